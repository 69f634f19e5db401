// quads.cu -- one quad per interior crossing edge, split into two or four
// triangles by the convex/concave analysis of Intersection-free Contouring
// (Sec. 4 "Polygonization", Sec. 5.4, A.1.5, Eqs. A1-A2).
//
// The four cells around an edge along axis a are ordered so that the
// triangle of the first three cell centres faces from the inside end of the
// edge to the outside end; each contributes the 3D point of its cycle
// through the edge.  Vertex c_k is concave when it lies below the oriented
// triangle (c_{k-1}, c_{k+1}, p_out) or above (c_{k-1}, c_{k+1}, p_in).
// Case 1 (diagonal c1 c3) needs c2 and c4 convex, case 2 (c2 c4) needs c1
// and c3 convex; otherwise case 3 fans four triangles around the 1D point.
// Pass 1 decides the case and counts; a scan gives offsets; pass 2 writes.
#include "kernels.h"
#include "odc_device.cuh"

namespace odc {

__device__ __forceinline__ float det3(float3 a, float3 b, float3 c, float3 o) {
    float ax = a.x - o.x, ay = a.y - o.y, az = a.z - o.z;
    float bx = b.x - o.x, by = b.y - o.y, bz = b.z - o.z;
    float cx = c.x - o.x, cy = c.y - o.y, cz = c.z - o.z;
    return ax * (by * cz - bz * cy) + ay * (bz * cx - bx * cz) + az * (bx * cy - by * cx);
}

__global__ void k_quad_case(GridDev g, const uint32_t* __restrict__ bits, const WordInfo* __restrict__ wi,
                            const uint32_t* __restrict__ cbase, const uint32_t* __restrict__ edges, uint32_t ne,
                            const unsigned long long* __restrict__ cycles, const uint32_t* __restrict__ vbase,
                            const float3* __restrict__ vlocal, int ic_split, uint8_t* __restrict__ qcase,
                            int4* __restrict__ qv, unsigned long long* __restrict__ cnt) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ne) return;
    uint32_t e = edges[i];
    int p[3];
    vid_xyz(g, e / 3u, &p[0], &p[1], &p[2]);
    int a = (int)(e % 3u), b = nxt3(a), c = prv3(a);
    if (p[b] < 1 || p[b] > g.n[b] - 1 || p[c] < 1 || p[c] > g.n[c] - 1) {
        qcase[i] = 0;
        cnt[i] = 0;
        return;
    }
    bool lower_in = label_at(g, bits, p[0], p[1], p[2]);
    const int dbs_in[4] = {0, 1, 1, 0}, dcs_in[4] = {0, 0, 1, 1};
    int vid[4];
    float3 P[4];
    for (int k = 0; k < 4; ++k) {
        int db = lower_in ? dbs_in[k] : dcs_in[k];
        int dc = lower_in ? dcs_in[k] : dbs_in[k];
        int q[3] = {p[0], p[1], p[2]};
        q[b] -= db;
        q[c] -= dc;
        uint32_t r = cell_rank(g, wi, cbase, q[0], q[1], q[2]);
        int le = 4 * a + db + 2 * dc;
        vid[k] = (int)(vbase[r] + nib(cycles[r], le));
        float3 v = vlocal[vid[k]];
        float o[3] = {v.x, v.y, v.z};
        o[b] -= (float)db;
        o[c] -= (float)dc;
        P[k] = make_float3(o[0], o[1], o[2]);
    }
    int cs = 1;
    if (ic_split) {
        float3 z = make_float3(0.f, 0.f, 0.f);
        float ea[3] = {0.f, 0.f, 0.f};
        ea[a] = 1.0f;
        float3 ua = make_float3(ea[0], ea[1], ea[2]);
        float3 pin = lower_in ? z : ua, pout = lower_in ? ua : z;
        bool conc[4];
        for (int k = 0; k < 4; ++k) {
            float3 pk = P[k], pp = P[(k + 3) & 3], pn = P[(k + 1) & 3];
            // (pk - o) . ((pp - o) x (pn - o)) = det3(pk, pp, pn, o)
            float d_out = det3(pk, pp, pn, pout);
            float d_in = det3(pk, pp, pn, pin);
            conc[k] = (d_out < 0.0f) || (d_in > 0.0f);
        }
        bool ok1 = !(conc[1] || conc[3]);
        bool ok2 = !(conc[0] || conc[2]);
        cs = ok1 ? 1 : (ok2 ? 2 : 3);
    }
    qcase[i] = (uint8_t)cs;
    qv[i] = make_int4(vid[0], vid[1], vid[2], vid[3]);
    cnt[i] = cs == 3 ? ((4ull << 32) | 1ull) : (2ull << 32);
}

__global__ void k_quad_emit(GridDev g, const uint32_t* __restrict__ edges, const uint32_t* __restrict__ T, uint32_t ne,
                            int k, const uint8_t* __restrict__ qcase, const int4* __restrict__ qv,
                            const unsigned long long* __restrict__ off, const uint32_t* __restrict__ v3tot,
                            float3* __restrict__ vworld, int3* __restrict__ tris) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ne) return;
    int cs = qcase[i];
    if (!cs) return;
    int4 v = qv[i];
    unsigned long long o = off[i];
    uint32_t t0 = (uint32_t)(o >> 32), x0 = (uint32_t)(o & 0xffffffffu);
    if (cs == 1) {
        tris[t0] = make_int3(v.x, v.y, v.z);
        tris[t0 + 1] = make_int3(v.x, v.z, v.w);
    } else if (cs == 2) {
        tris[t0] = make_int3(v.x, v.y, v.w);
        tris[t0 + 1] = make_int3(v.y, v.z, v.w);
    } else {
        int pe = (int)(*v3tot + x0);
        uint32_t e = edges[i];
        int p[3];
        vid_xyz(g, e / 3u, &p[0], &p[1], &p[2]);
        int a = (int)(e % 3u);
        float w[3] = {g.X[0][p[0]], g.X[1][p[1]], g.X[2][p[2]]};
        float tau = (float)T[i] * __int_as_float((127 - (k + 1)) << 23);
        w[a] = axis_world_ff(g.X[a], p[a], ff_make(tau)).hi;
        vworld[pe] = make_float3(w[0], w[1], w[2]);
        tris[t0] = make_int3(pe, v.x, v.y);
        tris[t0 + 1] = make_int3(pe, v.y, v.z);
        tris[t0 + 2] = make_int3(pe, v.z, v.w);
        tris[t0 + 3] = make_int3(pe, v.w, v.x);
    }
}

void launch_quad_case(const GridDev& g, const uint32_t* bits, const WordInfo* wi, const uint32_t* cbase,
                      const uint32_t* edges, uint32_t ne, const unsigned long long* cycles, const uint32_t* vbase,
                      const float3* vlocal, int ic_split, uint8_t* qcase, int4* qv, unsigned long long* cnt,
                      cudaStream_t st) {
    if (ne) { k_quad_case<<<(ne + 255) / 256, 256, 0, st>>>(g, bits, wi, cbase, edges, ne, cycles, vbase, vlocal,
                                                         ic_split, qcase, qv, cnt); note_launch(); }
}

void launch_quad_emit(const GridDev& g, const uint32_t* edges, const uint32_t* T, uint32_t ne, int k,
                      const uint8_t* qcase, const int4* qv, const unsigned long long* off,
                      const uint32_t* v3tot, float3* vworld, int3* tris, cudaStream_t st) {
    if (ne) { k_quad_emit<<<(ne + 255) / 256, 256, 0, st>>>(g, edges, T, ne, k, qcase, qv, off, v3tot, vworld, tris); note_launch(); }
}

}  // namespace odc
