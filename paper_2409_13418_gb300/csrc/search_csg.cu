// search_csg.cu -- grid labels and 1D and 2D point searches against the
// directly evaluated occupancies (CSG trees and voxel volumes), one thread per
// crossing edge / face segment running its whole search in registers (these
// queries cost tens to hundreds of flops, so no batching is needed).
//
// 1D (Sec. 5.1): k bisections of the edge keeping ends of opposite labels;
// the result is the midpoint of the final interval, stored as the odd integer
// T of T / 2^(k+1).
// 2D (Sec. 5.2, A.1.3, A.1.4): step 1 line-binary search from m along the
// perpendicular towards the opposite label; if it never leaves m, p_f = m;
// step 2 two line-binary searches from q parallel to l; step 3 intersects
// (p_e1, q1) and (p_e2, q2).
#include "kernels.h"
#include "search.cuh"
#include "voxel.cuh"

namespace odc {

struct CsgOcc {
    const PrimDev* prims;
    const float4* cull;
    int n;
    __device__ __forceinline__ uint32_t operator()(float3 p) const { return csg_label(prims, cull, n, p.x, p.y, p.z); }
};

template <class Occ>
__global__ void k_bisect(GridDev g, const uint32_t* __restrict__ bits, const uint32_t* __restrict__ edges,
                         uint32_t ne, int k, Occ occ, uint32_t* __restrict__ T) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ne) return;
    uint32_t e = edges[i];
    int p[3];
    vid_xyz(g, e / 3u, &p[0], &p[1], &p[2]);
    int a = (int)(e % 3u);
    uint32_t lab0 = label_at(g, bits, p[0], p[1], p[2]);
    float w[3] = {g.X[0][p[0]], g.X[1][p[1]], g.X[2][p[2]]};
    uint32_t lo = 0;   // numerator of the low end over 2^s
    for (int s = 0; s < k; ++s) {
        uint32_t mid = 2u * lo + 1u;   // over 2^(s+1)
        float u = (float)mid * __int_as_float((127 - (s + 1)) << 23);
        w[a] = axis_world_ff(g.X[a], p[a], ff_make(u)).hi;
        uint32_t lab = occ(make_float3(w[0], w[1], w[2]));
        lo = (lab == lab0) ? mid : 2u * lo;
    }
    T[i] = 2u * lo + 1u;
}

// Line-binary search (A.1.3) from p along unit d: returns J of the near end.
template <class Occ>
__device__ __forceinline__ uint32_t lbs(const GridDev& g, const FaceSeg& F, const Occ& occ, ff2 p, ff2 d, float R,
                                        int n, int b, uint32_t lab0, bool* found) {
    int first = n;
    *found = false;
    for (int i = 1; i <= n; ++i) {
        ff s = lbs_param(R, (uint32_t)i << b, n, b);
        if (occ(face_world2(g, F, ray_point(p, d, s))) != lab0) {
            first = i;
            *found = true;
            break;
        }
    }
    uint32_t Ja = (uint32_t)(first - 1) << b, Jc = (uint32_t)first << b;
    for (int t = 0; t < b; ++t) {
        uint32_t Jm = (Ja + Jc) >> 1;
        ff s = lbs_param(R, Jm, n, b);
        if (occ(face_world2(g, F, ray_point(p, d, s))) == lab0) Ja = Jm;
        else Jc = Jm;
    }
    return Ja;
}

template <class Occ>
__global__ void k_face(GridDev g, const uint32_t* __restrict__ bits, const uint32_t* __restrict__ flips,
                       const WordInfo* __restrict__ wi, const uint32_t* __restrict__ ebase,
                       const uint32_t* __restrict__ T, const uint32_t* __restrict__ faces,
                       const uint8_t* __restrict__ slots, uint32_t nf, SearchParams sp, Occ occ,
                       float4* __restrict__ pf, uint8_t* __restrict__ flags, FaceDecisions* __restrict__ dec) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    FaceSeg F;
    load_face(g, bits, flips, wi, ebase, T, sp.steps_1d, faces[i], slots[i], F);
    uint32_t lab_m = occ(face_world2(g, F, F.m));
    ff2 d = lab_m ? ff2{ff_neg(F.d.u), ff_neg(F.d.v)} : F.d;
    int fl = 0;
    bool f0 = false, f1 = false, f2 = false;
    uint32_t Jq = lbs(g, F, occ, F.m, d, sp.range1, sp.lin1, sp.bin1, lab_m, &f0);
    uint32_t J1 = 0, J2 = 0;
    float4 out;
    if (Jq == 0) {
        fl |= 1;
        out = ff2_pack(F.m);
    } else {
        ff2 q = ray_point(F.m, d, lbs_param(sp.range1, Jq, sp.lin1, sp.bin1));
        ff2 nu1 = {ff_neg(F.u1.u), ff_neg(F.u1.v)};
        J1 = lbs(g, F, occ, q, F.u1, sp.range2, sp.lin2, sp.bin2, lab_m, &f1);
        J2 = lbs(g, F, occ, q, nu1, sp.range2, sp.lin2, sp.bin2, lab_m, &f2);
        ff2 q1 = ray_point(q, F.u1, lbs_param(sp.range2, J1, sp.lin2, sp.bin2));
        ff2 q2 = ray_point(q, nu1, lbs_param(sp.range2, J2, sp.lin2, sp.bin2));
        out = face_intersect(F, q1, q2, &fl);
    }
    pf[i] = out;
    flags[i] = (uint8_t)fl;
    FaceDecisions D;
    D.Jq = Jq;
    D.J1 = J1;
    D.J2 = J2;
    D.lab_m = (uint8_t)lab_m;
    D.found = (uint8_t)(f0 | (f1 << 1) | (f2 << 2));
    D.pad0 = D.pad1 = 0;
    dec[i] = D;
}

template <class Occ>
__global__ void k_points(Occ occ, const float3* __restrict__ pts, int64_t n, uint8_t* __restrict__ labels) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    labels[i] = (uint8_t)occ(pts[i]);
}

// Per-axis sample coordinates of the grid's vertex coordinates (cell index
// and fraction, the fast path's float32 rounding): the label kernel then
// needs no division per vertex.
__global__ void k_vox_axes(GridDev g, VoxDev d, int* __restrict__ ci, float* __restrict__ fi) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int n0 = g.nv[0], n1 = g.nv[1], n2 = g.nv[2];
    if (t >= n0 + n1 + n2) return;
    const int a = t < n0 ? 0 : (t < n0 + n1 ? 1 : 2);
    const int i = t - (a == 0 ? 0 : (a == 1 ? n0 : n0 + n1));
    vox_axis32(d, a, g.X[a][i], &ci[t], &fi[t]);
}

// Grid labels of a voxel volume: one warp per (label word, row y), marching
// over kVoxZRun consecutive vertex layers z.  The float32 decision comes
// from the axis tables, with the samples of the upper volume layer kept in
// registers when the next vertex layer falls in the next volume cell (or
// the same one), so that a layer's samples are read once instead of twice;
// the full evaluation (float-float when near iso) decides what it leaves
// undecided.
constexpr int kVoxZRun = 8;
__global__ void k_vox_grid(GridDev g, VoxOcc occ, const int* __restrict__ ci, const float* __restrict__ fi,
                           uint32_t* __restrict__ bits) {
    const size_t wr = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;   // (word, row y, z run)
    const int l = threadIdx.x & 31;
    const int nzr = (g.nv[2] + kVoxZRun - 1) / kVoxZRun;
    if (wr >= (size_t)g.W * g.nv[1] * nzr) return;
    const int xw = (int)(wr % g.W);
    const size_t t = wr / g.W;
    const int y = (int)(t % g.nv[1]);
    const int z0 = (int)(t / g.nv[1]) * kVoxZRun, z1 = min(z0 + kVoxZRun, g.nv[2]);
    const int x = xw * 32 + l;
    const bool live = x < g.nv[0];
    const VoxDev& d = occ.d;
    const int cx = live ? __ldg(ci + x) : 0, cy = __ldg(ci + g.nv[0] + y);
    const float fx = live ? __ldg(fi + x) : 0.0f, fy = __ldg(fi + g.nv[0] + y);
    const int* cz = ci + g.nv[0] + g.nv[1];
    const float* fz = fi + g.nv[0] + g.nv[1];
    const int dmax = max(max(2, d.dims[0]), max(d.dims[1], d.dims[2]));
    const size_t sy = (size_t)d.dims[0], sz = (size_t)d.dims[0] * d.dims[1];
    const float* col = d.v + (size_t)cy * sy + (size_t)cx;   // (cx, cy) column of the volume
    int held = -2;                                            // volume layer whose 4 samples are in lo[]
    float lo[4] = {0.f, 0.f, 0.f, 0.f}, hi[4] = {0.f, 0.f, 0.f, 0.f};
    for (int z = z0; z < z1; ++z) {
        const int c = __ldg(cz + z);
        const float f = __ldg(fz + z);
        bool in = false;
        if (live) {
            if (c == held + 1) {          // the previous upper layer is this lower one
                for (int k = 0; k < 4; ++k) lo[k] = hi[k];
            } else if (c != held) {
                const float* b = col + (size_t)c * sz;
                lo[0] = __ldg(b); lo[1] = __ldg(b + 1); lo[2] = __ldg(b + sy); lo[3] = __ldg(b + sy + 1);
            }
            if (c != held) {
                const float* b = col + (size_t)(c + 1) * sz;
                hi[0] = __ldg(b); hi[1] = __ldg(b + 1); hi[2] = __ldg(b + sy); hi[3] = __ldg(b + sy + 1);
                held = c;
            }
            // the same float32 trilinear value and bound as the direct evaluation
            const float c00 = fmaf(lo[1] - lo[0], fx, lo[0]), c10 = fmaf(lo[3] - lo[2], fx, lo[2]);
            const float c01 = fmaf(hi[1] - hi[0], fx, hi[0]), c11 = fmaf(hi[3] - hi[2], fx, hi[2]);
            const float c0 = fmaf(c10 - c00, fy, c00), c1 = fmaf(c11 - c01, fy, c01);
            const float phi = fmaf(c1 - c0, f, c0);
            const float vmax = fmaxf(fmaxf(fmaxf(fabsf(lo[0]), fabsf(lo[1])), fmaxf(fabsf(lo[2]), fabsf(lo[3]))),
                                     fmaxf(fmaxf(fabsf(hi[0]), fabsf(hi[1])), fmaxf(fabsf(hi[2]), fabsf(hi[3]))));
            const float bound = vmax * (3e-6f * (float)(dmax - 1) + 4e-6f);
            if (phi - d.iso > bound) in = true;
            else if (d.iso - phi > bound) in = false;
            else in = occ(make_float3(g.X[0][x], g.X[1][y], g.X[2][z])) != 0;
        }
        const uint32_t word = __ballot_sync(0xffffffffu, in);
        if (l == 0) bits[((size_t)z * g.nv[1] + y) * g.W + xw] = word;
    }
}

void launch_csg_points(const PrimDev* prims, const float4* cull, int n_prims, const float3* pts, int64_t n,
                       uint8_t* labels, cudaStream_t st) {
    if (n <= 0) return;
    CsgOcc occ{prims, cull, n_prims};
    k_points<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(occ, pts, n, labels); note_launch();
}

void launch_bisect_csg(const GridDev& g, const uint32_t* bits, const uint32_t* edges, uint32_t ne, int k,
                       const PrimDev* prims, const float4* cull, int n_prims, uint32_t* T, cudaStream_t st) {
    if (!ne) return;
    CsgOcc occ{prims, cull, n_prims};
    k_bisect<<<(ne + 127) / 128, 128, 0, st>>>(g, bits, edges, ne, k, occ, T); note_launch();
}

void launch_face_csg(const GridDev& g, const uint32_t* bits, const uint32_t* flips, const WordInfo* wi,
                     const uint32_t* ebase, const uint32_t* T, const uint32_t* faces, const uint8_t* slots,
                     uint32_t nf, const SearchParams& sp, const PrimDev* prims, const float4* cull, int n_prims,
                     float4* pf, uint8_t* flags, FaceDecisions* dec, cudaStream_t st) {
    if (!nf) return;
    CsgOcc occ{prims, cull, n_prims};
    k_face<<<(nf + 127) / 128, 128, 0, st>>>(g, bits, flips, wi, ebase, T, faces, slots, nf, sp, occ, pf,
                                              flags, dec); note_launch();
}

void launch_vox_grid(const GridDev& g, const VoxDev& vox, int* axis_c, float* axis_f, uint32_t* bits,
                     cudaStream_t st) {
    const int na = g.nv[0] + g.nv[1] + g.nv[2];
    k_vox_axes<<<(na + 255) / 256, 256, 0, st>>>(g, vox, axis_c, axis_f); note_launch();
    const size_t runs = (size_t)(g.nv[2] + kVoxZRun - 1) / kVoxZRun;
    const size_t threads = (size_t)g.W * g.nv[1] * runs * 32;
    k_vox_grid<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(g, VoxOcc{vox}, axis_c, axis_f, bits); note_launch();
}

void launch_vox_points(const VoxDev& vox, const float3* pts, int64_t n, uint8_t* labels, cudaStream_t st) {
    if (n <= 0) return;
    k_points<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(VoxOcc{vox}, pts, n, labels); note_launch();
}

void launch_bisect_vox(const GridDev& g, const uint32_t* bits, const uint32_t* edges, uint32_t ne, int k,
                       const VoxDev& vox, uint32_t* T, cudaStream_t st) {
    if (!ne) return;
    k_bisect<<<(ne + 127) / 128, 128, 0, st>>>(g, bits, edges, ne, k, VoxOcc{vox}, T); note_launch();
}

void launch_face_vox(const GridDev& g, const uint32_t* bits, const uint32_t* flips, const WordInfo* wi,
                     const uint32_t* ebase, const uint32_t* T, const uint32_t* faces, const uint8_t* slots,
                     uint32_t nf, const SearchParams& sp, const VoxDev& vox, float4* pf, uint8_t* flags,
                     FaceDecisions* dec, cudaStream_t st) {
    if (!nf) return;
    k_face<<<(nf + 127) / 128, 128, 0, st>>>(g, bits, flips, wi, ebase, T, faces, slots, nf, sp, VoxOcc{vox}, pf,
                                              flags, dec); note_launch();
}

}  // namespace odc
