// slab.cu -- z-slab extraction support: the owned part of a slab
// extraction and its placement in the whole grid's mesh.
//
// A slab owns the cells, the 3D points (cycles) of those cells, the
// crossing edges whose lower end lies in its cell layers [z0, z1), and the
// quads of those edges with their IC case-3 edge points (Sec. 4
// "Polygonization"; A.1.5).  The extraction runs on the slab's cell layers
// plus halo layers on both sides (the quads of the slab's lowest edge layer
// use the 3D points of the layer below; the manifold fix and the face
// searches of a boundary cell look at its neighbour).  Because every list of
// the path is in linear (z-major) element order, the owned cells, edges,
// 3D points, triangles and edge points are contiguous ranges of that
// extraction, and the whole grid's mesh numbers them the same way: 3D
// points in cell order, then edge points in edge order, triangles in edge
// order.  Placing each slab's ranges at offsets from a prefix sum of the
// slabs' counts therefore gives the whole grid's mesh byte for byte -- as
// long as the manifold fix (A.1.1), whose flips can chain from cell to cell
// round by round, marks no face within two layers of a slab plane: then no
// chain crosses a plane and each slab's fix is the whole grid's.  The
// extraction counts such marks so that the caller can refuse the merge.
#include "kernels.h"
#include "odc_device.cuh"

namespace odc {

namespace {

// first index i of the ascending list a[0, n) with a[i] >= key
__device__ uint32_t lower_bound_u32(const uint32_t* a, uint32_t n, uint32_t key) {
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        uint32_t mid = lo + (hi - lo) / 2;
        if (a[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// out[0..5]: 3D points before / up to the owned cells, edge points before /
// up to the owned edges, triangles before / up to the owned edges.
__global__ void k_slab_ranges(const uint32_t* __restrict__ cells, uint32_t C, const uint32_t* __restrict__ vbase,
                              uint32_t V3, const uint32_t* __restrict__ edges, uint32_t E,
                              const unsigned long long* __restrict__ qoff, uint32_t N3, uint32_t NT,
                              uint32_t cell_lo, uint32_t cell_hi, uint32_t edge_lo, uint32_t edge_hi,
                              unsigned long long* __restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const uint32_t c0 = lower_bound_u32(cells, C, cell_lo), c1 = lower_bound_u32(cells, C, cell_hi);
    const uint32_t e0 = lower_bound_u32(edges, E, edge_lo), e1 = lower_bound_u32(edges, E, edge_hi);
    out[0] = c0 < C ? vbase[c0] : V3;
    out[1] = c1 < C ? vbase[c1] : V3;
    const unsigned long long q0 = e0 < E ? qoff[e0] : (((unsigned long long)NT << 32) | N3);
    const unsigned long long q1 = e1 < E ? qoff[e1] : (((unsigned long long)NT << 32) | N3);
    out[2] = q0 & 0xffffffffull;
    out[3] = q1 & 0xffffffffull;
    out[4] = q0 >> 32;
    out[5] = q1 >> 32;
}

// dst[t] = src[t] with 3D-point ids shifted by vshift and edge-point ids
// (>= v3) moved to c3dst + (id - v3 - c3skip)
__global__ void k_slab_tris(const int3* __restrict__ src, int64_t n, int64_t v3, int64_t vshift, int64_t c3skip,
                            int64_t c3dst, int3* __restrict__ dst) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    int3 v = src[t];
    int w[3] = {v.x, v.y, v.z};
#pragma unroll
    for (int i = 0; i < 3; ++i) w[i] = (int)(w[i] < v3 ? w[i] + vshift : c3dst + (w[i] - v3 - c3skip));
    dst[t] = make_int3(w[0], w[1], w[2]);
}

// ids at or above mark are edge points numbered from 0: move them behind v3 3D points
__global__ void k_slab_fix(int3* __restrict__ t, int64_t n, int mark, int v3) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int3 v = t[i];
    if (v.x >= mark) v.x = v.x - mark + v3;
    if (v.y >= mark) v.y = v.y - mark + v3;
    if (v.z >= mark) v.z = v.z - mark + v3;
    t[i] = v;
}

// marked faces whose vertex layer lies in [b0, b1) or [b2, b3) (local z)
__global__ void k_slab_watch(GridDev g, const uint32_t* __restrict__ faces, const uint8_t* __restrict__ mark,
                             uint32_t nf, int b0, int b1, int b2, int b3, unsigned long long* __restrict__ count) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf || !mark[i]) return;
    int x, y, z;
    vid_xyz(g, faces[i] / 3u, &x, &y, &z);
    if ((z >= b0 && z < b1) || (z >= b2 && z < b3)) atomicAdd(count, 1ull);
}

// ambiguous faces (slot 1) with local id < limit, appended (any order) to
// out[base ..] as id + offset
__global__ void k_amb_select(const uint32_t* __restrict__ faces, const uint8_t* __restrict__ slots, uint32_t nf,
                             uint32_t limit, uint32_t offset, uint32_t* __restrict__ out, uint32_t* __restrict__ count) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf || slots[i] != 1 || faces[i] >= limit) return;
    out[atomicAdd(count, 1u)] = faces[i] + offset;
}

}  // namespace

void launch_amb_select(const uint32_t* faces, const uint8_t* slots, uint32_t nf, uint32_t limit, uint32_t offset,
                       uint32_t* out, size_t base, uint32_t* count, cudaStream_t st) {
    cudaMemsetAsync(count, 0, 4, st);
    if (nf) {
        k_amb_select<<<(nf + 255) / 256, 256, 0, st>>>(faces, slots, nf, limit, offset, out + base, count);
        note_launch();
    }
}

void launch_slab_watch(const GridDev& g, const uint32_t* faces, const uint8_t* mark, uint32_t nf, const int* bands,
                       unsigned long long* count, cudaStream_t st) {
    if (nf) {
        k_slab_watch<<<(nf + 255) / 256, 256, 0, st>>>(g, faces, mark, nf, bands[0], bands[1], bands[2], bands[3],
                                                       count);
        note_launch();
    }
}

void launch_slab_ranges(const uint32_t* cells, uint32_t C, const uint32_t* vbase, uint32_t V3, const uint32_t* edges,
                        uint32_t E, const unsigned long long* qoff, uint32_t N3, uint32_t NT, uint32_t cell_lo,
                        uint32_t cell_hi, uint32_t edge_lo, uint32_t edge_hi, unsigned long long* out,
                        cudaStream_t st) {
    k_slab_ranges<<<1, 32, 0, st>>>(cells, C, vbase, V3, edges, E, qoff, N3, NT, cell_lo, cell_hi, edge_lo, edge_hi,
                                    out);
    note_launch();
}

void launch_slab_tris(const int3* src, int64_t n, int64_t v3, int64_t vshift, int64_t c3skip, int64_t c3dst,
                      int3* dst, cudaStream_t st) {
    if (n > 0) {
        k_slab_tris<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(src, n, v3, vshift, c3skip, c3dst, dst);
        note_launch();
    }
}

void launch_slab_fix(int3* t, int64_t n, int mark, int v3, cudaStream_t st) {
    if (n > 0) {
        k_slab_fix<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(t, n, mark, v3);
        note_launch();
    }
}

}  // namespace odc
