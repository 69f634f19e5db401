// mc.cu -- marching-cubes polygonization through the 1D points (the "MC" and
// "MC + 1D search" rows of Tab. A8): the mesh vertices are the 1D points of
// the crossing edges (edge order) and each cycle of each crossing cell
// (A.1.1 cycles, with the manifold fix) becomes a polygon walked in the
// oriented order of mc_next, fanned from its smallest local edge; cells in
// cell order, cycles in cycle order.  No 2D search, QEF or quads.
#include "kernels.h"
#include "odc_device.cuh"

namespace odc {

namespace {

__global__ void k_mc_verts(GridDev g, const uint32_t* __restrict__ edges, const uint32_t* __restrict__ T, uint32_t ne,
                           int k, float3* __restrict__ vworld) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ne) return;
    uint32_t e = edges[i];
    int p[3];
    vid_xyz(g, e / 3u, &p[0], &p[1], &p[2]);
    const int a = (int)(e % 3u);
    float w[3] = {g.X[0][p[0]], g.X[1][p[1]], g.X[2][p[2]]};
    const float tau = (float)T[i] * __int_as_float((127 - (k + 1)) << 23);
    w[a] = axis_world_ff(g.X[a], p[a], ff_make(tau)).hi;
    vworld[i] = make_float3(w[0], w[1], w[2]);
}

// Triangles per crossing cell: sum over its cycles of (length - 2).
__global__ void k_mc_count(const uint32_t* __restrict__ cells, const unsigned long long* __restrict__ cycles,
                           uint32_t nc, uint32_t* __restrict__ cnt) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    uint64_t cyc = cycles[i];
    uint32_t n = 0, ncyc = 0;
    for (int le = 0; le < 12; ++le)
        if (nib(cyc, le) != 0xF) {
            ++n;
            ncyc = max(ncyc, nib(cyc, le) + 1);
        }
    cnt[i] = n - 2 * ncyc;
    (void)cells;
}

__global__ void k_mc_emit(GridDev g, const uint32_t* __restrict__ flips, const WordInfo* __restrict__ wi,
                          const uint32_t* __restrict__ ebase, const uint32_t* __restrict__ cells,
                          const uint8_t* __restrict__ configs, const unsigned long long* __restrict__ cycles,
                          uint32_t nc, const uint32_t* __restrict__ off, const uint32_t* __restrict__ cnt,
                          int3* __restrict__ tris) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    int cp[3];
    cid_xyz(g, cells[i], &cp[0], &cp[1], &cp[2]);
    const uint32_t cfg = configs[i];
    const uint32_t fm = cell_flipmask(g, flips, cp[0], cp[1], cp[2]);
    const uint64_t cyc = cycles[i];
    int gid[12];
    int ncyc = 0;
    for (int le = 0; le < 12; ++le) {
        gid[le] = -1;
        if (nib(cyc, le) == 0xF) continue;
        ncyc = max(ncyc, (int)nib(cyc, le) + 1);
        const int a = le >> 2, d0 = edge_corner0(le);
        gid[le] = (int)edge_rank(g, wi, ebase, cp[0] + (d0 & 1), cp[1] + ((d0 >> 1) & 1), cp[2] + ((d0 >> 2) & 1), a);
    }
    uint32_t t = off[i];
    const uint32_t end = t + cnt[i];   // the counted triangles of this cell, never more
    for (int cy = 0; cy < ncyc; ++cy) {
        int le0 = -1;
        for (int le = 0; le < 12 && le0 < 0; ++le)
            if (nib(cyc, le) == (uint32_t)cy) le0 = le;
        int prev = mc_next(cfg, fm, le0);
        for (int guard = 0; guard < 12 && prev >= 0 && prev != le0; ++guard) {
            const int nx = mc_next(cfg, fm, prev);
            if (nx < 0 || nx == le0 || t >= end) break;
            tris[t++] = make_int3(gid[le0], gid[prev], gid[nx]);
            prev = nx;
        }
    }
}

}  // namespace

void launch_mc(const GridDev& g, const uint32_t* flips, const WordInfo* wi, const uint32_t* ebase,
               const uint32_t* edges, const uint32_t* T, uint32_t ne, int k, const uint32_t* cells,
               const uint8_t* configs, const unsigned long long* cycles, uint32_t nc, uint32_t* cnt, uint32_t* off,
               uint32_t* tmp, uint32_t* total, float3* vworld, int3* tris, cudaStream_t st) {
    if (ne) { k_mc_verts<<<(ne + 255) / 256, 256, 0, st>>>(g, edges, T, ne, k, vworld); note_launch(); }
    if (nc) { k_mc_count<<<(nc + 255) / 256, 256, 0, st>>>(cells, cycles, nc, cnt); note_launch(); }
    exclusive_scan<uint32_t>(cnt, off, nc, tmp, total, st);
    if (nc) { k_mc_emit<<<(nc + 127) / 128, 128, 0, st>>>(g, flips, wi, ebase, cells, configs, cycles, nc, off, cnt,
                                                         tris); note_launch(); }
}

}  // namespace odc
