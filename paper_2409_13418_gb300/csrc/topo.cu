// topo.cu -- manifold fix and per-cell cycles (A.1.1, Fig. A1).
//
// Each crossing cell's crossing edges form cycles by chaining the segments of
// its faces; one 3D point is placed per cycle.  Where two cells sharing an
// ambiguous face each close a single cycle through both of its segments, the
// dual edge between them would carry four quads; the face's pairing is then
// flipped for both cells, which splits both cycles.  Rounds of "mark all, then
// flip all" repeat until no face qualifies.
#include "kernels.h"
#include "odc_device.cuh"

namespace odc {

__global__ void k_manifold_mark(GridDev g, const uint32_t* __restrict__ bits, const uint32_t* __restrict__ flips,
                                const uint32_t* __restrict__ faces, const uint8_t* __restrict__ slots, uint32_t nf,
                                uint8_t* __restrict__ mark, uint32_t* __restrict__ counter) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    uint8_t m = 0;
    if (slots[i] == 1) {
        int x, y, z;
        uint32_t fid = faces[i];
        vid_xyz(g, fid / 3u, &x, &y, &z);
        int a = (int)(fid % 3u);
        int q[3] = {x, y, z};
        if (q[a] > 0 && q[a] < g.n[a]) {
            int b[3] = {x, y, z};
            b[a] -= 1;
            uint32_t cb = cell_config(g, bits, b[0], b[1], b[2]);
            uint32_t ca = cell_config(g, bits, x, y, z);
            bool sb = face_same_cycle(cb, cell_flipmask(g, flips, b[0], b[1], b[2]), 2 * a + 1);
            bool sa = face_same_cycle(ca, cell_flipmask(g, flips, x, y, z), 2 * a);
            m = (sb && sa) ? 1 : 0;
        }
    }
    mark[i] = m;
    if (m) atomicAdd(counter, 1u);
}

__global__ void k_manifold_apply(GridDev g, uint32_t* __restrict__ flips, const uint32_t* __restrict__ faces,
                                 const uint8_t* __restrict__ mark, uint32_t nf) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf || !mark[i]) return;
    int x, y, z;
    uint32_t fid = faces[i];
    vid_xyz(g, fid / 3u, &x, &y, &z);
    int a = (int)(fid % 3u);
    atomicXor(&flips[(((size_t)a * g.nv[2] + z) * g.nv[1] + y) * g.W + (x >> 5)], 1u << (x & 31));
}

__global__ void k_cells(GridDev g, const uint32_t* __restrict__ flips, const uint32_t* __restrict__ cells,
                        const uint8_t* __restrict__ configs, uint32_t nc, unsigned long long* __restrict__ cyc,
                        uint32_t* __restrict__ ncyc) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    int x, y, z;
    cid_xyz(g, cells[i], &x, &y, &z);
    int n;
    uint64_t c = cell_cycles(configs[i], cell_flipmask(g, flips, x, y, z), &n);
    cyc[i] = c;
    ncyc[i] = (uint32_t)n;
}

void launch_manifold_mark(const GridDev& g, const uint32_t* bits, const uint32_t* flips, const uint32_t* faces,
                          const uint8_t* slots, uint32_t nf, uint8_t* mark, uint32_t* counter, cudaStream_t st) {
    if (nf) { k_manifold_mark<<<(nf + 255) / 256, 256, 0, st>>>(g, bits, flips, faces, slots, nf, mark, counter); note_launch(); }
}

void launch_manifold_apply(const GridDev& g, uint32_t* flips, const uint32_t* faces, const uint8_t* mark, uint32_t nf,
                           cudaStream_t st) {
    if (nf) { k_manifold_apply<<<(nf + 255) / 256, 256, 0, st>>>(g, flips, faces, mark, nf); note_launch(); }
}

void launch_cells(const GridDev& g, const uint32_t* flips, const uint32_t* cells, const uint8_t* configs, uint32_t nc,
                  unsigned long long* cyc, uint32_t* ncyc, cudaStream_t st) {
    if (nc) { k_cells<<<(nc + 255) / 256, 256, 0, st>>>(g, flips, cells, configs, nc, cyc, ncyc); note_launch(); }
}

}  // namespace odc
