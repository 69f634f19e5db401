// ablation.cu -- the Manifold Dual Contouring variants of the paper's
// ablation (Sec. 6.3, Tab. 3) for CSG sources, which have a continuous
// implicit psi and its gradient:
//
//   * linear 1D points (Sec. 4, Eq. 1): p_e where psi, interpolated linearly
//     between the edge's ends, vanishes, instead of the binary search;
//   * gradient normals (Sec. 4, Eq. 3): grad psi at the 1D point as the plane
//     normal of the QEF, instead of the 2D points.
//
// psi and its gradient are csg_psi.cuh's, taken in FP32 without FMA
// contraction (this unit is compiled with -fmad=false), so the interpolation
// parameter, quantised to the 1D lattice of 2^-(k+1) edge, is a defined
// integer.
#include "csg_psi.cuh"
#include "kernels.h"
#include "odc_device.cuh"

namespace odc {

namespace {

// Eq. 1 along each crossing edge from its lower end: t = psi0 / (psi0 -
// psi1) (1/2 when the difference vanishes), clamped to [0, 1], rounded to the
// nearest multiple of 2^-(k+1) strictly inside the edge.
__global__ void k_linear_1d(GridDev g, const uint32_t* __restrict__ edges, uint32_t ne, int k,
                            const PrimDev* __restrict__ prims, int n_prims, uint32_t* __restrict__ T) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ne) return;
    uint32_t e = edges[i];
    int p[3];
    vid_xyz(g, e / 3u, &p[0], &p[1], &p[2]);
    const int a = (int)(e % 3u);
    float w0[3] = {g.X[0][p[0]], g.X[1][p[1]], g.X[2][p[2]]};
    float w1[3] = {w0[0], w0[1], w0[2]};
    w1[a] = g.X[a][p[a] + 1];
    const float psi0 = csg_psi<float>(prims, n_prims, w0[0], w0[1], w0[2], nullptr);
    const float psi1 = csg_psi<float>(prims, n_prims, w1[0], w1[1], w1[2], nullptr);
    const float den = psi0 - psi1;
    float t = den != 0.0f ? psi0 / den : 0.5f;
    t = fminf(fmaxf(t, 0.0f), 1.0f);
    const float full = (float)(1u << (k + 1));
    int q = (int)rintf(t * full);
    q = min(max(q, 1), (int)(1u << (k + 1)) - 1);
    T[i] = (uint32_t)q;
}

// grad psi at every crossing edge's 1D point (world units).
__global__ void k_edge_grad(GridDev g, const uint32_t* __restrict__ edges, const uint32_t* __restrict__ T,
                            uint32_t ne, int k, const PrimDev* __restrict__ prims, int n_prims,
                            float3* __restrict__ grad) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ne) return;
    uint32_t e = edges[i];
    int p[3];
    vid_xyz(g, e / 3u, &p[0], &p[1], &p[2]);
    const int a = (int)(e % 3u);
    float w[3] = {g.X[0][p[0]], g.X[1][p[1]], g.X[2][p[2]]};
    const float tau = (float)T[i] * __int_as_float((127 - (k + 1)) << 23);
    w[a] = axis_world_ff(g.X[a], p[a], ff_make(tau)).hi;
    float gr[3];
    csg_psi<float>(prims, n_prims, w[0], w[1], w[2], gr);
    grad[i] = make_float3(gr[0], gr[1], gr[2]);
}

}  // namespace

void launch_linear_1d(const GridDev& g, const uint32_t* edges, uint32_t ne, int k, const PrimDev* prims, int n_prims,
                      uint32_t* T, cudaStream_t st) {
    if (ne) { k_linear_1d<<<(ne + 255) / 256, 256, 0, st>>>(g, edges, ne, k, prims, n_prims, T); note_launch(); }
}

void launch_edge_grad(const GridDev& g, const uint32_t* edges, const uint32_t* T, uint32_t ne, int k,
                      const PrimDev* prims, int n_prims, float3* grad, cudaStream_t st) {
    if (ne) { k_edge_grad<<<(ne + 255) / 256, 256, 0, st>>>(g, edges, T, ne, k, prims, n_prims, grad); note_launch(); }
}

}  // namespace odc
