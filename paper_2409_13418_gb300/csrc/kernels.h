// kernels.h -- host launchers of the ODC kernels (one translation unit each).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "odc_internal.h"
#include "../../include/odc.h"

#include <string>

namespace odc {

// compact.cu
size_t scan_tmp_elems(size_t n);
template <typename T>
void exclusive_scan(const T* in, T* out, size_t n, T* tmp, T* total, cudaStream_t st);
void launch_csg_grid(const GridDev& g, const PrimDev* prims, const float4* cull, int n_prims, uint32_t* bits,
                     cudaStream_t st);
void launch_classify(const GridDev& g, const uint32_t* bits, WordInfo* wi, uint32_t* ce, uint32_t* cf, uint32_t* cc,
                     cudaStream_t st);
void launch_emit(const GridDev& g, const uint32_t* bits, const WordInfo* wi, const uint32_t* ebase,
                 const uint32_t* fbase, const uint32_t* cbase, uint32_t* edges, uint32_t* faces, uint8_t* slots,
                 uint32_t* cells, uint8_t* configs, cudaStream_t st);

// topo.cu
void launch_manifold_mark(const GridDev& g, const uint32_t* bits, const uint32_t* flips, const uint32_t* faces,
                          const uint8_t* slots, uint32_t nf, uint8_t* mark, uint32_t* counter, cudaStream_t st);
void launch_manifold_apply(const GridDev& g, uint32_t* flips, const uint32_t* faces, const uint8_t* mark, uint32_t nf,
                           cudaStream_t st);
void launch_cells(const GridDev& g, const uint32_t* flips, const uint32_t* cells, const uint8_t* configs, uint32_t nc,
                  unsigned long long* cyc, uint32_t* ncyc, cudaStream_t st);

// search_csg.cu
void launch_bisect_csg(const GridDev& g, const uint32_t* bits, const uint32_t* edges, uint32_t ne, int k,
                       const PrimDev* prims, const float4* cull, int n_prims, uint32_t* T, cudaStream_t st);
void launch_face_csg(const GridDev& g, const uint32_t* bits, const uint32_t* flips, const WordInfo* wi,
                     const uint32_t* ebase, const uint32_t* T, const uint32_t* faces, const uint8_t* slots,
                     uint32_t nf, const SearchParams& sp, const PrimDev* prims, const float4* cull, int n_prims,
                     float4* pf, uint8_t* flags, FaceDecisions* dec, cudaStream_t st);
void launch_csg_points(const PrimDev* prims, const float4* cull, int n_prims, const float3* pts, int64_t n,
                       uint8_t* labels, cudaStream_t st);

// search_csg.cu, voxel volumes
// axis_c / axis_f: scratch of nv[0] + nv[1] + nv[2] ints / floats
void launch_vox_grid(const GridDev& g, const VoxDev& vox, int* axis_c, float* axis_f, uint32_t* bits,
                     cudaStream_t st);
void launch_vox_points(const VoxDev& vox, const float3* pts, int64_t n, uint8_t* labels, cudaStream_t st);
void launch_bisect_vox(const GridDev& g, const uint32_t* bits, const uint32_t* edges, uint32_t ne, int k,
                       const VoxDev& vox, uint32_t* T, cudaStream_t st);
void launch_face_vox(const GridDev& g, const uint32_t* bits, const uint32_t* flips, const WordInfo* wi,
                     const uint32_t* ebase, const uint32_t* T, const uint32_t* faces, const uint8_t* slots,
                     uint32_t nf, const SearchParams& sp, const VoxDev& vox, float4* pf, uint8_t* flags,
                     FaceDecisions* dec, cudaStream_t st);

// qef.cu (gnorm: per crossing edge, grad psi at its 1D point replacing the
// 2D-point normals; null for ODC)
void launch_qef(const GridDev& g, const uint32_t* flips, const WordInfo* wi, const uint32_t* ebase,
                const uint32_t* fbase, const uint32_t* T, const float4* pf, const float3* gnorm, const uint32_t* cells,
                const uint8_t* configs, const unsigned long long* cycles, const uint32_t* vbase, uint32_t nc, int k,
                float3* vlocal, float3* vworld, cudaStream_t st);

// mc.cu (marching-cubes polygons through the 1D points)
void launch_mc(const GridDev& g, const uint32_t* flips, const WordInfo* wi, const uint32_t* ebase,
               const uint32_t* edges, const uint32_t* T, uint32_t ne, int k, const uint32_t* cells,
               const uint8_t* configs, const unsigned long long* cycles, uint32_t nc, uint32_t* cnt, uint32_t* off,
               uint32_t* tmp, uint32_t* total, float3* vworld, int3* tris, cudaStream_t st);

// ablation.cu (MDC variants of the ablation, CSG sources)
void launch_linear_1d(const GridDev& g, const uint32_t* edges, uint32_t ne, int k, const PrimDev* prims, int n_prims,
                      uint32_t* T, cudaStream_t st);
void launch_edge_grad(const GridDev& g, const uint32_t* edges, const uint32_t* T, uint32_t ne, int k,
                      const PrimDev* prims, int n_prims, float3* grad, cudaStream_t st);

// quads.cu
void launch_quad_case(const GridDev& g, const uint32_t* bits, const WordInfo* wi, const uint32_t* cbase,
                      const uint32_t* edges, uint32_t ne, const unsigned long long* cycles, const uint32_t* vbase,
                      const float3* vlocal, int ic_split, uint8_t* qcase, int4* qv, unsigned long long* cnt,
                      cudaStream_t st);
void launch_quad_emit(const GridDev& g, const uint32_t* edges, const uint32_t* T, uint32_t ne, int k,
                      const uint8_t* qcase, const int4* qv, const unsigned long long* off, const uint32_t* v3tot,
                      float3* vworld, int3* tris, cudaStream_t st);

// z-slab extraction (slab.cu)
void launch_slab_ranges(const uint32_t* cells, uint32_t C, const uint32_t* vbase, uint32_t V3, const uint32_t* edges,
                        uint32_t E, const unsigned long long* qoff, uint32_t N3, uint32_t NT, uint32_t cell_lo,
                        uint32_t cell_hi, uint32_t edge_lo, uint32_t edge_hi, unsigned long long* out,
                        cudaStream_t st);
void launch_slab_tris(const int3* src, int64_t n, int64_t v3, int64_t vshift, int64_t c3skip, int64_t c3dst,
                      int3* dst, cudaStream_t st);
void launch_slab_fix(int3* t, int64_t n, int mark, int v3, cudaStream_t st);
void launch_amb_select(const uint32_t* faces, const uint8_t* slots, uint32_t nf, uint32_t limit, uint32_t offset,
                       uint32_t* out, size_t base, uint32_t* count, cudaStream_t st);
void launch_slab_watch(const GridDev& g, const uint32_t* faces, const uint8_t* mark, uint32_t nf, const int* bands,
                       unsigned long long* count, cudaStream_t st);

// quality.cu (Sec. 6.1 metrics; mlp may be null for a CSG source)
struct MlpState;
odc_status mesh_quality(MlpState* mlp, const PrimDev* prims, int n_prims, const VoxDev* vox, const float3* v,
                        int64_t nv, const int3* t,
                        int64_t nt, float iso, int64_t n_samples, uint64_t seed, int what, cudaStream_t s,
                        odc_quality* out, std::string* err);

}  // namespace odc
