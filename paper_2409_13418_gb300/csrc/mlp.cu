// mlp.cu -- envelope-MLP occupancy network on the device.
//
// f(x) = W5 relu(W4 relu(W3 relu(W2 relu(W1 g(x) + b1) + b2) + b3) + b4) + b5,
// g(x) = [sin(2 pi B x), cos(2 pi B x)] (64 frequencies), z = scale (radius -
// |x| + amp f(x)).  The FP32 path (this file) is the plain reference path of
// the GPU: SIMT FMAs, register-tiled 64-query x 256-output tiles, the
// Fourier phase B.x formed exactly in float-float and reduced to one period
// before sincospi.  The BF16 tensor-core path lives in mlp_tc.cu.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "mlp.h"
#include "mlp_dev.cuh"
#include "odc_device.cuh"

namespace odc {

odc_status mlp_check(const odc_mlp* m, std::string* err) {
    if (!m) { *err = "MLP source without descriptor"; return ODC_ERR_INVALID_ARG; }
    if (m->n_freq != kNF || m->hidden != kH || m->n_hidden != kNL)
        { *err = "MLP shape must be 64 frequencies, 4 hidden layers of 256"; return ODC_ERR_INVALID_ARG; }
    if (m->latent_dim != 0 && m->latent_dim != 128) { *err = "latent_dim must be 0 or 128"; return ODC_ERR_INVALID_ARG; }
    if (m->latent_dim && !m->latent) { *err = "latent pointer missing"; return ODC_ERR_INVALID_ARG; }
    if (!m->B) { *err = "Fourier matrix missing"; return ODC_ERR_INVALID_ARG; }
    for (int l = 0; l <= kNL; ++l)
        if (!m->W[l] || !m->b[l]) { *err = "weight or bias pointer missing"; return ODC_ERR_INVALID_ARG; }
    if (m->precision != ODC_PREC_FP32 && m->precision != ODC_PREC_BF16)
        { *err = "precision must be FP32 or BF16"; return ODC_ERR_INVALID_ARG; }
    if (m->precision == ODC_PREC_BF16 && !(m->band >= 0.0f && m->band < 0.5f))
        { *err = "band must be in [0, 0.5)"; return ODC_ERR_INVALID_ARG; }
    if (!(m->split_zmargin >= 0.0f)) { *err = "split_zmargin must be >= 0"; return ODC_ERR_INVALID_ARG; }
    return ODC_OK;
}

float mlp_logit_threshold(float iso) { return (float)std::log((double)iso / (1.0 - (double)iso)); }

int mlp_precision(const MlpState* st) { return st->precision; }
int64_t mlp_split_count(const MlpState* st) { return st ? st->n_split : 0; }

#define MLP_CK(call)                                                                        \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) { *err = std::string(#call) + ": " + cudaGetErrorString(e_); \
                                 return ODC_ERR_CUDA; }                                     \
    } while (0)

odc_status mlp_scratch(MlpState* st, int slot, size_t bytes, void** out, std::string* err) {
    if (st->scr_cap[slot] < bytes) {
        if (st->scr[slot]) {
            MLP_CK(cudaDeviceSynchronize());
            cudaFree(st->scr[slot]);
            st->scr[slot] = nullptr;
            st->scr_cap[slot] = 0;
        }
        size_t want = bytes + bytes / 4 + 4096;
        cudaError_t e = cudaMalloc(&st->scr[slot], want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            *err = std::string("MLP scratch allocation failed: ") + cudaGetErrorString(e);
            return ODC_ERR_OOM;
        }
        st->scr_cap[slot] = want;
    }
    *out = st->scr[slot];
    return ODC_OK;
}

cudaEvent_t* mlp_ev_pair(MlpState* st, int kind) {
    if (st->ev_used >= 256) return nullptr;
    st->ev_kind[st->ev_used] = kind;
    cudaEvent_t* p = &st->ev[2 * st->ev_used];
    if (!p[0]) {
        if (cudaEventCreate(&p[0]) != cudaSuccess || cudaEventCreate(&p[1]) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
    }
    ++st->ev_used;
    return p;
}

void mlp_timing_begin(MlpState* st) {
    if (!st) return;
    st->ev_used = 0;
    st->flops[0] = st->flops[1] = st->flops[2] = 0.0;
    st->launches[0] = st->launches[1] = st->launches[2] = 0;
    st->n_split = 0;
}

void mlp_timing_collect(MlpState* st, int kind, float* ms, double* flops, int64_t* launches) {
    *ms = 0.0f;
    *flops = 0.0;
    *launches = 0;
    if (!st) return;
    for (int i = 0; i < st->ev_used; ++i) {
        if (st->ev_kind[i] != kind) continue;
        float t = 0.0f;
        if (cudaEventElapsedTime(&t, st->ev[2 * i], st->ev[2 * i + 1]) == cudaSuccess) *ms += t;
        else cudaGetLastError();
    }
    *flops = st->flops[kind];
    *launches = st->launches[kind];
}

void mlp_destroy(MlpState* st) {
    if (!st) return;
    for (auto& e : st->ev)
        if (e) cudaEventDestroy(e);
    if (st->wblob) cudaFree(st->wblob);
    for (int i = 0; i < kScratchSlots; ++i)
        if (st->scr[i]) cudaFree(st->scr[i]);
    mlp_tc_destroy(st);
    delete st;
}

// Upload weights: FP32 transposed copies for the SIMT path (W^T [in][out]),
// and the BF16 operand tiles of the tensor-core path.
odc_status mlp_prepare(MlpState** pst, const odc_mlp* m, cudaStream_t s, std::string* err) {
    odc_status r = mlp_check(m, err);
    if (r != ODC_OK) return r;
    if (!*pst) *pst = new MlpState();
    MlpState* st = *pst;
    st->precision = m->precision;
    st->band = m->band;
    st->split = m->no_split ? 0 : 1;
    st->zsplit = m->split_zmargin > 0.0f ? m->split_zmargin : 1e-4f;
    // |occ - 1/2| < band  <=>  |z| < 2 atanh(2 band)
    st->zband = (float)(2.0 * std::atanh(std::min(0.999999, 2.0 * (double)m->band)));
    st->scale = m->env_scale;
    st->radius = m->env_radius;
    st->amp = m->env_amp;
    const int din = 2 * kNF + m->latent_dim;
    std::vector<float> h(kBlobFloats, 0.0f);
    // B
    std::memcpy(&h[kOffB], m->B, sizeof(float) * kNF * 3);
    // layer 0: fold a constant latent into the bias (its columns multiply a
    // per-shape constant); W0^T for the Fourier columns only
    {
        const float* W = m->W[0];
        for (int k = 0; k < 2 * kNF; ++k)
            for (int n = 0; n < kH; ++n) h[kOffW[0] + (size_t)k * kH + n] = W[(size_t)n * din + m->latent_dim + k];
        for (int n = 0; n < kH; ++n) {
            double b = m->b[0][n];
            for (int j = 0; j < m->latent_dim; ++j) b += (double)W[(size_t)n * din + j] * (double)m->latent[j];
            h[kOffb[0] + n] = (float)b;
        }
    }
    for (int l = 1; l < kNL; ++l) {
        const float* W = m->W[l];
        for (int k = 0; k < kH; ++k)
            for (int n = 0; n < kH; ++n) h[kOffW[l] + (size_t)k * kH + n] = W[(size_t)n * kH + k];
        std::memcpy(&h[kOffb[l]], m->b[l], sizeof(float) * kH);
    }
    std::memcpy(&h[kOffW[kNL]], m->W[kNL], sizeof(float) * kH);
    h[kOffb[kNL]] = m->b[kNL][0];
    if (!st->wblob) MLP_CK(cudaMalloc((void**)&st->wblob, sizeof(float) * kBlobFloats));
    MLP_CK(cudaMemcpyAsync(st->wblob, h.data(), sizeof(float) * kBlobFloats, cudaMemcpyHostToDevice, s));
    r = mlp_tc_prepare(st, h.data(), s, err);
    if (r != ODC_OK) return r;
    return ODC_OK;
}

// ----------------------------------------------------------- FP32 network
#ifndef ODC_FP32_WARPS
#define ODC_FP32_WARPS 12
#endif
constexpr int kWarps = ODC_FP32_WARPS;   // one warp per 8 queries of the tile
constexpr int kTM = 8 * kWarps;          // queries per CTA
constexpr int kThreads = 32 * kWarps;
#ifndef ODC_FP32_KC
#define ODC_FP32_KC 32
#endif
constexpr int kKC = ODC_FP32_KC;         // weight rows per staged chunk
constexpr int kActStride = kH + 4;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// act[m][n] = relu(sum_k act[m][k] Wt[k][n] + b[n]) for the CTA's kTM queries,
// in place.  Thread (tr, tc): rows tr*8..tr*8+7, columns tc*4..tc*4+3 and
// 128+tc*4..+3.  The sums live in registers until every k has been read; the
// last chunk ends with a barrier before the epilogue overwrites the tile.
__device__ __forceinline__ void dense_relu(float* act, int K, const float* __restrict__ Wt,
                                           const float* __restrict__ bias, float* __restrict__ wbuf) {
    const int tid = threadIdx.x, tr = tid >> 5, tc = tid & 31;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
    const int nchunk = K / kKC;
    auto stage = [&](int c, int buf) {
        const float* src = Wt + (size_t)c * kKC * kH;
        float* dst = wbuf + buf * kKC * kH;
#pragma unroll
        for (int v = tid; v < kKC * kH / 4; v += kThreads) cp_async16(dst + 4 * v, src + 4 * v);
        cp_async_commit();
    };
    stage(0, 0);
    for (int c = 0; c < nchunk; ++c) {
        if (c + 1 < nchunk) {
            stage(c + 1, (c + 1) & 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const float* w = wbuf + (c & 1) * kKC * kH;
#pragma unroll
        for (int kk = 0; kk < kKC; kk += 4) {
            float4 a4[8];
#pragma unroll
            for (int i = 0; i < 8; ++i)
                a4[i] = *reinterpret_cast<const float4*>(act + (tr * 8 + i) * kActStride + c * kKC + kk);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float* wr = w + (kk + q) * kH;
                float4 w0 = *reinterpret_cast<const float4*>(wr + tc * 4);
                float4 w1 = *reinterpret_cast<const float4*>(wr + 128 + tc * 4);
                float wv[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    float av = q == 0 ? a4[i].x : (q == 1 ? a4[i].y : (q == 2 ? a4[i].z : a4[i].w));
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av, wv[j], acc[i][j]);
                }
            }
        }
        __syncthreads();
    }
    float4 b0 = *reinterpret_cast<const float4*>(bias + tc * 4);
    float4 b1 = *reinterpret_cast<const float4*>(bias + 128 + tc * 4);
    float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        float* o = act + (tr * 8 + i) * kActStride;
        float4 v0 = make_float4(fmaxf(acc[i][0] + bv[0], 0.f), fmaxf(acc[i][1] + bv[1], 0.f),
                                fmaxf(acc[i][2] + bv[2], 0.f), fmaxf(acc[i][3] + bv[3], 0.f));
        float4 v1 = make_float4(fmaxf(acc[i][4] + bv[4], 0.f), fmaxf(acc[i][5] + bv[5], 0.f),
                                fmaxf(acc[i][6] + bv[6], 0.f), fmaxf(acc[i][7] + bv[7], 0.f));
        *reinterpret_cast<float4*>(o + tc * 4) = v0;
        *reinterpret_cast<float4*>(o + 128 + tc * 4) = v1;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kThreads, 1)
    k_mlp_fp32(const float* __restrict__ wb, QuerySrc Q, int64_t n, float scale, float radius, float amp,
               float* __restrict__ zout) {
    extern __shared__ __align__(16) float sm[];
    float* act = sm;                         // [kTM][kActStride], layers run in place
    float* wbuf = sm + kTM * kActStride;     // two staged weight chunks
    __shared__ float3 xs[kTM];
    __shared__ float part[kTM][4];
    const int tid = threadIdx.x;
    const int64_t base = (int64_t)blockIdx.x * kTM;
    if (tid < kTM) {
        int64_t q = base + tid;
        xs[tid] = q < n ? query_point(Q, q) : make_float3(0.f, 0.f, 0.f);
    }
    __syncthreads();
    const float* B = wb + kOffB;
    for (int i = tid; i < kNF * kTM; i += kThreads) {
        int j = i / kTM, m = i % kTM;
        float2 sc = fourier_sincos(B[3 * j], B[3 * j + 1], B[3 * j + 2], xs[m]);
        act[m * kActStride + j] = sc.x;
        act[m * kActStride + kNF + j] = sc.y;
    }
    __syncthreads();
    for (int l = 0; l < kNL; ++l) dense_relu(act, l == 0 ? 2 * kNF : kH, wb + kOffW_(l), wb + kOffb_(l), wbuf);
    {
        int m = tid >> 2, p = tid & 3;
        const float* w5 = wb + kOffW[kNL];
        float s = 0.0f;
        for (int k = p * 64; k < p * 64 + 64; ++k) s = fmaf(act[m * kActStride + k], w5[k], s);
        part[m][p] = s;
    }
    __syncthreads();
    if (tid < kTM && base + tid < n) {
        float f = ((part[tid][0] + part[tid][1]) + (part[tid][2] + part[tid][3])) + wb[kOffb[kNL]];
        zout[base + tid] = envelope_logit(xs[tid], f, scale, radius, amp);
    }
}

static size_t fp32_smem() { return sizeof(float) * (kTM * kActStride + 2 * kKC * kH); }

static odc_status launch_fp32(MlpState* st, const QuerySrc& Q, int64_t n, float* z, cudaStream_t s, std::string* err) {
    if (n <= 0) return ODC_OK;
    static bool attr = false;
    if (!attr) {
        MLP_CK(cudaFuncSetAttribute(k_mlp_fp32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fp32_smem()));
        attr = true;
    }
    int64_t blocks = (n + kTM - 1) / kTM;
    cudaEvent_t* ev = mlp_ev_pair(st, 0);
    if (ev) MLP_CK(cudaEventRecord(ev[0], s));
    k_mlp_fp32<<<(unsigned)blocks, kThreads, fp32_smem(), s>>>(st->wblob, Q, n, st->scale, st->radius, st->amp, z); note_launch();
    if (ev) MLP_CK(cudaEventRecord(ev[1], s));
    MLP_CK(cudaGetLastError());
    int64_t real = n;
    if (!Q.pts) real = (int64_t)Q.g.nv[0] * Q.g.nv[1] * Q.g.nv[2];   // grid mode: padding lanes excluded
    st->flops[0] += kFlopsPerQuery * (double)real;
    st->launches[0] += 1;
    return ODC_OK;
}

// ------------------------------------------------------------ band re-eval
// Tier of every query: 0 = BF16 tensor-core pass first, 1 = split-FP16 pass
// first, 2 = FP32 directly.  hint[i] estimates |z_i - zt| (from the logits
// around the query in its search); no hint routes to the BF16 pass.
__global__ void k_route(const float* __restrict__ hint, int64_t n, float zs, float zb, int split,
                        uint8_t* __restrict__ r) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float h = hint ? hint[i] : INFINITY;
    r[i] = h < zs ? 2 : (h < zb ? (split ? 1 : 2) : 0);
}
// Queries of tier `from` whose logit lies within thr of t move to tier `to`;
// flag = the queries now in tier `to`.
__global__ void k_tier_flag(const float* __restrict__ z, int64_t n, float t, int from, int to, float thr,
                            uint8_t* __restrict__ r, uint32_t* __restrict__ flag) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int ri = r[i];
    if (ri == from && fabsf(z[i] - t) < thr) {
        ri = to;
        r[i] = (uint8_t)to;
    }
    flag[i] = ri == to ? 1u : 0u;
}
__global__ void k_band_gather(const uint32_t* __restrict__ flag, const uint32_t* __restrict__ off, int64_t n,
                              int* __restrict__ idx) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && flag[i]) idx[off[i]] = (int)i;
}
__global__ void k_band_scatter(const int* __restrict__ idx, const uint32_t* __restrict__ cnt,
                               const float* __restrict__ zr, float* __restrict__ z) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < *cnt) z[idx[i]] = zr[i];
}
__global__ void k_grid_points(GridDev g, const int* __restrict__ idx, const uint32_t* __restrict__ cnt,
                              float3* __restrict__ pts) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= *cnt) return;
    QuerySrc Q{nullptr, nullptr, g};
    pts[i] = query_point(Q, idx[i]);
}

__global__ void k_gather_pts(const float3* __restrict__ pts, const int* __restrict__ idx,
                             const uint32_t* __restrict__ cnt, float3* __restrict__ out) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < *cnt) out[i] = pts[idx[i]];
}

// Indices of the queries of tier `to` after promotion (see k_tier_flag), in
// increasing order (scratch slots base..base+3); the count is read back.
static odc_status tier_list(MlpState* st, const float* z, int64_t n, uint8_t* r, int from, int to, float thr,
                            int base, int** idx, uint32_t** dcnt, uint32_t* hcnt, cudaStream_t s, std::string* err) {
    void *pflag, *poff, *pidx, *pcnt;
    odc_status rc;
    if ((rc = mlp_scratch(st, base, n * 4 + 64, &pflag, err)) != ODC_OK) return rc;
    if ((rc = mlp_scratch(st, base + 1, n * 4 + scan_tmp_elems(n) * 8 + 64, &poff, err)) != ODC_OK) return rc;
    if ((rc = mlp_scratch(st, base + 2, n * 4 + 64, &pidx, err)) != ODC_OK) return rc;
    if ((rc = mlp_scratch(st, base + 3, 64, &pcnt, err)) != ODC_OK) return rc;
    uint32_t* flag = (uint32_t*)pflag;
    uint32_t* off = (uint32_t*)poff;
    uint32_t* tmp = off + ((n + 63) / 64) * 64;
    unsigned blocks = (unsigned)((n + 255) / 256);
    k_tier_flag<<<blocks, 256, 0, s>>>(z, n, st->zt, from, to, thr, r, flag); note_launch();
    exclusive_scan<uint32_t>(flag, off, (size_t)n, tmp, (uint32_t*)pcnt, s);
    k_band_gather<<<blocks, 256, 0, s>>>(flag, off, n, (int*)pidx); note_launch();
    MLP_CK(cudaMemcpyAsync(hcnt, pcnt, 4, cudaMemcpyDeviceToHost, s));
    MLP_CK(cudaStreamSynchronize(s));
    *idx = (int*)pidx;
    *dcnt = (uint32_t*)pcnt;
    return ODC_OK;
}

// Points of the listed queries (scratch slot ps).
static odc_status gather_points(MlpState* st, const QuerySrc& Q, const int* idx, const uint32_t* dcnt, uint32_t m,
                                int ps, float3** out, cudaStream_t s, std::string* err) {
    void* p;
    odc_status rc;
    if ((rc = mlp_scratch(st, ps, (size_t)m * 12 + 64, &p, err)) != ODC_OK) return rc;
    if (Q.idx) { *err = "nested gather"; return ODC_ERR_INTERNAL; }
    if (Q.pts) {
        k_gather_pts<<<(m + 255) / 256, 256, 0, s>>>(Q.pts, idx, dcnt, (float3*)p); note_launch();
    } else {
        k_grid_points<<<(m + 255) / 256, 256, 0, s>>>(Q.g, idx, dcnt, (float3*)p); note_launch();
    }
    *out = (float3*)p;
    return ODC_OK;
}

// Tiered evaluation (A.2.2 binary decision at iso): the sign of every logit
// equals the FP32 plain path's.  A logit of the BF16 pass is kept only
// outside the band |z - zt| >= zband; the split-FP16 tensor-core network
// (measured error below zsplit / 3) re-takes the band and keeps |z - zt| >=
// zsplit; the FP32 SIMT network takes the rest.  Without the split tier the
// whole band goes to FP32.  With hints, queries predicted inside the band
// (or inside zsplit) start at the split (or FP32) tier: the tiers' acceptance
// rules are unchanged, so only the cost depends on the hints.
static odc_status eval_tiered(MlpState* st, const QuerySrc& Q, int64_t n, float* z, const float* hint, cudaStream_t s,
                              int64_t* nrq, std::string* err) {
    odc_status r;
    void* pr;
    if ((r = mlp_scratch(st, 24, (size_t)n + 64, &pr, err)) != ODC_OK) return r;
    uint8_t* route = (uint8_t*)pr;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    k_route<<<blocks, 256, 0, s>>>(hint, n, st->zsplit, st->zband, st->split, route); note_launch();
    if (!hint) {
        if ((r = mlp_tc_eval(st, Q, n, z, s, err)) != ODC_OK) return r;
    } else {
        int* idx0;
        uint32_t *dc0, n0 = 0;
        if ((r = tier_list(st, z, n, route, -1, 0, 0.0f, 28, &idx0, &dc0, &n0, s, err)) != ODC_OK) return r;
        if (n0) {
            float3* p0;
            void* pz0;
            if ((r = gather_points(st, Q, idx0, dc0, n0, 32, &p0, s, err)) != ODC_OK) return r;
            if ((r = mlp_scratch(st, 33, (size_t)n0 * 4 + 64, &pz0, err)) != ODC_OK) return r;
            QuerySrc L0{p0, nullptr, Q.g};
            if ((r = mlp_tc_eval(st, L0, n0, (float*)pz0, s, err)) != ODC_OK) return r;
            k_band_scatter<<<(n0 + 255) / 256, 256, 0, s>>>(idx0, dc0, (const float*)pz0, z); note_launch();
        }
    }
    if (st->split) {
        int* idx1;
        uint32_t *dc1, n1 = 0;
        if ((r = tier_list(st, z, n, route, 0, 1, st->zband, 4, &idx1, &dc1, &n1, s, err)) != ODC_OK) return r;
        if ((r = mlp_tc_check(st, err)) != ODC_OK) return r;
        if (n1) {
            float3* p1;
            void* pz1;
            if ((r = gather_points(st, Q, idx1, dc1, n1, 8, &p1, s, err)) != ODC_OK) return r;
            if ((r = mlp_scratch(st, 9, (size_t)n1 * 4 + 64, &pz1, err)) != ODC_OK) return r;
            QuerySrc L1{p1, nullptr, Q.g};
            if ((r = mlp_tc3_eval(st, L1, n1, (float*)pz1, s, err)) != ODC_OK) return r;
            k_band_scatter<<<(n1 + 255) / 256, 256, 0, s>>>(idx1, dc1, (const float*)pz1, z); note_launch();
            st->n_split += n1;
        }
    }
    int* idx2;
    uint32_t *dc2, n2 = 0;
    const int from = st->split ? 1 : 0;
    const float thr = st->split ? st->zsplit : st->zband;
    if ((r = tier_list(st, z, n, route, from, 2, thr, 16, &idx2, &dc2, &n2, s, err)) != ODC_OK) return r;
    if ((r = mlp_tc_check(st, err)) != ODC_OK) return r;
    *nrq += n2;
    if (n2) {
        float3* p2;
        void* pz2;
        if ((r = gather_points(st, Q, idx2, dc2, n2, 20, &p2, s, err)) != ODC_OK) return r;
        if ((r = mlp_scratch(st, 21, (size_t)n2 * 4 + 64, &pz2, err)) != ODC_OK) return r;
        QuerySrc L2{p2, nullptr, Q.g};
        if ((r = launch_fp32(st, L2, n2, (float*)pz2, s, err)) != ODC_OK) return r;
        k_band_scatter<<<(n2 + 255) / 256, 256, 0, s>>>(idx2, dc2, (const float*)pz2, z); note_launch();
    }
    MLP_CK(cudaGetLastError());
    return ODC_OK;
}

static odc_status eval(MlpState* st, const QuerySrc& Q, int64_t n, float* z, int precision, const float* hint,
                       cudaStream_t s, int64_t* nrq, std::string* err) {
    if (precision < 0) precision = st->precision;
    if (precision == ODC_PREC_FP32) return launch_fp32(st, Q, n, z, s, err);
    if (precision == ODC_PREC_SPLIT) return mlp_tc3_eval(st, Q, n, z, s, err);
    return eval_tiered(st, Q, n, z, hint, s, nrq, err);
}

odc_status mlp_eval_list(MlpState* st, const float3* pts, int64_t n, float* z, int precision, cudaStream_t s,
                         int64_t* nrq, std::string* err, const float* hint) {
    QuerySrc Q{pts, nullptr, GridDev{}};
    return eval(st, Q, n, z, precision, hint, s, nrq, err);
}

odc_status mlp_eval_grid(MlpState* st, const GridDev& g, float* z, cudaStream_t s, int64_t* nrq, std::string* err) {
    QuerySrc Q{nullptr, nullptr, g};
    int64_t n = (int64_t)g.W * g.nv[1] * g.nv[2] * 32;
    return eval(st, Q, n, z, -1, nullptr, s, nrq, err);
}

__global__ void k_pts_labels(const float* __restrict__ z, int64_t n, float t, uint8_t* __restrict__ lab) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) lab[i] = z[i] > t ? 1 : 0;
}

odc_status mlp_points(MlpState* st, const float3* pts, int64_t n, float iso, int precision, uint8_t* labels,
                      float* logits, cudaStream_t s, std::string* err) {
    int64_t nrq = 0;
    st->zt = mlp_logit_threshold(iso);
    odc_status r = mlp_eval_list(st, pts, n, logits, precision, s, &nrq, err);
    if (r != ODC_OK) return r;
    k_pts_labels<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(logits, n, mlp_logit_threshold(iso), labels); note_launch();
    MLP_CK(cudaGetLastError());
    return ODC_OK;
}

}  // namespace odc
