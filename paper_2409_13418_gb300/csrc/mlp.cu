// mlp.cu -- envelope-MLP occupancy network on the device.
//
// f(x) = W5 relu(W4 relu(W3 relu(W2 relu(W1 g(x) + b1) + b2) + b3) + b4) + b5,
// g(x) = [sin(2 pi B x), cos(2 pi B x)] (64 frequencies), z = scale (radius -
// |x| + amp f(x)).  The FP32 path (this file) is the plain reference path of
// the GPU: SIMT FMAs, register-tiled 64-query x 256-output tiles, the
// Fourier phase B.x formed exactly in float-float and reduced to one period
// before sincospi.  The BF16 tensor-core path lives in mlp_tc.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "batch.h"
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
    if (m->precision != ODC_PREC_FP32 && m->precision != ODC_PREC_BF16 && m->precision != ODC_PREC_FP8)
        { *err = "precision must be FP32, BF16 or FP8"; return ODC_ERR_INVALID_ARG; }
    if (m->precision != ODC_PREC_FP32 && !(m->band >= 0.0f && m->band < 0.5f))
        { *err = "band must be in [0, 0.5)"; return ODC_ERR_INVALID_ARG; }
    if (!(m->split_zmargin >= 0.0f)) { *err = "split_zmargin must be >= 0"; return ODC_ERR_INVALID_ARG; }
    if (!(m->h16_zmargin >= 0.0f)) { *err = "h16_zmargin must be >= 0"; return ODC_ERR_INVALID_ARG; }
    if (!(m->split_acc_comp < 1e-3f)) { *err = "split_acc_comp must be below 1e-3"; return ODC_ERR_INVALID_ARG; }
    return ODC_OK;
}

float mlp_logit_threshold(float iso) { return (float)std::log((double)iso / (1.0 - (double)iso)); }

int mlp_precision(const MlpState* st) { return st->precision; }
void mlp_set_wait_limit(MlpState* st, unsigned long long ns, const int* gate) {
    if (!st) return;
    st->wait_ns = ns;
    st->gate = gate;
}
int64_t mlp_split_count(const MlpState* st) { return st ? (int64_t)st->hq[1] : 0; }
int64_t mlp_fp32_requery_count(const MlpState* st) { return st ? (int64_t)st->hq[2] : 0; }
int64_t mlp_h16_count(const MlpState* st) { return st ? (int64_t)st->hq[3] : 0; }
int64_t mlp_fp8_count(const MlpState* st) { return st ? (int64_t)st->hq[4] : 0; }

#define MLP_CK(call)                                                                        \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) { *err = std::string(#call) + ": " + cudaGetErrorString(e_); \
                                 return ODC_ERR_CUDA; }                                     \
    } while (0)

odc_status mlp_scratch(MlpState* st, int slot, size_t bytes, void** out, std::string* err) {
    if (st->scr_cap[slot] < bytes) {
        // stream-ordered on the stream of the current call: growth waits for
        // no other stream or context
        if (st->scr[slot]) {
            MLP_CK(cudaFreeAsync(st->scr[slot], st->stream));
            st->scr[slot] = nullptr;
            st->scr_cap[slot] = 0;
        }
        size_t want = bytes + bytes / 4 + 4096;
        cudaError_t e = cudaMallocAsync(&st->scr[slot], want, st->stream);
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

// Each tensor-core pass costs a search round a launch of ~25 us even when
// its list is short (one tile's chain of weight slices and four layers);
// per query the FP16 tier saves (1.33 - 0.65) ns and the BF16 pass (1.33 -
// 0.56) ns against the split tier.  With fewer crossing edges than this
// (about a 128^3 surface of the envelope networks) their search-round
// launches cost more than they save: the search queries then start at the
// split tier (or the FP32 tier) instead, with the same decisions.  The grid
// pass keeps every tier.
constexpr int64_t kSmallSurfaceEdges = 250000;
void mlp_size_tiers(MlpState* st, int64_t n_edges) {
    if (!st) return;
    st->h16_run = st->h16 && n_edges >= kSmallSurfaceEdges;
    st->first_run = n_edges >= kSmallSurfaceEdges;
}

void mlp_timing_begin(MlpState* st, cudaStream_t s) {
    if (!st) return;
    st->h16_run = st->h16;
    st->first_run = 1;
    st->ev_used = 0;
    for (auto& f : st->flops) f = 0.0;
    for (auto& l : st->launches) l = 0;
    for (auto& v : st->hq) v = 0;
    if (st->dq) cudaMemsetAsync(st->dq, 0, 16 * sizeof(unsigned long long), s);
}

void mlp_timing_finish(MlpState* st, cudaStream_t s) {
    if (!st || !st->dq) return;
    if (cudaMemcpyAsync(st->hq, st->dq, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(st->hq + 4, st->dq + 10, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        for (auto& v : st->hq) v = 0;
    }
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
    // device-sized lists: hq[0] BF16, hq[1] split-FP16 (three products), hq[2] FP32, hq[3] FP16, hq[4] FP8
    const double dev = kind == 0   ? (double)st->hq[2]
                       : kind == 1 ? (double)st->hq[0]
                       : kind == 2 ? 3.0 * (double)st->hq[1]
                       : kind == 3 ? (double)st->hq[3]
                                   : (double)st->hq[4];
    *flops = st->flops[kind] + kFlopsPerQuery * dev;
    *launches = st->launches[kind];
}

void mlp_destroy(MlpState* st) {
    if (!st) return;
    batch_unbind(st);
    if (st->bev) cudaEventDestroy(st->bev);
    for (auto& e : st->ev)
        if (e) cudaEventDestroy(e);
    if (st->wblob) cudaFree(st->wblob);
    if (st->dq) cudaFree(st->dq);
    for (int i = 0; i < kScratchSlots; ++i)
        if (st->scr[i]) cudaFree(st->scr[i]);
    mlp_tc_destroy(st);
    delete st;
}

size_t mlp_device_bytes(const MlpState* st) {
    if (!st) return 0;
    size_t b = st->wblob ? sizeof(float) * kBlobFloats : 0;
    for (int i = 0; i < kScratchSlots; ++i) b += st->scr_cap[i];
    return b + mlp_tc_device_bytes(st);
}

static odc_status fp32_kernel_setup(std::string* err);
static odc_status fp32_autotune(MlpState* st, cudaStream_t s, std::string* err);
static odc_status split_calibrate(MlpState* st, cudaStream_t s, std::string* err);
constexpr int kFp32VariantCount = 4;

// Upload weights: FP32 transposed copies for the SIMT path (W^T [in][out]),
// and the BF16 operand tiles of the tensor-core path.
odc_status mlp_prepare(MlpState** pst, const odc_mlp* m, cudaStream_t s, std::string* err) {
    odc_status r = mlp_check(m, err);
    if (r != ODC_OK) return r;
    if (!*pst) *pst = new MlpState();
    MlpState* st = *pst;
    st->stream = s;
    if (!st->sms) {
        int dev = 0;
        MLP_CK(cudaGetDevice(&dev));
        MLP_CK(cudaDeviceGetAttribute(&st->sms, cudaDevAttrMultiProcessorCount, dev));
    }
    if (!st->dq) {
        MLP_CK(cudaMalloc((void**)&st->dq, 16 * sizeof(unsigned long long)));
        odc_status r0 = fp32_kernel_setup(err);
        if (r0 != ODC_OK) return r0;
    }
    {
        const int f = (m->flags >> 8) & 0xf;
        if ((m->flags & ~(ODC_MLP_REUPLOAD | ODC_MLP_NO_F16_TIER | 0xf00)) || f > kFp32VariantCount) {
            *err = "unknown MLP flags";
            return ODC_ERR_INVALID_ARG;
        }
        st->fp32_forced = f - 1;
    }
    // FP8: the BF16 path's tiers behind an FP8 pass
    st->precision = m->precision == ODC_PREC_FP8 ? ODC_PREC_BF16 : m->precision;
    st->fp8 = m->precision == ODC_PREC_FP8 ? 1 : 0;
    st->band = m->band;
    st->split = m->no_split ? 0 : 1;
    st->h16 = (m->flags & ODC_MLP_NO_F16_TIER) ? 0 : 1;
    st->h16_run = st->h16;
    st->first_run = 1;
    st->zsplit_user = m->split_zmargin;
    st->zsplit = m->split_zmargin > 0.0f ? m->split_zmargin : (st->zsplit_cal > 0.0f ? st->zsplit_cal : 2e-5f);
    st->zh16 = m->h16_zmargin > 0.0f ? m->h16_zmargin : 0.025f;
    st->split_comp = m->split_acc_comp;
    // |occ - 1/2| < band  <=>  |z| < 2 atanh(2 band)
    st->zband = (float)(2.0 * std::atanh(std::min(0.999999, 2.0 * (double)m->band)));
    st->scale = m->env_scale;
    st->radius = m->env_radius;
    st->amp = m->env_amp;
    const int din = 2 * kNF + m->latent_dim;
    // Weights already on the device (same B, W, b; only the latent may
    // differ, as for latent-conditioned shapes of one network): refresh the
    // folded first-layer bias and keep everything else.
    std::vector<float> key;
    key.reserve(kBlobFloats + (size_t)kH * m->latent_dim + 8);
    key.push_back((float)m->latent_dim);
    key.push_back(st->split_comp);   // part of the prepared split-tier operands
    key.insert(key.end(), m->B, m->B + kNF * 3);
    for (int l = 0; l <= kNL; ++l) {
        size_t rows = l == kNL ? 1 : kH, cols = l == 0 ? (size_t)din : kH;
        key.insert(key.end(), m->W[l], m->W[l] + rows * cols);
        key.insert(key.end(), m->b[l], m->b[l] + rows);
    }
    if (st->wblob && !(m->flags & ODC_MLP_REUPLOAD) && key == st->wkey) {
        std::vector<float> b0(kH);
        for (int n = 0; n < kH; ++n) {
            double b = m->b[0][n];
            for (int j = 0; j < m->latent_dim; ++j) b += (double)m->W[0][(size_t)n * din + j] * (double)m->latent[j];
            b0[n] = (float)b;
        }
        MLP_CK(cudaMemcpyAsync(st->wblob + kOffb[0], b0.data(), sizeof(float) * kH, cudaMemcpyHostToDevice, s));
        MLP_CK(cudaStreamSynchronize(s));   // b0 is a host temporary
        st->b0host = b0;
        st->b0dirty = true;
        return ODC_OK;
    }
    const bool same_weights = st->wblob && key == st->wkey;   // a forced re-upload
    st->wkey.clear();   // set again once the upload below has succeeded
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
    st->b0host.assign(h.begin() + kOffb[0], h.begin() + kOffb[0] + kH);
    st->b0dirty = true;
    std::memcpy(&h[kOffW[kNL]], m->W[kNL], sizeof(float) * kH);
    h[kOffb[kNL]] = m->b[kNL][0];
    if (!st->wblob) MLP_CK(cudaMalloc((void**)&st->wblob, sizeof(float) * kBlobFloats));
    MLP_CK(cudaMemcpyAsync(st->wblob, h.data(), sizeof(float) * kBlobFloats, cudaMemcpyHostToDevice, s));
    r = mlp_tc_prepare(st, h.data(), s, err);
    if (r != ODC_OK) return r;
    if (st->fp32_variant < 0 && (r = fp32_autotune(st, s, err)) != ODC_OK) return r;
    // the split tier's accumulation compensation and margin for these weights
    if (same_weights && st->split_comp_used >= 0.0f && st->zsplit_cal > 0.0f) {
        r = mlp_tc_set_comp(st, st->split_comp_used, s, err);
    } else {
        r = split_calibrate(st, s, err);
    }
    if (r != ODC_OK) return r;
    st->zsplit = st->zsplit_user > 0.0f ? st->zsplit_user : st->zsplit_cal;
    st->wkey.swap(key);
    return ODC_OK;
}

// ----------------------------------------------------------- FP32 network
// Register tiles of 8 rows (queries) x 8 columns per thread; a warp's lanes
// form 4 x 8 threads (32 rows x 64 columns), the CTA's warps 4 column blocks
// x WARPS / 4 row blocks.  Activations sit transposed in shared memory
// (act[k][m], k-major), so that a thread's 8 rows at one k are two vector
// loads, shared by the 8 lanes of its row group.  The tile shape (warps,
// weight rows per staged chunk, chunks in flight) is a template parameter:
// every shape computes the same bits (each output sums its products in
// order k = 0..K-1 with one rounding per FMA), and the autotuner below picks
// the fastest on the device at hand.
template <int WARPS, int KC, int STAGES>
struct Fp32Tile {
    static constexpr int kWarps = WARPS;
    static constexpr int kTM = WARPS / 4 * 32;         // queries per CTA
    static constexpr int kThreads = 32 * WARPS;
    static constexpr int kKC = KC;                     // weight rows per staged chunk
    static constexpr int kWStages = STAGES;            // weight chunks in flight (ring)
    static constexpr int kActStride = kTM + 4;         // floats between consecutive k of act[k][m]
    static constexpr size_t kSmem = sizeof(float) * (kH * kActStride + STAGES * KC * kH);
    static_assert(WARPS % 4 == 0 && kTM <= kThreads && STAGES >= 2 && kSmem <= 220 * 1024, "FP32 tile shape");
};
constexpr int kFUnroll = 16;              // k steps unrolled in the inner loop

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// act[n][m] = relu(sum_k act[k][m] Wt[k][n] + b[n]) for the CTA's kTM queries,
// in place.  Lane (ty, tx) = (lane / 8, lane % 8) of warp w: rows
// (w / 4) 32 + ty 8 .. + 7, columns (w % 4) 64 + tx 4 .. + 3 and 32 more.
// The sums live in registers until every k has been read; the last chunk
// ends with a barrier before the epilogue overwrites the tile.
template <class T>
__device__ __forceinline__ void dense_relu(float* act, int K, const float* __restrict__ Wt,
                                           const float* __restrict__ bias, float* __restrict__ wbuf,
                                           const float* const* rowb = nullptr) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row0 = (warp >> 2) * 32 + (lane >> 3) * 8;
    const int col0 = (warp & 3) * 64 + (lane & 7) * 4;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
    const int nchunk = K / T::kKC;
    // ring of kWStages chunk buffers: chunk c + kWStages - 1 is issued at the
    // top of chunk c into the buffer chunk c - 1 used, which every thread
    // has left once it passed chunk c's barrier (one barrier per chunk)
    auto stage = [&](int c) {
        if (c < nchunk) {
            const float* src = Wt + (size_t)c * T::kKC * kH;
            float* dst = wbuf + (c % T::kWStages) * T::kKC * kH;
#pragma unroll
            for (int v = tid; v < T::kKC * kH / 4; v += T::kThreads) cp_async16(dst + 4 * v, src + 4 * v);
        }
        cp_async_commit();   // possibly empty: keeps the group count uniform
    };
#pragma unroll
    for (int c = 0; c < T::kWStages - 1; ++c) stage(c);
    for (int c = 0; c < nchunk; ++c) {
        cp_async_wait<T::kWStages - 2>();   // chunk c has landed (this thread's copies)
        __syncthreads();                    // ... and every thread's; chunk c - 1 is released
        stage(c + T::kWStages - 1);
        const float* w = wbuf + (c % T::kWStages) * T::kKC * kH + col0;
        const float* a = act + (size_t)(c * T::kKC) * T::kActStride + row0;
#pragma unroll kFUnroll
        for (int kk = 0; kk < T::kKC; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4*>(a + kk * T::kActStride);
            const float4 a1 = *reinterpret_cast<const float4*>(a + kk * T::kActStride + 4);
            const float4 w0 = *reinterpret_cast<const float4*>(w + kk * kH);
            const float4 w1 = *reinterpret_cast<const float4*>(w + kk * kH + 32);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float wv[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
            // column-outer order: measured 4% faster than row-outer on this part
#pragma unroll
            for (int j = 0; j < 8; ++j)
#pragma unroll
                for (int i = 0; i < 8; ++i) acc[i][j] = fmaf(av[i], wv[j], acc[i][j]);
        }
    }
    cp_async_wait<0>();
    __syncthreads();   // every thread has read the last chunk and the whole input tile
    if (rowb) {   // a bias row per query (rowb[m]: row of tile query m)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int col = col0 + (j < 4 ? j : 28 + j);
            float* o = act + (size_t)col * T::kActStride + row0;
            float b[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) b[i] = rowb[row0 + i][col];
            *reinterpret_cast<float4*>(o) = make_float4(fmaxf(acc[0][j] + b[0], 0.f), fmaxf(acc[1][j] + b[1], 0.f),
                                                        fmaxf(acc[2][j] + b[2], 0.f), fmaxf(acc[3][j] + b[3], 0.f));
            *reinterpret_cast<float4*>(o + 4) = make_float4(fmaxf(acc[4][j] + b[4], 0.f), fmaxf(acc[5][j] + b[5], 0.f),
                                                            fmaxf(acc[6][j] + b[6], 0.f), fmaxf(acc[7][j] + b[7], 0.f));
        }
    } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int col = col0 + (j < 4 ? j : 28 + j);
            const float b = bias[col];
            float* o = act + (size_t)col * T::kActStride + row0;
            *reinterpret_cast<float4*>(o) = make_float4(fmaxf(acc[0][j] + b, 0.f), fmaxf(acc[1][j] + b, 0.f),
                                                        fmaxf(acc[2][j] + b, 0.f), fmaxf(acc[3][j] + b, 0.f));
            *reinterpret_cast<float4*>(o + 4) = make_float4(fmaxf(acc[4][j] + b, 0.f), fmaxf(acc[5][j] + b, 0.f),
                                                            fmaxf(acc[6][j] + b, 0.f), fmaxf(acc[7][j] + b, 0.f));
        }
    }
    __syncthreads();
}

// Small lists: a full tile costs the same whatever its number of real
// queries (every chunk of every layer runs over all its rows), so a list of
// a few thousand queries would leave most SMs idle behind one long tile per
// SM.  Lists of at most kSmallN queries run as tiles of kSM = 32 queries
// instead, four times as many CTAs for the same list: lane (ty, tx) =
// (lane / 4, lane % 4) of warp w takes rows ty 4 .. + 3 and columns w 16 +
// tx 4 .. + 3.  Each output still sums its products in order k = 0..K-1,
// one rounding per FMA: the same bits as the full tiles.
constexpr int kSM = 32;                    // queries per small tile
constexpr int kSmallStride = kSM + 4;      // floats between consecutive k of the small act[k][m]
template <class T>
__device__ __forceinline__ void dense_relu_small(float* act, int K, const float* __restrict__ Wt,
                                                 const float* __restrict__ bias, float* __restrict__ wbuf,
                                                 const float* const* rowb) {
    static_assert(T::kWarps == 16, "small tiles: 16 warps x 16 columns");
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row0 = (lane >> 2) * 4;
    const int col0 = warp * 16 + (lane & 3) * 4;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
    const int nchunk = K / T::kKC;
    auto stage = [&](int c) {
        if (c < nchunk) {
            const float* src = Wt + (size_t)c * T::kKC * kH;
            float* dst = wbuf + (c % T::kWStages) * T::kKC * kH;
#pragma unroll
            for (int v = tid; v < T::kKC * kH / 4; v += T::kThreads) cp_async16(dst + 4 * v, src + 4 * v);
        }
        cp_async_commit();
    };
#pragma unroll
    for (int c = 0; c < T::kWStages - 1; ++c) stage(c);
    for (int c = 0; c < nchunk; ++c) {
        cp_async_wait<T::kWStages - 2>();
        __syncthreads();
        stage(c + T::kWStages - 1);
        const float* w = wbuf + (c % T::kWStages) * T::kKC * kH + col0;
        const float* a = act + (size_t)(c * T::kKC) * kSmallStride + row0;
#pragma unroll 8
        for (int kk = 0; kk < T::kKC; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4*>(a + kk * kSmallStride);
            const float4 w0 = *reinterpret_cast<const float4*>(w + kk * kH);
            const float av[4] = {a0.x, a0.y, a0.z, a0.w};
            const float wv[4] = {w0.x, w0.y, w0.z, w0.w};
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int i = 0; i < 4; ++i) acc[i][j] = fmaf(av[i], wv[j], acc[i][j]);
        }
    }
    cp_async_wait<0>();
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int col = col0 + j;
        float b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) b[i] = rowb ? rowb[row0 + i][col] : bias[col];
        *reinterpret_cast<float4*>(act + (size_t)col * kSmallStride + row0) =
            make_float4(fmaxf(acc[0][j] + b[0], 0.f), fmaxf(acc[1][j] + b[1], 0.f), fmaxf(acc[2][j] + b[2], 0.f),
                        fmaxf(acc[3][j] + b[3], 0.f));
    }
    __syncthreads();
}

// Persistent: each CTA walks the tiles blockIdx.x, blockIdx.x + gridDim.x, ...
// of min(n, *Q.cnt) queries (the tile loop is uniform within a CTA).
template <class T>
__global__ void __launch_bounds__(T::kThreads, 1)
    k_mlp_fp32(const float* __restrict__ wb, QuerySrc Q, int64_t n_max, float scale, float radius, float amp,
               float* __restrict__ zout) {
    extern __shared__ __align__(16) float sm[];
    float* act = sm;                            // [kH][kActStride], layers run in place
    float* wbuf = sm + kH * T::kActStride;      // kWStages staged weight chunks
    __shared__ float3 xs[T::kTM];
    __shared__ float part[T::kTM][4];
    __shared__ const float* rowb[T::kTM];   // per-query first-layer bias rows (Q.b0tab)
    const int tid = threadIdx.x;
    const int64_t n = query_count(Q, n_max);
    const float* B = wb + kOffB;
    // Full tiles cover whole waves of the grid; a remainder of at most three
    // small-tile rounds (and any list that small) runs as 32-query tiles over
    // the whole grid instead of a last, partly filled wave of full tiles.
    int64_t n_big = n;
    if constexpr (T::kWarps == 16) {
        const int64_t wave = (int64_t)gridDim.x * T::kTM;
        const int64_t rem = n % wave;
        if (rem <= (int64_t)gridDim.x * kSM * 3) n_big = n - rem;
    }
    for (int64_t base = (int64_t)blockIdx.x * T::kTM; base < n_big; base += (int64_t)gridDim.x * T::kTM) {
        if (tid < T::kTM) {
            int64_t q = base + tid;
            xs[tid] = q < n ? query_point(Q, q) : make_float3(0.f, 0.f, 0.f);
            if (Q.b0tab) rowb[tid] = q < n ? query_b0(Q, query_index(Q, q)) : wb + kOffb_(0);
        }
        __syncthreads();
        for (int i = tid; i < kNF * T::kTM; i += T::kThreads) {
            int j = i / T::kTM, m = i % T::kTM;
            float2 sc = fourier_sincos(B[3 * j], B[3 * j + 1], B[3 * j + 2], xs[m]);
            act[j * T::kActStride + m] = sc.x;
            act[(kNF + j) * T::kActStride + m] = sc.y;
        }
        __syncthreads();
        for (int l = 0; l < kNL; ++l)
            dense_relu<T>(act, l == 0 ? 2 * kNF : kH, wb + kOffW_(l), wb + kOffb_(l), wbuf,
                          l == 0 && Q.b0tab ? rowb : nullptr);
        for (int t = tid; t < 4 * T::kTM; t += T::kThreads) {
            const int m = t % T::kTM, p = t / T::kTM;
            const float* w5 = wb + kOffW[kNL];
            float s = 0.0f;
            for (int k = p * 64; k < p * 64 + 64; ++k) s = fmaf(act[k * T::kActStride + m], w5[k], s);
            part[m][p] = s;
        }
        __syncthreads();
        if (tid < T::kTM && base + tid < n) {
            float f = ((part[tid][0] + part[tid][1]) + (part[tid][2] + part[tid][3])) + wb[kOffb[kNL]];
            zout[query_index(Q, base + tid)] = envelope_logit(xs[tid], f, scale, radius, amp);
        }
    }
    __syncthreads();   // the small tiles reuse xs, part and the activation buffer
    if constexpr (T::kWarps == 16) {
        // the small-tile remainder [n_big, n)
        for (int64_t base = n_big + (int64_t)blockIdx.x * kSM; base < n; base += (int64_t)gridDim.x * kSM) {
            if (tid < kSM) {
                int64_t q = base + tid;
                xs[tid] = q < n ? query_point(Q, q) : make_float3(0.f, 0.f, 0.f);
                if (Q.b0tab) rowb[tid] = q < n ? query_b0(Q, query_index(Q, q)) : wb + kOffb_(0);
            }
            __syncthreads();
            for (int i = tid; i < kNF * kSM; i += T::kThreads) {
                int j = i / kSM, m = i % kSM;
                float2 sc = fourier_sincos(B[3 * j], B[3 * j + 1], B[3 * j + 2], xs[m]);
                act[j * kSmallStride + m] = sc.x;
                act[(kNF + j) * kSmallStride + m] = sc.y;
            }
            __syncthreads();
            for (int l = 0; l < kNL; ++l)
                dense_relu_small<T>(act, l == 0 ? 2 * kNF : kH, wb + kOffW_(l), wb + kOffb_(l), wbuf,
                                    l == 0 && Q.b0tab ? rowb : nullptr);
            for (int t = tid; t < 4 * kSM; t += T::kThreads) {
                const int m = t % kSM, p = t / kSM;
                const float* w5 = wb + kOffW[kNL];
                float s = 0.0f;
                for (int k = p * 64; k < p * 64 + 64; ++k) s = fmaf(act[k * kSmallStride + m], w5[k], s);
                part[m][p] = s;
            }
            __syncthreads();
            if (tid < kSM && base + tid < n) {
                float f = ((part[tid][0] + part[tid][1]) + (part[tid][2] + part[tid][3])) + wb[kOffb[kNL]];
                zout[query_index(Q, base + tid)] = envelope_logit(xs[tid], f, scale, radius, amp);
            }
            __syncthreads();   // part and xs are reused by the next tile
        }
    }
}

// The tile shapes the autotuner chooses from (warps, K chunk, chunks in
// flight); index 0 is the shape measured best on GB300 and the fallback.
using Fp32T0 = Fp32Tile<16, 32, 2>;
using Fp32T1 = Fp32Tile<16, 16, 3>;
using Fp32T2 = Fp32Tile<12, 32, 3>;
using Fp32T3 = Fp32Tile<8, 32, 3>;
constexpr int kFp32Variants = kFp32VariantCount;

template <class T>
static void launch_fp32_tile(const MlpState* st, const QuerySrc& Q, int64_t n, float* z, cudaStream_t s) {
    // enough CTAs for the small-list path's 32-query tiles when n is small
    const int64_t tiles = (n + kSM - 1) / kSM;
    const unsigned grid = (unsigned)std::min<int64_t>(tiles, (int64_t)std::max(st->sms, 1));
    k_mlp_fp32<T><<<grid, T::kThreads, T::kSmem, s>>>(st->wblob, Q, n, st->scale, st->radius, st->amp, z);
    note_launch();
}

static void launch_fp32_variant(int v, const MlpState* st, const QuerySrc& Q, int64_t n, float* z, cudaStream_t s) {
    switch (v) {
        case 1: launch_fp32_tile<Fp32T1>(st, Q, n, z, s); break;
        case 2: launch_fp32_tile<Fp32T2>(st, Q, n, z, s); break;
        case 3: launch_fp32_tile<Fp32T3>(st, Q, n, z, s); break;
        default: launch_fp32_tile<Fp32T0>(st, Q, n, z, s); break;
    }
}

static odc_status fp32_kernel_setup(std::string* err) {
    MLP_CK(cudaFuncSetAttribute(k_mlp_fp32<Fp32T0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Fp32T0::kSmem));
    MLP_CK(cudaFuncSetAttribute(k_mlp_fp32<Fp32T1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Fp32T1::kSmem));
    MLP_CK(cudaFuncSetAttribute(k_mlp_fp32<Fp32T2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Fp32T2::kSmem));
    MLP_CK(cudaFuncSetAttribute(k_mlp_fp32<Fp32T3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Fp32T3::kSmem));
    return ODC_OK;
}

// Deterministic calibration points in [-1, 1]^3 (a hash of the index).
__global__ void k_calib_points(float3* p, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t h = (uint64_t)i * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
    float c[3];
    for (int a = 0; a < 3; ++a) {
        h ^= h >> 29;
        h *= 0xBF58476D1CE4E5B9ull;
        h ^= h >> 32;
        c[a] = (float)(h >> 40) * (2.0f / 16777216.0f) - 1.0f;
    }
    p[i] = make_float3(c[0], c[1], c[2]);
}

// Autotuner: time every tile shape on a calibration list of 4 tiles per SM
// (three runs each, CUDA events on the stream, best of three) and keep the
// fastest.  Runs once per process and device; the choice never changes a
// result, only the time.
static int g_fp32_pick[64];
static float g_fp32_ms[64][kFp32Variants];
static bool g_fp32_init = false;

static std::mutex g_fp32_mu;   // request-loop slots prepare their networks on their own threads

static odc_status fp32_autotune(MlpState* st, cudaStream_t s, std::string* err) {
    int dev = 0;
    MLP_CK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_fp32_mu);
    if (!g_fp32_init) {
        for (int& v : g_fp32_pick) v = -1;
        g_fp32_init = true;
    }
    if (dev < 0 || dev >= 64) return ODC_OK;
    if (g_fp32_pick[dev] >= 0) {
        st->fp32_variant = g_fp32_pick[dev];
        return ODC_OK;
    }
    const int64_t n = (int64_t)4 * std::max(st->sms, 1) * 128;
    float3* pts = nullptr;
    float* z = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    MLP_CK(cudaMallocAsync((void**)&pts, n * sizeof(float3), s));
    MLP_CK(cudaMallocAsync((void**)&z, n * sizeof(float), s));
    MLP_CK(cudaEventCreate(&e0));
    MLP_CK(cudaEventCreate(&e1));
    k_calib_points<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(pts, n);
    note_launch();
    QuerySrc Q{pts, nullptr, GridDev{}, nullptr};
    int best = 0;
    float best_ms = 0.0f;
    for (int v = 0; v < kFp32Variants; ++v) {
        float vbest = 0.0f;
        for (int rep = 0; rep < 4; ++rep) {   // the first run warms up
            MLP_CK(cudaEventRecord(e0, s));
            launch_fp32_variant(v, st, Q, n, z, s);
            MLP_CK(cudaEventRecord(e1, s));
            MLP_CK(cudaEventSynchronize(e1));
            float ms = 0.0f;
            MLP_CK(cudaEventElapsedTime(&ms, e0, e1));
            if (rep > 0 && (rep == 1 || ms < vbest)) vbest = ms;
        }
        g_fp32_ms[dev][v] = vbest;
        if (v == 0 || vbest < best_ms) { best = v; best_ms = vbest; }
    }
    MLP_CK(cudaGetLastError());
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    MLP_CK(cudaFreeAsync(pts, s));
    MLP_CK(cudaFreeAsync(z, s));
    g_fp32_pick[dev] = best;
    st->fp32_variant = best;
    return ODC_OK;
}

int mlp_fp32_variant(const MlpState* st) {
    return !st ? -1 : (st->fp32_forced >= 0 ? st->fp32_forced : st->fp32_variant);
}

float mlp_fp32_variant_ms(int v) {
    int dev = 0;
    cudaGetDevice(&dev);
    return (g_fp32_init && dev >= 0 && dev < 64 && v >= 0 && v < kFp32Variants) ? g_fp32_ms[dev][v] : 0.0f;
}

// n is the query count, or with Q.cnt its upper bound (the count is then
// accumulated on the device for the FLOP accounting).
static odc_status launch_fp32(MlpState* st, const QuerySrc& Q, int64_t n, float* z, cudaStream_t s, std::string* err);

// Half of the split tier's calibration list: points on the shell 0.3 <=
// |x| <= 0.7 where the envelope networks' surfaces lie (hashed directions
// from a cube, rejected outside the unit ball, and radii).
__global__ void k_shell_points(float3* p, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t h = (uint64_t)(i + 0x5D1) * 0xD1B54A32D192ED03ull + 0x8CB92BA72F3D8DD7ull;
    auto next = [&]() {
        h ^= h >> 29;
        h *= 0xBF58476D1CE4E5B9ull;
        h ^= h >> 32;
        return (float)(h >> 40) * (1.0f / 16777216.0f);
    };
    float d[3], q = 0.0f;
    for (int t = 0; t < 16; ++t) {
        for (int a = 0; a < 3; ++a) d[a] = 2.0f * next() - 1.0f;
        q = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        if (q > 1e-4f && q <= 1.0f) break;
    }
    if (!(q > 1e-4f)) { d[0] = 1.0f; d[1] = d[2] = 0.0f; q = 1.0f; }
    const float r = (0.3f + 0.4f * next()) * rsqrtf(q);
    p[i] = make_float3(d[0] * r, d[1] * r, d[2] * r);
}

// Calibration of the split tier for the uploaded weights, on 65536 points
// (half hashed over the box, half on the surface shell).
//  * Accumulation compensation c (unless the source fixes it): the split
//    tier's logit error against the FP32 network is close to beta f (f the
//    network output, recovered from the FP32 logit), with beta linear in c;
//    beta is fitted by least squares at c = 0 and at c = kSplitCompProbe, and
//    c is set where the line crosses zero (kept within [0, 1e-6]).
//  * Margin: kSplitMarginFactor times the largest |split - FP32| logit
//    difference on the list at that c, and at least kSplitMarginFloor; on
//    eight networks of this shape the largest difference over 3 M points was
//    1.0 to 1.4 times the list's, so the margin is about twice the
//    large-sample error of each network.
// Rows the split tier hands on (out of FP16 range) and differences beyond
// 1e-3 are left out.
constexpr float kSplitMarginFactor = 2.5f;
constexpr float kSplitMarginFloor = 1.2e-5f;
static odc_status split_calibrate(MlpState* st, cudaStream_t s, std::string* err) {
    const int64_t n = 65536;
    float3* pts = nullptr;
    float* z = nullptr;
    MLP_CK(cudaMallocAsync((void**)&pts, n * sizeof(float3), s));
    MLP_CK(cudaMallocAsync((void**)&z, 3 * n * sizeof(float), s));
    k_calib_points<<<(unsigned)((n / 2 + 255) / 256), 256, 0, s>>>(pts, n / 2);
    note_launch();
    k_shell_points<<<(unsigned)((n / 2 + 255) / 256), 256, 0, s>>>(pts + n / 2, n / 2);
    note_launch();
    const QuerySrc Q{pts, nullptr, GridDev{}, nullptr};
    const bool fit = st->split_comp == 0.0f;
    odc_status r = launch_fp32(st, Q, n, z, s, err);
    if (fit) {
        if (r == ODC_OK) r = mlp_tc_set_comp(st, 0.0f, s, err);
        if (r == ODC_OK) r = mlp_tc3_eval(st, Q, n, z + n, s, err);
        if (r == ODC_OK) r = mlp_tc_set_comp(st, kSplitCompProbe, s, err);
        if (r == ODC_OK) r = mlp_tc3_eval(st, Q, n, z + 2 * n, s, err);
    }
    std::vector<float> hz((size_t)3 * n);
    std::vector<float3> hp((size_t)n);
    auto fetch = [&](size_t count) {
        if (r == ODC_OK &&
            (cudaMemcpyAsync(hz.data(), z, count * sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
             cudaMemcpyAsync(hp.data(), pts, hp.size() * sizeof(float3), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
             cudaStreamSynchronize(s) != cudaSuccess)) {
            *err = "split calibration: copy failed";
            r = ODC_ERR_CUDA;
        }
        if (r == ODC_OK) r = mlp_tc_check(st, s, err);
    };
    auto usable = [&](double z32, double d) { return std::isfinite(z32) && std::isfinite(d) && std::fabs(d) <= 1e-3; };
    double c = std::max(st->split_comp, 0.0f);
    if (fit) {
        fetch(hz.size());
        double sff = 0.0, sf0 = 0.0, sf1 = 0.0;
        for (int64_t i = 0; r == ODC_OK && i < n && st->amp != 0.0f && st->scale != 0.0f; ++i) {
            const double z32 = hz[i], d0 = (double)hz[n + i] - z32, d1 = (double)hz[2 * n + i] - z32;
            if (!usable(z32, d0) || !usable(z32, d1)) continue;
            const double x = hp[i].x, y = hp[i].y, w = hp[i].z;
            const double f = (z32 / st->scale - st->radius + std::sqrt(x * x + y * y + w * w)) / st->amp;
            sff += f * f;
            sf0 += d0 * f;
            sf1 += d1 * f;
        }
        c = 0.0;
        if (sff > 0.0 && sf1 != sf0) c = -sf0 * (double)kSplitCompProbe / (sf1 - sf0);
        c = std::min(std::max(c, 0.0), 1e-6);
    }
    // the margin, from the split tier at the compensation it keeps
    if (r == ODC_OK) r = mlp_tc_set_comp(st, (float)c, s, err);
    if (r == ODC_OK) r = mlp_tc3_eval(st, Q, n, z + n, s, err);
    fetch((size_t)2 * n);
    cudaFreeAsync(pts, s);
    cudaFreeAsync(z, s);
    if (r != ODC_OK) return r;
    double emax = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        const double z32 = hz[i], d = (double)hz[n + i] - z32;
        if (usable(z32, d)) emax = std::max(emax, std::fabs(d));
    }
    st->split_comp_used = (float)c;
    st->zsplit_cal = std::max(kSplitMarginFloor, (float)(kSplitMarginFactor * emax));
    return ODC_OK;
}

void mlp_split_settings(const MlpState* st, float* zmargin, float* comp) {
    *zmargin = st ? st->zsplit : 0.0f;
    *comp = st ? std::max(st->split_comp_used, 0.0f) : 0.0f;
}

static odc_status launch_fp32(MlpState* st, const QuerySrc& Q, int64_t n, float* z, cudaStream_t s, std::string* err) {
    if (n <= 0) return ODC_OK;
    const int v = st->fp32_forced >= 0 ? st->fp32_forced : std::max(st->fp32_variant, 0);
    cudaEvent_t* ev = mlp_ev_pair(st, 0);
    if (ev) MLP_CK(cudaEventRecord(ev[0], s));
    launch_fp32_variant(v, st, Q, n, z, s);
    if (ev) MLP_CK(cudaEventRecord(ev[1], s));
    MLP_CK(cudaGetLastError());
    if (!Q.cnt) {
        int64_t real = n;
        if (!Q.pts) real = (int64_t)Q.g.nv[0] * Q.g.nv[1] * Q.g.nv[2];   // grid mode: padding lanes excluded
        st->flops[0] += kFlopsPerQuery * (double)real;
    }
    st->launches[0] += 1;
    return ODC_OK;
}

// ------------------------------------------------------------ band re-eval
// Tiers: 0 BF16 pass, 1 FP16 tier, 2 split-FP16 tier, 3 FP32.  A query's
// first tier comes from hint[i], an estimate of |z_i - zt| (from the logits
// around the query in its search); no hint routes to the BF16 pass.
// With an FP8 pass, tier 4 comes first: queries predicted at |z - zt| >= z8
// (and every query without a hint) start there.
struct RouteArgs {
    const float* hint;
    float zs, zh, zb;
    int split, h16;
    float z8;
    int fp8;
    int first;   // the FP8 / BF16 passes take queries (0: every query starts at a later tier)
};
__device__ __forceinline__ int route_of(const RouteArgs& ra, int64_t i) {
    const float h = ra.hint ? ra.hint[i] : INFINITY;
    if (ra.first) {
        if (ra.fp8 && h >= ra.z8) return 4;
        if (h >= ra.zb) return 0;
    }
    if (h < ra.zs) return 3;
    if (h < ra.zh) return ra.split ? 2 : 3;
    return ra.h16 ? 1 : (ra.split ? 2 : 3);
}
__global__ void k_route(RouteArgs ra, int64_t n, uint8_t* __restrict__ r) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    r[i] = (uint8_t)route_of(ra, i);
}
// Queries of tier `from` whose logit lies within thr of t move to tier `to`
// (from < 0: every query takes its tier from the hints first); the queries
// now in tier `to` are appended to list (one atomic per block of
// kTierItems x kTierBlock queries: the list order varies between runs, the
// logits written back through it do not) and counted in *cnt and *total.
// Launched with kTierBlock threads.
constexpr int kTierBlock = 256;
constexpr int kTierItems = 4;              // queries per thread
__global__ void __launch_bounds__(kTierBlock)
    k_tier_list(const float* __restrict__ z, int64_t n, const unsigned long long* __restrict__ nlim, float t, int from,
                int to, float thr, RouteArgs ra, uint8_t* __restrict__ r, int* __restrict__ list,
                unsigned long long* __restrict__ cnt, unsigned long long* __restrict__ total) {
    constexpr int kWarps = kTierBlock / 32;
    __shared__ unsigned wbase[kTierItems][kWarps];
    __shared__ unsigned long long bbase;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (nlim) n = min(n, (int64_t)*nlim);   // device-sized query list
    const int64_t i0 = (int64_t)blockIdx.x * (kTierItems * kTierBlock) + threadIdx.x;
    uint32_t bal[kTierItems];
    bool fl[kTierItems];
#pragma unroll
    for (int it = 0; it < kTierItems; ++it) {
        const int64_t i = i0 + it * kTierBlock;
        bool f = false;
        if (i < n) {
            int ri;
            if (from < 0) {
                ri = route_of(ra, i);
                r[i] = (uint8_t)ri;
            } else {
                ri = r[i];
                if (ri == from && fabsf(z[i] - t) < thr) {
                    ri = to;
                    r[i] = (uint8_t)to;
                }
            }
            f = ri == to;
        }
        fl[it] = f;
        bal[it] = __ballot_sync(0xffffffffu, f);
        if (lane == 0) wbase[it][warp] = (unsigned)__popc(bal[it]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned tot = 0;
#pragma unroll
        for (int it = 0; it < kTierItems; ++it)
#pragma unroll
            for (int w = 0; w < kWarps; ++w) {
                const unsigned c = wbase[it][w];
                wbase[it][w] = tot;
                tot += c;
            }
        bbase = tot ? atomicAdd(cnt, (unsigned long long)tot) : 0ull;
        if (tot) atomicAdd(total, (unsigned long long)tot);
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kTierItems; ++it)
        if (fl[it])
            list[bbase + wbase[it][warp] + __popc(bal[it] & ((1u << lane) - 1u))] = (int)(i0 + it * kTierBlock);
}

// Tiered evaluation (A.2.2 binary decision at iso): the sign of every logit
// equals the FP32 plain path's.  A logit of the BF16 pass is kept only
// outside the band |z - zt| >= zband; the single-product FP16 tier (measured
// error 0.0091, below zh16 / 2) re-takes the band and keeps |z - zt| >= zh16; the
// split-FP16 tensor-core network (its accumulation bias compensated; zsplit
// calibrated per network at about twice its largest error) re-takes
// the rest and keeps |z - zt| >= zsplit; the FP32 SIMT network takes what is
// left.  A disabled tier passes its queries on with its predecessor's
// margin.  With hints, a query starts at the tier its predicted |z - zt|
// points to; the acceptance rules are unchanged, so only the cost depends on
// the hints.  Each tier's list is built and consumed on the device (its size
// stays there), so the evaluation needs no host round trip.
static odc_status eval_tiered(MlpState* st, const QuerySrc& Q, int64_t n, float* z, const float* hint, cudaStream_t s,
                              std::string* err, const unsigned long long* nlim = nullptr) {
    odc_status r;
    void *pr, *plist;
    if ((r = mlp_scratch(st, 24, (size_t)n + 64, &pr, err)) != ODC_OK) return r;
    // one list buffer for every tier: a tier's list is consumed (stream order)
    // before the next tier's list is built into the same buffer
    if ((r = mlp_scratch(st, 25, (size_t)n * 4 + 64, &plist, err)) != ODC_OK) return r;
    if (Q.idx) { *err = "nested query index"; return ODC_ERR_INTERNAL; }
    int* list = (int*)plist;
    uint8_t* route = (uint8_t*)pr;
    unsigned long long* cnt = st->dq + 4;
    const unsigned blocks = (unsigned)((n + kTierItems * kTierBlock - 1) / (kTierItems * kTierBlock));
    MLP_CK(cudaMemsetAsync(cnt, 0, 6 * sizeof(unsigned long long), s));   // tier lists 0..3, FP8 total and list
    // small surfaces: the search queries skip the FP8 / BF16 passes (their
    // launches would cost more than they save, mlp_size_tiers)
    const bool first_on = !hint || st->first_run;
    const RouteArgs ra{hint, st->zsplit, st->zh16, st->zband, st->split, st->h16_run, st->zb8, st->fp8,
                       first_on ? 1 : 0};
    // per tier: queries evaluated since the timing began
    unsigned long long* tot[4] = {st->dq + 0, st->dq + 3, st->dq + 1, st->dq + 2};
    unsigned long long* tot8 = st->dq + 10;
    unsigned long long* cnt8 = st->dq + 9;
    const int first = st->fp8 ? 4 : 0;
    // without the first passes the routing pass builds the first active
    // tier's list directly
    const int start = first_on ? first : (st->h16_run ? 1 : (st->split ? 2 : 3));
    if (!hint && !nlim) {
        k_route<<<(unsigned)((n + kTierBlock - 1) / kTierBlock), kTierBlock, 0, s>>>(ra, n, route); note_launch();
        if ((r = first == 4 ? mlp_tc8_eval(st, Q, n, z, s, err) : mlp_tc_eval(st, Q, n, z, s, err)) != ODC_OK)
            return r;
    } else {
        // routing and the first pass's list in one pass (no hint: every query
        // starts at the first pass)
        k_tier_list<<<blocks, kTierBlock, 0, s>>>(z, n, nlim, st->zt, -1, start, 0.0f, ra, route, list,
                                                  start == 4 ? cnt8 : cnt + start, start == 4 ? tot8 : tot[start]);
        note_launch();
        QuerySrc L0{Q.pts, list, Q.g, first == 4 ? cnt8 : cnt + 0, Q.seg, Q.b0tab};
        if (first_on &&
            (r = first == 4 ? mlp_tc8_eval(st, L0, n, z, s, err) : mlp_tc_eval(st, L0, n, z, s, err)) != ODC_OK)
            return r;
    }
    if (first == 4 && first_on) {
        // the BF16 pass re-takes the FP8 band and the queries routed to it
        k_tier_list<<<blocks, kTierBlock, 0, s>>>(z, n, nlim, st->zt, 4, 0, st->zb8, ra, route, list, cnt + 0,
                                                  tot[0]); note_launch();
        QuerySrc L0{Q.pts, list, Q.g, cnt + 0, Q.seg, Q.b0tab};
        if ((r = mlp_tc_eval(st, L0, n, z, s, err)) != ODC_OK) return r;
    }
    int from = 0;
    float thr = st->zband;
    for (int tier = 1; tier <= 3; ++tier) {
        const bool on = tier == 1 ? st->h16_run != 0 : tier == 2 ? st->split != 0 : true;
        if (!on) continue;
        if (tier != start) {   // else the routing pass built this list
            k_tier_list<<<blocks, kTierBlock, 0, s>>>(z, n, nlim, st->zt, from, tier, thr, ra, route, list,
                                                      cnt + tier, tot[tier]);
            note_launch();
        }
        QuerySrc L{Q.pts, list, Q.g, cnt + tier, Q.seg, Q.b0tab};
        r = tier == 1 ? mlp_tc16_eval(st, L, n, z, s, err)
            : tier == 2 ? mlp_tc3_eval(st, L, n, z, s, err)
                        : launch_fp32(st, L, n, z, s, err);
        if (r != ODC_OK) return r;
        from = tier;
        thr = tier == 1 ? st->zh16 : st->zsplit;
    }
    MLP_CK(cudaGetLastError());
    return ODC_OK;
}

static odc_status eval(MlpState* st, const QuerySrc& Q, int64_t n, float* z, int precision, const float* hint,
                       cudaStream_t s, std::string* err) {
    if (precision < 0) precision = st->precision;
    if (precision == ODC_PREC_FP32) return launch_fp32(st, Q, n, z, s, err);
    if (precision == ODC_PREC_SPLIT) return mlp_tc3_eval(st, Q, n, z, s, err);
    if (precision == ODC_PREC_F16) return mlp_tc16_eval(st, Q, n, z, s, err);
    if (precision == ODC_PREC_FP8_RAW) return mlp_tc8_eval(st, Q, n, z, s, err);
    return eval_tiered(st, Q, n, z, hint, s, err);
}

odc_status mlp_eval_list(MlpState* st, const float3* pts, int64_t n, float* z, int precision, cudaStream_t s,
                         std::string* err, const float* hint) {
    QuerySrc Q{pts, nullptr, GridDev{}, nullptr};
    st->stream = s;
    if (precision < 0 && batch_active(st)) return batch_eval(st, pts, n, nullptr, z, hint, s, err);
    return eval(st, Q, n, z, precision, hint, s, err);
}

// FP32 queries of a device-sized list, counted for the statistics
__global__ void k_count_add(const unsigned long long* __restrict__ n, int64_t n_max, unsigned long long* total) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *total += min((unsigned long long)n_max, *n);
}

odc_status mlp_eval_list_dev(MlpState* st, const float3* pts, int64_t n_max, const unsigned long long* n_dev, float* z,
                             cudaStream_t s, std::string* err, const float* hint) {
    QuerySrc Q{pts, nullptr, GridDev{}, nullptr};
    st->stream = s;
    if (n_max <= 0) return ODC_OK;
    if (batch_active(st)) return batch_eval(st, pts, n_max, n_dev, z, hint, s, err);
    if (st->precision != ODC_PREC_BF16) {
        QuerySrc L{pts, nullptr, GridDev{}, n_dev};
        odc_status r = launch_fp32(st, L, n_max, z, s, err);
        if (r != ODC_OK) return r;
        k_count_add<<<1, 32, 0, s>>>(n_dev, n_max, st->dq + 2); note_launch();
        return ODC_OK;
    }
    return eval_tiered(st, Q, n_max, z, hint, s, err, n_dev);
}

odc_status mlp_eval_merged(MlpState* st, const float3* pts, const float* hint, const uint16_t* seg,
                           const float* b0tab, int64_t n_max, const unsigned long long* n_dev, float* z,
                           cudaStream_t s, std::string* err) {
    st->stream = s;
    if (n_max <= 0) return ODC_OK;
    if (st->precision != ODC_PREC_BF16) {
        QuerySrc L{pts, nullptr, GridDev{}, n_dev, seg, b0tab};
        odc_status r = launch_fp32(st, L, n_max, z, s, err);
        if (r != ODC_OK) return r;
        k_count_add<<<1, 32, 0, s>>>(n_dev, n_max, st->dq + 2); note_launch();
        return ODC_OK;
    }
    QuerySrc Q{pts, nullptr, GridDev{}, nullptr, seg, b0tab};
    return eval_tiered(st, Q, n_max, z, hint, s, err, n_dev);
}

odc_status mlp_eval_grid(MlpState* st, const GridDev& g, float* z, cudaStream_t s, std::string* err) {
    QuerySrc Q{nullptr, nullptr, g, nullptr};
    int64_t n = (int64_t)g.W * g.nv[1] * g.nv[2] * 32;
    return eval(st, Q, n, z, -1, nullptr, s, err);
}

__global__ void k_pts_labels(const float* __restrict__ z, int64_t n, float t, uint8_t* __restrict__ lab) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) lab[i] = z[i] > t ? 1 : 0;
}

odc_status mlp_points(MlpState* st, const float3* pts, int64_t n, float iso, int precision, uint8_t* labels,
                      float* logits, cudaStream_t s, std::string* err) {
    st->zt = mlp_logit_threshold(iso);
    st->stream = s;
    odc_status r = mlp_eval_list(st, pts, n, logits, precision, s, err);
    if (r != ODC_OK) return r;
    k_pts_labels<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(logits, n, mlp_logit_threshold(iso), labels); note_launch();
    MLP_CK(cudaGetLastError());
    return mlp_tc_check(st, s, err);
}

}  // namespace odc
