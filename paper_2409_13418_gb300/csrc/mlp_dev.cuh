// mlp_dev.cuh -- device layout and shared helpers of the MLP occupancy path.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/odc.h"
#include "odc_device.cuh"

namespace odc {

constexpr int kNF = 64;    // Fourier frequencies
constexpr int kH = 256;    // hidden width
constexpr int kNL = 4;     // hidden layers
constexpr int kScratchSlots = 40;
// Split tier: the tensor core rounds each MMA's accumulated sum toward zero,
// so a layer sum of K products comes out short by about c K / 256 of its
// size (c from 1e-7 to 3e-7 on the networks measured); its weights are
// prepared as w (1 + c K / 256), which puts that back at no cost per query.  A ReLU network whose layer sums all shrink by
// the same fraction shrinks its output f by a fixed fraction, so the logit
// error is close to proportional to f: mlp_split_calibrate fits that slope
// at c = 0 and at c = kSplitCompProbe on a calibration list and takes the c
// where it vanishes, per network, at weight upload.
constexpr float kSplitCompProbe = 2e-7f;

// FP32 weight blob (floats): B [64][3] (padded to 256), W_l^T [in][out] for
// l = 0..3, w4 [256], biases b_0..b_3 [256], b_4 [1].
struct BlobLayout {
    static constexpr size_t B = 0;
    static constexpr size_t W0 = 256;
    static constexpr size_t W1 = W0 + 2 * kNF * kH;
    static constexpr size_t W2 = W1 + kH * kH;
    static constexpr size_t W3 = W2 + kH * kH;
    static constexpr size_t W4 = W3 + kH * kH;
    static constexpr size_t b0 = W4 + kH;
    static constexpr size_t b1 = b0 + kH;
    static constexpr size_t b2 = b1 + kH;
    static constexpr size_t b3 = b2 + kH;
    static constexpr size_t b4 = b3 + kH;
    static constexpr size_t total = b4 + 64;
};
#define kOffB (BlobLayout::B)
#define kBlobFloats (BlobLayout::total)
__host__ __device__ constexpr size_t kOffW_(int l) {
    return l == 0 ? BlobLayout::W0 : l == 1 ? BlobLayout::W1 : l == 2 ? BlobLayout::W2 : l == 3 ? BlobLayout::W3 : BlobLayout::W4;
}
__host__ __device__ constexpr size_t kOffb_(int l) {
    return l == 0 ? BlobLayout::b0 : l == 1 ? BlobLayout::b1 : l == 2 ? BlobLayout::b2 : l == 3 ? BlobLayout::b3 : BlobLayout::b4;
}
// array-like accessors kOffW[l], kOffb[l]
struct OffW { __host__ __device__ constexpr size_t operator[](int l) const { return kOffW_(l); } };
struct Offb { __host__ __device__ constexpr size_t operator[](int l) const { return kOffb_(l); } };
constexpr OffW kOffW{};
constexpr Offb kOffb{};

struct MlpTc;   // tensor-core path state (mlp_tc.cu)
struct BatchGroup;   // shared evaluations (batch.cu)
constexpr int kMaxTimedLaunches = 512;

struct MlpState {
    int precision = ODC_PREC_FP32;
    float band = 1e-3f;
    float zband = 0.004f;
    float scale = 20.f, radius = 0.5f, amp = 0.15f;
    float* wblob = nullptr;                 // FP32 weight blob (device)
    std::vector<float> wkey;                // host copy of the uploaded B, W, b (all but the latent)
    void* scr[kScratchSlots] = {};
    size_t scr_cap[kScratchSlots] = {};
    MlpTc* tc = nullptr;
    // per-launch CUDA events around the network kernels of one extract
    cudaEvent_t ev[2 * kMaxTimedLaunches] = {};
    int ev_kind[kMaxTimedLaunches] = {};   // 0: FP32, 1: BF16 pass, 2: split-FP16 tier, 3: FP16 tier, 4: FP8 pass
    int ev_used = 0;
    double flops[5] = {0.0, 0.0, 0.0, 0.0, 0.0};   // FLOPs of the network launches per kind (kind 2: tensor-pipe FLOPs)
    int64_t launches[5] = {0, 0, 0, 0, 0};
    int split = 1;              // use the split-FP16 tier for band re-evaluation
    int h16 = 1;                // use the single-product FP16 tier between the BF16 pass and the split tier
    int h16_run = 1;            // ... in the current extraction (off for small surfaces, mlp_size_tiers)
    int first_run = 1;          // search queries may start at the FP8 / BF16 passes (off for small surfaces)
    int fp8 = 0;                // an FP8 pass ahead of the BF16 pass (source precision ODC_PREC_FP8)
    float zb8 = 2.5f;           // |z - zt| below which an FP8-pass decision is re-taken by the BF16 pass
                                // (2.1 times the largest FP8 logit error measured, 1.19)
    float zh16 = 0.025f;        // |z - zt| below which an FP16-tier decision is re-taken by the split tier
    int fp32_variant = -1;      // FP32 network tile shape picked by the autotuner (-1: not yet)
    int fp32_forced = -1;       // tile shape forced by the source's flags (-1: the autotuner's)
    float zsplit = 2e-5f;       // |z - zt| below which a split-tier decision is re-taken in FP32
    float split_comp = 0.0f;    // requested split-tier compensation: 0 calibrate, < 0 none, > 0 this c
    float split_comp_used = -1.0f;   // c in effect for the uploaded weights (-1: none set yet)
    float zsplit_user = 0.0f;   // the source's split_zmargin (0: calibrated per network)
    float zsplit_cal = 0.0f;    // the calibrated margin of the uploaded weights (0: none yet)
    float zt = 0.0f;            // decision threshold logit(iso) of the current extract
    const float* zgrid = nullptr;   // grid logits of the current extract (label-word order)
    unsigned long long wait_ns = 0;   // limit of the single-CTA tensor-core kernels' pipeline waits (0: 2 s)
    const int* gate = nullptr;        // device go signal of those kernels (NULL: none)
    // batch group membership (batch.h): search-stage evaluations shared with
    // the group's other members when bcompat
    BatchGroup* group = nullptr;
    bool bcompat = false;
    bool bin_stage = false;           // inside a search stage (counted active by the group)
    int brow = -1;                    // the member's row of the group's first-layer bias table
    std::vector<float> b0host;        // the folded first-layer bias of the source last uploaded
    bool b0dirty = false;             // b0host not yet in the group's table
    cudaEvent_t bev = nullptr;        // the member's queries are ready (recorded per shared call)
    int sms = 0;                // SM count of the device
    cudaStream_t stream = nullptr;   // stream of the current call (scratch growth is ordered on it)
    // device counters: [0..3] queries evaluated from device-sized lists by the
    // BF16, split-FP16, FP32 and FP16 networks since mlp_timing_begin; [4..7]
    // the list sizes of the current evaluation
    // (FP8 pass: its list size in [9], its total in [10])
    unsigned long long* dq = nullptr;
    unsigned long long hq[5] = {0, 0, 0, 0, 0};   // host copy of dq[0..3] and dq[10] (mlp_timing_finish)
};

// Event pair around one network launch of the given kind (none once all are in use).
cudaEvent_t* mlp_ev_pair(MlpState* st, int kind);
constexpr double kFlopsPerQuery = 2.0 * (2.0 * kNF * kH + 3.0 * kH * kH + kH);

// Tensor-core path (mlp_tc.cu)
odc_status mlp_tc_prepare(MlpState* st, const float* host_blob, cudaStream_t s, std::string* err);
struct QuerySrc;
odc_status mlp_tc_eval(MlpState* st, const QuerySrc& Q, int64_t n, float* z, cudaStream_t s, std::string* err);
// Single-product FP16 network (FP16 activations, the split path's hi weights).
odc_status mlp_tc16_eval(MlpState* st, const QuerySrc& Q, int64_t n, float* z, cudaStream_t s, std::string* err);
// FP8 pass (E4M3 activations and weights, FP32 accumulation).
odc_status mlp_tc8_eval(MlpState* st, const QuerySrc& Q, int64_t n, float* z, cudaStream_t s, std::string* err);
void mlp_tc_destroy(MlpState* st);
size_t mlp_tc_device_bytes(const MlpState* st);
// ODC_ERR_TIMEOUT if a tensor-core launch since the last check hit a bounded wait.
odc_status mlp_tc_check(MlpState* st, cudaStream_t s, std::string* err);
// Device error flag of the tensor-core kernels (NULL before their preparation).
int* mlp_tc_err_flag(MlpState* st);
// Split-BF16 network (three BF16 products per layer, FP32 accumulation).
odc_status mlp_tc3_eval(MlpState* st, const QuerySrc& Q, int64_t n, float* z, cudaStream_t s, std::string* err);
// Split tier: prepare its weights for the accumulation compensation c (w (1 + c K / 256)).
odc_status mlp_tc_set_comp(MlpState* st, float c, cudaStream_t s, std::string* err);

// [sin(2 pi u), cos(2 pi u)] with u = b . x formed exactly in float-float and
// reduced to [-1/2, 1/2] turns before sincospi.
__device__ __forceinline__ float2 fourier_sincos(float b0, float b1, float b2, float3 x) {
    ff u = ff_add(ff_add(two_prod(b0, x.x), two_prod(b1, x.y)), two_prod(b2, x.z));
    float k = rintf(u.hi);
    float r = __fadd_rn(__fsub_rn(u.hi, k), u.lo);
    float s, c;
    sincospif(2.0f * r, &s, &c);
    return make_float2(s, c);
}

// The same features for the BF16 pass: the phase in FP32 (error ~1e-6
// turns for |B x| up to ~30), reduced to [-1/2, 1/2] turns, and the SFU
// sin/cos (absolute error ~3e-7 on [-pi, pi]): far below the BF16 rounding
// of the features (~4e-3), at a sixth of the instructions.
__device__ __forceinline__ float2 fourier_sincos_fast(float b0, float b1, float b2, float3 x) {
    float u = fmaf(b0, x.x, fmaf(b1, x.y, b2 * x.z));
    float r = u - rintf(u);
    float s, c;
    __sincosf(6.283185307179586f * r, &s, &c);
    return make_float2(s, c);
}

// z = scale (radius - |x| + amp f)
__device__ __forceinline__ float envelope_logit(float3 x, float f, float scale, float radius, float amp) {
    float r = __fsqrt_rn(x.x * x.x + x.y * x.y + x.z * x.z);
    return scale * ((radius - r) + amp * f);
}

// Query points either from a list or from the grid in label-word order.
// With idx, query q of a launch is query idx[q] of the source and its logit
// goes to z[idx[q]]; with cnt, the launch covers min(n, *cnt) queries (a
// device-side list size, so the host needs no count).
//
// seg and b0tab (optional, both set or both null): query q's first-layer
// bias is row seg[q] of b0tab ([rows][256]) instead of the network's b_0:
// queries of latent-conditioned shapes of one network (the latent folds into
// b_0) share one evaluation.
struct QuerySrc {
    const float3* pts;       // list mode when non-null
    const int* idx;          // optional indices into the source (and the output)
    GridDev g;               // grid mode
    const unsigned long long* cnt;   // optional device-side query count
    const uint16_t* seg;     // optional per-query row of b0tab (indexed like the output)
    const float* b0tab;
};
// first-layer bias row of source query q (seg and b0tab set)
__device__ __forceinline__ const float* query_b0(const QuerySrc& Q, int64_t qsrc) {
    return Q.b0tab + (size_t)Q.seg[qsrc] * 256;
}

__device__ __forceinline__ int64_t query_count(const QuerySrc& Q, int64_t n) {
    return Q.cnt ? min(n, (int64_t)*Q.cnt) : n;
}
__device__ __forceinline__ int64_t query_index(const QuerySrc& Q, int64_t q) { return Q.idx ? Q.idx[q] : q; }

__device__ __forceinline__ float3 query_point(const QuerySrc& Q, int64_t q0) {
    const int64_t q = query_index(Q, q0);
    if (Q.pts) return Q.pts[q];
    int64_t w = q >> 5;
    int l = (int)(q & 31);
    int xw = (int)(w % Q.g.W);
    int64_t row = w / Q.g.W;
    int y = (int)(row % Q.g.nv[1]);
    int z = (int)(row / Q.g.nv[1]);
    int x = min(xw * 32 + l, Q.g.nv[0] - 1);
    return make_float3(Q.g.X[0][x], Q.g.X[1][y], Q.g.X[2][z]);
}

// compact.cu
size_t scan_tmp_elems(size_t n);
template <typename T>
void exclusive_scan(const T* in, T* out, size_t n, T* tmp, T* total, cudaStream_t st);

}  // namespace odc
