// mlp.h -- MLP occupancy (envelope MLP over Fourier features) on the device.
//
// occ(x) = sigmoid(scale (radius - |x| + amp f(x))); decisions are taken on
// the logit z = scale (radius - |x| + amp f(x)) against logit(iso).  The
// searches batch their queries into wavefronts: one network evaluation per
// search step over all active edges or face segments.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/odc.h"
#include "odc_internal.h"

namespace odc {

struct MlpState;

odc_status mlp_check(const odc_mlp* m, std::string* err);
odc_status mlp_prepare(MlpState** st, const odc_mlp* m, cudaStream_t s, std::string* err);
void mlp_destroy(MlpState* st);
// Device bytes held by the network state (weights, operand tiles, scratch).
size_t mlp_device_bytes(const MlpState* st);
// FP32 network tile shape in use (forced, else autotuned; -1 before the
// first upload) and
// the autotuner's time for shape v on this device (ms, 0 if not measured).
int mlp_fp32_variant(const MlpState* st);
float mlp_fp32_variant_ms(int v);

// Device scratch owned by the MLP state (grows on demand, never shrinks).
odc_status mlp_scratch(MlpState* st, int slot, size_t bytes, void** out, std::string* err);

// Logits at n explicit points.  With BF16 precision, every logit within the
// band is re-taken by the split-FP16 and FP32 tiers (counted on the device,
// see mlp_timing_finish).  hint (device, n floats, optional): an estimate of |z - logit(iso)|
// per query that lets predicted band queries skip the BF16 pass; it changes
// the cost, never a decision.
odc_status mlp_eval_list(MlpState* st, const float3* pts, int64_t n, float* z, int precision, cudaStream_t s,
                         std::string* err, const float* hint = nullptr);
// The same over a device-sized list: n_dev (device) queries, at most n_max.
odc_status mlp_eval_list_dev(MlpState* st, const float3* pts, int64_t n_max, const unsigned long long* n_dev, float* z,
                             cudaStream_t s, std::string* err, const float* hint = nullptr);
// Logits at the grid vertices in label-word order (query q -> word q/32, lane q%32).
odc_status mlp_eval_grid(MlpState* st, const GridDev& g, float* z, cudaStream_t s, std::string* err);
int mlp_precision(const MlpState* st);
// Limit of every pipeline wait of the single-CTA tensor-core kernels (the
// BF16 pass and the FP16 tier), in ns of device global time; 0: 2 s.
void mlp_set_wait_limit(MlpState* st, unsigned long long ns, const int* gate);
float mlp_logit_threshold(float iso);

// Grid labels (a1): bit rows as in the CSG path.
odc_status mlp_grid(MlpState* st, const GridDev& g, float iso, uint32_t* bits, cudaStream_t s, int64_t* nq,
                    std::string* err);
// 1D search (a4) in k wavefronts over all crossing edges.
odc_status mlp_bisect(MlpState* st, const GridDev& g, const uint32_t* bits, const uint32_t* edges, uint32_t ne, int k,
                      float iso, uint32_t* T, cudaStream_t s, int64_t* nq, std::string* err);
// 2D search (a5) in wavefronts over all face segments.
odc_status mlp_faces(MlpState* st, const GridDev& g, const uint32_t* bits, const uint32_t* flips, const WordInfo* wi,
                     const uint32_t* ebase, const uint32_t* T, const uint32_t* faces, const uint8_t* slots,
                     uint32_t nf, const SearchParams& sp, float iso, float4* pf, uint8_t* flags, FaceDecisions* dec,
                     cudaStream_t s, int64_t* nq, std::string* err);
// Start / finish the per-extract accounting of network launches: total
// event-timed kernel milliseconds and algorithmic FLOPs.
void mlp_timing_begin(MlpState* st, cudaStream_t s);
// Per-extraction tier choice from the surface size (crossing edges).
void mlp_size_tiers(MlpState* st, int64_t n_edges);
// The split tier's margin and accumulation compensation in use.
void mlp_split_settings(const MlpState* st, float* zmargin, float* comp);
// Reads the device-side query counters (synchronises the stream).
void mlp_timing_finish(MlpState* st, cudaStream_t s);
// Per kind (0: FP32 SIMT network, 1: tensor-core network).
void mlp_timing_collect(MlpState* st, int kind, float* ms, double* flops, int64_t* launches);

// Queries re-taken by the split-FP16 and by the FP32 tier (after mlp_timing_finish).
int64_t mlp_split_count(const MlpState* st);
int64_t mlp_fp32_requery_count(const MlpState* st);
int64_t mlp_h16_count(const MlpState* st);   // FP16-tier re-evaluations since the timing began
int64_t mlp_fp8_count(const MlpState* st);   // FP8-pass evaluations from device-sized lists since the timing began

// One evaluation of a merged query list (shared evaluations, batch.cu):
// n_dev (device) of at most n_max queries at pts with routing hints, query q
// taking row seg[q] of b0tab as its first-layer bias.
odc_status mlp_eval_merged(MlpState* st, const float3* pts, const float* hint, const uint16_t* seg,
                           const float* b0tab, int64_t n_max, const unsigned long long* n_dev, float* z,
                           cudaStream_t s, std::string* err);

// Labels (and logits) at explicit points.
odc_status mlp_points(MlpState* st, const float3* pts, int64_t n, float iso, int precision, uint8_t* labels,
                      float* logits, cudaStream_t s, std::string* err);

}  // namespace odc
