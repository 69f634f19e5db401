// search_mlp.cu -- grid labels, 1D and 2D searches against an MLP occupancy,
// batched into wavefronts: every search step evaluates the network once over
// all active elements (Sec. 5.1 and 5.2 run "for all edges / faces at once";
// the network evaluation is the dense contraction).  A small kernel turns the
// logits of one step into the search-state update and the next step's query
// points; the state (integer bisection brackets, float-float geometry) stays
// on the device between steps.
#include <algorithm>

#include "batch.h"
#include "kernels.h"
#include "mlp.h"
#include "mlp_dev.cuh"
#include "search.cuh"

namespace odc {

#define S_CK(call)                                                                          \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) { *err = std::string(#call) + ": " + cudaGetErrorString(e_); \
                                 return ODC_ERR_CUDA; }                                     \
    } while (0)
#define S_TRY(call)                          \
    do {                                     \
        odc_status r_ = (call);              \
        if (r_ != ODC_OK) return r_;         \
    } while (0)

static inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// ------------------------------------------------------------------- grid
__global__ void k_pack_labels(GridDev g, const float* __restrict__ z, float t, uint32_t* __restrict__ bits) {
    size_t w = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int l = threadIdx.x & 31;
    size_t nw = (size_t)g.W * g.nv[1] * g.nv[2];
    if (w >= nw) return;
    int x = (int)(w % g.W) * 32 + l;
    bool in = x < g.nv[0] && z[w * 32 + l] > t;
    uint32_t word = __ballot_sync(0xffffffffu, in);
    if (l == 0) bits[w] = word;
}

odc_status mlp_grid(MlpState* st, const GridDev& g, float iso, uint32_t* bits, cudaStream_t s, int64_t* nq,
                    std::string* err) {
    size_t nw = (size_t)g.W * g.nv[1] * g.nv[2];
    void* pz;
    st->stream = s;
    S_TRY(mlp_scratch(st, 0, nw * 32 * 4, &pz, err));
    st->zt = mlp_logit_threshold(iso);
    st->zgrid = (const float*)pz;
    S_TRY(mlp_eval_grid(st, g, (float*)pz, s, err));
    k_pack_labels<<<nblk(nw * 32), 256, 0, s>>>(g, (const float*)pz, mlp_logit_threshold(iso), bits); note_launch();
    S_CK(cudaGetLastError());
    (void)nq;
    return mlp_tc_check(st, s, err);
}

// Routing hint for the midpoint of a bracket whose ends have logits za, zc
// (see mlp_eval_list): the best estimate of |z - t| at the midpoint, the
// linear prediction |(za + zc)/2 - t| plus kHintCurv of the bracket's logit
// span for curvature.  The hint only picks the first tier that evaluates a
// query; the tiers' acceptance rules take every decision, so a wrong hint
// costs one more evaluation and never changes a result.  An unbiased
// estimate (no allowance for the error of the ends' logits) routes best:
// on simulated 1D bisection traces of the 256^3 envelope network it cut the
// network cost by 6% against a worst-case bound (tier errors added, a
// quarter of the span), within 3% of routing by each query's final tier.
constexpr float kHintCurv = 0.01f;
__device__ __forceinline__ float bracket_hint(float za, float zc, float t, float zb, float zs) {
    (void)zb;
    (void)zs;
    return fabsf(0.5f * (za + zc) - t) + kHintCurv * fabsf(zc - za);
}

struct HintPar {
    float t, zb, zs;
};

// ------------------------------------------------------------------- 1D
__global__ void k_bis_gen(GridDev g, const uint32_t* __restrict__ edges, uint32_t ne, int s,
                          const uint32_t* __restrict__ lo, float3* __restrict__ pts) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ne) return;
    uint32_t e = edges[i];
    int p[3];
    vid_xyz(g, e / 3u, &p[0], &p[1], &p[2]);
    int a = (int)(e % 3u);
    float w[3] = {g.X[0][p[0]], g.X[1][p[1]], g.X[2][p[2]]};
    uint32_t mid = 2u * lo[i] + 1u;
    float u = (float)mid * __int_as_float((127 - (s + 1)) << 23);
    w[a] = axis_world_ff(g.X[a], p[a], ff_make(u)).hi;
    pts[i] = make_float3(w[0], w[1], w[2]);
}

__device__ __forceinline__ size_t grid_query(const GridDev& g, int x, int y, int z) {
    return (((size_t)z * g.nv[1] + y) * g.W + (x >> 5)) * 32 + (x & 31);
}

// Logits at both ends of every crossing edge (from the grid pass) and the
// routing hint of the first midpoint.
__global__ void k_bis_init(GridDev g, const uint32_t* __restrict__ edges, uint32_t ne, const float* __restrict__ zg,
                           HintPar hp, float2* __restrict__ zac, float* __restrict__ hint) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ne) return;
    uint32_t e = edges[i];
    int p[3];
    vid_xyz(g, e / 3u, &p[0], &p[1], &p[2]);
    float za = zg[grid_query(g, p[0], p[1], p[2])];
    p[e % 3u] += 1;
    float zc = zg[grid_query(g, p[0], p[1], p[2])];
    zac[i] = make_float2(za, zc);
    hint[i] = bracket_hint(za, zc, hp.t, hp.zb, hp.zs);
}

__global__ void k_bis_upd(GridDev g, const uint32_t* __restrict__ bits, const uint32_t* __restrict__ edges,
                          uint32_t ne, const float* __restrict__ z, float t, uint32_t* __restrict__ lo, int last,
                          uint32_t* __restrict__ T, HintPar hp, float2* __restrict__ zac, float* __restrict__ hint) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ne) return;
    uint32_t e = edges[i];
    int p[3];
    vid_xyz(g, e / 3u, &p[0], &p[1], &p[2]);
    uint32_t lab0 = label_at(g, bits, p[0], p[1], p[2]);
    float zm = z[i];
    uint32_t lab = zm > t;
    uint32_t l = lo[i], mid = 2u * l + 1u;
    l = (lab == lab0) ? mid : 2u * l;
    lo[i] = l;
    if (last) T[i] = 2u * l + 1u;
    if (hint) {
        float2 b = zac[i];
        if (lab == lab0) b.x = zm; else b.y = zm;
        zac[i] = b;
        hint[i] = bracket_hint(b.x, b.y, hp.t, hp.zb, hp.zs);
    }
}

static odc_status bisect_body(MlpState* st, const GridDev& g, const uint32_t* bits, const uint32_t* edges, uint32_t ne,
                              int k, float iso, uint32_t* T, cudaStream_t s, int64_t* nq, std::string* err) {
    if (!ne) return ODC_OK;
    st->stream = s;
    void *plo, *ppts, *pz;
    S_TRY(mlp_scratch(st, 1, ne * 4ull, &plo, err));
    S_TRY(mlp_scratch(st, 2, ne * 12ull, &ppts, err));
    S_TRY(mlp_scratch(st, 3, ne * 4ull, &pz, err));
    S_CK(cudaMemsetAsync(plo, 0, ne * 4ull, s));
    float t = mlp_logit_threshold(iso);
    st->zt = t;
    HintPar hp{t, st->zband, st->zsplit};
    float2* zac = nullptr;
    float* hint = nullptr;
    if (mlp_precision(st) == ODC_PREC_BF16 && st->zgrid) {
        void *pzac, *ph;
        S_TRY(mlp_scratch(st, 34, ne * 8ull, &pzac, err));
        S_TRY(mlp_scratch(st, 35, ne * 4ull, &ph, err));
        zac = (float2*)pzac;
        hint = (float*)ph;
        k_bis_init<<<nblk(ne), 256, 0, s>>>(g, edges, ne, st->zgrid, hp, zac, hint); note_launch();
    }
    for (int step = 0; step < k; ++step) {
        k_bis_gen<<<nblk(ne), 256, 0, s>>>(g, edges, ne, step, (const uint32_t*)plo, (float3*)ppts); note_launch();
        S_TRY(mlp_eval_list(st, (const float3*)ppts, ne, (float*)pz, -1, s, err, hint));
        k_bis_upd<<<nblk(ne), 256, 0, s>>>(g, bits, edges, ne, (const float*)pz, t, (uint32_t*)plo, step == k - 1, T,
                                           hp, zac, hint); note_launch();
        S_CK(cudaGetLastError());
    }
    *nq += (int64_t)ne * k;
    return mlp_tc_check(st, s, err);
}

// ------------------------------------------------------------------- 2D
struct FaceSt {
    FaceSeg F;
    ff2 d;        // step-1 ray (oriented by the label of m)
    ff2 q;        // step-1 result
    uint32_t lab_m, Ja, Jc, J1a, J1c, J2a, J2c, found;
    float zm;               // logit at m
    float za, zc;           // logits at the step-1 bracket ends (Ja, Jc)
    float z1a, z1c, z2a, z2c;   // logits at the step-2 bracket ends of both rays
};

// Routing hint of the midpoint queries m: a chord midpoint lies close to the
// isocurve through its two 1D points, so |z(m)| falls in the BF16 band for
// nine in ten faces of the 256^3 envelope network (measured on oracle
// traces); they start at the FP16 tier.
constexpr float kHintM = 0.06f;

__global__ void k_face_init(GridDev g, const uint32_t* __restrict__ bits, const uint32_t* __restrict__ flips,
                            const WordInfo* __restrict__ wi, const uint32_t* __restrict__ ebase,
                            const uint32_t* __restrict__ T, const uint32_t* __restrict__ faces,
                            const uint8_t* __restrict__ slots, uint32_t nf, int k, FaceSt* __restrict__ S,
                            float3* __restrict__ pts, float* __restrict__ hint) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    FaceSt st;
    load_face(g, bits, flips, wi, ebase, T, k, faces[i], slots[i], st.F);
    S[i] = st;
    pts[i] = face_world2(g, st.F, st.F.m);
    if (hint) hint[i] = kHintM;
}

// Append val to list with one atomic per block; every thread of the block
// calls it (a block-wide barrier).
template <int BLOCK>
__device__ __forceinline__ void block_append(bool f, uint32_t val, uint32_t* __restrict__ list,
                                             unsigned long long* __restrict__ cnt) {
    __shared__ unsigned wbase[BLOCK / 32];
    __shared__ unsigned long long bbase;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t b = __ballot_sync(0xffffffffu, f);
    if (lane == 0) wbase[warp] = (unsigned)__popc(b);
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned tot = 0;
        for (int w = 0; w < BLOCK / 32; ++w) {
            const unsigned c = wbase[w];
            wbase[w] = tot;
            tot += c;
        }
        bbase = tot ? atomicAdd(cnt, (unsigned long long)tot) : 0ull;
    }
    __syncthreads();
    if (f) list[bbase + wbase[warp] + __popc(b & ((1u << lane) - 1u))] = val;
}

__device__ __forceinline__ uint32_t n_of(const unsigned long long* cnt, uint32_t n) {
    return cnt ? (uint32_t)min((unsigned long long)n, *cnt) : n;
}
constexpr int kLinBlock = 128;
constexpr int kMaxLin = 65;   // line samples per search: at most 64 (odc_params)

// label of m -> step-1 ray.  zc holds the logit of the last line sample
// taken (m's before the first).
__global__ void k_face_m(uint32_t nf, const float* __restrict__ z, float t, FaceSt* __restrict__ S) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    FaceSt& st = S[i];
    uint32_t lab_m = z[i] > t;
    st.lab_m = lab_m;
    st.zm = z[i];
    st.zc = z[i];
    st.found = 0;
    st.d = lab_m ? ff2{ff_neg(st.F.d.u), ff_neg(st.F.d.v)} : st.F.d;
}

// Step-1 line samples one at a time (A.1.3: the first sample whose label
// differs from m's): round j queries sample j of the faces whose samples
// 1 .. j-1 kept m's label (list/cnt; every face for j = 1).  The hint of
// sample j > 1 is the previous sample's |z - t|.
__global__ void k_lin1_gen(GridDev g, uint32_t nf, int j, const uint32_t* __restrict__ list,
                           const unsigned long long* __restrict__ cnt, SearchParams sp, const FaceSt* __restrict__ S,
                           float3* __restrict__ lp, float* __restrict__ lh, float t) {
    uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_of(cnt, nf)) return;
    const FaceSt& st = S[list ? list[k] : k];
    lp[k] = face_world2(g, st.F, ray_point(st.F.m, st.d, lbs_param(sp.range1, (uint32_t)j << sp.bin1, sp.lin1, sp.bin1)));
    if (lh) lh[k] = j == 1 ? INFINITY : fabsf(st.zc - t);
}

// A sample whose label differs from m's (or the last one) closes the bracket
// [J - 1, J] and queues the first bisection query; the others search on.
__global__ void __launch_bounds__(kLinBlock)
    k_lin1_step(GridDev g, uint32_t nf, int j, const uint32_t* __restrict__ list,
                const unsigned long long* __restrict__ cnt, const float* __restrict__ lz, float t, SearchParams sp,
                FaceSt* __restrict__ S, float3* __restrict__ pts, HintPar hp, float* __restrict__ hint,
                uint32_t* __restrict__ list_out, unsigned long long* __restrict__ cnt_out) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    bool more = false;
    uint32_t i = 0;
    if (k < n_of(cnt, nf)) {
        i = list ? list[k] : k;
        FaceSt& st = S[i];
        const float zj = lz[k];
        const bool hit = (uint32_t)(zj > t) != st.lab_m;
        if (hit || j == sp.lin1) {
            if (hit) st.found = 1;
            st.Ja = (uint32_t)(j - 1) << sp.bin1;
            st.Jc = (uint32_t)j << sp.bin1;
            st.za = st.zc;
            st.zc = zj;
            if (sp.bin1 > 0) {
                pts[i] = face_world2(g, st.F, ray_point(st.F.m, st.d, lbs_param(sp.range1, (st.Ja + st.Jc) >> 1, sp.lin1, sp.bin1)));
                if (hint) hint[i] = bracket_hint(st.za, st.zc, hp.t, hp.zb, hp.zs);
            }
        } else {
            st.zc = zj;
            more = true;
        }
    }
    if (list_out) block_append<kLinBlock>(more, i, list_out, cnt_out);
}

__global__ void k_face_bin1(GridDev g, uint32_t nf, const float* __restrict__ z, float t, SearchParams sp, int step,
                            FaceSt* __restrict__ S, float3* __restrict__ pts, HintPar hp, float* __restrict__ hint) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    FaceSt& st = S[i];
    uint32_t Jm = (st.Ja + st.Jc) >> 1;
    float zm = z[i];
    if ((uint32_t)(zm > t) == st.lab_m) { st.Ja = Jm; st.za = zm; } else { st.Jc = Jm; st.zc = zm; }
    if (step + 1 < sp.bin1) {
        pts[i] = face_world2(g, st.F, ray_point(st.F.m, st.d, lbs_param(sp.range1, (st.Ja + st.Jc) >> 1, sp.lin1, sp.bin1)));
        if (hint) hint[i] = bracket_hint(st.za, st.zc, hp.t, hp.zb, hp.zs);
    }
}

// end of step 1: q == m gives p_f = m; else keep q and mark the face active
__global__ void k_face_fin1(uint32_t nf, SearchParams sp, FaceSt* __restrict__ S, float4* __restrict__ pf,
                            uint8_t* __restrict__ flags, uint32_t* __restrict__ active, FaceDecisions* __restrict__ dec) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    FaceSt& st = S[i];
    FaceDecisions D;
    D.Jq = st.Ja;
    D.J1 = D.J2 = 0;
    D.lab_m = (uint8_t)st.lab_m;
    D.found = (uint8_t)st.found;
    D.pad0 = D.pad1 = 0;
    dec[i] = D;
    if (st.Ja == 0) {
        pf[i] = ff2_pack(st.F.m);
        flags[i] = 1;
        active[i] = 0;
    } else {
        st.q = ray_point(st.F.m, st.d, lbs_param(sp.range1, st.Ja, sp.lin1, sp.bin1));
        st.z1c = st.z2c = st.za;   // logit of the last step-2 line sample of each ray (q's before the first)
        active[i] = 1;
    }
}

__global__ void k_list(const uint32_t* __restrict__ active, const uint32_t* __restrict__ off, uint32_t nf,
                       uint32_t* __restrict__ list) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nf && active[i]) list[off[i]] = i;
}

__device__ __forceinline__ ff2 ray2(const FaceSt& st, int r) {
    return r == 0 ? st.F.u1 : ff2{ff_neg(st.F.u1.u), ff_neg(st.F.u1.v)};
}

// Step-2 line samples of both rays, one at a time per ray: entry e < 2 na is
// ray r = e / na of active face flist[e % na]; round j queries sample j of
// the rays whose samples 1 .. j-1 kept m's label.  Hint: the ray leaves the
// isocurve through q about linearly, so sample 1's |z - t| is estimated as
// |z(m) - t| scaled by its distance over half the segment, and sample j > 1's
// as the previous sample's scaled by j / (j - 1).
__global__ void k_lin2_gen(GridDev g, const uint32_t* __restrict__ flist, uint32_t na, int j,
                           const uint32_t* __restrict__ list, const unsigned long long* __restrict__ cnt,
                           SearchParams sp, const FaceSt* __restrict__ S, float3* __restrict__ lp,
                           float* __restrict__ lh, float t) {
    uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_of(cnt, 2 * na)) return;
    const uint32_t e = list ? list[k] : k;
    const int r = e >= na;
    const FaceSt& st = S[flist[e - (uint32_t)r * na]];
    lp[k] = face_world2(g, st.F, ray_point(st.q, ray2(st, r), lbs_param(sp.range2, (uint32_t)j << sp.bin2, sp.lin2, sp.bin2)));
    if (lh) {
        if (j == 1) {
            const float half = fmaxf(0.5f * hypotf(st.F.p1.x - st.F.p2.x, st.F.p1.y - st.F.p2.y), 0.05f);
            lh[k] = fabsf(st.zm - t) * (sp.range2 / (float)sp.lin2) / half;
        } else {
            lh[k] = fabsf((r ? st.z2c : st.z1c) - t) * (float)j / (float)(j - 1);
        }
    }
}

__global__ void __launch_bounds__(kLinBlock)
    k_lin2_step(GridDev g, const uint32_t* __restrict__ flist, uint32_t na, int j, const uint32_t* __restrict__ list,
                const unsigned long long* __restrict__ cnt, const float* __restrict__ lz, float t, SearchParams sp,
                FaceSt* __restrict__ S, float3* __restrict__ pts, HintPar hp, float* __restrict__ hint,
                uint32_t* __restrict__ list_out, unsigned long long* __restrict__ cnt_out) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    bool more = false;
    uint32_t e = 0;
    if (k < n_of(cnt, 2 * na)) {
        e = list ? list[k] : k;
        const int r = e >= na;
        const uint32_t li = e - (uint32_t)r * na;
        FaceSt& st = S[flist[li]];   // the two rays of a face write disjoint fields (found: atomically)
        float* zprev = r ? &st.z2c : &st.z1c;
        const float zj = lz[k];
        const bool hit = (uint32_t)(zj > t) != st.lab_m;
        if (hit || j == sp.lin2) {
            if (hit) atomicOr(&st.found, 2u << r);
            const uint32_t Ja = (uint32_t)(j - 1) << sp.bin2, Jc = (uint32_t)j << sp.bin2;
            const float za = *zprev;
            if (r == 0) { st.J1a = Ja; st.J1c = Jc; st.z1a = za; st.z1c = zj; }
            else        { st.J2a = Ja; st.J2c = Jc; st.z2a = za; st.z2c = zj; }
            if (sp.bin2 > 0) {
                pts[(size_t)r * na + li] =
                    face_world2(g, st.F, ray_point(st.q, ray2(st, r), lbs_param(sp.range2, (Ja + Jc) >> 1, sp.lin2, sp.bin2)));
                if (hint) hint[(size_t)r * na + li] = bracket_hint(za, zj, hp.t, hp.zb, hp.zs);
            }
        } else {
            *zprev = zj;
            more = true;
        }
    }
    if (list_out) block_append<kLinBlock>(more, e, list_out, cnt_out);
}

__global__ void k_face_bin2(GridDev g, const uint32_t* __restrict__ list, uint32_t na, const float* __restrict__ z,
                            float t, SearchParams sp, int step, FaceSt* __restrict__ S, float3* __restrict__ pts,
                            HintPar hp, float* __restrict__ hint) {
    uint32_t li = blockIdx.x * blockDim.x + threadIdx.x;
    if (li >= na) return;
    FaceSt& st = S[list[li]];
    uint32_t* Ja[2] = {&st.J1a, &st.J2a};
    uint32_t* Jc[2] = {&st.J1c, &st.J2c};
    float* za[2] = {&st.z1a, &st.z2a};
    float* zc[2] = {&st.z1c, &st.z2c};
    for (int r = 0; r < 2; ++r) {
        uint32_t Jm = (*Ja[r] + *Jc[r]) >> 1;
        float zm = z[(size_t)r * na + li];
        if ((uint32_t)(zm > t) == st.lab_m) { *Ja[r] = Jm; *za[r] = zm; } else { *Jc[r] = Jm; *zc[r] = zm; }
        if (step + 1 < sp.bin2) {
            pts[(size_t)r * na + li] =
                face_world2(g, st.F, ray_point(st.q, ray2(st, r), lbs_param(sp.range2, (*Ja[r] + *Jc[r]) >> 1, sp.lin2, sp.bin2)));
            if (hint) hint[(size_t)r * na + li] = bracket_hint(*za[r], *zc[r], hp.t, hp.zb, hp.zs);
        }
    }
}

__global__ void k_face_fin2(const uint32_t* __restrict__ list, uint32_t na, SearchParams sp,
                            const FaceSt* __restrict__ S, float4* __restrict__ pf, uint8_t* __restrict__ flags,
                            FaceDecisions* __restrict__ dec) {
    uint32_t li = blockIdx.x * blockDim.x + threadIdx.x;
    if (li >= na) return;
    uint32_t i = list[li];
    const FaceSt& st = S[i];
    dec[i].J1 = st.J1a;
    dec[i].J2 = st.J2a;
    dec[i].found = (uint8_t)st.found;
    ff2 q1 = ray_point(st.q, ray2(st, 0), lbs_param(sp.range2, st.J1a, sp.lin2, sp.bin2));
    ff2 q2 = ray_point(st.q, ray2(st, 1), lbs_param(sp.range2, st.J2a, sp.lin2, sp.bin2));
    int fl = 0;
    pf[i] = face_intersect(st.F, q1, q2, &fl);
    flags[i] = (uint8_t)fl;
}

static odc_status faces_body(MlpState* st, const GridDev& g, const uint32_t* bits, const uint32_t* flips,
                             const WordInfo* wi, const uint32_t* ebase, const uint32_t* T, const uint32_t* faces,
                             const uint8_t* slots, uint32_t nf, const SearchParams& sp, float iso, float4* pf,
                             uint8_t* flags, FaceDecisions* dec, cudaStream_t s, int64_t* nq, std::string* err) {
    if (!nf) return ODC_OK;
    st->stream = s;
    const float t = mlp_logit_threshold(iso);
    st->zt = t;
    const HintPar hp{t, st->zband, st->zsplit};
    const size_t n2 = (size_t)nf * 2;   // queries of one wavefront at most (two rays per face)
    float *hint = nullptr, *lh = nullptr;
    if (mlp_precision(st) == ODC_PREC_BF16) {
        void *ph, *plh;
        S_TRY(mlp_scratch(st, 36, n2 * 4, &ph, err));
        S_TRY(mlp_scratch(st, 17, n2 * 4, &plh, err));
        hint = (float*)ph;
        lh = (float*)plh;
    }
    void *pS, *ppts, *pz, *pact, *poff, *plist, *pcnt, *plp, *plz, *pll, *plc;
    S_TRY(mlp_scratch(st, 10, (size_t)nf * sizeof(FaceSt), &pS, err));
    S_TRY(mlp_scratch(st, 2, n2 * 12, &ppts, err));
    S_TRY(mlp_scratch(st, 3, n2 * 4, &pz, err));
    S_TRY(mlp_scratch(st, 11, (size_t)nf * 4, &pact, err));
    S_TRY(mlp_scratch(st, 12, (size_t)nf * 4 + scan_tmp_elems(nf) * 8 + 64, &poff, err));
    S_TRY(mlp_scratch(st, 13, (size_t)nf * 4, &plist, err));
    S_TRY(mlp_scratch(st, 14, 64, &pcnt, err));
    S_TRY(mlp_scratch(st, 15, n2 * 12, &plp, err));     // line-sample points of a round (compact)
    S_TRY(mlp_scratch(st, 16, n2 * 4, &plz, err));      // their logits
    S_TRY(mlp_scratch(st, 18, n2 * 4 * 2, &pll, err));  // two lists of searches still sampling
    S_TRY(mlp_scratch(st, 19, 2 * kMaxLin * 8, &plc, err));   // their sizes: [j] step 1 round j + 1, [kMaxLin + j] step 2
    FaceSt* S = (FaceSt*)pS;
    float3* pts = (float3*)ppts;
    float* z = (float*)pz;
    uint32_t* act = (uint32_t*)pact;
    uint32_t* off = (uint32_t*)poff;
    uint32_t* tmp = off + ((nf + 63) / 64) * 64;
    uint32_t* list = (uint32_t*)plist;
    uint32_t* cnt = (uint32_t*)pcnt;
    float3* lp = (float3*)plp;
    float* lz = (float*)plz;
    uint32_t* L[2] = {(uint32_t*)pll, (uint32_t*)pll + n2};
    unsigned long long* C = (unsigned long long*)plc;
    unsigned long long hc[2 * kMaxLin] = {};
    S_CK(cudaMemsetAsync(C, 0, 2 * kMaxLin * 8, s));

    // step 1: m, line samples (one at a time, early exit), bisections
    k_face_init<<<nblk(nf, 128), 128, 0, s>>>(g, bits, flips, wi, ebase, T, faces, slots, nf, sp.steps_1d, S, pts,
                                              hint); note_launch();
    S_TRY(mlp_eval_list(st, pts, nf, z, -1, s, err, hint));
    k_face_m<<<nblk(nf, 128), 128, 0, s>>>(nf, z, t, S); note_launch();
    for (int j = 1; j <= sp.lin1; ++j) {
        const uint32_t* lin = j == 1 ? nullptr : L[j & 1];
        const unsigned long long* cin = j == 1 ? nullptr : C + (j - 1);
        uint32_t* lout = j < sp.lin1 ? L[(j + 1) & 1] : nullptr;
        k_lin1_gen<<<nblk(nf, 128), 128, 0, s>>>(g, nf, j, lin, cin, sp, S, lp, lh, t); note_launch();
        if (cin) S_TRY(mlp_eval_list_dev(st, lp, nf, cin, lz, s, err, lh));
        else S_TRY(mlp_eval_list(st, lp, nf, lz, -1, s, err, lh));
        k_lin1_step<<<nblk(nf, kLinBlock), kLinBlock, 0, s>>>(g, nf, j, lin, cin, lz, t, sp, S, pts, hp, hint, lout,
                                                             C + j); note_launch();
    }
    for (int b = 0; b < sp.bin1; ++b) {
        S_TRY(mlp_eval_list(st, pts, nf, z, -1, s, err, hint));
        k_face_bin1<<<nblk(nf, 128), 128, 0, s>>>(g, nf, z, t, sp, b, S, pts, hp, hint); note_launch();
    }
    k_face_fin1<<<nblk(nf), 256, 0, s>>>(nf, sp, S, pf, flags, act, dec); note_launch();
    // faces still active after step 1
    exclusive_scan<uint32_t>(act, off, nf, tmp, cnt, s);
    k_list<<<nblk(nf), 256, 0, s>>>(act, off, nf, list); note_launch();
    uint32_t na = 0;
    S_CK(cudaMemcpyAsync(&na, cnt, 4, cudaMemcpyDeviceToHost, s));
    S_CK(cudaMemcpyAsync(hc, C, kMaxLin * 8, cudaMemcpyDeviceToHost, s));
    S_CK(cudaStreamSynchronize(s));
    S_CK(cudaGetLastError());
    int64_t lin1_q = nf;
    for (int j = 1; j < sp.lin1; ++j) lin1_q += (int64_t)hc[j];
    *nq += (int64_t)nf * (1 + sp.bin1) + lin1_q;
    S_TRY(mlp_tc_check(st, s, err));
    if (!na) return ODC_OK;
    // step 2: both rays from q (line samples one at a time per ray), then step 3
    const uint32_t nr = 2 * na;
    for (int j = 1; j <= sp.lin2; ++j) {
        const uint32_t* lin = j == 1 ? nullptr : L[j & 1];
        const unsigned long long* cin = j == 1 ? nullptr : C + kMaxLin + (j - 1);
        uint32_t* lout = j < sp.lin2 ? L[(j + 1) & 1] : nullptr;
        k_lin2_gen<<<nblk(nr, 128), 128, 0, s>>>(g, list, na, j, lin, cin, sp, S, lp, lh, t); note_launch();
        if (cin) S_TRY(mlp_eval_list_dev(st, lp, nr, cin, lz, s, err, lh));
        else S_TRY(mlp_eval_list(st, lp, nr, lz, -1, s, err, lh));
        k_lin2_step<<<nblk(nr, kLinBlock), kLinBlock, 0, s>>>(g, list, na, j, lin, cin, lz, t, sp, S, pts, hp, hint,
                                                             lout, C + kMaxLin + j); note_launch();
    }
    for (int b = 0; b < sp.bin2; ++b) {
        S_TRY(mlp_eval_list(st, pts, (int64_t)na * 2, z, -1, s, err, hint));
        k_face_bin2<<<nblk(na, 128), 128, 0, s>>>(g, list, na, z, t, sp, b, S, pts, hp, hint); note_launch();
    }
    k_face_fin2<<<nblk(na, 128), 128, 0, s>>>(list, na, sp, S, pf, flags, dec); note_launch();
    S_CK(cudaGetLastError());
    S_CK(cudaMemcpyAsync(hc + kMaxLin, C + kMaxLin, kMaxLin * 8, cudaMemcpyDeviceToHost, s));
    S_CK(cudaStreamSynchronize(s));
    int64_t lin2_q = nr;
    for (int j = 1; j < sp.lin2; ++j) lin2_q += (int64_t)hc[kMaxLin + j];
    *nq += (int64_t)na * 2 * sp.bin2 + lin2_q;
    return mlp_tc_check(st, s, err);
}

// A search stage is one bracket of a batch group's membership: inside it
// the network evaluations are shared with the group's other members.
odc_status mlp_bisect(MlpState* st, const GridDev& g, const uint32_t* bits, const uint32_t* edges, uint32_t ne, int k,
                      float iso, uint32_t* T, cudaStream_t s, int64_t* nq, std::string* err) {
    mlp_size_tiers(st, (int64_t)ne);
    batch_enter(st);
    const odc_status r = bisect_body(st, g, bits, edges, ne, k, iso, T, s, nq, err);
    std::string e2;
    const odc_status r2 = batch_leave(st, &e2);
    if (r == ODC_OK && r2 != ODC_OK) *err = e2;
    return r != ODC_OK ? r : r2;
}

odc_status mlp_faces(MlpState* st, const GridDev& g, const uint32_t* bits, const uint32_t* flips, const WordInfo* wi,
                     const uint32_t* ebase, const uint32_t* T, const uint32_t* faces, const uint8_t* slots,
                     uint32_t nf, const SearchParams& sp, float iso, float4* pf, uint8_t* flags, FaceDecisions* dec,
                     cudaStream_t s, int64_t* nq, std::string* err) {
    batch_enter(st);
    const odc_status r = faces_body(st, g, bits, flips, wi, ebase, T, faces, slots, nf, sp, iso, pf, flags, dec, s, nq,
                                    err);
    std::string e2;
    const odc_status r2 = batch_leave(st, &e2);
    if (r == ODC_OK && r2 != ODC_OK) *err = e2;
    return r != ODC_OK ? r : r2;
}

}  // namespace odc
