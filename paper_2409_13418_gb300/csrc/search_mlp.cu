// search_mlp.cu -- grid labels, 1D and 2D searches against an MLP occupancy,
// batched into wavefronts: every search step evaluates the network once over
// all active elements (Sec. 5.1 and 5.2 run "for all edges / faces at once";
// the network evaluation is the dense contraction).  A small kernel turns the
// logits of one step into the search-state update and the next step's query
// points; the state (integer bisection brackets, float-float geometry) stays
// on the device between steps.
#include <algorithm>

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

odc_status mlp_bisect(MlpState* st, const GridDev& g, const uint32_t* bits, const uint32_t* edges, uint32_t ne, int k,
                      float iso, uint32_t* T, cudaStream_t s, int64_t* nq, std::string* err) {
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

__global__ void k_face_init(GridDev g, const uint32_t* __restrict__ bits, const uint32_t* __restrict__ flips,
                            const WordInfo* __restrict__ wi, const uint32_t* __restrict__ ebase,
                            const uint32_t* __restrict__ T, const uint32_t* __restrict__ faces,
                            const uint8_t* __restrict__ slots, uint32_t nf, int k, FaceSt* __restrict__ S,
                            float3* __restrict__ pts) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    FaceSt st;
    load_face(g, bits, flips, wi, ebase, T, k, faces[i], slots[i], st.F);
    S[i] = st;
    pts[i] = face_world2(g, st.F, st.F.m);
}

// label of m -> step-1 ray; queries: the N1 line samples
__global__ void k_face_m(GridDev g, uint32_t nf, const float* __restrict__ z, float t, SearchParams sp,
                         FaceSt* __restrict__ S, float3* __restrict__ pts) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    FaceSt& st = S[i];
    uint32_t lab_m = z[i] > t;
    st.lab_m = lab_m;
    st.zm = z[i];
    ff2 d = lab_m ? ff2{ff_neg(st.F.d.u), ff_neg(st.F.d.v)} : st.F.d;
    st.d = d;
    for (int j = 1; j <= sp.lin1; ++j)
        pts[(size_t)(j - 1) * nf + i] =
            face_world2(g, st.F, ray_point(st.F.m, d, lbs_param(sp.range1, (uint32_t)j << sp.bin1, sp.lin1, sp.bin1)));
}

// first line sample whose label differs -> bracket; first bisection query
__global__ void k_face_lin1(GridDev g, uint32_t nf, const float* __restrict__ z, float t, SearchParams sp,
                            FaceSt* __restrict__ S, float3* __restrict__ pts, HintPar hp, float* __restrict__ hint) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    FaceSt& st = S[i];
    int first = sp.lin1;
    st.found = 0;
    for (int j = 1; j <= sp.lin1; ++j)
        if ((uint32_t)(z[(size_t)(j - 1) * nf + i] > t) != st.lab_m) { first = j; st.found = 1; break; }
    st.Ja = (uint32_t)(first - 1) << sp.bin1;
    st.Jc = (uint32_t)first << sp.bin1;
    st.za = first > 1 ? z[(size_t)(first - 2) * nf + i] : st.zm;
    st.zc = z[(size_t)(first - 1) * nf + i];
    if (sp.bin1 > 0) {
        pts[i] = face_world2(g, st.F, ray_point(st.F.m, st.d, lbs_param(sp.range1, (st.Ja + st.Jc) >> 1, sp.lin1, sp.bin1)));
        if (hint) hint[i] = bracket_hint(st.za, st.zc, hp.t, hp.zb, hp.zs);
    }
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

// step 2 line samples of both rays: slot (r * N2 + j - 1) * na + li
__global__ void k_face_lin2_gen(GridDev g, const uint32_t* __restrict__ list, uint32_t na, SearchParams sp,
                                const FaceSt* __restrict__ S, float3* __restrict__ pts) {
    uint32_t li = blockIdx.x * blockDim.x + threadIdx.x;
    if (li >= na) return;
    const FaceSt& st = S[list[li]];
    for (int r = 0; r < 2; ++r) {
        ff2 d = ray2(st, r);
        for (int j = 1; j <= sp.lin2; ++j)
            pts[(size_t)(r * sp.lin2 + j - 1) * na + li] =
                face_world2(g, st.F, ray_point(st.q, d, lbs_param(sp.range2, (uint32_t)j << sp.bin2, sp.lin2, sp.bin2)));
    }
}

__global__ void k_face_lin2(GridDev g, const uint32_t* __restrict__ list, uint32_t na, const float* __restrict__ z,
                            float t, SearchParams sp, FaceSt* __restrict__ S, float3* __restrict__ pts, HintPar hp,
                            float* __restrict__ hint) {
    uint32_t li = blockIdx.x * blockDim.x + threadIdx.x;
    if (li >= na) return;
    FaceSt& st = S[list[li]];
    uint32_t Ja[2], Jc[2];
    float za[2], zc[2];
    for (int r = 0; r < 2; ++r) {
        int first = sp.lin2;
        for (int j = 1; j <= sp.lin2; ++j)
            if ((uint32_t)(z[(size_t)(r * sp.lin2 + j - 1) * na + li] > t) != st.lab_m) {
                first = j;
                st.found |= 2u << r;
                break;
            }
        Ja[r] = (uint32_t)(first - 1) << sp.bin2;
        Jc[r] = (uint32_t)first << sp.bin2;
        // the rays start at q, the step-1 bracket end Ja, whose logit is za
        za[r] = first > 1 ? z[(size_t)(r * sp.lin2 + first - 2) * na + li] : st.za;
        zc[r] = z[(size_t)(r * sp.lin2 + first - 1) * na + li];
        if (sp.bin2 > 0) {
            pts[(size_t)r * na + li] =
                face_world2(g, st.F, ray_point(st.q, ray2(st, r), lbs_param(sp.range2, (Ja[r] + Jc[r]) >> 1, sp.lin2, sp.bin2)));
            if (hint) hint[(size_t)r * na + li] = bracket_hint(za[r], zc[r], hp.t, hp.zb, hp.zs);
        }
    }
    st.J1a = Ja[0]; st.J1c = Jc[0]; st.J2a = Ja[1]; st.J2c = Jc[1];
    st.z1a = za[0]; st.z1c = zc[0]; st.z2a = za[1]; st.z2c = zc[1];
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

odc_status mlp_faces(MlpState* st, const GridDev& g, const uint32_t* bits, const uint32_t* flips, const WordInfo* wi,
                     const uint32_t* ebase, const uint32_t* T, const uint32_t* faces, const uint8_t* slots,
                     uint32_t nf, const SearchParams& sp, float iso, float4* pf, uint8_t* flags, FaceDecisions* dec,
                     cudaStream_t s, int64_t* nq, std::string* err) {
    if (!nf) return ODC_OK;
    st->stream = s;
    const float t = mlp_logit_threshold(iso);
    st->zt = t;
    const HintPar hp{t, st->zband, st->zsplit};
    size_t nmax = (size_t)nf * std::max(sp.lin1, 2 * sp.lin2);
    float* hint = nullptr;
    if (mlp_precision(st) == ODC_PREC_BF16) {
        void* ph;
        S_TRY(mlp_scratch(st, 36, (size_t)nf * 2 * 4, &ph, err));
        hint = (float*)ph;
    }
    void *pS, *ppts, *pz, *pact, *poff, *plist, *pcnt;
    S_TRY(mlp_scratch(st, 10, (size_t)nf * sizeof(FaceSt), &pS, err));
    S_TRY(mlp_scratch(st, 2, nmax * 12, &ppts, err));
    S_TRY(mlp_scratch(st, 3, nmax * 4, &pz, err));
    S_TRY(mlp_scratch(st, 11, (size_t)nf * 4, &pact, err));
    S_TRY(mlp_scratch(st, 12, (size_t)nf * 4 + scan_tmp_elems(nf) * 8 + 64, &poff, err));
    S_TRY(mlp_scratch(st, 13, (size_t)nf * 4, &plist, err));
    S_TRY(mlp_scratch(st, 14, 64, &pcnt, err));
    FaceSt* S = (FaceSt*)pS;
    float3* pts = (float3*)ppts;
    float* z = (float*)pz;
    uint32_t* act = (uint32_t*)pact;
    uint32_t* off = (uint32_t*)poff;
    uint32_t* tmp = off + ((nf + 63) / 64) * 64;
    uint32_t* list = (uint32_t*)plist;
    uint32_t* cnt = (uint32_t*)pcnt;

    // step 1: m, line samples, bisections
    k_face_init<<<nblk(nf, 128), 128, 0, s>>>(g, bits, flips, wi, ebase, T, faces, slots, nf, sp.steps_1d, S, pts); note_launch();
    S_TRY(mlp_eval_list(st, pts, nf, z, -1, s, err));
    k_face_m<<<nblk(nf, 128), 128, 0, s>>>(g, nf, z, t, sp, S, pts); note_launch();
    S_TRY(mlp_eval_list(st, pts, (int64_t)nf * sp.lin1, z, -1, s, err));
    k_face_lin1<<<nblk(nf, 128), 128, 0, s>>>(g, nf, z, t, sp, S, pts, hp, hint); note_launch();
    for (int b = 0; b < sp.bin1; ++b) {
        S_TRY(mlp_eval_list(st, pts, nf, z, -1, s, err, hint));
        k_face_bin1<<<nblk(nf, 128), 128, 0, s>>>(g, nf, z, t, sp, b, S, pts, hp, hint); note_launch();
    }
    k_face_fin1<<<nblk(nf), 256, 0, s>>>(nf, sp, S, pf, flags, act, dec); note_launch();
    *nq += (int64_t)nf * (1 + sp.lin1 + sp.bin1);
    // faces still active after step 1
    exclusive_scan<uint32_t>(act, off, nf, tmp, cnt, s);
    k_list<<<nblk(nf), 256, 0, s>>>(act, off, nf, list); note_launch();
    uint32_t na = 0;
    S_CK(cudaMemcpyAsync(&na, cnt, 4, cudaMemcpyDeviceToHost, s));
    S_CK(cudaStreamSynchronize(s));
    S_CK(cudaGetLastError());
    S_TRY(mlp_tc_check(st, s, err));
    if (!na) return ODC_OK;
    // step 2: both rays from q, then step 3
    k_face_lin2_gen<<<nblk(na, 128), 128, 0, s>>>(g, list, na, sp, S, pts); note_launch();
    S_TRY(mlp_eval_list(st, pts, (int64_t)na * 2 * sp.lin2, z, -1, s, err));
    k_face_lin2<<<nblk(na, 128), 128, 0, s>>>(g, list, na, z, t, sp, S, pts, hp, hint); note_launch();
    for (int b = 0; b < sp.bin2; ++b) {
        S_TRY(mlp_eval_list(st, pts, (int64_t)na * 2, z, -1, s, err, hint));
        k_face_bin2<<<nblk(na, 128), 128, 0, s>>>(g, list, na, z, t, sp, b, S, pts, hp, hint); note_launch();
    }
    k_face_fin2<<<nblk(na, 128), 128, 0, s>>>(list, na, sp, S, pf, flags, dec); note_launch();
    S_CK(cudaGetLastError());
    *nq += (int64_t)na * 2 * (sp.lin2 + sp.bin2);
    return mlp_tc_check(st, s, err);
}

}  // namespace odc
