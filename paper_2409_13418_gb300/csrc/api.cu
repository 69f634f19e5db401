// api.cu -- C ABI and host orchestration of the ODC path (include/odc.h).
//
// One extract runs every stage on one stream.  The host reads counts back
// from the device twice (crossing counts to size the lists; final vertex and
// triangle counts) plus once per manifold-fix round.  Device memory comes
// from two arenas owned by the context: one sized by the grid, one by the
// crossing counts; both grow on demand and are reused across calls.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <thread>

#include "../../include/odc.h"
#include "batch.h"
#include "kernels.h"
#include "mlp.h"
#include "odc_internal.h"

using namespace odc;

namespace {

thread_local std::string g_err;

odc_status fail(odc_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

#define ODC_CK(call)                                                                                  \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess) return fail(ODC_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

struct Arena {
    char* base = nullptr;
    size_t cap = 0;
    size_t off = 0;
    void reset() { off = 0; }
    void* take(size_t bytes) {
        size_t o = (off + 255) & ~(size_t)255;
        off = o + ((bytes + 255) & ~(size_t)255);
        return base + o;
    }
};

size_t al(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

void odc::set_last_error(const std::string& msg) { g_err = msg; }

struct odc_ctx {
    int device = 0;
    size_t budget = 0;
    cudaStream_t own = nullptr;
    Arena A, B, S;              // grid-sized, count-sized, source (prims / weights)
    uint32_t* h_cnt = nullptr;  // pinned host counters
    unsigned long long wait_ns = 0;   // limit of the tensor-core kernels' pipeline waits (0: default)
    const int* gate = nullptr;        // device go signal of the tensor-core kernels (NULL: none)
    BatchGroup* batch = nullptr;      // shared network evaluations (odc_ctx_join_batch)
    cudaEvent_t ev[9] = {};
    MlpState* mlp = nullptr;
    // resident source
    int res_kind = -1;
    int res_nprims = 0;
    PrimDev* res_prims = nullptr;
    float4* res_cull = nullptr;
    VoxDev res_vox{};
    // last extract
    GridDev g{};
    int k = 0;
    uint32_t E = 0, F = 0, C = 0, V3 = 0, NT = 0, N3 = 0, nflip = 0;
    uint32_t *bits = nullptr, *flips = nullptr, *edges = nullptr, *T = nullptr, *faces = nullptr, *cells = nullptr;
    uint8_t *slots = nullptr, *fflags = nullptr, *configs = nullptr, *qcase = nullptr;
    float4* pf = nullptr;
    FaceDecisions* dec = nullptr;
    unsigned long long* cycles = nullptr;
    float3 *vlocal = nullptr, *vworld = nullptr;
    int3* tris = nullptr;
    uint32_t* vbase = nullptr;           // exclusive scan of cycles per crossing cell
    unsigned long long* qoff = nullptr;  // exclusive scan of (triangles << 32 | edge points) per edge
    size_t nw = 0;
    // merged mesh of odc_extract_slabbed
    float3* sv = nullptr;       // vertices
    int3* stri = nullptr;       // triangles
    float3* sc3 = nullptr;      // edge points, staged until the 3D point count is known
    unsigned long long* sinfo = nullptr;   // slab range counters (device, 8)
    size_t sv_cap = 0, st_cap = 0, sc3_cap = 0;
    // whole-grid topology of a slabbed extraction: label words, flip words,
    // ambiguous faces
    uint32_t* gbits = nullptr;
    uint32_t* gflips = nullptr;
    uint32_t* gfaces = nullptr;
    size_t gb_cap = 0, gfl_cap = 0, gf_cap = 0;
    size_t nga = 0;
    size_t extra_bytes() const { return (sv_cap + st_cap + sc3_cap) * 12 + (gb_cap + gfl_cap + gf_cap) * 4; }
};

// Grow an arena (stream-ordered: the old block is freed and the new one
// allocated on the stream that uses them, so growth never waits for work of
// other streams or contexts).
static odc_status arena_ensure(odc_ctx* c, Arena& a, size_t need, cudaStream_t st) {
    if (need <= a.cap) {
        a.reset();
        return ODC_OK;
    }
    size_t others = c->A.cap + c->B.cap + c->S.cap - a.cap + c->extra_bytes();
    size_t want = std::max(need, a.cap + a.cap / 4);
    if (c->budget && others + want > c->budget) {
        want = need;
        if (others + want > c->budget)
            return fail(ODC_ERR_OOM, "device arena would exceed the context memory budget (" +
                                         std::to_string(others + want) + " > " + std::to_string(c->budget) + " bytes)");
    }
    if (a.base) {
        ODC_CK(cudaFreeAsync(a.base, st));
        a.base = nullptr;
        a.cap = 0;
    }
    cudaError_t e = cudaMallocAsync((void**)&a.base, want, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ODC_ERR_OOM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
    }
    a.cap = want;
    a.reset();
    return ODC_OK;
}

// Grow a device array (stream-ordered; the old contents are kept).
template <typename T>
static odc_status grow(odc_ctx* c, T** p, size_t* cap, size_t need, cudaStream_t st) {
    if (need <= *cap) return ODC_OK;
    size_t want = std::max(need, *cap + *cap / 2);
    size_t others = c->A.cap + c->B.cap + c->S.cap + c->extra_bytes() - *cap * sizeof(T);
    if (c->budget && others + want * sizeof(T) > c->budget) {
        want = need;
        if (others + want * sizeof(T) > c->budget)
            return fail(ODC_ERR_OOM, "merged slab mesh would exceed the context memory budget");
    }
    T* q = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&q, want * sizeof(T), st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ODC_ERR_OOM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
    }
    if (*p) {
        if (*cap) ODC_CK(cudaMemcpyAsync(q, *p, *cap * sizeof(T), cudaMemcpyDeviceToDevice, st));
        ODC_CK(cudaFreeAsync(*p, st));
    }
    *p = q;
    *cap = want;
    return ODC_OK;
}

extern "C" {

const char* odc_status_str(odc_status s) {
    switch (s) {
        case ODC_OK: return "ok";
        case ODC_ERR_INVALID_ARG: return "invalid argument";
        case ODC_ERR_OOM: return "out of memory";
        case ODC_ERR_CUDA: return "CUDA error";
        case ODC_ERR_TIMEOUT: return "timeout";
        case ODC_ERR_UNSUPPORTED: return "unsupported";
        case ODC_ERR_INTERNAL: return "internal error";
    }
    return "unknown status";
}

const char* odc_last_error(void) { return g_err.c_str(); }

int64_t odc_launch_count(void) { return (int64_t)launch_count(); }

odc_status odc_ctx_create(int device, size_t mem_budget, odc_ctx** out) {
    if (!out) return fail(ODC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int n = 0;
    ODC_CK(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) return fail(ODC_ERR_INVALID_ARG, "no such CUDA device");
    ODC_CK(cudaSetDevice(device));
    odc_ctx* c = new odc_ctx();
    c->device = device;
    c->budget = mem_budget;
    cudaError_t e = cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&c->h_cnt, 64 * sizeof(uint32_t));
    for (int i = 0; i < 9 && e == cudaSuccess; ++i) e = cudaEventCreate(&c->ev[i]);
    if (e != cudaSuccess) {
        odc_ctx_destroy(c);
        return fail(ODC_ERR_CUDA, std::string("context setup: ") + cudaGetErrorString(e));
    }
    *out = c;
    return ODC_OK;
}

odc_status odc_ctx_destroy(odc_ctx* c) {
    if (!c) return ODC_OK;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();   // arenas may still be in use on a caller's stream
    mlp_destroy(c->mlp);
    for (Arena* a : {&c->A, &c->B, &c->S})
        if (a->base) cudaFree(a->base);
    for (void* p : {(void*)c->sv, (void*)c->stri, (void*)c->sc3, (void*)c->sinfo, (void*)c->gbits, (void*)c->gflips,
                    (void*)c->gfaces})
        if (p) cudaFree(p);
    for (auto& e : c->ev)
        if (e) cudaEventDestroy(e);
    if (c->h_cnt) cudaFreeHost(c->h_cnt);
    if (c->own) cudaStreamDestroy(c->own);
    delete c;
    return ODC_OK;
}

static odc_status check_source(const odc_source* src) {
    if (!src) return fail(ODC_ERR_INVALID_ARG, "source is NULL");
    if (src->kind == ODC_SRC_RESIDENT) return ODC_OK;
    if (src->kind == ODC_SRC_CSG) {
        if (!src->prims) return fail(ODC_ERR_INVALID_ARG, "CSG source without primitives");
        if (src->n_prims < 1 || src->n_prims > kMaxPrims) return fail(ODC_ERR_INVALID_ARG, "n_prims out of [1, 4096]");
        for (int i = 0; i < src->n_prims; ++i) {
            const odc_csg_prim& p = src->prims[i];
            if (p.type < 0 || p.type > 4) return fail(ODC_ERR_INVALID_ARG, "unknown primitive type");
            if (p.op != 0 && p.op != 1) return fail(ODC_ERR_INVALID_ARG, "unknown primitive op");
        }
        return ODC_OK;
    }
    if (src->kind == ODC_SRC_MLP) return mlp_check(src->mlp, &g_err);
    if (src->kind == ODC_SRC_VOXEL) {
        const odc_voxels* v = src->voxels;
        if (!v || !v->values) return fail(ODC_ERR_INVALID_ARG, "voxel source without values");
        double n = 1.0;
        for (int a = 0; a < 3; ++a) {
            if (v->dims[a] < 2 || v->dims[a] > 2048) return fail(ODC_ERR_INVALID_ARG, "voxel dims out of [2, 2048]");
            if (!(v->lo[a] < v->hi[a])) return fail(ODC_ERR_INVALID_ARG, "voxel box: lo must be < hi");
            n *= v->dims[a];
        }
        if (n > 2147483648.0) return fail(ODC_ERR_INVALID_ARG, "voxel volume above 2^31 samples");
        return ODC_OK;
    }
    return fail(ODC_ERR_INVALID_ARG, "unknown source kind");
}

// Upload a CSG source: primitives and per-primitive culling spheres.
static odc_status upload_csg(odc_ctx* c, const odc_source* src, cudaStream_t st, PrimDev** d_prims,
                             float4** d_cull) {
    int n = src->n_prims;
    std::vector<float4> cull(n);
    for (int i = 0; i < n; ++i) {
        const odc_csg_prim& p = src->prims[i];
        double r;
        switch (p.type) {
            case ODC_PRIM_SPHERE: r = std::fabs((double)p.params[0]); break;
            case ODC_PRIM_AABB:
            case ODC_PRIM_OBOX:
                r = std::sqrt((double)p.params[0] * p.params[0] + (double)p.params[1] * p.params[1] +
                              (double)p.params[2] * p.params[2]);
                if (p.type == ODC_PRIM_OBOX) {   // rows of rot may not be exactly unit
                    double s = 0;
                    for (int k = 0; k < 9; ++k) s = std::max(s, std::fabs((double)p.rot[k]));
                    r *= std::max(1.0, 3.0 * s);
                }
                break;
            case ODC_PRIM_CYLINDER: {
                double an = std::sqrt((double)p.rot[6] * p.rot[6] + (double)p.rot[7] * p.rot[7] + (double)p.rot[8] * p.rot[8]);
                r = std::sqrt((double)p.params[0] * p.params[0] + (double)p.params[1] * p.params[1]) * std::max(1.0, 1.0 / std::max(an, 1e-3)) * 1.01;
                break;
            }
            default: {
                double an = std::sqrt((double)p.rot[6] * p.rot[6] + (double)p.rot[7] * p.rot[7] + (double)p.rot[8] * p.rot[8]);
                r = (std::fabs((double)p.params[0]) + std::fabs((double)p.params[1])) * std::max(1.0, 1.0 / std::max(an, 1e-3)) * 1.01;
            }
        }
        double rr = r * (1.0 + 1e-4) + 1e-6;
        cull[i] = make_float4(p.center[0], p.center[1], p.center[2], (float)(rr * rr));
    }
    size_t need = al(sizeof(PrimDev) * n) + al(sizeof(float4) * n);
    odc_status s = arena_ensure(c, c->S, need, st);
    if (s != ODC_OK) return s;
    *d_prims = (PrimDev*)c->S.take(sizeof(PrimDev) * n);
    *d_cull = (float4*)c->S.take(sizeof(float4) * n);
    ODC_CK(cudaMemcpyAsync(*d_prims, src->prims, sizeof(PrimDev) * n, cudaMemcpyHostToDevice, st));
    ODC_CK(cudaMemcpyAsync(*d_cull, cull.data(), sizeof(float4) * n, cudaMemcpyHostToDevice, st));
    return ODC_OK;
}

// Upload a voxel volume (values into the source arena).
static odc_status upload_voxels(odc_ctx* c, const odc_voxels* v, cudaStream_t st) {
    const size_t n = (size_t)v->dims[0] * v->dims[1] * v->dims[2];
    odc_status s = arena_ensure(c, c->S, al(n * 4), st);
    if (s != ODC_OK) return s;
    float* d = (float*)c->S.take(n * 4);
    ODC_CK(cudaMemcpyAsync(d, v->values, n * 4, cudaMemcpyHostToDevice, st));
    VoxDev& x = c->res_vox;
    x.v = d;
    for (int a = 0; a < 3; ++a) {
        x.dims[a] = v->dims[a];
        x.lo[a] = v->lo[a];
        // hi - lo as float-float: the rounded difference and its exact remainder
        const float hi = v->hi[a], lo = v->lo[a], r = hi - lo;
        const float bb = r - hi;
        x.rng_hi[a] = r;
        x.rng_lo[a] = (hi - (r - bb)) + (-lo - bb);
    }
    x.iso = 0.5f;
    return ODC_OK;
}

static odc_status upload_source(odc_ctx* c, const odc_source* src, cudaStream_t st) {
    odc_status s;
    c->res_kind = -1;
    if (src->kind == ODC_SRC_VOXEL) {
        s = upload_voxels(c, src->voxels, st);
        if (s != ODC_OK) return s;
    } else if (src->kind == ODC_SRC_CSG) {
        s = upload_csg(c, src, st, &c->res_prims, &c->res_cull);
        if (s != ODC_OK) return s;
        c->res_nprims = src->n_prims;
    } else {
        s = mlp_prepare(&c->mlp, src->mlp, st, &g_err);
        if (s != ODC_OK) return s;
    }
    c->res_kind = src->kind;
    return ODC_OK;
}

static void grid_coords(const odc_grid* grid, int a, std::vector<float>& X) {
    int n = grid->res[a];
    X.resize(n + 1);
    for (int i = 0; i <= n; ++i)
        X[i] = (float)((double)grid->lo[a] + ((double)grid->hi[a] - (double)grid->lo[a]) * (double)i / (double)n);
}

static odc_status check_params(const odc_params* prm) {
    if (prm->steps_1d < 1 || prm->steps_1d > 20) return fail(ODC_ERR_INVALID_ARG, "steps_1d out of [1, 20]");
    if (prm->s2d_lin1 < 1 || prm->s2d_lin2 < 1 || prm->s2d_bin1 < 0 || prm->s2d_bin2 < 0 || prm->s2d_lin1 > 64 ||
        prm->s2d_lin2 > 64 || prm->s2d_bin1 > 20 || prm->s2d_bin2 > 20 || !(prm->s2d_range1 > 0) ||
        !(prm->s2d_range2 > 0))
        return fail(ODC_ERR_INVALID_ARG, "2D search parameters out of range");
    if (!(prm->iso > 0.0f && prm->iso < 1.0f)) return fail(ODC_ERR_INVALID_ARG, "iso must be in (0, 1)");
    if (prm->flags & ~(ODC_ABL_LINEAR_1D | ODC_ABL_GRADIENT_NORMALS | ODC_POLY_MC))
        return fail(ODC_ERR_INVALID_ARG, "unknown flags");
    return ODC_OK;
}

// The whole path on the grid whose vertex coordinates per axis are Xh[a]
// (Xh[a].size() - 1 cells); arguments already checked.
static odc_status extract_impl(odc_ctx* c, const odc_source* src, const std::vector<float> (&Xh)[3],
                               const odc_params* prm, cudaStream_t st, odc_mesh* out,
                               const int* watch = nullptr, unsigned long long* watch_cnt = nullptr,
                               const uint32_t* ext_flips = nullptr, int ext_z0 = 0, int ext_nz = 0) {
    odc_status s = ODC_OK;
    std::memset(out, 0, sizeof(*out));

    // ---- source upload (skipped for a resident source)
    if (src->kind != ODC_SRC_RESIDENT) {
        s = upload_source(c, src, st);
        if (s != ODC_OK) return s;
    } else if (c->res_kind < 0) {
        return fail(ODC_ERR_INVALID_ARG, "no resident source on this context");
    }
    const int kind = c->res_kind;
    mlp_set_wait_limit(c->mlp, c->wait_ns, c->gate);
    if (c->mlp) {
        s = batch_bind(c->mlp, c->batch, src->kind == ODC_SRC_MLP ? src->mlp : nullptr, &g_err);
        if (s != ODC_OK) return s;
    }
    if ((prm->flags & (ODC_ABL_LINEAR_1D | ODC_ABL_GRADIENT_NORMALS)) && kind != ODC_SRC_CSG)
        return fail(ODC_ERR_UNSUPPORTED, "ablation variants need an implicit with a gradient: CSG sources only");
    const bool linear_1d = (prm->flags & ODC_ABL_LINEAR_1D) != 0;
    const bool mc = (prm->flags & ODC_POLY_MC) != 0;
    const bool grad_normals = !mc && (prm->flags & ODC_ABL_GRADIENT_NORMALS) != 0;
    PrimDev* d_prims = c->res_prims;
    float4* d_cull = c->res_cull;
    const int n_prims = c->res_nprims;

    // ---- grid-sized buffers
    GridDev g{};
    for (int a = 0; a < 3; ++a) {
        g.n[a] = (int)Xh[a].size() - 1;
        g.nv[a] = (int)Xh[a].size();
    }
    g.W = (g.nv[0] + 31) / 32;
    size_t nw = (size_t)g.W * g.nv[1] * g.nv[2];
    size_t nX = Xh[0].size() + Xh[1].size() + Xh[2].size();
    size_t stmp = scan_tmp_elems(nw);
    size_t needA = al(nX * 4) + al(nw * 4) + al(nw * sizeof(WordInfo)) + 6 * al(nw * 4) + al(3 * nw * 4) +
                   al(stmp * 8) + al(64 * 8) + 2 * al(nX * 4);
    s = arena_ensure(c, c->A, needA, st);
    if (s != ODC_OK) return s;
    float* dX = (float*)c->A.take(nX * 4);
    uint32_t* bits = (uint32_t*)c->A.take(nw * 4);
    WordInfo* wi = (WordInfo*)c->A.take(nw * sizeof(WordInfo));
    uint32_t* ce = (uint32_t*)c->A.take(nw * 4);
    uint32_t* cf = (uint32_t*)c->A.take(nw * 4);
    uint32_t* cc = (uint32_t*)c->A.take(nw * 4);
    uint32_t* ebase = (uint32_t*)c->A.take(nw * 4);
    uint32_t* fbase = (uint32_t*)c->A.take(nw * 4);
    uint32_t* cbase = (uint32_t*)c->A.take(nw * 4);
    uint32_t* flips = (uint32_t*)c->A.take(3 * nw * 4);
    void* tmp = c->A.take(stmp * 8);
    uint32_t* dcnt = (uint32_t*)c->A.take(64 * 8);
    int* axis_c = (int*)c->A.take(nX * 4);
    float* axis_f = (float*)c->A.take(nX * 4);
    g.X[0] = dX;
    g.X[1] = dX + Xh[0].size();
    g.X[2] = dX + Xh[0].size() + Xh[1].size();
    for (int a = 0; a < 3; ++a)
        ODC_CK(cudaMemcpyAsync((void*)g.X[a], Xh[a].data(), Xh[a].size() * 4, cudaMemcpyHostToDevice, st));
    ODC_CK(cudaMemsetAsync(flips, 0, 3 * nw * 4, st));
    ODC_CK(cudaMemsetAsync(dcnt, 0, 64 * 8, st));

    SearchParams sp{prm->steps_1d, prm->s2d_lin1, prm->s2d_bin1, prm->s2d_range1,
                    prm->s2d_lin2, prm->s2d_bin2, prm->s2d_range2, prm->ic_split};
    int64_t nq = 0;

    const long long launches0 = launch_count();
    mlp_timing_begin(c->mlp, st);
    ODC_CK(cudaEventRecord(c->ev[0], st));
    // ---- a1: grid occupancy
    VoxDev vox = c->res_vox;
    vox.iso = prm->iso;
    if (kind == ODC_SRC_CSG) {
        launch_csg_grid(g, d_prims, d_cull, n_prims, bits, st);
    } else if (kind == ODC_SRC_VOXEL) {
        launch_vox_grid(g, vox, axis_c, axis_f, bits, st);
    } else {
        s = mlp_grid(c->mlp, g, prm->iso, bits, st, &nq, &g_err);
        if (s != ODC_OK) return s;
    }
    nq += (int64_t)g.nv[0] * g.nv[1] * g.nv[2];
    ODC_CK(cudaGetLastError());
    ODC_CK(cudaEventRecord(c->ev[1], st));
    // ---- a2: compaction
    launch_classify(g, bits, wi, ce, cf, cc, st);
    exclusive_scan<uint32_t>(ce, ebase, nw, (uint32_t*)tmp, dcnt + 0, st);
    exclusive_scan<uint32_t>(cf, fbase, nw, (uint32_t*)tmp, dcnt + 1, st);
    exclusive_scan<uint32_t>(cc, cbase, nw, (uint32_t*)tmp, dcnt + 2, st);
    ODC_CK(cudaMemcpyAsync(c->h_cnt, dcnt, 3 * 4, cudaMemcpyDeviceToHost, st));
    ODC_CK(cudaStreamSynchronize(st));
    ODC_CK(cudaGetLastError());
    uint32_t E = c->h_cnt[0], F = c->h_cnt[1], C = c->h_cnt[2];

    // ---- count-sized buffers
    size_t stmpB = scan_tmp_elems(std::max<size_t>(std::max(E, C), 1));
    size_t needB = 2 * al(E * 4ull) + al(F * 4ull) + 3 * al(F) + al(F * 16ull) + al(F * sizeof(FaceDecisions)) + al(C * 4ull) + al(C) + al(C * 8ull) +
                   2 * al(C * 4ull) + al(4ull * C * 12) + al((4ull * C + E) * 12) + al(E) + al(E * 16ull) +
                   2 * al(E * 8ull) + al(4ull * E * 12) + al(stmpB * 8) + al(E * 12ull) + 2 * al(C * 4ull) + 1024;
    s = arena_ensure(c, c->B, needB, st);
    if (s != ODC_OK) return s;
    uint32_t* edges = (uint32_t*)c->B.take(E * 4ull);
    uint32_t* T = (uint32_t*)c->B.take(E * 4ull);
    uint32_t* faces = (uint32_t*)c->B.take(F * 4ull);
    uint8_t* slots = (uint8_t*)c->B.take(F);
    uint8_t* fflags = (uint8_t*)c->B.take(F);
    uint8_t* mark = (uint8_t*)c->B.take(F);
    float4* pf = (float4*)c->B.take(F * 16ull);
    FaceDecisions* dec = (FaceDecisions*)c->B.take(F * sizeof(FaceDecisions));
    uint32_t* cells = (uint32_t*)c->B.take(C * 4ull);
    uint8_t* configs = (uint8_t*)c->B.take(C);
    unsigned long long* cycles = (unsigned long long*)c->B.take(C * 8ull);
    uint32_t* ncyc = (uint32_t*)c->B.take(C * 4ull);
    uint32_t* vbase = (uint32_t*)c->B.take(C * 4ull);
    float3* vlocal = (float3*)c->B.take(4ull * C * 12);
    float3* vworld = (float3*)c->B.take((4ull * C + E) * 12);
    uint8_t* qcase = (uint8_t*)c->B.take(E);
    int4* qv = (int4*)c->B.take(E * 16ull);
    unsigned long long* qcnt = (unsigned long long*)c->B.take(E * 8ull);
    unsigned long long* qoff = (unsigned long long*)c->B.take(E * 8ull);
    int3* tris = (int3*)c->B.take(4ull * E * 12);
    void* tmpB = c->B.take(stmpB * 8);
    float3* gnorm = grad_normals ? (float3*)c->B.take(E * 12ull) : nullptr;
    uint32_t* mc_cnt = (uint32_t*)c->B.take(C * 4ull);
    uint32_t* mc_off = (uint32_t*)c->B.take(C * 4ull);

    launch_emit(g, bits, wi, ebase, fbase, cbase, edges, faces, slots, cells, configs, st);
    ODC_CK(cudaGetLastError());
    ODC_CK(cudaEventRecord(c->ev[2], st));

    // ---- a3: manifold fix rounds (or the whole grid's flips, for a window
    // of its vertex layers), cycles, 3D point ids
    int rounds = 0;
    uint32_t nflip = 0;
    if (ext_flips) {
        const size_t plane = (size_t)g.nv[1] * g.W;
        for (int a = 0; a < 3; ++a)
            ODC_CK(cudaMemcpyAsync(flips + (size_t)a * g.nv[2] * plane,
                                   ext_flips + ((size_t)a * (ext_nz + 1) + ext_z0) * plane, g.nv[2] * plane * 4,
                                   cudaMemcpyDeviceToDevice, st));
    }
    for (; !ext_flips;) {
        ODC_CK(cudaMemsetAsync(dcnt + 8, 0, 4, st));
        launch_manifold_mark(g, bits, flips, faces, slots, F, mark, dcnt + 8, st);
        ODC_CK(cudaMemcpyAsync(c->h_cnt + 8, dcnt + 8, 4, cudaMemcpyDeviceToHost, st));
        ODC_CK(cudaStreamSynchronize(st));
        uint32_t marked = c->h_cnt[8];
        if (!marked) break;
        if (watch) launch_slab_watch(g, faces, mark, F, watch, watch_cnt, st);
        launch_manifold_apply(g, flips, faces, mark, F, st);
        nflip += marked;   // faces flipped (each flip round toggles distinct faces)
        if (++rounds > 64) return fail(ODC_ERR_INTERNAL, "manifold fix did not converge");
    }
    launch_cells(g, flips, cells, configs, C, cycles, ncyc, st);
    exclusive_scan<uint32_t>(ncyc, vbase, C, (uint32_t*)tmpB, dcnt + 3, st);
    ODC_CK(cudaGetLastError());
    ODC_CK(cudaEventRecord(c->ev[3], st));

    // ---- a4: 1D search
    if (kind == ODC_SRC_CSG) {
        if (linear_1d) launch_linear_1d(g, edges, E, prm->steps_1d, d_prims, n_prims, T, st);
        else launch_bisect_csg(g, bits, edges, E, prm->steps_1d, d_prims, d_cull, n_prims, T, st);
        nq += (int64_t)E * prm->steps_1d;
    } else if (kind == ODC_SRC_VOXEL) {
        launch_bisect_vox(g, bits, edges, E, prm->steps_1d, vox, T, st);
        nq += (int64_t)E * prm->steps_1d;
    } else {
        s = mlp_bisect(c->mlp, g, bits, edges, E, prm->steps_1d, prm->iso, T, st, &nq, &g_err);
        if (s != ODC_OK) return s;
    }
    ODC_CK(cudaGetLastError());
    ODC_CK(cudaEventRecord(c->ev[4], st));

    uint32_t V3 = 0, NT = 0, N3 = 0, NV = 0;
    if (mc) {
        // ---- marching-cubes polygons through the 1D points: no 2D search, QEF or quads
        if (F) {
            ODC_CK(cudaMemsetAsync(pf, 0, F * 16ull, st));
            ODC_CK(cudaMemsetAsync(fflags, 0, F, st));
            ODC_CK(cudaMemsetAsync(dec, 0, F * sizeof(FaceDecisions), st));
        }
        if (E) ODC_CK(cudaMemsetAsync(qcase, 0, E, st));
        ODC_CK(cudaEventRecord(c->ev[5], st));
        ODC_CK(cudaEventRecord(c->ev[6], st));
        launch_mc(g, flips, wi, ebase, edges, T, E, prm->steps_1d, cells, configs, cycles, C, mc_cnt, mc_off,
                  (uint32_t*)tmpB, dcnt + 24, vworld, tris, st);
        ODC_CK(cudaGetLastError());
        ODC_CK(cudaEventRecord(c->ev[7], st));
        ODC_CK(cudaMemcpyAsync(c->h_cnt + 16, dcnt, 32 * 4, cudaMemcpyDeviceToHost, st));
        ODC_CK(cudaStreamSynchronize(st));
        NT = c->h_cnt[16 + 24];
        NV = E;
    } else {
        // ---- a5: 2D search
        if (grad_normals) {   // Eq. 3 normals replace the 2D points: no 2D search
            launch_edge_grad(g, edges, T, E, prm->steps_1d, d_prims, n_prims, gnorm, st);
            if (F) {
                ODC_CK(cudaMemsetAsync(pf, 0, F * 16ull, st));
                ODC_CK(cudaMemsetAsync(fflags, 0, F, st));
                ODC_CK(cudaMemsetAsync(dec, 0, F * sizeof(FaceDecisions), st));
            }
        } else if (kind == ODC_SRC_CSG) {
            launch_face_csg(g, bits, flips, wi, ebase, T, faces, slots, F, sp, d_prims, d_cull, n_prims, pf, fflags,
                            dec, st);
        } else if (kind == ODC_SRC_VOXEL) {
            launch_face_vox(g, bits, flips, wi, ebase, T, faces, slots, F, sp, vox, pf, fflags, dec, st);
        } else {
            s = mlp_faces(c->mlp, g, bits, flips, wi, ebase, T, faces, slots, F, sp, prm->iso, pf, fflags, dec, st, &nq,
                          &g_err);
            if (s != ODC_OK) return s;
        }
        ODC_CK(cudaGetLastError());
        ODC_CK(cudaEventRecord(c->ev[5], st));

        // ---- a6, a7: normals and QEF
        launch_qef(g, flips, wi, ebase, fbase, T, pf, gnorm, cells, configs, cycles, vbase, C, prm->steps_1d, vlocal,
                   vworld, st);
        ODC_CK(cudaGetLastError());
        ODC_CK(cudaEventRecord(c->ev[6], st));

        // ---- a8: quads with IC split
        launch_quad_case(g, bits, wi, cbase, edges, E, cycles, vbase, vlocal, prm->ic_split, qcase, qv, qcnt, st);
        exclusive_scan<unsigned long long>(qcnt, qoff, E, (unsigned long long*)tmpB, (unsigned long long*)(dcnt + 16), st);
        launch_quad_emit(g, edges, T, E, prm->steps_1d, qcase, qv, qoff, dcnt + 3, vworld, tris, st);
        ODC_CK(cudaGetLastError());
        ODC_CK(cudaEventRecord(c->ev[7], st));
        ODC_CK(cudaMemcpyAsync(c->h_cnt + 16, dcnt, 24 * 4, cudaMemcpyDeviceToHost, st));
        ODC_CK(cudaStreamSynchronize(st));
        V3 = c->h_cnt[16 + 3];
        unsigned long long qt = ((unsigned long long)c->h_cnt[16 + 17] << 32) | c->h_cnt[16 + 16];
        NT = (uint32_t)(qt >> 32);
        N3 = (uint32_t)(qt & 0xffffffffu);
        NV = V3 + N3;
    }

    c->g = g;
    c->k = prm->steps_1d;
    c->E = E; c->F = F; c->C = C; c->V3 = V3; c->NT = NT; c->N3 = N3; c->nflip = nflip;
    c->bits = bits; c->flips = flips; c->edges = edges; c->T = T; c->faces = faces; c->cells = cells;
    c->slots = slots; c->fflags = fflags; c->configs = configs; c->qcase = qcase; c->pf = pf; c->dec = dec; c->cycles = cycles;
    c->vlocal = vlocal; c->vworld = vworld; c->tris = tris; c->nw = nw;
    c->vbase = vbase; c->qoff = mc ? nullptr : qoff;

    out->n_verts = (int64_t)NV;
    out->n_tris = NT;
    out->d_verts = (const float*)vworld;
    out->d_tris = (const int32_t*)tris;
    odc_stats& S = out->stats;
    S.n_edges = E; S.n_face_segs = F; S.n_cells = C; S.n_verts3 = V3; S.n_case3 = N3;
    S.n_flips = nflip; S.fix_rounds = rounds; S.n_queries = nq; S.n_requeries = 0;
    for (int i = 0; i < 7; ++i) cudaEventElapsedTime(&S.stage_ms[i], c->ev[i], c->ev[i + 1]);
    cudaEventElapsedTime(&S.stage_ms[7], c->ev[0], c->ev[7]);
    S.n_launches = (int32_t)(launch_count() - launches0);
    if (kind == ODC_SRC_MLP) {
        mlp_timing_finish(c->mlp, st);
        S.n_requeries = mlp_fp32_requery_count(c->mlp);
        mlp_timing_collect(c->mlp, 0, &S.mlp_ms, &S.mlp_flops, &S.mlp_launches);
        mlp_timing_collect(c->mlp, 1, &S.tc_ms, &S.tc_flops, &S.tc_launches);
        mlp_timing_collect(c->mlp, 2, &S.split_ms, &S.split_flops, &S.split_launches);
        mlp_timing_collect(c->mlp, 3, &S.h16_ms, &S.h16_flops, &S.h16_launches);
        mlp_timing_collect(c->mlp, 4, &S.fp8_ms, &S.fp8_flops, &S.fp8_launches);
        S.n_split = mlp_split_count(c->mlp);
        S.n_h16 = mlp_h16_count(c->mlp);
        S.fp32_tile = mlp_fp32_variant(c->mlp);
        mlp_split_settings(c->mlp, &S.split_zmargin, &S.split_acc_comp);
    } else {
        S.fp32_tile = -1;
        S.split_zmargin = S.split_acc_comp = 0.0f;
    }
    return ODC_OK;
}

odc_status odc_extract(odc_ctx* c, const odc_source* src, const odc_grid* grid, const odc_params* prm,
                       void* cuda_stream, odc_mesh* out) {
    if (!c || !grid || !prm || !out) return fail(ODC_ERR_INVALID_ARG, "NULL argument");
    odc_status s = check_source(src);
    if (s != ODC_OK) return s;
    for (int a = 0; a < 3; ++a) {
        if (grid->res[a] < 1 || grid->res[a] > kMaxRes) return fail(ODC_ERR_INVALID_ARG, "res out of [1, 1024]");
        if (!(grid->lo[a] < grid->hi[a])) return fail(ODC_ERR_INVALID_ARG, "lo must be < hi");
    }
    s = check_params(prm);
    if (s != ODC_OK) return s;
    ODC_CK(cudaSetDevice(c->device));
    cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : c->own;
    std::vector<float> Xh[3];
    for (int a = 0; a < 3; ++a) grid_coords(grid, a, Xh[a]);
    return extract_impl(c, src, Xh, prm, st, out);
}

// ---- z-slab extraction
static odc_status check_slab_grid(const odc_grid* grid) {
    for (int a = 0; a < 3; ++a) {
        const int lim = a < 2 ? 2048 : 8192;
        if (grid->res[a] < 1 || grid->res[a] > lim)
            return fail(ODC_ERR_INVALID_ARG, "slab grid res out of [1, 2048] x [1, 2048] x [1, 8192]");
        if (!(grid->lo[a] < grid->hi[a])) return fail(ODC_ERR_INVALID_ARG, "lo must be < hi");
    }
    return ODC_OK;
}

static odc_status slab_extract(odc_ctx* c, const odc_source* src, const odc_grid* grid, const odc_params* prm,
                               const odc_slab* sl, cudaStream_t st, odc_mesh* out, odc_slab_info* info) {
    if (prm->flags & ODC_POLY_MC) return fail(ODC_ERR_UNSUPPORTED, "slab extraction of marching-cubes polygons");
    const int nz = grid->res[2];
    if (sl->z0 < 0 || sl->z1 <= sl->z0 || sl->z1 > nz || sl->halo < 1)
        return fail(ODC_ERR_INVALID_ARG, "slab needs 0 <= z0 < z1 <= res[2] and halo >= 1");
    const int za = std::max(0, sl->z0 - sl->halo), zb = std::min(nz, sl->z1 + sl->halo);
    const unsigned long long nv01 = (unsigned long long)(grid->res[0] + 1) * (grid->res[1] + 1);
    if (3ull * nv01 * (unsigned long long)(zb - za + 1) >= (1ull << 32))
        return fail(ODC_ERR_INVALID_ARG, "slab too deep for 32-bit element ids: use more slabs");
    std::vector<float> Xh[3], Xz;
    for (int a = 0; a < 3; ++a) grid_coords(grid, a, Xh[a]);
    Xh[2] = std::vector<float>(Xh[2].begin() + za, Xh[2].begin() + zb + 1);   // the whole grid's z coordinates
    if (!c->sinfo) ODC_CK(cudaMalloc((void**)&c->sinfo, 8 * sizeof(unsigned long long)));
    ODC_CK(cudaMemsetAsync(c->sinfo + 6, 0, sizeof(unsigned long long), st));
    // with the whole grid's flips the window takes them; otherwise it runs the
    // fix itself and counts marks within two layers of an inner slab plane
    int watch[4] = {0, 0, 0, 0};
    if (sl->z0 > 0) { watch[0] = std::max(0, sl->z0 - 2 - za); watch[1] = sl->z0 + 2 - za; }
    if (sl->z1 < nz) { watch[2] = sl->z1 - 2 - za; watch[3] = sl->z1 + 2 - za; }
    odc_status s = sl->flips ? extract_impl(c, src, Xh, prm, st, out, nullptr, nullptr, sl->flips, za, nz)
                             : extract_impl(c, src, Xh, prm, st, out, watch, c->sinfo + 6);
    if (s != ODC_OK) return s;
    const uint32_t n01 = (uint32_t)grid->res[0] * (uint32_t)grid->res[1];
    const uint32_t zl0 = (uint32_t)(sl->z0 - za), zl1 = (uint32_t)(sl->z1 - za);
    launch_slab_ranges(c->cells, c->C, c->vbase, c->V3, c->edges, c->E, c->qoff, c->N3, c->NT, n01 * zl0, n01 * zl1,
                       (uint32_t)(3ull * nv01 * zl0), (uint32_t)(3ull * nv01 * zl1), c->sinfo, st);
    unsigned long long h[7];
    ODC_CK(cudaMemcpyAsync(h, c->sinfo, sizeof(h), cudaMemcpyDeviceToHost, st));
    ODC_CK(cudaStreamSynchronize(st));
    ODC_CK(cudaGetLastError());
    info->verts3_local = c->V3;
    info->verts3_before = (int64_t)h[0];
    info->verts3_owned = (int64_t)(h[1] - h[0]);
    info->case3_before = (int64_t)h[2];
    info->case3_owned = (int64_t)(h[3] - h[2]);
    info->tris_before = (int64_t)h[4];
    info->tris_owned = (int64_t)(h[5] - h[4]);
    info->fix_near_plane = (int64_t)h[6];
    return ODC_OK;
}

static odc_status slab_place(odc_ctx* c, const odc_mesh* m, const odc_slab_info* in, int64_t verts3_base,
                             int64_t case3_base, int64_t tris_base, float3* dv, float3* dc3, int3* dt,
                             cudaStream_t st) {
    const float3* v = (const float3*)m->d_verts;
    if (in->verts3_owned)
        ODC_CK(cudaMemcpyAsync(dv + verts3_base, v + in->verts3_before, in->verts3_owned * 12,
                               cudaMemcpyDeviceToDevice, st));
    if (in->case3_owned)
        ODC_CK(cudaMemcpyAsync(dc3, v + in->verts3_local + in->case3_before, in->case3_owned * 12,
                               cudaMemcpyDeviceToDevice, st));
    // 3D points: local id i -> verts3_base + (i - verts3_before); edge points -> case3_base + ...
    launch_slab_tris((const int3*)m->d_tris + in->tris_before, in->tris_owned, in->verts3_local,
                     verts3_base - in->verts3_before, in->case3_before, case3_base, dt + tris_base, st);
    ODC_CK(cudaGetLastError());
    return ODC_OK;
}

// Label words of the whole grid's vertex layers [z0, z1] (grid-order word
// layout, W words per row) into bits_g: the grid stage alone on that window.
static odc_status labels_into(odc_ctx* c, const odc_grid* grid, const odc_params* prm, int z0, int z1,
                              uint32_t* bits_g, cudaStream_t st) {
    std::vector<float> Xh[3];
    for (int a = 0; a < 3; ++a) grid_coords(grid, a, Xh[a]);
    Xh[2] = std::vector<float>(Xh[2].begin() + z0, Xh[2].begin() + z1 + 1);
    GridDev g{};
    for (int a = 0; a < 3; ++a) {
        g.n[a] = (int)Xh[a].size() - 1;
        g.nv[a] = (int)Xh[a].size();
    }
    g.W = (g.nv[0] + 31) / 32;
    const size_t nw = (size_t)g.W * g.nv[1] * g.nv[2];
    const size_t nX = Xh[0].size() + Xh[1].size() + Xh[2].size();
    odc_status s = arena_ensure(c, c->A, 3 * al(nX * 4), st);
    if (s != ODC_OK) return s;
    float* dX = (float*)c->A.take(nX * 4);
    int* axis_c = (int*)c->A.take(nX * 4);
    float* axis_f = (float*)c->A.take(nX * 4);
    g.X[0] = dX;
    g.X[1] = dX + Xh[0].size();
    g.X[2] = dX + Xh[0].size() + Xh[1].size();
    for (int a = 0; a < 3; ++a)
        ODC_CK(cudaMemcpyAsync((void*)g.X[a], Xh[a].data(), Xh[a].size() * 4, cudaMemcpyHostToDevice, st));
    uint32_t* bits = bits_g + (size_t)z0 * g.nv[1] * g.W;   // rows of layers z0.. are contiguous
    const int kind = c->res_kind;
    if (kind == ODC_SRC_CSG) {
        launch_csg_grid(g, c->res_prims, c->res_cull, c->res_nprims, bits, st);
    } else if (kind == ODC_SRC_VOXEL) {
        VoxDev vox = c->res_vox;
        vox.iso = prm->iso;
        launch_vox_grid(g, vox, axis_c, axis_f, bits, st);
    } else {
        int64_t nq = 0;
        s = mlp_grid(c->mlp, g, prm->iso, bits, st, &nq, &g_err);
        if (s != ODC_OK) return s;
    }
    (void)nw;
    ODC_CK(cudaGetLastError());
    return ODC_OK;
}

// Ambiguous faces (second-segment entries, the only ones the manifold fix
// marks) of vertex layers [z0, z1) -- and of layer z1 when it is the grid's
// last -- as whole-grid face ids appended to c->gfaces.
static odc_status amb_faces_into(odc_ctx* c, const odc_grid* grid, const uint32_t* bits_g, int z0, int z1,
                                 cudaStream_t st) {
    GridDev g{};
    for (int a = 0; a < 3; ++a) {
        g.n[a] = a < 2 ? grid->res[a] : z1 - z0;
        g.nv[a] = g.n[a] + 1;
    }
    g.W = (g.nv[0] + 31) / 32;
    const size_t nw = (size_t)g.W * g.nv[1] * g.nv[2];
    const uint32_t* bits = bits_g + (size_t)z0 * g.nv[1] * g.W;
    size_t stmp = scan_tmp_elems(nw);
    odc_status s = arena_ensure(c, c->A, al(nw * sizeof(WordInfo)) + 6 * al(nw * 4) + al(stmp * 8) + al(64 * 8), st);
    if (s != ODC_OK) return s;
    WordInfo* wi = (WordInfo*)c->A.take(nw * sizeof(WordInfo));
    uint32_t* ce = (uint32_t*)c->A.take(nw * 4);
    uint32_t* cf = (uint32_t*)c->A.take(nw * 4);
    uint32_t* cc = (uint32_t*)c->A.take(nw * 4);
    uint32_t* ebase = (uint32_t*)c->A.take(nw * 4);
    uint32_t* fbase = (uint32_t*)c->A.take(nw * 4);
    uint32_t* cbase = (uint32_t*)c->A.take(nw * 4);
    void* tmp = c->A.take(stmp * 8);
    uint32_t* dcnt = (uint32_t*)c->A.take(64 * 8);
    ODC_CK(cudaMemsetAsync(dcnt, 0, 64 * 8, st));
    launch_classify(g, bits, wi, ce, cf, cc, st);
    exclusive_scan<uint32_t>(ce, ebase, nw, (uint32_t*)tmp, dcnt + 0, st);
    exclusive_scan<uint32_t>(cf, fbase, nw, (uint32_t*)tmp, dcnt + 1, st);
    exclusive_scan<uint32_t>(cc, cbase, nw, (uint32_t*)tmp, dcnt + 2, st);
    ODC_CK(cudaMemcpyAsync(c->h_cnt, dcnt, 3 * 4, cudaMemcpyDeviceToHost, st));
    ODC_CK(cudaStreamSynchronize(st));
    const uint32_t E = c->h_cnt[0], F = c->h_cnt[1], C = c->h_cnt[2];
    s = arena_ensure(c, c->B, al(E * 4ull) + al(F * 4ull) + al(F) + al(C * 4ull) + al(C) + 1024, st);
    if (s != ODC_OK) return s;
    uint32_t* edges = (uint32_t*)c->B.take(E * 4ull);
    uint32_t* faces = (uint32_t*)c->B.take(F * 4ull);
    uint8_t* slots = (uint8_t*)c->B.take(F);
    uint32_t* cells = (uint32_t*)c->B.take(C * 4ull);
    uint8_t* configs = (uint8_t*)c->B.take(C);
    launch_emit(g, bits, wi, ebase, fbase, cbase, edges, faces, slots, cells, configs, st);
    // keep layers < z1 - z0 (the next window owns layer z1) unless this is the last window
    const bool last = z1 == grid->res[2];
    const uint32_t limit = last ? 0xffffffffu : (uint32_t)(3ull * g.nv[0] * g.nv[1] * (uint32_t)(z1 - z0));
    const uint32_t offset = (uint32_t)(3ull * g.nv[0] * g.nv[1] * (uint32_t)z0);
    s = grow(c, &c->gfaces, &c->gf_cap, (size_t)c->nga + F, st);
    if (s != ODC_OK) return s;
    launch_amb_select(faces, slots, F, limit, offset, c->gfaces, c->nga, (uint32_t*)(dcnt + 32), st);
    ODC_CK(cudaMemcpyAsync(c->h_cnt + 32, dcnt + 32, 4, cudaMemcpyDeviceToHost, st));
    ODC_CK(cudaStreamSynchronize(st));
    ODC_CK(cudaGetLastError());
    c->nga += c->h_cnt[32];
    return ODC_OK;
}

// The manifold fix of the whole grid from its label words: rounds of mark
// all, flip all over the ambiguous faces (as in the extraction), into flips_g.
static odc_status global_fix(odc_ctx* c, const odc_grid* grid, const uint32_t* bits_g, uint32_t* flips_g,
                             cudaStream_t st, int64_t* n_flips) {
    GridDev g{};
    for (int a = 0; a < 3; ++a) {
        g.n[a] = grid->res[a];
        g.nv[a] = g.n[a] + 1;
    }
    g.W = (g.nv[0] + 31) / 32;
    const size_t nw = (size_t)g.W * g.nv[1] * g.nv[2];
    ODC_CK(cudaMemsetAsync(flips_g, 0, 3 * nw * 4, st));
    const uint32_t NA = (uint32_t)c->nga;
    odc_status s = arena_ensure(c, c->B, 2 * al(NA) + 1024, st);
    if (s != ODC_OK) return s;
    uint8_t* slots = (uint8_t*)c->B.take(NA);
    uint8_t* mark = (uint8_t*)c->B.take(NA);
    uint32_t* cnt = (uint32_t*)c->B.take(64);
    if (NA) ODC_CK(cudaMemsetAsync(slots, 1, NA, st));
    int64_t total = 0;
    for (int rounds = 0; NA; ++rounds) {
        ODC_CK(cudaMemsetAsync(cnt, 0, 4, st));
        launch_manifold_mark(g, bits_g, flips_g, c->gfaces, slots, NA, mark, cnt, st);
        ODC_CK(cudaMemcpyAsync(c->h_cnt + 8, cnt, 4, cudaMemcpyDeviceToHost, st));
        ODC_CK(cudaStreamSynchronize(st));
        const uint32_t marked = c->h_cnt[8];
        if (!marked) break;
        launch_manifold_apply(g, flips_g, c->gfaces, mark, NA, st);
        total += marked;
        if (rounds > 64) return fail(ODC_ERR_INTERNAL, "manifold fix did not converge");
    }
    ODC_CK(cudaGetLastError());
    if (n_flips) *n_flips = total;
    return ODC_OK;
}

odc_status odc_extract_slab(odc_ctx* c, const odc_source* src, const odc_grid* grid, const odc_params* prm,
                            const odc_slab* slab, void* cuda_stream, odc_mesh* out, odc_slab_info* info) {
    if (!c || !grid || !prm || !slab || !out || !info) return fail(ODC_ERR_INVALID_ARG, "NULL argument");
    odc_status s = check_source(src);
    if (s == ODC_OK) s = check_slab_grid(grid);
    if (s == ODC_OK) s = check_params(prm);
    if (s != ODC_OK) return s;
    ODC_CK(cudaSetDevice(c->device));
    cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : c->own;
    return slab_extract(c, src, grid, prm, slab, st, out, info);
}

odc_status odc_slab_place(odc_ctx* c, const odc_mesh* m, const odc_slab_info* info, int64_t verts3_base,
                          int64_t case3_base, int64_t tris_base, float* d_verts, int32_t* d_tris, void* cuda_stream) {
    if (!c || !m || !info || !d_verts || !d_tris) return fail(ODC_ERR_INVALID_ARG, "NULL argument");
    if (verts3_base < 0 || case3_base < 0 || tris_base < 0) return fail(ODC_ERR_INVALID_ARG, "negative base");
    if (m->d_tris != (const int32_t*)c->tris || info->verts3_local != (int64_t)c->V3)
        return fail(ODC_ERR_INVALID_ARG, "mesh is not this context's latest slab extraction");
    ODC_CK(cudaSetDevice(c->device));
    cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : c->own;
    float3* dv = (float3*)d_verts;
    return slab_place(c, m, info, verts3_base, case3_base, tris_base, dv, dv + case3_base, (int3*)d_tris, st);
}

odc_status odc_extract_slabbed(odc_ctx* c, const odc_source* src, const odc_grid* grid, const odc_params* prm,
                               int32_t n_slabs, int32_t halo, void* cuda_stream, odc_mesh* out) {
    if (!c || !grid || !prm || !out) return fail(ODC_ERR_INVALID_ARG, "NULL argument");
    odc_status s = check_source(src);
    if (s == ODC_OK) s = check_slab_grid(grid);
    if (s == ODC_OK) s = check_params(prm);
    if (s != ODC_OK) return s;
    if (n_slabs < 1 || n_slabs > grid->res[2]) return fail(ODC_ERR_INVALID_ARG, "n_slabs out of [1, res[2]]");
    ODC_CK(cudaSetDevice(c->device));
    cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : c->own;
    std::memset(out, 0, sizeof(*out));
    // edge points are numbered after every slab's 3D points: staged, and the
    // triangles' edge-point ids held at kMark + index until the count is known
    constexpr int64_t kMark = 1ll << 30;
    odc_source resident{};
    resident.kind = ODC_SRC_RESIDENT;
    if (src->kind != ODC_SRC_RESIDENT) {
        s = upload_source(c, src, st);
        if (s != ODC_OK) return s;
    } else if (c->res_kind < 0) {
        return fail(ODC_ERR_INVALID_ARG, "no resident source on this context");
    }
    auto zcut = [&](int i) { return (int32_t)((int64_t)grid->res[2] * i / n_slabs); };
    // ---- whole-grid topology: label words slab by slab, the ambiguous
    // faces, and one manifold fix over them (its flips chain across slabs)
    const size_t W = (size_t)(grid->res[0] + 32) / 32;
    const size_t nwg = W * (grid->res[1] + 1) * (size_t)(grid->res[2] + 1);
    if ((s = grow(c, &c->gbits, &c->gb_cap, nwg, st)) != ODC_OK ||
        (s = grow(c, &c->gflips, &c->gfl_cap, 3 * nwg, st)) != ODC_OK)
        return s;
    if (!c->sinfo) ODC_CK(cudaMalloc((void**)&c->sinfo, 8 * sizeof(unsigned long long)));
    for (int i = 0; i < n_slabs; ++i)
        if ((s = labels_into(c, grid, prm, zcut(i), zcut(i + 1), c->gbits, st)) != ODC_OK) return s;
    c->nga = 0;
    for (int i = 0; i < n_slabs; ++i)
        if ((s = amb_faces_into(c, grid, c->gbits, zcut(i), zcut(i + 1), st)) != ODC_OK) return s;
    int64_t gflip = 0;
    if ((s = global_fix(c, grid, c->gbits, c->gflips, st, &gflip)) != ODC_OK) return s;
    int64_t V = 0, N = 0, T = 0;
    odc_stats sum{};
    for (int i = 0; i < n_slabs; ++i) {
        odc_slab sl{zcut(i), zcut(i + 1), halo, c->gflips};
        odc_mesh m;
        odc_slab_info in;
        s = slab_extract(c, &resident, grid, prm, &sl, st, &m, &in);
        if (s != ODC_OK) return s;
        if (V + in.verts3_owned >= kMark || N + in.case3_owned >= kMark)
            return fail(ODC_ERR_INVALID_ARG, "merged mesh exceeds 2^30 vertices");
        if ((s = grow(c, &c->sv, &c->sv_cap, (size_t)(V + in.verts3_owned), st)) != ODC_OK ||
            (s = grow(c, &c->sc3, &c->sc3_cap, (size_t)(N + in.case3_owned), st)) != ODC_OK ||
            (s = grow(c, &c->stri, &c->st_cap, (size_t)(T + in.tris_owned), st)) != ODC_OK)
            return s;
        s = slab_place(c, &m, &in, V, kMark + N, T, c->sv, c->sc3 + N, c->stri, st);
        if (s != ODC_OK) return s;
        V += in.verts3_owned;
        N += in.case3_owned;
        T += in.tris_owned;
        const odc_stats& a = m.stats;
        sum.n_edges += a.n_edges; sum.n_face_segs += a.n_face_segs; sum.n_cells += a.n_cells;
        sum.n_verts3 += a.n_verts3; sum.n_case3 += a.n_case3; sum.n_flips += a.n_flips;
        sum.fix_rounds = std::max(sum.fix_rounds, a.fix_rounds);
        sum.n_queries += a.n_queries; sum.n_requeries += a.n_requeries;
        for (int k = 0; k < 8; ++k) sum.stage_ms[k] += a.stage_ms[k];
        sum.mlp_flops += a.mlp_flops; sum.mlp_ms += a.mlp_ms; sum.n_launches += a.n_launches;
        sum.mlp_launches += a.mlp_launches; sum.tc_flops += a.tc_flops; sum.tc_ms += a.tc_ms;
        sum.tc_launches += a.tc_launches; sum.split_flops += a.split_flops; sum.split_ms += a.split_ms;
        sum.split_launches += a.split_launches; sum.n_split += a.n_split;
        sum.h16_flops += a.h16_flops; sum.h16_ms += a.h16_ms; sum.h16_launches += a.h16_launches;
        sum.n_h16 += a.n_h16;
        sum.split_zmargin = a.split_zmargin;
        sum.split_acc_comp = a.split_acc_comp;
        // the next slab's extraction reuses the arenas: the placement must be done
        ODC_CK(cudaStreamSynchronize(st));
    }
    if ((s = grow(c, &c->sv, &c->sv_cap, (size_t)(V + N), st)) != ODC_OK) return s;
    if (N) ODC_CK(cudaMemcpyAsync(c->sv + V, c->sc3, N * 12, cudaMemcpyDeviceToDevice, st));
    launch_slab_fix(c->stri, T, (int)kMark, (int)V, st);
    ODC_CK(cudaStreamSynchronize(st));
    ODC_CK(cudaGetLastError());
    out->n_verts = V + N;
    out->n_tris = T;
    out->d_verts = (const float*)c->sv;
    out->d_tris = (const int32_t*)c->stri;
    out->stats = sum;
    out->stats.n_flips = gflip;
    out->stats.n_launches += 1;
    return ODC_OK;
}

odc_status odc_grid_labels(odc_ctx* c, const odc_source* src, const odc_grid* grid, const odc_params* prm, int32_t z0,
                           int32_t z1, uint32_t* d_bits, void* cuda_stream) {
    if (!c || !grid || !prm || !d_bits) return fail(ODC_ERR_INVALID_ARG, "NULL argument");
    odc_status s = check_source(src);
    if (s == ODC_OK) s = check_slab_grid(grid);
    if (s == ODC_OK) s = check_params(prm);
    if (s != ODC_OK) return s;
    if (z0 < 0 || z1 < z0 || z1 > grid->res[2]) return fail(ODC_ERR_INVALID_ARG, "need 0 <= z0 <= z1 <= res[2]");
    ODC_CK(cudaSetDevice(c->device));
    cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : c->own;
    if (src->kind != ODC_SRC_RESIDENT) {
        s = upload_source(c, src, st);
        if (s != ODC_OK) return s;
    } else if (c->res_kind < 0) {
        return fail(ODC_ERR_INVALID_ARG, "no resident source on this context");
    }
    s = labels_into(c, grid, prm, z0, z1, d_bits, st);
    if (s != ODC_OK) return s;
    ODC_CK(cudaStreamSynchronize(st));
    return ODC_OK;
}

odc_status odc_manifold_flips(odc_ctx* c, const odc_grid* grid, const uint32_t* d_bits, uint32_t* d_flips,
                              int32_t n_chunks, void* cuda_stream, int64_t* n_flips) {
    if (!c || !grid || !d_bits || !d_flips) return fail(ODC_ERR_INVALID_ARG, "NULL argument");
    odc_status s = check_slab_grid(grid);
    if (s != ODC_OK) return s;
    if (n_chunks < 1 || n_chunks > grid->res[2]) return fail(ODC_ERR_INVALID_ARG, "n_chunks out of [1, res[2]]");
    ODC_CK(cudaSetDevice(c->device));
    cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : c->own;
    c->nga = 0;
    for (int i = 0; i < n_chunks; ++i) {
        s = amb_faces_into(c, grid, d_bits, (int32_t)((int64_t)grid->res[2] * i / n_chunks),
                           (int32_t)((int64_t)grid->res[2] * (i + 1) / n_chunks), st);
        if (s != ODC_OK) return s;
    }
    int64_t nf = 0;
    s = global_fix(c, grid, d_bits, d_flips, st, &nf);
    if (s != ODC_OK) return s;
    ODC_CK(cudaStreamSynchronize(st));
    if (n_flips) *n_flips = nf;
    return ODC_OK;
}

odc_status odc_ctx_set_wait_limit(odc_ctx* c, uint64_t ns, const int32_t* d_gate) {
    if (!c) return fail(ODC_ERR_INVALID_ARG, "NULL context");
    c->wait_ns = ns;
    c->gate = d_gate;
    mlp_set_wait_limit(c->mlp, ns, d_gate);
    return ODC_OK;
}

}  // extern "C"

struct odc_batch {
    BatchGroup* g = nullptr;
    int device = 0;
};

extern "C" {

odc_status odc_batch_create(int device, odc_batch** out) {
    if (!out) return fail(ODC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int n = 0;
    ODC_CK(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) return fail(ODC_ERR_INVALID_ARG, "no such CUDA device");
    auto* b = new odc_batch();
    b->device = device;
    odc_status s = batch_create(device, &b->g, &g_err);
    if (s != ODC_OK) {
        delete b;
        return s;
    }
    *out = b;
    return ODC_OK;
}

odc_status odc_batch_destroy(odc_batch* b) {
    if (!b) return ODC_OK;
    batch_destroy(b->g);
    delete b;
    return ODC_OK;
}

odc_status odc_batch_stats(const odc_batch* b, int64_t* rounds, int64_t* calls) {
    if (!b || !rounds || !calls) return fail(ODC_ERR_INVALID_ARG, "NULL argument");
    batch_stats(b->g, rounds, calls);
    return ODC_OK;
}

odc_status odc_ctx_join_batch(odc_ctx* c, odc_batch* b) {
    if (!c) return fail(ODC_ERR_INVALID_ARG, "NULL context");
    if (b && b->device != c->device) return fail(ODC_ERR_INVALID_ARG, "batch and context are on different devices");
    c->batch = b ? b->g : nullptr;
    if (!c->batch) batch_unbind(c->mlp);   // a source uploaded later binds at its upload
    return ODC_OK;
}

odc_status odc_extract_many(odc_batch* b, int32_t n, odc_ctx* const* ctxs, const odc_source* srcs,
                            const odc_grid* grids, const odc_params* prms, odc_mesh* outs, odc_status* statuses) {
    if (n < 0 || (n > 0 && (!ctxs || !srcs || !grids || !prms || !outs || !statuses)))
        return fail(ODC_ERR_INVALID_ARG, "NULL argument");
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i]) return fail(ODC_ERR_INVALID_ARG, "NULL context");
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) return fail(ODC_ERR_INVALID_ARG, "a context appears twice");
        odc_status s = odc_ctx_join_batch(ctxs[i], b);
        if (s != ODC_OK) return s;
    }
    std::vector<std::string> errs(n);
    std::vector<std::thread> th;
    th.reserve(n);
    for (int i = 0; i < n; ++i)
        th.emplace_back([&, i] {
            statuses[i] = odc_extract(ctxs[i], &srcs[i], &grids[i], &prms[i], nullptr, &outs[i]);
            if (statuses[i] != ODC_OK) errs[i] = odc_last_error();
        });
    for (auto& t : th) t.join();
    for (int i = 0; i < n; ++i)
        if (statuses[i] != ODC_OK) return fail(statuses[i], "shape " + std::to_string(i) + ": " + errs[i]);
    return ODC_OK;
}

odc_status odc_ctx_memory(odc_ctx* c, size_t* bytes) {
    if (!c || !bytes) return fail(ODC_ERR_INVALID_ARG, "NULL argument");
    *bytes = c->A.cap + c->B.cap + c->S.cap + c->extra_bytes() + mlp_device_bytes(c->mlp);
    return ODC_OK;
}

odc_status odc_source_upload(odc_ctx* c, const odc_source* src) {
    if (!c) return fail(ODC_ERR_INVALID_ARG, "NULL context");
    if (src && src->kind == ODC_SRC_RESIDENT) return fail(ODC_ERR_INVALID_ARG, "cannot upload a resident source");
    odc_status s = check_source(src);
    if (s != ODC_OK) return s;
    ODC_CK(cudaSetDevice(c->device));
    s = upload_source(c, src, c->own);
    if (s != ODC_OK) return s;
    ODC_CK(cudaStreamSynchronize(c->own));
    return ODC_OK;
}

odc_status odc_mesh_copy(odc_ctx* c, const odc_mesh* m, float* verts, int32_t* tris, int dst_on_device) {
    if (!c || !m) return fail(ODC_ERR_INVALID_ARG, "NULL argument");
    ODC_CK(cudaSetDevice(c->device));
    cudaMemcpyKind k = dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (verts && m->n_verts) ODC_CK(cudaMemcpyAsync(verts, m->d_verts, m->n_verts * 12, k, c->own));
    if (tris && m->n_tris) ODC_CK(cudaMemcpyAsync(tris, m->d_tris, m->n_tris * 12, k, c->own));
    ODC_CK(cudaStreamSynchronize(c->own));
    return ODC_OK;
}

odc_status odc_mesh_release(odc_ctx* c, odc_mesh* m) {
    if (!c || !m) return fail(ODC_ERR_INVALID_ARG, "NULL argument");
    m->d_verts = nullptr;
    m->d_tris = nullptr;
    m->n_verts = m->n_tris = 0;
    return ODC_OK;
}

odc_status odc_debug_copy(odc_ctx* c, int what, void* dst, size_t max_bytes, int64_t* count, int32_t* elem_bytes) {
    if (!c || !count || !elem_bytes) return fail(ODC_ERR_INVALID_ARG, "NULL argument");
    const void* p = nullptr;
    int64_t n = 0;
    int eb = 0;
    std::vector<uint32_t> flipped;
    switch (what) {
        case ODC_DBG_LABELS: p = c->bits; n = (int64_t)c->nw; eb = 4; break;
        case ODC_DBG_EDGES: p = c->edges; n = c->E; eb = 4; break;
        case ODC_DBG_T: p = c->T; n = c->E; eb = 4; break;
        case ODC_DBG_FACES: p = c->faces; n = c->F; eb = 4; break;
        case ODC_DBG_SLOTS: p = c->slots; n = c->F; eb = 1; break;
        case ODC_DBG_FACE_PTS: p = c->pf; n = c->F; eb = 16; break;
        case ODC_DBG_FACE_FLAGS: p = c->fflags; n = c->F; eb = 1; break;
        case ODC_DBG_CELLS: p = c->cells; n = c->C; eb = 4; break;
        case ODC_DBG_CONFIGS: p = c->configs; n = c->C; eb = 1; break;
        case ODC_DBG_CYCLES: p = c->cycles; n = c->C; eb = 8; break;
        case ODC_DBG_VLOCAL: p = c->vlocal; n = c->V3; eb = 12; break;
        case ODC_DBG_QCASE: p = c->qcase; n = c->E; eb = 1; break;
        case ODC_DBG_SEARCH: p = c->dec; n = c->F; eb = (int)sizeof(FaceDecisions); break;
        case ODC_DBG_FLIPS: {
            // expand the flip bit planes into sorted face ids
            std::vector<uint32_t> h(3 * c->nw);
            if (c->nw) {
                ODC_CK(cudaSetDevice(c->device));
                ODC_CK(cudaMemcpy(h.data(), c->flips, h.size() * 4, cudaMemcpyDeviceToHost));
            }
            const GridDev& g = c->g;
            for (int z = 0; z < g.nv[2]; ++z)
                for (int y = 0; y < g.nv[1]; ++y)
                    for (int w = 0; w < g.W; ++w)
                        for (int a = 0; a < 3; ++a) {
                            uint32_t bitsw = h[(((size_t)a * g.nv[2] + z) * g.nv[1] + y) * g.W + w];
                            while (bitsw) {
                                int l = __builtin_ctz(bitsw);
                                bitsw &= bitsw - 1;
                                uint32_t v = (uint32_t)(w * 32 + l) + (uint32_t)g.nv[0] * ((uint32_t)y + (uint32_t)g.nv[1] * z);
                                flipped.push_back(3u * v + a);
                            }
                        }
            std::sort(flipped.begin(), flipped.end());
            *count = (int64_t)flipped.size();
            *elem_bytes = 4;
            if (dst) std::memcpy(dst, flipped.data(), std::min(max_bytes, flipped.size() * 4));
            return ODC_OK;
        }
        default: return fail(ODC_ERR_INVALID_ARG, "unknown debug buffer");
    }
    *count = n;
    *elem_bytes = eb;
    if (dst && p && n) {
        ODC_CK(cudaSetDevice(c->device));
        ODC_CK(cudaMemcpy(dst, p, std::min(max_bytes, (size_t)n * eb), cudaMemcpyDeviceToHost));
    }
    return ODC_OK;
}

odc_status odc_mesh_quality(odc_ctx* c, const odc_mesh* m, float iso, int64_t n_samples, uint64_t seed,
                            int32_t what, odc_quality* out) {
    if (!c || !m || !out || n_samples < 0) return fail(ODC_ERR_INVALID_ARG, "NULL argument");
    if ((m->n_verts && !m->d_verts) || (m->n_tris && !m->d_tris)) return fail(ODC_ERR_INVALID_ARG, "mesh without buffers");
    if ((what & ODC_Q_OCC) && c->res_kind < 0) return fail(ODC_ERR_INVALID_ARG, "no resident source on this context");
    ODC_CK(cudaSetDevice(c->device));
    std::memset(out, 0, sizeof(*out));
    MlpState* mlp = c->res_kind == ODC_SRC_MLP ? c->mlp : nullptr;
    const PrimDev* prims = c->res_kind == ODC_SRC_CSG ? c->res_prims : nullptr;
    const VoxDev* vox = c->res_kind == ODC_SRC_VOXEL ? &c->res_vox : nullptr;
    odc_status s = mesh_quality(mlp, prims, c->res_nprims, vox, (const float3*)m->d_verts, m->n_verts,
                                (const int3*)m->d_tris, m->n_tris, iso, n_samples, seed, what, c->own, out, &g_err);
    return s == ODC_OK ? s : fail(s, g_err);
}

odc_status odc_eval_points(odc_ctx* c, const odc_source* src, const float* points, int64_t n, float iso,
                           int precision, uint8_t* labels, float* logits) {
    if (!c || !points || !labels || n < 0) return fail(ODC_ERR_INVALID_ARG, "NULL argument");
    odc_status s = check_source(src);
    if (s != ODC_OK) return s;
    ODC_CK(cudaSetDevice(c->device));
    cudaStream_t st = c->own;
    if (n == 0) return ODC_OK;
    size_t need = al(n * 12) + al(n) + al(n * 4);
    if (src->kind != ODC_SRC_RESIDENT) {
        s = upload_source(c, src, st);
        if (s != ODC_OK) return s;
    } else if (c->res_kind < 0) {
        return fail(ODC_ERR_INVALID_ARG, "no resident source on this context");
    }
    PrimDev* d_prims = c->res_prims;
    float4* d_cull = c->res_cull;
    s = arena_ensure(c, c->B, need, st);
    if (s != ODC_OK) return s;
    float3* dp = (float3*)c->B.take(n * 12);
    uint8_t* dl = (uint8_t*)c->B.take(n);
    float* dz = (float*)c->B.take(n * 4);
    c->E = c->F = c->C = c->V3 = 0;   // the B arena no longer holds an extract
    ODC_CK(cudaMemcpyAsync(dp, points, n * 12, cudaMemcpyHostToDevice, st));
    if (c->res_kind == ODC_SRC_CSG) {
        launch_csg_points(d_prims, d_cull, c->res_nprims, dp, n, dl, st);
    } else if (c->res_kind == ODC_SRC_VOXEL) {
        VoxDev vox = c->res_vox;
        vox.iso = iso;
        launch_vox_points(vox, dp, n, dl, st);
    } else {
        mlp_set_wait_limit(c->mlp, c->wait_ns, c->gate);
        s = mlp_points(c->mlp, dp, n, iso, precision, dl, dz, st, &g_err);
        if (s != ODC_OK) return s;
    }
    ODC_CK(cudaGetLastError());
    ODC_CK(cudaMemcpyAsync(labels, dl, n, cudaMemcpyDeviceToHost, st));
    if (logits && c->res_kind == ODC_SRC_MLP) ODC_CK(cudaMemcpyAsync(logits, dz, n * 4, cudaMemcpyDeviceToHost, st));
    ODC_CK(cudaStreamSynchronize(st));
    return ODC_OK;
}

}  // extern "C"
