// quality.cu -- the mesh-quality measures of the paper's evaluation (Sec. 6.1
// "Evaluation Metrics") on the device, for a mesh in device memory:
//
//   * |phi - iso| at n points sampled uniformly by area on the mesh (Sec. 6.1
//     samples 2M points per shape), phi = sigmoid of the FP32 logit of the
//     context's MLP source.  Sample j draws three values 3j .. 3j + 2 of a
//     counter-based SplitMix64 stream (Steele, Lea and Flood, OOPSLA 2014):
//     the triangle by inverting the area CDF, then barycentric coordinates
//     (1 - sqrt u1, sqrt u1 (1 - u2), sqrt u1 u2).
//   * Manifoldness: every directed edge used once and its reverse once (a
//     hash table of directed edges), and the triangle fan around every vertex
//     a single cycle (a walk around each vertex through the table); Euler
//     characteristic V - E + F.
//   * Self-intersections: pairs of triangles whose closed sets meet, when
//     they share no vertex, or whose edge opposite their one shared vertex
//     meets the other triangle; triangles sharing an edge never count.
//     Candidate pairs come from a uniform grid (each triangle binned into
//     the cells its bounding box covers, a pair tested only in the lowest
//     cell common to both); triangles covering too many cells are tested
//     against all others.  Predicates are FP64 orientation tests, in
//     plain IEEE arithmetic (this unit is compiled without FMA contraction).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/odc.h"
#include "csg_psi.cuh"
#include "kernels.h"
#include "mlp.h"
#include "odc_internal.h"

namespace odc {

namespace {

constexpr unsigned long long kEmpty = ~0ull;
constexpr int kMaxCellsPerTri = 64;        // larger triangles go to the all-pairs list
constexpr uint64_t kMaxCells = 1ull << 24;  // binning grid size cap
constexpr int kMaxWalk = 1 << 16;          // fan walk bound (a valid fan is shorter)

#define Q_CK(call)                                                                           \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) { *err = std::string(#call) + ": " + cudaGetErrorString(e_); \
                                 return ODC_ERR_CUDA; }                                      \
    } while (0)

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long seed, unsigned long long i) {
    unsigned long long z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ double unit(unsigned long long r) { return (double)(r >> 11) * 0x1.0p-53; }

struct D3 {
    double x, y, z;
};
__device__ __forceinline__ D3 d3(float3 p) { return D3{(double)p.x, (double)p.y, (double)p.z}; }
__device__ __forceinline__ D3 sub(D3 a, D3 b) { return D3{a.x - b.x, a.y - b.y, a.z - b.z}; }

// ------------------------------------------------------------ sampling
__global__ void k_areas(const float3* __restrict__ v, const int3* __restrict__ t, int64_t nt, double* __restrict__ area) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    int3 f = t[i];
    D3 p0 = d3(v[f.x]), e1 = sub(d3(v[f.y]), p0), e2 = sub(d3(v[f.z]), p0);
    double cx = e1.y * e2.z - e1.z * e2.y, cy = e1.z * e2.x - e1.x * e2.z, cz = e1.x * e2.y - e1.y * e2.x;
    area[i] = 0.5 * sqrt(cx * cx + cy * cy + cz * cz);
}

__global__ void k_samples(const float3* __restrict__ v, const int3* __restrict__ t, int64_t nt,
                          const double* __restrict__ excl, const double* __restrict__ area,
                          const double* __restrict__ total, int64_t n, unsigned long long seed,
                          float3* __restrict__ out) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double u0 = unit(splitmix64(seed, 3ull * j)), u1 = unit(splitmix64(seed, 3ull * j + 1)),
           u2 = unit(splitmix64(seed, 3ull * j + 2));
    double target = u0 * *total;
    // first triangle whose inclusive CDF exceeds target
    int64_t lo = 0, hi = nt - 1;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (excl[mid] + area[mid] > target) hi = mid; else lo = mid + 1;
    }
    int3 f = t[lo];
    double s = sqrt(u1);
    double b0 = 1.0 - s, b1 = s * (1.0 - u2), b2 = s * u2;
    D3 p0 = d3(v[f.x]), p1 = d3(v[f.y]), p2 = d3(v[f.z]);
    out[j] = make_float3((float)((b0 * p0.x + b1 * p1.x) + b2 * p2.x), (float)((b0 * p0.y + b1 * p1.y) + b2 * p2.y),
                         (float)((b0 * p0.z + b1 * p1.z) + b2 * p2.z));
}

__device__ __forceinline__ void atomic_max_pos(double* a, double v) {
    unsigned long long* p = (unsigned long long*)a;
    unsigned long long x = (unsigned long long)__double_as_longlong(v), old = *p;
    while (__longlong_as_double((long long)old) < v) {
        unsigned long long prev = atomicCAS(p, old, x);
        if (prev == old) break;
        old = prev;
    }
}

__device__ __forceinline__ void block_sum_max(double d, double* acc) {
    __shared__ double ssum[8], smax[8];
    double s = d, m = d;
    for (int o = 16; o; o >>= 1) {
        s += __shfl_down_sync(0xffffffffu, s, o);
        m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    }
    int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { ssum[w] = s; smax[w] = m; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double S = 0.0, M = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { S += ssum[k]; M = fmax(M, smax[k]); }
        atomicAdd(&acc[0], S);
        atomic_max_pos(&acc[1], M);
    }
}

__global__ void k_deviation(const float* __restrict__ z, int64_t n, double iso, double* __restrict__ acc) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double d = 0.0;
    if (i < n) d = fabs(1.0 / (1.0 + exp(-(double)z[i])) - iso);
    block_sum_max(d, acc);
}

// |phi - iso| of a voxel volume: trilinear interpolation in FP64 (clamped).
__global__ void k_vox_deviation(const float3* __restrict__ pts, int64_t n, VoxDev d, double iso,
                                double* __restrict__ acc) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double dev = 0.0;
    if (i < n) {
        const float3 p = pts[i];
        const double pc[3] = {(double)p.x, (double)p.y, (double)p.z};
        int c[3];
        double f[3];
        for (int a = 0; a < 3; ++a) {
            const double lo = (double)d.lo[a], rng = (double)d.rng_hi[a] + (double)d.rng_lo[a];
            double u = (pc[a] - lo) / rng * (double)(d.dims[a] - 1);
            u = fmin(fmax(u, 0.0), (double)(d.dims[a] - 1));
            c[a] = min((int)floor(u), d.dims[a] - 2);
            f[a] = u - (double)c[a];
        }
        const size_t sy = (size_t)d.dims[0], sz = (size_t)d.dims[0] * d.dims[1];
        const float* b = d.v + (size_t)c[2] * sz + (size_t)c[1] * sy + (size_t)c[0];
        auto L = [](double x, double y, double t) { return x + (y - x) * t; };
        const double c00 = L(b[0], b[1], f[0]), c10 = L(b[sy], b[sy + 1], f[0]);
        const double c01 = L(b[sz], b[sz + 1], f[0]), c11 = L(b[sz + sy], b[sz + sy + 1], f[0]);
        dev = fabs(L(L(c00, c10, f[1]), L(c01, c11, f[1]), f[2]) - iso);
    }
    block_sum_max(dev, acc);
}

// First-order distance |psi| / |grad psi| of the CSG surface (FP64).
__global__ void k_csg_distance(const float3* __restrict__ pts, int64_t n, const PrimDev* __restrict__ prims,
                               int n_prims, double* __restrict__ acc) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double d = 0.0;
    if (i < n) {
        float3 p = pts[i];
        double gr[3];
        double psi = csg_psi<double>(prims, n_prims, (double)p.x, (double)p.y, (double)p.z, gr);
        double gn = sqrt(gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2]);
        d = gn > 0.0 ? fabs(psi) / gn : fabs(psi);
    }
    block_sum_max(d, acc);
}

__global__ void k_check_indices(const int3* __restrict__ t, int64_t nt, int64_t nv, unsigned long long* __restrict__ bad) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    int3 f = t[i];
    if (f.x < 0 || f.y < 0 || f.z < 0 || f.x >= nv || f.y >= nv || f.z >= nv) atomicAdd(bad, 1ull);
}

// ------------------------------------------------------------ manifold
__device__ __forceinline__ unsigned long long he_hash(unsigned long long k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    return k;
}

struct HeTable {
    unsigned long long* key;
    uint32_t* cnt;
    uint32_t* third;
    unsigned long long mask;
};

__device__ __forceinline__ int64_t he_find(const HeTable& H, unsigned long long k) {
    unsigned long long h = he_hash(k) & H.mask;
    for (unsigned long long probe = 0; probe <= H.mask; ++probe) {
        unsigned long long cur = H.key[h];
        if (cur == k) return (int64_t)h;
        if (cur == kEmpty) return -1;
        h = (h + 1) & H.mask;
    }
    return -1;
}

// Directed edges of every triangle; degenerate triangles (a repeated vertex)
// are counted and not inserted.  Vertex degrees and one incident triangle.
__global__ void k_he_insert(const int3* __restrict__ t, int64_t nt, HeTable H, uint32_t* __restrict__ deg,
                            uint32_t* __restrict__ start, unsigned long long* __restrict__ counters) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    int3 f = t[i];
    int c[3] = {f.x, f.y, f.z};
    if (c[0] == c[1] || c[1] == c[2] || c[0] == c[2]) {
        atomicAdd(&counters[0], 1ull);
        return;
    }
    for (int r = 0; r < 3; ++r) {
        uint32_t u = (uint32_t)c[r], w = (uint32_t)c[(r + 1) % 3], o = (uint32_t)c[(r + 2) % 3];
        atomicAdd(&deg[u], 1u);
        start[u] = (uint32_t)i;
        unsigned long long k = ((unsigned long long)u << 32) | w;
        unsigned long long h = he_hash(k) & H.mask;
        for (unsigned long long probe = 0; probe <= H.mask; ++probe) {
            unsigned long long prev = atomicCAS(&H.key[h], kEmpty, k);
            if (prev == kEmpty || prev == k) {
                atomicAdd(&H.cnt[h], 1u);
                H.third[h] = o;
                break;
            }
            h = (h + 1) & H.mask;
        }
    }
}

// Per table slot: a directed edge used more than once, or whose reverse is
// not used exactly once, is bad; undirected edges counted once.
__global__ void k_he_check(HeTable H, unsigned long long* __restrict__ counters) {
    unsigned long long h = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (h > H.mask) return;
    unsigned long long k = H.key[h];
    if (k == kEmpty) return;
    uint32_t u = (uint32_t)(k >> 32), w = (uint32_t)k;
    int64_t r = he_find(H, ((unsigned long long)w << 32) | u);
    uint32_t n = H.cnt[h], rn = r >= 0 ? H.cnt[r] : 0u;
    if (n != 1u || rn != 1u) atomicAdd(&counters[1], (unsigned long long)n);
    if (u < w || r < 0) atomicAdd(&counters[2], 1ull);
}

// Fan around each used vertex v: start at an incident triangle (v, a, b) and
// follow v->b to the triangle (v, b, w) until a is reached; a single cycle
// takes exactly deg(v) steps.
__global__ void k_fans(const int3* __restrict__ t, int64_t nv, HeTable H, const uint32_t* __restrict__ deg,
                       const uint32_t* __restrict__ start, unsigned long long* __restrict__ counters) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    uint32_t d = deg[v];
    if (!d) return;
    atomicAdd(&counters[3], 1ull);
    int3 f = t[start[v]];
    uint32_t a, b;
    if ((uint32_t)f.x == (uint32_t)v) { a = f.y; b = f.z; }
    else if ((uint32_t)f.y == (uint32_t)v) { a = f.z; b = f.x; }
    else { a = f.x; b = f.y; }
    uint32_t cur = b, steps = 1;
    bool ok = true;
    while (cur != a) {
        int64_t s = he_find(H, ((unsigned long long)v << 32) | cur);
        if (s < 0 || H.cnt[s] != 1u || steps > d || steps > (uint32_t)kMaxWalk) { ok = false; break; }
        cur = H.third[s];
        ++steps;
    }
    if (!ok || steps != d) atomicAdd(&counters[4], 1ull);
}

// ------------------------------------------------------------ self-intersection predicates
__device__ __forceinline__ double orient3(D3 a, D3 b, D3 c, D3 d) {
    D3 u = sub(b, a), v = sub(c, a), w = sub(d, a);
    return u.x * (v.y * w.z - v.z * w.y) + u.y * (v.z * w.x - v.x * w.z) + u.z * (v.x * w.y - v.y * w.x);
}
struct D2 {
    double x, y;
};
__device__ __forceinline__ double orient2(D2 a, D2 b, D2 c) { return (b.x - a.x) * (c.y - a.y) - (b.y - a.y) * (c.x - a.x); }
__device__ __forceinline__ bool on_seg2(D2 s0, D2 s1, D2 r, double d) {
    return d == 0.0 && fmin(s0.x, s1.x) <= r.x && r.x <= fmax(s0.x, s1.x) && fmin(s0.y, s1.y) <= r.y &&
           r.y <= fmax(s0.y, s1.y);
}
__device__ __forceinline__ bool seg_seg2(D2 p, D2 q, D2 a, D2 b) {
    double d1 = orient2(a, b, p), d2 = orient2(a, b, q), d3v = orient2(p, q, a), d4 = orient2(p, q, b);
    bool proper = ((d1 > 0 && d2 < 0) || (d1 < 0 && d2 > 0)) && ((d3v > 0 && d4 < 0) || (d3v < 0 && d4 > 0));
    return proper || on_seg2(a, b, p, d1) || on_seg2(a, b, q, d2) || on_seg2(p, q, a, d3v) || on_seg2(p, q, b, d4);
}
__device__ __forceinline__ bool in_tri2(D2 p, D2 a, D2 b, D2 c) {
    double s1 = orient2(a, b, p), s2 = orient2(b, c, p), s3 = orient2(c, a, p);
    return (s1 >= 0 && s2 >= 0 && s3 >= 0) || (s1 <= 0 && s2 <= 0 && s3 <= 0);
}
__device__ __forceinline__ D2 drop(D3 p, int ax) {
    return ax == 0 ? D2{p.y, p.z} : (ax == 1 ? D2{p.x, p.z} : D2{p.x, p.y});
}

// Closed segment pq meets closed triangle abc.
__device__ bool seg_tri(D3 p, D3 q, D3 a, D3 b, D3 c) {
    double d0 = orient3(a, b, c, p), d1 = orient3(a, b, c, q);
    if (d0 == 0.0 && d1 == 0.0) {
        D3 e1 = sub(b, a), e2 = sub(c, a);
        double nx = fabs(e1.y * e2.z - e1.z * e2.y), ny = fabs(e1.z * e2.x - e1.x * e2.z),
               nz = fabs(e1.x * e2.y - e1.y * e2.x);
        int ax = 0;
        double best = nx;
        if (ny > best) { ax = 1; best = ny; }
        if (nz > best) ax = 2;
        D2 P = drop(p, ax), Q = drop(q, ax), A = drop(a, ax), B = drop(b, ax), C = drop(c, ax);
        return in_tri2(P, A, B, C) || in_tri2(Q, A, B, C) || seg_seg2(P, Q, A, B) || seg_seg2(P, Q, B, C) ||
               seg_seg2(P, Q, C, A);
    }
    if ((d0 > 0 && d1 > 0) || (d0 < 0 && d1 < 0)) return false;
    double s1 = orient3(p, q, a, b), s2 = orient3(p, q, b, c), s3 = orient3(p, q, c, a);
    return (s1 >= 0 && s2 >= 0 && s3 >= 0) || (s1 <= 0 && s2 <= 0 && s3 <= 0);
}

__device__ bool tri_pair_hits(const float3* __restrict__ v, int3 fa, int3 fb) {
    int A[3] = {fa.x, fa.y, fa.z}, B[3] = {fb.x, fb.y, fb.z};
    int ns = 0, sa = -1, sb = -1;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            if (A[i] == B[j]) { ++ns; sa = i; sb = j; }
    if (ns >= 2) return false;
    D3 P[3] = {d3(v[A[0]]), d3(v[A[1]]), d3(v[A[2]])}, R[3] = {d3(v[B[0]]), d3(v[B[1]]), d3(v[B[2]])};
    if (ns == 0) {
        for (int e = 0; e < 3; ++e)
            if (seg_tri(P[e], P[(e + 1) % 3], R[0], R[1], R[2])) return true;
        for (int e = 0; e < 3; ++e)
            if (seg_tri(R[e], R[(e + 1) % 3], P[0], P[1], P[2])) return true;
        return false;
    }
    return seg_tri(P[(sa + 1) % 3], P[(sa + 2) % 3], R[0], R[1], R[2]) ||
           seg_tri(R[(sb + 1) % 3], R[(sb + 2) % 3], P[0], P[1], P[2]);
}

__device__ __forceinline__ bool boxes_meet(const float3* v, int3 fa, int3 fb) {
    float3 a0 = v[fa.x], a1 = v[fa.y], a2 = v[fa.z], b0 = v[fb.x], b1 = v[fb.y], b2 = v[fb.z];
    float alx = fminf(a0.x, fminf(a1.x, a2.x)), ahx = fmaxf(a0.x, fmaxf(a1.x, a2.x));
    float aly = fminf(a0.y, fminf(a1.y, a2.y)), ahy = fmaxf(a0.y, fmaxf(a1.y, a2.y));
    float alz = fminf(a0.z, fminf(a1.z, a2.z)), ahz = fmaxf(a0.z, fmaxf(a1.z, a2.z));
    float blx = fminf(b0.x, fminf(b1.x, b2.x)), bhx = fmaxf(b0.x, fmaxf(b1.x, b2.x));
    float bly = fminf(b0.y, fminf(b1.y, b2.y)), bhy = fmaxf(b0.y, fmaxf(b1.y, b2.y));
    float blz = fminf(b0.z, fminf(b1.z, b2.z)), bhz = fmaxf(b0.z, fmaxf(b1.z, b2.z));
    return blx <= ahx && alx <= bhx && bly <= ahy && aly <= bhy && blz <= ahz && alz <= bhz;
}

// ------------------------------------------------------------ binning
struct Bins {
    float lo[3];
    float inv;        // 1 / cell size
    int dim[3];
};

__device__ __forceinline__ void cell_range(const Bins& b, const float3* v, int3 f, int lo[3], int hi[3]) {
    float3 p[3] = {v[f.x], v[f.y], v[f.z]};
    float mn[3] = {fminf(p[0].x, fminf(p[1].x, p[2].x)), fminf(p[0].y, fminf(p[1].y, p[2].y)),
                   fminf(p[0].z, fminf(p[1].z, p[2].z))};
    float mx[3] = {fmaxf(p[0].x, fmaxf(p[1].x, p[2].x)), fmaxf(p[0].y, fmaxf(p[1].y, p[2].y)),
                   fmaxf(p[0].z, fmaxf(p[1].z, p[2].z))};
    for (int a = 0; a < 3; ++a) {
        lo[a] = min(max((int)floorf((mn[a] - b.lo[a]) * b.inv), 0), b.dim[a] - 1);
        hi[a] = min(max((int)floorf((mx[a] - b.lo[a]) * b.inv), 0), b.dim[a] - 1);
    }
}

__global__ void k_bin_count(const float3* __restrict__ v, const int3* __restrict__ t, int64_t nt, Bins b,
                            uint32_t* __restrict__ count, int* __restrict__ big, uint32_t* __restrict__ nbig) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    int lo[3], hi[3];
    cell_range(b, v, t[i], lo, hi);
    int64_t nc = (int64_t)(hi[0] - lo[0] + 1) * (hi[1] - lo[1] + 1) * (hi[2] - lo[2] + 1);
    if (nc > kMaxCellsPerTri) {
        big[atomicAdd(nbig, 1u)] = (int)i;
        return;
    }
    for (int z = lo[2]; z <= hi[2]; ++z)
        for (int y = lo[1]; y <= hi[1]; ++y)
            for (int x = lo[0]; x <= hi[0]; ++x)
                atomicAdd(&count[((size_t)z * b.dim[1] + y) * b.dim[0] + x], 1u);
}

__global__ void k_bin_fill(const float3* __restrict__ v, const int3* __restrict__ t, int64_t nt, Bins b,
                           const uint32_t* __restrict__ off, uint32_t* __restrict__ cursor,
                           uint32_t* __restrict__ list, uint32_t* __restrict__ list_cell) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    int lo[3], hi[3];
    cell_range(b, v, t[i], lo, hi);
    int64_t nc = (int64_t)(hi[0] - lo[0] + 1) * (hi[1] - lo[1] + 1) * (hi[2] - lo[2] + 1);
    if (nc > kMaxCellsPerTri) return;
    for (int z = lo[2]; z <= hi[2]; ++z)
        for (int y = lo[1]; y <= hi[1]; ++y)
            for (int x = lo[0]; x <= hi[0]; ++x) {
                size_t c = ((size_t)z * b.dim[1] + y) * b.dim[0] + x;
                uint32_t k = off[c] + atomicAdd(&cursor[c], 1u);
                list[k] = (uint32_t)i;
                list_cell[k] = (uint32_t)c;
            }
}

// Entry k of the binned list against the later entries of its cell; a pair
// is tested only in the lowest cell common to both bounding-box ranges.
__global__ void k_si_cells(const float3* __restrict__ v, const int3* __restrict__ t, Bins b, uint32_t nlist,
                           const uint32_t* __restrict__ list, const uint32_t* __restrict__ list_cell,
                           const uint32_t* __restrict__ off, const uint32_t* __restrict__ count,
                           uint8_t* __restrict__ flag, unsigned long long* __restrict__ counters) {
    uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nlist) return;
    uint32_t c = list_cell[k];
    uint32_t end = off[c] + count[c];
    uint32_t ia = list[k];
    int3 fa = t[ia];
    int alo[3], ahi[3];
    cell_range(b, v, fa, alo, ahi);
    for (uint32_t m = k + 1; m < end; ++m) {
        uint32_t ib = list[m];
        int3 fb = t[ib];
        int blo[3], bhi[3];
        cell_range(b, v, fb, blo, bhi);
        size_t home = ((size_t)max(alo[2], blo[2]) * b.dim[1] + max(alo[1], blo[1])) * b.dim[0] + max(alo[0], blo[0]);
        if (home != c) continue;
        if (!boxes_meet(v, fa, fb)) continue;
        if (tri_pair_hits(v, fa, fb)) {
            atomicAdd(&counters[5], 1ull);
            flag[ia] = 1;
            flag[ib] = 1;
        }
    }
}

// Triangles too large for the grid: one block each, against every triangle
// (pairs of two large triangles once, from the lower index).
__global__ void k_si_big(const float3* __restrict__ v, const int3* __restrict__ t, int64_t nt,
                         const int* __restrict__ big, const uint32_t* __restrict__ nbig,
                         const uint8_t* __restrict__ is_big, uint8_t* __restrict__ flag,
                         unsigned long long* __restrict__ counters) {
    if (blockIdx.x >= *nbig) return;
    int ia = big[blockIdx.x];
    int3 fa = t[ia];
    for (int64_t j = threadIdx.x; j < nt; j += blockDim.x) {
        if (j == ia || (is_big[j] && j < ia)) continue;
        int3 fb = t[j];
        if (!boxes_meet(v, fa, fb)) continue;
        if (tri_pair_hits(v, fa, fb)) {
            atomicAdd(&counters[5], 1ull);
            flag[ia] = 1;
            flag[j] = 1;
        }
    }
}

__global__ void k_mark_big(const int* __restrict__ big, const uint32_t* __restrict__ nbig, uint8_t* __restrict__ is_big) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < *nbig) is_big[big[i]] = 1;
}

__global__ void k_count_flags(const uint8_t* __restrict__ flag, int64_t n, unsigned long long* __restrict__ counters) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool f = i < n && flag[i];
    unsigned b = __ballot_sync(0xffffffffu, f);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(&counters[6], (unsigned long long)__popc(b));
}

}  // namespace

static inline unsigned nb(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

odc_status mesh_quality(MlpState* mlp, const PrimDev* prims, int n_prims, const VoxDev* vox, const float3* v,
                        int64_t nv, const int3* t,
                        int64_t nt, float iso, int64_t n_samples, uint64_t seed, int what, cudaStream_t s,
                        odc_quality* out, std::string* err) {
    out->n_tris = nt;
    out->n_samples = 0;
    out->occ_dev_mean = out->occ_dev_max = NAN;
    out->dist_mean = out->dist_max = NAN;
    unsigned long long* dcnt;
    Q_CK(cudaMallocAsync((void**)&dcnt, 16 * sizeof(unsigned long long), s));
    Q_CK(cudaMemsetAsync(dcnt, 0, 16 * sizeof(unsigned long long), s));
    unsigned long long hc[16] = {};
    void* to_free[16] = {};
    int nfree = 0;
    auto alloc = [&](size_t bytes, void** p) -> odc_status {
        cudaError_t e = cudaMallocAsync(p, std::max<size_t>(bytes, 16), s);
        if (e != cudaSuccess) { *err = std::string("quality scratch: ") + cudaGetErrorString(e); return ODC_ERR_OOM; }
        to_free[nfree++] = *p;
        return ODC_OK;
    };
    odc_status r = ODC_OK;
    if (nt > 0) {   // every index must name a vertex before any kernel reads through it
        k_check_indices<<<nb(nt), 256, 0, s>>>(t, nt, nv, dcnt + 15); note_launch();
        unsigned long long nbad = 0;
        Q_CK(cudaMemcpyAsync(&nbad, dcnt + 15, 8, cudaMemcpyDeviceToHost, s));
        Q_CK(cudaStreamSynchronize(s));
        if (nbad) {
            cudaFreeAsync(dcnt, s);
            *err = std::to_string(nbad) + " triangles index vertices outside [0, n_verts)";
            return ODC_ERR_INVALID_ARG;
        }
    }
    do {
        // ---- occupancy deviation on area-uniform samples
        if ((what & ODC_Q_OCC) && (mlp || prims || vox) && nt > 0 && n_samples > 0) {
            double *area, *excl, *acc;
            float3* pts;
            float* z;
            size_t stmp = scan_tmp_elems((size_t)nt);
            void *pa, *pe, *pt, *pp, *pz, *pacc;
            if ((r = alloc(nt * 8, &pa)) || (r = alloc(nt * 8, &pe)) || (r = alloc(stmp * 8 + 16, &pt)) ||
                (r = alloc(n_samples * 12, &pp)) || (r = alloc(n_samples * 4, &pz)) || (r = alloc(32, &pacc)))
                break;
            area = (double*)pa; excl = (double*)pe; pts = (float3*)pp; z = (float*)pz; acc = (double*)pacc;
            double* tmp = (double*)pt;
            double* total = tmp + stmp;
            k_areas<<<nb(nt), 256, 0, s>>>(v, t, nt, area); note_launch();
            exclusive_scan<double>(area, excl, (size_t)nt, tmp, total, s);
            k_samples<<<nb(n_samples), 256, 0, s>>>(v, t, nt, excl, area, total, n_samples, seed, pts); note_launch();
            Q_CK(cudaMemsetAsync(acc, 0, 16, s));
            if (mlp) {
                if ((r = mlp_eval_list(mlp, pts, n_samples, z, ODC_PREC_FP32, s, err)) != ODC_OK) break;
                k_deviation<<<nb(n_samples), 256, 0, s>>>(z, n_samples, (double)iso, acc); note_launch();
            } else if (vox) {
                k_vox_deviation<<<nb(n_samples), 256, 0, s>>>(pts, n_samples, *vox, (double)iso, acc); note_launch();
            } else {
                k_csg_distance<<<nb(n_samples), 256, 0, s>>>(pts, n_samples, prims, n_prims, acc); note_launch();
            }
            double h[2];
            Q_CK(cudaMemcpyAsync(h, acc, 16, cudaMemcpyDeviceToHost, s));
            Q_CK(cudaStreamSynchronize(s));
            out->n_samples = n_samples;
            (prims ? out->dist_mean : out->occ_dev_mean) = h[0] / (double)n_samples;
            (prims ? out->dist_max : out->occ_dev_max) = h[1];
        }
        // ---- manifoldness and Euler characteristic
        if (what & ODC_Q_MANIFOLD) {
            unsigned long long cap = 64;
            while (cap < 6ull * (unsigned long long)nt) cap <<= 1;
            void *pk, *pc, *p3, *pd, *ps;
            if ((r = alloc(cap * 8, &pk)) || (r = alloc(cap * 4, &pc)) || (r = alloc(cap * 4, &p3)) ||
                (r = alloc(nv * 4, &pd)) || (r = alloc(nv * 4, &ps)))
                break;
            HeTable H{(unsigned long long*)pk, (uint32_t*)pc, (uint32_t*)p3, cap - 1};
            Q_CK(cudaMemsetAsync(pk, 0xff, cap * 8, s));
            Q_CK(cudaMemsetAsync(pc, 0, cap * 4, s));
            Q_CK(cudaMemsetAsync(pd, 0, nv * 4, s));
            if (nt) { k_he_insert<<<nb(nt), 256, 0, s>>>(t, nt, H, (uint32_t*)pd, (uint32_t*)ps, dcnt); note_launch(); }
            k_he_check<<<nb((int64_t)cap), 256, 0, s>>>(H, dcnt); note_launch();
            if (nv) { k_fans<<<nb(nv), 256, 0, s>>>(t, nv, H, (const uint32_t*)pd, (const uint32_t*)ps, dcnt); note_launch(); }
        }
        // ---- self-intersections
        if ((what & ODC_Q_SI) && nt > 1) {
            // binning grid: the vertices' bounding box, cells of twice the
            // mean triangle extent (host-side, from a copy of the vertices)
            std::vector<float> hv((size_t)nv * 3);
            std::vector<int> ht((size_t)nt * 3);
            Q_CK(cudaMemcpyAsync(hv.data(), v, nv * 12, cudaMemcpyDeviceToHost, s));
            Q_CK(cudaMemcpyAsync(ht.data(), t, nt * 12, cudaMemcpyDeviceToHost, s));
            Q_CK(cudaStreamSynchronize(s));
            float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
            double ext = 0.0;
            for (int64_t i = 0; i < nt; ++i) {
                float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
                for (int c = 0; c < 3; ++c) {
                    const float* p = &hv[(size_t)ht[3 * i + c] * 3];
                    for (int a = 0; a < 3; ++a) { mn[a] = std::min(mn[a], p[a]); mx[a] = std::max(mx[a], p[a]); }
                }
                for (int a = 0; a < 3; ++a) {
                    lo[a] = std::min(lo[a], mn[a]);
                    hi[a] = std::max(hi[a], mx[a]);
                    ext += (double)(mx[a] - mn[a]) / 3.0;
                }
            }
            double cell = std::max(2.0 * ext / (double)nt, 1e-12);
            Bins b{};
            for (;;) {
                uint64_t tot = 1;
                for (int a = 0; a < 3; ++a) {
                    b.lo[a] = lo[a];
                    b.dim[a] = (int)std::min<double>(std::floor((hi[a] - lo[a]) / cell) + 1.0, 1 << 20);
                    tot *= (uint64_t)b.dim[a];
                }
                if (tot <= kMaxCells) break;
                cell *= 1.5;
            }
            b.inv = (float)(1.0 / cell);
            size_t ncell = (size_t)b.dim[0] * b.dim[1] * b.dim[2];
            size_t stmp = scan_tmp_elems(ncell);
            void *pcount, *poff, *ptmp, *pcur, *pbig, *pnbig, *pisbig, *pflag;
            if ((r = alloc(ncell * 4, &pcount)) || (r = alloc(ncell * 4, &poff)) || (r = alloc(stmp * 4 + 16, &ptmp)) ||
                (r = alloc(ncell * 4, &pcur)) || (r = alloc(nt * 4, &pbig)) || (r = alloc(16, &pnbig)) ||
                (r = alloc(nt, &pisbig)) || (r = alloc(nt, &pflag)))
                break;
            uint32_t* count = (uint32_t*)pcount;
            uint32_t* off = (uint32_t*)poff;
            uint32_t* tmp = (uint32_t*)ptmp;
            uint32_t* total = tmp + stmp;
            Q_CK(cudaMemsetAsync(count, 0, ncell * 4, s));
            Q_CK(cudaMemsetAsync(pcur, 0, ncell * 4, s));
            Q_CK(cudaMemsetAsync(pnbig, 0, 16, s));
            Q_CK(cudaMemsetAsync(pisbig, 0, nt, s));
            Q_CK(cudaMemsetAsync(pflag, 0, nt, s));
            k_bin_count<<<nb(nt), 256, 0, s>>>(v, t, nt, b, count, (int*)pbig, (uint32_t*)pnbig); note_launch();
            exclusive_scan<uint32_t>(count, off, ncell, tmp, total, s);
            uint32_t nlist = 0, nbig = 0;
            Q_CK(cudaMemcpyAsync(&nlist, total, 4, cudaMemcpyDeviceToHost, s));
            Q_CK(cudaMemcpyAsync(&nbig, pnbig, 4, cudaMemcpyDeviceToHost, s));
            Q_CK(cudaStreamSynchronize(s));
            void *plist, *plcell;
            if ((r = alloc((size_t)nlist * 4, &plist)) || (r = alloc((size_t)nlist * 4, &plcell))) break;
            k_bin_fill<<<nb(nt), 256, 0, s>>>(v, t, nt, b, off, (uint32_t*)pcur, (uint32_t*)plist, (uint32_t*)plcell); note_launch();
            if (nlist) {
                k_si_cells<<<nb(nlist, 128), 128, 0, s>>>(v, t, b, nlist, (const uint32_t*)plist, (const uint32_t*)plcell, off,
                                                     count, (uint8_t*)pflag, dcnt); note_launch();
            }
            if (nbig) {
                k_mark_big<<<nb(nbig), 256, 0, s>>>((const int*)pbig, (const uint32_t*)pnbig, (uint8_t*)pisbig); note_launch();
                k_si_big<<<nbig, 256, 0, s>>>(v, t, nt, (const int*)pbig, (const uint32_t*)pnbig,
                                              (const uint8_t*)pisbig, (uint8_t*)pflag, dcnt); note_launch();
            }
            k_count_flags<<<nb(nt), 256, 0, s>>>((const uint8_t*)pflag, nt, dcnt); note_launch();
            out->si_checked = 1;
        }
        Q_CK(cudaGetLastError());
        Q_CK(cudaMemcpyAsync(hc, dcnt, 16 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        Q_CK(cudaStreamSynchronize(s));
    } while (0);
    for (int i = 0; i < nfree; ++i) cudaFreeAsync(to_free[i], s);
    cudaFreeAsync(dcnt, s);
    if (r != ODC_OK) return r;
    if (what & ODC_Q_MANIFOLD) {
        out->n_degenerate = (int64_t)hc[0];
        out->n_bad_edges = (int64_t)hc[1];
        out->n_edges = (int64_t)hc[2];
        out->n_verts = (int64_t)hc[3];
        out->n_bad_verts = (int64_t)hc[4];
        out->euler = out->n_verts - out->n_edges + nt;
        out->manifold = (hc[0] == 0 && hc[1] == 0 && hc[4] == 0) ? 1 : 0;
    }
    if (what & ODC_Q_SI) {
        out->n_si_pairs = (int64_t)hc[5];
        out->n_si_tris = (int64_t)hc[6];
    }
    return ODC_OK;
}

}  // namespace odc
