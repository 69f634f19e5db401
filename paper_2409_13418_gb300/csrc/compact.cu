// compact.cu -- CSG grid occupancy, crossing classification, prefix scans and
// list emission (Sec. 3: labels at grid vertices, crossing edges E^S, the
// faces carrying 2D points and the crossing cells C^S).
//
// Labels live as bits: one 32-bit word holds 32 consecutive vertices of an
// x-row, rows padded to W = ceil((res0+1)/32) words.  All crossing tests are
// bitwise on whole words, so classification reads a handful of words per 32
// vertices; counts per word are prefix-scanned and the lists are emitted in
// id order (deterministic, no atomics).
#include "kernels.h"
#include "odc_device.cuh"

#include <atomic>

namespace odc {

static std::atomic<long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

// ---------------------------------------------------------------- grid phi
// One warp per label word: lane l evaluates vertex x = 32 w + l.  A primitive
// whose bounding sphere misses the warp's whole x-segment is skipped by the
// warp as a unit (a primitive outside its bounding sphere never changes the
// union/difference fold).
__global__ void k_csg_grid(GridDev g, const PrimDev* __restrict__ prims, const float4* __restrict__ cull,
                           int n_prims, uint32_t* __restrict__ bits) {
    size_t wid = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    size_t nw = (size_t)g.W * g.nv[1] * g.nv[2];
    if (wid >= nw) return;
    int xw = (int)(wid % g.W);
    size_t row = wid / g.W;
    int y = (int)(row % g.nv[1]);
    int z = (int)(row / g.nv[1]);
    int x = xw * 32 + lane;
    bool valid = x < g.nv[0];
    int xc = valid ? x : g.nv[0] - 1;
    float px = g.X[0][xc], py = g.X[1][y], pz = g.X[2][z];
    float xs = g.X[0][xw * 32], xe = g.X[0][min(xw * 32 + 31, g.nv[0] - 1)];
    uint32_t in = 0;
    for (int i = 0; i < n_prims; ++i) {
        float4 c = __ldg(&cull[i]);
        float sx = fminf(fmaxf(c.x, xs), xe) - c.x, sy = py - c.y, sz = pz - c.z;
        if (sx * sx + sy * sy + sz * sz > c.w) continue;   // uniform across the warp
        float dx = px - c.x;
        int s = 1;
        if (dx * dx + sy * sy + sz * sz <= c.w) s = prim_sign(prims[i], px, py, pz);
        if (i == 0 || prims[i].op == OP_UNION) in |= (s < 0);
        else in &= (s > 0);
    }
    uint32_t word = __ballot_sync(0xffffffffu, valid && in);
    if (lane == 0) bits[wid] = word;
}

// ------------------------------------------------------------ classify
__device__ __forceinline__ uint32_t shift_next(uint32_t L, uint32_t Lnext) { return (L >> 1) | (Lnext << 31); }

__global__ void k_classify(GridDev g, const uint32_t* __restrict__ bits, WordInfo* __restrict__ wi,
                           uint32_t* __restrict__ ce, uint32_t* __restrict__ cf, uint32_t* __restrict__ cc) {
    size_t w = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t nw = (size_t)g.W * g.nv[1] * g.nv[2];
    if (w >= nw) return;
    int xw = (int)(w % g.W);
    size_t row = w / g.W;
    int y = (int)(row % g.nv[1]);
    int z = (int)(row / g.nv[1]);
    bool last = (xw == g.W - 1);
    size_t rowW = g.W, sliceW = (size_t)g.W * g.nv[1];
    bool hy = y < g.n[1], hz = z < g.n[2];

    auto ld = [&](size_t idx) -> uint32_t { return bits[idx]; };
    uint32_t L = ld(w), Lx = shift_next(L, last ? 0u : ld(w + 1));
    uint32_t Ly = 0, Lyx = 0, Lz = 0, Lzx = 0, Lyz = 0, Lyzx = 0;
    if (hy) { Ly = ld(w + rowW); Lyx = shift_next(Ly, last ? 0u : ld(w + rowW + 1)); }
    if (hz) { Lz = ld(w + sliceW); Lzx = shift_next(Lz, last ? 0u : ld(w + sliceW + 1)); }
    if (hy && hz) { Lyz = ld(w + rowW + sliceW); Lyzx = shift_next(Lyz, last ? 0u : ld(w + rowW + sliceW + 1)); }

    int rem_v = g.nv[0] - xw * 32;            // vertices in this word
    int rem_e = g.n[0] - xw * 32;             // x-edges / cells in this word
    uint32_t vm = rem_v >= 32 ? ~0u : (rem_v <= 0 ? 0u : ((1u << rem_v) - 1u));
    uint32_t xm = rem_e >= 32 ? ~0u : (rem_e <= 0 ? 0u : ((1u << rem_e) - 1u));

    WordInfo r;
    r.m[0] = (L ^ Lx) & xm;
    r.m[1] = hy ? ((L ^ Ly) & vm) : 0u;
    r.m[2] = hz ? ((L ^ Lz) & vm) : 0u;
    auto face = [](uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t msk, uint32_t* has, uint32_t* amb) {
        *has = ((c0 ^ c1) | (c1 ^ c2) | (c2 ^ c3) | (c3 ^ c0)) & msk;
        *amb = ~(c0 ^ c2) & ~(c1 ^ c3) & (c0 ^ c1) & msk;
    };
    r.fhas[0] = r.famb[0] = r.fhas[1] = r.famb[1] = r.fhas[2] = r.famb[2] = 0;
    // face normal to x spans (y, z); normal to y spans (z, x); normal to z spans (x, y)
    if (hy && hz) face(L, Ly, Lyz, Lz, vm, &r.fhas[0], &r.famb[0]);
    if (hz) face(L, Lz, Lzx, Lx, xm, &r.fhas[1], &r.famb[1]);
    if (hy) face(L, Lx, Lyx, Ly, xm, &r.fhas[2], &r.famb[2]);
    r.cell = 0;
    if (hy && hz) {
        uint32_t A = L & Lx & Ly & Lyx & Lz & Lzx & Lyz & Lyzx;
        uint32_t O = L | Lx | Ly | Lyx | Lz | Lzx | Lyz | Lyzx;
        r.cell = ~A & O & xm;
    }
    wi[w] = r;
    ce[w] = __popc(r.m[0]) + __popc(r.m[1]) + __popc(r.m[2]);
    cf[w] = __popc(r.fhas[0]) + __popc(r.famb[0]) + __popc(r.fhas[1]) + __popc(r.famb[1]) + __popc(r.fhas[2]) +
            __popc(r.famb[2]);
    cc[w] = __popc(r.cell);
}

// ------------------------------------------------------------------- emit
// One warp per word, lane = vertex: each lane writes its own items at the
// rank given by popcounts of the lower lanes.
__global__ void k_emit(GridDev g, const uint32_t* __restrict__ bits, const WordInfo* __restrict__ wi,
                       const uint32_t* __restrict__ ebase, const uint32_t* __restrict__ fbase,
                       const uint32_t* __restrict__ cbase, uint32_t* __restrict__ edges,
                       uint32_t* __restrict__ faces, uint8_t* __restrict__ slots, uint32_t* __restrict__ cells,
                       uint8_t* __restrict__ configs) {
    size_t w = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int l = threadIdx.x & 31;
    size_t nw = (size_t)g.W * g.nv[1] * g.nv[2];
    if (w >= nw) return;
    WordInfo r = wi[w];
    uint32_t any = r.m[0] | r.m[1] | r.m[2] | r.fhas[0] | r.fhas[1] | r.fhas[2] | r.cell;
    if (((any >> l) & 1u) == 0) return;
    int xw = (int)(w % g.W);
    size_t row = w / g.W;
    int y = (int)(row % g.nv[1]);
    int z = (int)(row / g.nv[1]);
    int x = xw * 32 + l;
    uint32_t below = (1u << l) - 1u;
    uint32_t v = (uint32_t)x + (uint32_t)g.nv[0] * ((uint32_t)y + (uint32_t)g.nv[1] * (uint32_t)z);
    uint32_t eo = ebase[w] + __popc(r.m[0] & below) + __popc(r.m[1] & below) + __popc(r.m[2] & below);
    for (int a = 0; a < 3; ++a)
        if ((r.m[a] >> l) & 1u) edges[eo++] = 3u * v + a;
    uint32_t fo = fbase[w];
    for (int a = 0; a < 3; ++a) fo += __popc(r.fhas[a] & below) + __popc(r.famb[a] & below);
    for (int a = 0; a < 3; ++a) {
        if ((r.fhas[a] >> l) & 1u) { faces[fo] = 3u * v + a; slots[fo] = 0; ++fo; }
        if ((r.famb[a] >> l) & 1u) { faces[fo] = 3u * v + a; slots[fo] = 1; ++fo; }
    }
    if ((r.cell >> l) & 1u) {
        uint32_t co = cbase[w] + __popc(r.cell & below);
        cells[co] = (uint32_t)x + (uint32_t)g.n[0] * ((uint32_t)y + (uint32_t)g.n[1] * (uint32_t)z);
        configs[co] = (uint8_t)cell_config(g, bits, x, y, z);
    }
}

// ------------------------------------------------------------------- scan
// Exclusive prefix sum, three phases: tile sums, one block scans the tile
// sums with a running carry, tiles rescan and add their offset.
constexpr int kScanThreads = 512;
constexpr int kScanPer = 8;
constexpr int kScanTile = kScanThreads * kScanPer;

template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T* total) {
    __shared__ T warp_sums[kScanThreads / 32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_sums[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        T s = (lane < kScanThreads / 32) ? warp_sums[lane] : T(0);
        T si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T t = __shfl_up_sync(0xffffffffu, si, o);
            if (lane >= o) si += t;
        }
        if (lane < kScanThreads / 32) warp_sums[lane] = si - s;
        if (lane == kScanThreads / 32 - 1) *total = si;
    }
    __syncthreads();
    T r = warp_sums[wid] + inc - v;
    __syncthreads();
    return r;
}

template <typename T>
__global__ void k_scan_tiles(const T* __restrict__ in, size_t n, T* __restrict__ tile_sums) {
    size_t base = (size_t)blockIdx.x * kScanTile + (size_t)threadIdx.x * kScanPer;
    T s = 0;
#pragma unroll
    for (int i = 0; i < kScanPer; ++i)
        if (base + i < n) s += in[base + i];
    __shared__ T tot;
    block_excl_scan<T>(s, &tot);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

template <typename T>
__global__ void k_scan_sums(T* __restrict__ tile_sums, size_t nt, T* __restrict__ total) {
    __shared__ T carry_s;
    __shared__ T tot;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (size_t b = 0; b < nt; b += kScanThreads) {
        size_t i = b + threadIdx.x;
        T v = i < nt ? tile_sums[i] : T(0);
        T ex = block_excl_scan<T>(v, &tot);
        T carry = carry_s;
        if (i < nt) tile_sums[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry_s = carry + tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry_s;
}

template <typename T>
__global__ void k_scan_apply(const T* __restrict__ in, size_t n, const T* __restrict__ tile_sums, T* __restrict__ out) {
    size_t base = (size_t)blockIdx.x * kScanTile + (size_t)threadIdx.x * kScanPer;
    T loc[kScanPer];
    T s = 0;
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        loc[i] = (base + i < n) ? in[base + i] : T(0);
        s += loc[i];
    }
    __shared__ T tot;
    T ex = block_excl_scan<T>(s, &tot) + tile_sums[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        if (base + i < n) out[base + i] = ex;
        ex += loc[i];
    }
}

size_t scan_tmp_elems(size_t n) { return (n + kScanTile - 1) / kScanTile + 1; }

template <typename T>
void exclusive_scan(const T* in, T* out, size_t n, T* tmp, T* total, cudaStream_t st) {
    size_t nt = (n + kScanTile - 1) / kScanTile;
    if (nt == 0) {
        cudaMemsetAsync(total, 0, sizeof(T), st);
        return;
    }
    k_scan_tiles<T><<<(unsigned)nt, kScanThreads, 0, st>>>(in, n, tmp); note_launch();
    k_scan_sums<T><<<1, kScanThreads, 0, st>>>(tmp, nt, total); note_launch();
    k_scan_apply<T><<<(unsigned)nt, kScanThreads, 0, st>>>(in, n, tmp, out); note_launch();
}

template void exclusive_scan<uint32_t>(const uint32_t*, uint32_t*, size_t, uint32_t*, uint32_t*, cudaStream_t);
template void exclusive_scan<unsigned long long>(const unsigned long long*, unsigned long long*, size_t,
                                                 unsigned long long*, unsigned long long*, cudaStream_t);
template void exclusive_scan<double>(const double*, double*, size_t, double*, double*, cudaStream_t);

// --------------------------------------------------------------- launchers
void launch_csg_grid(const GridDev& g, const PrimDev* prims, const float4* cull, int n_prims, uint32_t* bits,
                     cudaStream_t st) {
    size_t nw = (size_t)g.W * g.nv[1] * g.nv[2];
    size_t threads = nw * 32;
    k_csg_grid<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(g, prims, cull, n_prims, bits); note_launch();
}

void launch_classify(const GridDev& g, const uint32_t* bits, WordInfo* wi, uint32_t* ce, uint32_t* cf, uint32_t* cc,
                     cudaStream_t st) {
    size_t nw = (size_t)g.W * g.nv[1] * g.nv[2];
    k_classify<<<(unsigned)((nw + 255) / 256), 256, 0, st>>>(g, bits, wi, ce, cf, cc); note_launch();
}

void launch_emit(const GridDev& g, const uint32_t* bits, const WordInfo* wi, const uint32_t* ebase,
                 const uint32_t* fbase, const uint32_t* cbase, uint32_t* edges, uint32_t* faces, uint8_t* slots,
                 uint32_t* cells, uint8_t* configs, cudaStream_t st) {
    size_t nw = (size_t)g.W * g.nv[1] * g.nv[2];
    size_t threads = nw * 32;
    k_emit<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(g, bits, wi, ebase, fbase, cbase, edges, faces, slots,
                                                            cells, configs); note_launch();
}

}  // namespace odc
