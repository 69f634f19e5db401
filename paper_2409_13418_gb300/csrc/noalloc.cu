// noalloc.cu -- crossing-edge compaction that allocates no memory.
//
// Some callers cannot call cudaMalloc: code running inside a CUDA stream
// capture that must not add allocation nodes, allocator-free embedded or
// real-time hosts, and plug-ins whose host application owns all device
// memory and forbids allocation after start-up.  For them this file offers
// one entry point, odc_compact_edges_noalloc, that lists the crossing edges
// of a label bitmask (the first half of the compaction stage) with all its
// scratch in a fixed, file-scope device array instead of the context arena.
//
// The scratch array (kNoAllocScratchBytes = 4 MiB) exists on every GPU that
// loads the library and stays there until the process exits.  Host code must
// not hand the symbol itself to a kernel (on the host it is only a stand-in):
// the device address is looked up once per device with cudaGetSymbolAddress
// and cached.  All calls on a device share the array, so calls that overlap
// on the GPU (different streams or threads without ordering) race.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/odc.h"
#include "kernels.h"
#include "odc_internal.h"

namespace odc {

constexpr size_t kNoAllocScratchBytes = 4u << 20;
constexpr size_t kNoAllocMaxWords = 520000;   // label words per grid: counts + offsets + scan partials fit

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {};

struct Dims {
    int n[3], nv[3], W;
};

// Crossing mask of the edges owned by the 32 vertices of one label word.
__device__ __forceinline__ void word_edges(const Dims& d, const uint32_t* __restrict__ bits, size_t w, uint32_t m[3]) {
    int xw = (int)(w % d.W);
    size_t row = w / d.W;
    int y = (int)(row % d.nv[1]);
    int z = (int)(row / d.nv[1]);
    bool last = (xw == d.W - 1);
    uint32_t L = bits[w];
    uint32_t Lx = (L >> 1) | ((last ? 0u : bits[w + 1]) << 31);
    int rem_v = d.nv[0] - xw * 32, rem_e = d.n[0] - xw * 32;
    uint32_t vm = rem_v >= 32 ? ~0u : (rem_v <= 0 ? 0u : ((1u << rem_v) - 1u));
    uint32_t xm = rem_e >= 32 ? ~0u : (rem_e <= 0 ? 0u : ((1u << rem_e) - 1u));
    m[0] = (L ^ Lx) & xm;
    m[1] = y < d.n[1] ? ((L ^ bits[w + d.W]) & vm) : 0u;
    m[2] = z < d.n[2] ? ((L ^ bits[w + (size_t)d.W * d.nv[1]]) & vm) : 0u;
}

__global__ void k_na_count(Dims d, const uint32_t* __restrict__ bits, size_t nw, uint32_t* __restrict__ cnt) {
    size_t w = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nw) return;
    uint32_t m[3];
    word_edges(d, bits, w, m);
    cnt[w] = __popc(m[0]) + __popc(m[1]) + __popc(m[2]);
}

__global__ void k_na_emit(Dims d, const uint32_t* __restrict__ bits, size_t nw, const uint32_t* __restrict__ base,
                          uint32_t* __restrict__ edges, uint32_t cap) {
    size_t w = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int l = threadIdx.x & 31;
    if (w >= nw) return;
    uint32_t m[3];
    word_edges(d, bits, w, m);
    if ((((m[0] | m[1] | m[2]) >> l) & 1u) == 0) return;
    uint32_t below = (1u << l) - 1u;
    uint32_t o = base[w] + __popc(m[0] & below) + __popc(m[1] & below) + __popc(m[2] & below);
    int xw = (int)(w % d.W);
    size_t row = w / d.W;
    uint32_t y = (uint32_t)(row % d.nv[1]), z = (uint32_t)(row / d.nv[1]);
    uint32_t v = (uint32_t)(xw * 32 + l) + (uint32_t)d.nv[0] * (y + (uint32_t)d.nv[1] * z);
    for (int a = 0; a < 3; ++a)
        if ((m[a] >> l) & 1u) {
            if (o < cap) edges[o] = 3u * v + a;
            ++o;
        }
}

odc_status na_fail(odc_status s, const std::string& msg) {
    set_last_error(msg);
    return s;
}

// Device address of the scratch array on the current device (set-up, once per
// device; the first call on a device performs it).
odc_status scratch_address(int dev, void** out) {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return na_fail(ODC_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return ODC_OK;
}
}  // namespace

}  // namespace odc

using namespace odc;

extern "C" odc_status odc_compact_edges_noalloc(const uint32_t* d_label_bits, const int32_t res[3], uint32_t* d_edges,
                                                uint32_t max_edges, uint32_t* d_count, uint32_t* h_count,
                                                void* cuda_stream) {
    if (!d_label_bits || !res || !d_count || (max_edges && !d_edges))
        return na_fail(ODC_ERR_INVALID_ARG, "NULL argument");
    Dims d;
    for (int a = 0; a < 3; ++a) {
        if (res[a] < 1 || res[a] > kMaxRes) return na_fail(ODC_ERR_INVALID_ARG, "res out of [1, 1024]");
        d.n[a] = res[a];
        d.nv[a] = res[a] + 1;
    }
    d.W = (d.nv[0] + 31) / 32;
    size_t nw = (size_t)d.W * d.nv[1] * d.nv[2];
    if (nw > kNoAllocMaxWords)
        return na_fail(ODC_ERR_INVALID_ARG,
                       "grid too large for the fixed scratch: " + std::to_string(nw) + " label words > " +
                           std::to_string(kNoAllocMaxWords) + " (4 MiB); use odc_extract");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) return na_fail(ODC_ERR_CUDA, "no current CUDA device");
    void* scr = nullptr;
    odc_status s = scratch_address(dev, &scr);
    if (s != ODC_OK) return s;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // scratch layout: counts [nw] | offsets [nw] | scan partials | total
    uint32_t* cnt = (uint32_t*)scr;
    uint32_t* off = cnt + kNoAllocMaxWords;
    uint32_t* tmp = off + kNoAllocMaxWords;
    uint32_t* total = (uint32_t*)scr + (kNoAllocScratchBytes / 4 - 1);
    if ((size_t)(total - tmp) < scan_tmp_elems(nw)) return na_fail(ODC_ERR_INTERNAL, "scan scratch too small");
    // Every scratch word this call reads (counts, offsets, scan partials and
    // the total, which the scan always writes) is written earlier in the same
    // call, so no result depends on what an earlier call left in the array.
    // What the calls share is the array itself: calls that overlap on the GPU
    // overwrite each other's words.
    k_na_count<<<(unsigned)((nw + 255) / 256), 256, 0, st>>>(d, d_label_bits, nw, cnt); note_launch();
    exclusive_scan<uint32_t>(cnt, off, nw, tmp, total, st);
    k_na_emit<<<(unsigned)((nw * 32 + 255) / 256), 256, 0, st>>>(d, d_label_bits, nw, off, d_edges, max_edges); note_launch();
    e = cudaMemcpyAsync(d_count, total, sizeof(uint32_t), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(ODC_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    if (h_count) {
        e = cudaMemcpyAsync(h_count, total, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return na_fail(ODC_ERR_CUDA, std::string("count readback: ") + cudaGetErrorString(e));
        if (*h_count > max_edges)
            return na_fail(ODC_ERR_OOM, "edge buffer too small: " + std::to_string(*h_count) + " crossing edges > " +
                                            std::to_string(max_edges));
    }
    return ODC_OK;
}
