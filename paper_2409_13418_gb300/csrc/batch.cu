// batch.cu -- network evaluations shared by several contexts (batch.h).
//
// Round protocol (host): a member's call records an event on its stream and
// queues itself; when the queued calls equal the members inside a search
// stage, the caller that completes the set (or a member leaving its stage
// with the rest queued) runs the round: the group's stream waits for every
// caller's event, a merge kernel concatenates their query lists (device
// counts read on the device), the tiered network evaluates the merged list
// once, a scatter kernel writes each caller's logits back, and every
// caller's stream waits for the round's event.  All waiting between rounds
// is host-side or stream-ordered; no kernel waits for another.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <mutex>
#include <string>
#include <vector>

#include "batch.h"
#include "mlp.h"
#include "mlp_dev.cuh"

namespace odc {

constexpr int kMaxMembers = 64;
// A queued call that no round has taken within this time leaves the queue
// and fails with ODC_ERR_TIMEOUT (its search stage then ends, so the other
// members' rounds no longer wait for it); a call already taken by a running
// round waits for that round.
constexpr int kRendezvousSeconds = 120;

struct BatchSeg {
    const float3* pts;
    const float* hint;             // NULL: no routing hint
    float* z;
    const unsigned long long* n_dev;   // NULL: n_max queries
    long long n_max;
    int row;                       // first-layer bias row of the member
    int pad;
};
struct BatchTable {
    BatchSeg s[kMaxMembers];
    int nseg;
};

__device__ __forceinline__ long long seg_count(const BatchSeg& s) {
    return s.n_dev ? (long long)min((unsigned long long)s.n_max, *s.n_dev) : s.n_max;
}

// blockIdx.y = segment: its queries go to the merged list at the sum of the
// counts of the segments before it.
__global__ void k_batch_merge(BatchTable T, float3* __restrict__ mp, float* __restrict__ mh,
                              uint16_t* __restrict__ mseg, unsigned long long* __restrict__ total) {
    __shared__ long long off, cnt;
    const int y = blockIdx.y;
    if (threadIdx.x == 0) {
        long long o = 0;
        for (int j = 0; j < y; ++j) o += seg_count(T.s[j]);
        off = o;
        cnt = seg_count(T.s[y]);
        if (blockIdx.x == 0 && y == T.nseg - 1) *total = (unsigned long long)(o + cnt);
    }
    __syncthreads();
    const BatchSeg& S = T.s[y];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (long long)gridDim.x * blockDim.x) {
        mp[off + i] = S.pts[i];
        mh[off + i] = S.hint ? S.hint[i] : INFINITY;
        mseg[off + i] = (uint16_t)S.row;
    }
}

__global__ void k_batch_scatter(BatchTable T, const float* __restrict__ mz) {
    __shared__ long long off, cnt;
    const int y = blockIdx.y;
    if (threadIdx.x == 0) {
        long long o = 0;
        for (int j = 0; j < y; ++j) o += seg_count(T.s[j]);
        off = o;
        cnt = seg_count(T.s[y]);
    }
    __syncthreads();
    const BatchSeg& S = T.s[y];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (long long)gridDim.x * blockDim.x)
        S.z[i] = mz[off + i];
}

struct Pending {
    MlpState* st;
    const float3* pts;
    int64_t n_max;
    const unsigned long long* n_dev;
    float* z;
    const float* hint;
    cudaStream_t s;
    float zt;
    bool done = false;
    odc_status status = ODC_OK;
    std::string err;
};

struct BatchGroup {
    int device = 0;
    std::mutex mu;                 // members, queue, counters
    std::condition_variable cv;
    std::mutex launch_mu;          // the group's stream and network state: one round enqueued at a time
    cudaStream_t stream = nullptr;
    cudaEvent_t done_ev = nullptr;
    MlpState* net = nullptr;       // the group's network
    bool net_ready = false;
    int precision = -1;
    std::vector<float> wkey;
    bool row_used[kMaxMembers] = {};
    int active = 0;                // members inside a search stage
    std::vector<Pending*> queue;
    float* b0tab = nullptr;        // [kMaxMembers][256] folded first-layer biases
    float3* mp = nullptr;          // merged query points, hints, logits, bias rows
    float* mh = nullptr;
    float* mz = nullptr;
    uint16_t* mseg = nullptr;
    unsigned long long* mtotal = nullptr;
    int* h_err = nullptr;          // pinned: the network's error flag, read at stage exits
    size_t cap = 0;
    int64_t rounds = 0, calls = 0;
};

odc_status batch_create(int device, BatchGroup** out, std::string* err) {
    *out = nullptr;
    auto* g = new BatchGroup();
    g->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->done_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc((void**)&g->b0tab, sizeof(float) * kMaxMembers * kH);
    if (e == cudaSuccess) e = cudaMalloc((void**)&g->mtotal, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&g->h_err, sizeof(int));
    if (e != cudaSuccess) {
        *err = std::string("batch group setup: ") + cudaGetErrorString(e);
        cudaGetLastError();
        batch_destroy(g);
        return ODC_ERR_CUDA;
    }
    *out = g;
    return ODC_OK;
}

void batch_destroy(BatchGroup* g) {
    if (!g) return;
    cudaSetDevice(g->device);
    if (g->stream) cudaStreamSynchronize(g->stream);
    mlp_destroy(g->net);
    for (void* p : {(void*)g->b0tab, (void*)g->mp, (void*)g->mh, (void*)g->mz, (void*)g->mseg, (void*)g->mtotal})
        if (p) cudaFree(p);
    if (g->h_err) cudaFreeHost(g->h_err);
    if (g->done_ev) cudaEventDestroy(g->done_ev);
    if (g->stream) cudaStreamDestroy(g->stream);
    delete g;
}

void batch_stats(const BatchGroup* g, int64_t* rounds, int64_t* calls) {
    auto* m = const_cast<BatchGroup*>(g);
    std::lock_guard<std::mutex> lk(m->mu);
    *rounds = g->rounds;
    *calls = g->calls;
}

odc_status batch_bind(MlpState* st, BatchGroup* g, const odc_mlp* m, std::string* err) {
    if (!st) return ODC_OK;
    if (!g) {
        batch_unbind(st);
        return ODC_OK;
    }
    if (!m && st->group == g) return ODC_OK;   // resident source: the binding of its upload holds
    if (st->group && st->group != g) batch_unbind(st);
    if (!m) return ODC_OK;                     // resident source uploaded before joining: evaluates alone
    {
        std::lock_guard<std::mutex> launch(g->launch_mu);
        std::lock_guard<std::mutex> lk(g->mu);
        if (!g->net_ready) {
            g->net_ready = true;
            g->wkey = st->wkey;
            g->precision = m->precision;
            odc_status r = mlp_prepare(&g->net, m, g->stream, err);
            if (r != ODC_OK) {
                g->net_ready = false;
                return r;
            }
        }
        if (!st->bev && cudaEventCreateWithFlags(&st->bev, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            *err = "batch: event creation failed";
            return ODC_ERR_CUDA;
        }
        st->group = g;
        st->bcompat = g->precision == m->precision && st->wkey == g->wkey;
        if (st->brow < 0) {
            for (int i = 0; i < kMaxMembers; ++i)
                if (!g->row_used[i]) {
                    g->row_used[i] = true;
                    st->brow = i;
                    break;
                }
            if (st->brow < 0) st->bcompat = false;   // more members than bias rows: evaluates alone
        }
        st->b0dirty = true;
    }
    return ODC_OK;
}

void batch_unbind(MlpState* st) {
    if (!st || !st->group) return;
    BatchGroup* g = st->group;
    {
        std::lock_guard<std::mutex> lk(g->mu);
        if (st->brow >= 0) g->row_used[st->brow] = false;
    }
    st->brow = -1;
    st->bcompat = false;
    st->group = nullptr;
}

bool batch_active(const MlpState* st) { return st && st->group && st->bcompat && st->bin_stage; }

// Run one round over ``batch`` (queued calls, removed from the queue).
static void run_round(BatchGroup* g, std::vector<Pending*>& batch) {
    std::lock_guard<std::mutex> launch(g->launch_mu);
    odc_status r = ODC_OK;
    std::string err;
    auto ck = [&](cudaError_t e, const char* what) {
        if (e != cudaSuccess && r == ODC_OK) {
            r = ODC_ERR_CUDA;
            err = std::string(what) + ": " + cudaGetErrorString(e);
        }
    };
    cudaSetDevice(g->device);
    for (Pending* p : batch) {
        ck(cudaStreamWaitEvent(g->stream, p->st->bev, 0), "stream wait");
        if (p->st->b0dirty) {   // the member is blocked in this round: its host row is stable
            ck(cudaMemcpyAsync(g->b0tab + (size_t)p->st->brow * kH, p->st->b0host.data(), sizeof(float) * kH,
                               cudaMemcpyHostToDevice, g->stream),
               "bias row upload");
            p->st->b0dirty = false;
        }
    }
    // one evaluation per threshold (members at the same iso level share it)
    std::vector<bool> taken(batch.size(), false);
    for (size_t a = 0; a < batch.size() && r == ODC_OK; ++a) {
        if (taken[a]) continue;
        BatchTable T{};
        int64_t total = 0;
        long long maxn = 0;
        for (size_t b = a; b < batch.size() && T.nseg < kMaxMembers; ++b) {
            if (taken[b] || batch[b]->zt != batch[a]->zt) continue;
            taken[b] = true;
            const Pending* p = batch[b];
            T.s[T.nseg++] = BatchSeg{p->pts, p->hint, p->z, p->n_dev, (long long)p->n_max, p->st->brow, 0};
            total += p->n_max;
            maxn = std::max<long long>(maxn, p->n_max);
        }
        if (total <= 0) continue;
        if ((size_t)total > g->cap) {
            const size_t want = std::max<size_t>((size_t)total, g->cap + g->cap / 2);
            for (void* p : {(void*)g->mp, (void*)g->mh, (void*)g->mz, (void*)g->mseg})
                if (p) ck(cudaFreeAsync(p, g->stream), "free");
            g->mp = nullptr;
            g->mh = g->mz = nullptr;
            g->mseg = nullptr;
            g->cap = 0;
            ck(cudaMallocAsync((void**)&g->mp, want * sizeof(float3), g->stream), "merged buffers");
            ck(cudaMallocAsync((void**)&g->mh, want * sizeof(float), g->stream), "merged buffers");
            ck(cudaMallocAsync((void**)&g->mz, want * sizeof(float), g->stream), "merged buffers");
            ck(cudaMallocAsync((void**)&g->mseg, want * sizeof(uint16_t), g->stream), "merged buffers");
            if (r != ODC_OK) break;
            g->cap = want;
        }
        const dim3 grid((unsigned)std::min<long long>(std::max<long long>((maxn + 255) / 256, 1), 1024),
                        (unsigned)T.nseg);
        k_batch_merge<<<grid, 256, 0, g->stream>>>(T, g->mp, g->mh, g->mseg, g->mtotal);
        note_launch();
        ck(cudaGetLastError(), "merge launch");
        if (r != ODC_OK) break;
        g->net->zt = batch[a]->zt;
        g->net->stream = g->stream;
        r = mlp_eval_merged(g->net, g->mp, g->mh, g->mseg, g->b0tab, total, g->mtotal, g->mz, g->stream, &err);
        if (r != ODC_OK) break;
        k_batch_scatter<<<grid, 256, 0, g->stream>>>(T, g->mz);
        note_launch();
        ck(cudaGetLastError(), "scatter launch");
    }
    ck(cudaEventRecord(g->done_ev, g->stream), "event record");
    for (Pending* p : batch) ck(cudaStreamWaitEvent(p->s, g->done_ev, 0), "stream wait");
    for (Pending* p : batch) {
        p->status = r;
        p->err = err;
    }
}

// Under g->mu (held by lk): if the queued calls complete the active set, take
// them and run their round (the lock is released meanwhile).
static void maybe_lead(BatchGroup* g, std::unique_lock<std::mutex>& lk) {
    if (g->queue.empty() || (int)g->queue.size() < g->active) return;
    std::vector<Pending*> batch;
    batch.swap(g->queue);
    g->rounds += 1;
    g->calls += (int64_t)batch.size();
    lk.unlock();
    run_round(g, batch);
    lk.lock();
    for (Pending* p : batch) p->done = true;
    g->cv.notify_all();
}

void batch_enter(MlpState* st) {
    if (!st || !st->group || !st->bcompat) return;
    BatchGroup* g = st->group;
    std::lock_guard<std::mutex> lk(g->mu);
    g->active += 1;
    st->bin_stage = true;
}

odc_status batch_leave(MlpState* st, std::string* err) {
    if (!st || !st->group || !st->bin_stage) return ODC_OK;
    BatchGroup* g = st->group;
    {
        std::unique_lock<std::mutex> lk(g->mu);
        g->active -= 1;
        st->bin_stage = false;
        maybe_lead(g, lk);   // the others may now be complete
    }
    // the network's error flag (an expired device wait in its kernels)
    cudaEvent_t ev = st->bev;
    {
        std::lock_guard<std::mutex> launch(g->launch_mu);
        if (!g->net || !mlp_tc_err_flag(g->net)) return ODC_OK;
        if (cudaMemcpyAsync(g->h_err, mlp_tc_err_flag(g->net), sizeof(int), cudaMemcpyDeviceToHost, g->stream) !=
                cudaSuccess ||
            cudaEventRecord(ev, g->stream) != cudaSuccess) {
            *err = "cannot read the shared network's error flag";
            return ODC_ERR_CUDA;
        }
    }
    if (cudaEventSynchronize(ev) != cudaSuccess) {
        *err = "cannot read the shared network's error flag";
        return ODC_ERR_CUDA;
    }
    if (*g->h_err) {
        std::lock_guard<std::mutex> launch(g->launch_mu);
        cudaMemsetAsync(mlp_tc_err_flag(g->net), 0, sizeof(int), g->stream);
        *err = "shared tensor-core evaluation: a pipeline wait expired";
        return ODC_ERR_TIMEOUT;
    }
    return ODC_OK;
}

odc_status batch_eval(MlpState* st, const float3* pts, int64_t n_max, const unsigned long long* n_dev, float* z,
                      const float* hint, cudaStream_t s, std::string* err) {
    BatchGroup* g = st->group;
    if (cudaEventRecord(st->bev, s) != cudaSuccess) {
        cudaGetLastError();
        *err = "batch: event record failed";
        return ODC_ERR_CUDA;
    }
    Pending p;
    p.st = st;
    p.pts = pts;
    p.n_max = n_max;
    p.n_dev = n_dev;
    p.z = z;
    p.hint = hint;
    p.s = s;
    p.zt = st->zt;
    std::unique_lock<std::mutex> lk(g->mu);
    g->queue.push_back(&p);
    maybe_lead(g, lk);
    if (!g->cv.wait_for(lk, std::chrono::seconds(kRendezvousSeconds), [&] { return p.done; })) {
        auto it = std::find(g->queue.begin(), g->queue.end(), &p);
        if (it != g->queue.end()) {
            g->queue.erase(it);
            *err = "batch: no shared evaluation round formed within " + std::to_string(kRendezvousSeconds) +
                   " s (" + std::to_string(g->queue.size()) + " other calls queued, " + std::to_string(g->active) +
                   " members in a search stage)";
            return ODC_ERR_TIMEOUT;
        }
        g->cv.wait(lk, [&] { return p.done; });   // taken by a round that is running: it completes
    }
    if (p.status != ODC_OK) *err = p.err;
    return p.status;
}

}  // namespace odc
