// serve.cu -- request loop: meshing requests of any grid size, admitted as
// slots and device memory free up, running concurrently on the GPU.
//
// Each slot owns a context (stream, device arenas, network state) and one
// worker thread.  A worker takes the oldest queued request once the memory
// estimate of the admitted requests and unreleased results leaves room for
// it, runs odc_extract on its own context, and copies the mesh into result
// buffers owned by the request (stream-ordered device allocations, plus host
// copies on request).  Requests on different slots overlap on the device:
// while one slot waits on a host round trip (a count read-back) or runs a
// latency-bound stage, the others keep the SMs busy.  Nothing of a request
// depends on the others, so every mesh is byte-identical to the one
// odc_extract produces alone.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/odc.h"
#include "odc_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

// Deep copy of one request's inputs.
struct Request {
    uint64_t id = 0;
    odc_source src{};
    std::vector<odc_csg_prim> prims;
    odc_voxels vox{};
    std::vector<float> vox_values;
    odc_mlp mlp{};
    std::vector<float> B, latent, W[8], b[8];
    odc_grid grid{};
    odc_params prm{};
    uint64_t est = 0;
    // outcome
    bool done = false;
    odc_status status = ODC_OK;
    std::string err;
    int slot = -1;
    double t_submit = 0, t_start = 0, t_end = 0;
    float* d_verts = nullptr;
    int32_t* d_tris = nullptr;
    uint64_t result_bytes = 0;
    odc_mesh mesh{};
    std::vector<float> h_verts;
    std::vector<int32_t> h_tris;
};

// Device memory a request may hold while it runs: the grid-sized arena
// (label words with their masks, scans and flips, ~90 B per word), the
// grid-sized network scratch of an MLP source (logits, routes and three tier
// lists: 17 B per vertex), and the crossing-sized buffers (about 8 N^2
// crossing edges for a closed surface spanning the grid; ~700 B per edge
// over the lists, search states and mesh), plus 64 MiB of weights and fixed
// buffers (plus the samples of a voxel source).
uint64_t estimate_bytes(const odc_source& src, const odc_grid& g) {
    const uint64_t nv0 = (uint64_t)g.res[0] + 1, nv1 = (uint64_t)g.res[1] + 1, nv2 = (uint64_t)g.res[2] + 1;
    const uint64_t W = (nv0 + 31) / 32, nw = W * nv1 * nv2, V = nw * 32;
    const uint64_t r = (uint64_t)std::max(g.res[0], std::max(g.res[1], g.res[2]));
    uint64_t b = nw * 90 + 8 * r * r * 700 + (64ull << 20);
    if (src.kind == ODC_SRC_MLP) b += V * 17;
    if (src.kind == ODC_SRC_VOXEL && src.voxels)
        b += 4ull * (uint64_t)src.voxels->dims[0] * src.voxels->dims[1] * src.voxels->dims[2];
    return b;
}

odc_status copy_source(const odc_source* s, Request& q, std::string* err) {
    q.src = *s;
    if (s->kind == ODC_SRC_CSG) {
        if (!s->prims || s->n_prims < 1 || s->n_prims > 4096) { *err = "CSG source: 1..4096 primitives required"; return ODC_ERR_INVALID_ARG; }
        q.prims.assign(s->prims, s->prims + s->n_prims);
        q.src.prims = q.prims.data();
        q.src.mlp = nullptr;
        return ODC_OK;
    }
    if (s->kind == ODC_SRC_VOXEL) {
        const odc_voxels* v = s->voxels;
        if (!v || !v->values) { *err = "voxel source without values"; return ODC_ERR_INVALID_ARG; }
        double n = 1.0;
        for (int a = 0; a < 3; ++a) n *= v->dims[a] >= 2 ? v->dims[a] : 0;
        if (n <= 0 || n > 2147483648.0) { *err = "voxel dims out of range"; return ODC_ERR_INVALID_ARG; }
        q.vox = *v;
        q.vox_values.assign(v->values, v->values + (size_t)n);
        q.vox.values = q.vox_values.data();
        q.src.voxels = &q.vox;
        q.src.prims = nullptr;
        q.src.mlp = nullptr;
        return ODC_OK;
    }
    if (s->kind != ODC_SRC_MLP) { *err = "odc_submit takes CSG, MLP or voxel sources (not resident ones)"; return ODC_ERR_INVALID_ARG; }
    const odc_mlp* m = s->mlp;
    if (!m || !m->B) { *err = "MLP source without descriptor or Fourier matrix"; return ODC_ERR_INVALID_ARG; }
    if (m->n_hidden < 1 || m->n_hidden > 7 || m->hidden < 1 || m->n_freq < 1 || m->latent_dim < 0)
        { *err = "MLP shape out of range"; return ODC_ERR_INVALID_ARG; }
    q.mlp = *m;
    q.B.assign(m->B, m->B + (size_t)m->n_freq * 3);
    q.mlp.B = q.B.data();
    for (int l = 0; l <= m->n_hidden; ++l) {
        if (!m->W[l] || !m->b[l]) { *err = "weight or bias pointer missing"; return ODC_ERR_INVALID_ARG; }
        size_t rows = l == m->n_hidden ? 1 : (size_t)m->hidden;
        size_t cols = l == 0 ? (size_t)m->latent_dim + 2 * (size_t)m->n_freq : (size_t)m->hidden;
        q.W[l].assign(m->W[l], m->W[l] + rows * cols);
        q.b[l].assign(m->b[l], m->b[l] + rows);
        q.mlp.W[l] = q.W[l].data();
        q.mlp.b[l] = q.b[l].data();
    }
    if (m->latent_dim) {
        if (!m->latent) { *err = "latent pointer missing"; return ODC_ERR_INVALID_ARG; }
        q.latent.assign(m->latent, m->latent + m->latent_dim);
        q.mlp.latent = q.latent.data();
    }
    q.src.mlp = &q.mlp;
    q.src.prims = nullptr;
    return ODC_OK;
}

}  // namespace

struct odc_server {
    odc_server_config cfg{};
    Clock::time_point t0;
    std::vector<odc_ctx*> ctx;
    std::vector<cudaStream_t> streams;
    odc_batch* batch = nullptr;  // shared network evaluations of the slots (share_network)
    cudaStream_t free_stream = nullptr;
    std::vector<std::thread> workers;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Request>> queue;
    std::unordered_map<uint64_t, std::shared_ptr<Request>> reqs;
    uint64_t charged = 0;        // admitted requests' estimates + held result bytes
    uint64_t next_id = 1;
    bool stop = false;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
    bool fits(uint64_t est) const { return cfg.mem_budget == 0 || charged + est <= cfg.mem_budget || charged == 0; }
    void run(int slot);
};

// One worker per slot.  Admission is strictly in arrival order: the head of
// the queue waits for memory rather than being overtaken.
void odc_server::run(int slot) {
    cudaSetDevice(cfg.device);
    for (;;) {
        std::shared_ptr<Request> q;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_work.wait(lk, [&] { return (!queue.empty() && fits(queue.front()->est)) || (stop && queue.empty()); });
            if (queue.empty()) return;   // stop requested and nothing left
            q = queue.front();
            queue.pop_front();
            charged += q->est;
            q->slot = slot;
            q->t_start = now();
        }
        odc_mesh m{};
        odc_status s = odc_extract(ctx[slot], &q->src, &q->grid, &q->prm, streams[slot], &m);
        std::string err = s == ODC_OK ? std::string() : std::string(odc_last_error());
        cudaStream_t st = streams[slot];
        if (s == ODC_OK) {
            const size_t vb = (size_t)m.n_verts * 12, tb = (size_t)m.n_tris * 12;
            cudaError_t e = cudaSuccess;
            if (vb) e = cudaMallocAsync((void**)&q->d_verts, vb, st);
            if (e == cudaSuccess && tb) e = cudaMallocAsync((void**)&q->d_tris, tb, st);
            if (e == cudaSuccess && vb) e = cudaMemcpyAsync(q->d_verts, m.d_verts, vb, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess && tb) e = cudaMemcpyAsync(q->d_tris, m.d_tris, tb, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess && cfg.host_copy) {
                q->h_verts.resize((size_t)m.n_verts * 3);
                q->h_tris.resize((size_t)m.n_tris * 3);
                if (vb) e = cudaMemcpyAsync(q->h_verts.data(), m.d_verts, vb, cudaMemcpyDeviceToHost, st);
                if (e == cudaSuccess && tb) e = cudaMemcpyAsync(q->h_tris.data(), m.d_tris, tb, cudaMemcpyDeviceToHost, st);
            }
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) {
                cudaGetLastError();
                s = ODC_ERR_CUDA;
                err = std::string("result copy: ") + cudaGetErrorString(e);
            } else {
                q->result_bytes = vb + tb;
                q->mesh = m;
                q->mesh.d_verts = q->d_verts;
                q->mesh.d_tris = q->d_tris;
            }
        }
        {
            std::lock_guard<std::mutex> lk(mu);
            q->status = s;
            q->err = err;
            q->t_end = now();
            q->done = true;
            charged = charged - q->est + q->result_bytes;
        }
        cv_done.notify_all();
        cv_work.notify_all();
    }
}

static odc_status srv_fail(odc_status s, const std::string& msg) {
    odc::set_last_error(msg);
    return s;
}

static void free_result(odc_server* srv, Request& q) {
    if (q.d_verts) cudaFreeAsync(q.d_verts, srv->free_stream);
    if (q.d_tris) cudaFreeAsync(q.d_tris, srv->free_stream);
    q.d_verts = nullptr;
    q.d_tris = nullptr;
}

extern "C" {

odc_status odc_server_create(const odc_server_config* cfg, odc_server** out) {
    if (!cfg || !out) return srv_fail(ODC_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (cfg->slots < 1 || cfg->slots > 64) return srv_fail(ODC_ERR_INVALID_ARG, "slots out of [1, 64]");
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || cfg->device < 0 || cfg->device >= n)
        return srv_fail(ODC_ERR_INVALID_ARG, "no such CUDA device");
    cudaSetDevice(cfg->device);
    // keep freed stream-ordered memory (result buffers) cached in this
    // process's default pool instead of returning it at every synchronisation
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, cfg->device) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
    auto* srv = new odc_server();
    srv->cfg = *cfg;
    srv->t0 = Clock::now();
    for (int i = 0; i < cfg->slots; ++i) {
        odc_ctx* c = nullptr;
        cudaStream_t st = nullptr;
        odc_status s = odc_ctx_create(cfg->device, 0, &c);
        if (s == ODC_OK && cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) s = ODC_ERR_CUDA;
        if (c) srv->ctx.push_back(c);
        if (st) srv->streams.push_back(st);
        if (s != ODC_OK) {
            std::string msg = odc_last_error();
            odc_server_destroy(srv);
            return srv_fail(s, "server slot setup: " + msg);
        }
    }
    if (cfg->share_network) {
        odc_status s = odc_batch_create(cfg->device, &srv->batch);
        for (int i = 0; s == ODC_OK && i < cfg->slots; ++i) s = odc_ctx_join_batch(srv->ctx[i], srv->batch);
        if (s != ODC_OK) {
            std::string msg = odc_last_error();
            odc_server_destroy(srv);
            return srv_fail(s, "server batch group setup: " + msg);
        }
    }
    if (cudaStreamCreateWithFlags(&srv->free_stream, cudaStreamNonBlocking) != cudaSuccess) {
        odc_server_destroy(srv);
        return srv_fail(ODC_ERR_CUDA, "server stream setup failed");
    }
    for (int i = 0; i < cfg->slots; ++i) srv->workers.emplace_back(&odc_server::run, srv, i);
    *out = srv;
    return ODC_OK;
}

odc_status odc_server_destroy(odc_server* srv) {
    if (!srv) return ODC_OK;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
    }
    srv->cv_work.notify_all();
    for (auto& t : srv->workers)
        if (t.joinable()) t.join();
    cudaSetDevice(srv->cfg.device);
    for (auto& kv : srv->reqs) free_result(srv, *kv.second);
    if (srv->free_stream) {
        cudaStreamSynchronize(srv->free_stream);
        cudaStreamDestroy(srv->free_stream);
    }
    for (auto* c : srv->ctx) odc_ctx_destroy(c);
    odc_batch_destroy(srv->batch);   // after its members
    for (auto st : srv->streams) cudaStreamDestroy(st);
    delete srv;
    return ODC_OK;
}

odc_status odc_submit(odc_server* srv, const odc_source* src, const odc_grid* grid, const odc_params* prm,
                      uint64_t* req_id) {
    if (!srv || !src || !grid || !prm || !req_id) return srv_fail(ODC_ERR_INVALID_ARG, "NULL argument");
    auto q = std::make_shared<Request>();
    std::string err;
    odc_status s = copy_source(src, *q, &err);
    if (s != ODC_OK) return srv_fail(s, err);
    for (int a = 0; a < 3; ++a)
        if (grid->res[a] < 1 || grid->res[a] > 1024 || !(grid->lo[a] < grid->hi[a]))
            return srv_fail(ODC_ERR_INVALID_ARG, "grid: res in [1, 1024] and lo < hi required");
    q->grid = *grid;
    q->prm = *prm;
    q->est = estimate_bytes(q->src, q->grid);
    if (srv->cfg.mem_budget && q->est > srv->cfg.mem_budget)
        return srv_fail(ODC_ERR_OOM, "request estimate (" + std::to_string(q->est) + " bytes) exceeds the server budget");
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->stop) return srv_fail(ODC_ERR_INVALID_ARG, "server is shutting down");
        q->id = srv->next_id++;
        q->t_submit = srv->now();
        srv->reqs[q->id] = q;
        srv->queue.push_back(q);
        *req_id = q->id;
    }
    srv->cv_work.notify_all();
    return ODC_OK;
}

odc_status odc_poll(odc_server* srv, uint64_t req_id, int32_t timeout_ms, odc_result* out) {
    if (!srv || !out) return srv_fail(ODC_ERR_INVALID_ARG, "NULL argument");
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(req_id);
    if (it == srv->reqs.end()) return srv_fail(ODC_ERR_INVALID_ARG, "unknown request id");
    std::shared_ptr<Request> q = it->second;
    auto ready = [&] { return q->done; };
    if (timeout_ms < 0) srv->cv_done.wait(lk, ready);
    else if (!srv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
        return srv_fail(ODC_ERR_TIMEOUT, "request not finished");
    std::memset(out, 0, sizeof(*out));
    out->status = q->status;
    out->slot = q->slot;
    out->mesh = q->mesh;
    out->h_verts = q->h_verts.empty() ? nullptr : q->h_verts.data();
    out->h_tris = q->h_tris.empty() ? nullptr : q->h_tris.data();
    out->t_submit = q->t_submit;
    out->t_start = q->t_start;
    out->t_end = q->t_end;
    out->est_bytes = q->est;
    if (q->status != ODC_OK) odc::set_last_error(q->err);
    return ODC_OK;
}

odc_status odc_result_release(odc_server* srv, uint64_t req_id) {
    if (!srv) return srv_fail(ODC_ERR_INVALID_ARG, "NULL argument");
    std::shared_ptr<Request> q;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        auto it = srv->reqs.find(req_id);
        if (it == srv->reqs.end()) return srv_fail(ODC_ERR_INVALID_ARG, "unknown request id");
        if (!it->second->done) return srv_fail(ODC_ERR_INVALID_ARG, "request not finished");
        q = it->second;
        srv->reqs.erase(it);
        srv->charged -= q->result_bytes;
    }
    cudaSetDevice(srv->cfg.device);
    free_result(srv, *q);
    srv->cv_work.notify_all();
    return ODC_OK;
}

double odc_server_clock(const odc_server* srv) { return srv ? srv->now() : 0.0; }

}  // extern "C"
