// Serving front end: a queue of kernel-column requests executed concurrently on a fixed set
// of CUDA streams, with admission by scratch footprint.
//
// Each request is one kb_krylov_apply call.  The server owns `streams` worker threads, each
// with its own CUDA stream; a worker takes the oldest pending request once the scratch it
// needs (kb_workspace_bytes) fits in the memory budget next to the requests in flight, runs
// it on its stream and waits for it (so the result's kb_info is available), then records
// the completion time.  Requests therefore complete out of submission order, but they are
// started in submission order (no request overtakes an older one that does not fit yet).
// Latency is measured on the host from kb_server_submit to the end of the solve.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "kb_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    kb_graph *g = nullptr;
    kb_method method = KB_CBL;
    kb_phi phi = KB_PHI_EXP;
    kb_params params{};
    std::vector<int32_t> nodes;
    int32_t m = 0;
    float *Y = nullptr;
    size_t bytes = 0;
    int state = 0;   // 0 pending, 1 running, 2 done
    int rc = KB_OK;
    std::string msg;
    kb_info info{};
    Clock::time_point t_submit, t_done;
};

}  // namespace

struct kb_server {
    int device = 0;
    size_t budget = 0;
    size_t in_use = 0;
    int32_t capacity = 0;
    int32_t fallback_sbl = 0;
    bool stopping = false;
    int64_t next_ticket = 1;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<int64_t> pending;
    std::unordered_map<int64_t, Request> reqs;
    std::vector<cudaStream_t> streams;
    std::vector<std::thread> workers;
};

namespace {

void worker_loop(kb_server *sv, int w) {
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    for (;;) {
        sv->cv_work.wait(lk, [&] {
            if (sv->pending.empty()) return sv->stopping;
            const Request &r = sv->reqs[sv->pending.front()];
            return sv->in_use + r.bytes <= sv->budget;
        });
        if (sv->pending.empty()) return;   // stopping with nothing left to run
        const int64_t ticket = sv->pending.front();
        sv->pending.pop_front();
        Request &r = sv->reqs[ticket];
        r.state = 1;
        sv->in_use += r.bytes;
        // the request is not erased while running (poll erases only finished requests)
        kb_graph *g = r.g;
        const kb_method method = r.method;
        const kb_phi phi = r.phi;
        const kb_params params = r.params;
        const int32_t *nodes = r.nodes.data();
        const int32_t M = int32_t(r.nodes.size());
        const int32_t m = r.m;
        float *Y = r.Y;
        const uint64_t r_bytes = r.bytes;
        lk.unlock();
        kb_info info{};
        int rc = kb_krylov_apply(g, method, phi, &params, nodes, M, m, Y, sv->streams[w], &info);
        if (rc == KB_ERR_BREAKDOWN && sv->fallback_sbl && (method == KB_CBL || method == KB_GBL)) {
            // rank-deficient block: one Lanczos process per column instead, when its scratch
            // fits what the request was admitted with
            kb_params p2 = params;
            p2.reorth = 0;
            p2.tol = 0.0;   // the stopping rule is a cbl feature: sbl runs the m steps
            uint64_t need = 0;
            if (kb_workspace_bytes(g, KB_SBL, phi, &p2, M, m, &need) == KB_OK && need <= r_bytes) {
                const int32_t bstep = info.breakdown_step;
                kb_info info2{};
                rc = kb_krylov_apply(g, KB_SBL, phi, &p2, nodes, M, m, Y, sv->streams[w], &info2);
                info = info2;
                info.breakdown_step = bstep;
            }
        }
        std::string msg = rc ? std::string(kb_last_error()) : std::string();
        const Clock::time_point t = Clock::now();
        lk.lock();
        Request &r2 = sv->reqs[ticket];
        r2.rc = rc;
        r2.msg = msg;
        r2.info = info;
        r2.t_done = t;
        r2.state = 2;
        sv->in_use -= r2.bytes;
        sv->cv_done.notify_all();
        sv->cv_work.notify_all();
    }
}

}  // namespace

using namespace kb;

extern "C" int kb_server_create(int32_t device, const kb_server_config *cfg, kb_server **out) {
    try {
        if (!cfg || !out) return fail(KB_ERR_ARG, "config or out is NULL");
        if (cfg->streams < 1 || cfg->streams > 64) return fail(KB_ERR_ARG, "streams must be in [1, 64]");
        if (cfg->queue_capacity < 1) return fail(KB_ERR_ARG, "queue_capacity must be >= 1");
        DeviceGuard dg;
        KB_CUDA_TRY(dg.set(device));
        size_t budget = 0;
        if (cfg->memory_budget > 0) {
            budget = size_t(cfg->memory_budget);
        } else {
            // the solves allocate from the device's stream-ordered pool, which keeps what
            // earlier solves freed (release threshold raised): memory it holds but does not
            // use counts as available too
            size_t fr = 0, tot = 0;
            KB_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
            cudaMemPool_t pool;
            if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
                uint64_t reserved = 0, used = 0;
                if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved) == cudaSuccess &&
                    cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) == cudaSuccess &&
                    reserved > used)
                    fr += size_t(reserved - used);
            }
            budget = fr / 4 * 3;
        }
        auto *sv = new kb_server();
        sv->device = device;
        sv->budget = budget;
        sv->capacity = cfg->queue_capacity;
        sv->fallback_sbl = cfg->fallback_sbl ? 1 : 0;
        for (int i = 0; i < cfg->streams; ++i) {
            cudaStream_t s = nullptr;
            cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
            if (e != cudaSuccess) {
                for (cudaStream_t s2 : sv->streams) cudaStreamDestroy(s2);
                delete sv;
                return cuda_fail(e, "cudaStreamCreateWithFlags");
            }
            sv->streams.push_back(s);
        }
        for (int i = 0; i < cfg->streams; ++i) sv->workers.emplace_back(worker_loop, sv, i);
        *out = sv;
        return KB_OK;
    } catch (const std::bad_alloc &) {
        return fail(KB_ERR_NOMEM, "host allocation failed");
    } catch (...) {
        return fail(KB_ERR_CUDA, "unexpected exception");
    }
}

extern "C" int kb_server_submit(kb_server *sv, kb_graph *g, kb_method method, kb_phi phi,
                                const kb_params *params, const int32_t *nodes, int32_t M,
                                int32_t m, float *Y, int64_t *ticket) {
    try {
        if (!sv || !g || !params || !nodes || !Y || !ticket) return fail(KB_ERR_ARG, "NULL argument");
        if (M < 1 || M > g->dev.n) return fail(KB_ERR_ARG, "M out of range");
        size_t bytes = 0;
        int rc = kb_workspace_bytes(g, method, phi, params, M, m, &bytes);
        if (rc) return rc;
        if (bytes > sv->budget) return fail(KB_ERR_NOMEM, "request scratch exceeds the server memory budget");
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->stopping) return fail(KB_ERR_ARG, "server is shutting down");
        if (int64_t(sv->reqs.size()) >= sv->capacity) return fail(KB_ERR_BUSY, "request queue is full");
        const int64_t t = sv->next_ticket++;
        Request &r = sv->reqs[t];
        r.g = g;
        r.method = method;
        r.phi = phi;
        r.params = *params;
        r.nodes.assign(nodes, nodes + M);
        r.m = m;
        r.Y = Y;
        r.bytes = bytes;
        r.t_submit = Clock::now();
        sv->pending.push_back(t);
        *ticket = t;
        sv->cv_work.notify_all();
        return KB_OK;
    } catch (const std::bad_alloc &) {
        return fail(KB_ERR_NOMEM, "host allocation failed");
    } catch (...) {
        return fail(KB_ERR_CUDA, "unexpected exception");
    }
}

extern "C" int kb_server_poll(kb_server *sv, int64_t ticket, int32_t wait_ms, kb_info *info,
                              double *latency_ms) {
    try {
        if (!sv) return fail(KB_ERR_ARG, "server is NULL");
        std::unique_lock<std::mutex> lk(sv->mu);
        auto it = sv->reqs.find(ticket);
        if (it == sv->reqs.end()) return fail(KB_ERR_ARG, "unknown ticket");
        if (it->second.state != 2 && wait_ms != 0) {
            auto done = [&] {
                auto j = sv->reqs.find(ticket);
                return j != sv->reqs.end() && j->second.state == 2;
            };
            if (wait_ms < 0) sv->cv_done.wait(lk, done);
            else sv->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), done);
            it = sv->reqs.find(ticket);
        }
        if (it->second.state != 2) return KB_PENDING;
        const Request &r = it->second;
        if (info) *info = r.info;
        if (latency_ms)
            *latency_ms = std::chrono::duration<double, std::milli>(r.t_done - r.t_submit).count();
        const int rc = r.rc;
        const std::string msg = r.msg;
        sv->reqs.erase(it);
        if (rc) return fail(rc, msg);
        return KB_OK;
    } catch (...) {
        return fail(KB_ERR_CUDA, "unexpected exception");
    }
}

extern "C" int kb_server_destroy(kb_server *sv) {
    if (!sv) return KB_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stopping = true;
        sv->cv_work.notify_all();
    }
    for (std::thread &t : sv->workers) t.join();
    for (cudaStream_t s : sv->streams) cudaStreamDestroy(s);
    delete sv;
    return KB_OK;
}
