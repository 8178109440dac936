// Serving layer of the application phase (include/defmm_serve.h): caller
// workspaces, graph-replayed batches of applies, and the request server.
// Every apply here is launch_apply, the kernels of defmm_apply; this file only
// organises scratch memory, streams, graphs and requests around it.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "defmm.h"
#include "defmm_serve.h"
#include "kernels.cuh"
#include "plan_state.h"

using defmm::set_error;

namespace {

defmm_status cuda_err(cudaError_t e, const char* what) {
    const defmm_status s = e == cudaErrorMemoryAllocation ? DEFMM_ERR_OOM : DEFMM_ERR_CUDA;
    cudaGetLastError();
    return set_error(s, std::string(what) + ": " + cudaGetErrorString(e));
}

size_t csize(defmm_dtype d) { return d == DEFMM_C64 ? 8 : 16; }
size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Scratch of one apply, carved from one region in this order at 256-byte
// boundaries: qs (ny), ps (nx), M (multipoles x p^3), Mhat (Fourier
// multipoles x NFpad), L (locals x p^3), part (near-field partial sums), each
// times R right-hand sides.
struct Carve {
    size_t qs, ps, M, Mhat, L, part, total;
};
Carve carve(const defmm::HostPlan& hp, int R, defmm_dtype d) {
    const size_t c = csize(d) * (size_t)R;
    Carve k{};
    size_t off = 0;
    auto take = [&](size_t count) {
        const size_t start = align256(off);
        off = start + count * c;
        return start;
    };
    k.qs = take((size_t)hp.ny);
    k.ps = take((size_t)hp.nx);
    k.M = take((size_t)std::max<int64_t>(1, hp.nM()) * hp.P3);
    k.Mhat = take(std::max<size_t>(1, hp.m2f_list.size()) * hp.NFpad);
    k.L = take((size_t)std::max<int64_t>(1, hp.nL()) * hp.P3);
    k.part = take((size_t)std::max<int64_t>(1, hp.p2p_parts));
    k.total = align256(off);
    return k;
}

defmm_status check_plan(defmm_plan plan) {
    if (!plan) return set_error(DEFMM_ERR_ARG, "plan is NULL");
    if (plan->host_only) return set_error(DEFMM_ERR_UNSUPPORTED, "plan was built with DEFMM_PLAN_HOST_ONLY");
    return DEFMM_OK;
}

}  // namespace

struct defmm_workspace_s {
    defmm_plan plan = nullptr;
    defmm_dtype dtype = DEFMM_C64;
    int R = 0;
    bool owned = false;
    unsigned char* mem = nullptr;
    Carve k{};
    int64_t launches = 0;   // kernels launched by the last apply through this workspace
};

namespace {

const defmm::DevTyped<float>& typed_tables(const defmm_plan_s* pl, float*) { return pl->tf; }
const defmm::DevTyped<double>& typed_tables(const defmm_plan_s* pl, double*) { return pl->td; }

template <typename T>
cudaError_t apply_with(defmm_plan pl, defmm_workspace ws, const void* q, void* p, int R, cudaStream_t stream) {
    using C = typename defmm::Cplx<T>::type;
    defmm::DevWork<T> w;
    w.R = R;
    w.qs = reinterpret_cast<C*>(ws->mem + ws->k.qs);
    w.ps = reinterpret_cast<C*>(ws->mem + ws->k.ps);
    w.M = reinterpret_cast<C*>(ws->mem + ws->k.M);
    w.Mhat = reinterpret_cast<C*>(ws->mem + ws->k.Mhat);
    w.L = reinterpret_cast<C*>(ws->mem + ws->k.L);
    w.part = reinterpret_cast<C*>(ws->mem + ws->k.part);
    w.nL = pl->hp.nL();
    const defmm::DevTyped<T>& typed = typed_tables(pl, (T*)nullptr);
    int launches = 0;
    // the whole operator whatever the plan's shard setting (documented in defmm_serve.h)
    cudaError_t e = defmm::launch_apply<T>(pl->common, typed, w, pl->m2m.data(), (int)pl->m2m.size(), pl->l2l.data(),
                                           pl->l2l_par.data(), (int)pl->l2l.size(), q, p, stream, &launches, nullptr);
    ws->launches = launches;
    return e;
}

defmm_status apply_ws_unchecked(defmm_plan plan, defmm_workspace ws, const void* q, void* p, int nrhs,
                                cudaStream_t stream) {
    cudaError_t e = ws->dtype == DEFMM_C64 ? apply_with<float>(plan, ws, q, p, nrhs, stream)
                                           : apply_with<double>(plan, ws, q, p, nrhs, stream);
    if (e != cudaSuccess) return cuda_err(e, "apply launch");
    return DEFMM_OK;
}

defmm_status new_workspace(defmm_plan plan, int nrhs, defmm_dtype dtype, void* mem, size_t bytes, bool own,
                           defmm_workspace* out) {
    defmm_status s = check_plan(plan);
    if (s != DEFMM_OK) return s;
    if (!out) return set_error(DEFMM_ERR_ARG, "out is NULL");
    if (nrhs < 1) return set_error(DEFMM_ERR_ARG, "nrhs must be >= 1");
    if (dtype != DEFMM_C64 && dtype != DEFMM_C128) return set_error(DEFMM_ERR_UNSUPPORTED, "dtype");
    const Carve k = carve(plan->hp, nrhs, dtype);
    if (own) {
        cudaError_t e = cudaMalloc(&mem, k.total);
        if (e != cudaSuccess) return cuda_err(e, "workspace allocation");
    } else {
        if (!mem) return set_error(DEFMM_ERR_ARG, "mem is NULL");
        if (reinterpret_cast<uintptr_t>(mem) % 256) return set_error(DEFMM_ERR_ARG, "mem must be 256-byte aligned");
        if (bytes < k.total)
            return set_error(DEFMM_ERR_ARG, "workspace memory too small: " + std::to_string(bytes) + " < " +
                                                std::to_string(k.total) + " bytes");
    }
    defmm_workspace ws = new defmm_workspace_s;
    ws->plan = plan;
    ws->dtype = dtype;
    ws->R = nrhs;
    ws->owned = own;
    ws->mem = static_cast<unsigned char*>(mem);
    ws->k = k;
    *out = ws;
    return DEFMM_OK;
}

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace

// ------------------------------------------------------------------ workspaces
extern "C" defmm_status defmm_workspace_bytes(defmm_plan plan, int nrhs, defmm_dtype dtype, size_t* bytes) {
    if (!plan || !bytes) return set_error(DEFMM_ERR_ARG, "plan and bytes must not be NULL");
    if (nrhs < 1) return set_error(DEFMM_ERR_ARG, "nrhs must be >= 1");
    if (dtype != DEFMM_C64 && dtype != DEFMM_C128) return set_error(DEFMM_ERR_UNSUPPORTED, "dtype");
    *bytes = carve(plan->hp, nrhs, dtype).total;
    return DEFMM_OK;
}

extern "C" defmm_status defmm_workspace_create(defmm_plan plan, int nrhs, defmm_dtype dtype, defmm_workspace* out) {
    return new_workspace(plan, nrhs, dtype, nullptr, 0, true, out);
}

extern "C" defmm_status defmm_workspace_wrap(defmm_plan plan, int nrhs, defmm_dtype dtype, void* mem, size_t bytes,
                                             defmm_workspace* out) {
    return new_workspace(plan, nrhs, dtype, mem, bytes, false, out);
}

extern "C" defmm_status defmm_workspace_destroy(defmm_workspace ws) {
    if (!ws) return DEFMM_OK;
    if (ws->owned) cudaFree(ws->mem);
    delete ws;
    return DEFMM_OK;
}

extern "C" defmm_status defmm_apply_ws(defmm_plan plan, defmm_workspace ws, const void* q, void* p, int nrhs,
                                       defmm_dtype dtype, void* stream) {
    defmm_status s = check_plan(plan);
    if (s != DEFMM_OK) return s;
    if (!ws) return set_error(DEFMM_ERR_ARG, "workspace is NULL");
    if (ws->plan != plan) return set_error(DEFMM_ERR_ARG, "workspace belongs to another plan");
    if (!q || !p) return set_error(DEFMM_ERR_ARG, "q and p must be device pointers");
    if (nrhs < 1 || nrhs > ws->R)
        return set_error(DEFMM_ERR_ARG, "nrhs must be in [1, " + std::to_string(ws->R) + "] for this workspace");
    if (dtype != ws->dtype) return set_error(DEFMM_ERR_ARG, "dtype differs from the workspace's");
    return apply_ws_unchecked(plan, ws, q, p, nrhs, (cudaStream_t)stream);
}

// ------------------------------------------------------------------ graph batches
struct defmm_batch_s {
    std::vector<defmm_plan> plans;
    std::vector<int> nrhs;
    defmm_dtype dtype = DEFMM_C64;
    std::vector<defmm_workspace> ws;
    cudaStream_t origin = nullptr;
    std::vector<cudaStream_t> side;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<const void*> q_last;
    std::vector<void*> p_last;
    int64_t launches = 0, nodes = 0;
    std::mutex busy;

    void release() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        for (cudaEvent_t e : join) cudaEventDestroy(e);
        if (fork) cudaEventDestroy(fork);
        for (cudaStream_t s : side) cudaStreamDestroy(s);
        if (origin) cudaStreamDestroy(origin);
        for (defmm_workspace w : ws) defmm_workspace_destroy(w);
    }
};

namespace {

// Records every entry's apply into a new graph: fork from the origin stream
// to the side streams, entry i on side stream i mod branches, join back.
defmm_status capture(defmm_batch b, const void* const* q, void* const* p, cudaGraph_t* out, int64_t* launches) {
    cudaError_t e = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_err(e, "begin graph capture");
    defmm_status st = DEFMM_OK;
    int64_t nl = 0;
    e = cudaEventRecord(b->fork, b->origin);
    for (size_t k = 0; e == cudaSuccess && k < b->side.size(); ++k) e = cudaStreamWaitEvent(b->side[k], b->fork, 0);
    for (size_t i = 0; e == cudaSuccess && st == DEFMM_OK && i < b->plans.size(); ++i) {
        st = apply_ws_unchecked(b->plans[i], b->ws[i], q[i], p[i], b->nrhs[i], b->side[i % b->side.size()]);
        nl += b->ws[i]->launches;
    }
    for (size_t k = 0; e == cudaSuccess && st == DEFMM_OK && k < b->side.size(); ++k) {
        e = cudaEventRecord(b->join[k], b->side[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->origin, b->join[k], 0);
    }
    cudaGraph_t g = nullptr;
    cudaError_t e_end = cudaStreamEndCapture(b->origin, &g);
    if (st != DEFMM_OK || e != cudaSuccess || e_end != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        if (st != DEFMM_OK) return st;
        return cuda_err(e != cudaSuccess ? e : e_end, "graph capture");
    }
    *out = g;
    *launches = nl;
    return DEFMM_OK;
}

}  // namespace

extern "C" defmm_status defmm_batch_create(const defmm_plan* plans, const int* nrhs, int n, defmm_dtype dtype,
                                           int branches, defmm_batch* out) {
    if (!plans || !nrhs || !out || n < 1) return set_error(DEFMM_ERR_ARG, "plans, nrhs, out and n >= 1 required");
    if (branches < 0 || branches > 64) return set_error(DEFMM_ERR_ARG, "branches must be in [0, 64]");
    if (dtype != DEFMM_C64 && dtype != DEFMM_C128) return set_error(DEFMM_ERR_UNSUPPORTED, "dtype");
    for (int i = 0; i < n; ++i) {
        defmm_status s = check_plan(plans[i]);
        if (s != DEFMM_OK) return s;
        if (nrhs[i] < 1) return set_error(DEFMM_ERR_ARG, "nrhs[i] must be >= 1");
    }
    if (branches == 0) branches = n < 8 ? n : 8;
    if (branches > n) branches = n;
    std::unique_ptr<defmm_batch_s> b(new defmm_batch_s);
    b->plans.assign(plans, plans + n);
    b->nrhs.assign(nrhs, nrhs + n);
    b->dtype = dtype;
    for (int i = 0; i < n; ++i) {
        defmm_workspace w = nullptr;
        defmm_status s = defmm_workspace_create(plans[i], nrhs[i], dtype, &w);
        if (s != DEFMM_OK) {
            b->release();
            return s;
        }
        b->ws.push_back(w);
    }
    cudaError_t e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    for (int k = 0; e == cudaSuccess && k < branches; ++k) {
        cudaStream_t s = nullptr;
        cudaEvent_t ev = nullptr;
        e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e == cudaSuccess) b->side.push_back(s);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) b->join.push_back(ev);
    }
    if (e != cudaSuccess) {
        b->release();
        return cuda_err(e, "batch streams");
    }
    *out = b.release();
    return DEFMM_OK;
}

extern "C" defmm_status defmm_batch_apply(defmm_batch b, const void* const* q, void* const* p, void* stream) {
    if (!b || !q || !p) return set_error(DEFMM_ERR_ARG, "batch, q and p must not be NULL");
    std::unique_lock<std::mutex> lk(b->busy, std::try_to_lock);
    if (!lk.owns_lock()) return set_error(DEFMM_ERR_BUSY, "batch is being applied by another thread");
    const size_t n = b->plans.size();
    for (size_t i = 0; i < n; ++i)
        if (!q[i] || !p[i]) return set_error(DEFMM_ERR_ARG, "q[i] and p[i] must be device pointers");
    bool same = b->exec != nullptr;
    for (size_t i = 0; same && i < n; ++i) same = b->q_last[i] == q[i] && b->p_last[i] == p[i];
    if (!same) {
        cudaGraph_t g = nullptr;
        int64_t nl = 0;
        defmm_status s = capture(b, q, p, &g, &nl);
        if (s != DEFMM_OK) return s;
        cudaError_t e = cudaSuccess;
        bool updated = false;
        if (b->exec) {
            cudaGraphExecUpdateResultInfo info;
            updated = cudaGraphExecUpdate(b->exec, g, &info) == cudaSuccess;
            if (!updated) {
                cudaGetLastError();
                cudaGraphExecDestroy(b->exec);
                b->exec = nullptr;
            }
        }
        if (!updated) e = cudaGraphInstantiate(&b->exec, g, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            b->exec = nullptr;
            return cuda_err(e, "graph instantiation");
        }
        if (b->graph) cudaGraphDestroy(b->graph);
        b->graph = g;
        size_t count = 0;
        cudaGraphGetNodes(g, nullptr, &count);
        b->nodes = (int64_t)count;
        b->launches = nl;
        b->q_last.assign(q, q + n);
        b->p_last.assign(p, p + n);
    }
    cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_err(e, "graph launch");
    return DEFMM_OK;
}

extern "C" defmm_status defmm_batch_info(defmm_batch b, int64_t* kernel_launches, int64_t* graph_nodes) {
    if (!b) return set_error(DEFMM_ERR_ARG, "batch is NULL");
    if (kernel_launches) *kernel_launches = b->launches;
    if (graph_nodes) *graph_nodes = b->nodes;
    return DEFMM_OK;
}

extern "C" defmm_status defmm_batch_destroy(defmm_batch b) {
    if (!b) return DEFMM_OK;
    {
        std::lock_guard<std::mutex> lk(b->busy);
    }
    b->release();
    delete b;
    return DEFMM_OK;
}

// ------------------------------------------------------------------ request server
namespace {

// First-fit allocator over one device region, 256-byte granules.
class Arena {
  public:
    void reset(size_t size) {
        free_.clear();
        if (size) free_[0] = size;
        size_ = size;
        used_ = 0;
    }
    bool alloc(size_t bytes, size_t* off) {
        bytes = align256(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            *off = it->first;
            const size_t rest = it->second - bytes, start = it->first + bytes;
            free_.erase(it);
            if (rest) free_[start] = rest;
            used_ += bytes;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = align256(bytes);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }
    size_t size() const { return size_; }

  private:
    std::map<size_t, size_t> free_;
    size_t size_ = 0, used_ = 0;
};

enum ReqState { kQueued, kRunning, kDone, kFailed };

struct Request {
    int g = 0, R = 0;
    const void* q = nullptr;
    void* p = nullptr;
    double t_submit = 0, t_done = 0;
    ReqState state = kQueued;
};

}  // namespace

struct defmm_server_s;

namespace {

struct Batch {
    defmm_server_s* server = nullptr;
    int stream = 0, g = 0, R = 0;
    std::vector<std::shared_ptr<Request>> reqs;
    size_t off = 0, bytes = 0;
    defmm_workspace ws = nullptr;
    bool done = false;
    double t_done = 0;
};

void CUDART_CB batch_done(void* arg);

}  // namespace

struct defmm_server_s {
    std::vector<defmm_plan> plans;
    defmm_dtype dtype = DEFMM_C64;
    defmm_server_options opt{};
    int device = 0;
    unsigned char* arena_mem = nullptr;
    Arena arena;
    std::vector<cudaStream_t> streams;
    std::vector<bool> stream_busy;
    std::deque<uint64_t> pending;
    std::unordered_map<uint64_t, std::shared_ptr<Request>> reqs;
    std::vector<Batch*> inflight;
    uint64_t next_id = 1;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false, failed = false, mem_blocked = false;
    std::string fail_msg;
    defmm_server_stats st{};
    std::thread worker;

    size_t batch_bytes(int g, int R) const {
        const defmm::HostPlan& hp = plans[g]->hp;
        return carve(hp, R, dtype).total + align256(csize(dtype) * (size_t)R * hp.ny) +
               align256(csize(dtype) * (size_t)R * hp.nx);
    }
    int free_stream() const {
        for (size_t k = 0; k < stream_busy.size(); ++k)
            if (!stream_busy[k]) return (int)k;
        return -1;
    }
    bool any_done() const {
        for (const Batch* b : inflight)
            if (b->done) return true;
        return false;
    }

    // Copies in, one apply, copies out, completion callback; no lock held.
    cudaError_t launch(Batch* b) {
        const defmm::HostPlan& hp = plans[b->g]->hp;
        const size_t cs = csize(dtype);
        const Carve k = carve(hp, b->R, dtype);
        unsigned char* base = arena_mem + b->off;
        unsigned char* qd = base + k.total;
        unsigned char* pd = qd + align256(cs * (size_t)b->R * hp.ny);
        defmm_workspace ws = nullptr;
        if (new_workspace(plans[b->g], b->R, dtype, base, k.total, false, &ws) != DEFMM_OK) return cudaErrorInvalidValue;
        b->ws = ws;
        cudaStream_t s = streams[b->stream];
        cudaError_t e = cudaSuccess;
        size_t col = 0;
        for (auto& r : b->reqs) {
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(qd + col * hp.ny * cs, r->q, cs * (size_t)r->R * hp.ny, cudaMemcpyHostToDevice, s);
            col += r->R;
        }
        if (e == cudaSuccess && apply_ws_unchecked(plans[b->g], ws, qd, pd, b->R, s) != DEFMM_OK)
            e = cudaErrorLaunchFailure;
        col = 0;
        for (auto& r : b->reqs) {
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(r->p, pd + col * hp.nx * cs, cs * (size_t)r->R * hp.nx, cudaMemcpyDeviceToHost, s);
            col += r->R;
        }
        if (e == cudaSuccess) e = cudaLaunchHostFunc(s, batch_done, b);
        return e;
    }

    void retire(std::unique_lock<std::mutex>&) {
        for (size_t i = 0; i < inflight.size();) {
            Batch* b = inflight[i];
            if (!b->done) {
                ++i;
                continue;
            }
            for (auto& r : b->reqs) {
                r->state = kDone;
                r->t_done = b->t_done;
                ++st.completed;
            }
            arena.release(b->off, b->bytes);
            stream_busy[b->stream] = false;
            delete b->ws;   // wrapped: owns no memory
            delete b;
            inflight.erase(inflight.begin() + (long)i);
            mem_blocked = false;
        }
        cv_done.notify_all();
    }

    // Oldest waiting request plus later ones on its geometry, up to max_batch_rhs.
    Batch* form(int stream_idx) {
        const uint64_t first = pending.front();
        const int g = reqs[first]->g;
        Batch* b = new Batch;
        b->server = this;
        b->stream = stream_idx;
        b->g = g;
        std::vector<uint64_t> take;
        int R = 0;
        for (uint64_t id : pending) {
            const auto& r = reqs[id];
            if (r->g != g) continue;
            if (!take.empty() && R + r->R > opt.max_batch_rhs) break;
            take.push_back(id);
            R += r->R;
            if (R >= opt.max_batch_rhs) break;
        }
        // shrink until it fits in the arena (a lone request always fits: checked at submit)
        while (true) {
            b->R = R;
            b->bytes = batch_bytes(g, R);
            if (arena.alloc(b->bytes, &b->off)) break;
            if (take.size() == 1) {
                delete b;
                return nullptr;
            }
            R -= reqs[take.back()]->R;
            take.pop_back();
        }
        for (uint64_t id : take) {
            auto& r = reqs[id];
            r->state = kRunning;
            b->reqs.push_back(r);
            for (auto it = pending.begin(); it != pending.end(); ++it)
                if (*it == id) {
                    pending.erase(it);
                    break;
                }
        }
        return b;
    }

    void run() {
        cudaSetDevice(device);
        std::unique_lock<std::mutex> lk(mu);
        while (true) {
            retire(lk);
            while (!failed && !pending.empty() && !mem_blocked) {
                const int k = free_stream();
                if (k < 0) break;
                Batch* b = form(k);
                if (!b) {
                    mem_blocked = true;   // wait for a running batch to free memory
                    break;
                }
                stream_busy[k] = true;
                inflight.push_back(b);
                ++st.batches;
                st.rhs_applied += b->R;
                if ((int64_t)b->reqs.size() > st.max_batch_requests) st.max_batch_requests = (int64_t)b->reqs.size();
                if ((int64_t)inflight.size() > st.max_inflight) st.max_inflight = (int64_t)inflight.size();
                if (arena.used() > st.peak_arena_bytes) st.peak_arena_bytes = arena.used();
                lk.unlock();
                const cudaError_t e = launch(b);
                lk.lock();
                if (b->ws) st.kernel_launches += b->ws->launches;
                if (e != cudaSuccess) {
                    failed = true;
                    fail_msg = std::string("server batch launch: ") + cudaGetErrorString(e);
                    cudaGetLastError();
                    // the stream may still run part of the batch: wait for it before failing the requests
                    lk.unlock();
                    cudaStreamSynchronize(streams[k]);
                    lk.lock();
                    for (auto& r : b->reqs) r->state = kFailed;
                    arena.release(b->off, b->bytes);
                    stream_busy[k] = false;
                    inflight.erase(std::find(inflight.begin(), inflight.end(), b));
                    delete b->ws;
                    delete b;
                    cv_done.notify_all();
                }
            }
            if (failed)
                for (uint64_t id : pending) reqs[id]->state = kFailed;
            if (failed) pending.clear(), cv_done.notify_all();
            if (stop && pending.empty() && inflight.empty()) break;
            cv_work.wait(lk, [&] {
                return any_done() || (stop && pending.empty() && inflight.empty()) ||
                       (!pending.empty() && !mem_blocked && free_stream() >= 0 && !failed);
            });
        }
    }
};

namespace {

void CUDART_CB batch_done(void* arg) {
    Batch* b = static_cast<Batch*>(arg);
    defmm_server_s* s = b->server;
    std::lock_guard<std::mutex> lk(s->mu);
    b->done = true;
    b->t_done = now_ms();
    s->cv_work.notify_one();
}

}  // namespace

extern "C" void defmm_server_default_options(defmm_server_options* opt) {
    if (!opt) return;
    opt->streams = 4;
    opt->max_batch_rhs = 16;
    opt->hbm_budget = size_t(4) << 30;
}

extern "C" defmm_status defmm_server_create(const defmm_plan* plans, int nplans, defmm_dtype dtype,
                                            const defmm_server_options* opt, defmm_server* out) {
    if (!plans || nplans < 1 || !out) return set_error(DEFMM_ERR_ARG, "plans, nplans >= 1 and out required");
    if (dtype != DEFMM_C64 && dtype != DEFMM_C128) return set_error(DEFMM_ERR_UNSUPPORTED, "dtype");
    for (int i = 0; i < nplans; ++i) {
        defmm_status s = check_plan(plans[i]);
        if (s != DEFMM_OK) return s;
    }
    defmm_server_options o;
    defmm_server_default_options(&o);
    if (opt) o = *opt;
    if (o.streams < 1 || o.streams > 32) return set_error(DEFMM_ERR_ARG, "streams must be in [1, 32]");
    if (o.max_batch_rhs < 1) return set_error(DEFMM_ERR_ARG, "max_batch_rhs must be >= 1");
    if (o.hbm_budget < 256) return set_error(DEFMM_ERR_ARG, "hbm_budget too small");
    std::unique_ptr<defmm_server_s> s(new defmm_server_s);
    s->plans.assign(plans, plans + nplans);
    s->dtype = dtype;
    s->opt = o;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaMalloc(&s->arena_mem, align256(o.hbm_budget));
    if (e != cudaSuccess) return cuda_err(e, "server arena");
    s->arena.reset(align256(o.hbm_budget));
    s->st.arena_bytes = s->arena.size();
    for (int k = 0; k < o.streams; ++k) {
        cudaStream_t st = nullptr;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
            cudaFree(s->arena_mem);
            return cuda_err(e, "server streams");
        }
        s->streams.push_back(st);
        s->stream_busy.push_back(false);
    }
    defmm_server_s* raw = s.release();
    raw->worker = std::thread([raw] { raw->run(); });
    *out = raw;
    return DEFMM_OK;
}

extern "C" defmm_status defmm_server_submit(defmm_server s, int geometry, const void* q_host, void* p_host, int nrhs,
                                            uint64_t* ticket) {
    if (!s || !q_host || !p_host || !ticket) return set_error(DEFMM_ERR_ARG, "server, q_host, p_host, ticket required");
    if (geometry < 0 || geometry >= (int)s->plans.size()) return set_error(DEFMM_ERR_ARG, "geometry out of range");
    if (nrhs < 1) return set_error(DEFMM_ERR_ARG, "nrhs must be >= 1");
    const size_t need = s->batch_bytes(geometry, nrhs);
    if (align256(need) > s->arena.size())
        return set_error(DEFMM_ERR_UNSUPPORTED, "request needs " + std::to_string(need) + " bytes, more than the " +
                                                    std::to_string(s->arena.size()) + "-byte arena");
    auto r = std::make_shared<Request>();
    r->g = geometry;
    r->R = nrhs;
    r->q = q_host;
    r->p = p_host;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->failed) return set_error(DEFMM_ERR_CUDA, s->fail_msg);
        if (s->stop) return set_error(DEFMM_ERR_ARG, "server is stopping");
        r->t_submit = now_ms();
        const uint64_t id = s->next_id++;
        s->reqs[id] = r;
        s->pending.push_back(id);
        ++s->st.submitted;
        *ticket = id;
    }
    s->cv_work.notify_one();
    return DEFMM_OK;
}

extern "C" defmm_status defmm_server_wait(defmm_server s, uint64_t ticket, double timeout_ms, double* latency_ms) {
    if (!s) return set_error(DEFMM_ERR_ARG, "server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return set_error(DEFMM_ERR_ARG, "unknown ticket");
    std::shared_ptr<Request> r = it->second;
    auto finished = [&] { return r->state == kDone || r->state == kFailed; };
    if (timeout_ms < 0) s->cv_done.wait(lk, finished);
    else s->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), finished);
    if (!finished()) return set_error(DEFMM_ERR_TIMEOUT, "request not finished yet");
    s->reqs.erase(ticket);
    if (r->state == kFailed) return set_error(DEFMM_ERR_CUDA, s->fail_msg.empty() ? "request failed" : s->fail_msg);
    if (latency_ms) *latency_ms = r->t_done - r->t_submit;
    return DEFMM_OK;
}

extern "C" defmm_status defmm_server_get_stats(defmm_server s, defmm_server_stats* out) {
    if (!s || !out) return set_error(DEFMM_ERR_ARG, "server and out must not be NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->st;
    return DEFMM_OK;
}

extern "C" defmm_status defmm_server_destroy(defmm_server s) {
    if (!s) return DEFMM_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_one();
    if (s->worker.joinable()) s->worker.join();
    for (cudaStream_t x : s->streams) {
        cudaStreamSynchronize(x);
        cudaStreamDestroy(x);
    }
    cudaFree(s->arena_mem);
    delete s;
    return DEFMM_OK;
}
