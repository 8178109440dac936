// defmm_plan_autotune: picks the launch shape of a geometry by measurement.
//
// The paper fixes Ncrit, the interpolation order and the FFT length by hand
// per experiment (Sec. 6); here the choices that change only the speed of an
// apply, never what it approximates beyond the order's accuracy, are timed on
// the caller's own geometry:
//  - leaf size Ncrit (plan time; candidates 16, 24, 32, 48, 64 within the
//    caller's range),
//  - DFT length N (plan time; 2p-1 and 2p, any N >= 2p-1 gives the same
//    result, Sec. 2.3),
//  - right-hand sides per M2L pass (apply time; 1, 2, 4 when nrhs > 1),
//  - the tensor-core near field on or off (apply time; nrhs >= 8, complex64),
//  - sibling targets per M2L block, 8 or 4 (apply time; complex64).
// Every candidate plan is built with the public entry points, applied to a
// fixed pseudo-random charge block of nrhs columns, and timed with CUDA events
// on the caller's stream (median of `reps` applies after two warm-up applies).
// At most two candidate plans are alive at once (the best so far and the one
// being timed).  The fastest becomes the returned plan.
//
// Tune cache: a text file with one line per tuned geometry,
//   defmm-tune <key> <leaf> <fft_n> <m2l_rhs_block> <tensor-core near field 0/1> <members> <ms>
// where key is a 64-bit FNV-1a hash of the coordinates, sizes, kappa, order,
// nrhs, dtype, the candidate range and the plan options.  A hit builds the
// plan directly with the stored choice; a miss tunes and appends a line.
#include <cuda_runtime.h>

#include <algorithm>
#include <cinttypes>
#include <cstdio>
#include <cstring>
#include <functional>
#include <mutex>
#include <string>
#include <vector>

#include "defmm.h"
#include "plan_state.h"

namespace {

struct Fnv {
    uint64_t h = 1469598103934665603ull;
    void add(const void* p, size_t n) {
        const unsigned char* b = static_cast<const unsigned char*>(p);
        for (size_t i = 0; i < n; ++i) {
            h ^= b[i];
            h *= 1099511628211ull;
        }
    }
    template <typename V> void val(const V& v) { add(&v, sizeof(v)); }
};

std::mutex g_cache_mutex;

struct Choice {
    int leaf = 0, fft_n = 0, rb = 0, tc = 0, mem = 0;
    double ms = 0;
};

bool cache_lookup(const char* path, uint64_t key, Choice* c) {
    if (!path || !*path) return false;
    std::lock_guard<std::mutex> lk(g_cache_mutex);
    FILE* f = std::fopen(path, "r");
    if (!f) return false;
    char line[256];
    bool found = false;
    while (std::fgets(line, sizeof line, f)) {
        uint64_t k;
        Choice v;
        if (std::sscanf(line, "defmm-tune %" SCNx64 " %d %d %d %d %d %lf", &k, &v.leaf, &v.fft_n, &v.rb, &v.tc, &v.mem,
                        &v.ms) == 7 &&
            k == key && v.leaf >= 1 && v.fft_n >= 0 && (v.rb == 0 || v.rb == 1 || v.rb == 2 || v.rb == 4) &&
            (v.tc == 0 || v.tc == 1) && (v.mem == 0 || v.mem == 4 || v.mem == 8 || v.mem == 12 || v.mem == 14)) {
            *c = v;   // the last matching line wins
            found = true;
        }
    }
    std::fclose(f);
    return found;
}

bool cache_store(const char* path, uint64_t key, const Choice& c) {
    if (!path || !*path) return true;
    std::lock_guard<std::mutex> lk(g_cache_mutex);
    FILE* f = std::fopen(path, "a");
    if (!f) return false;
    std::fprintf(f, "defmm-tune %016" PRIx64 " %d %d %d %d %d %.6f\n", key, c.leaf, c.fft_n, c.rb, c.tc, c.mem, c.ms);
    return std::fclose(f) == 0;
}

// Deterministic charges for timing (values do not change the work done).
void fill_charges(std::vector<unsigned char>& h, size_t count, bool dbl) {
    uint64_t s = 0x9e3779b97f4a7c15ull;
    auto next = [&s]() {
        s += 0x9e3779b97f4a7c15ull;
        uint64_t z = s;
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        return ((z ^ (z >> 31)) >> 11) * (1.0 / 9007199254740992.0) - 0.5;
    };
    h.resize(count * (dbl ? 16 : 8));
    for (size_t i = 0; i < 2 * count; ++i) {
        const double v = next();
        if (dbl) std::memcpy(&h[i * 8], &v, 8);
        else {
            const float f = (float)v;
            std::memcpy(&h[i * 4], &f, 4);
        }
    }
}

struct DeviceBuffers {
    void* q = nullptr;
    void* p = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~DeviceBuffers() {
        if (q) cudaFree(q);
        if (p) cudaFree(p);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
};

// Median time (ms, into *ms) of `reps` applies after two warm-up applies.
defmm_status time_applies(defmm_plan plan, DeviceBuffers& b, int nrhs, defmm_dtype dt, int reps,
                          cudaStream_t st, double* ms) {
    for (int w = 0; w < 2; ++w) {
        defmm_status s = defmm_apply(plan, b.q, b.p, nrhs, dt, st);
        if (s != DEFMM_OK) return s;
    }
    std::vector<float> t;
    for (int r = 0; r < reps; ++r) {
        cudaError_t e = cudaEventRecord(b.e0, st);
        if (e != cudaSuccess) return defmm::set_error(DEFMM_ERR_CUDA, std::string("autotune event: ") + cudaGetErrorString(e));
        defmm_status s = defmm_apply(plan, b.q, b.p, nrhs, dt, st);
        if (s != DEFMM_OK) return s;
        e = cudaEventRecord(b.e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(b.e1);
        float x = 0;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&x, b.e0, b.e1);
        if (e != cudaSuccess) return defmm::set_error(DEFMM_ERR_CUDA, std::string("autotune timing: ") + cudaGetErrorString(e));
        t.push_back(x);
    }
    std::sort(t.begin(), t.end());
    *ms = t[t.size() / 2];
    defmm_info info;
    defmm_status s = defmm_plan_info(plan, &info);
    if (s != DEFMM_OK) return s;
    if (info.device_error) return defmm::set_error(DEFMM_ERR_TIMEOUT, "autotune: a device-side wait gave up");
    return DEFMM_OK;
}

// Candidates, timing and the cache, for any plan factory (one geometry or a
// union): make(leaf, options, &plan) builds a candidate; nx / nys are the
// total target / source counts of an apply.
using Factory = std::function<defmm_status(int leaf, const defmm_options& o, defmm_plan* out)>;

defmm_status tune_with(const Factory& make, uint64_t key, int64_t nx, int64_t nys, int order,
                       const defmm_tune_options& t, const defmm_options& o, void* stream, defmm_plan* out,
                       defmm_tune_result* result) {
    cudaStream_t st = (cudaStream_t)stream;
    // candidates
    std::vector<int> leaves;
    for (int c : {16, 24, 32, 48, 64})
        if (c >= t.leaf_min && c <= t.leaf_max) leaves.push_back(c);
    if (leaves.empty() || leaves.back() != t.leaf_max) leaves.push_back(t.leaf_max);
    std::vector<int> ffts = {o.fft_n};
    if (t.tune_fft_n && o.fft_n == 0) ffts.push_back(2 * order);
    std::vector<int> rbs = {0};
    if (t.nrhs > 1 && t.dtype == DEFMM_C64) rbs = {1, 2, 4};
    std::vector<int> tcs = {0};
    if (t.nrhs >= 8 && t.dtype == DEFMM_C64) tcs = {0, 1};
    struct Launch { int tc, mem, rb; };   // apply-time choices timed on every candidate plan
    // members per M2L block: complex64 only; the splits by group size (12, 14)
    // exist for N = 7 with one column per pass
    auto launches_for = [&](int fft) {
        const int N = fft ? fft : 2 * order - 1;
        std::vector<Launch> v;
        for (int tc : tcs)
            for (int rb : rbs) {
                std::vector<int> mems = {0};
                if (t.dtype == DEFMM_C64) {
                    const bool one = rb == 1 || (rb == 0 && t.nrhs == 1);
                    if (order == 4 && N == 7 && one) mems = {14, 12, 8, 4};
                    else mems = {8, 4};
                }
                for (int mem : mems) v.push_back({tc, mem, rb});
            }
        return v;
    };

    defmm_tune_result res{};
    Choice hit;
    if (cache_lookup(t.cache_path, key, &hit)) {
        defmm_options oc = o;
        oc.fft_n = hit.fft_n;
        defmm_plan pl = nullptr;
        defmm_status s = make(hit.leaf, oc, &pl);
        if (s != DEFMM_OK) return s;
        defmm_tuning tn{hit.rb, hit.tc ? 1 : 0, hit.mem, 0};
        s = defmm_plan_set_tuning(pl, &tn);
        if (s != DEFMM_OK) { defmm_destroy(pl); return s; }
        res.leaf_size = hit.leaf; res.fft_n = hit.fft_n; res.m2l_rhs_block = hit.rb; res.p2p_tensor_cores = hit.tc;
        res.m2l_members_per_block = hit.mem;
        res.ms = hit.ms;
        res.candidates = 0; res.from_cache = 1;
        if (result) *result = res;
        *out = pl;
        return DEFMM_OK;
    }

    DeviceBuffers b;
    const bool dbl = t.dtype == DEFMM_C128;
    const size_t esz = dbl ? 16 : 8;
    cudaError_t e = cudaMalloc(&b.q, (size_t)nys * t.nrhs * esz);
    if (e == cudaSuccess) e = cudaMalloc(&b.p, (size_t)nx * t.nrhs * esz);
    if (e == cudaSuccess) e = cudaEventCreate(&b.e0);
    if (e == cudaSuccess) e = cudaEventCreate(&b.e1);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return defmm::set_error(e == cudaErrorMemoryAllocation ? DEFMM_ERR_OOM : DEFMM_ERR_CUDA,
                                std::string("autotune buffers: ") + cudaGetErrorString(e));
    }
    {
        std::vector<unsigned char> hq;
        fill_charges(hq, (size_t)nys * t.nrhs, dbl);
        e = cudaMemcpy(b.q, hq.data(), hq.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return defmm::set_error(DEFMM_ERR_CUDA, std::string("autotune charges: ") + cudaGetErrorString(e));
    }

    defmm_plan best = nullptr;
    Choice bc;
    bc.ms = 1e300;
    int timed = 0;
    for (int fft : ffts) {
        const std::vector<Launch> launches = launches_for(fft);
        for (int leaf : leaves) {
            defmm_options oc = o;
            oc.fft_n = fft;
            defmm_plan pl = nullptr;
            defmm_status s = make(leaf, oc, &pl);
            if (s == DEFMM_ERR_OOM) continue;            // over the budget: not a candidate
            if (s != DEFMM_OK) { if (best) defmm_destroy(best); return s; }
            bool kept = false;
            for (const Launch& lc : launches) {
                defmm_tuning tn{lc.rb, lc.tc ? 1 : 0, lc.mem, 0};
                s = defmm_plan_set_tuning(pl, &tn);
                double ms = 0;
                if (s == DEFMM_OK) s = time_applies(pl, b, t.nrhs, t.dtype, t.reps, st, &ms);
                if (s == DEFMM_ERR_OOM) break;   // this plan's workspace is over the budget
                if (s != DEFMM_OK) {
                    defmm_destroy(pl);
                    if (best) defmm_destroy(best);
                    return s;
                }
                ++timed;
                if (ms < bc.ms) {
                    bc.leaf = leaf; bc.fft_n = fft; bc.rb = lc.rb; bc.tc = lc.tc; bc.mem = lc.mem; bc.ms = ms;
                    if (!kept) {
                        if (best) defmm_destroy(best);
                        best = pl;
                        kept = true;
                    }
                }
            }
            if (!kept) defmm_destroy(pl);
        }
    }
    if (!best) return defmm::set_error(DEFMM_ERR_OOM, "autotune: no candidate fits the device or hbm_budget");
    defmm_tuning tn{bc.rb, bc.tc ? 1 : 0, bc.mem, 0};
    defmm_status s = defmm_plan_set_tuning(best, &tn);
    if (s != DEFMM_OK) { defmm_destroy(best); return s; }
    if (!cache_store(t.cache_path, key, bc)) {
        defmm_destroy(best);
        return defmm::set_error(DEFMM_ERR_ARG, std::string("autotune: cannot append to ") + t.cache_path);
    }
    res.leaf_size = bc.leaf; res.fft_n = bc.fft_n; res.m2l_rhs_block = bc.rb; res.p2p_tensor_cores = bc.tc;
    res.m2l_members_per_block = bc.mem;
    res.ms = bc.ms;
    res.candidates = timed; res.from_cache = 0;
    if (result) *result = res;
    *out = best;
    return DEFMM_OK;
}

defmm_status check_tune_args(const defmm_tune_options& t, const defmm_options& o, int order) {
    if (t.leaf_min < 1 || t.leaf_max < t.leaf_min) return defmm::set_error(DEFMM_ERR_ARG, "leaf range must satisfy 1 <= leaf_min <= leaf_max");
    if (t.nrhs < 1) return defmm::set_error(DEFMM_ERR_ARG, "nrhs must be >= 1");
    if (t.reps < 1) return defmm::set_error(DEFMM_ERR_ARG, "reps must be >= 1");
    if (t.dtype != DEFMM_C64 && t.dtype != DEFMM_C128) return defmm::set_error(DEFMM_ERR_UNSUPPORTED, "dtype");
    if (o.flags & DEFMM_PLAN_HOST_ONLY) return defmm::set_error(DEFMM_ERR_UNSUPPORTED, "autotuning needs a device plan");
    if (order < 2 || order > 8) return defmm::set_error(DEFMM_ERR_ARG, "order must be in [2, 8]");
    return DEFMM_OK;
}

// Host copy of n x 3 coordinates given in host or device memory.
defmm_status host_points(const double* P, int64_t n, std::vector<double>& h) {
    h.resize((size_t)n * 3);
    cudaPointerAttributes a{};
    const bool dev = cudaPointerGetAttributes(&a, P) == cudaSuccess && a.type == cudaMemoryTypeDevice;
    cudaGetLastError();
    if (dev) {
        cudaError_t e = cudaMemcpy(h.data(), P, h.size() * 8, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return defmm::set_error(DEFMM_ERR_CUDA, std::string("autotune: read points: ") + cudaGetErrorString(e));
    } else {
        std::memcpy(h.data(), P, h.size() * 8);
    }
    return DEFMM_OK;
}

void key_options(Fnv& key, const defmm_tune_options& t, const defmm_options& o, int order) {
    key.val(order);
    key.val(t.nrhs); key.val((int)t.dtype); key.val(t.leaf_min); key.val(t.leaf_max); key.val(t.tune_fft_n);
    key.val(o.eta); key.val(o.hf_kw); key.val(o.fft_n); key.val(o.self_eps); key.val(o.damping); key.val(o.radial_power);
    key.val(o.m2l_chunk_blocks);
}

}  // namespace

extern "C" {

void defmm_default_tune_options(defmm_tune_options* t) {
    if (!t) return;
    t->leaf_min = 16;
    t->leaf_max = 64;
    t->nrhs = 1;
    t->dtype = DEFMM_C64;
    t->reps = 5;
    t->tune_fft_n = 1;
    t->cache_path = nullptr;
}

defmm_status defmm_plan_autotune(const double* X, int64_t nx, const double* Y, int64_t ny, double kappa, int order,
                                 const defmm_options* opt, const defmm_tune_options* topt, void* stream,
                                 defmm_plan* out, defmm_tune_result* result) {
    if (!out) return defmm::set_error(DEFMM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!X || nx < 1) return defmm::set_error(DEFMM_ERR_ARG, "X is NULL or nx < 1");
    defmm_tune_options t;
    defmm_default_tune_options(&t);
    if (topt) t = *topt;
    defmm_options o;
    defmm_default_options(&o);
    if (opt) o = *opt;
    defmm_status s = check_tune_args(t, o, order);
    if (s != DEFMM_OK) return s;
    const bool same = (Y == nullptr) || (Y == X && ny == nx);
    const int64_t nys = same ? nx : ny;
    // cache key: coordinates (host or device), sizes, parameters
    Fnv key;
    std::vector<double> h;
    s = host_points(X, nx, h);
    if (s != DEFMM_OK) return s;
    key.add(h.data(), h.size() * 8);
    if (!same) {
        s = host_points(Y, ny, h);
        if (s != DEFMM_OK) return s;
        key.add(h.data(), h.size() * 8);
    }
    key.val(nx); key.val(nys); key.val(same); key.val(kappa);
    key_options(key, t, o, order);
    auto make = [&](int leaf, const defmm_options& oc, defmm_plan* pl) {
        return defmm_plan_create(X, nx, Y, ny, kappa, order, leaf, &oc, stream, pl);
    };
    return tune_with(make, key.h, nx, nys, order, t, o, stream, out, result);
}

defmm_status defmm_plan_autotune_union(int ngeo, const double* const* X, const int64_t* nx, const double* kappa,
                                       int order, const defmm_options* opt, const defmm_tune_options* topt,
                                       void* stream, defmm_plan* out, defmm_tune_result* result) {
    if (!out) return defmm::set_error(DEFMM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (ngeo < 1 || !X || !nx || !kappa) return defmm::set_error(DEFMM_ERR_ARG, "need ngeo >= 1 and X, nx, kappa arrays");
    defmm_tune_options t;
    defmm_default_tune_options(&t);
    if (topt) t = *topt;
    defmm_options o;
    defmm_default_options(&o);
    if (opt) o = *opt;
    defmm_status s = check_tune_args(t, o, order);
    if (s != DEFMM_OK) return s;
    Fnv key;
    int64_t total = 0;
    std::vector<double> h;
    for (int g = 0; g < ngeo; ++g) {
        if (!X[g] || nx[g] < 1) return defmm::set_error(DEFMM_ERR_ARG, "every geometry needs points (X[g] != NULL, nx[g] >= 1)");
        s = host_points(X[g], nx[g], h);
        if (s != DEFMM_OK) return s;
        key.add(h.data(), h.size() * 8);
        key.val(nx[g]); key.val(kappa[g]);
        total += nx[g];
    }
    key.val(ngeo);
    key_options(key, t, o, order);
    auto make = [&](int leaf, const defmm_options& oc, defmm_plan* pl) {
        return defmm_plan_create_union(ngeo, X, nx, kappa, order, leaf, &oc, stream, pl);
    };
    return tune_with(make, key.h, total, total, order, t, o, stream, out, result);
}

}  // extern "C"
