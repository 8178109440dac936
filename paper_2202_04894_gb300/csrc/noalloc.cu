// defmm_apply_noalloc: the application phase without any device allocation.
//
// Some callers cannot call cudaMalloc at the time they apply the operator:
// code running while a stream is being captured into a CUDA graph, runtimes
// whose device memory is owned by a pool or allocator that another component
// controls, or solvers that have reserved all device memory up front.  For
// them this entry point takes the application phase's scratch (Morton-ordered
// charges and potentials, multipole, Fourier-domain and local expansions,
// near-field partial sums)
// from a fixed array linked into the library instead of from cudaMalloc.
//
// Limits and rules:
//  - The array is a file-scope static __device__ array of kScratchBytes
//    (64 MiB).  Every GPU that loads the library reserves it until the
//    process exits.  Problems whose scratch does not fit are rejected with
//    DEFMM_ERR_UNSUPPORTED and a message giving both sizes.
//  - The first call on a device looks up the array's device address with
//    cudaGetSymbolAddress (with that device current) and caches it; make that
//    first call before any stream capture begins.
//  - All calls, from every plan and thread, share the one array, which keeps
//    the last call's contents.  Everything the apply needs zeroed is cleared
//    inside the call.  Calls whose GPU work overlaps (different streams, or
//    threads without ordering) race on the array and give wrong results; the
//    caller must order them.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "defmm.h"
#include "kernels.cuh"
#include "plan_state.h"

namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the array on the current device, looked up once per device.
defmm_status scratch_address(void** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return defmm::set_error(DEFMM_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return defmm::set_error(DEFMM_ERR_UNSUPPORTED, "device index out of range");
    std::lock_guard<std::mutex> lk(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return defmm::set_error(DEFMM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return DEFMM_OK;
}

const defmm::DevTyped<float>& typed_tables(const defmm_plan_s* pl, float*) { return pl->tf; }
const defmm::DevTyped<double>& typed_tables(const defmm_plan_s* pl, double*) { return pl->td; }

template <typename T>
defmm_status apply_static(defmm_plan_s* pl, const void* q, void* p, int R, cudaStream_t stream) {
    using C = typename defmm::Cplx<T>::type;
    const defmm::HostPlan& hp = pl->hp;
    auto carve = [](size_t& off, size_t count) {
        size_t start = (off + 255) / 256 * 256;
        off = start + count * sizeof(C);
        return start;
    };
    size_t off = 0;
    const size_t o_qs = carve(off, (size_t)R * hp.ny);
    const size_t o_ps = carve(off, (size_t)R * hp.nx);
    const size_t o_M = carve(off, (size_t)R * hp.nM() * hp.P3);
    const size_t o_Mh = carve(off, (size_t)R * hp.m2f_list.size() * hp.NFpad);
    const size_t o_L = carve(off, (size_t)R * hp.nL() * hp.P3);
    const size_t o_part = carve(off, (size_t)R * hp.p2p_parts);
    if (off > kScratchBytes)
        return defmm::set_error(DEFMM_ERR_UNSUPPORTED,
                                "defmm_apply_noalloc: this plan needs " + std::to_string(off) +
                                    " bytes of scratch for nrhs=" + std::to_string(R) +
                                    ", more than the library's fixed " + std::to_string(kScratchBytes) +
                                    " bytes; use defmm_apply");
    void* base = nullptr;
    defmm_status s = scratch_address(&base);
    if (s != DEFMM_OK) return s;
    unsigned char* b = static_cast<unsigned char*>(base);
    defmm::DevWork<T> w;
    w.R = R;
    w.qs = reinterpret_cast<C*>(b + o_qs);
    w.ps = reinterpret_cast<C*>(b + o_ps);
    w.M = reinterpret_cast<C*>(b + o_M);
    w.Mhat = reinterpret_cast<C*>(b + o_Mh);
    w.L = reinterpret_cast<C*>(b + o_L);
    w.part = reinterpret_cast<C*>(b + o_part);
    w.nL = hp.nL();
    const defmm::DevTyped<T>& typed = typed_tables(pl, (T*)nullptr);
    int launches = 0;
    const defmm::LevelList* l2l = nullptr;
    const defmm::DevCommon c = defmm::apply_tables(pl, &l2l);
    cudaError_t e = defmm::launch_apply<T>(c, typed, w, pl->m2m.data(), (int)pl->m2m.size(), l2l,
                                           pl->l2l_par.data(), (int)pl->l2l.size(), q, p, stream, &launches,
                                           pl->profiling ? pl->events : nullptr);
    pl->launches = launches;
    if (pl->profiling && e == cudaSuccess) pl->profiled = true;
    if (e != cudaSuccess)
        return defmm::set_error(DEFMM_ERR_CUDA, std::string("apply launch: ") + cudaGetErrorString(e));
    return DEFMM_OK;
}

}  // namespace

extern "C" defmm_status defmm_apply_noalloc(defmm_plan plan, const void* q, void* p, int nrhs, defmm_dtype dtype,
                                            void* stream) {
    if (!plan) return defmm::set_error(DEFMM_ERR_ARG, "plan is NULL");
    if (!q || !p) return defmm::set_error(DEFMM_ERR_ARG, "q and p must be device pointers");
    if (nrhs < 1) return defmm::set_error(DEFMM_ERR_ARG, "nrhs must be >= 1");
    if (dtype != DEFMM_C64 && dtype != DEFMM_C128) return defmm::set_error(DEFMM_ERR_UNSUPPORTED, "dtype");
    if (plan->host_only)
        return defmm::set_error(DEFMM_ERR_UNSUPPORTED, "plan was built with DEFMM_PLAN_HOST_ONLY");
    std::unique_lock<std::mutex> lk(plan->busy, std::try_to_lock);
    if (!lk.owns_lock()) return defmm::set_error(DEFMM_ERR_BUSY, "plan is in use by another thread");
    if (dtype == DEFMM_C64) return apply_static<float>(plan, q, p, nrhs, (cudaStream_t)stream);
    return apply_static<double>(plan, q, p, nrhs, (cudaStream_t)stream);
}
