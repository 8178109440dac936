// defmm_gmres: restarted GMRES on the device for (sigma I + A) x = b, where A
// is the plan's FMM operator (p = A q, Eq. 1.1 approximated by the directional
// FMM).  The paper applies the operator inside iterative boundary-integral
// solvers (Sec. 1, Sec. 7); this is that loop, with every matrix-vector product
// a defmm_apply on the caller's stream.
//
// Algorithm: GMRES(m) of Saad and Schultz (SIAM J. Sci. Stat. Comput. 7, 1986):
// Arnoldi with classical Gram-Schmidt applied twice (CGS2) for orthogonality,
// Givens rotations on the (m+1) x m Hessenberg matrix (host, float64 complex),
// restart after m products, the true residual b - (sigma x + A x) recomputed
// at every restart.  Vectors stay on the device in the apply's precision;
// inner products accumulate in float64 and are reduced in a fixed order
// (deterministic).  The host reads the projections and norms once per
// Arnoldi step (one stream synchronisation each).
#include <cuda_runtime.h>

#include <cmath>
#include <complex>
#include <string>
#include <vector>

#include "defmm.h"
#include "kernels.cuh"
#include "plan_state.h"

namespace {

using cd = std::complex<double>;
constexpr int kDotBlocks = 304;   // two per SM
constexpr int kDotThreads = 256;

__device__ __forceinline__ double2 to_d2(float2 v) { return make_double2((double)v.x, (double)v.y); }
__device__ __forceinline__ double2 to_d2(double2 v) { return v; }
template <typename C> __device__ __forceinline__ C from_d2(double2 v);
template <> __device__ __forceinline__ float2 from_d2<float2>(double2 v) { return make_float2((float)v.x, (float)v.y); }
template <> __device__ __forceinline__ double2 from_d2<double2>(double2 v) { return v; }

// part[i * gridDim.x + block] = sum over the block's slice of conj(V_i[j]) w[j]
template <typename C>
__global__ void __launch_bounds__(kDotThreads) k_dots(const C* __restrict__ V, int64_t ld, int k,
                                                      const C* __restrict__ w, int64_t n, double2* __restrict__ part) {
    __shared__ double2 red[kDotThreads];
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t j0 = (int64_t)blockIdx.x * chunk, j1 = j0 + chunk < n ? j0 + chunk : n;
    for (int i = 0; i < k; ++i) {
        double2 s = make_double2(0.0, 0.0);
        for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
            const double2 a = to_d2(V[(int64_t)i * ld + j]), b = to_d2(w[j]);
            s.x += a.x * b.x + a.y * b.y;
            s.y += a.x * b.y - a.y * b.x;
        }
        red[threadIdx.x] = s;
        __syncthreads();
        for (int h = blockDim.x / 2; h > 0; h >>= 1) {
            if (threadIdx.x < h) {
                red[threadIdx.x].x += red[threadIdx.x + h].x;
                red[threadIdx.x].y += red[threadIdx.x + h].y;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) part[(int64_t)i * gridDim.x + blockIdx.x] = red[0];
        __syncthreads();
    }
}

// out[i] = sum over blocks of part[i * nb + block], in a fixed tree order
__global__ void __launch_bounds__(kDotThreads) k_dots_reduce(const double2* __restrict__ part, int nb,
                                                             double2* __restrict__ out) {
    __shared__ double2 red[kDotThreads];
    double2 s = make_double2(0.0, 0.0);
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        s.x += part[(int64_t)blockIdx.x * nb + b].x;
        s.y += part[(int64_t)blockIdx.x * nb + b].y;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            red[threadIdx.x].x += red[threadIdx.x + h].x;
            red[threadIdx.x].y += red[threadIdx.x + h].y;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

// w[j] += sign * sum_i c[i] V_i[j]
template <typename C>
__global__ void k_combine(const C* __restrict__ V, int64_t ld, int k, const double2* __restrict__ c, double sign,
                          C* __restrict__ w, int64_t n) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        double2 s = to_d2(w[j]);
        for (int i = 0; i < k; ++i) {
            const double2 a = to_d2(V[(int64_t)i * ld + j]), h = c[i];
            s.x += sign * (h.x * a.x - h.y * a.y);
            s.y += sign * (h.x * a.y + h.y * a.x);
        }
        w[j] = from_d2<C>(s);
    }
}

// y = sigma * x + y (y holds A x), or with neg: y = b - (sigma * x + y)
template <typename C>
__global__ void k_shift(const C* __restrict__ x, C* __restrict__ y, const C* __restrict__ b, double2 sigma, int64_t n) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const double2 a = to_d2(x[j]), v = to_d2(y[j]);
        double2 s = make_double2(v.x + sigma.x * a.x - sigma.y * a.y, v.y + sigma.x * a.y + sigma.y * a.x);
        if (b) {
            const double2 bb = to_d2(b[j]);
            s = make_double2(bb.x - s.x, bb.y - s.y);
        }
        y[j] = from_d2<C>(s);
    }
}

template <typename C>
__global__ void k_scale(const C* __restrict__ w, C* __restrict__ v, double s, int64_t n) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const double2 a = to_d2(w[j]);
        v[j] = from_d2<C>(make_double2(a.x * s, a.y * s));
    }
}

struct Scratch {
    void* V = nullptr;
    void* w = nullptr;
    double2* part = nullptr;
    double2* dev = nullptr;
    ~Scratch() {
        if (V) cudaFree(V);
        if (w) cudaFree(w);
        if (part) cudaFree(part);
        if (dev) cudaFree(dev);
    }
};

defmm_status cuda_status(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return DEFMM_OK;
    return defmm::set_error(e == cudaErrorMemoryAllocation ? DEFMM_ERR_OOM : DEFMM_ERR_CUDA,
                            std::string("gmres: ") + what + ": " + cudaGetErrorString(e));
}

template <typename C>
defmm_status gmres_impl(defmm_plan plan, int64_t n, const C* b, C* x, defmm_dtype dt, const defmm_gmres_options& o,
                        cudaStream_t st, defmm_gmres_result* res) {
    const int m = o.restart;
    const double2 sigma = make_double2(o.shift_re, o.shift_im);
    Scratch s;
    cudaError_t e = cudaMalloc(&s.V, sizeof(C) * (size_t)n * (m + 1));
    if (e == cudaSuccess) e = cudaMalloc(&s.w, sizeof(C) * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&s.part, sizeof(double2) * (size_t)kDotBlocks * (m + 1));
    if (e == cudaSuccess) e = cudaMalloc(&s.dev, sizeof(double2) * (size_t)(m + 1));
    if (e != cudaSuccess) { cudaGetLastError(); return cuda_status(e, "scratch"); }
    C* V = static_cast<C*>(s.V);
    C* w = static_cast<C*>(s.w);
    const int eb = defmm::sm_count() * 4;
    std::vector<double2> hbuf(m + 1);

    // conj(V_i) . v for i < k, read back to the host
    auto dots = [&](const C* Vb, int k, const C* v, std::vector<cd>& out) -> defmm_status {
        k_dots<C><<<kDotBlocks, kDotThreads, 0, st>>>(Vb, n, k, v, n, s.part);
        k_dots_reduce<<<k, kDotThreads, 0, st>>>(s.part, kDotBlocks, s.dev);
        cudaError_t er = cudaMemcpyAsync(hbuf.data(), s.dev, sizeof(double2) * k, cudaMemcpyDeviceToHost, st);
        if (er == cudaSuccess) er = cudaStreamSynchronize(st);
        if (er != cudaSuccess) return cuda_status(er, "inner products");
        out.resize(k);
        for (int i = 0; i < k; ++i) out[i] = cd(hbuf[i].x, hbuf[i].y);
        return DEFMM_OK;
    };
    auto combine = [&](int k, const std::vector<cd>& c, double sign, C* dst) -> defmm_status {
        for (int i = 0; i < k; ++i) hbuf[i] = make_double2(c[i].real(), c[i].imag());
        cudaError_t er = cudaMemcpyAsync(s.dev, hbuf.data(), sizeof(double2) * k, cudaMemcpyHostToDevice, st);
        if (er != cudaSuccess) return cuda_status(er, "coefficients");
        k_combine<C><<<eb, 256, 0, st>>>(V, n, k, s.dev, sign, dst, n);
        // hbuf is reused by the next call: the copy above must have read it
        er = cudaStreamSynchronize(st);
        return cuda_status(er == cudaSuccess ? cudaGetLastError() : er, "combine");
    };
    // dst = b - (sigma src + A src), or (b == nullptr) dst = sigma src + A src
    auto op = [&](const C* src, C* dst, const C* rhs) -> defmm_status {
        defmm_status ss = defmm_apply(plan, src, dst, 1, dt, st);
        if (ss != DEFMM_OK) return ss;
        k_shift<C><<<eb, 256, 0, st>>>(src, dst, rhs, sigma, n);
        return cuda_status(cudaGetLastError(), "shift");
    };

    std::vector<cd> t;
    defmm_status ss = dots(b, 1, b, t);
    if (ss != DEFMM_OK) return ss;
    const double bnorm = std::sqrt(std::max(0.0, t[0].real()));
    defmm_gmres_result r{};
    if (bnorm == 0.0) {   // x = 0 solves it exactly
        e = cudaMemsetAsync(x, 0, sizeof(C) * (size_t)n, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_status(e, "zero solution");
        r.converged = 1;
        if (res) *res = r;
        return DEFMM_OK;
    }
    int total = 0;
    double rel = 0.0;
    std::vector<cd> H((size_t)(m + 1) * m), g(m + 1), cs(m), sn(m), h, h2;
    for (;;) {
        // true residual r0 = b - (sigma x + A x) into V_0
        ss = op(x, V, b);
        if (ss != DEFMM_OK) return ss;
        ss = dots(V, 1, V, t);
        if (ss != DEFMM_OK) return ss;
        const double beta = std::sqrt(std::max(0.0, t[0].real()));
        rel = beta / bnorm;
        if (rel <= o.tol || total >= o.max_iter || beta == 0.0) break;
        k_scale<C><<<eb, 256, 0, st>>>(V, V, 1.0 / beta, n);
        std::fill(H.begin(), H.end(), cd(0));
        std::fill(g.begin(), g.end(), cd(0));
        g[0] = beta;
        int kdim = 0;
        for (int j = 0; j < m && total < o.max_iter; ++j) {
            C* vj = V + (size_t)j * n;
            ss = op(vj, w, nullptr);
            if (ss != DEFMM_OK) return ss;
            ++total;
            // classical Gram-Schmidt, twice
            ss = dots(V, j + 1, w, h);
            if (ss == DEFMM_OK) ss = combine(j + 1, h, -1.0, w);
            if (ss == DEFMM_OK) ss = dots(V, j + 1, w, h2);
            if (ss == DEFMM_OK) ss = combine(j + 1, h2, -1.0, w);
            if (ss == DEFMM_OK) ss = dots(w, 1, w, t);
            if (ss != DEFMM_OK) return ss;
            const double hn = std::sqrt(std::max(0.0, t[0].real()));
            for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = h[i] + h2[i];
            H[(size_t)(j + 1) * m + j] = hn;
            // previous rotations, then a new one that zeroes H[j+1][j]
            for (int i = 0; i < j; ++i) {
                const cd a = H[(size_t)i * m + j], c2 = H[(size_t)(i + 1) * m + j];
                H[(size_t)i * m + j] = std::conj(cs[i]) * a + std::conj(sn[i]) * c2;
                H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * c2;
            }
            const cd a = H[(size_t)j * m + j];
            const double den = std::sqrt(std::norm(a) + hn * hn);
            cs[j] = den == 0.0 ? cd(1) : a / den;
            sn[j] = den == 0.0 ? cd(0) : cd(hn / den);
            H[(size_t)j * m + j] = den;
            H[(size_t)(j + 1) * m + j] = 0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = std::conj(cs[j]) * g[j];
            kdim = j + 1;
            if (std::abs(g[j + 1]) / bnorm <= o.tol || hn == 0.0) break;
            k_scale<C><<<eb, 256, 0, st>>>(w, V + (size_t)(j + 1) * n, 1.0 / hn, n);
        }
        if (kdim == 0) break;
        // y = H^{-1} g (upper triangular), x += V y
        std::vector<cd> y(kdim);
        for (int i = kdim - 1; i >= 0; --i) {
            cd acc = g[i];
            for (int l = i + 1; l < kdim; ++l) acc -= H[(size_t)i * m + l] * y[l];
            y[i] = acc / H[(size_t)i * m + i];
        }
        ss = combine(kdim, y, 1.0, x);
        if (ss != DEFMM_OK) return ss;
    }
    r.iterations = total;
    r.rel_residual = rel;
    r.converged = rel <= o.tol ? 1 : 0;
    defmm_info info;
    ss = defmm_plan_info(plan, &info);
    if (ss != DEFMM_OK) return ss;
    if (info.device_error) return defmm::set_error(DEFMM_ERR_TIMEOUT, "gmres: a device-side wait of an apply gave up");
    if (res) *res = r;
    return DEFMM_OK;
}

}  // namespace

extern "C" {

void defmm_default_gmres_options(defmm_gmres_options* o) {
    if (!o) return;
    o->shift_re = 1.0;
    o->shift_im = 0.0;
    o->tol = 1e-6;
    o->restart = 30;
    o->max_iter = 200;
}

defmm_status defmm_gmres(defmm_plan plan, const void* b, void* x, defmm_dtype dtype, const defmm_gmres_options* opt,
                         void* stream, defmm_gmres_result* result) {
    if (!plan) return defmm::set_error(DEFMM_ERR_ARG, "plan is NULL");
    if (!b || !x) return defmm::set_error(DEFMM_ERR_ARG, "b and x must be device pointers");
    if (dtype != DEFMM_C64 && dtype != DEFMM_C128) return defmm::set_error(DEFMM_ERR_UNSUPPORTED, "dtype");
    defmm_gmres_options o;
    defmm_default_gmres_options(&o);
    if (opt) o = *opt;
    if (o.restart < 1 || o.restart > 1000) return defmm::set_error(DEFMM_ERR_ARG, "restart must be in [1, 1000]");
    if (o.max_iter < 0) return defmm::set_error(DEFMM_ERR_ARG, "max_iter must be >= 0");
    if (!(o.tol >= 0.0)) return defmm::set_error(DEFMM_ERR_ARG, "tol must be >= 0");
    if (plan->host_only) return defmm::set_error(DEFMM_ERR_UNSUPPORTED, "plan was built with DEFMM_PLAN_HOST_ONLY");
    if (plan->hp.nx != plan->hp.ny) return defmm::set_error(DEFMM_ERR_ARG, "gmres needs as many targets as sources");
    if (plan->sh.nshards > 1) return defmm::set_error(DEFMM_ERR_UNSUPPORTED, "gmres needs the whole operator (plan is sharded)");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = plan->hp.nx;
    if (dtype == DEFMM_C64)
        return gmres_impl<float2>(plan, n, static_cast<const float2*>(b), static_cast<float2*>(x), dtype, o, st, result);
    return gmres_impl<double2>(plan, n, static_cast<const double2*>(b), static_cast<double2*>(x), dtype, o, st, result);
}

}  // extern "C"
