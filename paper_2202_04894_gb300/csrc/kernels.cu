// Application-phase kernels of the directional equispaced FMM on sm_103a.
//
//   gather   q -> Morton order
//   P2P      near field over the pairs of Alg. 1 (Sec. 2.2, Sec. 5.3); CUDA
//            cores (1, 4, 8 or 16 columns per pass) or, opt-in for many
//            columns, tcgen05 tensor cores (k_p2p_tc)
//   P2M      S_a^u[c](y) = exp(i kappa <y_a - y, u>) S_a[c](y)   (Sec. 2.2)
//   M2M      D0(v) (x)M^(p) D1(v), tensorised (Sec. 5.2.1, Eq. dlefturight)
//   M2F      F chi: zero-pad + forward DFT (Sec. 4.1.1)
//   M2L      Hadamard products with symmetry-permuted spectra, summed over
//            each target's list (Sec. 2.3, Eq. permuteM2L), fused with
//   F2L      chi^T F*: inverse DFT + crop (Sec. 4.1.1)
//   L2L      transpose of M2M (Sec. 2.2)
//   L2P      S_a^u[c](x) at the targets (Sec. 2.2)
//   scatter  p <- Morton order
//
// Every output is produced by exactly one thread block with a fixed
// summation order (no atomics), so results are deterministic.  The kernels
// take the plan's tables by value (DevCommon); a shard of the targets or a
// union of several geometries only changes which entries they visit and where
// a cell's wavenumber comes from.
#include <atomic>
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "kernels.cuh"
#include "plan.h"
#include "symmetry.h"
#include "tcgen05.cuh"

#include <nvtx3/nvToolsExt.h>

namespace defmm {

__constant__ int kPermDev[6][3] = DEFMM_PERM_TABLE;

// ------------------------------------------------------------------ complex
__device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {  // a * conj(b)
    return mk(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename C> __device__ __forceinline__ void cfma(C& acc, C a, C b) {
    acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return mk(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C cscale(C a, decltype(a.x) s) { return mk(a.x * s, a.y * s); }
template <typename C> __device__ __forceinline__ C czero() { return mk((decltype(C{}.x))0, (decltype(C{}.x))0); }

__device__ __forceinline__ void sincos_t(float a, float* s, float* c) { sincosf(a, s, c); }
__device__ __forceinline__ void sincos_t(double a, double* s, double* c) { sincos(a, s, c); }

// Lagrange basis l_m(t) on {0, 1/(p-1), ..., 1}, evaluated at s = (p-1) t.
template <typename T> __device__ __forceinline__ T lagrange(int p, int m, T s) {
    T v = (T)1;
    for (int n = 0; n < p; ++n)
        if (n != m) v *= (s - (T)n) / (T)(m - n);
    return v;
}

// Loads n consecutive values from shared memory with 16-byte loads where the
// type and count allow (the callers' rows start on 16-byte boundaries then).
template <int n> __device__ __forceinline__ void ld_vec(const float* src, float* dst) {
    if constexpr (n % 4 == 0) {
#pragma unroll
        for (int i = 0; i < n / 4; ++i) {
            const float4 v = reinterpret_cast<const float4*>(src)[i];
            dst[4 * i] = v.x, dst[4 * i + 1] = v.y, dst[4 * i + 2] = v.z, dst[4 * i + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < n; ++i) dst[i] = src[i];
    }
}
template <int n> __device__ __forceinline__ void ld_vec(const double* src, double* dst) {
#pragma unroll
    for (int i = 0; i < n; ++i) dst[i] = src[i];
}
template <int n> __device__ __forceinline__ void ld_vec(const float2* src, float2* dst) {
    if constexpr (n % 2 == 0) {
#pragma unroll
        for (int i = 0; i < n / 2; ++i) {
            const float4 v = reinterpret_cast<const float4*>(src)[i];
            dst[2 * i] = make_float2(v.x, v.y), dst[2 * i + 1] = make_float2(v.z, v.w);
        }
    } else {
#pragma unroll
        for (int i = 0; i < n; ++i) dst[i] = src[i];
    }
}
template <int n> __device__ __forceinline__ void ld_vec(const double2* src, double2* dst) {
#pragma unroll
    for (int i = 0; i < n; ++i) dst[i] = src[i];
}

constexpr double kInv4Pi = 0.0795774715459476678844418816863;  // 1/(4 pi)
constexpr double kInv2Pi = 0.159154943091895335768883763373;   // 1/(2 pi)
constexpr double kLog2E = 1.44269504088896340735992468100;     // log2(e)

// Wavenumber and self-distance of the geometry holding `cell` (a union plan
// holds several geometries; a plain plan has one).
__device__ __forceinline__ double kappa_of(const DevCommon& c, int cell) {
    return c.cell_geo ? c.geo_kappa[c.cell_geo[cell]] : c.kappa;
}
__device__ __forceinline__ double eps_of(const DevCommon& c, int cell) {
    return c.cell_geo ? c.geo_eps[c.cell_geo[cell]] : c.eps_self;
}

// ------------------------------------------------------------------ gather / scatter
template <typename C>
__global__ void k_gather(const C* __restrict__ q, C* __restrict__ qs, const int64_t* __restrict__ perm,
                         int64_t n, int R, int* err_flag) {
    const struct { int* err_flag; } c{err_flag};   // for the checked-build index test
    int64_t total = n * R;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = i / n, j = i - r * n;
        qs[i] = q[r * n + DEFMM_IX(c, perm[j], n)];
    }
}

template <typename C>
__global__ void k_scatter(const C* __restrict__ ps, C* __restrict__ p, const int64_t* __restrict__ perm,
                          int64_t n, int R, int64_t j0, int64_t j1, int* err_flag) {
    const struct { int* err_flag; } c{err_flag};   // for the checked-build index test
    // sorted targets j0 <= j < j1 (all of them unless the plan computes one shard)
    const int64_t m = j1 - j0, total = m * R;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = i / m, j = j0 + (i - r * m);
        p[r * n + DEFMM_IX(c, perm[j], n)] = ps[r * n + j];
    }
}

// A shard's potentials in sorted order: slice[r * ld + j] = ps[r * n + j0 + j].
template <typename C>
__global__ void k_slice(const C* __restrict__ ps, C* __restrict__ slice, int64_t n, int R, int64_t j0, int64_t j1,
                        int64_t ld) {
    const int64_t m = j1 - j0, total = m * R;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / m, j = i - r * m;
        slice[r * ld + j] = ps[r * n + j0 + j];
    }
}

// The inverse for one shard: p[r * n + perm[j0 + j]] = src[r * ld + j].
template <typename C>
__global__ void k_unslice(const C* __restrict__ src, int64_t ld, C* __restrict__ p, const int64_t* __restrict__ perm,
                          int64_t n, int R, int64_t j0, int64_t j1, int* err_flag) {
    const struct { int* err_flag; } c{err_flag};   // for the checked-build index test
    const int64_t m = j1 - j0, total = m * R;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / m, j = i - r * m;
        p[r * n + DEFMM_IX(c, perm[j0 + j], n)] = src[r * ld + j];
    }
}

// ------------------------------------------------------------------ P2P
// The hardware approximations (PTX rsqrt.approx / sin.approx / cos.approx,
// flush-to-zero): arguments here are never subnormal (r^2 > eps_self^2 is
// tested before use, phases are reduced to [-pi, pi]), so the flush changes
// nothing and saves the subnormal handling around each instruction.
__device__ __forceinline__ float rsqrt_hw(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float ex2_hw(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ void sincos_hw(float a, float* s, float* c) {
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(*s) : "f"(a));
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(*c) : "f"(a));
}

// The kernel family: G(r) = e^{(i kappa - lambda) r} / (4 pi r^P) with P = 1
// (Helmholtz; Laplace and Yukawa at kappa = 0) or P = 2 (an oscillatory kernel
// outside that family).  The method needs the kernel only to be
// asymptotically smooth (Sec. 1); it enters the transfer spectra (k_spectra)
// and the near field (the P2P kernels) and nothing else.
// Value for a difference d, zero when |d|^2 <= eps2 (Sec. 5.3), in float64.
__device__ __forceinline__ double2 helmholtz(double dx, double dy, double dz, double kappa, double eps2,
                                             double damping, int power) {
    double r2 = dx * dx + dy * dy + dz * dz;
    double r = sqrt(r2);
    double s, c;
    sincos(kappa * r, &s, &c);
    double g = kInv4Pi / r;
    if (power == 2) g /= r;
    if (damping > 0.0) g *= exp(-damping * r);
    double2 out = make_double2(c * g, s * g);
    if (!(r2 > eps2)) out = make_double2(0.0, 0.0);
    return out;
}

// e^{2 pi i t} for a phase given in turns, reduced exactly to [-1/2, 1/2].
__device__ __forceinline__ void turns_sincos(float t, float* s, float* c) {
    t -= __fadd_rn(__fadd_rn(t, 12582912.f), -12582912.f);
    sincos_hw(6.28318530717958647692f * t, s, c);
}
__device__ __forceinline__ void turns_sincos(double t, double* s, double* c) {
    t -= rint(t);
    sincospi(2.0 * t, s, c);
}

// Coordinates relative to the target leaf centre are kept as unevaluated sums
// hi + lo of two values of type T (lo = 0 in double precision), so that the
// difference of two nearby points is accurate to the precision of the
// difference itself, not of the coordinates: random clouds hold pairs far
// closer than the mean spacing, whose 1/r dominates the near field.
template <typename T> struct Split {
    T hi, lo;
};
template <typename T> __device__ __forceinline__ Split<T> split(double d) {
    Split<T> o;
    o.hi = (T)d;
    o.lo = sizeof(T) == 4 ? (T)(d - (double)o.hi) : (T)0;
    return o;
}

// Near field in the arithmetic type T (used for float64): one block per work
// unit (a target leaf and at most kP2PUnitSources of its near sources); the
// unit's partial sums go to part[] and are reduced per target by k_p2p_reduce.
template <typename T, int RB>
__global__ void __launch_bounds__(128) k_p2p(DevCommon c, const typename Cplx<T>::type* __restrict__ qs,
                                             typename Cplx<T>::type* __restrict__ part, int R, int rb0) {
    using C = typename Cplx<T>::type;
    constexpr bool kSplit = sizeof(T) == 4;
    __shared__ T sx[128], sy[128], sz[128];
    __shared__ T lx[kSplit ? 128 : 1], ly[kSplit ? 128 : 1], lz[kSplit ? 128 : 1];
    __shared__ C sq[RB][128];
    __shared__ C red[4][64][RB];
    const int u = c.sh_unit ? c.sh_unit[blockIdx.x] : (int)blockIdx.x;   // work unit (of the shard)
    const int cell = DEFMM_IX(c, c.p2p_leaf[DEFMM_IX(c, c.p2p_unit_leaf[u], c.n_leaf_all)], c.n_cell_t);
    const int tb = c.ct_beg[cell], te = c.ct_end[cell];
    const int64_t pbase = c.p2p_part[u];
    const double side = c.level_side[c.ct_level[cell]];
    const double cx = c.ct_corner[3 * cell] + 0.5 * side;
    const double cy = c.ct_corner[3 * cell + 1] + 0.5 * side;
    const double cz = c.ct_corner[3 * cell + 2] + 0.5 * side;
    const int nr = min(RB, R - rb0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double kap = kappa_of(c, cell), eps = eps_of(c, cell);
    const T kpar = kSplit ? (T)(kap * kInv2Pi) : (T)kap;
    const T eps2 = (T)(eps * eps);
    const int r0 = c.p2p_unit_off[u], r1 = c.p2p_unit_off[u + 1];
    for (int t0 = tb; t0 < te; t0 += 64) {
        const int ia = t0 + lane, ib = t0 + lane + 32;
        Split<T> xa{0, 0}, ya{0, 0}, za{0, 0}, xb{0, 0}, yb{0, 0}, zb{0, 0};
        if (ia < te) {
            xa = split<T>(c.Xs[3 * (int64_t)ia] - cx); ya = split<T>(c.Xs[3 * (int64_t)ia + 1] - cy);
            za = split<T>(c.Xs[3 * (int64_t)ia + 2] - cz);
        }
        if (ib < te) {
            xb = split<T>(c.Xs[3 * (int64_t)ib] - cx); yb = split<T>(c.Xs[3 * (int64_t)ib + 1] - cy);
            zb = split<T>(c.Xs[3 * (int64_t)ib + 2] - cz);
        }
        C acca[RB], accb[RB];
#pragma unroll
        for (int r = 0; r < RB; ++r) { acca[r] = czero<C>(); accb[r] = czero<C>(); }
        for (int rr = r0; rr < r1; ++rr) {
            const int sb = DEFMM_IX(c, c.p2p_sbeg[rr], c.ny + 1), se = DEFMM_IX(c, c.p2p_send[rr], c.ny + 1);
            for (int s0 = sb; s0 < se; s0 += 128) {
                const int ns = min(128, se - s0);
                __syncthreads();
                if (threadIdx.x < ns) {
                    const int64_t j = s0 + threadIdx.x;
                    const Split<T> ux = split<T>(c.Ys[3 * j] - cx), uy = split<T>(c.Ys[3 * j + 1] - cy),
                                   uz = split<T>(c.Ys[3 * j + 2] - cz);
                    sx[threadIdx.x] = ux.hi; sy[threadIdx.x] = uy.hi; sz[threadIdx.x] = uz.hi;
                    if (kSplit) { lx[threadIdx.x] = ux.lo; ly[threadIdx.x] = uy.lo; lz[threadIdx.x] = uz.lo; }
#pragma unroll
                    for (int r = 0; r < RB; ++r)
                        sq[r][threadIdx.x] = r < nr ? qs[(int64_t)(rb0 + r) * c.ny + j] : czero<C>();
                }
                __syncthreads();
                for (int k = warp; k < ns; k += 4) {
                    T dxa = xa.hi - sx[k], dya = ya.hi - sy[k], dza = za.hi - sz[k];
                    T dxb = xb.hi - sx[k], dyb = yb.hi - sy[k], dzb = zb.hi - sz[k];
                    if (kSplit) {
                        const T ex = lx[k], ey = ly[k], ez = lz[k];
                        dxa += xa.lo - ex; dya += ya.lo - ey; dza += za.lo - ez;
                        dxb += xb.lo - ex; dyb += yb.lo - ey; dzb += zb.lo - ez;
                    }
                    const C ga = helmholtz(dxa, dya, dza, kpar, eps2, (T)c.damping, c.radial_power);
                    const C gb = helmholtz(dxb, dyb, dzb, kpar, eps2, (T)c.damping, c.radial_power);
#pragma unroll
                    for (int r = 0; r < RB; ++r) {
                        const C qv = sq[r][k];
                        cfma(acca[r], ga, qv);
                        cfma(accb[r], gb, qv);
                    }
                }
            }
        }
#pragma unroll
        for (int r = 0; r < RB; ++r) { red[warp][lane][r] = acca[r]; red[warp][lane + 32][r] = accb[r]; }
        __syncthreads();
        if (threadIdx.x < 64) {
            const int i = t0 + threadIdx.x;
            if (i < te) {
                for (int r = 0; r < nr; ++r) {
                    C s = red[0][threadIdx.x][r];
                    s = cadd(s, red[1][threadIdx.x][r]);
                    s = cadd(s, red[2][threadIdx.x][r]);
                    s = cadd(s, red[3][threadIdx.x][r]);
                    part[(int64_t)(rb0 + r) * c.p2p_parts + pbase + (i - tb)] = s;
                }
            }
        }
        __syncthreads();
    }
}

// Single-precision near field.  One block per work unit (a target leaf and
// at most kP2PUnitSources of its near sources, heaviest first); pairs of the
// leaf's targets are spread over the 128 threads as target pair x
// source-split, so small leaves do not leave lanes idle.
// The leaf's source ranges are read as one concatenated sequence cut into
// full tiles of 128 (a thread finds its source by binary search in the
// ranges' prefix offsets), and the next tile is loaded into registers while
// the current one is consumed.
// Coordinates: every point is staged relative to a local origin o (the
// leaf's first target) as a single float v' = (hi - o_hi) + (lo - o_lo), from
// the hi + lo float pairs relative to the cube centre.  A difference
// t' - s' then carries an error of about 2^-24 (|t'| + |s'|), small against
// the distance r except for near-coincident pairs.  Those pairs, 64 r^2 <=
// |t'|^2 + |s'|^2 (r below about a sixth of |t'| + |s'|, so the single-float
// difference would keep fewer than about 21 bits), are formed again from the
// hi + lo pairs, where the difference is accurate to the precision of the
// difference itself (random clouds hold pairs far closer than the mean
// spacing, whose 1/r dominates the near field).  Coincident points (r^2 <=
// eps_self^2, Sec. 5.3) always take that branch (eps_self^2 is folded into
// the test) and get r^2 = 2^100: their term is below 2^-50 of the charge (zero
// once damped), nothing at single precision, without a select on every pair.
// Phase: with REDUCE the phase kappa r / (2 pi) is reduced exactly to
// [-1/2, 1/2] turns before the hardware sine and cosine on [-pi, pi]; without
// it (plans whose near-field phases are all below 90 pi, bounded on the host
// from the cell pairs) the hardware sine and cosine take kappa r directly:
// PTX documents sin.approx / cos.approx to 2^-20.5 absolute error on
// [-100 pi, 100 pi], and the rounding of the argument is the same as that of
// the reduced form.  Charges are pre-scaled by 1/(4 pi) when staged; partial
// sums are reduced over the splits in a fixed order.
constexpr int kP2PRanges = kP2PUnitRanges;   // ranges of a work unit, held in shared memory

// v - o for hi + lo pairs, as one float
__device__ __forceinline__ float3 local_coords(float4 h, float4 l, float4 oh, float4 ol) {
    return make_float3((h.x - oh.x) + (l.x - ol.x), (h.y - oh.y) + (l.y - ol.y), (h.z - oh.z) + (l.z - ol.z));
}

// e^{(i kappa - lambda) r} / r^P (times a staged 1/(4 pi) in the charges) for
// r^2: KIND 0 is P = 1 without damping, 1 is P = 1 with it, 2 is P = 2 (with
// the damping term, exact at lambda = 0).  kph is kappa / (2 pi) with REDUCE
// (phase in turns), else kappa (phase in radians).
template <int KIND, bool REDUCE>
__device__ __forceinline__ float2 near_kernel(float r2, float kph, float lam2) {
    const float rinv = rsqrt_hw(r2);
    const float r = r2 * rinv;
    float sn, cs;
    if (REDUCE) turns_sincos(r * kph, &sn, &cs);
    else sincos_hw(r * kph, &sn, &cs);
    float amp = KIND == 2 ? rinv * rinv : rinv;
    if (KIND >= 1) amp *= ex2_hw(-lam2 * r);
    return make_float2(cs * amp, sn * amp);
}

// r^2 of a near-coincident pair from the hi + lo pairs; 2^100 for coincident points
__device__ __forceinline__ float exact_r2(float4 th, float4 tl, float4 sh, float4 sl, float eps2) {
    const float dx = (th.x - sh.x) + (tl.x - sl.x);
    const float dy = (th.y - sh.y) + (tl.y - sl.y);
    const float dz = (th.z - sh.z) + (tl.z - sl.z);
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    return r2 > eps2 ? r2 : 0x1p100f;
}

template <int RB, int KIND = 0, bool REDUCE = true>
__global__ void __launch_bounds__(128, RB == 1 ? 8 : 1) k_p2p_f32(DevCommon c, const float2* __restrict__ qs,
                                                 float2* __restrict__ part, int R, int rb0) {
    __shared__ float4 sa[128];   // source relative to the local origin; w: |s'|^2 + 64 eps_self^2
    __shared__ float4 sh[128];   // hi x, y, z relative to the cube centre
    __shared__ float4 sl[128];   // lo x, y, z
    __shared__ float2 sq[RB][128];
    __shared__ float2 red[RB][128];
    __shared__ int rbeg[kP2PRanges], roff[kP2PRanges + 1];
    const int u = c.sh_unit ? c.sh_unit[blockIdx.x] : (int)blockIdx.x;   // work unit (of the shard)
    const int cell = DEFMM_IX(c, c.p2p_leaf[DEFMM_IX(c, c.p2p_unit_leaf[u], c.n_leaf_all)], c.n_cell_t);
    const int tb = c.ct_beg[cell], te = c.ct_end[cell];
    const int64_t pbase = c.p2p_part[u];
    const int nr = min(RB, R - rb0);
    const float kph = (float)(REDUCE ? kappa_of(c, cell) * kInv2Pi : kappa_of(c, cell));
    const float eps2 = (float)(eps_of(c, cell) * eps_of(c, cell));
    const float e64 = 64.f * eps2;
    const float inv4pi = (float)kInv4Pi;
    const float lam2 = (float)(c.damping * kLog2E);     // damping in powers of 2 per unit length
    const float4 oh = c.Xh[tb], ol = c.Xl[tb];          // local origin: the leaf's first target
    const int r0 = c.p2p_unit_off[u], r1 = c.p2p_unit_off[u + 1];
    for (int t0 = tb; t0 < te; t0 += 256) {
        // two targets per thread: target pairs (2i, 2i+1) x source splits
        const int nt = min(256, te - t0);
        const int np = (nt + 1) >> 1;
        const int splits = 128 / np;
        const int ti = threadIdx.x % np, sj = threadIdx.x / np;
        const bool active = sj < splits;
        const int ia = 2 * ti, ib = 2 * ti + 1;
        const bool has_b = ib < nt;
        float3 ta = make_float3(0.f, 0.f, 0.f), tb3 = ta;
        if (active) {
            ta = local_coords(c.Xh[t0 + ia], c.Xl[t0 + ia], oh, ol);
            tb3 = has_b ? local_coords(c.Xh[t0 + ib], c.Xl[t0 + ib], oh, ol) : ta;
        }
        const float na2 = fmaf(ta.x, ta.x, fmaf(ta.y, ta.y, ta.z * ta.z));
        const float nb2 = fmaf(tb3.x, tb3.x, fmaf(tb3.y, tb3.y, tb3.z * tb3.z));
        float2 acc[RB], bcc[RB];
#pragma unroll
        for (int r = 0; r < RB; ++r) { acc[r] = make_float2(0.f, 0.f); bcc[r] = make_float2(0.f, 0.f); }
        for (int g0 = r0; g0 < r1; g0 += kP2PRanges) {          // batches of ranges
            const int ng = min(kP2PRanges, r1 - g0);
            __syncthreads();
            for (int k = threadIdx.x; k < ng; k += blockDim.x) {
                rbeg[k] = c.p2p_sbeg[g0 + k];
                roff[k] = c.p2p_soff[g0 + k] - c.p2p_soff[g0];
            }
            if (threadIdx.x == 0) roff[ng] = c.p2p_soff[g0 + ng - 1] - c.p2p_soff[g0] + c.p2p_send[g0 + ng - 1] - c.p2p_sbeg[g0 + ng - 1];
            __syncthreads();
            const int total = roff[ng];
            auto source_of = [&](int f) {
                int lo = 0, hi = ng - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (roff[mid] <= f) lo = mid; else hi = mid - 1;
                }
                return rbeg[lo] + (f - roff[lo]);
            };
            float4 nh = make_float4(0.f, 0.f, 0.f, 0.f), nl = nh;
            float2 nq[RB];
            auto fetch = [&](int f0) {
                if (f0 + (int)threadIdx.x < total) {
                    const int64_t j = DEFMM_IX(c, (int64_t)source_of(f0 + threadIdx.x), c.ny);
                    nh = c.Yh[j];
                    nl = c.Yl[j];
#pragma unroll
                    for (int r = 0; r < RB; ++r)
                        nq[r] = r < nr ? qs[(int64_t)(rb0 + r) * c.ny + j] : make_float2(0.f, 0.f);
                }
            };
            fetch(0);
            for (int f0 = 0; f0 < total; f0 += 128) {
                const int ns = min(128, total - f0);
                __syncthreads();                 // previous tile consumed
                if (threadIdx.x < ns) {
                    const float3 s = local_coords(nh, nl, oh, ol);
                    sa[threadIdx.x] = make_float4(s.x, s.y, s.z, fmaf(s.x, s.x, fmaf(s.y, s.y, fmaf(s.z, s.z, e64))));
                    sh[threadIdx.x] = nh;
                    sl[threadIdx.x] = nl;
#pragma unroll
                    for (int r = 0; r < RB; ++r) sq[r][threadIdx.x] = make_float2(nq[r].x * inv4pi, nq[r].y * inv4pi);
                }
                __syncthreads();
                if (f0 + 128 < total) fetch(f0 + 128);   // in flight during the compute below
                if (active) {
                    for (int k = sj; k < ns; k += splits) {
                        const float4 s = sa[k];
                        float ra, rb;
                        {
                            const float dx = ta.x - s.x, dy = ta.y - s.y, dz = ta.z - s.z;
                            ra = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                        }
                        {
                            const float dx = tb3.x - s.x, dy = tb3.y - s.y, dz = tb3.z - s.z;
                            rb = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                        }
                        // near-coincident (or coincident) pairs, rare: the difference again from hi + lo
                        const bool ca = fmaf(ra, 64.f, -s.w) <= na2, cb = fmaf(rb, 64.f, -s.w) <= nb2;
                        if (__builtin_expect(ca || cb, 0)) {
                            const float4 h = sh[k], l = sl[k];
                            if (ca) ra = exact_r2(c.Xh[t0 + ia], c.Xl[t0 + ia], h, l, eps2);
                            if (cb) rb = exact_r2(c.Xh[t0 + (has_b ? ib : ia)], c.Xl[t0 + (has_b ? ib : ia)], h, l, eps2);
                        }
                        const float2 ga = near_kernel<KIND, REDUCE>(ra, kph, lam2);
                        const float2 gb = near_kernel<KIND, REDUCE>(rb, kph, lam2);
#pragma unroll
                        for (int r = 0; r < RB; ++r) {
                            const float2 q = sq[r][k];
                            acc[r].x = fmaf(ga.x, q.x, fmaf(-ga.y, q.y, acc[r].x));
                            acc[r].y = fmaf(ga.x, q.y, fmaf(ga.y, q.x, acc[r].y));
                            bcc[r].x = fmaf(gb.x, q.x, fmaf(-gb.y, q.y, bcc[r].x));
                            bcc[r].y = fmaf(gb.x, q.y, fmaf(gb.y, q.x, bcc[r].y));
                        }
                    }
                }
            }
        }
        // reduce over the splits in order: first the a targets, then the b targets
#pragma unroll
        for (int r = 0; r < RB; ++r) red[r][threadIdx.x] = acc[r];
        __syncthreads();
        if (active && sj == 0)
            for (int r = 0; r < nr; ++r) {
                float2 s = red[r][ti];
                for (int q = 1; q < splits; ++q) { s.x += red[r][ti + q * np].x; s.y += red[r][ti + q * np].y; }
                part[(int64_t)(rb0 + r) * c.p2p_parts + pbase + (t0 + ia - tb)] = s;
            }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < RB; ++r) red[r][threadIdx.x] = bcc[r];
        __syncthreads();
        if (active && sj == 0 && has_b)
            for (int r = 0; r < nr; ++r) {
                float2 s = red[r][ti];
                for (int q = 1; q < splits; ++q) { s.x += red[r][ti + q * np].x; s.y += red[r][ti + q * np].y; }
                part[(int64_t)(rb0 + r) * c.p2p_parts + pbase + (t0 + ib - tb)] = s;
            }
        __syncthreads();
    }
}

template <int KIND, bool REDUCE>
void launch_p2p_f32(int rb, unsigned nu, const DevCommon& c, const float2* qs, float2* part, int R, int rb0,
                    cudaStream_t stream) {
    if (rb == 1) k_p2p_f32<1, KIND, REDUCE><<<nu, 128, 0, stream>>>(c, qs, part, R, rb0);
    else if (rb == 16) k_p2p_f32<16, KIND, REDUCE><<<nu, 128, 0, stream>>>(c, qs, part, R, rb0);
    else if (rb == 8) k_p2p_f32<8, KIND, REDUCE><<<nu, 128, 0, stream>>>(c, qs, part, R, rb0);
    else k_p2p_f32<4, KIND, REDUCE><<<nu, 128, 0, stream>>>(c, qs, part, R, rb0);
}

// Sums each target's partial near-field sums over its leaf's work units, in
// the units' source order, into the potentials.
template <typename C>
__global__ void __launch_bounds__(128) k_p2p_reduce(DevCommon c, const C* __restrict__ part, C* __restrict__ ps, int R) {
    const int li = c.sh_leaf ? c.sh_leaf[blockIdx.x] : (int)blockIdx.x;  // leaf (of the shard)
    const int cell = DEFMM_IX(c, c.p2p_leaf[li], c.n_cell_t);
    const int tb = c.ct_beg[cell], te = c.ct_end[cell];
    const int u0 = c.p2p_leaf_off[li], u1 = c.p2p_leaf_off[li + 1];
    for (int r = 0; r < R; ++r)
        for (int j = tb + threadIdx.x; j < te; j += blockDim.x) {
            C s = czero<C>();
            for (int k = u0; k < u1; ++k) s = cadd(s, part[(int64_t)r * c.p2p_parts + c.p2p_part[c.p2p_leaf_units[k]] + (j - tb)]);
            ps[(int64_t)r * c.nx + j] = s;
        }
}

// ------------------------------------------------------------------ P2M
// The plane wave of S_a^u separates: exp(i kappa <y_a - y, u>) = P_u(a) conj(E_u(y))
// with E_u(y) = exp(i kappa <y - c, u>) (c the cell centre) and P_u(a) the
// tabulated node factors of the direction's slot, so
//   M_u[a] = P_u(a) * sum_y S_a(y_hat) (q(y) conj(E_u(y))),
// one phase per (particle, direction) and a real-basis contraction.
constexpr int kP2MChunk = 64;     // particles staged at a time
constexpr int kMaxExp = 32;       // expansions handled per pass

template <typename T, int RB, int PC = 0>
__global__ void __launch_bounds__(128) k_p2m(DevCommon c, DevTyped<T> t, const typename Cplx<T>::type* __restrict__ qs,
                                             typename Cplx<T>::type* __restrict__ M, int R, int rb0, int epass) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // [kP2MChunk][3][p] Lagrange values, then [RB][epass][kP2MChunk] modified charges
    T* lag = reinterpret_cast<T*>(smem_raw);
    const int p = PC ? PC : c.p, P3 = p * p * p;
    C* qm = reinterpret_cast<C*>(smem_raw + (((size_t)kP2MChunk * 3 * p * sizeof(T) + 15) / 16) * 16);
    const int cell = DEFMM_IX(c, c.p2m_cells[blockIdx.x], c.n_cell_s);
    const int b = c.cs_beg[cell], e = c.cs_end[cell];
    const double side = c.level_side[c.cs_level[cell]];
    const double h = side / (p - 1);
    const double cor[3] = {c.cs_corner[3 * cell], c.cs_corner[3 * cell + 1], c.cs_corner[3 * cell + 2]};
    const int nr = min(RB, R - rb0);
    const T k2pi = (T)(kappa_of(c, cell) * kInv2Pi);
    const int ex0 = DEFMM_IX(c, c.m_first[cell], c.n_mult + 1), nex = DEFMM_IX(c, c.m_count[cell], c.n_mult - ex0 + 1);
    for (int e0 = 0; e0 < nex; e0 += epass) {
        const int ne = min(epass, nex - e0);
        // outputs of this thread: (expansion, node) pairs o = threadIdx.x + 128 v (ne * P3 <= 16 * 128)
        const int nout = ne * P3;
        C acc[16][RB];      // up to 16 outputs per thread (ne * P3 <= 2048)
#pragma unroll
        for (int v = 0; v < 16; ++v)
#pragma unroll
            for (int r = 0; r < RB; ++r) acc[v][r] = czero<C>();
        for (int j0 = b; j0 < e; j0 += kP2MChunk) {
            const int nj = min(kP2MChunk, e - j0);
            __syncthreads();
            for (int idx = threadIdx.x; idx < nj * 3 * p; idx += blockDim.x) {
                const int j = idx / (3 * p), rem = idx - j * 3 * p, ax = rem / p, m = rem - ax * p;
                const double d = c.Ys[3 * (int64_t)(j0 + j) + ax] - cor[ax];
                lag[idx] = lagrange<T>(p, m, (T)(d / h));
                (void)j;
            }
            for (int idx = threadIdx.x; idx < ne * nj; idx += blockDim.x) {
                const int ee = idx / nj, j = idx - ee * nj;
                const int slot = DEFMM_IX(c, c.m_slot[ex0 + e0 + ee] + 1, c.n_slot + 1) - 1;
                C ph = mk((T)1, (T)0);
                if (slot >= 0) {
                    T arg = 0;
                    for (int ax = 0; ax < 3; ++ax)
                        arg += (T)(c.Ys[3 * (int64_t)(j0 + j) + ax] - cor[ax] - 0.5 * side) * (T)c.slot_u[3 * slot + ax];
                    T sn, cs;
                    turns_sincos(arg * k2pi, &sn, &cs);
                    ph = mk(cs, -sn);                                  // conj(E_u(y))
                }
#pragma unroll
                for (int r = 0; r < RB; ++r) {
                    const C q = r < nr ? qs[(int64_t)(rb0 + r) * c.ny + j0 + j] : czero<C>();
                    qm[((size_t)r * epass + ee) * kP2MChunk + j] = cmul(q, ph);
                }
            }
            __syncthreads();
#pragma unroll
            for (int v = 0; v < 16; ++v) {
                const int o = threadIdx.x + v * 128;
                if (o < nout) {
                    const int ee = o / P3, a = o - ee * P3;
                    const int a0 = a % p, a1 = (a / p) % p, a2 = a / (p * p);
                    for (int j = 0; j < nj; ++j) {
                        const T* lj = lag + j * 3 * p;
                        const T w = lj[a0] * lj[p + a1] * lj[2 * p + a2];
#pragma unroll
                        for (int r = 0; r < RB; ++r) {
                            const C q = qm[((size_t)r * epass + ee) * kP2MChunk + j];
                            acc[v][r].x = fma(w, q.x, acc[v][r].x);
                            acc[v][r].y = fma(w, q.y, acc[v][r].y);
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int v = 0; v < 16; ++v) {
            const int o = threadIdx.x + v * 128;
            if (o < nout) {
                const int ee = o / P3, a = o - ee * P3;
                const int ex = ex0 + e0 + ee;
                const int slot = DEFMM_IX(c, c.m_slot[ex] + 1, c.n_slot + 1) - 1;
                C ph = mk((T)1, (T)0);
                if (slot >= 0) {
                    const int a0 = a % p, a1 = (a / p) % p, a2 = a / (p * p);
                    const C* P = t.slot_P + (int64_t)slot * 3 * p;
                    ph = cmul(cmul(P[a0], P[p + a1]), P[2 * p + a2]);
                }
                for (int r = 0; r < nr; ++r) M[((int64_t)ex * R + rb0 + r) * P3 + a] = cmul(acc[v][r], ph);
            }
        }
    }
}

// Expansions per pass of k_p2m: at most 16 outputs per thread and 64 KB of modified charges.
__host__ int p2m_epass(int P3, int RB, size_t creal) {
    int ep = kMaxExp;
    ep = ep < (16 * 128) / P3 ? ep : (16 * 128) / P3;
    const int by_smem = (int)((64 * 1024) / ((size_t)RB * kP2MChunk * 2 * creal));
    ep = ep < by_smem ? ep : by_smem;
    return ep < 1 ? 1 : ep;
}
__host__ size_t p2m_smem(int p, int RB, int epass, size_t creal) {
    return ((size_t)kP2MChunk * 3 * p * creal + 15) / 16 * 16 + (size_t)RB * epass * kP2MChunk * 2 * creal;
}

// ------------------------------------------------------------------ warp-per-item helpers
// M2M, L2L and M2F work on one small expansion at a time: one warp per item,
// synchronised with __syncwarp only; blocks hold `wpb` independent warps.
// ------------------------------------------------------------------ M2M
// One warp per (father expansion, right-hand side) (entry: father id, 8 son ids or -1):
//   M_f^v[a] = P_v(a) sum_sons sum_b T_o[a, b] conj(Q_v,o(b)) M_son[b],
// T_o the tensor product of the 1-D son->father matrices, applied as three
// 1-D passes (Sec. 5.2.1).
template <typename T, int PC = 0>
__global__ void __launch_bounds__(256) k_m2m(DevCommon c, DevTyped<T> t, const int32_t* __restrict__ list, int64_t n,
                                             typename Cplx<T>::type* __restrict__ M, int R) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int p = PC ? PC : c.p, P3 = p * p * p;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __shared__ T m1s[2 * 8 * 8];
    for (int i = threadIdx.x; i < 2 * p * p; i += blockDim.x) m1s[i] = t.m1[i];
    __syncthreads();
    const int64_t wid = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;   // (item, right-hand side)
    const int64_t item = wid / R;
    const int rr = (int)(wid % R);
    if (item >= n) return;
    C* A = reinterpret_cast<C*>(smem_raw) + (size_t)warp * (2 * P3 + 72);
    C* B = A + P3;
    C* Ps = B + P3;          // [3][p]
    C* Qs = Ps + 24;         // [3][2][p]
    const int32_t* ent = list + 9 * item;
    const int ep = DEFMM_IX(c, ent[0], c.n_mult);
    const int slot = DEFMM_IX(c, c.m_slot[ep] + 1, c.n_slot + 1) - 1;
    for (int i = lane; i < 3 * p; i += 32) Ps[i] = slot >= 0 ? t.slot_P[(int64_t)slot * 3 * p + i] : mk((T)1, (T)0);
    for (int i = lane; i < 6 * p; i += 32) Qs[i] = slot >= 0 ? t.slot_Q[(int64_t)slot * 6 * p + i] : mk((T)1, (T)0);
    __syncwarp();
    {   // this warp's right-hand side
        const int r = rr;
        C acc[16];
#pragma unroll
        for (int v = 0; v < 16; ++v) acc[v] = czero<C>();
        for (int o = 0; o < 8; ++o) {
            const int ce = ent[1 + o] < 0 ? -1 : DEFMM_IX(c, ent[1 + o], c.n_mult);
            if (ce < 0) continue;
            const int ox = o & 1, oy = (o >> 1) & 1, oz = (o >> 2) & 1;
            const T* mx = m1s + ox * p * p;
            const T* my = m1s + oy * p * p;
            const T* mz = m1s + oz * p * p;
            for (int a = lane; a < P3; a += 32) {
                const int b0 = a % p, b1 = (a / p) % p, b2 = a / (p * p);
                const C q = cmul(cmul(Qs[(0 * 2 + ox) * p + b0], Qs[(1 * 2 + oy) * p + b1]), Qs[(2 * 2 + oz) * p + b2]);
                A[a] = cmulc(M[((int64_t)ce * R + r) * P3 + a], q);
            }
            __syncwarp();
            for (int a = lane; a < P3; a += 32) {  // x: (bz, by, ax)
                const int a0 = a % p, rest = a - a0;
                C s = czero<C>();
                for (int k = 0; k < p; ++k) { C v = A[rest + k]; T m = mx[a0 * p + k]; s.x += m * v.x; s.y += m * v.y; }
                B[a] = s;
            }
            __syncwarp();
            for (int a = lane; a < P3; a += 32) {  // y: (bz, ay, ax)
                const int a0 = a % p, a1 = (a / p) % p, a2 = a / (p * p);
                C s = czero<C>();
                for (int k = 0; k < p; ++k) { C v = B[(a2 * p + k) * p + a0]; T m = my[a1 * p + k]; s.x += m * v.x; s.y += m * v.y; }
                A[a] = s;
            }
            __syncwarp();
#pragma unroll
            for (int v = 0; v < 16; ++v) {  // z: (az, ay, ax), accumulate
                const int a = lane + v * 32;
                if (a < P3) {
                    const int a01 = a % (p * p), a2 = a / (p * p);
                    C s = acc[v];
                    for (int k = 0; k < p; ++k) { C w = A[k * p * p + a01]; T m = mz[a2 * p + k]; s.x += m * w.x; s.y += m * w.y; }
                    acc[v] = s;
                }
            }
            __syncwarp();
        }
#pragma unroll
        for (int v = 0; v < 16; ++v) {
            const int a = lane + v * 32;
            if (a < P3) {
                const int a0 = a % p, a1 = (a / p) % p, a2 = a / (p * p);
                const C ph = cmul(cmul(Ps[0 * p + a0], Ps[1 * p + a1]), Ps[2 * p + a2]);
                M[((int64_t)ep * R + r) * P3 + a] = cmul(acc[v], ph);
            }
        }
    }
}

// ------------------------------------------------------------------ M2F
// One warp per (Fourier multipole, right-hand side): zero-pad and forward DFT (F chi, Sec. 4.1.1),
// pruned to the p non-zero inputs per line.
template <typename T, int PC = 0, int NC = 0>
__global__ void __launch_bounds__(256) k_m2f(DevCommon c, DevTyped<T> t, const typename Cplx<T>::type* __restrict__ M,
                                             typename Cplx<T>::type* __restrict__ Mhat, int R) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int p = PC ? PC : c.p, N = NC ? NC : c.N, P3 = p * p * p, NF = N * N * N, NFpad = c.NFpad;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __shared__ C tws[16];
    if (threadIdx.x < N) tws[threadIdx.x] = mk(t.tw[threadIdx.x].x, -t.tw[threadIdx.x].y);   // e^{-2 pi i m / N}
    __syncthreads();
    const int64_t wid = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;   // (item, right-hand side)
    const int64_t item = wid / R;
    const int rr = (int)(wid % R);
    if (item >= c.n_m2f) return;
    C* A = reinterpret_cast<C*>(smem_raw) + (size_t)warp * (P3 + p * p * N + p * N * N);
    C* B = A + P3;              // [bz][by][xi_x]   p*p*N
    C* D = B + p * p * N;       // [bz][xi_y][xi_x] p*N*N
    const int e = DEFMM_IX(c, c.m2f_list[item], c.n_mult);
    {   // this warp's right-hand side
        const int r = rr;
        for (int a = lane; a < P3; a += 32) A[a] = M[((int64_t)e * R + r) * P3 + a];
        __syncwarp();
        for (int i = lane; i < p * p * N; i += 32) {
            const int xx = i % N, rest = i / N;  // rest = bz*p + by
            C s = czero<C>();
            for (int b = 0, w = 0; b < p; ++b) {   // w = xx * b mod N
                cfma(s, A[rest * p + b], tws[w]);
                w += xx;
                w -= w >= N ? N : 0;
            }
            B[i] = s;
        }
        __syncwarp();
        for (int i = lane; i < p * N * N; i += 32) {
            const int xx = i % N, yy = (i / N) % N, bz = i / (N * N);
            C s = czero<C>();
            for (int b = 0, w = 0; b < p; ++b) {   // w = yy * b mod N
                cfma(s, B[(bz * p + b) * N + xx], tws[w]);
                w += yy;
                w -= w >= N ? N : 0;
            }
            D[i] = s;
        }
        __syncwarp();
        C* out = Mhat + ((int64_t)item * R + r) * NFpad;
        for (int i = lane; i < NFpad; i += 32) {
            C s = czero<C>();
            if (i < NF) {
                const int xy = i % (N * N), zz = i / (N * N);
                for (int b = 0, w = 0; b < p; ++b) {   // w = zz * b mod N
                    cfma(s, D[b * N * N + xy], tws[w]);
                    w += zz;
                    w -= w >= N ? N : 0;
                }
            }
            out[i] = s;
        }
        __syncwarp();
    }
}

// Warps per block for the warp-per-item kernels, given the shared bytes of one warp.
__host__ int warps_per_block(size_t per_warp) {
    int w = (int)((180 * 1024) / (per_warp ? per_warp : 1));
    return w < 1 ? 1 : (w > 8 ? 8 : w);
}

// ------------------------------------------------------------------ M2L (+F2L)
// Asynchronous bulk copies (TMA, cp.async.bulk) into shared memory, completed
// on mbarriers.  Every wait is bounded; a wait that gives up raises the plan's
// error flag and the block stops.
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}
constexpr int kMaxSpin = 1 << 22;
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int spins = kMaxSpin) {
    for (int it = 0; it < spins; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Self-test of the bounded wait: one block waits on an mbarrier phase that no
// arrival completes, gives up after `spins` polls and raises *flag, exactly as
// the pipelined kernels do when a copy never lands; nothing faults or hangs.
__global__ void k_wait_probe(int* flag, int spins) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    const bool ok = mbar_wait(&bar, 0, spins);
    if (!ok && threadIdx.x == 0) atomicExch(flag, 1);
}

constexpr int kM2LMaxStages = 3;  // ring depth (runtime S <= this)
constexpr size_t kSmemLimit = 227 * 1024 - 2048;   // dynamic shared memory per block, with room for static

// One block per M2L group: up to 8 sibling target expansions sharing a father
// cell and a direction.  The group's pairs come in chunks; a chunk's blocks
// (the distinct canonical spectra and source Fourier multipoles it uses, one
// contiguous NFpad block each) are brought into a ring of S shared-memory
// stages by TMA bulk copies (cp.async.bulk) issued by thread 0 and completed
// on mbarriers, while the block computes an earlier chunk; every staged block
// serves all pairs of the chunk that use it.  Thread i owns the Fourier
// samples xi = i + v*blockDim (v < VPT) and accumulates, for each pair of
// member m, spectrum(xi') * Mhat(xi), xi'_{sigma(a)} = s_a xi_a mod N: the
// pair's symmetry is applied as a gather from shared memory.  The inverse DFT
// and the crop to the p^3 grid of each member follow in shared memory.
template <typename T, int VPT, int MAXT>
__global__ void __launch_bounds__(MAXT) k_m2l(DevCommon c, DevTyped<T> t, const typename Cplx<T>::type* __restrict__ Mhat,
                                              typename Cplx<T>::type* __restrict__ L, int R, int S) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int p = c.p, N = c.N, NF = c.NF, NFpad = c.NFpad, P3 = c.P3;
    const uint32_t blk_bytes = (uint32_t)(NFpad * sizeof(C));
    C* ring = reinterpret_cast<C*>(smem_raw);
    const int stage_elems = c.chk_stage_blocks[0] * NFpad;
    // F2L work arrays reuse the ring once every copy has landed
    C* Lh = ring;                              // NF
    C* T1 = Lh + NF;                           // [az][xi_y][xi_x]  p*N*N
    C* T2 = T1 + p * N * N;                    // [az][ay][xi_x]    p*p*N
    __shared__ __align__(8) uint64_t bars[kM2LMaxStages];
    __shared__ C tws[16];
    __shared__ int stride[6][3];               // N^sigma(a) for each axis permutation
    const int g = c.sh_grp ? c.sh_grp[blockIdx.x] : (int)blockIdx.x;   // group (of the shard)
    const int mem0 = c.grp_member_off[g], nm = c.grp_member_off[g + 1] - mem0;
    const int ch0 = c.grp_chunk_off[g], nchunks = c.grp_chunk_off[g + 1] - ch0;
    if (threadIdx.x < N) tws[threadIdx.x] = t.tw[threadIdx.x];
    if (threadIdx.x < 18) {
        const int q = kPermDev[threadIdx.x / 3][threadIdx.x % 3];
        stride[threadIdx.x / 3][threadIdx.x % 3] = q == 0 ? 1 : (q == 1 ? N : N * N);
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
        mbar_fence_init();
    }
    int xi[VPT], cp[VPT][3], cn[VPT][3];
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
        xi[v] = threadIdx.x + v * blockDim.x;
        const int f = xi[v] < NF ? xi[v] : 0;
        cp[v][0] = f % N; cp[v][1] = (f / N) % N; cp[v][2] = f / (N * N);
#pragma unroll
        for (int a = 0; a < 3; ++a) cn[v][a] = cp[v][a] == 0 ? 0 : N - cp[v][a];
    }
    __syncthreads();
    uint32_t use = 0;  // chunks consumed so far: stage = use % S, parity = (use / S) & 1
    const T scale = (T)1 / (T)NF;
    // producer: the blocks of chunk ch (right-hand side r) into stage st
    auto issue = [&](int ch, int r, int st) {
        const int cc = ch0 + ch;
        const int b0 = c.chk_blk_off[cc], nb = c.chk_blk_off[cc + 1] - b0, nsp = c.chk_nspec[cc];
        C* base = ring + (size_t)st * stage_elems;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&bars[st], (uint32_t)nb * blk_bytes);
        for (int b = 0; b < nb; ++b) {
            const int id = DEFMM_IX(c, c.chk_blk[b0 + b], b < nsp ? c.n_spec : c.n_m2f);
            const C* src = b < nsp ? t.spec + (int64_t)id * NFpad : Mhat + ((int64_t)id * R + r) * NFpad;
            tma_bulk_load(base + (size_t)b * NFpad, src, blk_bytes, &bars[st]);
        }
    };
    for (int r = 0; r < R; ++r) {
        if (threadIdx.x == 0)
            for (int k = 0; k < S - 1 && k < nchunks; ++k) issue(k, r, (use + k) % S);
        C acc[8][VPT];
#pragma unroll
        for (int m = 0; m < 8; ++m)
#pragma unroll
            for (int v = 0; v < VPT; ++v) acc[m][v] = czero<C>();
        for (int ch = 0; ch < nchunks; ++ch, ++use) {
            const int st = use % S;
            const bool ok = mbar_wait(&bars[st], (use / S) & 1);
            // one barrier per chunk: every thread has finished the previous chunk
            // (so its stage may be refilled) and the decision to stop is uniform
            if (__syncthreads_or(!ok)) {
                if (threadIdx.x == 0) {
                    atomicExch(c.err_flag, 1);
                    // give copies already issued a bounded chance to land before the block exits
                    const int last = min(nchunks - 1, ch + S - 2);
                    for (int k = ch; k <= last; ++k)
                        (void)mbar_wait(&bars[(use + k - ch) % S], ((use + k - ch) / S) & 1);
                }
                return;
            }
            if (threadIdx.x == 0 && ch + S - 1 < nchunks) issue(ch + S - 1, r, (use + S - 1) % S);
            const C* base = ring + (size_t)st * stage_elems;
            const int* opoff = c.chk_op_off + 9 * (ch0 + ch);
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                const int o1 = opoff[m + 1];
                for (int o = opoff[m]; o < o1; ++o) {
                    const int op = c.chk_op[o];
                    const int code = op >> 16, pid = code >> 3;
                    const int s0 = stride[pid][0], s1 = stride[pid][1], s2 = stride[pid][2];
                    const C* gs = base + (size_t)(op & 255) * NFpad;
                    const C* ms = base + (size_t)((op >> 8) & 255) * NFpad;
#pragma unroll
                    for (int v = 0; v < VPT; ++v) {
                        if (xi[v] < NF) {
                            const int idx = ((code & 1) ? cn[v][0] : cp[v][0]) * s0 +
                                            ((code & 2) ? cn[v][1] : cp[v][1]) * s1 +
                                            ((code & 4) ? cn[v][2] : cp[v][2]) * s2;
                            cfma(acc[m][v], gs[idx], ms[xi[v]]);
                        }
                    }
                }
            }
        }
        __syncthreads();   // every chunk read: the ring may now hold the F2L arrays
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            if (m >= nm) break;
#pragma unroll
            for (int v = 0; v < VPT; ++v)
                if (xi[v] < NF) Lh[xi[v]] = acc[m][v];
            __syncthreads();
            for (int q = threadIdx.x; q < p * N * N; q += blockDim.x) {  // z
                const int xy = q % (N * N), az = q / (N * N);
                C s = czero<C>();
                for (int k = 0; k < N; ++k) cfma(s, Lh[k * N * N + xy], tws[(k * az) % N]);
                T1[q] = s;
            }
            __syncthreads();
            for (int q = threadIdx.x; q < p * p * N; q += blockDim.x) {  // y
                const int xx = q % N, ay = (q / N) % p, az = q / (N * p);
                C s = czero<C>();
                for (int k = 0; k < N; ++k) cfma(s, T1[(az * N + k) * N + xx], tws[(k * ay) % N]);
                T2[q] = s;
            }
            __syncthreads();
            const int te = DEFMM_IX(c, c.grp_members[mem0 + m], c.n_local);
            for (int a = threadIdx.x; a < P3; a += blockDim.x) {  // x, crop, 1/N^3
                const int ax = a % p, rest = a / p;  // rest = az*p + ay
                C s = czero<C>();
                for (int k = 0; k < N; ++k) cfma(s, T2[rest * N + k], tws[(k * ax) % N]);
                L[((int64_t)te * R + r) * P3 + a] = cscale(s, scale);
            }
            __syncthreads();   // Lh, T1, T2 reused by the next member / the next prologue
        }
    }
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// The same group schedule with rows of samples and a warp-specialised
// pipeline.  A block takes the members of a group (at most MAXM: 8, 7 or 4;
// the group list of the launch, c.sh_grp, picks the groups) or, with MAXM =
// 4, one half of a larger group (its own pass over the group's chunks, using
// the ops of its members only).  Consumer thread (member m, lane l) of
// the first MAXM*TPM threads owns the x-rows l + j*TPM (j < ROWS) of member m; row (y, z) = (l mod N,
// l div N) holds the N samples xi = x + N*row.  Under a pair's symmetry
// (sigma, s) a row's permuted indices are base(y, z) + x*step (with a wrap
// for a negated x), so the permutation costs one row base per pair.  RB
// right-hand sides share a pass: a stage holds the chunk's spectra once and
// RB consecutive right-hand sides of each source multipole (contiguous in
// Mhat), so every gathered spectrum sample serves RB products.  The last warp
// is the producer: it keeps every stage of the ring loaded with TMA bulk
// copies, waiting on per-stage "empty" mbarriers that the consumer warps
// arrive on after reading a stage; consumers wait on per-stage "full"
// mbarriers that the copies complete.  There is no block-wide barrier in the
// main loop.  Every wait is bounded; a wait that gives up raises the plan's
// error flag and the block stops after its copies in flight have had a
// bounded chance to land.  F2L: each thread first takes the inverse DFT of
// its rows along x in registers (p outputs per row), then the y and z passes
// run in shared memory.  Needs N <= NX and N^2 <= ROWS*TPM.
template <typename T, int NX, int TPM, int ROWS, int RB, int MINB, int PC = 0, int NC = 0, int MAXM = 8>
__global__ void __launch_bounds__(MAXM * TPM + 32, MINB) k_m2l_rows(DevCommon c, DevTyped<T> t, const typename Cplx<T>::type* __restrict__ Mhat,
                                                                   typename Cplx<T>::type* __restrict__ L, int R, int S, int stage_elems) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int p = PC ? PC : c.p, N = NC ? NC : c.N, NFpad = c.NFpad, P3 = p * p * p;
    const int NN = N * N;
    const uint32_t blk_bytes = (uint32_t)(NFpad * sizeof(C));
    C* ring = reinterpret_cast<C*>(smem_raw);
    __shared__ __align__(8) uint64_t full[kM2LMaxStages], empty[kM2LMaxStages];
    __shared__ C tws[16];
    __shared__ int stride[6][3];
    __shared__ int abort_store, issued_sh, abort_at;
    volatile int& abort_sh = abort_store;   // written and polled by different warps
    int g = blockIdx.x, mb = 0;                  // group (of the shard), first member of this block
    if (MAXM == 4) {                             // grp_half holds the shard's half-groups when sharded
        const int code = c.grp_half[blockIdx.x];
        g = code >> 1;
        mb = 4 * (code & 1);
    } else if (c.sh_grp) {
        g = c.sh_grp[blockIdx.x];
    }
    const int mem0 = c.grp_member_off[g] + mb;
    const int nm = min(MAXM, c.grp_member_off[g + 1] - mem0);
    const int ch0 = c.grp_chunk_off[g], nchunks = c.grp_chunk_off[g + 1] - ch0;
    const bool producer = threadIdx.x >= MAXM * TPM;
    const int lane = threadIdx.x & 31;
    const int m = threadIdx.x / TPM, l = threadIdx.x % TPM;
    const bool member = !producer && m < nm;     // warp belongs to a member of the group
    int row[ROWS], yv[ROWS], zv[ROWS], yn[ROWS], zn[ROWS];
    bool act[ROWS];
#pragma unroll
    for (int j = 0; j < ROWS; ++j) {
        row[j] = l + j * TPM;
        act[j] = member && row[j] < NN;          // lane owns this row
        yv[j] = row[j] % N; zv[j] = row[j] / N;
        yn[j] = yv[j] == 0 ? 0 : N - yv[j];
        zn[j] = zv[j] == 0 ? 0 : N - zv[j];
    }
    const int consumer_warps = nm * (TPM / 32);
    if (threadIdx.x < N) tws[threadIdx.x] = t.tw[threadIdx.x];
    if (threadIdx.x < 18) {
        const int q = kPermDev[threadIdx.x / 3][threadIdx.x % 3];
        stride[threadIdx.x / 3][threadIdx.x % 3] = q == 0 ? 1 : (q == 1 ? N : N * N);
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], consumer_warps);
        }
        abort_sh = 0;
        issued_sh = 0;
        abort_at = 1 << 30;
        mbar_fence_init();
    }
    __syncthreads();
    uint32_t use0 = 0;   // chunks of earlier passes
    const T scale = (T)1 / (T)(N * NN);
    for (int r0 = 0; r0 < R; r0 += RB) {
        const int nrb = R - r0 < RB ? R - r0 : RB;   // right-hand sides in this pass
        C acc[ROWS][RB][NX];
#pragma unroll
        for (int j = 0; j < ROWS; ++j)
#pragma unroll
            for (int rr = 0; rr < RB; ++rr)
#pragma unroll
                for (int x = 0; x < NX; ++x) acc[j][rr][x] = czero<C>();
        if (producer) {
            // The whole warp feeds the ring: lane 9 holds a chunk's spectrum count and
            // lanes 10-11 its block range (loaded two chunks ahead), lane b the id of
            // its block b (loaded one chunk ahead, in parallel across the lanes); each
            // lane issues the bulk copies of its blocks after lane 0 has armed the
            // stage's mbarrier (whose phase then completes only when every block has
            // landed), so no global load latency sits between two chunks' copies.
            auto scalars = [&](int cc) -> int {
                if (lane == 9) return __ldg(&c.chk_nspec[cc]);
                if (lane == 10 || lane == 11) return __ldg(&c.chk_blk_off[cc + lane - 10]);
                return 0;
            };
            // block id of lane b of the chunk with scalars sc (b < 32)
            auto first_ids = [&](int sc) -> int {
                const int b0 = __shfl_sync(0xffffffffu, sc, 10), nb = __shfl_sync(0xffffffffu, sc, 11) - b0;
                return lane < nb ? __ldg(&c.chk_blk[b0 + lane]) : 0;
            };
            int sc_next = nchunks > 0 ? scalars(ch0) : 0;
            for (int k = 0; k < nchunks; ++k) {
                const int sc = sc_next;
                if (k + 1 < nchunks) sc_next = scalars(ch0 + k + 1);   // in flight during this chunk
                const int ids = first_ids(sc);
                const uint32_t u = use0 + k;
                const int st = u % S;
                int go = 1;
                if (lane == 0) {
                    if (u >= (uint32_t)S && !mbar_wait(&empty[st], ((u / S) - 1) & 1)) {
                        abort_sh = 1;
                        atomicExch(c.err_flag, 1);
                        go = 0;
                    }
                    if (abort_sh) go = 0;
                }
                if (!__shfl_sync(0xffffffffu, go, 0)) break;
                const int nsp = __shfl_sync(0xffffffffu, sc, 9), b0 = __shfl_sync(0xffffffffu, sc, 10);
                const int nb = __shfl_sync(0xffffffffu, sc, 11) - b0;
                if (lane == 0) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    mbar_expect_tx(&full[st], (uint32_t)(nsp + (nb - nsp) * nrb) * blk_bytes);
                }
                __syncwarp();
                C* base = ring + (size_t)st * stage_elems;
                for (int b = lane; b < nb; b += 32) {
                    const int id = DEFMM_IX(c, b < 32 ? ids : __ldg(&c.chk_blk[b0 + b]), b < nsp ? c.n_spec : c.n_m2f);
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    if (b < nsp)
                        tma_bulk_load(base + (size_t)b * NFpad, t.spec + (int64_t)id * NFpad, blk_bytes, &full[st]);
                    else   // right-hand sides r0 .. r0+nrb-1 of one source: one contiguous copy
                        tma_bulk_load(base + (size_t)(nsp + (b - nsp) * RB) * NFpad,
                                      Mhat + ((int64_t)id * R + r0) * NFpad, (uint32_t)nrb * blk_bytes, &full[st]);
                }
                if (lane == 0) issued_sh = k + 1;
            }
        } else if (member) {
            for (int k = 0; k < nchunks; ++k) {
                const uint32_t u = use0 + k;
                const int st = u % S;
                if (!mbar_wait(&full[st], (u / S) & 1) || abort_sh) {
                    abort_sh = 1;
                    atomicMin(&abort_at, k);
                    atomicExch(c.err_flag, 1);
                    break;
                }
                if (act[0]) {
                    const C* base = ring + (size_t)st * stage_elems;
                    const int* opoff = c.chk_op_off + 9 * (ch0 + k);
                    const int o0 = opoff[mb + m], o1 = opoff[mb + m + 1];
                    const int msh = RB == 1 ? 0 : (RB - 1) * __ldg(&c.chk_nspec[ch0 + k]);
                    int op_next = o0 < o1 ? __ldg(&c.chk_op[o0]) : 0;
                    for (int o = o0; o < o1; ++o) {
                        const int op = op_next;
                        if (o + 1 < o1) op_next = __ldg(&c.chk_op[o + 1]);   // in flight during this pair
                        const int code = op >> 16, pid = code >> 3;
                        const int s0 = stride[pid][0], s1 = stride[pid][1], s2 = stride[pid][2];
                        const C* gs = base + (size_t)(op & 255) * NFpad;
                        // source block b sits at nsp + (b - nsp) * RB blocks
                        const C* msrc = base + (size_t)(((op >> 8) & 255) * RB - msh) * NFpad;
                        const int xneg = code & 1;
                        const int dx = xneg ? -s0 : s0;
#pragma unroll
                        for (int j = 0; j < ROWS; ++j) {
                            if (j == 0 || act[j]) {
                                // permuted index of sample (x, y, z): f0(x) s0 + f1(y) s1 + f2(z) s2
                                const int rowb = ((code & 2) ? yn[j] : yv[j]) * s1 + ((code & 4) ? zn[j] : zv[j]) * s2;
                                const int b1 = xneg ? rowb + N * s0 : rowb;   // x >= 1: b1 + x * dx
                                const C* ms = msrc + (size_t)row[j] * N;
                                const C g0 = gs[rowb];
#pragma unroll
                                for (int rr = 0; rr < RB; ++rr) cfma(acc[j][rr][0], g0, ms[(size_t)rr * NFpad]);
#pragma unroll
                                for (int x = 1; x < NX; ++x)
                                    if (x < N) {
                                        const C gx = gs[b1 + x * dx];
#pragma unroll
                                        for (int rr = 0; rr < RB; ++rr) cfma(acc[j][rr][x], gx, ms[(size_t)rr * NFpad + x]);
                                    }
                            }
                        }
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[st]);
            }
        }
        __syncthreads();   // every chunk of this pass consumed (or the block gave up)
        if (abort_sh) {
            if (threadIdx.x == 0) {   // bounded drain of copies issued but never waited for
                const int first = abort_at < nchunks ? abort_at : 0;
                for (int k = first; k < issued_sh; ++k)
                    (void)mbar_wait(&full[(use0 + k) % S], ((use0 + k) / S) & 1);
            }
            __syncthreads();
            return;
        }
        use0 += nchunks;
        // F2L of every member in parallel, one right-hand side at a time; member
        // m uses its own arrays (aliasing the drained ring) and its TPM threads
        C* Tx = ring + (size_t)(member ? m : 0) * (NN * p + N * p * p);   // [z][y][ax]
        C* Ty = Tx + NN * p;                                               // [z][ay][ax]
        const int te = member ? DEFMM_IX(c, c.grp_members[mem0 + m], c.n_local) : 0;
#pragma unroll
        for (int rr = 0; rr < RB; ++rr) {
            if (rr >= nrb) break;
#pragma unroll
            for (int j = 0; j < ROWS; ++j)
                if (act[j])   // x: p outputs of the row, in registers
                    for (int ax = 0; ax < p; ++ax) {
                        C s = acc[j][rr][0];
#pragma unroll
                        for (int x = 1; x < NX; ++x)
                            if (x < N) cfma(s, acc[j][rr][x], tws[(x * ax) % N]);
                        Tx[row[j] * p + ax] = s;
                    }
            __syncthreads();
            if (member)
                for (int q = l; q < N * p * p; q += TPM) {  // y
                    const int ax = q % p, ay = (q / p) % p, zz = q / (p * p);
                    C s = czero<C>();
                    for (int k = 0, w = 0; k < N; ++k) {   // w = k * ay mod N
                        cfma(s, Tx[(zz * N + k) * p + ax], tws[w]);
                        w += ay;
                        w -= w >= N ? N : 0;
                    }
                    Ty[q] = s;
                }
            __syncthreads();
            if (member)
                for (int a = l; a < P3; a += TPM) {  // z, crop, 1/N^3
                    const int ax = a % p, ay = (a / p) % p, az = a / (p * p);
                    C s = czero<C>();
                    for (int k = 0, w = 0; k < N; ++k) {   // w = k * az mod N
                        cfma(s, Ty[(k * p + ay) * p + ax], tws[w]);
                        w += az;
                        w -= w >= N ? N : 0;
                    }
                    L[((int64_t)te * R + r0 + rr) * P3 + a] = cscale(s, scale);
                }
            __syncthreads();   // Tx, Ty reused by the next right-hand side / the next pass's ring
        }
    }
}

// Ring depth S and the dynamic shared memory of the per-sample M2L kernel:
// three stages of the largest chunk when they fit, else two; the F2L arrays of
// one member reuse the same memory.
template <typename T> __host__ void m2l_shape(const DevCommon& c, int* S, size_t* smem) {
    const size_t stage = (size_t)c.chk_stage_blocks[0] * c.NFpad * sizeof(typename Cplx<T>::type);
    int ss = kM2LMaxStages;
    while (ss > 2 && (size_t)ss * stage > kSmemLimit) --ss;
    const size_t ring = (size_t)ss * stage;
    const size_t f2l = ((size_t)c.NF + (size_t)c.p * c.N * c.N + (size_t)c.p * c.p * c.N) *
                       sizeof(typename Cplx<T>::type);
    *S = ss;
    *smem = ring > f2l ? ring : f2l;
}

// Shape of a row-kernel launch with RB right-hand sides per pass: the stage
// (in elements), the ring depth S (three stages if they fit in the shared
// memory one block may use at the wanted residency, else two) and the dynamic
// shared memory (ring, or the F2L arrays of `members` members if larger).
// Returns false if two stages or the F2L arrays do not fit in one block.
template <typename T> __host__ bool m2l_rows_shape(const DevCommon& c, int RB, int blocks_per_sm, int members, int* S,
                                                   int* stage_elems, size_t* smem) {
    const int v = RB == 1 ? 0 : (RB == 2 ? 1 : 2);
    const size_t esz = sizeof(typename Cplx<T>::type);
    *stage_elems = c.chk_stage_blocks[v] * c.NFpad;
    const size_t stage = (size_t)*stage_elems * esz;
    size_t budget = (228 * 1024) / (size_t)(blocks_per_sm < 1 ? 1 : blocks_per_sm) - 1024 - 2048;
    if (budget > kSmemLimit) budget = kSmemLimit;
    const size_t f2l = (size_t)members * ((size_t)c.N * c.N * c.p + (size_t)c.N * c.p * c.p) * esz;
    int ss = kM2LMaxStages;
    while (ss > 2 && (size_t)ss * stage > budget) --ss;
    const size_t ring = (size_t)ss * stage;
    *S = ss;
    *smem = ring > f2l ? ring : f2l;
    return *smem <= kSmemLimit;
}
// ------------------------------------------------------------------ L2L
// One warp per (son expansion, right-hand side) (entry: son id, octant, first, count into the
// list of father expansions feeding it), the transpose of M2M:
//   L_son[b] += sum_fathers Q_v,o(b) sum_a T_o[a, b] conj(P_v(a)) L_v[a].
template <typename T, int PC = 0>
__global__ void __launch_bounds__(256) k_l2l(DevCommon c, DevTyped<T> t, const int32_t* __restrict__ list, int64_t n,
                                             const int32_t* __restrict__ par, typename Cplx<T>::type* __restrict__ L, int R) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int p = PC ? PC : c.p, P3 = p * p * p;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __shared__ T m1s[2 * 8 * 8];
    for (int i = threadIdx.x; i < 2 * p * p; i += blockDim.x) m1s[i] = t.m1[i];
    __syncthreads();
    const int64_t wid = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;   // (item, right-hand side)
    const int64_t item = wid / R;
    const int rr = (int)(wid % R);
    if (item >= n) return;
    C* A = reinterpret_cast<C*>(smem_raw) + (size_t)warp * (2 * P3 + 72);
    C* B = A + P3;
    C* Ps = B + P3;          // [3][p]
    C* Qs = Ps + 24;         // [3][2][p]
    const int32_t* ent = list + 4 * item;
    const int ec = DEFMM_IX(c, ent[0], c.n_local), o = ent[1], first = ent[2], cnt = ent[3];
    const int ox = o & 1, oy = (o >> 1) & 1, oz = (o >> 2) & 1;
    const T* mx = m1s + ox * p * p;
    const T* my = m1s + oy * p * p;
    const T* mz = m1s + oz * p * p;
    {   // this warp's right-hand side
        const int r = rr;
        C acc[16];
#pragma unroll
        for (int v = 0; v < 16; ++v) acc[v] = czero<C>();
        for (int k = 0; k < cnt; ++k) {
            const int pe = DEFMM_IX(c, par[first + k], c.n_local);
            const int slot = DEFMM_IX(c, c.l_slot[pe] + 1, c.n_slot + 1) - 1;
            __syncwarp();
            for (int i = lane; i < 3 * p; i += 32) Ps[i] = slot >= 0 ? t.slot_P[(int64_t)slot * 3 * p + i] : mk((T)1, (T)0);
            for (int i = lane; i < 6 * p; i += 32) Qs[i] = slot >= 0 ? t.slot_Q[(int64_t)slot * 6 * p + i] : mk((T)1, (T)0);
            __syncwarp();
            for (int a = lane; a < P3; a += 32) {
                const int a0 = a % p, a1 = (a / p) % p, a2 = a / (p * p);
                const C ph = cmul(cmul(Ps[a0], Ps[p + a1]), Ps[2 * p + a2]);
                A[a] = cmulc(L[((int64_t)pe * R + r) * P3 + a], ph);
            }
            __syncwarp();
            for (int b = lane; b < P3; b += 32) {  // x: (az, ay, bx)
                const int b0 = b % p, rest = b - b0;
                C s = czero<C>();
                for (int q = 0; q < p; ++q) { C v = A[rest + q]; T m = mx[q * p + b0]; s.x += m * v.x; s.y += m * v.y; }
                B[b] = s;
            }
            __syncwarp();
            for (int b = lane; b < P3; b += 32) {  // y: (az, by, bx)
                const int b0 = b % p, b1 = (b / p) % p, b2 = b / (p * p);
                C s = czero<C>();
                for (int q = 0; q < p; ++q) { C v = B[(b2 * p + q) * p + b0]; T m = my[q * p + b1]; s.x += m * v.x; s.y += m * v.y; }
                A[b] = s;
            }
            __syncwarp();
#pragma unroll
            for (int v = 0; v < 16; ++v) {  // z: (bz, by, bx), times Q(v, o)
                const int b = lane + v * 32;
                if (b < P3) {
                    const int b0 = b % p, b1 = (b / p) % p, b01 = b % (p * p), b2 = b / (p * p);
                    C s = czero<C>();
                    for (int q = 0; q < p; ++q) { C w = A[q * p * p + b01]; T m = mz[q * p + b2]; s.x += m * w.x; s.y += m * w.y; }
                    const C qq = cmul(cmul(Qs[(0 * 2 + ox) * p + b0], Qs[(1 * 2 + oy) * p + b1]), Qs[(2 * 2 + oz) * p + b2]);
                    cfma(acc[v], s, qq);
                }
            }
        }
#pragma unroll
        for (int v = 0; v < 16; ++v) {
            const int b = lane + v * 32;
            if (b < P3) {
                C* dst = L + ((int64_t)ec * R + r) * P3 + b;
                *dst = cadd(*dst, acc[v]);
            }
        }
    }
}

// ------------------------------------------------------------------ L2P
// p(x) += sum_u E_u(x) sum_a S_a(x_hat) conj(P_u(a)) L_u[a], E_u(x) = exp(i kappa <x - c, u>):
// the leaf's expansions are pre-scaled by conj(P_u) into shared memory, each
// (particle, expansion) then costs one phase and a real-basis contraction.
// The leaf's n_t targets are spread over 128 threads as targets x
// expansion-splits; partial sums are reduced over the splits in order.
template <typename T, int RB, int PC = 0>
__global__ void __launch_bounds__(128) k_l2p(DevCommon c, DevTyped<T> t, const typename Cplx<T>::type* __restrict__ L,
                                             typename Cplx<T>::type* __restrict__ ps, int R, int rb0, int epass) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* Ls = reinterpret_cast<C*>(smem_raw);            // [RB][epass][P3]
    C* red = Ls + (size_t)RB * epass * c.P3;            // [RB][128]
    const int cell = DEFMM_IX(c, c.l2p_cells[blockIdx.x], c.n_cell_t);
    const int b = c.ct_beg[cell], e = c.ct_end[cell];
    const double side = c.level_side[c.ct_level[cell]];
    const int p = PC ? PC : c.p, P3 = p * p * p;
    const double h = side / (p - 1);
    const double cor[3] = {c.ct_corner[3 * cell], c.ct_corner[3 * cell + 1], c.ct_corner[3 * cell + 2]};
    const int nr = min(RB, R - rb0);
    const T k2pi = (T)(kappa_of(c, cell) * kInv2Pi);
    const int ex0 = DEFMM_IX(c, c.l_first[cell], c.n_local + 1), nex = DEFMM_IX(c, c.l_count[cell], c.n_local - ex0 + 1);
    for (int t0 = b; t0 < e; t0 += 128) {
        const int nt = min(128, e - t0);
        const int splits = 128 / nt;
        const int ti = threadIdx.x % nt, sj = threadIdx.x / nt;
        const bool active = sj < splits;
        const int j = t0 + ti;
        T lag[3][8], dc[3];
        for (int ax = 0; ax < 3; ++ax) {
            const double d = active ? c.Xs[3 * (int64_t)j + ax] - cor[ax] : 0.0;
            dc[ax] = (T)(d - 0.5 * side);
            for (int m = 0; m < p; ++m) lag[ax][m] = lagrange<T>(p, m, (T)(d / h));
        }
        C acc[RB];
#pragma unroll
        for (int r = 0; r < RB; ++r) acc[r] = czero<C>();
        for (int e0 = 0; e0 < nex; e0 += epass) {
            const int ne = min(epass, nex - e0);
            __syncthreads();
            for (int i = threadIdx.x; i < nr * ne * P3; i += blockDim.x) {
                const int r = i / (ne * P3), rem = i - r * ne * P3, ee = rem / P3, a = rem - ee * P3;
                const int ex = ex0 + e0 + ee;
                const int slot = DEFMM_IX(c, c.l_slot[ex] + 1, c.n_slot + 1) - 1;
                C v = L[((int64_t)ex * R + rb0 + r) * P3 + a];
                if (slot >= 0) {
                    const int a0 = a % p, a1 = (a / p) % p, a2 = a / (p * p);
                    const C* P = t.slot_P + (int64_t)slot * 3 * p;
                    v = cmulc(v, cmul(cmul(P[a0], P[p + a1]), P[2 * p + a2]));
                }
                Ls[((size_t)r * epass + ee) * P3 + a] = v;
            }
            __syncthreads();
            if (active) {
                for (int ee = sj; ee < ne; ee += splits) {
                    const int slot = DEFMM_IX(c, c.l_slot[ex0 + e0 + ee] + 1, c.n_slot + 1) - 1;
                    C E = mk((T)1, (T)0);
                    if (slot >= 0) {
                        const T arg = dc[0] * (T)c.slot_u[3 * slot] + dc[1] * (T)c.slot_u[3 * slot + 1] +
                                      dc[2] * (T)c.slot_u[3 * slot + 2];
                        T sn, cs;
                        turns_sincos(arg * k2pi, &sn, &cs);
                        E = mk(cs, sn);
                    }
                    for (int r = 0; r < nr; ++r) {
                        const C* Lr = Ls + ((size_t)r * epass + ee) * P3;
                        C sz = czero<C>();
                        for (int a2 = 0; a2 < p; ++a2) {
                            C sy = czero<C>();
                            for (int a1 = 0; a1 < p; ++a1) {
                                C sx = czero<C>();
                                const C* row = Lr + (a2 * p + a1) * p;
                                for (int a0 = 0; a0 < p; ++a0) {
                                    sx.x = fma(lag[0][a0], row[a0].x, sx.x);
                                    sx.y = fma(lag[0][a0], row[a0].y, sx.y);
                                }
                                sy.x = fma(lag[1][a1], sx.x, sy.x);
                                sy.y = fma(lag[1][a1], sx.y, sy.y);
                            }
                            sz.x = fma(lag[2][a2], sy.x, sz.x);
                            sz.y = fma(lag[2][a2], sy.y, sz.y);
                        }
                        cfma(acc[r], E, sz);
                    }
                }
            }
        }
#pragma unroll
        for (int r = 0; r < RB; ++r) red[r * 128 + threadIdx.x] = acc[r];
        __syncthreads();
        if (active && sj == 0)
            for (int r = 0; r < nr; ++r) {
                C s = red[r * 128 + ti];
                for (int q = 1; q < splits; ++q) s = cadd(s, red[r * 128 + ti + q * nt]);
                C* dst = ps + (int64_t)(rb0 + r) * c.nx + j;
                *dst = cadd(*dst, s);
            }
        __syncthreads();
    }
}

// Expansions per pass of k_l2p: at most 96 KB of pre-scaled local expansions.
__host__ int l2p_epass(int P3, int RB, size_t ccplx) {
    const int by_smem = (int)((96 * 1024) / ((size_t)RB * P3 * ccplx));
    int ep = kMaxExp < by_smem ? kMaxExp : by_smem;
    return ep < 1 ? 1 : ep;
}
__host__ size_t l2p_smem(int P3, int RB, int epass, size_t ccplx) {
    return ((size_t)RB * epass * P3 + (size_t)RB * 128) * ccplx;
}

// ------------------------------------------------------------------ P2M / L2P, one warp per leaf
// Leaves are small (tens of particles, mostly one expansion), so for orders
// known at compile time a warp, not a block, handles a leaf; blocks hold four
// independent warps synchronised with __syncwarp only.
constexpr int kLeafWarps = 4;
__host__ __device__ constexpr int p2m_items_per_lane(int RB) { return RB == 1 ? 4 : 1; }
__host__ int p2m_warp_epass(int p, int RB) {
    const int ep = p2m_items_per_lane(RB) * 32 / (p * p);
    return ep < 1 ? 1 : ep;
}
__host__ size_t p2m_warp_smem(int p, int RB, int epass, size_t creal) {
    return kLeafWarps * ((((size_t)32 * 3 * p * creal + 15) / 16) * 16 + (size_t)RB * epass * 32 * 2 * creal);
}

// P2M (Sec. 2.2) with the separated plane wave of k_p2m.  Lanes own items
// (expansion, a1, a2) of PC outputs along a0; per particle a lane reads the PC
// x-factors once and w = l_a1(y) l_a2(z) q conj(E_u(y)).  A leaf with a
// single expansion of at most 16 lines splits its particles between the
// half-warps (even / odd) and adds the two partial sums, lower half first;
// the rule depends on the leaf only, so a column's summation order does not
// depend on how many right-hand sides are blocked together.
template <typename T, int RB, int PC>
__global__ void __launch_bounds__(32 * kLeafWarps) k_p2m_warp(DevCommon c, DevTyped<T> t,
                                                              const typename Cplx<T>::type* __restrict__ qs,
                                                              typename Cplx<T>::type* __restrict__ M, int R, int rb0,
                                                              int epass) {
    using C = typename Cplx<T>::type;
    constexpr int P2 = PC * PC, P3 = P2 * PC, V = p2m_items_per_lane(RB), LW = 3 * PC;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int li = blockIdx.x * kLeafWarps + warp;
    if (li >= c.n_p2m) return;
    const size_t lag_bytes = (((size_t)32 * LW * sizeof(T) + 15) / 16) * 16;
    unsigned char* base = smem_raw + (size_t)warp * (lag_bytes + (size_t)RB * epass * 32 * sizeof(C));
    T* lag = reinterpret_cast<T*>(base);                 // [32][3][PC]
    C* qm = reinterpret_cast<C*>(base + lag_bytes);      // [RB][epass][32]
    const int cell = DEFMM_IX(c, c.p2m_cells[li], c.n_cell_s);
    const int b = c.cs_beg[cell], e = c.cs_end[cell];
    const double side = c.level_side[c.cs_level[cell]];
    const double h = side / (PC - 1);
    const double cx = c.cs_corner[3 * cell], cy = c.cs_corner[3 * cell + 1], cz = c.cs_corner[3 * cell + 2];
    const int nr = min(RB, R - rb0);
    const T k2pi = (T)(kappa_of(c, cell) * kInv2Pi);
    const int ex0 = DEFMM_IX(c, c.m_first[cell], c.n_mult + 1), nex = DEFMM_IX(c, c.m_count[cell], c.n_mult - ex0 + 1);
    for (int e0 = 0; e0 < nex; e0 += epass) {
        const int ne = min(epass, nex - e0);
        const int nitems = ne * P2;
        const int split = (nex == 1 && P2 <= 16) ? 2 : 1;   // depends on the leaf only, not on RB
        const int il = split == 2 ? (lane & 15) : lane, js = split == 2 ? (lane >> 4) : 0;
        const int stride = 32 / split;
        int yo[V], zo[V], qo[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int it = min(il + v * stride, nitems - 1);
            const int ee = it / P2, rem = it - ee * P2;
            yo[v] = PC + rem % PC;
            zo[v] = 2 * PC + rem / PC;
            qo[v] = ee * 32;
        }
        C acc[V][PC][RB];
#pragma unroll
        for (int v = 0; v < V; ++v)
#pragma unroll
            for (int a0 = 0; a0 < PC; ++a0)
#pragma unroll
                for (int r = 0; r < RB; ++r) acc[v][a0][r] = czero<C>();
        for (int j0 = b; j0 < e; j0 += 32) {
            const int nj = min(32, e - j0);
            __syncwarp();
            if (lane < nj) {
                const int64_t j = j0 + lane;
                const double d0 = c.Ys[3 * j] - cx, d1 = c.Ys[3 * j + 1] - cy, d2 = c.Ys[3 * j + 2] - cz;
                const T s0 = (T)(d0 / h), s1 = (T)(d1 / h), s2 = (T)(d2 / h);
#pragma unroll
                for (int m = 0; m < PC; ++m) {
                    lag[lane * LW + m] = lagrange<T>(PC, m, s0);
                    lag[lane * LW + PC + m] = lagrange<T>(PC, m, s1);
                    lag[lane * LW + 2 * PC + m] = lagrange<T>(PC, m, s2);
                }
                const T x0 = (T)(d0 - 0.5 * side), x1 = (T)(d1 - 0.5 * side), x2 = (T)(d2 - 0.5 * side);
                C q[RB];
#pragma unroll
                for (int r = 0; r < RB; ++r) q[r] = r < nr ? qs[(int64_t)(rb0 + r) * c.ny + j] : czero<C>();
                for (int ee = 0; ee < ne; ++ee) {
                    const int slot = DEFMM_IX(c, c.m_slot[ex0 + e0 + ee] + 1, c.n_slot + 1) - 1;
                    C ph = mk((T)1, (T)0);
                    if (slot >= 0) {
                        const T arg = x0 * (T)c.slot_u[3 * slot] + x1 * (T)c.slot_u[3 * slot + 1] +
                                      x2 * (T)c.slot_u[3 * slot + 2];
                        T sn, cs;
                        turns_sincos(arg * k2pi, &sn, &cs);
                        ph = mk(cs, -sn);                              // conj(E_u(y))
                    }
#pragma unroll
                    for (int r = 0; r < RB; ++r) qm[((size_t)r * epass + ee) * 32 + lane] = cmul(q[r], ph);
                }
            }
            __syncwarp();
            for (int j = js; j < nj; j += split) {
                const T* lj = lag + j * LW;
                T lx[PC];
                ld_vec<PC>(lj, lx);
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    if (il + v * stride < nitems) {
                        const T w = lj[yo[v]] * lj[zo[v]];
#pragma unroll
                        for (int r = 0; r < RB; ++r) {
                            const C q = qm[(size_t)r * epass * 32 + qo[v] + j];
                            const T wx = w * q.x, wy = w * q.y;
#pragma unroll
                            for (int a0 = 0; a0 < PC; ++a0) {
                                acc[v][a0][r].x = fma(lx[a0], wx, acc[v][a0][r].x);
                                acc[v][a0][r].y = fma(lx[a0], wy, acc[v][a0][r].y);
                            }
                        }
                    }
                }
            }
        }
        if (split == 2) {
#pragma unroll
            for (int a0 = 0; a0 < PC; ++a0)
#pragma unroll
                for (int r = 0; r < RB; ++r) {
                    acc[0][a0][r].x += __shfl_down_sync(0xffffffffu, acc[0][a0][r].x, 16);
                    acc[0][a0][r].y += __shfl_down_sync(0xffffffffu, acc[0][a0][r].y, 16);
                }
        }
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int it = il + v * stride;
            if (js == 0 && it < nitems) {
                const int ee = it / P2, rem = it - ee * P2;
                const int ex = ex0 + e0 + ee;
                const int slot = DEFMM_IX(c, c.m_slot[ex] + 1, c.n_slot + 1) - 1;
                const C* P = t.slot_P + (int64_t)(slot < 0 ? 0 : slot) * 3 * PC;
                const C p12 = slot >= 0 ? cmul(P[PC + rem % PC], P[2 * PC + rem / PC]) : mk((T)1, (T)0);
#pragma unroll
                for (int a0 = 0; a0 < PC; ++a0) {
                    const C ph = slot >= 0 ? cmul(P[a0], p12) : p12;
#pragma unroll
                    for (int r = 0; r < RB; ++r)
                        if (r < nr) M[((int64_t)ex * R + rb0 + r) * P3 + rem * PC + a0] = cmul(acc[v][a0][r], ph);
                }
            }
        }
    }
}

// L2P (Sec. 2.2): a lane per target; the leaf's expansions are staged epass at
// a time, pre-scaled by conj(P_u(a)), and each (target, expansion) costs one
// phase E_u(x) and a real-basis contraction over the staged rows.
__host__ int l2p_warp_epass(int P3, int RB, size_t ccplx) {
    const int ep = (int)(8192 / ((size_t)RB * P3 * ccplx));
    return ep < 1 ? 1 : (ep > 8 ? 8 : ep);
}
__host__ size_t l2p_warp_smem(int P3, int RB, int epass, size_t ccplx) {
    return kLeafWarps * (size_t)RB * epass * P3 * ccplx;
}

template <typename T, int RB, int PC>
__global__ void __launch_bounds__(32 * kLeafWarps) k_l2p_warp(DevCommon c, DevTyped<T> t,
                                                              const typename Cplx<T>::type* __restrict__ L,
                                                              typename Cplx<T>::type* __restrict__ ps, int R, int rb0,
                                                              int epass) {
    using C = typename Cplx<T>::type;
    constexpr int P3 = PC * PC * PC;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int li = blockIdx.x * kLeafWarps + warp;
    if (li >= c.n_l2p) return;
    C* Ls = reinterpret_cast<C*>(smem_raw) + (size_t)warp * RB * epass * P3;   // [epass][RB][P3]
    const int cell = DEFMM_IX(c, c.l2p_cells[li], c.n_cell_t);
    const int b = c.ct_beg[cell], e = c.ct_end[cell];
    const double side = c.level_side[c.ct_level[cell]];
    const double h = side / (PC - 1);
    const double cx = c.ct_corner[3 * cell], cy = c.ct_corner[3 * cell + 1], cz = c.ct_corner[3 * cell + 2];
    const int nr = min(RB, R - rb0);
    const T k2pi = (T)(kappa_of(c, cell) * kInv2Pi);
    const int ex0 = DEFMM_IX(c, c.l_first[cell], c.n_local + 1), nex = DEFMM_IX(c, c.l_count[cell], c.n_local - ex0 + 1);
    for (int t0 = b; t0 < e; t0 += 32) {
        const bool act = t0 + lane < e;
        const int64_t j = act ? t0 + lane : t0;
        const double d0 = c.Xs[3 * j] - cx, d1 = c.Xs[3 * j + 1] - cy, d2 = c.Xs[3 * j + 2] - cz;
        T lag[3][PC];
        {
            const T s0 = (T)(d0 / h), s1 = (T)(d1 / h), s2 = (T)(d2 / h);
#pragma unroll
            for (int m = 0; m < PC; ++m) {
                lag[0][m] = lagrange<T>(PC, m, s0);
                lag[1][m] = lagrange<T>(PC, m, s1);
                lag[2][m] = lagrange<T>(PC, m, s2);
            }
        }
        const T x0 = (T)(d0 - 0.5 * side), x1 = (T)(d1 - 0.5 * side), x2 = (T)(d2 - 0.5 * side);
        C acc[RB];
#pragma unroll
        for (int r = 0; r < RB; ++r) acc[r] = czero<C>();
        for (int e0 = 0; e0 < nex; e0 += epass) {
            const int ne = min(epass, nex - e0);
            __syncwarp();
            for (int i = lane; i < ne * nr * P3; i += 32) {
                const int ee = i / (nr * P3), rem = i - ee * nr * P3, r = rem / P3, a = rem - r * P3;
                const int ex = ex0 + e0 + ee;
                const int slot = DEFMM_IX(c, c.l_slot[ex] + 1, c.n_slot + 1) - 1;
                C v = L[((int64_t)ex * R + rb0 + r) * P3 + a];
                if (slot >= 0) {
                    const int a0 = a % PC, a1 = (a / PC) % PC, a2 = a / (PC * PC);
                    const C* P = t.slot_P + (int64_t)slot * 3 * PC;
                    v = cmulc(v, cmul(cmul(P[a0], P[PC + a1]), P[2 * PC + a2]));
                }
                Ls[((size_t)ee * RB + r) * P3 + a] = v;
            }
            __syncwarp();
            for (int ee = 0; ee < ne; ++ee) {
                const int slot = DEFMM_IX(c, c.l_slot[ex0 + e0 + ee] + 1, c.n_slot + 1) - 1;
                C E = mk((T)1, (T)0);
                if (slot >= 0) {
                    const T arg = x0 * (T)c.slot_u[3 * slot] + x1 * (T)c.slot_u[3 * slot + 1] + x2 * (T)c.slot_u[3 * slot + 2];
                    T sn, cs;
                    turns_sincos(arg * k2pi, &sn, &cs);
                    E = mk(cs, sn);
                }
#pragma unroll
                for (int r = 0; r < RB; ++r) {
                    if (r < nr) {
                        const C* Lr = Ls + ((size_t)ee * RB + r) * P3;
                        C sz = czero<C>();
#pragma unroll
                        for (int a2 = 0; a2 < PC; ++a2) {
                            C sy = czero<C>();
#pragma unroll
                            for (int a1 = 0; a1 < PC; ++a1) {
                                C lr[PC];
                                ld_vec<PC>(Lr + (a2 * PC + a1) * PC, lr);
                                C sx = czero<C>();
#pragma unroll
                                for (int a0 = 0; a0 < PC; ++a0) {
                                    sx.x = fma(lag[0][a0], lr[a0].x, sx.x);
                                    sx.y = fma(lag[0][a0], lr[a0].y, sx.y);
                                }
                                sy.x = fma(lag[1][a1], sx.x, sy.x);
                                sy.y = fma(lag[1][a1], sx.y, sy.y);
                            }
                            sz.x = fma(lag[2][a2], sy.x, sz.x);
                            sz.y = fma(lag[2][a2], sy.y, sz.y);
                        }
                        cfma(acc[r], E, sz);
                    }
                }
            }
        }
        if (act)
#pragma unroll
            for (int r = 0; r < RB; ++r)
                if (r < nr) {
                    C* dst = ps + (int64_t)(rb0 + r) * c.nx + j;
                    *dst = cadd(*dst, acc[r]);
                }
    }
}

// ------------------------------------------------------------------ spectra (float64)
// g(delta) = G(side*kbar + h*delta) placed at delta mod N, then an N^3 DFT
// with e^{-2 pi i xi.x / N} (unnormalised) along x, y and z.
__global__ void __launch_bounds__(256) k_spectra(const int32_t* __restrict__ spec_level, const int32_t* __restrict__ kbar,
                                                 const double* __restrict__ level_side, int p, int N, int NFpad,
                                                 double kappa0, const double* __restrict__ spec_kappa, double damping,
                                                 int power, double2* __restrict__ out_d, float2* __restrict__ out_f) {
    extern __shared__ unsigned char smem_raw[];
    const int NF = N * N * N;
    double2* A = reinterpret_cast<double2*>(smem_raw);
    double2* B = A + NF;
    __shared__ double2 tw[16];
    const int sid = blockIdx.x;
    const double side = level_side[spec_level[sid]];
    const double kappa = spec_kappa ? spec_kappa[sid] : kappa0;   // the spectrum's geometry
    const double h = side / (p - 1);
    const double k0 = kbar[3 * sid], k1 = kbar[3 * sid + 1], k2 = kbar[3 * sid + 2];
    if (threadIdx.x < N) {
        double s, c;
        sincospi(-2.0 * threadIdx.x / N, &s, &c);
        tw[threadIdx.x] = make_double2(c, s);
    }
    for (int i = threadIdx.x; i < NF; i += blockDim.x) A[i] = make_double2(0.0, 0.0);
    __syncthreads();
    const int W = 2 * p - 1;
    for (int i = threadIdx.x; i < W * W * W; i += blockDim.x) {
        const int dx = i % W - (p - 1), dy = (i / W) % W - (p - 1), dz = i / (W * W) - (p - 1);
        const double vx = side * k0 + h * dx, vy = side * k1 + h * dy, vz = side * k2 + h * dz;
        const double r = sqrt(vx * vx + vy * vy + vz * vz);
        double s, c;
        sincos(kappa * r, &s, &c);
        double g = kInv4Pi / r;
        if (power == 2) g /= r;
        if (damping > 0.0) g *= exp(-damping * r);
        const int ix = (dx + N) % N, iy = (dy + N) % N, iz = (dz + N) % N;
        A[(iz * N + iy) * N + ix] = make_double2(c * g, s * g);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < NF; i += blockDim.x) {  // x
        const int xx = i % N, rest = i - xx;
        double2 s = make_double2(0.0, 0.0);
        for (int k = 0; k < N; ++k) cfma(s, A[rest + k], tw[(xx * k) % N]);
        B[i] = s;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < NF; i += blockDim.x) {  // y
        const int xx = i % N, yy = (i / N) % N, zz = i / (N * N);
        double2 s = make_double2(0.0, 0.0);
        for (int k = 0; k < N; ++k) cfma(s, B[(zz * N + k) * N + xx], tw[(yy * k) % N]);
        A[i] = s;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < NFpad; i += blockDim.x) {  // z
        double2 s = make_double2(0.0, 0.0);
        if (i < NF) {
            const int xy = i % (N * N), zz = i / (N * N);
            for (int k = 0; k < N; ++k) cfma(s, A[k * N * N + xy], tw[(zz * k) % N]);
        }
        out_d[(int64_t)sid * NFpad + i] = s;
        out_f[(int64_t)sid * NFpad + i] = make_float2((float)s.x, (float)s.y);
    }
}

cudaError_t launch_spectra(const int32_t* spec_level, const int32_t* spec_kbar, int nspec,
                           const double* level_side, int p, int N, int NFpad, double kappa,
                           const double* spec_kappa, double damping, int power, double2* out_d, float2* out_f,
                           cudaStream_t stream) {
    if (nspec == 0) return cudaSuccess;
    size_t smem = 2 * (size_t)N * N * N * sizeof(double2);
    cudaError_t err = cudaFuncSetAttribute(k_spectra, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    k_spectra<<<nspec, 256, smem, stream>>>(spec_level, spec_kbar, level_side, p, N, NFpad, kappa, spec_kappa, damping,
                                            power, out_d, out_f);
    return cudaGetLastError();
}

// Tensor-core near field for many right-hand sides (complex64).  With R
// columns the near field of a work unit is the dense product
//   P[t, r] = sum_s G(x_t, y_s) Q[s, r],
// so per right-hand-side block of 32 columns one block computes it as a real
// GEMM on the tcgen05 tensor cores, M = 64 rows (Re and Im of 32 columns),
// N = the leaf's targets (a tile of <= 64, padded to a multiple of 8),
// K = 2 x (sources of a tile of 16):
//   D[(r, re), t] = sum_s Qr[s,r] Gr[t,s] - Qi[s,r] Gi[t,s],
//   D[(r, im), t] = sum_s Qi[s,r] Gr[t,s] + Qr[s,r] Gi[t,s],
// A = [[Qr, -Qi], [Qi, Qr]] interleaved per source (K index 2s + part),
// B[(s, part), t] = (Gr, Gi)[t, s].  The kernel values G are formed on the
// CUDA cores from the hi + lo coordinates of every pair with the reduced
// phase, once per interaction for all 32 columns.  Each operand is split into a tf32
// head and a tail (x = hi + lo, hi = tf32 rounding of x) and the three
// products lo*hi + hi*lo + hi*hi of a tile of 16 sources are summed in f32 in
// tensor memory (tf32 alone would leave ~1e-4 relative error).  The tensor
// cores' accumulation truncates, so its error grows with the number of MMAs
// summed into one accumulator: each tile therefore gets a fresh sum (12 MMAs)
// in one of two tensor-memory buffers, and the threads add finished tiles, in
// order, into f32 registers while the tensor cores work on the next tile.
// Operands live in shared memory as K-major core matrices without swizzle;
// two stages let the CUDA cores form the next tile while the tensor cores
// consume the previous one (completion tracked by tcgen05.commit on
// mbarriers).  Every wait is bounded; a wait that gives up raises the plan's
// error flag, the block waits (bounded) for its issued MMAs, frees its tensor
// memory and stops.
constexpr int kTcSrc = 16;               // sources per tile: K = 32
constexpr int kTcTgt = 64;               // targets per tile: N <= 64
constexpr int kTcStageFloats = 4 * 2048; // A hi, A lo, B hi, B lo: 64 x 32 floats each
constexpr size_t kTcSmem = 2 * kTcStageFloats * sizeof(float);

// Offset (floats) of element (row, k) of a 64 x 32 K-major operand: core
// matrix (k/4, row/8) at ((k/4)*8 + row/8) * 32 floats, row row%8 at +4*(row%8).
__device__ __forceinline__ int tc_off(int row, int k) {
    return (((k >> 2) << 3) + (row >> 3)) * 32 + ((row & 7) << 2) + (k & 3);
}

__device__ __forceinline__ void tc_split_store(float* hi, float* lo, int off, float a, float b) {
    const float ah = tc::to_tf32(a), bh = tc::to_tf32(b);
    *reinterpret_cast<float2*>(hi + off) = make_float2(ah, bh);
    *reinterpret_cast<float2*>(lo + off) = make_float2(a - ah, b - bh);
}

__global__ void __launch_bounds__(128) k_p2p_tc(DevCommon c, const float2* __restrict__ qs,
                                                float2* __restrict__ part, int R, int rb0) {
    extern __shared__ __align__(128) float tsm[];
    __shared__ float4 th[kTcTgt], tl[kTcTgt];      // target hi / lo coordinates
    __shared__ float4 sh[kTcSrc], sl[kTcSrc];      // source hi / lo coordinates of the tile
    __shared__ float2 qsm[kTcSrc][33];             // charges / (4 pi) of the tile, [source][column]
    __shared__ int rbeg[kP2PRanges], roff[kP2PRanges + 1];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ uint32_t taddr_sh;
    __shared__ int fail_sh;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int u = c.sh_unit ? c.sh_unit[blockIdx.x] : (int)blockIdx.x;   // work unit (of the shard)
    const int cell = DEFMM_IX(c, c.p2p_leaf[DEFMM_IX(c, c.p2p_unit_leaf[u], c.n_leaf_all)], c.n_cell_t);
    const int tb = c.ct_beg[cell], te = c.ct_end[cell];
    const int64_t pbase = c.p2p_part[u];
    const int nr = min(32, R - rb0);
    const float kap2pi = (float)(kappa_of(c, cell) * kInv2Pi);
    const float eps2 = (float)(eps_of(c, cell) * eps_of(c, cell));
    const float inv4pi = (float)kInv4Pi;
    const float lam2 = (float)(c.damping * kLog2E);
    const int r0 = c.p2p_unit_off[u], r1 = c.p2p_unit_off[u + 1];
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fail_sh = 0;
        mbar_fence_init();
    }
    if (warp == 0) tc::alloc(&taddr_sh, 128);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = taddr_sh;
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
    uint32_t uses[2] = {0, 0};   // commits issued on each stage's barrier (uniform)
    bool unread[2] = {false, false};
    int last_st = 0;
    int N = 8;
    // D row 16 w + i sits in TMEM lane 32 w + i (i < 16): Re rows from warps 0-1, Im from 2-3.
    // acc[col] is this thread's row of the target tile, summed over the source tiles in
    // f32 (each tile's own sum stays in the tensor cores, a short accumulation chain).
    float acc[kTcTgt];
#pragma unroll
    for (int j = 0; j < kTcTgt; ++j) acc[j] = 0.f;
    auto take = [&](int st) {    // adds the finished tile in TMEM buffer st to acc
        tc::fence_after_sync();
#pragma unroll
        for (int cc = 0; cc < kTcTgt / 16; ++cc)
            if (cc * 16 < N) {
                float v[16];
                tc::ld16(taddr + lane_base + (uint32_t)(64 * st + 16 * cc), v);
#pragma unroll
                for (int j = 0; j < 16; ++j) acc[16 * cc + j] += v[j];
            }
        tc::fence_before_sync();
        unread[st] = false;
    };
    for (int t0 = tb; t0 < te; t0 += kTcTgt) {
        const int nt = min(kTcTgt, te - t0);
        N = (nt + 7) & ~7;
        const uint32_t idesc = tc::idesc_tf32(64, N);
        if (tid < nt) { th[tid] = c.Xh[t0 + tid]; tl[tid] = c.Xl[t0 + tid]; }
        for (int g0 = r0; g0 < r1; g0 += kP2PRanges) {          // batches of ranges
            const int ng = min(kP2PRanges, r1 - g0);
            __syncthreads();
            for (int k = tid; k < ng; k += blockDim.x) {
                rbeg[k] = c.p2p_sbeg[g0 + k];
                roff[k] = c.p2p_soff[g0 + k] - c.p2p_soff[g0];
            }
            if (tid == 0) roff[ng] = c.p2p_soff[g0 + ng - 1] - c.p2p_soff[g0] + c.p2p_send[g0 + ng - 1] - c.p2p_sbeg[g0 + ng - 1];
            __syncthreads();
            const int total = roff[ng];
            auto source_of = [&](int f) {
                int lo = 0, hi = ng - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (roff[mid] <= f) lo = mid; else hi = mid - 1;
                }
                return rbeg[lo] + (f - roff[lo]);
            };
            // the next tile's sources and charges are fetched into registers while
            // the current tile is formed (coalesced over sources)
            float4 pf_h = make_float4(0.f, 0.f, 0.f, 0.f), pf_l = pf_h;
            float2 pf_q[4];
            auto fetch = [&](int f) {
                const int s = tid & 15;
                int64_t j = -1;
                if (f + s < total) j = DEFMM_IX(c, (int64_t)source_of(f + s), c.ny);
                if (tid < kTcSrc) {
                    pf_h = j >= 0 ? c.Yh[j] : make_float4(0.f, 0.f, 0.f, 0.f);
                    pf_l = j >= 0 ? c.Yl[j] : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int r = (tid >> 4) + 8 * k;
                    pf_q[k] = (j >= 0 && r < nr) ? qs[(int64_t)(rb0 + r) * c.ny + j] : make_float2(0.f, 0.f);
                }
            };
            fetch(0);
            for (int f0 = 0; f0 < total; f0 += kTcSrc) {
                const int ns = min(kTcSrc, total - f0);
                const int st = (int)((uses[0] + uses[1]) & 1);
                // the MMAs that last used this stage (its shared operands and its TMEM
                // buffer) must be done before either is rewritten; their tile is taken
                if (uses[st] > 0 && !mbar_wait(&bar[st], (uses[st] - 1) & 1)) fail_sh = 1;
                if (unread[st]) take(st);
                {
                    const int s = tid & 15;
                    if (tid < kTcSrc) { sh[s] = pf_h; sl[s] = pf_l; }
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        qsm[s][(tid >> 4) + 8 * k] = make_float2(pf_q[k].x * inv4pi, pf_q[k].y * inv4pi);
                }
                __syncthreads();
                if (fail_sh) break;
                if (f0 + kTcSrc < total) fetch(f0 + kTcSrc);   // in flight while this tile is formed
                float* Ahi = tsm + st * kTcStageFloats;
                float* Alo = Ahi + 2048;
                float* Bhi = Ahi + 4096;
                float* Blo = Ahi + 6144;
                // A: rows r (Re) and 32 + r (Im), columns 2s (Re q) and 2s + 1 (Im q)
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int s = warp + 4 * k, r = lane;
                    const float2 q = qsm[s][r];
                    tc_split_store(Ahi, Alo, tc_off(r, 2 * s), q.x, -q.y);
                    tc_split_store(Ahi, Alo, tc_off(32 + r, 2 * s), q.y, q.x);
                }
                // B: kernel values of the tile, zero outside the targets and sources.
                // Thread -> target t (a lane of 32 or 64) and a group of 4 or 8 sources.
                {
                    const bool narrow = N <= 32;
                    const int t = narrow ? (tid & 31) : (tid & 63);
                    const int sg = narrow ? (tid >> 5) : (tid >> 6);
                    const int spg = narrow ? 4 : 8;
                    if (t < N) {
                        const float4 xh = th[t], xl = tl[t];
                        for (int i = 0; i < spg; ++i) {
                            const int s = sg * spg + i;
                            float gr = 0.f, gi = 0.f;
                            if (t < nt && s < ns) {
                                const float4 a = sh[s], b = sl[s];
                                const float dx = (xh.x - a.x) + (xl.x - b.x);
                                const float dy = (xh.y - a.y) + (xl.y - b.y);
                                const float dz = (xh.z - a.z) + (xl.z - b.z);
                                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                                float rinv = rsqrt_hw(r2);
                                rinv = r2 > eps2 ? rinv : 0.f;
                                float sn, cs;
                                turns_sincos(r2 * rinv * kap2pi, &sn, &cs);
                                const float amp = c.radial_power == 2 ? rinv * rinv : rinv;
                                rinv = lam2 != 0.f ? amp * ex2_hw(-lam2 * (r2 * rinv)) : amp;
                                gr = cs * rinv;
                                gi = sn * rinv;
                            }
                            tc_split_store(Bhi, Blo, tc_off(t, 2 * s), gr, gi);
                        }
                    }
                }
                tc::fence_smem_to_async();
                __syncthreads();
                if (tid == 0) {
                    tc::fence_after_sync();
                    const uint32_t d = taddr + (uint32_t)(64 * st);
                    const uint32_t a0 = smem_u32(Ahi), l0 = smem_u32(Alo), b0 = smem_u32(Bhi), m0 = smem_u32(Blo);
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {   // K = 8 per MMA: two core matrices along K
                        const uint32_t o = ks * 2048;
                        const uint64_t ah = tc::smem_desc(a0 + o, 1024, 128), al = tc::smem_desc(l0 + o, 1024, 128);
                        const uint64_t bh = tc::smem_desc(b0 + o, 1024, 128), bl = tc::smem_desc(m0 + o, 1024, 128);
                        tc::mma_tf32(d, al, bh, idesc, ks > 0);   // a fresh sum per tile
                        tc::mma_tf32(d, ah, bl, idesc, true);
                        tc::mma_tf32(d, ah, bh, idesc, true);
                    }
                    tc::commit(&bar[st]);
                }
                ++uses[st];
                unread[st] = true;
                last_st = st;
            }
            if (fail_sh) break;
        }
        if (fail_sh) break;
        // take the last two tiles, older first
        for (int k = 0; k < 2; ++k) {
            const int st = k == 0 ? last_st ^ 1 : last_st;
            if (!unread[st]) continue;
            if (!mbar_wait(&bar[st], (uses[st] - 1) & 1)) fail_sh = 1;
            take(st);   // warp-collective load: taken even after a failed wait (results dropped)
        }
        __syncthreads();
        if (fail_sh) break;
        if (lane < 16) {
            const int r = (16 * warp + lane) & 31;
            if (r < nr) {
                float* dst = reinterpret_cast<float*>(part + (int64_t)(rb0 + r) * c.p2p_parts + pbase + (t0 - tb)) + (warp >= 2 ? 1 : 0);
#pragma unroll
                for (int j = 0; j < kTcTgt; ++j)
                    if (j < nt) dst[2 * j] = acc[j];
            }
        }
#pragma unroll
        for (int j = 0; j < kTcTgt; ++j) acc[j] = 0.f;
    }
    if (fail_sh) {
        if (tid == 0) {
            atomicExch(c.err_flag, 1);
            // bounded wait for the MMAs already issued before the memory they use is released
            if (uses[0] > 0) (void)mbar_wait(&bar[0], (uses[0] - 1) & 1);
            if (uses[1] > 0) (void)mbar_wait(&bar[1], (uses[1] - 1) & 1);
        }
        tc::fence_before_sync();
        __syncthreads();
    }
    tc::fence_after_sync();
    if (warp == 0) tc::dealloc(taddr, 128);
}

// ------------------------------------------------------------------ M2L launch
// Right-hand sides per row-kernel pass (complex64): the plan's choice when set,
// else 4 for N <= 8 (2 for two or three right-hand sides), 2 for N = 9 and 1
// for longer rows, whose accumulators would not fit in registers.
__host__ int m2l_pick_rb(const DevCommon& c, int R) {
    if (R == 1) return 1;
    int rb = c.m2l_rb > 0 ? c.m2l_rb : (c.N <= 8 ? (R >= 4 ? 4 : 2) : 2);
    if (c.N > 9) return 1;
    if (c.N == 9 && rb > 2) rb = 2;
    return rb >= 4 ? 4 : (rb >= 2 ? 2 : 1);
}

template <typename T, int NX, int TPM, int ROWS, int RB, int MINB, int PC, int NC, int MAXM = 8>
__host__ cudaError_t rows_config() {
    auto k = k_m2l_rows<T, NX, TPM, ROWS, RB, MINB, PC, NC, MAXM>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit);
    if (e != cudaSuccess) return e;
    // the row kernel's occupancy is set by shared memory: ask for the largest carveout
    return cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
}

// Launches one row-kernel variant; *fits = false (nothing launched) when its
// ring or F2L arrays do not fit in one block's shared memory.
template <typename T, int NX, int TPM, int ROWS, int RB, int MINB, int PC, int NC, int MAXM = 8>
__host__ void rows_launch(const DevCommon& c, const DevTyped<T>& t, const DevWork<T>& w, cudaStream_t stream,
                          bool* fits) {
    int S, stage;
    size_t sm;
    *fits = m2l_rows_shape<T>(c, RB, MINB, MAXM, &S, &stage, &sm);
    if (!*fits) return;
    const unsigned blocks = (unsigned)(MAXM == 4 ? c.n_grp_half : c.n_grp);
    k_m2l_rows<T, NX, TPM, ROWS, RB, MINB, PC, NC, MAXM><<<blocks, MAXM * TPM + 32, sm, stream>>>(
        c, t, w.Mhat, w.L, w.R, S, stage);
}

// The Hadamard M2L + F2L of one apply: the row kernel for N <= 12 (rows of N
// samples; N <= 8: 64 threads per member, N = 9: 96, N = 10..12: 64 threads
// with two rows each), the per-sample kernel beyond.
template <typename T>
cudaError_t launch_m2l(const DevCommon& c, const DevTyped<T>& t, const DevWork<T>& w, cudaStream_t stream,
                       int* nlaunch) {
    constexpr bool F = sizeof(T) == 4;
    const int N = c.N, p = c.p;
    bool fits = false;
    *nlaunch = 1;
    if (N <= 8) {
        if constexpr (F) {
            const int rb = m2l_pick_rb(c, w.R);
            if (p == 4 && N == 7) {
                if (rb == 1 && (c.m2l_members == 0 || c.m2l_members == 12 || c.m2l_members == 14)) {
                    // by group size: groups of at most 4 siblings whole in blocks of
                    // 4 (five per SM), 5-7 in blocks of 7 and 8 in blocks of 8 (three
                    // per SM; 0 and 14, the default), or more than 4 in blocks of 8
                    // (12), so few member warps idle
                    const bool three = c.m2l_members != 12;
                    bool fb = true, fs = true;
                    *nlaunch = 0;
                    if (!three && c.n_grp_big > 0) {
                        DevCommon cb = c;
                        cb.sh_grp = c.grp_big; cb.n_grp = c.n_grp_big;
                        rows_launch<T, 8, 64, 1, 1, 3, 4, 7>(cb, t, w, stream, &fb);
                        ++*nlaunch;
                    }
                    if (three && c.n_grp_large > 0) {
                        DevCommon cb = c;
                        cb.sh_grp = c.grp_large; cb.n_grp = c.n_grp_large;
                        rows_launch<T, 8, 64, 1, 1, 3, 4, 7>(cb, t, w, stream, &fb);
                        ++*nlaunch;
                    }
                    if (three && fb && c.n_grp_mid > 0) {
                        DevCommon cb = c;
                        cb.sh_grp = c.grp_mid; cb.n_grp = c.n_grp_mid;
                        rows_launch<T, 8, 64, 1, 1, 3, 4, 7, 7>(cb, t, w, stream, &fb);
                        ++*nlaunch;
                    }
                    if (fb && c.n_grp_small > 0) {
                        DevCommon cs = c;
                        cs.grp_half = c.grp_small; cs.n_grp_half = c.n_grp_small;
                        for (int v = 0; v < 3; ++v) cs.chk_stage_blocks[v] = c.chk_stage_small[v];   // smaller chunks
                        rows_launch<T, 8, 64, 1, 1, 5, 4, 7, 4>(cs, t, w, stream, &fs);
                        ++*nlaunch;
                    }
                    fits = fb && fs;
                    if (!fits) *nlaunch = 1;   // nothing launched: the fallback below runs alone
                }
                else if (rb == 1 && c.m2l_members == 4) rows_launch<T, 8, 64, 1, 1, 4, 4, 7, 4>(c, t, w, stream, &fits);
                else if (rb == 1) rows_launch<T, 8, 64, 1, 1, 3, 4, 7>(c, t, w, stream, &fits);
                else if (rb == 2) rows_launch<T, 8, 64, 1, 2, 2, 4, 7>(c, t, w, stream, &fits);
                else rows_launch<T, 8, 64, 1, 4, 1, 4, 7>(c, t, w, stream, &fits);
                // a stage of 4 (or 2) columns of the plan's largest chunk may not fit in
                // shared memory: fewer columns per pass (the same sums, so the same bits)
                if (!fits && rb == 4) rows_launch<T, 8, 64, 1, 2, 2, 4, 7>(c, t, w, stream, &fits);
                if (!fits && rb >= 2) rows_launch<T, 8, 64, 1, 1, 3, 4, 7>(c, t, w, stream, &fits);
            } else {
                if (rb == 1) rows_launch<T, 8, 64, 1, 1, 3, 0, 0>(c, t, w, stream, &fits);
                else if (rb == 2) rows_launch<T, 8, 64, 1, 2, 2, 0, 0>(c, t, w, stream, &fits);
                else rows_launch<T, 8, 64, 1, 4, 1, 0, 0>(c, t, w, stream, &fits);
                if (!fits && rb == 4) rows_launch<T, 8, 64, 1, 2, 2, 0, 0>(c, t, w, stream, &fits);
                if (!fits && rb >= 2) rows_launch<T, 8, 64, 1, 1, 3, 0, 0>(c, t, w, stream, &fits);
            }
        } else {
            if (p == 4 && N == 7) rows_launch<T, 8, 64, 1, 1, 1, 4, 7>(c, t, w, stream, &fits);
            else rows_launch<T, 8, 64, 1, 1, 1, 0, 0>(c, t, w, stream, &fits);
        }
    } else if (N <= 12) {
        if (p == 5 && N == 9) {
            bool one = true;
            if constexpr (F) {
                // one column per pass: blocks of 4 members (two per SM) measured faster;
                // two columns: blocks of 8 (the larger ring wins)
                one = m2l_pick_rb(c, w.R) == 1;
                if (!one && c.m2l_members == 4) rows_launch<T, 9, 96, 1, 2, 2, 5, 9, 4>(c, t, w, stream, &fits);
                else if (!one) rows_launch<T, 9, 96, 1, 2, 1, 5, 9>(c, t, w, stream, &fits);
                else if (c.m2l_members != 8) rows_launch<T, 9, 96, 1, 1, 2, 5, 9, 4>(c, t, w, stream, &fits);
            }
            if (one && !fits) rows_launch<T, 9, 96, 1, 1, 1, 5, 9>(c, t, w, stream, &fits);
        } else if (p == 6 && N == 11) {
            if constexpr (F) {   // complex64: blocks of 4 members, two per SM, unless 8 are asked for
                if (c.m2l_members != 8) rows_launch<T, 12, 64, 2, 1, 2, 6, 11, 4>(c, t, w, stream, &fits);
            }
            if (!fits) rows_launch<T, 12, 64, 2, 1, 1, 6, 11>(c, t, w, stream, &fits);
        } else {
            rows_launch<T, 12, 64, 2, 1, 1, 0, 0>(c, t, w, stream, &fits);
        }
    }
    if (fits) return cudaSuccess;
    int S;
    size_t sm;
    m2l_shape<T>(c, &S, &sm);
    if (sm > kSmemLimit) return cudaErrorInvalidConfiguration;
    if (c.NF <= 512) {          // two samples per thread, at most 256 threads
        const int threads = ((c.NF + 1) / 2 + 31) / 32 * 32;
        k_m2l<T, 2, 256><<<(unsigned)c.n_grp, threads, sm, stream>>>(c, t, w.Mhat, w.L, w.R, S);
    } else if (c.NF <= 1024) {  // four samples per thread, at most 256 threads
        const int threads = ((c.NF + 3) / 4 + 31) / 32 * 32;
        k_m2l<T, 4, 256><<<(unsigned)c.n_grp, threads, sm, stream>>>(c, t, w.Mhat, w.L, w.R, S);
    } else {                    // four samples per thread, up to 1024 threads
        const int threads = ((c.NF + 3) / 4 + 31) / 32 * 32;
        k_m2l<T, 4, 1024><<<(unsigned)c.n_grp, threads, sm, stream>>>(c, t, w.Mhat, w.L, w.R, S);
    }
    return cudaSuccess;
}

int sm_count() {
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    int v = cache[dev].load(std::memory_order_relaxed);
    if (v <= 0) {
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
            cudaGetLastError();
            v = 152;
        }
        cache[dev].store(v, std::memory_order_relaxed);
    }
    return v;
}

cudaError_t launch_wait_probe(int* flag, int spins, cudaStream_t stream) {
    k_wait_probe<<<1, 32, 0, stream>>>(flag, spins);
    return cudaGetLastError();
}

cudaError_t launch_unslice(const void* src, int64_t ld, void* p, const int64_t* perm, int64_t n, int R, int64_t j0,
                           int64_t j1, int elem_bytes, int* err_flag, cudaStream_t stream) {
    if (j1 <= j0) return cudaSuccess;
    const unsigned grid = (unsigned)(4 * sm_count());
    if (elem_bytes == 8)
        k_unslice<float2><<<grid, 256, 0, stream>>>(static_cast<const float2*>(src), ld, static_cast<float2*>(p), perm,
                                                    n, R, j0, j1, err_flag);
    else
        k_unslice<double2><<<grid, 256, 0, stream>>>(static_cast<const double2*>(src), ld, static_cast<double2*>(p),
                                                     perm, n, R, j0, j1, err_flag);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ orchestration
template <typename T>
cudaError_t launch_apply(const DevCommon& c, const DevTyped<T>& t, const DevWork<T>& w,
                         const LevelList* m2m, int n_m2m_levels, const LevelList* l2l,
                         const int32_t* const* l2l_par, int n_l2l_levels, const void* q, void* p,
                         cudaStream_t stream, int* launches, cudaEvent_t* phase_events) {
    using C = typename Cplx<T>::type;
    const int R = w.R;
    int nl = 0;
    int phase = 0;
    cudaError_t err;
    // phase boundaries: NVTX ranges for tracing tools (no-ops without one) and,
    // when profiling, CUDA events on the apply's stream
    static const char* const kPhaseName[kNumPhases] = {"defmm gather", "defmm p2p", "defmm p2m", "defmm m2m",
                                                       "defmm m2f", "defmm m2l+f2l", "defmm l2l", "defmm l2p",
                                                       "defmm scatter"};
    auto mark = [&]() -> cudaError_t {
        if (phase > 0) nvtxRangePop();
        if (phase < kNumPhases) nvtxRangePushA(kPhaseName[phase]);
        const int k = phase++;
        if (!phase_events) return cudaSuccess;
        return cudaEventRecord(phase_events[k], stream);
    };
#define DEFMM_MARK()                        \
    do {                                    \
        err = mark();                       \
        if (err != cudaSuccess) return err; \
    } while (0)
#define DEFMM_CHECK_LAUNCH()                      \
    do {                                          \
        ++nl;                                     \
        err = cudaGetLastError();                 \
        if (err != cudaSuccess) {                 \
            if (launches) *launches = nl;         \
            return err;                           \
        }                                         \
    } while (0)
    const int sms = sm_count() * 8;
    DEFMM_MARK();
    // gather charges into Morton order
    k_gather<C><<<sms, 256, 0, stream>>>(reinterpret_cast<const C*>(q), w.qs, c.perm_s, c.ny, R, c.err_flag);
    DEFMM_CHECK_LAUNCH();
    DEFMM_MARK();
    // near field: work units write partial sums, reduced per target in fixed order
    bool p2p_done = false;
    if constexpr (std::is_same<T, float>::value) {
        // many right-hand sides: the near field as tensor-core products, 32 columns per pass
        if (c.p2p_tc_min_rhs > 0 && R >= c.p2p_tc_min_rhs && c.n_p2p_units > 0) {
            for (int rb0 = 0; rb0 < R; rb0 += 32) {
                k_p2p_tc<<<(unsigned)c.n_p2p_units, 128, kTcSmem, stream>>>(c, w.qs, w.part, R, rb0);
                DEFMM_CHECK_LAUNCH();
            }
            p2p_done = true;
        }
    }
    // complex64: 8 columns per pass from 8 columns on, 16 from 16 on (each kernel value
    // serves that many products)
    const int p2p_rb = R == 1 ? 1 : (!std::is_same<T, float>::value ? 4 : (R >= 16 ? 16 : (R >= 8 ? 8 : 4)));
    for (int rb0 = 0; rb0 < R && !p2p_done; rb0 += p2p_rb) {
        if (c.n_p2p_units == 0) break;
        if constexpr (std::is_same<T, float>::value) {
            const unsigned nu = (unsigned)c.n_p2p_units;
            const bool direct = c.p2p_direct_phase && !c.p2p_reduce_phase;
            if (c.radial_power == 2) {
                if (direct) launch_p2p_f32<2, false>(p2p_rb, nu, c, w.qs, w.part, R, rb0, stream);
                else launch_p2p_f32<2, true>(p2p_rb, nu, c, w.qs, w.part, R, rb0, stream);
            } else if (c.damping > 0.0) {
                if (direct) launch_p2p_f32<1, false>(p2p_rb, nu, c, w.qs, w.part, R, rb0, stream);
                else launch_p2p_f32<1, true>(p2p_rb, nu, c, w.qs, w.part, R, rb0, stream);
            } else {
                if (direct) launch_p2p_f32<0, false>(p2p_rb, nu, c, w.qs, w.part, R, rb0, stream);
                else launch_p2p_f32<0, true>(p2p_rb, nu, c, w.qs, w.part, R, rb0, stream);
            }
        } else {
            if (R == 1) k_p2p<T, 1><<<(unsigned)c.n_p2p_units, 128, 0, stream>>>(c, w.qs, w.part, R, rb0);
            else k_p2p<T, 4><<<(unsigned)c.n_p2p_units, 128, 0, stream>>>(c, w.qs, w.part, R, rb0);
        }
        DEFMM_CHECK_LAUNCH();
    }
    if (c.n_p2p_leaf > 0) {
        k_p2p_reduce<C><<<(unsigned)c.n_p2p_leaf, 128, 0, stream>>>(c, w.part, w.ps, R);
        DEFMM_CHECK_LAUNCH();
    }
    DEFMM_MARK();
    // upward pass
    for (int rb0 = 0; rb0 < R; rb0 += (R == 1 ? 1 : 4)) {
        if (c.n_p2m == 0) break;
        const int rb = R == 1 ? 1 : 4;
        if (c.p == 4 || c.p == 5) {          // one warp per leaf
            const int ep = p2m_warp_epass(c.p, rb);
            const size_t sm = p2m_warp_smem(c.p, rb, ep, sizeof(T));
            const unsigned nb = (unsigned)((c.n_p2m + kLeafWarps - 1) / kLeafWarps);
            if (c.p == 4 && R == 1) k_p2m_warp<T, 1, 4><<<nb, 32 * kLeafWarps, sm, stream>>>(c, t, w.qs, w.M, R, rb0, ep);
            else if (c.p == 4) k_p2m_warp<T, 4, 4><<<nb, 32 * kLeafWarps, sm, stream>>>(c, t, w.qs, w.M, R, rb0, ep);
            else if (R == 1) k_p2m_warp<T, 1, 5><<<nb, 32 * kLeafWarps, sm, stream>>>(c, t, w.qs, w.M, R, rb0, ep);
            else k_p2m_warp<T, 4, 5><<<nb, 32 * kLeafWarps, sm, stream>>>(c, t, w.qs, w.M, R, rb0, ep);
        } else {
            const int ep = p2m_epass(c.P3, rb, sizeof(T));
            const size_t sm = p2m_smem(c.p, rb, ep, sizeof(T));
            if (R == 1) k_p2m<T, 1><<<(unsigned)c.n_p2m, 128, sm, stream>>>(c, t, w.qs, w.M, R, rb0, ep);
            else k_p2m<T, 4><<<(unsigned)c.n_p2m, 128, sm, stream>>>(c, t, w.qs, w.M, R, rb0, ep);
        }
        DEFMM_CHECK_LAUNCH();
    }
    DEFMM_MARK();
    const size_t per_warp_mm = (2 * (size_t)c.P3 + 72) * sizeof(C);
    const int wpb_mm = warps_per_block(per_warp_mm);
    for (int l = n_m2m_levels - 1; l >= 0; --l) {
        if (m2m[l].n == 0) continue;
        const unsigned blocks = (unsigned)((m2m[l].n * R + wpb_mm - 1) / wpb_mm);   // a warp per (item, column)
        if (c.p == 4) k_m2m<T, 4><<<blocks, 32 * wpb_mm, wpb_mm * per_warp_mm, stream>>>(c, t, m2m[l].data, m2m[l].n, w.M, R);
        else if (c.p == 5) k_m2m<T, 5><<<blocks, 32 * wpb_mm, wpb_mm * per_warp_mm, stream>>>(c, t, m2m[l].data, m2m[l].n, w.M, R);
        else if (c.p == 6) k_m2m<T, 6><<<blocks, 32 * wpb_mm, wpb_mm * per_warp_mm, stream>>>(c, t, m2m[l].data, m2m[l].n, w.M, R);
        else k_m2m<T><<<blocks, 32 * wpb_mm, wpb_mm * per_warp_mm, stream>>>(c, t, m2m[l].data, m2m[l].n, w.M, R);
        DEFMM_CHECK_LAUNCH();
    }
    DEFMM_MARK();
    if (c.n_m2f > 0) {
        const size_t per_warp = ((size_t)c.P3 + (size_t)c.p * c.p * c.N + (size_t)c.p * c.N * c.N) * sizeof(C);
        const int wpb = warps_per_block(per_warp);
        const unsigned blocks = (unsigned)((c.n_m2f * R + wpb - 1) / wpb);   // a warp per (item, column)
        if (c.p == 4 && c.N == 7) k_m2f<T, 4, 7><<<blocks, 32 * wpb, wpb * per_warp, stream>>>(c, t, w.M, w.Mhat, R);
        else if (c.p == 5 && c.N == 9) k_m2f<T, 5, 9><<<blocks, 32 * wpb, wpb * per_warp, stream>>>(c, t, w.M, w.Mhat, R);
        else if (c.p == 6 && c.N == 11) k_m2f<T, 6, 11><<<blocks, 32 * wpb, wpb * per_warp, stream>>>(c, t, w.M, w.Mhat, R);
        else k_m2f<T><<<blocks, 32 * wpb, wpb * per_warp, stream>>>(c, t, w.M, w.Mhat, R);
        DEFMM_CHECK_LAUNCH();
    }
    DEFMM_MARK();
    // transfer
    err = cudaMemsetAsync(w.L, 0, (size_t)w.nL * R * c.P3 * sizeof(C), stream);
    if (err != cudaSuccess) return err;
    if (c.n_grp > 0) {
        int k = 1;
        err = launch_m2l<T>(c, t, w, stream, &k);
        if (err != cudaSuccess) return err;
        nl += k - 1;
        DEFMM_CHECK_LAUNCH();
    }
    DEFMM_MARK();
    // downward pass
    for (int l = 1; l < n_l2l_levels; ++l) {
        if (l2l[l].n == 0) continue;
        const unsigned blocks = (unsigned)((l2l[l].n * R + wpb_mm - 1) / wpb_mm);   // a warp per (item, column)
        if (c.p == 4) k_l2l<T, 4><<<blocks, 32 * wpb_mm, wpb_mm * per_warp_mm, stream>>>(c, t, l2l[l].data, l2l[l].n, l2l_par[l], w.L, R);
        else if (c.p == 5) k_l2l<T, 5><<<blocks, 32 * wpb_mm, wpb_mm * per_warp_mm, stream>>>(c, t, l2l[l].data, l2l[l].n, l2l_par[l], w.L, R);
        else if (c.p == 6) k_l2l<T, 6><<<blocks, 32 * wpb_mm, wpb_mm * per_warp_mm, stream>>>(c, t, l2l[l].data, l2l[l].n, l2l_par[l], w.L, R);
        else k_l2l<T><<<blocks, 32 * wpb_mm, wpb_mm * per_warp_mm, stream>>>(c, t, l2l[l].data, l2l[l].n, l2l_par[l], w.L, R);
        DEFMM_CHECK_LAUNCH();
    }
    DEFMM_MARK();
    for (int rb0 = 0; rb0 < R; rb0 += (R == 1 ? 1 : 4)) {
        if (c.n_l2p == 0) break;
        const int rb = R == 1 ? 1 : 4;
        if (c.p == 4 || c.p == 5) {          // one warp per leaf
            const int ep = l2p_warp_epass(c.P3, rb, sizeof(C));
            const size_t sm = l2p_warp_smem(c.P3, rb, ep, sizeof(C));
            const unsigned nb = (unsigned)((c.n_l2p + kLeafWarps - 1) / kLeafWarps);
            if (c.p == 4 && R == 1) k_l2p_warp<T, 1, 4><<<nb, 32 * kLeafWarps, sm, stream>>>(c, t, w.L, w.ps, R, rb0, ep);
            else if (c.p == 4) k_l2p_warp<T, 4, 4><<<nb, 32 * kLeafWarps, sm, stream>>>(c, t, w.L, w.ps, R, rb0, ep);
            else if (R == 1) k_l2p_warp<T, 1, 5><<<nb, 32 * kLeafWarps, sm, stream>>>(c, t, w.L, w.ps, R, rb0, ep);
            else k_l2p_warp<T, 4, 5><<<nb, 32 * kLeafWarps, sm, stream>>>(c, t, w.L, w.ps, R, rb0, ep);
        } else {
            const int ep = l2p_epass(c.P3, rb, sizeof(C));
            const size_t sm = l2p_smem(c.P3, rb, ep, sizeof(C));
            if (R == 1) k_l2p<T, 1><<<(unsigned)c.n_l2p, 128, sm, stream>>>(c, t, w.L, w.ps, R, rb0, ep);
            else k_l2p<T, 4><<<(unsigned)c.n_l2p, 128, sm, stream>>>(c, t, w.L, w.ps, R, rb0, ep);
        }
        DEFMM_CHECK_LAUNCH();
    }
    DEFMM_MARK();
    if (w.slice) {   // the shard's potentials alone, in sorted order
        const int64_t j0 = c.sh_on ? c.sh_t0 : 0, j1 = c.sh_on ? c.sh_t1 : c.nx;
        if (j1 > j0) k_slice<C><<<sms, 256, 0, stream>>>(w.ps, w.slice, c.nx, R, j0, j1, w.slice_ld);
    } else {
        if (c.sh_on) {   // one shard: its targets, zeros elsewhere (the shards' outputs sum to the whole)
            err = cudaMemsetAsync(p, 0, (size_t)c.nx * R * sizeof(C), stream);
            if (err != cudaSuccess) return err;
        }
        if (!c.sh_on || c.sh_t1 > c.sh_t0)
            k_scatter<C><<<sms, 256, 0, stream>>>(w.ps, reinterpret_cast<C*>(p), c.perm_t, c.nx, R,
                                                  c.sh_on ? c.sh_t0 : 0, c.sh_on ? c.sh_t1 : c.nx, c.err_flag);
    }
    DEFMM_CHECK_LAUNCH();
    DEFMM_MARK();
#undef DEFMM_CHECK_LAUNCH
#undef DEFMM_MARK
    if (launches) *launches = nl;
    return cudaSuccess;
}

// Raises the dynamic shared-memory limit of the kernels that may need more
// than 48 KB (large orders / FFT lengths, float64).
template <typename T>
cudaError_t configure_kernels() {
    const int big = (int)kSmemLimit;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_m2l<T, 2, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, big)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_m2l<T, 4, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, big)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_m2l<T, 4, 1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, big)) != cudaSuccess) return e;
    if constexpr (sizeof(T) == 4) {
        if ((e = cudaFuncSetAttribute(k_p2p_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem)) != cudaSuccess) return e;
        if ((e = rows_config<T, 8, 64, 1, 1, 3, 4, 7>()) != cudaSuccess) return e;
        if ((e = rows_config<T, 8, 64, 1, 2, 2, 4, 7>()) != cudaSuccess) return e;
        if ((e = rows_config<T, 8, 64, 1, 4, 1, 4, 7>()) != cudaSuccess) return e;
        if ((e = rows_config<T, 8, 64, 1, 1, 3, 0, 0>()) != cudaSuccess) return e;
        if ((e = rows_config<T, 8, 64, 1, 2, 2, 0, 0>()) != cudaSuccess) return e;
        if ((e = rows_config<T, 8, 64, 1, 4, 1, 0, 0>()) != cudaSuccess) return e;
        if ((e = rows_config<T, 9, 96, 1, 2, 1, 5, 9>()) != cudaSuccess) return e;
        if ((e = rows_config<T, 8, 64, 1, 1, 4, 4, 7, 4>()) != cudaSuccess) return e;
        if ((e = rows_config<T, 8, 64, 1, 1, 5, 4, 7, 4>()) != cudaSuccess) return e;
        if ((e = rows_config<T, 8, 64, 1, 1, 3, 4, 7, 7>()) != cudaSuccess) return e;
        if ((e = rows_config<T, 9, 96, 1, 2, 2, 5, 9, 4>()) != cudaSuccess) return e;
        if ((e = rows_config<T, 9, 96, 1, 1, 2, 5, 9, 4>()) != cudaSuccess) return e;
        if ((e = rows_config<T, 12, 64, 2, 1, 2, 6, 11, 4>()) != cudaSuccess) return e;
    } else {
        if ((e = rows_config<T, 8, 64, 1, 1, 1, 4, 7>()) != cudaSuccess) return e;
        if ((e = rows_config<T, 8, 64, 1, 1, 1, 0, 0>()) != cudaSuccess) return e;
    }
    if ((e = rows_config<T, 9, 96, 1, 1, 1, 5, 9>()) != cudaSuccess) return e;
    if ((e = rows_config<T, 12, 64, 2, 1, 1, 6, 11>()) != cudaSuccess) return e;
    if ((e = rows_config<T, 12, 64, 2, 1, 1, 0, 0>()) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_m2f<T, 4, 7>, cudaFuncAttributeMaxDynamicSharedMemorySize, big)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_m2f<T, 5, 9>, cudaFuncAttributeMaxDynamicSharedMemorySize, big)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_m2f<T, 6, 11>, cudaFuncAttributeMaxDynamicSharedMemorySize, big)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_m2m<T, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize, big)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_l2l<T, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize, big)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_m2m<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, big)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_m2m<T, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize, big)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_l2l<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, big)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_l2l<T, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize, big)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_m2f<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_m2m<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_l2l<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_p2m<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_p2m<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, big)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_l2p<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_l2p<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, big)) != cudaSuccess) return e;
    return cudaSuccess;
}

template cudaError_t launch_apply<float>(const DevCommon&, const DevTyped<float>&, const DevWork<float>&,
                                         const LevelList*, int, const LevelList*, const int32_t* const*, int,
                                         const void*, void*, cudaStream_t, int*, cudaEvent_t*);
template cudaError_t launch_apply<double>(const DevCommon&, const DevTyped<double>&, const DevWork<double>&,
                                          const LevelList*, int, const LevelList*, const int32_t* const*, int,
                                          const void*, void*, cudaStream_t, int*, cudaEvent_t*);
template cudaError_t configure_kernels<float>();
template cudaError_t configure_kernels<double>();

}  // namespace defmm
