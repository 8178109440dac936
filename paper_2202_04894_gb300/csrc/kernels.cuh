// Device-side tables of a plan and the launchers of the application-phase
// kernels (Sec. 2.2 operators, Sec. 4.1.1 M2F/F2L, Sec. 4.3 symmetries,
// Sec. 5.3 near field).  All pointers are device pointers.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <type_traits>

namespace defmm {

template <typename T> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };

// Precision-independent tables.
struct DevCommon {
    int p, N, NF, NFpad, P3;
    int64_t nx, ny;
    double kappa, eps_self;
    double damping;          // lambda >= 0: G = exp((i kappa - lambda) r) / (4 pi r^P)
    int radial_power;        // P: 1 (Helmholtz family) or 2
    const double* Xs;        // nx*3 targets, Morton order
    const double* Ys;        // ny*3 sources, Morton order
    const float4* Xh;        // targets minus the cube centre, float hi part (w unused)
    const float4* Xl;        // the float remainder (x - c) - hi
    const float4* Yh;        // same for sources
    const float4* Yl;
    const int64_t* perm_t;   // sorted -> input
    const int64_t* perm_s;
    // target / source cells
    const int32_t *ct_beg, *ct_end, *ct_level;
    const double* ct_corner;  // 3 per cell
    const int32_t *cs_beg, *cs_end, *cs_level;
    const double* cs_corner;
    const double* level_side;  // per level
    // expansions
    const int32_t *m_first, *m_count, *m_slot;  // per source cell / per multipole
    const int32_t *l_first, *l_count, *l_slot;  // per target cell / per local
    const double* slot_u;                       // 3 per slot
    // tables
    const int32_t* m2f_list;  int64_t n_m2f;
    // M2L schedule: groups of sibling targets, chunks of staged blocks and pair ops
    const int32_t *grp_member_off, *grp_members, *grp_chunk_off;  int64_t n_grp;
    const int32_t* grp_half;  int64_t n_grp_half;   // blocks of <= 4 members: group * 2 + half
    // split by group size (members per block 12): groups of more than 4
    // members (ids) and the half-codes 2g of groups of at most 4
    const int32_t* grp_big;  int64_t n_grp_big;
    const int32_t* grp_small;  int64_t n_grp_small;
    // three classes (members per block 14 or 0): 5-7 members and 8 members
    const int32_t* grp_mid;  int64_t n_grp_mid;
    const int32_t* grp_large;  int64_t n_grp_large;
    const int32_t *chk_blk_off, *chk_nspec, *chk_blk, *chk_op_off, *chk_op;
    int chk_max_blocks;
    int chk_stage_blocks[3];  // largest stage (blocks) for 1, 2, 4 right-hand sides per pass
    int chk_stage_small[3];   // the same over the chunks of groups of at most 4 siblings
    int m2l_rb;               // right-hand sides per M2L pass (0: chosen from nrhs and N)
    int m2l_members;          // members per M2L block: 4, 8, 12 (4 or 8 by group size), 14 (4, 7
                              // or 8 by group size), 0 (default)
    int p2p_direct_phase;     // 1: every near-field phase kappa r is at most 90 pi (bounded on the
                              // host from the P2P cell pairs), within the range where the hardware
                              // sine and cosine are documented accurate without a reduction
    int p2p_reduce_phase;     // tuning: 1 reduces the phase exactly whatever the bound
    int p2p_tc_min_rhs;       // complex64 applies with at least this many columns use the
                              // tensor-core near field (0: never)
    const int32_t* p2m_cells;  int64_t n_p2m;
    const int32_t* l2p_cells;  int64_t n_l2p;
    // near field: work units (leaf x bounded source ranges) and leaves
    const int32_t *p2p_unit_leaf, *p2p_unit_off, *p2p_sbeg, *p2p_send, *p2p_soff, *p2p_part;
    int64_t n_p2p_units, p2p_parts;
    const int32_t *p2p_leaf, *p2p_leaf_off, *p2p_leaf_units;
    int64_t n_p2p_leaf;
    int* err_flag;           // set by a kernel whose bounded wait gave up (read by defmm_check)
    // One shard of the targets (sh_on): the M2L groups, P2P units and P2P leaves
    // to run (indices into the full tables) and the sorted targets written,
    // [sh_t0, sh_t1).  The L2L / L2P lists and grp_half are swapped for the
    // shard's own.  Off: every table entry in order.
    int sh_on;
    const int32_t *sh_grp, *sh_unit, *sh_leaf;
    int64_t sh_t0, sh_t1;
    // A union of several geometries: the geometry of each cell and the
    // per-geometry wavenumber and self-distance (null for one geometry: kappa,
    // eps_self above).  Cell levels are global level ids into level_side.
    const int32_t* cell_geo;
    const double *geo_kappa, *geo_eps;
    // table sizes, for the bounds checks of a checked build (DEFMM_CHECKED)
    int64_t n_cell_t, n_cell_s, n_mult, n_local, n_slot, n_spec;
    int64_t n_leaf_all;   // near-field leaves of the whole operator (n_p2p_leaf counts a shard's)
};

// A table index a kernel follows.  In a checked build (compiled with
// DEFMM_CHECKED) an index outside [0, n) raises the plan's error flag with the
// value 2 (the first such index also records its source line, value and
// bound in the flag's next three words) and is replaced by 0, so the access
// stays inside the table and no control flow changes (no thread leaves a
// barrier or a wait behind); the apply's results are then invalid and the host
// reports the flag.  Otherwise the index is used as it is.
#ifdef DEFMM_CHECKED
__device__ __forceinline__ int64_t checked_index(int* flag, int64_t i, int64_t n, int line) {
    if (i < 0 || i >= n) {
        if (atomicCAS(flag, 0, 2) == 0) {
            flag[1] = line;
            flag[2] = (int)i;
            flag[3] = (int)n;
        }
        return 0;
    }
    return i;
}
#define DEFMM_IX(c, i, n) \
    ((std::remove_cv_t<std::remove_reference_t<decltype(i)>>)::defmm::checked_index((c).err_flag, (int64_t)(i), (int64_t)(n), __LINE__))
#else
#define DEFMM_IX(c, i, n) (i)
#endif

// Tables in the arithmetic precision T.
template <typename T>
struct DevTyped {
    using C = typename Cplx<T>::type;
    const C* slot_P;   // [slot][3][p]
    const C* slot_Q;   // [slot][3][2][p]
    const T* m1;       // [2][p][p]
    const C* tw;       // [N]  e^{2 pi i m/N}
    const C* spec;     // [nspec][NFpad]
};

// Per-apply buffers.
template <typename T>
struct DevWork {
    using C = typename Cplx<T>::type;
    int R;
    C* qs;     // [R][ny]
    C* ps;     // [R][nx]
    C* part;   // [R][p2p_parts] near-field partial sums of the work units
    C* M;      // [nM][R][P3]
    C* Mhat;   // [nMhat][R][NFpad]
    C* L;      // [nL][R][P3]
    int64_t nL;
    // set: the apply writes its shard's potentials in sorted order, slice[r * slice_ld + j]
    // for sorted target sh_t0 + j (all targets unsharded), instead of p in the caller's order
    C* slice = nullptr;
    int64_t slice_ld = 0;
};

struct LevelList {
    const int32_t* data;  // device
    int64_t n;            // entries
};

// Launchers (enqueue on `stream`, return the launch error if any).
template <typename T>
cudaError_t launch_apply(const DevCommon& c, const DevTyped<T>& t, const DevWork<T>& w,
                         const LevelList* m2m, int n_m2m_levels, const LevelList* l2l,
                         const int32_t* const* l2l_par, int n_l2l_levels, const void* q, void* p,
                         cudaStream_t stream, int* launches, cudaEvent_t* phase_events);

constexpr int kNumPhases = 9;  // gather p2p p2m m2m m2f m2l l2l l2p scatter

// One block waiting, boundedly, on an mbarrier phase nothing completes; raises *flag.
cudaError_t launch_wait_probe(int* flag, int spins, cudaStream_t stream);

// p[r * n + perm[j0 + j]] = src[r * ld + j] for 0 <= j < j1 - j0, r < R: one shard's
// sorted-order slice put back in the caller's order (elem_bytes 8: complex64, 16: complex128).
cudaError_t launch_unslice(const void* src, int64_t ld, void* p, const int64_t* perm, int64_t n, int R, int64_t j0,
                           int64_t j1, int elem_bytes, int* err_flag, cudaStream_t stream);

// Streaming multiprocessors of the current device (queried once per device).
int sm_count();

// Forms the canonical transfer spectra in float64 (Sec. 2.3 Eq. FourierDiagonal).
cudaError_t launch_spectra(const int32_t* spec_level, const int32_t* spec_kbar, int nspec,
                           const double* level_side, int p, int N, int NFpad, double kappa,
                           const double* spec_kappa, double damping, int power, double2* out_d, float2* out_f,
                           cudaStream_t stream);

}  // namespace defmm
