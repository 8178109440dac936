/* defmm — GB300 application phase of the directional equispaced-interpolation
 * fast multipole method for the Helmholtz kernel (Chollet, Claeys, Fortin,
 * Grigori, arXiv 2202.04894).
 *
 *   p(x) = sum_{y in Y} G(x, y) q(y),   G(x, y) = exp(i kappa |x-y|) / (4 pi |x-y|)
 *
 * (Eq. 1.1, Sec. 1).  A plan holds the geometry-dependent part (Morton-sorted
 * Ncrit octree, Sec. 4.2.1; direction tree, Sec. 4.1.2; dual tree traversal,
 * Alg. 1; blank passes, Alg. 2-3; transfer spectra with cube symmetries,
 * Sec. 4.3).  An apply runs P2M, M2M, M2F, the Fourier-domain Hadamard M2L,
 * F2L, L2L, L2P and P2P on one GPU (Sec. 2.2, 4.1.1).
 *
 * Conventions shared by every entry point
 *  - Status codes, never exceptions.  On failure defmm_last_error() returns a
 *    message (thread-local, valid until the next call on the same thread).
 *  - Asynchronous device errors of an apply surface at the next call that
 *    synchronises (defmm_apply_host, defmm_plan_create, defmm_destroy) as
 *    DEFMM_ERR_CUDA.
 *  - Complex arrays are interleaved (re, im) in double (DEFMM_C128) or float
 *    (DEFMM_C64), column-major over right-hand sides: entry (j, r) at j + n*r.
 *  - Point arrays are n x 3 row-major float64 (x0 y0 z0 x1 y1 z1 ...).
 */
#ifndef DEFMM_H
#define DEFMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct defmm_plan_s* defmm_plan; /* opaque; owned by the library */

typedef enum {
    DEFMM_OK = 0,
    DEFMM_ERR_ARG = 1,         /* invalid argument (null pointer, bad size/order) */
    DEFMM_ERR_OOM = 2,         /* device or host allocation failed, or hbm_budget exceeded */
    DEFMM_ERR_CUDA = 3,        /* a CUDA call failed (message names it) */
    DEFMM_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up */
    DEFMM_ERR_UNSUPPORTED = 5, /* option or dtype not supported */
    DEFMM_ERR_BUSY = 6         /* plan is in use by another thread */
} defmm_status;

typedef enum { DEFMM_C64 = 0, DEFMM_C128 = 1 } defmm_dtype;

/* Plan options.  Obtain defaults with defmm_default_options().
 *  eta        - MAC parameter of Eq. (macdirref), Sec. 4.2.2 (default 1).
 *  hf_kw      - a level is high-frequency iff kappa * w > hf_kw, w the cell
 *               radius; the paper leaves this boundary open (default 1).
 *  fft_n      - DFT length N per axis, N >= 2*order - 1; 0 selects 2*order - 1.
 *               Any admissible N gives the same result (Sec. 2.3).
 *  self_eps   - pairs with |x - y| <= self_eps * D are skipped, D the side of
 *               the smallest box holding X and Y (Sec. 5.3; default 1e-10).
 *  flags      - DEFMM_PLAN_HOST_ONLY builds the host tables only (no device
 *               memory, no GPU needed); such a plan answers defmm_plan_info and
 *               defmm_plan_table, and defmm_apply returns DEFMM_ERR_UNSUPPORTED.
 *  hbm_budget - refuse plans whose device footprint exceeds this many bytes
 *               (0: no limit).  Checked at plan creation (plan tables and
 *               one-RHS workspace) and at each apply (workspace for nrhs).
 *  damping    - lambda >= 0: the kernel becomes exp((i kappa - lambda) r) /
 *               (4 pi r), the Helmholtz kernel of the complex wavenumber
 *               kappa + i lambda (default 0, the paper's kernel).  kappa = 0
 *               gives the Yukawa (modified Helmholtz) kernel, kappa = lambda =
 *               0 the Laplace kernel; the method holds for such asymptotically
 *               smooth kernels (Sec. 1).  kappa alone sets the directional
 *               (high-frequency) structure; lambda enters the near field and
 *               the transfer spectra only.
 *  m2l_chunk_blocks - most spectra + Fourier multipoles staged together by the
 *               M2L kernel (0: the library's default, 8 for N = 7 or 9; a
 *               positive value >= 2 may only lower it).  Smaller chunks use
 *               less shared memory per block; no result depends on it.
 *  radial_power - P in G(r) = exp((i kappa - lambda) r) / (4 pi r^P): 1 (the
 *               default, the Helmholtz family above) or 2, an oscillatory
 *               kernel outside that family; the method needs only an
 *               asymptotically smooth kernel (Sec. 1), and the kernel enters
 *               the transfer spectra and the near field only.               */
typedef struct {
    double eta;
    double hf_kw;
    int fft_n;
    int flags;
    double self_eps;
    size_t hbm_budget;
    double damping;
    int m2l_chunk_blocks;
    int radial_power;
} defmm_options;

#define DEFMM_PLAN_HOST_ONLY 1

void defmm_default_options(defmm_options* opt);

/* Builds a plan (Sec. 4.2, 4.3): bounding cube, Morton sort, Ncrit octree
 * (Sec. 4.2.1), per-level regime and directions (Sec. 4.1.2), dual tree
 * traversal (Alg. 1), blank DTT and blank downward pass (Alg. 2, 3), best
 * directions, canonical transfer spectra (formed on the GPU in float64, Sec.
 * 2.3 Eq. FourierDiagonal, Sec. 4.3 Eq. permuteM2L) and the interpolation
 * tables (Sec. 5.2.1).
 *  X, nx     - targets, nx x 3 float64, host or device memory (detected).
 *  Y, ny     - sources, ny x 3 float64.  Y == X with ny == nx (same pointer)
 *              or Y == NULL means sources = targets and a single tree.
 *  kappa     - wavenumber, >= 0.
 *  order     - interpolation points per dimension p, 2 <= p <= 8.
 *  leaf_size - Ncrit: cells holding more points are split, >= 1.
 *  opt       - NULL for defaults.
 *  stream    - cudaStream_t for the plan's device work (NULL: legacy stream);
 *              the call returns after that work is complete.
 *  out       - receives the plan.  X and Y are only read during the call.
 * Errors: DEFMM_ERR_ARG (also for damping < 0 or not finite, radial_power
 * not 1 or 2), DEFMM_ERR_OOM,
 * DEFMM_ERR_CUDA.                                                             */
defmm_status defmm_plan_create(const double* X, int64_t nx, const double* Y, int64_t ny,
                               double kappa, int order, int leaf_size,
                               const defmm_options* opt, void* stream, defmm_plan* out);

/* A union of several independent geometries in one plan: geometry g has
 * nx[g] points X[g] (sources = targets) and wavenumber kappa[g]; order, leaf
 * size and options are shared.  Each geometry's plan is built as by
 * defmm_plan_create and the tables are concatenated, so one defmm_apply runs
 * every phase as one kernel launch over all geometries (per tree level for
 * M2M and L2L) instead of one per geometry.  q and p hold the geometries'
 * points one after another (geometry 0 first), in each geometry's own point
 * order; there is no interaction between geometries, and each geometry's
 * result equals its own plan's bit for bit.  defmm_plan_info reports sums
 * over the geometries (nlevels: the deepest tree; d_aabb: the largest box);
 * cell levels in defmm_plan_table are global level ids (one range per
 * geometry).  The paper treats one geometry; this batches its application
 * phase across many.
 * Errors: DEFMM_ERR_ARG (ngeo < 1, NULL arrays, a geometry without points,
 * kappa < 0, the errors of defmm_plan_create), DEFMM_ERR_OOM, DEFMM_ERR_CUDA. */
defmm_status defmm_plan_create_union(int ngeo, const double* const* X, const int64_t* nx, const double* kappa,
                                     int order, int leaf_size, const defmm_options* opt, void* stream,
                                     defmm_plan* out);

/* Plan files.  defmm_plan_save writes the plan's host tables (octree,
 * traversal lists, expansions, phase tables, schedules) and the coordinates it
 * was built from to `path`; defmm_plan_load reads such a file and rebuilds the
 * device tables (the transfer spectra are formed again on the GPU), skipping
 * the tree construction, traversals and scheduling.  With the same tuning
 * and shard settings (which are not saved) a loaded plan computes the same
 * results as the saved one, bit for bit.  The format is this
 * library's own (magic "DEFMMPLN", version 2, native byte order, a 64-bit
 * FNV-1a checksum at the end); the paper has no counterpart.  Lengths are
 * checked against the file size and the checksum against the contents, which
 * catches damaged files; a plan file is otherwise trusted input (its tables
 * are indexes the kernels follow), like the library itself.  opt: only flags (DEFMM_PLAN_HOST_ONLY) and hbm_budget
 * apply at load, every other option is the saved plan's.  Tuning and shard
 * settings are not saved.
 * Errors: DEFMM_ERR_ARG (NULL arguments, unreadable, truncated or foreign
 * file, unwritable path), DEFMM_ERR_OOM, DEFMM_ERR_CUDA.                    */
defmm_status defmm_plan_save(defmm_plan plan, const char* path);
defmm_status defmm_plan_load(const char* path, const defmm_options* opt, void* stream, defmm_plan* out);

/* One application phase (Sec. 2.2 operators with M2F/F2L of Sec. 4.1.1):
 * P2M -> M2M -> M2F -> Hadamard M2L with permuted spectra -> F2L -> L2L -> L2P,
 * plus P2P over the near pairs of Alg. 1.
 *  q     - device, ny x nrhs complex charges in the caller's point order.
 *  p     - device, nx x nrhs complex potentials, overwritten.
 *  nrhs  - number of right-hand sides, >= 1.
 *  dtype - DEFMM_C64 (complex float arithmetic) or DEFMM_C128 (complex double).
 *  stream- cudaStream_t; all work is enqueued on it, no host synchronisation.
 * q and p are borrowed for the duration of the stream work.  The first call
 * for a given (nrhs, dtype) may allocate workspace; later calls do not.
 * Errors: DEFMM_ERR_ARG, DEFMM_ERR_OOM, DEFMM_ERR_CUDA, DEFMM_ERR_BUSY.        */
defmm_status defmm_apply(defmm_plan plan, const void* q, void* p, int nrhs,
                         defmm_dtype dtype, void* stream);

/* defmm_apply with host arrays: copies q to the device, applies, copies p back
 * and synchronises the stream before returning.  Page-locked host memory
 * gives asynchronous copies; pageable memory works but is slower.  Returns
 * DEFMM_ERR_TIMEOUT if a bounded device-side wait of the apply gave up.      */
defmm_status defmm_apply_host(defmm_plan plan, const void* q_host, void* p_host, int nrhs,
                              defmm_dtype dtype, void* stream);

/* defmm_apply for callers that cannot allocate device memory when they apply
 * (for example while a stream is captured into a CUDA graph, or when device
 * memory belongs to a pool another component owns).  The paper has no
 * counterpart: it is a property of this library's memory management.
 * The scratch comes from a fixed 64 MiB array linked into the library (held
 * by every GPU that loads it until exit); the call makes no cudaMalloc or
 * cudaFree.  Arguments, layouts and results are those of defmm_apply,
 * bit for bit, including a plan set to one shard (defmm_plan_set_shard).
 *  - Plans whose scratch for nrhs exceeds 64 MiB are rejected with
 *    DEFMM_ERR_UNSUPPORTED (the message gives both sizes).
 *  - The first call on a device looks the array's address up
 *    (cudaGetSymbolAddress); make that first call before any stream capture.
 *  - All calls share the array and it keeps the last call's contents; the
 *    call clears what must start at zero.  Calls whose GPU work overlaps race
 *    on the array: the caller must order them.
 * Errors: DEFMM_ERR_ARG, DEFMM_ERR_UNSUPPORTED, DEFMM_ERR_CUDA, DEFMM_ERR_BUSY. */
defmm_status defmm_apply_noalloc(defmm_plan plan, const void* q, void* p, int nrhs,
                                 defmm_dtype dtype, void* stream);

/* Apply-time tuning of a plan.  The paper has no counterpart: these are
 * launch choices of this library's kernels.
 *  m2l_rhs_block  - right-hand sides that share one pass of the complex64 M2L
 *                   kernel over a staged chunk of spectra and multipoles
 *                   (1, 2 or 4; 0 = the library's choice from nrhs and the
 *                   DFT length).  Values the kernel for the plan's DFT length
 *                   cannot take are lowered (N = 9: at most 2; N > 9: 1).
 *                   No output depends on it (bit for bit).
 *  p2p_tc_min_rhs - complex64 applies with at least this many right-hand
 *                   sides form the near field (Sec. 5.3) as tensor-core
 *                   products, 32 columns per pass, with three tf32 products
 *                   per operand pair (single-precision accuracy); fewer
 *                   columns use the CUDA-core kernel.  0 (the default) never
 *                   uses the tensor cores: with leaves of ~20 targets their
 *                   per-tile overhead makes them slower than the CUDA cores on
 *                   the measured workloads; defmm_plan_autotune times both.
 *                   The two kernels round differently (both within
 *                   single-precision accuracy of the same sum).
 *  m2l_members_per_block - sibling targets per M2L thread block: 4, 8, or by
 *                   group size, 12 or 14 (0 = the library's choice: 14 for
 *                   N = 7 with one column per pass, 4 for N = 9 with one
 *                   column per pass, else 8).  With 4, groups of more siblings
 *                   take two blocks, each staging the group's chunks; smaller
 *                   blocks fit more per SM.  By group size (order 4, N = 7, one
 *                   column per pass) each group runs whole in a block of its
 *                   size class, one launch per class, so few member warps
 *                   idle: 14 = at most 4 siblings in blocks of 4, 5-7 in
 *                   blocks of 7, 8 in blocks of 8; 12 = at most 4 in blocks
 *                   of 4, more in blocks of 8.  Elsewhere 12 and 14 act as 4.
 *                   Kernels without a 4-member variant use 8.
 *                   No output depends on it (bit for bit).
 *  p2p_reduce_phase - 1: the complex64 near field reduces every phase
 *                   kappa r / (2 pi) exactly to [-1/2, 1/2] turns before the
 *                   hardware sine and cosine.  0 (the default): it does so
 *                   only when some near-field phase of the plan may exceed
 *                   90 pi (bounded on the host from the near cell pairs), and
 *                   otherwise gives kappa r to the hardware sine and cosine
 *                   directly (documented to 2^-20.5 absolute error on
 *                   [-100 pi, 100 pi]).  Both are single-precision accurate;
 *                   they round differently.
 * The setting applies to applies enqueued after the call; CUDA graphs
 * captured earlier keep the value they were captured with.
 * Errors: DEFMM_ERR_ARG (NULL plan or tuning, m2l_rhs_block not in
 * {0, 1, 2, 4}, p2p_tc_min_rhs < 0, m2l_members_per_block not in {0, 4, 8, 12, 14},
 * p2p_reduce_phase not 0 or 1). */
typedef struct {
    int m2l_rhs_block;
    int p2p_tc_min_rhs;
    int m2l_members_per_block;
    int p2p_reduce_phase;
} defmm_tuning;

defmm_status defmm_plan_set_tuning(defmm_plan plan, const defmm_tuning* tuning);
defmm_status defmm_plan_get_tuning(defmm_plan plan, defmm_tuning* tuning);

/* Autotuned plan.  The paper sets Ncrit, the order and the FFT length by hand
 * per experiment (Sec. 6); this entry point picks, by timing applies on the
 * caller's geometry, the choices that change only the speed:
 *  - leaf size Ncrit among 16, 24, 32, 48, 64 within [leaf_min, leaf_max]
 *    (leaf_max itself is always a candidate),
 *  - DFT length N among 2p-1 and 2p when opt->fft_n is 0 and tune_fft_n is
 *    set (any N >= 2p-1 gives the same result, Sec. 2.3),
 *  - right-hand sides per M2L pass (1, 2, 4) when nrhs > 1 and complex64,
 *  - the tensor-core near field on or off when nrhs >= 8 and complex64
 *    (defmm_tuning.p2p_tc_min_rhs),
 *  - 8, 4 or by-group-size sibling targets per M2L block for complex64
 *    (defmm_tuning.m2l_members_per_block).
 * A smaller Ncrit changes the tree and so the approximation (within the
 * order's accuracy); the tensor-core near field changes rounding only; the
 * other choices change no result.
 * Each candidate plan is built with defmm_plan_create, applied to a fixed
 * charge block of nrhs columns (device buffers allocated for the call) and
 * timed with CUDA events on `stream` (median of reps applies after two
 * warm-ups).  Candidates over opt->hbm_budget are skipped.  The fastest plan
 * is returned in *out (owned by the caller, free with defmm_destroy) and its
 * choice in *result (may be NULL).
 *  cache_path - NULL, or a text file of earlier choices ("defmm-tune <key>
 *               <leaf> <fft_n> <m2l_rhs_block> <tc> <members> <ms>" lines, key a hash of the
 *               coordinates, sizes, kappa, order, nrhs, dtype, candidate range
 *               and plan options).  A matching line builds the plan with the
 *               stored choice without timing (result->from_cache = 1); after
 *               a tuning run a line is appended.
 * X, nx, Y, ny, kappa, order, opt, stream: as in defmm_plan_create.
 * Errors: those of defmm_plan_create and defmm_apply; DEFMM_ERR_ARG for a bad
 * range, nrhs or reps, or an unwritable cache file; DEFMM_ERR_OOM when no
 * candidate fits; DEFMM_ERR_TIMEOUT if a device-side wait gave up.          */
typedef struct {
    int leaf_min, leaf_max;  /* Ncrit range (default 16..64) */
    int nrhs;                /* columns the plan will be applied to (default 1) */
    defmm_dtype dtype;       /* arithmetic of those applies (default DEFMM_C64) */
    int reps;                /* timed applies per candidate (default 5) */
    int tune_fft_n;          /* also try N = 2p (default 1) */
    const char* cache_path;  /* tune cache file or NULL (default NULL) */
} defmm_tune_options;

typedef struct {
    int leaf_size, fft_n, m2l_rhs_block; /* the choice (fft_n 0: 2p-1) */
    int p2p_tensor_cores;                /* 1: tensor-core near field chosen */
    int m2l_members_per_block;           /* 8, 4, 12, 14 (0 for complex128: the default) */
    double ms;                           /* its median apply time when timed */
    int candidates;                      /* configurations timed (0 from the cache) */
    int from_cache;                      /* 1 if the choice came from cache_path */
} defmm_tune_result;

void defmm_default_tune_options(defmm_tune_options* topt);
defmm_status defmm_plan_autotune(const double* X, int64_t nx, const double* Y, int64_t ny, double kappa,
                                 int order, const defmm_options* opt, const defmm_tune_options* topt,
                                 void* stream, defmm_plan* out, defmm_tune_result* result);

/* The same search for a union plan (defmm_plan_create_union: ngeo
 * geometries, sources = targets): every candidate is a union plan of all the
 * geometries with one leaf size and DFT length, timed as one apply over all
 * of them (nrhs columns of the total point count).  The cache key hashes every
 * geometry's coordinates, point count and wavenumber.  Arguments and errors
 * as defmm_plan_create_union and defmm_plan_autotune.                         */
defmm_status defmm_plan_autotune_union(int ngeo, const double* const* X, const int64_t* nx, const double* kappa,
                                       int order, const defmm_options* opt, const defmm_tune_options* topt,
                                       void* stream, defmm_plan* out, defmm_tune_result* result);

/* Iterative solve with the FMM operator: restarted GMRES (Saad and Schultz,
 * 1986) for (sigma I + A) x = b, A the plan's operator (p = A q).  The paper
 * applies the operator repeatedly inside iterative boundary-integral solvers
 * (Sec. 1, Sec. 7); a shifted single-layer system is the simplest such use.
 *  b, x   - device, n complex values each (n = nx = ny, caller's point order);
 *           x holds the initial guess on entry and the solution on return.
 *  dtype  - DEFMM_C64 or DEFMM_C128: the precision of the applies and of the
 *           Krylov vectors (inner products accumulate in float64).
 *  opt    - NULL for defaults: sigma = 1, tol = 1e-6 (relative residual
 *           ||b - (sigma x + A x)|| / ||b||), restart 30, max_iter 200 applies.
 *  stream - all device work goes to it; the call synchronises it once per
 *           Arnoldi step and returns when done.
 * Every product is one defmm_apply; Arnoldi uses classical Gram-Schmidt twice;
 * the true residual is recomputed at each restart and reported in *result
 * (may be NULL): iterations (applies in the Arnoldi steps), rel_residual,
 * converged (rel_residual <= tol).  Not converging is not an error.
 * Allocates (n x (restart + 1)) complex values of device scratch per call.
 * Errors: DEFMM_ERR_ARG (NULL pointers, nx != ny, restart outside [1, 1000],
 * max_iter < 0, tol < 0), DEFMM_ERR_UNSUPPORTED (dtype, host-only plan, a plan
 * set to one shard by defmm_plan_set_shard),
 * DEFMM_ERR_OOM, DEFMM_ERR_CUDA, DEFMM_ERR_BUSY, DEFMM_ERR_TIMEOUT.          */
typedef struct {
    double shift_re, shift_im; /* sigma */
    double tol;
    int restart;
    int max_iter;
} defmm_gmres_options;

typedef struct {
    int iterations;
    double rel_residual;
    int converged;
} defmm_gmres_result;

void defmm_default_gmres_options(defmm_gmres_options* opt);
defmm_status defmm_gmres(defmm_plan plan, const void* b, void* x, defmm_dtype dtype,
                         const defmm_gmres_options* opt, void* stream, defmm_gmres_result* result);

/* One shard of the operator for a multi-GPU split of one geometry.  The
 * target leaves are cut, in Morton order, into nshards contiguous ranges of
 * about equal estimated work (near-field interactions plus the M2L pairs of
 * each leaf and its ancestors); shard s computes the potentials of its range.
 * The upward pass (P2M, M2M, M2F) is replicated on every shard, M2L and the
 * downward pass run only for target cells that hold targets of the shard
 * (cells on a range boundary are computed by each shard that needs them).
 * The paper's algorithm is single-core (Sec. 6); this split follows its tree.
 *
 * defmm_plan_set_shard makes later defmm_apply / defmm_apply_host calls on
 * this plan compute shard `shard` of `nshards` (nshards = 1: the whole
 * operator, the default): p receives the shard's potentials in the caller's
 * order and zeros elsewhere, so summing the nshards outputs (an all-reduce
 * across GPUs) gives the whole result, bit for bit.  defmm_apply_noalloc
 * follows the setting too; workspace, batch and server applies
 * (defmm_serve.h) always compute the whole operator.  The
 * call synchronises `stream` and the device, builds the shard's tables (one
 * device allocation held by the plan) and returns.
 * defmm_plan_shard_range gives the shard's targets in Morton (sorted) order:
 * positions [first, first + count) of defmm_plan_table(plan, "perm_t", ...);
 * it needs no GPU (host-only plans too).
 * Errors: DEFMM_ERR_ARG (NULL pointers, not 0 <= shard < nshards),
 * DEFMM_ERR_UNSUPPORTED (host-only plan, set_shard), DEFMM_ERR_BUSY,
 * DEFMM_ERR_CUDA.                                                            */
defmm_status defmm_plan_set_shard(defmm_plan plan, int nshards, int shard, void* stream);
defmm_status defmm_plan_shard_range(defmm_plan plan, int nshards, int shard, int64_t* first, int64_t* count);

/* Exchange of a sharded apply by all-gather instead of all-reduce.  Each rank
 * then sends only its own targets' potentials (1/nshards of p) and nothing is
 * summed.  The paper has no multi-GPU step (Sec. 6); the split is the one above.
 *
 * defmm_apply_slice: defmm_apply on the plan's current shard (the whole
 * operator when the plan is not sharded), writing only the shard's count
 * targets (defmm_plan_shard_range), in Morton (sorted) order:
 * slice[r * ld + j] is the potential of sorted target first + j for
 * 0 <= j < count, column r < nrhs; entries j >= count are left untouched.
 * q as in defmm_apply (device, nrhs columns of the caller's ny sources);
 * slice a device buffer of nrhs * ld elements of dtype; ld >= count.  The
 * values are bit for bit those defmm_apply writes for the same targets.
 *
 * defmm_assemble_slices: p (device, nrhs columns of the caller's nx targets,
 * as defmm_apply writes it) from the slices of all nshards shards, stored one
 * after another in `slices` (device): shard s's slice at element offset
 * s * nrhs * ld, laid out as defmm_apply_slice writes it.  starts (host,
 * nshards + 1 entries) are the shards' sorted-target boundaries:
 * starts[s] = first of shard s, starts[nshards] = nx, so
 * starts[s + 1] - starts[s] = count of shard s <= ld.  Every target of p is
 * written once; the result equals the whole operator's defmm_apply bit for bit.
 * Both calls only enqueue work on `stream`; the caller owns every buffer.
 * Errors: DEFMM_ERR_ARG (NULL pointers, nrhs < 1, ld below a shard's count,
 * starts not from 0 to nx or decreasing), DEFMM_ERR_UNSUPPORTED (dtype,
 * host-only plan), DEFMM_ERR_BUSY, DEFMM_ERR_OOM (workspace, as defmm_apply),
 * DEFMM_ERR_CUDA.                                                            */
defmm_status defmm_apply_slice(defmm_plan plan, const void* q, void* slice, int64_t ld, int nrhs, defmm_dtype dtype,
                               void* stream);
defmm_status defmm_assemble_slices(defmm_plan plan, int nshards, const int64_t* starts, const void* slices,
                                   int64_t ld, void* p, int nrhs, defmm_dtype dtype, void* stream);

/* Frees the plan and its device memory (synchronises the device first).       */
defmm_status defmm_destroy(defmm_plan plan);

typedef struct {
    int64_t nx, ny;
    int32_t order, fft_n;
    int32_t nlevels;         /* octree levels (target tree) */
    int32_t deepest_hf;      /* deepest high-frequency level, -1 if none */
    int64_t ncells_t, ncells_s;
    int64_t n_m2l_pairs, n_p2p_pairs;
    int64_t n_multipole, n_local;     /* effective expansions (Sec. 4.2.3) */
    int64_t n_fourier;                /* multipoles transformed by M2F */
    int64_t n_spectra;                /* canonical spectra stored (Sec. 4.3) */
    int64_t p2p_interactions;         /* sum over near pairs of n_t * n_s */
    size_t plan_bytes;                /* device bytes held by the plan tables */
    size_t workspace_bytes;           /* device bytes of the current workspace */
    int64_t launches_per_apply;       /* kernels launched by the last apply (0 before any) */
    int64_t device_error;             /* 1 if a bounded device-side wait of an apply gave up,
                                         2 if a table index was out of range (only a
                                         bounds-checked build, DEFMM_CHECKED, tests them)
                                         (that apply's results are invalid); this call
                                         synchronises with the device to read it */
    double d_aabb;                    /* side of the smallest box holding X, Y */
    double cube_side;                 /* side of the octree root */
    /* plan creation time (ms): the trees, the dual tree traversal, the best
       directions and the Alg. 2 marks, built on the device (device time from
       CUDA events, and the wall time of that step with its copies); the rest
       of the construction on the host; the upload of the tables with the
       spectra formed on the device.  Host-only plans build everything on the
       host (front times 0).                                                  */
    double plan_front_device_ms, plan_front_ms, plan_host_ms, plan_upload_ms;
} defmm_info;

defmm_status defmm_plan_info(defmm_plan plan, defmm_info* out);

/* Integer plan tables, for testing a plan against an independent build.
 * name: "perm_t", "perm_s" (sorted position -> input index),
 *       "cells_t", "cells_s" (per cell: level, ix, iy, iz, begin, end, parent),
 *       "m2l" (per pair: target cell, source cell, best direction or -1),
 *       "p2p" (per pair: target cell, source cell),
 *       "mult", "local" (per effective expansion: cell, direction or -1),
 *       "m2f_list" (Fourier-multipole slot -> multipole expansion id),
 *       "spectra" (per canonical spectrum: level, kbar x, y, z),
 *       the M2L schedule: "grp_member_off", "grp_members" (CSR: group ->
 *       local expansion ids), "grp_chunk_off" (CSR: group -> chunks),
 *       "chk_blk_off", "chk_nspec", "chk_blk" (CSR: chunk -> staged blocks,
 *       its first chk_nspec are spectrum ids, the rest Fourier-multipole
 *       slots), "chk_op_off" (9 per chunk: op ranges of members 0..7, end),
 *       "chk_op" (spectrum block | multipole block << 8 | symmetry code << 16;
 *       code bit a negates axis a, code >> 3 names the axis permutation),
 *       the near-field work units: "p2p_leaf" (near-field target leaf cells),
 *       "p2p_unit_leaf" (unit -> index into p2p_leaf), "p2p_unit_off" (CSR:
 *       unit -> source ranges), "p2p_unit_ranges" (per range: first, end
 *       sorted source position).
 * Copies min(count, capacity) int64 values to out (host) and sets *count to
 * the full length.  out may be NULL to query the length.                    */
defmm_status defmm_plan_table(defmm_plan plan, const char* name, int64_t* out,
                              int64_t capacity, int64_t* count);

/* Per-phase timing of the application phase, with CUDA events recorded on the
 * apply's own stream between its kernel groups.  enable = 1 turns recording on
 * for later defmm_apply calls on this plan (0 turns it off).  Phases, in
 * order: gather, p2p, p2m, m2m, m2f, m2l (Hadamard + F2L), l2l, l2p, scatter.
 * defmm_profile_read waits for the last profiled apply and writes up to
 * capacity phase durations in milliseconds to ms (host) and their number to
 * *nphase.  Errors: DEFMM_ERR_ARG (no profiled apply yet), DEFMM_ERR_CUDA.   */
defmm_status defmm_profile_enable(defmm_plan plan, int enable);
defmm_status defmm_profile_read(defmm_plan plan, double* ms, int capacity, int* nphase);

/* Self-test of the failure path every pipelined kernel uses (no counterpart
 * in the paper): one thread block waits on an mbarrier phase that nothing
 * completes, polls at most `spins` times, raises a device flag and returns,
 * as the M2L and tensor-core kernels do when a copy never lands (they then
 * raise the plan's flag, read by defmm_plan_info().device_error and reported
 * as DEFMM_ERR_TIMEOUT by defmm_apply_host).  Nothing faults or hangs and the
 * context stays usable.  Returns DEFMM_ERR_TIMEOUT when the flag was raised
 * (the expected outcome), DEFMM_OK otherwise.
 * Errors: DEFMM_ERR_ARG (spins outside [1, 2^22]), DEFMM_ERR_CUDA.           */
defmm_status defmm_selftest_bounded_wait(int spins, void* stream);

const char* defmm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DEFMM_H */
