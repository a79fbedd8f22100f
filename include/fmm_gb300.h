/*
 * fmm_gb300.h -- C-ABI of the GB300 Cartesian fast multipole library for the
 * 1/r kernel (Coles & Bieri, "An Optimizing Symbolic Algebra Approach for
 * Generating Fast Multipole Method Operators", arXiv:1811.06332).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Multi-indices follow App. D: n = (nx,ny,nz), |n| = nx+ny+nz,
 *    n! = nx!ny!nz!, r^n = x^nx y^ny z^nz.
 *  - Coefficient storage (App. A compressed form; App. E table of sizes):
 *      FMM_BASIS_SYM        C(p+3,3) components, ranks 0..p concatenated,
 *                           inside a rank descending nx then descending ny;
 *      FMM_BASIS_TRACELESS  (p+1)^2 independent components (nz <= 1) per
 *                           polytensor, inside rank j ordered
 *                           (j,0,0),(j-1,1,0),...,(0,j,0),(j-1,0,1),...,(0,j-1,1);
 *                           dependent components follow from the trace
 *                           condition A_{k+2ez} = -A_{k+2ex} - A_{k+2ey}
 *                           (App. B).
 *    fmm_ncoef(p, basis) returns the count.
 *  - Batched arrays are structure-of-arrays, coefficient-major:
 *    element (c, i) of an [ncoef][n] array lives at index c*n + i.
 *    Vectors are [3][n]: x components, then y, then z.
 *  - Normalisation of Sec. 2.1: M_n = sum_a q_a (-r_a)^n, M2L weights 1/m!,
 *    L2L weights delta^k/k!, L2P reads L at the particle.
 *  - Potentials and accelerations returned by fmm_l2p/fmm_p2p/fmm_evaluate
 *    use the astrophysical sign that Sec. 2.1 prescribes for gravity:
 *    pot_i = -sum_{j!=i} q_j/|x_i - x_j|,
 *    acc_i = sum_{j!=i} q_j (x_j - x_i)/|x_i - x_j|^3  (= +grad Phi of the paper).
 *    fmm_op_l2p returns the paper's own positive Phi and grad Phi.
 *  - Pointers: every array argument is a DEVICE pointer unless the entry
 *    point's name ends in _host.  The caller owns its inputs and outputs; a
 *    plan owns everything it allocates.  Work is queued on `stream` (a
 *    cudaStream_t passed as void*, NULL = legacy default stream) and is
 *    asynchronous unless stated otherwise.
 *  - Errors: every int-returning call returns an fmm_status.  Arguments are
 *    validated before any launch; nothing is thrown across the ABI.  The
 *    text of the last error is returned by fmm_last_error(plan), or by
 *    fmm_last_error(NULL) for the plan-less operator calls (thread-local).
 *  - Threading: a plan is used by one host thread at a time.
 */
#ifndef FMM_GB300_H
#define FMM_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FMM_OK = 0,
    FMM_ERR_ARG = -1,         /* invalid argument (size, pointer, p, basis) */
    FMM_ERR_CUDA = -2,        /* a CUDA call failed; see fmm_last_error     */
    FMM_ERR_OOM = -3,         /* device allocation failed                   */
    FMM_ERR_STATE = -4,       /* call made before fmm_build_tree            */
    FMM_ERR_TIMEOUT = -5,     /* a bounded device wait gave up              */
    FMM_ERR_UNSUPPORTED = -6  /* valid but not implemented combination      */
} fmm_status;

/* FMM_BASIS_TG (plans only; uniform octree, FMM_FP64): the paper's TG
 * variant (Sec. 3), multipoles in full symmetric storage (P2M and M2M
 * without a detracer), M2L from them to traceless local expansions (D is
 * traceless, so is L), L2L and L2P on traceless storage. */
typedef enum { FMM_BASIS_SYM = 0, FMM_BASIS_TRACELESS = 1, FMM_BASIS_TG = 2 } fmm_basis;

typedef enum {
    FMM_FP64 = 0,        /* every operator in FP64                                     */
    FMM_FP32 = 1,        /* operator arithmetic in FP32 (uniform trees: P2M, M2L, L2P,
                            P2P and, for p <= 8, M2M and L2L; adaptive trees: every
                            operator); tree geometry, D-tensor tables and every stored
                            expansion in FP64                                            */
    FMM_GEMM_TF32X3 = 2, /* as FMM_FP32, but M2L of the uniform levels >= 5 (class grids of
                            16+ cells per axis) as offset-grouped tensor-core GEMMs with
                            TF32 hi/lo operands, 3 products, FP32 accumulation; traceless
                            basis, p <= 8, uniform trees                                  */
    FMM_GEMM_BF16X3 = 3  /* the same with BF16 hi/lo operands                            */
} fmm_precision;

typedef struct {
    int p;                 /* expansion order, 0..10 (Eq. phi expansion, App. B)      */
    int basis;             /* fmm_basis                                                */
    int prec;              /* fmm_precision                                            */
    int adaptive;          /* 0: uniform octree of depth `depth` over [0,1)^3;
                              1: adaptive octree over the bounding cube of the data,
                              cells split while they hold more than max_leaf
                              particles, lists from a dual-tree traversal (App. C) */
    int depth;             /* uniform octree depth (leaves = 8^depth), 0..9            */
    int max_leaf;          /* adaptive trees: maximum particles per leaf               */
    double theta;          /* adaptive trees: opening parameter of the MAC (App. C)    */
    int learned_p;         /* adaptive trees, FMM_BASIS_SYM, 4 <= p <= 10: 1 gives every
                              M2L pair its own order in 0..p (chosen by the model set
                              with fmm_set_mlp, or given by fmm_set_pair_orders); p is
                              the order of every other operator and of the storage   */
    double target_rel_err; /* learned_p: the model picks, per pair, the lowest order
                              whose predicted error is at most
                              target_rel_err * kappa / sqrt(K_B), kappa stored with
                              the model, K_B the number of M2L pairs of the target
                              and its ancestors (errors of independent pairs add in
                              quadrature at a target)                                  */
    int use_graph;         /* 1 (non-default stream): adaptive trees capture the
                              operator sequence P2M..P2P of fmm_evaluate into a CUDA
                              graph after the first evaluation and replay it while
                              the tree keeps its sizes and buffers; uniform octrees
                              capture the whole step (tree and operators) at the
                              second evaluation and replay it while n, the input and
                              output arrays and the tensor-core kernel shape stay the
                              same                                                     */
    int autotune;          /* tensor-core forms: 1 takes the kernel shape stored for
                              this GPU, p, basis, form and depth in the tuning cache
                              (the JSON file FMM_TUNE_CACHE, else
                              $XDG_CACHE_HOME/fmm_gb300/tune.json, else
                              $HOME/.cache/fmm_gb300/tune.json); without an entry,
                              the first M2L that reaches a tensor-core level times
                              every candidate shape on the deepest level, keeps the
                              fastest and stores it.  0: the default shape          */
    int ap;                /* 1: the AP variant of Sec. 3 (astrophysics): adaptive tree,
                              traceless basis, FMM_FP64; expansion centres at the
                              centres of mass (summed bottom-up: a leaf over its
                              particles in sorted order, a cell over its children's
                              charge-weighted centres; a cell of zero charge keeps its
                              geometric centre), radii and MAC about them, the dipole
                              of every multipole set to 0 (it vanishes about the
                              centre of mass), and only the gradient evaluated: the
                              accelerations are written, pot is written as 0       */
    int binary_tree;       /* 1 (adaptive, FMM_FP64, not ap, not learned_p): the binary
                              median-split tree of App. C instead of the octree: a
                              cell of more than max_leaf particles is halved across
                              the longest side of its particles' bounding box (the
                              lower floor(n/2) by that coordinate, equal coordinates
                              by original index; the first of x, y, z when sides
                              tie), cells
                              shrink-wrapped and centred on their bounding boxes;
                              the same traversal, MAC and operators as the octree  */
} fmm_config;

typedef struct fmm_plan fmm_plan;

/* Number of stored coefficients of an order-p polytensor: C(p+3,3) for
 * FMM_BASIS_SYM, (p+1)^2 for FMM_BASIS_TRACELESS (App. E table).  Returns
 * FMM_ERR_ARG for p outside 0..10 or an unknown basis. */
int fmm_ncoef(int p, int basis);

/* ---------------------------------------------------------------------------
 * Plan-based FMM (App. C): tree, upward pass, interaction phase, downward
 * pass, near field.  Uniform octree over the unit cube: a particle belongs to
 * leaf i_d = min(floor(x_d 2^depth), 2^depth - 1) (coordinates outside
 * [0,1) are clamped into the boundary leaves); expansion centres are cell
 * centres (App. C); same-level cells at Chebyshev index distance >= 2 are
 * well separated, M2L runs over the children of the parent's neighbours
 * that are not adjacent (levels 2..depth) and adjacent leaves are summed
 * directly.
 * ------------------------------------------------------------------------- */

/* Creates a plan.  Validates cfg (p in 0..10, basis, prec, depth in 0..9;
 * adaptive plans: max_leaf >= 1, 0 <= theta <= 1, prec FMM_FP64 or
 * FMM_FP32; the tensor-core form needs the traceless basis and p <= 8) and
 * returns FMM_ERR_ARG / FMM_ERR_UNSUPPORTED otherwise.
 * *out receives the plan (NULL on failure).  Allocates no particle storage. */
int fmm_create(const fmm_config* cfg, fmm_plan** out);

/* Destroys a plan and frees everything it owns.  NULL is ignored.  The
 * caller must make sure no work of the plan is still running. */
void fmm_destroy(fmm_plan* plan);

/* Text of the last error of `plan` (or of the calling thread's last
 * plan-less call when plan == NULL).  Valid until the next call. */
const char* fmm_last_error(const fmm_plan* plan);

/* Sorts the n particles (device arrays x, y, z, q of length n, caller order)
 * into the leaves of the octree, stably by original index, and prepares the
 * interaction lists (App. C).  The plan keeps its own sorted copies; the
 * caller's arrays may be reused once the stream reaches this point.
 * n may be 0.  (Re)allocates plan storage when n or the tree changes. */
int fmm_build_tree(fmm_plan* plan, int64_t n, const double* x, const double* y,
                   const double* z, const double* q, void* stream);

/* P2M at every leaf (Eq. P2M, Sec. 2.1) about the leaf centre. */
int fmm_p2m(fmm_plan* plan, void* stream);
/* M2M bottom-up (Eq. M2M / M2M part 2, Sec. 2.1), delta = z_child - z_parent. */
int fmm_m2m(fmm_plan* plan, void* stream);
/* M2L over the interaction lists of levels 2..depth (Eq. M2L, Sec. 2.1),
 * r = z_target - z_source, in the plan's precision form. */
int fmm_m2l(fmm_plan* plan, void* stream);
/* M2L of the uniform levels lmin..lmax only (clamped to 2..depth; Eq. M2L,
 * Sec. 2.1).  Levels are independent, so calling it on disjoint ranges that
 * cover 2..depth computes what fmm_m2l computes (used to time the
 * tensor-core levels apart from the rest).  Adaptive plans:
 * FMM_ERR_UNSUPPORTED; lmin > lmax: FMM_ERR_ARG; before fmm_build_tree:
 * FMM_ERR_STATE. */
int fmm_m2l_levels(fmm_plan* plan, int lmin, int lmax, void* stream);
/* L2L top-down (Eq. L2L, Sec. 2.1), delta = z_child - z_parent. */
int fmm_l2l(fmm_plan* plan, void* stream);
/* L2P (Eq. L2P, Sec. 2.1): OVERWRITES pot, ax, ay, az (device, length n,
 * caller order) with the far-field potential and acceleration. */
int fmm_l2p(fmm_plan* plan, double* pot, double* ax, double* ay, double* az, void* stream);
/* Near field (App. C direct sum over adjacent leaves, self excluded):
 * ADDS into pot, ax, ay, az (device, length n, caller order). */
int fmm_p2p(fmm_plan* plan, double* pot, double* ax, double* ay, double* az, void* stream);
/* L2P followed by P2P in one pass: writes (does not add) pot and acc of
 * every particle with the far field of its leaf's local expansion and the
 * near field of its adjacent leaves.  The result is that of fmm_l2p then
 * fmm_p2p; plans of the FP32 and tensor-core forms on a uniform octree run
 * one kernel (each output written once), the others run the two steps. */
int fmm_l2p_p2p(fmm_plan* plan, double* pot, double* ax, double* ay, double* az, void* stream);

/* fmm_build_tree + p2m + m2m + m2l + l2l + l2p + p2p on `stream`.
 * All arrays are device arrays of length n in caller order; outputs are
 * overwritten.  With cfg.use_graph the sequence is captured into a CUDA
 * graph on the first call for a given (n, input/output pointers) and
 * replayed afterwards. */
int fmm_evaluate(fmm_plan* plan, int64_t n, const double* x, const double* y,
                 const double* z, const double* q, double* pot, double* ax,
                 double* ay, double* az, void* stream);

/* fmm_evaluate with point dipoles (App. B, "Dipoles and higher order
 * multipoles") beside the charges: particle i carries the charge q[i] and
 * the dipole moment (px[i], py[i], pz[i]) (device arrays, caller order; use
 * zeros for either).  A point dipole p at x_a acts as the limit of charges
 * +q at x_a + s and -q at x_a - s with p = 2 q s: P2M adds the pure dipole
 * M_{e_i} = -p_i shifted by M2M from x_a to the leaf centre, the near field
 * adds the dipole field (potential p.d/|d|^3, d = x - x_a), and M2M, M2L,
 * L2L, L2P are unchanged.  Outputs as fmm_evaluate (pot = -Phi, acc =
 * grad Phi).  Uniform plans in FMM_FP64 (either basis); others return
 * FMM_ERR_UNSUPPORTED. */
int fmm_evaluate_dipoles(fmm_plan* plan, int64_t n, const double* x, const double* y,
                         const double* z, const double* q, const double* px, const double* py,
                         const double* pz, double* pot, double* ax, double* ay, double* az,
                         void* stream);

/* fmm_evaluate on HOST arrays (length n, caller order): copies the inputs to
 * the device, evaluates, copies the outputs back and waits for the stream;
 * returns fmm_sync_status's verdict.
 * Uses plan-owned staging buffers; page-locked host memory gives full copy
 * speed but is not required.  Synchronous. */
int fmm_evaluate_host(fmm_plan* plan, int64_t n, const double* x, const double* y,
                      const double* z, const double* q, double* pot, double* ax,
                      double* ay, double* az, void* stream);

/* Waits for `stream`, then reports whether a bounded wait inside one of the
 * plan's tensor-core kernels (the M2L of the tensor-core forms, the order
 * model's inference of learned_p plans) gave up since the previous check:
 * FMM_ERR_TIMEOUT if so (the outputs of the work queued since that check are
 * undefined; the report clears the plan's device error word), FMM_OK
 * otherwise.  The queueing calls (fmm_m2l, fmm_evaluate, ...) return before
 * their kernels run and cannot see such a timeout; fmm_evaluate_host calls
 * this before it returns.  Synchronous. */
int fmm_sync_status(fmm_plan* plan, void* stream);

/* Self-test of the bounded waits of the tensor-core kernels (no counterpart
 * in the paper): one kernel waits, with the kernels' own bounded wait, on
 * an mbarrier that expects one arrival.  arrive != 0: the kernel arrives
 * first and the wait completes (FMM_OK).  arrive == 0: nothing arrives, the
 * wait gives up after `spin` polls, records its code in an error word and
 * the kernel returns; the call reports FMM_ERR_TIMEOUT and the context stays
 * usable.  FMM_ERR_ARG for spin < 1.  Synchronous on `stream`. */
int fmm_selftest_wait(int64_t spin, int arrive, void* stream);

/* ---------------------------------------------------------------------------
 * Operator-level batched entry points (independent items, physical units).
 * ------------------------------------------------------------------------- */

/* D-tensor D_k(r) = grad^k |r|^{-1} for all |k| <= p (Eq. traceless grad,
 * App. A).  r: [3][n] doubles, nonzero.  basis FMM_BASIS_SYM: D is
 * [C(p+3,3)][n] in full symmetric storage; FMM_BASIS_TRACELESS: D is
 * [(p+1)^2][n], the independent components (nz <= 1) of the traceless
 * storage (D is trace free, so they determine it).  Elements are doubles
 * (prec FMM_FP64) or floats (FMM_FP32, computed in FP32). */
int fmm_op_dtensor(int p, int basis, int prec, int64_t n, const double* r, void* D, void* stream);

/* P2M (Eq. P2M, Sec. 2.1; traceless: Mbar = D[M] per rank, Eq. Detracer of
 * App. A) for ncell particle groups: particles of group c are
 * start[c] .. start[c+1]-1 of x, y, z, q (device, doubles); start is an
 * int64 device array of ncell+1 nondecreasing offsets; centre: [3][ncell];
 * M: [ncoef][ncell] doubles, OVERWRITTEN. */
int fmm_op_p2m(int p, int basis, int64_t ncell, const int64_t* start, const double* x,
               const double* y, const double* z, const double* q, const double* centre,
               double* M, void* stream);

/* M2M (Eq. M2M / M2M part 2, Sec. 2.1): Mp[:,i] += shift of Mc[:,i] by
 * delta[:,i] = z_child - z_parent (traceless: followed by D[]).  Mc, Mp:
 * [ncoef][n] (distinct arrays) of doubles (prec FMM_FP64) or floats
 * (FMM_FP32, computed in FP32); delta: [3][n] doubles. */
int fmm_op_m2m(int p, int basis, int prec, int64_t n, const void* Mc, const double* delta,
               void* Mp, void* stream);

/* M2L (Eq. M2L, Sec. 2.1) for n independent pairs with the D-tensor computed
 * on the fly: L[:,i] (+)= sum_{|m|<=p-|n|} M_m[:,i]/m! D_{n+m}(r[:,i]).
 * prec FMM_FP64: M, L are doubles; FMM_FP32: floats.  r: [3][n] doubles,
 * r = z_target - z_source, nonzero.  accumulate = 0 overwrites L. */
int fmm_op_m2l(int p, int basis, int prec, int64_t n, const void* M, const double* r,
               void* L, int accumulate, void* stream);

/* M2M of traceless multipoles in the fused form of Eq. Detracer2 (Sec. 2.1):
 * the shift inserted into the detracer and regrouped by multipole
 * component, evaluated from a table of (coefficient, component, power)
 * terms built once per order.  Mp[:,i] += shifted Mc[:,i], delta[:,i] =
 * z_child - z_parent; Mc, Mp: [(p+1)^2][n] doubles in traceless storage
 * (distinct arrays); delta: [3][n].  Computes what fmm_op_m2m computes for
 * FMM_BASIS_TRACELESS, FMM_FP64.  The first call for an order on a device
 * allocates and uploads its table (synchronous). */
int fmm_op_m2m_fused(int p, int64_t n, const double* Mc, const double* delta, double* Mp,
                     void* stream);
/* Number of terms of the fused M2M table of order p (no GPU needed), or
 * FMM_ERR_ARG. */
int fmm_m2m_fused_terms(int p);

/* L2L (Eq. L2L, Sec. 2.1): Lc[:,i] += shift of Lp[:,i] by
 * delta[:,i] = z_child - z_parent.  Lp, Lc: [ncoef][n] (distinct arrays) of
 * doubles (prec FMM_FP64) or floats (FMM_FP32, computed in FP32); delta:
 * [3][n] doubles. */
int fmm_op_l2l(int p, int basis, int prec, int64_t n, const void* Lp, const double* delta,
               void* Lc, void* stream);

/* L2P (Eq. L2P, Sec. 2.1): out[0][i] = Phi, out[1..3][i] = grad Phi at
 * offset rb[:,i] from the expansion centre (the paper's positive sign).
 * L: [ncoef][n] and out: [4][n] (OVERWRITTEN) of doubles (prec FMM_FP64) or
 * floats (FMM_FP32, computed in FP32); rb: [3][n] doubles. */
int fmm_op_l2p(int p, int basis, int prec, int64_t n, const void* L, const double* rb,
               void* out, void* stream);

/* FP64 direct sum (Eq. PhiAB, App. B) of all n sources onto nt targets
 * (indices into the sources, int64 device array; NULL = all n, nt ignored),
 * with the astrophysical sign convention above.  Outputs have nt entries. */
int fmm_direct(int64_t n, const double* x, const double* y, const double* z,
               const double* q, int64_t nt, const int64_t* targets, double* pot,
               double* ax, double* ay, double* az, void* stream);

/* ---------------------------------------------------------------------------
 * No-allocation evaluation.  The paper has no counterpart to this entry
 * point; it exists for callers that must not allocate device memory --
 * applications that hand all device memory to their own pool allocator up
 * front, or that cannot afford the device-wide synchronisation which
 * cudaMalloc/cudaFree may cause in the middle of a time step.
 *
 * fmm_evaluate_noalloc runs the kernels that fmm_evaluate runs for a plan
 * with {p, basis, FMM_FP64, uniform octree of depth `depth`}, in the same
 * order, and its results agree with that plan's to within 1e-12 relative;
 * but it allocates nothing: no cudaMalloc, no cudaFree, no allocating
 * library routine.  Its working memory (sorted particles, leaf
 * ranges, tree-build counters, expansions, translation matrices, tables) is
 * one fixed __device__ array of FMM_NOALLOC_BYTES_APPROX bytes that every GPU
 * which loads this library holds until the process exits.  Limits:
 * 0 <= n <= FMM_NOALLOC_MAX_N, 0 <= p <= FMM_NOALLOC_MAX_P,
 * 0 <= depth <= FMM_NOALLOC_MAX_DEPTH; larger sizes return FMM_ERR_ARG with
 * a message, before any work is queued.  x, y, z, q, pot, ax, ay, az are
 * device arrays of length n in caller order (outputs overwritten).
 *
 * The first call on a device does the set-up (uploads constant tables into
 * the array; synchronous), and a call whose (p, basis) differs from the
 * previous call's on that device rebuilds the translation matrices and the
 * D-tensor table held in the array (synchronous).  Make the first call
 * before any stream capture.  A call that needs the set-up or a rebuild
 * while its stream is being captured returns FMM_ERR_STATE and queues
 * nothing.  The array's device address is looked up on every call, and a
 * changed address repeats the set-up; calling cudaDeviceReset between calls
 * is not supported.  Every call on a device shares the one array and
 * overwrites what the previous call left there; calls that overlap on the
 * GPU (different streams or threads without ordering between them) race and
 * corrupt each other's results.  Errors: fmm_last_error(NULL). */
#define FMM_NOALLOC_MAX_N 65536
#define FMM_NOALLOC_MAX_DEPTH 3
#define FMM_NOALLOC_MAX_P 6
#define FMM_NOALLOC_BYTES_APPROX 7540000
int fmm_evaluate_noalloc(int p, int basis, int depth, int64_t n, const double* x, const double* y,
                         const double* z, const double* q, double* pot, double* ax, double* ay,
                         double* az, void* stream);

/* Sizes of the plan's tree and lists after fmm_build_tree, written to
 * out[0..min(nout,19)): number of cells, leaves, M2L pairs, P2P (leaf) pairs,
 * M2L target cells, autotuned M2L blocks per SM (0 before the first M2L),
 * tree levels, 1 when a captured operator graph is held, then (learned_p
 * plans, after an M2L) the number of M2L pairs at each order 0..10.  For
 * uniform trees the list entries are 0 (the lists are implicit). */
int fmm_plan_stats(const fmm_plan* plan, int64_t* out, int nout);

/* Host-side layout of the TF32 form's tensor-core M2L kernel, the one that
 * streams each offset's precomputed matrix (no GPU needed; for diagnostics
 * and tests), for order p (1..8, traceless) and prec FMM_GEMM_TF32X3,
 * written to out[0..min(nout,42)):
 * N-chunk width cw, chunks nch, K-parts per offset np, matrix stages nbst,
 * MMA-issuing warps niss, bytes of a matrix stage, bytes of one offset's
 * packed matrix, dynamic shared bytes per CTA, then K-steps per chunk
 * kch[6], K-steps per part and chunk nk[2][6], byte offsets of the chunks in
 * a part's block boff[2][6], bytes of a part's block (hi or lo) pbytes[2],
 * byte offsets of the parts poff[2].  The chunk width follows the
 * FMM_TC_CHUNK environment variable as the kernel does.  Returns the count
 * written, or FMM_ERR_ARG. */
int fmm_tc_layout(int p, int prec, int* out, int nout);

/* Host-side layout of the BF16 form's tensor-core M2L kernel, which builds
 * each offset's matrix B_o(n, m) = D_{n+m}(-o) in shared memory from the
 * offset's D vector (no GPU needed; for diagnostics and tests), for order p
 * (1..8), chunk width cw (16, 32, 48 or 96 local rows; the hi and lo rows of
 * a chunk are stacked into one MMA of N = 2 cw) and niss (1 or 2)
 * MMA-issuing warps, written to out[0..min(nout,19)): cw, chunks nch, bytes
 * of a matrix stage, stages nb, niss, nonzero 16-byte groups of a matrix
 * ngroups, dynamic shared bytes per CTA, K-steps per chunk kch[6], byte
 * offsets of the chunks in a stage coff[6].  When gcap > 0, groups receives
 * up to gcap words of the group table, 4 per group: the symmetric storage
 * positions of n + m for its 8 multipole columns m (one byte each, 255 where
 * |n| + |m| > p), then the byte offsets of its hi and lo 16 bytes in a
 * stage.  Returns the count written to out, or FMM_ERR_ARG. */
int fmm_tc_gen_layout(int p, int cw, int niss, int* out, int nout, uint32_t* groups, int gcap);

/* Kernel shape of a tensor-core plan's M2L (Eq. M2L regrouped by offset).
 * kernel 0: each offset's matrix precomputed in global memory and streamed
 * into shared memory (BF16 or TF32 operands); kernel 1: each offset's matrix
 * built in shared memory from the offset's D vector (BF16 operands only);
 * kernel 2: the matrix as the A operand (M = 128 local components) and the
 * target cells of a tile as N (256 cells on levels >= 6, 128 on level 5),
 * BF16 operands only; kernel 3: kernel 2 with the multipole columns 0..47
 * on the tensor cores, then the columns >= 48 (which reach only the local
 * rows of rank <= p - 6) as FP32 products on the CUDA cores, added to L
 * (p = 6..8; the same as kernel 2 below p = 6).
 * cw: chunk width, the local components per MMA (16, 32, 48 or 96) for
 * kernels 0 and 1; 256 for kernels 2 and 3.
 * fmm_set_tc_shape fixes the shape (rebuilding the plan's offset tables;
 * synchronous); FMM_ERR_ARG for a shape the plan's form has not.
 * fmm_plan_tuning writes to out[0..min(nout, 5 + 4 ncand)): kernel, cw,
 * MMA-issuing warps, how the shape was chosen (0 default, 1 autotuned in
 * this plan, 2 read from the tuning cache, 3 set by fmm_set_tc_shape),
 * ncand, then per autotuner candidate kernel, cw, issuing warps and its
 * time on the deepest level in microseconds.  Returns the count written. */
int fmm_set_tc_shape(fmm_plan* plan, int kernel, int cw);
int fmm_plan_tuning(const fmm_plan* plan, int* out, int nout);

/* The tuning cache itself (host only; for tools and tests): a JSON object
 * {"<key>": {"kernel": k, "cw": c, "niss": n, "ms": t}, ...} in the file
 * `path`.  fmm_tune_cache_get writes vals[0..3) = {kernel, cw, niss} of
 * `key` and returns 1, or returns 0 when the file or the entry is missing
 * or malformed.  fmm_tune_cache_put stores vals[0..3) and ms under `key`
 * (replacing an earlier entry, creating the file's directories) and returns
 * FMM_OK, or FMM_ERR_STATE when the file cannot be written.  A plan's key
 * is "<GPU name>|p=<p>|basis=<basis>|prec=<prec>|depth=<depth>". */
int fmm_tune_cache_get(const char* path, const char* key, int* vals);
int fmm_tune_cache_put(const char* path, const char* key, const int* vals, double ms);

/* Number of kernels this library launched since it was loaded (all plans and
 * operator calls), counted on the host at each launch. */
int64_t fmm_kernel_launches(void);

/* ---------------------------------------------------------------------------
 * Learned per-pair M2L order.  The paper fixes one order p per run; these
 * calls add a model that picks an order for every M2L pair of an adaptive
 * tree from 12 features of the pair, so that pairs far inside the MAC use
 * fewer terms of Eq. M2L than pairs near its boundary.
 *
 * Features of a pair (source A, target B, d = z_B - z_A, radii r, particle
 * counts n, full symmetric multipoles M):
 *   a = max(r_A/|d|, 1e-6), b = max(r_B/|d|, 1e-6); f0 = ln(a+b) (the MAC
 *   ratio, App. C), f1 = ln a, f2 = ln b; f3..f6 = ln max(|M_A^(j)| /
 *   (|M_A,0| r_A^j), 1e-6) for j = 1..4 with |M^(j)|^2 = sum_{|m|=j} j!/m!
 *   M_m^2; f7, f8 = the same for M_B, j = 1, 2; f9 = ln min(n_A, 1024);
 *   f10 = ln min(n_B, 1024);
 *   f11 = ln max(g_AB / T_B, 1e-12), the pair's share of a far-field
 *   magnitude estimate: g_AB = |M_A,0| / |d|^2, T_B = the sum of g over the
 *   M2L lists of B and of all its ancestors.
 * Label of a pair at order q (q = 2..10): log10 max(e_q, 1e-12), e_q the
 * force error of the pair's order-q M2L + L2P (Eqs. M2L, L2P) at up to 64
 * particles of B (all when n_B <= 64, else sorted positions
 * b_B + floor(j n_B / 64)) against the direct sum over A's particles,
 * relative to the total force at those particles (direct sum over all
 * particles): sqrt(sum |g_q - g|^2 / sum |a|^2).
 *
 * Model: 12 -> 64 -> 64 -> 64 -> 9, ReLU; predicted log10 error at orders
 * 2..10.  Parameter blob (FMM_MLP_NBLOB floats): [0..8) header {6332, 2,
 * 12, 64, 9, 2, log10 kappa, 0}, [8..20) feature means, [20..32) feature
 * standard deviations, then W1 (64x12 row-major), b1, W2 (64x64), b2, W3,
 * b3, W4 (9x64), b4.  Inference rounds weights and the input of every layer
 * to BF16 (nearest even) and accumulates in FP32 on the tensor cores.
 * ------------------------------------------------------------------------- */
#define FMM_MLP_NF 12
#define FMM_MLP_NOUT 9
#define FMM_MLP_NBLOB 9769

/* M2L pair list of an adaptive plan after fmm_build_tree, grouped by target
 * (the order every per-pair array below uses): host arrays tgt[k], src[k]
 * (node indices; nodes are numbered level by level, children in octant
 * order).  *count receives the number of pairs; nothing is written when cap
 * is smaller.  Synchronous. */
int fmm_plan_pairs(fmm_plan* plan, int32_t* tgt, int32_t* src, int64_t cap, int64_t* count);

/* Features (device float [npair][FMM_MLP_NF]) and, when labels != NULL,
 * labels (device double [npair][FMM_MLP_NOUT]) of the plan's M2L pairs.
 * Runs P2M and M2M itself; labels also run an O(n^2) FP64 direct sum for
 * the total forces, so they need n <= 2^18, FMM_FP64, FMM_BASIS_SYM and
 * p = 10; features need p >= 4 and FMM_BASIS_SYM.  FMM_ERR_STATE before
 * fmm_build_tree. */
int fmm_pair_data(fmm_plan* plan, float* feat, double* labels, void* stream);

/* Mean squared error of the model over n samples (device feat [n][12],
 * labels [n][9], FP32) and its gradient with respect to blob[32..)
 * (host grad, FMM_MLP_NBLOB - 32 floats), in FP32.  Synchronous. */
int fmm_mlp_grad(const float* blob, int64_t n, const float* feat, const float* labels, float* loss,
                 float* grad, void* stream);

/* Trains the model in FP32 with Adam (beta1 0.9, beta2 0.999, eps 1e-8):
 * epochs passes over the samples in the order of `order` (device int32
 * permutation of 0..n-1, supplied by the caller), minibatches of `batch`,
 * learning rate lr.  blob (host, FMM_MLP_NBLOB floats) holds the initial
 * parameters and receives the trained ones; with fit_moments != 0 the
 * feature means and deviations are first set from the data.  loss_out
 * (host, epochs floats, may be NULL) receives each epoch's mean batch loss.
 * Allocates and frees its own scratch.  Synchronous. */
int fmm_mlp_train(float* blob, int64_t n, const float* feat, const float* labels, const int32_t* order,
                  int epochs, int batch, float lr, int fit_moments, float* loss_out, void* stream);

/* BF16 tensor-core inference: pred (device float [n][9]) from feat (device
 * float [n][12]).  blob is host memory. */
int fmm_mlp_predict(const float* blob, int64_t n, const float* feat, float* pred, void* stream);

/* Gives a learned_p plan its model (host blob, copied).  Synchronous. */
int fmm_set_mlp(fmm_plan* plan, const float* blob, int64_t nblob);

/* The order each M2L pair of the current tree used in the last M2L (host
 * int8, in the order of fmm_plan_pairs): the model's choice, or the orders
 * given by fmm_set_pair_orders.  *count receives the number of pairs;
 * nothing is written when cap is smaller.  FMM_ERR_STATE before
 * fmm_build_tree or before an M2L of the current tree.  Synchronous. */
int fmm_plan_pair_orders(fmm_plan* plan, int8_t* orders, int64_t cap, int64_t* count);

/* Gives every M2L pair of the current tree its order (host int8, n entries
 * in the order of fmm_plan_pairs, each in 0..p) instead of the model; NULL
 * returns to the model.  The orders stay in force while later builds keep
 * the same number of pairs.  Synchronous. */
int fmm_set_pair_orders(fmm_plan* plan, const int8_t* orders, int64_t n);

#ifdef __cplusplus
}
#endif
#endif /* FMM_GB300_H */
