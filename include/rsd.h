/*
 * rsd.h -- C ABI of the GB300 Recursive Schur Decomposition (RSD) library.
 *
 * The method (Sampath, Philip, Allu, Simunovic, "Recursive Schur Decomposition"):
 * a tree of nested sub-domains (Sec. 2); at every internal node the two (here: eight)
 * children are eliminated onto their shared interface I through the Schur complement
 * S = K_II - sum_c K_Ic K_cc^-1 K_cI (Eq. 3.2), and the children's unknowns are
 * recovered by back-substitution (Eq. 3.3); applied recursively down to the true
 * (leaf) sub-domains (Sec. 3.2, Algorithm 2), it preconditions a Krylov solve of K u = f.
 *
 * Conventions shared by every call:
 *   - Return value: RSD_OK (0) or a negative RSD_ERR_* code.  No call throws or aborts;
 *     rsd_strerror() names a code.  After RSD_ERR_CUDA the CUDA context may be unusable.
 *   - Matrices are CSR, 0-based, column indices sorted ascending within each row,
 *     FP64 values, symmetric positive definite (the SPD systems of Sec. 4).
 *   - "device" pointers are CUDA global memory of the current device; "host" pointers
 *     are ordinary (preferably pinned) host memory.  Each argument says which.
 *   - Vectors are FP64, length n, in the caller's DOF numbering.
 *   - Work is ordered on the stream given in rsd_options (or on the stream argument);
 *     calls on one handle must not run concurrently from several host threads.
 *   - The library never keeps a pointer the caller passed in: it copies what it needs.
 */
#ifndef RSD_H
#define RSD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------- */
#define RSD_OK              0
#define RSD_ERR_ARG        (-1)  /* bad argument: null pointer, size, tree, option value */
#define RSD_ERR_PARTITION  (-2)  /* K couples DOFs of two sub-domains that are not
                                    ancestor-related: the block structure of Eq. 3.1
                                    (K_LR = 0) does not hold for the given ownership */
#define RSD_ERR_NOT_SPD    (-3)  /* a pivot <= 0 (or NaN) in a sub-domain or interface
                                    factorisation */
#define RSD_ERR_NOMEM      (-4)  /* device or host allocation failed */
#define RSD_ERR_CUDA       (-5)  /* a CUDA runtime call failed */
#define RSD_ERR_TIMEOUT    (-6)  /* a bounded device-side wait gave up (see rsd_apply) */
#define RSD_ERR_NOCONV     (-7)  /* Krylov solve hit maxit; x and stats still filled */

/* ---- precisions of the stored factors and the arithmetic on them ----------------- */
#define RSD_PREC_FP64  0   /* FP64 storage, FP64 arithmetic on CUDA cores                */
#define RSD_PREC_FP32  1   /* FP32 storage, FP32 arithmetic on CUDA cores                */
#define RSD_PREC_TF32  2   /* FP32 storage; GEMM/TRSM updates on tcgen05 tensor cores in
                              TF32 with FP32 accumulation; diagonal blocks in FP32       */
#define RSD_PREC_FP16  3   /* as TF32, but the long Schur-complement updates (a panel's
                              update by all earlier panels, and U -= X X^T) read a 16-bit
                              copy of the finished panels on tcgen05 kind::f16 at twice the
                              TF32 rate: FP16, row i scaled by a power of two rs_i with
                              sqrt(K_ii) rs_i in [2^13, 2^14) (a symmetric diagonal scaling
                              of the front), FP32 accumulation, the scaling undone on the
                              result.  The factor entries are TF32 values (10-bit mantissa,
                              FP16's), so the copy holds them exactly down to 2^-27 sqrt(K_ii)
                              and the products equal TF32's.  The substitution sweeps read
                              the same copy.                                             */
#define RSD_PREC_BF16  4   /* as FP16 with a BF16 copy (8-bit mantissa) for those updates;
                              the sweeps read the FP32 factor.  A front whose pivot fails
                              (<= 0 or NaN) is factored again one precision up (BF16 or
                              FP16 -> TF32 -> FP32 on CUDA cores), with every ancestor that
                              consumed its Schur contribution; rsd_info_t.promoted counts
                              them.                                                      */

#define RSD_MODE_EXACT 0   /* exact recursive Schur complements (gamma -> infinity,
                              V-hat = V limit of Algorithm 2): the preconditioner is K^-1
                              up to the rounding of the stored factors                  */
#define RSD_MODE_PAPER 1   /* Algorithm 2 with the V-hat truncation of Sec. 3.2: each
                              interface solves S~ u_I = g, S~ = K_II minus the leaf terms
                              sum_l K_Il K_ll^-1 K_lI (Algorithm 1 with V-hat = the leaves
                              coupled to I), exactly (rsd_options.gamma = 0) or by gamma
                              GMRES iterations; g and the back-substitution use leaf
                              unknowns only.  Needs every leaf on the deepest level.
                              Not symmetric in general, and not linear for gamma > 0
                              (rsd_solve then runs FGMRES, the paper's outer GMRES in
                              flexible form); with gamma = 0 PCG still converges on the
                              SPD systems here.                                          */

/* outer Krylov method of rsd_solve */
#define RSD_KRYLOV_AUTO   0  /* PCG, except FGMRES for paper mode with gamma > 0           */
#define RSD_KRYLOV_PCG    1  /* preconditioned CG (needs a fixed SPD preconditioner)     */
#define RSD_KRYLOV_FGMRES 2  /* flexible right-preconditioned GMRES(restart), modified
                                Gram-Schmidt: the preconditioner may change from one
                                application to the next (finite gamma)                 */

#define RSD_MEM_HOST   0
#define RSD_MEM_DEVICE 1

/* ---- inputs ------------------------------------------------------------------------ */
typedef struct {
    int32_t        n;       /* rows = columns                                            */
    int64_t        nnz;
    const int64_t* rowptr;  /* n + 1 entries                                             */
    const int32_t* col;     /* nnz entries, ascending within a row                       */
    const double*  val;     /* nnz entries                                               */
    int32_t        mem;     /* RSD_MEM_HOST or RSD_MEM_DEVICE: where all three arrays live */
} rsd_csr;

/* Sub-domain tree of Sec. 2: node 0 is the whole domain; parent[t] < t for t > 0
 * (breadth-first ids), parent[0] = -1.  Leaves are the true sub-domains; every
 * internal node owns the interface DOFs that separate its children.               */
typedef struct {
    int32_t        n_nodes;
    const int32_t* parent;  /* host, n_nodes entries                                     */
} rsd_tree;

typedef struct {
    int32_t mode;        /* RSD_MODE_EXACT or RSD_MODE_PAPER                              */
    int32_t prec_leaf;   /* RSD_PREC_* of the leaf (true sub-domain) fronts               */
    int32_t prec_mid;    /* RSD_PREC_* of internal fronts below the root                  */
    int32_t prec_root;   /* RSD_PREC_* of the root interface                              */
    int32_t maxit;       /* rsd_solve iteration cap (<= 0: 200)                            */
    void*   stream;      /* cudaStream_t for every call on the handle (NULL: legacy default) */
    int32_t profile;     /* nonzero: record a CUDA event pair around every kernel launch of the
                            handle (see rsd_profile); adds ~2 us of host time per launch     */
    int64_t wait_cycles; /* bound of every wait of the substitution sweeps on another CTA's
                            progress, in SM clock cycles (<= 0: 4e9, about 2 s); a wait that
                            reaches it raises RSD_ERR_TIMEOUT (see rsd_apply)                */
    int32_t gamma;       /* paper mode only: 0 = each interface system S~ u = g is solved
                            exactly by a dense factorisation of S~ (formed at setup);
                            gamma > 0 = gamma GMRES iterations on it (Sec. 3.2, Algorithm 2),
                            x0 = 0, no restart, modified Gram-Schmidt, no inner
                            preconditioner, S~ applied matrix-free (Algorithm 1): no
                            interface front is formed or factored                          */
    int32_t krylov;      /* RSD_KRYLOV_*                                                    */
    int32_t restart;     /* FGMRES restart length (<= 0: 30)                                */
    const char* tune_cache; /* path of a table written by rsd_autotune (host string, read at
                            setup): the tile width and split-K count of the tensor-core
                            updates by size bucket; NULL = built-in rules                  */
    int32_t nonsymmetric;/* nonzero: K is not symmetric (its sparsity pattern must be): every
                            front is factored F_II = L U without pivoting (Eqs. 3.2-3.3 with
                            K_IL != K_LI^T, as the two-variable systems of Sec. 4, Eqs.
                            4.2-4.3, need), X = F_BI U^-1, Y = L^-1 F_IB, U_t = F_BB - X Y;
                            FP64 or FP32 on CUDA cores; rsd_solve runs FGMRES; exact mode, or
                            paper mode with gamma > 0.  A zero or non-finite pivot is
                            reported as RSD_ERR_NOT_SPD.                                    */
} rsd_options;

typedef struct {
    int32_t iterations;      /* PCG iterations taken                                      */
    double  relres;          /* ||f - K u|| / ||f|| recomputed in FP64 after the last step */
    double  relres_recursive;/* the recursively updated residual norm at exit             */
    double  history[64];     /* ||r_k|| / ||f|| for k = 0 .. min(iterations, 63)          */
} rsd_stats;

typedef struct {
    int32_t n;               /* DOFs                                                      */
    int32_t n_nodes;         /* tree nodes                                                */
    int32_t n_levels;        /* tree depth + 1                                            */
    int64_t factor_elems;    /* stored factor elements, sum_t (s_t^2/2 + s_t b_t)          */
    int64_t factor_bytes;    /* the same in bytes at each level's storage width           */
    double  setup_flops;     /* sum_t (s_t^3/3 + s_t^2 b_t + s_t b_t^2)                    */
    int64_t device_bytes;    /* bytes of device memory the handle holds                   */
    int32_t notspd_node;     /* first node whose pivot failed, or -1                      */
    int32_t promoted;        /* fronts factored again one precision up after a failed pivot
                                in a BF16 / FP16 / TF32 front (see RSD_PREC_BF16)          */
} rsd_info_t;

/* Per kernel class: launches, summed device time (CUDA events on the handle's stream)
 * and the algorithmic work of those launches (dense-front method: GEMM 2MNK flops;
 * substitution sweeps read every stored factor element once).  Classes:
 * 0 front assembly, 1 extend-add, 2 tcgen05 GEMM, 3 CUDA-core GEMM, 4 diagonal block
 * factor+inverse, 5 CUDA-core panel solve, 6 upward sweep, 7 downward sweep,
 * 8 sweep gathers, 9 Krylov vector/SpMV kernels, 10 FP16 copy of a TF32 level's factor
 * (the entries the sweeps read), 11 inner GMRES of paper mode with gamma > 0: its Arnoldi
 * steps (start vector, modified Gram-Schmidt, least-squares finish) of one interface
 * level, 12 tcgen05 GEMM on 16-bit operand copies (kind::f16; class 2 is then the
 * kind::tf32 launches only), 13 the leaf-coupling products of paper mode's S-MatVecs
 * (bytes = the X rows streamed), 14 the interface part of those S-MatVecs (K_II x less
 * the coupling terms).                                                                  */
#define RSD_PROFILE_CLASSES 15
typedef struct {
    int64_t launches[RSD_PROFILE_CLASSES];
    double  ms[RSD_PROFILE_CLASSES];
    double  flops[RSD_PROFILE_CLASSES];
    double  bytes[RSD_PROFILE_CLASSES];
    double  host_analysis_ms;    /* host-side analysis of the last rsd_setup             */
    double  host_parts_ms[6];    /* of which: structure copy to the host, ownership sort,
                                    Eq. 3.1 check, interface sets, extend-add maps, and the
                                    memory plan with its uploads                          */
    double  host_issue_ms;       /* host time spent issuing the numeric setup's launches
                                    (the device may still be working when it ends)        */
} rsd_profile_t;

/* one profiled launch (rsd_profile_trace): its class (as above), the stream it ran on
 * (0 = the caller's stream, 1 = the library's look-ahead stream used while factoring
 * levels with few fronts), device start and end in ms from the first recorded launch,
 * its algorithmic flops and bytes, and when the host issued it (ms from the first
 * record's issue; host and device times share no origin).                             */
typedef struct {
    int32_t cls;
    int32_t stream;
    double  start_ms, end_ms;
    double  flops, bytes;
    double  issue_ms;
} rsd_trace_rec;

typedef struct rsd_handle_s* rsd_handle;

/* ---- the three calls of the method --------------------------------------------- */

/* rsd_setup -- build the RSD hierarchy for K (Sec. 2 and Sec. 3.2; Eqs. 3.1-3.2).
 *   K        : the SPD matrix (host or device CSR, see rsd_csr.mem).
 *   dof_node : owner tree node of every DOF (n entries, same memory kind as K).
 *   T        : the sub-domain tree (host).
 *   opt      : options (host; NULL = exact mode, TF32 leaves/middle, FP64 root).
 *   out      : receives the handle; the handle owns all device memory it allocates.
 * Steps: validate the tree and the block structure of Eq. 3.1 (RSD_ERR_PARTITION),
 * form the interface index sets, then, level by level from the leaves up, assemble each
 * node's front from K and its children's Schur contributions, factor the interface block
 * and form the Schur contribution to the ancestors (Eq. 3.2).  All numeric work runs
 * in this library's CUDA kernels on opt->stream; the call returns after the stream has
 * drained and reports RSD_ERR_NOT_SPD if any pivot failed.  The caller may free K,
 * dof_node and T as soon as the call returns.                                         */
int rsd_setup(const rsd_csr* K, const int32_t* dof_node, const rsd_tree* T,
              const rsd_options* opt, rsd_handle* out);

/* rsd_setup_batched -- one hierarchy for nprob independent problems (many sub-domain
 * trees processed together: every tree level of every problem goes through the same
 * batched kernel launches).  K[p], dof_node[p], T[p] describe problem p exactly as for
 * rsd_setup (all K[p] in the same memory kind).  The problems are concatenated in order:
 * vectors passed to rsd_apply / rsd_solve hold problem 0's DOFs, then problem 1's, ...
 * Internally the trees hang under an empty super-root, so rsd_front_* node ids are
 * 1 + (sum of the earlier trees' sizes) + t.  rsd_solve runs one PCG on the
 * block-diagonal system (its inner products span all problems).                       */
int rsd_setup_batched(int32_t nprob, const rsd_csr* K, const int32_t* const* dof_node,
                      const rsd_tree* T, const rsd_options* opt, rsd_handle* out);

/* rsd_apply -- z = M r, one application of the preconditioner (Algorithm 2 in the exact
 * limit): an upward sweep that forms the interface right-hand sides g of Eq. 3.2 level by
 * level, and a downward sweep of back-substitutions (Eq. 3.3).
 *   r, z : device, n FP64 entries each, may not alias.  Stream-ordered on the handle's
 *          stream; returns without synchronising.  A device-side wait that exceeds its
 *          bound is reported as RSD_ERR_TIMEOUT by the next rsd_solve / rsd_check call. */
int rsd_apply(rsd_handle h, const double* r, double* z);

/* rsd_apply_static -- the same z = M r as rsd_apply, for callers that cannot have device
 * memory allocated on their behalf: a process that runs under a fixed device-memory
 * budget with every byte already handed out, or code inside a framework whose own
 * caching allocator owns the device (an allocation behind its back can fail, or force
 * the framework to release its cache).  The paper has no counterpart; it is a packaging
 * of rsd_apply.  The per-call scratch of the substitution sweeps (front vectors,
 * progress and ticket counters) is one file-scope device array of 4 MiB, which every
 * GPU that loads the library holds until the process exits; the call allocates nothing.
 * rsd_setup looks up that array's address on the handle's device and stores, in the
 * handle's own memory, a copy of the front descriptors that points into it, so the call
 * itself reads no host memory besides the handle.
 *   r, z : device, n FP64 entries each, may not alias (as rsd_apply).
 * Returns RSD_ERR_ARG if the hierarchy needs more than 4 MiB of scratch (roughly the sum
 * over tree nodes of (s + b + 32) entries at the level's storage width, plus two
 * counters per node), if the current device is not the handle's, or for a paper-mode
 * handle; rsd_last_error_detail names the reason.  The counters are cleared at the start
 * of every call; the array keeps the last call's vectors.  All calls on one device, from
 * every handle, stream and host thread, share the one array: calls that overlap on the
 * GPU race and must be serialised by the caller (for example by issuing them on one
 * stream).                                                                              */
int rsd_apply_static(rsd_handle h, const double* r, double* z);

/* rsd_solve -- preconditioned CG in FP64 on K u = f from u = 0 (the paper's outer Krylov
 * solve with RSD as preconditioner, Sec. 3 and Sec. 4), stopping when the recursively
 * updated residual satisfies ||r_k|| / ||f|| <= tol; then recomputes the true residual.
 *   f, u : device, n FP64 entries.   st : host, may be NULL.
 * Synchronises the stream once per iteration to test convergence.
 * Returns RSD_ERR_NOCONV if maxit iterations did not reach tol (u, st still valid).      */
int rsd_solve(rsd_handle h, const double* f, double* u, double tol, rsd_stats* st);

/* rsd_solve_adjoint -- the adjoint system K^T lam = g of the gradient of a loss L(u) with
 * u = K^-1 f (dL/df = lam, dL/dK = -lam u^T).  The paper has no counterpart: it is the
 * standard adjoint method applied to the solve above.  The hierarchy only holds
 * symmetric K (its fronts are Cholesky-factored), so K^T = K and the call runs the same
 * preconditioned CG on the same fronts, with no second setup.  RSD_ERR_ARG for a
 * nonsymmetric hierarchy.
 *   g, lam : device, n FP64 entries.  st : host, may be NULL.  Errors as rsd_solve.     */
int rsd_solve_adjoint(rsd_handle h, const double* g, double* lam, double tol, rsd_stats* st);

/* rsd_inject_drop_sweep_item -- fault injection for tests of the bounded waits (the paper
 * has no counterpart).  The next rsd_apply on h runs the upward sweep of tree level
 * `level` (0 = root) without that sweep's first work item (the first diagonal block of
 * the level's first front), as if the item were lost: the items that consume its result
 * wait on a progress counter that nothing raises.  Each such wait gives up after the
 * handle's wait_cycles, raises the timeout flag and lets its kernel finish, so the call
 * completes, the CUDA context stays usable and the next rsd_check / rsd_solve returns
 * RSD_ERR_TIMEOUT.  The handle's results are meaningless from then on: destroy it.
 * RSD_ERR_ARG for a bad level or a paper-mode handle.                                  */
int rsd_inject_drop_sweep_item(rsd_handle h, int32_t level);

/* rsd_check -- synchronise the handle's stream and report any device-side error flag
 * (timeout of a bounded wait, failed pivot) raised since setup.                        */
int rsd_check(rsd_handle h);

/* rsd_destroy -- release the handle.  Its device arena is kept in a one-slot per-device
 * cache and reused by the next rsd_setup on that device if large enough (the previously
 * cached block, if smaller, is freed); rsd_release_cache() frees the cached blocks.      */
void        rsd_destroy(rsd_handle h);
void        rsd_release_cache(void);
const char* rsd_strerror(int code);
/* detail of the last failure on the calling host thread (which CUDA call, which size). */
const char* rsd_last_error_detail(void);

/* ---- introspection (tests and benchmarks) --------------------------------------- */
int rsd_get_info(rsd_handle h, rsd_info_t* out);
/* s = |I_t| (interface / interior DOFs owned by node t), b = |B_t| (ancestor DOFs
 * coupled to the subtree of t); level = depth of t.                                   */
int rsd_front_dims(rsd_handle h, int32_t node, int32_t* s, int32_t* b, int32_t* level);
/* front DOF list I_t ++ B_t (host out, s + b entries, each part ascending).           */
int rsd_front_dofs(rsd_handle h, int32_t node, int32_t* out);
/* extend-add map of node t: positions of B_t inside its parent's front (host out, b). */
int rsd_front_map(rsd_handle h, int32_t node, int32_t* out);
/* factor of node t as FP64 row-major (s + b) x s (host out): rows 0..s-1 hold L_t,
 * the Cholesky factor of the interface Schur complement (lower triangle, zeros above);
 * rows s..s+b-1 hold X_t = K~_BI L_t^-T, the coupling to the ancestors.              */
int rsd_front_factor(rsd_handle h, int32_t node, double* out);
/* nonsymmetric fronts only: [U_t^T; Y_t^T] in the same (s + b) x s layout (rows 0..s-1 the
 * transposed upper factor, lower triangle; rows s.. Y_t^T = (L_t^-1 F_IB)^T); rsd_front_factor
 * returns [L_t; X_t] with the unit diagonal of L_t.  RSD_ERR_ARG for a symmetric hierarchy. */
int rsd_front_factor_upper(rsd_handle h, int32_t node, double* out);
/* FP16 copy of that factor which the substitution sweeps of a TF32 level read, unscaled
 * to FP64 in the same (s + b) x s layout: the entries below the NB x NB diagonal blocks
 * of L_t and all of X_t (Eq. 3.2 and 3.3 use L_t through its inverted diagonal blocks
 * and these entries); zeros elsewhere.  Row i is stored as rs_i times the entry, rs_i a
 * power of two with sqrt(K_ii) rs_i in [2^13, 2^14); every stored entry is a TF32 value
 * and |entry| <= sqrt(K_ii), so the copy equals rsd_front_factor except for entries
 * below 2^-27 sqrt(K_ii), which it holds to 2^-38 sqrt(K_ii).
 * Errors: RSD_ERR_ARG for a bad node or a node whose level has no copy (FP32 / FP64
 * fronts, paper mode).                                                                */
int rsd_front_factor16(rsd_handle h, int32_t node, double* out);

/* rsd_front_dinv -- the inverted diagonal blocks of node's front that the substitution
 * sweeps apply (Eqs. 3.2-3.3 split into NB-row blocks, NB = 128): block k of L_t's
 * diagonal, inverted, as stored (rounded to TF32 on tensor-core levels).  Writes
 * nd x 128 x 128 doubles (host, caller-owned), block k row-major at k * 128 * 128, with
 * nd = ceil(s / 128) and zeros above the diagonal and past s.  Synchronises the stream.
 * Errors: RSD_ERR_ARG for a bad node or a level that is not factored (paper mode's leaf
 * levels are; its interface levels are solved from S~).                              */
int rsd_front_dinv(rsd_handle h, int32_t node, double* out);

/* rsd_profile -- synchronise the handle's stream and sum the profile recorded since
 * setup or the last reset (all zeros unless rsd_options.profile was set).  reset != 0
 * clears it afterwards.                                                               */
int rsd_profile(rsd_handle h, rsd_profile_t* out, int32_t reset);

/* rsd_profile_trace -- the individual launch records behind rsd_profile, in issue order
 * (a timeline of setup and solve).  Synchronises like rsd_profile and must be called
 * before a resetting rsd_profile.  Writes min(cap, count) records to out (host; may be
 * NULL when cap = 0) and the total count to *n.                                       */
int rsd_profile_trace(rsd_handle h, rsd_trace_rec* out, int64_t cap, int64_t* n);

/* rsd_peak_gemm -- measured rate of this library's own dense GEMM kernel for one
 * precision, C -= A B^T on an n x n x n product of FP values in [-1, 1): the roofline
 * denominator of the Schur-complement updates of Eq. 3.2 (the paper reports no rates).
 *   prec    : RSD_PREC_TF32 / RSD_PREC_FP16 / RSD_PREC_BF16 (the persistent tcgen05
 *             128 x 256 kernel with FP32 / FP16 / BF16 operands, n a multiple of 256),
 *             RSD_PREC_FP32 or RSD_PREC_FP64 (the CUDA-core kernel, n a multiple of 64).
 *   reps    : timed single launches; *best_tflops = 2 n^3 / the shortest (TFLOP/s).
 *   seconds : then back-to-back launches for about this long; *sustained_tflops = their
 *             mean rate.  CUDA events on `stream` (cudaStream_t; NULL: legacy default).
 * Allocates and frees 3 n^2 elements of device memory.  RSD_ERR_ARG on a bad size or
 * precision, RSD_ERR_TIMEOUT if a bounded wait of the kernel gave up.                 */
int rsd_peak_gemm(int32_t prec, int32_t n, int32_t reps, double seconds, void* stream,
                  double* best_tflops, double* sustained_tflops);

/* rsd_autotune -- measure this library's tensor-core GEMM configurations and write the
 * fastest per size bucket to `path` (JSON: one object per bucket with the operand format
 * (0 TF32, 1 FP16/BF16), output tiles of 128 x 256, K, tile width, split-K count and the
 * measured and built-in-rule times in us).  The buckets: 1, 4, 16, 64, 256 tiles x K =
 * 512, 2048, 8192, 24576; the candidates: tile width 128 or 256 (TF32; 256 for 16-bit
 * operands) x 1..32 split-K slices of at least 4 K blocks; each timed as the best of 3
 * launches of C -= A B^T on synthetic operands through the factorisation's own launcher.
 * The paper has no counterpart (the tile shapes of the Schur-complement GEMMs of Eq. 3.2).
 * Allocates and frees about 5 GB of device memory; *seconds receives the wall time.
 * RSD_ERR_ARG if the file cannot be written.                                           */
int rsd_autotune(const char* path, double* seconds, void* stream);
/* rsd_tune_load -- parse and check a table written by rsd_autotune (host only, no GPU):
 * *entries receives the number of buckets; RSD_ERR_ARG for a missing or malformed file.  */
int rsd_tune_load(const char* path, int32_t* entries);

/* rsd_launch_count -- kernels this library has launched in this process so far.       */
int64_t rsd_launch_count(void);

/* ---- structured-grid FEM problems (the synthetic workloads) ---------------------- *
 * Unit cube, n x n x n nodes (h = 1/(n-1)), trilinear hexahedra, homogeneous Dirichlet
 * on the boundary (Sec. 4's setting in 3-D); unknowns are the (n-2)^3 interior nodes,
 * numbered x-1 + (n-2)*((y-1) + (n-2)*(z-1)).                                          */

/* sizes of the -div(kappa grad u) system: n_dof = (n-2)^3 and its nonzero count.       */
int rsd_grid_sizes(int32_t n, int64_t* n_dof, int64_t* nnz);
/* assemble K for kappa constant per element (element (ex,ey,ez) at ex + (n-1)*(ey +
 * (n-1)*ez)): kappa device ((n-1)^3), rowptr/col/val device (n_dof+1, nnz, nnz).      */
int rsd_grid_assemble(int32_t n, const double* kappa, int64_t* rowptr, int32_t* col,
                      double* val, void* stream);
/* load vector b = h^3 f (lumped mass) from nodal f; both device, n_dof entries.         */
int rsd_grid_load(int32_t n, const double* f, double* b, void* stream);
/* octree decomposition of the grid to the given depth (Sec. 2 generalised to 3-D: each
 * box splits at its integer mid-planes; a node belongs to the first box whose
 * mid-planes contain it, else to its leaf).  dof_node device (n_dof); parent host
 * ((8^(depth+1)-1)/7 entries, breadth-first ids).                                       */
int rsd_grid_partition(int32_t n, int32_t depth, int32_t* dof_node, int32_t* parent,
                       void* stream);
/* kappa = exp(m) per element, both device, (n-1)^3 entries (kappa's log parametrisation). */
int rsd_grid_exp(int32_t n, const double* m, double* kappa, void* stream);
/* per-element coefficient gradient for -div(kappa grad u) with kappa constant per
 * element: K = sum_e kappa_e K_e with K_e = h Khat on the element's interior nodes, so
 * for K^T lam = dL/du the gradient is dL/dkappa_e = -lam_e^T K_e u_e, and with kappa =
 * exp(m), dL/dm_e = kappa_e dL/dkappa_e.  The paper has no counterpart (the adjoint
 * method applied to Sec. 4's discretisation).
 *   u, lam : device, n_dof entries; kappa : device, (n-1)^3 (only read for dm);
 *   dkappa, dm : device, (n-1)^3 outputs, either may be NULL (not both).  One thread per
 * element, deterministic.  RSD_ERR_ARG on a bad n or pointer.                             */
int rsd_grid_coef_grad(int32_t n, const double* u, const double* lam, const double* kappa,
                       double* dkappa, double* dm, void* stream);

/* ---- 3-D linear elasticity on the same grids (three DOFs per node) ---------------- *
 * -div sigma(u) = f with sigma = lam tr(eps) I + 2 mu eps: the SPD Navier-Lame form of
 * Sec. 4's Problem 4 (Eq. 4.4, whose printed sign is read as this form), in 3-D.  DOF
 * 3 * node + c (c = 0, 1, 2 the displacement component), node the interior-node id above;
 * homogeneous Dirichlet on every component at the boundary.                           */

/* sizes: n_dof = 3 (n-2)^3 and the nonzero count (81 per interior row).                  */
int rsd_grid_elastic_sizes(int32_t n, int64_t* n_dof, int64_t* nnz);
/* assemble K with Young's modulus constant per leaf sub-domain of the octree of the given
 * depth (E_leaf device, 8^depth entries in breadth-first leaf order; an element spanning
 * [e, e+1] per coordinate lies in a box's lower child when e < its mid-plane) and
 * Poisson's ratio nu in (-1, 1/2); K_e = E_e h Khat(nu) with Khat the unit-cube element
 * matrix (exact integrals of the trilinear shape functions).  rowptr/col/val device
 * (n_dof + 1, nnz, nnz); one thread per row, deterministic.  RSD_ERR_ARG on bad sizes.  */
int rsd_grid_elastic_assemble(int32_t n, int32_t depth, const double* E_leaf, double nu,
                              int64_t* rowptr, int32_t* col, double* val, void* stream);
/* lumped load b = h^3 f per DOF; both device, n_dof entries.                             */
int rsd_grid_elastic_load(int32_t n, const double* f, double* b, void* stream);
/* the octree decomposition of rsd_grid_partition with every DOF owned by its node's owner:
 * dof_node device (n_dof), parent host (as rsd_grid_partition), node_scratch device
 * ((n-2)^3 ints, overwritten).                                                          */
int rsd_grid_elastic_partition(int32_t n, int32_t depth, int32_t* dof_node, int32_t* parent,
                               int32_t* node_scratch, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* RSD_H */
