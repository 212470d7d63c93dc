// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "rsd.h"

namespace rsd {

// Diagonal block size of the blocked partial Cholesky and of the substitution sweeps.
constexpr int NB = 128;

// Device-side error flags (one int array per handle).
enum ErrSlot { ERR_NOT_SPD = 0, ERR_TIMEOUT = 1, ERR_NOT_SPD_NODE = 2, ERR_SLOTS = 4 };

#define RSD_CUDA_TRY(expr)                                           \
    do {                                                             \
        cudaError_t _e = (expr);                                     \
        if (_e != cudaSuccess) {                                     \
            rsd::set_last_error(std::string(#expr) + ": " + cudaGetErrorString(_e)); \
            return RSD_ERR_CUDA;                                     \
        }                                                            \
    } while (0)

#define RSD_TRY(expr)                      \
    do {                                   \
        int _rc = (expr);                  \
        if (_rc != RSD_OK) return _rc;     \
    } while (0)

void set_last_error(const std::string& msg);

inline int elem_bytes(int prec) { return prec == RSD_PREC_FP64 ? 8 : 4; }
inline bool is_fp64(int prec) { return prec == RSD_PREC_FP64; }


// One tree node's dense front and factor, as the kernels see it.
// P is row-major N x ldp with N = s + b: rows 0..s-1 hold L (lower triangle; the
// diagonal NB x NB blocks are also kept inverted in Dinv), rows s..N-1 hold X = K_BI L^-T.
// U is row-major b x ldu (lower triangle): the Schur contribution to the ancestors.
struct FrontDesc {
    int node, s, b, N;
    int ldp, ldu, nd;          // row strides; nd = number of diagonal blocks
    int parent_slot;           // index of the parent in the next level's front array
    void* P;
    void* U;
    void* Dinv;                // nd x NB x NB, each block lower triangular (inverse of L_kk)
    const int* I;              // global DOFs of I_t (s)
    const int* Bd;             // global DOFs of B_t (b)
    const int* ea;             // positions of B_t in the parent front (b)
    // the inverse of the children's ea maps (the upward sweep's gather): for front position
    // p, gsrc[gptr[p] .. gptr[p + 1]) lists (child index, entry of that child's B), in the
    // order of the children
    const int* gptr;
    const int2* gsrc;
    void* vec;                 // apply: front vector (N entries, level accumulator type)
    int* flag;                 // apply: progress counters [forward, backward]
    int child_begin, child_count;   // into the level's child-slot table (previous level)
    // TF32 levels: FP16 copy of the factor entries the substitution sweeps read (the
    // off-diagonal blocks of L and X, same layout and ldp as P), row i scaled by the power
    // of two rs[i]; ri[i] = 1 / rs[i].  Every entry is TF32-rounded when final, and
    // |P_ij| <= sqrt(K_ii) (a Schur complement's diagonal never exceeds K's), so with
    // sqrt(K_ii) rs[i] in [2^13, 2^14) the copy is exact down to 2^-27 sqrt(K_ii).
    // nullptr elsewhere.
    void* P16;
    const float* rs;
    const float* ri;
    // nonsymmetric fronts (LU without pivoting): PU is [U^T; Y^T], N x ldp like P, with
    // F_II = L U (L unit lower in P), Y = L^-1 F_IB, X = F_BI U^-1 (rows s.. of P); DinvU
    // holds (U_kk^T)^-1 per diagonal block (Dinv then holds L_kk^-1).  nullptr otherwise.
    void* PU;
    void* DinvU;
};

// Batched GEMM task: C = beta*C - A * B^T over an M x N block (row-major operands,
// A is M x K, B is N x K).  beta is 0 or 1.  lower: C is symmetric, only tiles that
// meet the lower triangle are computed.
struct GemmTask {
    const void* A;
    const void* B;
    void* C;
    int lda, ldb, ldc;
    int M, N, K;
    int tiles_n;         // tiles along N
    int tile_begin;      // first global tile of this task
    int lower;
    int beta;
    int map_a, map_b;    // tensor-map slots (tensor-core path); -1 when unused
    int a_r0, a_c0, b_r0, b_c0;   // operand origins inside the tensor maps
    float alpha;         // general tensor-core kind only: C = alpha A B^T + beta C
    int round;           // general kind only: round stored results to TF32
    // 16-bit operand copies (TC_OP_F16 / TC_OP_BF16 launches): 1 / row scale of A's first
    // row and of B's first row (the product is multiplied by sa[i] sb[j])
    const float* sa;
    const float* sb;
};

// Operand formats of the tensor-core GEMM: FP32 storage read as TF32 (kind::tf32), or the
// row-scaled 16-bit copy of a front's factor (kind::f16 with FP16 or BF16 operands).
enum { TC_OP_TF32 = 0, TC_OP_F16 = 1, TC_OP_BF16 = 2 };

// Kernel classes for launch counting and the optional CUDA-event profile.
enum KClass { K_ASSEMBLE = 0, K_EXTEND, K_GEMM_TC, K_GEMM_SIMT, K_POTRF, K_TRSM, K_FWD, K_BWD,
              K_GATHER, K_KRYLOV, K_COPY16, K_GAMMA, K_GEMM_TC16, K_GAMMA_SMV, K_GAMMA_IFACE, K_CLASSES };

// Per-handle profile: one event pair per launch of a class, with the algorithmic
// flops and bytes of that launch; reduced on demand by rsd_profile().
struct Prof {
    bool on = false;
    struct Rec { int cls; double flops, bytes; cudaEvent_t a, b; int stream; double host_us; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    double host_ms = 0;                  // host-side analysis time of the last setup
    double host_part[6] = {0, 0, 0, 0, 0, 0};   // copy, sort, check, sets, maps, plan
    double host_issue_ms = 0;            // issuing the numeric setup's launches
};

void count_launch(int n = 1);

struct Level {
    int depth = 0;
    int prec = RSD_PREC_FP64;
    std::vector<int> nodes;              // tree node ids, in slot order
    std::vector<FrontDesc> fronts;       // host copy
    FrontDesc* d_fronts = nullptr;       // device copy
    int max_s = 0, max_b = 0, max_N = 0;
    int max_children = 0;
    // apply work lists (device): forward/backward items, (slot << 16 | block)
    int* d_fwd_items = nullptr;
    int n_fwd_items = 0;
    int* d_bwd_items = nullptr;
    int n_bwd_items = 0;
    // child slot table (device): for slot i of this level, child_begin.. -> slots of
    // the level below
    int* d_child_slots = nullptr;
    size_t bytes_P = 0, bytes_U = 0;
    bool h16 = false;                    // the sweeps read the FP16 factor copy (P16, rs, ri)
    // every front of the level has no B rows (the root level) and the sweeps read the FP16
    // copy: the sweeps run on clusters of SWEEP_CL CTAs, one diagonal block each, and the
    // work lists group SWEEP_CL diagonal blocks per item
    bool cl_sweep = false;
    // operand format of the long-K Schur updates (TC_OP_*): with a 16-bit format the
    // fronts carry its row-scaled copy (P16, rs, ri), written panel by panel
    int op16 = TC_OP_TF32;
    // paper mode: descriptors of the same fronts restricted to their interface block
    // (b = 0, no children) and forward items over interface blocks only, used by the
    // leaf and interface solves of the level-wise Algorithm 2
    FrontDesc* d_fronts_solve = nullptr;
    int* d_fwd_items_solve = nullptr;
    int n_fwd_items_solve = 0;
    // false for the interface levels of paper mode with gamma > 0: no front is stored
    bool factored = true;
    // nonsymmetric fronts: descriptors with P = PU and Dinv = DinvU for the backward sweeps
    // (and, in paper mode, for the backward leaf solves); nullptr for symmetric fronts
    FrontDesc* d_fronts_bwd = nullptr;
    FrontDesc* d_fronts_solve_bwd = nullptr;
};

// Paper mode with gamma inner GMRES iterations: one interface level's packed vectors and
// its couplings to the leaves (see paper_gamma.cu).  Interface slot i owns positions
// [if_off[i], if_off[i+1]); if_dofs maps a position to its global DOF.  cl_*: per leaf
// (CSR over leaf slots), the rows r of the leaf's X block that lie in the level's
// interfaces and their packed positions; ci_*: per packed position (CSR), the couplings
// (cl indices) that touch it, leaves ascending.
struct GammaLevel {
    int n_if = 0, S = 0;
    int *d_if_off = nullptr, *d_if_dofs = nullptr;
    int *d_cl_ptr = nullptr, *d_cl_row = nullptr, *d_cl_pos = nullptr;
    int* d_cl_leaf = nullptr;     // leaf slot of every coupling (cl index)
    int *d_ci_ptr = nullptr, *d_ci_k = nullptr;   // couplings (cl indices) per packed position
    int nk = 0;                   // couplings of the level
    double xbytes = 0;            // bytes of X one S-MatVec streams (its rows read twice)
};

// Levels factored with tcgen05 GEMMs (TF32 on the FP32 panels, or 16-bit operand copies).
inline bool tc_level(const Level& L) {
    return L.prec == RSD_PREC_TF32 || L.prec == RSD_PREC_FP16 || L.prec == RSD_PREC_BF16;
}
// Levels whose fronts carry a row-scaled 16-bit copy of the factor (P16, rs, ri).
inline bool copy16_level(const Level& L) { return L.h16 || L.op16 != TC_OP_TF32; }

// Diagonal blocks per substitution-sweep item: a single-front FP32 level (a root) pairs
// its blocks, halving the hand-offs of its long dependency chain; levels with many
// fronts keep one block per item, whose smaller footprint lets more CTAs stream the
// factor at once (an FP64 pair would not fit in shared memory).
inline int sweep_group(const Level& L) { return (!is_fp64(L.prec) && L.fronts.size() == 1) ? 2 : 1; }

// Paper mode with gamma > 0: the S-MatVec reads the leaves' FP16 copy when they have one
// (FP16-operand leaves, and TF32 leaves, whose solves read the copy too; not BF16 copies,
// FP64 or FP32 leaves, or the transposed upper factors of nonsymmetric leaves).
inline bool smv_reads_fp16(const Level& Ll) {
    return (Ll.op16 == TC_OP_F16 || Ll.h16) && !Ll.d_fronts_bwd && !is_fp64(Ll.prec);
}

// CTAs per cluster of the cluster sweeps (diagonal blocks per work item of a cl_sweep level)
constexpr int SWEEP_CL = 8;
inline int sweep_item_blocks(const Level& L) { return L.cl_sweep ? SWEEP_CL : sweep_group(L); }

// Per tree node: where its front lives (paper-mode scatter of leaf updates).
struct NodeRef {
    void* P;
    int ldp;
    int f64;
};

struct Handle {
    int n = 0;
    int n_nodes = 0;
    cudaStream_t stream = nullptr;
    rsd_options opt{};
    std::vector<int> parent, depth;
    std::vector<Level> levels;           // index 0 = root level, back() = deepest
    std::vector<int> node_level, node_slot;
    // host copies of the symbolic structure (introspection)
    std::vector<int> I_off, I_dofs, B_off, B_dofs;   // CSR-like per node
    // device buffers
    char* arena = nullptr;
    size_t arena_bytes = 0;
    size_t arena_capacity = 0;          // bytes of the block actually held (cache reuse)
    int device = 0;
    int* d_err = nullptr;
    int* d_front_bad = nullptr;          // per node: a pivot of its factorisation failed
    int promoted = 0;                    // fronts re-factored one precision up at setup
    bool lu = false;                     // nonsymmetric K: LU fronts (FrontDesc::PU, DinvU)
    int* d_ticket = nullptr;             // per-sweep ticket counters
    // CSR of K on the device (FP64), owned copy for the Krylov SpMV
    int64_t nnz = 0;
    int64_t* d_rowptr = nullptr;
    int* d_col = nullptr;
    double* d_val = nullptr;
    // Krylov work vectors
    double *d_r = nullptr, *d_p = nullptr, *d_q = nullptr, *d_z = nullptr;
    double* d_scal = nullptr;            // device scalars
    double* d_partial = nullptr;         // reduction partials
    double* h_scal = nullptr;            // pinned host mirror
    int64_t factor_elems = 0, factor_bytes = 0;
    double setup_flops = 0;
    int notspd_node = -1;
    int num_sms = 148;
    void* tc_state = nullptr;            // tensor-core GEMM state (tensor maps, task buffers)
    Prof prof;
    // paper mode (V-hat truncation, dense S~ per interface)
    bool paper = false;
    int* d_owner = nullptr;
    int* d_rank = nullptr;
    int* d_node_depth = nullptr;
    unsigned char* d_node_leaf = nullptr;
    NodeRef* d_node_ref = nullptr;
    double *d_pg = nullptr, *d_pw = nullptr, *d_pz = nullptr;   // g, w and leaf-solve scratch
    int* d_ticket_paper = nullptr;
    // leaf slots by colour class (no two leaves of a class share an interface DOF) for the
    // fixed-order accumulation of the leaf updates into S~
    std::vector<int> paper_color_off;
    int* d_paper_color_slots = nullptr;
    // pinned host staging for per-launch uploads (append-only; see stage_host)
    std::vector<std::pair<char*, size_t>> stage_blocks;
    size_t stage_cur = 0, stage_off = 0;
    // look-ahead factorisation of levels with few fronts: a high-priority stream runs the
    // diagonal-block chain beside the bulk updates on `stream` (created on first use)
    cudaStream_t chain = nullptr;
    cudaEvent_t ev_ready = nullptr, ev_join = nullptr;
    cudaEvent_t ev_diag[4] = {nullptr, nullptr, nullptr, nullptr};
    // PCG's preconditioner application as a captured graph (see pcg_apply)
    cudaGraphExec_t apply_exec = nullptr;
    int solve_calls = 0, apply_graph_launches = 0;
    // rsd_apply_static: descriptors whose vectors and counters point into the library's
    // file-scope device array (prepared at setup; static_ok false when it does not fit)
    FrontDesc* d_static_fronts = nullptr;
    std::vector<int> static_level_first;
    int* static_ticket = nullptr;
    size_t static_clear_bytes = 0, static_need = 0;
    bool static_ok = false;
    // paper mode, gamma > 0 (see GammaLevel); gamma_levels[d] for interface level d
    int gamma = 0;
    std::vector<GammaLevel> gamma_levels;
    int* d_pk_pos = nullptr;             // global DOF -> position in its level's packed vectors
    int* d_tl_off = nullptr;             // leaf slot -> offset of its t_l in d_tl
    double* d_tl = nullptr;              // X_l^T x per leaf
    double *d_gm_w = nullptr, *d_gm_V = nullptr, *d_gm_H = nullptr, *d_gm_beta = nullptr;
    double* d_gm_yl = nullptr;           // per coupling: X_l[row] . t_l
    int* d_gm_kused = nullptr;
    // outer Krylov method (RSD_KRYLOV_PCG or RSD_KRYLOV_FGMRES) and FGMRES storage
    int krylov = RSD_KRYLOV_PCG, restart = 30;
    double *d_fg_V = nullptr, *d_fg_Z = nullptr, *d_fg_H = nullptr, *d_fg_y = nullptr;
    double* h_fg = nullptr;              // pinned host mirror of H columns and y
    // bounded waits of the substitution sweeps: clock cycles before a wait gives up
    long long wait_cycles = 4000000000LL;
    // fault injection (rsd_inject_drop_sweep_item): level whose next upward sweep runs
    // without its first work item, or -1
    int inject_drop_level = -1;
};

// Copy `bytes` from host memory into the handle's pinned staging area and return the
// pinned copy, so that a following cudaMemcpyAsync is truly asynchronous.  The area is
// used append-only (another pinned block is added when it is full, never waiting for
// the device); stage_reset() rewinds it once every staged copy is known to be done.
const void* stage_host(Handle& h, const void* src, size_t bytes);
void stage_reset(Handle& h);
// give the handle's staging blocks back to the pool / destroy its profiling events
void stage_release(Handle& h);
void prof_release(Handle& h);

// Profile helpers: prof_begin records the start event (if profiling) and returns a
// record index; prof_end records the stop event and the launch's algorithmic work.
int prof_begin(Handle& h, int cls, cudaStream_t stream);
void prof_end(Handle& h, int idx, double flops, double bytes, cudaStream_t stream);
inline int prof_begin(Handle& h, int cls) { return prof_begin(h, cls, h.stream); }
inline void prof_end(Handle& h, int idx, double flops, double bytes) { prof_end(h, idx, flops, bytes, h.stream); }

// Tensor-core GEMM launch (gemm_tc.cu).  kind 0: inner panel update, 1: panel solve with
// an inverted diagonal block, 2: U -= X X^T (lower tiles), 3: outer panel update.
// `slot` selects the launch buffers (one per stream that launches concurrently);
// max_ctas > 0 caps the CTAs of the persistent kernel (leaving SMs to another stream).
constexpr int TC_SLOTS = 2;
constexpr int TC_GENERAL = 4;        // kind: explicit map indices, alpha and rounding
// Recorded launches: between record_begin and record_end, gemm_tc_launch only records
// each launch's task and tile lists; record_end uploads them in one copy on `stream`,
// and the next gemm_tc_launch calls, which must repeat the recorded sequence, launch
// from the uploaded lists; replay_end frees them (stream-ordered on `stream`).
int gemm_tc_record_begin(Handle& h);
int gemm_tc_record_end(Handle& h, cudaStream_t stream);
void gemm_tc_replay_end(Handle& h, cudaStream_t stream);
// Tensor maps for per-front scratch of the level being factored (the block-inverse panel
// solve): TC_SCR_MAPS per front slot -- Mt (512 x 512), Tt (512 x 128) and two Linv
// (512 x 512, alternating panels) -- encoded and uploaded on `stream`; returns the index
// of slot 0's first map.
constexpr int TC_SCR_MAPS = 4;
int gemm_tc_scratch_maps(Handle& h, const std::vector<float*>& mt, const std::vector<float*>& tt,
                         const std::vector<float*>& linv0, const std::vector<float*>& linv1,
                         cudaStream_t stream, int* base);
// map index of a node's [L; X] panel (P), of its inverted diagonal blocks, and of its
// 16-bit operand copy (P16)
constexpr int TC_NODE_MAPS = 3;
inline int tc_map_panel(int node) { return TC_NODE_MAPS * node; }
inline int tc_map_dinv(int node) { return TC_NODE_MAPS * node + 1; }
inline int tc_map_panel16(int node) { return TC_NODE_MAPS * node + 2; }
// op: TC_OP_F16 / TC_OP_BF16 run kinds 2 and 3 on the nodes' 16-bit copies (tasks carry
// sa / sb); TC_OP_TF32 on the FP32 panels.
int gemm_tc_launch(Handle& h, int li, const std::vector<GemmTask>& tasks, int kind, cudaStream_t stream,
                   int slot = 0, int max_ctas = 0, int op = TC_OP_TF32);

// ---- kernels launched from the host orchestration -------------------------------
// Zero the P and U storage of every front of level li (before its assembly).
int launch_zero_fronts(Handle& h, int li);
// FP16 copy of level li's factor (after its factorisation), read by the sweeps.
int launch_factor_copy16(Handle& h, int li);
int launch_assemble_fronts(Handle& h, int li, const int64_t* rowptr, const int* col,
                           const double* val, const int* owner, const int* rank,
                           const int* tin, const int* tout);
int launch_extend_add(Handle& h, int li);
int run_factor_level(Handle& h, int li);
// nonsymmetric fronts: assembly, extend-add and LU partial factorisation of level li
int launch_assemble_fronts_lu(Handle& h, int li, const int64_t* rowptr, const int* col, const double* val,
                              const int* owner, const int* rank, const int* tin, const int* tout);
int launch_extend_add_lu(Handle& h, int li);
int run_factor_level_lu(Handle& h, int li);
int run_apply(Handle& h, const double* r, double* z);
int run_apply_static(Handle& h, const double* r, double* z);
// descriptors of the allocation-free application, written to d_slots (n_nodes entries of
// the arena) at setup, with the handle's device current
int static_apply_prepare(Handle& h, FrontDesc* d_slots);
// one level of a substitution sweep with explicit descriptors/items: forward reads the
// right-hand side from `in` (through I), backward writes the solution to `out`
int sweep_with(Handle& h, int li, bool forward, const FrontDesc* fronts, const int* items, int n_items,
               const double* in, double* out, int* ticket);
int paper_extend_add(Handle& h);
// bytes one sweep of a level streams from its factor (with_x = false: L without X)
double level_factor_bytes(const Level& L, bool with_x);
// peak probes of this library's GEMM kernels (rsd_peak_gemm)
int gemm_tc_peak(int n, int reps, double seconds, cudaStream_t stream, int num_sms, double* best, double* sustained,
                 int op);
int gemm_simt_peak(int prec, int n, int reps, double seconds, cudaStream_t st, double* best, double* sustained);
int gemm_tc_autotune(const char* path, cudaStream_t stream, int num_sms, double* secs);
int tune_read(const char* path, void* out_table, int32_t* entries);
int run_apply_paper(Handle& h, const double* r, double* z);
int gamma_interface_solve(Handle& h, int li, double* z);
int fgmres(Handle& h, const double* f, double* u, double tol, rsd_stats* st);
int spmv(Handle& h, const double* x, double* y);

}  // namespace rsd
