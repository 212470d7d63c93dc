// Setup-phase kernels: front assembly, extend-add of the children's Schur contributions,
// and the blocked partial Cholesky that eliminates each node's interface block.
//
// Per tree node t with interface/interior DOFs I (s of them) and ancestor DOFs B (b):
//   F_t = K[I u B, I u B] restricted to rows/columns of I, plus sum_c U_c placed by the
//   extend-add maps; F_t[I,I] is then the interface Schur complement S_t of Eq. 3.2 (the
//   children's sub-domains already eliminated, Sec. 3.2).
//   L L^T = F_t[I,I],  X = F_t[B,I] L^-T,  U_t = -X X^T  (U_t's B x B block also carries the
//   children's contributions that land on B).
// Storage (row-major, lower triangles): P = [L; X] is N x ldp, U is b x ldu.
//
// The partial Cholesky is left-looking by NB-wide column panels, blocked in two levels
// (outer panels of WOUT = 4 NB columns starting at K0):
//   (a0) at k = K0: P[K0:N, K0:K0+WOUT] -= P[K0:N, 0:K0] P[K0:K0+WOUT, 0:K0]^T  (K = K0)
//   (a) P[k:N, k:k+w] -= P[k:N, K0:k] P[k:k+w, K0:k]^T      (GEMM, K = k - K0 < WOUT)
//   (b) L_kk L_kk^T = P[k:k+w, k:k+w]; Dinv_k = L_kk^-1         (one CTA per front)
//   (c) P[k+w:N, k:k+w] <- P[k+w:N, k:k+w] Dinv_k^T             (TRSM as a GEMM, K = w)
// and after the last panel
//   (d) U -= X X^T (lower tiles only)                           (GEMM, K = s)
#include <algorithm>
#include <cmath>
#include <type_traits>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "rsd_internal.cuh"

namespace rsd {

namespace {

template <typename T>
__device__ __forceinline__ T ld_nc(const T* p) { return __ldg(p); }

// ---------------------------------------------------------------------------------
// Front assembly: each warp takes rows of I_t and scatters K's entries into P.
// Entry (p, q) of row p (DOF I_t[p]) goes to the lower triangle at (q, p) when q >= p:
// q is the local index of the column DOF in I_t (q >= p) or s + position in B_t.
// Columns owned by descendants of t were placed by those descendants; entries with
// q < p inside I are placed by row q.  Every target is written exactly once.
// ---------------------------------------------------------------------------------
template <typename T>
__global__ void k_scatter_K(const FrontDesc* __restrict__ fronts, const int64_t* __restrict__ rowptr,
                            const int* __restrict__ col, const double* __restrict__ val,
                            const int* __restrict__ owner, const int* __restrict__ rank,
                            const int* __restrict__ tin, const int* __restrict__ tout) {
    const FrontDesc f = fronts[blockIdx.y];
    const int lane = threadIdx.x & 31;
    const int warps = blockDim.x >> 5;
    const int t = f.node;
    const int tin_t = tin[t], tout_t = tout[t];
    T* P = (T*)f.P;
    for (int p = blockIdx.x * warps + (threadIdx.x >> 5); p < f.s; p += gridDim.x * warps) {
        const int i = f.I[p];
        for (int64_t k = rowptr[i] + lane; k < rowptr[i + 1]; k += 32) {
            const int j = col[k];
            const int o = owner[j];
            int q;
            if (o == t) {
                q = rank[j];
                if (q < p) continue;
            } else if (tin[o] < tin_t && tout_t <= tout[o]) {      // proper ancestor of t
                int lo = 0, hi = f.b;                                 // lower_bound in B_t
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (f.Bd[mid] < j) lo = mid + 1; else hi = mid;
                }
                if (lo >= f.b || f.Bd[lo] != j) continue;            // not in this front
                q = f.s + lo;
            } else {
                continue;                                            // a descendant's DOF
            }
            P[(int64_t)q * f.ldp + p] = (T)val[k];
        }
    }
}

// Extend-add of child number `ci` of every front of the level: U_c (lower) is added at
// the parent positions ea_c, into P (column inside I) or U (both in B).  One launch per
// child index keeps the accumulation order fixed and race-free (within one child the
// targets of distinct entries are distinct: ea_c is injective).
//
// U_c is taken in 32 x 32 tiles; a work unit is a run of up to EA_CH tiles of one tile
// row, walked by one CTA.  Entry (i, j), j <= i, lands at
// (max(p_i, p_j), min(p_i, p_j)); the entries with p_j <= p_i are written by a warp per tile
// row (target row p_i, columns p_j increasing along the warp), the others, through a
// shared-memory transpose, by a warp per tile column (target row p_j, columns p_i), so
// both kinds of update run along parent rows (p restricted to the child's DOFs inside
// I_p or inside B_p is increasing).  Each thread issues all reads of its 8 targets before
// writing, and the next tile is loaded while the current one is added.
constexpr int EA_T = 32;
constexpr int EA_CH = 16;

template <typename Tc, typename Tp>
__global__ void __launch_bounds__(256, 4) k_extend_add(const FrontDesc* __restrict__ parents, const FrontDesc* __restrict__ kids,
                                                    const int* __restrict__ child_slots, int ci) {
    __shared__ Tp tile[2][EA_T][EA_T + 1];
    const FrontDesc fp = parents[blockIdx.y];
    if (ci >= fp.child_count) return;
    const FrontDesc fc = kids[child_slots[fp.child_begin + ci]];
    const Tc* U = (const Tc*)fc.U;
    Tp* P = (Tp*)fp.P;
    Tp* Up = (Tp*)fp.U;
    const int b = fc.b;
    const int nt = (b + EA_T - 1) / EA_T;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    auto at = [&](int r, int c) -> Tp* {
        return c < fp.s ? P + (int64_t)r * fp.ldp + c : Up + (int64_t)(r - fp.s) * fp.ldu + (c - fp.s);
    };
    int buf = 0;
    const int nch = (nt + EA_CH - 1) / EA_CH;
    for (int64_t unit = blockIdx.x; unit < (int64_t)nt * nch; unit += gridDim.x) {
        const int I = (int)(unit / nch), Jb = (int)(unit % nch) * EA_CH;
        if (Jb > I) continue;
        const int Je = min(I, Jb + EA_CH - 1);
        {
            const int i0 = I * EA_T;
            const int pi_lane = i0 + lane < b ? fc.ea[i0 + lane] : -1;      // row i0 + lane
            int pi_q[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = i0 + warp + 8 * u;
                pi_q[u] = i < b ? fc.ea[i] : -1;
            }
            // tile (I, J): this thread's entries (i0 + warp + 8u, j0 + lane)
            Tp cur[4];
            int pj_lane, pj_q[4];
            auto load = [&](int J, Tp* v, int& pl, int* pq) {
                const int j0 = J * EA_T;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int i = i0 + warp + 8 * u, j = j0 + lane;
                    v[u] = (i < b && j <= i) ? (Tp)U[(int64_t)i * fc.ldu + j] : (Tp)0;
                    pq[u] = j0 + warp + 8 * u < b ? fc.ea[j0 + warp + 8 * u] : -1;
                }
                pl = j0 + lane < b ? fc.ea[j0 + lane] : -1;
            };
            load(Jb, cur, pj_lane, pj_q);
            for (int J = Jb; J <= Je; ++J) {
                const int j0 = J * EA_T;
#pragma unroll
                for (int u = 0; u < 4; ++u) tile[buf][warp + 8 * u][lane] = cur[u];
                __syncthreads();
                Tp nxt[4];
                int nl = -1, nq[4] = {-1, -1, -1, -1};
                if (J < Je) load(J + 1, nxt, nl, nq);
                Tp* dst[8];
                Tp val[8];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int q = warp + 8 * u;
                    {                                      // rows: p_j <= p_i
                        const int i = i0 + q, j = j0 + lane;
                        const bool ok = i < b && j <= i && pj_lane <= pi_q[u];
                        dst[u] = ok ? at(pi_q[u], pj_lane) : nullptr;
                        val[u] = cur[u];
                    }
                    {                                      // columns: p_j > p_i
                        const int i = i0 + lane, j = j0 + q;
                        const bool ok = i < b && j <= i && pj_q[u] > pi_lane;
                        dst[4 + u] = ok ? at(pj_q[u], pi_lane) : nullptr;
                        val[4 + u] = tile[buf][lane][q];
                    }
                }
                Tp old[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) old[u] = dst[u] ? *dst[u] : (Tp)0;
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (dst[u]) *dst[u] = old[u] + val[u];
#pragma unroll
                for (int u = 0; u < 4; ++u) { cur[u] = nxt[u]; pj_q[u] = nq[u]; }
                pj_lane = nl;
                buf ^= 1;
            }
        }
    }
}

// ---------------------------------------------------------------------------------
// SIMT batched GEMM:  C = beta*C + alpha * A B^T, 64x64 tiles, 256 threads, 4x4 per thread.
// ---------------------------------------------------------------------------------
constexpr int SB = 64;     // tile edge
constexpr int WOUT = 4 * NB;   // outer panel width of the two-level left-looking update
template <typename T> struct SimtK { static constexpr int BK = 16; };
template <> struct SimtK<float> { static constexpr int BK = 32; };

__device__ __forceinline__ int find_task(const GemmTask* tasks, int ntask, int g) {
    int lo = 0, hi = ntask - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tasks[mid].tile_begin <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void decode_tile(const GemmTask& tk, int local, int& tm, int& tn) {
    if (tk.lower) {
        int r = (int)((sqrtf(8.0f * local + 1.0f) - 1.0f) * 0.5f);
        while ((r + 1) * (r + 2) / 2 <= local) ++r;
        while (r * (r + 1) / 2 > local) --r;
        tm = r;
        tn = local - r * (r + 1) / 2;
    } else {
        tm = local / tk.tiles_n;
        tn = local % tk.tiles_n;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_gemm_simt(const GemmTask* __restrict__ tasks, int ntask, T alpha) {
    constexpr int BK = SimtK<T>::BK;
    __shared__ T As[BK][SB + 1];
    __shared__ T Bs[BK][SB + 1];
    const int ti = find_task(tasks, ntask, blockIdx.x);
    const GemmTask tk = tasks[ti];
    int tm, tn;
    decode_tile(tk, blockIdx.x - tk.tile_begin, tm, tn);
    const int m0 = tm * SB, n0 = tn * SB;
    const T* A = (const T*)tk.A;
    const T* B = (const T*)tk.B;
    T* C = (T*)tk.C;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0;
    for (int k0 = 0; k0 < tk.K; k0 += BK) {
        for (int e = threadIdx.x; e < SB * BK; e += 256) {
            const int r = e / BK, kk = e % BK;
            const int gk = k0 + kk;
            const int ga = m0 + r, gb = n0 + r;
            As[kk][r] = (ga < tk.M && gk < tk.K) ? A[(int64_t)ga * tk.lda + gk] : (T)0;
            Bs[kk][r] = (gb < tk.N && gk < tk.K) ? B[(int64_t)gb * tk.ldb + gk] : (T)0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) { a[u] = As[kk][ty + 16 * u]; b[u] = Bs[kk][tx + 16 * u]; }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int r = m0 + ty + 16 * u;
        if (r >= tk.M) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int c = n0 + tx + 16 * v;
            if (c >= tk.N || (tk.lower && c > r)) continue;
            T* pc = C + (int64_t)r * tk.ldc + c;
            *pc = tk.beta ? (*pc + alpha * acc[u][v]) : alpha * acc[u][v];
        }
    }
}

// ---------------------------------------------------------------------------------
// Diagonal block: Cholesky of P[k:k+w, k:k+w] (w <= NB), written back to P, and its
// inverse stored as Dinv_k (NB x NB, zero padded).  One CTA per front whose interface
// extends past k.  The block lives in registers, distributed over a 16 x 16 thread grid:
// thread (tr, tc) holds e[a][b] = A[16a + tr][16b + tc].  The factorisation takes NB
// right-looking column steps (the owners of column j broadcast it through shared memory,
// every thread updates its 8 x 8 elements); the inverse takes NB right-looking row steps
// of X = L^-1 on the identity.  Entries above the diagonal of the broadcast vectors are
// zero, so the full-square updates leave finished columns intact; the upper triangle of
// the register block is never read back.  Beyond w the block is padded with the identity.
// ---------------------------------------------------------------------------------
constexpr int DLD = NB + 1;     // shared-memory row stride of L

template <typename T> __device__ __forceinline__ T rsqrt_t(T x);
template <> __device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double rsqrt_t(double x) { return 1.0 / sqrt(x); }

template <typename T>
__device__ __forceinline__ T store_round(T x, bool rnd);
template <>
__device__ __forceinline__ double store_round(double x, bool) { return x; }
template <>
__device__ __forceinline__ float store_round(float x, bool rnd) {
    if (!rnd) return x;
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

template <typename T>
__global__ void __launch_bounds__(256) k_potrf_diag(const FrontDesc* __restrict__ fronts, int k,
                                                   int* __restrict__ err, int round_tf32, int* __restrict__ bad_front) {
    extern __shared__ unsigned char smem_raw[];
    T* A = (T*)smem_raw;                 // L after the factorisation (upper part zero)
    T* vb = A + NB * DLD;                // two broadcast vectors
    const FrontDesc f = fronts[blockIdx.x];
    if (f.s <= k) return;
    const int w = min(NB, f.s - k);
    const int tid = threadIdx.x, tr = tid >> 4, tc = tid & 15;
    T* P = (T*)f.P;
    T e[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const int i = 16 * a + tr, c = 16 * b + tc;
            e[a][b] = (i < w && c <= i) ? P[(int64_t)(k + i) * f.ldp + (k + c)] : (i == c ? (T)1 : (T)0);
        }
    int bad = 0;
    // ---- Cholesky ----
#pragma unroll
    for (int jb = 0; jb < 8; ++jb) {
#pragma unroll 1
        for (int jj = 0; jj < 16; ++jj) {
            const int j = 16 * jb + jj;
            T* col = vb + (j & 1) * NB;
            T own[8];
            if (tc == jj) {
#pragma unroll
                for (int a = 0; a < 8; ++a) {
                    own[a] = e[a][jb];
                    col[16 * a + tr] = (16 * a + tr >= j) ? own[a] : (T)0;
                }
            }
            __syncthreads();
            T d = col[j];
            if (!(d > (T)0)) { bad = 1; d = (T)1; }
            const T inv = rsqrt_t(d), inv2 = inv * inv;
            // rows and columns before block jb see a zero column entry, and entries right
            // of the diagonal block (b > a) are never read: update the rest only
            T ci[8], ck[8];
#pragma unroll
            for (int a = jb; a < 8; ++a) ci[a] = col[16 * a + tr] * inv2;
#pragma unroll
            for (int b = jb; b < 8; ++b) ck[b] = col[16 * b + tc];
#pragma unroll
            for (int a = jb; a < 8; ++a)
#pragma unroll
                for (int b = jb; b <= a; ++b) e[a][b] -= ci[a] * ck[b];
            if (tc == jj) {
#pragma unroll
                for (int a = 0; a < 8; ++a) {
                    const int i = 16 * a + tr;
                    e[a][jb] = i > j ? own[a] * inv : (i == j ? d * inv : own[a]);
                }
            }
        }
    }
    if (bad) {
        atomicExch(&err[ERR_NOT_SPD], 1);
        atomicMin(&err[ERR_NOT_SPD_NODE], f.node);
        bad_front[f.node] = 1;
    }
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const int i = 16 * a + tr, c = 16 * b + tc;
            A[i * DLD + c] = c <= i ? e[a][b] : (T)0;
            if (i < w && c <= i) P[(int64_t)(k + i) * f.ldp + (k + c)] = store_round(e[a][b], round_tf32 != 0);
        }
    // ---- inverse X = L^-1 ----
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) e[a][b] = (16 * a + tr == 16 * b + tc) ? (T)1 : (T)0;
    __syncthreads();
#pragma unroll
    for (int rb = 0; rb < 8; ++rb) {
#pragma unroll 1
        for (int rr = 0; rr < 16; ++rr) {
            const int r = 16 * rb + rr;
            T* row = vb + (r & 1) * NB;
            const T ir = (T)1 / A[r * DLD + r];
            if (tr == rr) {
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    e[rb][b] *= ir;
                    row[16 * b + tc] = e[rb][b];
                }
            }
            __syncthreads();
            // X[i][c] -= L[i][r] X[r][c] touches rows i > r (blocks a >= rb) and columns
            // c <= r (blocks b <= rb) only
            T li[8], xr[8];
#pragma unroll
            for (int a = rb; a < 8; ++a) li[a] = (16 * a + tr > r) ? A[(16 * a + tr) * DLD + r] : (T)0;
#pragma unroll
            for (int b = 0; b <= rb; ++b) xr[b] = row[16 * b + tc];
#pragma unroll
            for (int a = rb; a < 8; ++a)
#pragma unroll
                for (int b = 0; b <= rb; ++b) e[a][b] -= li[a] * xr[b];
        }
    }
    T* D = (T*)f.Dinv + (int64_t)(k / NB) * NB * NB;
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const int i = 16 * a + tr, c = 16 * b + tc;
            D[i * NB + c] = (i < w && c <= i) ? store_round(e[a][b], round_tf32 != 0) : (T)0;
        }
}

// ---------------------------------------------------------------------------------
// FP32 diagonal block, blocked by 32: the same result as k_potrf_diag (Cholesky of
// P[k:k+w, k:k+w] written back, its inverse to Dinv_k) with a short critical path.
// Shared memory holds the block A (L in its lower triangle), the inverse X, the current
// 32-column panel transposed (LT[m][r] = L[r][32J + m]), the current diagonal inverse
// transposed (XT[c][r] = X_JJ[r][c]) and the columns of L_JJ, rotated so that row j
// starts at the diagonal (LJ[j][p] = l_{j+p, j}, zero where j + p wraps past 31).
// Per panel J the critical chain is
//   (1) warp 0: Cholesky of the 32 x 32 diagonal sub-block, lane = row, right-looking;
//       the lane row sits in registers rotated so that the current column is always
//       a[0], and each finished column is published once to LJ;
//   (2) rows below: y_c = (a_c - sum_{m<c} y_m l_cm) / l_cc, a warp per 32 rows (lane = row),
//       while warp 7 forms X_JJ = L_JJ^-1 (lane = column) with the same rotated sweep;
//   (3) the next diagonal tile, A_{J+1,J+1} -= L_{J+1,J} L_{J+1,J}^T, 8 rows per warp;
// and while warp 0 factors panel J+1 the other seven warps finish panel J off the chain:
//   - the remaining trailing tiles A_IK -= L_IJ L_KJ^T;
//   - the inverse by block rows (from L X = I): X_JK = -X_JJ T_JK for K < J, then
//     T_IK += L_IJ X_JK for I > J, K <= J, where T_IK = sum_{K<=M<I} L_IM X_MK collects in
//     A's unused upper block (K, I);
//   - the finished panel of L and row block of the inverse go out to global memory.
// Tile products give each lane a 4 x 8 piece of the 32 x 32 result, three float4 shared
// loads per 32 FMAs.  All per-column loops are rolled (the kernel runs from a cold
// instruction cache between other kernels).
// ---------------------------------------------------------------------------------
constexpr int DB = 32;                  // sub-block width
constexpr int XLD = NB + 4;             // row stride of A, X and LT (16-byte rows, 4 banks apart)
constexpr int XTLD = DB + 4;            // row stride of XT
constexpr size_t POTRF_BLK_SMEM = (size_t)(2 * NB * XLD + DB * XLD + DB * XTLD + DB * DB) * sizeof(float);

__device__ __forceinline__ float tf32_store(float x, bool rnd) {
    if (!rnd) return x;
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ float4 lds4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void sts4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }

__device__ __forceinline__ void load_row32(const float* __restrict__ row, float (&v)[DB]) {
#pragma unroll
    for (int t = 0; t < DB / 4; ++t) {
        const float4 q = lds4(row + 4 * t);
        v[4 * t + 0] = q.x; v[4 * t + 1] = q.y; v[4 * t + 2] = q.z; v[4 * t + 3] = q.w;
    }
}

__device__ __forceinline__ void store_row32(float* __restrict__ row, const float (&v)[DB]) {
#pragma unroll
    for (int t = 0; t < DB / 4; ++t) sts4(row + 4 * t, make_float4(v[4 * t], v[4 * t + 1], v[4 * t + 2], v[4 * t + 3]));
}

// v[p-1] = v[p] - y * col[p] for p = 1..31 (col: a 16-byte aligned shared row), v[31] = y
__device__ __forceinline__ void rotate_update32(float (&v)[DB], const float* __restrict__ col, float y) {
#pragma unroll
    for (int t = 0; t < DB / 4; ++t) {
        const float4 c4 = lds4(col + 4 * t);
        if (t > 0) v[4 * t - 1] = fmaf(-y, c4.x, v[4 * t]);
        v[4 * t + 0] = fmaf(-y, c4.y, v[4 * t + 1]);
        v[4 * t + 1] = fmaf(-y, c4.z, v[4 * t + 2]);
        v[4 * t + 2] = fmaf(-y, c4.w, v[4 * t + 3]);
    }
    v[DB - 1] = y;
}

// v[p-1] = v[p] - y * c[p] for p = 1..31 (c: one column held in registers), v[31] = y
__device__ __forceinline__ void rotate_update32_reg(float (&v)[DB], const float4 (&c)[DB / 4], float y) {
#pragma unroll
    for (int t = 0; t < DB / 4; ++t) {
        if (t > 0) v[4 * t - 1] = fmaf(-y, c[t].x, v[4 * t]);
        v[4 * t + 0] = fmaf(-y, c[t].y, v[4 * t + 1]);
        v[4 * t + 1] = fmaf(-y, c[t].z, v[4 * t + 2]);
        v[4 * t + 2] = fmaf(-y, c[t].w, v[4 * t + 3]);
    }
    v[DB - 1] = y;
}

__device__ __forceinline__ void load_col32(float4 (&c)[DB / 4], const float* __restrict__ col) {
#pragma unroll
    for (int t = 0; t < DB / 4; ++t) c[t] = lds4(col + 4 * t);
}

// Forward substitution with L_JJ, one right-hand side per lane: on entry v[p] = b_p, on
// return v[p] = x_p with x_c = (b_c - sum_{m<c} l_cm x_m) * scale[c].  Two columns per
// trip, each column's loads issued one step ahead of its use.
__device__ __forceinline__ void fsub32(float (&v)[DB], const float* __restrict__ LJ, const float* __restrict__ scale) {
    float4 ca[DB / 4], cb[DB / 4];
    load_col32(ca, LJ);
    float sa = scale[0], sb;
#pragma unroll 1
    for (int c = 0; c < DB; c += 2) {
        load_col32(cb, LJ + (c + 1) * DB);
        sb = scale[c + 1];
        rotate_update32_reg(v, ca, v[0] * sa);
        const int cn = (c + 2) & (DB - 1);            // the last trip prefetches column 0 again, unused
        load_col32(ca, LJ + cn * DB);
        sa = scale[cn];
        rotate_update32_reg(v, cb, v[0] * sb);
    }
}

// warp 0's step (1) for the diagonal sub-block at (o, o); returns 1 on a pivot that is not
// positive (replaced by 1 so that the rest stays finite).
// Lane i keeps A_j[i][j..], its row as updated by columns < j, rotated so that position p
// holds column j + p; finished entries l_i0..l_ij collect at the top and rotate down with
// the rest (the column entries that move them are zero).  The loop is software-pipelined:
// step j + 1's pivot chain runs ahead of step j's bulk update.  It needs column j + 1 and
// j + 2 after step j (a0n, a1n: from l_{j+1,j}, l_{j+2,j} by shuffle) and column j + 3 (one
// entry of the bulk update); the next pivot comes from lane j + 1's own update.
__device__ __forceinline__ int potrf_chol32(float* __restrict__ A, float* __restrict__ LJ, float* __restrict__ s_rs,
                                            float* __restrict__ s_ri, int o, int lane) {
    const unsigned full = 0xffffffffu;
    float a[DB];
    load_row32(A + (o + lane) * XLD + o, a);
    int bad = 0;
    float my_inv = 1.0f, my_ljj = 1.0f;
    // step 0's chain
    float d = __shfl_sync(full, a[0], 0);
    if (!(d > 0.0f)) { bad = 1; d = 1.0f; }
    float inv = rsqrtf(d);
    float lij = lane > 0 ? a[0] * inv : (lane == 0 ? d * inv : 0.0f);
    my_inv = lane == 0 ? inv : my_inv;
    my_ljj = lane == 0 ? d * inv : my_ljj;
    float dn = __shfl_sync(full, fmaf(-lij, lij, a[1]), 1);
    float a0n = fmaf(-lij, __shfl_sync(full, lij, 1), a[1]);
    float a1n = fmaf(-lij, __shfl_sync(full, lij, 2), a[2]);
#pragma unroll 1
    for (int j = 0; j < DB; ++j) {
        // (A) publish column j, fetch it back
        float* col = LJ + j * DB;
        col[(lane - j) & (DB - 1)] = lij;
        __syncwarp();
        float4 c[DB / 4];
#pragma unroll
        for (int t = 0; t < DB / 4; ++t) c[t] = lds4(col + 4 * t);
        // (B) step j + 1's chain (discarded after the last step)
        const float a2n = fmaf(-lij, c[0].w, a[3]);              // column j + 3 after step j
        const int j1 = j + 1;
        float d1 = dn;
        if (!(d1 > 0.0f)) { if (j1 < DB) bad = 1; d1 = 1.0f; }
        const float inv1 = rsqrtf(d1);
        const float ljj1 = d1 * inv1;
        const float lij1 = lane > j1 ? a0n * inv1 : (lane == j1 ? ljj1 : 0.0f);
        my_inv = lane == j1 ? inv1 : my_inv;
        my_ljj = lane == j1 ? ljj1 : my_ljj;
        dn = __shfl_sync(full, fmaf(-lij1, lij1, a1n), (j1 + 1) & (DB - 1));
        const float l1 = __shfl_sync(full, lij1, (j1 + 1) & (DB - 1));
        const float l2 = __shfl_sync(full, lij1, (j1 + 2) & (DB - 1));
        // (C) step j's bulk update: columns j + 4 .. j + 31 move down one position
#pragma unroll
        for (int t = 1; t < DB / 4; ++t) {
            a[4 * t - 1] = fmaf(-lij, c[t].x, a[4 * t]);
            a[4 * t + 0] = fmaf(-lij, c[t].y, a[4 * t + 1]);
            a[4 * t + 1] = fmaf(-lij, c[t].z, a[4 * t + 2]);
            a[4 * t + 2] = fmaf(-lij, c[t].w, a[4 * t + 3]);
        }
        a[DB - 1] = lij;
        a[0] = a0n;
        a[1] = a1n;
        a[2] = a2n;
        // step j + 1's first two columns after its own update
        a0n = fmaf(-lij1, l1, a1n);
        a1n = fmaf(-lij1, l2, a2n);
        lij = lij1;
    }
    s_rs[o + lane] = my_inv;
    s_ri[o + lane] = 1.0f / my_ljj;
    store_row32(A + (o + lane) * XLD + o, a);         // zero above the diagonal
    return bad;
}

// C (32 x 32, row stride ldc) = [C +] sgn * sum_{m<32} AT[m][r] B[m][c]; lane tile rows
// 4 (lane >> 2) + 0..3, columns 8 (lane & 3) + 0..7
template <bool ACC>
__device__ __forceinline__ void tile32_atb(const float* __restrict__ AT, int lda, const float* __restrict__ B, int ldb,
                                           float* __restrict__ C, int ldc, float sgn, int lane) {
    const int r0 = 4 * (lane >> 2), c0 = 8 * (lane & 3);
    float acc[4][8];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
#pragma unroll 4
    for (int m = 0; m < DB; ++m) {
        const float4 a = lds4(AT + m * lda + r0);
        const float4 b0 = lds4(B + m * ldb + c0), b1 = lds4(B + m * ldb + c0 + 4);
        const float av[4] = {a.x, a.y, a.z, a.w};
        const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float* row = C + (r0 + i) * ldc + c0;
        float4 o0 = make_float4(0.0f, 0.0f, 0.0f, 0.0f), o1 = o0;
        if (ACC) { o0 = lds4(row); o1 = lds4(row + 4); }
        o0.x = fmaf(sgn, acc[i][0], o0.x); o0.y = fmaf(sgn, acc[i][1], o0.y);
        o0.z = fmaf(sgn, acc[i][2], o0.z); o0.w = fmaf(sgn, acc[i][3], o0.w);
        o1.x = fmaf(sgn, acc[i][4], o1.x); o1.y = fmaf(sgn, acc[i][5], o1.y);
        o1.z = fmaf(sgn, acc[i][6], o1.z); o1.w = fmaf(sgn, acc[i][7], o1.w);
        sts4(row, o0);
        sts4(row + 4, o1);
    }
}

// rows 8 ch + 0..7 of C (32 x 32) -= sum_m AT[m][r] B[m][c]; lane tile 2 rows x 4 columns
__device__ __forceinline__ void chunk8_atb_sub(const float* __restrict__ AT, int lda, const float* __restrict__ B, int ldb,
                                               float* __restrict__ C, int ldc, int ch, int lane) {
    const int r0 = 8 * ch + 2 * (lane >> 3), c0 = 4 * (lane & 7);
    float acc[2][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
#pragma unroll 8
    for (int m = 0; m < DB; ++m) {
        const float2 a = *reinterpret_cast<const float2*>(AT + m * lda + r0);
        const float4 b = lds4(B + m * ldb + c0);
        const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            acc[0][j] = fmaf(a.x, bv[j], acc[0][j]);
            acc[1][j] = fmaf(a.y, bv[j], acc[1][j]);
        }
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        float* row = C + (r0 + i) * ldc + c0;
        float4 o = lds4(row);
        o.x -= acc[i][0]; o.y -= acc[i][1]; o.z -= acc[i][2]; o.w -= acc[i][3];
        sts4(row, o);
    }
}

// Panel K of L (rows 32K..w-1, columns 32K..32K+31, on or below the diagonal) to P
__device__ __forceinline__ void potrf_store_panel(const float* __restrict__ A, float* __restrict__ P, int64_t ldp, int k,
                                                  int w, int K, bool rnd, int t0, int nt) {
    const int r_lo = DB * K;
    for (int e = t0; e < (NB - r_lo) * (DB / 4); e += nt) {
        const int i = r_lo + e / (DB / 4), c = r_lo + 4 * (e % (DB / 4));
        if (i >= w || c > i) continue;
        const float4 l = lds4(A + i * XLD + c);
        float* dst = P + (int64_t)(k + i) * ldp + k + c;
        if (c + 3 <= i) {
            *reinterpret_cast<float4*>(dst) = make_float4(tf32_store(l.x, rnd), tf32_store(l.y, rnd), tf32_store(l.z, rnd), tf32_store(l.w, rnd));
        } else {
            dst[0] = tf32_store(l.x, rnd);
            if (c + 1 <= i) dst[1] = tf32_store(l.y, rnd);
            if (c + 2 <= i) dst[2] = tf32_store(l.z, rnd);
        }
    }
}

// Row block K of the inverse (rows 32K..32K+31, all 128 columns, zero above the diagonal
// and in rows past the front) to D
__device__ __forceinline__ void potrf_store_inverse(const float* __restrict__ X, float* __restrict__ D, int w, int K,
                                                    bool rnd, int t0, int nt) {
    for (int e = t0; e < DB * (NB / 4); e += nt) {
        const int i = DB * K + e / (NB / 4), c = 4 * (e % (NB / 4));
        float4 dv = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (i < w && c <= i) {
            const float4 x = lds4(X + i * XLD + c);
            dv.x = tf32_store(x.x, rnd);
            dv.y = c + 1 <= i ? tf32_store(x.y, rnd) : 0.0f;
            dv.z = c + 2 <= i ? tf32_store(x.z, rnd) : 0.0f;
            dv.w = c + 3 <= i ? tf32_store(x.w, rnd) : 0.0f;
        }
        *reinterpret_cast<float4*>(D + i * NB + c) = dv;
    }
}

struct PotrfOut {
    float* P;
    int64_t ldp;
    float* D;
    int k, w;
    bool rnd;
};

// panel K's work off the critical chain, by nw warps (index wi).  Part 1: trailing tiles
// and the finalised X row block K (warps left over store panel K of L); a named barrier
// over the nw warps (bar_id > 0); part 2: T accumulation (warps left over store row
// block K of the inverse).  With K = 3 only part 1 runs and nothing is stored.
__device__ __forceinline__ void potrf_background(float* __restrict__ A, float* __restrict__ X, const float* __restrict__ LT,
                                                 const float* __restrict__ XT, const PotrfOut& out, int K, int wi, int nw,
                                                 int bar_id, int lane) {
    constexpr int NBB = NB / DB;
    int ntrail = 0;                                   // trailing tiles except (K+1, K+1)
    for (int bk = K + 1; bk < NBB; ++bk) ntrail += NBB - bk;
    if (ntrail > 0) --ntrail;
    const int n1 = ntrail + K;
    for (int it = wi; it < n1; it += nw) {
        if (it < ntrail) {
            int cnt = 0, bi = 0, bk = 0;
            for (int q = K + 1; q < NBB; ++q)
                for (int p = q; p < NBB; ++p) {
                    if (p == K + 1 && q == K + 1) continue;
                    if (cnt == it) { bi = p; bk = q; }
                    ++cnt;
                }
            tile32_atb<true>(LT + DB * bi, XLD, LT + DB * bk, XLD, A + DB * bi * XLD + DB * bk, XLD, -1.0f, lane);
        } else {
            const int J = it - ntrail;                    // X_KJ = -X_KK T_KJ, T_KJ in A's block (J, K)
            tile32_atb<false>(XT, XTLD, A + DB * J * XLD + DB * K, XLD, X + DB * K * XLD + DB * J, XLD, -1.0f, lane);
        }
    }
    if (K + 1 >= NBB) return;
    if (wi >= n1) potrf_store_panel(A, out.P, out.ldp, out.k, out.w, K, out.rnd, 32 * (wi - n1) + lane, 32 * (nw - n1));
    if (bar_id > 0) asm volatile("bar.sync %0, %1;" :: "r"(bar_id), "r"(32 * nw) : "memory");
    const int n2 = (NBB - 1 - K) * (K + 1);           // T_IJ += L_IK X_KJ, I > K, J <= K
    for (int it = wi; it < n2; it += nw) {
        const int I = K + 1 + it / (K + 1), J = it % (K + 1);
        tile32_atb<true>(LT + DB * I, XLD, X + DB * K * XLD + DB * J, XLD, A + DB * J * XLD + DB * I, XLD, 1.0f, lane);
    }
    if (wi >= n2) potrf_store_inverse(X, out.D, out.w, K, out.rnd, 32 * (wi - n2) + lane, 32 * (nw - n2));
}

// rows [r_lo, r_hi) of the block into A (lower part; zero above the diagonal; identity
// rows past the front), float4 loads, nt threads (index ti), all loads before the stores
template <int MAXV>
__device__ __forceinline__ void potrf_load_rows(float* __restrict__ A, const float* __restrict__ P, int64_t ldp, int k, int w,
                                                int r_lo, int r_hi, int ti, int nt) {
    const int n4 = (r_hi - r_lo) * (NB / 4);
    float4 v[MAXV];
#pragma unroll
    for (int u = 0; u < MAXV; ++u) {
        const int e = ti + nt * u;
        v[u] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (e < n4) {
            const int i = r_lo + e / (NB / 4), c = 4 * (e % (NB / 4));
            if (i < w && c <= i) v[u] = *reinterpret_cast<const float4*>(P + (int64_t)(k + i) * ldp + k + c);
        }
    }
#pragma unroll
    for (int u = 0; u < MAXV; ++u) {
        const int e = ti + nt * u;
        if (e < n4) {
            const int i = r_lo + e / (NB / 4), c = 4 * (e % (NB / 4));
            float4 q = v[u];
            if (i < w) {
                if (c + 0 > i) q.x = 0.0f;
                if (c + 1 > i) q.y = 0.0f;
                if (c + 2 > i) q.z = 0.0f;
                if (c + 3 > i) q.w = 0.0f;
            } else {
                q = make_float4(c + 0 == i ? 1.0f : 0.0f, c + 1 == i ? 1.0f : 0.0f, c + 2 == i ? 1.0f : 0.0f, c + 3 == i ? 1.0f : 0.0f);
            }
            sts4(A + i * XLD + c, q);
        }
    }
}

__global__ void __launch_bounds__(256, 1) k_potrf_diag_blk(const FrontDesc* __restrict__ fronts, int k,
                                                       int* __restrict__ err, int round_tf32, int* __restrict__ bad_front) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* A = (float*)smem_raw;                  // 128 x XLD
    float* X = A + NB * XLD;                      // 128 x XLD
    float* LT = X + NB * XLD;                     // 32 x XLD
    float* XT = LT + DB * XLD;                    // 32 x XTLD
    float* LJ = XT + DB * XTLD;                   // 32 x 32
    __shared__ float s_rs[NB];                    // 1 / sqrt(pivot): scales the column below
    __shared__ float s_ri[NB];                    // 1 / l_jj
    __shared__ int s_bad;
    const FrontDesc f = fronts[blockIdx.x];
    if (f.s <= k) return;
    const int w = min(NB, f.s - k);
    const PotrfOut out{(float*)f.P, (int64_t)f.ldp, (float*)f.Dinv + (int64_t)(k / NB) * NB * NB, k, w, round_tf32 != 0};
    const float* P = (const float*)f.P;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_bad = 0;
    potrf_load_rows<4>(A, P, f.ldp, k, w, 0, DB, tid, 256);
    __syncthreads();
    for (int J = 0; J < NB / DB; ++J) {
        const int o = J * DB;
        const int nb_below = NB / DB - 1 - J;
        if (warp == 0) {
            if (potrf_chol32(A, LJ, s_rs, s_ri, o, lane) && lane == 0) s_bad = 1;
        } else if (J == 0) {
            // rows 32..127 in three batches of 32 rows (1024 float4, five per thread)
            for (int r0 = DB; r0 < NB; r0 += DB) potrf_load_rows<5>(A, P, f.ldp, k, w, r0, r0 + DB, tid - 32, 224);
        } else {
            potrf_background(A, X, LT, XT, out, J - 1, warp - 1, 7, 1, lane);
        }
        __syncthreads();
        if (warp < nb_below) {
            // (2) rows o + 32 (warp + 1) + lane, into A and transposed into LT
            const int r = o + DB * (warp + 1) + lane;
            float y[DB];
            load_row32(A + r * XLD + o, y);
            fsub32(y, LJ, s_rs + o);
            store_row32(A + r * XLD + o, y);
#pragma unroll
            for (int m = 0; m < DB; ++m) LT[m * XLD + r] = y[m];
        } else if (warp == 7) {
            // (2') X_JJ = L_JJ^-1, lane c forms column c
            float x[DB];
#pragma unroll
            for (int p = 0; p < DB; ++p) x[p] = p == lane ? 1.0f : 0.0f;
            fsub32(x, LJ, s_ri + o);
#pragma unroll
            for (int r = 0; r < DB; ++r) X[(o + r) * XLD + o + lane] = x[r];
            store_row32(XT + lane * XTLD, x);
        }
        __syncthreads();
        if (nb_below > 0) {
            // (3) the next diagonal tile, 8 rows per warp
            if (warp < 4) chunk8_atb_sub(LT + o + DB, XLD, LT + o + DB, XLD, A + (o + DB) * XLD + o + DB, XLD, warp, lane);
            __syncthreads();
        }
    }
    // the last X row block, the last panel of L (warps left over), then the last inverse rows
    potrf_background(A, X, LT, XT, out, NB / DB - 1, warp, 8, 0, lane);
    if (warp >= NB / DB - 1) potrf_store_panel(A, out.P, out.ldp, k, w, NB / DB - 1, out.rnd, 32 * (warp - (NB / DB - 1)) + lane, 32 * (8 - (NB / DB - 1)));
    __syncthreads();
    potrf_store_inverse(X, out.D, w, NB / DB - 1, out.rnd, tid, 256);
    if (tid == 0 && s_bad) {
        atomicExch(&err[ERR_NOT_SPD], 1);
        atomicMin(&err[ERR_NOT_SPD_NODE], f.node);
        bad_front[f.node] = 1;
    }
}

// ---------------------------------------------------------------------------------
// Panel solve in place: rows P[k+w:N, k:k+w] <- rows * Dinv_k^T (Dinv_k lower triangular).
// Each CTA owns 32 full-width rows, so reading and overwriting them cannot race.
// ---------------------------------------------------------------------------------
constexpr int TR_ROWS = 32;
template <typename T>
__global__ void __launch_bounds__(256) k_trsm_simt(const FrontDesc* __restrict__ fronts, int k, int sel) {
    extern __shared__ unsigned char smem_raw[];
    T* D = (T*)smem_raw;                     // NB x NB
    T* R = D + NB * NB;                      // TR_ROWS x (NB + 1)
    constexpr int LDR = NB + 1;
    const FrontDesc f = fronts[blockIdx.y];
    if (f.s <= k) return;
    const int w = min(NB, f.s - k);
    const int r0 = k + w + blockIdx.x * TR_ROWS;
    if (r0 >= f.N) return;
    const int nr = min(TR_ROWS, f.N - r0);
    // sel 0: (P, Dinv); nonsymmetric fronts: 1 = (P, DinvU), 2 = (PU, Dinv)
    const T* Dg = (const T*)(sel == 1 ? f.DinvU : f.Dinv) + (int64_t)(k / NB) * NB * NB;
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) D[e] = Dg[e];
    T* P = (T*)(sel == 2 ? f.PU : f.P);
    for (int e = threadIdx.x; e < TR_ROWS * NB; e += blockDim.x) {
        const int r = e / NB, c = e % NB;
        R[r * LDR + c] = (r < nr && c < w) ? P[(int64_t)(r0 + r) * f.ldp + k + c] : (T)0;
    }
    __syncthreads();
    // thread -> (row group of 4, column group of 4): 8 x 32 threads
    const int rg = threadIdx.x >> 5, cg = threadIdx.x & 31;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0;
    for (int l = 0; l < w; ++l) {
        T a[4], d[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) a[u] = R[(rg + 8 * u) * LDR + l];
#pragma unroll
        for (int v = 0; v < 4; ++v) d[v] = D[(cg + 32 * v) * NB + l];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], d[v], acc[u][v]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int r = rg + 8 * u;
        if (r >= nr) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int c = cg + 32 * v;
            if (c < w) P[(int64_t)(r0 + r) * f.ldp + k + c] = acc[u][v];
        }
    }
}

double gemm_flops(const std::vector<GemmTask>& tasks) {
    double f = 0;
    for (auto& t : tasks)
        f += t.lower ? (double)t.M * (t.M + 1) * t.K : 2.0 * t.M * t.N * t.K;
    return f;
}

double gemm_bytes(const std::vector<GemmTask>& tasks, size_t es) {
    double b = 0;
    for (auto& t : tasks) {
        const double c = t.lower ? 0.5 * t.M * (t.M + 1.0) : (double)t.M * t.N;
        b += es * ((double)t.M * t.K + (t.A == t.B && t.lower ? 0.0 : (double)t.N * t.K) + c * (t.beta ? 2 : 1));
    }
    return b;
}

template <typename T>
int launch_gemm_simt(Handle& h, const std::vector<GemmTask>& tasks, GemmTask* d_tasks, T alpha, cudaStream_t st) {
    if (tasks.empty()) return RSD_OK;
    RSD_CUDA_TRY(cudaMemcpyAsync(d_tasks, stage_host(h, tasks.data(), tasks.size() * sizeof(GemmTask)),
                                 tasks.size() * sizeof(GemmTask), cudaMemcpyHostToDevice, st));
    const GemmTask& last = tasks.back();
    const int tiles_last = last.lower ? ((last.M + SB - 1) / SB) * ((last.M + SB - 1) / SB + 1) / 2
                                      : ((last.M + SB - 1) / SB) * last.tiles_n;
    const int total = last.tile_begin + tiles_last;
    if (total <= 0) return RSD_OK;
    const int pi = prof_begin(h, K_GEMM_SIMT);
    k_gemm_simt<T><<<total, 256, 0, st>>>(d_tasks, (int)tasks.size(), alpha);
    count_launch();
    prof_end(h, pi, gemm_flops(tasks), gemm_bytes(tasks, sizeof(T)));
    RSD_CUDA_TRY(cudaGetLastError());
    return RSD_OK;
}

// Fill tile bookkeeping of a task list for tile edge `tile`; returns total tiles.
int finalize_tasks(std::vector<GemmTask>& tasks, int tile_m, int tile_n) {
    int total = 0;
    for (auto& t : tasks) {
        const int tm = (t.M + tile_m - 1) / tile_m;
        const int tn = (t.N + tile_n - 1) / tile_n;
        t.tiles_n = tn;
        t.tile_begin = total;
        total += t.lower ? tm * (tm + 1) / 2 : tm * tn;
    }
    return total;
}

// Peak probe of the CUDA-core GEMM: C -= A B^T on one n x n x n product, best of `reps`
// launches and the mean over back-to-back launches for about `seconds`.
template <typename T>
__global__ void k_fill_hash_t(T* __restrict__ p, int64_t n, uint32_t seed) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t x = (uint32_t)i * 2654435761u ^ seed;
        x ^= x >> 16; x *= 0x7feb352du; x ^= x >> 15; x *= 0x846ca68bu; x ^= x >> 16;
        p[i] = (T)((double)(x >> 8) * (1.0 / 8388608.0) - 1.0);
    }
}

template <typename T>
int gemm_simt_peak_t(int n, int reps, double seconds, cudaStream_t st, double* best, double* sustained) {
    const size_t elems = (size_t)n * n;
    std::vector<GemmTask> tasks(1);
    char* buf = nullptr;
    const size_t o_b = elems * sizeof(T), o_c = 2 * elems * sizeof(T), o_t = 3 * elems * sizeof(T);
    RSD_CUDA_TRY(cudaMalloc((void**)&buf, o_t + 256));
    struct Free { char* p; ~Free() { cudaFree(p); } } fr{buf};
    T* A = (T*)buf;
    k_fill_hash_t<T><<<1024, 256, 0, st>>>(A, (int64_t)elems, 0x9e3779b9u);
    k_fill_hash_t<T><<<1024, 256, 0, st>>>((T*)(buf + o_b), (int64_t)elems, 0x7f4a7c15u);
    RSD_CUDA_TRY(cudaMemsetAsync(buf + o_c, 0, elems * sizeof(T), st));
    GemmTask& t = tasks[0];
    t = GemmTask{};
    t.A = A; t.B = buf + o_b; t.C = buf + o_c;
    t.lda = t.ldb = t.ldc = n;
    t.M = t.N = t.K = n;
    t.lower = 0; t.beta = 1;
    const int total = finalize_tasks(tasks, SB, SB);
    RSD_CUDA_TRY(cudaMemcpyAsync(buf + o_t, tasks.data(), sizeof(GemmTask), cudaMemcpyHostToDevice, st));
    const GemmTask* dt = (const GemmTask*)(buf + o_t);
    auto launch = [&]() { k_gemm_simt<T><<<total, 256, 0, st>>>(dt, 1, (T)-1); count_launch(); };
    cudaEvent_t e0, e1;
    RSD_CUDA_TRY(cudaEventCreate(&e0));
    RSD_CUDA_TRY(cudaEventCreate(&e1));
    struct Ev { cudaEvent_t a, b; ~Ev() { cudaEventDestroy(a); cudaEventDestroy(b); } } ev{e0, e1};
    launch();
    float bms = 1e30f;
    for (int r = 0; r < reps; ++r) {
        RSD_CUDA_TRY(cudaEventRecord(e0, st));
        launch();
        RSD_CUDA_TRY(cudaEventRecord(e1, st));
        RSD_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0;
        RSD_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        bms = std::min(bms, ms);
    }
    const int loops = std::max(1, (int)(seconds * 1e3 / std::max(bms, 1e-3f)));
    RSD_CUDA_TRY(cudaEventRecord(e0, st));
    for (int r = 0; r < loops; ++r) launch();
    RSD_CUDA_TRY(cudaEventRecord(e1, st));
    RSD_CUDA_TRY(cudaEventSynchronize(e1));
    float tms = 0;
    RSD_CUDA_TRY(cudaEventElapsedTime(&tms, e0, e1));
    RSD_CUDA_TRY(cudaGetLastError());
    const double flops = 2.0 * n * (double)n * n;
    *best = flops / (bms * 1e-3) / 1e12;
    *sustained = flops * loops / (tms * 1e-3) / 1e12;
    return RSD_OK;
}

}  // namespace

int gemm_simt_peak(int prec, int n, int reps, double seconds, cudaStream_t st, double* best, double* sustained) {
    if (n < 64 || n % 64 || reps < 1 || !best || !sustained) return RSD_ERR_ARG;
    if (prec == RSD_PREC_FP64) return gemm_simt_peak_t<double>(n, reps, seconds, st, best, sustained);
    if (prec == RSD_PREC_FP32) return gemm_simt_peak_t<float>(n, reps, seconds, st, best, sustained);
    return RSD_ERR_ARG;
}

// Row scales of the FP16 factor copy: with sqrt(K_ii) = m 2^x, m in [0.5, 1), rs[i] =
// 2^(14 - x) puts sqrt(K_ii) rs[i] in [2^13, 2^14), a factor 4 below FP16's largest
// value, which bounds every entry of the row (the front's diagonal entry is a Schur
// complement's, at most K_ii).  ri[i] = 1 / rs[i] follows rs in memory.
__global__ void k_row_scale(const FrontDesc* __restrict__ fronts, const int64_t* __restrict__ rowptr,
                            const int* __restrict__ col, const double* __restrict__ val) {
    const FrontDesc f = fronts[blockIdx.x];
    float* rs = (float*)f.rs;
    for (int i = blockIdx.y * blockDim.x + threadIdx.x; i < f.N; i += gridDim.y * blockDim.x) {
        const int dof = i < f.s ? f.I[i] : f.Bd[i - f.s];
        double kii = 0.0;
        for (int64_t k = rowptr[dof]; k < rowptr[dof + 1]; ++k)
            if (col[k] == dof) { kii = val[k]; break; }
        int x = 0;
        if (kii > 0.0 && kii <= 1e300) frexp(sqrt(kii), &x);
        const int e = max(-120, min(120, 14 - x));
        rs[i] = ldexpf(1.0f, e);
        rs[f.N + i] = ldexpf(1.0f, -e);
    }
}

// Two values rounded to FP16 and packed in a word, the first in the low half (the lower
// address).
__device__ __forceinline__ uint32_t pack_h2(float lo, float hi) {
    return (uint32_t)__half_as_ushort(__float2half_rn(lo)) | ((uint32_t)__half_as_ushort(__float2half_rn(hi)) << 16);
}

// FP16 copy of the factor entries the sweeps read: row i, columns below its diagonal
// block (i < s) or all s columns (B rows), each scaled by rs[i].  One warp per row,
// eight entries (32 B in, 16 B out) per lane and step.  The entries are TF32 values, so
// the copy is exact wherever the scaled value is an FP16 normal.
__global__ void __launch_bounds__(256) k_copy16(const FrontDesc* __restrict__ fronts) {
    const FrontDesc f = fronts[blockIdx.x];
    const float* P = (const float*)f.P;
    __half* Q = (__half*)f.P16;
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int i = blockIdx.y * wpb + (threadIdx.x >> 5); i < f.N; i += gridDim.y * wpb) {
        const int cend = i < f.s ? (i / NB) * NB : f.s;
        const float sc = f.rs[i];
        const float* src = P + (int64_t)i * f.ldp;
        __half* dst = Q + (int64_t)i * f.ldp;
        for (int c = lane * 8; c < cend; c += 256) {
            if (c + 8 <= cend) {
                const float4 a = __ldcs((const float4*)(src + c)), b = __ldcs((const float4*)(src + c + 4));
                uint4 o;
                o.x = pack_h2(a.x * sc, a.y * sc);
                o.y = pack_h2(a.z * sc, a.w * sc);
                o.z = pack_h2(b.x * sc, b.y * sc);
                o.w = pack_h2(b.z * sc, b.w * sc);
                *reinterpret_cast<uint4*>(dst + c) = o;
            } else {
                for (int e = 0; c + e < cend; ++e) dst[c + e] = __float2half_rn(src[c + e] * sc);
            }
        }
    }
}

// 16-bit operand copy of one outer panel (columns [K0, K0 + WOUT)) of every front, once all
// its entries are final: the entries below the NB x NB diagonal blocks and the X rows, row
// i scaled by rs[i] (the same entries k_copy16 writes, panel by panel, so that the later
// panels' long-K updates can read them).  OUT is __half or __nv_bfloat16.
template <typename OUT> __device__ __forceinline__ unsigned short to16(float x);
template <> __device__ __forceinline__ unsigned short to16<__half>(float x) { return __half_as_ushort(__float2half_rn(x)); }
template <> __device__ __forceinline__ unsigned short to16<__nv_bfloat16>(float x) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}

template <typename OUT>
__global__ void __launch_bounds__(256) k_copy16_panel(const FrontDesc* __restrict__ fronts, int K0) {
    const FrontDesc f = fronts[blockIdx.x];
    if (f.s <= K0) return;
    const int c1 = min(K0 + WOUT, f.s);
    const float* P = (const float*)f.P;
    unsigned short* Q = (unsigned short*)f.P16;
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int i = K0 + blockIdx.y * wpb + (threadIdx.x >> 5); i < f.N; i += gridDim.y * wpb) {
        const int cend = i < f.s ? min(c1, (i / NB) * NB) : c1;
        if (cend <= K0) continue;
        const float sc = f.rs[i];
        const float* src = P + (int64_t)i * f.ldp;
        unsigned short* dst = Q + (int64_t)i * f.ldp;
        for (int c = K0 + lane * 8; c < cend; c += 256) {
            if (c + 8 <= cend) {
                const float4 a = *(const float4*)(src + c), b = *(const float4*)(src + c + 4);
                uint4 o;
                o.x = (uint32_t)to16<OUT>(a.x * sc) | ((uint32_t)to16<OUT>(a.y * sc) << 16);
                o.y = (uint32_t)to16<OUT>(a.z * sc) | ((uint32_t)to16<OUT>(a.w * sc) << 16);
                o.z = (uint32_t)to16<OUT>(b.x * sc) | ((uint32_t)to16<OUT>(b.y * sc) << 16);
                o.w = (uint32_t)to16<OUT>(b.z * sc) | ((uint32_t)to16<OUT>(b.w * sc) << 16);
                *reinterpret_cast<uint4*>(dst + c) = o;
            } else {
                for (int e = 0; c + e < cend; ++e) dst[c + e] = to16<OUT>(src[c + e] * sc);
            }
        }
    }
}

int launch_copy16_panel(Handle& h, int li, int K0, cudaStream_t st) {
    Level& L = h.levels[li];
    if (L.op16 == TC_OP_TF32 || L.fronts.empty() || K0 >= L.max_s) return RSD_OK;
    const int nf = (int)L.fronts.size();
    double bytes = 0;
    for (auto& f : L.fronts)
        if (f.s > K0) bytes += 6.0 * (double)(f.N - K0) * std::min(WOUT, f.s - K0);
    const dim3 g((unsigned)nf, (unsigned)std::max(1, std::min((L.max_N - K0 + 7) / 8, (h.num_sms * 8 + nf - 1) / nf)));
    const int pi = prof_begin(h, K_COPY16, st);
    if (L.op16 == TC_OP_BF16) k_copy16_panel<__nv_bfloat16><<<g, 256, 0, st>>>(L.d_fronts, K0);
    else k_copy16_panel<__half><<<g, 256, 0, st>>>(L.d_fronts, K0);
    count_launch();
    prof_end(h, pi, 0.0, bytes, st);
    RSD_CUDA_TRY(cudaGetLastError());
    return RSD_OK;
}

int launch_factor_copy16(Handle& h, int li) {
    Level& L = h.levels[li];
    // levels with 16-bit GEMM operands wrote their copy panel by panel
    if (!L.h16 || L.op16 != TC_OP_TF32 || L.fronts.empty()) return RSD_OK;
    const int nf = (int)L.fronts.size();
    double bytes = 0;
    for (auto& f : L.fronts) bytes += 6.0 * (0.5 * f.s * (f.s + 1.0) + (double)f.s * f.b);
    const dim3 g((unsigned)nf, (unsigned)std::max(1, std::min((L.max_N + 7) / 8, (h.num_sms * 8 + nf - 1) / nf)));
    const int pi = prof_begin(h, K_COPY16);
    k_copy16<<<g, 256, 0, h.stream>>>(L.d_fronts);
    count_launch();
    prof_end(h, pi, 0.0, bytes);
    RSD_CUDA_TRY(cudaGetLastError());
    return RSD_OK;
}

int launch_zero_fronts(Handle& h, int li) {
    Level& L = h.levels[li];
    if (L.fronts.empty()) return RSD_OK;
    RSD_CUDA_TRY(cudaMemsetAsync(L.fronts[0].P, 0, L.bytes_P, h.stream));
    if (L.bytes_U) RSD_CUDA_TRY(cudaMemsetAsync(L.fronts[0].U, 0, L.bytes_U, h.stream));
    return RSD_OK;
}

int launch_assemble_fronts(Handle& h, int li, const int64_t* rowptr, const int* col,
                           const double* val, const int* owner, const int* rank, const int* tin,
                           const int* tout) {
    Level& L = h.levels[li];
    if (L.fronts.empty()) return RSD_OK;
    dim3 grid((unsigned)std::max(1, std::min(64, (L.max_s + 7) / 8)), (unsigned)L.fronts.size());
    const int pi = prof_begin(h, K_ASSEMBLE);
    if (is_fp64(L.prec))
        k_scatter_K<double><<<grid, 256, 0, h.stream>>>(L.d_fronts, rowptr, col, val, owner, rank, tin, tout);
    else
        k_scatter_K<float><<<grid, 256, 0, h.stream>>>(L.d_fronts, rowptr, col, val, owner, rank, tin, tout);
    count_launch();
    if (copy16_level(L)) {
        const dim3 g((unsigned)L.fronts.size(), (unsigned)std::max(1, std::min(16, (L.max_N + 1023) / 1024)));
        k_row_scale<<<g, 256, 0, h.stream>>>(L.d_fronts, rowptr, col, val);
        count_launch();
    }
    {
        double rows = 0;
        for (auto& f : L.fronts) rows += f.s;
        prof_end(h, pi, 0.0, rows * 27.0 * (12.0 + elem_bytes(L.prec)));
    }
    RSD_CUDA_TRY(cudaGetLastError());
    return RSD_OK;
}

int launch_extend_add(Handle& h, int li) {
    if (li + 1 >= (int)h.levels.size()) return RSD_OK;
    Level& Lp = h.levels[li];
    Level& Lc = h.levels[li + 1];
    if (Lp.fronts.empty() || Lc.fronts.empty()) return RSD_OK;
    const bool p64 = is_fp64(Lp.prec), c64 = is_fp64(Lc.prec);
    const int64_t ntl = (Lc.max_b + EA_T - 1) / EA_T;
    const int64_t units = ntl * ((ntl + EA_CH - 1) / EA_CH);
    const int per_parent = (int)std::max<int64_t>(1, std::min<int64_t>(units,
                                                                       (8LL * h.num_sms + (int64_t)Lp.fronts.size() - 1) / (int64_t)Lp.fronts.size()));
    dim3 grid((unsigned)per_parent, (unsigned)Lp.fronts.size());
    double ea_bytes = 0;
    for (auto& f : Lc.fronts) ea_bytes += 0.5 * f.b * (f.b + 1.0) * (elem_bytes(Lc.prec) + 2.0 * elem_bytes(Lp.prec));
    ea_bytes /= std::max(1, Lp.max_children);
    for (int ci = 0; ci < Lp.max_children; ++ci) {
        const int pi = prof_begin(h, K_EXTEND);
        if (p64 && c64) k_extend_add<double, double><<<grid, 256, 0, h.stream>>>(Lp.d_fronts, Lc.d_fronts, Lp.d_child_slots, ci);
        else if (p64 && !c64) k_extend_add<float, double><<<grid, 256, 0, h.stream>>>(Lp.d_fronts, Lc.d_fronts, Lp.d_child_slots, ci);
        else if (!p64 && c64) k_extend_add<double, float><<<grid, 256, 0, h.stream>>>(Lp.d_fronts, Lc.d_fronts, Lp.d_child_slots, ci);
        else k_extend_add<float, float><<<grid, 256, 0, h.stream>>>(Lp.d_fronts, Lc.d_fronts, Lp.d_child_slots, ci);
        count_launch();
        prof_end(h, pi, 0.0, ea_bytes);
        RSD_CUDA_TRY(cudaGetLastError());
    }
    return RSD_OK;
}

// ---------------------------------------------------------------------------------
// Tensor-core levels: block-inverse panel solve and look-ahead.
//
// For each outer panel (columns K0 .. K0+W, W <= WOUT):
//   (a0) the outer update of the whole panel, as above;
//   (a)-(c) restricted to the W x W diagonal block of the panel (its 128-blocks factored
//        one after another: small GEMMs and the diagonal factor+inverse);
//   (e)  Mt = L_pp^-T for the W x W block L_pp, from its inverted diagonal blocks:
//        Mt_jj = Dinv_j^T and, block column i after block column i, for the rows j < i
//        Mt[j, i] = -(sum_{k<i} Mt[j, k] L_ik^T) Dinv_i^T    (from Mt L_pp^T = I);
//        then Linv = Mt^T;
//   (f)  the rows below the block in one step, X = A L_pp^-T = A Linv^T, in place: the
//        column tile [256, W) first (it reads A[:, 0:W]), then [0, 256) (it reads only
//        A[:, 0:256], which the first launch left untouched).
// (e)-(f) replace the per-128-column updates and solves of the rows below the block
// (many thin, memory-bound GEMMs) by two K = W GEMMs.
//
// Levels with few fronts (the root and the level below it) also look ahead: the
// diagonal-block work runs on a high-priority stream (the "chain") beside the bulk
// stream (the caller's), and the chain also takes the small steps that link one
// diagonal block to the next (the last K range of the next block's outer update, and
// the solve of the next block's rows), so that it never waits for the bulk's large
// GEMMs except the next panel's long outer update, which the bulk runs while the chain
// factors.  The bulk persistent GEMM leaves a wave of SMs to the chain.  Every entry
// receives the same products in either order; only the outer update's K range is
// summed in two parts, and the rows below a diagonal block are solved in two groups.
constexpr int LOOKAHEAD_FRONTS = 16;
constexpr int64_t SCR_MT = 512 * 512, SCR_TT = 512 * 128, SCR_LINV = 512 * 512;
constexpr int64_t SCR_FRONT = SCR_MT + SCR_TT + 2 * SCR_LINV;    // floats per front slot (two Linv)
static_assert(WOUT == 512, "scratch blocks are sized for 512-wide outer panels");

// Mt's diagonal blocks: Mt[j, j] = Dinv_j^T (upper triangular), j < ceil(W / NB).
__global__ void k_mt_diag(const FrontDesc* __restrict__ fronts, int K0, float* __restrict__ scr) {
    const FrontDesc f = fronts[blockIdx.z];
    if (f.s <= K0) return;
    const int W = min(WOUT, f.s - K0);
    const int j = blockIdx.y;
    if (j * NB >= W) return;
    float* Mt = scr + (int64_t)blockIdx.z * SCR_FRONT;
    const float* D = (const float*)f.Dinv + (int64_t)(K0 / NB + j) * NB * NB;
    __shared__ float t[32][33];
    const int bx = blockIdx.x & 3, by = blockIdx.x >> 2;     // 4 x 4 tiles of 32 x 32
    for (int r = threadIdx.y; r < 32; r += blockDim.y) t[r][threadIdx.x] = D[(by * 32 + r) * NB + bx * 32 + threadIdx.x];
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y)
        Mt[(int64_t)(j * NB + bx * 32 + r) * 512 + j * NB + by * 32 + threadIdx.x] = t[threadIdx.x][r];
}

// Linv = Mt^T on the W x W block, zero elsewhere in the 512 x 512 slot.
__global__ void k_linv_transpose(const FrontDesc* __restrict__ fronts, int K0, float* __restrict__ scr, int which) {
    const FrontDesc f = fronts[blockIdx.z];
    if (f.s <= K0) return;
    const int W = min(WOUT, f.s - K0);
    const float* Mt = scr + (int64_t)blockIdx.z * SCR_FRONT;
    float* Li = scr + (int64_t)blockIdx.z * SCR_FRONT + SCR_MT + SCR_TT + which * SCR_LINV;
    __shared__ float t[32][33];
    const int bx = blockIdx.x, by = blockIdx.y;               // 16 x 16 tiles of 32 x 32
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int row = by * 32 + r, col = bx * 32 + threadIdx.x;
        t[r][threadIdx.x] = (row < W && col < W) ? Mt[(int64_t)row * 512 + col] : 0.f;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y)
        Li[(int64_t)(bx * 32 + r) * 512 + by * 32 + threadIdx.x] = t[threadIdx.x][r];
}

static int ensure_chain(Handle& h) {
    if (h.chain) return RSD_OK;
    int lo = 0, hi = 0;
    RSD_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    RSD_CUDA_TRY(cudaStreamCreateWithPriority(&h.chain, cudaStreamNonBlocking, hi));
    for (cudaEvent_t* e : {&h.ev_ready, &h.ev_join, &h.ev_diag[0], &h.ev_diag[1], &h.ev_diag[2], &h.ev_diag[3]})
        RSD_CUDA_TRY(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    return RSD_OK;
}

static int factor_level_tc(Handle& h, int li, bool lookahead) {
    Level& L = h.levels[li];
    const size_t es = 4;
    const size_t potrf_smem = POTRF_BLK_SMEM;
    RSD_CUDA_TRY(cudaFuncSetAttribute(k_potrf_diag_blk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)potrf_smem));
    const int nf = (int)L.fronts.size();
    if (lookahead) RSD_TRY(ensure_chain(h));
    cudaStream_t B = h.stream, Cs = lookahead ? h.chain : h.stream;
    const int cslot = lookahead ? 1 : 0;
    // the bulk persistent GEMM leaves SMs for the chain's diagonal blocks and its small
    // GEMMs (one wave of them)
    const int bulk_ctas = lookahead ? h.num_sms - std::min(h.num_sms / 4, std::max(8, 2 * nf)) : 0;
    // per-front scratch: Mt, Tt, Linv (Mt's lower part stays zero)
    float* scr = nullptr;
    RSD_CUDA_TRY(cudaMallocAsync((void**)&scr, sizeof(float) * SCR_FRONT * nf, B));
    RSD_CUDA_TRY(cudaMemsetAsync(scr, 0, sizeof(float) * SCR_FRONT * nf, B));
    std::vector<float*> mt(nf), tt(nf), lv0(nf), lv1(nf);
    for (int i = 0; i < nf; ++i) {
        mt[i] = scr + SCR_FRONT * i;
        tt[i] = mt[i] + SCR_MT;
        lv0[i] = tt[i] + SCR_TT;
        lv1[i] = lv0[i] + SCR_LINV;
    }
    int mbase = 0;
    RSD_TRY(gemm_tc_scratch_maps(h, mt, tt, lv0, lv1, B, &mbase));
    auto map_mt = [&](int i) { return mbase + TC_SCR_MAPS * i; };
    auto map_tt = [&](int i) { return mbase + TC_SCR_MAPS * i + 1; };
    auto map_lv = [&](int i, int which) { return mbase + TC_SCR_MAPS * i + 2 + which; };

    std::vector<GemmTask> tasks;
    auto wend = [](const FrontDesc& f, int K0) { return std::min(K0 + WOUT, f.s); };
    auto P = [&](const FrontDesc& f, int r, int c) { return (char*)f.P + ((int64_t)r * f.ldp + c) * es; };
    // (a) rows [r0, r1) of column block k from the finished columns [K0, k)
    auto add_update = [&](const FrontDesc& f, int k, int K0, int r0, int r1) {
        if (f.s <= k || k <= K0 || r1 <= r0) return;
        GemmTask t{};
        t.A = P(f, r0, K0); t.B = P(f, k, K0); t.C = P(f, r0, k);
        t.lda = t.ldb = t.ldc = f.ldp;
        t.M = r1 - r0; t.N = std::min(NB, f.s - k); t.K = k - K0;
        t.lower = 0; t.beta = 1;
        t.map_a = t.map_b = f.node;
        t.a_r0 = r0; t.a_c0 = K0; t.b_r0 = k; t.b_c0 = K0;
        tasks.push_back(t);
    };
    // (c) rows [r0, r1) of column block k times the inverted diagonal block
    auto add_solve = [&](const FrontDesc& f, int k, int r0, int r1) {
        if (f.s <= k || r1 <= r0) return;
        GemmTask t{};
        t.A = P(f, r0, k); t.B = (const char*)f.Dinv + (int64_t)(k / NB) * NB * NB * es; t.C = P(f, r0, k);
        t.lda = t.ldc = f.ldp; t.ldb = NB;
        t.M = r1 - r0; t.N = std::min(NB, f.s - k); t.K = t.N;
        t.lower = 0; t.beta = 0;
        t.map_a = t.map_b = f.node;
        t.a_r0 = r0; t.a_c0 = k; t.b_r0 = (k / NB) * NB; t.b_c0 = 0;
        tasks.push_back(t);
    };
    // (a0) rows [r0, r1) of the panel at K0 from the columns [kb, ke)
    auto add_outer = [&](const FrontDesc& f, int K0, int kb, int ke, int r0, int r1) {
        if (f.s <= K0 || ke <= kb || r1 <= r0) return;
        GemmTask t{};
        t.A = P(f, r0, kb); t.B = P(f, K0, kb); t.C = P(f, r0, K0);
        t.lda = t.ldb = t.ldc = f.ldp;
        t.M = r1 - r0; t.N = std::min(WOUT, f.s - K0); t.K = ke - kb;
        t.lower = 0; t.beta = 1;
        t.map_a = t.map_b = f.node;
        t.a_r0 = r0; t.a_c0 = kb; t.b_r0 = K0; t.b_c0 = kb;
        t.sa = f.ri ? f.ri + r0 : nullptr;             // 16-bit operands: 1 / row scales
        t.sb = f.ri ? f.ri + K0 : nullptr;
        tasks.push_back(t);
    };
    auto general = [&](int ma, int a_r0, int a_c0, int mb, int b_r0, int b_c0, void* C, int ldc,
                       int M, int N, int K, float alpha) {
        GemmTask t{};
        t.C = C; t.ldc = ldc; t.M = M; t.N = N; t.K = K;
        t.lower = 0; t.beta = 0; t.alpha = alpha; t.round = 1;
        t.map_a = ma; t.map_b = mb;
        t.a_r0 = a_r0; t.a_c0 = a_c0; t.b_r0 = b_r0; t.b_c0 = b_c0;
        tasks.push_back(t);
    };

    // (a)-(c) and (e) for the diagonal block of every front at K0, on stream cs; the
    // block inverse goes to Linv buffer `which`
    // The level is issued twice: a dry pass in which the GEMM launcher only records each
    // launch's task and tile lists (and nothing else is launched), then, after one upload
    // of everything recorded, the real pass.  Per-launch uploads would stall the issuing
    // thread behind the streams' queues and serialise copies between the chain's kernels.
    bool dry = false;
    auto factor_block = [&](int K0, int which, cudaStream_t cs, int slot) -> int {
        for (int j = 0; j < WOUT / NB; ++j) {
            const int k = K0 + j * NB;
            if (k >= L.max_s) break;
            tasks.clear();
            for (auto& f : L.fronts) add_update(f, k, K0, k, wend(f, K0));
            RSD_TRY(gemm_tc_launch(h, li, tasks, 0, cs, slot));
            double pf = 0, pb = 0;
            for (auto& f : L.fronts)
                if (f.s > k) { const double w = std::min(NB, f.s - k); pf += 2.0 * w * w * w / 3.0; pb += (2.0 * w * w + NB * NB) * es; }
            if (!dry) {
                const int ppi = prof_begin(h, K_POTRF, cs);
                k_potrf_diag_blk<<<(unsigned)nf, 256, potrf_smem, cs>>>(L.d_fronts, k, h.d_err, 1, h.d_front_bad);
                count_launch();
                prof_end(h, ppi, pf, pb, cs);
                RSD_CUDA_TRY(cudaGetLastError());
            }
            tasks.clear();
            for (auto& f : L.fronts) add_solve(f, k, k + std::min(NB, std::max(0, f.s - k)), wend(f, K0));
            RSD_TRY(gemm_tc_launch(h, li, tasks, 1, cs, slot));
        }
        // (e) Mt = L_pp^-T, then Linv = Mt^T
        if (!dry) {
            k_mt_diag<<<dim3(16, WOUT / NB, (unsigned)nf), dim3(32, 8), 0, cs>>>(L.d_fronts, K0, scr);
            count_launch();
            RSD_CUDA_TRY(cudaGetLastError());
        }
        for (int i = 1; i < WOUT / NB; ++i) {
            const int k = K0 + i * NB;
            if (k >= L.max_s) break;
            tasks.clear();                              // Tt = Mt[0:i NB, 0:i NB] L_{i,<i}^T
            for (int q = 0; q < nf; ++q) {
                const FrontDesc& f = L.fronts[q];
                if (f.s <= k) continue;
                general(map_mt(q), 0, 0, tc_map_panel(f.node), k, K0, tt[q], 128,
                        i * NB, std::min(NB, f.s - k), i * NB, 1.0f);
            }
            RSD_TRY(gemm_tc_launch(h, li, tasks, TC_GENERAL, cs, slot));
            tasks.clear();                              // Mt[0:i NB, i] = -Tt Dinv_i^T
            for (int q = 0; q < nf; ++q) {
                const FrontDesc& f = L.fronts[q];
                if (f.s <= k) continue;
                const int w = std::min(NB, f.s - k);
                general(map_tt(q), 0, 0, tc_map_dinv(f.node), k, 0, mt[q] + i * NB, 512,
                        i * NB, w, w, -1.0f);
            }
            RSD_TRY(gemm_tc_launch(h, li, tasks, TC_GENERAL, cs, slot));
        }
        if (!dry) {
            k_linv_transpose<<<dim3(16, 16, (unsigned)nf), dim3(32, 8), 0, cs>>>(L.d_fronts, K0, scr, which);
            count_launch();
            RSD_CUDA_TRY(cudaGetLastError());
        }
        return RSD_OK;
    };
    // (f) X = A Linv^T in place for rows [rlo(f), rhi(f)) of the panel at K0: the column
    // tile [256, W) first (it reads A[:, 0:W]), then [0, 256) (it reads only A[:, 0:256])
    auto solve_rows = [&](int K0, int which, auto rlo, auto rhi, cudaStream_t cs, int slot, int ctas) -> int {
        for (int half = 1; half >= 0; --half) {
            tasks.clear();
            for (int q = 0; q < nf; ++q) {
                const FrontDesc& f = L.fronts[q];
                if (f.s <= K0) continue;
                const int W = std::min(WOUT, f.s - K0), r0 = rlo(f), r1 = rhi(f);
                const int c0 = half * 256, c1 = std::min(W, c0 + 256);
                if (c1 <= c0 || r1 <= r0) continue;
                general(tc_map_panel(f.node), r0, K0, map_lv(q, which), c0, 0, P(f, r0, K0 + c0), f.ldp,
                        r1 - r0, c1 - c0, c1, 1.0f);
            }
            RSD_TRY(gemm_tc_launch(h, li, tasks, TC_GENERAL, cs, slot, ctas));
        }
        return RSD_OK;
    };
    auto rows_to_end = [](const FrontDesc& f) { return f.N; };

    auto issue = [&]() -> int {
        const int np = (L.max_s + WOUT - 1) / WOUT;
        if (!lookahead) {
            for (int p = 0; p < np; ++p) {
                const int K0 = p * WOUT;
                if (p >= 1) {                                   // (a0) the whole outer update
                    tasks.clear();
                    for (auto& f : L.fronts) add_outer(f, K0, 0, K0, K0, f.N);
                    RSD_TRY(gemm_tc_launch(h, li, tasks, 3, B, 0, 0, L.op16));
                }
                RSD_TRY(factor_block(K0, 0, B, 0));
                RSD_TRY(solve_rows(K0, 0, [&](const FrontDesc& f) { return wend(f, K0); }, rows_to_end, B, 0, 0));
                if (!dry) RSD_TRY(launch_copy16_panel(h, li, K0, B));   // panel p is final
            }
        } else {
            // Look-ahead.  Chain(p): the part of panel p's outer update with K in [K0-W, K0)
            // restricted to its diagonal block, the block's factorisation and inverse, and the
            // solve of the next panel's diagonal-block rows ("X_next").  Bulk, meanwhile: the
            // K range [0, K0) of panel p+1's outer update (all its rows; it needs no result of
            // panels p-1 or p held by the chain), then, once the chain has them, the solve of
            // the remaining rows below and the K range [K0, K0+W) of panel p+1's outer update
            // for its rows below the diagonal block.  Events: ev_ready (bulk: panel p+1's long
            // update done), ev_diag[0] (chain: Linv of panel p), ev_diag[1 + p % 2] (chain:
            // X_next of panel p), ev_diag[3] (bulk: panel p's contribution to panel p+1 below
            // its diagonal block, which includes the rows chain(p+1)'s X_next overwrites; the
            // two short bulk launches before it finish while the chain factors its block).
            // Linv alternates between two buffers, so the chain can build panel p+1's while
            // the bulk still solves with panel p's.
            cudaEvent_t& ev_linv = h.ev_diag[0];
            cudaEvent_t& ev_rest = h.ev_diag[3];
            if (!dry) RSD_CUDA_TRY(cudaEventRecord(h.ev_ready, B));             // the fronts are assembled
            for (int p = 0; p < np; ++p) {
                const int K0 = p * WOUT, K0n = K0 + WOUT, which = p & 1;
                cudaEvent_t& ev_xnext = h.ev_diag[1 + which];
                // ---- chain(p)
                if (!dry) RSD_CUDA_TRY(cudaStreamWaitEvent(Cs, h.ev_ready, 0));
                if (p >= 1) {
                    tasks.clear();
                    for (auto& f : L.fronts) add_outer(f, K0, K0 - WOUT, K0, K0, wend(f, K0));
                    RSD_TRY(gemm_tc_launch(h, li, tasks, 3, Cs, cslot));
                }
                RSD_TRY(factor_block(K0, which, Cs, cslot));
                if (!dry) RSD_CUDA_TRY(cudaEventRecord(ev_linv, Cs));
                auto next_lo = [&](const FrontDesc& f) { return wend(f, K0); };
                auto next_hi = [&](const FrontDesc& f) { return f.s > K0n ? wend(f, K0n) : wend(f, K0); };
                if (p + 1 < np) {
                    // X_next overwrites rows that panel p-1's bulk update also writes
                    if (p >= 1 && !dry) RSD_CUDA_TRY(cudaStreamWaitEvent(Cs, ev_rest, 0));
                    RSD_TRY(solve_rows(K0, which, next_lo, next_hi, Cs, cslot, 0));
                }
                if (!dry) RSD_CUDA_TRY(cudaEventRecord(ev_xnext, Cs));
                // ---- bulk, panel p
                if (p + 1 < np) {
                    if (K0 > 0) {
                        tasks.clear();
                        for (auto& f : L.fronts) add_outer(f, K0n, 0, K0, K0n, f.N);
                        RSD_TRY(gemm_tc_launch(h, li, tasks, 3, B, 0, bulk_ctas, L.op16));
                    }
                    if (!dry) RSD_CUDA_TRY(cudaEventRecord(h.ev_ready, B));
                }
                if (!dry) RSD_CUDA_TRY(cudaStreamWaitEvent(B, ev_linv, 0));
                RSD_TRY(solve_rows(K0, which, next_hi, rows_to_end, B, 0, bulk_ctas));
                if (p + 1 < np) {
                    if (!dry) RSD_CUDA_TRY(cudaStreamWaitEvent(B, ev_xnext, 0));
                    if (!dry) RSD_TRY(launch_copy16_panel(h, li, K0, B));   // panel p is final
                    tasks.clear();
                    for (auto& f : L.fronts)
                        if (f.s > K0n) add_outer(f, K0n, K0, K0n, wend(f, K0n), f.N);
                    RSD_TRY(gemm_tc_launch(h, li, tasks, 3, B, 0, bulk_ctas));
                    if (!dry) RSD_CUDA_TRY(cudaEventRecord(ev_rest, B));
                } else if (!dry) {
                    RSD_TRY(launch_copy16_panel(h, li, K0, B));          // the last panel is final
                }
            }
            if (!dry) RSD_CUDA_TRY(cudaEventRecord(h.ev_join, Cs));
            if (!dry) RSD_CUDA_TRY(cudaStreamWaitEvent(B, h.ev_join, 0));
        }
        return RSD_OK;
    };
    dry = true;
    RSD_TRY(gemm_tc_record_begin(h));
    RSD_TRY(issue());
    RSD_TRY(gemm_tc_record_end(h, B));
    dry = false;
    const int rc_issue = issue();
    gemm_tc_replay_end(h, B);
    RSD_TRY(rc_issue);
    cudaFreeAsync(scr, B);
    return RSD_OK;
}

// Partial Cholesky of every front of level li (steps (a)-(d) above).
int run_factor_level(Handle& h, int li) {
    Level& L = h.levels[li];
    if (L.fronts.empty()) return RSD_OK;
    const bool f64 = is_fp64(L.prec);
    const bool tc = tc_level(L);
    const size_t es = f64 ? 8 : 4;
    // task buffer for this level: one slot per front per launch kind
    GemmTask* d_tasks = nullptr;
    RSD_CUDA_TRY(cudaMallocAsync((void**)&d_tasks, sizeof(GemmTask) * L.fronts.size() * 2 + 64, h.stream));
    const size_t potrf_smem = f64 ? (size_t)NB * DLD * es + (size_t)2 * NB * es : POTRF_BLK_SMEM;
    const size_t trsm_smem = (size_t)NB * NB * es + (size_t)TR_ROWS * (NB + 1) * es;
    if (f64) {
        RSD_CUDA_TRY(cudaFuncSetAttribute(k_potrf_diag<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)potrf_smem));
        RSD_CUDA_TRY(cudaFuncSetAttribute(k_trsm_simt<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)trsm_smem));
    } else {
        RSD_CUDA_TRY(cudaFuncSetAttribute(k_potrf_diag_blk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)potrf_smem));
        RSD_CUDA_TRY(cudaFuncSetAttribute(k_trsm_simt<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)trsm_smem));
    }
    std::vector<GemmTask> tasks;
    int rc = RSD_OK;
    auto run_gemm = [&](int kind) -> int {
        if (tasks.empty()) return RSD_OK;
        if (tc) return gemm_tc_launch(h, li, tasks, kind, h.stream);
        finalize_tasks(tasks, SB, SB);
        return f64 ? launch_gemm_simt<double>(h, tasks, d_tasks, -1.0, h.stream)
                   : launch_gemm_simt<float>(h, tasks, d_tasks, -1.0f, h.stream);
    };
    if (tc) rc = factor_level_tc(h, li, (int)L.fronts.size() <= LOOKAHEAD_FRONTS && L.max_s > WOUT);
    for (int k = 0; !tc && k < L.max_s && rc == RSD_OK; k += NB) {
        const int K0 = (k / WOUT) * WOUT;               // start of the enclosing outer panel
        // (a0) at an outer panel start: update the whole WOUT-wide panel from all columns
        //      left of it (one large-K GEMM per outer panel)
        if (k == K0 && K0 > 0) {
            tasks.clear();
            for (auto& f : L.fronts) {
                if (f.s <= K0) continue;
                const int W = std::min(WOUT, f.s - K0);
                GemmTask t{};
                t.A = (const char*)f.P + ((int64_t)K0 * f.ldp) * es;
                t.B = t.A;
                t.C = (char*)f.P + ((int64_t)K0 * f.ldp + K0) * es;
                t.lda = t.ldb = t.ldc = f.ldp;
                t.M = f.N - K0; t.N = W; t.K = K0;
                t.lower = 0; t.beta = 1;
                t.map_a = t.map_b = f.node;
                t.a_r0 = K0; t.a_c0 = 0; t.b_r0 = K0; t.b_c0 = 0;
                tasks.push_back(t);
            }
            rc = run_gemm(3);
            if (rc != RSD_OK) break;
        }
        // (a) inner update of the NB-wide panel from the finished columns K0..k of its
        //     outer panel
        if (k > K0) {
            tasks.clear();
            for (auto& f : L.fronts) {
                if (f.s <= k) continue;
                const int w = std::min(NB, f.s - k);
                GemmTask t{};
                t.A = (const char*)f.P + ((int64_t)k * f.ldp + K0) * es;
                t.B = t.A;
                t.C = (char*)f.P + ((int64_t)k * f.ldp + k) * es;
                t.lda = t.ldb = t.ldc = f.ldp;
                t.M = f.N - k; t.N = w; t.K = k - K0;
                t.lower = 0; t.beta = 1;
                t.map_a = t.map_b = f.node;
                t.a_r0 = k; t.a_c0 = K0; t.b_r0 = k; t.b_c0 = K0;
                tasks.push_back(t);
            }
            rc = run_gemm(0);
            if (rc != RSD_OK) break;
        }
        // (b) diagonal block factor + inverse
        double pf = 0, pb = 0;
        for (auto& f : L.fronts)
            if (f.s > k) { const double w = std::min(NB, f.s - k); pf += 2.0 * w * w * w / 3.0; pb += (2.0 * w * w + NB * NB) * es; }
        const int ppi = prof_begin(h, K_POTRF);
        if (f64) k_potrf_diag<double><<<(unsigned)L.fronts.size(), 256, potrf_smem, h.stream>>>(L.d_fronts, k, h.d_err, 0, h.d_front_bad);
        else k_potrf_diag_blk<<<(unsigned)L.fronts.size(), 256, potrf_smem, h.stream>>>(L.d_fronts, k, h.d_err, tc ? 1 : 0, h.d_front_bad);
        count_launch();
        prof_end(h, ppi, pf, pb);
        if (cudaGetLastError() != cudaSuccess) { rc = RSD_ERR_CUDA; break; }
        // (c) panel solve below the diagonal block
        if (tc) {
            tasks.clear();
            for (auto& f : L.fronts) {
                if (f.s <= k) continue;
                const int w = std::min(NB, f.s - k);
                if (f.N - k - w <= 0) continue;
                GemmTask t{};
                t.A = (const char*)f.P + ((int64_t)(k + w) * f.ldp + k) * es;
                t.B = (const char*)f.Dinv + (int64_t)(k / NB) * NB * NB * es;
                t.C = (char*)t.A;
                t.lda = t.ldc = f.ldp; t.ldb = NB;
                t.M = f.N - k - w; t.N = w; t.K = w;
                t.lower = 0; t.beta = 0;
                t.map_a = f.node; t.map_b = f.node;
                t.a_r0 = k + w; t.a_c0 = k; t.b_r0 = (k / NB) * NB; t.b_c0 = 0;
                tasks.push_back(t);
            }
            rc = gemm_tc_launch(h, li, tasks, 1, h.stream);
            if (rc != RSD_OK) break;
        } else {
            const int rows = L.max_N;   // upper bound on rows below the diagonal
            dim3 grid((unsigned)std::max(1, (rows - k + TR_ROWS - 1) / TR_ROWS), (unsigned)L.fronts.size());
            double tf = 0, tb = 0;
            for (auto& f : L.fronts)
                if (f.s > k) { const double w = std::min(NB, f.s - k), m = f.N - k - w; tf += m * w * w; tb += 2.0 * m * w * es; }
            const int tpi = prof_begin(h, K_TRSM);
            if (f64) k_trsm_simt<double><<<grid, 256, trsm_smem, h.stream>>>(L.d_fronts, k, 0);
            else k_trsm_simt<float><<<grid, 256, trsm_smem, h.stream>>>(L.d_fronts, k, 0);
            count_launch();
            prof_end(h, tpi, tf, tb);
            if (cudaGetLastError() != cudaSuccess) { rc = RSD_ERR_CUDA; break; }
        }
    }
    // (d) Schur contribution to the ancestors: U -= X X^T
    if (rc == RSD_OK) {
        tasks.clear();
        for (auto& f : L.fronts) {
            if (f.b == 0 || f.s == 0) continue;
            GemmTask t{};
            t.A = (const char*)f.P + ((int64_t)f.s * f.ldp) * es;
            t.B = t.A;
            t.C = f.U;
            t.lda = t.ldb = f.ldp; t.ldc = f.ldu;
            t.M = f.b; t.N = f.b; t.K = f.s;
            t.lower = 1; t.beta = 1;
            t.map_a = t.map_b = f.node;
            t.a_r0 = f.s; t.a_c0 = 0; t.b_r0 = f.s; t.b_c0 = 0;
            t.sa = t.sb = f.ri ? f.ri + f.s : nullptr;      // 16-bit operands: 1 / row scales
            tasks.push_back(t);
        }
        if (!tasks.empty()) {
            if (tc) rc = gemm_tc_launch(h, li, tasks, 2, h.stream, 0, 0, L.op16);
            else {
                finalize_tasks(tasks, SB, SB);
                rc = f64 ? launch_gemm_simt<double>(h, tasks, d_tasks, -1.0, h.stream)
                         : launch_gemm_simt<float>(h, tasks, d_tasks, -1.0f, h.stream);
            }
        }
    }
    cudaFreeAsync(d_tasks, h.stream);
    return rc;
}

// ---- CUDA-core kernels for the nonsymmetric (LU) fronts of factor_lu.cu -------------
int lu_gemm(Handle& h, const std::vector<GemmTask>& tasks_in, bool f64, cudaStream_t st) {
    if (tasks_in.empty()) return RSD_OK;
    std::vector<GemmTask> tasks = tasks_in;
    finalize_tasks(tasks, SB, SB);
    GemmTask* d_tasks = nullptr;
    RSD_CUDA_TRY(cudaMallocAsync((void**)&d_tasks, sizeof(GemmTask) * tasks.size(), st));
    const int rc = f64 ? launch_gemm_simt<double>(h, tasks, d_tasks, -1.0, st)
                       : launch_gemm_simt<float>(h, tasks, d_tasks, -1.0f, st);
    cudaFreeAsync(d_tasks, st);
    return rc;
}

int lu_trsm(Handle& h, int li, int k, int sel, bool f64, cudaStream_t st) {
    Level& L = h.levels[li];
    const size_t es = f64 ? 8 : 4;
    const size_t trsm_smem = (size_t)NB * NB * es + (size_t)TR_ROWS * (NB + 1) * es;
    if (f64) RSD_CUDA_TRY(cudaFuncSetAttribute(k_trsm_simt<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)trsm_smem));
    else RSD_CUDA_TRY(cudaFuncSetAttribute(k_trsm_simt<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)trsm_smem));
    dim3 grid((unsigned)std::max(1, (L.max_N - k + TR_ROWS - 1) / TR_ROWS), (unsigned)L.fronts.size());
    double tf = 0, tb = 0;
    for (auto& f : L.fronts)
        if (f.s > k) { const double w = std::min(NB, f.s - k), m = f.N - k - w; tf += m * w * w; tb += 2.0 * m * w * es; }
    const int tpi = prof_begin(h, K_TRSM, st);
    if (f64) k_trsm_simt<double><<<grid, 256, trsm_smem, st>>>(L.d_fronts, k, sel);
    else k_trsm_simt<float><<<grid, 256, trsm_smem, st>>>(L.d_fronts, k, sel);
    count_launch();
    prof_end(h, tpi, tf, tb, st);
    RSD_CUDA_TRY(cudaGetLastError());
    return RSD_OK;
}

}  // namespace rsd
