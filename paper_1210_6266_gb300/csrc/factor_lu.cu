// Nonsymmetric fronts: the exact recursion of Eqs. 3.2-3.3 with K_IL != K_LI^T (the
// two-variable systems of Sec. 4, Eqs. 4.2-4.3), LU without pivoting per front.
//
// Per front t with interface/interior DOFs I (s) and ancestor DOFs B (b):
//   F_II = L U (L unit lower), X = F_BI U^-1, Y = L^-1 F_IB, U_t = F_BB - X Y.
// Storage (row-major, N = s + b rows, ldp columns each):
//   P  = [L; X]      lower form: P[i, j] = L[i, j] (i > j), 1 on the diagonal; rows s.. X
//   PU = [U^T; Y^T]  lower form: PU[i, j] = U[j, i] (i >= j); rows s.. hold Y^T
// so that every update is C -= A B^T with A and B rows of P or PU, exactly the form of
// the symmetric kernels, and the substitution sweeps of the Cholesky fronts apply
// unchanged: the forward sweep to (P, Dinv = L_kk^-1), the backward sweep to (PU,
// DinvU = (U_kk^T)^-1), whose transpose is U_kk^-1.
// Before factorisation F is spread over P (entries on or below the diagonal of F_II, and
// F_BI) and PU (entries above it, transposed, and F_IB transposed).
//
// Left-looking by NB-column blocks k (CUDA cores, FP64 or FP32):
//   (a) P[k:N, blk]    -= P[k:N, 0:k]    PU[blk, 0:k]^T   (L and X columns, with the
//                                                          diagonal block's lower part)
//   (b) PU[k:N, blk]   -= PU[k:N, 0:k]   P[blk, 0:k]^T    (U^T and Y^T columns, with the
//                                                          diagonal block's upper part)
//   (c) the diagonal block's LU (lower part from P, upper part from PU) and the inverses
//       L_kk^-1, (U_kk^T)^-1
//   (d) P[k+w:N, blk]  <- P[k+w:N, blk]  DinvU^T          (= F U_kk^-1)
//       PU[k+w:N, blk] <- PU[k+w:N, blk] Dinv^T           (= (L_kk^-1 F)^T)
// then U_t -= X Y = P[s:N, :] PU[s:N, :]^T (all b x b entries).
#include <algorithm>
#include <cmath>

#include "rsd_internal.cuh"

namespace rsd {

// CUDA-core batched GEMM (C = C - A B^T) and panel solve (rows times an inverted diagonal
// block, transposed) of factor.cu; sel picks the panel solve's operands: 1 = (P, DinvU),
// 2 = (PU, Dinv)
int lu_gemm(Handle& h, const std::vector<GemmTask>& tasks, bool f64, cudaStream_t st);
int lu_trsm(Handle& h, int li, int k, int sel, bool f64, cudaStream_t st);

namespace {

// Assembly: warp per row p of I_t (DOF i); entry K[i, j]:
//   j in I_t (rank q):   q <= p -> P[p, q];  q > p -> PU[q, p]
//   j in B_t (pos):      PU[s + pos, p] = K[i, j]  and  P[s + pos, p] = K[j, i] (K[j, i]
//                        found in row j: the pattern is symmetric)
//   j owned by a descendant: placed by that descendant's rows.
template <typename T>
__global__ void k_scatter_K_lu(const FrontDesc* __restrict__ fronts, const int64_t* __restrict__ rowptr,
                               const int* __restrict__ col, const double* __restrict__ val,
                               const int* __restrict__ owner, const int* __restrict__ rank,
                               const int* __restrict__ tin, const int* __restrict__ tout) {
    const FrontDesc f = fronts[blockIdx.y];
    const int lane = threadIdx.x & 31, warps = blockDim.x >> 5;
    const int t = f.node;
    const int tin_t = tin[t], tout_t = tout[t];
    T* P = (T*)f.P;
    T* PU = (T*)f.PU;
    for (int p = blockIdx.x * warps + (threadIdx.x >> 5); p < f.s; p += gridDim.x * warps) {
        const int i = f.I[p];
        for (int64_t k = rowptr[i] + lane; k < rowptr[i + 1]; k += 32) {
            const int j = col[k];
            const int o = owner[j];
            if (o == t) {
                const int q = rank[j];
                if (q <= p) P[(int64_t)p * f.ldp + q] = (T)val[k];
                else PU[(int64_t)q * f.ldp + p] = (T)val[k];
            } else if (tin[o] < tin_t && tout_t <= tout[o]) {        // proper ancestor of t
                int lo = 0, hi = f.b;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (f.Bd[mid] < j) lo = mid + 1; else hi = mid;
                }
                if (lo >= f.b || f.Bd[lo] != j) continue;
                PU[(int64_t)(f.s + lo) * f.ldp + p] = (T)val[k];
                // K[j, i] in row j
                int64_t a = rowptr[j], e = rowptr[j + 1];
                while (a < e) {
                    const int64_t mid = (a + e) >> 1;
                    if (col[mid] < i) a = mid + 1; else e = mid;
                }
                P[(int64_t)(f.s + lo) * f.ldp + p] = (a < rowptr[j + 1] && col[a] == i) ? (T)val[a] : (T)0;
            }
        }
    }
}

// Extend-add of child number ci of every front of the level: U_c (b_c x b_c, all entries)
// added at parent positions (pi, pj) = (ea[i], ea[j]): both in B -> the parent's U;
// pi >= pj -> P[pi, pj]; pi < pj -> PU[pj, pi].  One thread per entry; within one child
// the targets are distinct (ea is injective), children are added in a fixed order.
template <typename Tc, typename Tp>
__global__ void k_extend_add_lu(const FrontDesc* __restrict__ parents, const FrontDesc* __restrict__ kids,
                                const int* __restrict__ child_slots, int ci) {
    const FrontDesc fp = parents[blockIdx.y];
    if (ci >= fp.child_count) return;
    const FrontDesc fc = kids[child_slots[fp.child_begin + ci]];
    const Tc* U = (const Tc*)fc.U;
    Tp* P = (Tp*)fp.P;
    Tp* PU = (Tp*)fp.PU;
    Tp* Up = (Tp*)fp.U;
    const int64_t nn = (int64_t)fc.b * fc.b;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nn; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / fc.b), j = (int)(e % fc.b);
        const int pi = fc.ea[i], pj = fc.ea[j];
        const Tp v = (Tp)U[(int64_t)i * fc.ldu + j];
        Tp* dst;
        if (pi >= fp.s && pj >= fp.s) dst = Up + (int64_t)(pi - fp.s) * fp.ldu + (pj - fp.s);
        else if (pi >= pj) dst = P + (int64_t)pi * fp.ldp + pj;
        else dst = PU + (int64_t)pj * fp.ldp + pi;
        *dst += v;
    }
}

// LU of the w x w diagonal block at k (w <= NB; one CTA per front), without pivoting.  The
// block of F (updated by steps (a) and (b)) is read from P on and below the diagonal and
// from PU (transposed) above it.  Writes L (unit) to P's block, U^T to PU's block, L^-1 to
// Dinv and (U^T)^-1 = (U^-1)^T to DinvU (NB x NB, zero padded).  A pivot that is zero or not finite marks the front (not factorable without
// pivoting) and is replaced by 1 so the kernel finishes.
template <typename T>
__global__ void __launch_bounds__(256) k_getrf_diag(const FrontDesc* __restrict__ fronts, int k, int* __restrict__ err,
                                                   int* __restrict__ bad_front) {
    extern __shared__ unsigned char smem_raw[];
    constexpr int LD = NB + 1;
    T* A = (T*)smem_raw;
    const FrontDesc f = fronts[blockIdx.x];
    if (f.s <= k) return;
    const int w = min(NB, f.s - k);
    T* P = (T*)f.P;
    T* PU = (T*)f.PU;
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        const int r = e / NB, c = e % NB;
        A[r * LD + c] = (r < w && c < w) ? (c <= r ? P[(int64_t)(k + r) * f.ldp + k + c] : PU[(int64_t)(k + c) * f.ldp + k + r])
                                         : (r == c ? (T)1 : (T)0);
    }
    __shared__ int s_bad;
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    for (int j = 0; j < w; ++j) {
        T piv = A[j * LD + j];
        if (!(piv != (T)0) || !isfinite((double)piv)) {
            if (threadIdx.x == 0) { s_bad = 1; A[j * LD + j] = (T)1; }
            piv = (T)1;
        }
        __syncthreads();
        const T inv = (T)1 / A[j * LD + j];
        for (int r = j + 1 + threadIdx.x; r < w; r += blockDim.x) A[r * LD + j] *= inv;
        __syncthreads();
        const int m = w - j - 1;
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
            const int r = j + 1 + e / m, c = j + 1 + e % m;
            A[r * LD + c] -= A[r * LD + j] * A[j * LD + c];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && s_bad) {
        atomicExch(&err[ERR_NOT_SPD], 1);
        atomicMin(&err[ERR_NOT_SPD_NODE], f.node);
        bad_front[f.node] = 1;
    }
    // L (unit) and U^T into the panels
    for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
        const int r = e / w, c = e % w;
        if (c < r) P[(int64_t)(k + r) * f.ldp + k + c] = A[r * LD + c];
        else if (c == r) P[(int64_t)(k + r) * f.ldp + k + c] = (T)1;
        if (c <= r) PU[(int64_t)(k + r) * f.ldp + k + c] = A[c * LD + r];
    }
    // inverses, one column per thread: Dinv column c of L^-1 (rows >= c), and row c of
    // DinvU = column c of U^-1 (rows <= c), each thread reading back only what it wrote
    T* D = (T*)f.Dinv + (int64_t)(k / NB) * NB * NB;
    T* DU = (T*)f.DinvU + (int64_t)(k / NB) * NB * NB;
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) { D[e] = (T)0; DU[e] = (T)0; }
    __syncthreads();
    for (int c = threadIdx.x; c < w; c += blockDim.x) {
        D[c * NB + c] = (T)1;
        for (int r = c + 1; r < w; ++r) {
            T x = (T)0;
            for (int m = c; m < r; ++m) x -= A[r * LD + m] * D[m * NB + c];
            D[r * NB + c] = x;
        }
        DU[c * NB + c] = (T)1 / A[c * LD + c];
        for (int r = c - 1; r >= 0; --r) {
            T x = (T)0;
            for (int m = r + 1; m <= c; ++m) x -= A[r * LD + m] * DU[c * NB + m];
            DU[c * NB + r] = x / A[r * LD + r];
        }
    }
}

}  // namespace

int launch_assemble_fronts_lu(Handle& h, int li, const int64_t* rowptr, const int* col, const double* val,
                              const int* owner, const int* rank, const int* tin, const int* tout) {
    Level& L = h.levels[li];
    if (L.fronts.empty()) return RSD_OK;
    dim3 grid((unsigned)std::max(1, std::min(64, (L.max_s + 7) / 8)), (unsigned)L.fronts.size());
    const int pi = prof_begin(h, K_ASSEMBLE);
    if (is_fp64(L.prec))
        k_scatter_K_lu<double><<<grid, 256, 0, h.stream>>>(L.d_fronts, rowptr, col, val, owner, rank, tin, tout);
    else
        k_scatter_K_lu<float><<<grid, 256, 0, h.stream>>>(L.d_fronts, rowptr, col, val, owner, rank, tin, tout);
    count_launch();
    double rows = 0;
    for (auto& f : L.fronts) rows += f.s;
    prof_end(h, pi, 0.0, rows * 27.0 * (12.0 + elem_bytes(L.prec)));
    RSD_CUDA_TRY(cudaGetLastError());
    return RSD_OK;
}

int launch_extend_add_lu(Handle& h, int li) {
    if (li + 1 >= (int)h.levels.size()) return RSD_OK;
    Level& Lp = h.levels[li];
    Level& Lc = h.levels[li + 1];
    if (Lp.fronts.empty() || Lc.fronts.empty()) return RSD_OK;
    const bool p64 = is_fp64(Lp.prec), c64 = is_fp64(Lc.prec);
    const int64_t nn = (int64_t)Lc.max_b * Lc.max_b;
    dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>((nn + 255) / 256,
                                                               (8LL * h.num_sms + (int64_t)Lp.fronts.size() - 1) /
                                                                   (int64_t)Lp.fronts.size())),
              (unsigned)Lp.fronts.size());
    for (int ci = 0; ci < Lp.max_children; ++ci) {
        const int pi = prof_begin(h, K_EXTEND);
        if (p64 && c64) k_extend_add_lu<double, double><<<grid, 256, 0, h.stream>>>(Lp.d_fronts, Lc.d_fronts, Lp.d_child_slots, ci);
        else if (p64) k_extend_add_lu<float, double><<<grid, 256, 0, h.stream>>>(Lp.d_fronts, Lc.d_fronts, Lp.d_child_slots, ci);
        else if (c64) k_extend_add_lu<double, float><<<grid, 256, 0, h.stream>>>(Lp.d_fronts, Lc.d_fronts, Lp.d_child_slots, ci);
        else k_extend_add_lu<float, float><<<grid, 256, 0, h.stream>>>(Lp.d_fronts, Lc.d_fronts, Lp.d_child_slots, ci);
        count_launch();
        prof_end(h, pi, 0.0, 0.0);
        RSD_CUDA_TRY(cudaGetLastError());
    }
    return RSD_OK;
}

int run_factor_level_lu(Handle& h, int li) {
    Level& L = h.levels[li];
    if (L.fronts.empty()) return RSD_OK;
    const bool f64 = is_fp64(L.prec);
    const size_t es = f64 ? 8 : 4;
    const size_t smem = (size_t)NB * (NB + 1) * es;
    if (f64) RSD_CUDA_TRY(cudaFuncSetAttribute(k_getrf_diag<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    else RSD_CUDA_TRY(cudaFuncSetAttribute(k_getrf_diag<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    auto at = [&](void* base, const FrontDesc& f, int r, int c) { return (char*)base + ((int64_t)r * f.ldp + c) * es; };
    std::vector<GemmTask> tasks;
    for (int k = 0; k < L.max_s; k += NB) {
        if (k > 0) {
            // (a) L and X columns, with the full diagonal block of F
            tasks.clear();
            for (auto& f : L.fronts) {
                if (f.s <= k) continue;
                GemmTask t{};
                t.A = at(f.P, f, k, 0); t.B = at(f.PU, f, k, 0); t.C = at(f.P, f, k, k);
                t.lda = t.ldb = t.ldc = f.ldp;
                t.M = f.N - k; t.N = std::min(NB, f.s - k); t.K = k;
                t.lower = 0; t.beta = 1;
                tasks.push_back(t);
            }
            RSD_TRY(lu_gemm(h, tasks, f64, h.stream));
            // (b) U^T and Y^T columns, from the diagonal block down
            tasks.clear();
            for (auto& f : L.fronts) {
                if (f.s <= k) continue;
                const int w = std::min(NB, f.s - k);
                GemmTask t{};
                t.A = at(f.PU, f, k, 0); t.B = at(f.P, f, k, 0); t.C = at(f.PU, f, k, k);
                t.lda = t.ldb = t.ldc = f.ldp;
                t.M = f.N - k; t.N = w; t.K = k;
                t.lower = 0; t.beta = 1;
                tasks.push_back(t);
            }
            RSD_TRY(lu_gemm(h, tasks, f64, h.stream));
        }
        // (c) the diagonal block
        double pf = 0;
        for (auto& f : L.fronts)
            if (f.s > k) { const double w = std::min(NB, f.s - k); pf += 2.0 * w * w * w / 3.0 + 2.0 * w * w * w / 3.0; }
        const int ppi = prof_begin(h, K_POTRF);
        if (f64) k_getrf_diag<double><<<(unsigned)L.fronts.size(), 256, smem, h.stream>>>(L.d_fronts, k, h.d_err, h.d_front_bad);
        else k_getrf_diag<float><<<(unsigned)L.fronts.size(), 256, smem, h.stream>>>(L.d_fronts, k, h.d_err, h.d_front_bad);
        count_launch();
        prof_end(h, ppi, pf, 0.0);
        RSD_CUDA_TRY(cudaGetLastError());
        // (d) the rows below: L/X panel with U_kk^-1 (DinvU^T), U^T/Y^T panel with Dinv^T
        RSD_TRY(lu_trsm(h, li, k, 1, f64, h.stream));
        RSD_TRY(lu_trsm(h, li, k, 2, f64, h.stream));
    }
    // the Schur contribution to the ancestors: U_t -= X Y, every entry
    tasks.clear();
    for (auto& f : L.fronts) {
        if (f.b == 0 || f.s == 0) continue;
        GemmTask t{};
        t.A = at(f.P, f, f.s, 0); t.B = at(f.PU, f, f.s, 0); t.C = f.U;
        t.lda = t.ldb = f.ldp; t.ldc = f.ldu;
        t.M = f.b; t.N = f.b; t.K = f.s;
        t.lower = 0; t.beta = 1;
        tasks.push_back(t);
    }
    RSD_TRY(lu_gemm(h, tasks, f64, h.stream));
    return RSD_OK;
}

}  // namespace rsd
