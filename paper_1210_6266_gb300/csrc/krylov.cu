// Outer Krylov solve: preconditioned CG in FP64 with the RSD preconditioner (the paper
// wraps RSD in GMRES on K u = f, zero initial guess, relative 2-norm stopping test,
// Sec. 3 and Sec. 4; K and M are SPD here, so CG is the short-recurrence choice).
// Dot products use a fixed grid and a fixed-order second pass, so results are
// bitwise reproducible run to run.  Step lengths stay on the device.
#include <cmath>
#include <vector>

#include "rsd_internal.cuh"

namespace rsd {
namespace {

constexpr int RT = 256;          // threads per block for vector kernels
constexpr int RED_BLOCKS = 1024; // fixed first-pass grid of the reductions

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum; result valid in thread 0.
__device__ double block_sum(double v) {
    __shared__ double s[RT / 32];
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0;
    if (threadIdx.x < 32) {
        t = threadIdx.x < RT / 32 ? s[threadIdx.x] : 0.0;
        t = warp_sum(t);
    }
    __syncthreads();
    return t;
}

// y = K x, four lanes per row.
__global__ void k_spmv(int n, const int64_t* __restrict__ rowptr, const int* __restrict__ col,
                       const double* __restrict__ val, const double* __restrict__ x, double* __restrict__ y) {
    const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t row = gt >> 2;
    const int sub = threadIdx.x & 3;
    double s = 0;
    if (row < n) {
        for (int64_t k = rowptr[row] + sub; k < rowptr[row + 1]; k += 4) s += val[k] * __ldg(x + col[k]);
    }
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    if (row < n && sub == 0) y[row] = s;
}

__global__ void k_dot_partial(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                              double* __restrict__ partial) {
    double s = 0;
    for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT) s += a[i] * b[i];
    s = block_sum(s);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void k_reduce_final(const double* __restrict__ partial, int np, double* __restrict__ out) {
    double s = 0;
    for (int i = threadIdx.x; i < np; i += RT) s += partial[i];
    s = block_sum(s);
    if (threadIdx.x == 0) *out = s;
}

// alpha = rz / pq;  u += alpha p;  r -= alpha q;  partial sums of r.r
__global__ void k_cg_update(int64_t n, const double* __restrict__ scal, int rz_slot, double* __restrict__ u,
                            double* __restrict__ r, const double* __restrict__ p, const double* __restrict__ q,
                            double* __restrict__ partial) {
    const double alpha = scal[rz_slot] / scal[1];
    double s = 0;
    for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT) {
        u[i] += alpha * p[i];
        const double ri = r[i] - alpha * q[i];
        r[i] = ri;
        s += ri * ri;
    }
    s = block_sum(s);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// beta = rz_new / rz_old;  p = z + beta p
__global__ void k_cg_direction(int64_t n, const double* __restrict__ scal, int new_slot, int old_slot,
                               const double* __restrict__ z, double* __restrict__ p) {
    const double beta = scal[new_slot] / scal[old_slot];
    for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT)
        p[i] = z[i] + beta * p[i];
}

__global__ void k_residual(int n, const int64_t* __restrict__ rowptr, const int* __restrict__ col,
                           const double* __restrict__ val, const double* __restrict__ x,
                           const double* __restrict__ f, double* __restrict__ r) {
    const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t row = gt >> 2;
    const int sub = threadIdx.x & 3;
    double s = 0;
    if (row < n)
        for (int64_t k = rowptr[row] + sub; k < rowptr[row + 1]; k += 4) s += val[k] * __ldg(x + col[k]);
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    if (row < n && sub == 0) r[row] = f[row] - s;
}

// One modified Gram-Schmidt step of FGMRES, fused with the next inner product:
// w -= h v (h read from the device, skipped when v is null), then per-block partial sums
// of w . next (next = w gives ||w||^2 after the update).
__global__ void k_mgs_step(int64_t n, const double* __restrict__ hval, const double* __restrict__ v,
                           double* __restrict__ w, const double* __restrict__ next, double* __restrict__ partial) {
    const double hv = v ? *hval : 0.0;
    double s = 0;
    for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT) {
        double wi = w[i];
        if (v) {
            wi -= hv * v[i];
            w[i] = wi;
        }
        s += wi * (next == w ? wi : next[i]);
    }
    s = block_sum(s);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// dst = src / sqrt(*nrm2) (left unchanged when the norm is zero); *hout = sqrt(*nrm2)
__global__ void k_scale_by_norm(int64_t n, const double* __restrict__ nrm2, const double* __restrict__ src,
                                double* __restrict__ dst, double* __restrict__ hout) {
    const double nv = sqrt(fmax(*nrm2, 0.0));
    if (blockIdx.x == 0 && threadIdx.x == 0 && hout) *hout = nv;
    if (!(nv > 0.0)) return;
    const double inv = 1.0 / nv;
    for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT) dst[i] = src[i] * inv;
}

// x += sum_q y_q Z_q, q = 0 .. k-1 in order
__global__ void k_fg_update(int64_t n, int k, const double* __restrict__ y, const double* __restrict__ Z,
                            double* __restrict__ x) {
    for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT) {
        double a = x[i];
        for (int q = 0; q < k; ++q) a += y[q] * Z[(int64_t)q * n + i];
        x[i] = a;
    }
}

int dot(Handle& h, const double* a, const double* b, int slot) {
    const int pi = prof_begin(h, K_KRYLOV);
    k_dot_partial<<<RED_BLOCKS, RT, 0, h.stream>>>(h.n, a, b, h.d_partial);
    k_reduce_final<<<1, RT, 0, h.stream>>>(h.d_partial, RED_BLOCKS, h.d_scal + slot);
    count_launch(2);
    prof_end(h, pi, 2.0 * h.n, 16.0 * h.n);
    RSD_CUDA_TRY(cudaGetLastError());
    return RSD_OK;
}

int fetch(Handle& h, int slot, double* out) {
    RSD_CUDA_TRY(cudaMemcpyAsync(h.h_scal + slot, h.d_scal + slot, sizeof(double), cudaMemcpyDeviceToHost, h.stream));
    RSD_CUDA_TRY(cudaStreamSynchronize(h.stream));
    *out = h.h_scal[slot];
    return RSD_OK;
}

}  // namespace

int spmv(Handle& h, const double* x, double* y) {
    const int64_t threads = (int64_t)h.n * 4;
    const int pi = prof_begin(h, K_KRYLOV);
    k_spmv<<<(unsigned)((threads + RT - 1) / RT), RT, 0, h.stream>>>(h.n, h.d_rowptr, h.d_col, h.d_val, x, y);
    count_launch();
    prof_end(h, pi, 2.0 * h.nnz, 12.0 * h.nnz + 24.0 * h.n);
    RSD_CUDA_TRY(cudaGetLastError());
    return RSD_OK;
}

// PCG's preconditioner application on its fixed vectors r -> z as a CUDA graph, for a
// handle that solves more than once (an adjoint solve, a sequence of right-hand sides):
// the second solve captures run_apply (on a private stream: the caller's stream may be
// the legacy default stream, which cannot be captured) and every later application
// replays it on the caller's stream.  A first solve keeps direct launches (capturing and
// instantiating would cost more than it saves once), as do a profiled handle, whose
// launch records are host-side, and paper mode.
static int pcg_apply(Handle& h, const double* r, double* z) {
    if (h.paper) return run_apply_paper(h, r, z);
    if (h.prof.on || h.solve_calls < 2) return run_apply(h, r, z);
    if (!h.apply_exec) {
        cudaStream_t cap = nullptr;
        RSD_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaStream_t user = h.stream;
        const int64_t l0 = rsd_launch_count();
        h.stream = cap;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        int rc = e == cudaSuccess ? run_apply(h, r, z) : RSD_ERR_CUDA;
        cudaGraph_t g = nullptr;
        if (e == cudaSuccess) e = cudaStreamEndCapture(cap, &g);
        h.stream = user;
        cudaStreamDestroy(cap);
        h.apply_graph_launches = (int)(rsd_launch_count() - l0);
        count_launch(-h.apply_graph_launches);            // counted when replayed
        if (rc == RSD_OK && e == cudaSuccess) e = cudaGraphInstantiate(&h.apply_exec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (rc != RSD_OK) return rc;
        if (e != cudaSuccess) { cudaGetLastError(); h.apply_exec = nullptr; set_last_error("apply graph capture failed"); return RSD_ERR_CUDA; }
    }
    RSD_CUDA_TRY(cudaGraphLaunch(h.apply_exec, h.stream));
    count_launch(h.apply_graph_launches);
    return RSD_OK;
}

// Flexible right-preconditioned GMRES(m) in FP64 from x = 0 (the outer solver when the
// preconditioner changes with its input, as paper mode's gamma inner iterations make it):
// per cycle r = f - K x, v_0 = r / ||r||; per step z_j = M v_j, w = K z_j, modified
// Gram-Schmidt against v_0..v_j, v_{j+1} = w / h_{j+1,j}; the Hessenberg columns come to
// the host (one synchronisation per step), where Givens rotations give the least-squares
// residual estimate |g_{j+1}| / ||f|| tested against tol; at the end of a cycle
// x += Z y.  Stops on the estimate, then recomputes the true residual in FP64.
int fgmres(Handle& h, const double* f, double* x, double tol, rsd_stats* st) {
    ++h.solve_calls;
    const int64_t n = h.n;
    const int m = h.restart;
    const int maxit = h.opt.maxit > 0 ? h.opt.maxit : 200;
    rsd_stats local{};
    rsd_stats* S = st ? st : &local;
    *S = rsd_stats{};
    double* V = h.d_fg_V;
    double* Z = h.d_fg_Z;
    double* Hd = h.d_fg_H;                       // column j at Hd + j (m + 1)
    double* w = h.d_q;
    RSD_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * n, h.stream));
    RSD_TRY(dot(h, f, f, 4));
    double ff;
    RSD_TRY(fetch(h, 4, &ff));
    const double fnorm = std::sqrt(ff);
    S->history[0] = 1.0;
    if (fnorm == 0.0) { S->relres = 0; return RSD_OK; }
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
    int it = 0;
    double est = 1.0;
    int rc = RSD_ERR_NOCONV;
    bool first = true;
    while (it < maxit) {
        // r = f - K x into v_0 and beta = ||r||
        if (first) {
            RSD_CUDA_TRY(cudaMemcpyAsync(V, f, sizeof(double) * n, cudaMemcpyDeviceToDevice, h.stream));
            RSD_CUDA_TRY(cudaMemcpyAsync(h.d_scal + 6, h.d_scal + 4, sizeof(double), cudaMemcpyDeviceToDevice, h.stream));
        } else {
            const int64_t threads = n * 4;
            k_residual<<<(unsigned)((threads + RT - 1) / RT), RT, 0, h.stream>>>(h.n, h.d_rowptr, h.d_col, h.d_val, x, f, V);
            count_launch();
            RSD_TRY(dot(h, V, V, 6));
        }
        double bb;
        RSD_TRY(fetch(h, 6, &bb));
        const double beta = std::sqrt(std::max(bb, 0.0));
        if (!first && beta / fnorm <= tol) { rc = RSD_OK; break; }
        first = false;
        k_scale_by_norm<<<RED_BLOCKS, RT, 0, h.stream>>>(n, h.d_scal + 6, V, V, nullptr);
        count_launch();
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int jl = -1;
        bool done = false;
        for (int j = 0; j < m; ++j) {
            double* zj = Z + (int64_t)j * n;
            const double* vj = V + (int64_t)j * n;
            RSD_TRY(h.paper ? run_apply_paper(h, vj, zj) : run_apply(h, vj, zj));
            RSD_TRY(spmv(h, zj, w));
            double* hc = Hd + (int64_t)j * (m + 1);
            const int pk = prof_begin(h, K_KRYLOV);
            for (int i = 0; i <= j + 1; ++i) {
                // step i: subtract h_{i-1,j} v_{i-1} (i > 0), then w . v_i (or ||w||^2 at i = j + 1)
                const double* vprev = i > 0 ? V + (int64_t)(i - 1) * n : nullptr;
                const double* nxt = i <= j ? V + (int64_t)i * n : w;
                k_mgs_step<<<RED_BLOCKS, RT, 0, h.stream>>>(n, i > 0 ? hc + i - 1 : nullptr, vprev, w, nxt, h.d_partial);
                k_reduce_final<<<1, RT, 0, h.stream>>>(h.d_partial, RED_BLOCKS, i <= j ? hc + i : h.d_scal + 7);
                count_launch(2);
            }
            k_scale_by_norm<<<RED_BLOCKS, RT, 0, h.stream>>>(n, h.d_scal + 7, w, V + (int64_t)(j + 1) * n, hc + j + 1);
            count_launch();
            prof_end(h, pk, (4.0 * (j + 2)) * n, (24.0 * (j + 2) + 16.0) * n);
            RSD_CUDA_TRY(cudaGetLastError());
            RSD_CUDA_TRY(cudaMemcpyAsync(h.h_fg, hc, sizeof(double) * (j + 2), cudaMemcpyDeviceToHost, h.stream));
            RSD_CUDA_TRY(cudaStreamSynchronize(h.stream));
            for (int i = 0; i <= j + 1; ++i) H[(size_t)i * m + j] = h.h_fg[i];
            for (int i = 0; i < j; ++i) {             // earlier rotations
                const double t0 = H[(size_t)i * m + j], t1 = H[(size_t)(i + 1) * m + j];
                H[(size_t)i * m + j] = cs[i] * t0 + sn[i] * t1;
                H[(size_t)(i + 1) * m + j] = -sn[i] * t0 + cs[i] * t1;
            }
            const double a = H[(size_t)j * m + j], b = H[(size_t)(j + 1) * m + j];
            const double den = std::hypot(a, b);
            cs[j] = den > 0 ? a / den : 1.0;
            sn[j] = den > 0 ? b / den : 0.0;
            H[(size_t)j * m + j] = den;
            H[(size_t)(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            ++it;
            jl = j;
            est = std::fabs(g[j + 1]) / fnorm;
            if (it < 64) S->history[it] = est;
            if (!(est == est)) { rc = RSD_ERR_NOT_SPD; done = true; break; }
            if (est <= tol || it >= maxit || !(b > 0.0)) break;
        }
        if (jl >= 0) {
            for (int r = jl; r >= 0; --r) {
                double t = g[r];
                for (int c = r + 1; c <= jl; ++c) t -= H[(size_t)r * m + c] * y[c];
                y[r] = H[(size_t)r * m + r] != 0.0 ? t / H[(size_t)r * m + r] : 0.0;
            }
            for (int q = 0; q <= jl; ++q) h.h_fg[128 + q] = y[q];
            RSD_CUDA_TRY(cudaMemcpyAsync(h.d_fg_y, h.h_fg + 128, sizeof(double) * (jl + 1), cudaMemcpyHostToDevice, h.stream));
            k_fg_update<<<RED_BLOCKS, RT, 0, h.stream>>>(n, jl + 1, h.d_fg_y, Z, x);
            count_launch();
            RSD_CUDA_TRY(cudaGetLastError());
            RSD_CUDA_TRY(cudaStreamSynchronize(h.stream));    // h_fg is rewritten by the next cycle
        }
        if (done) break;
        if (est <= tol) { rc = RSD_OK; break; }
    }
    S->iterations = it;
    S->relres_recursive = est;
    const int64_t threads = n * 4;
    k_residual<<<(unsigned)((threads + RT - 1) / RT), RT, 0, h.stream>>>(h.n, h.d_rowptr, h.d_col, h.d_val, x, f, w);
    count_launch();
    RSD_CUDA_TRY(cudaGetLastError());
    RSD_TRY(dot(h, w, w, 5));
    double tr;
    RSD_TRY(fetch(h, 5, &tr));
    S->relres = std::sqrt(tr) / fnorm;
    return rc;
}

// Scalar slots: 0 rz (even iterations), 1 pq, 2 rr, 3 rz (odd iterations), 4 ff, 5 true rr,
// 6 FGMRES ||r||^2, 7 FGMRES ||w||^2
int pcg(Handle& h, const double* f, double* u, double tol, rsd_stats* st) {
    ++h.solve_calls;
    const int64_t n = h.n;
    double* r = h.d_r;
    double* p = h.d_p;
    double* q = h.d_q;
    double* z = h.d_z;
    const int maxit = h.opt.maxit > 0 ? h.opt.maxit : 200;
    rsd_stats local{};
    rsd_stats* S = st ? st : &local;
    *S = rsd_stats{};
    RSD_CUDA_TRY(cudaMemsetAsync(u, 0, sizeof(double) * n, h.stream));
    RSD_CUDA_TRY(cudaMemcpyAsync(r, f, sizeof(double) * n, cudaMemcpyDeviceToDevice, h.stream));
    RSD_TRY(dot(h, f, f, 4));
    double ff;
    RSD_TRY(fetch(h, 4, &ff));
    const double fnorm = std::sqrt(ff);
    S->history[0] = 1.0;
    if (fnorm == 0.0) { S->relres = 0; return RSD_OK; }
    RSD_TRY(pcg_apply(h, r, z));
    RSD_CUDA_TRY(cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, h.stream));
    RSD_TRY(dot(h, r, z, 0));
    int it = 0;
    double rel = 1.0;
    int rc = RSD_ERR_NOCONV;
    for (it = 1; it <= maxit; ++it) {
        const int old_slot = (it & 1) ? 0 : 3, new_slot = (it & 1) ? 3 : 0;
        RSD_TRY(spmv(h, p, q));
        RSD_TRY(dot(h, p, q, 1));
        const int pu = prof_begin(h, K_KRYLOV);
        k_cg_update<<<RED_BLOCKS, RT, 0, h.stream>>>(n, h.d_scal, old_slot, u, r, p, q, h.d_partial);
        k_reduce_final<<<1, RT, 0, h.stream>>>(h.d_partial, RED_BLOCKS, h.d_scal + 2);
        count_launch(2);
        prof_end(h, pu, 6.0 * n, 48.0 * n);
        RSD_CUDA_TRY(cudaGetLastError());
        double rr;
        RSD_TRY(fetch(h, 2, &rr));
        rel = std::sqrt(std::max(rr, 0.0)) / fnorm;
        if (it < 64) S->history[it] = rel;
        if (!(rel == rel)) { rc = RSD_ERR_NOT_SPD; break; }
        if (rel <= tol) { rc = RSD_OK; break; }
        RSD_TRY(pcg_apply(h, r, z));
        RSD_TRY(dot(h, r, z, new_slot));
        const int pd = prof_begin(h, K_KRYLOV);
        k_cg_direction<<<RED_BLOCKS, RT, 0, h.stream>>>(n, h.d_scal, new_slot, old_slot, z, p);
        count_launch();
        prof_end(h, pd, 2.0 * n, 24.0 * n);
        RSD_CUDA_TRY(cudaGetLastError());
    }
    S->iterations = std::min(it, maxit);
    S->relres_recursive = rel;
    // true residual in FP64
    const int64_t threads = n * 4;
    const int pr = prof_begin(h, K_KRYLOV);
    k_residual<<<(unsigned)((threads + RT - 1) / RT), RT, 0, h.stream>>>(h.n, h.d_rowptr, h.d_col, h.d_val, u, f, q);
    count_launch();
    prof_end(h, pr, 2.0 * h.nnz, 12.0 * h.nnz + 32.0 * h.n);
    RSD_CUDA_TRY(cudaGetLastError());
    RSD_TRY(dot(h, q, q, 5));
    double tr;
    RSD_TRY(fetch(h, 5, &tr));
    S->relres = std::sqrt(tr) / fnorm;
    return rc;
}

}  // namespace rsd
