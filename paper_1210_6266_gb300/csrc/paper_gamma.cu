// Paper mode with gamma inner GMRES iterations (Sec. 3.2, Algorithms 1 and 2): every
// interface system S~_t u_t = g_t of a tree level is solved approximately by gamma
// GMRES iterations from u = 0 (no restart, modified Gram-Schmidt, no preconditioner),
// all interfaces of the level at once; S~ is never formed.
//
// S-MatVec (Algorithm 1) for interface t:
//     y = K_{I_t I_t} x - sum_{l in V-hat_t} K_{I_t l} K_ll^-1 K_{l I_t} x.
// Setup factors every leaf front [K_ll K_lB; K_Bl .] into L_l and X_l = K_{B_l l} L_l^-T
// (rows: the ancestor DOFs B_l coupled to l), so with R = the rows of X_l that lie in I_t,
//     K_{I_t l} K_ll^-1 K_{l I_t} = (K_{I_t l} L_l^-T)(L_l^-1 K_{l I_t}) = X_l[R] X_l[R]^T:
// the two leaf solves of Algorithm 1 become two streaming products with X_l[R]: t_l =
// X_l[R]^T x (column-parallel), then one row product X_l[row] . t_l per coupling, summed
// per interface DOF over the leaves that touch it in a fixed order.
// V-hat_t is exactly the set of leaves with a nonempty R for t (a leaf couples to its
// ancestors' DOFs only, Eq. 3.1).
//
// Vectors of a level are packed: interface slot i of the level owns positions
// [if_off[i], if_off[i+1]) in I_t order (pk_pos maps a global DOF to its position).
// Every reduction has a fixed order, so results are bitwise reproducible.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <type_traits>

#include "cluster.cuh"
#include "rsd_internal.cuh"

namespace rsd {
namespace {

constexpr int GT = 512;           // threads of the per-interface GMRES kernels
constexpr int GAMMA_MAX = 32;     // largest gamma (inner iterations) the kernels hold

// Block-wide sum in a fixed order; every thread receives the result.
__device__ double block_sum_all(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        double t = lane < nw ? red[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) red[32] = t;
    }
    __syncthreads();
    return red[32];
}

// Products with a leaf's X block accumulate in the block's own precision (A = T): FP32
// blocks of the mixed form in FP32, as the substitution sweeps do, FP64 blocks in FP64.
// With H16 (T = float) they read the leaf's FP16 copy instead: row i of P scaled by the
// power of two rs_i, so exactly the factor's TF32 values down to 2^-27 sqrt(K_ii); x enters
// scaled by ri of its row and a row product is scaled by ri once, at half the bytes.
template <typename T> struct VecOf;
template <> struct VecOf<float> { using V = float4; };
template <> struct VecOf<double> { using V = double2; };

template <typename T, bool H16> struct SmvElems { static constexpr int W = 16 / (int)sizeof(T); };
template <> struct SmvElems<float, true> { static constexpr int W = 8; };

// The W elements of one 16-byte load at p (a row of X, element offset c).
template <typename T, bool H16>
__device__ __forceinline__ void smv_load(const void* p, int64_t off, T (&o)[SmvElems<T, H16>::W]) {
    if constexpr (H16) {
        const uint4 u = __ldg((const uint4*)((const __half*)p + off));
        const __half2* h = reinterpret_cast<const __half2*>(&u);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 f = __half22float2(h[k]);
            o[2 * k] = f.x;
            o[2 * k + 1] = f.y;
        }
    } else {
        using V = typename VecOf<T>::V;
        const V v = __ldg((const V*)((const T*)p + off));
        const T* e = (const T*)&v;
#pragma unroll
        for (int k = 0; k < SmvElems<T, H16>::W; ++k) o[k] = e[k];
    }
}

// t_l = X_l[R_l]^T x for every leaf with rows coupled to the level; one CTA per (leaf, 32 x W
// columns), W columns per lane read with one 16-byte load per row.  The rows' offsets and x
// values are staged in shared memory 256 at a time; the eight warps take every eighth row
// (many loads in flight per column tile instead of one serial walk over the leaf's rows)
// and their partial sums are added in warp order.
template <typename T, bool H16>
__global__ void __launch_bounds__(256) k_smv_leaf(const FrontDesc* __restrict__ leaves, const int* __restrict__ cl_ptr,
                                                  const int* __restrict__ cl_row, const int* __restrict__ cl_pos,
                                                  const int* __restrict__ tl_off, const double* __restrict__ x,
                                                  T* __restrict__ tl) {
    constexpr int W = SmvElems<T, H16>::W, CT = 32 * W;
    __shared__ int s_row[256];
    __shared__ T s_x[256];
    __shared__ T s_red[8][CT];
    const int l = blockIdx.x;
    const int k0 = cl_ptr[l], k1 = cl_ptr[l + 1];
    const int s = leaves[l].s, ldp = leaves[l].ldp;
    const int c0 = blockIdx.y * CT;
    if (k0 == k1 || c0 >= s) return;
    const void* X = H16 ? (const void*)((const __half*)leaves[l].P16 + (int64_t)s * ldp)
                        : (const void*)((const T*)leaves[l].P + (int64_t)s * ldp);
    const float* ri = H16 ? leaves[l].ri + s : nullptr;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = c0 + lane * W;
    T acc[W];
#pragma unroll
    for (int e = 0; e < W; ++e) acc[e] = 0;
    for (int kb = k0; kb < k1; kb += 256) {
        const int nb = min(256, k1 - kb);
        __syncthreads();
        if ((int)threadIdx.x < nb) {
            const int row = cl_row[kb + threadIdx.x];
            s_row[threadIdx.x] = row;
            const T xv = (T)x[cl_pos[kb + threadIdx.x]];
            s_x[threadIdx.x] = H16 ? xv * (T)ri[row] : xv;
        }
        __syncthreads();
        if (c < s) {
#pragma unroll 4
            for (int q = warp; q < nb; q += 8) {
                T e[W];
                smv_load<T, H16>(X, (int64_t)s_row[q] * ldp + c, e);
                const T xv = s_x[q];
#pragma unroll
                for (int u = 0; u < W; ++u) acc[u] += e[u] * xv;
            }
        }
    }
#pragma unroll
    for (int e = 0; e < W; ++e) s_red[warp][lane * W + e] = acc[e];
    __syncthreads();
    T* out = tl + tl_off[l];
    for (int e = threadIdx.x; e < CT; e += blockDim.x) {
        if (c0 + e >= s) break;
        T v = 0;
#pragma unroll
        for (int w = 0; w < 8; ++w) v += s_red[w][e];
        out[c0 + e] = v;
    }
}

// The W entries of t at c (16- or 32-byte aligned: t_l slots start at multiples of 8
// elements and c is a multiple of W).
template <typename T, int W>
__device__ __forceinline__ void smv_tload(const T* t, T (&o)[W]) {
    if constexpr (sizeof(T) * W == 32) {
        const float4 a = __ldg((const float4*)t), b = __ldg((const float4*)t + 1);
        const float v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
        for (int q = 0; q < W; ++q) o[q] = v[q];
    } else {
        using V = typename VecOf<T>::V;
        const V v = __ldg((const V*)t);
        const T* e = (const T*)&v;
#pragma unroll
        for (int q = 0; q < W; ++q) o[q] = e[q];
    }
}

// yl_k = X_l[row_k] . t_l for every coupling k (a row of a leaf's X block that lies in the
// level's interfaces).  One warp per group of R consecutive couplings: couplings are grouped
// by leaf, so a group of one leaf reads each chunk of t_l once for its R rows (16-byte loads
// along the rows); a group that straddles two leaves takes its rows one at a time.  Either
// way a row's sum runs in the same order (lane-strided chunks, the ragged tail, then the
// butterfly), so the result does not depend on the grouping.
template <typename T, bool H16>
__global__ void __launch_bounds__(256) k_smv_rows(int nk, const int* __restrict__ cl_leaf, const int* __restrict__ cl_row,
                                                  const FrontDesc* __restrict__ leaves, const int* __restrict__ tl_off,
                                                  const T* __restrict__ tl, double* __restrict__ yl) {
    constexpr int W = SmvElems<T, H16>::W, R = 4;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t ng = ((int64_t)nk + R - 1) / R;
    for (int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; g < ng; g += warps) {
        const int64_t k0 = g * R;
        const int nr = (int)(nk - k0 < R ? nk - k0 : R);
        const bool shared = nr == R && cl_leaf[k0] == cl_leaf[k0 + R - 1];
        for (int r0 = 0; r0 < nr; r0 += shared ? R : 1) {
            const int m = shared ? R : 1;            // rows summed together
            const int l = cl_leaf[k0 + r0];
            const int s = leaves[l].s, ldp = leaves[l].ldp;
            const void* base = H16 ? (const void*)leaves[l].P16 : (const void*)leaves[l].P;
            const T* t = tl + tl_off[l];
            int64_t roff[R];
            T d[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                roff[r] = r < m ? (int64_t)(s + cl_row[k0 + r0 + r]) * ldp : 0;
                d[r] = 0;
            }
            const int sv = s / W * W;
#pragma unroll 1
            for (int c = lane * W; c < sv; c += 32 * W) {
                T tv[W];
                smv_tload<T, W>(t + c, tv);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if (r < m) {
                        T e[W];
                        smv_load<T, H16>(base, roff[r] + c, e);
#pragma unroll
                        for (int q = 0; q < W; ++q) d[r] += e[q] * tv[q];
                    }
                }
            }
            for (int c = sv + lane; c < s; c += 32) {
                const T tv = t[c];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if (r < m) {
                        const T v = H16 ? (T)__half2float(((const __half*)base)[roff[r] + c]) : ((const T*)base)[roff[r] + c];
                        d[r] += v * tv;
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) d[r] += __shfl_xor_sync(0xffffffffu, d[r], o);
                if (lane == 0 && r < m) {
                    const int64_t k = k0 + r0 + r;
                    yl[k] = H16 ? (double)(d[r] * (T)leaves[l].ri[s + cl_row[k]]) : (double)d[r];
                }
            }
        }
    }
}

// y_p = (K_{I_t I_t} x)_p - sum of yl_k over the couplings k of position p.  Eight lanes
// per packed position (four positions per warp): the lanes take every eighth entry of the
// row and every eighth coupling, and their partial sums meet in a fixed butterfly, so the
// gathers of four rows are in flight at once.
__global__ void __launch_bounds__(256) k_smv_iface(int S, const int* __restrict__ if_dofs, const int64_t* __restrict__ rowptr,
                                                   const int* __restrict__ col, const double* __restrict__ val,
                                                   const int* __restrict__ owner, const int* __restrict__ pk_pos,
                                                   const int* __restrict__ ci_ptr, const int* __restrict__ ci_k,
                                                   const double* __restrict__ yl, const double* __restrict__ x,
                                                   double* __restrict__ y) {
    const int lane = threadIdx.x & 31, sub = lane & 7;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    // warp-uniform trip count: every lane reaches the shuffles
    for (int64_t pw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; pw * 4 < S; pw += warps) {
        const int64_t p = pw * 4 + (lane >> 3);
        double acc = 0;
        if (p < S) {
            const int dof = if_dofs[p];
            const int o = owner[dof];
            for (int64_t k = rowptr[dof] + sub; k < rowptr[dof + 1]; k += 8) {
                const int j = col[k];
                if (owner[j] == o) acc += val[k] * x[pk_pos[j]];
            }
            for (int q = ci_ptr[p] + sub; q < ci_ptr[p + 1]; q += 8) acc -= yl[ci_k[q]];
        }
        acc += __shfl_xor_sync(0xffffffffu, acc, 4);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        if (sub == 0 && p < S) y[p] = acc;
    }
}

// The GMRES vector kernels give each interface a cluster of GC CTAs, CTA r of the cluster
// holding the r-th contiguous chunk of the interface's entries, so a long interface (the
// root's) is spread over GC SMs instead of one.
constexpr int GC = 8;

struct GmChunk {
    int i, o, s, lo, hi;        // interface, its offset and size; this CTA's entries [lo, hi)
};

__device__ __forceinline__ GmChunk gm_chunk(const int* __restrict__ if_off, int i, int r) {
    GmChunk c;
    c.i = i;
    c.o = if_off[i];
    c.s = if_off[i + 1] - c.o;
    const int per = (c.s + GC - 1) / GC;
    c.lo = min(c.s, r * per);
    c.hi = min(c.s, c.lo + per);
    return c;
}

// Sum over the cluster in a fixed order: each CTA's block sum (block_sum_all), then the GC
// partials added in rank order by every CTA, so every thread of the cluster gets the same
// bits.  part[] alternates between calls: a CTA rewrites part[p] only after the barrier of
// the call in between, which every CTA passes after its reads of part[p].
__device__ double cluster_sum_all(double v, double* red, double* part, double* tot, int& p) {
    const double b = block_sum_all(v, red);
    if (threadIdx.x == 0) part[p] = b;
    cl_sync();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int r = 0; r < GC; ++r) t += cl_ld_f64(cl_map(&part[p], (uint32_t)r));
        *tot = t;
    }
    __syncthreads();
    p ^= 1;
    return *tot;
}

// v_0 = g / beta on every interface of the level (g indexed by global DOF).
__global__ void __cluster_dims__(GC, 1, 1) __launch_bounds__(GT)
    k_gm_init(const int* __restrict__ if_off, const int* __restrict__ if_dofs, const double* __restrict__ g,
              double* __restrict__ V, double* __restrict__ beta, int* __restrict__ kused) {
    __shared__ double red[33], part[2], tot;
    const int r = (int)cl_rank();
    const GmChunk c = gm_chunk(if_off, blockIdx.x / GC, r);
    int p = 0;
    double a = 0;
    for (int e = c.lo + threadIdx.x; e < c.hi; e += blockDim.x) { const double v = g[if_dofs[c.o + e]]; a += v * v; }
    const double b = sqrt(cluster_sum_all(a, red, part, &tot, p));
    if (r == 0 && threadIdx.x == 0) { beta[c.i] = b; kused[c.i] = b > 0.0 ? 0 : -1; }
    const double inv = b > 0.0 ? 1.0 / b : 0.0;
    for (int e = c.lo + threadIdx.x; e < c.hi; e += blockDim.x) V[c.o + e] = g[if_dofs[c.o + e]] * inv;
    cl_sync();                                  // no CTA leaves while a peer reads its partials
}

// Arnoldi step j with modified Gram-Schmidt on w = S~ v_j, per interface: h_qj = <w, v_q>,
// w -= h_qj v_q for q = 0..j in turn, h_{j+1,j} = ||w||, v_{j+1} = w / h_{j+1,j}.  One pass
// over the chunk per q: the update by v_q and the product with v_{q+1} (or w's norm after
// the last) of the updated entries.  An interface whose h_{j+1,j} falls to 1e-14 beta
// (exact breakdown) stops with j + 1 columns; one that completes min(gamma, s) steps stops
// with that many.
__global__ void __cluster_dims__(GC, 1, 1) __launch_bounds__(GT)
    k_gm_mgs(int j, int gamma, int S, const int* __restrict__ if_off, double* __restrict__ w, double* __restrict__ V,
             double* __restrict__ H, const double* __restrict__ beta, int* __restrict__ kused) {
    __shared__ double red[33], part[2], tot;
    const int r = (int)cl_rank();
    const GmChunk c = gm_chunk(if_off, blockIdx.x / GC, r);
    const int m = min(gamma, c.s);
    if (kused[c.i] != 0 || j >= m) return;     // the whole cluster
    const bool lead = r == 0 && threadIdx.x == 0;
    double* Hi = H + (int64_t)c.i * (gamma + 1) * gamma;
    double* wi = w + c.o;
    int p = 0;
    double a = 0;
    for (int e = c.lo + threadIdx.x; e < c.hi; e += blockDim.x) a += wi[e] * V[c.o + e];
    double hq = cluster_sum_all(a, red, part, &tot, p);
    for (int q = 0; q <= j; ++q) {
        if (lead) Hi[q * gamma + j] = hq;
        const double* vq = V + (int64_t)q * S + c.o;
        a = 0;
        if (q < j) {
            const double* vn = vq + S;
#pragma unroll 4
            for (int e = c.lo + threadIdx.x; e < c.hi; e += blockDim.x) {
                const double x = wi[e] - hq * vq[e];
                wi[e] = x;
                a += x * vn[e];
            }
        } else {
#pragma unroll 4
            for (int e = c.lo + threadIdx.x; e < c.hi; e += blockDim.x) {
                const double x = wi[e] - hq * vq[e];
                wi[e] = x;
                a += x * x;
            }
        }
        hq = cluster_sum_all(a, red, part, &tot, p);
    }
    const double nrm = sqrt(hq);
    if (lead) Hi[(j + 1) * gamma + j] = nrm;
    if (nrm <= 1e-14 * beta[c.i]) {
        if (lead) kused[c.i] = j + 1;
    } else {
        double* vn = V + (int64_t)(j + 1) * S + c.o;
        for (int e = c.lo + threadIdx.x; e < c.hi; e += blockDim.x) vn[e] = wi[e] / nrm;
        if (j + 1 == m && lead) kused[c.i] = m;
    }
    cl_sync();                                  // no CTA leaves while a peer reads its partials
}

// u_t = V_k y with y the least-squares solution of min || beta e1 - H_k y || (H_k the
// (k+1) x k Hessenberg matrix; Givens rotations), written to z on the interface DOFs.
// Every CTA of an interface solves the small problem itself (the same bits) and writes
// its chunk.
__global__ void __launch_bounds__(GT) k_gm_finish(int gamma, int S, const int* __restrict__ if_off,
                                                  const int* __restrict__ if_dofs, const double* __restrict__ V,
                                                  const double* __restrict__ H, const double* __restrict__ beta,
                                                  const int* __restrict__ kused, double* __restrict__ z) {
    __shared__ double y[GAMMA_MAX];
    __shared__ double R[GAMMA_MAX + 1][GAMMA_MAX];      // rotated Hessenberg
    __shared__ double gv[GAMMA_MAX + 1];
    const GmChunk c = gm_chunk(if_off, blockIdx.x / GC, blockIdx.x % GC);
    const int ku = kused[c.i];
    const int k = ku < 0 ? 0 : (ku == 0 ? min(gamma, c.s) : ku);
    if (threadIdx.x == 0 && k > 0) {
        const double* Hi = H + (int64_t)c.i * (gamma + 1) * gamma;
        for (int r = 0; r <= k; ++r)
            for (int cc = 0; cc < k; ++cc) R[r][cc] = (r <= cc + 1) ? Hi[r * gamma + cc] : 0.0;
        for (int r = 0; r <= k; ++r) gv[r] = 0.0;
        gv[0] = beta[c.i];
        for (int cc = 0; cc < k; ++cc) {
            const double a = R[cc][cc], b = R[cc + 1][cc];
            const double den = hypot(a, b);
            const double cs = den > 0 ? a / den : 1.0, sn = den > 0 ? b / den : 0.0;
            for (int c2 = cc; c2 < k; ++c2) {
                const double t0 = R[cc][c2], t1 = R[cc + 1][c2];
                R[cc][c2] = cs * t0 + sn * t1;
                R[cc + 1][c2] = -sn * t0 + cs * t1;
            }
            const double g0 = gv[cc], g1 = gv[cc + 1];
            gv[cc] = cs * g0 + sn * g1;
            gv[cc + 1] = -sn * g0 + cs * g1;
        }
        for (int r = k - 1; r >= 0; --r) {
            double t = gv[r];
            for (int c2 = r + 1; c2 < k; ++c2) t -= R[r][c2] * y[c2];
            y[r] = R[r][r] != 0.0 ? t / R[r][r] : 0.0;
        }
    }
    __syncthreads();
    for (int e = c.lo + threadIdx.x; e < c.hi; e += blockDim.x) {
        double u = 0;
        for (int q = 0; q < k; ++q) u += y[q] * V[(int64_t)q * S + c.o + e];
        z[if_dofs[c.o + e]] = u;
    }
}

}  // namespace

// Apply-time launches of one level's inner GMRES: reads g (global DOF order, h.d_pg) on
// the level's interface DOFs and writes u_t = GMRES_gamma(S~_t, g_t) into z there.
int gamma_interface_solve(Handle& h, int li, double* z) {
    GammaLevel& G = h.gamma_levels[li];
    if (G.n_if == 0 || G.S == 0) return RSD_OK;
    const Level& Ll = h.levels.back();
    const int nleaf = (int)Ll.fronts.size();
    // t_l = (L_l^-1 K_{l I})[:, R] x reads Y^T (the backward descriptors) for nonsymmetric
    // leaves; for symmetric ones Y^T = X
    const FrontDesc* ty = Ll.d_fronts_bwd ? Ll.d_fronts_bwd : Ll.d_fronts;
    const bool f64 = is_fp64(Ll.prec);
    // the leaves' FP16 copy when they have one (16-bit operand levels; not the transposed
    // upper factors of nonsymmetric leaves)
    const bool c16 = smv_reads_fp16(Ll);
    const int gam = h.gamma;
    int pi = prof_begin(h, K_GAMMA);
    k_gm_init<<<G.n_if * GC, GT, 0, h.stream>>>(G.d_if_off, G.d_if_dofs, h.d_pg, h.d_gm_V, h.d_gm_beta, h.d_gm_kused);
    count_launch();
    prof_end(h, pi, 0.0, 0.0);
    const int wcol = f64 ? 2 : (c16 ? 8 : 4);     // columns per lane of k_smv_leaf
    const dim3 gl((unsigned)nleaf, (unsigned)std::max(1, (Ll.max_s + 32 * wcol - 1) / (32 * wcol)));
    const unsigned gi = (unsigned)std::max(1, std::min(h.num_sms * 8, (G.S + 31) / 32));   // 32 positions per CTA
    for (int j = 0; j < gam; ++j) {
        const double* vj = h.d_gm_V + (int64_t)j * G.S;
        const unsigned gr = (unsigned)std::max(1, std::min(h.num_sms * 4, (G.nk + 31) / 32));   // 8 warps of 4 rows
        pi = prof_begin(h, K_GAMMA_SMV);
        if (f64) {
            k_smv_leaf<double, false><<<gl, 256, 0, h.stream>>>(ty, G.d_cl_ptr, G.d_cl_row, G.d_cl_pos, h.d_tl_off, vj,
                                                                h.d_tl);
            k_smv_rows<double, false><<<gr, 256, 0, h.stream>>>(G.nk, G.d_cl_leaf, G.d_cl_row, Ll.d_fronts, h.d_tl_off,
                                                                h.d_tl, h.d_gm_yl);
        } else if (c16) {
            float* tl32 = (float*)h.d_tl;
            k_smv_leaf<float, true><<<gl, 256, 0, h.stream>>>(Ll.d_fronts, G.d_cl_ptr, G.d_cl_row, G.d_cl_pos, h.d_tl_off,
                                                              vj, tl32);
            k_smv_rows<float, true><<<gr, 256, 0, h.stream>>>(G.nk, G.d_cl_leaf, G.d_cl_row, Ll.d_fronts, h.d_tl_off, tl32,
                                                              h.d_gm_yl);
        } else {
            float* tl32 = (float*)h.d_tl;
            k_smv_leaf<float, false><<<gl, 256, 0, h.stream>>>(ty, G.d_cl_ptr, G.d_cl_row, G.d_cl_pos, h.d_tl_off, vj,
                                                               tl32);
            k_smv_rows<float, false><<<gr, 256, 0, h.stream>>>(G.nk, G.d_cl_leaf, G.d_cl_row, Ll.d_fronts, h.d_tl_off,
                                                               tl32, h.d_gm_yl);
        }
        prof_end(h, pi, 0.0, G.xbytes);
        pi = prof_begin(h, K_GAMMA_IFACE);
        k_smv_iface<<<gi, 256, 0, h.stream>>>(G.S, G.d_if_dofs, h.d_rowptr, h.d_col, h.d_val, h.d_owner, h.d_pk_pos,
                                              G.d_ci_ptr, G.d_ci_k, h.d_gm_yl, vj, h.d_gm_w);
        prof_end(h, pi, 0.0, 0.0);
        pi = prof_begin(h, K_GAMMA);
        k_gm_mgs<<<G.n_if * GC, GT, 0, h.stream>>>(j, gam, G.S, G.d_if_off, h.d_gm_w, h.d_gm_V, h.d_gm_H, h.d_gm_beta, h.d_gm_kused);
        prof_end(h, pi, 0.0, 0.0);
        count_launch(4);
    }
    pi = prof_begin(h, K_GAMMA);
    k_gm_finish<<<G.n_if * GC, GT, 0, h.stream>>>(gam, G.S, G.d_if_off, G.d_if_dofs, h.d_gm_V, h.d_gm_H, h.d_gm_beta,
                                             h.d_gm_kused, z);
    count_launch();
    prof_end(h, pi, 0.0, 0.0);
    RSD_CUDA_TRY(cudaGetLastError());
    return RSD_OK;
}

}  // namespace rsd
