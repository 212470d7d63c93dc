// Preconditioner application z = M r (Algorithm 2 in its exact limit).
//
// Upward sweep, deepest level first: each front gathers r on I_t and adds its children's
// contributions (the K_IL K_LL^-1 f_L terms of g in Eq. 3.2), solves L y = v_I and forms
// its own contribution v_B - X y for the parent.  Downward sweep, root first: each front
// gathers the ancestors' solution on B_t and back-substitutes L^T x_I = y - X^T x_B
// (Eq. 3.3), writing x_I into z.
//
// The triangular solves are split into NB-row (upward) / NB-column (downward) blocks.
// Blocks of all fronts of a level form one work list; a persistent grid takes blocks
// from the list with an atomic ticket, so a block only ever waits for blocks with a
// smaller ticket, which are already held by running CTAs (no deadlock without
// co-residency).  A block that consumes a result from another block polls that front's
// progress counter with a bounded wait; on timeout it raises ERR_TIMEOUT and proceeds.
// The factor is streamed once per sweep with 16-byte non-coherent loads.
#include <cuda_fp16.h>

#include <algorithm>
#include <climits>
#include <mutex>

#include "cluster.cuh"
#include "rsd_internal.cuh"

namespace rsd {
namespace {

constexpr int AT = 256;                  // threads per CTA
constexpr int AW = AT / 32;              // warps

template <typename T> struct Vec;
template <> struct Vec<float> { using V = float4; static constexpr int W = 4; };
template <> struct Vec<double> { using V = double2; static constexpr int W = 2; };

__device__ __forceinline__ float vget(const float4& v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }
__device__ __forceinline__ double vget(const double2& v, int i) { return i == 0 ? v.x : v.y; }

template <typename T> __device__ __forceinline__ T ld_cg(const T* p);
template <> __device__ __forceinline__ float ld_cg(const float* p) { return __ldcg(p); }
template <> __device__ __forceinline__ double ld_cg(const double* p) { return __ldcg(p); }

__device__ __forceinline__ int ld_volatile(const int* p) { return *(volatile const int*)p; }

// A level with the FP16 factor copy (H = true, T = float) streams it instead of P: row i
// holds rs[i] P[i, :] with rs[i] a power of two, so a sweep multiplies a row's partial
// sum by ri[i] (forward) or the row's x by ri[i] (backward) -- the products and sums of
// the FP32 factor, scaled by powers of two, except for entries below 2^-27 sqrt(K_ii),
// which the copy holds as FP16 subnormals.  A lane reads 8 entries (16 B) per load, so
// a step covers two column blocks (forward) or two row blocks (backward) with as many
// bytes in flight as the FP32 loop.
template <typename T, bool H> struct PType { using type = T; };
template <typename T> struct PType<T, true> { using type = __half; };

// Two FP16 entries packed in a word (lower address in the low half) widened to FP32.
__device__ __forceinline__ float h_lo(uint32_t w) { return __half2float(__ushort_as_half((unsigned short)(w & 0xffffu))); }
__device__ __forceinline__ float h_hi(uint32_t w) { return __half2float(__ushort_as_half((unsigned short)(w >> 16))); }

__device__ __forceinline__ void h8_to_f(const uint4& u, float (&o)[8]) {
    o[0] = h_lo(u.x); o[1] = h_hi(u.x); o[2] = h_lo(u.y); o[3] = h_hi(u.y);
    o[4] = h_lo(u.z); o[5] = h_hi(u.z); o[6] = h_lo(u.w); o[7] = h_hi(u.w);
}

// Shared-memory factor block entries as V (four entries; FP16 widened).
template <typename T, bool H>
__device__ __forceinline__ typename Vec<T>::V lds_v(const typename PType<T, H>::type* p) {
    if constexpr (H) {
        const uint2 u = *reinterpret_cast<const uint2*>(p);
        return make_float4(h_lo(u.x), h_hi(u.x), h_lo(u.y), h_hi(u.y));
    } else {
        return *reinterpret_cast<const typename Vec<T>::V*>(p);
    }
}

// Asynchronous copies into shared memory (16 B per cp.async, L2 only), committed by
// cp_async_commit() and completed by cp_async_wait() before use: `count` consecutive
// NB x NB inverted diagonal blocks, or `rows` rows of NB entries from a row-major panel.
template <typename T>
__device__ __forceinline__ void prefetch_blocks(T* dst, const T* src, int count) {
    const int chunks = count * NB * NB * (int)sizeof(T) / 16;
    const uint32_t d0 = (uint32_t)__cvta_generic_to_shared(dst);
    for (int c = threadIdx.x; c < chunks; c += blockDim.x)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d0 + 16 * c), "l"((const char*)src + 16 * c)
                     : "memory");
}

template <typename T>
__device__ __forceinline__ void prefetch_rows(T* dst, const T* src, int ld, int rows) {
    constexpr int RC = NB * (int)sizeof(T) / 16;         // 16-byte chunks per row
    const uint32_t d0 = (uint32_t)__cvta_generic_to_shared(dst);
    for (int c = threadIdx.x; c < rows * RC; c += blockDim.x) {
        const int r = c / RC, q = c % RC;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
                     ::"r"(d0 + (uint32_t)(r * NB * (int)sizeof(T) + 16 * q)),
                       "l"((const char*)(src + (int64_t)r * ld) + 16 * q) : "memory");
    }
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Wait until *flag >= target; returns the last value seen.  Thread 0 polls, the block syncs.
// After `limit` clock cycles (the handle's wait bound) the wait gives up, raises
// ERR_TIMEOUT and returns as if the target had been reached; once the flag is raised,
// every later wait of the launch returns at once.
__device__ int wait_flag(const int* flag, int target, int* err, int* s_val, long long limit) {
    if (threadIdx.x == 0) {
        int v = ld_volatile(flag);
        if (v < target) {
            const long long t0 = clock64();
            while ((v = ld_volatile(flag)) < target) {
                if (ld_volatile(&err[ERR_TIMEOUT]) || clock64() - t0 > limit) {
                    atomicExch(&err[ERR_TIMEOUT], 1);
                    v = target;
                    break;
                }
                __nanosleep(20);
            }
        }
        __threadfence();
        *s_val = v;
    }
    __syncthreads();
    return *s_val;
}

// Threads that stored results fence them; after the barrier one thread raises the flag.
__device__ void publish_flag(int* flag, int value, bool wrote) {
    if (wrote) __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) atomicExch(flag, value);
}

// ---- upward sweep ------------------------------------------------------------------
// Front vector of the upward sweep: v = r on I (0 on B) plus the children's
// contributions, children added in a fixed order.  blockIdx.y splits the front's
// positions into disjoint ranges; a CTA scans every child's map and applies the entries
// that land in its range (a child's map is injective, so no two threads of a CTA touch
// the same position).
template <typename A, typename Ac>
__global__ void k_fwd_gather(const FrontDesc* __restrict__ fronts, const FrontDesc* __restrict__ kids,
                             const int* __restrict__ child_slots, const double* __restrict__ r) {
    const FrontDesc f = fronts[blockIdx.x];
    const int len = (f.N + gridDim.y - 1) / gridDim.y;
    const int p0 = blockIdx.y * len, p1 = min(f.N, p0 + len);
    A* v = (A*)f.vec;
    for (int p = p0 + threadIdx.x; p < p1; p += blockDim.x) v[p] = p < f.s ? (A)r[f.I[p]] : (A)0;
    if (blockIdx.y == 0 && threadIdx.x == 0) { f.flag[0] = 0; f.flag[1] = 0; }
    for (int ci = 0; ci < f.child_count; ++ci) {
        __syncthreads();
        const FrontDesc c = kids[child_slots[f.child_begin + ci]];
        const Ac* cv = (const Ac*)c.vec;
        for (int i = threadIdx.x; i < c.b; i += blockDim.x) {
            const int p = c.ea[i];
            if (p >= p0 && p < p1) v[p] += (A)cv[c.s + i];
        }
    }
}

// The same vector from the inverse maps (gptr, gsrc): one thread per front position sums
// r and its children's contributions in the children's order -- the sums of
// k_fwd_gather, term for term, without every CTA scanning every child's map.
template <typename A, typename Ac>
__global__ void k_fwd_gather_inv(const FrontDesc* __restrict__ fronts, const FrontDesc* __restrict__ kids,
                                 const int* __restrict__ child_slots, const double* __restrict__ r) {
    const FrontDesc f = fronts[blockIdx.x];
    A* v = (A*)f.vec;
    if (blockIdx.y == 0 && threadIdx.x == 0) { f.flag[0] = 0; f.flag[1] = 0; }
    for (int p = blockIdx.y * blockDim.x + threadIdx.x; p < f.N; p += gridDim.y * blockDim.x) {
        A acc = p < f.s ? (A)r[f.I[p]] : (A)0;
        const int k1 = f.gptr[p + 1];
        for (int k = f.gptr[p]; k < k1; ++k) {
            const int2 e = f.gsrc[k];
            const int slot = child_slots[f.child_begin + e.x];
            acc += (A)((const Ac*)kids[slot].vec)[kids[slot].s + e.y];
        }
        v[p] = acc;
    }
}

// Forward item: either a group of up to GD consecutive diagonal row blocks [b0, b0 + nb)
// of one front (item code = b0), or one NB-row block of its B rows.  The item first
// streams acc_row = sum_{cb < ncb} P[row, cb] y_cb over the finished column blocks (the
// factor tile of a column block is requested before waiting for that block's y); a B
// block then stores its contribution v_row - acc_row.  A diagonal group finishes its
// blocks inside the CTA -- t_g = v_g - acc_g - sum_{g' < g} P[g, g'] y_g', y_g = Dinv_g t_g
// -- publishing the front's progress counter after each block, so the dependency chain
// between CTAs waits on one item per GD blocks while the next item already consumes
// the group's first block.
template <typename T, typename A, int GD, bool H>
__global__ void __launch_bounds__(AT, GD == 1 ? 2 : 1) k_fwd_sweep(const FrontDesc* __restrict__ fronts,
                                                     const int* __restrict__ items, int n_items,
                                                     int* __restrict__ ticket, int* __restrict__ err,
                                                     long long wait) {
    using V = typename Vec<T>::V;
    using PT = typename PType<T, H>::type;
    constexpr int VW = Vec<T>::W;
    constexpr int PASSES = NB / (32 * VW);
    constexpr int RPW = NB / AW;                 // rows per warp and block
    __shared__ int s_item, s_flag;
    __shared__ __align__(16) A s_t[GD * NB];
    __shared__ __align__(16) A s_y[NB];
    __shared__ float s_ri[H ? GD * NB : 1];      // row factors of the item's rows (FP16 copy)
    extern __shared__ __align__(16) unsigned char sweep_smem[];
    T* Ds = (T*)sweep_smem;                      // GD inverted diagonal blocks
    PT* Ls = (PT*)(Ds + GD * NB * NB);           // P[block b0+1 rows, block b0 columns]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(ticket, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= n_items) return;
        const int slot = items[it] >> 16, blk = items[it] & 0xffff;
        const FrontDesc f = fronts[slot];
        const bool diag = blk < f.nd;
        const int nb = diag ? min(GD, f.nd - blk) : 1;
        const PT* P = (const PT*)(H ? f.P16 : f.P);
        A* v = (A*)f.vec;
        const int r0 = diag ? blk * NB : f.s + (blk - f.nd) * NB;
        const int r1 = diag ? min(r0 + nb * NB, f.s) : min(r0 + NB, f.N);
        if (diag) {
            prefetch_blocks(Ds, (const T*)f.Dinv + (int64_t)blk * NB * NB, nb);
            if (GD > 1 && nb > 1) prefetch_rows(Ls, P + (int64_t)(r0 + NB) * f.ldp + r0, f.ldp, r1 - r0 - NB);
            cp_async_commit();
        }
        for (int q = threadIdx.x; q < GD * NB; q += AT) s_t[q] = (r0 + q < r1) ? ld_cg(v + r0 + q) : (A)0;
        if constexpr (H) {
            for (int q = threadIdx.x; q < GD * NB; q += AT) s_ri[q] = (r0 + q < r1) ? f.ri[r0 + q] : 0.f;
        }
        const int ncb = diag ? blk : f.nd;
        A acc[GD][RPW];
#pragma unroll
        for (int g = 0; g < GD; ++g)
#pragma unroll
            for (int u = 0; u < RPW; ++u) acc[g][u] = 0;
        int seen = 0;
        if constexpr (H) {
            const int cend = min(ncb * NB, f.s);
            for (int cb = 0; cb < ncb; cb += 2) {
                const int c0 = cb * NB, cw = min(2 * NB, cend - c0), cl = lane * 8;
                uint4 l[GD][RPW];
#pragma unroll
                for (int g = 0; g < GD; ++g)
#pragma unroll
                    for (int u = 0; u < RPW; ++u) {
                        const int row = r0 + g * NB + warp + AW * u;
                        l[g][u] = (g < nb && row < r1 && cl < cw) ? __ldg((const uint4*)(P + (int64_t)row * f.ldp + c0 + cl))
                                                                  : make_uint4(0u, 0u, 0u, 0u);
                    }
                const int need = min(cb + 2, ncb);
                if (seen < need) seen = wait_flag(&f.flag[0], need, err, &s_flag, wait);
                float y[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) y[e] = (cl + e < cw) ? ld_cg(v + c0 + cl + e) : 0.f;
                const int valid = cw - cl;               // entries of this lane's eight inside the step
#pragma unroll
                for (int g = 0; g < GD; ++g)
#pragma unroll
                    for (int u = 0; u < RPW; ++u) {
                        float pv[8];
                        h8_to_f(l[g][u], pv);
#pragma unroll
                        for (int e = 0; e < 8; ++e) acc[g][u] += (e < valid ? pv[e] : 0.f) * y[e];
                    }
            }
        } else {
        for (int cb = 0; cb < ncb; ++cb) {
            const int c0 = cb * NB;
            const int cw = min(NB, f.s - c0);
#pragma unroll
            for (int ps = 0; ps < PASSES; ++ps) {
                const int cl = ps * 32 * VW + lane * VW;   // column inside the block
                V l[GD][RPW];
#pragma unroll
                for (int g = 0; g < GD; ++g)
#pragma unroll
                    for (int u = 0; u < RPW; ++u) {
                        const int row = r0 + g * NB + warp + AW * u;
                        l[g][u] = (g < nb && row < r1 && cl < cw) ? __ldg((const V*)(P + (int64_t)row * f.ldp + c0 + cl)) : V{};
                    }
                if (ps == 0 && seen < cb + 1) seen = wait_flag(&f.flag[0], cb + 1, err, &s_flag, wait);
                A y[VW];
#pragma unroll
                for (int e = 0; e < VW; ++e) y[e] = (cl + e < cw) ? ld_cg(v + c0 + cl + e) : (A)0;
#pragma unroll
                for (int g = 0; g < GD; ++g)
#pragma unroll
                    for (int u = 0; u < RPW; ++u)
#pragma unroll
                        for (int e = 0; e < VW; ++e) acc[g][u] += (A)vget(l[g][u], e) * y[e];
            }
        }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int g = 0; g < GD; ++g)
#pragma unroll
                for (int u = 0; u < RPW; ++u) acc[g][u] += __shfl_xor_sync(0xffffffffu, acc[g][u], o);
        __syncthreads();                             // s_t holds v on the item's rows
        if (lane == 0) {
#pragma unroll
            for (int g = 0; g < GD; ++g)
#pragma unroll
                for (int u = 0; u < RPW; ++u) {
                    const int q = g * NB + warp + AW * u;
                    if constexpr (H) {
                        if (r0 + q < r1) s_t[q] -= acc[g][u] * s_ri[q];
                    } else {
                        if (r0 + q < r1) s_t[q] -= acc[g][u];
                    }
                }
        }
        __syncthreads();
        if (!diag) {
            for (int q = threadIdx.x; q < r1 - r0; q += AT) __stcg(v + r0 + q, s_t[q]);
            __syncthreads();
            continue;
        }
        cp_async_wait();
        __syncthreads();
        for (int g = 0; g < nb; ++g) {
            const int w = min(NB, r1 - r0 - g * NB);
            A part[RPW];
            if (g > 0) {
                // t_g -= P[g rows, g-1 columns] y_{g-1}   (only g = 1: GD <= 2)
#pragma unroll
                for (int u = 0; u < RPW; ++u) part[u] = 0;
#pragma unroll
                for (int ps = 0; ps < PASSES; ++ps) {
                    const int cl = ps * 32 * VW + lane * VW;
                    A yv[VW];
#pragma unroll
                    for (int e = 0; e < VW; ++e) yv[e] = s_y[cl + e];
#pragma unroll
                    for (int u = 0; u < RPW; ++u) {
                        const V d = lds_v<T, H>(Ls + (warp + AW * u) * NB + cl);
#pragma unroll
                        for (int e = 0; e < VW; ++e) part[u] += (A)vget(d, e) * yv[e];
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                    for (int u = 0; u < RPW; ++u) part[u] += __shfl_xor_sync(0xffffffffu, part[u], o);
                if (lane == 0) {
#pragma unroll
                    for (int u = 0; u < RPW; ++u) {
                        const int rr = warp + AW * u;
                        if constexpr (H) {
                            if (rr < w) s_t[g * NB + rr] -= part[u] * s_ri[g * NB + rr];
                        } else {
                            if (rr < w) s_t[g * NB + rr] -= part[u];
                        }
                    }
                }
                __syncthreads();
            }
            // y_g = Dinv_g t_g: each thread takes RPW rows x VW columns per pass, then a warp sum
            const T* D = Ds + g * NB * NB;
#pragma unroll
            for (int u = 0; u < RPW; ++u) part[u] = 0;
#pragma unroll
            for (int ps = 0; ps < PASSES; ++ps) {
                const int cl = ps * 32 * VW + lane * VW;
                A t[VW];
#pragma unroll
                for (int e = 0; e < VW; ++e) t[e] = cl + e < w ? s_t[g * NB + cl + e] : (A)0;
#pragma unroll
                for (int u = 0; u < RPW; ++u) {
                    const V d = *(const V*)(D + (warp + AW * u) * NB + cl);
#pragma unroll
                    for (int e = 0; e < VW; ++e) part[u] += (A)vget(d, e) * t[e];
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                for (int u = 0; u < RPW; ++u) part[u] += __shfl_xor_sync(0xffffffffu, part[u], o);
            if (lane == 0) {
#pragma unroll
                for (int u = 0; u < RPW; ++u) {
                    const int rr = warp + AW * u;
                    if (rr < w) {
                        __stcg(v + r0 + g * NB + rr, part[u]);
                        s_y[rr] = part[u];
                    }
                }
            }
            // each block is published as soon as it is done, so the next item can take
            // this block's column while the second block of the pair is solved
            publish_flag(&f.flag[0], blk + g + 1, lane == 0);
        }
        __syncthreads();
    }
}

// ---- downward sweep ----------------------------------------------------------------
template <typename A>
__global__ void k_bwd_gather(const FrontDesc* __restrict__ fronts, const double* __restrict__ z) {
    const FrontDesc f = fronts[blockIdx.x];
    A* v = (A*)f.vec;
    for (int i = blockIdx.y * blockDim.x + threadIdx.x; i < f.b; i += gridDim.y * blockDim.x) v[f.s + i] = (A)z[f.Bd[i]];
}

// Backward item: a group of up to GD consecutive column blocks [lo, hi] (item code = hi,
// lo = hi - nb + 1), solved from the highest: t = y - sum over the rows below the group of
// P[rows, group columns]^T x_rows (ancestor rows first, then the interface row blocks
// above hi as their owners finish; each row group's factor rows are requested before
// waiting for its x); then inside the CTA x_hi = Dinv_hi^T t_hi,
// t_lo -= P[hi rows, lo columns]^T x_hi, x_lo = Dinv_lo^T t_lo, each block published
// as soon as it is done.
template <typename T, typename A, int GD, bool H>
__global__ void __launch_bounds__(AT, GD == 1 ? 2 : 1) k_bwd_sweep(const FrontDesc* __restrict__ fronts,
                                                     const int* __restrict__ items, int n_items,
                                                     int* __restrict__ ticket, int* __restrict__ err,
                                                     double* __restrict__ z, long long wait) {
    using V = typename Vec<T>::V;
    using PT = typename PType<T, H>::type;
    constexpr int VW = Vec<T>::W;
    constexpr int PASSES = NB / (32 * VW);
    constexpr int RB = 16 / PASSES;              // rows per warp per batch (a whole row block for FP32)
    __shared__ int s_item, s_flag;
    __shared__ A s_red[AW][GD * NB];
    __shared__ A s_t[GD * NB];
    __shared__ A s_x[NB];
    __shared__ float s_rih[H && GD > 1 ? NB : 1];   // row factors of block hi (FP16 copy)
    extern __shared__ __align__(16) unsigned char sweep_smem[];
    T* Ds = (T*)sweep_smem;                      // Dinv_hi, Dinv_lo
    PT* Ls = (PT*)(Ds + GD * NB * NB);           // P[hi rows, lo columns]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(ticket, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= n_items) return;
        const int slot = items[it] >> 16, hi = items[it] & 0xffff;
        const FrontDesc f = fronts[slot];
        const int nb = min(GD, hi + 1), lo = hi - nb + 1;
        const PT* P = (const PT*)(H ? f.P16 : f.P);
        A* v = (A*)f.vec;
        const int c0 = lo * NB, c1 = min((hi + 1) * NB, f.s), cw = c1 - c0;
        const int whi = min(NB, f.s - hi * NB);
        prefetch_blocks(Ds, (const T*)f.Dinv + (int64_t)hi * NB * NB, 1);
        if (GD > 1 && nb > 1) {
            prefetch_blocks(Ds + NB * NB, (const T*)f.Dinv + (int64_t)lo * NB * NB, 1);
            prefetch_rows(Ls, P + (int64_t)hi * NB * f.ldp + lo * NB, f.ldp, whi);
        }
        cp_async_commit();
        if constexpr (H && GD > 1) {
            for (int q = threadIdx.x; q < NB; q += AT) s_rih[q] = q < whi ? f.ri[hi * NB + q] : 0.f;
        }
        int seen = 0;
        const int n_groups_B = (f.b + NB - 1) / NB;
        const int n_groups = n_groups_B + (f.nd - 1 - hi);
        if constexpr (H) {
            // row groups HW at a time (consecutive groups are adjacent row ranges); for a
            // single block the two half-warps take alternate rows, 16 lanes x 8 entries each
            constexpr int HW = GD == 1 ? 2 : 1;
            const int sub = GD == 1 ? lane >> 4 : 0;
            const int cl = GD == 1 ? (lane & 15) * 8 : lane * 8;
            float acc8[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) acc8[e] = 0.f;
            for (int gr = 0; gr < n_groups; gr += HW) {
                int rlo = INT_MAX, rhi = 0, need = 0;
                for (int k = 0; k < HW && gr + k < n_groups; ++k) {
                    const int gk = gr + k;
                    int g0, g1;
                    if (gk < n_groups_B) {
                        g0 = f.s + (n_groups_B - 1 - gk) * NB; g1 = min(g0 + NB, f.N);
                    } else {
                        const int rb = f.nd - 1 - (gk - n_groups_B);
                        need = max(need, f.nd - rb);
                        g0 = rb * NB; g1 = min(g0 + NB, f.s);
                    }
                    rlo = min(rlo, g0);
                    rhi = max(rhi, g1);
                }
                uint4 l[RB];
                float rsc[RB];
#pragma unroll
                for (int u = 0; u < RB; ++u) {
                    const int row = rlo + (warp + AW * u) * HW + sub;
                    const bool in = row < rhi;
                    l[u] = (in && cl < cw) ? __ldg((const uint4*)(P + (int64_t)row * f.ldp + c0 + cl)) : make_uint4(0u, 0u, 0u, 0u);
                    rsc[u] = in ? f.ri[row] : 0.f;
                }
                if (seen < need) seen = wait_flag(&f.flag[1], need, err, &s_flag, wait);
#pragma unroll
                for (int u = 0; u < RB; ++u) {
                    const int row = rlo + (warp + AW * u) * HW + sub;
                    const float x = row < rhi ? ld_cg(v + row) * rsc[u] : 0.f;
                    float pv[8];
                    h8_to_f(l[u], pv);
#pragma unroll
                    for (int e = 0; e < 8; ++e) acc8[e] += pv[e] * x;
                }
            }
            if (GD == 1) {
#pragma unroll
                for (int e = 0; e < 8; ++e) acc8[e] += __shfl_xor_sync(0xffffffffu, acc8[e], 16);
            }
            if (GD > 1 || lane < 16) {
#pragma unroll
                for (int e = 0; e < 8; ++e) s_red[warp][cl + e] = acc8[e];
            }
        } else {
        A acc[GD][PASSES][VW];
#pragma unroll
        for (int g = 0; g < GD; ++g)
#pragma unroll
            for (int ps = 0; ps < PASSES; ++ps)
#pragma unroll
                for (int e = 0; e < VW; ++e) acc[g][ps][e] = 0;
        for (int gr = 0; gr < n_groups; ++gr) {
            int g0, g1, need = 0;
            if (gr < n_groups_B) {
                g0 = f.s + (n_groups_B - 1 - gr) * NB; g1 = min(g0 + NB, f.N);
            } else {
                const int rb = f.nd - 1 - (gr - n_groups_B);     // I row block > hi
                need = f.nd - rb;                                  // blocks finished from the top
                g0 = rb * NB; g1 = min(g0 + NB, f.s);
            }
            for (int base = g0; base < g1; base += AW * RB) {
                V l[RB][GD][PASSES];
#pragma unroll
                for (int u = 0; u < RB; ++u) {
                    const int row = base + warp + AW * u;
#pragma unroll
                    for (int g = 0; g < GD; ++g)
#pragma unroll
                        for (int ps = 0; ps < PASSES; ++ps) {
                            const int cl = g * NB + ps * 32 * VW + lane * VW;
                            l[u][g][ps] = (row < g1 && cl < cw) ? __ldg((const V*)(P + (int64_t)row * f.ldp + c0 + cl)) : V{};
                        }
                }
                if (base == g0 && seen < need) seen = wait_flag(&f.flag[1], need, err, &s_flag, wait);
                A x[RB];
#pragma unroll
                for (int u = 0; u < RB; ++u) {
                    const int row = base + warp + AW * u;
                    x[u] = row < g1 ? ld_cg(v + row) : (A)0;
                }
#pragma unroll
                for (int u = 0; u < RB; ++u)
#pragma unroll
                    for (int g = 0; g < GD; ++g)
#pragma unroll
                        for (int ps = 0; ps < PASSES; ++ps)
#pragma unroll
                            for (int e = 0; e < VW; ++e) acc[g][ps][e] += (A)vget(l[u][g][ps], e) * x[u];
            }
        }
#pragma unroll
        for (int g = 0; g < GD; ++g)
#pragma unroll
            for (int ps = 0; ps < PASSES; ++ps)
#pragma unroll
                for (int e = 0; e < VW; ++e) s_red[warp][g * NB + ps * 32 * VW + lane * VW + e] = acc[g][ps][e];
        }
        __syncthreads();
        for (int c = threadIdx.x; c < GD * NB; c += AT) {
            A sum = 0;
#pragma unroll
            for (int w = 0; w < AW; ++w) sum += s_red[w][c];
            s_t[c] = c < cw ? ld_cg(v + c0 + c) - sum : (A)0;
        }
        cp_async_wait();
        __syncthreads();
        // blocks from the highest: x_g = Dinv_g^T t_g (lanes over columns, warps over rows)
        for (int k = 0; k < nb; ++k) {
            const int g = nb - 1 - k;                    // position of the block inside the group
            const int w = min(NB, cw - g * NB);
            const T* D = Ds + k * NB * NB;               // Dinv_hi first, then Dinv_lo
            if (k > 0) {
                // t_lo -= P[hi rows, lo columns]^T x_hi
                A part[PASSES][VW];
#pragma unroll
                for (int ps = 0; ps < PASSES; ++ps)
#pragma unroll
                    for (int e = 0; e < VW; ++e) part[ps][e] = 0;
                for (int rr = warp; rr < whi; rr += AW) {
                    A xr = s_x[rr];
                    if constexpr (H) xr *= s_rih[rr];
#pragma unroll
                    for (int ps = 0; ps < PASSES; ++ps) {
                        const V d = lds_v<T, H>(Ls + rr * NB + ps * 32 * VW + lane * VW);
#pragma unroll
                        for (int e = 0; e < VW; ++e) part[ps][e] += (A)vget(d, e) * xr;
                    }
                }
#pragma unroll
                for (int ps = 0; ps < PASSES; ++ps)
#pragma unroll
                    for (int e = 0; e < VW; ++e) s_red[warp][ps * 32 * VW + lane * VW + e] = part[ps][e];
                __syncthreads();
                for (int c = threadIdx.x; c < w; c += AT) {
                    A sum = 0;
#pragma unroll
                    for (int q = 0; q < AW; ++q) sum += s_red[q][c];
                    s_t[g * NB + c] -= sum;
                }
                __syncthreads();
            }
            {
                A part[PASSES][VW];
#pragma unroll
                for (int ps = 0; ps < PASSES; ++ps)
#pragma unroll
                    for (int e = 0; e < VW; ++e) part[ps][e] = 0;
                for (int rr = warp; rr < w; rr += AW) {
                    const A tr = s_t[g * NB + rr];
#pragma unroll
                    for (int ps = 0; ps < PASSES; ++ps) {
                        const V d = *(const V*)(D + rr * NB + ps * 32 * VW + lane * VW);
#pragma unroll
                        for (int e = 0; e < VW; ++e) part[ps][e] += (A)vget(d, e) * tr;
                    }
                }
#pragma unroll
                for (int ps = 0; ps < PASSES; ++ps)
#pragma unroll
                    for (int e = 0; e < VW; ++e) s_red[warp][ps * 32 * VW + lane * VW + e] = part[ps][e];
            }
            __syncthreads();
            for (int c = threadIdx.x; c < w; c += AT) {
                A sum = 0;
#pragma unroll
                for (int q = 0; q < AW; ++q) sum += s_red[q][c];
                __stcg(v + c0 + g * NB + c, sum);
                z[f.I[c0 + g * NB + c]] = (double)sum;
                s_x[c] = sum;
            }
            publish_flag(&f.flag[1], f.nd - hi + k, true);   // blocks >= hi - k are done
        }
        __syncthreads();
    }
}

// ---- cluster sweeps (levels of fronts without B rows, FP16 factor copy) ---------------
// A front with many diagonal blocks (the root) makes the sweeps chain-bound: every block
// waits for the previous one through global memory (the producer's fence, the flag poll,
// the vector reread), several microseconds per block.  Here a cluster of SWEEP_CL CTAs
// takes SWEEP_CL consecutive diagonal blocks, one each.  A CTA streams its own row block
// (forward) or column block (backward) over the blocks of earlier clusters as the
// per-CTA kernels do, waiting on the front's progress counter; the chain inside the
// cluster then runs through distributed shared memory: a CTA stores its finished block
// into the shared memory of each later CTA of the cluster and raises a per-sender counter
// there with a cluster-scope release; a CTA waits on its own counters (bounded, like every
// wait here) and reads the blocks locally.  The block, and the front's vector
// right-hand side it needs, are in shared memory before the chain reaches the CTA, so a
// hand-off costs a few hundred nanoseconds.  One hand-off in SWEEP_CL goes through global
// memory: every block still raises the front's progress counter, in block order (after
// its push and a fence), which the later clusters wait on.  Work items are taken with a ticket by the cluster's first CTA,
// so a cluster only waits on items with smaller tickets, held by running clusters.

__device__ __forceinline__ void cl_st_remote(uint32_t a, float v) {
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}

__device__ __forceinline__ void cl_st_release_remote(uint32_t a, int v) {
    asm volatile("st.release.cluster.shared::cluster.b32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

__device__ __forceinline__ int cl_ld_acquire_local(const int* p) {
    int v;
    asm volatile("ld.acquire.cluster.shared::cta.b32 %0, [%1];" : "=r"(v) : "r"((uint32_t)__cvta_generic_to_shared(p)) : "memory");
    return v;
}

// A finished block goes to the later CTAs of the cluster: the thread holding entry `row`
// (mine) stores it into in[rank][row] of each CTA rank + 1 .. last - 1 (distributed shared
// memory), the next CTA first; after the barrier thread q raises got[rank] = ep in CTA
// rank + 1 + q with a cluster-scope release, which orders the whole CTA's stores before
// it (one thread per receiver, so no receiver waits for another's flag).
__device__ void cl_push(float val, int row, bool mine, float (*in)[NB], int* got, uint32_t rank, int last, int ep) {
    if (mine)
        for (int m = (int)rank + 1; m < last; ++m) cl_st_remote(cl_map(&in[rank][row], (uint32_t)m), val);
    __syncthreads();
    const int m = (int)rank + 1 + (int)threadIdx.x;
    if (m < last) cl_st_release_remote(cl_map(&got[rank], (uint32_t)m), ep);
}

// Wait (bounded) until CTA `peer` has pushed its block of epoch `ep` into in[peer].
__device__ void cl_wait_in(const int* got, uint32_t peer, int ep, int* err, long long limit) {
    if (threadIdx.x == 0 && cl_ld_acquire_local(&got[peer]) < ep) {
        const long long t0 = clock64();
        while (cl_ld_acquire_local(&got[peer]) < ep) {
            if (ld_volatile(&err[ERR_TIMEOUT]) || clock64() - t0 > limit) {
                atomicExch(&err[ERR_TIMEOUT], 1);
                break;
            }
        }
    }
    __syncthreads();
}

// Raise a front's progress counter from `from` to `to` once it holds `from`: the blocks
// publish in order, so a counter value covers every block below it (each block's stores
// are fenced before its own step; a later block of the cluster can be done first, having
// received its predecessor through shared memory).  Thread 0; bounded like every wait.
__device__ void cl_publish_in_order(int* flag, int from, int to, int* err, long long limit) {
    if (threadIdx.x != 0) return;
    if (atomicCAS(flag, from, to) == from) return;
    const long long t0 = clock64();
    for (;;) {
        if (ld_volatile(flag) == from && atomicCAS(flag, from, to) == from) return;
        if (ld_volatile(&err[ERR_TIMEOUT]) || clock64() - t0 > limit) {
            atomicExch(&err[ERR_TIMEOUT], 1);
            atomicMax(flag, to);
            return;
        }
        __nanosleep(32);
    }
}

// The item of the cluster: the first CTA's ticket, read by every CTA (two cluster
// barriers: the ticket is in place, then read everywhere before it changes).
__device__ int cl_ticket(int* s_item, int* s_it, int* ticket, uint32_t rank) {
    if (rank == 0 && threadIdx.x == 0) *s_item = atomicAdd(ticket, 1);
    cl_sync();
    if (threadIdx.x == 0) *s_it = cl_ld(cl_map(s_item, 0));
    cl_sync();
    return *s_it;
}

// The factor tiles a CTA streams (NB x NB FP16, row-major) pass through a ring of
// CL_RING shared-memory stages filled with cp.async CL_RING - 1 steps ahead; a step's
// consumer reads them with lanes over four columns and warps over 16 rows.  A stage also
// carries the step's vector block (and its row factors, backward) when that block was
// already published when the stage was filled, which it is for all but the last blocks.
constexpr int CL_RING = 6;
constexpr int CL_STAGE = NB * NB * 2 + 2 * NB * 4;    // tile, then two NB-float vectors
constexpr int CL_SMEM = CL_RING * CL_STAGE;

__device__ __forceinline__ void cp16(uint32_t dst, const void* src, bool in) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(in ? 16 : 0) : "memory");
}

// Tile rows [row0, row0 + NB) (those below row_end), columns [col0, col0 + NB) (those
// starting below col_end) of the FP16 copy into a ring stage; the rest is zero-filled.
// With nv > 0 the stage's vectors receive a[e0 .. e0 + NB) (and b[..], nv = 2); callers
// pass whole blocks only (e0 + NB <= e_end).
__device__ __forceinline__ void cl_issue_tile(unsigned char* stage, const FrontDesc& f, int row0, int row_end, int col0, int col_end,
                                              int nv, const float* a, const float* b, int e0, int e_end) {
    const uint32_t d0 = (uint32_t)__cvta_generic_to_shared(stage);
    const __half* P = (const __half*)f.P16;
    for (int c = threadIdx.x; c < NB * 16; c += AT) {
        const int row = c >> 4, q = c & 15;
        const bool in = row0 + row < row_end && col0 + 8 * q < col_end;
        cp16(d0 + (uint32_t)(row * NB + 8 * q) * 2, in ? (const void*)(P + (int64_t)(row0 + row) * f.ldp + col0 + 8 * q) : (const void*)P, in);
    }
    // a (a front vector: 16-byte aligned, as is e0) in 16-byte chunks; b (row factors,
    // which start N floats into their region, so only 4-byte aligned) entry by entry
    if (nv >= 1 && (int)threadIdx.x < NB / 4)
        cp16(d0 + (uint32_t)(NB * NB * 2 + 16 * threadIdx.x), a + e0 + 4 * threadIdx.x, true);
    if (nv >= 2 && (int)threadIdx.x < NB)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d0 + (uint32_t)(NB * NB * 2 + NB * 4 + 4 * threadIdx.x)),
                     "l"(b + e0 + threadIdx.x) : "memory");
}

// Forward: CTA `rank` solves diagonal block blk = g0 + rank of the item's front: steps
// 0 .. blk-1 take the column blocks in order (those of earlier clusters after the front's
// progress counter, those of this cluster from the earlier CTAs' shared memory); a lane
// keeps partial sums of its warp's 16 rows over its four columns, reduced once:
// acc_r = sum_c P16[r, c] y_c, t_r = v_r - ri_r acc_r, y = Dinv t (two threads per row).
__global__ void __cluster_dims__(SWEEP_CL, 1, 1) __launch_bounds__(AT, 1)
k_fwd_sweep_cl(const FrontDesc* __restrict__ fronts, const int* __restrict__ items, int n_items,
               int* __restrict__ ticket, int* __restrict__ err, long long wait) {
    __shared__ int s_item, s_it, s_flag;
    __shared__ int s_got[SWEEP_CL];                  // epoch of the block pushed by each earlier CTA
    __shared__ __align__(16) float s_in[SWEEP_CL][NB];   // the blocks pushed by the earlier CTAs
    __shared__ __align__(16) float s_t[NB];
    __shared__ float s_v[NB], s_ri[NB];              // the block's v and row factors, read early
    extern __shared__ __align__(16) unsigned char cl_smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t rank = cl_rank();
    if (tid < SWEEP_CL) s_got[tid] = 0;
    if (tid == 0) s_item = 0;
    int ep = 0;
    for (;;) {
        const int it = cl_ticket(&s_item, &s_it, ticket, rank);
        ++ep;
        if (it >= n_items) return;
        const int slot = items[it] >> 16, g0 = items[it] & 0xffff;
        const FrontDesc f = fronts[slot];
        const int blk = g0 + (int)rank;
        if (blk >= f.nd) continue;
        const int r0 = blk * NB, w = min(NB, f.s - r0), rend = r0 + w;
        float* v = (float*)f.vec;
        const int r = tid >> 1, hf = tid & 1;
        float4 dv[16];                                // Dinv_blk[r, 64 hf .. 64 hf + 63]
        {
            const float4* D = reinterpret_cast<const float4*>((const float*)f.Dinv + (int64_t)blk * NB * NB + r * NB + hf * 64);
#pragma unroll
            for (int k = 0; k < 16; ++k) dv[k] = __ldg(D + k);
        }
        if (tid < NB) {                               // off the chain: loaded while the steps run
            s_v[tid] = tid < w ? __ldcg(v + r0 + tid) : 0.f;
            s_ri[tid] = tid < w ? f.ri[r0 + tid] : 0.f;
        }
        const int nsteps = blk;                       // column blocks 0 .. blk - 1
        int seen = 0;
        unsigned ymask = 0;                           // bit k: stage k holds its step's y block
        auto issue = [&](int q) {
            const int k = q % CL_RING;
            const bool yin = q < g0 && seen >= q + 1;     // (blocks before g0 are whole)
            cl_issue_tile(cl_smem + k * CL_STAGE, f, r0, rend, q * NB, f.s, yin ? 1 : 0, v, v, q * NB, f.s);
            ymask = yin ? (ymask | (1u << k)) : (ymask & ~(1u << k));
        };
#pragma unroll
        for (int q = 0; q < CL_RING - 1; ++q) {
            if (q < nsteps) issue(q);
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
        float acc[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) acc[u] = 0.f;
        for (int i = 0; i < nsteps; ++i) {
            asm volatile("cp.async.wait_group %0;" ::"n"(CL_RING - 2) : "memory");
            const unsigned char* stg = cl_smem + (i % CL_RING) * CL_STAGE;
            float4 y;
            if (i < g0) {
                const bool yin = (ymask >> (i % CL_RING)) & 1u;
                if (!yin && seen < i + 1) seen = wait_flag(&f.flag[0], i + 1, err, &s_flag, wait);
                __syncthreads();                      // the stage of step i is in place
                y = yin ? reinterpret_cast<const float4*>(stg + NB * NB * 2)[lane]
                        : __ldcg(reinterpret_cast<const float4*>(v + i * NB) + lane);
            } else {
                cl_wait_in(s_got, (uint32_t)(i - g0), ep, err, wait);
                y = reinterpret_cast<const float4*>(s_in[i - g0])[lane];
            }
            const int q = i + CL_RING - 1;            // refill the stage freed by step i - 1
            if (q < nsteps) issue(q);
            asm volatile("cp.async.commit_group;" ::: "memory");
            const __half* st = reinterpret_cast<const __half*>(stg) + (warp * 16) * NB + lane * 4;
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const uint2 pq = *reinterpret_cast<const uint2*>(st + u * NB);
                acc[u] = fmaf(h_lo(pq.x), y.x, acc[u]);
                acc[u] = fmaf(h_hi(pq.x), y.y, acc[u]);
                acc[u] = fmaf(h_lo(pq.y), y.z, acc[u]);
                acc[u] = fmaf(h_hi(pq.y), y.w, acc[u]);
            }
        }
        asm volatile("cp.async.wait_group 0;" ::: "memory");
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int u = 0; u < 16; ++u) acc[u] += __shfl_xor_sync(0xffffffffu, acc[u], o);
        __syncthreads();                              // s_v and s_ri (written at the item's start) are in place
        {
            float mine = acc[0];                      // lane u < 16 takes row 16 warp + u
#pragma unroll
            for (int u = 1; u < 16; ++u) mine = lane == u ? acc[u] : mine;
            const int rr = warp * 16 + lane;
            if (lane < 16) s_t[rr] = rr < w ? s_v[rr] - mine * s_ri[rr] : 0.f;
        }
        __syncthreads();
        float yq[4] = {0.f, 0.f, 0.f, 0.f};
        {
            const float4* t4 = reinterpret_cast<const float4*>(s_t + hf * 64);
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const float4 t = t4[k];
                yq[0] = fmaf(dv[k].x, t.x, yq[0]); yq[1] = fmaf(dv[k].y, t.y, yq[1]);
                yq[2] = fmaf(dv[k].z, t.z, yq[2]); yq[3] = fmaf(dv[k].w, t.w, yq[3]);
            }
        }
        float yr = (yq[0] + yq[1]) + (yq[2] + yq[3]);
        yr += __shfl_xor_sync(0xffffffffu, yr, 1);
        const bool rin = r < w;
        // the later CTAs of the cluster first, then the later clusters
        cl_push(rin ? yr : 0.f, r, hf == 0, s_in, s_got, rank, min(SWEEP_CL, f.nd - g0), ep);
        if (hf == 0 && rin) {
            __stcg(v + r0 + r, yr);
            __threadfence();
        }
        __syncthreads();
        cl_publish_in_order(&f.flag[0], blk, blk + 1, err, wait);
    }
}

// Backward: CTA `rank` solves column block cbk = hi - rank (the item's code is hi, the
// highest block): steps take the row blocks below it from the last up (those of earlier
// clusters after the front's progress counter, those of this cluster from the CTAs above
// in the cluster); lanes over four columns, warps over 16 rows:
// acc_c = sum_rows P16[row, c] (ri_row x_row), t = v - acc, x = Dinv^T t.  A CTA leaves
// ri_row x_row of its block for the CTAs below it in the cluster.
__global__ void __cluster_dims__(SWEEP_CL, 1, 1) __launch_bounds__(AT, 1)
k_bwd_sweep_cl(const FrontDesc* __restrict__ fronts, const int* __restrict__ items, int n_items,
               int* __restrict__ ticket, int* __restrict__ err, double* __restrict__ z, long long wait) {
    __shared__ int s_item, s_it, s_flag;
    __shared__ int s_got[SWEEP_CL];                  // epoch of the block pushed by each earlier CTA
    __shared__ __align__(16) float s_in[SWEEP_CL][NB];   // ri x of the blocks pushed by the earlier CTAs
    __shared__ __align__(16) float s_c[2][NB];       // ri x of the step's row block
    __shared__ __align__(16) float s_t[NB];
    __shared__ __align__(16) float s_red[AW][NB];
    __shared__ float s_v[NB], s_ri[NB];              // the block's v and row factors, read early
    extern __shared__ __align__(16) unsigned char cl_smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int c4 = lane * 4;                          // this thread's four columns of the block
    const uint32_t rank = cl_rank();
    if (tid < SWEEP_CL) s_got[tid] = 0;
    if (tid == 0) s_item = 0;
    int ep = 0;
    for (;;) {
        const int it = cl_ticket(&s_item, &s_it, ticket, rank);
        ++ep;
        if (it >= n_items) return;
        const int slot = items[it] >> 16, hi = items[it] & 0xffff;
        const FrontDesc f = fronts[slot];
        const int cbk = hi - (int)rank;
        if (cbk < 0) continue;
        const int c0 = cbk * NB, wc = min(NB, f.s - c0);
        float* v = (float*)f.vec;
        float4 dv[16];                                // Dinv_cbk[16 warp + u, c4 .. c4 + 3]
        {
            const float* D = (const float*)f.Dinv + (int64_t)cbk * NB * NB + (warp * 16) * NB + c4;
#pragma unroll
            for (int u = 0; u < 16; ++u) dv[u] = __ldg(reinterpret_cast<const float4*>(D + u * NB));
        }
        if (tid < NB) {                               // off the chain: loaded while the steps run
            s_v[tid] = tid < wc ? __ldcg(v + c0 + tid) : 0.f;
            s_ri[tid] = tid < wc ? f.ri[c0 + tid] : 0.f;
        }
        // step i takes row block rb(i): the earlier clusters' blocks nd-1 .. hi+1, then hi .. cbk+1
        const int nsteps = f.nd - 1 - cbk, n_glob = f.nd - 1 - hi;
        auto rb_of = [&](int i) { return f.nd - 1 - i; };
        int seen = 0;
        unsigned xmask = 0;                           // bit k: stage k holds its step's x and ri
        auto issue = [&](int q) {
            const int k = q % CL_RING, rb = rb_of(q);
            const bool xin = q < n_glob && seen >= f.nd - rb && (rb + 1) * NB <= f.s;   // whole blocks only
            cl_issue_tile(cl_smem + k * CL_STAGE, f, rb * NB, f.s, c0, f.s, xin ? 2 : 0, v, f.ri, rb * NB, f.s);
            xmask = xin ? (xmask | (1u << k)) : (xmask & ~(1u << k));
        };
#pragma unroll
        for (int q = 0; q < CL_RING - 1; ++q) {
            if (q < nsteps) issue(q);
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int i = 0; i < nsteps; ++i) {
            asm volatile("cp.async.wait_group %0;" ::"n"(CL_RING - 2) : "memory");
            const int rb = rb_of(i);
            const unsigned char* stg = cl_smem + (i % CL_RING) * CL_STAGE;
            const float* xs;                          // the step's x (ri applied when sc is null)
            const float* sc = nullptr;
            if (i < n_glob) {
                const bool xin = (xmask >> (i % CL_RING)) & 1u;
                if (xin) {
                    xs = reinterpret_cast<const float*>(stg + NB * NB * 2);
                    sc = xs + NB;
                } else {
                    const int need = f.nd - rb;
                    if (seen < need) seen = wait_flag(&f.flag[1], need, err, &s_flag, wait);
                    if (tid < NB) {
                        const int row = rb * NB + tid;
                        s_c[i & 1][tid] = row < f.s ? __ldcg(v + row) * f.ri[row] : 0.f;
                    }
                    xs = s_c[i & 1];
                }
                __syncthreads();                      // the stage and the x of step i are in place
            } else {
                cl_wait_in(s_got, (uint32_t)(i - n_glob), ep, err, wait);
                xs = s_in[i - n_glob];
            }
            const int q = i + CL_RING - 1;
            if (q < nsteps) issue(q);
            asm volatile("cp.async.commit_group;" ::: "memory");
            const __half* st = reinterpret_cast<const __half*>(stg) + (warp * 16) * NB + c4;
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const uint2 pq = *reinterpret_cast<const uint2*>(st + u * NB);
                const float x = sc ? xs[warp * 16 + u] * sc[warp * 16 + u] : xs[warp * 16 + u];
                acc[0] = fmaf(h_lo(pq.x), x, acc[0]); acc[1] = fmaf(h_hi(pq.x), x, acc[1]);
                acc[2] = fmaf(h_lo(pq.y), x, acc[2]); acc[3] = fmaf(h_hi(pq.y), x, acc[3]);
            }
        }
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        *reinterpret_cast<float4*>(&s_red[warp][c4]) = make_float4(acc[0], acc[1], acc[2], acc[3]);
        __syncthreads();
        if (tid < NB) {
            float sum = 0.f;
#pragma unroll
            for (int q = 0; q < AW; ++q) sum += s_red[q][tid];
            s_t[tid] = tid < wc ? s_v[tid] - sum : 0.f;
        }
        __syncthreads();
        float xp[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const float t = s_t[warp * 16 + u];
            xp[0] = fmaf(dv[u].x, t, xp[0]); xp[1] = fmaf(dv[u].y, t, xp[1]);
            xp[2] = fmaf(dv[u].z, t, xp[2]); xp[3] = fmaf(dv[u].w, t, xp[3]);
        }
        *reinterpret_cast<float4*>(&s_red[warp][c4]) = make_float4(xp[0], xp[1], xp[2], xp[3]);
        __syncthreads();
        float x = 0.f;
        if (tid < NB) {
#pragma unroll
            for (int q = 0; q < AW; ++q) x += s_red[q][tid];
        }
        // the later CTAs of the cluster first, then the later clusters
        cl_push(tid < wc ? x * s_ri[tid] : 0.f, tid, tid < NB, s_in, s_got, rank, min(SWEEP_CL, hi + 1), ep);
        if (tid < wc) {
            __stcg(v + c0 + tid, x);
            z[f.I[c0 + tid]] = (double)x;
            __threadfence();
        }
        __syncthreads();
        cl_publish_in_order(&f.flag[1], f.nd - 1 - cbk, f.nd - cbk, err, wait);
    }
}


// Dynamic shared memory of the sweep kernels: GD inverted diagonal blocks plus, for
// GD = 2, one factor block (FP16 when read from the copy).
template <typename T, int GD, bool H> constexpr int sweep_dsm() {
    return GD * NB * NB * (int)sizeof(T) + (GD > 1 ? NB * NB * (int)sizeof(typename PType<T, H>::type) : 0);
}

template <typename T, typename A, int GD, bool H>
int sweep_attr() {
    RSD_CUDA_TRY(cudaFuncSetAttribute(k_fwd_sweep<T, A, GD, H>, cudaFuncAttributeMaxDynamicSharedMemorySize, sweep_dsm<T, GD, H>()));
    RSD_CUDA_TRY(cudaFuncSetAttribute(k_bwd_sweep<T, A, GD, H>, cudaFuncAttributeMaxDynamicSharedMemorySize, sweep_dsm<T, GD, H>()));
    return RSD_OK;
}

template <typename T, typename A>
int sweep_smem_setup() {
    static bool done = false;
    if (!done) {
        RSD_TRY((sweep_attr<T, A, 1, false>()));
        if constexpr (sizeof(T) == 4) {
            RSD_TRY((sweep_attr<T, A, 2, false>()));
            RSD_TRY((sweep_attr<T, A, 1, true>()));
            RSD_TRY((sweep_attr<T, A, 2, true>()));
        }
        done = true;
    }
    return RSD_OK;
}

// Launch the upward / downward sweep kernel with the level's group size, reading the
// FP16 factor copy when the level has one.
template <typename T, typename A>
void launch_fwd(int gd, bool h16, int grid, cudaStream_t st, const FrontDesc* fr, const int* items, int n, int* tk,
                int* err, long long wait) {
    if constexpr (sizeof(T) == 4) {
        if (h16 && gd == 2) { k_fwd_sweep<T, A, 2, true><<<grid, AT, sweep_dsm<T, 2, true>(), st>>>(fr, items, n, tk, err, wait); return; }
        if (h16) { k_fwd_sweep<T, A, 1, true><<<grid, AT, sweep_dsm<T, 1, true>(), st>>>(fr, items, n, tk, err, wait); return; }
        if (gd == 2) { k_fwd_sweep<T, A, 2, false><<<grid, AT, sweep_dsm<T, 2, false>(), st>>>(fr, items, n, tk, err, wait); return; }
    }
    k_fwd_sweep<T, A, 1, false><<<grid, AT, sweep_dsm<T, 1, false>(), st>>>(fr, items, n, tk, err, wait);
}

template <typename T, typename A>
void launch_bwd(int gd, bool h16, int grid, cudaStream_t st, const FrontDesc* fr, const int* items, int n, int* tk,
                int* err, double* z, long long wait) {
    if constexpr (sizeof(T) == 4) {
        if (h16 && gd == 2) { k_bwd_sweep<T, A, 2, true><<<grid, AT, sweep_dsm<T, 2, true>(), st>>>(fr, items, n, tk, err, z, wait); return; }
        if (h16) { k_bwd_sweep<T, A, 1, true><<<grid, AT, sweep_dsm<T, 1, true>(), st>>>(fr, items, n, tk, err, z, wait); return; }
        if (gd == 2) { k_bwd_sweep<T, A, 2, false><<<grid, AT, sweep_dsm<T, 2, false>(), st>>>(fr, items, n, tk, err, z, wait); return; }
    }
    k_bwd_sweep<T, A, 1, false><<<grid, AT, sweep_dsm<T, 1, false>(), st>>>(fr, items, n, tk, err, z, wait);
}

// Clusters of the cluster sweeps resident at once on the current device (the persistent
// grid), looked up once per device.
int cl_grid(int n_items, int* out) {
    static int max_cl[64] = {};
    int dev = 0;
    RSD_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return RSD_ERR_ARG;
    if (!max_cl[dev]) {
        RSD_CUDA_TRY(cudaFuncSetAttribute(k_fwd_sweep_cl, cudaFuncAttributeMaxDynamicSharedMemorySize, CL_SMEM));
        RSD_CUDA_TRY(cudaFuncSetAttribute(k_bwd_sweep_cl, cudaFuncAttributeMaxDynamicSharedMemorySize, CL_SMEM));
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(SWEEP_CL * 64);
        cfg.blockDim = dim3(AT);
        cfg.dynamicSmemBytes = CL_SMEM;
        int n1 = 0, n2 = 0;
        RSD_CUDA_TRY(cudaOccupancyMaxActiveClusters(&n1, (void*)k_fwd_sweep_cl, &cfg));
        RSD_CUDA_TRY(cudaOccupancyMaxActiveClusters(&n2, (void*)k_bwd_sweep_cl, &cfg));
        max_cl[dev] = std::max(1, std::min(n1, n2));
    }
    *out = std::max(1, std::min(n_items, max_cl[dev]));
    return RSD_OK;
}

// Upward / downward sweep kernel of a level: the cluster kernels on a cl_sweep level,
// else the per-CTA kernels with the level's group size.
template <typename T, typename A>
int launch_fwd_level(const Level& L, int grid, cudaStream_t st, const FrontDesc* fr, const int* items, int n, int* tk,
                     int* err, long long wait) {
    if constexpr (sizeof(T) == 4) {
        if (L.cl_sweep) {
            int ncl = 0;
            RSD_TRY(cl_grid(n, &ncl));
            k_fwd_sweep_cl<<<ncl * SWEEP_CL, AT, CL_SMEM, st>>>(fr, items, n, tk, err, wait);
            return RSD_OK;
        }
    }
    launch_fwd<T, A>(sweep_group(L), L.h16, grid, st, fr, items, n, tk, err, wait);
    return RSD_OK;
}

template <typename T, typename A>
int launch_bwd_level(const Level& L, int grid, cudaStream_t st, const FrontDesc* fr, const int* items, int n, int* tk,
                     int* err, double* z, long long wait) {
    if constexpr (sizeof(T) == 4) {
        if (L.cl_sweep) {
            int ncl = 0;
            RSD_TRY(cl_grid(n, &ncl));
            k_bwd_sweep_cl<<<ncl * SWEEP_CL, AT, CL_SMEM, st>>>(fr, items, n, tk, err, z, wait);
            return RSD_OK;
        }
    }
    launch_bwd<T, A>(sweep_group(L), L.h16, grid, st, fr, items, n, tk, err, z, wait);
    return RSD_OK;
}

template <typename T, typename A>
int sweep_level(Handle& h, int li, bool forward, const double* r, double* z, int tk) {
    RSD_TRY((sweep_smem_setup<T, A>()));
    Level& L = h.levels[li];
    const int nf = (int)L.fronts.size();
    double gbytes = 0;
    for (auto& f : L.fronts) gbytes += (double)f.N * (sizeof(A) + 8.0);
    const double fbytes = level_factor_bytes(L, true);
    const int grid = std::max(1, std::min(forward ? L.n_fwd_items : L.n_bwd_items, h.num_sms * 4));
    if (forward) {
        const int gi = prof_begin(h, K_GATHER);
        // split each front into ranges of ~2048 positions when there are few fronts
        const dim3 gg((unsigned)nf, (unsigned)std::max(1, std::min((L.max_N + 255) / 256, (4 * h.num_sms + nf - 1) / nf)));
        if (li + 1 < (int)h.levels.size()) {
            const Level& Lc = h.levels[li + 1];
            if (is_fp64(Lc.prec)) k_fwd_gather_inv<A, double><<<gg, 256, 0, h.stream>>>(L.d_fronts, Lc.d_fronts, L.d_child_slots, r);
            else k_fwd_gather_inv<A, float><<<gg, 256, 0, h.stream>>>(L.d_fronts, Lc.d_fronts, L.d_child_slots, r);
        } else {
            k_fwd_gather_inv<A, A><<<gg, 256, 0, h.stream>>>(L.d_fronts, L.d_fronts, L.d_child_slots, r);
        }
        count_launch();
        prof_end(h, gi, 0.0, gbytes);
        RSD_CUDA_TRY(cudaGetLastError());
        if (L.n_fwd_items) {
            // fault injection: drop the first item (front slot 0's first diagonal block)
            const int drop = h.inject_drop_level == li && L.n_fwd_items > 1 ? 1 : 0;
            if (drop) h.inject_drop_level = -1;
            const int pi = prof_begin(h, K_FWD);
            RSD_TRY((launch_fwd_level<T, A>(L, grid, h.stream, L.d_fronts, L.d_fwd_items + drop, L.n_fwd_items - drop,
                                             h.d_ticket + tk, h.d_err, h.wait_cycles)));
            count_launch();
            prof_end(h, pi, fbytes / sizeof(T) * 2.0, fbytes);
        }
    } else {
        const int gi = prof_begin(h, K_GATHER);
        k_bwd_gather<A><<<dim3((unsigned)nf, (unsigned)std::max(1, std::min((L.max_b + 255) / 256, (4 * h.num_sms + nf - 1) / nf))),
                          256, 0, h.stream>>>(L.d_fronts, z);
        count_launch();
        prof_end(h, gi, 0.0, gbytes);
        RSD_CUDA_TRY(cudaGetLastError());
        if (L.n_bwd_items) {
            // nonsymmetric fronts: [U^T; Y^T] with (U_kk^T)^-1
            const FrontDesc* bf = L.d_fronts_bwd ? L.d_fronts_bwd : L.d_fronts;
            const int pi = prof_begin(h, K_BWD);
            RSD_TRY((launch_bwd_level<T, A>(L, grid, h.stream, bf, L.d_bwd_items, L.n_bwd_items, h.d_ticket + tk, h.d_err, z,
                                             h.wait_cycles)));
            count_launch();
            prof_end(h, pi, fbytes / sizeof(T) * 2.0, fbytes);
        }
    }
    RSD_CUDA_TRY(cudaGetLastError());
    return RSD_OK;
}

}  // namespace

// Bytes one sweep streams from the factor: the off-diagonal blocks of L and X (FP16 for a
// level with the FP16 copy) and the inverted diagonal blocks; with_x = false counts L alone
// (the leaf solves of paper mode).
double level_factor_bytes(const Level& L, bool with_x) {
    double e = 0, d = 0;
    for (auto& f : L.fronts) {
        e += 0.5 * f.s * (f.s + 1.0) + (with_x ? (double)f.s * f.b : 0.0);
        for (int k = 0; k < f.nd; ++k) {
            const double w = std::min(NB, f.s - k * NB);
            e -= 0.5 * w * (w + 1.0);
        }
        d += (double)f.nd * NB * NB;
    }
    return e * (L.h16 ? 2.0 : (double)elem_bytes(L.prec)) + d * elem_bytes(L.prec);
}

int run_apply(Handle& h, const double* r, double* z) {
    const int nl = (int)h.levels.size();
    RSD_CUDA_TRY(cudaMemsetAsync(h.d_ticket, 0, sizeof(int) * 2 * nl, h.stream));
    for (int li = nl - 1; li >= 0; --li) {
        const int rc = is_fp64(h.levels[li].prec) ? sweep_level<double, double>(h, li, true, r, z, li)
                                                  : sweep_level<float, float>(h, li, true, r, z, li);
        if (rc != RSD_OK) return rc;
    }
    for (int li = 0; li < nl; ++li) {
        const int rc = is_fp64(h.levels[li].prec) ? sweep_level<double, double>(h, li, false, r, z, nl + li)
                                                  : sweep_level<float, float>(h, li, false, r, z, nl + li);
        if (rc != RSD_OK) return rc;
    }
    return RSD_OK;
}

}  // namespace rsd

// ---- allocation-free variant of the preconditioner application ----------------------
// Same kernels as run_apply; the per-call scratch (front vectors, progress counters and
// ticket counters) lives in one file-scope device array instead of the handle's arena.
// rsd_setup prepares, with the handle's device current, a second copy of the handle's
// front descriptors whose vector and counter pointers point into that array, and stores
// it in the handle's arena; a call then only clears the counters and launches the
// sweeps.  Every handle on a device shares the array.
namespace rsd {
namespace {

constexpr size_t APPLY_STATIC_BYTES = (size_t)4 << 20;          // 4 MiB per device
__device__ __align__(256) unsigned char g_apply_scratch[APPLY_STATIC_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_scratch_mu;
void* g_apply_scratch_ptr[MAX_DEVICES] = {};

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Device address of the array on the current device (looked up once per device).
int scratch_address(int dev, char** out) {
    if (dev < 0 || dev >= MAX_DEVICES) return RSD_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_apply_scratch_ptr[dev]) {
        void* p = nullptr;
        RSD_CUDA_TRY(cudaGetSymbolAddress(&p, g_apply_scratch));
        g_apply_scratch_ptr[dev] = p;
    }
    *out = (char*)g_apply_scratch_ptr[dev];
    return RSD_OK;
}

template <typename T, typename A>
int sweep_level_static(Handle& h, int li, bool forward, const double* r, double* z, int* ticket) {
    RSD_TRY((sweep_smem_setup<T, A>()));
    Level& L = h.levels[li];
    const int nf = (int)L.fronts.size();
    const FrontDesc* fr = h.d_static_fronts + h.static_level_first[li];
    const int grid = std::max(1, std::min(forward ? L.n_fwd_items : L.n_bwd_items, h.num_sms * 4));
    if (forward) {
        const dim3 gg((unsigned)nf, (unsigned)std::max(1, std::min((L.max_N + 255) / 256, (4 * h.num_sms + nf - 1) / nf)));
        if (li + 1 < (int)h.levels.size()) {
            const Level& Lc = h.levels[li + 1];
            const FrontDesc* kids = h.d_static_fronts + h.static_level_first[li + 1];
            if (is_fp64(Lc.prec)) k_fwd_gather_inv<A, double><<<gg, 256, 0, h.stream>>>(fr, kids, L.d_child_slots, r);
            else k_fwd_gather_inv<A, float><<<gg, 256, 0, h.stream>>>(fr, kids, L.d_child_slots, r);
        } else {
            k_fwd_gather_inv<A, A><<<gg, 256, 0, h.stream>>>(fr, fr, L.d_child_slots, r);
        }
        count_launch();
        RSD_CUDA_TRY(cudaGetLastError());
        if (L.n_fwd_items) {
            RSD_TRY((launch_fwd_level<T, A>(L, grid, h.stream, fr, L.d_fwd_items, L.n_fwd_items, ticket, h.d_err, h.wait_cycles)));
            count_launch();
        }
    } else {
        k_bwd_gather<A><<<dim3((unsigned)nf, (unsigned)std::max(1, std::min((L.max_b + 255) / 256, (4 * h.num_sms + nf - 1) / nf))),
                          256, 0, h.stream>>>(fr, z);
        count_launch();
        RSD_CUDA_TRY(cudaGetLastError());
        if (L.n_bwd_items) {
            RSD_TRY((launch_bwd_level<T, A>(L, grid, h.stream, fr, L.d_bwd_items, L.n_bwd_items, ticket, h.d_err, z, h.wait_cycles)));
            count_launch();
        }
    }
    RSD_CUDA_TRY(cudaGetLastError());
    return RSD_OK;
}

}  // namespace

int static_apply_prepare(Handle& h, FrontDesc* d_slots) {
    h.static_ok = false;
    h.d_static_fronts = d_slots;
    if (h.paper || h.lu) return RSD_OK;
    char* base = nullptr;
    RSD_TRY(scratch_address(h.device, &base));
    const int nl = (int)h.levels.size();
    // layout: tickets | progress counters | front vectors
    size_t off = 0;
    const size_t o_ticket = off; off = align256(off + sizeof(int) * 2 * nl);
    const size_t o_flags = off;  off = align256(off + sizeof(int) * 2 * (size_t)h.n_nodes);
    h.static_clear_bytes = off;
    size_t vec_bytes = 0;
    for (auto& L : h.levels)
        for (auto& f : L.fronts) vec_bytes += align256((size_t)(f.N + 32) * elem_bytes(L.prec));
    const size_t o_vec = off;
    off += vec_bytes;
    h.static_need = off;
    if (off > APPLY_STATIC_BYTES) return RSD_OK;       // rsd_apply_static will refuse the handle
    std::vector<FrontDesc> desc;
    desc.reserve(h.n_nodes);
    h.static_level_first.assign(nl, 0);
    size_t voff = o_vec;
    for (int li = 0; li < nl; ++li) {
        Level& L = h.levels[li];
        h.static_level_first[li] = (int)desc.size();
        for (auto& f : L.fronts) {
            FrontDesc g = f;
            g.vec = base + voff;
            voff += align256((size_t)(f.N + 32) * elem_bytes(L.prec));
            g.flag = (int*)(base + o_flags) + 2 * f.node;
            desc.push_back(g);
        }
    }
    if (!desc.empty())
        RSD_CUDA_TRY(cudaMemcpyAsync(d_slots, stage_host(h, desc.data(), sizeof(FrontDesc) * desc.size()),
                                     sizeof(FrontDesc) * desc.size(), cudaMemcpyHostToDevice, h.stream));
    h.static_ticket = (int*)(base + o_ticket);
    h.static_ok = true;
    return RSD_OK;
}

size_t static_apply_limit() { return APPLY_STATIC_BYTES; }

int run_apply_static(Handle& h, const double* r, double* z) {
    int dev = -1;
    RSD_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != h.device) {
        set_last_error("rsd_apply_static: the current device (" + std::to_string(dev) +
                       ") is not the handle's device (" + std::to_string(h.device) + ")");
        return RSD_ERR_ARG;
    }
    if (h.lu) {
        set_last_error("rsd_apply_static: nonsymmetric (LU) hierarchies are not supported");
        return RSD_ERR_ARG;
    }
    if (!h.static_ok) {
        set_last_error("rsd_apply_static: this hierarchy needs " + std::to_string(h.static_need) +
                       " bytes of scratch; the static limit is " + std::to_string(APPLY_STATIC_BYTES));
        return RSD_ERR_ARG;
    }
    const int nl = (int)h.levels.size();
    RSD_CUDA_TRY(cudaMemsetAsync(h.static_ticket, 0, h.static_clear_bytes, h.stream));
    int* ticket = h.static_ticket;
    for (int li = nl - 1; li >= 0; --li) {
        const int rc = is_fp64(h.levels[li].prec)
                           ? sweep_level_static<double, double>(h, li, true, r, z, ticket + li)
                           : sweep_level_static<float, float>(h, li, true, r, z, ticket + li);
        if (rc != RSD_OK) return rc;
    }
    for (int li = 0; li < nl; ++li) {
        const int rc = is_fp64(h.levels[li].prec)
                           ? sweep_level_static<double, double>(h, li, false, r, z, ticket + nl + li)
                           : sweep_level_static<float, float>(h, li, false, r, z, ticket + nl + li);
        if (rc != RSD_OK) return rc;
    }
    return RSD_OK;
}

}  // namespace rsd

// ---- one level of a sweep with explicit descriptors (paper-mode leaf/interface solves) --
namespace rsd {

int sweep_with(Handle& h, int li, bool forward, const FrontDesc* fronts, const int* items, int n_items,
               const double* in, double* out, int* ticket) {
    Level& L = h.levels[li];
    const int nf = (int)L.fronts.size();
    const int grid = std::max(1, std::min(n_items, h.num_sms * 4));
    const bool f64 = is_fp64(L.prec);
    if (f64) { RSD_TRY((sweep_smem_setup<double, double>())); } else { RSD_TRY((sweep_smem_setup<float, float>())); }
    if (forward) {
        if (f64) k_fwd_gather<double, double><<<nf, 256, 0, h.stream>>>(fronts, fronts, L.d_child_slots, in);
        else k_fwd_gather<float, float><<<nf, 256, 0, h.stream>>>(fronts, fronts, L.d_child_slots, in);
        count_launch();
        RSD_CUDA_TRY(cudaGetLastError());
        if (n_items) {
            if (f64) launch_fwd<double, double>(sweep_group(L), false, grid, h.stream, fronts, items, n_items, ticket, h.d_err, h.wait_cycles);
            else launch_fwd<float, float>(sweep_group(L), L.h16, grid, h.stream, fronts, items, n_items, ticket, h.d_err, h.wait_cycles);
            count_launch();
        }
    } else if (n_items) {
        if (f64) launch_bwd<double, double>(sweep_group(L), false, grid, h.stream, fronts, items, n_items, ticket, h.d_err, out, h.wait_cycles);
        else launch_bwd<float, float>(sweep_group(L), L.h16, grid, h.stream, fronts, items, n_items, ticket, h.d_err, out, h.wait_cycles);
        count_launch();
    }
    RSD_CUDA_TRY(cudaGetLastError());
    return RSD_OK;
}

}  // namespace rsd
