// Tensor-core (tcgen05, TF32 in / FP32 accumulate) batched GEMM for the partial Cholesky
// of the fronts: the panel update (a), the panel solve by the inverted diagonal block (c)
// and the Schur contribution U -= X X^T (d) (see factor.cu).
//
//   C[M x N] = beta * C + alpha * A[M x K] * B[N x K]^T      (row-major, FP32 storage)
//
// One CTA computes one BM x BN tile:
//   warp 0      : TMA producer.  A and B tiles (32 FP32 = 128 B of K per row) are copied by
//                 cp.async.bulk.tensor with 128-byte swizzle into a STAGES-deep ring.
//   warp 1      : allocates the TMEM accumulator (BN columns x 128 lanes) and, from one
//                 thread, issues tcgen05.mma.kind::tf32 (M = 128, N = BN, K = 8) for each
//                 K slice; tcgen05.commit frees ring slots and finally signals the epilogue.
//   warps 2..5  : epilogue.  tcgen05.ld moves each accumulator row into registers (TMEM
//                 lane = tile row), then C is read-modified-written with 16-byte accesses
//                 (the persistent variant below: warps 2..9, two per row, half a row each).
// Operands stay in the front matrices: one 2-D tensor map per front covers its [L; X]
// panel (N rows x s columns) and one covers its stacked inverted diagonal blocks; TMA's
// zero fill handles ragged edges.  Every mbarrier wait is bounded; on timeout the CTA
// raises ERR_TIMEOUT, drains, frees its TMEM and exits.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "rsd_internal.cuh"

namespace rsd {

namespace {

constexpr int BM = 128;
constexpr int BK = 32;                       // FP32 elements per 128-byte swizzle row
// Operand formats: TF32 (FP32 storage, kind::tf32, 8 K per MMA) or a 16-bit copy (FP16
// or BF16, kind::f16, 16 K per MMA).  A K block is one 128-byte swizzle row either way:
// 32 FP32 or 64 16-bit elements, four MMAs.
template <int OP> struct OpT {
    static constexpr int BKE = OP == TC_OP_TF32 ? 32 : 64;      // elements per K block
    static constexpr uint32_t FMT = OP == TC_OP_TF32 ? 2u : (OP == TC_OP_BF16 ? 1u : 0u);
};
constexpr int TC_THREADS = 192;
// persistent kernel: producer, MMA issuer and 4 x TCP_SPLIT epilogue warps (TCP_SPLIT per
// TMEM lane quadrant, each taking 1 / TCP_SPLIT of the tile's columns)
constexpr int TCP_SPLIT = 2;
constexpr int TCP_THREADS = 64 + 128 * TCP_SPLIT;
constexpr long long TC_WAIT_CYCLES = 2000000000LL;   // ~1 s
constexpr int SPLIT_MIN_KB = 16;             // at least 16 x 32 K per split-K slice
constexpr int TILE_BAND = 16;                // row blocks per band of a wide output's tile order

// One CTA's work: output tile (tm, tn) of a task over K blocks [kb0, kb1).  ws_slot < 0:
// write C directly; otherwise write the raw partial product to workspace slot ws_slot
// (split-K), to be summed in fixed order by k_splitk_reduce.
struct TcTile { int task, tm, tn, kb0, kb1, ws_slot, pad0, pad1; };
// One split-K output tile: partials in slots [slot0, slot0 + nsplit).
struct TcRed { int task, tm, tn, slot0, nsplit, pad0, pad1, pad2; };

struct TcTask {               // device view of one GEMM task
    float* C;
    int ldc, M, N, K;
    int lower, beta;
    int map_a, map_b;
    int a_r0, a_c0, b_r0, b_c0;
    float alpha;
    int round_tf32;           // round stored results to the nearest TF32 value
    // 16-bit operands: row i of A (B) was stored scaled by 1 / sa[i] (1 / sb[i]), so the
    // product is multiplied by sa[row] sb[col]; null for TF32 operands
    const float* sa;
    const float* sb;
};

// Round to the nearest TF32 value (10-bit mantissa), kept as an FP32 bit pattern.
__device__ __forceinline__ float tf32_rn(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Pull the C rows an epilogue thread will read into L2 while the main loop runs, so the
// read-modify-write of the tile waits on L2 rather than on DRAM.
__device__ __forceinline__ void prefetch_c_row(const float* crow, int c_lo, int c_hi) {
    for (int c = c_lo; c < c_hi; c += 32) asm volatile("prefetch.global.L2 [%0];" ::"l"(crow + c));
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait; returns false (and raises the error flag) on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err) {
    if (mbar_try(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try(bar, parity)) {
        if (clock64() - t0 > TC_WAIT_CYCLES || *(volatile int*)&err[ERR_TIMEOUT]) {
            atomicExch(&err[ERR_TIMEOUT], 1);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);          // start address
    d |= (uint64_t)0 << 16;                           // leading byte offset (unused, swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;                 // stride byte offset
    d |= (uint64_t)1 << 46;                           // descriptor version
    d |= (uint64_t)2 << 61;                           // 128-byte swizzle
    return d;
}

// Instruction descriptor: D = F32, A = B of format fmt (TF32 2; F16 0; BF16 1), both
// K-major, M = 128, N = bn.
__host__ __device__ constexpr uint32_t idesc_of(uint32_t fmt, int bn) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(bn >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}
__host__ __device__ constexpr uint32_t idesc_tf32(int bn) { return idesc_of(2u, bn); }

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_f16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc)
        : "memory");
}

template <int OP>
__device__ __forceinline__ void mma_op(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    if constexpr (OP == TC_OP_TF32) mma_tf32(tmem, da, db, idesc, acc);
    else mma_f16(tmem, da, db, idesc, acc);
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

template <int BN, int ST>
struct Smem {
    static constexpr int STAGES = ST;
    static constexpr int A_BYTES = BM * BK * 4;
    static constexpr int B_BYTES = BN * BK * 4;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int TOTAL = STAGES * STAGE + 1024 /*align*/ + 256 /*barriers*/;
};

template <int BN, int ST>
__global__ void __launch_bounds__(TC_THREADS, ST <= 3 ? 2 : 1)
k_gemm_tc(const TcTask* __restrict__ tasks, const TcTile* __restrict__ tiles,
          const CUtensorMap* __restrict__ maps, float* __restrict__ ws, int* __restrict__ err) {
    extern __shared__ unsigned char smem_raw[];
    using S = Smem<BN, ST>;
    constexpr int STAGES = S::STAGES;
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023) & ~1023u;
    unsigned char* sbase = smem_raw + (base - raw);
    const uint32_t bar_full = base + STAGES * S::STAGE;            // STAGES x 8 B
    const uint32_t bar_empty = bar_full + 8 * STAGES;
    const uint32_t bar_done = bar_empty + 8 * STAGES;
    uint32_t* tmem_slot = (uint32_t*)(sbase + STAGES * S::STAGE + 24 * STAGES + 16);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    const TcTile tl = tiles[blockIdx.x];
    const TcTask tk = tasks[tl.task];
    const int m0 = tl.tm * BM, n0 = tl.tn * BN;
    const int kb0 = tl.kb0, nk = tl.kb1 - tl.kb0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(bar_full + 8 * s, 1);
            mbar_init(bar_empty + 8 * s, 1);
        }
        mbar_init(bar_done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tmem_slot)), "r"(BN) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            const CUtensorMap* ma = maps + tk.map_a;
            const CUtensorMap* mb = maps + tk.map_b;
            for (int kb = 0; kb < nk; ++kb) {
                const int s = kb % STAGES;
                const uint32_t ph = (kb / STAGES) & 1;
                if (!mbar_wait(bar_empty + 8 * s, ph ^ 1, err)) break;
                const uint32_t sa = base + s * S::STAGE;
                const uint32_t sb = sa + S::A_BYTES;
                mbar_expect_tx(bar_full + 8 * s, S::STAGE);
                const int kx = (kb0 + kb) * BK;
                tma_load_2d(sa, ma, tk.a_c0 + kx, tk.a_r0 + m0, bar_full + 8 * s);
#pragma unroll
                for (int h = 0; h < BN / 128; ++h)
                    tma_load_2d(sb + h * 128 * BK * 4, mb, tk.b_c0 + kx, tk.b_r0 + n0 + h * 128, bar_full + 8 * s);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_tf32(BN);
            bool ok = true;
            for (int kb = 0; kb < nk && ok; ++kb) {
                const int s = kb % STAGES;
                const uint32_t ph = (kb / STAGES) & 1;
                ok = mbar_wait(bar_full + 8 * s, ph, err);
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t sa = base + s * S::STAGE;
                const uint32_t sb = sa + S::A_BYTES;
#pragma unroll
                for (int k = 0; k < BK / 8; ++k)
                    mma_tf32(tmem, smem_desc(sa + k * 32), smem_desc(sb + k * 32), idesc, (kb | k) != 0);
                mma_commit(bar_empty + 8 * s);
            }
            mma_commit(bar_done);
        }
    } else {
        // epilogue: warp (2..5) reads TMEM lanes 32*(warp%4) .. +31
        const int quarter = warp & 3;
        const int row = quarter * 32 + lane;
        const int gr = m0 + row;
        float* crow = tk.C + (int64_t)gr * tk.ldc;
        if (tk.beta && tl.ws_slot < 0 && gr < tk.M)
            prefetch_c_row(crow, n0, min(n0 + BN, tk.lower ? min(tk.N, gr + 1) : tk.N));
        const bool ok = mbar_wait(bar_done, 0, err);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        float* wrow = tl.ws_slot >= 0 ? ws + ((int64_t)tl.ws_slot * BM + row) * BN : nullptr;
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 32) {
            uint32_t r[32];
            tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + c0, r);
            if (!ok) continue;
            if (wrow) {                                   // split-K partial: raw product
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    *(float4*)(wrow + c0 + 4 * q) = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                                                                __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
                continue;
            }
            if (gr >= tk.M) continue;
            const int gc0 = n0 + c0;
            if (gc0 >= tk.N) continue;
            if (tk.lower && gc0 > gr) continue;
            if (gc0 + 32 <= tk.N && (!tk.lower || gc0 + 31 <= gr)) {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    float4* p = (float4*)(crow + gc0 + 4 * q);
                    float4 o = tk.beta ? *p : make_float4(0.f, 0.f, 0.f, 0.f);
                    o.x += tk.alpha * __uint_as_float(r[4 * q + 0]);
                    o.y += tk.alpha * __uint_as_float(r[4 * q + 1]);
                    o.z += tk.alpha * __uint_as_float(r[4 * q + 2]);
                    o.w += tk.alpha * __uint_as_float(r[4 * q + 3]);
                    if (tk.round_tf32) { o.x = tf32_rn(o.x); o.y = tf32_rn(o.y); o.z = tf32_rn(o.z); o.w = tf32_rn(o.w); }
                    *p = o;
                }
            } else {
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    const int gc = gc0 + q;
                    if (gc < tk.N && (!tk.lower || gc <= gr)) {
                        float* p = crow + gc;
                        const float o = (tk.beta ? *p : 0.f) + tk.alpha * __uint_as_float(r[q]);
                        *p = tk.round_tf32 ? tf32_rn(o) : o;
                    }
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
    }
}

// Persistent variant for the long-K 128 x 256 tiles: one CTA per SM walks the tile list
// with stride gridDim.x.  The smem ring runs continuously across tiles, and the TMEM
// accumulator is double-buffered (2 x 256 columns), so the epilogue of one tile overlaps
// the main loop of the next.  Barriers: full/empty per ring stage, and acc_full/acc_empty
// per accumulator buffer (acc_empty counts the 256 epilogue threads).  The epilogue has
// two warps per TMEM lane quadrant, one per half of the tile's columns, so twice as many
// loads of C are in flight in the read-modify-write (at short K the tile's epilogue, not
// its MMAs, sets the pace).
template <int BN, int ST, int OP = TC_OP_TF32>
__global__ void __launch_bounds__(TCP_THREADS, 1)
k_gemm_tc_persist(const TcTask* __restrict__ tasks, const TcTile* __restrict__ tiles, int n_tiles,
                  const CUtensorMap* __restrict__ maps, float* __restrict__ ws, int* __restrict__ err) {
    extern __shared__ unsigned char smem_raw[];
    using S = Smem<BN, ST>;
    constexpr int STAGES = S::STAGES;
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023) & ~1023u;
    unsigned char* sbase = smem_raw + (base - raw);
    const uint32_t bar_full = base + STAGES * S::STAGE;            // STAGES x 8 B
    const uint32_t bar_empty = bar_full + 8 * STAGES;               // STAGES x 8 B
    const uint32_t bar_accf = bar_empty + 8 * STAGES;               // 2 x 8 B
    const uint32_t bar_acce = bar_accf + 16;                        // 2 x 8 B
    uint32_t* tmem_slot = (uint32_t*)(sbase + STAGES * S::STAGE + 16 * STAGES + 32 + 16);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(bar_full + 8 * s, 1);
            mbar_init(bar_empty + 8 * s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(bar_accf + 8 * b, 1);
            mbar_init(bar_acce + 8 * b, (TCP_THREADS / 32 - 2) * 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tmem_slot)), "r"(2 * BN) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            uint32_t it = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
                const TcTile tl = tiles[t];
                const TcTask tk = tasks[tl.task];
                const CUtensorMap* ma = maps + tk.map_a;
                const CUtensorMap* mb = maps + tk.map_b;
                const int m0 = tl.tm * BM, n0 = tl.tn * BN;
                for (int kb = tl.kb0; kb < tl.kb1; ++kb, ++it) {
                    const int s = it % STAGES;
                    const uint32_t ph = (it / STAGES) & 1;
                    if (!mbar_wait(bar_empty + 8 * s, ph ^ 1, err)) { ok = false; break; }
                    const uint32_t sa = base + s * S::STAGE;
                    const uint32_t sb = sa + S::A_BYTES;
                    mbar_expect_tx(bar_full + 8 * s, S::STAGE);
                    const int kx = kb * OpT<OP>::BKE;
                    tma_load_2d(sa, ma, tk.a_c0 + kx, tk.a_r0 + m0, bar_full + 8 * s);
#pragma unroll
                    for (int hh = 0; hh < BN / 128; ++hh)
                        tma_load_2d(sb + hh * 128 * 128, mb, tk.b_c0 + kx, tk.b_r0 + n0 + hh * 128, bar_full + 8 * s);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_of(OpT<OP>::FMT, BN);
            uint32_t it = 0, tcount = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x, ++tcount) {
                const TcTile tl = tiles[t];
                const uint32_t buf = tcount & 1, use = (tcount >> 1) & 1;
                if (!mbar_wait(bar_acce + 8 * buf, use ^ 1, err)) { ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t acc = tmem + buf * BN;
                for (int kb = tl.kb0; kb < tl.kb1; ++kb, ++it) {
                    const int s = it % STAGES;
                    const uint32_t ph = (it / STAGES) & 1;
                    if (!mbar_wait(bar_full + 8 * s, ph, err)) { ok = false; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t sa = base + s * S::STAGE;
                    const uint32_t sb = sa + S::A_BYTES;
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        mma_op<OP>(acc, smem_desc(sa + k * 32), smem_desc(sb + k * 32), idesc, (kb != tl.kb0 || k) ? 1u : 0u);
                    mma_commit(bar_empty + 8 * s);
                }
                mma_commit(bar_accf + 8 * buf);
            }
        }
    } else {
        const int quarter = warp & 3;
        const int row = quarter * 32 + lane;
        const int cb = ((warp - 2) >> 2) * (BN / TCP_SPLIT), ce = cb + BN / TCP_SPLIT;   // this warp's columns
        uint32_t tcount = 0;
        for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, ++tcount) {
            const TcTile tl = tiles[t];
            const TcTask tk = tasks[tl.task];
            const uint32_t buf = tcount & 1, use = (tcount >> 1) & 1;
            const int m0 = tl.tm * BM, n0 = tl.tn * BN;
            const int gr = m0 + row;
            float* crow = tk.C + (int64_t)gr * tk.ldc;
            if (tk.beta && tl.ws_slot < 0 && gr < tk.M)
                prefetch_c_row(crow, n0 + cb, min(n0 + ce, tk.lower ? min(tk.N, gr + 1) : tk.N));
            const bool ok = mbar_wait(bar_accf + 8 * buf, use, err);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            float* wrow = tl.ws_slot >= 0 ? ws + ((int64_t)tl.ws_slot * BM + row) * BN : nullptr;
#pragma unroll 1
            for (int c0 = cb; c0 < ce; c0 += 32) {
                uint32_t r[32];
                tmem_ld32(tmem + buf * BN + ((uint32_t)(quarter * 32) << 16) + c0, r);
                if (!ok) continue;
                if (wrow) {
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        *(float4*)(wrow + c0 + 4 * q) = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                                                                    __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
                    continue;
                }
                if (gr >= tk.M) continue;
                const int gc0 = n0 + c0;
                if (gc0 >= tk.N) continue;
                if (tk.lower && gc0 > gr) continue;
                if constexpr (OP != TC_OP_TF32) {
                    // undo the operands' row scales: entry (gr, gc) times sa[gr] sb[gc]
                    const float ar = tk.alpha * tk.sa[gr];
                    const int qe = min(32, tk.N - gc0);
#pragma unroll
                    for (int q = 0; q < 32; ++q)
                        r[q] = __float_as_uint(q < qe ? __uint_as_float(r[q]) * ar * __ldg(tk.sb + gc0 + q) : 0.f);
                }
                const float al = OP != TC_OP_TF32 ? 1.0f : tk.alpha;
                if (gc0 + 32 <= tk.N && (!tk.lower || gc0 + 31 <= gr)) {
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        float4* p = (float4*)(crow + gc0 + 4 * q);
                        float4 o = tk.beta ? *p : make_float4(0.f, 0.f, 0.f, 0.f);
                        o.x += al * __uint_as_float(r[4 * q + 0]);
                        o.y += al * __uint_as_float(r[4 * q + 1]);
                        o.z += al * __uint_as_float(r[4 * q + 2]);
                        o.w += al * __uint_as_float(r[4 * q + 3]);
                        if (tk.round_tf32) { o.x = tf32_rn(o.x); o.y = tf32_rn(o.y); o.z = tf32_rn(o.z); o.w = tf32_rn(o.w); }
                        *p = o;
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 32; ++q) {
                        const int gc = gc0 + q;
                        if (gc < tk.N && (!tk.lower || gc <= gr)) {
                            float* p = crow + gc;
                            const float o = (tk.beta ? *p : 0.f) + al * __uint_as_float(r[q]);
                            *p = tk.round_tf32 ? tf32_rn(o) : o;
                        }
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar_acce + 8 * buf) : "memory");
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * BN) : "memory");
    }
}

// Split-K reduction: C = beta*C + alpha * sum_s partial_s, summed in slot order.  A CTA
// takes RED_ROWS rows of one output tile (blockIdx.y), a thread the same column of
// RED_ROWS * BN / 256 of those rows: all of its partial-product loads are issued before
// its reads and writes of C.
constexpr int RED_ROWS = 8;
template <int BN>
__global__ void __launch_bounds__(256) k_splitk_reduce(const TcTask* __restrict__ tasks, const TcRed* __restrict__ reds,
                                                       const float* __restrict__ ws) {
    constexpr int PER = RED_ROWS * BN / 256;          // elements per thread
    constexpr int RSTEP = 256 / BN;                    // rows between a thread's elements
    const TcRed rd = reds[blockIdx.x];
    const TcTask tk = tasks[rd.task];
    const int m0 = rd.tm * BM, n0 = rd.tn * BN;
    const int col = threadIdx.x % BN;
    const int rbase = blockIdx.y * RED_ROWS + threadIdx.x / BN;
    float v[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) v[q] = 0.f;
    for (int sp = 0; sp < rd.nsplit; ++sp) {
        const float* w = ws + (int64_t)(rd.slot0 + sp) * BM * BN;
#pragma unroll
        for (int q = 0; q < PER; ++q) v[q] += w[(int64_t)(rbase + RSTEP * q) * BN + col];
    }
    const int gc = n0 + col;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int gr = m0 + rbase + RSTEP * q;
        if (gr >= tk.M || gc >= tk.N || (tk.lower && gc > gr)) continue;
        float x = v[q];
        if (tk.sa) x *= tk.sa[gr] * tk.sb[gc];        // 16-bit operands: undo the row scales
        float* p = tk.C + (int64_t)gr * tk.ldc + gc;
        const float o = (tk.beta ? *p : 0.f) + tk.alpha * x;
        *p = tk.round_tf32 ? tf32_rn(o) : o;
    }
}

// ---- host side ---------------------------------------------------------------------
using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn get_encode() {
    static EncodeFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeFn)p;
    }
    return fn;
}

// 2-D tensor map over a row-major matrix: boxes of 128 rows x 128 bytes (one swizzle
// row: 32 FP32 or 64 16-bit elements), 128-byte swizzle.
int encode_2d(CUtensorMap* m, void* base, int cols, int rows, int ld_elems, int op = TC_OP_TF32) {
    EncodeFn enc = get_encode();
    if (!enc) { set_last_error("cuTensorMapEncodeTiled unavailable"); return RSD_ERR_CUDA; }
    const int es_b = op == TC_OP_TF32 ? 4 : 2;
    cuuint64_t dims[2] = {(cuuint64_t)std::max(cols, 1), (cuuint64_t)std::max(rows, 1)};
    cuuint64_t strides[1] = {(cuuint64_t)ld_elems * es_b};
    cuuint32_t box[2] = {(cuuint32_t)(128 / es_b), 128};
    cuuint32_t es[2] = {1, 1};
    const CUtensorMapDataType dt = op == TC_OP_TF32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : op == TC_OP_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    CUresult r = enc(m, dt, 2, base, dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) { set_last_error("cuTensorMapEncodeTiled failed: " + std::to_string((int)r)); return RSD_ERR_CUDA; }
    return RSD_OK;
}

// Per-stream launch buffers: task/tile lists and the split-K workspace are rewritten by
// every launch, so two streams that launch concurrently each need their own set.
struct TcBuf {
    TcTask* d_tasks = nullptr;
    TcTile* d_tiles = nullptr;
    TcRed* d_reds = nullptr;
    float* d_ws = nullptr;              // split-K partial products
    size_t cap_tasks = 0, cap_tiles = 0, cap_reds = 0;
};

// Autotuned launch configurations (rsd_autotune / rsd_options.tune_cache): for an operand
// format, a launch's output tiles (counted at 128 x 256) and its longest K, the tile width
// and the split-K count that measured fastest on synthetic operands of that size.
struct TuneEntry { int op, tiles, k, bn, split; float us, us_rule; };

struct TcState {
    std::vector<TuneEntry> tune;        // empty: the built-in rules
    int force_bn = 0, force_split = 0;  // the tuner's candidate under measurement (0: none)
    CUtensorMap* d_maps = nullptr;      // TC_NODE_MAPS per tree node: [L; X] panel, inverted
                                        // diagonal blocks, 16-bit copy; then TC_SCR_MAPS per
                                        // front slot of the widest level
    int scr_base = 0, scr_slots = 0;
    TcBuf buf[TC_SLOTS];
    // recorded launches (gemm_tc_record_begin/end): lists built by a dry pass, uploaded
    // once, consumed in order by the real pass
    struct Rec { size_t o_tasks, o_tiles, o_reds; int n_tasks, n_tiles, n_reds, bn, max_kb; double fl, by; };
    int mode = 0;                       // 0 direct, 1 recording, 2 replaying
    std::vector<char> rec_buf;
    std::vector<Rec> recs;
    size_t cursor = 0;
    char* d_meta = nullptr;
    int ws_slots = 0;                   // split-K capacity per slot, in BM x 256 tiles
    bool attr_set = false;
};

std::vector<TcState*>& states() { static std::vector<TcState*> v; return v; }

TcState* state_of(Handle& h) { return (TcState*)h.tc_state; }

}  // namespace

// Nearest tuned bucket (log distance in tiles and K) for the operand format; 0 when the
// table has none for it.
static void tune_lookup(const std::vector<TuneEntry>& tab, int op, int tiles, int k, int* bn, int* split) {
    double best = 1e30;
    *bn = 0;
    *split = 0;
    for (const TuneEntry& e : tab) {
        if (e.op != op) continue;
        const double d = std::fabs(std::log2((double)std::max(tiles, 1) / std::max(e.tiles, 1))) +
                         std::fabs(std::log2((double)std::max(k, 1) / std::max(e.k, 1)));
        if (d < best) { best = d; *bn = e.bn; *split = e.split; }
    }
}

// Read a table written by rsd_autotune: one JSON object per line in its "entries" array.
// out_table: a std::vector<TuneEntry>* to fill, or null to validate only.
int tune_read(const char* path, void* out_table, int32_t* entries) {
    std::vector<TuneEntry>* out = (std::vector<TuneEntry>*)out_table;
    FILE* fp = std::fopen(path, "r");
    if (!fp) { set_last_error(std::string("tune cache not readable: ") + path); return RSD_ERR_ARG; }
    char line[512];
    std::vector<TuneEntry> tab;
    bool header = false;
    while (std::fgets(line, sizeof line, fp)) {
        if (std::strstr(line, "\"entries\"")) header = true;
        const char* q = std::strstr(line, "{\"op\":");
        if (!q) continue;
        TuneEntry e{};
        if (std::sscanf(q, "{\"op\": %d, \"tiles\": %d, \"k\": %d, \"bn\": %d, \"split\": %d, \"us\": %f, \"us_rule\": %f}",
                        &e.op, &e.tiles, &e.k, &e.bn, &e.split, &e.us, &e.us_rule) != 7 ||
            (e.bn != 128 && e.bn != 256) || e.split < 1 || e.split > 64 || e.tiles < 1 || e.k < 1 ||
            (e.op != TC_OP_TF32 && e.op != TC_OP_F16)) {
            std::fclose(fp);
            set_last_error(std::string("malformed tune cache entry in ") + path);
            return RSD_ERR_ARG;
        }
        tab.push_back(e);
    }
    std::fclose(fp);
    if (!header || tab.empty()) { set_last_error(std::string("tune cache without entries: ") + path); return RSD_ERR_ARG; }
    if (entries) *entries = (int32_t)tab.size();
    if (out) *out = std::move(tab);
    return RSD_OK;
}

int gemm_tc_prepare(Handle& h) {
    bool any = false;
    for (auto& L : h.levels) any |= tc_level(L) && L.factored;
    if (!any) return RSD_OK;
    auto* st = new TcState();
    h.tc_state = st;
    if (h.opt.tune_cache) RSD_TRY(tune_read(h.opt.tune_cache, &st->tune, nullptr));
    int widest = 0;
    for (auto& L : h.levels)
        if (tc_level(L) && L.factored) widest = std::max(widest, (int)L.fronts.size());
    st->scr_base = TC_NODE_MAPS * h.n_nodes;
    st->scr_slots = widest;
    std::vector<CUtensorMap> maps(TC_NODE_MAPS * (size_t)h.n_nodes + TC_SCR_MAPS * (size_t)widest);
    std::memset(maps.data(), 0, maps.size() * sizeof(CUtensorMap));
    for (auto& L : h.levels) {
        if (!tc_level(L) || !L.factored) continue;
        for (auto& f : L.fronts) {
            RSD_TRY(encode_2d(&maps[tc_map_panel(f.node)], f.P, f.s, f.N, f.ldp));
            RSD_TRY(encode_2d(&maps[tc_map_dinv(f.node)], f.Dinv, NB, std::max(1, f.nd) * NB, NB));
            if (L.op16 != TC_OP_TF32) RSD_TRY(encode_2d(&maps[tc_map_panel16(f.node)], f.P16, f.s, f.N, f.ldp, L.op16));
        }
    }
    RSD_CUDA_TRY(cudaMalloc((void**)&st->d_maps, maps.size() * sizeof(CUtensorMap)));
    st->ws_slots = 2 * h.num_sms;
    for (auto& b : st->buf)
        RSD_CUDA_TRY(cudaMalloc((void**)&b.d_ws, (size_t)st->ws_slots * BM * 256 * sizeof(float)));
    RSD_CUDA_TRY(cudaMemcpy(st->d_maps, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice));
    return RSD_OK;
}

int gemm_tc_scratch_maps(Handle& h, const std::vector<float*>& mt, const std::vector<float*>& tt,
                         const std::vector<float*>& linv0, const std::vector<float*>& linv1,
                         cudaStream_t stream, int* base) {
    TcState* st = state_of(h);
    const size_t n = mt.size();
    if (!st || tt.size() != n || linv0.size() != n || linv1.size() != n || (int)n > st->scr_slots) return RSD_ERR_ARG;
    std::vector<CUtensorMap> maps(TC_SCR_MAPS * n);
    for (size_t i = 0; i < n; ++i) {
        RSD_TRY(encode_2d(&maps[TC_SCR_MAPS * i + 0], mt[i], 512, 512, 512));
        RSD_TRY(encode_2d(&maps[TC_SCR_MAPS * i + 1], tt[i], 128, 512, 128));
        RSD_TRY(encode_2d(&maps[TC_SCR_MAPS * i + 2], linv0[i], 512, 512, 512));
        RSD_TRY(encode_2d(&maps[TC_SCR_MAPS * i + 3], linv1[i], 512, 512, 512));
    }
    if (n)
        RSD_CUDA_TRY(cudaMemcpyAsync(st->d_maps + st->scr_base, stage_host(h, maps.data(), maps.size() * sizeof(CUtensorMap)),
                                     maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice, stream));
    *base = st->scr_base;
    return RSD_OK;
}

int gemm_tc_record_begin(Handle& h) {
    TcState* st = state_of(h);
    if (!st || st->mode != 0) return RSD_ERR_ARG;
    st->mode = 1;
    st->rec_buf.clear();
    st->recs.clear();
    st->cursor = 0;
    return RSD_OK;
}

int gemm_tc_record_end(Handle& h, cudaStream_t stream) {
    TcState* st = state_of(h);
    if (!st || st->mode != 1) return RSD_ERR_ARG;
    st->mode = 2;
    st->d_meta = nullptr;
    if (st->rec_buf.empty()) return RSD_OK;
    RSD_CUDA_TRY(cudaMallocAsync((void**)&st->d_meta, st->rec_buf.size(), stream));
    RSD_CUDA_TRY(cudaMemcpyAsync(st->d_meta, stage_host(h, st->rec_buf.data(), st->rec_buf.size()),
                                 st->rec_buf.size(), cudaMemcpyHostToDevice, stream));
    return RSD_OK;
}

void gemm_tc_replay_end(Handle& h, cudaStream_t stream) {
    TcState* st = state_of(h);
    if (!st) return;
    if (st->d_meta) cudaFreeAsync(st->d_meta, stream);
    st->d_meta = nullptr;
    st->mode = 0;
    st->recs.clear();
    st->cursor = 0;
}

void gemm_tc_release(Handle& h) {
    TcState* st = state_of(h);
    if (!st) return;
    cudaFree(st->d_maps);
    for (auto& b : st->buf) {
        cudaFree(b.d_tasks);
        cudaFree(b.d_tiles);
        cudaFree(b.d_reds);
        cudaFree(b.d_ws);
    }
    delete st;
    h.tc_state = nullptr;
}

// ---- peak probe: the persistent 128 x 256 kernel on one n x n x n product --------------
namespace {

// Deterministic operand values in [-1, 1) from a counter hash (no host transfer).
__global__ void k_fill_hash(float* __restrict__ p, int64_t n, uint32_t seed) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t x = (uint32_t)i * 2654435761u ^ seed;
        x ^= x >> 16; x *= 0x7feb352du; x ^= x >> 15; x *= 0x846ca68bu; x ^= x >> 16;
        p[i] = (float)(x >> 8) * (1.0f / 8388608.0f) - 1.0f;
    }
}

}  // namespace

// 16-bit operand values from FP32 ones (probe inputs)
__global__ void k_to16(const float* __restrict__ src, unsigned short* __restrict__ dst, int64_t n, int bf16) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = bf16 ? __bfloat16_as_ushort(__float2bfloat16_rn(src[i])) : __half_as_ushort(__float2half_rn(src[i]));
}

int gemm_tc_peak(int n, int reps, double seconds, cudaStream_t stream, int num_sms, double* best, double* sustained,
                 int op) {
    if (n < 256 || n % 256 || reps < 1 || !best || !sustained) return RSD_ERR_ARG;
    const size_t elems = (size_t)n * n;
    char* buf = nullptr;
    const size_t o_b = elems * 4, o_c = 2 * elems * 4, o_maps = 3 * elems * 4;
    const int tm = n / BM, tn = n / 256;
    const int nkb = n / (op == TC_OP_TF32 ? BK : 64);
    std::vector<TcTile> tiles;
    for (int a0 = 0; a0 < tm; a0 += TILE_BAND)
        for (int b = 0; b < tn; ++b)
            for (int a = a0; a < std::min(tm, a0 + TILE_BAND); ++a) tiles.push_back({0, a, b, 0, nkb, -1, 0, 0});
    const size_t o_task = o_maps + 2 * sizeof(CUtensorMap);
    const size_t o_tiles = o_task + 256, o_ones = o_tiles + ((tiles.size() * sizeof(TcTile) + 255) & ~(size_t)255);
    const size_t o_err = o_ones + (size_t)n * 4;
    const size_t total = o_err + 256;
    RSD_CUDA_TRY(cudaMalloc((void**)&buf, total));
    struct Free { char* p; ~Free() { cudaFree(p); } } fr{buf};
    float* A = (float*)buf;
    float* B = (float*)(buf + o_b);
    float* Cm = (float*)(buf + o_c);
    k_fill_hash<<<1024, 256, 0, stream>>>(A, (int64_t)elems, 0x9e3779b9u);
    k_fill_hash<<<1024, 256, 0, stream>>>(B, (int64_t)elems, 0x7f4a7c15u);
    RSD_CUDA_TRY(cudaMemsetAsync(Cm, 0, elems * 4, stream));
    RSD_CUDA_TRY(cudaMemsetAsync(buf + o_err, 0, 256, stream));
    // 16-bit operands: converted copies in the C buffer's place before C is cleared
    void* Aop = A;
    void* Bop = B;
    if (op != TC_OP_TF32) {
        unsigned short* A16 = (unsigned short*)Cm;
        unsigned short* B16 = A16 + elems;
        k_to16<<<1024, 256, 0, stream>>>(A, A16, (int64_t)elems, op == TC_OP_BF16);
        k_to16<<<1024, 256, 0, stream>>>(B, B16, (int64_t)elems, op == TC_OP_BF16);
        RSD_CUDA_TRY(cudaMemcpyAsync(A, A16, elems * 2, cudaMemcpyDeviceToDevice, stream));
        RSD_CUDA_TRY(cudaMemcpyAsync(B, B16, elems * 2, cudaMemcpyDeviceToDevice, stream));
        RSD_CUDA_TRY(cudaMemsetAsync(Cm, 0, elems * 4, stream));
    }
    CUtensorMap maps[2];
    RSD_TRY(encode_2d(&maps[0], Aop, n, n, n, op));
    RSD_TRY(encode_2d(&maps[1], Bop, n, n, n, op));
    // unit row scales for the 16-bit epilogue
    float* ones = (float*)(buf + o_tiles) + ((tiles.size() * sizeof(TcTile) + 255) & ~(size_t)255) / 4;
    TcTask t{};
    t.C = Cm; t.ldc = n; t.M = n; t.N = n; t.K = n; t.lower = 0; t.beta = 1;
    t.map_a = 0; t.map_b = 1; t.alpha = -1.0f; t.round_tf32 = 0;
    t.sa = op != TC_OP_TF32 ? ones : nullptr;
    t.sb = t.sa;
    if (op != TC_OP_TF32) {
        std::vector<float> one((size_t)n, 1.0f);
        RSD_CUDA_TRY(cudaMemcpyAsync(ones, one.data(), sizeof(float) * n, cudaMemcpyHostToDevice, stream));
        RSD_CUDA_TRY(cudaStreamSynchronize(stream));
    }
    RSD_CUDA_TRY(cudaMemcpyAsync(buf + o_maps, maps, sizeof(maps), cudaMemcpyHostToDevice, stream));
    RSD_CUDA_TRY(cudaMemcpyAsync(buf + o_task, &t, sizeof(t), cudaMemcpyHostToDevice, stream));
    RSD_CUDA_TRY(cudaMemcpyAsync(buf + o_tiles, tiles.data(), tiles.size() * sizeof(TcTile), cudaMemcpyHostToDevice, stream));
    RSD_CUDA_TRY(cudaFuncSetAttribute(k_gemm_tc_persist<256, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem<256, 4>::TOTAL));
    RSD_CUDA_TRY(cudaFuncSetAttribute(k_gemm_tc_persist<256, 4, TC_OP_F16>, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem<256, 4>::TOTAL));
    RSD_CUDA_TRY(cudaFuncSetAttribute(k_gemm_tc_persist<256, 4, TC_OP_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem<256, 4>::TOTAL));
    int* err = (int*)(buf + o_err);
    const int ctas = std::min((int)tiles.size(), num_sms);
    auto launch = [&]() {
        const TcTask* tk = (const TcTask*)(buf + o_task);
        const TcTile* tl = (const TcTile*)(buf + o_tiles);
        const CUtensorMap* mp = (const CUtensorMap*)(buf + o_maps);
        if (op == TC_OP_F16)
            k_gemm_tc_persist<256, 4, TC_OP_F16><<<(unsigned)ctas, TCP_THREADS, Smem<256, 4>::TOTAL, stream>>>(tk, tl, (int)tiles.size(), mp, nullptr, err);
        else if (op == TC_OP_BF16)
            k_gemm_tc_persist<256, 4, TC_OP_BF16><<<(unsigned)ctas, TCP_THREADS, Smem<256, 4>::TOTAL, stream>>>(tk, tl, (int)tiles.size(), mp, nullptr, err);
        else
            k_gemm_tc_persist<256, 4><<<(unsigned)ctas, TCP_THREADS, Smem<256, 4>::TOTAL, stream>>>(tk, tl, (int)tiles.size(), mp, nullptr, err);
        count_launch();
    };
    cudaEvent_t e0, e1;
    RSD_CUDA_TRY(cudaEventCreate(&e0));
    RSD_CUDA_TRY(cudaEventCreate(&e1));
    struct Ev { cudaEvent_t a, b; ~Ev() { cudaEventDestroy(a); cudaEventDestroy(b); } } ev{e0, e1};
    const double flops = 2.0 * n * (double)n * n;
    launch();
    float bms = 1e30f;
    for (int r = 0; r < reps; ++r) {
        RSD_CUDA_TRY(cudaEventRecord(e0, stream));
        launch();
        RSD_CUDA_TRY(cudaEventRecord(e1, stream));
        RSD_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0;
        RSD_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        bms = std::min(bms, ms);
    }
    // back to back for about `seconds`
    const int loops = std::max(1, (int)(seconds * 1e3 / std::max(bms, 1e-3f)));
    RSD_CUDA_TRY(cudaEventRecord(e0, stream));
    for (int r = 0; r < loops; ++r) launch();
    RSD_CUDA_TRY(cudaEventRecord(e1, stream));
    RSD_CUDA_TRY(cudaEventSynchronize(e1));
    float tms = 0;
    RSD_CUDA_TRY(cudaEventElapsedTime(&tms, e0, e1));
    RSD_CUDA_TRY(cudaGetLastError());
    int errs[4] = {0, 0, 0, 0};
    RSD_CUDA_TRY(cudaMemcpy(errs, err, sizeof(errs), cudaMemcpyDeviceToHost));
    if (errs[ERR_TIMEOUT]) return RSD_ERR_TIMEOUT;
    *best = flops / (bms * 1e-3) / 1e12;
    *sustained = flops * loops / (tms * 1e-3) / 1e12;
    return RSD_OK;
}

// kind 0: inner panel update, 1: panel solve (B = inverted diagonal block),
// 2: U -= X X^T (lower tiles), 3: outer panel update, TC_GENERAL: map indices, alpha and
// rounding taken from the task (128- or 256-wide tiles by the widest N).
int gemm_tc_launch(Handle& h, int /*li*/, const std::vector<GemmTask>& tasks, int kind, cudaStream_t stream,
                   int buf_slot, int max_ctas, int op) {
    TcState* st = state_of(h);
    if (!st || tasks.empty()) return st ? RSD_OK : RSD_ERR_ARG;
    if (buf_slot < 0 || buf_slot >= TC_SLOTS) return RSD_ERR_ARG;
    TcBuf& bf = st->buf[buf_slot];
    const int sms = max_ctas > 0 ? std::min(max_ctas, h.num_sms) : h.num_sms;
    int max_n = 0;
    for (auto& g : tasks) max_n = std::max(max_n, g.N);
    int bn = (kind == 2 || kind == 3 || (kind == TC_GENERAL && max_n > 128)) ? 256 : 128;
    if (op != TC_OP_TF32 && kind != 2 && kind != 3) return RSD_ERR_ARG;     // 16-bit: long-K updates only
    // tuned configuration of the update kinds (0, 2, 3): the tile width (TF32 outer and
    // Schur updates; 16-bit operands run the 128 x 256 kernel only) and the split-K count
    int tuned_split = 0;
    if ((kind == 0 || kind == 2 || kind == 3) && (st->force_bn || !st->tune.empty())) {
        int t256 = 0, maxk = 0;
        for (auto& g : tasks) {
            const int tm = (g.M + BM - 1) / BM, tn = (g.N + 255) / 256;
            t256 += g.lower ? tm * (tn + 1) / 2 : tm * tn;
            maxk = std::max(maxk, g.K);
        }
        int tbn = 0;
        if (st->force_bn) { tbn = st->force_bn; tuned_split = st->force_split; }
        else tune_lookup(st->tune, op == TC_OP_TF32 ? TC_OP_TF32 : TC_OP_F16, t256, maxk, &tbn, &tuned_split);
        if (tbn && kind != 0 && op == TC_OP_TF32) bn = tbn;
    }
    std::vector<TcTask> tt(tasks.size());
    std::vector<std::array<int, 3>> out;            // (task, tm, tn) output tiles
    for (size_t i = 0; i < tasks.size(); ++i) {
        const GemmTask& g = tasks[i];
        TcTask& t = tt[i];
        t.C = (float*)g.C;
        t.ldc = g.ldc; t.M = g.M; t.N = g.N; t.K = g.K;
        t.lower = g.lower; t.beta = g.beta;
        t.map_a = kind == TC_GENERAL ? g.map_a : (op != TC_OP_TF32 ? tc_map_panel16(g.map_a) : tc_map_panel(g.map_a));
        t.map_b = kind == TC_GENERAL ? g.map_b : (kind == 1 ? tc_map_dinv(g.map_b)
                                                            : op != TC_OP_TF32 ? tc_map_panel16(g.map_b) : tc_map_panel(g.map_b));
        t.sa = op != TC_OP_TF32 ? g.sa : nullptr;
        t.sb = op != TC_OP_TF32 ? g.sb : nullptr;
        t.a_r0 = g.a_r0; t.a_c0 = g.a_c0; t.b_r0 = g.b_r0; t.b_c0 = g.b_c0;
        t.alpha = kind == TC_GENERAL ? g.alpha : (kind == 1 ? 1.0f : -1.0f);
        // panel-solve results are final factor entries
        t.round_tf32 = kind == TC_GENERAL ? g.round : (kind == 1);
        const int tm = (g.M + BM - 1) / BM, tn = (g.N + bn - 1) / bn;
        // The persistent kernel runs consecutive tiles at the same time.  Wide outputs
        // (U -= X X^T) are walked in bands of TILE_BAND row blocks, column block by
        // column block, so the tiles in flight share TILE_BAND A row blocks and a run of
        // B row blocks instead of one A row block and up to a wave of distinct B row
        // blocks, each as long as K.
        const int band = tn > 2 ? TILE_BAND : 1;
        for (int a0 = 0; a0 < tm; a0 += band)
            for (int b = 0; b < tn; ++b)
                for (int a = a0; a < std::min(tm, a0 + band); ++a) {
                    if (g.lower && b * bn > a * BM + BM - 1) continue;
                    out.push_back({(int)i, a, b});
                }
    }
    if (out.empty()) return RSD_OK;
    // split K when the output tiles cannot fill the GPU (never for the in-place panel solve)
    const int bke = op != TC_OP_TF32 ? 64 : BK;            // elements per K block
    int max_kb = 0;
    for (auto& g : tasks) max_kb = std::max(max_kb, (g.K + bke - 1) / bke);
    int nsplit = 1;
    if (tuned_split > 0) nsplit = std::max(1, std::min(tuned_split, max_kb / 4));
    else if (kind != 1 && kind != TC_GENERAL && (int)out.size() < sms)
        nsplit = std::max(1, std::min(sms / (int)out.size(), max_kb / SPLIT_MIN_KB));
    if ((int)out.size() * nsplit * (bn / 256 > 0 ? bn / 256 : 1) > st->ws_slots * (256 / bn)) nsplit = 1;
    std::vector<TcTile> tl;
    std::vector<TcRed> rd;
    int slot = 0;
    for (auto& o : out) {
        const int nkb = (tasks[o[0]].K + bke - 1) / bke;
        const int ns = std::max(1, std::min(nsplit, nkb / (tuned_split > 0 ? 4 : SPLIT_MIN_KB)));
        if (ns == 1) {
            tl.push_back({o[0], o[1], o[2], 0, nkb, -1, 0, 0});
            continue;
        }
        rd.push_back({o[0], o[1], o[2], slot, ns, 0, 0, 0});
        for (int sp = 0; sp < ns; ++sp)
            tl.push_back({o[0], o[1], o[2], (int)((int64_t)nkb * sp / ns), (int)((int64_t)nkb * (sp + 1) / ns), slot++, 0, 0});
    }
    double fl = 0, by = 0;
    for (auto& g : tasks) {
        const double c = g.lower ? 0.5 * g.M * (g.M + 1.0) : (double)g.M * g.N;
        fl += 2.0 * c * g.K;
        by += (op != TC_OP_TF32 ? 2.0 : 4.0) * ((double)g.M * g.K + (g.lower ? 0.0 : (double)g.N * g.K)) +
              4.0 * c * (g.beta ? 2 : 1);
    }
    if (st->mode == 1) {                                   // dry pass: record only
        auto put = [&](const void* p, size_t bytes) {
            const size_t o = (st->rec_buf.size() + 255) & ~(size_t)255;
            st->rec_buf.resize(o + bytes);
            if (bytes) std::memcpy(st->rec_buf.data() + o, p, bytes);
            return o;
        };
        TcState::Rec r{};
        r.o_tasks = put(tt.data(), tt.size() * sizeof(TcTask));
        r.o_tiles = put(tl.data(), tl.size() * sizeof(TcTile));
        r.o_reds = put(rd.data(), rd.size() * sizeof(TcRed));
        r.n_tasks = (int)tt.size(); r.n_tiles = (int)tl.size(); r.n_reds = (int)rd.size();
        r.bn = bn; r.max_kb = max_kb; r.fl = fl; r.by = by;
        st->recs.push_back(r);
        return RSD_OK;
    }
    TcTask* d_tasks = nullptr;
    TcTile* d_tiles = nullptr;
    TcRed* d_reds = nullptr;
    if (st->mode == 2) {                                   // real pass: the recorded lists
        if (st->cursor >= st->recs.size()) { set_last_error("recorded launch list exhausted"); return RSD_ERR_ARG; }
        const TcState::Rec& r = st->recs[st->cursor++];
        if (r.n_tasks != (int)tt.size() || r.n_tiles != (int)tl.size() || r.n_reds != (int)rd.size()) {
            set_last_error("recorded launch does not match");
            return RSD_ERR_ARG;
        }
        d_tasks = (TcTask*)(st->d_meta + r.o_tasks);
        d_tiles = (TcTile*)(st->d_meta + r.o_tiles);
        d_reds = (TcRed*)(st->d_meta + r.o_reds);
    }
    auto grow = [&](auto*& ptr, size_t& cap, size_t need, size_t elem) -> int {
        if (need <= cap) return RSD_OK;
        cudaFreeAsync(ptr, stream);
        cap = std::max(need, 2 * cap);
        RSD_CUDA_TRY(cudaMallocAsync((void**)&ptr, cap * elem, stream));
        return RSD_OK;
    };
    if (st->mode == 0) {                                   // direct: upload this launch's lists
        RSD_TRY(grow(bf.d_tasks, bf.cap_tasks, tt.size(), sizeof(TcTask)));
        RSD_TRY(grow(bf.d_tiles, bf.cap_tiles, tl.size(), sizeof(TcTile)));
        if (!rd.empty()) RSD_TRY(grow(bf.d_reds, bf.cap_reds, rd.size(), sizeof(TcRed)));
        d_tasks = bf.d_tasks;
        d_tiles = bf.d_tiles;
        d_reds = bf.d_reds;
        RSD_CUDA_TRY(cudaMemcpyAsync(d_tasks, stage_host(h, tt.data(), tt.size() * sizeof(TcTask)),
                                     tt.size() * sizeof(TcTask), cudaMemcpyHostToDevice, stream));
        RSD_CUDA_TRY(cudaMemcpyAsync(d_tiles, stage_host(h, tl.data(), tl.size() * sizeof(TcTile)),
                                     tl.size() * sizeof(TcTile), cudaMemcpyHostToDevice, stream));
        if (!rd.empty())
            RSD_CUDA_TRY(cudaMemcpyAsync(d_reds, stage_host(h, rd.data(), rd.size() * sizeof(TcRed)),
                                         rd.size() * sizeof(TcRed), cudaMemcpyHostToDevice, stream));
    }
    if (!st->attr_set) {
        RSD_CUDA_TRY(cudaFuncSetAttribute(k_gemm_tc<128, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem<128, 3>::TOTAL));
        RSD_CUDA_TRY(cudaFuncSetAttribute(k_gemm_tc<128, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem<128, 6>::TOTAL));
        RSD_CUDA_TRY(cudaFuncSetAttribute(k_gemm_tc<256, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem<256, 4>::TOTAL));
        RSD_CUDA_TRY(cudaFuncSetAttribute(k_gemm_tc_persist<256, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem<256, 4>::TOTAL));
        RSD_CUDA_TRY(cudaFuncSetAttribute(k_gemm_tc_persist<256, 4, TC_OP_F16>, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem<256, 4>::TOTAL));
        RSD_CUDA_TRY(cudaFuncSetAttribute(k_gemm_tc_persist<256, 4, TC_OP_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem<256, 4>::TOTAL));
        st->attr_set = true;
    }
    const int pi = prof_begin(h, op != TC_OP_TF32 ? K_GEMM_TC16 : K_GEMM_TC, stream);
    // short K (inner panel update, panel solve): 3-stage ring, two CTAs per SM so one
    // tile's epilogue overlaps the other's main loop; long K: deeper rings, one CTA per SM
    if (bn == 128 && max_kb <= 16)
        k_gemm_tc<128, 3><<<(unsigned)tl.size(), TC_THREADS, Smem<128, 3>::TOTAL, stream>>>(d_tasks, d_tiles, st->d_maps, bf.d_ws, h.d_err);
    else if (bn == 128)
        k_gemm_tc<128, 6><<<(unsigned)tl.size(), TC_THREADS, Smem<128, 6>::TOTAL, stream>>>(d_tasks, d_tiles, st->d_maps, bf.d_ws, h.d_err);
    else {
        const int ctas = std::min((int)tl.size(), sms);
        if (op == TC_OP_F16)
            k_gemm_tc_persist<256, 4, TC_OP_F16><<<(unsigned)ctas, TCP_THREADS, Smem<256, 4>::TOTAL, stream>>>(
                d_tasks, d_tiles, (int)tl.size(), st->d_maps, bf.d_ws, h.d_err);
        else if (op == TC_OP_BF16)
            k_gemm_tc_persist<256, 4, TC_OP_BF16><<<(unsigned)ctas, TCP_THREADS, Smem<256, 4>::TOTAL, stream>>>(
                d_tasks, d_tiles, (int)tl.size(), st->d_maps, bf.d_ws, h.d_err);
        else
            k_gemm_tc_persist<256, 4><<<(unsigned)ctas, TCP_THREADS, Smem<256, 4>::TOTAL, stream>>>(
                d_tasks, d_tiles, (int)tl.size(), st->d_maps, bf.d_ws, h.d_err);
    }
    count_launch();
    if (!rd.empty()) {
        const dim3 rg((unsigned)rd.size(), BM / RED_ROWS);
        if (bn == 128) k_splitk_reduce<128><<<rg, 256, 0, stream>>>(d_tasks, d_reds, bf.d_ws);
        else k_splitk_reduce<256><<<rg, 256, 0, stream>>>(d_tasks, d_reds, bf.d_ws);
        count_launch();
    }
    prof_end(h, pi, fl, by, stream);
    RSD_CUDA_TRY(cudaGetLastError());
    return RSD_OK;
}

// ---- autotuner ------------------------------------------------------------------------
// For each operand format (TF32; FP16, which BF16 shares) and each bucket of output tiles
// (1, 4, 16, 64, 256 tiles of 128 x 256) and K (512, 2048, 8192, 24576), time C -= A B^T
// on synthetic operands (one task, M = 128 tiles, N = 256) with the built-in rules and
// with every candidate tile width (TF32: 128 or 256; 16-bit operands: 256) and split-K
// count (1 .. 32 slices of at least 4 K blocks, within the split-K workspace), through the
// same launcher the factorisation uses (best of 3 launches, CUDA events around the GEMM and
// its split-K reduction), and write the fastest per bucket to `path`.
int gemm_tc_autotune(const char* path, cudaStream_t stream, int num_sms, double* secs) {
    const auto t_start = std::chrono::steady_clock::now();
    const int Ts[] = {1, 4, 16, 64, 256};
    const int Ks[] = {512, 2048, 8192, 24576};
    const int Mmax = 256 * BM, Kmax = 24576, Nn = 256;
    const size_t a32 = (size_t)Mmax * Kmax * 4, b32 = (size_t)Nn * Kmax * 4, c32 = (size_t)Mmax * Nn * 4;
    const size_t a16 = a32 / 2, b16 = b32 / 2;
    const size_t o_b = a32, o_c = o_b + b32, o_a16 = o_c + c32, o_b16 = o_a16 + a16, o_one = o_b16 + b16;
    const size_t o_err = o_one + (size_t)Mmax * 4, total = o_err + 256;
    char* buf = nullptr;
    RSD_CUDA_TRY(cudaMalloc((void**)&buf, total));
    struct Free { char* p; ~Free() { cudaFree(p); } } fr{buf};
    float* A = (float*)buf;
    float* B = (float*)(buf + o_b);
    float* Cm = (float*)(buf + o_c);
    k_fill_hash<<<1024, 256, 0, stream>>>(A, (int64_t)Mmax * Kmax, 0x9e3779b9u);
    k_fill_hash<<<1024, 256, 0, stream>>>(B, (int64_t)Nn * Kmax, 0x7f4a7c15u);
    k_to16<<<1024, 256, 0, stream>>>(A, (unsigned short*)(buf + o_a16), (int64_t)Mmax * Kmax, 0);
    k_to16<<<1024, 256, 0, stream>>>(B, (unsigned short*)(buf + o_b16), (int64_t)Nn * Kmax, 0);
    RSD_CUDA_TRY(cudaMemsetAsync(Cm, 0, c32, stream));
    RSD_CUDA_TRY(cudaMemsetAsync(buf + o_err, 0, 256, stream));
    {
        std::vector<float> one((size_t)Mmax, 1.0f);
        RSD_CUDA_TRY(cudaMemcpyAsync(buf + o_one, one.data(), sizeof(float) * Mmax, cudaMemcpyHostToDevice, stream));
        RSD_CUDA_TRY(cudaStreamSynchronize(stream));
    }
    // a stand-alone handle around the synthetic operands: node 0 is A, node 1 is B
    Handle h;
    h.stream = stream;
    h.num_sms = num_sms;
    h.prof.on = true;
    h.d_err = (int*)(buf + o_err);
    auto* st = new TcState();
    h.tc_state = st;
    struct Release { Handle& h; ~Release() { gemm_tc_release(h); stage_release(h); prof_release(h); } } rel{h};
    std::vector<CUtensorMap> maps(2 * TC_NODE_MAPS);
    std::memset(maps.data(), 0, maps.size() * sizeof(CUtensorMap));
    RSD_TRY(encode_2d(&maps[tc_map_panel(0)], A, Kmax, Mmax, Kmax));
    RSD_TRY(encode_2d(&maps[tc_map_panel16(0)], buf + o_a16, Kmax, Mmax, Kmax, TC_OP_F16));
    RSD_TRY(encode_2d(&maps[tc_map_panel(1)], B, Kmax, Nn, Kmax));
    RSD_TRY(encode_2d(&maps[tc_map_panel16(1)], buf + o_b16, Kmax, Nn, Kmax, TC_OP_F16));
    RSD_CUDA_TRY(cudaMalloc((void**)&st->d_maps, maps.size() * sizeof(CUtensorMap)));
    RSD_CUDA_TRY(cudaMemcpy(st->d_maps, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice));
    st->ws_slots = 2 * num_sms;
    for (auto& b : st->buf) RSD_CUDA_TRY(cudaMalloc((void**)&b.d_ws, (size_t)st->ws_slots * BM * 256 * sizeof(float)));
    auto time_one = [&](const GemmTask& t, int op, float* best) -> int {
        *best = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            h.prof.recs.clear();
            RSD_TRY(gemm_tc_launch(h, 0, std::vector<GemmTask>{t}, 3, stream, 0, 0, op));
            RSD_CUDA_TRY(cudaStreamSynchronize(stream));
            float ms = 0;
            const Prof::Rec r = h.prof.recs.back();
            h.prof.recs.clear();                    // its events go back to the pool, once
            for (auto e : {r.a, r.b}) h.prof.pool.push_back(e);
            RSD_CUDA_TRY(cudaEventElapsedTime(&ms, r.a, r.b));
            *best = std::min(*best, ms * 1000.0f);
        }
        return RSD_OK;
    };
    std::vector<TuneEntry> tab;
    for (int op : {TC_OP_TF32, TC_OP_F16}) {
        const int bke = op == TC_OP_TF32 ? BK : 64;
        for (int T : Ts)
            for (int K : Ks) {
                GemmTask t{};
                t.M = T * BM; t.N = Nn; t.K = K;
                t.C = Cm; t.ldc = Nn;
                t.lower = 0; t.beta = 1;
                t.map_a = 0; t.map_b = 1;
                t.sa = (const float*)(buf + o_one);
                t.sb = t.sa;
                st->force_bn = 0;
                float rule = 0;
                RSD_TRY(time_one(t, op, &rule));
                TuneEntry best{op, T, K, 256, 1, 1e30f, rule};
                for (int bn : {256, 128}) {
                    if (op != TC_OP_TF32 && bn != 256) continue;
                    for (int sp : {1, 2, 4, 8, 16, 32}) {
                        if (sp > 1 && sp > K / bke / 4) continue;
                        if (T * (bn == 128 ? 2 : 1) * sp > st->ws_slots * (256 / bn)) continue;
                        st->force_bn = bn;
                        st->force_split = sp;
                        float us = 0;
                        RSD_TRY(time_one(t, op, &us));
                        if (us < best.us) { best.us = us; best.bn = bn; best.split = sp; }
                    }
                }
                st->force_bn = 0;
                tab.push_back(best);
            }
    }
    int errs[ERR_SLOTS];
    RSD_CUDA_TRY(cudaMemcpy(errs, h.d_err, sizeof(errs), cudaMemcpyDeviceToHost));
    if (errs[ERR_TIMEOUT]) return RSD_ERR_TIMEOUT;
    FILE* fp = std::fopen(path, "w");
    if (!fp) { set_last_error(std::string("cannot write tune cache ") + path); return RSD_ERR_ARG; }
    cudaDeviceProp prop{};
    int dev = 0;
    cudaGetDevice(&dev);
    cudaGetDeviceProperties(&prop, dev);
    std::fprintf(fp, "{\"device\": \"%s\", \"sms\": %d, \"entries\": [\n", prop.name, num_sms);
    for (size_t i = 0; i < tab.size(); ++i) {
        const TuneEntry& e = tab[i];
        std::fprintf(fp, "  {\"op\": %d, \"tiles\": %d, \"k\": %d, \"bn\": %d, \"split\": %d, \"us\": %.2f, \"us_rule\": %.2f}%s\n",
                     e.op, e.tiles, e.k, e.bn, e.split, e.us, e.us_rule, i + 1 < tab.size() ? "," : "");
    }
    std::fprintf(fp, "]}\n");
    std::fclose(fp);
    *secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    return RSD_OK;
}

}  // namespace rsd
