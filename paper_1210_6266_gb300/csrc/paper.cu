// Paper mode: Algorithm 2 with the V-hat truncation of Sec. 3.2.  With gamma = 0 the
// interface systems are solved exactly (dense S~, the gamma -> infinity limit of the inner
// solve; this file); with gamma > 0 by gamma GMRES iterations (paper_gamma.cu).
//
// Setup: every leaf l is factored as in exact mode, which also yields its update
// U_l = -K_{B l} K_ll^-1 K_{l B}.  An interface t's front is only its s_t x s_t block
//     S~_t = K[I_t, I_t] + sum over leaves l below t of U_l restricted to I_t x I_t
// (the S-MatVec of Algorithm 1 applied to unit vectors: K_II minus the leaf terms of
// V-hat_t), factored densely.  The entries of U_l that couple two different interfaces
// are dropped: they are what the V-hat truncation leaves out.
//
// Apply (Algorithm 2 taken level by level, bottom-up, as the recursion orders it):
//   v_l = K_ll^-1 r_l for all leaves;
//   for each interface level d from the deepest up:
//     g_t = r_{I_t} - sum_l K_{I_t l} v_l               (coupling to leaf unknowns only)
//     u_t = S~_t^-1 g_t
//     v_l -= K_ll^-1 K_{l I_t} u_t for the leaves coupled to the level's interfaces.
// The result holds u_t on interfaces and the final v_l on leaves.
#include <algorithm>

#include "rsd_internal.cuh"

namespace rsd {
namespace {

// Leaf updates into the interface fronts: U_l(i, j) is added to S~_t when both B_l[i]
// and B_l[j] belong to t.  Leaves that share an interface DOF feed the same entries, so
// the leaves are split into colour classes with no shared DOF (setup) and added class by
// class, one launch per class: within a launch every target has one writer, and every
// entry receives its leaves' terms in a fixed order.
template <typename Tu>
__global__ void k_paper_extend_add(const FrontDesc* __restrict__ leaves, const int* __restrict__ slots,
                                   const NodeRef* __restrict__ refs, const int* __restrict__ owner,
                                   const int* __restrict__ rank) {
    const FrontDesc f = leaves[slots[blockIdx.y]];
    const Tu* U = (const Tu*)f.U;
    for (int i = blockIdx.x; i < f.b; i += gridDim.x) {
        const int gi = f.Bd[i];
        const int oi = owner[gi], ri = rank[gi];
        const NodeRef ref = refs[oi];
        for (int j = threadIdx.x; j <= i; j += blockDim.x) {
            const int gj = f.Bd[j];
            if (owner[gj] != oi) continue;
            const int rj = rank[gj];
            const int r = max(ri, rj), c = min(ri, rj);
            const Tu v = U[(int64_t)i * f.ldu + j];
            if (ref.f64) ((double*)ref.P)[(int64_t)r * ref.ldp + c] += (double)v;
            else ((float*)ref.P)[(int64_t)r * ref.ldp + c] += (float)v;
        }
    }
}

// g_i = r_i - sum over leaf columns K_ij z_j, for the interface rows of one level.
__global__ void k_paper_g(const FrontDesc* __restrict__ fronts, const int64_t* __restrict__ rowptr,
                          const int* __restrict__ col, const double* __restrict__ val,
                          const int* __restrict__ owner, const unsigned char* __restrict__ leaf,
                          const double* __restrict__ r, const double* __restrict__ z, double* __restrict__ g) {
    const FrontDesc f = fronts[blockIdx.y];
    const int lane = threadIdx.x & 31, warps = blockDim.x >> 5;
    for (int p = blockIdx.x * warps + (threadIdx.x >> 5); p < f.s; p += gridDim.x * warps) {
        const int i = f.I[p];
        double s = 0;
        for (int64_t k = rowptr[i] + lane; k < rowptr[i + 1]; k += 32) {
            const int j = col[k];
            if (leaf[owner[j]]) s += val[k] * z[j];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) g[i] = r[i] - s;
    }
}

// w_i = sum over columns owned by depth-d interfaces K_ij z_j, for every leaf row.
__global__ void k_paper_w(const FrontDesc* __restrict__ leaves, const int64_t* __restrict__ rowptr,
                          const int* __restrict__ col, const double* __restrict__ val,
                          const int* __restrict__ owner, const int* __restrict__ node_depth, int d,
                          const double* __restrict__ z, double* __restrict__ w) {
    const FrontDesc f = leaves[blockIdx.y];
    const int lane = threadIdx.x & 31, warps = blockDim.x >> 5;
    for (int p = blockIdx.x * warps + (threadIdx.x >> 5); p < f.s; p += gridDim.x * warps) {
        const int i = f.I[p];
        double s = 0;
        for (int64_t k = rowptr[i] + lane; k < rowptr[i + 1]; k += 32) {
            const int j = col[k];
            if (node_depth[owner[j]] == d) s += val[k] * z[j];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) w[i] = s;
    }
}

// z_i -= c_i on the leaf unknowns.
__global__ void k_paper_sub(const FrontDesc* __restrict__ leaves, const double* __restrict__ c, double* __restrict__ z) {
    const FrontDesc f = leaves[blockIdx.y];
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < f.s; p += gridDim.x * blockDim.x) {
        const int i = f.I[p];
        z[i] -= c[i];
    }
}

}  // namespace

int paper_extend_add(Handle& h) {
    const int dl = (int)h.levels.size() - 1;              // all leaves live on the deepest level
    Level& L = h.levels[dl];
    if (L.fronts.empty() || L.max_b == 0) return RSD_OK;
    const int pi = prof_begin(h, K_EXTEND);
    for (size_t c = 0; c + 1 < h.paper_color_off.size(); ++c) {
        const int n = h.paper_color_off[c + 1] - h.paper_color_off[c];
        if (n == 0) continue;
        const int* slots = h.d_paper_color_slots + h.paper_color_off[c];
        dim3 grid((unsigned)std::max(1, std::min(4096, L.max_b)), (unsigned)n);
        if (is_fp64(L.prec))
            k_paper_extend_add<double><<<grid, 256, 0, h.stream>>>(L.d_fronts, slots, h.d_node_ref, h.d_owner, h.d_rank);
        else
            k_paper_extend_add<float><<<grid, 256, 0, h.stream>>>(L.d_fronts, slots, h.d_node_ref, h.d_owner, h.d_rank);
        count_launch();
        RSD_CUDA_TRY(cudaGetLastError());
    }
    double bytes = 0;
    for (auto& f : L.fronts) bytes += 0.5 * f.b * (f.b + 1.0) * 3.0 * elem_bytes(L.prec);
    prof_end(h, pi, 0.0, bytes);
    RSD_CUDA_TRY(cudaGetLastError());
    return RSD_OK;
}

static int leaf_solve(Handle& h, const double* in, double* out, int*& ticket) {
    const int dl = (int)h.levels.size() - 1;
    Level& L = h.levels[dl];
    const int p1 = prof_begin(h, K_FWD);
    RSD_TRY(sweep_with(h, dl, true, L.d_fronts_solve, L.d_fwd_items_solve, L.n_fwd_items_solve, in, out, ticket++));
    double fl = 0;
    for (auto& f : L.fronts) fl += f.s * (f.s + 1.0);
    const double fb = level_factor_bytes(L, false);
    prof_end(h, p1, fl, fb);
    const int p2 = prof_begin(h, K_BWD);
    RSD_TRY(sweep_with(h, dl, false, L.d_fronts_solve_bwd ? L.d_fronts_solve_bwd : L.d_fronts_solve, L.d_bwd_items,
                       L.n_bwd_items, in, out, ticket++));
    prof_end(h, p2, fl, fb);
    return RSD_OK;
}

int run_apply_paper(Handle& h, const double* r, double* z) {
    const int nl = (int)h.levels.size();
    const int dl = nl - 1;
    Level& Lleaf = h.levels[dl];
    const int n_tickets = 2 + 4 * nl;
    RSD_CUDA_TRY(cudaMemsetAsync(h.d_ticket_paper, 0, sizeof(int) * n_tickets, h.stream));
    int* ticket = h.d_ticket_paper;
    RSD_TRY(leaf_solve(h, r, z, ticket));                 // v_l = K_ll^-1 r_l
    const int nleaf = (int)Lleaf.fronts.size();
    for (int d = dl - 1; d >= 0; --d) {
        Level& L = h.levels[d];
        const int nf = (int)L.fronts.size();
        if (L.max_s == 0) continue;
        // g on the interface rows of level d
        dim3 gg((unsigned)std::max(1, std::min(64, (L.max_s + 7) / 8)), (unsigned)nf);
        k_paper_g<<<gg, 256, 0, h.stream>>>(L.d_fronts_solve, h.d_rowptr, h.d_col, h.d_val, h.d_owner,
                                            h.d_node_leaf, r, z, h.d_pg);
        count_launch();
        RSD_CUDA_TRY(cudaGetLastError());
        // u = S~^-1 g (dense factor) or gamma GMRES iterations on S~ u = g, written into z
        // on the level's interfaces
        if (h.gamma > 0) {
            RSD_TRY(gamma_interface_solve(h, d, z));
        } else {
            RSD_TRY(sweep_with(h, d, true, L.d_fronts_solve, L.d_fwd_items_solve, L.n_fwd_items_solve, h.d_pg, z, ticket++));
            RSD_TRY(sweep_with(h, d, false, L.d_fronts_solve, L.d_bwd_items, L.n_bwd_items, h.d_pg, z, ticket++));
        }
        // leaf corrections
        dim3 gw((unsigned)std::max(1, std::min(64, (Lleaf.max_s + 7) / 8)), (unsigned)nleaf);
        k_paper_w<<<gw, 256, 0, h.stream>>>(Lleaf.d_fronts_solve, h.d_rowptr, h.d_col, h.d_val, h.d_owner,
                                            h.d_node_depth, d, z, h.d_pw);
        count_launch();
        RSD_CUDA_TRY(cudaGetLastError());
        RSD_TRY(leaf_solve(h, h.d_pw, h.d_pz, ticket));
        dim3 gs((unsigned)std::max(1, std::min(64, (Lleaf.max_s + 255) / 256)), (unsigned)nleaf);
        k_paper_sub<<<gs, 256, 0, h.stream>>>(Lleaf.d_fronts_solve, h.d_pz, z);
        count_launch();
        RSD_CUDA_TRY(cudaGetLastError());
    }
    return RSD_OK;
}

}  // namespace rsd
