// Structured-grid FEM problems: assembly of -div(kappa grad u) with trilinear hexahedra on
// the unit cube, the lumped load vector, and the octree decomposition of Sec. 2 (binary
// halving of a strip there; mid-plane octree splits here, as the paper's conclusions
// propose for 3-D).  Row-parallel kernels: each thread builds one CSR row by gathering the
// (up to 8) elements around its node, so no atomics and a deterministic result.
#include "rsd_internal.cuh"

namespace rsd {
namespace {

// 1-D linear-element matrices on the unit interval: stiffness [[1,-1],[-1,1]] and mass
// [[1/3,1/6],[1/6,1/3]].  The trilinear stiffness on the unit cube is the sum of the three
// tensor products with the stiffness factor in one direction.
__device__ __forceinline__ double k1(int a, int b) { return a == b ? 1.0 : -1.0; }
__device__ __forceinline__ double m1(int a, int b) { return a == b ? (1.0 / 3.0) : (1.0 / 6.0); }

__device__ __forceinline__ double khat(int a, int b) {
    int ax = a & 1, ay = (a >> 1) & 1, az = a >> 2;
    int bx = b & 1, by = (b >> 1) & 1, bz = b >> 2;
    return k1(ax, bx) * m1(ay, by) * m1(az, bz) + m1(ax, bx) * k1(ay, by) * m1(az, bz) +
           m1(ax, bx) * m1(ay, by) * k1(az, bz);
}

__device__ __forceinline__ int cnt1(int v, int m) {   // valid offsets of coordinate v in 1..m
    return 3 - (v == 1) - (v == m);
}

__device__ __forceinline__ int64_t prefix1(int v, int m) {   // sum of cnt1 over 1..v-1
    if (v <= 1) return 0;
    return 2 + 3 * (int64_t)(v - 2);
}

__global__ void k_grid_assemble(int n, const double* __restrict__ kappa, int64_t* rowptr,
                                int* col, double* val) {
    const int m = n - 2;
    const int64_t ndof = (int64_t)m * m * m;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= ndof) return;
    const int x = (int)(i % m) + 1, y = (int)((i / m) % m) + 1, z = (int)(i / ((int64_t)m * m)) + 1;
    const int64_t C = (m >= 2) ? 3 * (int64_t)m - 2 : 1;
    const int cx = m >= 2 ? cnt1(x, m) : 1, cy = m >= 2 ? cnt1(y, m) : 1, cz = m >= 2 ? cnt1(z, m) : 1;
    int64_t start = prefix1(z, m) * C * C + cz * (prefix1(y, m) * C + cy * prefix1(x, m));
    if (m < 2) start = 0;
    rowptr[i] = start;
    if (i == ndof - 1) rowptr[ndof] = C * C * C;
    const double h = 1.0 / (n - 1);
    const int ne = n - 1;
    int64_t k = start;
    for (int dz = -1; dz <= 1; ++dz) {
        const int zj = z + dz;
        if (zj < 1 || zj > m) continue;
        for (int dy = -1; dy <= 1; ++dy) {
            const int yj = y + dy;
            if (yj < 1 || yj > m) continue;
            for (int dx = -1; dx <= 1; ++dx) {
                const int xj = x + dx;
                if (xj < 1 || xj > m) continue;
                double v = 0.0;
                // elements with origin (x-1+ax, y-1+ay, z-1+az)
                for (int az = 0; az < 2; ++az) {
                    const int lzi = 1 - az, lzj = lzi + dz;
                    if (lzj < 0 || lzj > 1) continue;
                    for (int ay = 0; ay < 2; ++ay) {
                        const int lyi = 1 - ay, lyj = lyi + dy;
                        if (lyj < 0 || lyj > 1) continue;
                        for (int ax = 0; ax < 2; ++ax) {
                            const int lxi = 1 - ax, lxj = lxi + dx;
                            if (lxj < 0 || lxj > 1) continue;
                            const int64_t e = (x - 1 + ax) + (int64_t)ne * ((y - 1 + ay) + (int64_t)ne * (z - 1 + az));
                            v += kappa[e] * khat(lxi + 2 * lyi + 4 * lzi, lxj + 2 * lyj + 4 * lzj);
                        }
                    }
                }
                col[k] = (xj - 1) + m * ((yj - 1) + m * (zj - 1));
                val[k] = h * v;
                ++k;
            }
        }
    }
}

__global__ void k_grid_load(int64_t ndof, double h3, const double* __restrict__ f, double* b) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < ndof) b[i] = h3 * f[i];
}

__global__ void k_grid_partition(int n, int depth, int* owner) {
    const int m = n - 2;
    const int64_t ndof = (int64_t)m * m * m;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= ndof) return;
    int p[3] = {(int)(i % m) + 1, (int)((i / m) % m) + 1, (int)(i / ((int64_t)m * m)) + 1};
    int lo[3] = {0, 0, 0}, hi[3] = {n - 1, n - 1, n - 1};
    int node = 0;
    for (int level = 0; level < depth; ++level) {
        int mid[3];
        bool on_plane = false;
        for (int d = 0; d < 3; ++d) {
            mid[d] = lo[d] + (hi[d] - lo[d]) / 2;
            on_plane |= (p[d] == mid[d]);
        }
        if (on_plane) { owner[i] = node; return; }
        int c = 0;
        for (int d = 0; d < 3; ++d) {
            if (p[d] > mid[d]) { c |= 1 << d; lo[d] = mid[d]; } else { hi[d] = mid[d]; }
        }
        node = 8 * node + 1 + c;
    }
    owner[i] = node;
}

// kappa_e = exp(m_e): the log-coefficient parametrisation used by the gradient workload.
__global__ void k_grid_exp(int64_t ne3, const double* __restrict__ m, double* __restrict__ kappa) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < ne3) kappa[e] = exp(m[e]);
}

// Adjoint coefficient gradient, one thread per element e: K depends linearly on kappa_e
// through K_e = h Khat (Sec. 4's discretisation), so d(lam^T K u)/dkappa_e = lam_e^T K_e u_e
// and dL/dkappa_e = -lam_e^T K_e u_e when K^T lam = dL/du.  Boundary nodes carry 0.
// Threads of a warp take consecutive ex, so the nodal gathers are coalesced rows.
__global__ void k_grid_coef_grad(int n, const double* __restrict__ u, const double* __restrict__ lam,
                                 const double* __restrict__ kappa, double* __restrict__ dkappa,
                                 double* __restrict__ dm) {
    const int m = n - 2, ne = n - 1;
    const int64_t ne3 = (int64_t)ne * ne * ne;
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= ne3) return;
    const int ex = (int)(e % ne), ey = (int)((e / ne) % ne), ez = (int)(e / ((int64_t)ne * ne));
    double ue[8], le[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const int x = ex + (a & 1), y = ey + ((a >> 1) & 1), z = ez + (a >> 2);
        const bool in = x >= 1 && x <= m && y >= 1 && y <= m && z >= 1 && z <= m;
        const int64_t id = (x - 1) + (int64_t)m * ((y - 1) + (int64_t)m * (z - 1));
        ue[a] = in ? u[id] : 0.0;
        le[a] = in ? lam[id] : 0.0;
    }
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        double w = 0.0;
#pragma unroll
        for (int b = 0; b < 8; ++b) w += khat(a, b) * ue[b];
        s += le[a] * w;
    }
    const double g = -s / (n - 1);                          // h = 1/(n-1)
    if (dkappa) dkappa[e] = g;
    if (dm) dm[e] = kappa[e] * g;
}

// ---- 3-D linear elasticity (three DOFs per node) ------------------------------------
// -div sigma(u) = f, sigma = lam tr(eps) I + 2 mu eps (the SPD Navier-Lame form of Sec. 4's
// Problem 4 in 3-D).  For u = N_b e_q and v = N_a e_p the element bilinear form is
//   int lam d_p N_a d_q N_b + mu (d_q N_a d_p N_b + delta_pq grad N_a . grad N_b),
// and on the unit cube every int d_r N_a d_s N_b is a product of 1-D integrals of the
// linear shape functions: K1 (both derivatives), G1 (one derivative), M1 (none).
__device__ __forceinline__ double g1(int ad, int bd) { return ad ? 0.5 : -0.5; }   // int N_a' N_b

__device__ __forceinline__ double jrs(int r, int s, int a, int b) {
    double v = 1.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int ad = (a >> d) & 1, bd = (b >> d) & 1;
        if (d == r && d == s) v *= k1(ad, bd);
        else if (d == r) v *= g1(ad, bd);
        else if (d == s) v *= g1(bd, ad);
        else v *= m1(ad, bd);
    }
    return v;
}

// Element stiffness entry ((a, p), (b, q)) on the unit cube for E = 1.
__device__ __forceinline__ double khat_el(int a, int p, int b, int q, double lam, double mu) {
    double v = lam * jrs(p, q, a, b) + mu * jrs(q, p, a, b);
    if (p == q) v += mu * (jrs(0, 0, a, b) + jrs(1, 1, a, b) + jrs(2, 2, a, b));
    return v;
}

// Leaf (breadth-first order among the leaves) of element (ex, ey, ez): an element spans
// [e, e + 1] and lies in the lower child of a box [lo, hi] when e < lo + (hi - lo) / 2.
__device__ __forceinline__ int leaf_of_element(int n, int depth, int ex, int ey, int ez) {
    int e[3] = {ex, ey, ez}, lo[3] = {0, 0, 0}, hi[3] = {n - 1, n - 1, n - 1};
    int node = 0;
    for (int level = 0; level < depth; ++level) {
        int c = 0;
        for (int d = 0; d < 3; ++d) {
            const int mid = lo[d] + (hi[d] - lo[d]) / 2;
            if (e[d] >= mid) { c |= 1 << d; lo[d] = mid; } else { hi[d] = mid; }
        }
        node = 8 * node + 1 + c;
    }
    int first = 0, w = 1;
    for (int d = 0; d < depth; ++d) { first += w; w *= 8; }
    return node - first;
}

// One thread per row (node i, component p): the row of the scalar stencil times three
// components, columns 3 j + q ascending; E of each element from its leaf.
__global__ void k_grid_elastic_assemble(int n, int depth, const double* __restrict__ E_leaf, double lam, double mu,
                                        int64_t* rowptr, int* col, double* val) {
    const int m = n - 2;
    const int64_t nn = (int64_t)m * m * m;
    const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (row >= 3 * nn) return;
    const int64_t i = row / 3;
    const int p = (int)(row % 3);
    const int x = (int)(i % m) + 1, y = (int)((i / m) % m) + 1, z = (int)(i / ((int64_t)m * m)) + 1;
    const int64_t C = (m >= 2) ? 3 * (int64_t)m - 2 : 1;
    const int cx = m >= 2 ? cnt1(x, m) : 1, cy = m >= 2 ? cnt1(y, m) : 1, cz = m >= 2 ? cnt1(z, m) : 1;
    int64_t start = prefix1(z, m) * C * C + cz * (prefix1(y, m) * C + cy * prefix1(x, m));
    if (m < 2) start = 0;
    const int64_t cnt = (int64_t)cx * cy * cz;                 // neighbour nodes of i
    const int64_t k0 = 9 * start + 3 * cnt * p;
    rowptr[row] = k0;
    if (row == 3 * nn - 1) rowptr[3 * nn] = 9 * C * C * C;
    // moduli of the 8 elements around node i (origin (x - 1 + ax, ...))
    double Ee[8];
    for (int q = 0; q < 8; ++q)
        Ee[q] = E_leaf[leaf_of_element(n, depth, x - 1 + (q & 1), y - 1 + ((q >> 1) & 1), z - 1 + (q >> 2))];
    const double h = 1.0 / (n - 1);
    int64_t k = k0;
    for (int dz = -1; dz <= 1; ++dz) {
        const int zj = z + dz;
        if (zj < 1 || zj > m) continue;
        for (int dy = -1; dy <= 1; ++dy) {
            const int yj = y + dy;
            if (yj < 1 || yj > m) continue;
            for (int dx = -1; dx <= 1; ++dx) {
                const int xj = x + dx;
                if (xj < 1 || xj > m) continue;
                const int64_t j = (xj - 1) + (int64_t)m * ((yj - 1) + (int64_t)m * (zj - 1));
                for (int q = 0; q < 3; ++q) {
                    double v = 0.0;
                    for (int az = 0; az < 2; ++az) {
                        const int lzi = 1 - az, lzj = lzi + dz;
                        if (lzj < 0 || lzj > 1) continue;
                        for (int ay = 0; ay < 2; ++ay) {
                            const int lyi = 1 - ay, lyj = lyi + dy;
                            if (lyj < 0 || lyj > 1) continue;
                            for (int ax = 0; ax < 2; ++ax) {
                                const int lxi = 1 - ax, lxj = lxi + dx;
                                if (lxj < 0 || lxj > 1) continue;
                                v += Ee[ax + 2 * ay + 4 * az] *
                                     khat_el(lxi + 2 * lyi + 4 * lzi, p, lxj + 2 * lyj + 4 * lzj, q, lam, mu);
                            }
                        }
                    }
                    col[k] = (int)(3 * j + q);
                    val[k] = h * v;
                    ++k;
                }
            }
        }
    }
}

// Owner of DOF c * i + comp: the owner of node i (the octree of k_grid_partition).
__global__ void k_grid_expand_owner(int64_t nn, int ncomp, const int* __restrict__ node_owner, int* __restrict__ dof_owner) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < nn * ncomp) dof_owner[k] = node_owner[k / ncomp];
}

}  // namespace
}  // namespace rsd

using namespace rsd;

extern "C" int rsd_grid_elastic_sizes(int32_t n, int64_t* n_dof, int64_t* nnz) {
    int64_t nd, nz;
    if (!n_dof || !nnz) return RSD_ERR_ARG;
    RSD_TRY(rsd_grid_sizes(n, &nd, &nz));
    if (3 * nd > INT32_MAX) return RSD_ERR_ARG;
    *n_dof = 3 * nd;
    *nnz = 9 * nz;
    return RSD_OK;
}

extern "C" int rsd_grid_elastic_assemble(int32_t n, int32_t depth, const double* E_leaf, double nu,
                                         int64_t* rowptr, int32_t* col, double* val, void* stream) {
    int64_t ndof, nnz;
    RSD_TRY(rsd_grid_elastic_sizes(n, &ndof, &nnz));
    if (depth < 0 || depth > 6 || !E_leaf || !rowptr || !col || !val || !(nu > -1.0 && nu < 0.5)) return RSD_ERR_ARG;
    const double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), mu = 1.0 / (2.0 * (1.0 + nu));   // E = 1
    const int T = 128;
    k_grid_elastic_assemble<<<(unsigned)((ndof + T - 1) / T), T, 0, (cudaStream_t)stream>>>(n, depth, E_leaf, lam, mu,
                                                                                            rowptr, col, val);
    count_launch();
    RSD_CUDA_TRY(cudaGetLastError());
    return RSD_OK;
}

extern "C" int rsd_grid_elastic_partition(int32_t n, int32_t depth, int32_t* dof_node, int32_t* parent,
                                          int32_t* node_scratch, void* stream) {
    int64_t nd, nz;
    RSD_TRY(rsd_grid_sizes(n, &nd, &nz));
    if (!node_scratch || !dof_node) return RSD_ERR_ARG;
    RSD_TRY(rsd_grid_partition(n, depth, node_scratch, parent, stream));
    const int T = 256;
    k_grid_expand_owner<<<(unsigned)((3 * nd + T - 1) / T), T, 0, (cudaStream_t)stream>>>(nd, 3, node_scratch, dof_node);
    count_launch();
    RSD_CUDA_TRY(cudaGetLastError());
    return RSD_OK;
}

extern "C" int rsd_grid_sizes(int32_t n, int64_t* n_dof, int64_t* nnz) {
    if (n < 3 || !n_dof || !nnz) return RSD_ERR_ARG;
    const int64_t m = n - 2;
    if (m * m * m > INT32_MAX) return RSD_ERR_ARG;
    *n_dof = m * m * m;
    const int64_t C = m >= 2 ? 3 * m - 2 : 1;
    *nnz = C * C * C;
    return RSD_OK;
}

extern "C" int rsd_grid_assemble(int32_t n, const double* kappa, int64_t* rowptr, int32_t* col,
                                 double* val, void* stream) {
    int64_t ndof, nnz;
    RSD_TRY(rsd_grid_sizes(n, &ndof, &nnz));
    if (!kappa || !rowptr || !col || !val) return RSD_ERR_ARG;
    const int T = 256;
    k_grid_assemble<<<(unsigned)((ndof + T - 1) / T), T, 0, (cudaStream_t)stream>>>(n, kappa, rowptr, col, val);
    count_launch();
    RSD_CUDA_TRY(cudaGetLastError());
    return RSD_OK;
}

extern "C" int rsd_grid_elastic_load(int32_t n, const double* f, double* b, void* stream) {
    int64_t ndof, nnz;
    RSD_TRY(rsd_grid_elastic_sizes(n, &ndof, &nnz));
    if (!f || !b) return RSD_ERR_ARG;
    const double h = 1.0 / (n - 1);
    const int T = 256;
    k_grid_load<<<(unsigned)((ndof + T - 1) / T), T, 0, (cudaStream_t)stream>>>(ndof, h * h * h, f, b);
    count_launch();
    RSD_CUDA_TRY(cudaGetLastError());
    return RSD_OK;
}

extern "C" int rsd_grid_load(int32_t n, const double* f, double* b, void* stream) {
    int64_t ndof, nnz;
    RSD_TRY(rsd_grid_sizes(n, &ndof, &nnz));
    if (!f || !b) return RSD_ERR_ARG;
    const double h = 1.0 / (n - 1);
    const int T = 256;
    k_grid_load<<<(unsigned)((ndof + T - 1) / T), T, 0, (cudaStream_t)stream>>>(ndof, h * h * h, f, b);
    count_launch();
    RSD_CUDA_TRY(cudaGetLastError());
    return RSD_OK;
}

extern "C" int rsd_grid_partition(int32_t n, int32_t depth, int32_t* dof_node, int32_t* parent,
                                  void* stream) {
    int64_t ndof, nnz;
    RSD_TRY(rsd_grid_sizes(n, &ndof, &nnz));
    if (depth < 0 || depth > 6 || !dof_node || !parent) return RSD_ERR_ARG;
    int64_t n_nodes = 0, w = 1;
    for (int d = 0; d <= depth; ++d) { n_nodes += w; w *= 8; }
    for (int64_t t = 0; t < n_nodes; ++t) parent[t] = t == 0 ? -1 : (int32_t)((t - 1) / 8);
    const int T = 256;
    k_grid_partition<<<(unsigned)((ndof + T - 1) / T), T, 0, (cudaStream_t)stream>>>(n, depth, dof_node);
    count_launch();
    RSD_CUDA_TRY(cudaGetLastError());
    return RSD_OK;
}

extern "C" int rsd_grid_exp(int32_t n, const double* m, double* kappa, void* stream) {
    if (n < 3 || !m || !kappa) return RSD_ERR_ARG;
    const int64_t ne3 = (int64_t)(n - 1) * (n - 1) * (n - 1);
    const int T = 256;
    k_grid_exp<<<(unsigned)((ne3 + T - 1) / T), T, 0, (cudaStream_t)stream>>>(ne3, m, kappa);
    count_launch();
    RSD_CUDA_TRY(cudaGetLastError());
    return RSD_OK;
}

extern "C" int rsd_grid_coef_grad(int32_t n, const double* u, const double* lam, const double* kappa,
                                  double* dkappa, double* dm, void* stream) {
    int64_t ndof, nnz;
    RSD_TRY(rsd_grid_sizes(n, &ndof, &nnz));
    if (!u || !lam || (!dkappa && !dm) || (dm && !kappa)) return RSD_ERR_ARG;
    const int64_t ne3 = (int64_t)(n - 1) * (n - 1) * (n - 1);
    const int T = 256;
    k_grid_coef_grad<<<(unsigned)((ne3 + T - 1) / T), T, 0, (cudaStream_t)stream>>>(n, u, lam, kappa, dkappa, dm);
    count_launch();
    RSD_CUDA_TRY(cudaGetLastError());
    return RSD_OK;
}
