// C ABI entry points and the host-side analysis of the sub-domain hierarchy.
//
// Analysis (integer work, multithreaded C++ on the host):
//   1. the tree of Sec. 2: depth, children, Euler-tour intervals (ancestor tests);
//   2. I_t: the DOFs each node owns, ascending (stable counting sort);
//   3. Eq. 3.1's block structure: every nonzero K_ij couples ancestor-related owners;
//   4. B_t = (adj(I_t) u B_children) restricted to proper ancestors' DOFs, ascending;
//      equivalently the ancestor DOFs adjacent to the subtree of t;
//   5. extend-add maps ea_t: position of each B_t DOF inside the parent's front I_p ++ B_p.
// Numeric setup and every later step run in the CUDA kernels of this library.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <functional>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <thread>

#include <cuda_fp16.h>

#include "rsd_internal.cuh"

namespace rsd {

static thread_local std::string g_last_error;
void set_last_error(const std::string& msg) { g_last_error = msg; }

static std::atomic<long long> g_launches(0);

// One cached arena per device: rsd_destroy parks its arena here instead of freeing it and
// the next rsd_setup on that device reuses it when it is large enough (the arena of a
// factorisation is tens of GB; mapping and unmapping it costs tens of milliseconds).
// rsd_release_cache() returns it to the driver.
struct ArenaCache { char* ptr = nullptr; size_t bytes = 0; };
static std::mutex g_cache_mu;
static ArenaCache g_cache[64];

static char* arena_take(size_t bytes, int dev, size_t* got) {
    {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        ArenaCache& c = g_cache[dev & 63];
        if (c.ptr && c.bytes >= bytes) {
            char* p = c.ptr;
            *got = c.bytes;
            c = ArenaCache{};
            return p;
        }
        if (c.ptr) { cudaFree(c.ptr); c = ArenaCache{}; }   // too small: give it back first
    }
    char* p = nullptr;
    if (cudaMalloc((void**)&p, bytes) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    *got = bytes;
    return p;
}

// Pinned staging blocks (64 MB or more), cached across handles: a handle takes blocks
// as its uploads need them and gives them back when it is destroyed.
static std::mutex g_pin_mu;
static std::vector<std::pair<char*, size_t>> g_pin_free;

static char* pinned_take(size_t bytes, size_t* got) {
    {
        std::lock_guard<std::mutex> lk(g_pin_mu);
        for (size_t i = 0; i < g_pin_free.size(); ++i)
            if (g_pin_free[i].second >= bytes) {
                char* p = g_pin_free[i].first;
                *got = g_pin_free[i].second;
                g_pin_free.erase(g_pin_free.begin() + (int64_t)i);
                return p;
            }
    }
    char* p = nullptr;
    if (cudaMallocHost((void**)&p, bytes) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    *got = bytes;
    return p;
}

static void pinned_give(char* p, size_t bytes) {
    std::lock_guard<std::mutex> lk(g_pin_mu);
    if (g_pin_free.size() >= 4) { cudaFreeHost(p); return; }
    g_pin_free.push_back({p, bytes});
}

// Second one-slot pinned cache: host copies of a device CSR structure for the analysis.
static std::mutex g_pin2_mu;
static char* g_pin2_ptr = nullptr;
static size_t g_pin2_bytes = 0;

static char* pinned2_take(size_t bytes, size_t* got) {
    {
        std::lock_guard<std::mutex> lk(g_pin2_mu);
        if (g_pin2_ptr && g_pin2_bytes >= bytes) {
            char* p = g_pin2_ptr;
            *got = g_pin2_bytes;
            g_pin2_ptr = nullptr;
            g_pin2_bytes = 0;
            return p;
        }
    }
    char* p = nullptr;
    if (cudaMallocHost((void**)&p, bytes) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    *got = bytes;
    return p;
}

static void pinned2_give(char* p, size_t bytes) {
    std::lock_guard<std::mutex> lk(g_pin2_mu);
    if (g_pin2_ptr && g_pin2_bytes >= bytes) { cudaFreeHost(p); return; }
    if (g_pin2_ptr) cudaFreeHost(g_pin2_ptr);
    g_pin2_ptr = p;
    g_pin2_bytes = bytes;
}

const void* stage_host(Handle& h, const void* src, size_t bytes) {
    const size_t need = (bytes + 255) & ~(size_t)255;
    for (;;) {
        if (h.stage_cur < h.stage_blocks.size()) {
            auto& blk = h.stage_blocks[h.stage_cur];
            if (h.stage_off + need <= blk.second) break;
            if (h.stage_cur + 1 < h.stage_blocks.size()) { ++h.stage_cur; h.stage_off = 0; continue; }
        }
        // every block is in use by copies that may still be pending: add one
        size_t got = 0;
        char* p = pinned_take(std::max(need, (size_t)64 << 20), &got);
        if (!p) return src;                            // fall back to a pageable (staged) copy
        h.stage_blocks.push_back({p, got});
        h.stage_cur = h.stage_blocks.size() - 1;
        h.stage_off = 0;
        break;
    }
    char* dst = h.stage_blocks[h.stage_cur].first + h.stage_off;
    std::memcpy(dst, src, bytes);
    h.stage_off += need;
    return dst;
}

void stage_reset(Handle& h) {
    h.stage_cur = 0;
    h.stage_off = 0;
}

void stage_release(Handle& h) {
    if (h.stream) cudaStreamSynchronize(h.stream);
    for (auto& blk : h.stage_blocks) pinned_give(blk.first, blk.second);
    h.stage_blocks.clear();
    stage_reset(h);
}

void prof_release(Handle& h) {
    for (auto& r : h.prof.recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : h.prof.pool) cudaEventDestroy(e);
    h.prof.recs.clear();
    h.prof.pool.clear();
}

static void arena_give(char* p, size_t bytes, int dev) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    ArenaCache& c = g_cache[dev & 63];
    if (c.ptr && c.bytes >= bytes) { cudaFree(p); return; }
    if (c.ptr) cudaFree(c.ptr);
    c.ptr = p;
    c.bytes = bytes;
}
void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int prof_begin(Handle& h, int cls, cudaStream_t stream) {
    if (!h.prof.on) return -1;
    const double host_us = std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now().time_since_epoch()).count();
    Prof::Rec r{cls, 0.0, 0.0, nullptr, nullptr, (h.chain && stream == h.chain) ? 1 : 0, host_us};
    for (cudaEvent_t* e : {&r.a, &r.b}) {
        if (!h.prof.pool.empty()) { *e = h.prof.pool.back(); h.prof.pool.pop_back(); }
        else if (cudaEventCreate(e) != cudaSuccess) { cudaGetLastError(); return -1; }
    }
    cudaEventRecord(r.a, stream);
    h.prof.recs.push_back(r);
    return (int)h.prof.recs.size() - 1;
}

void prof_end(Handle& h, int idx, double flops, double bytes, cudaStream_t stream) {
    if (idx < 0 || idx >= (int)h.prof.recs.size()) return;
    Prof::Rec& r = h.prof.recs[idx];
    r.flops = flops;
    r.bytes = bytes;
    cudaEventRecord(r.b, stream);
}

int pcg(Handle& h, const double* f, double* u, double tol, rsd_stats* st);
int gemm_tc_prepare(Handle& h);     // tensor maps for the tensor-core levels (gemm_tc.cu)
void gemm_tc_release(Handle& h);

namespace {

// Persistent worker pool (created on first use) for the host analysis loops.
class Pool {
public:
    static Pool& get() { static Pool p; return p; }
    int size() const { return (int)workers_.size() + 1; }
    // run fn(i) for i in [0, n) on the pool and the calling thread
    void run(int64_t n, const std::function<void(int64_t)>& fn) {
        std::unique_lock<std::mutex> lk(mu_);
        job_ = &fn;
        n_ = n;
        next_.store(0);
        active_ = (int)workers_.size();
        ++gen_;
        cv_.notify_all();
        lk.unlock();
        for (int64_t i; (i = next_.fetch_add(1)) < n;) fn(i);
        lk.lock();
        done_.wait(lk, [&] { return active_ == 0; });
        job_ = nullptr;
    }
    ~Pool() {
        {
            std::lock_guard<std::mutex> lk(mu_);
            stop_ = true;
            ++gen_;
        }
        cv_.notify_all();
        for (auto& t : workers_) t.join();
    }

private:
    Pool() {
        const int nt = (int)std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
        for (int t = 0; t + 1 < nt; ++t)
            workers_.emplace_back([this] {
                uint64_t seen = 0;
                for (;;) {
                    std::unique_lock<std::mutex> lk(mu_);
                    cv_.wait(lk, [&] { return stop_ || gen_ != seen; });
                    if (stop_) return;
                    seen = gen_;
                    const std::function<void(int64_t)>* fn = job_;
                    const int64_t n = n_;
                    lk.unlock();
                    for (int64_t i; (i = next_.fetch_add(1)) < n;) (*fn)(i);
                    lk.lock();
                    if (--active_ == 0) done_.notify_all();
                }
            });
    }
    std::vector<std::thread> workers_;
    std::mutex mu_;
    std::condition_variable cv_, done_;
    const std::function<void(int64_t)>* job_ = nullptr;
    int64_t n_ = 0;
    std::atomic<int64_t> next_{0};
    int active_ = 0;
    uint64_t gen_ = 0;
    bool stop_ = false;
};

std::mutex g_pool_mu;     // one analysis at a time uses the pool

template <typename F>
void parallel_for(int64_t n, F fn) {
    if (n < 2) {
        for (int64_t i = 0; i < n; ++i) fn(i);
        return;
    }
    std::lock_guard<std::mutex> lk(g_pool_mu);
    const std::function<void(int64_t)> f = fn;
    Pool::get().run(n, f);
}

template <typename F>
void parallel_chunks(int64_t n, F fn) {   // fn(begin, end)
    const int nt = (int)std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    const int64_t chunks = std::min<int64_t>(n, nt * 8);
    if (chunks <= 1) { fn((int64_t)0, n); return; }
    parallel_for(chunks, [&](int64_t c) { fn(n * c / chunks, n * (c + 1) / chunks); });
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
int round_up(int v, int a) { return (v + a - 1) / a * a; }

struct Analysis {
    int n = 0, n_nodes = 0;
    std::vector<int> parent, depth, tin, tout;
    std::vector<std::vector<int>> children;
    std::vector<int> owner, rank;
    std::vector<int> I_off, I_dofs;
    std::vector<std::vector<int>> B, ea;
    int max_depth = 0;
};

int analyse_tree(Analysis& a, const rsd_tree* T) {
    a.n_nodes = T->n_nodes;
    if (a.n_nodes <= 0 || a.n_nodes > (1 << 24) || !T->parent) return RSD_ERR_ARG;
    a.parent.assign(T->parent, T->parent + a.n_nodes);
    if (a.parent[0] != -1) return RSD_ERR_ARG;
    a.children.assign(a.n_nodes, {});
    a.depth.assign(a.n_nodes, 0);
    for (int t = 1; t < a.n_nodes; ++t) {
        const int p = a.parent[t];
        if (p < 0 || p >= t) return RSD_ERR_ARG;
        a.children[p].push_back(t);
        a.depth[t] = a.depth[p] + 1;
        a.max_depth = std::max(a.max_depth, a.depth[t]);
    }
    a.tin.assign(a.n_nodes, 0);
    a.tout.assign(a.n_nodes, 0);
    int clock = 0;
    std::vector<std::pair<int, size_t>> stack{{0, 0}};
    a.tin[0] = clock++;
    while (!stack.empty()) {
        auto& [t, k] = stack.back();
        if (k < a.children[t].size()) {
            const int c = a.children[t][k++];
            a.tin[c] = clock++;
            stack.push_back({c, 0});
        } else {
            a.tout[t] = clock++;
            stack.pop_back();
        }
    }
    return RSD_OK;
}

inline bool anc_or_self(const Analysis& a, int x, int y) {   // x is ancestor-or-self of y
    return a.tin[x] <= a.tin[y] && a.tout[y] <= a.tout[x];
}

// Ownership: validate the owner array and sort the DOFs stably by owner (I_t lists in
// natural order, rank = position within I_t), in parallel over DOF chunks.
int sort_owners(Analysis& a, const int* owner) {
    const int n = a.n;
    a.owner.assign(owner, owner + n);
    for (int i = 0; i < n; ++i)
        if (a.owner[i] < 0 || a.owner[i] >= a.n_nodes) return RSD_ERR_ARG;
    // stable counting sort by owner, in parallel over DOF chunks (per-chunk histograms)
    a.I_off.assign(a.n_nodes + 1, 0);
    a.I_dofs.resize(n);
    a.rank.resize(n);
    {
        const int nc = (int)std::max<int64_t>(1, std::min<int64_t>(32, n / 65536 + 1));
        std::vector<int> cnt((size_t)nc * a.n_nodes, 0);
        parallel_for(nc, [&](int64_t c) {
            int* h = cnt.data() + (size_t)c * a.n_nodes;
            for (int64_t i = n * c / nc; i < n * (c + 1) / nc; ++i) h[a.owner[i]]++;
        });
        for (int t = 0; t < a.n_nodes; ++t) {
            int run = 0;
            for (int c = 0; c < nc; ++c) {
                const int v = cnt[(size_t)c * a.n_nodes + t];
                cnt[(size_t)c * a.n_nodes + t] = run;           // chunk start within node t
                run += v;
            }
            a.I_off[t + 1] = a.I_off[t] + run;
        }
        parallel_for(nc, [&](int64_t c) {
            int* h = cnt.data() + (size_t)c * a.n_nodes;
            for (int64_t i = n * c / nc; i < n * (c + 1) / nc; ++i) {
                const int t = a.owner[i];
                const int r = h[t]++;
                a.rank[i] = r;
                a.I_dofs[a.I_off[t] + r] = (int)i;
            }
        });
    }
    return RSD_OK;
}

// Extend-add maps: position of each of B_c's DOFs in the parent's front (I_p then B_p).
void ea_maps(Analysis& a) {
    a.ea.assign(a.n_nodes, {});
    parallel_for(a.n_nodes, [&](int64_t tt) {
        const int t = (int)tt;
        const int p = a.parent[t];
        if (p < 0) return;
        const int sp = a.I_off[p + 1] - a.I_off[p];
        auto& m = a.ea[t];
        m.resize(a.B[t].size());
        for (size_t k = 0; k < a.B[t].size(); ++k) {
            const int j = a.B[t][k];
            if (a.owner[j] == p) m[k] = a.rank[j];
            else m[k] = sp + (int)(std::lower_bound(a.B[p].begin(), a.B[p].end(), j) - a.B[p].begin());
        }
    });
}

// Host structure pass (CSR in host memory): Eq. 3.1 check and B sets.
int analyse_structure(Analysis& a, const int64_t* rowptr, const int* col, const int* owner, double* part) {
    using clk = std::chrono::steady_clock;
    auto ms_since = [](clk::time_point t) { return std::chrono::duration<double, std::milli>(clk::now() - t).count(); };
    auto t0 = clk::now();
    const int n = a.n;
    if (rowptr[0] != 0) return RSD_ERR_ARG;
    for (int i = 0; i < n; ++i)
        if (rowptr[i + 1] < rowptr[i]) return RSD_ERR_ARG;
    RSD_TRY(sort_owners(a, owner));
    part[0] = ms_since(t0);
    t0 = clk::now();
    // Eq. 3.1: no coupling between owners that are not ancestor-related
    std::atomic<int> bad(0);
    parallel_chunks(n, [&](int64_t b, int64_t e) {
        for (int64_t i = b; i < e && !bad.load(std::memory_order_relaxed); ++i) {
            const int oi = a.owner[i];
            for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
                const int j = col[k];
                if (j < 0 || j >= n) { bad = 2; break; }
                const int oj = a.owner[j];
                if (oi != oj && !anc_or_self(a, oi, oj) && !anc_or_self(a, oj, oi)) { bad = 1; break; }
            }
        }
    });
    if (bad == 2) return RSD_ERR_ARG;
    if (bad == 1) return RSD_ERR_PARTITION;
    part[1] = ms_since(t0);
    t0 = clk::now();
    // B sets, bottom-up by depth, nodes of one depth in parallel
    a.B.assign(a.n_nodes, {});
    std::vector<std::vector<int>> by_depth(a.max_depth + 1);
    for (int t = 0; t < a.n_nodes; ++t) by_depth[a.depth[t]].push_back(t);
    for (int d = a.max_depth; d >= 0; --d) {
        const auto& nodes = by_depth[d];
        parallel_for((int64_t)nodes.size(), [&](int64_t idx) {
            const int t = nodes[idx];
            // one bitmap per proper ancestor, indexed by the DOF's rank in that ancestor
            thread_local std::vector<uint64_t> bits;
            thread_local std::vector<int> anc, base;
            anc.clear();
            base.clear();
            size_t words = 0;
            for (int x = a.parent[t]; x >= 0; x = a.parent[x]) {
                anc.push_back(x);
                base.push_back((int)words);
                words += (size_t)(a.I_off[x + 1] - a.I_off[x] + 63) / 64;
            }
            bits.assign(words, 0);
            auto mark = [&](int j) {
                const int o = a.owner[j];
                for (size_t q = 0; q < anc.size(); ++q)
                    if (anc[q] == o) {
                        const int r = a.rank[j];
                        bits[base[q] + (r >> 6)] |= (uint64_t)1 << (r & 63);
                        return;
                    }
            };
            for (int p = a.I_off[t]; p < a.I_off[t + 1]; ++p) {
                const int i = a.I_dofs[p];
                for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
                    const int o = a.owner[col[k]];
                    if (o != t && anc_or_self(a, o, t)) mark(col[k]);
                }
            }
            for (int c : a.children[t])
                for (int j : a.B[c]) mark(j);
            // each ancestor's list is ascending (I lists are); merge them
            std::vector<int> out;
            for (size_t q = 0; q < anc.size(); ++q) {
                const int x = anc[q];
                const int sx = a.I_off[x + 1] - a.I_off[x];
                const size_t mid = out.size();
                for (int wd = 0; wd < (sx + 63) / 64; ++wd) {
                    uint64_t m = bits[base[q] + wd];
                    while (m) {
                        const int bt = __builtin_ctzll(m);
                        m &= m - 1;
                        out.push_back(a.I_dofs[a.I_off[x] + wd * 64 + bt]);
                    }
                }
                std::inplace_merge(out.begin(), out.begin() + mid, out.end());
            }
            a.B[t] = std::move(out);
        });
    }
    part[2] = ms_since(t0);
    t0 = clk::now();
    ea_maps(a);
    part[3] = ms_since(t0);
    return RSD_OK;
}

// ---- device structure pass (CSR in device memory) ---------------------------------
// Only the ownership array crosses to the host (for the sort); the Eq. 3.1 check and
// the B sets run on the GPU over the CSR, and the sets come back as bitmaps: for every
// node t one bitmap per proper ancestor x (parent first), bit r set when the DOF of rank
// r in I_x belongs to B_t.  A row of t marks the ancestor DOFs it couples to; then,
// level by level from the deepest, every node ORs its bitmaps for the ancestors beyond
// its parent into its parent's (B_parent contains B_child minus I_parent).

enum { SF_ROWPTR = 0, SF_COL, SF_PARTITION, SF_SLOTS };

__global__ void k_struct_mark(int n, int64_t nnz, const int64_t* __restrict__ rowptr, const int* __restrict__ col,
                              const int* __restrict__ owner, const int* __restrict__ rank,
                              const int* __restrict__ tin, const int* __restrict__ tout,
                              const int* __restrict__ depth, const int64_t* __restrict__ anc_word,
                              const int* __restrict__ anc_first, uint32_t* __restrict__ bm, int* __restrict__ flags) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    if (blockIdx.x == 0 && threadIdx.x == 0 && (rowptr[0] != 0 || rowptr[n] != nnz)) flags[SF_ROWPTR] = 1;
    for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
        const int64_t b = rowptr[i], e = rowptr[i + 1];
        if (b < 0 || e < b || e > nnz) { if (lane == 0) flags[SF_ROWPTR] = 1; continue; }
        const int oi = owner[i];
        const int ti = tin[oi], to = tout[oi], di = depth[oi];
        for (int64_t k = b + lane; k < e; k += 32) {
            const int j = col[k];
            if (j < 0 || j >= n) { flags[SF_COL] = 1; continue; }
            const int oj = owner[j];
            if (oj == oi) continue;
            if (tin[oj] <= ti && to <= tout[oj]) {            // oj is a proper ancestor of oi
                const int r = rank[j];
                const int64_t w = anc_word[anc_first[oi] + (di - depth[oj] - 1)] + (r >> 5);
                atomicOr(bm + w, 1u << (r & 31));
            } else if (!(ti <= tin[oj] && tout[oj] <= to)) {
                flags[SF_PARTITION] = 1;                       // neither ancestor nor descendant
            }
        }
    }
}

// bm[parent's words] |= bm[child's words beyond its parent's bitmap], one CTA per child
__global__ void k_struct_up(const int* __restrict__ nodes, const int* __restrict__ parent,
                            const int64_t* __restrict__ anc_word, const int* __restrict__ anc_first,
                            const int64_t* __restrict__ words_total, uint32_t* __restrict__ bm) {
    const int c = nodes[blockIdx.x];
    const int t = parent[c];
    const int64_t n = words_total[t];
    if (n == 0) return;
    const uint32_t* src = bm + anc_word[anc_first[c] + 1];
    uint32_t* dst = bm + anc_word[anc_first[t]];
    for (int64_t w = threadIdx.x; w < n; w += blockDim.x) {
        const uint32_t v = src[w];
        if (v) atomicOr(dst + w, v);
    }
}

int analyse_structure_device(Analysis& a, const rsd_csr* K, const int* d_owner, cudaStream_t st, double* part) {
    using clk = std::chrono::steady_clock;
    auto ms_since = [](clk::time_point t) { return std::chrono::duration<double, std::milli>(clk::now() - t).count(); };
    auto t0 = clk::now();
    const int n = a.n, nn = a.n_nodes;
    // ownership to the host, stable sort there
    size_t pin_bytes = 0;
    char* pin = pinned2_take(sizeof(int) * (size_t)n, &pin_bytes);
    struct PinGuard { char* p; size_t b; ~PinGuard() { if (p) pinned2_give(p, b); } } guard{pin, pin_bytes};
    std::vector<int> own_pageable;
    int* own = (int*)pin;
    if (!own) { own_pageable.resize(n); own = own_pageable.data(); }
    RSD_CUDA_TRY(cudaMemcpyAsync(own, d_owner, sizeof(int) * n, cudaMemcpyDeviceToHost, st));
    RSD_CUDA_TRY(cudaStreamSynchronize(st));
    part[0] = ms_since(t0);
    t0 = clk::now();
    RSD_TRY(sort_owners(a, own));
    // bitmap layout: node t holds depth(t) bitmaps (parent first), words(x) = ceil(s_x / 32)
    std::vector<int> anc_first(nn + 1, 0);
    for (int t = 0; t < nn; ++t) anc_first[t + 1] = anc_first[t] + a.depth[t];
    std::vector<int64_t> anc_word(std::max(1, anc_first[nn])), words_total(nn, 0);
    int64_t W = 0;
    for (int t = 0; t < nn; ++t) {
        int q = 0;
        for (int x = a.parent[t]; x >= 0; x = a.parent[x], ++q) {
            anc_word[anc_first[t] + q] = W;
            const int64_t wx = (a.I_off[x + 1] - a.I_off[x] + 31) / 32;
            W += wx;
            words_total[t] += wx;
        }
    }
    part[1] = ms_since(t0);
    t0 = clk::now();
    // device buffers: rank, tree arrays, layout, bitmaps, flags
    const size_t b_rank = sizeof(int) * n, b_tree = sizeof(int) * nn;
    const size_t b_aw = sizeof(int64_t) * anc_word.size(), b_af = sizeof(int) * (nn + 1);
    const size_t b_wt = sizeof(int64_t) * nn, b_bm = sizeof(uint32_t) * std::max<int64_t>(W, 1);
    auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
    const size_t total = al(b_rank) + 4 * al(b_tree) + al(b_aw) + al(b_af) + al(b_wt) + al(b_bm) + al(sizeof(int) * SF_SLOTS);
    char* dbuf = nullptr;
    RSD_CUDA_TRY(cudaMallocAsync((void**)&dbuf, total, st));
    struct Free { char* p; cudaStream_t s; ~Free() { if (p) cudaFreeAsync(p, s); } } fr{dbuf, st};
    char* cur = dbuf;
    auto take = [&](size_t b) { char* r = cur; cur += al(b); return r; };
    int* d_rank = (int*)take(b_rank);
    int* d_tin = (int*)take(b_tree);
    int* d_tout = (int*)take(b_tree);
    int* d_depth = (int*)take(b_tree);
    int* d_parent = (int*)take(b_tree);
    int64_t* d_aw = (int64_t*)take(b_aw);
    int* d_af = (int*)take(b_af);
    int64_t* d_wt = (int64_t*)take(b_wt);
    uint32_t* d_bm = (uint32_t*)take(b_bm);
    int* d_flags = (int*)take(sizeof(int) * SF_SLOTS);
    std::vector<int> parent_tab(a.parent);
    RSD_CUDA_TRY(cudaMemcpyAsync(d_rank, a.rank.data(), b_rank, cudaMemcpyHostToDevice, st));
    RSD_CUDA_TRY(cudaMemcpyAsync(d_tin, a.tin.data(), b_tree, cudaMemcpyHostToDevice, st));
    RSD_CUDA_TRY(cudaMemcpyAsync(d_tout, a.tout.data(), b_tree, cudaMemcpyHostToDevice, st));
    RSD_CUDA_TRY(cudaMemcpyAsync(d_depth, a.depth.data(), b_tree, cudaMemcpyHostToDevice, st));
    RSD_CUDA_TRY(cudaMemcpyAsync(d_parent, parent_tab.data(), b_tree, cudaMemcpyHostToDevice, st));
    RSD_CUDA_TRY(cudaMemcpyAsync(d_aw, anc_word.data(), b_aw, cudaMemcpyHostToDevice, st));
    RSD_CUDA_TRY(cudaMemcpyAsync(d_af, anc_first.data(), b_af, cudaMemcpyHostToDevice, st));
    RSD_CUDA_TRY(cudaMemcpyAsync(d_wt, words_total.data(), b_wt, cudaMemcpyHostToDevice, st));
    RSD_CUDA_TRY(cudaMemsetAsync(d_bm, 0, b_bm, st));
    RSD_CUDA_TRY(cudaMemsetAsync(d_flags, 0, sizeof(int) * SF_SLOTS, st));
    int sms = 148, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    k_struct_mark<<<(unsigned)(sms * 8), 256, 0, st>>>(n, K->nnz, K->rowptr, K->col, d_owner, d_rank, d_tin, d_tout,
                                                        d_depth, d_aw, d_af, d_bm, d_flags);
    count_launch();
    RSD_CUDA_TRY(cudaGetLastError());
    // propagate level by level, deepest first (children of depth d into depth d-1)
    std::vector<int> nodes_by_depth;
    std::vector<int> doff(a.max_depth + 2, 0);
    for (int t = 0; t < nn; ++t) doff[a.depth[t] + 1]++;
    for (int d = 0; d <= a.max_depth; ++d) doff[d + 1] += doff[d];
    nodes_by_depth.resize(nn);
    {
        std::vector<int> fill(doff.begin(), doff.end() - 1);
        for (int t = 0; t < nn; ++t) nodes_by_depth[fill[a.depth[t]]++] = t;
    }
    int* d_nodes = nullptr;
    RSD_CUDA_TRY(cudaMallocAsync((void**)&d_nodes, sizeof(int) * nn, st));
    struct Free2 { int* p; cudaStream_t s; ~Free2() { if (p) cudaFreeAsync(p, s); } } fr2{d_nodes, st};
    RSD_CUDA_TRY(cudaMemcpyAsync(d_nodes, nodes_by_depth.data(), sizeof(int) * nn, cudaMemcpyHostToDevice, st));
    for (int d = a.max_depth; d >= 2; --d) {
        const int cnt = doff[d + 1] - doff[d];
        if (cnt == 0) continue;
        k_struct_up<<<(unsigned)cnt, 256, 0, st>>>(d_nodes + doff[d], d_parent, d_aw, d_af, d_wt, d_bm);
        count_launch();
        RSD_CUDA_TRY(cudaGetLastError());
    }
    std::vector<uint32_t> bm((size_t)std::max<int64_t>(W, 1));
    int flags[SF_SLOTS];
    RSD_CUDA_TRY(cudaMemcpyAsync(flags, d_flags, sizeof(flags), cudaMemcpyDeviceToHost, st));
    RSD_CUDA_TRY(cudaMemcpyAsync(bm.data(), d_bm, b_bm, cudaMemcpyDeviceToHost, st));
    RSD_CUDA_TRY(cudaStreamSynchronize(st));
    if (flags[SF_ROWPTR] || flags[SF_COL]) return RSD_ERR_ARG;
    if (flags[SF_PARTITION]) return RSD_ERR_PARTITION;
    part[2] = ms_since(t0);
    t0 = clk::now();
    // B lists: each ancestor's bits in rank order are ascending natural ids; merge them
    a.B.assign(nn, {});
    parallel_for(nn, [&](int64_t tt) {
        const int t = (int)tt;
        std::vector<int> out;
        int q = 0;
        for (int x = a.parent[t]; x >= 0; x = a.parent[x], ++q) {
            const int sx = a.I_off[x + 1] - a.I_off[x];
            const uint32_t* bits = bm.data() + anc_word[anc_first[t] + q];
            const size_t mid = out.size();
            for (int wd = 0; wd < (sx + 31) / 32; ++wd) {
                uint32_t m = bits[wd];
                while (m) {
                    const int bt = __builtin_ctz(m);
                    m &= m - 1;
                    out.push_back(a.I_dofs[a.I_off[x] + wd * 32 + bt]);
                }
            }
            std::inplace_merge(out.begin(), out.begin() + mid, out.end());
        }
        a.B[t] = std::move(out);
    });
    part[3] = ms_since(t0);
    t0 = clk::now();
    ea_maps(a);
    part[4] = ms_since(t0);
    return RSD_OK;
}

int level_precision(const rsd_options& o, int depth, bool all_leaves) {
    if (depth == 0) return o.prec_root;
    return all_leaves ? o.prec_leaf : o.prec_mid;
}

bool valid_prec(int p) {
    return p == RSD_PREC_FP64 || p == RSD_PREC_FP32 || p == RSD_PREC_TF32 || p == RSD_PREC_FP16 || p == RSD_PREC_BF16;
}

}  // namespace

// Breakdown handling of the low-precision factorisations (failed pivot: <= 0 or NaN).
// Every front whose pivot failed is factored again one precision up (BF16 / FP16 ->
// TF32 -> FP32 on CUDA cores), and every ancestor, whose front consumed the failed
// front's Schur contribution, again at its own precision; level by level from the
// deepest, each group of one level and precision as a sub-level of those fronts only
// (the other fronts, and the children's contributions, stay as they are).  Repeats while
// pivots fail; a failure in an FP32 or FP64 front is final.
static int promote_failed_fronts(Handle& h, int* d_owner, int* d_rank, int* d_tin, int* d_tout) {
    cudaStream_t st = h.stream;
    const int nl = (int)h.levels.size();
    std::vector<int> node_prec(h.n_nodes);
    for (int t = 0; t < h.n_nodes; ++t) node_prec[t] = h.levels[h.node_level[t]].prec;
    for (int round = 0; round < 4; ++round) {
        std::vector<int> bad(h.n_nodes);
        RSD_CUDA_TRY(cudaStreamSynchronize(st));
        RSD_CUDA_TRY(cudaMemcpy(bad.data(), h.d_front_bad, sizeof(int) * h.n_nodes, cudaMemcpyDeviceToHost));
        std::vector<char> mark(h.n_nodes, 0);
        bool any = false;
        for (int t = 0; t < h.n_nodes; ++t) {
            if (!bad[t]) continue;
            int& p = node_prec[t];
            if (p == RSD_PREC_BF16 || p == RSD_PREC_FP16) p = RSD_PREC_TF32;
            else if (p == RSD_PREC_TF32) p = RSD_PREC_FP32;
            else return RSD_OK;                       // FP32 / FP64 pivot: reported by the caller
            ++h.promoted;
            any = true;
            for (int x = t; x >= 0; x = h.parent[x]) mark[x] = 1;
        }
        if (!any) return RSD_OK;
        const int big = 0x7fffffff;
        RSD_CUDA_TRY(cudaMemsetAsync(h.d_front_bad, 0, sizeof(int) * h.n_nodes, st));
        RSD_CUDA_TRY(cudaMemsetAsync(h.d_err + ERR_NOT_SPD, 0, sizeof(int), st));
        RSD_CUDA_TRY(cudaMemcpyAsync(h.d_err + ERR_NOT_SPD_NODE, &big, sizeof(int), cudaMemcpyHostToDevice, st));
        for (int d = nl - 1; d >= 0; --d) {
            Level& L = h.levels[d];
            std::vector<std::pair<int, std::vector<int>>> groups;     // (precision, slots)
            for (size_t sl = 0; sl < L.nodes.size(); ++sl) {
                const int t = L.nodes[sl];
                if (!mark[t]) continue;
                auto it = std::find_if(groups.begin(), groups.end(), [&](auto& g) { return g.first == node_prec[t]; });
                if (it == groups.end()) groups.push_back({node_prec[t], {(int)sl}});
                else it->second.push_back((int)sl);
            }
            for (auto& [prec, slots] : groups) {
                Level sub;
                sub.depth = L.depth;
                sub.prec = prec;
                sub.h16 = L.h16;                      // the level's sweeps keep reading what they read
                sub.op16 = prec == RSD_PREC_FP16 ? TC_OP_F16 : prec == RSD_PREC_BF16 ? TC_OP_BF16 : TC_OP_TF32;
                sub.d_child_slots = L.d_child_slots;
                for (int sl : slots) {
                    const FrontDesc& f = L.fronts[sl];
                    sub.nodes.push_back(L.nodes[sl]);
                    sub.fronts.push_back(f);
                    sub.max_s = std::max(sub.max_s, f.s);
                    sub.max_b = std::max(sub.max_b, f.b);
                    sub.max_N = std::max(sub.max_N, f.N);
                    sub.max_children = std::max(sub.max_children, f.child_count);
                    const size_t es = elem_bytes(L.prec);
                    RSD_CUDA_TRY(cudaMemsetAsync(f.P, 0, (size_t)f.N * f.ldp * es, st));
                    if (f.b) RSD_CUDA_TRY(cudaMemsetAsync(f.U, 0, (size_t)f.b * f.ldu * es, st));
                }
                RSD_CUDA_TRY(cudaMallocAsync((void**)&sub.d_fronts, sizeof(FrontDesc) * sub.fronts.size(), st));
                RSD_CUDA_TRY(cudaMemcpyAsync(sub.d_fronts, stage_host(h, sub.fronts.data(), sizeof(FrontDesc) * sub.fronts.size()),
                                             sizeof(FrontDesc) * sub.fronts.size(), cudaMemcpyHostToDevice, st));
                std::swap(h.levels[d], sub);
                int rc = launch_assemble_fronts(h, d, h.d_rowptr, h.d_col, h.d_val, d_owner, d_rank, d_tin, d_tout);
                if (rc == RSD_OK) rc = launch_extend_add(h, d);
                if (rc == RSD_OK) rc = run_factor_level(h, d);
                if (rc == RSD_OK) rc = launch_factor_copy16(h, d);
                std::swap(h.levels[d], sub);
                cudaFreeAsync(sub.d_fronts, st);
                RSD_TRY(rc);
            }
        }
    }
    return RSD_OK;
}

// Build the handle's levels, memory plan and device copies from an analysis.
static int build_handle(Handle& h, Analysis& a, const int64_t* rowptr, const int* col, const double* val) {
    const auto t_plan = std::chrono::steady_clock::now();
    h.n = a.n;
    h.n_nodes = a.n_nodes;
    h.parent = a.parent;
    h.depth = a.depth;
    h.I_off = a.I_off;
    h.I_dofs = a.I_dofs;
    h.B_off.assign(a.n_nodes + 1, 0);
    for (int t = 0; t < a.n_nodes; ++t) h.B_off[t + 1] = h.B_off[t] + (int)a.B[t].size();
    h.B_dofs.resize(h.B_off.back());
    for (int t = 0; t < a.n_nodes; ++t) std::copy(a.B[t].begin(), a.B[t].end(), h.B_dofs.begin() + h.B_off[t]);
    std::vector<int> ea_all(h.B_off.back());
    for (int t = 0; t < a.n_nodes; ++t) std::copy(a.ea[t].begin(), a.ea[t].end(), ea_all.begin() + h.B_off[t]);
    // inverse of the extend-add maps: per node t and front position p, the contributions
    // (child index, entry of the child's B) in the order of t's children
    std::vector<int64_t> gp_off(a.n_nodes + 1, 0), gs_off(a.n_nodes + 1, 0);
    for (int t = 0; t < a.n_nodes; ++t) {
        gp_off[t + 1] = gp_off[t] + (a.I_off[t + 1] - a.I_off[t]) + (int64_t)a.B[t].size() + 1;
        int64_t nb = 0;
        for (int c : a.children[t]) nb += (int64_t)a.ea[c].size();
        gs_off[t + 1] = gs_off[t] + nb;
    }
    std::vector<int> gptr_all(gp_off.back());
    std::vector<int2> gsrc_all(std::max<int64_t>(1, gs_off.back()));
    parallel_for(a.n_nodes, [&](int64_t tt) {
        const int t = (int)tt;
        const int Nt = (int)(gp_off[t + 1] - gp_off[t] - 1);
        int* ptr = gptr_all.data() + gp_off[t];
        std::fill(ptr, ptr + Nt + 1, 0);
        for (int c : a.children[t])
            for (int q : a.ea[c]) ++ptr[q + 1];
        for (int q = 0; q < Nt; ++q) ptr[q + 1] += ptr[q];
        std::vector<int> cur(ptr, ptr + Nt);
        int2* src = gsrc_all.data() + gs_off[t];
        int ci = 0;
        for (int c : a.children[t]) {
            const auto& m = a.ea[c];
            for (int i = 0; i < (int)m.size(); ++i) src[cur[m[i]]++] = make_int2(ci, i);
            ++ci;
        }
    });

    const int nl = a.max_depth + 1;
    const bool paper = h.opt.mode == RSD_MODE_PAPER;
    h.paper = paper;
    // paper mode with gamma inner GMRES iterations: only the leaf fronts are stored
    const bool gmode = paper && h.opt.gamma > 0;
    h.gamma = gmode ? h.opt.gamma : 0;
    h.lu = h.opt.nonsymmetric != 0;
    h.krylov = h.opt.krylov == RSD_KRYLOV_AUTO ? ((gmode || h.lu) ? RSD_KRYLOV_FGMRES : RSD_KRYLOV_PCG) : h.opt.krylov;
    h.restart = h.opt.restart > 0 ? h.opt.restart : 30;
    // paper mode keeps only the interface block of internal fronts (V-hat truncation);
    // leaves keep their coupling block, which yields the updates scattered into S~
    auto beff = [&](int t) { return (paper && !a.children[t].empty()) ? 0 : (int)a.B[t].size(); };
    if (paper)
        for (int t = 0; t < a.n_nodes; ++t)
            if (a.children[t].empty() && a.depth[t] != a.max_depth) {
                set_last_error("paper mode needs every leaf on the deepest tree level");
                return RSD_ERR_ARG;
            }
    h.levels.assign(nl, Level{});
    h.node_level.assign(a.n_nodes, 0);
    h.node_slot.assign(a.n_nodes, 0);
    for (int t = 0; t < a.n_nodes; ++t) {
        Level& L = h.levels[a.depth[t]];
        h.node_level[t] = a.depth[t];
        h.node_slot[t] = (int)L.nodes.size();
        L.nodes.push_back(t);
    }
    for (int d = 0; d < nl; ++d) {
        Level& L = h.levels[d];
        L.depth = d;
        bool leaves = true;
        for (int t : L.nodes) leaves &= a.children[t].empty();
        L.prec = level_precision(h.opt, d, leaves);
        if (!valid_prec(L.prec)) return RSD_ERR_ARG;
        L.factored = !(gmode && d < nl - 1);
    }
    // ---- memory plan ----
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t o = off; off = align_up(off + bytes, 1024); return o; };
    const size_t o_rowptr = take(sizeof(int64_t) * (a.n + 1));
    const size_t o_col = take(sizeof(int) * h.nnz);
    const size_t o_val = take(sizeof(double) * h.nnz);
    const size_t o_owner = take(sizeof(int) * a.n);
    const size_t o_rank = take(sizeof(int) * a.n);
    const size_t o_tin = take(sizeof(int) * a.n_nodes);
    const size_t o_tout = take(sizeof(int) * a.n_nodes);
    const size_t o_I = take(sizeof(int) * a.n);
    const size_t o_B = take(sizeof(int) * std::max<size_t>(1, h.B_dofs.size()));
    const size_t o_ea = take(sizeof(int) * std::max<size_t>(1, ea_all.size()));
    const size_t o_gptr = take(sizeof(int) * gptr_all.size());
    const size_t o_gsrc = take(sizeof(int2) * gsrc_all.size());
    const size_t o_flags = take(sizeof(int) * 2 * a.n_nodes);
    struct FrontPlan { size_t P, U, D, V, H, R, PU, DU; };
    std::vector<FrontPlan> fp(a.n_nodes);
    std::vector<size_t> lvlP(nl), lvlU(nl);
    h.factor_elems = 0; h.factor_bytes = 0; h.setup_flops = 0;
    for (int d = nl - 1; d >= 0; --d) {
        Level& L = h.levels[d];
        const size_t es = L.factored ? elem_bytes(L.prec) : 0;   // unfactored: no storage
        // paper mode: the leaves' solves read the copy too (its interface factors S~ are
        // solved from the FP32 panels)
        L.h16 = (L.prec == RSD_PREC_TF32 || L.prec == RSD_PREC_FP16) && (!paper || d == nl - 1);
        L.op16 = L.prec == RSD_PREC_FP16 ? TC_OP_F16 : L.prec == RSD_PREC_BF16 ? TC_OP_BF16 : TC_OP_TF32;
        // P regions of a level are contiguous, then the U regions
        lvlP[d] = off;
        for (int t : L.nodes) {
            const int s = a.I_off[t + 1] - a.I_off[t], b = beff(t);
            const int ldp = std::max(32, round_up(s, 32));
            fp[t].P = take((size_t)(s + b) * ldp * es);
            if (!L.factored) continue;
            h.factor_elems += (int64_t)s * (s + 1) / 2 + (int64_t)s * b;
            h.factor_bytes += ((int64_t)s * (s + 1) / 2 + (int64_t)s * b) * (int64_t)es;
            h.setup_flops += (double)s * s * s / 3.0 + (double)s * s * b + (double)s * b * b;
        }
        if (h.lu)                                    // [U^T; Y^T] panels right after the P panels
            for (int t : L.nodes) {
                const int s = a.I_off[t + 1] - a.I_off[t], b = beff(t);
                const int ldp = std::max(32, round_up(s, 32));
                fp[t].PU = take((size_t)(s + b) * ldp * es);
                if (!L.factored) continue;
                h.factor_elems += (int64_t)s * (s - 1) / 2 + (int64_t)s * b;
                h.factor_bytes += ((int64_t)s * (s - 1) / 2 + (int64_t)s * b) * (int64_t)es;
                h.setup_flops += (double)s * s * s / 3.0 + (double)s * s * b;
            }
        L.bytes_P = off - lvlP[d];
        lvlU[d] = off;
        for (int t : L.nodes) {
            const int b = beff(t);
            const int ldu = std::max(32, round_up(b, 32));
            fp[t].U = take((size_t)b * ldu * es);
        }
        L.bytes_U = off - lvlU[d];
        for (int t : L.nodes) {
            const int s = a.I_off[t + 1] - a.I_off[t], b = beff(t);
            const int nd = (s + NB - 1) / NB;
            fp[t].D = take((size_t)(L.factored ? std::max(1, nd) : 0) * NB * NB * es);
            if (h.lu) fp[t].DU = take((size_t)(L.factored ? std::max(1, nd) : 0) * NB * NB * es);
            fp[t].V = take((size_t)(s + b + 32) * es);
        }
        if (copy16_level(L))                         // 16-bit factor copies after the level's other regions
            for (int t : L.nodes) {
                const int s = a.I_off[t + 1] - a.I_off[t], b = beff(t);
                const int ldp = std::max(32, round_up(s, 32));
                fp[t].H = take((size_t)(s + b) * ldp * 2);
                fp[t].R = take((size_t)2 * (s + b) * sizeof(float));
            }
    }
    const size_t o_fronts = take(sizeof(FrontDesc) * a.n_nodes);
    const size_t o_sfronts = take(sizeof(FrontDesc) * a.n_nodes);
    const size_t o_bfronts = h.lu ? take(sizeof(FrontDesc) * a.n_nodes) : 0;          // backward sweeps
    const size_t o_bsolve = h.lu && paper ? take(sizeof(FrontDesc) * a.n_nodes) : 0;   // backward leaf solves
    size_t n_items = 16;
    for (int t = 0; t < a.n_nodes; ++t) {
        const size_t s = a.I_off[t + 1] - a.I_off[t], b = beff(t);
        n_items += 3 * ((s + NB - 1) / NB) + (b + NB - 1) / NB;
    }
    const size_t o_items = take(sizeof(int) * n_items);
    // paper mode extras
    const size_t o_pvec = paper ? take(sizeof(double) * 3 * (size_t)a.n) : 0;
    const size_t o_nref = paper ? take(sizeof(NodeRef) * a.n_nodes) : 0;
    // paper mode, gamma = 0: colour the leaves so that no two leaves of a class share an
    // interface DOF (greedy, in slot order); their updates are added into S~ class by class
    std::vector<int> color_slots;
    if (paper && !gmode) {
        const Level& Ll = h.levels[nl - 1];
        const int nleaf = (int)Ll.nodes.size();
        std::vector<int> cnt(a.n + 1, 0);
        for (int t : Ll.nodes)
            for (int dof : a.B[t]) cnt[dof + 1]++;
        for (int i = 0; i < a.n; ++i) cnt[i + 1] += cnt[i];
        std::vector<int> lst(cnt[a.n]), fill(cnt.begin(), cnt.end() - 1);
        for (int l = 0; l < nleaf; ++l)
            for (int dof : a.B[Ll.nodes[l]]) lst[fill[dof]++] = l;
        std::vector<int> color(nleaf, 0), stamp;
        int ncol = 0;
        for (int l = 0; l < nleaf; ++l) {
            for (int dof : a.B[Ll.nodes[l]])
                for (int q = cnt[dof]; q < cnt[dof + 1] && lst[q] < l; ++q) {
                    const int c = color[lst[q]];
                    if ((int)stamp.size() <= c) stamp.resize(c + 1, -1);
                    stamp[c] = l;
                }
            int c = 0;
            while (c < (int)stamp.size() && stamp[c] == l) ++c;
            color[l] = c;
            ncol = std::max(ncol, c + 1);
        }
        h.paper_color_off.assign(ncol + 1, 0);
        for (int l = 0; l < nleaf; ++l) h.paper_color_off[color[l] + 1]++;
        for (int c = 0; c < ncol; ++c) h.paper_color_off[c + 1] += h.paper_color_off[c];
        color_slots.resize(nleaf);
        std::vector<int> pos(h.paper_color_off.begin(), h.paper_color_off.end() - 1);
        for (int l = 0; l < nleaf; ++l) color_slots[pos[color[l]]++] = l;
    }
    const size_t o_pcolor = take(sizeof(int) * std::max<size_t>(1, color_slots.size()));
    const size_t o_nleaf = paper ? take(a.n_nodes) : 0;
    const size_t o_ndepth = paper ? take(sizeof(int) * a.n_nodes) : 0;
    const size_t o_fsolve = paper ? take(sizeof(FrontDesc) * a.n_nodes) : 0;
    const size_t o_tpaper = paper ? take(sizeof(int) * (2 + 4 * nl)) : 0;
    // paper mode with gamma > 0: packed interface vectors and leaf couplings per level
    struct GammaHost { std::vector<int> if_off, if_dofs, cl_ptr, cl_row, cl_pos, cl_leaf, ci_ptr, ci_k; double xbytes = 0; };
    std::vector<GammaHost> gh;
    std::vector<int> pk_pos, tl_off;
    size_t o_gamma = 0, gamma_bytes = 0, gm_maxS = 0, gm_maxIf = 0, gm_maxK = 0;
    if (gmode) {
        if (h.gamma > 32) { set_last_error("gamma > 32"); return RSD_ERR_ARG; }
        gh.resize(nl - 1);
        pk_pos.assign(a.n, -1);
        const Level& Ll = h.levels[nl - 1];
        const size_t les = (Ll.op16 == TC_OP_F16 || Ll.h16) && !h.lu ? 2 : elem_bytes(Ll.prec);   // smv_reads_fp16
        for (int d = 0; d < nl - 1; ++d) {
            GammaHost& G = gh[d];
            G.if_off.assign(1, 0);
            for (int t : h.levels[d].nodes) {
                for (int q = a.I_off[t]; q < a.I_off[t + 1]; ++q) {
                    pk_pos[a.I_dofs[q]] = (int)G.if_dofs.size();
                    G.if_dofs.push_back(a.I_dofs[q]);
                }
                G.if_off.push_back((int)G.if_dofs.size());
            }
            gm_maxS = std::max(gm_maxS, G.if_dofs.size());
            gm_maxIf = std::max(gm_maxIf, h.levels[d].nodes.size());
        }
        tl_off.assign(1, 0);
        for (int t : Ll.nodes)                       // slots of 8 elements: vector loads of t_l
            tl_off.push_back(tl_off.back() + round_up(a.I_off[t + 1] - a.I_off[t], 8));
        for (int d = 0; d < nl - 1; ++d) {
            GammaHost& G = gh[d];
            const int S = (int)G.if_dofs.size();
            G.cl_ptr.assign(1, 0);
            std::vector<int> cnt(S + 1, 0);
            for (int t : Ll.nodes) {
                const int sl = a.I_off[t + 1] - a.I_off[t];
                for (size_t r = 0; r < a.B[t].size(); ++r) {
                    const int dof = a.B[t][r];
                    if (a.depth[a.owner[dof]] != d) continue;
                    G.cl_row.push_back((int)r);
                    G.cl_pos.push_back(pk_pos[dof]);
                    G.cl_leaf.push_back((int)(G.cl_ptr.size() - 1));
                    cnt[pk_pos[dof] + 1]++;
                    G.xbytes += 2.0 * sl * (double)les;
                }
                G.cl_ptr.push_back((int)G.cl_row.size());
            }
            for (int p = 0; p < S; ++p) cnt[p + 1] += cnt[p];
            G.ci_ptr = cnt;
            G.ci_k.resize(G.cl_row.size());
            std::vector<int> fill(cnt.begin(), cnt.end() - 1);
            for (size_t k = 0; k < G.cl_row.size(); ++k) G.ci_k[fill[G.cl_pos[k]]++] = (int)k;
            gm_maxK = std::max(gm_maxK, G.cl_row.size());
        }
        size_t gb = 0;
        auto acc = [&](size_t bytes) { gb += align_up(std::max<size_t>(bytes, 4), 256); };
        for (auto& G : gh)
            for (auto* v : {&G.if_off, &G.if_dofs, &G.cl_ptr, &G.cl_row, &G.cl_pos, &G.cl_leaf, &G.ci_ptr, &G.ci_k})
                acc(sizeof(int) * v->size());
        acc(sizeof(int) * pk_pos.size());
        acc(sizeof(int) * tl_off.size());
        acc(sizeof(double) * (size_t)tl_off.back());
        acc(sizeof(double) * gm_maxS);
        acc(sizeof(double) * gm_maxS * (h.gamma + 1));
        acc(sizeof(double) * gm_maxIf * (h.gamma + 1) * h.gamma);
        acc(sizeof(double) * gm_maxIf);
        acc(sizeof(int) * gm_maxIf);
        acc(sizeof(double) * gm_maxK);
        gamma_bytes = gb;
        o_gamma = take(gamma_bytes);
    }
    const bool fg = h.krylov == RSD_KRYLOV_FGMRES;
    const int m = h.restart;
    if (fg && m > 64) { set_last_error("FGMRES restart > 64"); return RSD_ERR_ARG; }
    const size_t o_fg = fg ? take(sizeof(double) * ((size_t)(2 * m + 1) * a.n + (size_t)(m + 1) * m + m + 64)) : 0;
    const size_t o_child = take(sizeof(int) * a.n_nodes);
    const size_t o_vecs = take(sizeof(double) * 4 * (size_t)a.n + 4096);
    const size_t o_partial = take(sizeof(double) * 2048);
    const size_t o_scal = take(sizeof(double) * 16);
    const size_t o_err = take(sizeof(int) * ERR_SLOTS);
    const size_t o_bad = take(sizeof(int) * a.n_nodes);
    const size_t o_ticket = take(sizeof(int) * 2 * nl + 16);
    h.arena_bytes = off;
    {
        int dev = 0;
        cudaGetDevice(&dev);
        h.device = dev;
        size_t got = 0;
        h.arena = arena_take(h.arena_bytes, dev, &got);
        if (!h.arena) {
            set_last_error("device arena of " + std::to_string(h.arena_bytes) + " bytes");
            return RSD_ERR_NOMEM;
        }
        h.arena_capacity = got;
    }
    char* A = h.arena;
    h.d_rowptr = (int64_t*)(A + o_rowptr);
    h.d_col = (int*)(A + o_col);
    h.d_val = (double*)(A + o_val);
    h.d_err = (int*)(A + o_err);
    h.d_front_bad = (int*)(A + o_bad);
    h.d_ticket = (int*)(A + o_ticket);
    h.d_partial = (double*)(A + o_partial);
    h.d_scal = (double*)(A + o_scal);
    double* vecs = (double*)(A + o_vecs);
    h.d_r = vecs; h.d_p = vecs + a.n; h.d_q = vecs + 2 * (size_t)a.n; h.d_z = vecs + 3 * (size_t)a.n;
    int* d_owner = (int*)(A + o_owner);
    int* d_rank = (int*)(A + o_rank);
    int* d_tin = (int*)(A + o_tin);
    int* d_tout = (int*)(A + o_tout);
    int* d_I = (int*)(A + o_I);
    int* d_B = (int*)(A + o_B);
    int* d_ea = (int*)(A + o_ea);
    int* d_gptr = (int*)(A + o_gptr);
    int2* d_gsrc = (int2*)(A + o_gsrc);
    int* d_flags = (int*)(A + o_flags);
    FrontDesc* d_fronts = (FrontDesc*)(A + o_fronts);
    int* d_items = (int*)(A + o_items);
    int* d_child = (int*)(A + o_child);
    cudaStream_t st = h.stream;
    RSD_CUDA_TRY(cudaMemcpyAsync(h.d_rowptr, rowptr, sizeof(int64_t) * (a.n + 1), cudaMemcpyDefault, st));
    RSD_CUDA_TRY(cudaMemcpyAsync(h.d_col, col, sizeof(int) * h.nnz, cudaMemcpyDefault, st));
    RSD_CUDA_TRY(cudaMemcpyAsync(h.d_val, val, sizeof(double) * h.nnz, cudaMemcpyDefault, st));
    RSD_CUDA_TRY(cudaMemcpyAsync(d_owner, stage_host(h, a.owner.data(), sizeof(int) * a.n), sizeof(int) * a.n, cudaMemcpyHostToDevice, st));
    RSD_CUDA_TRY(cudaMemcpyAsync(d_rank, stage_host(h, a.rank.data(), sizeof(int) * a.n), sizeof(int) * a.n, cudaMemcpyHostToDevice, st));
    RSD_CUDA_TRY(cudaMemcpyAsync(d_tin, stage_host(h, a.tin.data(), sizeof(int) * a.n_nodes), sizeof(int) * a.n_nodes, cudaMemcpyHostToDevice, st));
    RSD_CUDA_TRY(cudaMemcpyAsync(d_tout, stage_host(h, a.tout.data(), sizeof(int) * a.n_nodes), sizeof(int) * a.n_nodes, cudaMemcpyHostToDevice, st));
    RSD_CUDA_TRY(cudaMemcpyAsync(d_I, stage_host(h, a.I_dofs.data(), sizeof(int) * a.n), sizeof(int) * a.n, cudaMemcpyHostToDevice, st));
    if (!h.B_dofs.empty()) {
        RSD_CUDA_TRY(cudaMemcpyAsync(d_B, stage_host(h, h.B_dofs.data(), sizeof(int) * h.B_dofs.size()), sizeof(int) * h.B_dofs.size(), cudaMemcpyHostToDevice, st));
        RSD_CUDA_TRY(cudaMemcpyAsync(d_ea, stage_host(h, ea_all.data(), sizeof(int) * ea_all.size()), sizeof(int) * ea_all.size(), cudaMemcpyHostToDevice, st));
    }
    RSD_CUDA_TRY(cudaMemcpyAsync(d_gptr, stage_host(h, gptr_all.data(), sizeof(int) * gptr_all.size()), sizeof(int) * gptr_all.size(), cudaMemcpyHostToDevice, st));
    RSD_CUDA_TRY(cudaMemcpyAsync(d_gsrc, stage_host(h, gsrc_all.data(), sizeof(int2) * gsrc_all.size()), sizeof(int2) * gsrc_all.size(), cudaMemcpyHostToDevice, st));
    RSD_CUDA_TRY(cudaMemsetAsync(h.d_err, 0, sizeof(int) * ERR_SLOTS, st));
    RSD_CUDA_TRY(cudaMemsetAsync(h.d_front_bad, 0, sizeof(int) * a.n_nodes, st));
    {
        const int big = 0x7fffffff;
        RSD_CUDA_TRY(cudaMemcpyAsync(h.d_err + ERR_NOT_SPD_NODE, &big, sizeof(int), cudaMemcpyHostToDevice, st));
    }
    // ---- fronts, child tables, work lists ----
    size_t front_cursor = 0, item_cursor = 0;
    std::vector<int> child_tab;
    std::vector<int> items_all;
    for (int d = 0; d < nl; ++d) {
        Level& L = h.levels[d];
        L.fronts.resize(L.nodes.size());
        L.max_s = L.max_b = L.max_N = 0;
        L.max_children = 0;
        const size_t child_base = child_tab.size();
        for (size_t sidx = 0; sidx < L.nodes.size(); ++sidx) {
            const int t = L.nodes[sidx];
            FrontDesc& f = L.fronts[sidx];
            f.node = t;
            f.s = a.I_off[t + 1] - a.I_off[t];
            f.b = beff(t);
            f.N = f.s + f.b;
            f.ldp = std::max(32, round_up(f.s, 32));
            f.ldu = std::max(32, round_up(f.b, 32));
            f.nd = (f.s + NB - 1) / NB;
            f.parent_slot = a.parent[t] >= 0 ? h.node_slot[a.parent[t]] : -1;
            f.P = A + fp[t].P;
            f.PU = h.lu ? A + fp[t].PU : nullptr;
            f.DinvU = h.lu ? A + fp[t].DU : nullptr;
            f.U = A + fp[t].U;
            f.Dinv = A + fp[t].D;
            f.vec = A + fp[t].V;
            const bool c16 = copy16_level(L);
            f.P16 = c16 ? A + fp[t].H : nullptr;
            f.rs = c16 ? (const float*)(A + fp[t].R) : nullptr;
            f.ri = c16 ? f.rs + f.N : nullptr;
            f.I = d_I + a.I_off[t];
            f.Bd = d_B + h.B_off[t];
            f.ea = d_ea + h.B_off[t];
            f.gptr = d_gptr + gp_off[t];
            f.gsrc = d_gsrc + gs_off[t];
            f.flag = d_flags + 2 * t;
            f.child_begin = (int)(child_tab.size() - child_base);
            f.child_count = (int)a.children[t].size();
            for (int c : a.children[t]) child_tab.push_back(h.node_slot[c]);
            L.max_s = std::max(L.max_s, f.s);
            L.max_b = std::max(L.max_b, f.b);
            L.max_N = std::max(L.max_N, f.N);
            L.max_children = std::max(L.max_children, f.child_count);
        }
        L.d_fronts = d_fronts + front_cursor;
        front_cursor += L.fronts.size();
        L.d_child_slots = d_child + child_base;
        // forward items: key = block index (I blocks, then B blocks), fronts interleaved
        // a diagonal item covers gd consecutive blocks: forward groups start at multiples
        // of gd from the top-left, backward groups are counted from the last block up
        L.cl_sweep = L.h16 && !h.lu && !paper && !L.fronts.empty() &&
                     std::all_of(L.fronts.begin(), L.fronts.end(), [](const FrontDesc& f) { return f.b == 0; });
        const int gd = sweep_item_blocks(L);
        std::vector<std::pair<int, int>> fw, bw;   // (key, item)
        for (size_t sidx = 0; sidx < L.fronts.size(); ++sidx) {
            const FrontDesc& f = L.fronts[sidx];
            const int nbB = (f.b + NB - 1) / NB;
            for (int blk = 0; blk < f.nd; blk += gd) fw.push_back({blk, (int)(sidx << 16) | blk});
            for (int blk = f.nd; blk < f.nd + nbB; ++blk) fw.push_back({blk, (int)(sidx << 16) | blk});
            for (int hi = f.nd - 1; hi >= 0; hi -= gd) bw.push_back({f.nd - 1 - hi, (int)(sidx << 16) | hi});
        }
        std::stable_sort(fw.begin(), fw.end(), [](auto& x, auto& y) { return x.first < y.first; });
        std::stable_sort(bw.begin(), bw.end(), [](auto& x, auto& y) { return x.first < y.first; });
        L.d_fwd_items = d_items + item_cursor;
        L.n_fwd_items = (int)fw.size();
        for (auto& x : fw) items_all.push_back(x.second);
        item_cursor += fw.size();
        L.d_bwd_items = d_items + item_cursor;
        L.n_bwd_items = (int)bw.size();
        for (auto& x : bw) items_all.push_back(x.second);
        item_cursor += bw.size();
        if (paper) {
            std::vector<std::pair<int, int>> fs;
            for (size_t sidx = 0; sidx < L.fronts.size(); ++sidx)
                for (int blk = 0; blk < L.fronts[sidx].nd; blk += gd) fs.push_back({blk, (int)(sidx << 16) | blk});
            std::stable_sort(fs.begin(), fs.end(), [](auto& x, auto& y) { return x.first < y.first; });
            L.d_fwd_items_solve = d_items + item_cursor;
            L.n_fwd_items_solve = (int)fs.size();
            for (auto& x : fs) items_all.push_back(x.second);
            item_cursor += fs.size();
        }
    }
    if (items_all.size() > n_items) { set_last_error("work list overflow"); return RSD_ERR_ARG; }
    for (int d = 0; d < nl; ++d) {
        Level& L = h.levels[d];
        RSD_CUDA_TRY(cudaMemcpyAsync(L.d_fronts, stage_host(h, L.fronts.data(), sizeof(FrontDesc) * L.fronts.size()), sizeof(FrontDesc) * L.fronts.size(), cudaMemcpyHostToDevice, st));
    }
    if (h.lu) {
        // the backward sweeps read [U^T; Y^T] with (U_kk^T)^-1: the same descriptors with
        // P and Dinv exchanged for PU and DinvU
        FrontDesc* d_b = (FrontDesc*)(A + o_bfronts);
        std::vector<FrontDesc> bw;
        for (int d = 0; d < nl; ++d) {
            Level& L = h.levels[d];
            L.d_fronts_bwd = d_b + bw.size();
            for (FrontDesc g : L.fronts) {
                g.P = g.PU;
                g.Dinv = g.DinvU;
                bw.push_back(g);
            }
        }
        RSD_CUDA_TRY(cudaMemcpyAsync(d_b, stage_host(h, bw.data(), sizeof(FrontDesc) * bw.size()), sizeof(FrontDesc) * bw.size(),
                                     cudaMemcpyHostToDevice, st));
    }
    if (!items_all.empty())
        RSD_CUDA_TRY(cudaMemcpyAsync(d_items, stage_host(h, items_all.data(), sizeof(int) * items_all.size()), sizeof(int) * items_all.size(), cudaMemcpyHostToDevice, st));
    if (!child_tab.empty())
        RSD_CUDA_TRY(cudaMemcpyAsync(d_child, stage_host(h, child_tab.data(), sizeof(int) * child_tab.size()), sizeof(int) * child_tab.size(), cudaMemcpyHostToDevice, st));
    RSD_CUDA_TRY(cudaMemsetAsync(d_flags, 0, sizeof(int) * 2 * a.n_nodes, st));
    h.d_owner = d_owner;
    h.d_rank = d_rank;
    if (paper) {
        h.d_pg = (double*)(A + o_pvec);
        h.d_pw = h.d_pg + a.n;
        h.d_pz = h.d_pw + a.n;
        h.d_node_ref = (NodeRef*)(A + o_nref);
        h.d_node_leaf = (unsigned char*)(A + o_nleaf);
        h.d_node_depth = (int*)(A + o_ndepth);
        h.d_ticket_paper = (int*)(A + o_tpaper);
        std::vector<NodeRef> refs(a.n_nodes);
        std::vector<unsigned char> leaf(a.n_nodes);
        std::vector<FrontDesc> solve, solve_b;
        FrontDesc* d_solve = (FrontDesc*)(A + o_fsolve);
        FrontDesc* d_solve_b = h.lu ? (FrontDesc*)(A + o_bsolve) : nullptr;
        for (int d = 0; d < nl; ++d) {
            Level& L = h.levels[d];
            L.d_fronts_solve = d_solve + solve.size();
            if (h.lu) L.d_fronts_solve_bwd = d_solve_b + solve.size();
            for (auto& f : L.fronts) {
                refs[f.node] = NodeRef{f.P, f.ldp, is_fp64(L.prec) ? 1 : 0};
                FrontDesc g = f;
                g.b = 0;
                g.N = g.s;
                g.child_count = 0;
                solve.push_back(g);
                g.P = g.PU;
                g.Dinv = g.DinvU;
                solve_b.push_back(g);
            }
        }
        if (h.lu)
            RSD_CUDA_TRY(cudaMemcpyAsync(d_solve_b, stage_host(h, solve_b.data(), sizeof(FrontDesc) * solve_b.size()),
                                         sizeof(FrontDesc) * solve_b.size(), cudaMemcpyHostToDevice, st));
        for (int t = 0; t < a.n_nodes; ++t) leaf[t] = a.children[t].empty() ? 1 : 0;
        RSD_CUDA_TRY(cudaMemcpyAsync(h.d_node_ref, stage_host(h, refs.data(), sizeof(NodeRef) * refs.size()), sizeof(NodeRef) * refs.size(), cudaMemcpyHostToDevice, st));
        RSD_CUDA_TRY(cudaMemcpyAsync(h.d_node_leaf, stage_host(h, leaf.data(), leaf.size()), leaf.size(), cudaMemcpyHostToDevice, st));
        RSD_CUDA_TRY(cudaMemcpyAsync(h.d_node_depth, stage_host(h, a.depth.data(), sizeof(int) * a.n_nodes), sizeof(int) * a.n_nodes, cudaMemcpyHostToDevice, st));
        RSD_CUDA_TRY(cudaMemcpyAsync(d_solve, stage_host(h, solve.data(), sizeof(FrontDesc) * solve.size()), sizeof(FrontDesc) * solve.size(), cudaMemcpyHostToDevice, st));
        RSD_CUDA_TRY(cudaStreamSynchronize(st));     // host vectors above go out of scope
    }
    if (!color_slots.empty()) {
        h.d_paper_color_slots = (int*)(A + o_pcolor);
        RSD_CUDA_TRY(cudaMemcpyAsync(h.d_paper_color_slots, stage_host(h, color_slots.data(), sizeof(int) * color_slots.size()),
                                     sizeof(int) * color_slots.size(), cudaMemcpyHostToDevice, st));
    }
    if (gmode) {
        char* cur = A + o_gamma;
        auto put = [&](const std::vector<int>& v) -> int* {
            int* d = (int*)cur;
            cur += align_up(std::max<size_t>(sizeof(int) * v.size(), 4), 256);
            return d;
        };
        auto upload = [&](int* d, const std::vector<int>& v) -> int {
            if (!v.empty())
                RSD_CUDA_TRY(cudaMemcpyAsync(d, stage_host(h, v.data(), sizeof(int) * v.size()), sizeof(int) * v.size(),
                                             cudaMemcpyHostToDevice, st));
            return RSD_OK;
        };
        h.gamma_levels.assign(nl - 1, GammaLevel{});
        for (int d = 0; d < nl - 1; ++d) {
            GammaHost& G = gh[d];
            GammaLevel& D = h.gamma_levels[d];
            D.n_if = (int)h.levels[d].nodes.size();
            D.S = (int)G.if_dofs.size();
            D.xbytes = G.xbytes;
            D.nk = (int)G.cl_row.size();
            int** dst[8] = {&D.d_if_off, &D.d_if_dofs, &D.d_cl_ptr, &D.d_cl_row, &D.d_cl_pos, &D.d_cl_leaf, &D.d_ci_ptr, &D.d_ci_k};
            const std::vector<int>* src[8] = {&G.if_off, &G.if_dofs, &G.cl_ptr, &G.cl_row, &G.cl_pos, &G.cl_leaf, &G.ci_ptr, &G.ci_k};
            for (int q = 0; q < 8; ++q) {
                *dst[q] = put(*src[q]);
                RSD_TRY(upload(*dst[q], *src[q]));
            }
        }
        h.d_pk_pos = put(pk_pos);
        RSD_TRY(upload(h.d_pk_pos, pk_pos));
        h.d_tl_off = put(tl_off);
        RSD_TRY(upload(h.d_tl_off, tl_off));
        auto dput = [&](size_t count) {
            double* d = (double*)cur;
            cur += align_up(std::max<size_t>(sizeof(double) * count, 4), 256);
            return d;
        };
        h.d_tl = dput((size_t)tl_off.back());
        h.d_gm_w = dput(gm_maxS);
        h.d_gm_V = dput(gm_maxS * (h.gamma + 1));
        h.d_gm_H = dput(gm_maxIf * (h.gamma + 1) * h.gamma);
        h.d_gm_beta = dput(gm_maxIf);
        h.d_gm_kused = (int*)cur;
        cur += align_up(sizeof(int) * std::max<size_t>(gm_maxIf, 1), 256);
        h.d_gm_yl = dput(gm_maxK);
        if ((size_t)(cur - (A + o_gamma)) > gamma_bytes) { set_last_error("gamma plan overflow"); return RSD_ERR_ARG; }
    }
    if (fg) {
        h.d_fg_V = (double*)(A + o_fg);
        h.d_fg_Z = h.d_fg_V + (size_t)(m + 1) * a.n;
        h.d_fg_H = h.d_fg_Z + (size_t)m * a.n;
        h.d_fg_y = h.d_fg_H + (size_t)(m + 1) * m;
        if (!h.h_fg && cudaMallocHost((void**)&h.h_fg, sizeof(double) * 256) != cudaSuccess) {
            cudaGetLastError();
            return RSD_ERR_NOMEM;
        }
    }
    RSD_TRY(static_apply_prepare(h, (FrontDesc*)(A + o_sfronts)));
    // the tensor-core levels need tensor maps over the fronts just placed
    RSD_TRY(gemm_tc_prepare(h));
    h.prof.host_part[5] = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_plan).count();
    // ---- numeric setup, deepest level first ----
    // Every level's fronts (disjoint arena regions) are zeroed and receive their K entries
    // up front, leaves first: the device does this while the host plans the leaf level.
    for (int d = nl - 1; d >= 0; --d) {
        if (!h.levels[d].factored) continue;
        RSD_TRY(launch_zero_fronts(h, d));
        if (h.lu) RSD_TRY(launch_assemble_fronts_lu(h, d, h.d_rowptr, h.d_col, h.d_val, d_owner, d_rank, d_tin, d_tout));
        else RSD_TRY(launch_assemble_fronts(h, d, h.d_rowptr, h.d_col, h.d_val, d_owner, d_rank, d_tin, d_tout));
    }
    if (!paper) {
        const auto t_issue = std::chrono::steady_clock::now();
        for (int d = nl - 1; d >= 0; --d) {
            if (h.lu) {
                RSD_TRY(launch_extend_add_lu(h, d));
                RSD_TRY(run_factor_level_lu(h, d));
                continue;
            }
            RSD_TRY(launch_extend_add(h, d));
            RSD_TRY(run_factor_level(h, d));
            RSD_TRY(launch_factor_copy16(h, d));
        }
        h.prof.host_issue_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_issue).count();
    } else {
        // every interface front is K_II plus leaf updates: factor the leaves, scatter
        // their updates into S~, then factor the interfaces
        RSD_TRY(h.lu ? run_factor_level_lu(h, nl - 1) : run_factor_level(h, nl - 1));
        if (!h.lu) RSD_TRY(launch_factor_copy16(h, nl - 1));   // TF32 leaves: the copy their solves read
        if (!gmode) {
            RSD_TRY(paper_extend_add(h));
            for (int d = nl - 2; d >= 0; --d) RSD_TRY(run_factor_level(h, d));
        }
    }
    RSD_CUDA_TRY(cudaStreamSynchronize(st));
    stage_reset(h);                                   // every staged upload has completed
    int err[ERR_SLOTS];
    RSD_CUDA_TRY(cudaMemcpy(err, h.d_err, sizeof(err), cudaMemcpyDeviceToHost));
    if (err[ERR_NOT_SPD] && !paper && !h.lu) {
        RSD_TRY(promote_failed_fronts(h, d_owner, d_rank, d_tin, d_tout));
        RSD_CUDA_TRY(cudaStreamSynchronize(st));
        stage_reset(h);
        RSD_CUDA_TRY(cudaMemcpy(err, h.d_err, sizeof(err), cudaMemcpyDeviceToHost));
    }
    if (err[ERR_NOT_SPD]) {
        h.notspd_node = err[ERR_NOT_SPD_NODE];
        set_last_error("pivot <= 0 in node " + std::to_string(h.notspd_node));
        return RSD_ERR_NOT_SPD;
    }
    return RSD_OK;
}

}  // namespace rsd

using namespace rsd;

struct rsd_handle_s {
    Handle h;
};

extern "C" const char* rsd_strerror(int code) {
    switch (code) {
        case RSD_OK: return "ok";
        case RSD_ERR_ARG: return "invalid argument";
        case RSD_ERR_PARTITION: return "matrix couples sub-domains that are not ancestor-related (Eq. 3.1 violated)";
        case RSD_ERR_NOT_SPD: return "non-positive pivot in a factorisation";
        case RSD_ERR_NOMEM: return "out of memory";
        case RSD_ERR_CUDA: return "CUDA error";
        case RSD_ERR_TIMEOUT: return "bounded device wait timed out";
        case RSD_ERR_NOCONV: return "Krylov solve did not converge within maxit";
        default: return "unknown error";
    }
}

extern "C" const char* rsd_last_error_detail(void) { return g_last_error.c_str(); }

extern "C" int64_t rsd_launch_count(void) { return (int64_t)g_launches.load(); }

extern "C" void rsd_release_cache(void) {
    {
        std::lock_guard<std::mutex> lk(g_pin2_mu);
        if (g_pin2_ptr) cudaFreeHost(g_pin2_ptr);
        g_pin2_ptr = nullptr;
        g_pin2_bytes = 0;
    }
    {
        std::lock_guard<std::mutex> lk(g_pin_mu);
        for (auto& blk : g_pin_free) cudaFreeHost(blk.first);
        g_pin_free.clear();
    }
    std::lock_guard<std::mutex> lk(g_cache_mu);
    int cur = 0;
    cudaGetDevice(&cur);
    for (int d = 0; d < 64; ++d) {
        if (!g_cache[d].ptr) continue;
        cudaSetDevice(d);
        cudaFree(g_cache[d].ptr);
        g_cache[d] = ArenaCache{};
    }
    cudaSetDevice(cur);
}

static_assert(K_CLASSES == RSD_PROFILE_CLASSES, "profile classes of the ABI and the kernels differ");

extern "C" int rsd_profile(rsd_handle hh, rsd_profile_t* out, int32_t reset) {
    if (!hh || !out) return RSD_ERR_ARG;
    Handle& h = hh->h;
    std::memset(out, 0, sizeof(*out));
    RSD_CUDA_TRY(cudaStreamSynchronize(h.stream));
    for (auto& r : h.prof.recs) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) { cudaGetLastError(); ms = 0; }
        out->launches[r.cls] += 1;
        out->ms[r.cls] += ms;
        out->flops[r.cls] += r.flops;
        out->bytes[r.cls] += r.bytes;
    }
    out->host_analysis_ms = h.prof.host_ms + h.prof.host_part[5];
    for (int i = 0; i < 6; ++i) out->host_parts_ms[i] = h.prof.host_part[i];
    out->host_issue_ms = h.prof.host_issue_ms;
    if (reset) {
        for (auto& r : h.prof.recs) { h.prof.pool.push_back(r.a); h.prof.pool.push_back(r.b); }
        h.prof.recs.clear();
    }
    return RSD_OK;
}

extern "C" int rsd_profile_trace(rsd_handle hh, rsd_trace_rec* out, int64_t cap, int64_t* n) {
    if (!hh || !n || cap < 0 || (cap > 0 && !out)) return RSD_ERR_ARG;
    Handle& h = hh->h;
    RSD_CUDA_TRY(cudaStreamSynchronize(h.stream));
    if (h.chain) RSD_CUDA_TRY(cudaStreamSynchronize(h.chain));
    *n = (int64_t)h.prof.recs.size();
    for (int64_t i = 0; i < std::min(cap, *n); ++i) {
        const Prof::Rec& r = h.prof.recs[i];
        float t0 = 0, t1 = 0;
        if (cudaEventElapsedTime(&t0, h.prof.recs[0].a, r.a) != cudaSuccess) { cudaGetLastError(); t0 = 0; }
        if (cudaEventElapsedTime(&t1, h.prof.recs[0].a, r.b) != cudaSuccess) { cudaGetLastError(); t1 = 0; }
        out[i] = rsd_trace_rec{r.cls, r.stream, t0, t1, r.flops, r.bytes,
                               (r.host_us - h.prof.recs[0].host_us) / 1000.0};
    }
    return RSD_OK;
}

extern "C" void rsd_destroy(rsd_handle hh) {
    if (!hh) return;
    Handle& h = hh->h;
    if (h.stream) cudaStreamSynchronize(h.stream);
    if (h.chain) {
        cudaStreamSynchronize(h.chain);
        cudaStreamDestroy(h.chain);
    }
    for (cudaEvent_t e : {h.ev_ready, h.ev_join, h.ev_diag[0], h.ev_diag[1], h.ev_diag[2], h.ev_diag[3]})
        if (e) cudaEventDestroy(e);
    if (h.apply_exec) cudaGraphExecDestroy(h.apply_exec);
    gemm_tc_release(h);
    for (auto& r : h.prof.recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : h.prof.pool) cudaEventDestroy(e);
    if (h.arena) arena_give(h.arena, h.arena_capacity, h.device);
    for (auto& blk : h.stage_blocks) pinned_give(blk.first, blk.second);
    if (h.h_scal) cudaFreeHost(h.h_scal);
    if (h.h_fg) cudaFreeHost(h.h_fg);
    delete hh;
}

extern "C" int rsd_setup(const rsd_csr* K, const int32_t* dof_node, const rsd_tree* T,
                         const rsd_options* opt, rsd_handle* out) {
    if (!K || !dof_node || !T || !out || K->n <= 0 || K->nnz <= 0 || !K->rowptr || !K->col || !K->val)
        return RSD_ERR_ARG;
    if (K->mem != RSD_MEM_HOST && K->mem != RSD_MEM_DEVICE) return RSD_ERR_ARG;
    *out = nullptr;
    rsd_options o{};
    o.mode = RSD_MODE_EXACT;
    o.prec_leaf = RSD_PREC_TF32;
    o.prec_mid = RSD_PREC_TF32;
    o.prec_root = RSD_PREC_FP64;
    o.maxit = 200;
    if (opt) o = *opt;
    if (o.mode != RSD_MODE_EXACT && o.mode != RSD_MODE_PAPER) return RSD_ERR_ARG;
    if (o.gamma < 0 || (o.gamma > 0 && o.mode != RSD_MODE_PAPER)) return RSD_ERR_ARG;
    if (o.krylov < RSD_KRYLOV_AUTO || o.krylov > RSD_KRYLOV_FGMRES) return RSD_ERR_ARG;
    if (o.nonsymmetric) {
        const int ps[3] = {o.prec_leaf, o.prec_mid, o.prec_root};
        for (int p : ps)
            if (p != RSD_PREC_FP64 && p != RSD_PREC_FP32) {
                set_last_error("nonsymmetric fronts (LU) are factored in FP64 or FP32 on CUDA cores");
                return RSD_ERR_ARG;
            }
        if (o.krylov == RSD_KRYLOV_PCG || (o.mode == RSD_MODE_PAPER && o.gamma == 0)) {
            set_last_error("nonsymmetric K: FGMRES only, and paper mode needs gamma > 0");
            return RSD_ERR_ARG;
        }
    }
    if (o.krylov == RSD_KRYLOV_PCG && o.gamma > 0) {
        set_last_error("PCG needs a fixed preconditioner: gamma > 0 makes it change with its input");
        return RSD_ERR_ARG;
    }
    const auto t_host0 = std::chrono::steady_clock::now();
    Analysis a;
    a.n = K->n;
    RSD_TRY(analyse_tree(a, T));
    cudaStream_t st = (cudaStream_t)o.stream;
    using clk = std::chrono::steady_clock;
    auto ms_since = [](clk::time_point t) { return std::chrono::duration<double, std::milli>(clk::now() - t).count(); };
    double part[6] = {0, 0, 0, 0, 0, 0};
    // A host CSR is uploaded first when a device is present, so that the structure pass
    // runs on the GPU too (the handle copies the uploaded structure, not the host one);
    // without a device the host pass checks it.  Its values follow once the structure pass
    // is done, while the host plans the hierarchy (the device is idle then), so that the
    // handle copies them device to device.
    const int64_t* rowptr_src = K->rowptr;
    const int* col_src = K->col;
    const double* val_src = K->val;
    struct Tmp { char* p = nullptr; cudaStream_t s = nullptr; ~Tmp() { if (p) cudaFreeAsync(p, s); } } tmp;
    int ndev = 0;
    if (K->mem == RSD_MEM_HOST && (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0)) { cudaGetLastError(); ndev = 0; }
    if (K->mem == RSD_MEM_DEVICE) {
        RSD_TRY(analyse_structure_device(a, K, dof_node, st, part));
    } else if (ndev > 0) {
        const auto t0 = clk::now();
        if (K->rowptr[0] != 0 || K->rowptr[K->n] != K->nnz) return RSD_ERR_ARG;
        const size_t b_rp = sizeof(int64_t) * ((size_t)K->n + 1), b_cl = sizeof(int) * (size_t)K->nnz;
        const size_t b_ow = sizeof(int) * (size_t)K->n, b_vl = sizeof(double) * (size_t)K->nnz;
        const size_t o_cl = (b_rp + 255) & ~(size_t)255, o_ow = (o_cl + b_cl + 255) & ~(size_t)255;
        const size_t o_vl = (o_ow + b_ow + 255) & ~(size_t)255;
        RSD_CUDA_TRY(cudaMallocAsync((void**)&tmp.p, o_vl + b_vl, st));
        tmp.s = st;
        RSD_CUDA_TRY(cudaMemcpyAsync(tmp.p, K->rowptr, b_rp, cudaMemcpyHostToDevice, st));
        RSD_CUDA_TRY(cudaMemcpyAsync(tmp.p + o_cl, K->col, b_cl, cudaMemcpyHostToDevice, st));
        RSD_CUDA_TRY(cudaMemcpyAsync(tmp.p + o_ow, dof_node, b_ow, cudaMemcpyHostToDevice, st));
        rsd_csr Kd = *K;
        Kd.rowptr = (const int64_t*)tmp.p;
        Kd.col = (const int*)(tmp.p + o_cl);
        Kd.mem = RSD_MEM_DEVICE;
        rowptr_src = Kd.rowptr;
        col_src = Kd.col;
        const double up = ms_since(t0);
        RSD_TRY(analyse_structure_device(a, &Kd, (const int*)(tmp.p + o_ow), st, part));
        part[0] += up;
        RSD_CUDA_TRY(cudaMemcpyAsync(tmp.p + o_vl, K->val, b_vl, cudaMemcpyHostToDevice, st));
        val_src = (const double*)(tmp.p + o_vl);
    } else {
        const auto t0 = clk::now();
        if (K->rowptr[K->n] != K->nnz) return RSD_ERR_ARG;
        part[0] = ms_since(t0);
        RSD_TRY(analyse_structure(a, K->rowptr, K->col, dof_node, part + 1));
    }
    auto* hh = new (std::nothrow) rsd_handle_s();
    if (!hh) return RSD_ERR_NOMEM;
    Handle& h = hh->h;
    h.opt = o;
    h.stream = st;
    if (o.wait_cycles > 0) h.wait_cycles = o.wait_cycles;
    h.prof.on = o.profile != 0;
    for (int i = 0; i < 5; ++i) h.prof.host_part[i] = part[i];
    h.prof.host_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_host0).count();
    h.nnz = K->nnz;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&h.num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaMallocHost((void**)&h.h_scal, sizeof(double) * 16) != cudaSuccess) {
        cudaGetLastError();
        delete hh;
        return RSD_ERR_NOMEM;
    }
    // numeric values come from the caller's memory directly (device or host)
    const int rc = build_handle(h, a, rowptr_src, col_src, val_src);
    if (rc != RSD_OK) {
        h.notspd_node = h.notspd_node;
        if (rc == RSD_ERR_NOT_SPD) { *out = hh; return rc; }   // handle kept for introspection
        rsd_destroy(hh);
        return rc;
    }
    *out = hh;
    return RSD_OK;
}

extern "C" int rsd_apply(rsd_handle hh, const double* r, double* z) {
    if (!hh || !r || !z || r == z) return RSD_ERR_ARG;
    return hh->h.paper ? run_apply_paper(hh->h, r, z) : run_apply(hh->h, r, z);
}

extern "C" int rsd_apply_static(rsd_handle hh, const double* r, double* z) {
    if (!hh || !r || !z || r == z || hh->h.paper) return RSD_ERR_ARG;
    return run_apply_static(hh->h, r, z);
}

extern "C" int rsd_peak_gemm(int32_t prec, int32_t n, int32_t reps, double seconds, void* stream,
                             double* best_tflops, double* sustained_tflops) {
    if (!best_tflops || !sustained_tflops || reps < 1 || !(seconds >= 0)) return RSD_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == RSD_PREC_TF32 || prec == RSD_PREC_FP16 || prec == RSD_PREC_BF16) {
        int dev = 0, sms = 148;
        RSD_CUDA_TRY(cudaGetDevice(&dev));
        RSD_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const int op = prec == RSD_PREC_FP16 ? TC_OP_F16 : prec == RSD_PREC_BF16 ? TC_OP_BF16 : TC_OP_TF32;
        return gemm_tc_peak(n, reps, seconds, st, sms, best_tflops, sustained_tflops, op);
    }
    return gemm_simt_peak(prec, n, reps, seconds, st, best_tflops, sustained_tflops);
}

extern "C" int rsd_inject_drop_sweep_item(rsd_handle hh, int32_t level) {
    if (!hh || hh->h.paper || level < 0 || level >= (int)hh->h.levels.size()) return RSD_ERR_ARG;
    hh->h.inject_drop_level = level;
    return RSD_OK;
}

extern "C" int rsd_autotune(const char* path, double* seconds, void* stream) {
    if (!path || !seconds) return RSD_ERR_ARG;
    int dev = 0, sms = 148;
    RSD_CUDA_TRY(cudaGetDevice(&dev));
    RSD_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    return gemm_tc_autotune(path, (cudaStream_t)stream, sms, seconds);
}

extern "C" int rsd_tune_load(const char* path, int32_t* entries) {
    if (!path || !entries) return RSD_ERR_ARG;
    return tune_read(path, nullptr, entries);
}

extern "C" int rsd_check(rsd_handle hh) {
    if (!hh) return RSD_ERR_ARG;
    Handle& h = hh->h;
    RSD_CUDA_TRY(cudaStreamSynchronize(h.stream));
    int err[ERR_SLOTS];
    RSD_CUDA_TRY(cudaMemcpy(err, h.d_err, sizeof(err), cudaMemcpyDeviceToHost));
    if (err[ERR_TIMEOUT]) return RSD_ERR_TIMEOUT;
    if (err[ERR_NOT_SPD]) return RSD_ERR_NOT_SPD;
    return RSD_OK;
}

extern "C" int rsd_solve(rsd_handle hh, const double* f, double* u, double tol, rsd_stats* st) {
    if (!hh || !f || !u || !(tol > 0)) return RSD_ERR_ARG;
    const int rc = hh->h.krylov == RSD_KRYLOV_FGMRES ? fgmres(hh->h, f, u, tol, st) : pcg(hh->h, f, u, tol, st);
    const int chk = rsd_check(hh);
    if (chk != RSD_OK) return chk;
    return rc;
}

extern "C" int rsd_solve_adjoint(rsd_handle hh, const double* g, double* lam, double tol, rsd_stats* st) {
    if (hh && hh->h.lu) {
        set_last_error("rsd_solve_adjoint: the hierarchy holds a nonsymmetric K");
        return RSD_ERR_ARG;
    }
    // Every matrix the hierarchy holds is symmetric (its fronts are Cholesky-factored), so
    // K^T lam = g is the same system as K lam = g: same fronts, same PCG, no new setup.
    return rsd_solve(hh, g, lam, tol, st);
}

extern "C" int rsd_get_info(rsd_handle hh, rsd_info_t* out) {
    if (!hh || !out) return RSD_ERR_ARG;
    const Handle& h = hh->h;
    out->n = h.n;
    out->n_nodes = h.n_nodes;
    out->n_levels = (int)h.levels.size();
    out->factor_elems = h.factor_elems;
    out->factor_bytes = h.factor_bytes;
    out->setup_flops = h.setup_flops;
    out->device_bytes = (int64_t)h.arena_bytes;
    out->notspd_node = h.notspd_node;
    out->promoted = h.promoted;
    return RSD_OK;
}

extern "C" int rsd_front_dims(rsd_handle hh, int32_t node, int32_t* s, int32_t* b, int32_t* level) {
    if (!hh || node < 0 || node >= hh->h.n_nodes) return RSD_ERR_ARG;
    const Handle& h = hh->h;
    const FrontDesc& f = h.levels[h.node_level[node]].fronts[h.node_slot[node]];
    if (s) *s = f.s;
    if (b) *b = f.b;
    if (level) *level = h.depth[node];
    return RSD_OK;
}

extern "C" int rsd_front_dofs(rsd_handle hh, int32_t node, int32_t* out) {
    if (!hh || !out || node < 0 || node >= hh->h.n_nodes) return RSD_ERR_ARG;
    const Handle& h = hh->h;
    const FrontDesc& f = h.levels[h.node_level[node]].fronts[h.node_slot[node]];
    std::copy(h.I_dofs.begin() + h.I_off[node], h.I_dofs.begin() + h.I_off[node + 1], out);
    std::copy(h.B_dofs.begin() + h.B_off[node], h.B_dofs.begin() + h.B_off[node] + f.b, out + f.s);
    return RSD_OK;
}

extern "C" int rsd_front_map(rsd_handle hh, int32_t node, int32_t* out) {
    if (!hh || !out || node < 0 || node >= hh->h.n_nodes) return RSD_ERR_ARG;
    Handle& h = hh->h;
    const Level& L = h.levels[h.node_level[node]];
    const FrontDesc& f = L.fronts[h.node_slot[node]];
    if (f.b == 0) return RSD_OK;
    RSD_CUDA_TRY(cudaMemcpy(out, f.ea, sizeof(int) * f.b, cudaMemcpyDeviceToHost));
    return RSD_OK;
}

extern "C" int rsd_front_factor16(rsd_handle hh, int32_t node, double* out) {
    if (!hh || !out || node < 0 || node >= hh->h.n_nodes) return RSD_ERR_ARG;
    Handle& h = hh->h;
    const Level& L = h.levels[h.node_level[node]];
    const FrontDesc& f = L.fronts[h.node_slot[node]];
    if (!f.P16 || !L.h16) return RSD_ERR_ARG;
    RSD_CUDA_TRY(cudaStreamSynchronize(h.stream));
    std::vector<__half> q((size_t)f.N * f.ldp);
    std::vector<float> rs((size_t)2 * f.N);
    if (!q.empty()) RSD_CUDA_TRY(cudaMemcpy(q.data(), f.P16, q.size() * sizeof(__half), cudaMemcpyDeviceToHost));
    if (!rs.empty()) RSD_CUDA_TRY(cudaMemcpy(rs.data(), f.rs, rs.size() * sizeof(float), cudaMemcpyDeviceToHost));
    for (int r = 0; r < f.N; ++r)
        for (int c = 0; c < f.s; ++c) {
            const bool read = r >= f.s || c / NB < r / NB;       // what the sweeps read
            out[(size_t)r * f.s + c] = read ? (double)__half2float(q[(size_t)r * f.ldp + c]) * (double)rs[f.N + r] : 0.0;
        }
    return RSD_OK;
}

extern "C" int rsd_front_dinv(rsd_handle hh, int32_t node, double* out) {
    if (!hh || !out || node < 0 || node >= hh->h.n_nodes) return RSD_ERR_ARG;
    Handle& h = hh->h;
    const Level& L = h.levels[h.node_level[node]];
    if (!L.factored) return RSD_ERR_ARG;
    const FrontDesc& f = L.fronts[h.node_slot[node]];
    RSD_CUDA_TRY(cudaStreamSynchronize(h.stream));
    const size_t n = (size_t)f.nd * NB * NB;
    if (!n) return RSD_OK;
    if (is_fp64(L.prec)) {
        RSD_CUDA_TRY(cudaMemcpy(out, f.Dinv, n * sizeof(double), cudaMemcpyDeviceToHost));
    } else {
        std::vector<float> buf(n);
        RSD_CUDA_TRY(cudaMemcpy(buf.data(), f.Dinv, n * sizeof(float), cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < n; ++i) out[i] = buf[i];
    }
    return RSD_OK;
}

extern "C" int rsd_front_factor_upper(rsd_handle hh, int32_t node, double* out) {
    if (!hh || !out || node < 0 || node >= hh->h.n_nodes || !hh->h.lu) return RSD_ERR_ARG;
    Handle& h = hh->h;
    RSD_CUDA_TRY(cudaStreamSynchronize(h.stream));
    const Level& L = h.levels[h.node_level[node]];
    if (!L.factored) return RSD_ERR_ARG;
    const FrontDesc& f = L.fronts[h.node_slot[node]];
    const size_t es = elem_bytes(L.prec);
    std::vector<char> buf((size_t)f.N * f.ldp * es);
    if (!buf.empty()) RSD_CUDA_TRY(cudaMemcpy(buf.data(), f.PU, buf.size(), cudaMemcpyDeviceToHost));
    for (int r = 0; r < f.N; ++r)
        for (int c = 0; c < f.s; ++c) {
            const double v = es == 8 ? ((const double*)buf.data())[(size_t)r * f.ldp + c]
                                     : (double)((const float*)buf.data())[(size_t)r * f.ldp + c];
            out[(size_t)r * f.s + c] = (r < f.s && c > r) ? 0.0 : v;
        }
    return RSD_OK;
}

extern "C" int rsd_front_factor(rsd_handle hh, int32_t node, double* out) {
    if (!hh || !out || node < 0 || node >= hh->h.n_nodes) return RSD_ERR_ARG;
    Handle& h = hh->h;
    RSD_CUDA_TRY(cudaStreamSynchronize(h.stream));
    const Level& L = h.levels[h.node_level[node]];
    if (!L.factored) return RSD_ERR_ARG;
    const FrontDesc& f = L.fronts[h.node_slot[node]];
    const size_t es = elem_bytes(L.prec);
    std::vector<char> buf((size_t)f.N * f.ldp * es);
    if (!buf.empty()) RSD_CUDA_TRY(cudaMemcpy(buf.data(), f.P, buf.size(), cudaMemcpyDeviceToHost));
    for (int r = 0; r < f.N; ++r)
        for (int c = 0; c < f.s; ++c) {
            double v = es == 8 ? ((const double*)buf.data())[(size_t)r * f.ldp + c]
                               : (double)((const float*)buf.data())[(size_t)r * f.ldp + c];
            out[(size_t)r * f.s + c] = (r < f.s && c > r) ? 0.0 : v;
        }
    return RSD_OK;
}


// ---- many independent problems in one hierarchy (batched form) ----------------------
namespace rsd {
namespace {

struct ConcatDesc {
    const int64_t* rowptr;
    const int* col;
    const int* owner;
    int n;
    int dof_off;
    int64_t nnz_off;
    int node_off;
    int pad;
};

// Problem p's rows are shifted by dof_off, its nonzeros by nnz_off, its tree nodes by
// node_off; one CTA row-block per problem (blockIdx.y).
__global__ void k_concat(const ConcatDesc* __restrict__ d, int64_t* rowptr, int* col, int* owner) {
    const ConcatDesc c = d[blockIdx.y];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < c.n; i += gridDim.x * blockDim.x) {
        const int64_t r0 = c.rowptr[i], r1 = c.rowptr[i + 1];
        rowptr[c.dof_off + i] = c.nnz_off + r0;
        owner[c.dof_off + i] = c.owner[i] + c.node_off;
        for (int64_t k = r0; k < r1; ++k) col[c.nnz_off + k] = c.col[k] + c.dof_off;
    }
}

}  // namespace
}  // namespace rsd

extern "C" int rsd_setup_batched(int32_t nprob, const rsd_csr* K, const int32_t* const* dof_node,
                                 const rsd_tree* T, const rsd_options* opt, rsd_handle* out) {
    if (nprob <= 0 || !K || !dof_node || !T || !out) return RSD_ERR_ARG;
    *out = nullptr;
    const int mem = K[0].mem;
    int64_t n = 0, nnz = 0, nodes = 1;
    for (int p = 0; p < nprob; ++p) {
        if (K[p].mem != mem || K[p].n <= 0 || K[p].nnz <= 0 || !K[p].rowptr || !K[p].col || !K[p].val ||
            !dof_node[p] || T[p].n_nodes <= 0 || !T[p].parent)
            return RSD_ERR_ARG;
        n += K[p].n;
        nnz += K[p].nnz;
        nodes += T[p].n_nodes;
    }
    if (n > INT32_MAX || nodes > (1 << 24)) return RSD_ERR_ARG;
    // the forest under an empty super-root (node 0)
    std::vector<int> parent(nodes);
    parent[0] = -1;
    std::vector<int> node_off(nprob);
    {
        int64_t base = 1;
        for (int p = 0; p < nprob; ++p) {
            node_off[p] = (int)base;
            for (int t = 0; t < T[p].n_nodes; ++t) {
                const int pp = T[p].parent[t];
                if ((t == 0 && pp != -1) || (t > 0 && (pp < 0 || pp >= t))) return RSD_ERR_ARG;
                parent[base + t] = t == 0 ? 0 : (int)(base + pp);
            }
            base += T[p].n_nodes;
        }
    }
    cudaStream_t st = opt ? (cudaStream_t)opt->stream : nullptr;
    rsd_tree tree{(int32_t)nodes, parent.data()};
    rsd_csr all{};
    all.n = (int32_t)n;
    all.nnz = nnz;
    all.mem = mem;
    int rc;
    if (mem == RSD_MEM_HOST) {
        std::vector<int64_t> rp(n + 1);
        std::vector<int> cl(nnz), ow(n);
        std::vector<double> vl(nnz);
        int64_t dof = 0, nz = 0;
        for (int p = 0; p < nprob; ++p) {
            for (int i = 0; i < K[p].n; ++i) {
                rp[dof + i] = nz + K[p].rowptr[i];
                ow[dof + i] = dof_node[p][i] + node_off[p];
            }
            for (int64_t k = 0; k < K[p].nnz; ++k) {
                cl[nz + k] = K[p].col[k] + (int)dof;
                vl[nz + k] = K[p].val[k];
            }
            dof += K[p].n;
            nz += K[p].nnz;
        }
        rp[n] = nnz;
        all.rowptr = rp.data();
        all.col = cl.data();
        all.val = vl.data();
        rc = rsd_setup(&all, ow.data(), &tree, opt, out);
    } else {
        int64_t* rp = nullptr;
        int* cl = nullptr;
        int* ow = nullptr;
        double* vl = nullptr;
        ConcatDesc* dd = nullptr;
        std::vector<ConcatDesc> desc(nprob);
        int64_t dof = 0, nz = 0;
        int maxn = 0;
        for (int p = 0; p < nprob; ++p) {
            desc[p] = ConcatDesc{K[p].rowptr, K[p].col, dof_node[p], K[p].n, (int)dof, nz, node_off[p], 0};
            dof += K[p].n;
            nz += K[p].nnz;
            maxn = std::max(maxn, K[p].n);
        }
        RSD_CUDA_TRY(cudaMallocAsync((void**)&rp, sizeof(int64_t) * (n + 1), st));
        RSD_CUDA_TRY(cudaMallocAsync((void**)&cl, sizeof(int) * nnz, st));
        RSD_CUDA_TRY(cudaMallocAsync((void**)&ow, sizeof(int) * n, st));
        RSD_CUDA_TRY(cudaMallocAsync((void**)&vl, sizeof(double) * nnz, st));
        RSD_CUDA_TRY(cudaMallocAsync((void**)&dd, sizeof(ConcatDesc) * nprob, st));
        RSD_CUDA_TRY(cudaMemcpyAsync(dd, desc.data(), sizeof(ConcatDesc) * nprob, cudaMemcpyHostToDevice, st));
        for (int p = 0; p < nprob; ++p)
            RSD_CUDA_TRY(cudaMemcpyAsync(vl + desc[p].nnz_off, K[p].val, sizeof(double) * K[p].nnz,
                                         cudaMemcpyDeviceToDevice, st));
        RSD_CUDA_TRY(cudaMemcpyAsync(rp + n, &nnz, sizeof(int64_t), cudaMemcpyHostToDevice, st));
        dim3 grid((unsigned)std::max(1, std::min(1024, (maxn + 255) / 256)), (unsigned)nprob);
        k_concat<<<grid, 256, 0, st>>>(dd, rp, cl, ow);
        count_launch();
        RSD_CUDA_TRY(cudaGetLastError());
        RSD_CUDA_TRY(cudaStreamSynchronize(st));
        all.rowptr = rp;
        all.col = cl;
        all.val = vl;
        rc = rsd_setup(&all, ow, &tree, opt, out);
        cudaFreeAsync(rp, st);
        cudaFreeAsync(cl, st);
        cudaFreeAsync(ow, st);
        cudaFreeAsync(vl, st);
        cudaFreeAsync(dd, st);
        cudaStreamSynchronize(st);
    }
    return rc;
}
