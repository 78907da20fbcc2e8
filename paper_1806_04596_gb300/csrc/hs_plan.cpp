// Plan construction: everything the operators derive from the uv coverage.
//
//  * grid coordinates t = u K / (2 pi) per axis, split into the cell floor(t)
//    (mod K) and the fraction; FP32 plans store both in one 32-bit fixed-point
//    word per axis (fraction resolution 2^-23 .. 2^-20 cells, computed in FP64
//    so the FP32 kernels never form t themselves), FP64 plans store the exact
//    FP64 fraction;
//  * a per-channel sort of the visibilities by the 32 x 32 grid tile holding
//    the start of their 8 x 8 window, then by cell, so that consecutive
//    visibilities touch neighbouring grid cells;
//  * the gridding lists, consumed without atomics: for grids of at least
//    64 x 64 cells, per (channel, 32-column strip, row range) the windows that
//    reach it, grouped by start row into disjoint column ranges (sweep
//    kernel); otherwise, and for the compensated kernel, per (channel, 32 x 32
//    tile) the windows that overlap it (a window straddles at most 2 x 2 tiles);
//  * the Kaiser-Bessel polynomial pieces, the Z scaling, the FFT twiddles;
//  * all scratch buffers, so that no compute call allocates.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>
#include <vector>

#include "hs_internal.h"

namespace hs {

hs_status dwt_init();
hs_status fft_init();
hs_status nufft_init();
hs_status prox_init();
hs_status eig_init();
int64_t gram_part_doubles(int L);

// Device memory held by the library's plans and PD states (process-wide), and
// the optional cap on it (hs_set_device_limit; 0: none).
static std::atomic<int64_t> g_lib_bytes{0};
static std::atomic<int64_t> g_lib_limit{0};

void set_device_limit(int64_t bytes) { g_lib_limit.store(bytes < 0 ? 0 : bytes); }
int64_t device_bytes_held() { return g_lib_bytes.load(); }

hs_status lib_alloc(void** ptr, size_t bytes) {
    *ptr = nullptr;
    const int64_t lim = g_lib_limit.load();
    const int64_t now = g_lib_bytes.fetch_add((int64_t)bytes) + (int64_t)bytes;
    if (lim > 0 && now > lim) {
        g_lib_bytes.fetch_sub((int64_t)bytes);
        return fail(HS_ERR_NOMEM, "allocation of %zu bytes would pass the library's device limit (%lld of %lld held)",
                    bytes, (long long)(now - (int64_t)bytes), (long long)lim);
    }
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *ptr = nullptr;
        g_lib_bytes.fetch_sub((int64_t)bytes);
        return fail(HS_ERR_NOMEM, "cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
    }
    return HS_OK;
}

void lib_free(void* ptr, size_t bytes) {
    if (ptr) {
        cudaFree(ptr);
        g_lib_bytes.fetch_sub((int64_t)bytes);
    }
}

hs_status plan_alloc(Plan* p, void** ptr, size_t bytes) {
    *ptr = nullptr;
    if (bytes == 0) return HS_OK;
    HS_TRY(lib_alloc(ptr, bytes));
    p->allocs.push_back(*ptr);
    p->alloc_bytes.push_back(bytes);
    p->device_bytes += (int64_t)bytes;
    return HS_OK;
}

// Free one allocation of the plan (lists rebuilt at creation).
static void plan_release(Plan* p, void* ptr) {
    for (size_t k = 0; k < p->allocs.size(); ++k)
        if (p->allocs[k] == ptr) {
            lib_free(ptr, p->alloc_bytes[k]);
            p->device_bytes -= (int64_t)p->alloc_bytes[k];
            p->allocs.erase(p->allocs.begin() + k);
            p->alloc_bytes.erase(p->alloc_bytes.begin() + k);
            return;
        }
}

void plan_free(Plan* p) {
    if (p->fft_ev_col) cudaEventDestroy(p->fft_ev_col);
    if (p->fft_ev_join) cudaEventDestroy(p->fft_ev_join);
    if (p->fft_side) cudaStreamDestroy(p->fft_side);
    p->fft_ev_col = p->fft_ev_join = nullptr;
    p->fft_side = nullptr;
    for (size_t k = 0; k < p->allocs.size(); ++k) lib_free(p->allocs[k], p->alloc_bytes[k]);
    p->allocs.clear();
    p->alloc_bytes.clear();
}

static bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }
// x mod K for any x (grids need not be powers of two).
static inline int modk(int64_t x, int K) { return (int)(((x % K) + K) % K); }
// Image sides the kernels support: r 2^a with r in {1, 3, 5} (FFT lines of
// 2 r 2^a), at least 16, and multiples of 16 unless powers of two (gridding
// tiles and strips of 32 cells).
static bool side_ok(int n) {
    if (n < 16 || n > 2048) return false;
    if (pow2(n)) return true;
    int m = n;
    if (m % 5 == 0) m /= 5;
    else if (m % 3 == 0) m /= 3;
    return pow2(m) && n % 16 == 0;
}
static int ilog2(int v) {
    int r = 0;
    while ((1 << r) < v) ++r;
    return r;
}

template <typename T> static hs_status upload(Plan* p, void** dst, const std::vector<T>& h) {
    HS_TRY(plan_alloc(p, dst, h.size() * sizeof(T)));
    if (!h.empty()) HS_CHECK_CUDA(cudaMemcpy(*dst, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    return HS_OK;
}

template <typename R>
static hs_status upload_real(Plan* p, void** dst, const std::vector<double>& h) {
    std::vector<R> v(h.size());
    for (size_t i = 0; i < h.size(); ++i) v[i] = (R)h[i];
    return upload(p, dst, v);
}

static hs_status download_real(const Plan* p, const void* src, int64_t n, std::vector<double>& out,
                               cudaStream_t s) {
    out.assign((size_t)n, 0.0);
    if (n == 0) return HS_OK;
    if (p->prec == HS_F32) {
        std::vector<float> tmp((size_t)n);
        HS_CHECK_CUDA(cudaMemcpyAsync(tmp.data(), src, n * sizeof(float), cudaMemcpyDeviceToHost, s));
        HS_CHECK_CUDA(cudaStreamSynchronize(s));
        for (int64_t i = 0; i < n; ++i) out[i] = tmp[i];
    } else {
        HS_CHECK_CUDA(cudaMemcpyAsync(out.data(), src, n * sizeof(double), cudaMemcpyDeviceToHost, s));
        HS_CHECK_CUDA(cudaStreamSynchronize(s));
    }
    return HS_OK;
}

// Gridding lists of the sweep kernel (grids of at least 64 x 64 cells). A work
// item is one channel, one 32-column strip and its output rows [row0, row1);
// its list holds every window that overlaps the strip and starts in rows
// row0 - 7 .. row1 - 1 (circularly), as groups of 4 slots (-1 pads) whose
// windows cover disjoint columns of the strip (slots in increasing start
// column) and start in the same 4-row band (relative start row y, band
// floor(y / 4)), so that they all lie in that band and the next two. Windows are
// placed in increasing start row, first fit over the band's groups; groups are
// stored by band. Rows are cut after hmax rows, or earlier once the list
// would pass cap windows (at least one row per item). Items are stored
// heaviest first.
// Host part: window start cells k0x[r], k0y[r] in the order the kernel indexes
// them (list entries are these positions r), channel ranges off[0..L].
hs_status sweep_lists(int Kx, int Ky, int L, const int64_t* off, const int* k0xs, const int* k0ys, int hmax_req,
                      int cap, std::vector<SweepItem>& items, std::vector<int>& ent) {
    const int nstrip = Kx / GRID_TILE;
    const int hmax = std::min(hmax_req, Ky - 8);
    struct Win {
        int y, x, r;   // start row (absolute, then relative to row0), start column relative to the strip
    };
    std::vector<std::vector<Win>> strips(nstrip);
    std::vector<int64_t> rowcnt(Ky);
    std::vector<Win> seg;
    items.clear();
    ent.clear();
    struct Grp {
        int y, m;        // band, windows held
        uint32_t mask;   // strip columns covered
        int e[4], x[4];  // sorted visibility indices and start columns, by start column
    };
    std::vector<Grp> open;
    for (int l = 0; l < L; ++l) {
        for (auto& v : strips) v.clear();
        for (int64_t r = off[l]; r < off[l + 1]; ++r) {
            const int k0x = k0xs[r], k0y = k0ys[r];
            const int s0 = k0x / GRID_TILE, s1 = modk(k0x + 7, Kx) / GRID_TILE;
            strips[s0].push_back({k0y, k0x - s0 * GRID_TILE, (int)r});
            if (s1 != s0) strips[s1].push_back({k0y, modk(k0x - s1 * GRID_TILE + 7, Kx) - 7, (int)r});
        }
        for (int st = 0; st < nstrip; ++st) {
            std::vector<Win>& ws = strips[st];
            // by start row (then column, index): a row range is a contiguous run
            std::sort(ws.begin(), ws.end(), [](const Win& a, const Win& b) {
                return a.y != b.y ? a.y < b.y : (a.x != b.x ? a.x < b.x : a.r < b.r);
            });
            auto row_at = [&](int y) {   // first window starting in row >= y
                return std::lower_bound(ws.begin(), ws.end(), y, [](const Win& w, int v) { return w.y < v; });
            };
            std::fill(rowcnt.begin(), rowcnt.end(), 0);
            for (const Win& w : ws) ++rowcnt[w.y];
            for (int row0 = 0; row0 < Ky;) {
                int64_t cnt = 0;
                for (int d = 1; d <= 7; ++d) cnt += rowcnt[modk(row0 - d, Ky)];
                int row1 = row0;
                while (row1 < Ky && row1 - row0 < hmax && (row1 == row0 || cnt + rowcnt[row1] <= cap))
                    cnt += rowcnt[row1++];
                // windows starting in rows row0 - 7 .. row1 - 1 (circularly), in order of
                // their start row relative to row0 (the wrapped rows come first)
                seg.clear();
                auto take = [&](int ya, int yb) {
                    for (auto it = row_at(ya); it != ws.end() && it->y < yb; ++it)
                        seg.push_back({modk(it->y - row0 + 7, Ky) - 7, it->x, it->r});
                };
                if (row0 >= 7) {
                    take(row0 - 7, row1);
                } else {
                    take(Ky + row0 - 7, Ky);
                    take(0, row1);
                }
                const int e0 = (int)ent.size();
                open.clear();
                size_t first = 0;
                for (const Win& w : seg) {
                    const int b = std::max(w.x, 0), e = std::min(w.x + 8, GRID_TILE);
                    const uint32_t mask = (uint32_t)(((uint64_t)1 << e) - ((uint64_t)1 << b));
                    const int band = (w.y + 8) / 4 - 2;   // floor(y / 4), y >= -7
                    while (first < open.size() && open[first].y < band) ++first;
                    size_t gi = first;
                    while (gi < open.size() && (open[gi].m == 4 || (open[gi].mask & mask))) ++gi;
                    if (gi == open.size()) open.push_back({band, 0, 0u, {-1, -1, -1, -1}, {0, 0, 0, 0}});
                    Grp& gr = open[gi];
                    int k = gr.m++;   // keep the slots in increasing start column
                    for (; k > 0 && gr.x[k - 1] > w.x; --k) {
                        gr.e[k] = gr.e[k - 1];
                        gr.x[k] = gr.x[k - 1];
                    }
                    gr.e[k] = w.r;
                    gr.x[k] = w.x;
                    gr.mask |= mask;
                }
                for (const Grp& gr : open) ent.insert(ent.end(), gr.e, gr.e + 4);
                if (ent.size() >= ((size_t)1 << 31)) return fail(HS_ERR_ARG, "too many gridding list entries");
                items.push_back({l, st, row0, row1, e0, (int)ent.size()});
                row0 = row1;
            }
        }
    }
    std::stable_sort(items.begin(), items.end(), [](const SweepItem& a, const SweepItem& b) {
        return (a.e1 - a.e0) + 4 * (a.row1 - a.row0) > (b.e1 - b.e0) + 4 * (b.row1 - b.row0);
    });
    return HS_OK;
}

static hs_status build_sweep(Plan* p, const std::vector<int>& perm, const std::vector<int>& cellx,
                             const std::vector<int>& celly) {
    const int Kx = p->g.Kx, Ky = p->g.Ky;
    const int64_t M = p->off_h[p->g.L];
    std::vector<int> k0x(M), k0y(M);
    for (int64_t r = 0; r < M; ++r) {
        const int64_t i = perm[r];
        k0x[r] = modk(cellx[i] - 3, Kx);
        k0y[r] = modk(celly[i] - 3, Ky);
    }
    std::vector<SweepItem> items;
    std::vector<int> ent;
    HS_TRY(sweep_lists(Kx, Ky, p->g.L, p->off_h.data(), k0x.data(), k0y.data(), p->sweep_hmax, p->sweep_cap, items,
                       ent));
    if (p->sw_items) {   // rebuilt by the autotuner: replace the previous lists
        plan_release(p, p->sw_items);
        plan_release(p, p->sw_ent);
        p->sw_items = nullptr;
        p->sw_ent = nullptr;
    }
    p->n_sw_items = (int64_t)items.size();
    p->n_sw_ent = (int64_t)ent.size();
    HS_TRY(upload(p, &p->sw_items, items));
    HS_TRY(upload(p, (void**)&p->sw_ent, ent));
    return HS_OK;
}

// ---------------------------------------------------------------- autotuner
// Plan-time choice of the parameters that depend on the problem's size and
// sampling density, by timing the candidates on this plan with CUDA events
// (inputs: zeroed plan scratch; the values do not change the work):
//   * sweep gridding row cut and list cap, (32, 512), (64, 1024), (128, 2048):
//     short items balance dense coverage, tall items cut the halo rows;
//   * FP32 Gram matrix of the nuclear prox on the tensor cores or the CUDA
//     cores (the tensor-core form streams 64-pixel chunks per SM and wins on
//     large cubes; the CUDA-core form wins when N L is small);
//   * F^H in one column-pass / row-pass pair over all channels, or in channel
//     chunks sized to keep the intermediate in L2.
// Choices are cached per process by (grid, L, visibilities, precision, flags),
// so plans of the same shape skip the timing.
namespace {
struct TuneKey {
    int Kx, Ky, L, prec;
    unsigned flags;
    int64_t M;
    bool operator<(const TuneKey& o) const {
        return std::tie(Kx, Ky, L, prec, flags, M) < std::tie(o.Kx, o.Ky, o.L, o.prec, o.flags, o.M);
    }
};
struct TuneVal {
    int gram_tc, hmax, cap, fft_chunk;
    double grid_ms[3], gram_ms[2], fft_ms[2];
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune_cache;
}  // namespace

static hs_status time_ms(cudaStream_t s, int reps, const std::function<hs_status()>& fn, double* out) {
    HS_TRY(fn());   // warm-up
    cudaEvent_t e0, e1;
    HS_CHECK_CUDA(cudaEventCreate(&e0));
    HS_CHECK_CUDA(cudaEventCreate(&e1));
    hs_status st = HS_OK;
    HS_CHECK_CUDA(cudaEventRecord(e0, s));
    for (int r = 0; r < reps && st == HS_OK; ++r) st = fn();
    HS_CHECK_CUDA(cudaEventRecord(e1, s));
    HS_CHECK_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    HS_CHECK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *out = ms / reps;
    return st;
}

static hs_status autotune(Plan* p, const std::vector<int>& perm, const std::vector<int>& cellx,
                          const std::vector<int>& celly, bool sweep, cudaStream_t s) {
    const auto t0 = std::chrono::steady_clock::now();
    const TuneKey key{p->g.Kx, p->g.Ky, p->g.L, (int)p->prec, p->flags, p->M_total};
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            const TuneVal& v = it->second;
            p->gram_tc = v.gram_tc;
            p->fft_adj_chunk = v.fft_chunk;
            std::copy(v.grid_ms, v.grid_ms + 3, p->tune_grid_ms);
            std::copy(v.gram_ms, v.gram_ms + 2, p->tune_gram_ms);
            std::copy(v.fft_ms, v.fft_ms + 2, p->tune_fft_ms);
            if (sweep && (v.hmax != p->sweep_hmax || v.cap != p->sweep_cap)) {
                p->sweep_hmax = v.hmax;
                p->sweep_cap = v.cap;
                HS_TRY(build_sweep(p, perm, cellx, celly));
            }
            p->tuned = 2;
            p->tune_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            return HS_OK;
        }
    }
    const int L = p->g.L;
    const int64_t N = p->N();
    const int reps = 3;
    if (sweep && !(p->flags & HS_PLAN_COMPENSATED) && p->M_total > 0) {
        static const int cand[3][2] = {{32, 512}, {64, 1024}, {128, 2048}};
        HS_CHECK_CUDA(cudaMemsetAsync(p->vis, 0, (size_t)p->M_total * p->csize(), s));
        int best = -1;
        for (int c = 0; c < 3; ++c) {
            p->sweep_hmax = cand[c][0];
            p->sweep_cap = cand[c][1];
            HS_TRY(build_sweep(p, perm, cellx, celly));
            GridArgs a{};
            a.mode = GIN_SORTED;
            a.in = p->vis;
            HS_TRY(time_ms(s, reps, [&]() { return grid(p, a, s); }, &p->tune_grid_ms[c]));
            if (best < 0 || p->tune_grid_ms[c] < p->tune_grid_ms[best]) best = c;
        }
        if (best != 2) {
            p->sweep_hmax = cand[best][0];
            p->sweep_cap = cand[best][1];
            HS_TRY(build_sweep(p, perm, cellx, celly));
        }
    }
    if (p->prec == HS_F32 && !(p->flags & HS_PLAN_GRAM_FMA) && L <= MAX_L_NUC) {
        HS_CHECK_CUDA(cudaMemsetAsync(p->xbuf, 0, (size_t)L * N * p->rsize(), s));
        HS_CHECK_CUDA(cudaMemsetAsync(p->xbuf2, 0, (size_t)L * N * p->rsize(), s));
        for (int c = 0; c < 2; ++c) {
            p->gram_tc = c == 0;
            HS_TRY(time_ms(s, reps, [&]() { return gram_matrix(p, p->xbuf, p->xbuf2, s); }, &p->tune_gram_ms[c]));
        }
        p->gram_tc = p->tune_gram_ms[0] <= p->tune_gram_ms[1];
    }
    if (!(p->flags & HS_PLAN_FFT_CHUNKED)) {   // F^H: all channels in one pass pair, or L2-sized channel chunks
        const int C = fft_adjoint_chunk(p);
        if (C < L) {
            p->fft_adj_chunk = 0;
            HS_TRY(time_ms(s, reps, [&]() { return fft_adjoint(p, p->xbuf, s); }, &p->tune_fft_ms[0]));
            p->fft_adj_chunk = C;
            HS_TRY(time_ms(s, reps, [&]() { return fft_adjoint(p, p->xbuf, s); }, &p->tune_fft_ms[1]));
            if (p->tune_fft_ms[1] >= p->tune_fft_ms[0]) p->fft_adj_chunk = 0;
        }
    }
    HS_CHECK_CUDA(cudaStreamSynchronize(s));
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        TuneVal v{p->gram_tc, p->sweep_hmax, p->sweep_cap, p->fft_adj_chunk, {}, {}, {}};
        std::copy(p->tune_grid_ms, p->tune_grid_ms + 3, v.grid_ms);
        std::copy(p->tune_gram_ms, p->tune_gram_ms + 2, v.gram_ms);
        std::copy(p->tune_fft_ms, p->tune_fft_ms + 2, v.fft_ms);
        g_tune_cache[key] = v;
    }
    p->tuned = 1;
    p->tune_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return HS_OK;
}

static hs_status build(Plan* p, const int64_t* vis_offsets, int nblocks, const int64_t* block_offsets,
                       const void* uv, const void* weights, const void* precond, cudaStream_t s) {
    Geo& g = p->g;
    const int L = g.L;
    p->off_h.assign(vis_offsets, vis_offsets + L + 1);
    if (p->off_h[0] != 0) return fail(HS_ERR_ARG, "vis_offsets[0] must be 0");
    int64_t Mmax = 0;
    for (int l = 0; l < L; ++l) {
        const int64_t m = p->off_h[l + 1] - p->off_h[l];
        if (m < 0) return fail(HS_ERR_ARG, "vis_offsets must be nondecreasing (channel %d)", l);
        Mmax = std::max(Mmax, m);
    }
    const int64_t M = p->off_h[L];
    if (M >= ((int64_t)1 << 31)) return fail(HS_ERR_ARG, "total visibilities must be < 2^31");
    if (M > 0 && uv == nullptr) return fail(HS_ERR_ARG, "uv is null");
    p->M_total = M;
    p->Mmax = (int)Mmax;
    // data blocks (Sec. 2.1, M_l^b): contiguous caller ranges inside channels
    if (block_offsets == nullptr) {
        p->blk_off_h = p->off_h;
    } else {
        if (nblocks < L) return fail(HS_ERR_ARG, "nblocks (%d) must be >= L (%d)", nblocks, L);
        p->blk_off_h.assign(block_offsets, block_offsets + nblocks + 1);
        if (p->blk_off_h[0] != 0 || p->blk_off_h[nblocks] != M)
            return fail(HS_ERR_ARG, "block_offsets must run from 0 to the total visibility count");
        for (int k = 0; k < nblocks; ++k)
            if (p->blk_off_h[k + 1] < p->blk_off_h[k]) return fail(HS_ERR_ARG, "block_offsets must be nondecreasing");
        for (int l = 1; l < L; ++l)   // every channel boundary must be a block boundary
            if (!std::binary_search(p->blk_off_h.begin(), p->blk_off_h.end(), p->off_h[l]))
                return fail(HS_ERR_ARG, "block_offsets must contain every channel boundary (channel %d)", l);
    }
    p->nblk = (int)p->blk_off_h.size() - 1;
    p->blk_ch.assign(p->nblk, 0);
    for (int k = 0; k < p->nblk; ++k) {   // channel of a block: the last channel starting at or before it
        const int64_t x = p->blk_off_h[k];
        const int l = (int)(std::upper_bound(p->off_h.begin(), p->off_h.end() - 1, x) - p->off_h.begin()) - 1;
        p->blk_ch[k] = std::max(0, std::min(L - 1, l));
    }

    std::vector<double> uvh, wh, uh;
    HS_TRY(download_real(p, uv, 2 * M, uvh, s));
    if (weights) HS_TRY(download_real(p, weights, M, wh, s));
    if (precond) HS_TRY(download_real(p, precond, M, uh, s));
    for (int64_t i = 0; i < 2 * M; ++i) {
        const double v = uvh[i];
        if (!std::isfinite(v) || v < -M_PI || v >= M_PI)
            return fail(HS_ERR_ARG, "uv[%lld] = %g outside [-pi, pi)", (long long)(i / 2), v);
    }
    for (int64_t i = 0; i < (int64_t)uh.size(); ++i)
        if (!(uh[i] > 0.0) || !std::isfinite(uh[i]))
            return fail(HS_ERR_ARG, "precond[%lld] must be finite and > 0", (long long)i);

    const int Kx = g.Kx, Ky = g.Ky, TX = g.tx, TY = g.ty;
    // per-visibility cells and fractions (FP64, same expression as t = u K / (2 pi))
    std::vector<int> cellx(M), celly(M);
    std::vector<double> fx(M), fy(M);
    for (int64_t i = 0; i < M; ++i) {
        const double tu = uvh[2 * i] * Kx / (2.0 * M_PI);
        const double tv = uvh[2 * i + 1] * Ky / (2.0 * M_PI);
        const double flu = std::floor(tu), flv = std::floor(tv);
        fx[i] = tu - flu;
        fy[i] = tv - flv;
        cellx[i] = (int)((((int64_t)flu % Kx) + Kx) % Kx);
        celly[i] = (int)((((int64_t)flv % Ky) + Ky) % Ky);
    }
    // sort each block (each channel without blocks) by (tile of the window start, cell)
    std::vector<int> perm(M);
    std::vector<uint64_t> keys;
    for (int kb = 0; kb < p->nblk; ++kb) {
        const int64_t a = p->blk_off_h[kb], b = p->blk_off_h[kb + 1];
        keys.resize(b - a);
        for (int64_t i = a; i < b; ++i) {
            const int k0x = modk(cellx[i] - 3, Kx), k0y = modk(celly[i] - 3, Ky);
            const uint64_t tile = (uint64_t)(k0y / TY) * g.ntx + (uint64_t)(k0x / TX);
            const uint64_t key = (tile * TY + (uint64_t)(k0y % TY)) * TX + (uint64_t)(k0x % TX);
            keys[i - a] = (key << 32) | (uint64_t)(i - a);
        }
        std::sort(keys.begin(), keys.end());
        for (int64_t r = 0; r < b - a; ++r) perm[a + r] = (int)(a + (int64_t)(keys[r] & 0xffffffffu));
    }
    HS_TRY(upload(p, (void**)&p->perm, perm));
    if (p->nblk != L) {   // block of every sorted visibility (gridding scale lookup)
        std::vector<int> bid(M);
        for (int kb = 0; kb < p->nblk; ++kb)
            for (int64_t r = p->blk_off_h[kb]; r < p->blk_off_h[kb + 1]; ++r) bid[r] = kb;
        HS_TRY(upload(p, (void**)&p->blk_id, bid));
    }
    // de-gridding work items: runs of one window-start tile in each block's
    // sorted range (cells before the fixed-point carry, as in the sort key), split
    // into chunks of at most DEGRID_CHUNK visibilities; slot = block * items_max + k
    {
        std::vector<int> items;
        const int nb = p->nblk;
        std::vector<int> per_b(nb, 0);
        const int64_t ntl = (int64_t)g.ntx * g.nty;
        for (int kb = 0; kb < nb; ++kb) {
            const int l = p->blk_ch[kb];
            const int64_t a = p->blk_off_h[kb], b = p->blk_off_h[kb + 1];
            int64_t r = a;
            while (r < b) {
                auto tile_of = [&](int64_t rr) {
                    const int64_t i = perm[rr];
                    const int k0x = modk(cellx[i] - 3, Kx), k0y = modk(celly[i] - 3, Ky);
                    return (int64_t)(k0y / TY) * g.ntx + k0x / TX;
                };
                const int64_t t = tile_of(r);
                int64_t e = r + 1;
                while (e < b && tile_of(e) == t) ++e;
                for (int64_t c0 = r; c0 < e; c0 += DEGRID_CHUNK) {
                    const int64_t c1 = std::min<int64_t>(e, c0 + DEGRID_CHUNK);
                    items.insert(items.end(), {(int)(l * ntl + t), (int)c0, (int)c1, kb});
                    ++per_b[kb];
                }
                r = e;
            }
        }
        int mx = 1;
        for (int kb = 0; kb < nb; ++kb) mx = std::max(mx, per_b[kb]);
        std::vector<int> seen(nb, 0);
        for (size_t k = 0; k < items.size(); k += 4) {   // slot = block * items_max + rank in block
            const int kb = items[k + 3];
            items[k + 3] = kb * mx + seen[kb]++;
        }
        p->dg_items_max = mx;
        p->n_dg_items = (int64_t)items.size() / 4;
        HS_TRY(upload(p, &p->dg_items, items));
    }

    if (p->prec == HS_F32) {
        std::vector<uint32_t> c((size_t)2 * M);
        for (int64_t r = 0; r < M; ++r) {
            const int64_t i = perm[r];
            int cxv = cellx[i], cyv = celly[i];
            uint64_t qx = (uint64_t)std::llround(std::ldexp(fx[i], g.fbx));
            uint64_t qy = (uint64_t)std::llround(std::ldexp(fy[i], g.fby));
            if (qx >= (1ull << g.fbx)) {
                qx = 0;
                cxv = modk(cxv + 1, Kx);
            }
            if (qy >= (1ull << g.fby)) {
                qy = 0;
                cyv = modk(cyv + 1, Ky);
            }
            c[2 * r] = ((uint32_t)cxv << g.fbx) | (uint32_t)qx;
            c[2 * r + 1] = ((uint32_t)cyv << g.fby) | (uint32_t)qy;
            cellx[i] = cxv;   // tile membership below uses the stored cell
            celly[i] = cyv;
        }
        HS_TRY(upload(p, &p->coords, c));
    } else {
        std::vector<Coord64> c(M);
        for (int64_t r = 0; r < M; ++r) {
            const int64_t i = perm[r];
            c[r].fx = fx[i];
            c[r].fy = fy[i];
            c[r].cx = cellx[i];
            c[r].cy = celly[i];
        }
        HS_TRY(upload(p, &p->coords, c));
    }
    if (!wh.empty()) {
        std::vector<double> ws(M);
        for (int64_t r = 0; r < M; ++r) ws[r] = wh[perm[r]];
        HS_TRY(p->prec == HS_F32 ? upload_real<float>(p, &p->w_sorted, ws)
                                 : upload_real<double>(p, &p->w_sorted, ws));
    }
    if (!uh.empty()) {
        std::vector<double> us(M);
        for (int64_t r = 0; r < M; ++r) us[r] = uh[perm[r]];
        HS_TRY(p->prec == HS_F32 ? upload_real<float>(p, &p->u_sorted, us)
                                 : upload_real<double>(p, &p->u_sorted, us));
    }

    // gridding lists: the sweep kernel's for grids of at least 64 x 64 cells;
    // per-tile lists for smaller grids and the compensated kernel
    const bool sweep = Kx >= 2 * GRID_TILE && Ky >= 2 * GRID_TILE;
    if (sweep) HS_TRY(build_sweep(p, perm, cellx, celly));
    if (!sweep || (p->flags & HS_PLAN_COMPENSATED)) {
        // gridding lists: every (channel, tile) overlapped by a window
        const int64_t nt = p->ntiles();
        std::vector<int64_t> toff((size_t)L * nt + 1, 0);
        auto tiles_of = [&](int64_t r, int* txs, int* tys, int& ntx_, int& nty_) {
            const int64_t i = perm[r];
            const int k0x = modk(cellx[i] - 3, Kx), k0y = modk(celly[i] - 3, Ky);
            txs[0] = k0x / TX;
            txs[1] = modk(k0x + 7, Kx) / TX;
            tys[0] = k0y / TY;
            tys[1] = modk(k0y + 7, Ky) / TY;
            ntx_ = txs[1] != txs[0] ? 2 : 1;
            nty_ = tys[1] != tys[0] ? 2 : 1;
        };
        for (int l = 0; l < L; ++l)
            for (int64_t r = p->off_h[l]; r < p->off_h[l + 1]; ++r) {
                int txs[2], tys[2], a, b;
                tiles_of(r, txs, tys, a, b);
                for (int yy = 0; yy < b; ++yy)
                    for (int xx = 0; xx < a; ++xx) ++toff[1 + (size_t)l * nt + tys[yy] * g.ntx + txs[xx]];
            }
        for (size_t k = 1; k < toff.size(); ++k) toff[k] += toff[k - 1];
        if (toff.back() >= ((int64_t)1 << 30)) return fail(HS_ERR_ARG, "too many gridding list entries");
        std::vector<int> ent((size_t)toff.back());
        {
            std::vector<int64_t> fill(toff.begin(), toff.end() - 1);
            for (int l = 0; l < L; ++l)
                for (int64_t r = p->off_h[l]; r < p->off_h[l + 1]; ++r) {
                    int txs[2], tys[2], a, b;
                    tiles_of(r, txs, tys, a, b);
                    for (int yy = 0; yy < b; ++yy)
                        for (int xx = 0; xx < a; ++xx)
                            ent[fill[(size_t)l * nt + tys[yy] * g.ntx + txs[xx]]++] = (int)r;
                }
        }
        // Regroup every list into groups of 4 entries whose windows do not overlap
        // (circular distance >= 8 cells in x or y), padding with -1, so that the
        // gridding kernel can add the 4 windows of a group at once without atomics.
        // Greedy, in list order: an entry joins the first open group it fits; at
        // most GROUP_OPEN groups are open, the oldest is closed (padded) to make room.
        std::vector<int64_t> goff((size_t)L * nt + 1, 0);
        std::vector<int> gent;
        gent.reserve((size_t)(toff.back() + toff.back() / 4 + 64));
        {
            constexpr int GROUP_OPEN = 64;
            struct Group {
                int m;
                int e[4], x[4], y[4];
            };
            auto circ = [](int d, int K) {
                d &= K - 1;
                return d < K - d ? d : K - d;
            };
            std::vector<Group> open;
            auto emit = [&](const Group& g) {
                for (int k = 0; k < 4; ++k) gent.push_back(k < g.m ? g.e[k] : -1);
            };
            for (int64_t tix = 0; tix < (int64_t)L * nt; ++tix) {
                open.clear();
                for (int64_t q = toff[tix]; q < toff[tix + 1]; ++q) {
                    const int r = ent[q];
                    const int64_t i = perm[r];
                    const int x = modk(cellx[i] - 3, Kx), y = modk(celly[i] - 3, Ky);
                    bool placed = false;
                    for (size_t gi = 0; gi < open.size() && !placed; ++gi) {
                        Group& g = open[gi];
                        bool fits = true;
                        for (int k = 0; k < g.m && fits; ++k)
                            fits = circ(x - g.x[k], Kx) >= 8 || circ(y - g.y[k], Ky) >= 8;
                        if (!fits) continue;
                        g.e[g.m] = r;
                        g.x[g.m] = x;
                        g.y[g.m] = y;
                        if (++g.m == 4) {
                            emit(g);
                            open.erase(open.begin() + gi);
                        }
                        placed = true;
                    }
                    if (placed) continue;
                    if ((int)open.size() == GROUP_OPEN) {
                        emit(open.front());
                        open.erase(open.begin());
                    }
                    Group g{};
                    g.m = 1;
                    g.e[0] = r;
                    g.x[0] = x;
                    g.y[0] = y;
                    open.push_back(g);
                }
                for (const Group& g : open) emit(g);
                goff[tix + 1] = (int64_t)gent.size();
            }
        }
        p->n_ent = goff.back();
        if (p->n_ent >= ((int64_t)1 << 31)) return fail(HS_ERR_ARG, "too many gridding list entries");
        HS_TRY(upload(p, (void**)&p->tile_off, goff));
        HS_TRY(upload(p, (void**)&p->tile_ent, gent));
        // work items: lists longer than GRID_CAP entries are split at group
        // boundaries; split tiles are merged
        {
            std::vector<int> items, merges;
            int slots = 0;
            for (int64_t tix = 0; tix < (int64_t)L * nt; ++tix) {
                const int64_t a = goff[tix], b = goff[tix + 1];
                const int64_t ng = (b - a) / 4;
                const int parts = ng * 4 <= GRID_CAP ? 1 : (int)((ng * 4 + GRID_CAP - 1) / GRID_CAP);
                if (parts == 1) {
                    items.insert(items.end(), {(int)tix, (int)a, (int)b, -1});
                } else {
                    merges.insert(merges.end(), {(int)tix, slots, parts});
                    for (int k = 0; k < parts; ++k) {
                        const int64_t e0 = a + 4 * (ng * k / parts), e1 = a + 4 * (ng * (k + 1) / parts);
                        items.insert(items.end(), {(int)tix, (int)e0, (int)e1, slots + k});
                    }
                    slots += parts;
                }
            }
            p->n_items = (int64_t)items.size() / 4;
            p->n_merges = (int64_t)merges.size() / 3;
            HS_TRY(upload(p, &p->grid_items, items));
            HS_TRY(upload(p, &p->grid_merges, merges));
            HS_TRY(plan_alloc(p, &p->grid_partial, (size_t)std::max(slots, 1) * g.tx * g.ty * p->csize()));
        }
    }
    if (sweep && !(p->flags & HS_PLAN_COMPENSATED)) p->n_ent = p->n_sw_ent;
    HS_TRY(upload(p, (void**)&p->off_d, p->off_h));

    // tables
    std::vector<double> kbc;
    p->kb_terms = p->prec == HS_F32 ? KB_TERMS_F32 : KB_TERMS_F64;
    p->kb_fit_err = kb_poly_fit(p->J, p->beta, p->kb_terms, &kbc);
    p->kbc_h = kbc;
    std::vector<double> cx(g.nx), cy(g.ny);
    for (int i = 0; i < g.nx; ++i) cx[i] = 1.0 / kb_phihat((double)(i - g.nx / 2) / Kx, p->J, p->beta);
    for (int i = 0; i < g.ny; ++i) cy[i] = 1.0 / kb_phihat((double)(i - g.ny / 2) / Ky, p->J, p->beta);
    std::vector<double> twx(2 * (size_t)Kx), twy(2 * (size_t)Ky);
    for (int m = 0; m < Kx; ++m) {
        twx[2 * m] = std::cos(2.0 * M_PI * m / Kx);
        twx[2 * m + 1] = -std::sin(2.0 * M_PI * m / Kx);
    }
    for (int m = 0; m < Ky; ++m) {
        twy[2 * m] = std::cos(2.0 * M_PI * m / Ky);
        twy[2 * m + 1] = -std::sin(2.0 * M_PI * m / Ky);
    }
    if (p->prec == HS_F32) {
        HS_TRY(upload_real<float>(p, &p->kbc, kbc));
        HS_TRY(upload_real<float>(p, &p->cxs, cx));
        HS_TRY(upload_real<float>(p, &p->cys, cy));
        HS_TRY(upload_real<float>(p, &p->twx, twx));
        HS_TRY(upload_real<float>(p, &p->twy, twy));
    } else {
        HS_TRY(upload_real<double>(p, &p->kbc, kbc));
        HS_TRY(upload_real<double>(p, &p->cxs, cx));
        HS_TRY(upload_real<double>(p, &p->cys, cy));
        HS_TRY(upload_real<double>(p, &p->twx, twx));
        HS_TRY(upload_real<double>(p, &p->twy, twy));
    }

    // scratch
    const size_t rs = p->rsize(), cs = p->csize();
    const int64_t N = p->N();
    HS_TRY(plan_alloc(p, &p->grid, (size_t)L * Ky * Kx * cs));
    HS_TRY(plan_alloc(p, &p->tmp, (size_t)L * g.ny * Kx * cs));
    HS_TRY(plan_alloc(p, &p->vis, (size_t)std::max<int64_t>(M, 1) * cs));
    HS_TRY(plan_alloc(p, &p->dwt_a, (size_t)NW * L * N * rs));
    HS_TRY(plan_alloc(p, &p->dwt_b, (size_t)NW * L * N * rs));
    HS_TRY(plan_alloc(p, &p->xbuf, (size_t)L * N * rs));
    HS_TRY(plan_alloc(p, &p->xbuf2, (size_t)L * N * rs));
    const int64_t nbx = (Mmax + DEGRID_CHUNK - 1) / DEGRID_CHUNK;
    p->part_n = std::max<int64_t>({(int64_t)L * std::max<int64_t>(nbx, 1),
                                   gram_part_doubles(std::min(L, MAX_L_NUC)), 8192});
    HS_TRY(plan_alloc(p, (void**)&p->part, (size_t)p->part_n * sizeof(double)));
    HS_TRY(plan_alloc(p, (void**)&p->gram, sizeof(double) * MAX_L_NUC * MAX_L_NUC));
    HS_TRY(plan_alloc(p, (void**)&p->eigf, sizeof(double) * LR_TOTAL_DOUBLES));
    HS_TRY(plan_alloc(p, (void**)&p->sv, sizeof(double) * MAX_L_NUC));
    HS_TRY(plan_alloc(p, (void**)&p->dscal, sizeof(double) * 6 * std::max(L, 1)));
    HS_TRY(plan_alloc(p, (void**)&p->err_d, sizeof(int)));
    HS_CHECK_CUDA(cudaStreamCreateWithFlags(&p->fft_side, cudaStreamNonBlocking));
    HS_CHECK_CUDA(cudaEventCreateWithFlags(&p->fft_ev_col, cudaEventDisableTiming));
    HS_CHECK_CUDA(cudaEventCreateWithFlags(&p->fft_ev_join, cudaEventDisableTiming));
    HS_CHECK_CUDA(cudaMemsetAsync(p->err_d, 0, sizeof(int), s));
    if (p->flags & HS_PLAN_GRAM_FMA) p->gram_tc = 0;
    if (p->flags & HS_PLAN_FFT_CHUNKED) p->fft_adj_chunk = fft_adjoint_chunk(p);
    if (!(p->flags & HS_PLAN_NO_TUNE)) HS_TRY(autotune(p, perm, cellx, celly, sweep, s));
    HS_CHECK_CUDA(cudaStreamSynchronize(s));
    return HS_OK;
}

hs_status plan_create(Plan** out, int nx, int ny, int L, const int64_t* vis_offsets, int nblocks,
                      const int64_t* block_offsets, const void* uv, const void* weights, const void* precond,
                      int oversample, int J, double kb_beta, int levels, hs_prec prec, unsigned flags,
                      cudaStream_t s) {
    if (out == nullptr) return fail(HS_ERR_ARG, "out is null");
    *out = nullptr;
    if (vis_offsets == nullptr) return fail(HS_ERR_ARG, "vis_offsets is null");
    if (!side_ok(nx) || !side_ok(ny))
        return fail(HS_ERR_ARG, "nx, ny must be in [16, 2048] and powers of two, or 3 or 5 times a power of two "
                                "and multiples of 16 (got %d x %d)", nx, ny);
    if (L < 1 || L > 1024) return fail(HS_ERR_ARG, "L must be in [1, 1024] (got %d)", L);
    if (oversample != 2) return fail(HS_ERR_ARG, "oversample must be 2 (got %d)", oversample);
    if (J != 8) return fail(HS_ERR_ARG, "J must be 8 (got %d)", J);
    if (levels < 1 || levels > 8 || (nx >> levels) < 1 || (ny >> levels) < 1 ||
        nx % (1 << levels) || ny % (1 << levels))
        return fail(HS_ERR_ARG, "wavelet_levels %d incompatible with %d x %d", levels, nx, ny);
    for (int lev = 0; lev < levels; ++lev) {   // DWT tiles: 16 coefficients per subband side, or one tile
        const int hy = ny >> (lev + 1), hx = nx >> (lev + 1);
        if ((hy >= 16 && hy % 16) || (hx >= 16 && hx % 16))
            return fail(HS_ERR_ARG, "wavelet_levels %d: level %d subbands of %d x %d are not multiples of 16",
                        levels, lev, hy, hx);
    }
    if (prec != HS_F32 && prec != HS_F64) return fail(HS_ERR_ARG, "bad precision %d", (int)prec);
    if (flags & ~(unsigned)(HS_PLAN_COMPENSATED | HS_PLAN_GRAM_FMA | HS_PLAN_NO_TUNE | HS_PLAN_FFT_CHUNKED))
        return fail(HS_ERR_ARG, "unknown plan flags 0x%x", flags);
    HS_TRY(dwt_init());
    HS_TRY(fft_init());
    HS_TRY(nufft_init());
    HS_TRY(prox_init());
    HS_TRY(eig_init());
    std::unique_ptr<Plan> p(new Plan());
    p->prec = prec;
    p->flags = flags;
    p->levels = levels;
    p->J = J;
    p->o = oversample;
    p->beta = kb_beta > 0 ? kb_beta
                          : M_PI * std::sqrt((double)(J * J) / (oversample * oversample) *
                                                 (oversample - 0.5) * (oversample - 0.5) - 0.8);
    Geo& g = p->g;
    g.nx = nx;
    g.ny = ny;
    g.L = L;
    g.Kx = oversample * nx;
    g.Ky = oversample * ny;
    g.fbx = std::min(23, 32 - ilog2(g.Kx));
    g.fby = std::min(23, 32 - ilog2(g.Ky));
    g.kxm = pow2(g.Kx) ? g.Kx - 1 : -1;
    g.kym = pow2(g.Ky) ? g.Ky - 1 : -1;
    g.tx = std::min(GRID_TILE, g.Kx);
    g.ty = std::min(GRID_TILE, g.Ky);
    g.ntx = g.Kx / g.tx;
    g.nty = g.Ky / g.ty;
    hs_status st = build(p.get(), vis_offsets, nblocks, block_offsets, uv, weights, precond, s);
    if (st != HS_OK) {
        plan_free(p.get());
        return st;
    }
    *out = p.release();
    return HS_OK;
}

}  // namespace hs
