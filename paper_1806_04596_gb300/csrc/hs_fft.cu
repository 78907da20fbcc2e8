// Batched 2-D FFT of the oversampled grid with the zero-padding / scaling Z
// fused into the first pass and the crop / scale / real part of Z^T fused
// into the last pass (Sec. 2.1: Phi_l = Theta_l G_l F Z).
//
// F is applied as two batches of 1-D transforms (rows, then columns). Each
// CTA transforms G lines held in shared memory with a self-sorting Stockham
// schedule of radix-8 passes (one 8-point DFT per thread per pass, operands in
// registers) and one final radix-4 or radix-2 pass when log2 K is not a
// multiple of 3. The first pass loads straight from global memory through the
// mode's gather (padding, scaling), the last pass stores straight to global
// memory through the mode's scatter (layout, crop), so each line costs one
// global read and one global write.
//
// Forward Phi:  X (L x ny x nx real) --rows--> tmp (L x ny x Kx) --cols--> grid (L x Ky x Kx)
// Adjoint:      grid --cols, inverse, keep ny rows--> tmp --rows, inverse, crop--> X
// Only the ny image rows are ever transformed along x: the other Ky - ny rows
// of Z x are zero in the forward direction and discarded by Z^T in the adjoint.
//
// Lines whose length is not a power of two (K = r 2^m, r = 3 or 5: images
// such as 1280 x 1280, grids of 2560) use k_fft_mr: the same gather / scatter
// modes around a mixed-radix Stockham schedule (one radix-r pass, then radix
// 4 and 2) with each pass's small DFT evaluated directly, ping-ponging between
// two shared-memory copies of the CTA's lines.
#include <algorithm>

#include "hs_device.cuh"
#include "hs_internal.h"

namespace hs {

enum FftMode { ROW_FWD = 0, COL_FWD = 1, COL_INV = 2, ROW_INV = 3 };

template <typename R> struct FftArgs {
    const void* in;
    void* out;
    const Cx<R>* tw;   // exp(-2 pi i m / K), m < K
    const R* cxs;      // Z scale along x (nx)
    const R* cys;      // Z scale along y (ny)
    int K, G, n8, rlast, npass;
    int lgK, lgG;      // log2 K, log2 G
    int nx, ny, Kx, Ky;
    int lgny, lgKx;    // log2 ny, log2 Kx
};

// A line is a row (l, iy) of the row modes or a column (l, kx) of the column
// modes; la = channel, lb = iy or kx.
template <typename R, int MODE>
__device__ __forceinline__ void line_of(const FftArgs<R>& a, int line, int& la, int& lb) {
    if (MODE == COL_FWD || MODE == COL_INV) {
        la = line >> a.lgKx;
        lb = line & (a.Kx - 1);
    } else {
        la = line >> a.lgny;
        lb = line & (a.ny - 1);
    }
}

template <typename R, int MODE>
__device__ __forceinline__ Cx<R> fft_load(const FftArgs<R>& a, int la, int lb, int k) {
    typedef Cx<R> CT;
    if (MODE == ROW_FWD) {   // Z: pad and scale
        const int h = a.nx >> 1;
        int ix;
        if (k < h) ix = k + h;
        else if (k >= a.Kx - h) ix = k - a.Kx + h;
        else return cx<R>(0, 0);
        const R* X = (const R*)a.in;
        return cx<R>(a.cys[lb] * a.cxs[ix] * X[((int64_t)la * a.ny + lb) * a.nx + ix], (R)0);
    } else if (MODE == COL_FWD) {   // only the ny image rows are nonzero
        const int h = a.ny >> 1;
        int iy;
        if (k < h) iy = k + h;
        else if (k >= a.Ky - h) iy = k - a.Ky + h;
        else return cx<R>(0, 0);
        return ((const CT*)a.in)[((int64_t)la * a.ny + iy) * a.Kx + lb];
    } else if (MODE == COL_INV) {
        return ((const CT*)a.in)[((int64_t)la * a.Ky + k) * a.Kx + lb];
    } else {   // ROW_INV
        return ((const CT*)a.in)[((int64_t)la * a.ny + lb) * a.Kx + k];
    }
}

template <typename R, int MODE>
__device__ __forceinline__ void fft_store(const FftArgs<R>& a, int la, int lb, int k, Cx<R> v) {
    typedef Cx<R> CT;
    if (MODE == ROW_FWD) {
        ((CT*)a.out)[((int64_t)la * a.ny + lb) * a.Kx + k] = v;
    } else if (MODE == COL_FWD) {
        ((CT*)a.out)[((int64_t)la * a.Ky + k) * a.Kx + lb] = v;
    } else if (MODE == COL_INV) {   // keep the ny image rows
        const int h = a.ny >> 1;
        int iy;
        if (k < h) iy = k + h;
        else if (k >= a.Ky - h) iy = k - a.Ky + h;
        else return;
        ((CT*)a.out)[((int64_t)la * a.ny + iy) * a.Kx + lb] = v;
    } else {   // ROW_INV: crop, scale, real part
        const int h = a.nx >> 1;
        int ix;
        if (k < h) ix = k + h;
        else if (k >= a.Kx - h) ix = k - a.Kx + h;
        else return;
        ((R*)a.out)[((int64_t)la * a.ny + lb) * a.nx + ix] = a.cys[lb] * a.cxs[ix] * v.x;
    }
}

// One Stockham pass of radix RAD (LGR = log2 RAD) over the CTA's G lines:
// every thread owns NREP x 8 / RAD butterflies (8 NREP operands, all in
// registers; NREP > 1 lets long column lines come G = 4 to a CTA, so that
// every 32-byte sector of a column load is used, within 512 threads).
// LGK_ / LGG_ > 0 fix log2 K and log2 G at compile time (0: from the arguments).
template <typename R, int DIR, int MODE, int RAD, int LGR, int LGK_, int LGG_, int NREP>
__device__ __forceinline__ void fft_pass(const FftArgs<R>& a, Cx<R>* sm, int lgNs, bool first,
                                         bool last, int line0) {
    typedef Cx<R> CT;
    constexpr bool COLS = (MODE == COL_FWD || MODE == COL_INV);
    constexpr int PER = 8 / RAD * NREP;
    const int lgK = LGK_ > 0 ? LGK_ : a.lgK;
    const int lgG = LGG_ > 0 || LGK_ > 0 ? LGG_ : a.lgG;
    const int K = 1 << lgK, G = 1 << lgG;
    const int nthr = LGK_ > 0 ? ((G << lgK) >> 3) / NREP : blockDim.x, tid = threadIdx.x;
    const int lgnb = lgK - LGR;
    const int nb = 1 << lgnb;
    const int lgstep = lgK - lgNs - LGR;
    CT v[8 * NREP];
    int gs[PER], js[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int w = tid + i * nthr;
        const int g = COLS ? (w & (G - 1)) : (w >> lgnb);
        const int j = COLS ? (w >> lgG) : (w & (nb - 1));
        gs[i] = g;
        js[i] = j;
        int la = 0, lb = 0;
        if (first) line_of<R, MODE>(a, line0 + g, la, lb);
#pragma unroll
        for (int r = 0; r < RAD; ++r) {
            const int k = j + r * nb;
            v[i * RAD + r] = first ? fft_load<R, MODE>(a, la, lb, k)
                                   : sm[COLS ? (k * G + g) : (g * K + k)];
        }
    }
    if (!first) __syncthreads();   // every read of this pass precedes any write
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int j = js[i];
        const int kk = j & ((1 << lgNs) - 1);
        CT* u = v + i * RAD;
        if (lgNs > 0) {   // the first pass has unit twiddles
            if (RAD == 8) {
                // w^1, w^2, w^4 from the table, the others as products (one rounding each)
                CT t[8];
                t[1] = a.tw[kk << lgstep];
                t[2] = a.tw[(2 * kk) << lgstep];
                t[4] = a.tw[(4 * kk) << lgstep];
                t[3] = cmul(t[1], t[2]);
                t[5] = cmul(t[1], t[4]);
                t[6] = cmul(t[2], t[4]);
                t[7] = cmul(t[3], t[4]);
#pragma unroll
                for (int r = 1; r < 8; ++r) {
                    if (DIR > 0) t[r].y = -t[r].y;
                    u[r] = cmul(u[r], t[r]);
                }
            } else {
#pragma unroll
                for (int r = 1; r < RAD; ++r) {
                    CT t = a.tw[(kk * r) << lgstep];
                    if (DIR > 0) t.y = -t.y;
                    u[r] = cmul(u[r], t);
                }
            }
        }
        if (RAD == 8) {
            dft8<R, DIR>(u);
        } else if (RAD == 4) {
            dft4<DIR>(u[0], u[1], u[2], u[3]);
        } else {
            CT t0 = cadd(u[0], u[1]);
            u[1] = csub(u[0], u[1]);
            u[0] = t0;
        }
        const int base = ((j >> lgNs) << (lgNs + LGR)) + kk;
        const int g = gs[i];
        int la = 0, lb = 0;
        if (last) line_of<R, MODE>(a, line0 + g, la, lb);
#pragma unroll
        for (int r = 0; r < RAD; ++r) {
            const int k = base + (r << lgNs);
            if (last) fft_store<R, MODE>(a, la, lb, k, u[r]);
            else sm[COLS ? (k * G + g) : (g * K + k)] = u[r];
        }
    }
    __syncthreads();
}

// DIR = -1: forward transform (exp(-2 pi i kn / K)); DIR = +1: unnormalised inverse.
// LGK_ > 0: K = 2^LGK_ lines of G = 2^LGG_ per CTA fixed at compile time (the
// pass schedule and every index computation fold to constants); 0: generic.
template <typename R, int DIR, int MODE, int LGK_, int LGG_, int NREP = 1>
__global__ void __launch_bounds__(512, NREP > 1 ? 1 : (sizeof(R) == 4 ? 3 : 2)) k_fft(FftArgs<R> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx<R>* sm = reinterpret_cast<Cx<R>*>(smem_raw);
    if constexpr (LGK_ > 0) {
        constexpr int N8 = LGK_ / 3, REM = LGK_ % 3, NPASS = N8 + (REM ? 1 : 0);
        const int line0 = blockIdx.x << LGG_;
#pragma unroll
        for (int pass = 0; pass < NPASS; ++pass) {
            const bool first = (pass == 0), last = (pass == NPASS - 1);
            if (pass < N8) fft_pass<R, DIR, MODE, 8, 3, LGK_, LGG_, NREP>(a, sm, 3 * pass, first, last, line0);
            else if (REM == 2) fft_pass<R, DIR, MODE, 4, 2, LGK_, LGG_, NREP>(a, sm, 3 * pass, first, last, line0);
            else fft_pass<R, DIR, MODE, 2, 1, LGK_, LGG_, NREP>(a, sm, 3 * pass, first, last, line0);
        }
    } else {
        const int line0 = blockIdx.x * a.G;
        int lgNs = 0;
        for (int pass = 0; pass < a.npass; ++pass) {
            const bool first = (pass == 0), last = (pass == a.npass - 1);
            if (pass < a.n8) {
                fft_pass<R, DIR, MODE, 8, 3, 0, 0, 1>(a, sm, lgNs, first, last, line0);
                lgNs += 3;
            } else if (a.rlast == 4) {
                fft_pass<R, DIR, MODE, 4, 2, 0, 0, 1>(a, sm, lgNs, first, last, line0);
                lgNs += 2;
            } else {
                fft_pass<R, DIR, MODE, 2, 1, 0, 0, 1>(a, sm, lgNs, first, last, line0);
                lgNs += 1;
            }
        }
    }
}

// ---------------------------------------------------------------- mixed radix (K = r 2^m)
constexpr int MR_MAXPASS = 16;
struct MrPlan {
    int npass;
    int radix[MR_MAXPASS];
};

// Line index -> (channel, row or column), any K.
template <int MODE>
__device__ __forceinline__ void line_of_any(int line, int Kx, int ny, int& la, int& lb) {
    if (MODE == COL_FWD || MODE == COL_INV) {
        la = line / Kx;
        lb = line - la * Kx;
    } else {
        la = line / ny;
        lb = line - la * ny;
    }
}

// Self-sorting Stockham transform of G lines of length K = prod(radix) held in
// shared memory: pass with radix q and sub-transform length Ns reads
// x_t = in[j + t K/q] (t < q), multiplies by w_{Ns q}^{t (j mod Ns)}, takes the
// q-point DFT and writes it to out[(j / Ns) Ns q + (j mod Ns) + u Ns] (u < q);
// after all passes the lines are in natural order. Twiddles come from the
// K-point table w^m = exp(-2 pi i m / K) (conjugated for DIR = +1).
template <typename R, int DIR, int MODE>
__global__ void __launch_bounds__(512) k_fft_mr(FftArgs<R> a, MrPlan mp) {
    typedef Cx<R> CT;
    constexpr bool COLS = (MODE == COL_FWD || MODE == COL_INV);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int K = a.K, G = a.G, GK = G * K;
    CT* src = reinterpret_cast<CT*>(smem_raw);
    CT* dst = src + GK;
    const int line0 = blockIdx.x * G, tid = threadIdx.x, nthr = blockDim.x;
    for (int e = tid; e < GK; e += nthr) {   // consecutive threads: consecutive columns / row elements
        const int g = COLS ? e % G : e / K, k = COLS ? e / G : e % K;
        int la, lb;
        line_of_any<MODE>(line0 + g, a.Kx, a.ny, la, lb);
        src[g * K + k] = fft_load<R, MODE>(a, la, lb, k);
    }
    __syncthreads();
    auto tw = [&](int m) {
        CT t = a.tw[m];
        if (DIR > 0) t.y = -t.y;
        return t;
    };
    int Ns = 1;
    for (int pass = 0; pass < mp.npass; ++pass) {
        const int q = mp.radix[pass], nb = K / q, step = K / q;
        for (int e = tid; e < G * nb; e += nthr) {
            const int g = e / nb, j = e - g * nb;
            const int k = j % Ns;
            CT x[5], y[5];
#pragma unroll
            for (int t = 0; t < 5; ++t)
                if (t < q) x[t] = src[g * K + j + t * nb];
            if (Ns > 1) {
                const int tstep = K / (Ns * q);
#pragma unroll
                for (int t = 1; t < 5; ++t)
                    if (t < q) x[t] = cmul(x[t], tw(t * k * tstep));
            }
#pragma unroll
            for (int u = 0; u < 5; ++u) {
                if (u >= q) break;
                CT acc = x[0];
#pragma unroll
                for (int t = 1; t < 5; ++t)
                    if (t < q) acc = cadd(acc, cmul(x[t], tw(((u * t) % q) * step)));
                y[u] = acc;
            }
            const int base = (j / Ns) * Ns * q + k;
#pragma unroll
            for (int u = 0; u < 5; ++u)
                if (u < q) dst[g * K + base + u * Ns] = y[u];
        }
        __syncthreads();
        CT* t = src;
        src = dst;
        dst = t;
        Ns *= q;
    }
    for (int e = tid; e < GK; e += nthr) {
        const int g = COLS ? e % G : e / K, k = COLS ? e / G : e % K;
        int la, lb;
        line_of_any<MODE>(line0 + g, a.Kx, a.ny, la, lb);
        fft_store<R, MODE>(a, la, lb, k, src[g * K + k]);
    }
}

static bool mr_plan(int K, MrPlan* mp) {
    mp->npass = 0;
    for (int r : {5, 3}) {
        if (K % r == 0) {
            mp->radix[mp->npass++] = r;
            K /= r;
        }
    }
    while (K % 4 == 0 && mp->npass < MR_MAXPASS) {
        mp->radix[mp->npass++] = 4;
        K /= 4;
    }
    if (K == 2 && mp->npass < MR_MAXPASS) {
        mp->radix[mp->npass++] = 2;
        K = 1;
    }
    return K == 1;
}

static bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

static void radix_plan(int K, int* n8, int* rlast, int* npass) {
    int p = 0;
    while ((1 << p) < K) ++p;
    *n8 = p / 3;
    const int rem = p % 3;
    *rlast = rem == 0 ? 8 : (1 << rem);
    *npass = *n8 + (rem ? 1 : 0);
}

// nl channels starting at in / out (a channel range of the plan's cube).
template <typename R, int DIR, int MODE>
static hs_status launch_fft(Plan* p, const void* in, void* out, int nl, cudaStream_t s) {
    FftArgs<R> a;
    a.in = in;
    a.out = out;
    a.nx = p->g.nx;
    a.ny = p->g.ny;
    a.Kx = p->g.Kx;
    a.Ky = p->g.Ky;
    a.cxs = (const R*)p->cxs;
    a.cys = (const R*)p->cys;
    constexpr bool cols = (MODE == COL_FWD || MODE == COL_INV);
    const int K = cols ? p->g.Ky : p->g.Kx;
    a.K = K;
    a.tw = (const Cx<R>*)(cols ? p->twy : p->twx);
    if (!is_pow2(K) || !is_pow2(cols ? p->g.Kx : p->g.ny)) {   // mixed radix, generic indexing
        MrPlan mp;
        if (!mr_plan(K, &mp)) return fail(HS_ERR_ARG, "FFT: line length %d is not r 2^m with r in {1, 3, 5}", K);
        int G = 1;
        if (cols) {   // whole 32-byte sectors per column load where shared memory allows
            const int want = (int)(32 / sizeof(Cx<R>)) > 0 ? (int)(32 / sizeof(Cx<R>)) : 1;
            G = std::max(1, want);
            while (G > 1 && (p->g.Kx % G != 0 || (size_t)2 * G * K * sizeof(Cx<R>) > (size_t)200 * 1024)) G >>= 1;
        }
        a.G = G;
        const int nlines = nl * (cols ? p->g.Kx : p->g.ny);
        const size_t smem = (size_t)2 * G * K * sizeof(Cx<R>);
        if (smem > (size_t)200 * 1024) return fail(HS_ERR_ARG, "FFT: line length %d too long", K);
        k_fft_mr<R, DIR, MODE><<<nlines / G, 512, smem, s>>>(a, mp);
        HS_CHECK_LAUNCH();
        return HS_OK;
    }
    radix_plan(K, &a.n8, &a.rlast, &a.npass);
    auto lg2 = [](int v) {
        int r = 0;
        while ((1 << r) < v) ++r;
        return r;
    };
    a.lgK = lg2(K);
    a.lgny = lg2(p->g.ny);
    a.lgKx = lg2(p->g.Kx);
    int G, nlines, nrep = 1;
    if (cols) {
        // 512 threads per CTA so two CTAs share an SM (one loads while the other computes);
        // lines longer than 1024 come 4 to a CTA (2 for FP64 at 4096: shared memory) with
        // several butterflies per thread, so column loads use whole 32-byte sectors
        G = 512 / (K / 8);
        if (G > 16) G = 16;
        if (K >= 2048) {
            G = (sizeof(R) == 8 && K >= 4096) ? 2 : 4;
            nrep = G * K / 8 / 512;
        }
        if (G > p->g.Kx) G = p->g.Kx;
        nlines = nl * p->g.Kx;
    } else {
        G = 256 / (K / 8);
        if (G < 1) G = 1;
        if (G > p->g.ny) G = p->g.ny;
        nlines = nl * p->g.ny;
    }
    if (G < 1) G = 1;
    a.G = G;
    a.lgG = lg2(G);
    const int threads = G * K / 8 / nrep;
    const size_t smem = (size_t)G * K * sizeof(Cx<R>);
    const int blocks = nlines / G;
    if (blocks == 0) return HS_OK;
    // compile-time sizes for the common grids (G as chosen above for these K)
#define HS_FFT_CT(LK, LG) \
    if (a.lgK == LK && a.lgG == LG && nrep == 1) { \
        k_fft<R, DIR, MODE, LK, LG><<<blocks, threads, smem, s>>>(a); \
        HS_CHECK_LAUNCH(); \
        return HS_OK; \
    }
#define HS_FFT_CT_REP(LK, LG, NR) \
    if (a.lgK == LK && a.lgG == LG && nrep == NR) { \
        k_fft<R, DIR, MODE, LK, LG, NR><<<blocks, threads, smem, s>>>(a); \
        HS_CHECK_LAUNCH(); \
        return HS_OK; \
    }
    if constexpr (cols) {
        HS_FFT_CT(9, 3)
        HS_FFT_CT(10, 2)
        HS_FFT_CT_REP(11, 2, 2)
        if constexpr (sizeof(R) == 4) {
            HS_FFT_CT_REP(12, 2, 4)
        } else {
            HS_FFT_CT_REP(12, 1, 2)
        }
    } else {
        HS_FFT_CT(9, 2)
        HS_FFT_CT(10, 1)
        HS_FFT_CT(11, 0)
        HS_FFT_CT(12, 0)
    }
#undef HS_FFT_CT
#undef HS_FFT_CT_REP
    if (nrep != 1) return fail(HS_ERR_ARG, "FFT: no kernel for K = %d with %d lines per CTA", K, G);
    k_fft<R, DIR, MODE, 0, 0><<<blocks, threads, smem, s>>>(a);
    HS_CHECK_LAUNCH();
    return HS_OK;
}

template <typename R, int DIR, int MODE, int LK, int LG, int NR = 1> static hs_status fft_attr1() {
    HS_CHECK_CUDA(cudaFuncSetAttribute(k_fft<R, DIR, MODE, LK, LG, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       200 * 1024));
    return HS_OK;
}

template <typename R, int DIR, int MODE> static hs_status fft_attr() {
    constexpr bool cols = (MODE == COL_FWD || MODE == COL_INV);
    HS_CHECK_CUDA(cudaFuncSetAttribute(k_fft_mr<R, DIR, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       200 * 1024));
    HS_TRY((fft_attr1<R, DIR, MODE, 0, 0>()));
    HS_TRY((fft_attr1<R, DIR, MODE, 9, cols ? 3 : 2>()));
    HS_TRY((fft_attr1<R, DIR, MODE, 10, cols ? 2 : 1>()));
    if constexpr (cols) {
        HS_TRY((fft_attr1<R, DIR, MODE, 11, 2, 2>()));
        if constexpr (sizeof(R) == 4) {
            HS_TRY((fft_attr1<R, DIR, MODE, 12, 2, 4>()));
        } else {
            HS_TRY((fft_attr1<R, DIR, MODE, 12, 1, 2>()));
        }
    } else {
        HS_TRY((fft_attr1<R, DIR, MODE, 11, 0>()));
        HS_TRY((fft_attr1<R, DIR, MODE, 12, 0>()));
    }
    return HS_OK;
}

// Opt the FFT kernels into large dynamic shared memory (once per process, at
// plan creation, outside any stream capture).
static int64_t g_l2_bytes = 0;

hs_status fft_init() {
    static bool done = false;
    if (done) return HS_OK;
    int dev = 0, l2 = 0;
    HS_CHECK_CUDA(cudaGetDevice(&dev));
    HS_CHECK_CUDA(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev));
    g_l2_bytes = l2;
    HS_TRY((fft_attr<float, -1, ROW_FWD>()));
    HS_TRY((fft_attr<float, -1, COL_FWD>()));
    HS_TRY((fft_attr<float, 1, COL_INV>()));
    HS_TRY((fft_attr<float, 1, ROW_INV>()));
    HS_TRY((fft_attr<double, -1, ROW_FWD>()));
    HS_TRY((fft_attr<double, -1, COL_FWD>()));
    HS_TRY((fft_attr<double, 1, COL_INV>()));
    HS_TRY((fft_attr<double, 1, ROW_INV>()));
    done = true;
    return HS_OK;
}

hs_status fft_forward(Plan* p, const void* X, cudaStream_t s) {
    const int L = p->g.L;
    if (p->prec == HS_F32) {
        HS_TRY((launch_fft<float, -1, ROW_FWD>(p, X, p->tmp, L, s)));
        HS_TRY((launch_fft<float, -1, COL_FWD>(p, p->tmp, p->grid, L, s)));
    } else {
        HS_TRY((launch_fft<double, -1, ROW_FWD>(p, X, p->tmp, L, s)));
        HS_TRY((launch_fft<double, -1, COL_FWD>(p, p->tmp, p->grid, L, s)));
    }
    return HS_OK;
}

// Channels per adjoint chunk that keep a chunk's traffic within half the L2:
// the column pass of a chunk streams its grid (Ky Kx cells per channel) and
// writes the ny x Kx intermediate, which the row pass reads right after, so the
// intermediate can stay on chip instead of going through HBM and back. The row
// pass of chunk c runs on the plan's side stream, overlapping the column pass
// of chunk c + 1 (two chunks in flight fill the L2); the plan's autotuner keeps
// the chunked form only where it measures faster (p->fft_adj_chunk, default
// all channels).
int fft_adjoint_chunk(const Plan* p) {
    const int64_t per = ((int64_t)p->g.Ky * p->g.Kx + (int64_t)p->g.ny * p->g.Kx) * (int64_t)p->csize();
    const int64_t budget = g_l2_bytes > 0 ? g_l2_bytes / 2 : ((int64_t)32 << 20);
    return (int)std::max<int64_t>(1, std::min<int64_t>(p->g.L, budget / std::max<int64_t>(per, 1)));
}

hs_status fft_adjoint(Plan* p, void* X, cudaStream_t s) {
    const int L = p->g.L, C = std::max(1, std::min(L, p->fft_adj_chunk > 0 ? p->fft_adj_chunk : L));
    const int64_t gch = (int64_t)p->g.Ky * p->g.Kx, tch = (int64_t)p->g.ny * p->g.Kx, xch = p->N();
    const bool side = C < L && p->fft_side != nullptr;
    cudaStream_t s2 = side ? p->fft_side : s;
    for (int l0 = 0; l0 < L; l0 += C) {
        const int n = std::min(C, L - l0);
        if (p->prec == HS_F32) {
            const float2* g = (const float2*)p->grid + l0 * gch;
            float2* t = (float2*)p->tmp + l0 * tch;
            HS_TRY((launch_fft<float, 1, COL_INV>(p, g, t, n, s)));
            if (side) {
                HS_CHECK_CUDA(cudaEventRecord(p->fft_ev_col, s));
                HS_CHECK_CUDA(cudaStreamWaitEvent(s2, p->fft_ev_col, 0));
            }
            HS_TRY((launch_fft<float, 1, ROW_INV>(p, t, (float*)X + l0 * xch, n, s2)));
        } else {
            const double2* g = (const double2*)p->grid + l0 * gch;
            double2* t = (double2*)p->tmp + l0 * tch;
            HS_TRY((launch_fft<double, 1, COL_INV>(p, g, t, n, s)));
            if (side) {
                HS_CHECK_CUDA(cudaEventRecord(p->fft_ev_col, s));
                HS_CHECK_CUDA(cudaStreamWaitEvent(s2, p->fft_ev_col, 0));
            }
            HS_TRY((launch_fft<double, 1, ROW_INV>(p, t, (double*)X + l0 * xch, n, s2)));
        }
    }
    if (side) {
        HS_CHECK_CUDA(cudaEventRecord(p->fft_ev_join, s2));
        HS_CHECK_CUDA(cudaStreamWaitEvent(s, p->fft_ev_join, 0));
    }
    return HS_OK;
}

}  // namespace hs
