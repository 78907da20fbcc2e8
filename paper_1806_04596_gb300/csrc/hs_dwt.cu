// SARA dictionary (Sec. 2.3): Psi^dagger = [Dirac, db1, ..., db8]^dagger / 3.
//
// Each Daubechies basis is the periodic orthonormal 2-D DWT, computed level by
// level with separable filter kernels (no lifting): a row pass and a column
// pass per level, all 8 wavelets and all L channels in one launch per pass.
// One level on a length-m line (m even, indices mod m):
//   analysis   a[k] = sum_j h[j] x[2k + j],   d[k] = sum_j g[j] x[2k + j]
//   synthesis  x[i] = sum_{j = i mod 2} h[j] a[(i - j) / 2] + g[j] d[(i - j) / 2]
// with g[j] = (-1)^j h[F-1-j]. The synthesis is the transpose of the analysis,
// which also holds when the level is shorter than the filter (the periodic
// wrap is applied to the index, so taps that alias onto the same sample add).
// Coefficients use the Mallat layout in an ny x nx array per (basis, channel).
#include "hs_device.cuh"
#include "hs_internal.h"

namespace hs {

__constant__ float c_filt_f[NW][2][MAXF];
__constant__ double c_filt_d[NW][2][MAXF];

template <typename R> __device__ __forceinline__ R filt(int d, int hg, int j);
template <> __device__ __forceinline__ float filt<float>(int d, int hg, int j) { return c_filt_f[d][hg][j]; }
template <> __device__ __forceinline__ double filt<double>(int d, int hg, int j) { return c_filt_d[d][hg][j]; }

// Dirac basis: A[0][l] = X[l] / 3
template <typename R>
__global__ void k_scale_copy(const R* __restrict__ in, R* __restrict__ out, int64_t n, R s) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = s * in[i];
}

// Analysis row pass on the my x mx block of every (wavelet d, channel l).
// src: level 0 -> X (shared by all wavelets, scaled by 1/3); else the LL block of A[1+d].
template <typename R>
__global__ void k_dwt_rows_fwd(const R* __restrict__ X, const R* __restrict__ A, R* __restrict__ S,
                               int L, int ny, int nx, int my, int mx, int lev0, R s0) {
    const int dl = blockIdx.y;
    const int d = dl / L, l = dl - d * L;
    const int half = mx >> 1;
    const int64_t N = (int64_t)ny * nx;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)my * half) return;
    const int y = (int)(t / half), k = (int)(t - (int64_t)y * half);
    const R* row = lev0 ? X + (int64_t)l * N + (int64_t)y * nx
                        : A + ((int64_t)(1 + d) * L + l) * N + (int64_t)y * nx;
    const int F = 2 * (d + 1);
    R lo = 0, hi = 0;
    for (int j = 0; j < F; ++j) {
        const R xv = row[(2 * k + j) & (mx - 1)];
        lo = fma(filt<R>(d, 0, j), xv, lo);
        hi = fma(filt<R>(d, 1, j), xv, hi);
    }
    if (lev0) {
        lo *= s0;
        hi *= s0;
    }
    R* out = S + ((int64_t)d * L + l) * N + (int64_t)y * nx;
    out[k] = lo;
    out[half + k] = hi;
}

// Analysis column pass: S block -> A[1+d] block (top half low-pass, bottom high-pass).
template <typename R>
__global__ void k_dwt_cols_fwd(const R* __restrict__ S, R* __restrict__ A, int L, int ny, int nx,
                               int my, int mx) {
    const int dl = blockIdx.y;
    const int d = dl / L, l = dl - d * L;
    const int half = my >> 1;
    const int64_t N = (int64_t)ny * nx;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)half * mx) return;
    const int k = (int)(t / mx), x = (int)(t - (int64_t)k * mx);
    const R* col = S + ((int64_t)d * L + l) * N + x;
    const int F = 2 * (d + 1);
    R lo = 0, hi = 0;
    for (int j = 0; j < F; ++j) {
        const R v = col[(int64_t)((2 * k + j) & (my - 1)) * nx];
        lo = fma(filt<R>(d, 0, j), v, lo);
        hi = fma(filt<R>(d, 1, j), v, hi);
    }
    R* out = A + ((int64_t)(1 + d) * L + l) * N + x;
    out[(int64_t)k * nx] = lo;
    out[(int64_t)(half + k) * nx] = hi;
}

// Synthesis column pass on the my x mx block: the LL quadrant comes from `LLsrc`
// (A itself at the coarsest level, else the previous level's output T1), the
// detail quadrants from A[1+d]. Output T2 block.
template <typename R>
__global__ void k_dwt_cols_inv(const R* __restrict__ A, const R* __restrict__ T1, int ll_from_a,
                               R* __restrict__ T2, int L, int ny, int nx, int my, int mx) {
    const int dl = blockIdx.y;
    const int d = dl / L, l = dl - d * L;
    const int64_t N = (int64_t)ny * nx;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)my * mx) return;
    const int i = (int)(t / mx), x = (int)(t - (int64_t)i * mx);
    const int hy = my >> 1, hx = mx >> 1;
    const R* a_col = A + ((int64_t)(1 + d) * L + l) * N + x;
    const R* top = (x < hx && !ll_from_a) ? T1 + ((int64_t)d * L + l) * N + x : a_col;
    const int F = 2 * (d + 1);
    R acc = 0;
    for (int j = (i & 1); j < F; j += 2) {
        const int k = ((i - j) & (my - 1)) >> 1;
        acc = fma(filt<R>(d, 0, j), top[(int64_t)k * nx], acc);
        acc = fma(filt<R>(d, 1, j), a_col[(int64_t)(hy + k) * nx], acc);
    }
    T2[((int64_t)d * L + l) * N + (int64_t)i * nx + x] = acc;
}

// Synthesis row pass for levels > 0: T2 block -> T1 block.
template <typename R>
__global__ void k_dwt_rows_inv(const R* __restrict__ T2, R* __restrict__ T1, int L, int ny, int nx,
                               int my, int mx) {
    const int dl = blockIdx.y;
    const int d = dl / L, l = dl - d * L;
    const int64_t N = (int64_t)ny * nx;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)my * mx) return;
    const int y = (int)(t / mx), i = (int)(t - (int64_t)y * mx);
    const int hx = mx >> 1;
    const R* row = T2 + ((int64_t)d * L + l) * N + (int64_t)y * nx;
    const int F = 2 * (d + 1);
    R acc = 0;
    for (int j = (i & 1); j < F; j += 2) {
        const int k = ((i - j) & (mx - 1)) >> 1;
        acc = fma(filt<R>(d, 0, j), row[k], acc);
        acc = fma(filt<R>(d, 1, j), row[hx + k], acc);
    }
    T1[((int64_t)d * L + l) * N + (int64_t)y * nx + i] = acc;
}

// Level-0 synthesis row pass fused with the sum over the 9 bases:
// X[l] = (A[0][l] + sum_d W_d^T A[1+d][l]) / 3.
template <typename R>
__global__ void k_dwt_rows_inv_sum(const R* __restrict__ T2, const R* __restrict__ A,
                                   R* __restrict__ X, int L, int ny, int nx, R s) {
    const int64_t N = (int64_t)ny * nx;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)L * N) return;
    const int l = (int)(t / N);
    const int64_t pix = t - (int64_t)l * N;
    const int y = (int)(pix / nx), i = (int)(pix - (int64_t)y * nx);
    const int hx = nx >> 1;
    R acc = A[t];   // basis 0 (Dirac) of channel l
    for (int d = 0; d < NW; ++d) {
        const R* row = T2 + ((int64_t)d * L + l) * N + (int64_t)y * nx;
        const int F = 2 * (d + 1);
        for (int j = (i & 1); j < F; j += 2) {
            const int k = ((i - j) & (nx - 1)) >> 1;
            acc = fma(filt<R>(d, 0, j), row[k], acc);
            acc = fma(filt<R>(d, 1, j), row[hx + k], acc);
        }
    }
    X[t] = s * acc;
}

static hs_status upload_filters() {
    static bool done = false;
    if (done) return HS_OK;
    double hd[NW][2][MAXF] = {};
    float hf[NW][2][MAXF] = {};
    for (int d = 0; d < NW; ++d) {
        const int F = 2 * (d + 1);
        double h[MAXF];
        HS_TRY(daubechies_lowpass(d + 1, h));
        for (int j = 0; j < F; ++j) {
            hd[d][0][j] = h[j];
            hd[d][1][j] = (j & 1 ? -1.0 : 1.0) * h[F - 1 - j];
            hf[d][0][j] = (float)hd[d][0][j];
            hf[d][1][j] = (float)hd[d][1][j];
        }
    }
    HS_CHECK_CUDA(cudaMemcpyToSymbol(c_filt_d, hd, sizeof(hd)));
    HS_CHECK_CUDA(cudaMemcpyToSymbol(c_filt_f, hf, sizeof(hf)));
    done = true;
    return HS_OK;
}

hs_status dwt_init() { return upload_filters(); }

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <typename R> static hs_status analysis_t(Plan* p, const R* X, R* A, cudaStream_t s) {
    const int L = p->g.L, ny = p->g.ny, nx = p->g.nx;
    const int64_t N = p->N();
    R* S = (R*)p->dwt_a;
    const R third = (R)(1.0 / 3.0);
    k_scale_copy<R><<<nblk(L * N, 256) > 4096 ? 4096 : nblk(L * N, 256), 256, 0, s>>>(X, A, L * N, third);
    HS_CHECK_LAUNCH();
    for (int lev = 0; lev < p->levels; ++lev) {
        const int my = ny >> lev, mx = nx >> lev;
        dim3 g1(nblk((int64_t)my * (mx / 2), 256), NW * L);
        k_dwt_rows_fwd<R><<<g1, 256, 0, s>>>(X, A, S, L, ny, nx, my, mx, lev == 0, third);
        HS_CHECK_LAUNCH();
        dim3 g2(nblk((int64_t)(my / 2) * mx, 256), NW * L);
        k_dwt_cols_fwd<R><<<g2, 256, 0, s>>>(S, A, L, ny, nx, my, mx);
        HS_CHECK_LAUNCH();
    }
    return HS_OK;
}

template <typename R> static hs_status synthesis_t(Plan* p, const R* A, R* X, cudaStream_t s) {
    const int L = p->g.L, ny = p->g.ny, nx = p->g.nx;
    const int64_t N = p->N();
    R* T1 = (R*)p->dwt_a;
    R* T2 = (R*)p->dwt_b;
    for (int lev = p->levels - 1; lev >= 0; --lev) {
        const int my = ny >> lev, mx = nx >> lev;
        dim3 g1(nblk((int64_t)my * mx, 256), NW * L);
        k_dwt_cols_inv<R><<<g1, 256, 0, s>>>(A, T1, lev == p->levels - 1, T2, L, ny, nx, my, mx);
        HS_CHECK_LAUNCH();
        if (lev > 0) {
            k_dwt_rows_inv<R><<<g1, 256, 0, s>>>(T2, T1, L, ny, nx, my, mx);
        } else {
            k_dwt_rows_inv_sum<R><<<nblk((int64_t)L * N, 256), 256, 0, s>>>(T2, A, X, L, ny, nx,
                                                                            (R)(1.0 / 3.0));
        }
        HS_CHECK_LAUNCH();
    }
    return HS_OK;
}

hs_status dwt_analysis(Plan* p, const void* X, void* A, cudaStream_t s) {
    if (p->prec == HS_F32) return analysis_t<float>(p, (const float*)X, (float*)A, s);
    return analysis_t<double>(p, (const double*)X, (double*)A, s);
}

hs_status dwt_synthesis(Plan* p, const void* A, void* X, cudaStream_t s) {
    if (p->prec == HS_F32) return synthesis_t<float>(p, (const float*)A, (float*)X, s);
    return synthesis_t<double>(p, (const double*)A, (double*)X, s);
}

}  // namespace hs
