// SARA dictionary (Sec. 2.3): Psi^dagger = [Dirac, db1, ..., db8]^dagger / 3.
//
// Each Daubechies basis is the periodic orthonormal 2-D DWT, computed level by
// level with separable filter kernels (no lifting). One launch per level does
// both separable passes for all 8 wavelets and all L channels: a CTA loads a
// tile of the level's input with its periodic halo into shared memory, filters
// the rows, then the columns, and writes the four subbands once (analysis), or
// loads the four subband tiles with halo and reconstructs a 2q x 2q output tile
// (synthesis). The last synthesis level also sums the 9 bases.
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

constexpr int DQ = 16;                    // coefficients per subband and axis in one tile
constexpr int DIN = 2 * DQ + MAXF - 2;    // analysis input region side (46)
constexpr int DC = DQ + MAXF / 2 - 1;     // synthesis coefficient region side (23)

// One analysis level for every (wavelet d, channel l). Input: the my x mx block
// (level 0: X / 3, row stride nx; otherwise the previous level's LL, compact
// with stride mx, in `src`). The three detail subbands go to A[1+d] at their
// Mallat positions (stride nx); LL goes to `ll_out` (compact, stride mx / 2),
// or to A[1+d] at the last level. 256 threads as 8 rows of 32 lanes.
template <typename R>
__global__ void __launch_bounds__(256) k_dwt_fwd_level(const R* __restrict__ X, const R* __restrict__ src,
                                                      R* __restrict__ A, R* __restrict__ ll_out, int L,
                                                      int ny, int nx, int my, int mx, int lev0, int last,
                                                      R s0) {
    __shared__ R in[DIN][DIN + 1];
    __shared__ R ro[DIN][2 * DQ + 1];
    const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
    const int d = blockIdx.y / L, l = blockIdx.y - d * L;
    const int F = 2 * (d + 1);
    const int hy = my >> 1, hx = mx >> 1;
    const int qy = min(DQ, hy), qx = min(DQ, hx);
    const int ntx = hx / qx;
    const int ty = blockIdx.x / ntx, tx = blockIdx.x - ty * ntx;
    const int k0y = ty * qy, k0x = tx * qx;
    const int ry = 2 * qy + F - 2, rx = 2 * qx + F - 2;
    const int64_t N = (int64_t)ny * nx;
    const R* base;
    int64_t stride;
    if (lev0) {
        base = X + (int64_t)l * N;
        stride = nx;
    } else {
        base = src + ((int64_t)d * L + l) * (int64_t)my * mx;
        stride = mx;
    }
    const R sc = lev0 ? s0 : (R)1;
    for (int r = wy; r < ry; r += 8) {
        const R* row = base + (int64_t)((2 * k0y + r) & (my - 1)) * stride;
        for (int c = lane; c < rx; c += 32) in[r][c] = sc * row[(2 * k0x + c) & (mx - 1)];
    }
    __syncthreads();
    {   // rows: lanes 0-15 row r, lanes 16-31 row r + 1; lane computes both halves
        const int c = lane & (DQ - 1), rofs = lane >> 4;
        if (c < qx)
            for (int r = 2 * wy + rofs; r < ry; r += 16) {
                R lo = 0, hi = 0;
                for (int j = 0; j < F; ++j) {
                    const R v = in[r][2 * c + j];
                    lo = fma(filt<R>(d, 0, j), v, lo);
                    hi = fma(filt<R>(d, 1, j), v, hi);
                }
                ro[r][c] = lo;
                ro[r][qx + c] = hi;
            }
    }
    __syncthreads();
    R* Ad = A + ((int64_t)(1 + d) * L + l) * N;
    R* LLo = last ? Ad : ll_out + ((int64_t)d * L + l) * (int64_t)hy * hx;
    const int64_t lls = last ? nx : hx;
    if (lane < 2 * qx) {   // columns + stores: lane = output column of the row-filtered tile
        const bool xlow = lane < qx;
        const int ox = xlow ? k0x + lane : hx + k0x + (lane - qx);
        for (int r = wy; r < qy; r += 8) {
            R lo = 0, hi = 0;
            for (int j = 0; j < F; ++j) {
                const R v = ro[2 * r + j][lane];
                lo = fma(filt<R>(d, 0, j), v, lo);
                hi = fma(filt<R>(d, 1, j), v, hi);
            }
            const int oy = k0y + r;
            if (xlow) LLo[(int64_t)oy * lls + ox] = lo;
            else Ad[(int64_t)oy * nx + ox] = lo;
            Ad[(int64_t)(hy + oy) * nx + ox] = hi;
        }
    }
}

// Loads the four subband tiles (with the periodic halo of the synthesis
// filters) of one (d, l) and reconstructs the 2q x 2q output tile; thread
// (lane, wy) accumulates output rows wy, wy + 8, ... (up to 4) at column lane.
template <typename R>
__device__ __forceinline__ void dwt_inv_tile(const R* __restrict__ Ad, const R* __restrict__ ll,
                                             int64_t lls, int d, int nx, int my, int mx, int ty, int tx,
                                             R (*cf)[DC][DC + 1], R (*cl)[2][DC + 1], R* acc) {
    const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
    const int F = 2 * (d + 1);
    const int hy = my >> 1, hx = mx >> 1;
    const int qy = min(DQ, hy), qx = min(DQ, hx);
    const int h2 = F / 2 - 1;
    const int cyn = qy + h2, cxn = qx + h2;
    const int ky0 = ty * qy - h2, kx0 = tx * qx - h2;
    __syncthreads();   // previous use of cf / cl is finished
    for (int q = 0; q < 4; ++q) {
        const int yb = q >> 1, xb = q & 1;
        for (int yy = wy; yy < cyn; yy += 8) {
            const int gy = (ky0 + yy) & (hy - 1);
            const R* row = (q == 0) ? ll + (int64_t)gy * lls : Ad + (int64_t)(yb * hy + gy) * nx + xb * hx;
            for (int xx = lane; xx < cxn; xx += 32) cf[q][yy][xx] = row[(kx0 + xx) & (hx - 1)];
        }
    }
    __syncthreads();
    // columns: output row i (0..2qy), coefficient column xx, x-half b
    for (int i = wy; i < 2 * qy; i += 8)
        for (int xx = lane; xx < 2 * cxn; xx += 32) {
            const int b = xx >= cxn, x = xx - b * cxn;
            R v = 0;
            for (int j = (i & 1); j < F; j += 2) {
                const int kk = ((i - j) >> 1) + h2;
                v = fma(filt<R>(d, 0, j), cf[b][kk][x], v);
                v = fma(filt<R>(d, 1, j), cf[2 + b][kk][x], v);
            }
            cl[i][b][x] = v;
        }
    __syncthreads();
    if (lane < 2 * qx) {
        const int c = lane;
#pragma unroll
        for (int e = 0; e < 4; ++e) {   // rows
            const int i = wy + 8 * e;
            if (i >= 2 * qy) break;
            R v = 0;
            for (int j = (c & 1); j < F; j += 2) {
                const int kk = ((c - j) >> 1) + h2;
                v = fma(filt<R>(d, 0, j), cl[i][0][kk], v);
                v = fma(filt<R>(d, 1, j), cl[i][1][kk], v);
            }
            acc[e] += v;
        }
    }
}

// One synthesis level > 0 for every (d, l): reconstructs the my x mx block
// (compact, stride mx, into `out`) from its LL (`ll`: A[1+d] at the coarsest
// level, else the coarser level's output, compact stride mx / 2) and A[1+d].
template <typename R>
__global__ void __launch_bounds__(256) k_dwt_inv_level(const R* __restrict__ A, const R* __restrict__ llbuf,
                                                      int ll_from_a, R* __restrict__ out, int L, int ny,
                                                      int nx, int my, int mx) {
    __shared__ R cf[4][DC][DC + 1];
    __shared__ R cl[2 * DQ][2][DC + 1];
    const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
    const int d = blockIdx.y / L, l = blockIdx.y - d * L;
    const int hy = my >> 1, hx = mx >> 1;
    const int qy = min(DQ, hy), qx = min(DQ, hx);
    const int ntx = hx / qx;
    const int ty = blockIdx.x / ntx, tx = blockIdx.x - ty * ntx;
    const int64_t N = (int64_t)ny * nx;
    const R* Ad = A + ((int64_t)(1 + d) * L + l) * N;
    const R* ll = ll_from_a ? Ad : llbuf + ((int64_t)d * L + l) * (int64_t)hy * hx;
    const int64_t lls = ll_from_a ? nx : hx;
    R acc[4] = {0, 0, 0, 0};
    dwt_inv_tile<R>(Ad, ll, lls, d, nx, my, mx, ty, tx, cf, cl, acc);
    R* o = out + ((int64_t)d * L + l) * (int64_t)my * mx;
    if (lane < 2 * qx)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int i = wy + 8 * e;
            if (i >= 2 * qy) break;
            o[(int64_t)(2 * ty * qy + i) * mx + 2 * tx * qx + lane] = acc[e];
        }
}

// Level-0 synthesis summed over the 9 bases: X[l] = (A[0][l] + sum_d W_d^T A[1+d][l]) / 3.
// One CTA per (channel, output tile); the wavelets are accumulated in registers.
template <typename R>
__global__ void __launch_bounds__(256) k_dwt_inv_level0_sum(const R* __restrict__ A, const R* __restrict__ llbuf,
                                                           int ll_from_a, R* __restrict__ X, int L, int ny,
                                                           int nx, R s) {
    __shared__ R cf[4][DC][DC + 1];
    __shared__ R cl[2 * DQ][2][DC + 1];
    const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
    const int l = blockIdx.y;
    const int hy = ny >> 1, hx = nx >> 1;
    const int qy = min(DQ, hy), qx = min(DQ, hx);
    const int ntx = hx / qx;
    const int ty = blockIdx.x / ntx, tx = blockIdx.x - ty * ntx;
    const int64_t N = (int64_t)ny * nx;
    R acc[4] = {0, 0, 0, 0};
    for (int d = 0; d < NW; ++d) {
        const R* Ad = A + ((int64_t)(1 + d) * L + l) * N;
        const R* ll = ll_from_a ? Ad : llbuf + ((int64_t)d * L + l) * (int64_t)hy * hx;
        const int64_t lls = ll_from_a ? nx : hx;
        dwt_inv_tile<R>(Ad, ll, lls, d, nx, ny, nx, ty, tx, cf, cl, acc);
    }
    const R* A0 = A + (int64_t)l * N;
    R* o = X + (int64_t)l * N;
    if (lane < 2 * qx)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int i = wy + 8 * e;
            if (i >= 2 * qy) break;
            const int64_t idx = (int64_t)(2 * ty * qy + i) * nx + 2 * tx * qx + lane;
            o[idx] = s * (acc[e] + A0[idx]);
        }
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

static inline unsigned ntiles(int my, int mx) {
    const int hy = my >> 1, hx = mx >> 1;
    const int qy = hy < DQ ? hy : DQ, qx = hx < DQ ? hx : DQ;
    return (unsigned)((hy / qy) * (hx / qx));
}

template <typename R> static hs_status analysis_t(Plan* p, const R* X, R* A, cudaStream_t s) {
    const int L = p->g.L, ny = p->g.ny, nx = p->g.nx;
    const int64_t N = p->N();
    R* buf[2] = {(R*)p->dwt_a, (R*)p->dwt_b};
    const R third = (R)(1.0 / 3.0);
    const unsigned gs = nblk(L * N, 256);
    k_scale_copy<R><<<gs > 4096 ? 4096 : gs, 256, 0, s>>>(X, A, L * N, third);
    HS_CHECK_LAUNCH();
    for (int lev = 0; lev < p->levels; ++lev) {
        const int my = ny >> lev, mx = nx >> lev;
        dim3 g(ntiles(my, mx), NW * L);
        k_dwt_fwd_level<R><<<g, 256, 0, s>>>(X, lev ? buf[(lev - 1) & 1] : nullptr, A, buf[lev & 1], L, ny,
                                             nx, my, mx, lev == 0, lev == p->levels - 1, third);
        HS_CHECK_LAUNCH();
    }
    return HS_OK;
}

template <typename R> static hs_status synthesis_t(Plan* p, const R* A, R* X, cudaStream_t s) {
    const int L = p->g.L, ny = p->g.ny, nx = p->g.nx;
    R* buf[2] = {(R*)p->dwt_a, (R*)p->dwt_b};
    const int top = p->levels - 1;
    for (int lev = top; lev >= 1; --lev) {
        const int my = ny >> lev, mx = nx >> lev;
        dim3 g(ntiles(my, mx), NW * L);
        k_dwt_inv_level<R><<<g, 256, 0, s>>>(A, lev == top ? nullptr : buf[(lev + 1) & 1], lev == top,
                                             buf[lev & 1], L, ny, nx, my, mx);
        HS_CHECK_LAUNCH();
    }
    dim3 g0(ntiles(ny, nx), L);
    k_dwt_inv_level0_sum<R><<<g0, 256, 0, s>>>(A, top == 0 ? nullptr : buf[1], top == 0, X, L, ny, nx,
                                               (R)(1.0 / 3.0));
    HS_CHECK_LAUNCH();
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
