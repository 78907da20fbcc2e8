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

constexpr int DQ = 16;                    // coefficients per subband and axis in one tile
constexpr int DIN = 2 * DQ + MAXF - 2;    // analysis input region side (46)
constexpr int SIN = DIN + 4;              // its row stride (50: pair loads hit distinct banks)
constexpr int SRO = 48;                   // row-filtered tile stride: lowpass at 0, highpass at 16
constexpr int DC = DQ + MAXF / 2 - 1;     // synthesis coefficient region side (23)
constexpr int SCF = 24;                   // row stride of the column-filtered halves
constexpr int SCS = 28;                   // row stride of the staged coefficients (16-byte chunks)
constexpr int SCL = 2 * SCF + 1;          // column-filtered tile stride (x-lowpass at 0, highpass at 24)
constexpr int FWD_SMEM = DIN * SIN + 2 * DIN * SRO;        // reals
constexpr int INV_SMEM = 2 * 4 * DC * SCS + 2 * DQ * SCL;  // reals
static_assert(2 * DQ * (DQ * 2 + 1) <= 2 * DQ * SCL, "output transpose fits the column tile");

// Runs CALL(D) for the runtime wavelet index d (0..7) with D a compile-time
// constant, so every filter loop unrolls with constant taps.
#define HS_DWT_DISPATCH(d, CALL)  \
    switch (d) {                  \
        case 0: CALL(0); break;   \
        case 1: CALL(1); break;   \
        case 2: CALL(2); break;   \
        case 3: CALL(3); break;   \
        case 4: CALL(4); break;   \
        case 5: CALL(5); break;   \
        case 6: CALL(6); break;   \
        default: CALL(7); break;  \
    }

// ---- asynchronous global -> shared staging (the halo loads never stall a warp)
template <typename R> __device__ __forceinline__ void cp_async(R* dst, const R* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if constexpr (sizeof(R) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <typename R> __device__ __forceinline__ Cx<R> ld2(const R* p) { return *reinterpret_cast<const Cx<R>*>(p); }
__device__ __forceinline__ void st4(float* p, float a, float b, float c, float d) {
    *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}
__device__ __forceinline__ void st4(double* p, double a, double b, double c, double d) {
    reinterpret_cast<double2*>(p)[0] = make_double2(a, b);
    reinterpret_cast<double2*>(p)[1] = make_double2(c, d);
}

// x mod n for x in [-n, 2n): the mask when every level of the image is a power
// of two (P2, the common case, a compile-time choice), else one conditional
// correction each way (sides 3 or 5 times a power of two).
template <bool P2> __device__ __forceinline__ int wrapp(int x, int n) {
    if constexpr (P2) {
        return x & (n - 1);
    } else {
        x += x < 0 ? n : 0;
        return x >= n ? x - n : x;
    }
}

// Stages rows [y0, y0 + ry) x columns [x0, x0 + rx) of a periodic ysz x xsz
// block (indices wrapped with wrapp; y0, x0 >= 0 and the region shorter than
// the block) into in[r * SIN + c].
// FP32 with an 8-byte aligned block (`pairs`): x0, rx and the block width are
// even, so columns move as 8-byte pairs that never straddle the periodic wrap.
template <typename R, bool P2>
__device__ __forceinline__ void stage_region(R* in, const R* __restrict__ base, int64_t stride, int ysz,
                                             int xsz, int y0, int x0, int ry, int rx, bool pairs) {
    const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
    if (sizeof(R) == 4 && pairs) {
        for (int r = wy; r < ry; r += 8) {
            const R* row = base + (int64_t)wrapp<P2>(y0 + r, ysz) * stride;
            for (int c = 2 * lane; c < rx; c += 64) cp_async8(in + r * SIN + c, row + wrapp<P2>(x0 + c, xsz));
        }
    } else {
        for (int r = wy; r < ry; r += 8) {
            const R* row = base + (int64_t)wrapp<P2>(y0 + r, ysz) * stride;
            for (int c = lane; c < rx; c += 32) cp_async(in + r * SIN + c, row + wrapp<P2>(x0 + c, xsz));
        }
    }
    cp_async_commit();
}

// Analysis along x of wavelet D (F = 2D + 2 taps): thread (r, g) filters input
// row r into the 4 lowpass and 4 highpass outputs 4g .. 4g + 3, reading the
// F + 6 inputs they share once, as pairs.
template <typename R, int D>
__device__ __forceinline__ void fwd_rows(const R* __restrict__ in, R* __restrict__ ro, int ry, int qx) {
    constexpr int F = 2 * (D + 1);
    constexpr int NV = F + 6;
    const int r = threadIdx.x >> 2, g = threadIdx.x & 3;
    if (r >= ry || 4 * g >= qx) return;
    R v[NV];
    const R* p = in + r * SIN + 8 * g;
#pragma unroll
    for (int k = 0; k < NV / 2; ++k) {
        const Cx<R> t = ld2(p + 2 * k);
        v[2 * k] = t.x;
        v[2 * k + 1] = t.y;
    }
    R lo[4], hi[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        R a = 0, b = 0;
#pragma unroll
        for (int j = 0; j < F; ++j) {
            a = fma(filt<R>(D, 0, j), v[2 * u + j], a);
            b = fma(filt<R>(D, 1, j), v[2 * u + j], b);
        }
        lo[u] = a;
        hi[u] = b;
    }
    st4(ro + r * SRO + 4 * g, lo[0], lo[1], lo[2], lo[3]);
    st4(ro + r * SRO + 16 + 4 * g, hi[0], hi[1], hi[2], hi[3]);
}

// Analysis along y of the row-filtered tile and the subband stores: thread
// (col, g) makes output rows 2g, 2g + 1 of tile column col (0-15: x-lowpass,
// 16-31: x-highpass), lowpass and highpass in y, scaled by sc.
template <typename R, int D>
__device__ __forceinline__ void fwd_cols(const R* __restrict__ ro, R sc, R* __restrict__ Ad,
                                         R* __restrict__ LLo, int64_t lls, int nx, int hy, int hx, int k0y,
                                         int k0x, int qy, int qx) {
    constexpr int F = 2 * (D + 1);
    constexpr int NV = F + 2;
    const int col = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int c = col & 15;
    const bool xhi = col >= 16;
    if (c >= qx || 2 * g >= qy) return;
    R v[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = ro[(4 * g + k) * SRO + col];
    R lo0 = 0, hi0 = 0, lo1 = 0, hi1 = 0;
#pragma unroll
    for (int j = 0; j < F; ++j) {
        lo0 = fma(filt<R>(D, 0, j), v[j], lo0);
        hi0 = fma(filt<R>(D, 1, j), v[j], hi0);
        lo1 = fma(filt<R>(D, 0, j), v[j + 2], lo1);
        hi1 = fma(filt<R>(D, 1, j), v[j + 2], hi1);
    }
    const int oy = k0y + 2 * g;
    const bool two = 2 * g + 1 < qy;
    if (xhi) {
        R* o = Ad + (int64_t)oy * nx + hx + k0x + c;
        o[0] = sc * lo0;
        if (two) o[nx] = sc * lo1;
    } else {
        R* o = LLo + (int64_t)oy * lls + k0x + c;
        o[0] = sc * lo0;
        if (two) o[lls] = sc * lo1;
    }
    R* o = Ad + (int64_t)(hy + oy) * nx + (xhi ? hx : 0) + k0x + c;
    o[0] = sc * hi0;
    if (two) o[nx] = sc * hi1;
}

template <typename R> struct FwdCtx {
    const R* in;
    R* ro;
    R* A;
    R* ll_out;
    int64_t N;
    int L, l, nx, hy, hx, k0y, k0x, qy, qx, last;
    R sc;
};

// All eight wavelets of level 0 from the one staged input tile; the
// row-filtered tile is double-buffered, so one barrier per wavelet suffices.
template <typename R, int D> __device__ __forceinline__ void fwd_all(const FwdCtx<R>& c) {
    if constexpr (D < NW) {
        constexpr int F = 2 * (D + 1);
        R* rb = c.ro + (D & 1) * DIN * SRO;
        fwd_rows<R, D>(c.in, rb, 2 * c.qy + F - 2, c.qx);
        __syncthreads();
        R* Ad = c.A + ((int64_t)(1 + D) * c.L + c.l) * c.N;
        R* LLo = c.last ? Ad : c.ll_out + ((int64_t)D * c.L + c.l) * (int64_t)c.hy * c.hx;
        fwd_cols<R, D>(rb, c.sc, Ad, LLo, c.last ? c.nx : c.hx, c.nx, c.hy, c.hx, c.k0y, c.k0x, c.qy, c.qx);
        fwd_all<R, D + 1>(c);
    }
}

// Level 0 of Psi^dagger for one (output tile, channel): the Dirac block
// A[0] = X / 3 and the first level of all 8 wavelets. LL goes to the compact
// buffer ll_out (stride nx / 2), or to A[1+d] when there is a single level.
template <typename R, bool P2>
__global__ void __launch_bounds__(256) k_psi_fwd_l0(const R* __restrict__ X, R* __restrict__ A,
                                                   R* __restrict__ ll_out, int L, int ny, int nx, int last,
                                                   R sc, int pairs) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* in = reinterpret_cast<R*>(smem_raw);
    const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
    const int l = blockIdx.y;
    const int hy = ny >> 1, hx = nx >> 1;
    const int qy = min(DQ, hy), qx = min(DQ, hx);
    const int ntx = hx / qx;
    const int ty = blockIdx.x / ntx, tx = blockIdx.x - ty * ntx;
    const int k0y = ty * qy, k0x = tx * qx;
    const int64_t N = (int64_t)ny * nx;
    stage_region<R, P2>(in, X + l * N, nx, ny, nx, 2 * k0y, 2 * k0x, 2 * qy + MAXF - 2, 2 * qx + MAXF - 2,
                 pairs != 0);
    cp_async_wait<0>();
    __syncthreads();
    R* A0 = A + l * N + (int64_t)(2 * k0y) * nx + 2 * k0x;
    for (int r = wy; r < 2 * qy; r += 8)
        if (lane < 2 * qx) A0[(int64_t)r * nx + lane] = sc * in[r * SIN + lane];
    FwdCtx<R> c{in, in + DIN * SIN, A, ll_out, N, L, l, nx, hy, hx, k0y, k0x, qy, qx, last, sc};
    fwd_all<R, 0>(c);
}

// One analysis level > 0 for every (wavelet d, channel l): input the previous
// level's LL (compact my x mx in `src`); details to A[1+d] at their Mallat
// positions, LL to `ll_out` (compact) or to A[1+d] at the last level.
template <typename R, bool P2>
__global__ void __launch_bounds__(256) k_dwt_fwd_level(const R* __restrict__ src, R* __restrict__ A,
                                                      R* __restrict__ ll_out, int L, int ny, int nx, int my,
                                                      int mx, int last) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* in = reinterpret_cast<R*>(smem_raw);
    R* ro = in + DIN * SIN;
    const int d = blockIdx.y / L, l = blockIdx.y - d * L;
    const int hy = my >> 1, hx = mx >> 1;
    const int qy = min(DQ, hy), qx = min(DQ, hx);
    const int ntx = hx / qx;
    const int ty = blockIdx.x / ntx, tx = blockIdx.x - ty * ntx;
    const int k0y = ty * qy, k0x = tx * qx;
    const int64_t N = (int64_t)ny * nx;
    const R* base = src + ((int64_t)d * L + l) * (int64_t)my * mx;
    R* Ad = A + ((int64_t)(1 + d) * L + l) * N;
    R* LLo = last ? Ad : ll_out + ((int64_t)d * L + l) * (int64_t)hy * hx;
    const int64_t lls = last ? nx : hx;
#define HS_FWD(DD)                                                                                       \
    {                                                                                                    \
        constexpr int F = 2 * (DD + 1);                                                                  \
        stage_region<R, P2>(in, base, mx, my, mx, 2 * k0y, 2 * k0x, 2 * qy + F - 2, 2 * qx + F - 2, true); \
        cp_async_wait<0>();                                                                              \
        __syncthreads();                                                                                 \
        fwd_rows<R, DD>(in, ro, 2 * qy + F - 2, qx);                                                     \
        __syncthreads();                                                                                 \
        fwd_cols<R, DD>(ro, (R)1, Ad, LLo, lls, nx, hy, hx, k0y, k0x, qy, qx);                           \
    }
    HS_DWT_DISPATCH(d, HS_FWD)
#undef HS_FWD
}

// ---- synthesis
// Column offset of a staged coefficient tile: the staged columns start at the
// 16-byte boundary at or below the tile's first column kx0 = t q - D, which is
// kx0 - inv_co columns (q is a multiple of the chunk, or the tile is alone).
template <typename R, int D> __host__ __device__ constexpr int inv_co() {
    constexpr int EPC = 16 / (int)sizeof(R);
    return (EPC - D % EPC) % EPC;
}

// Stages the four subband regions of one (d, l) tile: rows ky0 .. ky0 + cyn
// and columns kx0 .. kx0 + cxn (periodic) into cf[s][row][CO + col], s = 2 yb + xb;
// subband 0 (LL) comes from `ll` (row stride lls). With 16-byte aligned
// coefficients (`chunks`), subbands at least one 16-byte chunk wide move in
// aligned chunks (which never straddle the wrap).
template <typename R, int CO, bool P2>
__device__ __forceinline__ void inv_stage(R* cf, const R* __restrict__ Ad, const R* __restrict__ ll,
                                          int64_t lls, int nx, int hy, int hx, int ky0, int kx0, int cyn,
                                          int cxn, bool chunks) {
    constexpr int EPC = 16 / (int)sizeof(R);   // reals per chunk
    constexpr int LPR = EPC == 4 ? 8 : 16;     // lanes per staged row (chunks per row <= LPR)
    const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
    if (chunks && hx >= EPC) {
        const int nch = (cxn + CO + EPC - 1) / EPC;
        const int cc = lane % LPR, rr = lane / LPR;
        const int gx = wrapp<P2>(kx0 - CO + EPC * cc, hx);
        if (cc < nch) {
#pragma unroll
            for (int s = 0; s < 4; ++s)
                for (int yy = (32 / LPR) * wy + rr; yy < cyn; yy += 8 * (32 / LPR)) {
                    const int gy = wrapp<P2>(ky0 + yy, hy);
                    const R* src = (s == 0) ? ll + (int64_t)gy * lls + gx
                                            : Ad + (int64_t)((s >> 1) * hy + gy) * nx + (s & 1) * hx + gx;
                    cp_async16(cf + (s * DC + yy) * SCS + EPC * cc, src);
                }
        }
    } else if (lane < cxn) {
        const int gx = wrapp<P2>(kx0 + lane, hx);
#pragma unroll
        for (int s = 0; s < 4; ++s)
            for (int yy = wy; yy < cyn; yy += 8) {
                const int gy = wrapp<P2>(ky0 + yy, hy);
                const R* src = (s == 0) ? ll + (int64_t)gy * lls + gx
                                        : Ad + (int64_t)((s >> 1) * hy + gy) * nx + (s & 1) * hx + gx;
                cp_async(cf + (s * DC + yy) * SCS + CO + lane, src);
            }
    }
    cp_async_commit();
}

// Synthesis along y: thread (x, b, mg) makes rows 2m, 2m + 1 for m = 4mg .. 4mg + 3
// of column x of the x-lowpass (b = 0) or x-highpass (b = 1) half. Output row
// 2m + p takes taps h[2k + p], g[2k + p] on coefficient rows m - k.
template <typename R, int D>
__device__ __forceinline__ void inv_cols(const R* __restrict__ cf, R* __restrict__ cl, int qy, int cxn) {
    constexpr int H = D + 1;   // taps per parity
    constexpr int NV = H + 3;
    const int x = threadIdx.x & 31, b = (threadIdx.x >> 5) & 1, m0 = 4 * (threadIdx.x >> 6);
    if (x >= cxn || m0 >= qy) return;
    R a[NV], e[NV];
#pragma unroll
    for (int t = 0; t < NV; ++t) {
        a[t] = cf[(b * DC + m0 + t) * SCS + inv_co<R, D>() + x];
        e[t] = cf[((2 + b) * DC + m0 + t) * SCS + inv_co<R, D>() + x];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        R v0 = 0, v1 = 0;
#pragma unroll
        for (int k = 0; k < H; ++k) {
            const int t = u - k + H - 1;
            v0 = fma(filt<R>(D, 0, 2 * k), a[t], v0);
            v0 = fma(filt<R>(D, 1, 2 * k), e[t], v0);
            v1 = fma(filt<R>(D, 0, 2 * k + 1), a[t], v1);
            v1 = fma(filt<R>(D, 1, 2 * k + 1), e[t], v1);
        }
        if (m0 + u < qy) {
            cl[(2 * (m0 + u)) * SCL + b * SCF + x] = v0;
            cl[(2 * (m0 + u) + 1) * SCL + b * SCF + x] = v1;
        }
    }
}

// Synthesis along x, accumulated: thread (i, ng) adds output columns
// 4ng .. 4ng + 3 of tile row i into acc.
template <typename R, int D>
__device__ __forceinline__ void inv_rows(const R* __restrict__ cl, R* acc, int qy, int qx) {
    constexpr int H = D + 1;
    constexpr int NV = H + 1;
    const int i = threadIdx.x & 31, n0 = 2 * (threadIdx.x >> 5);
    if (i >= 2 * qy || n0 >= qx) return;
    R a[NV], e[NV];
#pragma unroll
    for (int t = 0; t < NV; ++t) {
        a[t] = cl[i * SCL + n0 + t];
        e[t] = cl[i * SCL + SCF + n0 + t];
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        R v0 = 0, v1 = 0;
#pragma unroll
        for (int k = 0; k < H; ++k) {
            const int t = u - k + H - 1;
            v0 = fma(filt<R>(D, 0, 2 * k), a[t], v0);
            v0 = fma(filt<R>(D, 1, 2 * k), e[t], v0);
            v1 = fma(filt<R>(D, 0, 2 * k + 1), a[t], v1);
            v1 = fma(filt<R>(D, 1, 2 * k + 1), e[t], v1);
        }
        acc[2 * u] += v0;
        acc[2 * u + 1] += v1;
    }
}

// Writes the 2qy x 2qx tile held in acc (thread (i, ng): row i, columns
// 4ng .. 4ng + 3) through the shared transpose buffer T with coalesced rows:
// out[r * stride + c] = s * (T[r][c] + (add ? add[r * stride + c] : 0)).
template <typename R>
__device__ __forceinline__ void tile_store(R* T, const R* acc, R* __restrict__ out, const R* __restrict__ add,
                                           int64_t stride, int qy, int qx, R s) {
    constexpr int ST = 2 * DQ + 1;
    const int i = threadIdx.x & 31, c0 = 4 * (threadIdx.x >> 5);
    if (i < 2 * qy && c0 < 2 * qx)
#pragma unroll
        for (int u = 0; u < 4; ++u) T[i * ST + c0 + u] = acc[u];
    __syncthreads();
    const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
    if (lane < 2 * qx)
        for (int r = wy; r < 2 * qy; r += 8) {
            const int64_t o = (int64_t)r * stride + lane;
            R v = T[r * ST + lane];
            if (add) v += add[o];
            out[o] = s * v;
        }
}

// One synthesis level > 0 for every (d, l): reconstructs the my x mx block
// (compact, stride mx, into `out`) from its LL (`llbuf`: A[1+d] at the coarsest
// level, else the coarser level's output, compact stride mx / 2) and A[1+d].
template <typename R, bool P2>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 4 : 1)
    k_dwt_inv_level(const R* __restrict__ A, const R* __restrict__ llbuf,
                    int ll_from_a, R* __restrict__ out, int L, int ny,
                    int nx, int my, int mx, int chunks) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* cf = reinterpret_cast<R*>(smem_raw);
    R* cl = cf + 2 * 4 * DC * SCS;
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
#define HS_INV(DD)                                                                                   \
    {                                                                                                \
        constexpr int H = DD + 1;                                                                    \
        inv_stage<R, inv_co<R, DD>(), P2>(cf, Ad, ll, lls, nx, hy, hx, ty * qy - (H - 1),            \
                                      tx * qx - (H - 1), qy + H - 1, qx + H - 1, chunks != 0);       \
        cp_async_wait<0>();                                                                          \
        __syncthreads();                                                                             \
        inv_cols<R, DD>(cf, cl, qy, qx + H - 1);                                                     \
        __syncthreads();                                                                             \
        inv_rows<R, DD>(cl, acc, qy, qx);                                                            \
    }
    HS_DWT_DISPATCH(d, HS_INV)
#undef HS_INV
    __syncthreads();
    R* o = out + ((int64_t)d * L + l) * (int64_t)my * mx + (int64_t)(2 * ty * qy) * mx + 2 * tx * qx;
    tile_store<R>(cl, acc, o, nullptr, mx, qy, qx, (R)1);
}

template <typename R> struct InvCtx {
    R* cf;
    R* cl;
    const R* A;
    const R* llbuf;
    int64_t N;
    int L, l, nx, hy, hx, ty, tx, qy, qx, ll_from_a, chunks;
};

template <typename R, int D, bool P2> __device__ __forceinline__ void inv_stage_d(const InvCtx<R>& c) {
    constexpr int H = D + 1;
    const R* Ad = c.A + ((int64_t)(1 + D) * c.L + c.l) * c.N;
    const R* ll = c.ll_from_a ? Ad : c.llbuf + ((int64_t)D * c.L + c.l) * (int64_t)c.hy * c.hx;
    inv_stage<R, inv_co<R, D>(), P2>(c.cf + (D & 1) * 4 * DC * SCS, Ad, ll, c.ll_from_a ? c.nx : c.hx, c.nx, c.hy,
                                 c.hx, c.ty * c.qy - (H - 1), c.tx * c.qx - (H - 1), c.qy + H - 1, c.qx + H - 1,
                                 c.chunks != 0);
}

// Level-0 synthesis of all eight wavelets, the next wavelet's subbands staged
// while the current one is filtered.
template <typename R, int D, bool P2> __device__ __forceinline__ void inv_all(const InvCtx<R>& c, R* acc) {
    if constexpr (D < NW) {
        if constexpr (D + 1 < NW) {
            inv_stage_d<R, D + 1, P2>(c);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        inv_cols<R, D>(c.cf + (D & 1) * 4 * DC * SCS, c.cl, c.qy, c.qx + D);
        __syncthreads();
        inv_rows<R, D>(c.cl, acc, c.qy, c.qx);
        inv_all<R, D + 1, P2>(c, acc);
    }
}

// Level-0 synthesis summed over the 9 bases: X[l] = (A[0][l] + sum_d W_d^T A[1+d][l]) / 3,
// one CTA per (output tile, channel).
template <typename R, bool P2>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 4 : 1)
    k_psi_adj_l0(const R* __restrict__ A, const R* __restrict__ llbuf,
                 int ll_from_a, R* __restrict__ X, int L, int ny, int nx,
                 R s, int chunks) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* cf = reinterpret_cast<R*>(smem_raw);
    R* cl = cf + 2 * 4 * DC * SCS;
    const int l = blockIdx.y;
    const int hy = ny >> 1, hx = nx >> 1;
    const int qy = min(DQ, hy), qx = min(DQ, hx);
    const int ntx = hx / qx;
    const int ty = blockIdx.x / ntx, tx = blockIdx.x - ty * ntx;
    const int64_t N = (int64_t)ny * nx;
    InvCtx<R> c{cf, cl, A, llbuf, N, L, l, nx, hy, hx, ty, tx, qy, qx, ll_from_a, chunks};
    inv_stage_d<R, 0, P2>(c);
    R acc[4] = {0, 0, 0, 0};
    inv_all<R, 0, P2>(c, acc);
    __syncthreads();
    const int64_t t0 = (int64_t)(2 * ty * qy) * nx + 2 * tx * qx;
    tile_store<R>(cl, acc, X + l * N + t0, A + l * N + t0, nx, qy, qx, s);
}

// ---- coarse levels of one (wavelet, channel) in shared memory
// When a level's input block fits in shared memory, one CTA per (wavelet d,
// channel l) runs that level and every coarser one without leaving the SM: X
// holds the level's block (top-left my x mx, row stride S), Y the intermediate
// of the two separable passes. Row passes take lane = row and 16-byte chunks
// along the row (S = 4 words mod 32 puts a quarter-warp's chunks in distinct
// banks); column passes take lane = column. Every level of the tail has sides
// that are multiples of 8, so chunks never straddle the periodic wrap.
constexpr int TAIL_THREADS = 512;
constexpr int TAIL_SMEM_MAX = 160 * 1024;   // bytes of X and Y together

// Row stride of X and Y, fixed at compile time so that every shared-memory
// address in the passes is a base plus an immediate offset: 132 floats or 66
// doubles (4 words mod 32), for blocks at most 128 floats or 64 doubles wide.
template <typename R> __host__ __device__ constexpr int tail_stride() { return sizeof(R) == 4 ? 132 : 66; }
template <typename R> __host__ __device__ constexpr int tail_max_width() {
    return tail_stride<R>() - 16 / (int)sizeof(R);
}
template <typename R> __host__ __device__ constexpr size_t tail_smem(int my) {
    return (size_t)2 * my * tail_stride<R>() * sizeof(R);
}

// x mod n for x >= 0
template <bool P2> __device__ __forceinline__ int modp(int x, int n) {
    if constexpr (P2) return x & (n - 1);
    else return x < n ? x : x % n;
}

template <typename R> __device__ __forceinline__ void ld_chunk(const R* p, R* v) {
    if constexpr (sizeof(R) == 4) {
        const float4 t = *reinterpret_cast<const float4*>(p);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else {
        const double2 t = *reinterpret_cast<const double2*>(p);
        v[0] = t.x; v[1] = t.y;
    }
}

// Copies rows [0, ry) x columns [c0, c0 + cw) of a global block (row stride gs)
// into X (row stride S) with asynchronous copies, all in flight at once: 16-byte
// chunks when the block is 16-byte aligned (cw, c0 multiples of the chunk), else
// single elements. Warps take rows, lanes take chunks.
template <typename R>
__device__ __forceinline__ void tail_stage(R* X, int S, const R* __restrict__ g, int64_t gs, int r0, int ry,
                                           int c0, int cw, bool chunks) {
    constexpr int EPC = 16 / (int)sizeof(R);
    const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (chunks) {
        for (int r = r0 + wy; r < r0 + ry; r += nw)
            for (int c = c0 + EPC * lane; c < c0 + cw; c += 32 * EPC) cp_async16(X + r * S + c, g + r * gs + c);
    } else {
        for (int r = r0 + wy; r < r0 + ry; r += nw)
            for (int c = c0 + lane; c < c0 + cw; c += 32) cp_async(X + r * S + c, g + r * gs + c);
    }
}

// Work items (q, c) = (it mod m, it / m) for it = threadIdx.x, threadIdx.x +
// blockDim.x, ... below m * nc, stepped without a division per item.
struct TailIter {
    int q, c, dq, dc, m;
    __device__ __forceinline__ TailIter(int m_) : m(m_) {
        c = threadIdx.x / m;
        q = threadIdx.x - c * m;
        dc = blockDim.x / m;
        dq = blockDim.x - dc * m;
    }
    __device__ __forceinline__ void next() {
        q += dq;
        c += dc;
        if (q >= m) {
            q -= m;
            ++c;
        }
    }
};

// Analysis along x: Y[r][k] = sum_j h[j] X[r][2k + j], Y[r][hx + k] = sum_j g[j] X[r][2k + j]
// (columns mod mx); a work item is one row and 4 consecutive output pairs.
template <typename R, int D, bool P2>
__device__ __forceinline__ void tail_fwd_rows(const R* X, R* Y, int S, int my, int mx) {
    constexpr int F = 2 * (D + 1);
    constexpr int EPC = 16 / (int)sizeof(R);
    constexpr int NCH = (F + 6 + EPC - 1) / EPC;
    const int hx = mx >> 1, nck = hx >> 2;
    for (TailIter t(my); t.c < nck; t.next()) {
        const int r = t.q, c = t.c;
        const R* row = X + r * S;
        R v[NCH * EPC];
        if (8 * c + NCH * EPC <= mx) {
#pragma unroll
            for (int k = 0; k < NCH; ++k) ld_chunk(row + 8 * c + EPC * k, v + EPC * k);
        } else {
#pragma unroll
            for (int k = 0; k < NCH; ++k) ld_chunk(row + modp<P2>(8 * c + EPC * k, mx), v + EPC * k);
        }
        R lo[4], hi[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            R a = 0, b = 0;
#pragma unroll
            for (int j = 0; j < F; ++j) {
                a = fma(filt<R>(D, 0, j), v[2 * u + j], a);
                b = fma(filt<R>(D, 1, j), v[2 * u + j], b);
            }
            lo[u] = a;
            hi[u] = b;
        }
        st4(Y + r * S + 4 * c, lo[0], lo[1], lo[2], lo[3]);
        st4(Y + r * S + hx + 4 * c, hi[0], hi[1], hi[2], hi[3]);
    }
}

// Analysis along y of the row-filtered block and the subband stores; a work
// item is one column and 4 consecutive output rows. LL goes to X (compact at
// the top-left, the next level's input) or, at the last level, to Ad.
template <typename R, int D, bool P2>
__device__ __forceinline__ void tail_fwd_cols(const R* Y, R* X, int S, int my, int mx, R* __restrict__ Ad,
                                              int nx, bool last) {
    constexpr int F = 2 * (D + 1);
    constexpr int NV = F + 6;
    const int hy = my >> 1, hx = mx >> 1, ncy = hy >> 2;
    for (TailIter t(mx); t.c < ncy; t.next()) {
        const int x = t.q, c = t.c;
        R v[NV];
        if (8 * c + NV <= my) {
            const R* col = Y + 8 * c * S + x;
#pragma unroll
            for (int k = 0; k < NV; ++k) v[k] = col[k * S];
        } else {
#pragma unroll
            for (int k = 0; k < NV; ++k) v[k] = Y[modp<P2>(8 * c + k, my) * S + x];
        }
        R lo[4], hi[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            R a = 0, b = 0;
#pragma unroll
            for (int j = 0; j < F; ++j) {
                a = fma(filt<R>(D, 0, j), v[2 * u + j], a);
                b = fma(filt<R>(D, 1, j), v[2 * u + j], b);
            }
            lo[u] = a;
            hi[u] = b;
        }
        const int oy = 4 * c;
        R* o = Ad + (int64_t)oy * nx + x;
        if (x < hx && !last) {
#pragma unroll
            for (int u = 0; u < 4; ++u) X[(oy + u) * S + x] = lo[u];
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) o[(int64_t)u * nx] = lo[u];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) o[(int64_t)(hy + u) * nx] = hi[u];
    }
}

// Synthesis along y: Y[2m + p][x] = sum_k h[2k + p] a[m - k] + g[2k + p] e[m - k]
// with a = X[.][x] (rows 0 .. hy - 1) and e = X[hy + .][x] (rows mod hy); a work
// item is one column and 4 consecutive coefficient rows.
template <typename R, int D, bool P2>
__device__ __forceinline__ void tail_inv_cols(const R* X, R* Y, int S, int my, int mx) {
    constexpr int H = D + 1;
    constexpr int NV = H + 3;
    const int hy = my >> 1, ncy = hy >> 2;
    for (TailIter it(mx); it.c < ncy; it.next()) {
        const int x = it.q, m0 = 4 * it.c;
        R a[NV], e[NV];
        if (m0 >= H - 1 && m0 + 4 <= hy) {
            const R* col = X + (m0 - (H - 1)) * S + x;
#pragma unroll
            for (int t = 0; t < NV; ++t) {
                a[t] = col[t * S];
                e[t] = col[(hy + t) * S];
            }
        } else {
#pragma unroll
            for (int t = 0; t < NV; ++t) {
                const int row = modp<P2>(m0 - (H - 1) + t + 8 * hy, hy);
                a[t] = X[row * S + x];
                e[t] = X[(hy + row) * S + x];
            }
        }
        R* o = Y + 2 * m0 * S + x;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            R v0 = 0, v1 = 0;
#pragma unroll
            for (int k = 0; k < H; ++k) {
                const int t = u - k + H - 1;
                v0 = fma(filt<R>(D, 0, 2 * k), a[t], v0);
                v0 = fma(filt<R>(D, 1, 2 * k), e[t], v0);
                v1 = fma(filt<R>(D, 0, 2 * k + 1), a[t], v1);
                v1 = fma(filt<R>(D, 1, 2 * k + 1), e[t], v1);
            }
            o[(2 * u) * S] = v0;
            o[(2 * u + 1) * S] = v1;
        }
    }
}

// Synthesis along x: out[i][2n + p] = sum_k h[2k + p] Y[i][n - k] + g[2k + p] Y[i][hx + n - k]
// (columns mod hx); a work item is one row and 4 consecutive coefficient columns
// (8 consecutive outputs), written to X (row stride S) or to a compact block.
template <typename R, int D, bool P2>
__device__ __forceinline__ void tail_inv_rows(const R* Y, R* out, int ostride, int S, int my, int mx) {
    constexpr int H = D + 1;
    constexpr int EPC = 16 / (int)sizeof(R);
    constexpr int BACK = ((H - 1 + EPC - 1) / EPC) * EPC;   // chunk-aligned look-back
    constexpr int NL = BACK + 4;                            // loaded values per half
    constexpr int OFF = BACK - (H - 1);                     // position of coefficient n0 - H + 1
    const int hx = mx >> 1, nck = hx >> 2;
    for (TailIter it(my); it.c < nck; it.next()) {
        const int i = it.q, n0 = 4 * it.c;
        const R* row = Y + i * S;
        R a[NL], e[NL];
        if (n0 >= BACK && n0 + 4 <= hx) {
#pragma unroll
            for (int k = 0; k < NL / EPC; ++k) {
                ld_chunk(row + n0 - BACK + EPC * k, a + EPC * k);
                ld_chunk(row + hx + n0 - BACK + EPC * k, e + EPC * k);
            }
        } else {
#pragma unroll
            for (int k = 0; k < NL / EPC; ++k) {
                const int n = modp<P2>(n0 - BACK + EPC * k + 8 * hx, hx);
                ld_chunk(row + n, a + EPC * k);
                ld_chunk(row + hx + n, e + EPC * k);
            }
        }
        R o[8];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            R v0 = 0, v1 = 0;
#pragma unroll
            for (int k = 0; k < H; ++k) {
                const int t = OFF + u - k + H - 1;
                v0 = fma(filt<R>(D, 0, 2 * k), a[t], v0);
                v0 = fma(filt<R>(D, 1, 2 * k), e[t], v0);
                v1 = fma(filt<R>(D, 0, 2 * k + 1), a[t], v1);
                v1 = fma(filt<R>(D, 1, 2 * k + 1), e[t], v1);
            }
            o[2 * u] = v0;
            o[2 * u + 1] = v1;
        }
        R* dst = out + (int64_t)i * ostride + 8 * it.c;
        st4(dst, o[0], o[1], o[2], o[3]);
        st4(dst + 4, o[4], o[5], o[6], o[7]);
    }
}

// Analysis levels lev0 .. top for one (d, l): input the compact my0 x mx0 LL of
// level lev0 - 1 (`src`); details (and the last LL) to A[1+d] at their Mallat
// positions.
template <typename R, bool P2>
__global__ void __launch_bounds__(TAIL_THREADS) k_dwt_fwd_tail(const R* __restrict__ src, R* __restrict__ A,
                                                              int L, int ny, int nx, int my0, int mx0,
                                                              int nlev) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int S = tail_stride<R>();
    R* X = reinterpret_cast<R*>(smem_raw);
    R* Y = X + my0 * S;
    const int dr = blockIdx.x / L, l = blockIdx.x - dr * L;
    const int d = NW - 1 - dr;   // longest filters first: the short ones fill the last wave
    const R* in = src + ((int64_t)d * L + l) * (int64_t)my0 * mx0;
    R* Ad = A + ((int64_t)(1 + d) * L + l) * (int64_t)ny * nx;
    tail_stage<R>(X, S, in, mx0, 0, my0, 0, mx0, true);   // plan scratch: 16-byte aligned
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
#define HS_FTAIL(DD)                                                          \
    for (int j = 0; j < nlev; ++j) {                                          \
        const int my = my0 >> j, mx = mx0 >> j;                               \
        tail_fwd_rows<R, DD, P2>(X, Y, S, my, mx);                            \
        __syncthreads();                                                      \
        tail_fwd_cols<R, DD, P2>(Y, X, S, my, mx, Ad, nx, j == nlev - 1);     \
        __syncthreads();                                                      \
    }
    HS_DWT_DISPATCH(d, HS_FTAIL)
#undef HS_FTAIL
}

// Synthesis levels top .. lev0 for one (d, l): the coarsest LL and every
// level's details from A[1+d]; the reconstructed my0 x mx0 input of level lev0
// to the compact buffer `out`.
template <typename R, bool P2>
__global__ void __launch_bounds__(TAIL_THREADS) k_dwt_inv_tail(const R* __restrict__ A, R* __restrict__ out,
                                                              int L, int ny, int nx, int my0, int mx0,
                                                              int nlev, int chunks) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int S = tail_stride<R>();
    R* X = reinterpret_cast<R*>(smem_raw);
    R* Y = X + my0 * S;
    const int dr = blockIdx.x / L, l = blockIdx.x - dr * L;
    const int d = NW - 1 - dr;   // longest filters first: the short ones fill the last wave
    const R* Ad = A + ((int64_t)(1 + d) * L + l) * (int64_t)ny * nx;
    R* o = out + ((int64_t)d * L + l) * (int64_t)my0 * mx0;
#define HS_ITAIL(DD)                                                                          \
    /* a level's details lie outside the coarser level's block, so they are fetched     \
       while the coarser level is synthesised */                                            \
    {                                                                                         \
        const int my = my0 >> (nlev - 1), mx = mx0 >> (nlev - 1);                            \
        tail_stage<R>(X, S, Ad, nx, 0, my, 0, mx, chunks != 0);                               \
        cp_async_commit();                                                                    \
    }                                                                                         \
    for (int j = nlev - 1; j >= 0; --j) {                                                     \
        const int my = my0 >> j, mx = mx0 >> j;                                               \
        if (j > 0) {                                                                          \
            tail_stage<R>(X, S, Ad, nx, 0, my, mx, mx, chunks != 0);                          \
            tail_stage<R>(X, S, Ad, nx, my, my, 0, 2 * mx, chunks != 0);                      \
            cp_async_commit();                                                                \
            cp_async_wait<1>();                                                               \
        } else {                                                                              \
            cp_async_wait<0>();                                                               \
        }                                                                                     \
        __syncthreads();                                                                      \
        tail_inv_cols<R, DD, P2>(X, Y, S, my, mx);                                            \
        __syncthreads();                                                                      \
        if (j > 0) tail_inv_rows<R, DD, P2>(Y, X, S, S, my, mx);                              \
        else tail_inv_rows<R, DD, P2>(Y, o, mx0, S, my, mx);                                  \
        __syncthreads();                                                                      \
    }
    HS_DWT_DISPATCH(d, HS_ITAIL)
#undef HS_ITAIL
}

// First level of the shared-memory tail: the finest level lev >= 1 whose input
// block fits (both sides multiples of 8 at every level down to the top), or 0
// when no level qualifies.
template <typename R> static int tail_level(const Plan* p) {
    const int top = p->levels - 1;
    for (int lev = 1; lev <= top; ++lev) {
        const int my = p->g.ny >> lev, mx = p->g.nx >> lev;
        if (mx > tail_max_width<R>() || tail_smem<R>(my) > (size_t)TAIL_SMEM_MAX) continue;
        for (int j = lev; j <= top; ++j)
            if (((p->g.ny >> j) % 8) || ((p->g.nx >> j) % 8)) return 0;
        return lev;
    }
    return 0;
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

template <typename K> static hs_status smem_attr(K k, int bytes) {
    HS_CHECK_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    return HS_OK;
}

hs_status dwt_init() {
    HS_TRY(upload_filters());
    HS_TRY(smem_attr(k_dwt_fwd_tail<float, true>, TAIL_SMEM_MAX));
    HS_TRY(smem_attr(k_dwt_fwd_tail<float, false>, TAIL_SMEM_MAX));
    HS_TRY(smem_attr(k_dwt_fwd_tail<double, true>, TAIL_SMEM_MAX));
    HS_TRY(smem_attr(k_dwt_fwd_tail<double, false>, TAIL_SMEM_MAX));
    HS_TRY(smem_attr(k_dwt_inv_tail<float, true>, TAIL_SMEM_MAX));
    HS_TRY(smem_attr(k_dwt_inv_tail<float, false>, TAIL_SMEM_MAX));
    HS_TRY(smem_attr(k_dwt_inv_tail<double, true>, TAIL_SMEM_MAX));
    HS_TRY(smem_attr(k_dwt_inv_tail<double, false>, TAIL_SMEM_MAX));
    HS_TRY(smem_attr(k_psi_fwd_l0<float, true>, FWD_SMEM * 4));
    HS_TRY(smem_attr(k_psi_fwd_l0<double, true>, FWD_SMEM * 8));
    HS_TRY(smem_attr(k_dwt_fwd_level<float, true>, FWD_SMEM * 4));
    HS_TRY(smem_attr(k_dwt_fwd_level<double, true>, FWD_SMEM * 8));
    HS_TRY(smem_attr(k_dwt_inv_level<float, true>, INV_SMEM * 4));
    HS_TRY(smem_attr(k_dwt_inv_level<double, true>, INV_SMEM * 8));
    HS_TRY(smem_attr(k_psi_adj_l0<float, true>, INV_SMEM * 4));
    HS_TRY(smem_attr(k_psi_adj_l0<double, true>, INV_SMEM * 8));
    HS_TRY(smem_attr(k_psi_fwd_l0<float, false>, FWD_SMEM * 4));
    HS_TRY(smem_attr(k_psi_fwd_l0<double, false>, FWD_SMEM * 8));
    HS_TRY(smem_attr(k_dwt_fwd_level<float, false>, FWD_SMEM * 4));
    HS_TRY(smem_attr(k_dwt_fwd_level<double, false>, FWD_SMEM * 8));
    HS_TRY(smem_attr(k_dwt_inv_level<float, false>, INV_SMEM * 4));
    HS_TRY(smem_attr(k_dwt_inv_level<double, false>, INV_SMEM * 8));
    HS_TRY(smem_attr(k_psi_adj_l0<float, false>, INV_SMEM * 4));
    HS_TRY(smem_attr(k_psi_adj_l0<double, false>, INV_SMEM * 8));
    return HS_OK;
}

static inline unsigned ntiles(int my, int mx) {
    const int hy = my >> 1, hx = mx >> 1;
    const int qy = hy < DQ ? hy : DQ, qx = hx < DQ ? hx : DQ;
    return (unsigned)((hy / qy) * (hx / qx));
}

template <typename R, bool P2> static hs_status analysis_t(Plan* p, const R* X, R* A, cudaStream_t s) {
    const int L = p->g.L, ny = p->g.ny, nx = p->g.nx;
    R* buf[2] = {(R*)p->dwt_a, (R*)p->dwt_b};
    const int top = p->levels - 1;
    const int pairs = ((uintptr_t)X % 8) == 0;   // caller's image: 8-byte pairs only when aligned
    k_psi_fwd_l0<R, P2><<<dim3(ntiles(ny, nx), L), 256, FWD_SMEM * sizeof(R), s>>>(X, A, buf[0], L, ny, nx, top == 0,
                                                                              (R)(1.0 / 3.0), pairs);
    HS_CHECK_LAUNCH();
    const int t = tail_level<R>(p);
    for (int lev = 1; lev <= top && (t == 0 || lev < t); ++lev) {
        const int my = ny >> lev, mx = nx >> lev;
        dim3 g(ntiles(my, mx), NW * L);
        k_dwt_fwd_level<R, P2><<<g, 256, FWD_SMEM * sizeof(R), s>>>(buf[(lev - 1) & 1], A, buf[lev & 1], L, ny, nx,
                                                                my, mx, lev == top);
        HS_CHECK_LAUNCH();
    }
    if (t > 0) {
        const int my = ny >> t, mx = nx >> t;
        k_dwt_fwd_tail<R, P2><<<NW * L, TAIL_THREADS, tail_smem<R>(my), s>>>(buf[(t - 1) & 1], A, L, ny, nx,
                                                                                my, mx, top - t + 1);
        HS_CHECK_LAUNCH();
    }
    return HS_OK;
}

template <typename R, bool P2> static hs_status synthesis_t(Plan* p, const R* A, R* X, cudaStream_t s) {
    const int chunks = ((uintptr_t)A % 16) == 0;   // caller's coefficients: 16-byte chunks only when aligned
    const int L = p->g.L, ny = p->g.ny, nx = p->g.nx;
    R* buf[2] = {(R*)p->dwt_a, (R*)p->dwt_b};
    const int top = p->levels - 1;
    const int t = tail_level<R>(p);
    if (t > 0) {
        const int my = ny >> t, mx = nx >> t;
        k_dwt_inv_tail<R, P2><<<NW * L, TAIL_THREADS, tail_smem<R>(my), s>>>(A, buf[t & 1], L, ny, nx, my, mx,
                                                                                top - t + 1, chunks);
        HS_CHECK_LAUNCH();
    }
    for (int lev = t > 0 ? t - 1 : top; lev >= 1; --lev) {
        const int my = ny >> lev, mx = nx >> lev;
        dim3 g(ntiles(my, mx), NW * L);
        k_dwt_inv_level<R, P2><<<g, 256, INV_SMEM * sizeof(R), s>>>(A, lev == top ? nullptr : buf[(lev + 1) & 1],
                                                                lev == top, buf[lev & 1], L, ny, nx, my, mx,
                                                                chunks);
        HS_CHECK_LAUNCH();
    }
    k_psi_adj_l0<R, P2><<<dim3(ntiles(ny, nx), L), 256, INV_SMEM * sizeof(R), s>>>(
        A, top == 0 ? nullptr : buf[1], top == 0, X, L, ny, nx, (R)(1.0 / 3.0), chunks);
    HS_CHECK_LAUNCH();
    return HS_OK;
}

static bool pow2_image(const Plan* p) { return wrap_mask(p->g.nx) >= 0 && wrap_mask(p->g.ny) >= 0; }

hs_status dwt_analysis(Plan* p, const void* X, void* A, cudaStream_t s) {
    const bool p2 = pow2_image(p);
    if (p->prec == HS_F32)
        return p2 ? analysis_t<float, true>(p, (const float*)X, (float*)A, s)
                  : analysis_t<float, false>(p, (const float*)X, (float*)A, s);
    return p2 ? analysis_t<double, true>(p, (const double*)X, (double*)A, s)
              : analysis_t<double, false>(p, (const double*)X, (double*)A, s);
}

hs_status dwt_synthesis(Plan* p, const void* A, void* X, cudaStream_t s) {
    const bool p2 = pow2_image(p);
    if (p->prec == HS_F32)
        return p2 ? synthesis_t<float, true>(p, (const float*)A, (float*)X, s)
                  : synthesis_t<float, false>(p, (const float*)A, (float*)X, s);
    return p2 ? synthesis_t<double, true>(p, (const double*)A, (double*)X, s)
              : synthesis_t<double, false>(p, (const double*)A, (double*)X, s);
}

}  // namespace hs
