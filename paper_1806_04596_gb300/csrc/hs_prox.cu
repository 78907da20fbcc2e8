// Proximity operators of Sec. 3.3 and the primal update of Algorithm 2.
//
//  l2,1      rows (basis, pixel) across the L channels (Eq. "prox-L21"), with
//            the Moreau dual form a min(1, lambda / ||a||) used in step 7.
//  l2 ball   per-channel projection onto B(y_l, eps_l) (functions g_l), norms
//            accumulated in FP64 as deterministic per-CTA partial sums.
//  nuclear   Eq. "prox-L*" through the L x L Gram matrix S = Z^T Z (per-tile
//            products, FP64 combine), its eigendecomposition in one CTA
//            (hs_eig.cu), and the apply Z V diag(f) V^T with f the
//            per-singular-value factor.
//  primal    steps 20-23: G = k1 P + k2 A~ + k3 Phi^dagger v, X = P_+(X - tau G),
//            X~ = 2 X - X_prev, beta partial sums.
#include <cmath>

#include <algorithm>

#include "hs_device.cuh"
#include "hs_internal.h"

namespace hs {

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// ---------------------------------------------------------------- reductions
// out[c] = sum_b part[c * nb + b] for c < nc, one block per c, fixed order.
__global__ void k_reduce_rows(const double* __restrict__ part, int nb, double* __restrict__ out) {
    __shared__ double red[32];
    const int c = blockIdx.x;
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s += part[(int64_t)c * nb + b];
    s = block_sum(s, red);
    if (threadIdx.x == 0) out[c] = s;
}

// ---------------------------------------------------------------- l2,1
// One thread per row (basis b, pixel n) of the coefficient cube: q_l = A + W
// over the L channels (stride N), the row norm, and the scaled row. For
// L <= LMAX the row is held in registers (each input read once); LMAX = 0 is
// the general form that reads the row twice.
template <typename R, int LMAX>
__global__ void __launch_bounds__(256) k_l21(const R* __restrict__ A, const R* __restrict__ W,
                                             const R* __restrict__ w_rows, R thr, int dual,
                                             R* __restrict__ out, int L, int64_t N) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)NB * N) return;
    const int b = (int)(t / N);
    const int64_t pix = t - (int64_t)b * N;
    const int64_t base = (int64_t)b * L * N + pix;
    R s = 0;
    R q[LMAX > 0 ? LMAX : 1];
    if (LMAX > 0) {
#pragma unroll
        for (int l = 0; l < LMAX; ++l)
            if (l < L) {
                R v = A[base + (int64_t)l * N];
                if (W) v += W[base + (int64_t)l * N];
                q[l] = v;
            }
#pragma unroll
        for (int l = 0; l < LMAX; ++l)
            if (l < L) s = fma(q[l], q[l], s);
    } else {
        for (int l = 0; l < L; ++l) {
            R v = A[base + (int64_t)l * N];
            if (W) v += W[base + (int64_t)l * N];
            s = fma(v, v, s);
        }
    }
    const R nrm = sqrt(s);
    const R lam = thr * (w_rows ? w_rows[t] : (R)1);
    R f;
    if (dual == 2) f = (nrm > (R)0) ? lam / nrm : (R)0;   // direction: gradient of lam ||q||
    else if (dual) f = (nrm > lam) ? lam / nrm : (R)1;
    else f = (nrm > lam) ? (nrm - lam) / nrm : (R)0;
    if (LMAX > 0) {
#pragma unroll
        for (int l = 0; l < LMAX; ++l)
            if (l < L) out[base + (int64_t)l * N] = q[l] * f;
    } else {
        for (int l = 0; l < L; ++l) {
            R v = A[base + (int64_t)l * N];
            if (W) v += W[base + (int64_t)l * N];
            out[base + (int64_t)l * N] = v * f;
        }
    }
}

// FP32 form with the channels of a row split over the 4 warps of a CTA
// (channel l to warp l mod 4): a CTA covers 32 pixel pairs of one basis, every
// lane keeps at most LW channels of its pair in registers (LW = ceil(L / 4)),
// and the 4 warps' partial sums of squares meet in shared memory, added in the
// same order by every warp. With at most 16 channels of a pair per thread,
// many more loads are in flight per SM than with a whole row per thread (the
// kernel streams A and W once and writes the dual once).
template <int LW>
__global__ void __launch_bounds__(128) k_l21_split(const float* __restrict__ A, const float* __restrict__ W,
                                                   const float* __restrict__ w_rows, float thr, int dual,
                                                   float* __restrict__ out, int L, int64_t N) {
    __shared__ float2 part[4][32];
    const int64_t Nh = N >> 1;
    const int64_t nq = (Nh + 31) >> 5;   // CTAs per basis
    const int b = (int)(blockIdx.x / nq);
    const int64_t pp = (blockIdx.x - (int64_t)b * nq) * 32 + (threadIdx.x & 31);
    const int wv = threadIdx.x >> 5;
    const bool in = pp < Nh;
    const int64_t base = (int64_t)b * L * N + 2 * pp;
    float2 q[LW];
    float s0 = 0.f, s1 = 0.f;
#pragma unroll
    for (int c = 0; c < LW; ++c) {
        const int l = wv + 4 * c;
        if (in && l < L) {
            float2 v = *reinterpret_cast<const float2*>(A + base + (int64_t)l * N);
            if (W) {
                const float2 u = *reinterpret_cast<const float2*>(W + base + (int64_t)l * N);
                v.x += u.x;
                v.y += u.y;
            }
            q[c] = v;
            s0 = fmaf(v.x, v.x, s0);
            s1 = fmaf(v.y, v.y, s1);
        }
    }
    part[wv][threadIdx.x & 31] = make_float2(s0, s1);
    __syncthreads();
    if (!in) return;
    const float2 p0 = part[0][threadIdx.x & 31], p1 = part[1][threadIdx.x & 31];
    const float2 p2 = part[2][threadIdx.x & 31], p3 = part[3][threadIdx.x & 31];
    const float n0 = sqrtf((p0.x + p1.x) + (p2.x + p3.x)), n1 = sqrtf((p0.y + p1.y) + (p2.y + p3.y));
    float2 wr = make_float2(1.f, 1.f);
    if (w_rows) wr = *reinterpret_cast<const float2*>(w_rows + (int64_t)b * N + 2 * pp);
    const float lam0 = thr * wr.x, lam1 = thr * wr.y;
    float f0, f1;
    if (dual == 2) {   // direction: gradient of lam ||q||
        f0 = (n0 > 0.f) ? lam0 / n0 : 0.f;
        f1 = (n1 > 0.f) ? lam1 / n1 : 0.f;
    } else if (dual) {
        f0 = (n0 > lam0) ? lam0 / n0 : 1.f;
        f1 = (n1 > lam1) ? lam1 / n1 : 1.f;
    } else {
        f0 = (n0 > lam0) ? (n0 - lam0) / n0 : 0.f;
        f1 = (n1 > lam1) ? (n1 - lam1) / n1 : 0.f;
    }
#pragma unroll
    for (int c = 0; c < LW; ++c) {
        const int l = wv + 4 * c;
        if (l < L)
            *reinterpret_cast<float2*>(out + base + (int64_t)l * N) = make_float2(q[c].x * f0, q[c].y * f1);
    }
}

template <typename R>
__global__ void k_l21_norm(const R* __restrict__ A, const R* __restrict__ w_rows, int L, int64_t N,
                           double* __restrict__ part) {
    __shared__ double red[32];
    double acc = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)NB * N;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(t / N);
        const int64_t pix = t - (int64_t)b * N;
        const int64_t base = (int64_t)b * L * N + pix;
        double s = 0.0;
        for (int l = 0; l < L; ++l) {
            const double q = (double)A[base + (int64_t)l * N];
            s += q * q;
        }
        acc += sqrt(s) * (w_rows ? (double)w_rows[t] : 1.0);
    }
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

hs_status l21_apply(Plan* p, const void* A, const void* Wadd, const void* w_rows, double thr,
                    int dual, void* out, cudaStream_t s) {
    const int64_t N = p->N();
    const unsigned g = nblk((int64_t)NB * N, 256);
    const int L = p->g.L;
#define HS_L21(R, LM)                                                                                    \
    k_l21<R, LM><<<g, 256, 0, s>>>((const R*)A, (const R*)Wadd, (const R*)w_rows, (R)thr, dual, (R*)out, L, \
                                   N)
    auto al8 = [](const void* q) { return ((uintptr_t)q % 8) == 0; };
    const bool pairs = (N % 2) == 0 && al8(A) && al8(Wadd) && al8(w_rows) && al8(out);
    if (p->prec == HS_F32 && pairs && L <= 64) {
        const int64_t nq = (N / 2 + 31) / 32;
        const unsigned g2 = (unsigned)(NB * nq);
        if (L <= 16)
            k_l21_split<4><<<g2, 128, 0, s>>>((const float*)A, (const float*)Wadd, (const float*)w_rows,
                                              (float)thr, dual, (float*)out, L, N);
        else
            k_l21_split<16><<<g2, 128, 0, s>>>((const float*)A, (const float*)Wadd, (const float*)w_rows,
                                               (float)thr, dual, (float*)out, L, N);
    } else if (p->prec == HS_F32) {
        if (L <= 16) HS_L21(float, 16);
        else if (L <= 64) HS_L21(float, 64);
        else HS_L21(float, 0);
    } else {
        if (L <= 16) HS_L21(double, 16);
        else if (L <= 64) HS_L21(double, 64);
        else HS_L21(double, 0);
    }
#undef HS_L21
    HS_CHECK_LAUNCH();
    return HS_OK;
}

// SARA prior (Sec. 4.2): every coefficient on its own. Dual form (step 7 with
// the l1 norm): out = clip(A + W, -thr w, thr w); prox form: soft threshold.
template <typename R>
__global__ void __launch_bounds__(256) k_l1(const R* __restrict__ A, const R* __restrict__ W,
                                           const R* __restrict__ w, R thr, int dual, R* __restrict__ out,
                                           int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        R q = A[i];
        if (W) q += W[i];
        const R lam = thr * (w ? w[i] : (R)1);
        const R c = fmin(fmax(q, -lam), lam);
        out[i] = dual ? c : q - c;
    }
}

hs_status l1_apply(Plan* p, const void* A, const void* Wadd, const void* w, double thr, int dual, void* out,
                   cudaStream_t s) {
    const int64_t n = (int64_t)NB * p->g.L * p->N();
    const unsigned g = std::min<unsigned>(nblk(n, 256), 152u * 16u);
    if (p->prec == HS_F32)
        k_l1<float><<<g, 256, 0, s>>>((const float*)A, (const float*)Wadd, (const float*)w, (float)thr, dual,
                                      (float*)out, n);
    else
        k_l1<double><<<g, 256, 0, s>>>((const double*)A, (const double*)Wadd, (const double*)w, thr, dual,
                                       (double*)out, n);
    HS_CHECK_LAUNCH();
    return HS_OK;
}

hs_status l21_norm(Plan* p, const void* A, const void* w_rows, double* out_dev, cudaStream_t s) {
    const int64_t N = p->N();
    const int nb = 512;
    if (p->prec == HS_F32)
        k_l21_norm<float><<<nb, 256, 0, s>>>((const float*)A, (const float*)w_rows, p->g.L, N, p->part);
    else
        k_l21_norm<double><<<nb, 256, 0, s>>>((const double*)A, (const double*)w_rows, p->g.L, N,
                                              p->part);
    HS_CHECK_LAUNCH();
    k_reduce_rows<<<1, 256, 0, s>>>(p->part, nb, out_dev);
    HS_CHECK_LAUNCH();
    return HS_OK;
}

// ---------------------------------------------------------------- l2 ball
// Per-CTA partial ||z - y||^2 over [off[l] + bx * CH, ...), grid (nbx, L).
template <typename R>
__global__ void k_ball_norm(const Cx<R>* __restrict__ Z, const Cx<R>* __restrict__ Y,
                            const int64_t* __restrict__ off, int nbx, double* __restrict__ part) {
    __shared__ double red[32];
    const int l = blockIdx.y;
    const int64_t beg = off[l] + (int64_t)blockIdx.x * DEGRID_CHUNK;
    const int64_t end = min(off[l + 1], beg + DEGRID_CHUNK);
    double s = 0.0;
    for (int64_t i = beg + threadIdx.x; i < end; i += blockDim.x) {
        const Cx<R> d = csub(Z[i], Y[i]);
        s += (double)d.x * d.x + (double)d.y * d.y;
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) part[(int64_t)l * nbx + blockIdx.x] = s;
}

// rho_l = sqrt(sum of partials); scale_l = max(0, 1 - eps_l / rho_l) (0 when rho = 0).
template <typename R>
__global__ void k_ball_scale(const double* __restrict__ part, int nb, const double* __restrict__ eps,
                             double* __restrict__ rho, R* __restrict__ scale) {
    __shared__ double red[32];
    const int l = blockIdx.x;
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s += part[(int64_t)l * nb + b];
    s = block_sum(s, red);
    if (threadIdx.x == 0) {
        const double r = sqrt(s);
        if (rho) rho[l] = r;
        const double e = eps[l];
        scale[l] = (R)((r > e) ? (1.0 - e / r) : 0.0);
    }
}

template <typename R>
__global__ void k_ball_apply(const Cx<R>* __restrict__ Z, const Cx<R>* __restrict__ Y,
                             const int64_t* __restrict__ off, int L, const R* __restrict__ scale,
                             int dual, Cx<R>* __restrict__ out, int64_t total) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = L;   // channel: off[lo] <= i < off[lo+1]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (off[mid] <= i) lo = mid;
            else hi = mid;
        }
        const R sc = scale[lo];
        const Cx<R> d = csub(Z[i], Y[i]);
        // (z - y) * max(0, 1 - eps/rho) is z - P_B(z); P_B(z) = z - that
        const Cx<R> r = cscale(d, sc);
        out[i] = dual ? r : csub(Z[i], r);
    }
}

// One CTA per data block of the plan (p->nblk; one per channel without blocks).
hs_status ball_scale_from_partials(Plan* p, const double* part, int nparts, const double* eps,
                                   double* rho, void* scale_real, cudaStream_t s) {
    if (p->prec == HS_F32)
        k_ball_scale<float><<<p->nblk, 256, 0, s>>>(part, nparts, eps, rho, (float*)scale_real);
    else
        k_ball_scale<double><<<p->nblk, 256, 0, s>>>(part, nparts, eps, rho, (double*)scale_real);
    HS_CHECK_LAUNCH();
    return HS_OK;
}

// Algorithm 2 steps 13-19, one CTA per block: rho_b = ||y_b - Phi_b x~|| from
// the de-gridding partials; when beta^{(t-1)} < lambda_1, t - vartheta_b >
// vartheta_bar and |rho_b - eps_b| / eps_b > lambda_2, eps_b <- lambda_3 rho_b
// + (1 - lambda_3) eps_b and vartheta_b <- t (t = completed iterations + 1).
__global__ void k_adapt(int nparts, AdaptArgs a) {
    __shared__ double red[32];
    const int b = blockIdx.x;
    double s = 0.0;
    for (int k = threadIdx.x; k < nparts; k += blockDim.x) s += a.rpart[(int64_t)b * nparts + k];
    s = block_sum(s, red);
    if (threadIdx.x == 0) {
        const double rho = sqrt(s);
        a.resid[b] = rho;
        const int64_t t = *a.t + 1;
        const double e = a.eps[b];
        if (*a.beta < a.lambda1 && t - a.theta[b] > a.min_gap && fabs(rho - e) / e > a.lambda2) {
            a.eps[b] = a.lambda3 * rho + (1.0 - a.lambda3) * e;
            a.theta[b] = t;
        }
    }
}

hs_status adapt_bounds(int nblk, int nparts, const AdaptArgs& a, cudaStream_t s) {
    k_adapt<<<nblk, 128, 0, s>>>(nparts, a);
    HS_CHECK_LAUNCH();
    return HS_OK;
}

hs_status ball_project(Plan* p, const void* Z, const void* Yd, const double* eps, int dual,
                       void* out, double* rho_out, cudaStream_t s) {
    const int nbx = degrid_blocks_x(p);
    const int L = p->g.L;
    if (L == 0 || p->M_total == 0) {
        if (rho_out && L) HS_CHECK_CUDA(cudaMemsetAsync(rho_out, 0, sizeof(double) * L, s));
        return HS_OK;
    }
    dim3 g(nbx, L);
    void* scale = p->dscal + 2 * L;   // L reals (fits in 2 L doubles)
    if (p->prec == HS_F32) {
        k_ball_norm<float><<<g, 256, 0, s>>>((const float2*)Z, (const float2*)Yd, p->off_d, nbx, p->part);
        HS_CHECK_LAUNCH();
        k_ball_scale<float><<<L, 256, 0, s>>>(p->part, nbx, eps, rho_out, (float*)scale);
        HS_CHECK_LAUNCH();
        k_ball_apply<float><<<nblk(p->M_total, 256) > 8192 ? 8192 : nblk(p->M_total, 256), 256, 0, s>>>(
            (const float2*)Z, (const float2*)Yd, p->off_d, L, (const float*)scale, dual, (float2*)out,
            p->M_total);
    } else {
        k_ball_norm<double><<<g, 256, 0, s>>>((const double2*)Z, (const double2*)Yd, p->off_d, nbx,
                                              p->part);
        HS_CHECK_LAUNCH();
        k_ball_scale<double><<<L, 256, 0, s>>>(p->part, nbx, eps, rho_out, (double*)scale);
        HS_CHECK_LAUNCH();
        k_ball_apply<double><<<nblk(p->M_total, 256) > 8192 ? 8192 : nblk(p->M_total, 256), 256, 0, s>>>(
            (const double2*)Z, (const double2*)Yd, p->off_d, L, (const double*)scale, dual,
            (double2*)out, p->M_total);
    }
    HS_CHECK_LAUNCH();
    return HS_OK;
}

// ---------------------------------------------------------------- nuclear norm
constexpr int GRAM_PIX = 64;      // pixels per shared-memory tile
constexpr int GRAM_CTAS = 304;    // 2 per SM
constexpr int GRAM_LDZ = MAX_L_NUC + 4;   // pixel-major tile row (16-byte aligned)

__device__ __forceinline__ void ld4(const float* p, float* v) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x;
    v[1] = t.y;
    v[2] = t.z;
    v[3] = t.w;
}
__device__ __forceinline__ void ld4(const double* p, double* v) {
    const double2 t0 = reinterpret_cast<const double2*>(p)[0], t1 = reinterpret_cast<const double2*>(p)[1];
    v[0] = t0.x;
    v[1] = t0.y;
    v[2] = t1.x;
    v[3] = t1.y;
}

// Partial Gram matrices S_ij = sum_n z_in z_jn, z = X (+ Xa), for L <= 64:
// thread (bi, bj) of a 16 x 16 grid owns the 4 x 4 block of rows 4 bi .. 4 bi + 3
// and columns 4 bj .. 4 bj + 3 (register blocking: per pixel two 4-wide shared
// loads feed 16 FMAs). Runs of 32 pixels are summed in R and added into a
// (hi, lo) pair with the error-free two-sum (Knuth), so the accumulation across
// runs is as exact as in FP64 without FP64 arithmetic; each CTA writes its
// upper-triangle partials in FP64.
template <typename R>
__global__ void __launch_bounds__(256) k_gram(const R* __restrict__ X, const R* __restrict__ Xa,
                                              int L, int64_t N, double* __restrict__ part) {
    __shared__ __align__(16) R zs[GRAM_PIX][GRAM_LDZ];   // pixel-major tile
    const int tid = threadIdx.x;
    const int bi = tid >> 4, bj = tid & 15;
    R hi[16], lo[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        hi[q] = 0;
        lo[q] = 0;
    }
    const int64_t ntile = N / GRAM_PIX;   // N is a multiple of 64 (nx, ny >= 16, powers of two)
    // thread tid stages channels (tid >> 6) + 4 m, m < 16, of pixel tid & 63; the
    // next tile's values are loaded into registers while the current one is used
    constexpr int PER = MAX_L_NUC * GRAM_PIX / 256;
    const int px0 = tid & (GRAM_PIX - 1), l0 = tid >> 6;
    R pre[PER];
    auto fetch = [&](int64_t tile) {
        const int64_t n = tile * GRAM_PIX + px0;
#pragma unroll
        for (int m = 0; m < PER; ++m) {
            const int l = l0 + 4 * m;
            R z = 0;
            if (l < L && tile < ntile) {
                z = X[(int64_t)l * N + n];
                if (Xa) z += Xa[(int64_t)l * N + n];
            }
            pre[m] = z;
        }
    };
    fetch(blockIdx.x);
    for (int64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
        __syncthreads();
#pragma unroll
        for (int m = 0; m < PER; ++m) zs[px0][l0 + 4 * m] = pre[m];
        __syncthreads();
        fetch(tile + gridDim.x);
#pragma unroll
        for (int half = 0; half < GRAM_PIX / 32; ++half) {
            R acc[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) acc[q] = 0;
#pragma unroll 4
            for (int px = 32 * half; px < 32 * half + 32; ++px) {
                R a[4], b[4];
                ld4(&zs[px][4 * bi], a);
                ld4(&zs[px][4 * bj], b);
#pragma unroll
                for (int t = 0; t < 4; ++t)
#pragma unroll
                    for (int u = 0; u < 4; ++u) acc[4 * t + u] = fma(a[t], b[u], acc[4 * t + u]);
            }
#pragma unroll
            for (int q = 0; q < 16; ++q) {   // (hi, lo) += acc, hi + e = old hi + acc exactly
                const R sum = hi[q] + acc[q];
                const R bp = sum - hi[q];
                const R e = (hi[q] - (sum - bp)) + (acc[q] - bp);
                hi[q] = sum;
                lo[q] += e;
            }
        }
    }
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = 4 * bi + t, j = 4 * bj + u;
            if (i <= j && j < L) {
                const int e = i * L - i * (i - 1) / 2 + (j - i);   // row-major rank in the upper triangle
                part[(int64_t)e * gridDim.x + blockIdx.x] = (double)hi[4 * t + u] + (double)lo[4 * t + u];
            }
        }
}

// Sum the per-CTA partials (fixed order) and expand to the full symmetric matrix.
__global__ void k_gram_reduce(const double* __restrict__ part, int nb, int L, double* __restrict__ S) {
    __shared__ double red[32];
    const int e = blockIdx.x;
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s += part[(int64_t)e * nb + b];
    s = block_sum(s, red);
    if (threadIdx.x == 0) {
        int i = 0, rem = e;
        while (rem >= L - i) {
            rem -= L - i;
            ++i;
        }
        const int j = i + rem;
        S[i * L + j] = s;
        S[j * L + i] = s;
    }
}

// out[:, n] = M z_n with z = X (+ Xa) and M = base I + sum_{c < r} g_c x_c x_c^T
// (low-rank form written by the eigensolver): per pixel, r projections
// q_c = g_c (x_c . z), then out = base z + sum_c q_c x_c, the pixel's L values
// in registers (overwritten in place by the output), q_c in shared memory, x_c
// read with uniform (broadcast) loads. In FP32 the FP64 vectors are carried as
// two FP32 parts (hi + lo), so that their rounding does not enter the result:
// the output is often a small remainder of a large z (the dual form keeps the
// small singular values).
constexpr int LR_BS = 128;   // pixels (threads) per CTA
static_assert(LR_DOUBLES % 2 == 0 && LRF_XL % 4 == 0 && MAX_L_NUC % 4 == 0, "16-byte aligned FP32 factor rows");

template <typename R, int LMAX>
__global__ void __launch_bounds__(LR_BS) k_lowrank_apply(const R* __restrict__ X, const R* __restrict__ Xa,
                                                         const double* __restrict__ F, int L, int64_t N,
                                                         R* __restrict__ out) {
    constexpr bool SPLIT = sizeof(R) == 4;
    __shared__ R qs[LMAX * LR_BS];
    const int r = max(0, min((int)F[LR_R], L));   // the active count, always <= L
    const bool base = F[LR_BASE] != 0.0;
    const float* Ff = reinterpret_cast<const float*>(F + LR_DOUBLES);
    const int t = threadIdx.x;
    const int64_t n = blockIdx.x * (int64_t)LR_BS + t;
    if (n >= N) return;
    R z[LMAX];
#pragma unroll
    for (int i = 0; i < LMAX; ++i) {
        z[i] = 0;
        if (i < L) {
            z[i] = X[(int64_t)i * N + n];
            if (Xa) z[i] += Xa[(int64_t)i * N + n];
        }
    }
    for (int c = 0; c < r; ++c) {
        R p = 0, p2 = 0;
        if constexpr (SPLIT) {   // the factor rows as 16-byte broadcast loads, same FMA order
#pragma unroll
            for (int i = 0; i < LMAX; i += 4)
                if (i < L) {
                    const float4 h = *reinterpret_cast<const float4*>(Ff + LRF_XH + c * MAX_L_NUC + i);
                    const float4 o = *reinterpret_cast<const float4*>(Ff + LRF_XL + c * MAX_L_NUC + i);
                    const float hh[4] = {h.x, h.y, h.z, h.w}, oo[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (i + k < L) {
                            p = fma(z[i + k], (R)hh[k], p);
                            p2 = fma(z[i + k], (R)oo[k], p2);
                        }
                }
        } else {
#pragma unroll
            for (int i = 0; i < LMAX; ++i)
                if (i < L) p = fma(z[i], (R)F[LR_X + c * MAX_L_NUC + i], p);
        }
        qs[c * LR_BS + t] = (SPLIT ? (R)Ff[LRF_G + c] : (R)F[LR_G + c]) * (p + p2);
    }
    if (!base)
#pragma unroll
        for (int i = 0; i < LMAX; ++i) z[i] = 0;
    for (int c = 0; c < r; ++c) {
        const R q = qs[c * LR_BS + t];
        if constexpr (SPLIT) {
#pragma unroll
            for (int i = 0; i < LMAX; i += 4)
                if (i < L) {
                    const float4 h = *reinterpret_cast<const float4*>(Ff + LRF_XH + c * MAX_L_NUC + i);
                    const float4 o = *reinterpret_cast<const float4*>(Ff + LRF_XL + c * MAX_L_NUC + i);
                    const float hh[4] = {h.x, h.y, h.z, h.w}, oo[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (i + k < L) {
                            z[i + k] = fma(q, (R)hh[k], z[i + k]);
                            z[i + k] = fma(q, (R)oo[k], z[i + k]);
                        }
                }
        } else {
#pragma unroll
            for (int i = 0; i < LMAX; ++i)
                if (i < L) z[i] = fma(q, (R)F[LR_X + c * MAX_L_NUC + i], z[i]);
        }
    }
#pragma unroll
    for (int i = 0; i < LMAX; ++i)
        if (i < L) out[(int64_t)i * N + n] = z[i];
}

// FP32 form with the channels of a pixel split over the 4 warps of a CTA
// (channel i to warp i mod 4; 32 pixels per CTA): each warp forms partial
// projections of its channels on 8 components at a time, the partials meet in
// shared memory (added in the same order by every warp), and every lane then
// updates its own channels in component order, as in k_lowrank_apply. At most
// LW = ceil(L / 4) channels per lane in registers, so far more pixels are in
// flight per SM than with one pixel's whole spectrum per thread.
constexpr int LRS_CC = 8;   // components per shared-memory round
template <int LW>
__global__ void __launch_bounds__(128) k_lowrank_split(const float* __restrict__ X, const float* __restrict__ Xa,
                                                       const double* __restrict__ F, int L, int64_t N,
                                                       float* __restrict__ out) {
    __shared__ float2 part[LRS_CC][4][32];
    const int r = max(0, min((int)F[LR_R], L));   // the active count, always <= L
    const bool base = F[LR_BASE] != 0.0;
    const float* Ff = reinterpret_cast<const float*>(F + LR_DOUBLES);
    const int lane = threadIdx.x & 31, wv = threadIdx.x >> 5;
    const int64_t n = blockIdx.x * (int64_t)32 + lane;
    const bool in = n < N;
    float z[LW], acc[LW];
#pragma unroll
    for (int k = 0; k < LW; ++k) {
        const int i = wv + 4 * k;
        z[k] = 0.f;
        if (in && i < L) {
            z[k] = X[(int64_t)i * N + n];
            if (Xa) z[k] += Xa[(int64_t)i * N + n];
        }
        acc[k] = base ? z[k] : 0.f;
    }
    for (int c0 = 0; c0 < r; c0 += LRS_CC) {
        const int nc = min(LRS_CC, r - c0);
        for (int cc = 0; cc < nc; ++cc) {
            const int c = c0 + cc;
            float p = 0.f, p2 = 0.f;
#pragma unroll
            for (int k = 0; k < LW; ++k) {
                const int i = wv + 4 * k;
                if (i < L) {
                    p = fmaf(z[k], Ff[LRF_XH + c * MAX_L_NUC + i], p);
                    p2 = fmaf(z[k], Ff[LRF_XL + c * MAX_L_NUC + i], p2);
                }
            }
            part[cc][wv][lane] = make_float2(p, p2);
        }
        __syncthreads();
        for (int cc = 0; cc < nc; ++cc) {
            const int c = c0 + cc;
            const float2 a = part[cc][0][lane], b = part[cc][1][lane], d = part[cc][2][lane], e = part[cc][3][lane];
            const float q = Ff[LRF_G + c] * (((a.x + b.x) + (d.x + e.x)) + ((a.y + b.y) + (d.y + e.y)));
#pragma unroll
            for (int k = 0; k < LW; ++k) {
                const int i = wv + 4 * k;
                if (i < L) {
                    acc[k] = fmaf(q, Ff[LRF_XH + c * MAX_L_NUC + i], acc[k]);
                    acc[k] = fmaf(q, Ff[LRF_XL + c * MAX_L_NUC + i], acc[k]);
                }
            }
        }
        __syncthreads();
    }
    if (!in) return;
#pragma unroll
    for (int k = 0; k < LW; ++k) {
        const int i = wv + 4 * k;
        if (i < L) out[(int64_t)i * N + n] = acc[k];
    }
}

template <typename R>
static hs_status lowrank_apply_t(Plan* p, const void* X, const void* Xa, void* out, cudaStream_t s) {
    const int L = p->g.L;
    const int64_t N = p->N();
    const unsigned g = nblk(N, LR_BS);
    if constexpr (sizeof(R) == 4) {
        const unsigned g4 = (unsigned)((N + 31) / 32);
        if (L <= 16) k_lowrank_split<4><<<g4, 128, 0, s>>>((const float*)X, (const float*)Xa, p->eigf, L, N, (float*)out);
        else k_lowrank_split<16><<<g4, 128, 0, s>>>((const float*)X, (const float*)Xa, p->eigf, L, N, (float*)out);
        HS_CHECK_LAUNCH();
        return HS_OK;
    }
#define HS_LR(LM) \
    k_lowrank_apply<R, LM><<<g, LR_BS, 0, s>>>((const R*)X, (const R*)Xa, p->eigf, L, N, (R*)out)
    if (L <= 8) HS_LR(8);
    else if (L <= 16) HS_LR(16);
    else if (L <= 32) HS_LR(32);
    else HS_LR(64);
#undef HS_LR
    HS_CHECK_LAUNCH();
    return HS_OK;
}

// Partial Gram matrices of Z = X (+ Xa) into p->part and their fixed-order sum
// into p->gram (L x L, row-major): tensor cores (tcgen05,
// exact BF16 digits) for FP32 plans whose buffers allow it, register-blocked
// FMA otherwise (and for FP64 plans).
hs_status gram_matrix(Plan* p, const void* X, const void* Xadd, cudaStream_t s) {
    const int L = p->g.L;
    const int64_t N = p->N();
    const int P = L * (L + 1) / 2;
    int nb = GRAM_CTAS;
    if (p->prec == HS_F32 && p->gram_tc && gram_tc_usable(X, Xadd, L, N)) {
        HS_TRY(gram_tc_launch((const float*)X, (const float*)Xadd, L, N, p->part, GRAM_CTAS, p->err_d, &nb, s));
    } else if (p->prec == HS_F32) {
        k_gram<float><<<GRAM_CTAS, 256, 0, s>>>((const float*)X, (const float*)Xadd, L, N, p->part);
    } else {
        k_gram<double><<<GRAM_CTAS, 256, 0, s>>>((const double*)X, (const double*)Xadd, L, N, p->part);
    }
    HS_CHECK_LAUNCH();
    k_gram_reduce<<<P, 128, 0, s>>>(p->part, nb, L, p->gram);
    HS_CHECK_LAUNCH();
    return HS_OK;
}

hs_status nuclear_apply(Plan* p, const void* X, const void* Xadd, const double* w_sv, double thr,
                        int dual, void* out, double* sv_out, float* warm, int* r_out,
                        cudaStream_t s) {
    const int L = p->g.L;
    if (L > MAX_L_NUC) return fail(HS_ERR_ARG, "nuclear prox: L = %d exceeds %d", L, MAX_L_NUC);
    HS_TRY(gram_matrix(p, X, Xadd, s));
    if (p->prec == HS_F32) {
        // FP32 Jacobi (warm-started) + FP64 refinement of the active eigenpairs
        HS_TRY(eig_mixed_launch(p->gram, L, w_sv, thr, dual, p->eigf, sv_out, warm, r_out, s));
    } else {
        // FP64 plans: cyclic Jacobi entirely in FP64
        HS_TRY(eig_f64_launch(p->gram, L, w_sv, thr, dual, p->eigf, sv_out, r_out, s));
    }
    if (p->prec == HS_F32) return lowrank_apply_t<float>(p, X, Xadd, out, s);
    return lowrank_apply_t<double>(p, X, Xadd, out, s);
}

// Singular values of the N x L matrix X (descending, FP64 buffer of L): the
// Gram route of the nuclear prox with threshold 0 (every pair with a positive
// eigenvalue is refined in FP64 in FP32 plans), cold-started.
hs_status nuclear_svals(Plan* p, const void* X, double* sv_out, cudaStream_t s) {
    const int L = p->g.L;
    if (L > MAX_L_NUC) return fail(HS_ERR_ARG, "singular values: L = %d exceeds %d", L, MAX_L_NUC);
    HS_TRY(gram_matrix(p, X, nullptr, s));
    if (p->prec == HS_F32) return eig_mixed_launch(p->gram, L, nullptr, 0.0, 1, p->eigf, sv_out, nullptr, nullptr, s);
    return eig_f64_launch(p->gram, L, nullptr, 0.0, 1, p->eigf, sv_out, nullptr, s);
}

// ---------------------------------------------------------------- re-weighting (Algorithm 1)
// w_n = gamma / (gamma + ||A_n||_2) for every row n = (basis, pixel) of the
// coefficient cube A (norm across the L channels).
template <typename R>
__global__ void __launch_bounds__(256) k_rw_rows(const R* __restrict__ A, int L, int64_t N, double gamma,
                                                R* __restrict__ w) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)NB * N) return;
    const int b = (int)(t / N);
    const int64_t base = (int64_t)b * L * N + (t - (int64_t)b * N);
    R s = 0;
    for (int l = 0; l < L; ++l) {
        const R q = A[base + (int64_t)l * N];
        s = fma(q, q, s);
    }
    w[t] = (R)(gamma / (gamma + (double)sqrt(s)));
}

// SARA weights: w_i = gamma / (gamma + |a_i|) for every coefficient.
template <typename R>
__global__ void __launch_bounds__(256) k_rw_coef(const R* __restrict__ A, int64_t n, double gamma,
                                                R* __restrict__ w) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        w[i] = (R)(gamma / (gamma + fabs((double)A[i])));
}

hs_status reweight_coef(Plan* p, const void* A, double gamma, void* w_out, cudaStream_t s) {
    const int64_t n = (int64_t)NB * p->g.L * p->N();
    const unsigned g = std::min<unsigned>(nblk(n, 256), 152u * 16u);
    if (p->prec == HS_F32)
        k_rw_coef<float><<<g, 256, 0, s>>>((const float*)A, n, gamma, (float*)w_out);
    else
        k_rw_coef<double><<<g, 256, 0, s>>>((const double*)A, n, gamma, (double*)w_out);
    HS_CHECK_LAUNCH();
    return HS_OK;
}

// w_j = gamma / (gamma + sigma_j)
__global__ void k_rw_sv(const double* __restrict__ sv, int L, double gamma, double* __restrict__ w) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < L) w[j] = gamma / (gamma + sv[j]);
}

hs_status reweight_rows(Plan* p, const void* A, double gamma, void* w_out, cudaStream_t s) {
    const int64_t N = p->N();
    const unsigned g = nblk((int64_t)NB * N, 256);
    if (p->prec == HS_F32)
        k_rw_rows<float><<<g, 256, 0, s>>>((const float*)A, p->g.L, N, gamma, (float*)w_out);
    else
        k_rw_rows<double><<<g, 256, 0, s>>>((const double*)A, p->g.L, N, gamma, (double*)w_out);
    HS_CHECK_LAUNCH();
    return HS_OK;
}

hs_status reweight_sv(const double* sv, int L, double gamma, double* w_out, cudaStream_t s) {
    k_rw_sv<<<(L + 127) / 128, 128, 0, s>>>(sv, L, gamma, w_out);
    HS_CHECK_LAUNCH();
    return HS_OK;
}

hs_status prox_init() { return gram_tc_init(); }

int64_t gram_part_doubles(int L) { return (int64_t)(L * (L + 1) / 2) * GRAM_CTAS; }

// ---------------------------------------------------------------- primal update
template <typename R>
__global__ void k_primal(int64_t n, const R* __restrict__ P, const R* __restrict__ At,
                         const R* __restrict__ D, R k1, R k2, R k3, R tau, R* __restrict__ X,
                         R* __restrict__ Xt, double* __restrict__ part) {
    __shared__ double red[32];
    R ddr = 0, xxr = 0;   // this thread's sums (few terms); FP64 for the block sums
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        R g = k3 * D[i];
        if (P) g = fma(k1, P[i], g);
        if (At) g = fma(k2, At[i], g);
        const R xo = X[i];
        R xn = xo - tau * g;
        xn = xn > (R)0 ? xn : (R)0;
        X[i] = xn;
        Xt[i] = (R)2 * xn - xo;
        const R df = xn - xo;
        ddr = fma(df, df, ddr);
        xxr = fma(xn, xn, xxr);
    }
    const double dd = block_sum((double)ddr, red);
    const double xx = block_sum((double)xxr, red);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = dd;
        part[2 * blockIdx.x + 1] = xx;
    }
}

// FP32 form of k_primal on 16-byte vectors (n a multiple of 4, buffers 16-byte
// aligned): four elements per load, so each thread keeps several 16-byte loads
// in flight instead of one 4-byte load per loop trip.
__global__ void k_primal4(int64_t n4, const float4* __restrict__ P, const float4* __restrict__ At,
                          const float4* __restrict__ D, float k1, float k2, float k3, float tau,
                          float4* __restrict__ X, float4* __restrict__ Xt, double* __restrict__ part) {
    __shared__ double red[32];
    float ddr = 0.f, xxr = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float4 d = D[i], xo = X[i];
        const float4 pp = P ? P[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 aa = At ? At[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float dv[4] = {d.x, d.y, d.z, d.w}, xv[4] = {xo.x, xo.y, xo.z, xo.w};
        const float pv[4] = {pp.x, pp.y, pp.z, pp.w}, av[4] = {aa.x, aa.y, aa.z, aa.w};
        float xn[4], xt[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float g = k3 * dv[k];
            if (P) g = fmaf(k1, pv[k], g);
            if (At) g = fmaf(k2, av[k], g);
            float v = xv[k] - tau * g;
            v = v > 0.f ? v : 0.f;
            xn[k] = v;
            xt[k] = 2.f * v - xv[k];
            const float df = v - xv[k];
            ddr = fmaf(df, df, ddr);
            xxr = fmaf(v, v, xxr);
        }
        X[i] = make_float4(xn[0], xn[1], xn[2], xn[3]);
        Xt[i] = make_float4(xt[0], xt[1], xt[2], xt[3]);
    }
    const double dd = block_sum((double)ddr, red);
    const double xx = block_sum((double)xxr, red);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = dd;
        part[2 * blockIdx.x + 1] = xx;
    }
}

__global__ void k_beta(const double* __restrict__ part, int nb, double* __restrict__ beta,
                       int64_t* __restrict__ t_count) {
    __shared__ double red[32];
    double dd = 0.0, xx = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        dd += part[2 * b];
        xx += part[2 * b + 1];
    }
    dd = block_sum(dd, red);
    xx = block_sum(xx, red);
    if (threadIdx.x == 0) {
        *beta = (xx > 0.0) ? sqrt(dd / xx) : INFINITY;
        if (t_count) *t_count += 1;   // completed iterations (adaptive bounds)
    }
}

hs_status primal_update(Plan* p, int64_t n, const void* P, const void* At, const void* D,
                        double k1, double k2, double k3, double tau, int use_p, int use_a,
                        void* X, void* Xt, double* part, int nparts, cudaStream_t s) {
    auto a16 = [](const void* q) { return ((uintptr_t)q % 16) == 0; };
    if (p->prec == HS_F32 && n % 4 == 0 && a16(P) && a16(At) && a16(D) && a16(X) && a16(Xt))
        k_primal4<<<nparts, 256, 0, s>>>(n / 4, use_p ? (const float4*)P : nullptr,
                                         use_a ? (const float4*)At : nullptr, (const float4*)D, (float)k1,
                                         (float)k2, (float)k3, (float)tau, (float4*)X, (float4*)Xt, part);
    else if (p->prec == HS_F32)
        k_primal<float><<<nparts, 256, 0, s>>>(n, use_p ? (const float*)P : nullptr,
                                               use_a ? (const float*)At : nullptr, (const float*)D,
                                               (float)k1, (float)k2, (float)k3, (float)tau,
                                               (float*)X, (float*)Xt, part);
    else
        k_primal<double><<<nparts, 256, 0, s>>>(n, use_p ? (const double*)P : nullptr,
                                                use_a ? (const double*)At : nullptr,
                                                (const double*)D, k1, k2, k3, tau, (double*)X,
                                                (double*)Xt, part);
    HS_CHECK_LAUNCH();
    return HS_OK;
}

hs_status beta_from_partials(const double* part, int nparts, double* beta, int64_t* t_count, cudaStream_t s) {
    k_beta<<<1, 256, 0, s>>>(part, nparts, beta, t_count);
    HS_CHECK_LAUNCH();
    return HS_OK;
}

// ---------------------------------------------------------------- channel norms (power iteration)
template <typename R>
__global__ void k_channel_norm(const R* __restrict__ X, int64_t N, double* __restrict__ out) {
    __shared__ double red[32];
    const int l = blockIdx.x;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
        const double v = (double)X[(int64_t)l * N + i];
        s += v * v;
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) out[l] = sqrt(s);
}

template <typename R>
__global__ void k_channel_scale(R* __restrict__ X, int64_t N, const double* __restrict__ nrm) {
    const int l = blockIdx.y;
    const double nv = nrm[l];
    const R f = (R)(nv > 0.0 ? 1.0 / nv : 0.0);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x)
        X[(int64_t)l * N + i] *= f;
}

hs_status channel_norms(Plan* p, const void* X, double* out_dev, cudaStream_t s) {
    if (p->prec == HS_F32) k_channel_norm<float><<<p->g.L, 512, 0, s>>>((const float*)X, p->N(), out_dev);
    else k_channel_norm<double><<<p->g.L, 512, 0, s>>>((const double*)X, p->N(), out_dev);
    HS_CHECK_LAUNCH();
    return HS_OK;
}

hs_status scale_channels(Plan* p, void* X, const double* norms, cudaStream_t s) {
    dim3 g(64, p->g.L);
    if (p->prec == HS_F32) k_channel_scale<float><<<g, 256, 0, s>>>((float*)X, p->N(), norms);
    else k_channel_scale<double><<<g, 256, 0, s>>>((double*)X, p->N(), norms);
    HS_CHECK_LAUNCH();
    return HS_OK;
}

// out[l] = 1 / max_n X[l][n] (0 when the maximum is not positive): the PSF
// normalisation eta_l of the dirty cube.
template <typename R>
__global__ void k_channel_inv_max(const R* __restrict__ X, int64_t N, double* __restrict__ out) {
    __shared__ double red[32];
    const int l = blockIdx.x;
    double m = -1e300;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) m = fmax(m, (double)X[(int64_t)l * N + i]);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = red[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) b = fmax(b, red[w]);
        out[l] = b > 0.0 ? 1.0 / b : 0.0;
    }
}

// X[l][n] *= f[l]
template <typename R>
__global__ void k_channel_mul(R* __restrict__ X, int64_t N, const double* __restrict__ f) {
    const int l = blockIdx.y;
    const R v = (R)f[l];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        X[(int64_t)l * N + i] *= v;
}

// The unit image at the phase centre (pixel (ny / 2, nx / 2)) in every channel.
template <typename R> __global__ void k_set_delta(R* __restrict__ X, int64_t N, int64_t centre) {
    X[(int64_t)blockIdx.x * N + centre] = (R)1;
}

hs_status psf_inv_peak(Plan* p, void* X, double* eta, cudaStream_t s) {
    const int L = p->g.L;
    const int64_t N = p->N(), centre = (int64_t)(p->g.ny / 2) * p->g.nx + p->g.nx / 2;
    HS_CHECK_CUDA(cudaMemsetAsync(X, 0, (size_t)L * N * p->rsize(), s));
    if (p->prec == HS_F32) k_set_delta<float><<<L, 1, 0, s>>>((float*)X, N, centre);
    else k_set_delta<double><<<L, 1, 0, s>>>((double*)X, N, centre);
    HS_CHECK_LAUNCH();
    if (p->M_total > 0) {
        HS_TRY(fft_forward(p, X, s));
        DegridArgs da{};
        da.mode = DOUT_SORTED;
        da.out = p->vis;
        HS_TRY(degrid(p, da, s));
        GridArgs ga{};
        ga.mode = GIN_SORTED;
        ga.in = p->vis;
        HS_TRY(grid(p, ga, s));
        HS_TRY(fft_adjoint(p, X, s));
    } else {
        HS_CHECK_CUDA(cudaMemsetAsync(X, 0, (size_t)L * N * p->rsize(), s));
    }
    if (p->prec == HS_F32) k_channel_inv_max<float><<<L, 256, 0, s>>>((const float*)X, N, eta);
    else k_channel_inv_max<double><<<L, 256, 0, s>>>((const double*)X, N, eta);
    HS_CHECK_LAUNCH();
    return HS_OK;
}

hs_status mul_channels(Plan* p, void* X, const double* f, cudaStream_t s) {
    dim3 g(64, p->g.L);
    if (p->prec == HS_F32) k_channel_mul<float><<<g, 256, 0, s>>>((float*)X, p->N(), f);
    else k_channel_mul<double><<<g, 256, 0, s>>>((double*)X, p->N(), f);
    HS_CHECK_LAUNCH();
    return HS_OK;
}

}  // namespace hs
