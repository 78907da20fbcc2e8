// Eigendecomposition of the L x L Gram matrix S = Z^T Z for the nuclear-norm
// prox (Eq. "prox-L*") of FP32 plans, in one CTA.
//
// The prox needs V diag(f) V^T with f_j = min(1, c_j / sigma_j) (dual form,
// Algorithm 2 step 5) or max(0, 1 - c_j / sigma_j) (prox form), sigma_j =
// sqrt(lambda_j). Only eigenpairs with sigma_j > c_j make f_j differ from its
// limit (1 for the dual, 0 for the prox), so only those "active" pairs must be
// accurate; on GB300 FP64 is ~1/64 of the FP32 rate, so the work is split:
//
//  1. FP32 cyclic Jacobi (round-robin parallel ordering) on S, warm-started
//     from the previous call's eigenvectors V0 (A = V0^T S V0), gives every
//     eigenpair to FP32 accuracy; warm calls skip it while V0 still
//     diagonalises S to 2e-5 (late in a solve, when S changes slowly).
//  2. The active eigenvectors are refined in FP64 against the rest of the
//     basis with first-order correction steps (one from a warm basis, two
//     cold) of an approximate eigendecomposition (Ogita & Aishima 2018): with
//     b_j the basis (the active vectors themselves, then the inactive FP32
//     eigenvectors), T = B^T S X, R = I - B^T X, lambda_c = T_cc / (1 - R_cc),
//     the correction of x_c along b_j (j != c) is
//     (T_jc + lambda_c R_jc) / (lambda_c - lambda_j), and R_jc / 2
//     (orthogonalisation only) along x_c itself or for near-equal eigenvalues
//     (their mixing leaves f, continuous in sigma, unchanged to first order).
//     The eigenvalues are the last step's Rayleigh quotients lambda_c.
//  3. Cholesky QR keeps the active vectors orthonormal in FP64.
//  4. The factor is returned in low-rank form: M = I - sum_active (1 - f) x x^T
//     (dual) or sum_active f x x^T (prox), as r, g and the active x.
#include <cmath>

#include "hs_device.cuh"
#include "hs_internal.h"

namespace hs {

constexpr int EIG_T = 1024;
constexpr int LD32 = MAX_L_NUC + 1;

// Block-wide sum of doubles, returned to every thread (red: 33 doubles).
__device__ __forceinline__ double eig_bsum(double v, double* red) { return block_sum_all(v, red); }

// Round-robin (circle method) schedule for n indices, n even: in round r the
// index n-1 meets r and (r + i) meets (r - i) (mod n-1) for i = 1 .. n/2-1.
// pairs[r * n/2 + k] = p | q << 8 (p < q) is the k-th pair of round r (thread r
// lists its round).
__device__ void rr_schedule(int n, unsigned short* pairs) {
    for (int r = threadIdx.x; r < n - 1; r += blockDim.x) {
        int k = 0;
        for (int i = 0; i < n; ++i) {
            int pi;
            if (i == n - 1) pi = r;
            else if (i == r) pi = n - 1;
            else pi = ((2 * r - i) % (n - 1) + (n - 1)) % (n - 1);
            if (i < pi) pairs[r * (n / 2) + k++] = (unsigned short)(i | (pi << 8));
        }
    }
}

// Rotation (c, s) that zeroes a_pq of the 2 x 2 block [[a_pp, a_pq], [a_pq, a_qq]]
// (Golub & Van Loan Alg. 8.4.1). FP32: fast reciprocal and reciprocal square
// root (the FP32 sweeps only need FP32-orthogonal rotations); FP64: IEEE.
__device__ __forceinline__ void jac_rot(float app, float aqq, float apq, float& c, float& s) {
    const float tau = __fdividef(aqq - app, 2.f * apq);
    const float t = copysignf(1.f, tau) * __frcp_rn(fabsf(tau) + sqrtf(fmaf(tau, tau, 1.f)));
    c = rsqrtf(fmaf(t, t, 1.f));
    s = t * c;
}
__device__ __forceinline__ void jac_rot(double app, double aqq, double apq, double& c, double& s) {
    const double tau = (aqq - app) / (2.0 * apq);
    const double t = copysign(1.0, tau) / (fabs(tau) + sqrt(fma(tau, tau, 1.0)));
    c = rsqrt(fma(t, t, 1.0));
    s = t * c;
}

// Cyclic Jacobi, round-robin parallel ordering, on the symmetric N x N matrix
// in A (leading dimension LDJ), accumulating V <- V J. Each round, thread k < N/2
// computes the rotation (c_k, s_k) of pair k = (p, q) from a_pp, a_qq, a_pq
// (J_pp = J_qq = c, J_pq = s, J_qp = -s); then thread (i, j) of the (N/2)^2
// grid applies A <- J^T A J to the 2 x 2 block (rows of pair i, columns of
// pair j):
//   rows   (p, q) <- (c_i row_p - s_i row_q, s_i row_p + c_i row_q)
//   cols   (p, q) <- (c_j col_p - s_j col_q, s_j col_p + c_j col_q),
// and rotates columns (p_j, q_j) of V in rows i and i + N/2. Every entry belongs
// to one thread per round, so A and V are updated in place. A rotation is
// applied only when |a_pq| exceeds skip sqrt(|a_pp a_qq|) and floor_rel ||A||_F;
// sweeps stop when the off-diagonal Frobenius norm is at most off_rel ||A||_F,
// when a sweep applies no rotation, or after max_sweeps.
template <typename T, int N>
__device__ void jacobi_blocks(T* A, T* V, unsigned short* pairs, double skip, double floor_rel,
                              double off_rel, int max_sweeps, Cx<T>* cs, double* red, int* flag) {
    constexpr int LDJ = MAX_L_NUC + 1;
    constexpr int NP = N / 2;
    constexpr int LG = (N >= 64) ? 6 : (N >= 32) ? 5 : (N >= 16) ? 4 : (N >= 8) ? 3 : (N >= 4) ? 2 : 1;
    const int tid = threadIdx.x, nt = blockDim.x;
    const T skip2 = (T)(skip * skip);
    const int bi = tid / NP, bj = tid - (tid / NP) * NP;   // block of this thread (tid < NP^2)
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        T nrmT = 0, offT = 0;   // per-thread partial sums in the working precision
        for (int k = tid; k < N * N; k += nt) {
            const int i = k >> LG, j = k & (N - 1);
            const T x = A[i * LDJ + j];
            nrmT = fma(x, x, nrmT);
            if (i != j) offT = fma(x, x, offT);
        }
        const double nrm = eig_bsum((double)nrmT, red);
        const double off = eig_bsum((double)offT, red);
        if (!(off > off_rel * off_rel * nrm)) break;
        if (sweep == 0) {   // the round-robin schedule, built only when a sweep runs
            rr_schedule(N, pairs);
            __syncthreads();
        }
        const T flo = (T)(floor_rel * sqrt(nrm));
        if (tid == 0) *flag = 0;
        __syncthreads();
        for (int r = 0; r < N - 1; ++r) {
            const unsigned short* pr = pairs + r * NP;
            if (tid < NP) {
                const int pq = pr[tid], p = pq & 0xff, q = pq >> 8;
                const T apq = A[p * LDJ + q], app = A[p * LDJ + p], aqq = A[q * LDJ + q];
                T c = 1, s = 0;
                const T ab = fabs(apq);
                if (ab > flo && ab * ab > skip2 * fabs(app * aqq)) {
                    jac_rot(app, aqq, apq, c, s);
                    *flag = 1;
                }
                Cx<T> v;
                v.x = c;
                v.y = s;
                cs[tid] = v;
            }
            __syncthreads();
            if (tid < NP * NP) {
                const int pqi = pr[bi], pqj = pr[bj];
                const int pi = pqi & 0xff, qi = pqi >> 8, pj = pqj & 0xff, qj = pqj >> 8;
                const Cx<T> csi = cs[bi], csj = cs[bj];
                const T ci = csi.x, si = csi.y, cj = csj.x, sj = csj.y;
                const T a00 = A[pi * LDJ + pj], a01 = A[pi * LDJ + qj];
                const T a10 = A[qi * LDJ + pj], a11 = A[qi * LDJ + qj];
                const T v00 = V[bi * LDJ + pj], v01 = V[bi * LDJ + qj];
                const T v10 = V[(bi + NP) * LDJ + pj], v11 = V[(bi + NP) * LDJ + qj];
                const T r0x = ci * a00 - si * a10, r0y = ci * a01 - si * a11;
                const T r1x = si * a00 + ci * a10, r1y = si * a01 + ci * a11;
                T b00 = cj * r0x - sj * r0y, b01 = sj * r0x + cj * r0y;
                T b10 = cj * r1x - sj * r1y, b11 = sj * r1x + cj * r1y;
                if (bi == bj && si != T(0)) {   // the rotated pair is decoupled
                    b01 = T(0);
                    b10 = T(0);
                }
                A[pi * LDJ + pj] = b00;
                A[pi * LDJ + qj] = b01;
                A[qi * LDJ + pj] = b10;
                A[qi * LDJ + qj] = b11;
                V[bi * LDJ + pj] = cj * v00 - sj * v01;
                V[bi * LDJ + qj] = sj * v00 + cj * v01;
                V[(bi + NP) * LDJ + pj] = cj * v10 - sj * v11;
                V[(bi + NP) * LDJ + qj] = sj * v10 + cj * v11;
            }
            __syncthreads();
        }
        const int any = *flag;
        __syncthreads();
        if (!any) break;
    }
}

// Dispatch on the padded size n (power of two, 2..64). B and W are unused
// scratch kept for the callers' layouts.
template <typename T>
__device__ void jacobi_n(int n, T* A, T* B, T* V, T* W, unsigned short* pairs, double skip,
                         double floor_rel, double off_rel, int max_sweeps, Cx<T>* cs, double* red, int* flag) {
    (void)B;
    (void)W;
#define HS_JAC(NN) jacobi_blocks<T, NN>(A, V, pairs, skip, floor_rel, off_rel, max_sweeps, cs, red, flag)
    switch (n) {
        case 2: HS_JAC(2); break;
        case 4: HS_JAC(4); break;
        case 8: HS_JAC(8); break;
        case 16: HS_JAC(16); break;
        case 32: HS_JAC(32); break;
        default: HS_JAC(64); break;
    }
#undef HS_JAC
}

// One CTA of EIG_T threads; dynamic shared memory layout below.
__global__ void __launch_bounds__(EIG_T) k_eig_mixed(const double* __restrict__ Sg, int L,
                                                    const double* __restrict__ w_sv, double thr,
                                                    int dual, double* __restrict__ Mf,
                                                    double* __restrict__ sv_out,
                                                    float* __restrict__ warm, int* __restrict__ r_out) {
    extern __shared__ __align__(16) unsigned char eig_smem[];
    constexpr int SL = MAX_L_NUC * LD32;                 // one 64 x 65 slot
    float* V32 = (float*)eig_smem;                       // slot 0
    float* W32 = V32 + SL;                               // slot 1 (Jacobi scratch)
    float* A32 = W32 + SL;                               // slot 2
    float* B32 = A32 + SL;                               // slot 3 (Jacobi scratch, warm-start temp)
    float* T32 = B32;
    double* Sd = (double*)(B32 + SL);                    // 64 x 65 doubles each from here
    double* X = Sd + SL;                                 // active vectors (columns)
    double* Y = X + SL;
    double* Rb = Y + SL;
    // FP64 view over float slots 2-3 once the FP32 Jacobi matrix is dead
    double* Tb = (double*)A32;
    __shared__ double red[33];
    __shared__ float2 cs32[MAX_L_NUC / 2];
    __shared__ unsigned short partner[(MAX_L_NUC - 1) * MAX_L_NUC / 2];
    __shared__ int flag;
    __shared__ double lam32[MAX_L_NUC], lamr[MAX_L_NUC], fv[MAX_L_NUC];
    __shared__ float lamf[MAX_L_NUC];
    __shared__ int order[MAX_L_NUC];
    __shared__ int r_act;
    const int tid = threadIdx.x, nt = blockDim.x;
    int n = 2;
    while (n < L) n <<= 1;
    // ---- load S (FP64) and its FP32 copy
    for (int k = tid; k < n * n; k += nt) {
        const int i = k / n, j = k - i * n;
        const double v = (i < L && j < L) ? Sg[i * L + j] : 0.0;
        Sd[i * MAX_L_NUC + j] = v;
        A32[i * LD32 + j] = (float)v;
        V32[i * LD32 + j] = (warm && i < L && j < L) ? warm[i * L + j] : (i == j ? 1.f : 0.f);
    }
    __syncthreads();
    if (warm) {   // A = V0^T S V0 (FP32), then symmetrise; 2 x 2 output blocks per thread
        const int nh = n >> 1;
        for (int k = tid; k < nh * nh; k += nt) {   // T = S V0
            const int i = 2 * (k / nh), j = 2 * (k % nh);
            float a00 = 0.f, a01 = 0.f, a10 = 0.f, a11 = 0.f;
            for (int m = 0; m < n; ++m) {
                const float s0 = A32[i * LD32 + m], s1 = A32[(i + 1) * LD32 + m];
                const float v0 = V32[m * LD32 + j], v1 = V32[m * LD32 + j + 1];
                a00 = fmaf(s0, v0, a00);
                a01 = fmaf(s0, v1, a01);
                a10 = fmaf(s1, v0, a10);
                a11 = fmaf(s1, v1, a11);
            }
            T32[i * LD32 + j] = a00;
            T32[i * LD32 + j + 1] = a01;
            T32[(i + 1) * LD32 + j] = a10;
            T32[(i + 1) * LD32 + j + 1] = a11;
        }
        __syncthreads();
        for (int k = tid; k < nh * nh; k += nt) {   // A = V0^T T
            const int i = 2 * (k / nh), j = 2 * (k % nh);
            float a00 = 0.f, a01 = 0.f, a10 = 0.f, a11 = 0.f;
            for (int m = 0; m < n; ++m) {
                const float u0 = V32[m * LD32 + i], u1 = V32[m * LD32 + i + 1];
                const float t0 = T32[m * LD32 + j], t1 = T32[m * LD32 + j + 1];
                a00 = fmaf(u0, t0, a00);
                a01 = fmaf(u0, t1, a01);
                a10 = fmaf(u1, t0, a10);
                a11 = fmaf(u1, t1, a11);
            }
            A32[i * LD32 + j] = a00;
            A32[i * LD32 + j + 1] = a01;
            A32[(i + 1) * LD32 + j] = a10;
            A32[(i + 1) * LD32 + j + 1] = a11;
        }
        __syncthreads();
        for (int k = tid; k < n * n; k += nt) {
            const int i = k / n, j = k - i * n;
            if (i < j) {
                const float a = 0.5f * (A32[i * LD32 + j] + A32[j * LD32 + i]);
                A32[i * LD32 + j] = a;
                A32[j * LD32 + i] = a;
            }
        }
        __syncthreads();
    }
    // ---- 1. FP32 Jacobi on every eigenpair
    // warm-started calls run at most one FP32 sweep, and none while the previous
    // basis still diagonalises S to 2e-5 (relative off-diagonal Frobenius norm,
    // about twice the FP32 rounding of V0^T S V0): the active pairs are made exact in
    // FP64 below from a basis that accurate, and the basis is swept again as
    // soon as S has drifted further
    jacobi_n<float>(n, A32, B32, V32, W32, partner, 1e-7, 2e-7, warm ? 2e-5 : 2e-6, warm ? 1 : 15, cs32, red,
                    &flag);
    // ---- eigenvalues, descending order (rank by counting), warm start for the next call
    if (tid < L) {
        lamf[tid] = A32[tid * LD32 + tid];
        lam32[tid] = (double)lamf[tid];
    }
    if (tid == 0) r_act = 0;
    __syncthreads();
    if (tid < L) {   // rank of eigenvalue tid; active when sigma > c_rank (1 - 1e-3)
        // a NaN (from a non-finite input) ranks below every number, so the ranks stay a
        // permutation and every index taken from `order` stays in range
        int rk = 0;
        const float li = isnan(lamf[tid]) ? -INFINITY : lamf[tid];
        for (int j = 0; j < L; ++j) {
            const float lj = isnan(lamf[j]) ? -INFINITY : lamf[j];
            rk += (lj > li) || (lj == li && j < tid);
        }
        order[rk] = tid;
        const double c = thr * (w_sv ? w_sv[rk] : 1.0) * (1.0 - 1e-3);
        if ((double)fmaxf(li, 0.f) > c * c) atomicMax(&r_act, rk + 1);
    }
    if (warm)
        for (int k = tid; k < L * L; k += nt) warm[k] = V32[(k / L) * LD32 + (k % L)];
    __syncthreads();
    if (tid == 0 && r_out) *r_out = r_act;
    const int r = r_act;
    if (r > 0) {
        // active vectors in FP64
        for (int k = tid; k < L * r; k += nt) {
            const int i = k / r, c = k - i * r;
            X[i * MAX_L_NUC + c] = (double)V32[i * LD32 + order[c]];
        }
        __syncthreads();
        // ---- 2. FP64 correction steps of the active vectors against the whole basis
        // (the first-order step squares the FP32 error: one suffices from a warm basis)
        const int nsteps = warm ? 1 : 2;
        for (int step = 0; step < nsteps; ++step) {
            // Y = S X
            for (int k = tid; k < L * r; k += nt) {
                const int i = k / r, c = k - i * r;
                double acc = 0.0;
                for (int m = 0; m < L; ++m) acc = fma(Sd[i * MAX_L_NUC + m], X[m * MAX_L_NUC + c], acc);
                Y[i * MAX_L_NUC + c] = acc;
            }
            __syncthreads();
            // T_jc = b_j . Y_c, R_jc = delta_jc - b_j . X_c   (b_j = X_j for j < r, else V32 column)
            for (int k = tid; k < L * r; k += nt) {
                const int j = k / r, c = k - j * r;
                double t = 0.0, q = 0.0;
                if (j < r) {
                    for (int m = 0; m < L; ++m) {
                        const double b = X[m * MAX_L_NUC + j];
                        t = fma(b, Y[m * MAX_L_NUC + c], t);
                        q = fma(b, X[m * MAX_L_NUC + c], q);
                    }
                } else {
                    const int col = order[j];
                    for (int m = 0; m < L; ++m) {
                        const double b = (double)V32[m * LD32 + col];
                        t = fma(b, Y[m * MAX_L_NUC + c], t);
                        q = fma(b, X[m * MAX_L_NUC + c], q);
                    }
                }
                Tb[j * MAX_L_NUC + c] = t;
                Rb[j * MAX_L_NUC + c] = (j == c ? 1.0 : 0.0) - q;
            }
            __syncthreads();
            if (tid < r) lamr[tid] = Tb[tid * MAX_L_NUC + tid] / (1.0 - Rb[tid * MAX_L_NUC + tid]);
            __syncthreads();
            const double delta = 1e-5 * fmax(fabs(lamr[0]), 1e-300);
            // E_jc into Tb (overwrites T in place: each entry read once by its own thread)
            for (int k = tid; k < L * r; k += nt) {
                const int j = k / r, c = k - j * r;
                const double t = Tb[j * MAX_L_NUC + c], q = Rb[j * MAX_L_NUC + c];
                double e;
                const double gap = lamr[c] - (j < r ? lamr[j] : lam32[order[j]]);
                e = (j != c && fabs(gap) > delta) ? (t + lamr[c] * q) / gap : 0.5 * q;
                Tb[j * MAX_L_NUC + c] = e;
            }
            __syncthreads();
            // X_new = X + B E  (into Y)
            for (int k = tid; k < L * r; k += nt) {
                const int i = k / r, c = k - i * r;
                double acc = X[i * MAX_L_NUC + c];
                for (int j = 0; j < r; ++j) acc = fma(X[i * MAX_L_NUC + j], Tb[j * MAX_L_NUC + c], acc);
                for (int j = r; j < L; ++j)
                    acc = fma((double)V32[i * LD32 + order[j]], Tb[j * MAX_L_NUC + c], acc);
                Y[i * MAX_L_NUC + c] = acc;
            }
            __syncthreads();
            for (int k = tid; k < L * r; k += nt) {
                const int i = k / r, c = k - i * r;
                X[i * MAX_L_NUC + c] = Y[i * MAX_L_NUC + c];
            }
            __syncthreads();
        }
        // ---- 3. orthonormalise the active vectors (Cholesky QR: G = X^T X = R^T R,
        //      X <- X R^{-1}; X is orthonormal to first order already, so G ~ I)
        for (int k = tid; k < r * r; k += nt) {
            const int a = k / r, b = k - a * r;
            if (a <= b) {
                double acc = 0.0;
                for (int m = 0; m < L; ++m) acc = fma(X[m * MAX_L_NUC + a], X[m * MAX_L_NUC + b], acc);
                Tb[a * LD32 + b] = acc;
            }
        }
        __syncthreads();
        if (tid < 32) {   // upper-triangular R in place of G, one warp, lanes over columns
            for (int j = 0; j < r; ++j) {
                if (tid == 0) {
                    double d = Tb[j * LD32 + j];
                    for (int k = 0; k < j; ++k) d -= Tb[k * LD32 + j] * Tb[k * LD32 + j];
                    Tb[j * LD32 + j] = sqrt(fmax(d, 1e-300));
                }
                __syncwarp();
                const double rjj = Tb[j * LD32 + j];
                for (int i = j + 1 + tid; i < r; i += 32) {
                    double v = Tb[j * LD32 + i];
                    for (int k = 0; k < j; ++k) v -= Tb[k * LD32 + j] * Tb[k * LD32 + i];
                    Tb[j * LD32 + i] = v / rjj;
                }
                __syncwarp();
            }
        }
        __syncthreads();
        for (int m = tid; m < L; m += nt) {   // row m of X times R^{-1} (forward substitution)
            for (int j = 0; j < r; ++j) {
                double v = X[m * MAX_L_NUC + j];
                for (int k = 0; k < j; ++k) v -= X[m * MAX_L_NUC + k] * Tb[k * LD32 + j];
                X[m * MAX_L_NUC + j] = v / Tb[j * LD32 + j];
            }
        }
        __syncthreads();
        // eigenvalues: the last step's Rayleigh quotients (second-order accurate)
        if (tid < r) {
            const double sig = sqrt(fmax(lamr[tid], 0.0));
            const double c = thr * (w_sv ? w_sv[tid] : 1.0);
            double f;
            if (dual) f = (sig > c) ? c / sig : 1.0;
            else f = (sig > c) ? 1.0 - c / sig : 0.0;
            if (sv_out) sv_out[tid] = sig;
            fv[tid] = f;   // factor of active vector tid
        }
        __syncthreads();
    }
    if (sv_out)
        for (int j = r + tid; j < L; j += nt) sv_out[j] = sqrt(fmax(lam32[order[j]], 0.0));
    // ---- 4. low-rank factor: M = I + sum_c (f_c - 1) y_c y_c^T (dual) or sum_c f_c y_c y_c^T
    if (tid == 0) {
        Mf[LR_R] = (double)r;
        Mf[LR_BASE] = dual ? 1.0 : 0.0;
    }
    float* Ff = reinterpret_cast<float*>(Mf + LR_DOUBLES);   // FP32 copies for the apply kernel
    if (tid < r) {
        const double g = dual ? fv[tid] - 1.0 : fv[tid];
        Mf[LR_G + tid] = g;
        Ff[LRF_G + tid] = (float)g;
    }
    for (int k = tid; k < L * r; k += nt) {
        const int i = k / r, c = k - i * r;
        const double x = X[i * MAX_L_NUC + c];
        const float xh = (float)x;
        Mf[LR_X + c * MAX_L_NUC + i] = x;
        Ff[LRF_XH + c * MAX_L_NUC + i] = xh;
        Ff[LRF_XL + c * MAX_L_NUC + i] = (float)(x - (double)xh);
    }
}

size_t eig_mixed_smem() {
    return (size_t)4 * MAX_L_NUC * LD32 * sizeof(float) + (size_t)4 * MAX_L_NUC * LD32 * sizeof(double);
}

// FP64 plans: the whole Gram matrix is diagonalised by the FP64 Jacobi method;
// f and the low-rank factor as in k_eig_mixed (all eigenpairs are FP64-accurate).
__global__ void __launch_bounds__(EIG_T) k_eig_f64(const double* __restrict__ Sg, int L,
                                                  const double* __restrict__ w_sv, double thr, int dual,
                                                  double* __restrict__ Mf, double* __restrict__ sv_out,
                                                  int* __restrict__ r_out) {
    extern __shared__ __align__(16) unsigned char eig_smem[];
    constexpr int SL = MAX_L_NUC * LD32;
    double* A = (double*)eig_smem;
    double* B = A + SL;
    double* V = B + SL;
    double* W = V + SL;
    __shared__ double red[33];
    __shared__ double lam[MAX_L_NUC], fv[MAX_L_NUC];
    __shared__ double2 cs[MAX_L_NUC / 2];
    __shared__ int order[MAX_L_NUC];
    __shared__ unsigned short partner[(MAX_L_NUC - 1) * MAX_L_NUC / 2];
    __shared__ int flag;
    const int tid = threadIdx.x, nt = blockDim.x;
    int n = 2;
    while (n < L) n <<= 1;
    for (int k = tid; k < n * n; k += nt) {
        const int i = k / n, j = k - i * n;
        A[i * LD32 + j] = (i < L && j < L) ? Sg[i * L + j] : 0.0;
        V[i * LD32 + j] = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();
    jacobi_n<double>(n, A, B, V, W, partner, 1e-17, 1e-18, 1e-16, 40, cs, red, &flag);
    if (tid < L) lam[tid] = A[tid * LD32 + tid];
    __syncthreads();
    if (tid < L) {   // NaN ranks last (the ranks stay a permutation)
        int rk = 0;
        const double li = isnan(lam[tid]) ? -INFINITY : lam[tid];
        for (int j = 0; j < L; ++j) {
            const double lj = isnan(lam[j]) ? -INFINITY : lam[j];
            rk += (lj > li) || (lj == li && j < tid);
        }
        order[rk] = tid;
    }
    __syncthreads();
    if (tid == 0) {
        int r = 0;
        for (int j = 0; j < L; ++j) {
            const double sig = sqrt(fmax(lam[order[j]], 0.0));
            const double c = thr * (w_sv ? w_sv[j] : 1.0);
            double f;
            if (dual) f = (sig > c) ? c / sig : 1.0;
            else f = (sig > c) ? 1.0 - c / sig : 0.0;
            fv[j] = f;
            if (sv_out) sv_out[j] = sig;
            if (sig > c) r = j + 1;
        }
        if (r_out) *r_out = r;
    }
    __syncthreads();
    // low-rank factor over the pairs with sigma > c (f differs from its limit only there)
    __shared__ int r_act;
    if (tid == 0) {
        int r = 0;
        for (int j = 0; j < L; ++j)
            if (sqrt(fmax(lam[order[j]], 0.0)) > thr * (w_sv ? w_sv[j] : 1.0)) r = j + 1;
        r_act = r;
        Mf[LR_R] = (double)r;
        Mf[LR_BASE] = dual ? 1.0 : 0.0;
    }
    __syncthreads();
    const int r = r_act;
    if (tid < r) Mf[LR_G + tid] = dual ? fv[tid] - 1.0 : fv[tid];
    for (int k = tid; k < L * r; k += nt) {
        const int i = k / r, c = k - i * r;
        Mf[LR_X + c * MAX_L_NUC + i] = V[i * LD32 + order[c]];
    }
}

hs_status eig_f64_launch(const double* S, int L, const double* w_sv, double thr, int dual, double* Mf,
                         double* sv_out, int* r_out, cudaStream_t s) {
    const size_t sm = (size_t)4 * MAX_L_NUC * LD32 * sizeof(double);
    k_eig_f64<<<1, EIG_T, sm, s>>>(S, L, w_sv, thr, dual, Mf, sv_out, r_out);
    HS_CHECK_LAUNCH();
    return HS_OK;
}

hs_status eig_init() {
    static bool done = false;
    if (done) return HS_OK;
    HS_CHECK_CUDA(cudaFuncSetAttribute(k_eig_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)eig_mixed_smem()));
    HS_CHECK_CUDA(cudaFuncSetAttribute(k_eig_f64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(4 * MAX_L_NUC * LD32 * sizeof(double))));
    done = true;
    return HS_OK;
}

hs_status eig_mixed_launch(const double* S, int L, const double* w_sv, double thr, int dual,
                           double* Mf, double* sv_out, float* warm, int* r_out, cudaStream_t s) {
    k_eig_mixed<<<1, EIG_T, eig_mixed_smem(), s>>>(S, L, w_sv, thr, dual, Mf, sv_out, warm, r_out);
    HS_CHECK_LAUNCH();
    return HS_OK;
}

}  // namespace hs
