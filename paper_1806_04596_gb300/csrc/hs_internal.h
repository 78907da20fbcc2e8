// Internal declarations of the HyperSARA GB300 library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/hypersara.h"

namespace hs {

// ---------------------------------------------------------------- errors
hs_status fail(hs_status st, const char* fmt, ...);
void clear_error();

#define HS_CHECK_CUDA(call)                                                              \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return ::hs::fail(HS_ERR_CUDA, "%s:%d %s: %s", __FILE__, __LINE__, #call,    \
                              cudaGetErrorString(e_));                                   \
    } while (0)

#define HS_CHECK_LAUNCH() HS_CHECK_CUDA(cudaGetLastError())

#define HS_TRY(expr)                          \
    do {                                      \
        hs_status s_ = (expr);                \
        if (s_ != HS_OK) return s_;           \
    } while (0)

// ---------------------------------------------------------------- constants
constexpr int KB_J = 8;              // interpolation support (cells per axis)
constexpr int NB = 9;                // SARA bases: Dirac + db1..db8
constexpr int NW = 8;                // wavelet bases
constexpr int MAXF = 16;             // longest filter (db8)
constexpr int KB_TERMS_F32 = 9;      // polynomial coefficients per unit piece, FP32
constexpr int KB_TERMS_F64 = 14;     // ... FP64
constexpr int KB_HALF = 7;           // even (or odd) coefficients of a piece, at most
constexpr int GRID_TILE = 32;        // gridding tile side (cells)
constexpr int GRID_WARPS = 4;        // warps per gridding CTA (private accumulators)
constexpr int GRID_CAP = 512;        // most list entries one gridding CTA processes
constexpr int DEGRID_CHUNK = 256;    // visibilities per degridding CTA
constexpr int SWEEP_HMAX = 64;       // most output rows of one sweep-gridding work item
constexpr int SWEEP_CAP = 1024;      // windows above which a sweep item's rows are cut short

// Sweep-gridding work item (grids of at least 64 x 64 cells): channel l, the
// 32-column strip `strip`, output rows [row0, row1); list range [e0, e1) of
// groups of 4 slots (see the plan builder).
struct SweepItem {
    int l, strip, row0, row1, e0, e1;
};
constexpr int MAX_L_NUC = 64;        // largest L for the nuclear-norm prox
// Low-rank form of the nuclear prox factor M = base I + sum_c g_c x_c x_c^T
// (doubles in Plan::eigf): [LR_R] active count r, [LR_BASE] 1 (dual) or 0,
// [LR_G + c] g_c, [LR_X + c * MAX_L_NUC + i] component i of x_c.
// Followed by FP32 copies for FP32 plans, as floats from double offset LR_DOUBLES:
// [LRF_XH + c * MAX_L_NUC + i] hi part of x_ci, [LRF_XL + ...] lo part
// (x = hi + lo to FP64 rounding), [LRF_G + c] g_c.
constexpr int LR_R = 0, LR_BASE = 1, LR_G = 2, LR_X = 2 + MAX_L_NUC;
constexpr int LR_DOUBLES = LR_X + MAX_L_NUC * MAX_L_NUC;
constexpr int LRF_XH = 0, LRF_XL = MAX_L_NUC * MAX_L_NUC, LRF_G = 2 * MAX_L_NUC * MAX_L_NUC;
constexpr int LR_TOTAL_DOUBLES = LR_DOUBLES + (LRF_G + MAX_L_NUC + 1) / 2;

// Coordinates of one visibility in an FP64 plan: window start cells and the
// fractional part of t = u K / (2 pi) (exact in FP64).
struct Coord64 {
    double fx, fy;
    int cx, cy;   // floor(t) mod K per axis
};

// Sizes passed by value to kernels.
struct Geo {
    int nx, ny, L, Kx, Ky;
    int fbx, fby;          // fractional bits of the FP32 fixed-point coordinates
    int tx, ty, ntx, nty;  // gridding tile size and tiles per axis
    int kxm, kym;          // Kx - 1, Ky - 1 for powers of two, else -1 (wrapn)
};

// ---------------------------------------------------------------- plan
struct Plan {
    Geo g{};
    int levels = 4;
    int J = 8, o = 2;
    hs_prec prec = HS_F32;
    unsigned flags = 0;
    double beta = 0.0;
    int kb_terms = 0;
    double kb_fit_err = 0.0;
    int64_t M_total = 0;
    int Mmax = 0;
    std::vector<int64_t> off_h;
    std::vector<int64_t> blk_off_h;    // data blocks (caller = sorted boundaries), nblk + 1
    std::vector<int> blk_ch;           // channel of every block
    int nblk = 0;
    int* blk_id = nullptr;             // block of every sorted visibility (only when nblk != L)
    int64_t* off_d = nullptr;          // L+1
    int* perm = nullptr;               // sorted index -> caller index
    void* coords = nullptr;            // FP32: uint2 fixed point; FP64: Coord64
    void* w_sorted = nullptr;          // Theta in sorted order (real) or null
    void* u_sorted = nullptr;          // U in sorted order (real) or null
    int64_t n_ent = 0;
    int64_t* tile_off = nullptr;       // L * ntiles + 1
    void* dg_items = nullptr;          // de-gridding work items {tix, e0, e1, slot}
    int64_t n_dg_items = 0;
    int dg_items_max = 0;              // most items of one channel (partial-sum stride)
    int* tile_ent = nullptr;           // per (channel, tile): groups of 4 sorted visibility indices
                                       // with non-overlapping windows, -1 = padding
    void* grid_items = nullptr;        // gridding work items {tix, e0, e1, slot}
    int64_t n_items = 0;
    void* grid_merges = nullptr;       // split tiles {tix, slot0, nslot}
    int64_t n_merges = 0;
    void* grid_partial = nullptr;      // partial tiles of split tiles (complex, slots x tile)
    void* sw_items = nullptr;          // sweep-gridding work items (SweepItem), heaviest first
    int64_t n_sw_items = 0;
    int* sw_ent = nullptr;             // sweep lists: groups of 4 sorted visibility indices, -1 = padding
    int64_t n_sw_ent = 0;
    void* kbc = nullptr;               // 8 * kb_terms reals
    std::vector<double> kbc_h;         // the same on the host
    cudaStream_t fft_side = nullptr;   // row passes of a chunked F^H (overlap the next chunk's column pass)
    cudaEvent_t fft_ev_col = nullptr, fft_ev_join = nullptr;
    void* cxs = nullptr;               // nx reals (Z scale along x)
    void* cys = nullptr;               // ny reals
    void* twx = nullptr;               // Kx complex, exp(-2 pi i m / Kx)
    void* twy = nullptr;               // Ky complex
    void* filt = nullptr;              // 8 * 2 * MAXF reals: lowpass, highpass per db_p
    // scratch
    void* grid = nullptr;              // L * Ky * Kx complex
    void* tmp = nullptr;               // L * ny * Kx complex
    void* vis = nullptr;               // M_total complex (sorted order)
    void* dwt_a = nullptr;             // 8 * L * N reals
    void* dwt_b = nullptr;             // 8 * L * N reals
    double* part = nullptr;            // partial sums (size part_n doubles)
    int64_t part_n = 0;
    double* gram = nullptr;            // MAX_L_NUC^2 doubles
    double* eigf = nullptr;            // LR_TOTAL_DOUBLES: low-rank prox factor (layout above)
    double* sv = nullptr;              // MAX_L_NUC doubles
    double* dscal = nullptr;           // small per-channel doubles (4 * L)
    int* err_d = nullptr;              // device error flag: a bounded device-side wait expired
    // parameters chosen by the plan-time autotuner (defaults without it)
    int gram_tc = 1;                   // FP32 Gram matrix on the tensor cores (else CUDA cores)
    int sweep_hmax = SWEEP_HMAX;       // sweep gridding: most output rows per work item
    int sweep_cap = SWEEP_CAP;         // ... windows above which an item's rows are cut short
    int fft_adj_chunk = 0;             // channels per F^H chunk (0: all at once)
    int tuned = 0;                     // 1: timed at creation, 2: taken from the process cache
    double tune_ms = 0.0;              // host time spent tuning
    double tune_grid_ms[3] = {0, 0, 0};   // gridding launch time per candidate
    double tune_gram_ms[2] = {0, 0};      // Gram time: tensor cores, CUDA cores
    double tune_fft_ms[2] = {0, 0};       // F^H time: all channels at once, L2-sized chunks
    void* xbuf = nullptr;              // L * N reals (power iteration, misc)
    void* xbuf2 = nullptr;             // L * N reals
    int64_t device_bytes = 0;
    std::vector<void*> allocs;
    std::vector<size_t> alloc_bytes;

    int64_t N() const { return (int64_t)g.nx * g.ny; }
    int64_t ntiles() const { return (int64_t)g.ntx * g.nty; }
    size_t rsize() const { return prec == HS_F64 ? 8 : 4; }
    size_t csize() const { return 2 * rsize(); }
};

// Device allocation tracked by the plan (freed in destroy).
hs_status plan_alloc(Plan* p, void** ptr, size_t bytes);
// Every device allocation of the library goes through these (process-wide
// accounting and the optional limit of hs_set_device_limit).
hs_status lib_alloc(void** ptr, size_t bytes);
void lib_free(void* ptr, size_t bytes);
void set_device_limit(int64_t bytes);
int64_t device_bytes_held();

// ---------------------------------------------------------------- host tables
hs_status daubechies_lowpass(int p, double* out);
double kb_phi(double x, int J, double beta);
double kb_phihat(double f, int J, double beta);
// Fits phi(m + f), f in [0,1), m = -J/2 .. J/2-1, as polynomials in s = 2f - 1
// with `terms` coefficients each (ascending powers). Returns the max error / phi(0).
double kb_poly_fit(int J, double beta, int terms, std::vector<double>* coef);
// Sweep-gridding work lists (host only): windows with start cells k0x[r], k0y[r],
// channel ranges off[0..L]; list entries are the positions r.
// Rows are cut after hmax rows, or earlier once a list would pass cap windows.
hs_status sweep_lists(int Kx, int Ky, int L, const int64_t* off, const int* k0x, const int* k0y, int hmax,
                      int cap, std::vector<SweepItem>& items, std::vector<int>& ent);

// ---------------------------------------------------------------- launches
// Visibility input / output modes of the gridding and de-gridding kernels.
enum DegridOut { DOUT_CALLER = 0, DOUT_SORTED = 1, DOUT_SORTED_U = 2, DOUT_PD = 3 };
enum GridIn { GIN_CALLER = 0, GIN_SORTED = 1, GIN_PD = 2 };

// FFT stages (hs_fft.cu)
hs_status fft_forward(Plan* p, const void* X, cudaStream_t s);           // X -> p->grid
hs_status fft_adjoint(Plan* p, void* X, cudaStream_t s);                 // p->grid -> X

// NUFFT interpolation (hs_nufft.cu)
struct DegridArgs {
    int mode;
    void* out;              // DOUT_CALLER / DOUT_SORTED / DOUT_SORTED_U: destination
    void* v;                // DOUT_PD: dual v (read), sorted
    const void* y;          // DOUT_PD: data, sorted
    void* d;                // DOUT_PD: output d = U^{-1/2} vbar - y, sorted
    double* part;           // DOUT_PD: per-item partial ||d||^2, [blocks][items_max]
    double* rpart;          // DOUT_PD: per-item partial ||y - Phi x~||^2, same layout, or null
};
hs_status degrid(Plan* p, const DegridArgs& a, cudaStream_t s);
int degrid_blocks_x(const Plan* p);   // chunks of DEGRID_CHUNK per channel (l2-ball partials)
int degrid_items_max(const Plan* p);  // partial-sum stride of the PD de-gridding (>= 1)

struct GridArgs {
    int mode;
    const void* in;         // GIN_CALLER / GIN_SORTED: visibilities
    const void* d;          // GIN_PD: d from the de-gridding pass
    const void* scale;      // GIN_PD: per-block real factor max(0, 1 - eps / rho)
    void* v;                // GIN_PD: dual output v (home tile writes), sorted
};
hs_status grid(Plan* p, const GridArgs& a, cudaStream_t s);

// l2-ball helpers (hs_prox.cu)
struct AdaptArgs {          // Algorithm 2 steps 13-19 on the device
    const double* rpart;    // per-item residual partials, [nblk][nparts]
    double* eps;            // bounds (updated in place for the next iteration)
    int64_t* theta;         // iteration of each block's last update
    const int64_t* t;       // completed iterations (this one is t + 1)
    const double* beta;     // beta of the previous iteration
    double* resid;          // out: ||y_b - Phi_b x~||
    double lambda1, lambda2, lambda3;
    int64_t min_gap;
};
hs_status adapt_bounds(int nblk, int nparts, const AdaptArgs& a, cudaStream_t s);
hs_status ball_scale_from_partials(Plan* p, const double* part, int nparts, const double* eps,
                                   double* rho, void* scale_real, cudaStream_t s);

// Wavelets (hs_dwt.cu)
hs_status dwt_analysis(Plan* p, const void* X, void* A, cudaStream_t s);
hs_status dwt_synthesis(Plan* p, const void* A, void* X, cudaStream_t s);

// Proximal operators and PD pieces (hs_prox.cu)
hs_status l21_apply(Plan* p, const void* A, const void* Wadd, const void* w_rows, double thr,
                    int dual, void* out, cudaStream_t s);
hs_status l21_norm(Plan* p, const void* A, const void* w_rows, double* out_dev, cudaStream_t s);
hs_status nuclear_svals(Plan* p, const void* X, double* sv_out, cudaStream_t s);
hs_status reweight_rows(Plan* p, const void* A, double gamma, void* w_out, cudaStream_t s);
hs_status reweight_sv(const double* sv, int L, double gamma, double* w_out, cudaStream_t s);
hs_status reweight_coef(Plan* p, const void* A, double gamma, void* w_out, cudaStream_t s);
hs_status l1_apply(Plan* p, const void* A, const void* Wadd, const void* w, double thr, int dual, void* out,
                   cudaStream_t s);
hs_status nuclear_apply(Plan* p, const void* X, const void* Xadd, const double* w_sv, double thr,
                        int dual, void* out, double* sv_out, float* warm, int* r_out, cudaStream_t s);
// S = Z^T Z of Z = X (+ Xadd) into p->gram (L x L, row-major).
hs_status gram_matrix(Plan* p, const void* X, const void* Xadd, cudaStream_t s);
// Channels per F^H chunk that fit half the L2 (fft_adjoint below).
int fft_adjoint_chunk(const Plan* p);
// Tensor-core Gram matrix of FP32 plans (hs_gram_tc.cu): set-up once per plan
// creation, the conditions it needs (L <= 64, N a multiple of 64, 16-byte
// aligned buffers), and the launch writing per-CTA upper-triangle partials
// part[e * g + b], b < g = *ctas_out <= nparts; a bounded wait that expires
// sets *err.
hs_status gram_tc_init();
bool gram_tc_usable(const void* X, const void* Xa, int L, int64_t N);
hs_status gram_tc_launch(const float* X, const float* Xa, int L, int64_t N, double* part, int nparts, int* err,
                         int* ctas_out, cudaStream_t s);
// FP32 plans: mixed-precision eigendecomposition of the Gram matrix (hs_eig.cu).
// warm: L x L FP32 eigenvectors of the previous call (updated in place) or null.
hs_status eig_mixed_launch(const double* S, int L, const double* w_sv, double thr, int dual,
                           double* Mf, double* sv_out, float* warm, int* r_out, cudaStream_t s);
// FP64 plans: FP64 Jacobi on the whole Gram matrix (hs_eig.cu).
hs_status eig_f64_launch(const double* S, int L, const double* w_sv, double thr, int dual, double* Mf,
                         double* sv_out, int* r_out, cudaStream_t s);
hs_status ball_project(Plan* p, const void* Z, const void* Yd, const double* eps, int dual,
                       void* out, double* rho_out, cudaStream_t s);
hs_status primal_update(Plan* p, int64_t n, const void* P, const void* At, const void* D,
                        double k1, double k2, double k3, double tau, int use_p, int use_a,
                        void* X, void* Xt, double* part, int nparts, cudaStream_t s);
hs_status beta_from_partials(const double* part, int nparts, double* beta, int64_t* t_count, cudaStream_t s);
hs_status channel_norms(Plan* p, const void* X, double* out_dev, cudaStream_t s);
// eta_l = 1 / max(Phi_l^dagger Phi_l delta) into eta (device L); X: L x N scratch.
hs_status psf_inv_peak(Plan* p, void* X, double* eta, cudaStream_t s);
// X[l] *= f[l] (device L doubles).
hs_status mul_channels(Plan* p, void* X, const double* f, cudaStream_t s);
hs_status scale_channels(Plan* p, void* X, const double* norms, cudaStream_t s);

}  // namespace hs
