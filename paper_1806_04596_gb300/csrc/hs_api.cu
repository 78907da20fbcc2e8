// C ABI of the HyperSARA GB300 library: argument checks, plan / state
// lifetime, operator entry points and the primal-dual iteration (Algorithm 2).
#include <cmath>
#include <cstring>
#include <memory>
#include <vector>

#include <algorithm>

#include "hs_internal.h"

namespace hs {
const char* last_error();
hs_status plan_create(Plan** out, int nx, int ny, int L, const int64_t* vis_offsets, int nblocks,
                      const int64_t* block_offsets, const void* uv, const void* weights, const void* precond,
                      int oversample, int J, double kb_beta, int levels, hs_prec prec, unsigned flags,
                      cudaStream_t s);
void plan_free(Plan* p);
}  // namespace hs

using namespace hs;

struct hs_plan {
    Plan* p;
};

// Primal-dual state: variables of Algorithm 2 plus its own scratch, so that a
// state never shares partial-sum buffers between its two concurrent branches.
struct hs_pd_state {
    Plan* p = nullptr;
    hs_pd_params prm{};
    void* X = nullptr;      // L x N reals: primal estimate
    void* Xt = nullptr;     // L x N: extrapolated 2 X - X_prev
    void* P = nullptr;      // L x N: nuclear dual
    void* A = nullptr;      // 9 x L x N: sparsity duals
    void* W = nullptr;      // 9 x L x N: Psi^dagger X~ scratch
    void* At = nullptr;     // L x N: sum_d Psi_d A_d
    void* D = nullptr;      // L x N: Phi^dagger v
    void* v = nullptr;      // M complex (plan order): data duals
    void* y = nullptr;      // M complex (plan order): data
    void* d = nullptr;      // M complex: U^{-1/2} vbar - y
    double* eps = nullptr;  // L
    double* rho = nullptr;  // L
    void* scale = nullptr;  // L reals
    double* beta = nullptr; // 1
    double* ppart = nullptr;   // primal partial sums
    double* dpart = nullptr;   // de-gridding partial sums [L][nbx] (one slot per work item)
    float* warm = nullptr;     // L x L eigenvectors of the previous nuclear step (FP32 plans)
    double* sv = nullptr;      // L singular values of the last nuclear step
    double* sv_rw = nullptr;   // L singular values of X for the re-weighting
    double* rpart = nullptr;   // de-gridding partial ||y - Phi x~||^2 [nblk][nbx] (adaptive bounds)
    int64_t* theta = nullptr;  // nblk: iteration of each block's last bound update
    int64_t* tcnt = nullptr;   // completed iterations (device)
    double* resid = nullptr;   // nblk: ||y_b - Phi_b x~|| of the last iteration (adaptive bounds)
    hs_adapt_params adapt{};   // adaptive bounds, off unless set
    int* nact = nullptr;       // active count of the last nuclear step
    int nprim = 0;
    int nbx = 0;
    int64_t iters = 0;
    cudaStream_t side = nullptr, side2 = nullptr, cap = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_join2 = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    void* ystage = nullptr;   // caller-order y staged from host memory (hs_pd_set_data_host)
    std::vector<void*> allocs;
    std::vector<size_t> alloc_bytes;
};

static cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

#define CHECK_PLAN(pl)                                                         \
    do {                                                                       \
        if ((pl) == nullptr || (pl)->p == nullptr)                             \
            return fail(HS_ERR_ARG, "%s: plan is null", __func__);             \
    } while (0)

extern "C" {

const char* hs_version(void) { return "hypersara-gb300 0.1 (sm_103a)"; }

const char* hs_last_error(void) { return hs::last_error(); }

hs_status hs_daubechies_lowpass(int p, double* out) {
    clear_error();
    return daubechies_lowpass(p, out);
}

hs_status hs_kb_poly_fit(int J, double beta, int terms, double* max_rel_err) {
    clear_error();
    if (J != 8 || terms < 2 || terms > 40 || max_rel_err == nullptr || !(beta > 0))
        return fail(HS_ERR_ARG, "hs_kb_poly_fit: need J = 8, 2 <= terms <= 40, beta > 0");
    std::vector<double> c;
    *max_rel_err = kb_poly_fit(J, beta, terms, &c);
    return HS_OK;
}

hs_status hs_kb_poly_coefs(int J, double beta, int terms, double* coef_out) {
    clear_error();
    if (J != 8 || terms < 2 || terms > 40 || coef_out == nullptr || !(beta > 0))
        return fail(HS_ERR_ARG, "hs_kb_poly_coefs: need J = 8, 2 <= terms <= 40, beta > 0");
    std::vector<double> c;
    kb_poly_fit(J, beta, terms, &c);
    std::copy(c.begin(), c.end(), coef_out);
    return HS_OK;
}

hs_status hs_sweep_lists(int Kx, int Ky, int L, const int64_t* offsets, const int* k0x, const int* k0y, int hmax,
                         int cap, int* items, int64_t* n_items, int* ent, int64_t* n_ent) {
    clear_error();
    if (Kx % hs::GRID_TILE || Ky % 8 || Kx < 2 * hs::GRID_TILE || Ky < 2 * hs::GRID_TILE)
        return fail(HS_ERR_ARG, "hs_sweep_lists: Kx must be a multiple of %d and Ky of 8, both >= %d", hs::GRID_TILE,
                    2 * hs::GRID_TILE);
    if (L < 1 || offsets == nullptr || n_items == nullptr || n_ent == nullptr || offsets[0] != 0)
        return fail(HS_ERR_ARG, "hs_sweep_lists: need L >= 1, offsets from 0 and the count pointers");
    for (int l = 0; l < L; ++l)
        if (offsets[l + 1] < offsets[l]) return fail(HS_ERR_ARG, "hs_sweep_lists: offsets must be nondecreasing");
    const int64_t M = offsets[L];
    if (M >= ((int64_t)1 << 31)) return fail(HS_ERR_ARG, "hs_sweep_lists: too many windows");
    if (M > 0 && (k0x == nullptr || k0y == nullptr)) return fail(HS_ERR_ARG, "hs_sweep_lists: null start cells");
    for (int64_t r = 0; r < M; ++r)
        if (k0x[r] < 0 || k0x[r] >= Kx || k0y[r] < 0 || k0y[r] >= Ky)
            return fail(HS_ERR_ARG, "hs_sweep_lists: start cell %lld outside the grid", (long long)r);
    std::vector<hs::SweepItem> it;
    std::vector<int> en;
    HS_TRY(hs::sweep_lists(Kx, Ky, L, offsets, k0x, k0y, hmax > 0 ? hmax : hs::SWEEP_HMAX,
                           cap > 0 ? cap : hs::SWEEP_CAP, it, en));
    if (items != nullptr && ent != nullptr) {
        if (*n_items < (int64_t)it.size() || *n_ent < (int64_t)en.size())
            return fail(HS_ERR_ARG, "hs_sweep_lists: buffers hold %lld items / %lld entries, need %lld / %lld",
                        (long long)*n_items, (long long)*n_ent, (long long)it.size(), (long long)en.size());
        for (size_t k = 0; k < it.size(); ++k) {
            const hs::SweepItem& q = it[k];
            const int v[6] = {q.l, q.strip, q.row0, q.row1, q.e0, q.e1};
            for (int c = 0; c < 6; ++c) items[6 * k + c] = v[c];
        }
        std::copy(en.begin(), en.end(), ent);
    }
    *n_items = (int64_t)it.size();
    *n_ent = (int64_t)en.size();
    return HS_OK;
}

hs_status hs_plan_create(hs_plan_t* out, int nx, int ny, int L, const int64_t* vis_offsets,
                         const void* uv, const void* weights, const void* precond, int oversample,
                         int J, double kb_beta, int wavelet_levels, hs_prec prec, unsigned flags,
                         void* stream) {
    return hs_plan_create_blocks(out, nx, ny, L, vis_offsets, 0, nullptr, uv, weights, precond, oversample, J,
                                 kb_beta, wavelet_levels, prec, flags, stream);
}

hs_status hs_plan_create_blocks(hs_plan_t* out, int nx, int ny, int L, const int64_t* vis_offsets, int nblocks,
                                const int64_t* block_offsets, const void* uv, const void* weights,
                                const void* precond, int oversample, int J, double kb_beta, int wavelet_levels,
                                hs_prec prec, unsigned flags, void* stream) {
    clear_error();
    if (out == nullptr) return fail(HS_ERR_ARG, "hs_plan_create: out is null");
    *out = nullptr;
    if ((block_offsets == nullptr) != (nblocks == 0))
        return fail(HS_ERR_ARG, "hs_plan_create_blocks: block_offsets and nblocks must be given together");
    Plan* p = nullptr;
    HS_TRY(plan_create(&p, nx, ny, L, vis_offsets, nblocks, block_offsets, uv, weights, precond, oversample, J,
                       kb_beta, wavelet_levels, prec, flags, S(stream)));
    hs_plan* h = new (std::nothrow) hs_plan;
    if (h == nullptr) {
        plan_free(p);
        delete p;
        return fail(HS_ERR_NOMEM, "hs_plan_create: host allocation failed");
    }
    h->p = p;
    *out = h;
    return HS_OK;
}

hs_status hs_plan_destroy(hs_plan_t plan) {
    clear_error();
    if (plan == nullptr) return HS_OK;
    if (plan->p) {
        plan_free(plan->p);
        delete plan->p;
    }
    delete plan;
    return HS_OK;
}

hs_status hs_plan_info(hs_plan_t plan, hs_plan_info_t* info) {
    clear_error();
    CHECK_PLAN(plan);
    if (info == nullptr) return fail(HS_ERR_ARG, "hs_plan_info: info is null");
    const Plan* p = plan->p;
    std::memset(info, 0, sizeof(*info));
    info->nx = p->g.nx;
    info->ny = p->g.ny;
    info->L = p->g.L;
    info->Kx = p->g.Kx;
    info->Ky = p->g.Ky;
    info->levels = p->levels;
    info->prec = (int)p->prec;
    info->flags = (int)p->flags;
    info->total_vis = p->M_total;
    info->grid_tile_entries = p->n_ent;
    info->tile_x = p->g.tx;
    info->tile_y = p->g.ty;
    info->kb_terms = p->kb_terms;
    info->kb_beta = p->beta;
    info->kb_fit_max_err = p->kb_fit_err;
    info->device_bytes = p->device_bytes;
    info->nblocks = p->nblk;
    info->gram_tc = p->prec == HS_F32 ? p->gram_tc : 0;
    info->sweep_hmax = p->sweep_hmax;
    info->sweep_cap = p->sweep_cap;
    info->tuned = p->tuned;
    info->tune_ms = p->tune_ms;
    for (int c = 0; c < 3; ++c) info->tune_grid_ms[c] = p->tune_grid_ms[c];
    for (int c = 0; c < 2; ++c) info->tune_gram_ms[c] = p->tune_gram_ms[c];
    info->fft_adj_chunk = p->fft_adj_chunk;
    for (int c = 0; c < 2; ++c) info->tune_fft_ms[c] = p->tune_fft_ms[c];
    return HS_OK;
}

// Read and clear the plan's device error flag (the stream is synchronised).
static hs_status take_device_error(Plan* p, cudaStream_t s) {
    int err = 0;
    HS_CHECK_CUDA(cudaMemcpyAsync(&err, p->err_d, sizeof(int), cudaMemcpyDeviceToHost, s));
    HS_CHECK_CUDA(cudaStreamSynchronize(s));
    if (err == 0) return HS_OK;
    HS_CHECK_CUDA(cudaMemsetAsync(p->err_d, 0, sizeof(int), s));
    HS_CHECK_CUDA(cudaStreamSynchronize(s));
    if (err & 1) return fail(HS_ERR_TIMEOUT, "a bounded device-side wait expired (tensor-core Gram)");
    return fail(HS_ERR_ARG, "an input magnitude reached 2^60, beyond the tensor-core Gram's range");
}

hs_status hs_set_device_limit(int64_t bytes) {
    clear_error();
    if (bytes < 0) return fail(HS_ERR_ARG, "hs_set_device_limit: bytes must be >= 0");
    set_device_limit(bytes);
    return HS_OK;
}

hs_status hs_device_bytes(int64_t* out) {
    clear_error();
    if (out == nullptr) return fail(HS_ERR_ARG, "hs_device_bytes: out is null");
    *out = device_bytes_held();
    return HS_OK;
}

hs_status hs_plan_check(hs_plan_t plan, void* stream) {
    clear_error();
    CHECK_PLAN(plan);
    return take_device_error(plan->p, S(stream));
}

hs_status hs_phi_fwd(hs_plan_t plan, const void* X, void* Y, void* stream) {
    clear_error();
    CHECK_PLAN(plan);
    Plan* p = plan->p;
    if (X == nullptr || (Y == nullptr && p->M_total > 0))
        return fail(HS_ERR_ARG, "hs_phi_fwd: null buffer");
    if (p->M_total == 0) return HS_OK;
    HS_TRY(fft_forward(p, X, S(stream)));
    DegridArgs a{};
    a.mode = DOUT_CALLER;
    a.out = Y;
    return degrid(p, a, S(stream));
}

hs_status hs_phi_adj(hs_plan_t plan, const void* Y, void* X, void* stream) {
    clear_error();
    CHECK_PLAN(plan);
    Plan* p = plan->p;
    if (X == nullptr || (Y == nullptr && p->M_total > 0))
        return fail(HS_ERR_ARG, "hs_phi_adj: null buffer");
    GridArgs a{};
    a.mode = GIN_CALLER;
    a.in = Y;
    HS_TRY(grid(p, a, S(stream)));
    return fft_adjoint(p, X, S(stream));
}

hs_status hs_psi_fwd(hs_plan_t plan, const void* X, void* A, void* stream) {
    clear_error();
    CHECK_PLAN(plan);
    if (X == nullptr || A == nullptr) return fail(HS_ERR_ARG, "hs_psi_fwd: null buffer");
    if (X == A) return fail(HS_ERR_ARG, "hs_psi_fwd: X and A must not alias");
    return dwt_analysis(plan->p, X, A, S(stream));
}

hs_status hs_psi_adj(hs_plan_t plan, const void* A, void* X, void* stream) {
    clear_error();
    CHECK_PLAN(plan);
    if (X == nullptr || A == nullptr) return fail(HS_ERR_ARG, "hs_psi_adj: null buffer");
    if (X == A) return fail(HS_ERR_ARG, "hs_psi_adj: X and A must not alias");
    return dwt_synthesis(plan->p, A, X, S(stream));
}

hs_status hs_prox_l21(hs_plan_t plan, const void* A, const void* w_rows, double thr, int dual,
                      void* out, void* stream) {
    clear_error();
    CHECK_PLAN(plan);
    if (A == nullptr || out == nullptr) return fail(HS_ERR_ARG, "hs_prox_l21: null buffer");
    if (!(thr >= 0.0) || !std::isfinite(thr)) return fail(HS_ERR_ARG, "hs_prox_l21: thr must be >= 0");
    if (dual != 0 && dual != 1) return fail(HS_ERR_ARG, "hs_prox_l21: dual must be 0 or 1");
    return l21_apply(plan->p, A, nullptr, w_rows, thr, dual, out, S(stream));
}

hs_status hs_l21_grad(hs_plan_t plan, const void* A, const void* w_rows, void* out, void* stream) {
    clear_error();
    CHECK_PLAN(plan);
    if (A == nullptr || out == nullptr) return fail(HS_ERR_ARG, "hs_l21_grad: null buffer");
    return l21_apply(plan->p, A, nullptr, w_rows, 1.0, 2, out, S(stream));
}

hs_status hs_prox_nuclear(hs_plan_t plan, const void* X, const double* w_sv, double thr, int dual,
                          void* out, double* sv_out, void* stream) {
    clear_error();
    CHECK_PLAN(plan);
    if (X == nullptr || out == nullptr) return fail(HS_ERR_ARG, "hs_prox_nuclear: null buffer");
    if (!(thr >= 0.0) || !std::isfinite(thr))
        return fail(HS_ERR_ARG, "hs_prox_nuclear: thr must be >= 0");
    if (dual != 0 && dual != 1) return fail(HS_ERR_ARG, "hs_prox_nuclear: dual must be 0 or 1");
    if (plan->p->g.L > MAX_L_NUC)
        return fail(HS_ERR_ARG, "hs_prox_nuclear: L = %d exceeds %d", plan->p->g.L, MAX_L_NUC);
    return nuclear_apply(plan->p, X, nullptr, w_sv, thr, dual, out, sv_out, nullptr, nullptr,
                         S(stream));
}

hs_status hs_gram(hs_plan_t plan, const void* X, const void* Xadd, int form, double* S_out, void* stream) {
    clear_error();
    CHECK_PLAN(plan);
    if (X == nullptr || S_out == nullptr) return fail(HS_ERR_ARG, "hs_gram: null buffer");
    if (form < 0 || form > 2) return fail(HS_ERR_ARG, "hs_gram: form must be 0, 1 or 2");
    Plan* p = plan->p;
    const int L = p->g.L;
    if (L > MAX_L_NUC) return fail(HS_ERR_ARG, "hs_gram: L = %d exceeds %d", L, MAX_L_NUC);
    cudaStream_t s = S(stream);
    const int keep = p->gram_tc;
    if (form) p->gram_tc = form == 1;
    const hs_status st = gram_matrix(p, X, Xadd, s);
    p->gram_tc = keep;
    HS_TRY(st);
    HS_CHECK_CUDA(cudaMemcpyAsync(S_out, p->gram, (size_t)L * L * sizeof(double), cudaMemcpyDeviceToDevice, s));
    return HS_OK;
}

hs_status hs_proj_l2ball(hs_plan_t plan, const void* Z, const void* Yd, const double* eps, int dual,
                         void* out, double* rho_out, void* stream) {
    clear_error();
    CHECK_PLAN(plan);
    Plan* p = plan->p;
    if (eps == nullptr || ((Z == nullptr || Yd == nullptr || out == nullptr) && p->M_total > 0))
        return fail(HS_ERR_ARG, "hs_proj_l2ball: null buffer");
    if (dual != 0 && dual != 1) return fail(HS_ERR_ARG, "hs_proj_l2ball: dual must be 0 or 1");
    return ball_project(p, Z, Yd, eps, dual, out, rho_out, S(stream));
}

hs_status hs_norm_l21(hs_plan_t plan, const void* A, const void* w_rows, double* out_host,
                      void* stream) {
    clear_error();
    CHECK_PLAN(plan);
    if (A == nullptr || out_host == nullptr) return fail(HS_ERR_ARG, "hs_norm_l21: null buffer");
    Plan* p = plan->p;
    HS_TRY(l21_norm(p, A, w_rows, p->dscal, S(stream)));
    HS_CHECK_CUDA(cudaMemcpyAsync(out_host, p->dscal, sizeof(double), cudaMemcpyDeviceToHost, S(stream)));
    HS_CHECK_CUDA(cudaStreamSynchronize(S(stream)));
    return HS_OK;
}

static hs_status run_stage(Plan* p, int stage, const void* in, void* out, cudaStream_t s) {
    switch (stage) {
        case HS_STAGE_FFT_FWD: return fft_forward(p, in, s);
        case HS_STAGE_DEGRID: {
            DegridArgs a{};
            a.mode = DOUT_CALLER;
            a.out = out;
            return degrid(p, a, s);
        }
        case HS_STAGE_GRID: {
            GridArgs a{};
            a.mode = GIN_CALLER;
            a.in = in;
            return grid(p, a, s);
        }
        case HS_STAGE_FFT_ADJ: return fft_adjoint(p, out, s);
        case HS_STAGE_PSI_FWD: return dwt_analysis(p, in, out, s);
        case HS_STAGE_PSI_ADJ: return dwt_synthesis(p, in, out, s);
        default: return fail(HS_ERR_ARG, "hs_time_stage: unknown stage %d", stage);
    }
}

hs_status hs_time_stage(hs_plan_t plan, int stage, const void* in, void* out, int reps, float* avg_ms,
                        void* stream) {
    clear_error();
    CHECK_PLAN(plan);
    if (avg_ms == nullptr || reps < 1) return fail(HS_ERR_ARG, "hs_time_stage: need avg_ms, reps >= 1");
    const bool needs_in = stage == HS_STAGE_FFT_FWD || stage == HS_STAGE_GRID || stage == HS_STAGE_PSI_FWD ||
                          stage == HS_STAGE_PSI_ADJ;
    const bool needs_out = stage == HS_STAGE_DEGRID || stage == HS_STAGE_FFT_ADJ ||
                           stage == HS_STAGE_PSI_FWD || stage == HS_STAGE_PSI_ADJ;
    if ((needs_in && in == nullptr && plan->p->M_total > 0) || (needs_out && out == nullptr))
        return fail(HS_ERR_ARG, "hs_time_stage: missing buffer for stage %d", stage);
    cudaStream_t s = S(stream);
    Plan* p = plan->p;
    HS_TRY(run_stage(p, stage, in, out, s));   // warm
    cudaEvent_t e0, e1;
    HS_CHECK_CUDA(cudaEventCreate(&e0));
    HS_CHECK_CUDA(cudaEventCreate(&e1));
    hs_status st = HS_OK;
    cudaEventRecord(e0, s);
    for (int i = 0; i < reps && st == HS_OK; ++i) st = run_stage(p, stage, in, out, s);
    cudaEventRecord(e1, s);
    cudaError_t ce = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != HS_OK) return st;
    if (ce != cudaSuccess) return fail(HS_ERR_CUDA, "hs_time_stage: %s", cudaGetErrorString(ce));
    *avg_ms = ms / reps;
    return HS_OK;
}

// splitmix64 followed by Box-Muller: a fixed, documented start vector.
static uint64_t splitmix64(uint64_t& x) {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

hs_status hs_estimate_mu(hs_plan_t plan, const void* Y, void* A_work, double* eta_out, void* Xd_out,
                         double* mu_host, void* stream) {
    clear_error();
    CHECK_PLAN(plan);
    Plan* p = plan->p;
    if (A_work == nullptr || mu_host == nullptr || (Y == nullptr && p->M_total > 0))
        return fail(HS_ERR_ARG, "hs_estimate_mu: null argument");
    const int L = p->g.L;
    if (L > MAX_L_NUC) return fail(HS_ERR_ARG, "hs_estimate_mu: L = %d exceeds %d", L, MAX_L_NUC);
    cudaStream_t s = S(stream);
    double* eta = eta_out ? eta_out : p->dscal + 2 * L;
    HS_TRY(psf_inv_peak(p, p->xbuf, eta, s));
    void* Xd = Xd_out ? Xd_out : p->xbuf2;
    if (p->M_total > 0) {   // dirty cube eta_l Phi_l^dagger y_l
        GridArgs ga{};
        ga.mode = GIN_CALLER;
        ga.in = Y;
        HS_TRY(grid(p, ga, s));
        HS_TRY(fft_adjoint(p, Xd, s));
    } else {
        HS_CHECK_CUDA(cudaMemsetAsync(Xd, 0, (size_t)L * p->N() * p->rsize(), s));
    }
    HS_TRY(mul_channels(p, Xd, eta, s));
    HS_TRY(nuclear_svals(p, Xd, p->sv, s));
    HS_TRY(dwt_analysis(p, Xd, A_work, s));
    HS_TRY(l21_norm(p, A_work, nullptr, p->dscal, s));
    std::vector<double> sv(L);
    double l21 = 0.0;
    HS_CHECK_CUDA(cudaMemcpyAsync(sv.data(), p->sv, L * sizeof(double), cudaMemcpyDeviceToHost, s));
    HS_CHECK_CUDA(cudaMemcpyAsync(&l21, p->dscal, sizeof(double), cudaMemcpyDeviceToHost, s));
    HS_TRY(take_device_error(p, s));
    double nuc = 0.0;
    for (int l = 0; l < L; ++l) nuc += sv[l];
    *mu_host = l21 > 0.0 ? nuc / l21 : 0.0;
    return HS_OK;
}

hs_status hs_op_norm2(hs_plan_t plan, int iters, double tol, uint64_t seed, double* out_host,
                      void* stream) {
    clear_error();
    CHECK_PLAN(plan);
    if (out_host == nullptr || iters < 1 || !(tol >= 0.0))
        return fail(HS_ERR_ARG, "hs_op_norm2: need out_host, iters >= 1, tol >= 0");
    Plan* p = plan->p;
    cudaStream_t s = S(stream);
    const int L = p->g.L;
    const int64_t n = (int64_t)L * p->N();
    std::vector<double> h((size_t)n);
    uint64_t st = seed;
    for (int64_t i = 0; i < n; i += 2) {
        const double u1 = ((splitmix64(st) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        const double u2 = ((splitmix64(st) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        const double r = std::sqrt(-2.0 * std::log(u1));
        h[i] = r * std::cos(2.0 * M_PI * u2);
        if (i + 1 < n) h[i + 1] = r * std::sin(2.0 * M_PI * u2);
    }
    if (p->prec == HS_F32) {
        std::vector<float> f(h.begin(), h.end());
        HS_CHECK_CUDA(cudaMemcpyAsync(p->xbuf, f.data(), n * sizeof(float), cudaMemcpyHostToDevice, s));
        HS_CHECK_CUDA(cudaStreamSynchronize(s));
    } else {
        HS_CHECK_CUDA(cudaMemcpyAsync(p->xbuf, h.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
        HS_CHECK_CUDA(cudaStreamSynchronize(s));
    }
    double* nrm = p->dscal;
    HS_TRY(channel_norms(p, p->xbuf, nrm, s));
    HS_TRY(scale_channels(p, p->xbuf, nrm, s));
    std::vector<double> lam(L, 0.0), prev(L, 0.0);
    for (int it = 0; it < iters; ++it) {
        if (p->M_total > 0) {
            HS_TRY(fft_forward(p, p->xbuf, s));
            DegridArgs da{};
            da.mode = DOUT_SORTED_U;
            da.out = p->vis;
            HS_TRY(degrid(p, da, s));
            GridArgs ga{};
            ga.mode = GIN_SORTED;
            ga.in = p->vis;
            HS_TRY(grid(p, ga, s));
            HS_TRY(fft_adjoint(p, p->xbuf, s));
        } else {
            HS_CHECK_CUDA(cudaMemsetAsync(p->xbuf, 0, n * p->rsize(), s));
        }
        HS_TRY(channel_norms(p, p->xbuf, nrm, s));
        HS_CHECK_CUDA(cudaMemcpyAsync(lam.data(), nrm, sizeof(double) * L, cudaMemcpyDeviceToHost, s));
        HS_CHECK_CUDA(cudaStreamSynchronize(s));
        HS_TRY(scale_channels(p, p->xbuf, nrm, s));
        bool conv = it > 0;
        for (int l = 0; l < L; ++l)
            if (std::fabs(lam[l] - prev[l]) > tol * lam[l]) conv = false;
        prev = lam;
        if (conv) break;
    }
    HS_CHECK_CUDA(cudaStreamSynchronize(s));
    double best = 0.0;
    for (int l = 0; l < L; ++l) best = std::max(best, lam[l]);
    *out_host = best;
    return HS_OK;
}

// ------------------------------------------------------------------ primal-dual state
static hs_status st_alloc(hs_pd_state* st, void** ptr, size_t bytes) {
    *ptr = nullptr;
    if (bytes == 0) bytes = 16;
    HS_TRY(lib_alloc(ptr, bytes));
    st->allocs.push_back(*ptr);
    st->alloc_bytes.push_back(bytes);
    return HS_OK;
}

static void st_free(hs_pd_state* st) {
    if (st->gexec) cudaGraphExecDestroy(st->gexec);
    if (st->graph) cudaGraphDestroy(st->graph);
    if (st->ev_fork) cudaEventDestroy(st->ev_fork);
    if (st->ev_join) cudaEventDestroy(st->ev_join);
    if (st->ev_join2) cudaEventDestroy(st->ev_join2);
    if (st->side) cudaStreamDestroy(st->side);
    if (st->side2) cudaStreamDestroy(st->side2);
    if (st->cap) cudaStreamDestroy(st->cap);
    for (size_t k = 0; k < st->allocs.size(); ++k) lib_free(st->allocs[k], st->alloc_bytes[k]);
    st->allocs.clear();
    st->alloc_bytes.clear();
}

__global__ void k_gather_c2(const float2* __restrict__ in, const int* __restrict__ perm,
                            float2* __restrict__ out, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[perm[i]];
}
__global__ void k_gather_z2(const double2* __restrict__ in, const int* __restrict__ perm,
                            double2* __restrict__ out, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[perm[i]];
}

hs_status hs_pd_state_create(hs_plan_t plan, const void* Y, const double* eps,
                             const hs_pd_params* prm, hs_pd_state_t* out, void* stream) {
    clear_error();
    CHECK_PLAN(plan);
    if (out == nullptr || prm == nullptr || eps == nullptr || (Y == nullptr && plan->p->M_total > 0))
        return fail(HS_ERR_ARG, "hs_pd_state_create: null argument");
    *out = nullptr;
    if (!(prm->tau > 0.0) || !std::isfinite(prm->kappa1) || !std::isfinite(prm->kappa2) ||
        !std::isfinite(prm->kappa3) || !(prm->mu >= 0.0) || !(prm->psi_norm2 > 0.0))
        return fail(HS_ERR_ARG, "hs_pd_state_create: invalid parameters");
    Plan* p = plan->p;
    if (prm->sparsity != 0 && prm->sparsity != 1)
        return fail(HS_ERR_ARG, "hs_pd_state_create: sparsity must be 0 (l2,1) or 1 (l1)");
    if (prm->use_nuclear && p->g.L > MAX_L_NUC)
        return fail(HS_ERR_ARG, "hs_pd_state_create: nuclear prior needs L <= %d", MAX_L_NUC);
    cudaStream_t s = S(stream);
    std::unique_ptr<hs_pd_state> st(new hs_pd_state());
    st->p = p;
    st->prm = *prm;
    const int L = p->g.L;
    const int64_t N = p->N();
    const size_t rs = p->rsize(), cs = p->csize();
    const int64_t M = p->M_total;
    hs_status e = HS_OK;
#define ALLOC(ptr, bytes)                                   \
    do {                                                    \
        e = st_alloc(st.get(), (void**)&(ptr), (bytes));    \
        if (e != HS_OK) {                                   \
            st_free(st.get());                              \
            return e;                                       \
        }                                                   \
    } while (0)
    ALLOC(st->X, L * N * rs);
    ALLOC(st->Xt, L * N * rs);
    ALLOC(st->P, L * N * rs);
    ALLOC(st->A, NB * L * N * rs);
    ALLOC(st->W, NB * L * N * rs);
    ALLOC(st->At, L * N * rs);
    ALLOC(st->D, L * N * rs);
    ALLOC(st->v, M * cs);
    ALLOC(st->y, M * cs);
    ALLOC(st->d, M * cs);
    const int nb = p->nblk;   // data blocks (one per channel unless the plan has blocks)
    ALLOC(st->eps, nb * sizeof(double));
    ALLOC(st->rho, nb * sizeof(double));
    ALLOC(st->scale, nb * rs);
    ALLOC(st->theta, nb * sizeof(int64_t));
    ALLOC(st->resid, nb * sizeof(double));
    ALLOC(st->tcnt, sizeof(int64_t));
    ALLOC(st->beta, sizeof(double));
    st->nprim = 1024;
    ALLOC(st->ppart, 2 * st->nprim * sizeof(double));
    st->nbx = degrid_items_max(p);   // slots block * nbx + k; slots without a work item stay 0
    ALLOC(st->dpart, (size_t)nb * st->nbx * sizeof(double));
    ALLOC(st->rpart, (size_t)nb * st->nbx * sizeof(double));
    ALLOC(st->warm, (size_t)MAX_L_NUC * MAX_L_NUC * sizeof(float));
    ALLOC(st->sv, (size_t)std::max(L, 1) * sizeof(double));
    ALLOC(st->sv_rw, (size_t)std::max(L, 1) * sizeof(double));
    ALLOC(st->nact, sizeof(int));
#undef ALLOC
    auto cu = [&](cudaError_t ce, const char* what) -> hs_status {
        if (ce == cudaSuccess) return HS_OK;
        st_free(st.get());
        return fail(HS_ERR_CUDA, "hs_pd_state_create: %s: %s", what, cudaGetErrorString(ce));
    };
    HS_TRY(cu(cudaMemsetAsync(st->X, 0, L * N * rs, s), "memset"));
    HS_TRY(cu(cudaMemsetAsync(st->Xt, 0, L * N * rs, s), "memset"));
    HS_TRY(cu(cudaMemsetAsync(st->P, 0, L * N * rs, s), "memset"));
    HS_TRY(cu(cudaMemsetAsync(st->A, 0, NB * L * N * rs, s), "memset"));
    HS_TRY(cu(cudaMemsetAsync(st->At, 0, L * N * rs, s), "memset"));
    HS_TRY(cu(cudaMemsetAsync(st->v, 0, std::max<int64_t>(M, 1) * cs, s), "memset"));
    HS_TRY(cu(cudaMemsetAsync(st->rho, 0, nb * sizeof(double), s), "memset"));
    HS_TRY(cu(cudaMemsetAsync(st->sv, 0, L * sizeof(double), s), "memset"));
    HS_TRY(cu(cudaMemsetAsync(st->nact, 0, sizeof(int), s), "memset"));
    HS_TRY(cu(cudaMemsetAsync(st->dpart, 0, (size_t)nb * st->nbx * sizeof(double), s), "memset"));
    HS_TRY(cu(cudaMemsetAsync(st->rpart, 0, (size_t)nb * st->nbx * sizeof(double), s), "memset"));
    HS_TRY(cu(cudaMemsetAsync(st->theta, 0, nb * sizeof(int64_t), s), "memset"));
    HS_TRY(cu(cudaMemsetAsync(st->resid, 0, nb * sizeof(double), s), "memset"));
    HS_TRY(cu(cudaMemsetAsync(st->tcnt, 0, sizeof(int64_t), s), "memset"));
    {   // beta^{(0)} undefined: +inf, so the first iteration never adjusts a bound
        static const double inf = INFINITY;
        HS_TRY(cu(cudaMemcpyAsync(st->beta, &inf, sizeof(double), cudaMemcpyHostToDevice, s), "beta"));
        HS_TRY(cu(cudaStreamSynchronize(s), "beta"));
    }
    HS_TRY(cu(cudaMemcpyAsync(st->eps, eps, nb * sizeof(double), cudaMemcpyDeviceToDevice, s), "eps"));
    if (L <= MAX_L_NUC) {   // warm start of the eigensolver: identity
        std::vector<float> eye((size_t)L * L, 0.f);
        for (int i = 0; i < L; ++i) eye[(size_t)i * L + i] = 1.f;
        HS_TRY(cu(cudaMemcpyAsync(st->warm, eye.data(), eye.size() * sizeof(float),
                                  cudaMemcpyHostToDevice, s), "warm"));
        HS_TRY(cu(cudaStreamSynchronize(s), "sync"));
    }
    if (M > 0) {
        const unsigned g = (unsigned)std::min<int64_t>((M + 255) / 256, 8192);
        if (p->prec == HS_F32) k_gather_c2<<<g, 256, 0, s>>>((const float2*)Y, p->perm, (float2*)st->y, M);
        else k_gather_z2<<<g, 256, 0, s>>>((const double2*)Y, p->perm, (double2*)st->y, M);
        HS_TRY(cu(cudaGetLastError(), "gather"));
    }
    HS_TRY(cu(cudaStreamCreateWithFlags(&st->side, cudaStreamNonBlocking), "stream"));
    HS_TRY(cu(cudaStreamCreateWithFlags(&st->side2, cudaStreamNonBlocking), "stream"));
    HS_TRY(cu(cudaEventCreateWithFlags(&st->ev_join2, cudaEventDisableTiming), "event"));
    HS_TRY(cu(cudaStreamCreateWithFlags(&st->cap, cudaStreamNonBlocking), "stream"));
    HS_TRY(cu(cudaEventCreateWithFlags(&st->ev_fork, cudaEventDisableTiming), "event"));
    HS_TRY(cu(cudaEventCreateWithFlags(&st->ev_join, cudaEventDisableTiming), "event"));
    HS_TRY(cu(cudaStreamSynchronize(s), "sync"));
    *out = st.release();
    return HS_OK;
}

hs_status hs_pd_set_data(hs_pd_state_t st, const void* Y, const double* eps, void* stream) {
    clear_error();
    if (st == nullptr || eps == nullptr || (Y == nullptr && st->p->M_total > 0))
        return fail(HS_ERR_ARG, "hs_pd_set_data: null argument");
    Plan* p = st->p;
    cudaStream_t s = S(stream);
    const int64_t M = p->M_total;
    HS_CHECK_CUDA(cudaMemcpyAsync(st->eps, eps, p->nblk * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (M > 0) {
        const unsigned g = (unsigned)std::min<int64_t>((M + 255) / 256, 8192);
        if (p->prec == HS_F32) k_gather_c2<<<g, 256, 0, s>>>((const float2*)Y, p->perm, (float2*)st->y, M);
        else k_gather_z2<<<g, 256, 0, s>>>((const double2*)Y, p->perm, (double2*)st->y, M);
        HS_CHECK_LAUNCH();
    }
    return HS_OK;
}

hs_status hs_pd_set_data_host(hs_pd_state_t st, const void* Y_host, const double* eps_host, void* stream) {
    clear_error();
    if (st == nullptr || eps_host == nullptr || (Y_host == nullptr && st->p->M_total > 0))
        return fail(HS_ERR_ARG, "hs_pd_set_data_host: null argument");
    Plan* p = st->p;
    cudaStream_t s = S(stream);
    const int64_t M = p->M_total;
    if (M > 0 && st->ystage == nullptr) HS_TRY(st_alloc(st, &st->ystage, (size_t)M * p->csize()));
    HS_CHECK_CUDA(cudaMemcpyAsync(st->eps, eps_host, p->nblk * sizeof(double), cudaMemcpyHostToDevice, s));
    if (M > 0) {
        HS_CHECK_CUDA(cudaMemcpyAsync(st->ystage, Y_host, (size_t)M * p->csize(), cudaMemcpyHostToDevice, s));
        const unsigned g = (unsigned)std::min<int64_t>((M + 255) / 256, 8192);
        if (p->prec == HS_F32) k_gather_c2<<<g, 256, 0, s>>>((const float2*)st->ystage, p->perm, (float2*)st->y, M);
        else k_gather_z2<<<g, 256, 0, s>>>((const double2*)st->ystage, p->perm, (double2*)st->y, M);
        HS_CHECK_LAUNCH();
    }
    return HS_OK;
}

hs_status hs_pd_get_host(hs_pd_state_t st, void* X_host, double* beta_host, double* rho_host, void* stream) {
    clear_error();
    if (st == nullptr || X_host == nullptr) return fail(HS_ERR_ARG, "hs_pd_get_host: null argument");
    cudaStream_t s = S(stream);
    Plan* p = st->p;
    HS_CHECK_CUDA(cudaMemcpyAsync(X_host, st->X, (size_t)p->g.L * p->N() * p->rsize(), cudaMemcpyDeviceToHost, s));
    if (beta_host) HS_CHECK_CUDA(cudaMemcpyAsync(beta_host, st->beta, sizeof(double), cudaMemcpyDeviceToHost, s));
    if (rho_host)
        HS_CHECK_CUDA(cudaMemcpyAsync(rho_host, st->rho, sizeof(double) * p->nblk, cudaMemcpyDeviceToHost, s));
    return take_device_error(p, s);
}

hs_status hs_pd_state_destroy(hs_pd_state_t st) {
    clear_error();
    if (st == nullptr) return HS_OK;
    st_free(st);
    delete st;
    return HS_OK;
}

// One iteration of Algorithm 2 on stream s. The two prior branches (step 5;
// steps 7-8) run on the state's two side streams, forked and joined with
// events, so they overlap each other and the data-fidelity branch (steps 4,
// 10-12 and Phi^dagger of step 20). They use disjoint scratch: the nuclear
// branch the Gram buffers, the sparsity branch the wavelet buffers.
static hs_status pd_step_launch(hs_pd_state* st, cudaStream_t s) {
    Plan* p = st->p;
    const hs_pd_params& q = st->prm;
    const int64_t n = (int64_t)p->g.L * p->N();
    HS_CHECK_CUDA(cudaEventRecord(st->ev_fork, s));
    HS_CHECK_CUDA(cudaStreamWaitEvent(st->side, st->ev_fork, 0));
    HS_CHECK_CUDA(cudaStreamWaitEvent(st->side2, st->ev_fork, 0));
    // ---- priors (side stream)
    if (q.use_nuclear)   // step 5: P = (I - S*_w)(P + X~), threshold w / kappa1
        HS_TRY(nuclear_apply(p, st->P, st->Xt, q.w_nuc, 1.0 / q.kappa1, 1, st->P, st->sv, st->warm,
                             st->nact, st->side));
    HS_CHECK_CUDA(cudaEventRecord(st->ev_join, st->side));
    if (q.use_l21) {     // steps 7-8
        HS_TRY(dwt_analysis(p, st->Xt, st->W, st->side2));
        // A_d = (I - S^{l21}_{w mu ||Psi||^2})(A_d + Psi_d^dagger X~)
        if (q.sparsity == 1)   // SARA: per-coefficient l1 dual
            HS_TRY(l1_apply(p, st->A, st->W, q.w_l21, q.mu * q.psi_norm2, 1, st->A, st->side2));
        else
            HS_TRY(l21_apply(p, st->A, st->W, q.w_l21, q.mu * q.psi_norm2, 1, st->A, st->side2));
        HS_TRY(dwt_synthesis(p, st->A, st->At, st->side2));
    }
    HS_CHECK_CUDA(cudaEventRecord(st->ev_join2, st->side2));
    // ---- data fidelity (main stream)
    if (p->M_total > 0) {
        HS_TRY(fft_forward(p, st->Xt, s));                        // step 4
        DegridArgs da{};
        da.mode = DOUT_PD;
        da.v = st->v;
        da.y = st->y;
        da.d = st->d;
        da.part = st->dpart;
        da.rpart = st->adapt.enable ? st->rpart : nullptr;
        HS_TRY(degrid(p, da, s));                                  // step 10 (+ residual norms)
        HS_TRY(ball_scale_from_partials(p, st->dpart, st->nbx, st->eps, st->rho, st->scale, s));
        if (st->adapt.enable) {   // steps 13-19: bounds for the next iteration
            AdaptArgs aa{};
            aa.rpart = st->rpart;
            aa.eps = st->eps;
            aa.theta = st->theta;
            aa.t = st->tcnt;
            aa.beta = st->beta;
            aa.resid = st->resid;
            aa.lambda1 = st->adapt.lambda1;
            aa.lambda2 = st->adapt.lambda2;
            aa.lambda3 = st->adapt.lambda3;
            aa.min_gap = st->adapt.min_gap;
            HS_TRY(adapt_bounds(p->nblk, st->nbx, aa, s));
        }
        GridArgs ga{};
        ga.mode = GIN_PD;
        ga.d = st->d;
        ga.scale = st->scale;
        ga.v = st->v;
        HS_TRY(grid(p, ga, s));                                    // steps 11-12
        HS_TRY(fft_adjoint(p, st->D, s));                          // Z^T F^H of step 20
    } else {
        HS_CHECK_CUDA(cudaMemsetAsync(st->D, 0, n * p->rsize(), s));
    }
    HS_CHECK_CUDA(cudaStreamWaitEvent(s, st->ev_join, 0));
    HS_CHECK_CUDA(cudaStreamWaitEvent(s, st->ev_join2, 0));
    // ---- steps 20-23
    HS_TRY(primal_update(p, n, st->P, st->At, st->D, q.kappa1, q.kappa2, q.kappa3, q.tau,
                         q.use_nuclear, q.use_l21, st->X, st->Xt, st->ppart, st->nprim, s));
    HS_TRY(beta_from_partials(st->ppart, st->nprim, st->beta, st->tcnt, s));
    return HS_OK;
}

hs_status hs_pd_step(hs_pd_state_t st, void* stream) {
    clear_error();
    if (st == nullptr) return fail(HS_ERR_ARG, "hs_pd_step: state is null");
    HS_TRY(pd_step_launch(st, S(stream)));
    st->iters += 1;
    return HS_OK;
}

hs_status hs_pd_solve(hs_pd_state_t st, int iters, int graph, void* stream) {
    clear_error();
    if (st == nullptr) return fail(HS_ERR_ARG, "hs_pd_solve: state is null");
    if (iters < 0 || (graph != 0 && graph != 1)) return fail(HS_ERR_ARG, "hs_pd_solve: bad arguments");
    cudaStream_t s = S(stream);
    if (!graph) {
        for (int i = 0; i < iters; ++i) {
            HS_TRY(pd_step_launch(st, s));
            st->iters += 1;
        }
        return HS_OK;
    }
    if (st->gexec == nullptr) {
        // capture one iteration on the state's own stream (the caller's stream may be the
        // legacy default stream, which cannot be captured)
        HS_CHECK_CUDA(cudaStreamBeginCapture(st->cap, cudaStreamCaptureModeThreadLocal));
        hs_status e = pd_step_launch(st, st->cap);
        cudaGraph_t g = nullptr;
        cudaError_t ce = cudaStreamEndCapture(st->cap, &g);
        if (e != HS_OK) {
            if (g) cudaGraphDestroy(g);
            return e;
        }
        if (ce != cudaSuccess) return fail(HS_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(ce));
        st->graph = g;
        HS_CHECK_CUDA(cudaGraphInstantiate(&st->gexec, g, 0));
    }
    for (int i = 0; i < iters; ++i) {
        HS_CHECK_CUDA(cudaGraphLaunch(st->gexec, s));
        st->iters += 1;
    }
    return HS_OK;
}

hs_status hs_pd_get(hs_pd_state_t st, void* X, double* beta_host, double* rho_host, void* stream) {
    clear_error();
    if (st == nullptr) return fail(HS_ERR_ARG, "hs_pd_get: state is null");
    cudaStream_t s = S(stream);
    Plan* p = st->p;
    if (X) HS_CHECK_CUDA(cudaMemcpyAsync(X, st->X, (size_t)p->g.L * p->N() * p->rsize(),
                                         cudaMemcpyDeviceToDevice, s));
    if (beta_host) HS_CHECK_CUDA(cudaMemcpyAsync(beta_host, st->beta, sizeof(double), cudaMemcpyDeviceToHost, s));
    if (rho_host) HS_CHECK_CUDA(cudaMemcpyAsync(rho_host, st->rho, sizeof(double) * p->nblk,
                                                cudaMemcpyDeviceToHost, s));
    if (beta_host || rho_host) return take_device_error(p, s);
    return HS_OK;
}

hs_status hs_pd_graph_kernels(hs_pd_state_t st, int* out) {
    clear_error();
    if (st == nullptr || out == nullptr) return fail(HS_ERR_ARG, "hs_pd_graph_kernels: null argument");
    *out = 0;
    if (st->graph == nullptr) return HS_OK;
    size_t n = 0;
    HS_CHECK_CUDA(cudaGraphGetNodes(st->graph, nullptr, &n));
    std::vector<cudaGraphNode_t> nodes(n);
    HS_CHECK_CUDA(cudaGraphGetNodes(st->graph, nodes.data(), &n));
    int k = 0;
    for (size_t i = 0; i < n; ++i) {
        cudaGraphNodeType t;
        HS_CHECK_CUDA(cudaGraphNodeGetType(nodes[i], &t));
        if (t == cudaGraphNodeTypeKernel) ++k;
    }
    *out = k;
    return HS_OK;
}

hs_status hs_pd_nuclear_info(hs_pd_state_t st, double* sv_host, int* active_host, void* stream) {
    clear_error();
    if (st == nullptr) return fail(HS_ERR_ARG, "hs_pd_nuclear_info: state is null");
    cudaStream_t s = S(stream);
    if (sv_host)
        HS_CHECK_CUDA(cudaMemcpyAsync(sv_host, st->sv, sizeof(double) * st->p->g.L,
                                      cudaMemcpyDeviceToHost, s));
    if (active_host)
        HS_CHECK_CUDA(cudaMemcpyAsync(active_host, st->nact, sizeof(int), cudaMemcpyDeviceToHost, s));
    HS_CHECK_CUDA(cudaStreamSynchronize(s));
    return HS_OK;
}

hs_status hs_pd_reweight(hs_pd_state_t st, double gamma_l21, double gamma_nuc, void* w_l21, double* w_nuc,
                         double* sv_out, void* stream) {
    clear_error();
    if (st == nullptr) return fail(HS_ERR_ARG, "hs_pd_reweight: state is null");
    if (w_l21 == nullptr && w_nuc == nullptr && sv_out == nullptr)
        return fail(HS_ERR_ARG, "hs_pd_reweight: no output requested");
    if (w_l21 && !(gamma_l21 > 0.0 && std::isfinite(gamma_l21)))
        return fail(HS_ERR_ARG, "hs_pd_reweight: gamma_l21 must be finite and > 0");
    if (w_nuc && !(gamma_nuc > 0.0 && std::isfinite(gamma_nuc)))
        return fail(HS_ERR_ARG, "hs_pd_reweight: gamma_nuc must be finite and > 0");
    Plan* p = st->p;
    if ((w_nuc || sv_out) && p->g.L > MAX_L_NUC)
        return fail(HS_ERR_ARG, "hs_pd_reweight: nuclear weights need L <= %d", MAX_L_NUC);
    cudaStream_t s = S(stream);
    if (w_l21) {   // Eq. "weights-l21" from Psi^dagger X (the state's analysis scratch)
        HS_TRY(dwt_analysis(p, st->X, st->W, s));
        if (st->prm.sparsity == 1) HS_TRY(reweight_coef(p, st->W, gamma_l21, w_l21, s));
        else HS_TRY(reweight_rows(p, st->W, gamma_l21, w_l21, s));
    }
    if (w_nuc || sv_out) {   // Eq. "weights-n" from the singular values of X
        double* sv = sv_out ? sv_out : st->sv_rw;
        HS_TRY(nuclear_svals(p, st->X, sv, s));
        if (w_nuc) HS_TRY(reweight_sv(sv, p->g.L, gamma_nuc, w_nuc, s));
    }
    return HS_OK;
}

hs_status hs_pd_set_adaptive(hs_pd_state_t st, const hs_adapt_params* a) {
    clear_error();
    if (st == nullptr) return fail(HS_ERR_ARG, "hs_pd_set_adaptive: state is null");
    hs_adapt_params q{};
    if (a != nullptr && a->enable) {
        if (!(a->lambda1 >= 0.0) || !(a->lambda2 >= 0.0) || !(a->lambda3 > 0.0 && a->lambda3 <= 1.0) ||
            a->min_gap < 0)
            return fail(HS_ERR_ARG, "hs_pd_set_adaptive: need lambda1, lambda2 >= 0, 0 < lambda3 <= 1, min_gap >= 0");
        q = *a;
    }
    st->adapt = q;
    if (st->gexec) {   // the captured iteration changes: capture again at the next graph solve
        cudaGraphExecDestroy(st->gexec);
        st->gexec = nullptr;
    }
    if (st->graph) {
        cudaGraphDestroy(st->graph);
        st->graph = nullptr;
    }
    return HS_OK;
}

hs_status hs_pd_bounds(hs_pd_state_t st, double* eps_host, double* resid_host, int64_t* theta_host, void* stream) {
    clear_error();
    if (st == nullptr) return fail(HS_ERR_ARG, "hs_pd_bounds: state is null");
    cudaStream_t s = S(stream);
    const int nb = st->p->nblk;
    if (eps_host) HS_CHECK_CUDA(cudaMemcpyAsync(eps_host, st->eps, nb * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (resid_host)
        HS_CHECK_CUDA(cudaMemcpyAsync(resid_host, st->resid, nb * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (theta_host)
        HS_CHECK_CUDA(cudaMemcpyAsync(theta_host, st->theta, nb * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    HS_CHECK_CUDA(cudaStreamSynchronize(s));
    return HS_OK;
}

hs_status hs_pd_iterations(hs_pd_state_t st, int64_t* out) {
    clear_error();
    if (st == nullptr || out == nullptr) return fail(HS_ERR_ARG, "hs_pd_iterations: null argument");
    *out = st->iters;
    return HS_OK;
}

}  // extern "C"
