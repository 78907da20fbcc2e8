// Host-side tables of the HyperSARA library: error strings, Daubechies
// filters, Kaiser-Bessel kernel and its piecewise-polynomial fit.
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <vector>

#include "hs_internal.h"

namespace hs {

static thread_local std::string g_err;

hs_status fail(hs_status st, const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

void clear_error() { g_err.clear(); }

const char* last_error() { return g_err.c_str(); }

// ----------------------------------------------------------------------------
// Daubechies db_p low-pass filter (Daubechies, Ten Lectures on Wavelets, 6.1).
// |m0(w)|^2 = cos^{2p}(w/2) P(sin^2(w/2)) with P(y) = sum_{k<p} C(p-1+k, k) y^k.
// The roots y_r of P are found with the Aberth-Ehrlich simultaneous iteration
// (Aberth 1973) followed by Newton polishing; each y_r gives the reciprocal
// pair z, 1/z of z^2 + (4 y_r - 2) z + 1 = 0 and the root inside the unit
// circle is kept (minimum phase). m0 ~ (1 + z)^p prod (z - z_r), normalised
// to sum sqrt(2); the taps are the coefficients from the highest power down,
// so that db2 = [(1+sqrt3), (3+sqrt3), (3-sqrt3), (1-sqrt3)] / (4 sqrt2).
// ----------------------------------------------------------------------------
using cd = std::complex<double>;

static cd poly_eval(const std::vector<double>& a, cd z) {   // ascending coefficients
    cd r = 0.0;
    for (int k = (int)a.size() - 1; k >= 0; --k) r = r * z + a[k];
    return r;
}

static cd poly_deriv(const std::vector<double>& a, cd z) {
    cd r = 0.0;
    for (int k = (int)a.size() - 1; k >= 1; --k) r = r * z + (double)k * a[k];
    return r;
}

hs_status daubechies_lowpass(int p, double* out) {
    if (p < 1 || p > 8 || out == nullptr)
        return fail(HS_ERR_ARG, "daubechies_lowpass: p must be 1..8 and out non-null");
    std::vector<cd> q{cd(1.0)};   // ascending coefficients of prod (z - z_r)
    if (p > 1) {
        const int n = p - 1;
        std::vector<double> a(p);
        for (int k = 0; k < p; ++k) {
            double c = 1.0;   // C(p-1+k, k)
            for (int i = 1; i <= k; ++i) c = c * (p - 1 + i) / i;
            a[k] = c;
        }
        std::vector<cd> r(n);
        const double R = std::pow(std::fabs(a[0] / a[n]), 1.0 / n);
        for (int i = 0; i < n; ++i) r[i] = std::polar(R, 2.0 * M_PI * i / n + 0.4);
        for (int it = 0; it < 500; ++it) {
            double step = 0.0;
            for (int i = 0; i < n; ++i) {
                cd ratio = poly_eval(a, r[i]) / poly_deriv(a, r[i]);
                cd sum = 0.0;
                for (int j = 0; j < n; ++j)
                    if (j != i) sum += 1.0 / (r[i] - r[j]);
                cd w = ratio / (1.0 - ratio * sum);
                r[i] -= w;
                step = std::max(step, std::abs(w) / std::max(1e-300, std::abs(r[i])));
            }
            if (step < 1e-17) break;
        }
        for (int i = 0; i < n; ++i)
            for (int it = 0; it < 3; ++it) r[i] -= poly_eval(a, r[i]) / poly_deriv(a, r[i]);
        for (int i = 0; i < n; ++i) {
            cd b = 1.0 - 2.0 * r[i];
            cd disc = std::sqrt(b * b - 1.0);
            cd z1 = b + disc, z2 = b - disc;
            cd z = std::abs(z1) < 1.0 ? z1 : z2;
            std::vector<cd> nq(q.size() + 1, cd(0.0));
            for (size_t k = 0; k < q.size(); ++k) {
                nq[k + 1] += q[k];
                nq[k] -= z * q[k];
            }
            q.swap(nq);
        }
    }
    for (int i = 0; i < p; ++i) {   // times (1 + z)^p
        std::vector<cd> nq(q.size() + 1, cd(0.0));
        for (size_t k = 0; k < q.size(); ++k) {
            nq[k] += q[k];
            nq[k + 1] += q[k];
        }
        q.swap(nq);
    }
    double s = 0.0;
    for (auto& c : q) s += c.real();
    const int F = 2 * p;
    for (int j = 0; j < F; ++j) out[j] = q[F - 1 - j].real() * std::sqrt(2.0) / s;
    return HS_OK;
}

// ----------------------------------------------------------------------------
// Kaiser-Bessel kernel phi(x) = I0(beta sqrt(1 - (2x/J)^2)), |x| <= J/2, and
// its continuous Fourier transform J sinh(sqrt(beta^2 - (pi J f)^2)) / sqrt(...)
// (Jackson et al. 1991). I0 by its power series, all terms positive.
// ----------------------------------------------------------------------------
static double bessel_i0(double z) {
    double s = 1.0, term = 1.0;
    const double q = 0.25 * z * z;
    for (int k = 1; k < 500; ++k) {
        term *= q / ((double)k * (double)k);
        s += term;
        if (term < 1e-18 * s) break;
    }
    return s;
}

double kb_phi(double x, int J, double beta) {
    const double h = 0.5 * J;
    if (std::fabs(x) > h) return 0.0;
    const double r = 1.0 - (x / h) * (x / h);
    return bessel_i0(beta * std::sqrt(r > 0.0 ? r : 0.0));
}

double kb_phihat(double f, int J, double beta) {
    const double a = beta * beta - (M_PI * J * f) * (M_PI * J * f);
    if (a > 0.0) {
        const double s = std::sqrt(a);
        return J * std::sinh(s) / s;
    }
    if (a < 0.0) {
        const double s = std::sqrt(-a);
        return J * std::sin(s) / s;
    }
    return (double)J;
}

// Chebyshev interpolation of g(s) = phi(m + (s + 1) / 2) on [-1, 1] at `terms`
// Chebyshev points of the first kind, converted to monomials in s.
double kb_poly_fit(int J, double beta, int terms, std::vector<double>* coef) {
    const int half = J / 2;
    const double peak = kb_phi(0.0, J, beta);
    coef->assign((size_t)J * terms, 0.0);
    double max_err = 0.0;
    std::vector<double> c(terms), tk_prev(terms), tk(terms), tk_next(terms), mono(terms);
    for (int piece = 0; piece < J; ++piece) {
        const int m = piece - half;
        for (int k = 0; k < terms; ++k) {
            double acc = 0.0;
            for (int i = 0; i < terms; ++i) {
                const double th = M_PI * (i + 0.5) / terms;
                const double s = std::cos(th);
                acc += kb_phi(m + 0.5 * (s + 1.0), J, beta) * std::cos(k * th);
            }
            c[k] = acc * 2.0 / terms;
        }
        c[0] *= 0.5;
        std::fill(mono.begin(), mono.end(), 0.0);
        std::fill(tk_prev.begin(), tk_prev.end(), 0.0);
        std::fill(tk.begin(), tk.end(), 0.0);
        tk_prev[0] = 1.0;                // T0
        if (terms > 1) tk[1] = 1.0;      // T1
        for (int k = 0; k < terms; ++k) {
            const std::vector<double>& Tk = (k == 0) ? tk_prev : tk;
            for (int j = 0; j < terms; ++j) mono[j] += c[k] * Tk[j];
            if (k >= 1 && k + 1 < terms) {
                std::fill(tk_next.begin(), tk_next.end(), 0.0);
                for (int j = 0; j + 1 < terms; ++j) tk_next[j + 1] += 2.0 * tk[j];
                for (int j = 0; j < terms; ++j) tk_next[j] -= tk_prev[j];
                tk_prev = tk;
                tk = tk_next;
            }
        }
        for (int j = 0; j < terms; ++j) (*coef)[(size_t)piece * terms + j] = mono[j];
        for (int i = 0; i <= 2000; ++i) {
            const double f = i / 2000.0 * (1.0 - 1e-12);
            const double s = 2.0 * f - 1.0;
            double v = 0.0;
            for (int j = terms - 1; j >= 0; --j) v = v * s + mono[j];
            max_err = std::max(max_err, std::fabs(v - kb_phi(m + f, J, beta)) / peak);
        }
    }
    return max_err;
}

}  // namespace hs
