// Host planner for PSWF fast Ewald summation.
//
//  * Prolate: psi_0^c from its even Legendre expansion (App. B).  The ODE
//    (eq. ode) becomes a symmetric tridiagonal eigenproblem in the orthonormal
//    basis sqrt(k+1/2) P_k; the smallest eigenvalue chi_0 is located by Sturm
//    bisection and the coefficients by inverse iteration (App. B, "Computation
//    of eigenpairs").  lambda_0 = (1/psi(0)) int psi by Gauss-Legendre quadrature.
//  * Alg. 3 (Sec. 6.4) with Lambert W by Halley iteration.
//  * Piecewise window polynomials (Remark on Horner evaluation, Sec. 4.3) and
//    radial polynomials for the residual kernel R (eq. R, eq. Phi_cs).
//  * Diagonal scaling tables for Alg. 2 step 3.
#include "planner.h"

#include <algorithm>
#include <cmath>
#include <stdexcept>

namespace pswf {

namespace {

constexpr double kPi = 3.14159265358979323846;

// ---------------------------------------------------------- double-double ----
// Unevaluated sums hi + lo of two doubles (about 32 significant digits) from plain IEEE double
// operations: Knuth's error-free two-sum, the fma residual of a product, and one Newton correction
// for quotients and square roots.  The same operations give the same bits on every IEEE-754 host,
// unlike long double (80-bit on x86-64, 128-bit software arithmetic on AArch64).
struct DD {
    double hi = 0, lo = 0;
};

inline DD two_sum(double a, double b) {
    const double s = a + b, bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
inline DD fast_two_sum(double a, double b) {   // |a| >= |b| (or a == 0)
    const double s = a + b;
    return {s, b - (s - a)};
}
inline DD dd(double a) { return {a, 0.0}; }
inline DD operator+(DD a, DD b) {
    DD s = two_sum(a.hi, b.hi);
    const DD t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return fast_two_sum(s.hi, s.lo);
}
inline DD operator-(DD a) { return {-a.hi, -a.lo}; }
inline DD operator-(DD a, DD b) { return a + (-b); }
inline DD operator*(DD a, DD b) {
    const double p = a.hi * b.hi;
    double e = std::fma(a.hi, b.hi, -p);
    e += a.hi * b.lo + a.lo * b.hi;
    return fast_two_sum(p, e);
}
inline DD operator*(DD a, double b) {
    const double p = a.hi * b;
    double e = std::fma(a.hi, b, -p);
    e += a.lo * b;
    return fast_two_sum(p, e);
}
inline DD operator/(DD a, double b) {
    const double q1 = a.hi / b;
    const double p = q1 * b, pe = std::fma(q1, b, -p);   // q1 b = p + pe exactly
    DD r = two_sum(a.hi, -p);
    r.lo += a.lo - pe;
    return fast_two_sum(q1, (r.hi + r.lo) / b);
}
inline DD operator/(DD a, DD b) {
    const double q1 = a.hi / b.hi;
    const DD r = a - b * q1;
    const double q2 = r.hi / b.hi;
    const DD r2 = r - b * q2;
    return fast_two_sum(q1, q2) + dd(r2.hi / b.hi);
}
inline DD dd_sqrt(DD a) {   // a >= 0
    if (!(a.hi > 0)) return dd(0.0);
    const double x = std::sqrt(a.hi);
    const DD r = a - DD{x * x, std::fma(x, x, -x * x)};
    return fast_two_sum(x, (r.hi + r.lo) / (2.0 * x));
}
inline double to_double(DD a) { return a.hi + a.lo; }

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_N.
void gauss_legendre(int N, std::vector<double>& x, std::vector<double>& w) {
    x.assign(N, 0.0);
    w.assign(N, 0.0);
    for (int i = 0; i < (N + 1) / 2; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (N + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= N; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            // p1 = P_N(z), p0 = P_{N-1}(z)
            dp = N * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = -z;
        x[N - 1 - i] = z;
        double wt = 2.0 / ((1.0 - z * z) * dp * dp);
        w[i] = wt;
        w[N - 1 - i] = wt;
    }
}

// Number of eigenvalues of the symmetric tridiagonal (d, e) below sigma.
int sturm_count(const std::vector<double>& d, const std::vector<double>& e, double sigma) {
    int cnt = 0;
    double q = d[0] - sigma;
    if (q < 0) ++cnt;
    for (size_t i = 1; i < d.size(); ++i) {
        if (q == 0.0) q = 1e-300;
        q = d[i] - sigma - e[i - 1] * e[i - 1] / q;
        if (q < 0) ++cnt;
    }
    return cnt;
}

// Solve (T) y = b for a general tridiagonal T (sub, diag, super) with partial pivoting.
void tridiag_solve(std::vector<double> sub, std::vector<double> diag, std::vector<double> sup,
                   std::vector<double>& b) {
    const int n = static_cast<int>(diag.size());
    std::vector<double> sup2(n, 0.0);
    for (int i = 0; i < n - 1; ++i) {
        if (std::fabs(diag[i]) >= std::fabs(sub[i])) {
            if (diag[i] == 0.0) diag[i] = 1e-300;
            double f = sub[i] / diag[i];
            diag[i + 1] -= f * sup[i];
            b[i + 1] -= f * b[i];
        } else {
            // swap rows i and i+1
            double f = diag[i] / sub[i];
            diag[i] = sub[i];
            double t = diag[i + 1];
            diag[i + 1] = sup[i] - f * t;
            if (i < n - 2) {
                sup2[i] = sup[i + 1];
                sup[i + 1] = -f * sup2[i];
            }
            sup[i] = t;
            double tb = b[i];
            b[i] = b[i + 1];
            b[i + 1] = tb - f * b[i + 1];
        }
    }
    if (diag[n - 1] == 0.0) diag[n - 1] = 1e-300;
    b[n - 1] /= diag[n - 1];
    if (n > 1) b[n - 2] = (b[n - 2] - sup[n - 2] * b[n - 1]) / diag[n - 2];
    for (int i = n - 3; i >= 0; --i) b[i] = (b[i] - sup[i] * b[i + 1] - sup2[i] * b[i + 2]) / diag[i];
}

}  // namespace

double horner(const double* c, int deg, double x) {
    double r = c[deg];
    for (int k = deg - 1; k >= 0; --k) r = r * x + c[k];
    return r;
}

// ---------------------------------------------------------------- Prolate ----
Prolate::Prolate(double cc) : c(cc) {
    if (!(c > 0)) throw std::invalid_argument("PSWF bandlimit must be positive");
    const int K = static_cast<int>(std::ceil(1.2 * c)) + 24;   // App. B: K ~ 1.2 c, plus margin
    std::vector<double> d(K), e(K - 1);
    for (int i = 0; i < K; ++i) {
        const double k = 2.0 * i;
        d[i] = k * (k + 1) + c * c * (2 * k * (k + 1) - 1) / ((2 * k + 3) * (2 * k - 1));
        if (i < K - 1) e[i] = c * c * (k + 1) * (k + 2) / ((2 * k + 3) * std::sqrt((2 * k + 1) * (2 * k + 5)));
    }
    // Sturm bisection for the smallest eigenvalue (Gershgorin lower bound, Rayleigh upper bound)
    double lo = d[0] - std::fabs(e[0]);
    for (int i = 1; i < K; ++i)
        lo = std::min(lo, d[i] - std::fabs(e[i - 1]) - (i < K - 1 ? std::fabs(e[i]) : 0.0));
    double hi = d[0] + 1e-9 * (1.0 + std::fabs(d[0]));
    for (int it = 0; it < 200 && hi - lo > 4e-16 * std::max(1.0, std::fabs(hi)); ++it) {
        double mid = 0.5 * (lo + hi);
        if (sturm_count(d, e, mid) >= 1) hi = mid; else lo = mid;
    }
    chi = 0.5 * (lo + hi);
    // inverse iteration
    std::vector<double> v(K, 1.0);
    const double shift = chi + 1e-13 * std::max(1.0, std::fabs(chi));
    for (int it = 0; it < 4; ++it) {
        std::vector<double> dd(K), sub(e), sup(e);
        for (int i = 0; i < K; ++i) dd[i] = d[i] - shift;
        tridiag_solve(sub, dd, sup, v);
        double nrm = 0;
        for (double t : v) nrm += t * t;
        nrm = std::sqrt(nrm);
        for (double& t : v) t /= nrm;
    }
    a.resize(K);
    for (int i = 0; i < K; ++i) a[i] = v[i] * std::sqrt(2.0 * i + 0.5);
    if (psi(0.0) < 0)
        for (double& t : a) t = -t;
    psi0 = psi(0.0);
    psi1 = psi(1.0);
    std::vector<double> gx, gw;
    gauss_legendre(K + 10, gx, gw);
    double s = 0;
    for (size_t i = 0; i < gx.size(); ++i) s += gw[i] * psi(gx[i]);
    lambda = s / psi0;   // App. B: lambda_0 = (1/psi(0)) int psi
}

double Prolate::psi(double x) const {
    const int nmax = 2 * static_cast<int>(a.size()) - 2;
    double p0 = 1.0, p1 = x, s = a[0];
    for (int n = 1; n < nmax; ++n) {
        double p2 = ((2.0 * n + 1.0) * x * p1 - n * p0) / (n + 1.0);   // P_{n+1}
        p0 = p1;
        p1 = p2;
        if ((n + 1) % 2 == 0) s += a[(n + 1) / 2] * p1;
    }
    return s;
}

double Prolate::dpsi(double x) const {
    // P'_{n+1} = P'_{n-1} + (2n+1) P_n, alongside the three-term recurrence of P_n
    const int nmax = 2 * static_cast<int>(a.size()) - 2;
    double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0, s = 0.0;   // P_{n-1}, P_n, P'_{n-1}, P'_n at n = 1
    for (int n = 1; n < nmax; ++n) {
        const double p2 = ((2.0 * n + 1.0) * x * p1 - n * p0) / (n + 1.0);
        const double d2 = d0 + (2.0 * n + 1.0) * p1;
        if ((n + 1) % 2 == 0) s += a[(n + 1) / 2] * d2;
        p0 = p1;
        p1 = p2;
        d0 = d1;
        d1 = d2;
    }
    return s;   // the P_0 term has zero derivative
}

void Prolate::psi_int0_dd(double xhi, double xlo, double* psi_out, double* int0_out) const {
    // psi(x) = sum_i a_i P_{2i}(x) and int_0^x psi = a_0 x + sum_{i>=1} a_i (P_{2i+1} - P_{2i-1})(x) / (4i+1)
    // (int_0^x P_n = (P_{n+1} - P_{n-1}) / (2n+1)), both from one run of the Legendre recurrence
    const int K = static_cast<int>(a.size());
    const DD x{xhi, xlo};
    DD p0 = dd(1.0), p1 = x, sp = dd(a[0]), si = x * a[0];
    for (int n = 1; n <= 2 * K - 2; ++n) {
        const DD p2 = (x * p1 * (2.0 * n + 1.0) - p0 * static_cast<double>(n)) / (n + 1.0);   // P_{n+1}
        if (n % 2 == 1) {
            if ((n + 1) / 2 < K) sp = sp + p2 * a[(n + 1) / 2];
        } else {
            si = si + (p2 - p0) * a[n / 2] / (2.0 * n + 1.0);
        }
        p0 = p1;
        p1 = p2;
    }
    psi_out[0] = sp.hi;
    psi_out[1] = sp.lo;
    int0_out[0] = si.hi;
    int0_out[1] = si.lo;
}

double Prolate::cos_transform(double omega) const {
    CosQuadrature q(*this, std::fabs(omega));
    return q(omega);
}

CosQuadrature::CosQuadrature(const Prolate& f, double omega_max) {
    const int N = static_cast<int>(f.a.size()) + static_cast<int>(0.6 * omega_max) + 48;
    gauss_legendre(N, x, w);
    for (int i = 0; i < N; ++i) w[i] *= f.psi(x[i]);
}

double CosQuadrature::operator()(double omega) const {
    double s = 0;
    for (size_t i = 0; i < x.size(); ++i) s += w[i] * std::cos(omega * x[i]);
    return s;
}

// --------------------------------------------------------------- Lambert W --
double lambert_w(int branch, double z) {
    const double em1 = 0.36787944117144233;   // 1/e
    if (branch != 0 && branch != -1) throw std::invalid_argument("Lambert W: branch must be 0 or -1");
    if (!(z >= -em1 - 1e-15)) throw std::invalid_argument("Lambert W: z < -1/e or not a number");
    if (branch == -1 && !(z < 0)) throw std::invalid_argument("Lambert W_{-1}: z must be in [-1/e, 0)");
    double w;
    if (branch == 0) {
        if (z > 3.0) {
            const double l1 = std::log(z), l2 = std::log(l1);
            w = l1 - l2 + l2 / l1;
        } else if (z > -0.25) {
            w = std::log1p(z);
        } else {
            w = -1.0 + std::sqrt(std::max(0.0, 2.0 * (1.0 + z / em1)));
        }
    } else {
        if (z < -0.25) {
            w = -1.0 - std::sqrt(std::max(0.0, 2.0 * (1.0 + z / em1)));
        } else {
            const double l1 = std::log(-z), l2 = std::log(-l1);
            w = l1 - l2 + l2 / l1;
        }
    }
    for (int it = 0; it < 100; ++it) {
        const double ew = std::exp(w);
        const double f = w * ew - z;
        const double wp1 = w + 1.0;
        if (wp1 == 0.0) break;
        const double dw = f / (ew * wp1 - (w + 2.0) * f / (2.0 * wp1));
        w -= dw;
        if (std::fabs(dw) <= 1e-15 * (1.0 + std::fabs(w))) break;
    }
    return w;
}

double kappa_constant() {
    // sum_{k in Z^3 \ 0} |k|^-4 = sum_n r3(n)/n^2; tail sum_{n > N} r3(n)/n^2 ~ 4 pi / sqrt(N + 1/2)
    const long N = 40000;
    const int K = static_cast<int>(std::sqrt(static_cast<double>(N))) + 1;
    double s = 0;
    for (int i = -K; i <= K; ++i)
        for (int j = -K; j <= K; ++j)
            for (int k = -K; k <= K; ++k) {
                const long q = static_cast<long>(i) * i + static_cast<long>(j) * j + static_cast<long>(k) * k;
                if (q > 0 && q <= N) s += 1.0 / (static_cast<double>(q) * q);
            }
    s += 4.0 * kPi / std::sqrt(N + 0.5);
    return s / (kPi * kPi);
}

int good_size(int m, int mult) {
    m = std::max(m, mult);
    for (;; ++m) {
        if (m % mult) continue;
        int r = m;
        for (int p : {2, 3, 5, 7})
            while (r % p == 0) r /= p;
        if (r == 1) return m;
    }
}

ewald_opts default_opts() {
    ewald_opts o{};
    o.precision = EWALD_FP64;
    o.rc = 0.0;
    o.grid_density = 0.0;
    o.tol_safety = 0.25;
    o.sr_reach = 0;
    o.window_extra = 0;
    o.autotune = 0;
    o.spread_kernel = 0;
    return o;
}

// ------------------------------------------------------------------- fits ---
namespace {

// Chebyshev interpolant of f at deg+1 first-kind nodes on [-1, 1], converted to monomials.  The
// coefficient sums and the conversion (whose T_k coefficients reach 2^(k-1)) run in double-double.
template <class F>
std::vector<double> cheb_monomial_fit(F f, int deg) {
    const int N = deg + 1;
    std::vector<double> fv(N);
    std::vector<DD> ch(N);
    for (int j = 0; j < N; ++j) fv[j] = f(std::cos(kPi * (j + 0.5) / N));
    for (int k = 0; k < N; ++k) {
        DD s;
        for (int j = 0; j < N; ++j) s = s + dd(fv[j]) * std::cos(kPi * k * (j + 0.5) / N);
        ch[k] = s * (k == 0 ? 1.0 : 2.0) / static_cast<double>(N);
    }
    // monomial coefficients of T_k by the recurrence T_{k+1} = 2 z T_k - T_{k-1} (exact integers)
    std::vector<DD> tm1(N), t0(N), mono(N);
    t0[0] = dd(1.0);
    for (int k = 0; k < N; ++k) {
        for (int i = 0; i < N; ++i) mono[i] = mono[i] + ch[k] * t0[i];
        std::vector<DD> t1(N);
        if (k == 0) {                      // T_1 = z
            if (N > 1) t1[1] = dd(1.0);
        } else {
            for (int i = 0; i + 1 < N; ++i) t1[i + 1] = t0[i] * 2.0;
            for (int i = 0; i < N; ++i) t1[i] = t1[i] - tm1[i];
        }
        tm1 = t0;
        t0 = t1;
    }
    std::vector<double> out(N);
    for (int i = 0; i < N; ++i) out[i] = to_double(mono[i]);
    return out;
}

template <class F>
double max_fit_error(F f, const std::vector<double>& c, int deg, int nsample) {
    double e = 0;
    for (int i = 0; i <= nsample; ++i) {
        const double z = -1.0 + 2.0 * i / nsample;
        e = std::max(e, std::fabs(horner(c.data(), deg, z) - static_cast<double>(f(z))));
    }
    return e;
}

}  // namespace

std::vector<double> fit_window(const Prolate& pw, int P, int deg, bool deriv, double* max_err) {
    std::vector<double> out;
    double err = 0;
    for (int a = 0; a < P; ++a) {
        auto f = [&](double z) {
            const double s = (z + P - 1 - 2.0 * a) / P;
            return (deriv ? pw.dpsi(s) : pw.psi(s)) / pw.psi0;
        };
        auto c = cheb_monomial_fit(f, deg);
        err = std::max(err, max_fit_error(f, c, deg, 8 * (deg + 1)));
        out.insert(out.end(), c.begin(), c.end());
    }
    if (max_err) *max_err = err;
    return out;
}

// P1(u) = Phi(x) / (x r_c) and Q(u) = (x Phi'(x) - Phi(x)) / (x^3 r_c^3), x = r / r_c = sqrt((u + 1)/2),
// with Phi(x) = 2 / (lambda_0 psi(0)) int_0^x psi (eq. Phi_cs).  Q's numerator is O(x^3) while both of
// its terms are O(x): double-double keeps the digits that the subtraction cancels.
RadialFitter::RadialFitter(const Prolate& ps, double rc) : ps_(ps), rc_(rc) {}

void RadialFitter::values(double u, double* p1, double* q) const {
    const DD norm = dd(2.0) / (dd(ps_.lambda) * ps_.psi0);
    const DD x = dd_sqrt(two_sum(u, 1.0) * 0.5);
    double pv[2], iv[2];
    ps_.psi_int0_dd(x.hi, x.lo, pv, iv);
    const DD Phi = norm * DD{iv[0], iv[1]};
    const DD rc = dd(rc_);
    if (p1) *p1 = to_double(Phi / (x * rc));
    if (q) {
        const DD dPhi = norm * DD{pv[0], pv[1]};
        *q = to_double((dPhi * x - Phi) / (x * x * x) / (rc * rc * rc));
    }
}

double RadialFitter::value(double u, int which) const {
    double v = 0;
    values(u, which == 0 ? &v : nullptr, which == 0 ? nullptr : &v);
    return v;
}

std::vector<double> RadialFitter::fit(int deg, int which, double* rel_err) {
    auto c = cheb_monomial_fit([&](double u) { return value(u, which); }, deg);
    if (rel_err) {
        // error measured away from u = -1, where x -> 0 and both functions approach finite limits
        // that the sampled form reaches only through the cancellation; both functions are sampled
        // at the check points on first use
        constexpr int kCheck = 1000;
        auto check_u = [](int i) { return -1.0 + 1e-4 + (2.0 - 1e-4) * i / kCheck; };
        if (check_[0].empty()) {
            check_[0].resize(kCheck + 1);
            check_[1].resize(kCheck + 1);
            for (int i = 0; i <= kCheck; ++i) values(check_u(i), &check_[0][i], &check_[1][i]);
        }
        const std::vector<double>& v = check_[which];
        double e = 0, sm = 0;
        for (int i = 0; i <= kCheck; ++i) {
            sm = std::max(sm, std::fabs(v[i]));
            e = std::max(e, std::fabs(horner(c.data(), deg, check_u(i)) - v[i]));
        }
        *rel_err = e / sm;
    }
    return c;
}

std::vector<double> fit_radial(const Prolate& ps, double rc, int deg, int which, double* rel_err) {
    RadialFitter f(ps, rc);
    return f.fit(deg, which, rel_err);
}

void scale_tables(const ewald_params& p, const Prolate& ps, const Prolate& pw, std::vector<double>& iw,
                  std::vector<double>& mtab) {
    if (!(p.box[0] == p.box[1] && p.box[1] == p.box[2] && p.grid[0] == p.grid[1] && p.grid[1] == p.grid[2])) {
        // cuboid: 1/(phihat_d/h_d)^2 per axis (x, then y, then z entries); M-hat from the gamma polynomial
        iw.clear();
        for (int d = 0; d < 3; ++d) {
            const int m = p.grid[d];
            const double L = p.box[d], h = L / m, alpha = p.P * h / 2.0;
            const CosQuadrature qw(pw, kPi * (m / 2) * alpha * 2.0 / L + 1.0);
            for (int i = 0; i < m; ++i) {
                const int k = i < m / 2 ? i : i - m;
                const double ph = alpha * qw(2.0 * kPi * k / L * alpha) / (pw.psi0 * h);
                iw.push_back(1.0 / (ph * ph));
            }
        }
        mtab.clear();
        return;
    }
    const int m = p.m;
    const double L = p.L;
    iw.resize(m);
    const CosQuadrature qw(pw, kPi * (m / 2) * p.alpha * 2.0 / L + 1.0);
    for (int i = 0; i < m; ++i) {
        const int k = i < m / 2 ? i : i - m;
        const double w = 2.0 * kPi * k / L;
        const double ph = p.alpha * qw(w * p.alpha) / (pw.psi0 * p.h);   // phihat_1d(k) / h
        iw[i] = 1.0 / (ph * ph);
    }
    const int qmax = (m / 2) * (m / 2);
    mtab.assign(qmax + 1, 0.0);
    const double V = L * L * L;
    const CosQuadrature qs(ps, 2.0 * kPi * (m / 2) / L * p.rc + 1.0);
    for (int q = 1; q <= qmax; ++q) {
        const double omega = 2.0 * kPi * std::sqrt(static_cast<double>(q)) / L;
        const double gh = qs(omega * p.rc) / (ps.lambda * ps.psi0);   // eq. gammahatintegral (with 1/lambda_0)
        mtab[q] = L * L / (kPi * q) * gh / V;                          // eq. MhatPSWF and the 1/V of step 3
    }
}

// In-band mollifier transform for cuboid boxes: gammahat(omega) = psi(s)/psi(0), s = omega r_c/c_s
// (Lemma 2 applied to eq. gammahatintegral; every retained mode has s < 1).  Fitted as a polynomial in
// u = 2 s^2 - 1 (Chebyshev nodes, monomial coefficients); max_err is absolute (the function is <= 1).
std::vector<double> fit_gamma(const Prolate& ps, int deg, double* max_err) {
    auto f = [&](double u) {
        const double sv = std::sqrt(std::max(0.0, (u + 1.0) / 2.0));
        return ps.psi(sv) / ps.psi0;
    };
    auto c = cheb_monomial_fit(f, deg);
    if (max_err) *max_err = max_fit_error(f, c, deg, 8 * (deg + 1));
    return c;
}

HostPlan make_plan(double L, int64_t n, double tol, const ewald_opts& o) {
    const double box[3] = {L, L, L};
    return make_plan_box(box, n, tol, o);
}

HostPlan make_plan_box(const double* box, int64_t n, double tol, const ewald_opts& o) {
    for (int d = 0; d < 3; ++d)
        if (!(box[d] > 0) || !std::isfinite(box[d])) throw std::invalid_argument("box edges must be positive and finite");
    const bool cube = box[0] == box[1] && box[1] == box[2];
    const double L = std::min(box[0], std::min(box[1], box[2]));   // the cube's edge, or the shortest edge
    const double V = box[0] * box[1] * box[2];
    if (n < 2) throw std::invalid_argument("n must be at least 2");
    if (!(tol >= 1e-13 && tol <= 1e-2)) throw std::invalid_argument("tol must lie in [1e-13, 1e-2]");
    if (o.precision != EWALD_FP64 && o.precision != EWALD_MIXED && o.precision != EWALD_FLOATFLOAT)
        throw std::invalid_argument("unknown precision");
    if (std::isnan(o.rc)) throw std::invalid_argument("rc must be a number (<= 0: automatic cutoff)");
    if (!(o.tol_safety > 0 && o.tol_safety <= 1)) throw std::invalid_argument("tol_safety must lie in (0, 1]");
    if (!(o.grid_density >= 0) || !std::isfinite(o.grid_density))
        throw std::invalid_argument("grid_density must be 0 (automatic) or positive");
    if (o.window_extra < 0 || o.window_extra > 8) throw std::invalid_argument("window_extra must lie in [0, 8]");
    if (o.autotune != 0 && o.autotune != 1) throw std::invalid_argument("autotune must be 0 or 1");
    if (o.sr_reach < 0 || o.sr_reach > 4) throw std::invalid_argument("sr_reach must lie in [0, 4]");
    if (o.spread_kernel < 0 || o.spread_kernel > 2) throw std::invalid_argument("spread_kernel must be 0, 1 or 2");

    const double As = 5.0, Aw = 3.1;                      // Secs. 5.1.1 and 5.2.1
    static const double kappa = kappa_constant();
    // grid density of the cutoff rule: automatic (0) = the measured optima of the GB300 kernels, 6 for
    // float32 plans (tile 8) and 3 for the float64 / float-float ones (tile 4)
    const bool f32_plan = o.precision == EWALD_MIXED && tol >= 1e-7;
    const double gdens = o.grid_density > 0 ? o.grid_density : (f32_plan ? 6.0 : 3.0);
    const double t_pot = tol * o.tol_safety;   // potential target (window / aliasing side)
    double t = t_pot;                            // split target (tightened for forces below)
    auto cs_at = [&](double rcl, double tt) {
        const double bs_eps = As * std::sqrt(rcl) / (std::sqrt(kappa) * tt);
        return 0.5 * lambert_w(0, 2.0 * bs_eps * bs_eps);   // eq. cs_dimless
    };
    auto cs_of = [&](double rcl) { return cs_at(rcl, t); };
    auto cutoff = [&]() {
        double rcl;
        if (o.rc > 0) {
            rcl = std::min(o.rc / L, 0.5);
        } else {
            // cube: m* = (g n)^{1/3} points per edge; cuboid (in units of the shortest edge L):
            // m* = L / h with the common spacing h = (V / (g n))^{1/3}
            const double mstar = cube ? std::cbrt(gdens * static_cast<double>(n))
                                      : L / std::cbrt(V / (gdens * static_cast<double>(n)));
            rcl = 0.1;
            for (int it = 0; it < 12; ++it) rcl = std::min(cs_of(rcl) / (kPi * mstar), 0.5);
        }
        return rcl;
    };
    double rcl = cutoff();
    // Forces: their relative error, measured against the oracle, is ~m/10 times the potential's
    // (the band-edge modes of the truncation carry the factor |k| ~ m/2 into the gradient); the
    // potential target is tightened accordingly (factor min(1, 10/m0), m0 the unrounded grid size).
    const double m0 = cs_of(rcl) / (kPi * rcl);
    if (m0 > 10.0) {
        t *= 10.0 / m0;
        rcl = cutoff();
    }
    const double cs = cs_of(rcl);
    const double mraw = std::ceil(cs / (kPi * rcl));      // eq. m_cs_dimless
    if (mraw > 1024) throw std::length_error("grid beyond 1024^3");
    // float32 plans tile the grid by 8, the others by 4 (spreading tile edge; m is a multiple of it)
    const int precision = (o.precision == EWALD_MIXED && tol < 1e-7) ? EWALD_FLOATFLOAT : o.precision;
    const int tile = precision == EWALD_MIXED ? 8 : 4;
    int mv[3];
    double hmax = 0;
    if (cube) {
        mv[0] = mv[1] = mv[2] = good_size(static_cast<int>(mraw), tile);
    } else {
        // cuboid: m_d = ceil(c_s L_d / (pi r_c)) per axis, rounded like the cube's m
        for (int d = 0; d < 3; ++d) {
            const double md = std::ceil(cs * (box[d] / L) / (kPi * rcl));
            if (md > 1024) throw std::length_error("grid beyond 1024 points on an axis");
            mv[d] = good_size(static_cast<int>(md), tile);
            hmax = std::max(hmax, box[d] / mv[d]);
        }
    }
    const int m = mv[0];
    if (mv[0] > 1024 || mv[1] > 1024 || mv[2] > 1024) throw std::length_error("grid beyond 1024^3");
    // eq. csrc holds exactly (on the coarsest axis of a cuboid: r_c = c_s h_max / pi)
    rcl = cube ? cs / (kPi * m) : cs * hmax / (kPi * L);
    const double bw = (As / Aw) * std::sqrt(rcl);
    // eq. cwW balances the aliasing error against the potential target: the force factor above
    // tightens the split only (forces follow the split truncation, not the window; see the sizing notes)
    const double cs_w = cs_at(rcl, t_pot);
    const double cw_t = -0.5 * lambert_w(-1, -2.0 * bw * bw * std::exp(-2.0 * cs_w) / cs_w);
    const double alpha_over_L = rcl * cw_t / cs;          // eq. alpha
    // eq. P_dimless (cuboid: P = ceil(2 alpha / h_max), the support in points of the coarsest axis)
    int P = static_cast<int>(std::ceil(2.0 * alpha_over_L * (cube ? m : L / hmax)));
    P = std::max(P + o.window_extra, 3);
    if (P > 24) throw std::length_error("window support P > 24 (tolerance too tight)");

    HostPlan hp;
    ewald_params& p = hp.p;
    for (int d = 0; d < 3; ++d) {
        p.box[d] = box[d];
        p.grid[d] = mv[d];
    }
    p.L = box[0];
    p.n = n;
    p.tol = tol;
    p.m = m;
    p.P = P;
    p.h = box[0] / m;
    p.rc = rcl * L;
    p.cs = cs;
    p.cw_target = cw_t;
    p.cw = kPi * P / 2.0;                                 // eq. cwP
    p.alpha = P * p.h / 2.0;
    // float32 products cannot reach tol < 1e-7; below it MIXED runs the float-float kernels
    p.precision = precision;
    p.tile = tile;
    // real-space cells of edge >= rc / reach.  float32 plans: columns of edge >= rc / reach in x and y
    // (reach 1 by default) cut into cells of edge >= rc / 4 along z, which the float32 kernel walks as
    // z windows per target.  Otherwise cubic cells; the automatic reach aims at ~3 particles per cell,
    // or ~1.5 for float-float plans, whose pairs cost ~15x a float32 pair: finer cells approximate the
    // cutoff sphere better (fewer candidates per pair) and fit the kernel's 4 targets per pass
    int reach = o.sr_reach;
    if (reach <= 0) {
        if (precision == EWALD_MIXED) {
            reach = 1;
        } else {
            const double per_cell = precision == EWALD_FLOATFLOAT ? 1.5 : 3.0;
            reach = static_cast<int>(std::lround(rcl * std::cbrt(static_cast<double>(n) / per_cell)));
            reach = std::max(1, std::min(reach, 4));
        }
    }
    const int reach_z = precision == EWALD_MIXED ? 4 : reach;
    p.sr_reach = reach;
    p.sr_reach_z = reach_z;
    for (int d = 0; d < 3; ++d) {   // cells of edge L_d / ncell_d >= rc / reach_d on every axis
        const int rd = d == 2 ? reach_z : reach;
        int nc = static_cast<int>(std::floor(rd * (box[d] / L) / rcl));
        p.cells[d] = std::max(1, std::min(nc, 1024));
    }
    p.ncell = p.cells[0];
    p.fit_tol = std::max(0.02 * t, p.precision == EWALD_MIXED ? 1e-8 : 5e-15);
    // spreading kernel: tensor cores on request for float32 plans whose tile block fits the accumulator
    // (P <= 14); automatic = CUDA cores: timed alone the tensor-core kernel is faster at tol >= 1e-5
    // (53 vs 59 us at n = 1e5, tol 1e-4), but inside the step, concurrent with the real-space sum, the
    // whole step measured 1-2% slower with it (0.336 vs 0.333 ms at 1e-5, 0.389 vs 0.381 ms at 1e-6)
    const bool tc_ok = p.precision == EWALD_MIXED && P <= 14;
    p.spread_kernel = tc_ok && o.spread_kernel == 2 ? 2 : 1;

    const Prolate ps(p.cs), pw(p.cw);
    p.lambda_s = ps.lambda;
    p.lambda_w = pw.lambda;
    p.self_coeff = 2.0 / (ps.lambda * p.rc);

    // ---- window polynomials: smallest degree meeting fit_tol
    {
        double dmax = 0;
        for (int i = 0; i <= 400; ++i) dmax = std::max(dmax, std::fabs(pw.dpsi(-1.0 + i / 200.0)) / pw.psi0);
        bool ok = false;
        for (int deg = 4; deg <= kDegWMax && !ok; ++deg) {
            double err = 0, derr = 0;
            auto wc = fit_window(pw, P, deg, false, &err);
            auto dwc = fit_window(pw, P, deg, true, &derr);
            if (err <= p.fit_tol && derr <= p.fit_tol * dmax) {
                ok = true;
                p.deg_w = deg;
                hp.wc = wc;
                hp.dwc = dwc;
            }
        }
        if (!ok) throw std::runtime_error("window polynomial fit did not converge");
    }
    // ---- radial polynomials in u = 2 r^2/rc^2 - 1
    {
        bool ok = false;
        RadialFitter rf(ps, p.rc);
        for (int deg = 4; deg <= kDegRMax && !ok; ++deg) {
            double e1 = 0, e2 = 0;
            auto c1 = rf.fit(deg, 0, &e1);
            auto c2 = rf.fit(deg, 1, &e2);
            if (e1 <= p.fit_tol && e2 <= p.fit_tol) {
                ok = true;
                p.deg_r = deg;
                hp.p1c = c1;
                hp.qc = c2;
            }
        }
        if (!ok) throw std::runtime_error("radial polynomial fit did not converge");
    }
    // ---- cuboid boxes: mollifier transform polynomial for the scaling step
    p.deg_g = 0;
    if (!cube) {
        bool ok = false;
        for (int deg = 4; deg <= kDegRMax && !ok; ++deg) {
            double e = 0;
            auto gc = fit_gamma(ps, deg, &e);
            if (e <= p.fit_tol) {
                ok = true;
                p.deg_g = deg;
                hp.gc = gc;
            }
        }
        if (!ok) throw std::runtime_error("mollifier transform fit did not converge");
    }
    scale_tables(p, ps, pw, hp.iw, hp.mtab);
    return hp;
}

}  // namespace pswf
