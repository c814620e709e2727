// Host-side planner: PSWF evaluation, Alg. 3 parameters, polynomial fits and
// scaling tables.  Pure C++ (no CUDA); shared by the C ABI and the device setup.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "pswf_ewald.h"

namespace pswf {

// psi_0^c on [-1, 1] as a Legendre series (App. B).
struct Prolate {
    double c = 0, chi = 0, lambda = 0, psi0 = 0, psi1 = 0;
    std::vector<double> a;   // coefficients of P_0, P_2, P_4, ... (standard Legendre normalisation)

    explicit Prolate(double c);
    double psi(double x) const;
    double dpsi(double x) const;
    // psi(x) and int_0^x psi in double-double (x = xhi + xlo; each result as {hi, lo})
    void psi_int0_dd(double xhi, double xlo, double* psi, double* int0) const;
    double cos_transform(double omega) const;     // int_{-1}^{1} psi(u) cos(omega u) du
};

// Gauss-Legendre rule for int_{-1}^{1} psi(u) cos(omega u) du, |omega| <= omega_max.
struct CosQuadrature {
    std::vector<double> x, w;   // nodes and weights already multiplied by psi(node)
    CosQuadrature(const Prolate& f, double omega_max);
    double operator()(double omega) const;
};

double lambert_w(int branch, double z);
double kappa_constant();                           // pi^-2 sum_{k != 0} |k|^-4
int good_size(int m, int mult);

// Complete host plan: parameters and every table the device path needs.
struct HostPlan {
    ewald_params p{};
    // window polynomials: coefficient k of weight a at wc[a*(deg_w+1) + k] (monomials in z)
    std::vector<double> wc, dwc;    // dwc fits psi'(s)/psi(0) (the 1/alpha is applied on the device)
    // radial polynomials in u = 2 r^2/rc^2 - 1: R(r) = 1/r - P1(u), -R'(r)/r = 1/r^3 + Q(u)
    std::vector<double> p1c, qc;
    // scaling: S(k) = mtab[|k|^2] * iw[kx] * iw[ky] * iw[kz] for 0 < |k|^2 < (m/2)^2, else 0
    std::vector<double> iw;         // indexed by grid index 0..m-1 (cuboids: m_x + m_y + m_z entries, by axis)
    std::vector<double> mtab;       // indexed by |k|^2 = 0..(m/2)^2, mtab[0] = 0 (cubes only)
    // cuboids: gammahat(omega) = g(2 s^2 - 1), s = |omega| r_c / c_s, monomial coefficients of g
    std::vector<double> gc;
};

constexpr int kDegWMax = 40, kDegRMax = 60;

std::vector<double> fit_window(const Prolate& pw, int P, int deg, bool deriv, double* max_err);
std::vector<double> fit_radial(const Prolate& ps, double rc, int deg, int which, double* rel_err);

// The two radial functions sampled once for a degree search: fit(deg, which, &rel_err) equals
// fit_radial(ps, rc, deg, which, &rel_err) and reuses the error-check samples across degrees.
class RadialFitter {
public:
    RadialFitter(const Prolate& ps, double rc);
    std::vector<double> fit(int deg, int which, double* rel_err);
    double value(double u, int which) const;   // P1 (which = 0) or Q (which = 1) at u = 2 r^2/rc^2 - 1
    void values(double u, double* p1, double* q) const;   // both (either pointer may be NULL)

private:
    const Prolate& ps_;
    double rc_;
    std::vector<double> check_[2];   // both functions at the error-check points (filled on first use)
};
void scale_tables(const ewald_params& p, const Prolate& ps, const Prolate& pw, std::vector<double>& iw,
                  std::vector<double>& mtab);

// Throws std::invalid_argument / std::runtime_error with a message on failure.
HostPlan make_plan(double L, int64_t n, double tol, const ewald_opts& opts);
HostPlan make_plan_box(const double* box, int64_t n, double tol, const ewald_opts& opts);   // box[3]
std::vector<double> fit_gamma(const Prolate& ps, int deg, double* max_err);
ewald_opts default_opts();

// Sets the thread-local message returned by ewald_last_error() (defined in api.cu).
void record_error(const std::string& msg);

double horner(const double* c, int deg, double x);

}  // namespace pswf
