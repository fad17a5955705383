// Host-side setup of the PML-BIE modal solver: geometry, graded grid, PML
// tables, Alpert quadrature, close-pair lists and the diagonal term.
//
// Sections of Wang & Lu, arXiv 2412.11162, restated here:
//   Sec. 2     interface, normal toward the lower medium, reference field.
//   Sec. 3.1   PML stretching (Eqs. (rhot), (sgm1)), conormal nu_c = A^T nu.
//   Sec. 3.2   solid-angle diagonal (Lemmas 3.1-3.3).
//   Sec. 4     graded parametrisation (Eq. (sxi)), Alpert's hybrid
//              Gauss-trapezoid rule of order 10 (Sec. 5) with Lagrange
//              interpolation of the off-grid density values.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <mutex>
#include <stdexcept>
#include <thread>

#include "internal.h"

#if defined(__x86_64__)
#include <quadmath.h>
#endif

namespace pmlbie {

// binary128 arithmetic for the Alpert generator: __float128 on x86-64
// (libquadmath), long double on aarch64 (binary128 there).
namespace q128 {
#if defined(__x86_64__)
using real = __float128;
inline real exp_(real x) { return expq(x); }
inline real log_(real x) { return logq(x); }
inline real pow_(real x, real y) { return powq(x, y); }
inline real abs_(real x) { return fabsq(x); }
inline bool finite_(real x) { return finiteq(x); }
inline real pi_() { return 4 * atanq((real)1); }
#else
using real = long double;
inline real exp_(real x) { return expl(x); }
inline real log_(real x) { return logl(x); }
inline real pow_(real x, real y) { return powl(x, y); }
inline real abs_(real x) { return fabsl(x); }
inline bool finite_(real x) { return std::isfinite(x); }
inline real pi_() { return 4 * atanl((real)1); }
#endif
}  // namespace q128

static thread_local std::string g_err = "no error";
thread_local long g_launches = 0;
void set_error(const std::string& msg) { g_err = msg; }
int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}
const char* error_text() { return g_err.c_str(); }

namespace {

constexpr double kPi = 3.14159265358979323846;
const q128::real kPiQ = q128::pi_();

// Run f(lo, hi) over [0, n) split into contiguous chunks on the host cores.
template <typename F>
void parallel_rows(int n, F f) {
    int nt = (int)std::thread::hardware_concurrency();
    nt = std::max(1, std::min(nt, 64));
    if (n < 64 || nt == 1) {
        f(0, n);
        return;
    }
    std::vector<std::thread> th;
    int chunk = (n + nt - 1) / nt;
    for (int t = 0; t < nt; ++t) {
        int lo = t * chunk, hi = std::min(n, lo + chunk);
        if (lo >= hi) break;
        th.emplace_back([=, &f] { f(lo, hi); });
    }
    for (auto& x : th) x.join();
}

// ---------------------------------------------------------------------------
// Gauss-Legendre nodes on [-1, 1] (Newton on P_n).
// ---------------------------------------------------------------------------
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
    x.resize(n);
    w.resize(n);
    for (int i = 0; i < n; ++i) {
        long double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
        long double dp = 0;
        for (int it = 0; it < 100; ++it) {
            long double p0 = 1, p1 = z;
            for (int k = 2; k <= n; ++k) {
                long double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1);
            long double dz = p1 / dp;
            z -= dz;
            if (std::fabs((double)dz) < 1e-19) break;
        }
        x[i] = (double)z;
        w[i] = (double)(2.0L / ((1 - z * z) * dp * dp));
    }
}

struct GL {
    std::vector<double> x, w;
    explicit GL(int n) { gauss_legendre(n, x, w); }
};

// ---------------------------------------------------------------------------
// PML profile (Eq. (sgm1)) and its integral.
// ---------------------------------------------------------------------------
struct Pml {
    double a1, T, S, L;
    int p;
    double sigma(double rho) const {
        if (rho <= a1) return 0.0;
        if (rho >= L) return S;
        double rb = (rho - L) / T;
        double f1 = (0.5 - 1.0 / p) * rb * rb * rb + rb / p + 0.5;
        double f2 = 1.0 - f1;
        double f1p = std::pow(f1, p), f2p = std::pow(f2, p);
        return 2.0 * S * f1p / (f1p + f2p);
    }
    // int_lo^hi sigma, lo <= hi, composite 24-point Gauss-Legendre
    double integral(double lo, double hi, int panels = 6) const {
        static const GL g(24);
        lo = std::max(lo, a1);
        hi = std::max(hi, a1);
        if (hi <= lo) return 0.0;
        double tot = 0.0;
        for (int k = 0; k < panels; ++k) {
            double a = lo + (hi - lo) * k / panels, b = lo + (hi - lo) * (k + 1) / panels;
            double mid = 0.5 * (a + b), half = 0.5 * (b - a), s = 0.0;
            for (size_t i = 0; i < g.x.size(); ++i) s += g.w[i] * sigma(mid + half * g.x[i]);
            tot += half * s;
        }
        return tot;
    }
    // I(r2 + dr) - I(r2) for an accurately known separation dr: integrated
    // directly over [r2, r2 + dr] when the radii are close (where the
    // difference of tabulated values would cancel), else the difference of
    // the tabulated integrals I1 = I(r2 + dr), I2 = I(r2).
    // (sigma is C^(p-1) at a1, so a short interval that reaches below a1 is
    // integrated from a1 only.)
    double delta(double r2, double dr, double I1, double I2) const {
        if (std::fabs(dr) > 0.05 * T) return I1 - I2;
        double lo = std::min(r2, r2 + dr), hi = std::max(r2, r2 + dr);
        double start = lo, width = std::fabs(dr);   // the interval [start, start + width]
        if (lo < a1) {
            if (hi <= a1) return 0.0;
            start = a1;
            width = hi - a1;
        }
        static const GL g(16);
        double tot = 0.0;
        const int panels = 4;
        for (int k = 0; k < panels; ++k)
            for (size_t i = 0; i < g.x.size(); ++i) {
                double xs = (k + 0.5 * (g.x[i] + 1.0)) / panels;
                tot += 0.5 / panels * g.w[i] * sigma(start + width * xs);
            }
        return (dr < 0 ? -width : width) * tot;
    }
};

// ---------------------------------------------------------------------------
// Curve segments r(s), s in [0, 1]
// ---------------------------------------------------------------------------
// Grading exponent of a segment that leaves the axis at an angle (the surface
// has a conical point there).  With the Sec. 5 exponent 6 the graded nodes
// next to the tip sit at rho ~ 1e-8 .. 1e-6, where the double-layer kernel of
// the targets scales like 1/rho^2 over neighbours spaced geometrically in rho,
// and the Alpert-corrected rule does not resolve it; exponent 2 keeps the tip
// nodes at rho ~ h^2.
constexpr int kConicalP = 2;

struct Segment {
    int p = 0;                           // grading exponent (0: the problem's p)
    bool gauss = false, wavy = false;
    double h = 0, w = 1, R = 1;          // Gaussian bump
    double wR = 1, eps = 0;              // wavy dent: radius, relative amplitude,
    int wm = 1;                          // half-waves of the perturbation
    double r0 = 0, z0 = 0, r1 = 0, z1 = 0;  // line
    void eval(double s, double& rho, double& z, double& drho, double& dz) const {
        if (wavy) {
            // Sec. 5, Example 2: rho = f sin(pi s/2), z = -f cos(pi s/2),
            // f = R (1 - eps sin(m pi s)), from (0, -R) on the axis to (R, 0)
            const double f = wR * (1.0 - eps * std::sin(wm * kPi * s));
            const double df = -wR * eps * wm * kPi * std::cos(wm * kPi * s);
            const double c = std::cos(0.5 * kPi * s), si = std::sin(0.5 * kPi * s);
            rho = f * si;
            z = -f * c;
            drho = df * si + 0.5 * kPi * f * c;
            dz = -df * c + 0.5 * kPi * f * si;
        } else if (gauss) {
            rho = R * s;
            double e0 = std::exp(-R * R / w), g = std::exp(-rho * rho / w);
            z = h * (g - e0) / (1.0 - e0);
            drho = R;
            dz = R * h * (-2.0 * rho / w) * g / (1.0 - e0);
        } else {
            rho = r0 + s * (r1 - r0);
            z = z0 + s * (z1 - z0);
            drho = r1 - r0;
            dz = z1 - z0;
        }
    }
    // r(s) - r(0) (end 0) or r(s) - r(1) (end 1) without cancellation; sc = 1 - s
    void offset(double s, double sc, int end, double& orho, double& oz) const {
        if (wavy) {
            // 1 - cos x = 2 sin^2(x/2); near s = 1, sin(m pi s) = (-1)^(m+1) sin(m pi sc)
            // and sin(pi s/2) = cos(pi sc/2)
            if (end == 0) {
                double z, dr, dz;
                eval(s, orho, z, dr, dz);
                const double q = std::sin(0.25 * kPi * s);
                oz = 2.0 * wR * q * q + wR * eps * std::sin(wm * kPi * s) * std::cos(0.5 * kPi * s);
            } else {
                const double sm = ((wm & 1) ? 1.0 : -1.0) * std::sin(wm * kPi * sc);
                const double q = std::sin(0.25 * kPi * sc);
                orho = -2.0 * wR * q * q - wR * eps * sm * std::cos(0.5 * kPi * sc);
                oz = -wR * (1.0 - eps * sm) * std::sin(0.5 * kPi * sc);
            }
        } else if (gauss) {
            double c = h / (1.0 - std::exp(-R * R / w));
            if (end == 0) {
                orho = R * s;
                oz = c * std::expm1(-(R * s) * (R * s) / w);
            } else {
                orho = -R * sc;
                oz = c * std::exp(-R * R / w) * std::expm1(R * R * sc * (1.0 + s) / w);
            }
        } else if (end == 0) {
            orho = s * (r1 - r0);
            oz = s * (z1 - z0);
        } else {
            orho = -sc * (r1 - r0);
            oz = -sc * (z1 - z0);
        }
    }
    double length() const {
        static const GL g(48);
        double s = 0;
        for (size_t i = 0; i < g.x.size(); ++i) {
            double r, z, dr, dz;
            eval(0.5 * (g.x[i] + 1), r, z, dr, dz);
            s += g.w[i] * std::hypot(dr, dz);
        }
        return 0.5 * s;
    }
};

// Graded map of Eq. (sxi), oriented so that u = 0 -> s = 0: s(u), 1 - s(u)
// (computed separately, accurate near u = 1) and ds/du.
void graded_map(double u, int p, double& s, double& sc, double& ds) {
    double xi = 2.0 * u - 1.0, A = 0.5 - 1.0 / p;
    double x1 = (2.0 * u) * (A * xi * xi - A * xi + 0.5);        // (xi+1)(A xi^2 - A xi + 1/2)
    double x2 = (2.0 * (1.0 - u)) * (A * xi * xi + A * xi + 0.5);  // (1-xi)(A xi^2 + A xi + 1/2)
    double x1p = std::pow(x1, p), x2p = std::pow(x2, p), den = x1p + x2p;
    s = x1p / den;
    sc = x2p / den;
    double dx1 = 3.0 * A * xi * xi + 1.0 / p;
    ds = p * std::pow(x1, p - 1) * std::pow(x2, p - 1) / (den * den) * dx1 * 2.0;
}

struct Curve {
    std::vector<Segment> segs;
    std::vector<int> brk;   // breakpoint grid indices
    int Nt = 0;
    double h = 0;
    int p = 6;
    struct Pt {
        double rho, z, speed, nu_r, nu_z;
        int bk;          // nearest breakpoint (index into brk)
        double ox, oz;   // r - r(breakpoint), accurate
    };
    Pt at(double t) const {
        int k = 0;
        while (k + 1 < (int)segs.size() && t >= brk[k + 1] * h) ++k;
        double t0 = brk[k] * h, t1 = brk[k + 1] * h;
        double u = (t - t0) / (t1 - t0), s, sc, ds;
        graded_map(u, segs[k].p ? segs[k].p : p, s, sc, ds);
        double r, z, dr, dz;
        segs[k].eval(s, r, z, dr, dz);
        int end = u > 0.5 ? 1 : 0;
        double ox, oz;
        segs[k].offset(s, sc, end, ox, oz);
        double dsdt = ds / (t1 - t0);
        dr *= dsdt;
        dz *= dsdt;
        Pt o;
        o.rho = r;
        o.z = z;
        o.bk = k + end;
        o.ox = ox;
        o.oz = oz;
        o.speed = std::hypot(dr, dz);
        if (o.speed > 0) {
            o.nu_r = dz / o.speed;   // tangent rotated by -90 degrees: toward Omega_2
            o.nu_z = -dr / o.speed;
        } else {
            o.nu_r = 0;
            o.nu_z = -1;
        }
        return o;
    }
};

// ---------------------------------------------------------------------------
// Hurwitz zeta zeta(-p, a) and d/ds zeta(s, a) at s = -p (integer p >= 0,
// real a > 0) from the Euler-Maclaurin expansion about a, which terminates for
// the value and converges quickly for the derivative when a = 10.
// ---------------------------------------------------------------------------
q128::real bernoulli_even(int n2) {   // B_{n2}, n2 even >= 2
    static const q128::real small[] = {(q128::real)1 / 6, (q128::real)-1 / 30, (q128::real)1 / 42, (q128::real)-1 / 30, (q128::real)5 / 66,
                                        (q128::real)-691 / 2730, (q128::real)7 / 6, (q128::real)-3617 / 510, (q128::real)43867 / 798};
    if (n2 <= 18) return small[n2 / 2 - 1];
    // B_{2j} = (-1)^{j+1} 2 (2j)! zeta(2j) / (2 pi)^{2j}
    q128::real z = 0;
    for (int n = 1; n <= 60; ++n) z += q128::pow_((q128::real)n, (q128::real)(-n2));
    q128::real f = 1;
    for (int i = 2; i <= n2; ++i) f *= i;
    q128::real tp = q128::pow_(2 * kPiQ, (q128::real)n2);
    int j = n2 / 2;
    return ((j + 1) % 2 == 0 ? (q128::real)1 : (q128::real)-1) * 2 * f * z / tp;
}

void hurwitz_at_neg_int(int p, q128::real a, q128::real& val, q128::real& der) {
    q128::real s = -p, la = q128::log_(a);
    q128::real ap1 = q128::pow_(a, 1 - s), ams = q128::pow_(a, -s);
    val = ap1 / (s - 1) + ams / 2;
    der = ap1 * (-la / (s - 1) - 1 / ((s - 1) * (s - 1))) - la * ams / 2;
    q128::real fact = 1;   // (2j)!
    for (int j = 1; j <= 30; ++j) {
        fact *= (2 * j - 1) * (2 * j);
        q128::real c = bernoulli_even(2 * j) / fact;
        // rising factorial (s)_{2j-1} and its derivative at s = -p
        q128::real prod = 1, dprod = 0;
        for (int i = 0; i <= 2 * j - 2; ++i) {
            q128::real f = s + i;
            dprod = dprod * f + prod;
            prod *= f;
        }
        q128::real pw = q128::pow_(a, -s - 2 * j + 1);
        val += c * prod * pw;
        der += c * (dprod - prod * la) * pw;
    }
}

// Solve a dense n x n system in place (partial pivoting), q128::real.
bool solve_ld(std::vector<q128::real>& A, std::vector<q128::real>& b, int n) {
    for (int k = 0; k < n; ++k) {
        int piv = k;
        for (int i = k + 1; i < n; ++i)
            if (q128::abs_(A[i * n + k]) > q128::abs_(A[piv * n + k])) piv = i;
        if (A[piv * n + k] == 0) return false;
        if (piv != k) {
            for (int j = 0; j < n; ++j) std::swap(A[k * n + j], A[piv * n + j]);
            std::swap(b[k], b[piv]);
        }
        for (int i = k + 1; i < n; ++i) {
            q128::real f = A[i * n + k] / A[k * n + k];
            for (int j = k; j < n; ++j) A[i * n + j] -= f * A[k * n + j];
            b[i] -= f * b[k];
        }
    }
    for (int k = n - 1; k >= 0; --k) {
        q128::real s = b[k];
        for (int j = k + 1; j < n; ++j) s -= A[k * n + j] * b[j];
        b[k] = s / A[k * n + k];
    }
    return true;
}

}  // namespace

// ---------------------------------------------------------------------------
// Alpert's log-singular end correction (j nodes, skip a): nodes x_k in (0, a)
// and weights w_k with  sum_k w_k x_k^p = -zeta(-p, a)  and
// sum_k w_k x_k^p log x_k = zeta'(-p, a),  p = 0..j-1, solved by Newton's
// method along a homotopy of the right-hand side, in binary128.  Each
// equation p is scaled by a^-p.
// ---------------------------------------------------------------------------
void alpert_log_rule(int j, int a, std::vector<double>& xo, std::vector<double>& wo) {
    static std::mutex mu;
    static std::vector<double> cx, cw;
    static int cj = -1, ca = -1;
    std::lock_guard<std::mutex> lk(mu);
    if (cj == j && ca == a) {
        xo = cx;
        wo = cw;
        return;
    }
    const int n = 2 * j;
    std::vector<q128::real> tgt(n), scale(j);
    for (int p = 0; p < j; ++p) {
        q128::real v, d;
        hurwitz_at_neg_int(p, a, v, d);
        scale[p] = q128::pow_((q128::real)a, (q128::real)-p);
        tgt[p] = -v * scale[p];
        tgt[j + p] = d * scale[p];
    }
    std::vector<q128::real> u(n);
    for (int k = 0; k < j; ++k) {
        q128::real f = ((q128::real)k + (q128::real)0.5) / j;
        u[k] = q128::log_(a * f * f);
        u[j + k] = (q128::real)a / j * 2 * f;
    }
    auto moments = [&](const std::vector<q128::real>& v, std::vector<q128::real>& F,
                       std::vector<q128::real>* J) {
        for (int p = 0; p < j; ++p) {
            q128::real s0 = 0, s1 = 0;
            for (int k = 0; k < j; ++k) {
                q128::real x = q128::exp_(v[k]), lx = v[k], w = v[j + k];
                q128::real xp = q128::pow_(x, (q128::real)p) * scale[p];
                s0 += w * xp;
                s1 += w * xp * lx;
                if (J) {
                    (*J)[p * n + k] = w * p * xp;
                    (*J)[p * n + j + k] = xp;
                    (*J)[(j + p) * n + k] = w * (p * xp * lx + xp);
                    (*J)[(j + p) * n + j + k] = xp * lx;
                }
            }
            F[p] = s0;
            F[j + p] = s1;
        }
    };
    std::vector<q128::real> b0(n), F(n), Jm(n * n), r(n);
    moments(u, b0, nullptr);
    // Newton from v toward the system with right-hand side rhs(l2); returns the
    // final max-norm residual (or -1 on a failed step).  Path points are
    // accepted at 1e-14 (scaled); the end point is polished until the residual
    // stops decreasing.
    auto newton = [&](std::vector<q128::real>& v, q128::real l2, bool polish) -> q128::real {
        q128::real best = -1;
        std::vector<q128::real> vbest = v;
        for (int it = 0; it < 60; ++it) {
            moments(v, F, &Jm);
            q128::real nr = 0;
            bool finite = true;
            for (int i = 0; i < n; ++i) {
                r[i] = -(F[i] - (b0[i] * (1 - l2) + tgt[i] * l2));
                if (!q128::finite_(r[i])) finite = false;
                if (q128::abs_(r[i]) > nr) nr = q128::abs_(r[i]);
            }
            if (!finite) return -1;
            if (best < 0 || nr < best) {
                best = nr;
                vbest = v;
            } else if (polish) {
                break;   // no further progress at working precision
            }
            if (!polish && nr < (q128::real)1e-24) break;
            if (!solve_ld(Jm, r, n)) return -1;
            q128::real nd = 0;
            for (int i = 0; i < n; ++i) if (q128::abs_(r[i]) > nd) nd = q128::abs_(r[i]);
            if (!(nd <= 1)) return best < (q128::real)1e-24 ? best : -1;
            for (int i = 0; i < n; ++i) v[i] += r[i];
        }
        v = vbest;
        return best;
    };
    q128::real lam = 0, dl = (q128::real)0.01;
    while (lam < 1) {
        q128::real l2 = lam + dl < 1 ? lam + dl : (q128::real)1;
        std::vector<q128::real> v = u;
        q128::real res = newton(v, l2, false);
        if (res >= 0 && res < (q128::real)1e-24) {
            u = v;
            lam = l2;
            dl = dl * (q128::real)1.5 < (q128::real)0.2 ? dl * (q128::real)1.5 : (q128::real)0.2;
        } else {
            dl /= 4;
            if (dl < (q128::real)1e-12) throw std::runtime_error("Alpert rule: homotopy failed");
        }
    }
    if (!(newton(u, (q128::real)1, true) >= 0)) throw std::runtime_error("Alpert rule: final polish failed");
    for (int k = 0; k < j; ++k)
        if (!(u[k] < q128::log_((q128::real)a)) || !(u[j + k] > 0))
            throw std::runtime_error("Alpert rule: nodes outside (0, a) or non-positive weights");
    std::vector<std::pair<double, double>> xw(j);
    for (int k = 0; k < j; ++k) xw[k] = {(double)q128::exp_(u[k]), (double)u[j + k]};
    std::sort(xw.begin(), xw.end());
    cx.resize(j);
    cw.resize(j);
    for (int k = 0; k < j; ++k) {
        cx[k] = xw[k].first;
        cw[k] = xw[k].second;
    }
    cj = j;
    ca = a;
    xo = cx;
    wo = cw;
}

namespace {

// Complete elliptic integrals K(k), E(k) for 0 <= k < 1 given k' = sqrt(1-k^2)
// (arithmetic-geometric mean, in double: the diagonal sums agree with an
// extended-precision evaluation to ~2e-14; the loop stops once a and b agree
// to rounding, before the doubling weight could amplify rounding in c_n).
void ellip_KE(double k2, double kp, double& K, double& E) {
    double a = 1, b = kp, sum = 0.5 * k2, pw = 0.5;
    for (int it = 0; it < 60; ++it) {
        double an = 0.5 * (a + b), bn = std::sqrt(a * b), cn = 0.5 * (a - b);
        pw *= 2;
        sum += pw * cn * cn;
        a = an;
        b = bn;
        if (std::fabs(cn) <= 5e-16 * std::fabs(a)) break;
    }
    K = 3.141592653589793 / (2 * a);
    E = K * (1 - sum);
}

// int_{-pi}^{pi} dG0/dnu' dpsi, unstretched Laplace double layer, mode 0:
// -(1/(pi sqrt(Q))) [A E(k)/d^2 + nu'_rho K(k)/(2 rho')],
// Q = (rho+rho')^2 + dz^2, d^2 = (rho-rho')^2 + dz^2, k^2 = 4 rho rho'/Q,
// A = nu'_rho (rho' - rho) + nu'_z (z' - z) - nu'_rho d^2/(2 rho');
// drho = rho - rho', dzz = z - z' are passed in (accurate separations).
double laplace_dl0(double rho, double rs, double drho, double dzz, double nr, double nz) {
    double dr = drho, dz = dzz;
    double d2 = dr * dr + dz * dz;
    double Q = (rho + rs) * (rho + rs) + dz * dz;
    double k2 = 4.0 * rho * rs / Q, kp = std::sqrt(d2 / Q);
    double K, E;
    ellip_KE(k2, kp, K, E);
    double A = -nr * dr - nz * dz - nr * d2 / (2.0 * rs);
    double v = -(A * E / d2 + nr * K / (2.0 * rs)) / (3.141592653589793 * std::sqrt(Q));
    return v;
}

// Solid angle of the disc {rho' <= Lr, z' = 0} seen from (rho, 0, h), rho < Lr.
double disc_solid_angle(double rho, double hgt, double Lr) {
    if (hgt == 0.0) return 2.0 * kPi;
    const int n = 4096;
    double s = 0;
    for (int i = 0; i < n; ++i) {
        double th = 2.0 * kPi * i / n;
        double sn = rho * std::sin(th);
        double d = -rho * std::cos(th) + std::sqrt(Lr * Lr - sn * sn);
        s += 1.0 - std::fabs(hgt) / std::sqrt(hgt * hgt + d * d);
    }
    return 2.0 * kPi * s / n;
}

}  // namespace

// ---------------------------------------------------------------------------
// All host tables of one problem.
// ---------------------------------------------------------------------------
int build_tables(pmlbie_problem* prob) {
    const pmlbie_params& P = prob->P;
    HostTables& H = prob->H;
    const double Lr = P.a1 + P.T;
    Pml pml{P.a1, P.T, P.S, Lr, P.p};

    // segments
    Curve C;
    C.p = P.p;
    if (P.curve_kind == PMLBIE_CURVE_GAUSS_BUMP) {
        Segment g;
        g.gauss = true;
        g.h = P.bump_h;
        g.w = P.bump_w;
        g.R = P.bump_R;
        C.segs.push_back(g);
        Segment f;
        f.r0 = P.bump_R;
        f.r1 = Lr;
        C.segs.push_back(f);
    } else if (P.curve_kind == PMLBIE_CURVE_WAVY_DENT) {
        Segment d;
        d.p = kConicalP;   // leaves the axis at an angle
        d.wavy = true;
        d.wR = P.wavy_R;
        d.eps = P.wavy_eps;
        d.wm = P.wavy_m;
        C.segs.push_back(d);
        Segment f;
        f.r0 = P.wavy_R;
        f.r1 = Lr;
        C.segs.push_back(f);
    } else {
        const std::vector<double>& V = prob->vertices;
        int nv = (int)V.size() / 2;
        for (int i = 0; i + 1 < nv; ++i) {
            Segment f;
            f.r0 = V[2 * i];
            f.z0 = V[2 * i + 1];
            f.r1 = V[2 * i + 2];
            f.z1 = V[2 * i + 3];
            if (i == 0 && f.z1 != f.z0) f.p = kConicalP;   // leaves the axis at an angle
            C.segs.push_back(f);
        }
        if (std::fabs(V[2 * nv - 2] - Lr) > 1e-14 || std::fabs(V[2 * nv - 1]) > 1e-14) {
            Segment f;
            f.r0 = V[2 * nv - 2];
            f.z0 = V[2 * nv - 1];
            f.r1 = Lr;
            f.z1 = 0;
            C.segs.push_back(f);
        }
    }
    const int nseg = (int)C.segs.size();
    H.N = P.N;
    H.M = P.M;
    H.Nt = P.N + nseg;
    H.h = 1.0 / H.Nt;
    C.Nt = H.Nt;
    C.h = H.h;
    // whole steps per segment, proportional to length, at least 2a + 4
    std::vector<double> len(nseg);
    double tot = 0;
    for (int k = 0; k < nseg; ++k) tot += (len[k] = C.segs[k].length());
    std::vector<int> steps(nseg);
    int sum = 0, imax = 0;
    const int min_steps = 2 * kAlpertA + 4;
    for (int k = 0; k < nseg; ++k) {
        steps[k] = std::max(min_steps, (int)std::lround(H.Nt * len[k] / tot));
        sum += steps[k];
        if (len[k] > len[imax]) imax = k;
    }
    steps[imax] += H.Nt - sum;
    for (int k = 0; k < nseg; ++k)
        if (steps[k] < min_steps) return fail(PMLBIE_EINVAL, "N too small for the curve's segments");
    C.brk.assign(nseg + 1, 0);
    for (int k = 0; k < nseg; ++k) C.brk[k + 1] = C.brk[k] + steps[k];

    // unknowns: non-breakpoint grid nodes
    std::vector<char> isbrk(H.Nt + 1, 0);
    for (int b : C.brk) isbrk[b] = 1;
    H.unk_grid.clear();
    H.unk_of_grid.assign(H.Nt + 1, -1);
    for (int i = 0; i <= H.Nt; ++i)
        if (!isbrk[i]) {
            H.unk_of_grid[i] = (int)H.unk_grid.size();
            H.unk_grid.push_back(i);
        }
    if ((int)H.unk_grid.size() != P.N) return fail(PMLBIE_EINVAL, "internal: unknown count");

    // every quantity of one curve point (node or Alpert correction point)
    struct CP {
        double rho, z, speed, nr, nz, I;
        cd rt, ncr, ncz;
        int bk;            // nearest breakpoint
        double ox, oz;     // offset from it, accurate
    };
    auto fill_point = [&](double t) {
        Curve::Pt q = C.at(t);
        CP c;
        c.rho = q.rho;
        c.z = q.z;
        c.speed = q.speed;
        c.nr = q.nu_r;
        c.nz = q.nu_z;
        c.bk = q.bk;
        c.ox = q.ox;
        c.oz = q.oz;
        c.I = pml.integral(P.a1, c.rho);
        c.rt = cd(c.rho, c.I);
        cd alpha(1.0, pml.sigma(c.rho));
        cd ratio = c.rho > 0 ? c.rt / c.rho : cd(1.0, 0.0);
        c.ncr = c.nr * ratio / alpha;   // nu_rho rho~ alpha_z / (rho alpha_rho), alpha_z = 1
        c.ncz = c.nz * ratio * alpha;   // nu_z rho~ alpha_rho / (rho alpha_z)
        return c;
    };
    // (rho_t - rho_s, z_t - z_s): from breakpoint offsets when both points are
    // nearest to the same breakpoint (close points of a graded cluster)
    auto separation = [](const CP& a, const CP& b, double& dr, double& dz) {
        if (a.bk == b.bk) {
            dr = a.ox - b.ox;
            dz = a.oz - b.oz;
        } else {
            dr = a.rho - b.rho;
            dz = a.z - b.z;
        }
    };

    const int N = P.N;
    H.t.resize(N);
    H.rho.resize(N);
    H.z.resize(N);
    H.speed.resize(N);
    H.nu_r.resize(N);
    H.nu_z.resize(N);
    H.I.resize(N);
    H.Wu.resize(N);
    H.Wphi.resize(N);
    H.rho_t.resize(N);
    H.nuc_r.resize(N);
    H.nuc_z.resize(N);
    std::vector<CP> npts(N);
    H.bk.resize(N);
    H.off.resize(N);
    for (int l = 0; l < N; ++l) {
        double t = H.unk_grid[l] * H.h;
        H.t[l] = t;
        const CP c = npts[l] = fill_point(t);
        H.rho[l] = c.rho;
        H.z[l] = c.z;
        H.speed[l] = c.speed;
        H.nu_r[l] = c.nr;
        H.nu_z[l] = c.nz;
        H.I[l] = c.I;
        H.rho_t[l] = c.rt;
        H.nuc_r[l] = c.ncr;
        H.nuc_z[l] = c.ncz;
        H.bk[l] = c.bk;
        H.off[l] = make_double2(c.ox, c.oz);
        H.Wu[l] = 2.0 * H.rho[l] * H.speed[l];
        H.Wphi[l] = 2.0 * H.rho[l];
    }

    // Alpert rule and correction points
    try {
        alpert_log_rule(kAlpertJ, kAlpertA, H.ax, H.aw);
    } catch (const std::exception& e) {
        return fail(PMLBIE_EINVAL, e.what());
    }
    H.corr_target.clear();
    H.corr_tau.clear();
    H.corr_m.clear();
    H.corr_coef.clear();
    std::vector<CP> cpts;
    for (int l = 0; l < N; ++l) {
        for (int sg = -1; sg <= 1; sg += 2) {
            for (int k = 0; k < kAlpertJ; ++k) {
                double tau = H.unk_grid[l] * H.h + sg * H.ax[k] * H.h;
                if (tau <= 0.0 || tau >= 1.0) continue;
                int i0 = (int)std::floor(tau / H.h) - (kStencil / 2 - 1);
                i0 = std::min(std::max(i0, 0), H.Nt + 1 - kStencil);
                for (int a = 0; a < kStencil; ++a) {
                    double ta = (i0 + a) * H.h, Lv = 1.0;
                    for (int b = 0; b < kStencil; ++b)
                        if (b != a) Lv *= (tau - (i0 + b) * H.h) / (ta - (i0 + b) * H.h);
                    int m = H.unk_of_grid[i0 + a];
                    H.corr_m.push_back(m);
                    H.corr_coef.push_back(m >= 0 ? H.aw[k] * H.h * Lv : 0.0);
                }
                H.corr_target.push_back(l);
                H.corr_tau.push_back(tau);
            }
        }
    }
    const int ncorr = (int)H.corr_target.size();
    // correction points by target (they come ordered by target) and the
    // column window of each target's stencils, for the per-target assembly
    H.corr_start.assign(N + 1, 0);
    H.corr_cmin.assign(N, 0);
    H.corr_w.assign(N, 0);
    H.corr_wmax = 0;
    for (int c = 0; c < ncorr; ++c) H.corr_start[H.corr_target[c] + 1]++;
    for (int l = 0; l < N; ++l) H.corr_start[l + 1] += H.corr_start[l];
    for (int l = 0; l < N; ++l) {
        int lo = N, hi = -1;
        for (int c = H.corr_start[l]; c < H.corr_start[l + 1]; ++c)
            for (int a = 0; a < kStencil; ++a) {
                const int m = H.corr_m[(size_t)c * kStencil + a];
                if (m >= 0) lo = std::min(lo, m), hi = std::max(hi, m);
            }
        H.corr_cmin[l] = hi >= lo ? lo : 0;
        H.corr_w[l] = hi >= lo ? hi - lo + 1 : 0;
        H.corr_wmax = std::max(H.corr_wmax, H.corr_w[l]);
    }
    // the points themselves (curve, PML integral and conormal of each) in parallel
    cpts.resize(ncorr);
    parallel_rows(ncorr, [&](int lo, int hi) {
        for (int c = lo; c < hi; ++c) cpts[c] = fill_point(H.corr_tau[c]);
    });

    // pair classes and close-pair table
    const double eta = prob->eta_split;
    auto pair_sep = [&](const CP& tg, const CP& src, double& dr, double& dz, double& dI) {
        separation(tg, src, dr, dz);
        dI = (tg.rho > P.a1 || src.rho > P.a1) ? pml.delta(src.rho, dr, tg.I, src.I) : 0.0;
    };
    auto make_pair_sep = [&](int l, const CP& src, NearPair& np, double dr, double dz, double dI) -> bool {
        const CP& tg = npts[l];
        cd drt(dr, dI);                   // rho~ - rho~'
        cd d2 = drt * drt + dz * dz;
        cd rr = tg.rt * src.rt;
        cd x = d2 / rr;
        double re_sqrt = std::sqrt(std::max(0.5 * (std::abs(x) + x.real()), 0.0));
        np.d2 = make_double2(d2.real(), d2.imag());
        np.rr = make_double2(rr.real(), rr.imag());
        np.rho_t = make_double2(tg.rt.real(), tg.rt.imag());
        np.rho_s = make_double2(src.rt.real(), src.rt.imag());
        np.drt = make_double2(-drt.real(), -drt.imag());
        np.nuc_r = make_double2(src.ncr.real(), src.ncr.imag());
        np.nuc_z = make_double2(src.ncz.real(), src.ncz.imag());
        np.dz = dz;
        np.tgt = l;
        np.flags = (!P.subst_off && (tg.I > 0 || src.I > 0)) ? kFlagSubst : 0;
        return re_sqrt < eta;
    };
    auto make_pair = [&](int l, const CP& src, NearPair& np) -> bool {
        double dr, dz, dI;
        pair_sep(npts[l], src, dr, dz, dI);
        return make_pair_sep(l, src, np, dr, dz, dI);
    };
    // The same criterion in real arithmetic (x = d~^2 / (rho~ rho~'): |x| and
    // Re x without the complex division), used only to skip the pairs whose
    // value exceeds the split threshold by 1 % -- far beyond any rounding
    // difference, so every pair near the threshold still takes make_pair's test.
    auto clearly_far = [&](int l, const CP& src, double dr, double dz, double dI) -> bool {
        const CP& tg = npts[l];
        const double a = dr * dr - dI * dI + dz * dz, b = 2.0 * dr * dI;          // d~^2
        const std::complex<double> rr = tg.rt * src.rt;
        const double c = rr.real(), d = rr.imag(), nr2 = c * c + d * d;
        if (!(nr2 > 0.0)) return false;
        const double re_x = (a * c + b * d) / nr2, abs_x = std::sqrt((a * a + b * b) / nr2);
        const double v2 = 0.5 * (abs_x + re_x);                                   // (Re sqrt x)^2
        return std::isfinite(v2) && v2 > 1.0201 * eta * eta;
    };
    H.cls.assign((size_t)N * N, kFar);
    H.near.clear();
    {
        int nt = std::max(1, std::min((int)std::thread::hardware_concurrency(), 64));
        std::vector<std::vector<NearPair>> part(nt);
        int chunk = (N + nt - 1) / nt;
        std::vector<std::thread> th;
        for (int t = 0; t < nt; ++t) {
            int lo = t * chunk, hi = std::min(N, lo + chunk);
            if (lo >= hi) break;
            th.emplace_back([&, t, lo, hi] {
                for (int l = lo; l < hi; ++l)
                    for (int m = 0; m < N; ++m) {
                        if (std::abs(H.unk_grid[l] - H.unk_grid[m]) < kAlpertA) {
                            H.cls[(size_t)l * N + m] = kSkip;
                            continue;
                        }
                        double dr, dz, dI;
                        pair_sep(npts[l], npts[m], dr, dz, dI);
                        if (clearly_far(l, npts[m], dr, dz, dI)) continue;
                        NearPair np;
                        if (make_pair_sep(l, npts[m], np, dr, dz, dI)) {
                            np.src = m;
                            H.cls[(size_t)l * N + m] = kNear;
                            part[t].push_back(np);
                        }
                    }
            });
        }
        for (auto& x : th) x.join();
        for (auto& v : part) H.near.insert(H.near.end(), v.begin(), v.end());
    }
    H.n_grid_near = (int)H.near.size();
    {
        // mirror pairs: the exact modal Laplace kernels depend on the pair only
        // through chi (symmetric) and the normal factor, so one recurrence
        // serves both orientations.  The grid list is ordered by (target,
        // source): row starts, then a binary search of source l in row m.
        const int ng = H.n_grid_near;
        auto before = [](const NearPair& a, const NearPair& b) {
            return a.tgt < b.tgt || (a.tgt == b.tgt && a.src < b.src);
        };
        if (!std::is_sorted(H.near.begin(), H.near.begin() + ng, before))
            std::sort(H.near.begin(), H.near.begin() + ng, before);
        std::vector<int> row(N + 1, 0);
        for (int i = 0; i < ng; ++i) ++row[H.near[i].tgt + 1];
        for (int l = 0; l < N; ++l) row[l + 1] += row[l];
        std::vector<int> srcs(ng);
        for (int i = 0; i < ng; ++i) srcs[i] = H.near[i].src;
        parallel_rows(ng, [&](int lo, int hi) {
            for (int i = lo; i < hi; ++i) {
                const int l = H.near[i].tgt, m = H.near[i].src;
                const int* b = srcs.data() + row[m];
                const int* e = srcs.data() + row[m + 1];
                const int* it = std::lower_bound(b, e, l);
                H.near[i].mirror = (it != e && *it == l) ? (int)(it - srcs.data()) : -1;
            }
        });
    }
    H.near.resize((size_t)H.n_grid_near + ncorr);
    parallel_rows(ncorr, [&](int lo, int hi) {
        for (int c = lo; c < hi; ++c) {
            NearPair np;
            bool nr = make_pair(H.corr_target[c], cpts[c], np);
            np.src = c;
            np.flags |= kFlagCorr | (nr ? 0 : kFlagFar);
            H.near[(size_t)H.n_grid_near + c] = np;
        }
    });
    {
        // Close pairs whose exact modal Laplace kernels a thread computes: not
        // far by the criterion, and of a pair and its mirror the lower index.
        // Ordered so that a warp holds pairs of one arithmetic class (real:
        // both points physical; complex otherwise) and of similar recurrence
        // length (upward: M steps; Miller: M + 20 / Re(eta)): a warp's FP64
        // instruction costs the same issue slot whatever its active lanes.
        const int np = (int)H.near.size();
        auto cx_zero = [](double2 v) { return v.y == 0.0; };
        // keys in pair order (-1: not a leader), computed in parallel
        std::vector<long long> kp(np, -1);
        parallel_rows(np, [&](int lo, int hi) {
            for (int p = lo; p < hi; ++p) {
                const NearPair& q = H.near[p];
                if (q.flags & kFlagFar) continue;
                if (q.mirror >= 0 && q.mirror < p) continue;
                bool real = cx_zero(q.d2) && cx_zero(q.rr) && cx_zero(q.rho_t) && cx_zero(q.rho_s) &&
                            cx_zero(q.drt) && cx_zero(q.nuc_r) && cx_zero(q.nuc_z);
                if (real && q.mirror >= 0)
                    real = cx_zero(H.near[q.mirror].nuc_r) && cx_zero(H.near[q.mirror].nuc_z);
                // Re acosh(chi), chi - 1 = d~^2 / (2 rho~ rho~')
                const std::complex<double> d2(q.d2.x, q.d2.y), rr(q.rr.x, q.rr.y);
                const std::complex<double> chim1 = d2 / (2.0 * rr), chi = 1.0 + chim1;
                const double reeta = std::fabs(std::log(chi + std::sqrt(chim1) * std::sqrt(chi + 1.0)).real());
                long long steps = P.M;
                if (!(reeta * P.M < kRecUpward) && reeta > 0.0) steps += (long long)std::ceil(20.0 / reeta);
                kp[p] = (real ? 0LL : (1LL << 40)) + steps;
            }
        });
        std::vector<std::pair<long long, int>> key;
        key.reserve(np);
        for (int p = 0; p < np; ++p)
            if (kp[p] >= 0) key.push_back({kp[p], p});
        std::stable_sort(key.begin(), key.end(),
                         [](const std::pair<long long, int>& a, const std::pair<long long, int>& b) {
                             return a.first < b.first;
                         });
        H.near_lead.resize(key.size());
        for (size_t i = 0; i < key.size(); ++i) H.near_lead[i] = key[i].second;
    }

    // diagonal term: K0_AB 1 by the same quadrature (mode-0 Laplace double layer,
    // physical normal), plus K0_+ 1 from the disc solid angle (Lemma 3.3)
    H.Da.assign(N, 0.0);
    H.Db.assign(N, 0.0);
    std::vector<double> K0(N, 0.0);
    parallel_rows(N, [&](int lo, int hi) {
        for (int l = lo; l < hi; ++l) {
            double s = 0;
            for (int m = 0; m < N; ++m) {
                if (H.cls[(size_t)l * N + m] == kSkip) continue;
                double dr, dz;
                separation(npts[l], npts[m], dr, dz);
                s += H.h * H.Wu[m] * laplace_dl0(H.rho[l], H.rho[m], dr, dz, H.nu_r[m], H.nu_z[m]);
            }
            K0[l] = s;
        }
    });
    // correction kernels in parallel; their sums in the serial order
    std::vector<double> vc(ncorr);
    parallel_rows(ncorr, [&](int lo, int hi) {
        for (int c = lo; c < hi; ++c) {
            const int l = H.corr_target[c];
            const CP& q = cpts[c];
            double dr, dz;
            separation(npts[l], q, dr, dz);
            vc[c] = laplace_dl0(H.rho[l], q.rho, dr, dz, q.nr, q.nz);
        }
    });
    for (int c = 0; c < ncorr; ++c) {
        const int l = H.corr_target[c];
        const double v = vc[c];
        for (int a = 0; a < kStencil; ++a) {
            int m = H.corr_m[(size_t)c * kStencil + a];
            if (m >= 0) K0[l] += H.corr_coef[(size_t)c * kStencil + a] * H.Wu[m] * v;
        }
    }
    parallel_rows(N, [&](int lo, int hi) {
        for (int l = lo; l < hi; ++l) {
            double Od = disc_solid_angle(H.rho[l], H.z[l], Lr);
            double Op = H.z[l] > 0 ? 4.0 * kPi - Od : (H.z[l] < 0 ? Od : 2.0 * kPi);
            H.Da[l] = K0[l] - Op / (2.0 * kPi);
            H.Db[l] = -K0[l] - (4.0 * kPi - Op) / (2.0 * kPi);
        }
    });
    return PMLBIE_OK;
}

}  // namespace pmlbie
