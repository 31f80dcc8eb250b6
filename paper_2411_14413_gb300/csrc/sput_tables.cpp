// sput_tables.cpp -- FP64 host construction of the interaction tables.
//
// The tables hold the parts of the transport that are smooth functions of one
// variable and too costly to solve per collision on the device:
//   * b_max(eps)/a: impact parameter whose CM deflection equals chi_min, in
//     reduced Moliere units (eps = a E_r / (Z1 Z2 e^2)); the cross section is
//     sigma = pi b_max^2 (angle cut-off of the screened-Coulomb interaction,
//     Sec. "The SIMTRA model");
//   * the head-on apsis x_h(eps), root of Phi(x) = eps x, a lower bound that
//     starts the device's Newton iteration for the closest approach;
//   * K(v) = <sigma(g) g> over a Maxwellian gas at T, so that the mean free
//     path is lambda_m(v) = v / (n_g K(v)) (velocity-dependent lambda_m of the
//     Eq. for lambda, gas in thermal equilibrium);
//   * M(v) = max_{g <= v + 6 s} sigma(g) g, the bound of the partner rejection;
//   * first guesses for the racetrack inverse CDF.
// Everything here is double precision; the device receives FP32 cubic pieces.
#include "sput_tables.h"

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <thread>

#include "sput_internal.h"

namespace sput {

namespace {

constexpr double kC[3] = {0.35, 0.55, 0.10};
constexpr double kD[3] = {0.3, 1.2, 6.0};

// Gauss-Mehler: N = 256 nodes on [-1,1], 128 evaluations by symmetry.
constexpr int kHostGM = 128;
struct GMNodes {
    double u[kHostGM], inv1pu[kHostGM], uo[kHostGM], r[kHostGM];
    GMNodes()
    {
        const int N = 2 * kHostGM;
        for (int j = 0; j < kHostGM; ++j) {
            double th = (2.0 * (j + 1) - 1.0) * kPi / (2.0 * N);
            double c = std::cos(th), s = std::sin(th);
            u[j] = c;
            inv1pu[j] = 1.0 / (1.0 + c);
            uo[j] = c / (s * s);
            r[j] = 2.0 * std::sin(0.5 * th) * std::sin(0.5 * th) / c;  // 1/u - 1
        }
    }
};
const GMNodes& gm_nodes()
{
    static const GMNodes g;
    return g;
}

double phi(double x) { return kC[0] * std::exp(-kD[0] * x) + kC[1] * std::exp(-kD[1] * x) + kC[2] * std::exp(-kD[2] * x); }

// Gauss-Legendre nodes on [-1,1] (Newton on P_n).
struct GL {
    std::vector<double> x, w;
    explicit GL(int n) : x(n), w(n)
    {
        for (int i = 0; i < n; ++i) {
            double z = std::cos(kPi * (i + 0.75) / (n + 0.5)), dp = 1.0;
            for (int it = 0; it < 100; ++it) {
                double p0 = 1.0, p1 = z;
                for (int k = 2; k <= n; ++k) {
                    double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                    p0 = p1;
                    p1 = p2;
                }
                dp = n * (z * p1 - p0) / (z * z - 1.0);
                double dz = p1 / dp;
                z -= dz;
                if (std::fabs(dz) < 1e-16) break;
            }
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            x[i] = z;
            w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
        }
    }
};
const GL& gl24()
{
    static const GL g(24);
    return g;
}

}  // namespace

float4 cubic_from_thirds(double f0, double f1, double f2, double f3)
{
    // Newton forward differences on t = 0, 1/3, 2/3, 1 expanded in powers of t
    double d1 = f1 - f0, d2 = f2 - 2.0 * f1 + f0, d3 = f3 - 3.0 * f2 + 3.0 * f1 - f0;
    return make_float4((float)f0, (float)(3.0 * d1 - 1.5 * d2 + d3), (float)(4.5 * d2 - 4.5 * d3), (float)(4.5 * d3));
}

double head_on_apsis64(double eps)
{
    // Phi(x) = eps x has one root in (0, 1/eps]; bisection in ln x
    double lo = std::log(1e-12), hi = std::log(1.0 / eps) + 1e-9;
    for (int it = 0; it < 200; ++it) {
        double m = 0.5 * (lo + hi), x = std::exp(m);
        if (phi(x) > eps * x) lo = m;
        else hi = m;
        if (hi - lo < 1e-15) break;
    }
    return std::exp(0.5 * (lo + hi));
}

double apsis64(double eps, double beta)
{
    // root of g(x) = 1 - beta^2/x^2 - Phi(x)/(eps x): increasing and concave, so
    // Newton from the lower bound max(beta, x_h) approaches monotonically
    double x = std::max(beta, head_on_apsis64(eps));
    for (int it = 0; it < 200; ++it) {
        double e0 = kC[0] * std::exp(-kD[0] * x), e1 = kC[1] * std::exp(-kD[1] * x), e2 = kC[2] * std::exp(-kD[2] * x);
        double ph = e0 + e1 + e2, dph = -(kD[0] * e0 + kD[1] * e1 + kD[2] * e2);
        double g = 1.0 - beta * beta / (x * x) - ph / (eps * x);
        double gp = 2.0 * beta * beta / (x * x * x) - (dph * x - ph) / (x * x * eps);
        double dx = g / gp;
        x -= dx;
        if (std::fabs(dx) <= 1e-15 * x) break;
    }
    return x;
}

double chi_moliere64(double eps, double beta)
{
    if (beta <= 0.0) return kPi;
    const GMNodes& G = gm_nodes();
    double x0 = apsis64(eps, beta);
    double bt = beta / x0;
    double pref[3];
    for (int i = 0; i < 3; ++i) pref[i] = kC[i] * std::exp(-kD[i] * x0) / (eps * x0);
    // chi = (2 pi / N) sum_j D_j / (S_j (S_j + bt)), S_j = sqrt(bt^2 + D_j): the
    // Gauss-Mehler sum of pi - 2 bt int_0^1 du / sqrt(1-u^2) / sqrt(bt^2 + D(u)),
    // D(u) = [V(r0) - V(r0/u)] / (E_r (1 - u^2)), written without cancellation
    double s = 0.0;
    for (int j = 0; j < kHostGM; ++j) {
        double D = 0.0;
        for (int i = 0; i < 3; ++i) {
            double y = kD[i] * x0 * G.r[j];
            D += pref[i] * (G.inv1pu[j] + G.uo[j] * (-std::expm1(-y)));
        }
        double S = std::sqrt(bt * bt + D);
        s += D / (S * (S + bt));
    }
    return 2.0 * kPi / (2.0 * kHostGM) * s;
}

static double bmax64(double eps, double chi_min)
{
    // chi decreases monotonically with beta from pi to 0
    double lo = 0.0, hi = std::max(1.0, head_on_apsis64(eps));
    while (chi_moliere64(eps, hi) > chi_min) {
        lo = hi;
        hi *= 2.0;
    }
    double flo = (lo > 0.0 ? chi_moliere64(eps, lo) : kPi) - chi_min, fhi = chi_moliere64(eps, hi) - chi_min;
    for (int it = 0; it < 200 && hi - lo > 1e-14 * hi; ++it) {
        // secant step clipped to the bracket, bisection every third step
        double m = (it % 3 == 2) ? 0.5 * (lo + hi) : (lo * fhi - hi * flo) / (fhi - flo);
        if (!(m > lo && m < hi)) m = 0.5 * (lo + hi);
        double fm = chi_moliere64(eps, m) - chi_min;
        if (fm == 0.0) return m;
        if (fm > 0.0) {
            lo = m;
            flo = fm;
        } else {
            hi = m;
            fhi = fm;
        }
    }
    return 0.5 * (lo + hi);
}

double BmaxTable::eval(double ln_eps) const
{
    double x = (ln_eps - lo) / h;
    if (x <= 0.0) x = 0.0;
    if (x >= n) x = n;
    int i = std::min((int)x, n - 1);
    double t = x - i;
    const double* f = &third[3 * i];
    double d1 = f[1] - f[0], d2 = f[2] - 2.0 * f[1] + f[0], d3 = f[3] - 3.0 * f[2] + 3.0 * f[1] - f[0];
    double c1 = 3.0 * d1 - 1.5 * d2 + d3, c2 = 4.5 * d2 - 4.5 * d3, c3 = 4.5 * d3;
    return f[0] + t * (c1 + t * (c2 + t * c3));
}

const BmaxTable& bmax_table(double chi_min)
{
    static std::mutex mu;
    static std::map<double, BmaxTable*> cache;
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(chi_min);
    if (it != cache.end()) return *it->second;
    BmaxTable* T = new BmaxTable();
    T->chi_min = chi_min;
    T->n = (int)std::lround((6.0 - T->lo) / T->h);
    int m = 3 * T->n + 1;
    T->third.assign(m, 0.0);
    T->xh.assign(T->n + 1, 0.0f);
    unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; ++t)
        th.emplace_back([T, m, nt, t, chi_min]() {
            for (int j = (int)t; j < m; j += (int)nt) T->third[j] = bmax64(std::exp(T->lo + T->h * j / 3.0), chi_min);
        });
    for (auto& x : th) x.join();
    T->cubic.resize(T->n);
    for (int i = 0; i < T->n; ++i) {
        const double* f = &T->third[3 * i];
        T->cubic[i] = cubic_from_thirds(f[0], f[1], f[2], f[3]);
    }
    for (int i = 0; i <= T->n; ++i) T->xh[i] = (float)head_on_apsis64(std::exp(T->lo + T->h * i));
    cache[chi_min] = T;
    return *T;
}

PairPhys make_pair(double Z1, double m1, double Z2, double m2, int hard_sphere, double hs_d, double chi_min)
{
    PairPhys p;
    p.Z1 = Z1;
    p.Z2 = Z2;
    p.m1 = m1;
    p.m2 = m2;
    // Firsov screening length
    p.a = 0.8853 * kBohrA * std::pow(std::sqrt(Z1) + std::sqrt(Z2), -2.0 / 3.0);
    p.zze2 = Z1 * Z2 * kE2EVA;
    double mu = m1 * m2 / (m1 + m2);
    // E_r = mu g^2 / 2 (eV with g in km/s); eps = a E_r / (Z1 Z2 e^2)
    p.kappa = p.a * 0.5 * mu * kEnergyUnit / p.zze2;
    p.hard_sphere = hard_sphere;
    p.hs_d = hs_d;
    p.chi_min = chi_min;
    return p;
}

double sigma64(const PairPhys& pp, const BmaxTable* bt, double g)
{
    if (pp.hard_sphere) return kPi * pp.hs_d * pp.hs_d;
    double eps = pp.kappa * g * g;
    double b = bt->eval(std::log(std::max(eps, 1e-300))) * pp.a;
    return kPi * b * b;
}

// density of the relative speed g = |v - V| for V Maxwellian with per-axis std s
static double rel_pdf(double g, double v, double s)
{
    const double c = 1.0 / (s * std::sqrt(2.0 * kPi));
    if (v < 1e-9 * s) return 2.0 * g * g * c / (s * s) * std::exp(-g * g / (2.0 * s * s));
    double a = (g - v) / s;
    return g / v * c * std::exp(-0.5 * a * a) * (-std::expm1(-2.0 * g * v / (s * s)));
}

double K64(const PairPhys& pp, const BmaxTable* bt, double s, int thermal, double v)
{
    if (!thermal) return sigma64(pp, bt, v) * v;
    const GL& G = gl24();
    double a = std::max(0.0, v - 10.0 * s), b = v + 10.0 * s;
    const int panels = 8;
    double sum = 0.0;
    for (int p = 0; p < panels; ++p) {
        double x0 = a + (b - a) * p / panels, x1 = a + (b - a) * (p + 1) / panels;
        double hm = 0.5 * (x1 - x0), mm = 0.5 * (x1 + x0);
        for (size_t i = 0; i < G.x.size(); ++i) {
            double g = mm + hm * G.x[i];
            sum += hm * G.w[i] * sigma64(pp, bt, g) * g * rel_pdf(g, v, s);
        }
    }
    return sum;
}

int h_monotone(const PairPhys& pp, const BmaxTable* bt, double g_top)
{
    double prev = 0.0;
    for (int j = 1; j <= 4000; ++j) {
        double g = g_top * j / 4000.0, hv = sigma64(pp, bt, g) * g;
        if (hv < prev) return 0;
        prev = hv;
    }
    return 1;
}

double M64(const PairPhys& pp, const BmaxTable* bt, double s, double v, int monotone)
{
    double G = v + kMajorantSigmas * s;
    double m = sigma64(pp, bt, G) * G;
    if (monotone) return m;
    for (int j = 1; j < 4000; ++j) {
        double g = G * j / 4000.0;
        m = std::max(m, sigma64(pp, bt, g) * g);
    }
    return m;
}

void build_w_tables(const PairPhys& pp, const BmaxTable* bt, double s, int thermal, double v_top, double h_w,
                    std::vector<float4>& K, std::vector<float4>& M, std::vector<float4>& G, int& n_w)
{
    double w_top = std::log1p(v_top / s);
    n_w = std::max(4, (int)std::ceil(w_top / h_w));
    int mono = h_monotone(pp, bt, v_top + 20.0 * s);
    std::vector<double> kv(3 * n_w + 1), mv(3 * n_w + 1), gv(3 * n_w + 1);
    unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; ++t)
        th.emplace_back([&, t]() {
            for (int j = (int)t; j < 3 * n_w + 1; j += (int)nt) {
                double v = s * std::expm1(h_w * j / 3.0);
                // stationary gas: tabulate sigma(v) = K(v)/v, so that the inverse mean free
                // path n sigma(v) stays finite when the speed decays towards zero
                kv[j] = thermal ? K64(pp, bt, s, 1, v) : sigma64(pp, bt, v);
                mv[j] = thermal ? M64(pp, bt, s, v, mono) : 0.0;
                // d ln K / d ln s at fixed v by a central difference in s (gas at rest: 0)
                const double hs = 1e-4;
                gv[j] = thermal ? (K64(pp, bt, s * (1.0 + hs), 1, v) - K64(pp, bt, s * (1.0 - hs), 1, v)) /
                                      (2.0 * hs * kv[j])
                                : 0.0;
            }
        });
    for (auto& x : th) x.join();
    K.resize(n_w);
    M.resize(n_w);
    G.resize(n_w);
    for (int i = 0; i < n_w; ++i) {
        K[i] = cubic_from_thirds(kv[3 * i], kv[3 * i + 1], kv[3 * i + 2], kv[3 * i + 3]);
        M[i] = cubic_from_thirds(mv[3 * i], mv[3 * i + 1], mv[3 * i + 2], mv[3 * i + 3]);
        G[i] = cubic_from_thirds(gv[3 * i], gv[3 * i + 1], gv[3 * i + 2], gv[3 * i + 3]);
    }
}

double sigma_m64(const PairPhys& pp, const BmaxTable* bt, double g)
{
    if (pp.hard_sphere) return kPi * pp.hs_d * pp.hs_d;  // isotropic CM scattering: sigma_m = sigma
    // 1 - cos chi = 2 sin^2(chi/2) over beta = b/a, out to where chi < 1e-9 rad
    const double eps = std::max(pp.kappa * g * g, 1e-40);
    double B = std::max(1.0, bt->eval(std::log(eps)));
    while (chi_moliere64(eps, B) > 1e-9 && B < 1e4) B *= 1.5;
    const GL& G = gl24();
    const int panels = 24;
    double sum = 0.0;
    for (int p = 0; p < panels; ++p) {
        double x0 = B * p / panels, x1 = B * (p + 1) / panels;
        double hm = 0.5 * (x1 - x0), mm = 0.5 * (x1 + x0);
        for (size_t i = 0; i < G.x.size(); ++i) {
            double beta = mm + hm * G.x[i];
            double sh = std::sin(0.5 * chi_moliere64(eps, beta));
            sum += hm * G.w[i] * 2.0 * sh * sh * beta;
        }
    }
    return 2.0 * kPi * pp.a * pp.a * sum;
}

double sigma_D64(const PairPhys& pp, const BmaxTable* bt, double T)
{
    const double kT = kBoltzmannJ * T;
    const double mu = pp.m1 * pp.m2 / (pp.m1 + pp.m2) * kAmuKg;        // kg
    const double g_per_y = std::sqrt(2.0 * kT / mu) * 1e-3;             // km/s per unit y
    // Omega11 / sqrt(kT/(2 pi mu)) = int_0^inf e^{-y^2} y^5 sigma_m dy on [0, 6] (Angstrom^2;
    // the rest of the range weighs below 1e-12)
    const GL& G = gl24();
    const int panels = 8;
    double I = 0.0;
    for (int p = 0; p < panels; ++p) {
        double y0 = 6.0 * p / panels, y1 = 6.0 * (p + 1) / panels;
        double hm = 0.5 * (y1 - y0), mm = 0.5 * (y1 + y0);
        for (size_t i = 0; i < G.x.size(); ++i) {
            double y = mm + hm * G.x[i];
            I += hm * G.w[i] * std::exp(-y * y) * std::pow(y, 5) * sigma_m64(pp, bt, y * g_per_y);
        }
    }
    const double omega = std::sqrt(kT / (2.0 * kPi * mu)) * I;          // Angstrom^2 m/s
    const double vbar1 = std::sqrt(8.0 * kT / (kPi * pp.m1 * kAmuKg));  // m/s
    return 16.0 * mu * vbar1 * omega / (9.0 * kT);                       // Angstrom^2
}

double racetrack_F64(double r0, double sg, double r)
{
    // integral of rho exp(-(rho-r0)^2/(2 sg^2)) over [0, r]
    double k = 1.0 / (sg * std::sqrt(2.0));
    return sg * sg * (std::exp(-r0 * r0 * k * k) - std::exp(-(r - r0) * (r - r0) * k * k)) +
           r0 * sg * std::sqrt(kPi / 2.0) * (std::erf((r - r0) * k) + std::erf(r0 * k));
}

void racetrack_table(double r0, double sg, double R, int n, float4* out)
{
    // Inverse of the radial CDF as cubic pieces: n pieces in s = sqrt(u) on
    // [0, sqrt(1/2)] (lower half), then n pieces in q = sqrt(1-u) on the same
    // interval (upper half); each piece interpolates four exact inverses.
    const double FR = racetrack_F64(r0, sg, R), half = std::sqrt(0.5);
    auto inv = [&](double u) {
        double tgt = u * FR, lo = 0.0, hi = R;
        for (int it = 0; it < 200 && hi - lo > 1e-15 * R; ++it) {
            double m = 0.5 * (lo + hi);
            if (racetrack_F64(r0, sg, m) < tgt) lo = m;
            else hi = m;
        }
        return 0.5 * (lo + hi);
    };
    for (int side = 0; side < 2; ++side)
        for (int i = 0; i < n; ++i) {
            double f[4];
            for (int j = 0; j < 4; ++j) {
                double x = half * (i + j / 3.0) / n;
                f[j] = inv(side ? 1.0 - x * x : x * x);
            }
            out[side * n + i] = cubic_from_thirds(f[0], f[1], f[2], f[3]);
        }
}

}  // namespace sput
