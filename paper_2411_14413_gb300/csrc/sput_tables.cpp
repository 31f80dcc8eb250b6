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
//   * the partner envelope A(v), B(v): the line A + B rho (rho = |V|/s) on the
//     upper concave hull of H(rho) = max sigma(g) g over the relative speeds a
//     partner of speed rho s can give, which bounds the rejection's weight;
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

namespace {

// Slopes of the C2 cubic spline through (t_i, f_i), i < n (n >= 4), with the end
// slopes of the cubic through the four end nodes; t strictly increasing.
void spline_slopes(const double* t, const double* f, int n, double* s)
{
    auto end_slope = [](const double* tt, const double* ff, int at) {
        // derivative at tt[at] of the Lagrange cubic through the four points
        double d = 0.0;
        for (int k = 0; k < 4; ++k) {
            double num = 0.0, den = 1.0;
            for (int m = 0; m < 4; ++m)
                if (m != k) den *= tt[k] - tt[m];
            for (int m = 0; m < 4; ++m) {
                if (m == k) continue;
                double prod = 1.0;
                for (int r = 0; r < 4; ++r)
                    if (r != k && r != m) prod *= tt[at] - tt[r];
                num += prod;
            }
            d += ff[k] * num / den;
        }
        return d;
    };
    s[0] = end_slope(t, f, 0);
    s[n - 1] = end_slope(t + n - 4, f + n - 4, 3);
    // h_i s_{i-1} + 2 (h_{i-1} + h_i) s_i + h_{i-1} s_{i+1} = 3 (h_i d_{i-1} + h_{i-1} d_i)
    std::vector<double> a(n), b(n), c(n), r(n);
    for (int i = 1; i < n - 1; ++i) {
        const double h0 = t[i] - t[i - 1], h1 = t[i + 1] - t[i];
        const double d0 = (f[i] - f[i - 1]) / h0, d1 = (f[i + 1] - f[i]) / h1;
        a[i] = h1;
        b[i] = 2.0 * (h0 + h1);
        c[i] = h0;
        r[i] = 3.0 * (h1 * d0 + h0 * d1);
    }
    r[1] -= a[1] * s[0];
    r[n - 2] -= c[n - 2] * s[n - 1];
    for (int i = 2; i < n - 1; ++i) {  // Thomas elimination
        const double w = a[i] / b[i - 1];
        b[i] -= w * c[i - 1];
        r[i] -= w * r[i - 1];
    }
    s[n - 2] = r[n - 2] / b[n - 2];
    for (int i = n - 3; i >= 1; --i) s[i] = (r[i] - c[i] * s[i + 1]) / b[i];
}

}  // namespace

bool ChiTable::eval(double ln_eps, double ln_s, double& q) const
{
    const double fx = (ln_eps - kChiX0) / kChiHx;
    if (!(fx >= 0.0 && fx < kChiNx) || !(ln_s >= kChiY0) || ln_s > 0.0) return false;
    const int i = std::min((int)fx, kChiNx - 1);
    const double tx = fx - i;
    int j;
    double ty;
    if (ln_s < kChiY1) {
        const double fy = (ln_s - kChiY0) / kChiHyC;
        j = std::min((int)fy, kChiNyC - 1);
        ty = fy - j;
    } else {
        const double fy = (ln_s - kChiY1) / kChiHyF;
        j = std::min((int)fy, kChiNyF - 1);
        ty = fy - j;
        j += kChiNyC;
    }
    const double* a = &a64[16 * ((size_t)i * kChiNy + j)];
    double p = 0.0;
    for (int k = 3; k >= 0; --k) {
        const double ck = a[4 * k] + ty * (a[4 * k + 1] + ty * (a[4 * k + 2] + ty * a[4 * k + 3]));
        p = p * tx + ck;
    }
    q = p;
    return true;
}

const ChiTable& chi_table(double chi_min)
{
    static std::mutex mu;
    static std::map<double, ChiTable*> cache;
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(chi_min);
    if (it != cache.end()) return *it->second;
    // nodes of the table's cells plus kExt more on every side: the splines' end
    // slopes then fall outside the stored cells (y > 0 is b > b_max, chi < chi_min)
    constexpr int kExt = 4;
    const int NX = kChiNx + 1 + 2 * kExt, NY = kChiNy + 1 + 2 * kExt;
    std::vector<double> X(NX), Y(NY);
    for (int i = 0; i < NX; ++i) X[i] = kChiX0 + (double)kChiHx * (i - kExt);
    for (int j = 0; j < NY; ++j) {
        const int k = j - kExt;  // node index of the table's own grid
        Y[j] = k <= kChiNyC ? kChiY0 + (double)kChiHyC * k : kChiY1 + (double)kChiHyF * (k - kChiNyC);
    }
    const int j_zero = kExt + kChiNy;  // the node y = 0, b = b_max
    // node values q = ln tan(chi/2) at b = b_max(eps) e^y, rows of x in parallel
    std::vector<double> Q((size_t)NX * NY), Qx(Q.size()), Qy(Q.size()), Qxy(Q.size());
    unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; ++t)
        th.emplace_back([&, t]() {
            for (int i = (int)t; i < NX; i += (int)nt) {
                const double eps = std::exp(X[i]);
                const double bm = bmax64(eps, chi_min);
                for (int j = 0; j < NY; ++j) {
                    const double chi = j == j_zero ? chi_min : chi_moliere64(eps, bm * std::exp(Y[j]));
                    Q[(size_t)i * NY + j] = std::log(std::tan(0.5 * chi));
                }
            }
        });
    for (auto& x : th) x.join();
    std::vector<double> col(NX), sl(std::max(NX, NY));
    for (int i = 0; i < NX; ++i) spline_slopes(Y.data(), &Q[(size_t)i * NY], NY, &Qy[(size_t)i * NY]);
    for (int j = 0; j < NY; ++j) {
        for (int i = 0; i < NX; ++i) col[i] = Q[(size_t)i * NY + j];
        spline_slopes(X.data(), col.data(), NX, sl.data());
        for (int i = 0; i < NX; ++i) Qx[(size_t)i * NY + j] = sl[i];
        for (int i = 0; i < NX; ++i) col[i] = Qy[(size_t)i * NY + j];
        spline_slopes(X.data(), col.data(), NX, sl.data());
        for (int i = 0; i < NX; ++i) Qxy[(size_t)i * NY + j] = sl[i];
    }
    // cubic Hermite basis in power form: value and slope at t = 0, value and slope at t = 1
    static const double H[4][4] = {{1, 0, -3, 2}, {0, 1, -2, 1}, {0, 0, 3, -2}, {0, 0, -1, 1}};
    ChiTable* T = new ChiTable();
    T->chi_min = chi_min;
    T->a64.assign((size_t)kChiCells * 16, 0.0);
    T->cells.resize((size_t)kChiCells * 4);
    for (int i = 0; i < kChiNx; ++i)
        for (int j = 0; j < kChiNy; ++j) {
            const int ni = i + kExt, nj = j + kExt;
            const double dx = X[ni + 1] - X[ni], dy = Y[nj + 1] - Y[nj];
            double* a = &T->a64[16 * ((size_t)i * kChiNy + j)];
            for (int ci = 0; ci < 2; ++ci)
                for (int cj = 0; cj < 2; ++cj) {
                    const size_t n = (size_t)(ni + ci) * NY + (nj + cj);
                    // (value, y slope; x slope, cross slope) scaled to the cell's unit square
                    const double v[2][2] = {{Q[n], Qy[n] * dy}, {Qx[n] * dx, Qxy[n] * dx * dy}};
                    for (int dxo = 0; dxo < 2; ++dxo)
                        for (int dyo = 0; dyo < 2; ++dyo) {
                            const double* hx = H[2 * ci + dxo];
                            const double* hy = H[2 * cj + dyo];
                            for (int k = 0; k < 4; ++k)
                                for (int l = 0; l < 4; ++l) a[4 * k + l] += v[dxo][dyo] * hx[k] * hy[l];
                        }
                }
            for (int k = 0; k < 4; ++k)
                T->cells[4 * ((size_t)i * kChiNy + j) + k] =
                    make_float4((float)a[4 * k], (float)a[4 * k + 1], (float)a[4 * k + 2], (float)a[4 * k + 3]);
        }
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

void envelope64(const PairPhys& pp, const BmaxTable* bt, double s, double v, double& A, double& B)
{
    // H(rho): the largest h = sigma(g) g over [max(0, v - s rho), v + s rho], sampled at
    // kEnvN + 1 equally spaced rho in [0, kEnvRhoMax]
    double rho[kEnvN + 1], H[kEnvN + 1];
    double hm = sigma64(pp, bt, v) * v;
    for (int k = 0; k <= kEnvN; ++k) {
        rho[k] = kEnvRhoMax * k / kEnvN;
        const double gh = v + s * rho[k];
        hm = std::max(hm, sigma64(pp, bt, gh) * gh);
        const double gl = v - s * rho[k];
        if (gl > 0.0) hm = std::max(hm, sigma64(pp, bt, gl) * gl);
        H[k] = hm;
    }
    // the edge of the upper concave hull of (rho, H) that spans kEnvM
    int hull[kEnvN + 1], nh = 0;
    for (int k = 0; k <= kEnvN; ++k) {
        while (nh >= 2) {
            const int i = hull[nh - 2], j = hull[nh - 1];
            const double cross = (rho[j] - rho[i]) * (H[k] - H[i]) - (H[j] - H[i]) * (rho[k] - rho[i]);
            if (cross >= 0.0) --nh;
            else break;
        }
        hull[nh++] = k;
    }
    int e = 0;
    while (e + 2 < nh && rho[hull[e + 1]] <= kEnvM) ++e;
    const int i = hull[e], j = hull[e + 1];
    const double b = (H[j] - H[i]) / (rho[j] - rho[i]);
    A = (H[i] - b * rho[i]) * (1.0 + kEnvMargin);
    B = b * (1.0 + kEnvMargin);
}

void build_w_tables(const PairPhys& pp, const BmaxTable* bt, double s, int thermal, double v_top, double h_w,
                    std::vector<float4>& K, std::vector<float4>& EA, std::vector<float4>& EB, std::vector<float4>& G,
                    int& n_w)
{
    double w_top = std::log1p(v_top / s);
    n_w = std::max(4, (int)std::ceil(w_top / h_w));
    std::vector<double> kv(3 * n_w + 1), av(3 * n_w + 1), bv(3 * n_w + 1), gv(3 * n_w + 1);
    unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; ++t)
        th.emplace_back([&, t]() {
            for (int j = (int)t; j < 3 * n_w + 1; j += (int)nt) {
                double v = s * std::expm1(h_w * j / 3.0);
                // stationary gas: tabulate sigma(v) = K(v)/v, so that the inverse mean free
                // path n sigma(v) stays finite when the speed decays towards zero
                kv[j] = thermal ? K64(pp, bt, s, 1, v) : sigma64(pp, bt, v);
                av[j] = bv[j] = 0.0;
                if (thermal) envelope64(pp, bt, s, v, av[j], bv[j]);
                // d ln K / d ln s at fixed v by a central difference in s (gas at rest: 0)
                const double hs = 1e-4;
                gv[j] = thermal ? (K64(pp, bt, s * (1.0 + hs), 1, v) - K64(pp, bt, s * (1.0 - hs), 1, v)) /
                                      (2.0 * hs * kv[j])
                                : 0.0;
            }
        });
    for (auto& x : th) x.join();
    K.resize(n_w);
    EA.resize(n_w);
    EB.resize(n_w);
    G.resize(n_w);
    for (int i = 0; i < n_w; ++i) {
        K[i] = cubic_from_thirds(kv[3 * i], kv[3 * i + 1], kv[3 * i + 2], kv[3 * i + 3]);
        EA[i] = cubic_from_thirds(av[3 * i], av[3 * i + 1], av[3 * i + 2], av[3 * i + 3]);
        EB[i] = cubic_from_thirds(bv[3 * i], bv[3 * i + 1], bv[3 * i + 2], bv[3 * i + 3]);
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
