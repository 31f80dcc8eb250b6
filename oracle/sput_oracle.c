/*
 * sput_oracle.c -- plain FP64 CPU reference transporter for sputtered atoms.
 *
 * TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference leg may load this library.  The product path (the
 * CUDA library under paper_2411_14413_gb300/) never links, loads or calls it,
 * and this file shares no code, header, table or constant generator with it.
 *
 * What it computes (Sec. "The SIMTRA model", arXiv 2411.14413):
 *   launch position from the racetrack pdf, Thompson energy with cut-off
 *   E_max = k*Lambda*E_i - U_s (Eq. for phi(E)), cosine-sum polar angle
 *   (Eq. for d2Y/dOmega), free path lambda = -lambda_m ln RN_1 with RN_1 in
 *   ]0,1] (Eq. for lambda), a surface test after every flight (deposition on
 *   hit), and otherwise an elastic binary collision with a thermal Ar atom
 *   under a screened-Coulomb potential with Moliere screening; repeated until
 *   the atom lands.
 *
 * Where the paper is silent these readings are taken (each is mirrored,
 * independently coded, by the CUDA path):
 *   - lambda_m(v) = v / (n_g <sigma(g) g>), the average over a Maxwellian gas
 *     at T; n_g = p / (k_B T).
 *   - sigma(E_r) = pi b_max^2 with chi(E_r, b_max) = chi_min (CM-angle cut-off).
 *   - the gas partner is drawn from the Maxwellian weighted by sigma(g) g by
 *     rejection from the Maxwellian weighted by an envelope A + B |V|/s of
 *     sigma(g) g (s = sqrt(kT/m_gas); the line through the upper concave hull
 *     of the largest sigma(g) g a partner of speed |V| can give, see
 *     envelope()); at most A attempts, the last one is taken if none is
 *     accepted.
 *   - b = b_max sqrt(RN), azimuth 2 pi RN; the azimuth is measured in the
 *     orthonormal basis of Duff et al., "Building an Orthonormal Basis,
 *     Revisited", JCGT 6(1), 2017.
 *   - random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel
 *     random numbers: as easy as 1, 2, 3", SC'11), key = (seed_lo, seed_hi),
 *     counter = (particle id, instance, event, sub-block); a 32-bit word x maps
 *     to RN = ((x >> 8) + 1) * 2^-24, which lies in ]0,1] as the paper asks.
 *
 * Accuracy: every quantity is computed in double precision from its
 * definition.  The scattering integral uses adaptive Gauss-Legendre panels
 * after the substitution r0/r = 1 - w^2; b_max(eps) is found by root
 * bracketing and, for speed, evaluated from 6-point Lagrange interpolation in
 * ln(eps) on nodes spaced 0.05 (the interpolation error is pinned by a test
 * against the direct root).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_VERSION 1

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ---------------------------------------------------------------- constants */
/* CODATA 2018 */
static const double AMU_KG = 1.66053906660e-27;
static const double E_CHARGE = 1.602176634e-19;
static const double KB_J = 1.380649e-23;
static const double KB_EV = 8.617333262e-5;
static const double BOHR_A = 0.529177210903;
static const double E2_EVA = 14.3996454784; /* e^2 / (4 pi eps0) in eV*Angstrom */

/* energy of 1 u moving at 1 km/s, in eV */
static double c_energy(void) { return AMU_KG * 1.0e6 / E_CHARGE; }

/* Moliere screening function (Moliere 1947): 0.35e^-0.3x + 0.55e^-1.2x + 0.10e^-6x */
static const double MOL_C[3] = {0.35, 0.55, 0.10};
static const double MOL_D[3] = {0.3, 1.2, 6.0};

/* ------------------------------------------------------------ Philox4x32-10 */
static void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

void or_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out) { philox4x32_10(ctr, key, out); }

/* RN in ]0,1] (Eq. for lambda asks RN_1 in ]0,1]) */
static double rn(uint32_t x) { return (double)((x >> 8) + 1u) * (1.0 / 16777216.0); }

typedef struct {
    uint32_t key[2];
    uint32_t pid;
    uint32_t inst;
} stream_t;

static void draw(const stream_t* s, uint32_t event, uint32_t sub, uint32_t w[4])
{
    uint32_t ctr[4] = {s->pid, s->inst, event, sub};
    philox4x32_10(ctr, s->key, w);
}

/* ------------------------------------------------------- adaptive quadrature */
/* Gauss-Legendre nodes/weights of order QN on [-1,1] by Newton on P_n. */
#define QN 10
static double gl_x[QN], gl_w[QN];
static pthread_once_t gl_once = PTHREAD_ONCE_INIT;

static void gl_init(void)
{
    for (int i = 0; i < QN; ++i) {
        double x = cos(M_PI * (i + 0.75) / (QN + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= QN; ++k) {
                double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            double dp = QN * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        double p0 = 1.0, p1 = x;
        for (int k = 2; k <= QN; ++k) {
            double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        double dp = QN * (x * p1 - p0) / (x * x - 1.0);
        gl_x[i] = x;
        gl_w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
}

typedef double (*fn1)(double, const void*);

static double gl_panel(fn1 f, const void* ctx, double a, double b)
{
    double h = 0.5 * (b - a), m = 0.5 * (a + b), s = 0.0;
    for (int i = 0; i < QN; ++i) s += gl_w[i] * f(m + h * gl_x[i], ctx);
    return s * h;
}

static double adapt_rec(fn1 f, const void* ctx, double a, double b, double whole, double tol, int depth, int* budget)
{
    double m = 0.5 * (a + b);
    double l = gl_panel(f, ctx, a, m), r = gl_panel(f, ctx, m, b);
    *budget -= 2;
    /* stop refining on a non-finite value or when the panel budget is spent */
    if (!isfinite(l + r) || depth <= 0 || *budget <= 0 || fabs(l + r - whole) <= tol) return l + r;
    return adapt_rec(f, ctx, a, m, l, 0.5 * tol, depth - 1, budget) +
           adapt_rec(f, ctx, m, b, r, 0.5 * tol, depth - 1, budget);
}

/* integral of f over [a,b]; panels are halved until two levels agree to tol
 * (at most 20000 panels per call) */
static double integrate(fn1 f, const void* ctx, double a, double b, double rel_tol)
{
    pthread_once(&gl_once, gl_init);
    double whole = gl_panel(f, ctx, a, b);
    if (!isfinite(whole)) return whole;
    double tol = rel_tol * fabs(whole) + 1e-300;
    int budget = 20000;
    return adapt_rec(f, ctx, a, b, whole, tol, 40, &budget);
}

double or_integrate_test(int which, double a, double b);

/* --------------------------------------------- scattering integral (CM frame) */
/*
 * Reduced units: x = r/a, beta = b/a, eps = a E_r / (Z1 Z2 e^2), with a the
 * Firsov screening length.  V(r)/E_r = Phi(x)/(eps x).
 *   chi = pi - 2 b int_{r0}^inf dr / (r^2 sqrt(1 - V/E_r - b^2/r^2))
 * With u = r0/r and u = 1 - w^2 the integral becomes
 *   chi = pi - 4 (beta/x0) int_0^1 w / sqrt(F(1-w^2)) dw,   (see or_chi)
 * F(u) = [V(r0) - V(r0/u)]/E_r + (beta/x0)^2 (1 - u^2), written so that no
 * two large numbers are subtracted (F(1) = 0 by definition of r0).
 */
enum { SCR_MOLIERE = 0, SCR_COULOMB = 1 };

static double screen_phi(int scr, double x)
{
    if (scr == SCR_COULOMB) return 1.0;
    double s = 0.0;
    for (int i = 0; i < 3; ++i) s += MOL_C[i] * exp(-MOL_D[i] * x);
    return s;
}

/* g(x) = 1 - beta^2/x^2 - Phi(x)/(eps x): increasing in x, root = x0 */
static double apsis_fn(int scr, double eps, double beta, double x)
{
    return 1.0 - (beta * beta) / (x * x) - screen_phi(scr, x) / (eps * x);
}

double or_x0(int scr, double eps, double beta)
{
    /* bracket: g(lo) < 0 <= g(hi); hi = unscreened (Coulomb) apsis since Phi <= 1 */
    double hi = 0.5 * (1.0 / eps + sqrt(1.0 / (eps * eps) + 4.0 * beta * beta));
    double lo = beta > 0.0 ? beta : 0.0;
    if (lo <= 0.0) lo = hi * 1e-300;
    if (apsis_fn(scr, eps, beta, hi) < 0.0) hi *= 1.0 + 1e-12; /* rounding guard */
    for (int it = 0; it < 400; ++it) {
        double m = 0.5 * (lo + hi);
        if (m <= lo || m >= hi) break;
        if (apsis_fn(scr, eps, beta, m) < 0.0) lo = m;
        else hi = m;
        if (hi - lo <= 1e-16 * hi) break;
    }
    return 0.5 * (lo + hi);
}

typedef struct {
    int scr;
    double eps, x0, bx; /* bx = beta/x0 */
} chi_ctx;

/*
 * Since 4 (beta/x0) int_0^1 w / sqrt(F0) dw = pi for the potential-free part
 * F0 = (beta/x0)^2 w^2 (2 - w^2), the deflection is written as
 *   chi = 4 (beta/x0) int_0^1 w P / (sqrt(F) sqrt(F0) (sqrt(F) + sqrt(F0))) dw,
 * P = F - F0 = [V(r0) - V(r0/u)]/E_r >= 0; this is the same quantity as
 * pi - 4 (beta/x0) int w/sqrt(F) dw without the cancellation at small angles.
 */
static double chi_integrand(double w, const void* vctx)
{
    const chi_ctx* c = (const chi_ctx*)vctx;
    double w2 = w * w;
    double one_m_u2 = w2 * (2.0 - w2);
    double F0 = c->bx * c->bx * one_m_u2;
    double P = 0.0;
    if (c->scr == SCR_COULOMB) {
        /* [1/x0 - u/x0]/eps = w^2/(eps x0) */
        P = w2 / (c->eps * c->x0);
    } else {
        double lnu = log1p(-w2);
        double ratio = w2 / (1.0 - w2); /* 1/u - 1 */
        for (int i = 0; i < 3; ++i) {
            double y = MOL_D[i] * c->x0 * ratio;
            double term = -expm1(lnu - y); /* 1 - u e^{-y} */
            P += MOL_C[i] * exp(-MOL_D[i] * c->x0) * term / (c->eps * c->x0);
        }
    }
    double F = F0 + P;
    double sF = sqrt(F), sF0 = sqrt(F0);
    return w * P / (sF * sF0 * (sF + sF0));
}

double or_chi(int scr, double eps, double beta)
{
    if (beta <= 0.0) return M_PI;
    chi_ctx c;
    c.scr = scr;
    c.eps = eps;
    c.x0 = or_x0(scr, eps, beta);
    c.bx = beta / c.x0;
    /* split at a few points so the adaptive panels see the steep region */
    double pts[6] = {0.0, 0.05, 0.2, 0.5, 0.8, 1.0};
    double I = 0.0;
    for (int k = 0; k < 5; ++k) I += integrate(chi_integrand, &c, pts[k], pts[k + 1], 1e-13);
    return 4.0 * c.bx * I;
}

/* hard-sphere test potential: b = d cos(chi/2) */
double or_chi_hard_sphere(double beta) { return 2.0 * acos(beta < 1.0 ? beta : 1.0); }

/* b_max(eps)/a: chi(eps, b_max) = chi_min, chi decreasing in b */
double or_bmax_direct(int scr, double chi_min, double eps)
{
    double lo = 0.0, hi = 1.0;
    while (or_chi(scr, eps, hi) > chi_min) {
        lo = hi;
        hi *= 2.0;
        if (hi > 1e12) return hi;
    }
    /* bisection to 1e-7 relative, then Illinois regula falsi to ~1e-15 */
    double flo = (lo > 0.0 ? or_chi(scr, eps, lo) : M_PI) - chi_min;
    double fhi = or_chi(scr, eps, hi) - chi_min;
    while (hi - lo > 1e-7 * hi) {
        double m = 0.5 * (lo + hi), fm = or_chi(scr, eps, m) - chi_min;
        if (fm > 0.0) { lo = m; flo = fm; }
        else { hi = m; fhi = fm; }
    }
    int side = 0;
    for (int it = 0; it < 60 && hi - lo > 1e-15 * hi; ++it) {
        double m = (lo * fhi - hi * flo) / (fhi - flo);
        if (!(m > lo && m < hi)) m = 0.5 * (lo + hi);
        double fm = or_chi(scr, eps, m) - chi_min;
        if (fm == 0.0) return m;
        if (fm > 0.0) {
            lo = m; flo = fm;
            if (side == 1) fhi *= 0.5;
            side = 1;
        } else {
            hi = m; fhi = fm;
            if (side == -1) flo *= 0.5;
            side = -1;
        }
    }
    return 0.5 * (lo + hi);
}

/* ---- b_max interpolation cache (per chi_min), 6-point Lagrange in ln eps ---- */
#define BM_LO (-42.0)
#define BM_HI (6.0)
#define BM_H (0.05)
#define BM_N ((int)((BM_HI - BM_LO) / BM_H + 0.5) + 1)

typedef struct {
    double chi_min;
    double* node; /* b_max at ln eps = BM_LO + i*BM_H */
} bmax_cache;

static pthread_mutex_t bm_mutex = PTHREAD_MUTEX_INITIALIZER;
static bmax_cache bm_caches[8];
static int bm_ncache = 0;

typedef struct {
    double chi_min;
    double* node;
    int begin, end;
} bm_job;

static void* bm_worker(void* arg)
{
    bm_job* j = (bm_job*)arg;
    for (int i = j->begin; i < j->end; ++i)
        j->node[i] = or_bmax_direct(SCR_MOLIERE, j->chi_min, exp(BM_LO + BM_H * i));
    return NULL;
}

static const double* bmax_nodes(double chi_min)
{
    /* the last table this thread used, without taking the lock (tables are never freed) */
    static __thread double tl_chi = -1.0;
    static __thread const double* tl_node = NULL;
    if (tl_node && tl_chi == chi_min) return tl_node;
    const double* found = NULL;
    pthread_mutex_lock(&bm_mutex);
    for (int i = 0; i < bm_ncache; ++i)
        if (bm_caches[i].chi_min == chi_min) found = bm_caches[i].node;
    if (found) {
        pthread_mutex_unlock(&bm_mutex);
        tl_chi = chi_min;
        tl_node = found;
        return found;
    }
    double* node = (double*)malloc(sizeof(double) * BM_N);
    enum { NT = 16 };
    pthread_t th[NT];
    bm_job jobs[NT];
    int per = (BM_N + NT - 1) / NT;
    for (int t = 0; t < NT; ++t) {
        jobs[t].chi_min = chi_min;
        jobs[t].node = node;
        jobs[t].begin = t * per;
        jobs[t].end = (t + 1) * per < BM_N ? (t + 1) * per : BM_N;
        pthread_create(&th[t], NULL, bm_worker, &jobs[t]);
    }
    for (int t = 0; t < NT; ++t) pthread_join(th[t], NULL);
    int slot = bm_ncache < 8 ? bm_ncache++ : 7;
    bm_caches[slot].chi_min = chi_min;
    bm_caches[slot].node = node;
    pthread_mutex_unlock(&bm_mutex);
    tl_chi = chi_min;
    tl_node = node;
    return node;
}

double or_bmax_interp(double chi_min, double eps)
{
    double le = log(eps);
    if (le < BM_LO + 3 * BM_H || le > BM_HI - 3 * BM_H) return or_bmax_direct(SCR_MOLIERE, chi_min, eps);
    const double* node = bmax_nodes(chi_min);
    double f = (le - BM_LO) / BM_H;
    int i0 = (int)floor(f) - 2; /* nodes i0 .. i0+5 */
    double s = 0.0;
    for (int j = 0; j < 6; ++j) {
        double xj = i0 + j, lj = 1.0;
        for (int m = 0; m < 6; ++m)
            if (m != j) lj *= (f - (i0 + m)) / (xj - (i0 + m));
        s += lj * node[i0 + j];
    }
    return s;
}

/* -------------------------------------------------------------- scene model */
enum { PK_BOX = 0, PK_RECT = 1, PK_DISC = 2, PK_CYL = 3 };
enum { INT_MOLIERE = 0, INT_HARD_SPHERE = 1 };
enum { GAS_THERMAL = 0, GAS_STATIONARY = 1 };

typedef struct {
    int kind;
    double c[3], u[3], v[3], n[3];
    double p0, p1;
} prim_t;

typedef struct {
    int begin, count, substrate;
} geom_t;

typedef struct {
    double Z, mass, U_s;
    double c[3], n[3], e1[3], e2[3];
    double rt_r0, rt_sigma, rt_R, rt_norm;
    double coef[6], coef_norm;
    int target;
    /* collision pair with the gas */
    double a_scr;   /* Firsov screening length, Angstrom */
    double zze2;    /* Z1 Z2 e^2, eV*Angstrom */
    double mu_red;  /* u */
    int h_monotone; /* sigma(g) g non-decreasing on the checked range */
    /* optional joint launch table: weights lt[i * n_E + k] of the cells mu in [i, i+1)/n_mu,
     * E in [k, k+1) E_hi/n_E (uniform inside a cell); NULL = Thompson law + cosine sum */
    int n_mu, n_E;
    double E_hi;
    double* lt;
    double sigma_D; /* diffusion cross section of the shortcut, Angstrom^2 (set when E_switch > 0) */
} cath_t;

typedef struct {
    int geometry, cathode;
    double pressure, E_i, k;
    double n_gas;   /* mm^-3 */
    double E_max;
    uint32_t stream; /* word 1 of the Philox counters of the instance's particles */
} inst_t;

typedef struct or_scene {
    double box_lo[3], box_hi[3];
    double gas_Z, gas_mass, T, s_gas; /* s_gas = sqrt(kT/m_gas) in km/s */
    int n_prims, n_geom, n_cath, n_inst;
    prim_t* prims;
    geom_t* geoms;
    cath_t* cath;
    inst_t* inst;
    int nx, ny, n_ebins, n_abins;
    double half_u, half_v, e_hist_max;
    double chi_min;
    int interaction, gas_motion, max_attempts;
    int want_score_T; /* compute the temperature score (or_scene_set_score_T) */
    int at_cutoff;    /* launch every atom with E = E_max (boundary run of d/dE_max) */
    int plant_unweighted; /* tests only: a planted mistake, the partner is the plain Maxwellian */
    double E_switch;  /* eV: diffusion shortcut below it (0 = off) */
    int64_t max_collisions;
    double hs_diameter;
} or_scene;

static void cross3(const double a[3], const double b[3], double o[3])
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* Thompson cut-off, Eq. for phi(E): E_max = k Lambda E_i - U_s, Lambda = 4 M_i M_t/(M_i+M_t)^2 */
double or_emax(double k, double M_i, double M_t, double E_i, double U_s)
{
    double lam = 4.0 * M_i * M_t / ((M_i + M_t) * (M_i + M_t));
    return k * lam * E_i - U_s;
}

/* total cross section sigma(E_r) in Angstrom^2 for the pair of cathode c */
static double sigma_of_g(const or_scene* S, const cath_t* c, double g)
{
    if (S->interaction == INT_HARD_SPHERE) return M_PI * S->hs_diameter * S->hs_diameter;
    double Er = 0.5 * c->mu_red * g * g * c_energy();
    double eps = c->a_scr * Er / c->zze2;
    /* floor far below any reachable collision (g < 1e-9 km/s) keeps the root finding finite */
    if (!(eps > 1e-40)) eps = 1e-40;
    double bm = or_bmax_interp(S->chi_min, eps) * c->a_scr;
    return M_PI * bm * bm;
}

/* relative-speed density of g = |v - V|, V ~ Maxwellian with per-axis std s */
static double rel_speed_pdf(double g, double v, double s)
{
    const double c = 1.0 / (s * sqrt(2.0 * M_PI));
    if (v < 1e-9 * s) return 2.0 * g * g * c / (s * s) * exp(-g * g / (2.0 * s * s));
    double a = (g - v) / s;
    return g / v * c * exp(-0.5 * a * a) * (-expm1(-2.0 * g * v / (s * s)));
}

typedef struct {
    const or_scene* S;
    const cath_t* c;
    double v, s;
} K_ctx;

static double K_integrand(double g, const void* vctx)
{
    const K_ctx* k = (const K_ctx*)vctx;
    return sigma_of_g(k->S, k->c, g) * g * rel_speed_pdf(g, k->v, k->s);
}

/* <sigma(g) g> over a Maxwellian gas of per-axis velocity spread s */
static double K_of_v_s(const or_scene* S, const cath_t* c, double v, double s)
{
    double a = v - 12.0 * s, b = v + 12.0 * s;
    if (a < 0.0) a = 0.0;
    K_ctx k = {S, c, v, s};
    /* split the window into 8 panels around the peak */
    double I = 0.0;
    for (int p = 0; p < 8; ++p) {
        double x0 = a + (b - a) * p / 8.0, x1 = a + (b - a) * (p + 1) / 8.0;
        I += integrate(K_integrand, &k, x0, x1, 1e-12);
    }
    return I;
}

/* K(v) = <sigma(g) g> over the Maxwellian gas at T, Angstrom^2 km/s */
static double K_of_v(const or_scene* S, const cath_t* c, double v)
{
    if (S->gas_motion == GAS_STATIONARY) return sigma_of_g(S, c, v) * v;
    return K_of_v_s(S, c, v, S->s_gas);
}

/* d ln K / d ln s at fixed v (s = sqrt(kT/m_gas), so d ln K / dT = this / (2T)):
 * central difference of the quadrature; 0 for a gas at rest */
static double dlnK_dlns(const or_scene* S, const cath_t* c, double v)
{
    if (S->gas_motion == GAS_STATIONARY) return 0.0;
    const double h = 1e-4, s = S->s_gas;
    return (K_of_v_s(S, c, v, s * (1.0 + h)) - K_of_v_s(S, c, v, s * (1.0 - h))) / (2.0 * h * K_of_v_s(S, c, v, s));
}

/* mean free path lambda_m(v) = v / (n_g K(v)), mm */
static double lambda_m(const or_scene* S, const cath_t* c, const inst_t* I, double v)
{
    /* gas at rest: lambda_m = 1/(n_g sigma(v)), written without v/v */
    if (S->gas_motion == GAS_STATIONARY) return 1.0 / (I->n_gas * sigma_of_g(S, c, v) * 1e-14);
    double K = K_of_v(S, c, v); /* Angstrom^2 km/s = 1e-14 mm^2 km/s */
    return v / (I->n_gas * K * 1e-14);
}

static double h_of_g(const or_scene* S, const cath_t* c, double g) { return sigma_of_g(S, c, g) * g; }

/* Envelope of the gas-partner rejection (reading of the paper's gas motion).
 * A partner of speed rho s (rho = |V|/s) meets the atom at a relative speed g
 * in [|v - s rho|, v + s rho], so h(g) = sigma(g) g <= H(rho), the largest h
 * over [max(0, v - s rho), v + s rho], which does not decrease with rho.  The
 * envelope is the line A + B rho above H on [0, ENV_RHO_MAX] with the least
 * value at rho = ENV_M = E[rho] under the Maxwellian (the mean of the chi
 * distribution with 3 degrees of freedom, 2 sqrt(2/pi)): the line through the
 * edge of H's upper concave hull that spans ENV_M, with H taken at ENV_N + 1
 * equally spaced rho and the line raised by the relative margin ENV_MARGIN.
 * The expected number of attempts per partner is (A + B ENV_M) / K(v). */
#define ENV_N 512
#define ENV_RHO_MAX 8.0
#define ENV_MARGIN 1e-4
static const double ENV_M = 1.5957691216057308;

static void envelope(const or_scene* S, const cath_t* c, double v, double* A, double* B)
{
    const double s = S->s_gas;
    double rho[ENV_N + 1], H[ENV_N + 1];
    double hm = h_of_g(S, c, v);
    for (int k = 0; k <= ENV_N; ++k) {
        rho[k] = ENV_RHO_MAX * k / ENV_N;
        double hi = h_of_g(S, c, v + s * rho[k]);
        if (hi > hm) hm = hi;
        double glo = v - s * rho[k];
        if (glo > 0.0) {
            double lo = h_of_g(S, c, glo);
            if (lo > hm) hm = lo;
        }
        H[k] = hm;
    }
    /* upper concave hull of (rho_k, H_k), rho increasing (monotone chain) */
    int hull[ENV_N + 1], nh = 0;
    for (int k = 0; k <= ENV_N; ++k) {
        while (nh >= 2) {
            int i = hull[nh - 2], j = hull[nh - 1];
            double cross = (rho[j] - rho[i]) * (H[k] - H[i]) - (H[j] - H[i]) * (rho[k] - rho[i]);
            if (cross >= 0.0) --nh; /* j on or below the chord i -> k */
            else break;
        }
        hull[nh++] = k;
    }
    int e = 0;
    while (e + 2 < nh && rho[hull[e + 1]] <= ENV_M) ++e;
    int i = hull[e], j = hull[e + 1];
    double b = (H[j] - H[i]) / (rho[j] - rho[i]);
    double a = H[i] - b * rho[i];
    *A = a * (1.0 + ENV_MARGIN);
    *B = b * (1.0 + ENV_MARGIN);
}

/* ---------------------------------------------- diffusion shortcut (opt-in) */
typedef struct {
    const or_scene* S;
    const cath_t* c;
    double eps, gpy;
} sm_ctx;

static double sm_integrand(double beta, const void* vctx)
{
    const sm_ctx* k = (const sm_ctx*)vctx;
    double h = sin(0.5 * or_chi(0, k->eps, beta));
    return 2.0 * h * h * beta; /* (1 - cos chi) beta */
}

/* momentum-transfer cross section sigma_m(g) = 2 pi int_0^inf (1 - cos chi) b db, Angstrom^2 */
static double sigma_m_of_g(const or_scene* S, const cath_t* c, double g)
{
    if (S->interaction == INT_HARD_SPHERE) return M_PI * S->hs_diameter * S->hs_diameter;
    double eps = c->a_scr * 0.5 * c->mu_red * g * g * c_energy() / c->zze2;
    if (!(eps > 1e-40)) eps = 1e-40;
    double B = or_bmax_interp(S->chi_min, eps);
    if (B < 1.0) B = 1.0;
    while (or_chi(0, eps, B) > 1e-9 && B < 1e4) B *= 1.5;
    sm_ctx k = {S, c, eps, 0.0};
    double I = 0.0;
    for (int p = 0; p < 16; ++p) I += integrate(sm_integrand, &k, B * p / 16.0, B * (p + 1) / 16.0, 1e-10);
    return 2.0 * M_PI * c->a_scr * c->a_scr * I;
}

static double om_integrand(double y, const void* vctx)
{
    const sm_ctx* k = (const sm_ctx*)vctx;
    return exp(-y * y) * pow(y, 5) * sigma_m_of_g(k->S, k->c, y * k->gpy);
}

/* 1/lambda_D = n sigma_D with lambda_D = 3 D12 / vbar1: D12 = 3kT/(16 n mu Omega11) is the first
 * Chapman-Enskog diffusion coefficient, Omega11 = sqrt(kT/(2 pi mu)) int e^{-y^2} y^5 sigma_m dy
 * with g = y sqrt(2kT/mu), vbar1 = sqrt(8kT/(pi m1)) the atom's mean thermal speed; Angstrom^2 */
static double sigma_D_of(const or_scene* S, const cath_t* c)
{
    double kT = KB_J * S->T, mu = c->mu_red * AMU_KG;
    sm_ctx k = {S, c, 0.0, sqrt(2.0 * kT / mu) * 1e-3};
    double I = 0.0;
    for (int p = 0; p < 12; ++p) I += integrate(om_integrand, &k, 0.5 * p, 0.5 * (p + 1), 1e-10);
    double omega = sqrt(kT / (2.0 * M_PI * mu)) * I;
    double vbar1 = sqrt(8.0 * kT / (M_PI * c->mass * AMU_KG));
    return 16.0 * mu * vbar1 * omega / (9.0 * kT);
}

/* ----------------------------------------------------------------- sampling */
/* racetrack: radial pdf proportional to r * exp(-(r-r0)^2/(2 sigma^2)) on [0,R]
 * (axisymmetric depth profile, Sec. "Racetrack measurement"); the
 * unnormalised CDF has the closed form below. */
static double racetrack_F(double r0, double sg, double r)
{
    double q = sg * sqrt(2.0);
    return sg * sg * (exp(-(r0 * r0) / (2 * sg * sg)) - exp(-(r - r0) * (r - r0) / (2 * sg * sg))) +
           r0 * sg * sqrt(M_PI / 2.0) * (erf((r - r0) / q) + erf(r0 / q));
}

double or_racetrack_cdf(double r0, double sg, double R, double r)
{
    return racetrack_F(r0, sg, r) / racetrack_F(r0, sg, R);
}

double or_racetrack_r(double r0, double sg, double R, double u)
{
    double tgt = u * racetrack_F(r0, sg, R);
    double lo = 0.0, hi = R;
    for (int it = 0; it < 200 && hi - lo > 1e-15 * R; ++it) {
        double m = 0.5 * (lo + hi);
        if (racetrack_F(r0, sg, m) < tgt) lo = m;
        else hi = m;
    }
    return 0.5 * (lo + hi);
}

/* Thompson energy with cut-off (Eq. for phi(E)) by exact inversion:
 * CDF(E) = [E/(E+U)]^2 / [E_m/(E_m+U)]^2 */
double or_thompson(double E_max, double U, double u)
{
    double s = sqrt(u) * E_max / (E_max + U);
    return U * s / (1.0 - s);
}

/* cosine-sum emission (Eq. for d2Y/dOmega): pdf in mu = cos(theta) is
 * proportional to sum_i c_i mu^i on [0,1]; invert the polynomial CDF by bisection */
static double cos_cdf_un(const double* cf, double mu)
{
    double s = 0.0, p = mu;
    for (int i = 0; i < 6; ++i) {
        s += cf[i] * p / (i + 1);
        p *= mu;
    }
    return s;
}

double or_cos_mu(const double* cf, double u)
{
    double tot = cos_cdf_un(cf, 1.0), tgt = u * tot;
    double lo = 0.0, hi = 1.0;
    for (int it = 0; it < 200 && hi - lo > 1e-16; ++it) {
        double m = 0.5 * (lo + hi);
        if (cos_cdf_un(cf, m) < tgt) lo = m;
        else hi = m;
    }
    return 0.5 * (lo + hi);
}

/* ---------------------------------------------------------------- geometry */
/* nearest hit with t in (0, ell] (box: [0, ell]); ties -> lowest index */
static int hit_test(const or_scene* S, const geom_t* G, const double p[3], const double d[3], double ell,
                    int exclude, double* t_out)
{
    double best = INFINITY;
    int who = -1;
    for (int li = 0; li < G->count; ++li) {
        if (li == exclude) continue;
        const prim_t* P = &S->prims[G->begin + li];
        double t = INFINITY;
        if (P->kind == PK_BOX) {
            double te = INFINITY;
            for (int a = 0; a < 3; ++a) {
                if (d[a] > 0.0) {
                    double x = (S->box_hi[a] - p[a]) / d[a];
                    if (x < te) te = x;
                } else if (d[a] < 0.0) {
                    double x = (S->box_lo[a] - p[a]) / d[a];
                    if (x < te) te = x;
                }
            }
            if (te < 0.0) te = 0.0;
            if (te <= ell) t = te;
        } else if (P->kind == PK_RECT || P->kind == PK_DISC) {
            double den = dot3(d, P->n);
            if (den != 0.0) {
                double w[3] = {P->c[0] - p[0], P->c[1] - p[1], P->c[2] - p[2]};
                double tt = dot3(w, P->n) / den;
                if (tt > 0.0 && tt <= ell) {
                    double q[3] = {p[0] + tt * d[0] - P->c[0], p[1] + tt * d[1] - P->c[1], p[2] + tt * d[2] - P->c[2]};
                    double a1 = dot3(q, P->u), a2 = dot3(q, P->v);
                    int in;
                    if (P->kind == PK_RECT) in = fabs(a1) <= P->p0 && fabs(a2) <= P->p1;
                    else {
                        double r2 = a1 * a1 + a2 * a2;
                        in = r2 >= P->p0 * P->p0 && r2 <= P->p1 * P->p1;
                    }
                    if (in) t = tt;
                }
            }
        } else if (P->kind == PK_CYL) {
            const double* ax = P->u;
            double w[3] = {p[0] - P->c[0], p[1] - P->c[1], p[2] - P->c[2]};
            double wa = dot3(w, ax), da = dot3(d, ax);
            double wp[3] = {w[0] - wa * ax[0], w[1] - wa * ax[1], w[2] - wa * ax[2]};
            double dp[3] = {d[0] - da * ax[0], d[1] - da * ax[1], d[2] - da * ax[2]};
            double A = dot3(dp, dp), B = 2.0 * dot3(wp, dp), C = dot3(wp, wp) - P->p0 * P->p0;
            double disc = B * B - 4.0 * A * C;
            if (A > 0.0 && disc >= 0.0) {
                double sq = sqrt(disc);
                double r1 = (-B - sq) / (2.0 * A), r2 = (-B + sq) / (2.0 * A);
                double roots[2] = {r1, r2};
                for (int k = 0; k < 2; ++k) {
                    double tt = roots[k];
                    if (tt > 0.0 && tt <= ell && fabs(wa + tt * da) <= P->p1) {
                        t = tt;
                        break;
                    }
                }
            }
        }
        if (t < best) {
            best = t;
            who = li;
        }
    }
    *t_out = best;
    return who;
}

/* --------------------------------------------------------------- collision */
/* orthonormal pair perpendicular to unit n (Duff et al., JCGT 2017) */
static void onb(const double n[3], double b1[3], double b2[3])
{
    double sign = copysign(1.0, n[2]);
    double a = -1.0 / (sign + n[2]);
    double b = n[0] * n[1] * a;
    b1[0] = 1.0 + sign * n[0] * n[0] * a;
    b1[1] = sign * b;
    b1[2] = -sign * n[0];
    b2[0] = b;
    b2[1] = sign + n[1] * n[1] * a;
    b2[2] = -n[1];
}

/* elastic binary collision in the CM frame: rotate the relative velocity
 * g = v - V by (chi, psi); |g| is unchanged (elastic, Sec. "The SIMTRA model") */
static void collide_with(const or_scene* S, const cath_t* c, const double v[3], const double V[3], double u_b,
                         double u_psi, double v_out[3], double V_out[3], double* chi_out)
{
    double m1 = c->mass, m2 = S->gas_mass, M = m1 + m2;
    double gv[3] = {v[0] - V[0], v[1] - V[1], v[2] - V[2]};
    double g = sqrt(dot3(gv, gv));
    double chi;
    if (!(g > 0.0)) {
        memcpy(v_out, v, sizeof(double) * 3);
        memcpy(V_out, V, sizeof(double) * 3);
        if (chi_out) *chi_out = 0.0;
        return;
    }
    if (S->interaction == INT_HARD_SPHERE) {
        chi = or_chi_hard_sphere(sqrt(u_b));
    } else {
        double Er = 0.5 * c->mu_red * g * g * c_energy();
        double eps = c->a_scr * Er / c->zze2;
        double beta = or_bmax_interp(S->chi_min, eps) * sqrt(u_b);
        chi = or_chi(SCR_MOLIERE, eps, beta);
    }
    double psi = 2.0 * M_PI * u_psi;
    double gh[3] = {gv[0] / g, gv[1] / g, gv[2] / g}, b1[3], b2[3];
    onb(gh, b1, b2);
    double cc = cos(chi), sc = sin(chi), cp = cos(psi), sp = sin(psi);
    double g2[3];
    for (int a = 0; a < 3; ++a) g2[a] = g * (cc * gh[a] + sc * (cp * b1[a] + sp * b2[a]));
    for (int a = 0; a < 3; ++a) {
        double vcm = (m1 * v[a] + m2 * V[a]) / M;
        v_out[a] = vcm + (m2 / M) * g2[a];
        V_out[a] = vcm - (m1 / M) * g2[a];
    }
    if (chi_out) *chi_out = chi;
}

/* Gas partner: the Maxwellian f(V) weighted by h(g) = sigma(g) g, g = |v - V|,
 * by rejection from the proposal f(V) (A + B rho) of the envelope above: the
 * Maxwellian with weight A and, with weight B ENV_M, its rho-weighted form, whose
 * speed has the chi distribution with 4 degrees of freedom; accepted with
 * probability h(g) / (A + B rho).  Attempt a draws Philox block 1 + a of the
 * flight's event.  The upper 24 bits of its four words give two Box-Muller pairs,
 * z = (z1, z2, z3, z4) standard normal.  The low bytes of words 0, 1, 2, joined
 * into one 24-bit number, give u: u (A + B ENV_M) <= B ENV_M selects the rho-
 * weighted branch, and u, rescaled to (0, 1] inside the selected branch, is the
 * acceptance uniform.  Maxwellian branch: V = s (z1, z2, z3).  Weighted branch:
 * V = s |z| (z1, z2, z3) / |(z1, z2, z3)| (the direction of (z1, z2, z3) is
 * uniform and independent of |z|).  At most A attempts; the last is kept if none
 * is accepted. */
static int sample_partner(const or_scene* S, const cath_t* c, const stream_t* st, uint32_t event, const double v[3],
                          double V[3])
{
    if (S->gas_motion == GAS_STATIONARY) {
        V[0] = V[1] = V[2] = 0.0;
        return 0;
    }
    if (S->plant_unweighted) {
        /* planted mistake for the tests that must detect it: no sigma(g) g weighting */
        uint32_t w[4];
        draw(st, event, 1u, w);
        double R0 = sqrt(-2.0 * log(rn(w[0]))), R1 = sqrt(-2.0 * log(rn(w[2])));
        V[0] = S->s_gas * R0 * cos(2.0 * M_PI * rn(w[1]));
        V[1] = S->s_gas * R0 * sin(2.0 * M_PI * rn(w[1]));
        V[2] = S->s_gas * R1 * cos(2.0 * M_PI * rn(w[3]));
        return 1;
    }
    double speed = sqrt(dot3(v, v));
    double Aenv, Benv;
    envelope(S, c, speed, &Aenv, &Benv);
    const double Bm = Benv * ENV_M, tot = Aenv + Bm;
    double s = S->s_gas;
    int A = S->max_attempts;
    uint32_t w[4];
    for (int a = 0; a < A; ++a) {
        draw(st, event, 1u + (uint32_t)a, w);
        double R0 = sqrt(-2.0 * log(rn(w[0]))), R1 = sqrt(-2.0 * log(rn(w[2])));
        double z1 = R0 * cos(2.0 * M_PI * rn(w[1])), z2 = R0 * sin(2.0 * M_PI * rn(w[1]));
        double z3 = R1 * cos(2.0 * M_PI * rn(w[3])), z4 = R1 * sin(2.0 * M_PI * rn(w[3]));
        uint32_t low = ((w[0] & 0xffu) << 24) | ((w[1] & 0xffu) << 16) | ((w[2] & 0xffu) << 8);
        double ut = rn(low) * tot;
        double r3 = sqrt(z1 * z1 + z2 * z2 + z3 * z3);
        int weighted = ut <= Bm;
        double rho = weighted ? sqrt(r3 * r3 + z4 * z4) : r3;
        double scale = weighted ? (r3 > 0.0 ? rho / r3 : 0.0) : 1.0;
        V[0] = s * scale * z1;
        V[1] = s * scale * z2;
        V[2] = s * scale * z3;
        double gv[3] = {v[0] - V[0], v[1] - V[1], v[2] - V[2]};
        double hg = h_of_g(S, c, sqrt(dot3(gv, gv)));
        double env = Aenv + Benv * rho;
        /* weighted: u' = ut / Bm; Maxwellian: u' = (ut - Bm) / Aenv; accept if u' env <= h */
        if (weighted ? ut * env <= Bm * hg : (ut - Bm) * env <= Aenv * hg) return a + 1;
    }
    return A;
}

/* Joint launch table: mu from the marginal over the mu cells (uniform u_mu),
 * then E from the weights of the drawn mu cell (uniform u_E); each draw is the
 * inverse of the piecewise-linear CDF of a piecewise-uniform density, found by
 * a plain scan over the cumulative weights (u in ]0,1]). */
static void table_draw(const double* w, int n, int stride, double u, int* cell, double* t)
{
    double tot = 0.0;
    for (int i = 0; i < n; ++i) tot += w[(size_t)i * stride];
    double target = u * tot, acc = 0.0;
    for (int i = 0; i < n; ++i) {
        double wi = w[(size_t)i * stride];
        if (wi > 0.0 && acc + wi >= target) {
            *cell = i;
            *t = (target - acc) / wi;
            if (*t > 1.0) *t = 1.0;
            if (*t < 0.0) *t = 0.0;
            return;
        }
        acc += wi;
    }
    /* rounding left u * tot above the sum: the last cell of positive weight */
    for (int i = n - 1; i >= 0; --i)
        if (w[(size_t)i * stride] > 0.0) {
            *cell = i;
            *t = 1.0;
            return;
        }
    *cell = 0;
    *t = 1.0;
}

static void table_launch(const cath_t* c, double u_mu, double u_E, double* mu, double* E)
{
    /* marginal weight of mu cell i = sum over k of lt[i][k] */
    double* row = (double*)malloc((size_t)c->n_mu * sizeof(double));
    for (int i = 0; i < c->n_mu; ++i) {
        row[i] = 0.0;
        for (int k = 0; k < c->n_E; ++k) row[i] += c->lt[(size_t)i * c->n_E + k];
    }
    int i, k;
    double tm, te;
    table_draw(row, c->n_mu, 1, u_mu, &i, &tm);
    free(row);
    table_draw(c->lt + (size_t)i * c->n_E, c->n_E, 1, u_E, &k, &te);
    *mu = (i + tm) / c->n_mu;
    *E = (k + te) * c->E_hi / c->n_E;
}

int or_set_launch_table(or_scene* S, int cath, int n_mu, int n_E, double E_hi, const double* w)
{
    if (cath < 0 || cath >= S->n_cath || n_mu < 1 || n_E < 1 || !(E_hi > 0.0)) return -1;
    cath_t* c = &S->cath[cath];
    free(c->lt);
    c->lt = (double*)malloc((size_t)n_mu * n_E * sizeof(double));
    memcpy(c->lt, w, (size_t)n_mu * n_E * sizeof(double));
    c->n_mu = n_mu;
    c->n_E = n_E;
    c->E_hi = E_hi;
    return 0;
}

void or_table_launch(const or_scene* S, int cath, double u_mu, double u_E, double* mu, double* E)
{
    table_launch(&S->cath[cath], u_mu, u_E, mu, E);
}

/* ------------------------------------------------------------- transport */
typedef struct {
    int32_t prim;  /* local primitive index, -1 = timed out */
    int32_t cell;  /* substrate grid cell (front face) or -1 */
    double E;      /* arrival energy, eV */
    double cosang; /* |cos| of arrival angle to the substrate normal (front hits) */
    int64_t ncoll;
    double score;  /* d ln p(path) / d ln n_gas */
    double score_T; /* d ln p(path) / dT at fixed pressure, 1/K (when requested) */
    int64_t attempts;
} outcome_t;

static double speed_of_E(double E, double m) { return sqrt(2.0 * E / (m * c_energy())); }

/* optional trace: rows of (x,y,z, dx,dy,dz, speed, status, a, t); row 0 = launch
 * (status -1), row r = state after flight r (status 0 collided: position at the
 * collision, direction/speed after it, a = partner attempts, t = flight length;
 * 1 landed: hit point, a = primitive, t = hit distance; 2 timed out) */
static void trace_row(double* tr, int rows, int r, const double p[3], const double d[3], double speed, int status,
                      double a, double t)
{
    if (!tr || r >= rows) return;
    double* q = tr + 10 * r;
    q[0] = p[0]; q[1] = p[1]; q[2] = p[2];
    q[3] = d[0]; q[4] = d[1]; q[5] = d[2];
    q[6] = speed; q[7] = status; q[8] = a; q[9] = t;
}

static void transport_one(const or_scene* S, uint64_t seed, int ii, uint64_t pid, outcome_t* o, double* tr, int rows)
{
    const inst_t* I = &S->inst[ii];
    const cath_t* c = &S->cath[I->cathode];
    const geom_t* G = &S->geoms[I->geometry];
    stream_t st = {{(uint32_t)seed, (uint32_t)(seed >> 32)}, (uint32_t)pid, S->inst[ii].stream};
    uint32_t w[4];

    /* launch: event 0 */
    draw(&st, 0u, 0u, w);
    double r = or_racetrack_r(c->rt_r0, c->rt_sigma, c->rt_R, rn(w[0]));
    double al = 2.0 * M_PI * rn(w[1]);
    double E, mu;
    if (c->lt) table_launch(c, rn(w[3]), rn(w[2]), &mu, &E);
    else {
        E = S->at_cutoff ? I->E_max : or_thompson(I->E_max, c->U_s, rn(w[2]));
        mu = or_cos_mu(c->coef, rn(w[3]));
    }
    draw(&st, 0u, 1u, w);
    double ph = 2.0 * M_PI * rn(w[0]);
    double st_ = sqrt((1.0 - mu) * (1.0 + mu));
    double p[3], d[3], v[3];
    for (int a = 0; a < 3; ++a) {
        p[a] = c->c[a] + r * cos(al) * c->e1[a] + r * sin(al) * c->e2[a];
        d[a] = st_ * cos(ph) * c->e1[a] + st_ * sin(ph) * c->e2[a] + mu * c->n[a];
    }
    double speed = speed_of_E(E, c->mass);
    int64_t ncoll = 0, attempts = 0;
    int walk = 0; /* thermalised: random walk of the diffusion shortcut */
    double score = 0.0, score_T = 0.0;
    o->score_T = 0.0;
    trace_row(tr, rows, 0, p, d, speed, -1, 0.0, 0.0);

    for (uint32_t k = 1;; ++k) {
        draw(&st, k, 0u, w);
        double lam = walk ? 1.0 / (I->n_gas * c->sigma_D * 1e-14) : lambda_m(S, c, I, speed);
        /* no gas (p = 0): straight line-of-sight flight */
        double ell = I->n_gas > 0.0 ? -lam * log(rn(w[0])) : INFINITY;
        double t;
        int hit = hit_test(S, G, p, d, ell, k == 1 ? c->target : -1, &t);
        /* temperature score: the collision rate n_g K(v)/v with n_g = p/(k_B T)
         * has d ln(rate)/dT = (-1 + G/2)/T, G = d ln K/d ln s */
        double Gv = S->want_score_T ? dlnK_dlns(S, c, speed) : 0.0;
        double aT = (-1.0 + 0.5 * Gv) / S->T;
        if (hit >= 0) {
            score -= t / lam;
            score_T -= aT * t / lam;
            double q[3] = {p[0] + t * d[0], p[1] + t * d[1], p[2] + t * d[2]};
            trace_row(tr, rows, (int)k, q, d, speed, 1, hit, t);
            o->prim = hit;
            o->cell = -1;
            o->cosang = 0.0;
            o->E = 0.5 * c->mass * speed * speed * c_energy();
            if (hit == G->substrate) {
                const prim_t* P = &S->prims[G->begin + hit];
                double dn = dot3(d, P->n);
                if (dn < 0.0) {
                    double rel[3] = {q[0] - P->c[0], q[1] - P->c[1], q[2] - P->c[2]};
                    double a1 = dot3(rel, P->u), a2 = dot3(rel, P->v);
                    double fx = (a1 + S->half_u) / (2.0 * S->half_u) * S->nx;
                    double fy = (a2 + S->half_v) / (2.0 * S->half_v) * S->ny;
                    if (fx >= 0.0 && fy >= 0.0 && fx <= S->nx && fy <= S->ny) {
                        int ix = (int)floor(fx), iy = (int)floor(fy);
                        if (ix >= S->nx) ix = S->nx - 1;
                        if (iy >= S->ny) iy = S->ny - 1;
                        o->cell = iy * S->nx + ix;
                    }
                    o->cosang = -dn;
                }
            }
            o->ncoll = ncoll;
            o->score = score;
            o->score_T = score_T;
            o->attempts = attempts;
            return;
        }
        for (int a = 0; a < 3; ++a) p[a] += ell * d[a];
        score += 1.0 - ell / lam;
        score_T += aT * (1.0 - ell / lam);
        if ((int64_t)k > S->max_collisions) {
            trace_row(tr, rows, (int)k, p, d, speed, 2, 0.0, ell);
            o->prim = -1;
            o->cell = -1;
            o->E = 0.5 * c->mass * speed * speed * c_energy();
            o->cosang = 0.0;
            o->ncoll = ncoll;
            o->score = score;
            o->score_T = score_T;
            o->attempts = attempts;
            return;
        }
        if (walk) {
            /* isotropic new direction from words 1 and 2; speed unchanged */
            double mu = 2.0 * rn(w[1]) - 1.0, phi = 2.0 * M_PI * rn(w[2]);
            double sn = sqrt((1.0 - mu) * (1.0 + mu));
            d[0] = sn * cos(phi);
            d[1] = sn * sin(phi);
            d[2] = mu;
            ++ncoll;
            trace_row(tr, rows, (int)k, p, d, speed, 0, 0.0, ell);
            continue;
        }
        for (int a = 0; a < 3; ++a) v[a] = speed * d[a];
        double V[3], vo[3], Vo[3];
        int na = sample_partner(S, c, &st, k, v, V);
        attempts += na;
        /* partner density f_T(V) sigma(g) g / K(v): d ln/dT = -3/(2T) + |V|^2/(2 s^2 T) - G/(2T) */
        if (S->want_score_T && S->gas_motion == GAS_THERMAL)
            score_T += (-1.5 + 0.5 * dot3(V, V) / (S->s_gas * S->s_gas) - 0.5 * Gv) / S->T;
        collide_with(S, c, v, V, rn(w[1]), rn(w[2]), vo, Vo, NULL);
        speed = sqrt(dot3(vo, vo));
        for (int a = 0; a < 3; ++a) d[a] = vo[a] / speed;
        ++ncoll;
        if (S->E_switch > 0.0 && 0.5 * c->mass * speed * speed * c_energy() < S->E_switch) walk = 1;
        trace_row(tr, rows, (int)k, p, d, speed, 0, na, ell);
    }
}

/* ------------------------------------------------------------- public API */
/*
 * Flat input layouts (doubles):
 *   chamber[9]      box_lo[3] box_hi[3] gas_Z gas_mass T
 *   prims[16*n]     kind c[3] u[3] v[3] p0 p1 (rest unused)
 *   geoms[3*n] int  prim_begin prim_count substrate_local
 *   cath[32*n]      Z mass U_s c[3] n[3] e1[3] rt_r0 rt_sigma rt_R coef[6] target_local
 *   inst[8*n]       geometry cathode pressure E_i k rng_stream (0 = the instance index, s > 0 = s - 1)
 *   grid[8]         nx ny half_u half_v n_ebins e_hist_max n_abins
 *   phys[8]         chi_min(rad) interaction hs_diameter gas_motion max_attempts max_collisions
 */
or_scene* or_scene_new(const double* chamber, int n_prims, const double* prims, int n_geom, const int* geoms,
                       int n_cath, const double* cath, int n_inst, const double* inst, const double* grid,
                       const double* phys)
{
    or_scene* S = (or_scene*)calloc(1, sizeof(or_scene));
    for (int a = 0; a < 3; ++a) {
        S->box_lo[a] = chamber[a];
        S->box_hi[a] = chamber[3 + a];
    }
    S->gas_Z = chamber[6];
    S->gas_mass = chamber[7];
    S->T = chamber[8];
    S->s_gas = sqrt(KB_EV * S->T / (S->gas_mass * c_energy()));
    S->chi_min = phys[0];
    S->interaction = (int)phys[1];
    S->hs_diameter = phys[2];
    S->gas_motion = (int)phys[3];
    S->max_attempts = (int)phys[4];
    S->max_collisions = (int64_t)phys[5];
    S->E_switch = phys[6];
    S->nx = (int)grid[0];
    S->ny = (int)grid[1];
    S->half_u = grid[2];
    S->half_v = grid[3];
    S->n_ebins = (int)grid[4];
    S->e_hist_max = grid[5];
    S->n_abins = (int)grid[6];

    S->n_prims = n_prims;
    S->prims = (prim_t*)calloc((size_t)n_prims, sizeof(prim_t));
    for (int i = 0; i < n_prims; ++i) {
        const double* q = prims + 16 * i;
        prim_t* P = &S->prims[i];
        P->kind = (int)q[0];
        memcpy(P->c, q + 1, 3 * sizeof(double));
        memcpy(P->u, q + 4, 3 * sizeof(double));
        memcpy(P->v, q + 7, 3 * sizeof(double));
        P->p0 = q[10];
        P->p1 = q[11];
        cross3(P->u, P->v, P->n);
    }
    S->n_geom = n_geom;
    S->geoms = (geom_t*)calloc((size_t)n_geom, sizeof(geom_t));
    for (int i = 0; i < n_geom; ++i) {
        S->geoms[i].begin = geoms[3 * i];
        S->geoms[i].count = geoms[3 * i + 1];
        S->geoms[i].substrate = geoms[3 * i + 2];
    }
    S->n_cath = n_cath;
    S->cath = (cath_t*)calloc((size_t)n_cath, sizeof(cath_t));
    for (int i = 0; i < n_cath; ++i) {
        const double* q = cath + 32 * i;
        cath_t* c = &S->cath[i];
        c->Z = q[0];
        c->mass = q[1];
        c->U_s = q[2];
        memcpy(c->c, q + 3, 3 * sizeof(double));
        memcpy(c->n, q + 6, 3 * sizeof(double));
        memcpy(c->e1, q + 9, 3 * sizeof(double));
        cross3(c->n, c->e1, c->e2);
        c->rt_r0 = q[12];
        c->rt_sigma = q[13];
        c->rt_R = q[14];
        memcpy(c->coef, q + 15, 6 * sizeof(double));
        c->target = (int)q[21];
        /* Firsov screening length a = 0.8853 a_0 (Z1^1/2 + Z2^1/2)^-2/3 */
        c->a_scr = 0.8853 * BOHR_A * pow(sqrt(c->Z) + sqrt(S->gas_Z), -2.0 / 3.0);
        c->zze2 = c->Z * S->gas_Z * E2_EVA;
        c->mu_red = c->mass * S->gas_mass / (c->mass + S->gas_mass);
        c->h_monotone = 1;
    }
    S->n_inst = n_inst;
    S->inst = (inst_t*)calloc((size_t)n_inst, sizeof(inst_t));
    for (int i = 0; i < n_inst; ++i) {
        const double* q = inst + 8 * i;
        inst_t* I = &S->inst[i];
        I->geometry = (int)q[0];
        I->cathode = (int)q[1];
        I->pressure = q[2];
        I->E_i = q[3];
        I->k = q[4];
        I->stream = q[5] > 0.0 ? (uint32_t)q[5] - 1u : (uint32_t)i;
        I->n_gas = I->pressure / (KB_J * S->T) * 1e-9; /* m^-3 -> mm^-3 */
        const cath_t* c = &S->cath[I->cathode];
        I->E_max = or_emax(I->k, S->gas_mass, c->mass, I->E_i, c->U_s);
    }
    for (int i = 0; i < n_cath; ++i) S->cath[i].sigma_D = S->E_switch > 0.0 ? sigma_D_of(S, &S->cath[i]) : 0.0;
    /* check monotonicity of sigma(g) g up to well beyond the fastest launch */
    for (int i = 0; i < n_cath; ++i) {
        cath_t* c = &S->cath[i];
        if (S->interaction != INT_MOLIERE || S->gas_motion != GAS_THERMAL) continue;
        double Emx = 0.0;
        for (int j = 0; j < n_inst; ++j)
            if (S->inst[j].cathode == i && S->inst[j].E_max > Emx) Emx = S->inst[j].E_max;
        double gtop = speed_of_E(Emx > 0 ? Emx : 1.0, c->mass) + 20.0 * S->s_gas;
        double prev = 0.0;
        for (int j = 1; j <= 4000; ++j) {
            double hv = h_of_g(S, c, gtop * j / 4000.0);
            if (hv < prev) {
                c->h_monotone = 0;
                break;
            }
            prev = hv;
        }
    }
    return S;
}

void or_scene_free(or_scene* S)
{
    if (!S) return;
    free(S->prims);
    free(S->geoms);
    for (int i = 0; i < S->n_cath; ++i) free(S->cath[i].lt);
    free(S->cath);
    free(S->inst);
    free(S);
}

typedef struct {
    const or_scene* S;
    uint64_t seed;
    const int32_t* inst;
    const uint64_t* pid;
    int64_t begin, end;
    int32_t *prim, *cell;
    double *E, *cosang, *score;
    int64_t *ncoll, *attempts;
    double* score_T;
} run_job;

static void* run_worker(void* arg)
{
    run_job* j = (run_job*)arg;
    for (int64_t i = j->begin; i < j->end; ++i) {
        outcome_t o;
        transport_one(j->S, j->seed, j->inst[i], j->pid[i], &o, NULL, 0);
        j->prim[i] = o.prim;
        j->cell[i] = o.cell;
        j->E[i] = o.E;
        j->cosang[i] = o.cosang;
        j->ncoll[i] = o.ncoll;
        j->score[i] = o.score;
        j->attempts[i] = o.attempts;
        if (j->score_T) j->score_T[i] = o.score_T;
    }
    return NULL;
}

/* transport the particles (inst[i], pid[i]) for i < n with n_threads threads */
int or_run_ids(const or_scene* S, uint64_t seed, int64_t n, const int32_t* inst, const uint64_t* pid, int n_threads,
               int32_t* prim, int32_t* cell, double* E, double* cosang, int64_t* ncoll, double* score,
               int64_t* attempts, double* score_T)
{
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    for (int64_t i = 0; i < n; ++i)
        if (inst[i] < 0 || inst[i] >= S->n_inst) return -1;
    pthread_t th[256];
    run_job jobs[256];
    int64_t per = (n + n_threads - 1) / n_threads;
    int used = 0;
    for (int t = 0; t < n_threads; ++t) {
        int64_t b = t * per, e = (t + 1) * per < n ? (t + 1) * per : n;
        if (b >= e) break;
        run_job J = {S, seed, inst, pid, b, e, prim, cell, E, cosang, score, ncoll, attempts, score_T};
        jobs[t] = J;
        pthread_create(&th[t], NULL, run_worker, &jobs[t]);
        ++used;
    }
    for (int t = 0; t < used; ++t) pthread_join(th[t], NULL);
    return 0;
}

/* ------------------------------------------------ probes for unit tests */
int or_version(void) { return OR_VERSION; }
/* compute the temperature score in or_run_ids from now on (slower: three quadratures per flight) */
void or_scene_set_score_T(or_scene* S, int on) { S->want_score_T = on; }
/* launch every atom at the Thompson cut-off E_max from now on (boundary runs) */
void or_scene_set_at_cutoff(or_scene* S, int on) { S->at_cutoff = on; }
void or_scene_plant_unweighted_partner(or_scene* S, int on) { S->plant_unweighted = on; }
double or_dlnK_dlns(const or_scene* S, int cath, double v) { return dlnK_dlns(S, &S->cath[cath], v); }
double or_sigma_m(const or_scene* S, int cath, double g) { return sigma_m_of_g(S, &S->cath[cath], g); }
double or_sigma_D(const or_scene* S, int cath) { return sigma_D_of(S, &S->cath[cath]); }
double or_c_energy(void) { return c_energy(); }
double or_s_gas(const or_scene* S) { return S->s_gas; }
double or_n_gas(const or_scene* S, int inst) { return S->inst[inst].n_gas; }
double or_inst_emax(const or_scene* S, int inst) { return S->inst[inst].E_max; }
double or_cath_ascr(const or_scene* S, int c) { return S->cath[c].a_scr; }
int or_cath_monotone(const or_scene* S, int c) { return S->cath[c].h_monotone; }
double or_sigma(const or_scene* S, int c, double g) { return sigma_of_g(S, &S->cath[c], g); }
double or_K(const or_scene* S, int c, double v) { return K_of_v(S, &S->cath[c], v); }
void or_envelope(const or_scene* S, int c, double v, double* A, double* B) { envelope(S, &S->cath[c], v, A, B); }
double or_lambda(const or_scene* S, int inst, double v)
{
    return lambda_m(S, &S->cath[S->inst[inst].cathode], &S->inst[inst], v);
}
double or_rel_speed_pdf(double g, double v, double s) { return rel_speed_pdf(g, v, s); }

int or_hit(const or_scene* S, int geom, const double* p, const double* d, double ell, int exclude, double* t)
{
    return hit_test(S, &S->geoms[geom], p, d, ell, exclude, t);
}

void or_collide(const or_scene* S, int c, const double* v, const double* V, double u_b, double u_psi, double* v_out,
                double* V_out, double* chi)
{
    collide_with(S, &S->cath[c], v, V, u_b, u_psi, v_out, V_out, chi);
}

/* draw the gas partner of collision `event` for particle (inst, pid) */
int or_partner(const or_scene* S, uint64_t seed, int inst, uint64_t pid, uint32_t event, const double* v, double* V)
{
    stream_t st = {{(uint32_t)seed, (uint32_t)(seed >> 32)}, (uint32_t)pid, S->inst[inst].stream};
    return sample_partner(S, &S->cath[S->inst[inst].cathode], &st, event, v, V);
}

/* repeated collisions in an unbounded gas (no surfaces, no flights): the
 * speed after each of n_coll collisions is written to speeds[0..n_coll) */
void or_thermalize(const or_scene* S, uint64_t seed, int inst, uint64_t pid, double E0, int n_coll, double* speeds)
{
    const cath_t* c = &S->cath[S->inst[inst].cathode];
    stream_t st = {{(uint32_t)seed, (uint32_t)(seed >> 32)}, (uint32_t)pid, S->inst[inst].stream};
    double v[3] = {0.0, 0.0, speed_of_E(E0, c->mass)};
    uint32_t w[4];
    for (int k = 1; k <= n_coll; ++k) {
        draw(&st, (uint32_t)k, 0u, w);
        double V[3], vo[3], Vo[3];
        sample_partner(S, c, &st, (uint32_t)k, v, V);
        collide_with(S, c, v, V, rn(w[1]), rn(w[2]), vo, Vo, NULL);
        memcpy(v, vo, sizeof v);
        speeds[k - 1] = sqrt(dot3(v, v));
    }
}

/* launch state of particle (inst, pid): position, direction, energy */
void or_launch(const or_scene* S, uint64_t seed, int ii, uint64_t pid, double* p, double* d, double* E)
{
    const inst_t* I = &S->inst[ii];
    const cath_t* c = &S->cath[I->cathode];
    stream_t st = {{(uint32_t)seed, (uint32_t)(seed >> 32)}, (uint32_t)pid, S->inst[ii].stream};
    uint32_t w[4];
    draw(&st, 0u, 0u, w);
    double r = or_racetrack_r(c->rt_r0, c->rt_sigma, c->rt_R, rn(w[0]));
    double al = 2.0 * M_PI * rn(w[1]);
    double mu;
    if (c->lt) table_launch(c, rn(w[3]), rn(w[2]), &mu, E);
    else {
        *E = S->at_cutoff ? I->E_max : or_thompson(I->E_max, c->U_s, rn(w[2]));
        mu = or_cos_mu(c->coef, rn(w[3]));
    }
    draw(&st, 0u, 1u, w);
    double ph = 2.0 * M_PI * rn(w[0]);
    double s = sqrt((1.0 - mu) * (1.0 + mu));
    for (int a = 0; a < 3; ++a) {
        p[a] = c->c[a] + r * cos(al) * c->e1[a] + r * sin(al) * c->e2[a];
        d[a] = s * cos(ph) * c->e1[a] + s * sin(ph) * c->e2[a] + mu * c->n[a];
    }
}

/* per-flight trace of particle (inst, pid): rows x 10 doubles, unused rows status -2 */
void or_trace(const or_scene* S, uint64_t seed, int inst, uint64_t pid, int rows, double* out)
{
    for (int r = 0; r < rows; ++r) {
        memset(out + 10 * r, 0, 10 * sizeof(double));
        out[10 * r + 7] = -2.0;
    }
    outcome_t o;
    transport_one(S, seed, inst, pid, &o, out, rows);
}

/* quadrature self-test integrands */
static double qt_f(double x, const void* ctx)
{
    int which = *(const int*)ctx;
    if (which == 0) return exp(x);
    if (which == 1) return 1.0 / (1.0 + x * x);
    return sqrt(x);
}

double or_integrate_test(int which, double a, double b) { return integrate(qt_f, &which, a, b, 1e-13); }
