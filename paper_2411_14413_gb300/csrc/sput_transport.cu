// sput_transport.cu -- persistent Monte Carlo transport kernel for sm_103a.
//
// One thread carries one sputtered atom at a time; a warp refills its dead
// lanes from a warp-private pool of tickets that it takes in chunks from one
// global counter, so every lane runs exactly one free flight per loop
// iteration (Sec. "The SIMTRA model": launch, free flight, surface test,
// binary collision, repeated until the atom lands).  The geometry and the small
// interaction tables are staged in shared memory; the rate tables, the
// deflection table and the cell masks are read through L1/L2.  The scattering
// angle comes from a bicubic table of ln tan(chi/2) built from the classical
// deflection integral, and from Gauss-Mehler quadrature in FP32 outside the
// table's range.  Counts are integer atomics (bit-exact, order independent);
// energy and score sums are FP64 atomics.
#include <cuda.h>
#include <cuda_runtime.h>
#include <math_constants.h>

#include <cstdint>
#include <map>
#include <mutex>
#include <utility>

#include "sput_internal.h"

namespace sput {

namespace {

constexpr unsigned kFull = 0xffffffffu;
// kernel instances: the exact transport, with the temperature score, or with the
// diffusion shortcut for thermalised atoms (the two options exclude each other)
enum { kModePlain = 0, kModeScoreT = 1, kModeWalk = 2 };

// ----------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of two 32x32
// multiplies with the published multipliers, keyed by the seed's key schedule
// (Weyl increments), which the host writes into the kernel parameters
// (set_philox_keys): each round's key is an operand from the parameter bank, not
// an addition.  Inlined: an out-of-line call made the caller save registers
// around it at 64 registers a thread.
__device__ __forceinline__ uint4 philox(const Params& P, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
        c0 = hi1 ^ c1 ^ P.rk0[r];
        c1 = lo1;
        c2 = hi0 ^ c3 ^ P.rk1[r];
        c3 = lo0;
    }
    return make_uint4(c0, c1, c2, c3);
}

// RN in ]0,1]: ((x >> 8) + 1) 2^-24, exact in FP32
__device__ __forceinline__ float rn(uint32_t x) { return (float)((x >> 8) + 1u) * 5.9604644775390625e-8f; }

// ------------------------------------------------------------- checked build
// Built with SPUT_CHECKED, every table window, cell, primitive, instance,
// counter and record index is tested against its buffer before the access: an
// index outside sets kStatusBadIndex in the run's status word and the access
// is skipped (a read falls back to index 0, a write is dropped), so the run
// ends normally and the call reports SPUT_ERR_DEVICE_CHECK.  The regular build
// compiles every test to true.
__device__ __forceinline__ bool idx_ok(unsigned int* status, long long i, long long n)
{
#ifdef SPUT_CHECKED
    if (i >= 0 && i < n) return true;
    if (status) atomicOr(status, kStatusBadIndex);  // the probe kernel runs without a status word
    return false;
#else
    (void)status;
    (void)i;
    (void)n;
    return true;
#endif
}

// ------------------------------------------------------------- tables
__device__ __forceinline__ float cubic_eval(const float4* tab, int n, float x)
{
    // x in piece units; clamped to [0, n]
    x = fminf(fmaxf(x, 0.0f), (float)n);
    int i = min((int)x, n - 1);
    float t = x - (float)i;
    float4 c = tab[i];
    return fmaf(t, fmaf(t, fmaf(t, c.w, c.z), c.y), c.x);
}

struct TableView {
    const float4* bm;
    const float* xh;
    const float4* w;
    const float4* gm;  // Gauss-Mehler nodes: kGMHalf of the kGMNodes rule, then kGMHalfLo of the kGMNodesLo rule
    const DevPair* pairs;
    const DevGeom* geoms;
    int n_bm;
    int n_w;           // entries of w (bounds of the checked build)
    float bm_lo, bm_inv_h;
    unsigned int* status;
    const uint32_t* stream;  // Philox stream word per instance (shared memory), or null: read P.inst
};

// word 1 of the Philox counters of instance `inst`'s particles
__device__ __forceinline__ uint32_t stream_of(const TableView& T, const Params& P, uint32_t inst)
{
    return T.stream ? T.stream[inst] : P.inst[inst].stream;
}

__device__ __forceinline__ float bmax_eval(const TableView& T, float ln_eps)
{
    return cubic_eval(T.bm, T.n_bm, (ln_eps - T.bm_lo) * T.bm_inv_h);
}

__device__ __forceinline__ float xh_eval(const TableView& T, float ln_eps)
{
    float x = fminf(fmaxf((ln_eps - T.bm_lo) * T.bm_inv_h, 0.0f), (float)T.n_bm);
    int i = min((int)x, T.n_bm - 1);
    float t = x - (float)i;
    return fmaf(t, T.xh[i + 1] - T.xh[i], T.xh[i]);
}

// The rate tables' coordinate w = ln(1 + v/s), from the MUFU logarithm: its error
// (about 4e-7 absolute) moves K, A and B far less than their interpolation error.
__device__ __forceinline__ float w_of(const DevPair& pr, float v) { return __logf(1.0f + v * pr.inv_s); }

// K(v), A(v) or B(v) of a pair: cubic pieces in w = ln(1 + v/s), at a given w.  The
// tables are read through L1 from global memory (a few KB per pair, L1-resident), which
// keeps them out of shared memory so that four blocks fit on an SM.
__device__ __forceinline__ float wtab_at(const TableView& T, const DevPair& pr, int off, float w)
{
    if (!idx_ok(T.status, (long long)off + pr.n_w - 1, T.n_w) || !idx_ok(T.status, off, T.n_w)) return 0.0f;
    const float x = fminf(fmaxf(w * pr.w_inv_h, 0.0f), (float)pr.n_w);
    const int i = min((int)x, pr.n_w - 1);
    const float t = x - (float)i;
    const float4 c = __ldg(T.w + off + i);
    return fmaf(t, fmaf(t, fmaf(t, c.w, c.z), c.y), c.x);
}

__device__ __forceinline__ float wtab_eval(const TableView& T, const DevPair& pr, int off, float v)
{
    return wtab_at(T, pr, off, w_of(pr, v));
}

// sigma(g) g in A^2 km/s
__device__ __forceinline__ float h_of_g(const TableView& T, const DevPair& pr, float g, float g2)
{
    if (pr.hard_sphere) return pr.sigma_scale * g;
    float b = bmax_eval(T, __logf(pr.kappa * g2));
    return pr.sigma_scale * b * b * g;
}

// 1 - exp(-y) without cancellation for small y
__device__ __forceinline__ float one_minus_exp_neg(float y)
{
    if (y < 0.5f) {
        float s = 1.0f - y * (1.0f / 10.0f);
        s = 1.0f - y * (1.0f / 9.0f) * s;
        s = 1.0f - y * (1.0f / 8.0f) * s;
        s = 1.0f - y * (1.0f / 7.0f) * s;
        s = 1.0f - y * (1.0f / 6.0f) * s;
        s = 1.0f - y * (1.0f / 5.0f) * s;
        s = 1.0f - y * (1.0f / 4.0f) * s;
        s = 1.0f - y * (1.0f / 3.0f) * s;
        s = 1.0f - y * (1.0f / 2.0f) * s;
        return y * s;
    }
    return 1.0f - expf(-y);
}

// CM deflection for the Moliere potential in reduced units (eps, beta), in
// units of pi: apsis by Newton from the head-on lower bound max(beta, x_h),
// then the Gauss-Mehler sum chi / pi = (2 / N) sum_j D_j / (S_j (S_j + beta/x0))
// with N = kGMNodesLo below ln eps = kGMLoLnEps, else kGMNodes (2/N is a power
// of two, so the scaling is exact).
__device__ float chi_over_pi_moliere(float eps, float ln_eps, float beta, float xh, const float4* gm)
{
    const float ie = 1.0f / eps;
    const float b2 = beta * beta;
    float x = fmaxf(beta, xh);
    // Terms of Phi with d_i = 1.2 and 6.0 are dropped, lane by lane, where their
    // share of the potential is below 1e-8: c_i d_i e^{-d_i x} < 1e-8 c_0 d_0 e^{-d_0 x}
    // for x > 23 (d = 1.2) and x > 4 (d = 6.0).  Both x-bounds hold from the start
    // of the apsis iteration onwards because x only grows from max(beta, x_h).
    const bool t1 = x < 23.0f, t2 = x < 4.0f;
    // loops are not unrolled: a compact kernel misses the instruction cache less
#pragma unroll 1
    for (int it = 0; it < kApsisIters; ++it) {
        float e0 = kMolC0 * expf(-kMolD0 * x);
        float e1 = t1 ? kMolC1 * expf(-kMolD1 * x) : 0.0f;
        float e2 = t2 ? kMolC2 * expf(-kMolD2 * x) : 0.0f;
        float ph = e0 + e1 + e2;
        float dph = -(kMolD0 * e0 + kMolD1 * e1 + kMolD2 * e2);
        float ix = __frcp_rn(x);
        float ix2 = ix * ix;
        float g = 1.0f - b2 * ix2 - ph * ix * ie;
        float gp = 2.0f * b2 * ix2 * ix - (dph * x - ph) * ix2 * ie;
        x -= __fdividef(g, gp);
    }
    const float x0 = x;
    const float bt = beta / x0;
    const float bt2 = bt * bt;
    const float iex = ie / x0;
    const bool u1 = x0 < 23.0f, u2 = x0 < 4.0f;
    const float p0 = kMolC0 * expf(-kMolD0 * x0) * iex;
    const float p1 = u1 ? kMolC1 * expf(-kMolD1 * x0) * iex : 0.0f;
    const float p2 = u2 ? kMolC2 * expf(-kMolD2 * x0) * iex : 0.0f;
    const float y0 = kMolD0 * x0, y1 = kMolD1 * x0, y2 = kMolD2 * x0;
    const bool lo = ln_eps < kGMLoLnEps;
    const float4* nodes = lo ? gm + kGMHalf : gm;
    const int nh = lo ? kGMHalfLo : kGMHalf;
    float s = 0.0f;
#pragma unroll 1
    for (int j = 0; j < nh; ++j) {
        const float4 nd = nodes[j];  // (u, 1/(1+u), u/(1-u^2), 1/u - 1)
        float D = p0 * fmaf(nd.z, one_minus_exp_neg(y0 * nd.w), nd.y);
        if (u1) D = fmaf(p1, fmaf(nd.z, one_minus_exp_neg(y1 * nd.w), nd.y), D);
        if (u2) D = fmaf(p2, fmaf(nd.z, one_minus_exp_neg(y2 * nd.w), nd.y), D);
        // S = sqrt(q), q = (beta/x0)^2 + D > 0; approximate reciprocal square root
        // and division (2 ulp) are well inside the quadrature error
        const float q = bt2 + D;
        const float S = q * rsqrtf(q);
        s += __fdividef(D, S * (S + bt));
    }
    return s * (lo ? 2.0f / (float)kGMNodesLo : 2.0f / (float)kGMNodes);
}

// Deflection from the table: q = ln tan(chi/2) at x = ln eps, y = ln(b/b_max) (y <= 0),
// bicubic in the cell; false outside the table (the caller integrates instead).
__device__ __forceinline__ bool chi_table_q(const float4* tab, unsigned int* status, float x, float y, float& q)
{
    const float fx = (x - kChiX0) * (1.0f / kChiHx);
    if (!(fx >= 0.0f && fx < (float)kChiNx && y >= kChiY0)) return false;
    const int i = min((int)fx, kChiNx - 1);
    const float tx = fx - (float)i;
    int j;
    float ty;
    if (y < kChiY1) {
        const float fy = (y - kChiY0) * (1.0f / kChiHyC);
        j = min((int)fy, kChiNyC - 1);
        ty = fy - (float)j;
    } else {
        const float fy = (y - kChiY1) * (1.0f / kChiHyF);
        j = min((int)fy, kChiNyF - 1);
        ty = fminf(fy - (float)j, 1.0f);
        j += kChiNyC;
    }
    const int cell = i * kChiNy + j;
    if (!idx_ok(status, cell, kChiCells)) return false;
    const float4* c = tab + 4 * cell;
    const float4 r0 = __ldg(c), r1 = __ldg(c + 1), r2 = __ldg(c + 2), r3 = __ldg(c + 3);
    const float c0 = fmaf(ty, fmaf(ty, fmaf(ty, r0.w, r0.z), r0.y), r0.x);
    const float c1 = fmaf(ty, fmaf(ty, fmaf(ty, r1.w, r1.z), r1.y), r1.x);
    const float c2 = fmaf(ty, fmaf(ty, fmaf(ty, r2.w, r2.z), r2.y), r2.x);
    const float c3 = fmaf(ty, fmaf(ty, fmaf(ty, r3.w, r3.z), r3.y), r3.x);
    q = fmaf(tx, fmaf(tx, fmaf(tx, c3, c2), c1), c0);
    return true;
}

// cos and sin of the deflection from q = ln tan(chi/2): with T = e^q,
// cos chi = (1 - T^2)/(1 + T^2), sin chi = 2T/(1 + T^2)
__device__ __forceinline__ void chi_cos_sin(float q, float& cc, float& sc)
{
    const float Tq = __expf(fminf(q, 40.0f));
    const float T2 = Tq * Tq;
    const float inv = __fdividef(1.0f, 1.0f + T2);
    cc = (1.0f - T2) * inv;
    sc = 2.0f * Tq * inv;
}

// (sin 2 pi u, cos 2 pi u) for u in (0, 1] from the MUFU sine and cosine, whose
// absolute error bound (about 2^-21.4) holds on [-pi, pi]: 2 pi u = 2 pi (u - 1/2) + pi,
// and u - 1/2 is exact for u = m 2^-24
__device__ __forceinline__ void sincos_2pi_fast(float u, float* s, float* c)
{
    float ss, cc;
    __sincosf(6.283185307179586f * (u - 0.5f), &ss, &cc);
    *s = -ss;
    *c = -cc;
}

// -ln u for u in (0, 1] from the MUFU logarithm (absolute error about 2^-21.4 near 1,
// 3 ulp elsewhere), clamped at 0 where the approximation rounds above zero
__device__ __forceinline__ float neg_log_fast(float u) { return fmaxf(-__logf(u), 0.0f); }

// sqrt(x) for x >= 0 as x / sqrt(x) from the MUFU reciprocal square root (about 2 ulp); 0 at 0
__device__ __forceinline__ float sqrt_fast(float x) { return x > 0.0f ? x * rsqrtf(x) : 0.0f; }

// orthonormal pair perpendicular to unit n (Duff et al., JCGT 6(1), 2017)
__device__ __forceinline__ void onb(float nx, float ny, float nz, float3& b1, float3& b2)
{
    float sgn = copysignf(1.0f, nz);
    float a = __fdividef(-1.0f, sgn + nz);
    float b = nx * ny * a;
    b1 = make_float3(1.0f + sgn * nx * nx * a, sgn * b, -sgn * nx);
    b2 = make_float3(b, sgn + ny * ny * a, -ny);
}

// ------------------------------------------------------------- launch
struct Lane {
    float px, py, pz, dx, dy, dz, speed, score;
    float scoreT;  // d ln p(path)/dT (kernel instance with the temperature score only)
    bool diff;     // thermalised: random walk of the diffusion shortcut
    uint32_t pid, inst, k, ncoll;
    int geom, pair;  // geometry index (its record is read from TableView::geoms), gas pair
    float ng14, E_per_v2;
};

__device__ __forceinline__ float racetrack_r(const DevCathode& C, const float4* rt_tab, int rt_n, int n_rt_all,
                                            unsigned int* status, float u)
{
    // inverse radial CDF: cubic pieces in sqrt(u) below the median, in
    // sqrt(1-u) above it (1 - u is exact for RN = m 2^-24)
    const bool upper = u > 0.5f;
    const float q = upper ? 1.0f - u : u;
    const float x = sqrtf(q) * ((float)rt_n * 1.41421356237309515f);
    const int i = min((int)x, rt_n - 1);
    const float t = x - (float)i;
    int k = C.rt_tab + (upper ? rt_n : 0) + i;
    if (!idx_ok(status, k, n_rt_all)) k = 0;
    const float4 c = rt_tab[k];
    return fminf(fmaxf(fmaf(t, fmaf(t, fmaf(t, c.w, c.z), c.y), c.x), 0.0f), C.rt_R);
}

__device__ float cosine_sum_mu(const DevCathode& C, float u)
{
    if (!C.cos_general) return sqrtf(u);
    // bisection on the polynomial CDF sum c_i mu^{i+1}/(i+1)
    const float tgt = u * C.coef_norm;
    float lo = 0.0f, hi = 1.0f;
    for (int it = 0; it < 26; ++it) {
        float m = 0.5f * (lo + hi);
        float F = C.coef[5] * (1.0f / 6.0f);
        F = fmaf(F, m, C.coef[4] * (1.0f / 5.0f));
        F = fmaf(F, m, C.coef[3] * (1.0f / 4.0f));
        F = fmaf(F, m, C.coef[2] * (1.0f / 3.0f));
        F = fmaf(F, m, C.coef[1] * (1.0f / 2.0f));
        F = fmaf(F, m, C.coef[0]);
        F *= m;
        if (F < tgt) lo = m;
        else hi = m;
    }
    return 0.5f * (lo + hi);
}

// Inverse CDF of a piecewise-uniform density over n cells: F[0..n] the
// cumulative weights (F[0] = 0, F[n] = 1), u in ]0,1].  Returns the first cell
// i with F[i+1] >= u (cells of zero weight are never returned) and the position
// t in ]0,1] of u inside it.
__device__ int table_pick(const float* F, int n, float u, float& t)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (F[mid + 1] >= u) hi = mid;
        else lo = mid + 1;
    }
    const float f0 = F[lo], d = F[lo + 1] - f0;
    t = d > 0.0f ? fminf(fmaxf((u - f0) / d, 0.0f), 1.0f) : 1.0f;
    return lo;
}

// Joint table draw (kept out of line: rare, and off the registers of the hot loop):
// mu from the marginal CDF F (u_mu), E from the conditional CDF of the drawn mu cell (u_E).
__device__ __noinline__ void table_launch(const float* F, int nmu, int nE, float dE, float u_mu, float u_E, float& mu,
                                          float& E)
{
    float tm, te;
    const int i = table_pick(F, nmu, u_mu, tm);
    const int k = table_pick(F + (nmu + 1) + i * (nE + 1), nE, u_E, te);
    mu = ((float)i + tm) / (float)nmu;
    E = ((float)k + te) * dE;
}

__device__ void launch_state(const Params& P, const float4* rt_tab, uint32_t inst, uint32_t pid, float& px,
                             float& py, float& pz, float& dx, float& dy, float& dz, float& E)
{
    const DevInstance& I = P.inst[inst];
    const DevCathode& C = P.cath[I.cathode];
    const uint4 w0 = philox(P, pid, I.stream, 0u, 0u);
    const uint4 w1 = philox(P, pid, I.stream, 0u, 1u);
    const float r = racetrack_r(C, rt_tab, P.rt_n, P.n_rt_all, P.status, rn(w0.x));
    float sa, ca;
    sincospif(2.0f * rn(w0.y), &sa, &ca);
    float mu;
    if (C.lt_off >= 0 &&
        idx_ok(P.status, (long long)C.lt_off + (C.lt_nmu + 1) + (long long)C.lt_nmu * (C.lt_nE + 1) - 1, P.n_lt_all)) {
        table_launch(P.lt_tab + C.lt_off, C.lt_nmu, C.lt_nE, C.lt_dE, rn(w0.w), rn(w0.z), mu, E);
    } else {
        // Thompson inverse CDF at u_E; E_max itself in a boundary run
        const float s = P.launch_at_cutoff ? I.thompson_q : sqrtf(rn(w0.z)) * I.thompson_q;
        E = I.U_s * s / (1.0f - s);
        mu = cosine_sum_mu(C, rn(w0.w));
    }
    float sp, cp;
    sincospif(2.0f * rn(w1.x), &sp, &cp);
    const float st = sqrtf((1.0f - mu) * (1.0f + mu));
    const float rc = r * ca, rs = r * sa, tc = st * cp, ts = st * sp;
    px = C.c[0] + rc * C.e1[0] + rs * C.e2[0];
    py = C.c[1] + rc * C.e1[1] + rs * C.e2[1];
    pz = C.c[2] + rc * C.e1[2] + rs * C.e2[2];
    dx = tc * C.e1[0] + ts * C.e2[0] + mu * C.n[0];
    dy = tc * C.e1[1] + ts * C.e2[1] + mu * C.n[1];
    dz = tc * C.e1[2] + ts * C.e2[2] + mu * C.n[2];
}

// ------------------------------------------------------------- geometry
__device__ __forceinline__ float hit_prim(const DevPrim& Q, const Params& P, float px, float py, float pz, float dx,
                                          float dy, float dz)
{
    float t = CUDART_INF_F;
    if (Q.kind == SPUT_PRIM_BOX) {
        // approximate quotients (2 ulp): a hit distance needs no correctly rounded division
        const float tx = dx > 0.0f ? __fdividef(P.box_hi[0] - px, dx)
                                   : (dx < 0.0f ? __fdividef(P.box_lo[0] - px, dx) : CUDART_INF_F);
        const float ty = dy > 0.0f ? __fdividef(P.box_hi[1] - py, dy)
                                   : (dy < 0.0f ? __fdividef(P.box_lo[1] - py, dy) : CUDART_INF_F);
        const float tz = dz > 0.0f ? __fdividef(P.box_hi[2] - pz, dz)
                                   : (dz < 0.0f ? __fdividef(P.box_lo[2] - pz, dz) : CUDART_INF_F);
        t = fmaxf(fminf(tx, fminf(ty, tz)), 0.0f);
    } else if (Q.kind == SPUT_PRIM_CYLINDER) {
        const float wx = px - Q.cx, wy = py - Q.cy, wz = pz - Q.cz;
        const float wa = wx * Q.ux + wy * Q.uy + wz * Q.uz;
        const float da = dx * Q.ux + dy * Q.uy + dz * Q.uz;
        const float wpx = wx - wa * Q.ux, wpy = wy - wa * Q.uy, wpz = wz - wa * Q.uz;
        const float dpx = dx - da * Q.ux, dpy = dy - da * Q.uy, dpz = dz - da * Q.uz;
        const float A = dpx * dpx + dpy * dpy + dpz * dpz;
        const float B = 2.0f * (wpx * dpx + wpy * dpy + wpz * dpz);
        const float Cc = wpx * wpx + wpy * wpy + wpz * wpz - Q.p0sq;
        const float disc = B * B - 4.0f * A * Cc;
        if (A > 0.0f && disc >= 0.0f) {
            const float sq = sqrtf(disc);
            const float q = -0.5f * (B + copysignf(sq, B));
            float r1 = __fdividef(q, A), r2 = q != 0.0f ? __fdividef(Cc, q) : r1;
            const float tlo = fminf(r1, r2), thi = fmaxf(r1, r2);
            if (tlo > 0.0f && fabsf(fmaf(tlo, da, wa)) <= Q.p1) t = tlo;
            else if (thi > 0.0f && fabsf(fmaf(thi, da, wa)) <= Q.p1) t = thi;
        }
    } else {
        const float den = dx * Q.nx + dy * Q.ny + dz * Q.nz;
        if (den != 0.0f) {
            const float num = (Q.cx - px) * Q.nx + (Q.cy - py) * Q.ny + (Q.cz - pz) * Q.nz;
            const float tt = __fdividef(num, den);
            if (tt > 0.0f) {
                const float qx = fmaf(tt, dx, px) - Q.cx, qy = fmaf(tt, dy, py) - Q.cy, qz = fmaf(tt, dz, pz) - Q.cz;
                const float a1 = qx * Q.ux + qy * Q.uy + qz * Q.uz;
                const float a2 = qx * Q.vx + qy * Q.vy + qz * Q.vz;
                bool in;
                if (Q.kind == SPUT_PRIM_RECT) in = fabsf(a1) <= Q.p0 && fabsf(a2) <= Q.p1;
                else {
                    const float r2 = a1 * a1 + a2 * a2;
                    in = r2 >= Q.p0sq && r2 <= Q.p1 * Q.p1;
                }
                if (in) t = tt;
            }
        }
    }
    return t;
}

// ------------------------------------------------------------- particle start
// A prepared launch: position, direction and speed of particle (inst, pid).
struct Launch {
    float px, py, pz, dx, dy, dz, speed;
    uint32_t inst, pid;
};
constexpr int kLaunchWords = 9;  // 32-bit words of a Launch in a warp's shared-memory queue

__device__ Launch prepare_launch(const Params& P, uint32_t inst, uint32_t pid)
{
    if (!idx_ok(P.status, inst, P.n_inst)) inst = 0;
    const DevCathode& C = P.cath[P.inst[inst].cathode];
    Launch L;
    float E;
    launch_state(P, P.rt_tab, inst, pid, L.px, L.py, L.pz, L.dx, L.dy, L.dz, E);
    L.speed = C.v_per_sqrtE * sqrtf(E);
    L.inst = inst;
    L.pid = pid;
    return L;
}

// The lane takes up the prepared particle.
__device__ void start_from(Lane& S, const Params& P, const Launch& L)
{
    const uint32_t inst = L.inst;
    const DevInstance& I = P.inst[inst];
    S.inst = inst;
    S.pid = L.pid;
    S.geom = idx_ok(P.status, I.geometry, P.n_geoms) ? I.geometry : 0;
    S.pair = idx_ok(P.status, I.pair, P.n_pairs) ? I.pair : 0;
    S.ng14 = I.ng14;
    S.E_per_v2 = P.cath[I.cathode].E_per_v2;
    S.px = L.px;
    S.py = L.py;
    S.pz = L.pz;
    S.dx = L.dx;
    S.dy = L.dy;
    S.dz = L.dz;
    S.speed = L.speed;
    // failure-path test aid (SPUT_RUN_INJECT_NONFINITE): a non-finite state that the
    // flight step retires with the non-finite status bit
    if (P.inject_nonfinite && L.pid == 0u) S.speed = CUDART_NAN_F;
    S.k = 0u;
    S.ncoll = 0u;
    S.score = 0.0f;
    S.scoreT = 0.0f;
    S.diff = false;
}

__device__ void start_particle(Lane& S, const Params& P, uint32_t inst, uint32_t pid)
{
    start_from(S, P, prepare_launch(P, inst, pid));
}

// ------------------------------------------------------------- one flight
enum { kStepNone = -1, kStepCollided = 0, kStepLanded = 1, kStepTimedOut = 2 };

struct StepOut {
    float t;        // landing: distance to the hit; otherwise the flight length
    int prim;       // landing: local primitive index
    int attempts;   // partner attempts of this collision
    int nonfinite;  // the state became NaN/Inf
    float Gv;       // d ln K / d ln s at the flight's speed (temperature score only)
};

// Free flight k+1 of the atom in S and the surface test.  Landing: S keeps the
// pre-flight position and out.t is the hit distance.  Otherwise the atom moves
// to the collision point; w is the flight's Philox block (words 1 and 2, the
// impact parameter and azimuth, are used by the collision; word 3 is unused).
template <int kMode, bool kMasks>
__device__ int flight_move(Lane& S, const Params& P, const TableView& T, const DevPrim* prims, const DevPair* pairs,
                           StepOut& out, uint4& w)
{
    S.k += 1u;
    out.attempts = 0;
    out.nonfinite = 0;
    out.prim = -1;
    w = philox(P, S.pid, stream_of(T, P, S.inst), S.k, 0u);
    const DevPair pr = pairs[S.pair];
    // inverse mean free path n_g <sigma g>/v (thermal) or n_g sigma(v) (gas at rest)
    const float Kv = wtab_eval(T, pr, pr.K_off, S.speed);
    float inv_lam = P.gas_thermal ? S.ng14 * Kv / S.speed : S.ng14 * Kv;
    // diffusion shortcut: exponential steps of mean lambda_D, 1/lambda_D = n sigma_D
    if (kMode == kModeWalk && S.diff) inv_lam = S.ng14 * pr.sigma_D;
    constexpr bool kScoreT = kMode == kModeScoreT;
    const float ell = S.ng14 > 0.0f ? __fdividef(neg_log_fast(rn(w.x)), inv_lam) : CUDART_INF_F;
    // temperature score: d ln(n_g K(v)/v)/dT = (-1 + G/2)/T with n_g = p/(k_B T), G = d ln K/d ln s
    float aT = 0.0f;
    if (kScoreT) {
        // (this table stays in global memory: w_tab + G_off, read through L1)
        out.Gv = idx_ok(P.status, (long long)pr.G_off + pr.n_w - 1, P.n_w_all)
                     ? cubic_eval(P.w_tab + pr.G_off, pr.n_w, w_of(pr, S.speed) * pr.w_inv_h)
                     : 0.0f;
        aT = (0.5f * out.Gv - 1.0f) * P.inv_T;
    }

    // surface test: nearest hit, ties to the lowest index; the emitting target
    // is skipped on the first flight.  Every primitive whose bounding sphere lies
    // within min(ell, best t) is tested (margin covers FP32 rounding): no hit
    // beyond that can be the landing.
    float tb = CUDART_INF_F;
    int hb = -1;
    // the emitting target is skipped on the first flight (read only then)
    const DevGeom G = T.geoms[S.geom];
    const int excl = S.k == 1u ? P.cath[P.inst[S.inst].cathode].target : -1;
    if (!kMasks) {
        for (int li = 0; li < G.count; ++li) {
            if (li == excl) continue;
            if (!idx_ok(P.status, G.begin + li, P.n_prims)) break;
            const DevPrim& Q = prims[G.begin + li];
            if (Q.kind != SPUT_PRIM_BOX) {
                const float ex = Q.bx - S.px, ey = Q.by - S.py, ez = Q.bz - S.pz;
                const float reach = fminf(ell, tb) * 1.0001f + Q.br + 1e-3f;
                if (ex * ex + ey * ey + ez * ez > reach * reach) continue;
            }
            const float t = hit_prim(Q, P, S.px, S.py, S.pz, S.dx, S.dy, S.dz);
            if (t < tb) {
                tb = t;
                hb = li;
            }
        }
    } else {
        // candidates as 32-bit masks of local indices, visited in ascending order; a
        // flight of length <= h (2 h) takes its cell's mask of the primitives it can
        // reach, which leaves the result unchanged
        unsigned long long near = ~0ull;
        if (ell <= 2.0f * P.cell_h) {
            const int ix = min(max((int)floorf((S.px - P.cell_lo[0]) * P.cell_inv_h), 0), P.cell_n[0] - 1);
            const int iy = min(max((int)floorf((S.py - P.cell_lo[1]) * P.cell_inv_h), 0), P.cell_n[1] - 1);
            const int iz = min(max((int)floorf((S.pz - P.cell_lo[2]) * P.cell_inv_h), 0), P.cell_n[2] - 1);
            const int c = (iz * P.cell_n[1] + iy) * P.cell_n[0] + ix;
            near = __ldg(P.cell_mask + G.cell_base + 2 * c + (ell <= P.cell_h ? 0 : 1));
        }
        for (int base = 0; base < G.count; base += 32) {
            const int left = G.count - base;
            unsigned mask = left >= 32 ? 0xffffffffu : ((1u << left) - 1u);
            if (base < 64) mask &= (unsigned)(near >> base);
            if (excl >= base && excl < base + 32) mask &= ~(1u << (excl - base));
            while (mask) {
                const int li = base + __ffs(mask) - 1;
                mask &= mask - 1u;
                if (!idx_ok(P.status, G.begin + li, P.n_prims)) break;
                const DevPrim& Q = prims[G.begin + li];
                if (Q.kind != SPUT_PRIM_BOX) {
                    const float ex = Q.bx - S.px, ey = Q.by - S.py, ez = Q.bz - S.pz;
                    const float reach = fminf(ell, tb) * 1.0001f + Q.br + 1e-3f;
                    if (ex * ex + ey * ey + ez * ez > reach * reach) continue;
                }
                const float t = hit_prim(Q, P, S.px, S.py, S.pz, S.dx, S.dy, S.dz);
                if (t < tb) {
                    tb = t;
                    hb = li;
                }
            }
        }
    }
    if (hb >= 0 && tb <= ell) {
        S.score -= tb * inv_lam;
        if (kScoreT) S.scoreT -= aT * tb * inv_lam;
        out.t = tb;
        out.prim = hb;
        return kStepLanded;
    }
    out.t = ell;
    S.px = fmaf(ell, S.dx, S.px);
    S.py = fmaf(ell, S.dy, S.py);
    S.pz = fmaf(ell, S.dz, S.pz);
    S.score += 1.0f - ell * inv_lam;
    if (kScoreT) S.scoreT += aT * (1.0f - ell * inv_lam);
    if (!isfinite(S.px + S.py + S.pz + S.speed)) {
        out.nonfinite = 1;
        return kStepTimedOut;
    }
    if ((long long)S.k > P.max_collisions) return kStepTimedOut;
    return kStepCollided;
}

// correctly rounded 1/d for d = 1..33 (the values __frcp_rn gives), indexed by warp-uniform d
__constant__ float kRcpSmall[34] = {0.0f, 1.0f / 1.0f, 1.0f / 2.0f, 1.0f / 3.0f, 1.0f / 4.0f, 1.0f / 5.0f, 1.0f / 6.0f, 1.0f / 7.0f, 1.0f / 8.0f, 1.0f / 9.0f, 1.0f / 10.0f, 1.0f / 11.0f, 1.0f / 12.0f, 1.0f / 13.0f, 1.0f / 14.0f, 1.0f / 15.0f, 1.0f / 16.0f, 1.0f / 17.0f, 1.0f / 18.0f, 1.0f / 19.0f, 1.0f / 20.0f, 1.0f / 21.0f, 1.0f / 22.0f, 1.0f / 23.0f, 1.0f / 24.0f, 1.0f / 25.0f, 1.0f / 26.0f, 1.0f / 27.0f, 1.0f / 28.0f, 1.0f / 29.0f, 1.0f / 30.0f, 1.0f / 31.0f, 1.0f / 32.0f, 1.0f / 33.0f};

// position of the n-th (0-based) set bit of mask; mask has more than n set bits
__device__ __forceinline__ int nth_set_bit(unsigned mask, int n)
{
    int pos = 0;
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1)
        if (__popc(mask & ((1u << (pos + w)) - 1u)) <= n) pos += w;
    return pos;
}

// Gas partners of every lane with `need`, drawn by the whole warp: the
// Maxwellian f(V) weighted by h(g) = sigma(g) g, by rejection from the
// proposal f(V) (EA + EB rho), rho = |V|/s, where EA + EB rho bounds h over the
// relative speeds a partner of speed rho s can give (the pair's envelope tables
// at the atom's speed).  The proposal is the Maxwellian with weight EA and, with
// weight EB E[rho], its rho-weighted form, whose speed follows the chi law with
// 4 degrees of freedom.  Attempt a of a particle uses its own Philox block 1 + a:
// the upper 24 bits of the four words give two Box-Muller pairs z1..z4, the low
// bytes of words 0-2 one more uniform u that selects the branch
// (u (EA + EB E[rho]) <= EB E[rho]: rho-weighted) and, rescaled within the
// branch, is the acceptance uniform.  Maxwellian branch: V = s (z1, z2, z3);
// rho-weighted branch: V = s |z| (z1, z2, z3)/|(z1, z2, z3)|.  The first
// accepted attempt is kept (attempt A-1 if none is).  Each round spreads the
// pending particles' next attempts over all 32 lanes (consecutive attempts per
// particle, the first 32 mod np particles one more), so the result is the
// sequential rejection loop's result while every lane stays busy.  Must be
// called by all 32 lanes together.
__device__ void partner_sample_warp(bool need, const Params& P, const TableView& T, const DevPair* pairs,
                                    uint32_t pid, uint32_t strm, uint32_t k, int pair, float vx, float vy, float vz,
                                    float EA, float EB, float& Vx, float& Vy, float& Vz, int& attempts)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int A = P.max_attempts;
    unsigned pending = __ballot_sync(kFull, need);
    int next_a = 0;
    Vx = Vy = Vz = 0.0f;
    attempts = 0;
    while (pending) {
        // np pending particles share 32 lanes: the first `extra` get m + 1 lanes, the rest m
        // (small-integer quotients through a correctly rounded reciprocal from a
        // table, d = 1..33: 32/np is exact as np <= 32 divides 32 only as a power of
        // two, and (l + 1/2)/d stays at least 1/66 away from an integer for l < 32)
        const int np = __popc(pending);
        const int m = (int)(32.0f * kRcpSmall[np]);
        const int extra = 32 - m * np;
        const int cut = extra * (m + 1);
        int slot, j;
        if (lane < cut) {
            slot = (int)(((float)lane + 0.5f) * kRcpSmall[m + 1]);
            j = lane - slot * (m + 1);
        } else {
            const int r = (int)(((float)(lane - cut) + 0.5f) * kRcpSmall[m]);
            slot = extra + r;
            j = lane - cut - r * m;
        }
        const int owner = nth_set_bit(pending, slot);
        const uint32_t o_pid = __shfl_sync(kFull, pid, owner);
        const uint32_t o_strm = __shfl_sync(kFull, strm, owner);
        const uint32_t o_k = __shfl_sync(kFull, k, owner);
        const int o_pair = __shfl_sync(kFull, pair, owner);
        const float o_vx = __shfl_sync(kFull, vx, owner);
        const float o_vy = __shfl_sync(kFull, vy, owner);
        const float o_vz = __shfl_sync(kFull, vz, owner);
        const float o_A = __shfl_sync(kFull, EA, owner);
        const float o_B = __shfl_sync(kFull, EB, owner);
        const int o_next = __shfl_sync(kFull, next_a, owner);
        const int a = o_next + j;
        bool acc = false;
        float cx = 0.0f, cy = 0.0f, cz = 0.0f;
        if (a < A) {
            const uint4 wn = philox(P, o_pid, o_strm, o_k, 1u + (uint32_t)a);
            const float R0 = sqrt_fast(2.0f * neg_log_fast(rn(wn.x)));
            const float R1 = sqrt_fast(2.0f * neg_log_fast(rn(wn.z)));
            float s1, c1, s3, c3;
            sincos_2pi_fast(rn(wn.y), &s1, &c1);
            sincos_2pi_fast(rn(wn.w), &s3, &c3);
            const float z1 = R0 * c1, z2 = R0 * s1, z3 = R1 * c3, z4 = R1 * s3;
            // low bytes of words 0, 1, 2 as one more 24-bit uniform
            const uint32_t lowb = ((wn.x & 0xffu) << 24) | ((wn.y & 0xffu) << 16) | ((wn.z & 0xffu) << 8);
            const float Bm = o_B * (float)kEnvM;
            const float ut = rn(lowb) * (o_A + Bm);
            const bool weighted = ut <= Bm;
            const float r32 = z1 * z1 + z2 * z2 + z3 * z3;
            const float ir3 = r32 > 0.0f ? rsqrtf(r32) : 0.0f;
            const float r3 = r32 * ir3;
            const float rho = weighted ? sqrt_fast(r32 + z4 * z4) : r3;
            const float sc = P.s_gas * (weighted ? rho * ir3 : 1.0f);
            cx = sc * z1;
            cy = sc * z2;
            cz = sc * z3;
            const float gx = o_vx - cx, gy = o_vy - cy, gz = o_vz - cz;
            const float g2 = gx * gx + gy * gy + gz * gz;
            const int op = idx_ok(T.status, o_pair, P.n_pairs) ? o_pair : 0;
            const float hg = h_of_g(T, pairs[op], sqrt_fast(g2), g2);
            const float env = fmaf(o_B, rho, o_A);
            // the branch's own uniform, rescaled to (0, 1], times the envelope against h
            acc = (weighted ? ut * env <= Bm * hg : (ut - Bm) * env <= o_A * hg) || a == A - 1;
        }
        const unsigned accm = __ballot_sync(kFull, acc);
        const bool is_owner = (pending >> lane) & 1u;
        int src = lane, first = 0;
        bool done = false;
        if (is_owner) {
            const int my_slot = __popc(pending & lt);
            const int my_m = my_slot < extra ? m + 1 : m;
            const int my_lo = my_slot < extra ? my_slot * (m + 1) : cut + (my_slot - extra) * m;
            const unsigned range = (my_m >= 32 ? kFull : ((1u << my_m) - 1u)) << my_lo;
            const unsigned hit = accm & range;
            if (hit) {
                src = __ffs(hit) - 1;
                first = src - my_lo;
                done = true;
            } else {
                next_a += my_m;
            }
        }
        const float sx = __shfl_sync(kFull, cx, src);
        const float sy = __shfl_sync(kFull, cy, src);
        const float sz = __shfl_sync(kFull, cz, src);
        if (done) {
            Vx = sx;
            Vy = sy;
            Vz = sz;
            attempts = next_a + first + 1;
        }
        pending &= ~__ballot_sync(kFull, done);
    }
}

// Binary collision in the CM frame: rotate g = v - V by (chi, psi), |g| kept.
__device__ void scatter(Lane& S, const Params& P, const TableView& T, const DevPair& pr, float vx, float vy, float vz,
                        float Vx, float Vy, float Vz, const uint4& w)
{
    const float gx = vx - Vx, gy = vy - Vy, gz = vz - Vz;
    const float g2 = gx * gx + gy * gy + gz * gz;
    if (g2 > 0.0f) {
        const float ig = rsqrtf(g2);
        const float g = g2 * ig;
        const float hx = gx * ig, hy = gy * ig, hz = gz * ig;
        float sc, cc, sp, cp;
        const float ub = rn(w.y);  // impact parameter b = b_max sqrt(ub)
        float q;
        if (pr.hard_sphere) {
            sincospif(acosf(sqrtf(ub)) * (2.0f / 3.14159265358979f), &sc, &cc);
        } else {
            const float eps = pr.kappa * g2;
            const float le = logf(eps);
            if (chi_table_q(P.chi_tab, P.status, le, 0.5f * logf(ub), q)) {
                chi_cos_sin(q, cc, sc);
            } else {
                const float beta = bmax_eval(T, le) * sqrtf(ub);
                sincospif(chi_over_pi_moliere(eps, le, beta, xh_eval(T, le), T.gm), &sc, &cc);
            }
        }
        sincos_2pi_fast(rn(w.z), &sp, &cp);
        float3 b1, b2;
        onb(hx, hy, hz, b1, b2);
        const float gpx = g * (cc * hx + sc * (cp * b1.x + sp * b2.x));
        const float gpy = g * (cc * hy + sc * (cp * b1.y + sp * b2.y));
        const float gpz = g * (cc * hz + sc * (cp * b1.z + sp * b2.z));
        const float nvx = pr.m1M * vx + pr.m2M * Vx + pr.m2M * gpx;
        const float nvy = pr.m1M * vy + pr.m2M * Vy + pr.m2M * gpy;
        const float nvz = pr.m1M * vz + pr.m2M * Vz + pr.m2M * gpz;
        // an atom slowed to ~1e-15 km/s or below (gas at rest) would underflow the
        // squares: scale by the exact power of two 2^60 first
        const float up = nvx * nvx + nvy * nvy + nvz * nvz < 1e-30f ? 0x1p60f : 1.0f;
        const float ux = nvx * up, uy = nvy * up, uz = nvz * up;
        const float sp2 = ux * ux + uy * uy + uz * uz;
        if (sp2 > 0.0f) {
            const float is = rsqrtf(sp2);
            const float sn = sp2 * is;
            S.speed = up == 1.0f ? sn : sn * 0x1p-60f;
            S.dx = ux * is;
            S.dy = uy * is;
            S.dz = uz * is;
        } else {
            S.speed = 0.0f;  // at rest: the direction is kept
        }
    }
    ++S.ncoll;
}

// One flight of every active lane of the warp (flight, surface test, then for
// the lanes that collide: warp-wide partner sampling and the scattering).
// Must be called by all 32 lanes together; inactive lanes return kStepNone.
template <int kMode, bool kMasks>
__device__ int flight_step_warp(bool active, Lane& S, const Params& P, const TableView& T, const DevPrim* prims,
                                const DevPair* pairs, StepOut& out)
{
    uint4 w = make_uint4(0u, 0u, 0u, 0u);
    int res = kStepNone;
    out.attempts = 0;
    constexpr bool kScoreT = kMode == kModeScoreT;
    if (kScoreT) out.Gv = 0.0f;
    if (active) res = flight_move<kMode, kMasks>(S, P, T, prims, pairs, out, w);
    // a thermalised atom (diffusion shortcut) turns isotropically at the end of its step
    const bool walk = kMode == kModeWalk && res == kStepCollided && S.diff;
    const bool coll = res == kStepCollided && !walk;
    const DevPair pr = pairs[S.pair];
    const float vx = S.speed * S.dx, vy = S.speed * S.dy, vz = S.speed * S.dz;
    float Vx = 0.0f, Vy = 0.0f, Vz = 0.0f;
    if (P.gas_thermal) {
        float EA = 0.0f, EB = 0.0f;
        if (coll) {
            const float w = w_of(pr, S.speed);
            EA = wtab_at(T, pr, pr.A_off, w);
            EB = wtab_at(T, pr, pr.B_off, w);
        }
        // the owner's Philox stream word travels with it (one shuffle instead of a lookup per attempt)
        partner_sample_warp(coll, P, T, pairs, S.pid, stream_of(T, P, S.inst), S.k, S.pair, vx, vy, vz, EA, EB, Vx,
                            Vy, Vz, out.attempts);
        // partner density f_T(V) sigma(g) g / K(v): d ln/dT = (|V|^2/(2 s^2) - 3/2 - G/2)/T
        if (kScoreT && coll)
            S.scoreT += (0.5f * (Vx * Vx + Vy * Vy + Vz * Vz) * P.inv_s2 - 1.5f - 0.5f * out.Gv) * P.inv_T;
    }
    if (coll) {
        scatter(S, P, T, pr, vx, vy, vz, Vx, Vy, Vz, w);
        if (kMode == kModeWalk && S.E_per_v2 * S.speed * S.speed < P.E_switch) S.diff = true;
    } else if (walk) {
        // isotropic direction from the flight block's words 1 and 2
        const float mu = 2.0f * rn(w.y) - 1.0f;
        const float st = sqrtf(fmaxf(0.0f, (1.0f - mu) * (1.0f + mu)));
        float sp, cp;
        sincospif(2.0f * rn(w.z), &sp, &cp);
        S.dx = st * cp;
        S.dy = st * sp;
        S.dz = mu;
        ++S.ncoll;
    }
    return res;
}

// ------------------------------------------------------------- kernel
struct SmemLayout {
    size_t prims, geoms, pairs, bm, prefix, xh, gm, stream, pool, queue, counters, total;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline SmemLayout smem_layout(const Params& p)
{
    SmemLayout L;
    size_t o = 0;
    L.prims = o;
    o = align16(o + sizeof(DevPrim) * p.n_prims);
    L.geoms = o;
    o = align16(o + sizeof(DevGeom) * p.n_geoms);
    L.pairs = o;
    o = align16(o + sizeof(DevPair) * p.n_pairs);
    L.bm = o;
    o = align16(o + sizeof(float4) * p.n_bm);
    L.prefix = o;
    o = align16(o + sizeof(unsigned long long) * (p.n_inst + 1));
    L.xh = o;
    o = align16(o + sizeof(float) * (p.n_bm + 1));
    L.gm = o;
    o = align16(o + sizeof(float4) * (kGMHalf + kGMHalfLo));
    L.stream = o;
    o = align16(o + sizeof(uint32_t) * p.n_inst);
    L.pool = o;
    o = align16(o + sizeof(unsigned long long) * 4 * 8);
    L.queue = o;
    o = align16(o + sizeof(uint32_t) * kLaunchWords * 32 * 8);
    L.counters = o;
    o = align16(o + (p.smem_counters ? sizeof(unsigned int) * (size_t)p.n_inst * (p.max_prims + 1) : 0));
    L.total = o;
    return L;
}

__device__ __forceinline__ void copy16(void* dst, const void* src, size_t bytes)
{
    const uint4* s = reinterpret_cast<const uint4*>(src);
    uint4* d = reinterpret_cast<uint4*>(dst);
    for (size_t i = threadIdx.x; i < bytes / 16; i += blockDim.x) d[i] = s[i];
    const unsigned char* sb = reinterpret_cast<const unsigned char*>(src);
    unsigned char* db = reinterpret_cast<unsigned char*>(dst);
    for (size_t i = (bytes / 16) * 16 + threadIdx.x; i < bytes; i += blockDim.x) db[i] = sb[i];
}

// Persistent warp pool.  Four blocks of 256 threads per SM (32 warps, 64 registers a
// thread): the issue-bound loop gains more from the extra warps than it loses to the
// few spills at 64 registers; the lane state is kept small for it (a geometry index
// instead of the geometry's fields, the ticket recomputed from (instance, id), the
// warp's ticket pool in shared memory).
template <bool kCount64, int kMode, bool kMasks>
__global__ void __launch_bounds__(256, 4) transport_kernel(const Params P)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const SmemLayout L = smem_layout(P);
    DevPrim* s_prims = reinterpret_cast<DevPrim*>(smem + L.prims);
    DevGeom* s_geoms = reinterpret_cast<DevGeom*>(smem + L.geoms);
    DevPair* s_pairs = reinterpret_cast<DevPair*>(smem + L.pairs);
    float4* s_bm = reinterpret_cast<float4*>(smem + L.bm);
    unsigned long long* s_prefix = reinterpret_cast<unsigned long long*>(smem + L.prefix);
    float* s_xh = reinterpret_cast<float*>(smem + L.xh);
    float4* s_gm = reinterpret_cast<float4*>(smem + L.gm);
    uint32_t* s_stream = reinterpret_cast<uint32_t*>(smem + L.stream);
    unsigned long long* s_pool = reinterpret_cast<unsigned long long*>(smem + L.pool);
    uint32_t* s_queue = reinterpret_cast<uint32_t*>(smem + L.queue);
    unsigned int* s_cnt = reinterpret_cast<unsigned int*>(smem + L.counters);

    copy16(s_prims, P.prims, sizeof(DevPrim) * P.n_prims);
    copy16(s_geoms, P.geoms, sizeof(DevGeom) * P.n_geoms);
    copy16(s_pairs, P.pairs, sizeof(DevPair) * P.n_pairs);
    copy16(s_bm, P.bm_tab, sizeof(float4) * P.n_bm);
    copy16(s_prefix, P.prefix, sizeof(unsigned long long) * (P.n_inst + 1));
    copy16(s_xh, P.xh_tab, sizeof(float) * (P.n_bm + 1));
    if (threadIdx.x < kGMHalf) s_gm[threadIdx.x] = P.gm[threadIdx.x];
    else if (threadIdx.x < kGMHalf + kGMHalfLo) s_gm[threadIdx.x] = P.gm_lo[threadIdx.x - kGMHalf];
    for (int i = threadIdx.x; i < P.n_inst; i += blockDim.x) s_stream[i] = P.inst[i].stream;
    const int n_cnt = P.smem_counters ? P.n_inst * (P.max_prims + 1) : 0;
    for (int i = threadIdx.x; i < n_cnt; i += blockDim.x) s_cnt[i] = 0u;
    __syncthreads();

    TableView T;
    T.bm = s_bm;
    T.xh = s_xh;
    T.w = P.w_tab;
    T.gm = s_gm;
    T.pairs = s_pairs;
    T.geoms = s_geoms;
    T.n_bm = P.n_bm;
    T.n_w = P.n_w_all;
    T.bm_lo = P.bm_lo;
    T.bm_inv_h = P.bm_inv_h;
    T.status = P.status;
    T.stream = s_stream;

    const int lane = threadIdx.x & 31;
    const unsigned lane_lt = (1u << lane) - 1u;
    const int ncell = P.nx * P.ny;

    Lane S;
    S.px = S.py = S.pz = S.dx = S.dy = S.dz = S.speed = S.score = S.scoreT = 0.0f;
    S.pid = S.inst = S.k = S.ncoll = 0u;
    S.geom = S.pair = 0;
    S.ng14 = S.E_per_v2 = 0.0f;
    bool alive = false;

    // per-lane statistics; particles = landed + timed out, flights = landed + timed out + collided
    uint32_t c_landed = 0, c_timed = 0, c_coll = 0, c_att = 0;
    // the warp's ticket pool [next, end) lives in shared memory (warp-uniform, read only
    // when the warp refills); the pool is exhausted once its end reaches ticket_end
    // and its queue of prepared launches: s_wpool[2] entries of kLaunchWords words
    unsigned long long* s_wpool = s_pool + 4 * (threadIdx.x >> 5);
    uint32_t* s_wqueue = s_queue + kLaunchWords * 32 * (threadIdx.x >> 5);
    if (lane == 0) s_wpool[0] = s_wpool[1] = s_wpool[2] = 0ull;
    __syncwarp();

    for (;;) {
        // ---------------------------------------------------- refill (warp-uniform)
        // Dead lanes take prepared launches from the warp's queue at once.  When the
        // queue runs short, the whole warp prepares the next launches together, one
        // per lane, so the launch code runs with every lane busy instead of once for
        // a few dead lanes while the others wait.
        const unsigned need = __ballot_sync(kFull, !alive);
        if (need) {
            const unsigned n = __popc(need);
            const unsigned rank = __popc(need & lane_lt);
            unsigned qn = (unsigned)s_wpool[2];  // prepared launches in the queue (warp-uniform)
            if (qn < n) {
                // the whole warp prepares launches for up to 32 - qn new tickets, one per lane,
                // so that the launch code runs with every lane busy
                const unsigned want = 32u - qn;
                unsigned long long pool_next = s_wpool[0], pool_end = s_wpool[1];
                const bool exhausted = pool_end == P.ticket_end;
                const unsigned long long avail = pool_end - pool_next;
                unsigned long long t = ~0ull;
                if ((unsigned)lane < want && lane < avail) t = pool_next + lane;
                if (want > avail && !exhausted) {
                    const unsigned long long more = want - avail;
                    const unsigned long long grab = more > (unsigned long long)P.chunk ? more : (unsigned long long)P.chunk;
                    unsigned long long base = 0ull;
                    if (lane == 0) base = atomicAdd(P.ticket_counter, grab);
                    base = __shfl_sync(kFull, base, 0) + P.ticket_begin;
                    if ((unsigned)lane < want && lane >= avail && base + (lane - avail) < P.ticket_end)
                        t = base + (lane - avail);
                    const unsigned long long ne = base + grab < P.ticket_end ? base + grab : P.ticket_end;
                    const unsigned long long nn = base + more < ne ? base + more : ne;
                    pool_next = nn;
                    pool_end = ne;
                } else {
                    pool_next += (want < avail ? want : avail);
                }
                if (t != ~0ull) {
                    // ticket -> (instance, particle id) by binary search over the instance prefix
                    int lo = 0, hi = P.n_inst;
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        if (s_prefix[mid] <= t) lo = mid;
                        else hi = mid;
                    }
                    const Launch Ln = prepare_launch(P, (uint32_t)lo, (uint32_t)(t - s_prefix[lo]));
                    uint32_t* e = s_wqueue + kLaunchWords * (qn + lane);
                    e[0] = __float_as_uint(Ln.px);
                    e[1] = __float_as_uint(Ln.py);
                    e[2] = __float_as_uint(Ln.pz);
                    e[3] = __float_as_uint(Ln.dx);
                    e[4] = __float_as_uint(Ln.dy);
                    e[5] = __float_as_uint(Ln.dz);
                    e[6] = __float_as_uint(Ln.speed);
                    e[7] = Ln.inst;
                    e[8] = Ln.pid;
                }
                qn += __popc(__ballot_sync(kFull, t != ~0ull));  // the lanes with tickets are a prefix
                __syncwarp();
                if (lane == 0) {
                    s_wpool[0] = pool_next;
                    s_wpool[1] = pool_end;
                }
            }
            // the dead lanes take launches from the top of the queue
            if (!alive && rank < qn) {
                const uint32_t* e = s_wqueue + kLaunchWords * (qn - 1u - rank);
                Launch Ln;
                Ln.px = __uint_as_float(e[0]);
                Ln.py = __uint_as_float(e[1]);
                Ln.pz = __uint_as_float(e[2]);
                Ln.dx = __uint_as_float(e[3]);
                Ln.dy = __uint_as_float(e[4]);
                Ln.dz = __uint_as_float(e[5]);
                Ln.speed = __uint_as_float(e[6]);
                Ln.inst = e[7];
                Ln.pid = e[8];
                start_from(S, P, Ln);
                alive = true;
            }
            __syncwarp();
            if (lane == 0) s_wpool[2] = qn - (n < qn ? n : qn);
            __syncwarp();
        }
        if (!__any_sync(kFull, alive)) break;

        // ---------------------------------------------------- one flight (all lanes together)
        StepOut so;
        const int res = flight_step_warp<kMode, kMasks>(alive, S, P, T, s_prims, s_pairs, so);
        c_att += so.attempts;
        if (res == kStepLanded) {
            // ------------------------------------------------ landing tally
            const float tb = so.t;
            const int hb = so.prim;
            const float E = S.E_per_v2 * S.speed * S.speed;
            int cell = -1;
            float cosang = 0.0f;
            const DevGeom G = s_geoms[S.geom];
            if (hb == G.substrate) {
                const DevPrim& Q = s_prims[G.begin + hb];
                const float dn = S.dx * Q.nx + S.dy * Q.ny + S.dz * Q.nz;
                if (dn < 0.0f) {
                    const float qx = fmaf(tb, S.dx, S.px) - Q.cx, qy = fmaf(tb, S.dy, S.py) - Q.cy,
                                qz = fmaf(tb, S.dz, S.pz) - Q.cz;
                    const float a1 = qx * Q.ux + qy * Q.uy + qz * Q.uz;
                    const float a2 = qx * Q.vx + qy * Q.vy + qz * Q.vz;
                    const float fx = (a1 + P.half_u) * P.cells_per_mm_u;
                    const float fy = (a2 + P.half_v) * P.cells_per_mm_v;
                    if (fx >= 0.0f && fy >= 0.0f && fx <= (float)P.nx && fy <= (float)P.ny) {
                        const int ix = min((int)fx, P.nx - 1), iy = min((int)fy, P.ny - 1);
                        cell = iy * P.nx + ix;
                    }
                    cosang = -dn;
                }
            }
            if (cell >= 0 && idx_ok(P.status, (long long)S.inst * ncell + cell, (long long)P.n_inst * ncell)) {
                const size_t ci = (size_t)S.inst * ncell + cell;
                if (P.counts) {
                    if (kCount64) atomicAdd(reinterpret_cast<unsigned long long*>(P.counts) + ci, 1ull);
                    else atomicAdd(reinterpret_cast<unsigned int*>(P.counts) + ci, 1u);
                }
                if (P.energy) atomicAdd(P.energy + ci, (double)E);
                if (P.score) atomicAdd(P.score + ci, (double)S.score);
                if (kMode == kModeScoreT) atomicAdd(P.score_T + ci, (double)S.scoreT);
                if (P.hist_E) {
                    int b = min(max((int)(E * P.ebin_per_eV), 0), P.n_ebins - 1);
                    atomicAdd(reinterpret_cast<unsigned long long*>(P.hist_E) + (size_t)S.inst * P.n_ebins + b, 1ull);
                }
                if (P.hist_A) {
                    const float th = acosf(fminf(cosang, 1.0f)) * (57.29577951308232f / 90.0f);
                    int b = min(max((int)(th * (float)P.n_abins), 0), P.n_abins - 1);
                    atomicAdd(reinterpret_cast<unsigned long long*>(P.hist_A) + (size_t)S.inst * P.n_abins + b, 1ull);
                }
            }
            if (!idx_ok(P.status, hb, P.max_prims)) {
                // dropped: the checked build reports it
            } else if (P.smem_counters) atomicAdd(&s_cnt[S.inst * (P.max_prims + 1) + hb], 1u);
            else if (P.prim_counts)
                atomicAdd(reinterpret_cast<unsigned long long*>(P.prim_counts) + (size_t)S.inst * P.max_prims + hb, 1ull);
            if (P.records && idx_ok(P.status, (long long)(s_prefix[S.inst] + S.pid - P.ticket_begin),
                                    (long long)(P.ticket_end - P.ticket_begin))) {
                sput_record rec;
                rec.prim = hb;
                rec.cell = cell;
                rec.energy = E;
                rec.cos_angle = cosang;
                rec.n_collisions = S.ncoll;
                rec.score = S.score;
                P.records[s_prefix[S.inst] + S.pid - P.ticket_begin] = rec;
            }
            ++c_landed;
            alive = false;
        } else if (res == kStepTimedOut) {
            if (so.nonfinite) atomicOr(P.status, kStatusNonFinite);
            if (P.smem_counters) atomicAdd(&s_cnt[S.inst * (P.max_prims + 1) + P.max_prims], 1u);
            else if (P.timed_out) atomicAdd(reinterpret_cast<unsigned long long*>(P.timed_out) + S.inst, 1ull);
            if (P.records && idx_ok(P.status, (long long)(s_prefix[S.inst] + S.pid - P.ticket_begin),
                                    (long long)(P.ticket_end - P.ticket_begin))) {
                sput_record rec;
                rec.prim = -1;
                rec.cell = -1;
                rec.energy = S.E_per_v2 * S.speed * S.speed;
                rec.cos_angle = 0.0f;
                rec.n_collisions = S.ncoll;
                rec.score = S.score;
                P.records[s_prefix[S.inst] + S.pid - P.ticket_begin] = rec;
            }
            ++c_timed;
            alive = false;
        } else if (res == kStepCollided) {
            ++c_coll;
        }
    }

    // ---------------------------------------------------- flush counters
    unsigned long long v[kNumStats] = {c_landed + c_timed, c_landed, c_timed, c_landed + c_timed + c_coll, c_coll, c_att};
#pragma unroll
    for (int i = 0; i < kNumStats; ++i) {
        unsigned long long x = v[i];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(kFull, x, o);
        if (lane == 0 && x) atomicAdd(P.stats + i, x);
    }
    if (P.smem_counters) {
        __syncthreads();
        for (int i = threadIdx.x; i < n_cnt; i += blockDim.x) {
            const unsigned int c = s_cnt[i];
            if (!c) continue;
            const int inst = i / (P.max_prims + 1), li = i % (P.max_prims + 1);
            if (li < P.max_prims) {
                if (P.prim_counts)
                    atomicAdd(reinterpret_cast<unsigned long long*>(P.prim_counts) + (size_t)inst * P.max_prims + li,
                              (unsigned long long)c);
            } else if (P.timed_out) {
                atomicAdd(reinterpret_cast<unsigned long long*>(P.timed_out) + inst, (unsigned long long)c);
            }
        }
    }
}

// ------------------------------------------------------------- probes
__global__ void probe_kernel(const Params P, int what, int idx, int n, const double* x, double* y)
{
    __shared__ float4 s_gm[kGMHalf + kGMHalfLo];
    if (threadIdx.x < kGMHalf) s_gm[threadIdx.x] = P.gm[threadIdx.x];
    else if (threadIdx.x < kGMHalf + kGMHalfLo) s_gm[threadIdx.x] = P.gm_lo[threadIdx.x - kGMHalf];
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    TableView T;
    T.bm = P.bm_tab;
    T.xh = P.xh_tab;
    T.w = P.w_tab;
    T.gm = s_gm;
    T.pairs = P.pairs;
    T.geoms = P.geoms;
    T.n_bm = P.n_bm;
    T.n_w = P.n_w_all;
    T.bm_lo = P.bm_lo;
    T.bm_inv_h = P.bm_inv_h;
    T.status = P.status;
    T.stream = nullptr;
    if (what == SPUT_PROBE_TRACE) {
        // state after each flight of particle x[i] of instance idx, kTraceRows rows of 10;
        // the flight step is warp-collective, so lanes past n take part without a particle
        const bool valid = i < n;
        Lane S;
        S.px = S.py = S.pz = S.dx = S.dy = S.dz = S.speed = S.score = S.scoreT = 0.0f;
        S.pid = S.inst = S.k = S.ncoll = 0u;
        S.geom = S.pair = 0;
        S.ng14 = S.E_per_v2 = 0.0f;
        double* o = valid ? y + (size_t)i * kTraceRows * 10 : nullptr;
        if (valid) {
            start_particle(S, P, (uint32_t)idx, (uint32_t)x[i]);
            for (int r = 0; r < kTraceRows * 10; ++r) o[r] = 0.0;
            for (int r = 1; r < kTraceRows; ++r) o[r * 10 + 7] = -2.0;
            o[0] = S.px; o[1] = S.py; o[2] = S.pz; o[3] = S.dx; o[4] = S.dy; o[5] = S.dz; o[6] = S.speed;
            o[7] = -1.0;
        }
        bool running = valid;
        for (int r = 1; r < kTraceRows; ++r) {
            if (!__any_sync(kFull, running)) break;
            StepOut so;
            const int status = P.E_switch > 0.0f
                                   ? (P.cell_mask ? flight_step_warp<kModeWalk, true>(running, S, P, T, P.prims, P.pairs, so)
                                                  : flight_step_warp<kModeWalk, false>(running, S, P, T, P.prims, P.pairs, so))
                                   : (P.cell_mask ? flight_step_warp<kModePlain, true>(running, S, P, T, P.prims, P.pairs, so)
                                                  : flight_step_warp<kModePlain, false>(running, S, P, T, P.prims, P.pairs, so));
            if (running) {
                double* q = o + (size_t)r * 10;
                float px = S.px, py = S.py, pz = S.pz;
                if (status == kStepLanded) {
                    px = fmaf(so.t, S.dx, S.px);
                    py = fmaf(so.t, S.dy, S.py);
                    pz = fmaf(so.t, S.dz, S.pz);
                }
                q[0] = px; q[1] = py; q[2] = pz; q[3] = S.dx; q[4] = S.dy; q[5] = S.dz; q[6] = S.speed;
                q[7] = status; q[8] = status == kStepLanded ? so.prim : so.attempts; q[9] = so.t;
                if (status != kStepCollided) running = false;
            }
        }
        return;
    }
    if (i >= n) return;
    if (what == SPUT_PROBE_CHI) {
        const float eps = (float)x[2 * i], beta = (float)x[2 * i + 1];
        const float le = logf(eps);
        y[i] = 3.141592653589793 * (double)chi_over_pi_moliere(eps, le, beta, xh_eval(T, le), T.gm);
    } else if (what == SPUT_PROBE_CHI_U) {
        // the collision's path: table inside its range, direct integration outside
        const float eps = (float)x[2 * i], ub = (float)x[2 * i + 1];
        const float le = logf(eps);
        float q;
        if (chi_table_q(P.chi_tab, P.status, le, 0.5f * logf(ub), q)) {
            y[i] = 2.0 * atan(exp((double)q));
        } else {
            const float beta = bmax_eval(T, le) * sqrtf(ub);
            y[i] = 3.141592653589793 * (double)chi_over_pi_moliere(eps, le, beta, xh_eval(T, le), T.gm);
        }
    } else if (what == SPUT_PROBE_BMAX) {
        y[i] = bmax_eval(T, logf((float)x[i]));
    } else if (what == SPUT_PROBE_K) {
        const DevPair pr = P.pairs[idx];
        const float v = (float)x[i];
        float val = wtab_eval(T, pr, pr.K_off, v);
        if (!P.gas_thermal) val *= v;  // the table holds sigma(v) = K/v
        y[i] = val;
    } else if (what == SPUT_PROBE_M) {
        // rejection envelope (A, B) of the pair at speed v
        const DevPair pr = P.pairs[idx];
        const float w = w_of(pr, (float)x[i]);
        y[2 * i] = wtab_at(T, pr, pr.A_off, w);
        y[2 * i + 1] = wtab_at(T, pr, pr.B_off, w);
    } else if (what == SPUT_PROBE_LAUNCH) {
        float px, py, pz, dx, dy, dz, E;
        launch_state(P, P.rt_tab, (uint32_t)idx, (uint32_t)x[i], px, py, pz, dx, dy, dz, E);
        double* o = y + 7 * (size_t)i;
        o[0] = px;
        o[1] = py;
        o[2] = pz;
        o[3] = dx;
        o[4] = dy;
        o[5] = dz;
        o[6] = E;
    }
}

}  // namespace

size_t transport_smem_bytes(const Params& p) { return smem_layout(p).total; }

namespace {

using KernelFn = void (*)(const Params);

// the instances [count type][mode][surface-test loop]
KernelFn kernel_for(int count64, int mode, int masks)
{
    static const KernelFn tab[2][3][2] = {
        {{transport_kernel<false, kModePlain, false>, transport_kernel<false, kModePlain, true>},
         {transport_kernel<false, kModeScoreT, false>, transport_kernel<false, kModeScoreT, true>},
         {transport_kernel<false, kModeWalk, false>, transport_kernel<false, kModeWalk, true>}},
        {{transport_kernel<true, kModePlain, false>, transport_kernel<true, kModePlain, true>},
         {transport_kernel<true, kModeScoreT, false>, transport_kernel<true, kModeScoreT, true>},
         {transport_kernel<true, kModeWalk, false>, transport_kernel<true, kModeWalk, true>}}};
    return tab[count64 ? 1 : 0][mode][masks ? 1 : 0];
}

}  // namespace

int transport_max_blocks_per_sm(int count64, int threads, size_t smem)
{
    // the smallest occupancy of the instances of this count type
    int m = 1 << 30;
    for (int mode = 0; mode < 3; ++mode)
        for (int masks = 0; masks < 2; ++masks) {
            int nb = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel_for(count64, mode, masks), threads, smem) !=
                cudaSuccess)
                return 0;
            m = nb < m ? nb : m;
        }
    return m;
}

int transport_configure(int max_dynamic_smem)
{
    const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
    for (int c64 = 0; c64 < 2; ++c64)
        for (int mode = 0; mode < 3; ++mode)
            for (int masks = 0; masks < 2; ++masks) {
                const cudaError_t e = cudaFuncSetAttribute(kernel_for(c64, mode, masks), a, max_dynamic_smem);
                if (e != cudaSuccess) return (int)e;
            }
    return 0;
}

int transport_launch(const Params& p, int count64, int blocks, int threads, size_t smem, void* stream)
{
    const int mode = p.score_T ? kModeScoreT : (p.E_switch > 0.0f ? kModeWalk : kModePlain);
    kernel_for(count64, mode, p.cell_mask != nullptr)<<<blocks, threads, smem, reinterpret_cast<cudaStream_t>(stream)>>>(p);
    return (int)cudaGetLastError();
}

int probe_launch(const Params& p, int what, int idx, int n, const double* x_dev, double* y_dev, void* stream)
{
    if (n <= 0) return 0;
    probe_kernel<<<(n + 127) / 128, 128, 0, reinterpret_cast<cudaStream_t>(stream)>>>(p, what, idx, n, x_dev, y_dev);
    return (int)cudaGetLastError();
}

// ------------------------------------------------------- static run scratch
// Run scratch for sput_run_noalloc: ticket counter, statistics and status word
// in module memory, so that a run needs no device allocation at all.  Every
// device that loads the library holds these kStaticScratchBytes until the
// process exits.  In host code the name below is only a stand-in for the
// device symbol; its device address is looked up with the device current.
static __device__ __align__(256) unsigned long long g_static_run_scratch[kStaticScratchBytes / 8];

namespace {
// The address is cached per CUDA context, identified by the driver's context
// id: a context torn down and created again (cudaDeviceReset) gets a new id,
// so a stale address is never reused.  The two driver entry points are taken
// through the runtime, which needs no link against the driver library.
typedef CUresult (*PfnCtxGetCurrent)(CUcontext*);
typedef CUresult (*PfnCtxGetId)(CUcontext, unsigned long long*);

int current_context_id(unsigned long long* id)
{
    static PfnCtxGetCurrent get_current = nullptr;
    static PfnCtxGetId get_id = nullptr;
    if (!get_current || !get_id) {
        void* f0 = nullptr;
        void* f1 = nullptr;
        cudaDriverEntryPointQueryResult q0, q1;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000, cudaEnableDefault, &q0);
        if (e == cudaSuccess)
            e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault, &q1);
        if (e != cudaSuccess) return (int)e;
        if (q0 != cudaDriverEntryPointSuccess || q1 != cudaDriverEntryPointSuccess || !f0 || !f1)
            return (int)cudaErrorNotSupported;
        get_current = reinterpret_cast<PfnCtxGetCurrent>(f0);
        get_id = reinterpret_cast<PfnCtxGetId>(f1);
    }
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return (int)cudaErrorDeviceUninitialized;
    if (get_id(ctx, id) != CUDA_SUCCESS) return (int)cudaErrorDeviceUninitialized;
    return 0;
}
}  // namespace

int static_scratch_address(int device, unsigned long long** out)
{
    static std::mutex mu;
    static std::map<std::pair<int, unsigned long long>, unsigned long long*> cache;
    std::lock_guard<std::mutex> lock(mu);
    unsigned long long ctx_id = 0;
    int e0 = current_context_id(&ctx_id);
    if (e0 != 0) return e0;
    const auto key = std::make_pair(device, ctx_id);
    auto it = cache.find(key);
    if (it != cache.end()) {
        *out = it->second;
        return 0;
    }
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_run_scratch);
    if (e != cudaSuccess) return (int)e;
    cache[key] = reinterpret_cast<unsigned long long*>(ptr);
    *out = cache[key];
    return 0;
}

}  // namespace sput
