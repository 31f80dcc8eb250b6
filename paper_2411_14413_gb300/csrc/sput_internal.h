// sput_internal.h -- device-side scene layout shared by the host library and
// the CUDA kernels of libsput.so (not part of the public ABI).
#pragma once

#include <cstdint>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "sput.h"

namespace sput {

// Scattering integral: Gauss-Mehler (Gauss-Chebyshev) quadrature with
// kGMNodes nodes on [-1,1]; by symmetry kGMNodes/2 evaluations.  Below
// ln eps = kGMLoLnEps the 16-node rule already meets the FP32 rounding level
// (quadrature error < 2e-7 rad over all impact parameters, against < 4e-7
// for the 32-node rule up to ln eps = -3), so it is used there.
constexpr int kGMNodes = 32;
constexpr int kGMHalf = kGMNodes / 2;
constexpr int kGMNodesLo = 16;
constexpr int kGMHalfLo = kGMNodesLo / 2;
constexpr float kGMLoLnEps = -7.0f;
// Newton steps for the apsis from the head-on lower bound (converges to
// < 2e-8 relative within 5 steps over the whole eps, b range; one spare).
constexpr int kApsisIters = 6;

// Deflection table of the Moliere potential, q = ln tan(chi/2) over
// x = ln eps and y = ln(b / b_max(eps)) (b_max: chi(eps, b_max) = chi_min), bicubic
// cells: x in [kChiX0, kChiX0 + kChiNx kChiHx] in steps of kChiHx; y in [kChiY0, kChiY1]
// in steps of kChiHyC, then in [kChiY1, 0] in steps of kChiHyF, where screening
// makes chi fall from tenths of a radian to chi_min over a few hundredths of y at
// small eps.  Outside (rare) the device integrates the deflection directly.  The
// steps are powers of two, so node positions and cell indices are exact in FP32.
constexpr float kChiX0 = -26.0f, kChiHx = 0.25f;
constexpr int kChiNx = 88;
constexpr float kChiY0 = -6.0f, kChiY1 = -1.0f, kChiHyC = 0.03125f, kChiHyF = 0.0078125f;
constexpr int kChiNyC = 160, kChiNyF = 128, kChiNy = kChiNyC + kChiNyF;
constexpr int kChiCells = kChiNx * kChiNy;

// Moliere screening: Phi(x) = sum c_i exp(-d_i x) (Moliere 1947).
constexpr float kMolC0 = 0.35f, kMolC1 = 0.55f, kMolC2 = 0.10f;
constexpr float kMolD0 = 0.3f, kMolD1 = 1.2f, kMolD2 = 6.0f;

// Envelope of the gas-partner rejection (see envelope64 in sput_tables.h): H sampled at
// kEnvN + 1 points of rho = |V|/s in [0, kEnvRhoMax], the line raised by kEnvMargin;
// kEnvM = 2 sqrt(2/pi), the mean of |V|/s under the Maxwellian.
constexpr int kEnvN = 512;
constexpr double kEnvRhoMax = 8.0;
constexpr double kEnvMargin = 1e-4;
constexpr double kEnvM = 1.5957691216057308;

// Device status bits (sput_run_stats.device_status).
enum : uint32_t {
    kStatusNonFinite = 1u << 0,   // a particle state became NaN/Inf; the particle was retired as timed out
    kStatusBadIndex = 1u << 1,    // a tally or table index fell outside its buffer; the write was skipped
};

// One primitive, 80 bytes; n = u x v precomputed; (bx, by, bz, br) bounds it.
struct alignas(16) DevPrim {
    float cx, cy, cz;
    int kind;
    float ux, uy, uz;
    float p0;
    float vx, vy, vz;
    float p1;
    float nx, ny, nz;
    float p0sq;  // disc: inner radius^2; cylinder: radius^2
    float bx, by, bz, br;  // bounding sphere (centre, radius); unused for the box
};

struct alignas(16) DevGeom {
    int begin, count, substrate;
    int cell_base;  // offset of this geometry's cell masks in Params::cell_mask (-1: none)
};

struct alignas(16) DevCathode {
    float c[3], n[3], e1[3], e2[3];
    // racetrack: inverse radial CDF as cubic pieces, rt_n per half (see rt_tab of Params)
    float rt_R;
    // joint (mu, E) launch table: float offset in Params::lt_tab of the marginal CDF over
    // lt_nmu cells of mu (lt_nmu + 1 values) followed by lt_nmu conditional CDFs over
    // lt_nE energy cells (lt_nE + 1 values each); lt_off < 0 = Thompson law + cosine sum
    int lt_off, lt_nmu, lt_nE;
    float lt_dE;                           // eV per energy cell
    float rt_pad[7];
    float coef[6];
    float coef_norm;                       // sum c_i/(i+1)
    int cos_general;                       // 0 = pure cosine (mu = sqrt(u))
    int target;                            // local index of the target disc
    int pair;                              // interaction pair (tables)
    int rt_tab;                            // float4 offset of this cathode's 2 rt_n racetrack pieces
    int pad0;
    float v_per_sqrtE;                     // speed (km/s) = v_per_sqrtE * sqrt(E / eV)
    float E_per_v2;                        // E (eV) = E_per_v2 * v^2
    float pad1, pad2;
};

struct alignas(16) DevPair {
    float kappa;        // eps = kappa * g^2 (g in km/s)
    float ln_kappa;
    float sigma_scale;  // sigma (A^2) = sigma_scale * (b_max/a)^2  (hard sphere: pi d^2)
    float m1M;          // m1 / (m1 + m2)
    float m2M;          // m2 / (m1 + m2)
    int hard_sphere;
    int K_off;          // float4 offset of the <sigma g>(w) table
    int A_off, B_off;   // float4 offsets of the rejection-envelope coefficient tables A(w), B(w)
    int n_w;            // intervals of the w tables
    float w_inv_h;      // 1 / Delta w
    float inv_s;        // 1 / s_gas, w = ln(1 + v / s_gas)
    int G_off;          // float4 offset of the d ln K / d ln s table (zero for a gas at rest)
    float sigma_D;      // diffusion cross section (A^2) of the thermalised-atom shortcut: 1/lambda_D = n sigma_D
    float pad_d[2];
};

struct alignas(16) DevInstance {
    int geometry, cathode, pair;
    uint32_t n;           // particles
    float ng14;           // n_gas (mm^-3) * 1e-14: inverse mean free path = ng14 * K / v
    float thompson_q;     // E_max / (E_max + U_s)
    float U_s;
    float kLambda;        // d E_max / d E_i = k Lambda
    unsigned long long ticket_begin;
    uint32_t stream;      // word 1 of every Philox counter of this instance's particles
    uint32_t pad2;
};

// Everything the transport kernel needs; passed by value (kernel parameter).
struct Params {
    // scene (device pointers)
    const DevPrim* prims;
    const DevGeom* geoms;
    const DevCathode* cath;
    const DevPair* pairs;
    const DevInstance* inst;
    const unsigned long long* prefix;  // n_inst + 1 ticket offsets
    const float4* bm_tab;              // n_bm cubic pieces of b_max/a over ln eps
    const float* xh_tab;               // n_bm + 1 head-on apsis values (linear)
    const float4* w_tab;               // all pairs' K and M pieces, then their d ln K/d ln s pieces
    const float4* rt_tab;              // racetrack inverse-CDF pieces (2 rt_n per cathode)
    const float* lt_tab;               // joint launch-table CDFs (see DevCathode::lt_off)
    const float4* chi_tab;             // deflection table: kChiCells cells of 4 float4 (null: hard spheres)
    // cell masks of the surface test (null: off): per geometry and cell of a uniform grid over
    // the chamber, the local primitives a flight of length <= h (word 0) or <= 2 h (word 1)
    // starting in the cell can reach
    const unsigned long long* cell_mask;
    float cell_lo[3], cell_h, cell_inv_h;
    int cell_n[3];
    int n_prims, n_geoms, n_pairs, n_inst;
    int n_bm;
    int n_w_all, n_rt_all, n_lt_all;   // entries of w_tab, rt_tab and lt_tab (bounds of the checked build)
    float bm_lo, bm_inv_h;
    float box_lo[3], box_hi[3];
    float s_gas;
    float inv_T, inv_s2;               // 1/T (1/K), 1/s_gas^2
    int gas_thermal;
    int max_attempts;
    int max_prims;
    long long max_collisions;
    int rt_n;                          // racetrack pieces per half
    // grid
    int nx, ny;
    float half_u, half_v, cells_per_mm_u, cells_per_mm_v;
    int n_ebins, n_abins;
    float ebin_per_eV;
    // tallies (caller-owned device memory, may be null)
    void* counts;
    double* energy;
    double* score;
    double* score_T;                   // temperature score tally (null = off)
    long long* prim_counts;
    long long* timed_out;
    long long* hist_E;
    long long* hist_A;
    sput_record* records;
    // run
    uint32_t key0, key1;
    // the Philox key schedule of this seed, (key0 + r W0, key1 + r W1) for rounds r = 0..9,
    // set by set_philox_keys (the kernel reads it from the parameter bank)
    uint32_t rk0[10], rk1[10];
    unsigned long long ticket_begin, ticket_end;
    int chunk;
    int smem_counters;                 // prim/timed-out counters privatised in shared memory
    int launch_at_cutoff;              // launch energy = E_max (SPUT_RUN_LAUNCH_AT_CUTOFF)
    float E_switch;                    // eV; below it after a collision the atom turns diffusive (0 = off)
    int inject_nonfinite;              // SPUT_RUN_INJECT_NONFINITE: particle 0 of each instance starts with a NaN speed
    // scratch (library-owned device memory)
    unsigned long long* ticket_counter;
    unsigned long long* stats;         // [particles, landed, timed_out, flights, collisions, attempts]
    unsigned int* status;
    // Gauss-Mehler node constants per evaluation j: (u_j, 1/(1+u_j), u_j/(1-u_j^2), 1/u_j - 1)
    float4 gm[kGMHalf];       // kGMNodes-point rule
    float4 gm_lo[kGMHalfLo];  // kGMNodesLo-point rule (ln eps < kGMLoLnEps)
};

constexpr int kNumStats = 6;
// rows of one SPUT_PROBE_TRACE record (launch state + 63 flights)
constexpr int kTraceRows = 64;

// Launchers implemented in sput_transport.cu.
int transport_configure(int max_dynamic_smem);
int transport_launch(const Params& p, int count64, int blocks, int threads, size_t smem, void* stream);
// (the launch picks the kernel instance with the temperature score when p.score_T is set)
size_t transport_smem_bytes(const Params& p);
int transport_max_blocks_per_sm(int count64, int threads, size_t smem);
int probe_launch(const Params& p, int what, int idx, int n, const double* x_dev, double* y_dev, void* stream);

// Device copy of the scene's instance table (for the adjoint kernels).
const DevInstance* scene_device_instances(const sput_scene* scene);

// NVTX range over one entry point (scene upload, run, backward): shows the
// library's calls on a profiler timeline; header-only, no cost without a tool.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Error text for sput_last_error from other translation units.
void set_last_error(const char* msg);

// Static run scratch of sput_run_noalloc (module memory, no allocation).
constexpr size_t kRunScratchBytes = 64;      // ticket counter + kNumStats statistics + status word
constexpr size_t kStaticScratchBytes = 256;  // capacity of the static array
// Device address of the static scratch for `device` (must be current); looked
// up with cudaGetSymbolAddress on the first call in each CUDA context of the
// device, then cached under the context's id (a reset device gets a new one).
int static_scratch_address(int device, unsigned long long** out);

}  // namespace sput
