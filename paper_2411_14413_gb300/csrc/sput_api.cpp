// sput_api.cpp -- C ABI of libsput.so: scene validation and packing, device
// upload, launch of the transport kernel, statistics and diagnostics.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <thread>
#include <vector>

#include "sput.h"
#include "sput_internal.h"
#include "sput_tables.h"

using namespace sput;

namespace {

thread_local std::string g_last_error;

sput_status fail(sput_status s, const std::string& msg)
{
    g_last_error = msg;
    return s;
}

sput_status cuda_fail(cudaError_t e, const char* where)
{
    g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
    return SPUT_ERR_CUDA;
}

#define CUDA_TRY(call)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

bool finite3(const double* v) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }
double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
void cross3(const double* a, const double* b, double* o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
bool unit3(const double* v) { return finite3(v) && std::fabs(dot3(v, v) - 1.0) < 1e-6; }

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Thompson cut-off (Eq. for phi(E)): E_max = k Lambda E_i - U_s, Lambda = 4 M_i M_t / (M_i + M_t)^2
double thompson_emax(double k, double Mi, double Mt, double Ei, double Us)
{
    return k * 4.0 * Mi * Mt / ((Mi + Mt) * (Mi + Mt)) * Ei - Us;
}

// Philox4x32-10 key of a run (the seed's two 32-bit halves) and its key schedule: round r
// uses (key0 + r W0, key1 + r W1) with the published Weyl increments, modulo 2^32.
void set_philox_keys(sput::Params& p, uint64_t seed)
{
    p.key0 = (uint32_t)seed;
    p.key1 = (uint32_t)(seed >> 32);
    for (uint32_t r = 0; r < 10; ++r) {
        p.rk0[r] = p.key0 + r * 0x9E3779B9u;
        p.rk1[r] = p.key1 + r * 0xBB67AE85u;
    }
}

}  // namespace

void sput::set_last_error(const char* msg) { g_last_error = msg; }

struct sput_scene {
    int device = 0;
    int n_sm = 0;
    size_t smem_optin = 0;
    sput_chamber chamber{};
    sput_grid grid{};
    sput_physics physics{};
    std::vector<sput_primitive> prims;
    std::vector<sput_geometry> geoms;
    std::vector<sput_cathode> cathodes;
    std::vector<sput_instance> instances;
    // packed host copies
    std::vector<DevPrim> dprims;
    std::vector<DevGeom> dgeoms;
    // cell masks of the surface test (empty: a geometry has more than 64 primitives)
    std::vector<unsigned long long> cell_masks;
    double cell_lo[3] = {0, 0, 0}, cell_h = 0.0;
    int cell_n[3] = {0, 0, 0};
    std::vector<DevCathode> dcath;
    std::vector<DevPair> dpairs;
    std::vector<DevInstance> dinst;
    std::vector<unsigned long long> prefix;
    std::vector<float4> wtab;
    std::vector<float4> rt;
    std::vector<std::vector<double>> lt_weights;  // copies of the cathodes' joint launch tables
    std::vector<float> lt;                        // their CDFs (DevCathode::lt_off)
    std::vector<PairPhys> pair_phys;
    std::vector<double> pair_E_top;
    const BmaxTable* bt = nullptr;
    double s_gas = 0.0;
    int max_prims = 0;
    unsigned long long n_tickets = 0;
    // device memory
    unsigned char* d_blob = nullptr;
    size_t off_prims = 0, off_geoms = 0, off_cath = 0, off_pairs = 0, off_inst = 0, off_prefix = 0, off_bm = 0,
           off_xh = 0, off_w = 0, off_rt = 0, off_lt = 0, off_chi = 0, off_cell = 0, blob_bytes = 0;
    // run scratch (allocated on the first run): ticket counter, stats, status word
    unsigned long long* d_scratch = nullptr;
    unsigned long long* h_scratch = nullptr;  // pinned
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // device staging of sput_run_host
    void* d_stage = nullptr;
    size_t stage_bytes = 0;
    cudaStream_t own_stream = nullptr;
    Params base{};
    int smem_counters_fit = 0;  // per-primitive counters fit in shared memory
    // launch shape for opts fields left 0 (set by sput_autotune)
    int def_threads = 256, def_bps = 0, def_chunk = 32, def_flags = 0;
};

namespace {

sput_status validate(const sput_scene_desc* d)
{
    if (!d) return fail(SPUT_ERR_INVALID_ARG, "desc is NULL");
    if (d->abi_version != SPUT_ABI_VERSION) return fail(SPUT_ERR_INVALID_ARG, "abi_version mismatch");
    if (d->n_prims < 1 || d->n_geoms < 1 || d->n_cathodes < 1 || d->n_instances < 1)
        return fail(SPUT_ERR_INVALID_ARG, "scene needs at least one primitive, geometry, cathode and instance");
    if (!d->prims || !d->geoms || !d->cathodes || !d->instances)
        return fail(SPUT_ERR_INVALID_ARG, "NULL scene array");
    const sput_chamber& ch = d->chamber;
    for (int a = 0; a < 3; ++a)
        if (!(ch.box_lo[a] < ch.box_hi[a])) return fail(SPUT_ERR_INVALID_SCENE, "chamber box_lo must be < box_hi");
    if (ch.gas_Z < 1 || !(ch.gas_mass > 0.0) || !(ch.gas_T > 0.0) || !std::isfinite(ch.gas_T))
        return fail(SPUT_ERR_INVALID_SCENE, "gas Z, mass and temperature must be positive");
    for (int i = 0; i < d->n_prims; ++i) {
        const sput_primitive& P = d->prims[i];
        char buf[96];
        std::snprintf(buf, sizeof buf, "primitive %d: ", i);
        if (P.kind < SPUT_PRIM_BOX || P.kind > SPUT_PRIM_CYLINDER) return fail(SPUT_ERR_INVALID_SCENE, std::string(buf) + "bad kind");
        if (P.kind == SPUT_PRIM_BOX) continue;
        if (!finite3(P.center) || !unit3(P.u)) return fail(SPUT_ERR_INVALID_SCENE, std::string(buf) + "centre/axis not finite or u not unit");
        if (!(P.p0 >= 0.0) || !(P.p1 > 0.0) || !std::isfinite(P.p0) || !std::isfinite(P.p1))
            return fail(SPUT_ERR_INVALID_SCENE, std::string(buf) + "sizes must be finite, p0 >= 0, p1 > 0");
        if (P.kind == SPUT_PRIM_RECT || P.kind == SPUT_PRIM_DISC) {
            if (!unit3(P.v) || std::fabs(dot3(P.u, P.v)) > 1e-6) return fail(SPUT_ERR_INVALID_SCENE, std::string(buf) + "v must be unit and orthogonal to u");
            if (P.kind == SPUT_PRIM_RECT && !(P.p0 > 0.0)) return fail(SPUT_ERR_INVALID_SCENE, std::string(buf) + "rect half sizes must be > 0");
            if (P.kind == SPUT_PRIM_DISC && !(P.p0 < P.p1)) return fail(SPUT_ERR_INVALID_SCENE, std::string(buf) + "disc needs inner radius < outer radius");
        }
        if (P.kind == SPUT_PRIM_CYLINDER && !(P.p0 > 0.0)) return fail(SPUT_ERR_INVALID_SCENE, std::string(buf) + "cylinder radius must be > 0");
    }
    for (int g = 0; g < d->n_geoms; ++g) {
        const sput_geometry& G = d->geoms[g];
        if (G.prim_begin < 0 || G.prim_count < 1 || G.prim_begin + G.prim_count > d->n_prims)
            return fail(SPUT_ERR_INVALID_SCENE, "geometry primitive range out of bounds");
        if (G.substrate < 0 || G.substrate >= G.prim_count) return fail(SPUT_ERR_INVALID_SCENE, "substrate index outside the geometry");
        int k = d->prims[G.prim_begin + G.substrate].kind;
        if (k != SPUT_PRIM_RECT && k != SPUT_PRIM_DISC) return fail(SPUT_ERR_INVALID_SCENE, "substrate must be a RECT or DISC");
    }
    for (int c = 0; c < d->n_cathodes; ++c) {
        const sput_cathode& C = d->cathodes[c];
        if (C.Z < 1 || !(C.mass > 0.0) || !(C.U_s > 0.0)) return fail(SPUT_ERR_INVALID_SCENE, "cathode Z, mass, U_s must be positive");
        if (!finite3(C.center) || !unit3(C.normal) || !unit3(C.e1) || std::fabs(dot3(C.normal, C.e1)) > 1e-6)
            return fail(SPUT_ERR_INVALID_SCENE, "cathode pose: normal and e1 must be orthonormal");
        if (!(C.rt_sigma > 0.0) || !(C.rt_R > 0.0) || !(C.rt_r0 >= 0.0) || !std::isfinite(C.rt_r0))
            return fail(SPUT_ERR_INVALID_SCENE, "racetrack needs sigma > 0, R > 0, r0 >= 0");
        double sum = 0.0;
        for (int i = 0; i < 6; ++i) {
            if (!(C.cos_coef[i] >= 0.0) || !std::isfinite(C.cos_coef[i])) return fail(SPUT_ERR_INVALID_SCENE, "cosine coefficients must be >= 0");
            sum += C.cos_coef[i];
        }
        if (!(sum > 0.0)) return fail(SPUT_ERR_INVALID_SCENE, "cosine coefficients must not all be zero");
        if (C.launch_table) {
            if (C.n_mu < 1 || C.n_mu > 256 || C.n_E < 1 || C.n_E > 256)
                return fail(SPUT_ERR_INVALID_SCENE, "launch table needs 1 <= n_mu, n_E <= 256");
            if (!(C.E_hi > 0.0) || !std::isfinite(C.E_hi)) return fail(SPUT_ERR_INVALID_SCENE, "launch table needs E_hi > 0");
            double tot = 0.0;
            for (int i = 0; i < C.n_mu * C.n_E; ++i) {
                const double w = C.launch_table[i];
                if (!(w >= 0.0) || !std::isfinite(w)) return fail(SPUT_ERR_INVALID_SCENE, "launch table weights must be finite and >= 0");
                tot += w;
            }
            if (!(tot > 0.0) || !std::isfinite(tot)) return fail(SPUT_ERR_INVALID_SCENE, "launch table weights must not all be zero");
        }
    }
    const sput_grid& gr = d->grid;
    if (gr.nx < 1 || gr.ny < 1 || !(gr.half_u > 0.0) || !(gr.half_v > 0.0)) return fail(SPUT_ERR_INVALID_SCENE, "grid needs nx, ny >= 1 and positive extent");
    if ((long long)gr.nx * gr.ny > (1LL << 30)) return fail(SPUT_ERR_INVALID_SCENE, "grid too large");
    if (gr.count_type != SPUT_COUNT_INT32 && gr.count_type != SPUT_COUNT_INT64) return fail(SPUT_ERR_INVALID_SCENE, "bad count_type");
    if (gr.n_ebins < 0 || gr.n_abins < 0 || (gr.n_ebins > 0 && !(gr.e_hist_max > 0.0))) return fail(SPUT_ERR_INVALID_SCENE, "bad histogram settings");
    const sput_physics& ph = d->physics;
    if (!(ph.chi_min > 0.0 && ph.chi_min < kPi)) return fail(SPUT_ERR_INVALID_SCENE, "chi_min must lie in (0, pi)");
    if (ph.interaction != SPUT_INTERACTION_MOLIERE && ph.interaction != SPUT_INTERACTION_HARD_SPHERE) return fail(SPUT_ERR_INVALID_SCENE, "bad interaction");
    if (ph.interaction == SPUT_INTERACTION_HARD_SPHERE && !(ph.hs_diameter > 0.0)) return fail(SPUT_ERR_INVALID_SCENE, "hard-sphere diameter must be > 0");
    if (ph.gas_motion != SPUT_GAS_THERMAL && ph.gas_motion != SPUT_GAS_STATIONARY) return fail(SPUT_ERR_INVALID_SCENE, "bad gas_motion");
    if (ph.max_attempts < 1 || ph.max_attempts > 64) return fail(SPUT_ERR_INVALID_SCENE, "max_attempts must be 1..64");
    if (ph.max_collisions < 0 || ph.max_collisions > 0xFFFFFFF0LL) return fail(SPUT_ERR_INVALID_SCENE, "max_collisions out of range");
    if (!(ph.thermal_switch_eV >= 0.0) || !std::isfinite(ph.thermal_switch_eV))
        return fail(SPUT_ERR_INVALID_SCENE, "thermal_switch_eV must be >= 0");
    if (ph.thermal_switch_eV > 0.0 && ph.gas_motion != SPUT_GAS_THERMAL)
        return fail(SPUT_ERR_INVALID_SCENE, "the diffusion shortcut needs a thermal gas");
    return SPUT_OK;
}

sput_status validate_instances(const sput_scene* S, const sput_instance* inst, int n, const sput_cathode* cath,
                               int n_cath, const sput_geometry* geoms, int n_geoms, const sput_primitive* prims,
                               int count_type, double gas_mass)
{
    unsigned long long total = 0;
    for (int i = 0; i < n; ++i) {
        const sput_instance& I = inst[i];
        if (I.geometry < 0 || I.geometry >= n_geoms || I.cathode < 0 || I.cathode >= n_cath)
            return fail(SPUT_ERR_INVALID_SCENE, "instance geometry/cathode index out of range");
        const sput_cathode& C = cath[I.cathode];
        const sput_geometry& G = geoms[I.geometry];
        if (C.target < 0 || C.target >= G.prim_count || prims[G.prim_begin + C.target].kind != SPUT_PRIM_DISC)
            return fail(SPUT_ERR_INVALID_SCENE, "cathode target must be a DISC of the instance geometry");
        if (!(I.pressure >= 0.0) || !std::isfinite(I.pressure) || !(I.E_i > 0.0) || !(I.k > 0.0))
            return fail(SPUT_ERR_INVALID_SCENE, "instance needs pressure >= 0, E_i > 0, k > 0");
        // the Thompson distribution needs a positive cut-off (a launch table brings its own range)
        if (!C.launch_table && !(thompson_emax(I.k, gas_mass, C.mass, I.E_i, C.U_s) > 0.0))
            return fail(SPUT_ERR_INVALID_SCENE, "E_max = k Lambda E_i - U_s must be > 0");
        if (I.n_particles >= (1ull << 32)) return fail(SPUT_ERR_INVALID_SCENE, "more than 2^32-1 particles in one instance");
        total += I.n_particles;
    }
    if (count_type == SPUT_COUNT_INT32 && total > 0x7FFFFFFFull) return fail(SPUT_ERR_INVALID_SCENE, "int32 counts need fewer than 2^31 particles");
    (void)S;
    return SPUT_OK;
}

}  // namespace

extern "C" {

int sput_version(void) { return SPUT_ABI_VERSION; }

const char* sput_status_str(sput_status s)
{
    switch (s) {
    case SPUT_OK: return "ok";
    case SPUT_ERR_INVALID_ARG: return "invalid argument";
    case SPUT_ERR_INVALID_SCENE: return "invalid scene";
    case SPUT_ERR_CUDA: return "CUDA error";
    case SPUT_ERR_TIMEOUT: return "timeout";
    case SPUT_ERR_DEVICE_CHECK: return "device check failed";
    case SPUT_ERR_UNSUPPORTED: return "unsupported";
    case SPUT_ERR_NO_MEMORY: return "out of memory";
    }
    return "unknown status";
}

const char* sput_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

const sput::DevInstance* sput::scene_device_instances(const sput_scene* S) { return S ? S->base.inst : nullptr; }

extern "C" {

static sput_status pack_instances(sput_scene* S)
{
    const double kT = kBoltzmannJ * S->chamber.gas_T;
    S->dinst.assign(S->instances.size(), DevInstance{});
    S->prefix.assign(S->instances.size() + 1, 0ull);
    for (size_t i = 0; i < S->instances.size(); ++i) {
        const sput_instance& I = S->instances[i];
        const sput_cathode& C = S->cathodes[I.cathode];
        double Em = thompson_emax(I.k, S->chamber.gas_mass, C.mass, I.E_i, C.U_s);
        if (!(Em > 0.0)) return fail(SPUT_ERR_INVALID_SCENE, "E_max = k Lambda E_i - U_s must be > 0");
        int pair = S->dcath[I.cathode].pair;
        if (!C.launch_table && Em > S->pair_E_top[pair] * (1.0 + 1e-12))
            return fail(SPUT_ERR_INVALID_ARG, "E_max beyond the range of the scene's tables; recreate the scene");
        DevInstance& D = S->dinst[i];
        D.geometry = I.geometry;
        D.cathode = I.cathode;
        D.pair = pair;
        D.n = (uint32_t)I.n_particles;
        // n_g = p / (k_B T) in m^-3 -> mm^-3 (1e-9); sigma in A^2 -> mm^2 (1e-14)
        D.ng14 = (float)(I.pressure / kT * 1e-9 * 1e-14);
        D.thompson_q = (float)(Em / (Em + C.U_s));
        D.U_s = (float)C.U_s;
        D.kLambda = (float)(I.k * 4.0 * S->chamber.gas_mass * C.mass /
                            ((S->chamber.gas_mass + C.mass) * (S->chamber.gas_mass + C.mass)));
        D.ticket_begin = S->prefix[i];
        D.stream = I.rng_stream ? I.rng_stream - 1u : (uint32_t)i;
        S->prefix[i + 1] = S->prefix[i] + I.n_particles;
    }
    S->n_tickets = S->prefix.back();
    return SPUT_OK;
}

// Cell masks of the surface test.  A uniform grid of cubic cells (edge h, 32 along the
// chamber's longest side) covers the chamber box.  For every geometry, cell c and
// r = 1, 2, a 64-bit mask holds the local primitives that a flight of length at most
// r h starting in c can reach: those whose bounding sphere meets the block of cells
// within r of c (grown by a margin for FP32 rounding), and the chamber box when that
// block touches a wall.  A flight that long cannot leave the block, so testing the
// mask's primitives in ascending order finds the same nearest hit, with the same
// tie-breaking, as testing every primitive.  Geometries of more than 64 primitives
// leave the masks out (every flight tests every primitive).
static void build_cell_masks(sput_scene* S)
{
    S->cell_masks.clear();
    S->cell_h = 0.0;
    for (const sput_geometry& g : S->geoms)
        if (g.prim_count > 64) return;
    double ext[3], emax = 0.0;
    for (int a = 0; a < 3; ++a) {
        S->cell_lo[a] = S->chamber.box_lo[a];
        ext[a] = S->chamber.box_hi[a] - S->chamber.box_lo[a];
        emax = std::max(emax, ext[a]);
    }
    const double h = emax / 32.0;
    for (int a = 0; a < 3; ++a) S->cell_n[a] = std::max(1, std::min(32, (int)std::ceil(ext[a] / h - 1e-9)));
    S->cell_h = h;
    const int nx = S->cell_n[0], ny = S->cell_n[1], nz = S->cell_n[2];
    const size_t ncell = (size_t)nx * ny * nz;
    const double margin = 1e-3 * h + 1e-3;
    S->cell_masks.assign(S->geoms.size() * ncell * 2, 0ull);
    for (size_t g = 0; g < S->geoms.size(); ++g) {
        const sput_geometry& G = S->geoms[g];
        S->dgeoms[g].cell_base = (int)(g * ncell * 2);
        for (int iz = 0; iz < nz; ++iz)
            for (int iy = 0; iy < ny; ++iy)
                for (int ix = 0; ix < nx; ++ix) {
                    const int idx[3] = {ix, iy, iz};
                    for (int r = 1; r <= 2; ++r) {
                        double blo[3], bhi[3];
                        bool wall = false;
                        for (int a = 0; a < 3; ++a) {
                            blo[a] = S->cell_lo[a] + (idx[a] - r) * h - margin;
                            bhi[a] = S->cell_lo[a] + (idx[a] + 1 + r) * h + margin;
                            if (idx[a] - r <= 0 || idx[a] + r >= S->cell_n[a] - 1) wall = true;
                        }
                        unsigned long long m = 0ull;
                        for (int li = 0; li < G.prim_count; ++li) {
                            const DevPrim& Q = S->dprims[G.prim_begin + li];
                            bool in;
                            if (Q.kind == SPUT_PRIM_BOX) {
                                in = wall;
                            } else {
                                const double c[3] = {Q.bx, Q.by, Q.bz};
                                double d2 = 0.0;
                                for (int a = 0; a < 3; ++a) {
                                    const double d = std::max(0.0, std::max(blo[a] - c[a], c[a] - bhi[a]));
                                    d2 += d * d;
                                }
                                const double rr = (double)Q.br + margin;
                                in = d2 <= rr * rr;
                            }
                            if (in) m |= 1ull << li;
                        }
                        S->cell_masks[(size_t)S->dgeoms[g].cell_base + 2 * (((size_t)iz * ny + iy) * nx + ix) + (r - 1)] = m;
                    }
                }
    }
}

sput_status sput_scene_create(const sput_scene_desc* desc, int device, sput_scene** out)
{
    sput::NvtxRange nvtx("sput_scene_create");
    if (!out) return fail(SPUT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    sput_status st = validate(desc);
    if (st != SPUT_OK) return st;
    st = validate_instances(nullptr, desc->instances, desc->n_instances, desc->cathodes, desc->n_cathodes, desc->geoms,
                            desc->n_geoms, desc->prims, desc->grid.count_type, desc->chamber.gas_mass);
    if (st != SPUT_OK) return st;
    int ndev = 0;
    CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(SPUT_ERR_INVALID_ARG, "device index out of range");
    DeviceGuard guard(device);
    if (!guard.ok) return fail(SPUT_ERR_CUDA, "cudaSetDevice failed");

    int n_sm = 0, optin = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device));
    CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
    sput_scene* S = new sput_scene();
    S->device = device;
    S->n_sm = n_sm;
    S->smem_optin = (size_t)optin;
    S->chamber = desc->chamber;
    S->grid = desc->grid;
    S->physics = desc->physics;
    S->prims.assign(desc->prims, desc->prims + desc->n_prims);
    S->geoms.assign(desc->geoms, desc->geoms + desc->n_geoms);
    S->cathodes.assign(desc->cathodes, desc->cathodes + desc->n_cathodes);
    S->lt_weights.resize(S->cathodes.size());
    for (size_t c = 0; c < S->cathodes.size(); ++c) {
        sput_cathode& C = S->cathodes[c];
        if (C.launch_table) S->lt_weights[c].assign(C.launch_table, C.launch_table + (size_t)C.n_mu * C.n_E);
        C.launch_table = S->lt_weights[c].empty() ? nullptr : S->lt_weights[c].data();
    }
    S->instances.assign(desc->instances, desc->instances + desc->n_instances);

    const bool hard = S->physics.interaction == SPUT_INTERACTION_HARD_SPHERE;
    const int thermal = S->physics.gas_motion == SPUT_GAS_THERMAL;
    S->s_gas = std::sqrt(kBoltzmannEV * S->chamber.gas_T / (S->chamber.gas_mass * kEnergyUnit));
    S->bt = hard ? nullptr : &bmax_table(S->physics.chi_min);

    // primitives
    S->dprims.resize(S->prims.size());
    for (size_t i = 0; i < S->prims.size(); ++i) {
        const sput_primitive& P = S->prims[i];
        DevPrim& D = S->dprims[i];
        double n[3];
        cross3(P.u, P.v, n);
        D.cx = (float)P.center[0];
        D.cy = (float)P.center[1];
        D.cz = (float)P.center[2];
        D.kind = P.kind;
        D.ux = (float)P.u[0];
        D.uy = (float)P.u[1];
        D.uz = (float)P.u[2];
        D.p0 = (float)P.p0;
        D.vx = (float)P.v[0];
        D.vy = (float)P.v[1];
        D.vz = (float)P.v[2];
        D.p1 = (float)P.p1;
        D.nx = (float)n[0];
        D.ny = (float)n[1];
        D.nz = (float)n[2];
        D.p0sq = (float)(P.p0 * P.p0);
        // bounding sphere about the centre
        double br = 0.0;
        if (P.kind == SPUT_PRIM_RECT) br = std::sqrt(P.p0 * P.p0 + P.p1 * P.p1);
        else if (P.kind == SPUT_PRIM_DISC) br = P.p1;
        else if (P.kind == SPUT_PRIM_CYLINDER) br = std::sqrt(P.p0 * P.p0 + P.p1 * P.p1);
        D.bx = D.cx;
        D.by = D.cy;
        D.bz = D.cz;
        D.br = (float)(br * (1.0 + 1e-6));
    }
    S->dgeoms.resize(S->geoms.size());
    S->max_prims = 0;
    for (size_t g = 0; g < S->geoms.size(); ++g) {
        S->dgeoms[g] = DevGeom{S->geoms[g].prim_begin, S->geoms[g].prim_count, S->geoms[g].substrate, -1};
        S->max_prims = std::max(S->max_prims, S->geoms[g].prim_count);
    }
    build_cell_masks(S);

    // interaction pairs (one per distinct cathode element) and their E range
    std::map<std::pair<int, double>, int> pair_of;
    std::vector<int> cath_pair(S->cathodes.size());
    for (size_t c = 0; c < S->cathodes.size(); ++c) {
        auto key = std::make_pair(S->cathodes[c].Z, S->cathodes[c].mass);
        auto it = pair_of.find(key);
        if (it == pair_of.end()) {
            int id = (int)S->pair_phys.size();
            pair_of[key] = id;
            S->pair_phys.push_back(make_pair(S->cathodes[c].Z, S->cathodes[c].mass, S->chamber.gas_Z,
                                             S->chamber.gas_mass, hard ? 1 : 0, S->physics.hs_diameter,
                                             S->physics.chi_min));
            S->pair_E_top.push_back(0.0);
            cath_pair[c] = id;
        } else {
            cath_pair[c] = it->second;
        }
    }
    for (const sput_instance& I : S->instances) {
        const sput_cathode& C = S->cathodes[I.cathode];
        // highest launch energy: the Thompson cut-off, or the table's upper end
        double Em = C.launch_table ? C.E_hi : thompson_emax(I.k, S->chamber.gas_mass, C.mass, I.E_i, C.U_s);
        double& top = S->pair_E_top[cath_pair[I.cathode]];
        top = std::max(top, std::max(2.0 * Em, 200.0));
    }
    S->dpairs.resize(S->pair_phys.size());
    const double h_w = 0.02;
    std::vector<std::vector<float4>> g_tabs(S->pair_phys.size());
    for (size_t p = 0; p < S->pair_phys.size(); ++p) {
        const PairPhys& pp = S->pair_phys[p];
        double v_top = std::sqrt(2.0 * S->pair_E_top[p] / (pp.m1 * kEnergyUnit)) + 12.0 * S->s_gas;
        std::vector<float4> K, EA, EB, Gt;
        int n_w = 0;
        build_w_tables(pp, S->bt, S->s_gas, thermal, v_top, h_w, K, EA, EB, Gt, n_w);
        DevPair& D = S->dpairs[p];
        D.kappa = (float)pp.kappa;
        D.ln_kappa = (float)std::log(pp.kappa);
        D.sigma_scale = (float)(hard ? kPi * pp.hs_d * pp.hs_d : kPi * pp.a * pp.a);
        D.m1M = (float)(pp.m1 / (pp.m1 + pp.m2));
        D.m2M = (float)(pp.m2 / (pp.m1 + pp.m2));
        D.hard_sphere = hard ? 1 : 0;
        D.K_off = (int)S->wtab.size();
        S->wtab.insert(S->wtab.end(), K.begin(), K.end());
        D.A_off = (int)S->wtab.size();
        S->wtab.insert(S->wtab.end(), EA.begin(), EA.end());
        D.B_off = (int)S->wtab.size();
        S->wtab.insert(S->wtab.end(), EB.begin(), EB.end());
        g_tabs[p] = std::move(Gt);
        D.sigma_D = S->physics.thermal_switch_eV > 0.0 ? (float)sigma_D64(pp, S->bt, S->chamber.gas_T) : 0.0f;
        D.pad_d[0] = D.pad_d[1] = 0.0f;
        D.n_w = n_w;
        D.w_inv_h = (float)(1.0 / h_w);
        D.inv_s = (float)(1.0 / S->s_gas);
    }
    // the d ln K/d ln s tables follow every K, A and B table (read by the temperature-score
    // instance only); the kernel reads all of them through L1
    for (size_t p = 0; p < S->pair_phys.size(); ++p) {
        S->dpairs[p].G_off = (int)S->wtab.size();
        S->wtab.insert(S->wtab.end(), g_tabs[p].begin(), g_tabs[p].end());
    }

    // cathodes
    const int rt_n = 512;
    S->dcath.resize(S->cathodes.size());
    S->rt.clear();
    for (size_t c = 0; c < S->cathodes.size(); ++c) {
        const sput_cathode& C = S->cathodes[c];
        DevCathode& D = S->dcath[c];
        double e2[3];
        cross3(C.normal, C.e1, e2);
        for (int a = 0; a < 3; ++a) {
            D.c[a] = (float)C.center[a];
            D.n[a] = (float)C.normal[a];
            D.e1[a] = (float)C.e1[a];
            D.e2[a] = (float)e2[a];
        }
        D.rt_R = (float)C.rt_R;
        for (int q = 0; q < 7; ++q) D.rt_pad[q] = 0.0f;
        D.lt_off = -1;
        D.lt_nmu = D.lt_nE = 0;
        D.lt_dE = 0.0f;
        if (C.launch_table) {
            // marginal CDF over mu cells, then one conditional CDF over E per mu cell
            const int nm = C.n_mu, ne = C.n_E;
            D.lt_off = (int)S->lt.size();
            D.lt_nmu = nm;
            D.lt_nE = ne;
            D.lt_dE = (float)(C.E_hi / ne);
            std::vector<double> row(nm, 0.0);
            double tot = 0.0;
            for (int i = 0; i < nm; ++i) {
                for (int k = 0; k < ne; ++k) row[i] += C.launch_table[(size_t)i * ne + k];
                tot += row[i];
            }
            double acc = 0.0;
            S->lt.push_back(0.0f);
            for (int i = 0; i < nm; ++i) {
                acc += row[i];
                S->lt.push_back(i + 1 == nm ? 1.0f : (float)(acc / tot));
            }
            for (int i = 0; i < nm; ++i) {
                double a2 = 0.0;
                S->lt.push_back(0.0f);
                for (int k = 0; k < ne; ++k) {
                    a2 += C.launch_table[(size_t)i * ne + k];
                    // a row of zero weight is never drawn; give it a valid ramp
                    S->lt.push_back(k + 1 == ne ? 1.0f : (float)(row[i] > 0.0 ? a2 / row[i] : (k + 1.0) / ne));
                }
            }
        }
        double norm = 0.0;
        bool pure = true;
        for (int i = 0; i < 6; ++i) {
            D.coef[i] = (float)C.cos_coef[i];
            norm += C.cos_coef[i] / (i + 1);
            if (C.cos_coef[i] != (i == 1 ? 1.0 : 0.0)) pure = false;
        }
        D.coef_norm = (float)norm;
        D.cos_general = pure ? 0 : 1;
        D.target = C.target;
        D.pair = cath_pair[c];
        // cathodes with the same racetrack profile share one table
        int same = -1;
        for (size_t c2 = 0; c2 < c; ++c2)
            if (S->cathodes[c2].rt_r0 == C.rt_r0 && S->cathodes[c2].rt_sigma == C.rt_sigma &&
                S->cathodes[c2].rt_R == C.rt_R) {
                same = (int)c2;
                break;
            }
        if (same >= 0) {
            D.rt_tab = S->dcath[same].rt_tab;
        } else {
            D.rt_tab = (int)S->rt.size();
            S->rt.resize(S->rt.size() + 2 * rt_n);
            racetrack_table(C.rt_r0, C.rt_sigma, C.rt_R, rt_n, &S->rt[D.rt_tab]);
        }
        D.v_per_sqrtE = (float)std::sqrt(2.0 / (C.mass * kEnergyUnit));
        D.E_per_v2 = (float)(0.5 * C.mass * kEnergyUnit);
    }
    st = pack_instances(S);
    if (st != SPUT_OK) {
        delete S;
        return st;
    }

    // one device allocation for every table
    size_t o = 0;
    auto place = [&](size_t bytes) {
        size_t at = o;
        o = align_up(o + bytes, 256);
        return at;
    };
    S->off_prims = place(sizeof(DevPrim) * S->dprims.size());
    S->off_geoms = place(sizeof(DevGeom) * S->dgeoms.size());
    S->off_cath = place(sizeof(DevCathode) * S->dcath.size());
    S->off_pairs = place(sizeof(DevPair) * S->dpairs.size());
    S->off_inst = place(sizeof(DevInstance) * S->dinst.size());
    S->off_prefix = place(sizeof(unsigned long long) * S->prefix.size());
    const BmaxTable* bt = S->bt;
    std::vector<float4> bm_hs(1, make_float4(1.0f, 0.0f, 0.0f, 0.0f));
    std::vector<float> xh_hs(2, 0.0f);
    const std::vector<float4>& bm = bt ? bt->cubic : bm_hs;
    const std::vector<float>& xh = bt ? bt->xh : xh_hs;
    S->off_bm = place(sizeof(float4) * bm.size());
    S->off_xh = place(sizeof(float) * xh.size());
    S->off_w = place(sizeof(float4) * S->wtab.size());
    S->off_rt = place(sizeof(float4) * S->rt.size());
    S->off_lt = place(sizeof(float) * S->lt.size());
    const ChiTable* ct = hard ? nullptr : &chi_table(S->physics.chi_min);
    S->off_chi = place(ct ? sizeof(float4) * ct->cells.size() : 0);
    S->off_cell = place(sizeof(unsigned long long) * S->cell_masks.size());
    S->blob_bytes = o;
    cudaError_t e = cudaMalloc(&S->d_blob, S->blob_bytes);
    if (e != cudaSuccess) {
        delete S;
        return fail(SPUT_ERR_NO_MEMORY, std::string("cudaMalloc scene: ") + cudaGetErrorString(e));
    }
    std::vector<unsigned char> h(S->blob_bytes, 0);
    auto put = [&](size_t off, const void* src, size_t bytes) {
        if (bytes) std::memcpy(h.data() + off, src, bytes);
    };
    put(S->off_prims, S->dprims.data(), sizeof(DevPrim) * S->dprims.size());
    put(S->off_geoms, S->dgeoms.data(), sizeof(DevGeom) * S->dgeoms.size());
    put(S->off_cath, S->dcath.data(), sizeof(DevCathode) * S->dcath.size());
    put(S->off_pairs, S->dpairs.data(), sizeof(DevPair) * S->dpairs.size());
    put(S->off_inst, S->dinst.data(), sizeof(DevInstance) * S->dinst.size());
    put(S->off_prefix, S->prefix.data(), sizeof(unsigned long long) * S->prefix.size());
    put(S->off_bm, bm.data(), sizeof(float4) * bm.size());
    put(S->off_xh, xh.data(), sizeof(float) * xh.size());
    put(S->off_w, S->wtab.data(), sizeof(float4) * S->wtab.size());
    put(S->off_rt, S->rt.data(), sizeof(float4) * S->rt.size());
    put(S->off_lt, S->lt.data(), sizeof(float) * S->lt.size());
    if (ct) put(S->off_chi, ct->cells.data(), sizeof(float4) * ct->cells.size());
    put(S->off_cell, S->cell_masks.data(), sizeof(unsigned long long) * S->cell_masks.size());
    e = cudaMemcpy(S->d_blob, h.data(), S->blob_bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMallocHost(&S->h_scratch, 64);
    if (e == cudaSuccess) e = cudaEventCreate(&S->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&S->ev1);
    if (e != cudaSuccess) {
        sput_scene_destroy(S);
        return cuda_fail(e, "scene upload");
    }

    Params& p = S->base;
    std::memset(&p, 0, sizeof p);
    set_philox_keys(p, 0);  // the probe kernel's draws use key 0
    p.prims = reinterpret_cast<const DevPrim*>(S->d_blob + S->off_prims);
    p.geoms = reinterpret_cast<const DevGeom*>(S->d_blob + S->off_geoms);
    p.cath = reinterpret_cast<const DevCathode*>(S->d_blob + S->off_cath);
    p.pairs = reinterpret_cast<const DevPair*>(S->d_blob + S->off_pairs);
    p.inst = reinterpret_cast<const DevInstance*>(S->d_blob + S->off_inst);
    p.prefix = reinterpret_cast<const unsigned long long*>(S->d_blob + S->off_prefix);
    p.bm_tab = reinterpret_cast<const float4*>(S->d_blob + S->off_bm);
    p.xh_tab = reinterpret_cast<const float*>(S->d_blob + S->off_xh);
    p.w_tab = reinterpret_cast<const float4*>(S->d_blob + S->off_w);
    p.rt_tab = reinterpret_cast<const float4*>(S->d_blob + S->off_rt);
    p.lt_tab = reinterpret_cast<const float*>(S->d_blob + S->off_lt);
    p.chi_tab = ct ? reinterpret_cast<const float4*>(S->d_blob + S->off_chi) : nullptr;
    p.cell_mask = S->cell_masks.empty() ? nullptr
                                        : reinterpret_cast<const unsigned long long*>(S->d_blob + S->off_cell);
    for (int a = 0; a < 3; ++a) {
        p.cell_lo[a] = (float)S->cell_lo[a];
        p.cell_n[a] = S->cell_n[a];
    }
    p.cell_h = (float)S->cell_h;
    p.cell_inv_h = S->cell_h > 0.0 ? (float)(1.0 / S->cell_h) : 0.0f;
    p.n_prims = (int)S->dprims.size();
    p.n_geoms = (int)S->dgeoms.size();
    p.n_pairs = (int)S->dpairs.size();
    p.n_inst = (int)S->dinst.size();
    p.n_bm = (int)bm.size();
    p.n_w_all = (int)S->wtab.size();
    p.n_rt_all = (int)S->rt.size();
    p.n_lt_all = (int)S->lt.size();
    p.bm_lo = bt ? (float)bt->lo : 0.0f;
    p.bm_inv_h = bt ? (float)(1.0 / bt->h) : 1.0f;
    for (int a = 0; a < 3; ++a) {
        p.box_lo[a] = (float)S->chamber.box_lo[a];
        p.box_hi[a] = (float)S->chamber.box_hi[a];
    }
    p.s_gas = (float)S->s_gas;
    p.inv_T = (float)(1.0 / S->chamber.gas_T);
    p.E_switch = (float)S->physics.thermal_switch_eV;
    p.inv_s2 = (float)(1.0 / (S->s_gas * S->s_gas));
    p.gas_thermal = thermal;
    p.max_attempts = S->physics.max_attempts;
    p.max_prims = S->max_prims;
    p.max_collisions = S->physics.max_collisions;
    p.rt_n = rt_n;
    p.nx = S->grid.nx;
    p.ny = S->grid.ny;
    p.half_u = (float)S->grid.half_u;
    p.half_v = (float)S->grid.half_v;
    p.cells_per_mm_u = (float)(S->grid.nx / (2.0 * S->grid.half_u));
    p.cells_per_mm_v = (float)(S->grid.ny / (2.0 * S->grid.half_v));
    p.n_ebins = S->grid.n_ebins;
    p.n_abins = S->grid.n_abins;
    p.ebin_per_eV = S->grid.n_ebins > 0 ? (float)(S->grid.n_ebins / S->grid.e_hist_max) : 0.0f;
    // Gauss-Mehler constants: theta_j = (2j-1) pi / (2N), j = 1..N/2
    auto gm_node = [](int j, int N) {
        double th = (2.0 * (j + 1) - 1.0) * kPi / (2.0 * N);
        double c = std::cos(th), s = std::sin(th);
        return make_float4((float)c, (float)(1.0 / (1.0 + c)), (float)(c / (s * s)),
                           (float)(2.0 * std::sin(0.5 * th) * std::sin(0.5 * th) / c));
    };
    for (int j = 0; j < kGMHalf; ++j) p.gm[j] = gm_node(j, kGMNodes);
    for (int j = 0; j < kGMHalfLo; ++j) p.gm_lo[j] = gm_node(j, kGMNodesLo);
    if (transport_configure((int)S->smem_optin) != 0) {
        sput_scene_destroy(S);
        return fail(SPUT_ERR_CUDA, "cudaFuncSetAttribute on the transport kernel failed");
    }
    // privatise per-primitive counters in shared memory while they fit
    p.smem_counters = (size_t)p.n_inst * (p.max_prims + 1) <= 12288 ? 1 : 0;
    if (transport_smem_bytes(p) > S->smem_optin) {
        p.smem_counters = 0;
        if (transport_smem_bytes(p) > S->smem_optin) {
            sput_scene_destroy(S);
            return fail(SPUT_ERR_UNSUPPORTED, "scene tables exceed the shared memory of one block");
        }
    }
    S->smem_counters_fit = p.smem_counters;
    *out = S;
    return SPUT_OK;
}

sput_status sput_instances_set(sput_scene* S, const sput_instance* instances, int n)
{
    sput::NvtxRange nvtx("sput_instances_set");
    if (!S || !instances) return fail(SPUT_ERR_INVALID_ARG, "NULL argument");
    if (n != (int)S->instances.size()) return fail(SPUT_ERR_INVALID_ARG, "number of instances must not change");
    for (int i = 0; i < n; ++i)
        if (instances[i].geometry != S->instances[i].geometry || instances[i].cathode != S->instances[i].cathode)
            return fail(SPUT_ERR_INVALID_ARG, "instance geometry and cathode must not change");
    sput_status st = validate_instances(S, instances, n, S->cathodes.data(), (int)S->cathodes.size(), S->geoms.data(),
                                        (int)S->geoms.size(), S->prims.data(), S->grid.count_type,
                                        S->chamber.gas_mass);
    if (st != SPUT_OK) return st;
    std::vector<sput_instance> old = S->instances;
    S->instances.assign(instances, instances + n);
    st = pack_instances(S);
    if (st != SPUT_OK) {
        S->instances = old;
        pack_instances(S);
        return st;
    }
    DeviceGuard guard(S->device);
    CUDA_TRY(cudaMemcpy(S->d_blob + S->off_inst, S->dinst.data(), sizeof(DevInstance) * S->dinst.size(),
                        cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(S->d_blob + S->off_prefix, S->prefix.data(), sizeof(unsigned long long) * S->prefix.size(),
                        cudaMemcpyHostToDevice));
    return SPUT_OK;
}

sput_status sput_tally_layout_get(const sput_scene* S, sput_tally_layout* out)
{
    if (!S || !out) return fail(SPUT_ERR_INVALID_ARG, "NULL argument");
    out->n_instances = (int)S->instances.size();
    out->nx = S->grid.nx;
    out->ny = S->grid.ny;
    out->max_prims = S->max_prims;
    out->n_ebins = S->grid.n_ebins;
    out->n_abins = S->grid.n_abins;
    out->count_type = S->grid.count_type;
    out->reserved = 0;
    out->n_tickets = S->n_tickets;
    return SPUT_OK;
}

}  // extern "C"

namespace {

struct TallySizes {
    size_t counts, energy, score, prim_counts, timed_out, hist_E, hist_A, score_T;
};

TallySizes tally_sizes(const sput_scene* S)
{
    const size_t ni = S->instances.size(), nc = (size_t)S->grid.nx * S->grid.ny;
    TallySizes t;
    t.counts = ni * nc * (S->grid.count_type == SPUT_COUNT_INT64 ? 8 : 4);
    t.energy = ni * nc * 8;
    t.score = ni * nc * 8;
    t.prim_counts = ni * S->max_prims * 8;
    t.timed_out = ni * 8;
    t.hist_E = ni * S->grid.n_ebins * 8;
    t.hist_A = ni * S->grid.n_abins * 8;
    t.score_T = ni * nc * 8;
    return t;
}

sput_status ensure_scratch(sput_scene* S)
{
    if (S->d_scratch) return SPUT_OK;
    cudaError_t e = cudaMalloc(&S->d_scratch, 64);
    if (e != cudaSuccess) return fail(SPUT_ERR_NO_MEMORY, std::string("cudaMalloc scratch: ") + cudaGetErrorString(e));
    return SPUT_OK;
}

sput_status run_impl(sput_scene* S, const sput_run_opts* opts, cudaStream_t stream, const sput_tallies* T,
                     sput_run_stats* stats, unsigned long long* scratch, int* blocks_out = nullptr,
                     int* threads_out = nullptr)
{
    if (!opts || !T) return fail(SPUT_ERR_INVALID_ARG, "NULL argument");
    if (T->hist_E && S->grid.n_ebins == 0) return fail(SPUT_ERR_INVALID_ARG, "hist_E requested but n_ebins = 0");
    if (T->hist_A && S->grid.n_abins == 0) return fail(SPUT_ERR_INVALID_ARG, "hist_A requested but n_abins = 0");
    unsigned long long tb = opts->ticket_begin, te = opts->ticket_end ? opts->ticket_end : S->n_tickets;
    if (tb > te || te > S->n_tickets) return fail(SPUT_ERR_INVALID_ARG, "ticket range outside [0, n_tickets]");
    int threads = opts->block_threads ? opts->block_threads : S->def_threads;
    if (threads < 32 || threads > 256 || threads % 32) return fail(SPUT_ERR_INVALID_ARG, "block_threads must be a multiple of 32 in [32, 256]");
    int chunk = opts->ticket_chunk ? opts->ticket_chunk : S->def_chunk;
    if (chunk < 1 || chunk > (1 << 20)) return fail(SPUT_ERR_INVALID_ARG, "ticket_chunk out of range");
    if (opts->flags &
        ~(SPUT_RUN_NO_SMEM_COUNTERS | SPUT_RUN_SMEM_COUNTERS | SPUT_RUN_LAUNCH_AT_CUTOFF | SPUT_RUN_INJECT_NONFINITE |
          SPUT_RUN_NO_CELL_MASKS | SPUT_RUN_CELL_MASKS))
        return fail(SPUT_ERR_INVALID_ARG, "unknown flags");
    const int cutoff = opts->flags & SPUT_RUN_LAUNCH_AT_CUTOFF;
    const int fsm = opts->flags & (SPUT_RUN_NO_SMEM_COUNTERS | SPUT_RUN_SMEM_COUNTERS);
    const int flags = (fsm ? fsm : S->def_flags) | cutoff;
    if (T->score_T && S->physics.thermal_switch_eV > 0.0)
        return fail(SPUT_ERR_UNSUPPORTED, "the temperature score is not defined with the diffusion shortcut");
    if (cutoff)
        for (const sput_cathode& C : S->cathodes)
            if (C.launch_table) return fail(SPUT_ERR_UNSUPPORTED, "launch at the cut-off needs Thompson cathodes only");
    const int bps_req = opts->blocks_per_sm ? opts->blocks_per_sm : S->def_bps;

    Params p = S->base;
    p.counts = T->counts;
    p.energy = T->energy;
    p.score = T->score;
    p.score_T = T->score_T;
    p.prim_counts = reinterpret_cast<long long*>(T->prim_counts);
    p.timed_out = reinterpret_cast<long long*>(T->timed_out);
    p.hist_E = reinterpret_cast<long long*>(T->hist_E);
    p.hist_A = reinterpret_cast<long long*>(T->hist_A);
    p.records = T->records;
    set_philox_keys(p, opts->seed);
    p.ticket_begin = tb;
    p.ticket_end = te;
    p.chunk = chunk;
    p.ticket_counter = scratch;
    p.stats = scratch + 1;
    p.status = reinterpret_cast<unsigned int*>(scratch + 1 + kNumStats);
    p.smem_counters = (flags & SPUT_RUN_NO_SMEM_COUNTERS) ? 0 : S->smem_counters_fit;
    p.launch_at_cutoff = cutoff ? 1 : 0;
    p.inject_nonfinite = (opts->flags & SPUT_RUN_INJECT_NONFINITE) ? 1 : 0;
    // the masked surface test pays where geometries have many primitives (see SPUT_RUN_CELL_MASKS)
    const bool masks = (opts->flags & SPUT_RUN_CELL_MASKS) ||
                       (!(opts->flags & SPUT_RUN_NO_CELL_MASKS) && S->max_prims > 32);
    if (!masks) p.cell_mask = nullptr;

    const TallySizes sz = tally_sizes(S);
    if (!opts->accumulate) {
        if (T->counts) CUDA_TRY(cudaMemsetAsync(T->counts, 0, sz.counts, stream));
        if (T->energy) CUDA_TRY(cudaMemsetAsync(T->energy, 0, sz.energy, stream));
        if (T->score) CUDA_TRY(cudaMemsetAsync(T->score, 0, sz.score, stream));
        if (T->prim_counts) CUDA_TRY(cudaMemsetAsync(T->prim_counts, 0, sz.prim_counts, stream));
        if (T->timed_out) CUDA_TRY(cudaMemsetAsync(T->timed_out, 0, sz.timed_out, stream));
        if (T->hist_E) CUDA_TRY(cudaMemsetAsync(T->hist_E, 0, sz.hist_E, stream));
        if (T->hist_A) CUDA_TRY(cudaMemsetAsync(T->hist_A, 0, sz.hist_A, stream));
        if (T->score_T) CUDA_TRY(cudaMemsetAsync(T->score_T, 0, sz.score_T, stream));
    }
    CUDA_TRY(cudaMemsetAsync(scratch, 0, 64, stream));

    const int c64 = S->grid.count_type == SPUT_COUNT_INT64;
    const size_t smem = transport_smem_bytes(p);
    int bps = transport_max_blocks_per_sm(c64, threads, smem);
    if (bps < 1) return fail(SPUT_ERR_UNSUPPORTED, "launch shape does not fit on an SM");
    if (bps_req > 0) bps = std::min(bps, bps_req);
    unsigned long long need = (te - tb + threads - 1) / threads;
    int blocks = (int)std::max<unsigned long long>(1ull, std::min<unsigned long long>((unsigned long long)S->n_sm * bps, need));
    if (te == tb) blocks = 1;
    if (blocks_out) *blocks_out = blocks;
    if (threads_out) *threads_out = threads;
    CUDA_TRY(cudaEventRecord(S->ev0, stream));
    int le = transport_launch(p, c64, blocks, threads, smem, stream);
    if (le != 0) return cuda_fail((cudaError_t)le, "transport kernel launch");
    CUDA_TRY(cudaEventRecord(S->ev1, stream));
    if (!stats) return SPUT_OK;

    CUDA_TRY(cudaMemcpyAsync(S->h_scratch, scratch, 64, cudaMemcpyDeviceToHost, stream));
    cudaEvent_t done;
    CUDA_TRY(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
    cudaError_t e = cudaEventRecord(done, stream);
    if (e != cudaSuccess) {
        cudaEventDestroy(done);
        return cuda_fail(e, "cudaEventRecord");
    }
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        e = cudaEventQuery(done);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) {
            cudaEventDestroy(done);
            return cuda_fail(e, "transport kernel");
        }
        if (opts->timeout_ms > 0 &&
            std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count() >
                opts->timeout_ms) {
            cudaEventDestroy(done);
            return fail(SPUT_ERR_TIMEOUT, "transport did not finish within timeout_ms (device left running)");
        }
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    cudaEventDestroy(done);
    const unsigned long long* h = S->h_scratch;
    stats->particles = h[1];
    stats->landed = h[2];
    stats->timed_out = h[3];
    stats->flights = h[4];
    stats->collisions = h[5];
    stats->attempts = h[6];
    stats->device_status = (uint32_t)(h[1 + kNumStats] & 0xffffffffu);
    stats->grid_blocks = (uint32_t)blocks;
    stats->block_threads = (uint32_t)threads;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, S->ev0, S->ev1);
    stats->kernel_ms = ms;
    if (stats->device_status) return fail(SPUT_ERR_DEVICE_CHECK, "device status bits set");
    return SPUT_OK;
}

}  // namespace

extern "C" {

sput_status sput_run(sput_scene* S, const sput_run_opts* opts, void* stream, const sput_tallies* T,
                     sput_run_stats* stats)
{
    sput::NvtxRange nvtx("sput_run");
    if (!S) return fail(SPUT_ERR_INVALID_ARG, "scene is NULL");
    DeviceGuard guard(S->device);
    sput_status st = ensure_scratch(S);
    if (st != SPUT_OK) return st;
    return run_impl(S, opts, reinterpret_cast<cudaStream_t>(stream), T, stats, S->d_scratch);
}

sput_status sput_run_host(sput_scene* S, const sput_run_opts* opts, const sput_tallies* H, sput_run_stats* stats)
{
    sput::NvtxRange nvtx("sput_run_host");
    if (!S || !opts || !H) return fail(SPUT_ERR_INVALID_ARG, "NULL argument");
    if (H->records) return fail(SPUT_ERR_UNSUPPORTED, "records are device-only; use sput_run");
    DeviceGuard guard(S->device);
    sput_status st = ensure_scratch(S);
    if (st != SPUT_OK) return st;
    const TallySizes sz = tally_sizes(S);
    size_t off[8], o = 0;
    const size_t bytes[8] = {sz.counts, sz.energy, sz.score, sz.prim_counts, sz.timed_out, sz.hist_E, sz.hist_A,
                             sz.score_T};
    for (int i = 0; i < 8; ++i) {
        off[i] = o;
        o = align_up(o + bytes[i], 256);
    }
    if (S->stage_bytes < o) {
        if (S->d_stage) cudaFree(S->d_stage);
        S->d_stage = nullptr;
        S->stage_bytes = 0;
        cudaError_t e = cudaMalloc(&S->d_stage, o);
        if (e != cudaSuccess) return fail(SPUT_ERR_NO_MEMORY, "cudaMalloc staging tallies");
        S->stage_bytes = o;
    }
    if (!S->own_stream) CUDA_TRY(cudaStreamCreateWithFlags(&S->own_stream, cudaStreamNonBlocking));
    unsigned char* base = reinterpret_cast<unsigned char*>(S->d_stage);
    void* hp[8] = {H->counts, H->energy, H->score, H->prim_counts, H->timed_out, H->hist_E, H->hist_A, H->score_T};
    sput_tallies D{};
    void** dp[8] = {&D.counts, reinterpret_cast<void**>(&D.energy), reinterpret_cast<void**>(&D.score),
                    reinterpret_cast<void**>(&D.prim_counts), reinterpret_cast<void**>(&D.timed_out),
                    reinterpret_cast<void**>(&D.hist_E), reinterpret_cast<void**>(&D.hist_A),
                    reinterpret_cast<void**>(&D.score_T)};
    for (int i = 0; i < 8; ++i) *dp[i] = hp[i] ? base + off[i] : nullptr;
    sput_run_opts o2 = *opts;
    if (o2.accumulate) {
        // accumulate into the caller's host values: upload them first
        for (int i = 0; i < 8; ++i)
            if (hp[i]) CUDA_TRY(cudaMemcpyAsync(base + off[i], hp[i], bytes[i], cudaMemcpyHostToDevice, S->own_stream));
    }
    sput_run_stats local{};
    st = run_impl(S, &o2, S->own_stream, &D, stats ? stats : &local, S->d_scratch);
    if (st != SPUT_OK) return st;
    for (int i = 0; i < 8; ++i)
        if (hp[i]) CUDA_TRY(cudaMemcpyAsync(hp[i], base + off[i], bytes[i], cudaMemcpyDeviceToHost, S->own_stream));
    CUDA_TRY(cudaStreamSynchronize(S->own_stream));
    return SPUT_OK;
}

sput_status sput_run_noalloc(sput_scene* S, const sput_run_opts* opts, void* stream, const sput_tallies* T,
                             sput_run_stats* stats)
{
    sput::NvtxRange nvtx("sput_run_noalloc");
    // Same transport as sput_run, but the run scratch (ticket counter, statistics,
    // status word) is the library's static device array instead of a per-scene
    // cudaMalloc, and the statistics wait polls the stream instead of creating
    // an event: nothing here allocates.
    if (!S) return fail(SPUT_ERR_INVALID_ARG, "scene is NULL");
    if (kRunScratchBytes > kStaticScratchBytes)
        return fail(SPUT_ERR_UNSUPPORTED, "run scratch of " + std::to_string(kRunScratchBytes) +
                                              " bytes exceeds the static scratch of " +
                                              std::to_string(kStaticScratchBytes) + " bytes");
    DeviceGuard guard(S->device);
    if (!guard.ok) return fail(SPUT_ERR_CUDA, "cudaSetDevice failed");
    unsigned long long* scratch = nullptr;
    int e0 = static_scratch_address(S->device, &scratch);
    if (e0 != 0) return cuda_fail((cudaError_t)e0, "cudaGetSymbolAddress(static run scratch)");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int blocks = 0, threads = 0;
    sput_status rs = run_impl(S, opts, st, T, nullptr, scratch, &blocks, &threads);
    if (rs != SPUT_OK || !stats) return rs;
    CUDA_TRY(cudaMemcpyAsync(S->h_scratch, scratch, kRunScratchBytes, cudaMemcpyDeviceToHost, st));
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t q = cudaStreamQuery(st);
        if (q == cudaSuccess) break;
        if (q != cudaErrorNotReady) return cuda_fail(q, "transport kernel");
        if (opts->timeout_ms > 0 &&
            std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count() >
                opts->timeout_ms)
            return fail(SPUT_ERR_TIMEOUT, "transport did not finish within timeout_ms (device left running)");
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    const unsigned long long* h = S->h_scratch;
    stats->particles = h[1];
    stats->landed = h[2];
    stats->timed_out = h[3];
    stats->flights = h[4];
    stats->collisions = h[5];
    stats->attempts = h[6];
    stats->device_status = (uint32_t)(h[1 + kNumStats] & 0xffffffffu);
    stats->grid_blocks = (uint32_t)blocks;
    stats->block_threads = (uint32_t)threads;
    // the kernel time comes from the scene's two timing events, which every run of
    // the scene records: a run of the same scene that overlaps this one overwrites
    // them (the same race as on the scratch array)
    float ms = 0.0f;
    CUDA_TRY(cudaEventElapsedTime(&ms, S->ev0, S->ev1));
    stats->kernel_ms = ms;
    if (stats->device_status) return fail(SPUT_ERR_DEVICE_CHECK, "device status bits set");
    return SPUT_OK;
}

sput_status sput_autotune(sput_scene* S, const sput_run_opts* base, void* stream, const sput_tallies* T,
                          uint64_t sample_tickets, sput_tune_result* out)
{
    if (!S || !base || !T || !out) return fail(SPUT_ERR_INVALID_ARG, "NULL argument");
    DeviceGuard guard(S->device);
    sput_status st = ensure_scratch(S);
    if (st != SPUT_OK) return st;
    std::memset(out, 0, sizeof *out);
    const unsigned long long n = S->n_tickets;
    if (n == 0) return fail(SPUT_ERR_INVALID_ARG, "scene has no particles");
    // four equal ticket ranges spread over the ticket space
    const unsigned long long per = std::max<unsigned long long>(1ull, std::min<unsigned long long>(sample_tickets / 4, n / 4 ? n / 4 : n));
    unsigned long long rb[4], re[4];
    int nr = 0;
    for (int i = 0; i < 4; ++i) {
        unsigned long long b = (n / 4) * i;
        if (b >= n) break;
        rb[nr] = b;
        re[nr] = std::min(n, b + per);
        ++nr;
    }
    struct Cand { int threads, bps, chunk, flags; };
    std::vector<Cand> cands;
    const int c64 = S->grid.count_type == SPUT_COUNT_INT64;
    for (int threads : {128, 192, 256}) {
        Params probe = S->base;
        probe.smem_counters = S->smem_counters_fit;
        const int occ = transport_max_blocks_per_sm(c64, threads, transport_smem_bytes(probe));
        for (int fl : {SPUT_RUN_SMEM_COUNTERS, SPUT_RUN_NO_SMEM_COUNTERS}) {
            if (fl == SPUT_RUN_SMEM_COUNTERS && !S->smem_counters_fit) continue;
            Params pr = S->base;
            pr.smem_counters = fl == SPUT_RUN_SMEM_COUNTERS ? 1 : 0;
            const int maxb = transport_max_blocks_per_sm(c64, threads, transport_smem_bytes(pr));
            if (maxb < 1) continue;
            for (int bps : {maxb, maxb - 1})
                if (bps >= 1 && (bps == maxb || bps >= occ - 1))
                    for (int chunk : {32, 128}) cands.push_back(Cand{threads, bps, chunk, fl});
        }
    }
    if (cands.size() > 32) cands.resize(32);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    double best = -1.0;
    Cand bestc = cands.empty() ? Cand{256, 0, 32, 0} : cands[0];
    for (size_t ci = 0; ci <= cands.size(); ++ci) {
        // candidate 0 is timed twice: the first pass warms up
        const Cand c = cands[ci == 0 ? 0 : ci - 1];
        double coll = 0.0, ms = 0.0;
        for (int r = 0; r < nr; ++r) {
            sput_run_opts o = *base;
            o.ticket_begin = rb[r];
            o.ticket_end = re[r];
            o.block_threads = c.threads;
            o.blocks_per_sm = c.bps;
            o.ticket_chunk = c.chunk;
            o.flags = c.flags;
            o.accumulate = 0;
            sput_run_stats rs{};
            st = run_impl(S, &o, s, T, &rs, S->d_scratch);
            if (st != SPUT_OK) return st;
            coll += (double)rs.collisions;
            ms += rs.kernel_ms;
        }
        if (ci == 0) continue;
        const double rate = ms > 0.0 ? coll / (ms * 1e-3) : 0.0;
        const int k = out->n_candidates++;
        out->cand_threads[k] = c.threads;
        out->cand_bps[k] = c.bps;
        out->cand_chunk[k] = c.chunk;
        out->cand_flags[k] = c.flags;
        out->cand_rate[k] = (float)rate;
        if (rate > best) {
            best = rate;
            bestc = c;
        }
    }
    S->def_threads = bestc.threads;
    S->def_bps = bestc.bps;
    S->def_chunk = bestc.chunk;
    S->def_flags = bestc.flags;
    out->block_threads = bestc.threads;
    out->blocks_per_sm = bestc.bps;
    out->ticket_chunk = bestc.chunk;
    out->flags = bestc.flags;
    out->best_rate = (float)best;
    return SPUT_OK;
}

}  // extern "C"

struct sput_graph {
    sput_scene* S = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t knode = nullptr;
    cudaKernelNodeParams kp{};
    Params params{};
    void* args[1] = {nullptr};
    cudaStream_t cs = nullptr;
};

extern "C" {

sput_status sput_graph_create(sput_scene* S, const sput_run_opts* opts, void* stream, const sput_tallies* T,
                              sput_graph** out)
{
    if (!S || !opts || !T || !out) return fail(SPUT_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    DeviceGuard guard(S->device);
    sput_status st = ensure_scratch(S);
    if (st != SPUT_OK) return st;
    sput_graph* G = new sput_graph();
    G->S = S;
    (void)stream;
    cudaError_t e = cudaStreamCreateWithFlags(&G->cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(G->cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        sput_graph_destroy(G);
        return cuda_fail(e, "graph capture begin");
    }
    st = run_impl(S, opts, G->cs, T, nullptr, S->d_scratch);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(G->cs, &g);
    G->graph = g;
    if (st != SPUT_OK) {
        sput_graph_destroy(G);
        return st;
    }
    if (e != cudaSuccess) {
        sput_graph_destroy(G);
        return cuda_fail(e, "graph capture end");
    }
    size_t nn = 0;
    e = cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (e == cudaSuccess && nn) e = cudaGraphGetNodes(g, nodes.data(), &nn);
    for (size_t i = 0; e == cudaSuccess && i < nn; ++i) {
        cudaGraphNodeType ty;
        e = cudaGraphNodeGetType(nodes[i], &ty);
        if (e == cudaSuccess && ty == cudaGraphNodeTypeKernel) G->knode = nodes[i];
    }
    if (e == cudaSuccess && G->knode) e = cudaGraphKernelNodeGetParams(G->knode, &G->kp);
    if (e != cudaSuccess || !G->knode) {
        sput_graph_destroy(G);
        return e != cudaSuccess ? cuda_fail(e, "graph inspection") : fail(SPUT_ERR_CUDA, "no kernel node in the captured graph");
    }
    std::memcpy(&G->params, G->kp.kernelParams[0], sizeof(Params));
    e = cudaGraphInstantiate(&G->exec, g, 0);
    if (e != cudaSuccess) {
        sput_graph_destroy(G);
        return cuda_fail(e, "cudaGraphInstantiate");
    }
    *out = G;
    return SPUT_OK;
}

sput_status sput_graph_launch(sput_graph* G, uint64_t seed, void* stream)
{
    if (!G) return fail(SPUT_ERR_INVALID_ARG, "graph is NULL");
    DeviceGuard guard(G->S->device);
    set_philox_keys(G->params, seed);
    G->args[0] = &G->params;
    cudaKernelNodeParams kp = G->kp;
    kp.kernelParams = G->args;
    kp.extra = nullptr;
    CUDA_TRY(cudaGraphExecKernelNodeSetParams(G->exec, G->knode, &kp));
    CUDA_TRY(cudaGraphLaunch(G->exec, reinterpret_cast<cudaStream_t>(stream)));
    return SPUT_OK;
}

void sput_graph_destroy(sput_graph* G)
{
    if (!G) return;
    {
        DeviceGuard guard(G->S ? G->S->device : 0);
        if (G->exec) cudaGraphExecDestroy(G->exec);
        if (G->graph) cudaGraphDestroy(G->graph);
        if (G->cs) cudaStreamDestroy(G->cs);
    }
    delete G;
}

void sput_scene_destroy(sput_scene* S)
{
    if (!S) return;
    {
        DeviceGuard guard(S->device);
        if (S->d_blob) cudaFree(S->d_blob);
        if (S->d_scratch) cudaFree(S->d_scratch);
        if (S->d_stage) cudaFree(S->d_stage);
        if (S->h_scratch) cudaFreeHost(S->h_scratch);
        if (S->ev0) cudaEventDestroy(S->ev0);
        if (S->ev1) cudaEventDestroy(S->ev1);
        if (S->own_stream) cudaStreamDestroy(S->own_stream);
    }
    delete S;
}

sput_status sput_deflection_table_eval(double chi_min, int n, const double* eps, const double* u, double* chi)
{
    if (!eps || !u || !chi || n < 0) return fail(SPUT_ERR_INVALID_ARG, "NULL argument or negative n");
    if (!(chi_min > 0.0 && chi_min < 0.5 * kPi)) return fail(SPUT_ERR_INVALID_ARG, "chi_min must be in (0, pi/2)");
    const ChiTable& ct = chi_table(chi_min);
    const BmaxTable& bt = bmax_table(chi_min);
    for (int i = 0; i < n; ++i) {
        if (!(eps[i] > 0.0) || !(u[i] > 0.0 && u[i] <= 1.0)) return fail(SPUT_ERR_INVALID_ARG, "need eps > 0, 0 < u <= 1");
        double q;
        if (ct.eval(std::log(eps[i]), 0.5 * std::log(u[i]), q)) {
            chi[i] = 2.0 * std::atan(std::exp(q));
        } else {
            // outside the table the device integrates; here the FP64 deflection
            chi[i] = chi_moliere64(eps[i], bt.eval(std::log(eps[i])) * std::sqrt(u[i]));
        }
    }
    return SPUT_OK;
}

sput_status sput_probe(sput_scene* S, int what, int idx, int n, const double* x, double* y)
{
    if (!S || !x || !y || n < 0) return fail(SPUT_ERR_INVALID_ARG, "NULL argument or negative n");
    if (what < SPUT_PROBE_CHI || what > SPUT_PROBE_CHI_U) return fail(SPUT_ERR_INVALID_ARG, "unknown probe");
    if ((what == SPUT_PROBE_K || what == SPUT_PROBE_M) && (idx < 0 || idx >= (int)S->dpairs.size()))
        return fail(SPUT_ERR_INVALID_ARG, "pair index out of range");
    if ((what == SPUT_PROBE_LAUNCH || what == SPUT_PROBE_TRACE) && (idx < 0 || idx >= (int)S->dinst.size()))
        return fail(SPUT_ERR_INVALID_ARG, "instance index out of range");
    if ((what == SPUT_PROBE_CHI || what == SPUT_PROBE_BMAX || what == SPUT_PROBE_CHI_U) && !S->bt)
        return fail(SPUT_ERR_UNSUPPORTED, "no Moliere tables in a hard-sphere scene");
    if (n == 0) return SPUT_OK;
    DeviceGuard guard(S->device);
    const size_t nx = (size_t)n * (what == SPUT_PROBE_CHI || what == SPUT_PROBE_CHI_U ? 2 : 1);
    const size_t ny = (size_t)n * (what == SPUT_PROBE_LAUNCH   ? 7
                                   : what == SPUT_PROBE_TRACE  ? kTraceRows * 10
                                   : what == SPUT_PROBE_M      ? 2
                                                               : 1);
    double *dx = nullptr, *dy = nullptr;
    CUDA_TRY(cudaMalloc(&dx, nx * sizeof(double)));
    cudaError_t e = cudaMalloc(&dy, ny * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(dx, x, nx * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = (cudaError_t)probe_launch(S->base, what, idx, n, dx, dy, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(y, dy, ny * sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(dx);
    if (dy) cudaFree(dy);
    if (e != cudaSuccess) return cuda_fail(e, "probe");
    return SPUT_OK;
}

}  // extern "C"
