/*
 * sput.h -- C ABI of the GB300 sputtered-atom transport library (libsput.so).
 *
 * The library runs the per-particle Monte Carlo transport of sputtered atoms
 * through the process gas described in Sec. "The SIMTRA model" of
 * arXiv 2411.14413 (Thelen et al., pySIMTRA):
 *   - launch point sampled from the racetrack profile (racetrack pdf),
 *   - launch energy from the Thompson distribution with cut-off
 *     E_max = k * Lambda * E_i - U_s, Lambda = 4 M_i M_t / (M_i + M_t)^2
 *     (Eq. for phi(E)),
 *   - launch direction from the six-term cosine sum
 *     d2Y/dOmega = sum_{i=0..5} c_i cos^i(theta) (Eq. for d2Y/dOmega),
 *   - free flights lambda = -lambda_m ln RN_1, RN_1 in ]0,1] (Eq. for lambda),
 *     with lambda_m depending on the atom and gas velocities,
 *   - after each flight a test whether the path reaches a surface ("dummy"
 *     objects, the chamber and the cathodes), which deposits the atom,
 *   - otherwise an elastic binary collision with a thermal gas atom under a
 *     screened-Coulomb potential with Moliere screening,
 * repeated until the atom lands; landings are tallied on a substrate grid
 * together with arrival energy and angle.
 *
 * Readings where the paper gives no formula (all fixed here, see each field):
 *   lambda_m(v) = v / (n_g <sigma(g) g>) averaged over a Maxwellian gas at T,
 *   n_g = p / (k_B T); sigma = pi b_max^2 with the CM deflection at b_max equal
 *   to chi_min; the gas partner is drawn from the Maxwellian weighted by
 *   sigma(g) g, by rejection from the Maxwellian weighted by a line
 *   A(v) + B(v) |V|/s (s = sqrt(kT/m_gas)) that bounds sigma(g) g over every
 *   relative speed a partner of speed |V| can give: the edge of the upper
 *   concave hull of that bound spanning the Maxwellian's mean |V|/s (at most
 *   max_attempts attempts, the last attempt is kept);
 *   impact parameter b = b_max sqrt(RN); azimuth 2 pi RN in the orthonormal
 *   basis of Duff et al. (JCGT 2017); Firsov screening length
 *   a = 0.8853 a_0 (Z1^1/2 + Z2^1/2)^(-2/3).
 *
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11) with key = (seed low
 * word, seed high word) and counter = (particle id, stream, event, block), the
 * stream being the instance index unless sput_instance.rng_stream sets it.
 * Event 0 is the launch (block 0: racetrack radius, racetrack azimuth, energy,
 * polar cosine; block 1 word 0: emission azimuth).  Event k >= 1 is flight k
 * (block 0: flight length, impact parameter, scattering azimuth; block 1+a,
 * a < max_attempts: partner attempt a, two Box-Muller pairs from its four
 * words, and one more uniform from the low bytes of words 0, 1, 2 joined as
 * x = (w0 & 255) << 24 | (w1 & 255) << 16 | (w2 & 255) << 8, which selects the
 * proposal's branch and, rescaled within it, is the acceptance uniform).  A 32-bit word x maps to RN = ((x >> 8) + 1) * 2^-24,
 * which uses only its upper 24 bits.
 * Every particle therefore has its own stream: integer tallies are bit-exact
 * and independent of launch configuration, order and chunking.
 *
 * Units: mm, eV, u (atomic mass units), K, Pa, radians.
 *
 * Conventions for every entry point:
 *   - Return value: SPUT_OK (0) or an error code; no exception or signal ever
 *     crosses the ABI, and a device error is reported, never trapped.
 *   - Ownership: sput_scene handles are created and freed by the library.
 *     Tally and record buffers are owned by the caller; the library never
 *     frees or reallocates them.  Input arrays are copied during the call and
 *     may be freed afterwards.
 *   - Device pointers are plain CUDA device addresses on the scene's device;
 *     `stream` is a cudaStream_t (NULL = legacy default stream).
 */
#ifndef SPUT_H
#define SPUT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SPUT_ABI_VERSION 5

typedef enum sput_status {
    SPUT_OK = 0,
    SPUT_ERR_INVALID_ARG = 1,     /* NULL pointer, bad size, bad enum value */
    SPUT_ERR_INVALID_SCENE = 2,   /* geometry / cathode / instance inconsistency */
    SPUT_ERR_CUDA = 3,            /* a CUDA runtime call failed (message via sput_last_error) */
    SPUT_ERR_TIMEOUT = 4,         /* host-side wait exceeded the caller's limit; device not reset */
    SPUT_ERR_DEVICE_CHECK = 5,    /* the kernel raised a status bit (see sput_run_stats.device_status) */
    SPUT_ERR_UNSUPPORTED = 6,     /* feature not available in this build */
    SPUT_ERR_NO_MEMORY = 7        /* host or device allocation failed */
} sput_status;

/* Surface primitives (Sec. "The SIMTRA Python wrapper": chamber, magnetron
 * body and "dummy" objects; every surface collects the atoms that reach it). */
typedef enum sput_prim_kind {
    SPUT_PRIM_BOX = 0,       /* the chamber box interior (sput_chamber.box_lo/hi); hit from inside */
    SPUT_PRIM_RECT = 1,      /* plane rectangle: |(q-c).u| <= p0, |(q-c).v| <= p1, normal u x v */
    SPUT_PRIM_DISC = 2,      /* plane disc / annulus: p0 <= |q-c| <= p1 in the (u, v) plane */
    SPUT_PRIM_CYLINDER = 3   /* open tube: axis u through c, radius p0, |(q-c).u| <= p1 */
} sput_prim_kind;

typedef enum sput_interaction {
    SPUT_INTERACTION_MOLIERE = 0,     /* screened Coulomb, Moliere screening (paper's choice) */
    SPUT_INTERACTION_HARD_SPHERE = 1  /* test potential: diameter hs_diameter, chi = 2 acos(b/d) */
} sput_interaction;

typedef enum sput_gas_motion {
    SPUT_GAS_THERMAL = 0,    /* Maxwellian gas at T (the paper accounts for the motion of the gas) */
    SPUT_GAS_STATIONARY = 1  /* gas atoms at rest (test mode) */
} sput_gas_motion;

typedef enum sput_count_type { SPUT_COUNT_INT32 = 0, SPUT_COUNT_INT64 = 1 } sput_count_type;

typedef struct sput_chamber {
    double box_lo[3], box_hi[3]; /* chamber interior, mm */
    int gas_Z;                   /* process gas atomic number (Ar: 18) */
    int reserved;
    double gas_mass;             /* u */
    double gas_T;                /* K, homogeneous gas in thermal equilibrium */
} sput_chamber;

typedef struct sput_primitive {
    int kind;                    /* sput_prim_kind */
    int reserved;
    double center[3];
    double u[3], v[3];           /* unit vectors (cylinder: u = axis, v unused) */
    double p0, p1;               /* sizes, see sput_prim_kind */
} sput_primitive;

typedef struct sput_geometry {
    int prim_begin, prim_count;  /* a contiguous range of the scene's primitives */
    int substrate;               /* index (within the range) of the tallied RECT or DISC */
    int reserved;
} sput_geometry;

typedef struct sput_cathode {
    int Z;                       /* target element atomic number */
    int target;                  /* index, within each geometry that uses it, of the target DISC */
    double mass;                 /* u */
    double U_s;                  /* surface binding energy, eV */
    double center[3], normal[3], e1[3]; /* target-surface centre, outward unit normal, in-plane unit axis */
    double rt_r0, rt_sigma, rt_R;       /* racetrack depth d(r) = exp(-(r-r0)^2/(2 sigma^2)) on [0, R];
                                            radial pdf proportional to r d(r) (axisymmetric profile) */
    double cos_coef[6];          /* c_0..c_5 of the emission cosine sum; (0,1,0,0,0,0) = cosine */
    /* Optional joint launch distribution in (polar cosine, energy), e.g. binned output of a
     * binary-collision code for the target (angle-dependent energy distributions, Sec. "The
     * SIMTRA model").  launch_table[i * n_E + k] >= 0 is the weight of the cell
     * mu = cos(theta) in [i, i+1) / n_mu and E in [k, k+1) * E_hi / n_E, with a uniform density
     * inside each cell.  The polar cosine is drawn from the marginal over mu (launch word u_mu),
     * the energy from the row of the drawn mu cell (word u_E); Thompson law, E_i, k and
     * cos_coef are then not used for this cathode.  NULL = off.  Copied during
     * sput_scene_create; 1 <= n_mu, n_E <= 256, E_hi > 0, weights finite, sum > 0. */
    const double* launch_table;
    int n_mu, n_E;
    double E_hi;                 /* eV, upper end of the table's energy range */
} sput_cathode;

typedef struct sput_instance {   /* one (cathode, process condition) pair */
    int geometry, cathode;
    double pressure;             /* Pa */
    double E_i;                  /* incident ion energy, eV (set by the discharge voltage) */
    double k;                    /* head-on factor of the cut-off, 0.4 in the paper */
    uint64_t n_particles;        /* < 2^32 per instance */
    uint32_t rng_stream;         /* word 1 of the Philox counter: 0 = the instance index; s > 0 = s - 1.
                                    Instances with the same stream draw the same random numbers for the
                                    same particle ids (common random numbers across conditions, e.g. the
                                    tilts of a scan) */
    uint32_t reserved;
} sput_instance;

typedef struct sput_grid {
    int nx, ny;                  /* cells along substrate u and v */
    double half_u, half_v;       /* grid covers [-half_u, half_u] x [-half_v, half_v] around the centre */
    int count_type;              /* sput_count_type of the per-cell counts */
    int n_ebins;                 /* arrival-energy histogram bins on [0, e_hist_max] (0 = off) */
    double e_hist_max;           /* eV */
    int n_abins;                 /* arrival-angle histogram bins on [0, 90] degrees (0 = off) */
    int reserved;
} sput_grid;

typedef struct sput_physics {
    double chi_min;              /* rad, CM deflection that defines sigma (default 1 degree) */
    double hs_diameter;          /* Angstrom, hard-sphere test potential only */
    int interaction;             /* sput_interaction */
    int gas_motion;              /* sput_gas_motion */
    int max_attempts;            /* partner rejection attempts per collision, 1..64 */
    int reserved;
    int64_t max_collisions;      /* per particle; beyond it the atom counts as timed out */
    double thermal_switch_eV;    /* diffusion shortcut for thermalised atoms (0 = off, the exact model):
                                    once a collision leaves the atom below this energy, it moves on as
                                    an isotropic random walk with exponential steps of mean
                                    lambda_D = 3 D_12 / vbar_1 (D_12 the first Chapman-Enskog diffusion
                                    coefficient from the momentum-transfer cross section, vbar_1 the mean
                                    thermal speed of the atom), speed frozen; thermal gas only; not
                                    combined with the temperature score */
} sput_physics;

typedef struct sput_scene_desc {
    uint32_t abi_version;        /* SPUT_ABI_VERSION */
    int n_prims, n_geoms, n_cathodes, n_instances;
    sput_chamber chamber;
    const sput_primitive* prims;
    const sput_geometry* geoms;
    const sput_cathode* cathodes;
    const sput_instance* instances;
    sput_grid grid;
    sput_physics physics;
} sput_scene_desc;

typedef struct sput_scene sput_scene;

/* Per-particle record (optional), indexed by ticket = instance prefix + id. */
typedef struct sput_record {
    int32_t prim;                /* local primitive index hit, -1 = timed out */
    int32_t cell;                /* substrate cell (front face), -1 otherwise */
    float energy;                /* arrival energy, eV */
    float cos_angle;             /* |cos| of the arrival angle to the substrate normal (front hits) */
    uint32_t n_collisions;
    float score;                 /* d ln p(path) / d ln n_gas, likelihood-ratio score */
} sput_record;

/* Caller-owned DEVICE buffers; NULL = not requested.  Layouts (row-major):
 *   counts       [n_instances][ny][nx]   int32 or int64 (grid.count_type)
 *   energy       [n_instances][ny][nx]   double, sum of arrival energies (eV)
 *   score        [n_instances][ny][nx]   double, sum of the landing atoms' scores
 *   prim_counts  [n_instances][max_prims] int64, landings per local primitive
 *   timed_out    [n_instances]           int64
 *   hist_E       [n_instances][n_ebins]  int64 (front substrate hits)
 *   hist_A       [n_instances][n_abins]  int64 (front substrate hits)
 *   records      [ticket_end - ticket_begin] sput_record, row = ticket - ticket_begin
 * max_prims = the largest prim_count of any geometry; n_tickets = sum of n_particles;
 * ticket = (sum of n_particles of the earlier instances) + particle id. */
typedef struct sput_tallies {
    void* counts;
    double* energy;
    double* score;
    int64_t* prim_counts;
    int64_t* timed_out;
    int64_t* hist_E;
    int64_t* hist_A;
    sput_record* records;
    double* score_T;             /* [inst][ny][nx] sum over landings of d ln p(path)/dT at fixed
                                    pressure (1/K): the collision rate through n_g = p/(k_B T) and
                                    <sigma g>(v; T), and the Maxwellian partner density */
} sput_tallies;

typedef struct sput_tally_layout {
    int n_instances, nx, ny, max_prims, n_ebins, n_abins;
    int count_type;
    int reserved;
    uint64_t n_tickets;
} sput_tally_layout;

typedef struct sput_run_opts {
    uint64_t seed;
    uint64_t ticket_begin, ticket_end; /* run tickets [begin, end); end = 0 means all */
    int accumulate;              /* 0: zero the requested tallies first; 1: add into them */
    int block_threads;           /* 0 = scene default (256, or the autotuned value); else a multiple of 32 in [32, 256] */
    int blocks_per_sm;           /* 0 = scene default (occupancy limit, or the autotuned value) */
    int ticket_chunk;            /* tickets a warp takes per refill; 0 = scene default (32, or autotuned) */
    int timeout_ms;              /* host wait limit when stats are requested; 0 = none */
    int flags;                   /* SPUT_RUN_* bits */
} sput_run_opts;

/* sput_run_opts.flags */
#define SPUT_RUN_NO_SMEM_COUNTERS 1 /* count landings per primitive with global atomics only */
#define SPUT_RUN_SMEM_COUNTERS 2    /* privatise them in shared memory (when they fit); default: scene choice */
#define SPUT_RUN_LAUNCH_AT_CUTOFF 4 /* every atom launches with E = E_max (all other draws unchanged): the
                                       boundary run of the derivative with respect to the Thompson cut-off,
                                       d E[f]/dE_max = p(E_max) (E[f | E = E_max] - E[f]),
                                       p(E_max) = 2 U_s / (E_max (E_max + U_s)); Thompson cathodes only */
#define SPUT_RUN_NO_CELL_MASKS 16   /* surface test over every primitive, by a counted loop */
#define SPUT_RUN_CELL_MASKS 32      /* surface test restricted by the cell masks: a flight of length <= h (2 h)
                                       tests only the primitives whose bounding sphere meets the cells within 1
                                       (2) of its start, h = the chamber's longest side / 32 (geometries of at
                                       most 64 primitives).  Default: on when the largest geometry has more than
                                       32 primitives.  Results are identical either way; only the speed differs */
#define SPUT_RUN_INJECT_NONFINITE 8 /* failure-path test aid: particle 0 of every instance starts with a NaN
                                       speed; the kernel retires it as timed out, sets the non-finite bit of
                                       device_status and the call returns SPUT_ERR_DEVICE_CHECK (with stats) */

typedef struct sput_run_stats {
    uint64_t particles;          /* particles that completed (landed or timed out) */
    uint64_t landed;
    uint64_t timed_out;
    uint64_t flights;            /* free flights (one per cycle) */
    uint64_t collisions;         /* binary collisions */
    uint64_t attempts;           /* partner rejection attempts */
    uint32_t device_status;      /* bit mask of device checks, 0 = clean */
    uint32_t grid_blocks;        /* launch shape that ran */
    uint32_t block_threads;
    float kernel_ms;             /* device time of the transport kernel (CUDA events) */
} sput_run_stats;

/* Library version (SPUT_ABI_VERSION) and status text. */
int sput_version(void);
const char* sput_status_str(sput_status s);
/* Text of the last error on this thread (CUDA error string or validation message). */
const char* sput_last_error(void);

/* Validate the description, build the interaction tables (FP64 on the host:
 * b_max(eps) and the head-on apsis in reduced Moliere units, <sigma g>(v) and
 * the partner rejection envelope per cathode/gas pair, the deflection table,
 * racetrack guesses, the surface test's cell masks) and copy
 * scene and tables to `device`.  On success *out owns device memory until
 * sput_scene_destroy.  Errors: INVALID_ARG, INVALID_SCENE (found on the host
 * before any CUDA call, e.g. an instance whose Thompson cut-off
 * E_max = k Lambda E_i - U_s is not positive), CUDA, NO_MEMORY, and UNSUPPORTED
 * when the primitives and small tables a block stages do not fit its shared
 * memory (about 2800 primitives).  Geometries of more than 64 primitives run the
 * surface test without cell masks. */
sput_status sput_scene_create(const sput_scene_desc* desc, int device, sput_scene** out);

/* Replace the instance table (pressures, ion energies, k, particle counts).
 * The number of instances and each instance's geometry and cathode must stay
 * the same (tables do not depend on them).  Synchronous host->device copy. */
sput_status sput_instances_set(sput_scene* scene, const sput_instance* instances, int n_instances);

/* Sizes of the tally buffers (see sput_tallies). */
sput_status sput_tally_layout_get(const sput_scene* scene, sput_tally_layout* out);

/* Transport the tickets of opts on `stream`.  Tallies are device pointers
 * owned by the caller.  With stats == NULL the call only enqueues work (no
 * host synchronisation).  With stats != NULL it waits for the kernel (at most
 * opts->timeout_ms when > 0, else SPUT_ERR_TIMEOUT without touching the
 * device) and fills the counters.  Concurrent runs of one scene on different
 * streams race on the scene's scratch counters: serialise them. */
sput_status sput_run(sput_scene* scene, const sput_run_opts* opts, void* stream, const sput_tallies* tallies,
                     sput_run_stats* stats);

/* Same as sput_run with HOST tally buffers (any subset non-NULL, same layouts):
 * the library runs into scene-owned device buffers and copies the requested
 * tallies back before returning.  Always synchronous. */
sput_status sput_run_host(sput_scene* scene, const sput_run_opts* opts, const sput_tallies* host_tallies,
                          sput_run_stats* stats);

/* Same transport as sput_run, for callers that must not allocate device memory
 * at run time: code recorded into a CUDA graph under a global-mode stream
 * capture (where cudaMalloc is not permitted), processes whose device memory
 * is owned by another allocator that has reserved it, or latency-critical
 * loops that keep the driver allocator (which may synchronise the device) off
 * their path.  sput_run allocates its run scratch (ticket counter, statistics,
 * status word: 64 bytes) on its first call for a scene; this variant instead
 * uses a static array of 256 bytes in the library's module memory, which every
 * GPU that loads the library holds until the process exits.  It never calls
 * cudaMalloc, cudaFree or any other allocating routine; the scene (inputs) and
 * the tallies (outputs) are passed in exactly as for sput_run.
 *   - The first call in a CUDA context of a device looks up the array's device
 *     address with that device current and caches it under the context's id
 *     (a context created again after cudaDeviceReset looks it up afresh); make
 *     that first call before any stream capture.
 *   - All calls on one device share the array and it keeps the last call's
 *     contents; each call clears the counters it needs before its kernel.
 *     Calls whose work overlaps on the GPU (other streams, other threads,
 *     other scenes on the same device) race on it: serialise them.
 *   - A run whose scratch would exceed the array's capacity is rejected with
 *     SPUT_ERR_UNSUPPORTED and a message naming both sizes.
 *   - With stats != NULL the call waits for the stream (opts->timeout_ms
 *     applies) and also reuses the scene's pinned statistics buffer and its two
 *     timing events for kernel_ms; a run of the same scene that overlaps this
 *     one overwrites them, which is one more reason to serialise such calls.
 * The paper has no counterpart of this entry point. */
sput_status sput_run_noalloc(sput_scene* scene, const sput_run_opts* opts, void* stream, const sput_tallies* tallies,
                             sput_run_stats* stats);

/* Autotuner: time candidate launch shapes (threads per block, blocks per SM,
 * ticket chunk, shared-memory counters) on `sample_tickets` tickets taken as
 * four equal ranges spread over the scene's ticket space, and keep the fastest
 * (most collisions per second of kernel time) as the scene default for runs
 * whose opts leave those fields 0.  Uses `tallies` as scratch output (their
 * contents are overwritten).  Synchronous.  The results of every candidate are
 * reported in *out. */
typedef struct sput_tune_result {
    int block_threads, blocks_per_sm, ticket_chunk, flags; /* the chosen shape */
    float best_rate;             /* collisions per second of kernel time on the sample */
    int n_candidates;
    int reserved;
    int cand_threads[32], cand_bps[32], cand_chunk[32], cand_flags[32];
    float cand_rate[32];
} sput_tune_result;

sput_status sput_autotune(sput_scene* scene, const sput_run_opts* base, void* stream, const sput_tallies* tallies,
                          uint64_t sample_tickets, sput_tune_result* out);

/* CUDA graph of one run (tally clearing when opts->accumulate == 0, scratch
 * clearing and the transport kernel), captured on `stream` and instantiated.
 * sput_graph_launch replays it on `stream` with a new seed (the kernel node's
 * parameters are updated in the executable graph).  The graph keeps the
 * tally pointers and ticket range it was made with.  The scene must outlive
 * the graph; a run or launch of the scene must not overlap another. */
typedef struct sput_graph sput_graph;

sput_status sput_graph_create(sput_scene* scene, const sput_run_opts* opts, void* stream, const sput_tallies* tallies,
                              sput_graph** out);
sput_status sput_graph_launch(sput_graph* graph, uint64_t seed, void* stream);
void sput_graph_destroy(sput_graph* graph);

/* Likelihood-ratio backward pass for the gas pressure.  Pressure enters only
 * through the free flights (Eq. for lambda with lambda_m = v/(n_g <sigma g>),
 * n_g = p/(k_B T)); the forward run accumulates, per tally cell, the score
 * S = sum over collisions (1 - l_k/lambda_k) - t_land/lambda_land = d ln p(path)/d ln n_g
 * of every landing atom (sput_tallies.score).  Then d E[count]/d ln p equals the
 * expected score tally, and for a loss L
 *   grad_log_pressure[i] = sum_cells grad_counts[i][cell] * score_tally[i][cell]
 * estimates dL/d ln p_i.  All pointers are DEVICE arrays in the tally layout of
 * `scene` ([n_instances][ny][nx], double; output [n_instances]).  Asynchronous on
 * `stream`.  The paper computes no gradients; this is the adjoint of its transport. */
sput_status sput_backward(const sput_scene* scene, const double* grad_counts, const double* score_tally,
                          double* grad_log_pressure, void* stream);

/* Arrival counts -> composition in at.% (Methods paragraph after Table 1: arrival
 * fractions weighted with the sputter rates, then with bulk density and atomic
 * mass).  For cathode j and measurement point m,
 *   a_j(m) = R_j(P_j) N_j(m)/N_j(ref) rho_j/M_j,   composition[m][j] = 100 a_j(m) / sum_k a_k(m),
 * N_j(m) the counts of cathode j summed over the cells with patch_of_cell == m, ref
 * the reference point, R_j(P) the line through the two calibration points.
 *   counts         DEVICE int64 [n_cathodes][n_cells] (the first n_cathodes instances' counts)
 *   patch_of_cell  DEVICE int32 [n_cells], point index or -1
 *   calibration    HOST double [n_cathodes][6] = (P_a, R_a, P_b, R_b, density, atomic mass)
 *   power          HOST double [n_cathodes]
 *   patch_counts   DEVICE double [n_cathodes][n_points] (output, kept for the backward pass)
 *   composition    DEVICE double [n_points][n_cathodes] (output)
 * n_cathodes <= 16.  Asynchronous on `stream`. */
sput_status sput_composition(int n_cathodes, int n_cells, int n_points, const int64_t* counts,
                             const int32_t* patch_of_cell, int ref_point, const double* calibration,
                             const double* power, double* patch_counts, double* composition, void* stream);

/* Derivative with respect to the incident ion energy E_i of every instance, through the
 * Thompson cut-off E_max = k Lambda E_i - U_s (Eq. for phi(E)); E_i follows the discharge
 * voltage, hence the cathode power.  The launch density moves its support with E_max, so
 *   d E[count_c]/dE_max = p(E_max) (E[count_c | E = E_max] - E[count_c]),
 *   p(E_max) = 2 U_s / (E_max (E_max + U_s)),
 * and grad_ion_energy[i] = k Lambda p(E_max) sum_c grad_counts[i][c] (counts_cutoff[i][c] - counts[i][c]).
 * counts: a run's count tally; counts_cutoff: the same particles and seed run with
 * SPUT_RUN_LAUNCH_AT_CUTOFF (DEVICE, the scene's count type, [inst][ny][nx]); grad_counts
 * DEVICE double [inst][ny][nx]; grad_ion_energy DEVICE double [inst], per eV.  Thompson
 * cathodes only (a launch table has no cut-off).  Asynchronous on `stream`. */
sput_status sput_emax_backward(const sput_scene* scene, const double* grad_counts, const void* counts,
                               const void* counts_cutoff, double* grad_ion_energy, void* stream);

/* Incident ion energy from the cathode power through the discharge voltage.  Table S1
 * gives the discharge voltage (DC) or bias (RF) of every element and supply at two
 * powers; the voltage is read as the line through them, and singly charged ions give
 * E_i = e V (so E_i in eV equals V in volts):
 *   ion_energy[j] = V_a + (V_b - V_a) (power[j] - P_a) / (P_b - P_a),
 * voltage HOST double [n][4] = (P_a, V_a, P_b, V_b) per cathode (W, V), power HOST [n] (W),
 * ion_energy HOST [n] (eV, output; feed it to sput_instances_set).  1 <= n <= 4096; the
 * two points of a line must be finite with P_a != P_b, else SPUT_ERR_INVALID_ARG.
 * Host only, synchronous, touches no device. */
sput_status sput_ion_energy(int n, const double* voltage, const double* power, double* ion_energy);

/* The power's path through the discharge voltage to the Thompson cut-off, in one call:
 * the sput_emax_backward contraction per instance, grad_ion_energy[i] = dL/dE_i (DEVICE
 * double [n_instances], written), and then
 *   grad_power[i] += grad_ion_energy[i] * dE_i/dP_i,   dE_i/dP_i = (V_b - V_a)/(P_b - P_a)
 * (DEVICE double [n_instances], accumulated into, e.g. after sput_composition_backward has
 * written the rate-line term).  voltage HOST [n_instances][4] as for sput_ion_energy;
 * counts / counts_cutoff / grad_counts as for sput_emax_backward.  At most 16 instances
 * (one per cathode of a composition map).  Asynchronous on `stream`. */
sput_status sput_voltage_backward(const sput_scene* scene, const double* voltage, const double* grad_counts,
                                  const void* counts, const void* counts_cutoff, double* grad_ion_energy,
                                  double* grad_power, void* stream);

/* Backward pass of sput_composition: from grad_composition (DEVICE [n_points][n_cathodes])
 * and the forward's patch_counts, writes grad_patch (DEVICE [n_cathodes][n_points], scratch
 * owned by the caller), grad_counts (DEVICE double [n_cathodes][n_cells]) and grad_power
 * (DEVICE double [n_cathodes], through dR_j/dP_j).  Asynchronous on `stream`. */
sput_status sput_composition_backward(int n_cathodes, int n_cells, int n_points, const double* patch_counts,
                                      const int32_t* patch_of_cell, int ref_point, const double* calibration,
                                      const double* power, const double* grad_composition, double* grad_patch,
                                      double* grad_counts, double* grad_power, void* stream);

/* Measured throughput of the units the transport kernel issues to, for its roofline
 * (no counterpart in the paper; measurement only).  One kernel per call, launched with
 * SMs x 8 blocks of 256 threads; a warm-up launch, then one launch timed with CUDA events
 * on `stream`.  Synchronous.
 *   SPUT_MB_FFMA      FP32 fused multiply-adds (lane-ops)
 *   SPUT_MB_MUFU_*    lg2 / ex2 / rsqrt / sin on the MUFU (XU) pipe, approximate forms (lane-ops)
 *   SPUT_MB_PHILOX    Philox4x32-10 blocks (10 rounds of the generator the transport uses)
 *   SPUT_MB_RED_*     L2 reductions (atomic adds whose result is unused, as in the landing
 *                     tally) of int32 / int64 / fp64 at pseudo-random slots of an array of
 *                     n_slots elements
 * scratch: DEVICE buffer owned by the caller; the reductions use its first n_slots
 * elements (cleared first), the other kinds need room for SMs * 8 * 256 floats (a sink
 * that is written only under a condition that never holds).  iters in [1, 2^24] sets the
 * work per thread.  out->ops counts the lane-ops (or blocks, or reductions) of the timed
 * launch, out->ms its device time. */
typedef enum sput_microbench_kind {
    SPUT_MB_FFMA = 0,
    SPUT_MB_MUFU_LG2 = 1,
    SPUT_MB_MUFU_EX2 = 2,
    SPUT_MB_MUFU_RSQ = 3,
    SPUT_MB_MUFU_SIN = 4,
    SPUT_MB_PHILOX = 5,
    SPUT_MB_RED_I32 = 6,
    SPUT_MB_RED_I64 = 7,
    SPUT_MB_RED_F64 = 8
} sput_microbench_kind;

typedef struct sput_microbench_result {
    double ops;                  /* units of work in the timed launch */
    double ms;                   /* its device time */
    double ops_per_s;
    int blocks, threads;         /* launch shape */
} sput_microbench_result;

sput_status sput_microbench(int device, int kind, int n_slots, void* scratch, size_t scratch_bytes, int iters,
                            void* stream, sput_microbench_result* out);

/* Free the scene and its device memory. */
void sput_scene_destroy(sput_scene* scene);

/* Diagnostics: evaluate one step of the device code path on given inputs
 * (device functions identical to those of the transport kernel), for parity
 * tests.  `x` and `y` are HOST arrays; layouts per `what`:
 *   SPUT_PROBE_CHI      x[2n] = (eps, beta) reduced units, pair p -> y[n] = chi (rad) by the direct
 *                       Gauss-Mehler integration (the device's path outside the deflection table)
 *   SPUT_PROBE_CHI_U    x[2n] = (eps, u)          -> y[n] = chi (rad) as a collision computes it from
 *                       the impact-parameter uniform u (b = b_max(eps) sqrt(u)): the deflection
 *                       table inside its range, the direct integration outside
 *   SPUT_PROBE_BMAX     x[n]  = eps                        -> y[n] = b_max / a
 *   SPUT_PROBE_K        x[n]  = speed (km/s), pair p       -> y[n] = <sigma g> (A^2 km/s)
 *   SPUT_PROBE_M        x[n]  = speed (km/s), pair p       -> y[2n] = (A, B): the partner-rejection
 *                       envelope A + B |V|/s (A^2 km/s) at atom speed v
 *   SPUT_PROBE_LAUNCH   x[n]  = particle id, instance p    -> y[7n] = (x,y,z, dx,dy,dz, E)
 *   SPUT_PROBE_TRACE    x[n]  = particle id, instance p    -> y[640n]: 64 rows of
 *       (x,y,z, dx,dy,dz, speed, status, a, t): row 0 the launch (status -1), row r the
 *       state after flight r (status 0 collided: position = collision point, direction and
 *       speed after the collision, a = partner attempts, t = flight length; 1 landed:
 *       position = hit point, a = primitive, t = hit distance; 2 timed out; -2 unused)
 * p is the pair index (one per distinct cathode element) or the instance index.
 * This call allocates and frees temporary device buffers. */
typedef enum sput_probe_kind {
    SPUT_PROBE_CHI = 0,
    SPUT_PROBE_BMAX = 1,
    SPUT_PROBE_K = 2,
    SPUT_PROBE_M = 3,
    SPUT_PROBE_LAUNCH = 4,
    SPUT_PROBE_TRACE = 5,
    SPUT_PROBE_CHI_U = 6
} sput_probe_kind;

sput_status sput_probe(sput_scene* scene, int what, int p, int n, const double* x, double* y);

/* Host evaluation, in FP64, of the deflection table the device uses for the Moliere
 * potential (the paper's screened Coulomb interaction, Sec. "The SIMTRA model"), built
 * once per chi_min: q = ln tan(chi/2) over x = ln eps and y = ln(b/b_max) = (ln u)/2 as
 * bicubic cells through FP64 node values of the classical deflection integral
 * (x in [-26, -4] step 1/4; y in [-6, -1] step 1/32 and [-1, 0] step 1/128).  For each
 * i < n: chi[i] (rad) at reduced energy eps[i] > 0 and impact-parameter uniform
 * 0 < u[i] <= 1; outside the table the FP64 deflection at b = b_max sqrt(u).  HOST arrays;
 * no device is touched.  Errors: INVALID_ARG. */
sput_status sput_deflection_table_eval(double chi_min, int n, const double* eps, const double* u, double* chi);

#ifdef __cplusplus
}
#endif
#endif /* SPUT_H */
