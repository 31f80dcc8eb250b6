// sput_adjoint.cu -- likelihood-ratio backward pass and the arrival-count ->
// composition map with its backward pass (sm_103a).
//
// Pressure enters the transport only through the free flights (Eq. for
// lambda: lambda_m = v / (n_g <sigma g>), n_g = p / (k_B T)).  The forward
// kernel accumulates for every landing atom the score
//   S = sum over collisions (1 - l_k/lambda_k) - t_land/lambda_land
//     = d ln p(path) / d ln n_g,
// per tally cell.  Hence d E[count_c] / d ln p = E[sum_{atoms in c} S]; the
// backward kernel contracts dL/dcount with that score tally.
//
// Composition (Methods paragraph after Table 1: arrival fractions weighted
// with the sputter rates, then with bulk density and atomic mass, in at.%):
//   a_j(m) = R_j(P_j) * N_j(m) / N_j(ref) * rho_j / M_j,   c_j(m) = 100 a_j(m) / sum_k a_k(m),
// N_j(m) the arrivals of cathode j summed over measurement patch m, ref the
// central patch, R_j linear in power through two calibration points.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>

#include "sput.h"
#include "sput_internal.h"

namespace {

constexpr int kMaxCath = 16;

struct CompParams {
    int n_cath, n_cells, n_points, ref;
    double R[kMaxCath];      // R_j(P_j)
    double dRdP[kMaxCath];   // slope of the rate line
    double w[kMaxCath];      // rho_j / M_j
};

__device__ double warp_sum(double x)
{
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    return x;
}

// grad[i] = sum_c g[i][c] * score[i][c], one block per instance
__global__ void lr_backward_kernel(const double* g, const double* score, double* grad, long long n_cells)
{
    __shared__ double part[32];
    const long long base = (long long)blockIdx.x * n_cells;
    double s = 0.0;
    for (long long c = threadIdx.x; c < n_cells; c += blockDim.x) s += g[base + c] * score[base + c];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
        t = warp_sum(t);
        if (threadIdx.x == 0) grad[blockIdx.x] = t;
    }
}

// Derivative with respect to the Thompson cut-off.  The launch energy has the
// density p(E) = E/(E+U)^3 / Z(E_max) on (0, E_max], Z = E_max^2 / (2U (E_max+U)^2),
// so d ln p(E)/dE_max = -p(E_max) for every E inside the support, and the moving
// end of the support adds p(E_max) E[f | E = E_max]:
//   d E[f]/dE_max = p(E_max) (E[f | E = E_max] - E[f]),  p(E_max) = 2U / (E_max (E_max + U)).
// With a boundary run of the same particles launched at E_max (counts_cut) and
// dE_max/dE_i = k Lambda, one block per instance forms
//   grad[i] = k Lambda p(E_max) sum_c g[i][c] (counts_cut[i][c] - counts[i][c]).
// Voltage lines V_i(P) = V_a + (V_b - V_a)(P - P_a)/(P_b - P_a) (Table S1), with
// E_i = e V for singly charged ions: dE_i/dP_i in eV/W per instance.
struct VoltParams {
    double dEdP[kMaxCath];
};

// grad_power (optional) gets grad[i] * dE_i/dP_i added: the path from the cathode
// power through the discharge voltage to the cut-off.
template <typename CountT>
__global__ void emax_backward_kernel(const double* g, const CountT* counts, const CountT* counts_cut,
                                     const sput::DevInstance* inst, double* grad, long long n_cells,
                                     double* grad_power, VoltParams vp)
{
    __shared__ double part[32];
    const long long base = (long long)blockIdx.x * n_cells;
    double s = 0.0;
    for (long long c = threadIdx.x; c < n_cells; c += blockDim.x)
        s += g[base + c] * ((double)counts_cut[base + c] - (double)counts[base + c]);
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
        t = warp_sum(t);
        if (threadIdx.x == 0) {
            const sput::DevInstance I = inst[blockIdx.x];
            const double q = I.thompson_q, U = I.U_s;
            const double Em = U * q / (1.0 - q);
            const double gE = (double)I.kLambda * 2.0 * U / (Em * (Em + U)) * t;
            grad[blockIdx.x] = gE;
            if (grad_power) grad_power[blockIdx.x] += gE * vp.dEdP[blockIdx.x];
        }
    }
}

// N[j][m] = sum of counts of cathode j over the cells of patch m
__global__ void patch_sum_kernel(const long long* counts, const int32_t* patch, double* N, int n_cath, int n_cells,
                                 int n_points)
{
    const long long total = (long long)n_cath * n_cells;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(i / n_cells), c = (int)(i % n_cells);
        const int m = patch[c];
        if (m >= 0 && m < n_points && counts[i]) atomicAdd(N + (size_t)j * n_points + m, (double)counts[i]);
    }
}

__global__ void composition_kernel(const double* N, double* comp, CompParams cp)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= cp.n_points) return;
    double a[kMaxCath], A = 0.0;
    for (int j = 0; j < cp.n_cath; ++j) {
        const double nref = N[(size_t)j * cp.n_points + cp.ref];
        a[j] = nref > 0.0 ? cp.R[j] * N[(size_t)j * cp.n_points + m] / nref * cp.w[j] : 0.0;
        A += a[j];
    }
    for (int j = 0; j < cp.n_cath; ++j) comp[(size_t)m * cp.n_cath + j] = A > 0.0 ? 100.0 * a[j] / A : 0.0;
}

// dL/dN[j][m] and dL/dP_j from dL/dc[m][j]; one block of >= n_points threads
__global__ void composition_backward_kernel(const double* N, const double* gc, double* gN, double* gP, CompParams cp)
{
    __shared__ double ref_acc[kMaxCath];
    __shared__ double rate_acc[kMaxCath];
    if (threadIdx.x < kMaxCath) {
        ref_acc[threadIdx.x] = 0.0;
        rate_acc[threadIdx.x] = 0.0;
    }
    __syncthreads();
    for (int m = threadIdx.x; m < cp.n_points; m += blockDim.x) {
        double a[kMaxCath], A = 0.0, gdotc = 0.0;
        for (int j = 0; j < cp.n_cath; ++j) {
            const double nref = N[(size_t)j * cp.n_points + cp.ref];
            a[j] = nref > 0.0 ? cp.R[j] * N[(size_t)j * cp.n_points + m] / nref * cp.w[j] : 0.0;
            A += a[j];
        }
        if (A <= 0.0) {
            for (int j = 0; j < cp.n_cath; ++j) gN[(size_t)j * cp.n_points + m] = 0.0;
            continue;
        }
        for (int j = 0; j < cp.n_cath; ++j) gdotc += gc[(size_t)m * cp.n_cath + j] * 100.0 * a[j] / A;
        for (int j = 0; j < cp.n_cath; ++j) {
            // dL/da_j = (100/A) (g_j - sum_k g_k c_k / 100)
            const double ga = 100.0 / A * (gc[(size_t)m * cp.n_cath + j] - gdotc / 100.0);
            const double nref = N[(size_t)j * cp.n_points + cp.ref];
            gN[(size_t)j * cp.n_points + m] = nref > 0.0 ? ga * cp.R[j] * cp.w[j] / nref : 0.0;
            // a_j(m) depends on N_j(ref) through 1/N_j(ref) and on R_j linearly
            if (nref > 0.0) atomicAdd(&ref_acc[j], -ga * a[j] / nref);
            if (cp.R[j] != 0.0) atomicAdd(&rate_acc[j], ga * a[j] / cp.R[j]);
        }
    }
    __syncthreads();
    if (threadIdx.x < cp.n_cath) {
        gN[(size_t)threadIdx.x * cp.n_points + cp.ref] += ref_acc[threadIdx.x];
        gP[threadIdx.x] = rate_acc[threadIdx.x] * cp.dRdP[threadIdx.x];
    }
}

// dL/dcount[j][c] = dL/dN[j][patch(c)]
__global__ void scatter_kernel(const double* gN, const int32_t* patch, double* gcounts, int n_cath, int n_cells,
                               int n_points)
{
    const long long total = (long long)n_cath * n_cells;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(i / n_cells), c = (int)(i % n_cells);
        const int m = patch[c];
        gcounts[i] = (m >= 0 && m < n_points) ? gN[(size_t)j * n_points + m] : 0.0;
    }
}

sput_status adj_fail(sput_status s, const char* msg)
{
    sput::set_last_error(msg);
    return s;
}

sput_status comp_params(int n_cath, int n_cells, int n_points, int ref, const double* cal, const double* power,
                        CompParams& cp)
{
    if (n_cath < 1 || n_cath > kMaxCath) return adj_fail(SPUT_ERR_INVALID_ARG, "n_cathodes must be 1..16");
    if (n_cells < 1 || n_points < 1 || ref < 0 || ref >= n_points) return adj_fail(SPUT_ERR_INVALID_ARG, "bad sizes");
    if (!cal || !power) return adj_fail(SPUT_ERR_INVALID_ARG, "NULL calibration or power");
    std::memset(&cp, 0, sizeof cp);
    cp.n_cath = n_cath;
    cp.n_cells = n_cells;
    cp.n_points = n_points;
    cp.ref = ref;
    for (int j = 0; j < n_cath; ++j) {
        const double* q = cal + 6 * j;  // P_a, R_a, P_b, R_b, density, mass
        if (q[2] == q[0] || !(q[5] > 0.0)) return adj_fail(SPUT_ERR_INVALID_ARG, "bad calibration row");
        const double slope = (q[3] - q[1]) / (q[2] - q[0]);
        cp.R[j] = q[1] + slope * (power[j] - q[0]);
        cp.dRdP[j] = slope;
        cp.w[j] = q[4] / q[5];
    }
    return SPUT_OK;
}

}  // namespace

extern "C" {

sput_status sput_backward(const sput_scene* scene, const double* grad_counts, const double* score_tally,
                          double* grad_log_pressure, void* stream)
{
    sput::NvtxRange nvtx("sput_backward");
    if (!scene || !grad_counts || !score_tally || !grad_log_pressure) return adj_fail(SPUT_ERR_INVALID_ARG, "NULL argument");
    sput_tally_layout L;
    sput_status st = sput_tally_layout_get(scene, &L);
    if (st != SPUT_OK) return st;
    const long long n_cells = (long long)L.nx * L.ny;
    lr_backward_kernel<<<L.n_instances, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(grad_counts, score_tally,
                                                                                        grad_log_pressure, n_cells);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return adj_fail(SPUT_ERR_CUDA, cudaGetErrorString(e));
    return SPUT_OK;
}

}  // extern "C"

namespace {

sput_status emax_backward_launch(const sput_scene* scene, const double* grad_counts, const void* counts,
                                 const void* counts_cutoff, double* grad_ion_energy, double* grad_power,
                                 const VoltParams& vp, void* stream)
{
    sput_tally_layout L;
    sput_status st = sput_tally_layout_get(scene, &L);
    if (st != SPUT_OK) return st;
    if (grad_power && L.n_instances > kMaxCath)
        return adj_fail(SPUT_ERR_INVALID_ARG, "the voltage path supports at most 16 instances");
    const long long n_cells = (long long)L.nx * L.ny;
    const sput::DevInstance* inst = sput::scene_device_instances(scene);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (L.count_type == SPUT_COUNT_INT64)
        emax_backward_kernel<<<L.n_instances, 256, 0, s>>>(grad_counts, static_cast<const long long*>(counts),
                                                           static_cast<const long long*>(counts_cutoff), inst,
                                                           grad_ion_energy, n_cells, grad_power, vp);
    else
        emax_backward_kernel<<<L.n_instances, 256, 0, s>>>(grad_counts, static_cast<const int*>(counts),
                                                           static_cast<const int*>(counts_cutoff), inst,
                                                           grad_ion_energy, n_cells, grad_power, vp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return adj_fail(SPUT_ERR_CUDA, cudaGetErrorString(e));
    return SPUT_OK;
}

// slope dV/dP of each voltage line (P_a, V_a, P_b, V_b); E_i = e V, so dE_i/dP in eV/W
sput_status voltage_slopes(int n, const double* voltage, double* slope)
{
    if (n < 1 || !voltage) return adj_fail(SPUT_ERR_INVALID_ARG, "NULL voltage lines or no instance");
    for (int j = 0; j < n; ++j) {
        const double* q = voltage + 4 * j;
        if (!(q[2] != q[0]) || !std::isfinite(q[0]) || !std::isfinite(q[1]) || !std::isfinite(q[2]) ||
            !std::isfinite(q[3]))
            return adj_fail(SPUT_ERR_INVALID_ARG, "voltage line needs two finite points at distinct powers");
        slope[j] = (q[3] - q[1]) / (q[2] - q[0]);
    }
    return SPUT_OK;
}

}  // namespace

extern "C" {

sput_status sput_emax_backward(const sput_scene* scene, const double* grad_counts, const void* counts,
                               const void* counts_cutoff, double* grad_ion_energy, void* stream)
{
    sput::NvtxRange nvtx("sput_emax_backward");
    if (!scene || !grad_counts || !counts || !counts_cutoff || !grad_ion_energy)
        return adj_fail(SPUT_ERR_INVALID_ARG, "NULL argument");
    VoltParams vp;
    std::memset(&vp, 0, sizeof vp);
    return emax_backward_launch(scene, grad_counts, counts, counts_cutoff, grad_ion_energy, nullptr, vp, stream);
}

sput_status sput_ion_energy(int n, const double* voltage, const double* power, double* ion_energy)
{
    if (!power || !ion_energy) return adj_fail(SPUT_ERR_INVALID_ARG, "NULL argument");
    if (n > 4096) return adj_fail(SPUT_ERR_INVALID_ARG, "at most 4096 lines");
    for (int j = 0; j < n; ++j) {
        double slope;
        sput_status st = voltage_slopes(1, voltage + 4 * j, &slope);
        if (st != SPUT_OK) return st;
        if (!std::isfinite(power[j])) return adj_fail(SPUT_ERR_INVALID_ARG, "power must be finite");
        const double* q = voltage + 4 * j;
        ion_energy[j] = q[1] + slope * (power[j] - q[0]);  // singly charged ions: eV = e * volts
    }
    return n >= 1 ? SPUT_OK : adj_fail(SPUT_ERR_INVALID_ARG, "no voltage line");
}

sput_status sput_voltage_backward(const sput_scene* scene, const double* voltage, const double* grad_counts,
                                  const void* counts, const void* counts_cutoff, double* grad_ion_energy,
                                  double* grad_power, void* stream)
{
    sput::NvtxRange nvtx("sput_voltage_backward");
    if (!scene || !grad_counts || !counts || !counts_cutoff || !grad_ion_energy || !grad_power)
        return adj_fail(SPUT_ERR_INVALID_ARG, "NULL argument");
    sput_tally_layout L;
    sput_status st = sput_tally_layout_get(scene, &L);
    if (st != SPUT_OK) return st;
    if (L.n_instances > kMaxCath) return adj_fail(SPUT_ERR_INVALID_ARG, "the voltage path supports at most 16 instances");
    VoltParams vp;
    std::memset(&vp, 0, sizeof vp);
    st = voltage_slopes(L.n_instances, voltage, vp.dEdP);
    if (st != SPUT_OK) return st;
    return emax_backward_launch(scene, grad_counts, counts, counts_cutoff, grad_ion_energy, grad_power, vp, stream);
}

sput_status sput_composition(int n_cathodes, int n_cells, int n_points, const int64_t* counts, const int32_t* patch_of_cell,
                             int ref_point, const double* calibration, const double* power, double* patch_counts,
                             double* composition, void* stream)
{
    CompParams cp;
    sput_status st = comp_params(n_cathodes, n_cells, n_points, ref_point, calibration, power, cp);
    if (st != SPUT_OK) return st;
    if (!counts || !patch_of_cell || !patch_counts || !composition) return adj_fail(SPUT_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(patch_counts, 0, sizeof(double) * (size_t)n_cathodes * n_points, s);
    if (e != cudaSuccess) return adj_fail(SPUT_ERR_CUDA, cudaGetErrorString(e));
    patch_sum_kernel<<<304, 256, 0, s>>>(reinterpret_cast<const long long*>(counts), patch_of_cell, patch_counts,
                                         n_cathodes, n_cells, n_points);
    composition_kernel<<<(n_points + 127) / 128, 128, 0, s>>>(patch_counts, composition, cp);
    e = cudaGetLastError();
    if (e != cudaSuccess) return adj_fail(SPUT_ERR_CUDA, cudaGetErrorString(e));
    return SPUT_OK;
}

sput_status sput_composition_backward(int n_cathodes, int n_cells, int n_points, const double* patch_counts,
                                      const int32_t* patch_of_cell, int ref_point, const double* calibration,
                                      const double* power, const double* grad_composition, double* grad_patch,
                                      double* grad_counts, double* grad_power, void* stream)
{
    sput::NvtxRange nvtx("sput_composition_backward");
    CompParams cp;
    sput_status st = comp_params(n_cathodes, n_cells, n_points, ref_point, calibration, power, cp);
    if (st != SPUT_OK) return st;
    if (!patch_counts || !patch_of_cell || !grad_composition || !grad_patch || !grad_counts || !grad_power)
        return adj_fail(SPUT_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    composition_backward_kernel<<<1, 512, 0, s>>>(patch_counts, grad_composition, grad_patch, grad_power, cp);
    scatter_kernel<<<304, 256, 0, s>>>(grad_patch, patch_of_cell, grad_counts, n_cathodes, n_cells, n_points);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return adj_fail(SPUT_ERR_CUDA, cudaGetErrorString(e));
    return SPUT_OK;
}

}  // extern "C"
