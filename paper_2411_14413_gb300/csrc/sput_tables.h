// sput_tables.h -- FP64 host construction of the interaction tables of
// libsput.so (cross section, head-on apsis, collision rate, rejection bound,
// racetrack guesses).  Internal to the library.
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

namespace sput {

// Physical constants (CODATA 2018).
constexpr double kAmuKg = 1.66053906660e-27;
constexpr double kElemCharge = 1.602176634e-19;
constexpr double kBoltzmannJ = 1.380649e-23;
constexpr double kBoltzmannEV = 8.617333262e-5;
constexpr double kBohrA = 0.529177210903;
constexpr double kE2EVA = 14.3996454784;  // e^2/(4 pi eps0), eV*Angstrom
constexpr double kPi = 3.14159265358979323846;
// kinetic energy (eV) of 1 u at 1 km/s
constexpr double kEnergyUnit = kAmuKg * 1.0e6 / kElemCharge;

// b_max / a of the Moliere potential over ln(eps), piecewise cubic on a
// uniform grid; each piece interpolates four exactly root-found values.
struct BmaxTable {
    double chi_min = 0.0;
    double lo = -42.0, h = 0.05;
    int n = 0;                       // pieces
    std::vector<double> third;       // 3n+1 values at lo + h*j/3
    std::vector<float4> cubic;       // per piece c0 + t(c1 + t(c2 + t c3)), t in [0,1]
    std::vector<float> xh;           // head-on apsis at the n+1 nodes
    double eval(double ln_eps) const;  // FP64 evaluation of the same pieces
};

// Cached per chi_min (thread-safe).
const BmaxTable& bmax_table(double chi_min);

// Deflection table (layout constants kChi* in sput_internal.h): node values
// q = ln tan(chi/2) from the FP64 deflection at b = b_max(eps) e^y; slopes in x,
// y and the cross slope from C2 cubic splines through the nodes (end slopes from
// the cubic through the four end nodes); each cell the bicubic Hermite patch of
// its four corners, stored as p(tx, ty) = sum_k tx^k sum_l a[k][l] ty^l,
// tx, ty in [0, 1], row k of the cell in float4 k.
struct ChiTable {
    double chi_min = 0.0;
    std::vector<float4> cells;       // 4 per cell, cell (i, j) at 4 (i kChiNy + j)
    std::vector<double> a64;         // the same coefficients in FP64, 16 per cell
    // FP64 evaluation of the same cells; returns false outside the table
    bool eval(double ln_eps, double ln_s, double& q) const;
};

const ChiTable& chi_table(double chi_min);

// Reduced-unit Moliere scattering: closest approach and CM deflection (FP64).
double head_on_apsis64(double eps);
double apsis64(double eps, double beta);
double chi_moliere64(double eps, double beta);

struct PairPhys {
    double Z1, Z2, m1, m2;
    double a;          // Firsov screening length, Angstrom
    double zze2;       // Z1 Z2 e^2, eV*Angstrom
    double kappa;      // eps = kappa g^2
    int hard_sphere;
    double hs_d;       // Angstrom
    double chi_min;
};

PairPhys make_pair(double Z1, double m1, double Z2, double m2, int hard_sphere, double hs_d, double chi_min);

// sigma(g) in Angstrom^2 (g in km/s)
double sigma64(const PairPhys& pp, const BmaxTable* bt, double g);

// Envelope of the gas-partner rejection at atom speed v: the line A + B rho (rho = |V|/s)
// above H(rho), the largest sigma(g) g over [max(0, v - s rho), v + s rho], on
// [0, kEnvRhoMax], with the least value at rho = kEnvM (the Maxwellian's mean |V|/s):
// the edge of H's upper concave hull that spans kEnvM, from H at kEnvN + 1 equally
// spaced rho, raised by the relative margin kEnvMargin.
void envelope64(const PairPhys& pp, const BmaxTable* bt, double s_gas, double v, double& A, double& B);

// Tables in w = ln(1 + v/s) with pieces of width h_w up to w(v_top):
// K(v) = <sigma(g) g> over the Maxwellian gas (gas at rest: sigma(v) = K(v)/v), the
// envelope coefficients A(v), B(v) and G(v) = d ln K / d ln s.
void build_w_tables(const PairPhys& pp, const BmaxTable* bt, double s_gas, int gas_thermal, double v_top,
                    double h_w, std::vector<float4>& K, std::vector<float4>& EA, std::vector<float4>& EB,
                    std::vector<float4>& G, int& n_w);

// Momentum-transfer cross section sigma_m(g) = 2 pi int_0^inf (1 - cos chi) b db (Angstrom^2)
// and the diffusion cross section sigma_D (Angstrom^2) of the shortcut for thermalised atoms:
// 1/lambda_D = n sigma_D with lambda_D = 3 D_12 / vbar_1, D_12 = 3 kT / (16 n mu Omega11),
// Omega11 = sqrt(kT / (2 pi mu)) int_0^inf exp(-y^2) y^5 sigma_m(y sqrt(2kT/mu)) dy.
double sigma_m64(const PairPhys& pp, const BmaxTable* bt, double g);
double sigma_D64(const PairPhys& pp, const BmaxTable* bt, double T);

// FP64 host values used by tests through the probe entry point.
double K64(const PairPhys& pp, const BmaxTable* bt, double s_gas, int gas_thermal, double v);


// Racetrack inverse CDF: n cubic pieces in sqrt(u), then n in sqrt(1-u), over [0, sqrt(1/2)].
void racetrack_table(double r0, double sigma, double R, int n, float4* out);
double racetrack_F64(double r0, double sigma, double r);

// Cubic through f(0), f(1/3), f(2/3), f(1) on t in [0,1].
float4 cubic_from_thirds(double f0, double f1, double f2, double f3);

}  // namespace sput
