// dugks_common.cuh -- device-side types and lattice constants of the two-phase
// DUGKS library (Zhang, Yang & Guo, arXiv:1802.02868, Sec. 2.2).
#pragma once
#include <cstdint>

namespace dugks {

constexpr int Q = 9;

// D2Q9 velocities, Eq. (D2Q9) with c = 1: rest, four axis, four diagonal.
__host__ __device__ constexpr int cx(int q) { return (q == 1 || q == 5 || q == 8) ? 1 : ((q == 3 || q == 6 || q == 7) ? -1 : 0); }
__host__ __device__ constexpr int cy(int q) { return (q == 2 || q == 5 || q == 6) ? 1 : ((q == 4 || q == 7 || q == 8) ? -1 : 0); }
__host__ __device__ constexpr int opp(int q) { return q == 0 ? 0 : (q <= 4 ? ((q + 1) % 4) + 1 : ((q - 3) % 4) + 5); }
// Weights omega_i (Sec. 2.2, after Eq. Hi).
__host__ __device__ constexpr double wq(int q) { return q == 0 ? 4.0 / 9.0 : (q < 5 ? 1.0 / 9.0 : 1.0 / 36.0); }
// velocity component along axis a
__host__ __device__ constexpr int ca(int q, int a) { return a == 0 ? cx(q) : cy(q); }

static_assert(opp(1) == 3 && opp(2) == 4 && opp(3) == 1 && opp(4) == 2, "opp axis");
static_assert(opp(5) == 7 && opp(6) == 8 && opp(7) == 5 && opp(8) == 6, "opp diag");

// Per-axis geometry record of cell index k along one axis.  Coefficients act
// on (value at km, value at k, value at kp):
//   c1*: first derivative of a macroscopic field, Eq. (nonphi), mirror ghost at walls;
//   c2*: second derivative, Eq. (nonphi2), mirror ghost at walls;
//   e1*: first derivative of a distribution: Eq. (nonphi) between real cells,
//        one-sided two-point difference next to a wall;
//   wL, wR, invd: the face between k and kp ("high face"): distance weights of
//        cell k and cell kp and 1 / (centre distance).
struct AxisRec {
    double d;
    double c1m, c10, c1p;
    double c2m, c20, c2p;
    double e1m, e10, e1p;
    double wL, wR, invd;
    int km, kp;       // neighbour indices (periodic wrap; self for a wall ghost)
    int lo_wall, hi_wall;
    double pad_;
};
static_assert(sizeof(AxisRec) == 128, "AxisRec layout");

// Per-instance constants.
struct InstDev {
    int nx, ny, nxp, bcx, bcy, pad0;
    long long cell0;   // first cell of the instance in the batch cell space
    long long gx_off;  // index of the x-axis records in the geometry table
    long long gy_off;
    int tile0, ntiles; // tile range of the instance in the tile table
    // model parameters
    double phiA, phiB, rhoA, rhoB, muA, muB, lambda, tau_g, beta, kappa, gxa, gya, rho_ref;
    // derived: dt (Eq. cfl), h = dt/2, eta (Eq. kineticandmobility), gamma (Eq. Gama),
    // drho = d rho / d phi (Eq. oderrho)
    double dt, h, eta, gamma, drho;
};

// All device planes of a simulation.  Distribution planes are [Q][N], the
// rest [N], N = total padded cells of all instances.
template <typename T>
struct Planes {
    T *f, *g;      // tracked tilde distributions
    T *fbp, *gbp;  // bar-plus at cell centres (step 2)
    // phi is FP64 in both precisions: in FP32 mode it is the authoritative
    // order parameter, advanced by the conservative flux form of the update
    double *phi;
    T *mu, *lapmu, *gmux, *gmuy, *gphix, *gphiy, *p, *ux, *uy, *gpx, *gpy, *rho;
    long long N;
    int *status;   // per instance, bit 0 = non-finite seen
};

constexpr int TX = 32;
constexpr int TY = 8;

enum KernelId { K_MU = 0, K_MACRO = 1, K_CELL = 2, K_FACE = 3, K_INIT = 4, K_REDUCE = 5, K_COUNT = 6 };

}  // namespace dugks
