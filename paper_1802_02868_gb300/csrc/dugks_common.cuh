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
    double xc;        // cell-centre coordinate (the low face of the axis at 0)
};
static_assert(sizeof(AxisRec) == 128, "AxisRec layout");

// Storage of the order parameter phi.  FP64 mode: a double.  FP32 mode: an
// unevaluated pair of floats (hi + lo, |lo| <= ulp(hi)/2), so that the
// differences that feed lap(phi) and grad(phi), and the conservative update of
// phi, keep about 48 bits without a single FP64 instruction in the kernels.
template <typename T>
struct PhiS;
template <>
struct PhiS<double> { using type = double; };
template <>
struct PhiS<float> { using type = float2; };
template <typename T>
using phi_t = typename PhiS<T>::type;

__device__ __forceinline__ double phi_val(double v) { return v; }
__device__ __forceinline__ float phi_val(float2 v) { return v.x + v.y; }
// a - b
__device__ __forceinline__ double phi_sub(double a, double b) { return a - b; }
__device__ __forceinline__ float phi_sub(float2 a, float2 b) { return (a.x - b.x) + (a.y - b.y); }
// a + d: exact two-sum of the high parts, error folded into the low part
__device__ __forceinline__ double phi_add(double a, double d) { return a + d; }
__device__ __forceinline__ float2 phi_add(float2 a, float d)
{
    const float s = a.x + d;
    const float bb = s - a.x;
    const float e = (a.x - (s - bb)) + (d - bb);
    const float lo = a.y + e;
    const float hi = s + lo;
    return make_float2(hi, lo - (hi - s));
}
__device__ __forceinline__ void phi_from_zero(double &v) { v = 0.0; }
__device__ __forceinline__ void phi_from_zero(float2 &v) { v = make_float2(0.f, 0.f); }
__device__ __forceinline__ double phi_to_double(double v) { return v; }
__device__ __forceinline__ double phi_to_double(float2 v) { return (double)v.x + (double)v.y; }
__device__ __forceinline__ void phi_from_double(double d, double &out) { out = d; }
__device__ __forceinline__ void phi_from_double(double d, float2 &out)
{
    const float hi = (float)d;
    out = make_float2(hi, (float)(d - (double)hi));
}

// Model parameters of one instance in the arithmetic type T (precomputed on
// the host so that FP32 kernels execute no conversion from FP64).
template <typename T>
struct ParT {
    T phiA, phiB, rhoA, rhoB, muA, muB, lambda, tau_g, beta, kappa, gxa, gya, rho_ref;
    T dt, h, eta, gamma, drho;
    // relaxation weights: with K = muA muB (phiA - phiB), h muA, h muB and the
    // numerators 6K, 3Kh, 9Kh of the f weights; the g weights of a cell
    // (2 tau_g - h, 3h, 3 tau_g h over 2 tau_g + dt)
    T hmuA, hmuB, k6, k3h, k9h;
    T gca, gcb, gcc;
};

// A constant of the phi storage: the double and its float pair (hi, lo).
struct PhiC {
    double d;
    float hi, lo;
};
__device__ __forceinline__ double phi_subc(double a, const PhiC &c) { return a - c.d; }
__device__ __forceinline__ float phi_subc(float2 a, const PhiC &c) { return (a.x - c.hi) + (a.y - c.lo); }
// a - t for a value t of the arithmetic type
__device__ __forceinline__ double phi_subt(double a, double t) { return a - t; }
__device__ __forceinline__ float phi_subt(float2 a, float t) { return (a.x - t) + a.y; }

// Geometry record of one axis position in the arithmetic type T (same fields
// as AxisRec).
template <typename T>
struct AxisRecT {
    T d, c1m, c10, c1p, c2m, c20, c2p, e1m, e10, e1p, wL, wR, invd;
    int km, kp, lo_wall, hi_wall;
    T xc;
    T d_lo;   // d - (T)d of the FP64 width: d + d_lo is the width to about 48 bits in FP32
};

// A pair (f, g) of values of the two distribution kinds.  In FP32 the pair
// arithmetic maps to the packed two-lane instructions of sm_100+ (one issue
// for two FP32 FMAs), which the fused step uses wherever f and g undergo the
// same operation; in FP64 it is two scalar operations.
template <typename T>
struct PairS;
template <>
struct PairS<float> { using type = float2; };
template <>
struct PairS<double> { using type = double2; };
template <typename T>
using pair_t = typename PairS<T>::type;

__device__ __forceinline__ float2 pr(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 pr(double a, double b) { return make_double2(a, b); }
__device__ __forceinline__ float2 pr(float a) { return make_float2(a, a); }
__device__ __forceinline__ double2 pr(double a) { return make_double2(a, a); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ double2 pfma(double2 a, double2 b, double2 c)
{
    return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ double2 pmul(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ double2 padd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
// a - b
__device__ __forceinline__ float2 psub(float2 a, float2 b) { return __ffma2_rn(make_float2(-1.f, -1.f), b, a); }
__device__ __forceinline__ double2 psub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

// Per-instance constants.
struct InstDev {
    int nx, ny, nxp, bcx, bcy;
    int uni;           // uniform spacing on both axes, both periodic
    long long cell0;   // first cell of the instance in the batch cell space
    long long gx_off;  // index of the x-axis records in the geometry table
    long long gy_off;
    int tile0, ntiles; // tile range of the instance in the tile table
    // model parameters
    double phiA, phiB, rhoA, rhoB, muA, muB, lambda, tau_g, beta, kappa, gxa, gya, rho_ref;
    // derived: dt (Eq. cfl), h = dt/2, eta (Eq. kineticandmobility), gamma (Eq. Gama),
    // drho = d rho / d phi (Eq. oderrho)
    double dt, h, eta, gamma, drho;
    double vol;        // total volume (sum dx)(sum dy)
    // phiA, phiB and (phiA + phiB)/2 as constants of the phi storage
    PhiC cA, cB, cM;
    ParT<double> pd;
    ParT<float> pf;
};

template <typename T>
__device__ __forceinline__ const ParT<T> &par(const InstDev &I);
template <>
__device__ __forceinline__ const ParT<double> &par<double>(const InstDev &I) { return I.pd; }
template <>
__device__ __forceinline__ const ParT<float> &par<float>(const InstDev &I) { return I.pf; }

// All device planes of a simulation.  Distribution planes are [Q][N], the
// rest [N], N = total padded cells of all instances.
template <typename T>
struct Planes {
    T *f, *g;      // tracked tilde distributions
    T *fbp, *gbp;  // bar-plus at cell centres (step 2)
    // phi is FP64 in both precisions: in FP32 mode it is the authoritative
    // order parameter, advanced by the conservative flux form of the update
    phi_t<T> *phi;
    T *mu, *lapmu, *gmux, *gmuy, *gphix, *gphiy, *p, *ux, *uy, *gpx, *gpy, *rho;
    long long N;
    int *status;   // per instance, bit 0 = non-finite seen
};

constexpr int TX = 32;
constexpr int TY = 8;

// Per-instance status bits: set by the kernels when a non-finite value
// appears (the instance is masked from then on), and by the host to hold an
// instance still while the rest of a batch steps.
constexpr int ST_NONFINITE = 1;
constexpr int ST_PAUSED = 2;

enum KernelId { K_MU = 0, K_MACRO = 1, K_CELL = 2, K_FACE = 3, K_INIT = 4, K_REDUCE = 5, K_STEP = 6, K_DIAG = 7, K_COUNT = 8 };

}  // namespace dugks
