// dugks_diag.cuh -- on-device diagnostics of a state, in FP64.
//
//   Laplace pressure (Sec. 3.1, Laplace's law):
//       P = p0 - kappa phi lap(phi) + kappa |grad phi|^2 / 2 + p,
//       p0 = phi psi'(phi) - psi(phi),  psi = beta (phi - phiA)^2 (phi - phiB)^2
//   with the cell stencils of Eqs. (nonphi), (nonphi2) and mirror ghosts at
//   walls; p, u from the macro kernels (Eqs. u, P).
//   Region A: cells with c = (phi - phiB)/(phiA - phiB) > 1/2.  Its volume is
//   the droplet mass of Table A1; its centroid and mean velocity follow the
//   rising bubble (Sec. 3.3).  Bulk pressures: volume means of P over c > 0.9
//   and c < 0.1 (their difference is the Laplace jump).
//   Front and tip (Sec. 3.4): each pair of vertically adjacent cells with
//   c < 1/2 below and c >= 1/2 above holds a crossing of the median level,
//   placed by linear interpolation between the centres; the highest and the
//   lowest crossing (pairs across a periodic y boundary do not count).
//
// k_diag forms per-tile partial sums and extremes; k_diag_inst adds the tiles
// of each instance in tile order, so the result does not depend on timing.
#pragma once
#include "dugks_kernels.cuh"

namespace dugks {

constexpr int DIAG_SUMS = 9;   // V_A, sum x, sum y, sum ux, sum uy (over A); sum P, V over bulk A; sum P, V over bulk B
struct DiagPart {
    double s[DIAG_SUMS];
    double front, tip;
};
// result of one instance, field for field the public dugks_diag
struct DiagOut {
    double mass, xc, yc, ux, uy, p_bulk_A, p_bulk_B, front_y, tip_y;
};

__device__ __forceinline__ double diag_nan() { return __longlong_as_double(0x7ff8000000000000LL); }

// Arithmetic in the sim's precision T: FP32 sims sum each tile in FP32 (the
// FP64 pipe of GB300 runs at 1/64 of the FP32 rate) and the tiles of an
// instance in FP64; the crossing heights are placed and compared in FP64.
template <typename T>
__global__ void __launch_bounds__(TX *TY) k_diag(const InstDev *__restrict__ insts, const int4 *__restrict__ tiles,
                                                 const AxisRecT<T> *__restrict__ geoT, const AxisRec *__restrict__ geo,
                                                 Planes<T> P, DiagPart *parts, double *p_dense,
                                                 const long long *__restrict__ dense0)
{
    __shared__ T red[TX * TY / 32][DIAG_SUMS];
    __shared__ unsigned long long s_front, s_tip;   // bit patterns of positive doubles order as integers
    __shared__ int s_ncross;
    const int4 t = tiles[blockIdx.x];
    const InstDev &I = insts[t.x];
    const ParT<T> &Pr = par<T>(I);
    const int i = t.y + threadIdx.x, j = t.z + threadIdx.y;
    const int tid = threadIdx.y * TX + threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        s_front = 0ull;
        s_tip = 0x7ff0000000000000ull;   // +inf
        s_ncross = 0;
    }
    __syncthreads();
    T v[DIAG_SUMS];
#pragma unroll
    for (int k = 0; k < DIAG_SUMS; k++) v[k] = T(0);
    if (!(P.status[t.x] & ST_NONFINITE) && i < I.nx && j < I.ny) {
        const AxisRecT<T> &ax = geoT[I.gx_off + i];
        const AxisRecT<T> &ay = geoT[I.gy_off + j];
        const long long c = cell_of(I, i, j);
        const phi_t<T> p0 = P.phi[c];
        const T fxm = phi_sub(P.phi[cell_of(I, ax.km, j)], p0), fxp = phi_sub(P.phi[cell_of(I, ax.kp, j)], p0);
        const T fym = phi_sub(P.phi[cell_of(I, i, ay.km)], p0), fyp = phi_sub(P.phi[cell_of(I, i, ay.kp)], p0);
        const T gx = ax.c1m * fxm + ax.c1p * fxp;
        const T gy = ay.c1m * fym + ay.c1p * fyp;
        const T lap = (ax.c2m * fxm + ax.c2p * fxp) + (ay.c2m * fym + ay.c2p * fyp);
        const T f0 = T(phi_val(p0));
        const T a = f0 - Pr.phiA, b = f0 - Pr.phiB;
        const T psi = Pr.beta * a * a * b * b;
        const T dpsi = T(2) * Pr.beta * a * b * (a + b);
        const T Pv = (f0 * dpsi - psi) - Pr.kappa * f0 * lap + T(0.5) * Pr.kappa * (gx * gx + gy * gy) + P.p[c];
        if (p_dense) p_dense[dense0[t.x] + (long long)j * I.nx + i] = (double)Pv;
        const T vol = ax.d * ay.d;
        const T inv = T(1) / (Pr.phiA - Pr.phiB);
        const T cn = b * inv;
        if (cn > T(0.5)) {
            v[0] = vol;
            v[1] = vol * ax.xc;
            v[2] = vol * ay.xc;
            v[3] = vol * P.ux[c];
            v[4] = vol * P.uy[c];
        }
        if (cn > T(0.9)) { v[5] = vol * Pv; v[6] = vol; }
        if (cn < T(0.1)) { v[7] = vol * Pv; v[8] = vol; }
        if (j + 1 < I.ny && cn < T(0.5)) {
            const T c1 = (T(phi_val(P.phi[cell_of(I, i, j + 1)])) - Pr.phiB) * inv;
            if (c1 >= T(0.5)) {
                const double y0 = geo[I.gy_off + j].xc, y1 = geo[I.gy_off + j + 1].xc;
                const double y = y0 + (double)((T(0.5) - cn) / (c1 - cn)) * (y1 - y0);
                const unsigned long long bits = (unsigned long long)__double_as_longlong(y);
                atomicMax(&s_front, bits);
                atomicMin(&s_tip, bits);
                atomicAdd(&s_ncross, 1);
            }
        }
    }
    // fixed-order reduction in T: warp shuffles, then the warps in order, and
    // one conversion per tile (a warp-wide FP64 instruction occupies GB300's
    // FP64 pipe for 16 cycles even with one lane active)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int k = 0; k < DIAG_SUMS; k++) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    }
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < DIAG_SUMS; k++) red[warp][k] = v[k];
    }
    __syncthreads();
    if (tid == 0) {
        DiagPart out;
        for (int k = 0; k < DIAG_SUMS; k++) {
            T a = red[0][k];
            for (int w = 1; w < TX * TY / 32; w++) a += red[w][k];
            out.s[k] = (double)a;
        }
        out.front = s_ncross ? __longlong_as_double((long long)s_front) : -INFINITY;
        out.tip = s_ncross ? __longlong_as_double((long long)s_tip) : INFINITY;
        parts[blockIdx.x] = out;
    }
}

// One block per instance: its tiles' partials in tile order (a strided pass
// per thread, then the threads in order), then the quotients.
constexpr int DIAG_INST_THREADS = 128;
__global__ void __launch_bounds__(DIAG_INST_THREADS) k_diag_inst(const InstDev *__restrict__ insts, const int *status,
                                                                 const DiagPart *__restrict__ parts, DiagOut *out)
{
    __shared__ DiagPart red[DIAG_INST_THREADS];
    const InstDev &I = insts[blockIdx.x];
    DiagPart a;
    for (int k = 0; k < DIAG_SUMS; k++) a.s[k] = 0.0;
    a.front = -INFINITY;
    a.tip = INFINITY;
    for (int t = I.tile0 + threadIdx.x; t < I.tile0 + I.ntiles; t += DIAG_INST_THREADS) {
        const DiagPart &p = parts[t];
        for (int k = 0; k < DIAG_SUMS; k++) a.s[k] += p.s[k];
        a.front = fmax(a.front, p.front);
        a.tip = fmin(a.tip, p.tip);
    }
    red[threadIdx.x] = a;
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int w = 1; w < DIAG_INST_THREADS; w++) {
        for (int k = 0; k < DIAG_SUMS; k++) a.s[k] += red[w].s[k];
        a.front = fmax(a.front, red[w].front);
        a.tip = fmin(a.tip, red[w].tip);
    }
    const double nan = diag_nan();
    DiagOut o;
    if (status[blockIdx.x] & ST_NONFINITE) {
        o.mass = o.xc = o.yc = o.ux = o.uy = o.p_bulk_A = o.p_bulk_B = o.front_y = o.tip_y = nan;
    } else {
        const double m = a.s[0];
        o.mass = m;
        o.xc = m > 0 ? a.s[1] / m : nan;
        o.yc = m > 0 ? a.s[2] / m : nan;
        o.ux = m > 0 ? a.s[3] / m : nan;
        o.uy = m > 0 ? a.s[4] / m : nan;
        o.p_bulk_A = a.s[6] > 0 ? a.s[5] / a.s[6] : nan;
        o.p_bulk_B = a.s[8] > 0 ? a.s[7] / a.s[8] : nan;
        o.front_y = a.front > -INFINITY ? a.front : nan;
        o.tip_y = a.tip < INFINITY ? a.tip : nan;
    }
    out[blockIdx.x] = o;
}

}  // namespace dugks
