// dugks_diag.cuh -- on-device diagnostics of a state.
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
// k_diag_f forms per-strip partial sums and extremes in one pass over the
// state; k_diag_inst adds the strips of each instance in strip order, so the
// result does not depend on timing.
#pragma once
#include "dugks_fused.cuh"
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

// Arithmetic in the sim's precision T: FP32 sims sum each strip in FP32 (the
// FP64 pipe of GB300 runs at 1/64 of the FP32 rate) and the strips of an
// instance in FP64; the crossing heights are placed and compared in FP64.
// The sums of each tile of a strip of up to SB tiles (32 columns, 8 SB rows)
// in one pass over the state.  A block stages phi of the strip and a
// two-cell ring and the geometry of its columns and rows in shared memory,
// computes mu on the strip and a one-cell ring (Eq. chemicalpotential), then
// walks the strip's tiles: for each cell grad mu, lap mu, grad phi, F, u and
// p (Eqs. u, P) as k_mu and k_macro form them (in FP32 with the fast
// division), the Laplace pressure and the region sums, with the next tile's
// tilde f already in flight.  Each thread accumulates its cells' terms over
// the strip in T; the block reduces them once (warp shuffles, then the warps
// in order) into one partial per strip, at the strip's index, and
// k_diag_inst adds an instance's strips in order.  Writes nothing else (and
// P if asked).
constexpr int DIAG_SB = 8;
template <typename T>
__global__ void __launch_bounds__(TX *TY, sizeof(T) == sizeof(float) ? 4 : 2) k_diag_f(const InstDev *__restrict__ insts, const int4 *__restrict__ strips,
                                                   const AxisRecT<T> *__restrict__ geoT, const AxisRec *__restrict__ geo,
                                                   Planes<T> P, DiagPart *parts, double *p_dense,
                                                   const long long *__restrict__ dense0)
{
    constexpr int SB = DIAG_SB, W2 = TX + 4, H2 = SB * TY + 4, W1 = TX + 2, H1 = SB * TY + 2, NE = W2 + H2;
    __shared__ phi_t<T> sphi[H2 * W2];          // columns -2..TX+1, rows -2..SB TY+1
    __shared__ T smu[H1 * W1];                  // columns -1..TX, rows -1..SB TY
    // geometry of the region's columns (entries 0..W2-1) and rows (W2..NE-1):
    // c1m, c1p, c10, c2m, c2p, c20, d, xc, and the neighbour steps (0 at a wall ghost)
    __shared__ T sgeo[8][NE];
    __shared__ signed char smo[NE], spo[NE];
    __shared__ double syc[H2];                  // FP64 row centres, for the crossing heights
    __shared__ T red[TX * TY / 32][DIAG_SUMS];
    __shared__ unsigned long long s_front, s_tip;
    __shared__ int s_ncross;
    // the instance's parameters and phase constants, read by every cell: one
    // shared copy instead of a global load per use
    __shared__ ParT<T> sPr;
    __shared__ PhiC sC[3];
    const int4 st = strips[blockIdx.x];
    const InstDev &I = insts[st.x];
    const ParT<T> &Pr = sPr;   // filled before the first barrier
    const int i0 = st.y, j0 = st.z, nb = st.w;
    const int tid = threadIdx.y * TX + threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool live = !(P.status[st.x] & ST_NONFINITE);
    const long long N = P.N;
    const int rows = nb * TY;
    auto i2 = [](int x, int y) { return (y + 2) * W2 + (x + 2); };
    auto i1 = [](int x, int y) { return (y + 1) * W1 + (x + 1); };
    auto wrap = [&](bool isx, int g) -> int {
        const int n = isx ? I.nx : I.ny;
        if ((isx ? I.bcx : I.bcy) == 0) {
            while (g < 0) g += n;
            while (g >= n) g -= n;
            return g;
        }
        return (g < 0 || g >= n) ? -1 : g;
    };
    if (tid == 0) {
        s_front = 0ull;
        s_tip = 0x7ff0000000000000ull;   // +inf
        s_ncross = 0;
        sC[0] = I.cA;
        sC[1] = I.cB;
        sC[2] = I.cM;
    }
    static_assert(sizeof(ParT<T>) % sizeof(T) == 0 && sizeof(ParT<T>) / sizeof(T) <= TX * TY, "parameter copy");
    if (tid < (int)(sizeof(ParT<T>) / sizeof(T))) ((T *)&sPr)[tid] = ((const T *)&par<T>(I))[tid];
    const int x = threadIdx.x, y = threadIdx.y;
    const int i = i0 + x;
    // tilde f of the thread's cell in tile rb
    T fv[Q];
    auto load_f = [&](int rb) {
        const int j = j0 + rb * TY + y;
        if (live && i < I.nx && j < I.ny) {
            const long long c = cell_of(I, i, j);
#pragma unroll
            for (int q = 0; q < Q; q++) fv[q] = P.f[q * N + c];
        }
    };
    load_f(0);
    if (live) {
        // the phi region in asynchronous copies, in flight while the geometry is staged
        for (int r = tid; r < W2 * (rows + 4); r += TX * TY) {
            const int gi = wrap(true, i0 + r % W2 - 2), gj = wrap(false, j0 + r / W2 - 2);
            if (gi >= 0 && gj >= 0) {
                cp_async<sizeof(phi_t<T>)>(sphi + r, P.phi + cell_of(I, gi, gj));
            } else {
                phi_t<T> v;
                phi_from_zero(v);
                sphi[r] = v;
            }
        }
        cp_commit();
        for (int e = tid; e < W2 + rows + 4; e += TX * TY) {
            const bool isx = e < W2;
            const int g = wrap(isx, isx ? i0 + e - 2 : j0 + (e - W2) - 2);
            T v[8] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
            int m = 0, pp = 0;
            if (g >= 0) {
                const AxisRecT<T> &R = geoT[(isx ? I.gx_off : I.gy_off) + g];
                v[0] = R.c1m; v[1] = R.c1p; v[2] = R.c10; v[3] = R.c2m; v[4] = R.c2p; v[5] = R.c20; v[6] = R.d; v[7] = R.xc;
                m = R.km == g ? 0 : -1;
                pp = R.kp == g ? 0 : 1;
                if (!isx) syc[e - W2] = geo[I.gy_off + g].xc;
            }
#pragma unroll
            for (int k = 0; k < 8; k++) sgeo[k][e] = v[k];
            smo[e] = (signed char)m;
            spo[e] = (signed char)pp;
        }
        cp_wait<0>();
    }
    __syncthreads();
    // geometry accessors: column x (entry x + 2), row y (entry W2 + y + 2)
    auto gx = [&](int k, int xx) { return sgeo[k][xx + 2]; };
    auto gy = [&](int k, int yy) { return sgeo[k][W2 + yy + 2]; };
    if (live) {
        // mu on the strip and a one-cell ring (k_mu)
        for (int r = tid; r < W1 * (rows + 2); r += TX * TY) {
            const int xx = r % W1 - 1, yy = r / W1 - 1;
            T mu = 0;
            if (gx(6, xx) != T(0) && gy(6, yy) != T(0)) {   // a cell of the domain
                const phi_t<T> p0 = sphi[i2(xx, yy)];
                const T lap = (gx(3, xx) * phi_sub(sphi[i2(xx + smo[xx + 2], yy)], p0) + gx(4, xx) * phi_sub(sphi[i2(xx + spo[xx + 2], yy)], p0))
                            + (gy(3, yy) * phi_sub(sphi[i2(xx, yy + smo[W2 + yy + 2])], p0) + gy(4, yy) * phi_sub(sphi[i2(xx, yy + spo[W2 + yy + 2])], p0));
                const T dpsi = T(4) * Pr.beta * phi_subc(p0, sC[0]) * phi_subc(p0, sC[1]) * phi_subc(p0, sC[2]);
                mu = dpsi - Pr.kappa * lap;
            }
            smu[r] = mu;
        }
    }
    __syncthreads();
    T v[DIAG_SUMS];   // the thread's sums over its cells of the strip
#pragma unroll
    for (int k = 0; k < DIAG_SUMS; k++) v[k] = T(0);
    for (int rb = 0; rb < nb; rb++) {
        T cur[Q];
#pragma unroll
        for (int q = 0; q < Q; q++) cur[q] = fv[q];
        if (rb + 1 < nb) load_f(rb + 1);   // the next tile's tilde f is in flight while this tile runs
        const int yr = rb * TY + y, j = j0 + yr;
        if (live && i < I.nx && j < I.ny) {
            const T cs2 = Cst<T>::cs2;
            const int xm = x + smo[x + 2], xp = x + spo[x + 2], ym = yr + smo[W2 + yr + 2], yp = yr + spo[W2 + yr + 2];
            // the macros of k_macro
            const phi_t<T> p0 = sphi[i2(x, yr)];
            const T phi = T(phi_val(p0)), mu = smu[i1(x, yr)];
            const T gmx = gx(0, x) * smu[i1(xm, yr)] + gx(2, x) * mu + gx(1, x) * smu[i1(xp, yr)];
            const T gmy = gy(0, yr) * smu[i1(x, ym)] + gy(2, yr) * mu + gy(1, yr) * smu[i1(x, yp)];
            const T fxm = phi_sub(sphi[i2(xm, yr)], p0), fxp = phi_sub(sphi[i2(xp, yr)], p0);
            const T fym = phi_sub(sphi[i2(x, ym)], p0), fyp = phi_sub(sphi[i2(x, yp)], p0);
            const T gfx = gx(0, x) * fxm + gx(1, x) * fxp;
            const T gfy = gy(0, yr) * fym + gy(1, yr) * fyp;
            const T lmu = (gx(3, x) * smu[i1(xm, yr)] + gx(5, x) * mu + gx(4, x) * smu[i1(xp, yr)])
                        + (gy(3, yr) * smu[i1(x, ym)] + gy(5, yr) * mu + gy(4, yr) * smu[i1(x, yp)]);
            const T rho = Pr.rhoB + Pr.drho * (phi - Pr.phiB);   // Eq. (oderrho), as rho_of forms it
            const T Fx = -phi * gmx + (rho - Pr.rho_ref) * Pr.gxa;
            const T Fy = -phi * gmy + (rho - Pr.rho_ref) * Pr.gya;
            T sf = 0, mx = 0, my = 0;
#pragma unroll
            for (int q = 0; q < Q; q++) {
                sf += cur[q];
                if (cx(q)) mx += T(cx(q)) * cur[q];
                if (cy(q)) my += T(cy(q)) * cur[q];
            }
            const T hdt = T(0.5) * Pr.dt;
            const T ux = fdiv(mx + hdt * cs2 * Fx, cs2 * rho);
            const T uy = fdiv(my + hdt * cs2 * Fy, cs2 * rho);
            const T grx = Pr.drho * gfx, gry = Pr.drho * gfy;
            const T pv = sf + hdt * cs2 * (ux * grx + uy * gry - Pr.gamma * rho * Pr.lambda * lmu);
            // the Laplace pressure (the gradients of phi are those of k_macro) and the region sums
            const T lap = (gx(3, x) * fxm + gx(4, x) * fxp) + (gy(3, yr) * fym + gy(4, yr) * fyp);
            const T a = phi - Pr.phiA, b = phi - Pr.phiB;
            const T psi = Pr.beta * a * a * b * b;
            const T dpsi = T(2) * Pr.beta * a * b * (a + b);
            const T Pv = (phi * dpsi - psi) - Pr.kappa * phi * lap + T(0.5) * Pr.kappa * (gfx * gfx + gfy * gfy) + pv;
            if (p_dense) p_dense[dense0[st.x] + (long long)j * I.nx + i] = (double)Pv;
            const T vol = gx(6, x) * gy(6, yr);
            const T inv = fdiv(T(1), Pr.phiA - Pr.phiB);
            const T cn = b * inv;
            if (cn > T(0.5)) {
                v[0] += vol;
                v[1] += vol * gx(7, x);
                v[2] += vol * gy(7, yr);
                v[3] += vol * ux;
                v[4] += vol * uy;
            }
            if (cn > T(0.9)) { v[5] += vol * Pv; v[6] += vol; }
            if (cn < T(0.1)) { v[7] += vol * Pv; v[8] += vol; }
            if (j + 1 < I.ny && cn < T(0.5)) {
                const T c1 = (T(phi_val(sphi[i2(x, yr + 1)])) - Pr.phiB) * inv;
                if (c1 >= T(0.5)) {
                    const double y0 = syc[yr + 2], y1 = syc[yr + 3];
                    const double yy = y0 + (double)((T(0.5) - cn) / (c1 - cn)) * (y1 - y0);
                    const unsigned long long bits = (unsigned long long)__double_as_longlong(yy);
                    atomicMax(&s_front, bits);
                    atomicMin(&s_tip, bits);
                    atomicAdd(&s_ncross, 1);
                }
            }
        }
    }
    // fixed-order reduction of the strip in T: warp shuffles, then the warps
    // in order, and one conversion per strip (a warp-wide FP64 instruction
    // occupies GB300's FP64 pipe for 16 cycles even with one lane active)
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

// One block per instance: its strips' partials in strip order (a strided
// pass per thread, then the threads in order), then the quotients.  srng[k]
// = (first strip, number of strips) of instance k.
constexpr int DIAG_INST_THREADS = 128;
__global__ void __launch_bounds__(DIAG_INST_THREADS) k_diag_inst(const int2 *__restrict__ srng, const int *status,
                                                                 const DiagPart *__restrict__ parts, DiagOut *out)
{
    __shared__ DiagPart red[DIAG_INST_THREADS];
    const int2 R = srng[blockIdx.x];
    DiagPart a;
    for (int k = 0; k < DIAG_SUMS; k++) a.s[k] = 0.0;
    a.front = -INFINITY;
    a.tip = INFINITY;
    for (int t = R.x + threadIdx.x; t < R.x + R.y; t += DIAG_INST_THREADS) {
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
