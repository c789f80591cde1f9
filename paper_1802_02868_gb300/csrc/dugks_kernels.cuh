// dugks_kernels.cuh -- CUDA kernels of one two-phase DUGKS step (sm_103a).
//
// One step of the procedure of Sec. 2.2 runs as four launches over a table of
// 32x8-cell tiles that covers every instance of a batch:
//   k_mu    : mu = psi'(phi) - kappa lap(phi)                    (Eq. chemicalpotential)
//   k_macro : grad mu, lap mu, grad phi, F, u, p                  (Eqs. u, P)
//   k_cell  : grad p, tau_f, equilibria, sources, bar-plus        (Eqs. feq, geq, F, G, relations1)
//   k_face  : face reconstruction, face macros, originals, flux,
//             tilde update in place, phi = sum g for the next step (Eqs. fbar_h, original-function,
//                                                                   microfluxf, updatef, relations2)
// plus k_init (step 1) and k_reduce / k_reduce_f32 (FP64 conservation sums).
#pragma once
#include "dugks_common.cuh"

namespace dugks {

template <typename T>
struct Cst {
    static constexpr T cs2 = T(1.0 / 3.0);   // c_s^2 = RT = 1/3
    static constexpr T half = T(0.5);
};

// a / b: IEEE division in FP64 mode; in FP32 mode the fast reciprocal-based
// division (within 2 ulp), used only for 1/rho, the relaxation weights, the
// mixed viscosity and dt/|V|, all well away from overflow.
__device__ __forceinline__ double fdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }
// a * b + c with one rounding
__device__ __forceinline__ double tfma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float tfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }

__device__ __forceinline__ long long cell_of(const InstDev &I, int i, int j)
{
    return I.cell0 + (long long)j * I.nxp + i;
}

template <typename T>
__device__ __forceinline__ T rho_of(const InstDev &I, T phi)
{
    const ParT<T> &Pr = par<T>(I);
    // Eq. (oderrho) written as rhoB + (rhoA - rhoB)(phi - phiB)/(phiA - phiB)
    return Pr.rhoB + Pr.drho * (phi - Pr.phiB);
}

template <typename T>
__device__ __forceinline__ T tauf_of(const InstDev &I, T phi, T rho)
{
    const ParT<T> &Pr = par<T>(I);
    // Eq. (mixvis) and tau_f = nu / c_s^2 with nu = mu / rho (Eq. kineticandmobility)
    T muA = Pr.muA, muB = Pr.muB;
    T mu = fdiv(muA * muB * (Pr.phiA - Pr.phiB), (phi - Pr.phiB) * muB + (Pr.phiA - phi) * muA);
    return fdiv(T(3) * mu, rho);
}

// Weights of the f relaxation with tau_f = 3K/(D rho) (Eq. mixvis and
// Eq. kineticandmobility; K = muA muB (phiA - phiB), D = (phi - phiB) muB +
// (phiA - phi) muA).  At a face (Eq. relations2 with h): 2tau/(2tau + h),
// h/(2tau + h), tau h/(2tau + h), which are 6K, X and 3Kh over 6K + X with
// X = h D rho.  At a cell (Eq. relations1): (2tau - h)/(2tau + dt),
// 3h/(2tau + dt), 3 tau h/(2tau + dt), which are 6K - X, 3X and 9Kh over
// 6K + 2X.  One reciprocal per point.
template <typename T>
__device__ __forceinline__ void face_weights(const ParT<T> &Pr, T phi, T rho, T &a, T &b, T &c)
{
    const T X = ((phi - Pr.phiB) * Pr.hmuB + (Pr.phiA - phi) * Pr.hmuA) * rho;
    const T r = fdiv(T(1), Pr.k6 + X);
    a = Pr.k6 * r;
    b = X * r;
    c = Pr.k3h * r;
}
template <typename T>
__device__ __forceinline__ void cell_weights(const ParT<T> &Pr, T phi, T rho, T &a, T &b, T &c)
{
    const T X = ((phi - Pr.phiB) * Pr.hmuB + (Pr.phiA - phi) * Pr.hmuA) * rho;
    const T r = fdiv(T(1), Pr.k6 + T(2) * X);
    a = (Pr.k6 - X) * r;
    b = T(3) * X * r;
    c = Pr.k9h * r;
}

// Point state from which equilibria and sources follow.
template <typename T>
struct Pt {
    T phi, rho, ux, uy, p, mu, lapmu, Fx, Fy, grx, gry, gpx, gpy, tauf;
};

// Per-point factors shared by the nine directions.  With c_s^2 = 1/3 the
// divisions of Eq. (su) become the exact multipliers 3, 4.5 and 1.5.
template <typename T>
struct PtInv {
    T uu15;    // u.u / (2 c_s^2)
    T prho;    // c_s^2 rho
    T emu;     // eta mu
    T srcF;    // c_s^2 rho gamma lambda lap(mu)
    T fg;      // phi / (c_s^2 rho)
    T Gx, Gy;  // F - grad p
    T cgx, cgy;  // c_s^2 grad rho
    T uF, ucg, uG;  // u.F, u.(c_s^2 grad rho), u.(F - grad p)
};

template <typename T>
__device__ __forceinline__ PtInv<T> pt_inv_p(const ParT<T> &Pr, const Pt<T> &s)
{
    const T cs2 = Cst<T>::cs2;
    PtInv<T> v;
    v.uu15 = T(1.5) * (s.ux * s.ux + s.uy * s.uy);
    v.prho = cs2 * s.rho;
    v.emu = Pr.eta * s.mu;
    v.srcF = cs2 * s.rho * Pr.gamma * Pr.lambda * s.lapmu;
    v.fg = fdiv(T(3) * s.phi, s.rho);
    v.Gx = s.Fx - s.gpx;
    v.Gy = s.Fy - s.gpy;
    v.cgx = cs2 * s.grx;
    v.cgy = cs2 * s.gry;
    v.uF = s.ux * s.Fx + s.uy * s.Fy;
    v.ucg = s.ux * v.cgx + s.uy * v.cgy;
    v.uG = s.ux * v.Gx + s.uy * v.Gy;
    return v;
}

template <typename T>
__device__ __forceinline__ PtInv<T> pt_inv(const InstDev &I, const Pt<T> &s)
{
    return pt_inv_p<T>(par<T>(I), s);
}

// xi_q . (ax, ay) with the zero components of xi_q left out.
template <typename T>
__device__ __forceinline__ T xi_dot(int q, T ax, T ay)
{
    return cx(q) == 0 ? (cy(q) == 0 ? T(0) : T(cy(q)) * ay)
                      : (cy(q) == 0 ? T(cx(q)) * ax : T(cx(q)) * ax + T(cy(q)) * ay);
}

// f^eq, g^eq (Eqs. feq, geq, su, Hi) and F^f, F^g (Eqs. F, G) of direction q
// (index 0) and of its opposite opp(q) (index 1).  With xi_opp = -xi_q the two
// share w, (xi.u)^2 and, up to sign, xi.u, xi.F, xi.(c_s^2 grad rho) and
// xi.(F - grad p); (xi - u).X is formed as xi.X - u.X.  For q = 0 both
// entries are those of the rest direction.
template <typename T>
__device__ __forceinline__ void eq_src2(const Pt<T> &s, const PtInv<T> &v, int q, T (&feq)[2], T (&geq)[2], T (&Ff)[2],
                                        T (&Fg)[2])
{
    const T w = T(wq(q));
    const T xu = xi_dot<T>(q, s.ux, s.uy);
    const T a = tfma(T(4.5 * wq(q)), xu * xu, -(w * v.uu15));   // even part of s_i
    const T b = T(3.0 * wq(q)) * xu;                 // odd part of s_i
    const T xF = xi_dot<T>(q, s.Fx, s.Fy), xc = xi_dot<T>(q, v.cgx, v.cgy), xG = xi_dot<T>(q, v.Gx, v.Gy);
    const T H = (q == 0) ? s.phi - T(1.0 - wq(q)) * v.emu : w * v.emu;
    const T wp = w * s.p, wsrc = w * v.srcF;
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const T si = k == 0 ? a + b : a - b;
        feq[k] = wp + v.prho * si;
        geq[k] = H + s.phi * si;
        const T G = w + si;
        const T eF = (k == 0 ? xF : -xF) - v.uF;
        const T ec = (k == 0 ? xc : -xc) - v.ucg;
        const T eG = (k == 0 ? xG : -xG) - v.uG;
        Ff[k] = tfma(G, eF, tfma(si, ec, -wsrc));
        Fg[k] = v.fg * eG * G;
    }
}

// The same for one direction q; bit for bit the entry that eq_src2 gives for q.
template <typename T>
__device__ __forceinline__ void eq_src(const Pt<T> &s, const PtInv<T> &v, int q, T &feq, T &geq, T &Ff, T &Fg)
{
    const bool base = q == 0 || q == 1 || q == 2 || q == 5 || q == 6;
    T e[2], g[2], f1[2], f2[2];
    eq_src2<T>(s, v, base ? q : opp(q), e, g, f1, f2);
    const int k = base ? 0 : 1;
    feq = e[k];
    geq = g[k];
    Ff = f1[k];
    Fg = f2[k];
}

// compatibility wrapper: equilibria and sources of one direction
template <typename T>
__device__ __forceinline__ void eq_src(const InstDev &I, const Pt<T> &s, int q, T &feq, T &geq, T &Ff, T &Fg)
{
    eq_src<T>(s, pt_inv<T>(I, s), q, feq, geq, Ff, Fg);
}

// ---------------------------------------------------------------------------
// k_mu: chemical potential (Eq. chemicalpotential) with the 5-point Laplacian
// of Eq. (nonphi2) on both axes.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(TX *TY) k_mu(const InstDev *__restrict__ insts, const int4 *__restrict__ tiles,
                                               const AxisRecT<T> *__restrict__ geo, Planes<T> P)
{
    const int4 t = tiles[blockIdx.x];
    const InstDev &I = insts[t.x];
    const ParT<T> &Pr = par<T>(I);
    if (P.status[t.x] & ST_NONFINITE) return;   // masked: non-finite instance of a batch (a paused one still gets its macros)
    const int i = t.y + threadIdx.x, j = t.z + threadIdx.y;
    if (i >= I.nx || j >= I.ny) return;
    const auto &ax = geo[I.gx_off + i];
    const auto &ay = geo[I.gy_off + j];
    const long long c = cell_of(I, i, j);
    // Differences of the stored phi are formed first, so that the Laplacian
    // keeps the precision of the stored phi in FP32 mode (the stencil weights
    // sum to zero: c2m + c20 + c2p = 0).
    const phi_t<T> p0 = P.phi[c];
    T lap = (T(ax.c2m) * phi_sub(P.phi[cell_of(I, ax.km, j)], p0) + T(ax.c2p) * phi_sub(P.phi[cell_of(I, ax.kp, j)], p0))
          + (T(ay.c2m) * phi_sub(P.phi[cell_of(I, i, ay.km)], p0) + T(ay.c2p) * phi_sub(P.phi[cell_of(I, i, ay.kp)], p0));
    T dpsi = T(4) * Pr.beta * phi_subc(p0, I.cA) * phi_subc(p0, I.cB)
           * phi_subc(p0, I.cM);
    P.mu[c] = dpsi - Pr.kappa * lap;
}

// first derivatives of a cell field along x and y (mirror ghosts)
template <typename T, typename R>
__device__ __forceinline__ void grad_field(const InstDev &I, const T *__restrict__ F, const R &ax,
                                           const R &ay, int i, int j, T f0, T &gx, T &gy)
{
    gx = T(ax.c1m) * F[cell_of(I, ax.km, j)] + T(ax.c10) * f0 + T(ax.c1p) * F[cell_of(I, ax.kp, j)];
    gy = T(ay.c1m) * F[cell_of(I, i, ay.km)] + T(ay.c10) * f0 + T(ay.c1p) * F[cell_of(I, i, ay.kp)];
}

// first derivatives of the stored order parameter, difference form (weights sum to zero)
template <typename T, typename R>
__device__ __forceinline__ void grad_phi(const InstDev &I, const phi_t<T> *__restrict__ F, const R &ax,
                                         const R &ay, int i, int j, phi_t<T> f0, T &gx, T &gy)
{
    gx = T(ax.c1m) * phi_sub(F[cell_of(I, ax.km, j)], f0) + T(ax.c1p) * phi_sub(F[cell_of(I, ax.kp, j)], f0);
    gy = T(ay.c1m) * phi_sub(F[cell_of(I, i, ay.km)], f0) + T(ay.c1p) * phi_sub(F[cell_of(I, i, ay.kp)], f0);
}

// ---------------------------------------------------------------------------
// k_macro: grad mu, lap mu, grad phi, total force F = -phi grad mu + F_b, and
// Eqs. (u), (P) from the tracked f.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(TX *TY) k_macro(const InstDev *__restrict__ insts, const int4 *__restrict__ tiles,
                                                  const AxisRecT<T> *__restrict__ geo, Planes<T> P, int write_rho)
{
    const int4 t = tiles[blockIdx.x];
    const InstDev &I = insts[t.x];
    const ParT<T> &Pr = par<T>(I);
    if (P.status[t.x] & ST_NONFINITE) return;   // masked: non-finite instance of a batch (a paused one still gets its macros)
    const int i = t.y + threadIdx.x, j = t.z + threadIdx.y;
    if (i >= I.nx || j >= I.ny) return;
    const auto &ax = geo[I.gx_off + i];
    const auto &ay = geo[I.gy_off + j];
    const long long c = cell_of(I, i, j);
    const long long N = P.N;
    const T cs2 = Cst<T>::cs2;
    const T phi = T(phi_val(P.phi[c])), mu = P.mu[c];
    T gmx, gmy, gfx, gfy;
    grad_field(I, P.mu, ax, ay, i, j, mu, gmx, gmy);
    grad_phi<T>(I, P.phi, ax, ay, i, j, P.phi[c], gfx, gfy);
    T lmu = (T(ax.c2m) * P.mu[cell_of(I, ax.km, j)] + T(ax.c20) * mu + T(ax.c2p) * P.mu[cell_of(I, ax.kp, j)])
          + (T(ay.c2m) * P.mu[cell_of(I, i, ay.km)] + T(ay.c20) * mu + T(ay.c2p) * P.mu[cell_of(I, i, ay.kp)]);
    T rho = rho_of<T>(I, phi);
    T Fx = -phi * gmx + (rho - Pr.rho_ref) * Pr.gxa;
    T Fy = -phi * gmy + (rho - Pr.rho_ref) * Pr.gya;
    T sf = 0, mx = 0, my = 0;
#pragma unroll
    for (int q = 0; q < Q; q++) {
        T v = P.f[q * N + c];
        sf += v;
        if (cx(q)) mx += T(cx(q)) * v;
        if (cy(q)) my += T(cy(q)) * v;
    }
    T hdt = T(0.5) * Pr.dt;
    T ux = (mx + hdt * cs2 * Fx) / (cs2 * rho);
    T uy = (my + hdt * cs2 * Fy) / (cs2 * rho);
    T grx = Pr.drho * gfx, gry = Pr.drho * gfy;
    T p = sf + hdt * cs2 * (ux * grx + uy * gry - Pr.gamma * rho * Pr.lambda * lmu);
    P.gmux[c] = gmx;
    P.gmuy[c] = gmy;
    P.lapmu[c] = lmu;
    P.gphix[c] = gfx;
    P.gphiy[c] = gfy;
    P.ux[c] = ux;
    P.uy[c] = uy;
    P.p[c] = p;
    if (write_rho) P.rho[c] = rho;
}

template <typename T>
__device__ __forceinline__ void cell_point(const InstDev &I, const Planes<T> &P, long long c, T gpx, T gpy, Pt<T> &s)
{
    const ParT<T> &Pr = par<T>(I);
    s.phi = T(phi_val(P.phi[c]));
    s.rho = rho_of<T>(I, s.phi);
    s.ux = P.ux[c];
    s.uy = P.uy[c];
    s.p = P.p[c];
    s.mu = P.mu[c];
    s.lapmu = P.lapmu[c];
    T gmx = P.gmux[c], gmy = P.gmuy[c];
    s.Fx = -s.phi * gmx + (s.rho - Pr.rho_ref) * Pr.gxa;
    s.Fy = -s.phi * gmy + (s.rho - Pr.rho_ref) * Pr.gya;
    s.grx = Pr.drho * P.gphix[c];
    s.gry = Pr.drho * P.gphiy[c];
    s.gpx = gpx;
    s.gpy = gpy;
    s.tauf = tauf_of<T>(I, s.phi, s.rho);
}

// ---------------------------------------------------------------------------
// k_cell: grad p, then bar-plus of both distributions at the cell centre
// (step 2, Eq. relations1).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(TX *TY) k_cell(const InstDev *__restrict__ insts, const int4 *__restrict__ tiles,
                                                 const AxisRec *__restrict__ geo, Planes<T> P)
{
    const int4 t = tiles[blockIdx.x];
    const InstDev &I = insts[t.x];
    const ParT<T> &Pr = par<T>(I);
    if (P.status[t.x]) return;   // masked (non-finite) or paused instance of a batch
    const int i = t.y + threadIdx.x, j = t.z + threadIdx.y;
    if (i >= I.nx || j >= I.ny) return;
    const AxisRec &ax = geo[I.gx_off + i];
    const AxisRec &ay = geo[I.gy_off + j];
    const long long c = cell_of(I, i, j);
    const long long N = P.N;
    T gpx, gpy;
    grad_field(I, P.p, ax, ay, i, j, P.p[c], gpx, gpy);
    P.gpx[c] = gpx;
    P.gpy[c] = gpy;
    Pt<T> s;
    cell_point(I, P, c, gpx, gpy, s);
    const T dt = Pr.dt, h = Pr.h, tg = Pr.tau_g, tf = s.tauf;
    // Eq. (relations1) coefficients
    const T af = (T(2) * tf - h) / (T(2) * tf + dt), bf = T(3) * h / (T(2) * tf + dt), cf = T(3) * tf * h / (T(2) * tf + dt);
    const T ag = (T(2) * tg - h) / (T(2) * tg + dt), bg = T(3) * h / (T(2) * tg + dt), cg = T(3) * tg * h / (T(2) * tg + dt);
#pragma unroll
    for (int q = 0; q < Q; q++) {
        T feq, geq, Ff, Fg;
        eq_src<T>(I, s, q, feq, geq, Ff, Fg);
        P.fbp[q * N + c] = af * P.f[q * N + c] + bf * feq + cf * Ff;
        P.gbp[q * N + c] = ag * P.g[q * N + c] + bg * geq + cg * Fg;
    }
}

// Face macroscopic variables from the bar distributions at t+h (Eq.
// conservedVariable with h and bar), then equilibria, sources and the original
// distributions of Eq. (original-function) for every direction.
template <typename T>
struct FaceAux {
    T mu, lapmu, gmux, gmuy, gpx, gpy, gphix, gphiy;
};

template <typename T>
__device__ __forceinline__ void face_originals(const InstDev &I, const T (&fb)[Q], const T (&gb)[Q],
                                               const FaceAux<T> &ax, bool wall, T (&fo)[Q], T (&go)[Q])
{
    const ParT<T> &Pr = par<T>(I);
    const T cs2 = Cst<T>::cs2;
    const T h = Pr.h;
    T phi = 0, sf = 0, mx = 0, my = 0;
#pragma unroll
    for (int q = 0; q < Q; q++) {
        phi += gb[q];
        sf += fb[q];
        if (cx(q)) mx += T(cx(q)) * fb[q];
        if (cy(q)) my += T(cy(q)) * fb[q];
    }
    Pt<T> s;
    s.phi = phi;
    s.rho = rho_of<T>(I, phi);
    s.Fx = -phi * ax.gmux + (s.rho - Pr.rho_ref) * Pr.gxa;
    s.Fy = -phi * ax.gmuy + (s.rho - Pr.rho_ref) * Pr.gya;
    s.grx = Pr.drho * ax.gphix;
    s.gry = Pr.drho * ax.gphiy;
    if (wall) {
        s.ux = 0;
        s.uy = 0;
    } else {
        s.ux = (mx + T(0.5) * h * cs2 * s.Fx) / (cs2 * s.rho);
        s.uy = (my + T(0.5) * h * cs2 * s.Fy) / (cs2 * s.rho);
    }
    s.p = sf + T(0.5) * h * cs2 * (s.ux * s.grx + s.uy * s.gry - Pr.gamma * s.rho * Pr.lambda * ax.lapmu);
    s.mu = ax.mu;
    s.lapmu = ax.lapmu;
    s.gpx = ax.gpx;
    s.gpy = ax.gpy;
    s.tauf = tauf_of<T>(I, phi, s.rho);
    const T tf = s.tauf, tg = Pr.tau_g;
    const T a1 = T(2) * tf / (T(2) * tf + h), b1 = h / (T(2) * tf + h), c1 = tf * h / (T(2) * tf + h);
    const T a2 = T(2) * tg / (T(2) * tg + h), b2 = h / (T(2) * tg + h), c2 = tg * h / (T(2) * tg + h);
#pragma unroll
    for (int q = 0; q < Q; q++) {
        T feq, geq, Ff, Fg;
        eq_src<T>(I, s, q, feq, geq, Ff, Fg);
        fo[q] = a1 * fb[q] + b1 * feq + c1 * Ff;
        go[q] = a2 * gb[q] + b2 * geq + c2 * Fg;
    }
}

// Interior (or periodic) face on axis A between cell L = (iL, jL) and the next
// cell R = (iR, jR); returns the original distributions at the face (steps 3-4).
template <typename T, int A>
__device__ void interior_face(const InstDev &I, const Planes<T> &P, const AxisRec *__restrict__ geo, int iL, int jL,
                              int iR, int jR, T (&fo)[Q], T (&go)[Q])
{
    const ParT<T> &Pr = par<T>(I);
    const long long N = P.N;
    const AxisRec &rn = (A == 0) ? geo[I.gx_off + iL] : geo[I.gy_off + jL];
    const AxisRec &rt = (A == 0) ? geo[I.gy_off + jL] : geo[I.gx_off + iL];
    const T wL = T(rn.wL), wR = T(rn.wR), invd = T(rn.invd);
    const T em = T(rt.e1m), e0 = T(rt.e10), ep = T(rt.e1p);
    const long long cL = cell_of(I, iL, jL), cR = cell_of(I, iR, jR);
    long long cLm, cLp, cRm, cRp;
    if (A == 0) {
        cLm = cell_of(I, iL, rt.km); cLp = cell_of(I, iL, rt.kp);
        cRm = cell_of(I, iR, rt.km); cRp = cell_of(I, iR, rt.kp);
    } else {
        cLm = cell_of(I, rt.km, jL); cLp = cell_of(I, rt.kp, jL);
        cRm = cell_of(I, rt.km, jR); cRp = cell_of(I, rt.kp, jR);
    }
    const T h = Pr.h;
    T fb[Q], gb[Q];
#pragma unroll
    for (int q = 0; q < Q; q++) {
        const T *Pf = P.fbp + q * N;
        const T *Pg = P.gbp + q * N;
        T bL = Pf[cL], bR = Pf[cR];
        T tL = em * Pf[cLm] + e0 * bL + ep * Pf[cLp];
        T tR = em * Pf[cRm] + e0 * bR + ep * Pf[cRp];
        fb[q] = (wL * bL + wR * bR) - h * (T(ca(q, A)) * ((bR - bL) * invd) + T(ca(q, 1 - A)) * (wL * tL + wR * tR));
        bL = Pg[cL]; bR = Pg[cR];
        tL = em * Pg[cLm] + e0 * bL + ep * Pg[cLp];
        tR = em * Pg[cRm] + e0 * bR + ep * Pg[cRp];
        gb[q] = (wL * bL + wR * bR) - h * (T(ca(q, A)) * ((bR - bL) * invd) + T(ca(q, 1 - A)) * (wL * tL + wR * tR));
    }
    FaceAux<T> ax;
    ax.mu = wL * P.mu[cL] + wR * P.mu[cR];
    ax.lapmu = wL * P.lapmu[cL] + wR * P.lapmu[cR];
    ax.gmux = wL * P.gmux[cL] + wR * P.gmux[cR];
    ax.gmuy = wL * P.gmuy[cL] + wR * P.gmuy[cR];
    ax.gpx = wL * P.gpx[cL] + wR * P.gpx[cR];
    ax.gpy = wL * P.gpy[cL] + wR * P.gpy[cR];
    ax.gphix = wL * P.gphix[cL] + wR * P.gphix[cR];
    ax.gphiy = wL * P.gphiy[cL] + wR * P.gphiy[cR];
    face_originals<T>(I, fb, gb, ax, false, fo, go);
}

// Wall face on axis A of cell (i, j), side = +1 (high end) or -1 (low end).
// Outgoing and parallel bar distributions by Taylor reconstruction from the
// cell centre, incoming ones by bounce-back; wall velocity zero; aux values
// of the cell with zero normal gradient; incoming originals by bounce-back.
template <typename T, int A>
__device__ void wall_face(const InstDev &I, const Planes<T> &P, const AxisRec *__restrict__ geo, int i, int j,
                          int side, T (&fo)[Q], T (&go)[Q])
{
    const ParT<T> &Pr = par<T>(I);
    const long long N = P.N;
    const AxisRec &rn = (A == 0) ? geo[I.gx_off + i] : geo[I.gy_off + j];
    const AxisRec &rt = (A == 0) ? geo[I.gy_off + j] : geo[I.gx_off + i];
    const long long c = cell_of(I, i, j);
    long long cnm, cnp, ctm, ctp;
    if (A == 0) {
        cnm = cell_of(I, rn.km, j); cnp = cell_of(I, rn.kp, j);
        ctm = cell_of(I, i, rt.km); ctp = cell_of(I, i, rt.kp);
    } else {
        cnm = cell_of(I, i, rn.km); cnp = cell_of(I, i, rn.kp);
        ctm = cell_of(I, rt.km, j); ctp = cell_of(I, rt.kp, j);
    }
    const T h = Pr.h, half_d = T(0.5) * T(rn.d);
    const T nm = T(rn.e1m), n0 = T(rn.e10), np = T(rn.e1p);
    const T tm = T(rt.e1m), t0 = T(rt.e10), tp = T(rt.e1p);
    T fb[Q], gb[Q];
#pragma unroll
    for (int q = 0; q < Q; q++) {
        if (ca(q, A) * side < 0) continue;
        const T *Pf = P.fbp + q * N;
        const T *Pg = P.gbp + q * N;
        const T off = T(side) * half_d - h * T(ca(q, A));
        const T ht = h * T(ca(q, 1 - A));
        T b = Pf[c];
        fb[q] = b + off * (nm * Pf[cnm] + n0 * b + np * Pf[cnp]) - ht * (tm * Pf[ctm] + t0 * b + tp * Pf[ctp]);
        b = Pg[c];
        gb[q] = b + off * (nm * Pg[cnm] + n0 * b + np * Pg[cnp]) - ht * (tm * Pg[ctm] + t0 * b + tp * Pg[ctp]);
    }
#pragma unroll
    for (int q = 0; q < Q; q++) {
        if (ca(q, A) * side < 0) {
            fb[q] = fb[opp(q)];
            gb[q] = gb[opp(q)];
        }
    }
    FaceAux<T> ax;
    ax.mu = P.mu[c];
    ax.lapmu = P.lapmu[c];
    ax.gmux = (A == 0) ? T(0) : P.gmux[c];
    ax.gmuy = (A == 1) ? T(0) : P.gmuy[c];
    ax.gpx = (A == 0) ? T(0) : P.gpx[c];
    ax.gpy = (A == 1) ? T(0) : P.gpy[c];
    ax.gphix = (A == 0) ? T(0) : P.gphix[c];
    ax.gphiy = (A == 1) ? T(0) : P.gphiy[c];
    face_originals<T>(I, fb, gb, ax, true, fo, go);
#pragma unroll
    for (int q = 0; q < Q; q++) {
        if (ca(q, A) * side < 0) {
            fo[q] = fo[opp(q)];
            go[q] = go[opp(q)];
        }
    }
}

// ---------------------------------------------------------------------------
// k_face: flux through the four faces of each cell (steps 3-5) and the update
// tilde^{n+1} = 4/3 bar-plus - 1/3 tilde - dt/|V| J (Eqs. relations2, updatef),
// in place; then phi = sum g for the next step and the non-finite flag.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(TX *TY) k_face(const InstDev *__restrict__ insts, const int4 *__restrict__ tiles,
                                                 const AxisRec *__restrict__ geo, Planes<T> P)
{
    const int4 t = tiles[blockIdx.x];
    const InstDev &I = insts[t.x];
    const ParT<T> &Pr = par<T>(I);
    if (P.status[t.x]) return;   // masked (non-finite) or paused instance of a batch
    const int i = t.y + threadIdx.x, j = t.z + threadIdx.y;
    if (i >= I.nx || j >= I.ny) return;
    const AxisRec &ax = geo[I.gx_off + i];
    const AxisRec &ay = geo[I.gy_off + j];
    const long long c = cell_of(I, i, j);
    const long long N = P.N;
    T Jf[Q], Jg[Q], fo[Q], go[Q];
#pragma unroll
    for (int q = 0; q < Q; q++) { Jf[q] = 0; Jg[q] = 0; }
    // x faces, area dy
    const T ay_area = T(ay.d), ax_area = T(ax.d);
    // west face
    if (ax.lo_wall) wall_face<T, 0>(I, P, geo, i, j, -1, fo, go);
    else interior_face<T, 0>(I, P, geo, ax.km, j, i, j, fo, go);
#pragma unroll
    for (int q = 0; q < Q; q++) if (cx(q)) { Jf[q] -= T(cx(q)) * fo[q] * ay_area; Jg[q] -= T(cx(q)) * go[q] * ay_area; }
    // east face
    if (ax.hi_wall) wall_face<T, 0>(I, P, geo, i, j, +1, fo, go);
    else interior_face<T, 0>(I, P, geo, i, j, ax.kp, j, fo, go);
#pragma unroll
    for (int q = 0; q < Q; q++) if (cx(q)) { Jf[q] += T(cx(q)) * fo[q] * ay_area; Jg[q] += T(cx(q)) * go[q] * ay_area; }
    // south face
    if (ay.lo_wall) wall_face<T, 1>(I, P, geo, i, j, -1, fo, go);
    else interior_face<T, 1>(I, P, geo, i, ay.km, i, j, fo, go);
#pragma unroll
    for (int q = 0; q < Q; q++) if (cy(q)) { Jf[q] -= T(cy(q)) * fo[q] * ax_area; Jg[q] -= T(cy(q)) * go[q] * ax_area; }
    // north face
    if (ay.hi_wall) wall_face<T, 1>(I, P, geo, i, j, +1, fo, go);
    else interior_face<T, 1>(I, P, geo, i, j, i, ay.kp, fo, go);
#pragma unroll
    for (int q = 0; q < Q; q++) if (cy(q)) { Jf[q] += T(cy(q)) * fo[q] * ax_area; Jg[q] += T(cy(q)) * go[q] * ax_area; }

    const T dtv = Pr.dt / (ax_area * ay_area);
    bool finite = true;
    if constexpr (sizeof(T) == sizeof(double)) {
        T phi = 0;
#pragma unroll
        for (int q = 0; q < Q; q++) {
            T fn = T(4.0 / 3.0) * P.fbp[q * N + c] - T(1.0 / 3.0) * P.f[q * N + c] - dtv * Jf[q];
            T gn = T(4.0 / 3.0) * P.gbp[q * N + c] - T(1.0 / 3.0) * P.g[q * N + c] - dtv * Jg[q];
            P.f[q * N + c] = fn;
            P.g[q * N + c] = gn;
            phi += gn;
            finite = finite && isfinite(fn) && isfinite(gn);
        }
        P.phi[c] = phi;
    } else {
        // FP32 storage: sum_i g~+_i = phi exactly (Eqs. relations1/2), so the
        // order parameter advances by the flux balance alone; it is carried in
        // FP64 and the rest distribution g~_0 is rebuilt from it.
        T jsum = 0, gsum = 0;
#pragma unroll
        for (int q = 0; q < Q; q++) {
            T fn = T(4.0 / 3.0) * P.fbp[q * N + c] - T(1.0 / 3.0) * P.f[q * N + c] - dtv * Jf[q];
            P.f[q * N + c] = fn;
            finite = finite && isfinite(fn);
            jsum += Jg[q];
            if (q > 0) {
                T gn = T(4.0 / 3.0) * P.gbp[q * N + c] - T(1.0 / 3.0) * P.g[q * N + c] - dtv * Jg[q];
                P.g[q * N + c] = gn;
                gsum += gn;
                finite = finite && isfinite(gn);
            }
        }
        const phi_t<T> phi = phi_add(P.phi[c], -(dtv * jsum));
        P.phi[c] = phi;
        P.g[c] = phi_subt(phi, gsum);
        finite = finite && isfinite(phi_val(phi));
    }
    if (!finite) atomicOr(P.status + t.x, 1);
}

// ---------------------------------------------------------------------------
// k_init: step 1, tilde = eq - dt/2 F with the given phi, u, p (planes phi,
// ux, uy, p already hold them; mu was computed by k_mu).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(TX *TY) k_init(const InstDev *__restrict__ insts, const int4 *__restrict__ tiles,
                                                 const AxisRec *__restrict__ geo, Planes<T> P)
{
    const int4 t = tiles[blockIdx.x];
    const InstDev &I = insts[t.x];
    const ParT<T> &Pr = par<T>(I);
    const int i = t.y + threadIdx.x, j = t.z + threadIdx.y;
    if (i >= I.nx || j >= I.ny) return;
    const AxisRec &ax = geo[I.gx_off + i];
    const AxisRec &ay = geo[I.gy_off + j];
    const long long c = cell_of(I, i, j);
    const long long N = P.N;
    Pt<T> s;
    s.phi = T(phi_val(P.phi[c]));
    s.rho = rho_of<T>(I, s.phi);
    s.ux = P.ux[c];
    s.uy = P.uy[c];
    s.p = P.p[c];
    s.mu = P.mu[c];
    T gmx, gmy, gfx, gfy, gpx, gpy;
    grad_field(I, P.mu, ax, ay, i, j, s.mu, gmx, gmy);
    grad_phi<T>(I, P.phi, ax, ay, i, j, P.phi[c], gfx, gfy);
    grad_field(I, P.p, ax, ay, i, j, s.p, gpx, gpy);
    s.lapmu = (T(ax.c2m) * P.mu[cell_of(I, ax.km, j)] + T(ax.c20) * s.mu + T(ax.c2p) * P.mu[cell_of(I, ax.kp, j)])
            + (T(ay.c2m) * P.mu[cell_of(I, i, ay.km)] + T(ay.c20) * s.mu + T(ay.c2p) * P.mu[cell_of(I, i, ay.kp)]);
    s.Fx = -s.phi * gmx + (s.rho - Pr.rho_ref) * Pr.gxa;
    s.Fy = -s.phi * gmy + (s.rho - Pr.rho_ref) * Pr.gya;
    s.grx = Pr.drho * gfx;
    s.gry = Pr.drho * gfy;
    s.gpx = gpx;
    s.gpy = gpy;
    s.tauf = tauf_of<T>(I, s.phi, s.rho);
    const T hdt = T(0.5) * Pr.dt;
    bool finite = true;
    T gsum = 0;
#pragma unroll
    for (int q = 0; q < Q; q++) {
        T feq, geq, Ff, Fg;
        eq_src<T>(I, s, q, feq, geq, Ff, Fg);
        T fv = feq - hdt * Ff, gv = geq - hdt * Fg;
        P.f[q * N + c] = fv;
        P.g[q * N + c] = gv;
        if (q > 0) gsum += gv;
        finite = finite && isfinite(fv) && isfinite(gv);
    }
    // FP32 storage: the rest distribution is rebuilt from the stored phi (sum g = phi)
    if constexpr (sizeof(T) != sizeof(double)) P.g[c] = phi_subt(P.phi[c], gsum);
    if (!finite) atomicOr(P.status + t.x, 1);
}

// phi = sum g (after init or a state load), in index order 0..8
template <typename T>
__global__ void __launch_bounds__(TX *TY) k_phi(const InstDev *__restrict__ insts, const int4 *__restrict__ tiles,
                                                Planes<T> P)
{
    const int4 t = tiles[blockIdx.x];
    const InstDev &I = insts[t.x];
    const ParT<T> &Pr = par<T>(I);
    const int i = t.y + threadIdx.x, j = t.z + threadIdx.y;
    if (i >= I.nx || j >= I.ny) return;
    const long long c = cell_of(I, i, j);
    double phi = 0;
#pragma unroll
    for (int q = 0; q < Q; q++) phi += (double)P.g[q * P.N + c];
    phi_from_double(phi, P.phi[c]);
}

// ---------------------------------------------------------------------------
// Conservation sums (Eq. locallyconserved): per-tile FP64 partials of |V| phi
// and |V| rho (k_reduce for FP64 sims, k_reduce_f32 for FP32 sims); a second
// pass (k_reduce_inst) adds the partials of each instance in tile order.
// ---------------------------------------------------------------------------
// One record per tile for the FP32 conservation sums (k_reduce_f32): the
// cell of the tile's first column and row, the first x and y geometry records,
// the instance's row pitch, and the tile's valid columns and rows.
struct __align__(16) RedTile {
    long long c0;
    int gx, gy, pitch, ncol, nrow, pad;
};

// Double-float arithmetic for the FP32 sums: a value is an unevaluated pair
// hi + lo of floats.  ff_sum is Knuth's TwoSum, ff_mul Dekker's product with
// the FMA giving the exact error of hi * hi; both keep about 48 bits, the
// precision of the stored order parameter.  The _rn intrinsics keep the
// compiler from contracting the steps whose rounding the algorithms rely on.
__device__ __forceinline__ void ff_sum(float ah, float al, float bh, float bl, float &sh, float &sl)
{
    const float s = __fadd_rn(ah, bh);
    const float v = __fsub_rn(s, ah);
    const float e = __fadd_rn(__fsub_rn(ah, __fsub_rn(s, v)), __fsub_rn(bh, v));
    const float t = __fadd_rn(__fadd_rn(e, al), bl);
    sh = __fadd_rn(s, t);
    sl = __fsub_rn(t, __fsub_rn(sh, s));
}
__device__ __forceinline__ void ff_mul(float ah, float al, float bh, float bl, float &ph, float &pl)
{
    const float p = __fmul_rn(ah, bh);
    const float e = __fadd_rn(fmaf(ah, bh, -p), fmaf(ah, bl, __fmul_rn(al, bh)));
    ph = __fadd_rn(p, e);
    pl = __fsub_rn(e, __fsub_rn(ph, p));
}

// k_reduce: per-tile partial sums of |V| phi and |V| rho of FP64 sims, one
// thread block per tile; a second pass (k_reduce_inst) adds the partials of
// each instance in tile order.
template <typename T>
__global__ void __launch_bounds__(TX *TY) k_reduce(const InstDev *__restrict__ insts, const int4 *__restrict__ tiles,
                                                   const AxisRec *__restrict__ geo, Planes<T> P, double2 *partials)
{
    const int lane = (threadIdx.y * TX + threadIdx.x) & 31, warp = (threadIdx.y * TX + threadIdx.x) >> 5;
    __shared__ double2 red[TX * TY / 32];
    const int4 t = tiles[blockIdx.x];
    const InstDev &I = insts[t.x];
    const int i = t.y + threadIdx.x, j = t.z + threadIdx.y;
    double a = 0.0, b = 0.0;
    if (i < I.nx && j < I.ny) {
        const long long c = cell_of(I, i, j);
        const double phi = phi_to_double(P.phi[c]);
        double vol = geo[I.gx_off + i].d * geo[I.gy_off + j].d;
        a = vol * phi;
        b = vol * (I.rhoB + I.drho * (phi - I.phiB));
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if (lane == 0) red[warp] = make_double2(a, b);
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        double2 s = red[0];
        for (int w = 1; w < TX * TY / 32; w++) { s.x += red[w].x; s.y += red[w].y; }
        partials[blockIdx.x] = s;
    }
}

// The FP32 sims' sums |V| phi, one warp per tile over a grid of the blocks the
// SMs hold at once.  Each tile has one record (RedTile) with the addresses the
// warp needs, so a tile costs one dependent load before its data, and the next
// record is in flight while a tile is summed.  Lane l holds column l: it adds
// dy_r phi_r over the tile's rows in double-float, multiplies the sum by its
// dx once, and the lanes are added in a fixed tree; the sum is converted to
// FP64 once per tile (a warp-wide FP64 instruction occupies GB300's FP64 pipe
// for 16 cycles even with one lane active).  gd: the widths {d, d_lo} of the
// geometry records.  Their |V| rho sum is formed per instance from sum |V| phi,
// because rho is linear in phi (Eq. oderrho): sum |V| rho = rhoB V + drho
// (sum |V| phi - phiB V).
__global__ void __launch_bounds__(256) k_reduce_f32(const RedTile *__restrict__ rt, int n_tiles,
                                                    const float2 *__restrict__ gd, const float2 *__restrict__ phi,
                                                    double2 *__restrict__ partials)
{
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * (blockDim.x >> 5);
    int tt = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (tt >= n_tiles) return;
    RedTile t = rt[tt];
    for (; tt < n_tiles; tt += nw) {
        const RedTile nt = rt[tt + nw < n_tiles ? tt + nw : tt];
        const bool col = lane < t.ncol;
        const float2 dx = col ? gd[t.gx + lane] : make_float2(0.f, 0.f);
        float2 ph[TY], dy[TY];
#pragma unroll
        for (int r = 0; r < TY; r++) {
            const bool row = r < t.nrow;
            ph[r] = col && row ? phi[t.c0 + (long long)r * t.pitch + lane] : make_float2(0.f, 0.f);
            dy[r] = row ? gd[t.gy + r] : make_float2(0.f, 0.f);
        }
        float ah = 0.f, al = 0.f;
#pragma unroll
        for (int r = 0; r < TY; r++) {
            float ch, cl;
            ff_mul(dy[r].x, dy[r].y, ph[r].x, ph[r].y, ch, cl);
            ff_sum(ah, al, ch, cl, ah, al);
        }
        ff_mul(ah, al, dx.x, dx.y, ah, al);
        for (int o = 16; o > 0; o >>= 1) {
            const float oh = __shfl_down_sync(0xffffffffu, ah, o), ol = __shfl_down_sync(0xffffffffu, al, o);
            ff_sum(ah, al, oh, ol, ah, al);
        }
        if (lane == 0) partials[tt] = make_double2((double)ah + (double)al, 0.0);
        t = nt;
    }
}

// One warp per instance: lane l adds tiles l, l + 32, ... in order, then the
// lanes are added in a fixed tree.  rho_from_phi: form sum |V| rho from sum
// |V| phi and the total volume (FP32 sims).
__global__ void k_reduce_inst(const InstDev *__restrict__ insts, int n_inst, const double2 *__restrict__ partials,
                              double2 *out, int rho_from_phi)
{
    const int k = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (k >= n_inst) return;
    const InstDev &I = insts[k];
    double2 s = make_double2(0.0, 0.0);
    // unrolled so that several partials are in flight; the additions keep
    // their order
#pragma unroll 8
    for (int t = lane; t < I.ntiles; t += 32) {
        const double2 v = partials[I.tile0 + t];
        s.x += v.x;
        s.y += v.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
        s.x += __shfl_down_sync(0xffffffffu, s.x, o);
        s.y += __shfl_down_sync(0xffffffffu, s.y, o);
    }
    if (lane != 0) return;
    if (rho_from_phi) s.y = I.rhoB * I.vol + I.drho * (s.x - I.phiB * I.vol);
    out[k] = s;
}

// Gather the stored phi plane into a dense double array and back.
template <typename S>
__global__ void k_pack_phi(const InstDev *__restrict__ insts, const int4 *__restrict__ tiles, const S *__restrict__ src,
                           double *__restrict__ dst, const long long *__restrict__ dense0)
{
    const int4 t = tiles[blockIdx.x];
    const InstDev &I = insts[t.x];
    const int i = t.y + threadIdx.x, j = t.z + threadIdx.y;
    if (i >= I.nx || j >= I.ny) return;
    dst[dense0[t.x] + (long long)j * I.nx + i] = phi_to_double(src[cell_of(I, i, j)]);
}

template <typename S>
__global__ void k_unpack_phi(const InstDev *__restrict__ insts, const int4 *__restrict__ tiles,
                             const double *__restrict__ src, S *__restrict__ dst, const long long *__restrict__ dense0)
{
    const int4 t = tiles[blockIdx.x];
    const InstDev &I = insts[t.x];
    const int i = t.y + threadIdx.x, j = t.z + threadIdx.y;
    if (i >= I.nx || j >= I.ny) return;
    phi_from_double(src[dense0[t.x] + (long long)j * I.nx + i], dst[cell_of(I, i, j)]);
}

// Set *flag (zeroed by the caller) when a[0..n) holds a non-finite value: the
// init inputs are checked on the device after the upload, one pass at HBM
// speed, instead of by a host loop over the caller's array.
__global__ void k_any_nonfinite(const double *__restrict__ a, long long n, int *flag)
{
    bool bad = false;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
        bad |= !isfinite(a[c]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

// Gather a padded plane (type T) into a dense double array and back.
template <typename T>
__global__ void k_pack(const InstDev *__restrict__ insts, const int4 *__restrict__ tiles, const T *__restrict__ src,
                       double *__restrict__ dst, const long long *__restrict__ dense0)
{
    const int4 t = tiles[blockIdx.x];
    const InstDev &I = insts[t.x];
    const ParT<T> &Pr = par<T>(I);
    const int i = t.y + threadIdx.x, j = t.z + threadIdx.y;
    if (i >= I.nx || j >= I.ny) return;
    dst[dense0[t.x] + (long long)j * I.nx + i] = (double)src[cell_of(I, i, j)];
}

template <typename T>
__global__ void k_unpack(const InstDev *__restrict__ insts, const int4 *__restrict__ tiles, const double *__restrict__ src,
                         T *__restrict__ dst, const long long *__restrict__ dense0)
{
    const int4 t = tiles[blockIdx.x];
    const InstDev &I = insts[t.x];
    const ParT<T> &Pr = par<T>(I);
    const int i = t.y + threadIdx.x, j = t.z + threadIdx.y;
    if (i >= I.nx || j >= I.ny) return;
    dst[cell_of(I, i, j)] = (T)src[dense0[t.x] + (long long)j * I.nx + i];
}

}  // namespace dugks
