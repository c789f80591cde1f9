// dugks_adjoint.cuh -- reverse-mode (adjoint) sweep of one DUGKS step and of
// the initialisation, written by hand as the transpose of the forward kernels
// of dugks_kernels.cuh (Sec. 2.2 procedure).
//
// Forward step n (the four-kernel form, whose intermediates the adjoint reads):
//   k_mu    mu = psi'(phi) - kappa lap(phi)
//   k_macro grad mu, lap mu, grad phi, F, u, p
//   k_cell  grad p, equilibria, sources, bar-plus (Eq. relations1)
//   k_face  reconstruction, face macros, originals, flux, update (Eq. updatef)
// Reverse, given the adjoint xb of the state at n+1:
//   ka_face_t update and faces  -> adjoint of bar-plus and of the face aux fields
//   ka_cell   bar-plus          -> adjoint of tilde, of u, p, phi, mu and gradients
//   ka_macro  transpose grad p, then p, u, F -> adjoint of tilde f, phi, grad mu, ...
//   ka_mu     transpose grad mu, lap mu, then mu -> adjoint of phi, lap phi
//   ka_phi    transpose grad phi, lap phi, then phi = sum g -> adjoint of tilde g
// The parameters kappa and lambda (the mobility) collect their adjoints per
// instance in FP64.
#pragma once
#include "dugks_fused.cuh"

namespace dugks {

template <typename T>
struct AdjPlanes {
    const T *xf, *xg;   // adjoint of the tracked state at step n+1 [Q][N]
    T *af, *ag;         // adjoint of the tracked state at step n   [Q][N]
    T *bp;              // adjoint of bar-plus [2Q][N]
    T *phi, *mu, *lapmu, *gmx, *gmy, *gfx, *gfy, *gpx, *gpy, *p, *ux, *uy, *lapphi;  // [N]
    double *pk;         // [2 * n_inst]: d/dlambda, d/dkappa per instance
    long long N;
};

template <typename T>
struct PtBar {
    T phi, rho, ux, uy, p, mu, lapmu, Fx, Fy, grx, gry, gpx, gpy;
};

template <typename T>
struct InvBar {
    T uu15, prho, emu, srcF, fg, Gx, Gy, cgx, cgy;
};

template <typename T>
__device__ __forceinline__ PtBar<T> ptbar_zero()
{
    PtBar<T> b;
    b.phi = b.rho = b.ux = b.uy = b.p = b.mu = b.lapmu = b.Fx = b.Fy = b.grx = b.gry = b.gpx = b.gpy = T(0);
    return b;
}

template <typename T>
__device__ __forceinline__ InvBar<T> invbar_zero()
{
    InvBar<T> b;
    b.uu15 = b.prho = b.emu = b.srcF = b.fg = b.Gx = b.Gy = b.cgx = b.cgy = T(0);
    return b;
}

// transpose of eq_src: adjoints of (feq, geq, Ff, Fg) of direction q into s, v
template <typename T>
__device__ __forceinline__ void eq_src_adj(const Pt<T> &s, const PtInv<T> &v, int q, T feqb, T geqb, T Ffb, T Fgb,
                                           PtBar<T> &sb, InvBar<T> &vb)
{
    const T w = T(wq(q));
    const T xu = T(cx(q)) * s.ux + T(cy(q)) * s.uy;
    const T si = w * (T(3) * xu + T(4.5) * xu * xu - v.uu15);
    const T G = w + si;
    const T ex = T(cx(q)) - s.ux, ey = T(cy(q)) - s.uy;
    const T A = s.Fx * G + si * v.cgx, B = s.Fy * G + si * v.cgy;
    const T C = ex * v.Gx + ey * v.Gy;
    T sib = 0, Gb = 0;
    // feq = w p + prho si
    sb.p += w * feqb;
    vb.prho += si * feqb;
    sib += v.prho * feqb;
    // geq = H + phi si, H_0 = phi - (1 - w) emu, H_q = w emu
    sb.phi += si * geqb;
    sib += s.phi * geqb;
    if (q == 0) {
        sb.phi += geqb;
        vb.emu -= (T(1) - w) * geqb;
    } else {
        vb.emu += w * geqb;
    }
    // Ff = ex A + ey B - w srcF
    const T Ab = ex * Ffb, Bb = ey * Ffb;
    T exb = A * Ffb, eyb = B * Ffb;
    vb.srcF -= w * Ffb;
    sb.Fx += G * Ab;
    sb.Fy += G * Bb;
    Gb += s.Fx * Ab + s.Fy * Bb;
    sib += v.cgx * Ab + v.cgy * Bb;
    vb.cgx += si * Ab;
    vb.cgy += si * Bb;
    // Fg = fg C G
    vb.fg += C * G * Fgb;
    const T Cb = v.fg * G * Fgb;
    Gb += v.fg * C * Fgb;
    exb += v.Gx * Cb;
    eyb += v.Gy * Cb;
    vb.Gx += ex * Cb;
    vb.Gy += ey * Cb;
    sb.ux -= exb;
    sb.uy -= eyb;
    // G = w + si, si = w (3 xu + 4.5 xu^2 - uu15)
    sib += Gb;
    const T xub = w * (T(3) + T(9) * xu) * sib;
    vb.uu15 -= w * sib;
    sb.ux += T(cx(q)) * xub;
    sb.uy += T(cy(q)) * xub;
}

// transpose of pt_inv; lamb collects d/dlambda (eta = 3 lambda / tau_g, srcF)
template <typename T>
__device__ __forceinline__ void pt_inv_adj(const ParT<T> &Pr, const Pt<T> &s, const PtInv<T> &v, const InvBar<T> &vb,
                                           PtBar<T> &sb, T &lamb)
{
    const T cs2 = Cst<T>::cs2;
    sb.ux += T(3) * s.ux * vb.uu15;
    sb.uy += T(3) * s.uy * vb.uu15;
    sb.rho += cs2 * vb.prho;
    sb.mu += Pr.eta * vb.emu;
    lamb += T(3) / Pr.tau_g * s.mu * vb.emu;
    sb.rho += cs2 * Pr.gamma * Pr.lambda * s.lapmu * vb.srcF;
    sb.lapmu += cs2 * s.rho * Pr.gamma * Pr.lambda * vb.srcF;
    lamb += cs2 * s.rho * Pr.gamma * s.lapmu * vb.srcF;
    sb.phi += T(3) / s.rho * vb.fg;
    sb.rho -= v.fg / s.rho * vb.fg;
    sb.Fx += vb.Gx;
    sb.Fy += vb.Gy;
    sb.gpx -= vb.Gx;
    sb.gpy -= vb.Gy;
    sb.grx += cs2 * vb.cgx;
    sb.gry += cs2 * vb.cgy;
}

// transpose of tau_f(phi, rho) = 3 mu_mix(phi) / rho (Eqs. mixvis, kineticandmobility)
template <typename T>
__device__ __forceinline__ void tauf_adj(const ParT<T> &Pr, T phi, T rho, T taub, T &phib, T &rhob)
{
    const T K = Pr.muA * Pr.muB * (Pr.phiA - Pr.phiB);
    const T den = (phi - Pr.phiB) * Pr.muB + (Pr.phiA - phi) * Pr.muA;
    const T mu = K / den;
    phib += taub * T(3) / rho * (-K * (Pr.muB - Pr.muA) / (den * den));
    rhob -= taub * T(3) * mu / (rho * rho);
}

// Face of axis A: forward face macros and originals (as face_originals) and
// their transpose.  Ffb/Fgb are the adjoints of the flux values
// (xi . e_A) phi_i |S| of the six flux-carrying directions; outputs are the
// adjoints of the nine bar distributions of each kind and of the face aux.
template <typename T, int A>
__device__ void face_adj(const ParT<T> &Pr, const T (&fb)[Q], const T (&gb)[Q], const FaceAux<T> &ax, bool wall,
                         int side, T area, const T (&Ffb)[6], const T (&Fgb)[6], T (&fbb)[Q], T (&gbb)[Q],
                         FaceAux<T> &axb, T &lamb)
{
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
    s.rho = Pr.rhoB + Pr.drho * (phi - Pr.phiB);
    const T irho = T(1) / s.rho;
    s.Fx = -phi * ax.gmux + (s.rho - Pr.rho_ref) * Pr.gxa;
    s.Fy = -phi * ax.gmuy + (s.rho - Pr.rho_ref) * Pr.gya;
    s.grx = Pr.drho * ax.gphix;
    s.gry = Pr.drho * ax.gphiy;
    if (wall) {
        s.ux = 0;
        s.uy = 0;
    } else {
        s.ux = (T(3) * mx + T(0.5) * h * s.Fx) * irho;
        s.uy = (T(3) * my + T(0.5) * h * s.Fy) * irho;
    }
    s.p = sf + T(0.5) * h * cs2 * (s.ux * s.grx + s.uy * s.gry - Pr.gamma * s.rho * Pr.lambda * ax.lapmu);
    s.mu = ax.mu;
    s.lapmu = ax.lapmu;
    s.gpx = ax.gpx;
    s.gpy = ax.gpy;
    const T K = Pr.muA * Pr.muB * (Pr.phiA - Pr.phiB);
    const T tf = T(3) * (K / ((phi - Pr.phiB) * Pr.muB + (Pr.phiA - phi) * Pr.muA)) / s.rho;
    const T tg = Pr.tau_g;
    const PtInv<T> v = pt_inv_p<T>(Pr, s);
    const T r1 = T(1) / (T(2) * tf + h), r2 = T(1) / (T(2) * tg + h);
    const T a1 = T(2) * tf * r1, b1 = h * r1, c1 = tf * h * r1;
    const T a2 = T(2) * tg * r2, b2 = h * r2, c2 = tg * h * r2;
    // adjoints of the originals
    T fob[Q], gob[Q];
#pragma unroll
    for (int q = 0; q < Q; q++) { fob[q] = 0; gob[q] = 0; fbb[q] = 0; gbb[q] = 0; }
#pragma unroll
    for (int k = 0; k < 6; k++) {
        const int q = fset<A>(k);
        const T vf = T(ca(q, A)) * area * Ffb[k], vg = T(ca(q, A)) * area * Fgb[k];
        const int dst = (wall && ca(q, A) * side < 0) ? opp(q) : q;
        fob[dst] += vf;
        gob[dst] += vg;
    }
    PtBar<T> sb = ptbar_zero<T>();
    InvBar<T> vb = invbar_zero<T>();
    T a1b = 0, b1b = 0, c1b = 0;
#pragma unroll
    for (int k = 0; k < 6; k++) {
        const int q = fset<A>(k);
        if (wall && ca(q, A) * side < 0) continue;
        T feq, geq, F1, F2;
        eq_src<T>(s, v, q, feq, geq, F1, F2);
        fbb[q] += a1 * fob[q];
        a1b += fb[q] * fob[q];
        b1b += feq * fob[q];
        c1b += F1 * fob[q];
        gbb[q] += a2 * gob[q];
        eq_src_adj<T>(s, v, q, b1 * fob[q], b2 * gob[q], c1 * fob[q], c2 * gob[q], sb, vb);
    }
    // a1 = 2 tf r1, b1 = h r1, c1 = tf h r1 with r1 = 1 / (2 tf + h)
    const T taub = (a1b - b1b) * T(2) * h * r1 * r1 + c1b * h * h * r1 * r1;
    pt_inv_adj<T>(Pr, s, v, vb, sb, lamb);
    tauf_adj<T>(Pr, phi, s.rho, taub, sb.phi, sb.rho);
    // p = sf + h/2 c_s^2 (u . grad rho - gamma rho lambda lap mu)
    const T pk = T(0.5) * h * cs2 * sb.p;
    const T sfb = sb.p;
    T uxb = sb.ux + pk * s.grx, uyb = sb.uy + pk * s.gry;
    T grxb = sb.grx + pk * s.ux, gryb = sb.gry + pk * s.uy;
    T rhob = sb.rho - pk * Pr.gamma * Pr.lambda * ax.lapmu;
    const T lapmub = sb.lapmu - pk * Pr.gamma * s.rho * Pr.lambda;
    lamb -= pk * Pr.gamma * s.rho * ax.lapmu;
    // u = (3 m + h/2 F) / rho
    T mxb = 0, myb = 0, Fxb = sb.Fx, Fyb = sb.Fy;
    if (!wall) {
        mxb = T(3) * irho * uxb;
        myb = T(3) * irho * uyb;
        Fxb += T(0.5) * h * irho * uxb;
        Fyb += T(0.5) * h * irho * uyb;
        rhob -= (s.ux * uxb + s.uy * uyb) * irho;
    }
    // F = -phi grad mu + (rho - rho_ref) g
    T phib = sb.phi - ax.gmux * Fxb - ax.gmuy * Fyb;
    rhob += Pr.gxa * Fxb + Pr.gya * Fyb;
    axb.gmux = -phi * Fxb;
    axb.gmuy = -phi * Fyb;
    axb.gphix = Pr.drho * grxb;
    axb.gphiy = Pr.drho * gryb;
    phib += Pr.drho * rhob;
    axb.mu = sb.mu;
    axb.lapmu = lapmub;
    axb.gpx = sb.gpx;
    axb.gpy = sb.gpy;
#pragma unroll
    for (int q = 0; q < Q; q++) {
        fbb[q] += sfb + T(cx(q)) * mxb + T(cy(q)) * myb;
        gbb[q] += phib;
    }
}


// sum over a block of one instance's per-thread parameter adjoint, added in FP64
template <typename T>
__device__ __forceinline__ void block_add_param(double *dst, T v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(dst, (double)v);
}

// ---------------------------------------------------------------------------
// faces: the transposes of the interior and wall faces (Eqs. fbar_h,
// conservedVariable with h, original-function, microfluxf) for a TX x TY tile
// per thread block.  Bar-plus, the face aux fields and the incoming adjoints
// of the tile and its one-cell ring are staged in shared memory with
// coalesced loads, the scatter of the face transposes goes into shared
// accumulators, and each accumulator slot is added to global memory once.
// Each cell owns its west and south faces, and the wall faces at the high end.
// ---------------------------------------------------------------------------
template <typename T>
struct AdjTile {
    static constexpr int W = TX + 2, H = TY + 2, A = W * H;   // region: columns -1..TX, rows -1..TY
    static constexpr int NG = W + H;                          // geometry entries: columns, then rows
    static constexpr int BP = 0, AUX = 2 * Q, XF = 2 * Q + 8, XG = 3 * Q + 8;
    static constexpr int NIN = 4 * Q + 8;                     // staged planes
    static constexpr int NACC = 2 * Q + 8;                    // accumulators: bar-plus, then aux adjoints
    static constexpr size_t al(size_t v) { return (v + 15) / 16 * 16; }
    static constexpr size_t o_in = al((sizeof(T) * 7 + sizeof(int) * 2) * NG);
    static constexpr size_t o_acc = al(o_in + sizeof(T) * NIN * A);
    static constexpr size_t bytes = al(o_acc + sizeof(T) * NACC * A);
    static __device__ __forceinline__ int ri(int x, int y) { return (y + 1) * W + (x + 1); }
    static __device__ __forceinline__ int ex(int x) { return x + 1; }
    static __device__ __forceinline__ int ey(int y) { return W + y + 1; }
};

template <typename T>
struct AdjTileView {
    using AT = AdjTile<T>;
    const T *ga;     // [7][NG]: d, e1m, e10, e1p, wL, wR, invd
    const int *gf;   // [NG] flags: 1 low neighbour, 2 high neighbour, 4 low wall, 8 high wall
    const T *in;     // [NIN][A]
    T *acc;          // [NACC][A]
    __device__ __forceinline__ T g(int k, int e) const { return ga[k * AT::NG + e]; }
    __device__ __forceinline__ T v(int plane, int r) const { return in[plane * AT::A + r]; }
    __device__ __forceinline__ void add(int plane, int r, T val) const { atomicAdd(acc + plane * AT::A + r, val); }
};

template <typename T, int A>
__device__ void interior_face_adj_t(const ParT<T> &Pr, const AdjTileView<T> &V, int xL, int yL, int xR, int yR, T &lamb)
{
    using AT = AdjTile<T>;
    const int rL = AT::ri(xL, yL), rR = AT::ri(xR, yR);
    const int en = A == 0 ? AT::ex(xL) : AT::ey(yL);     // normal axis: the high face of L
    const int et = A == 0 ? AT::ey(yL) : AT::ex(xL);     // tangential axis
    const T wL = V.g(4, en), wR = V.g(5, en), invd = V.g(6, en);
    const T em = V.g(1, et), e0 = V.g(2, et), ep = V.g(3, et);
    const T area = V.g(0, et);
    const int ft = V.gf[et], tstep = A == 0 ? AT::W : 1;
    const int tm = (ft & 1) ? -tstep : 0, tp = (ft & 2) ? tstep : 0;   // a wall ghost is the cell itself
    const T h = Pr.h;
    T fb[Q], gb[Q];
#pragma unroll
    for (int q = 0; q < Q; q++) {
#pragma unroll
        for (int kind = 0; kind < 2; kind++) {
            const int pl = AT::BP + kind * Q + q;
            const T bL = V.v(pl, rL), bR = V.v(pl, rR);
            const T tL = em * V.v(pl, rL + tm) + e0 * bL + ep * V.v(pl, rL + tp);
            const T tR = em * V.v(pl, rR + tm) + e0 * bR + ep * V.v(pl, rR + tp);
            (kind == 0 ? fb : gb)[q] = (wL * bL + wR * bR) - h * (T(ca(q, A)) * ((bR - bL) * invd) + T(ca(q, 1 - A)) * (wL * tL + wR * tR));
        }
    }
    FaceAux<T> ax;
    ax.mu = wL * V.v(AT::AUX + 0, rL) + wR * V.v(AT::AUX + 0, rR);
    ax.lapmu = wL * V.v(AT::AUX + 1, rL) + wR * V.v(AT::AUX + 1, rR);
    ax.gmux = wL * V.v(AT::AUX + 2, rL) + wR * V.v(AT::AUX + 2, rR);
    ax.gmuy = wL * V.v(AT::AUX + 3, rL) + wR * V.v(AT::AUX + 3, rR);
    ax.gpx = wL * V.v(AT::AUX + 4, rL) + wR * V.v(AT::AUX + 4, rR);
    ax.gpy = wL * V.v(AT::AUX + 5, rL) + wR * V.v(AT::AUX + 5, rR);
    ax.gphix = wL * V.v(AT::AUX + 6, rL) + wR * V.v(AT::AUX + 6, rR);
    ax.gphiy = wL * V.v(AT::AUX + 7, rL) + wR * V.v(AT::AUX + 7, rR);
    // the flux value enters J_L with + and J_R with -; J-bar = -dt/|V| x-bar
    const T dtvL = Pr.dt / (V.g(0, AT::ex(xL)) * V.g(0, AT::ey(yL)));
    const T dtvR = Pr.dt / (V.g(0, AT::ex(xR)) * V.g(0, AT::ey(yR)));
    T Ffb[6], Fgb[6];
#pragma unroll
    for (int k = 0; k < 6; k++) {
        const int q = fset<A>(k);
        Ffb[k] = dtvR * V.v(AT::XF + q, rR) - dtvL * V.v(AT::XF + q, rL);
        Fgb[k] = dtvR * V.v(AT::XG + q, rR) - dtvL * V.v(AT::XG + q, rL);
    }
    T fbb[Q], gbb[Q];
    FaceAux<T> axb;
    face_adj<T, A>(Pr, fb, gb, ax, false, 0, area, Ffb, Fgb, fbb, gbb, axb, lamb);
#pragma unroll
    for (int q = 0; q < Q; q++) {
#pragma unroll
        for (int kind = 0; kind < 2; kind++) {
            const T bb = (kind == 0 ? fbb : gbb)[q];
            const int pl = kind * Q + q;
            const T k1 = h * T(ca(q, A)) * invd;
            V.add(pl, rL, (wL + k1) * bb);
            V.add(pl, rR, (wR - k1) * bb);
            if (ca(q, 1 - A)) {
                const T kt = -h * T(ca(q, 1 - A)) * bb;
                V.add(pl, rL + tm, kt * wL * em);
                V.add(pl, rL, kt * wL * e0);
                V.add(pl, rL + tp, kt * wL * ep);
                V.add(pl, rR + tm, kt * wR * em);
                V.add(pl, rR, kt * wR * e0);
                V.add(pl, rR + tp, kt * wR * ep);
            }
        }
    }
    const T vals[8] = {axb.mu, axb.lapmu, axb.gmux, axb.gmuy, axb.gpx, axb.gpy, axb.gphix, axb.gphiy};
#pragma unroll
    for (int k = 0; k < 8; k++) {
        V.add(2 * Q + k, rL, wL * vals[k]);
        V.add(2 * Q + k, rR, wR * vals[k]);
    }
}

template <typename T, int A>
__device__ void wall_face_adj_t(const ParT<T> &Pr, const AdjTileView<T> &V, int x, int y, int side, T &lamb)
{
    using AT = AdjTile<T>;
    const int r = AT::ri(x, y);
    const int en = A == 0 ? AT::ex(x) : AT::ey(y), et = A == 0 ? AT::ey(y) : AT::ex(x);
    const int fn = V.gf[en], ft = V.gf[et];
    const int nstep = A == 0 ? 1 : AT::W, tstep = A == 0 ? AT::W : 1;
    const int nmo = (fn & 1) ? -nstep : 0, npo = (fn & 2) ? nstep : 0;   // a wall ghost is the cell itself
    const int tmo = (ft & 1) ? -tstep : 0, tpo = (ft & 2) ? tstep : 0;
    const T h = Pr.h, half_d = T(0.5) * V.g(0, en);
    const T nm = V.g(1, en), n0 = V.g(2, en), np = V.g(3, en);
    const T tm = V.g(1, et), t0 = V.g(2, et), tp = V.g(3, et);
    const T area = V.g(0, et);
    T fb[Q], gb[Q];
#pragma unroll
    for (int q = 0; q < Q; q++) {
        if (ca(q, A) * side < 0) continue;
        const T off = T(side) * half_d - h * T(ca(q, A));
        const T ht = h * T(ca(q, 1 - A));
#pragma unroll
        for (int kind = 0; kind < 2; kind++) {
            const int pl = AT::BP + kind * Q + q;
            const T b = V.v(pl, r);
            (kind == 0 ? fb : gb)[q] = b + off * (nm * V.v(pl, r + nmo) + n0 * b + np * V.v(pl, r + npo))
                                     - ht * (tm * V.v(pl, r + tmo) + t0 * b + tp * V.v(pl, r + tpo));
        }
    }
#pragma unroll
    for (int q = 0; q < Q; q++) {
        if (ca(q, A) * side < 0) {
            fb[q] = fb[opp(q)];
            gb[q] = gb[opp(q)];
        }
    }
    FaceAux<T> ax;
    ax.mu = V.v(AT::AUX + 0, r);
    ax.lapmu = V.v(AT::AUX + 1, r);
    ax.gmux = (A == 0) ? T(0) : V.v(AT::AUX + 2, r);
    ax.gmuy = (A == 1) ? T(0) : V.v(AT::AUX + 3, r);
    ax.gpx = (A == 0) ? T(0) : V.v(AT::AUX + 4, r);
    ax.gpy = (A == 1) ? T(0) : V.v(AT::AUX + 5, r);
    ax.gphix = (A == 0) ? T(0) : V.v(AT::AUX + 6, r);
    ax.gphiy = (A == 1) ? T(0) : V.v(AT::AUX + 7, r);
    // the flux value enters J_c with the sign of the side
    const T dtv = Pr.dt / (V.g(0, AT::ex(x)) * V.g(0, AT::ey(y)));
    T Ffb[6], Fgb[6];
#pragma unroll
    for (int k = 0; k < 6; k++) {
        const int q = fset<A>(k);
        Ffb[k] = -T(side) * dtv * V.v(AT::XF + q, r);
        Fgb[k] = -T(side) * dtv * V.v(AT::XG + q, r);
    }
    T fbb[Q], gbb[Q];
    FaceAux<T> axb;
    face_adj<T, A>(Pr, fb, gb, ax, true, side, area, Ffb, Fgb, fbb, gbb, axb, lamb);
    // incoming bars were copies of the opposite outgoing ones
#pragma unroll
    for (int q = 0; q < Q; q++) {
        if (ca(q, A) * side < 0) {
            fbb[opp(q)] += fbb[q];
            gbb[opp(q)] += gbb[q];
        }
    }
#pragma unroll
    for (int q = 0; q < Q; q++) {
        if (ca(q, A) * side < 0) continue;
        const T off = T(side) * half_d - h * T(ca(q, A));
        const T ht = h * T(ca(q, 1 - A));
#pragma unroll
        for (int kind = 0; kind < 2; kind++) {
            const T bb = (kind == 0 ? fbb : gbb)[q];
            const int pl = kind * Q + q;
            V.add(pl, r, (T(1) + off * n0 - ht * t0) * bb);
            V.add(pl, r + nmo, off * nm * bb);
            V.add(pl, r + npo, off * np * bb);
            V.add(pl, r + tmo, -ht * tm * bb);
            V.add(pl, r + tpo, -ht * tp * bb);
        }
    }
    V.add(2 * Q + 0, r, axb.mu);
    V.add(2 * Q + 1, r, axb.lapmu);
    if (A == 1) { V.add(2 * Q + 2, r, axb.gmux); V.add(2 * Q + 4, r, axb.gpx); V.add(2 * Q + 6, r, axb.gphix); }
    if (A == 0) { V.add(2 * Q + 3, r, axb.gmuy); V.add(2 * Q + 5, r, axb.gpy); V.add(2 * Q + 7, r, axb.gphiy); }
}

// update and faces of a tile: x_new = 4/3 bar-plus - 1/3 x - dt/|V| J
// (Eqs. relations2, updatef)
template <typename T>
__global__ void __launch_bounds__(TX *TY, sizeof(T) == 4 ? 2 : 1)
    ka_face_t(const InstDev *__restrict__ insts, const int4 *__restrict__ tiles, const AxisRecT<T> *__restrict__ geo,
              Planes<T> P, AdjPlanes<T> Ad)
{
    using AT = AdjTile<T>;
    extern __shared__ __align__(16) unsigned char smem[];
    T *ga = (T *)smem;
    int *gg = (int *)(ga + 7 * AT::NG), *gf = gg + AT::NG;
    T *in = (T *)(smem + AT::o_in);
    T *acc = (T *)(smem + AT::o_acc);
    const int4 t = tiles[blockIdx.x];
    const InstDev &I = insts[t.x];
    const ParT<T> &Pr = par<T>(I);
    const int tid = threadIdx.y * TX + threadIdx.x;
    const int i0 = t.y, j0 = t.z;
    const long long N = P.N;
    // geometry of the region's columns and rows (wrapped on a periodic axis,
    // -1 outside the domain)
    for (int e = tid; e < AT::NG; e += TX * TY) {
        const bool isx = e < AT::W;
        const int n = isx ? I.nx : I.ny;
        int g = isx ? i0 + e - 1 : j0 + (e - AT::W) - 1;
        if ((isx ? I.bcx : I.bcy) == 0) {
            while (g < 0) g += n;
            while (g >= n) g -= n;
        } else if (g < 0 || g >= n) {
            g = -1;
        }
        T v[7] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
        int fl = 0;
        if (g >= 0) {
            const AxisRecT<T> &R = geo[(isx ? I.gx_off : I.gy_off) + g];
            v[0] = R.d; v[1] = R.e1m; v[2] = R.e10; v[3] = R.e1p; v[4] = R.wL; v[5] = R.wR; v[6] = R.invd;
            fl = (R.km == g ? 0 : 1) | (R.kp == g ? 0 : 2) | (R.lo_wall ? 4 : 0) | (R.hi_wall ? 8 : 0);
        }
#pragma unroll
        for (int k = 0; k < 7; k++) ga[k * AT::NG + e] = v[k];
        gg[e] = g;
        gf[e] = fl;
    }
    __syncthreads();
    // staged planes; the accumulators start from the update's 4/3 x-bar in the
    // tile's own cells, whose new x-bar (-1/3 x-bar) is written here
    for (int r = tid; r < AT::A; r += TX * TY) {
        const int x = r % AT::W - 1, y = r / AT::W - 1;
        const int gi = gg[AT::ex(x)], gj = gg[AT::ey(y)];
        const bool inside = gi >= 0 && gj >= 0;
        const bool own = x >= 0 && x < TX && y >= 0 && y < TY && i0 + x < I.nx && j0 + y < I.ny;
        const long long c = inside ? cell_of(I, gi, gj) : 0;
#pragma unroll
        for (int q = 0; q < Q; q++) {
            const T xf = inside ? Ad.xf[q * N + c] : T(0), xg = inside ? Ad.xg[q * N + c] : T(0);
            in[(AT::BP + q) * AT::A + r] = inside ? P.fbp[q * N + c] : T(0);
            in[(AT::BP + Q + q) * AT::A + r] = inside ? P.gbp[q * N + c] : T(0);
            in[(AT::XF + q) * AT::A + r] = xf;
            in[(AT::XG + q) * AT::A + r] = xg;
            acc[q * AT::A + r] = own ? T(4.0 / 3.0) * xf : T(0);
            acc[(Q + q) * AT::A + r] = own ? T(4.0 / 3.0) * xg : T(0);
            if (own) {
                Ad.af[q * N + c] = -T(1.0 / 3.0) * xf;
                Ad.ag[q * N + c] = -T(1.0 / 3.0) * xg;
            }
        }
        const T *aux[8] = {P.mu, P.lapmu, P.gmux, P.gmuy, P.gpx, P.gpy, P.gphix, P.gphiy};
#pragma unroll
        for (int k = 0; k < 8; k++) {
            in[(AT::AUX + k) * AT::A + r] = inside ? aux[k][c] : T(0);
            acc[(2 * Q + k) * AT::A + r] = T(0);
        }
    }
    __syncthreads();
    const AdjTileView<T> V{ga, gf, in, acc};
    T lamb = 0;
    {
        const int x = threadIdx.x, y = threadIdx.y;
        if (i0 + x < I.nx && j0 + y < I.ny) {
            const int fx = gf[AT::ex(x)], fy = gf[AT::ey(y)];
            if (fx & 4) wall_face_adj_t<T, 0>(Pr, V, x, y, -1, lamb);
            else interior_face_adj_t<T, 0>(Pr, V, x - 1, y, x, y, lamb);
            if (fx & 8) wall_face_adj_t<T, 0>(Pr, V, x, y, +1, lamb);
            if (fy & 4) wall_face_adj_t<T, 1>(Pr, V, x, y, -1, lamb);
            else interior_face_adj_t<T, 1>(Pr, V, x, y - 1, x, y, lamb);
            if (fy & 8) wall_face_adj_t<T, 1>(Pr, V, x, y, +1, lamb);
        }
    }
    __syncthreads();
    // every accumulator slot of a cell of the domain, added once
    T *const aux_out[8] = {Ad.mu, Ad.lapmu, Ad.gmx, Ad.gmy, Ad.gpx, Ad.gpy, Ad.gfx, Ad.gfy};
    for (int r = tid; r < AT::A; r += TX * TY) {
        const int gi = gg[AT::ex(r % AT::W - 1)], gj = gg[AT::ey(r / AT::W - 1)];
        if (gi < 0 || gj < 0) continue;
        const long long c = cell_of(I, gi, gj);
#pragma unroll
        for (int k = 0; k < 2 * Q; k++) {
            const T v = acc[k * AT::A + r];
            if (v != T(0)) atomicAdd(Ad.bp + k * N + c, v);
        }
#pragma unroll
        for (int k = 0; k < 8; k++) {
            const T v = acc[(2 * Q + k) * AT::A + r];
            if (v != T(0)) atomicAdd(aux_out[k] + c, v);
        }
    }
    block_add_param(Ad.pk + 2 * t.x, lamb);
}

// ---------------------------------------------------------------------------
// cells
// ---------------------------------------------------------------------------
// transpose of F = -phi grad mu + (rho - rho_ref) g and grad rho = drho grad phi
template <typename T>
__device__ __forceinline__ void force_adj(const ParT<T> &Pr, T phi, T gmx, T gmy, PtBar<T> &sb, T &gmxb, T &gmyb,
                                          T &gfxb, T &gfyb)
{
    sb.phi += -gmx * sb.Fx - gmy * sb.Fy;
    gmxb += -phi * sb.Fx;
    gmyb += -phi * sb.Fy;
    sb.rho += Pr.gxa * sb.Fx + Pr.gya * sb.Fy;
    gfxb += Pr.drho * sb.grx;
    gfyb += Pr.drho * sb.gry;
}

// bar-plus at the cell centre (Eq. relations1) and its equilibria and sources
template <typename T>
__global__ void __launch_bounds__(TX *TY, sizeof(T) == 4 ? 2 : 1) ka_cell(const InstDev *__restrict__ insts, const int4 *__restrict__ tiles,
                                                  const AxisRec *__restrict__ geo, Planes<T> P, AdjPlanes<T> Ad)
{
    const int4 t = tiles[blockIdx.x];
    const InstDev &I = insts[t.x];
    const ParT<T> &Pr = par<T>(I);
    const int i = t.y + threadIdx.x, j = t.z + threadIdx.y;
    T lamb = 0;
    if (i < I.nx && j < I.ny) {
        const long long c = cell_of(I, i, j);
        const long long N = P.N;
        Pt<T> s;
        cell_point(I, P, c, P.gpx[c], P.gpy[c], s);
        const PtInv<T> v = pt_inv_p<T>(Pr, s);
        const T dt = Pr.dt, h = Pr.h, tf = s.tauf, tg = Pr.tau_g;
        const T rf = T(1) / (T(2) * tf + dt), rg = T(1) / (T(2) * tg + dt);
        const T af = (T(2) * tf - h) * rf, bf = T(3) * h * rf, cf = T(3) * tf * h * rf;
        const T ag = (T(2) * tg - h) * rg, bg = T(3) * h * rg, cg = T(3) * tg * h * rg;
        PtBar<T> sb = ptbar_zero<T>();
        InvBar<T> vb = invbar_zero<T>();
        T afb = 0, bfb = 0, cfb = 0;
        // every input of the nine directions is loaded before any store, so
        // that the loads are in flight together
        T pf[Q], pg[Q], fv[Q], xa[Q], xg[Q];
#pragma unroll
        for (int q = 0; q < Q; q++) {
            pf[q] = Ad.bp[q * N + c];
            pg[q] = Ad.bp[(Q + q) * N + c];
            fv[q] = P.f[q * N + c];
            xa[q] = Ad.af[q * N + c];
            xg[q] = Ad.ag[q * N + c];
        }
#pragma unroll
        for (int q = 0; q < Q; q++) {
            T feq, geq, Ff, Fg;
            eq_src<T>(s, v, q, feq, geq, Ff, Fg);
            afb += fv[q] * pf[q];
            bfb += feq * pf[q];
            cfb += Ff * pf[q];
            eq_src_adj<T>(s, v, q, bf * pf[q], bg * pg[q], cf * pf[q], cg * pg[q], sb, vb);
        }
#pragma unroll
        for (int q = 0; q < Q; q++) {
            Ad.af[q * N + c] = xa[q] + af * pf[q];
            Ad.ag[q * N + c] = xg[q] + ag * pg[q];
        }
        // af = (2 tf - h) rf, bf = 3 h rf, cf = 3 tf h rf, rf = 1 / (2 tf + dt)
        const T taub = afb * T(3) * dt * rf * rf - bfb * T(6) * h * rf * rf + cfb * T(3) * h * dt * rf * rf;
        pt_inv_adj<T>(Pr, s, v, vb, sb, lamb);
        tauf_adj<T>(Pr, s.phi, s.rho, taub, sb.phi, sb.rho);
        T gmxb = 0, gmyb = 0, gfxb = 0, gfyb = 0;
        force_adj<T>(Pr, s.phi, P.gmux[c], P.gmuy[c], sb, gmxb, gmyb, gfxb, gfyb);
        sb.phi += Pr.drho * sb.rho;
        Ad.phi[c] += sb.phi;
        Ad.mu[c] += sb.mu;
        Ad.lapmu[c] += sb.lapmu;
        Ad.gmx[c] += gmxb;
        Ad.gmy[c] += gmyb;
        Ad.gfx[c] += gfxb;
        Ad.gfy[c] += gfyb;
        Ad.gpx[c] += sb.gpx;
        Ad.gpy[c] += sb.gpy;
        Ad.p[c] = sb.p;
        Ad.ux[c] = sb.ux;
        Ad.uy[c] = sb.uy;
    }
    block_add_param(Ad.pk + 2 * t.x, lamb);
}

// Transpose of a three-point stencil along axis a: the sum over the cells whose
// stencil reads cell (i, j), of their coefficient times the adjoint there.
// KIND 0: first derivative (c1m, c10, c1p); 1: first derivative in difference
// form (centre weight -(c1m + c1p)); 2: second derivative (c2m, c20, c2p);
// 3: second derivative in difference form.
template <int KIND>
__device__ __forceinline__ double coef(const AxisRec &r, int which)
{
    const double m = (KIND < 2) ? r.c1m : r.c2m, p = (KIND < 2) ? r.c1p : r.c2p;
    const double z = (KIND == 0) ? r.c10 : (KIND == 2) ? r.c20 : -(m + p);
    return which < 0 ? m : which > 0 ? p : z;
}

template <typename T, int KIND>
__device__ __forceinline__ T stencil_t(const InstDev &I, const AxisRec *__restrict__ geo, const T *__restrict__ Ab,
                                       int a, int i, int j)
{
    const long long off = a == 0 ? I.gx_off : I.gy_off;
    const int k = a == 0 ? i : j;
    const AxisRec &r = geo[off + k];
    auto at = [&](int kk) -> T { return Ab[a == 0 ? cell_of(I, kk, j) : cell_of(I, i, kk)]; };
    T s = T(coef<KIND>(r, 0)) * at(k);
    if (r.km == k) s += T(coef<KIND>(r, -1)) * at(k);
    else s += T(coef<KIND>(geo[off + r.km], +1)) * at(r.km);
    if (r.kp == k) s += T(coef<KIND>(r, +1)) * at(k);
    else s += T(coef<KIND>(geo[off + r.kp], -1)) * at(r.kp);
    return s;
}

// p, u, F of the cell (Eqs. u, P), after the transpose of grad p
template <typename T>
__global__ void __launch_bounds__(TX *TY) ka_macro(const InstDev *__restrict__ insts, const int4 *__restrict__ tiles,
                                                   const AxisRec *__restrict__ geo, Planes<T> P, AdjPlanes<T> Ad)
{
    const int4 t = tiles[blockIdx.x];
    const InstDev &I = insts[t.x];
    const ParT<T> &Pr = par<T>(I);
    const int i = t.y + threadIdx.x, j = t.z + threadIdx.y;
    T lamb = 0;
    if (i < I.nx && j < I.ny) {
        const long long c = cell_of(I, i, j);
        const long long N = P.N;
        const T cs2 = Cst<T>::cs2;
        const T hdt = T(0.5) * Pr.dt;
        const T pb = Ad.p[c] + stencil_t<T, 0>(I, geo, Ad.gpx, 0, i, j) + stencil_t<T, 0>(I, geo, Ad.gpy, 1, i, j);
        T uxb = Ad.ux[c], uyb = Ad.uy[c];
        const T phi = T(phi_val(P.phi[c]));
        const T rho = Pr.rhoB + Pr.drho * (phi - Pr.phiB);
        const T ux = P.ux[c], uy = P.uy[c];
        const T grx = Pr.drho * P.gphix[c], gry = Pr.drho * P.gphiy[c];
        const T lmu = P.lapmu[c];
        const T pk = hdt * cs2 * pb;
        // p = sum f + dt/2 c_s^2 (u . grad rho - gamma rho lambda lap mu)
        const T sfb = pb;
        uxb += pk * grx;
        uyb += pk * gry;
        PtBar<T> sb = ptbar_zero<T>();
        sb.grx = pk * ux;
        sb.gry = pk * uy;
        sb.rho = -pk * Pr.gamma * Pr.lambda * lmu;
        const T lmub = -pk * Pr.gamma * rho * Pr.lambda;
        lamb -= pk * Pr.gamma * rho * lmu;
        // u = (3 m + dt/2 F) / rho
        const T mxb = T(3) * uxb / rho, myb = T(3) * uyb / rho;
        sb.Fx = hdt * uxb / rho;
        sb.Fy = hdt * uyb / rho;
        sb.rho -= (ux * uxb + uy * uyb) / rho;
        T gmxb = 0, gmyb = 0, gfxb = 0, gfyb = 0;
        force_adj<T>(Pr, phi, P.gmux[c], P.gmuy[c], sb, gmxb, gmyb, gfxb, gfyb);
        sb.phi += Pr.drho * sb.rho;
#pragma unroll
        for (int q = 0; q < Q; q++) Ad.af[q * N + c] += sfb + T(cx(q)) * mxb + T(cy(q)) * myb;
        Ad.phi[c] += sb.phi;
        Ad.gmx[c] += gmxb;
        Ad.gmy[c] += gmyb;
        Ad.gfx[c] += gfxb;
        Ad.gfy[c] += gfyb;
        Ad.lapmu[c] += lmub;
    }
    block_add_param(Ad.pk + 2 * t.x, lamb);
}

// mu = psi'(phi) - kappa lap(phi) (Eq. chemicalpotential), after the transposes
// of grad mu and lap mu; writes the adjoint of lap(phi)
template <typename T>
__global__ void __launch_bounds__(TX *TY) ka_mu(const InstDev *__restrict__ insts, const int4 *__restrict__ tiles,
                                                const AxisRec *__restrict__ geo, Planes<T> P, AdjPlanes<T> Ad)
{
    const int4 t = tiles[blockIdx.x];
    const InstDev &I = insts[t.x];
    const ParT<T> &Pr = par<T>(I);
    const int i = t.y + threadIdx.x, j = t.z + threadIdx.y;
    T kapb = 0;
    if (i < I.nx && j < I.ny) {
        const long long c = cell_of(I, i, j);
        const AxisRec &ax = geo[I.gx_off + i];
        const AxisRec &ay = geo[I.gy_off + j];
        const T mub = Ad.mu[c] + stencil_t<T, 0>(I, geo, Ad.gmx, 0, i, j) + stencil_t<T, 0>(I, geo, Ad.gmy, 1, i, j)
                    + stencil_t<T, 2>(I, geo, Ad.lapmu, 0, i, j) + stencil_t<T, 2>(I, geo, Ad.lapmu, 1, i, j);
        const phi_t<T> p0 = P.phi[c];
        const T phi = T(phi_val(p0));
        const T a = phi - Pr.phiA, b = phi - Pr.phiB, m = phi - T(0.5) * (Pr.phiA + Pr.phiB);
        const T d2psi = T(4) * Pr.beta * (b * m + a * m + a * b);
        const T lap = (T(ax.c2m) * phi_sub(P.phi[cell_of(I, ax.km, j)], p0) + T(ax.c2p) * phi_sub(P.phi[cell_of(I, ax.kp, j)], p0))
                    + (T(ay.c2m) * phi_sub(P.phi[cell_of(I, i, ay.km)], p0) + T(ay.c2p) * phi_sub(P.phi[cell_of(I, i, ay.kp)], p0));
        Ad.phi[c] += d2psi * mub;
        Ad.lapphi[c] = -Pr.kappa * mub;
        kapb = -lap * mub;
    }
    block_add_param(Ad.pk + 2 * t.x + 1, kapb);
}

// phi = sum_i g~_i, after the transposes of grad phi and lap phi
template <typename T>
__global__ void __launch_bounds__(TX *TY) ka_phi(const InstDev *__restrict__ insts, const int4 *__restrict__ tiles,
                                                 const AxisRec *__restrict__ geo, Planes<T> P, AdjPlanes<T> Ad,
                                                 double *phi0_out, const long long *__restrict__ dense0)
{
    const int4 t = tiles[blockIdx.x];
    const InstDev &I = insts[t.x];
    const int i = t.y + threadIdx.x, j = t.z + threadIdx.y;
    if (i >= I.nx || j >= I.ny) return;
    const long long c = cell_of(I, i, j);
    const long long N = P.N;
    const T phib = Ad.phi[c] + stencil_t<T, 1>(I, geo, Ad.gfx, 0, i, j) + stencil_t<T, 1>(I, geo, Ad.gfy, 1, i, j)
                 + stencil_t<T, 3>(I, geo, Ad.lapphi, 0, i, j) + stencil_t<T, 3>(I, geo, Ad.lapphi, 1, i, j);
    if (phi0_out) {
        // initialisation: phi is the input field itself
        phi0_out[dense0[t.x] + (long long)j * I.nx + i] = (double)phib;
        return;
    }
#pragma unroll
    for (int q = 0; q < Q; q++) Ad.ag[q * N + c] += phib;
}

// Step 1 (Eq. auxf a with the original distribution at equilibrium):
// tilde = eq - dt/2 F; the adjoint of the tracked state is in xf, xg.
template <typename T>
__global__ void __launch_bounds__(TX *TY) ka_init(const InstDev *__restrict__ insts, const int4 *__restrict__ tiles,
                                                  const AxisRec *__restrict__ geo, Planes<T> P, AdjPlanes<T> Ad)
{
    const int4 t = tiles[blockIdx.x];
    const InstDev &I = insts[t.x];
    const ParT<T> &Pr = par<T>(I);
    const int i = t.y + threadIdx.x, j = t.z + threadIdx.y;
    T lamb = 0;
    if (i < I.nx && j < I.ny) {
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
        const PtInv<T> v = pt_inv_p<T>(Pr, s);
        const T hdt = T(0.5) * Pr.dt;
        PtBar<T> sb = ptbar_zero<T>();
        InvBar<T> vb = invbar_zero<T>();
#pragma unroll
        for (int q = 0; q < Q; q++) {
            const T xf = Ad.xf[q * N + c], xg = Ad.xg[q * N + c];
            eq_src_adj<T>(s, v, q, xf, xg, -hdt * xf, -hdt * xg, sb, vb);
        }
        pt_inv_adj<T>(Pr, s, v, vb, sb, lamb);
        T gmxb = 0, gmyb = 0, gfxb = 0, gfyb = 0;
        force_adj<T>(Pr, s.phi, gmx, gmy, sb, gmxb, gmyb, gfxb, gfyb);
        sb.phi += Pr.drho * sb.rho;
        // u, p and grad p are inputs held fixed
        Ad.phi[c] = sb.phi;
        Ad.mu[c] = sb.mu;
        Ad.lapmu[c] = sb.lapmu;
        Ad.gmx[c] = gmxb;
        Ad.gmy[c] = gmyb;
        Ad.gfx[c] = gfxb;
        Ad.gfy[c] = gfyb;
    }
    block_add_param(Ad.pk + 2 * t.x, lamb);
}

// L = sum_cells (phi - phi*)^2: per-tile FP64 partial loss and the seed
// adjoint of the state (dL/dg~_i = 2 (phi - phi*), dL/df~_i = 0).
template <typename T>
__global__ void __launch_bounds__(TX *TY) ka_seed(const InstDev *__restrict__ insts, const int4 *__restrict__ tiles,
                                                  Planes<T> P, T *xf, T *xg, const double *__restrict__ target,
                                                  const long long *__restrict__ dense0, double *loss)
{
    const int4 t = tiles[blockIdx.x];
    const InstDev &I = insts[t.x];
    const int i = t.y + threadIdx.x, j = t.z + threadIdx.y;
    double l = 0.0;
    if (i < I.nx && j < I.ny) {
        const long long c = cell_of(I, i, j);
        const long long N = P.N;
        double phi = 0.0;
#pragma unroll
        for (int q = 0; q < Q; q++) phi += (double)P.g[q * N + c];
        const double d = phi - target[dense0[t.x] + (long long)j * I.nx + i];
        l = d * d;
#pragma unroll
        for (int q = 0; q < Q; q++) {
            xf[q * N + c] = T(0);
            xg[q * N + c] = T(2.0 * d);
        }
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss + t.x, l);
}

}  // namespace dugks
