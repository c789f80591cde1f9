// dugks_ring.cuh -- the DUGKS step (Sec. 2.2, steps 2-7) for a strip of
// blocks, with every shared-memory region a ring of rows and the phases of
// consecutive blocks merged.
//
// A thread block owns BX columns of one instance and marches up a run of
// blocks of BY = 8 rows, like k_strip (dugks_strip.cuh), with the same
// regions: phi on a 4-cell ring, mu on 3, p on 2, bar-plus and the face aux
// fields on 1.  Here each region is a ring of rows addressed by the row's
// position in the strip (phi, mu and the row geometry: 32 slots; p: 16;
// bar-plus and aux: 10), so nothing is shifted between blocks, and the work
// of later blocks runs in the phases of earlier ones.  Block b takes three
// phases:
//   X_b  bar-plus and aux of its rows 1..8 (Eq. relations1)  +  mu of the rows
//        of block b+1 (Eq. chemicalpotential)
//   F_b  its faces (Eqs. fbar_h, conservedVariable with h, original-function,
//        microfluxf), while the tilde rows of block b+1 and the phi rows of
//        block b+2 are copied in (cp.async)
//   U_b  the update of its cells (Eqs. relations2, updatef)  +  p of the rows
//        of block b+1 (Eqs. u, P)
// so three barriers per block, and each phase's items fill the threads evenly
// (with BX = 32 and 288 threads: 272 + 304 items in X, 520 in F, 256 + 288 in
// U).  The arithmetic of every item is that of k_step and k_strip, bit for
// bit.
#pragma once
#include "dugks_strip.cuh"

namespace dugks {

template <typename T, int BX, int BY>
struct RingLayout {
    static_assert(BY == 8, "the ring sizes below hold the rows of an 8-row block and its neighbours");
    static constexpr int W1 = BX + 2, W2 = BX + 4, W3 = BX + 6, W4 = BX + 8;
    static constexpr int R32 = 32, R16 = 16, R1 = BY + 2;   // ring rows: phi, mu, row geometry / p / bar-plus and aux
    static constexpr int A1 = W1 * R1;                      // one bar-plus or aux plane
    static constexpr int NG = W4 + R32 + 1;   // geometry: x positions -4..BX+3, 32 row slots, the y record of a uniform axis
    static constexpr int NFX = (BX + 1) * BY, NFY = BX * BY, NFT = NFX + NFY;
    static constexpr int FROWS = BY + 1, GROWS = BY;        // staged tilde rows of a block (f: 1..BY+1, g: 1..BY)
    static constexpr int NR1 = 7 + 18;
    static constexpr size_t al(size_t v) { return (v + 15) / 16 * 16; }
    static constexpr size_t o_geo = 0;
    static constexpr size_t o_phi = al(o_geo + (sizeof(T) * 11 + sizeof(int) * 2) * NG);
    static constexpr size_t o_mu = al(o_phi + sizeof(phi_t<T>) * R32 * W4);
    static constexpr size_t o_p = al(o_mu + sizeof(T) * R32 * W3);
    static constexpr size_t o_r1 = al(o_p + sizeof(T) * R16 * W2);
    static constexpr size_t o_st = al(o_r1 + sizeof(T) * NR1 * A1);
    static constexpr size_t o_flux = al(o_st + sizeof(T) * Q * (FROWS * W2 + GROWS * W1));
    static constexpr size_t o_keep = al(o_flux + sizeof(pair_t<T>) * 6 * NFT);
    static constexpr size_t bytes = al(o_keep + sizeof(pair_t<T>) * 2 * 6 * BX);
};

// Shared-memory views of a ring strip, with the accessors of Tile
// (dugks_fused.cuh) so that tile_face serves both.  Row y is relative to the
// current block; rb = BY b + 8 is the strip row of its y = 0 (the 8 keeps
// y >= -8 non-negative) and r1b = BY b mod 10.
template <typename T, int BX, int BY, bool UNI>
struct RingTile {
    using L = RingLayout<T, BX, BY>;
    T *ga;
    int *gg, *gf;
    phi_t<T> *phi;
    T *mu, *p;
    T *gmx, *gmy, *lmu, *gfx, *gfy, *gpx, *gpy;
    pair_t<T> *bp;
    int rb = 8, r1b = 0;
    __device__ RingTile(unsigned char *sm)
    {
        ga = (T *)(sm + L::o_geo);
        gg = (int *)(ga + 11 * L::NG);
        gf = gg + L::NG;
        phi = (phi_t<T> *)(sm + L::o_phi);
        mu = (T *)(sm + L::o_mu);
        p = (T *)(sm + L::o_p);
        T *r1 = (T *)(sm + L::o_r1);
        gmx = r1; gmy = r1 + L::A1; lmu = r1 + 2 * L::A1; gfx = r1 + 3 * L::A1; gfy = r1 + 4 * L::A1;
        gpx = r1 + 5 * L::A1; gpy = r1 + 6 * L::A1;
        bp = (pair_t<T> *)(r1 + 7 * L::A1);
    }
    __device__ __forceinline__ int s32(int y) const { return (rb + y) & 31; }
    __device__ __forceinline__ int s16(int y) const { return (rb + y) & 15; }
    // slot of row y in [-1, BY] of the 10-row rings
    __device__ __forceinline__ int s10(int y) const
    {
        const int s = r1b + y + 1;
        return s >= L::R1 ? s - L::R1 : s;
    }
    __device__ __forceinline__ int i1(int x, int y) const { return s10(y) * L::W1 + (x + 1); }
    __device__ __forceinline__ int i2(int x, int y) const { return s16(y) * L::W2 + (x + 2); }
    __device__ __forceinline__ int i3(int x, int y) const { return s32(y) * L::W3 + (x + 3); }
    __device__ __forceinline__ int i4(int x, int y) const { return s32(y) * L::W4 + (x + 4); }
    __device__ __forceinline__ int ge(int axis, int pos) const { return axis == 0 ? pos + 4 : L::W4 + s32(pos); }
    __device__ __forceinline__ int gidx(int axis, int pos) const { return gg[ge(axis, pos)]; }
    __device__ __forceinline__ bool ok(int axis, int pos) const { return UNI || gg[ge(axis, pos)] >= 0; }
    __device__ __forceinline__ int om(int axis, int pos) const { return UNI ? -1 : (gf[ge(axis, pos)] & 1) ? -1 : 0; }
    __device__ __forceinline__ int op(int axis, int pos) const { return UNI ? 1 : (gf[ge(axis, pos)] & 2) ? 1 : 0; }
    __device__ __forceinline__ T c(int k, int axis, int pos) const
    {
        return ga[k * L::NG + (UNI ? (axis == 0 ? 4 : L::W4 + L::R32) : ge(axis, pos))];
    }
    __device__ __forceinline__ int rs1(int y, int d) const { return (s10(y + d) - s10(y)) * L::W1; }
};

template <typename T, int BX, int BY, int NT, int MINB, bool UNI>
__global__ void __launch_bounds__(NT, MINB) k_ring(const InstDev *__restrict__ insts, const int4 *__restrict__ chunks,
                                                   const AxisRecT<T> *__restrict__ geo, StepIO<T> io)
{
    static_assert(NT % 32 == 0 && NT >= BX * BY, "thread count");
    using RL = RingLayout<T, BX, BY>;
    using TL = RingTile<T, BX, BY, UNI>;
    extern __shared__ __align__(16) unsigned char smem[];
    TL S(smem);
    T *stf = (T *)(smem + RL::o_st);                      // staged tilde f [Q][FROWS][W2]
    T *stg = stf + Q * RL::FROWS * RL::W2;                // staged tilde g [Q][GROWS][W1]
    pair_t<T> *flux = (pair_t<T> *)(smem + RL::o_flux);  // [6][NFT]
    // two [6][BX] buffers: block b reads its bottom y faces from buffer b % 2
    // and leaves its top y faces, the next block's bottom ones, in the other
    pair_t<T> *const keep0 = (pair_t<T> *)(smem + RL::o_keep);
    const int4 t = chunks[blockIdx.x];
    const InstDev &I = insts[t.x];
    const ParT<T> &Pr = par<T>(I);
    const int i0 = t.y, j0 = t.z, nblk = t.w;
    const int tid = threadIdx.x;
    const long long N = io.N;
    auto cell = [&](int gi, int gj) -> long long { return I.cell0 + (long long)gj * I.nxp + gi; };
    {
        const int st = io.status[t.x];
        if (st & ST_NONFINITE) return;   // masked: non-finite instance of a batch
        if (st & ST_PAUSED) {            // paused: the state passes to the other buffer unchanged
            for (int r = tid; r < BX * BY * nblk; r += NT) {
                const int gi = i0 + r % BX, gj = j0 + r / BX;
                if (gi >= I.nx || gj >= I.ny) continue;
                const long long c = cell(gi, gj);
#pragma unroll
                for (int q = 0; q < Q; q++) {
                    io.f_out[q * N + c] = io.f_in[q * N + c];
                    io.g_out[q * N + c] = io.g_in[q * N + c];
                }
                io.phi_out[c] = io.phi_in[c];
            }
            return;
        }
    }
    const T cs2 = Cst<T>::cs2;
    const T hdt = T(0.5) * Pr.dt, dt = Pr.dt;
    const T ag = Pr.gca, bg = Pr.gcb, cg = Pr.gcc;
    int jb = j0;   // global row of y = 0 of the current block (before wrapping)
    auto gwrap = [&](bool isx, int g) -> int {
        const int n = isx ? I.nx : I.ny;
        if ((isx ? I.bcx : I.bcy) == 0) {
            while (g < 0) g += n;
            while (g >= n) g -= n;
            return g;
        }
        return (g < 0 || g >= n) ? -1 : g;
    };
    auto grow = [&](int y) -> int { return gwrap(false, jb + y); };
    // geometry entry e: global index, record and flags
    auto set_geo = [&](int e, bool isx, int g, bool record) {
        S.gg[e] = g;
        if (!record) return;
        T v[11];
        int fl = 0;
        if (g >= 0) {
            const AxisRecT<T> &R = geo[(isx ? I.gx_off : I.gy_off) + g];
            v[0] = R.c1m; v[1] = R.c1p; v[2] = R.c2m; v[3] = R.c2p;
            v[4] = R.e1m; v[5] = R.e10; v[6] = R.e1p;
            v[7] = R.wL; v[8] = R.wR; v[9] = R.invd; v[10] = R.d;
            fl = (R.km == g ? 0 : 1) | (R.kp == g ? 0 : 2) | (R.lo_wall ? 4 : 0) | (R.hi_wall ? 8 : 0);
        } else {
#pragma unroll
            for (int k = 0; k < 11; k++) v[k] = T(0);
        }
#pragma unroll
        for (int k = 0; k < 11; k++) S.ga[k * RL::NG + e] = v[k];
        S.gf[e] = fl;
    };
    // geometry of rows [y0, y1) of the current block (a uniform instance needs none)
    auto set_rows = [&](int y0, int y1) {
        if (UNI) return;
        for (int r = tid; r < y1 - y0; r += NT) set_geo(RL::W4 + S.s32(y0 + r), false, grow(y0 + r), true);
    };
    // phi rows [y0, y1) into the phi ring (zero outside the domain)
    auto load_phi = [&](int y0, int y1) {
        for (int r = tid; r < (y1 - y0) * RL::W4; r += NT) {
            const int x = r % RL::W4 - 4, y = y0 + r / RL::W4;
            const int gi = S.gidx(0, x), gj = grow(y);
            if (UNI || (gi >= 0 && gj >= 0)) {
                cp_async<sizeof(phi_t<T>)>(S.phi + S.i4(x, y), io.phi_in + cell(gi, gj));
            } else {
                phi_t<T> z;
                phi_from_zero(z);
                S.phi[S.i4(x, y)] = z;
            }
        }
    };
    // tilde f rows [fy0, fy1) and tilde g rows [gy0, gy1) into the staging rows
    // from 0 (zero outside the domain)
    auto load_fg = [&](int fy0, int fy1, int gy0, int gy1) {
        for (int r = tid; r < (fy1 - fy0) * RL::W2; r += NT) {
            const int x = r % RL::W2 - 2, yy = r / RL::W2;
            const int gi = S.gidx(0, x), gj = grow(fy0 + yy);
            T *d = stf + yy * RL::W2 + (x + 2);
            if (UNI || (gi >= 0 && gj >= 0)) {
                const long long c = cell(gi, gj);
#pragma unroll
                for (int q = 0; q < Q; q++) cp_async<sizeof(T)>(d + q * RL::FROWS * RL::W2, io.f_in + q * N + c);
            } else {
#pragma unroll
                for (int q = 0; q < Q; q++) d[q * RL::FROWS * RL::W2] = T(0);
            }
        }
        for (int r = tid; r < (gy1 - gy0) * RL::W1; r += NT) {
            const int x = r % RL::W1 - 1, yy = r / RL::W1;
            const int gi = S.gidx(0, x), gj = grow(gy0 + yy);
            T *d = stg + yy * RL::W1 + (x + 1);
            if (UNI || (gi >= 0 && gj >= 0)) {
                const long long c = cell(gi, gj);
#pragma unroll
                for (int q = 0; q < Q; q++) cp_async<sizeof(T)>(d + q * RL::GROWS * RL::W1, io.g_in + q * N + c);
            } else {
#pragma unroll
                for (int q = 0; q < Q; q++) d[q * RL::GROWS * RL::W1] = T(0);
            }
        }
    };

    // item r of mu on rows from y0 (Eq. chemicalpotential)
    auto mu_item = [&](int r, int y0) {
        const int x = r % RL::W3 - 3, y = y0 + r / RL::W3;
        T mu = 0;
        if (S.ok(0, x) && S.ok(1, y)) {
            const phi_t<T> p0 = S.phi[S.i4(x, y)];
            const T lap = (S.c(2, 0, x) * phi_sub(S.phi[S.i4(x + S.om(0, x), y)], p0)
                         + S.c(3, 0, x) * phi_sub(S.phi[S.i4(x + S.op(0, x), y)], p0))
                        + (S.c(2, 1, y) * phi_sub(S.phi[S.i4(x, y + S.om(1, y))], p0)
                         + S.c(3, 1, y) * phi_sub(S.phi[S.i4(x, y + S.op(1, y))], p0));
            const T dpsi = T(4) * Pr.beta * phi_subc(p0, I.cA) * phi_subc(p0, I.cB) * phi_subc(p0, I.cM);
            mu = dpsi - Pr.kappa * lap;
        }
        S.mu[S.i3(x, y)] = mu;
    };
    // item r of p on rows from y0 (Eqs. u, P); tilde f staged from row fr0
    auto p_item = [&](int r, int y0, int fr0) {
        const int x = r % RL::W2 - 2, y = y0 + r / RL::W2;
        T vp = 0;
        if (S.ok(0, x) && S.ok(1, y)) {
            const T m0 = S.mu[S.i3(x, y)];
            const T mxm = S.mu[S.i3(x + S.om(0, x), y)] - m0, mxp = S.mu[S.i3(x + S.op(0, x), y)] - m0;
            const T mym = S.mu[S.i3(x, y + S.om(1, y))] - m0, myp = S.mu[S.i3(x, y + S.op(1, y))] - m0;
            const T gmx = S.c(0, 0, x) * mxm + S.c(1, 0, x) * mxp;
            const T gmy = S.c(0, 1, y) * mym + S.c(1, 1, y) * myp;
            const T lmu = (S.c(2, 0, x) * mxm + S.c(3, 0, x) * mxp) + (S.c(2, 1, y) * mym + S.c(3, 1, y) * myp);
            const phi_t<T> p0 = S.phi[S.i4(x, y)];
            const T gfx = S.c(0, 0, x) * phi_sub(S.phi[S.i4(x + S.om(0, x), y)], p0)
                        + S.c(1, 0, x) * phi_sub(S.phi[S.i4(x + S.op(0, x), y)], p0);
            const T gfy = S.c(0, 1, y) * phi_sub(S.phi[S.i4(x, y + S.om(1, y))], p0)
                        + S.c(1, 1, y) * phi_sub(S.phi[S.i4(x, y + S.op(1, y))], p0);
            const T phi = T(phi_val(p0));
            const T rho = rho_of<T>(I, phi);
            const T Fx = -phi * gmx + (rho - Pr.rho_ref) * Pr.gxa;
            const T Fy = -phi * gmy + (rho - Pr.rho_ref) * Pr.gya;
            const T *fr = stf + (y - fr0) * RL::W2 + (x + 2);
            T sf = 0, mx = 0, my = 0;
#pragma unroll
            for (int q = 0; q < Q; q++) {
                const T v = fr[q * RL::FROWS * RL::W2];
                sf += v;
                if (cx(q)) mx += T(cx(q)) * v;
                if (cy(q)) my += T(cy(q)) * v;
            }
            const T irho = fdiv(T(1), rho);
            const T ux = (T(3) * mx + hdt * Fx) * irho;
            const T uy = (T(3) * my + hdt * Fy) * irho;
            vp = sf + hdt * cs2 * (ux * Pr.drho * gfx + uy * Pr.drho * gfy - Pr.gamma * rho * Pr.lambda * lmu);
        }
        S.p[S.i2(x, y)] = vp;
    };
    // item r of grad p, the face aux fields and bar-plus on rows from y0
    // (Eq. relations1); tilde f staged from row fr0, tilde g from row gr0
    auto r1_item = [&](int r, int y0, int fr0, int gr0) {
        const int x = r % RL::W1 - 1, y = y0 + r / RL::W1;
        const int k1 = S.i1(x, y);
        if (!S.ok(0, x) || !S.ok(1, y)) {
            S.gmx[k1] = 0; S.gmy[k1] = 0; S.lmu[k1] = 0; S.gfx[k1] = 0; S.gfy[k1] = 0; S.gpx[k1] = 0; S.gpy[k1] = 0;
#pragma unroll
            for (int q = 0; q < Q; q++) S.bp[q * RL::A1 + k1] = pr(T(0));
            return;
        }
        const T p0 = S.p[S.i2(x, y)];
        const T gpx = S.c(0, 0, x) * (S.p[S.i2(x + S.om(0, x), y)] - p0) + S.c(1, 0, x) * (S.p[S.i2(x + S.op(0, x), y)] - p0);
        const T gpy = S.c(0, 1, y) * (S.p[S.i2(x, y + S.om(1, y))] - p0) + S.c(1, 1, y) * (S.p[S.i2(x, y + S.op(1, y))] - p0);
        const T m0 = S.mu[S.i3(x, y)];
        const T mxm = S.mu[S.i3(x + S.om(0, x), y)] - m0, mxp = S.mu[S.i3(x + S.op(0, x), y)] - m0;
        const T mym = S.mu[S.i3(x, y + S.om(1, y))] - m0, myp = S.mu[S.i3(x, y + S.op(1, y))] - m0;
        const T gmx = S.c(0, 0, x) * mxm + S.c(1, 0, x) * mxp;
        const T gmy = S.c(0, 1, y) * mym + S.c(1, 1, y) * myp;
        const T lmu = (S.c(2, 0, x) * mxm + S.c(3, 0, x) * mxp) + (S.c(2, 1, y) * mym + S.c(3, 1, y) * myp);
        const phi_t<T> ph0 = S.phi[S.i4(x, y)];
        const T gfx = S.c(0, 0, x) * phi_sub(S.phi[S.i4(x + S.om(0, x), y)], ph0)
                    + S.c(1, 0, x) * phi_sub(S.phi[S.i4(x + S.op(0, x), y)], ph0);
        const T gfy = S.c(0, 1, y) * phi_sub(S.phi[S.i4(x, y + S.om(1, y))], ph0)
                    + S.c(1, 1, y) * phi_sub(S.phi[S.i4(x, y + S.op(1, y))], ph0);
        S.gmx[k1] = gmx; S.gmy[k1] = gmy; S.lmu[k1] = lmu; S.gfx[k1] = gfx; S.gfy[k1] = gfy; S.gpx[k1] = gpx; S.gpy[k1] = gpy;
        const T *fr = stf + (y - fr0) * RL::W2 + (x + 2);
        const T *gr = stg + (y - gr0) * RL::W1 + (x + 1);
        T fv[Q];
        T mx = 0, my = 0;
#pragma unroll
        for (int q = 0; q < Q; q++) {
            fv[q] = fr[q * RL::FROWS * RL::W2];
            if (cx(q)) mx += T(cx(q)) * fv[q];
            if (cy(q)) my += T(cy(q)) * fv[q];
        }
        Pt<T> s;
        s.phi = T(phi_val(ph0));
        s.rho = rho_of<T>(I, s.phi);
        s.Fx = -s.phi * gmx + (s.rho - Pr.rho_ref) * Pr.gxa;
        s.Fy = -s.phi * gmy + (s.rho - Pr.rho_ref) * Pr.gya;
        const T irho = fdiv(T(1), s.rho);
        s.ux = (T(3) * mx + hdt * s.Fx) * irho;
        s.uy = (T(3) * my + hdt * s.Fy) * irho;
        s.p = p0;
        s.mu = m0;
        s.lapmu = lmu;
        s.grx = Pr.drho * gfx;
        s.gry = Pr.drho * gfy;
        s.gpx = gpx;
        s.gpy = gpy;
        T af, bf, cf;
        cell_weights<T>(Pr, s.phi, s.rho, af, bf, cf);
        const PtInv<T> v = pt_inv<T>(I, s);
#pragma unroll
        for (int k = 0; k < 5; k++) {
            // the rest direction, then the opposite pairs 1|3, 2|4, 5|7, 6|8
            const int q = k == 0 ? 0 : k < 3 ? k : k + 2;
            T feq[2], geq[2], Ff[2], Fg[2];
            eq_src2<T>(s, v, q, feq, geq, Ff, Fg);
#pragma unroll
            for (int e = 0; e < (k == 0 ? 1 : 2); e++) {
                const int qq = e == 0 ? q : opp(q);
                S.bp[qq * RL::A1 + k1] = pfma(pr(af, ag), pr(fv[qq], gr[qq * RL::GROWS * RL::W1]),
                                              pfma(pr(bf, bg), pr(feq[e], geq[e]), pmul(pr(cf, cg), pr(Ff[e], Fg[e]))));
            }
        }
    };
    // update of cell (x, y) of the current block (Eqs. relations2, updatef)
    auto update_item = [&](int x, int y, int b) {
        const int gi = i0 + x, gj = jb + y;
        if (gi >= I.nx || gj >= I.ny) return;
        pair_t<T> J[Q];
#pragma unroll
        for (int q = 0; q < Q; q++) J[q] = pr(T(0));
        const int kw = y * (BX + 1) + x, ke = kw + 1;
        const int kn = RL::NFX + y * BX + x;              // face between rows y and y + 1
#pragma unroll
        for (int m = 0; m < 6; m++) {
            const int qx = xset(m), qy = yset(m);
            const pair_t<T> south = (y == 0) ? keep0[(b & 1) * 6 * BX + m * BX + x] : flux[m * RL::NFT + kn - BX];
            J[qx] = padd(J[qx], psub(flux[m * RL::NFT + ke], flux[m * RL::NFT + kw]));
            J[qy] = padd(J[qy], psub(flux[m * RL::NFT + kn], south));
        }
        const long long c = cell(gi, gj);
        const int r1 = S.i1(x, y);
        const T dtv = fdiv(dt, S.c(10, 0, x) * S.c(10, 1, y));
        pair_t<T> nw[Q];
#pragma unroll
        for (int q = 0; q < Q; q++)
            nw[q] = pfma(pr(T(4.0 / 3.0)), S.bp[q * RL::A1 + r1],
                         pfma(pr(T(-1.0 / 3.0)), pr(io.f_in[q * N + c], io.g_in[q * N + c]), pmul(pr(-dtv), J[q])));
        bool finite = true;
        if constexpr (sizeof(T) == sizeof(double)) {
            T phi = 0;
#pragma unroll
            for (int q = 0; q < Q; q++) {
                io.f_out[q * N + c] = nw[q].x;
                io.g_out[q * N + c] = nw[q].y;
                phi += nw[q].y;
                finite = finite && isfinite(nw[q].x) && isfinite(nw[q].y);
            }
            io.phi_out[c] = phi;
        } else {
            T jsum = 0, gsum = 0;
#pragma unroll
            for (int q = 0; q < Q; q++) {
                io.f_out[q * N + c] = nw[q].x;
                finite = finite && isfinite(nw[q].x);
                jsum += J[q].y;
                if (q > 0) {
                    io.g_out[q * N + c] = nw[q].y;
                    gsum += nw[q].y;
                    finite = finite && isfinite(nw[q].y);
                }
            }
            const phi_t<T> phi = phi_add(S.phi[S.i4(x, y)], -(dtv * jsum));
            io.phi_out[c] = phi;
            io.g_out[c] = phi_subt(phi, gsum);
            finite = finite && isfinite(phi_val(phi));
        }
        if (!finite) atomicOr(io.status + t.x, ST_NONFINITE);
    };

    // ---- prologue.  Geometry of the columns, of the rows -4..BY+11 and of a
    // uniform instance's one row record; then phi on those rows, mu on rows
    // -3..BY+2, p on -2..BY+1 and bar-plus on -1..0 of block 0.
    const int ph1 = nblk > 1 ? 2 * BY + 4 : BY + 4;    // phi rows of blocks 0 and 1
    for (int r = tid; r < RL::W4; r += NT) set_geo(r, true, gwrap(true, i0 + r - 4), !UNI || r == 4);
    if (UNI && tid == 0) set_geo(RL::W4 + RL::R32, false, gwrap(false, j0), true);
    set_rows(-4, ph1);
    __syncthreads();
    load_phi(-4, ph1);
    load_fg(-2, 2, -1, 1);
    cp_commit();
    cp_wait<0>();
    __syncthreads();
    for (int r = tid; r < (BY + 6) * RL::W3; r += NT) mu_item(r, -3);
    __syncthreads();
    for (int r = tid; r < 4 * RL::W2; r += NT) p_item(r, -2, -2);
    __syncthreads();
    for (int r = tid; r < 2 * RL::W1; r += NT) r1_item(r, -1, -2, -1);
    __syncthreads();
    load_fg(1, BY + 2, 1, BY + 1);
    cp_commit();
    cp_wait<0>();
    __syncthreads();
    for (int r = tid; r < BY * RL::W2; r += NT) p_item(r, 2, 1);
    __syncthreads();

    constexpr int NX1 = BY * RL::W1, NX3 = BY * RL::W3, NU = BX * BY, NU2 = BY * RL::W2;
    for (int b = 0; b < nblk; b++) {
        const bool more = b + 1 < nblk;
        // ---- X_b: bar-plus of rows 1..BY of this block, mu of the next block's
        // rows (BY + 3 .. 2 BY + 2 here)
        for (int k = tid; k < NX1 + (more ? NX3 : 0); k += NT) {
            if (k < NX1) r1_item(k, 1, 1, 1);
            else mu_item(k - NX1, BY + 3);
        }
        __syncthreads();
        // ---- F_b: the next block's tilde rows (rows 1..BY+1 of block b+1, into
        // the staging rows, free once X_b ends) and the phi rows and row
        // geometry of block b+2 are copied in while the faces run
        if (more) load_fg(BY + 1, 2 * BY + 2, BY + 1, 2 * BY + 1);
        if (b + 2 < nblk) {
            set_rows(2 * BY + 4, 3 * BY + 4);
            load_phi(2 * BY + 4, 3 * BY + 4);
        }
        cp_commit();
        // faces: x faces of the block rows and y faces 0|1 .. BY-1|BY; the first
        // block also forms its bottom faces -1|0; later blocks carry them over
        const int nf = RL::NFT + (b == 0 ? BX : 0);
        for (int k = tid; k < nf; k += NT) {
            pair_t<T> F2o[6];
            if (k < RL::NFX) tile_face<T, 0, UNI>(I, S, k % (BX + 1) - 1, k / (BX + 1), F2o);
            else if (k < RL::NFT) tile_face<T, 1, UNI>(I, S, (k - RL::NFX) % BX, (k - RL::NFX) / BX, F2o);
            else tile_face<T, 1, UNI>(I, S, k - RL::NFT, -1, F2o);
            pair_t<T> *dst = k < RL::NFT ? flux + k : keep0 + (k - RL::NFT);   // block 0: buffer 0
            const int stride = k < RL::NFT ? RL::NFT : BX;
#pragma unroll
            for (int m = 0; m < 6; m++) dst[m * stride] = F2o[m];
            if (k >= RL::NFT - BX && k < RL::NFT) {   // top row: also the next block's bottom faces
#pragma unroll
                for (int m = 0; m < 6; m++) keep0[((b + 1) & 1) * 6 * BX + m * BX + (k - (RL::NFT - BX))] = F2o[m];
            }
        }
        cp_wait<0>();
        __syncthreads();
        // ---- U_b: the update of the block's cells, p of the next block's rows
        // (BY + 2 .. 2 BY + 1 here; tilde f staged from row BY + 1)
        for (int k = tid; k < NU + (more ? NU2 : 0); k += NT) {
            if (k < NU) update_item(k % BX, k / BX, b);
            else p_item(k - NU, BY + 2, BY + 1);
        }
        __syncthreads();
        S.rb += BY;
        S.r1b = S.r1b + BY >= RL::R1 ? S.r1b + BY - RL::R1 : S.r1b + BY;
        jb += BY;
    }
}

}  // namespace dugks
