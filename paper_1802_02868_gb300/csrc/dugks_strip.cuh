// dugks_strip.cuh -- the DUGKS step (Sec. 2.2, steps 2-7) for a strip of
// blocks: a thread block owns BX columns and marches up a run of blocks of BY
// rows (the strip length comes from the strip table), bottom to top.
//
// The per-block regions and phases are those of k_step (dugks_fused.cuh):
// phi on a 4-cell ring, mu on 3, p on 2, bar-plus and the face aux fields on
// 1, then the faces and the update.  Consecutive blocks share the top rows of
// these rings, so each block computes only its BY new rows of every region and
// shifts the shared rows, and the geometry of the rows, down afterwards; the y
// faces between two blocks are computed once and carried over.  A prologue
// computes the bottom rows of the first block's rings.  Shared memory does not
// grow with the strip length.  The thread count NT is chosen so that the new
// rows of a phase fill whole passes of the threads (with BX = 32, BY = 8 and
// 288 threads: p 288 items, bar-plus 272, the 520 faces in two passes).
//
// Loads of a later block overlap the work of the one before: its new phi rows
// are copied into a staging area while the faces and the update run, and its
// tilde f and g rows into the (then free) flux bytes while the rings shift.
// The shift refills the phi rows it moves down from the staging area, so a
// block starts without a load wait of its own.
#pragma once
#include "dugks_fused.cuh"

namespace dugks {

template <typename T, int BX, int BY>
struct StripLayout {
    using L = FusedLayout<T, BX, BY, false>;
    static_assert(BY == 8, "the shifted ring rows are the rows that the next block's new rows replace");
    // face items of a block, in the order the threads take them and the flux
    // buffer stores them: the x faces on the pitch of the R1 planes (XP items
    // a row, the last one idle), so that a warp's faces read consecutive R1
    // entries across a row change; then, from item Y0 (a whole number of
    // warps), the y faces one row of BX per warp.  Either way no warp reads
    // two R1 entries of one shared-memory bank.
    static constexpr int XP = BX + 2;
    static constexpr int NXI = XP * BY;
    static constexpr int Y0 = (NXI + 31) / 32 * 32;
    static constexpr int NFY = BX * BY;                   // y faces per block (the bottom row is carried)
    static constexpr int NFT = Y0 + NFY;
    static constexpr int FROWS = BY + 1, GROWS = BY;      // staged tilde rows of a block (f: 1..BY+1, g: 1..BY)
    static constexpr size_t al(size_t v) { return (v + 15) / 16 * 16; }
    static constexpr size_t o_un = L::o_un;               // after the R1 planes
    // staging rows on pitch SP with column x at SO + x: x = 0 on a 16-byte
    // boundary, so that a uniform row can arrive in 16-byte copies
    static constexpr int SP = BX + 8, SO = 4;
    static constexpr size_t st_f = sizeof(T) * Q * FROWS * SP;
    static constexpr size_t st_g = sizeof(T) * Q * GROWS * SP;
    static constexpr size_t st_flux = sizeof(pair_t<T>) * 6 * NFT;
    static constexpr size_t un = (st_f + st_g > st_flux) ? st_f + st_g : st_flux;
    static constexpr size_t o_st = o_un;                  // staging: the flux bytes, free after the update
    static constexpr size_t o_phst = al(o_un + un);  // the next block's new phi rows [BY][W4]
    static constexpr size_t o_keep = al(o_phst + sizeof(phi_t<T>) * BY * L::W4);      // carried y-face rows [2][6][BX] pairs (by block parity)
    static constexpr size_t bytes = al(o_keep + sizeof(pair_t<T>) * 2 * 6 * BX);
};

template <typename T, int BX, int BY, int NT, int MINB, bool UNI>
__global__ void __launch_bounds__(NT, MINB) k_strip(const InstDev *__restrict__ insts, const int4 *__restrict__ chunks,
                                                    const AxisRecT<T> *__restrict__ geo, StepIO<T> io)
{
    static_assert(NT % 32 == 0 && NT >= BX * BY, "thread count");
    using SL = StripLayout<T, BX, BY>;
    using L = typename SL::L;
    using TL = Tile<T, BX, BY, UNI, false>;
    extern __shared__ __align__(16) unsigned char smem[];
    TL S(smem);
    T *stf = (T *)(smem + SL::o_st);                      // staged tilde f [Q][FROWS][SP]
    T *stg = stf + Q * SL::FROWS * SL::SP;                // staged tilde g [Q][GROWS][SP]
    phi_t<T> *phst = (phi_t<T> *)(smem + SL::o_phst);    // staged phi rows 4 .. BY + 3 of the next block
    pair_t<T> *flux = (pair_t<T> *)(smem + SL::o_un);    // [6][NFT], by face item
    // two [6][BX] buffers: block b reads its bottom y faces from buffer b % 2
    // and leaves its top y faces, the next block's bottom ones, in the other
    pair_t<T> *const keep0 = (pair_t<T> *)(smem + SL::o_keep);
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
    // 16-byte staging copies: FP32, uniform periodic, a width that is a
    // multiple of 4 (row pitches and instance offsets are multiples of 32)
    // and 16-byte aligned planes
    const bool wide = UNI && sizeof(T) == 4 && I.nx % 4 == 0 &&
                      ((reinterpret_cast<unsigned long long>(io.f_in) | reinterpret_cast<unsigned long long>(io.g_in) |
                        (unsigned long long)(N * sizeof(T))) & 15) == 0;
    const bool wide_phi = wide && (reinterpret_cast<unsigned long long>(io.phi_in) & 15) == 0;
    const T ag = Pr.gca, bg = Pr.gcb, cg = Pr.gcc;
    // global index of a column (x) or of row y of block b (wrapped on a periodic
    // axis, -1 outside the domain)
    auto gwrap = [&](bool isx, int g) -> int {
        const int n = isx ? I.nx : I.ny;
        if ((isx ? I.bcx : I.bcy) == 0) {
            while (g < 0) g += n;
            while (g >= n) g -= n;
            return g;
        }
        return (g < 0 || g >= n) ? -1 : g;
    };
    auto grow = [&](int b, int y) -> int { return gwrap(false, j0 + b * BY + y); };
    // geometry entry r: global index, record and flags (on a uniform periodic
    // instance only position 0 of each axis carries the record)
    auto set_geo = [&](int r, bool isx, int pos, int g) {
        S.gg[r] = g;
        if (UNI && pos != 0) return;
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
        for (int k = 0; k < 11; k++) S.ga[k * L::NG + r] = v[k];
        S.gf[r] = fl;
    };

    // ---- geometry of the columns and of the first block's rows -4..3
    for (int r = tid; r < L::W4 + 8; r += NT) {
        if (r < L::W4) set_geo(r, true, r - 4, gwrap(true, i0 + r - 4));
        else set_geo(r, false, r - L::W4 - 4, grow(0, r - L::W4 - 4));
    }
    __syncthreads();

    // rows of block b: phi [ph0, ph1) into the phi ring and the geometry of
    // the rows [4, BY + 4) that are new to it
    auto load_phi = [&](int b, int ph0, int ph1) {
        if (b >= 0)
            for (int r = tid; r < BY; r += NT) set_geo(L::W4 + 8 + r, false, 4 + r, grow(b, 4 + r));
        const int bb = b < 0 ? 0 : b;
        for (int r = tid; r < (ph1 - ph0) * L::W4; r += NT) {
            const int x = r % L::W4 - 4, y = ph0 + r / L::W4;
            const int gi = S.gidx(0, x), gj = grow(bb, y);
            if (UNI || (gi >= 0 && gj >= 0)) {
                cp_async<sizeof(phi_t<T>)>(S.phi + TL::i4(x, y), io.phi_in + cell(gi, gj));
            } else {
                phi_t<T> z;
                phi_from_zero(z);
                S.phi[TL::i4(x, y)] = z;
            }
        }
    };
    // the new phi rows 4 .. BY + 3 of block b into the phi staging rows
    auto load_phi_next = [&](int b) {
        if (wide_phi) {
            // two cells per 16-byte copy: x even and an even width, so a pair
            // never straddles the periodic wrap
            for (int r = tid; r < BY * (L::W4 / 2); r += NT) {
                const int x = 2 * (r % (L::W4 / 2)) - 4, y = 4 + r / (L::W4 / 2);
                cp_async<16>(phst + (y - 4) * L::W4 + (x + 4), io.phi_in + cell(S.gidx(0, x), grow(b, y)));
            }
            return;
        }
        for (int r = tid; r < BY * L::W4; r += NT) {
            const int x = r % L::W4 - 4, y = 4 + r / L::W4;
            const int gi = S.gidx(0, x), gj = grow(b, y);
            if (UNI || (gi >= 0 && gj >= 0)) {
                cp_async<sizeof(phi_t<T>)>(phst + r, io.phi_in + cell(gi, gj));
            } else {
                phi_t<T> z;
                phi_from_zero(z);
                phst[r] = z;
            }
        }
    };
    // tilde f rows [fr0, fr1) and tilde g rows [gr0, gr1) of block b into the
    // staging area (zero outside the domain); the f copies are committed as a
    // group, the g copies are left for the caller to commit
    auto load_fg = [&](int b, int fr0, int fr1, int gr0, int gr1) {
        const int bb = b < 0 ? 0 : b;
        if (wide) {
            // per row ten copies of each plane: the 32 interior columns in
            // 16-byte pieces of four, and the halo (f: x = -2..-1 and 32..33 in
            // 8-byte pairs; g: x = -1 and 32).  A piece never straddles the
            // periodic wrap: the width and the strip origin are multiples of 4.
            for (int r = tid; r < (fr1 - fr0) * 10; r += NT) {
                const int yy = r / 10, k = r % 10;
                const int x = k < 8 ? 4 * k : k == 8 ? -2 : BX;
                const long long c = cell(S.gidx(0, x), grow(bb, fr0 + yy));
                T *d = stf + yy * SL::SP + (x + SL::SO);
                if (k < 8) {
#pragma unroll
                    for (int q = 0; q < Q; q++) cp_async<16>(d + q * SL::FROWS * SL::SP, io.f_in + q * N + c);
                } else {
#pragma unroll
                    for (int q = 0; q < Q; q++) cp_async<8>(d + q * SL::FROWS * SL::SP, io.f_in + q * N + c);
                }
            }
            cp_commit();   // f and g in groups of their own: p waits for f only
            for (int r = tid; r < (gr1 - gr0) * 10; r += NT) {
                const int yy = r / 10, k = r % 10;
                const int x = k < 8 ? 4 * k : k == 8 ? -1 : BX;
                const long long c = cell(S.gidx(0, x), grow(bb, gr0 + yy));
                T *d = stg + yy * SL::SP + (x + SL::SO);
                if (k < 8) {
#pragma unroll
                    for (int q = 0; q < Q; q++) cp_async<16>(d + q * SL::GROWS * SL::SP, io.g_in + q * N + c);
                } else {
#pragma unroll
                    for (int q = 0; q < Q; q++) cp_async<4>(d + q * SL::GROWS * SL::SP, io.g_in + q * N + c);
                }
            }
            return;
        }
        for (int r = tid; r < (fr1 - fr0) * L::W2; r += NT) {
            const int x = r % L::W2 - 2, yy = r / L::W2;
            const int gi = S.gidx(0, x), gj = grow(bb, fr0 + yy);
            T *d = stf + yy * SL::SP + (x + SL::SO);
            if (UNI || (gi >= 0 && gj >= 0)) {
                const long long c = cell(gi, gj);
#pragma unroll
                for (int q = 0; q < Q; q++) cp_async<sizeof(T)>(d + q * SL::FROWS * SL::SP, io.f_in + q * N + c);
            } else {
#pragma unroll
                for (int q = 0; q < Q; q++) d[q * SL::FROWS * SL::SP] = T(0);
            }
        }
        cp_commit();   // f and g in groups of their own: p waits for f only
        for (int r = tid; r < (gr1 - gr0) * L::W1; r += NT) {
            const int x = r % L::W1 - 1, yy = r / L::W1;
            const int gi = S.gidx(0, x), gj = grow(bb, gr0 + yy);
            T *d = stg + yy * SL::SP + (x + SL::SO);
            if (UNI || (gi >= 0 && gj >= 0)) {
                const long long c = cell(gi, gj);
#pragma unroll
                for (int q = 0; q < Q; q++) cp_async<sizeof(T)>(d + q * SL::GROWS * SL::SP, io.g_in + q * N + c);
            } else {
#pragma unroll
                for (int q = 0; q < Q; q++) d[q * SL::GROWS * SL::SP] = T(0);
            }
        }
    };
    auto load_wait = [&]() {
        cp_commit();
        cp_wait<0>();
        __syncthreads();
    };

    // mu on R3 rows [y0, y1) (Eq. chemicalpotential)
    auto mu_rows = [&](int y0, int y1) {
        for (int r = tid; r < (y1 - y0) * L::W3; r += NT) {
            int x, y;
            TL::ring_item(r, y1 - y0, 3, y0, x, y);
            T mu = 0;
            if (S.ok(0, x) && S.ok(1, y)) {
                const phi_t<T> p0 = S.phi[TL::i4(x, y)];
                const T lap = (S.c(2, 0, x) * phi_sub(S.phi[TL::i4(x + S.om(0, x), y)], p0)
                             + S.c(3, 0, x) * phi_sub(S.phi[TL::i4(x + S.op(0, x), y)], p0))
                            + (S.c(2, 1, y) * phi_sub(S.phi[TL::i4(x, y + S.om(1, y))], p0)
                             + S.c(3, 1, y) * phi_sub(S.phi[TL::i4(x, y + S.op(1, y))], p0));
                const T dpsi = T(4) * Pr.beta * phi_subc(p0, I.cA) * phi_subc(p0, I.cB) * phi_subc(p0, I.cM);
                mu = dpsi - Pr.kappa * lap;
            }
            S.mu[TL::i3(x, y)] = mu;
        }
        cp_wait<1>();   // the block's tilde f rows (issued during the shift) are in
        __syncthreads();
    };

    // p on R2 rows [y0, y1) (Eqs. u, P); tilde f staged from row fr0
    auto p_rows = [&](int y0, int y1, int fr0) {
        for (int r = tid; r < (y1 - y0) * L::W2; r += NT) {
            int x, y;
            TL::ring_item(r, y1 - y0, 2, y0, x, y);
            T vp = 0;
            if (S.ok(0, x) && S.ok(1, y)) {
                const T m0 = S.mu[TL::i3(x, y)];
                const T mxm = S.mu[TL::i3(x + S.om(0, x), y)] - m0, mxp = S.mu[TL::i3(x + S.op(0, x), y)] - m0;
                const T mym = S.mu[TL::i3(x, y + S.om(1, y))] - m0, myp = S.mu[TL::i3(x, y + S.op(1, y))] - m0;
                const T gmx = S.c(0, 0, x) * mxm + S.c(1, 0, x) * mxp;
                const T gmy = S.c(0, 1, y) * mym + S.c(1, 1, y) * myp;
                const T lmu = (S.c(2, 0, x) * mxm + S.c(3, 0, x) * mxp) + (S.c(2, 1, y) * mym + S.c(3, 1, y) * myp);
                const phi_t<T> p0 = S.phi[TL::i4(x, y)];
                const T gfx = S.c(0, 0, x) * phi_sub(S.phi[TL::i4(x + S.om(0, x), y)], p0)
                            + S.c(1, 0, x) * phi_sub(S.phi[TL::i4(x + S.op(0, x), y)], p0);
                const T gfy = S.c(0, 1, y) * phi_sub(S.phi[TL::i4(x, y + S.om(1, y))], p0)
                            + S.c(1, 1, y) * phi_sub(S.phi[TL::i4(x, y + S.op(1, y))], p0);
                const T phi = T(phi_val(p0));
                const T rho = rho_of<T>(I, phi);
                const T Fx = -phi * gmx + (rho - Pr.rho_ref) * Pr.gxa;
                const T Fy = -phi * gmy + (rho - Pr.rho_ref) * Pr.gya;
                const T *fr = stf + (y - fr0) * SL::SP + (x + SL::SO);
                T sf = 0, mx = 0, my = 0;
#pragma unroll
                for (int q = 0; q < Q; q++) {
                    const T v = fr[q * SL::FROWS * SL::SP];
                    sf += v;
                    if (cx(q)) mx += T(cx(q)) * v;
                    if (cy(q)) my += T(cy(q)) * v;
                }
                const T irho = fdiv(T(1), rho);
                const T ux = (T(3) * mx + hdt * Fx) * irho;
                const T uy = (T(3) * my + hdt * Fy) * irho;
                vp = sf + hdt * cs2 * (ux * Pr.drho * gfx + uy * Pr.drho * gfy - Pr.gamma * rho * Pr.lambda * lmu);
            }
            S.p[TL::i2(x, y)] = vp;
        }
        cp_wait<0>();   // and the tilde g rows
        __syncthreads();
    };

    // grad p, the face aux fields and bar-plus on R1 rows [y0, y1) (Eq. relations1);
    // tilde f staged from row fr0, tilde g from row gr0
    auto r1_rows = [&](int y0, int y1, int fr0, int gr0) {
        for (int r = tid; r < (y1 - y0) * L::W1; r += NT) {
            int x, y;
            TL::ring_item(r, y1 - y0, 1, y0, x, y);
            const int k1 = TL::i1(x, y);
            if (!S.ok(0, x) || !S.ok(1, y)) {
                S.gmx[k1] = 0; S.gmy[k1] = 0; S.lmu[k1] = 0; S.gfx[k1] = 0; S.gfy[k1] = 0; S.gpx[k1] = 0; S.gpy[k1] = 0;
#pragma unroll
                for (int q = 0; q < Q; q++) S.bp[q * L::A1 + k1] = pr(T(0));
                continue;
            }
            const T p0 = S.p[TL::i2(x, y)];
            const T gpx = S.c(0, 0, x) * (S.p[TL::i2(x + S.om(0, x), y)] - p0) + S.c(1, 0, x) * (S.p[TL::i2(x + S.op(0, x), y)] - p0);
            const T gpy = S.c(0, 1, y) * (S.p[TL::i2(x, y + S.om(1, y))] - p0) + S.c(1, 1, y) * (S.p[TL::i2(x, y + S.op(1, y))] - p0);
            const T m0 = S.mu[TL::i3(x, y)];
            const T mxm = S.mu[TL::i3(x + S.om(0, x), y)] - m0, mxp = S.mu[TL::i3(x + S.op(0, x), y)] - m0;
            const T mym = S.mu[TL::i3(x, y + S.om(1, y))] - m0, myp = S.mu[TL::i3(x, y + S.op(1, y))] - m0;
            const T gmx = S.c(0, 0, x) * mxm + S.c(1, 0, x) * mxp;
            const T gmy = S.c(0, 1, y) * mym + S.c(1, 1, y) * myp;
            const T lmu = (S.c(2, 0, x) * mxm + S.c(3, 0, x) * mxp) + (S.c(2, 1, y) * mym + S.c(3, 1, y) * myp);
            const phi_t<T> ph0 = S.phi[TL::i4(x, y)];
            const T gfx = S.c(0, 0, x) * phi_sub(S.phi[TL::i4(x + S.om(0, x), y)], ph0)
                        + S.c(1, 0, x) * phi_sub(S.phi[TL::i4(x + S.op(0, x), y)], ph0);
            const T gfy = S.c(0, 1, y) * phi_sub(S.phi[TL::i4(x, y + S.om(1, y))], ph0)
                        + S.c(1, 1, y) * phi_sub(S.phi[TL::i4(x, y + S.op(1, y))], ph0);
            S.gmx[k1] = gmx; S.gmy[k1] = gmy; S.lmu[k1] = lmu; S.gfx[k1] = gfx; S.gfy[k1] = gfy; S.gpx[k1] = gpx; S.gpy[k1] = gpy;
            const T *fr = stf + (y - fr0) * SL::SP + (x + SL::SO);
            const T *gr = stg + (y - gr0) * SL::SP + (x + SL::SO);
            T fv[Q];
            T mx = 0, my = 0;
#pragma unroll
            for (int q = 0; q < Q; q++) {
                fv[q] = fr[q * SL::FROWS * SL::SP];
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
                    S.bp[qq * L::A1 + k1] = pfma(pr(af, ag), pr(fv[qq], gr[qq * SL::GROWS * SL::SP]),
                                                 pfma(pr(bf, bg), pr(feq[e], geq[e]), pmul(pr(cf, cg), pr(Ff[e], Fg[e]))));
                }
            }
        }
        __syncthreads();
    };

    // ---- prologue: the bottom rows of the first block's rings
    load_phi(-1, -4, 4);
    load_fg(-1, -2, 2, -1, 1);
    load_wait();
    mu_rows(-3, 3);
    p_rows(-2, 2, -2);
    r1_rows(-1, 1, -2, -1);

    // the ring shift: word k of the rows that move down by BY; the rows of a
    // ring are contiguous and 16-byte aligned, so they move in 16-byte words
    constexpr int PHB = (int)(sizeof(phi_t<T>) * 8 * L::W4 / 16);
    constexpr int MUB = (int)(sizeof(T) * 6 * L::W3 / 16);
    constexpr int PB = (int)(sizeof(T) * 4 * L::W2 / 16);
    constexpr int AB = (int)(sizeof(T) * 2 * L::W1 / 16);               // one aux plane
    constexpr int BB = (int)(sizeof(pair_t<T>) * 2 * L::W1 / 16);       // one bar-plus plane
    static_assert(sizeof(pair_t<T>) * BX % 16 == 0 && sizeof(phi_t<T>) * 8 * L::W4 % 16 == 0 &&
                      sizeof(T) * 6 * L::W3 % 16 == 0 && sizeof(T) * 4 * L::W2 % 16 == 0 &&
                      sizeof(T) * 2 * L::W1 % 16 == 0 && sizeof(T) * L::A1 % 16 == 0 &&
                      sizeof(T) * BY * L::W3 % 16 == 0 && sizeof(T) * BY * L::W2 % 16 == 0 &&
                      sizeof(T) * BY * L::W1 % 16 == 0 && sizeof(pair_t<T>) * SL::NFT % 16 == 0 &&
                      sizeof(pair_t<T>) * (SL::Y0 + (BY - 1) * BX) % 16 == 0,
                  "16-byte ring rows");
    constexpr int NPHI = PHB, NMU = NPHI + MUB, NP = NMU + PB, NAUX = NP + 7 * AB;
    constexpr int NALL = NAUX + Q * BB;
    auto shift_word = [&](int k) {
        float4 *d;
        const float4 *src;
        if (k < NPHI) {
            // the thread that moves a word down also refills it with the
            // next block's staged row
            float4 *up = (float4 *)(S.phi + BY * L::W4) + k;
            ((float4 *)S.phi)[k] = *up;
            *up = ((const float4 *)phst)[k];
            return;
        } else if (k < NMU) {
            d = (float4 *)S.mu + (k - NPHI);
            src = (const float4 *)(S.mu + BY * L::W3) + (k - NPHI);
        } else if (k < NP) {
            d = (float4 *)S.p + (k - NMU);
            src = (const float4 *)(S.p + BY * L::W2) + (k - NMU);
        } else if (k < NAUX) {
            const int pl = (k - NP) / AB, w = (k - NP) % AB;
            d = (float4 *)(S.gmx + pl * L::A1) + w;
            src = (const float4 *)(S.gmx + pl * L::A1 + BY * L::W1) + w;
        } else {
            const int q = (k - NAUX) / BB, w = (k - NAUX) % BB;
            d = (float4 *)(S.bp + q * L::A1) + w;
            src = (const float4 *)(S.bp + q * L::A1 + BY * L::W1) + w;
        }
        *d = *src;
    };
    const int x = tid % BX, y = tid / BX;
    for (int b = 0; b < nblk; b++) {
        // ---- the new rows of every region; those of a later block were
        // loaded during the block before
        if (b == 0) {
            load_phi(0, 4, BY + 4);
            load_fg(0, 1, BY + 2, 1, BY + 1);
            load_wait();
        }
        mu_rows(3, BY + 3);
        p_rows(2, BY + 2, 1);
        r1_rows(1, BY + 1, 1, 1);
        // the next block's new phi rows land while the faces and the update run
        if (b + 1 < nblk) {
            load_phi_next(b + 1);
            cp_commit();
        }
        // ---- faces: x faces of the block rows and y faces 0|1 .. BY-1|BY; the
        // first block also forms its bottom faces -1|0 (a wall face there
        // differences bar-plus up to row 1); later blocks carry them over
        const int nf = SL::NFT + (b == 0 ? BX : 0);
        for (int k = tid; k < nf; k += NT) {
            pair_t<T> F2o[6];
            if (k < SL::NXI) {
                const int xa = k % SL::XP - 1;
                if (xa >= BX) continue;                   // the idle item of an x-face row
                tile_face<T, 0, UNI>(I, S, xa, k / SL::XP, F2o);
            } else if (k < SL::Y0) {
                continue;
            } else if (k < SL::NFT) {
                tile_face<T, 1, UNI>(I, S, (k - SL::Y0) % BX, (k - SL::Y0) / BX, F2o);
            } else {
                tile_face<T, 1, UNI>(I, S, k - SL::NFT, -1, F2o);
            }
            pair_t<T> *dst = k < SL::NFT ? flux + k : keep0 + (k - SL::NFT);   // block 0: buffer 0
            const int stride = k < SL::NFT ? SL::NFT : BX;
#pragma unroll
            for (int m = 0; m < 6; m++) dst[m * stride] = F2o[m];
            if (k >= SL::NFT - BX && k < SL::NFT) {   // top row: also the next block's bottom faces
#pragma unroll
                for (int m = 0; m < 6; m++) keep0[((b + 1) & 1) * 6 * BX + m * BX + (k - (SL::NFT - BX))] = F2o[m];
            }
        }
        __syncthreads();
        // ---- update of the block's cell (Eqs. relations2, updatef)
        const int gi = i0 + x, gj = j0 + b * BY + y;
        if (tid < BX * BY && gi < I.nx && gj < I.ny) {
            pair_t<T> J[Q];
#pragma unroll
            for (int q = 0; q < Q; q++) J[q] = pr(T(0));
            const int kw = y * SL::XP + x, ke = kw + 1;       // faces x - 1 | x and x | x + 1
            const int kn = SL::Y0 + y * BX + x;               // face between rows y and y + 1
#pragma unroll
            for (int m = 0; m < 6; m++) {
                const int qx = xset(m), qy = yset(m);
                const pair_t<T> south = (y == 0) ? keep0[(b & 1) * 6 * BX + m * BX + x] : flux[m * SL::NFT + kn - BX];
                J[qx] = padd(J[qx], psub(flux[m * SL::NFT + ke], flux[m * SL::NFT + kw]));
                J[qy] = padd(J[qy], psub(flux[m * SL::NFT + kn], south));
            }
            const long long c = cell(gi, gj);
            const int r1 = TL::i1(x, y);
            const T dtv = fdiv(dt, S.c(10, 0, x) * S.c(10, 1, y));
            pair_t<T> nw[Q];
#pragma unroll
            for (int q = 0; q < Q; q++)
                nw[q] = pfma(pr(T(4.0 / 3.0)), S.bp[q * L::A1 + r1],
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
                const phi_t<T> phi = phi_add(S.phi[TL::i4(x, y)], -(dtv * jsum));
                io.phi_out[c] = phi;
                io.g_out[c] = phi_subt(phi, gsum);
                finite = finite && isfinite(phi_val(phi));
            }
            if (!finite) atomicOr(io.status + t.x, ST_NONFINITE);
        }
        // the threads that the update leaves idle shift the mu, p and aux
        // rings, which the update does not read
        constexpr int IDLE = NT - BX * BY;
        if constexpr (IDLE > 0) {
            if (tid >= BX * BY && b + 1 < nblk)
                for (int k = NPHI + (tid - BX * BY); k < NAUX; k += IDLE) shift_word(k);
        }
        cp_wait<0>();   // the next block's phi rows are in; the barrier makes them visible
        __syncthreads();
        if (b + 1 == nblk) break;
        // ---- the next block's tilde rows into the staging bytes (free once the
        // update has read the fluxes); while they are in flight, shift the
        // phi and bar-plus ring rows and the row geometry down by BY (a
        // uniform instance keeps its one row record) and write the new rows'
        // phi and geometry.
        load_fg(b + 1, 1, BY + 2, 1, BY + 1);
        cp_commit();
        // the phi and bar-plus rings (mu, p and the aux planes were shifted
        // during the update by the threads it leaves idle, if any)
        if constexpr (NT > BX * BY) {
            for (int k = tid; k < NPHI + (NALL - NAUX); k += NT) shift_word(k < NPHI ? k : k + (NAUX - NPHI));
        } else {
            for (int k = tid; k < NALL; k += NT) shift_word(k);
        }
        for (int r = tid; r < 8; r += NT) {
            S.gg[L::W4 + r] = S.gg[L::W4 + BY + r];
            if (!UNI) {
                S.gf[L::W4 + r] = S.gf[L::W4 + BY + r];
#pragma unroll
                for (int k = 0; k < 11; k++) S.ga[k * L::NG + L::W4 + r] = S.ga[k * L::NG + L::W4 + BY + r];
            }
            // the same thread then writes the geometry of the next block's new row r
            set_geo(L::W4 + 8 + r, false, 4 + r, grow(b + 1, 4 + r));
        }
        // the next block's tilde rows land during its mu (f) and p (g) phases
        __syncthreads();
    }
}

}  // namespace dugks
