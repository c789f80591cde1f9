// dugks_fused.cuh -- the whole DUGKS step (Sec. 2.2, steps 2-7) as one tiled
// kernel for sm_103a.
//
// A CTA owns a BX x BY tile of one instance and keeps everything it needs in
// shared memory, so the step reads the tracked state once and writes it once:
//   phase 1  phi on the tile plus a 4-cell ring                   (R4)
//   phase 2  mu = psi'(phi) - kappa lap(phi)                      (R3, Eq. chemicalpotential)
//   phase 3  p from f~ and F = -phi grad mu + F_b                 (R2, Eqs. u, P)
//   phase 4  grad p, tau_f, equilibria, sources, bar-plus         (R1, Eq. relations1)
//   phase 5  all faces of the tile, each once: reconstruction at t+h, face
//            macros, originals, flux                              (Eqs. fbar_h, conservedVariable
//                                                                  with h, original-function, microfluxf)
//   phase 6  tilde^{n+1} = 4/3 bar-plus - 1/3 tilde - dt/|V| J    (Eqs. relations2, updatef)
// Only the six flux-carrying directions of a face get equilibria, sources and
// originals.  The ring cells are recomputed by the neighbouring tiles instead
// of being written to and re-read from HBM; the state is double-buffered
// because tiles read the old state of their ring.
#pragma once
#include "dugks_kernels.cuh"

namespace dugks {

template <typename T>
struct StepIO {
    const T *f_in, *g_in;
    const phi_t<T> *phi_in;
    T *f_out, *g_out;
    phi_t<T> *phi_out;
    long long N;
    int *status;
};

template <typename T, int BX, int BY, bool SEP = false>
struct FusedLayout {
    static constexpr int W1 = BX + 2, H1 = BY + 2, A1 = W1 * H1;
    static constexpr int W2 = BX + 4, H2 = BY + 4, A2 = W2 * H2;
    static constexpr int W3 = BX + 6, H3 = BY + 6, A3 = W3 * H3;
    static constexpr int W4 = BX + 8, H4 = BY + 8, A4 = W4 * H4;
    static constexpr int NG = W4 + H4;                       // geometry entries (x then y)
    static constexpr int NFX = (BX + 1) * BY, NFY = BX * (BY + 1);
    // face items, in the order the threads take them and the flux buffer
    // stores them: the x faces on the pitch of the R1 planes (XP items a row,
    // the last one idle), so that a warp's faces read consecutive R1 entries
    // across a row change; then, from item Y0 (a whole number of warps), the
    // y faces one row of BX per warp.  Either way no warp reads two R1
    // entries of one shared-memory bank.
    static constexpr int XP = W1, NXI = XP * BY, Y0 = (NXI + 31) / 32 * 32, NFT = Y0 + NFY;
    static constexpr int NR1 = 7 + 18;                       // R1 planes
    static constexpr size_t al(size_t v) { return (v + 15) / 16 * 16; }
    static constexpr size_t o_geo = 0;                       // 11 T arrays + 2 int arrays of NG
    static constexpr size_t o_phi = al(o_geo + (sizeof(T) * 11 + sizeof(int) * 2) * NG);
    static constexpr size_t o_mu = al(o_phi + sizeof(phi_t<T>) * A4);
    static constexpr size_t o_p = al(o_mu + sizeof(T) * A3);
    static constexpr size_t o_r1 = al(o_p + sizeof(T) * A2);
    // tilde f on R2 and tilde g on R1 (phases 1-4); the face fluxes (phase
    // 5-6) reuse the same bytes once the bar-plus phase is done, unless SEP
    // gives them their own (then the update reads its tilde values here)
    static constexpr size_t o_un = al(o_r1 + sizeof(T) * NR1 * A1);
    static constexpr size_t un_fg = sizeof(T) * Q * (A2 + A1);
    static constexpr size_t un_flux = sizeof(T) * 12 * NFT;
    static constexpr size_t o_f = o_un;
    static constexpr size_t o_g = o_un + sizeof(T) * Q * A2;
    static constexpr size_t o_flux = SEP ? al(o_un + un_fg) : o_un;
    static constexpr size_t bytes = SEP ? al(o_flux + un_flux) : al(o_un + (un_fg > un_flux ? un_fg : un_flux));
};

// Asynchronous global -> shared copies (cp.async), grouped and awaited.
template <int BYTES>
__device__ __forceinline__ void cp_async(void *dst_smem, const void *src_gmem)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(src_gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Flux-carrying directions of x faces (cx != 0) and of y faces (cy != 0).
__host__ __device__ constexpr int xset(int k) { return k == 0 ? 1 : k == 1 ? 3 : k + 3; }   // 1,3,5,6,7,8
__host__ __device__ constexpr int yset(int k) { return k == 0 ? 2 : k == 1 ? 4 : k + 3; }   // 2,4,5,6,7,8
template <int A>
__host__ __device__ constexpr int fset(int k) { return A == 0 ? xset(k) : yset(k); }

// Geometry of one region position on one axis, read from the SoA arrays.
template <typename T>
struct G1 {
    T c1m, c1p, c2m, c2p, e1m, e10, e1p, wL, wR, invd, d;
    int g, om, op, lo, hi;
};

// Shared-memory views of one CTA.  UNI marks an instance whose spacing is
// uniform on each axis and whose axes are both periodic: every position then
// has the same geometry record (the records depend only on the spacings of a
// cell and its two neighbours), every neighbour exists, and there are no wall
// faces, so the accessors below return the record of position 0 and constant
// neighbour offsets.  The arithmetic is that of the general path, bit for bit.
template <typename T, int BX, int BY, bool UNI = false, bool SEP = false>
struct Tile {
    using L = FusedLayout<T, BX, BY, SEP>;
    T *ga;          // [11][NG] geometry coefficients, positions x -4..BX+3 then y -4..BY+3
    int *gg, *gf;   // [NG] global index (-1 outside), flags: 1 om=-1, 2 op=+1, 4 lo wall, 8 hi wall
    phi_t<T> *phi;  // R4
    pair_t<T> *flux;  // [6][NFT] (f, g) flux pairs by face item; unless SEP, aliases sf and sg (dead once phase 4 ends)
    T *mu;          // R3
    T *p;           // R2
    T *gmx, *gmy, *lmu, *gfx, *gfy, *gpx, *gpy;  // R1
    pair_t<T> *bp;  // [9][A1]: (f, g) bar-plus pairs
    T *sf;          // tilde f on R2 [Q][A2]
    T *sg;          // tilde g on R1 [Q][A1]
    __device__ Tile(unsigned char *sm)
    {
        ga = (T *)(sm + L::o_geo);
        gg = (int *)(ga + 11 * L::NG);
        gf = gg + L::NG;
        phi = (phi_t<T> *)(sm + L::o_phi);
        flux = (pair_t<T> *)(sm + L::o_flux);
        mu = (T *)(sm + L::o_mu);
        p = (T *)(sm + L::o_p);
        T *r1 = (T *)(sm + L::o_r1);
        gmx = r1; gmy = r1 + L::A1; lmu = r1 + 2 * L::A1; gfx = r1 + 3 * L::A1; gfy = r1 + 4 * L::A1;
        gpx = r1 + 5 * L::A1; gpy = r1 + 6 * L::A1;
        bp = (pair_t<T> *)(r1 + 7 * L::A1);
        sf = (T *)(sm + L::o_f);
        sg = (T *)(sm + L::o_g);
    }
    static __device__ __forceinline__ int i1(int x, int y) { return (y + 1) * L::W1 + (x + 1); }
    static __device__ __forceinline__ int i2(int x, int y) { return (y + 2) * L::W2 + (x + 2); }
    static __device__ __forceinline__ int i3(int x, int y) { return (y + 3) * L::W3 + (x + 3); }
    static __device__ __forceinline__ int i4(int x, int y) { return (y + 4) * L::W4 + (x + 4); }
    // entry of x position x (axis 0) or y position y (axis 1)
    static __device__ __forceinline__ int ge(int axis, int pos) { return axis == 0 ? pos + 4 : L::W4 + pos + 4; }
    __device__ __forceinline__ int gidx(int axis, int pos) const { return gg[ge(axis, pos)]; }
    // position inside the domain (always, on a periodic axis)
    __device__ __forceinline__ bool ok(int axis, int pos) const { return UNI || gg[ge(axis, pos)] >= 0; }
    __device__ __forceinline__ G1<T> geo(int axis, int pos) const
    {
        const int e = ge(axis, pos);
        G1<T> G;
        G.c1m = ga[0 * L::NG + e]; G.c1p = ga[1 * L::NG + e]; G.c2m = ga[2 * L::NG + e]; G.c2p = ga[3 * L::NG + e];
        G.e1m = ga[4 * L::NG + e]; G.e10 = ga[5 * L::NG + e]; G.e1p = ga[6 * L::NG + e];
        G.wL = ga[7 * L::NG + e]; G.wR = ga[8 * L::NG + e]; G.invd = ga[9 * L::NG + e]; G.d = ga[10 * L::NG + e];
        const int f = gf[e];
        G.g = gg[e];
        G.om = (f & 1) ? -1 : 0;
        G.op = (f & 2) ? 1 : 0;
        G.lo = (f >> 2) & 1;
        G.hi = (f >> 3) & 1;
        return G;
    }
    __device__ __forceinline__ int om(int axis, int pos) const { return UNI ? -1 : (gf[ge(axis, pos)] & 1) ? -1 : 0; }
    __device__ __forceinline__ int op(int axis, int pos) const { return UNI ? 1 : (gf[ge(axis, pos)] & 2) ? 1 : 0; }
    __device__ __forceinline__ T c(int k, int axis, int pos) const { return ga[k * L::NG + ge(axis, UNI ? 0 : pos)]; }
    // index step from row y to row y + d of the R1 planes
    __device__ __forceinline__ int rs1(int y, int d) const { return d * L::W1; }
    // position of item r of a phase over the H rows of a ring of radius R
    // (width BX + 2R) starting at row y0: the first H * BX items one row of BX
    // (a warp) each, then the 2R right-hand columns of every row, so that a
    // warp reads one row of every ring and no two of its lanes hit one
    // shared-memory bank
    static __device__ __forceinline__ void ring_item(int r, int H, int R, int y0, int &x, int &y)
    {
        if (r < H * BX) {
            x = r % BX - R;
            y = y0 + r / BX;
        } else {
            const int k = r - H * BX;
            x = BX - R + k % (2 * R);
            y = y0 + k / (2 * R);
        }
    }
};

// Face macroscopic variables from the nine bar distributions of each kind at
// t+h (Eq. conservedVariable with h, bar for tilde), then the originals of
// Eq. (original-function) of the six flux-carrying directions of axis A,
// returned as (xi . e_A) phi_i |S|.
template <typename T, int A>
__device__ __forceinline__ void face_tail(const InstDev &I, const T (&fb)[Q], const T (&gb)[Q], const FaceAux<T> &ax,
                                          bool wall, int side, T area, pair_t<T> (&F2o)[6])
{
    const ParT<T> &Pr = par<T>(I);
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
    const T irho = fdiv(T(1), s.rho);
    s.Fx = -phi * ax.gmux + (s.rho - Pr.rho_ref) * Pr.gxa;
    s.Fy = -phi * ax.gmuy + (s.rho - Pr.rho_ref) * Pr.gya;
    s.grx = Pr.drho * ax.gphix;
    s.gry = Pr.drho * ax.gphiy;
    if (wall) {
        s.ux = 0;
        s.uy = 0;
    } else {
        // (sum xi f + h/2 c_s^2 F) / (c_s^2 rho)
        s.ux = (T(3) * mx + T(0.5) * h * s.Fx) * irho;
        s.uy = (T(3) * my + T(0.5) * h * s.Fy) * irho;
    }
    s.p = sf + T(0.5) * h * Cst<T>::cs2 * (s.ux * s.grx + s.uy * s.gry - Pr.gamma * s.rho * Pr.lambda * ax.lapmu);
    s.mu = ax.mu;
    s.lapmu = ax.lapmu;
    s.gpx = ax.gpx;
    s.gpy = ax.gpy;
    const PtInv<T> v = pt_inv<T>(I, s);
    T a1, b1, c1;
    face_weights<T>(Pr, phi, s.rho, a1, b1, c1);
    // the g weights (Eq. original-function with h), formed here rather than
    // loaded, which keeps fewer values live
    const T tg = Pr.tau_g, r2 = fdiv(T(1), T(2) * tg + h);
    const pair_t<T> ca2 = pr(a1, T(2) * tg * r2), cb2 = pr(b1, h * r2), cc2 = pr(c1, tg * h * r2);
    pair_t<T> o[Q];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        // the six directions as three opposite pairs; at a wall the incoming
        // originals are formed too but replaced by bounce-back below
        const int q = k == 0 ? fset<A>(0) : k + 4;   // 1|3 or 2|4, 5|7, 6|8
        T feq[2], geq[2], F1[2], F2[2];
        eq_src2<T>(s, v, q, feq, geq, F1, F2);
        o[q] = pfma(ca2, pr(fb[q], gb[q]), pfma(cb2, pr(feq[0], geq[0]), pmul(cc2, pr(F1[0], F2[0]))));
        const int r = opp(q);
        o[r] = pfma(ca2, pr(fb[r], gb[r]), pfma(cb2, pr(feq[1], geq[1]), pmul(cc2, pr(F1[1], F2[1]))));
    }
#pragma unroll
    for (int k = 0; k < 6; k++) {
        const int q = fset<A>(k);
        const pair_t<T> vo = (wall && ca(q, A) * side < 0) ? o[opp(q)] : o[q];
        F2o[k] = pmul(pr(T(ca(q, A)) * area), vo);
    }
}

// Flux values of the face between positions a (low side) and b = a + e_A of a
// tile, or of the wall face of whichever of the two lies in the domain.
template <typename T, int A, bool UNI, typename TL>
__device__ __forceinline__ void tile_face(const InstDev &I, const TL &S, int xa, int ya, pair_t<T> (&F2o)[6])
{
    const ParT<T> &Pr = par<T>(I);
    constexpr int A1 = TL::L::A1;
    const int xb = xa + (A == 0 ? 1 : 0), yb = ya + (A == 1 ? 1 : 0);
    const int pa = A == 0 ? xa : ya, pb = A == 0 ? xb : yb, pt = A == 0 ? ya : xa;
#pragma unroll
    for (int k = 0; k < 6; k++) F2o[k] = pr(T(0));
    if (!S.ok(1 - A, pt)) return;
    const bool va = S.ok(A, pa), vb = S.ok(A, pb);
    const T h = Pr.h;
    const T area = S.c(10, 1 - A, pt);
    const T te1m = S.c(4, 1 - A, pt), te10 = S.c(5, 1 - A, pt), te1p = S.c(6, 1 - A, pt);
    // tangential neighbours: a row step for x faces, a column step for y faces
    const int tm = A == 0 ? S.rs1(pt, S.om(1, pt)) : S.om(0, pt);
    const int tp = A == 0 ? S.rs1(pt, S.op(1, pt)) : S.op(0, pt);
    T fb[Q], gb[Q];
    FaceAux<T> ax;
    if (UNI || (va && vb)) {
        const int ia = S.i1(xa, ya), ib = S.i1(xb, yb);
        const T wL = S.c(7, A, pa), wR = S.c(8, A, pa), invd = S.c(9, A, pa);
#pragma unroll
        for (int q = 0; q < Q; q++) {
            // (wL bL + wR bR) - h xi_A (bR - bL) / d - h xi_t (wL tL + wR tR), for f and g at once
            const pair_t<T> *B = S.bp + q * A1;
            const pair_t<T> bL = B[ia], bR = B[ib];
            const T k1 = h * T(ca(q, A)) * invd;
            pair_t<T> v = pfma(pr(wL + k1), bL, pmul(pr(wR - k1), bR));
            if (ca(q, 1 - A)) {
                // the centre weight is exactly 0 on a uniform periodic axis
                const pair_t<T> tL = UNI ? pfma(pr(te1m), B[ia + tm], pmul(pr(te1p), B[ia + tp]))
                                         : pfma(pr(te1m), B[ia + tm], pfma(pr(te10), bL, pmul(pr(te1p), B[ia + tp])));
                const pair_t<T> tR = UNI ? pfma(pr(te1m), B[ib + tm], pmul(pr(te1p), B[ib + tp]))
                                         : pfma(pr(te1m), B[ib + tm], pfma(pr(te10), bR, pmul(pr(te1p), B[ib + tp])));
                const T kt = -h * T(ca(q, 1 - A));
                v = pfma(pr(kt * wL), tL, pfma(pr(kt * wR), tR, v));
            }
            fb[q] = v.x;
            gb[q] = v.y;
        }
        const int ma = S.i3(xa, ya), mb = S.i3(xb, yb);
        ax.mu = wL * S.mu[ma] + wR * S.mu[mb];
        ax.lapmu = wL * S.lmu[ia] + wR * S.lmu[ib];
        ax.gmux = wL * S.gmx[ia] + wR * S.gmx[ib];
        ax.gmuy = wL * S.gmy[ia] + wR * S.gmy[ib];
        ax.gphix = wL * S.gfx[ia] + wR * S.gfx[ib];
        ax.gphiy = wL * S.gfy[ia] + wR * S.gfy[ib];
        ax.gpx = wL * S.gpx[ia] + wR * S.gpx[ib];
        ax.gpy = wL * S.gpy[ia] + wR * S.gpy[ib];
        face_tail<T, A>(I, fb, gb, ax, false, 0, area, F2o);
        return;
    }
    int side, xc, yc, pc;
    if (!va && vb && (S.gf[S.ge(A, pb)] & 4)) { side = -1; xc = xb; yc = yb; pc = pb; }
    else if (va && !vb && (S.gf[S.ge(A, pa)] & 8)) { side = +1; xc = xa; yc = ya; pc = pa; }
    else return;
    // wall face of cell c: Taylor reconstruction from the cell centre for the
    // outgoing and parallel directions, bounce-back for the incoming ones
    const int ic = S.i1(xc, yc);
    const int nm = A == 0 ? S.om(0, pc) : S.rs1(yc, S.om(1, pc));
    const int np = A == 0 ? S.op(0, pc) : S.rs1(yc, S.op(1, pc));
    const T ne1m = S.c(4, A, pc), ne10 = S.c(5, A, pc), ne1p = S.c(6, A, pc);
    const T half_d = T(0.5) * S.c(10, A, pc);
#pragma unroll
    for (int q = 0; q < Q; q++) {
        if (ca(q, A) * side < 0) continue;
        const T off = T(side) * half_d - h * T(ca(q, A));
        const T ht = h * T(ca(q, 1 - A));
        const pair_t<T> *B = S.bp + q * A1;
        const pair_t<T> b = B[ic];
        const pair_t<T> dn = pfma(pr(ne1m), B[ic + nm], pfma(pr(ne10), b, pmul(pr(ne1p), B[ic + np])));
        const pair_t<T> dtg = pfma(pr(te1m), B[ic + tm], pfma(pr(te10), b, pmul(pr(te1p), B[ic + tp])));
        const pair_t<T> v = pfma(pr(-ht), dtg, pfma(pr(off), dn, b));
        fb[q] = v.x;
        gb[q] = v.y;
    }
#pragma unroll
    for (int q = 0; q < Q; q++) {
        if (ca(q, A) * side < 0) {
            fb[q] = fb[opp(q)];
            gb[q] = gb[opp(q)];
        }
    }
    ax.mu = S.mu[S.i3(xc, yc)];
    ax.lapmu = S.lmu[ic];
    ax.gmux = A == 0 ? T(0) : S.gmx[ic];
    ax.gmuy = A == 1 ? T(0) : S.gmy[ic];
    ax.gphix = A == 0 ? T(0) : S.gfx[ic];
    ax.gphiy = A == 1 ? T(0) : S.gfy[ic];
    ax.gpx = A == 0 ? T(0) : S.gpx[ic];
    ax.gpy = A == 1 ? T(0) : S.gpy[ic];
    face_tail<T, A>(I, fb, gb, ax, true, side, area, F2o);
}

// NT threads (a multiple of 32, at least BX * BY) share the phases of a
// BX x BY tile; the first BX * BY of them own one cell each in the update.
template <typename T, int BX, int BY, int NT, int MINB, bool UNI, bool SEP>
__global__ void __launch_bounds__(NT, MINB) k_step(const InstDev *__restrict__ insts, const int4 *__restrict__ tiles,
                                                   const AxisRecT<T> *__restrict__ geo, StepIO<T> io)
{
    static_assert(NT % 32 == 0 && NT >= BX * BY, "thread count");
    using TL = Tile<T, BX, BY, UNI, SEP>;
    using L = typename TL::L;
    extern __shared__ __align__(16) unsigned char smem[];
    TL S(smem);
    const int4 t = tiles[blockIdx.x];
    const InstDev &I = insts[t.x];
    const ParT<T> &Pr = par<T>(I);
    const int i0 = t.y, j0 = t.z;
    const int tid = threadIdx.x;
    {
        const int st = io.status[t.x];
        if (st & ST_NONFINITE) return;   // masked: non-finite instance of a batch
        if (st & ST_PAUSED) {            // paused: the state passes to the other buffer unchanged
            const int x = tid % BX, y = tid / BX;
            if (tid < BX * BY && i0 + x < I.nx && j0 + y < I.ny) {
                const long long c = I.cell0 + (long long)(j0 + y) * I.nxp + (i0 + x);
#pragma unroll
                for (int q = 0; q < Q; q++) {
                    io.f_out[q * io.N + c] = io.f_in[q * io.N + c];
                    io.g_out[q * io.N + c] = io.g_in[q * io.N + c];
                }
                io.phi_out[c] = io.phi_in[c];
            }
            return;
        }
    }
    const long long N = io.N;

    // global index of every region column and row (wrapped on periodic axes,
    // -1 outside the domain), kept in shared memory for all later phases
    for (int r = tid; r < L::NG; r += NT) {
        const bool isx = r < L::W4;
        const int n = isx ? I.nx : I.ny;
        int g = (isx ? i0 : j0) + (isx ? r - 4 : r - L::W4 - 4);
        if ((isx ? I.bcx : I.bcy) == 0) {
            while (g < 0) g += n;
            while (g >= n) g -= n;
        } else if (g < 0 || g >= n) {
            g = -1;
        }
        S.gg[r] = g;
    }
    __syncthreads();
    auto gpos = [&](bool isx, int pos) -> int { return S.gg[isx ? pos + 4 : L::W4 + pos + 4]; };
    auto cell = [&](int gi, int gj) -> long long { return I.cell0 + (long long)gj * I.nxp + gi; };

    // ---- phase 1: asynchronous copies of phi (R4), then of tilde f (R2) and
    // tilde g (R1); positions outside the domain are zero-filled.  They are
    // issued first so that their latency overlaps the geometry set-up.
    for (int r = tid; r < L::A4; r += NT) {
        const int gi = gpos(true, r % L::W4 - 4), gj = gpos(false, r / L::W4 - 4);
        if (UNI || (gi >= 0 && gj >= 0)) {
            cp_async<sizeof(phi_t<T>)>(S.phi + r, io.phi_in + cell(gi, gj));
        } else {
            phi_t<T> v;
            phi_from_zero(v);
            S.phi[r] = v;
        }
    }
    cp_commit();
    for (int r = tid; r < L::A2; r += NT) {
        const int gi = gpos(true, r % L::W2 - 2), gj = gpos(false, r / L::W2 - 2);
        if (UNI || (gi >= 0 && gj >= 0)) {
            const long long c = cell(gi, gj);
#pragma unroll
            for (int q = 0; q < Q; q++) cp_async<sizeof(T)>(S.sf + q * L::A2 + r, io.f_in + q * N + c);
        } else {
#pragma unroll
            for (int q = 0; q < Q; q++) S.sf[q * L::A2 + r] = T(0);
        }
    }
    for (int r = tid; r < L::A1; r += NT) {
        const int gi = gpos(true, r % L::W1 - 1), gj = gpos(false, r / L::W1 - 1);
        if (UNI || (gi >= 0 && gj >= 0)) {
            const long long c = cell(gi, gj);
#pragma unroll
            for (int q = 0; q < Q; q++) cp_async<sizeof(T)>(S.sg + q * L::A1 + r, io.g_in + q * N + c);
        } else {
#pragma unroll
            for (int q = 0; q < Q; q++) S.sg[q * L::A1 + r] = T(0);
        }
    }
    cp_commit();

    // ---- geometry of the region columns and rows (SoA)
    for (int r = tid; r < L::NG; r += NT) {
        const bool isx = r < L::W4;
        const int pos = isx ? r - 4 : r - L::W4 - 4;
        const int g = S.gg[r];
        if (UNI && pos != 0) continue;   // every position carries the record of position 0
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
    }
    cp_wait<1>();   // phi has landed
    __syncthreads();

    // ---- phase 2: mu on R3 (Eq. chemicalpotential), differences of the stored phi
    for (int r = tid; r < L::A3; r += NT) {
        int x, y;
        TL::ring_item(r, L::H3, 3, -3, x, y);
        T mu = 0;
        if (S.ok(0, x) && S.ok(1, y)) {
            const phi_t<T> p0 = S.phi[TL::i4(x, y)];
            const T lap = (S.c(2, 0, x) * phi_sub(S.phi[TL::i4(x + S.om(0, x), y)], p0)
                         + S.c(3, 0, x) * phi_sub(S.phi[TL::i4(x + S.op(0, x), y)], p0))
                        + (S.c(2, 1, y) * phi_sub(S.phi[TL::i4(x, y + S.om(1, y))], p0)
                         + S.c(3, 1, y) * phi_sub(S.phi[TL::i4(x, y + S.op(1, y))], p0));
            const T dpsi = T(4) * Pr.beta * phi_subc(p0, I.cA)
                         * phi_subc(p0, I.cB)
                         * phi_subc(p0, I.cM);
            mu = dpsi - Pr.kappa * lap;
        }
        S.mu[TL::i3(x, y)] = mu;
    }
    cp_wait<0>();   // tilde f and g have landed
    __syncthreads();

    const T hdt = T(0.5) * Pr.dt;
    const T cs2 = Cst<T>::cs2;
    // ---- phase 3: p on R2 (Eqs. u, P); needs grad mu, lap mu, grad phi and f~
    for (int r = tid; r < L::A2; r += NT) {
        int x, y;
        TL::ring_item(r, L::H2, 2, -2, x, y);
        const int k2 = TL::i2(x, y);
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
            T sf = 0, mx = 0, my = 0;
#pragma unroll
            for (int q = 0; q < Q; q++) {
                const T v = S.sf[q * L::A2 + k2];
                sf += v;
                if (cx(q)) mx += T(cx(q)) * v;
                if (cy(q)) my += T(cy(q)) * v;
            }
            const T irho = fdiv(T(1), rho);
            const T ux = (T(3) * mx + hdt * Fx) * irho;
            const T uy = (T(3) * my + hdt * Fy) * irho;
            vp = sf + hdt * cs2 * (ux * Pr.drho * gfx + uy * Pr.drho * gfy - Pr.gamma * rho * Pr.lambda * lmu);
        }
        S.p[k2] = vp;
    }
    __syncthreads();

    // ---- phase 4: grad p, u and bar-plus of both distributions on R1 (Eq. relations1)
    const T dt = Pr.dt;
    const T ag = Pr.gca, bg = Pr.gcb, cg = Pr.gcc;
    for (int r = tid; r < L::A1; r += NT) {
        int x, y;
        TL::ring_item(r, L::H1, 1, -1, x, y);
        const int k1 = TL::i1(x, y);
        if (!S.ok(0, x) || !S.ok(1, y)) {
            S.gmx[k1] = 0; S.gmy[k1] = 0; S.lmu[k1] = 0; S.gfx[k1] = 0; S.gfy[k1] = 0; S.gpx[k1] = 0; S.gpy[k1] = 0;
#pragma unroll
            for (int q = 0; q < Q; q++) S.bp[q * L::A1 + k1] = pr(T(0));
            continue;
        }
        const int k2 = TL::i2(x, y);
        const T p0 = S.p[k2];
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
        T fv[Q];
        T mx = 0, my = 0;
#pragma unroll
        for (int q = 0; q < Q; q++) {
            fv[q] = S.sf[q * L::A2 + k2];
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
                S.bp[qq * L::A1 + k1] = pfma(pr(af, ag), pr(fv[qq], S.sg[qq * L::A1 + k1]),
                                            pfma(pr(bf, bg), pr(feq[e], geq[e]), pmul(pr(cf, cg), pr(Ff[e], Fg[e]))));
            }
        }
    }
    __syncthreads();

    const int x = tid % BX, y = tid / BX;
    const int gi = i0 + x, gj = j0 + y;
    const bool own = tid < BX * BY && gi < I.nx && gj < I.ny;
    const long long c = own ? cell(gi, gj) : 0;

    // ---- phase 5: every face of the tile once (x faces first in the item space)
    for (int k = tid; k < L::NFT; k += NT) {
        pair_t<T> F2o[6];
        if (k < L::NXI) {
            const int xa = k % L::XP - 1;
            if (xa >= BX) continue;                       // the idle item of an x-face row
            tile_face<T, 0, UNI>(I, S, xa, k / L::XP, F2o);
        } else if (k < L::Y0) {
            continue;
        } else {
            tile_face<T, 1, UNI>(I, S, (k - L::Y0) % BX, (k - L::Y0) / BX - 1, F2o);
        }
#pragma unroll
        for (int m = 0; m < 6; m++) S.flux[m * L::NFT + k] = F2o[m];
    }
    __syncthreads();

    // ---- phase 6: update of the tile cell (Eqs. relations2, updatef)
    if (!own) return;
    // J of both kinds at once: east minus west for the x set, north minus south for the y set
    pair_t<T> J[Q];
#pragma unroll
    for (int q = 0; q < Q; q++) J[q] = pr(T(0));
    {
        const int kw = y * L::XP + x, ke = kw + 1;                    // west and east faces
        const int ks = L::Y0 + y * BX + x, kn = ks + BX;             // south and north faces
#pragma unroll
        for (int m = 0; m < 6; m++) {
            const int qx = xset(m), qy = yset(m);
            J[qx] = padd(J[qx], psub(S.flux[m * L::NFT + ke], S.flux[m * L::NFT + kw]));
            J[qy] = padd(J[qy], psub(S.flux[m * L::NFT + kn], S.flux[m * L::NFT + ks]));
        }
    }
    const int r1 = TL::i1(x, y);
    const T dtv = fdiv(dt, S.c(10, 0, x) * S.c(10, 1, y));
    // tilde^{n+1} = 4/3 bar-plus - 1/3 tilde - dt/|V| J
    pair_t<T> nw[Q];
    const int r2 = TL::i2(x, y);
#pragma unroll
    for (int q = 0; q < Q; q++) {
        // the cell's own tilde values: still in shared memory with SEP, else an L2 hit (read in phase 1)
        const pair_t<T> old = SEP ? pr(S.sf[q * L::A2 + r2], S.sg[q * L::A1 + r1]) : pr(io.f_in[q * N + c], io.g_in[q * N + c]);
        nw[q] = pfma(pr(T(4.0 / 3.0)), S.bp[q * L::A1 + r1], pfma(pr(T(-1.0 / 3.0)), old, pmul(pr(-dtv), J[q])));
    }
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
        // sum_i g~+_i = phi exactly, so phi advances by the flux balance alone
        // (kept as a float pair); the rest distribution g~_0 is rebuilt from it
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
    if (!finite) atomicOr(io.status + t.x, 1);
}

}  // namespace dugks
