/*
 * dugks_oracle.c -- plain, slow, FP64 CPU oracle of the two-phase DUGKS step
 * (Zhang, Yang & Guo, "A discrete unified gas-kinetic scheme for immiscible
 * two-phase flows", Sec. 2.2).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this file.  It shares no code, header,
 * table or helper with the CUDA library; it is written from the paper's
 * equations, in the paper's order (the seven steps of the procedure at the end
 * of Sec. 2.2), with cell loops that a reader can check by eye.
 *
 * Notation follows the paper: f_i carries the pressure and momentum, g_i the
 * order parameter phi (Eqs. bgkf, bgkg, phiup).  The tracked state is the pair
 * of "tilde" distributions (Eq. auxf a); everything else is recomputed from it
 * every step.  Arrays are [Q][ny][nx], x fastest.
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *  - face values of phi-bar-plus: linear interpolation between the two cell
 *    centres; normal derivative = two-point difference; tangential derivative
 *    = the same interpolation of the cells' tangential derivatives (Eq. nonphi);
 *  - face values of mu, lap(mu) and of the gradients of mu, p, phi: the same
 *    linear interpolation of cell values at t_n;
 *  - face macroscopic variables: Eq. conservedVariable with h for dt and the
 *    bar distributions for the tilde ones;
 *  - gradient ghosts at walls for phi, mu, p: mirror ghost (zero normal
 *    gradient); for the distributions: one-sided two-point difference;
 *  - walls: bounce-back of the bar distributions and of the original
 *    distributions at the wall face, wall velocity zero;
 *  - body force F_b = (rho - rho_ref) g;  eta = lambda / (c_s^2 tau_g).
 *
 * Compiled with -ffp-contract=off so that x86 and Arm give the same bits.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* The arithmetic type.  The default build is plain double.  Built with
 * -DORACLE_COMPLEX the same code runs in double complex arithmetic, which
 * gives exact first derivatives by the complex step: perturb an input by
 * i*eps (eps ~ 1e-30) and read d(output)/d(input) = Im(output)/eps, free of
 * subtractive cancellation.  Mesh geometry stays real in both builds. */
#ifdef ORACLE_COMPLEX
#include <complex.h>
typedef double complex real;
#define FINITE(x) (isfinite(creal(x)) && isfinite(cimag(x)))
#define creal_or_same(x) creal(x)
#else
typedef double real;
#define FINITE(x) isfinite(x)
#define creal_or_same(x) (x)
#endif

#define Q 9
#define BC_PERIODIC 0
#define BC_WALL 1

/* D2Q9 velocities, Eq. (D2Q9) with c = sqrt(3RT) = 1:
   0: rest; 1-4: (cos,sin) of (i-1)pi/2; 5-8: sqrt(2)(cos,sin) of (i-5)pi/2+pi/4 */
static const int XI[Q][2] = {{0, 0}, {1, 0}, {0, 1}, {-1, 0}, {0, -1},
                             {1, 1}, {-1, 1}, {-1, -1}, {1, -1}};
/* weights omega_i (Sec. 2.2, after Eq. Hi) */
static const double WT[Q] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
/* opposite direction (bounce-back) */
static const int OPP[Q] = {0, 3, 4, 1, 2, 7, 8, 5, 6};

/* RT = c_s^2 = 1/3 in all the paper's runs (start of Sec. 3) */
static const double CS2 = 1.0 / 3.0;

typedef struct {
    int nx, ny;
    int bc[2];
    double *d[2];    /* cell widths along x (nx) and y (ny) */
    /* parameters */
    real phiA, phiB, rhoA, rhoB, nuA, nuB, lambda, tau_g, beta, kappa, gx, gy, rho_ref;
    double cfl;
    /* derived */
    double dt, h;
    real eta, gamma, muA, muB;
    /* tracked state: tilde distributions */
    real *f, *g;
    /* per-cell macroscopic fields at t_n */
    real *phi, *rho, *lap_phi, *mu, *lap_mu, *gphi[2], *gmu[2], *F[2], *u[2], *p, *gp[2], *tauf;
    /* per-cell bar-plus and tilde-plus distributions (step 2) */
    real *fbp, *gbp, *ftp, *gtp;
    /* flux accumulators J (Eq. microfluxf) */
    real *Jf, *Jg;
} osim;

static inline int IDX(const osim *s, int i, int j) { return j * s->nx + i; }

/* ------------------------------------------------------------------------- */
/* Model relations                                                            */
/* ------------------------------------------------------------------------- */

/* Eq. (oderrho): density linear in phi */
static real rho_of(const osim *s, real phi)
{
    return (phi - s->phiB) / (s->phiA - s->phiB) * s->rhoA + (s->phiA - phi) / (s->phiA - s->phiB) * s->rhoB;
}

/* Eq. (mixvis) mixed dynamic viscosity, then nu = mu/rho and tau_f = nu/c_s^2
   (Eq. kineticandmobility) */
static real tauf_of(const osim *s, real phi, real rho)
{
    real mu = s->muA * s->muB * (s->phiA - s->phiB) / ((phi - s->phiB) * s->muB + (s->phiA - phi) * s->muA);
    real nu = mu / rho;
    return nu / CS2;
}

/* Eq. (chemicalpotential), bulk part psi'(phi) */
static real dpsi(const osim *s, real phi)
{
    return 4.0 * s->beta * (phi - s->phiA) * (phi - s->phiB) * (phi - 0.5 * (s->phiA + s->phiB));
}

/* Eq. (su) */
static real s_i(int i, real ux, real uy)
{
    real xu = XI[i][0] * ux + XI[i][1] * uy;
    real uu = ux * ux + uy * uy;
    return WT[i] * (xu / CS2 + xu * xu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
}

/* Eq. (feq): f_i^eq = omega_i p + c_s^2 rho s_i(u) */
void oracle_feq(real p, real rho, real ux, real uy, real *out)
{
    for (int i = 0; i < Q; i++) out[i] = WT[i] * p + CS2 * rho * s_i(i, ux, uy);
}

/* Eqs. (geq), (Hi): g_i^eq = H_i + phi s_i(u) */
void oracle_geq(real phi, real mu, real eta, real ux, real uy, real *out)
{
    for (int i = 0; i < Q; i++) {
        real H = (i == 0) ? phi - (1.0 - WT[0]) * eta * mu : WT[i] * eta * mu;
        out[i] = H + phi * s_i(i, ux, uy);
    }
}

/* Eq. (F): F_i^f = (xi_i - u).[F Gamma_i + s_i c_s^2 grad rho] - omega_i c_s^2 rho gamma div(lambda grad mu),
   with Gamma_i = omega_i + s_i and div(lambda grad mu) = lambda lap(mu) (constant lambda) */
void oracle_src_f(real ux, real uy, real Fx, real Fy, real grx, real gry, real rho,
                  real gamma, real lambda, real lap_mu, real *out)
{
    for (int i = 0; i < Q; i++) {
        real si = s_i(i, ux, uy);
        real Gi = WT[i] + si;
        real cx = XI[i][0] - ux, cy = XI[i][1] - uy;
        out[i] = cx * (Fx * Gi + si * CS2 * grx) + cy * (Fy * Gi + si * CS2 * gry)
               - WT[i] * CS2 * rho * gamma * lambda * lap_mu;
    }
}

/* Eq. (G): F_i^g = phi/(c_s^2 rho) (xi_i - u).(F - grad p) Gamma_i */
void oracle_src_g(real phi, real rho, real ux, real uy, real Fx, real Fy, real gpx,
                  real gpy, real *out)
{
    for (int i = 0; i < Q; i++) {
        real Gi = WT[i] + s_i(i, ux, uy);
        real cx = XI[i][0] - ux, cy = XI[i][1] - uy;
        out[i] = phi / (CS2 * rho) * (cx * (Fx - gpx) + cy * (Fy - gpy)) * Gi;
    }
}

/* Eq. (relations1): cell-centre bar-plus from the tilde distribution */
real oracle_bar_plus(real tilde, real eq, real src, real tau, double dt)
{
    double h = 0.5 * dt;
    return (2.0 * tau - h) / (2.0 * tau + dt) * tilde + 3.0 * h / (2.0 * tau + dt) * eq
         + 3.0 * tau * h / (2.0 * tau + dt) * src;
}

/* Eq. (relations2) */
real oracle_tilde_plus(real bar_plus, real tilde)
{
    return 4.0 / 3.0 * bar_plus - 1.0 / 3.0 * tilde;
}

/* Eq. (original-function): original distribution from the bar one at t+h */
real oracle_original(real bar, real eq, real src, real tau, double h)
{
    return 2.0 * tau / (2.0 * tau + h) * bar + h / (2.0 * tau + h) * eq + tau * h / (2.0 * tau + h) * src;
}

/* ------------------------------------------------------------------------- */
/* Mesh neighbours and the non-uniform differences of Eqs. (nonphi), (nonphi2) */
/* ------------------------------------------------------------------------- */

/* Neighbour of index k on axis a on side (-1 / +1).  Returns 1 for a real
   (possibly periodic) cell, 0 for a wall ghost; *dist is the distance between
   the two centres.  The wall ghost is the cell mirrored about the wall: its
   centre lies d[k] away and it carries the same index. */
static int neighbour(const osim *s, int a, int k, int side, int *kn, double *dist)
{
    int n = a == 0 ? s->nx : s->ny;
    const double *d = s->d[a];
    int k2 = k + side;
    if (k2 >= 0 && k2 < n) {
        *kn = k2;
        *dist = 0.5 * (d[k] + d[k2]);
        return 1;
    }
    if (s->bc[a] == BC_PERIODIC) {
        k2 = (k2 + n) % n;
        *kn = k2;
        *dist = 0.5 * (d[k] + d[k2]);
        return 1;
    }
    *kn = k;
    *dist = d[k];
    return 0;
}

/* value of field Fd at the cell reached from (i,j) by moving to index k on axis a */
static real at(const osim *s, const real *Fd, int a, int i, int j, int k)
{
    return a == 0 ? Fd[IDX(s, k, j)] : Fd[IDX(s, i, k)];
}

/* Eq. (nonphi): first derivative along axis a with theta_l, theta_r, a, b, c;
   delta is the mean of the two step lengths (any delta gives the same value) */
static real nonphi(real Fm, real F0, real Fp, double dl, double dr)
{
    double delta = 0.5 * (dl + dr);
    double tl = dl / delta, tr = dr / delta;
    double A = tl * tr, B = tl + tr, C = tr - tl;
    return (tl * tl * Fp + B * C * F0 - tr * tr * Fm) / (A * B * delta);
}

/* Eq. (nonphi2): second derivative along axis a */
static real nonphi2(real Fm, real F0, real Fp, double dl, double dr)
{
    double delta = 0.5 * (dl + dr);
    double tl = dl / delta, tr = dr / delta;
    double A = tl * tr, B = tl + tr;
    return 2.0 / (A * B * delta * delta) * (tl * Fp - B * F0 + tr * Fm);
}

/* derivative of a macroscopic cell field along axis a, mirror ghosts at walls */
static real d1_field(const osim *s, const real *Fd, int a, int i, int j)
{
    int k = a == 0 ? i : j, km, kp;
    double dl, dr;
    neighbour(s, a, k, -1, &km, &dl);
    neighbour(s, a, k, +1, &kp, &dr);
    return nonphi(at(s, Fd, a, i, j, km), Fd[IDX(s, i, j)], at(s, Fd, a, i, j, kp), dl, dr);
}

static real d2_field(const osim *s, const real *Fd, int a, int i, int j)
{
    int k = a == 0 ? i : j, km, kp;
    double dl, dr;
    neighbour(s, a, k, -1, &km, &dl);
    neighbour(s, a, k, +1, &kp, &dr);
    return nonphi2(at(s, Fd, a, i, j, km), Fd[IDX(s, i, j)], at(s, Fd, a, i, j, kp), dl, dr);
}

/* derivative of a distribution plane along axis a: Eq. (nonphi) between real
   cells; one-sided two-point difference next to a wall */
static real d1_dist(const osim *s, const real *Fd, int a, int i, int j)
{
    int k = a == 0 ? i : j, km, kp;
    double dl, dr;
    int hasm = neighbour(s, a, k, -1, &km, &dl);
    int hasp = neighbour(s, a, k, +1, &kp, &dr);
    real F0 = Fd[IDX(s, i, j)];
    if (hasm && hasp) return nonphi(at(s, Fd, a, i, j, km), F0, at(s, Fd, a, i, j, kp), dl, dr);
    if (hasp) return (at(s, Fd, a, i, j, kp) - F0) / dr;
    if (hasm) return (F0 - at(s, Fd, a, i, j, km)) / dl;
    return 0.0;
}

/* ------------------------------------------------------------------------- */
/* Step 7 / start of a step: macroscopic variables at the cell centres         */
/* ------------------------------------------------------------------------- */

static void cell_macros(osim *s)
{
    int nx = s->nx, ny = s->ny, N = nx * ny;
    real drho = (s->rhoA - s->rhoB) / (s->phiA - s->phiB);
    /* Eq. (phi), Eq. (oderrho) */
    for (int c = 0; c < N; c++) {
        real phi = 0.0;
        for (int i = 0; i < Q; i++) phi += s->g[i * N + c];
        s->phi[c] = phi;
        s->rho[c] = rho_of(s, phi);
    }
    /* Eq. (chemicalpotential) with the 5-point Laplacian of Eq. (nonphi2) */
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            int c = IDX(s, i, j);
            s->lap_phi[c] = d2_field(s, s->phi, 0, i, j) + d2_field(s, s->phi, 1, i, j);
            s->mu[c] = dpsi(s, s->phi[c]) - s->kappa * s->lap_phi[c];
        }
    /* grad mu, lap mu, grad phi, F = -phi grad mu + F_b, Eq. (u), Eq. (P), tau_f */
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            int c = IDX(s, i, j);
            real gmx = d1_field(s, s->mu, 0, i, j), gmy = d1_field(s, s->mu, 1, i, j);
            real lmu = d2_field(s, s->mu, 0, i, j) + d2_field(s, s->mu, 1, i, j);
            real gfx = d1_field(s, s->phi, 0, i, j), gfy = d1_field(s, s->phi, 1, i, j);
            real phi = s->phi[c], rho = s->rho[c];
            real Fx = -phi * gmx + (rho - s->rho_ref) * s->gx;
            real Fy = -phi * gmy + (rho - s->rho_ref) * s->gy;
            real sf = 0.0, mx = 0.0, my = 0.0;
            for (int q = 0; q < Q; q++) {
                real fq = s->f[q * N + c];
                sf += fq;
                mx += XI[q][0] * fq;
                my += XI[q][1] * fq;
            }
            real ux = (mx + 0.5 * s->dt * CS2 * Fx) / (CS2 * rho);
            real uy = (my + 0.5 * s->dt * CS2 * Fy) / (CS2 * rho);
            real grx = drho * gfx, gry = drho * gfy;
            real p = sf + 0.5 * s->dt * CS2 * (ux * grx + uy * gry - s->gamma * rho * s->lambda * lmu);
            s->gmu[0][c] = gmx; s->gmu[1][c] = gmy; s->lap_mu[c] = lmu;
            s->gphi[0][c] = gfx; s->gphi[1][c] = gfy;
            s->F[0][c] = Fx; s->F[1][c] = Fy;
            s->u[0][c] = ux; s->u[1][c] = uy; s->p[c] = p;
            s->tauf[c] = tauf_of(s, phi, rho);
        }
    /* grad p */
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            int c = IDX(s, i, j);
            s->gp[0][c] = d1_field(s, s->p, 0, i, j);
            s->gp[1][c] = d1_field(s, s->p, 1, i, j);
        }
}

/* equilibria and sources of both distributions at a point */
typedef struct {
    real phi, rho, ux, uy, p, mu, lap_mu, Fx, Fy, grx, gry, gpx, gpy, tauf;
} point_state;

static void point_eq_src(const osim *s, const point_state *ps, real *feq, real *geq, real *Ff,
                         real *Fg)
{
    oracle_feq(ps->p, ps->rho, ps->ux, ps->uy, feq);
    oracle_geq(ps->phi, ps->mu, s->eta, ps->ux, ps->uy, geq);
    oracle_src_f(ps->ux, ps->uy, ps->Fx, ps->Fy, ps->grx, ps->gry, ps->rho, s->gamma, s->lambda, ps->lap_mu, Ff);
    oracle_src_g(ps->phi, ps->rho, ps->ux, ps->uy, ps->Fx, ps->Fy, ps->gpx, ps->gpy, Fg);
}

static void cell_point(const osim *s, int c, point_state *ps)
{
    real drho = (s->rhoA - s->rhoB) / (s->phiA - s->phiB);
    ps->phi = s->phi[c]; ps->rho = s->rho[c];
    ps->ux = s->u[0][c]; ps->uy = s->u[1][c]; ps->p = s->p[c];
    ps->mu = s->mu[c]; ps->lap_mu = s->lap_mu[c];
    ps->Fx = s->F[0][c]; ps->Fy = s->F[1][c];
    ps->grx = drho * s->gphi[0][c]; ps->gry = drho * s->gphi[1][c];
    ps->gpx = s->gp[0][c]; ps->gpy = s->gp[1][c];
    ps->tauf = s->tauf[c];
}

/* ------------------------------------------------------------------------- */
/* Step 2: bar-plus and tilde-plus at the cell centres                        */
/* ------------------------------------------------------------------------- */

static void cell_auxiliaries(osim *s)
{
    int N = s->nx * s->ny;
#pragma omp parallel for schedule(static)
    for (int c = 0; c < N; c++) {
        point_state ps;
        real feq[Q], geq[Q], Ff[Q], Fg[Q];
        cell_point(s, c, &ps);
        point_eq_src(s, &ps, feq, geq, Ff, Fg);
        for (int i = 0; i < Q; i++) {
            real fb = oracle_bar_plus(s->f[i * N + c], feq[i], Ff[i], ps.tauf, s->dt);
            real gb = oracle_bar_plus(s->g[i * N + c], geq[i], Fg[i], s->tau_g, s->dt);
            s->fbp[i * N + c] = fb;
            s->gbp[i * N + c] = gb;
            s->ftp[i * N + c] = oracle_tilde_plus(fb, s->f[i * N + c]);
            s->gtp[i * N + c] = oracle_tilde_plus(gb, s->g[i * N + c]);
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Steps 3-5: faces                                                           */
/* ------------------------------------------------------------------------- */

/* Face macroscopic variables (Eq. conservedVariable with h and bar), then the
   equilibria, sources and original distributions (Eq. original-function).
   aux holds the interpolated mu, lap mu, grad mu, grad p, grad phi. */
typedef struct {
    real mu, lap_mu, gmu[2], gp[2], gphi[2];
} face_aux;

static void face_originals(const osim *s, const real *fbar, const real *gbar, const face_aux *ax,
                           int wall, real *forig, real *gorig)
{
    real drho = (s->rhoA - s->rhoB) / (s->phiA - s->phiB);
    double h = s->h;
    point_state ps;
    real phi = 0.0, sf = 0.0, mx = 0.0, my = 0.0;
    for (int i = 0; i < Q; i++) {
        phi += gbar[i];
        sf += fbar[i];
        mx += XI[i][0] * fbar[i];
        my += XI[i][1] * fbar[i];
    }
    real rho = rho_of(s, phi);
    real Fx = -phi * ax->gmu[0] + (rho - s->rho_ref) * s->gx;
    real Fy = -phi * ax->gmu[1] + (rho - s->rho_ref) * s->gy;
    real grx = drho * ax->gphi[0], gry = drho * ax->gphi[1];
    real ux, uy;
    if (wall) {
        ux = 0.0;
        uy = 0.0;
    } else {
        ux = (mx + 0.5 * h * CS2 * Fx) / (CS2 * rho);
        uy = (my + 0.5 * h * CS2 * Fy) / (CS2 * rho);
    }
    real p = sf + 0.5 * h * CS2 * (ux * grx + uy * gry - s->gamma * rho * s->lambda * ax->lap_mu);
    ps.phi = phi; ps.rho = rho; ps.ux = ux; ps.uy = uy; ps.p = p;
    ps.mu = ax->mu; ps.lap_mu = ax->lap_mu; ps.Fx = Fx; ps.Fy = Fy;
    ps.grx = grx; ps.gry = gry; ps.gpx = ax->gp[0]; ps.gpy = ax->gp[1];
    ps.tauf = tauf_of(s, phi, rho);
    real feq[Q], geq[Q], Ff[Q], Fg[Q];
    point_eq_src(s, &ps, feq, geq, Ff, Fg);
    for (int i = 0; i < Q; i++) {
        forig[i] = oracle_original(fbar[i], feq[i], Ff[i], ps.tauf, h);
        gorig[i] = oracle_original(gbar[i], geq[i], Fg[i], s->tau_g, h);
    }
}

/* Interior (or periodic) face between cell L and cell R = next along axis a.
   Adds (xi.n) phi_i |S| to J of both cells (n outward for each). */
static void interior_face(osim *s, int a, int iL, int jL, int iR, int jR)
{
    int N = s->nx * s->ny, t = 1 - a;
    int cL = IDX(s, iL, jL), cR = IDX(s, iR, jR);
    double dL = 0.5 * s->d[a][a == 0 ? iL : jL];
    double dR = 0.5 * s->d[a][a == 0 ? iR : jR];
    double wL = dR / (dL + dR), wR = dL / (dL + dR);
    double area = a == 0 ? s->d[1][jL] : s->d[0][iL];
    real fbar[Q], gbar[Q], forig[Q], gorig[Q];
    /* step 3: bar-plus at x_b by linear interpolation, gradient sigma_b, then
       Eq. (fbar) with the Taylor form Eq. (fbar_h) */
    for (int i = 0; i < Q; i++) {
        const real *Pf = s->fbp + i * N, *Pg = s->gbp + i * N;
        real vf = wL * Pf[cL] + wR * Pf[cR];
        real vg = wL * Pg[cL] + wR * Pg[cR];
        real nf = (Pf[cR] - Pf[cL]) / (dL + dR);
        real ng = (Pg[cR] - Pg[cL]) / (dL + dR);
        real tf = wL * d1_dist(s, Pf, t, iL, jL) + wR * d1_dist(s, Pf, t, iR, jR);
        real tg = wL * d1_dist(s, Pg, t, iL, jL) + wR * d1_dist(s, Pg, t, iR, jR);
        fbar[i] = vf - s->h * (XI[i][a] * nf + XI[i][t] * tf);
        gbar[i] = vg - s->h * (XI[i][a] * ng + XI[i][t] * tg);
    }
    /* step 4: face macroscopic variables from interpolated cell values at t_n */
    face_aux ax;
    ax.mu = wL * s->mu[cL] + wR * s->mu[cR];
    ax.lap_mu = wL * s->lap_mu[cL] + wR * s->lap_mu[cR];
    for (int k = 0; k < 2; k++) {
        ax.gmu[k] = wL * s->gmu[k][cL] + wR * s->gmu[k][cR];
        ax.gp[k] = wL * s->gp[k][cL] + wR * s->gp[k][cR];
        ax.gphi[k] = wL * s->gphi[k][cL] + wR * s->gphi[k][cR];
    }
    face_originals(s, fbar, gbar, &ax, 0, forig, gorig);
    /* step 5: micro-flux, Eq. (microfluxf) */
    for (int i = 0; i < Q; i++) {
        double xn = XI[i][a];
        s->Jf[i * N + cL] += xn * forig[i] * area;
        s->Jg[i * N + cL] += xn * gorig[i] * area;
        s->Jf[i * N + cR] -= xn * forig[i] * area;
        s->Jg[i * N + cR] -= xn * gorig[i] * area;
    }
}

/* Wall face of cell c on axis a, side = +1 (high end) or -1 (low end);
   n = side * e_a is the outward normal of the cell. */
static void wall_face(osim *s, int a, int i, int j, int side)
{
    int N = s->nx * s->ny, t = 1 - a, c = IDX(s, i, j);
    double dc = s->d[a][a == 0 ? i : j];
    double area = a == 0 ? s->d[1][j] : s->d[0][i];
    real fbar[Q], gbar[Q], forig[Q], gorig[Q];
    /* outgoing and parallel directions: Taylor reconstruction from the cell
       centre, x_b - xi h - x_c = (side dc/2 - xi_a h) e_a - xi_t h e_t */
    for (int q = 0; q < Q; q++) {
        if (XI[q][a] * side < 0) continue;
        const real *Pf = s->fbp + q * N, *Pg = s->gbp + q * N;
        double off = side * 0.5 * dc - s->h * XI[q][a];
        fbar[q] = Pf[c] + off * d1_dist(s, Pf, a, i, j) - s->h * XI[q][t] * d1_dist(s, Pf, t, i, j);
        gbar[q] = Pg[c] + off * d1_dist(s, Pg, a, i, j) - s->h * XI[q][t] * d1_dist(s, Pg, t, i, j);
    }
    /* incoming directions: bounce-back of the bar distributions */
    for (int q = 0; q < Q; q++) {
        if (XI[q][a] * side < 0) {
            fbar[q] = fbar[OPP[q]];
            gbar[q] = gbar[OPP[q]];
        }
    }
    /* mirror interpolation of the cell values: value kept, normal gradient 0 */
    face_aux ax;
    ax.mu = s->mu[c];
    ax.lap_mu = s->lap_mu[c];
    ax.gmu[a] = 0.0; ax.gmu[t] = s->gmu[t][c];
    ax.gp[a] = 0.0; ax.gp[t] = s->gp[t][c];
    ax.gphi[a] = 0.0; ax.gphi[t] = s->gphi[t][c];
    face_originals(s, fbar, gbar, &ax, 1, forig, gorig);
    /* incoming originals: bounce-back */
    for (int q = 0; q < Q; q++) {
        if (XI[q][a] * side < 0) {
            forig[q] = forig[OPP[q]];
            gorig[q] = gorig[OPP[q]];
        }
    }
    for (int q = 0; q < Q; q++) {
        double xn = XI[q][a] * side;
        s->Jf[q * N + c] += xn * forig[q] * area;
        s->Jg[q * N + c] += xn * gorig[q] * area;
    }
}

static void all_faces(osim *s)
{
    int nx = s->nx, ny = s->ny, N = nx * ny;
    memset(s->Jf, 0, sizeof(real) * Q * N);
    memset(s->Jg, 0, sizeof(real) * Q * N);
    /* x faces, one row at a time (rows touch disjoint cells) */
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; j++) {
        for (int i = 0; i + 1 < nx; i++) interior_face(s, 0, i, j, i + 1, j);
        if (s->bc[0] == BC_PERIODIC) {
            interior_face(s, 0, nx - 1, j, 0, j);
        } else {
            wall_face(s, 0, 0, j, -1);
            wall_face(s, 0, nx - 1, j, +1);
        }
    }
    /* y faces, one column at a time */
#pragma omp parallel for schedule(static)
    for (int i = 0; i < nx; i++) {
        for (int j = 0; j + 1 < ny; j++) interior_face(s, 1, i, j, i, j + 1);
        if (s->bc[1] == BC_PERIODIC) {
            interior_face(s, 1, i, ny - 1, i, 0);
        } else {
            wall_face(s, 1, i, 0, -1);
            wall_face(s, 1, i, ny - 1, +1);
        }
    }
}

/* Step 6: Eq. (updatef) */
static void update_cells(osim *s)
{
    int nx = s->nx, ny = s->ny, N = nx * ny;
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            int c = IDX(s, i, j);
            double vol = s->d[0][i] * s->d[1][j];
            for (int q = 0; q < Q; q++) {
                s->f[q * N + c] = s->ftp[q * N + c] - s->dt / vol * s->Jf[q * N + c];
                s->g[q * N + c] = s->gtp[q * N + c] - s->dt / vol * s->Jg[q * N + c];
            }
        }
}

/* ------------------------------------------------------------------------- */
/* Public entry points (ctypes)                                               */
/* ------------------------------------------------------------------------- */

void oracle_destroy(void *h);

/* params: phiA, phiB, rhoA, rhoB, nuA, nuB, lambda, tau_g, beta, kappa, gx, gy, rho_ref, cfl */
void *oracle_create(int nx, int ny, int bcx, int bcy, const double *dx, const double *dy,
                    const real *prm)
{
    if (nx < 1 || ny < 1) return NULL;
    osim *s = (osim *)calloc(1, sizeof(osim));
    if (!s) return NULL;
    int N = nx * ny;
    s->nx = nx; s->ny = ny; s->bc[0] = bcx; s->bc[1] = bcy;
    s->d[0] = (double *)malloc(sizeof(double) * nx);
    s->d[1] = (double *)malloc(sizeof(double) * ny);
    memcpy(s->d[0], dx, sizeof(double) * nx);
    memcpy(s->d[1], dy, sizeof(double) * ny);
    s->phiA = prm[0]; s->phiB = prm[1]; s->rhoA = prm[2]; s->rhoB = prm[3];
    s->nuA = prm[4]; s->nuB = prm[5]; s->lambda = prm[6]; s->tau_g = prm[7];
    s->beta = prm[8]; s->kappa = prm[9]; s->gx = prm[10]; s->gy = prm[11];
    s->rho_ref = prm[12]; s->cfl = creal_or_same(prm[13]);
    /* Eq. (cfl): dt = alpha dx_min / C_max with C_max = sqrt(6 RT) */
    double dmin = dx[0];
    for (int i = 0; i < nx; i++) if (dx[i] < dmin) dmin = dx[i];
    for (int j = 0; j < ny; j++) if (dy[j] < dmin) dmin = dy[j];
    s->dt = s->cfl * dmin / sqrt(6.0 * CS2);
    s->h = 0.5 * s->dt;
    /* Eq. (kineticandmobility): lambda = c_s^2 tau_g eta */
    s->eta = s->lambda / (CS2 * s->tau_g);
    /* Eq. (Gama) with rho_r = rhoA / rhoB */
    real rr = s->rhoA / s->rhoB;
    s->gamma = (rr - 1.0) / (s->phiA - s->phiB * rr);
    s->muA = s->rhoA * s->nuA;
    s->muB = s->rhoB * s->nuB;
    real **bufs[] = {&s->f, &s->g, &s->phi, &s->rho, &s->lap_phi, &s->mu, &s->lap_mu, &s->gphi[0],
                       &s->gphi[1], &s->gmu[0], &s->gmu[1], &s->F[0], &s->F[1], &s->u[0], &s->u[1],
                       &s->p, &s->gp[0], &s->gp[1], &s->tauf};
    int nb = (int)(sizeof(bufs) / sizeof(bufs[0]));
    for (int k = 0; k < nb; k++) {
        int m = (k < 2) ? Q * N : N;
        *bufs[k] = (real *)calloc((size_t)m, sizeof(real));
        if (!*bufs[k]) { oracle_destroy(s); return NULL; }
    }
    real **qb[] = {&s->fbp, &s->gbp, &s->ftp, &s->gtp, &s->Jf, &s->Jg};
    for (int k = 0; k < 6; k++) {
        *qb[k] = (real *)calloc((size_t)Q * N, sizeof(real));
        if (!*qb[k]) { oracle_destroy(s); return NULL; }
    }
    return s;
}

void oracle_destroy(void *h)
{
    osim *s = (osim *)h;
    if (!s) return;
    void *all[] = {s->d[0], s->d[1], s->f, s->g, s->phi, s->rho, s->lap_phi, s->mu, s->lap_mu,
                     s->gphi[0], s->gphi[1], s->gmu[0], s->gmu[1], s->F[0], s->F[1], s->u[0], s->u[1],
                     s->p, s->gp[0], s->gp[1], s->tauf, s->fbp, s->gbp, s->ftp, s->gtp, s->Jf, s->Jg};
    for (size_t k = 0; k < sizeof(all) / sizeof(all[0]); k++) free(all[k]);
    free(s);
}

double oracle_dt(void *h) { return ((osim *)h)->dt; }

/* Step 1: from phi, u, p at the cells, the tilde distributions are
   tilde = eq - dt/2 F (Eq. auxf a with the original distribution at equilibrium).
   ux, uy, p may be NULL (zero). */
int oracle_init(void *hd, const real *phi, const real *ux, const real *uy, const real *p)
{
    osim *s = (osim *)hd;
    int nx = s->nx, ny = s->ny, N = nx * ny;
    for (int c = 0; c < N; c++) {
        s->phi[c] = phi[c];
        s->rho[c] = rho_of(s, phi[c]);
        s->u[0][c] = ux ? ux[c] : 0.0;
        s->u[1][c] = uy ? uy[c] : 0.0;
        s->p[c] = p ? p[c] : 0.0;
    }
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            int c = IDX(s, i, j);
            s->lap_phi[c] = d2_field(s, s->phi, 0, i, j) + d2_field(s, s->phi, 1, i, j);
            s->mu[c] = dpsi(s, s->phi[c]) - s->kappa * s->lap_phi[c];
        }
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            int c = IDX(s, i, j);
            s->gmu[0][c] = d1_field(s, s->mu, 0, i, j);
            s->gmu[1][c] = d1_field(s, s->mu, 1, i, j);
            s->lap_mu[c] = d2_field(s, s->mu, 0, i, j) + d2_field(s, s->mu, 1, i, j);
            s->gphi[0][c] = d1_field(s, s->phi, 0, i, j);
            s->gphi[1][c] = d1_field(s, s->phi, 1, i, j);
            s->gp[0][c] = d1_field(s, s->p, 0, i, j);
            s->gp[1][c] = d1_field(s, s->p, 1, i, j);
            s->F[0][c] = -s->phi[c] * s->gmu[0][c] + (s->rho[c] - s->rho_ref) * s->gx;
            s->F[1][c] = -s->phi[c] * s->gmu[1][c] + (s->rho[c] - s->rho_ref) * s->gy;
            s->tauf[c] = tauf_of(s, s->phi[c], s->rho[c]);
        }
    for (int c = 0; c < N; c++) {
        point_state ps;
        real feq[Q], geq[Q], Ff[Q], Fg[Q];
        cell_point(s, c, &ps);
        point_eq_src(s, &ps, feq, geq, Ff, Fg);
        for (int i = 0; i < Q; i++) {
            s->f[i * N + c] = feq[i] - 0.5 * s->dt * Ff[i];
            s->g[i * N + c] = geq[i] - 0.5 * s->dt * Fg[i];
        }
    }
    for (int c = 0; c < Q * N; c++)
        if (!FINITE(s->f[c]) || !FINITE(s->g[c])) return -3;
    return 0;
}

/* Steps 7, 2, 3-5, 6 repeated n times. Returns -3 if the state becomes non-finite. */
int oracle_step(void *hd, long n)
{
    osim *s = (osim *)hd;
    int N = s->nx * s->ny;
    for (long k = 0; k < n; k++) {
        cell_macros(s);
        cell_auxiliaries(s);
        all_faces(s);
        update_cells(s);
    }
    for (int c = 0; c < Q * N; c++)
        if (!FINITE(s->f[c]) || !FINITE(s->g[c])) return -3;
    return 0;
}

/* Macroscopic fields from the current tilde state (Eqs. phi, oderrho, u, P);
   any output pointer may be NULL. */
void oracle_moments(void *hd, real *phi, real *rho, real *ux, real *uy, real *p)
{
    osim *s = (osim *)hd;
    int N = s->nx * s->ny;
    cell_macros(s);
    for (int c = 0; c < N; c++) {
        if (phi) phi[c] = s->phi[c];
        if (rho) rho[c] = s->rho[c];
        if (ux) ux[c] = s->u[0][c];
        if (uy) uy[c] = s->u[1][c];
        if (p) p[c] = s->p[c];
    }
}

/* Cell fields of the last macro evaluation: mu, lap_mu, grad mu, grad p, grad phi, tau_f */
void oracle_aux(void *hd, real *mu, real *lap_mu, real *gmux, real *gmuy, real *gpx,
                real *gpy, real *gphix, real *gphiy, real *tauf)
{
    osim *s = (osim *)hd;
    int N = s->nx * s->ny;
    for (int c = 0; c < N; c++) {
        if (mu) mu[c] = s->mu[c];
        if (lap_mu) lap_mu[c] = s->lap_mu[c];
        if (gmux) gmux[c] = s->gmu[0][c];
        if (gmuy) gmuy[c] = s->gmu[1][c];
        if (gpx) gpx[c] = s->gp[0][c];
        if (gpy) gpy[c] = s->gp[1][c];
        if (gphix) gphix[c] = s->gphi[0][c];
        if (gphiy) gphiy[c] = s->gphi[1][c];
        if (tauf) tauf[c] = s->tauf[c];
    }
}

void oracle_get_state(void *hd, real *f, real *g)
{
    osim *s = (osim *)hd;
    size_t n = (size_t)Q * s->nx * s->ny;
    memcpy(f, s->f, n * sizeof(real));
    memcpy(g, s->g, n * sizeof(real));
}

void oracle_set_state(void *hd, const real *f, const real *g)
{
    osim *s = (osim *)hd;
    size_t n = (size_t)Q * s->nx * s->ny;
    memcpy(s->f, f, n * sizeof(real));
    memcpy(s->g, g, n * sizeof(real));
}

/* Volume-weighted totals of phi and rho (Eq. locallyconserved) */
void oracle_conservation(void *hd, real *sum_phi, real *sum_rho)
{
    osim *s = (osim *)hd;
    int nx = s->nx, ny = s->ny, N = nx * ny;
    real a = 0.0, b = 0.0;
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            int c = IDX(s, i, j);
            real phi = 0.0;
            for (int q = 0; q < Q; q++) phi += s->g[q * N + c];
            double vol = s->d[0][i] * s->d[1][j];
            a += vol * phi;
            b += vol * rho_of(s, phi);
        }
    *sum_phi = a;
    *sum_rho = b;
}

/* Non-uniform first and second derivative of a cell field (mirror ghosts), for pins */
void oracle_derivatives(void *hd, const real *F, real *dx, real *dy, real *lap)
{
    osim *s = (osim *)hd;
    for (int j = 0; j < s->ny; j++)
        for (int i = 0; i < s->nx; i++) {
            int c = IDX(s, i, j);
            if (dx) dx[c] = d1_field(s, F, 0, i, j);
            if (dy) dy[c] = d1_field(s, F, 1, i, j);
            if (lap) lap[c] = d2_field(s, F, 0, i, j) + d2_field(s, F, 1, i, j);
        }
}

/* Cell-centre bar-plus distributions of the current state (step 2), [Q][N] each */
void oracle_bar_plus_fields(void *hd, real *fbp, real *gbp)
{
    osim *s = (osim *)hd;
    size_t n = (size_t)Q * s->nx * s->ny;
    cell_macros(s);
    cell_auxiliaries(s);
    if (fbp) memcpy(fbp, s->fbp, n * sizeof(real));
    if (gbp) memcpy(gbp, s->gbp, n * sizeof(real));
}

void oracle_derived(void *hd, real *out /* dt, h, eta, gamma, muA, muB */)
{
    osim *s = (osim *)hd;
    out[0] = s->dt; out[1] = s->h; out[2] = s->eta; out[3] = s->gamma; out[4] = s->muA; out[5] = s->muB;
}

/* Eqs. (thickness) and (sigma): interface width and surface tension from beta, kappa */
void oracle_width_sigma(double beta, double kappa, double phiA, double phiB, double *W, double *sigma)
{
    *W = sqrt(8.0 * kappa / beta) / (phiA - phiB);
    *sigma = pow(fabs(phiA - phiB), 3.0) / 6.0 * sqrt(2.0 * kappa * beta);
}
