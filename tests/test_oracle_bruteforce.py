"""An independent extended-precision step on tiny meshes, compared with the
oracle's step.

The oracle advances the tilde distributions with the shortcut relations of
Sec. 2.2 (Eq. relations1 for bar-plus from tilde, Eq. original-function at the
faces, Eq. relations2 for tilde-plus) and the closed forms of Eqs. (u), (P)
for the macroscopic variables.  This step does not use any of them.  It goes
through the defining auxiliary distributions instead, in 50-digit arithmetic
(mpmath):

* the original distribution at a cell solves tilde = f - dt/2 Omega(f)
  (Eq. auxf a), found by fixed-point iteration with the macroscopic variables
  taken as plain moments of f itself (p = sum f, c_s^2 rho u = sum xi f;
  phi = sum tilde g, Eq. phi);
* bar-plus = f + h/2 Omega(f) (Eq. auxfbar b) and tilde-plus = f + dt/2
  Omega(f) (Eq. auxf b) at the cells;
* at a face, the original distribution solves bar = f - h/2 Omega(f)
  (Eq. auxfbar a), again by fixed-point iteration on its own moments (the
  wall velocity held at zero at a wall face);
* the update is tilde^{n+1} = tilde-plus - dt/|V| J (Eq. updatef).

The gradients, the face interpolation and the wall treatment are the readings
the oracle documents (values and tangential derivatives interpolated between
the two cell centres, mirror ghosts for phi, mu and p, one-sided derivatives
of distributions next to walls, bounce-back of the incoming bar and original
distributions).  A mistake in the shortcut relations, in the tilde-based
moments, in an index or a sign of the oracle's step shows up here as an O(1)
relative difference; rounding alone stays near 1e-14.
"""
import numpy as np
import pytest

import oracle
from paper_1802_02868_gb300 import inputs as I

mp = pytest.importorskip("mpmath")
mp.mp.dps = 50

XI = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
OPP = [0, 3, 4, 1, 2, 7, 8, 5, 6]
Q = 9


class Brute:
    """One step of the scheme on a tiny mesh in mpmath arithmetic."""

    def __init__(self, mesh, prm):
        M = mp.mpf
        self.nx, self.ny = mesh.nx, mesh.ny
        self.d = [[M(v) for v in mesh.dx], [M(v) for v in mesh.dy]]
        self.bc = [mesh.bc_x, mesh.bc_y]
        P = prm
        self.phiA, self.phiB, self.rhoA, self.rhoB = M(P.phiA), M(P.phiB), M(P.rhoA), M(P.rhoB)
        self.muA, self.muB = M(P.rhoA) * M(P.nuA), M(P.rhoB) * M(P.nuB)
        self.lam, self.tau_g, self.beta, self.kappa = M(P.mobility), M(P.tau_g), M(P.beta), M(P.kappa)
        self.g = (M(P.gx), M(P.gy))
        self.rho_ref = M(P.rho_ref)
        self.cs2 = M(1) / 3
        self.w = [M(4) / 9] + [M(1) / 9] * 4 + [M(1) / 36] * 4
        dmin = min(min(self.d[0]), min(self.d[1]))
        # Eq. (cfl) with C_max = sqrt(6 RT) = sqrt(2)
        self.dt = M(P.cfl) * dmin / mp.sqrt(2)
        self.h = self.dt / 2
        self.eta = self.lam / (self.cs2 * self.tau_g)
        rr = self.rhoA / self.rhoB
        self.gamma = (rr - 1) / (self.phiA - self.phiB * rr)
        self.drho = (self.rhoA - self.rhoB) / (self.phiA - self.phiB)

    # -- model relations (Sec. 2.1, 2.2)
    def rho(self, phi):
        return self.rhoB + self.drho * (phi - self.phiB)

    def tauf(self, phi, rho):
        mu = self.muA * self.muB * (self.phiA - self.phiB) / ((phi - self.phiB) * self.muB + (self.phiA - phi) * self.muA)
        return mu / rho / self.cs2

    def s(self, i, u):
        xu = XI[i][0] * u[0] + XI[i][1] * u[1]
        uu = u[0] ** 2 + u[1] ** 2
        c = self.cs2
        return self.w[i] * (xu / c + xu * xu / (2 * c * c) - uu / (2 * c))

    def omega_f(self, f, st):
        """BGK collision plus source of f (Eqs. bgkf, feq, F) at a point."""
        u, rho = st["u"], st["rho"]
        out = []
        for i in range(Q):
            si = self.s(i, u)
            feq = self.w[i] * st["p"] + self.cs2 * rho * si
            G = self.w[i] + si
            src = sum((XI[i][a] - u[a]) * (st["F"][a] * G + si * self.cs2 * st["grho"][a]) for a in range(2)) \
                - self.w[i] * self.cs2 * rho * self.gamma * self.lam * st["lapmu"]
            out.append((feq - f[i]) / st["tauf"] + src)
        return out

    def omega_g(self, g, st):
        """Collision plus source of g (Eqs. bgkg, geq, Hi, G) at a point."""
        u, rho, phi = st["u"], st["rho"], st["phi"]
        out = []
        for i in range(Q):
            si = self.s(i, u)
            H = phi - (1 - self.w[0]) * self.eta * st["mu"] if i == 0 else self.w[i] * self.eta * st["mu"]
            geq = H + phi * si
            src = phi / (self.cs2 * rho) * sum((XI[i][a] - u[a]) * (st["F"][a] - st["gp"][a]) for a in range(2)) \
                * (self.w[i] + si)
            out.append((geq - g[i]) / self.tau_g + src)
        return out

    def solve_f(self, given, k, st, wall=False):
        """Original f with given = f - k Omega_f(f) (k = +dt/2 from tilde, +h/2
        from bar): fixed point of f = given + k Omega_f(f), the macroscopic
        variables being moments of f (u = 0 held at a wall face)."""
        f = list(given)
        for _ in range(400):
            st["p"] = sum(f)
            st["u"] = (mp.mpf(0), mp.mpf(0)) if wall else tuple(
                sum(XI[i][a] * f[i] for i in range(Q)) / (self.cs2 * st["rho"]) for a in range(2))
            om = self.omega_f(f, st)
            new = [given[i] + k * om[i] for i in range(Q)]
            if max(abs(new[i] - f[i]) for i in range(Q)) < mp.mpf(10) ** -45:
                f = new
                break
            f = new
        else:
            raise AssertionError("fixed point did not converge")
        st["p"] = sum(f)
        if not wall:
            st["u"] = tuple(sum(XI[i][a] * f[i] for i in range(Q)) / (self.cs2 * st["rho"]) for a in range(2))
        return f

    def solve_g(self, given, k, st):
        g = list(given)
        for _ in range(400):
            om = self.omega_g(g, st)
            new = [given[i] + k * om[i] for i in range(Q)]
            if max(abs(new[i] - g[i]) for i in range(Q)) < mp.mpf(10) ** -45:
                return new
            g = new
        raise AssertionError("fixed point did not converge")

    # -- mesh differences (Eqs. nonphi, nonphi2; mirror ghosts at walls)
    def nb(self, a, k, side):
        n = self.nx if a == 0 else self.ny
        k2 = k + side
        if 0 <= k2 < n:
            return k2, (self.d[a][k] + self.d[a][k2]) / 2, True
        if self.bc[a] == I.PERIODIC:
            k2 %= n
            return k2, (self.d[a][k] + self.d[a][k2]) / 2, True
        return k, self.d[a][k], False

    def val(self, F, a, i, j, k):
        return F[j][k] if a == 0 else F[k][i]

    def d1(self, F, a, i, j, dist=False):
        k = i if a == 0 else j
        km, dl, hm = self.nb(a, k, -1)
        kp, dr, hp = self.nb(a, k, +1)
        Fm, F0, Fp = self.val(F, a, i, j, km), F[j][i], self.val(F, a, i, j, kp)
        if dist and not (hm and hp):
            if hp:
                return (Fp - F0) / dr
            if hm:
                return (F0 - Fm) / dl
            return mp.mpf(0)
        delta = (dl + dr) / 2
        tl, tr = dl / delta, dr / delta
        return (tl * tl * Fp + (tl + tr) * (tr - tl) * F0 - tr * tr * Fm) / (tl * tr * (tl + tr) * delta)

    def d2(self, F, a, i, j):
        k = i if a == 0 else j
        km, dl, _ = self.nb(a, k, -1)
        kp, dr, _ = self.nb(a, k, +1)
        Fm, F0, Fp = self.val(F, a, i, j, km), F[j][i], self.val(F, a, i, j, kp)
        delta = (dl + dr) / 2
        tl, tr = dl / delta, dr / delta
        return 2 / (tl * tr * (tl + tr) * delta * delta) * (tl * Fp - (tl + tr) * F0 + tr * Fm)

    # -- one step
    def step(self, ft, gt):
        nx, ny, M = self.nx, self.ny, mp.mpf
        cells = [(i, j) for j in range(ny) for i in range(nx)]
        grid = lambda: [[M(0)] * nx for _ in range(ny)]
        phi, rho, mu = grid(), grid(), grid()
        for i, j in cells:
            phi[j][i] = sum(gt[q][j][i] for q in range(Q))      # Eq. (phi)
            rho[j][i] = self.rho(phi[j][i])
        for i, j in cells:
            lap = self.d2(phi, 0, i, j) + self.d2(phi, 1, i, j)
            p0 = phi[j][i]
            mu[j][i] = 4 * self.beta * (p0 - self.phiA) * (p0 - self.phiB) * (p0 - (self.phiA + self.phiB) / 2) \
                - self.kappa * lap
        st = {}
        for i, j in cells:
            s = {"phi": phi[j][i], "rho": rho[j][i], "mu": mu[j][i],
                 "gmu": (self.d1(mu, 0, i, j), self.d1(mu, 1, i, j)),
                 "lapmu": self.d2(mu, 0, i, j) + self.d2(mu, 1, i, j),
                 "gphi": (self.d1(phi, 0, i, j), self.d1(phi, 1, i, j))}
            s["F"] = tuple(-s["phi"] * s["gmu"][a] + (s["rho"] - self.rho_ref) * self.g[a] for a in range(2))
            s["grho"] = tuple(self.drho * s["gphi"][a] for a in range(2))
            s["tauf"] = self.tauf(s["phi"], s["rho"])
            st[(i, j)] = s
        # originals of f at the cells (p and u from their moments), then grad p
        forig, p = {}, grid()
        for i, j in cells:
            forig[(i, j)] = self.solve_f([ft[q][j][i] for q in range(Q)], self.dt / 2, st[(i, j)])
            p[j][i] = st[(i, j)]["p"]
        for i, j in cells:
            st[(i, j)]["gp"] = (self.d1(p, 0, i, j), self.d1(p, 1, i, j))
        fbp = [grid() for _ in range(Q)]
        gbp = [grid() for _ in range(Q)]
        ftp = [grid() for _ in range(Q)]
        gtp = [grid() for _ in range(Q)]
        for i, j in cells:
            s = st[(i, j)]
            f = forig[(i, j)]
            g = self.solve_g([gt[q][j][i] for q in range(Q)], self.dt / 2, s)
            of, og = self.omega_f(f, s), self.omega_g(g, s)
            for q in range(Q):
                fbp[q][j][i] = f[q] + self.h / 2 * of[q]      # Eq. (auxfbar b)
                gbp[q][j][i] = g[q] + self.h / 2 * og[q]
                ftp[q][j][i] = f[q] + self.dt / 2 * of[q]     # Eq. (auxf b)
                gtp[q][j][i] = g[q] + self.dt / 2 * og[q]
        Jf = [grid() for _ in range(Q)]
        Jg = [grid() for _ in range(Q)]

        def face_state(phib, aux, wall):
            s = {"phi": phib, "rho": self.rho(phib), "mu": aux["mu"], "lapmu": aux["lapmu"],
                 "gp": aux["gp"]}
            s["F"] = tuple(-phib * aux["gmu"][a] + (s["rho"] - self.rho_ref) * self.g[a] for a in range(2))
            s["grho"] = tuple(self.drho * aux["gphi"][a] for a in range(2))
            s["tauf"] = self.tauf(phib, s["rho"])
            return s

        def originals(fb, gb, aux, wall):
            s = face_state(sum(gb), aux, wall)
            f = self.solve_f(fb, self.h / 2, s, wall=wall)
            return f, self.solve_g(gb, self.h / 2, s)

        def interp(L, R, wL, wR):
            return {"mu": wL * st[L]["mu"] + wR * st[R]["mu"], "lapmu": wL * st[L]["lapmu"] + wR * st[R]["lapmu"],
                    "gmu": tuple(wL * st[L]["gmu"][a] + wR * st[R]["gmu"][a] for a in range(2)),
                    "gp": tuple(wL * st[L]["gp"][a] + wR * st[R]["gp"][a] for a in range(2)),
                    "gphi": tuple(wL * st[L]["gphi"][a] + wR * st[R]["gphi"][a] for a in range(2))}

        def interior(a, L, R):
            t = 1 - a
            (iL, jL), (iR, jR) = L, R
            dL = self.d[a][iL if a == 0 else jL] / 2
            dR = self.d[a][iR if a == 0 else jR] / 2
            wL, wR = dR / (dL + dR), dL / (dL + dR)
            area = self.d[1][jL] if a == 0 else self.d[0][iL]
            fb, gb = [], []
            for q in range(Q):
                for B, out in ((fbp, fb), (gbp, gb)):
                    v = wL * B[q][jL][iL] + wR * B[q][jR][iR]
                    nrm = (B[q][jR][iR] - B[q][jL][iL]) / (dL + dR)
                    tan = wL * self.d1(B[q], t, iL, jL, dist=True) + wR * self.d1(B[q], t, iR, jR, dist=True)
                    out.append(v - self.h * (XI[q][a] * nrm + XI[q][t] * tan))   # Eqs. (fbar), (fbar_h)
            f, g = originals(fb, gb, interp(L, R, wL, wR), False)
            for q in range(Q):
                for J, o in ((Jf, f), (Jg, g)):
                    J[q][jL][iL] += XI[q][a] * o[q] * area
                    J[q][jR][iR] -= XI[q][a] * o[q] * area

        def wall(a, c, side):
            t = 1 - a
            i, j = c
            dc = self.d[a][i if a == 0 else j]
            area = self.d[1][j] if a == 0 else self.d[0][i]
            fb, gb = [None] * Q, [None] * Q
            for q in range(Q):
                if XI[q][a] * side < 0:
                    continue
                off = side * dc / 2 - self.h * XI[q][a]
                for B, out in ((fbp, fb), (gbp, gb)):
                    out[q] = B[q][j][i] + off * self.d1(B[q], a, i, j, dist=True) \
                        - self.h * XI[q][t] * self.d1(B[q], t, i, j, dist=True)
            for q in range(Q):
                if XI[q][a] * side < 0:
                    fb[q], gb[q] = fb[OPP[q]], gb[OPP[q]]
            s = st[c]
            aux = {"mu": s["mu"], "lapmu": s["lapmu"],
                   "gmu": tuple(M(0) if k == a else s["gmu"][k] for k in range(2)),
                   "gp": tuple(M(0) if k == a else s["gp"][k] for k in range(2)),
                   "gphi": tuple(M(0) if k == a else s["gphi"][k] for k in range(2))}
            f, g = originals(fb, gb, aux, True)
            for q in range(Q):
                if XI[q][a] * side < 0:
                    f[q], g[q] = f[OPP[q]], g[OPP[q]]
            for q in range(Q):
                Jf[q][j][i] += XI[q][a] * side * f[q] * area
                Jg[q][j][i] += XI[q][a] * side * g[q] * area

        for j in range(ny):
            for i in range(nx - 1):
                interior(0, (i, j), (i + 1, j))
            if self.bc[0] == I.PERIODIC:
                interior(0, (nx - 1, j), (0, j))
            else:
                wall(0, (0, j), -1)
                wall(0, (nx - 1, j), +1)
        for i in range(nx):
            for j in range(ny - 1):
                interior(1, (i, j), (i, j + 1))
            if self.bc[1] == I.PERIODIC:
                interior(1, (i, ny - 1), (i, 0))
            else:
                wall(1, (i, 0), -1)
                wall(1, (i, ny - 1), +1)
        fn = [grid() for _ in range(Q)]
        gn = [grid() for _ in range(Q)]
        for i, j in cells:
            vol = self.d[0][i] * self.d[1][j]
            for q in range(Q):
                fn[q][j][i] = ftp[q][j][i] - self.dt / vol * Jf[q][j][i]   # Eq. (updatef)
                gn[q][j][i] = gtp[q][j][i] - self.dt / vol * Jg[q][j][i]
        return fn, gn


def _mpgrid(a):
    return [[[mp.mpf(float(v)) for v in row] for row in plane] for plane in a]


def _case(nx, ny, bcx, bcy, seed, stretch):
    rng = np.random.default_rng(seed)
    dx = 1.0 + stretch * rng.random(nx)
    dy = 1.0 + stretch * rng.random(ny)
    mesh = I.Mesh(dx, dy, bcx, bcy)
    beta, kappa = I.params_from_sigma_width(1e-2, 2.0)
    prm = I.Params(rhoA=2.0, rhoB=1.0, nuA=0.3, nuB=0.2, mobility=0.2, tau_g=0.5, beta=beta, kappa=kappa,
                   gx=2e-3, gy=-3e-3, rho_ref=1.5, cfl=0.5)
    phi = 0.5 + 0.4 * np.tanh(rng.normal(size=(ny, nx)))
    ux, uy, p = (1e-2 * rng.normal(size=(ny, nx)) for _ in range(3))
    return mesh, prm, phi, ux, uy, p


@pytest.mark.parametrize("nx,ny,bcx,bcy,stretch", [
    (3, 3, I.PERIODIC, I.PERIODIC, 0.0),
    (4, 4, I.WALL, I.WALL, 0.0),
    (4, 4, I.PERIODIC, I.WALL, 0.6),
    (3, 4, I.WALL, I.PERIODIC, 0.6),
])
def test_step_equals_extended_precision_step_through_the_auxiliary_definitions(nx, ny, bcx, bcy, stretch):
    mesh, prm, phi, ux, uy, p = _case(nx, ny, bcx, bcy, 7 + nx * ny + bcx + 2 * bcy, stretch)
    o = oracle.Oracle(mesh, prm).init(phi, ux, uy, p)
    o.step(2)                      # a generic state, off the initial equilibrium
    f0, g0 = o.state()
    o.step(1)
    f1, g1 = o.state()
    B = Brute(mesh, prm)
    assert abs(float(B.dt) - o.dt) <= 1e-15 * o.dt
    fn, gn = B.step(_mpgrid(f0), _mpgrid(g0))
    fb = np.array([[[float(v) for v in row] for row in plane] for plane in fn])
    gb = np.array([[[float(v) for v in row] for row in plane] for plane in gn])
    # the one-step increments, where the scheme's work shows, agree to rounding
    for new, old, ref in ((f1, f0, fb), (g1, g0, gb)):
        inc, inc_ref = new - old, ref - old
        assert np.abs(inc - inc_ref).max() <= 1e-11 * np.abs(inc_ref).max(), \
            np.abs(inc - inc_ref).max() / np.abs(inc_ref).max()
        assert np.abs(new - ref).max() <= 1e-13 * np.abs(ref).max()
