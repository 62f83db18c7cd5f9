"""Second, independently written FP64 oracle in NumPy, for tiny lattices.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``). It restates the same method
as ``lbm_oracle.c`` in array form -- velocity set generated rather than tabulated,
streaming by ``np.roll`` with masks for the walls, the near-contact ray as a plain
Python loop over interface nodes -- so that an indexing or transcription slip in
either version shows up as a disagreement. Arrays are indexed [.., z, y, x].

Readings (identical to the C oracle, where the paper is silent):
  * D3Q19: rest + 6 faces + 12 edges, w = 1/3, 1/18, 1/36, c_s^2 = 1/3.
  * omega_eff = 2 c_s^2 / (2 nu + c_s^2), 1/nu = sum_k (rho_k/rho)/nu_k  (Eqs. 4, 7, 8).
  * Total-population BGK + EDM source (Eqs. 1, 2, 5, 6, 9) with bare u = j/rho.
  * Colour gradient 3 sum w c phi(x+c), wall neighbour -> phi(x).
  * Perturbation (A/2)|G|(w (c.n)^2 - B), A = 9 omega sigma / 2,
    B = -2/9, 1/54, 1/27; recolouring with beta (Latva-Kokko & Rothman);
    both skipped where |G| < 1e-6.
  * Near-contact force A_h[h] G (Eq. 11); h is measured on the lagged colour field,
    along minus its own gradient, by linear zero-crossing location between
    consecutive half-unit samples that carry a sign (|phi| > 1e-5).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

CS2 = 1.0 / 3.0


def velocity_set():
    vecs = [v for v in itertools.product((-1, 0, 1), repeat=3) if sum(a * a for a in v) <= 2]
    c = np.array(vecs, dtype=np.int64)            # [19, 3] as (cx, cy, cz)
    c2 = (c * c).sum(1)
    w = np.where(c2 == 0, 1 / 3, np.where(c2 == 1, 1 / 18, 1 / 36))
    B = np.where(c2 == 0, -2 / 9, np.where(c2 == 1, 1 / 54, 1 / 27))
    opp = np.array([int(np.nonzero((c == -c[i]).all(1))[0][0]) for i in range(len(c))])
    return c, w, B, opp


C_, W_, B_, OPP_ = velocity_set()


def equilibrium(rho, u):
    """rho [...], u [3, ...] -> f^eq [19, ...] (Eq. 2)."""
    cu = np.einsum("ia,a...->i...", C_.astype(float), u)
    usq = (u * u).sum(0)
    return W_.reshape((-1,) + (1,) * rho.ndim) * rho * (
        1 + cu / CS2 + 0.5 * cu * cu / CS2 ** 2 - 0.5 * usq / CS2)


class MiniLattice:
    def __init__(self, nx, ny, nz, *, wall_y=0, wall_z=0, tau_r=1.0, tau_b=None, sigma=0.0,
                 beta=0.7, A_nc=0.0, h_min=3.0, h_cut=None, g=(0, 0, 0), kolmogorov_amp=0.0,
                 wall_u=0.0, model="colour", G_sc=0.0):
        self.n = (nz, ny, nx)
        self.wall_y, self.wall_z = bool(wall_y), bool(wall_z)
        self.tau_r = tau_r
        self.tau_b = tau_r if tau_b is None else tau_b
        self.sigma, self.beta = sigma, beta
        self.A_nc, self.h_min = A_nc, h_min
        self.h_cut = 2 * h_min if h_cut is None else h_cut
        self.g = np.asarray(g, dtype=float)
        self.kamp = kolmogorov_amp
        self.wall_u = float(wall_u)
        self.shan_chen = model == "shan_chen"
        self.G_sc = float(G_sc)
        z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        self.X, self.Y, self.Z = x, y, z

    # --- fields ----------------------------------------------------------------
    def set_fields(self, rho_r, rho_b, u=None):
        u = np.zeros((3,) + self.n) if u is None else np.asarray(u, float)
        self.fr = equilibrium(np.asarray(rho_r, float), u)
        self.fb = equilibrium(np.asarray(rho_b, float), u)
        self.phi_lag = (rho_r - rho_b) / (rho_r + rho_b)

    def _outside(self, dy, dz):
        """mask of nodes whose neighbour at (y+dy, z+dz) is outside the fluid."""
        m = np.zeros(self.n, dtype=bool)
        nz, ny, _ = self.n
        if self.wall_y:
            m |= (self.Y + dy < 0) | (self.Y + dy >= ny)
        if self.wall_z:
            m |= (self.Z + dz < 0) | (self.Z + dz >= nz)
        return m

    def _shift_from(self, a, c):
        """value of field a at x - c (periodic roll), array [z, y, x]."""
        return np.roll(a, shift=(c[2], c[1], c[0]), axis=(0, 1, 2))

    def stream(self):
        gr = np.empty_like(self.fr)
        gb = np.empty_like(self.fb)
        for i, c in enumerate(C_):
            out = self._outside(-c[1], -c[2])
            gr[i] = np.where(out, self.fr[OPP_[i]], self._shift_from(self.fr[i], c))
            gb[i] = np.where(out, self.fb[OPP_[i]], self._shift_from(self.fb[i], c))
        if self.wall_y and self.wall_u != 0.0:
            # sliding y-walls (+U at the top, -U at the bottom, along x): a link that
            # came back from a wall moving with u_w gains 6 w_i rho_k c_i.u_w
            ny = self.n[1]
            rr, rb = gr.sum(0), gb.sum(0)
            for i, c in enumerate(C_):
                uw = np.where(self.Y - c[1] >= ny, self.wall_u,
                              np.where(self.Y - c[1] < 0, -self.wall_u, 0.0))
                gr[i] = gr[i] + 6.0 * W_[i] * rr * c[0] * uw
                gb[i] = gb[i] + 6.0 * W_[i] * rb * c[0] * uw
        return gr, gb

    def grad(self, phi):
        G = np.zeros((3,) + self.n)
        for i, c in enumerate(C_):
            if not c.any():
                continue
            nb = self._shift_from(phi, -c)                  # phi(x + c)
            nb = np.where(self._outside(c[1], c[2]), phi, nb)
            for a in range(3):
                G[a] += 3 * W_[i] * c[a] * nb
        return G

    # --- near contact ----------------------------------------------------------
    def _interp(self, fld, node, off):
        """trilinear value at node + off (cell and weights from the offset)."""
        nz, ny, nx = self.n
        dims = [(nx, False), (ny, self.wall_y), (nz, self.wall_z)]
        lo, hi, fr = [], [], []
        for a, (n, walled) in enumerate(dims):
            fl = math.floor(off[a])
            b, f = node[a] + fl, off[a] - fl
            if walled:
                if b < 0 or b > n - 1 or (b == n - 1 and f > 0):
                    return None
                if n == 1:
                    lo.append(0); hi.append(0); fr.append(0.0)
                    continue
                if b == n - 1:
                    b, f = n - 2, 1.0
                lo.append(b); hi.append(b + 1); fr.append(f)
            else:
                lo.append(b % n); hi.append((b + 1) % n); fr.append(f)
        v = 0.0
        for cz in (0, 1):
            for cy in (0, 1):
                for cx in (0, 1):
                    wgt = ((fr[0] if cx else 1 - fr[0]) * (fr[1] if cy else 1 - fr[1])
                           * (fr[2] if cz else 1 - fr[2]))
                    v += wgt * fld[hi[2] if cz else lo[2], hi[1] if cy else lo[1],
                                   hi[0] if cx else lo[0]]
        return v

    def _Ah(self, h):
        if h <= self.h_min:
            return self.A_nc
        if h >= self.h_cut:
            return 0.0
        return self.A_nc * ((self.h_min / h) ** 3 - (self.h_min / self.h_cut) ** 3) / (
            1 - (self.h_min / self.h_cut) ** 3)

    def nc_force(self, phi_ray, G):
        """A_h measured on phi_ray (its own gradient gives the ray direction) times G."""
        F = np.zeros((3,) + self.n)
        if self.A_nc == 0:
            return F
        Gr = self.grad(phi_ray)
        gm = np.sqrt((Gr * Gr).sum(0))
        ts = [-1 + 0.5 * s for s in range(int(math.floor(2 * (self.h_cut + 3))) + 1)]
        for z, y, x in zip(*np.nonzero(gm >= 1e-3)):
            nrm = -Gr[:, z, y, x] / gm[z, y, x]
            vals = []
            for t in ts:
                v = self._interp(phi_ray, (x, y, z), (t * nrm[0], t * nrm[1], t * nrm[2]))
                if v is None:
                    break
                if abs(v) > 1e-5:          # samples within 1e-5 of zero carry no sign
                    vals.append((t, v))
            t_d = t_u = None
            for (t0, v0), (t1, v1) in zip(vals, vals[1:]):
                if t_d is None and v0 > 0 > v1:
                    t_d = t0 + (t1 - t0) * v0 / (v0 - v1)
                elif t_d is not None and v0 < 0 < v1:
                    t_u = t0 + (t1 - t0) * v0 / (v0 - v1)
                    break
            if t_d is not None and t_u is not None:
                F[:, z, y, x] = self._Ah(t_u - t_d) * G[:, z, y, x]
        return F

    # --- one step ----------------------------------------------------------------
    def step(self, nsteps=1):
        Cf = C_.astype(float)
        for _ in range(nsteps):
            gr, gb = self.stream()
            rr, rb = gr.sum(0), gb.sum(0)
            f = gr + gb
            rho = rr + rb
            j = np.einsum("ia,i...->a...", Cf, f)
            phi = (rr - rb) / rho
            G = self.grad(phi)
            F = np.zeros((3,) + self.n)
            F[0] += self.g[0] + self.kamp * np.sin(2 * np.pi * self.Y / self.n[1])
            F[1] += self.g[1]
            F[2] += self.g[2]
            nu_r, nu_b = CS2 * (self.tau_r - 0.5), CS2 * (self.tau_b - 0.5)
            nu = 1.0 / ((rr / rho) / nu_r + (rb / rho) / nu_b)
            om = 2 * CS2 / (2 * nu + CS2)
            if self.shan_chen:
                # cohesive shifts F^k / rho_k = -G sum_i w_i rho_kbar(x + c_i) c_i (a
                # neighbour beyond a wall takes the node's own density); per-species
                # BGK towards f^eq(rho_k, u) plus the EDM source of F^k + (rho_k/rho) F
                u = j / rho
                sr = np.zeros((3,) + self.n)
                sb = np.zeros((3,) + self.n)
                for i, c in enumerate(C_):
                    if not c.any():
                        continue
                    out = self._outside(c[1], c[2])
                    nr = np.where(out, rr, self._shift_from(rr, -c))
                    nb = np.where(out, rb, self._shift_from(rb, -c))
                    for a in range(3):
                        sr[a] -= self.G_sc * W_[i] * nb * c[a]
                        sb[a] -= self.G_sc * W_[i] * nr * c[a]
                er0, eb0 = equilibrium(rr, u), equilibrium(rb, u)
                er1 = equilibrium(rr, u + sr + F / rho)
                eb1 = equilibrium(rb, u + sb + F / rho)
                self.fr = (1 - om) * gr + om * er0 + (er1 - er0)
                self.fb = (1 - om) * gb + om * eb0 + (eb1 - eb0)
                Ftot = rr * sr + rb * sb + F
                self.phi_lag = phi
                self.last = {"rho_r": rr, "rho_b": rb, "phi": phi, "u": (j + 0.5 * Ftot) / rho,
                             "F": Ftot, "G": G}
                continue
            F += self.nc_force(self.phi_lag, G)
            u = j / rho
            fe = equilibrium(rho, u)
            S = equilibrium(rho, u + F / rho) - fe
            f1 = f - om * (f - fe) + S
            gm = np.sqrt((G * G).sum(0))
            ok = gm >= 1e-6
            safe = np.where(ok, gm, 1.0)
            cg = np.einsum("ia,a...->i...", Cf, G)
            A = 4.5 * om * self.sigma
            pert = 0.5 * A * gm * (W_[:, None, None, None] * cg * cg / (safe * safe)
                                   - B_[:, None, None, None])
            f2 = f1 + np.where(ok, pert, 0.0)
            cn = np.sqrt((C_ * C_).sum(1)).astype(float)
            cn[cn == 0] = 1.0
            cos = np.where(ok, cg / (cn[:, None, None, None] * safe), 0.0)
            seg = self.beta * (rr * rb / rho) * W_[:, None, None, None] * cos
            self.fr = (rr / rho) * f2 + seg
            self.fb = (rb / rho) * f2 - seg
            self.phi_lag = phi
            self.last = {"rho_r": rr, "rho_b": rb, "phi": phi, "u": (j + 0.5 * F) / rho,
                         "F": F, "G": G}
