"""FP64 CPU oracle of the 2D cylindrically symmetric (r-z) mode (test infrastructure only).

Only ``tests/`` may import this module.  It follows the thesis' section on
the 2D cylindrically symmetric algorithms (ch. 3):

* grid: the 2D Cartesian grid with x1 -> z, x2 -> r and E1, E2, E3 -> Ez, Er,
  Etheta (B and j likewise); the axis runs through the middle of the first
  cell, so node row j sits at r_j = (j - 1/2) dr and half row j + 1/2 at
  r = j dr (the axis is half row 1/2 of row 0);
* field solve: the Cartesian 2D stencils, except the z components, whose
  r-derivatives carry the radius (eq. "2d-field-solve-cyl"), and Bz on the
  axis, advanced from the integral form of Faraday's law around a loop half a
  cell off the axis (eq. "2d-field-solve-cyl-b1-axis"); axial parity:
  components perpendicular to the axis are odd in r, parallel ones and rho
  even;
* push: the Cartesian Boris update of (pz, pr, ptheta); then a "pseudo" 3D
  move from (z, r, 0) and a rotation back into the r-z plane (eqs.
  "2d-cyl-position-update-1..3"), ptheta from the conservation of angular
  momentum of a ring particle;
* deposit: the 2D Cartesian current deposit of the particles' current I,
  then j = I / V(r) with V(r) = r dr dz per radian.

The Cartesian pieces (gather, Boris, Villasenor-Buneman deposit) are the
pinned routines of ``oracle`` run on an index grid of nz columns and nr + 1
rows whose x2 origin is -dr/2.

Readings of points the thesis leaves open (also listed in the design notes):

C1  The printed Ez update subtracts r_{i2-1/2} B_Theta,i1-1,i2; the r-derivative
    of r B_Theta at (i1 + 1/2, i2) needs B_Theta at (i1 + 1/2, i2 - 1/2), i.e.
    B_Theta,i1,i2-1, which is what is used.
C2  A particle is a ring; a uniform density needs a ring charge proportional to
    its radius: each particle carries q * w * r_load (w: its own weight, 1
    unless given), constant in time.  Totals (charge, energies) are over the
    full 2 pi.
C3  V(r) is taken at the radius of the quantity: r_j dr dz for rho, jz and
    jtheta on node rows, j dr * dr dz for jr on half rows; jr on the axis
    (j = 0) is 0 by parity.
C4  Row 0 (r = -dr/2) mirrors row 1: what the deposit puts on row 0 is folded
    onto row 1 with the parity sign (rho, jz: +; jtheta: -).
C5  Field rows at the axis: Ez_0 = Ez_1, Etheta_0 = -Etheta_1, Br_0 = -Br_1
    (mirror row), Er_0 = Btheta_0 = 0 (odd, on the axis), Bz_0 from the axis
    formula.
C6  The upper r boundary is the appendix's boundary type 5, "conducting
    boundary with particle absorption" (the lower one is type 20, the axial
    boundary of this mode): a perfectly conducting wall at node row nr,
    r_max = (nr - 1/2) dr, with Ez = Etheta = Br = 0 there and every field
    beyond it 0.  A particle whose move reaches r_max is
    absorbed: its path is deposited up to the wall (out-of-plane current for
    that fraction of the step) and its slot is kept with r = -1, u = 0.
C7  The out-of-plane current of a move uses ptheta before the rotation (the
    Cartesian deposit routine is reused unchanged).
C8  Lattice points of cell 0 below the axis are reflected to -r (input
    recipe, workload.load_cylindrical).
C9  Field energy: (1/2) sum F^2 V 2 pi with V = r dr dz at each component's
    radius; the on-axis half-row values (Bz_0) use the disc volume
    (dr/2)^2 / 2 * dz per radian; the mirror row and the wall row are left
    out.  Kinetic energy: sum 2 pi q w |rqm| (gamma - 1) -- q rqm > 0 for every
    species.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import boris as _boris
from . import deposit_vb as _deposit_vb
from . import gather as _gather

TWO_PI = 2.0 * math.pi


@dataclasses.dataclass
class _IndexGrid:
    """The Cartesian grid the pinned 2D routines run on (x1 = z, x2 = r)."""
    ndim: int
    nx: tuple
    dx: tuple
    xmin: tuple
    dt: float
    e0: tuple
    b0: tuple
    smooth_level: tuple = (0, 0, 0)
    smooth_w: tuple = ((1.0, 2.0, 1.0),) * 3
    rho_bg: float = 0.0


class CylState:
    """State of an r-z simulation: fields F[c][j, i] (c: Ez, Er, Etheta, Bz, Br,
    Btheta; rows j = 0..nr, row nr the wall), currents, and the species."""

    def __init__(self, nz, nr, dz, dr, dt, zmin=0.0, e0=(0.0, 0.0, 0.0), b0=(0.0, 0.0, 0.0), rho_bg=0.0):
        self.nz, self.nr, self.dz, self.dr, self.dt = int(nz), int(nr), float(dz), float(dr), float(dt)
        self.zmin = float(zmin)
        self.rho_bg = float(rho_bg)
        self.rmax = (self.nr - 0.5) * self.dr
        self.g = _IndexGrid(2, (self.nz, self.nr + 1, 1), (self.dz, self.dr, 1.0), (self.zmin, -0.5 * self.dr, 0.0),
                            self.dt, tuple(map(float, e0)), tuple(map(float, b0)))
        self.F = [np.zeros((self.nr + 1, self.nz)) for _ in range(6)]
        self.J = [np.zeros((self.nr + 1, self.nz)) for _ in range(3)]
        self.species = []
        self.steps = 0

    # radii
    def r_node(self, j):
        return (np.asarray(j, dtype=np.float64) - 0.5) * self.dr

    def r_half(self, j):
        return np.asarray(j, dtype=np.float64) * self.dr

    def add_species(self, x, u, q, rqm, w=None):
        """Particles at x[:, 0] = z, x[:, 1] = r (0 <= r < r_max), momenta u =
        (pz, pr, ptheta); ring charge q * w * r (reading C2)."""
        x = np.array(x, dtype=np.float64).reshape(-1, 3)
        u = np.array(u, dtype=np.float64).reshape(-1, 3)
        assert np.all(x[:, 1] >= 0.0) and np.all(x[:, 1] < self.rmax)
        x[:, 2] = 0.0
        w0 = np.ones(x.shape[0]) if w is None else np.array(w, dtype=np.float64)
        self.species.append({"x": x, "u": u, "w": w0 * x[:, 1], "q": float(q), "rqm": float(rqm)})

    # ------------------------------------------------------------ boundaries
    def boundary_fields(self):
        """Axis rows by parity (C5), the conducting wall and beyond (C6)."""
        Ez, Er, Et, Bz, Br, Bt = self.F
        Ez[0] = Ez[1]
        Et[0] = -Et[1]
        Br[0] = -Br[1]
        Er[0] = 0.0
        Bt[0] = 0.0
        n = self.nr
        Ez[n] = 0.0
        Et[n] = 0.0
        Br[n] = 0.0
        Er[n] = 0.0  # half row n + 1/2 lies beyond the wall
        Bz[n] = 0.0
        Bt[n] = 0.0

    # ------------------------------------------------------------ particles
    def push_species(self, sp, J):
        """Gather, Boris, pseudo-3D move + rotation, deposit of I, absorption."""
        g, dt = self.g, self.dt
        x, u, w = sp["x"], sp["u"], sp["w"]
        for p in range(x.shape[0]):
            z, r = x[p, 0], x[p, 1]
            if r < 0.0:  # absorbed earlier
                continue
            f = _gather(g, [c.reshape(1, self.nr + 1, self.nz) for c in self.F], np.array([z, r, 0.0]))
            un = _boris(u[p], f[:3], f[3:], sp["rqm"], dt)
            gam = math.sqrt(1.0 + un[0] * un[0] + un[1] * un[1] + un[2] * un[2])
            # eq. 2d-cyl-position-update-1: the move in 3D Cartesian space from (z, r, 0)
            zn = z + dt * un[0] / gam
            x2 = r + dt * un[1] / gam
            x3 = dt * un[2] / gam
            rn = math.hypot(x2, x3)  # eq. 2d-cyl-position-update-2
            qp = sp["q"] * w[p]
            v3 = un[2] / gam  # C7
            if rn >= self.rmax:  # C6: absorbed at the wall
                t = (self.rmax - r) / (rn - r)
                zc = z + t * (zn - z)
                d = _deposit_vb(g, np.array([z, r, 0.0]), np.array([zc, self.rmax, 0.0]), v3 * t, qp)
                for c in range(3):
                    J[c] += d[c][0]
                x[p] = (z, -1.0, 0.0)
                u[p] = 0.0
                continue
            d = _deposit_vb(g, np.array([z, r, 0.0]), np.array([zn, rn, 0.0]), v3, qp)
            for c in range(3):
                J[c] += d[c][0]
            # eq. 2d-cyl-position-update-3: momenta in the rotated frame; ptheta
            # from the conservation of angular momentum (r^n ptheta = r^n+1 ptheta')
            if rn > 0.0:
                pr = (un[1] * x2 + un[2] * x3) / rn
                pt = un[2] * r / rn
            else:
                pr, pt = math.hypot(un[1], un[2]), 0.0
            L = self.nz * self.dz
            zw = zn - L * math.floor((zn - self.zmin) / L)
            x[p] = (zw, rn, 0.0)
            u[p] = (un[0], pr, pt)

    def currents_to_density(self, J):
        """Deposited current (Cartesian area units, q dx / (dt dz dr)) to j = I / V(r):
        fold row 0 onto row 1 with the parity sign (C4), then divide by the
        radius of each component (C3)."""
        Jz, Jr, Jt = J
        Jz[1] += Jz[0]
        Jt[1] -= Jt[0]
        Jz[0] = 0.0
        Jt[0] = 0.0
        Jr[0] = 0.0
        rows = np.arange(1, self.nr + 1)
        Jz[1:] /= self.r_node(rows)[:, None]
        Jt[1:] /= self.r_node(rows)[:, None]
        Jr[1:] /= self.r_half(rows)[:, None]
        Jz[self.nr] = 0.0  # on the wall: no tangential field is advanced there
        Jt[self.nr] = 0.0
        Jr[self.nr] = 0.0

    # ------------------------------------------------------------ field solve
    def b_half(self):
        """B advanced by dt/2 from E (eqs. 2d-field-solve-b-part1 / -cyl / -cyl-b1-axis)."""
        Ez, Er, Et, Bz, Br, Bt = self.F
        h, dz, dr, n = 0.5 * self.dt, self.dz, self.dr, self.nr
        j = np.arange(1, n)
        rj = self.r_node(np.arange(n + 1))
        dEt_dz = (np.roll(Et, -1, axis=1) - Et) / dz
        dEr_dz = (np.roll(Er, -1, axis=1) - Er) / dz
        Bz_axis = Bz[0] - h * 4.0 * Et[1] / dr
        Bz[j] -= h * (rj[j + 1, None] * Et[j + 1] - rj[j, None] * Et[j]) / (self.r_half(j)[:, None] * dr)
        Bz[0] = Bz_axis
        Br[j] += h * dEt_dz[j]
        Bt[j] -= h * (dEr_dz[j] - (Ez[j + 1] - Ez[j]) / dr)
        self.boundary_fields()

    def e_full(self):
        """E advanced by dt from B and j (eqs. 2d-field-solve-e / -cyl, reading C1)."""
        Ez, Er, Et, Bz, Br, Bt = self.F
        Jz, Jr, Jt = self.J
        dt, dz, dr, n = self.dt, self.dz, self.dr, self.nr
        j = np.arange(1, n)
        rh = self.r_half(np.arange(n + 1))
        dBt_dz = (Bt - np.roll(Bt, 1, axis=1)) / dz
        dBr_dz = (Br - np.roll(Br, 1, axis=1)) / dz
        Ez[j] += dt * ((rh[j, None] * Bt[j] - rh[j - 1, None] * Bt[j - 1]) / (self.r_node(j)[:, None] * dr) - Jz[j])
        Er[j] += dt * (-dBt_dz[j] - Jr[j])
        Et[j] += dt * (dBr_dz[j] - (Bz[j] - Bz[j - 1]) / dr - Jt[j])
        self.boundary_fields()

    def step(self, n=1):
        for _ in range(n):
            self.boundary_fields()
            J = [np.zeros((self.nr + 1, self.nz)) for _ in range(3)]
            for sp in self.species:
                self.push_species(sp, J)
            self.currents_to_density(J)
            self.J = J
            self.b_half()
            self.e_full()
            self.b_half()
            self.steps += 1

    # ------------------------------------------------------------ diagnostics
    def rho(self):
        """Charge density of the particles on node rows (linear weights, row 0
        folded onto row 1, divided by r_j dz dr; C3/C4); background excluded."""
        Q = np.zeros((self.nr + 1, self.nz))
        for sp in self.species:
            x = sp["x"]
            live = x[:, 1] >= 0.0
            g1 = (x[live, 0] - self.zmin) / self.dz
            g2 = (x[live, 1] + 0.5 * self.dr) / self.dr
            i0, j0 = np.floor(g1), np.floor(g2)
            e1, e2 = g1 - i0, g2 - j0
            qp = sp["q"] * sp["w"][live]
            for c2 in (0, 1):
                for c1 in (0, 1):
                    wt = (e1 if c1 else 1.0 - e1) * (e2 if c2 else 1.0 - e2)
                    np.add.at(Q, ((j0 + c2).astype(int), (i0 + c1).astype(int) % self.nz), qp * wt)
        Q[1] += Q[0]
        Q[0] = 0.0
        rows = np.arange(1, self.nr + 1)
        Q[1:] /= self.r_node(rows)[:, None] * self.dz * self.dr
        return Q

    def div_e(self):
        """Discrete div E on node rows 1..nr-1: (Ez_i - Ez_i-1)/dz + (1/r_j)
        (r_j+1/2 Er_j - r_j-1/2 Er_j-1)/dr."""
        Ez, Er = self.F[0], self.F[1]
        j = np.arange(1, self.nr)
        dz_term = (Ez[j] - np.roll(Ez, 1, axis=1)[j]) / self.dz
        dr_term = (self.r_half(j)[:, None] * Er[j] - self.r_half(j - 1)[:, None] * Er[j - 1]) / (
            self.r_node(j)[:, None] * self.dr)
        return dz_term + dr_term

    def div_j(self):
        """The same divergence of j (continuity check)."""
        Jz, Jr = self.J[0], self.J[1]
        j = np.arange(1, self.nr)
        return (Jz[j] - np.roll(Jz, 1, axis=1)[j]) / self.dz + (
            self.r_half(j)[:, None] * Jr[j] - self.r_half(j - 1)[:, None] * Jr[j - 1]) / (self.r_node(j)[:, None] * self.dr)

    def gauss_residual(self):
        """div E - rho - rho_bg on node rows 1..nr-1."""
        return self.div_e() - self.rho()[1:self.nr] - self.rho_bg

    def div_b(self):
        """Discrete div B over the cells (i + 1/2, j + 1/2), j = 0..nr-1, in flux
        form: the axis cell (j = 0) is the disc of radius dr/2, whose side
        flux is 2 pi (dr/2) dz Br_1 and whose end flux is pi (dr/2)^2 dBz_0."""
        Bz, Br = self.F[3], self.F[4]
        out = np.empty((self.nr, self.nz))
        dBz = (np.roll(Bz, -1, axis=1) - Bz) / self.dz
        out[0] = 4.0 * Br[1] / self.dr + dBz[0]
        j = np.arange(1, self.nr)
        out[1:] = (self.r_node(j + 1)[:, None] * Br[j + 1] - self.r_node(j)[:, None] * Br[j]) / (
            self.r_half(j)[:, None] * self.dr) + dBz[j]
        return out

    def field_energy(self):
        """(1/2) sum F^2 V 2 pi (C9)."""
        n, dz, dr = self.nr, self.dz, self.dr
        vn = self.r_node(np.arange(1, n)) * dr * dz   # node rows 1..nr-1
        vh = self.r_half(np.arange(0, n)) * dr * dz   # half rows 0..nr-1
        vh[0] = 0.125 * dr * dr * dz                  # the axis disc (per radian)
        s = 0.0
        for c, half in ((0, False), (1, True), (2, False), (3, True), (4, False), (5, True)):
            f = self.F[c]
            if half:
                s += float(np.sum(f[0:n] ** 2 * vh[:, None]))
            else:
                s += float(np.sum(f[1:n] ** 2 * vn[:, None]))
        return 0.5 * s * TWO_PI

    def kinetic_energy(self):
        s = 0.0
        for sp in self.species:
            live = sp["x"][:, 1] >= 0.0
            u = sp["u"][live]
            s += sp["q"] * sp["rqm"] * float(np.sum(sp["w"][live] * (np.sqrt(1.0 + np.sum(u * u, axis=1)) - 1.0)))
        return s * TWO_PI

    def total_charge(self):
        return TWO_PI * sum(sp["q"] * float(np.sum(sp["w"][sp["x"][:, 1] >= 0.0])) for sp in self.species)
