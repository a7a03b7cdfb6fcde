"""Seeded synthetic inputs for the EM-PIC hot path.

This module is the only code that both sides of every comparison share: the
FP64 CPU oracle (``oracle/``) and the CUDA library.  It produces input data
only -- grids, initial particle positions and momenta, random test fields --
and contains none of the arithmetic of the PIC method (no gather, push,
deposit, smoothing or field solve).

Random numbers come from one counter-based generator, SplitMix64
(G. L. Steele, D. Lea, C. H. Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014; the constants are those of the published
reference implementation), turned into uniforms on [0, 1) with 53 bits and
into normals with the Box-Muller transform (cos branch only, so that each
normal deviate has its own pair of counters).  Draw number ``c`` of stream
``seed`` is ``splitmix64(seed + (c + 1) * GAMMA)``, so any particle can be
regenerated on its own from its index.  The CUDA loader implements the same
published definitions independently.

Particle loading follows the species input of the paper's appendix (input
sections ``nl_species`` / ``nl_profile``): ``num_par_x`` particles per cell
direction on a regular sub-lattice, thermal spread ``vth`` read as the
standard deviation of each momentum component u = p/(m c), fluid momentum
``vfl``.  Particle ``p`` is sub-lattice point ``s`` of cell ``c`` with
``p = c * ppc + s``, cells in x1-fastest order, sub-lattice points in
x1-fastest order.
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
MIX1 = np.uint64(0xBF58476D1CE4E5B9)
MIX2 = np.uint64(0x94D049BB133111EB)
_U53 = 1.0 / 9007199254740992.0  # 2**-53


def splitmix64(seed: int, counter) -> np.ndarray:
    """Output number ``counter`` (0-based, array) of the SplitMix64 stream ``seed``."""
    c = np.asarray(counter, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (c + np.uint64(1)) * GAMMA
        z = (z ^ (z >> np.uint64(30))) * MIX1
        z = (z ^ (z >> np.uint64(27))) * MIX2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, counter) -> np.ndarray:
    """Uniform double on [0, 1): top 53 bits of the SplitMix64 output."""
    return (splitmix64(seed, counter) >> np.uint64(11)).astype(np.float64) * _U53


def normal(seed: int, counter) -> np.ndarray:
    """Standard normal deviate number ``counter``: Box-Muller on draws 2c, 2c+1."""
    c = np.asarray(counter, dtype=np.uint64)
    u1 = 1.0 - uniform01(seed, np.uint64(2) * c)          # (0, 1]
    u2 = uniform01(seed, np.uint64(2) * c + np.uint64(1))  # [0, 1)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


# ----------------------------------------------------------------------------
# Problem descriptions
# ----------------------------------------------------------------------------

@dataclass
class Grid:
    """Simulation box in normalised units (t in 1/w_p, x in c/w_p)."""
    ndim: int
    nx: tuple                      # cells per direction (3 entries; nx[2] = 1 in 2D)
    dx: tuple                      # cell size per direction
    xmin: tuple = (0.0, 0.0, 0.0)
    dt: float = 0.0
    e0: tuple = (0.0, 0.0, 0.0)    # constant external fields
    b0: tuple = (0.0, 0.0, 0.0)
    smooth_level: tuple = (0, 0, 0)
    smooth_w: tuple = ((1.0, 2.0, 1.0),) * 3
    rho_bg: float = 1.0            # fixed neutralising ion background density
    init_e_gauss_x1: bool = False  # initial E1 from the discrete Gauss law along x1
    move_window: bool = False      # window moving at c in x1 (x1 open; periodic in x2, x3)
    window_start: float = 0.0      # time from which the window moves (before it: x1 open, static)
    deposit: str = "vb"            # current deposit: "vb" (TRISTAN / Villasenor-Buneman) or "isis" (2D)
    coords: str = "cartesian"      # "cylindrical": 2D r-z (x1 = z, x2 = r), xmin[1] = -dx[1]/2

    @property
    def ncells(self) -> int:
        return int(self.nx[0]) * int(self.nx[1]) * int(self.nx[2])

    @property
    def dvol(self) -> float:
        v = self.dx[0] * self.dx[1]
        return v * self.dx[2] if self.ndim == 3 else v


@dataclass
class Species:
    rqm: float = -1.0              # m/q in units of m_e/e; electrons -1
    ppc: tuple = (1, 1, 1)         # num_par_x
    uth: tuple = (0.0, 0.0, 0.0)   # vth, std-dev of each u component
    ufl: tuple = (0.0, 0.0, 0.0)   # vfl
    density: float = 1.0           # uniform density in units of n0
    seed: int = 0
    # sinusoidal x1 displacement: x1 -> x1 + (delta/k) cos(k (x1 - xmin1)),
    # giving density ~ 1 + delta sin(k x1) to first order
    perturb_delta: float = 0.0
    perturb_k: float = 0.0
    # density profile (nl_num_x / nl_profile): per direction None or (x points,
    # f values) of a piecewise-linear function, constant beyond its ends; the
    # density is density * prod_d f_d(x_d).  A particle's charge is scaled by
    # the profile at its initial position; no particle is created where the
    # density is not above den_min.
    profile: tuple = None
    den_min: float = 0.0

    @property
    def ppc_total(self) -> int:
        return int(self.ppc[0]) * int(self.ppc[1]) * int(self.ppc[2])


@dataclass
class Laser:
    """A pulse (the thesis' pulse section): wavetype 1 moves in +x1, 2 in +x2;
    vosc = peak normalised vector potential a0, rkkp = wavenumber k (= omega0
    / omega_p), w0 = spot size, rise / length / fall = envelope distances,
    start = distance of the pulse front from the side of the box it moves
    towards, pol = polarisation angle in degrees from the in-plane transverse
    axis towards x3, phase, offset = transverse offset of the axis from the box
    centre, focus = distance of the focal plane from that side (None: the
    waist profile everywhere)."""
    vosc: float = 1.0
    rkkp: float = 10.0
    w0: float = 4.0
    rise: float = 1.0
    fall: float = 1.0
    length: float = 0.0
    start: float = 1.0
    pol: float = 0.0
    phase: float = 0.0
    offset: tuple = (0.0, 0.0)
    wavetype: int = 1
    focus: object = None
    antenna: bool = False          # enters through the lower x1 boundary; its front crosses it at time `start`


def courant_dt(dx, ndim: int, frac: float = 0.99) -> float:
    """``frac`` times the multi-dimensional Courant limit 1/sqrt(sum dx_d^-2)."""
    return frac / math.sqrt(sum(1.0 / (dx[d] * dx[d]) for d in range(ndim)))


def macro_charge(grid: Grid, sp: Species) -> float:
    """Charge per macroparticle so that ppc particles carry density ``sp.density``."""
    sign = -1.0 if sp.rqm < 0 else 1.0
    return sign * sp.density * grid.dvol / sp.ppc_total


def n_particles(grid: Grid, sp: Species) -> int:
    return grid.ncells * sp.ppc_total


def profile_weight(sp: Species, x):
    """Product of the piecewise-linear profile functions at positions x[n,3]
    (1 where a direction has none); None for a species without a profile."""
    if sp.profile is None:
        return None
    x = np.asarray(x, dtype=np.float64)
    w = np.ones(x.shape[0])
    for d, prof in enumerate(sp.profile):
        if prof is None:
            continue
        xs, fs = (np.asarray(v, dtype=np.float64) for v in prof)
        w = w * np.interp(x[:, d], xs, fs)
    return w


def load_weighted(grid: Grid, sp: Species):
    """The loader with the density profile applied: (x, u, w, ids) of the
    particles that are created (density * w > den_min), ids = their lattice
    indices.  w is None for a species without a profile (all of them kept)."""
    x, u = load_particles(grid, sp)
    w = profile_weight(sp, x)
    ids = np.arange(x.shape[0], dtype=np.int64)
    if w is None:
        return x, u, None, ids
    keep = sp.density * w > sp.den_min
    return np.ascontiguousarray(x[keep]), np.ascontiguousarray(u[keep]), np.ascontiguousarray(w[keep]), ids[keep]


def load_particles(grid: Grid, sp: Species, index=None):
    """Initial x^0 (global, FP64) and u^{-1/2} (FP64) of the particles ``index``.

    ``index`` defaults to all particles.  Returns (x[n,3], u[n,3]); in 2D the
    third position column is 0.
    """
    n_total = n_particles(grid, sp)
    if index is None:
        index = np.arange(n_total, dtype=np.int64)
    p = np.asarray(index, dtype=np.int64)
    ppc = sp.ppc_total
    cell = p // ppc
    sub = p % ppc
    nx, ny = int(grid.nx[0]), int(grid.nx[1])
    ci = cell % nx
    cj = (cell // nx) % ny
    ck = cell // (nx * ny)
    npx, npy = int(sp.ppc[0]), int(sp.ppc[1])
    si = sub % npx
    sj = (sub // npx) % npy
    sk = sub // (npx * npy)
    x = np.zeros((p.size, 3), dtype=np.float64)
    for d, (c, s) in enumerate(((ci, si), (cj, sj), (ck, sk))):
        if d >= grid.ndim:
            break
        off = (s.astype(np.float64) + 0.5) / float(sp.ppc[d])
        x[:, d] = grid.xmin[d] + (c.astype(np.float64) + off) * grid.dx[d]
    if sp.perturb_delta != 0.0:
        L = grid.nx[0] * grid.dx[0]
        x1 = x[:, 0] + (sp.perturb_delta / sp.perturb_k) * np.cos(sp.perturb_k * (x[:, 0] - grid.xmin[0]))
        x1 = np.where(x1 >= grid.xmin[0] + L, x1 - L, x1)
        x1 = np.where(x1 < grid.xmin[0], x1 + L, x1)
        x[:, 0] = x1
    u = np.empty((p.size, 3), dtype=np.float64)
    pu = p.astype(np.uint64)
    for d in range(3):
        u[:, d] = sp.ufl[d] + sp.uth[d] * normal(sp.seed, np.uint64(3) * pu + np.uint64(d)) if sp.uth[d] != 0.0 \
            else np.full(p.size, float(sp.ufl[d]))
    return x, u


def random_fields(grid: Grid, seed: int, amp: float = 0.1, ncomp: int = 6):
    """``ncomp`` grid arrays [nz][ny][nx] of uniform noise on [-amp, amp)."""
    shape = (int(grid.nx[2]), int(grid.nx[1]), int(grid.nx[0]))
    n = int(np.prod(shape))
    out = []
    for c in range(ncomp):
        cnt = np.arange(n, dtype=np.uint64) + np.uint64(c * n)
        out.append((2.0 * uniform01(seed, cnt) - 1.0).reshape(shape) * amp)
    return out


# ----------------------------------------------------------------------------
# The five workloads of the hot path (sizes and physics parameters)
# ----------------------------------------------------------------------------

def config0(seed: int = 20001):
    """2D3V periodic electron plasma, 64x64 cells, 16 ppc, 1% x1 perturbation, 100 steps."""
    dx = (0.1, 0.1, 1.0)
    g = Grid(ndim=2, nx=(64, 64, 1), dx=dx, dt=courant_dt(dx, 2), init_e_gauss_x1=True)
    k = 2.0 * math.pi / (64 * 0.1)
    s = Species(rqm=-1.0, ppc=(4, 4, 1), uth=(0.01, 0.01, 0.01), seed=seed,
                perturb_delta=0.01, perturb_k=k)
    return g, [s], 100


def config1(seed: int = 20002, vacuum_gap: float = None):
    """2D3V laser wakefield: 2048 x 256 cells, dx1 = 0.05, dx2 = 0.2, 8 ppc (4 x 2)
    cold uniform electrons, window moving at c in x1, a pulse a0 = 2,
    omega0/omega_p = 10, spot 4, polarised in x2, with the thesis' polynomial
    rise and fall of 1.945 each: the intensity f^2 of the envelope then has a
    full width at half maximum of 1.5 (the duration given); front 1.0 behind
    the +x1 edge; 2000 steps.  The plasma fills the window from the start; with
    ``vacuum_gap`` it begins that far ahead of the pulse front instead (a
    density profile: vacuum, then density 1), so the window meets it as it
    moves."""
    dx = (0.05, 0.2, 1.0)
    g = Grid(ndim=2, nx=(2048, 256, 1), dx=dx, dt=courant_dt(dx, 2), move_window=True)
    s = Species(rqm=-1.0, ppc=(4, 2, 1), uth=(0.0, 0.0, 0.0), seed=seed)
    las = Laser(vosc=2.0, rkkp=10.0, w0=4.0, rise=1.945, length=0.0, fall=1.945, start=1.0)
    if vacuum_gap is not None:
        edge = g.nx[0] * dx[0] - las.start + vacuum_gap  # lab x1 where the plasma begins
        s = dataclasses.replace(s, profile=(((0.0, edge, edge + 1e-9, 1e9), (0.0, 0.0, 1.0, 1.0)), None),
                                den_min=1e-6)
    return g, [s], las, 2000


def beam_particles(grid: Grid, n: int, center, sigma1: float, sigma_r: float, gamma: float, peak_density: float,
                   seed: int):
    """A bi-Gaussian electron driver of n macroparticles: x1 ~ N(center1,
    sigma1), x2, x3 ~ N(center, sigma_r) (draw 3p + d of the SplitMix64 /
    Box-Muller stream ``seed`` for particle p), longitudinal x1 clipped to the
    box, transverse wrapped (periodic); every u = (sqrt(gamma^2 - 1), 0, 0).
    The macro-charge makes the peak density ``peak_density``: total charge
    -peak (2 pi)^(d/2) sigma1 sigma_r^(d-1).  Returns (x, u, q)."""
    p = np.arange(n, dtype=np.uint64)
    x = np.zeros((n, 3))
    for d in range(grid.ndim):
        z = normal(seed, np.uint64(3) * p + np.uint64(d))
        sig = sigma1 if d == 0 else sigma_r
        x[:, d] = center[d] + sig * z
        lo, L = grid.xmin[d], grid.nx[d] * grid.dx[d]
        if d == 0:
            x[:, 0] = np.clip(x[:, 0], lo, np.nextafter(lo + L, lo))
        else:
            x[:, d] = lo + np.mod(x[:, d] - lo, L)
    u = np.zeros((n, 3))
    u[:, 0] = math.sqrt(gamma * gamma - 1.0)
    vol = (2.0 * math.pi) ** (grid.ndim / 2.0) * sigma1 * sigma_r ** (grid.ndim - 1)
    q = -peak_density * vol / n
    return x, u, q


def config2(seed: int = 20003, nx=(256, 128, 128), nbeam: int = 4194304):
    """3D3V beam-driven wake: 256 x 128 x 128 cells, dx1 = 0.05, dx2 = dx3 = 0.1,
    8 ppc (2 x 2 x 2) cold electrons plus a bi-Gaussian driver (gamma = 60000,
    sigma_z = 1, sigma_r = 0.3, peak n_b/n_0 = 5, ``nbeam`` macroparticles)
    centred 3 behind the +x1 edge on the axis, window moving at c; 500 steps.
    Returns (grid, [plasma, beam species], (x, u, q) of the beam, steps)."""
    dx = (0.05, 0.1, 0.1)
    g = Grid(ndim=3, nx=tuple(nx), dx=dx, dt=courant_dt(dx, 3), move_window=True)
    plasma = Species(rqm=-1.0, ppc=(2, 2, 2), uth=(0.0, 0.0, 0.0), seed=seed)
    beam = Species(rqm=-1.0, ppc=(0, 0, 0), seed=seed + 1)
    L = [g.nx[d] * g.dx[d] for d in range(3)]
    centre = (L[0] - 3.0, 0.5 * L[1], 0.5 * L[2])
    bx, bu, bq = beam_particles(g, nbeam, centre, 1.0, 0.3, 60000.0, 5.0, seed + 1)
    return g, [plasma, beam], (bx, bu, bq), 500


def config3(ppc_total: int = 8, seed: int = 20004, nx=(512, 256, 256)):
    """3D3V periodic thermal plasma, 512x256x256 cells, u_th = 0.05, 200 steps."""
    lattice = {1: (1, 1, 1), 2: (2, 1, 1), 4: (2, 2, 1), 8: (2, 2, 2), 16: (4, 2, 2)}[ppc_total]
    dx = (0.1, 0.1, 0.1)
    g = Grid(ndim=3, nx=tuple(nx), dx=dx, dt=courant_dt(dx, 3))
    s = Species(rqm=-1.0, ppc=lattice, uth=(0.05, 0.05, 0.05), seed=seed)
    return g, [s], 200


def config4(seed: int = 20005, nsims: int = 64):
    """Batched parameter scan of 2D3V laser-wakefield runs: ``nsims``
    independent members of uneven size drawn from the seed, 500 steps each.

    Draw i uses counters 8i .. 8i+4 of the SplitMix64 stream ``seed``: grid
    nx1 in {128, 256, 512, 1024} x nx2 in {64, 128, 256, 512}, ppc in
    {4, 8, 16, 32} (lattices 2x2, 4x2, 4x4, 8x4), plasma density scale n
    U[0.5, 2) in units of the density n0 that sets w_p, and laser strength a0
    U[0.5, 3); dx1 = 0.05, dx2 = 0.2, dt = 0.99 of the Courant limit.  Each
    member is a wakefield run like the single 2D one: cold electrons of density
    n over a fixed ion background of the same density, filling a window that
    moves at c in x1 (open x1, fresh plasma injected at the front), and a pulse
    placed in the box, polarised in x2, with omega0 = 10 w_p (omega0 over the
    member's own plasma frequency: 10 n^-1/2), the polynomial rise and fall of
    1.945 each, front 1.0 behind the +x1 edge and spot min(4, a quarter of the
    transverse box).
    Returns a list of (Grid, [Species], Laser) and the step count.
    """
    lattices = {4: (2, 2, 1), 8: (4, 2, 1), 16: (4, 4, 1), 32: (8, 4, 1)}
    dx = (0.05, 0.2, 1.0)
    dt = courant_dt(dx, 2)
    out = []
    for i in range(nsims):
        r = uniform01(seed, np.arange(8 * i, 8 * i + 5, dtype=np.uint64))
        nx1 = (128, 256, 512, 1024)[int(r[0] * 4)]
        nx2 = (64, 128, 256, 512)[int(r[1] * 4)]
        ppc = (4, 8, 16, 32)[int(r[2] * 4)]
        dens = 0.5 + 1.5 * float(r[3])
        a0 = 0.5 + 2.5 * float(r[4])
        g = Grid(ndim=2, nx=(nx1, nx2, 1), dx=dx, dt=dt, rho_bg=dens, move_window=True)
        s = Species(rqm=-1.0, ppc=lattices[ppc], density=dens, seed=seed + 1000 * (i + 1))
        las = Laser(vosc=a0, rkkp=10.0, w0=min(4.0, 0.25 * nx2 * dx[1]), rise=1.945, length=0.0, fall=1.945,
                    start=1.0)
        out.append((g, [s], las))
    return out, 500


def inject_column(grid: Grid, sp: Species, xmin1: float, first_index: int):
    """Fresh plasma for the front column (cell index nx1 - 1) of a window whose
    x1 edge is now ``xmin1``: the particles of the column's cells in cell order
    (x3 slowest), each cell's sub-lattice as the loader's, momenta from draws
    of global particle indices first_index, first_index + 1, ... (the loader's
    stream continued).  Returns (x[n,3], u[n,3])."""
    nx, ny = int(grid.nx[0]), int(grid.nx[1])
    nz = int(grid.nx[2]) if grid.ndim == 3 else 1
    ppc = sp.ppc_total
    if ppc == 0:  # a species without a lattice (a beam) gets no fresh plasma
        return np.zeros((0, 3)), np.zeros((0, 3))
    k = np.arange(ny * nz * ppc, dtype=np.int64)
    col = k // ppc
    sub = k % ppc
    cj, ck = col % ny, col // ny
    npx, npy = int(sp.ppc[0]), int(sp.ppc[1])
    si, sj, sk = sub % npx, (sub // npx) % npy, sub // (npx * npy)
    x = np.zeros((k.size, 3))
    x[:, 0] = xmin1 + ((nx - 1) + (si + 0.5) / float(sp.ppc[0])) * grid.dx[0]
    x[:, 1] = grid.xmin[1] + (cj + (sj + 0.5) / float(sp.ppc[1])) * grid.dx[1]
    if grid.ndim == 3:
        x[:, 2] = grid.xmin[2] + (ck + (sk + 0.5) / float(sp.ppc[2])) * grid.dx[2]
    gidx = np.uint64(first_index) + k.astype(np.uint64)
    u = np.zeros((k.size, 3))
    for d in range(3):
        u[:, d] = sp.ufl[d] + sp.uth[d] * normal(sp.seed, np.uint64(3) * gidx + np.uint64(d)) if sp.uth[d] != 0.0 \
            else np.full(k.size, float(sp.ufl[d]))
    return x, u


# ---------------------------------------------------------------- r-z geometry
def cyl_grid(nz: int, nr: int, dz: float, dr: float, zmin: float = 0.0, frac: float = 0.99,
             b0=(0.0, 0.0, 0.0), e0=(0.0, 0.0, 0.0), rho_bg: float = 0.0) -> Grid:
    """2D cylindrically symmetric box: x1 = z (periodic), x2 = r with the axis
    through the middle of the first cell (xmin[1] = -dr/2) and a wall at
    r = (nr - 1/2) dr."""
    return Grid(ndim=2, nx=(int(nz), int(nr), 1), dx=(float(dz), float(dr), 1.0), xmin=(float(zmin), -0.5 * dr, 0.0),
                dt=cyl_courant_dt(dz, dr, frac), e0=tuple(e0), b0=tuple(b0), rho_bg=rho_bg,
                coords="cylindrical")


# Largest eigenvalue of the radial part of the r-z field solve (the Etheta, Bz,
# Br family with the axis rule), in units of 4/dr^2: a mode bound to the axis,
# the same for every nr >= 10 (smaller grids have a smaller one).  The leapfrog
# is stable for dt < 1 / sqrt(1/dz^2 + CYL_RADIAL_EIG / dr^2).
CYL_RADIAL_EIG = 1.2105


def cyl_courant_dt(dz: float, dr: float, frac: float = 0.99) -> float:
    return frac / math.sqrt(1.0 / dz ** 2 + CYL_RADIAL_EIG / dr ** 2)


def load_cylindrical(grid: Grid, sp: Species, index=None):
    """Lattice particles of an r-z box: the Cartesian lattice of the (z, r)
    cells with r measured from the lower edge -dr/2 of the first cell, and the
    points of that cell below the axis reflected to -r.  Returns (x[n,3] with
    columns z, r, 0; u[n,3] = (pz, pr, ptheta))."""
    assert grid.coords == "cylindrical"
    x, u = load_particles(grid, sp, index)
    x[:, 1] = np.abs(x[:, 1])
    return x, u


def config_cyl(seed: int = 20006, nz: int = 2048, nr: int = 512, ppc=(2, 2, 1), uth: float = 0.05):
    """r-z thermal plasma column (uniform density 1 out to the wall, fixed ion
    background): nz x nr cells of 0.1 c/w_p, electrons."""
    g = cyl_grid(nz, nr, 0.1, 0.1, rho_bg=1.0)
    sp = Species(rqm=-1.0, ppc=tuple(ppc), uth=(uth, uth, uth), density=1.0, seed=seed)
    return g, [sp], 200

