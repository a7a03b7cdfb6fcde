"""FP64 CPU oracle of the EM-PIC step (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The C source ``pic_oracle.c`` is built
with gcc into ``oracle/_build/liboracle.so`` on first use (or by ``build()``).

Every function follows a passage of Hemker's thesis (arxiv 1503.00276), ch. 3:
field weighting eq. "2d-field-weighting-e3", Boris push eq. "momentum-update",
position update eq. "2d-position-update", TRISTAN / Villasenor-Buneman
current deposit (average of orthogonal moves, path split at cell faces), field
solve eqs. "2d-field-solve-b-part1/-e/-b-part2" and the 3D extension, and the
appendix's smoothing section (nl_smooth).  See the header of pic_oracle.c for
the readings of garbled passages and the list of pins.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import math
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_STAMP = os.path.join(_BUILD, "machine.txt")
_SRC = os.path.join(_HERE, "pic_oracle.c")
_lock = threading.Lock()
_lib = None

MAX_PASS = 8


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    same_machine = os.path.exists(_STAMP) and open(_STAMP).read().strip() == platform.machine()
    if (not force and same_machine and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC),
                                                   os.path.getmtime(os.path.join(_HERE, "pic_oracle.h")))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    with open(_STAMP, "w") as f:
        f.write(platform.machine())
    return _LIB_PATH


class OraGrid(C.Structure):
    _fields_ = [("ndim", C.c_int), ("nx", C.c_int * 3), ("dx", C.c_double * 3), ("xmin", C.c_double * 3),
                ("dt", C.c_double), ("e0", C.c_double * 3), ("b0", C.c_double * 3),
                ("smooth_level", C.c_int * 3), ("smooth_w", ((C.c_double * 3) * MAX_PASS) * 3),
                ("rho_bg", C.c_double), ("open_x1", C.c_int), ("isis", C.c_int),
                ("inc_b2", C.POINTER(C.c_double)), ("inc_b3", C.POINTER(C.c_double))]


class OraSpecies(C.Structure):
    _fields_ = [("rqm", C.c_double), ("q", C.c_double), ("n", C.c_longlong),
                ("x", C.POINTER(C.c_double)), ("u", C.POINTER(C.c_double)), ("w", C.POINTER(C.c_double))]


_DP = C.POINTER(C.c_double)
_DPP = _DP * 6


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB_PATH)
            gp = C.POINTER(OraGrid)
            sp = C.POINTER(OraSpecies)
            L.ora_gather.argtypes = [gp, C.POINTER(_DP), _DP, _DP]
            L.ora_boris.argtypes = [_DP, _DP, _DP, C.c_double, C.c_double]
            L.ora_gamma.argtypes = [_DP]
            L.ora_gamma.restype = C.c_double
            L.ora_move.argtypes = [gp, _DP, _DP]
            L.ora_wrap.argtypes = [gp, _DP]
            L.ora_deposit_vb.argtypes = [gp, C.POINTER(_DP), _DP, _DP, C.c_double, C.c_double]
            L.ora_deposit_isis.argtypes = [gp, C.POINTER(_DP), _DP, _DP, C.c_double, C.c_double]
            L.ora_deposit_rho.argtypes = [gp, _DP, _DP, C.c_longlong, C.c_double]
            L.ora_smooth.argtypes = [gp, _DP]
            L.ora_field_solve.argtypes = [gp, C.POINTER(_DP), C.POINTER(_DP)]
            L.ora_advance_particles.argtypes = [gp, C.POINTER(_DP), C.c_double, C.c_longlong, _DP, _DP, C.c_int]
            L.ora_particle_phase.argtypes = [gp, C.POINTER(_DP), C.POINTER(_DP), sp, C.c_int]
            L.ora_step.argtypes = [gp, C.POINTER(_DP), C.POINTER(_DP), sp, C.c_int, C.c_int]
            L.ora_rho.argtypes = [gp, sp, C.c_int, _DP]
            L.ora_gauss_residual.argtypes = [gp, C.POINTER(_DP), _DP]
            L.ora_gauss_residual.restype = C.c_double
            L.ora_field_energy.argtypes = [gp, C.POINTER(_DP)]
            L.ora_field_energy.restype = C.c_double
            L.ora_kinetic_energy.argtypes = [sp, C.c_int]
            L.ora_kinetic_energy.restype = C.c_double
            L.ora_init_e_gauss_x1.argtypes = [gp, _DP, _DP]
            L.ora_tile_bin.argtypes = [gp, C.POINTER(C.c_int), C.c_longlong, _DP, C.POINTER(C.c_longlong),
                                       C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_DP)


def make_grid(g) -> OraGrid:
    """ctypes grid from a ``workload.Grid``."""
    og = OraGrid()
    og.ndim = g.ndim
    for d in range(3):
        og.nx[d] = int(g.nx[d])
        og.dx[d] = float(g.dx[d])
        og.xmin[d] = float(g.xmin[d])
        og.e0[d] = float(g.e0[d])
        og.b0[d] = float(g.b0[d])
        og.smooth_level[d] = int(g.smooth_level[d])
        for p in range(MAX_PASS):
            w = g.smooth_w[d] if not isinstance(g.smooth_w[d][0], (tuple, list)) else g.smooth_w[d][min(p, len(g.smooth_w[d]) - 1)]
            for m in range(3):
                og.smooth_w[d][p][m] = float(w[m])
    og.dt = float(g.dt)
    og.rho_bg = float(g.rho_bg)
    og.open_x1 = int(bool(getattr(g, "move_window", False)))
    og.isis = int(getattr(g, "deposit", "vb") == "isis")
    return og


class State:
    """Oracle simulation state: six field arrays, three current arrays, species."""

    def __init__(self, grid, species_list, xs, us, charges, fields=None, weights=None, ids=None, created=None):
        self.grid = grid
        self.species = list(species_list)
        if getattr(grid, "deposit", "vb") == "isis" and grid.ndim != 2:
            raise ValueError("the ISIS deposit is defined for 2D3V only")
        self.og = make_grid(grid)
        self.nstep = 0
        self.shifts = 0
        # particle ids (initial generator index; injected particles continue it)
        self.ids = [np.arange(np.asarray(x).shape[0], dtype=np.int64) if ids is None or ids[s] is None
                    else np.asarray(ids[s], dtype=np.int64).copy() for s, x in enumerate(xs)]
        # particles ever created, counting the lattice places a profile skipped:
        # the id and draw index of the next injected particle
        self.created = [int(created[s]) if created is not None else
                        (np.asarray(xs[s]).shape[0] if ids is None or ids[s] is None
                         else (int(self.ids[s][-1]) + 1 if self.ids[s].size else 0)) for s in range(len(xs))]
        # per-particle charge weights (density profile); None: all 1
        self.w = [None if weights is None or weights[s] is None
                  else np.ascontiguousarray(weights[s], dtype=np.float64).copy() for s in range(len(xs))]
        shape = (int(grid.nx[2]), int(grid.nx[1]), int(grid.nx[0]))
        self.fld = [np.zeros(shape) if fields is None else np.ascontiguousarray(fields[c], dtype=np.float64).copy()
                    for c in range(6)]
        self.cur = [np.zeros(shape) for _ in range(3)]
        self.x = [np.ascontiguousarray(x, dtype=np.float64).copy() for x in xs]
        self.u = [np.ascontiguousarray(u, dtype=np.float64).copy() for u in us]
        self.rqm = [float(s.rqm) for s in species_list]
        self.q = [float(q) for q in charges]
        self._refresh()

    def _refresh(self):
        self._fp = _DPP(*[_dp(f) for f in self.fld])
        self._cp = (_DP * 3)(*[_dp(c) for c in self.cur])
        n = len(self.x)
        self._sp = (OraSpecies * n)()
        for i in range(n):
            self._sp[i].rqm = self.rqm[i]
            self._sp[i].q = self.q[i]
            self._sp[i].n = self.x[i].shape[0]
            self._sp[i].x = _dp(self.x[i])
            self._sp[i].u = _dp(self.u[i])
            self._sp[i].w = _dp(self.w[i]) if self.w[i] is not None else None

    @property
    def nsp(self):
        return len(self.x)

    def step(self, nsteps: int = 1):
        if getattr(self.grid, "move_window", False):
            for _ in range(int(nsteps)):
                self.window_step()
            return
        lib().ora_step(C.byref(self.og), self._fp, self._cp, self._sp, self.nsp, int(nsteps))
        self.nstep += int(nsteps)

    # -- moving window (thesis: dynamic simulation spaces) --------------------
    def window_step(self):
        """One step of a window moving at c in +x1.  The front boundary moves
        outward and the back boundary inward at c; the window is shifted by one
        cell when it lags c t by a cell (the step that reaches t = (n+1) dt):
        then every field value moves one cell back, the back column of cells and
        its plasma are discarded, and the new front column gets zero fields and
        fresh plasma.  x1 is open (no wrap); particles outside the window after
        the step are removed.  Order: particle phase, removal, smoothing and
        field solve, then the shift of the fields and the injection."""
        g = self.grid
        dx1 = float(g.dx[0])
        # the window moves at c from time window_start on
        lag = float(self.nstep + 1) * float(g.dt) - float(getattr(g, "window_start", 0.0))
        shift = lag > 0.0 and int(math.floor(lag / dx1)) > self.shifts
        self.particle_phase()
        lo = self.og.xmin[0] + (dx1 if shift else 0.0)
        hi = lo + int(g.nx[0]) * dx1
        for s in range(self.nsp):
            keep = (self.x[s][:, 0] >= lo) & (self.x[s][:, 0] < hi)
            if not keep.all():
                self.x[s] = np.ascontiguousarray(self.x[s][keep])
                self.u[s] = np.ascontiguousarray(self.u[s][keep])
                self.ids[s] = self.ids[s][keep]
                if self.w[s] is not None:
                    self.w[s] = np.ascontiguousarray(self.w[s][keep])
        self._refresh()
        self.smooth_current()
        self.field_solve()
        if shift:
            for f in self.fld:
                f[..., :-1] = f[..., 1:].copy()
                f[..., -1] = 0.0
            self.og.xmin[0] = lo
            self.shifts += 1
            import workload
            for s in range(self.nsp):
                gx = dataclasses.replace(g, xmin=(lo, g.xmin[1], g.xmin[2]))
                sp = self.species[s]
                xn, un = workload.inject_column(gx, sp, lo, self.created[s])
                idn = self.created[s] + np.arange(xn.shape[0])
                self.created[s] += xn.shape[0]
                wn = workload.profile_weight(sp, xn)  # the profile at the lab-frame positions
                if wn is not None:
                    keep = sp.density * wn > sp.den_min
                    xn, un, wn, idn = xn[keep], un[keep], wn[keep], idn[keep]
                    self.w[s] = np.ascontiguousarray(np.concatenate([self.w[s], wn]))
                self.x[s] = np.ascontiguousarray(np.concatenate([self.x[s], xn]))
                self.u[s] = np.ascontiguousarray(np.concatenate([self.u[s], un]))
                self.ids[s] = np.concatenate([self.ids[s], idn])
            self._refresh()
        self.nstep += 1

    def particle_phase(self):
        self._refresh()
        lib().ora_particle_phase(C.byref(self.og), self._fp, self._cp, self._sp, self.nsp)

    def smooth_current(self):
        for c in self.cur:
            lib().ora_smooth(C.byref(self.og), _dp(c))

    def add_antenna(self, laser):
        """A pulse entering through the lower x1 boundary (open x1 only)."""
        assert getattr(self.grid, "move_window", False), "an antenna needs the open x1 boundary"
        if not hasattr(self, "antennas"):
            self.antennas = []
            self.xmin1_initial = float(self.og.xmin[0])
        self.antennas.append(laser)

    def field_solve(self):
        ants = getattr(self, "antennas", [])
        if ants:  # B just below the lower x1 boundary at t = (n + 1/2) dt
            tt = (self.nstep + 0.5) * float(self.grid.dt)
            b2 = b3 = 0.0
            for las in ants:
                p2, p3 = antenna_planes(self.grid, las, tt, float(self.og.xmin[0]), self.xmin1_initial)
                b2, b3 = b2 + p2, b3 + p3
            self._inc = (np.ascontiguousarray(b2, dtype=np.float64), np.ascontiguousarray(b3, dtype=np.float64))
            self.og.inc_b2 = _dp(self._inc[0])
            self.og.inc_b3 = _dp(self._inc[1])
        lib().ora_field_solve(C.byref(self.og), self._fp, self._cp)
        self.og.inc_b2 = None
        self.og.inc_b3 = None

    def rho(self) -> np.ndarray:
        r = np.zeros_like(self.cur[0])
        lib().ora_rho(C.byref(self.og), self._sp, self.nsp, _dp(r))
        return r

    def gauss_residual(self, rho=None) -> float:
        r = self.rho() if rho is None else rho
        return lib().ora_gauss_residual(C.byref(self.og), self._fp, _dp(r))

    def field_energy(self) -> float:
        return lib().ora_field_energy(C.byref(self.og), self._fp)

    def kinetic_energy(self) -> float:
        return lib().ora_kinetic_energy(self._sp, self.nsp)

    def init_e_gauss_x1(self):
        lib().ora_init_e_gauss_x1(C.byref(self.og), _dp(self.rho()), _dp(self.fld[0]))


def from_workload(grid, species_list, fields=None, index=None):
    """Oracle state loaded from the seeded generator (all particles, or ``index``)."""
    import workload
    xs, us, qs, ws, ids, created = [], [], [], [], [], []
    for s in species_list:
        if s.profile is not None:
            assert index is None, "a density profile needs the whole lattice"
            x, u, w, idx = workload.load_weighted(grid, s)
        else:
            x, u = workload.load_particles(grid, s, index)
            w, idx = None, None
        xs.append(x)
        us.append(u)
        ws.append(w)
        ids.append(idx)
        created.append(workload.n_particles(grid, s) if index is None else x.shape[0])
        qs.append(workload.macro_charge(grid, s))
    st = State(grid, species_list, xs, us, qs, fields, weights=ws, ids=ids, created=created)
    if grid.init_e_gauss_x1:
        st.init_e_gauss_x1()
    return st


# --- single-operation helpers for the pins ---------------------------------

def gather(grid, fields, x) -> np.ndarray:
    og = make_grid(grid)
    fl = [np.ascontiguousarray(f, dtype=np.float64) for f in fields]
    fp = _DPP(*[_dp(f) for f in fl])
    xx = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros(6)
    lib().ora_gather(C.byref(og), fp, _dp(xx), _dp(out))
    return out


def boris(u, e, b, rqm, dt) -> np.ndarray:
    uu = np.array(u, dtype=np.float64)
    ee = np.array(e, dtype=np.float64)
    bb = np.array(b, dtype=np.float64)
    lib().ora_boris(_dp(uu), _dp(ee), _dp(bb), float(rqm), float(dt))
    return uu


def deposit_vb(grid, xold, xnew, v3, q):
    og = make_grid(grid)
    shape = (int(grid.nx[2]), int(grid.nx[1]), int(grid.nx[0]))
    cur = [np.zeros(shape) for _ in range(3)]
    cp = (_DP * 3)(*[_dp(c) for c in cur])
    lib().ora_deposit_vb(C.byref(og), cp, _dp(np.ascontiguousarray(xold, dtype=np.float64)),
                         _dp(np.ascontiguousarray(xnew, dtype=np.float64)), float(v3), float(q))
    return cur


def deposit_isis(grid, xold, xnew, v3, q):
    """ISIS deposit of one path (2D3V only)."""
    assert grid.ndim == 2, "the thesis defines the ISIS deposit for 2D"
    og = make_grid(grid)
    shape = (int(grid.nx[2]), int(grid.nx[1]), int(grid.nx[0]))
    cur = [np.zeros(shape) for _ in range(3)]
    cp = (_DP * 3)(*[_dp(c) for c in cur])
    lib().ora_deposit_isis(C.byref(og), cp, _dp(np.ascontiguousarray(xold, dtype=np.float64)),
                           _dp(np.ascontiguousarray(xnew, dtype=np.float64)), float(v3), float(q))
    return cur


def deposit_rho(grid, x, q, bg: float = 0.0):
    og = make_grid(grid)
    shape = (int(grid.nx[2]), int(grid.nx[1]), int(grid.nx[0]))
    r = np.full(shape, bg)
    xx = np.ascontiguousarray(np.atleast_2d(x), dtype=np.float64)
    lib().ora_deposit_rho(C.byref(og), _dp(r), _dp(xx), xx.shape[0], float(q))
    return r


def smooth(grid, f):
    og = make_grid(grid)
    ff = np.ascontiguousarray(f, dtype=np.float64).copy()
    lib().ora_smooth(C.byref(og), _dp(ff))
    return ff


def field_solve(grid, fields, currents):
    og = make_grid(grid)
    fl = [np.ascontiguousarray(f, dtype=np.float64).copy() for f in fields]
    cu = [np.ascontiguousarray(c, dtype=np.float64) for c in currents]
    lib().ora_field_solve(C.byref(og), _DPP(*[_dp(f) for f in fl]), (_DP * 3)(*[_dp(c) for c in cu]))
    return fl


def advance_particles(grid, fields, rqm, x, u, wrap=True):
    og = make_grid(grid)
    fl = [np.ascontiguousarray(f, dtype=np.float64) for f in fields]
    xx = np.ascontiguousarray(x, dtype=np.float64).copy()
    uu = np.ascontiguousarray(u, dtype=np.float64).copy()
    lib().ora_advance_particles(C.byref(og), _DPP(*[_dp(f) for f in fl]), float(rqm), xx.shape[0],
                                _dp(xx), _dp(uu), int(wrap))
    return xx, uu


def tile_bin(grid, tile, x):
    og = make_grid(grid)
    nt = [int(grid.nx[d]) // int(tile[d]) if d < grid.ndim else 1 for d in range(3)]
    ntiles = nt[0] * nt[1] * nt[2]
    xx = np.ascontiguousarray(x, dtype=np.float64)
    n = xx.shape[0]
    tid = np.zeros(n, dtype=np.int64)
    counts = np.zeros(ntiles, dtype=np.int64)
    order = np.zeros(n, dtype=np.int64)
    t = (C.c_int * 3)(*[int(v) for v in tile])
    LLP = C.POINTER(C.c_longlong)
    lib().ora_tile_bin(C.byref(og), t, n, _dp(xx), tid.ctypes.data_as(LLP), counts.ctypes.data_as(LLP),
                       order.ctypes.data_as(LLP))
    return tid, counts, order


# --- laser pulse initialisation ----------------------------------------------

def laser_envelope(xi, rise, length, fall):
    """Longitudinal envelope behind the pulse front (xi >= 0 behind it), the
    thesis' temporal profile: it rises as 10 s^3 - 15 s^4 + 6 s^5 with s =
    xi / rise (ch. on injection simulations; the appendix calls the rise and
    fall "approximately Gaussian"), stays 1 over `length` and falls as the
    mirror image over `fall`; 0 elsewhere (reading R21)."""
    xi = np.asarray(xi, dtype=np.float64)

    def poly(s):
        return 10.0 * s ** 3 - 15.0 * s ** 4 + 6.0 * s ** 5

    f = np.zeros_like(xi)
    a = (xi >= 0) & (xi < rise)
    f[a] = poly(xi[a] / rise)
    b = (xi >= rise) & (xi < rise + length)
    f[b] = 1.0
    c = (xi >= rise + length) & (xi < rise + length + fall)
    f[c] = poly(1.0 - (xi[c] - rise - length) / fall)
    return f


def _pulse_amp(laser, ndim, x, a, xfront, ct, c3, xfocus):
    """-vosc k f g T sin(psi) of a pulse moving in +x_a at positions x (three
    arrays), for the front at xfront, the transverse axis at (ct, c3) and the
    focal plane at xfocus (None: the waist profile everywhere); see
    laser_fields."""
    t = 1 - a
    k = laser.rkkp
    r2 = (x[t] - ct) ** 2
    if ndim == 3:
        r2 = r2 + (x[2] - c3) ** 2
    f = laser_envelope(xfront - x[a], laser.rise, laser.length, laser.fall)
    w2 = laser.w0 ** 2 * np.ones(np.shape(r2))
    g = np.ones(np.shape(r2))
    psi = k * (x[a] - xfront) + laser.phase
    if xfocus is not None:
        zr = 0.5 * k * laser.w0 ** 2
        z = x[a] - xfocus
        q = 1.0 + (z / zr) ** 2
        w2 = laser.w0 ** 2 * q
        g = q ** -0.5 if ndim == 3 else q ** -0.25
        with np.errstate(divide="ignore", invalid="ignore"):
            curv = np.where(z != 0.0, k * r2 / (2.0 * (z + zr * zr / z)), 0.0)
        gouy = np.arctan(z / zr)
        psi = psi + curv - (gouy if ndim == 3 else 0.5 * gouy)
    return -laser.vosc * k * f * g * np.exp(-r2 / w2) * np.sin(psi)


def laser_fields(grid, laser, xmin1=None):
    """E and B of a pulse at t = 0, each component at its own staggered
    position.  The pulse moves in +x_a (wavetype 1: a = x1, 2: a = x2); with
    the vector potential A = vosc f(xi) g T cos(psi) along p = cos(pol) e_t +
    sin(pol) e_3 (e_t the in-plane transverse axis), the slowly varying
    envelope approximation gives E = -dA/dt = -vosc k f g T sin(psi) p and
    B = e_a x E.  Without a focal plane g = 1, T = exp(-r^2 / w0^2) and
    psi = k (x_a - x_front) + phase.  With one (the thesis' Hermite-Gaussian
    beam, its laser-beam section): z = x_a - x_focus, z_R = k w0^2 / 2, w = w0
    sqrt(1 + (z/z_R)^2), T = exp(-r^2 / w^2), g = w0 / w in 3D and sqrt(w0 / w)
    for the 2D slab beam, psi += k r^2 / (2 R) - Gouy with R = z + z_R^2 / z and
    Gouy = atan(z / z_R) (half in 2D).  Returns the six arrays [nz][ny][nx]."""
    nx, ny = int(grid.nx[0]), int(grid.nx[1])
    nz = int(grid.nx[2]) if grid.ndim == 3 else 1
    dx = grid.dx
    a = 1 if int(getattr(laser, "wavetype", 1)) == 2 else 0
    t = 1 - a
    xmin = [float(grid.xmin[0] if xmin1 is None else xmin1), float(grid.xmin[1]), float(grid.xmin[2])]
    nn = [nx, ny, nz]
    upper = xmin[a] + nn[a] * dx[a]
    xfront = upper - laser.start
    ct = xmin[t] + 0.5 * nn[t] * dx[t] + laser.offset[0]
    c3 = (xmin[2] + 0.5 * nz * dx[2] + laser.offset[1]) if grid.ndim == 3 else 0.0
    focus = getattr(laser, "focus", None)
    xfocus = None if focus is None else upper - focus
    th = math.radians(laser.pol)
    k_, j_, i_ = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")

    def amp(s1, s2, s3):
        x = [xmin[0] + (i_ + s1) * dx[0], xmin[1] + (j_ + s2) * dx[1],
             xmin[2] + (k_ + s3) * dx[2] if grid.ndim == 3 else np.zeros(i_.shape)]
        return _pulse_amp(laser, grid.ndim, x, a, xfront, ct, c3, xfocus)

    zero = np.zeros((nz, ny, nx))
    s3 = 0.5 if grid.ndim == 3 else 0.0
    out = [zero.copy() for _ in range(6)]
    if a == 0:  # E2, E3; B3 = E2, B2 = -E3
        out[1] = amp(0.0, 0.5, 0.0) * math.cos(th)
        out[2] = amp(0.0, 0.0, s3) * math.sin(th)
        out[4] = -amp(0.5, 0.0, s3) * math.sin(th)
        out[5] = amp(0.5, 0.5, 0.0) * math.cos(th)
    else:  # E1, E3; B1 = E3, B3 = -E1
        out[0] = amp(0.5, 0.0, 0.0) * math.cos(th)
        out[2] = amp(0.0, 0.0, s3) * math.sin(th)
        out[3] = amp(0.0, 0.5, s3) * math.sin(th)
        out[5] = -amp(0.5, 0.5, 0.0) * math.cos(th)
    return out


def antenna_planes(grid, laser, time, xlo1, xmin1_initial):
    """B2 and B3 ([nz][ny]) just below the lower x1 boundary (x1 = xlo1 -
    dx1/2) at `time`, of a pulse that enters the box through that boundary
    moving in +x1 (the antenna form of the pulse input): its front crosses the
    boundary at time `start`, so x_front = xlo1 + (time - start); the focal
    plane (if any) lies `focus` into the box from the initial boundary
    xmin1_initial; otherwise as laser_fields (B3 = E2, B2 = -E3)."""
    ny = int(grid.nx[1])
    nz = int(grid.nx[2]) if grid.ndim == 3 else 1
    dx = grid.dx
    ct = grid.xmin[1] + 0.5 * ny * dx[1] + laser.offset[0]
    c3 = (grid.xmin[2] + 0.5 * nz * dx[2] + laser.offset[1]) if grid.ndim == 3 else 0.0
    focus = getattr(laser, "focus", None)
    xfocus = None if focus is None else xmin1_initial + focus
    xfront = xlo1 + (time - laser.start)
    th = math.radians(laser.pol)
    k_, j_ = np.meshgrid(np.arange(nz), np.arange(ny), indexing="ij")
    x1 = np.full(j_.shape, xlo1 - 0.5 * dx[0])
    s3 = 0.5 if grid.ndim == 3 else 0.0

    def amp(s2, s3_):
        x = [x1, grid.xmin[1] + (j_ + s2) * dx[1],
             grid.xmin[2] + (k_ + s3_) * dx[2] if grid.ndim == 3 else np.zeros(j_.shape)]
        return _pulse_amp(laser, grid.ndim, x, 0, xfront, ct, c3, xfocus)

    b2 = -amp(0.0, s3) * math.sin(th)
    b3 = amp(0.5, 0.0) * math.cos(th)
    return np.ascontiguousarray(b2), np.ascontiguousarray(b3)
