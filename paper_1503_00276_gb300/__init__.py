"""GB300 (sm_103a) hot path of the electromagnetic PIC method of Hemker's OSIRIS
thesis (arxiv 1503.00276): gather E,B -> relativistic Boris push -> position
update -> TRISTAN / Villasenor-Buneman charge-conserving current deposit, with
the Yee field solve, current smoothing and the per-tile particle sort as
supporting kernels.

Every step runs in the CUDA kernels of ``libpicgb.so`` behind the C ABI of
``include/pic.h``.  This module only marshals arguments; PyTorch (when
present) supplies device memory through its caching allocator and the CUDA
stream.  There is no CPU fallback: without the built library and a GPU every
call raises.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _capi
from ._capi import FIELD_NAMES, PIC_FP32_CELLOFF, PIC_FP64_PLAIN, PicError, check, load  # noqa: F401

__all__ = ["Simulation", "Batch", "autotune", "batch_autotune", "bin_tiles", "bin_tiles_noalloc", "load", "PicError", "PIC_FP64_PLAIN", "PIC_FP32_CELLOFF", "FIELD_NAMES"]


def _torch():
    try:
        import torch
        return torch
    except Exception:  # pragma: no cover
        return None


class _TorchAllocator:
    """pic_allocator backed by torch's caching allocator on the given stream."""

    def __init__(self, torch, device, stream):
        self.torch, self.device, self.stream = torch, device, stream
        self._alloc = _capi.ALLOC_FN(self._do_alloc)
        self._free = _capi.FREE_FN(self._do_free)
        self.struct = _capi.PicAllocator(None, self._alloc, self._free)

    def _do_alloc(self, ctx, nbytes):
        try:
            return int(self.torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream))
        except Exception:
            return None

    def _do_free(self, ctx, ptr, nbytes):
        self.torch.cuda.caching_allocator_delete(ptr)


def _grid_struct(grid, precision, tile=None, slack=0.0, sort_period=0, ctas_per_sm=0):
    g = _capi.PicGrid()
    g.ndim = int(grid.ndim)
    for d in range(3):
        g.nx[d] = int(grid.nx[d]) if d < grid.ndim else 1
        g.dx[d] = float(grid.dx[d]) if d < grid.ndim else 1.0
        g.xmin[d] = float(grid.xmin[d])
        g.e0[d] = float(grid.e0[d])
        g.b0[d] = float(grid.b0[d])
        g.smooth_level[d] = int(grid.smooth_level[d]) if d < grid.ndim else 0
        sw = grid.smooth_w[d]
        per_pass = isinstance(sw[0], (tuple, list))
        for p in range(_capi.MAX_SMOOTH):
            w = sw[min(p, len(sw) - 1)] if per_pass else sw
            for m in range(3):
                g.smooth_w[d][p][m] = float(w[m])
        g.bc[d][0] = g.bc[d][1] = 0
        g.tile[d] = int(tile[d]) if tile is not None and d < len(tile) else 0
    g.dt = float(grid.dt)
    g.rho_bg = float(grid.rho_bg)
    g.init_e_gauss_x1 = int(bool(getattr(grid, "init_e_gauss_x1", False)))
    g.precision = int(precision)
    g.slack = float(slack)
    g.sort_period = int(sort_period)
    g.ctas_per_sm = int(ctas_per_sm)
    g.move_window = int(bool(getattr(grid, "move_window", False)))
    dep = getattr(grid, "deposit", "vb")
    if dep not in ("vb", "isis"):
        raise ValueError(f"unknown deposit {dep!r} (vb or isis)")
    g.deposit = 1 if dep == "isis" else 0
    g.window_start = float(getattr(grid, "window_start", 0.0))
    g.coords = 1 if getattr(grid, "coords", "cartesian") == "cylindrical" else 0
    if g.coords:  # r-z: the axial boundary below, the conducting, absorbing wall above
        g.bc[1][0], g.bc[1][1] = _capi.PIC_BC_AXIAL, _capi.PIC_BC_CONDUCT_ABSORB
    return g


def _species_struct(sp, explicit=None, track_ids=False, np_max=0):
    s = _capi.PicSpecies()
    s.rqm = float(sp.rqm)
    for d in range(3):
        s.ppc[d] = int(sp.ppc[d])
        s.uth[d] = float(sp.uth[d])
        s.ufl[d] = float(sp.ufl[d])
    s.density = float(getattr(sp, "density", 1.0))
    s.seed = int(getattr(sp, "seed", 0)) & 0xFFFFFFFFFFFFFFFF
    s.track_ids = int(bool(track_ids))
    s.np_max = int(np_max)
    keep = []
    prof = getattr(sp, "profile", None)
    if explicit is None and prof is not None:
        for d, pd in enumerate(prof):
            if pd is None:
                continue
            xs, fs = (np.ascontiguousarray(v, dtype=np.float64) for v in pd)
            assert xs.shape == fs.shape and xs.ndim == 1 and xs.size > 0
            s.prof_n[d] = xs.size
            s.prof_x[d] = xs.ctypes.data_as(C.POINTER(C.c_double))
            s.prof_f[d] = fs.ctypes.data_as(C.POINTER(C.c_double))
            keep += [xs, fs]
        s.den_min = float(getattr(sp, "den_min", 0.0))
    if explicit is not None:
        x, u, q = explicit[:3]
        x = np.ascontiguousarray(x, dtype=np.float64)
        u = np.ascontiguousarray(u, dtype=np.float64)
        assert x.shape == u.shape and x.ndim == 2 and x.shape[1] == 3
        s.n_explicit = x.shape[0]
        s.x0 = x.ctypes.data_as(C.POINTER(C.c_double))
        s.u0 = u.ctypes.data_as(C.POINTER(C.c_double))
        s.q_explicit = float(q)
        keep += [x, u]
        if len(explicit) > 3 and explicit[3] is not None:  # per-particle charge weights
            w = np.ascontiguousarray(explicit[3], dtype=np.float64)
            assert w.shape == (x.shape[0],)
            s.w0 = w.ctypes.data_as(C.POINTER(C.c_double))
            keep.append(w)
    return s, keep


class Simulation:
    """One simulation handle (pic_init ... pic_destroy).

    grid / species: objects with the attributes of ``pic_grid`` / ``pic_species``
    (ndim, nx, dx, xmin, dt, e0, b0, smooth_level, smooth_w, rho_bg,
    init_e_gauss_x1 / rqm, ppc, uth, ufl, density, seed).  ``explicit``: optional
    list, per species, of (x[n,3], u[n,3], q[, w[n]]) host arrays that replace the
    lattice loader (w: per-particle charge weights).  A species' ``profile`` /
    ``den_min`` (see ``workload.Species``) give its density profile.  ``precision``: "fp64" (plain form) or "fp32" (cell-offset tiled form).
    """

    def __init__(self, grid, species, precision="fp64", explicit=None, tile=None, track_ids=False, slack=0.0,
                 stream=None, use_torch_allocator=True, np_max=0, sort_period=0, ctas_per_sm=0):
        self._lib = load()
        torch = _torch()
        prec = PIC_FP32_CELLOFF if precision in ("fp32", PIC_FP32_CELLOFF) else PIC_FP64_PLAIN
        self.precision = prec
        self.ndim = int(grid.ndim)
        self.shape = (int(grid.nx[2]) if grid.ndim == 3 else 1, int(grid.nx[1]), int(grid.nx[0]))
        self._g = _grid_struct(grid, prec, tile, slack, sort_period, ctas_per_sm)
        specs = (_capi.PicSpecies * max(len(species), 1))()
        self._keep = []
        for k, sp in enumerate(species):
            ex = explicit[k] if explicit is not None else None
            s, keep = _species_struct(sp, ex, track_ids, np_max)
            specs[k] = s
            self._keep.append(keep)
        self.nspecies = len(species)
        self._torch = torch
        self._alloc = None
        stream_ptr = None
        if torch is not None and torch.cuda.is_available():
            st = stream if stream is not None else torch.cuda.current_stream()
            self.stream = st
            stream_ptr = C.c_void_p(st.cuda_stream)
            if use_torch_allocator:
                self._alloc = _TorchAllocator(torch, torch.cuda.current_device(), st)
        else:
            self.stream = None
        h = C.c_void_p()
        code = self._lib.pic_init(C.byref(self._g), specs, len(species),
                                  C.byref(self._alloc.struct) if self._alloc else None, stream_ptr, C.byref(h))
        self._keep = None
        check(code, "pic_init")
        self._h = h

    # -- laser ----------------------------------------------------------------
    def add_laser(self, laser):
        """pic_laser_add: a pulse moving in +x1 or +x2 (attributes of workload.Laser)."""
        L = _capi.PicLaser()
        for f in ("vosc", "rkkp", "w0", "rise", "fall", "length", "start", "pol", "phase"):
            setattr(L, f, float(getattr(laser, f)))
        off = tuple(getattr(laser, "offset", (0.0, 0.0)))
        L.offset[0], L.offset[1] = float(off[0]), float(off[1] if len(off) > 1 else 0.0)
        L.wavetype = int(getattr(laser, "wavetype", 1))
        focus = getattr(laser, "focus", None)
        L.focus_on = int(focus is not None)
        L.focus = float(focus) if focus is not None else 0.0
        L.antenna = int(bool(getattr(laser, "antenna", False)))
        check(self._lib.pic_laser_add(self._h, C.byref(L)), "pic_laser_add")

    # -- checkpoint / restart ---------------------------------------------------
    def save(self, path: str):
        """pic_checkpoint_save: the full state (particles, E/B, step) to a file."""
        check(self._lib.pic_checkpoint_save(self._h, str(path).encode()), "pic_checkpoint_save")

    @classmethod
    def load(cls, path: str, stream=None, use_torch_allocator=True) -> "Simulation":
        """pic_checkpoint_load: a new simulation from a checkpoint file."""
        self = cls.__new__(cls)
        self._lib = load()
        torch = _torch()
        self._torch = torch
        self._alloc = None
        stream_ptr = None
        self.stream = None
        if torch is not None and torch.cuda.is_available():
            st = stream if stream is not None else torch.cuda.current_stream()
            self.stream = st
            stream_ptr = C.c_void_p(st.cuda_stream)
            if use_torch_allocator:
                self._alloc = _TorchAllocator(torch, torch.cuda.current_device(), st)
        h = C.c_void_p()
        check(self._lib.pic_checkpoint_load(str(path).encode(), C.byref(self._alloc.struct) if self._alloc else None,
                                            stream_ptr, C.byref(h)), "pic_checkpoint_load")
        self._h = h
        g = _capi.PicGrid()
        nsp = C.c_int()
        check(self._lib.pic_info(h, C.byref(g), C.byref(nsp), None), "pic_info")
        self._g = g
        self.precision = int(g.precision)
        self.ndim = int(g.ndim)
        self.shape = (int(g.nx[2]) if g.ndim == 3 else 1, int(g.nx[1]), int(g.nx[0]))
        self.nspecies = int(nsp.value)
        self._keep = None
        return self

    def info(self) -> dict:
        g = _capi.PicGrid()
        nsp = C.c_int()
        step = C.c_longlong()
        check(self._lib.pic_info(self._h, C.byref(g), C.byref(nsp), C.byref(step)), "pic_info")
        return {"tile": tuple(g.tile), "sort_period": int(g.sort_period), "ctas_per_sm": int(g.ctas_per_sm),
                "nspecies": int(nsp.value), "step": int(step.value), "precision": int(g.precision),
                "coords": int(g.coords)}

    # -- lifecycle ----------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            self._lib.pic_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- stepping -------------------------------------------------------------
    def step(self, n: int = 1):
        check(self._lib.pic_step(self._h, int(n)), "pic_step")

    # -- grid data ------------------------------------------------------------
    def _which(self, which):
        return FIELD_NAMES[which] if isinstance(which, str) else int(which)

    def fields(self, which) -> np.ndarray:
        out = np.empty(self.shape, dtype=np.float64)
        check(self._lib.pic_fields(self._h, self._which(which), out.ctypes.data_as(C.c_void_p), out.nbytes, 0),
              "pic_fields")
        return out

    def fields_device(self, which):
        torch = self._torch
        out = torch.empty(self.shape, dtype=torch.float64, device="cuda")
        check(self._lib.pic_fields(self._h, self._which(which), C.c_void_p(out.data_ptr()), out.numel() * 8, 1),
              "pic_fields")
        return out

    def set_field(self, which, arr):
        a = np.ascontiguousarray(np.asarray(arr, dtype=np.float64).reshape(self.shape))
        check(self._lib.pic_set_field(self._h, self._which(which), a.ctypes.data_as(C.c_void_p), a.nbytes, 0),
              "pic_set_field")

    # -- particles --------------------------------------------------------------
    def n_particles(self, species: int = 0) -> int:
        n = C.c_longlong()
        self._lib.pic_particles(self._h, species, None, None, 0, C.byref(n), 0)
        return int(n.value)

    def particles(self, species: int = 0):
        n = self.n_particles(species)
        x = np.empty((n, 3), dtype=np.float64)
        u = np.empty((n, 3), dtype=np.float64)
        got = C.c_longlong()
        check(self._lib.pic_particles(self._h, species, x.ctypes.data_as(C.c_void_p), u.ctypes.data_as(C.c_void_p),
                                      n, C.byref(got), 0), "pic_particles")
        return x, u

    def particles_into(self, x, u, species: int = 0) -> int:
        """Copy into caller buffers (numpy host arrays or torch CUDA tensors)."""
        on_dev = int(hasattr(x, "data_ptr"))
        px = C.c_void_p(x.data_ptr() if on_dev else x.ctypes.data)
        pu = C.c_void_p(u.data_ptr() if on_dev else u.ctypes.data)
        got = C.c_longlong()
        check(self._lib.pic_particles(self._h, species, px, pu, int(x.shape[0]), C.byref(got), on_dev),
              "pic_particles")
        return int(got.value)

    def ids(self, species: int = 0) -> np.ndarray:
        n = self.n_particles(species)
        out = np.empty(n, dtype=np.int32)
        got = C.c_longlong()
        check(self._lib.pic_particle_ids(self._h, species, out.ctypes.data_as(C.c_void_p), n, C.byref(got), 0),
              "pic_particle_ids")
        return out

    def weights(self, species: int = 0) -> np.ndarray:
        """pic_particle_weights: charge weight of each particle (1 without a profile)."""
        n = self.n_particles(species)
        out = np.empty(n, dtype=np.float64)
        got = C.c_longlong()
        check(self._lib.pic_particle_weights(self._h, species, out.ctypes.data_as(C.c_void_p), n, C.byref(got), 0),
              "pic_particle_weights")
        return out

    def tile_counts(self, species: int = 0) -> np.ndarray:
        nt = C.c_longlong()
        self._lib.pic_tile_counts(self._h, species, None, 0, C.byref(nt))
        out = np.empty(int(nt.value), dtype=np.int64)
        check(self._lib.pic_tile_counts(self._h, species, out.ctypes.data_as(C.POINTER(C.c_longlong)), out.size,
                                        C.byref(nt)), "pic_tile_counts")
        return out

    # -- diagnostics ------------------------------------------------------------
    def diag(self) -> dict:
        d = _capi.PicDiag()
        check(self._lib.pic_diag(self._h, C.byref(d)), "pic_diag")
        return {k: getattr(d, k) for k, _ in _capi.PicDiag._fields_}

    def timing_enable(self, on: bool = True):
        check(self._lib.pic_timing_enable(self._h, int(on)), "pic_timing_enable")

    def timing_read(self, reset: bool = False):
        ms = (C.c_double * 6)()
        n = (C.c_longlong * 6)()
        check(self._lib.pic_timing_read(self._h, ms, n, 6, int(reset)), "pic_timing_read")
        names = ["particles", "current", "fields", "rebuild", "step", "launches"]
        return {names[k]: (ms[k], n[k]) for k in range(6)}


def bin_tiles(nx, tile, cell, stream=None):
    """Tile binning of device int32 cells[n,3] (torch CUDA tensor) through pic_bin_tiles.
    Returns (tile_count int32, tile_start int64, perm int64) as torch tensors."""
    torch = _torch()
    lib = load()
    assert cell.is_cuda and cell.dtype == torch.int32 and cell.is_contiguous()
    n = cell.shape[0]
    nt = 1
    for d in range(3):
        nt *= int(nx[d]) // int(tile[d])
    counts = torch.empty(nt, dtype=torch.int32, device=cell.device)
    start = torch.empty(nt, dtype=torch.int64, device=cell.device)
    perm = torch.empty(max(n, 1), dtype=torch.int64, device=cell.device)
    st = stream if stream is not None else torch.cuda.current_stream()
    alloc = _TorchAllocator(torch, cell.device.index, st)
    nxa = (C.c_int * 3)(*[int(v) for v in nx])
    ta = (C.c_int * 3)(*[int(v) for v in tile])
    check(lib.pic_bin_tiles(nxa, ta, n, C.c_void_p(cell.data_ptr()), C.c_void_p(counts.data_ptr()),
                            C.c_void_p(start.data_ptr()), C.c_void_p(perm.data_ptr()), C.byref(alloc.struct),
                            C.c_void_p(st.cuda_stream)), "pic_bin_tiles")
    return counts, start, perm[:n]


def bin_tiles_noalloc(nx, tile, cell, stream=None):
    """pic_bin_tiles_noalloc: same result as bin_tiles, scratch from the fixed
    device array compiled into the library (no allocation inside the call).
    Output tensors are allocated here by torch, outside the C call."""
    torch = _torch()
    lib = load()
    assert cell.is_cuda and cell.dtype == torch.int32 and cell.is_contiguous()
    n = cell.shape[0]
    nt = 1
    for d in range(3):
        nt *= int(nx[d]) // int(tile[d])
    counts = torch.empty(nt, dtype=torch.int32, device=cell.device)
    start = torch.empty(nt, dtype=torch.int64, device=cell.device)
    perm = torch.empty(max(n, 1), dtype=torch.int64, device=cell.device)
    st = stream if stream is not None else torch.cuda.current_stream()
    nxa = (C.c_int * 3)(*[int(v) for v in nx])
    ta = (C.c_int * 3)(*[int(v) for v in tile])
    check(lib.pic_bin_tiles_noalloc(nxa, ta, n, C.c_void_p(cell.data_ptr()), C.c_void_p(counts.data_ptr()),
                                    C.c_void_p(start.data_ptr()), C.c_void_p(perm.data_ptr()),
                                    C.c_void_p(st.cuda_stream)), "pic_bin_tiles_noalloc")
    return counts, start, perm[:n]


class _Member(Simulation):
    """Borrowed handle of one member of a Batch: read-out and set_field only."""

    def __init__(self, batch, handle, grid, nspecies):
        self._lib = batch._lib
        self._torch = batch._torch
        self._batch = batch  # keeps the batch alive
        self._h = handle
        self.precision = PIC_FP32_CELLOFF
        self.ndim = int(grid.ndim)
        self.shape = (int(grid.nx[2]) if grid.ndim == 3 else 1, int(grid.nx[1]), int(grid.nx[0]))
        self.nspecies = nspecies
        self.stream = batch.stream
        self._alloc = None

    def close(self):
        self._h = None  # owned by the batch

    def step(self, n: int = 1):
        raise RuntimeError("a batch member is stepped by Batch.step")


class Batch:
    """Many independent FP32 cell-offset simulations advanced together
    (pic_batch_init ... pic_batch_destroy): one persistent tile-kernel launch
    for the particles of all members, one launch per field stage for all
    members, and one CUDA graph launch per step.

    ``members``: list of (grid, [species, ...]) with the same number of
    species each, or of (grid, [species, ...], laser) where laser is None, one
    pulse or a list of pulses given to that member's pic_laser_add after
    pic_batch_init.  ``tile``: common tile shape (None: the library's choice).
    """

    def __init__(self, members, tile=None, track_ids=False, slack=0.0, stream=None, use_torch_allocator=True,
                 ctas_per_sm=0):
        self._lib = load()
        torch = _torch()
        self._torch = torch
        n = len(members)
        nsp = len(members[0][1])
        assert n >= 1 and nsp >= 1 and all(len(m[1]) == nsp for m in members)
        grids = (_capi.PicGrid * n)()
        specs = (_capi.PicSpecies * (n * nsp))()
        for i, m in enumerate(members):
            g, sps = m[0], m[1]
            grids[i] = _grid_struct(g, PIC_FP32_CELLOFF, tile, slack, 1, ctas_per_sm)
            for k, sp in enumerate(sps):
                specs[i * nsp + k] = _species_struct(sp, None, track_ids)[0]
        self._members = members
        self.nspecies = nsp
        self._alloc = None
        stream_ptr = None
        if torch is not None and torch.cuda.is_available():
            st = stream if stream is not None else torch.cuda.current_stream()
            self.stream = st
            stream_ptr = C.c_void_p(st.cuda_stream)
            if use_torch_allocator:
                self._alloc = _TorchAllocator(torch, torch.cuda.current_device(), st)
        else:
            self.stream = None
        h = C.c_void_p()
        code = self._lib.pic_batch_init(n, grids, specs, nsp, C.byref(self._alloc.struct) if self._alloc else None,
                                        stream_ptr, C.byref(h))
        check(code, "pic_batch_init")
        self._h = h
        for i, m in enumerate(members):
            lasers = m[2] if len(m) > 2 else None
            if lasers is None:
                continue
            for las in (lasers if isinstance(lasers, (list, tuple)) else [lasers]):
                self.sim(i).add_laser(las)

    def __len__(self):
        return len(self._members)

    def step(self, n: int = 1):
        check(self._lib.pic_batch_step(self._h, int(n)), "pic_batch_step")

    def sim(self, i: int) -> Simulation:
        h = C.c_void_p()
        check(self._lib.pic_batch_sim(self._h, int(i), C.byref(h)), "pic_batch_sim")
        return _Member(self, h, self._members[i][0], self.nspecies)

    def info(self) -> dict:
        steps, launches = C.c_longlong(), C.c_longlong()
        tile = (C.c_int * 3)()
        check(self._lib.pic_batch_info(self._h, C.byref(steps), C.byref(launches), tile), "pic_batch_info")
        return {"steps": int(steps.value), "launches": int(launches.value), "tile": tuple(tile)}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.pic_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def _tune_result(best, tried, n):
    def one(c):
        return {"tile": tuple(c.tile), "ctas_per_sm": int(c.ctas_per_sm), "sort_period": int(c.sort_period),
                "ms_per_step": float(c.ms_per_step)}
    return one(best), [one(tried[k]) for k in range(min(n, len(tried)))]


def _stream_and_alloc(stream, use_torch_allocator):
    torch = _torch()
    if torch is None or not torch.cuda.is_available():
        return None, None
    st = stream if stream is not None else torch.cuda.current_stream()
    alloc = _TorchAllocator(torch, torch.cuda.current_device(), st) if use_torch_allocator else None
    return C.c_void_p(st.cuda_stream), alloc


def autotune(grid, species, warmup=3, steps=5, slack=0.0, stream=None, use_torch_allocator=True):
    """pic_autotune: time every (tile shape, blocks per SM, sort period)
    candidate of the FP32 form on this workload; returns (best, all tried)."""
    lib = load()
    g = _grid_struct(grid, PIC_FP32_CELLOFF, None, slack)
    specs = (_capi.PicSpecies * len(species))(*[_species_struct(sp)[0] for sp in species])
    st, alloc = _stream_and_alloc(stream, use_torch_allocator)
    best = _capi.PicTuneChoice()
    tried = (_capi.PicTuneChoice * 32)()
    n = C.c_int()
    check(lib.pic_autotune(C.byref(g), specs, len(species), C.byref(alloc.struct) if alloc else None, st,
                           int(warmup), int(steps), C.byref(best), tried, 32, C.byref(n)), "pic_autotune")
    return _tune_result(best, tried, n.value)


def batch_autotune(members, warmup=2, steps=3, slack=0.0, stream=None, use_torch_allocator=True):
    """pic_batch_autotune for the members of a Batch; returns (best, all tried)."""
    lib = load()
    n = len(members)
    nsp = len(members[0][1])
    grids = (_capi.PicGrid * n)()
    specs = (_capi.PicSpecies * (n * nsp))()
    for i, m in enumerate(members):  # (grid, species[, lasers]): the candidates run without the pulses
        g, sps = m[0], m[1]
        grids[i] = _grid_struct(g, PIC_FP32_CELLOFF, None, slack, 1)
        for k, sp in enumerate(sps):
            specs[i * nsp + k] = _species_struct(sp)[0]
    st, alloc = _stream_and_alloc(stream, use_torch_allocator)
    best = _capi.PicTuneChoice()
    tried = (_capi.PicTuneChoice * 32)()
    cnt = C.c_int()
    check(lib.pic_batch_autotune(n, grids, specs, nsp, C.byref(alloc.struct) if alloc else None, st, int(warmup),
                                 int(steps), C.byref(best), tried, 32, C.byref(cnt)), "pic_batch_autotune")
    return _tune_result(best, tried, cnt.value)
