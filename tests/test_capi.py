"""C ABI checks that need no GPU: the library builds and loads, exports every
function include/pic.h declares, and validates arguments on the host
(Courant condition, dimensions, boundary types) before touching a device."""
import ctypes as C
import os
import re

import pytest

import workload

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def capi():
    from paper_1503_00276_gb300 import _capi, build
    build.build()
    _capi.load()
    return _capi


def _declared():
    src = open(os.path.join(ROOT, "include", "pic.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pic_[a-z_0-9]+)\s*\(", src)))


def test_header_declarations_are_exported(capi):
    names = _declared()
    assert "pic_init" in names and "pic_step" in names and len(names) >= 13
    lib = C.CDLL(capi.library_path())
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(capi.PROTOTYPES) == names


def test_struct_layouts_match_header(capi, tmp_path):
    """sizeof/offsetof of the ABI structs as the C compiler sees include/pic.h."""
    import subprocess
    prog = tmp_path / "layout.c"
    fields = {"pic_grid": capi.PicGrid, "pic_species": capi.PicSpecies, "pic_diag_t": capi.PicDiag,
              "pic_allocator": capi.PicAllocator, "pic_tune_choice": capi.PicTuneChoice, "pic_laser": capi.PicLaser}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pic.h"', "int main(void) {"]
    for cname, cls in fields.items():
        lines.append(f'  printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("  return 0; }")
    prog.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True, check=True)
               .stdout.splitlines())
    for cname, cls in fields.items():
        assert int(out[cname]) == C.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert int(out[f"{cname}.{f}"]) == getattr(cls, f).offset, (cname, f)


def _grid(dt_frac=0.99, ndim=2, bc=0):
    dx = (0.1, 0.1, 0.1)
    g = workload.Grid(ndim=ndim, nx=(16, 16, 16), dx=dx, dt=workload.courant_dt(dx, ndim, dt_frac))
    from paper_1503_00276_gb300 import _grid_struct
    s = _grid_struct(g, 0)
    s.bc[0][0] = bc
    return s


def _init(capi, g):
    h = C.c_void_p()
    sp = capi.PicSpecies()
    sp.rqm = -1.0
    sp.ppc[0] = sp.ppc[1] = sp.ppc[2] = 1
    sp.density = 1.0
    code = capi.load().pic_init(C.byref(g), C.byref(sp), 1, None, None, C.byref(h))
    return code, h


def test_courant_violation_is_rejected(capi):
    code, h = _init(capi, _grid(dt_frac=1.0001))
    assert code == -4 and not h.value
    assert b"Courant" in capi.load().pic_last_error()


def test_bad_arguments_are_rejected(capi):
    g = _grid()
    g.ndim = 4
    assert _init(capi, g)[0] == -1
    assert _init(capi, _grid(bc=5))[0] == -8
    lib = capi.load()
    assert lib.pic_destroy(None) == 0
    h = C.c_void_p()
    assert lib.pic_init(None, None, 0, None, None, C.byref(h)) == -1
    nx = (C.c_int * 3)(16, 16, 1)
    bad_tile = (C.c_int * 3)(5, 4, 1)
    assert lib.pic_bin_tiles(nx, bad_tile, 0, None, C.c_void_p(8), C.c_void_p(8), None, None, None) == -1


def test_deposit_choice_is_checked(capi):
    g = _grid(ndim=3)
    g.deposit = 1  # ISIS: defined for 2D3V only
    assert _init(capi, g)[0] == -8
    assert b"ISIS" in capi.load().pic_last_error()
    g = _grid()
    g.deposit = 7
    assert _init(capi, g)[0] == -1


def test_valid_grid_without_device_reports_cuda_error(capi):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    code, h = _init(capi, _grid())
    assert code == -3 and not h.value


def test_batch_arguments_are_checked_before_any_device_work(capi):
    from paper_1503_00276_gb300 import _grid_struct, _species_struct
    lib = capi.load()
    h = C.c_void_p()
    assert lib.pic_batch_init(0, None, None, 1, None, None, C.byref(h)) == -1
    dx = (0.1, 0.1, 0.1)
    g2 = workload.Grid(ndim=2, nx=(64, 32, 1), dx=dx, dt=workload.courant_dt(dx, 2))
    g3 = workload.Grid(ndim=3, nx=(16, 16, 16), dx=dx, dt=workload.courant_dt(dx, 3))
    sp = workload.Species(ppc=(1, 1, 1))
    grids = (capi.PicGrid * 2)(_grid_struct(g2, 1), _grid_struct(g3, 1))
    specs = (capi.PicSpecies * 2)(_species_struct(sp)[0], _species_struct(sp)[0])
    assert lib.pic_batch_init(2, grids, specs, 1, None, None, C.byref(h)) == -1  # mixed ndim
    grids = (capi.PicGrid * 2)(_grid_struct(g2, 1), _grid_struct(g2, 0))
    assert lib.pic_batch_init(2, grids, specs, 1, None, None, C.byref(h)) == -1  # FP64 member
    assert b"FP32" in lib.pic_last_error()
    # an r-z member is refused (the batched step has no cylindrical kernels);
    # moving-window members are accepted and run on the device
    grz = _grid_struct(g2, 1)
    grz.coords = capi.PIC_COORDS_CYLINDRICAL
    grids = (capi.PicGrid * 2)(_grid_struct(g2, 1), grz)
    assert lib.pic_batch_init(2, grids, specs, 1, None, None, C.byref(h)) == -8  # PIC_EUNSUPPORTED
    assert b"simulation 1" in lib.pic_last_error() and b"r-z" in lib.pic_last_error()
    assert not h.value
    assert lib.pic_batch_destroy(None) == 0


def test_autotune_arguments_are_checked_before_any_device_work(capi):
    from paper_1503_00276_gb300 import _grid_struct, _species_struct
    lib = capi.load()
    best = capi.PicTuneChoice()
    dx = (0.1, 0.1, 0.1)
    g = workload.Grid(ndim=2, nx=(20, 12, 1), dx=dx, dt=workload.courant_dt(dx, 2))  # no tile shape divides it
    gs = _grid_struct(g, 1)
    sp = _species_struct(workload.Species(ppc=(1, 1, 1)))[0]
    n = C.c_int()
    assert lib.pic_autotune(C.byref(gs), C.byref(sp), 1, None, None, 1, 2, C.byref(best), None, 0, C.byref(n)) == -1
    assert b"divides" in lib.pic_last_error()
    assert lib.pic_autotune(C.byref(gs), C.byref(sp), 1, None, None, 1, 0, C.byref(best), None, 0, None) == -1
    g64 = _grid_struct(workload.Grid(ndim=2, nx=(64, 32, 1), dx=dx, dt=workload.courant_dt(dx, 2)), 0)
    assert lib.pic_autotune(C.byref(g64), C.byref(sp), 1, None, None, 1, 2, C.byref(best), None, 0, None) == -1


def test_checkpoint_load_rejects_missing_and_foreign_files(capi, tmp_path):
    lib = capi.load()
    h = C.c_void_p()
    assert lib.pic_checkpoint_load(str(tmp_path / "none.ckpt").encode(), None, None, C.byref(h)) == -1
    bad = tmp_path / "bad.ckpt"
    bad.write_bytes(b"NOTACKPT" + bytes(200))
    assert lib.pic_checkpoint_load(str(bad).encode(), None, None, C.byref(h)) == -1
    assert b"not a checkpoint" in lib.pic_last_error()
    trunc = tmp_path / "trunc.ckpt"
    trunc.write_bytes(b"PICGBCK1" + bytes(6))
    assert lib.pic_checkpoint_load(str(trunc).encode(), None, None, C.byref(h)) == -1
    assert not h.value
    assert lib.pic_checkpoint_save(None, b"x") == -1


def _cyl_grid(frac=0.99):
    g = workload.cyl_grid(16, 8, 0.1, 0.1, frac=frac)
    from paper_1503_00276_gb300 import _grid_struct
    return _grid_struct(g, 0)


def test_r_z_arguments_are_checked_before_any_device_work(capi):
    """The r-z mode's grid rules (axial and conducting-absorbing r boundaries,
    the axis through the first cell, its own time-step bound, the options it
    does not combine with) are checked before any device work."""
    import torch
    lib = capi.load()
    g = _cyl_grid()
    assert g.bc[1][0] == capi.PIC_BC_AXIAL and g.bc[1][1] == capi.PIC_BC_CONDUCT_ABSORB
    g.bc[1][0] = capi.PIC_BC_PERIODIC
    assert _init(capi, g)[0] == -1 and b"PIC_BC_AXIAL" in lib.pic_last_error()
    g = _cyl_grid()
    g.xmin[1] = 0.0
    assert _init(capi, g)[0] == -1 and b"axis" in lib.pic_last_error()
    # inside the Cartesian bound, outside the r-z one
    g = _cyl_grid(frac=1.001)
    assert _init(capi, g)[0] == -4 and b"r-z" in lib.pic_last_error()
    g = _cyl_grid()
    g.smooth_level[0] = 1
    assert _init(capi, g)[0] == -8
    g = _cyl_grid()
    g.coords = 2
    g.bc[1][0] = g.bc[1][1] = capi.PIC_BC_PERIODIC
    assert _init(capi, g)[0] == -1 and b"coords" in lib.pic_last_error()
    if not torch.cuda.is_available():
        assert _init(capi, _cyl_grid())[0] == -3


def test_enum_values_match_header(capi, tmp_path):
    """The binding's constants equal the header's enums as the C compiler sees them."""
    import subprocess
    names = ["PIC_OK", "PIC_FP64_PLAIN", "PIC_FP32_CELLOFF", "PIC_BC_PERIODIC", "PIC_BC_CONDUCT_ABSORB",
             "PIC_BC_AXIAL", "PIC_COORDS_CARTESIAN", "PIC_COORDS_CYLINDRICAL", "PIC_E1", "PIC_B3", "PIC_J1",
             "PIC_RHO"]
    prog = tmp_path / "enums.c"
    lines = ['#include <stdio.h>', '#include "pic.h"', "int main(void) {"]
    lines += [f'  printf("{n} %d\\n", (int){n});' for n in names]
    lines.append("  return 0; }")
    prog.write_text("\n".join(lines))
    exe = tmp_path / "enums"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True, check=True)
               .stdout.splitlines())
    for n in names:
        assert int(out[n]) == getattr(capi, n), n
