"""The seeded input generator: SplitMix64 against its published test vectors,
Box-Muller moments, the num_par_x lattice loader and macroparticle charge."""
import math
import os

import numpy as np

import workload

HERE = os.path.dirname(os.path.abspath(__file__))


def test_splitmix64_published_vectors():
    for line in open(os.path.join(HERE, "golden", "splitmix64_vectors.txt")):
        if line.startswith("#") or not line.strip():
            continue
        seed, *vals = line.split()
        got = workload.splitmix64(int(seed), np.arange(len(vals)))
        assert [int(v) for v in got] == [int(v, 16) for v in vals]


def test_uniform_and_normal_moments():
    u = workload.uniform01(7, np.arange(200000))
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 3e-3
    n = workload.normal(7, np.arange(200000))
    assert abs(n.mean()) < 1e-2 and abs(n.std() - 1) < 1e-2
    assert abs(np.mean(n ** 4) - 3) < 0.05


def test_lattice_loader_positions_and_charge():
    g = workload.Grid(ndim=3, nx=(4, 3, 2), dx=(0.1, 0.2, 0.3), dt=0.01)
    sp = workload.Species(ppc=(2, 1, 2), uth=(0.1, 0.0, 0.2), ufl=(0.0, 0.5, 0.0), seed=5)
    x, u = workload.load_particles(g, sp)
    assert x.shape == (4 * 3 * 2 * 4, 3)
    # particle 0: cell (0,0,0), sub-lattice (0,0,0) -> offsets (1/4, 1/2, 1/4)
    np.testing.assert_array_equal(x[0], [0.025, 0.1, 0.075])
    # particle 1: sub-lattice x1 index 1 -> offset 3/4
    np.testing.assert_allclose(x[1], [0.075, 0.1, 0.075], rtol=1e-15)
    # particle ppc: next cell in x1
    np.testing.assert_allclose(x[4], [0.125, 0.1, 0.075])
    assert np.all(u[:, 1] == 0.5)
    # regenerate a subset by index: identical
    idx = np.array([7, 31, 60])
    xs, us = workload.load_particles(g, sp, idx)
    np.testing.assert_array_equal(xs, x[idx])
    np.testing.assert_array_equal(us, u[idx])
    q = workload.macro_charge(g, sp)
    assert math.isclose(q * x.shape[0], -g.dvol * g.ncells)


def test_config_shapes():
    g, sp, steps = workload.config0()
    assert g.nx == (64, 64, 1) and workload.n_particles(g, sp[0]) == 65536 and steps == 100
    assert abs(g.dt - 0.99 / math.sqrt(200)) < 1e-15
    g3, sp3, steps3 = workload.config3()
    assert workload.n_particles(g3, sp3[0]) == 268435456 and steps3 == 200


def test_config4_scan_draws():
    sims, steps = workload.config4()
    assert len(sims) == 64 and steps == 500
    again, _ = workload.config4()
    assert [(g.nx, s[0].ppc, s[0].density, las.vosc) for g, s, las in sims] == \
        [(g.nx, s[0].ppc, s[0].density, las.vosc) for g, s, las in again]
    for g, (sp,), las in sims:
        assert g.nx[0] in (128, 256, 512, 1024) and g.nx[1] in (64, 128, 256, 512) and g.nx[2] == 1
        assert sp.ppc_total in (4, 8, 16, 32)
        assert 0.5 <= sp.density < 2.0 and 0.5 <= las.vosc < 3.0
        assert g.rho_bg == sp.density and g.move_window  # neutral, window at c
        assert sp.uth == (0.0, 0.0, 0.0) and sp.ufl == (0.0, 0.0, 0.0)  # cold
        assert abs(g.dt - 0.99 / math.sqrt(1 / 0.05 ** 2 + 1 / 0.2 ** 2)) < 1e-15
        # omega0 = 10 w_p: 10 n^-1/2 of the member's own plasma frequency
        assert las.rkkp == 10.0 and las.wavetype == 1 and not las.antenna
        assert las.w0 <= 0.25 * g.nx[1] * g.dx[1] + 1e-12
        # the whole pulse (front 1.0 behind the edge, rise + fall behind it) is in the box
        assert g.nx[0] * g.dx[0] - las.start - las.rise - las.fall > 0.0
    # uneven sizes: several distinct grids and particle counts
    assert len({g.nx for g, _, _ in sims}) > 8
    assert len({workload.n_particles(g, s[0]) for g, s, _ in sims}) > 8
    assert len({round(las.vosc, 6) for _, _, las in sims}) == 64


def test_config1_pulse_intensity_fwhm_is_the_stated_duration():
    """The 2D wakefield stand-in's pulse: intensity (envelope squared) full width
    at half maximum 1.5 with the thesis' polynomial rise and fall."""
    import oracle
    _, _, las, _ = workload.config1()
    xi = np.linspace(0.0, las.rise + las.length + las.fall, 200001)
    inten = oracle.laser_envelope(xi, las.rise, las.length, las.fall) ** 2
    above = xi[inten >= 0.5]
    assert abs((above[-1] - above[0]) - 1.5) < 2e-3


def test_config1_vacuum_gap_puts_the_plasma_edge_ahead_of_the_pulse():
    g, sps, las, _ = workload.config1(vacuum_gap=2.0)
    edge = g.nx[0] * g.dx[0] - las.start + 2.0
    x = np.array([[edge - 1e-3, 1.0, 0.0], [edge + 1e-3, 1.0, 0.0]])
    w = workload.profile_weight(sps[0], x)
    assert w[0] == 0.0 and w[1] == 1.0
    assert workload.load_weighted(g, sps[0])[0].shape[0] == 0  # the window starts in vacuum


def test_cylindrical_recipe():
    """r-z input recipe: the Cartesian lattice of the (z, r) cells from r =
    -dr/2, the first cell's points below the axis reflected; positions in
    [0, r_max); dt at 0.99 of the r-z bound, below the Cartesian one."""
    import math
    import numpy as np
    g = workload.cyl_grid(8, 6, 0.1, 0.2)
    assert g.coords == "cylindrical" and g.xmin[1] == -0.1
    assert abs(g.dt - 0.99 / math.sqrt(1 / 0.1 ** 2 + workload.CYL_RADIAL_EIG / 0.2 ** 2)) < 1e-15
    assert g.dt < workload.courant_dt((0.1, 0.2, 1.0), 2)
    sp = workload.Species(rqm=-1.0, ppc=(2, 2, 1), uth=(0.1,) * 3, seed=3)
    x, u = workload.load_cylindrical(g, sp)
    xc, uc = workload.load_particles(g, sp)
    rmax = (6 - 0.5) * 0.2
    assert np.all(x[:, 1] >= 0.0) and np.all(x[:, 1] < rmax)
    np.testing.assert_array_equal(x[:, 1], np.abs(xc[:, 1]))
    np.testing.assert_array_equal(x[:, 0], xc[:, 0])
    np.testing.assert_array_equal(u, uc)
    below = xc[:, 1] < 0.0
    assert below.sum() == 8 * 2  # one of the two r points of each first-row cell, per z point
