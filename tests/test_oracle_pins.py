"""Pins of the FP64 oracle against what the physics and the mathematics fix.

These tests check the oracle (``oracle/``) against closed forms, invariants,
textbook special cases and exact rational brute force -- never against a copy
of its own formulas.  Each test names the passage of Hemker's thesis
(arxiv 1503.00276, ch. 3) that the checked function follows.
"""
import math
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle
import workload

# staggering of E1,E2,E3,B1,B2,B3 as read off the difference stencils of the
# field equations (eqs. 2d-field-solve-*), in cell units
STAG = np.array([[0.5, 0, 0], [0, 0.5, 0], [0, 0, 0.5], [0, 0.5, 0.5], [0.5, 0, 0.5], [0.5, 0.5, 0]])


def _grid(ndim, nx, dx, dt=None, **kw):
    nx = tuple(nx) + (1,) * (3 - len(nx))
    dx = tuple(dx) + (1.0,) * (3 - len(dx))
    if dt is None:
        dt = workload.courant_dt(dx, ndim)
    return workload.Grid(ndim=ndim, nx=nx, dx=dx, dt=dt, **kw)


def _zeros(g):
    return [np.zeros((g.nx[2], g.nx[1], g.nx[0])) for _ in range(6)]


# ---------------------------------------------------------------------------
# Boris push (eq. momentum-update) and position update (eq. 2d-position-update)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("bdir", [(0, 0, 1.0), (0.3, -0.5, 0.8)])
def test_gyration_phase_radius_and_speed(bdir):
    """Uniform B, E = 0: each step rotates u_perp by exactly 2 atan(|t|),
    |t| = |(q/m)(dt/2) B| / gamma; |u| is conserved to rounding; the positions lie
    on a circle of radius (dt |u_perp| / gamma) / (2 sin(theta/2))."""
    b = np.array(bdir) / np.linalg.norm(bdir) * 1.3
    g = _grid(3, (16, 16, 16), (0.1, 0.1, 0.1), dt=0.05, b0=tuple(b))
    rqm = -1.0
    f = _zeros(g)
    x = np.array([[0.8, 0.8, 0.8]])
    u = np.array([[0.4, -0.2, 0.3]])
    bh = b / np.linalg.norm(b)
    upar = u[0] @ bh
    gam = math.sqrt(1 + u[0] @ u[0])
    tmag = abs(g.dt / (2 * rqm)) * np.linalg.norm(b) / gam
    theta = 2 * math.atan(tmag)
    uperp_mag = np.linalg.norm(u[0] - upar * bh)
    R = (g.dt * uperp_mag / gam) / (2 * math.sin(theta / 2))
    xs, us = [x[0].copy()], [u[0].copy()]
    for _ in range(300):
        x, u = oracle.advance_particles(g, f, rqm, x, u, wrap=False)
        xs.append(x[0].copy())
        us.append(u[0].copy())
    us = np.array(us)
    xs = np.array(xs)
    # speed conserved exactly up to rounding
    speeds = np.linalg.norm(us, axis=1)
    assert np.max(np.abs(speeds / speeds[0] - 1)) < 1e-14
    # parallel momentum unchanged
    assert np.max(np.abs(us @ bh - upar)) < 1e-14
    # rotation angle per step (electron: rotates in the +B sense)
    e1 = us[0] - upar * bh
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(bh, e1)
    perp = us - np.outer(us @ bh, bh)
    ang = np.unwrap(np.arctan2(perp @ e2, perp @ e1))
    assert np.max(np.abs(np.diff(ang) - theta)) < 1e-13
    # circle: centre from the perpendicular projection of the guiding centre
    xp = xs - np.outer(xs @ bh, bh)
    p0, p1, p2 = xp[0], xp[1], xp[2]
    # circumcentre of three points in the perpendicular plane
    a, bb = p1 - p0, p2 - p0
    axb = np.cross(a, bb)
    centre = p0 + np.cross((a @ a) * bb - (bb @ bb) * a, axb) / (2 * (axb @ axb))
    radii = np.linalg.norm(xp - centre, axis=1)
    assert np.max(np.abs(radii / R - 1)) < 1e-11
    # continuous limit: omega_c = |B/rqm|/gamma, r_L = |u_perp| |rqm| / |B|
    assert abs(theta / g.dt / (np.linalg.norm(b) / gam) - 1) < (g.dt * 1.3) ** 2
    assert abs(R / (uperp_mag / np.linalg.norm(b)) - 1) < (g.dt * 1.3) ** 2


def test_e_only_acceleration_is_exact():
    """B = 0: u^{n+1/2} = u^{n-1/2} + (q/m) E dt exactly."""
    e = np.array([0.2, -0.1, 0.05])
    g = _grid(2, (8, 8), (0.1, 0.1), dt=0.05, e0=tuple(e))
    f = _zeros(g)
    x = np.array([[0.4, 0.4, 0.0]])
    u = np.array([[0.1, 0.0, -0.2]])
    for n in range(1, 41):
        x, u = oracle.advance_particles(g, f, -1.0, x, u)
        np.testing.assert_allclose(u[0], np.array([0.1, 0.0, -0.2]) - n * g.dt * e, rtol=0, atol=4e-15)


def test_free_streaming_and_periodic_wrap():
    """Zero fields: x^n = x^0 + n dt u/gamma (mod L); only in-plane components move in 2D."""
    g = _grid(2, (8, 6), (0.1, 0.2))
    f = _zeros(g)
    x0 = np.array([[0.05, 1.1, 0.0], [0.79, 0.01, 0.0]])
    u0 = np.array([[0.9, -0.4, 0.3], [-2.0, 1.5, -0.7]])
    x, u = x0.copy(), u0.copy()
    nsteps = 57
    for _ in range(nsteps):
        x, u = oracle.advance_particles(g, f, -1.0, x, u)
    np.testing.assert_array_equal(u, u0)
    gam = np.sqrt(1 + np.sum(u0 ** 2, axis=1))
    L = np.array([0.8, 1.2])
    expect = np.mod(x0[:, :2] + nsteps * g.dt * u0[:, :2] / gam[:, None], L)
    np.testing.assert_allclose(x[:, :2], expect, atol=1e-12)
    assert np.all(x[:, 2] == 0.0)
    assert np.all((x[:, :2] >= 0) & (x[:, :2] < L))


def test_exb_drift():
    """Crossed uniform E and B with |E| < |B|: the averaged velocity is E x B / B^2."""
    E, B = 0.1, 1.0
    g = _grid(2, (8, 8), (0.1, 0.1), dt=0.1, e0=(0.0, E, 0.0), b0=(0.0, 0.0, B))
    f = _zeros(g)
    x = np.array([[0.4, 0.4, 0.0]])
    u = np.zeros((1, 3))
    xs = [x[0, 0]]
    for _ in range(20000):
        x, u = oracle.advance_particles(g, f, -1.0, x, u, wrap=False)
        xs.append(x[0, 0])
    xs = np.array(xs)
    # least-squares slope over the whole run removes the gyration
    t = np.arange(xs.size) * g.dt
    slope = np.polyfit(t, xs, 1)[0]
    assert abs(slope / (E / B) - 1) < 2e-4


# ---------------------------------------------------------------------------
# Field weighting (eq. 2d-field-weighting-e3 and its 3D extension)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("ndim", [2, 3])
def test_gather_reproduces_linear_fields(ndim):
    """Linear interpolation from each component's own staggered lattice is exact
    for fields that are linear in position."""
    rng = np.random.default_rng(5)
    nx = (10, 9, 8)[:ndim]
    dx = (0.1, 0.15, 0.12)[:ndim]
    e0, b0 = (0.01, 0.02, 0.03), (-0.01, 0.04, 0.05)
    g = _grid(ndim, nx, dx, e0=e0, b0=b0)
    a = rng.normal(size=6)
    bvec = rng.normal(size=(6, 3))
    kk, jj, ii = np.meshgrid(np.arange(g.nx[2]), np.arange(g.nx[1]), np.arange(g.nx[0]), indexing="ij")
    idx = [ii, jj, kk]
    fields = []
    for c in range(6):
        val = np.full(ii.shape, a[c])
        for d in range(ndim):
            val = val + bvec[c, d] * (idx[d] + STAG[c, d]) * g.dx[d]
        fields.append(val)
    for _ in range(50):
        x = np.zeros(3)
        for d in range(ndim):
            x[d] = rng.uniform(1.5, g.nx[d] - 2.0) * g.dx[d]
        got = oracle.gather(g, fields, x)
        for c in range(6):
            want = a[c] + sum(bvec[c, d] * x[d] for d in range(ndim)) + (e0 + b0)[c]
            assert abs(got[c] - want) < 1e-13


def test_gathered_b_sits_where_the_curl_puts_it():
    """B made by the solver's own half step from a smooth E, gathered at arbitrary
    points, equals -(dt/2) curl E of the continuous field to O((k dx)^2); a B
    lattice shifted by half a cell would give O(k dx) errors."""
    g = _grid(3, (40, 40, 40), (0.1, 0.1, 0.1))
    L = 4.0
    k = 2 * math.pi / L
    kk, jj, ii = np.meshgrid(np.arange(40), np.arange(40), np.arange(40), indexing="ij")
    idx = [ii, jj, kk]

    def pos(c, d):
        return (idx[d] + STAG[c, d]) * 0.1

    f = _zeros(g)
    f[0] = np.sin(k * pos(0, 1)) * np.cos(k * pos(0, 2))         # E1(y, z)
    f[1] = np.cos(k * pos(1, 2)) + 0.5 * np.sin(k * pos(1, 0))   # E2(z, x)
    f[2] = np.sin(k * pos(2, 0)) * np.sin(k * pos(2, 1))         # E3(x, y)
    # one solve from E^n with B^n = 0, J = 0: B^{n+1} = -dt curl E^n + O(dt^3 k^3)
    out = oracle.field_solve(g, f, [np.zeros_like(f[0])] * 3)
    rng = np.random.default_rng(1)

    def curlE(x):
        X, Y, Z = x
        dE3dy = k * np.sin(k * X) * np.cos(k * Y)
        dE2dz = -k * np.sin(k * Z)
        dE1dz = -k * np.sin(k * Y) * np.sin(k * Z)
        dE3dx = k * np.cos(k * X) * np.sin(k * Y)
        dE2dx = 0.5 * k * np.cos(k * X)
        dE1dy = k * np.cos(k * Y) * np.cos(k * Z)
        return np.array([dE3dy - dE2dz, dE1dz - dE3dx, dE2dx - dE1dy])

    for _ in range(40):
        x = rng.uniform(0.5, 3.5, size=3)
        got = oracle.gather(g, out, x)[3:]
        want = -g.dt * curlE(x)
        err = np.max(np.abs(got - want)) / (g.dt * k)
        assert err < 0.02, err


# ---------------------------------------------------------------------------
# Charge-conserving deposit (TRISTAN / Villasenor-Buneman), eq. continuity
# ---------------------------------------------------------------------------

def _div_j(g, cur):
    div = (cur[0] - np.roll(cur[0], 1, axis=2)) / g.dx[0] + (cur[1] - np.roll(cur[1], 1, axis=1)) / g.dx[1]
    if g.ndim == 3:
        div = div + (cur[2] - np.roll(cur[2], 1, axis=0)) / g.dx[2]
    return div


def _paths(ndim, rng, g, n):
    """Random paths with |dx_d| < dx_d, plus face, corner and exact-node cases."""
    out = []
    for _ in range(n):
        x0 = np.zeros(3)
        d = np.zeros(3)
        for k in range(ndim):
            x0[k] = rng.uniform(0, g.nx[k]) * g.dx[k]
            d[k] = rng.uniform(-0.99, 0.99) * g.dx[k]
        out.append((x0, x0 + d))
    # corner crossing through the shared edge/vertex
    x0 = np.array([2.75, 3.75, 4.75])[:3] * np.array(g.dx)
    out.append((x0, x0 + 0.5 * np.array(g.dx) * np.array([1, 1, 1 if ndim == 3 else 0])))
    # start exactly on a node, move backwards across every face
    x0 = np.array([3.0, 2.0, 5.0]) * np.array(g.dx)
    out.append((x0, x0 - 0.3 * np.array(g.dx) * np.array([1, 1, 1 if ndim == 3 else 0])))
    # end exactly on a face
    x0 = np.array([3.25, 2.5, 1.5]) * np.array(g.dx)
    out.append((x0, x0 + np.array([0.75, 0.0, 0.0]) * np.array(g.dx)))
    # across the periodic seam
    x0 = np.array([0.02, 0.03, 0.01]) * np.array(g.dx)
    out.append((x0, x0 - np.array([0.5, 0.4, 0.3 if ndim == 3 else 0]) * np.array(g.dx)))
    for o in out:
        if ndim == 2:
            o[0][2] = o[1][2] = 0.0
    return out


@pytest.mark.parametrize("ndim", [2, 3])
def test_deposit_satisfies_discrete_continuity(ndim):
    """(rho^{n+1} - rho^n)/dt + div J^{n+1/2} = 0 at every node, to rounding, for
    every path: the property both deposit schemes of the thesis are built on."""
    rng = np.random.default_rng(11 + ndim)
    g = _grid(ndim, (7, 6, 5)[:ndim], (0.1, 0.13, 0.11)[:ndim])
    q = -0.37
    for xo, xn in _paths(ndim, rng, g, 200):
        cur = oracle.deposit_vb(g, xo, xn, 0.1, q)
        xw = xn.copy()
        L = np.array(g.nx) * np.array(g.dx)
        for d in range(ndim):
            xw[d] = xw[d] % L[d]
        r0 = oracle.deposit_rho(g, xo, q)
        r1 = oracle.deposit_rho(g, xw, q)
        resid = (r1 - r0) / g.dt + _div_j(g, cur)
        scale = abs(q) / g.dvol / g.dt
        assert np.max(np.abs(resid)) < 1e-13 * scale


def _hat(s):
    a = abs(s)
    return 1 - a if a < 1 else Fr(0)


def _exact_current(ndim, a, b, v3):
    """Exact current of the straight path a -> b (cell units, dx = dt = q = 1):
    J_d(face m+1/2, nodes n_t) = integral over the step of
    v_d * [x_d(t) in cell m] * prod_t W(x_t(t) - n_t), W the linear hat; 2D3V J3
    at node (n_1, n_2) = integral of v3 * W W.  Piecewise-polynomial integrand
    of degree <= 2 between breakpoints, so Simpson's rule is exact."""
    dims = list(range(ndim))
    ts = {Fr(0), Fr(1)}
    for d in dims:
        if b[d] != a[d]:
            lo, hi = min(a[d], b[d]), max(a[d], b[d])
            for m in range(math.floor(lo), math.ceil(hi) + 1):
                t = (Fr(m) - a[d]) / (b[d] - a[d])
                if 0 < t < 1:
                    ts.add(t)
    ts = sorted(ts)
    J = {}

    def xat(t):
        return [a[d] + t * (b[d] - a[d]) for d in dims]

    for t0, t1 in zip(ts[:-1], ts[1:]):
        tm = (t0 + t1) / 2
        cell = [math.floor(v) for v in xat(tm)]
        h = t1 - t0
        for d in dims:
            tr = [e for e in dims if e != d]
            for corner in range(1 << len(tr)):
                nodes = [cell[e] + ((corner >> r) & 1) for r, e in enumerate(tr)]

                def f(t):
                    x = xat(t)
                    w = Fr(1)
                    for e, nd in zip(tr, nodes):
                        w *= _hat(x[e] - nd)
                    return (b[d] - a[d]) * w

                val = h / 6 * (f(t0) + 4 * f(tm) + f(t1))
                key = [0, 0, 0]
                key[d] = cell[d]
                for e, nd in zip(tr, nodes):
                    key[e] = nd
                key = (d,) + tuple(key)
                J[key] = J.get(key, Fr(0)) + val
        if ndim == 2:
            for corner in range(4):
                nodes = [cell[0] + (corner & 1), cell[1] + (corner >> 1)]

                def f3(t):
                    x = xat(t)
                    return v3 * _hat(x[0] - nodes[0]) * _hat(x[1] - nodes[1])

                val = h / 6 * (f3(t0) + 4 * f3(tm) + f3(t1))
                key = (2, nodes[0], nodes[1], 0)
                J[key] = J.get(key, Fr(0)) + val
    return J


@pytest.mark.parametrize("ndim", [2, 3])
def test_deposit_equals_exact_shape_flux_integral(ndim):
    """Brute force in rational arithmetic: the oracle's orthogonal-move average,
    segment by segment, equals the exact time integral of the shape-weighted
    flux (this pins the Delta y Delta z / 12 cross terms of the 3D scheme and the
    2D3V J3)."""
    rng = np.random.default_rng(100 + ndim)
    n = 8
    g = _grid(ndim, (n,) * ndim, (1.0,) * ndim, dt=1.0)
    cases = []
    for _ in range(60):
        a = [Fr(int(rng.integers(2, 5))) + Fr(int(rng.integers(0, 1024)), 1024) for _ in range(ndim)]
        dd = [Fr(int(rng.integers(-1000, 1001)), 1024) for _ in range(ndim)]
        cases.append((a, [a[i] + dd[i] for i in range(ndim)]))
    cases.append(([Fr(3, 4)] * ndim, [Fr(5, 4)] * ndim))                     # corner crossing
    cases.append(([Fr(3)] * ndim, [Fr(3) - Fr(3, 10)] * ndim))               # from a node backwards
    cases.append(([Fr(9, 4)] + [Fr(5, 2)] * (ndim - 1), [Fr(3)] + [Fr(5, 2)] * (ndim - 1)))  # end on a face
    v3 = Fr(3, 7)
    for a, b in cases:
        af = np.zeros(3)
        bf = np.zeros(3)
        af[:ndim] = [float(v) for v in a]
        bf[:ndim] = [float(v) for v in b]
        cur = oracle.deposit_vb(g, af, bf, float(v3), 1.0)
        exact = _exact_current(ndim, a, b, v3)
        got = {}
        for c in range(3):
            nz = np.argwhere(cur[c] != 0.0)
            for k, j, i in nz:
                got[(c, int(i), int(j), int(k))] = cur[c][k, j, i]
        keys = set(got) | {(c, i % n, j % n, (k % n) if ndim == 3 else 0) for (c, i, j, k) in exact}
        ex = {}
        for (c, i, j, k), v in exact.items():
            kk = (c, i % n, j % n, (k % n) if ndim == 3 else 0)
            ex[kk] = ex.get(kk, Fr(0)) + v
        for key in keys:
            assert abs(got.get(key, 0.0) - float(ex.get(key, 0))) < 1e-15, (key, a, b)


# ---------------------------------------------------------------------------
# Field solve (eqs. 2d-field-solve-b-part1, -e, -b-part2; 3D extension)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("ndim,m", [(2, (1, 2, 0)), (2, (3, 0, 0)), (3, (1, 2, 1)), (3, (0, 1, 3))])
def test_yee_amplification_matches_discrete_dispersion(ndim, m):
    """The solver's one-step map on a single Fourier mode, measured by applying it
    to basis fields, has eigenvalues exp(+-i w dt) (twice: two polarisations)
    and 1 (twice: the longitudinal modes), with
    (sin(w dt/2)/dt)^2 = sum_d (sin(k_d dx_d/2)/dx_d)^2."""
    nx = (8, 8, 8)[:ndim]
    dx = (0.1, 0.13, 0.07)[:ndim]
    g = _grid(ndim, nx, dx)
    L = [g.nx[d] * g.dx[d] for d in range(3)]
    k = np.array([2 * math.pi * m[d] / L[d] if d < ndim else 0.0 for d in range(3)])
    kk, jj, ii = np.meshgrid(np.arange(g.nx[2]), np.arange(g.nx[1]), np.arange(g.nx[0]), indexing="ij")
    idx = [ii, jj, kk]

    def phase(c):
        return sum(k[d] * (idx[d] + STAG[c, d]) * g.dx[d] for d in range(ndim))

    N = ii.size
    zero_j = [np.zeros(ii.shape)] * 3
    M = np.zeros((6, 6), dtype=complex)
    for c in range(6):
        for kind in ("cos", "sin"):
            f = _zeros(g)
            f[c] = np.cos(phase(c)) if kind == "cos" else np.sin(phase(c))
            out = oracle.field_solve(g, f, zero_j)
            col = np.array([np.sum(out[c2] * np.exp(-1j * phase(c2))) * 2 / N for c2 in range(6)])
            col = col if kind == "cos" else col * 1j
            if kind == "cos":
                M[:, c] = col
            else:
                np.testing.assert_allclose(col, M[:, c], atol=1e-12)
    lam = np.linalg.eigvals(M)
    np.testing.assert_allclose(np.abs(lam), 1.0, atol=1e-12)
    s = math.sqrt(sum((math.sin(k[d] * g.dx[d] / 2) / g.dx[d]) ** 2 for d in range(ndim)))
    w = 2 * math.asin(g.dt * s) / g.dt
    args = np.sort(np.angle(lam))
    want = np.sort([-w * g.dt] * 2 + [0.0] * 2 + [w * g.dt] * 2)
    np.testing.assert_allclose(args, want, atol=1e-12)


# ---------------------------------------------------------------------------
# Smoothing (appendix nl_smooth)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("weights", [(1.0, 2.0, 1.0), (1.0, 6.0, 1.0)])
def test_smoothing_transfer_function(weights):
    """One pass of (w0,w1,w0)/sum on cos(k x) multiplies it by
    (w1 + 2 w0 cos(k dx))/(w1 + 2 w0); for (1,2,1) that is cos^2(k dx/2).
    Passes and directions multiply."""
    g = _grid(2, (32, 16), (0.1, 0.2), smooth_level=(2, 1, 0), smooth_w=(weights, weights, weights))
    kx = 2 * math.pi * 3 / (32 * 0.1)
    ky = 2 * math.pi * 2 / (16 * 0.2)
    jj, ii = np.meshgrid(np.arange(16), np.arange(32), indexing="ij")
    f = np.cos(kx * ii * 0.1) * np.cos(ky * jj * 0.2)
    out = oracle.smooth(g, f[None])[0]
    w0, w1, _ = weights

    def T(k, d):
        return (w1 + 2 * w0 * math.cos(k * d)) / (w1 + 2 * w0)

    want = f * T(kx, 0.1) ** 2 * T(ky, 0.2)
    np.testing.assert_allclose(out, want, atol=1e-14)
    if weights == (1.0, 2.0, 1.0):
        assert abs(T(kx, 0.1) - math.cos(kx * 0.1 / 2) ** 2) < 1e-15


# ---------------------------------------------------------------------------
# Whole step: Gauss law, cold plasma oscillation, energy, diagnostics
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("ndim", [2, 3])
def test_gauss_law_preserved_over_steps(ndim):
    """Yee + a charge-conserving deposit keep div E - rho constant to rounding."""
    if ndim == 2:
        g = _grid(2, (24, 16), (0.1, 0.12), init_e_gauss_x1=True)
        sp = workload.Species(ppc=(2, 2, 1), uth=(0.2, 0.2, 0.2), seed=3, perturb_delta=0.05,
                              perturb_k=2 * math.pi / 2.4)
    else:
        g = _grid(3, (8, 8, 6), (0.1, 0.1, 0.1))
        sp = workload.Species(ppc=(2, 1, 1), uth=(0.2, 0.2, 0.2), seed=4)
    st = oracle.from_workload(g, [sp])
    r0 = st.gauss_residual()
    assert r0 < 1e-12
    for _ in range(5):
        st.step(8)
        assert abs(st.gauss_residual() - r0) < 1e-12


def test_cold_plasma_oscillation_frequency():
    """Cold uniform plasma, small x1 displacement, k dx << 1: leapfrog gives
    sin(w dt/2) = w_p dt/2 with w_p = 1 (normalised units); the amplitude stays
    constant (a field sampled half a cell off would grow or damp it)."""
    nx = 512
    g = _grid(2, (nx, 2), (0.2, 0.2), init_e_gauss_x1=True)
    L = nx * 0.2
    k = 2 * math.pi / L
    sp = workload.Species(ppc=(4, 1, 1), seed=1, perturb_delta=1e-3, perturb_k=k)
    st = oracle.from_workload(g, [sp])
    xg = (np.arange(nx) + 0.5) * 0.2
    amps = []
    nsteps = 260
    for _ in range(nsteps):
        amps.append(np.sum(st.fld[0][0, 0, :] * np.cos(k * xg)) * 2 / nx)
        st.step(1)
    a = np.array(amps)
    zc = []
    for n in range(len(a) - 1):
        if a[n] == 0 or a[n] * a[n + 1] < 0:
            zc.append(n + a[n] / (a[n] - a[n + 1]))
    half_periods = np.diff(zc)
    w = math.pi / (np.mean(half_periods) * g.dt)
    w_expect = 2 * math.asin(g.dt / 2) / g.dt
    assert abs(w / w_expect - 1) < 3e-4
    peaks = [np.max(np.abs(a[int(zc[i]):int(zc[i + 1]) + 1])) for i in range(len(zc) - 1)]
    assert abs(peaks[-1] / peaks[0] - 1) < 2e-3


def test_energy_roughly_conserved_and_diag_closed_forms():
    """Field energy of a known field, kinetic energy of one particle, rho of a
    particle on a node, total charge; total energy drift over a short run."""
    g = _grid(2, (8, 8), (0.1, 0.1))
    f = _zeros(g)
    f[2][0, 3, 4] = 2.0
    st = oracle.State(g, [workload.Species()], [np.array([[0.3, 0.4, 0.0]])], [np.array([[0.3, 0.4, 0.0]])],
                      [-0.01], fields=f)
    assert abs(st.field_energy() - 0.5 * 4.0 * 0.01) < 1e-15
    assert abs(st.kinetic_energy() - 0.01 * (math.sqrt(1.25) - 1)) < 1e-15
    r = oracle.deposit_rho(g, np.array([0.3, 0.4, 0.0]), -0.01)
    assert abs(r[0, 4, 3] + 1.0) < 1e-13 and abs(np.sum(r) * g.dvol + 0.01) < 1e-15
    assert np.count_nonzero(np.abs(r) > 1e-15) == 1
    # thermal plasma: total energy conserved to a small fraction of the kinetic energy
    g2 = _grid(2, (32, 32), (0.1, 0.1))
    sp = workload.Species(ppc=(2, 2, 1), uth=(0.05, 0.05, 0.05), seed=9)
    st2 = oracle.from_workload(g2, [sp])
    e0 = st2.field_energy() + st2.kinetic_energy()
    st2.step(40)
    e1 = st2.field_energy() + st2.kinetic_energy()
    assert abs(e1 - e0) < 0.02 * e0


# ---------------------------------------------------------------------------
# Tile binning (not in the paper)
# ---------------------------------------------------------------------------

def test_tile_binning_matches_brute_force():
    g = _grid(3, (16, 8, 8), (0.1, 0.1, 0.1))
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, size=(500, 3)) * np.array([1.6, 0.8, 0.8])
    x[:5] = [[0, 0, 0], [1.6 - 1e-15, 0.8 - 1e-15, 0.8 - 1e-15], [0.4, 0.4, 0.4], [0.8, 0, 0], [0.39999, 0, 0]]
    tile = (4, 4, 2)
    tid, counts, order = oracle.tile_bin(g, tile, x)
    nt = (4, 2, 4)
    want_tid = []
    for p in range(x.shape[0]):
        c = [min(int(math.floor(x[p, d] / 0.1)), g.nx[d] - 1) for d in range(3)]
        want_tid.append(((c[2] // tile[2]) * nt[1] + c[1] // tile[1]) * nt[0] + c[0] // tile[0])
    np.testing.assert_array_equal(tid, want_tid)
    np.testing.assert_array_equal(counts, np.bincount(want_tid, minlength=32))
    np.testing.assert_array_equal(order, np.argsort(np.array(want_tid), kind="stable"))
