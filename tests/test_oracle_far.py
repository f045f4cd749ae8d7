"""Pins of the oracle's far field past the cutoff (orc_far_tail): eq. (17) for
every pair beyond r_cut, with the lattice images beyond r_cut replaced by the
lattice continuum (section 7's asymptote-accelerated image sums; sections 3
and 6.2 repeat the cell until the energy converges), for one, two and three
periodic axes."""
import numpy as np
import pytest

C_ASYM = 12.0 * (4.0 * np.pi / 9.0) ** 3


def _pref(n, q, dV):
    """1/2 dV^2 n_i n_j (-C / (q_i^2 q_j^2 (q_i^2 + q_j^2))) for all ordered pairs."""
    u = q ** 2
    return 0.5 * dV ** 2 * np.outer(n, n) * (-C_ASYM / (np.outer(u, u) * (u[:, None] + u[None, :])))


def _positions(idx, dims, cell):
    return (np.asarray(idx, dtype=float) / np.asarray(dims, dtype=float)) @ cell


@pytest.mark.parametrize("skew", [False, True])
def test_two_axis_continuum_is_the_radial_integral(oracle_mod, skew):
    """Two periodic axes: each pair's factor is (1/A) times the integral of r^-6 over
    the plane of images outside the cutoff sphere, done here by scipy's adaptive
    quadrature (in the radius rho within the plane), for pairs whose normal
    separation |z| is below and above r_cut; the normal comes from the cell."""
    quad = pytest.importorskip("scipy.integrate").quad
    dims = (10, 12, 40)
    cell = np.array([[10.0, 0, 0], [0.0, 12.0, 0], [0, 0, 40.0]])
    if skew:
        cell = np.array([[10.0, 0, 0], [5.0, 11.0, 0], [1.5, -2.0, 40.0]])
    idx = np.array([[0, 0, 0], [3, 4, 5], [7, 1, 31], [2, 9, 18]])
    n = np.array([0.7, 1.3, 0.4, 0.9])
    q = np.array([0.5, 1.1, 0.35, 2.0])
    rc = 9.0
    e = np.cross(cell[0], cell[1])
    A = np.linalg.norm(e)
    e /= A
    pos = _positions(idx, dims, cell)
    K = np.zeros((4, 4))
    for i in range(4):
        for j in range(4):
            z = abs(np.dot(pos[i] - pos[j], e))
            lo = np.sqrt(rc * rc - z * z) if z < rc else 0.0
            val, _ = quad(lambda rho: 2 * np.pi * rho * (rho * rho + z * z) ** -3, lo, np.inf,
                          epsabs=0, epsrel=1e-13, limit=200)
            K[i, j] = val / A
    dV = abs(np.linalg.det(cell)) / np.prod(dims)
    ref = float(np.sum(_pref(n, q, dV) * K))
    got = oracle_mod.far_tail_points(idx[:, 0], idx[:, 1], idx[:, 2], n, q, dims, cell, (1, 1, 0), rc)
    assert abs(got - ref) < 1e-11 * abs(ref), (got, ref)


def test_three_axis_continuum_is_the_radial_integral(oracle_mod):
    quad = pytest.importorskip("scipy.integrate").quad
    dims = (8, 8, 8)
    cell = np.array([[9.0, 0, 0], [1.0, 9.5, 0], [0.5, 0.7, 10.0]])
    idx = np.array([[0, 0, 0], [3, 4, 5], [7, 1, 2]])
    n = np.array([0.7, 1.3, 0.4])
    q = np.array([0.5, 1.1, 0.35])
    rc = 12.0
    V = abs(np.linalg.det(cell))
    val, _ = quad(lambda r: 4 * np.pi * r * r * r ** -6, rc, np.inf, epsabs=0, epsrel=1e-13)
    ref = float(np.sum(_pref(n, q, V / 512) * (val / V)))
    got = oracle_mod.far_tail_points(idx[:, 0], idx[:, 1], idx[:, 2], n, q, dims, cell, (1, 1, 1), rc)
    assert abs(got - ref) < 1e-11 * abs(ref), (got, ref)
    with pytest.raises(ValueError):   # an open cell: no lattice images
        oracle_mod.far_tail_points(idx[:, 0], idx[:, 1], idx[:, 2], n, q, dims, cell, (0, 0, 0), rc)


@pytest.mark.parametrize("rho", [0.0, 1e-4, 0.3, 2.0, 4.4, 4.5, 7.0, 9.99, 10.0, 10.01, 13.0, 30.0])
def test_line_integral_matches_quadrature(oracle_mod, rho):
    """orc_line_tail_integral, int_{x0}^inf dx / (rho^2 + x^2)^3 with
    x0 = sqrt(max(0, r_c^2 - rho^2)), r_c = 10, against scipy's adaptive quadrature:
    the series branch (rho / x0 < 1/2, up to rho = 4.47), the closed form beyond
    it, and x0 = 0 past the cutoff."""
    quad = pytest.importorskip("scipy.integrate").quad
    rc = 10.0
    x0 = np.sqrt(max(0.0, rc * rc - rho * rho))
    ref, _ = quad(lambda x: (rho * rho + x * x) ** -3, x0, np.inf, epsabs=0, epsrel=1e-13, limit=400)
    got = oracle_mod.line_tail_integral(rho, x0)
    assert abs(got - ref) < 2e-12 * abs(ref), (rho, got, ref)


def test_one_axis_continuum_is_the_line_integral(oracle_mod):
    """One periodic axis (the second lattice vector of a skewed cell): each pair's
    factor is (1/|a|) times the integral of r^-6 along the line of images outside
    the cutoff sphere, done here by scipy's adaptive quadrature with the pair's
    distance rho from the axis direction taken from the cell."""
    quad = pytest.importorskip("scipy.integrate").quad
    dims = (12, 10, 14)
    cell = np.array([[14.0, 0, 0], [3.0, 9.0, 0], [1.0, -2.0, 15.0]])
    idx = np.array([[0, 0, 0], [3, 4, 5], [7, 1, 11], [2, 9, 8], [11, 6, 3]])
    n = np.array([0.7, 1.3, 0.4, 0.9, 0.2])
    q = np.array([0.5, 1.1, 0.35, 2.0, 0.8])
    rc = 9.0
    a = cell[1]
    alen = np.linalg.norm(a)
    e = a / alen
    pos = _positions(idx, dims, cell)
    K = np.zeros((5, 5))
    for i in range(5):
        for j in range(5):
            d = pos[i] - pos[j]
            rho = np.linalg.norm(d - np.dot(d, e) * e)
            x0 = np.sqrt(rc * rc - rho * rho) if rho < rc else 0.0
            val, _ = quad(lambda x: (rho * rho + x * x) ** -3, x0, np.inf, epsabs=0, epsrel=1e-13, limit=400)
            K[i, j] = 2.0 * val / alen
    assert np.max(K) > 5 * np.min(K)           # pairs near and far from the axis
    dV = abs(np.linalg.det(cell)) / np.prod(dims)
    ref = float(np.sum(_pref(n, q, dV) * K))
    got = oracle_mod.far_tail_points(idx[:, 0], idx[:, 1], idx[:, 2], n, q, dims, cell, (0, 1, 0), rc)
    assert abs(got - ref) < 1e-11 * abs(ref), (got, ref)


def test_one_axis_factor_at_the_cutoff_radius(oracle_mod):
    """A pair whose distance from the axis is r_cut exactly (6 grid steps of
    16.4/8 bohr = 12.3 bohr = r_cut): x0 = sqrt(r_cut^2 - rho^2) is 0, and the
    factor is (2/|a|) 3 pi / (16 r_cut^5).  In floating point rho^2 comes out
    5.7e-14 below r_cut^2 here; the factor's square-root singularity at rho = r_cut
    would turn that into a 3e-8 change, so differences within 1e-12 r_cut^2 count
    as zero (as the pair sum's inclusive cutoff treats distances equal to r_cut)."""
    dims = (8, 5, 5)
    cell = np.diag([16.4, 9.0, 9.0])
    rc = 12.3
    n = np.array([1.0, 1.0])
    q = np.array([0.6, 0.9])
    dV = abs(np.linalg.det(cell)) / np.prod(dims)
    P = _pref(n, q, dV)
    idx = np.array([[0, 0, 0], [6, 0, 0]])
    both = oracle_mod.far_tail_points(idx[:, 0], idx[:, 1], idx[:, 2], n, q, dims, cell, (0, 1, 0), rc)
    only0 = oracle_mod.far_tail_points(idx[:1, 0], idx[:1, 1], idx[:1, 2], n[:1], q[:1], dims, cell, (0, 1, 0), rc)
    only1 = oracle_mod.far_tail_points(idx[1:, 0], idx[1:, 1], idx[1:, 2], n[1:], q[1:], dims, cell, (0, 1, 0), rc)
    K01 = (both - only0 - only1) / (2 * P[0, 1])
    ref = 2.0 / 9.0 * 3.0 * np.pi / (16.0 * rc ** 5)
    assert abs(K01 - ref) < 1e-12 * ref, (K01, ref)


@pytest.mark.parametrize("rc", [10.0, 25.0])
def test_one_axis_continuum_is_the_offset_average_of_the_lattice_sum(oracle_mod, rc):
    """The continuum stands for the images beyond r_cut.  For one periodic axis the
    lattice sum of r^-6 over the images beyond r_cut jumps as images cross the
    cutoff sphere, but its average over the pair's offset along the axis is the
    continuum: 20000 offsets across one period against the oracle's factor for
    pairs at several distances from the axis (2e-4)."""
    dims = (40, 8, 8)
    cell = np.array([[6.0, 0, 0], [0, 30.0, 0], [0, 0, 30.0]])
    n = np.array([1.0, 1.0])
    q = np.array([0.6, 0.9])
    dV = abs(np.linalg.det(cell)) / np.prod(dims)
    P = _pref(n, q, dV)
    for jb, jc in ((0, 0), (1, 0), (2, 3), (4, 5)):
        idx = np.array([[0, 0, 0], [0, jb, jc]])
        both = oracle_mod.far_tail_points(idx[:, 0], idx[:, 1], idx[:, 2], n, q, dims, cell, (1, 0, 0), rc)
        only0 = oracle_mod.far_tail_points(idx[:1, 0], idx[:1, 1], idx[:1, 2], n[:1], q[:1], dims, cell, (1, 0, 0), rc)
        only1 = oracle_mod.far_tail_points(idx[1:, 0], idx[1:, 1], idx[1:, 2], n[1:], q[1:], dims, cell, (1, 0, 0), rc)
        K01 = (both - only0 - only1) / (2 * P[0, 1])      # the cross term's factor
        rho = np.hypot(jb * 30.0 / 8, jc * 30.0 / 8)
        x = (np.arange(20000) + 0.5) / 20000 * 6.0
        M = int(np.ceil(8 * rc / 6.0)) + 2
        y = x[:, None] + 6.0 * np.arange(-M, M + 1)[None, :]
        r2 = y * y + rho * rho
        S = np.where(r2 > rc * rc, r2, np.inf) ** -3
        tail = 2.0 / 6.0 * oracle_mod.line_tail_integral(rho, 6.0 * M - 6.0)  # images past the window
        lat = float(np.mean(S.sum(axis=1))) + tail
        assert abs(K01 - lat) < 2e-4 * abs(lat), (rc, jb, jc, K01, lat)


def test_continuum_approaches_the_lattice_sum(oracle_mod):
    """The continuum stands for the images beyond r_cut.  Against the lattice sum of
    eq. (17) over those images (summed directly out to 8 r_cut, the continuum past
    that), for 48 points spread over a skewed cell: within 3 % at r_cut = 10, 20
    and within 1 % at 40, 80.  (For one pair alone the images just past r_cut make
    the error jump about with r_cut; over offsets spread across the cell the lattice
    sum averages to the continuum.)"""
    dims = (10, 12, 40)
    cell = np.array([[10.0, 0, 0], [4.0, 11.0, 0], [0, 0, 40.0]])
    rng = np.random.default_rng(5)
    K = 48
    idx = np.stack([rng.integers(0, 10, K), rng.integers(0, 12, K), rng.integers(15, 25, K)], 1)
    n = rng.uniform(0.3, 1.5, K)
    q = rng.uniform(0.3, 1.5, K)
    pos = _positions(idx, dims, cell)
    A = np.linalg.norm(np.cross(cell[0], cell[1]))
    dV = abs(np.linalg.det(cell)) / np.prod(dims)
    P = _pref(n, q, dV)
    for rc, tol in ((10.0, 0.03), (20.0, 0.03), (40.0, 0.01), (80.0, 0.01)):
        Rb = 8 * rc
        M = int(np.ceil(Rb / 9.0)) + 2
        m0, m1 = np.meshgrid(np.arange(-M, M + 1), np.arange(-M, M + 1), indexing="ij")
        L = m0.ravel()[:, None] * cell[0] + m1.ravel()[:, None] * cell[1]
        lat = 0.0
        for i in range(K):
            d = pos[i] - pos
            r = np.linalg.norm(d[:, None, :] + L[None, :, :], axis=2)
            sel = (r > rc) & (r <= Rb)
            S = np.sum(np.where(sel, r, np.inf) ** -6, axis=1) + (2 * np.pi / A) / (4 * np.maximum(Rb, np.abs(d[:, 2])) ** 4)
            lat += float(np.dot(P[i], S))
        got = oracle_mod.far_tail_points(idx[:, 0], idx[:, 1], idx[:, 2], n, q, dims, cell, (1, 1, 0), rc)
        assert abs(got - lat) < tol * abs(lat), (rc, got, lat)


def test_energy_plus_tail_converges(oracle_mod, oracle_spline):
    """Coarse periodic monolayer: the oracle's direct sums E(r_cut) and E(r_cut) + T(r_cut)
    at r_cut = 15, 25, 35 bohr.  The tail takes up what the direct sum still gains
    past each cutoff: against r_cut = 35, E + T moves by under a tenth of what E moves
    from 15 and under a hundredth from 25."""
    from paper_0810_2273_gb300 import inputs
    w = inputs.xe_monolayer((8, 14, 20))
    Es, Ts = [], []
    for rc in (15.0, 25.0, 35.0):
        P = oracle_mod.Problem(w["density"], w["lengths"], w["periodic"], w["n_cut"], rc, oracle_spline)
        Es.append(P.energy()["E"])
        Ts.append(P.far_tail())
    Es, Ts = np.array(Es), np.array(Ts)
    assert np.all(Ts < 0) and abs(Ts[0]) > abs(Ts[1]) > abs(Ts[2])
    d_direct = abs(Es[0] - Es[2]), abs(Es[1] - Es[2])
    d_tail = abs(Es[0] + Ts[0] - Es[2] - Ts[2]), abs(Es[1] + Ts[1] - Es[2] - Ts[2])
    assert d_tail[0] < 0.1 * d_direct[0] and d_tail[1] < 0.01 * d_direct[1], (d_direct, d_tail)


def test_energy_plus_tail_converges_on_a_wire(oracle_mod, oracle_spline):
    """A chain of rare-gas atoms 6 bohr apart, periodic along the chain only: the
    oracle's direct sums E(r_cut) and E(r_cut) + T(r_cut) at r_cut = 15, 20, 25, 35.
    Against r_cut = 35, E + T moves by under a twentieth of what E moves from 15
    and under a hundredth from 20 and from 25."""
    from paper_0810_2273_gb300 import inputs
    L, dims = (6.0, 14.0, 14.0), (8, 18, 18)
    n = inputs.density(dims, L, [((3.0, 7.0, 7.0), inputs.rare_gas_shells())], periodic=(1, 0, 0))
    Es, Ts = [], []
    for rc in (15.0, 20.0, 25.0, 35.0):
        P = oracle_mod.Problem(n, L, (1, 0, 0), 1e-6, rc, oracle_spline)
        Es.append(P.energy()["E"])
        Ts.append(P.far_tail())
    Es, Ts = np.array(Es), np.array(Ts)
    assert np.all(Ts < 0) and np.all(np.diff(np.abs(Ts)) < 0)
    d_direct = np.abs(Es[:3] - Es[3])
    d_tail = np.abs(Es[:3] + Ts[:3] - Es[3] - Ts[3])
    assert d_tail[0] < 0.05 * d_direct[0] and np.all(d_tail[1:] < 0.01 * d_direct[1:]), (d_direct, d_tail)


@pytest.mark.parametrize("periodic", [(1, 1, 0), (0, 1, 1), (1, 1, 1), (1, 0, 0), (0, 0, 1)])
def test_tail_potential_is_derivative_of_tail(oracle_mod, oracle_spline, periodic):
    """The far field's potential v_T = dT/dn_m / dV (mask frozen) against central
    differences of the oracle's T, at active points and at inactive points next
    to the active region (where only the gradient term of q0 acts)."""
    rng = np.random.default_rng(41)
    dims = (9, 8, 10)
    L = (6.0, 6.4, 7.0)
    n = 0.02 + 0.5 * rng.uniform(0, 1, size=dims) * np.exp(-rng.uniform(0, 3, size=dims))
    n_cut = 0.05
    n[np.abs(n - n_cut) < 0.01] += 0.03
    rc = 5.0
    P = oracle_mod.Problem(n, L, periodic, n_cut, rc, oracle_spline)
    v = P.far_tail_potential()
    flat = n.ravel()
    act = np.nonzero(flat >= 2 * n_cut)[0]
    ina = np.nonzero(flat < 0.5 * n_cut)[0]
    pts = np.concatenate([rng.choice(act, 6, replace=False), rng.choice(ina, 4, replace=False)])
    for m in pts:
        hstep = 1e-4 * flat[m]

        def T_at(delta):
            nn = flat.copy()
            nn[m] += delta
            return oracle_mod.Problem(nn.reshape(dims), L, periodic, n_cut, rc, oracle_spline).far_tail()
        fd = (T_at(hstep) - T_at(-hstep)) / (2 * hstep) / P.dV
        assert abs(fd - v.ravel()[m]) < 1e-6 * np.max(np.abs(v)), (m, fd, v.ravel()[m])


def test_tail_potential_is_derivative_of_tail_skewed(oracle_mod, oracle_spline):
    """The same on a skewed cell (periodic along its first two lattice vectors, the
    third tilted), where the planes' normal separation comes from the cell."""
    rng = np.random.default_rng(43)
    dims = (8, 9, 10)
    cell = np.array([[6.0, 0.0, 0.0], [2.5, 6.2, 0.0], [1.0, -0.8, 7.0]])
    n = 0.02 + 0.5 * rng.uniform(0, 1, size=dims) * np.exp(-rng.uniform(0, 3, size=dims))
    n_cut = 0.05
    n[np.abs(n - n_cut) < 0.01] += 0.03
    rc = 5.0
    per = (1, 1, 0)
    P = oracle_mod.Problem(n, None, per, n_cut, rc, oracle_spline, cell=cell)
    v = P.far_tail_potential()
    flat = n.ravel()
    act = np.nonzero(flat >= 2 * n_cut)[0]
    ina = np.nonzero(flat < 0.5 * n_cut)[0]
    pts = np.concatenate([rng.choice(act, 5, replace=False), rng.choice(ina, 3, replace=False)])
    for m in pts:
        hstep = 1e-4 * flat[m]

        def T_at(delta):
            nn = flat.copy()
            nn[m] += delta
            return oracle_mod.Problem(nn.reshape(dims), None, per, n_cut, rc, oracle_spline, cell=cell).far_tail()
        fd = (T_at(hstep) - T_at(-hstep)) / (2 * hstep) / P.dV
        assert abs(fd - v.ravel()[m]) < 1e-6 * np.max(np.abs(v)), (m, fd, v.ravel()[m])
