"""Pins of the oracle's tensor-product cubic spline through the phi table."""
import numpy as np
import pytest


def _grid(nD=40, Dmax=30.0, nd=20):
    D = Dmax * np.arange(nD) / (nD - 1)
    dl = np.arange(nd) / nd
    return D, dl


def test_spline_reproduces_nodes(oracle_mod):
    rng = np.random.default_rng(3)
    D, dl = _grid()
    nodes = rng.normal(size=(len(D), len(dl)))
    s = oracle_mod.Spline(nodes, D[-1])
    DD, LL = np.meshgrid(D, dl, indexing="ij")
    p, _, _ = s.eval(DD.ravel(), LL.ravel())
    assert np.max(np.abs(p - nodes.ravel())) < 1e-12


def test_spline_exact_on_cubics_meeting_boundary_conditions(oracle_mod):
    """f(D) g(delta) with f = D^2 - D^3/(3 Dmax), g = d^2 - d^3/(3 d_last) has zero
    slope at 0 and zero curvature at the last node in both variables, and lies in the
    tensor spline space: the interpolant must equal it everywhere, with derivatives."""
    D, dl = _grid()
    Dmax, dlast = D[-1], dl[-1]
    f = lambda x: x ** 2 - x ** 3 / (3 * Dmax)
    fp = lambda x: 2 * x - x ** 2 / Dmax
    g = lambda x: x ** 2 - x ** 3 / (3 * dlast)
    gp = lambda x: 2 * x - x ** 2 / dlast
    nodes = f(D)[:, None] * g(dl)[None, :]
    s = oracle_mod.Spline(nodes, Dmax)
    rng = np.random.default_rng(4)
    x = rng.uniform(0, Dmax, 500)
    y = rng.uniform(0, dlast, 500)
    p, pD, pd = s.eval(x, y)
    scale = np.max(np.abs(nodes))
    assert np.max(np.abs(p - f(x) * g(y))) < 1e-12 * scale
    assert np.max(np.abs(pD - fp(x) * g(y))) < 1e-11 * scale
    assert np.max(np.abs(pd - f(x) * gp(y))) < 1e-10 * scale


def test_spline_matches_library_1d_splines(oracle_mod):
    """Along node lines the tensor spline is the 1-D cubic spline with the same end
    conditions; off the lines it is the composition of the two 1-D interpolations.
    scipy's CubicSpline with bc_type ((1, 0), (2, 0)) is the independent reference."""
    sp = pytest.importorskip("scipy.interpolate")
    rng = np.random.default_rng(9)
    D, dl = _grid(30, 30.0, 16)
    nodes = rng.normal(size=(len(D), len(dl)))
    s = oracle_mod.Spline(nodes, D[-1])
    bc = ((1, 0.0), (2, 0.0))
    # composition: spline along delta for each D row at y, then along D at x
    for _ in range(40):
        x = rng.uniform(0, D[-1])
        y = rng.uniform(0, dl[-1])
        col = np.array([sp.CubicSpline(dl, nodes[k], bc_type=bc)(y) for k in range(len(D))])
        ref = sp.CubicSpline(D, col, bc_type=bc)(x)
        got = s.eval([x], [y])[0][0]
        assert abs(got - ref) < 1e-12 * np.max(np.abs(nodes))


def test_kernel_branches(oracle_mod, oracle_spline):
    """D > 30 takes eq. (17) with its analytic d1-derivative; below, the spline; a
    delta above the last node is clamped (and counted) with zero delta-slope."""
    s = oracle_spline
    C = oracle_mod.C_ASYM
    r, qi, qj = 12.0, 3.1, 2.7         # D = 34.8
    p, rd, ncl = s.kernel([r], [qi], [qj])
    d1, d2 = qi * r, qj * r
    pa = -C / (d1 ** 2 * d2 ** 2 * (d1 ** 2 + d2 ** 2))
    assert abs(p[0] - pa) < 1e-15 * abs(pa) and ncl == 0
    h = 1e-6 * d1
    dp = (oracle_mod.phi_asym(d1 + h, d2) - oracle_mod.phi_asym(d1 - h, d2)) / (2 * h)
    assert abs(rd[0] - r * dp) < 1e-7 * abs(r * dp)
    # inside the table: r dphi/dd1 from a central difference of the spline kernel in q_i
    r, qi, qj = 2.0, 1.3, 0.9
    p0, rd0, _ = s.kernel([r], [qi], [qj])
    e = 1e-6
    pp, _, _ = s.kernel([r], [qi + e], [qj])
    pm, _, _ = s.kernel([r], [qi - e], [qj])
    # d phi / d q_i = r dphi/dd1  (d1 = q_i r)
    assert abs((pp[0] - pm[0]) / (2 * e) - rd0[0]) < 1e-7
    # clamping: delta = (8 - 0.01)/(8 + 0.01) > 0.995 with D = 0.5 * 0.5 * 8.01 < 30
    _, _, ncl = s.kernel([0.5], [8.0], [0.01])
    assert ncl == 1
