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


def _rho_reference(oracle_mod, s):
    """rho(delta): scipy cubic spline (zero slope at 0, zero curvature at the end) through
    the last table row divided by eq. (17) at D = Dmax, at the delta nodes."""
    sp = pytest.importorskip("scipy.interpolate")
    dl = np.arange(s.nd) * s.hd
    ratio = s.f[-1] / oracle_mod.phi_asym(s.Dmax * (1 + dl), s.Dmax * (1 - dl))
    return sp.CubicSpline(dl, ratio, bc_type=((1, 0.0), (2, 0.0)))


def _far_factor(oracle_mod, s, rho, d1, d2):
    """The factor g that multiplies eq. (17) past the table, from its reading:
    rho at delta* = max(0, 1 - min(d1, d2)/Dmax), the delta at which the last
    table row has the same smaller argument, plus (1 - rho(0)) (1 - (Dmax/D)^2)."""
    D = 0.5 * (d1 + d2)
    dstar = max(0.0, 1.0 - min(d1, d2) / s.Dmax)
    dlast = (s.nd - 1) * s.hd
    if dstar > dlast:  # linear continuation past the last node
        val = rho(dlast) + rho(dlast, 1) * (dstar - dlast)
    else:
        val = rho(dstar)
    return val + (1.0 - rho(0.0)) * (1.0 - (s.Dmax / D) ** 2)


# (r, q_i, q_j) past the table: delta* clamped at 0 (both arguments above Dmax);
# delta* > 0 with d1 the smaller argument, then d2; delta* past the last node
FAR_PAIRS = [(12.0, 3.1, 2.7), (10.0, 0.3, 6.0), (10.0, 6.0, 0.3), (5.0, 0.02, 12.1)]


def test_kernel_branches(oracle_mod, oracle_spline):
    """D > Dmax takes eq. (17) times g (see _far_factor) with the analytic
    d1-derivative; below, the spline; a delta above the last node is counted."""
    s = oracle_spline
    rho = _rho_reference(oracle_mod, s)
    e = 1e-6
    for r, qi, qj in FAR_PAIRS:
        assert 0.5 * r * (qi + qj) > s.Dmax
        p, rd, ncl = s.kernel([r], [qi], [qj])
        d1, d2 = qi * r, qj * r
        pa = _far_factor(oracle_mod, s, rho, d1, d2) * oracle_mod.phi_asym(d1, d2)
        assert abs(p[0] - pa) < 1e-12 * abs(pa), (r, qi, qj, p[0], pa)
        # r dphi/dd1 by a central difference in q_i (d1 = q_i r moves, d2 fixed)
        h = e * qi
        pp, _, _ = s.kernel([r], [qi + h], [qj])
        pm, _, _ = s.kernel([r], [qi - h], [qj])
        fd = (pp[0] - pm[0]) / (2 * h)   # dphi/dq_i = r dphi/dd1
        assert abs(fd - rd[0]) < 1e-6 * abs(rd[0]), (r, qi, qj, fd, rd[0])
    # inside the table: the same check
    r, qi, qj = 2.0, 1.3, 0.9
    p0, rd0, _ = s.kernel([r], [qi], [qj])
    pp, _, _ = s.kernel([r], [qi + e], [qj])
    pm, _, _ = s.kernel([r], [qi - e], [qj])
    assert abs((pp[0] - pm[0]) / (2 * e) - rd0[0]) < 1e-7
    # clamping: delta = (8 - 0.01)/(8 + 0.01) > 0.995 with D = 0.5 * 0.5 * 8.01 < 30
    _, _, ncl = s.kernel([0.5], [8.0], [0.01])
    assert ncl == 1


@pytest.mark.parametrize("dl", [0.0, 0.8, 0.9, 0.94])
def test_kernel_tends_to_eq17_at_large_D(oracle_mod, oracle_spline, dl):
    """Eq. (17) is the kernel's limit when both arguments are large (section 2: it
    is used "for large D"): at fixed delta the kernel as used, divided by eq. (17)
    written out here, tends to 1 as D grows, and is within 1e-5 of it at D = 1000."""
    s = oracle_spline
    C = 12.0 * (4.0 * np.pi / 9.0) ** 3
    dev = []
    for D in (100.0, 300.0, 1000.0):
        qi, qj = 1.0 + dl, 1.0 - dl
        r = D                                   # D = r (q_i + q_j) / 2
        d1, d2 = qi * r, qj * r
        p17 = -C / (d1 ** 2 * d2 ** 2 * (d1 ** 2 + d2 ** 2))
        p, _, _ = s.kernel([r], [qi], [qj])
        dev.append(abs(p[0] / p17 - 1.0))
    assert dev[1] < dev[0] and dev[2] < dev[1], dev
    assert dev[2] < 1e-5, dev


@pytest.mark.parametrize("D", [60.0, 120.0])
def test_kernel_past_table_matches_quadrature(oracle_mod, oracle_spline, D):
    """Past the table the kernel as used agrees with direct quadrature of eq. (14)
    at large delta, where eq. (17) alone is off by up to 97 % (min(d1, d2) of a few
    bohr^-1 q): within 1 % for delta = 0.9, 0.95, 0.99 at D = 60 and 120."""
    s = oracle_spline
    for dl in (0.9, 0.95, 0.99):
        qi, qj = 1.0 + dl, 1.0 - dl
        r = D
        p, _, _ = s.kernel([r], [qi], [qj])
        pq = oracle_mod.phi([qi * r], [qj * r], oracle_mod.QUAD_REFERENCE)[0]
        assert abs(p[0] / pq - 1.0) < 1e-2, (D, dl, p[0], pq)


def test_kernel_continuous_at_table_edge(oracle_mod, oracle_spline):
    """phi is continuous across D = Dmax: at the delta nodes exactly (rho interpolates
    the ratio there), in between up to the interpolation error; rho = 1 where eq. (17)
    is accurate (delta = 0; this table's quadrature is good to ~1e-11 absolute, i.e.
    5e-4 of phi(30, 0) = -2.2e-8)."""
    s = oracle_spline
    rho = _rho_reference(oracle_mod, s)
    assert abs(rho(0.0) - 1.0) < 2e-3
    for dl in list(np.arange(0, 199, 13) / 200.0) + [0.2537, 0.61, 0.9033]:
        q = 1.7
        qi, qj = q * (1 + dl), q * (1 - dl)
        r_edge = 2 * s.Dmax / (qi + qj)
        inside, _, _ = s.kernel([r_edge * (1 - 1e-12)], [qi], [qj])
        outside, _, _ = s.kernel([r_edge * (1 + 1e-12)], [qi], [qj])
        on_node = abs(dl * s.nd - round(dl * s.nd)) < 1e-9
        tol = 1e-9 if on_node else 1e-6
        assert abs(inside[0] - outside[0]) <= tol * abs(inside[0]), (dl, inside, outside)


@pytest.mark.parametrize("D", [2.0, 17.3, 29.99, 31.0, 45.0])
def test_kernel_continued_past_last_delta_node(oracle_mod, oracle_spline, D):
    """Above the last delta node the kernel is the spline's linear continuation (the
    spline has zero curvature there): value and delta-slope continuous across the node,
    and r dphi/dd1 of the continued kernel equals a central difference in q_i."""
    s = oracle_spline
    dlast = (s.nd - 1) * s.hd
    q = 2.0
    def at(dl, eps_q=0.0):
        qi, qj = q * (1 + dl), q * (1 - dl)
        r = 2 * D / (qi + qj)
        return s.kernel([r], [qi + eps_q], [qj])
    # second differences across the node: O(e^2) if smooth, O(e) for a kink, O(1) for
    # a jump -- so the ratio of second difference to e^2 must not grow as e shrinks
    ratios = []
    for e in (1e-4, 1e-5):
        below, _, n0 = at(dlast - e)
        mid, _, _ = at(dlast)
        above, _, n1 = at(dlast + e)
        assert n0 == 0 and n1 == 1
        ratios.append(abs(above[0] - 2 * mid[0] + below[0]) / e ** 2)
    assert ratios[1] <= 2.0 * ratios[0] + 1e-6 * abs(mid[0])
    dl = 0.9985
    p0, rd, n2 = at(dl)
    assert n2 == 1
    h = 1e-6
    pp, _, _ = at(dl, h)
    pm, _, _ = at(dl, -h)
    assert abs((pp[0] - pm[0]) / (2 * h) - rd[0]) <= 1e-6 * abs(rd[0])
