"""Pins of the oracle on general (non-orthogonal) cells: the pair sum, the
gradient along skewed grid axes and its transpose, checked against properties
that hold for any correct implementation."""
import numpy as np
import pytest

HEX = np.array([[9.0, 0.0, 0.0], [4.5, 7.794228634059948, 0.0], [0.0, 0.0, 8.0]])  # 60 degrees


def _smooth(cell, dims, seed=0, n0=0.02):
    """A positive periodic density sum_k A_k cos(2 pi m_k . u + p_k) + n0 on the grid of
    the cell, with its exact Cartesian gradient (m_k integer, u fractional)."""
    rng = np.random.default_rng(seed)
    u = np.meshgrid(*[np.arange(d) / d for d in dims], indexing="ij")
    B = np.linalg.inv(cell).T
    n = np.full(dims, n0)
    g = np.zeros((3,) + tuple(dims))
    for _ in range(4):
        m = rng.integers(-2, 3, size=3)
        A = rng.uniform(0.001, 0.004)
        p = rng.uniform(0, 2 * np.pi)
        ph = 2 * np.pi * (m[0] * u[0] + m[1] * u[1] + m[2] * u[2]) + p
        n += A * np.cos(ph)
        G = 2 * np.pi * (m[0] * B[0] + m[1] * B[1] + m[2] * B[2])   # Cartesian wave vector
        for c in range(3):
            g[c] -= A * np.sin(ph) * G[c]
    return n, g


def test_diagonal_cell_equals_orthorhombic(oracle_mod, oracle_spline):
    rng = np.random.default_rng(1)
    L = (5.0, 6.0, 4.0)
    n = 10 ** rng.uniform(-3, -0.5, size=(8, 9, 7))
    a = oracle_mod.Problem(n, L, (1, 1, 0), 1e-3, 5.0, oracle_spline)
    b = oracle_mod.Problem(n, None, (1, 1, 0), 1e-3, 5.0, oracle_spline, cell=np.diag(L))
    ea, eb = a.energy(), b.energy()
    assert ea["pairs"] == eb["pairs"]
    assert abs(ea["E"] - eb["E"]) <= 1e-13 * abs(ea["E"])
    assert np.max(np.abs(ea["U"] - eb["U"])) <= 1e-12 * np.max(np.abs(ea["U"]))
    va, vb = a.potential(ea["A"], ea["U"]), b.potential(eb["A"], eb["U"])
    assert np.max(np.abs(va - vb)) <= 1e-12 * np.max(np.abs(va))


@pytest.mark.parametrize("ms", [(1, 0, 0), (2, -1, 0), (1, 2, 1), (0, 3, -2)])
def test_gradient_cell_fourier_symbol(oracle_mod, ms):
    """f = cos(2 pi m . u): the stencil along axis a gives df/du_a times the
    known symbol (8 sin t - sin 2t)/(6 t), t = 2 pi m_a / N_a; the Cartesian
    gradient is sum_a (df/du_a) B_a."""
    dims = (12, 10, 9)
    u = np.meshgrid(*[np.arange(d) / d for d in dims], indexing="ij")
    ph = 2 * np.pi * sum(m * uu for m, uu in zip(ms, u))
    f = np.cos(ph)
    B = np.linalg.inv(HEX).T
    ref = np.zeros((3,) + dims)
    for a in range(3):
        t = 2 * np.pi * ms[a] / dims[a]
        sym = (8 * np.sin(t) - np.sin(2 * t)) / (6 * t) if ms[a] else 0.0
        dfu = -2 * np.pi * ms[a] * np.sin(ph) * sym
        for c in range(3):
            ref[c] += dfu * B[a, c]
    g = oracle_mod.gradient_cell(f, HEX)
    assert np.max(np.abs(g - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_gradient_cell_adjoint_identity(oracle_mod):
    rng = np.random.default_rng(2)
    dims = (7, 8, 6)
    f = rng.normal(size=dims)
    w = rng.normal(size=(3,) + dims)
    lhs = np.sum(oracle_mod.gradient_cell(f, HEX) * w)
    rhs = np.sum(f * oracle_mod.gradient_T_cell(w, HEX))
    assert abs(lhs - rhs) <= 1e-12 * np.sum(np.abs(f)) * np.max(np.abs(w)) * 10


def test_lattice_basis_invariance(oracle_mod, oracle_spline):
    """The same periodic density on the same points, described with the basis
    (a, b, c) and with (a, a + b, c) (N_0 = N_1): point (i', j', k) of the second
    is point ((i' + j') mod N, j', k) of the first.  With the same Cartesian
    gradient both must give the same E and pair count."""
    dims = (10, 10, 8)
    n, g = _smooth(HEX, dims, seed=3)
    cell2 = HEX.copy()
    cell2[1] = HEX[0] + HEX[1]
    i = np.arange(dims[0])[:, None]
    j = np.arange(dims[1])[None, :]
    src = (i + j) % dims[0]
    n2 = n[src, j, :]
    g2 = g[:, src, j, :]
    a = oracle_mod.Problem(n, None, (1, 1, 0), 1e-3, 7.0, oracle_spline, cell=HEX, g=g).energy()
    b = oracle_mod.Problem(n2, None, (1, 1, 0), 1e-3, 7.0, oracle_spline, cell=cell2, g=g2).energy()
    assert a["pairs"] == b["pairs"] > 0
    assert abs(a["E"] - b["E"]) <= 1e-12 * abs(a["E"])


def test_rotation_invariance(oracle_mod, oracle_spline):
    dims = (9, 9, 6)
    n, g = _smooth(HEX, dims, seed=4)
    th = 0.7
    R = np.array([[np.cos(th), -np.sin(th), 0.2], [np.sin(th), np.cos(th), 0.0], [0.0, 0.0, 1.0]])
    R, _ = np.linalg.qr(R)
    cellR = HEX @ R.T
    gR = np.einsum("ck,k...->c...", R, g)
    a = oracle_mod.Problem(n, None, (1, 1, 0), 1e-3, 6.5, oracle_spline, cell=HEX, g=g).energy()
    b = oracle_mod.Problem(n, None, (1, 1, 0), 1e-3, 6.5, oracle_spline, cell=cellR, g=gR).energy()
    assert a["pairs"] == b["pairs"]
    assert abs(a["E"] - b["E"]) <= 1e-12 * abs(a["E"])


def test_skewed_pair_counts_brute_force(oracle_mod, oracle_spline):
    """Ordered pairs within rc (self term excluded) by brute force over a
    generous image range, against the oracle's bounded image loops."""
    rng = np.random.default_rng(5)
    dims = (6, 5, 4)
    cell = np.array([[4.0, 0.0, 0.0], [3.2, 2.1, 0.0], [0.3, -0.4, 3.5]])   # strongly skewed
    n = 10 ** rng.uniform(-2, -0.5, size=dims)
    rc = 6.3
    P = oracle_mod.Problem(n, None, (1, 1, 1), 1e-3, rc, oracle_spline, cell=cell)
    e = P.energy()
    idx = np.stack(np.unravel_index(P.active, dims), axis=1) / np.array(dims)
    pos = idx @ cell
    K = 8
    rng_m = np.arange(-K, K + 1)
    L = np.array(np.meshgrid(rng_m, rng_m, rng_m, indexing="ij")).reshape(3, -1).T @ cell
    cnt = 0
    for a in range(len(pos)):
        d = pos[a] - pos[:, None, :] + L[None, :, :]
        r2 = (d ** 2).sum(-1)
        cnt += int(np.count_nonzero(r2 <= rc * rc * (1 + 1e-12))) - 1
    assert e["pairs"] == cnt


def test_skewed_potential_is_derivative_of_energy(oracle_mod, oracle_spline):
    """v = dE/dn / dV on a skewed periodic cell, against central differences of the
    FP64 E, through the skewed stencil and its transpose."""
    rng = np.random.default_rng(6)
    dims = (8, 8, 6)
    cell = np.array([[6.0, 0.0, 0.0], [3.0, 5.196152422706632, 0.0], [0.0, 0.0, 5.0]])
    n, _ = _smooth(cell, dims, seed=7, n0=0.03)
    P = oracle_mod.Problem(n, None, (1, 1, 1), 1e-4, 5.5, oracle_spline, cell=cell)
    e = P.energy()
    v = P.potential(e["A"], e["U"])
    vmax = np.max(np.abs(v))
    for m in rng.choice(n.size, 4, replace=False):
        h = 1e-4 * n.flat[m]
        npl, nmi = n.copy(), n.copy()
        npl.flat[m] += h
        nmi.flat[m] -= h
        Ep = oracle_mod.Problem(npl, None, (1, 1, 1), 1e-4, 5.5, oracle_spline, cell=cell).energy()["E"]
        Em = oracle_mod.Problem(nmi, None, (1, 1, 1), 1e-4, 5.5, oracle_spline, cell=cell).energy()["E"]
        fd = (Ep - Em) / (2 * h * P.dV)
        assert abs(fd - v.flat[m]) <= 1e-6 * vmax, (m, fd, v.flat[m])
    # and potential_at agrees with the whole-grid potential
    pts = rng.choice(n.size, 5, replace=False)
    assert np.max(np.abs(P.potential_at(pts) - v.ravel()[pts])) <= 1e-12 * vmax
