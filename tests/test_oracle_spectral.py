"""Pins of the oracle's spectral (FFT) gradient, the paper's FFTW gradient option
(section 3): closed-form derivatives of band-limited fields on orthorhombic and
skewed cells, the Nyquist convention, the textbook circulant form of the same
operator, its adjoint, spectral accuracy on a smooth field, and the potential
as the derivative of E with this gradient."""
import numpy as np
import pytest


def _skewed_cell():
    return np.array([[9.0, 0.0, 0.0], [4.5, 7.794228634059948, 0.0], [0.7, -0.4, 11.0]])


@pytest.mark.parametrize("shape", [(12, 10, 14), (9, 11, 8)])
@pytest.mark.parametrize("skew", [False, True])
def test_plane_waves_exact(oracle_mod, shape, skew):
    """f = sum_G a_G cos(G.r + p_G) over reciprocal lattice vectors G = 2 pi sum m_a B_a
    with |m_a| < N_a/2 has grad f = -sum a_G G sin(G.r + p_G) exactly."""
    cell = _skewed_cell() if skew else np.diag([9.0, 8.0, 11.0])
    B = np.linalg.inv(cell).T
    idx = np.stack(np.meshgrid(*[np.arange(n) for n in shape], indexing="ij"), axis=-1)
    r = (idx / np.array(shape, float)) @ cell          # r = sum_a u_a M_a
    rng = np.random.default_rng(11)
    f = np.zeros(shape)
    g = np.zeros((3,) + shape)
    for _ in range(6):
        m = np.array([rng.integers(-((n - 1) // 2), (n - 1) // 2 + 1) for n in shape])
        G = 2 * np.pi * (m @ B)
        a, p = rng.normal(), rng.uniform(0, 2 * np.pi)
        ph = r @ G + p
        f += a * np.cos(ph)
        g -= a * G[:, None, None, None] * np.sin(ph)[None]
    got = oracle_mod.gradient_spectral(f, cell if skew else np.diag(cell))
    assert np.max(np.abs(got - g)) < 1e-11 * np.max(np.abs(g))


def test_nyquist_mode_has_no_derivative(oracle_mod):
    """On an even axis the alternating field (-1)^i is its own mirror frequency:
    its band-limited derivative at the grid points is zero."""
    shape = (10, 6, 8)
    f = np.broadcast_to(((-1.0) ** np.arange(10))[:, None, None], shape).copy()
    g = oracle_mod.gradient_spectral(f, (5.0, 3.0, 4.0))
    assert np.max(np.abs(g)) < 1e-12


@pytest.mark.parametrize("N", [8, 9, 16, 15])
def test_circulant_form(oracle_mod, N):
    """Along one axis the operator is the circulant matrix of the periodic sinc
    interpolant: D[l, k] = c_(l-k) with c_j = pi (-1)^j cot(pi j / N) for even N
    and pi (-1)^j / sin(pi j / N) for odd N (d/du, period 1; c_0 = 0)."""
    j = np.arange(1, N)
    c = np.zeros(N)
    c[1:] = np.pi * (-1.0) ** j / (np.tan(np.pi * j / N) if N % 2 == 0 else np.sin(np.pi * j / N))
    D = np.array([[c[(l - k) % N] for k in range(N)] for l in range(N)])
    rng = np.random.default_rng(N)
    f = rng.normal(size=(N, 3, 4))
    L = 6.0
    got = oracle_mod.gradient_spectral(f, (L, 3.0, 4.0))[0]
    ref = np.einsum("lk,kab->lab", D, f) / L
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("skew", [False, True])
def test_adjoint_identity(oracle_mod, skew):
    """<grad u, w> = <u, D^T w> with D^T from its own (conjugate-multiplier) formula,
    and D^T = -div of the same operator (the multipliers are purely imaginary)."""
    shape = (10, 9, 12)
    geom = _skewed_cell() if skew else (7.0, 6.0, 9.0)
    rng = np.random.default_rng(5)
    u = rng.normal(size=shape)
    w = rng.normal(size=(3,) + shape)
    lhs = np.sum(oracle_mod.gradient_spectral(u, geom) * w)
    rhs = np.sum(u * oracle_mod.gradient_spectral_T(w, geom))
    assert abs(lhs - rhs) < 1e-11 * np.sum(np.abs(u)) * np.max(np.abs(w))


def test_spectral_accuracy(oracle_mod):
    """A smooth periodic field that is not band-limited: the FFT gradient is exact
    to ~1e-10 on a 32-point axis where the 4th-order stencil errs by ~1e-4."""
    N, L = 32, 10.0
    u = np.arange(N) / N
    f1 = np.exp(np.cos(2 * np.pi * u))
    df1 = -2 * np.pi / L * np.sin(2 * np.pi * u) * f1
    f = np.broadcast_to(f1[:, None, None], (N, 4, 4)).copy()
    gs = oracle_mod.gradient_spectral(f, (L, 2.0, 2.0))[0, :, 0, 0]
    gf = oracle_mod.gradient(f, (L / N, 0.5, 0.5))[0, :, 0, 0]
    assert np.max(np.abs(gs - df1)) < 1e-10 * np.max(np.abs(df1))
    assert np.max(np.abs(gf - df1)) > 1e-5 * np.max(np.abs(df1))


def test_potential_is_derivative_with_spectral_gradient(oracle_mod, oracle_spline):
    """v from the spectral adjoint equals central differences of E computed with
    the spectral gradient, at points where the trimming mask does not move."""
    from paper_0810_2273_gb300 import inputs
    w = inputs.kr_dimer((12, 10, 10))
    n = w["density"]
    P = oracle_mod.Problem(n, w["lengths"], w["periodic"], w["n_cut"], w["r_cut"], oracle_spline,
                           gradient="spectral")
    e = P.energy()
    v = P.potential(e["A"], e["U"])
    rng = np.random.default_rng(2)
    flat = n.ravel()
    cand = np.nonzero(flat > 4 * w["n_cut"])[0]
    for m in rng.choice(cand, 5, replace=False):
        h = 1e-4 * flat[m]
        Es = []
        for sgn in (1, -1):
            nn = flat.copy()
            nn[m] += sgn * h
            Es.append(oracle_mod.Problem(nn.reshape(n.shape), w["lengths"], w["periodic"], w["n_cut"],
                                         w["r_cut"], oracle_spline, gradient="spectral").energy()["E"])
        fd = (Es[0] - Es[1]) / (2 * h * P.dV)
        assert abs(fd - v.ravel()[m]) < 1e-6 * np.max(np.abs(v)) + 1e-7 * abs(fd), (m, fd, v.ravel()[m])
