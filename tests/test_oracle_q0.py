"""Pins of the oracle's q0 (Dion eqs. 11-12 with PW92 LDA correlation) and of
its 4th-order periodic finite-difference gradient (paper section 3)."""
import numpy as np

from conftest import golden_dict, read_golden


def _rs(n):
    return (3.0 / (4.0 * np.pi * n)) ** (1.0 / 3.0)


def test_lda_correlation_against_uniform_gas_energies(oracle_mod):
    rows = [r for r in read_golden("lda_correlation.txt") if len(r) == 2 and r[0][0].isdigit()]
    rs = np.array([float(r[0]) for r in rows])
    ref = np.array([float(r[1]) for r in rows])
    e, _ = oracle_mod.eps_c(rs)
    assert np.max(np.abs(e - ref)) < 3e-4


def test_lda_correlation_high_density_limit(oracle_mod):
    c0 = golden_dict("lda_correlation.txt")["c0"]
    e, _ = oracle_mod.eps_c(np.array([1e-10, 1e-11]))
    slope = (e[0] - e[1]) / np.log(10.0)
    assert abs(slope - c0) < 2e-5 * c0


def test_lda_correlation_high_density_constant(oracle_mod):
    """eps_c - c0 ln rs -> -c1 as rs -> 0, with the slope c0 measured between
    rs = 1e-11 and 1e-10 (where the next terms are ~1e-7)."""
    g = golden_dict("lda_correlation.txt")
    e, _ = oracle_mod.eps_c(np.array([1e-10, 1e-11]))
    slope = (e[0] - e[1]) / np.log(10.0)
    assert abs((e[0] - slope * np.log(1e-10)) + g["c1"]) < 2e-6


def test_lda_correlation_derivative(oracle_mod):
    rs = np.array([0.3, 1.0, 4.0, 30.0, 300.0])
    h = 1e-6 * rs
    e, de = oracle_mod.eps_c(rs)
    ep, _ = oracle_mod.eps_c(rs + h)
    em, _ = oracle_mod.eps_c(rs - h)
    assert np.max(np.abs((ep - em) / (2 * h) - de) / np.abs(de)) < 1e-7


def test_q0_hand_values(oracle_mod):
    """n = 1/(3 pi^2) gives k_F = 1: without gradient q0 = 1 - (4 pi/3) eps_c; with
    |grad n| = 2 s n the gradient term adds -(Zab/9) k_F s^2 = 0.8491 s^2 / 9
    (s = 1, 2 and 1/2, so that the power of s shows)."""
    g = golden_dict("dion_kernel.txt")
    n0 = 1.0 / (3.0 * np.pi ** 2)
    svals = (1.0, 2.0, 0.5)
    n = np.full((1, 1, 1 + len(svals)), n0)
    grad = np.zeros((3, 1, 1, 1 + len(svals)))
    for k, sv in enumerate(svals):
        grad[(k % 3), 0, 0, 1 + k] = 2.0 * sv * n0
    q, _, _ = oracle_mod.q0(n, grad)
    ec, _ = oracle_mod.eps_c(np.array([_rs(n0)]))
    assert abs(q[0, 0, 0] - (1.0 - 4.0 * np.pi / 3.0 * ec[0])) < 1e-14
    for k, sv in enumerate(svals):
        assert abs((q[0, 0, 1 + k] - q[0, 0, 0]) - (-g["Zab"] / 9.0) * sv ** 2) < 1e-14


def test_q0_partials_against_finite_differences(oracle_mod):
    rng = np.random.default_rng(21)
    N = 40
    n = 10 ** rng.uniform(-5, 1, N).reshape(1, 1, N)
    grad = rng.normal(size=(3, 1, 1, N)) * n[None] * rng.uniform(0.1, 5, N)
    q, qn, qg = oracle_mod.q0(n, grad)
    h = 1e-6 * n
    qp, _, _ = oracle_mod.q0(n + h, grad)
    qm, _, _ = oracle_mod.q0(n - h, grad)
    fd = (qp - qm) / (2 * h)
    assert np.max(np.abs(fd - qn) / (np.abs(qn) + np.abs(q) / n)) < 1e-7
    for ax in range(3):
        hg = 1e-3 * (np.abs(grad[ax]) + n)   # q0 is quadratic in grad n: no truncation error
        gp = grad.copy()
        gp[ax] += hg
        gm = grad.copy()
        gm[ax] -= hg
        fd = (oracle_mod.q0(n, gp)[0] - oracle_mod.q0(n, gm)[0]) / (2 * hg)
        assert np.max(np.abs(fd - qg[ax]) / (np.abs(qg[ax]) + 1e-12)) < 1e-6


def test_gradient_fourier_symbol(oracle_mod):
    """On the periodic grid the stencil maps sin(theta m) to
    (8 sin theta - sin 2 theta)/(6 h) cos(theta m), exactly (its Fourier symbol)."""
    n0, n1, n2 = 20, 12, 16
    h = (0.7, 0.45, 0.3)
    for ax, nn in enumerate((n0, n1, n2)):
        for k in (1, 2, 5):
            th = 2 * np.pi * k / nn
            m = np.arange(nn)
            shape = [1, 1, 1]
            shape[ax] = nn
            f = np.broadcast_to(np.sin(th * m + 0.3).reshape(shape), (n0, n1, n2))
            g = oracle_mod.gradient(f, h)
            sym = (8 * np.sin(th) - np.sin(2 * th)) / (6 * h[ax])
            ref = np.broadcast_to((sym * np.cos(th * m + 0.3)).reshape(shape), (n0, n1, n2))
            assert np.max(np.abs(g[ax] - ref)) < 1e-12
            for other in range(3):
                if other != ax:
                    assert np.max(np.abs(g[other])) < 1e-12


def test_gradient_adjoint_identity(oracle_mod):
    """<D u, w> = <u, D^T w> and D^T = -D (central differences are antisymmetric)."""
    rng = np.random.default_rng(2)
    shape = (9, 7, 11)
    h = (0.5, 0.31, 0.77)
    u = rng.normal(size=shape)
    w = rng.normal(size=(3,) + shape)
    lhs = np.sum(oracle_mod.gradient(u, h) * w)
    rhs = np.sum(u * oracle_mod.gradient_T(w, h))
    assert abs(lhs - rhs) < 1e-12 * np.sum(np.abs(u)) * np.max(np.abs(w))
    gw = sum(oracle_mod.gradient(w[ax], h)[ax] for ax in range(3))
    assert np.max(np.abs(oracle_mod.gradient_T(w, h) + gw)) < 1e-12
