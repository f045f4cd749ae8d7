"""Pins of the oracle's kernel phi (Dion eq. 14, eq. 17) against facts that the
mathematics fixes, independent of the oracle's own code path."""
import numpy as np
import pytest

from conftest import golden_dict


def test_W_matches_printed_formula_high_precision(oracle_mod):
    """The oracle evaluates W from a factored form; compare it with the formula
    as printed by Dion (eq. 14), evaluated at 50 digits, over small and large
    arguments (the printed form cancels badly at small a, b in FP64)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50

    def W_printed(a, b):
        a = mp.mpf(a)
        b = mp.mpf(b)
        num = ((3 - a ** 2) * b * mp.cos(b) * mp.sin(a) + (3 - b ** 2) * a * mp.cos(a) * mp.sin(b)
               + (a ** 2 + b ** 2 - 3) * mp.sin(a) * mp.sin(b) - 3 * a * b * mp.cos(a) * mp.cos(b))
        return 2 * num / (a ** 3 * b ** 3)

    rng = np.random.default_rng(7)
    pts = list(zip(10 ** rng.uniform(-4, 2, 60), 10 ** rng.uniform(-4, 2, 60)))
    pts += [(1e-3, 1e-3), (0.2, 0.26), (0.25, 0.25), (30.0, 1e-2), (80.0, 79.5)]
    for a, b in pts:
        ref = float(W_printed(a, b))
        got = float(oracle_mod.W(a, b)[0])
        assert abs(got - ref) <= 1e-13 * max(1.0, abs(ref)), (a, b, got, ref)
    # W(0, 0) = 2/3 is what sets the small-D logarithm below
    assert abs(float(oracle_mod.W(1e-6, 1e-6)[0]) - 2.0 / 3.0) < 1e-12


def test_phi_symmetric_in_arguments(oracle_mod):
    """phi(d1, d2) = phi(d2, d1): the kernel is symmetric in r, r' (eq. 1)."""
    rng = np.random.default_rng(11)
    d1 = rng.uniform(0.05, 25.0, 40)
    d2 = rng.uniform(0.05, 25.0, 40)
    q = oracle_mod.QUAD_TABLE
    a = oracle_mod.phi(d1, d2, q)
    b = oracle_mod.phi(d2, d1, q)
    assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(a))


def test_phi_zero_integral(oracle_mod):
    """int_0^inf 4 pi D^2 phi(D, 0) dD = 0 (vdW-DF has no nonlocal correlation for a
    uniform density).  [0, 30] by composite Gauss-Legendre, [30, inf) from eq. (17):
    int_30^inf 4 pi D^2 (-C / (2 D^6)) dD = -2 pi C / (3 * 30^3)."""
    g = golden_dict("dion_kernel.txt")
    x, w = np.polynomial.legendre.leggauss(12)
    edges = [0, 1e-4, 1e-3, 1e-2, 0.05, 0.1, 0.25, 0.5, 0.75, 1.0] + list(np.arange(1.5, 30.01, 0.5))
    D, Wt = [], []
    for lo, hi in zip(edges[:-1], edges[1:]):
        D += list(0.5 * (lo + hi) + 0.5 * (hi - lo) * x)
        Wt += list(0.5 * (hi - lo) * w)
    D = np.array(D)
    Wt = np.array(Wt)
    f = 4 * np.pi * D ** 2 * oracle_mod.phi(D, D, oracle_mod.QUAD_REFERENCE)
    tail = -2 * np.pi * g["C_asym"] / (3 * 30.0 ** 3)
    total = np.sum(Wt * f) + tail
    scale = np.sum(Wt * np.abs(f))
    assert abs(total - g["zero_integral"]) <= 1e-9 * scale, (total, scale)


@pytest.mark.parametrize("dl", [0.0, 0.3, 0.6])
def test_phi_large_D_asymptote(oracle_mod, dl):
    """phi -> -C/(d1^2 d2^2 (d1^2 + d2^2)), C = 12 (4 pi/9)^3 (Dion eq. 17): the
    relative deviation falls steadily with D and is small by D = 30."""
    g = golden_dict("dion_kernel.txt")
    assert abs(g["C_asym"] - 12 * (4 * np.pi / 9) ** 3) < 1e-12
    D = np.array([10.0, 15.0, 20.0, 25.0, 30.0])
    p = oracle_mod.phi(D * (1 + dl), D * (1 - dl), oracle_mod.QUAD_REFERENCE)
    d1, d2 = D * (1 + dl), D * (1 - dl)
    pa = -g["C_asym"] / (d1 ** 2 * d2 ** 2 * (d1 ** 2 + d2 ** 2))
    rel = np.abs(p / pa - 1)
    # decreasing until quadrature noise (absolute ~1e-16 against phi ~ 1e-8)
    assert rel[1] < rel[0] and rel[2] < rel[1]
    assert rel[-1] < {0.0: 1e-7, 0.3: 1e-7, 0.6: 1e-5}[dl]
    assert np.all(p < 0)


def test_phi_small_D_logarithm(oracle_mod):
    """phi(D, 0) = -(2/pi) ln D + c + O(D): the remainder converges."""
    g = golden_dict("dion_kernel.txt")
    D = np.array([1e-2, 1e-3, 1e-4])
    p = oracle_mod.phi(D, D, oracle_mod.QUAD_REFERENCE)
    c = p + g["small_D_log_coef"] * np.log(D)
    d1, d2 = abs(c[0] - c[1]), abs(c[1] - c[2])
    assert d2 < 1e-3
    assert 3.0 < d1 / d2 < 30.0      # O(D) remainder: steps shrink ~10x


def test_quadrature_converged(oracle_mod):
    """Reference quadrature vs a finer one (wider range, more points)."""
    rng = np.random.default_rng(5)
    D = rng.uniform(0.05, 30, 12)
    dl = rng.uniform(0, 0.99, 12)
    fine = dict(a_min=3e-8, log_ratio=1.4, n_log=10, m_half=320, n_osc=12)
    a = oracle_mod.phi(D * (1 + dl), D * (1 - dl), oracle_mod.QUAD_REFERENCE)
    b = oracle_mod.phi(D * (1 + dl), D * (1 - dl), fine)
    assert np.max(np.abs(a - b)) < 1e-10


def test_table_row0_rule_and_layout(oracle_mod):
    """Node table layout (D outer, delta inner) and the D = 0 row rule."""
    q = oracle_mod.QUAD_FAST
    t = oracle_mod.phi_table(6, 1.0, 4, q)
    D = 1.0 * np.arange(6) / 5
    for k in (1, 3, 5):
        for l in (0, 2, 3):
            dl = l / 4
            ref = oracle_mod.phi([D[k] * (1 + dl)], [D[k] * (1 - dl)], q)[0]
            assert abs(t[k, l] - ref) < 1e-14 * max(1, abs(ref))
    assert np.allclose(t[0], (4 * t[1] - t[2]) / 3, rtol=1e-15, atol=0)
