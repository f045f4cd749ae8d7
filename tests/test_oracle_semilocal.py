"""Pins of the oracle's semilocal energies (eq. 3 terms: LDA, PBE and revPBE
exchange, PW92 and PBE correlation), each against a property the definitions fix:
exact uniform scaling of exchange, the uniform-gas limit, and the analytic limits
of the PBE enhancement factor and gradient correction."""
import numpy as np
import pytest

from conftest import read_golden

BETA = 0.06672455060314922


def _blobs(shape, lengths, seed=0):
    """A smooth positive periodic density: a few Gaussians plus a floor."""
    rng = np.random.default_rng(seed)
    ax = [np.arange(d) * L / d for d, L in zip(shape, lengths)]
    X = np.meshgrid(*ax, indexing="ij")
    n = np.full(shape, 1e-4)
    for _ in range(3):
        c = rng.uniform(0, 1, 3) * np.array(lengths)
        a = rng.uniform(0.8, 1.5)
        r2 = sum(np.minimum(np.abs(X[k] - c[k]), lengths[k] - np.abs(X[k] - c[k])) ** 2 for k in range(3))
        n += rng.uniform(0.05, 0.3) * np.exp(-r2 / a ** 2)
    return n


@pytest.mark.parametrize("lam", [0.5, 2.0, 3.0])
def test_exchange_uniform_scaling(oracle_mod, lam):
    """n_lam(r) = lam^3 n(lam r) gives E_x[n_lam] = lam E_x[n] for LDA and both GGAs
    (s is scale invariant).  On the grid the scaled density is the same array
    times lam^3 on a cell shrunk by lam, and the 4th-order gradient scales by
    lam^4 exactly, so the identity holds to rounding."""
    L = (7.0, 8.0, 9.0)
    n = _blobs((14, 16, 18), L)
    e1 = oracle_mod.semilocal(n, L)
    el = oracle_mod.semilocal(lam ** 3 * n, tuple(x / lam for x in L))
    for k in ("Ex_lda", "Ex_pbe", "Ex_revpbe"):
        assert abs(el[k] - lam * e1[k]) <= 1e-12 * abs(lam * e1[k]), k
    # correlation is not scale-linear (a wrong power in it would show here)
    assert abs(el["Ec_lda"] - lam * e1["Ec_lda"]) > 1e-3 * abs(e1["Ec_lda"])


def test_uniform_gas(oracle_mod):
    """grad n = 0: the GGAs reduce to LDA; E_x^LDA = -(3/4)(3/pi)^(1/3) n^(4/3) V;
    E_c^LDA = N eps_c(rs) with the uniform-gas correlation energies tabulated by
    Perdew and Wang (golden file, their quoted accuracy)."""
    rows = [r for r in read_golden("lda_correlation.txt") if len(r) == 2 and r[0][0].isdigit()]
    for rs, ec_ref in ((float(a), float(b)) for a, b in rows):
        n0 = 3.0 / (4.0 * np.pi * rs ** 3)
        L = (4.0, 5.0, 6.0)
        e = oracle_mod.semilocal(np.full((4, 5, 6), n0), L)
        V = L[0] * L[1] * L[2]
        assert e["n_points"] == 120
        assert abs(e["Ex_lda"] - (-0.75 * (3.0 / np.pi) ** (1.0 / 3.0) * n0 ** (4.0 / 3.0) * V)) <= 1e-13 * abs(e["Ex_lda"])
        assert e["Ex_pbe"] == pytest.approx(e["Ex_lda"], rel=1e-15)
        assert e["Ex_revpbe"] == pytest.approx(e["Ex_lda"], rel=1e-15)
        assert e["Ec_pbe"] == pytest.approx(e["Ec_lda"], rel=1e-15)
        assert abs(e["Ec_lda"] / (n0 * V) - ec_ref) < 3e-4


@pytest.mark.parametrize("kappa", [0.804, 1.245])
def test_enhancement_factor_limits(oracle_mod, kappa):
    """F_x(0) = 1; F_x = 1 + mu s^2 + O(s^4) with mu = beta pi^2/3 (the PBE choice
    that cancels the gradient term of correlation); F_x -> 1 + kappa as s -> inf
    (the Lieb-Oxford bound for PBE)."""
    mu = BETA * np.pi ** 2 / 3.0
    f = oracle_mod.fx([0.0, 1e-3, 1e-2, 1e8], kappa)
    assert f[0] == 1.0
    assert abs((f[1] - 1.0) / 1e-6 - mu) <= 1e-6 * mu + mu * mu / kappa * 1e-6 * 2
    assert abs((f[2] - 1.0) / 1e-4 - mu) <= 2 * mu * mu / kappa * 1e-4
    assert abs(f[3] - (1.0 + kappa)) <= 1e-12


def test_pbe_gradient_correction_limits(oracle_mod):
    """H(rs, 0) = 0; H = beta t^2 + O(t^4) (second-order gradient expansion of
    correlation); eps_c + H -> 0 as t -> inf (correlation vanishes for rapidly
    varying densities)."""
    rs = np.array([0.1, 1.0, 5.0, 30.0])
    assert np.all(oracle_mod.pbe_H(rs, 0.0) == 0.0)
    t = 1e-4
    h = oracle_mod.pbe_H(rs, t)
    assert np.all(np.abs(h / t ** 2 - BETA) <= 1e-4 * BETA)
    ec = np.array([oracle_mod.eps_c(np.array([r]))[0][0] for r in rs])
    hinf = oracle_mod.pbe_H(rs, 1e7)
    assert np.all(np.abs(ec + hinf) <= 1e-9 * np.abs(ec))


def test_pbe_correlation_high_density_scaling(oracle_mod):
    """Under uniform scaling to high density (lam -> inf) PBE correlation tends to a
    constant while LDA correlation diverges like -0.0311 N ln lam: the gradient
    correction must cancel the logarithm, which holds only with
    gamma = (1 - ln 2)/pi^2 matching the high-density coefficient of PW92."""
    L = (7.0, 8.0, 9.0)
    n = _blobs((14, 16, 18), L, seed=3)
    e = [oracle_mod.semilocal(lam ** 3 * n, tuple(x / lam for x in L)) for lam in (1e3, 1e4, 1e5)]
    d_lda = abs(e[2]["Ec_lda"] - e[1]["Ec_lda"])
    d_pbe = abs(e[2]["Ec_pbe"] - e[1]["Ec_pbe"])
    assert d_lda > 0.05 * abs(e[1]["Ec_lda"]) / np.log(1e4)
    assert d_pbe < 1e-2 * d_lda
    assert abs(e[2]["Ec_pbe"] - e[1]["Ec_pbe"]) < abs(e[1]["Ec_pbe"] - e[0]["Ec_pbe"])


def test_gradient_argument_matches_stencil(oracle_mod):
    """Passing the oracle's own stencil gradient equals the default path; a
    density with n <= 0 points skips them."""
    L = (6.0, 6.0, 6.0)
    n = _blobs((10, 10, 10), L, seed=5)
    n[0, 0, :3] = [-1e-6, 0.0, -2e-7]
    h = [x / d for x, d in zip(L, n.shape)]
    a = oracle_mod.semilocal(n, L)
    b = oracle_mod.semilocal(n, L, oracle_mod.gradient(n, h))
    assert a == b
    assert a["n_points"] == 1000 - 3


def test_second_order_gradient_coefficients(oracle_mod):
    """A weakly modulated density n0 (1 + eps cos(2 pi x / L)): to second order in
    the gradient, E_c^PBE - E_c^LDA = +C_MB G and E_x^PBE - E_x^LDA = -C_MB G
    (revPBE the same), G = integral |grad n|^2 / n^(4/3), with the Ma-Brueckner
    coefficient C_MB (golden file).  This fixes the scale of s, t and k_s."""
    from conftest import golden_dict
    C = golden_dict("gradient_coefficients.txt")["C_MB"]
    L = (10.0, 2.0, 2.0)
    shape = (64, 2, 2)
    x = np.arange(shape[0]) * L[0] / shape[0]
    for n0, eps in ((0.05, 2e-3), (1.0, 2e-3), (20.0, 1e-3)):
        n = np.broadcast_to((n0 * (1.0 + eps * np.cos(2 * np.pi * x / L[0])))[:, None, None], shape).copy()
        h = [a / d for a, d in zip(L, shape)]
        g = oracle_mod.gradient(n, h)
        G = np.sum((g ** 2).sum(0) / n ** (4.0 / 3.0)) * h[0] * h[1] * h[2]
        e = oracle_mod.semilocal(n, L)
        assert abs((e["Ec_pbe"] - e["Ec_lda"]) / G - C) <= 2e-4 * C + 1e-3 * C
        assert abs((e["Ex_pbe"] - e["Ex_lda"]) / G + C) <= 1e-3 * C
        assert abs((e["Ex_revpbe"] - e["Ex_lda"]) / G + C) <= 1e-3 * C


def test_exchange_ordering(oracle_mod):
    """F_x >= 1 grows with kappa at every s, so E_x^revPBE <= E_x^PBE <= E_x^LDA < 0
    for any density with gradients (kappa_revPBE = 1.245 > kappa_PBE = 0.804)."""
    L = (6.0, 7.0, 8.0)
    e = oracle_mod.semilocal(_blobs((12, 14, 16), L, seed=7), L)
    assert e["Ex_revpbe"] < e["Ex_pbe"] < e["Ex_lda"] < 0.0
