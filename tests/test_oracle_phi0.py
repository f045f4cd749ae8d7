"""Pins of the oracle's voxel-averaged diagonal phi0(q) (the reading of the
paper's undocumented "phi0" step): the exact small-voxel logarithmic law, the
exact scale duality between voxel size and q, and Monte Carlo averages of the
kernel over pairs of uniform points in a voxel (box and skewed)."""
import numpy as np
import pytest

BOX = np.diag([0.35, 0.30, 0.28])
SKEW = np.array([[0.34, 0.0, 0.0], [0.17, 0.296, 0.0], [0.02, -0.03, 0.33]])


def _small_d_model(oracle_spline):
    s = oracle_spline
    D1, D2 = s.hD, 2 * s.hD
    psi1 = s.f[1, 0] + (2 / np.pi) * np.log(D1)
    psi2 = s.f[2, 0] + (2 / np.pi) * np.log(D2)
    psi0 = (4 * psi1 - psi2) / 3
    return D1, psi0, (psi1 - psi0) / D1 ** 2


def _mc_pairs(vox, n, seed):
    """Differences r - r' of n pairs of uniform points in the voxel spanned by vox."""
    rng = np.random.default_rng(seed)
    t = rng.uniform(0, 1, (n, 3)) - rng.uniform(0, 1, (n, 3))
    return t @ vox


def _phi_delta0(oracle_spline, D):
    D1, psi0, c2 = _small_d_model(oracle_spline)
    out = np.empty_like(D)
    small = D < D1
    out[small] = -(2 / np.pi) * np.log(D[small]) + psi0 + c2 * D[small] ** 2
    if np.any(~small):
        Dl = D[~small]
        out[~small] = oracle_spline.kernel(Dl, np.ones_like(Dl), np.ones_like(Dl))[0]
    return out


def test_small_voxel_logarithmic_law(oracle_spline):
    """For q |r - r'| < D_1 the model is -(2/pi) ln(q s) + psi0 + c2 (q s)^2, so
    phi0(q) = -(2/pi)(ln q + <ln s>) + psi0 + c2 q^2 <s^2>, with <s^2> = sum |v_a|^2 / 6
    exactly and <ln s> from Monte Carlo; the slope in ln q is exactly -2/pi."""
    _, psi0, c2 = _small_d_model(oracle_spline)
    for vox in (BOX, SKEW):
        q = np.array([1e-3, 2e-3, 4e-3])
        p = oracle_spline.phi0(vox, q, 7, 8)
        s2 = np.sum(vox ** 2) / 6.0
        # the quadratic term is below 1e-9 here; the log slope is exact
        lin = p - c2 * q ** 2 * s2
        assert abs((lin[0] - lin[1]) - (2 / np.pi) * np.log(2)) < 1e-8
        assert abs((lin[1] - lin[2]) - (2 / np.pi) * np.log(2)) < 1e-8
        d = _mc_pairs(vox, 4_000_000, 7)
        ln_s = np.log(np.sqrt((d ** 2).sum(1)))
        mean_ln, err = ln_s.mean(), 4 * ln_s.std() / np.sqrt(len(ln_s))
        pred = -(2 / np.pi) * (np.log(q[0]) + mean_ln) + psi0
        assert abs(lin[0] - pred) < (2 / np.pi) * err + 1e-6


def test_scale_duality(oracle_spline):
    """phi0(q; lam V) = phi0(lam q; V): only q |r - r'| enters."""
    for lam in (0.5, 3.0):
        for q in (0.4, 2.5):
            a = oracle_spline.phi0(lam * SKEW, [q], 6, 6)[0]
            b = oracle_spline.phi0(SKEW, [lam * q], 6, 6)[0]
            assert abs(a - b) <= 1e-12 * abs(a) + 1e-15


@pytest.mark.parametrize("q", [0.5, 2.0, 6.0])
def test_monte_carlo_voxel_average(oracle_spline, q):
    """phi0(q) is the mean of phi(q |r - r'|, delta = 0) over pairs of uniform points
    in the voxel: compare with 3e5-pair Monte Carlo averages within 4 standard errors."""
    for vox, seed in ((BOX, 1), (SKEW, 2)):
        d = _mc_pairs(vox, 300_000, seed + int(10 * q))
        vals = _phi_delta0(oracle_spline, q * np.sqrt((d ** 2).sum(1)))
        mean, err = vals.mean(), 4 * vals.std() / np.sqrt(len(vals))
        p = oracle_spline.phi0(vox, [q], 7, 8)[0]
        assert abs(p - mean) < err + 1e-6, (q, p, mean, err)


def test_quadrature_converged(oracle_spline):
    """The graded tensor rule: two refinements agree to 1e-5 relative (the kinks of
    the integrand at q s = D_1 and q s = Dmax are not aligned with the panels)."""
    for q in (0.3, 1.5, 5.0):
        a = oracle_spline.phi0(SKEW, [q], 6, 6)[0]
        b = oracle_spline.phi0(SKEW, [q], 8, 10)[0]
        assert abs(a - b) <= 1e-5 * abs(b) + 1e-8
