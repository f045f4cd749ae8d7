"""Pins of the oracle's double sum E_c^nl (paper eq. 2, section 3: trimming and
periodic images) and of its adjoint potential v = dE/dn / dV."""
import numpy as np
import pytest

from conftest import golden_dict


def _blob(shape, rng, lo=0.05, hi=0.6, zero_border=0):
    n = rng.uniform(lo, hi, size=shape)
    if zero_border:
        b = zero_border
        m = np.zeros(shape, dtype=bool)
        m[b:-b, b:-b, b:-b] = True
        n = np.where(m, n, 0.0)
    return n


def test_brute_force_direct_quadrature(oracle_mod, oracle_spline):
    """Same sum with phi from direct quadrature of eq. (14) at every pair instead of
    the spline: the two differ only by the interpolation error of the table."""
    rng = np.random.default_rng(17)
    n = 0.05 + 0.3 * np.exp(-rng.uniform(0, 2, size=(6, 6, 6)))
    P = oracle_mod.Problem(n, (3.0, 3.0, 3.0), (0, 0, 0), 0.0, 0.0, oracle_spline)
    e = P.energy()
    Eb = P.brute_energy(oracle_mod.QUAD_TABLE)
    off_tab = e["E"] - e["E_diag"]
    off_bru = Eb - e["E_diag"]
    assert abs(off_tab - off_bru) < 1e-5 * abs(off_bru), (off_tab, off_bru)
    assert e["pairs"] == P.n_active * (P.n_active - 1)


def test_translation_invariance_periodic(oracle_mod, oracle_spline):
    """A density periodic in all axes, shifted by whole grid steps, has the same
    E (the pair set is only relabelled)."""
    rng = np.random.default_rng(23)
    n = _blob((8, 7, 6), rng)
    L = (3.2, 3.1, 2.9)
    args = dict(lengths=L, periodic=(1, 1, 1), n_cut=0.1, rc=3.0, spline=oracle_spline)
    E0 = oracle_mod.Problem(n, **args).energy()
    for sh in [(1, 0, 0), (0, 3, 0), (2, 5, 4)]:
        E1 = oracle_mod.Problem(np.roll(n, sh, axis=(0, 1, 2)), **args).energy()
        assert abs(E1["E"] - E0["E"]) < 1e-12 * abs(E0["E"])
        assert E1["pairs"] == E0["pairs"]


def test_far_fragments_cross_term_is_asymptotic_sum(oracle_mod, oracle_spline):
    """Two compactly supported blobs so far apart that every cross pair has D > 30:
    E_AB - E_A - E_B must equal dV^2 sum_{i in A, j in B} n_i n_j g phi_17(q_i r, q_j r),
    with the factor g of the kernel past the table, written out here with numpy and
    scipy (the factor 1/2 and the two orderings give 1)."""
    sp = pytest.importorskip("scipy.interpolate")
    g = golden_dict("dion_kernel.txt")
    rng = np.random.default_rng(29)
    dims = (40, 8, 8)
    L = (40.0, 8.0, 8.0)
    nA = np.zeros(dims)
    nB = np.zeros(dims)
    nA[3:8, 2:6, 2:6] = rng.uniform(0.5, 2.0, size=(5, 4, 4))
    nB[30:35, 2:6, 2:6] = rng.uniform(0.5, 2.0, size=(5, 4, 4))
    args = dict(lengths=L, periodic=(0, 0, 0), n_cut=0.25, rc=0.0, spline=oracle_spline)
    PA = oracle_mod.Problem(nA, **args)
    PB = oracle_mod.Problem(nB, **args)
    PAB = oracle_mod.Problem(nA + nB, **args)
    EA, EB, EAB = PA.energy()["E"], PB.energy()["E"], PAB.energy()["E"]
    h = np.array(L) / np.array(dims)
    rA = np.stack([PA.i0, PA.i1, PA.i2], 1) * h
    rB = np.stack([PB.i0, PB.i1, PB.i2], 1) * h
    r = np.linalg.norm(rA[:, None, :] - rB[None, :, :], axis=-1)
    d1 = PA.qa[:, None] * r
    d2 = PB.qa[None, :] * r
    assert np.min(0.5 * (d1 + d2)) > 30.0
    s = oracle_spline
    dln = np.arange(s.nd) * s.hd
    ratio = s.f[-1] / (-g["C_asym"] / ((s.Dmax * (1 + dln)) ** 2 * (s.Dmax * (1 - dln)) ** 2 *
                                      ((s.Dmax * (1 + dln)) ** 2 + (s.Dmax * (1 - dln)) ** 2)))
    rho = sp.CubicSpline(dln, ratio, bc_type=((1, 0.0), (2, 0.0)))
    # eq. (17) times g = rho(delta*) + (1 - rho(0)) (1 - (Dmax/D)^2), with
    # delta* = max(0, 1 - min(d1, d2)/Dmax) (linear past the last delta node)
    D = 0.5 * (d1 + d2)
    dstar = np.maximum(0.0, 1.0 - np.minimum(d1, d2) / s.Dmax)
    past = np.maximum(dstar - dln[-1], 0.0)
    gfac = rho(np.minimum(dstar, dln[-1])) + rho(dln[-1], 1) * past
    gfac = gfac + (1.0 - rho(0.0)) * (1.0 - (s.Dmax / D) ** 2)
    phi = gfac * (-g["C_asym"] / (d1 ** 2 * d2 ** 2 * (d1 ** 2 + d2 ** 2)))
    cross = PA.dV ** 2 * np.sum(PA.na[:, None] * PB.na[None, :] * phi)
    assert abs((EAB - EA - EB) - cross) < 1e-6 * abs(cross)
    assert abs(EA) > 1e3 * abs(cross)


def test_self_term_and_prefactor(oracle_mod, oracle_spline):
    """One active point: E = 1/2 dV^2 n^2 phi(0, 0) = E_diag, no pairs."""
    n = np.zeros((5, 5, 5))
    n[2, 2, 2] = 0.7
    P = oracle_mod.Problem(n, (2.5, 2.5, 2.5), (0, 0, 0), 0.1, 0.0, oracle_spline)
    e = P.energy()
    dV = 0.5 ** 3
    assert abs(e["E"] - 0.5 * dV ** 2 * 0.49 * oracle_spline.f[0, 0]) < 1e-15
    assert abs(e["E"] - e["E_diag"]) < 1e-15 * abs(e["E"]) and e["pairs"] == 0


def test_periodic_cutoff_counts(oracle_mod, oracle_spline):
    """Ordered pair count with images under a spherical cutoff, by brute force."""
    rng = np.random.default_rng(31)
    n = _blob((5, 4, 6), rng)
    L = (2.0, 1.8, 3.0)
    rc = 2.5
    P = oracle_mod.Problem(n, L, (1, 1, 0), 0.2, rc, oracle_spline)
    e = P.energy()
    h = np.array(L) / np.array(n.shape)
    pos = np.stack([P.i0, P.i1, P.i2], 1) * h
    cnt = 0
    for m0 in range(-3, 4):
        for m1 in range(-3, 4):
            d = pos[:, None, :] - pos[None, :, :] + np.array([m0 * L[0], m1 * L[1], 0.0])
            r2 = np.sum(d * d, axis=-1)
            cnt += int(np.sum(r2 <= rc * rc * (1 + 1e-12)))
    cnt -= P.n_active          # self terms
    assert e["pairs"] == cnt


@pytest.mark.parametrize("periodic", [(0, 0, 0), (1, 1, 0)])
def test_potential_is_derivative_of_energy(oracle_mod, oracle_spline, periodic):
    """v_m = dE/dn_m / dV by central differences of the FP64 E (mask frozen:
    perturbed points stay on their side of n_cut), at active points and at
    inactive points next to the active region (divergence term only)."""
    rng = np.random.default_rng(37)
    dims = (8, 8, 7)
    L = (4.0, 4.4, 3.5)
    n = 0.02 + 0.5 * rng.uniform(0, 1, size=dims) * np.exp(-rng.uniform(0, 3, size=dims))
    n_cut = 0.05
    n[np.abs(n - n_cut) < 0.01] += 0.03
    rc = 3.0 if any(periodic) else 0.0
    P = oracle_mod.Problem(n, L, periodic, n_cut, rc, oracle_spline)
    v = P.potential()
    flat = n.ravel()
    act = np.nonzero(flat >= 2 * n_cut)[0]
    ina = np.nonzero(flat < 0.5 * n_cut)[0]
    pts = np.concatenate([rng.choice(act, 6, replace=False), rng.choice(ina, 4, replace=False)])
    for m in pts:
        hstep = 1e-4 * flat[m]
        def E_at(delta):
            nn = flat.copy()
            nn[m] += delta
            return oracle_mod.Problem(nn.reshape(dims), L, periodic, n_cut, rc, oracle_spline).energy()["E"]
        fd = (E_at(hstep) - E_at(-hstep)) / (2 * hstep) / P.dV
        assert abs(fd - v.ravel()[m]) < 1e-6 * np.max(np.abs(v)), (m, fd, v.ravel()[m])
    vp = P.potential_at(pts)
    assert np.max(np.abs(vp - v.ravel()[pts])) < 1e-13 * np.max(np.abs(v))
