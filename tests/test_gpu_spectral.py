"""The spectral (FFT) gradient option through the C ABI against the oracle's FFT
gradient: the gradient itself (even and odd axes, skewed cells, an axis long
enough to shrink the kernel's tile), q0, the semilocal energies, E and v of the
pair sum in both precisions, the voxel diagonal's potential, and the batched
path.  Tolerances as the finite-difference path: E 1e-10 (FP64) / 1e-6 (FP32),
v 1e-10 / 1e-5 of max|v|; the gradient 1e-12 of its largest component."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import __graft_entry__
    __graft_entry__.build()
    import paper_0810_2273_gb300 as V
    return V


@pytest.fixture(scope="module")
def dev():
    import torch
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def gtable(V, oracle_table):
    return V.Table.from_nodes(oracle_table, 30.0)


def _t(a, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(dev)


def _hex_cell(c=12.0):
    return np.array([[8.2, 0.0, 0.0], [4.1, 8.2 * np.sqrt(3) / 2, 0.0], [0.0, 0.0, c]])


@pytest.mark.parametrize("case", ["even", "odd", "skew", "long"])
def test_gradient_matches_oracle(V, dev, oracle_mod, case):
    rng = np.random.default_rng(21)
    if case == "even":
        shape, geom = (24, 18, 20), (9.0, 7.0, 8.0)
    elif case == "odd":
        shape, geom = (15, 21, 9), (6.0, 8.5, 4.0)
    elif case == "skew":
        shape, geom = (16, 16, 24), _hex_cell()
    else:  # 900 points along axis 0 with 80 columns: the tile holds 16 of them
        shape, geom = (900, 2, 40), (90.0, 1.0, 4.0)
    n = np.exp(rng.normal(size=shape) * 0.3)
    g = V.gradient(_t(n, dev), geom, "spectral").cpu().numpy()
    ref = oracle_mod.gradient_spectral(n, geom)
    assert np.max(np.abs(g - ref)) < 1e-12 * np.max(np.abs(ref)) * np.sqrt(max(shape))
    gf = V.gradient(_t(n, dev), geom, "fd").cpu().numpy()
    if np.asarray(geom).shape == (3, 3):
        reff = oracle_mod.gradient_cell(n, geom)
    else:
        reff = oracle_mod.gradient(n, [L / d for L, d in zip(geom, shape)])
    assert np.max(np.abs(gf - reff)) < 1e-12 * np.max(np.abs(reff))


def test_q0_and_semilocal(V, dev, oracle_mod):
    from paper_0810_2273_gb300 import inputs
    w = inputs.kr_dimer()
    n = w["density"]
    g = oracle_mod.gradient_spectral(n, w["lengths"])
    q, qn, qg = oracle_mod.q0(n, g)
    gq, gqn, gqg = V.q0(_t(n, dev), w["lengths"], gradient="spectral")
    for a, b in ((gq, q), (gqn, qn)):
        a = a.cpu().numpy()
        assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))
    # dq0/dgrad n = -Zab grad n / (18 k_F n^2): the spectral gradient's rounding is
    # absolute (each value sums a whole line), and 1/n^2 magnifies it where n is
    # tiny, so compare n^2 dq0/dgrad n
    a = gqg.cpu().numpy() * n ** 2
    b = qg * n ** 2
    assert np.max(np.abs(a - b)) <= 1e-10 * np.max(np.abs(b))
    so = oracle_mod.semilocal(n, w["lengths"], g=g)
    sg = V.semilocal(_t(n, dev), w["lengths"], w["periodic"], gradient="spectral")
    for k in ("Ex_lda", "Ec_lda", "Ex_pbe", "Ec_pbe", "Ex_revpbe"):
        assert abs(sg[k] - so[k]) <= 1e-12 * abs(so[k]), k


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
@pytest.mark.parametrize("case", ["molecule", "monolayer", "hex"])
def test_energy_and_potential(V, dev, gtable, oracle_mod, oracle_spline, prec, tol, case):
    from paper_0810_2273_gb300 import inputs
    if case == "molecule":
        w = inputs.molecule24((18, 18, 18))
    elif case == "monolayer":
        w = inputs.xe_monolayer((14, 24, 34))
    else:
        w = inputs.xe_monolayer_hex((16, 16, 36))
    geom = w.get("cell", w["lengths"])
    cell = w.get("cell")
    P = oracle_mod.Problem(w["density"], w["lengths"], w["periodic"], w["n_cut"], w["r_cut"], oracle_spline,
                           cell=cell, gradient="spectral")
    e = P.energy()
    vo = P.potential(e["A"], e["U"])
    E, v, res = V.potential(_t(w["density"], dev), geom, w["periodic"], w["n_cut"], w["r_cut"], gtable, prec,
                            gradient="spectral")
    Etol = tol if prec == "fp64" else 1e-6
    assert abs(E - e["E"]) <= Etol * abs(e["E"])
    assert np.max(np.abs(v.cpu().numpy() - vo)) <= tol * np.max(np.abs(vo))
    assert res["pairs"] == e["pairs"]
    Ee, _ = V.energy(_t(w["density"], dev), geom, w["periodic"], w["n_cut"], w["r_cut"], gtable, prec,
                     gradient="spectral")
    assert abs(Ee - e["E"]) <= Etol * abs(e["E"])
    # the option changes q0 and so E: the finite-difference E differs
    Ef, _ = V.energy(_t(w["density"], dev), geom, w["periodic"], w["n_cut"], w["r_cut"], gtable, prec)
    assert Ef != Ee


def test_diag_voxel_potential_and_batched(V, dev, gtable):
    """The voxel diagonal with the spectral gradient equals the same call given
    that gradient explicitly; its potential is the central difference of its
    FP64 energy; batched spectral energies equal one-at-a-time calls."""
    from paper_0810_2273_gb300 import inputs
    w = inputs.kr_dimer((16, 12, 12))
    n = _t(w["density"], dev)
    L = w["lengths"]
    rs = V.diag_voxel(n, L, w["periodic"], w["n_cut"], gtable, gradient="spectral")
    g = V.gradient(n, L, "spectral")
    rg = V.diag_voxel(n, L, w["periodic"], w["n_cut"], gtable, grad=g)
    assert rs["E_diag_voxel"] == rg["E_diag_voxel"]
    _, dv = V.diag_voxel_potential(n, L, w["periodic"], w["n_cut"], gtable, gradient="spectral")
    dv = dv.cpu().numpy()
    flat = w["density"].ravel()
    dV = np.prod(L) / flat.size
    rng = np.random.default_rng(4)
    for m in rng.choice(np.nonzero(flat > 4 * w["n_cut"])[0], 4, replace=False):
        h = 1e-4 * flat[m]
        Es = []
        for sgn in (1, -1):
            nn = flat.copy()
            nn[m] += sgn * h
            r = V.diag_voxel(_t(nn.reshape(w["density"].shape), dev), L, w["periodic"], w["n_cut"], gtable,
                             gradient="spectral")
            Es.append(r["E_diag_voxel"] - r["E_diag_table"])
        fd = (Es[0] - Es[1]) / (2 * h * dV)
        assert abs(fd - dv.ravel()[m]) <= 1e-6 * np.max(np.abs(dv)) + 1e-6 * abs(fd)
    ws = [inputs.kr_dimer((16, 12, 12)), inputs.kr_dimer((20, 15, 15))]
    ns = [_t(x["density"], dev) for x in ws]
    Es, _ = V.energy_batched(ns, [x["lengths"] for x in ws], [x["periodic"] for x in ws], ws[0]["n_cut"],
                             ws[0]["r_cut"], gtable, "fp64", gradient="spectral")
    for x, nx, Eb in zip(ws, ns, Es):
        E1, _ = V.energy(nx, x["lengths"], x["periodic"], x["n_cut"], x["r_cut"], gtable, "fp64",
                         gradient="spectral")
        assert abs(Eb - E1) <= 1e-12 * abs(E1)
