"""GPU path (through the C ABI) against the FP64 CPU oracle on the same seeded
inputs.  Tolerances: E relative 1e-10 (FP64 path), 1e-6 (FP32 path); v max-norm
relative 1e-10 (FP64), 1e-5 (FP32); integer counts exact."""
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


def _problem(oracle_mod, spline, w):
    return oracle_mod.Problem(w["density"], w["lengths"], w["periodic"], w["n_cut"], w["r_cut"], spline)


def _relerr(a, b):
    return abs(a - b) / abs(b)


def test_kernel_eval_matches_oracle(V, dev, gtable, oracle_spline):
    """Interpolation + the branch past the table in isolation, incl. the last cells,
    clamping, and each case of delta* past the table."""
    rng = np.random.default_rng(3)
    n = 20000
    r = rng.uniform(0.0, 25.0, n)
    qi = 10 ** rng.uniform(-0.7, 0.9, n)
    qj = 10 ** rng.uniform(-0.7, 0.9, n)
    # exact end nodes and a few clamped deltas
    r[:4] = [0.0, 30.0 / 2.0, 60.0 / 4.0, 1e-3]
    qi[:4] = [1.0, 1.0, 2.0, 1.0]
    qj[:4] = [1.0, 1.0, 2.0, 1.0]
    qi[4:8] = [8.0, 9.0, 7.5, 8.0]
    qj[4:8] = [0.01, 0.02, 0.015, 0.0101]
    r[4:8] = [0.5, 0.3, 0.2, 1.0]
    # past the table: delta* > 0 with either argument the smaller, delta* past the
    # last delta node, and D of several hundred (delta* clamped at 0)
    r[8:14] = [10.0, 10.0, 5.0, 5.0, 400.0, 800.0]
    qi[8:14] = [0.3, 6.0, 0.02, 12.1, 1.9, 0.05]
    qj[8:14] = [6.0, 0.3, 12.1, 0.02, 0.1, 2.5]
    p_o, rd_o, _ = oracle_spline.kernel(r, qi, qj)
    p64, rd64 = V.kernel_eval(gtable, _t(r, dev), _t(qi, dev), _t(qj, dev), "fp64")
    p32, rd32 = V.kernel_eval(gtable, _t(r, dev), _t(qi, dev), _t(qj, dev), "fp32")
    p64, rd64, p32, rd32 = (x.cpu().numpy() for x in (p64, rd64, p32, rd32))
    pmax, rmax = np.max(np.abs(p_o)), np.max(np.abs(rd_o))
    # |got - ref| <= rtol |ref| + atol, atol a small fraction of the largest value
    assert np.all(np.abs(p64 - p_o) <= 1e-11 * np.abs(p_o) + 1e-14 * pmax)
    assert np.all(np.abs(rd64 - rd_o) <= 1e-9 * np.abs(rd_o) + 1e-13 * rmax)
    # FP32: the same with single-precision tolerances; the derivative has a kink at
    # D = Dmax (the asymptotic branch is continuous there but not its slope), so
    # pairs within rounding of it are left out
    D = 0.5 * r * (qi + qj)
    away = np.abs(D / 30.0 - 1) > 1e-5
    assert np.all(np.abs(p32 - p_o) <= 1e-5 * np.abs(p_o) + 1e-7 * pmax)
    # r dphi/dd1 = r cD phi_t + cd/(q_i + q_j) sign(ds)(1 -+ ds) phi_u: each term is a
    # cell-coordinate derivative of the spline (a difference of O(phi) coefficients,
    # rounded at 2^-24) scaled by r cD or cd/(q_i + q_j), so its FP32 error is bounded
    # by a few eps32 (r cD + cd/(q_i + q_j)) max|phi|, whatever the size of the derivative
    nD, Dmax, nd = gtable.info()
    cD = 0.5 * (nD - 1) / Dmax
    cd = float(nd)
    eps32 = 2.0 ** -24
    atol = 16 * eps32 * (r * cD + cd / (qi + qj)) * pmax
    err = np.abs(rd32 - rd_o)
    ok = (err <= 1e-4 * np.abs(rd_o) + atol) | ~away
    if not np.all(ok):
        bad = np.argsort(-(err - atol))[:5]
        raise AssertionError("FP32 r dphi/dd1 off: " + "; ".join(
            f"r={r[b]:.4g} qi={qi[b]:.4g} qj={qj[b]:.4g} got={rd32[b]:.6g} ref={rd_o[b]:.6g} atol={atol[b]:.3g}"
            for b in bad))


def test_q0_matches_oracle(V, dev, oracle_mod):
    rng = np.random.default_rng(5)
    n = 10 ** rng.uniform(-6, 0.5, size=(10, 13, 7))
    L = (5.0, 6.5, 3.5)
    h = [l / d for l, d in zip(L, n.shape)]
    g = oracle_mod.gradient(n, h)
    q, qn, qg = oracle_mod.q0(n, g)
    gq, gqn, gqg = V.q0(_t(n, dev), L)
    for a, b in ((gq, q), (gqn, qn), (gqg, qg)):
        a = a.cpu().numpy()
        assert np.max(np.abs(a - b) / (np.abs(b) + 1e-300)) < 1e-12


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-6)])
def test_energy_kr_dimer(V, dev, gtable, oracle_mod, oracle_spline, prec, tol):
    """Rare-gas dimer, 24x18x18, open cell, all 7,776 points active."""
    from paper_0810_2273_gb300 import inputs
    w = inputs.kr_dimer()
    e = _problem(oracle_mod, oracle_spline, w).energy()
    E, res = V.energy(_t(w["density"], dev), w["lengths"], w["periodic"], w["n_cut"], w["r_cut"],
                      gtable, prec)
    assert _relerr(E, e["E"]) < tol, (E, e["E"])
    assert _relerr(res["E_diag"], e["E_diag"]) < 1e-12
    assert res["pairs"] == e["pairs"] == 7776 * 7775
    assert res["n_active"] == 7776
    if prec == "fp64":
        assert res["n_clamped"] == e["clamped"]


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-6)])
def test_energy_periodic_monolayer_small(V, dev, gtable, oracle_mod, oracle_spline, prec, tol):
    """Monolayer cell on a coarse 12x21x30 grid, periodic x, y, 20 bohr cutoff:
    spans several tiles with a ragged last tile; pair counts exact."""
    from paper_0810_2273_gb300 import inputs
    w = inputs.xe_monolayer((12, 21, 30))
    e = _problem(oracle_mod, oracle_spline, w).energy()
    E, res = V.energy(_t(w["density"], dev), w["lengths"], w["periodic"], w["n_cut"], w["r_cut"],
                      gtable, prec)
    assert res["n_active"] % 256 != 0
    assert _relerr(E, e["E"]) < tol, (E, e["E"])
    assert res["pairs"] == e["pairs"]


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_potential_small(V, dev, gtable, oracle_mod, oracle_spline, prec, tol):
    """E and v on a 20^3 molecule grid and on a periodic slab, whole grid vs the oracle."""
    from paper_0810_2273_gb300 import inputs
    for w in (inputs.molecule24((20, 20, 20)), inputs.xe_monolayer((14, 24, 34))):
        P = _problem(oracle_mod, oracle_spline, w)
        e = P.energy()
        vo = P.potential(e["A"], e["U"])
        E, v, res, A, U = V.potential(_t(w["density"], dev), w["lengths"], w["periodic"], w["n_cut"],
                                      w["r_cut"], gtable, prec, want_AU=True)
        v = v.cpu().numpy()
        assert _relerr(E, e["E"]) < (tol if prec == "fp64" else 1e-6), (w["name"], E, e["E"])
        assert np.max(np.abs(v - vo)) < tol * np.max(np.abs(vo)), w["name"]
        flat = w["density"].ravel() >= w["n_cut"]
        Ag = A.cpu().numpy().ravel()[flat]
        Ug = U.cpu().numpy().ravel()[flat]
        assert np.max(np.abs(Ag - e["A"])) < tol * np.max(np.abs(e["A"]))
        assert np.max(np.abs(Ug - e["U"])) < tol * np.max(np.abs(e["U"]))
        assert res["pairs"] == e["pairs"]


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_potential_far_pairs(V, dev, gtable, oracle_mod, oracle_spline, prec, tol):
    """A metal-like slab under a 20 bohr cutoff on a coarse 24x20x40 grid: dense
    layers (q0 up to ~4) put almost half of the pairs at D above 30 258/399 (past
    the table rows the FP32 kernel keeps in shared memory) and a tenth past the
    table (D > 30, eq. 17 times the factor g).  E, A, U and v against the oracle."""
    from paper_0810_2273_gb300 import inputs
    w = inputs.slab_adsorbate((24, 20, 40))
    P = _problem(oracle_mod, oracle_spline, w)
    # the case does reach those D: a sample of 300 i points against every j and image
    rng = np.random.default_rng(12)
    dims = np.array(P.dims)
    h = np.array(w["lengths"]) / dims
    idx = np.array([P.i0, P.i1, P.i2], dtype=np.float64).T
    I = rng.choice(P.n_active, 300, replace=False)
    Ds = []
    for m0 in range(-2, 3):
        for m1 in range(-2, 3):
            d = (idx[I][:, None, :] - idx[None, :, :] + np.array([m0, m1, 0]) * dims) * h
            r = np.sqrt((d * d).sum(2))
            Ds.append((0.5 * r * (P.qa[I][:, None] + P.qa[None, :]))[r <= w["r_cut"]])
    D = np.concatenate(Ds)
    assert np.mean(D > 30.0 * 258 / 399) > 0.3 and np.mean(D > 30.0) > 0.05
    e = P.energy()
    vo = P.potential(e["A"], e["U"])
    E, v, res, A, U = V.potential(_t(w["density"], dev), w["lengths"], w["periodic"], w["n_cut"],
                                  w["r_cut"], gtable, prec, want_AU=True)
    assert _relerr(E, e["E"]) < (tol if prec == "fp64" else 1e-6), (E, e["E"])
    flat = w["density"].ravel() >= w["n_cut"]
    Ag = A.cpu().numpy().ravel()[flat]
    Ug = U.cpu().numpy().ravel()[flat]
    assert np.max(np.abs(Ag - e["A"])) < tol * np.max(np.abs(e["A"]))
    assert np.max(np.abs(Ug - e["U"])) < tol * np.max(np.abs(e["U"]))
    assert np.max(np.abs(v.cpu().numpy() - vo)) < tol * np.max(np.abs(vo))
    assert res["pairs"] == e["pairs"]
    Ee, rese = V.energy(_t(w["density"], dev), w["lengths"], w["periodic"], w["n_cut"], w["r_cut"],
                        gtable, prec)
    assert _relerr(Ee, e["E"]) < (tol if prec == "fp64" else 1e-6) and rese["pairs"] == e["pairs"]


def test_edge_cases(V, dev, gtable, oracle_mod, oracle_spline):
    """No active point; one active point; grid sides not multiples of 4; huge cutoff."""
    rng = np.random.default_rng(8)
    L = (3.5, 4.2, 5.4)
    n = rng.uniform(0.01, 0.5, size=(5, 7, 9))
    for prec in ("fp64", "fp32"):
        E, res = V.energy(_t(n, dev), L, (0, 0, 0), 10.0, 0.0, gtable, prec)
        assert E == 0.0 and res["n_active"] == 0 and res["pairs"] == 0
        one = np.full((5, 7, 9), 1e-3)
        one[2, 3, 4] = 0.8
        E, res = V.energy(_t(one, dev), L, (0, 0, 0), 0.1, 0.0, gtable, prec)
        ref = 0.5 * (np.prod(L) / one.size) ** 2 * 0.64 * oracle_spline.f[0, 0]
        assert abs(E - ref) < (1e-12 if prec == "fp64" else 1e-6) * abs(ref) and res["pairs"] == 0
        P = oracle_mod.Problem(n, L, (0, 0, 0), 0.2, 0.0, oracle_spline)
        e = P.energy()
        E, res = V.energy(_t(n, dev), L, (0, 0, 0), 0.2, 0.0, gtable, prec)
        assert _relerr(E, e["E"]) < (1e-10 if prec == "fp64" else 1e-6)
        assert res["pairs"] == e["pairs"]
        Pp = oracle_mod.Problem(n, L, (1, 1, 1), 0.2, 6.0, oracle_spline)
        ep = Pp.energy()
        E, res = V.energy(_t(n, dev), L, (1, 1, 1), 0.2, 6.0, gtable, prec)
        assert _relerr(E, ep["E"]) < (1e-10 if prec == "fp64" else 1e-6)
        assert res["pairs"] == ep["pairs"]


def test_batched_matches_single(V, dev, gtable):
    """Several uneven densities in one graph-captured launch equal one-at-a-time calls,
    also on replay with changed density values."""
    import torch
    from paper_0810_2273_gb300 import inputs
    ws = [inputs.kr_dimer((16, 12, 12)), inputs.kr_dimer((20, 15, 15)), inputs.molecule24((14, 14, 14))]
    ns = [_t(w["density"], dev) for w in ws]
    for prec, tol in (("fp64", 1e-12), ("fp32", 1e-6)):
        Es, _ = V.energy_batched(ns, [w["lengths"] for w in ws], [w["periodic"] for w in ws], 1e-6, 0.0,
                                 gtable, prec)
        for w, nt, Eb in zip(ws, ns, Es):
            E1, _ = V.energy(nt, w["lengths"], w["periodic"], 1e-6, 0.0, gtable, "fp64")
            assert _relerr(Eb, E1) < tol
        with torch.no_grad():
            ns[1].mul_(1.1)
        Es2, _ = V.energy_batched(ns, [w["lengths"] for w in ws], [w["periodic"] for w in ws], 1e-6, 0.0,
                                  gtable, prec)
        E1, _ = V.energy(ns[1], ws[1]["lengths"], ws[1]["periodic"], 1e-6, 0.0, gtable, "fp64")
        assert _relerr(Es2[1], E1) < tol and _relerr(Es2[0], Es[0]) < 1e-14
        with torch.no_grad():
            ns[1].div_(1.1)


def test_autograd_function(V, dev, gtable):
    import torch
    from paper_0810_2273_gb300 import inputs
    w = inputs.kr_dimer((16, 12, 12))
    n = _t(w["density"], dev).requires_grad_(True)
    spec = dict(lengths=w["lengths"], periodic=w["periodic"], n_cut=w["n_cut"], r_cut=w["r_cut"],
                table=gtable, precision="fp64")
    E = V.nonlocal_energy(n, spec)
    E.backward()
    _, v, _ = V.potential(n.detach(), w["lengths"], w["periodic"], w["n_cut"], w["r_cut"], gtable, "fp64")
    dV = np.prod(w["lengths"]) / n.numel()
    assert torch.allclose(n.grad, dV * v, rtol=1e-12, atol=1e-14 * float(torch.max(torch.abs(dV * v))))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_every_pattern_of_periodic_axes(V, dev, gtable, oracle_mod, oracle_spline, prec, tol):
    """One and two periodic axes in every direction (a wire along each axis, a
    slab normal to each axis) and a skewed cell periodic along its second axis
    only: E, v, A, U and the pair count against the oracle.  Each pattern drops
    the images of different axes, which the culling and the image lists must
    follow."""
    from paper_0810_2273_gb300 import inputs
    rng = np.random.default_rng(77)
    dims, L = (10, 11, 12), (8.0, 8.8, 9.6)
    atoms = [(tuple(rng.uniform(0.2, 0.8, 3) * np.asarray(L)), inputs.single_exponential(z, a))
             for z, a in ((6.0, 0.7), (4.0, 0.6), (1.0, 0.5))]
    patterns = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 0, 1), (0, 1, 1)]
    for per in patterns:
        n = inputs.density(dims, L, atoms, periodic=per)
        P = oracle_mod.Problem(n, L, per, 1e-4, 9.0, oracle_spline)
        e = P.energy()
        vo = P.potential(e["A"], e["U"])
        E, v, res, A, U = V.potential(_t(n, dev), L, per, 1e-4, 9.0, gtable, prec, want_AU=True)
        assert _relerr(E, e["E"]) < (tol if prec == "fp64" else 1e-6), (per, E, e["E"])
        assert res["pairs"] == e["pairs"], per
        v = v.cpu().numpy()
        assert np.max(np.abs(v - vo)) < tol * np.max(np.abs(vo)), per
        act = n.ravel() >= 1e-4
        assert np.max(np.abs(A.cpu().numpy().ravel()[act] - e["A"])) < tol * np.max(np.abs(e["A"])), per
        assert np.max(np.abs(U.cpu().numpy().ravel()[act] - e["U"])) < tol * np.max(np.abs(e["U"])), per
    cell = np.array([[8.0, 0.0, 0.0], [3.0, 8.8, 0.0], [1.0, -0.5, 9.6]])
    per = (0, 1, 0)
    n = inputs.density_cell(dims, cell, atoms, periodic=per)
    P = oracle_mod.Problem(n, None, per, 1e-4, 9.0, oracle_spline, cell=cell)
    e = P.energy()
    vo = P.potential(e["A"], e["U"])
    E, v, res = V.potential(_t(n, dev), cell, per, 1e-4, 9.0, gtable, prec)
    assert _relerr(E, e["E"]) < (tol if prec == "fp64" else 1e-6), ("skewed", E, e["E"])
    assert res["pairs"] == e["pairs"]
    assert np.max(np.abs(v.cpu().numpy() - vo)) < tol * np.max(np.abs(vo))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-6)])
def test_tiny_and_cell_sized_cutoffs(V, dev, gtable, oracle_mod, oracle_spline, prec, tol):
    """r_cut below the grid spacing: no pair is inside, and E is the self term
    alone.  r_cut just past one cell length along the only periodic axis: every
    point meets its own first images (self-images are ordinary pairs), which the
    pair count and E of the oracle show too."""
    rng = np.random.default_rng(19)
    L = (3.5, 4.2, 5.4)
    n = rng.uniform(0.01, 0.5, size=(7, 8, 9))
    per = (1, 0, 0)
    E, res = V.energy(_t(n, dev), L, per, 0.2, 0.3, gtable, prec)   # h = 0.5, 0.525, 0.6 bohr
    P = oracle_mod.Problem(n, L, per, 0.2, 0.3, oracle_spline)
    e = P.energy()
    assert res["pairs"] == 0 == e["pairs"]
    # (the FP32 path sums the self term with the FP32 table's phi(0,0); E_diag is FP64)
    assert abs(E - res["E_diag"]) <= tol * abs(E) and abs(E - e["E"]) <= tol * abs(e["E"])
    E, res = V.energy(_t(n, dev), L, per, 0.2, 3.6, gtable, prec)
    P = oracle_mod.Problem(n, L, per, 0.2, 3.6, oracle_spline)
    e = P.energy()
    assert res["pairs"] == e["pairs"] and res["pairs"] >= 2 * res["n_active"]
    assert _relerr(E, e["E"]) < tol, (E, e["E"])
