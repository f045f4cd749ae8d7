"""General (non-orthogonal) cells through the C ABI against the oracle: the
hexagonal monolayer cell (60 degrees), energy and potential in both
precisions, with the skewed gradient, its adjoint and the full metric in the
pair sum; invariances that any correct implementation keeps."""
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


def _smooth(cell, dims, seed, n0=0.02):
    """Positive periodic density on the cell's grid with its exact gradient."""
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
        G = 2 * np.pi * (m[0] * B[0] + m[1] * B[1] + m[2] * B[2])
        for c in range(3):
            g[c] -= A * np.sin(ph) * G[c]
    return n, g


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-6)])
def test_hex_monolayer_energy_and_potential(V, dev, gtable, oracle_mod, oracle_spline, prec, tol):
    from paper_0810_2273_gb300 import inputs
    w = inputs.xe_monolayer_hex((12, 12, 30))
    cell = w["cell"]
    P = oracle_mod.Problem(w["density"], None, w["periodic"], w["n_cut"], w["r_cut"], oracle_spline, cell=cell)
    e = P.energy()
    vo = P.potential(e["A"], e["U"])
    n = _t(w["density"], dev)
    E, v, res, A, U = V.potential(n, cell, w["periodic"], w["n_cut"], w["r_cut"], gtable, prec, want_AU=True)
    assert res["pairs"] == e["pairs"] > 0
    assert abs(E - e["E"]) <= (tol if prec == "fp64" else 1e-6) * abs(e["E"])
    vtol = 1e-10 if prec == "fp64" else 1e-5
    assert np.max(np.abs(v.cpu().numpy() - vo)) <= vtol * np.max(np.abs(vo))
    flat = w["density"].ravel() >= w["n_cut"]
    assert np.max(np.abs(U.cpu().numpy().ravel()[flat] - e["U"])) <= vtol * np.max(np.abs(e["U"]))
    E2, res2 = V.energy(n, cell, w["periodic"], w["n_cut"], w["r_cut"], gtable, prec)
    assert abs(E2 - e["E"]) <= (tol if prec == "fp64" else 1e-6) * abs(e["E"])
    assert res2["pairs"] == e["pairs"]


def test_lattice_basis_and_rotation_invariance(V, dev, gtable):
    """The same density on the same points with the basis (a, b, c), with
    (a, a + b, c), and with the cell rotated: equal E and pair counts through the
    GPU (FP64), given the same Cartesian gradient (rotated with the cell)."""
    cell = np.array([[9.0, 0.0, 0.0], [4.5, 7.794228634059948, 0.0], [0.0, 0.0, 8.0]])
    dims = (10, 10, 8)
    n, g = _smooth(cell, dims, seed=3)
    cell2 = cell.copy()
    cell2[1] = cell[0] + cell[1]
    i = np.arange(dims[0])[:, None]
    j = np.arange(dims[1])[None, :]
    src = (i + j) % dims[0]
    n2, g2 = n[src, j, :], g[:, src, j, :]
    th = 0.7
    R = np.array([[np.cos(th), -np.sin(th), 0.0], [np.sin(th), np.cos(th), 0.0], [0.0, 0.0, 1.0]])
    cellR = cell @ R.T
    gR = np.einsum("ck,k...->c...", R, g)
    out = []
    for c, nn, gg in ((cell, n, g), (cell2, n2, g2), (cellR, n, gR)):
        E, r = V.energy(_t(nn, dev), c, (1, 1, 0), 1e-3, 7.0, gtable, "fp64", grad=_t(gg, dev))
        out.append((E, r["pairs"]))
    assert out[0][1] == out[1][1] == out[2][1] > 0
    for E, _ in out[1:]:
        assert abs(E - out[0][0]) <= 1e-12 * abs(out[0][0])


def test_hex_monolayer_full_size(V, dev, gtable, oracle_mod, oracle_spline):
    """48x48x120 hexagonal cell at the bench's launch configuration: FP32 against
    FP64 E, and sampled v against the oracle (v at points from A, U of their
    stencil neighbourhoods)."""
    from paper_0810_2273_gb300 import inputs
    w = inputs.xe_monolayer_hex()
    cell = w["cell"]
    n = _t(w["density"], dev)
    a = (cell, w["periodic"], w["n_cut"], w["r_cut"], gtable)
    E32, v32, r32 = V.potential(n, *a, precision="fp32")
    E64, v64, r64 = V.potential(n, *a, precision="fp64")
    assert r32["pairs"] == r64["pairs"] > 0
    assert abs(E32 - E64) <= 1e-6 * abs(E64)
    v32, v64 = v32.cpu().numpy().ravel(), v64.cpu().numpy().ravel()
    vmax = np.max(np.abs(v64))
    assert np.max(np.abs(v32 - v64)) <= 1e-5 * vmax
    P = oracle_mod.Problem(w["density"], None, w["periodic"], w["n_cut"], w["r_cut"], oracle_spline, cell=cell)
    rng = np.random.default_rng(4)
    flat = w["density"].ravel()
    pts = rng.choice(np.nonzero(flat >= 1e-3)[0], 3, replace=False)
    vo = P.potential_at(pts)
    assert np.max(np.abs(v64[pts] - vo)) <= 1e-10 * vmax


def test_hex_semilocal(V, dev, oracle_mod):
    from paper_0810_2273_gb300 import inputs
    w = inputs.xe_monolayer_hex((24, 24, 60))
    ref = oracle_mod.semilocal(w["density"], None, cell=w["cell"])
    got = V.semilocal(_t(w["density"], dev), w["cell"], w["periodic"])
    for k in ("Ex_lda", "Ec_lda", "Ex_pbe", "Ec_pbe", "Ex_revpbe"):
        assert abs(got[k] - ref[k]) <= 1e-12 * abs(ref[k]), k
    assert got["n_points"] == ref["n_points"]


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_many_images_skewed_potential(V, dev, gtable, oracle_mod, oracle_spline, prec, tol):
    """A small, strongly skewed cell periodic along all axes with a cutoff of about
    twice the cell: more than 32 candidate images per tile pair, so the image
    lists are processed in chunks; energy, v and U against the oracle."""
    rng = np.random.default_rng(12)
    cell = np.array([[4.0, 0.0, 0.0], [2.6, 3.3, 0.0], [0.5, -0.7, 4.4]])
    n = 10 ** rng.uniform(-2.5, -0.5, size=(6, 7, 8))
    P = oracle_mod.Problem(n, None, (1, 1, 1), 5e-3, 8.5, oracle_spline, cell=cell)
    e = P.energy()
    vo = P.potential(e["A"], e["U"])
    E, v, res, A, U = V.potential(_t(n, dev), cell, (1, 1, 1), 5e-3, 8.5, gtable, prec, want_AU=True)
    assert res["pairs"] == e["pairs"]
    assert abs(E - e["E"]) <= (tol if prec == "fp64" else 1e-6) * abs(e["E"])
    assert np.max(np.abs(v.cpu().numpy() - vo)) <= tol * np.max(np.abs(vo))
    flat = n.ravel() >= 5e-3
    assert np.max(np.abs(U.cpu().numpy().ravel()[flat] - e["U"])) <= tol * np.max(np.abs(e["U"]))
