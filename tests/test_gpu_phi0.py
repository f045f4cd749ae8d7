"""The voxel-averaged diagonal (reading of the paper's phi0 step) through the C
ABI against the oracle: phi0(q) for box, skewed and hexagonal voxels, and the
diagonal energy of small grids.  Tolerance: the two sides use different graded
tensor rules whose difference is below 2e-5 |phi0| + 2e-8 (the kinks of the
integrand at q s = D_1 and Dmax are not aligned with either rule)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

VOXELS = {
    "box": np.diag([0.35, 0.30, 0.28]),
    "skew": np.array([[0.34, 0.0, 0.0], [0.17, 0.296, 0.0], [0.02, -0.03, 0.33]]),
    "hex": np.array([[16.4, 0, 0], [8.2, 14.2028166, 0], [0, 0, 40.0]]) / np.array([[48.0], [48.0], [120.0]]),
}


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


@pytest.mark.parametrize("name", list(VOXELS))
def test_phi0_matches_oracle(V, dev, gtable, oracle_spline, name):
    vox = VOXELS[name]
    q = np.array([0.02, 0.1, 0.3, 0.8, 2.0, 5.0, 12.0, 40.0])
    ref = oracle_spline.phi0(vox, q, 10, 12)
    got = V.phi0_eval(gtable, vox, _t(q, dev)).cpu().numpy()
    assert np.all(np.abs(got - ref) <= 2e-5 * np.abs(ref) + 2e-8), (got, ref)


@pytest.mark.parametrize("name,dims,n_cut,cell", [
    ("kr_dimer", None, 0.02, None),
    ("xe_monolayer_hex", (12, 12, 30), 0.01, "cell"),
])
def test_diag_voxel_matches_oracle(V, dev, gtable, oracle_mod, oracle_spline, name, dims, n_cut, cell):
    """The diagonal energy from the GPU's phi0 table (interpolated in ln q) against
    the oracle's per-point quadrature, and the table self term against the pair
    sum's own E_diag."""
    from paper_0810_2273_gb300 import inputs
    w = getattr(inputs, name)(dims) if dims else getattr(inputs, name)()
    c = w["cell"] if cell else None
    P = oracle_mod.Problem(w["density"], None if c is not None else w["lengths"], w["periodic"], n_cut,
                           w["r_cut"], oracle_spline, cell=c)
    ref = P.diag_voxel(7, 8)
    n = _t(w["density"], dev)
    geom = c if c is not None else w["lengths"]
    got = V.diag_voxel(n, geom, w["periodic"], n_cut, gtable)
    assert got["n_active"] == P.n_active > 0
    assert abs(got["E_diag_voxel"] - ref["E_diag_voxel"]) <= 2e-5 * abs(ref["E_diag_voxel"])
    assert abs(got["E_diag_table"] - ref["E_diag_table"]) <= 1e-12 * abs(ref["E_diag_table"])
    E, res = V.energy(n, geom, w["periodic"], n_cut, w["r_cut"], gtable, "fp64")
    assert abs(res["E_diag"] - got["E_diag_table"]) <= 1e-12 * abs(got["E_diag_table"])
    # more table points move the result by no more than the interpolation error
    fine = V.diag_voxel(n, geom, w["periodic"], n_cut, gtable, nphi0=400)
    assert abs(fine["E_diag_voxel"] - got["E_diag_voxel"]) <= 1e-6 * abs(got["E_diag_voxel"])


def test_diag_voxel_potential_is_derivative(V, dev, gtable, oracle_mod, oracle_spline):
    """dv = (1/dV) d(E_diag_voxel - E_diag_table)/dn at points with n >= 2 n_cut (mask
    unchanged) whose stencil neighbourhoods are not at the q0 extremes (table range
    unchanged): against central differences of the GPU's own FP64 sums, and at two
    points against central differences of the oracle's diagonal."""
    import torch
    from paper_0810_2273_gb300 import inputs
    w = inputs.xe_monolayer_hex((12, 12, 30))
    cell, n_cut = w["cell"], 0.01
    n = w["density"].copy()
    res, dv = V.diag_voxel_potential(_t(n, dev), cell, w["periodic"], n_cut, gtable)
    dv = dv.cpu().numpy()
    dV = abs(np.linalg.det(cell)) / n.size
    q0 = V.q0(_t(n, dev), cell)[0].cpu().numpy()
    act = n >= n_cut
    qa = q0[act]
    lo, hi = np.sort(qa)[3], np.sort(qa)[-4]
    rng = np.random.default_rng(3)
    cand = [m for m in rng.permutation(n.size) if n.flat[m] >= 2 * n_cut]
    picked = []
    for m in cand:
        i = np.unravel_index(m, n.shape)
        nb = [tuple((np.array(i) + d) % np.array(n.shape)) for d in
              [np.eye(3, dtype=int)[a] * s for a in range(3) for s in (-2, -1, 0, 1, 2)]]
        if all(lo < q0[j] < hi for j in nb):
            picked.append(m)
        if len(picked) == 4:
            break
    vmax = np.max(np.abs(dv))

    def e_diag(nn):
        r = V.diag_voxel(_t(nn, dev), cell, w["periodic"], n_cut, gtable)
        return r["E_diag_voxel"] - r["E_diag_table"]

    for m in picked:
        h = 1e-4 * n.flat[m]
        npl, nmi = n.copy(), n.copy()
        npl.flat[m] += h
        nmi.flat[m] -= h
        fd = (e_diag(npl) - e_diag(nmi)) / (2 * h * dV)
        assert abs(fd - dv.flat[m]) <= 1e-6 * vmax + 1e-8 * abs(dv.flat[m]), (m, fd, dv.flat[m])
    for m in picked[:2]:
        h = 1e-4 * n.flat[m]
        vals = []
        for s in (1, -1):
            nn = n.copy()
            nn.flat[m] += s * h
            P = oracle_mod.Problem(nn, None, w["periodic"], n_cut, w["r_cut"], oracle_spline, cell=cell)
            d = P.diag_voxel(6, 8)
            vals.append(d["E_diag_voxel"] - d["E_diag_table"])
        fd = (vals[0] - vals[1]) / (2 * h * dV)
        assert abs(fd - dv.flat[m]) <= 1e-3 * abs(dv.flat[m]) + 1e-5 * vmax, (m, fd, dv.flat[m])
