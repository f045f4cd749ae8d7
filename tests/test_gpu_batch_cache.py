"""The batched path's recorded CUDA graphs are replayed only for calls that
would record the same graph: each case below changes one thing the recording
bakes in (the off-diagonal cell, the gradient kind, the table behind a handle,
more plans than the cache holds) and checks the batched energies against
single-instance calls of vdwdf_energy on the same inputs."""
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


def _t(a, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(dev)


def _blob(dims, lengths, seed):
    from paper_0810_2273_gb300 import inputs
    rng = np.random.default_rng(seed)
    atoms = [(rng.uniform(0.3, 0.7, 3) * np.asarray(lengths), inputs.rare_gas_shells()) for _ in range(2)]
    return inputs.density(dims, lengths, atoms)


def _single(V, n, cell, periodic, r_cut, table, prec, gradient="fd"):
    return V.energy(n, cell, periodic, 1e-6, r_cut, table, prec, gradient=gradient)[0]


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-6)])
def test_skewed_cells_sharing_a_diagonal(V, dev, oracle_table, prec, tol):
    """Two cells with the same diagonal and opposite off-diagonal entries: the
    second batched call must not replay the graph recorded for the first."""
    table = V.Table.from_nodes(oracle_table, 30.0)
    dims = (16, 16, 12)
    n = _t(_blob(dims, (9.0, 9.0, 7.0), 1), dev)
    per = (1, 1, 0)
    cells = [np.array([[9.0, 0, 0], [s * 4.5, 9.0, 0], [0, 0, 7.0]]) for s in (1.0, -1.0)]
    for cell in cells:
        Eb, _ = V.energy_batched([n], [cell], [per], 1e-6, 8.0, table, prec)
        Es = _single(V, n, cell, per, 8.0, table, prec)
        assert abs(Eb[0] - Es) <= tol * abs(Es), (cell, Eb[0], Es)
    e0 = _single(V, n, cells[0], per, 8.0, table, prec)
    e1 = _single(V, n, cells[1], per, 8.0, table, prec)
    assert abs(e0 - e1) > 1e-4 * abs(e0)   # the two cells really differ
    table.free()


def test_gradient_kind_switch(V, dev, oracle_table):
    """The same tensors with the finite-difference, then the FFT gradient."""
    table = V.Table.from_nodes(oracle_table, 30.0)
    dims = (20, 16, 16)
    L = (10.0, 8.0, 8.0)
    ns = [_t(_blob(dims, L, s), dev) for s in (2, 3)]
    for kind in ("fd", "spectral", "fd"):
        Eb, _ = V.energy_batched(ns, [L, L], [(0, 0, 0)] * 2, 1e-6, 0.0, table, "fp64", gradient=kind)
        for k in range(2):
            Es = _single(V, ns[k], L, (0, 0, 0), 0.0, table, "fp64", gradient=kind)
            assert abs(Eb[k] - Es) <= 1e-10 * abs(Es), (kind, k, Eb[k], Es)
    table.free()


def test_table_freed_and_replaced(V, dev, oracle_table):
    """A graph recorded with one table is dropped when that table is freed: a new
    table (its handle may reuse the freed address) gives its own energies."""
    dims = (16, 12, 12)
    L = (10.0, 8.0, 8.0)
    n = _t(_blob(dims, L, 4), dev)
    scales = (1.0, 1.5, 0.5)
    for sc in scales:
        table = V.Table.from_nodes(oracle_table * sc, 30.0)
        Eb, _ = V.energy_batched([n], [L], [(0, 0, 0)], 1e-6, 0.0, table, "fp64")
        Es = _single(V, n, L, (0, 0, 0), 0.0, table, "fp64")
        assert abs(Eb[0] - Es) <= 1e-10 * abs(Es), (sc, Eb[0], Es)
        table.free()


def test_more_plans_than_the_cache_holds(V, dev, oracle_table):
    """Twelve different inputs (more than the eight recorded graphs kept), then
    the first ones again: evicted plans are recorded anew, kept ones replayed."""
    table = V.Table.from_nodes(oracle_table, 30.0)
    dims = (12, 12, 12)
    L = (8.0, 8.0, 8.0)
    ns = [_t(_blob(dims, L, 10 + s), dev) for s in range(12)]
    ref = [_single(V, x, L, (0, 0, 0), 0.0, table, "fp64") for x in ns]
    for rounds in range(2):
        for k, x in enumerate(ns):
            Eb, _ = V.energy_batched([x], [L], [(0, 0, 0)], 1e-6, 0.0, table, "fp64")
            assert abs(Eb[0] - ref[k]) <= 1e-10 * abs(ref[k]), (rounds, k)
    table.free()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-6)])
def test_more_instances_than_one_launch_holds(V, dev, oracle_table, prec, tol):
    """Thirty uneven densities (one pair launch holds 24, so two launches in one
    graph), among them one with no point above the cutoff and one with a single
    point, against one-at-a-time calls; then the graph's replay with new values."""
    table = V.Table.from_nodes(oracle_table, 30.0)
    rng = np.random.default_rng(30)
    shapes = [tuple(int(x) for x in rng.integers(8, 15, 3)) for _ in range(30)]
    Ls = [tuple(0.55 * d for d in s) for s in shapes]
    hosts = [_blob(s, L, 40 + k) for k, (s, L) in enumerate(zip(shapes, Ls))]
    hosts[7] = np.full(shapes[7], 1e-8)              # nothing above the cutoff
    hosts[19] = np.full(shapes[19], 1e-8)
    hosts[19][3, 4, 5] = 0.3                         # a single active point
    ns = [_t(h, dev) for h in hosts]
    per = [(0, 0, 0)] * 30
    for scale in (1.0, 1.25):
        if scale != 1.0:
            for x in ns:
                x.mul_(scale)                        # same tensors: the recorded graph replays
        Eb, _ = V.energy_batched(ns, Ls, per, 1e-6, 0.0, table, prec)
        for k in range(30):
            Es, res = V.energy(ns[k], Ls[k], per[k], 1e-6, 0.0, table, prec)
            if k == 7:
                assert Eb[k] == 0.0 and Es == 0.0 and res["n_active"] == 0
                continue
            if k == 19:
                assert res["n_active"] == 1 and res["pairs"] == 0
            assert abs(Eb[k] - Es) <= tol * abs(Es), (scale, k, Eb[k], Es)
    table.free()
