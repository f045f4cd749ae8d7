"""vdwdf_energy_noalloc, the energy with all scratch in a static device array,
against vdwdf_energy on the same inputs: the same energies and counts on two
calls in a row (the scratch is reused; what must start at zero is cleared by
each call) on orthorhombic and skewed cells and with both gradients, no change
in free device memory across calls, its refusals (grid too large, table not
yet on the device), and a call that stops at the work-loop cap followed by an
ordinary one.  Collected last, so it also runs
after every other GPU test."""
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


def _cases():
    from paper_0810_2273_gb300 import inputs
    curve = inputs.binding_curve()
    hexa = inputs.xe_monolayer_hex((16, 16, 40))      # skewed cell: Cartesian tile boxes
    spec = inputs.xe_monolayer((12, 21, 30))
    spec["name"] = spec["name"] + " (FFT gradient)"
    spec["gradient"] = "spectral"                       # gradient and coefficients carved too
    return [inputs.kr_dimer(), inputs.xe_monolayer((12, 21, 30)), curve[0], curve[15],  # 64x32x32
            hexa, spec]


def _geom(w):
    return w["cell"] if "cell" in w else w["lengths"]


def test_noalloc_matches_energy_twice(V, dev, oracle_table):
    import torch
    T = V.Table.from_nodes(oracle_table, 30.0)
    for w in _cases():
        assert w["density"].size <= 65536
        n = _t(w["density"], dev)
        args = (_geom(w), w["periodic"], w["n_cut"], w["r_cut"], T)
        kind = w.get("gradient", "fd")
        for prec in ("fp64", "fp32"):
            E_ref, r_ref = V.energy(n, *args, precision=prec, gradient=kind)  # also puts T on the device
            E0, _ = V.energy_noalloc(n, *args, precision=prec, gradient=kind)  # first call: set-up
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info(dev)[0]
            for call in range(2):
                E, r = V.energy_noalloc(n, *args, precision=prec, gradient=kind)
                assert abs(E - E_ref) <= 1e-13 * abs(E_ref), (w["name"], prec, call, E, E_ref)
                assert abs(r["E_diag"] - r_ref["E_diag"]) <= 1e-12 * abs(r_ref["E_diag"])
                for k in ("n_active", "pairs", "pairs_evaluated", "n_clamped"):
                    assert r[k] == r_ref[k], (w["name"], prec, call, k, r[k], r_ref[k])
                assert r["q0_min"] == r_ref["q0_min"] and r["q0_max"] == r_ref["q0_max"]
                assert r["ms_pairs"] == 0.0 and r["launches"] > 0
            torch.cuda.synchronize()
            assert torch.cuda.mem_get_info(dev)[0] == free0, (w["name"], prec)
            assert abs(E0 - E_ref) <= 1e-13 * abs(E_ref)


def test_noalloc_refusals(V, dev, oracle_table):
    from paper_0810_2273_gb300 import inputs
    w = inputs.kr_dimer()
    fresh = V.Table.from_nodes(oracle_table, 30.0)  # never used on the device
    n = _t(w["density"], dev)
    with pytest.raises(V.VdwdfError) as e:
        V.energy_noalloc(n, w["lengths"], w["periodic"], w["n_cut"], w["r_cut"], fresh)
    assert e.value.status == -6  # VDWDF_ENOTABLE: making the table resident would allocate
    big = _t(np.full((64, 64, 17), 1e-3), dev)
    with pytest.raises(V.VdwdfError) as e:
        V.energy_noalloc(big, (20.0, 20.0, 6.0), (0, 0, 0), 1e-6, 0.0, fresh)
    assert e.value.status == -2  # VDWDF_EUNSUPPORTED: more than 65536 grid points


def test_noalloc_timeout_then_ordinary_call(V, dev, oracle_table, monkeypatch):
    """A work-loop cap of one item per CTA (host-side fault injection) makes the
    call return VDWDF_ETIMEOUT after its kernels ran on the shared array; the call
    has finished with the array when it returns, and the next call gives the same
    energy as vdwdf_energy."""
    from paper_0810_2273_gb300 import inputs
    T = V.Table.from_nodes(oracle_table, 30.0)
    w = inputs.xe_monolayer((12, 21, 30))
    n = _t(w["density"], dev)
    args = (w["lengths"], w["periodic"], w["n_cut"], w["r_cut"], T)
    for prec in ("fp32", "fp64"):
        E_ref, r_ref = V.energy(n, *args, precision=prec)
        monkeypatch.setenv("VDWDF_MAX_ITERS", "1")
        with pytest.raises(V.VdwdfError) as e:
            V.energy_noalloc(n, *args, precision=prec)
        assert e.value.status == -5  # VDWDF_ETIMEOUT
        monkeypatch.delenv("VDWDF_MAX_ITERS")
        E, r = V.energy_noalloc(n, *args, precision=prec)
        assert abs(E - E_ref) <= 1e-13 * abs(E_ref), (prec, E, E_ref)
        assert r["pairs"] == r_ref["pairs"]
