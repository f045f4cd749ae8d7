"""Failure detection on the GPU without a GPU fault: the library's host-side
fault injection (an allocation that fails, a work-loop cap that trips the
persistent kernel's iteration guard) and non-finite inputs return their status
codes, and the next ordinary call gives the same result as before."""
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
def setup(V, oracle_table):
    import torch
    from paper_0810_2273_gb300 import inputs
    T = V.Table.from_nodes(oracle_table, 30.0)
    w = inputs.xe_monolayer((12, 21, 30))
    n = torch.from_numpy(w["density"]).to("cuda:0")
    args = (w["lengths"], w["periodic"], w["n_cut"], w["r_cut"], T)
    E0, r0 = V.energy(n, *args, precision="fp32")
    return n, args, E0, r0


def test_allocation_failure_hook(V, setup, monkeypatch):
    n, args, E0, r0 = setup
    monkeypatch.setenv("VDWDF_FAIL_ALLOC", "1")
    for call in (lambda: V.energy(n, *args), lambda: V.potential(n, *args),
                 lambda: V.semilocal(n, args[0], args[1]),
                 lambda: V.far_tail(n, args[0], args[1], args[2], args[3])):
        with pytest.raises(V.VdwdfError) as e:
            call()
        assert e.value.status == -4  # VDWDF_EALLOC
    monkeypatch.delenv("VDWDF_FAIL_ALLOC")
    E, r = V.energy(n, *args, precision="fp32")
    assert E == E0 and r["pairs"] == r0["pairs"]


def test_work_loop_cap_returns_timeout(V, setup, monkeypatch):
    """A cap of one work item per CTA stops the persistent kernel early through
    its bounded loop (no spin, no fault): VDWDF_ETIMEOUT, in both modes."""
    n, args, E0, r0 = setup
    monkeypatch.setenv("VDWDF_MAX_ITERS", "1")
    for prec in ("fp32", "fp64"):
        with pytest.raises(V.VdwdfError) as e:
            V.energy(n, *args, precision=prec)
        assert e.value.status == -5  # VDWDF_ETIMEOUT
        with pytest.raises(V.VdwdfError) as e:
            V.potential(n, *args, precision=prec)
        assert e.value.status == -5
    monkeypatch.delenv("VDWDF_MAX_ITERS")
    E, r = V.energy(n, *args, precision="fp32")
    assert E == E0 and r["pairs"] == r0["pairs"]


def test_nonfinite_density_is_rejected(V, setup):
    import torch
    n, args, E0, r0 = setup
    bad = n.clone()
    bad[6, 10, 15] = float("inf")
    with pytest.raises(V.VdwdfError) as e:
        V.energy(bad, *args)
    assert e.value.status == -1  # VDWDF_EINVAL
    with pytest.raises(V.VdwdfError) as e:
        V.far_tail(bad, args[0], args[1], args[2], args[3])
    assert e.value.status == -1
    bad = n.clone()
    idx = torch.nonzero(n >= args[2])[0]
    bad[tuple(idx.tolist())] = float("nan")
    bad[(idx[0] + 1) % n.shape[0], idx[1], idx[2]] = float("nan")
    with pytest.raises(V.VdwdfError) as e:
        V.potential(bad, *args)
    assert e.value.status == -1
    E, r = V.energy(n, *args, precision="fp32")
    assert E == E0
