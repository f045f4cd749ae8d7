"""The C-ABI library: loads without a GPU, exports what include/vdwdf.h declares,
rejects bad arguments on the host, and its host-side kernel table agrees with
the oracle's independent quadrature of Dion eq. (14)."""
import ctypes
import os
import re

import numpy as np
import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "vdwdf.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    return sorted(set(re.findall(r"\b(vdwdf_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def native():
    from paper_0810_2273_gb300 import _native, build
    build.build()
    return _native


def test_library_exports_every_declared_symbol(native):
    lib = native.load()
    names = _declared_functions()
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(native.PROTOTYPES), set(names) ^ set(native.PROTOTYPES)
    assert lib.vdwdf_version() == 10000
    for s in (0, -1, -2, -3, -4, -5, -6):
        assert lib.vdwdf_strerror(s)


def test_struct_layouts_match_header(native, tmp_path):
    """ctypes structs vs the C compiler's layout of include/vdwdf.h."""
    import subprocess
    fields = {"vdwdf_grid": native.vdwdf_grid, "vdwdf_result": native.vdwdf_result,
              "vdwdf_tuning": native.vdwdf_tuning, "vdwdf_semilocal_result": native.vdwdf_semilocal_result,
              "vdwdf_diag_result": native.vdwdf_diag_result, "vdwdf_tail_result": native.vdwdf_tail_result}
    src = ["#include <stdio.h>", "#include <stddef.h>", '#include "vdwdf.h"', "int main(void) {"]
    for s, cls in fields.items():
        src.append('printf("%s size %%zu\\n", sizeof(%s));' % (s, s))
        for f, _ in cls._fields_:
            src.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (s, f, s, f))
    src.append("return 0; }")
    c = os.path.join(tmp_path, "layout.c")
    exe = os.path.join(tmp_path, "layout")
    open(c, "w").write("\n".join(src))
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    for line in filter(None, out):
        s, f, v = line.split()
        got = ctypes.sizeof(fields[s]) if f == "size" else getattr(fields[s], f).offset
        assert got == int(v), line


def test_host_side_argument_errors(native):
    """Invalid inputs are rejected before any device work (no GPU needed)."""
    lib = native.load()
    h = ctypes.c_void_p()
    assert lib.vdwdf_table_build(2, 30.0, 200, 1, None, ctypes.byref(h)) == -1
    assert lib.vdwdf_table_build(400, -1.0, 200, 1, None, ctypes.byref(h)) == -1
    assert lib.vdwdf_table_build(400, 30.0, 200, 7, None, ctypes.byref(h)) == -1
    nodes = np.zeros((4, 4))
    nodes[1, 1] = np.inf
    assert lib.vdwdf_table_from_nodes(4, 30.0, 4, nodes.ctypes.data_as(ctypes.c_void_p), ctypes.byref(h)) == -1
    g = native.vdwdf_grid()
    for a in range(3):
        g.cell[a][a] = 10.0
        g.n[a] = 8
    res = native.vdwdf_result()
    # null density pointer
    assert lib.vdwdf_energy(ctypes.byref(g), None, None, 1e-6, 0.0, ctypes.c_void_p(1), 0, None,
                            ctypes.byref(res), None) == -1
    # no table
    assert lib.vdwdf_energy(ctypes.byref(g), ctypes.c_void_p(8), None, 1e-6, 0.0, None, 0, None,
                            ctypes.byref(res), None) == -6
    # periodic without a cutoff
    g.periodic[0] = 1
    assert lib.vdwdf_energy(ctypes.byref(g), ctypes.c_void_p(8), None, 1e-6, 0.0, ctypes.c_void_p(1), 0,
                            None, ctypes.byref(res), None) == -1
    g.periodic[0] = 0
    # more than 64 image shifts along a periodic axis (r_cut of 70 cell lengths)
    g.periodic[0] = 1
    assert lib.vdwdf_energy(ctypes.byref(g), ctypes.c_void_p(8), None, 1e-6, 700.0, ctypes.c_void_p(1), 0,
                            None, ctypes.byref(res), None) == -1
    g.periodic[0] = 0
    # non-positive density cutoff, bad precision
    assert lib.vdwdf_energy(ctypes.byref(g), ctypes.c_void_p(8), None, 0.0, 0.0, ctypes.c_void_p(1), 0,
                            None, ctypes.byref(res), None) == -1
    assert lib.vdwdf_energy(ctypes.byref(g), ctypes.c_void_p(8), None, 1e-6, 0.0, ctypes.c_void_p(1), 5,
                            None, ctypes.byref(res), None) == -1
    # singular cell (two parallel lattice vectors)
    g.cell[1][0], g.cell[1][1] = 10.0, 0.0
    assert lib.vdwdf_energy(ctypes.byref(g), ctypes.c_void_p(8), None, 1e-6, 0.0, ctypes.c_void_p(1), 0,
                            None, ctypes.byref(res), None) == -1
    g.cell[1][0], g.cell[1][1] = 0.0, 10.0
    # batched: bad count (at least 1, at most 4096 instances)
    assert lib.vdwdf_energy_batched(0, None, None, 1e-6, 0.0, ctypes.c_void_p(1), 0, None, None, None,
                                    None) == -1
    gs = (native.vdwdf_grid * 4097)(*([g] * 4097))
    ptrs = (ctypes.c_void_p * 4097)(*([8] * 4097))
    E_out = (ctypes.c_double * 4097)()
    assert lib.vdwdf_energy_batched(4097, gs, ptrs, 1e-6, 0.0, ctypes.c_void_p(1), 0, None, E_out, None,
                                    None) == -1
    # semilocal energies: null density or result, singular cell
    sres = native.vdwdf_semilocal_result()
    assert lib.vdwdf_semilocal(ctypes.byref(g), None, None, ctypes.byref(sres), None) == -1
    assert lib.vdwdf_semilocal(ctypes.byref(g), ctypes.c_void_p(8), None, None, None) == -1
    g.cell[2][0], g.cell[2][2] = 10.0, 0.0
    assert lib.vdwdf_semilocal(ctypes.byref(g), ctypes.c_void_p(8), None, ctypes.byref(sres), None) == -1
    g.cell[2][0], g.cell[2][2] = 0.0, 10.0
    # voxel diagonal: no table, bad table size, null result
    dres = native.vdwdf_diag_result()
    assert lib.vdwdf_diag_voxel(ctypes.byref(g), ctypes.c_void_p(8), None, 1e-6, None, 0, ctypes.byref(dres),
                                None) == -6
    assert lib.vdwdf_diag_voxel(ctypes.byref(g), ctypes.c_void_p(8), None, 1e-6, ctypes.c_void_p(1), 2,
                                ctypes.byref(dres), None) == -1
    assert lib.vdwdf_diag_voxel(ctypes.byref(g), ctypes.c_void_p(8), None, 1e-6, ctypes.c_void_p(1), 0, None,
                                None) == -1
    vox = (ctypes.c_double * 9)(*([0.3] * 9))
    assert lib.vdwdf_phi0_eval(None, vox, 1, ctypes.c_void_p(8), ctypes.c_void_p(8), None) == -6
    # gradient kind: only finite differences (0) and spectral (1); spectral axes up to 12800
    g.gradient = 2
    assert lib.vdwdf_energy(ctypes.byref(g), ctypes.c_void_p(8), None, 1e-6, 0.0, ctypes.c_void_p(1), 0, None,
                            ctypes.byref(res), None) == -1
    g.gradient = 1
    g.n[2] = 12801
    assert lib.vdwdf_gradient(ctypes.byref(g), ctypes.c_void_p(8), ctypes.c_void_p(8), None) == -2
    g.n[2] = 8
    assert lib.vdwdf_gradient(ctypes.byref(g), None, ctypes.c_void_p(8), None) == -1
    assert lib.vdwdf_gradient(ctypes.byref(g), ctypes.c_void_p(8), None, None) == -1
    g.gradient = 0
    # launch shapes outside the documented values, and thread counts without a skewed kernel
    tu = native.vdwdf_tuning()
    for field, value in (("threads", 300), ("items_per_sm", -1), ("smem_rows", -2), ("smem_row0", -5)):
        tu = native.vdwdf_tuning()
        setattr(tu, field, value)
        assert lib.vdwdf_energy(ctypes.byref(g), ctypes.c_void_p(8), None, 1e-6, 0.0, ctypes.c_void_p(1), 0,
                                ctypes.byref(tu), ctypes.byref(res), None) == -1, field
    tu = native.vdwdf_tuning()
    tu.threads = 1024
    g.cell[1][0] = 5.0  # skewed
    assert lib.vdwdf_energy(ctypes.byref(g), ctypes.c_void_p(8), None, 1e-6, 0.0, ctypes.c_void_p(1), 0,
                            ctypes.byref(tu), ctypes.byref(res), None) == -2
    tu.threads = 448
    g.cell[1][0] = 0.0
    # no-allocation energy: a grid larger than its static scratch holds is refused
    g.cell[0][1] = 0.0
    g.n[0], g.n[1], g.n[2] = 64, 64, 17
    assert lib.vdwdf_energy_noalloc(ctypes.byref(g), ctypes.c_void_p(8), None, 1e-6, 0.0, ctypes.c_void_p(1),
                                    0, ctypes.byref(res), None) == -2
    # lane-rate measurement: unknown kind, no output, duration outside 1..1000 ms
    rate = ctypes.c_double()
    assert lib.vdwdf_lane_rate(3, 20.0, ctypes.byref(rate), None, None) == -1
    assert lib.vdwdf_lane_rate(-1, 20.0, ctypes.byref(rate), None, None) == -1
    assert lib.vdwdf_lane_rate(0, 20.0, None, None, None) == -1
    for ms in (0.5, 1001.0, float("nan")):
        assert lib.vdwdf_lane_rate(2, ms, ctypes.byref(rate), None, None) == -1


def test_table_build_matches_oracle_quadrature(oracle_mod):
    """Library table (its own quadrature: octave panels, pi/4-aligned panels, truncation
    at 63.5 pi with an integration-by-parts tail) vs the oracle's reference quadrature
    (ratio-1.5 log panels, unit-pi panels, truncation at 255.5 pi, no tail term)."""
    from paper_0810_2273_gb300 import Table
    T = Table.build(13, 30.0, 8, 1)
    nodes = T.nodes
    D = 30.0 * np.arange(13) / 12
    dl = np.arange(8) / 8
    DD, LL = np.meshgrid(D[1:], dl, indexing="ij")
    ref = oracle_mod.phi((DD * (1 + LL)).ravel(), (DD * (1 - LL)).ravel(),
                         oracle_mod.QUAD_REFERENCE).reshape(DD.shape)
    assert np.max(np.abs(nodes[1:] - ref)) < 5e-12
    assert np.allclose(nodes[0], (4 * nodes[1] - nodes[2]) / 3, rtol=1e-15, atol=0)
    assert T.info() == (13, 30.0, 8)


def test_standard_table_at_random_nodes(oracle_mod):
    """The standard 400 x 200 build (0 <= D <= 30, quadrature level 1) against the
    oracle's reference quadrature at 240 random nodes of rows 1..399 (the spot-point
    pin of the node table, within 1e-9 of max|phi|), and its row 0 rule."""
    import os
    from paper_0810_2273_gb300 import Table
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), ".cache",
                        "vdwdf_table_400x200_D30_q1.npz")
    T = Table.load(path) if os.path.exists(path) else Table.build(400, 30.0, 200, 1)
    nodes = T.nodes
    assert nodes.shape == (400, 200)
    rng = np.random.default_rng(2024)
    k = rng.integers(1, 400, 240)
    l = rng.integers(0, 200, 240)
    D = 30.0 * k / 399
    dl = l / 200.0
    ref = oracle_mod.phi(D * (1 + dl), D * (1 - dl), oracle_mod.QUAD_REFERENCE)
    scale = np.max(np.abs(nodes))
    # the two quadratures differ by up to 2e-10 absolute, at D < 1 where the
    # integrand's switch h(a/d) sits at small a; the bound is 1e-9 max|phi|
    assert np.max(np.abs(nodes[k, l] - ref)) < 1e-9 * scale, np.max(np.abs(nodes[k, l] - ref))
    assert np.allclose(nodes[0], (4 * nodes[1] - nodes[2]) / 3, rtol=1e-15, atol=0)


def test_table_roundtrip_from_nodes(tmp_path):
    from paper_0810_2273_gb300 import Table
    rng = np.random.default_rng(0)
    nodes = rng.normal(size=(9, 6))
    T = Table.from_nodes(nodes, 12.0)
    assert np.array_equal(T.nodes, nodes)
    p = os.path.join(tmp_path, "t.npz")
    T.save(p)
    T2 = Table.load(p)
    assert np.array_equal(T2.nodes, nodes) and T2.info() == (9, 12.0, 6)


def test_total_energy_assembly():
    """Eq. 3 (host arithmetic behind the C ABI) with PBE exchange leaves E_tot^DFT - E_c^PBE + E_c^LDA + E_c^nl (the
    correction printed as the "needed number" in the paper's sample output); with
    revPBE exchange it adds E_x^revPBE - E_x^PBE on top."""
    import paper_0810_2273_gb300 as V
    semi = {"Ex_lda": -1.0, "Ec_lda": -0.30, "Ex_pbe": -1.10, "Ec_pbe": -0.20, "Ex_revpbe": -1.12}
    E = V.total_energy_nl(-50.0, semi, 0.05)
    assert E == pytest.approx(-50.0 - (-0.20) + (-0.30) + 0.05, abs=1e-15)
    Er = V.total_energy_nl(-50.0, semi, 0.05, exchange="revpbe")
    assert Er == pytest.approx(E + (-1.12) - (-1.10), abs=1e-15)
    with pytest.raises(ValueError):
        V.total_energy_nl(-50.0, semi, 0.05, exchange="lda")
    # the C entry point refuses a NULL pointer, another exchange and a non-finite sum
    import ctypes
    from paper_0810_2273_gb300 import _native
    lib = _native.load()
    s = _native.vdwdf_semilocal_result()
    out = ctypes.c_double(7.0)
    assert lib.vdwdf_total_energy_nl(-50.0, None, 0.05, 0, ctypes.byref(out)) == -1
    assert lib.vdwdf_total_energy_nl(-50.0, ctypes.byref(s), 0.05, 2, ctypes.byref(out)) == -1
    assert lib.vdwdf_total_energy_nl(float("nan"), ctypes.byref(s), 0.05, 0, ctypes.byref(out)) == -1
    assert out.value == 7.0


def test_python_grid_and_tuning_marshalling():
    """grid() carries the gradient kind and _tuning() the four launch fields, as the
    header defines them; a bad kind is refused before any library call."""
    from paper_0810_2273_gb300 import grid, _tuning, _native
    g = grid((10.0, 11.0, 12.0), (8, 9, 10), (True, False, True))
    assert g.gradient == 0 and list(g.periodic) == [1, 0, 1] and list(g.n) == [8, 9, 10]
    assert g.cell[0][0] == 10.0 and g.cell[1][1] == 11.0 and g.cell[0][1] == 0.0
    gs = grid(np.diag([3.0, 4.0, 5.0]), (4, 4, 4), gradient="spectral")
    assert gs.gradient == 1 and gs.cell[2][2] == 5.0
    with pytest.raises(ValueError):
        grid((1.0, 1.0, 1.0), (2, 2, 2), gradient="fft")
    t = _tuning({"threads": 448, "items_per_sm": 256, "smem_row0": -1})._obj
    assert (t.threads, t.items_per_sm, t.smem_rows, t.smem_row0) == (448, 256, 0, -1)
    assert _tuning(None) is None
    r = _native.vdwdf_result()
    assert "smem_row0" in r.as_dict() and "pair_threads" in r.as_dict()
