"""GB300-native vdW-DF nonlocal correlation: the hot path of JuNoLo
(Lazic et al., arXiv 0810.2273) as a CUDA library for sm_103a.

    E_c^nl = 1/2 sum_i sum_j n_i phi(q0_i r_ij, q0_j r_ij) n_j dV^2      (paper eq. 2)

over grid points above a density cutoff, with periodic images under a pair
cutoff, and its potential v = dE/dn / dV.  This module is a thin binding of
``libvdwdf`` (C ABI in include/vdwdf.h): it passes torch CUDA tensors'
device pointers and the current CUDA stream; every step runs in the
library's kernels.  Tensors: FP64, contiguous, shape (n0, n1, n2).
"""
import ctypes

import numpy as np

from . import _native
from ._native import (VDWDF_FP32, VDWDF_FP64, VdwdfError, vdwdf_diag_result, vdwdf_grid, vdwdf_result,
                      vdwdf_semilocal_result, vdwdf_tuning)

__all__ = ["Table", "grid", "energy", "energy_noalloc", "potential", "energy_batched", "q0", "kernel_eval",
           "semilocal", "total_energy_nl", "far_tail", "phi0_eval", "diag_voxel", "diag_voxel_potential",
           "autotune", "launch_count", "lane_rate", "NonlocalEnergy", "nonlocal_energy", "VdwdfError",
           "VDWDF_FP32", "VDWDF_FP64"]


def _prec(p):
    if p in (VDWDF_FP32, "fp32", "float32"):
        return VDWDF_FP32
    if p in (VDWDF_FP64, "fp64", "float64"):
        return VDWDF_FP64
    raise ValueError("precision must be 'fp32' or 'fp64'")


class Table:
    """Kernel table phi(D_k, delta_l), D_k = Dmax k/(nD-1), delta_l = l/ndelta, with its
    bicubic spline (library-owned; paper section 2 and section 7)."""

    def __init__(self, handle):
        self._h = ctypes.c_void_p(handle)

    @classmethod
    def build(cls, nD=400, Dmax=30.0, ndelta=200, quad_level=1):
        """Tabulate Dion's eq. (14) by double quadrature on the host (FP64, OpenMP)."""
        lib = _native.load()
        h = ctypes.c_void_p()
        _native.check(lib.vdwdf_table_build(nD, float(Dmax), ndelta, quad_level, None, ctypes.byref(h)),
                      "vdwdf_table_build")
        return cls(h.value)

    @classmethod
    def from_nodes(cls, nodes, Dmax=30.0):
        lib = _native.load()
        a = np.ascontiguousarray(nodes, dtype=np.float64)
        nD, nd = a.shape
        h = ctypes.c_void_p()
        _native.check(lib.vdwdf_table_from_nodes(nD, float(Dmax), nd, a.ctypes.data_as(ctypes.c_void_p),
                                                 ctypes.byref(h)), "vdwdf_table_from_nodes")
        return cls(h.value)

    @classmethod
    def load(cls, path):
        """Load nodes saved by ``save`` (the kernel-file path of paper section 5)."""
        with np.load(path) as z:
            return cls.from_nodes(z["nodes"], float(z["Dmax"]))

    def save(self, path):
        np.savez(path, nodes=self.nodes, Dmax=self.info()[1])

    def info(self):
        lib = _native.load()
        nD, nd = ctypes.c_int(), ctypes.c_int()
        Dm = ctypes.c_double()
        _native.check(lib.vdwdf_table_info(self._h, ctypes.byref(nD), ctypes.byref(Dm), ctypes.byref(nd)),
                      "vdwdf_table_info")
        return nD.value, Dm.value, nd.value

    @property
    def nodes(self):
        nD, _, nd = self.info()
        out = np.zeros((nD, nd))
        _native.check(_native.load().vdwdf_table_nodes(self._h, out.ctypes.data_as(ctypes.c_void_p)),
                      "vdwdf_table_nodes")
        return out

    @property
    def handle(self):
        return self._h

    def free(self):
        if self._h is not None and self._h.value:
            _native.load().vdwdf_table_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


_GRADIENTS = {"fd": 0, "spectral": 1}


def grid(lengths, dims, periodic=(False, False, False), gradient="fd"):
    """vdwdf_grid for an orthorhombic cell lengths[0] x lengths[1] x lengths[2] bohr, or,
    when ``lengths`` is 3x3, for the general cell whose rows are the lattice vectors.
    gradient: "fd" (4th-order finite differences) or "spectral" (the band-limited,
    FFT derivative), the library's gradient wherever it computes one."""
    if gradient not in _GRADIENTS:
        raise ValueError("gradient: 'fd' or 'spectral'")
    g = vdwdf_grid()
    g.gradient = _GRADIENTS[gradient]
    cell = np.asarray(lengths, dtype=np.float64)
    for a in range(3):
        for b in range(3):
            if cell.shape == (3, 3):
                g.cell[a][b] = float(cell[a, b])
            else:
                g.cell[a][b] = float(cell[a]) if a == b else 0.0
        g.n[a] = int(dims[a])
        g.periodic[a] = 1 if periodic[a] else 0
    return g


def _cell_volume(lengths):
    """Volume of the orthorhombic cell lengths, or of the general cell (3x3 rows)."""
    cell = np.asarray(lengths, dtype=np.float64)
    return abs(float(np.linalg.det(cell))) if cell.shape == (3, 3) else float(np.prod(cell))


def _torch():
    import torch
    return torch


def _check_tensor(t, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError("%s must be contiguous float64" % name)


def _stream(t):
    torch = _torch()
    return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)


def _tuning(tu):
    if tu is None:
        return None
    if isinstance(tu, vdwdf_tuning):
        return ctypes.byref(tu)
    t = vdwdf_tuning()
    for k in ("threads", "items_per_sm", "smem_rows", "smem_row0"):
        setattr(t, k, int(tu.get(k, 0)))
    return ctypes.byref(t)


def energy(n, lengths, periodic, n_cut, r_cut, table, precision="fp32", grad=None, tuning=None, gradient="fd"):
    """E_c^nl (Hartree) of density n on the grid; returns (E, result dict)."""
    _check_tensor(n, "n")
    if grad is not None:
        _check_tensor(grad, "grad")
    torch = _torch()
    lib = _native.load()
    g = grid(lengths, n.shape, periodic, gradient)
    res = vdwdf_result()
    with torch.cuda.device(n.device):
        st = lib.vdwdf_energy(ctypes.byref(g), ctypes.c_void_p(n.data_ptr()),
                              ctypes.c_void_p(grad.data_ptr()) if grad is not None else None,
                              float(n_cut), float(r_cut), table.handle, _prec(precision), _tuning(tuning),
                              ctypes.byref(res), _stream(n))
    _native.check(st, "vdwdf_energy")
    return res.E, res.as_dict()


def energy_noalloc(n, lengths, periodic, n_cut, r_cut, table, precision="fp32", grad=None, gradient="fd"):
    """As energy, through vdwdf_energy_noalloc: no allocation during the call (grids
    of at most 65536 points; the table must already be resident on n's device)."""
    _check_tensor(n, "n")
    if grad is not None:
        _check_tensor(grad, "grad")
    torch = _torch()
    lib = _native.load()
    g = grid(lengths, n.shape, periodic, gradient)
    res = vdwdf_result()
    with torch.cuda.device(n.device):
        st = lib.vdwdf_energy_noalloc(ctypes.byref(g), ctypes.c_void_p(n.data_ptr()),
                                      ctypes.c_void_p(grad.data_ptr()) if grad is not None else None,
                                      float(n_cut), float(r_cut), table.handle, _prec(precision),
                                      ctypes.byref(res), _stream(n))
    _native.check(st, "vdwdf_energy_noalloc")
    return res.E, res.as_dict()


def semilocal(n, lengths, periodic, grad=None, gradient="fd"):
    """E_x^LDA, E_c^LDA, E_x^PBE, E_c^PBE, E_x^revPBE (Hartree) of density n over all
    points with n > 0, through vdwdf_semilocal; returns the result dict."""
    _check_tensor(n, "n")
    if grad is not None:
        _check_tensor(grad, "grad")
    torch = _torch()
    lib = _native.load()
    g = grid(lengths, n.shape, periodic, gradient)
    res = vdwdf_semilocal_result()
    with torch.cuda.device(n.device):
        st = lib.vdwdf_semilocal(ctypes.byref(g), ctypes.c_void_p(n.data_ptr()),
                                 ctypes.c_void_p(grad.data_ptr()) if grad is not None else None,
                                 ctypes.byref(res), _stream(n))
    _native.check(st, "vdwdf_semilocal")
    return res.as_dict()


def far_tail(n, lengths, periodic, n_cut, r_cut, grad=None, gradient="fd", want_v=False):
    """The far field past r_cut from eq. (17) and the lattice continuum
    (vdwdf_far_tail): E(r_cut -> inf) reads E(r_cut) + T.  Returns the result dict
    (T in Hartree), and with want_v also T's potential on the grid."""
    _check_tensor(n, "n")
    if grad is not None:
        _check_tensor(grad, "grad")
    torch = _torch()
    lib = _native.load()
    g = grid(lengths, n.shape, periodic, gradient)
    res = _native.vdwdf_tail_result()
    v = torch.empty_like(n) if want_v else None
    with torch.cuda.device(n.device):
        st = lib.vdwdf_far_tail(ctypes.byref(g), ctypes.c_void_p(n.data_ptr()),
                                ctypes.c_void_p(grad.data_ptr()) if grad is not None else None,
                                float(n_cut), float(r_cut), ctypes.c_void_p(v.data_ptr()) if want_v else None,
                                ctypes.byref(res), _stream(n))
    _native.check(st, "vdwdf_far_tail")
    return (res.as_dict(), v) if want_v else res.as_dict()


def phi0_eval(table, voxel, q):
    """The voxel-averaged kernel at delta = 0, phi0(q), for the voxel spanned by the
    rows of ``voxel`` (3x3, bohr), at the values of the CUDA FP64 tensor q."""
    _check_tensor(q, "q")
    torch = _torch()
    lib = _native.load()
    vox = np.ascontiguousarray(np.asarray(voxel, dtype=np.float64).reshape(9))
    out = torch.empty_like(q)
    with torch.cuda.device(q.device):
        st = lib.vdwdf_phi0_eval(table.handle, vox.ctypes.data_as(ctypes.c_void_p), int(q.numel()),
                                 ctypes.c_void_p(q.data_ptr()), ctypes.c_void_p(out.data_ptr()), _stream(q))
    _native.check(st, "vdwdf_phi0_eval")
    return out


def diag_voxel(n, lengths, periodic, n_cut, table, nphi0=0, grad=None, gradient="fd"):
    """The voxel-averaged self term 1/2 dV^2 sum n_i^2 phi0(q0_i) over the points with
    n >= n_cut, and the table self term it replaces; returns the result dict.  E_c^nl
    with this diagonal is E - E_diag_table + E_diag_voxel."""
    _check_tensor(n, "n")
    if grad is not None:
        _check_tensor(grad, "grad")
    torch = _torch()
    lib = _native.load()
    g = grid(lengths, n.shape, periodic, gradient)
    res = vdwdf_diag_result()
    with torch.cuda.device(n.device):
        st = lib.vdwdf_diag_voxel(ctypes.byref(g), ctypes.c_void_p(n.data_ptr()),
                                  ctypes.c_void_p(grad.data_ptr()) if grad is not None else None,
                                  float(n_cut), table.handle, int(nphi0), ctypes.byref(res), _stream(n))
    _native.check(st, "vdwdf_diag_voxel")
    return res.as_dict()


def diag_voxel_potential(n, lengths, periodic, n_cut, table, nphi0=0, gradient="fd"):
    """(result dict, dv): the voxel diagonal as diag_voxel and the change dv of the
    potential when it replaces the table self term (v + dv belongs to
    E - E_diag_table + E_diag_voxel)."""
    _check_tensor(n, "n")
    torch = _torch()
    lib = _native.load()
    g = grid(lengths, n.shape, periodic, gradient)
    res = vdwdf_diag_result()
    dv = torch.empty_like(n)
    with torch.cuda.device(n.device):
        st = lib.vdwdf_diag_voxel_potential(ctypes.byref(g), ctypes.c_void_p(n.data_ptr()), float(n_cut),
                                            table.handle, int(nphi0), ctypes.c_void_p(dv.data_ptr()),
                                            ctypes.byref(res), _stream(n))
    _native.check(st, "vdwdf_diag_voxel_potential")
    return res.as_dict(), dv


def total_energy_nl(E_tot_dft, semi, E_c_nl, exchange="pbe"):
    """Eq. 3 through vdwdf_total_energy_nl: the total energy with the nonlocal
    correlation, from the DFT total energy of a PBE calculation, the semilocal
    terms of that density (the dict of semilocal()) and E_c^nl, with E_x^PBE or,
    for exchange="revpbe", E_x^revPBE in the bracket."""
    if exchange not in ("pbe", "revpbe"):
        raise ValueError("exchange must be 'pbe' or 'revpbe'")
    lib = _native.load()
    s = _native.vdwdf_semilocal_result()
    for k in ("Ex_lda", "Ec_lda", "Ex_pbe", "Ec_pbe", "Ex_revpbe"):
        setattr(s, k, float(semi[k]))
    out = ctypes.c_double()
    st = lib.vdwdf_total_energy_nl(float(E_tot_dft), ctypes.byref(s), float(E_c_nl),
                                   0 if exchange == "pbe" else 1, ctypes.byref(out))
    _native.check(st, "vdwdf_total_energy_nl")
    return out.value


def potential(n, lengths, periodic, n_cut, r_cut, table, precision="fp32", tuning=None,
              want_AU=False, out=None, gradient="fd"):
    """E_c^nl and v = dE/dn / dV on the grid; returns (E, v, result dict[, A, U])."""
    _check_tensor(n, "n")
    torch = _torch()
    lib = _native.load()
    g = grid(lengths, n.shape, periodic, gradient)
    v = out if out is not None else torch.empty_like(n)
    _check_tensor(v, "out")
    A = torch.empty_like(n) if want_AU else None
    U = torch.empty_like(n) if want_AU else None
    res = vdwdf_result()
    with torch.cuda.device(n.device):
        st = lib.vdwdf_potential(ctypes.byref(g), ctypes.c_void_p(n.data_ptr()), float(n_cut),
                                 float(r_cut), table.handle, _prec(precision), _tuning(tuning),
                                 ctypes.c_void_p(v.data_ptr()),
                                 ctypes.c_void_p(A.data_ptr()) if want_AU else None,
                                 ctypes.c_void_p(U.data_ptr()) if want_AU else None,
                                 ctypes.byref(res), _stream(n))
    _native.check(st, "vdwdf_potential")
    if want_AU:
        return res.E, v, res.as_dict(), A, U
    return res.E, v, res.as_dict()


def energy_batched(ns, lengths, periodic, n_cut, r_cut, table, precision="fp32", tuning=None, gradient="fd"):
    """E_c^nl of several densities in one persistent launch (CUDA graph, replayed for the
    same tensors).  lengths / periodic: one entry per density.  Returns (E array, result)."""
    torch = _torch()
    lib = _native.load()
    k = len(ns)
    grids = (vdwdf_grid * k)()
    ptrs = (ctypes.c_void_p * k)()
    for i, t in enumerate(ns):
        _check_tensor(t, "ns[%d]" % i)
        grids[i] = grid(lengths[i], t.shape, periodic[i], gradient)
        ptrs[i] = t.data_ptr()
    E = np.zeros(k)
    res = vdwdf_result()
    with torch.cuda.device(ns[0].device):
        st = lib.vdwdf_energy_batched(k, grids, ptrs, float(n_cut), float(r_cut), table.handle,
                                      _prec(precision), _tuning(tuning),
                                      E.ctypes.data_as(ctypes.c_void_p), ctypes.byref(res), _stream(ns[0]))
    _native.check(st, "vdwdf_energy_batched")
    return E, res.as_dict()


def q0(n, lengths, grad=None, want_partials=True, gradient="fd"):
    """q0 and (optionally) dq0/dn, dq0/dgrad n on the grid (Dion eqs. 11-12)."""
    _check_tensor(n, "n")
    torch = _torch()
    lib = _native.load()
    g = grid(lengths, n.shape, gradient=gradient)
    q = torch.empty_like(n)
    qn = torch.empty_like(n) if want_partials else None
    qg = torch.empty((3,) + tuple(n.shape), dtype=n.dtype, device=n.device) if want_partials else None
    with torch.cuda.device(n.device):
        st = lib.vdwdf_q0(ctypes.byref(g), ctypes.c_void_p(n.data_ptr()),
                          ctypes.c_void_p(grad.data_ptr()) if grad is not None else None, 0.0,
                          ctypes.c_void_p(q.data_ptr()),
                          ctypes.c_void_p(qn.data_ptr()) if want_partials else None,
                          ctypes.c_void_p(qg.data_ptr()) if want_partials else None, _stream(n))
    _native.check(st, "vdwdf_q0")
    return q, qn, qg


def gradient(n, lengths, kind="fd"):
    """The library's gradient of n (Cartesian, [3, *n.shape]) on the orthorhombic
    cell ``lengths`` or the general cell (3x3 rows): kind "fd" (4th-order finite
    differences) or "spectral" (the band-limited, FFT derivative)."""
    _check_tensor(n, "n")
    torch = _torch()
    lib = _native.load()
    g = grid(lengths, n.shape, gradient=kind)
    out = torch.empty((3,) + tuple(n.shape), dtype=torch.float64, device=n.device)
    with torch.cuda.device(n.device):
        st = lib.vdwdf_gradient(ctypes.byref(g), ctypes.c_void_p(n.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                _stream(n))
    _native.check(st, "vdwdf_gradient")
    return out


def kernel_eval(table, r, qi, qj, precision="fp32"):
    """phi and r dphi/dd1 at pairs (r, q_i, q_j) through the library's interpolation."""
    torch = _torch()
    lib = _native.load()
    for t, nm in ((r, "r"), (qi, "qi"), (qj, "qj")):
        _check_tensor(t, nm)
    phi = torch.empty_like(r)
    rd = torch.empty_like(r)
    with torch.cuda.device(r.device):
        st = lib.vdwdf_kernel_eval(table.handle, _prec(precision), r.numel(), ctypes.c_void_p(r.data_ptr()),
                                   ctypes.c_void_p(qi.data_ptr()), ctypes.c_void_p(qj.data_ptr()),
                                   ctypes.c_void_p(phi.data_ptr()), ctypes.c_void_p(rd.data_ptr()), _stream(r))
    _native.check(st, "vdwdf_kernel_eval")
    return phi, rd


def autotune(n, lengths, periodic, n_cut, r_cut, table, precision="fp32", gradient="fd"):
    """Fastest launch shape of the pair kernel on this problem (a sampled energy pass)."""
    _check_tensor(n, "n")
    torch = _torch()
    lib = _native.load()
    g = grid(lengths, n.shape, periodic, gradient)
    best = vdwdf_tuning()
    with torch.cuda.device(n.device):
        st = lib.vdwdf_autotune(ctypes.byref(g), ctypes.c_void_p(n.data_ptr()), float(n_cut), float(r_cut),
                                table.handle, _prec(precision), ctypes.byref(best), _stream(n))
    _native.check(st, "vdwdf_autotune")
    return {k: getattr(best, k) for k, _ in vdwdf_tuning._fields_}


def launch_count():
    """Kernels the library has launched in this process."""
    return int(_native.load().vdwdf_launch_count())


LANE_RATE_KINDS = {"fp32": 0, "fp32x2": 1, "fp64": 2}


def lane_rate(kind="fp32", target_ms=20.0, device=None):
    """Measured arithmetic rate of the device (vdwdf_lane_rate): lane operations
    per second for kind "fp32" (FMA), "fp32x2" (packed FMA, two lane operations
    per instruction) or "fp64" (FMA), and the timed launch's milliseconds."""
    if kind not in LANE_RATE_KINDS:
        raise ValueError("kind must be one of %s" % sorted(LANE_RATE_KINDS))
    torch = _torch()
    lib = _native.load()
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    rate, ms = ctypes.c_double(), ctypes.c_double()
    with torch.cuda.device(dev):
        stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
        st = lib.vdwdf_lane_rate(LANE_RATE_KINDS[kind], float(target_ms), ctypes.byref(rate), ctypes.byref(ms),
                                 stream)
    _native.check(st, "vdwdf_lane_rate")
    return rate.value, ms.value


def _make_function():
    torch = _torch()

    class NonlocalEnergy(torch.autograd.Function):
        """E_c^nl as a differentiable function of the density tensor n.

        forward(n, spec) -> E (0-d FP64 tensor); backward gives grad * dE/dn_m =
        grad * dV * v_m, from the library's fused pair pass and the adjoint of its gradient."""

        @staticmethod
        def forward(ctx, n, spec):
            E, v, _ = potential(n, spec["lengths"], spec["periodic"], spec["n_cut"], spec["r_cut"],
                                spec["table"], spec.get("precision", "fp32"), spec.get("tuning"),
                                gradient=spec.get("gradient", "fd"))
            dV = _cell_volume(spec["lengths"]) / float(n.numel())
            ctx.save_for_backward(v)
            ctx.dV = dV
            return torch.tensor(E, dtype=torch.float64, device=n.device)

        @staticmethod
        def backward(ctx, gE):
            (v,) = ctx.saved_tensors
            return gE * ctx.dV * v, None

    return NonlocalEnergy


_FN = None


def nonlocal_energy(n, spec):
    """Differentiable E_c^nl(n); spec: dict(lengths, periodic, n_cut, r_cut, table[, precision,
    tuning, gradient])."""
    global _FN
    if _FN is None:
        _FN = _make_function()
    return _FN.apply(n, spec)


def __getattr__(name):
    if name == "NonlocalEnergy":
        global _FN
        if _FN is None:
            _FN = _make_function()
        return _FN
    raise AttributeError(name)
