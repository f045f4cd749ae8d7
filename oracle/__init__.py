"""Plain FP64 CPU oracle for the vdW-DF nonlocal correlation hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
this package.  The library (``paper_0810_2273_gb300``) never imports it, and
it never imports the library: the two share no code.  Inputs come from the
seeded generators in ``paper_0810_2273_gb300.inputs`` (which hold none of the
method's arithmetic) as plain NumPy arrays.

The arithmetic lives in ``oracle.c`` (FP64, OpenMP over independent outputs);
this module is marshalling plus the grid-level assembly, each step citing the
passage it follows.  Paper: Lazic et al., "JuNoLo", arXiv 0810.2273.

Parity status: see the header of ``oracle.c``.  The paper's own Appendix
energies are *parity unpinned* (the density file they come from is absent).
"""
import ctypes
import os

import numpy as np

from . import build as _build

# Quadrature settings for Dion eq. (14): (a_min, log_ratio, n_log, m_half, n_osc);
# the a- and b-integrals are truncated at A = (m_half + 1/2) pi, where cos A = 0.
# REFERENCE: A = 255.5 pi ~ 803, truncation error ~ 4/A^4 ~ 1e-11.
QUAD_REFERENCE = dict(a_min=1e-7, log_ratio=1.5, n_log=8, m_half=255, n_osc=10)
# TABLE: the node table the parity tests feed to both sides (A ~ 99, ~4e-8).
QUAD_TABLE = dict(a_min=1e-7, log_ratio=2.0, n_log=8, m_half=31, n_osc=10)
# FAST: per-pair direct quadrature in the brute-force pin (A ~ 49, ~7e-7).
QUAD_FAST = dict(a_min=1e-6, log_ratio=2.0, n_log=6, m_half=15, n_osc=8)

C_ASYM = 12.0 * (4.0 * np.pi / 9.0) ** 3   # Dion eq. (17)
ZAB = -0.8491                               # Dion eq. (12)

_LIB = None
_d = ctypes.c_double
_i = ctypes.c_int
_p = ctypes.c_void_p


def load_library(path):
    """The oracle's C functions from the shared library at ``path``, with their
    ctypes signatures (tests also load deliberately broken builds this way)."""
    L = ctypes.CDLL(path)
    L.orc_grid_size.restype = _i
    L.orc_grid_size.argtypes = [_d, _d, _i, _i, _i]
    L.orc_grid.restype = _i
    L.orc_grid.argtypes = [_d, _d, _i, _i, _i, _p, _p]
    L.orc_W.restype = _d
    L.orc_W.argtypes = [_d, _d]
    L.orc_phi_many.restype = _i
    L.orc_phi_many.argtypes = [_i, _p, _p, _p, _d, _d, _i, _i, _i]
    L.orc_phi_table.restype = _i
    L.orc_phi_table.argtypes = [_i, _d, _i, _p, _d, _d, _i, _i, _i]
    L.orc_spline_prepare.restype = _i
    L.orc_spline_prepare.argtypes = [_i, _d, _i, _d, _p, _p, _p, _p, _p, _p]
    L.orc_spline_eval_many.restype = _i
    L.orc_spline_eval_many.argtypes = [_i, _d, _i, _d, _p, _p, _p, _p, _i, _p, _p, _p, _p, _p]
    L.orc_kernel_many.restype = _i
    L.orc_kernel_many.argtypes = [_i, _d, _i, _d, _p, _p, _p, _p, _p, _p, _i, _p, _p, _p, _p, _p]
    L.orc_pair_AU.restype = _i
    L.orc_pair_AU.argtypes = ([_i, _p, _p, _p, _p, _p, _i, _i, _i, _d, _d, _d, _i, _i, _i, _d,
                               _i, _d, _i, _d, _p, _p, _p, _p, _p, _p, _i, _p, _p, _p, _p, _p])
    L.orc_pair_brute.restype = _i
    L.orc_pair_brute.argtypes = ([_i, _p, _p, _p, _p, _p, _i, _i, _i, _d, _d, _d, _i, _i, _i,
                                  _d, _d, _d, _d, _d, _i, _i, _i, _p])
    L.orc_gradient.restype = _i
    L.orc_gradient.argtypes = [_i, _i, _i, _d, _d, _d, _p, _p]
    L.orc_gradient_T.restype = _i
    L.orc_gradient_T.argtypes = [_i, _i, _i, _d, _d, _d, _p, _p]
    L.orc_eps_c.restype = _i
    L.orc_eps_c.argtypes = [_i, _p, _p, _p]
    L.orc_q0.restype = _i
    L.orc_q0.argtypes = [_i, _p, _p, _p, _p, _p]
    L.orc_pair_AU_cell.restype = _i
    L.orc_pair_AU_cell.argtypes = ([_i, _p, _p, _p, _p, _p, _i, _i, _i, _p, _i, _i, _i, _d,
                                    _i, _d, _i, _d, _p, _p, _p, _p, _p, _p, _i, _p, _p, _p, _p, _p])
    L.orc_gradient_cell.restype = _i
    L.orc_gradient_cell.argtypes = [_i, _i, _i, _p, _p, _p]
    L.orc_gradient_T_cell.restype = _i
    L.orc_gradient_T_cell.argtypes = [_i, _i, _i, _p, _p, _p]
    L.orc_phi0_many.restype = _i
    L.orc_phi0_many.argtypes = [_i, _d, _i, _d, _p, _p, _p, _p, _p, _p, _p, _i, _p, _p, _i, _i]
    L.orc_fx_many.restype = _i
    L.orc_fx_many.argtypes = [_i, _p, _d, _p]
    L.orc_pbe_H_many.restype = _i
    L.orc_pbe_H_many.argtypes = [_i, _p, _p, _p]
    L.orc_far_tail.restype = _i
    L.orc_far_tail.argtypes = [_i, _p, _p, _p, _p, _p, _i, _i, _i, _p, _i, _i, _i, _d, _p]
    L.orc_line_tail_integral.restype = _d
    L.orc_line_tail_integral.argtypes = [_d, _d]
    L.orc_far_tail_AB.restype = _i
    L.orc_far_tail_AB.argtypes = [_i, _p, _p, _p, _p, _p, _i, _i, _i, _p, _i, _i, _i, _d, _i, _p, _p, _p]
    L.orc_semilocal.restype = _i
    L.orc_semilocal.argtypes = [_i, _p, _p, _p, _p]
    return L


def lib():
    """Load (building first if needed) the oracle's shared library."""
    global _LIB
    if _LIB is None:
        _LIB = load_library(_build.build())
    return _LIB


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _q(quad):
    return (quad["a_min"], quad["log_ratio"], quad["n_log"], quad["m_half"], quad["n_osc"])


# --------------------------------------------------------------------------
# Kernel phi (section 2; Dion eq. 14 and 17)
# --------------------------------------------------------------------------
def grid(quad=QUAD_REFERENCE):
    """Quadrature nodes and weights on (0, (m_half + 1/2) pi]."""
    L = lib()
    n = L.orc_grid_size(*_q(quad))
    a = np.zeros(n)
    w = np.zeros(n)
    if L.orc_grid(*_q(quad), _ptr(a), _ptr(w)) != n:
        raise ValueError("bad quadrature settings")
    return a, w


def W(a, b):
    """Dion's W(a, b) (eq. 14), from the factored form (see oracle.c)."""
    L = lib()
    a = np.atleast_1d(np.asarray(a, dtype=np.float64))
    b = np.atleast_1d(np.asarray(b, dtype=np.float64))
    a, b = np.broadcast_arrays(a, b)
    return np.array([L.orc_W(float(x), float(y)) for x, y in zip(a.ravel(), b.ravel())]).reshape(a.shape)


def phi(d1, d2, quad=QUAD_REFERENCE):
    """phi(d1, d2) by direct quadrature of Dion eq. (14)."""
    d1 = np.atleast_1d(_f64(d1))
    d2 = np.atleast_1d(_f64(d2))
    d1, d2 = np.broadcast_arrays(d1, d2)
    d1 = _f64(d1.ravel())
    d2 = _f64(d2.ravel())
    out = np.zeros_like(d1)
    rc = lib().orc_phi_many(len(d1), _ptr(d1), _ptr(d2), _ptr(out), *_q(quad))
    if rc != 0:
        raise RuntimeError("orc_phi_many failed (%d)" % rc)
    return out


def phi_asym(d1, d2):
    """Large-D asymptote, Dion eq. (17): -C / (d1^2 d2^2 (d1^2 + d2^2))."""
    d1 = np.asarray(d1, dtype=np.float64)
    d2 = np.asarray(d2, dtype=np.float64)
    return -C_ASYM / (d1 ** 2 * d2 ** 2 * (d1 ** 2 + d2 ** 2))


def phi_table(nD=400, Dmax=30.0, ndelta=200, quad=QUAD_TABLE):
    """Node table phi(D_k, delta_l), D_k = Dmax k/(nD-1), delta_l = l/ndelta.

    Row 0 (D = 0, where eq. 14 diverges logarithmically) holds
    (4 phi(D_1) - phi(D_2)) / 3, the even quadratic through rows 1 and 2.
    """
    nodes = np.zeros((nD, ndelta))
    rc = lib().orc_phi_table(nD, Dmax, ndelta, _ptr(nodes), *_q(quad))
    if rc != 0:
        raise RuntimeError("orc_phi_table failed (%d)" % rc)
    return nodes


class Spline:
    """Tensor-product cubic spline through the node table (M form).

    Boundary conditions: zero slope at D = 0 and delta = 0, zero curvature at
    the last node of each axis.  ``kernel`` adds the D > Dmax branch: eq. (17)
    times g = rho(delta*) + (1 - rho(0)) (1 - (Dmax/D)^2), rho the 1-D spline
    through phi(Dmax, delta_l) / phi17(Dmax, delta_l) and
    delta* = max(0, 1 - min(d1, d2)/Dmax).
    """

    def __init__(self, nodes, Dmax=30.0):
        self.f = _f64(nodes)
        self.nD, self.nd = self.f.shape
        self.Dmax = float(Dmax)
        self.hD = self.Dmax / (self.nD - 1)
        self.hd = 1.0 / self.nd
        self.fDD = np.zeros_like(self.f)
        self.fdd = np.zeros_like(self.f)
        self.fDDdd = np.zeros_like(self.f)
        self.rho = np.zeros(self.nd)
        self.rhoM = np.zeros(self.nd)
        rc = lib().orc_spline_prepare(self.nD, self.hD, self.nd, self.hd, _ptr(self.f),
                                      _ptr(self.fDD), _ptr(self.fdd), _ptr(self.fDDdd),
                                      _ptr(self.rho), _ptr(self.rhoM))
        if rc != 0:
            raise RuntimeError("orc_spline_prepare failed (%d)" % rc)

    def _args(self):
        return (self.nD, self.hD, self.nd, self.hd, _ptr(self.f), _ptr(self.fDD),
                _ptr(self.fdd), _ptr(self.fDDdd))

    def _kargs(self):
        return self._args() + (_ptr(self.rho), _ptr(self.rhoM))

    def eval(self, D, dl):
        """Spline value and partials (phi, dphi/dD, dphi/ddelta) inside the table."""
        D = np.atleast_1d(_f64(D))
        dl = np.atleast_1d(_f64(dl))
        D, dl = np.broadcast_arrays(D, dl)
        D = _f64(D.ravel())
        dl = _f64(dl.ravel())
        p, pD, pd = (np.zeros_like(D) for _ in range(3))
        lib().orc_spline_eval_many(*self._args(), len(D), _ptr(D), _ptr(dl), _ptr(p), _ptr(pD), _ptr(pd))
        return p, pD, pd

    def phi0(self, vox, q, panels=6, npts=6):
        """Voxel-averaged kernel at delta = 0, phi0(q), for the voxel spanned by the
        rows of vox (v_a = M_a / N_a), at each q (see orc_phi0_many)."""
        vox = _f64(vox).reshape(3, 3)
        q = np.atleast_1d(_f64(q))
        out = np.zeros_like(q)
        rc = lib().orc_phi0_many(*self._kargs(), _ptr(vox), len(q), _ptr(q), _ptr(out), int(panels), int(npts))
        if rc != 0:
            raise RuntimeError("orc_phi0_many failed (%d)" % rc)
        return out

    def kernel(self, r, qi, qj):
        """phi and r dphi/dd1 for pairs (d1 = qi r, d2 = qj r); returns (phi, rdphi1, nclamped)."""
        r, qi, qj = (np.atleast_1d(_f64(x)) for x in (r, qi, qj))
        r, qi, qj = (_f64(x.ravel()) for x in np.broadcast_arrays(r, qi, qj))
        p = np.zeros_like(r)
        rd = np.zeros_like(r)
        ncl = lib().orc_kernel_many(*self._kargs(), len(r), _ptr(r), _ptr(qi), _ptr(qj), _ptr(p), _ptr(rd))
        return p, rd, ncl


# --------------------------------------------------------------------------
# Gradient and q0 (section 3 "gradient"; Dion eqs. 11-12)
# --------------------------------------------------------------------------
def gradient(f, h):
    """4th-order periodic central differences along the three axes -> (3, n0, n1, n2)."""
    f = _f64(f)
    g = np.zeros((3,) + f.shape)
    lib().orc_gradient(*f.shape, *map(float, h), _ptr(f), _ptr(g))
    return g


_gradient_fd = gradient  # Problem's keyword ``gradient`` shadows the name there


def gradient_T(w, h):
    """sum over axes of the transposed stencil applied to w (3, n0, n1, n2)."""
    w = _f64(w)
    out = np.zeros(w.shape[1:])
    lib().orc_gradient_T(*w.shape[1:], *map(float, h), _ptr(w), _ptr(out))
    return out


def eps_c(rs):
    """PW92 LDA correlation energy per electron and d eps_c / d rs (Hartree)."""
    rs = np.atleast_1d(_f64(rs))
    e = np.zeros_like(rs)
    de = np.zeros_like(rs)
    lib().orc_eps_c(len(rs), _ptr(rs), _ptr(e), _ptr(de))
    return e, de


def gradient_cell(f, cell):
    """Gradient on a general cell (rows of cell: lattice vectors, bohr): the
    4th-order stencil along each grid axis gives df/du_a, and grad f =
    sum_a (df/du_a) B_a with the reciprocal rows B_a.  Returns [3][...]."""
    f = _f64(f)
    cell = _f64(cell).reshape(3, 3)
    g = np.zeros((3,) + f.shape)
    if lib().orc_gradient_cell(*f.shape, _ptr(cell), _ptr(f), _ptr(g)) != 0:
        raise ValueError("singular cell")
    return g


def gradient_T_cell(w, cell):
    """Transpose of gradient_cell applied to w [3][...]."""
    w = _f64(w)
    cell = _f64(cell).reshape(3, 3)
    out = np.zeros(w.shape[1:])
    if lib().orc_gradient_T_cell(*w.shape[1:], _ptr(cell), _ptr(w), _ptr(out)) != 0:
        raise ValueError("singular cell")
    return out


def _recip_rows(cell_or_lengths, shape):
    """Reciprocal rows B_a (B_a . M_b = delta_ab) of a cell given as 3 lengths
    (orthorhombic) or as 3x3 rows of lattice vectors."""
    c = _f64(cell_or_lengths)
    cell = np.diag(c) if c.shape == (3,) else c.reshape(3, 3)
    return np.linalg.inv(cell).T


def _spectral_multipliers(shape):
    """2 pi i m_a along each axis for the DFT frequencies m_a in (-N/2, N/2); the
    Nyquist frequency m_a = N_a/2 of an even axis gets 0 (it is its own mirror
    image, so a real field has no odd part there: the real part of the inverse
    transform drops it)."""
    mult = []
    for a, N in enumerate(shape):
        m = np.fft.fftfreq(N, 1.0 / N)
        k = 2j * np.pi * m
        if N % 2 == 0:
            k[N // 2] = 0.0
        sh = [1, 1, 1]
        sh[a] = N
        mult.append(k.reshape(sh))
    return mult


def gradient_spectral(f, cell_or_lengths):
    """The FFT gradient (section 3 of the paper, the FFTW option): df/du_a by
    multiplying the discrete Fourier transform along u_a (fractional coordinate,
    period 1) by 2 pi i m_a, then grad f = sum_a (df/du_a) B_a.  Returns [3][...]."""
    f = _f64(f)
    B = _recip_rows(cell_or_lengths, f.shape)
    F = np.fft.fftn(f)
    d = [np.real(np.fft.ifftn(k * F)) for k in _spectral_multipliers(f.shape)]
    return np.stack([sum(B[a, c] * d[a] for a in range(3)) for c in range(3)])


def gradient_spectral_T(w, cell_or_lengths):
    """Transpose of gradient_spectral applied to w [3][...]: sum_c D_c^T w_c.  With
    F the DFT, D_c = F^-1 Lambda_c F for purely imaginary Lambda_c, so
    D_c^T = F^-1 conj(Lambda_c) F; written with the conjugate multipliers."""
    w = _f64(w)
    shape = w.shape[1:]
    B = _recip_rows(cell_or_lengths, shape)
    mult = _spectral_multipliers(shape)
    out = np.zeros(shape)
    for a in range(3):
        Wa = sum(B[a, c] * w[c] for c in range(3))
        out += np.real(np.fft.ifftn(np.conj(mult[a]) * np.fft.fftn(Wa)))
    return out


def q0(n, g):
    """q0 and its partials dq0/dn, dq0/dgrad n at every grid point."""
    n = _f64(n)
    g = _f64(g).reshape((3,) + n.shape)
    N = n.size
    q = np.zeros(n.shape)
    qn = np.zeros(n.shape)
    qg = np.zeros((3,) + n.shape)
    lib().orc_q0(N, _ptr(n), _ptr(g), _ptr(q), _ptr(qn), _ptr(qg))
    return q, qn, qg


# --------------------------------------------------------------------------
# Semilocal energies of eq. 3 (section 2): LDA, PBE, revPBE
# --------------------------------------------------------------------------
KAPPA_PBE = 0.804     # Perdew, Burke, Ernzerhof 1996
KAPPA_REVPBE = 1.245  # Zhang and Yang 1998


def fx(s, kappa):
    """GGA exchange enhancement factor F_x(s) = 1 + kappa - kappa/(1 + mu s^2/kappa)."""
    s = _f64(s)
    out = np.zeros(s.shape)
    lib().orc_fx_many(s.size, _ptr(s), float(kappa), _ptr(out))
    return out


def pbe_H(rs, t):
    """Gradient correction H(rs, t) of the PBE correlation (unpolarised)."""
    rs, t = np.broadcast_arrays(_f64(rs), _f64(t))
    rs, t = _f64(rs), _f64(t)
    out = np.zeros(rs.shape)
    lib().orc_pbe_H_many(rs.size, _ptr(rs), _ptr(t), _ptr(out))
    return out


def semilocal(n, lengths, g=None, cell=None):
    """E_x^LDA, E_c^LDA (PW92), E_x^PBE, E_c^PBE, E_x^revPBE (Hartree) of the density
    n on an orthorhombic grid of the given cell lengths (or on the general cell
    ``cell``, rows = lattice vectors), summed over points with n > 0;
    g: [3][n0][n1][n2] Cartesian gradient, or None for the 4th-order stencil."""
    n = _f64(n)
    if cell is not None:
        cell = _f64(cell).reshape(3, 3)
        if g is None:
            g = gradient_cell(n, cell)
        dV = abs(float(np.linalg.det(cell))) / n.size
    else:
        h = [float(L) / d for L, d in zip(lengths, n.shape)]
        if g is None:
            g = gradient(n, h)
        dV = h[0] * h[1] * h[2]
    g = _f64(g).reshape((3,) + n.shape)
    sums = np.zeros(5)
    count = ctypes.c_int64()
    lib().orc_semilocal(n.size, _ptr(n), _ptr(g), _ptr(sums), ctypes.byref(count))
    keys = ("Ex_lda", "Ec_lda", "Ex_pbe", "Ec_pbe", "Ex_revpbe")
    out = {k: dV * v for k, v in zip(keys, sums)}
    out["n_points"] = count.value
    return out


# --------------------------------------------------------------------------
# The double sum and its adjoint (section 2 eq. 2; section 3)
# --------------------------------------------------------------------------
class Problem:
    """A density on a periodic grid, trimmed at n_cut.

    dims: (n0, n1, n2); lengths: (L0, L1, L2) bohr of an orthorhombic cell, or
    cell: 3x3 rows = lattice vectors (bohr) of a general cell (then lengths is
    ignored); periodic: 3 flags; rc: spherical pair cutoff in bohr (<= 0: none;
    required if periodic); g: the gradient [3][...] (Cartesian) to use instead
    of the library-style stencil.
    """

    def __init__(self, density, lengths, periodic, n_cut, rc, spline, cell=None, g=None, gradient="fd"):
        self.n = _f64(density)
        self.dims = self.n.shape
        self.periodic = tuple(int(bool(p)) for p in periodic)
        self.n_cut = float(n_cut)
        self.rc = float(rc)
        self.spline = spline
        if cell is None:
            self.cell = None
            self.lengths = tuple(float(x) for x in lengths)
            self.h = tuple(L / d for L, d in zip(self.lengths, self.dims))
            self.dV = float(np.prod(self.lengths)) / float(np.prod(self.dims))
        else:
            self.cell = _f64(cell).reshape(3, 3)
            self.lengths = None
            self.h = None
            self.dV = abs(float(np.linalg.det(self.cell))) / float(np.prod(self.dims))
        if gradient not in ("fd", "spectral"):
            raise ValueError("gradient: 'fd' or 'spectral'")
        self.gradient_kind = gradient
        geom = self.lengths if self.cell is None else self.cell
        if g is not None:
            self.g = _f64(g).reshape((3,) + self.dims)
        elif gradient == "spectral":
            self.g = gradient_spectral(self.n, geom)
        else:
            self.g = _gradient_fd(self.n, self.h) if self.cell is None else gradient_cell(self.n, self.cell)
        self.q0, self.dq0dn, self.dq0dg = q0(self.n, self.g)
        flat = self.n.ravel()
        self.active = np.nonzero(flat >= self.n_cut)[0]          # row-major order
        self.slot = -np.ones(flat.size, dtype=np.int64)
        self.slot[self.active] = np.arange(len(self.active))
        i0, i1, i2 = np.unravel_index(self.active, self.dims)
        self.i0, self.i1, self.i2 = _i32(i0), _i32(i1), _i32(i2)
        self.na = _f64(flat[self.active])
        self.qa = _f64(self.q0.ravel()[self.active])

    @property
    def n_active(self):
        return len(self.active)

    def AU(self, queries=None):
        """A_i, U_i, pair counts and clamp counts for active slots ``queries``."""
        if queries is None:
            queries = np.arange(self.n_active)
        qidx = _i32(queries)
        A = np.zeros(len(qidx))
        U = np.zeros(len(qidx))
        npairs = np.zeros(len(qidx), dtype=np.int64)
        ncl = np.zeros(len(qidx), dtype=np.int64)
        s = self.spline
        if self.cell is None:
            rc = lib().orc_pair_AU(self.n_active, _ptr(self.i0), _ptr(self.i1), _ptr(self.i2),
                                   _ptr(self.na), _ptr(self.qa), *self.dims, *self.lengths,
                                   *self.periodic, self.rc, *s._kargs(), len(qidx), _ptr(qidx),
                                   _ptr(A), _ptr(U), _ptr(npairs), _ptr(ncl))
        else:
            rc = lib().orc_pair_AU_cell(self.n_active, _ptr(self.i0), _ptr(self.i1), _ptr(self.i2),
                                        _ptr(self.na), _ptr(self.qa), *self.dims, _ptr(self.cell),
                                        *self.periodic, self.rc, *s._kargs(), len(qidx), _ptr(qidx),
                                        _ptr(A), _ptr(U), _ptr(npairs), _ptr(ncl))
        if rc != 0:
            raise RuntimeError("orc_pair_AU failed (%d)" % rc)
        return A, U, npairs, ncl

    def energy(self):
        """E = 1/2 dV^2 sum_i n_i A_i, its self-term part, pair count (all active points)."""
        A, U, npairs, ncl = self.AU()
        E = 0.5 * self.dV ** 2 * float(np.dot(self.na, A))
        E_diag = 0.5 * self.dV ** 2 * float(np.dot(self.na, self.na)) * self.spline.f[0, 0]
        return dict(E=E, E_diag=E_diag, pairs=int(npairs.sum()), clamped=int(ncl.sum()), A=A, U=U)

    def potential(self, A=None, U=None):
        """v = dE/dn / dV on the whole grid (mask frozen):
        v_m = dV [chi_m (A_m + U_m dq0/dn_m) + sum_ax (D_ax^T w_ax)_m],
        w_ax = chi U dq0/dgrad_ax.  Needs A, U at every active point."""
        if A is None or U is None:
            A, U, _, _ = self.AU()
        flat_n = self.n.size
        Ag = np.zeros(flat_n)
        Ug = np.zeros(flat_n)
        Ag[self.active] = A
        Ug[self.active] = U
        w = self.dq0dg.reshape(3, -1) * Ug[None, :]
        if self.gradient_kind == "spectral":
            geom = self.lengths if self.cell is None else self.cell
            div = gradient_spectral_T(w.reshape((3,) + self.dims), geom).ravel()
        elif self.cell is None:
            div = gradient_T(w.reshape((3,) + self.dims), self.h).ravel()
        else:
            div = gradient_T_cell(w.reshape((3,) + self.dims), self.cell).ravel()
        chi = np.zeros(flat_n)
        chi[self.active] = 1.0
        v = self.dV * (chi * (Ag + Ug * self.dq0dn.ravel()) + div)
        return v.reshape(self.dims)

    def potential_at(self, points):
        """v at flat grid indices ``points`` from A, U at only the active points
        in their stencil neighbourhoods (each point and +-1, +-2 along each axis).
        Finite-difference gradient only (the spectral one couples whole lines)."""
        if self.gradient_kind != "fd":
            raise NotImplementedError("potential_at: finite-difference gradient only")
        points = np.asarray(points, dtype=np.int64)
        d = self.dims
        need = set()
        coords = np.stack(np.unravel_index(points, d), axis=1)
        for c in coords:
            for ax in range(3):
                for o in (-2, -1, 0, 1, 2):
                    cc = list(c)
                    cc[ax] = (cc[ax] + o) % d[ax]
                    m = np.ravel_multi_index(cc, d)
                    if self.slot[m] >= 0:
                        need.add(int(self.slot[m]))
        need = np.array(sorted(need), dtype=np.int64)
        A, U, _, _ = self.AU(need)
        Amap = dict(zip(need.tolist(), A.tolist()))
        Umap = dict(zip(need.tolist(), U.tolist()))
        c4 = (1.0 / 12.0, -8.0 / 12.0, 0.0, 8.0 / 12.0, -1.0 / 12.0)
        out = np.zeros(len(points))
        qn = self.dq0dn.ravel()
        qg = self.dq0dg.reshape(3, -1)
        # (D_ax^T applied to (B_ax . w)), B_ax the reciprocal row scaled by N_ax; on an
        # orthorhombic cell B_ax . w = w_ax / L_ax and N_ax / L_ax = 1 / h_ax
        if self.cell is None:
            Bs = np.diag([1.0 / h for h in self.h])
        else:
            Bs = np.linalg.inv(self.cell).T * np.array(d, dtype=float)[:, None]
        for t, (m, c) in enumerate(zip(points, coords)):
            val = 0.0
            s = int(self.slot[m])
            if s >= 0:
                val += Amap[s] + Umap[s] * qn[m]
            # sum_ax (D^T w)_m = sum_ax sum_o c_o w_{m-o} / h_ax
            for ax in range(3):
                for o in (-2, -1, 1, 2):
                    cc = list(c)
                    cc[ax] = (cc[ax] - o) % d[ax]
                    mm = int(np.ravel_multi_index(cc, d))
                    ss = int(self.slot[mm])
                    if ss >= 0:
                        val += c4[o + 2] * Umap[ss] * float(np.dot(Bs[ax], qg[:, mm]))
            out[t] = self.dV * val
        return out

    def far_tail(self):
        """The far field past the cutoff from eq. (17) and the lattice continuum
        (see orc_far_tail): T such that E(r_cut -> inf) reads E(r_cut) + T."""
        cell = np.diag(self.lengths) if self.cell is None else self.cell
        return far_tail_points(self.i0, self.i1, self.i2, self.na, self.qa, self.dims, cell,
                               self.periodic, self.rc)

    def far_tail_potential(self):
        """The potential of the far field T (far_tail): v_T = dT/dn / dV with the mask
        frozen.  T has the pair sum's adjoint form with
            A_m = -C sum_j n_j f(u_m, u_j) K_mj,
            U_m = dT/dq_m / dV^2 = -C n_m 2 q_m sum_j n_j df/da(u_m, u_j) K_mj,
        f(a, b) = 1 / (a b (a + b)), u = q0^2 (orc_far_tail_AB), so the grid
        assembly of ``potential`` applies."""
        cell = np.diag(self.lengths) if self.cell is None else self.cell
        cell = _f64(cell).reshape(3, 3)
        qidx = _i32(np.arange(self.n_active))
        AT = np.zeros(self.n_active)
        BT = np.zeros(self.n_active)
        rc_ = lib().orc_far_tail_AB(self.n_active, _ptr(self.i0), _ptr(self.i1), _ptr(self.i2),
                                    _ptr(self.na), _ptr(self.qa), *map(int, self.dims), _ptr(cell),
                                    *self.periodic, self.rc, len(qidx), _ptr(qidx), _ptr(AT), _ptr(BT))
        if rc_ != 0:
            raise ValueError("far tail needs a periodic axis and rc > 0")
        return self.potential(A=-C_ASYM * AT, U=-C_ASYM * self.na * 2.0 * self.qa * BT)

    def voxel(self):
        """Rows v_a = M_a / N_a spanning one voxel."""
        cell = np.diag(self.lengths) if self.cell is None else self.cell
        return cell / np.array(self.dims, dtype=float)[:, None]

    def diag_voxel(self, panels=5, npts=5):
        """The voxel-averaged self term 1/2 dV^2 sum_i n_i^2 phi0(q_i) over the active
        points (each phi0 by direct quadrature), and the table self term it replaces."""
        p0 = self.spline.phi0(self.voxel(), self.qa, panels, npts)
        E = 0.5 * self.dV ** 2 * float(np.dot(self.na * self.na, p0))
        E_tab = 0.5 * self.dV ** 2 * float(np.dot(self.na, self.na)) * self.spline.f[0, 0]
        return dict(E_diag_voxel=E, E_diag_table=E_tab, phi0=p0)

    def brute_energy(self, quad=QUAD_FAST):
        """E from direct quadrature of eq. (14) at every pair (no table)."""
        out = ctypes.c_double(0.0)
        rc = lib().orc_pair_brute(self.n_active, _ptr(self.i0), _ptr(self.i1), _ptr(self.i2),
                                  _ptr(self.na), _ptr(self.qa), *self.dims, *self.lengths,
                                  *self.periodic, self.rc, self.spline.Dmax,
                                  float(self.spline.f[0, 0]), *_q(quad), ctypes.byref(out))
        if rc != 0:
            raise RuntimeError("orc_pair_brute failed (%d)" % rc)
        return 0.5 * self.dV ** 2 * out.value


def line_tail_integral(rho, x0):
    """orc_line_tail_integral: int_{x0}^inf dx / (rho^2 + x^2)^3."""
    return float(lib().orc_line_tail_integral(float(rho), float(x0)))


def far_tail_points(i0, i1, i2, n, q, dims, cell, periodic, rc):
    """orc_far_tail on given points (grid indices), densities and q0 values."""
    i0, i1, i2 = _i32(i0), _i32(i1), _i32(i2)
    n, q = _f64(n), _f64(q)
    cell = _f64(cell).reshape(3, 3)
    out = ctypes.c_double(0.0)
    rc_ = lib().orc_far_tail(len(n), _ptr(i0), _ptr(i1), _ptr(i2), _ptr(n), _ptr(q), *map(int, dims),
                             _ptr(cell), *[int(bool(p)) for p in periodic], float(rc), ctypes.byref(out))
    if rc_ != 0:
        raise ValueError("far tail needs a periodic axis and rc > 0")
    return out.value


_TABLE_CACHE = {}


def cached_table(nD=400, Dmax=30.0, ndelta=200, quad=QUAD_TABLE, cache_dir=None):
    """phi_table(), memoised in-process and on disk (under .cache/ at the repo root)."""
    key = (nD, float(Dmax), ndelta) + _q(quad)
    if key in _TABLE_CACHE:
        return _TABLE_CACHE[key]
    if cache_dir is None:
        cache_dir = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), ".cache")
    name = "oracle_phi_%d_%g_%d_%g_%g_%d_%d_%d.npy" % key
    path = os.path.join(cache_dir, name)
    if os.path.exists(path):
        nodes = np.load(path)
    else:
        nodes = phi_table(nD, Dmax, ndelta, quad)
        os.makedirs(cache_dir, exist_ok=True)
        tmp = path + ".tmp%d.npy" % os.getpid()
        np.save(tmp, nodes)
        os.replace(tmp, path)
    _TABLE_CACHE[key] = nodes
    return nodes
