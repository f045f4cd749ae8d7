"""Seeded synthetic densities for the five standard workloads.

This module holds no arithmetic of the method (no kernel, no q0, no pair
sum): it only builds charge densities on grids, shaped like the paper's two
examples (section 6: a rare-gas dimer and a rare-gas monolayer) and three
larger stand-ins.  The paper's own DFT densities are not available, so these
stand in for them.  Every array is FP64, row-major [n0][n1][n2], with grid
point (i, j, k) at (i L0/n0, j L1/n1, k L2/n2) bohr.

Workloads (``config(i)``):
  0 kr_dimer        two rare-gas atoms 7.6 bohr apart, 24x18x18, open
  1 xe_monolayer    8-atom hexagonal monolayer cell, 48x84x120, periodic x,y
  2 molecule24      24 random atoms, 64^3, open
  3 binding_curve   16 dimers (6.0..12.0 bohr) + 2 single atoms, open
  4 slab_adsorbate  4-layer 144-atom slab + 30-atom flake, 128x112x200,
                    periodic x,y
  5 xe_monolayer_hex  the monolayer in a 4-atom hexagonal cell (60 degrees),
                    48x48x120, periodic along the in-plane lattice vectors
Seeds: NumPy PCG64, 20081021 + workload index.  Workloads on a general cell
carry it as w["cell"] (rows: lattice vectors); w["lengths"] is then only its
diagonal and must not be used as the cell.
"""
import math

import numpy as np

SEED_BASE = 20081021


def _rng(idx):
    return np.random.Generator(np.random.PCG64(SEED_BASE + idx))


def rare_gas_shells():
    """Two-exponential valence density of 8 electrons, 3:1 in electron count:
    A1 exp(-r/0.35) + A2 exp(-r/1.1), A = N_e / (8 pi a^3)."""
    a1, a2 = 0.35, 1.1
    return [(6.0 / (8.0 * math.pi * a1 ** 3), a1), (2.0 / (8.0 * math.pi * a2 ** 3), a2)]


def single_exponential(Z, a):
    """Z electrons as Z / (8 pi a^3) exp(-r / a)."""
    return [(Z / (8.0 * math.pi * a ** 3), a)]


def density(dims, lengths, atoms, periodic=(False, False, False), floor=1e-14):
    """Sum of exponential atoms on the grid.

    atoms: list of (position (3,), [(amplitude, decay length), ...]).
    Periodic axes add the atom's images one cell either side.  Each
    component is evaluated only where it exceeds ``floor`` (far below any
    density cutoff used here).
    """
    dims = tuple(int(d) for d in dims)
    L = np.asarray(lengths, dtype=np.float64)
    h = L / np.asarray(dims, dtype=np.float64)
    out = np.zeros(dims, dtype=np.float64)
    axes = [np.arange(d, dtype=np.float64) * hh for d, hh in zip(dims, h)]
    shifts = [(-1, 0, 1) if p else (0,) for p in periodic]
    for pos, comps in atoms:
        pos = np.asarray(pos, dtype=np.float64)
        rmax = max(a * math.log(max(A / floor, 1.0)) for A, a in comps)
        for s0 in shifts[0]:
            for s1 in shifts[1]:
                for s2 in shifts[2]:
                    c = pos + np.array([s0, s1, s2]) * L
                    lo = [max(0, int(math.floor((c[k] - rmax) / h[k]))) for k in range(3)]
                    hi = [min(dims[k], int(math.ceil((c[k] + rmax) / h[k])) + 1) for k in range(3)]
                    if any(l >= u for l, u in zip(lo, hi)):
                        continue
                    dx = (axes[0][lo[0]:hi[0]] - c[0]) ** 2
                    dy = (axes[1][lo[1]:hi[1]] - c[1]) ** 2
                    dz = (axes[2][lo[2]:hi[2]] - c[2]) ** 2
                    r = np.sqrt(dx[:, None, None] + dy[None, :, None] + dz[None, None, :])
                    blk = out[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]]
                    for A, a in comps:
                        blk += A * np.exp(-r / a)
    return out


def density_cell(dims, cell, atoms, periodic=(False, False, False), floor=1e-14):
    """As density(), on a general cell: rows of ``cell`` are the lattice vectors,
    grid point (i, j, k) sits at i/n0 M_0 + j/n1 M_1 + k/n2 M_2.  Periodic axes add
    the atom's images one cell either side (by lattice vectors)."""
    dims = tuple(int(d) for d in dims)
    M = np.asarray(cell, dtype=np.float64).reshape(3, 3)
    u = np.meshgrid(*[np.arange(d, dtype=np.float64) / d for d in dims], indexing="ij")
    P = u[0][..., None] * M[0] + u[1][..., None] * M[1] + u[2][..., None] * M[2]
    out = np.zeros(dims, dtype=np.float64)
    shifts = [(-1, 0, 1) if p else (0,) for p in periodic]
    for pos, comps in atoms:
        pos = np.asarray(pos, dtype=np.float64)
        for s0 in shifts[0]:
            for s1 in shifts[1]:
                for s2 in shifts[2]:
                    c = pos + s0 * M[0] + s1 * M[1] + s2 * M[2]
                    r = np.sqrt(((P - c) ** 2).sum(-1))
                    for A, a in comps:
                        e = A * np.exp(-r / a)
                        out += np.where(e > floor, e, 0.0)
    return out


def _noise(n, rng, amp):
    """Multiplicative seeded noise n (1 + amp U(-1, 1))."""
    return n * (1.0 + amp * rng.uniform(-1.0, 1.0, size=n.shape))


def _workload(name, idx, dens, lengths, periodic, n_cut, r_cut, **extra):
    w = dict(name=name, index=idx, density=dens, lengths=tuple(float(x) for x in lengths),
             periodic=tuple(bool(p) for p in periodic), n_cut=float(n_cut), r_cut=float(r_cut),
             seed=SEED_BASE + idx)
    w.update(extra)
    return w


def kr_dimer(dims=(24, 18, 18)):
    """Rare-gas dimer, atoms at (8 +- 3.8, 6, 6) in a 16 x 12 x 12 bohr open cell."""
    L = (16.0, 12.0, 12.0)
    atoms = [((8.0 - 3.8, 6.0, 6.0), rare_gas_shells()), ((8.0 + 3.8, 6.0, 6.0), rare_gas_shells())]
    n = density(dims, L, atoms)
    return _workload("kr_dimer", 0, n, L, (False, False, False), 1e-6, 0.0, atoms=atoms)


def xe_monolayer(dims=(48, 84, 120)):
    """Hexagonal rare-gas monolayer, nearest neighbours 8.2 bohr, in a 16.4 x 28.4
    surface cell (2 x 2 rectangular cells of the hexagonal lattice: 8 atoms), 40 bohr
    high with the layer at z = 20.  Periodic in x and y, 20 bohr pair cutoff,
    1% multiplicative noise, density cutoff 1e-6."""
    L = (16.4, 28.4, 40.0)
    atoms = []
    for j in range(4):
        for i in range(2):
            atoms.append(((i * 8.2 + (j % 2) * 4.1, j * 7.1, 20.0), rare_gas_shells()))
    n = density(dims, L, atoms, periodic=(True, True, False))
    n = _noise(n, _rng(1), 0.01)
    return _workload("xe_monolayer", 1, n, L, (True, True, False), 1e-6, 20.0, atoms=atoms)


def xe_monolayer_hex(dims=(48, 48, 120)):
    """The rare-gas monolayer of xe_monolayer in a hexagonal cell, as the paper's
    own Xe cell is (section 6.2): a 2 x 2 supercell of the primitive cell with
    nearest neighbours 8.2 bohr, M_0 = (16.4, 0, 0), M_1 = (8.2, 14.2028, 0)
    (60 degrees), M_2 = (0, 0, 40); 4 atoms at z = 20; periodic along M_0, M_1;
    20 bohr pair cutoff, 1% multiplicative noise, density cutoff 1e-6.  The
    grid spacing along the in-plane axes is 0.342 bohr, as in xe_monolayer."""
    a = 8.2
    p1 = np.array([a, 0.0, 0.0])
    p2 = np.array([a / 2.0, a * math.sqrt(3.0) / 2.0, 0.0])
    cell = np.array([2 * p1, 2 * p2, [0.0, 0.0, 40.0]])
    atoms = [(tuple(i * p1 + j * p2 + np.array([0.0, 0.0, 20.0])), rare_gas_shells())
             for i in range(2) for j in range(2)]
    n = density_cell(dims, cell, atoms, periodic=(True, True, False))
    n = _noise(n, _rng(5), 0.01)
    w = _workload("xe_monolayer_hex", 5, n, np.diag(cell), (True, True, False), 1e-6, 20.0, atoms=atoms)
    w["cell"] = cell
    return w


def rare_gas_chain(dims=(24, 72, 72)):
    """A chain of rare-gas atoms 8.2 bohr apart along x (one per 8.2 x 24 x 24 cell,
    at the centre of the cross-section), periodic along x only: the one-axis
    counterpart of xe_monolayer, with its grid spacing (0.34 bohr), 20 bohr pair
    cutoff, 1% multiplicative noise and density cutoff 1e-6."""
    L = (8.2, 24.0, 24.0)
    atoms = [((4.1, 12.0, 12.0), rare_gas_shells())]
    n = density(dims, L, atoms, periodic=(True, False, False))
    n = _noise(n, _rng(6), 0.01)
    return _workload("rare_gas_chain", 6, n, L, (True, False, False), 1e-6, 20.0, atoms=atoms)


def molecule24(dims=(64, 64, 64)):
    """24 atoms uniform in [3, 21]^3 (minimum separation 2.5 bohr) in a 24 bohr open
    cube; each Z / (8 pi a^3) exp(-r / a), a ~ U[0.4, 0.9], Z from {1, 4, 6}."""
    rng = _rng(2)
    pos = []
    while len(pos) < 24:
        p = rng.uniform(3.0, 21.0, size=3)
        if all(np.linalg.norm(p - q) >= 2.5 for q in pos):
            pos.append(p)
    a = rng.uniform(0.4, 0.9, size=24)
    Z = rng.choice(np.array([1.0, 4.0, 6.0]), size=24)
    L = (24.0, 24.0, 24.0)
    atoms = [(tuple(p), single_exponential(z, aa)) for p, z, aa in zip(pos, Z, a)]
    n = density(dims, L, atoms)
    return _workload("molecule24", 2, n, L, (False, False, False), 1e-6, 0.0, atoms=atoms)


def _round_half_up(x):
    return int(math.floor(x + 0.5))


def binding_curve():
    """16 rare-gas dimers at separations 6.0 .. 12.0 bohr (step 0.4) plus a single
    atom in the smallest and in the largest cell; 0.5 bohr spacing, open cells,
    nx = 32 + 4 round(8 (s - 6)/6), ny = nz = 24 + 4 round(2 (s - 6)/6).
    Returns a list of workloads (instances); atoms sit at the cell centre +- s/2."""
    out = []
    for k in range(16):
        s = 6.0 + 0.4 * k
        nx = 32 + 4 * _round_half_up(8.0 * (s - 6.0) / 6.0)
        ny = 24 + 4 * _round_half_up(2.0 * (s - 6.0) / 6.0)
        dims = (nx, ny, ny)
        L = tuple(0.5 * d for d in dims)
        c = np.array(L) / 2.0
        atoms = [((c[0] - s / 2, c[1], c[2]), rare_gas_shells()),
                 ((c[0] + s / 2, c[1], c[2]), rare_gas_shells())]
        out.append(_workload("dimer_%.1f" % s, 3, density(dims, L, atoms), L,
                             (False, False, False), 1e-6, 0.0, separation=s, atoms=atoms))
    for dims in ((32, 24, 24), (64, 32, 32)):
        L = tuple(0.5 * d for d in dims)
        c = tuple(x / 2.0 for x in L)
        atoms = [(c, rare_gas_shells())]
        out.append(_workload("atom_%dx%dx%d" % dims, 3, density(dims, L, atoms), L,
                             (False, False, False), 1e-6, 0.0, separation=None, atoms=atoms))
    return out


def slab_adsorbate(dims=(128, 112, 200)):
    """4-layer fcc(111)-like slab, 36 atoms a layer (nearest neighbours 5 bohr, layers
    at z = 8 + k 5 sqrt(2/3), ABC stacking), each Z = 11, a = 0.6; a 30-atom flat
    flake 6 bohr above the top layer: 6 Z=6 atoms at radius 2.7, 12 Z=6 at 5.0 and
    12 Z=1 at 7.0 around the cell centre, a ~ U[0.4, 0.7].  Cell 30 x 26 x 48,
    periodic x, y, 20 bohr pair cutoff, 0.5% noise, density cutoff 1e-5."""
    rng = _rng(4)
    L = (30.0, 26.0, 48.0)
    atoms = []
    dz = 5.0 * math.sqrt(2.0 / 3.0)
    for k in range(4):
        sx, sy = 2.5 * k, (26.0 / 18.0) * k
        for j in range(6):
            for i in range(6):
                x = (i * 5.0 + (j % 2) * 2.5 + sx) % L[0]
                y = (j * 26.0 / 6.0 + sy) % L[1]
                atoms.append(((x, y, 8.0 + k * dz), single_exponential(11.0, 0.6)))
    zf = 8.0 + 3 * dz + 6.0
    ring = [(2.7, 6, 6.0), (5.0, 12, 6.0), (7.0, 12, 1.0)]
    flake = []
    for rad, cnt, Z in ring:
        for m in range(cnt):
            t = 2.0 * math.pi * m / cnt
            flake.append(((15.0 + rad * math.cos(t), 13.0 + rad * math.sin(t), zf), Z))
    a_fl = rng.uniform(0.4, 0.7, size=len(flake))
    for (p, Z), a in zip(flake, a_fl):
        atoms.append((p, single_exponential(Z, a)))
    n = density(dims, L, atoms, periodic=(True, True, False))
    n = _noise(n, rng, 0.005)
    return _workload("slab_adsorbate", 4, n, L, (True, True, False), 1e-5, 20.0, atoms=atoms)


def config(idx, dims=None):
    """Workload ``idx`` (0..4) at its standard grid, or on ``dims`` (same cell)."""
    makers = {0: kr_dimer, 1: xe_monolayer, 2: molecule24, 4: slab_adsorbate}
    if idx == 3:
        return binding_curve()
    if idx not in makers:
        raise ValueError("workload index must be 0..4")
    return makers[idx]() if dims is None else makers[idx](dims)
