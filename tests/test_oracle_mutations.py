"""The oracle's pins catch plausible mistakes.  Each case plants one mistake in a
copy of oracle/oracle.c (a flipped sign, a wrong index, a dropped term or
factor, a mistyped constant, a shifted boundary), builds it with gcc into a
temporary library, loads it in place of the oracle's own, and checks that the
pin meant to guard that part now fails.  The oracle itself is never changed;
the last cases do the same to the numpy FFT gradient by substituting
functions for the duration of the test."""
import os
import subprocess

import numpy as np
import pytest

from conftest import ROOT

import test_oracle_cell as CELL
import test_oracle_far as FAR
import test_oracle_kernel as K
import test_oracle_phi0 as PHI0
import test_oracle_q0 as Q
import test_oracle_semilocal as SEMI
import test_oracle_spectral as SP
import test_oracle_spline as SPL
import test_oracle_sum as SUM

ORACLE_C = os.path.join(ROOT, "oracle", "oracle.c")

# (name, text in oracle.c, planted text, occurrence, pin, its arguments: a
#  string names a fixture, anything else is passed as it is)
MUTATIONS = [
    ("W: sign of the cos a cos b term",
     "return 2.0 * (sa * ub + sb * ua - 3.0 * ua * ub);",
     "return 2.0 * (sa * ub + sb * ua + 3.0 * ua * ub);", 0,
     K.test_W_matches_printed_formula_high_precision, ("oracle_mod",)),
    ("T: y + z written y + x",
     "return 0.5 * (1.0 / (w + x) + 1.0 / (y + z)) *",
     "return 0.5 * (1.0 / (w + x) + 1.0 / (y + x)) *", 0,
     K.test_phi_symmetric_in_arguments, ("oracle_mod",)),
    ("q0: s instead of s^2 in the gradient term",
     "double exc0 = ec + ex * (1.0 - (Zab / 9.0) * s * s);",
     "double exc0 = ec + ex * (1.0 - (Zab / 9.0) * s);", 0,
     Q.test_q0_hand_values, ("oracle_mod",)),
    ("gradient stencil: +-1 neighbours swapped",
     "static const double orc_fd_c[5] = {1.0 / 12.0, -8.0 / 12.0, 0.0, 8.0 / 12.0, -1.0 / 12.0};",
     "static const double orc_fd_c[5] = {1.0 / 12.0, 8.0 / 12.0, 0.0, -8.0 / 12.0, -1.0 / 12.0};", 0,
     Q.test_gradient_fourier_symbol, ("oracle_mod",)),
    ("transposed stencil: shifted the wrong way",
     "jj[ax] = ((idx[ax] - o) % dims[ax] + dims[ax]) % dims[ax];",
     "jj[ax] = ((idx[ax] + o) % dims[ax] + dims[ax]) % dims[ax];", 0,
     Q.test_gradient_adjoint_identity, ("oracle_mod",)),
    # (beta3, beta4 and alpha1 are fitted to the QMC energies, which resolve about
    # 0.1 mHa; beta1 is fixed by the exact high-density constant c1)
    ("PW92: beta1 mistyped 7.5597",
     "PW_b1 = 7.5957", "PW_b1 = 7.5597", 0,
     Q.test_lda_correlation_high_density_constant, ("oracle_mod",)),
    ("pair sum: self term dropped",
     "a += n[i] * phi00;", "a += 0.0 * phi00;", 0,
     SUM.test_self_term_and_prefactor, ("oracle_mod", "oracle_spline")),
    ("pair sum: cutoff made exclusive",
     "if (rc > 0.0 && r2 > rc * rc * (1.0 + 1e-12)) continue;",
     "if (rc > 0.0 && r2 >= rc * rc * (1.0 - 1e-12)) continue;", 0,
     SUM.test_periodic_cutoff_counts, ("oracle_mod", "oracle_spline")),
    ("spline: end condition row 2 M0 + M1 written 4 M0 + M1",
     "sub = 0.0; diag = 2.0; sup = 1.0;", "sub = 0.0; diag = 4.0; sup = 1.0;", 0,
     SPL.test_spline_exact_on_cubics_meeting_boundary_conditions, ("oracle_mod",)),
    ("adjoint: the n_i factor of U dropped",
     "U[t] = n[i] * u;", "U[t] = u;", 0,
     SUM.test_potential_is_derivative_of_energy, ("oracle_mod", "oracle_spline", (0, 0, 0))),
    ("kernel: d delta/d d1 with (1 + ds) for (1 - ds)",
     "*rdphi1 = r * (0.5 * pD + (1.0 - ds) / (2.0 * D) * sgn * pd);",
     "*rdphi1 = r * (0.5 * pD + (1.0 + ds) / (2.0 * D) * sgn * pd);", 0,
     SPL.test_kernel_branches, ("oracle_mod", "oracle_spline")),
    ("general-cell gradient: reciprocal matrix transposed",
     "for (int k = 0; k < 3; ++k) g[k * N + m] = du[0] * B[k] + du[1] * B[3 + k] + du[2] * B[6 + k];",
     "for (int k = 0; k < 3; ++k) g[k * N + m] = du[0] * B[3 * k] + du[1] * B[3 * k + 1] + du[2] * B[3 * k + 2];",
     0, CELL.test_gradient_cell_fourier_symbol, ("oracle_mod", (1, 2, 1))),
    ("GGA exchange: mu s instead of mu s^2",
     "return 1.0 + kappa - kappa / (1.0 + pbe_mu() * s * s / kappa);",
     "return 1.0 + kappa - kappa / (1.0 + pbe_mu() * s / kappa);", 0,
     SEMI.test_enhancement_factor_limits, ("oracle_mod", 0.804)),
    ("kernel: gamma of h(y) = 1 - exp(-gamma y^2) as 4 pi/3",
     "const double gam = 4.0 * M_PI / 9.0;", "const double gam = 4.0 * M_PI / 3.0;", 0,
     K.test_phi_large_D_asymptote, ("oracle_mod", 0.0)),
    ("voxel diagonal: one tent factor (1 - |t|) dropped",
     "double wt = w[i] * w[j] * w[k] * (1.0 - x[i]) * (1.0 - x[j]) * (1.0 - x[k]);",
     "double wt = w[i] * w[j] * w[k] * (1.0 - x[i]) * (1.0 - x[j]);", 0,
     PHI0.test_monte_carlo_voxel_average, ("oracle_spline", 2.0)),
    ("general-cell pair sum: image shift with the transposed cell",
     "d[c] = ri[c] - rj[c] + m0 * cell[c] + m1 * cell[3 + c] + m2 * cell[6 + c];",
     "d[c] = ri[c] - rj[c] + m0 * cell[3 * c] + m1 * cell[3 * c + 1] + m2 * cell[3 * c + 2];", 0,
     CELL.test_skewed_pair_counts_brute_force, ("oracle_mod", "oracle_spline")),
    ("kernel: nu(y) = y^2/h without the 1/2",
     "return 0.5 * y * y / h;", "return y * y / h;", 0,
     K.test_phi_large_D_asymptote, ("oracle_mod", 0.0)),
    ("spline: the two linear basis weights swapped",
     "double al[2] = {1.0 - t, t};", "double al[2] = {t, 1.0 - t};", 0,
     SPL.test_spline_reproduces_nodes, ("oracle_mod",)),
    ("past the table: the larger argument taken for the smaller",
     "double dsmall = (d1 < d2) ? d1 : d2;", "double dsmall = (d1 < d2) ? d2 : d1;", 0,
     SPL.test_kernel_past_table_matches_quadrature, ("oracle_mod", "oracle_spline", 60.0)),
    ("past the table: the (1 - rho(0)) term dropped",
     "double g = rho + (1.0 - rho0) * (1.0 - Dr * Dr);", "double g = rho;", 0,
     SPL.test_kernel_tends_to_eq17_at_large_D, ("oracle_mod", "oracle_spline", 0.9)),
    ("past the table: the rho'(delta*) term of r dphi/dd1 with the wrong sign",
     "if (d1 < d2 && dstar > 0.0) rdg -= drho * r / Dmax;",
     "if (d1 < d2 && dstar > 0.0) rdg += drho * r / Dmax;", 0,
     SPL.test_kernel_branches, ("oracle_mod", "oracle_spline")),
    ("far tail: the normal separation |z| ignored (R = r_cut for every pair)",
     "double R = fabs(z) > rc ? fabs(z) : rc;", "double R = rc;", 0,
     FAR.test_two_axis_continuum_is_the_radial_integral, ("oracle_mod", False)),
    ("far tail: 2 pi / A written pi / A",
     "return (2.0 * M_PI / g->A) / (4.0 * R * R * R * R);", "return (M_PI / g->A) / (4.0 * R * R * R * R);", 0,
     FAR.test_continuum_approaches_the_lattice_sum, ("oracle_mod",)),
    ("far tail, one axis: the factor 2 of the two half-lines dropped",
     "return (2.0 / g->alen) * orc_line_tail_integral(rho, x0);",
     "return (1.0 / g->alen) * orc_line_tail_integral(rho, x0);", 0,
     FAR.test_one_axis_continuum_is_the_offset_average_of_the_lattice_sum, ("oracle_mod", 10.0)),
    ("far tail, one axis: rho taken as the full distance (axial part not removed)",
     "double p2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] - z * z;",
     "double p2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];", 0,
     FAR.test_one_axis_continuum_is_the_line_integral, ("oracle_mod",)),
    ("far tail, one axis: no allowance at rho = r_cut (rounding decides x0)",
     "double x0 = t > 1e-12 * rc * rc ? sqrt(t) : 0.0;", "double x0 = t > 0.0 ? sqrt(t) : 0.0;", 0,
     FAR.test_one_axis_factor_at_the_cutoff_radius, ("oracle_mod",)),
    ("line integral: the series' alternating sign dropped",
     "sum += (k % 2) ? -term : term;", "sum += term;", 0,
     FAR.test_line_integral_matches_quadrature, ("oracle_mod", 2.0)),
    ("line integral: closed form's second term with (rho^2 + x0^2) once, not squared",
     "x0 / (4.0 * r2 * s2 * s2)", "x0 / (4.0 * r2 * s2)", 0,
     FAR.test_line_integral_matches_quadrature, ("oracle_mod", 7.0)),
    ("far tail's potential: the 1/(a + b) term of df/da dropped",
     "sb += n[j] * (-f * (1.0 / ui + 1.0 / (ui + uj))) * K;", "sb += n[j] * (-f * (1.0 / ui)) * K;", 0,
     FAR.test_tail_potential_is_derivative_of_tail, ("oracle_mod", "oracle_spline", (1, 1, 0))),
    ("PBE correlation: A^2 t^4 written A t^4",
     "double den = 1.0 + A * t2 + A * A * t2 * t2;", "double den = 1.0 + A * t2 + A * t2 * t2;", 0,
     SEMI.test_pbe_gradient_correction_limits, ("oracle_mod",)),
]


def _build_mutant(tmp_path, old, new, which):
    src = open(ORACLE_C).read()
    at = -1
    for _ in range(which + 1):
        at = src.index(old, at + 1)
    mutated = src[:at] + new + src[at + len(old):]
    c = os.path.join(tmp_path, "oracle_mutant.c")
    so = os.path.join(tmp_path, "liboracle_mutant.so")
    open(c, "w").write(mutated)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
                    "-o", so, c, "-lm"], check=True)
    return so


@pytest.mark.parametrize("case", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pin_catches_planted_mistake(oracle_mod, request, tmp_path, case):
    name, old, new, which, pin, spec = case
    so = _build_mutant(str(tmp_path), old, new, which)
    args = [request.getfixturevalue(f) if isinstance(f, str) else f for f in spec]
    real = oracle_mod.lib()
    # the pin passes on the oracle as it is ...
    pin(*args)
    # ... and fails with the mistake planted
    oracle_mod._LIB = oracle_mod.load_library(so)
    try:
        with pytest.raises(AssertionError):
            pin(*args)
    finally:
        oracle_mod._LIB = real


def _mutated_function(module, name, old, new):
    """module.name rebuilt from its own source with ``old`` replaced by ``new``."""
    import inspect
    import textwrap
    src = textwrap.dedent(inspect.getsource(getattr(module, name)))
    assert src.count(old) == 1, (name, old)
    ns = dict(module.__dict__)
    exec(compile(src.replace(old, new), "<mutant %s>" % name, "exec"), ns)
    return ns[name]


def _mutated_method(cls, name, old, new, module):
    """cls.name rebuilt from its own source with ``old`` replaced by ``new``."""
    import inspect
    import textwrap
    src = textwrap.dedent(inspect.getsource(getattr(cls, name)))
    assert src.count(old) == 1, (name, old)
    ns = dict(module.__dict__)
    exec(compile(src.replace(old, new), "<mutant %s.%s>" % (cls.__name__, name), "exec"), ns)
    return ns[name]


PY_MUTATIONS = [
    ("E: dV instead of dV^2", "energy", "E = 0.5 * self.dV ** 2 * float(np.dot(self.na, A))",
     "E = 0.5 * self.dV * float(np.dot(self.na, A))", SUM.test_self_term_and_prefactor,
     ("oracle_mod", "oracle_spline")),
    ("v: divergence term added with the wrong sign", "potential",
     "v = self.dV * (chi * (Ag + Ug * self.dq0dn.ravel()) + div)",
     "v = self.dV * (chi * (Ag + Ug * self.dq0dn.ravel()) - div)", SUM.test_potential_is_derivative_of_energy,
     ("oracle_mod", "oracle_spline", (0, 0, 0))),
]


@pytest.mark.parametrize("case", PY_MUTATIONS, ids=[m[0] for m in PY_MUTATIONS])
def test_pin_catches_planted_mistake_in_assembly(oracle_mod, request, monkeypatch, case):
    """The same for the grid-level assembly that the oracle does in Python."""
    name, method, old, new, pin, spec = case
    args = [request.getfixturevalue(f) if isinstance(f, str) else f for f in spec]
    pin(*args)
    monkeypatch.setattr(oracle_mod.Problem, method, _mutated_method(oracle_mod.Problem, method, old, new, oracle_mod))
    with pytest.raises(AssertionError):
        pin(*args)


def test_spectral_pins_catch_planted_mistakes(oracle_mod, monkeypatch):
    """The FFT gradient: frequencies 0..N-1 without aliasing the upper half to
    negative ones, and the transpose without its conjugate multipliers."""
    SP.test_plane_waves_exact(oracle_mod, (12, 10, 14), False)
    SP.test_adjoint_identity(oracle_mod, True)
    bad = _mutated_function(oracle_mod, "_spectral_multipliers", "m = np.fft.fftfreq(N, 1.0 / N)",
                            "m = np.arange(N, dtype=np.float64)")
    monkeypatch.setattr(oracle_mod, "_spectral_multipliers", bad)
    with pytest.raises(AssertionError):
        SP.test_plane_waves_exact(oracle_mod, (12, 10, 14), False)
    monkeypatch.undo()
    bad = _mutated_function(oracle_mod, "gradient_spectral_T", "np.conj(mult[a])", "mult[a]")
    monkeypatch.setattr(oracle_mod, "gradient_spectral_T", bad)
    with pytest.raises(AssertionError):
        SP.test_adjoint_identity(oracle_mod, True)
