"""Planted mistakes in the oracle: each case copies the oracle into a scratch directory,
plants one plausible slip in its C source (a dropped or doubled term, a wrong sign, a
shifted index, a transposed operand, a wrong stage time or weight, a wrong power of h)
and runs the pin that must catch it against that copy.  The repository's oracle is never
modified.

By default a representative case per oracle function runs (operator, profile, layout,
RK4, sources, energy, norms, walls, transpose, adjoint, dJ/dsigma); with
PML_ORACLE_MUTANTS=all every case runs.  Three further slips were tried and change
nothing, so no pin can catch them: the step guard of the interior-run search (it only
binds when the whole axis is free, where the other loop already covers it) and forcing
the support flags inside dJ/dsigma's contraction to 1 (the transposed stage vectors are
zero off the supports of Phi and Psi).
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = "tests/test_oracle_pins.py::"

# (name, original text, planted text, occurrence, pin that catches it, in the default set)
MUTANTS = [
    ("laplacian centre", "- 2.0 * U[i] + at(U, im)) / (h * h)", "- 1.9 * U[i] + at(U, im)) / (h * h)", 0,
     "test_plane_wave_is_eigenvector_1d_random_sigma", True),
    ("laplacian power of h", "at(U, im)) / (h * h);", "at(U, im)) / h;", 0, "test_plane_wave_dx_not_one", False),
    ("damping term sign", "pml += (s_i * at(Psi, ip) - s_im * at(Phi, im)) / h;",
     "pml += (s_i * at(Psi, ip) + s_im * at(Phi, im)) / h;", 0, "test_plane_wave_is_eigenvector_1d_random_sigma", False),
    ("damping term Psi index", "pml += (s_i * at(Psi, ip)", "pml += (s_i * at(Psi, im)", 0,
     "test_plane_wave_is_eigenvector_1d_random_sigma", True),
    ("damping term sigma swap", "pml += (s_i * at(Psi, ip) - s_im * at(Phi, im)) / h;",
     "pml += (s_im * at(Psi, ip) - s_i * at(Phi, im)) / h;", 0, "test_plane_wave_is_eigenvector_1d_random_sigma", False),
    ("damping term power of h", "- s_im * at(Phi, im)) / h;", "- s_im * at(Phi, im)) / (h * h);", 0,
     "test_plane_wave_dx_not_one", True),
    ("Phi sigma swap", "-0.5 * (s_im * at(Phi, im) + s_i * Phi[i]) - dU", "-0.5 * (s_i * at(Phi, im) + s_im * Phi[i]) - dU",
     0, "test_plane_wave_is_eigenvector_1d_random_sigma", False),
    ("Psi sigma swap", "-0.5 * (s_im * Psi[i] + s_i * at(Psi, ip)) - dU", "-0.5 * (s_i * Psi[i] + s_im * at(Psi, ip)) - dU",
     0, "test_plane_wave_is_eigenvector_1d_random_sigma", True),
    ("Phi half", "? -0.5 * (s_im * at(Phi, im)", "? -1.0 * (s_im * at(Phi, im)", 0,
     "test_plane_wave_is_eigenvector_1d_random_sigma", False),
    ("Phi gradient sign", "+ s_i * Phi[i]) - dU", "+ s_i * Phi[i]) + dU", 0,
     "test_plane_wave_is_eigenvector_1d_random_sigma", False),
    ("Psi gradient sign", "+ s_i * at(Psi, ip)) - dU", "+ s_i * at(Psi, ip)) + dU", 0,
     "test_plane_wave_is_eigenvector_1d_random_sigma", False),
    ("centred difference 2h", "double dU = (at(U, ip) - at(U, im)) / (2.0 * h);", "double dU = (at(U, ip) - at(U, im)) / h;",
     0, "test_plane_wave_is_eigenvector_1d_random_sigma", False),
    ("Phi support", "oPhi[i] = (s_i != 0.0) ? -0.5", "oPhi[i] = (s_im != 0.0) ? -0.5", 0,
     "test_plane_wave_is_eigenvector_1d_random_sigma", False),
    ("Psi support", "oPsi[i] = (s_im != 0.0) ? -0.5", "oPsi[i] = (s_i != 0.0) ? -0.5", 0,
     "test_dense_spectral_radius_stable", True),
    ("sigma of edge i-1", "const double s_im = g->sig[a][(c[a] - 1 + Ta) % Ta];",
     "const double s_im = g->sig[a][(c[a] + 1) % Ta];", 0, "test_plane_wave_is_eigenvector_1d_random_sigma", False),
    ("RK4 first stage", "for (j = 0; j < len; j++) Y[j] = y[j] + 0.5 * dt * k1[j];",
     "for (j = 0; j < len; j++) Y[j] = y[j] + dt * k1[j];", 0, "test_rk4_single_mode_exact", False),
    ("RK4 second stage", "Y[j] = y[j] + 0.5 * dt * k2[j];", "Y[j] = y[j] + dt * k2[j];", 0, "test_rk4_single_mode_exact",
     True),
    ("RK4 weights", "(k1[j] + 2.0 * k2[j] + 2.0 * k3[j] + k4[j])", "(k1[j] + 2.0 * k2[j] + 2.0 * k3[j] + 1.1 * k4[j])", 0,
     "test_rk4_single_mode_exact", False),
    ("RK4 stage time", "rhs(&g, Y, k3, sp, t + 0.5 * dt);", "rhs(&g, Y, k3, sp, t + dt);", 0,
     "test_source_stage_times_simpson", True),
    ("receiver sample", "trace[k * nr + r] = y[rec_idx[r]];", "trace[k * nr + r] = k1[rec_idx[r]];", 0,
     "test_adjoint_gradients_vs_central_differences", False),
    ("source sign", "oV[src->idx[s]] += src->amp[s] * orc_ricker", "oV[src->idx[s]] -= src->amp[s] * orc_ricker", 0,
     "test_source_stage_times_simpson", False),
    ("Ricker factor 2", "return (1.0 - 2.0 * a) * exp(-a);", "return (1.0 - a) * exp(-a);", 0,
     "test_source_stage_times_simpson", True),
    ("Ricker exponent", "return (1.0 - 2.0 * a) * exp(-a);", "return (1.0 - 2.0 * a) * exp(-0.5 * a);", 0,
     "test_source_stage_times_simpson", False),
    ("energy power of h", "double d = (at(y, shifted(&g, c, a, +1)) - y[i]) / h;",
     "double d = (at(y, shifted(&g, c, a, +1)) - y[i]);", 0, "test_rk4_single_mode_exact", True),
    ("energy elastic half", "return 0.5 * kin + 0.5 * ela;", "return 0.5 * kin + ela;", 0, "test_rk4_single_mode_exact",
     False),
    ("energy backward difference", "double d = (at(y, shifted(&g, c, a, +1)) - y[i]) / h;",
     "double d = (at(y, shifted(&g, c, a, -1)) - y[i]) / h;", 0, "test_energy_of_a_point_at_the_window_corners", True),
    ("energy window bound", "if (c[a] < lo[a] || c[a] > hi[a]) inside = 0;\n        if (!inside) continue;\n        kin",
     "if (c[a] < lo[a] || c[a] >= hi[a]) inside = 0;\n        if (!inside) continue;\n        kin", 0,
     "test_energy_is_additive_over_windows", False),
    ("norms L2", "s2 += U[i] * U[i];", "s2 += fabs(U[i]);", 0, "test_norms_over_a_window", False),
    ("norms window bound",
     "if (c[a] < lo[a] || c[a] > hi[a]) inside = 0;\n        if (!inside) continue;\n        if (fabs",
     "if (c[a] <= lo[a] || c[a] > hi[a]) inside = 0;\n        if (!inside) continue;\n        if (fabs", 0,
     "test_norms_over_a_window", True),
    ("norms distance", "if (ref) d2 += (U[i] - ref[i]) * (U[i] - ref[i]);",
     "if (ref) d2 += (U[i] - ref[i]) * (U[i] + ref[i]);", 0, "test_norms_over_a_window", False),
    ("profile depth", "if (a - 1 - e > d) d = a - 1 - e;", "if (a - e > d) d = a - e;", 0, "test_sigma_profile_shapes",
     True),
    ("profile power law", "pow((double)d / (double)w, order)", "pow((double)(d - 1) / (double)w, order)", 0,
     "test_sigma_profile_shapes", False),
    ("interior run reach", "for (k = -2; k <= 1; k++)", "for (k = -1; k <= 1; k++)", 0,
     "test_interior_run_is_where_layer_terms_vanish", True),
    ("Psi support table", "psi_active[i] = (uint8_t)(sig[(i - 1 + T) % T] != 0.0);",
     "psi_active[i] = (uint8_t)(sig[i] != 0.0);", 0, "test_interior_run_is_where_layer_terms_vanish", False),
    ("wall at the upper end", "if (g->wall && (d[a] + s < 0 || d[a] + s >= g->T[a])) return -1;",
     "if (g->wall && (d[a] + s < 0 || d[a] + s > g->T[a])) return -1;", 0, "test_wall_box_sine_mode_exact", True),
    ("wall at the lower end", "if (g->wall && (d[a] + s < 0 || d[a] + s >= g->T[a])) return -1;",
     "if (g->wall && (d[a] + s < -1 || d[a] + s >= g->T[a])) return -1;", 0, "test_wall_box_sine_mode_exact", False),
    ("transpose Laplacian power of h", "acc += (at(Vb, ip) - 2.0 * Vb[i] + at(Vb, im)) / (h * h);",
     "acc += (at(Vb, ip) - 2.0 * Vb[i] + at(Vb, im)) / h;", 0, "test_transpose_matches_dense", True),
    ("transpose Phi sign", "acc += (phib_p - phib_m) / (2.0 * h)", "acc += (phib_m - phib_p) / (2.0 * h)", 0,
     "test_transpose_matches_dense", False),
    ("transpose Psi support", "double psib_m = (g->sig[a][iamm] != 0.0)", "double psib_m = (g->sig[a][iam] != 0.0)", 0,
     "test_transpose_matches_dense", False),
    ("transpose Phi index", "oPhi[i] = (s_i != 0.0) ? -s_i * at(Vb, ip) / h", "oPhi[i] = (s_i != 0.0) ? -s_i * at(Vb, im) / h",
     0, "test_transpose_matches_dense", False),
    ("transpose Psi sign", "oPsi[i] = (s_im != 0.0) ? s_im * at(Vb, im) / h", "oPsi[i] = (s_im != 0.0) ? -s_im * at(Vb, im) / h",
     0, "test_transpose_matches_dense", False),
    ("transpose Psi pair", "- 0.5 * s_im * (psib_0 + psib_m)", "- 0.5 * s_im * (psib_0 - psib_m)", 0,
     "test_transpose_matches_dense", False),
    ("transpose V row", "out[n + i] = Ub[i];", "out[n + i] = 0.5 * Ub[i];", 0, "test_transpose_matches_dense", False),
    ("adjoint kb3 update", "for (j = 0; j < len; j++) { yb_out[j] += Yb[j]; kb3[j] += dt * Yb[j]; }",
     "for (j = 0; j < len; j++) { yb_out[j] += Yb[j]; kb3[j] += 0.5 * dt * Yb[j]; }", 0, "test_adjoint_dot_product", True),
    ("adjoint kb1 update", "for (j = 0; j < len; j++) { yb_out[j] += Yb[j]; kb1[j] += 0.5 * dt * Yb[j]; }",
     "for (j = 0; j < len; j++) { yb_out[j] += Yb[j]; kb1[j] += dt * Yb[j]; }", 0, "test_adjoint_dot_product", False),
    ("adjoint weights", "kb2[j] = dt / 3.0 * yb[j];", "kb2[j] = dt / 6.0 * yb[j];", 0, "test_adjoint_dot_product", False),
    ("adjoint source time", "+ orc_ricker(t + dt, f_peak, t_delay) * kb4[v];", "+ orc_ricker(t, f_peak, t_delay) * kb4[v];",
     0, "test_adjoint_gradients_vs_central_differences", True),
    ("adjoint source stages", "+ orc_ricker(t + 0.5 * dt, f_peak, t_delay) * (kb2[v] + kb3[v])",
     "+ orc_ricker(t + 0.5 * dt, f_peak, t_delay) * (kb2[v] + kb2[v])", 0,
     "test_adjoint_gradients_vs_central_differences", False),
    ("adjoint residual sign", "yb[rec_idx[r]] += residual[k * nr + r];", "yb[rec_idx[r]] -= residual[k * nr + r];", 0,
     "test_adjoint_gradients_vs_central_differences", False),
    ("dJ/dsigma kb3 update", "for (j = 0; j < len; j++) { yb_out[j] += Yb[j]; kb3[j] += dt * Yb[j]; }",
     "for (j = 0; j < len; j++) { yb_out[j] += Yb[j]; kb3[j] += 0.5 * dt * Yb[j]; }", 1,
     "test_grad_sigma_matches_central_differences", False),
    ("dJ/dsigma V entry", "sum += kV[i] * at(Psi, ip) / h;", "sum += kV[i] * Psi[i] / h;", 0,
     "test_grad_sigma_matches_central_differences", True),
    ("dJ/dsigma Phi half", "sum += -0.5 * kPhi[i] * Phi[i];", "sum += -1.0 * kPhi[i] * Phi[i];", 0,
     "test_grad_sigma_matches_central_differences", False),
    ("dJ/dsigma Psi entry", "sum += -0.5 * kPsi[i] * Psi[i];", "sum += -0.5 * kPsi[i] * at(Psi, im);", 0,
     "test_grad_sigma_matches_central_differences", False),
    ("dJ/dsigma stage pairing", "dA_contract(&g, a, e, kb2, Y2) +", "dA_contract(&g, a, e, kb2, Y3) +", 0,
     "test_grad_sigma_matches_central_differences", False),
    ("dJ/dsigma last stage input", "for (j = 0; j < len; j++) Y4[j] = y[j] + dt * k3[j];",
     "for (j = 0; j < len; j++) Y4[j] = y[j] + 0.5 * dt * k3[j];", 0, "test_grad_sigma_matches_central_differences", False),
    ("misfit half", "*J += 0.5 * d * d;", "*J += d * d;", 0, "test_grad_sigma_matches_central_differences", False),
]

_ALL = os.environ.get("PML_ORACLE_MUTANTS", "") == "all"
CASES = [m for m in MUTANTS if _ALL or m[5]]


def _replace_nth(s, old, new, n):
    i = -1
    for _ in range(n + 1):
        i = s.index(old, i + 1)
    return s[:i] + new + s[i + len(old):]


@pytest.fixture(scope="module")
def tree(tmp_path_factory):
    """A scratch copy of what the pins import: the oracle, the seeded input generator, the
    binding (for the layer-design call one pin makes) and the pins with their fixtures."""
    lib = os.path.join(ROOT, "paper_1804_01390_gb300", "_build", "libpml.so")
    if not os.path.exists(lib):
        pytest.skip("libpml.so is not built")
    d = tmp_path_factory.mktemp("mutants")
    os.makedirs(d / "oracle")
    shutil.copy(os.path.join(ROOT, "oracle", "__init__.py"), d / "oracle")
    os.makedirs(d / "paper_1804_01390_gb300")
    for f in ("__init__.py", "workloads.py", "_lib.py"):
        shutil.copy(os.path.join(ROOT, "paper_1804_01390_gb300", f), d / "paper_1804_01390_gb300")
    os.symlink(os.path.join(ROOT, "paper_1804_01390_gb300", "_build"), d / "paper_1804_01390_gb300" / "_build")
    os.makedirs(d / "tests")
    for f in ("__init__.py", "conftest.py", "test_oracle_pins.py", "test_golden_figures.py"):
        shutil.copy(os.path.join(ROOT, "tests", f), d / "tests")
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), d / "tests" / "golden")
    return d


def _pins(tree, source, tests):
    open(tree / "oracle" / "pml_oracle.c", "w").write(source)
    shutil.rmtree(tree / "oracle" / "_build", ignore_errors=True)
    return subprocess.run([sys.executable, "-m", "pytest", *[PINS + t for t in tests], "-x", "-q",
                           "-p", "no:cacheprovider"], cwd=tree, capture_output=True, text=True, timeout=900)


def test_unmodified_copy_passes(tree):
    """The copy with the oracle as it is passes every pin the cases below use."""
    src = open(os.path.join(ROOT, "oracle", "pml_oracle.c")).read()
    r = _pins(tree, src, sorted({m[4] for m in CASES}))
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("name,old,new,nth,pin,default", CASES, ids=[m[0] for m in CASES])
def test_planted_mistake_is_caught(tree, name, old, new, nth, pin, default):
    src = open(os.path.join(ROOT, "oracle", "pml_oracle.c")).read()
    assert src.count(old) > nth, "the text to change is not in the oracle any more"
    r = _pins(tree, _replace_nth(src, old, new, nth), [pin])
    assert r.returncode == 1 and " failed" in r.stdout, (name, r.stdout[-1500:])
