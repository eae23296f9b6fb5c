"""Do the oracle's pins catch plausible mistakes?

Each case plants one mistake in a temporary copy of the oracle's C source (a
dropped factor, a flipped sign, a transposed or shifted index, a wrong axis, a
perturbed coefficient), compiles that copy and runs the oracle pin tests
(tests/test_oracle_*.py) against it in a subprocess; at least one pin must
fail.  The real oracle is never modified."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PIN_FILES = ["test_oracle_stencils.py", "test_oracle_rk.py", "test_oracle_physics.py"]

# name: (text in oracle/fd_oracle.c, mistaken text); each original occurs exactly once.
# (Storing the velocity gradients transposed is not among them: the residual uses
# only their diagonal and the symmetric sum tau_ij G_ij, so it computes the same.)
MUTATIONS = {
    # first and second differences (Section 2, fourth-order central stencils)
    "d1_scale": ("(8.0 * (fp1 - fm1) - (fp2 - fm2)) / (12.0 * h)", "(8.0 * (fp1 - fm1) - (fp2 - fm2)) / (12.5 * h)"),
    "d1_outer_sign": ("(8.0 * (fp1 - fm1) - (fp2 - fm2)) / (12.0 * h)", "(8.0 * (fp1 - fm1) + (fp2 - fm2)) / (12.0 * h)"),
    "d2_centre_weight": ("- 30.0 * f0 +", "- 29.0 * f0 +"),
    "d2_wrong_tap": ("16.0 * fp1 - fp2)", "16.0 * fp1 - fm2)"),
    # initial condition and equation of state (Section 3; Eqs. 6-7)
    "ic_pressure": ("(cos(2.0 * z) + 2.0) / 16.0", "(cos(2.0 * z) + 2.0) / 15.0"),
    "eos_half_dropped": ("(Q[4 * n + q] - 0.5 * rho * (u * u + v * v + w * w))",
                         "(Q[4 * n + q] - rho * (u * u + v * v + w * w))"),
    "temperature_mach_power": ("prim[4 * n + q] = gamma * mach * mach * p / rho;",
                               "prim[4 * n + q] = gamma * mach * p / rho;"),
    # residual (Eqs. 1-5, skew-symmetric convection, expanded viscous terms)
    "skew_half_dropped": ("Rf[q] -= 0.5 * (d[q] + u[j][q] * d2[q] + rphi[q] * divj[q]);",
                          "Rf[q] -= (d[q] + u[j][q] * d2[q] + rphi[q] * divj[q]);"),
    "skew_weights": ("Rf[q] -= 0.5 * (d[q] + u[j][q] * d2[q] + rphi[q] * divj[q]);",
                     "Rf[q] -= 0.5 * (d[q] + 1.5 * u[j][q] * d2[q] + 0.5 * rphi[q] * divj[q]);"),
    "convection_wrong_axis": ("or_d1(rphi, nx, ny, nz, j, h[j], d2);", "or_d1(rphi, nx, ny, nz, (j + 1) % 3, h[j], d2);"),
    "pressure_gradient_sign": ("for (long q = 0; q < n; ++q) Rm[q] -= d[q];",
                               "for (long q = 0; q < n; ++q) Rm[q] += d[q];"),
    "pressure_work_axis": ("or_d1(work, nx, ny, nz, j, h[j], d);\n        double* RE",
                           "or_d1(work, nx, ny, nz, (j + 1) % 3, h[j], d);\n        double* RE"),
    "viscous_third_dropped": ("visc[q] += d2[q] / 3.0;", "visc[q] += 0.0 * d2[q];"),
    "mixed_as_pure_second": ("if (k == i)\n                or_d2", "if (1)\n                or_d2"),
    "heat_flux_sign": ("RE[q] += kappa * d2[q];", "RE[q] -= kappa * d2[q];"),
    "stress_index": ("s += tau * G[(3 * i + j) * n + q];", "s += tau * G[(3 * i + i) * n + q];"),
    "viscous_work_dropped": ("RE[q] += u[i][q] * (nu * visc[q]);", "RE[q] += 0.0;"),
    "pressure_work_sign": ("for (long q = 0; q < n; ++q) RE[q] -= d[q];", "for (long q = 0; q < n; ++q) RE[q] += d[q];"),
    "viscosity_scale": ("double nu = 1.0 / P->Re;", "double nu = 1.0 / (2.0 * P->Re);"),
    "conductivity_prandtl_dropped": ("P->Mach * P->Mach * P->Pr * P->Re);", "P->Mach * P->Mach * P->Re);"),
    "dissipation_two_thirds": ("(i == j ? 2.0 / 3.0 * dk : 0.0)", "(i == j ? 1.0 / 3.0 * dk : 0.0)"),
    "dissipation_symmetric_part": ("G[(3 * i + j) * n + q] + G[(3 * j + i) * n + q] -",
                                   "G[(3 * i + j) * n + q] + G[(3 * i + j) * n + q] -"),
    "divergence_index": ("double dk = G[0 * n + q] + G[4 * n + q] + G[8 * n + q];",
                         "double dk = G[0 * n + q] + G[4 * n + q] + G[7 * n + q];"),
    "ic_velocity_sign": ("double v = -cos(x) * sin(y) * cos(z);", "double v = cos(x) * sin(y) * cos(z);"),
    "d1_wrapped_tap": ("double* out) {\n#pragma omp parallel for schedule(static)\n    for (int z = 0; z < nz; ++z)\n"
                       "        for (int y = 0; y < ny; ++y)\n            for (int x = 0; x < nx; ++x) {\n"
                       "                double fm2, fm1, fp1, fp2;\n                if (axis == 0) {\n"
                       "                    fm2 = f[at(nx, ny, wrap(x - 2, nx), y, z)];",
                       "double* out) {\n#pragma omp parallel for schedule(static)\n    for (int z = 0; z < nz; ++z)\n"
                       "        for (int y = 0; y < ny; ++y)\n            for (int x = 0; x < nx; ++x) {\n"
                       "                double fm2, fm1, fp1, fp2;\n                if (axis == 0) {\n"
                       "                    fm2 = f[at(nx, ny, wrap(x - 3, nx), y, z)];"),
    # low-storage RK3 (Section 2, Fig. 1)
    "rk_a_coefficient": ("{2.0 / 3.0, 5.0 / 12.0, 3.0 / 5.0}", "{2.0 / 3.0, 5.0 / 12.0, 0.6000001}"),
    "rk_b_coefficient": ("{1.0 / 4.0, 3.0 / 20.0, 0.0}", "{1.0 / 4.0, 3.0 / 19.0, 0.0}"),
    "rk_register_kept_one_stage_short": ("if (s < 2) Qs[q] = qs + OR_RK_B[s] * dt * R[q];",
                                         "if (s < 1) Qs[q] = qs + OR_RK_B[s] * dt * R[q];"),
    # diagnostics (Section 3)
    "vorticity_sign": ("double oy = G[(3 * 0 + 2) * n + q] - G[(3 * 2 + 0) * n + q];",
                       "double oy = G[(3 * 0 + 2) * n + q] + G[(3 * 2 + 0) * n + q];"),
    "kinetic_energy_unweighted": ("a += 0.5 * rho * (u * u + v * v + w * w);", "a += 0.5 * (u * u + v * v + w * w);"),
}


def _copy_tree(dst):
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(dst, "oracle"),
                    ignore=shutil.ignore_patterns("*.so", "*.tmp*", "__pycache__"))
    tdst = os.path.join(dst, "tests")
    os.makedirs(tdst)
    for f in ["__init__.py", "conftest.py", "inputs.py"] + PIN_FILES:
        shutil.copy(os.path.join(ROOT, "tests", f), tdst)
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(tdst, "golden"))


def test_every_mutation_site_exists_once():
    src = open(os.path.join(ROOT, "oracle", "fd_oracle.c")).read()
    for name, (a, b) in MUTATIONS.items():
        assert src.count(a) == 1, name
        assert a != b, name


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, tmp_path):
    a, b = MUTATIONS[name]
    _copy_tree(str(tmp_path))
    path = os.path.join(str(tmp_path), "oracle", "fd_oracle.c")
    src = open(path).read()
    with open(path, "w") as f:
        f.write(src.replace(a, b, 1))
    env = dict(os.environ, PYTHONPATH=str(tmp_path), OMP_NUM_THREADS="4")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider"]
                       + [os.path.join("tests", f) for f in PIN_FILES],
                       cwd=str(tmp_path), env=env, capture_output=True, text=True, timeout=600)
    # pytest exit code 1: tests ran and at least one failed (2-5: harness problems)
    assert r.returncode == 1 and " failed" in r.stdout, (name, r.returncode, r.stdout[-2000:], r.stderr[-2000:])
