"""The oracle's pins are sharp enough to catch plausible slips.

Each case copies oracle.c to a temporary directory, plants one mistake in the
copy (on the CPU, never in the committed file), rebuilds it and runs the pin
tests (forward, integrator, adjoint, the random-system properties and the FP32
listing restatement) against
the mutant; every mutant must fail at least one pin.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = {
    "force_exponent_1": ("w = mass[j] * rinv * rinv * rinv", "w = mass[j] * rinv * rinv"),
    "self_term_kept_with_softening": ("if (j == i) continue;\n        const double dx",
                                      "if (j == i && eps2 == 0.0) continue;\n        const double dx"),
    "potential_sign": ("p -= mass[j] * rinv;", "p += mass[j] * rinv;"),
    "transposed_coordinate": ("const double dy = pos[3 * j + 1] - yi", "const double dy = pos[3 * j + 0] - yi"),
    "softening_dropped": ("const double s = dx * dx + dy * dy + dz * dz + eps2;\n        const double rinv = 1.0 / sqrt(s);\n        const double w = mass[j]",
                          "const double s = dx * dx + dy * dy + dz * dz;\n        const double rinv = 1.0 / sqrt(s);\n        const double w = mass[j]"),
    "full_kick_instead_of_half": ("oracle_accel(n, pos, mass, eps, a, NULL);\n    const double h = 0.5 * dt;",
                                  "oracle_accel(n, pos, mass, eps, a, NULL);\n    const double h = dt;"),
    "sink_mass_instead_of_source": ("const double w = mass[j] *", "const double w = mass[i] *"),
    "drift_uses_old_velocity_sign": ("pos[k] += dt * vel[k];", "pos[k] -= dt * vel[k];"),
    "energy_half_missing": ("w += 0.5 * mass[i] * phi[i];", "w += mass[i] * phi[i];"),
    "vjp_tidal_factor_3_dropped": ("- 3.0 * s52 * d[a] * d[b]", "- s52 * d[a] * d[b]"),
    "vjp_sink_term_dropped": ("g[a] -= mass[i] * T[a][b] * lk[b];", "g[a] -= 0.0 * lk[b];"),
    "vjp_mass_gradient_sign": ("gm += (li[0] * d[0]", "gm -= (li[0] * d[0]"),
    "vjp_potential_masses_swapped": ("(mu[i] * mass[k] + mu[k] * mass[i])", "(mu[k] * mass[k] + mu[i] * mass[i])"),
    "adjoint_drift_uses_half_step": ("lv[k] += dt * gx0[k];", "lv[k] += h * gx0[k];"),
    "sink_source_pot_sign": ("p -= jmass[j] * rinv;", "p += jmass[j] * rinv;"),
    "sink_source_coordinate": ("jpos[3 * j + 2] - ipos[3 * i + 2]", "jpos[3 * j + 2] - ipos[3 * i + 1]"),
    "listing_fma_chain_reordered": ("fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, eps2)))",
                                    "fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)))"),
    "listing_weight_not_cubed": ("        w = w * (w * w);", "        w = w * w;"),
    "listing_rsqrt_rounded_once_in_fp64": ("float w = 1.0f / sqrtf(r2);", "float w = (float)(1.0 / sqrt((double)r2));"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(os.path.join(ROOT, "oracle", "oracle.c")).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found"
    shutil.copytree(os.path.join(ROOT, "oracle"), tmp_path / "oracle",
                    ignore=shutil.ignore_patterns("*.so", "*.tmp*", "__pycache__"))
    (tmp_path / "oracle" / "oracle.c").write_text(src.replace(old, new))
    shutil.copytree(os.path.join(ROOT, "nbody_inputs"), tmp_path / "nbody_inputs",
                    ignore=shutil.ignore_patterns("__pycache__"))
    os.makedirs(tmp_path / "tests")
    for f in ("conftest.py", "test_oracle_pins.py", "test_oracle_integrator.py", "test_oracle_adjoint.py",
              "test_oracle_properties.py", "test_oracle_listing_f32.py"):
        shutil.copy(os.path.join(ROOT, "tests", f), tmp_path / "tests" / f)
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        "tests/test_oracle_pins.py", "tests/test_oracle_integrator.py",
                        "tests/test_oracle_adjoint.py", "tests/test_oracle_properties.py",
                        "tests/test_oracle_listing_f32.py"],
                       cwd=tmp_path, capture_output=True, text=True, timeout=300)
    assert r.returncode == 1, f"mutant {name} passed every pin:\n{r.stdout[-2000:]}"
