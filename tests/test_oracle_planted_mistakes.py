"""The oracle's pins catch plausible mistakes.

No GPU.  Each case copies the oracle, the input generators and the tests
into a temporary directory, plants one mistake in the copied oracle (a
dropped term, a wrong sign, a swapped operand or index, a wrong step), runs
the pins that should catch it, and requires at least one of them to fail.
The repository's own oracle is never modified.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (oracle file, original text, planted text, pins to run)
PLANTS = [
    ("sw_lagmean.py", "Nu = self.f0 * vh + self.spec(zeta * v) - self.dx(B)",
     "Nu = -self.f0 * vh + self.spec(zeta * v) - self.dx(B)",
     "tests/test_oracle_pins.py::test_uniform_inertial_oscillation"),
    ("sw_lagmean.py", 'out["P"] = [s * uh_adv - self.spec(adx), s * vh_adv - self.spec(ady)]',
     'out["P"] = [-self.spec(adx), -self.spec(ady)]',
     "tests/test_oracle_pins.py::test_uniform_advection_strategy1_closed_form"),
    ("sw_lagmean.py", "return 1j * self.ky * zh * inv, -1j * self.kx * zh * inv",
     "return 1j * self.kx * zh * inv, -1j * self.ky * zh * inv",
     "tests/test_oracle_euler2d.py::test_velocity_from_vorticity_and_steady_cellular_flow"),
    ("sw_lagmean.py", "wx = 0.5 * au", "wx = 1.0 * au",
     "tests/test_oracle_steppers.py::test_strategy2_uniform_flow_exact"),
    ("sw_lagmean.py", 'even = lm["done"] % 2 == 0', 'even = lm["done"] % 2 == 1',
     "tests/test_oracle_steppers.py::test_xi_first_uniform_flow_exact"),
    ("gbla.py", "ddx, ddy = -dt * ux, -dt * uy", "ddx, ddy = dt * ux, dt * uy",
     "tests/test_oracle_gbla.py::test_one_cell_per_step_matches_characteristic_sums"),
    ("remap.py", "return fbar, X + xi_x, Y + xi_y, resid", "return fbar, X - xi_x, Y - xi_y, resid",
     "tests/test_oracle_remap.py::test_whole_cell_shift_is_an_exact_roll"),
    ("sw_lagmean.py", "yn = m(lambda yy, aa, bb, e: e * e * yy + (dt / 2.0) * (e * e * aa + bb), y, a, b, E)",
     "yn = m(lambda yy, aa, bb, e: e * e * yy + (dt / 2.0) * (aa + bb), y, a, b, E)",
     "tests/test_oracle_steppers.py::test_laplacian_integrating_factor_exact"),
    ("sw_lagmean.py", "e_h = np.ones_like(k8) if self.visc_p == 1 else e_sw", "e_h = e_sw",
     "tests/test_oracle_steppers.py::test_viscosity_placement_on_depth"),
    ("remap.py", "return {k: bilinear_at_displacement(v, pos_x - X, pos_y - Y) for k, v in fields.items()}",
     "return {k: bilinear_at_displacement(v, X - pos_x, Y - pos_y) for k, v in fields.items()}",
     "tests/test_oracle_diagnostics.py::test_lift_exact_cases"),
    ("remap.py", "np.add.at(out, sh[box], 0.5 * np.abs(F[box]) ** 2)", "np.add.at(out, sh[box], np.abs(F[box]) ** 2)",
     "tests/test_oracle_diagnostics.py::test_spectrum_single_modes_and_box"),
]


@pytest.mark.parametrize("fname,orig,planted,pins", PLANTS, ids=[f"{p[0]}:{i}" for i, p in enumerate(PLANTS)])
def test_planted_mistake_fails_a_pin(tmp_path, fname, orig, planted, pins):
    for d in ("oracle", "sw_inputs", "tests"):
        shutil.copytree(os.path.join(ROOT, d), tmp_path / d,
                        ignore=shutil.ignore_patterns("__pycache__", "*.pyc"))
    target = tmp_path / "oracle" / fname
    text = target.read_text()
    assert text.count(orig) == 1, "the planted line is not where this test expects it"
    target.write_text(text.replace(orig, planted))
    env = dict(os.environ, PYTHONDONTWRITEBYTECODE="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", pins],
                       cwd=tmp_path, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1, r.stdout[-2000:] + r.stderr[-2000:]
