"""The oracle's pins are strong enough to catch plausible mistakes: each mutation
below plants one (a dropped factor, a wrong sign, an index swapped, a wrong
coefficient) in a copy of oracle/vpm_oracle.c, builds it, and runs the pin tests
against it in a subprocess; every mutant must make at least one pin fail.  The same
is done for the oracle's near-wake time loop (oracle/wake_loop.py)."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "vpm_oracle.c")
PINS = ["tests/test_oracle_blob.py", "tests/test_oracle_segments.py", "tests/test_oracle_local.py",
        "tests/test_oracle_rk3_lu_adjoint.py", "tests/test_oracle_wake.py"]

MUTATIONS = {
    "taylor_denominator": ("qs += term / (2.0 * k + 3.0);", "qs += term / (2.0 * k + 5.0);"),
    "closed_form_drops_rho": ("const double g = erf(rho / sqrt(2.0)) - SQRT_2_OVER_PI * rho * e;",
                              "const double g = erf(rho / sqrt(2.0)) - SQRT_2_OVER_PI * e;"),
    "kernel_2pi": ("*K = q / (4.0 * PI * s3);", "*K = q / (2.0 * PI * s3);"),
    "cross_sign": ("out[0] = p[1] * q[2] - p[2] * q[1];", "out[0] = p[2] * q[1] - p[1] * q[2];"),
    "gradient_transposed": ("Ji[3 * a + b] += K * t + H * c[a] * r[b];", "Ji[3 * a + b] += K * t + H * c[b] * r[a];"),
    "segment_d_sign": ("const double d = dot(r0, r1) / n1 - dot(r0, r2) / n2;",
                       "const double d = dot(r0, r1) / n1 + dot(r0, r2) / n2;"),
    "vatistas_core_length": ("const double e = pow(rc * L, 2.0 * vn);", "const double e = pow(rc, 2.0 * vn);"),
    "vreman_delta": ("be[i][j] = delta * delta * s;", "be[i][j] = delta * s;"),
    "stretch_not_transposed": ("t += classic ? Jp[3 * a + b] * G[b] : Jp[3 * b + a] * G[b];",
                               "t += classic ? Jp[3 * a + b] * G[b] : Jp[3 * a + b] * G[b];"),
    "pse_factor": ("p[a] = 2.0 / (sigma * sigma) * acc[a];", "p[a] = 1.0 / (sigma * sigma) * acc[a];"),
    "stretch_dropped": ("            s[3 * p + a] = t;", "            s[3 * p + a] = 0.0 * t;"),
    "rk3_coefficient": ("-153.0 / 128.0", "-153.0 / 126.0"),
    "lu_no_pivoting": ("if (fabs(A[n * i + k]) > fabs(A[n * piv + k])) piv = i;", "if (0) piv = i;"),
    "adjoint_sign": ("ax[b] -= t;", "ax[b] += t;"),
    "aic_normal_index": ("A[n * k + l] = dot(tot, &normal[4 * k]);", "A[n * k + l] = dot(tot, &normal[4 * l]);"),
    "wake_count_floor": ("const double v = ceil((len / ds_tip) * (double)n_tip);",
                         "const double v = floor((len / ds_tip) * (double)n_tip);"),
    "wake_position_offset": ("const double t = ((double)k + 0.5) / (double)n;", "const double t = (double)k / (double)n;"),
    "wake_neighbour_sign": ("? gamma[i] - gamma_nb[i] : gamma[i]; /* Eq. 7 */", "? gamma[i] + gamma_nb[i] : gamma[i]; /* Eq. 7 */"),
    "wake_back_edge_direction": ("memcpy(&a[3 * e], &D[3 * (p + 1)], 3 * sizeof(double));\n        memcpy(&b[3 * e], &D[3 * p], 3 * sizeof(double));",
                                 "memcpy(&a[3 * e], &D[3 * p], 3 * sizeof(double));\n        memcpy(&b[3 * e], &D[3 * (p + 1)], 3 * sizeof(double));"),
}


def _run_pins(src_text, tmp_path):
    mutant = tmp_path / "mutant.c"
    mutant.write_text(src_text)
    lib = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", str(lib), str(mutant), "-lm"],
                   check=True)
    env = dict(os.environ, VPM_ORACLE_LIB=str(lib), OMP_NUM_THREADS="4")
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *PINS], cwd=ROOT,
                          env=env, capture_output=True, text=True, timeout=600)


@pytest.mark.slow
def test_unmutated_copy_passes_the_pins(tmp_path):
    res = _run_pins(open(SRC).read(), tmp_path)
    assert res.returncode == 0, res.stdout[-2000:]


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    res = _run_pins(src.replace(old, new), tmp_path)
    assert res.returncode != 0, f"no pin caught mutation {name}:\n{res.stdout[-2000:]}"


# Mistakes planted in the oracle's near-wake time loop (oracle/wake_loop.py) and in its
# blade kinematics (oracle/kinematics.py): a copy of the oracle package with the mutated
# file is put first on the import path of a subprocess that runs the pins (the C
# routines are the unmutated library).  The kinematics mutants run against the
# kinematics pins without the comparison with the product's generator, so that the
# oracle's own pins (schedules read back, central differences, hover) must catch them.
LOOP_PINS = ["tests/test_oracle_wake_loop.py"]
KIN_PINS = ["tests/test_oracle_kinematics.py", "-k", "not agrees"]
LOOP_MUTATIONS = {
    "nodes_drop_free_stream": ("wake_loop.py", LOOP_PINS,
                               "self.nodes = (pts + self.dt * (_f32(u_n) + self.u_inf)).reshape(self.nodes.shape)",
                               "self.nodes = (pts + self.dt * _f32(u_n)).reshape(self.nodes.shape)"),
    "particles_drop_free_stream": ("wake_loop.py", LOOP_PINS, "seg_core=self.core, u_inf=self.u_inf, cast_f32=True)",
                                   "seg_core=self.core, cast_f32=True)"),
    "kutta_sign": ("wake_loop.py", LOOP_PINS, "shed = -gam[te_idx.ravel()].reshape(1, self.nb, self.S)",
                   "shed = gam[te_idx.ravel()].reshape(1, self.nb, self.S)"),
    "flap_rate_sign": ("kinematics.py", KIN_PINS, "- dbe * (Z @ _dry(-be) @ X)", "+ dbe * (Z @ _dry(-be) @ X)"),
    "flap_about_wrong_axis": ("kinematics.py", KIN_PINS, "Z, Y, X = _rz(psi), _ry(-be), _rx(th)",
                              "Z, Y, X = _rz(psi), _ry(be), _rx(th)"),
    "pitch_schedule_sine_sign": ("kinematics.py", KIN_PINS, "a = c0 + c1c * np.cos(psi) + c1s * np.sin(psi)",
                                 "a = c0 + c1c * np.cos(psi) - c1s * np.sin(psi)"),
    "v_rel_sign": ("kinematics.py", KIN_PINS, "v_rel.append(u_inf - np.cross(w, y - hub))",
                   "v_rel.append(u_inf + np.cross(w, y - hub))"),
}


def _run_loop_pins(fname, text, pins, tmp_path):
    import glob
    import shutil

    pkg = tmp_path / "oracle"
    pkg.mkdir()
    for f in glob.glob(os.path.join(ROOT, "oracle", "*.py")):
        shutil.copy(f, pkg / os.path.basename(f))
    (pkg / fname).write_text(text)
    os.symlink(os.path.join(ROOT, "paper_2511_11430_gb300"), tmp_path / "paper_2511_11430_gb300")
    os.symlink(os.path.join(ROOT, "tests"), tmp_path / "tests")
    lib = os.path.join(ROOT, "oracle", "liboracle.so")
    env = dict(os.environ, VPM_ORACLE_LIB=lib, OMP_NUM_THREADS="4")
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *pins],
                          cwd=str(tmp_path), env=env, capture_output=True, text=True, timeout=900)


@pytest.mark.slow
def test_unmutated_loop_passes_its_pins(tmp_path):
    import oracle

    oracle.build()
    src = open(os.path.join(ROOT, "oracle", "wake_loop.py")).read()
    res = _run_loop_pins("wake_loop.py", src, LOOP_PINS + ["tests/test_oracle_kinematics.py"], tmp_path)
    assert res.returncode == 0, res.stdout[-2000:]


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(LOOP_MUTATIONS))
def test_loop_pins_catch_planted_mistake(name, tmp_path):
    import oracle

    oracle.build()
    fname, pins, old, new = LOOP_MUTATIONS[name]
    src = open(os.path.join(ROOT, "oracle", fname)).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    res = _run_loop_pins(fname, src.replace(old, new), pins, tmp_path)
    assert res.returncode != 0, f"no pin caught mutation {name}:\n{res.stdout[-2000:]}"
