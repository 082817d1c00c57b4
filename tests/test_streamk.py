"""Host-side check of the stream-K work split of the pair sweeps (no GPU): the
helper in csrc/vpm_common.cuh is compiled for the host by nvcc and exercised over
many tile counts, unit weights and grid sizes."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_stream_k_split_covers_every_unit_once(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc) and shutil.which("nvcc") is None:
        pytest.skip("nvcc not available")
    exe = tmp_path / "streamk_check"
    src = os.path.join(ROOT, "tests", "host", "streamk_check.cu")
    inc = os.path.join(ROOT, "paper_2511_11430_gb300", "csrc")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-O1", "-I" + inc, src, "-o",
                    str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.startswith("OK"), out.stdout + out.stderr


def test_near_field_series_coefficients_match_oracle(tmp_path):
    """The kernels' incomplete-gamma series for q = g/rho^3 and f = F/rho^5, evaluated
    on the host with their own float coefficient table, agree with the FP64 oracle to
    float precision (a wrong coefficient shows up as a relative error >> 1e-7)."""
    import numpy as np

    import oracle

    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc) and shutil.which("nvcc") is None:
        pytest.skip("nvcc not available")
    exe = tmp_path / "series_check"
    src = os.path.join(ROOT, "tests", "host", "series_check.cu")
    inc = os.path.join(ROOT, "paper_2511_11430_gb300", "csrc")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-I" + inc, src, "-o",
                    str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    vals = np.array(out, dtype=np.float64).reshape(-1, 3)
    rho = vals[:, 0]
    g, F = oracle.blob_gF(rho)
    np.testing.assert_allclose(vals[:, 1], g / rho ** 3, rtol=3e-7)
    np.testing.assert_allclose(vals[:, 2], F / rho ** 5, rtol=3e-7)
