"""The adjoint kernel's per-substep vector-Jacobian product (mg_device.cuh,
compiled for the host in FP64) against central differences of the forward
substep: the product is the transpose of the forward map, term by term
(Eq. 1-3 with the actuators of Sec. III-D), for the vehicle alone (diagonal
inverse), with a payload (combined body about the origin, full inverse), and
for a class with fins and a servo-tilted propeller; with the semi-implicit
Euler substep and with RK4. No GPU: the device functions are
host/device code; nvcc compiles them for the host."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


def test_vjp_matches_central_differences(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "vjp_fd")
    subprocess.check_call([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-O2",
                           "-I", os.path.join(ROOT, "paper_2503_09203_b300", "csrc"),
                           "-I", os.path.join(ROOT, "include"),
                           os.path.join(HERE, "host", "vjp_fd.cu"), "-o", exe])
    out = subprocess.check_output([exe, "1"], text=True).split()
    vals = dict(zip(out[0::2], map(float, out[1::2])))
    # FP64 central differences at h = 1e-6: truncation ~1e-12, rounding ~1e-10.
    assert vals["worst"] <= 1e-8, vals
    assert vals["worst_payload"] <= 1e-8, vals
    assert vals["worst_generic"] <= 1e-8, vals
    assert vals["worst_rk4"] <= 1e-8, vals
    # A 1% error in one gradient term is seen.
    assert vals["scaled"] >= 1e-5, vals
    assert vals["scaled_payload"] >= 1e-5, vals
    assert vals["scaled_generic"] >= 1e-5, vals
    assert vals["scaled_rk4"] >= 1e-5, vals
