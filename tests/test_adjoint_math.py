"""The adjoint's hand-written vector-Jacobian products (stress, impedance, simplex geometry,
velocity gradient, nodal solve with BC projectors, node moments, cell predictor and cell
update, orders 1 and 2, 2D and 3D) against central finite differences of their forward
functions, on random inputs. Runs on the CPU: the functions compile for host and device."""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2104_02139_gb300", "csrc")


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="needs nvcc")
def test_vjps_against_finite_differences():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = os.path.join(tempfile.mkdtemp(), "adjcheck")
    subprocess.check_call([nvcc, "-std=c++17", "-O2", "-x", "cu", "-I", CSRC,
                           os.path.join(HERE, "adjoint_math_check.cu"), "-o", exe])
    out = subprocess.check_output([exe], text=True)
    names = set()
    for line in out.strip().splitlines():
        name, fd, an = line.split()
        fd, an = float(fd), float(an)
        names.add(name)
        assert abs(fd - an) <= 1e-6 * max(abs(fd), 1e-9), (name, fd, an)
    for d in (2, 3):
        for part in ("stress", "stressr1_", "stressr1T_", "stressfam", "stressfamT", "stressfamNH", "sgpsi", "sgstress", "sgstressT", "sgimp",
                     "impedance", "faces", "velgrad", "nodesolve", "nodesolvebc", "moments"):
            assert f"{part}{d}" in names
        for o in (1, 2):
            assert f"predict{d}_ord{o}" in names and f"update{d}_ord{o}" in names
            assert f"updateF1in{d}_ord{o}" in names and f"updatestride{d}_ord{o}" in names
            assert f"predictfam{d}_ord{o}" in names and f"predictsg{d}_ord{o}" in names
        assert f"predictbj{d}" in names and f"predictbjlimited{d}" in names
