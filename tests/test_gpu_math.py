"""The step's own FP64 log and J^{-1/3} (Taylor and atanh series near 1, chosen by the exponent
of J - 1, with the tier boundaries sampled on both sides / single-precision seed with a
third-order correction) against CUDA's log and rcbrt on the device (-m gpu)."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2104_02139_gb300", "csrc")


def test_log_and_rcbrt_against_cuda():
    so = os.path.join(tempfile.mkdtemp(), "mathcheck.so")
    subprocess.check_call(["nvcc", "-shared", "-Xcompiler", "-fPIC", "-O3", "-std=c++17",
                           "-gencode", "arch=compute_103a,code=sm_103a", "-I", CSRC,
                           os.path.join(HERE, "gpu_math_check.cu"), "-o", so])
    lib = ctypes.CDLL(so)
    rng = np.random.default_rng(0)
    J = np.concatenate([np.linspace(0.3, 3.0, 100001), 1 + np.linspace(-0.13, 0.13, 100001),
                        1 + rng.normal(0, 1e-4, 50000), 1 + rng.normal(0, 1e-9, 20000),
                        1 + rng.normal(0, 1e-14, 20000), [1.0, 0.875, 1.125, np.nextafter(1.125, 2)],
                        [1 + sgn * 2.0 ** -k * f for k in (12, 6, 3) for sgn in (1, -1)
                         for f in (1.0, 1 - 2.0 ** -52, 1 + 2.0 ** -52)]])
    out = np.zeros(4 * J.size)
    assert lib.eval_math(J.ctypes.data_as(ctypes.c_void_p), J.size, out.ctypes.data_as(ctypes.c_void_p)) == 0
    lg, lg_ref, rc, rc_ref = out.reshape(4, -1)
    # log: within 2 ulp of |log J| (absolute 2 ulp of 1/8 ~ 6e-17 near the switch-over)
    assert np.all(np.abs(lg - lg_ref) <= 4.5e-16 * np.abs(lg_ref) + 1e-17)
    assert lg[np.where(J == 1.0)[0][0]] == 0.0
    # J^{-1/3}: within 2 ulp
    assert np.all(np.abs(rc - rc_ref) <= 4.5e-16 * rc_ref)


def test_order_keys_compare_like_doubles():
    """The integer keys the detection and the density ranges compare: a >= b, min and max agree
    with the FP64 ones for every finite and infinite value, zeros of both signs aside (which
    the keys order -0 < +0)."""
    so = os.path.join(tempfile.mkdtemp(), "keycheck.so")
    subprocess.check_call(["nvcc", "-shared", "-Xcompiler", "-fPIC", "-O3", "-std=c++17",
                           "-gencode", "arch=compute_103a,code=sm_103a", "-I", CSRC,
                           os.path.join(HERE, "gpu_math_check.cu"), "-o", so])
    lib = ctypes.CDLL(so)
    rng = np.random.default_rng(1)
    special = np.array([0.0, 1.0, -1.0, 2.0, -2.0, 1e-300, -1e-300, 5e-324, -5e-324, 1e300, -1e300,
                        np.inf, -np.inf, np.nextafter(1.0, 2.0), np.nextafter(1.0, 0.0)])
    a = np.concatenate([rng.normal(size=50000) * 10.0 ** rng.integers(-20, 20, 50000), np.repeat(special, special.size),
                        rng.normal(size=1000)])
    b = np.concatenate([rng.normal(size=50000) * 10.0 ** rng.integers(-20, 20, 50000), np.tile(special, special.size),
                        np.zeros(1000) + rng.normal(size=1000)])
    n = a.size
    ge = np.zeros(2 * n, dtype=np.int32)
    mm = np.zeros(2 * n)
    assert lib.eval_keys(a.ctypes.data_as(ctypes.c_void_p), b.ctypes.data_as(ctypes.c_void_p), n,
                         ge.ctypes.data_as(ctypes.c_void_p), mm.ctypes.data_as(ctypes.c_void_p)) == 0
    keep = ~((a == 0) & (b == 0))
    assert np.array_equal(ge[:n][keep], ge[n:][keep])
    assert np.array_equal(mm[:n][keep], np.minimum(a, b)[keep])
    assert np.array_equal(mm[n:][keep], np.maximum(a, b)[keep])
