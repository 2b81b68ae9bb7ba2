"""The phase reduction of the FP64-accurate double-float form (RAD_FP64_DF), run on the GPU and
checked against exact rational arithmetic.

The kernel forms the oracle's FP64 phase phi = w* A_k(n) (Sec. II) and reduces it as
phi = j pi/1024 + r with |r| <= pi/2048: by a fixed-point (Payne-Hanek) reduction with integer
multiplies for 2^-10 <= |phi| < 2^22, by an FP64 Cody-Waite reduction above and with r = phi
below. It returns j (modulo 2^16 on the integer path; the table takes it modulo 2048) and r as a
float pair (xh, xl). Here phi is an exact binary number, pi/1024 is taken from pi to 60 decimal
digits, and for every phase, with t = phi 1024/pi:
  j = J (mod 2048) for a neighbour J of t with |t - J| <= 1/2 + 1e-4 (the Cody-Waite path rounds
  an FP64 quotient, whose relative error of about 1e-16 reaches 4e-5 of a step at |phi| = 2^30,
  so within that distance of a tie it may take the farther neighbour; r is then exact for it);
  |xh + xl - (phi - J pi/1024)| <= 3e-16 rad, the bound the kernel's error budget states;
  |xh + xl| <= (1/2 + 1e-4) pi/1024.
"""
import ctypes
import os
import subprocess
import tempfile
from fractions import Fraction

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
PI = Fraction("3.141592653589793238462643383279502884197169399375105820974944")
STEP = PI / 1024


@pytest.fixture(scope="module")
def probe():
    out = os.path.join(tempfile.mkdtemp(), "df_reduce_probe.so")
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-shared",
                           "-Xcompiler", "-fPIC", os.path.join(HERE, "df_reduce_probe.cu"), "-o", out])
    lib = ctypes.CDLL(out)
    P = ctypes.c_void_p
    lib.reduce_probe.argtypes = [P, ctypes.c_int, P, P, P]
    lib.reduce_probe.restype = ctypes.c_int
    return lib


def run(lib, phi):
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    n = phi.size
    j = np.zeros(n, np.int32)
    xh = np.zeros(n, np.float32)
    xl = np.zeros(n, np.float32)
    rc = lib.reduce_probe(phi.ctypes.data, n, j.ctypes.data, xh.ctypes.data, xl.ctypes.data)
    assert rc == 0, f"CUDA error {rc}"
    return j, xh, xl


def phases(seed):
    rng = np.random.default_rng(seed)
    out = []
    # every binade from 2^-14 to 2^30: both sides of the integer path's range [2^-10, 2^22)
    for e in range(-14, 31):
        out.append(rng.uniform(1.0, 2.0, 300) * 2.0 ** e)
    # exact binade edges and the path boundaries
    out.append(np.array([2.0 ** -10, np.nextafter(2.0 ** -10, 0), 2.0 ** 22, np.nextafter(2.0 ** 22, 0),
                         np.pi / 2048, np.pi / 1024, np.pi, 2 * np.pi, 1.0, 0.0]))
    # near multiples of pi/1024 and near the half-way points between them
    k = rng.integers(1, 1 << 31, 3000).astype(np.float64)
    near = k * (np.pi / 1024)
    out.append(near * (1 + rng.normal(0, 1e-15, k.size)))
    out.append((k + 0.5) * (np.pi / 1024) * (1 + rng.normal(0, 1e-15, k.size)))
    p = np.concatenate(out)
    p = p[(p < 2.0 ** 30)]
    sign = np.where(rng.random(p.size) < 0.5, -1.0, 1.0)
    return p * sign


@pytest.mark.parametrize("seed", [1, 2])
def test_reduction_exact_within_3e_16(probe, seed):
    phi = phases(seed)
    j, xh, xl = run(probe, phi)
    worst = Fraction(0)
    slack = Fraction(1, 2) + Fraction(1, 10 ** 4)
    for i in range(phi.size):
        f = Fraction(float(phi[i]))
        t = f / STEP
        lo = t.numerator // t.denominator  # floor(t)
        cands = [J for J in (lo, lo + 1) if (int(j[i]) - J) % 2048 == 0]
        assert len(cands) == 1, (phi[i], int(j[i]), lo)
        J = cands[0]
        assert abs(t - J) <= slack, (phi[i], float(t - J))
        r = Fraction(float(xh[i])) + Fraction(float(xl[i]))
        err = abs(r - (f - J * STEP))
        assert err <= Fraction(3, 10 ** 16), (phi[i], float(err))
        assert abs(r) <= slack * STEP, (phi[i], float(r))
        worst = max(worst, err)
    print("max |r - exact| =", float(worst))


def test_reduction_is_odd(probe):
    """phi and -phi give j and -j (mod 2048) and opposite remainders, bit for bit."""
    phi = np.abs(phases(3))
    j1, h1, l1 = run(probe, phi)
    j2, h2, l2 = run(probe, -phi)
    assert np.all((j1 + j2) % 2048 == 0)
    assert np.array_equal(h1, -h2) and np.array_equal(l1, -l2)
