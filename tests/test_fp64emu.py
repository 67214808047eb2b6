"""The integer-pipe binary64 addition of the z move (csrc/rlt2_fp64emu.cuh),
compiled for the host, against the host's IEEE 754 addition (numpy, round to
nearest, ties to even) bit for bit: random operands over the whole exponent
range, subnormals, cancellations, exact ties, signed zeros, large exponent gaps
and overflow to infinity."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_1710_03732_gb300", "csrc")
SHIM = r"""
#include <cstdint>
#include "rlt2_fp64emu.cuh"
extern "C" void emu_add_many(long long n, const uint64_t* a, const uint64_t* b, int sub, uint64_t* out) {
  for (long long i = 0; i < n; ++i) out[i] = rlt2::emu_add_bits(a[i], sub ? (b[i] ^ 0x8000000000000000ull) : b[i]);
}
"""


@pytest.fixture(scope="module")
def emu(tmp_path_factory):
    d = tmp_path_factory.mktemp("emu")
    src, lib = d / "shim.cpp", d / "libemu.so"
    src.write_text(SHIM)
    r = subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-I" + HDR, str(src), "-o", str(lib)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    L = ctypes.CDLL(str(lib))
    u64p = ctypes.POINTER(ctypes.c_uint64)
    L.emu_add_many.argtypes = [ctypes.c_longlong, u64p, u64p, ctypes.c_int, u64p]

    def run(a, b, sub=False):
        a = np.ascontiguousarray(a, dtype=np.float64).view(np.uint64)
        b = np.ascontiguousarray(b, dtype=np.float64).view(np.uint64)
        out = np.empty_like(a)
        L.emu_add_many(a.size, a.ctypes.data_as(u64p), b.ctypes.data_as(u64p), int(sub), out.ctypes.data_as(u64p))
        return out
    return run


def _check(emu, a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    with np.errstate(over="ignore", invalid="ignore"):
        ref_add, ref_sub = (a + b).view(np.uint64), (a - b).view(np.uint64)
    got_add, got_sub = emu(a, b), emu(a, b, sub=True)
    bad = np.nonzero((got_add != ref_add) | (got_sub != ref_sub))[0]
    assert bad.size == 0, [(a[i], b[i], got_add[i], ref_add[i], got_sub[i], ref_sub[i]) for i in bad[:5]]


def _random_bits(rng, n):
    """Doubles with uniformly random sign, exponent field 0..2046 and fraction."""
    sign = rng.integers(0, 2, n, dtype=np.uint64) << np.uint64(63)
    ex = rng.integers(0, 2047, n, dtype=np.uint64) << np.uint64(52)
    fr = rng.integers(0, 1 << 52, n, dtype=np.uint64)
    return (sign | ex | fr).view(np.float64)


def test_random_over_the_exponent_range(emu):
    rng = np.random.default_rng(1)
    _check(emu, _random_bits(rng, 200000), _random_bits(rng, 200000))


def test_close_exponents_and_cancellation(emu):
    """Operands within a few binades (every alignment shift 0..60) and nearly
    equal magnitudes of opposite sign (massive cancellation)."""
    rng = np.random.default_rng(2)
    n = 200000
    a = rng.normal(size=n) * 10.0 ** rng.integers(-5, 6, n)
    b = a * (1 + rng.normal(size=n) * 10.0 ** rng.integers(-16, 0, n)) * rng.choice([-1.0, 1.0], n)
    _check(emu, a, b)
    shift = rng.integers(0, 64, n).astype(np.float64)
    _check(emu, a, a * np.exp2(-shift) * rng.choice([-1.0, 1.0], n))
    # neighbours: a and -nextafter(a)
    _check(emu, a, -np.nextafter(a, np.inf))


def test_exact_ties_round_to_even(emu):
    """1 + k*2^-53 for odd and even significands: exactly halfway between two
    doubles, rounded to the even one; the same across binades."""
    rng = np.random.default_rng(3)
    base = 1.0 + rng.integers(0, 1 << 20, 5000) * 2.0 ** -52
    scale = 2.0 ** rng.integers(-1000, 1000, 5000).astype(np.float64)
    half = 2.0 ** -53
    _check(emu, base * scale, half * scale)
    _check(emu, base * scale, -half * scale)
    _check(emu, base * scale, 3 * half * scale)
    _check(emu, base * scale, half * scale * (1 + 2.0 ** -30))  # just above half


def test_subnormals_zeros_and_overflow(emu):
    rng = np.random.default_rng(4)
    n = 100000
    tiny = rng.integers(0, 1 << 53, n).astype(np.float64) * 5e-324 * rng.choice([-1.0, 1.0], n)
    _check(emu, tiny, _random_bits(rng, n) * 1e-300)
    _check(emu, tiny, np.roll(tiny, 1))
    mn = np.finfo(float).tiny
    _check(emu, np.full(4, mn), np.array([-5e-324, -mn, mn, -mn / 2]))
    z = np.array([0.0, -0.0, 0.0, -0.0, 1.0, -1.0, 5e-324])
    _check(emu, np.repeat(z, z.size), np.tile(z, z.size))
    big = np.finfo(float).max
    _check(emu, np.array([big, big, -big, big / 2, 1e308]), np.array([big, -big, -big, big, 9e307]))


@pytest.mark.gpu
def test_device_emulation_equals_the_fp64_pipe(emu):
    """The same inputs through the device build (rlt2_fp64_add_emulated, C ABI)
    against the FP64 pipe (torch float64 add and sub on the GPU) and against
    the host build, bit for bit."""
    torch = pytest.importorskip("torch")
    from paper_1710_03732_gb300 import build, rlt2
    build.build()
    rng = np.random.default_rng(9)
    n = 300000
    a = np.concatenate([_random_bits(rng, n), rng.normal(size=n) * 1e3,
                        rng.integers(0, 1 << 53, n).astype(np.float64) * 5e-324])
    b = np.concatenate([_random_bits(rng, n), -a[n:2 * n] * (1 + rng.normal(size=n) * 1e-12),
                        rng.integers(0, 1 << 53, n).astype(np.float64) * -5e-324])
    base = 1.0 + rng.integers(0, 1 << 20, n) * 2.0 ** -52
    a = np.concatenate([a, base, [0.0, -0.0, 0.0, 5e-324]])
    b = np.concatenate([b, np.full(n, 2.0 ** -53), [-0.0, -0.0, 0.0, -5e-324]])
    ta, tb = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    s, d = torch.empty_like(ta), torch.empty_like(ta)
    rlt2.rlt2_fp64_add_emulated(ta, tb, s, d)
    pipe_s, pipe_d = (ta + tb).cpu().numpy().view(np.uint64), (ta - tb).cpu().numpy().view(np.uint64)
    got_s, got_d = s.cpu().numpy().view(np.uint64), d.cpu().numpy().view(np.uint64)
    finite = np.isfinite(a + b) & np.isfinite(a - b)
    assert np.array_equal(got_s[finite], pipe_s[finite]) and np.array_equal(got_d[finite], pipe_d[finite])
    assert np.array_equal(got_s, emu(a, b)) and np.array_equal(got_d, emu(a, b, sub=True))
