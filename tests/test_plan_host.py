"""The FFT planning code shared by every launcher (csrc/plan.h), on the CPU:
a host-only driver (tests/plan_check.cpp, compiled here with g++) prints the
plans, and each is checked against definitions written out independently:
the radices multiply to L and fit the kernels' element count, the Stockham
stage table follows from the radices, every twiddle is exp(-2 pi i r k /
(R ns)), a Stockham transform run in numpy from the plan's own stage table
and twiddle table is the DFT (forward plan) and L times the inverse DFT
(reversed plan, conjugate twiddles), and the tile choice obeys its rules.
A plan that failed any of these would make the pass kernels compute a
different transform than the filter (Section 4, Eq. df2) needs."""

import json
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = "/usr/local/cuda/include"
LENGTHS = [8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024, 1536, 2048, 3072, 4096]


def pick_e(n):
    return 24 if n % 3 == 0 else 16


@pytest.fixture(scope="module")
def plans(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("plan") / "plan_check")
    subprocess.run([gxx, "-std=c++17", "-O1", "-I" + os.path.join(ROOT, "include"),
                    "-I" + os.path.join(ROOT, "paper_1707_09177_gb300", "csrc"), "-I" + CUDA_INC,
                    os.path.join(ROOT, "tests", "plan_check.cpp"), "-o", exe], check=True)
    args = ["%d:%d" % (n, pick_e(n)) for n in LENGTHS] + ["10:16", "5:16", "48:16", "9216:24"]
    out = subprocess.run([exe] + args, check=True, capture_output=True, text=True).stdout
    return {(d["L"], d["E"]): d for d in map(json.loads, out.strip().splitlines())}


def _stockham(x, radices, tw, inverse):
    """Stockham autosort transform of the plan: stage (R, ns) reads butterfly j's
    inputs at j + r L/R, multiplies input r by the table's factor (r, k = j mod
    ns), takes an R-point DFT (exp(-+2 pi i r m / R)) and writes output m at
    (j - k) R + k + m ns."""
    L = len(x)
    x = x.astype(np.complex128)
    ns, off = 1, 0
    for R in radices:
        lr = L // R
        y = np.empty_like(x)
        sgn = 1.0 if inverse else -1.0
        dft = np.exp(sgn * 2j * np.pi * np.outer(np.arange(R), np.arange(R)) / R)
        for j in range(lr):
            k = j % ns
            v = x[j + lr * np.arange(R)].copy()
            for r in range(1, R):
                e = off + (r - 1) * ns + k
                w = tw[e]
                v[r] *= np.conj(w) if inverse else w
            y[(j - k) * R + k + ns * np.arange(R)] = dft @ v
        x = y
        off += (R - 1) * ns
        ns *= R
    return x


def _table(d, key):
    t = np.array(d[key])
    return t[0::2] + 1j * t[1::2]


@pytest.mark.parametrize("n", LENGTHS)
def test_radices_and_stage_table(plans, n):
    d = plans[(n, pick_e(n))]
    rad, E = d["radices"], d["E"]
    assert d["plan_ok"] and 1 <= len(rad) <= 5
    assert int(np.prod(rad)) == n
    assert all(E % r == 0 for r in rad)
    k3 = sum(1 for r in rad if r == 3)
    assert rad[:k3] == [3] * k3 and all(r != 3 for r in rad[k3:])          # the factors 3 first
    p2 = rad[k3:]
    assert p2 == sorted(p2, reverse=True) and max(p2, default=1) <= (16 if E % 16 == 0 else 8)
    ns, off = 1, 0
    for (R, s_ns, s_off), r in zip(d["stages"], rad):
        assert (R, s_ns, s_off) == (r, ns, off)
        off += (r - 1) * ns
        ns *= r
    assert off == n - 1 and d["reversed"] == rad[::-1]


@pytest.mark.parametrize("n", LENGTHS)
def test_twiddles_are_the_stage_roots_of_unity(plans, n):
    d = plans[(n, pick_e(n))]
    for key, rad in (("twiddles", d["radices"]), ("reversed_twiddles", d["reversed"])):
        tw = _table(d, key)
        ns, off = 1, 0
        for R in rad:
            for r in range(1, R):
                k = np.arange(ns)
                want = np.exp(-2j * np.pi * r * k / (R * ns))
                # the table is computed in long double; this float64 reference carries up to
                # |angle| 2^-53 (~7e-16) of its own argument rounding
                np.testing.assert_allclose(tw[off + (r - 1) * ns + k], want, rtol=0, atol=2e-15)
            off += (R - 1) * ns
            ns *= R


@pytest.mark.parametrize("n", LENGTHS)
def test_plan_transforms_are_the_dft(plans, n):
    d = plans[(n, pick_e(n))]
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    fwd = _stockham(x, d["radices"], _table(d, "twiddles"), inverse=False)
    assert np.linalg.norm(fwd - np.fft.fft(x)) <= 1e-13 * np.linalg.norm(fwd)
    inv = _stockham(x, d["reversed"], _table(d, "reversed_twiddles"), inverse=True)
    assert np.linalg.norm(inv - n * np.fft.ifft(x)) <= 1e-13 * np.linalg.norm(inv)


def test_lengths_without_a_plan(plans):
    assert plans[(10, 16)]["radices"] == []        # a factor 5
    assert plans[(5, 16)]["radices"] == []
    assert plans[(48, 16)]["radices"] == []        # a factor 3 needs E divisible by 3
    assert plans[(9216, 24)]["radices"] == []      # 9 x 2^10 would take 6 stages at E = 24


def _phys(i):
    return i + (i >> 4)


@pytest.mark.parametrize("n", LENGTHS + [10])
def test_tile_choice(plans, n):
    E = 16 if n == 10 else pick_e(n)
    d = plans[(n, E)]
    slots = n + 1
    ld = _phys(slots - 1) + 1
    ld += (ld + 1) % 2                                # odd row stride
    for div, ok, W, T, got_ld, smem in d["tiles"]:
        cands = []
        Wc = 1
        while Wc <= 4096 and (div == 0 or div % Wc == 0):
            if (Wc * n) % E == 0 and 1 <= Wc * n // E <= 256 and Wc * ld * 8 <= 100 * 1024:
                cands.append((abs(np.log2(Wc * n / E / 256.0)), Wc))
            Wc *= 2
        if not cands:
            assert ok == 0
            continue
        best = min(cands)[1]                           # closest to 256 threads, the narrower tile on a tie
        assert ok == 1 and W == best and T == W * n // E and got_ld == ld and smem == W * ld * 8
