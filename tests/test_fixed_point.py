"""The solver's integer-pipe reductions against exact rational sums (CPU only).

Dot products inside the persistent CG kernel are summed as fixed-point
integers aligned to a common exponent (per warp, per block and across
blocks) and converted back to the nearest double: 128-bit and exact for the
plain reductions, 64-bit with a bounded truncation for the tagged ones of
the iterations.  These tests build the same arithmetic on the host and
compare it with the exact sum of the same doubles, computed with Python
fractions.
"""
import math
import os
import shutil
import struct
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    out = tmp_path_factory.mktemp("fx") / "fx_harness"
    subprocess.check_call([cxx, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2003_00082_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "fixed_point_harness.cpp"), "-o", str(out)])
    return str(out)


def bits(v):
    return struct.unpack("<Q", struct.pack("<d", float(v)))[0]


def run(harness, groups, red=None, warps_per_block=None):
    text = "" if red is None else f"R {red}\n"
    if warps_per_block is not None:
        text += f"W {warps_per_block}\n"
    text += "".join(f"G {len(g)}\n" + " ".join(f"{bits(v):x}" for v in g) + "\n" for g in groups)
    r = subprocess.run([harness], input=text, capture_output=True, text=True, check=True)
    return struct.unpack("<d", struct.pack("<Q", int(r.stdout.strip(), 16)))[0]


def exact(groups):
    return float(sum((Fraction(float(v)) for g in groups for v in g), Fraction(0)))


def ulp_diff(a, b):
    if a == b:
        return 0
    return abs(a - b) / math.ulp(max(abs(a), abs(b)))


@pytest.mark.parametrize("seed", range(12))
def test_fixed_point_sum_is_the_correctly_rounded_sum(harness, seed):
    rng = np.random.default_rng(seed)
    ngroups = int(rng.integers(1, 40))
    groups = []
    for _ in range(ngroups):
        n = int(rng.integers(1, 64))
        scale = 10.0 ** rng.uniform(-8, 8, size=n)
        groups.append(list(rng.standard_normal(n) * scale))
    got = run(harness, groups)
    want = exact(groups)
    assert ulp_diff(got, want) <= 1, (got, want)


def test_cancellation_and_signs(harness):
    groups = [[1e16, 1.0, -1e16], [3.0, -3.0], [2.0 ** -40]]
    assert run(harness, groups) == exact(groups)
    groups = [[0.1] * 10, [-0.1] * 10]
    assert run(harness, groups) == 0.0
    assert run(harness, [[0.0, -0.0]]) == 0.0


def test_ties_round_to_even(harness):
    # 2^53 + 1 is a tie between 2^53 and 2^53 + 2: rounds to the even 2^53
    groups = [[2.0 ** 53, 1.0]]
    assert run(harness, groups) == 2.0 ** 53
    groups = [[2.0 ** 53, 3.0]]
    assert run(harness, groups) == 2.0 ** 53 + 4.0


def test_subnormal_and_tiny_values(harness):
    tiny = 5e-324
    assert run(harness, [[tiny, tiny]]) == 2 * tiny
    groups = [[1e-310, 2e-310], [-5e-311]]
    assert run(harness, groups) == exact(groups)


def test_non_finite_input_gives_nan(harness):
    assert math.isnan(run(harness, [[1.0, float("inf")], [2.0]]))
    assert math.isnan(run(harness, [[float("nan")]]))


def test_large_sums_do_not_overflow(harness):
    groups = [[1.7e308 / 4096] * 64 for _ in range(32)]     # 2048 terms near the top of the range
    got = run(harness, groups)
    want = exact(groups)
    assert ulp_diff(got, want) <= 1


# ---------------------------------------------------------------------------
# the tagged slot encoding: a block's partial travels through an 80-bit
# mantissa with its exponent and the reduction's tags (here a 128-bit partial
# shifted into the field)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(8))
def test_tagged_slots_keep_the_sum_correctly_rounded(harness, seed):
    rng = np.random.default_rng(100 + seed)
    groups = []
    for _ in range(int(rng.integers(1, 300))):       # up to a few hundred blocks
        n = int(rng.integers(1, 64))
        scale = 10.0 ** rng.uniform(-6, 6, size=n)
        groups.append(list(rng.standard_normal(n) * scale))
    red = int(rng.integers(2, 1 << 22))
    got = run(harness, groups, red=red)
    assert ulp_diff(got, exact(groups)) <= 1, (got, exact(groups))


@pytest.mark.parametrize("red", [2, 3, 255, 256, 257, (1 << 23) - 1, 1 << 23, (1 << 23) + 5])
def test_tagged_slots_reject_stale_torn_and_empty_words(harness, red):
    # the harness exits non-zero if a current slot fails its check or a torn / stale / zero one passes;
    # values straddle the 56-bit split of the mantissa and both signs
    groups = [[1.0, -3.5e-7], [-2.0 ** 60, 5.0], [1e-300], [-7.25e12, 1.0 / 3.0]]
    got = run(harness, groups, red=red)
    assert ulp_diff(got, exact(groups)) <= 1


def test_tagged_slots_cancel_and_propagate_non_finite(harness):
    assert run(harness, [[1e16, 1.0, -1e16], [3.0, -3.0]], red=7) == 1.0
    assert run(harness, [[0.0], [-0.0]], red=9) == 0.0
    assert math.isnan(run(harness, [[1.0], [float("inf")]], red=11))


# ---------------------------------------------------------------------------
# the 64-bit tagged reductions of the solver's iterations: warp sums of 64-bit
# images, block sums with 5 bits of headroom, unshifted tagged slots
# ---------------------------------------------------------------------------
def bound64(groups, warps_per_block, got):
    """Truncation bound: under 2^(E - 1079) per term, 2^(E - 1074) per warp and per block, E the largest
    biased exponent of the inputs; then the rounding of the result."""
    vals = [float(v) for g in groups for v in g]
    emax = max((math.frexp(v)[1] + 1022 if v != 0.0 else 1) for v in vals)
    nblocks = (len(groups) + warps_per_block - 1) // warps_per_block
    unit = 2.0 ** (emax - 1074)
    return len(vals) * unit / 32 + (len(groups) + nblocks) * unit + 0.5 * math.ulp(abs(got))


@pytest.mark.parametrize("seed", range(8))
def test_64bit_tagged_sums_stay_within_the_truncation_bound(harness, seed):
    rng = np.random.default_rng(300 + seed)
    wpb = int(rng.choice([1, 4, 12, 16, 32]))
    groups = []
    for _ in range(int(rng.integers(1, 600))):       # up to a few hundred blocks of warps
        n = int(rng.integers(1, 33))
        scale = 10.0 ** rng.uniform(-6, 6, size=n)
        groups.append(list(rng.standard_normal(n) * scale))
    got = run(harness, groups, red=int(rng.integers(2, 1 << 22)), warps_per_block=wpb)
    want = exact(groups)
    assert abs(got - want) <= bound64(groups, wpb, got), (got, want)


def test_64bit_tagged_sums_are_exact_on_one_scale_and_cancel(harness):
    # values on a common grid of the largest exponent carry no truncation
    groups = [[1.0, 2.0, 3.5], [-0.25, 0.125], [4.0]]
    assert run(harness, groups, red=5, warps_per_block=2) == exact(groups)
    # a sum far below its largest term keeps only what the truncation bound allows (the 1.0 here
    # sits 2^-53 below 1e16, under the block level's unit)
    groups = [[1e16, 1.0, -1e16], [3.0, -3.0]]
    got = run(harness, groups, red=7, warps_per_block=16)
    assert abs(got - 1.0) <= bound64(groups, 16, got)
    assert run(harness, [[0.0], [-0.0]], red=9, warps_per_block=1) == 0.0
    assert math.isnan(run(harness, [[1.0], [float("inf")]], red=11, warps_per_block=1))
    # every slot checked against stale, torn and empty words (exit status otherwise)
    for red in (2, 255, 256, (1 << 23) + 5):
        groups = [[1.0, -3.5e-7], [-2.0 ** 60, 5.0], [1e-300], [-7.25e12, 1.0 / 3.0]]
        got = run(harness, groups, red=red, warps_per_block=2)
        assert abs(got - exact(groups)) <= bound64(groups, 2, got)
