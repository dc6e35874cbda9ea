"""The stochastic rounding of the 16-bit storages on the device (the
conversion the step kernels store every pair with, through
lbm_debug_sr_pairs).

For each test value and every one of the 65536 values of the half-word of
random bits that decides it:
  * the code is one of the two 16-bit neighbours of x in magnitude (x itself
    when x is representable);
  * the neighbour away from zero comes up frac * 2^16 times (to one count),
    frac = (|x| - |lower|) / spacing, so the mean code equals x: BF16 and
    normal FP16 values, whose dropped bits (16, 13) the random bits resolve
    fully;
  * FP16 subnormals drop more than 13 bits and the conversion resolves 13 of
    them: the count is frac * 2^16 rounded down to a multiple of 8 (a bias
    toward zero under 2^-13 of a spacing);
  * the other half-word's random bits do not change it.
Values: the FP16 storage's scaled deviations (2^15 x 1e-9 .. 1e-1, FP16
subnormals included), binade ends, both signs, exact values, zero; for BF16
the unscaled deviations.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    from paper_2011_15073_gb300 import lbm as m
    m.lib()
    return m


def _values(fmt):
    rng = np.random.default_rng(2011)
    mag = 10.0 ** rng.uniform(-9.0, -1.0, 40)
    if fmt == "f16":
        mag = mag * 32768.0
        special = [0.0, 1.0, 0.5, 2.0 ** -24, 3 * 2.0 ** -25, 6.0e-5, 6.2e-5, 2.0 ** -14, 1.0 + 2.0 ** -23,
                   2.0 - 2.0 ** -23, 1000.123, 2.0 ** -20 * (1 + 0x1234 * 2.0 ** -23),
                   2.0 ** -15 * (1 + 0x5A5A5 * 2.0 ** -23)]
    else:
        special = [0.0, 1.0, 0.5, 1.0 + 2.0 ** -23, 2.0 - 2.0 ** -23, 1e-30, 0.0123]
    v = np.concatenate([mag, special]).astype(np.float32)
    sign = np.where(np.arange(v.size) % 2 == 1, -1.0, 1.0).astype(np.float32)
    return v * sign


def _decode(codes, fmt):
    if fmt == "f16":
        return codes.view(np.float16).astype(np.float64)
    return (codes.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def _neighbours(x, fmt):
    """(lower, upper) 16-bit neighbours of x in magnitude and frac of the way up."""
    x = np.float32(x)
    if fmt == "f16":
        lo = np.float16(x)
        if abs(float(lo)) > abs(float(x)):
            lo = np.nextafter(lo, np.float16(0))
        hi = np.nextafter(lo, np.float16(np.inf) if x >= 0 else np.float16(-np.inf))
        lo, hi = float(lo), float(hi)
    else:
        u = np.array([x], np.float32).view(np.uint32)[0]
        lo = float(np.array([u & 0xFFFF0000], np.uint32).view(np.float32)[0])
        hi = float(np.array([(u & 0xFFFF0000) + 0x10000], np.uint32).view(np.float32)[0])
    frac = 0.0 if hi == lo else (abs(float(x)) - abs(lo)) / (abs(hi) - abs(lo))
    return lo, hi, frac


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
@pytest.mark.parametrize("half", ["low", "high"])
def test_pair_rounding_is_unbiased_and_brackets(lbm, fmt, half):
    vals = _values(fmt)
    s = np.arange(65536, dtype=np.uint32)
    other = np.random.default_rng(7).integers(0, 65536, 65536, dtype=np.uint32)
    n = vals.size * 65536
    x = np.zeros(2 * n, np.float32)
    r = np.empty(n, np.uint32)
    for j, v in enumerate(vals):
        sl = slice(j * 65536, (j + 1) * 65536)
        if half == "low":
            x[2 * j * 65536:2 * (j + 1) * 65536:2] = v
            x[2 * j * 65536 + 1:2 * (j + 1) * 65536:2] = 0.3   # the other half: fixed value
            r[sl] = (other << 16) | s
        else:
            x[2 * j * 65536 + 1:2 * (j + 1) * 65536:2] = v
            x[2 * j * 65536:2 * (j + 1) * 65536:2] = 0.3
            r[sl] = (s << 16) | other
    codes = lbm.debug_sr_pairs(fmt, x, r)
    mine = _decode(codes[0::2] if half == "low" else codes[1::2], fmt).reshape(vals.size, 65536)
    for j, v in enumerate(vals):
        lo, hi, frac = _neighbours(v, fmt)
        got = mine[j]
        if lo == float(v):
            assert np.all(got == lo), (fmt, half, float(v))
            continue
        assert np.all((got == lo) | (got == hi)), (fmt, half, float(v), np.unique(got)[:4], lo, hi)
        ups = int(np.count_nonzero(got == hi))
        if fmt == "f16" and abs(float(v)) < 2.0 ** -14:   # FP16 subnormal: 13 of the dropped bits resolved
            assert ups % 8 == 0 and frac * 65536.0 - 8.0 < ups <= frac * 65536.0 + 1e-6, (float(v), ups, frac)
            continue
        assert abs(ups - frac * 65536.0) <= 1.0, (fmt, half, float(v), ups, frac * 65536.0)
        assert abs(got.mean() - float(v)) <= abs(hi - lo) * 2.0 ** -16 * 1.0001


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
def test_each_half_is_decided_by_its_own_random_bits(lbm, fmt):
    """Sweeping one half-word of r leaves the other half's rounding unchanged."""
    v = np.float32(1.0 + 0x0A5A * 2.0 ** -23 if fmt == "f16" else 1.0 + 0x5A5A * 2.0 ** -23)
    s = np.arange(65536, dtype=np.uint32)
    x = np.full(2 * 65536, v, np.float32)
    for shift, fixed_half in ((0, 1), (16, 0)):   # sweep low bits -> high value fixed, and vice versa
        codes = lbm.debug_sr_pairs(fmt, x, (s << shift) | (np.uint32(0x1234) << (16 - shift)))
        assert np.unique(codes[fixed_half::2]).size == 1
        assert np.unique(codes[1 - fixed_half::2]).size == 2
