"""Host checks (numpy, IEEE arithmetic) of the floating-point facts the mixed
path's kernels rely on. Each test restates a fact the device code assumes and
checks it on inputs of the kind the kernels see, edge cases included."""
import numpy as np


def _f32_pairs(rng, n):
    """FP32 pairs (hi, lo) as the double-float arithmetic leaves them: lo
    within about half an ulp of hi, plus pairs far apart and ties."""
    hi = (rng.standard_normal(n) * 10.0 ** rng.integers(-20, 20, n)).astype(np.float32)
    ulp = np.spacing(np.abs(hi)).astype(np.float64)
    lo = (rng.uniform(-0.5, 0.5, n) * ulp).astype(np.float32)
    far = (rng.standard_normal(n // 4) * ulp[: n // 4] * 2.0 ** -rng.integers(0, 40, n // 4)).astype(np.float32)
    lo[: n // 4] = far
    # exact midpoints between FP32 neighbours of hi, and one bit past them
    k = n // 8
    lo[n // 4: n // 4 + k] = (0.5 * ulp[n // 4: n // 4 + k]).astype(np.float32)
    lo[n // 4 + k: n // 4 + 2 * k] = np.nextafter((0.5 * ulp[n // 4 + k: n // 4 + 2 * k]).astype(np.float32),
                                                  np.float32(np.inf))
    return hi, lo


def test_pair_sum_rounded_once_in_fp32_equals_fp32_of_the_fp64_sum():
    """The assembly writes an FP32 plane as hi + lo rounded in FP32 and the FP64
    plane as hi + lo rounded in FP64: the FP32 plane must equal the FP64
    plane's FP32 rounding bit for bit (double rounding through 53 bits is
    innocuous for a sum of two 24-bit numbers: 53 >= 2 * 24 + 1)."""
    rng = np.random.default_rng(20230318)
    hi, lo = _f32_pairs(rng, 200_000)
    direct = (hi + lo).astype(np.float32)                      # one FP32 rounding
    via64 = (hi.astype(np.float64) + lo.astype(np.float64)).astype(np.float32)
    assert np.array_equal(direct.view(np.uint32), via64.view(np.uint32))


def test_power_of_two_scaling_commutes_with_fp32_rounding():
    """The staged residual is rounded to FP32 after scaling by 2^e on the
    exponent field: for FP64 values whose scaled value is a normal FP32
    number, rounding d * 2^e equals rounding d and scaling the result."""
    rng = np.random.default_rng(7)
    d = rng.standard_normal(100_000) * 10.0 ** rng.integers(-30, 30, 100_000)
    for e in (-60, -17, 0, 9, 45):
        scaled = d * 2.0 ** e                                   # exact in FP64 here
        ok = (np.abs(scaled) >= np.finfo(np.float32).tiny) & (np.abs(scaled) < np.finfo(np.float32).max / 2)
        a = scaled[ok].astype(np.float32)
        b = (d[ok] * 2.0 ** e).astype(np.float32)
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
        # and the FP32 rounding of d, scaled in FP32 where that stays normal, agrees too
        ok2 = ok & (np.abs(d) >= np.finfo(np.float32).tiny) & (np.abs(d) < np.finfo(np.float32).max / 2)
        c = (d[ok2].astype(np.float32) * np.float32(2.0 ** e)).astype(np.float32)
        assert np.array_equal(c.view(np.uint32), scaled[ok2].astype(np.float32).view(np.uint32))


def _chunked_fp32_norm2(v, chunk=16):
    """Sum of squares as the FP32 transform path forms it: FP32 partial sums
    of at most `chunk` fused squares, each partial added to an FP64 total."""
    total = 0.0
    part = np.float32(0.0)
    k = 0
    for x in v.astype(np.float32):
        # fmaf(x, x, part): x * x is exact in FP64; the sum rounded to FP64
        # and then to FP32 is within an FP32 ulp of the fused result
        part = np.float32(np.float64(x) * np.float64(x) + np.float64(part))
        k += 1
        if k == chunk:
            total += float(part)
            part = np.float32(0.0)
            k = 0
    return total + float(part)


def test_chunked_fp32_norm_stays_inside_the_convergence_margin():
    """A transform sweep is declared converged when its FP32-summed norm times
    1 + 2^-16 meets the tolerance; the FP32 norm must be within that margin
    of the FP64 norm of the same staged values (values of a staged residual:
    at most a few units, down to tiny)."""
    rng = np.random.default_rng(11)
    margin = 1.0 + 2.0 ** -16
    for trial in range(40):
        n = int(rng.integers(1, 600))
        scale = 10.0 ** rng.uniform(-8, 0)
        v = (rng.standard_normal(n) * scale * 10.0 ** rng.uniform(-3, 0, n)).astype(np.float32)
        exact = np.sqrt(np.sum(v.astype(np.float64) ** 2))
        got = np.sqrt(_chunked_fp32_norm2(v))
        assert got * margin >= exact, (trial, got, exact)
        assert got <= exact * margin, (trial, got, exact)
