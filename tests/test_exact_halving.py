"""Two FP32 kernels fold a factor 1/2 into their operands and rely on the halving being
exact, so that the values are the same as before the fold:

- the torus transfer computes (1 - e^-x) / 2 as fma(e, -1/2, 1/2) and, for small x, as
  x (1/2 - x (1/4 - x / 12)) in place of x (1 - x (1/2 - x / 6)) / 2;
- the surrogate's inference kernel packs the weights and biases of layers 1-4 halved (BF16
  and FP32) so that its accumulators hold z / 2.

Halving a binary floating-point number is exact away from the subnormal range, and so is a
rounded operation on halved operands (round(x / 2) = round(x) / 2).  Here the constants and
the operation chains are replayed in float32 on the CPU (an FMA emulated in float64, where
the product of two float32 values is exact) over sampled inputs."""
import numpy as np


def _fma32(a, b, c):
    # float32 fma: a * b is exact in float64; a single rounding of a*b + c to float32
    # matches the hardware FMA whenever the float64 sum is exact, which holds for the
    # magnitudes sampled here (all operands within a few binades of each other)
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def test_series_constants_halve_exactly():
    assert np.float32(1.0 / 12.0) == np.float32(1.0 / 6.0) / np.float32(2.0)
    assert np.float32(0.25) == np.float32(0.5) / np.float32(2.0)


def test_halved_series_is_half_the_series():
    rng = np.random.default_rng(7)
    x = rng.uniform(0.0, 1.0 / 32.0, 200_000).astype(np.float32)
    f32 = np.float32
    full = x * _fma32(x, _fma32(x, np.full_like(x, f32(1 / 6)), np.full_like(x, f32(-0.5))),
                      np.full_like(x, f32(1.0)))
    half = x * _fma32(x, _fma32(x, np.full_like(x, f32(1 / 12)), np.full_like(x, f32(-0.25))),
                      np.full_like(x, f32(0.5)))
    assert np.array_equal(half, full / f32(2.0))


def test_halved_difference_is_half_the_difference():
    rng = np.random.default_rng(8)
    e = np.exp(-rng.uniform(1.0 / 32.0, 40.0, 200_000)).astype(np.float32)
    full = _fma32(e, np.full_like(e, np.float32(-1.0)), np.full_like(e, np.float32(1.0)))
    half = _fma32(e, np.full_like(e, np.float32(-0.5)), np.full_like(e, np.float32(0.5)))
    assert np.array_equal(half, full / np.float32(2.0))


def test_halved_bf16_weights_are_exact():
    """BF16 is float32 with the low 16 bits dropped: halving keeps the 8-bit mantissa."""
    rng = np.random.default_rng(9)
    w = rng.normal(0.0, 0.1, 200_000).astype(np.float32)
    bf = (w.view(np.uint32) & np.uint32(0xFFFF0000)).view(np.float32)  # a BF16 value
    halved = bf / np.float32(2.0)
    assert np.array_equal(halved.view(np.uint32) & np.uint32(0x0000FFFF),
                          np.zeros_like(halved.view(np.uint32)))  # still a BF16 value
    assert np.array_equal(halved * np.float32(2.0), bf)
