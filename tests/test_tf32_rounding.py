"""The integer form of TF32 rounding used by the split-precision kernels, (u + 0x1000) &
0xFFFFE000 on the FP32 bit pattern u, against the definition of the rounding it replaces
(cvt.rna.tf32.f32: round to the nearest value with 10 explicit fraction bits, ties away from
zero), computed here from that definition in exact float64 arithmetic.  Also the exactness of
the three-slice cut f = s1 + s2 + s3 that the subspace kernels rely on (11 + 11 + 2 bits)."""
import numpy as np


def tf32_bits(u):
    """The kernels' integer form, on uint32 bit patterns."""
    return ((u.astype(np.uint64) + 0x1000) & 0xFFFFE000).astype(np.uint32)


def tf32_definition(f):
    """Round each finite float32 value to 10 fraction bits, nearest, ties away from zero
    (float64 holds every intermediate exactly)."""
    x = np.abs(f.astype(np.float64))
    out = np.zeros_like(x)
    nz = x > 0
    # spacing of 10-fraction-bit values around x: 2^(e - 10) for normals (e = exponent of x),
    # 2^(-126 - 10) throughout the float32 subnormal range, as in TF32's own subnormals
    e = np.floor(np.log2(x[nz]))
    e = np.maximum(e, -126.0)
    # guard the floor of log2 at exact powers of two and just below them
    two_e = np.exp2(e)
    e = np.where(x[nz] < two_e, e - 1, e)
    e = np.where(x[nz] >= 2 * np.exp2(e), e + 1, e)
    e = np.maximum(e, -126.0)
    ulp = np.exp2(e - 10.0)
    n = x[nz] / ulp                      # exact: x has at most 24 significant bits
    out[nz] = np.floor(n + 0.5) * ulp    # ties (n + 0.5 integral) go up: away from zero
    return np.where(np.signbit(f), -out, out)


def _check(u):
    f = u.view(np.float32)
    fin = np.isfinite(f)
    u, f = u[fin], f[fin]
    got = tf32_bits(u).view(np.float32).astype(np.float64)
    want = tf32_definition(f)
    # values that round past the largest finite float become infinity in both
    big = np.abs(want) > np.finfo(np.float32).max
    assert np.all(np.isinf(got[big]))
    ok = ~big
    assert np.array_equal(got[ok], want[ok]), np.nonzero(got[ok] != want[ok])[0][:5]


def test_integer_tf32_rounding_equals_the_definition_exhaustively_on_binades():
    # every pattern (both signs) of the binades [1, 2), [2^-20, 2^-19), [2^100, 2^101), the
    # top binade below infinity and the float32 subnormals' top range
    for biased in (127, 107, 227, 254, 0, 1):
        m = np.arange(1 << 23, dtype=np.uint32)
        for sign in (0, 1):
            _check((np.uint32(sign << 31) | (np.uint32(biased) << np.uint32(23)) | m).astype(np.uint32))


def test_integer_tf32_rounding_equals_the_definition_on_random_patterns():
    rng = np.random.default_rng(20261204)
    _check(rng.integers(0, 1 << 32, size=1 << 22, dtype=np.uint64).astype(np.uint32))


def test_three_slices_are_exact():
    """f = s1 + s2 + s3 exactly for FP32 values (the subspace kernels' operand cut), with each
    slice a TF32 value and every subtraction exact in FP32."""
    rng = np.random.default_rng(7)
    f = (rng.standard_normal(1 << 20) * np.exp2(rng.integers(-60, 60, 1 << 20))).astype(np.float32)
    s1 = tf32_bits(f.view(np.uint32)).view(np.float32)
    r1 = (f - s1).astype(np.float32)
    s2 = tf32_bits(r1.view(np.uint32)).view(np.float32)
    r2 = (r1 - s2).astype(np.float32)
    s3 = tf32_bits(r2.view(np.uint32)).view(np.float32)
    for s in (s1, s2, s3):
        assert np.all((s.view(np.uint32) & 0x1FFF) == 0)          # 10 fraction bits
    total = s1.astype(np.float64) + s2.astype(np.float64) + s3.astype(np.float64)
    assert np.array_equal(total, f.astype(np.float64))
