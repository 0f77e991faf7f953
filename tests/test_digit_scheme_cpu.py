"""CPU pins of the arithmetic the tcgen05 kernels rest on.

complex128 (exact digit split of Q56 fixed point, level sums in float32,
re-assembly): each formula is checked bit for bit against plain integer
arithmetic on random and extreme inputs, with the kernel's constants written
out.  complex64 (bfloat16 triple split): the residuals are exact and the
three parts, and the six part products kept, carry float32 accuracy.

The kernels (paper_2502_11385_gb300/csrc/kernels.cu, namespaces t05 and t32)
are not imported: these tests fix what their arithmetic must equal."""
import math

import numpy as np

M64 = (1 << 64) - 1
M32 = (1 << 32) - 1
MAGIC = np.float32(12582912.0)  # 1.5 * 2^23
MAGIC_BITS = 0x4B400000
PAIR_OFFSET = 0x8B400000                # 257 * MAGIC_BITS mod 2^32
LEVEL_BIAS = 0x74BF74BF29800000         # removes the three pair offsets and level 6's
DIGIT_BIAS = (1 << 56) + 0x808080808080  # u = v + DIGIT_BIAS
Q56_ONE = 1 << 56


def f32_bits(x):
    return int(np.array(x, dtype=np.float32).view(np.uint32))


def half_value(bits16):
    return float(np.array([bits16], dtype=np.uint16).view(np.float16)[0])


def s64(v):
    v &= M64
    return v - (1 << 64) if v >> 63 else v


def digits_plain(v):
    """Balanced base-256 digits: v = sum_j X_j 256^(6 - j), X_1..6 in [-128, 127]."""
    x = []
    r = v
    for j in range(6, 0, -1):
        d = ((r + 128) % 256) - 128
        x.append(d)
        r = (r - d) // 256
    x.append(r)
    return x[::-1]


def digits_kernel(v):
    """The kernel's split: bytes of u = v + 2^56 + 0x808080808080 under the
    float16 exponent of 1024, minus 1024 + 128 (the top 16 bits minus 1024 +
    256)."""
    u = (v + DIGIT_BIAS) & M64
    top = u >> 48
    assert top <= 512
    x = [half_value(0x6400 | top) - 1280.0]
    for j in range(6):
        b = (u >> (8 * (5 - j))) & 255
        x.append(half_value(0x6400 | b) - 1152.0)
    return [int(d) for d in x]


def test_constants():
    assert (257 * MAGIC_BITS) & M32 == PAIR_OFFSET
    assert LEVEL_BIAS == (-(PAIR_OFFSET * ((1 << 32) + (1 << 16) + 1)) - MAGIC_BITS) & M64
    # the accumulator preload: fp16 3072 (0x6A00) times fp16 4096 (0x6C00)
    assert half_value(0x6A00) * half_value(0x6C00) == float(MAGIC) == 1.5 * 2 ** 23


def test_digit_split_matches_balanced_digits():
    rng = np.random.default_rng(11)
    vals = [0, 1, -1, Q56_ONE, -Q56_ONE, Q56_ONE - 1, -(Q56_ONE - 1), 1 << 55, -(1 << 55), 127, 128, -128, -129]
    vals += [int(v) for v in rng.integers(-Q56_ONE, Q56_ONE + 1, size=20000)]
    vals += [int(v) << int(s) for v, s in zip(rng.integers(-(1 << 20), 1 << 20, size=5000),
                                               rng.integers(0, 36, size=5000))]
    for v in vals:
        v = max(-Q56_ONE, min(Q56_ONE, v))
        x = digits_kernel(v)
        assert x == digits_plain(v), v
        assert sum(d * 256 ** (6 - j) for j, d in enumerate(x)) == v
        assert abs(x[0]) <= 256 and all(-128 <= d <= 127 for d in x[1:])


def reassemble_kernel(z):
    """Accumulator bits w = 0x4B400000 + z (the float 1.5 * 2^23 + z), level
    pairs w_a * 256 + w_b (mod 2^32), widened into one 64-bit sum."""
    w = [f32_bits(np.float32(zl) + MAGIC) for zl in z]
    p = [(w[2 * q] * 256 + w[2 * q + 1]) & M32 for q in range(3)]
    # level 6: (accumulator - 1.5 * 2^23 + 128) exactly, then x / 256 + 1.5 * 2^23 rounded down
    t = float(np.float32(np.float32(z[6]) + MAGIC) + np.float32(128.0 - 12582912.0))
    assert t == z[6] + 128
    w6 = f32_bits(np.float32(math.floor(t / 256 + 12582912.0)))
    y = ((p[0] + (LEVEL_BIAS >> 32)) & M32) << 32 | (LEVEL_BIAS & M32)
    y = (y + w6) & M64
    y = (y + p[2]) & M64
    y = (y + p[1] * 65536) & M64
    return s64(y)


def test_reassembly_equals_exact_level_sum():
    rng = np.random.default_rng(12)
    lim = 1 << 22
    cases = [[lim] * 7, [-lim] * 7, [0] * 7, [lim, -lim, lim, -lim, lim, -lim, 127],
             [1, 2, 3, 4, 5, 6, 128], [0, 0, 0, 0, 0, 0, -129]]
    cases += [[int(v) for v in rng.integers(-lim, lim + 1, size=7)] for _ in range(20000)]
    cases += [[int(rng.choice([-lim, lim, 0, -1, 1, 127, 128, -128, -129, 255, 256])) for _ in range(7)]
              for _ in range(5000)]
    for z in cases:
        # each pair, offset, lies in [0, 2^32): no wrap before it is widened
        for q in range(3):
            assert 0 <= 256 * z[2 * q] + z[2 * q + 1] + PAIR_OFFSET < 1 << 32
        exact = sum(z[l] * (1 << (8 * (5 - l))) for l in range(6)) + math.floor((z[6] + 128) / 256)
        assert reassemble_kernel(z) == exact, z


def test_level_sums_exact_in_float32_with_preload():
    """Digit products summed in float32 from the preload 1.5 * 2^23, in any
    order, stay exact while the sum of their magnitudes is at most 2^22 (the
    host's per-block check)."""
    rng = np.random.default_rng(13)
    for _ in range(300):
        n = int(rng.integers(1, 200))
        a = rng.integers(-128, 128, size=n)
        b = rng.integers(-128, 128, size=n)
        prods = [int(x) * int(y) for x, y in zip(a, b)]
        scale = sum(abs(p) for p in prods)
        if scale > 1 << 22:
            continue
        acc = MAGIC
        for k in rng.permutation(n):
            acc = np.float32(acc + np.float32(prods[k]))
        assert f32_bits(acc) - MAGIC_BITS == sum(prods)


# ---------------------------------------------------------------------------
# complex64: the bfloat16 triple split of float32 components
# ---------------------------------------------------------------------------
def bf16_rn(x):
    """float32 -> bfloat16 (round to nearest, ties to even), returned as float32."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32)


def triple_split(x):
    x = np.asarray(x, dtype=np.float32)
    h = bf16_rn(x)
    r1 = (x - h).astype(np.float32)
    m = bf16_rn(r1)
    r2 = (r1 - m).astype(np.float32)
    return h, m, bf16_rn(r2), r1, r2


def test_triple_split_residuals_exact_and_bounded():
    rng = np.random.default_rng(21)
    x = np.concatenate([rng.standard_normal(200000).astype(np.float32),
                        (rng.standard_normal(20000) * 10.0 ** rng.integers(-30, 30, 20000)).astype(np.float32),
                        np.float32([1.0, -1.0, 0.5, 3.0, 1.0 / 3.0, 2.0 ** -100])])
    h, m, l, r1, r2 = triple_split(x)
    x64, h64, m64, l64 = (v.astype(np.float64) for v in (x, h, m, l))
    # both residuals are exact in float32
    assert np.array_equal(r1.astype(np.float64), x64 - h64)
    assert np.array_equal(r2.astype(np.float64), x64 - h64 - m64)
    # the three parts carry float32 accuracy
    err = np.abs(x64 - h64 - m64 - l64)
    assert np.all(err <= 2.0 ** -24 * np.abs(x64))


def test_triple_split_products_keep_float32_accuracy():
    """Dot products from the six part products with i + j <= 2 (levels 0..2,
    the dropped ones below 2^-24 relative), summed in float32, stay within a
    few float32 ulps of the exact result."""
    rng = np.random.default_rng(22)
    for _ in range(200):
        n = int(rng.integers(8, 65))
        a = rng.standard_normal(n).astype(np.float32)
        b = rng.standard_normal(n).astype(np.float32)
        pa, pb = triple_split(a)[:3], triple_split(b)[:3]
        acc = np.float32(0)
        for i in range(3):
            for j in range(3 - i):
                acc = np.float32(acc + np.float32(np.dot(pa[i].astype(np.float64), pb[j].astype(np.float64))))
        exact = float(np.dot(a.astype(np.float64), b.astype(np.float64)))
        scale = float(np.dot(np.abs(a.astype(np.float64)), np.abs(b.astype(np.float64))))
        assert abs(float(acc) - exact) <= 8 * 2.0 ** -24 * scale
