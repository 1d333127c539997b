"""The exactness argument behind the encrypted model's multiply-accumulate on the
tensor cores, checked with plain integers and numpy's IEEE fp16 / f32 on the CPU
(no GPU, no library code): a residue of a prime below 2^55, centred, is seven
balanced base-256 digits; the digits are exact in fp16 and so are their products;
an f32 sum of up to 256 digit products is exact in any order; the f32 -> integer
conversion by adding 1.5 * 2^23 is exact on [-2^22, 2^22]; and the 49 digit-pair
sums, rebuilt in 128-bit arithmetic with the conversion biases removed, give the
product sum of the residues exactly, so one reduction mod q yields the residue the
plain 64-bit modular arithmetic gives (the diagonal method of Section 4.3 with the
model encrypted, Section 8.3)."""
import numpy as np

BIAS = 0x0080808080808080          # 128 in bytes 0-6
MAGIC = np.float32(12582912.0)     # 1.5 * 2^23
MAGIC_BITS = 0x4B400000
M128 = (1 << 128) - 1


def _primes_below_2_55(n, seed=1):
    """n random primes just below 2^55 (Miller-Rabin with the first 12 prime bases, exact below 3.3e24)."""
    def is_prime(x):
        if x < 2:
            return False
        for p in (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37):
            if x % p == 0:
                return x == p
        d, s = x - 1, 0
        while d % 2 == 0:
            d, s = d // 2, s + 1
        for a in (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37):
            y = pow(a, d, x)
            if y in (1, x - 1):
                continue
            for _ in range(s - 1):
                y = y * y % x
                if y == x - 1:
                    break
            else:
                return False
        return True
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        c = (1 << 55) - 1 - 2 * int(rng.integers(0, 1 << 40))
        if is_prime(c):
            out.append(c)
    return out


def _digits(v, q):
    """Seven balanced digits of the centred residue of v, from the bytes of v' + BIAS."""
    vc = v - q if v > q // 2 else v
    w = vc + BIAS
    assert 0 <= w < 1 << 63 and (w >> 56) == 0        # byte 7 is zero: no carry lost
    return vc, [((w >> (8 * i)) & 0xFF) - 128 for i in range(7)]


def test_balanced_digits_rebuild_the_centred_residue():
    rng = np.random.default_rng(7)
    for q in _primes_below_2_55(4):
        vals = [0, 1, q // 2, q // 2 + 1, q - 1] + [int(x) for x in rng.integers(0, q, 2000, dtype=np.uint64)]
        for v in vals:
            vc, s = _digits(v, q)
            assert all(-128 <= d <= 127 for d in s)
            assert sum(d * 256 ** i for i, d in enumerate(s)) == vc
            assert vc % q == v


def test_fp16_digits_from_bytes_are_exact():
    """0x6400 | byte is the fp16 of 1024 + byte; less 1152 it is byte - 128, exactly."""
    b = np.arange(256, dtype=np.uint16)
    h = (np.uint16(0x6400) | b).view(np.float16)
    assert np.array_equal(h.astype(np.float64), 1024.0 + b)
    s = h - np.float16(1152)
    assert np.array_equal(s.astype(np.int64), b.astype(np.int64) - 128)
    # every digit product is exact in fp16 x fp16 -> f32 (|product| <= 2^14)
    d = np.arange(-128, 128, dtype=np.float32)
    assert np.array_equal(np.outer(d, d).astype(np.int64), np.outer(d.astype(np.int64), d.astype(np.int64)))


def test_f32_sums_of_256_digit_products_are_exact_in_any_order():
    rng = np.random.default_rng(3)
    cases = [np.full(256, 128 * 128), np.full(256, -128 * 127)]
    cases += [rng.integers(-128, 128, 256) * rng.integers(-128, 128, 256) for _ in range(200)]
    for p in cases:
        exact = int(np.sum(p.astype(np.int64)))
        assert abs(exact) <= 1 << 22
        for order in (np.arange(256), rng.permutation(256), np.argsort(p)):
            acc = np.float32(0)
            for x in p[order]:
                acc = np.float32(acc + np.float32(x))
            assert int(acc) == exact


def test_magic_conversion_is_exact_on_the_sum_range():
    xs = np.concatenate([np.arange(-(1 << 22), -(1 << 22) + 1000), np.arange(-5000, 5000),
                         np.arange((1 << 22) - 1000, (1 << 22) + 1),
                         np.random.default_rng(1).integers(-(1 << 22), (1 << 22) + 1, 20000)])
    f = xs.astype(np.float32)
    assert np.array_equal(f.astype(np.int64), xs)                # the integers are f32 values
    bits = (f + MAGIC).view(np.uint32).astype(np.int64)
    assert np.array_equal(bits, xs + MAGIC_BITS)


def test_digit_pair_sums_rebuild_the_product_sum_mod_q():
    """One output of one run: D_ab = sum_j s_a(R_j) s_b(d_j) over up to 256 baby steps, taken
    through f32 and the biased conversion, rebuilt as sum_ab (D_ab + MAGIC_BITS) 256^(a+b) over
    a < 8, b < 7 (digit 7 of R is the zero row) mod 2^128, minus the biases; as a signed 128-bit
    value it is the integer sum_j R'_j d'_j, so its residue is sum_j R_j d_j mod q."""
    S8 = sum(1 << (8 * i) for i in range(8))
    S7 = sum(1 << (8 * i) for i in range(7))
    bias = MAGIC_BITS * S8 * S7 & M128
    rng = np.random.default_rng(11)
    for q in _primes_below_2_55(3, seed=5):
        for nj in (1, 16, 255, 256):
            for extreme in (False, True):
                if extreme:      # every residue at the most negative centred value: the largest |sum|
                    R = [q // 2 + 1] * nj
                    d = [q // 2 + 1] * nj
                else:
                    R = [int(x) for x in rng.integers(0, q, nj, dtype=np.uint64)]
                    d = [int(x) for x in rng.integers(0, q, nj, dtype=np.uint64)]
                Rs = [_digits(v, q)[1] + [0] for v in R]      # eight rows, the last zero
                ds = [_digits(v, q)[1] for v in d]
                t = 0
                for a in range(8):
                    for b in range(7):
                        acc = np.float32(0)
                        for j in range(nj):
                            acc = np.float32(acc + np.float32(Rs[j][a] * ds[j][b]))
                        u = int((acc + MAGIC).view(np.uint32))
                        t = (t + (u << (8 * (a + b)))) & M128
                t = (t - bias) & M128
                signed = t - (1 << 128) if t >> 127 else t
                want = sum(_digits(x, q)[0] * _digits(y, q)[0] for x, y in zip(R, d))
                assert signed == want and abs(want) < 1 << 116
                assert signed % q == sum(x * y for x, y in zip(R, d)) % q
