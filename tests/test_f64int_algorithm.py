"""The integer algorithms behind the FP64 kernels' double multiplications and
additions (fe_f64int.cuh), restated step by step with Python integers on the bit
patterns, against IEEE binary64 products and sums (numpy, round to nearest even):
random operands over the whole normal range, ties, cancellations, every exponent
difference of an addition and the edges of the fast path. The GPU self-test
(tests/test_gpu_f64int.py) compares the compiled code with the hardware
instructions; this checks the steps themselves on the CPU."""
import struct

import numpy as np
import pytest

M64 = (1 << 64) - 1


def bits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def dbl(u):
    return struct.unpack("<d", struct.pack("<Q", u & M64))[0]


def emu_mul(a, b):
    ua, ub = bits(a), bits(b)
    ah, al, bh, bl = ua >> 32, ua & 0xFFFFFFFF, ub >> 32, ub & 0xFFFFFFFF
    ea, eb = (ah >> 20) & 0x7FF, (bh >> 20) & 0x7FF
    e0 = ea + eb - 1023
    za, zb = (ua & 0x7FFFFFFFFFFFFFFF) == 0, (ub & 0x7FFFFFFFFFFFFFFF) == 0
    na, nb = 1 <= ea <= 2046, 1 <= eb <= 2046
    if (za and (nb or zb)) or (zb and na):
        return dbl(((ah ^ bh) & 0x80000000) << 32)     # a zero operand: the signed zero
    if not (na and nb and 1 <= e0 <= 2044):
        return None                                    # left to the hardware instruction
    mah, mbh = (ah & 0xFFFFF) | 0x100000, (bh & 0xFFFFF) | 0x100000
    t0 = al * bl
    t1 = mah * bl + (t0 >> 32)
    t2 = al * mbh + (t1 & 0xFFFFFFFF)
    H = mah * mbh + (t1 >> 32) + (t2 >> 32)
    M, L = t2 & 0xFFFFFFFF, t0 & 0xFFFFFFFF
    s = H >> 41
    Q = ((H << 12) | (M >> 20)) & M64
    m = Q >> s
    rbit = (Q & 1) if s else ((M >> 19) & 1)
    sticky = (M & (0xFFFFF if s else 0x7FFFF)) | L
    m += rbit & (int(sticky != 0) | (m & 1))
    r = (((e0 + s - 1) << 52) + m) | (((ah ^ bh) & 0x80000000) << 32)
    return dbl(r)


def clz64(v):
    return 64 - v.bit_length()


def emu_add(a, b):
    ua, ub = bits(a), bits(b)
    ea, eb = (ua >> 52) & 0x7FF, (ub >> 52) & 0x7FF
    if not (1 <= ea <= 2046 and 1 <= eb <= 2046):
        return None
    swap = (ub & 0x7FFFFFFFFFFFFFFF) > (ua & 0x7FFFFFFFFFFFFFFF)
    x, y = (ub, ua) if swap else (ua, ub)
    ex, ey = (eb, ea) if swap else (ea, eb)
    mx = ((x & 0xFFFFFFFFFFFFF) | (1 << 52)) << 10
    my = ((y & 0xFFFFFFFFFFFFF) | (1 << 52)) << 10
    d = min(ex - ey, 63)
    lost = my & ((1 << d) - 1)
    my = (my >> d) | int(lost != 0)
    S = (mx - my) if ((x ^ y) >> 63) else (mx + my)
    if S == 0:
        return 0.0
    lz = clz64(S)
    e = ex + 1 - lz
    if not (1 <= e <= 2045):
        return None
    S = ((S >> 1) | (S & 1)) if lz == 0 else ((S << (lz - 1)) & M64)
    m = S >> 10
    rbit = (S >> 9) & 1
    m += rbit & (int((S & 0x1FF) != 0) | (m & 1))
    r = (((e - 1) << 52) + m) | (x & 0x8000000000000000)
    return dbl(r)


def emu_add_nz(a, b):
    """i64_dadd_nz: normal or zero operands with a normal or zero result on the
    integer path (a zero operand returns the other one, two zeros the AND of
    their bit patterns); None where the kernel reports a special case."""
    ua, ub = bits(a), bits(b)
    ea, eb = (ua >> 52) & 0x7FF, (ub >> 52) & 0x7FF
    na, nb = 1 <= ea <= 2046, 1 <= eb <= 2046
    za, zb = ((ua << 1) & M64) == 0, ((ub << 1) & M64) == 0
    if not ((na or za) and (nb or zb)):
        return None
    if za:
        return dbl(ua & ub) if zb else dbl(ub)
    if zb:
        return dbl(ua)
    return emu_add(a, b)


def _check(op, emu, pairs):
    n_fast = 0
    for a, b in pairs:
        got = emu(a, b)
        with np.errstate(all="ignore"):
            ref = float(op(np.float64(a), np.float64(b)))
        if got is None:
            continue
        n_fast += 1
        assert bits(got) == bits(ref), (a, b, got, ref)
    return n_fast


def _operands(rng, n, lo=-300, hi=300):
    mant = rng.uniform(1.0, 2.0, n) * rng.choice([-1.0, 1.0], n)
    return mant * 2.0 ** rng.integers(lo, hi, n).astype(float)


def test_mul_random_and_edges():
    rng = np.random.default_rng(5)
    a, b = _operands(rng, 40000), _operands(rng, 40000)
    pairs = list(zip(a, b))
    # ties and near-ties: short significands whose exact product has a half-ulp tail
    for _ in range(4000):
        x = float(rng.integers(1 << 26, 1 << 27)) * 2.0 ** -26 + 2.0 ** -52 * rng.integers(0, 2)
        y = float(rng.integers(1 << 26, 1 << 27)) * 2.0 ** -26
        pairs.append((x, y))
        pairs.append((1.0 + 2.0 ** -52 * rng.integers(0, 1 << 20), 1.0 + 2.0 ** -52 * rng.integers(0, 1 << 20)))
    # the edges of the fast path: results near the smallest and largest normals
    for ea in (1, 2, 500, 1022, 1023, 1024, 1500, 2045, 2046):
        for eb in (1, 2, 1, 1023, 1024, 2044, 2046):
            x = (1.0 + rng.random()) * 2.0 ** (ea - 1023)
            y = (1.0 + rng.random()) * 2.0 ** (eb - 1023)
            pairs.append((x, y))
            pairs.append((-x, y))
    pairs += [(0.0, 1.5), (1.5, -0.0), (-0.0, -2.5), (0.0, 0.0), (-0.0, 0.0), (0.0, 1e300), (1e-300, -0.0),
              (1e-310, 3.0), (0.0, 1e-310), (0.0, np.inf), (np.inf, 2.0), (np.nan, 1.0), (1.0, 1.0), (-1.0, 1.0)]
    assert _check(np.multiply, emu_mul, pairs) > 40000


def test_add_random_exponent_differences_and_cancellation():
    rng = np.random.default_rng(6)
    pairs = list(zip(_operands(rng, 30000), _operands(rng, 30000)))
    # every exponent difference 0..70, both signs
    for d in range(0, 71):
        for _ in range(150):
            x = (1.0 + rng.random()) * 2.0 ** rng.integers(-20, 20)
            y = (1.0 + rng.random()) * x * 2.0 ** -d * rng.choice([-1.0, 1.0])
            pairs.append((x, y))
            pairs.append((y, x))
    # cancellation: nearby values of opposite sign, and exact cancellation
    for _ in range(5000):
        x = (1.0 + rng.random()) * 2.0 ** rng.integers(-50, 50)
        k = int(rng.integers(1, 1 << 30))
        y = -dbl(bits(x) + k * int(rng.choice([-1, 1])))
        pairs.append((x, y))
        pairs.append((x, -x))
    # ties on addition: a value and a half ulp of it, with either parity
    for _ in range(3000):
        x = dbl(bits(1.0 + rng.random()) | int(rng.integers(0, 2)))
        pairs.append((x, float(np.spacing(x)) / 2))
        pairs.append((x, -float(np.spacing(x)) / 2))
    # near the smallest normals and the overflow threshold
    for e in (1, 2, 3, 2044, 2045, 2046):
        x = (1.0 + rng.random()) * 2.0 ** (e - 1023)
        pairs += [(x, x), (x, -x * 0.75), (x, x * 2.0 ** -3)]
    pairs += [(0.0, 1.0), (-0.0, 0.0), (1e-310, 1.0), (np.inf, 1.0), (np.nan, 2.0), (1.0, -1.0), (-1.0, 1.0)]
    assert _check(np.add, emu_add, pairs) > 50000


def test_add_nz_matches_ieee_and_zero_rules():
    """The reporting form of the integer addition (i64_dadd_nz): the same sums as
    the fast path where it is taken, zero operands by the sign rule of IEEE
    round-to-nearest addition, and a report (None) for subnormal, infinite and NaN
    operands and for results that leave the normal range."""
    rng = np.random.default_rng(7)
    pairs = list(zip(_operands(rng, 20000), _operands(rng, 20000)))
    for _ in range(3000):
        x = (1.0 + rng.random()) * 2.0 ** rng.integers(-50, 50)
        pairs.append((x, -x))
        pairs.append((x, -dbl(bits(x) + int(rng.integers(1, 1 << 20)))))
    zeros = [(0.0, 0.0), (-0.0, 0.0), (0.0, -0.0), (-0.0, -0.0), (0.0, 1.5), (-0.0, -2.5), (3.0, -0.0),
             (1e300, 0.0), (-0.0, 1e-300)]
    pairs += zeros
    assert _check(np.add, emu_add_nz, pairs) > 20000
    for a, b in zeros:
        assert emu_add_nz(a, b) is not None
    for a, b in [(1e-310, 1.0), (0.0, 1e-310), (np.inf, 1.0), (1.0, np.nan),
                 (2.0 ** -1022 * 1.5, -2.0 ** -1022), (1.7e308, 1.7e308)]:
        assert emu_add_nz(a, b) is None
