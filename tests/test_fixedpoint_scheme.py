"""The numerical scheme of the MLEM pass's fixed-point accumulator, checked on
CPU by exact emulation (rational arithmetic with single-precision rounding):

- the split of a term v/D (v = P rho' <= D) into H = floor(x 2^12) and
  L = round((x 2^12 - H) 2^20) by three fused multiply-adds with the magic
  2^23: H <= 4097, L <= 2^20, the represented value within 2^-33 of v * (1/D);
- the word sums: adding the raw bits (magic + H, magic + L) modulo 2^32 over up
  to 4000 nonzero terms and any number of zero terms, sum H is the H word's
  low 24 bits and sum L the L word minus the H word's top byte, exactly.

These are the bounds the device header states for kAccWords / kItemMaxEvents.
"""
import math
import random
from fractions import Fraction as F

import numpy as np

MAGIC = F(2) ** 23
MAGIC_BITS = 0x4B000000


def f32_round(x: F, mode: str) -> F:
    """x rounded to the nearest float32 ('rn', ties to even) or towards zero ('rz')."""
    if x == 0:
        return F(0)
    s = -1 if x < 0 else 1
    a = abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    while F(2) ** e > a:
        e -= 1
    while F(2) ** (e + 1) <= a:
        e += 1
    ulp = F(2) ** (e - 23)
    q = a / ulp
    fl = q.numerator // q.denominator
    r = q - fl
    if mode == "rz":
        n = fl
    else:
        n = fl + 1 if (r > F(1, 2) or (r == F(1, 2) and fl % 2 == 1)) else fl
    return s * n * ulp


def f32(x: float) -> F:
    return F(float(np.float32(x)))


def split(v: F, D: F):
    """The kernel's three FMAs for one term: returns (H, L, 1/D as float32)."""
    invD = f32_round(F(1) / D, "rn")
    s2, sl = invD * 4096, invD * F(2) ** 32                     # exact power-of-two scalings
    t1 = f32_round(v * s2 + MAGIC, "rz")                          # magic + floor(x 2^12)
    c = f32_round(t1 * F(-(2 ** 20)) + (F(2) ** 43 + MAGIC), "rn")
    t2 = f32_round(v * sl + c, "rn")                              # magic + L
    return t1 - MAGIC, t2 - MAGIC, invD, c


def test_split_bounds_and_error():
    rng = random.Random(3)
    worst = F(0)
    for _ in range(4000):
        D = f32(rng.uniform(1e-6, 1e3))
        frac = rng.choice([rng.random(), rng.random() ** 8, 1.0, 1e-9 * rng.random(), 0.0])
        v = min(f32(float(D) * frac), D)
        H, L, invD, c = split(v, D)
        assert H.denominator == 1 and 0 <= H <= 4097
        assert L.denominator == 1 and 0 <= L <= 2 ** 20
        assert c == MAGIC - H * 2 ** 20                               # the FMA is exact
        err = abs((H + L / 2 ** 20) / 4096 - v * invD)
        worst = max(worst, err)
    assert worst <= F(1, 2 ** 33)


def test_word_sums_recover_exactly():
    rng = np.random.Generator(np.random.PCG64(9))
    for trial in range(200):
        n_nz = int(rng.integers(0, 4001))                 # nonzero terms of one item
        n_zero = int(rng.integers(0, 50000))              # zero adds (idle lanes, masked pixels)
        H = rng.integers(0, 4098, n_nz)
        L = rng.integers(0, 2 ** 20 + 1, n_nz)
        if trial == 0:                                    # the worst case of the bound
            n_nz, H, L = 4000, np.full(4000, 4097), np.full(4000, 2 ** 20)
        wh = (int(H.sum()) + (n_nz + n_zero) * MAGIC_BITS) % 2 ** 32
        wl = (int(L.sum()) + (n_nz + n_zero) * MAGIC_BITS) % 2 ** 32
        sh = wh & 0xFFFFFF
        sl = (wl - (wh & 0xFF000000)) % 2 ** 32
        assert sh == int(H.sum()) and sl == int(L.sum())
    assert 4000 * 4097 < 2 ** 24 and 4000 * 2 ** 20 < 2 ** 32
    assert math.log2(4000 * 4097) < 24
