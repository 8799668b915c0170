"""Brute-force rounding checker (pure Python, exact rationals).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  This module pins the C
oracle: it shares no code or formula with it.  Instead of integer arithmetic on
significands it

1. lists every finite value of a small format ``1/E/M`` as an exact
   ``fractions.Fraction``, sorted;
2. forms the exact result of ``x + y`` or ``x * y`` as a Fraction;
3. finds the correctly rounded neighbour by binary search in that list:
   round to nearest with ties to the neighbour whose encoding is even, or
   round toward zero (the two modes of the paper's Sec. 4), with IEEE-754
   overflow (RN: to infinity once the magnitude reaches max + half an ulp;
   RZ: to the largest finite value) and IEEE signed zeros.

With flush to zero (rounding modes 2 = RN and 3 = RZ with flush; an optional
mode, not in the paper) every encoding with exponent field 0 reads as a zero
of its sign, an exact result of magnitude below the smallest normal is a zero
of its sign, and the search runs over the normal values only.

Only practical for formats of up to about 12 bits.
"""
from __future__ import annotations

import bisect
from fractions import Fraction
from functools import lru_cache

RN, RZ, RN_FTZ, RZ_FTZ = 0, 1, 2, 3


class Format:
    def __init__(self, E: int, M: int):
        self.E, self.M = E, M
        self.B = 1 + E + M
        self.bias = 2 ** (E - 1) - 1
        self.emax = 2 ** E - 1
        # all non-negative finite encodings, in increasing value order
        self.pos_codes = [(e << M) | f for e in range(self.emax) for f in range(2 ** M)]
        self.pos_vals = [self.value(c) for c in self.pos_codes]
        assert all(a < b for a, b in zip(self.pos_vals, self.pos_vals[1:]))
        self.max_finite = self.pos_vals[-1]
        # the rounding boundary to infinity in RN: max + half an ulp of the top binade
        top_ulp = Fraction(2) ** (self.emax - 1 - self.bias - M)
        self.ovf_rn = self.max_finite + top_ulp / 2
        self.nan = (self.emax << M) | (1 << (M - 1))
        self.sign_bit = 1 << (E + M)
        self.min_normal = Fraction(2) ** (1 - self.bias)
        # the normal encodings only (exponent field >= 1), for flush to zero
        self.norm_codes = [c for c in self.pos_codes if c >> M]
        self.norm_vals = [self.value(c) for c in self.norm_codes]

    # -- decoding ---------------------------------------------------------------
    def fields(self, code: int):
        M, E = self.M, self.E
        return (code >> (E + M)) & 1, (code >> M) & (2 ** E - 1), code & (2 ** M - 1)

    def value(self, code: int) -> Fraction:
        """Exact value of a finite encoding (IEEE-754 style reading)."""
        s, e, f = self.fields(code)
        assert e != self.emax
        if e == 0:
            v = Fraction(f, 2 ** self.M) * Fraction(2) ** (1 - self.bias)
        else:
            v = (1 + Fraction(f, 2 ** self.M)) * Fraction(2) ** (e - self.bias)
        return -v if s else v

    def operand(self, code: int, rnd: int) -> Fraction:
        """Value of a finite operand under the rounding mode's zero rule."""
        if rnd & 2 and self.fields(code)[1] == 0:
            return Fraction(0)
        return self.value(code)

    def is_nan(self, code):
        _, e, f = self.fields(code)
        return e == self.emax and f != 0

    def is_inf(self, code):
        _, e, f = self.fields(code)
        return e == self.emax and f == 0

    def inf(self, s):
        return (s << (self.E + self.M)) | (self.emax << self.M)

    # -- rounding ---------------------------------------------------------------
    def round(self, v: Fraction, rnd: int) -> int:
        """Correctly rounded encoding of a nonzero exact value."""
        assert v != 0
        s = 1 if v < 0 else 0
        a = -v if s else v
        sgn = s * self.sign_bit
        rz, ftz = rnd & 1, rnd & 2
        if ftz and a < self.min_normal:
            return sgn                            # tiny: a zero of the result's sign
        if not rz:
            if a >= self.ovf_rn:
                return self.inf(s)
        else:
            if a > self.max_finite:
                return sgn | self.pos_codes[-1]
        codes, vals = (self.norm_codes, self.norm_vals) if ftz else (self.pos_codes, self.pos_vals)
        i = bisect.bisect_right(vals, a) - 1      # vals[i] <= a
        if vals[i] == a:
            return sgn | codes[i]
        if rz:
            return sgn | codes[i]
        lo, hi = vals[i], vals[i + 1] if i + 1 < len(vals) else None
        if hi is None:                            # between max and the RN boundary
            return sgn | codes[i]
        dl, dh = a - lo, hi - a
        if dl < dh:
            return sgn | codes[i]
        if dh < dl:
            return sgn | codes[i + 1]
        # tie: the neighbour with an even encoding
        return sgn | (codes[i] if codes[i] % 2 == 0 else codes[i + 1])

    # -- operations ---------------------------------------------------------------
    def add(self, x: int, y: int, rnd: int) -> int:
        if self.is_nan(x) or self.is_nan(y):
            return self.nan
        sx, sy = self.fields(x)[0], self.fields(y)[0]
        if self.is_inf(x) and self.is_inf(y):
            return self.inf(sx) if sx == sy else self.nan
        if self.is_inf(x):
            return self.inf(sx)
        if self.is_inf(y):
            return self.inf(sy)
        v = self.operand(x, rnd) + self.operand(y, rnd)
        if v == 0:
            # exact zero: -0 only for (-0) + (-0); otherwise +0 (RN and RZ)
            return self.sign_bit if (sx and sy) else 0
        return self.round(v, rnd)

    def sub(self, x: int, y: int, rnd: int) -> int:
        return self.add(x, y ^ self.sign_bit, rnd)

    def mul(self, x: int, y: int, rnd: int) -> int:
        if self.is_nan(x) or self.is_nan(y):
            return self.nan
        sx, sy = self.fields(x)[0], self.fields(y)[0]
        s = sx ^ sy
        if self.is_inf(x) or self.is_inf(y):
            other = y if self.is_inf(x) else x
            if not self.is_inf(other) and self.operand(other, rnd) == 0:
                return self.nan
            return self.inf(s)
        v = self.operand(x, rnd) * self.operand(y, rnd)
        if v == 0:
            return s * self.sign_bit
        r = self.round(v, rnd)
        # a nonzero product that rounds to zero keeps the sign of the exact result
        return r

    def div(self, x: int, y: int, rnd: int) -> int:
        """IEEE-754 division: NaN for NaN operands, 0/0 and Inf/Inf; x/0 and
        Inf/y are infinities, x/Inf and 0/y zeros, signed by XOR."""
        if self.is_nan(x) or self.is_nan(y):
            return self.nan
        s = self.fields(x)[0] ^ self.fields(y)[0]
        xi, yi = self.is_inf(x), self.is_inf(y)
        if xi and yi:
            return self.nan
        if xi:
            return self.inf(s)
        if yi:
            return s * self.sign_bit
        vx, vy = self.operand(x, rnd), self.operand(y, rnd)
        if vy == 0:
            return self.nan if vx == 0 else self.inf(s)
        if vx == 0:
            return s * self.sign_bit
        return self.round(vx / vy, rnd)

    def from_value(self, v, s: int, rnd: int) -> int:
        """Encoding of an exact value v (a Fraction; s its sign, for zero)
        rounded in mode rnd: the conversion of another format's value."""
        if v == 0:
            return s * self.sign_bit
        return self.round(v, rnd)

    def fma2(self, x: int, y: int, z: int, rnd: int) -> int:
        return self.add(self.mul(x, y, rnd), z, rnd)


@lru_cache(maxsize=None)
def fmt(E: int, M: int) -> Format:
    return Format(E, M)
