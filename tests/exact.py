"""Exact rational helpers for the oracle pins (test infrastructure).

Everything here is Python ``fractions.Fraction`` / big-integer arithmetic,
independent of the C oracle: a float converts to a Fraction exactly, and
``float(Fraction)`` rounds to nearest (ties to even) in CPython.
"""

from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

U = Fraction(1, 2**53)   # unit roundoff of binary64


def F(x) -> Fraction:
    return Fraction(float(x))


def value(terms) -> Fraction:
    return sum((F(t) for t in terms), Fraction(0))


def ulp(x: float) -> Fraction:
    """ulp of a nonzero finite double."""
    m, e = math.frexp(abs(x))
    return Fraction(2) ** (e - 53)


def greedy(x: Fraction, nterms: int):
    out = []
    for _ in range(nterms):
        t = float(x)
        out.append(t)
        x -= Fraction(t)
    return out


def non_overlapping(terms) -> bool:
    for a, b in zip(terms[:-1], terms[1:]):
        if a == 0:
            if b != 0:
                return False
            continue
        if abs(F(b)) > ulp(a) / 2:
            return False
    return True


# ---------------------------------------------------------------- multi-limb

def mp_words_to_fraction(words, w: int) -> Fraction:
    words = [int(x) for x in words]
    e = np.uint32(words[0]).view(np.int32).item()
    flags = words[1]
    if flags & 2:
        return Fraction(0)
    M = sum(words[2 + i] << (32 * i) for i in range(w))
    v = Fraction(M) * Fraction(2) ** (e - 32 * w)
    return -v if flags & 1 else v


def mp_words(e: int, sign: int, M: int, w: int):
    out = np.zeros(2 + w, dtype=np.uint32)
    if M == 0:
        out[1] = 2 | sign
        return out
    out[0] = np.int32(e).view(np.uint32)
    out[1] = sign
    for i in range(w):
        out[2 + i] = (M >> (32 * i)) & 0xFFFFFFFF
    return out


def mp_round_fraction(x: Fraction, w: int):
    """RN_p(x), ties to even, as (e, sign, M); p = 32 w.  Plain rational
    arithmetic: M = round(|x| 2^(p - e)) with 2^(e-1) <= |x| < 2^e."""
    p = 32 * w
    if x == 0:
        return 0, 0, 0
    sign = 1 if x < 0 else 0
    a = abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    while Fraction(2) ** e <= a:
        e += 1
    while Fraction(2) ** (e - 1) > a:
        e -= 1
    t = a * Fraction(2) ** (p - e)
    q, r = divmod(t.numerator, t.denominator)
    twice = 2 * r
    if twice > t.denominator or (twice == t.denominator and q & 1):
        q += 1
    if q == 1 << p:
        q >>= 1
        e += 1
    return e, sign, q


def mp_from_mpmath(mpf, w: int):
    """(e, sign, M) of an mpmath mpf tuple normalised to p = 32 w bits."""
    sign, man, exp, bc = mpf
    p = 32 * w
    if man == 0:
        return 0, 0, 0
    shift = p - bc
    M = man << shift if shift >= 0 else None
    assert M is not None and M >> (p - 1) == 1
    return exp - shift + p, sign, M
