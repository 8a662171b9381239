"""Unit roundoff and dynamic range of IEEE-754 style formats (oracle; test infrastructure).

* Table 1 lists formats 1-e-m with their unit roundoff; the table's own annotation gives it
  as 2^-(m+1) (the implicit leading bit).
* Table 2 lists the dynamic range, the base-10 logarithm of the ratio between the largest
  finite and the smallest (subnormal) positive value, rounded down.
"""
import math


def unit_roundoff(m: int) -> float:
    """Unit roundoff 2^-(m+1) of a format with m stored mantissa bits (Table 1)."""
    return 2.0 ** (-(m + 1))


def bits(e: int, m: int) -> int:
    """Total width 1 + e + m of a 1-e-m format (Table 1)."""
    return 1 + e + m


def dynamic_range(e: int, m: int) -> int:
    """floor(log10(max_finite / min_subnormal)) of an IEEE-style 1-e-m format (Table 2).

    With bias 2^(e-1)-1: max_finite = (2 - 2^-m) * 2^bias, min_subnormal = 2^(1 - bias - m).
    Computed with exact integer/log arithmetic in log space.
    """
    bias = 2 ** (e - 1) - 1
    log2_ratio = math.log2(2.0 - 2.0 ** (-m)) + bias - (1 - bias - m)
    return math.floor(log2_ratio * math.log10(2.0))

