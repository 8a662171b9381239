"""Pins of the format helpers against Table 1 and Table 2 (values printed in the paper)."""
import math
import os

from oracle import formats

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLD, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def test_table1_unit_roundoff_and_bits():
    for name, e, m, nbits, printed in _rows("table1_ieee_formats.txt"):
        e, m, nbits = int(e), int(m), int(nbits)
        assert formats.bits(e, m) == nbits, name
        u = formats.unit_roundoff(m)
        # Table 1 prints two significant digits, rounded half up (0.0625 -> 6.3e-2)
        exp10 = math.floor(math.log10(u))
        mant = math.floor(u / 10.0 ** exp10 * 10.0 + 0.5) / 10.0
        assert math.isclose(mant * 10.0 ** exp10, float(printed), rel_tol=1e-12), (name, u, printed)


def test_table2_dynamic_range():
    for name, e, m, printed in _rows("table2_dynamic_range.txt"):
        assert formats.dynamic_range(int(e), int(m)) == int(printed), name

