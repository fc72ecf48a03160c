"""Readers of the values the paper prints (tests/golden/*.txt; each file
cites its section and equations).  Plain text: '#' starts a comment, fields
are separated by blanks, numbers are exact fractions or decimals."""
from fractions import Fraction
from pathlib import Path

GOLDEN = Path(__file__).resolve().parent / "golden"


def _rows(name):
    for line in (GOLDEN / name).read_text().splitlines():
        line = line.split("#", 1)[0].strip()
        if line:
            yield line.split()


def dispersion():
    """{closure: (a, b, c)} of the O(mu) dispersion relation, Fractions."""
    return {r[0]: tuple(Fraction(v) for v in r[1:4]) for r in _rows("dispersion_o_mu.txt")}


def spatial_setup():
    """{name: value} of the spatially resolved runs' setup, Fractions."""
    return {r[0]: Fraction(r[1]) for r in _rows("spatial_setup.txt")}
