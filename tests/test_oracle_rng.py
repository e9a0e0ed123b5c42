"""Pins for the oracle's counter-based generator (SplitMix64)."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_vectors.txt")


def _vectors():
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        seed, n, out = (int(v) for v in line.split())
        yield seed, n, out


def test_splitmix64_published_vectors(orc):
    rows = list(_vectors())
    assert len(rows) == 5
    for seed, n, out in rows:
        assert orc.splitmix64(seed, n) == out


def test_draw_streams_are_distinct_and_deterministic(orc):
    a = [orc.draw(7, 3, 2, 1, i) for i in range(64)]
    assert a == [orc.draw(7, 3, 2, 1, i) for i in range(64)]
    assert len(set(a)) == 64
    # changing any coordinate of the counter changes the stream
    for alt in ((8, 3, 2, 1), (7, 4, 2, 1), (7, 3, 3, 1), (7, 3, 2, 2)):
        b = [orc.draw(*alt, i) for i in range(64)]
        assert len(set(a) & set(b)) == 0


def test_draw_high_bits_uniform(orc):
    # 4096 draws in 16 bins of the top 4 bits: chi-square with 15 dof, p ~ 1e-6 bound
    vals = np.array([orc.draw(1, 0, 0, 4, i) >> 60 for i in range(4096)])
    counts = np.bincount(vals, minlength=16)
    chi2 = ((counts - 256.0) ** 2 / 256.0).sum()
    assert chi2 < 50.0
