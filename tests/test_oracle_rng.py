"""Pins for the oracle's counter-based generator (Philox4x32-10) and the
uniform it derives.  CPU only."""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            v = [int(t, 16) for t in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_kat_file_has_vectors():
    assert len(_kat_rows()) == 3


@pytest.mark.parametrize("ctr,key,out", _kat_rows())
def test_philox_known_answers(orc, ctr, key, out):
    assert orc.philox4x32_10(ctr, key) == out


def test_uniform_is_24_bit_and_keyed_by_all_counter_fields(orc):
    base = orc.uniform(1, 0, 0, 0, 0, 0)
    assert 0.0 <= base < 1.0
    assert base * 2 ** 24 == int(base * 2 ** 24)
    # every field of the counter and the key must change the stream
    others = [orc.uniform(2, 0, 0, 0, 0, 0), orc.uniform(1, 1, 0, 0, 0, 0),
              orc.uniform(1, 0, 1, 0, 0, 0), orc.uniform(1, 0, 0, 1, 0, 0),
              orc.uniform(1, 0, 0, 0, 1, 0), orc.uniform(1, 0, 0, 0, 0, 1),
              orc.uniform(1 << 32, 0, 0, 0, 0, 0)]
    assert all(o != base for o in others)


def test_uniform_word_layout(orc):
    """Columns 4m..4m+3 of a row share one Philox call and use words 0..3."""
    seed, chain, tag, sweep, row = 0x123456789ABCDEF, 7, 0, 11, 5
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for m in range(3):
        words = orc.philox4x32_10([m, row, sweep, (tag << 24) | chain], key)
        for j in range(4):
            u = orc.uniform(seed, chain, tag, sweep, row, 4 * m + j)
            assert u == (words[j] >> 8) / 2 ** 24


def test_uniform_statistics(orc):
    """Chi-square on 256 bins and mean of 2^16 uniforms from one sweep plane."""
    n_r, n_c = 64, 1024
    u = np.array([[orc.uniform(99, 3, 0, 4, r, c) for c in range(n_c)] for r in range(n_r)])
    u = u.reshape(-1)
    counts = np.bincount((u * 256).astype(int), minlength=256)
    exp = u.size / 256
    chi2 = float(((counts - exp) ** 2 / exp).sum())
    # 255 dof: mean 255, sd ~22.6; 6 sd band
    assert 120 < chi2 < 390
    assert abs(u.mean() - 0.5) < 6 * (1 / np.sqrt(12 * u.size))
