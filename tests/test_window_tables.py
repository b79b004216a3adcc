"""The windowed sweep's tent arithmetic, replayed on the CPU.

The windowed kernels find the tent sums Pb(s) = sum_j max(T - |x_j - s|, 0)
of a chunk of 8 labels from a table indexed by d = x_j - 8c (clamped to a
zero entry outside (-T, T + 7)), add the neighbours' 8-byte entries as two
32-bit words, and evaluate only the chunks of the hull
[x_min - T + 1, x_max + T - 1] of the present neighbours, taking every other
chunk's sum from the outside table (Pb = 0 there).  This test replays that
index arithmetic with numpy -- the table built from its definition, the
unsigned clamp, the byte-wise word sums -- and checks it against Pb computed
label by label for random neighbourhoods: inside the hull the bytes equal
Pb, outside it Pb is zero, and no byte sum carries into its neighbour."""
import numpy as np
import pytest

MISSING = 1024


def tent_table(T):
    """2T + 8 entries of two little-endian 32-bit words (bytes k = 0..7)."""
    ent = np.zeros((2 * T + 8, 2), np.uint64)
    for i in range(2 * T + 8):
        d = i - T
        b = [max(T - abs(d - k), 0) for k in range(8)]
        ent[i, 0] = sum(b[k] << (8 * k) for k in range(4))
        ent[i, 1] = sum(b[4 + k] << (8 * k) for k in range(4))
    return ent


def chunk_words(tab, T, x, c):
    zero_i = 2 * T + 7
    lo = hi = 0
    for xj in x:
        i = min((xj + T - 8 * c) & 0xFFFFFFFF, zero_i)     # the kernel's unsigned clamp
        lo = (lo + int(tab[i, 0])) & 0xFFFFFFFF
        hi = (hi + int(tab[i, 1])) & 0xFFFFFFFF
    return lo, hi


def hull(x, T, L):
    pres = [v for v in x if v < MISSING]
    nc = (L + 7) // 8
    if not pres:
        return 0, 0
    clo = max(min(pres) - T + 1, 0) >> 3
    return clo, min((max(pres) + T - 1) >> 3, nc - 1) - clo + 1


@pytest.mark.parametrize("L,T,nbhd", [(256, 30, 4), (256, 33, 4), (201, 25, 8), (33, 1, 8),
                                      (64, 2, 4), (9, 31, 8), (100, 31, 8)])
def test_tent_bytes_and_hull_match_the_definition(L, T, nbhd):
    if nbhd * T > 255:
        pytest.skip("not a windowed model")
    rng = np.random.default_rng(L * 100 + T)
    tab = tent_table(T)
    nc = (L + 7) // 8
    s = np.arange(nc * 8)
    for trial in range(400):
        x = list(rng.integers(0, L, nbhd))
        if trial % 5 == 0:   # image edges: missing neighbours
            for j in rng.choice(nbhd, size=int(rng.integers(1, nbhd + 1)), replace=False):
                x[j] = MISSING
        if trial % 7 == 0:   # clustered labels
            base = int(rng.integers(0, L))
            x = [min(L - 1, max(0, base + int(v))) for v in rng.integers(-3, 4, nbhd)]
        pb = np.zeros(nc * 8, np.int64)
        for xj in x:
            if xj < MISSING:
                pb += np.maximum(T - np.abs(xj - s), 0)
        assert pb.max() <= nbhd * T <= 255
        clo, cnt = hull(x, T, L)
        for c in range(nc):
            if clo <= c < clo + cnt:
                lo, hi = chunk_words(tab, T, x, c)
                got = [(lo >> (8 * k)) & 0xFF for k in range(4)] + \
                      [(hi >> (8 * k)) & 0xFF for k in range(4)]
                assert got == list(pb[8 * c:8 * c + 8]), (x, c)
            else:
                assert not pb[8 * c:8 * c + 8].any(), (x, c)   # outside table: Pb = 0


def test_missing_neighbours_and_far_chunks_read_the_zero_entry():
    T = 30
    tab = tent_table(T)
    assert not tab[2 * T + 7].any() and not tab[0].any()
    for c in range(32):
        assert chunk_words(tab, T, [MISSING] * 4, c) == (0, 0)
    # a label 40 below the chunk and one 40 above it: clamped, zero
    assert chunk_words(tab, T, [8 * 20 - 40, 8 * 20 + 47], 20) == (0, 0)
