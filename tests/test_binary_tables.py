"""The two-label kernels' configuration index, replayed on the CPU.

The resident kernel and the two-label sweep draw a site from the entry
e = 2 (b + n1) + x_i of a threshold table, b = (g (NB + 1) + nm) (NB + 1),
where n1 counts the label-1 neighbours inside the image and nm the
neighbours outside it.  The sweep computes it four sites at a time: label
bytes packed in 32-bit words (zero outside the image and beyond W), the
neighbour counts by byte-wise adds of shifted words, the base from the
observation word times (NB + 1)^2 plus nm (NB + 1) on the image border.
This test replays that word arithmetic with Python integers and checks
every site's entry against n1, nm, g and x_i counted from their
definitions, and that no byte sum carries into the next site's byte."""
import numpy as np
import pytest

M32 = 0xFFFFFFFF


def words(plane, H, W):
    """Rows of 32-bit little-endian words with one zero word on each side and
    a zero row above and below (the staged tile of the whole image)."""
    Wq = (W + 3) // 4
    X = np.zeros((H + 2, Wq + 2), dtype=np.int64)
    for r in range(H):
        for q in range(Wq):
            w = 0
            for j in range(4):
                c = 4 * q + j
                if c < W:
                    w |= int(plane[r, c]) << (8 * j)
            X[r + 1, q + 1] = w
    return X


def quad_keys(x, g, NB):
    H, W = x.shape
    X = words(x, H, W)
    G = words(g, H, W)
    Wq = (W + 3) // 4
    keys = np.full((H, W), -1, dtype=np.int64)
    for r in range(H):
        for q in range(Wq):
            R, Q = r + 1, q + 1
            M, U, D = int(X[R, Q]), int(X[R - 1, Q]), int(X[R + 1, Q])
            left = ((M << 8) | (int(X[R, Q - 1]) >> 24)) & M32
            right = ((M >> 8) | (int(X[R, Q + 1]) << 24)) & M32
            S = U + D + left + right
            if NB == 8:
                Ul, Ur = int(X[R - 1, Q - 1]), int(X[R - 1, Q + 1])
                Dl, Dr = int(X[R + 1, Q - 1]), int(X[R + 1, Q + 1])
                S += (((U << 8) | (Ul >> 24)) & M32) + (((U >> 8) | (Ur << 24)) & M32)
                S += (((D << 8) | (Dl >> 24)) & M32) + (((D >> 8) | (Dr << 24)) & M32)
            nv = min(4, W - 4 * q)
            act = M32 if nv >= 4 else (1 << (8 * nv)) - 1
            S += (int(G[R, Q]) & act & 0x01010101) * (NB + 1) * (NB + 1)
            if r == 0 or r == H - 1 or q == 0 or 4 * q + 4 >= W:
                for j in range(4):
                    c = 4 * q + j
                    nm = (r == 0) + (r == H - 1) + (c == 0) + (c == W - 1)
                    if NB == 8:
                        nm += ((r == 0 or c == 0) + (r == 0 or c == W - 1) +
                               (r == H - 1 or c == 0) + (r == H - 1 or c == W - 1))
                    S += (nm * (NB + 1)) << (8 * j)
            assert S <= M32   # a 32-bit word
            for j in range(nv):
                b = (S >> (8 * j)) & 0xFF
                keys[r, 4 * q + j] = 2 * b + ((M >> (8 * j)) & 1)
    return keys


def defined_keys(x, g, NB):
    H, W = x.shape
    offs = [(-1, 0), (1, 0), (0, -1), (0, 1)]
    if NB == 8:
        offs += [(-1, -1), (-1, 1), (1, -1), (1, 1)]
    keys = np.zeros((H, W), dtype=np.int64)
    for r in range(H):
        for c in range(W):
            n1 = nm = 0
            for dr, dc in offs:
                rr, cc = r + dr, c + dc
                if 0 <= rr < H and 0 <= cc < W:
                    n1 += int(x[rr, cc])
                else:
                    nm += 1
            b = (int(g[r, c]) * (NB + 1) + nm) * (NB + 1)
            keys[r, c] = 2 * (b + n1) + int(x[r, c])
    return keys


@pytest.mark.parametrize("NB", [4, 8])
@pytest.mark.parametrize("H,W", [(1, 1), (1, 9), (7, 1), (5, 12), (6, 13), (9, 30), (3, 4)])
def test_quad_keys_match_the_configuration_definition(NB, H, W):
    rng = np.random.default_rng(H * 100 + W + NB)
    for trial in range(3):
        x = rng.integers(0, 2, (H, W)).astype(np.uint8)
        g = rng.integers(0, 2, (H, W)).astype(np.uint8)
        if trial == 1:
            x[:] = 1   # the largest neighbour counts
        keys = quad_keys(x, g, NB)
        assert np.array_equal(keys, defined_keys(x, g, NB))
        assert keys.max() < 4 * (NB + 1) * (NB + 1)   # inside the table
