"""Tile and box index arithmetic of the tiled kernels, replayed on the CPU.

* The small-label kernel's TMA form: output tiles of 64 x 46 sites, each
  read from the 96 x 48 box at (x0 - 16, y0 - 1) of the plane maps; a
  thread's 4-site group (qr, qc) of a tile sits at box row 1 + qr and box
  columns 16 + 4 qc .. 19 + 4 qc.  Every image site must be written by
  exactly one tile, every neighbour it reads must lie inside the box, the
  box's x origin must be a multiple of 16 bytes (the TMA rule), and the
  tiles called interior (no bounds tests) must have their halo inside the
  image.
* The two-label sweep: tiles of 16 rows x 32 words staged with a one-word
  halo; the same coverage and the same neighbour words as the whole-image
  staging."""
import numpy as np
import pytest

TM_OUT_W, TM_OUT_H, TM_BOX_W, TM_BOX_H, TM_COL_OFF = 64, 46, 96, 48, 16


def small_tma_tiles(H, W):
    tiles_x = (W + TM_OUT_W - 1) // TM_OUT_W
    tiles_y = (H + TM_OUT_H - 1) // TM_OUT_H
    for t in range(tiles_x * tiles_y):
        ty, tx = divmod(t, tiles_x)
        yield tx * TM_OUT_W, ty * TM_OUT_H


@pytest.mark.parametrize("NB", [4, 8])
@pytest.mark.parametrize("H,W", [(1, 1), (46, 64), (47, 65), (93, 200), (140, 129), (5, 300)])
def test_small_tma_tiles_cover_the_image_and_read_inside_the_box(NB, H, W):
    offs = [(-1, 0), (1, 0), (0, -1), (0, 1)]
    if NB == 8:
        offs += [(-1, -1), (-1, 1), (1, -1), (1, 1)]
    written = np.zeros((H, W), np.int64)
    for x0, y0 in small_tma_tiles(H, W):
        bx, by = x0 - TM_COL_OFF, y0 - 1
        assert bx % 16 == 0   # the box's x origin, in bytes of a uint8 plane
        interior = x0 >= 1 and y0 >= 1 and x0 + TM_OUT_W < W and y0 + TM_OUT_H < H
        for qd in range(TM_OUT_H * TM_OUT_W // 4):
            qr, qc = divmod(qd, TM_OUT_W // 4)
            lr, lc0 = 1 + qr, TM_COL_OFF + 4 * qc
            gr, gc0 = y0 + qr, x0 + 4 * qc
            for q in range(4):
                lc, gc = lc0 + q, gc0 + q
                assert (by + lr, bx + lc) == (gr, gc)   # box coordinates map to the site
                if not (gr < H and gc < W):
                    assert not interior
                    continue
                written[gr, gc] += 1
                for dr, dc in offs:
                    assert 0 <= lr + dr < TM_BOX_H and 0 <= lc + dc < TM_BOX_W
                    if interior:
                        assert 0 <= gr + dr < H and 0 <= gc + dc < W
    assert (written == 1).all()


BIN_ROWS, BIN_QW = 16, 32
BIN_PW = BIN_QW + 2


def staged_words(x, r0, q0):
    """The two-label sweep's staged tile: rows r0 - 1 .. r0 + 16, words
    q0 - 1 .. q0 + 32, zero outside the image and beyond W."""
    H, W = x.shape
    Wq = (W + 3) // 4
    X = np.zeros((BIN_ROWS + 2, BIN_PW), np.int64)
    for i in range(X.size):
        lr, lw = divmod(i, BIN_PW)
        gr, gq = r0 - 1 + lr, q0 - 1 + lw
        if 0 <= gr < H and 0 <= gq < Wq:
            w = 0
            for j in range(4):
                c = 4 * gq + j
                if c < W:
                    w |= int(x[gr, c]) << (8 * j)
            X[lr, lw] = w
    return X


@pytest.mark.parametrize("H,W", [(1, 5), (17, 129), (33, 260), (16, 128), (40, 513)])
def test_binary_tiles_stage_the_neighbour_words_of_every_quad(H, W):
    rng = np.random.default_rng(H * 1000 + W)
    x = rng.integers(0, 2, (H, W)).astype(np.uint8)
    Wq = (W + 3) // 4
    tiles_x = (Wq + BIN_QW - 1) // BIN_QW
    ntiles = tiles_x * ((H + BIN_ROWS - 1) // BIN_ROWS)
    seen = np.zeros((H, Wq), np.int64)
    for tile in range(ntiles):
        ty, tx = divmod(tile, tiles_x)
        r0, q0 = ty * BIN_ROWS, tx * BIN_QW
        X = staged_words(x, r0, q0)
        for k in range(BIN_ROWS * BIN_QW):
            lr, lq = divmod(k, BIN_QW)
            gr, gq = r0 + lr, q0 + lq
            if gr >= H or gq >= Wq:
                continue
            seen[gr, gq] += 1
            o_r, o_w = lr + 1, 1 + lq
            # the 3 x 3 words around the quad equal the image's words there
            for dr in (-1, 0, 1):
                for dw in (-1, 0, 1):
                    rr, ww = gr + dr, gq + dw
                    want = 0
                    if 0 <= rr < H and 0 <= ww < Wq:
                        for j in range(4):
                            c = 4 * ww + j
                            if c < W:
                                want |= int(x[rr, c]) << (8 * j)
                    assert X[o_r + dr, o_w + dw] == want
    assert (seen == 1).all()
