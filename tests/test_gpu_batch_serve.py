"""Batched chains and the continuous-batching server against chains run
alone (which the parity tests tie to the oracle): every chain's sample and
posterior mean must be bit-identical, whatever else shares the launches."""
import numpy as np
import pytest

import oracle
from pcad_inputs import Model, flip_noise, gaussian_noise, greyscale_scene, shapes_binary

pytestmark = pytest.mark.gpu

POTTS, TL, GAUSS, FLIP = 0, 1, 0, 1


@pytest.fixture(scope="module")
def pc():
    import paper_2507_14869_gb300 as pc
    pc.lib()
    return pc


def _grey(seed, H, W, L, sigma):
    return gaussian_noise(seed + 1, greyscale_scene(seed, H, W, L, n_shapes=6), sigma, L)


def _jobs():
    bin_g = flip_noise(9, shapes_binary(8, 50, 71), 0.1)
    return [
        (bin_g, Model(L=2, pair=POTTS, pair_coef=1.2, noise=FLIP, flip_p=0.1, inertia=1.0), 1, 0, 10),
        (bin_g, Model(L=2, pair=POTTS, pair_coef=1.2, noise=FLIP, flip_p=0.1, inertia=1.0), 1, 1, 10),
        (_grey(2, 67, 45, 16, 1.0), Model(L=16, pair=TL, pair_coef=0.85, pair_T=2, sigma=1.0, inertia=2.0), 5, 3, 7),
        (_grey(3, 1, 1, 16, 1.0), Model(L=16, pair=TL, pair_coef=0.85, pair_T=2, sigma=1.0, inertia=2.0), 5, 4, 0),
        (_grey(4, 3, 130, 256, 20.0), Model(L=256, pair=TL, pair_coef=0.05, pair_T=30, sigma=20.0, inertia=2.0), 6, 5, 12),
        (_grey(5, 40, 33, 256, 20.0), Model(L=256, pair=TL, pair_coef=0.05, pair_T=30, sigma=20.0, inertia=2.0), 6, 6, 12),
        (_grey(6, 45, 52, 5, 1.0), Model(L=5, nbhd=8, pair=POTTS, pair_coef=0.8, sigma=1.0, inertia=0.7), 7, 7, 3),
        (_grey(7, 29, 64, 33, 3.0), Model(L=33, nbhd=8, pair=POTTS, pair_coef=0.8, sigma=3.0, inertia=0.4), 7, 8, 3),
        (_grey(8, 100, 100, 16, 1.2), Model(L=16, pair=TL, pair_coef=0.6, pair_T=3, sigma=1.2, inertia=0.0), 9, 9, 20),
        # a second tensor-core group (8-neighbourhood, T = 25, L % 8 != 0)
        (_grey(10, 50, 61, 201, 18.0), Model(L=201, nbhd=8, pair=TL, pair_coef=0.05, pair_T=25, sigma=18.0, inertia=1.5), 11, 10, 6),
    ]


def _alone(pc, g, m, seed, chain, burn, n):
    with pc.Chain(g, m, seed=seed, chain_id=chain, burn_in=burn) as ch:
        ch.run(n)
        return ch.sample(), ch.mean()


@pytest.mark.parametrize("autotune", [False, True])
def test_batch_is_bit_identical_to_chains_alone(pc, autotune):
    jobs = _jobs()
    b = pc.pcad_batch_create(jobs, autotune=autotune)
    try:
        for n_total, step in ((37, 37), (57, 20)):
            pc.pcad_batch_run(b, step)
            for i, (g, m, seed, chain, burn) in enumerate(jobs):
                H, W = g.shape
                xs, ms = _alone(pc, g, m, seed, chain, burn, n_total)
                assert np.array_equal(pc.pcad_batch_read_sample(b, i, H, W), xs), (i, n_total)
                assert np.array_equal(pc.pcad_batch_read_mean(b, i, H, W), ms), (i, n_total)
        info = pc.pcad_batch_info(b)
        assert info["t"] == 57 and info["tile_rows"] in (4, 8, 16)
        # reset restarts every chain from its observation
        pc.pcad_batch_reset(b)
        pc.pcad_batch_run(b, 37)
        g, m, seed, chain, burn = jobs[5]
        xs, _ = _alone(pc, g, m, seed, chain, burn, 37)
        assert np.array_equal(pc.pcad_batch_read_sample(b, 5, *g.shape), xs)
    finally:
        pc.pcad_batch_destroy(b)


@pytest.mark.parametrize("rows,order", [(4, 2), (8, 2), (12, 2), (16, 0), (8, 1), (24, 2), (64, 0)])
def test_batch_tilings_are_bit_identical(pc, rows, order):
    """Every tiling, the wavefront included, gives each chain's own result; a
    run length that is not a multiple of 16 ends inside a wavefront slice."""
    jobs = _jobs()
    b = pc.pcad_batch_create(jobs, autotune=False)
    try:
        pc.pcad_batch_set_tiling(b, rows, order)
        info = pc.pcad_batch_info(b)
        assert (info["tile_rows"], info["lpt_order"]) == (rows, order)
        pc.pcad_batch_run(b, 21)
        pc.pcad_batch_run(b, 30)
        pc.pcad_batch_sync(b)
        for i, (g, m, seed, chain, burn) in enumerate(jobs):
            xs, ms = _alone(pc, g, m, seed, chain, burn, 51)
            assert np.array_equal(pc.pcad_batch_read_sample(b, i, *g.shape), xs), i
            assert np.array_equal(pc.pcad_batch_read_mean(b, i, *g.shape), ms), i
        for bad in ((0, 2), (6, 1), (68, 0), (8, 3)):
            with pytest.raises(pc.PcadError):
                pc.pcad_batch_set_tiling(b, *bad)
    finally:
        pc.pcad_batch_destroy(b)


def test_batch_chain_matches_oracle(pc):
    """One batched chain checked directly against the FP64 oracle."""
    jobs = _jobs()
    b = pc.pcad_batch_create(jobs, autotune=False)
    try:
        pc.pcad_batch_run(b, 25)
        g, m, seed, chain, burn = jobs[2]
        x, acc, nacc, _ = oracle.run_chain(m, g, 25, burn, seed=seed, chain=chain)
        assert np.array_equal(pc.pcad_batch_read_sample(b, 2, *g.shape), x)
        np.testing.assert_allclose(pc.pcad_batch_read_mean(b, 2, *g.shape), acc / nacc,
                                   rtol=1e-6, atol=0)
    finally:
        pc.pcad_batch_destroy(b)


def _serve_until_done(pc, sv, ids, shapes, slice_sweeps=16, max_steps=10000):
    out = {}
    for _ in range(max_steps):
        pc.pcad_server_step(sv, slice_sweeps)
        for rid in list(ids):
            st, smp, mean = pc.pcad_server_poll(sv, rid, *shapes[rid])
            if st == 2:
                out[rid] = (smp, mean)
                ids.remove(rid)
        if not ids:
            return out
    raise AssertionError("server did not finish")


def test_server_result_is_the_same_alone_and_in_the_mix(pc):
    jobs = _jobs()
    budgets = [40, 73, 16, 5, 33, 29, 50, 21, 64, 27]
    target = 5
    g, m, seed, chain, burn = jobs[target]
    ref = _alone(pc, g, m, seed, chain, burn, budgets[target])
    # alone in a server
    sv = pc.pcad_server_create(8, 1 << 30)
    try:
        rid = pc.pcad_server_submit(sv, g, m, seed, chain, burn, budgets[target])
        res = _serve_until_done(pc, sv, [rid], {rid: g.shape}, slice_sweeps=7)
        assert np.array_equal(res[rid][0], ref[0]) and np.array_equal(res[rid][1], ref[1])
    finally:
        pc.pcad_server_destroy(sv)
    # in a mix: others arrive before and after, with other slice lengths
    sv = pc.pcad_server_create(4, 1 << 30)
    try:
        shapes, ids, order = {}, [], [0, 2, 6, target, 1, 9, 3, 4, 7, 8]
        for k, i in enumerate(order):
            gi, mi, si, ci, bi = jobs[i]
            rid = pc.pcad_server_submit(sv, gi, mi, si, ci, bi, budgets[i])
            shapes[rid] = gi.shape
            ids.append(rid)
            if i == target:
                tid = rid
            if k % 2 == 1:
                pc.pcad_server_step(sv, 3)
        want = {rid: i for rid, i in zip(ids, order)}
        res = _serve_until_done(pc, sv, list(ids), shapes, slice_sweeps=11)
        assert np.array_equal(res[tid][0], ref[0]) and np.array_equal(res[tid][1], ref[1])
        for rid, (smp, mean) in res.items():
            gi, mi, si, ci, bi = jobs[want[rid]]
            xs, ms = _alone(pc, gi, mi, si, ci, bi, budgets[want[rid]])
            assert np.array_equal(smp, xs)
            assert np.array_equal(mean, ms)
    finally:
        pc.pcad_server_destroy(sv)


def test_server_admission_waits_for_budget_and_slots(pc):
    jobs = _jobs()
    g, m, seed, chain, burn = jobs[8]          # 100x100 L=16
    sv = pc.pcad_server_create(16, 100_000)     # room for one 100x100 request at a time
    try:
        ids = [pc.pcad_server_submit(sv, g, m, seed, chain + k, burn, 32) for k in range(3)]
        act, pend, fin = pc.pcad_server_step(sv, 16)
        assert act == 1 and pend == 2 and fin == 0
        assert pc.pcad_server_info(sv)["hbm_used"] <= 200_000
        res = _serve_until_done(pc, sv, list(ids), {r: g.shape for r in ids})
        for k, rid in enumerate(ids):
            xs, ms = _alone(pc, g, m, seed, chain + k, burn, 32)
            assert np.array_equal(res[rid][0], xs)
        with pytest.raises(pc.PcadError):
            pc.pcad_server_submit(sv, np.zeros((400, 400), np.uint8), m, 1, 0, 0, 10)
    finally:
        pc.pcad_server_destroy(sv)


def test_server_wavefront_across_many_tiles(pc):
    """Requests spanning hundreds of 4 x 32 tiles, so that a slice's sweeps of
    one chain overlap inside the wavefront launch; budgets end inside slices."""
    reqs = [
        (_grey(11, 301, 257, 16, 1.0),
         Model(L=16, nbhd=8, pair=TL, pair_coef=0.85, pair_T=2, sigma=1.0, inertia=2.0), 3, 1, 9, 48),
        (_grey(12, 200, 333, 256, 20.0),
         Model(L=256, pair=TL, pair_coef=0.05, pair_T=30, sigma=20.0, inertia=2.0), 4, 2, 5, 35),
        (flip_noise(13, shapes_binary(14, 97, 640), 0.1),
         Model(L=2, pair=POTTS, pair_coef=1.2, noise=FLIP, flip_p=0.1, inertia=1.0), 5, 3, 4, 40),
        (_grey(15, 130, 7, 33, 3.0),
         Model(L=33, nbhd=8, pair=POTTS, pair_coef=0.8, sigma=3.0, inertia=0.4), 6, 4, 2, 21),
    ]
    sv = pc.pcad_server_create(8, 1 << 31)
    try:
        ids, shapes = [], {}
        for g, m, seed, chain, burn, n in reqs:
            rid = pc.pcad_server_submit(sv, g, m, seed, chain, burn, n)
            ids.append(rid)
            shapes[rid] = g.shape
        res = _serve_until_done(pc, sv, list(ids), shapes, slice_sweeps=16)
        for rid, (g, m, seed, chain, burn, n) in zip(ids, reqs):
            xs, ms = _alone(pc, g, m, seed, chain, burn, n)
            assert np.array_equal(res[rid][0], xs)
            assert np.array_equal(res[rid][1], ms)
        assert pc.pcad_server_info(sv)["hbm_used"] == 0
    finally:
        pc.pcad_server_destroy(sv)
    # one of them straight against the oracle
    g, m, seed, chain, burn, n = reqs[3]
    x, acc, nacc, _ = oracle.run_chain(m, g, n, burn, seed=seed, chain=chain)
    assert np.array_equal(res[ids[3]][0], x)
    np.testing.assert_allclose(res[ids[3]][1], acc / nacc, rtol=1e-6, atol=0)


def test_large_tensor_core_slots_in_batch_and_server(pc):
    """A tensor-core eligible image of at least 1216 tiles runs as its own
    launch inside the batch's and the server's slices (planes chosen by the
    device sweep counter, the budget capping the last slice): results equal
    the chains run alone, for runs and budgets that end inside slices."""
    big = (_grey(20, 330, 512, 256, 20.0),
           Model(L=256, pair=TL, pair_coef=0.05, pair_T=30, sigma=20.0, inertia=2.0), 21, 3, 7)
    small = (_grey(21, 40, 33, 256, 15.0),
             Model(L=256, pair=TL, pair_coef=0.05, pair_T=30, sigma=15.0, inertia=2.0), 22, 4, 5)
    other = (_grey(22, 100, 100, 16, 1.2),
             Model(L=16, pair=TL, pair_coef=0.6, pair_T=3, sigma=1.2, inertia=1.0), 23, 5, 9)
    jobs = [big, small, other]
    b = pc.pcad_batch_create(jobs, autotune=False)
    try:
        pc.pcad_batch_run(b, 21)
        pc.pcad_batch_run(b, 30)
        pc.pcad_batch_sync(b)
        for i, (g, m, seed, chain, burn) in enumerate(jobs):
            xs, ms = _alone(pc, g, m, seed, chain, burn, 51)
            assert np.array_equal(pc.pcad_batch_read_sample(b, i, *g.shape), xs), i
            assert np.array_equal(pc.pcad_batch_read_mean(b, i, *g.shape), ms), i
    finally:
        pc.pcad_batch_destroy(b)
    budgets = [37, 20, 45]
    sv = pc.pcad_server_create(8, 1 << 31)
    try:
        ids, shapes = [], {}
        for (g, m, seed, chain, burn), n in zip(jobs, budgets):
            rid = pc.pcad_server_submit(sv, g, m, seed, chain, burn, n)
            ids.append(rid)
            shapes[rid] = g.shape
        res = _serve_until_done(pc, sv, list(ids), shapes, slice_sweeps=16)
        for rid, (g, m, seed, chain, burn), n in zip(ids, jobs, budgets):
            xs, ms = _alone(pc, g, m, seed, chain, burn, n)
            assert np.array_equal(res[rid][0], xs)
            assert np.array_equal(res[rid][1], ms)
    finally:
        pc.pcad_server_destroy(sv)


def test_server_admission_cap(pc):
    """With an admission cap, a request waits while the admitted ones hold
    enough sites (but is admitted when nothing else runs); results are the
    same as without the cap."""
    jobs = _jobs()
    g, m, seed, chain, burn = jobs[8]            # 100 x 100
    sv = pc.pcad_server_create(16, 1 << 30)
    try:
        pc.pcad_server_set_policy(sv, pc.SERVE_FIFO)
        pc.pcad_server_set_limits(sv, 15_000)     # one 100 x 100 request at a time
        ids = [pc.pcad_server_submit(sv, g, m, seed, chain + k, burn, 32) for k in range(3)]
        act, pend, fin = pc.pcad_server_step(sv, 16)
        assert act == 1 and pend == 2 and fin == 0
        res = _serve_until_done(pc, sv, list(ids), {r: g.shape for r in ids})
        for k, rid in enumerate(ids):
            xs, ms = _alone(pc, g, m, seed, chain + k, burn, 32)
            assert np.array_equal(res[rid][0], xs) and np.array_equal(res[rid][1], ms)
        # a request larger than the cap still runs when nothing else is admitted
        pc.pcad_server_set_limits(sv, 100)
        rid = pc.pcad_server_submit(sv, g, m, seed, chain, burn, 25)
        res = _serve_until_done(pc, sv, [rid], {rid: g.shape})
        assert np.array_equal(res[rid][0], _alone(pc, g, m, seed, chain, burn, 25)[0])
    finally:
        pc.pcad_server_destroy(sv)


def test_server_srpt_runs_short_requests_first_and_pauses_long_ones(pc):
    """Shortest remaining work first: with a run set of one request, a short
    request submitted while a long one runs preempts it and finishes first;
    the long one pauses (its state stays on the device) and resumes.  Both
    results equal the chains run alone, and equal the FIFO server's."""
    jobs = _jobs()
    lg, lm, ls, lc, lb = jobs[8]            # 100 x 100, L = 16
    sg, sm, ss, sc, sb = jobs[2]            # 67 x 45, L = 16
    outs = {}
    for policy in (pc.SERVE_SRPT, pc.SERVE_FIFO):
        sv = pc.pcad_server_create(8, 1 << 30)
        try:
            pc.pcad_server_set_policy(sv, policy, 0.0)
            pc.pcad_server_set_limits(sv, 1)  # SRPT: one request per slice; FIFO: one admitted
            lid = pc.pcad_server_submit(sv, lg, lm, ls, lc, lb, 80)
            pc.pcad_server_step(sv, 16)       # the long request runs 16 sweeps
            sid = pc.pcad_server_submit(sv, sg, sm, ss, sc, sb, 32)
            finished_first = None
            res = {}
            for _ in range(100):
                pc.pcad_server_step(sv, 16)
                for rid, shape in ((lid, lg.shape), (sid, sg.shape)):
                    if rid in res:
                        continue
                    st, smp, mean = pc.pcad_server_poll(sv, rid, *shape)
                    if st == 2:
                        res[rid] = (smp, mean)
                        finished_first = finished_first or rid
                if len(res) == 2:
                    break
            assert len(res) == 2
            if policy == pc.SERVE_SRPT:
                assert finished_first == sid   # 32 x 3015 sites left against 64 x 10^4
            else:
                assert finished_first == lid
            outs[policy] = (res[lid], res[sid])
        finally:
            pc.pcad_server_destroy(sv)
    xl, ml = _alone(pc, lg, lm, ls, lc, lb, 80)
    xs, ms = _alone(pc, sg, sm, ss, sc, sb, 32)
    for (l_out, s_out) in outs.values():
        assert np.array_equal(l_out[0], xl) and np.array_equal(l_out[1], ml)
        assert np.array_equal(s_out[0], xs) and np.array_equal(s_out[1], ms)


def test_server_policy_is_validated(pc):
    sv = pc.pcad_server_create(2, 1 << 20)
    try:
        for policy, aging in ((2, 0.1), (-1, 0.1), (1, -0.5), (1, float("nan"))):
            with pytest.raises(pc.PcadError) as e:
                pc.pcad_server_set_policy(sv, policy, aging)
            assert e.value.status == 1
        pc.pcad_server_set_policy(sv, pc.SERVE_FIFO, 0.0)
        pc.pcad_server_set_policy(sv, pc.SERVE_SRPT, 3.0)
    finally:
        pc.pcad_server_destroy(sv)


def test_large_small_label_slots_in_batch_and_server(pc):
    """Chains of at least 1216 tiles of 16 x 32 sites with a small-label model
    (3 <= L <= 16) run the small-label kernel as their own launches inside the
    batch's and the server's slices (planes chosen by the device sweep
    counter, budgets ending inside slices): results equal the chains run
    alone."""
    big16 = (_grey(30, 800, 800, 16, 1.0),
             Model(L=16, pair=TL, pair_coef=0.05, pair_T=30, sigma=1.0, inertia=2.0), 31, 6, 9)
    big8 = (_grey(31, 640, 1000, 8, 1.5),
            Model(L=8, nbhd=8, pair=POTTS, pair_coef=0.7, sigma=1.5, inertia=0.6), 32, 7, 4)
    other = (_grey(32, 90, 70, 16, 1.2),
             Model(L=16, pair=TL, pair_coef=0.6, pair_T=3, sigma=1.2, inertia=1.0), 33, 8, 5)
    jobs = [big16, big8, other]
    b = pc.pcad_batch_create(jobs, autotune=False)
    try:
        pc.pcad_batch_run(b, 21)
        pc.pcad_batch_run(b, 30)
        pc.pcad_batch_sync(b)
        for i, (g, m, seed, chain, burn) in enumerate(jobs):
            xs, ms = _alone(pc, g, m, seed, chain, burn, 51)
            assert np.array_equal(pc.pcad_batch_read_sample(b, i, *g.shape), xs), i
            assert np.array_equal(pc.pcad_batch_read_mean(b, i, *g.shape), ms), i
    finally:
        pc.pcad_batch_destroy(b)
    budgets = [37, 20, 45]
    sv = pc.pcad_server_create(8, 1 << 31)
    try:
        ids, shapes = [], {}
        for (g, m, seed, chain, burn), n in zip(jobs, budgets):
            rid = pc.pcad_server_submit(sv, g, m, seed, chain, burn, n)
            ids.append(rid)
            shapes[rid] = g.shape
        res = _serve_until_done(pc, sv, list(ids), shapes, slice_sweeps=16)
        for rid, (g, m, seed, chain, burn), n in zip(ids, jobs, budgets):
            xs, ms = _alone(pc, g, m, seed, chain, burn, n)
            assert np.array_equal(res[rid][0], xs)
            assert np.array_equal(res[rid][1], ms)
    finally:
        pc.pcad_server_destroy(sv)


@pytest.mark.parametrize("slice_sweeps,rows,order", [(8, 4, 2), (32, 8, 2), (32, 16, 0)])
def test_batch_slice_lengths_are_bit_identical(pc, slice_sweeps, rows, order):
    """Every slice length (sweeps per captured slice, sweeps per wavefront
    launch) gives each chain its own result, for runs ending inside a slice."""
    jobs = _jobs()
    b = pc.pcad_batch_create(jobs, autotune=False)
    try:
        pc.pcad_batch_set_tiling(b, rows, order)
        assert pc.pcad_batch_slice(b, slice_sweeps) == slice_sweeps
        pc.pcad_batch_run(b, 21)
        pc.pcad_batch_run(b, 30)
        pc.pcad_batch_sync(b)
        for i, (g, m, seed, chain, burn) in enumerate(jobs):
            xs, ms = _alone(pc, g, m, seed, chain, burn, 51)
            assert np.array_equal(pc.pcad_batch_read_sample(b, i, *g.shape), xs), i
            assert np.array_equal(pc.pcad_batch_read_mean(b, i, *g.shape), ms), i
        assert pc.pcad_batch_slice(b) == slice_sweeps
        for bad in (1, 12, 64, -8):
            with pytest.raises(pc.PcadError):
                pc.pcad_batch_slice(b, bad)
    finally:
        pc.pcad_batch_destroy(b)


def test_large_windowed_slots_in_batch_and_server(pc):
    """Tensor-core eligible images of at least 8 blocks of 4 x 32 sites per
    SM run the windowed sweep as their own launches inside the batch's and
    the server's slices -- the wavefront form one launch per slice, from 100
    blocks per SM one launch per sweep -- (planes chosen by the device sweep
    counter, budgets ending inside slices), one of them changing its
    coefficients between runs: results equal the chains run alone."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    big4 = (_grey(40, 640, 520, 256, 20.0),
            Model(L=256, pair=TL, pair_coef=0.05, pair_T=30, sigma=20.0, inertia=2.0), 41, 3, 7)
    big8 = (_grey(41, 700, 500, 201, 18.0),
            Model(L=201, nbhd=8, pair=TL, pair_coef=0.05, pair_T=25, sigma=18.0, inertia=1.5),
            42, 4, 5)
    small = (_grey(42, 40, 33, 256, 15.0),
             Model(L=256, pair=TL, pair_coef=0.05, pair_T=30, sigma=15.0, inertia=2.0), 43, 5, 5)
    huge = (_grey(43, 1600, 1300, 256, 25.0),
            Model(L=256, pair=TL, pair_coef=0.05, pair_T=30, sigma=25.0, inertia=2.0), 44, 6, 9)
    jobs = [big4, big8, small, huge]
    tiles = [((g.shape[1] + 31) // 32) * ((g.shape[0] + 3) // 4) for g, *_ in jobs]
    assert all(8 * sms <= n < 100 * sms for n in tiles[:2])   # the wavefront form
    assert tiles[3] >= 100 * sms                                 # one launch per sweep
    m_new = Model(L=256, pair=TL, pair_coef=0.08, pair_T=30, sigma=20.0, inertia=1.0)
    b = pc.pcad_batch_create(jobs, autotune=False)
    try:
        pc.pcad_batch_run(b, 21)
        pc.pcad_batch_set_model(b, 0, m_new)
        pc.pcad_batch_run(b, 30)
        pc.pcad_batch_sync(b)
        for i, (g, m, seed, chain, burn) in enumerate(jobs):
            with pc.Chain(g, m, seed=seed, chain_id=chain, burn_in=burn) as ch:
                ch.run(21)
                if i == 0:
                    ch.set_model(m_new)
                ch.run(30)
                xs, ms = ch.sample(), ch.mean()
            assert np.array_equal(pc.pcad_batch_read_sample(b, i, *g.shape), xs), i
            assert np.array_equal(pc.pcad_batch_read_mean(b, i, *g.shape), ms), i
    finally:
        pc.pcad_batch_destroy(b)
    budgets = [37, 20, 45, 23]
    sv = pc.pcad_server_create(8, 1 << 31)
    try:
        ids, shapes = [], {}
        for (g, m, seed, chain, burn), n in zip(jobs, budgets):
            rid = pc.pcad_server_submit(sv, g, m, seed, chain, burn, n)
            ids.append(rid)
            shapes[rid] = g.shape
        res = _serve_until_done(pc, sv, list(ids), shapes, slice_sweeps=16)
        for rid, (g, m, seed, chain, burn), n in zip(ids, jobs, budgets):
            xs, ms = _alone(pc, g, m, seed, chain, burn, n)
            assert np.array_equal(res[rid][0], xs)
            assert np.array_equal(res[rid][1], ms)
    finally:
        pc.pcad_server_destroy(sv)
