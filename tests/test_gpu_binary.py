"""The two-label sweep (PCAD_KERNEL_BINARY: one launch per sweep, each site
drawn by a read of the resident kernel's threshold table and a compare)
against the general CUDA-core kernel and the FP64 oracle: free-running
chains are label-for-label identical with the same FP64 re-draw count, AUTO
takes it for two-label images of 2^18 sites and more, and batches and the
server run their large two-label chains on it with the chains' results."""
import numpy as np
import pytest

import oracle
from pcad_inputs import Model, flip_noise, shapes_binary

pytestmark = pytest.mark.gpu

CUDA_CORE, RESIDENT, BINARY = 1, 5, 8
POTTS, FLIP = 0, 1


@pytest.fixture(scope="module")
def pc():
    import paper_2507_14869_gb300 as pc
    pc.lib()
    return pc


def _binary(seed, H, W, p=0.1):
    return flip_noise(seed + 1, shapes_binary(seed, H, W, n_shapes=max(4, H * W // 4096)), p)


def _ising(nbhd=4, coef=1.2, p=0.1, inertia=1.0):
    return Model(L=2, nbhd=nbhd, pair=POTTS, pair_coef=coef, noise=FLIP, flip_p=p,
                 inertia=inertia)


CASES = [
    ("ragged_4nb", lambda: _binary(1, 130, 257), _ising()),
    ("ragged_8nb", lambda: _binary(2, 97, 203), _ising(nbhd=8, coef=0.6)),
    ("one_row", lambda: _binary(3, 1, 301), _ising()),
    ("one_col_8nb", lambda: _binary(4, 77, 1), _ising(nbhd=8, coef=0.5)),
    ("w129_h33_no_inertia", lambda: _binary(5, 33, 129, p=0.2), _ising(coef=0.9, p=0.2,
                                                                        inertia=0.0)),
    ("w128_h40_strong", lambda: _binary(6, 40, 128, p=0.3), _ising(coef=2.5, p=0.3,
                                                                    inertia=3.0)),
]


@pytest.mark.parametrize("name,make,m", CASES, ids=[c[0] for c in CASES])
def test_binary_sweep_equals_general_kernel_and_oracle(pc, name, make, m):
    g = make()
    outs = {}
    for kind in (BINARY, CUDA_CORE):
        with pc.Chain(g, m, seed=11, chain_id=4, burn_in=7) as ch:
            ch.set_kernel(kind)
            assert ch.kernel_in_use() == kind
            ch.run(40)
            outs[kind] = (ch.sample(), ch.mean(), ch.fp64_draws())
    assert np.array_equal(outs[BINARY][0], outs[CUDA_CORE][0])
    assert np.array_equal(outs[BINARY][1], outs[CUDA_CORE][1])
    assert outs[BINARY][2] == outs[CUDA_CORE][2]   # the same draws go to FP64
    xo, acc, nacc, _ = oracle.run_chain(m, g, 40, 7, seed=11, chain=4)
    assert np.array_equal(outs[BINARY][0], xo)
    np.testing.assert_allclose(outs[BINARY][1], acc / nacc, rtol=1e-6, atol=0)


def test_auto_rule_and_validation(pc):
    m = _ising()
    for shape, expect in (((64, 64), RESIDENT), ((511, 512), CUDA_CORE), ((512, 512), BINARY),
                          ((700, 700), BINARY), ((5, 52429), BINARY)):
        with pc.Chain(_binary(7, *shape), m, seed=1) as ch:
            assert ch.kernel_in_use() == expect, shape
    g = _binary(8, 40, 40)
    with pc.Chain(g, Model(L=2, pair=POTTS, pair_coef=1.0, noise=FLIP, flip_p=0.1,
                           sampler=1), seed=1) as ch:
        with pytest.raises(pc.PcadError):
            ch.set_kernel(BINARY)
    with pc.Chain(np.minimum(g, 1) * 2, Model(L=3, pair=POTTS, pair_coef=1.0, sigma=1.0),
                  seed=1) as ch:
        with pytest.raises(pc.PcadError):
            ch.set_kernel(BINARY)


def test_large_binary_chain_with_blocking_and_model_change(pc):
    """At 2048^2 (AUTO: the two-label sweep) a run with a coefficient change
    mid-run equals the general kernel's; temporal blocking takes over from
    it with the same labels."""
    g = _binary(9, 2048, 2048)
    m = _ising()
    m2 = _ising(coef=0.8, inertia=0.5)
    res = []
    for kind, k in ((0, 0), (CUDA_CORE, 0), (0, 4)):
        with pc.Chain(g, m, seed=3, chain_id=1, burn_in=5) as ch:
            ch.set_kernel(kind)
            ch.set_blocking(k)
            assert ch.kernel_in_use() == (BINARY if (kind, k) == (0, 0) else
                                          CUDA_CORE if k == 0 else -k)
            ch.run(17)
            ch.set_model(m2)
            ch.run(16)
            res.append((ch.sample(), ch.mean()))
    for x, mu in res[1:]:
        assert np.array_equal(x, res[0][0]) and np.array_equal(mu, res[0][1])


def _alone(pc, g, m, seed, chain, burn, n):
    with pc.Chain(g, m, seed=seed, chain_id=chain, burn_in=burn) as ch:
        ch.run(n)
        return ch.sample(), ch.mean()


def test_large_binary_slots_in_batch_and_server(pc):
    """Two-label images of at least one wave of the two-label sweep's tiles
    run it as their own launches inside the batch's and the server's slices
    (planes chosen by the device sweep counter, budgets ending inside a
    slice, one chain changing its coefficients between runs): results equal
    the chains run alone."""
    big = (_binary(10, 1700, 1600), _ising(), 21, 3, 7)
    big8 = (_binary(11, 1601, 1599), _ising(nbhd=8, coef=0.6), 22, 4, 5)
    small = (_binary(12, 64, 64), _ising(), 23, 5, 3)
    mid = (_binary(13, 300, 257), _ising(coef=0.9), 24, 6, 4)
    jobs = [big, big8, small, mid]
    assert all(g.size >= 1216 * 16 * 128 for g, *_ in jobs[:2])
    m_new = _ising(coef=0.7, inertia=0.3)
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
    from test_gpu_batch_serve import _serve_until_done
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
