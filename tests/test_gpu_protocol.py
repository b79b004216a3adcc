"""The paper protocol on the GPU against the oracle:

* annealed schedules (coefficients changed between stages, state and
  sweep counter carried on) give exactly the oracle's chain, for the lazy
  PCA and for 4-colour Gibbs;
* prior-only Gibbs sampling (the synthetic MRF images) equals the oracle's;
* the batched q grid (per-chain coefficient changes between stages) gives
  each chain's result as when run alone;
* set_model refuses structural changes."""
import numpy as np
import pytest

import oracle
from pcad_inputs import Model, gaussian_noise, random_lattice

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pc():
    import paper_2507_14869_gb300 as pc
    pc.lib()
    return pc


def _oracle_schedule(models, sweeps, g, seed, chain, sampler):
    x, acc, t = g.copy(), None, 0
    for m, n in zip(models, sweeps):
        x, acc, _, _ = oracle.run_chain(Model(**m), g, n, 0, seed=seed, chain=chain,
                                        sampler=sampler, x0=x, acc=acc, t0=t)
        t += n
    return x, acc


@pytest.mark.parametrize("sampler", [0, 1])
@pytest.mark.parametrize("L,sigma,shape", [(5, 0.25, (23, 37)), (33, 0.1, (19, 40))])
def test_annealed_schedule_matches_oracle(pc, sampler, L, sigma, shape):
    from paper_2507_14869_gb300 import protocol as pr
    clean = random_lattice(3, *shape, L)
    g = gaussian_noise(4, clean, sigma * (L - 1), L)
    ms, sw = pr.schedule(L, J=1 / 3, q=0.46, sigma=sigma, sampler=sampler, stage_sweeps=6)
    sw = [6, 11, 33, 4]   # a graph block inside one stage, ragged remainders
    with pc.Chain(g, ms[0], seed=7, chain_id=2, burn_in=0) as ch:
        ch.run_schedule(ms, sw)
        xg, mg = ch.sample(), ch.mean()
    x, acc = _oracle_schedule(ms, sw, g, 7, 2, sampler)
    assert np.array_equal(xg, x)
    np.testing.assert_allclose(mg, acc / sum(sw), rtol=1e-6, atol=0)


def test_mrf_image_matches_oracle_prior_sampling(pc):
    from paper_2507_14869_gb300 import protocol as pr
    init = random_lattice(9, 41, 37, 9)
    img = pr.mrf_image(init, L=9, J=1 / 3, beta=1.5, sweeps=40, seed=5)
    m = Model(L=9, nbhd=8, pair=0, pair_coef=2 * 1.5 / 3, noise=2, sampler=1)
    x, _, _, _ = oracle.run_chain(m, init, 40, 40, seed=5, chain=0, sampler=1)
    assert np.array_equal(img, x)
    # prior sampling in the ordered phase coarsens the random start
    pairs = lambda a: np.count_nonzero(a[:, 1:] == a[:, :-1]) + np.count_nonzero(a[1:] == a[:-1])
    assert pairs(img) > 3 * pairs(init)


def test_q_grid_batch_equals_single_chains(pc):
    from paper_2507_14869_gb300 import protocol as pr
    L, sigma = 9, 0.2
    clean = random_lattice(11, 30, 45, L)
    g = gaussian_noise(12, clean, sigma * (L - 1), L)
    qs, runs = (0.06, 0.46), 2
    sched = dict(stage_sweeps=5)
    res, xs = pr.q_grid(g, clean, L, J=1 / 3, sigma=sigma, seed=3, qs=qs, runs=runs,
                        return_samples=True, **sched)
    for qi, q in enumerate(qs):
        for r in range(runs):
            k = qi * runs + r
            x = pr.restore(g, L, J=1 / 3, q=q, sigma=sigma, seed=3, chain_id=k, **sched)
            assert np.array_equal(xs[q][r], x)
            # the GPU metric reductions use FP64 atomics: equal up to summation order
            np.testing.assert_allclose(res[q][r], pr.metrics(x, clean, L), rtol=1e-12)
    # and one of them against the oracle
    ms, sw = pr.schedule(L, 1 / 3, qs[1], sigma, **sched)
    xo, _ = _oracle_schedule(ms, sw, g, 3, runs, 0)
    assert np.array_equal(xs[qs[1]][0], xo)


def test_set_model_refuses_structural_changes(pc):
    g = random_lattice(1, 10, 10, 5)
    m = dict(L=5, nbhd=8, pair=0, pair_coef=0.5, noise=0, sigma=1.0, inertia=0.5)
    with pc.Chain(g, m, seed=1) as ch:
        for bad in (dict(L=6), dict(nbhd=4), dict(pair=1, pair_T=2), dict(noise=2)):
            with pytest.raises(pc.PcadError):
                ch.set_model({**m, **bad})
        ch.set_model({**m, "pair_coef": 0.9, "inertia": 1.0, "sigma": 2.0})
        ch.run(3)
