"""Posterior energy on the GPU (exact integer reduction + FP64 combination)
against the oracle, and minimum-energy tracking along chains that are
bit-identical to the oracle's: every recorded energy equals the oracle
energy of the oracle chain's state after that sweep, and the kept state is
the first one of lowest energy."""
import numpy as np
import pytest

import oracle
from oracle import energy as oen
from pcad_inputs import Model, flip_noise, gaussian_noise, greyscale_scene, shapes_binary

pytestmark = pytest.mark.gpu

POTTS, TL, FLIP = 0, 1, 1


@pytest.fixture(scope="module")
def pc():
    import paper_2507_14869_gb300 as pc
    pc.lib()
    return pc


def _grey(seed, H, W, L, sigma):
    return gaussian_noise(seed + 1, greyscale_scene(seed, H, W, L, n_shapes=6), sigma, L)


CASES = [
    ("tl_L16_37x53", lambda: (_grey(1, 37, 53, 16, 1.2),
                              Model(L=16, pair=TL, pair_coef=0.6, pair_T=3, sigma=1.2, inertia=1.0))),
    ("tl_L256_8nb_29x70", lambda: (_grey(2, 29, 70, 256, 20.0),
                                   Model(L=256, nbhd=8, pair=TL, pair_coef=0.05, pair_T=30,
                                         sigma=20.0, inertia=2.0))),
    ("flip_potts_40x33", lambda: (flip_noise(3, shapes_binary(4, 40, 33), 0.1),
                                  Model(L=2, pair=POTTS, pair_coef=1.2, noise=FLIP, flip_p=0.1,
                                        inertia=1.0))),
    ("potts_L5_8nb_31x31", lambda: (_grey(5, 31, 31, 5, 0.9),
                                    Model(L=5, nbhd=8, pair=POTTS, pair_coef=0.8, sigma=0.9,
                                          inertia=0.7))),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_energy_matches_oracle(pc, name, make):
    g, m = make()
    with pc.Chain(g, m, seed=4, chain_id=1, burn_in=0) as ch:
        for n in (0, 7):
            ch.run(n)
            x = ch.sample()
            e, pair, data = ch.energy()
            opair, odata = oen.energy_terms(m, g, x)
            assert (pair, data) == (opair, odata)
            assert e == pytest.approx(oen.posterior_energy(m, g, x), rel=1e-12, abs=1e-9)


@pytest.mark.parametrize("sampler", [0, 1])
@pytest.mark.parametrize("name,make", CASES[:3], ids=[c[0] for c in CASES[:3]])
def test_tracking_follows_oracle_chain(pc, name, make, sampler):
    g, m = make()
    m = Model(**{**m.as_dict(), "sampler": sampler})
    n = 45   # one 32-sweep graph block and a remainder
    with pc.Chain(g, m, seed=6, chain_id=3, burn_in=0) as ch:
        ch.track_energy(64)
        ch.run(20)
        ch.run(n - 20)
        trace = ch.energies()
        xmin, emin, smin = ch.min_state()
    assert trace.shape == (n,)
    x = g.copy()
    ref = []
    states = []
    for t in range(n):
        x, _, _, _ = oracle.run_chain(m, g, 1, 0, seed=6, chain=3, sampler=sampler, x0=x, t0=t)
        ref.append(oen.posterior_energy(m, g, x))
        states.append(x.copy())
    np.testing.assert_allclose(trace, ref, rtol=1e-12, atol=1e-9)
    k = int(np.argmin(trace))   # first occurrence of the minimum
    assert smin == k + 1
    assert emin == trace[k]
    assert np.array_equal(xmin, states[k])


def test_tracking_capacity_reset_and_blocking(pc):
    g, m = CASES[0][1]()
    with pc.Chain(g, m, seed=1) as ch:
        ch.track_energy(5)
        ch.run(9)
        assert ch.energies().shape == (5,)
        ch.reset()
        with pytest.raises(pc.PcadError):
            ch.min_state()                    # nothing tracked since the reset
        ch.run(3)
        assert ch.energies().shape == (3,)
        with pytest.raises(pc.PcadError):
            ch.set_blocking(2)
        ch.track_energy(0)
        with pytest.raises(pc.PcadError):
            ch.energies()
        ch.set_blocking(2)
        with pytest.raises(pc.PcadError):
            ch.track_energy(4)
