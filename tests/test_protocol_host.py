"""Host-side pieces of the paper protocol and the prior-only model:

* the oracle's conditional without likelihood is the Potts prior's
  conditional, exp(c_P n(s)) normalised (closed form), and its joint is the
  prior, exp(c_P * equal pairs) (exhaustive enumeration against the energy);
* the annealing schedule, the q grid and the concavity count of the
  protocol module (no GPU needed: no library call is made)."""
import numpy as np
import pytest

from oracle import energy, exact
from pcad_inputs import Model, random_lattice

POTTS, TL, NONE = 0, 1, 2


def test_prior_only_conditional_closed_form(orc):
    m = Model(L=4, nbhd=8, pair=POTTS, pair_coef=0.9, noise=NONE, inertia=0.0)
    nbrs = [0, 2, 2, 3, 2, 1, 0, 2]
    for g in (0, 3):   # the observation plays no part
        p = np.asarray(orc.site_probs(m, g, 1, nbrs, 0.0))
        n = np.array([sum(1 for x in nbrs if x == s) for s in range(4)])
        ref = np.exp(np.float32(0.9).item() * n)   # parameters arrive as FP32
        np.testing.assert_allclose(p, ref / ref.sum(), rtol=1e-12)


def test_prior_only_joint_is_potts_prior():
    m = Model(L=3, nbhd=4, pair=POTTS, pair_coef=0.8, noise=NONE)
    g = random_lattice(5, 2, 3, 3)
    logw = exact.posterior_logweights(m, g)
    X = exact.states(6, 3)
    for k in range(X.shape[0]):
        x = X[k].reshape(2, 3).astype(np.uint8)
        pair, data = energy.energy_terms(m, g, x)
        assert data == 0
        assert -logw[k] == pytest.approx(-np.float32(0.8).item() * pair, abs=1e-12)


def test_protocol_schedule_and_grid():
    from paper_2507_14869_gb300 import protocol as pr
    assert pr.betas() == [1.25, 1.5, 1.75, 2.0]
    assert len(pr.Q_GRID) == 14 and pr.Q_GRID[0] == 0.06 and pr.Q_GRID[-1] == 0.71
    ms, sw = pr.schedule(L=9, J=1 / 3, q=0.46, sigma=0.2)
    assert sw == [250] * 4 and sum(sw) == 1000
    for b, m in zip(pr.betas(), ms):
        assert m["pair_coef"] == pytest.approx(2 * b / 3)
        assert m["inertia"] == pytest.approx(b * 0.46)
        assert m["sigma"] == pytest.approx(0.2 * 8)   # intensity units -> label units
        assert m["nbhd"] == 8 and m["pair"] == POTTS
    c = pr.concavity([1.0, 2.0, 2.5, 2.6, 2.4])
    assert c == dict(positive=0, max=pytest.approx(-0.3), n=3)
    assert pr.concavity([1.0, 0.0, 1.0])["positive"] == 1
