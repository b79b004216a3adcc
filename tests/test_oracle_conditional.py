"""Pins for the oracle's per-site conditional and draw against quantities the
paper and the mathematics fix independently of it:

* the Gibbs conditional equals the ratio of joint posterior weights
  (Eq. gibbs_sampler_elementary_step vs Eq. mrf_gauss_noise_posterior_distribution);
* the lazy-PCA transition built from per-site conditionals equals
  exp(-H~(x,w)) / Z_x from the symmetric lifted pair Hamiltonian
  (Eq. double_hamiltonian_pca_general_form, Section 5.2);
* detailed balance and stationarity of pi~ = Z_x / Z (Eq. pca_detailed_balance);
* the J = 0 closed form and its large-inertia limit;
* the inverse-CDF draw against the exact probabilities on a grid of u.
CPU only."""
import numpy as np
import pytest

from oracle import exact
from pcad_inputs import Model, random_lattice

POTTS, TL, GAUSS, FLIP = 0, 1, 0, 1


def _models():
    return [
        ("potts_flip_2x3", Model(L=2, nbhd=4, pair=POTTS, pair_coef=1.2, noise=FLIP,
                                 flip_p=0.1, inertia=0.7), (2, 3)),
        ("tl_gauss_L3_2x2", Model(L=3, nbhd=4, pair=TL, pair_coef=0.8, pair_T=1,
                                  noise=GAUSS, sigma=0.9, inertia=0.5), (2, 2)),
        ("tl_gauss_L4_T2_1x3", Model(L=4, nbhd=4, pair=TL, pair_coef=0.6, pair_T=2,
                                     noise=GAUSS, sigma=1.3, inertia=1.1), (1, 3)),
        ("potts8_gauss_3x3", Model(L=2, nbhd=8, pair=POTTS, pair_coef=0.9, noise=GAUSS,
                                   sigma=0.8, inertia=0.9), (3, 3)),
        ("potts_gauss_L3_2x2_8", Model(L=3, nbhd=8, pair=POTTS, pair_coef=0.7,
                                       noise=GAUSS, sigma=1.0, inertia=0.4), (2, 2)),
        # L1 / L2 inertia norms on intensities (Section 3)
        ("tl_gauss_L4_T2_1x3_l1", Model(L=4, nbhd=4, pair=TL, pair_coef=0.6, pair_T=2,
                                        noise=GAUSS, sigma=1.3, inertia=1.7, inertia_norm=1),
         (1, 3)),
        ("tl_gauss_L3_2x2_l2", Model(L=3, nbhd=4, pair=TL, pair_coef=0.8, pair_T=1,
                                     noise=GAUSS, sigma=0.9, inertia=2.5, inertia_norm=2), (2, 2)),
        ("potts_gauss_L5_1x3_l2_8", Model(L=5, nbhd=8, pair=POTTS, pair_coef=0.7, noise=GAUSS,
                                          sigma=1.1, inertia=3.0, inertia_norm=2), (1, 3)),
    ]


@pytest.mark.parametrize("name,m,shape", _models(), ids=[x[0] for x in _models()])
def test_gibbs_conditional_is_joint_ratio(orc, name, m, shape):
    H, W = shape
    g = random_lattice(11, H, W, m.L)
    X = exact.states(H * W, m.L)
    logw = exact.posterior_logweights(m, g)
    nb = exact.neighbours(H, W, m.nbhd)
    rng = np.random.default_rng(5)
    strides = m.L ** np.arange(H * W)
    for _ in range(20):
        a = int(rng.integers(0, X.shape[0]))
        x = X[a]
        for i in range(H * W):
            idx = [a + (s - x[i]) * strides[i] for s in range(m.L)]
            lw = logw[idx]
            p_joint = np.exp(lw - lw.max())
            p_joint /= p_joint.sum()
            p_orc = orc.site_probs(m, g.reshape(-1)[i], x[i], [x[j] for j in nb[i]], 0.0)
            np.testing.assert_allclose(p_orc, p_joint, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("name,m,shape", _models()[:3] + _models()[4:],
                         ids=[x[0] for x in _models()[:3] + _models()[4:]])
def test_pca_transition_matches_pair_hamiltonian(orc, name, m, shape):
    H, W = shape
    g = random_lattice(12, H, W, m.L)
    P_cond = exact.pca_transition_from_conditionals(m, g)
    P_pair = exact.pca_transition_from_pair(m, g)
    np.testing.assert_allclose(P_cond, P_pair, rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(P_cond.sum(axis=1), 1.0, rtol=1e-12)


@pytest.mark.parametrize("name,m,shape", _models()[:3] + _models()[4:],
                         ids=[x[0] for x in _models()[:3] + _models()[4:]])
def test_pca_detailed_balance_and_stationarity(orc, name, m, shape):
    H, W = shape
    g = random_lattice(13, H, W, m.L)
    P = exact.pca_transition_from_conditionals(m, g)
    pi = exact.normalise_log(exact.pca_stationary_logweights(m, g))
    flow = pi[:, None] * P
    np.testing.assert_allclose(flow, flow.T, rtol=1e-9, atol=1e-15)
    np.testing.assert_allclose(pi @ P, pi, rtol=1e-9, atol=1e-15)


def test_pca_stationary_differs_from_posterior(orc):
    """The lazy PCA targets pi~, not pi_post, at finite inertia (Section 3)."""
    m = Model(L=2, nbhd=4, pair=POTTS, pair_coef=1.2, noise=FLIP, flip_p=0.1, inertia=1.0)
    g = random_lattice(14, 3, 3, 2)
    p_pca = exact.normalise_log(exact.pca_stationary_logweights(m, g))
    p_post = exact.normalise_log(exact.posterior_logweights(m, g))
    assert exact.tv(p_pca, p_post) > 0.05


def test_large_inertia_limit_is_doubled_posterior(orc):
    """As lambda -> inf, Z_i(x) -> exp(-E_i(x_i|x)), so pi~ -> pi_post^2
    (the posterior with every energy doubled).  The distance to pi_post^2 must
    shrink monotonically with lambda while the distance to pi_post does not."""
    g = random_lattice(15, 3, 3, 2)
    base = dict(L=2, nbhd=4, pair=POTTS, pair_coef=0.8, noise=FLIP, flip_p=0.15)
    post = exact.posterior_logweights(Model(**base, inertia=0.0), g)
    sq = exact.normalise_log(2.0 * post)
    p1 = exact.normalise_log(post)
    d_sq, d_p = [], []
    for lam in (0.5, 1.0, 2.0, 4.0, 8.0, 16.0):
        p = exact.normalise_log(exact.pca_stationary_logweights(Model(**base, inertia=lam), g))
        d_sq.append(exact.tv(p, sq))
        d_p.append(exact.tv(p, p1))
    assert all(b < a for a, b in zip(d_sq, d_sq[1:]))
    assert d_sq[-1] < 1e-4
    assert d_p[-1] > 0.05


@pytest.mark.parametrize("L,sigma,lam", [(2, 0.6, 0.5), (16, 2.0, 1.0), (256, 20.0, 2.0)])
def test_j0_closed_form_matches_single_site_chain(orc, L, sigma, lam):
    m = Model(L=L, nbhd=4, pair=TL, pair_coef=0.0, pair_T=1, noise=GAUSS, sigma=sigma,
              inertia=lam)
    for gi in (0, L // 3, L - 1):
        cf = exact.j0_pca_marginal(m, gi)
        ev = exact.single_site_chain_stationary(m, gi)
        np.testing.assert_allclose(cf, ev, rtol=1e-8, atol=1e-14)


@pytest.mark.parametrize("L,sigma,lam,norm", [(16, 2.0, 1.5, 1), (16, 2.0, 3.0, 2),
                                               (256, 20.0, 2.0, 1), (5, 0.7, 4.0, 2)])
def test_j0_closed_form_matches_single_site_chain_norms(orc, L, sigma, lam, norm):
    m = Model(L=L, nbhd=4, pair=TL, pair_coef=0.0, pair_T=1, noise=GAUSS, sigma=sigma,
              inertia=lam, inertia_norm=norm)
    for gi in (0, L // 3, L - 1):
        cf = exact.j0_pca_marginal(m, gi)
        ev = exact.single_site_chain_stationary(m, gi)
        np.testing.assert_allclose(cf, ev, rtol=1e-8, atol=1e-14)


@pytest.mark.parametrize("norm,E", [(1, (3.0, 1.5, 3.0)), (2, (3.0, 1.0, 3.0))])
def test_hand_worked_norm_conditional(orc, norm, E):
    """L = 3, truncated linear c = 0.5, T = 1, Gaussian sigma = 1, lambda = 2,
    g = 2, x_i = 0, two neighbours at label 1:
      s = 0: prior 0.5 (1 + 1) = 1, data (2-0)^2/2 = 2, inertia 0
      s = 1: prior 0, data 1/2, inertia 2 (1/2)^p = 1 (p = 1) or 1/2 (p = 2)
      s = 2: prior 1, data 0, inertia 2 (2/2)^p = 2."""
    m = Model(L=3, nbhd=4, pair=TL, pair_coef=0.5, pair_T=1, noise=GAUSS, sigma=1.0,
              inertia=2.0, inertia_norm=norm)
    p = orc.site_probs(m, 2, 0, [1, 1], 2.0)
    w = np.exp(-np.array(E))
    np.testing.assert_allclose(p, w / w.sum(), rtol=1e-13)


def test_j0_conditional_is_data_term_only(orc):
    m = Model(L=16, nbhd=4, pair=TL, pair_coef=0.0, pair_T=3, noise=GAUSS, sigma=2.5,
              inertia=0.0)
    p = orc.site_probs(m, 5, 9, [1, 2, 14, 15], 0.0)
    np.testing.assert_allclose(p, exact.j0_gibbs_marginal(m, 5), rtol=1e-12)


def test_potts_equals_truncated_linear_with_T1(orc):
    """c_P 1{s=t} reward == c_P min(|s-t|,1) cost up to a constant: the two
    priors give the same conditional."""
    mp = Model(L=9, nbhd=8, pair=POTTS, pair_coef=0.9, noise=GAUSS, sigma=1.5, inertia=0.3)
    mt = Model(L=9, nbhd=8, pair=TL, pair_coef=0.9, pair_T=1, noise=GAUSS, sigma=1.5,
               inertia=0.3)
    rng = np.random.default_rng(3)
    for _ in range(50):
        nbrs = list(rng.integers(0, 9, size=int(rng.integers(3, 9))))
        g, xi = int(rng.integers(0, 9)), int(rng.integers(0, 9))
        np.testing.assert_allclose(orc.site_probs(mp, g, xi, nbrs, 0.3),
                                   orc.site_probs(mt, g, xi, nbrs, 0.3), rtol=1e-12)


def test_hand_worked_binary_conditional(orc):
    """Ising site, two neighbours equal to label 1, observed g = 0 under flip
    noise p = 0.25, c_P = 1, lambda = 0.5, previous label x_i = 0:
      E(0) = -ln(0.75)               + 0
      E(1) = -2 - ln(0.25)           + 0.5
      p(1) = 1 / (1 + exp(E(1) - E(0))),
      E(1) - E(0) = -2 + 0.5 - ln(0.25) + ln(0.75) = -1.5 + ln 3."""
    m = Model(L=2, nbhd=4, pair=POTTS, pair_coef=1.0, noise=FLIP, flip_p=0.25, inertia=0.5)
    p = orc.site_probs(m, 0, 0, [1, 1], 0.5)
    d = -1.5 + np.log(3.0)
    assert abs(p[1] - 1.0 / (1.0 + np.exp(d))) < 1e-14


def test_draw_inverse_cdf_on_grid(orc):
    m = Model(L=7, nbhd=4, pair=TL, pair_coef=0.4, pair_T=2, noise=GAUSS, sigma=1.7,
              inertia=0.8)
    nbrs, g, xi = [1, 3, 6], 2, 5
    p = orc.site_probs(m, g, xi, nbrs, 0.8)
    F = np.cumsum(p)
    N = 4096
    counts = np.zeros(m.L)
    for k in range(N):
        lab, _ = orc.site_draw(m, g, xi, nbrs, 0.8, (k + 0.5) / N)
        counts[lab] += 1
    np.testing.assert_allclose(counts / N, p, atol=1.5 / N)
    # direction and strictness at each boundary
    for k in range(m.L - 1):
        lo, _ = orc.site_draw(m, g, xi, nbrs, 0.8, F[k] - 1e-9)
        hi, near = orc.site_draw(m, g, xi, nbrs, 0.8, F[k] + 1e-9)
        assert lo == k and hi == k + 1 and near


def test_zero_weight_labels_never_drawn(orc):
    """A label whose weight underflows to 0 in FP64 is never chosen."""
    m = Model(L=256, nbhd=4, pair=TL, pair_coef=0.0, pair_T=1, noise=GAUSS, sigma=0.5,
              inertia=0.0)
    for u in (0.0, 0.5, 1.0 - 2 ** -24):
        lab, _ = orc.site_draw(m, 0, 0, [], 0.0, u)
        assert lab in (0, 1, 2)
