"""Pins for the oracle's samplers as Markov chains: empirical state laws
against exact enumeration, J = 0 closed forms, bookkeeping invariants.
CPU only (each long chain is ~1-2 s of C)."""
import numpy as np
import pytest

from oracle import exact
from pcad_inputs import Model, random_lattice

POTTS, TL, GAUSS, FLIP = 0, 1, 0, 1
SWEEPS = 1_000_000


def _structured_binary(H, W, flips=((1, 1),)):
    """A block pattern (left half 0, right half 1) with a few flipped pixels,
    so the posterior concentrates and 1e6 sweeps resolve it to TV < 0.01."""
    g = np.zeros((H, W), dtype=np.uint8)
    g[:, W // 2:] = 1
    for r, c in flips:
        g[r, c] ^= 1
    return g


CASES = [
    # name, model, g, gibbs order
    ("ising_flip_4x4", Model(L=2, nbhd=4, pair=POTTS, pair_coef=1.2, noise=FLIP, flip_p=0.1,
                             inertia=1.0), _structured_binary(4, 4, ((1, 1), (2, 3)))),
    ("ising_flip_3x4", Model(L=2, nbhd=4, pair=POTTS, pair_coef=0.9, noise=FLIP, flip_p=0.15,
                             inertia=0.6), _structured_binary(3, 4, ((0, 3),))),
    ("potts8_gauss_3x3", Model(L=2, nbhd=8, pair=POTTS, pair_coef=0.7, noise=GAUSS, sigma=0.7,
                               inertia=0.8), random_lattice(21, 3, 3, 2)),
    ("tl_L3_2x3", Model(L=3, nbhd=4, pair=TL, pair_coef=0.7, pair_T=1, noise=GAUSS, sigma=0.4,
                        inertia=0.5), random_lattice(22, 2, 3, 3)),
]


@pytest.mark.parametrize("name,m,g", CASES, ids=[c[0] for c in CASES])
def test_pca_chain_law_matches_exact_stationary_measure(orc, name, m, g):
    p_exact = exact.normalise_log(exact.pca_stationary_logweights(m, g))
    assert exact.tv_noise_floor(p_exact, SWEEPS / 4) < 0.008
    h = orc.state_histogram(m, g, SWEEPS, seed=101, sampler=0)
    tv = exact.tv(h / h.sum(), p_exact)
    assert tv < 0.01, tv
    # discriminating: the same chain is far from the posterior
    p_post = exact.normalise_log(exact.posterior_logweights(m, g))
    assert exact.tv(h / h.sum(), p_post) > 3 * tv


@pytest.mark.parametrize("order", [0, 1, 2], ids=["row", "column", "colour"])
@pytest.mark.parametrize("name,m,g", CASES, ids=[c[0] for c in CASES])
def test_gibbs_chain_law_matches_exact_posterior(orc, name, m, g, order):
    p_exact = exact.normalise_log(exact.posterior_logweights(m, g))
    h = orc.state_histogram(m, g, SWEEPS, seed=202 + order, sampler=1, order=order)
    tv = exact.tv(h / h.sum(), p_exact)
    assert tv < 0.01, tv


def _batch_se(samples, nb=50):
    """Standard error of a time average by batch means."""
    n = samples.shape[0] // nb * nb
    b = samples[:n].reshape(nb, -1, *samples.shape[1:]).mean(axis=1)
    return b.std(axis=0, ddof=1) / np.sqrt(nb)


@pytest.mark.parametrize("L,sigma,lam", [(16, 1.5, 1.0), (256, 20.0, 2.0)])
def test_j0_posterior_mean_matches_closed_form(orc, L, sigma, lam):
    """J = 0: sites are independent; PCA per-site law from the closed form,
    Gibbs per-site law exp(-U(s)).  Time averages within 5 standard errors."""
    m = Model(L=L, nbhd=4, pair=TL, pair_coef=0.0, pair_T=1, noise=GAUSS, sigma=sigma,
              inertia=lam)
    g = random_lattice(31, 2, 8, L)
    labels = np.arange(L)
    for sampler, law in ((0, exact.j0_pca_marginal), (1, exact.j0_gibbs_marginal)):
        x = g.copy()
        traj = []
        for t in range(4000):
            if sampler == 0:
                x, _ = orc.pca_sweep(m, g, x, 77, 0, t)
            else:
                x, _ = orc.gibbs_sweep(m, g, x, 77, 0, t)
            traj.append(x.astype(np.float64))
        traj = np.array(traj[200:])
        mean = traj.mean(axis=0)
        se = np.maximum(_batch_se(traj), 1e-3)
        exact_mean = np.array([[float(labels @ law(m, int(gv))) for gv in row] for row in g])
        z = np.abs(mean - exact_mean) / se
        assert z.max() < 5.0, (sampler, z.max())


def test_sweep_uses_previous_state_and_keyed_uniforms(orc):
    """A PCA sweep equals independent per-site draws from the previous state
    with the uniform keyed by (seed, chain, tag 0, sweep, row, col)."""
    m = Model(L=5, nbhd=8, pair=TL, pair_coef=0.5, pair_T=2, noise=GAUSS, sigma=1.2,
              inertia=0.7)
    g = random_lattice(41, 5, 7, 5)
    x = random_lattice(42, 5, 7, 5)
    xn, _ = orc.pca_sweep(m, g, x, 9, 3, 17)
    nb = exact.neighbours(5, 7, 8)
    for i in range(35):
        r, c = divmod(i, 7)
        u = orc.uniform(9, 3, 0, 17, r, c)
        lab, _ = orc.site_draw(m, g.reshape(-1)[i], x.reshape(-1)[i],
                               [x.reshape(-1)[j] for j in nb[i]], 0.7, u)
        assert xn[r, c] == lab


def test_chain_split_and_accumulator(orc):
    """run(300) then run(200) == run(500); the accumulator counts only sweeps
    after burn-in; the initial state is the observation."""
    m = Model(L=16, nbhd=4, pair=TL, pair_coef=0.4, pair_T=3, noise=GAUSS, sigma=2.0,
              inertia=1.0)
    g = random_lattice(51, 9, 13, 16)
    for sampler in (0, 1):
        xa, acca, na, _ = orc.run_chain(m, g, 500, 120, seed=5, sampler=sampler)
        xb, accb, nb_, _ = orc.run_chain(m, g, 300, 120, seed=5, sampler=sampler)
        xb, accb, nb2, _ = orc.run_chain(m, g, 200, 120, seed=5, sampler=sampler, x0=xb,
                                         acc=accb, t0=300)
        assert np.array_equal(xa, xb)
        assert np.array_equal(acca, accb)
        assert na == 380 and nb_ + nb2 == 380
        x0, acc0, n0, _ = orc.run_chain(m, g, 0, 0, seed=5, sampler=sampler)
        assert np.array_equal(x0, g) and n0 == 0


def test_gibbs_orders_agree_on_colour_independent_sites(orc):
    """In colour order the last colour's draws see the others' fresh labels:
    a checkerboard sweep equals row-major order restricted to two phases."""
    m = Model(L=3, nbhd=4, pair=TL, pair_coef=0.6, pair_T=1, noise=GAUSS, sigma=1.0)
    g = random_lattice(61, 6, 5, 3)
    x = random_lattice(62, 6, 5, 3)
    xc, _ = orc.gibbs_sweep(m, g, x, 1, 0, 0, order=2)
    # replay by hand: colour 0 then colour 1, each from the state after the previous phase
    y = x.copy()
    nb = exact.neighbours(6, 5, 4)
    for q in (0, 1):
        for i in range(30):
            r, c = divmod(i, 5)
            if (r + c) % 2 != q:
                continue
            u = orc.uniform(1, 0, 1, 0, r, c)
            lab, _ = orc.site_draw(m, g[r, c], y[r, c], [y.reshape(-1)[j] for j in nb[i]],
                                   0.0, u)
            y[r, c] = lab
    assert np.array_equal(xc, y)
