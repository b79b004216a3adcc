"""The small-label draw's selection logic, replayed in FP32 on the CPU and
checked against the FP64 oracle draw.

The small-label kernel finds the chunk of 4 labels by comparing the chunk
ends with t or t - delta (delta the inertia correction, added at and above
x_i), joins the chosen chunk's prefix sums to Gp or fl(Gp + delta), and
certifies the label only when t lies more than the per-site margin inside
its CDF interval.  This test replays those FP32 operations in numpy (both
exponent forms: fl(alpha q + fl(gam P)) and, from the data-term table,
fl(gam P + fl(alpha q))), with uniforms placed on and around every CDF
boundary, and asserts that every draw the replay calls certain picks the
label of the oracle's FP64 inverse-CDF draw (`orc_site_draw`, Eq.
posterior_pca_transition_matrix), and that most draws are certain."""
import numpy as np
import pytest

f32, f64 = np.float32, np.float64


@pytest.fixture(scope="module")
def pc():
    import paper_2507_14869_gb300 as pc
    pc.lib()
    return pc


def _fma32(a, b, c):
    return (np.asarray(a, f64) * np.asarray(b, f64) + np.asarray(c, f64)).astype(f32)


def replay(mg, model, g, xi, nbrs, ub, aq_form):
    """The FP32 draw of one site for uniform numerators ub (array); returns
    (labels, certain)."""
    L, T = model["L"], model["T"]
    s = np.arange(16)
    P = np.zeros(16, np.int64)
    for x in nbrs:
        P += np.minimum(np.abs(s - x), T)
    q = (g - s) ** 2
    alpha, gam = f32(mg["alpha"]), f32(mg["gam"])
    if aq_form:
        v = _fma32(gam, P, (f64(alpha) * q).astype(f32))
    else:
        v = _fma32(alpha, q, (f64(gam) * P).astype(f32))
    w = np.exp2(v.astype(f64)).astype(f32)
    w[s >= L] = f32(0.0)
    G = np.zeros(4, f32)
    for c in range(4):
        p3 = f32(f32(f32(w[4 * c] + w[4 * c + 1]) + w[4 * c + 2]) + w[4 * c + 3])
        G[c] = p3 if c == 0 else f32(G[c - 1] + p3)
    em1 = f32(np.expm1(f64(f32(model["inertia"]))))
    delta = f32(w[xi] * em1) if model["inertia"] > 0 else f32(0.0)
    Z = f32(G[3] + delta)
    lgZ = f32(np.log2(f64(Z)))
    eta = f32(_fma32(mg["kb1"], f32(f32(mg["hb"]) - lgZ), mg["kb0"]) +
              f32(f32(mg["kbr"]) * f32(delta / Z)))
    margin = f32(eta * Z)
    labels, certain = [], []
    for u in ub:
        t = f32(f32(f32(u) * f32(1.0 / 16777216.0)) * Z)
        tmd = f32(t - delta)
        cs, Gp = 0, f32(0.0)
        for c in range(3):
            if G[c] <= (tmd if 4 * c + 3 >= xi else t):
                cs += 1
                Gp = G[c]
        base = 4 * cs
        wc = w[base:base + 4]
        p = [wc[0]]
        p.append(f32(wc[0] + wc[1]))
        p.append(f32(p[1] + wc[2]))
        p.append(f32(p[2] + wc[3]))
        Gpd = f32(Gp + delta)
        C = [f32((Gpd if base + k >= xi else Gp) + p[k]) for k in range(4)]
        b = [C[0] <= t, C[1] <= t, C[2] <= t]
        k = int(b[0]) + int(b[1]) + int(b[2])
        hiC = C[k]
        Cm = Gpd if base - 1 >= xi else Gp
        loC = C[k - 1] if k > 0 else Cm
        sl = base + k
        ok = (t < hiC) and (sl < L) and (sl == L - 1 or f32(hiC - t) > margin) and \
             (sl == 0 or f32(t - loC) > margin)
        labels.append(min(sl, L - 1))
        certain.append(bool(ok))
    return np.array(labels), np.array(certain)


MODELS = [
    dict(L=16, nbhd=4, pair=1, pair_coef=0.05, pair_T=30, noise=0, sigma=1.0, inertia=2.0),
    dict(L=16, nbhd=4, pair=1, pair_coef=0.85, pair_T=2, noise=0, sigma=2.0, inertia=1.0),
    dict(L=13, nbhd=8, pair=1, pair_coef=0.4, pair_T=3, noise=0, sigma=1.5, inertia=0.7),
    dict(L=16, nbhd=4, pair=1, pair_coef=0.3, pair_T=6, noise=0, sigma=3.0, inertia=0.0),
    dict(L=5, nbhd=8, pair=0, pair_coef=0.833, pair_T=1, noise=0, sigma=1.0, inertia=0.7),
]


@pytest.mark.parametrize("aq_form", [False, True])
@pytest.mark.parametrize("i", range(len(MODELS)))
def test_certified_small_draws_pick_the_fp64_label(pc, orc, i, aq_form):
    model = dict(MODELS[i])
    model["T"] = 1 if model["pair"] == 0 else model["pair_T"]
    mg = pc.pcad_model_margins(dict(model, flip_p=0.1, sampler=0))
    om = dict(model, flip_p=0.1, sampler=0)
    L, nbhd = model["L"], model["nbhd"]
    rng = np.random.default_rng(500 + i)
    n_rand = n_rand_certain = n_near_certain = 0
    for _ in range(60):
        g = int(rng.integers(0, L))
        xi = int(rng.integers(0, L))
        nn = int(rng.integers(1, nbhd + 1))   # present neighbours (the rest outside)
        nbrs = [int(v) for v in np.clip(xi + rng.integers(-3, 4, nn), 0, L - 1)]
        probs = orc.site_probs(om, g, xi, nbrs, model["inertia"])
        cdf = np.cumsum(probs)
        nr = 32
        ub = list(rng.integers(0, 1 << 24, nr))
        for c in cdf[:-1]:   # on and around every boundary, inside and outside the margin
            centre = int(c * (1 << 24))
            ub += [min(max(centre + d, 0), (1 << 24) - 1)
                   for d in (-3, -1, 0, 1, 2, 40, -40, 400, -400, 4000, -4000)]
        labels, certain = replay(mg, model, g, xi, nbrs, ub, aq_form)
        for u, lab, ok in zip(ub, labels, certain):
            want, _ = orc.site_draw(om, g, xi, nbrs, model["inertia"], u / float(1 << 24))
            if ok:
                assert lab == want, (g, xi, nbrs, u)
        n_rand += nr
        n_rand_certain += int(certain[:nr].sum())
        n_near_certain += int(certain[nr:].sum())
    assert n_rand_certain > 0.99 * n_rand   # random uniforms: almost all certain
    assert n_near_certain > 0               # the boundary sample reaches certain draws too
