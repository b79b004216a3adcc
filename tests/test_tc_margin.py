"""The certified margins of the FP32 draw, checked by brute force on the CPU:
the per-site margin (tensor-core sweep, and CUDA-core sweeps with a
non-negative prior coefficient) and the constant margin the CUDA-core sweeps
keep for a negative one.

For random sites of several models, the FP32 arithmetic of the window
weights (2^(alpha (g-s)^2 + mu Pb + cb) with two roundings, ex2 off by up to
2 ulp in the direction that hurts most), the chunk sums, the Kahan prefix and
the inertia correction is replayed in numpy and every CDF value C_k / Z is
compared with the exact conditional CDF of Eq. posterior_pca_transition_matrix
(§5.2; FP64).  The library's per-site margin (pcad_model_margins: eta =
kb1 (hb - log2 Z) + kb0 + kbr delta / Z, of which two thirds are the bound and
one third slack) must exceed the worst error plus the rounding of t = u Z at
every site.  CPU only: the coefficients come from the host side of the
library, no kernel runs."""
import numpy as np
import pytest

U = 2.0 ** -24
LOG2E = 1.4426950408889634074
f32, f64 = np.float32, np.float64


@pytest.fixture(scope="module")
def pc():
    import paper_2507_14869_gb300 as pc
    pc.lib()
    return pc


def _fma32(a, b, c):
    # exact in FP64 for these magnitudes (24-bit x 24-bit products, integer
    # q and Pb), then one rounding: the FP32 fused multiply-add
    return (np.asarray(a, f64) * np.asarray(b, f64) + np.asarray(c, f64)).astype(f32)


def _sites(rng, n, L, nbhd, spread):
    x = np.where(rng.random((n, 1)) < 0.5,
                 rng.integers(0, L, (n, nbhd)),
                 np.clip(rng.integers(0, L, (n, 1)) + rng.integers(-spread, spread + 1, (n, nbhd)),
                         0, L - 1))
    present = rng.random((n, nbhd)) < 0.9            # missing neighbours: image border
    present[:, 0] = True
    g = np.where(rng.random(n) < 0.7, np.clip(x[:, 0] + rng.integers(-40, 41, n), 0, L - 1),
                 rng.integers(0, L, n))
    xi = np.where(rng.random(n) < 0.6, x[:, 0], rng.integers(0, L, n))
    return x, present, g, xi


def _worst_error(mg, model, x, present, g, xi, sign_split, form="tc"):
    """Max over k of |C_k / Z - F_k| with the FP32 replay and the site's
    margin.  form "tc": the tensor-core weights 2^fl(alpha q + fl(mu Pb + cb))
    (Pb the tent sum of the present neighbours); "cc": the CUDA-core weights
    2^fl(alpha q + fl(gam P)) (P = sum of min(|x_j - s|, T), T for a missing
    neighbour)."""
    L, T, nbhd = model["L"], model["T"], model["nbhd"]
    s = np.arange(L)
    Pb = (np.maximum(T - np.abs(s[None, None, :] - x[:, :, None]), 0) * present[:, :, None]).sum(1)
    q = (g[:, None] - s[None, :]) ** 2
    alpha, gam, cb = f32(mg["alpha"]), f32(mg["gam"]), f32(mg["cb"])
    mu = -gam
    if form == "tc":
        v = _fma32(alpha, q, _fma32(mu, Pb, cb))
    else:
        # "cc": a missing neighbour contributes T; "small" (the small-label
        # kernel's pair table): it contributes nothing
        P = (np.where(present[:, :, None], np.minimum(np.abs(s[None, None, :] - x[:, :, None]), T),
                      T if form == "cc" else 0)).sum(1)
        if form == "small_aq":   # the data term from a table: fl(gam P + fl(alpha q))
            v = _fma32(gam, P, (f64(alpha) * q).astype(f32))
        else:
            v = _fma32(alpha, q, (f64(gam) * P).astype(f32))
    # ex2 within 2 ulp: correctly rounded, moved by 2u up for labels <= the
    # split and down above it, rounded again
    w = np.exp2(v.astype(f64)).astype(f32)
    up = s[None, :] <= sign_split[:, None]
    w = (w.astype(f64) * np.where(up, 1.0 + 2 * U, 1.0 - 2 * U)).astype(f32)
    w = np.where(v < -126.0, f32(0.0), w)
    n = len(g)
    nc = (L + 7) // 8
    wp = np.zeros((n, nc * 8), f32)
    wp[:, :L] = w
    # chunk sums (sequential), Kahan prefix over chunks, in-chunk prefixes
    pref = np.zeros((n, nc * 8), f32)
    S = np.zeros(n, f32)
    for k in range(nc * 8):
        S = S + wp[:, k] if k % 8 else wp[:, k].copy()
        pref[:, k] = S
    chunk = pref[:, 7::8]
    if form == "tc":   # window chunk sums: a pairwise tree ((w0+w1)+(w2+w3))+((w4+w5)+(w6+w7))
        w8 = wp.reshape(n, nc, 8)
        pairs = w8[:, :, 0::2] + w8[:, :, 1::2]
        chunk = (pairs[:, :, 0] + pairs[:, :, 1]) + (pairs[:, :, 2] + pairs[:, :, 3])
    G = np.zeros(n, f32)
    comp = np.zeros(n, f32)
    Gc = np.zeros((n, nc), f32)
    for c in range(nc):
        y = chunk[:, c] - comp
        tt = G + y
        comp = (tt - G) - y
        G = tt
        Gc[:, c] = G
    if form.startswith("small"):
        # chunks of 4 labels: in-chunk sequential prefix, sequential chunk
        # prefix, no compensation
        nc = (L + 3) // 4
        wp = np.zeros((n, nc * 4), f32)
        wp[:, :L] = w
        pref = np.zeros((n, nc * 4), f32)
        for k in range(nc * 4):
            pref[:, k] = pref[:, k - 1] + wp[:, k] if k % 4 else wp[:, k]
        Gc = np.zeros((n, nc), f32)
        for c in range(nc):
            Gc[:, c] = pref[:, 4 * c + 3] if c == 0 else Gc[:, c - 1] + pref[:, 4 * c + 3]
        G = Gc[:, -1].copy()
    # the model's parameters as the library receives them (FP32 fields)
    lam = float(f32(model["inertia"]))
    c_e, sig_e = float(f32(model["pair_coef"])), float(f32(model["sigma"]))
    em1 = f32(np.expm1(lam))
    delta = (w[np.arange(n), xi].astype(f64) * f64(em1)).astype(f32) if lam > 0 else np.zeros(n, f32)
    Z = (G + delta).astype(f32)
    Gprev = np.concatenate([np.zeros((n, 1), f32), Gc[:, :-1]], axis=1)
    if form.startswith("small"):
        # the small-label kernel joins the in-chunk prefix to Gprev or to
        # fl(Gprev + delta) (at and above x_i)
        Gp = np.repeat(Gprev, 4, axis=1)[:, :L]
        Gpd = (Gp + delta[:, None]).astype(f32)
        C = (np.where(s[None, :] >= xi[:, None], Gpd, Gp) + pref[:, :L]).astype(f32)
    else:
        C = (np.repeat(Gprev, 8, axis=1)[:, :L] + pref[:, :L]).astype(f32)
        C = (C + np.where(s[None, :] >= xi[:, None], delta[:, None], f32(0.0))).astype(f32)
    # exact conditional
    mu_e = c_e * LOG2E
    alpha_e = -LOG2E / (2.0 * sig_e ** 2) if model["noise"] == 0 else 0.0
    # every label's prior sum, a missing neighbour contributing T (a constant)
    P_all = np.where(present[:, :, None], np.minimum(np.abs(s[None, None, :] - x[:, :, None]), T),
                     T).sum(1)
    W = np.exp2(alpha_e * q - mu_e * P_all - np.max(alpha_e * q - mu_e * P_all, axis=1,
                                                       keepdims=True))
    dW = np.expm1(lam) * W[np.arange(n), xi]
    Fk = (np.cumsum(W, axis=1) + np.where(s[None, :] >= xi[:, None], dW[:, None], 0.0)) / \
         (W.sum(1) + dW)[:, None]
    err = np.abs(C.astype(f64) / Z.astype(f64)[:, None] - Fk).max(1)
    if form == "cc" and mg["gam"] > 0:   # c < 0 on the CUDA cores: the constant margin
        eta = np.full(n, mg["eta"])
    else:
        eta = mg["kb1"] * (mg["hb"] - np.log2(Z.astype(f64))) + mg["kb0"] + \
            mg["kbr"] * delta.astype(f64) / Z.astype(f64)
    return err, eta, Fk


MODELS = [
    dict(L=256, nbhd=4, pair=1, pair_coef=0.05, pair_T=30, noise=0, sigma=20.0, inertia=2.0),
    dict(L=256, nbhd=8, pair=1, pair_coef=0.15, pair_T=33, noise=0, sigma=25.0, inertia=1.0),
    dict(L=100, nbhd=4, pair=1, pair_coef=0.5, pair_T=10, noise=0, sigma=4.0, inertia=0.3),
    dict(L=64, nbhd=4, pair=1, pair_coef=4.9, pair_T=2, noise=0, sigma=2.0, inertia=5.0),
    dict(L=128, nbhd=8, pair=0, pair_coef=4.5, pair_T=1, noise=0, sigma=6.0, inertia=0.0),
    dict(L=256, nbhd=4, pair=1, pair_coef=-0.08, pair_T=30, noise=0, sigma=30.0, inertia=1.5),
    dict(L=200, nbhd=4, pair=1, pair_coef=0.3, pair_T=20, noise=2, sigma=1.0, inertia=2.5),
    dict(L=256, nbhd=8, pair=1, pair_coef=0.02, pair_T=25, noise=0, sigma=200.0, inertia=0.05),
]


CASES = [(i, "tc") for i in range(len(MODELS))] + [(i, "cc") for i in range(len(MODELS))]


@pytest.mark.parametrize("i,form", CASES, ids=[f"{f}{i}" for i, f in CASES])
def test_margin_covers_worst_fp32_error(pc, i, form):
    model = dict(MODELS[i])
    model["T"] = 1 if model["pair"] == 0 else model["pair_T"]
    mg = pc.pcad_model_margins(dict(model, flip_p=0.1, sampler=0))
    assert mg["alpha"] == pytest.approx(-LOG2E / (2 * model["sigma"] ** 2) if model["noise"] == 0
                                        else 0.0, rel=1e-6)
    rng = np.random.default_rng(100 + i)
    x, present, g, xi = _sites(rng, 600, model["L"], model["nbhd"], spread=6)
    worst = 0.0
    for split_kind in range(3):
        if split_kind == 0:
            split = np.full(len(g), -1)                # every weight low
        elif split_kind == 1:
            split = np.full(len(g), model["L"])        # every weight high
        else:                                          # around each site's median
            _, _, Fk = _worst_error(mg, model, x, present, g, xi, np.full(len(g), -1), form)
            split = (Fk < 0.5).sum(1)
        err, eta, _ = _worst_error(mg, model, x, present, g, xi, split, form)
        bound = eta / 1.5 - U                          # without the slack, less t's rounding
        assert np.all(err <= bound), (float(err.max()), float(bound[np.argmax(err / bound)]))
        worst = max(worst, float((err / bound).max()))
    assert worst < 1.0


SMALL_MODELS = [
    dict(L=16, nbhd=4, pair=1, pair_coef=0.05, pair_T=30, noise=0, sigma=1.0, inertia=2.0),
    dict(L=16, nbhd=8, pair=1, pair_coef=0.6, pair_T=4, noise=0, sigma=4.0, inertia=0.5),
    dict(L=5, nbhd=8, pair=0, pair_coef=0.833, pair_T=1, noise=0, sigma=1.0, inertia=0.7),
    dict(L=9, nbhd=4, pair=1, pair_coef=0.85, pair_T=2, noise=0, sigma=1.6, inertia=0.26),
    dict(L=13, nbhd=4, pair=1, pair_coef=2.4, pair_T=3, noise=0, sigma=0.7, inertia=4.0),
    dict(L=3, nbhd=4, pair=1, pair_coef=0.3, pair_T=1, noise=2, sigma=1.0, inertia=1.0),
    dict(L=16, nbhd=4, pair=1, pair_coef=0.0, pair_T=3, noise=0, sigma=60.0, inertia=0.0),
]


@pytest.mark.parametrize("form", ["small", "small_aq"])
@pytest.mark.parametrize("i", range(len(SMALL_MODELS)))
def test_margin_covers_the_small_label_kernel(pc, i, form):
    """The small-label kernel: the same weight formula with a missing
    neighbour contributing nothing (or, on TMA tiles, the data term from a
    table: fl(gam P + fl(alpha q))), chunks of 4 labels summed without
    compensation -- inside the same per-site margin."""
    model = dict(SMALL_MODELS[i])
    model["T"] = 1 if model["pair"] == 0 else model["pair_T"]
    mg = pc.pcad_model_margins(dict(model, flip_p=0.1, sampler=0))
    assert mg["gam"] <= 0
    rng = np.random.default_rng(300 + i)
    x, present, g, xi = _sites(rng, 1500, model["L"], model["nbhd"], spread=3)
    worst = 0.0
    for split_kind in range(3):
        if split_kind == 0:
            split = np.full(len(g), -1)
        elif split_kind == 1:
            split = np.full(len(g), model["L"])
        else:
            _, _, Fk = _worst_error(mg, model, x, present, g, xi, np.full(len(g), -1), form)
            split = (Fk < 0.5).sum(1)
        err, eta, _ = _worst_error(mg, model, x, present, g, xi, split, form)
        bound = eta / 1.5 - U
        assert np.all(err <= bound), (float(err.max()), float(bound[np.argmax(err / bound)]))
        worst = max(worst, float((err / bound).max()))
    assert worst < 1.0


def test_margin_is_tighter_than_worst_case_constant(pc):
    """At the bench model the per-site margin of typical sites is a small
    multiple of 2^-24, well below the worst-case constant margin of the
    CUDA-core kernels."""
    model = dict(MODELS[0], T=30)
    mg = pc.pcad_model_margins(dict(model, flip_p=0.1, sampler=0))
    rng = np.random.default_rng(7)
    x, present, g, xi = _sites(rng, 400, 256, 4, spread=4)
    _, eta, _ = _worst_error(mg, model, x, present, g, xi, np.full(len(g), -1))
    assert np.median(eta) < 0.5 * mg["eta"]
    assert mg["cb"] == pytest.approx(-0.05 * LOG2E * 120, rel=1e-6)


def test_model_margins_rejects_bad_arguments(pc):
    import ctypes
    good = dict(MODELS[0], flip_p=0.1, sampler=0)
    m = pc.as_model(good)
    out = (ctypes.c_double * 4)()
    assert pc.lib().pcad_model_margins(ctypes.byref(m), out, 4) == 1     # n < PCAD_N_MARGINS
    with pytest.raises(pc.PcadError):
        pc.pcad_model_margins(dict(good, pair_coef=1.0))                 # prior range > 40
    with pytest.raises(pc.PcadError):
        pc.pcad_model_margins(dict(good, sigma=-1.0))
    mg = pc.pcad_model_margins(dict(good, pair_coef=-0.05))
    assert mg["cb"] == 0.0 and mg["gam"] > 0                             # c < 0: no offset
