"""Exhaustive enumeration on tiny lattices -- TEST INFRASTRUCTURE.

Written from the joint (global) formulas of the paper, independently of the
per-site conditional in ``pcad_oracle.c``:

  * posterior Gibbs measure, Eq. (mrf_gauss_noise_posterior_distribution):
    pi_post(x) ~ exp{-[ sum_{unordered edges <ij>} V(x_i, x_j) + sum_i U_i(x_i) ]}
    where V(s,t) = -c_P 1{s=t} (Potts, c_P = 2 beta J: the per-edge weight that
    makes its single-site conditional the one of Eq.
    gibbs_sampler_elementary_step) or c_T min(|s-t|, T);
  * the lazy-PCA pair Hamiltonian, symmetric lift of Section 5.2 with the
    L0 inertia of Section 3:
    H~(x,w) = sum_i sum_{j in N(i)} V(w_i, x_j) + sum_i [U_i(w_i) + U_i(x_i)]
              + lambda sum_i rho(w_i, x_i),
    with the inertia price rho = 1{w != x} (L0) or (|w - x| / (L - 1))^p for
    the L1 / L2 norms on intensities (Section 3),
    its transition matrix P(x,w) = exp(-H~(x,w)) / Z_x
    (Eq. double_hamiltonian_pca_general_form) and stationary measure
    pi~(x) = Z_x / Z (Eq. symm_ham_pca_stationary_measure);
  * the J = 0 closed forms (independent sites).
"""
from __future__ import annotations

import itertools

import numpy as np

from . import FLIP, GAUSS, POTTS, _f32, site_probs

_D8 = [(-1, 0), (1, 0), (0, -1), (0, 1), (-1, -1), (-1, 1), (1, -1), (1, 1)]


def _params(m):
    d = m.as_dict() if hasattr(m, "as_dict") else dict(m)
    return dict(L=int(d["L"]), nbhd=int(d.get("nbhd", 4)), pair=int(d.get("pair", 1)),
                T=int(d.get("pair_T", 1)), noise=int(d.get("noise", 0)),
                c=_f32(d.get("pair_coef", 0.0)), sigma=_f32(d.get("sigma", 1.0)),
                p=_f32(d.get("flip_p", 0.1)), lam=_f32(d.get("inertia", 0.0)),
                norm=int(d.get("inertia_norm", 0)))


def inertia_price(P, a, b):
    """rho(a, b): 1{a != b}, or (|a - b| / (L - 1))^p for p = inertia_norm."""
    a = np.asarray(a, dtype=np.int64)
    b = np.asarray(b, dtype=np.int64)
    if P["norm"] == 0:
        return (a != b).astype(np.float64)
    d = np.abs(a - b) / float(P["L"] - 1)
    return d if P["norm"] == 1 else d * d


def states(n: int, L: int) -> np.ndarray:
    """All L**n configurations; row k has label (k // L**i) % L at site i."""
    idx = np.arange(L ** n, dtype=np.int64)
    return np.stack([(idx // (L ** i)) % L for i in range(n)], axis=1)


def neighbours(H: int, W: int, nbhd: int):
    nb = []
    for r in range(H):
        for c in range(W):
            lst = []
            for dr, dc in _D8[:nbhd]:
                rr, cc = r + dr, c + dc
                if 0 <= rr < H and 0 <= cc < W:
                    lst.append(rr * W + cc)
            nb.append(lst)
    return nb


def edges(H: int, W: int, nbhd: int):
    nb = neighbours(H, W, nbhd)
    return [(i, j) for i in range(H * W) for j in nb[i] if i < j]


def pair_V(P, a, b):
    a = np.asarray(a, dtype=np.int64)
    b = np.asarray(b, dtype=np.int64)
    if P["pair"] == POTTS:
        return -P["c"] * (a == b)
    return P["c"] * np.minimum(np.abs(a - b), P["T"])


def data_U(P, g, s):
    s = np.asarray(s, dtype=np.int64)
    if P["noise"] == GAUSS:
        return (np.asarray(g, dtype=np.int64) - s) ** 2 / (2.0 * P["sigma"] * P["sigma"])
    if P["noise"] != FLIP:   # no likelihood
        return np.zeros(np.shape(s))
    same = -np.log(1.0 - P["p"])
    diff = -np.log(P["p"])
    return np.where(s == g, same, diff)


def posterior_logweights(m, g: np.ndarray) -> np.ndarray:
    """Unnormalised log pi_post over all states (state index as in states())."""
    P = _params(m)
    H, W = g.shape
    gf = g.reshape(-1).astype(np.int64)
    X = states(H * W, P["L"])
    logw = np.zeros(X.shape[0])
    for i, j in edges(H, W, P["nbhd"]):
        logw -= pair_V(P, X[:, i], X[:, j])
    for i in range(H * W):
        logw -= data_U(P, gf[i], X[:, i])
    return logw


def _site_energy_all(P, X, nb, gf, i, s):
    """E_i(s | x) for every state x (rows of X): the lazy-PCA conditional energy."""
    e = data_U(P, gf[i], s) + P["lam"] * inertia_price(P, X[:, i], s)
    for j in nb[i]:
        e = e + pair_V(P, s, X[:, j])
    return e


def pca_stationary_logweights(m, g: np.ndarray) -> np.ndarray:
    """log Z_x = -sum_i U_i(x_i) + sum_i log sum_s exp(-E_i(s|x))  (+ const)."""
    P = _params(m)
    H, W = g.shape
    gf = g.reshape(-1).astype(np.int64)
    X = states(H * W, P["L"])
    nb = neighbours(H, W, P["nbhd"])
    logw = np.zeros(X.shape[0])
    for i in range(H * W):
        logw -= data_U(P, gf[i], X[:, i])
        Es = np.stack([_site_energy_all(P, X, nb, gf, i, s) for s in range(P["L"])], axis=1)
        emin = Es.min(axis=1, keepdims=True)
        logw += np.log(np.exp(-(Es - emin)).sum(axis=1)) - emin[:, 0]
    return logw


def pair_hamiltonian(m, g: np.ndarray) -> np.ndarray:
    """Matrix H~(x, w) over all pairs of states of a tiny lattice."""
    P = _params(m)
    H, W = g.shape
    n = H * W
    gf = g.reshape(-1).astype(np.int64)
    X = states(n, P["L"])
    nb = neighbours(H, W, P["nbhd"])
    Xr = X[:, None, :]        # x (rows)
    Wc = X[None, :, :]        # w (cols)
    Ht = np.zeros((X.shape[0], X.shape[0]))
    for i in range(n):
        for j in nb[i]:
            Ht += pair_V(P, Wc[..., i], Xr[..., j])
        Ht += data_U(P, gf[i], Wc[..., i]) + data_U(P, gf[i], Xr[..., i])
        Ht += P["lam"] * inertia_price(P, Wc[..., i], Xr[..., i])
    return Ht


def pca_transition_from_pair(m, g: np.ndarray) -> np.ndarray:
    """P(x, w) = exp(-H~(x,w)) / sum_w exp(-H~(x,w))."""
    Ht = pair_hamiltonian(m, g)
    Ht = Ht - Ht.min(axis=1, keepdims=True)
    Pm = np.exp(-Ht)
    return Pm / Pm.sum(axis=1, keepdims=True)


def pca_transition_from_conditionals(m, g: np.ndarray) -> np.ndarray:
    """P(x, w) = prod_i p_i(w_i | x), with p_i from the C oracle's conditional."""
    P = _params(m)
    H, W = g.shape
    n = H * W
    gf = g.reshape(-1).astype(np.int64)
    X = states(n, P["L"])
    nb = neighbours(H, W, P["nbhd"])
    T = np.ones((X.shape[0], X.shape[0]))
    for a, x in enumerate(X):
        for i in range(n):
            p = site_probs(m, gf[i], x[i], [x[j] for j in nb[i]], P["lam"])
            T[a, :] *= p[X[:, i]]
    return T


def normalise_log(logw: np.ndarray) -> np.ndarray:
    w = np.exp(logw - logw.max())
    return w / w.sum()


def tv(p: np.ndarray, q: np.ndarray) -> float:
    return 0.5 * float(np.abs(np.asarray(p) - np.asarray(q)).sum())


def tv_noise_floor(p: np.ndarray, n_eff: float) -> float:
    """Expected TV of an empirical histogram of n_eff independent draws from p
    (normal approximation: E|N(0, p(1-p)/n)| summed over states, halved)."""
    p = np.asarray(p)
    return 0.5 * float(np.sum(np.sqrt(2.0 * p * (1.0 - p) / (np.pi * n_eff))))


def j0_gibbs_marginal(m, g_i: int) -> np.ndarray:
    """J = 0: the posterior factorises; site law p(s) ~ exp(-U(s))."""
    P = _params(m)
    u = data_U(P, g_i, np.arange(P["L"]))
    w = np.exp(-(u - u.min()))
    return w / w.sum()


def j0_pca_marginal(m, g_i: int) -> np.ndarray:
    """J = 0 lazy PCA: independent single-site chains with transition
    P(x, s) ~ exp(-U(s) - lambda rho(s, x)), rho symmetric; detailed balance
    gives pi(x) ~ exp(-U(x)) sum_s exp(-U(s) - lambda rho(s, x)), which for the
    L0 price is exp(-U(x)) [exp(-lambda) Z_U + (1 - exp(-lambda)) exp(-U(x))]."""
    P = _params(m)
    L = P["L"]
    u = data_U(P, g_i, np.arange(L))
    eu = np.exp(-(u - u.min()))
    if P["norm"] == 0:
        ZU = eu.sum()
        el = np.exp(-P["lam"])
        w = eu * (el * ZU + (1.0 - el) * eu)
    else:
        s = np.arange(L)
        R = inertia_price(P, s[:, None], s[None, :])
        w = eu * (np.exp(-P["lam"] * R) @ eu)
    return w / w.sum()


def single_site_chain_stationary(m, g_i: int) -> np.ndarray:
    """J = 0 lazy PCA, by linear algebra: left eigenvector of the L x L
    single-site transition matrix (independent of the closed form above)."""
    P = _params(m)
    L = P["L"]
    u = data_U(P, g_i, np.arange(L))
    K = np.zeros((L, L))
    for x in range(L):
        e = u + P["lam"] * inertia_price(P, np.arange(L), x)
        w = np.exp(-(e - e.min()))
        K[x] = w / w.sum()
    vals, vecs = np.linalg.eig(K.T)
    k = int(np.argmin(np.abs(vals - 1.0)))
    v = np.real(vecs[:, k])
    return v / v.sum()


def all_pairs(n):
    return list(itertools.combinations(range(n), 2))
