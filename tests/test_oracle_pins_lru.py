"""Pins of the FP64 oracle of the deep 1D LRU (Sec. II.B Eq. lru, Sec. II.G 1D
residual, Sec. III.B architecture) against facts fixed by the paper and by
mathematics:

- autoregressive normalisation over all 2^N configurations (also with u1);
- the closed form of the complex diagonal recurrence with a constant input,
  h_t = e^gamma beta (1 - lambda^t) / (1 - lambda), lambda =
  exp(-e^nu + i e^theta), read through y = Re(C h);
- the GLU block (W_a y + b_a) * sigmoid(W_g y + b_g) and the one-hot D at
  layer 0, with the recurrence switched off;
- the residual x^(l+1) = GLU(y^(l)) + x^(l) from layer 1 on only;
- E_loc against an independently built sparse Hamiltonian (TFIM and
  Heisenberg chains) and the variational bound;
- a chi^2 test of the sampler.
"""
import numpy as np
import pytest
from scipy.special import expit, logsumexp
from scipy.stats import chi2

from oracle import ed
from paper_2605_13807_gb300 import inputs


def _views(theta, n_layers, H):
    """Named views of the flat LRU parameter vector (layout convention)."""
    out, off = [], 0
    for l in range(n_layers):
        din = 2 if l == 0 else H
        d = {}
        for name, shape in (("nu", (H,)), ("theta", (H,)), ("gamma", (H,)), ("B_re", (H, din)),
                            ("B_im", (H, din)), ("C_re", (H, H)), ("C_im", (H, H)),
                            ("D", (H, 2) if l == 0 else (H,)), ("W_a", (H, H)), ("b_a", (H,)),
                            ("W_g", (H, H)), ("b_g", (H,))):
            size = int(np.prod(shape))
            d[name] = theta[off:off + size].reshape(shape)
            off += size
        out.append(d)
    Wo = theta[off:off + 2 * H].reshape(2, H)
    bo = theta[off + 2 * H:off + 2 * H + 2]
    assert off + 2 * H + 2 == theta.size
    return out, Wo, bo


def _theta(oracle_mod, nL, H, seed, scale=1.0):
    P = oracle_mod.param_count_lru(nL, H)
    return scale * (2.0 * inputs.uniform(seed, (P,)) - 1.0)


def _site_logp(Wo, bo, x, s):
    logits = x @ Wo.T + bo
    return logits[np.arange(len(s)), s] - logsumexp(logits, axis=1)


def test_param_count_formula(oracle_mod):
    for H in (4, 32, 64):
        assert oracle_mod.param_count_lru(3, H) == 16 * H * H + 25 * H + 2
        assert oracle_mod.param_count_lru(1, H) == 4 * H * H + 11 * H + 2 * H + 2


@pytest.mark.parametrize("N,u1", [(10, False), (10, True), (7, False)])
def test_normalisation_over_all_configurations(oracle_mod, N, u1):
    theta = _theta(oracle_mod, 3, 4, seed=500 + N, scale=1.2)
    cfg = ed.all_configs(N)
    p = np.exp(2 * oracle_mod.logpsi_lru(theta, 3, 4, cfg, u1=u1))
    assert abs(p.sum() - 1.0) < 1e-12
    if u1:
        assert np.all(p[cfg.sum(axis=1) != N // 2] == 0.0)


def test_complex_recurrence_closed_form(oracle_mod):
    """One layer, one unit: B u_t = beta for t >= 1 (equal columns), 0 at
    t = 0; D = 0; GLU reduced to the identity (W_a = 1, b_a = 0, W_g = 0,
    b_g = 40).  Then y_t = Re(c e^gamma beta (1 - lambda^t) / (1 - lambda))."""
    N, H = 12, 1
    theta = _theta(oracle_mod, 1, H, seed=510)
    (L,), Wo, bo = _views(theta, 1, H)
    nu, th, ga = -0.4, 0.9, 0.3
    beta = 0.7 - 0.5j
    c = 1.2 + 0.8j
    L["nu"][:] = nu
    L["theta"][:] = th
    L["gamma"][:] = ga
    L["B_re"][:] = beta.real
    L["B_im"][:] = beta.imag
    L["C_re"][:] = c.real
    L["C_im"][:] = c.imag
    L["D"][:] = 0.0
    L["W_a"][:] = 1.0
    L["b_a"][:] = 0.0
    L["W_g"][:] = 0.0
    L["b_g"][:] = 40.0
    s = inputs.random_spins(511, 1, N)[0]
    _, lp = oracle_mod.logpsi_lru(theta, 1, H, s, per_site=True)
    lam = np.exp(-np.exp(nu) + 1j * np.exp(th))
    t = np.arange(N)
    h = np.exp(ga) * beta * (1 - lam ** t) / (1 - lam)
    y = np.real(c * h) * expit(40.0)
    assert np.max(np.abs(lp[0] - _site_logp(Wo, bo, y[:, None], s))) < 1e-12


def test_glu_and_one_hot_input(oracle_mod):
    """Recurrence off (B = 0): y_t = D^(0) onehot(s_{t-1}) and
    x_t = (W_a y + b_a) * sigmoid(W_g y + b_g)."""
    N, H = 9, 3
    theta = _theta(oracle_mod, 1, H, seed=520, scale=1.3)
    (L,), Wo, bo = _views(theta, 1, H)
    L["B_re"][:] = 0.0
    L["B_im"][:] = 0.0
    s = inputs.random_spins(521, 1, N)[0]
    _, lp = oracle_mod.logpsi_lru(theta, 1, H, s, per_site=True)
    u = np.zeros((N, 2))
    u[np.arange(1, N), s[:-1]] = 1.0
    y = u @ L["D"].T
    x = (y @ L["W_a"].T + L["b_a"]) * expit(y @ L["W_g"].T + L["b_g"])
    assert np.max(np.abs(lp[0] - _site_logp(Wo, bo, x, s))) < 1e-12


def test_residual_from_layer_one_only(oracle_mod):
    """Layer 1 with B = 0 and D = 0 has y = 0, so x^(2) = b_a sigmoid(b_g) +
    x^(1), with x^(1) the GLU output of layer 0 (no residual there)."""
    N, H = 9, 3
    theta = _theta(oracle_mod, 2, H, seed=530, scale=1.3)
    (L0, L1), Wo, bo = _views(theta, 2, H)
    L0["B_re"][:] = 0.0
    L0["B_im"][:] = 0.0
    L1["B_re"][:] = 0.0
    L1["B_im"][:] = 0.0
    L1["D"][:] = 0.0
    s = inputs.random_spins(531, 1, N)[0]
    _, lp = oracle_mod.logpsi_lru(theta, 2, H, s, per_site=True)
    u = np.zeros((N, 2))
    u[np.arange(1, N), s[:-1]] = 1.0
    y0 = u @ L0["D"].T
    x1 = (y0 @ L0["W_a"].T + L0["b_a"]) * expit(y0 @ L0["W_g"].T + L0["b_g"])
    x2 = L1["b_a"] * expit(L1["b_g"]) + x1
    assert np.max(np.abs(lp[0] - _site_logp(Wo, bo, x2, s))) < 1e-12


@pytest.mark.parametrize("kind,N,pbc,u1", [(1, 8, False, False), (1, 8, True, False),
                                           (0, 10, False, True), (0, 8, True, False)])
def test_mean_local_energy_equals_hamiltonian_expectation(oracle_mod, kind, N, pbc, u1):
    theta = _theta(oracle_mod, 3, 4, seed=540 + N + kind, scale=1.2)
    cfg = ed.all_configs(N)
    psi = np.exp(oracle_mod.logpsi_lru(theta, 3, 4, cfg, u1=u1))
    keep = psi > 0
    hf = 1.0
    eloc = oracle_mod.local_energy_lru(theta, 3, 4, cfg[keep], kind, N, 1, pbc=pbc, marshall=True,
                                       J=1.0, h=hf, u1=u1)
    mean = np.sum(psi[keep] ** 2 * eloc)
    pairs = oracle_mod.bonds(N, 1, pbc)
    if kind == 0:
        Hm = ed.heisenberg(N, pairs, J=1.0)
        phys = psi * ed.marshall_sign(cfg, np.arange(0, N, 2))
    else:
        Hm = ed.tfim(N, pairs, J=1.0, h=hf)
        phys = psi
    assert abs(mean - ed.expectation(Hm, phys)) < 1e-10
    E0, _ = ed.ground_state(Hm)
    assert mean >= E0 - 1e-10


def test_sampler_frequencies_chi2(oracle_mod):
    N, n = 6, 40000
    theta = _theta(oracle_mod, 2, 4, seed=550, scale=1.5)
    u = inputs.uniform(551, (n, N))
    s, lps = oracle_mod.sample_lru(theta, 2, 4, N, u)
    assert np.max(np.abs(lps - oracle_mod.logpsi_lru(theta, 2, 4, s))) < 1e-12
    cfg = ed.all_configs(N)
    p = np.exp(2 * oracle_mod.logpsi_lru(theta, 2, 4, cfg))
    idx = (s.astype(np.int64) << (N - 1 - np.arange(N))).sum(axis=1)
    obs = np.bincount(idx, minlength=2 ** N)
    stat = np.sum((obs - p * n) ** 2 / (p * n))
    assert chi2.sf(stat, df=2 ** N - 1) > 1e-4
