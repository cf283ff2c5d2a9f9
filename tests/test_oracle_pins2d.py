"""Pins of the FP64 oracle of the two-dimensional patched minGRU (Sec. II.F
two-dimensional recurrences, Sec. II.G residual) against facts fixed by the
paper and by mathematics:

- autoregressive normalisation over all 2^N spin configurations (also on the
  zero-magnetisation sector), which any causal model satisfies;
- the predecessor rule H = (i - (-1)^j, j), V = (i, j - 1) on the patch
  lattice, read off the conditionals' dependence on earlier patches;
- closed forms of the horizontal scan along a row (row start at zero, the
  zigzag direction) and of the vertical coupling h~ = W_h [u, h_V];
- the residual wiring s_l = h_{l-1} for l >= 2 only;
- E_loc against an independently built sparse Hamiltonian;
- a chi^2 test of the sampler.
"""
import numpy as np
import pytest
from scipy.special import erf, logsumexp
from scipy.stats import chi2

from oracle import ed
from paper_2605_13807_gb300 import inputs


def _gelu(x):
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def _views(theta, n_layers, H):
    """Named views of the flat 2D parameter vector (layout convention)."""
    out, off = [], 0
    for l in range(n_layers):
        din = 32 if l == 0 else H
        d = {}
        for name, shape in (("Wz", (H, din)), ("bz", (H,)), ("Wh", (H, din + H)), ("bh", (H,)),
                            ("C", (H, H)), ("D", (H, din))):
            size = int(np.prod(shape))
            d[name] = theta[off:off + size].reshape(shape)
            off += size
        out.append(d)
    Wo = theta[off:off + 16 * H].reshape(16, H)
    bo = theta[off + 16 * H:off + 16 * H + 16]
    assert off + 16 * H + 16 == theta.size
    return out, Wo, bo


def _random_theta(oracle_mod, n_layers, H, seed, scale=1.0):
    P = oracle_mod.param_count2d(n_layers, H)
    return scale * (2.0 * inputs.uniform(seed, (P,)) - 1.0)


def _path(Px, Py):
    """(pi, pj) of each patch in path order (zigzag over the patch lattice)."""
    return [((k if pj % 2 == 0 else Px - 1 - k), pj) for pj in range(Py) for k in range(Px)]


def test_param_count_formula(oracle_mod):
    for H in (4, 32, 128):
        assert oracle_mod.param_count2d(3, H) == 12 * H * H + 118 * H + 16
        assert oracle_mod.param_count2d(1, H) == 2 * H * H + 98 * H + 16 * H + 16


@pytest.mark.parametrize("Lx,Ly,u1", [(4, 4, False), (4, 4, True), (4, 2, False), (2, 6, False),
                                      (6, 2, True)])
def test_normalisation_over_all_configurations(oracle_mod, Lx, Ly, u1):
    N = Lx * Ly
    theta = _random_theta(oracle_mod, 3, 4, seed=300 + N + Lx, scale=1.2)
    cfg = ed.all_configs(N)
    lp = oracle_mod.logpsi2d(theta, 3, 4, Lx, Ly, cfg, u1=u1)
    p = np.exp(2 * lp)
    assert abs(p.sum() - 1.0) < 1e-12
    if u1:
        assert np.all(p[cfg.sum(axis=1) != N // 2] == 0.0)


def test_predecessor_rule(oracle_mod):
    """One layer with C = 0: x1 = GELU(D (x0_H, x0_V)), so a patch's
    conditional depends on exactly its two causal predecessors."""
    Lx = Ly = 6
    Px = Py = 3
    H = 4
    theta = _random_theta(oracle_mod, 1, H, seed=310, scale=1.5)
    (layer,), _, _ = _views(theta, 1, H)
    layer["C"][:] = 0.0
    s = inputs.random_spins(311, 1, Lx * Ly)
    _, base = oracle_mod.logpsi2d(theta, 1, H, Lx, Ly, s, per_site=True)
    path = _path(Px, Py)
    index = {pq: t for t, pq in enumerate(path)}
    for t, (pi, pj) in enumerate(path):
        preds = set()
        hi = pi - (1 if pj % 2 == 0 else -1)
        if 0 <= hi < Px:
            preds.add(index[(hi, pj)])
        if pj > 0:
            preds.add(index[(pi, pj - 1)])
        for tp in range(t):
            qi, qj = path[tp]
            s2 = s.copy()
            s2[0, inputs.seq_pos(Lx, 2 * qi, 2 * qj)] ^= 1  # changes the value of patch tp only
            _, lp2 = oracle_mod.logpsi2d(theta, 1, H, Lx, Ly, s2, per_site=True)
            changed = abs(lp2[0, t] - base[0, t]) > 1e-12
            assert changed == (tp in preds), (t, tp)


def _closed_form_logp(Wo, bo, x_per_patch, vals):
    logits = x_per_patch @ Wo.T + bo
    return logits[np.arange(len(vals)), vals] - logsumexp(logits, axis=1)


def _patch_values(s, Lx, Ly):
    Px, Py = Lx // 2, Ly // 2
    vals = []
    for pi, pj in _path(Px, Py):
        v = 0
        for dy in range(2):
            for dx in range(2):
                v |= int(s[inputs.seq_pos(Lx, 2 * pi + dx, 2 * pj + dy)]) << (2 * dy + dx)
        vals.append(v)
    return np.array(vals)


def test_horizontal_scan_closed_form(oracle_mod):
    """z = sigma(beta_z) constant, h~ = beta_h: along each row, in path order,
    h_k = beta_h (1 - a^(k+1)) from zero at the row start."""
    Lx, Ly, H = 10, 6, 1
    Px, Py = Lx // 2, Ly // 2
    theta = _random_theta(oracle_mod, 1, H, seed=320)
    (layer,), Wo, bo = _views(theta, 1, H)
    layer["Wz"][:] = 0.0
    layer["Wh"][:] = 0.0
    layer["D"][:] = 0.0
    bz, bh, c = 0.7, -1.3, 0.9
    layer["bz"][:] = bz
    layer["bh"][:] = bh
    layer["C"][:] = c
    s = inputs.random_spins(321, 1, Lx * Ly)[0]
    _, lp = oracle_mod.logpsi2d(theta, 1, H, Lx, Ly, s, per_site=True)
    a = 1.0 / (1.0 + np.exp(-bz))
    k = np.tile(np.arange(Px), Py)  # position within the row, in path order
    h = bh * (1.0 - a ** (k + 1))
    x = _gelu(c * h)[:, None]
    assert np.max(np.abs(lp[0] - _closed_form_logp(Wo, bo, x, _patch_values(s, Lx, Ly)))) < 1e-12


def test_vertical_coupling_closed_form(oracle_mod):
    """z = 0, h~ = M h_V + beta with a non-symmetric M: row j holds
    (1 + M + ... + M^j) beta."""
    Lx, Ly, H = 6, 8, 2
    Px, Py = Lx // 2, Ly // 2
    theta = _random_theta(oracle_mod, 1, H, seed=330)
    (layer,), Wo, bo = _views(theta, 1, H)
    layer["Wz"][:] = 0.0
    layer["bz"][:] = -60.0  # sigma = 9e-27
    layer["Wh"][:] = 0.0
    M = np.array([[0.5, -0.9], [0.2, 0.3]])
    beta = np.array([0.6, -0.4])
    Cm = np.array([[1.1, 0.3], [-0.5, 0.8]])
    layer["Wh"][:, 32:] = M
    layer["bh"][:] = beta
    layer["D"][:] = 0.0
    layer["C"][:] = Cm
    s = inputs.random_spins(331, 1, Lx * Ly)[0]
    _, lp = oracle_mod.logpsi2d(theta, 1, H, Lx, Ly, s, per_site=True)
    rows, h = [], np.zeros(H)
    for _ in range(Py):
        h = M @ h + beta
        rows.append(h.copy())
    x = np.array([_gelu(Cm @ rows[t // Px]) for t in range(Px * Py)])
    assert np.max(np.abs(lp[0] - _closed_form_logp(Wo, bo, x, _patch_values(s, Lx, Ly)))) < 1e-12


def test_residual_only_from_layer_two(oracle_mod):
    """Layer 1: z = 0, h~ = beta (so h1 = beta), C1 = D1 = 0; layer 2: C2 = 0.
    With s_l = h_{l-1} for l >= 2 only, x2 = GELU(0) = 0 and
    x3 = GELU(D2 x2 + h1) = GELU(beta) at every patch."""
    Lx, Ly, H = 6, 4, 3
    theta = _random_theta(oracle_mod, 3, H, seed=340)
    layers, Wo, bo = _views(theta, 3, H)
    beta = np.array([0.4, -1.1, 0.8])
    layers[1]["Wz"][:] = 0.0
    layers[1]["bz"][:] = -60.0
    layers[1]["Wh"][:] = 0.0
    layers[1]["bh"][:] = beta
    layers[1]["C"][:] = 0.0
    layers[1]["D"][:] = 0.0
    layers[2]["C"][:] = 0.0
    s = inputs.random_spins(341, 1, Lx * Ly)[0]
    _, lp = oracle_mod.logpsi2d(theta, 3, H, Lx, Ly, s, per_site=True)
    vals = _patch_values(s, Lx, Ly)
    x = np.tile(_gelu(beta), (len(vals), 1))
    assert np.max(np.abs(lp[0] - _closed_form_logp(Wo, bo, x, vals))) < 1e-12


def _sublattice_a(Lx, Ly):
    return np.array([inputs.seq_pos(Lx, i, j) for j in range(Ly) for i in range(Lx)
                     if (i + j) % 2 == 0])


@pytest.mark.parametrize("kind,Lx,Ly,u1", [(0, 4, 2, False), (0, 4, 4, True), (1, 4, 2, False),
                                           (0, 2, 6, True)])
def test_mean_local_energy_equals_hamiltonian_expectation(oracle_mod, kind, Lx, Ly, u1):
    N = Lx * Ly
    theta = _random_theta(oracle_mod, 3, 4, seed=350 + N + kind, scale=1.2)
    cfg = ed.all_configs(N)
    lp = oracle_mod.logpsi2d(theta, 3, 4, Lx, Ly, cfg, u1=u1)
    psi = np.exp(lp)
    keep = psi > 0
    hf = 3.044
    eloc = oracle_mod.local_energy2d(theta, 3, 4, cfg[keep], kind, Lx, Ly, pbc=False,
                                     marshall=True, J=1.0, h=hf, u1=u1)
    mean = np.sum(psi[keep] ** 2 * eloc)
    pairs = oracle_mod.bonds(Lx, Ly, False)
    if kind == 0:
        Hm = ed.heisenberg(N, pairs, J=1.0)
        phys = psi * ed.marshall_sign(cfg, _sublattice_a(Lx, Ly))
    else:
        Hm = ed.tfim(N, pairs, J=1.0, h=hf)
        phys = psi
    assert abs(mean - ed.expectation(Hm, phys)) < 1e-10
    E0, _ = ed.ground_state(Hm)
    assert mean >= E0 - 1e-10


def test_sampler_frequencies_chi2(oracle_mod):
    Lx, Ly, n = 4, 2, 40000
    theta = _random_theta(oracle_mod, 2, 4, seed=360, scale=1.5)
    u = inputs.uniform(361, (n, 2))
    s, lps = oracle_mod.sample2d(theta, 2, 4, Lx, Ly, u)
    assert np.max(np.abs(lps - oracle_mod.logpsi2d(theta, 2, 4, Lx, Ly, s))) < 1e-12
    cfg = ed.all_configs(8)
    p = np.exp(2 * oracle_mod.logpsi2d(theta, 2, 4, Lx, Ly, cfg))
    idx = (s.astype(np.int64) << (7 - np.arange(8))).sum(axis=1)
    obs = np.bincount(idx, minlength=256)
    stat = np.sum((obs - p * n) ** 2 / (p * n))
    assert chi2.sf(stat, df=255) > 1e-4


def test_sampler_respects_u1(oracle_mod):
    Lx, Ly = 4, 4
    theta = _random_theta(oracle_mod, 2, 4, seed=362, scale=1.5)
    s, lps = oracle_mod.sample2d(theta, 2, 4, Lx, Ly, inputs.uniform(363, (500, 4)), u1=True)
    assert np.all(s.sum(axis=1) == 8)
    assert np.all(np.isfinite(lps))


def test_conditionals_are_the_log_probabilities(oracle_mod):
    """The 16-way conditionals sum to one, vanish on masked values, and at the
    configuration's own values reproduce its per-patch log P."""
    Lx, Ly, H = 6, 4, 4
    theta = _random_theta(oracle_mod, 2, H, seed=370, scale=1.2)
    s = inputs.zero_magnetisation_spins(371, 5, Lx * Ly)
    probs = oracle_mod.conditionals2d(theta, 2, H, Lx, Ly, s, u1=True)
    assert np.allclose(probs.sum(axis=2), 1.0, atol=1e-13)
    _, lp = oracle_mod.logpsi2d(theta, 2, H, Lx, Ly, s, u1=True, per_site=True)
    vals = np.array([_patch_values(x, Lx, Ly) for x in s])
    own = np.take_along_axis(probs, vals[:, :, None], axis=2)[:, :, 0]
    assert np.max(np.abs(np.log(own) - lp)) < 1e-12
    assert np.any(probs == 0.0)  # the mask removes values near the end
