"""Pins of the FP64 oracle of c4v symmetrisation and of the VMC step
(oracle/vmc.py) against facts fixed by the definitions and by mathematics:

- the 8 index maps form the group c4v (distinct, closed, identity present);
- the symmetrised amplitude is invariant under the group and normalised;
- it equals the plain amplitude for a model that is already invariant;
- E_loc of psi_sym against an independently built sparse Hamiltonian;
- d log psi_sym / d theta against central finite differences;
- the energy-gradient estimator, fed every configuration with its exact
  probability, against finite differences of <psi|H|psi>;
- Adam against its closed form from a zero state.
"""
import numpy as np
import pytest

from oracle import ed
from oracle import vmc
from paper_2605_13807_gb300 import inputs


def _theta(n_layers, H, seed, scale=1.2):
    return inputs.random_params(n_layers, H, seed=seed, scale=scale).astype(np.float64)


def test_c4v_maps_form_the_group():
    for L in (3, 4, 5):
        maps = vmc.c4v_maps(L)
        keys = {tuple(m) for m in maps}
        assert len(keys) == 8
        assert tuple(range(L * L)) in keys  # identity
        for m in maps:
            assert sorted(m) == list(range(L * L))  # a permutation of the sites
            for k in maps:
                assert tuple(m[k]) in keys  # closed under composition


def test_symmetrised_amplitude_is_invariant_and_normalised(oracle_mod):
    L, nL, H = 4, 2, 4
    theta = _theta(nL, H, seed=700)

    def lp(x):
        return oracle_mod.logpsi(theta, nL, H, x)

    s = inputs.random_spins(701, 6, L * L)
    base = vmc.logpsi_sym(lp, s, L)
    for img in vmc.c4v_images(s, L):
        assert np.max(np.abs(vmc.logpsi_sym(lp, img, L) - base)) < 1e-12
    L3 = 3  # normalisation over all 2^9 configurations of the 3 x 3 lattice
    cfg = ed.all_configs(L3 * L3)
    assert abs(np.sum(np.exp(2 * vmc.logpsi_sym(lp, cfg, L3))) - 1.0) < 1e-12


def test_invariant_model_is_unchanged(oracle_mod):
    """All weights zero: psi depends only on the number of up spins, so it is
    c4v-invariant and psi_sym = psi."""
    L, nL, H = 4, 2, 4
    theta = np.zeros(oracle_mod.param_count(nL, H))
    theta[-2:] = [0.3, -0.5]  # b_o

    def lp(x):
        return oracle_mod.logpsi(theta, nL, H, x)

    s = inputs.random_spins(702, 8, L * L)
    assert np.max(np.abs(vmc.logpsi_sym(lp, s, L) - lp(s))) < 1e-12


@pytest.mark.parametrize("kind", [0, 1])
def test_mean_symmetrised_local_energy_equals_expectation(oracle_mod, kind):
    L, nL, H = 3, 2, 4
    N = L * L
    theta = _theta(nL, H, seed=710 + kind)

    def lp(x):
        return oracle_mod.logpsi(theta, nL, H, x)

    cfg = ed.all_configs(N)
    psi = np.exp(vmc.logpsi_sym(lp, cfg, L))
    hf = 3.044
    eloc = vmc.local_energy_sym(lp, cfg, kind, L, marshall=True, J=1.0, h=hf)
    mean = np.sum(psi ** 2 * eloc)
    pairs = oracle_mod.bonds(L, L, False)
    if kind == 0:
        Hm = ed.heisenberg(N, pairs, J=1.0)
        sub_a = np.array([oracle_mod.seq_pos(L, i, j) for j in range(L) for i in range(L)
                          if (i + j) % 2 == 0])
        phys = psi * ed.marshall_sign(cfg, sub_a)
    else:
        Hm = ed.tfim(N, pairs, J=1.0, h=hf)
        phys = psi
    assert abs(mean - ed.expectation(Hm, phys)) < 1e-10
    assert mean >= ed.ground_state(Hm)[0] - 1e-10


def test_symmetrised_gradient_matches_finite_differences(oracle_mod):
    L, nL, H = 3, 2, 4
    theta = _theta(nL, H, seed=720)
    s = inputs.random_spins(721, 3, L * L)
    g = vmc.grad_logpsi_sym(theta, nL, H, s, L)
    rng = np.random.default_rng(0)
    eps = 1e-4
    for k in rng.choice(theta.size, 12, replace=False):
        tp, tm = theta.copy(), theta.copy()
        tp[k] += eps
        tm[k] -= eps
        fp = vmc.logpsi_sym(lambda x: oracle_mod.logpsi(tp, nL, H, x), s, L)
        fm = vmc.logpsi_sym(lambda x: oracle_mod.logpsi(tm, nL, H, x), s, L)
        fd = (fp - fm) / (2 * eps)
        assert np.max(np.abs(fd - g[:, k])) <= 1e-7 * max(1.0, np.max(np.abs(g[:, k])))


def test_energy_gradient_estimator_matches_exact_energy_derivative(oracle_mod):
    """With every configuration weighted by its exact probability the
    estimator 2 <(E_loc - E) O> is the derivative of <psi|H|psi>."""
    N, nL, H = 8, 2, 4
    theta = _theta(nL, H, seed=730)
    cfg = ed.all_configs(N)
    pairs = oracle_mod.bonds(N, 1, False)
    Hm = ed.tfim(N, pairs, J=1.0, h=1.0)

    def energy(th):
        return ed.expectation(Hm, np.exp(oracle_mod.logpsi(th, nL, H, cfg)))

    lps, ok = oracle_mod.grad(theta, nL, H, cfg)
    eloc = oracle_mod.local_energy(theta, nL, H, cfg, 1, N, 1, h=1.0)
    g, mean = vmc.energy_gradient(eloc, ok, weights=np.exp(2 * lps))
    assert abs(mean - energy(theta)) < 1e-10
    rng = np.random.default_rng(1)
    eps = 1e-5
    for _ in range(4):
        d = rng.standard_normal(theta.size)
        fd = (energy(theta + eps * d) - energy(theta - eps * d)) / (2 * eps)
        assert abs(fd - g @ d) <= 1e-6 * max(1.0, abs(fd))


def test_adam_closed_form():
    rng = np.random.default_rng(2)
    theta = rng.standard_normal(50)
    g1 = rng.standard_normal(50)
    lr, eps = 1e-3, 1e-8
    t1, m, v = vmc.adam(theta, g1, np.zeros(50), np.zeros(50), 1, lr, eps=eps)
    # first step from zero moments: theta - lr g / (|g| + eps)
    assert np.max(np.abs(t1 - (theta - lr * g1 / (np.abs(g1) + eps)))) < 1e-15
    g2 = rng.standard_normal(50)
    t2, _, _ = vmc.adam(t1, g2, m, v, 2, lr, eps=eps)
    m2 = 0.9 * 0.1 * g1 + 0.1 * g2
    v2 = 0.999 * 0.001 * g1 ** 2 + 0.001 * g2 ** 2
    ref = t1 - lr * (m2 / (1 - 0.81)) / (np.sqrt(v2 / (1 - 0.999 ** 2)) + eps)
    assert np.max(np.abs(t2 - ref)) < 1e-15


def test_energy_gradient_ignores_a_constant_energy_shift(oracle_mod):
    """Adding a constant to H leaves the gradient unchanged on any sample
    set: the estimator is centred on the sample mean."""
    N, nL, H = 10, 2, 4
    theta = _theta(nL, H, seed=740)
    s = inputs.random_spins(741, 30, N)
    _, ok = oracle_mod.grad(theta, nL, H, s)
    e = inputs.uniform(742, (30,)) * 4 - 7
    g0, m0 = vmc.energy_gradient(e, ok)
    g1, m1 = vmc.energy_gradient(e + 5.0, ok)
    assert abs(m1 - m0 - 5.0) < 1e-12
    assert np.max(np.abs(g1 - g0)) < 1e-12 * max(1.0, np.max(np.abs(g0)))


def test_finite_difference_gradient_helper_matches_reverse_mode(oracle_mod):
    """The GPU tests' oracle-only energy-gradient reference (tests/fdcheck.py)
    agrees with the energy-gradient estimator over the oracle's analytic
    reverse-mode O_k (chain model, plain and c4v-symmetrised), and rejects a
    gradient with the centring dropped or the image weights replaced by 1/8."""
    import fdcheck

    nL, H, L = 2, 4, 4
    theta = _theta(nL, H, seed=720)
    s = inputs.zero_magnetisation_spins(721, 24, L * L)
    e = inputs.uniform(722, (24,)) * 3.0 - 1.0   # any energies: the helper only weights them
    _, ok = oracle_mod.grad(theta, nL, H, s, u1=True)
    g, _ = vmc.energy_gradient(e, ok)
    lp = lambda t: oracle_mod.logpsi(t, nL, H, s, u1=True)  # noqa: E731
    fdcheck.check_energy_gradient(g, lp, theta, e, seed=723, n_top=8, n_rand=8)
    with pytest.raises(AssertionError):  # centring dropped
        fdcheck.check_energy_gradient(2.0 * (e @ ok) / e.size, lp, theta, e, seed=723, n_top=8, n_rand=8)
    ok_sym = vmc.grad_logpsi_sym(theta, nL, H, s, L, u1=True)
    g_sym, _ = vmc.energy_gradient(e, ok_sym)
    lps = lambda t: vmc.logpsi_sym(lambda x: oracle_mod.logpsi(t, nL, H, x, u1=True), s, L)  # noqa: E731
    fdcheck.check_energy_gradient(g_sym, lps, theta, e, seed=724, n_top=8, n_rand=8)
    imgs = vmc.c4v_images(s, L)
    ok_avg = np.mean([oracle_mod.grad(theta, nL, H, x, u1=True)[1] for x in imgs], axis=0)
    with pytest.raises(AssertionError):  # equal image weights instead of psi(g s)^2
        fdcheck.check_energy_gradient(vmc.energy_gradient(e, ok_avg)[0], lps, theta, e, seed=724,
                                      n_top=8, n_rand=8)
