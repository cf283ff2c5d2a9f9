"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test ties one oracle function to something other than itself:
printed values (Table I), closed forms (geometric scan, product states,
the unrolled kernel of Sec. II.E), invariants (autoregressive normalisation,
zero-variance of an exact eigenstate, the variational bound), an
independently built sparse Hamiltonian (Kronecker products of Pauli
matrices), central finite differences and a chi^2 test of the sampler.
"""
import math
import os

import numpy as np
import pytest
from scipy.special import erf
from scipy.stats import chi2

from oracle import ed
from paper_2605_13807_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _gelu(x):
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def _layer_views(theta, n_layers, H):
    """Named views of the flat parameter vector (layout convention)."""
    out = {}
    off = 0
    for name, shape, _ in inputs.param_shapes(n_layers, H):
        n = int(np.prod(shape))
        out[name] = np.asarray(theta[off:off + n], dtype=np.float64).reshape(shape)
        off += n
    return out


def _set(theta, n_layers, H, name, value):
    off = 0
    for nm, shape, _ in inputs.param_shapes(n_layers, H):
        n = int(np.prod(shape))
        if nm == name:
            theta[off:off + n] = np.broadcast_to(value, shape).ravel()
            return theta
        off += n
    raise KeyError(name)


# ------------------------------------------------------------------ ED pins

def test_tfim_exact_energies_match_table_I(oracle_mod):
    """ED of the 1D TFIM (OBC, h=1) reproduces the paper's exact column."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "tfim_obc_h1_exact.txt"))
            if l.strip() and not l.startswith("#")]
    table = {int(a): float(b) for a, b in rows}
    for N, e_tab in table.items():
        closed = (1.0 - 1.0 / math.sin(math.pi / (2 * (2 * N + 1)))) / N
        assert abs(closed - e_tab) < 6e-8, (N, closed, e_tab)
        if N <= 16:
            pairs = oracle_mod.bonds(N, 1, False)
            E0, _ = ed.ground_state(ed.tfim(N, pairs, J=1.0, h=1.0))
            assert abs(E0 / N - e_tab) < 6e-8, (N, E0 / N, e_tab)
    # large-N series of App. B
    N = 256
    closed = (1.0 - 1.0 / math.sin(math.pi / (2 * (2 * N + 1)))) / N
    series = -4 / math.pi + (math.pi - 2) / math.pi / N - math.pi / 24 / N**2 + math.pi / 48 / N**3
    assert abs(closed - series) < 1e-9


def test_heisenberg_small_exact_energies(oracle_mod):
    E2, _ = ed.ground_state(ed.heisenberg(2, oracle_mod.bonds(2, 1, False)))
    assert abs(E2 + 0.75) < 1e-12  # singlet
    E4, _ = ed.ground_state(ed.heisenberg(4, oracle_mod.bonds(4, 1, False)))
    assert abs(E4 + (3 + 2 * math.sqrt(3)) / 4) < 1e-10  # open 4-site chain


# ---------------------------------------------------------- lattice / bonds

@pytest.mark.parametrize("Lx,Ly", [(5, 1), (4, 3), (3, 4), (6, 6)])
def test_zigzag_predecessors(oracle_mod, Lx, Ly):
    """Sequence predecessor of (i,j) is (i-(-1)^j, j), or (i, j-1) at a row start."""
    where = {}
    for j in range(Ly):
        for i in range(Lx):
            where[oracle_mod.seq_pos(Lx, i, j)] = (i, j)
    assert sorted(where) == list(range(Lx * Ly))
    for pos in range(1, Lx * Ly):
        i, j = where[pos]
        pi, pj = where[pos - 1]
        hor = (i - (-1) ** j, j)
        if 0 <= hor[0] < Lx:
            assert (pi, pj) == hor
        else:
            assert (pi, pj) == (i, j - 1)


@pytest.mark.parametrize("Lx,Ly,pbc", [(10, 1, False), (10, 1, True), (4, 3, False),
                                       (4, 4, True), (6, 5, False), (3, 3, True)])
def test_bonds_are_all_nearest_neighbour_pairs(oracle_mod, Lx, Ly, pbc):
    b = oracle_mod.bonds(Lx, Ly, pbc)
    got = {tuple(x) for x in b.tolist()}
    assert len(got) == len(b)
    want = set()
    coords = [(i, j) for j in range(Ly) for i in range(Lx)]
    for (i1, j1) in coords:
        for (i2, j2) in coords:
            di = abs(i1 - i2)
            dj = abs(j1 - j2)
            if pbc and Lx >= 3:
                di = min(di, Lx - di)
            if pbc and Ly >= 3:
                dj = min(dj, Ly - dj)
            if di + dj == 1:
                p = oracle_mod.seq_pos(Lx, i1, j1)
                q = oracle_mod.seq_pos(Lx, i2, j2)
                want.add((min(p, q), max(p, q)))
    assert got == want
    assert all(p < q for p, q in b.tolist())


# ----------------------------------------------------------------- scans

@pytest.mark.parametrize("N", [1, 2, 3, 7, 64, 100, 257])
def test_blelloch_equals_sequential(oracle_mod, N):
    u = inputs.uniform(11 + N, (2, N))
    a = u[0]
    b = 2 * u[1] - 1
    hs = oracle_mod.scan_sequential(a, b, 0.3)
    hb = oracle_mod.scan_blelloch(a, b, 0.3)
    assert np.max(np.abs(hs - hb)) <= 1e-12 * max(1.0, np.max(np.abs(hs)))


def test_scan_constant_coefficients_closed_form(oracle_mod):
    """Constant a, b: h_t = a^{t+1} h0 + b (1 - a^{t+1}) / (1 - a)."""
    N, a, b, h0 = 200, 0.93, -0.7, 0.25
    t = np.arange(N)
    want = a ** (t + 1) * h0 + b * (1 - a ** (t + 1)) / (1 - a)
    for fn in (oracle_mod.scan_sequential, oracle_mod.scan_blelloch):
        got = fn(np.full(N, a), np.full(N, b), h0)
        assert np.max(np.abs(got - want)) < 1e-12


# ------------------------------------------------------- network structure

def _all_configs(N):
    return ed.all_configs(N)


@pytest.mark.parametrize("n_layers,H,N", [(1, 4, 9), (3, 6, 10), (4, 5, 8)])
def test_autoregressive_normalisation(oracle_mod, n_layers, H, N):
    theta = inputs.random_params(n_layers, H, seed=100 + N, scale=1.5)
    cfg = _all_configs(N)
    lp = oracle_mod.logpsi(theta, n_layers, H, cfg)
    assert abs(np.sum(np.exp(2 * lp)) - 1.0) < 1e-12


def test_u1_normalisation_over_zero_magnetisation_sector(oracle_mod):
    n_layers, H, N = 3, 5, 10
    theta = inputs.random_params(n_layers, H, seed=7, scale=1.5)
    cfg = _all_configs(N)
    lp = oracle_mod.logpsi(theta, n_layers, H, cfg, u1=True)
    in_sector = cfg.sum(axis=1) == N // 2
    assert np.all(np.isneginf(lp[~in_sector]))
    assert abs(np.sum(np.exp(2 * lp[in_sector])) - 1.0) < 1e-12


def test_constant_gate_layer_is_the_unrolled_kernel(oracle_mod):
    """W_z = 0 gives a constant gate a, and the layer becomes the linear
    time-invariant filter h_t = sum_{i<=t} (1-a) a^{t-i} h~_i (Sec. II.E)."""
    n_layers, H, N = 1, 4, 12
    theta = inputs.random_params(n_layers, H, seed=3, scale=1.0).astype(np.float64)
    theta = _set(theta, n_layers, H, "W_z0", 0.0)
    v = _layer_views(theta, n_layers, H)
    s = np.array([0, 1, 1, 0, 1, 0, 0, 0, 1, 1, 1, 0], dtype=np.uint8)
    _, h, x, _ = oracle_mod.trace(theta, n_layers, H, s)
    a = 1.0 / (1.0 + np.exp(-v["b_z0"]))
    u = np.zeros((N, 2))
    u[np.arange(1, N), s[:-1]] = 1.0  # one-hot of the previous spin, zero at t=0
    cand = u @ v["W_h0"].T + v["b_h0"]
    for t in range(N):
        want = sum((1 - a) * a ** (t - i) * cand[i] for i in range(t + 1))
        assert np.max(np.abs(h[t, 0] - want)) < 1e-12
    # output map x = GELU(C h + D u) with C, D read as [out][in]
    want_x = _gelu(h[:, 0] @ v["C0"].T + u @ v["D0"].T)
    assert np.max(np.abs(x[:, 0] - want_x)) < 1e-12


def test_residual_enters_from_the_previous_layer_for_l_ge_2(oracle_mod):
    n_layers, H, N = 3, 4, 7
    theta = inputs.random_params(n_layers, H, seed=5, scale=1.0).astype(np.float64)
    for l in (1, 2):
        theta = _set(theta, n_layers, H, f"C{l}", 0.0)
        theta = _set(theta, n_layers, H, f"D{l}", 0.0)
    s = np.array([1, 0, 0, 1, 1, 0, 1], dtype=np.uint8)
    _, h, x, _ = oracle_mod.trace(theta, n_layers, H, s)
    assert np.max(np.abs(x[:, 1])) == 0.0             # no residual at l = 1
    assert np.max(np.abs(x[:, 2] - _gelu(h[:, 1]))) < 1e-14  # s^(2) = h^(1)


# ---------------------------------------------------------- product states

def _product_theta(n_layers, H, beta, seed=9):
    theta = inputs.random_params(n_layers, H, seed=seed, scale=1.0).astype(np.float64)
    theta = _set(theta, n_layers, H, "W_o", 0.0)
    return _set(theta, n_layers, H, "b_o", np.asarray(beta, dtype=np.float64))


def test_product_state_logpsi_closed_form(oracle_mod):
    n_layers, H, N = 3, 4, 11
    beta = np.array([0.3, -0.8])
    theta = _product_theta(n_layers, H, beta)
    s = inputs.random_spins(1, 16, N)
    lsm = beta - np.log(np.sum(np.exp(beta)))
    want = 0.5 * lsm[s].sum(axis=1)
    assert np.max(np.abs(oracle_mod.logpsi(theta, n_layers, H, s) - want)) < 1e-13
    theta0 = _product_theta(n_layers, H, [0.0, 0.0])
    assert np.max(np.abs(oracle_mod.logpsi(theta0, n_layers, H, s) + 0.5 * N * np.log(2))) < 1e-13


@pytest.mark.parametrize("Lx,Ly,pbc", [(10, 1, False), (10, 1, True), (4, 3, False)])
def test_product_state_heisenberg_eloc(oracle_mod, Lx, Ly, pbc):
    """Exchanging an antiparallel pair keeps the spin multiset, so the ratio
    is 1: E_loc = (J/4) sum sigma sigma - (J/2) n_anti with the Marshall sign."""
    n_layers, H, N, J = 2, 3, Lx * Ly, 1.3
    theta = _product_theta(n_layers, H, [0.4, -0.1])
    s = inputs.random_spins(2, 12, N)
    got = oracle_mod.local_energy(theta, n_layers, H, s, oracle_mod.HEISENBERG, Lx, Ly,
                                  pbc=pbc, marshall=True, J=J)
    b = oracle_mod.bonds(Lx, Ly, pbc)
    sig = 2.0 * s - 1.0
    zz = (sig[:, b[:, 0]] * sig[:, b[:, 1]]).sum(axis=1)
    n_anti = (s[:, b[:, 0]] != s[:, b[:, 1]]).sum(axis=1)
    assert np.max(np.abs(got - (0.25 * J * zz - 0.5 * J * n_anti))) < 1e-12


def test_product_state_tfim_eloc_and_mean(oracle_mod):
    n_layers, H, Lx, Ly, J, hf = 2, 3, 3, 3, 0.7, 3.044
    N = Lx * Ly
    beta = np.array([0.5, -0.2])
    theta = _product_theta(n_layers, H, beta)
    s = inputs.random_spins(3, 10, N)
    got = oracle_mod.local_energy(theta, n_layers, H, s, oracle_mod.TFIM, Lx, Ly, J=J, h=hf)
    b = oracle_mod.bonds(Lx, Ly, False)
    sig = 2.0 * s - 1.0
    zz = (sig[:, b[:, 0]] * sig[:, b[:, 1]]).sum(axis=1)
    p = np.exp(beta - np.log(np.sum(np.exp(beta))))
    ratio = np.sqrt(p[1 - s] / p[s]).sum(axis=1)
    assert np.max(np.abs(got - (-J * zz - hf * ratio))) < 1e-12
    # beta = 0: <E> = -h N exactly (sum over all 2^N configurations)
    theta0 = _product_theta(n_layers, H, [0.0, 0.0])
    cfg = _all_configs(N)
    e = oracle_mod.local_energy(theta0, n_layers, H, cfg, oracle_mod.TFIM, Lx, Ly, J=J, h=hf)
    w = np.exp(2 * oracle_mod.logpsi(theta0, n_layers, H, cfg))
    assert abs(np.sum(w * e) + hf * N) < 1e-10


# ------------------------------------------------ E_loc against sparse H

def _sublattice_a(Lx, Ly, oracle_mod):
    return np.array([oracle_mod.seq_pos(Lx, i, j) for j in range(Ly) for i in range(Lx)
                     if (i + j) % 2 == 0])


@pytest.mark.parametrize("kind,Lx,Ly,pbc,u1", [
    (0, 10, 1, False, False), (0, 10, 1, True, True), (0, 4, 3, False, True),
    (0, 4, 3, False, False), (1, 10, 1, False, False), (1, 3, 3, False, False)])
def test_mean_local_energy_equals_hamiltonian_expectation(oracle_mod, kind, Lx, Ly, pbc, u1):
    n_layers, H = 3, 4
    N = Lx * Ly
    J, hf = 1.0, (3.044 if Ly > 1 else 1.0)
    theta = inputs.random_params(n_layers, H, seed=20 + N + kind, scale=1.5)
    cfg = _all_configs(N)
    lp = oracle_mod.logpsi(theta, n_layers, H, cfg, u1=u1)
    psi = np.exp(lp)
    keep = psi > 0
    eloc = np.zeros(len(cfg))
    eloc[keep] = oracle_mod.local_energy(theta, n_layers, H, cfg[keep], kind, Lx, Ly, pbc=pbc,
                                         marshall=True, J=J, h=hf, u1=u1)
    mean = np.sum(psi[keep] ** 2 * eloc[keep])
    pairs = oracle_mod.bonds(Lx, Ly, pbc)
    if kind == 0:
        Hm = ed.heisenberg(N, pairs, J=J)
        phys = psi * ed.marshall_sign(cfg, _sublattice_a(Lx, Ly, oracle_mod))
    else:
        Hm = ed.tfim(N, pairs, J=J, h=hf)
        phys = psi
    assert abs(mean - ed.expectation(Hm, phys)) < 1e-10
    E0, _ = ed.ground_state(Hm)
    assert mean >= E0 - 1e-10  # variational bound


@pytest.mark.parametrize("kind,Lx,Ly", [(0, 8, 1), (0, 4, 2), (1, 8, 1)])
def test_exact_ground_state_has_zero_variance(oracle_mod, kind, Lx, Ly):
    """E_loc of the exact ground state is E0 on every configuration."""
    N = Lx * Ly
    pairs = oracle_mod.bonds(Lx, Ly, False)
    cfg = _all_configs(N)
    if kind == 0:
        Hm = ed.heisenberg(N, pairs)
        E0, v = ed.ground_state(Hm)
        v = np.real(v * ed.marshall_sign(cfg, _sublattice_a(Lx, Ly, oracle_mod)))
    else:
        Hm = ed.tfim(N, pairs, J=1.0, h=1.0)
        E0, v = ed.ground_state(Hm)
        v = np.real(v)
    v = v * np.sign(v[np.argmax(np.abs(v))])
    assert np.min(v) > -1e-10  # positive in the rotated basis
    table = np.log(np.abs(v))
    index = {tuple(c): k for k, c in enumerate(cfg.tolist())}
    coeff = oracle_mod.offdiag_coeff(kind, 1.0, 1.0, True)
    offs, ent, diag = oracle_mod.connected(kind, Lx, Ly, False, cfg)
    for k in np.flatnonzero(np.abs(v) > 1e-6):
        lps = []
        for e in range(offs[k], offs[k + 1]):
            sp = cfg[k].copy()
            sp[ent[e, 1]] ^= 1
            if ent[e, 2] >= 0:
                sp[ent[e, 2]] ^= 1
            lps.append(table[index[tuple(sp.tolist())]])
        el = oracle_mod.eloc_combine(diag[k], coeff, table[k], np.array(lps))
        assert abs(el - E0) < 1e-8


# ---------------------------------------------------------------- gradient

@pytest.mark.parametrize("u1", [False, True])
def test_gradient_matches_central_finite_differences(oracle_mod, u1):
    n_layers, H, N = 3, 5, 10
    theta = inputs.random_params(n_layers, H, seed=31, scale=1.2).astype(np.float64)
    s = inputs.zero_magnetisation_spins(4, 1, N)[0]
    lp, g = oracle_mod.grad(theta, n_layers, H, s, u1=u1)
    eps = 1e-4
    fd = np.empty_like(theta)
    for k in range(theta.size):
        tp = theta.copy(); tp[k] += eps
        tm = theta.copy(); tm[k] -= eps
        fd[k] = (oracle_mod.logpsi(tp, n_layers, H, s, u1=u1)[0]
                 - oracle_mod.logpsi(tm, n_layers, H, s, u1=u1)[0]) / (2 * eps)
    assert abs(lp[0] - oracle_mod.logpsi(theta, n_layers, H, s, u1=u1)[0]) < 1e-14
    assert np.max(np.abs(g[0] - fd)) <= 1e-7 * max(1.0, np.max(np.abs(fd)))


# ----------------------------------------------------------------- sampler

def test_sampler_frequencies_chi2(oracle_mod):
    n_layers, H, N, n = 2, 4, 6, 40000
    theta = inputs.random_params(n_layers, H, seed=41, scale=1.5)
    u = inputs.uniform(42, (n, N))
    s, lps = oracle_mod.sample(theta, n_layers, H, N, u)
    assert np.max(np.abs(lps - oracle_mod.logpsi(theta, n_layers, H, s))) < 1e-12
    cfg = _all_configs(N)
    p = np.exp(2 * oracle_mod.logpsi(theta, n_layers, H, cfg))
    idx = (s.astype(np.int64) << (N - 1 - np.arange(N))).sum(axis=1)
    obs = np.bincount(idx, minlength=2 ** N)
    exp = p * n
    stat = np.sum((obs - exp) ** 2 / exp)
    assert chi2.sf(stat, df=2 ** N - 1) > 1e-4


def test_sampler_respects_u1(oracle_mod):
    n_layers, H, N = 2, 4, 10
    theta = inputs.random_params(n_layers, H, seed=43, scale=1.5)
    s, lps = oracle_mod.sample(theta, n_layers, H, N, inputs.uniform(44, (500, N)), u1=True)
    assert np.all(s.sum(axis=1) == N // 2)
    assert np.all(np.isfinite(lps))


def test_stats_unbiased_variance(oracle_mod):
    e = inputs.uniform(5, (1000,)) * 3 - 1
    m, v, se = oracle_mod.stats(e)
    assert abs(m - np.mean(e)) < 1e-13
    assert abs(v - np.var(e, ddof=1)) < 1e-13
    assert abs(se - np.sqrt(np.var(e, ddof=1) / e.size)) < 1e-13


def test_param_count_formula(oracle_mod):
    for H in (4, 32, 64, 128):
        assert oracle_mod.param_count(3, H) == 9 * H * H + 14 * H + 2
        assert oracle_mod.param_count(3, H) == inputs.param_count(3, H)
