"""GPU 2D patched minGRU (psr2d_logpsi, psr2d_local_energy) against the FP64
oracle of the same model.

Tolerances as for the chain model's FP32 path: |d log psi| <= 1e-5 +
1e-6 |log psi|; E_loc error <= 1e-3 of |diag| + |E_loc - diag|.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2605_13807_gb300 import api, binding as B, inputs  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    yield


def _theta(oracle_mod, nL, H, seed, scale):
    P = oracle_mod.param_count2d(nL, H)
    assert P == api.param_count2d(nL, H)
    # uniform entries of size scale / sqrt(fan-in) keep activations O(1)
    return (scale * (2.0 * inputs.uniform(seed, (P,)) - 1.0) / np.sqrt(H)).astype(np.float32)


def _spins(seed, n, Lx, Ly, u1):
    N = Lx * Ly
    return inputs.zero_magnetisation_spins(seed, n, N) if u1 else inputs.random_spins(seed, n, N)


@pytest.mark.parametrize("Lx,Ly,H,nL,u1", [(4, 4, 32, 3, False), (6, 4, 64, 2, True),
                                           (10, 10, 128, 3, True), (8, 6, 32, 1, False),
                                           (64, 4, 32, 2, False), (2, 8, 64, 3, True),
                                           (8, 6, 256, 3, True), (20, 4, 64, 2, True),
                                           (32, 2, 32, 3, False), (34, 2, 128, 2, True)])
def test_logpsi_matches_oracle(oracle_mod, Lx, Ly, H, nL, u1):
    theta = _theta(oracle_mod, nL, H, seed=400 + Lx + Ly + H, scale=2.0)
    s = _spins(401 + Lx, 40, Lx, Ly, u1)
    cfg = api.ModelConfig(nL, H, u1, "fp32")
    got = api.logpsi2d(torch.from_numpy(theta).cuda(), torch.from_numpy(s).cuda(), cfg, Lx, Ly)
    api.sync()
    ref = oracle_mod.logpsi2d(theta.astype(np.float64), nL, H, Lx, Ly, s, u1=u1)
    got = got.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(got) == np.isfinite(ref))
    fin = np.isfinite(ref)
    assert np.all(np.abs(got[fin] - ref[fin]) <= 1e-5 + 1e-6 * np.abs(ref[fin]))


@pytest.mark.parametrize("kind,Lx,Ly,H,u1,hf", [(0, 4, 4, 32, True, 0.0), (0, 6, 6, 64, True, 0.0),
                                                (1, 4, 6, 32, False, 3.044),
                                                (0, 10, 10, 128, True, 0.0),
                                                (0, 6, 4, 256, True, 0.0), (0, 18, 4, 64, True, 0.0)])
def test_local_energy_matches_oracle(oracle_mod, kind, Lx, Ly, H, u1, hf):
    nL = 3
    theta = _theta(oracle_mod, nL, H, seed=410 + Lx * Ly + kind, scale=2.0)
    n = 4 if Lx * Ly >= 100 else 12
    s = (inputs.neel_like_spins(411, n, Lx, Ly) if kind == 0 else inputs.random_spins(411, n, Lx * Ly))
    ham = B.make_hamiltonian(kind, Lx, Ly, False, True, 1.0, hf)
    cfg = api.ModelConfig(nL, H, u1, "fp32")
    e, st = api.local_energy2d(torch.from_numpy(theta).cuda(), torch.from_numpy(s).cuda(), cfg, ham)
    api.sync()
    ref = oracle_mod.local_energy2d(theta.astype(np.float64), nL, H, s, kind, Lx, Ly, pbc=False,
                                    marshall=True, J=1.0, h=hf, u1=u1)
    _, _, diag = oracle_mod.connected(kind, Lx, Ly, False, s)
    scale = np.abs(diag) + np.abs(ref - diag)
    assert np.all(np.abs(e.cpu().numpy() - ref) <= 1e-3 * scale)
    m, v, se = oracle_mod.stats(e.cpu().numpy().astype(np.float64))
    assert abs(st[0].item() - m) <= 1e-9 * max(1.0, abs(m))


def test_rejected_shapes_and_precision():
    theta = torch.zeros(api.param_count2d(3, 32), device="cuda")
    s = torch.zeros((2, 5 * 4), dtype=torch.uint8, device="cuda")
    out = torch.empty(2, device="cuda")
    with pytest.raises(B.PsrError) as ei:  # odd Lx
        B.psr2d_logpsi(B.make_params(theta, 3, 32), s, 5, 4, out)
    assert ei.value.code == B.PSR_EINVAL
    s2 = torch.zeros((2, 66 * 2), dtype=torch.uint8, device="cuda")
    with pytest.raises(B.PsrError) as ei:  # 33 patches in a row
        B.psr2d_logpsi(B.make_params(theta, 3, 32), s2, 66, 2, out)
    assert ei.value.code == B.PSR_EUNSUPPORTED
    s3 = torch.zeros((2, 16), dtype=torch.uint8, device="cuda")
    with pytest.raises(B.PsrError) as ei:  # tensor-core path: hidden 128 or 256 only
        B.psr2d_logpsi(B.make_params(theta, 3, 32, False, "bf16"), s3, 4, 4, out)
    assert ei.value.code == B.PSR_EUNSUPPORTED


def test_52x52_resume_equals_full_forwards(oracle_mod):
    """52x52, hidden 128, three layers, zero magnetisation: E_loc of two
    samples (connected configurations resumed at their patch row) equals the
    combination of full forwards of every connected configuration, and
    sampled log psi values agree with the oracle."""
    Lx = Ly = 52
    nL, H = 3, 128
    theta = inputs.glorot_params2d(nL, H, seed=0)
    assert theta.size == oracle_mod.param_count2d(nL, H)
    s = inputs.neel_like_spins(421, 2, Lx, Ly)
    ham = B.make_hamiltonian("heisenberg", Lx, Ly, False, True, 1.0, 0.0)
    cfg = api.ModelConfig(nL, H, True, "fp32")
    th = torch.from_numpy(theta).cuda()
    e, _ = api.local_energy2d(th, torch.from_numpy(s).cuda(), cfg, ham)
    offsets, entries, diag = oracle_mod.connected(0, Lx, Ly, False, s)
    flipped = np.repeat(s, np.diff(offsets), axis=0)
    rows = np.arange(flipped.shape[0])
    flipped[rows, entries[:, 1]] ^= 1
    flipped[rows, entries[:, 2]] ^= 1
    lp_s = api.logpsi2d(th, torch.from_numpy(s).cuda(), cfg, Lx, Ly).cpu().numpy().astype(np.float64)
    lp_f = api.logpsi2d(th, torch.from_numpy(flipped).cuda(), cfg, Lx, Ly).cpu().numpy().astype(np.float64)
    api.sync()
    full = np.array([diag[i] - 0.5 * np.sum(np.exp(lp_f[offsets[i]:offsets[i + 1]] - lp_s[i]))
                     for i in range(2)])
    scale = np.abs(diag) + np.abs(full - diag)
    assert np.all(np.abs(e.cpu().numpy() - full) <= 1e-4 * scale)
    pick = np.random.default_rng(0).choice(flipped.shape[0], 6, replace=False)
    ref = oracle_mod.logpsi2d(theta.astype(np.float64), nL, H, Lx, Ly,
                              np.concatenate([s, flipped[pick]]), u1=True)
    got = np.concatenate([lp_s, lp_f[pick]])
    assert np.all(np.abs(got - ref) <= 1e-5 + 1e-6 * np.abs(ref))


def _patch_vals(s, Lx, Ly):
    """[n, Np] patch values in path order (value bit 2 dy + dx)."""
    Px, Py = Lx // 2, Ly // 2
    out = np.zeros((s.shape[0], Px * Py), dtype=np.int64)
    t = 0
    for pj in range(Py):
        for k in range(Px):
            pi = k if pj % 2 == 0 else Px - 1 - k
            for dy in range(2):
                for dx in range(2):
                    out[:, t] |= s[:, inputs.seq_pos(Lx, 2 * pi + dx, 2 * pj + dy)].astype(np.int64) << (2 * dy + dx)
            t += 1
    return out


@pytest.mark.parametrize("Lx,Ly,H,nL,u1", [(6, 4, 32, 3, True), (8, 6, 64, 2, False),
                                           (10, 10, 128, 3, True), (8, 8, 256, 3, True)])
def test_sampler_follows_oracle_conditionals(oracle_mod, Lx, Ly, H, nL, u1):
    """Each patch's value is the first whose cumulative oracle probability
    exceeds its uniform, except within 1e-4 of a boundary (FP32 rounding);
    log psi of the draw matches the oracle."""
    theta = _theta(oracle_mod, nL, H, seed=430 + H, scale=2.0)
    n, Np = 120, (Lx // 2) * (Ly // 2)
    u = inputs.uniform(431, (n, Np)).astype(np.float32)
    cfg = api.ModelConfig(nL, H, u1, "fp32")
    s, lp = api.sample2d(torch.from_numpy(theta).cuda(), torch.from_numpy(u).cuda(), cfg, Lx, Ly)
    api.sync()
    s = s.cpu().numpy()
    if u1:
        assert np.all(s.sum(axis=1) == Lx * Ly // 2)
    probs = oracle_mod.conditionals2d(theta.astype(np.float64), nL, H, Lx, Ly, s, u1=u1)
    cdf = np.cumsum(probs, axis=2)
    v = _patch_vals(s, Lx, Ly)
    lo = np.where(v > 0, np.take_along_axis(cdf, np.maximum(v - 1, 0)[:, :, None], axis=2)[:, :, 0], 0.0)
    hi = np.take_along_axis(cdf, v[:, :, None], axis=2)[:, :, 0]
    u64 = u.astype(np.float64)
    inside = (u64 >= lo) & (u64 < hi)
    near = np.minimum(np.abs(u64 - lo), np.abs(u64 - hi)) <= 1e-4
    assert np.all(inside | near)
    assert np.count_nonzero(~inside) <= max(2, 1e-3 * inside.size)
    assert np.all(np.take_along_axis(probs, v[:, :, None], axis=2) > 0)  # never a masked value
    ref = oracle_mod.logpsi2d(theta.astype(np.float64), nL, H, Lx, Ly, s, u1=u1)
    assert np.all(np.abs(lp.cpu().numpy() - ref) <= 1e-5 + 1e-6 * np.abs(ref))


def test_sampler_frequencies_chi2(oracle_mod):
    from scipy.stats import chi2
    Lx, Ly, nL, H, n = 4, 2, 2, 32, 40000
    theta = _theta(oracle_mod, nL, H, seed=440, scale=3.0)
    u = inputs.uniform(441, (n, 2)).astype(np.float32)
    s, _ = api.sample2d(torch.from_numpy(theta).cuda(), torch.from_numpy(u).cuda(),
                        api.ModelConfig(nL, H, False, "fp32"), Lx, Ly)
    api.sync()
    s = s.cpu().numpy()
    cfg = ((np.arange(256)[:, None] >> (7 - np.arange(8))[None, :]) & 1).astype(np.uint8)
    p = np.exp(2 * oracle_mod.logpsi2d(theta.astype(np.float64), nL, H, Lx, Ly, cfg))
    idx = (s.astype(np.int64) << (7 - np.arange(8))).sum(axis=1)
    obs = np.bincount(idx, minlength=256)
    keep = p * n > 1e-9
    stat = np.sum((obs[keep] - p[keep] * n) ** 2 / (p[keep] * n))
    assert chi2.sf(stat, df=int(keep.sum()) - 1) > 1e-4


def test_sampler_tuned_tile_draws_identical_samples(oracle_mod):
    Lx, Ly, nL, H = 8, 8, 3, 128
    theta = torch.from_numpy(_theta(oracle_mod, nL, H, seed=450, scale=2.0)).cuda()
    u = torch.from_numpy(inputs.uniform(451, (50, 16)).astype(np.float32)).cuda()
    cfg = api.ModelConfig(nL, H, True, "fp32")
    s0, lp0 = api.sample2d(theta, u, cfg, Lx, Ly)
    api.set_autotune(True)
    try:
        s1, lp1 = api.sample2d(theta, u, cfg, Lx, Ly)
    finally:
        api.set_autotune(False)
    api.sync()
    assert torch.equal(s0, s1) and torch.equal(lp0, lp1)


@pytest.mark.parametrize("Lx,Ly,H,nL,u1", [(6, 6, 32, 3, True), (8, 4, 64, 2, False),
                                           (4, 8, 32, 1, False), (6, 4, 128, 3, True),
                                           (18, 4, 32, 2, True), (34, 2, 32, 1, False),
                                           (32, 4, 32, 1, True), (56, 2, 32, 1, False)])
def test_gradient_matches_oracle_finite_differences(oracle_mod, Lx, Ly, H, nL, u1):
    """Per-sample O_k against central differences of the FP64 oracle's
    log psi: 80 sampled components (|dO_k| <= 1e-3 max|O|) and 3 random
    directions (|dO.d| <= 1e-3 ||O|| ||d||)."""
    theta = _theta(oracle_mod, nL, H, seed=460 + H + Lx, scale=2.0)
    th64 = theta.astype(np.float64)
    n = 3
    s = _spins(461, n, Lx, Ly, u1)
    cfg = api.ModelConfig(nL, H, u1, "fp32")
    ok = api.grad2d(torch.from_numpy(theta).cuda(), torch.from_numpy(s).cuda(), cfg, Lx, Ly)
    api.sync()
    ok = ok.cpu().numpy().astype(np.float64)
    P = theta.size
    rng = np.random.default_rng(462)
    eps = 1e-5

    def lp(t):
        return oracle_mod.logpsi2d(t, nL, H, Lx, Ly, s, u1=u1)

    for k in rng.choice(P, 80, replace=False):
        tp, tm = th64.copy(), th64.copy()
        tp[k] += eps
        tm[k] -= eps
        fd = (lp(tp) - lp(tm)) / (2 * eps)
        assert np.all(np.abs(ok[:, k] - fd) <= 1e-3 * np.max(np.abs(ok), axis=1) + 1e-6), k
    for _ in range(3):
        d = rng.standard_normal(P)
        fd = (lp(th64 + eps * d) - lp(th64 - eps * d)) / (2 * eps)
        assert np.all(np.abs(ok @ d - fd) <= 1e-3 * np.linalg.norm(ok, axis=1) * np.linalg.norm(d))


def test_gradient_weighted_sum_and_determinism(oracle_mod):
    Lx, Ly, H, nL = 6, 6, 64, 3
    theta = torch.from_numpy(_theta(oracle_mod, nL, H, seed=470, scale=2.0)).cuda()
    s = torch.from_numpy(_spins(471, 40, Lx, Ly, True)).cuda()
    cfg = api.ModelConfig(nL, H, True, "fp32")
    rows = api.grad2d(theta, s, cfg, Lx, Ly)
    w = torch.from_numpy(inputs.uniform(472, (40,)).astype(np.float32) - 0.5).cuda()
    tot = api.grad2d(theta, s, cfg, Lx, Ly, dout=w)
    tot2 = api.grad2d(theta, s, cfg, Lx, Ly, dout=w)
    rows2 = api.grad2d(theta, s, cfg, Lx, Ly)
    api.sync()
    ref = (w[:, None].double() * rows.double()).sum(0)
    assert torch.allclose(tot.double(), ref, rtol=1e-4, atol=1e-5 * ref.abs().max().item())
    assert torch.equal(tot, tot2) and torch.equal(rows, rows2)
