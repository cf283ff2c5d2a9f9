"""Exact sampler, reverse-mode gradient and on-device VMC step of the deep
1D LRU ansatz (psr_lru_sample, psr_lru_grad, psr_lru_vmc_step) against the
FP64 oracle of the same model.

Sampler: validity against the oracle's conditionals on the drawn sample
(a decision may differ from the oracle's only within `band` of P(up), and
rarely), log psi at the FP32 tolerance, and identical samples however the
samples are grouped into CTAs.  Gradient: per-sample O_k against central
differences of the oracle's FP64 log psi (sampled components within 1e-3 of
max|O|, random directions within 1e-3 ||O|| ||d||).  VMC step: E_loc at the
E_loc tolerance; the energy gradient element by element (largest and random
components) and along random directions against central differences of the
oracle's FP64 log psi weighted by the oracle's centred E_loc (1e-3); Adam.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from fdcheck import check_energy_gradient  # noqa: E402
from oracle import vmc  # noqa: E402
from paper_2605_13807_gb300 import api, binding as B, inputs  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    yield


def _theta(oracle_mod, nL, H, seed, kind):
    P = oracle_mod.param_count_lru(nL, H)
    if kind == "ring":
        th = inputs.lru_params(nL, H, seed=seed)
    else:  # every entry random (biases, nu, theta and gamma included)
        th = ((2.0 * inputs.uniform(seed, (P,)) - 1.0) * 2.0 / np.sqrt(H)).astype(np.float32)
    assert th.size == P
    return th


def _spins(seed, n, N, u1):
    return inputs.zero_magnetisation_spins(seed, n, N) if u1 else inputs.random_spins(seed, n, N)


# ------------------------------------------------------------------ sampler

@pytest.mark.parametrize("N,H,nL,u1,kind", [(16, 32, 3, False, "random"), (100, 64, 3, True, "ring"),
                                            (37, 128, 2, False, "random"), (64, 32, 1, True, "random")])
def test_samples_follow_oracle_conditionals(oracle_mod, N, H, nL, u1, kind):
    theta = _theta(oracle_mod, nL, H, 700 + N + H, kind)
    n = 200
    u = inputs.uniform(701 + N, (n, N)).astype(np.float32)
    cfg = api.ModelConfig(nL, H, u1, "fp32")
    s, lp = api.sample_lru(torch.from_numpy(theta).cuda(), torch.from_numpy(u).cuda(), cfg)
    api.sync()
    s = s.cpu().numpy()
    lp = lp.cpu().numpy().astype(np.float64)
    if u1:
        assert np.all(s.sum(axis=1) == N // 2)
    ref, lps = oracle_mod.logpsi_lru(theta.astype(np.float64), nL, H, s, u1=u1, per_site=True)
    assert np.all(np.isfinite(lps)), "a sample left the support (mask violated)"
    p_actual = np.exp(lps)
    p_up = np.where(s == 1, p_actual, 1.0 - p_actual)
    differ = s != (u.astype(np.float64) < p_up).astype(np.uint8)
    assert np.all(np.abs(u - p_up)[differ] <= 1e-4)
    assert int(differ.sum()) <= max(2, 1e-3 * s.size)
    assert np.all(np.abs(lp - ref) <= 1e-5 + 1e-6 * np.abs(ref)), np.max(np.abs(lp - ref))
    s_orc, lp_orc = oracle_mod.sample_lru(theta, nL, H, N, u.astype(np.float64), u1=u1)
    assert np.mean(np.all(s == s_orc, axis=1)) >= 0.95


def test_samples_do_not_depend_on_the_cta_grouping():
    """n = 64, 1280 and 2560 run 4, 8 and 16 samples per CTA on a 152-SM
    part; the rows drawn from the same uniforms must be identical."""
    nL, H, N = 3, 64, 48
    theta = torch.from_numpy(inputs.lru_params(nL, H, seed=710)).cuda()
    u = torch.from_numpy(inputs.uniform(711, (2560, N)).astype(np.float32)).cuda()
    cfg = api.ModelConfig(nL, H, False, "fp32")
    outs = [api.sample_lru(theta, u[:n].contiguous(), cfg) for n in (64, 1280, 2560)]
    api.sync()
    for s, lp in outs[1:]:
        assert torch.equal(s[:64], outs[0][0]) and torch.equal(lp[:64], outs[0][1])
    assert torch.equal(outs[1][0], outs[2][0][:1280])
    # the autotuner's measured choice draws the same samples
    api.set_autotune(True)
    try:
        s_t, lp_t = api.sample_lru(theta, u[:1280].contiguous(), cfg)
        s_t2, _ = api.sample_lru(theta, u[:1280].contiguous(), cfg)  # cached choice
    finally:
        api.set_autotune(False)
    api.sync()
    assert torch.equal(s_t, outs[1][0]) and torch.equal(lp_t, outs[1][1]) and torch.equal(s_t2, s_t)


def test_sampler_frequencies_chi2(oracle_mod):
    from scipy.stats import chi2
    nL, H, N, n = 2, 32, 6, 40000
    theta = _theta(oracle_mod, nL, H, 720, "random")
    u = torch.from_numpy(inputs.uniform(721, (n, N)).astype(np.float32)).cuda()
    s, _ = api.sample_lru(torch.from_numpy(theta).cuda(), u, api.ModelConfig(nL, H, False, "fp32"))
    api.sync()
    s = s.cpu().numpy()
    cfg = ((np.arange(2 ** N)[:, None] >> (N - 1 - np.arange(N))[None, :]) & 1).astype(np.uint8)
    p = np.exp(2 * oracle_mod.logpsi_lru(theta.astype(np.float64), nL, H, cfg))
    assert abs(p.sum() - 1.0) < 1e-9
    idx = (s.astype(np.int64) << (N - 1 - np.arange(N))).sum(axis=1)
    obs = np.bincount(idx, minlength=2 ** N)
    stat = np.sum((obs - p * n) ** 2 / (p * n))
    assert chi2.sf(stat, df=2 ** N - 1) > 1e-4


# ------------------------------------------------------------------ gradient

@pytest.mark.parametrize("N,H,nL,u1,kind", [(16, 32, 3, False, "random"), (40, 32, 3, True, "ring"),
                                            (64, 64, 2, False, "random"), (38, 128, 2, True, "random"),
                                            (100, 32, 1, False, "ring")])
def test_gradient_matches_oracle_finite_differences(oracle_mod, N, H, nL, u1, kind):
    theta = _theta(oracle_mod, nL, H, 730 + N + H, kind)
    th64 = theta.astype(np.float64)
    n = 3
    s = _spins(731, n, N, u1)
    cfg = api.ModelConfig(nL, H, u1, "fp32")
    ok = api.grad_lru(torch.from_numpy(theta).cuda(), torch.from_numpy(s).cuda(), cfg)
    api.sync()
    ok = ok.cpu().numpy().astype(np.float64)
    P = theta.size
    assert ok.shape == (n, P)
    rng = np.random.default_rng(732)
    eps = 1e-5

    def lp(t):
        return oracle_mod.logpsi_lru(t, nL, H, s, u1=u1)

    # every tensor's first entries, then random components
    shapes = inputs.param_shapes_lru(nL, H)
    starts = np.cumsum([0] + [int(np.prod(sh)) for _, sh in shapes])[:-1]
    comps = np.concatenate([starts, rng.choice(P, 60, replace=False)])
    for k in comps:
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
    nL, H, N, n = 3, 64, 70, 300
    theta = torch.from_numpy(_theta(oracle_mod, nL, H, 740, "ring")).cuda()
    s = torch.from_numpy(_spins(741, n, N, True)).cuda()
    cfg = api.ModelConfig(nL, H, True, "fp32")
    rows = api.grad_lru(theta, s, cfg)
    w = torch.from_numpy(inputs.uniform(742, (n,)).astype(np.float32) - 0.5).cuda()
    tot = api.grad_lru(theta, s, cfg, dout=w)
    tot2 = api.grad_lru(theta, s, cfg, dout=w)
    rows2 = api.grad_lru(theta, s, cfg)
    api.sync()
    ref = (w[:, None].double() * rows.double()).sum(0)
    assert torch.allclose(tot.double(), ref, rtol=1e-4, atol=1e-5 * ref.abs().max().item())
    # samples go to CTAs in a fixed order and every address has one writer
    assert torch.equal(rows, rows2) and torch.equal(tot, tot2)


def test_gradient_of_host_arrays_equals_device_result(oracle_mod):
    nL, H, N, n = 2, 32, 20, 5
    theta = _theta(oracle_mod, nL, H, 750, "random")
    s = _spins(751, n, N, False)
    p_host = B.make_params(theta, nL, H, False, "fp32", api._ctx())
    g_host = np.empty((n, theta.size), dtype=np.float32)
    B.psr_lru_grad(p_host, s, None, g_host)
    g_dev = api.grad_lru(torch.from_numpy(theta).cuda(), torch.from_numpy(s).cuda(),
                         api.ModelConfig(nL, H, False, "fp32"))
    api.sync()
    assert np.array_equal(g_host, g_dev.cpu().numpy())


# ------------------------------------------------------------------ VMC step

@pytest.mark.parametrize("kind,N,u1,hf", [(1, 16, False, 1.0), (0, 20, True, 0.0)])
def test_vmc_step_matches_oracle(oracle_mod, kind, N, u1, hf):
    nL, H, n = 3, 32, 64
    theta = _theta(oracle_mod, nL, H, 760 + N, "ring")
    th = torch.from_numpy(theta).cuda()
    ham = B.make_hamiltonian(kind, N, 1, False, True, 1.0, hf)
    cfg = api.ModelConfig(nL, H, u1, "fp32")
    u = torch.from_numpy(inputs.uniform(761, (n, N)).astype(np.float32)).cuda()
    adam = api.Adam(theta.size, "cuda", lr=1e-2)
    out = api.vmc_step_lru(th, cfg, ham, u, adam)
    api.sync()
    s = out["spins"].cpu().numpy()
    if u1:
        assert np.all(s.sum(axis=1) == N // 2)
    s_ref, _ = api.sample_lru(th, u, cfg)
    api.sync()
    assert np.array_equal(s, s_ref.cpu().numpy())
    e = out["eloc"].cpu().numpy().astype(np.float64)
    ref_e = oracle_mod.local_energy_lru(theta.astype(np.float64), nL, H, s, kind, N, 1, pbc=False,
                                        marshall=True, J=1.0, h=hf, u1=u1)
    _, _, diag = oracle_mod.connected(kind, N, 1, False, s)
    assert np.all(np.abs(e - ref_e) <= 1e-3 * (np.abs(diag) + np.abs(ref_e - diag)))
    m, _, _ = oracle_mod.stats(e)
    assert abs(out["stats"][0].item() - m) <= 1e-9 * max(1.0, abs(m))
    # energy gradient against the oracle alone: central differences of its
    # FP64 log psi weighted by its own centred E_loc
    g = out["grad"].cpu().numpy().astype(np.float64)
    th64 = theta.astype(np.float64)
    check_energy_gradient(g, lambda t: oracle_mod.logpsi_lru(t, nL, H, s, u1=u1), th64, ref_e,
                          seed=762 + N)
    t1, m1, v1 = vmc.adam(theta, g, np.zeros_like(g), np.zeros_like(g), 1, 1e-2)
    assert np.max(np.abs(out["theta"].cpu().numpy() - t1)) <= 1e-6 + 1e-6 * np.max(np.abs(t1))
    # a second step from the updated parameters carries the Adam moments
    th2 = out["theta"].clone()
    out2 = api.vmc_step_lru(th2, cfg, ham, u, adam)
    api.sync()
    g2 = out2["grad"].cpu().numpy().astype(np.float64)
    t2, _, _ = vmc.adam(th2.cpu().numpy(), g2, m1, v1, 2, 1e-2)
    assert np.max(np.abs(out2["theta"].cpu().numpy() - t2)) <= 1e-5


def test_rejections():
    nL, H, N = 3, 32, 16
    theta = torch.zeros(api.param_count_lru(nL, H), device="cuda")
    cfg = api.ModelConfig(nL, H, False, "fp32")
    ham = B.make_hamiltonian("tfim", N, 1, False, True, 1.0, 1.0)
    adam = api.Adam(theta.numel(), "cuda")
    adam.step = 1
    p = B.make_params(theta, nL, H)
    u_host = inputs.uniform(770, (8, N)).astype(np.float32)
    with pytest.raises(B.PsrError) as ei:  # the VMC step takes device arrays only
        B.psr_lru_vmc_step(p, ham, u_host, adam.state(), torch.empty_like(theta))
    assert ei.value.code == B.PSR_EINVAL
    with pytest.raises(B.PsrError) as ei:  # odd length with the zero-magnetisation mask
        api.sample_lru(theta, torch.zeros((4, 9), device="cuda"), api.ModelConfig(nL, H, True, "fp32"))
    assert ei.value.code == B.PSR_EINVAL
    with pytest.raises(B.PsrError) as ei:  # BF16 is not a precision of this model
        api.grad_lru(theta, torch.zeros((4, N), dtype=torch.uint8, device="cuda"),
                     api.ModelConfig(nL, H, False, "bf16"))
    assert ei.value.code == B.PSR_EUNSUPPORTED
    # spin bytes other than 0 / 1: reported by the next synchronisation
    api.grad_lru(theta, torch.full((4, N), 2, dtype=torch.uint8, device="cuda"), cfg)
    with pytest.raises(B.PsrError) as ei:
        api.sync()
    assert ei.value.code == B.PSR_EDEVICE
    api.sync()  # cleared
