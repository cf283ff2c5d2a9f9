"""GPU exact autoregressive sampler (psr_sample) against the FP64 oracle.

Sampling turns floating point into integers (s_t = 1 iff u_t < P(up)), and
the GPU evaluates P(up) in FP32 (or, at BF16 precision, from the BF16 model
on the tensor cores) while the oracle uses FP64, so a uniform that falls
within the GPU's error of P(up) may legitimately go either way.  The check
is therefore on validity: the oracle evaluates its own conditionals on the
GPU's sample (same prefix); a site may carry a decision other than the
oracle's only when its uniform lies within `band` of the oracle's P(up), and
such sites must be rare.  log psi of the drawn sample is compared with the
oracle's at the path's tolerance (FP32, or the BF16 bound).
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


def _draw(theta_np, u_np, cfg):
    theta = torch.from_numpy(theta_np).cuda()
    u = torch.from_numpy(u_np).cuda()
    s, lp = api.sample(theta, u, cfg)
    api.sync()
    return s.cpu().numpy(), lp.cpu().numpy().astype(np.float64)


def _check_valid(orc, theta_np, cfg, u_np, s, lp, band, rows=None):
    rows = range(s.shape[0]) if rows is None else rows
    s = s[list(rows)]
    u = u_np[list(rows)].astype(np.float64)
    lp = lp[list(rows)]
    ref, lps = orc.logpsi(theta_np, cfg.n_layers, cfg.hidden, s, u1=cfg.u1, per_site=True)
    assert np.all(np.isfinite(lps)), "a sample left the support (mask violated)"
    p_actual = np.exp(lps)
    p_up = np.where(s == 1, p_actual, 1.0 - p_actual)
    decided = (u < p_up).astype(np.uint8)
    differ = s != decided
    # every decision that differs from the oracle's is a near-tie ...
    assert np.all(np.abs(u - p_up)[differ] <= band), np.abs(u - p_up)[differ].max()
    # ... and such ties are rare (the GPU's error of P(up) is far below band)
    assert int(differ.sum()) <= max(2, 1e-3 * s.size), int(differ.sum())
    tol = (1e-5 + 1e-6 * np.abs(ref)) if cfg.precision == "fp32" else (2e-2 + 2e-5 * np.abs(ref))
    assert np.all(np.abs(lp - ref) <= tol), np.max(np.abs(lp - ref))
    return int(differ.sum())


@pytest.mark.parametrize("n_layers,H,N,u1,precision", [
    (3, 32, 16, False, "fp32"),     # 16-site chain, hidden 32
    (3, 64, 100, True, "fp32"),     # 100-site chain with zero magnetisation
    (3, 128, 100, True, "bf16"),    # 10x10 lattice size, hidden 128 (tensor-core sampler)
    (2, 32, 37, False, "fp32"),     # odd length, two layers
])
def test_samples_follow_oracle_conditionals(oracle_mod, n_layers, H, N, u1, precision):
    theta = inputs.random_params(n_layers, H, seed=60 + H, scale=1.0)
    n = 300
    u = inputs.uniform(61 + N, (n, N)).astype(np.float32)
    cfg = api.ModelConfig(n_layers, H, u1, precision)
    s, lp = _draw(theta, u, cfg)
    if u1:
        assert np.all(s.sum(axis=1) == N // 2)
    _check_valid(oracle_mod, theta, cfg, u, s, lp, band=1e-4 if precision == "fp32" else 1e-3)
    # nearly every sample is the oracle's own draw from the same uniforms
    s_orc, _ = oracle_mod.sample(theta, n_layers, H, N, u.astype(np.float64), u1=u1)
    same = np.mean(np.all(s == s_orc, axis=1))
    assert same >= 0.95, same


def test_frequencies_chi2(oracle_mod):
    from scipy.stats import chi2
    n_layers, H, N, n = 2, 32, 6, 40000
    theta = inputs.random_params(n_layers, H, seed=70, scale=1.5)
    u = inputs.uniform(71, (n, N)).astype(np.float32)
    s, _ = _draw(theta, u, api.ModelConfig(n_layers, H, False, "fp32"))
    cfg = ((np.arange(2 ** N)[:, None] >> (N - 1 - np.arange(N))[None, :]) & 1).astype(np.uint8)
    p = np.exp(2 * oracle_mod.logpsi(theta, n_layers, H, cfg))
    idx = (s.astype(np.int64) << (N - 1 - np.arange(N))).sum(axis=1)
    obs = np.bincount(idx, minlength=2 ** N)
    stat = np.sum((obs - p * n) ** 2 / (p * n))
    assert chi2.sf(stat, df=2 ** N - 1) > 1e-4


def test_tc_sampler_does_not_depend_on_the_grouping():
    """BF16 (the tensor-core sampler, blocks of 32 samples spread over the
    CTAs): the rows drawn from the same uniforms are identical whether 32,
    1000 or 9000 samples are drawn."""
    theta = torch.from_numpy(inputs.glorot_params(3, 128, seed=0)).cuda()
    u = torch.from_numpy(inputs.uniform(77, (9000, 64)).astype(np.float32)).cuda()
    cfg = api.ModelConfig(3, 128, True, "bf16")
    outs = [api.sample(theta, u[:n].contiguous(), cfg) for n in (32, 1000, 9000)]
    api.sync()
    for s_, lp_ in outs[1:]:
        assert torch.equal(s_[:32], outs[0][0]) and torch.equal(lp_[:32], outs[0][1])
    assert torch.equal(outs[1][0], outs[2][0][:1000]) and torch.equal(outs[1][1], outs[2][1][:1000])
    assert torch.all(outs[2][0].sum(dim=1) == 32)


def test_tuned_tile_draws_identical_samples():
    theta = torch.from_numpy(inputs.glorot_params(3, 128, seed=0)).cuda()
    n, N = 200, 64
    u = torch.from_numpy(inputs.uniform(72, (n, N)).astype(np.float32)).cuda()
    cfg = api.ModelConfig(3, 128, True, "fp32")
    s0, lp0 = api.sample(theta, u, cfg)
    api.sync()
    ctx = B.context()
    assert B.psr_sample_tile_for(ctx, n, N, 3, 128) == (8, False)
    api.set_autotune(True)
    try:
        s1, lp1 = api.sample(theta, u, cfg)
        api.sync()
    finally:
        api.set_autotune(False)
    per, tuned = B.psr_sample_tile_for(ctx, n, N, 3, 128)
    assert tuned and per in (4, 8, 16, 32)
    assert torch.equal(s0, s1) and torch.equal(lp0, lp1)


def test_host_arrays_and_bad_arguments(oracle_mod):
    theta = inputs.random_params(3, 32, seed=73, scale=1.0)
    u = inputs.uniform(74, (10, 20)).astype(np.float32)
    s = np.empty((10, 20), dtype=np.uint8)
    lp = np.empty(10, dtype=np.float32)
    p = B.make_params(theta, 3, 32, False, "fp32")
    B.psr_sample(p, u, s, lp)
    _check_valid(oracle_mod, theta, api.ModelConfig(3, 32, False, "fp32"), u, s,
                 lp.astype(np.float64), band=1e-4)
    with pytest.raises(B.PsrError) as ei:  # odd length with the zero-magnetisation mask
        B.psr_sample(B.make_params(theta, 3, 32, True, "fp32"), u[:, :19].copy(), s[:, :19].copy())
    assert ei.value.code == B.PSR_EINVAL


def test_52x52_sampled_rows(oracle_mod):
    """The 52x52 configuration (hidden 128, 3 layers, zero magnetisation),
    256 samples; oracle validity on 4 sampled rows of 2704 sites."""
    Lx = Ly = 52
    N = Lx * Ly
    theta = inputs.glorot_params(3, 128, seed=0)
    n = 256
    u = inputs.uniform(75, (n, N)).astype(np.float32)
    cfg = api.ModelConfig(3, 128, True, "bf16")
    s, lp = _draw(theta, u, cfg)
    assert np.all(s.sum(axis=1) == N // 2)
    _check_valid(oracle_mod, theta, cfg, u, s, lp, band=1e-3, rows=[0, 77, 190, 255])
