"""GPU deep 1D LRU on the tensor cores (precisions "fp16" and "bf16", hidden
64: psr_lru_logpsi and psr_lru_local_energy through lru_tc_kernel, 16-bit
operands with FP32 accumulation, complex scan, GLU and readout) against the
FP64 oracle of the same model (Sec. II.B Eq. lru, Sec. II.G, Sec. III.B).

Tolerances, the stated bounds of the 16-bit path:
  log psi : |d| <= 2e-2 + 2e-5 |log psi|
  E_loc   : |d| <= 1e-3 (|diag| + |E_loc - diag|)
FP16 operands meet both.  BF16 operands are held to twice the log psi bound
and three times the E_loc bound (2.1e-3 measured on the 256-site TFIM
chain): regression bounds, as for the 2D model's BF16 path.
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


H = 64


def _theta(oracle_mod, nL, seed, kind):
    P = oracle_mod.param_count_lru(nL, H)
    assert P == api.param_count_lru(nL, H)
    if kind == "ring":
        th = inputs.lru_params(nL, H, seed=seed)
    else:  # every entry random (biases, nu, theta and gamma included)
        th = ((2.0 * inputs.uniform(seed, (P,)) - 1.0) / np.sqrt(H)).astype(np.float32)
    return th


def _spins(seed, n, N, u1):
    return inputs.zero_magnetisation_spins(seed, n, N) if u1 else inputs.random_spins(seed, n, N)


@pytest.mark.parametrize("N,nL,u1,kind", [(16, 3, False, "random"), (100, 3, True, "ring"),
                                          (256, 3, False, "ring"), (37, 2, False, "random"),
                                          (70, 1, True, "random"), (34, 3, True, "ring")])
@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_logpsi_lru_tc_matches_oracle(oracle_mod, N, nL, u1, kind, prec):
    theta = _theta(oracle_mod, nL, 700 + N + nL, kind)
    s = _spins(701, 40, N, u1)
    cfg = api.ModelConfig(nL, H, u1, prec)
    got = api.logpsi_lru(torch.from_numpy(theta).cuda(), torch.from_numpy(s).cuda(), cfg)
    api.sync()
    ref = oracle_mod.logpsi_lru(theta.astype(np.float64), nL, H, s, u1=u1)
    got = got.cpu().numpy().astype(np.float64)
    scale = 1.0 if prec == "fp16" else 2.0
    assert np.all(np.isfinite(got) == np.isfinite(ref))
    fin = np.isfinite(ref)
    err = np.abs(got[fin] - ref[fin])
    assert np.all(err <= scale * (2e-2 + 2e-5 * np.abs(ref[fin]))), (err.max(), np.abs(ref).max())


@pytest.mark.parametrize("N,nL,u1", [(1, 3, False), (2, 3, True), (33, 2, False), (64, 4, True), (31, 4, False),
                                     (1000, 3, True)])
def test_logpsi_lru_tc_edge_sizes(oracle_mod, N, nL, u1):
    """Degenerate and boundary chains on the tensor-core path: a single site,
    the smallest zero-magnetisation chain, one site past a chunk, an exact
    multiple of the chunk, the deepest supported model (4 layers), and a
    1000-site chain (32 chunks, ragged last chunk)."""
    theta = _theta(oracle_mod, nL, 740 + N + nL, "random")
    s = _spins(741, 24, N, u1)
    ref = oracle_mod.logpsi_lru(theta.astype(np.float64), nL, H, s, u1=u1)
    for prec, scale in (("fp16", 1.0), ("bf16", 2.0)):
        got = api.logpsi_lru(torch.from_numpy(theta).cuda(), torch.from_numpy(s).cuda(),
                             api.ModelConfig(nL, H, u1, prec))
        api.sync()
        got = got.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(got) == np.isfinite(ref))
        fin = np.isfinite(ref)
        err = np.abs(got[fin] - ref[fin])
        assert np.all(err <= scale * (2e-2 + 2e-5 * np.abs(ref[fin]))), (prec, err.max())


@pytest.mark.parametrize("kind,N,pbc,u1,hf", [(1, 16, False, False, 1.0), (1, 16, True, False, 1.0),
                                              (0, 20, False, True, 0.0), (1, 256, False, False, 1.0),
                                              (0, 66, True, True, 0.0)])
@pytest.mark.parametrize("prec,tol", [("fp16", 1e-3), ("bf16", 3e-3)])
def test_local_energy_lru_tc_matches_oracle(oracle_mod, kind, N, pbc, u1, hf, prec, tol):
    nL = 3
    theta = _theta(oracle_mod, nL, 710 + N, "ring")
    n = 3 if N >= 256 else 12
    s = _spins(711, n, N, u1)
    ham = B.make_hamiltonian(kind, N, 1, pbc, True, 1.0, hf)
    cfg = api.ModelConfig(nL, H, u1, prec)
    e, st = api.local_energy_lru(torch.from_numpy(theta).cuda(), torch.from_numpy(s).cuda(), cfg, ham)
    api.sync()
    ref = oracle_mod.local_energy_lru(theta.astype(np.float64), nL, H, s, kind, N, 1, pbc=pbc,
                                      marshall=True, J=1.0, h=hf, u1=u1)
    _, _, diag = oracle_mod.connected(kind, N, 1, pbc, s)
    scale = np.abs(diag) + np.abs(ref - diag)
    err = np.abs(e.cpu().numpy() - ref)
    assert np.all(err <= tol * scale), (err / scale).max()
    m, _, _ = oracle_mod.stats(e.cpu().numpy().astype(np.float64))
    assert abs(st[0].item() - m) <= 1e-9 * max(1.0, abs(m))


def test_lru_tc_at_the_benchmark_size(oracle_mod):
    """The benchmark's LRU workload in its own launch shape (TFIM chain N =
    256, OBC, h = 1, 1024 samples, ring parameters seed 0, FP16 operands):
    log psi of every sample, and E_loc of sampled rows (first, middle, last),
    against the oracle."""
    N, nL, n = 256, 3, 1024
    theta = inputs.lru_params(nL, H, seed=0)
    s = inputs.random_spins(2000, n, N)
    ham = B.make_hamiltonian("tfim", N, 1, False, True, 1.0, 1.0)
    cfg = api.ModelConfig(nL, H, False, "fp16")
    th, sp = torch.from_numpy(theta).cuda(), torch.from_numpy(s).cuda()
    lp = api.logpsi_lru(th, sp, cfg)
    e, _ = api.local_energy_lru(th, sp, cfg, ham)
    api.sync()
    ref = oracle_mod.logpsi_lru(theta.astype(np.float64), nL, H, s, u1=False)
    err = np.abs(lp.cpu().numpy().astype(np.float64) - ref)
    assert np.all(err <= 2e-2 + 2e-5 * np.abs(ref)), err.max()
    pick = [0, n // 2, n - 1]
    sub = s[pick]
    eref = oracle_mod.local_energy_lru(theta.astype(np.float64), nL, H, sub, 1, N, 1, pbc=False, marshall=True,
                                       J=1.0, h=1.0, u1=False)
    _, _, diag = oracle_mod.connected(1, N, 1, False, sub)
    got = e.cpu().numpy()[pick]
    assert np.all(np.abs(got - eref) <= 1e-3 * (np.abs(diag) + np.abs(eref - diag))), (got, eref)


def test_lru_tc_many_jobs_and_determinism():
    """More sequences than the CTAs hold slots (8 per CTA), so slots take new
    jobs mid-launch; within the 16-bit bound of the (oracle-checked) FP32
    path, and two runs bitwise equal."""
    N, nL, n = 96, 3, 3000
    theta = torch.from_numpy(inputs.lru_params(nL, H, seed=4)).cuda()
    s = torch.from_numpy(_spins(721, n, N, True)).cuda()
    a = api.logpsi_lru(theta, s, api.ModelConfig(nL, H, True, "fp16"))
    b = api.logpsi_lru(theta, s, api.ModelConfig(nL, H, True, "fp16"))
    r = api.logpsi_lru(theta, s, api.ModelConfig(nL, H, True, "fp32"))
    api.sync()
    assert torch.equal(a, b)
    err = (a.double() - r.double()).abs()
    assert torch.all(err <= 2e-2 + 2e-5 * r.double().abs())


@pytest.mark.parametrize("N,nL,u1,kind", [(16, 3, False, "random"), (100, 3, True, "ring"), (37, 2, False, "random"),
                                          (64, 1, True, "random"), (256, 3, False, "ring")])
@pytest.mark.parametrize("prec,ptol,frac", [("fp16", 2e-3, 2e-3), ("bf16", 1e-2, 1e-2)])
def test_tc_sampler_follows_oracle_conditionals(oracle_mod, N, nL, u1, kind, prec, ptol, frac):
    """psr_lru_sample at 16-bit precision (the tensor-core sampler): every draw
    agrees with the oracle's conditional P(s_t = 1 | s_<t) at the drawn
    prefix, except where the uniform lies within ptol of it (the 16-bit
    model's conditionals differ from the exact ones by less); the zero-
    magnetisation mask holds; the returned log psi is the 16-bit forward's
    within its bound."""
    theta = _theta(oracle_mod, nL, 750 + N + nL, kind)
    n = 200
    u = inputs.uniform(751 + N, (n, N)).astype(np.float32)
    cfg = api.ModelConfig(nL, H, u1, prec)
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
    assert np.all(np.abs(u - p_up)[differ] <= ptol), np.abs(u - p_up)[differ].max()
    assert int(differ.sum()) <= max(2, frac * s.size)
    scale = 1.0 if prec == "fp16" else 2.0
    assert np.all(np.abs(lp - ref) <= scale * (2e-2 + 2e-5 * np.abs(ref))), np.max(np.abs(lp - ref))


def test_tc_sampler_does_not_depend_on_the_grouping():
    """Blocks of 32 samples, spread over the CTAs: the rows drawn from the
    same uniforms are identical whether 32, 1000 or 9000 samples are drawn
    (one block, 32 blocks, several blocks per CTA)."""
    nL, N = 3, 48
    theta = torch.from_numpy(inputs.lru_params(nL, H, seed=760)).cuda()
    u = torch.from_numpy(inputs.uniform(761, (9000, N)).astype(np.float32)).cuda()
    cfg = api.ModelConfig(nL, H, False, "fp16")
    outs = [api.sample_lru(theta, u[:n].contiguous(), cfg) for n in (32, 1000, 9000)]
    api.sync()
    for s_, lp_ in outs[1:]:
        assert torch.equal(s_[:32], outs[0][0]) and torch.equal(lp_[:32], outs[0][1])
    assert torch.equal(outs[1][0], outs[2][0][:1000]) and torch.equal(outs[1][1], outs[2][1][:1000])


def test_lru_vmc_step_fp16_local_energies(oracle_mod):
    """The LRU VMC step at precision fp16: samples from the tensor-core
    sampler, gradient FP32, local energies from the tensor-core forward,
    within the E_loc bound of the oracle; the samples are nearly all those
    the FP32 step draws from the same uniforms."""
    N, nL, n = 32, 3, 64
    theta = inputs.lru_params(nL, H, seed=5)
    ham = B.make_hamiltonian("tfim", N, 1, False, True, 1.0, 1.0)
    g = torch.Generator(device="cuda")
    g.manual_seed(9)
    u = torch.rand((n, N), generator=g, device="cuda")
    th = torch.from_numpy(theta).cuda()
    outs = {}
    for prec in ("fp32", "fp16"):
        adam = api.Adam(th.numel(), th.device, lr=1e-3)
        outs[prec] = api.vmc_step_lru(th, api.ModelConfig(nL, H, False, prec), ham, u, adam)
    api.sync()
    same = torch.all(outs["fp32"]["spins"] == outs["fp16"]["spins"], dim=1).float().mean().item()
    assert same >= 0.9, same
    s = outs["fp16"]["spins"].cpu().numpy()
    ref = oracle_mod.local_energy_lru(theta.astype(np.float64), nL, H, s, 1, N, 1, pbc=False, marshall=True,
                                      J=1.0, h=1.0, u1=False)
    _, _, diag = oracle_mod.connected(1, N, 1, False, s)
    e = outs["fp16"]["eloc"].cpu().numpy()
    assert np.all(np.abs(e - ref) <= 1e-3 * (np.abs(diag) + np.abs(ref - diag)))


def test_lru_tc_rejects_unsupported_shapes():
    """The 16-bit path holds hidden 64 and up to 4 layers; other shapes at
    fp16 or bf16 return PSR_EUNSUPPORTED (FP32 takes them)."""
    for nL, Hh in ((5, 64), (3, 128)):
        theta = torch.from_numpy(inputs.lru_params(nL, Hh, seed=1)).cuda()
        s = torch.from_numpy(_spins(731, 4, 16, False)).cuda()
        with pytest.raises(B.PsrError) as ei:
            api.logpsi_lru(theta, s, api.ModelConfig(nL, Hh, False, "fp16"))
        assert ei.value.code == B.PSR_EUNSUPPORTED
