"""The 2D patched minGRU at the paper's 2D configuration: c4v-symmetrised
log psi and E_loc (psr2d_sym_logpsi, psr2d_sym_local_energy), the gradient
at hidden 256 and the symmetrised on-device VMC step (psr2d_vmc_step with
symmetrize), against the FP64 oracle of the 2D model composed with the
oracle's c4v symmetrisation (oracle/vmc.py).

Tolerances: log psi FP32 1e-5 + 1e-6 |log psi|; E_loc 1e-3 of
|diag| + |E_loc - diag|; O_k against central differences of the oracle's
FP64 log psi (sampled components within 1e-3 of max|O|, random directions
within 1e-3 ||O|| ||d||); the step's gradient element by element (largest
and random components, 1e-3 of the largest) and along random directions
against central differences of the oracle's symmetrised FP64 log psi
weighted by the oracle's centred E_loc.
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


def _theta(oracle_mod, nL, H, seed, scale=2.0):
    P = oracle_mod.param_count2d(nL, H)
    return ((2.0 * inputs.uniform(seed, (P,)) - 1.0) * scale / np.sqrt(H)).astype(np.float32)


def _spins(seed, n, N, u1):
    return inputs.zero_magnetisation_spins(seed, n, N) if u1 else inputs.random_spins(seed, n, N)


@pytest.mark.parametrize("L,H,nL,u1", [(4, 32, 3, True), (6, 64, 2, False), (4, 256, 3, True)])
def test_sym_logpsi2d_matches_oracle(oracle_mod, L, H, nL, u1):
    theta = _theta(oracle_mod, nL, H, 900 + L + H)
    s = _spins(901, 12, L * L, u1)
    cfg = api.ModelConfig(nL, H, u1, "fp32")
    got = api.sym_logpsi2d(torch.from_numpy(theta).cuda(), torch.from_numpy(s).cuda(), cfg, L)
    api.sync()
    th64 = theta.astype(np.float64)
    ref = vmc.logpsi_sym(lambda x: oracle_mod.logpsi2d(th64, nL, H, L, L, x, u1=u1), s, L)
    got = got.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - ref) <= 1e-5 + 1e-6 * np.abs(ref)), np.max(np.abs(got - ref))
    # invariance: every image of a configuration has the same psi_sym
    imgs = vmc.c4v_images(s, L)
    for g in (1, 6):
        gi = api.sym_logpsi2d(torch.from_numpy(theta).cuda(),
                              torch.from_numpy(np.ascontiguousarray(imgs[g])).cuda(), cfg, L)
        api.sync()
        assert np.all(np.abs(gi.cpu().numpy() - got) <= 2e-5 + 2e-6 * np.abs(ref))


@pytest.mark.parametrize("kind,L,H,u1,hf", [(0, 4, 32, True, 0.0), (1, 4, 32, False, 3.044),
                                            (0, 6, 64, True, 0.0)])
def test_sym_local_energy2d_matches_oracle(oracle_mod, kind, L, H, u1, hf):
    nL = 3
    theta = _theta(oracle_mod, nL, H, 910 + L + kind)
    n = 6
    s = inputs.neel_like_spins(911, n, L, L) if kind == 0 else inputs.random_spins(911, n, L * L)
    ham = B.make_hamiltonian(kind, L, L, False, True, 1.0, hf)
    e, st = api.sym_local_energy2d(torch.from_numpy(theta).cuda(), torch.from_numpy(s).cuda(),
                                   api.ModelConfig(nL, H, u1, "fp32"), ham)
    api.sync()
    th64 = theta.astype(np.float64)
    ref = vmc.local_energy_sym(lambda x: oracle_mod.logpsi2d(th64, nL, H, L, L, x, u1=u1), s, kind, L,
                               marshall=True, J=1.0, h=hf)
    _, _, diag = oracle_mod.connected(kind, L, L, False, s)
    scale = np.abs(diag) + np.abs(ref - diag)
    assert np.all(np.abs(e.cpu().numpy() - ref) <= 1e-3 * scale)
    m, _, _ = oracle_mod.stats(e.cpu().numpy().astype(np.float64))
    assert abs(st[0].item() - m) <= 1e-9 * max(1.0, abs(m))


def test_sym_rejects_rectangular_lattices(oracle_mod):
    theta = torch.from_numpy(_theta(oracle_mod, 3, 32, 920)).cuda()
    s = torch.zeros((2, 24), dtype=torch.uint8, device="cuda")
    with pytest.raises(B.PsrError) as ei:
        B.psr2d_sym_logpsi(B.make_params(theta, 3, 32), s, 6, 4, torch.empty(2, device="cuda"))
    assert ei.value.code == B.PSR_EINVAL


@pytest.mark.parametrize("L,nL,u1", [(4, 3, True), (6, 2, False)])
def test_gradient_at_hidden_256_matches_oracle_finite_differences(oracle_mod, L, nL, u1):
    H = 256
    theta = _theta(oracle_mod, nL, H, 930 + L)
    th64 = theta.astype(np.float64)
    n = 2
    s = _spins(931, n, L * L, u1)
    cfg = api.ModelConfig(nL, H, u1, "fp32")
    ok = api.grad2d(torch.from_numpy(theta).cuda(), torch.from_numpy(s).cuda(), cfg, L, L)
    api.sync()
    ok = ok.cpu().numpy().astype(np.float64)
    P = theta.size
    rng = np.random.default_rng(932)
    eps = 1e-5

    def lp(t):
        return oracle_mod.logpsi2d(t, nL, H, L, L, s, u1=u1)

    for k in rng.choice(P, 60, replace=False):
        tp, tm = th64.copy(), th64.copy()
        tp[k] += eps
        tm[k] -= eps
        fd = (lp(tp) - lp(tm)) / (2 * eps)
        assert np.all(np.abs(ok[:, k] - fd) <= 1e-3 * np.max(np.abs(ok), axis=1) + 1e-6), k
    for _ in range(2):
        d = rng.standard_normal(P)
        fd = (lp(th64 + eps * d) - lp(th64 - eps * d)) / (2 * eps)
        assert np.all(np.abs(ok @ d - fd) <= 1e-3 * np.linalg.norm(ok, axis=1) * np.linalg.norm(d))


def test_gradient_at_hidden_256_weighted_sum(oracle_mod):
    L, nL, H, n = 6, 3, 256, 20
    theta = torch.from_numpy(_theta(oracle_mod, nL, H, 940)).cuda()
    s = torch.from_numpy(_spins(941, n, L * L, True)).cuda()
    cfg = api.ModelConfig(nL, H, True, "fp32")
    rows = api.grad2d(theta, s, cfg, L, L)
    w = torch.from_numpy(inputs.uniform(942, (n,)).astype(np.float32) - 0.5).cuda()
    tot = api.grad2d(theta, s, cfg, L, L, dout=w)
    api.sync()
    ref = (w[:, None].double() * rows.double()).sum(0)
    assert torch.allclose(tot.double(), ref, rtol=1e-4, atol=1e-5 * ref.abs().max().item())


def test_symmetrised_vmc_step_of_the_2d_model(oracle_mod):
    L, nL, H, n = 4, 3, 32, 32
    N, Np = L * L, (L // 2) * (L // 2)
    theta = _theta(oracle_mod, nL, H, 950)
    th = torch.from_numpy(theta).cuda()
    ham = B.make_hamiltonian("heisenberg", L, L, False, True, 1.0, 0.0)
    cfg = api.ModelConfig(nL, H, True, "fp32")
    u = torch.from_numpy(inputs.uniform(951, (n, Np)).astype(np.float32)).cuda()
    us = torch.from_numpy(inputs.uniform(952, (n,)).astype(np.float32)).cuda()
    adam = api.Adam(theta.size, "cuda", lr=1e-2)
    out = api.vmc_step2d(th, cfg, ham, u, adam, symmetrize=True, sym_uniforms=us)
    api.sync()
    s = out["spins"].cpu().numpy()
    assert np.all(s.sum(axis=1) == N // 2)
    # the samples are the sampler's draws mapped by the chosen images
    s0, _ = api.sample2d(th, u, cfg, L, L)
    api.sync()
    imgs0 = vmc.c4v_images(s0.cpu().numpy(), L)
    g = np.minimum(7, np.floor(8 * us.cpu().numpy()).astype(int))
    assert np.array_equal(s, imgs0[g, np.arange(n)])
    th64 = theta.astype(np.float64)

    def lp(x):
        return oracle_mod.logpsi2d(th64, nL, H, L, L, x, u1=True)

    e = out["eloc"].cpu().numpy().astype(np.float64)
    ref_e = vmc.local_energy_sym(lp, s, 0, L, marshall=True, J=1.0, h=0.0)
    _, _, diag = oracle_mod.connected(0, L, L, False, s)
    assert np.all(np.abs(e - ref_e) <= 1e-3 * (np.abs(diag) + np.abs(ref_e - diag)))
    # energy gradient against the oracle alone: central differences of the
    # oracle's symmetrised FP64 log psi (its own image weighting) weighted by
    # the oracle's centred E_loc
    grad = out["grad"].cpu().numpy().astype(np.float64)
    check_energy_gradient(grad, lambda t: vmc.logpsi_sym(
        lambda x: oracle_mod.logpsi2d(t, nL, H, L, L, x, u1=True), s, L), th64, ref_e, seed=953)
    t1, _, _ = vmc.adam(theta, grad, np.zeros(theta.size), np.zeros(theta.size), 1, 1e-2)
    assert np.max(np.abs(out["theta"].cpu().numpy() - t1)) <= 1e-6 + 1e-6 * np.max(np.abs(t1))


def test_sym_local_energy2d_host_arrays_equal_device_result(oracle_mod):
    L, nL, H = 4, 2, 32
    theta = _theta(oracle_mod, nL, H, 960)
    s = inputs.neel_like_spins(961, 5, L, L)
    ham = B.make_hamiltonian("heisenberg", L, L, False, True, 1.0, 0.0)
    p_host = B.make_params(theta, nL, H, True, "fp32", api._ctx())
    e_host = np.empty(5, dtype=np.float32)
    st_host = np.empty(3, dtype=np.float64)
    B.psr2d_sym_local_energy(p_host, s, ham, e_host, st_host)
    e_dev, st_dev = api.sym_local_energy2d(torch.from_numpy(theta).cuda(), torch.from_numpy(s).cuda(),
                                           api.ModelConfig(nL, H, True, "fp32"), ham)
    api.sync()
    assert np.array_equal(e_host, e_dev.cpu().numpy())
    assert np.array_equal(st_host, st_dev.cpu().numpy())


def test_vmc_step2d_rejections(oracle_mod):
    L, nL, H = 4, 2, 32
    theta = torch.from_numpy(_theta(oracle_mod, nL, H, 970)).cuda()
    p = B.make_params(theta, nL, H, True, "fp32")
    adam = api.Adam(theta.numel(), "cuda")
    adam.step = 1
    out = torch.empty_like(theta)
    u = torch.zeros((8, 4), device="cuda")
    us = torch.zeros(8, device="cuda")
    rect = B.make_hamiltonian("heisenberg", 4, 8, False, True, 1.0, 0.0)
    with pytest.raises(B.PsrError) as ei:  # c4v needs a square lattice
        B.psr2d_vmc_step(p, rect, True, torch.zeros((8, 8), device="cuda"), us, adam.state(), out)
    assert ei.value.code == B.PSR_EINVAL
    sq = B.make_hamiltonian("heisenberg", L, L, False, True, 1.0, 0.0)
    with pytest.raises(B.PsrError) as ei:  # symmetrize without its uniforms
        B.psr2d_vmc_step(p, sq, True, u, None, adam.state(), out)
    assert ei.value.code == B.PSR_EINVAL
    with pytest.raises(B.PsrError) as ei:  # host uniforms
        B.psr2d_vmc_step(p, sq, False, u.cpu().numpy(), None, adam.state(), out)
    assert ei.value.code == B.PSR_EINVAL
