"""c4v-symmetrised amplitudes and the on-device VMC step against the FP64
oracle (oracle/vmc.py).

Tolerances: log psi as the model's path (FP32 1e-5 + 1e-6 |log psi|, BF16
2e-2 + 2e-5 |log psi|); E_loc 1e-3 of |diag| + |E_loc - diag|; gradient
||dg|| <= 1e-3 ||g||; the Adam update is checked against the oracle's Adam
applied to the GPU's own gradient (FP32 rounding only).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import vmc  # noqa: E402
from paper_2605_13807_gb300 import api, binding as B, inputs  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    yield


def _params(nL, H, seed, precision):
    if precision == "bf16":
        return inputs.glorot_params(nL, H, seed=seed)
    return inputs.random_params(nL, H, seed=seed, scale=1.0)


@pytest.mark.parametrize("L,H,u1,precision", [(4, 32, True, "fp32"), (6, 64, False, "fp32"),
                                              (10, 128, True, "bf16")])
def test_sym_logpsi_matches_oracle(oracle_mod, L, H, u1, precision):
    nL = 3
    theta = _params(nL, H, 800 + L, precision)
    N = L * L
    s = inputs.zero_magnetisation_spins(801, 24, N) if u1 else inputs.random_spins(801, 24, N)
    got = api.sym_logpsi(torch.from_numpy(theta).cuda(), torch.from_numpy(s).cuda(),
                         api.ModelConfig(nL, H, u1, precision), L)
    api.sync()
    ref = vmc.logpsi_sym(lambda x: oracle_mod.logpsi(theta, nL, H, x, u1=u1), s, L)
    tol = (1e-5 + 1e-6 * np.abs(ref)) if precision == "fp32" else (2e-2 + 2e-5 * np.abs(ref))
    assert np.all(np.abs(got.cpu().numpy() - ref) <= tol)


@pytest.mark.parametrize("kind,L,H,u1,precision,hf", [(0, 4, 32, True, "fp32", 0.0),
                                                      (1, 4, 32, False, "fp32", 3.044),
                                                      (0, 6, 128, True, "bf16", 0.0)])
def test_sym_local_energy_matches_oracle(oracle_mod, kind, L, H, u1, precision, hf):
    nL = 3
    theta = _params(nL, H, 810 + L + kind, precision)
    N = L * L
    n = 8
    s = inputs.neel_like_spins(811, n, L, L) if kind == 0 else inputs.random_spins(811, n, N)
    ham = B.make_hamiltonian(kind, L, L, False, True, 1.0, hf)
    e, st = api.sym_local_energy(torch.from_numpy(theta).cuda(), torch.from_numpy(s).cuda(),
                                 api.ModelConfig(nL, H, u1, precision), ham)
    api.sync()
    ref = vmc.local_energy_sym(lambda x: oracle_mod.logpsi(theta, nL, H, x, u1=u1), s, kind, L,
                               marshall=True, J=1.0, h=hf)
    _, _, diag = oracle_mod.connected(kind, L, L, False, s)
    scale = np.abs(diag) + np.abs(ref - diag)
    assert np.all(np.abs(e.cpu().numpy() - ref) <= 1e-3 * scale)


def _check_step(oracle_mod, out, theta, nL, H, u1, kind, Lx, Ly, hf, sym, adam_lr):
    s = out["spins"].cpu().numpy()
    e = out["eloc"].cpu().numpy().astype(np.float64)
    g = out["grad"].cpu().numpy().astype(np.float64)
    if sym:
        def lp(x):
            return oracle_mod.logpsi(theta, nL, H, x, u1=u1)
        ref_e = vmc.local_energy_sym(lp, s, kind, Lx, marshall=True, J=1.0, h=hf)
        okl = vmc.grad_logpsi_sym(theta, nL, H, s, Lx, u1=u1)
    else:
        ref_e = oracle_mod.local_energy(theta, nL, H, s, kind, Lx, Ly, marshall=True, J=1.0, h=hf, u1=u1)
        _, okl = oracle_mod.grad(theta, nL, H, s, u1=u1)
    _, _, diag = oracle_mod.connected(kind, Lx, Ly, False, s)
    assert np.all(np.abs(e - ref_e) <= 1e-3 * (np.abs(diag) + np.abs(ref_e - diag)))
    st = out["stats"].cpu().numpy()
    m, v, se = oracle_mod.stats(e)
    assert abs(st[0] - m) <= 1e-9 * max(1.0, abs(m))
    ref_g, _ = vmc.energy_gradient(ref_e, okl)
    assert np.linalg.norm(g - ref_g) <= 1e-3 * np.linalg.norm(ref_g)
    return g


@pytest.mark.parametrize("sym", [False, True])
def test_vmc_step_matches_oracle(oracle_mod, sym):
    nL, H = 3, 32
    if sym:
        kind, Lx, Ly, u1, hf = 0, 4, 4, True, 0.0
    else:
        kind, Lx, Ly, u1, hf = 1, 16, 1, False, 1.0
    N = Lx * Ly
    n = 64
    theta = _params(nL, H, 820 + int(sym), "fp32")
    th = torch.from_numpy(theta).cuda()
    ham = B.make_hamiltonian(kind, Lx, Ly, False, True, 1.0, hf)
    cfg = api.ModelConfig(nL, H, u1, "fp32")
    u = torch.from_numpy(inputs.uniform(821, (n, N)).astype(np.float32)).cuda()
    us = torch.from_numpy(inputs.uniform(822, (n,)).astype(np.float32)).cuda() if sym else None
    adam = api.Adam(theta.size, "cuda", lr=1e-2)
    out = api.vmc_step(th, cfg, ham, u, adam, symmetrize=sym, sym_uniforms=us)
    api.sync()
    s = out["spins"].cpu().numpy()
    if u1:
        assert np.all(s.sum(axis=1) == N // 2)
    g = _check_step(oracle_mod, out, theta, nL, H, u1, kind, Lx, Ly, hf, sym, 1e-2)
    t1, m1, v1 = vmc.adam(theta, g, np.zeros_like(g), np.zeros_like(g), 1, 1e-2)
    assert np.max(np.abs(out["theta"].cpu().numpy() - t1)) <= 1e-6 + 1e-6 * np.max(np.abs(t1))
    # a second step from the updated parameters carries the Adam moments
    th2 = out["theta"].clone()
    out2 = api.vmc_step(th2, cfg, ham, u, adam, symmetrize=sym, sym_uniforms=us)
    api.sync()
    g2 = out2["grad"].cpu().numpy().astype(np.float64)
    t2, _, _ = vmc.adam(th2.cpu().numpy(), g2, m1, v1, 2, 1e-2)
    assert np.max(np.abs(out2["theta"].cpu().numpy() - t2)) <= 1e-5


def test_vmc_step_rejects_host_arrays_and_bad_constants():
    nL, H, N = 3, 32, 16
    theta = torch.from_numpy(_params(nL, H, 830, "fp32")).cuda()
    ham = B.make_hamiltonian("tfim", N, 1, False, True, 1.0, 1.0)
    p = B.make_params(theta, nL, H)
    u_host = inputs.uniform(831, (8, N)).astype(np.float32)
    adam = api.Adam(theta.numel(), "cuda")
    adam.step = 1
    out = torch.empty_like(theta)
    with pytest.raises(B.PsrError) as ei:
        B.psr_vmc_step(p, ham, False, u_host, None, adam.state(), out)
    assert ei.value.code == B.PSR_EINVAL
    u = torch.from_numpy(u_host).cuda()
    bad = api.Adam(theta.numel(), "cuda", beta1=1.0)
    bad.step = 1
    with pytest.raises(B.PsrError) as ei:
        B.psr_vmc_step(p, ham, False, u, None, bad.state(), out)
    assert ei.value.code == B.PSR_EINVAL
    sym_ham = B.make_hamiltonian("heisenberg", 4, 2, False, True, 1.0, 0.0)
    with pytest.raises(B.PsrError) as ei:  # c4v needs a square lattice
        B.psr_vmc_step(p, sym_ham, True, torch.zeros((8, 8), device="cuda"),
                       torch.zeros(8, device="cuda"), adam.state(), out)
    assert ei.value.code == B.PSR_EINVAL


def test_vmc_step_of_the_2d_model(oracle_mod):
    """psr2d_vmc_step: its E_loc match the oracle on the drawn samples, its
    gradient is the centred estimator over the per-sample O_k of psr2d_grad
    (themselves checked against finite differences), and its update is Adam."""
    Lx = Ly = 6
    nL, H, n = 3, 32, 64
    N, Np = Lx * Ly, (Lx // 2) * (Ly // 2)
    P = oracle_mod.param_count2d(nL, H)
    theta = ((2.0 * inputs.uniform(840, (P,)) - 1.0) * 2.0 / np.sqrt(H)).astype(np.float32)
    th = torch.from_numpy(theta).cuda()
    ham = B.make_hamiltonian("heisenberg", Lx, Ly, False, True, 1.0, 0.0)
    cfg = api.ModelConfig(nL, H, True, "fp32")
    u = torch.from_numpy(inputs.uniform(841, (n, Np)).astype(np.float32)).cuda()
    adam = api.Adam(P, "cuda", lr=1e-2)
    out = api.vmc_step2d(th, cfg, ham, u, adam)
    api.sync()
    s = out["spins"].cpu().numpy()
    assert np.all(s.sum(axis=1) == N // 2)
    e = out["eloc"].cpu().numpy().astype(np.float64)
    ref_e = oracle_mod.local_energy2d(theta.astype(np.float64), nL, H, s, 0, Lx, Ly, u1=True)
    _, _, diag = oracle_mod.connected(0, Lx, Ly, False, s)
    assert np.all(np.abs(e - ref_e) <= 1e-3 * (np.abs(diag) + np.abs(ref_e - diag)))
    ok = api.grad2d(th, out["spins"], cfg, Lx, Ly)
    api.sync()
    ref_g, _ = vmc.energy_gradient(e, ok.cpu().numpy().astype(np.float64))
    g = out["grad"].cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g - ref_g) <= 1e-4 * np.linalg.norm(ref_g)
    t1, _, _ = vmc.adam(theta, g, np.zeros(P), np.zeros(P), 1, 1e-2)
    assert np.max(np.abs(out["theta"].cpu().numpy() - t1)) <= 1e-6 + 1e-6 * np.max(np.abs(t1))
