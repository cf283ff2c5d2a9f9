"""Shapes of the fused forward kernels and their autotuner.

BF16 (tcgen05) forward: one sequence per MMA stream (four streams per SM,
N = 32) or two side by side (two streams, N = 64).  Each sequence's
arithmetic is the same in both, so log psi and E_loc must be identical bit
for bit, and both must match the FP64 oracle at the BF16 tolerances
(|d log psi| <= 2e-2 + 2e-5 |log psi|; E_loc 1e-3 of |diag| + sum |c ratio|).
Odd sample counts leave sequences of a two-sequence stream idle while the
other still runs; that must change nothing.
FP32 (SIMT) forward: scan chunks of 32 or 16 sites, both at the FP32
tolerance (1e-5 + 1e-6 |log psi|; E_loc 1e-3).
Autotuner: with it on, the first call of a shape times both candidates,
keeps the faster one and computes with it.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2605_13807_gb300 import api, binding as B, inputs  # noqa: E402

NL, H = 3, 128


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    yield
    api.set_fwd_shape("bf16", 0)
    api.set_fwd_shape("fp32", 0)


def _shaped(precision, shape, fn):
    api.set_fwd_shape(precision, shape)
    try:
        out = fn()
        api.sync()
        return out
    finally:
        api.set_fwd_shape(precision, 0)


def _spins(kind, seed, n, Lx, Ly, u1):
    if kind == 0 and Ly > 1:
        return inputs.neel_like_spins(seed, n, Lx, Ly)
    N = Lx * Ly
    return inputs.zero_magnetisation_spins(seed, n, N) if u1 else inputs.random_spins(seed, n, N)


@pytest.mark.parametrize("N,n,u1", [(1, 3, False), (2, 5, True), (31, 7, False), (33, 9, False),
                                    (64, 1, False), (100, 13, True), (200, 40, False), (97, 6, False)])
def test_bf16_shapes_give_identical_logpsi(oracle_mod, N, n, u1):
    theta_np = inputs.glorot_params(NL, H, seed=N)
    spins_np = inputs.zero_magnetisation_spins(N + 1, n, N) if u1 else inputs.random_spins(N + 1, n, N)
    theta = torch.from_numpy(theta_np).cuda()
    spins = torch.from_numpy(spins_np).cuda()
    cfg = api.ModelConfig(NL, H, u1, "bf16")
    a = _shaped("bf16", 1, lambda: api.logpsi(theta, spins, cfg))
    b = _shaped("bf16", 2, lambda: api.logpsi(theta, spins, cfg))
    assert torch.equal(a, b)
    ref = oracle_mod.logpsi(theta_np, NL, H, spins_np, u1=u1)
    got = a.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - ref) <= 2e-2 + 2e-5 * np.abs(ref)), np.abs(got - ref).max()


@pytest.mark.parametrize("kind,Lx,Ly,pbc,u1,hf,n,check", [
    (0, 10, 10, False, True, 0.0, 7, True), (0, 100, 1, True, True, 0.0, 5, True),
    (1, 9, 8, False, False, 3.044, 3, True), (0, 16, 16, False, True, 0.0, 9, False),
    (1, 20, 20, False, False, 3.044, 5, False)])
def test_bf16_shapes_give_identical_local_energy(oracle_mod, kind, Lx, Ly, pbc, u1, hf, n, check):
    theta_np = inputs.glorot_params(NL, H, seed=0)
    spins_np = _spins(kind, 31 + Lx, n, Lx, Ly, u1)
    theta = torch.from_numpy(theta_np).cuda()
    spins = torch.from_numpy(spins_np).cuda()
    cfg = api.ModelConfig(NL, H, u1, "bf16")
    ham = B.make_hamiltonian(kind, Lx, Ly, pbc, True, 1.0, hf)
    e1, s1 = _shaped("bf16", 1, lambda: api.local_energy(theta, spins, cfg, ham))
    e2, s2 = _shaped("bf16", 2, lambda: api.local_energy(theta, spins, cfg, ham))
    assert torch.equal(e1, e2) and torch.equal(s1, s2)
    if check:
        ref = oracle_mod.local_energy(theta_np, NL, H, spins_np, kind, Lx, Ly, pbc=pbc, marshall=True,
                                      J=1.0, h=hf, u1=u1)
        _, _, diag = oracle_mod.connected(kind, Lx, Ly, pbc, spins_np)
        scale = np.abs(diag) + np.abs(ref - diag)
        e = e1.cpu().numpy().astype(np.float64)
        assert np.all(np.abs(e - ref) <= 1e-3 * scale), (np.abs(e - ref) / scale).max()


@pytest.mark.parametrize("shape", [32, 16])
def test_fp32_chunk_shapes_match_oracle(oracle_mod, shape):
    theta_np = inputs.random_params(NL, 64, seed=5, scale=1.0)
    theta = torch.from_numpy(theta_np).cuda()
    cfg = api.ModelConfig(NL, 64, True, "fp32")
    spins_np = inputs.zero_magnetisation_spins(6, 9, 70)
    lp = _shaped("fp32", shape, lambda: api.logpsi(theta, torch.from_numpy(spins_np).cuda(), cfg))
    ref = oracle_mod.logpsi(theta_np, NL, 64, spins_np, u1=True)
    got = lp.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - ref) <= 1e-5 + 1e-6 * np.abs(ref)), np.abs(got - ref).max()
    s2 = inputs.neel_like_spins(7, 5, 6, 6)
    ham = B.make_hamiltonian("heisenberg", 6, 6, False, True, 1.0, 0.0)
    e, _ = _shaped("fp32", shape, lambda: api.local_energy(theta, torch.from_numpy(s2).cuda(), cfg, ham))
    ref_e = oracle_mod.local_energy(theta_np, NL, 64, s2, 0, 6, 6, marshall=True, J=1.0, h=0.0, u1=True)
    _, _, diag = oracle_mod.connected(0, 6, 6, False, s2)
    scale = np.abs(diag) + np.abs(ref_e - diag)
    assert np.all(np.abs(e.cpu().numpy() - ref_e) <= 1e-3 * scale)


def test_invalid_shapes_are_rejected():
    ctx = api._ctx()
    for prec, bad in (("bf16", 3), ("bf16", 32), ("fp32", 2), ("fp32", 64)):
        with pytest.raises(B.PsrError) as ei:
            B.psr_context_set_fwd_shape(ctx, prec, bad)
        assert ei.value.code == B.PSR_EINVAL


@pytest.mark.parametrize("precision", ["bf16", "fp32"])
def test_autotuner_picks_keeps_and_uses_a_shape(precision):
    L, n = 12, 64
    theta = torch.from_numpy(inputs.glorot_params(NL, H, seed=3)).cuda()
    spins = torch.from_numpy(inputs.neel_like_spins(4, n, L, L)).cuda()
    cfg = api.ModelConfig(NL, H, True, precision)
    ham = B.make_hamiltonian("heisenberg", L, L, False, True, 1.0, 0.0)
    shape0, tuned0 = api.fwd_shape_for(precision, 1, n, L * L)
    assert not tuned0
    api.set_autotune(True)
    try:
        e, st = api.local_energy(theta, spins, cfg, ham)
        api.sync()
    finally:
        api.set_autotune(False)
    shape, tuned = api.fwd_shape_for(precision, 1, n, L * L)
    assert tuned and shape in ((1, 2) if precision == "bf16" else (16, 32))
    # the tuned call computed with the shape it kept
    e_fixed, st_fixed = _shaped(precision, shape, lambda: api.local_energy(theta, spins, cfg, ham))
    assert torch.equal(e, e_fixed) and torch.equal(st, st_fixed)
    # a call without the tuner uses the kept shape too
    e_again, _ = api.local_energy(theta, spins, cfg, ham)
    api.sync()
    assert torch.equal(e, e_again)
