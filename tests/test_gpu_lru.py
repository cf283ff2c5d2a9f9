"""GPU deep 1D LRU (psr_lru_logpsi, psr_lru_local_energy) against the FP64
oracle of the same model.  Tolerances as for the chain minGRU's FP32 path:
|d log psi| <= 1e-5 + 1e-6 |log psi|; E_loc error <= 1e-3 of
|diag| + |E_loc - diag|."""
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


def _theta(oracle_mod, nL, H, seed, kind):
    P = oracle_mod.param_count_lru(nL, H)
    assert P == api.param_count_lru(nL, H)
    if kind == "ring":
        th = inputs.lru_params(nL, H, seed=seed)
    else:  # every entry random (biases, nu, theta and gamma included)
        th = ((2.0 * inputs.uniform(seed, (P,)) - 1.0) / np.sqrt(H)).astype(np.float32)
    assert th.size == P
    return th


@pytest.mark.parametrize("N,H,nL,u1,kind", [(16, 32, 3, False, "random"), (100, 64, 3, True, "ring"),
                                            (256, 64, 3, False, "ring"), (37, 128, 2, False, "random"),
                                            (70, 32, 1, True, "random")])
def test_logpsi_matches_oracle(oracle_mod, N, H, nL, u1, kind):
    theta = _theta(oracle_mod, nL, H, 600 + N + H, kind)
    s = (inputs.zero_magnetisation_spins(601, 32, N) if u1 else inputs.random_spins(601, 32, N))
    cfg = api.ModelConfig(nL, H, u1, "fp32")
    got = api.logpsi_lru(torch.from_numpy(theta).cuda(), torch.from_numpy(s).cuda(), cfg)
    api.sync()
    ref = oracle_mod.logpsi_lru(theta.astype(np.float64), nL, H, s, u1=u1)
    got = got.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - ref) <= 1e-5 + 1e-6 * np.abs(ref)), np.max(np.abs(got - ref))


@pytest.mark.parametrize("kind,N,pbc,u1,hf", [(1, 16, False, False, 1.0), (1, 16, True, False, 1.0),
                                              (0, 20, False, True, 0.0), (1, 256, False, False, 1.0)])
def test_local_energy_matches_oracle(oracle_mod, kind, N, pbc, u1, hf):
    nL, H = 3, 64
    theta = _theta(oracle_mod, nL, H, 610 + N, "ring")
    n = 3 if N >= 256 else 12
    s = (inputs.zero_magnetisation_spins(611, n, N) if u1 else inputs.random_spins(611, n, N))
    ham = B.make_hamiltonian(kind, N, 1, pbc, True, 1.0, hf)
    cfg = api.ModelConfig(nL, H, u1, "fp32")
    e, st = api.local_energy_lru(torch.from_numpy(theta).cuda(), torch.from_numpy(s).cuda(), cfg, ham)
    api.sync()
    ref = oracle_mod.local_energy_lru(theta.astype(np.float64), nL, H, s, kind, N, 1, pbc=pbc,
                                      marshall=True, J=1.0, h=hf, u1=u1)
    _, _, diag = oracle_mod.connected(kind, N, 1, pbc, s)
    scale = np.abs(diag) + np.abs(ref - diag)
    assert np.all(np.abs(e.cpu().numpy() - ref) <= 1e-3 * scale)
    m, _, _ = oracle_mod.stats(e.cpu().numpy().astype(np.float64))
    assert abs(st[0].item() - m) <= 1e-9 * max(1.0, abs(m))


def test_rejects_bf16_and_odd_u1():
    theta = torch.zeros(api.param_count_lru(3, 32), device="cuda")
    out = torch.empty(2, device="cuda")
    s = torch.zeros((2, 10), dtype=torch.uint8, device="cuda")
    with pytest.raises(B.PsrError) as ei:
        B.psr_lru_logpsi(B.make_params(theta, 3, 32, False, "bf16"), s, out)
    assert ei.value.code == B.PSR_EUNSUPPORTED
    s9 = torch.zeros((2, 9), dtype=torch.uint8, device="cuda")
    with pytest.raises(B.PsrError) as ei:
        B.psr_lru_logpsi(B.make_params(theta, 3, 32, True, "fp32"), s9, out)
    assert ei.value.code == B.PSR_EINVAL
