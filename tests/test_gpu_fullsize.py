"""Parity at the full benchmark size, in the launch configuration the
benchmark times: 52x52 open Heisenberg lattice, 4096 Neel-like samples
(the benchmark's seed), hidden 128, 3 layers, BF16 projections.

The oracle cannot evaluate E_loc of a 52x52 sample in test time (about 3,800
full forwards of 2,704 sites each), so the check combines:
- a property that holds at any size: for sampled samples of the full-size
  call, E_loc equals diag + sum_e c_e exp(log psi(s'_e) - log psi(s))
  assembled from full (non-resumed) log psi evaluations of every connected
  configuration of that sample, and the reported mean is the FP64 mean;
- oracle values one by one: log psi of sampled connected configurations of
  those samples against the FP64 oracle at the BF16 tolerance.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2605_13807_gb300 import api, binding as B, inputs  # noqa: E402

NL, H, L, NS = 3, 128, 52, 4096


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    yield


def test_full_size_local_energy_in_the_benchmark_configuration(oracle_mod):
    theta_np = inputs.glorot_params(NL, H, seed=0)
    spins_np = inputs.neel_like_spins(1000, NS, L, L)
    theta = torch.from_numpy(theta_np).cuda()
    spins = torch.from_numpy(spins_np).cuda()
    cfg = api.ModelConfig(NL, H, True, "bf16")
    ham = B.make_hamiltonian("heisenberg", L, L, False, True, 1.0, 0.0)
    e, st = api.local_energy(theta, spins, cfg, ham)
    api.sync()
    e = e.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(e))
    assert abs(st[0].item() - np.mean(e)) <= 1e-6 * max(1.0, abs(np.mean(e)))
    rng = np.random.default_rng(1001)
    picked = [0, int(rng.integers(1, NS - 1)), NS - 1]
    checked = 0
    for i in picked:
        offs, ent, diag = api.connected(spins[i:i + 1].contiguous(), ham)
        ent = ent.cpu().numpy()
        diag = float(diag.cpu().numpy()[0])
        assert ent.shape[0] > 2000  # a Neel-like 52x52 sample has thousands
        sp = np.repeat(spins_np[i:i + 1], ent.shape[0], axis=0)
        r = np.arange(ent.shape[0])
        sp[r, ent[:, 1]] ^= 1
        sp[r, ent[:, 2]] ^= 1
        lp_c = api.logpsi(theta, torch.from_numpy(sp).cuda(), cfg)
        lp_s = api.logpsi(theta, spins[i:i + 1].contiguous(), cfg)
        api.sync()
        lp_c = lp_c.cpu().numpy().astype(np.float64)
        lp_s = float(lp_s.cpu().numpy()[0])
        want = diag - 0.5 * np.sum(np.exp(lp_c - lp_s))  # Heisenberg + Marshall: c_e = -J/2
        assert abs(e[i] - want) <= 1e-4 * (abs(diag) + abs(want - diag)), (i, e[i], want)
        # log psi of two of its connected configurations against the oracle
        for k in rng.choice(ent.shape[0], 2, replace=False):
            ref = oracle_mod.logpsi(theta_np, NL, H, sp[k:k + 1], u1=True)[0]
            assert abs(lp_c[k] - ref) <= 2e-2 + 2e-5 * abs(ref), (i, k, lp_c[k], ref)
            checked += 1
    assert checked == 6


def test_full_size_per_sample_gradient_row_against_the_oracle(oracle_mod):
    """O_k rows of the full 4096-sample gradient call (FP32 reverse scan, the
    benchmark's psr_grad launch) against the oracle's FP64 reverse mode for
    sampled samples: ||dg|| <= 1e-3 ||g|| and max|dg_k| <= 1e-3 max|g|."""
    theta_np = inputs.glorot_params(NL, H, seed=0)
    spins_np = inputs.neel_like_spins(1000, NS, L, L)
    cfg = api.ModelConfig(NL, H, True, "bf16")
    ok = api.grad(torch.from_numpy(theta_np).cuda(), torch.from_numpy(spins_np).cuda(), cfg)
    api.sync()
    assert ok.shape == (NS, theta_np.size)
    for i in (5, NS - 2):
        row = ok[i].cpu().numpy().astype(np.float64)
        _, ref = oracle_mod.grad(theta_np, NL, H, spins_np[i:i + 1], u1=True)
        ref = ref[0]
        assert np.linalg.norm(row - ref) <= 1e-3 * np.linalg.norm(ref)
        assert np.max(np.abs(row - ref)) <= 1e-3 * np.max(np.abs(ref))
