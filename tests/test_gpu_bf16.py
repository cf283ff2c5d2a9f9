"""GPU parity of the tcgen05 BF16 path (hidden 128, 3 layers) against the
FP64 oracle, through the C ABI.

The BF16 path rounds the operands of every dense projection (weights and
activations) to BF16 and accumulates in FP32; gates, scan carry, softmax and
sums stay FP32.  Tolerances:
  log psi : |d| <= 2e-2 + 2e-5 |log psi|   (spec 2e-2 for N <= 100; the
            relative term covers the growth of independent per-site rounding
            errors with N)
  E_loc   : |d| <= 1e-3 (|diag| + sum_e |c_e ratio_e|)  (the stated relative
            bound; a connected configuration shares its prefix with the
            sample, so most of the BF16 rounding cancels in the ratio)
With BF16-representable parameters the weight rounding vanishes and only
activation rounding remains; those runs use tolerances 5x tighter.
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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _bf16_representable(theta):
    t = torch.from_numpy(theta).to(torch.bfloat16).to(torch.float32)
    return t.numpy()


def _lp(theta, spins, u1, prec="bf16"):
    out = api.logpsi(_dev(theta), _dev(spins), api.ModelConfig(NL, H, u1, prec))
    api.sync()
    return out.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("N,u1,seed", [(64, False, 1), (1, False, 2), (2, True, 3), (36, True, 4),
                                       (63, False, 5), (65, False, 6), (100, True, 7), (128, True, 8),
                                       (200, False, 9), (31, False, 10), (32, True, 11), (33, False, 12)])
def test_logpsi_bf16_matches_oracle(oracle_mod, N, u1, seed):
    theta = inputs.glorot_params(NL, H, seed=seed)
    n = 40
    spins = (inputs.zero_magnetisation_spins(seed, n, N) if u1 else inputs.random_spins(seed, n, N))
    got = _lp(theta, spins, u1)
    ref = oracle_mod.logpsi(theta, NL, H, spins, u1=u1)
    err = np.abs(got - ref)
    assert np.all(err <= 2e-2 + 2e-5 * np.abs(ref)), (err.max(), np.abs(ref).max())
    thb = _bf16_representable(theta)
    got_b = _lp(thb, spins, u1)
    ref_b = oracle_mod.logpsi(thb, NL, H, spins, u1=u1)
    err_b = np.abs(got_b - ref_b)
    assert np.all(err_b <= 4e-3 + 4e-6 * np.abs(ref_b)), err_b.max()


def test_bf16_random_parameters_every_entry(oracle_mod):
    """Nonzero biases and larger weights exercise every packed parameter."""
    theta = inputs.random_params(NL, H, seed=17, scale=1.0)
    spins = inputs.random_spins(18, 32, 130)
    got = _lp(theta, spins, False)
    ref = oracle_mod.logpsi(theta, NL, H, spins)
    assert np.max(np.abs(got - ref)) <= 2e-2 + 2e-5 * np.max(np.abs(ref))


def test_bf16_deterministic_and_host_buffers():
    theta = inputs.glorot_params(NL, H, seed=3)
    spins = inputs.random_spins(4, 300, 150)
    a = _lp(theta, spins, False)
    b = _lp(theta, spins, False)
    assert np.array_equal(a, b)
    host = api.logpsi(torch.from_numpy(theta), torch.from_numpy(spins),
                      api.ModelConfig(NL, H, False, "bf16")).numpy()
    assert np.array_equal(a.astype(np.float32), host)


def _eloc(theta, spins, kind, Lx, Ly, pbc, u1, hf, prec):
    ham = B.make_hamiltonian(kind, Lx, Ly, pbc, True, 1.0, hf)
    e, st = api.local_energy(_dev(theta), _dev(spins), api.ModelConfig(NL, H, u1, prec), ham)
    api.sync()
    return e.cpu().numpy().astype(np.float64), st.cpu().numpy()


@pytest.mark.parametrize("kind,Lx,Ly,pbc,u1,hf,n", [(0, 10, 10, False, True, 0.0, 6),
                                                    (0, 100, 1, True, True, 0.0, 6),
                                                    (1, 9, 8, False, False, 3.044, 4)])
def test_local_energy_bf16_matches_oracle(oracle_mod, kind, Lx, Ly, pbc, u1, hf, n):
    theta = inputs.glorot_params(NL, H, seed=0)
    N = Lx * Ly
    spins = (inputs.neel_like_spins(5, n, Lx, Ly) if kind == 0 else inputs.random_spins(5, n, N))
    e, st = _eloc(theta, spins, kind, Lx, Ly, pbc, u1, hf, "bf16")
    ref = oracle_mod.local_energy(theta, NL, H, spins, kind, Lx, Ly, pbc=pbc, marshall=True, J=1.0,
                                  h=hf, u1=u1)
    _, _, diag = oracle_mod.connected(kind, Lx, Ly, pbc, spins)
    scale = np.abs(diag) + np.abs(ref - diag)
    assert np.all(np.abs(e - ref) <= 1e-3 * scale), (np.abs(e - ref) / scale).max()
    assert abs(st[0] - np.mean(e)) <= 1e-6 * max(1.0, abs(st[0]))


def test_local_energy_path_equals_logpsi_path_bf16(oracle_mod):
    """E_loc from the resumed-suffix path equals E_loc assembled from full
    log psi evaluations of every connected configuration (same kernel)."""
    Lx = Ly = 12
    N = Lx * Ly
    theta = inputs.glorot_params(NL, H, seed=0)
    spins = inputs.neel_like_spins(6, 3, Lx, Ly)
    ham = B.make_hamiltonian(0, Lx, Ly, False, True, 1.0, 0.0)
    e, _ = _eloc(theta, spins, 0, Lx, Ly, False, True, 0.0, "bf16")
    offs, ent, diag = api.connected(_dev(spins), ham)
    offs, ent, diag = offs.cpu().numpy(), ent.cpu().numpy(), diag.cpu().numpy()
    sp = spins[ent[:, 0]].copy()
    r = np.arange(len(ent))
    sp[r, ent[:, 1]] ^= 1
    sp[r, ent[:, 2]] ^= 1
    lp_s = _lp(theta, spins, True)
    lp_c = _lp(theta, sp, True)
    for i in range(len(spins)):
        sl = slice(offs[i], offs[i + 1])
        want = diag[i] - 0.5 * np.sum(np.exp(lp_c[sl] - lp_s[i]))
        assert abs(e[i] - want) <= 1e-4 * (abs(diag[i]) + abs(want - diag[i]))


def test_bf16_full_lattice_sampled_outputs(oracle_mod):
    """52x52 (2704 sites): log psi of sampled configurations against the oracle."""
    Lx = Ly = 52
    theta = inputs.glorot_params(NL, H, seed=0)
    spins = inputs.neel_like_spins(7, 4, Lx, Ly)
    got = _lp(theta, spins, True)
    ref = oracle_mod.logpsi(theta, NL, H, spins, u1=True)
    assert np.all(np.abs(got - ref) <= 2e-2 + 2e-5 * np.abs(ref)), np.abs(got - ref).max()
    got32 = _lp(theta, spins, True, "fp32")
    assert np.all(np.abs(got32 - ref) <= 1e-5 + 1e-6 * np.abs(ref)), np.abs(got32 - ref).max()
