"""GPU parity of the FP32 path against the FP64 oracle, through the C ABI.

Tolerances (FP32 arithmetic against FP64):
  log psi: |d| <= 1e-5 + 1e-6 |log psi|   (1e-5 absolute for the small lattices;
           the relative term covers the FP32 resolution of sums of N terms)
  E_loc  : |d| <= 1e-3 (|diag| + sum_e |c_e ratio_e|)  per sample
  grad   : ||d||_2 <= 1e-3 ||g||_2 and |d_k| <= 1e-3 ||g||_inf
  generator: bit-exact.
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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _logpsi_tol(ref):
    return 1e-5 + 1e-6 * np.abs(ref)


def _run_logpsi(theta, spins, cfg):
    out = api.logpsi(_dev(theta), _dev(spins), cfg)
    api.sync()
    return out.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("n_layers,H,N,u1,seed", [
    (3, 32, 16, False, 0), (3, 64, 100, True, 1), (3, 128, 36, True, 2), (1, 32, 33, False, 3),
    (4, 64, 65, False, 4), (3, 128, 100, True, 5), (2, 32, 1, False, 6), (3, 32, 2, True, 7),
    (3, 64, 31, False, 8), (3, 64, 32, False, 9), (3, 64, 64, True, 10)])
def test_logpsi_matches_oracle(oracle_mod, n_layers, H, N, u1, seed):
    theta = inputs.random_params(n_layers, H, seed=seed, scale=1.0)
    n = 48
    spins = (inputs.zero_magnetisation_spins(seed + 100, n, N) if u1
             else inputs.random_spins(seed + 100, n, N))
    cfg = api.ModelConfig(n_layers, H, u1, "fp32")
    got = _run_logpsi(theta, spins, cfg)
    ref = oracle_mod.logpsi(theta, n_layers, H, spins, u1=u1)
    assert np.all(np.abs(got - ref) <= _logpsi_tol(ref)), np.max(np.abs(got - ref))


def test_logpsi_c1_model_samples(oracle_mod):
    """1D chain N=16, hidden 32, Glorot seed 0, 1024 samples drawn from the model."""
    n_layers, H, N, n = 3, 32, 16, 1024
    theta = inputs.glorot_params(n_layers, H, seed=0)
    spins, ref = oracle_mod.sample(theta, n_layers, H, N, inputs.uniform(1, (n, N)))
    got = _run_logpsi(theta, spins, api.ModelConfig(n_layers, H, False, "fp32"))
    assert np.max(np.abs(got - ref)) <= 1e-5


def test_logpsi_outside_u1_sector_is_minus_inf(oracle_mod):
    n_layers, H, N = 3, 32, 10
    theta = inputs.random_params(n_layers, H, seed=3)
    spins = np.zeros((2, N), dtype=np.uint8)
    spins[1, :6] = 1
    got = _run_logpsi(theta, spins, api.ModelConfig(n_layers, H, True, "fp32"))
    assert np.all(np.isneginf(got))


def test_host_buffers_give_the_same_result(oracle_mod):
    n_layers, H, N = 3, 64, 50
    theta = inputs.random_params(n_layers, H, seed=11)
    spins = inputs.random_spins(12, 20, N)
    cfg = api.ModelConfig(n_layers, H, False, "fp32")
    dev = _run_logpsi(theta, spins, cfg)
    host = api.logpsi(torch.from_numpy(theta), torch.from_numpy(spins), cfg).numpy()
    assert np.array_equal(dev.astype(np.float32), host)


def test_deterministic_bits():
    n_layers, H, N = 3, 128, 70
    theta = inputs.random_params(n_layers, H, seed=13)
    spins = inputs.random_spins(14, 40, N)
    cfg = api.ModelConfig(n_layers, H, False, "fp32")
    a = _run_logpsi(theta, spins, cfg)
    b = _run_logpsi(theta, spins, cfg)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("kind,Lx,Ly,pbc", [(0, 16, 1, False), (0, 100, 1, True), (0, 10, 10, False),
                                            (0, 7, 6, False), (1, 20, 20, False), (1, 5, 1, False),
                                            (0, 4, 4, True)])
def test_connected_generator_is_bit_exact(oracle_mod, kind, Lx, Ly, pbc):
    N = Lx * Ly
    spins = inputs.random_spins(20 + N, 33, N)
    ham = B.make_hamiltonian(kind, Lx, Ly, pbc, True, 1.0, 3.044)
    offs, ent, diag = api.connected(_dev(spins), ham)
    r_off, r_ent, r_diag = oracle_mod.connected(kind, Lx, Ly, pbc, spins)
    assert np.array_equal(offs.cpu().numpy(), r_off)
    assert np.array_equal(ent.cpu().numpy(), r_ent)
    assert np.array_equal(diag.cpu().numpy().astype(np.float64), r_diag)


def _eloc_check(oracle_mod, theta, n_layers, H, spins, kind, Lx, Ly, pbc, u1, hfield, precision="fp32"):
    cfg = api.ModelConfig(n_layers, H, u1, precision)
    ham = B.make_hamiltonian(kind, Lx, Ly, pbc, True, 1.0, hfield)
    e, st = api.local_energy(_dev(theta), _dev(spins), cfg, ham)
    api.sync()
    e = e.cpu().numpy().astype(np.float64)
    st = st.cpu().numpy()
    ref = oracle_mod.local_energy(theta, n_layers, H, spins, kind, Lx, Ly, pbc=pbc, marshall=True,
                                  J=1.0, h=hfield, u1=u1)
    # scale of each sample's terms for the relative bound
    # |diag| + sum_e |c_e ratio_e|: every c_e has the same sign, so the sum is |E_loc - diag|
    _, _, diag = oracle_mod.connected(kind, Lx, Ly, pbc, spins)
    scale = np.abs(diag) + np.abs(ref - diag)
    assert np.all(np.abs(e - ref) <= 1e-3 * np.maximum(scale, 1e-3)), np.max(np.abs(e - ref))
    m, v, se = oracle_mod.stats(e)
    assert abs(st[0] - m) <= 1e-9 * max(1, abs(m))
    assert abs(st[1] - v) <= 1e-9 * max(1, abs(v))
    assert abs(st[0] - np.mean(ref)) <= 1e-3 * abs(np.mean(ref))
    return e, ref


def test_local_energy_c1(oracle_mod):
    n_layers, H, N, n = 3, 32, 16, 1024
    theta = inputs.glorot_params(n_layers, H, seed=0)
    spins, _ = oracle_mod.sample(theta, n_layers, H, N, inputs.uniform(1, (n, N)))
    _eloc_check(oracle_mod, theta, n_layers, H, spins, 0, N, 1, False, False, 0.0)


def test_local_energy_chain_pbc_u1(oracle_mod):
    n_layers, H, N, n = 3, 64, 100, 48
    theta = inputs.random_params(n_layers, H, seed=21, scale=1.0)
    spins, _ = oracle_mod.sample(theta, n_layers, H, N, inputs.uniform(22, (n, N)), u1=True)
    _eloc_check(oracle_mod, theta, n_layers, H, spins, 0, N, 1, True, True, 0.0)


def test_local_energy_2d_heisenberg_h128(oracle_mod):
    n_layers, H, Lx, Ly, n = 3, 128, 6, 6, 12
    theta = inputs.glorot_params(n_layers, H, seed=0)
    spins = inputs.neel_like_spins(23, n, Lx, Ly)
    _eloc_check(oracle_mod, theta, n_layers, H, spins, 0, Lx, Ly, False, True, 0.0)


def test_local_energy_2d_tfim(oracle_mod):
    n_layers, H, Lx, Ly, n = 3, 64, 5, 5, 16
    theta = inputs.random_params(n_layers, H, seed=24, scale=1.0)
    spins = inputs.random_spins(25, n, Lx * Ly)
    _eloc_check(oracle_mod, theta, n_layers, H, spins, 1, Lx, Ly, False, False, 3.044)


def _grad_ok(got, ref):
    d = got - ref
    assert np.linalg.norm(d) <= 1e-3 * np.linalg.norm(ref), np.linalg.norm(d) / np.linalg.norm(ref)
    assert np.max(np.abs(d)) <= 1e-3 * np.max(np.abs(ref))


@pytest.mark.parametrize("n_layers,H,N,u1,n", [(3, 32, 16, False, 8), (3, 64, 100, True, 3),
                                               (3, 128, 40, False, 2), (4, 32, 70, True, 2)])
def test_per_sample_gradient_matches_oracle(oracle_mod, n_layers, H, N, u1, n):
    theta = inputs.random_params(n_layers, H, seed=30 + N, scale=1.0)
    spins = (inputs.zero_magnetisation_spins(31, n, N) if u1 else inputs.random_spins(31, n, N))
    cfg = api.ModelConfig(n_layers, H, u1, "fp32")
    g = api.grad(_dev(theta), _dev(spins), cfg)
    api.sync()
    g = g.cpu().numpy().astype(np.float64)
    _, ref = oracle_mod.grad(theta, n_layers, H, spins, u1=u1)
    for i in range(n):
        _grad_ok(g[i], ref[i])


def test_summed_gradient_and_autograd(oracle_mod):
    n_layers, H, N, n = 3, 64, 48, 6
    theta = inputs.random_params(n_layers, H, seed=40, scale=1.0)
    spins = inputs.random_spins(41, n, N)
    dout = (inputs.uniform(42, (n,)) - 0.5).astype(np.float32)
    cfg = api.ModelConfig(n_layers, H, False, "fp32")
    g = api.grad(_dev(theta), _dev(spins), cfg, dout=_dev(dout))
    api.sync()
    _, ref = oracle_mod.grad(theta, n_layers, H, spins)
    want = (dout.astype(np.float64)[:, None] * ref).sum(axis=0)
    _grad_ok(g.cpu().numpy().astype(np.float64), want)
    th = _dev(theta).requires_grad_(True)
    lp = api.LogPsi.apply(th, _dev(spins), cfg)
    (lp * _dev(dout)).sum().backward()
    _grad_ok(th.grad.cpu().numpy().astype(np.float64), want)


def test_invalid_spin_byte_is_reported():
    theta = inputs.random_params(3, 32, seed=1)
    spins = np.zeros((2, 8), dtype=np.uint8)
    spins[0, 3] = 2
    cfg = api.ModelConfig(3, 32, False, "fp32")
    api.logpsi(_dev(theta), _dev(spins), cfg)
    with pytest.raises(B.PsrError) as ei:
        api.sync()
    assert ei.value.code == B.PSR_EDEVICE
    api.sync()  # cleared


def test_argument_errors():
    theta = _dev(inputs.random_params(3, 64, seed=1))
    spins = _dev(inputs.random_spins(1, 4, 9))
    with pytest.raises(B.PsrError) as ei:
        api.logpsi(theta, spins, api.ModelConfig(3, 64, True, "fp32"))  # odd N with u1
    assert ei.value.code == B.PSR_EINVAL
    with pytest.raises(B.PsrError) as ei:
        api.logpsi(theta, spins, api.ModelConfig(3, 64, False, "bf16"))
    assert ei.value.code == B.PSR_EUNSUPPORTED
    ham = B.make_hamiltonian(0, 5, 1, True, True)  # odd periodic chain is not bipartite
    with pytest.raises(B.PsrError) as ei:
        api.local_energy(theta, _dev(inputs.random_spins(1, 4, 5)), api.ModelConfig(3, 64), ham)
    assert ei.value.code == B.PSR_EINVAL


def test_gradient_is_deterministic():
    """Gradient updates are reductions with one writer per address, so two
    runs give identical bits (per-sample rows and the dout-weighted sum)."""
    n_layers, H, N, n = 3, 128, 70, 12
    theta = _dev(inputs.random_params(n_layers, H, seed=50, scale=1.0))
    spins = _dev(inputs.random_spins(51, n, N))
    dout = _dev((inputs.uniform(52, (n,)) - 0.5).astype(np.float32))
    cfg = api.ModelConfig(n_layers, H, False, "fp32")
    a = api.grad(theta, spins, cfg).clone()
    b = api.grad(theta, spins, cfg)
    api.sync()
    assert torch.equal(a, b)
    c = api.grad(theta, spins, cfg, dout=dout).clone()
    d = api.grad(theta, spins, cfg, dout=dout)
    api.sync()
    assert torch.equal(c, d)
