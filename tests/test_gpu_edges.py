"""Degenerate and ragged inputs of the chain model's local energy and log psi
against the FP64 oracle: a lattice without bonds, samples without any
antiparallel bond next to samples with many (ragged connected sets), a
single sample, a transverse field of zero, and empty calls."""
import ctypes as C

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


def _eloc(theta, s, cfg, ham):
    e, st = api.local_energy(torch.from_numpy(theta).cuda(), torch.from_numpy(s).cuda(), cfg, ham)
    api.sync()
    return e.cpu().numpy().astype(np.float64), st.cpu().numpy()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_ragged_connected_sets(oracle_mod, precision):
    """Ferromagnetic samples have no antiparallel bond (no entries); Neel
    samples have one per bond."""
    Lx = Ly = 6
    N = Lx * Ly
    H = 128
    theta = inputs.glorot_params(3, H, seed=3)
    up = np.ones((1, N), np.uint8)
    down = np.zeros((1, N), np.uint8)
    neel = np.array([[(i + j) % 2 for j in range(Ly) for i in range(Lx)]], np.uint8)
    neel = inputs.to_sequence(neel.reshape(1, Ly, Lx), Lx, Ly)
    mixed = inputs.random_spins(4, 3, N)
    s = np.concatenate([up, mixed[:1], down, neel, mixed[1:]]).astype(np.uint8)
    ham = B.make_hamiltonian("heisenberg", Lx, Ly, False, True, 1.0, 0.0)
    e, _ = _eloc(theta, s, api.ModelConfig(3, H, False, precision), ham)
    ref = oracle_mod.local_energy(theta, 3, H, s, 0, Lx, Ly)
    offsets, _, diag = oracle_mod.connected(0, Lx, Ly, False, s)
    counts = np.diff(offsets)
    assert counts[0] == 0 and counts[2] == 0 and counts[3] == 60
    assert e[0] == diag[0] and e[2] == diag[2]  # no off-diagonal term at all
    scale = np.abs(diag) + np.abs(ref - diag)
    assert np.all(np.abs(e - ref) <= 1e-3 * scale)


def test_lattice_without_bonds_and_zero_field(oracle_mod):
    theta = inputs.random_params(3, 32, seed=5, scale=1.0)
    cfg = api.ModelConfig(3, 32, False, "fp32")
    s1 = inputs.random_spins(6, 5, 1)
    e, st = _eloc(theta, s1, cfg, B.make_hamiltonian("heisenberg", 1, 1, False, True, 1.0, 0.0))
    assert np.all(e == 0.0) and st[0] == 0.0  # one site: no bond, no energy
    e, _ = _eloc(theta, s1, cfg, B.make_hamiltonian("tfim", 1, 1, False, True, 1.0, 0.7))
    ref = oracle_mod.local_energy(theta, 3, 32, s1, 1, 1, 1, h=0.7)
    assert np.all(np.abs(e - ref) <= 1e-5 * (1 + np.abs(ref)))
    s = inputs.random_spins(7, 6, 12)
    e, _ = _eloc(theta, s, cfg, B.make_hamiltonian("tfim", 12, 1, False, True, 1.0, 0.0))
    _, _, diag = oracle_mod.connected(1, 12, 1, False, s)
    assert np.all(e == diag.astype(np.float32))  # h = 0: only the diagonal


def test_single_sample_and_statistics(oracle_mod):
    theta = inputs.random_params(3, 64, seed=8, scale=1.0)
    s = inputs.zero_magnetisation_spins(9, 1, 20)
    e, st = _eloc(theta, s, api.ModelConfig(3, 64, True, "fp32"),
                  B.make_hamiltonian("heisenberg", 20, 1, False, True, 1.0, 0.0))
    ref = oracle_mod.local_energy(theta, 3, 64, s, 0, 20, 1, u1=True)
    assert abs(e[0] - ref[0]) <= 1e-3 * (1 + abs(ref[0]))
    assert st[0] == e[0]
    assert st[1] == 0.0 and st[2] == 0.0  # one sample: the variance is reported as zero


def test_empty_calls_are_rejected():
    theta = torch.zeros(B.psr_param_count(3, 32), device="cuda")
    p = B.make_params(theta, 3, 32)
    out = torch.empty(1, device="cuda")
    s = torch.zeros((1, 4), dtype=torch.uint8, device="cuda")
    L = B.lib()
    assert L.psr_logpsi(C.byref(p), C.c_void_p(s.data_ptr()), 0, 4,
                        C.c_void_p(out.data_ptr())) == B.PSR_EINVAL
    ham = B.make_hamiltonian("tfim", 4, 1, False, True, 1.0, 1.0)
    assert L.psr_local_energy(C.byref(p), C.c_void_p(s.data_ptr()), 0, C.byref(ham),
                              C.c_void_p(out.data_ptr()), None) == B.PSR_EINVAL
    assert L.psr_logpsi(C.byref(p), C.c_void_p(s.data_ptr()), 1, 0,
                        C.c_void_p(out.data_ptr())) == B.PSR_EINVAL
