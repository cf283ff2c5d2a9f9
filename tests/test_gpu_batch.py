"""Mixed persistent batch (psr_local_energy_batch): several lattices and both
Hamiltonians in one launch, optionally replayed from a CUDA graph.

Each item must get exactly what psr_local_energy gives it alone (the per-job
arithmetic does not depend on scheduling, so the comparison is bitwise), and
small items are checked against the FP64 oracle.
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


def _items(seed=0):
    spec = [("heisenberg", 6, 6, 48, True, 0.0), ("heisenberg", 8, 8, 24, True, 0.0),
            ("heisenberg", 10, 10, 12, True, 0.0), ("tfim", 5, 4, 20, False, 3.044)]
    out = []
    for k, (kind, Lx, Ly, n, u1, hf) in enumerate(spec):
        if kind == "heisenberg":
            s = inputs.neel_like_spins(seed + 10 * k, n, Lx, Ly)
        else:
            s = inputs.random_spins(seed + 10 * k, n, Lx * Ly)
        ham = B.make_hamiltonian(kind, Lx, Ly, False, True, 1.0, hf)
        out.append((torch.from_numpy(s).cuda(), ham, u1, s))
    return out


@pytest.mark.parametrize("precision", ["bf16", "fp32"])
def test_batch_equals_single_calls(precision):
    theta = torch.from_numpy(inputs.glorot_params(NL, H, seed=0)).cuda()
    items = _items()
    outs, stats = api.local_energy_batch(theta, [(s, h, u1) for s, h, u1, _ in items],
                                         api.ModelConfig(NL, H, False, precision))
    api.sync()
    for (s, h, u1, _), o, st in zip(items, outs, stats):
        e, st1 = api.local_energy(theta, s, api.ModelConfig(NL, H, u1, precision), h)
        api.sync()
        assert torch.equal(o, e)
        assert torch.equal(st, st1)


def test_batch_matches_oracle_fp32(oracle_mod):
    theta_np = inputs.glorot_params(NL, H, seed=0)
    theta = torch.from_numpy(theta_np).cuda()
    items = _items(seed=5)[::3]  # 6x6 Heisenberg and 5x4 TFIM
    outs, _ = api.local_energy_batch(theta, [(s, h, u1) for s, h, u1, _ in items],
                                     api.ModelConfig(NL, H, False, "fp32"))
    api.sync()
    for (s, h, u1, s_np), o in zip(items, outs):
        ref = oracle_mod.local_energy(theta_np, NL, H, s_np, h.kind, h.Lx, h.Ly, pbc=False,
                                      marshall=True, J=1.0, h=h.h, u1=u1)
        _, _, diag = oracle_mod.connected(h.kind, h.Lx, h.Ly, False, s_np)
        scale = np.abs(diag) + np.abs(ref - diag)
        assert np.all(np.abs(o.cpu().numpy() - ref) <= 1e-3 * scale)


def test_graph_capture_and_replay():
    theta = torch.from_numpy(inputs.glorot_params(NL, H, seed=0)).cuda()
    stream = torch.cuda.Stream()
    ctx = B.context(stream)
    B.psr_context_set_graphs(ctx, True)
    items = _items(seed=7)
    fresh = _items(seed=11)
    outs = [torch.empty(s.shape[0], dtype=torch.float32, device="cuda") for s, *_ in items]
    stats = [torch.empty(3, dtype=torch.float64, device="cuda") for _ in items]
    torch.cuda.synchronize()
    p = B.make_params(theta, NL, H, False, "bf16", ctx)
    args = [(s, h, u1, o, st) for (s, h, u1, _), o, st in zip(items, outs, stats)]
    with torch.cuda.stream(stream):
        B.psr_local_energy_batch(p, args)      # capture + launch
        B.psr_context_sync(ctx)
        first = [o.clone() for o in outs]
        B.psr_local_energy_batch(p, args)      # replay
        B.psr_context_sync(ctx)
        for a, b in zip(first, outs):
            assert torch.equal(a, b)
        # new contents in the same buffers: the replay must use them
        for (s, *_), (s2, *_) in zip(items, fresh):
            s.copy_(s2)
        B.psr_local_energy_batch(p, args)
        B.psr_context_sync(ctx)
    torch.cuda.synchronize()
    for (s, h, u1, _), o in zip(items, outs):
        e, _ = api.local_energy(theta, s, api.ModelConfig(NL, H, u1, "bf16"), h)
        api.sync()
        assert torch.equal(o, e)
    B.psr_context_set_graphs(ctx, False)
