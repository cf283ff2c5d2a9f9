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


# ------------------------------------------- psr_step_batch: the whole step

def _single(theta, s, h, u1, precision):
    cfg = api.ModelConfig(NL, H, u1, precision)
    lp = api.logpsi(theta, s, cfg)
    e, st = api.local_energy(theta, s, cfg, h)
    g = api.grad(theta, s, cfg)
    api.sync()
    return lp, e, st, g


@pytest.mark.parametrize("precision,shape", [("bf16", 1), ("bf16", 2), ("fp32", 32), ("fp32", 16)])
def test_step_batch_equals_single_calls(precision, shape):
    theta = torch.from_numpy(inputs.glorot_params(NL, H, seed=0)).cuda()
    items = _items(seed=3)
    api.set_fwd_shape(precision, shape)
    try:
        outs = api.step_batch(theta, [(s, h, u1) for s, h, u1, _ in items],
                              api.ModelConfig(NL, H, False, precision))
        api.sync()
        for (s, h, u1, _), o in zip(items, outs):
            lp, e, st, g = _single(theta, s, h, u1, precision)
            assert torch.equal(o["logpsi"], lp)
            assert torch.equal(o["eloc"], e) and torch.equal(o["stats"], st)
            assert torch.equal(o["grad"], g)
    finally:
        api.set_fwd_shape(precision, 0)


def test_step_batch_partial_outputs_and_host_arrays():
    theta_np = inputs.glorot_params(NL, H, seed=1)
    theta = torch.from_numpy(theta_np).cuda()
    items = _items(seed=4)
    cfg = api.ModelConfig(NL, H, False, "bf16")
    p = B.make_params(theta, NL, H, False, "bf16", api._ctx())
    P = theta.numel()
    (s0, h0, u0, s0_np), (s1, h1, u1_, s1_np) = items[0], items[3]
    g0 = torch.empty((s0.shape[0], P), device="cuda")
    lp1 = torch.empty(s1.shape[0], device="cuda")
    B.psr_step_batch(p, [(s0, h0, u0, None, None, None, g0), (s1, h1, u1_, lp1, None, None, None)])
    api.sync()
    assert torch.equal(g0, api.grad(theta, s0, api.ModelConfig(NL, H, u0, "bf16")))
    assert torch.equal(lp1, api.logpsi(theta, s1, api.ModelConfig(NL, H, u1_, "bf16")))
    # host arrays everywhere: staged through the workspace, same values
    ph = B.make_params(theta_np, NL, H, False, "bf16", api._ctx())
    lph = np.empty(s0_np.shape[0], dtype=np.float32)
    elh = np.empty(s0_np.shape[0], dtype=np.float32)
    sth = np.empty(3, dtype=np.float64)
    gh = np.empty((s0_np.shape[0], P), dtype=np.float32)
    B.psr_step_batch(ph, [(s0_np, h0, u0, lph, elh, sth, gh)])
    lp, e, st, g = _single(theta, s0, h0, u0, "bf16")
    assert np.array_equal(lph, lp.cpu().numpy()) and np.array_equal(elh, e.cpu().numpy())
    assert np.array_equal(sth, st.cpu().numpy()) and np.array_equal(gh, g.cpu().numpy())
    # rejected: no output, stats without eloc
    with pytest.raises(B.PsrError) as ei:
        B.psr_step_batch(p, [(s0, h0, u0, None, None, None, None)])
    assert ei.value.code == B.PSR_EINVAL
    st_d = torch.empty(3, dtype=torch.float64, device="cuda")
    with pytest.raises(B.PsrError) as ei:
        B.psr_step_batch(p, [(s0, h0, u0, lp1[:0], None, st_d, None)])
    assert ei.value.code == B.PSR_EINVAL


def _mixed_lattice_items(n):
    """16x16, 24x24, 32x32 open Heisenberg (Neel-like, zero magnetisation) and
    the 20x20 open TFIM at h/J = 3.044 (uniform random spins)."""
    spec = [("heisenberg", 16, True, 0.0), ("heisenberg", 24, True, 0.0), ("heisenberg", 32, True, 0.0),
            ("tfim", 20, False, 3.044)]
    out = []
    for k, (kind, L, u1, hf) in enumerate(spec):
        s = (inputs.neel_like_spins(2000 + k, n, L, L) if kind == "heisenberg"
             else inputs.random_spins(2000 + k, n, L * L))
        out.append((torch.from_numpy(s).cuda(), B.make_hamiltonian(kind, L, L, False, True, 1.0, hf), u1, s))
    return out


def test_step_batch_at_the_mixed_lattice_sizes(oracle_mod):
    """The mixed batch at its full size (2048 samples per lattice, BF16):
    every output bitwise equal to the single calls; sampled outputs against
    the FP64 oracle (log psi of samples of every lattice, E_loc of a 16x16 and
    a 20x20 sample assembled from the oracle's log psi of all their connected
    configurations, O_k rows of 16x16 samples); graph replay unchanged."""
    n = 2048
    theta_np = inputs.glorot_params(NL, H, seed=0)
    theta = torch.from_numpy(theta_np).cuda()
    items = _mixed_lattice_items(n)
    cfg = api.ModelConfig(NL, H, False, "bf16")
    outs = api.step_batch(theta, [(s, h, u1) for s, h, u1, _ in items], cfg)
    api.sync()
    for (s, h, u1, s_np), o in zip(items, outs):
        lp, e, st, g = _single(theta, s, h, u1, "bf16")
        assert torch.equal(o["logpsi"], lp)
        assert torch.equal(o["eloc"], e) and torch.equal(o["stats"], st)
        assert torch.equal(o["grad"], g)
        del lp, e, st, g
        assert torch.all(torch.isfinite(o["eloc"]))
        # log psi of sampled samples against the oracle
        pick = [0, 777, n - 1]
        ref = oracle_mod.logpsi(theta_np, NL, H, s_np[pick], u1=u1, threads=16)
        got = o["logpsi"][pick].cpu().numpy().astype(np.float64)
        assert np.all(np.abs(got - ref) <= 2e-2 + 2e-5 * np.abs(ref)), (h.Lx, np.abs(got - ref).max())
    # E_loc of one 16x16 and one 20x20 sample from the oracle's log psi of
    # every connected configuration
    for k in (0, 3):
        s, h, u1, s_np = items[k]
        i = 5
        offs, ent, diag = oracle_mod.connected(h.kind, h.Lx, h.Ly, False, s_np[i:i + 1])
        sp = np.repeat(s_np[i:i + 1], ent.shape[0], axis=0)
        r = np.arange(ent.shape[0])
        sp[r, ent[:, 1]] ^= 1
        q = ent[:, 2] >= 0
        sp[r[q], ent[q, 2]] ^= 1
        lp_c = oracle_mod.logpsi(theta_np, NL, H, sp, u1=u1, threads=16)
        lp_s = oracle_mod.logpsi(theta_np, NL, H, s_np[i:i + 1], u1=u1)[0]
        c = oracle_mod.offdiag_coeff(h.kind, J=1.0, h=h.h, marshall=True)
        ref = oracle_mod.eloc_combine(diag[0], c, lp_s, lp_c)
        got = float(outs[k]["eloc"][i].item())
        scale = abs(diag[0]) + abs(ref - diag[0])
        assert abs(got - ref) <= 1e-3 * scale, (h.Lx, got, ref)
    # O_k rows of 16x16 samples against the oracle's reverse mode
    s, h, u1, s_np = items[0]
    _, ref_g = oracle_mod.grad(theta_np, NL, H, s_np[[1, 1000]], u1=u1)
    g = outs[0]["grad"][[1, 1000]].cpu().numpy().astype(np.float64)
    for a, b in zip(g, ref_g):
        assert np.linalg.norm(a - b) <= 1e-3 * np.linalg.norm(b)
    # graph capture and replay of the whole step
    first = [{k: v.clone() for k, v in o.items()} for o in outs]
    stream = torch.cuda.Stream()
    ctx = B.context(stream)
    B.psr_context_set_graphs(ctx, True)
    try:
        p = B.make_params(theta, NL, H, False, "bf16", ctx)
        args = [(s, h, u1, o["logpsi"], o["eloc"], o["stats"], o["grad"]) for (s, h, u1, _), o in zip(items, outs)]
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            for _ in range(2):  # capture + launch, then replay
                for o in outs:
                    for v in o.values():
                        v.zero_()
                B.psr_step_batch(p, args)
                B.psr_context_sync(ctx)
                for a, b in zip(first, outs):
                    for key in a:
                        assert torch.equal(a[key], b[key]), key
    finally:
        B.psr_context_set_graphs(ctx, False)
