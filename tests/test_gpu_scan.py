"""Standalone chunked scan psr_scan (h_t = a_t h_{t-1} + b_t over [n, N, H])
against the FP64 oracle's strictly sequential recurrence, column by column.

Tolerance: the FP32 kernel composes affine maps in a different order than the
sequential loop, so each h_t carries a few rounding errors of the size of the
terms that build it.  The bound is 1e-5 * M_t, where M_t is the same
recurrence run on |a|, |b|, |h0| (the largest value any partial sum can take),
i.e. about 170 FP32 ulps of that magnitude.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2605_13807_gb300 import api, binding as B, inputs  # noqa: E402

TILES = [(4, 32), (16, 96), (32, 100), (128, 64), (4, 10 ** 9), (16, 10 ** 9), (32, 10 ** 9),
         (128, 10 ** 9), (128, 1000)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    yield


def _oracle_columns(orc, a, b, h0, cols):
    """(reference, magnitude bound) for the listed (sequence, unit) columns."""
    ref, mag = [], []
    for i, u in cols:
        x0 = 0.0 if h0 is None else float(h0[i, u])
        ref.append(orc.scan_sequential(a[i, :, u], b[i, :, u], x0))
        mag.append(orc.scan_sequential(np.abs(a[i, :, u]), np.abs(b[i, :, u]), abs(x0)))
    return np.array(ref), np.array(mag)


def _check(orc, a, b, h0, h, cols=None):
    n, N, H = a.shape
    if cols is None:
        cols = [(i, u) for i in range(n) for u in range(H)]
    ref, mag = _oracle_columns(orc, a, b, h0, cols)
    got = np.array([h[i, :, u] for i, u in cols], dtype=np.float64)
    err = np.abs(got - ref)
    assert np.all(err <= 1e-5 * mag), (err / mag).max()


@pytest.mark.parametrize("tile", TILES)
@pytest.mark.parametrize("shape,with_h0", [((3, 1000, 128), True), ((2, 777, 64), False)])
def test_every_tile_shape_matches_oracle(oracle_mod, tile, shape, with_h0):
    n, N, H = shape
    if H % tile[0]:
        pytest.skip("unit block does not divide H")
    a, b, h0 = inputs.scan_inputs(11, n, N, H)
    ta, tb, th0 = (torch.from_numpy(x).cuda() for x in (a, b, h0))
    h = api.scan(ta, tb, th0 if with_h0 else None, tile=tile)
    api.sync()
    _check(oracle_mod, a, b, h0 if with_h0 else None, h.cpu().numpy())


def test_long_single_sequence_many_chunks(oracle_mod):
    # one sequence of 20 000 sites, 4 units: 625 chunks of 32 chained by look-back
    a, b, h0 = inputs.scan_inputs(12, 1, 20000, 4)
    ta, tb, th0 = (torch.from_numpy(x).cuda() for x in (a, b, h0))
    for tile in [(4, 32), (4, 256), (4, 20000)]:
        h = api.scan(ta, tb, th0, tile=tile)
        api.sync()
        _check(oracle_mod, a, b, h0, h.cpu().numpy())


def test_default_and_autotuned_tiles(oracle_mod):
    a, b, h0 = inputs.scan_inputs(13, 4, 600, 32)
    ta, tb, th0 = (torch.from_numpy(x).cuda() for x in (a, b, h0))
    ctx = B.context()
    tile, tuned = B.psr_scan_tile_for(ctx, 4, 600, 32)
    assert not tuned and 32 % tile[0] == 0
    h = api.scan(ta, tb, th0)
    api.sync()
    _check(oracle_mod, a, b, h0, h.cpu().numpy())
    api.set_autotune(True)
    try:
        h2 = api.scan(ta, tb, th0)
        api.sync()
        tile2, tuned2 = B.psr_scan_tile_for(ctx, 4, 600, 32)
        assert tuned2 and 32 % tile2[0] == 0 and tile2[0] in (4, 16, 32, 128)
        _check(oracle_mod, a, b, h0, h2.cpu().numpy())
        # a tuned shape is remembered: the next call uses it without re-tuning
        h3 = api.scan(ta, tb, th0)
        api.sync()
        assert torch.equal(h3, h2)
    finally:
        api.set_autotune(False)


def test_host_arrays_and_in_place(oracle_mod):
    a, b, h0 = inputs.scan_inputs(14, 2, 300, 16)
    h = np.empty_like(a)
    B.psr_scan(B.context(), a, b, h, h0=h0, tile=(16, 64))
    _check(oracle_mod, a, b, h0, h)
    # h may alias b
    ta, tb, th0 = (torch.from_numpy(x).cuda() for x in (a, b, h0))
    B.psr_scan(B.context(), ta, tb, tb, h0=th0, tile=(4, 32))
    api.sync()
    _check(oracle_mod, a, b, h0, tb.cpu().numpy())


def test_rejects_bad_arguments():
    a = torch.rand((2, 50, 8), device="cuda")
    h = torch.empty_like(a)
    ctx = B.context()
    with pytest.raises(B.PsrError) as ei:  # units must divide H
        B.psr_scan(ctx, a, a, h, tile=(16, 32))
    assert ei.value.code == B.PSR_EINVAL
    with pytest.raises(B.PsrError) as ei:  # not a unit-block width
        B.psr_scan(ctx, a, a, h, tile=(8, 32))
    assert ei.value.code == B.PSR_EINVAL
    bad = torch.rand((2, 50, 6), device="cuda")  # H not a multiple of 4
    with pytest.raises(B.PsrError) as ei:
        B.psr_scan(ctx, bad, bad, torch.empty_like(bad))
    assert ei.value.code == B.PSR_EINVAL
    import ctypes as C
    base = torch.rand(2 * 50 * 8 + 1, device="cuda")
    rc = B.lib().psr_scan(C.c_void_p(ctx), C.c_void_p(base.data_ptr() + 4), C.c_void_p(a.data_ptr()),
                          None, 2, 50, 8, C.c_void_p(h.data_ptr()))
    assert rc == B.PSR_EINVAL  # misaligned device array
    rc = B.lib().psr_scan(C.c_void_p(ctx), C.c_void_p(a.data_ptr()), C.c_void_p(a.data_ptr()),
                          None, 0, 50, 8, C.c_void_p(h.data_ptr()))
    assert rc == B.PSR_EINVAL  # no sequences


def test_full_size_sampled_columns(oracle_mod):
    """4096 sequences x 2704 sites x 128 units (the 52x52 workload's layer
    shape), default and tuned tiles, checked on 48 sampled columns."""
    n, N, H = 4096, 2704, 128
    ta, tb, th0 = inputs.scan_inputs_device(15, n, N, H, "cuda")
    h = api.scan(ta, tb, th0)
    api.sync()
    rng = np.random.default_rng(0)
    cols = [(int(i), int(u)) for i, u in zip(rng.integers(0, n, 48), rng.integers(0, H, 48))]
    cols += [(0, 0), (n - 1, H - 1)]
    idx_i = torch.tensor([c[0] for c in cols], device="cuda")
    idx_u = torch.tensor([c[1] for c in cols], device="cuda")

    def columns(x):
        return x[idx_i, :, idx_u].cpu().numpy()   # [cols, N]

    a_c, b_c, h_c = columns(ta), columns(tb), columns(h)
    h0_c = th0[idx_i, idx_u].cpu().numpy()
    a_s = a_c[:, None, :].transpose(0, 2, 1)      # as [cols, N, 1] sequences
    b_s = b_c[:, None, :].transpose(0, 2, 1)
    sub = [(k, 0) for k in range(len(cols))]
    _check(oracle_mod, a_s, b_s, h0_c[:, None], h_c[:, :, None], sub)


def test_bounded_wait_expires_and_context_recovers(oracle_mod):
    """A look-back wait on a flag that nothing sets gives up after its limit,
    reports PSR_ETIMEOUT through the status word and leaves the context
    usable (failure detection without a GPU fault)."""
    ctx = B.context()
    rc, ms = B.psr_selftest_wait_timeout(ctx)
    assert rc == B.PSR_ETIMEOUT
    assert 1500.0 <= ms <= 20000.0, ms
    B.psr_context_sync(ctx)  # the status word was cleared
    a, b, h0 = inputs.scan_inputs(16, 2, 300, 16)
    ta, tb, th0 = (torch.from_numpy(x).cuda() for x in (a, b, h0))
    h = api.scan(ta, tb, th0, tile=(16, 64))
    api.sync()
    _check(oracle_mod, a, b, h0, h.cpu().numpy())
