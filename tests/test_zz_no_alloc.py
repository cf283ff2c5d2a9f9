"""psr_logpsi_noalloc, the variant of psr_logpsi for callers that may not
allocate device memory (its scratch is a fixed array inside the library).

It must give what psr_logpsi gives, within the tolerances the other GPU tests
use, on consecutive calls that reuse the shared array, and it must leave the
device's free memory unchanged.  This file is collected last on purpose.
"""
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


def _case(n_layers, H, N, n, u1, precision, seed):
    theta = torch.from_numpy(inputs.random_params(n_layers, H, seed=seed, scale=1.0)
                             if precision == "fp32" else inputs.glorot_params(n_layers, H, seed=seed)).cuda()
    spins_np = (inputs.zero_magnetisation_spins(seed, n, N) if u1 else inputs.random_spins(seed, n, N))
    spins = torch.from_numpy(spins_np).cuda()
    return theta, spins, api.ModelConfig(n_layers, H, u1, precision)


def _params(theta, cfg):
    """psr_params without a context (the no-allocation call ignores it)."""
    return B.psr_params(cfg.n_layers, cfg.hidden, int(cfg.u1), B._PRECISION[cfg.precision],
                        B._ptr(theta), None)


def _noalloc(theta, spins, cfg):
    out = torch.full((spins.shape[0],), float("nan"), dtype=torch.float32, device="cuda")
    B.psr_logpsi_noalloc(_params(theta, cfg), spins, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def _reference(theta, spins, cfg):
    out = api.logpsi(theta, spins, cfg)
    api.sync()
    return out.cpu().numpy().astype(np.float64)


def _close(got, ref, precision):
    if precision == "fp32":
        tol = 1e-5 + 1e-6 * np.abs(ref)
    else:
        tol = 2e-2 + 2e-5 * np.abs(ref)
    assert np.all(np.isfinite(got) == np.isfinite(ref))
    fin = np.isfinite(ref)
    assert np.all(np.abs(got[fin] - ref[fin]) <= tol[fin]), np.max(np.abs(got[fin] - ref[fin]))


def test_two_calls_in_a_row_match_psr_logpsi():
    first = _case(3, 64, 100, 300, True, "fp32", 1)
    # 12000 samples of 2704 sites need two batches through the fixed array
    # (11,915 rows of 44 words each fit its 4 MiB spin region)
    second = _case(3, 128, 2704, 12000, True, "bf16", 2)
    ref1 = _reference(*first)
    ref2 = _reference(*second)
    got1 = _noalloc(*first)
    got2 = _noalloc(*second)
    _close(got1, ref1, "fp32")
    _close(got2, ref2, "bf16")
    assert B.psr_noalloc_status() == B.PSR_OK
    # the array keeps the last call's contents; a later call must not depend on them
    _close(_noalloc(*first), ref1, "fp32")


def test_device_free_memory_is_unchanged():
    theta, spins, cfg = _case(3, 128, 100, 500, False, "bf16", 3)
    _noalloc(theta, spins, cfg)  # set-up on this device already done
    out = torch.empty(500, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        B.psr_logpsi_noalloc(_params(theta, cfg), spins, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_rejects_host_arrays_and_oversized_configurations():
    theta, spins, cfg = _case(3, 32, 16, 4, False, "fp32", 4)
    out = torch.empty(4, dtype=torch.float32, device="cuda")
    p = _params(theta, cfg)
    with pytest.raises(B.PsrError) as ei:
        B.psr_logpsi_noalloc(p, spins.cpu(), out)
    assert ei.value.code == B.PSR_EINVAL
    # one configuration longer than the array can hold: rejected on the host
    rc = B.lib().psr_logpsi_noalloc(C.byref(p), C.c_void_p(spins.data_ptr()), 1, 33554369,
                                    C.c_void_p(out.data_ptr()), None)
    assert rc == B.PSR_EINVAL


def test_device_side_failure_is_visible_through_the_status_query():
    """A spin byte other than 0/1 is found by a kernel, after the call has
    returned PSR_OK; the status query reports it, and the next clean call
    clears it."""
    theta, spins, cfg = _case(3, 32, 16, 4, False, "fp32", 5)
    out = torch.empty(4, dtype=torch.float32, device="cuda")
    bad = spins.clone()
    bad[2, 7] = 2
    B.psr_logpsi_noalloc(_params(theta, cfg), bad, out)
    assert B.psr_noalloc_status() == B.PSR_EDEVICE
    got = _noalloc(theta, spins, cfg)
    assert B.psr_noalloc_status() == B.PSR_OK
    _close(got, _reference(theta, spins, cfg), "fp32")
