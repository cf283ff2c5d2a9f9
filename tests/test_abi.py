"""The C-ABI library loads and exports every symbol declared in include/psr.h
(no compute calls: these run without a GPU)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(psr[a-z0-9]*_\w+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpsr():
    from paper_2605_13807_gb300 import binding
    if not os.path.exists(binding.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return binding.lib()


def test_every_declared_symbol_is_exported(libpsr):
    declared = _declared()
    assert "psr_logpsi" in declared and "psr_local_energy" in declared and "psr_grad" in declared
    for name in declared:
        assert hasattr(libpsr, name), name


def test_param_count_host_only(libpsr):
    from paper_2605_13807_gb300 import binding, inputs
    for H in (32, 64, 128):
        assert binding.psr_param_count(3, H) == 9 * H * H + 14 * H + 2 == inputs.param_count(3, H)
    P = C.c_int64()
    assert libpsr.psr_param_count(0, 32, C.byref(P)) == binding.PSR_EINVAL
    assert libpsr.psr_param_count(3, 32, None) == binding.PSR_EINVAL


def test_param_counts_of_the_other_models(libpsr):
    from paper_2605_13807_gb300 import binding, inputs
    for H in (32, 64, 128):
        assert binding.psr2d_param_count(3, H) == 12 * H * H + 118 * H + 16
        assert binding.psr2d_param_count(3, H) == inputs.glorot_params2d(3, H).size
        assert binding.psr_lru_param_count(3, H) == 16 * H * H + 25 * H + 2
        assert binding.psr_lru_param_count(3, H) == inputs.lru_params(3, H).size
    P = C.c_int64()
    assert libpsr.psr2d_param_count(9, 32, C.byref(P)) == binding.PSR_EINVAL
    assert libpsr.psr_lru_param_count(3, 32, None) == binding.PSR_EINVAL


def test_null_arguments_are_rejected_without_touching_the_device(libpsr):
    from paper_2605_13807_gb300 import binding
    assert libpsr.psr_logpsi(None, None, 1, 1, None) == binding.PSR_EINVAL
    assert libpsr.psr_local_energy(None, None, 1, None, None, None) == binding.PSR_EINVAL
    assert libpsr.psr_grad(None, None, 1, 1, None, None) == binding.PSR_EINVAL
    assert libpsr.psr_connected(None, None, 1, None, None, None, 0, None, None) == binding.PSR_EINVAL
    assert libpsr.psr_context_sync(None) == binding.PSR_EINVAL
    assert libpsr.psr2d_logpsi(None, None, 1, 4, 4, None) == binding.PSR_EINVAL
    assert libpsr.psr_lru_logpsi(None, None, 1, 4, None) == binding.PSR_EINVAL
    assert libpsr.psr_lru_sample(None, None, 1, 4, None, None) == binding.PSR_EINVAL
    assert libpsr.psr_lru_grad(None, None, 1, 4, None, None) == binding.PSR_EINVAL
    assert libpsr.psr_lru_vmc_step(None, None, None, 1, None, None, None, None, None, None) == binding.PSR_EINVAL
    assert libpsr.psr2d_sym_logpsi(None, None, 1, 4, 4, None) == binding.PSR_EINVAL
    assert libpsr.psr2d_sym_local_energy(None, None, 1, None, None, None) == binding.PSR_EINVAL
    assert libpsr.psr2d_vmc_step(None, None, 0, None, None, 1, None, None, None, None, None,
                                 None) == binding.PSR_EINVAL
    assert libpsr.psr_sample(None, None, 1, 4, None, None) == binding.PSR_EINVAL
    assert libpsr.psr_scan(None, None, None, None, 1, 4, 4, None) == binding.PSR_EINVAL
    assert libpsr.psr_selftest_wait_timeout(None, None) == binding.PSR_EINVAL
    assert libpsr.psr_context_destroy(None) == binding.PSR_EINVAL
    assert binding.strerror(binding.PSR_ETIMEOUT) == "bounded device wait expired"


def test_library_has_no_oracle_dependency():
    """The product path must not link or import the oracle."""
    from paper_2605_13807_gb300 import binding
    pkg = os.path.join(ROOT, "paper_2605_13807_gb300")
    for mod in os.listdir(pkg):
        if mod.endswith(".py"):
            src = open(os.path.join(pkg, mod)).read()
            assert not re.search(r"^\s*(from|import)\s+oracle\b", src, flags=re.M), mod
            assert "liboracle" not in src, mod
    csrc = os.path.join(ROOT, "paper_2605_13807_gb300", "csrc")
    for f in os.listdir(csrc):
        assert "psr_oracle" not in open(os.path.join(csrc, f)).read()
    assert binding.LIB_PATH.endswith("libpsr.so")


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without libpsr.so every entry point raises: there is no CPU path."""
    import numpy as np

    from paper_2605_13807_gb300 import api, binding, inputs
    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(binding, "LIB_PATH", str(tmp_path / "libpsr.so"))
    with pytest.raises(ImportError):
        binding.lib()
    theta = inputs.glorot_params(3, 32, seed=0)
    spins = np.zeros((2, 8), dtype=np.uint8)
    with pytest.raises(ImportError):
        # (a placeholder context handle: the call must fail before using it)
        binding.psr_logpsi(binding.make_params(theta, 3, 32, ctx=1), spins, np.empty(2, np.float32))
    with pytest.raises(ImportError):
        api.param_count(3, 32)
