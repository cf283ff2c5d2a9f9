"""Thin ctypes binding of libpsr (argument marshalling only).

Every function here forwards to the C entry point of the same name declared
in include/psr.h; no computation happens in Python.  Arrays are torch tensors
(device or host) or numpy arrays (host); their data pointers are passed as
is, and the library itself stages host arrays.  If libpsr.so has not been
built this module raises at import of the library, never falls back.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpsr.so")

PSR_OK, PSR_EINVAL, PSR_ENOMEM, PSR_ECUDA, PSR_ETIMEOUT, PSR_EDEVICE, PSR_EUNSUPPORTED = range(7)
PSR_FP32, PSR_BF16, PSR_FP16 = 0, 1, 2
PSR_HEISENBERG, PSR_TFIM = 0, 1

_PRECISION = {"fp32": PSR_FP32, "bf16": PSR_BF16, "fp16": PSR_FP16, PSR_FP32: PSR_FP32, PSR_BF16: PSR_BF16,
              PSR_FP16: PSR_FP16}


class PsrError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} (code {code})")


class psr_params(C.Structure):
    _fields_ = [("n_layers", C.c_int32), ("hidden", C.c_int32), ("u1_mask", C.c_int32),
                ("precision", C.c_int32), ("theta", C.c_void_p), ("ctx", C.c_void_p)]


class psr_hamiltonian(C.Structure):
    _fields_ = [("kind", C.c_int32), ("Lx", C.c_int32), ("Ly", C.c_int32), ("pbc", C.c_int32),
                ("marshall", C.c_int32), ("J", C.c_double), ("h", C.c_double)]


class psr_scan_tile(C.Structure):
    _fields_ = [("units", C.c_int32), ("chunk", C.c_int32)]


class psr_adam(C.Structure):
    _fields_ = [("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("step", C.c_int32), ("m", C.c_void_p), ("v", C.c_void_p)]


class psr_batch_item(C.Structure):
    _fields_ = [("samples", C.c_void_p), ("n", C.c_int64), ("ham", psr_hamiltonian),
                ("u1_mask", C.c_int32), ("out", C.c_void_p), ("stats", C.c_void_p)]


class psr_step_item(C.Structure):
    _fields_ = [("samples", C.c_void_p), ("n", C.c_int64), ("ham", psr_hamiltonian),
                ("u1_mask", C.c_int32), ("logpsi", C.c_void_p), ("eloc", C.c_void_p),
                ("stats", C.c_void_p), ("grad", C.c_void_p)]


EXPORTED = ("psr_context_create", "psr_context_destroy", "psr_context_sync", "psr_param_count",
            "psr_logpsi", "psr_local_energy", "psr_connected", "psr_grad", "psr_strerror",
            "psr_context_set_profiling", "psr_context_stage_ms", "psr_logpsi_noalloc",
            "psr_local_energy_batch", "psr_context_set_graphs", "psr_scan", "psr_scan_tiled",
            "psr_scan_tile_for", "psr_context_set_autotune", "psr_sample", "psr_sample_tile_for",
            "psr2d_param_count", "psr2d_logpsi", "psr2d_local_energy", "psr_selftest_wait_timeout",
            "psr_lru_param_count", "psr_lru_logpsi", "psr_lru_local_energy", "psr_sym_logpsi",
            "psr_sym_local_energy", "psr_vmc_step", "psr2d_sample", "psr2d_grad", "psr2d_vmc_step",
            "psr_lru_sample", "psr_lru_grad", "psr_lru_vmc_step", "psr2d_sym_logpsi",
            "psr2d_sym_local_energy", "psr_noalloc_status", "psr_step_batch",
            "psr_context_set_fwd_shape", "psr_fwd_shape_for")
STAGES = ("pack", "generator", "fwd_samples", "fwd_connected", "gather", "bwd", "scan", "sample")

_lib = None
_lock = threading.Lock()


def lib():
    """The loaded libpsr.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        with _lock:
            if _lib is None:
                if not os.path.exists(LIB_PATH):
                    raise ImportError(f"{LIB_PATH} is missing: build it with "
                                      "`python -c 'import __graft_entry__ as g; g.build()'`")
                L = C.CDLL(LIB_PATH)
                vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
                L.psr_context_create.argtypes = [C.POINTER(vp), vp]
                L.psr_context_destroy.argtypes = [vp]
                L.psr_context_sync.argtypes = [vp]
                L.psr_param_count.argtypes = [i32, i32, C.POINTER(i64)]
                L.psr_logpsi.argtypes = [C.POINTER(psr_params), vp, i64, i32, vp]
                L.psr_local_energy.argtypes = [C.POINTER(psr_params), vp, i64,
                                               C.POINTER(psr_hamiltonian), vp, vp]
                L.psr_connected.argtypes = [vp, vp, i64, C.POINTER(psr_hamiltonian), vp, vp, i64, vp,
                                            C.POINTER(i64)]
                L.psr_grad.argtypes = [C.POINTER(psr_params), vp, i64, i32, vp, vp]
                L.psr_logpsi_noalloc.argtypes = [C.POINTER(psr_params), vp, i64, i32, vp, vp]
                L.psr_noalloc_status.argtypes = [vp]
                L.psr_local_energy_batch.argtypes = [C.POINTER(psr_params), C.POINTER(psr_batch_item), i32]
                L.psr_step_batch.argtypes = [C.POINTER(psr_params), C.POINTER(psr_step_item), i32]
                L.psr_context_set_fwd_shape.argtypes = [vp, i32, i32]
                L.psr_fwd_shape_for.argtypes = [vp, i32, i32, i32, C.POINTER(i64), C.POINTER(i32),
                                                C.POINTER(i32), C.POINTER(i32)]
                L.psr_context_set_graphs.argtypes = [vp, C.c_int]
                L.psr_context_set_profiling.argtypes = [vp, C.c_int]
                L.psr_context_stage_ms.argtypes = [vp, C.c_int, C.POINTER(C.c_float)]
                L.psr_scan.argtypes = [vp, vp, vp, vp, i64, i32, i32, vp]
                L.psr_scan_tiled.argtypes = [vp, vp, vp, vp, i64, i32, i32, vp, C.POINTER(psr_scan_tile)]
                L.psr_scan_tile_for.argtypes = [vp, i64, i32, i32, C.POINTER(psr_scan_tile),
                                                C.POINTER(i32)]
                L.psr_context_set_autotune.argtypes = [vp, C.c_int]
                L.psr_sample.argtypes = [C.POINTER(psr_params), vp, i64, i32, vp, vp]
                L.psr_sample_tile_for.argtypes = [vp, i64, i32, i32, i32, C.POINTER(i32), C.POINTER(i32)]
                L.psr2d_param_count.argtypes = [i32, i32, C.POINTER(i64)]
                L.psr2d_logpsi.argtypes = [C.POINTER(psr_params), vp, i64, i32, i32, vp]
                L.psr2d_local_energy.argtypes = [C.POINTER(psr_params), vp, i64,
                                                 C.POINTER(psr_hamiltonian), vp, vp]
                L.psr_selftest_wait_timeout.argtypes = [vp, C.POINTER(C.c_float)]
                L.psr_lru_param_count.argtypes = [i32, i32, C.POINTER(i64)]
                L.psr_lru_logpsi.argtypes = [C.POINTER(psr_params), vp, i64, i32, vp]
                L.psr_lru_local_energy.argtypes = [C.POINTER(psr_params), vp, i64,
                                                   C.POINTER(psr_hamiltonian), vp, vp]
                L.psr_sym_logpsi.argtypes = [C.POINTER(psr_params), vp, i64, i32, i32, vp]
                L.psr_sym_local_energy.argtypes = [C.POINTER(psr_params), vp, i64,
                                                   C.POINTER(psr_hamiltonian), vp, vp]
                L.psr_vmc_step.argtypes = [C.POINTER(psr_params), C.POINTER(psr_hamiltonian), i32, vp, vp,
                                           i64, C.POINTER(psr_adam), vp, vp, vp, vp, vp]
                L.psr2d_sample.argtypes = [C.POINTER(psr_params), vp, i64, i32, i32, vp, vp]
                L.psr2d_grad.argtypes = [C.POINTER(psr_params), vp, i64, i32, i32, vp, vp]
                L.psr2d_vmc_step.argtypes = [C.POINTER(psr_params), C.POINTER(psr_hamiltonian), i32, vp, vp,
                                             i64, C.POINTER(psr_adam), vp, vp, vp, vp, vp]
                L.psr2d_sym_logpsi.argtypes = [C.POINTER(psr_params), vp, i64, i32, i32, vp]
                L.psr2d_sym_local_energy.argtypes = [C.POINTER(psr_params), vp, i64,
                                                     C.POINTER(psr_hamiltonian), vp, vp]
                L.psr_lru_sample.argtypes = [C.POINTER(psr_params), vp, i64, i32, vp, vp]
                L.psr_lru_grad.argtypes = [C.POINTER(psr_params), vp, i64, i32, vp, vp]
                L.psr_lru_vmc_step.argtypes = [C.POINTER(psr_params), C.POINTER(psr_hamiltonian), vp, i64,
                                               C.POINTER(psr_adam), vp, vp, vp, vp, vp]
                L.psr_strerror.argtypes = [C.c_int]
                L.psr_strerror.restype = C.c_char_p
                for name in EXPORTED:
                    if name != "psr_strerror":
                        getattr(L, name).restype = C.c_int
                _lib = L
    return _lib


def strerror(code: int) -> str:
    return lib().psr_strerror(int(code)).decode()


def _check(code, where):
    if code != PSR_OK:
        raise PsrError(code, where)


# ------------------------------------------------------------------ contexts

_contexts = {}


def context(stream=None):
    """A psr_context bound to a CUDA stream (default: torch's current stream)."""
    import torch
    dev = torch.cuda.current_device()
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    handle = int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream or 0)
    key = (dev, handle)
    ctx = _contexts.get(key)
    if ctx is None:
        out = C.c_void_p()
        _check(lib().psr_context_create(C.byref(out), C.c_void_p(handle)), "psr_context_create")
        ctx = out.value
        _contexts[key] = ctx
    return ctx


def psr_context_sync(ctx=None):
    _check(lib().psr_context_sync(C.c_void_p(ctx if ctx else context())), "psr_context_sync")


def psr_context_set_profiling(ctx, enable=True):
    _check(lib().psr_context_set_profiling(C.c_void_p(ctx), int(bool(enable))),
           "psr_context_set_profiling")


def psr_context_stage_ms(ctx):
    """{stage name: ms} of the most recent call on the context."""
    out = {}
    for i, name in enumerate(STAGES):
        ms = C.c_float()
        _check(lib().psr_context_stage_ms(C.c_void_p(ctx), i, C.byref(ms)), "psr_context_stage_ms")
        out[name] = float(ms.value)
    return out


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return C.c_void_p(a.ctypes.data)
    assert a.is_contiguous()
    return C.c_void_p(a.data_ptr())


def make_params(theta, n_layers, hidden, u1=False, precision="fp32", ctx=None):
    return psr_params(int(n_layers), int(hidden), int(bool(u1)), _PRECISION[precision],
                      _ptr(theta), C.c_void_p(ctx if ctx else context()))


def make_hamiltonian(kind, Lx, Ly=1, pbc=False, marshall=True, J=1.0, h=0.0):
    k = {"heisenberg": PSR_HEISENBERG, "tfim": PSR_TFIM}.get(kind, kind)
    return psr_hamiltonian(int(k), int(Lx), int(Ly), int(bool(pbc)), int(bool(marshall)),
                           float(J), float(h))


# ------------------------------------------------------------- entry points

def psr_param_count(n_layers, hidden):
    P = C.c_int64()
    _check(lib().psr_param_count(int(n_layers), int(hidden), C.byref(P)), "psr_param_count")
    return int(P.value)


def psr_logpsi(params, spins, out):
    n, L = spins.shape
    _check(lib().psr_logpsi(C.byref(params), _ptr(spins), int(n), int(L), _ptr(out)), "psr_logpsi")
    return out


def psr_local_energy(params, samples, ham, out, stats=None):
    n = samples.shape[0]
    _check(lib().psr_local_energy(C.byref(params), _ptr(samples), int(n), C.byref(ham), _ptr(out),
                                  _ptr(stats)), "psr_local_energy")
    return out


def psr_connected(ctx, samples, ham, offsets, entries, diag):
    n = samples.shape[0]
    total = C.c_int64()
    _check(lib().psr_connected(C.c_void_p(ctx), _ptr(samples), int(n), C.byref(ham), _ptr(offsets),
                               _ptr(entries), int(entries.shape[0]), _ptr(diag), C.byref(total)),
           "psr_connected")
    return int(total.value)


def psr_grad(params, spins, dout, dparams):
    n, L = spins.shape
    _check(lib().psr_grad(C.byref(params), _ptr(spins), int(n), int(L), _ptr(dout), _ptr(dparams)),
           "psr_grad")
    return dparams


def psr_logpsi_noalloc(params, spins, out, stream=None):
    """log psi with the library's fixed scratch array (no device allocation);
    queued on `stream` (a torch stream or a raw handle; default: torch's
    current stream) without synchronising."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    handle = int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream or 0)
    n, L = spins.shape
    _check(lib().psr_logpsi_noalloc(C.byref(params), _ptr(spins), int(n), int(L), _ptr(out),
                                    C.c_void_p(handle)), "psr_logpsi_noalloc")
    return out


def psr_noalloc_status(stream=None):
    """Device-side status code of the last psr_logpsi_noalloc call on the
    current device (waits for `stream`; allocates nothing)."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    handle = int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream or 0)
    return int(lib().psr_noalloc_status(C.c_void_p(handle)))


def psr_context_set_graphs(ctx, enable=True):
    _check(lib().psr_context_set_graphs(C.c_void_p(ctx), int(bool(enable))), "psr_context_set_graphs")


def psr_local_energy_batch(params, items):
    """items: sequence of (samples, hamiltonian, u1_mask, out, stats-or-None)."""
    arr = (psr_batch_item * len(items))()
    for k, (samples, ham, u1, out, stats) in enumerate(items):
        arr[k].samples = _ptr(samples)
        arr[k].n = int(samples.shape[0])
        arr[k].ham = ham
        arr[k].u1_mask = int(bool(u1))
        arr[k].out = _ptr(out)
        arr[k].stats = _ptr(stats)
    _check(lib().psr_local_energy_batch(C.byref(params), arr, len(items)), "psr_local_energy_batch")


def psr_step_batch(params, items):
    """items: sequence of (samples, hamiltonian, u1_mask, logpsi, eloc, stats, grad),
    each output an array or None."""
    arr = (psr_step_item * len(items))()
    for k, (samples, ham, u1, logpsi, eloc, stats, grad) in enumerate(items):
        arr[k].samples = _ptr(samples)
        arr[k].n = int(samples.shape[0])
        arr[k].ham = ham
        arr[k].u1_mask = int(u1)
        arr[k].logpsi = _ptr(logpsi)
        arr[k].eloc = _ptr(eloc)
        arr[k].stats = _ptr(stats)
        arr[k].grad = _ptr(grad)
    _check(lib().psr_step_batch(C.byref(params), arr, len(items)), "psr_step_batch")


def psr_context_set_fwd_shape(ctx, precision, shape):
    """Fixes the fused forward's shape (BF16: 1 or 2 sequences per MMA stream;
    FP32: 32- or 16-site chunks); 0 returns the choice to the context."""
    _check(lib().psr_context_set_fwd_shape(C.c_void_p(ctx), _PRECISION[precision], int(shape)),
           "psr_context_set_fwd_shape")


def psr_fwd_shape_for(ctx, precision, what, n, L):
    """(shape, tuned) a call would use: what 0 = log psi, 1 = E_loc (n, L
    integers), 2 = a batch whose items all ask for E_loc (n, L sequences)."""
    ns = [int(x) for x in (n if what == 2 else [n])]
    Ls = [int(x) for x in (L if what == 2 else [L])]
    na = (C.c_int64 * len(ns))(*ns)
    la = (C.c_int32 * len(Ls))(*Ls)
    shape = C.c_int32()
    tuned = C.c_int32()
    _check(lib().psr_fwd_shape_for(C.c_void_p(ctx), _PRECISION[precision], int(what), len(ns), na, la,
                                   C.byref(shape), C.byref(tuned)), "psr_fwd_shape_for")
    return shape.value, bool(tuned.value)


def psr_scan(ctx, a, b, h, h0=None, tile=None):
    """h_t = a_t h_{t-1} + b_t over [n, N, H] arrays; tile = (units, chunk)
    forces a tile shape (psr_scan_tiled), None lets the context choose."""
    n, N, H = a.shape
    if tile is None:
        _check(lib().psr_scan(C.c_void_p(ctx), _ptr(a), _ptr(b), _ptr(h0), int(n), int(N), int(H),
                              _ptr(h)), "psr_scan")
    else:
        t = psr_scan_tile(int(tile[0]), int(tile[1]))
        _check(lib().psr_scan_tiled(C.c_void_p(ctx), _ptr(a), _ptr(b), _ptr(h0), int(n), int(N),
                                    int(H), _ptr(h), C.byref(t)), "psr_scan_tiled")
    return h


def psr_scan_tile_for(ctx, n, N, H):
    """((units, chunk), tuned) that psr_scan would use for this shape."""
    t = psr_scan_tile()
    tuned = C.c_int32()
    _check(lib().psr_scan_tile_for(C.c_void_p(ctx), int(n), int(N), int(H), C.byref(t),
                                   C.byref(tuned)), "psr_scan_tile_for")
    return (int(t.units), int(t.chunk)), bool(tuned.value)


def psr_context_set_autotune(ctx, enable=True):
    _check(lib().psr_context_set_autotune(C.c_void_p(ctx), int(bool(enable))),
           "psr_context_set_autotune")


def psr_sample(params, uniforms, spins, logpsi=None):
    """Exact autoregressive samples: spins[i, t] = 1 iff uniforms[i, t] < P(up)."""
    n, L = uniforms.shape
    _check(lib().psr_sample(C.byref(params), _ptr(uniforms), int(n), int(L), _ptr(spins),
                            _ptr(logpsi)), "psr_sample")
    return spins


def psr_sample_tile_for(ctx, n, L, n_layers, hidden):
    """(samples per CTA, tuned) that psr_sample would use for this shape."""
    per = C.c_int32()
    tuned = C.c_int32()
    _check(lib().psr_sample_tile_for(C.c_void_p(ctx), int(n), int(L), int(n_layers), int(hidden),
                                     C.byref(per), C.byref(tuned)), "psr_sample_tile_for")
    return int(per.value), bool(tuned.value)


def psr2d_param_count(n_layers, hidden):
    P = C.c_int64()
    _check(lib().psr2d_param_count(int(n_layers), int(hidden), C.byref(P)), "psr2d_param_count")
    return int(P.value)


def psr2d_logpsi(params, spins, Lx, Ly, out):
    n = spins.shape[0]
    _check(lib().psr2d_logpsi(C.byref(params), _ptr(spins), int(n), int(Lx), int(Ly), _ptr(out)),
           "psr2d_logpsi")
    return out


def psr2d_local_energy(params, samples, ham, out, stats=None):
    n = samples.shape[0]
    _check(lib().psr2d_local_energy(C.byref(params), _ptr(samples), int(n), C.byref(ham), _ptr(out),
                                    _ptr(stats)), "psr2d_local_energy")
    return out


def psr_selftest_wait_timeout(ctx):
    """(return code, device ms) of the bounded-wait self-test; the code is
    PSR_ETIMEOUT when the bound works."""
    ms = C.c_float()
    rc = lib().psr_selftest_wait_timeout(C.c_void_p(ctx), C.byref(ms))
    return int(rc), float(ms.value)


def psr_lru_param_count(n_layers, hidden):
    P = C.c_int64()
    _check(lib().psr_lru_param_count(int(n_layers), int(hidden), C.byref(P)), "psr_lru_param_count")
    return int(P.value)


def psr_lru_logpsi(params, spins, out):
    n, L = spins.shape
    _check(lib().psr_lru_logpsi(C.byref(params), _ptr(spins), int(n), int(L), _ptr(out)),
           "psr_lru_logpsi")
    return out


def psr_lru_local_energy(params, samples, ham, out, stats=None):
    n = samples.shape[0]
    _check(lib().psr_lru_local_energy(C.byref(params), _ptr(samples), int(n), C.byref(ham), _ptr(out),
                                      _ptr(stats)), "psr_lru_local_energy")
    return out


def psr_sym_logpsi(params, spins, Lx, Ly, out):
    n = spins.shape[0]
    _check(lib().psr_sym_logpsi(C.byref(params), _ptr(spins), int(n), int(Lx), int(Ly), _ptr(out)),
           "psr_sym_logpsi")
    return out


def psr_sym_local_energy(params, samples, ham, out, stats=None):
    n = samples.shape[0]
    _check(lib().psr_sym_local_energy(C.byref(params), _ptr(samples), int(n), C.byref(ham), _ptr(out),
                                      _ptr(stats)), "psr_sym_local_energy")
    return out


def psr_vmc_step(params, ham, symmetrize, uniforms, sym_uniforms, adam, theta_out, spins_out=None,
                 eloc_out=None, stats_out=None, grad_out=None):
    n = uniforms.shape[0]
    _check(lib().psr_vmc_step(C.byref(params), C.byref(ham), int(bool(symmetrize)), _ptr(uniforms),
                              _ptr(sym_uniforms), int(n), C.byref(adam), _ptr(theta_out),
                              _ptr(spins_out), _ptr(eloc_out), _ptr(stats_out), _ptr(grad_out)),
           "psr_vmc_step")
    return theta_out


def psr2d_sample(params, uniforms, Lx, Ly, spins, logpsi=None):
    n = uniforms.shape[0]
    _check(lib().psr2d_sample(C.byref(params), _ptr(uniforms), int(n), int(Lx), int(Ly), _ptr(spins),
                              _ptr(logpsi)), "psr2d_sample")
    return spins


def psr2d_grad(params, spins, Lx, Ly, dout, dparams):
    n = spins.shape[0]
    _check(lib().psr2d_grad(C.byref(params), _ptr(spins), int(n), int(Lx), int(Ly), _ptr(dout),
                            _ptr(dparams)), "psr2d_grad")
    return dparams


def psr2d_vmc_step(params, ham, symmetrize, uniforms, sym_uniforms, adam, theta_out, spins_out=None,
                   eloc_out=None, stats_out=None, grad_out=None):
    n = uniforms.shape[0]
    _check(lib().psr2d_vmc_step(C.byref(params), C.byref(ham), int(bool(symmetrize)), _ptr(uniforms),
                                _ptr(sym_uniforms), int(n), C.byref(adam), _ptr(theta_out),
                                _ptr(spins_out), _ptr(eloc_out), _ptr(stats_out), _ptr(grad_out)),
           "psr2d_vmc_step")
    return theta_out


def psr2d_sym_logpsi(params, spins, Lx, Ly, out):
    n = spins.shape[0]
    _check(lib().psr2d_sym_logpsi(C.byref(params), _ptr(spins), int(n), int(Lx), int(Ly), _ptr(out)),
           "psr2d_sym_logpsi")
    return out


def psr2d_sym_local_energy(params, samples, ham, out, stats=None):
    n = samples.shape[0]
    _check(lib().psr2d_sym_local_energy(C.byref(params), _ptr(samples), int(n), C.byref(ham), _ptr(out),
                                        _ptr(stats)), "psr2d_sym_local_energy")
    return out


def psr_lru_sample(params, uniforms, spins, logpsi=None):
    n, L = uniforms.shape
    _check(lib().psr_lru_sample(C.byref(params), _ptr(uniforms), int(n), int(L), _ptr(spins), _ptr(logpsi)),
           "psr_lru_sample")
    return spins


def psr_lru_grad(params, spins, dout, dparams):
    n, L = spins.shape
    _check(lib().psr_lru_grad(C.byref(params), _ptr(spins), int(n), int(L), _ptr(dout), _ptr(dparams)),
           "psr_lru_grad")
    return dparams


def psr_lru_vmc_step(params, ham, uniforms, adam, theta_out, spins_out=None, eloc_out=None,
                     stats_out=None, grad_out=None):
    n = uniforms.shape[0]
    _check(lib().psr_lru_vmc_step(C.byref(params), C.byref(ham), _ptr(uniforms), int(n), C.byref(adam),
                                  _ptr(theta_out), _ptr(spins_out), _ptr(eloc_out), _ptr(stats_out),
                                  _ptr(grad_out)), "psr_lru_vmc_step")
    return theta_out
