"""Python front end of the FP64 CPU oracle (test infrastructure only).

Only tests/, ``__graft_entry__.smoke()`` and the cpu_baseline / reference
legs of bench.py may import this module.  It loads ``liboracle.so`` compiled
from ``psr_oracle.c`` (plain C, double precision, strictly sequential) and
adds the exact-diagonalisation routines used to pin it.  It shares nothing
with the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "psr_oracle.c")
_SRCS = (_SRC, os.path.join(_HERE, "psr_oracle2d.c"), os.path.join(_HERE, "psr_oracle_lru.c"))
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")

HEISENBERG = 0
TFIM = 1


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (no architecture-specific flags)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    newest = max(os.path.getmtime(x) for x in _SRCS)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, *_SRCS, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d, i, l, vp = C.c_double, C.c_int, C.c_long, C.c_void_p
        _lib.psro_param_count.restype = l
        _lib.psro_param_count.argtypes = [i, i]
        _lib.psro_logpsi.restype = d
        _lib.psro_logpsi.argtypes = [vp, i, i, i, vp, i, vp]
        _lib.psro_trace.restype = d
        _lib.psro_trace.argtypes = [vp, i, i, i, vp, i, vp, vp, vp]
        _lib.psro_grad.restype = d
        _lib.psro_grad.argtypes = [vp, i, i, i, vp, i, vp]
        _lib.psro_sample.restype = None
        _lib.psro_sample.argtypes = [vp, i, i, i, i, l, vp, vp, vp]
        _lib.psro_seq_pos.restype = i
        _lib.psro_seq_pos.argtypes = [i, i, i]
        _lib.psro_bonds.restype = i
        _lib.psro_bonds.argtypes = [i, i, i, vp]
        _lib.psro_count_connected.restype = None
        _lib.psro_count_connected.argtypes = [i, d, vp, i, vp, i, l, vp, vp]
        _lib.psro_fill_connected.restype = None
        _lib.psro_fill_connected.argtypes = [i, vp, i, vp, i, l, vp]
        _lib.psro_offdiag_coeff.restype = d
        _lib.psro_offdiag_coeff.argtypes = [i, d, d, i]
        _lib.psro_eloc_combine.restype = d
        _lib.psro_eloc_combine.argtypes = [d, d, d, vp, l]
        _lib.psro_local_energy.restype = None
        _lib.psro_local_energy.argtypes = [vp, i, i, i, i, i, i, i, i, d, d, vp, i, l, vp]
        _lib.psro_stats.restype = None
        _lib.psro_stats.argtypes = [vp, l, vp]
        _lib.psro_scan_sequential.restype = None
        _lib.psro_scan_sequential.argtypes = [vp, vp, i, d, vp]
        _lib.psro_scan_blelloch.restype = None
        _lib.psro_scan_blelloch.argtypes = [vp, vp, i, d, vp]
        _lib.psro2d_param_count.restype = l
        _lib.psro2d_param_count.argtypes = [i, i]
        _lib.psro2d_logpsi.restype = d
        _lib.psro2d_logpsi.argtypes = [vp, i, i, i, i, i, vp, vp]
        _lib.psro2d_sample.restype = None
        _lib.psro2d_sample.argtypes = [vp, i, i, i, i, i, l, vp, vp, vp]
        _lib.psro2d_conditionals.restype = None
        _lib.psro2d_conditionals.argtypes = [vp, i, i, i, i, i, vp, vp]
        _lib.psro_lru_param_count.restype = l
        _lib.psro_lru_param_count.argtypes = [i, i]
        _lib.psro_lru_logpsi.restype = d
        _lib.psro_lru_logpsi.argtypes = [vp, i, i, i, vp, i, vp]
        _lib.psro_lru_sample.restype = None
        _lib.psro_lru_sample.argtypes = [vp, i, i, i, i, l, vp, vp, vp]
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _theta64(theta):
    return np.ascontiguousarray(np.asarray(theta, dtype=np.float64))


def _spins(s):
    s = np.ascontiguousarray(np.asarray(s, dtype=np.uint8))
    return s.reshape(1, -1) if s.ndim == 1 else s


def _threads(threads):
    return max(1, threads if threads else (os.cpu_count() or 1))


# ------------------------------------------------------------- model calls

def param_count(n_layers: int, hidden: int) -> int:
    return int(lib().psro_param_count(n_layers, hidden))


def logpsi(theta, n_layers, hidden, spins, u1=False, threads=None, per_site=False):
    """log psi for every row of spins [n, N]; optionally per-site log P [n, N]."""
    th = _theta64(theta)
    s = _spins(spins)
    n, N = s.shape
    out = np.empty(n)
    lp = np.empty((n, N)) if per_site else None
    L = lib()

    def one(i):
        row = np.ascontiguousarray(s[i])
        buf = np.empty(N) if per_site else None
        out[i] = L.psro_logpsi(_p(th), n_layers, hidden, int(u1), _p(row), N,
                               _p(buf) if per_site else None)
        if per_site:
            lp[i] = buf

    _map(one, n, threads)
    return (out, lp) if per_site else out


def trace(theta, n_layers, hidden, spins, u1=False):
    """Per-site hidden states h[N, nL, H], layer outputs x[N, nL, H], logits[N, 2]."""
    th = _theta64(theta)
    s = np.ascontiguousarray(np.asarray(spins, dtype=np.uint8).ravel())
    N = s.size
    h = np.empty((N, n_layers, hidden))
    x = np.empty((N, n_layers, hidden))
    lg = np.empty((N, 2))
    r = lib().psro_trace(_p(th), n_layers, hidden, int(u1), _p(s), N, _p(h), _p(x), _p(lg))
    return r, h, x, lg


def grad(theta, n_layers, hidden, spins, u1=False, threads=None):
    """(log psi [n], O_k = d log psi / d theta [n, P]) per configuration."""
    th = _theta64(theta)
    s = _spins(spins)
    n, N = s.shape
    P = param_count(n_layers, hidden)
    g = np.empty((n, P))
    lps = np.empty(n)
    L = lib()

    def one(i):
        row = np.ascontiguousarray(s[i])
        buf = np.empty(P)
        lps[i] = L.psro_grad(_p(th), n_layers, hidden, int(u1), _p(row), N, _p(buf))
        g[i] = buf

    _map(one, n, threads)
    return lps, g


def sample(theta, n_layers, hidden, N, uniforms, u1=False):
    """Exact autoregressive samples from the given uniforms [n, N]."""
    th = _theta64(theta)
    u = np.ascontiguousarray(np.asarray(uniforms, dtype=np.float64))
    n = u.shape[0]
    out = np.empty((n, N), dtype=np.uint8)
    lps = np.empty(n)
    lib().psro_sample(_p(th), n_layers, hidden, int(u1), N, n, _p(u), _p(out), _p(lps))
    return out, lps


# ------------------------------------------------------- Hamiltonian calls

def seq_pos(Lx, i, j):
    return int(lib().psro_seq_pos(Lx, i, j))


def bonds(Lx, Ly, pbc=False):
    buf = np.empty(2 * (2 * Lx * Ly + 2), dtype=np.int32)
    nb = lib().psro_bonds(Lx, Ly, int(pbc), _p(buf))
    return buf[: 2 * nb].reshape(nb, 2).copy()


def connected(kind, Lx, Ly, pbc, spins, J=1.0):
    """(offsets [n+1] int64, entries [E, 3] int32, diag [n] float64)."""
    s = _spins(spins)
    n, N = s.shape
    pq = np.ascontiguousarray(bonds(Lx, Ly, pbc))
    nb = pq.shape[0]
    counts = np.empty(n, dtype=np.int64)
    diag = np.empty(n)
    L = lib()
    L.psro_count_connected(kind, J, _p(pq), nb, _p(s), N, n, _p(counts), _p(diag))
    offsets = np.zeros(n + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(counts)
    ent = np.empty((int(offsets[-1]), 3), dtype=np.int32)
    if ent.size:
        L.psro_fill_connected(kind, _p(pq), nb, _p(s), N, n, _p(ent))
    return offsets, ent, diag


def offdiag_coeff(kind, J=1.0, h=0.0, marshall=True):
    return float(lib().psro_offdiag_coeff(kind, J, h, int(marshall)))


def eloc_combine(diag, coeff, logpsi_s, logpsi_sp):
    v = np.ascontiguousarray(np.asarray(logpsi_sp, dtype=np.float64))
    return float(lib().psro_eloc_combine(float(diag), float(coeff), float(logpsi_s),
                                         _p(v) if v.size else None, v.size))


def local_energy(theta, n_layers, hidden, spins, kind, Lx, Ly, pbc=False, marshall=True,
                 J=1.0, h=0.0, u1=False, threads=None):
    """E_loc per sample with every connected configuration recomputed in full."""
    th = _theta64(theta)
    s = _spins(spins)
    n, N = s.shape
    out = np.empty(n)
    L = lib()

    def one(i):
        row = np.ascontiguousarray(s[i])
        buf = np.empty(1)
        L.psro_local_energy(_p(th), n_layers, hidden, int(u1), kind, Lx, Ly, int(pbc),
                            int(marshall), J, h, _p(row), N, 1, _p(buf))
        out[i] = buf[0]

    _map(one, n, threads)
    return out


def stats(e):
    e = np.ascontiguousarray(np.asarray(e, dtype=np.float64))
    out = np.empty(3)
    lib().psro_stats(_p(e), e.size, _p(out))
    return out


def scan_sequential(a, b, h0=0.0):
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    h = np.empty_like(a)
    lib().psro_scan_sequential(_p(a), _p(b), a.size, h0, _p(h))
    return h


def scan_blelloch(a, b, h0=0.0):
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    h = np.empty_like(a)
    lib().psro_scan_blelloch(_p(a), _p(b), a.size, h0, _p(h))
    return h


def _map(fn, n, threads):
    t = min(_threads(threads), max(1, n))
    if t == 1:
        for i in range(n):
            fn(i)
        return
    with ThreadPoolExecutor(max_workers=t) as ex:
        list(ex.map(fn, range(n)))


# --------------------------------------------- two-dimensional patched minGRU

def param_count2d(n_layers: int, hidden: int) -> int:
    return int(lib().psro2d_param_count(n_layers, hidden))


def logpsi2d(theta, n_layers, hidden, Lx, Ly, spins, u1=False, threads=None, per_site=False):
    """log psi of the 2D patched minGRU for every row of spins [n, Lx*Ly]
    (sequence order); optionally the per-patch log P [n, Lx*Ly/4]."""
    th = _theta64(theta)
    s = _spins(spins)
    n, N = s.shape
    assert N == Lx * Ly
    Np = (Lx // 2) * (Ly // 2)
    out = np.empty(n)
    lp = np.empty((n, Np)) if per_site else None
    L = lib()

    def one(i):
        row = np.ascontiguousarray(s[i])
        buf = np.empty(Np) if per_site else None
        out[i] = L.psro2d_logpsi(_p(th), n_layers, hidden, int(u1), Lx, Ly, _p(row),
                                 _p(buf) if per_site else None)
        if per_site:
            lp[i] = buf

    _map(one, n, threads)
    return (out, lp) if per_site else out


def sample2d(theta, n_layers, hidden, Lx, Ly, uniforms, u1=False):
    """Exact samples of the 2D model from uniforms [n, Lx*Ly/4] (one per patch)."""
    th = _theta64(theta)
    u = np.ascontiguousarray(np.asarray(uniforms, dtype=np.float64))
    n = u.shape[0]
    out = np.empty((n, Lx * Ly), dtype=np.uint8)
    lps = np.empty(n)
    lib().psro2d_sample(_p(th), n_layers, hidden, int(u1), Lx, Ly, n, _p(u), _p(out), _p(lps))
    return out, lps


def conditionals2d(theta, n_layers, hidden, Lx, Ly, spins, u1=False, threads=None):
    """[n, Np, 16] conditional distributions of every patch (path order)."""
    th = _theta64(theta)
    s = _spins(spins)
    n = s.shape[0]
    Np = (Lx // 2) * (Ly // 2)
    out = np.empty((n, Np, 16))
    L = lib()

    def one(i):
        row = np.ascontiguousarray(s[i])
        buf = np.empty((Np, 16))
        L.psro2d_conditionals(_p(th), n_layers, hidden, int(u1), Lx, Ly, _p(row), _p(buf))
        out[i] = buf

    _map(one, n, threads)
    return out


def local_energy2d(theta, n_layers, hidden, spins, kind, Lx, Ly, pbc=False, marshall=True,
                   J=1.0, h=0.0, u1=False, threads=None):
    """E_loc of the 2D model: the connected configurations of the bond /
    site flips, each evaluated by a full forward, combined with the diagonal
    energy (the same steps as the one-dimensional E_loc)."""
    s = _spins(spins)
    n, N = s.shape
    offsets, ent, diag = connected(kind, Lx, Ly, pbc, s, J=J)
    flipped = np.repeat(s, np.diff(offsets), axis=0)
    rows = np.arange(flipped.shape[0])
    if flipped.shape[0]:
        flipped[rows, ent[:, 1]] ^= 1
        has_q = ent[:, 2] >= 0
        flipped[rows[has_q], ent[has_q, 2]] ^= 1
    lp_s = logpsi2d(theta, n_layers, hidden, Lx, Ly, s, u1=u1, threads=threads)
    lp_sp = logpsi2d(theta, n_layers, hidden, Lx, Ly, flipped, u1=u1, threads=threads) \
        if flipped.shape[0] else np.empty(0)
    c = offdiag_coeff(kind, J=J, h=h, marshall=marshall)
    return np.array([eloc_combine(diag[i], c, lp_s[i], lp_sp[offsets[i]:offsets[i + 1]])
                     for i in range(n)])


# --------------------------------------------------------- deep 1D LRU model

def param_count_lru(n_layers: int, hidden: int) -> int:
    return int(lib().psro_lru_param_count(n_layers, hidden))


def logpsi_lru(theta, n_layers, hidden, spins, u1=False, threads=None, per_site=False):
    """log psi of the deep LRU for every row of spins [n, N]; optionally the
    per-site log P [n, N]."""
    th = _theta64(theta)
    s = _spins(spins)
    n, N = s.shape
    out = np.empty(n)
    lp = np.empty((n, N)) if per_site else None
    L = lib()

    def one(i):
        row = np.ascontiguousarray(s[i])
        buf = np.empty(N) if per_site else None
        out[i] = L.psro_lru_logpsi(_p(th), n_layers, hidden, int(u1), _p(row), N,
                                   _p(buf) if per_site else None)
        if per_site:
            lp[i] = buf

    _map(one, n, threads)
    return (out, lp) if per_site else out


def sample_lru(theta, n_layers, hidden, N, uniforms, u1=False):
    th = _theta64(theta)
    u = np.ascontiguousarray(np.asarray(uniforms, dtype=np.float64))
    n = u.shape[0]
    out = np.empty((n, N), dtype=np.uint8)
    lps = np.empty(n)
    lib().psro_lru_sample(_p(th), n_layers, hidden, int(u1), N, n, _p(u), _p(out), _p(lps))
    return out, lps


def local_energy_lru(theta, n_layers, hidden, spins, kind, Lx, Ly, pbc=False, marshall=True,
                     J=1.0, h=0.0, u1=False, threads=None):
    """E_loc of the deep LRU: connected configurations evaluated by full
    forwards and combined with the diagonal energy."""
    s = _spins(spins)
    n, N = s.shape
    offsets, ent, diag = connected(kind, Lx, Ly, pbc, s, J=J)
    flipped = np.repeat(s, np.diff(offsets), axis=0)
    rows = np.arange(flipped.shape[0])
    if flipped.shape[0]:
        flipped[rows, ent[:, 1]] ^= 1
        has_q = ent[:, 2] >= 0
        flipped[rows[has_q], ent[has_q, 2]] ^= 1
    lp_s = logpsi_lru(theta, n_layers, hidden, s, u1=u1, threads=threads)
    lp_sp = logpsi_lru(theta, n_layers, hidden, flipped, u1=u1, threads=threads) \
        if flipped.shape[0] else np.empty(0)
    c = offdiag_coeff(kind, J=J, h=h, marshall=marshall)
    return np.array([eloc_combine(diag[i], c, lp_s[i], lp_sp[offsets[i]:offsets[i + 1]])
                     for i in range(n)])
