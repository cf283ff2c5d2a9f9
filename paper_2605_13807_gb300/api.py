"""Tensor-level wrappers over the C ABI (allocation and marshalling only).

    logpsi(theta, spins, ...)            -> float32 [n]
    local_energy(theta, samples, ham)    -> (float32 [n] E_loc, float64 [3] stats)
    connected(samples, ham)              -> (int64 [n+1], int32 [E, 3], float32 [n])
    scan(a, b, h0=None)                  -> float32 [n, N, H], h_t = a_t h_{t-1} + b_t
    sample(theta, uniforms, cfg)         -> (uint8 [n, L] exact samples, float32 [n] log psi)
    logpsi2d / local_energy2d            -> the 2D patched minGRU (Lx, Ly even)
    logpsi_lru / local_energy_lru        -> the deep 1D LRU ansatz
    sym_logpsi / sym_local_energy        -> c4v-symmetrised amplitude and its E_loc
    vmc_step(theta, cfg, ham, u, adam)   -> one on-device VMC step (sample, E_loc, gradient, Adam)
    grad(theta, spins, dout=None)        -> float32 [n, P] (O_k) or [P]
    LogPsi.apply(theta, spins, cfg)      -> differentiable log psi; backward = psr_grad

Outputs live where the inputs live (a CUDA tensor in, CUDA tensors out).
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import binding as B


@dataclass(frozen=True)
class ModelConfig:
    n_layers: int = 3
    hidden: int = 128
    u1: bool = False
    precision: str = "fp32"  # "fp32", "bf16" or (2D patched model) "fp16"


def _device_of(*ts):
    for t in ts:
        if isinstance(t, torch.Tensor) and t.is_cuda:
            return t.device
    return torch.device("cpu")


def _ctx():
    return B.context()


def param_count(n_layers: int = 3, hidden: int = 128) -> int:
    return B.psr_param_count(n_layers, hidden)


def logpsi(theta, spins, cfg: ModelConfig, out=None):
    dev = _device_of(spins, theta)
    if out is None:
        out = torch.empty(spins.shape[0], dtype=torch.float32, device=dev)
    p = B.make_params(theta, cfg.n_layers, cfg.hidden, cfg.u1, cfg.precision, _ctx())
    return B.psr_logpsi(p, spins, out)


def local_energy(theta, samples, cfg: ModelConfig, ham: B.psr_hamiltonian, out=None, stats=None):
    dev = _device_of(samples, theta)
    if out is None:
        out = torch.empty(samples.shape[0], dtype=torch.float32, device=dev)
    if stats is None:
        stats = torch.empty(3, dtype=torch.float64, device=dev)
    p = B.make_params(theta, cfg.n_layers, cfg.hidden, cfg.u1, cfg.precision, _ctx())
    B.psr_local_energy(p, samples, ham, out, stats)
    return out, stats


def local_energy_batch(theta, batch, cfg: ModelConfig, outs=None, stats=None):
    """batch: list of (samples, hamiltonian, u1_mask).  Returns lists of E_loc
    and stats tensors; all items run in one persistent launch."""
    dev = _device_of(theta, *[b[0] for b in batch])
    if outs is None:
        outs = [torch.empty(b[0].shape[0], dtype=torch.float32, device=dev) for b in batch]
    if stats is None:
        stats = [torch.empty(3, dtype=torch.float64, device=dev) for _ in batch]
    p = B.make_params(theta, cfg.n_layers, cfg.hidden, cfg.u1, cfg.precision, _ctx())
    B.psr_local_energy_batch(p, [(s, h, u1, o, st) for (s, h, u1), o, st in zip(batch, outs, stats)])
    return outs, stats


def step_batch(theta, batch, cfg: ModelConfig, want=("logpsi", "eloc", "grad"), outs=None):
    """One hot-path step (log psi, E_loc with stats, per-sample O_k) for several
    sample sets in one call: batch is a list of (samples, hamiltonian,
    u1_mask).  Returns a list of dicts with the requested outputs."""
    dev = _device_of(theta, *[b[0] for b in batch])
    P = theta.numel()
    if outs is None:
        outs = []
        for s, _, _ in batch:
            n = s.shape[0]
            o = {}
            if "logpsi" in want:
                o["logpsi"] = torch.empty(n, dtype=torch.float32, device=dev)
            if "eloc" in want:
                o["eloc"] = torch.empty(n, dtype=torch.float32, device=dev)
                o["stats"] = torch.empty(3, dtype=torch.float64, device=dev)
            if "grad" in want:
                o["grad"] = torch.empty((n, P), dtype=torch.float32, device=dev)
            outs.append(o)
    p = B.make_params(theta, cfg.n_layers, cfg.hidden, cfg.u1, cfg.precision, _ctx())
    B.psr_step_batch(p, [(s, h, u1, o.get("logpsi"), o.get("eloc"), o.get("stats"), o.get("grad"))
                         for (s, h, u1), o in zip(batch, outs)])
    return outs


def set_fwd_shape(precision, shape):
    """Fixes the fused forward's shape on the context (0: autotuned / default)."""
    B.psr_context_set_fwd_shape(_ctx(), precision, shape)


def fwd_shape_for(precision, what, n, L):
    return B.psr_fwd_shape_for(_ctx(), precision, what, n, L)


def max_entries(ham: B.psr_hamiltonian, n: int) -> int:
    N = ham.Lx * ham.Ly
    if ham.kind == B.PSR_TFIM:
        return n * N
    wx = 1 if (ham.pbc and ham.Lx >= 3) else 0
    wy = 1 if (ham.pbc and ham.Ly >= 3) else 0
    return n * (ham.Ly * (ham.Lx - 1 + wx) + ham.Lx * (ham.Ly - 1 + wy))


def connected(samples, ham: B.psr_hamiltonian):
    n = samples.shape[0]
    dev = _device_of(samples)
    cap = max_entries(ham, n)
    offsets = torch.empty(n + 1, dtype=torch.int64, device=dev)
    entries = torch.empty((max(cap, 1), 3), dtype=torch.int32, device=dev)
    diag = torch.empty(n, dtype=torch.float32, device=dev)
    total = B.psr_connected(_ctx(), samples, ham, offsets, entries, diag)
    return offsets, entries[:total], diag


def grad(theta, spins, cfg: ModelConfig, dout=None, out=None):
    dev = _device_of(spins, theta)
    P = param_count(cfg.n_layers, cfg.hidden)
    if out is None:
        shape = (P,) if dout is not None else (spins.shape[0], P)
        out = torch.empty(shape, dtype=torch.float32, device=dev)
    p = B.make_params(theta, cfg.n_layers, cfg.hidden, cfg.u1, cfg.precision, _ctx())
    return B.psr_grad(p, spins, dout, out)


def scan(a, b, h0=None, tile=None, out=None):
    """h_t = a_t h_{t-1} + b_t over float32 [n, N, H] tensors (psr_scan)."""
    if out is None:
        out = torch.empty_like(a)
    return B.psr_scan(_ctx(), a, b, out, h0=h0, tile=tile)


def sample(theta, uniforms, cfg: ModelConfig, spins=None, logpsi=None):
    """Exact autoregressive samples from the caller's uniforms [n, L]:
    (uint8 spins [n, L] in sequence order, float32 log psi [n])."""
    dev = _device_of(uniforms, theta)
    n, L = uniforms.shape
    if spins is None:
        spins = torch.empty((n, L), dtype=torch.uint8, device=dev)
    if logpsi is None:
        logpsi = torch.empty(n, dtype=torch.float32, device=dev)
    p = B.make_params(theta, cfg.n_layers, cfg.hidden, cfg.u1, cfg.precision, _ctx())
    B.psr_sample(p, uniforms, spins, logpsi)
    return spins, logpsi


def param_count2d(n_layers: int = 3, hidden: int = 128) -> int:
    return B.psr2d_param_count(n_layers, hidden)


def logpsi2d(theta, spins, cfg: ModelConfig, Lx: int, Ly: int, out=None):
    """log psi of the 2D patched minGRU (spins [n, Lx*Ly] in sequence order)."""
    dev = _device_of(spins, theta)
    if out is None:
        out = torch.empty(spins.shape[0], dtype=torch.float32, device=dev)
    p = B.make_params(theta, cfg.n_layers, cfg.hidden, cfg.u1, cfg.precision, _ctx())
    return B.psr2d_logpsi(p, spins, Lx, Ly, out)


def local_energy2d(theta, samples, cfg: ModelConfig, ham: B.psr_hamiltonian, out=None, stats=None):
    dev = _device_of(samples, theta)
    if out is None:
        out = torch.empty(samples.shape[0], dtype=torch.float32, device=dev)
    if stats is None:
        stats = torch.empty(3, dtype=torch.float64, device=dev)
    p = B.make_params(theta, cfg.n_layers, cfg.hidden, cfg.u1, cfg.precision, _ctx())
    B.psr2d_local_energy(p, samples, ham, out, stats)
    return out, stats


def sample2d(theta, uniforms, cfg: ModelConfig, Lx: int, Ly: int, spins=None, logpsi=None):
    """Exact samples of the 2D patched minGRU from uniforms [n, Np]."""
    dev = _device_of(uniforms, theta)
    n = uniforms.shape[0]
    if spins is None:
        spins = torch.empty((n, Lx * Ly), dtype=torch.uint8, device=dev)
    if logpsi is None:
        logpsi = torch.empty(n, dtype=torch.float32, device=dev)
    p = B.make_params(theta, cfg.n_layers, cfg.hidden, cfg.u1, cfg.precision, _ctx())
    B.psr2d_sample(p, uniforms, Lx, Ly, spins, logpsi)
    return spins, logpsi


def grad2d(theta, spins, cfg: ModelConfig, Lx: int, Ly: int, dout=None, out=None):
    """d log psi / d theta of the 2D model: [n, P] per sample, or [P] with dout."""
    dev = _device_of(spins, theta)
    P = param_count2d(cfg.n_layers, cfg.hidden)
    if out is None:
        shape = (P,) if dout is not None else (spins.shape[0], P)
        out = torch.empty(shape, dtype=torch.float32, device=dev)
    p = B.make_params(theta, cfg.n_layers, cfg.hidden, cfg.u1, cfg.precision, _ctx())
    return B.psr2d_grad(p, spins, Lx, Ly, dout, out)


def param_count_lru(n_layers: int = 3, hidden: int = 64) -> int:
    return B.psr_lru_param_count(n_layers, hidden)


def logpsi_lru(theta, spins, cfg: ModelConfig, out=None):
    """log psi of the deep 1D LRU ansatz (spins [n, L] in sequence order)."""
    dev = _device_of(spins, theta)
    if out is None:
        out = torch.empty(spins.shape[0], dtype=torch.float32, device=dev)
    p = B.make_params(theta, cfg.n_layers, cfg.hidden, cfg.u1, cfg.precision, _ctx())
    return B.psr_lru_logpsi(p, spins, out)


def local_energy_lru(theta, samples, cfg: ModelConfig, ham: B.psr_hamiltonian, out=None, stats=None):
    dev = _device_of(samples, theta)
    if out is None:
        out = torch.empty(samples.shape[0], dtype=torch.float32, device=dev)
    if stats is None:
        stats = torch.empty(3, dtype=torch.float64, device=dev)
    p = B.make_params(theta, cfg.n_layers, cfg.hidden, cfg.u1, cfg.precision, _ctx())
    B.psr_lru_local_energy(p, samples, ham, out, stats)
    return out, stats


def sample_lru(theta, uniforms, cfg: ModelConfig, spins=None, logpsi=None):
    """Exact samples of the LRU ansatz from uniforms [n, L]."""
    dev = _device_of(uniforms, theta)
    n, L = uniforms.shape
    if spins is None:
        spins = torch.empty((n, L), dtype=torch.uint8, device=dev)
    if logpsi is None:
        logpsi = torch.empty(n, dtype=torch.float32, device=dev)
    p = B.make_params(theta, cfg.n_layers, cfg.hidden, cfg.u1, cfg.precision, _ctx())
    B.psr_lru_sample(p, uniforms, spins, logpsi)
    return spins, logpsi


def grad_lru(theta, spins, cfg: ModelConfig, dout=None, out=None):
    """d log psi / d theta of the LRU ansatz: [n, P] per sample, or [P] with dout."""
    dev = _device_of(spins, theta)
    P = param_count_lru(cfg.n_layers, cfg.hidden)
    if out is None:
        shape = (P,) if dout is not None else (spins.shape[0], P)
        out = torch.empty(shape, dtype=torch.float32, device=dev)
    p = B.make_params(theta, cfg.n_layers, cfg.hidden, cfg.u1, cfg.precision, _ctx())
    return B.psr_lru_grad(p, spins, dout, out)


def sym_logpsi2d(theta, spins, cfg: ModelConfig, L: int, out=None):
    """c4v-symmetrised log psi of the 2D patched model on an L x L lattice."""
    dev = _device_of(spins, theta)
    if out is None:
        out = torch.empty(spins.shape[0], dtype=torch.float32, device=dev)
    p = B.make_params(theta, cfg.n_layers, cfg.hidden, cfg.u1, cfg.precision, _ctx())
    return B.psr2d_sym_logpsi(p, spins, L, L, out)


def sym_local_energy2d(theta, samples, cfg: ModelConfig, ham: B.psr_hamiltonian, out=None, stats=None):
    dev = _device_of(samples, theta)
    if out is None:
        out = torch.empty(samples.shape[0], dtype=torch.float32, device=dev)
    if stats is None:
        stats = torch.empty(3, dtype=torch.float64, device=dev)
    p = B.make_params(theta, cfg.n_layers, cfg.hidden, cfg.u1, cfg.precision, _ctx())
    B.psr2d_sym_local_energy(p, samples, ham, out, stats)
    return out, stats


def sym_logpsi(theta, spins, cfg: ModelConfig, L: int, out=None):
    """c4v-symmetrised log psi on an L x L lattice."""
    dev = _device_of(spins, theta)
    if out is None:
        out = torch.empty(spins.shape[0], dtype=torch.float32, device=dev)
    p = B.make_params(theta, cfg.n_layers, cfg.hidden, cfg.u1, cfg.precision, _ctx())
    return B.psr_sym_logpsi(p, spins, L, L, out)


def sym_local_energy(theta, samples, cfg: ModelConfig, ham: B.psr_hamiltonian, out=None, stats=None):
    dev = _device_of(samples, theta)
    if out is None:
        out = torch.empty(samples.shape[0], dtype=torch.float32, device=dev)
    if stats is None:
        stats = torch.empty(3, dtype=torch.float64, device=dev)
    p = B.make_params(theta, cfg.n_layers, cfg.hidden, cfg.u1, cfg.precision, _ctx())
    B.psr_sym_local_energy(p, samples, ham, out, stats)
    return out, stats


class Adam:
    """Adam moments for psr_vmc_step (device tensors, updated in place)."""

    def __init__(self, P, device, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.m = torch.zeros(P, dtype=torch.float32, device=device)
        self.v = torch.zeros(P, dtype=torch.float32, device=device)
        self.lr, self.beta1, self.beta2, self.eps = lr, beta1, beta2, eps
        self.step = 0

    def state(self):
        return B.psr_adam(self.lr, self.beta1, self.beta2, self.eps, self.step, B._ptr(self.m),
                          B._ptr(self.v))


def vmc_step(theta, cfg: ModelConfig, ham: B.psr_hamiltonian, uniforms, adam: Adam,
             symmetrize=False, sym_uniforms=None, theta_out=None):
    """One VMC step on the device: exact samples from `uniforms` [n, N],
    E_loc, energy gradient, Adam update.  Returns a dict with the updated
    parameters, the samples, E_loc, FP64 statistics and the gradient."""
    n, N = uniforms.shape
    dev = uniforms.device
    if theta_out is None:
        theta_out = torch.empty_like(theta)
    out = {"theta": theta_out,
           "spins": torch.empty((n, N), dtype=torch.uint8, device=dev),
           "eloc": torch.empty(n, dtype=torch.float32, device=dev),
           "stats": torch.empty(3, dtype=torch.float64, device=dev),
           "grad": torch.empty_like(theta)}
    adam.step += 1
    p = B.make_params(theta, cfg.n_layers, cfg.hidden, cfg.u1, cfg.precision, _ctx())
    B.psr_vmc_step(p, ham, symmetrize, uniforms, sym_uniforms, adam.state(), theta_out,
                   out["spins"], out["eloc"], out["stats"], out["grad"])
    return out


def vmc_step2d(theta, cfg: ModelConfig, ham: B.psr_hamiltonian, uniforms, adam: Adam, theta_out=None,
               symmetrize=False, sym_uniforms=None):
    """One on-device VMC step of the 2D patched minGRU (uniforms [n, Np]);
    with symmetrize, of its c4v-symmetrised amplitude (sym_uniforms [n])."""
    n = uniforms.shape[0]
    dev = uniforms.device
    N = ham.Lx * ham.Ly
    if theta_out is None:
        theta_out = torch.empty_like(theta)
    out = {"theta": theta_out,
           "spins": torch.empty((n, N), dtype=torch.uint8, device=dev),
           "eloc": torch.empty(n, dtype=torch.float32, device=dev),
           "stats": torch.empty(3, dtype=torch.float64, device=dev),
           "grad": torch.empty_like(theta)}
    adam.step += 1
    p = B.make_params(theta, cfg.n_layers, cfg.hidden, cfg.u1, cfg.precision, _ctx())
    B.psr2d_vmc_step(p, ham, symmetrize, uniforms, sym_uniforms, adam.state(), theta_out, out["spins"],
                     out["eloc"], out["stats"], out["grad"])
    return out


def vmc_step_lru(theta, cfg: ModelConfig, ham: B.psr_hamiltonian, uniforms, adam: Adam, theta_out=None):
    """One on-device VMC step of the LRU ansatz (uniforms [n, N])."""
    n = uniforms.shape[0]
    dev = uniforms.device
    N = ham.Lx * ham.Ly
    if theta_out is None:
        theta_out = torch.empty_like(theta)
    out = {"theta": theta_out,
           "spins": torch.empty((n, N), dtype=torch.uint8, device=dev),
           "eloc": torch.empty(n, dtype=torch.float32, device=dev),
           "stats": torch.empty(3, dtype=torch.float64, device=dev),
           "grad": torch.empty_like(theta)}
    adam.step += 1
    p = B.make_params(theta, cfg.n_layers, cfg.hidden, cfg.u1, cfg.precision, _ctx())
    B.psr_lru_vmc_step(p, ham, uniforms, adam.state(), theta_out, out["spins"], out["eloc"], out["stats"],
                       out["grad"])
    return out


def set_autotune(enable=True):
    B.psr_context_set_autotune(_ctx(), enable)


def sync():
    B.psr_context_sync(_ctx())


class LogPsi(torch.autograd.Function):
    """log psi(s; theta) with a backward that calls the reverse-scan adjoint
    (psr_grad with dout = the incoming gradient)."""

    @staticmethod
    def forward(ctx, theta, spins, cfg: ModelConfig):
        ctx.save_for_backward(theta, spins)
        ctx.cfg = cfg
        return logpsi(theta.detach().contiguous(), spins, cfg)

    @staticmethod
    def backward(ctx, g):
        theta, spins = ctx.saved_tensors
        dtheta = grad(theta.detach().contiguous(), spins, ctx.cfg,
                      dout=g.detach().to(torch.float32).contiguous())
        return dtheta, None, None
