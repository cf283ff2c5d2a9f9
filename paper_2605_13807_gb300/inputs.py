"""Seeded synthetic inputs for the PSR-NQS hot path.

This module holds no arithmetic of the method itself: it only produces
parameters and spin configurations from counter-based random numbers, so that
the CUDA library and the FP64 oracle can be fed identical bytes.

Generator: splitmix64 evaluated at counter values (Steele, Lea, Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014): value i of
stream ``seed`` is mix64(seed + (i + 1) * 0x9E3779B97F4A7C15); a uniform
double in [0, 1) is its top 53 bits times 2**-53.

Layouts follow the library's parameter order (per layer: W_z, b_z, W_h, b_h,
C, D; then W_o, b_o) and the zigzag sequence order of the lattice
(Sec. II.F of the paper: row j runs left to right when j is even).
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """``count`` raw 64-bit outputs of stream ``seed`` starting at ``offset``."""
    i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, shape, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) with the given shape."""
    n = int(np.prod(shape))
    z = splitmix64(seed, n, offset)
    return ((z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)).reshape(shape)


# ---------------------------------------------------------------- parameters

def param_shapes(n_layers: int, hidden: int):
    """(name, shape, is_weight) in the flat parameter order."""
    out = []
    for l in range(n_layers):
        din = 2 if l == 0 else hidden
        out += [(f"W_z{l}", (hidden, din), True), (f"b_z{l}", (hidden,), False),
                (f"W_h{l}", (hidden, din), True), (f"b_h{l}", (hidden,), False),
                (f"C{l}", (hidden, hidden), True), (f"D{l}", (hidden, din), True)]
    out += [("W_o", (2, hidden), True), ("b_o", (2,), False)]
    return out


def param_count(n_layers: int, hidden: int) -> int:
    return int(sum(int(np.prod(s)) for _, s, _ in param_shapes(n_layers, hidden)))


def glorot_params(n_layers: int, hidden: int, seed: int = 0) -> np.ndarray:
    """Glorot-uniform weights U(+-sqrt(6/(fan_in+fan_out))), zero biases, FP32."""
    parts = []
    off = 0
    for _, shape, is_w in param_shapes(n_layers, hidden):
        n = int(np.prod(shape))
        if is_w:
            fan_out, fan_in = shape
            lim = np.sqrt(6.0 / (fan_in + fan_out))
            u = uniform(seed, (n,), offset=off)
            parts.append((2.0 * u - 1.0) * lim)
        else:
            parts.append(np.zeros(n))
        off += n
    return np.concatenate(parts).astype(np.float32)


def param_shapes2d(n_layers: int, hidden: int):
    """(name, shape, is_weight) in the flat parameter order of the 2D patched
    model (layer-0 input: two 16-value one-hots; W_h also acts on h_V)."""
    out = []
    for l in range(n_layers):
        din = 32 if l == 0 else hidden
        out += [(f"W_z{l}", (hidden, din), True), (f"b_z{l}", (hidden,), False),
                (f"W_h{l}", (hidden, din + hidden), True), (f"b_h{l}", (hidden,), False),
                (f"C{l}", (hidden, hidden), True), (f"D{l}", (hidden, din), True)]
    out += [("W_o", (16, hidden), True), ("b_o", (16,), False)]
    return out


def glorot_params2d(n_layers: int, hidden: int, seed: int = 0) -> np.ndarray:
    """Glorot-uniform weights, zero biases, for the 2D patched model; FP32."""
    parts = []
    off = 0
    for _, shape, is_w in param_shapes2d(n_layers, hidden):
        n = int(np.prod(shape))
        if is_w:
            fan_out, fan_in = shape
            lim = np.sqrt(6.0 / (fan_in + fan_out))
            parts.append((2.0 * uniform(seed, (n,), offset=off) - 1.0) * lim)
        else:
            parts.append(np.zeros(n))
        off += n
    return np.concatenate(parts).astype(np.float32)


def random_params(n_layers: int, hidden: int, seed: int, scale: float = 0.5) -> np.ndarray:
    """Every entry (biases included) uniform in +-scale/sqrt(fan_in); FP32.
    Used by tests to exercise every parameter."""
    parts = []
    off = 0
    for _, shape, _ in param_shapes(n_layers, hidden):
        n = int(np.prod(shape))
        fan_in = shape[1] if len(shape) == 2 else 1
        u = uniform(seed, (n,), offset=off)
        parts.append((2.0 * u - 1.0) * scale / np.sqrt(max(fan_in, 1)))
        off += n
    return np.concatenate(parts).astype(np.float32)


# ------------------------------------------------------------ configurations

def seq_pos(Lx: int, i, j):
    """Zigzag sequence position of lattice site (i, j)."""
    i = np.asarray(i)
    j = np.asarray(j)
    return j * Lx + np.where(j % 2 == 0, i, Lx - 1 - i)


def to_sequence(lattice_spins: np.ndarray, Lx: int, Ly: int) -> np.ndarray:
    """[n, Ly, Lx] lattice spins -> [n, N] spins in zigzag sequence order."""
    n = lattice_spins.shape[0]
    out = np.empty((n, Lx * Ly), dtype=lattice_spins.dtype)
    jj, ii = np.meshgrid(np.arange(Ly), np.arange(Lx), indexing="ij")
    out[:, seq_pos(Lx, ii, jj).ravel()] = lattice_spins.reshape(n, -1)
    return out


def random_spins(seed: int, n: int, N: int) -> np.ndarray:
    """Independent uniform spins {0,1}, uint8 [n, N]."""
    return (uniform(seed, (n, N)) < 0.5).astype(np.uint8)


def zero_magnetisation_spins(seed: int, n: int, N: int) -> np.ndarray:
    """Uniform configurations with exactly N/2 ones (random permutation)."""
    assert N % 2 == 0
    keys = uniform(seed, (n, N))
    order = np.argsort(keys, axis=1, kind="stable")
    out = np.zeros((n, N), dtype=np.uint8)
    rows = np.arange(n)[:, None]
    out[rows, order[:, : N // 2]] = 1
    return out


def neel_like_spins(seed: int, n: int, Lx: int, Ly: int, anti_fraction: float = 0.72) -> np.ndarray:
    """Antiferromagnetically correlated S^z = 0 configurations.

    Start from the Neel pattern (up where i + j is even) and exchange k up
    spins with k down spins chosen uniformly, k = round(f * N/2), where f
    solves f^2 + (1 - f)^2 = anti_fraction so that a bond keeps its
    antiparallel state with probability ~anti_fraction.  Returned in zigzag
    sequence order, uint8 [n, Lx*Ly].  Requires an even site count.
    """
    N = Lx * Ly
    assert N % 2 == 0
    f = 0.5 * (1.0 - np.sqrt(max(0.0, 2.0 * anti_fraction - 1.0)))
    k = int(round(f * N / 2))
    jj, ii = np.meshgrid(np.arange(Ly), np.arange(Lx), indexing="ij")
    neel_lat = ((ii + jj) % 2 == 0).astype(np.uint8)
    neel = to_sequence(neel_lat[None], Lx, Ly)[0]
    ups = np.flatnonzero(neel == 1)
    dns = np.flatnonzero(neel == 0)
    if len(ups) != len(dns):  # odd dimensions: fall back to an exact half split
        ups = ups[: N // 2]
        dns = np.setdiff1d(np.arange(N), ups)
    out = np.tile(neel, (n, 1))
    out[:, ups] = 1
    out[:, dns] = 0
    rows = np.arange(n)[:, None]
    if k > 0:
        ku = np.argsort(uniform(seed, (n, len(ups))), axis=1)[:, :k]
        kd = np.argsort(uniform(seed ^ 0x5A5A5A5A, (n, len(dns))), axis=1)[:, :k]
        out[rows, ups[ku]] = 0
        out[rows, dns[kd]] = 1
    return out


def scan_inputs(seed: int, n: int, N: int, H: int):
    """Coefficients of a diagonal linear recurrence h_t = a_t h_{t-1} + b_t
    shaped like a minGRU layer's gates: a in (0.001, 1) with many values
    close to 1 (long memory), b and h0 uniform in (-1, 1).  float32
    [n, N, H], [n, N, H], [n, H]."""
    u = uniform(seed, (3, n * N * H + n * H))
    a = (1.0 - 0.999 * u[0, : n * N * H] ** 2).astype(np.float32).reshape(n, N, H)
    b = (2.0 * u[1, : n * N * H] - 1.0).astype(np.float32).reshape(n, N, H)
    h0 = (2.0 * u[2, n * N * H:] - 1.0).astype(np.float32).reshape(n, H)
    return a, b, h0


def scan_inputs_device(seed: int, n: int, N: int, H: int, device):
    """The distribution of scan_inputs drawn on the device with torch's seeded
    generator (for sizes where host generation is too slow)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    a = torch.rand((n, N, H), generator=g, device=device, dtype=torch.float32)
    a.pow_(2).mul_(-0.999).add_(1.0)
    b = torch.rand((n, N, H), generator=g, device=device, dtype=torch.float32).mul_(2.0).sub_(1.0)
    h0 = torch.rand((n, H), generator=g, device=device, dtype=torch.float32).mul_(2.0).sub_(1.0)
    return a, b, h0


def param_shapes_lru(n_layers: int, hidden: int):
    """(name, shape) in the flat parameter order of the deep 1D LRU."""
    out = []
    for l in range(n_layers):
        din = 2 if l == 0 else hidden
        out += [(f"nu{l}", (hidden,)), (f"theta{l}", (hidden,)), (f"gamma{l}", (hidden,)),
                (f"B_re{l}", (hidden, din)), (f"B_im{l}", (hidden, din)),
                (f"C_re{l}", (hidden, hidden)), (f"C_im{l}", (hidden, hidden)),
                (f"D{l}", (hidden, 2) if l == 0 else (hidden,)),
                (f"W_a{l}", (hidden, hidden)), (f"b_a{l}", (hidden,)),
                (f"W_g{l}", (hidden, hidden)), (f"b_g{l}", (hidden,))]
    out += [("W_o", (2, hidden)), ("b_o", (2,))]
    return out


def lru_params(n_layers: int, hidden: int, seed: int = 0) -> np.ndarray:
    """Seeded LRU parameters in the usual ring initialisation: |lambda| =
    exp(-e^nu) uniform in [0.9, 0.999], phase e^theta uniform in
    [0.01, 0.1 * 2 pi], gamma = log sqrt(1 - |lambda|^2) (unit-variance
    states); matrices U(+-1/sqrt(fan_in)), biases 0; FP32."""
    parts = []
    off = 0
    for name, shape in param_shapes_lru(n_layers, hidden):
        n = int(np.prod(shape))
        u = uniform(seed, (n,), offset=off)
        off += n
        base = name.rstrip("0123456789")
        if base == "nu":
            r = 0.9 + 0.099 * u
            parts.append(np.log(-np.log(r)))
            r_last = r
        elif base == "theta":
            parts.append(np.log(0.01 + (0.2 * np.pi - 0.01) * u))
        elif base == "gamma":
            parts.append(np.log(np.sqrt(1.0 - r_last ** 2)))
        elif base in ("b_a", "b_g", "b_o"):
            parts.append(np.zeros(n))
        else:
            fan_in = shape[1] if len(shape) == 2 else 1
            parts.append((2.0 * u - 1.0) / np.sqrt(fan_in))
    return np.concatenate(parts).astype(np.float32)
