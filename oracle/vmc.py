"""FP64 oracle of c4v symmetrisation and of one VMC step (test infrastructure
only: only tests/, __graft_entry__.smoke() and the cpu_baseline / reference
legs of bench.py may import it).

- c4v acts on an L x L lattice by its 8 operations (identity, the three
  rotations, the reflections in x and in y, the two diagonal reflections);
  the symmetrised amplitude of a positive wave function is
  psi_sym(s) = sqrt(1/8 sum_g psi(g s)^2)   (Sec. III.C imposes the c4v
  point group; the formula is the one of the RNN wave-function work the
  paper cites for it);
- the VMC energy gradient of a real positive wave function over samples
  s_i ~ |psi|^2 is grad E = 2/n sum_i (E_loc(s_i) - E) d log psi(s_i) / d theta,
  with d log psi_sym = sum_g w_g d log psi(g s), w_g = psi(g s)^2 / sum_h
  psi(h s)^2 (Sec. III.B: stochastic energy-gradient estimates);
- Adam (Sec. III.B; Kingma and Ba): m = b1 m + (1 - b1) g,
  v = b2 v + (1 - b2) g^2, theta -= lr m / (1 - b1^t) / (sqrt(v / (1 - b2^t)) + eps).
"""
from __future__ import annotations

import numpy as np

from . import oracle as orc


def c4v_maps(L: int):
    """[8, L*L] index maps: image g of a configuration s (sequence order)
    has (g s)[pos(g(i, j))] = s[pos(i, j)]; returned as src indices, i.e.
    (g s) = s[maps[g]]."""
    ops = [
        lambda i, j: (i, j),                  # identity
        lambda i, j: (L - 1 - j, i),          # rotation by 90 degrees
        lambda i, j: (L - 1 - i, L - 1 - j),  # rotation by 180 degrees
        lambda i, j: (j, L - 1 - i),          # rotation by 270 degrees
        lambda i, j: (L - 1 - i, j),          # reflection in x
        lambda i, j: (i, L - 1 - j),          # reflection in y
        lambda i, j: (j, i),                  # reflection in the diagonal
        lambda i, j: (L - 1 - j, L - 1 - i),  # reflection in the anti-diagonal
    ]
    maps = np.empty((8, L * L), dtype=np.int64)
    for g, op in enumerate(ops):
        for j in range(L):
            for i in range(L):
                gi, gj = op(i, j)
                maps[g, orc.seq_pos(L, gi, gj)] = orc.seq_pos(L, i, j)
    return maps


def c4v_images(spins, L: int):
    """[8, n, N] images of every configuration."""
    s = np.asarray(spins, dtype=np.uint8)
    s = s.reshape(1, -1) if s.ndim == 1 else s
    return np.stack([s[:, m] for m in c4v_maps(L)])


def logpsi_sym(logpsi_fn, spins, L):
    """Symmetrised log amplitude from a model's log psi function."""
    imgs = c4v_images(spins, L)
    lp = np.stack([logpsi_fn(x) for x in imgs])  # [8, n]
    m = np.max(2 * lp, axis=0)
    return 0.5 * (m + np.log(np.sum(np.exp(2 * lp - m), axis=0)) - np.log(8.0))


def local_energy_sym(logpsi_fn, spins, kind, L, pbc=False, marshall=True, J=1.0, h=0.0):
    """E_loc of psi_sym: every connected configuration's symmetrised
    amplitude by its 8 images."""
    s = np.asarray(spins, dtype=np.uint8)
    s = s.reshape(1, -1) if s.ndim == 1 else s
    offsets, ent, diag = orc.connected(kind, L, L, pbc, s, J=J)
    flipped = np.repeat(s, np.diff(offsets), axis=0)
    rows = np.arange(flipped.shape[0])
    if flipped.shape[0]:
        flipped[rows, ent[:, 1]] ^= 1
        q = ent[:, 2] >= 0
        flipped[rows[q], ent[q, 2]] ^= 1
    ls = logpsi_sym(logpsi_fn, s, L)
    lf = logpsi_sym(logpsi_fn, flipped, L) if flipped.shape[0] else np.empty(0)
    c = orc.offdiag_coeff(kind, J=J, h=h, marshall=marshall)
    return np.array([orc.eloc_combine(diag[i], c, ls[i], lf[offsets[i]:offsets[i + 1]])
                     for i in range(s.shape[0])])


def energy_gradient(eloc, okl, weights=None):
    """2 sum_i w_i (E_i - E) O_i over samples (w_i = 1/n for samples drawn
    from |psi|^2; exact probabilities when enumerating), E = sum_i w_i E_i."""
    e = np.asarray(eloc, dtype=np.float64)
    w = np.full(e.size, 1.0 / e.size) if weights is None else np.asarray(weights, dtype=np.float64)
    mean = np.sum(w * e)
    return 2.0 * ((w * (e - mean)) @ np.asarray(okl, dtype=np.float64)), mean


def grad_logpsi_sym(theta, n_layers, hidden, spins, L, u1=False):
    """d log psi_sym / d theta [n, P] of the chain minGRU model."""
    imgs = c4v_images(spins, L)
    lps, oks = [], []
    for x in imgs:
        lp, ok = orc.grad(theta, n_layers, hidden, x, u1=u1)
        lps.append(lp)
        oks.append(ok)
    lps = np.stack(lps)            # [8, n]
    w = np.exp(2 * lps - np.max(2 * lps, axis=0))
    w /= w.sum(axis=0)
    return np.einsum("gn,gnp->np", w, np.stack(oks))


def adam(theta, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update; returns (theta, m, v) as new arrays (step counts from 1)."""
    g = np.asarray(grad, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return np.asarray(theta, dtype=np.float64) - lr * mh / (np.sqrt(vh) + eps), m, v
