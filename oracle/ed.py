"""Exact diagonalisation and dense-state helpers (test infrastructure only).

Builds the Hamiltonians of the paper directly from Pauli matrices with
Kronecker products, independently of the oracle's bond/flip generator:
  - Heisenberg  H = J sum_<ij> S_i . S_j,  S = sigma/2   (Sec. III.C)
  - TFIM        H = -J sum_<ij> sz_i sz_j - h sum_i sx_i (Sec. III.B)
Basis: sites in sequence order; basis index = sum_t s_t 2^(N-1-t) with local
state s = 1 meaning spin up (sigma^z = +1).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as sla

# local basis (s=0 -> down, s=1 -> up)
_SX = sp.csr_matrix(np.array([[0.0, 1.0], [1.0, 0.0]]))
_SY = sp.csr_matrix(np.array([[0.0, 1.0j], [-1.0j, 0.0]]))  # <s|sy|s'> with s=1 up
_SZ = sp.csr_matrix(np.array([[-1.0, 0.0], [0.0, 1.0]]))


def _op(single, site, N):
    left = sp.identity(2 ** site, format="csr")
    right = sp.identity(2 ** (N - site - 1), format="csr")
    return sp.kron(sp.kron(left, single, format="csr"), right, format="csr")


def heisenberg(N, pairs, J=1.0):
    H = sp.csr_matrix((2 ** N, 2 ** N), dtype=np.complex128)
    for p, q in pairs:
        for s in (_SX, _SY, _SZ):
            H = H + 0.25 * J * (_op(s, p, N) @ _op(s, q, N))
    return H


def tfim(N, pairs, J=1.0, h=1.0):
    H = sp.csr_matrix((2 ** N, 2 ** N), dtype=np.complex128)
    for p, q in pairs:
        H = H - J * (_op(_SZ, p, N) @ _op(_SZ, q, N))
    for i in range(N):
        H = H - h * _op(_SX, i, N)
    return H


def all_configs(N):
    """[2^N, N] uint8 in basis-index order."""
    idx = np.arange(2 ** N, dtype=np.int64)
    return ((idx[:, None] >> (N - 1 - np.arange(N))[None, :]) & 1).astype(np.uint8)


def marshall_sign(configs, sublattice_a):
    """(-1)^(number of up spins on sublattice A)."""
    n_up_a = configs[:, sublattice_a].sum(axis=1)
    return np.where(n_up_a % 2 == 0, 1.0, -1.0)


def ground_state(H, k=1):
    """Lowest eigenpair of a Hermitian sparse matrix."""
    n = H.shape[0]
    if n <= 64:
        w, v = np.linalg.eigh(H.toarray())
        return w[0], v[:, 0]
    w, v = sla.eigsh(H, k=k, which="SA", tol=1e-12)
    i = int(np.argmin(w))
    return w[i], v[:, i]


def expectation(H, psi):
    psi = np.asarray(psi)
    return float(np.real(np.vdot(psi, H @ psi)) / np.real(np.vdot(psi, psi)))
