"""Oracle-only reference for a VMC energy gradient (test helper, not a test).

For samples s_i with local energies E_i (mean E) the stochastic
energy-gradient estimate of Sec. III.B is

    g = (2/n) sum_i (E_i - E) d log psi(s_i) / d theta,

which is the gradient, at fixed weights c_i = (2/n)(E_i - E), of the scalar
F(theta) = sum_i c_i log psi_theta(s_i).  Its component along any direction d
is (F(theta + eps d) - F(theta - eps d)) / (2 eps) up to O(eps^2), so it is
computed here from the FP64 oracle's log psi and the oracle's local energies
alone: nothing of the CUDA path enters the reference.  A mistake shared by a
device step and its O_k kernel (the image weights of a symmetrised
amplitude, the centring of E_loc) changes g but not this reference.
"""
from __future__ import annotations

import numpy as np


def energy_gradient_fd(logpsi_fn, theta, eloc_ref, dirs, eps=1e-5):
    """Directional derivatives of F along each row of dirs (FP64)."""
    th = np.asarray(theta, dtype=np.float64)
    e = np.asarray(eloc_ref, dtype=np.float64)
    c = 2.0 * (e - e.mean()) / e.size
    out = []
    for d in dirs:
        fp = c @ logpsi_fn(th + eps * d)
        fm = c @ logpsi_fn(th - eps * d)
        out.append((fp - fm) / (2 * eps))
    return np.array(out)


def check_energy_gradient(g, logpsi_fn, theta, eloc_ref, seed, n_top=24, n_rand=24, n_dir=4,
                          tol=1e-3):
    """Checks a device energy gradient g [P] element by element on n_top of
    its largest and n_rand random coordinates, and along n_dir random
    directions, against the finite-difference reference.  Element bound:
    tol of the largest reference component among the checked ones;
    direction bound: tol of ||g|| ||d||."""
    g = np.asarray(g, dtype=np.float64)
    P = g.size
    rng = np.random.default_rng(seed)
    top = np.argsort(-np.abs(g))[:n_top]
    rest = np.setdiff1d(np.arange(P), top)
    coords = np.concatenate([top, rng.choice(rest, n_rand, replace=False)])
    eye = np.zeros((coords.size, P))
    eye[np.arange(coords.size), coords] = 1.0
    ref_k = energy_gradient_fd(logpsi_fn, theta, eloc_ref, eye)
    scale = np.max(np.abs(ref_k))
    assert scale > 0.0
    err = np.abs(g[coords] - ref_k)
    assert np.all(err <= tol * scale), (err.max() / scale, coords[np.argmax(err)])
    dirs = rng.standard_normal((n_dir, P))
    ref_d = energy_gradient_fd(logpsi_fn, theta, eloc_ref, dirs)
    bound = tol * np.linalg.norm(g) * np.linalg.norm(dirs, axis=1)
    assert np.all(np.abs(dirs @ g - ref_d) <= bound), (np.abs(dirs @ g - ref_d) / bound).max()
    return ref_k
