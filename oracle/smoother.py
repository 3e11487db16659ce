"""Learned gauge-covariant smoother (not in the paper: an extension of the
multigrid V-cycle's smoothing step).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The smoother is one linear layer of link-transported one-hop terms:

    (S r)(x)_{o,a} = sum_{d=0..8} sum_{i=0..3} w[d, o, i] (T_d r)(x)_{i,a},

with o, i spin indices, a colour, and the transports
T_0 r(x) = r(x), T_{1+mu} r(x) = U_mu(x) r(x + mu),
T_{5+mu} r(x) = U_mu(x - mu)^H r(x - mu).  Colour is only ever moved by the
links, so S commutes with every gauge transformation (links
U_mu(x) -> g(x) U_mu(x) g(x+mu)^H, fields r(x) -> g(x) r(x)).  The Wilson
operator is the member with w[0] = (4 + m0) 1, w[1+mu] = -(1 - gamma_mu)/2,
w[5+mu] = -(1 + gamma_mu)/2.

Training: given pairs (e_j, r_j), the weights minimise sum_j ||e_j - S r_j||^2.
S r is linear in w and the rows of different output spins o do not share
weights, so for each o this is one linear least-squares problem with the 36
features f = [(T_d r)(x)_{i,a}]_{(d, i)} per (x, a, j) row; numpy's lstsq
solves it (a library routine standing in for the normal equations).

Pins (tests/test_oracle_smoother.py): the Wilson weights reproduce
``wilson.dirac_apply``; a fit to pairs made by planted weights recovers them;
gauge covariance; w[0] = 1, others 0 is the identity.
"""

import numpy as np

from . import lattice, wilson


def transport(U, r, dims, d):
    """T_d r for a field r of shape (V, 4, 3[, s]) (d = 0..8)."""
    r = np.asarray(r, dtype=np.complex128)
    if d == 0:
        return r.copy()
    nb = lattice.neighbours(dims)
    if d <= 4:
        mu = d - 1
        M = U[mu]                                   # U_mu(x)
        src = r[nb[0, mu]]                          # r(x + mu)
    else:
        mu = d - 5
        M = np.conj(np.swapaxes(U[mu][nb[1, mu]], -1, -2))  # U_mu(x - mu)^H
        src = r[nb[1, mu]]                          # r(x - mu)
    return np.einsum("vab,vsb...->vsa...", M, src)


def apply(U, w, r, dims):
    """S r for weights w of shape (9, 4, 4)."""
    w = np.asarray(w, dtype=np.complex128)
    out = np.zeros_like(np.asarray(r, dtype=np.complex128))
    for d in range(9):
        out += np.einsum("oi,via...->voa...", w[d], transport(U, r, dims, d))
    return out


def wilson_weights(m0):
    """The weights for which S is the Wilson operator A(m0)."""
    g = wilson.gammas()
    one = np.eye(4, dtype=np.complex128)
    w = np.zeros((9, 4, 4), dtype=np.complex128)
    w[0] = (4.0 + m0) * one
    for mu in range(4):
        w[1 + mu] = -0.5 * (one - g[mu])
        w[5 + mu] = -0.5 * (one + g[mu])
    return w


def fit(U, E, R, dims):
    """Least-squares weights for pairs (e_j, r_j), fields of shape (V, 4, 3, s)."""
    R = np.asarray(R, dtype=np.complex128)
    E = np.asarray(E, dtype=np.complex128)
    V, s = R.shape[0], R.shape[3]
    # F[(v, a, j), (d, i)] = (T_d r_j)(v)_{i, a}
    F = np.empty((V, 3, s, 9, 4), dtype=np.complex128)
    for d in range(9):
        F[:, :, :, d, :] = np.transpose(transport(U, R, dims, d), (0, 2, 3, 1))
    F = F.reshape(V * 3 * s, 36)
    w = np.zeros((9, 4, 4), dtype=np.complex128)
    for o in range(4):
        y = E[:, o, :, :].reshape(V * 3 * s)       # rows (v, a, j)
        sol, *_ = np.linalg.lstsq(F, y, rcond=None)
        w[:, o, :] = sol.reshape(9, 4)
    return w
