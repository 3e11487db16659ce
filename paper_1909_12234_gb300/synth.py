"""Seeded synthetic inputs: random SU(3) gauge fields and plain random fields.

This module holds no arithmetic of the method itself.  It makes the inputs
that both the GPU library and its independent CPU checker consume, in the
canonical host layout of ``include/qdtrace.h``:

* gauge links: complex128 array ``(4, V, 3, 3)``, ``U[mu, lex]`` on the link
  from site lex to lex + mu; use :func:`links_to_canonical` to get the
  ``[V][4][3][3]`` order the C-ABI reads;
* fermion fields: complex128 ``(V, 4, 3[, s])``, lexicographic sites.

Gauge recipe (stands in for the paper's clover ensembles 32^3x64 and
64^3x128 at beta = 6.3, which are not available): per link draw a 3x3 matrix
G with i.i.d. entries N(0,1) + i N(0,1), take the Hermitian traceless part
H = (G + G^H)/2 - tr(...)/3, and set U = exp(i eps H) through the eigen-
decomposition of H.  eps = 0 (or ``unit=True``) gives the free field.
"""

import numpy as np


def random_su3_links(dims, eps, seed, unit=False):
    V = int(np.prod(dims))
    if unit or eps == 0.0:
        return np.broadcast_to(np.eye(3, dtype=np.complex128), (4, V, 3, 3)).copy()
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((4, V, 3, 3)) + 1j * rng.standard_normal((4, V, 3, 3))
    H = 0.5 * (G + np.conj(np.swapaxes(G, -1, -2)))
    tr = np.trace(H, axis1=-2, axis2=-1).real / 3.0
    H = H - tr[..., None, None] * np.eye(3)
    w, Q = np.linalg.eigh(H)
    phase = np.exp(1j * eps * w)
    U = np.einsum("...ij,...j,...kj->...ik", Q, phase, Q.conj())
    return U


def gauge_transform(U, dims, seed):
    """Random SU(3) gauge transformation g(n): U_mu(n) -> g(n) U_mu(n) g(n+mu)^H.

    Returns (U', g).  Used only to build test inputs for gauge covariance.
    """
    V = int(np.prod(dims))
    g = random_su3_links(dims, 1.0, seed)[0]
    Lx, Ly, Lz, Lt = dims
    lex = np.arange(V)
    c = np.stack([lex % Lx, (lex // Lx) % Ly, (lex // (Lx * Ly)) % Lz, lex // (Lx * Ly * Lz)], 1)
    out = np.empty_like(U)
    for mu in range(4):
        cp = c.copy()
        cp[:, mu] = (cp[:, mu] + 1) % dims[mu]
        fwd = cp[:, 0] + Lx * (cp[:, 1] + Ly * (cp[:, 2] + Lz * cp[:, 3]))
        out[mu] = g @ U[mu] @ np.conj(np.swapaxes(g[fwd], -1, -2))
    return out, g


def links_to_canonical(U):
    """(4, V, 3, 3) -> contiguous (V, 4, 3, 3), the C-ABI's host link layout."""
    return np.ascontiguousarray(np.transpose(U, (1, 0, 2, 3)))


def random_field(dims, nrhs, seed):
    """Complex Gaussian fermion field (V, 4, 3, nrhs)."""
    V = int(np.prod(dims))
    rng = np.random.default_rng(seed)
    shape = (V, 4, 3, nrhs)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
