"""Lattice geometry: site indexing, even-odd maps, neighbours and aggregates.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

* Sec. 1 names red-black (even-odd) partitioning, and Sec. 3 (the paragraph
  after Algorithm 2) builds the solver on the odd-even operator; the parity of
  site n is (x+y+z+t) mod 2.
* Sec. 2 ("blocking") splits the lattice into disjoint subdomains D_j; here
  they are the hypercubic blocks of Table 2 (e.g. 2^4 sites).

Even-odd index (this library's reading; the paper fixes no storage order):
``eo(n) = parity(n) * V/2 + lex(n) // 2``, which needs an even Lx.

Pinned by brute force over every site in ``tests/test_oracle_lattice.py``.
"""

import functools
import itertools

import numpy as np


def volume(dims):
    return int(np.prod(dims))


@functools.lru_cache(maxsize=32)
def _coords(dims):
    V = volume(dims)
    out = np.empty((V, 4), dtype=np.int64)
    for n, (t, z, y, x) in enumerate(itertools.product(*[range(L) for L in dims[::-1]])):
        out[n] = (x, y, z, t)
    out.setflags(write=False)
    return out


def coords(dims):
    """(V, 4) int array: coordinates of every lexicographic site."""
    return _coords(tuple(int(d) for d in dims))


def lex_index(dims, c):
    """Lexicographic index of coordinates c (..., 4)."""
    c = np.asarray(c)
    Lx, Ly, Lz, _ = dims
    return c[..., 0] + Lx * (c[..., 1] + Ly * (c[..., 2] + Lz * c[..., 3]))


def parity(dims):
    c = coords(dims)
    return c.sum(axis=1) % 2


def eo_index(dims):
    """eo_index(dims)[lex] = even-odd index of that site."""
    if dims[0] % 2:
        raise ValueError("even-odd ordering needs an even Lx")
    V = volume(dims)
    lex = np.arange(V)
    return parity(dims) * (V // 2) + lex // 2


def neighbours(dims):
    """(2, 4, V) lexicographic indices: [0, mu, n] = n + mu, [1, mu, n] = n - mu."""
    return _neighbours(tuple(int(d) for d in dims))


@functools.lru_cache(maxsize=32)
def _neighbours(dims):
    c = coords(dims)
    out = np.empty((2, 4, len(c)), dtype=np.int64)
    for mu in range(4):
        step = np.zeros(4, dtype=np.int64)
        step[mu] = 1
        out[0, mu] = lex_index(dims, (c + step) % np.asarray(dims))
        out[1, mu] = lex_index(dims, (c - step) % np.asarray(dims))
    out.setflags(write=False)
    return out


def coarse_dims(dims, block):
    for L, b in zip(dims, block):
        if L % b:
            raise ValueError(f"block {block} does not divide lattice {dims}")
    return tuple(L // b for L, b in zip(dims, block))


def aggregate_of(dims, block):
    """aggregate_of(dims, block)[lex] = lexicographic index of its aggregate
    on the coarse lattice dims // block (the subdomain D_j of Sec. 2)."""
    cd = coarse_dims(dims, block)
    c = coords(dims) // np.asarray(block)
    return lex_index(cd, c)


def aggregate_members(dims, block):
    """(V_c, b) array: the fine lexicographic sites of each aggregate, in
    increasing lexicographic order."""
    agg = aggregate_of(dims, block)
    Vc = volume(coarse_dims(dims, block))
    b = volume(dims) // Vc
    out = np.empty((Vc, b), dtype=np.int64)
    for a in range(Vc):
        out[a] = np.nonzero(agg == a)[0]
    return out
