"""Pins for oracle.lattice by brute force over every site."""
import numpy as np
import pytest

from oracle import lattice

DIMS = [(4, 4, 4, 4), (6, 6, 6, 6), (8, 8, 8, 4), (4, 2, 6, 8), (2, 2, 2, 2)]


@pytest.mark.parametrize("dims", DIMS)
def test_coords_roundtrip(dims):
    c = lattice.coords(dims)
    V = lattice.volume(dims)
    assert c.shape == (V, 4)
    assert np.array_equal(lattice.lex_index(dims, c), np.arange(V))
    assert np.all(c >= 0) and np.all(c < np.asarray(dims))
    # brute force: every coordinate tuple appears exactly once
    assert len({tuple(r) for r in c}) == V


@pytest.mark.parametrize("dims", DIMS)
def test_even_odd_map(dims):
    V = lattice.volume(dims)
    eo = lattice.eo_index(dims)
    par = lattice.parity(dims)
    assert np.array_equal(np.sort(eo), np.arange(V))
    assert np.all((eo < V // 2) == (par == 0))
    # brute force: within a parity the order follows the lexicographic order
    for p in (0, 1):
        lex_p = np.nonzero(par == p)[0]
        assert np.array_equal(eo[lex_p], p * V // 2 + np.arange(V // 2))


def test_even_odd_needs_even_lx():
    with pytest.raises(ValueError):
        lattice.eo_index((3, 4, 4, 4))


@pytest.mark.parametrize("dims", DIMS)
def test_neighbours(dims):
    c = lattice.coords(dims)
    nb = lattice.neighbours(dims)
    for mu in range(4):
        step = np.zeros(4, dtype=int)
        step[mu] = 1
        for n in range(len(c)):
            assert tuple(c[nb[0, mu, n]]) == tuple((c[n] + step) % dims)
            assert tuple(c[nb[1, mu, n]]) == tuple((c[n] - step) % dims)
        assert np.array_equal(nb[1, mu][nb[0, mu]], np.arange(len(c)))
        # even-odd: every neighbour has the opposite parity when all L are even
        if all(L % 2 == 0 for L in dims):
            par = lattice.parity(dims)
            assert np.all(par[nb[0, mu]] != par)


@pytest.mark.parametrize("dims,block", [((4, 4, 4, 4), (2, 2, 2, 2)),
                                        ((8, 8, 8, 4), (2, 2, 2, 2)),
                                        ((4, 2, 6, 8), (2, 1, 3, 4))])
def test_aggregates(dims, block):
    c = lattice.coords(dims)
    agg = lattice.aggregate_of(dims, block)
    cd = lattice.coarse_dims(dims, block)
    mem = lattice.aggregate_members(dims, block)
    assert mem.shape == (lattice.volume(cd), int(np.prod(block)))
    assert np.array_equal(np.sort(mem.ravel()), np.arange(len(c)))
    for a in range(mem.shape[0]):
        cc = c[mem[a]] // np.asarray(block)
        assert np.all(cc == cc[0])
        assert lattice.lex_index(cd, cc[0]) == a
        assert np.all(agg[mem[a]] == a)
    with pytest.raises(ValueError):
        lattice.coarse_dims(dims, (3, 3, 3, 3))
