"""FP64 CPU oracle for the deflated Hutchinson estimator of tr(A^-1).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of what the GPU library computes, written from the paper
"Multigrid deflation for Lattice QCD" (Romero, Stathopoulos, Orginos,
arXiv:1909.12234).  Only the test suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The product path (``paper_1909_12234_gb300``) never imports, links or runs
anything here, and nothing here imports the product.

Conventions shared by every module (all FP64 / complex128):

* lattice dims ``(Lx, Ly, Lz, Lt)``, direction mu = 0..3 <-> x, y, z, t,
  periodic boundaries;
* lexicographic site index ``x + Lx*(y + Ly*(z + Lz*t))``;
* a fermion field is an array of shape ``(V, 4, 3)`` (spin, colour) or
  ``(V, 4, 3, s)`` for s right-hand sides, sites in lexicographic order;
* gauge links ``U`` have shape ``(4, V, 3, 3)``: ``U[mu, n]`` lives on the
  link from site n to n + mu.

Modules:

* ``philox``     counter-based generator (Salmon et al., SC'11) and the
                 Rademacher noise of Sec. 1 (the x_j of Eq. 1);
* ``lattice``    site indexing, even-odd maps, neighbours, aggregates (Sec. 2);
* ``wilson``     gamma matrices and the Wilson-Dirac operator;
* ``dense``      dense assembly, LU trace, exact variances (Eq. 2);
* ``krylov``     GCR / minimal-residual solvers (Sec. 1 inexact solve, Sec. 2);
* ``multigrid``  adaptive setup, blocking, W^H A W, V-cycle (Sec. 2);
* ``deflation``  Algorithm 1 and Algorithm 2 deflation spaces and projectors;
* ``smoother``   the learned gauge-covariant smoother (an extension; the paper
                 has no counterpart) and its least-squares fit;
* ``estimator``  the Hutchinson loop, t0 + t1, statistics and jackknife.

Pinned functions are checked by ``tests/test_oracle_*.py`` against closed
forms, brute force and published known-answer values.  Functions without
such a pin say "parity unpinned" in their docstring.
"""
