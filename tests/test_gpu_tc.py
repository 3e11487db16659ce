"""The coarsest solve of the FP32 V-cycle on tcgen05 tensor cores (BF16
operands, FP32 accumulate) against the oracle's solve with its own coarse
operator C = W^H A W (null_maxit = 0: both sides block the same Philox
starts), for several right-hand-side counts including a ragged 16-column tail
and a chunked batch.

The GPU applies X = C^{-1} computed once by FP32 Gauss-Jordan with partial
pivoting, rounded to BF16 (u = 2^-8) together with the input, products summed
in FP32.  Tolerance per output i, against y = C^{-1} x from the oracle's
sparse LU (scipy splu):
  (2u + u^2 + 2^-22) S_i  with S = P(C^{-1}) P(x), P(z) = |Re z| + |Im z|,
for the BF16 rounding of both operands and the FP32 sums, plus
  4 sqrt(n) 2^-24 kappa_inf(C) ||C^{-1}||_inf ||x||_inf
for the FP32 inversion (the typical error of Gauss-Jordan with partial
pivoting, u kappa with sqrt(n) growth of rounding errors, times the factor 4).
The FP32 CUDA-core product of the same inverse is held to the second term
plus 2^-22 S_i."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import multigrid as omg
from paper_1909_12234_gb300 import synth

from gpu_util import host, need_gpu, torch

pytestmark = pytest.mark.gpu

U_BF16 = 2.0 ** -8


@pytest.fixture(scope="module")
def qd():
    need_gpu()
    from paper_1909_12234_gb300 import qdtrace
    qdtrace.load()
    return qdtrace


@pytest.fixture(scope="module")
def ctx(qd):
    return qd.Context(0)


def _P(M):
    return np.abs(M.real) + np.abs(M.imag)


def _oracle(U, dims, m0, nv):
    H = omg.setup(U, m0, dims, [(2, 2, 2, 2)], [nv], seed=5, null_maxit=0)
    C = H.matrices[0].tocsc()
    lu = spla.splu(C)
    Cinv = np.linalg.inv(C.toarray())
    Cd = C.toarray()
    kappa = np.abs(Cd).sum(axis=1).max() * np.abs(Cinv).sum(axis=1).max()
    return lu, Cinv, kappa


def _gpu_solve(qd, mg, n, s, x):
    x32 = torch.from_numpy(np.ascontiguousarray(x.astype(np.complex64))).to("cuda:0")
    y32 = torch.empty((n, s), dtype=torch.complex64, device="cuda:0")
    qd.coarse_solve_f32(mg, 1, s, x32, y32)
    return host(y32).astype(np.complex128), x32


@pytest.mark.parametrize("dims,m0,nv,svals", [((4, 4, 4, 4), -0.4, 6, [3, 64]),
                                              ((8, 8, 8, 8), -0.8, 12, [64, 5, 130])])
def test_tensor_core_coarsest_solve_against_oracle(qd, ctx, dims, m0, nv, svals):
    U = synth.random_su3_links(dims, 0.3, 2)
    g = qd.Gauge(ctx, dims, U)
    n = (int(np.prod(dims)) // 16) * 2 * nv
    lu, Cinv, kappa = _oracle(U, dims, m0, nv)
    inv_norm = np.abs(Cinv).sum(axis=1).max()
    for bf16 in (1, 0):
        mg = qd.Multigrid(ctx, g, m0, 0.0, qd.mg_params(1, [(2, 2, 2, 2)], [nv], null_maxit=0, seed=5,
                                                       coarsest_bf16=bf16))
        rng = np.random.default_rng(11)
        for s in svals:
            x = rng.standard_normal((n, s)) + 1j * rng.standard_normal((n, s))
            got, x32 = _gpu_solve(qd, mg, n, s, x)
            xs = host(x32).astype(np.complex128)  # the FP32 input both sides solve with
            ref = lu.solve(xs)
            S = _P(Cinv) @ _P(xs)
            inv_term = 4.0 * np.sqrt(n) * 2.0 ** -24 * kappa * inv_norm * np.abs(xs).max(axis=0)
            coef = (2 * U_BF16 + U_BF16 ** 2 + 2.0 ** -22) if bf16 else 2.0 ** -22
            tol = coef * S + inv_term[None, :]
            err = np.abs(got - ref)
            assert np.all(err <= tol), (bf16, s, float((err / tol).max()))
            # not vacuous: the column errors are at the operands' rounding level
            colerr = np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)
            assert colerr.max() < (3e-2 if bf16 else 1e-3), (bf16, s, colerr.max())
        mg.close()
    g.close()
