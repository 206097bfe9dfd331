"""Tensor-core multi-vector products (bie_matmat) vs the oracle's matrix.

Y_r = A X_r with the FP16 / BF16 storage: every stored entry carries a
relative rounding of 2^-11 (FP16) or 2^-8 (BF16) and every column of X is
rounded once to the same type, so each output obeys
  |Y - A X|_m <= 2 u sum_l |A_ml| |x_l| + (FP32 accumulation),
u the storage's unit roundoff; the test allows 3u.  Cases: 640 unknowns,
1001 (ragged tiles and K ranges), 6 to 64 right-hand sides (padding of the
MMA's N = 16 / 32 / 64).
"""
import numpy as np
import pytest

import workloads as W
from oracle import bie as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2108_01786_gb300 as P
    from paper_2108_01786_gb300 import _build
    _build.build()
    return P


def _check(P, g, f, ph, prec, nrhs, u):
    import torch
    A = O.assemble(g)
    X = np.random.default_rng(nrhs).standard_normal((nrhs, g.N))
    X[0] *= 1e3                       # columns of very different size
    if nrhs > 1:
        X[1] *= 1e-4
    prob = P.Problem(g, f, ph)
    try:
        prob.assemble(prec)
        Xd = torch.as_tensor(X, device="cuda").contiguous()
        Yd = torch.empty_like(Xd)
        P.bie_matmat(prob.ctx, Xd, Yd)
        Y = Yd.cpu().numpy()
        ref = X @ A.T
        bound = 3 * u * (np.abs(X) @ np.abs(A).T) + 1e-12 * np.abs(ref)
        assert np.all(np.abs(Y - ref) <= bound), np.max(np.abs(Y - ref) / bound)
        # agrees with one inner-storage product per column within the same bound
        y0 = torch.empty(g.N, dtype=torch.float64, device="cuda")
        P.bie_matvec(prob.ctx, 0, Xd[nrhs - 1].contiguous(), y0)
        assert np.all(np.abs(Y[nrhs - 1] - y0.cpu().numpy()) <= 2 * bound[nrhs - 1])
    finally:
        prob.close()


@pytest.mark.parametrize("nrhs", [6, 16, 17, 40, 64])
def test_matmat_fp16_matches_oracle(P, nrhs):
    _check(P, *W.config1(), "fp16_ir", nrhs, 2.0 ** -11)


@pytest.mark.parametrize("prec,u", [("fp16_ir", 2.0 ** -11), ("bf16_ir", 2.0 ** -8)])
def test_matmat_ragged(P, prec, u):
    _check(P, *W.config1_type(np.random.default_rng(3), 1001), prec, 9, u)


def test_matmat_errors(P):
    import torch
    g, f, ph = W.config1()
    prob = P.Problem(g, f, ph)
    try:
        X = torch.zeros((4, g.N), dtype=torch.float64, device="cuda")
        prob.assemble("fp32_ir")
        with pytest.raises(P.BieError) as e:
            P.bie_matmat(prob.ctx, X, torch.empty_like(X))
        assert e.value.status == P.BIE_ERR_STATE
        prob.assemble("fp16_ir")
        X65 = torch.zeros((65, g.N), dtype=torch.float64, device="cuda")
        with pytest.raises(P.BieError) as e:
            P.bie_matmat(prob.ctx, X65, torch.empty_like(X65))
        assert e.value.status == P.BIE_ERR_ARG
    finally:
        prob.close()
