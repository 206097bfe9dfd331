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
    _check(P, *W.one_ellipse_640(), "fp16_ir", nrhs, 2.0 ** -11)


@pytest.mark.parametrize("prec,u", [("fp16_ir", 2.0 ** -11), ("bf16_ir", 2.0 ** -8)])
def test_matmat_ragged(P, prec, u):
    _check(P, *W.random_geometry(np.random.default_rng(3), 1001), prec, 9, u)


def test_matmat_errors(P):
    import torch
    g, f, ph = W.one_ellipse_640()
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


# ---------------------------------------------------------------------------
# bie_solve_multi: several right-hand sides on one matrix.  Every column is an
# ordinary system of eq. lin:sys, so the bounds are the single-solve parity
# bounds: relative 2-norm error of omega and U within 1e-11 of the oracle's
# dense FP64 LU solution, relative residual 1e-14.
# ---------------------------------------------------------------------------

def _phits(M0, nrhs, seed):
    rng = np.random.default_rng(seed)
    amps = 0.05 * 10.0 ** rng.uniform(-3, 1, nrhs)     # columns of very different size
    return np.stack([W.filtered_noise(rng, M0, a, int(rng.integers(4, 40))) for a in amps])


def _solve_multi(P, g, f, PH, prec, **kw):
    import torch
    prob = P.Problem(g, f, PH[0])
    try:
        prob.assemble(prec)
        ph = torch.as_tensor(PH, device="cuda").contiguous()
        om = torch.empty((len(PH), g.N), dtype=torch.float64, device="cuda")
        U = torch.empty((len(PH), g.M[0]), dtype=torch.float64, device="cuda")
        infos = P.bie_solve_multi(prob.ctx, ph, om, U, P.bie_default_opts(**kw))
        return om.cpu().numpy(), U.cpu().numpy(), infos
    finally:
        prob.close()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("prec,nrhs", [("fp16_ir", 5), ("bf16_ir", 5), ("fp16_ir", 17),
                                       ("bf16_ir", 40)])
def test_solve_multi_matches_oracle(P, prec, nrhs):
    g, f, _ = W.random_geometry(np.random.default_rng(11), 1001)
    PH = _phits(g.M[0], nrhs, nrhs)
    om, U, infos = _solve_multi(P, g, f, PH, prec)
    for r in range(nrhs):
        om_ref, U_ref, _ = O.solve(g, f, PH[r])
        assert infos[r].converged and infos[r].rel_resid <= 1e-14, (r, infos[r].as_dict())
        assert _rel(om[r], om_ref) <= 1e-11, (r, _rel(om[r], om_ref))
        assert _rel(U[r], U_ref) <= 1e-11, (r, _rel(U[r], U_ref))


def test_solve_multi_paper_problem_and_single_solves(P):
    """A worked-example geometry of Sec. 5 with 3 columns; each agrees with a
    single bie_solve of the same storage."""
    import torch
    g, f, ph = W.paper_problem(3)
    PH = np.stack([ph, 0.3 * ph[::-1].copy(), _phits(g.M[0], 1, 5)[0]])
    om, U, infos = _solve_multi(P, g, f, PH, "fp16_ir")
    for r in range(3):
        om_ref, U_ref, _ = O.solve(g, f, PH[r])
        assert _rel(om[r], om_ref) <= 1e-11 and _rel(U[r], U_ref) <= 1e-11
        prob = P.Problem(g, f, PH[r])
        try:
            prob.assemble("fp16_ir")
            prob.solve()
            assert _rel(om[r], prob.omega.cpu().numpy()) <= 1e-12
            assert _rel(U[r], prob.U.cpu().numpy()) <= 1e-11
        finally:
            prob.close()


def test_solve_multi_degenerate_columns(P):
    """No flow and a zero column: b = 0 there, the column is done before the
    first Arnoldi step (omega = U = 0 exactly) while the others iterate; one
    column alone; a repeated column gives the same answer."""
    g = W.simple_channel(M0=256, M1=144, h=1.2)
    f = W.Flow(V1=0.0, a=np.array([]))
    base = _phits(256, 3, 9)
    PH = np.stack([base[0], np.zeros(256), base[1], base[0], base[2]])
    om, U, infos = _solve_multi(P, g, f, PH, "fp16_ir")
    assert np.all(om[1] == 0.0) and np.all(U[1] == 0.0)
    assert infos[1].converged and infos[1].iters == 0
    for r in (0, 2, 4):
        om_ref, U_ref, _ = O.solve(g, f, PH[r])
        assert infos[r].converged and infos[r].iters > 0
        assert _rel(om[r], om_ref) <= 1e-11 and _rel(U[r], U_ref) <= 1e-11
    assert _rel(om[3], om[0]) <= 1e-13 and _rel(U[3], U[0]) <= 1e-13
    om1, U1, inf1 = _solve_multi(P, g, f, PH[2:3], "bf16_ir")
    assert inf1[0].converged and _rel(om1[0], om[2]) <= 1e-12 and _rel(U1[0], U[2]) <= 1e-11


def test_solve_multi_errors(P):
    import torch
    g, f, ph = W.one_ellipse_640()
    prob = P.Problem(g, f, ph)
    try:
        PH = torch.zeros((3, g.M[0]), dtype=torch.float64, device="cuda")
        om = torch.empty((3, g.N), dtype=torch.float64, device="cuda")
        U = torch.empty((3, g.M[0]), dtype=torch.float64, device="cuda")
        with pytest.raises(P.BieError) as e:           # not assembled
            P.bie_solve_multi(prob.ctx, PH, om, U)
        assert e.value.status == P.BIE_ERR_STATE
        prob.assemble("fp32_ir")
        with pytest.raises(P.BieError) as e:           # no tensor-core storage
            P.bie_solve_multi(prob.ctx, PH, om, U)
        assert e.value.status == P.BIE_ERR_STATE
        prob.assemble("bf16_ir")
        with pytest.raises(P.BieError) as e:
            P.bie_solve_multi(prob.ctx, PH, om, U, P.bie_default_opts(restart=64))
        assert e.value.status == P.BIE_ERR_ARG
        PH65 = torch.zeros((65, g.M[0]), dtype=torch.float64, device="cuda")
        with pytest.raises(P.BieError) as e:
            P.bie_solve_multi(prob.ctx, PH65, om, U)
        assert e.value.status == P.BIE_ERR_ARG
        # one cycle of 2 steps cannot reach 1e-14: NOCONV, with omega written
        infos = P.bie_solve_multi(prob.ctx, PH + 0.01, om, U,
                                  P.bie_default_opts(restart=2, max_cycles=1),
                                  raise_on_noconv=False)
        assert not any(i.converged for i in infos)
        assert all(i.cycles == 1 and 1 <= i.iters <= 2 for i in infos)
    finally:
        prob.close()


def test_solve_multi_full_size_sampled(P):
    """The 16383-unknown workload (8192 + 4096 + 3 x 1365) with 16 right-hand sides: every column
    converges; sampled rows of the oracle's system are solved to 1e-12 of
    ||b||_inf and sampled U values match the oracle's evaluation."""
    import torch
    g, f, ph = W.three_ellipses_16383()
    PH = _phits(g.M[0], 16, 2)
    om, U, infos = _solve_multi(P, g, f, PH, "fp16_ir")
    assert all(i.converged for i in infos)
    rows = np.random.default_rng(0).choice(g.N, 24, replace=False)
    rows = np.unique(np.concatenate([rows, g.offsets()[:-1], g.offsets()[1:] - 1]))
    K = O.kernel_rows(g, rows)
    tg = np.sort(np.random.default_rng(1).choice(g.M[0], 8, replace=False))
    for r in (0, 7, 15):
        b = O.rhs(g, f, PH[r])
        res = b[rows] - K @ om[r]
        assert np.abs(res).max() <= 1e-12 * np.abs(b).max(), r
        Uref = O.normal_velocity(g, f, om[r], targets=tg)
        assert np.abs(U[r][tg] - Uref).max() <= 1e-11 * np.abs(Uref).max(), r


@pytest.mark.parametrize("nrhs,prec", [(8, "fp16_ir"), (32, "fp16_ir"), (3, "fp16_ir"),
                                       (12, "bf16_ir")])
def test_solve_multi_reported_residual_is_the_true_one(P, nrhs, prec):
    """Once every refining column's residual is the full-accuracy one and small,
    the multi-column solver updates the residuals from the last increments
    with as many exact slices as the residual needs (8 columns or more; with
    fewer it keeps direct products); the residual each column reports must be
    that of its returned omega, measured with the hi + lo product of the same
    storage."""
    import torch
    g, f, _ = W.three_ellipses_16383()
    PH = _phits(g.M[0], nrhs, 5)
    prob = P.Problem(g, f, PH[0])
    try:
        prob.assemble(prec)
        ph = torch.as_tensor(PH, device="cuda").contiguous()
        om = torch.empty((nrhs, g.N), dtype=torch.float64, device="cuda")
        U = torch.empty((nrhs, g.M[0]), dtype=torch.float64, device="cuda")
        infos = P.bie_solve_multi(prob.ctx, ph, om, U, P.bie_default_opts())
        b = torch.empty(g.N, dtype=torch.float64, device="cuda")
        y = torch.empty_like(b)
        for r in range(nrhs):
            P.bie_rhs(prob.ctx, ph[r].contiguous(), b)
            P.bie_matvec(prob.ctx, 1, om[r].contiguous(), y)
            true = ((b - y).norm() / b.norm()).item()
            assert infos[r].converged and true <= 1.2e-14, (r, true, infos[r].as_dict())
            # (an update does not see the rounding of omega itself, ~1e-16 of
            # ||A|| ||omega|| per update; the exact-slice products truncate below
            # 2^-50 of each row's scale): up to 7e-16 measured, a tenth of rtol
            assert abs(true - infos[r].rel_resid) <= 1e-15, (r, true, infos[r].rel_resid)
    finally:
        prob.close()


# ---------------------------------------------------------------------------
# bie_matmat_full: the hi + lo operator on the tensor cores by exact slices.
# The slice GEMMs are exact; what remains is the storage's own ~2^-48 and the
# truncation below 2^-50 of each row's scale, so the product matches the
# oracle's FP64 A x to 1e-13 of sum_l |A_ml| |x_l| and the double-float
# hi + lo GEMV (bie_matvec, which = 1) to 1e-14 of that scale.
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec,nrhs", [("fp16_ir", 1), ("fp16_ir", 7), ("fp32_ir", 24),
                                       ("bf16_ir", 64)])
def test_matmat_full_is_exact(P, prec, nrhs):
    import torch
    g, f, ph = W.random_geometry(np.random.default_rng(6), 1001)
    A = O.assemble(g)
    X = np.random.default_rng(nrhs).standard_normal((nrhs, g.N))
    X[0] *= 1e4
    if nrhs > 2:
        X[2] *= 1e-6
    prob = P.Problem(g, f, ph)
    try:
        prob.assemble(prec)
        Xd = torch.as_tensor(X, device="cuda").contiguous()
        Yd = torch.empty_like(Xd)
        P.bie_matmat_full(prob.ctx, Xd, Yd)
        Y = Yd.cpu().numpy()
        scale = np.abs(X) @ np.abs(A).T
        assert np.all(np.abs(Y - X @ A.T) <= 1e-13 * scale)
        for r in sorted({0, nrhs - 1}):
            y1 = torch.empty(g.N, dtype=torch.float64, device="cuda")
            P.bie_matvec(prob.ctx, 1, Xd[r].contiguous(), y1)
            assert np.all(np.abs(Y[r] - y1.cpu().numpy()) <= 1e-14 * scale[r]), r
        # a second call reuses the slices of this assembly and gives the same bits
        Y2 = torch.empty_like(Xd)
        P.bie_matmat_full(prob.ctx, Xd, Y2)
        assert torch.equal(Yd, Y2)
    finally:
        prob.close()


def test_matmat_full_full_size(P):
    """16383 unknowns (ld = 16384, the exactness limit of one accumulation):
    sampled rows against the oracle's rows."""
    import torch
    g, f, ph = W.three_ellipses_16383()
    X = np.random.default_rng(1).standard_normal((5, g.N))
    prob = P.Problem(g, f, ph)
    try:
        prob.assemble("fp16_ir")
        Xd = torch.as_tensor(X, device="cuda").contiguous()
        Yd = torch.empty_like(Xd)
        P.bie_matmat_full(prob.ctx, Xd, Yd)
        rows = np.unique(np.concatenate([np.random.default_rng(2).choice(g.N, 24, replace=False),
                                         g.offsets()[:-1], g.offsets()[1:] - 1]))
        K = O.kernel_rows(g, rows)
        ref = X @ K.T
        scale = np.abs(X) @ np.abs(K).T
        assert np.all(np.abs(Yd.cpu().numpy()[:, rows] - ref) <= 1e-13 * scale)
    finally:
        prob.close()
