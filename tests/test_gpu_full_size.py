"""Full-size checks at 32768 unknowns (the large-solve + interior-field workload).

The oracle cannot factor this system in a test's time, so the checks use
outputs it computes one by one, or properties that hold at any size:
  * the GPU densities solve the oracle's system: residual of sampled rows,
    rows assembled by the oracle (kernel_rows), relative to ||b||_inf;
  * the normal velocity of a seeded smooth density on sampled surface nodes
    (oracle normal_velocity with a target subset);
  * far-field velocities of sampled grid targets (oracle velocity_far);
  * the exact field of a DtN pair on a 32768-node channel, at ~10^4 targets
    including targets within 2 node spacings of the boundaries (Helsing),
    within four times the FP64 floor of the method at that size.
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


@pytest.fixture(scope="module")
def four_ellipses_32768():
    return W.four_ellipses_32768()


def _ct(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.complex128, device="cuda")


def test_32768_solve_residual_sampled_rows(P, four_ellipses_32768):
    g, f, ph = four_ellipses_32768
    b = O.rhs(g, f, ph)
    rows = np.random.default_rng(7).choice(g.N, 48, replace=False)
    rows = np.unique(np.concatenate([rows, g.offsets()[:-1], g.offsets()[1:] - 1]))
    A_rows = O.kernel_rows(g, rows)
    prob = P.Problem(g, f, ph)
    try:
        prob.assemble("fp32_ir")
        info = prob.solve()
        assert info.converged
        om = prob.omega.cpu().numpy()
        r = b[rows] - A_rows @ om
        assert np.abs(r).max() <= 1e-12 * np.abs(b).max()
    finally:
        prob.close()


def test_32768_normal_velocity_sampled_nodes(P, four_ellipses_32768):
    import torch
    g, f, ph = four_ellipses_32768
    om = W.smooth_density(g, seed=3)
    tg = np.sort(np.random.default_rng(8).choice(g.M[0], 64, replace=False))
    ref = O.normal_velocity(g, f, om, targets=tg)
    prob = P.Problem(g, f, ph)
    try:
        prob.assemble("fp32_ir")     # U through the stored surface U-matrix
        U = torch.empty(g.M[0], dtype=torch.float64, device="cuda")
        P.bie_normal_velocity(prob.ctx, torch.as_tensor(om, device="cuda"), U)
        got = U.cpu().numpy()[tg]
        assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()
    finally:
        prob.close()


def test_32768_targets_far_sample(P, four_ellipses_32768):
    import torch
    g, f, ph = four_ellipses_32768
    om = W.smooth_density(g, seed=4)
    zg, zn = W.targets_32768(g)
    z = np.concatenate([zg, zn])
    prob = P.Problem(g, f, ph)
    try:
        uv = torch.empty(len(z), dtype=torch.complex128, device="cuda")
        nn = P.bie_eval_velocity(prob.ctx, torch.as_tensor(om, device="cuda"), _ct(z), uv,
                                 mode=P.VEL_AUTO, near_spacings=2.0, count_near=True)
        assert nn >= len(zn)           # every near-boundary target went to Helsing
        got = uv.cpu().numpy()
        assert np.all(np.isfinite(got))
        # grid targets at least 6 node spacings from every boundary: FP32 sums
        rng = np.random.default_rng(9)
        cand = rng.choice(len(zg), 3000, replace=False)
        h = np.abs(g.dzeta) * 2 * np.pi / np.asarray(g.M, float)[O.block_ids(g.M)]
        dn = np.array([(np.abs(zg[i] - g.zeta) / h).min() for i in cand])
        far = cand[dn > 6.0][:200]
        ref = O.velocity_far(g, f, om, zg[far])
        assert np.abs(got[far] - ref).max() <= 2e-5 * np.abs(ref).max()
    finally:
        prob.close()


def test_helsing_exact_field_max_size(P):
    import torch
    h = 1.3
    c = {1: 0.3, 2: -0.1, 3: 0.05}
    Phit = lambda z: sum(ck * np.cos(k * (z + 1j * h)) for k, ck in c.items())
    dPhit = lambda z: sum(-ck * k * np.sin(k * (z + 1j * h)) for k, ck in c.items())
    f = W.Flow(V1=0.7, a=np.array([]))
    g = W.simple_channel(M0=16384, M1=16384, h=h)
    z0 = g.zeta[: g.M[0]]
    prob = P.Problem(g, f, np.real(Phit(z0)))
    try:
        prob.assemble("fp32_ir")
        info = prob.solve()
        assert info.converged
        # Phi' on the boundary carries the FP64 floor of the method itself: the
        # oracle, on this same channel, misses the exact U by 3.2e-12 (M=1024),
        # 1.3e-11 (2048), 5.9e-11 (4096), i.e. ~3.5e-18 M^2 (kernel values of
        # size ~M, then a spectral derivative).  Bound: 4x that floor at M_0.
        floor = 3.5e-18 * g.M[0] ** 2
        fb = torch.empty(g.N, dtype=torch.complex128, device="cuda")
        P.bie_boundary_velocity(prob.ctx, prob.omega, fb)
        ex_b = dPhit(g.zeta) + f.V1
        assert np.abs(fb.cpu().numpy() - ex_b).max() <= 4 * floor
        zn = W.near_boundary_targets(g, 5000, seed=2, max_spacings=2.0)
        zi = W.fluid_grid(g, 120, 40, margin=0.05)
        z = np.concatenate([zn, zi])
        exact = dPhit(z) + f.V1
        uv = torch.empty(len(z), dtype=torch.complex128, device="cuda")
        P.bie_eval_velocity(prob.ctx, prob.omega, _ct(z), uv, mode=P.VEL_AUTO, near_spacings=4.0)
        got = uv.cpu().numpy()
        scale = np.abs(exact).max()
        assert np.abs(got[: len(zn)] - exact[: len(zn)]).max() <= 4 * floor
        assert np.abs(got[len(zn):] - exact[len(zn):]).max() <= 2e-5 * scale
    finally:
        prob.close()


@pytest.mark.parametrize("prec", ["fp16_ir", "bf16_ir", "fp32_ir"])
def test_16383_updated_residual_is_the_true_one(P, prec):
    """The last refinement residuals are updated from the last increment with
    the FP32 part or the inner storage of A (when the storage's rounding times
    the residual stays below 6e-15 ||b||); the residual the solve reports must
    still be that of omega: against the hi + lo product of the final omega
    (relative 2-norm, Sec. 7.1's tolerance) and against rows of the oracle's
    own FP64 matrix (max norm)."""
    import torch
    g, f, ph = W.three_ellipses_16383(seed=0)
    prob = P.Problem(g, f, ph)
    try:
        prob.assemble(prec)
        info = prob.solve(rtol=1e-14)
        assert info.converged and info.rel_resid <= 1e-14
        b = torch.empty(g.N, dtype=torch.float64, device="cuda")
        P.bie_rhs(prob.ctx, prob.phit, b)
        y = torch.empty_like(b)
        P.bie_matvec(prob.ctx, 1, prob.omega, y)
        true = ((b - y).norm() / b.norm()).item()
        assert true <= 1.2e-14, true
        assert abs(true - info.rel_resid) <= 2e-16, (true, info.rel_resid)
        rows = np.unique(np.concatenate([np.random.default_rng(3).choice(g.N, 32, replace=False),
                                         g.offsets()[:-1], g.offsets()[1:] - 1]))
        bo = O.rhs(g, f, ph)
        r = bo[rows] - O.kernel_rows(g, rows) @ prob.omega.cpu().numpy()
        assert np.abs(r).max() <= 1e-13 * np.abs(bo).max()
    finally:
        prob.close()


@pytest.mark.parametrize("prec", ["fp16_ir", "fp32_ir"])
def test_16383_initial_guess_residual_is_the_true_one(P, prec):
    """A solve from a perturbed solution (x0, as the evolution drivers start
    every stage): its first residuals come from the FP32 part alone while they
    are above 1e-4 ||b||, and no later residual may be updated from one of
    those; the reported residual must be that of the final omega."""
    import torch
    g, f, ph = W.three_ellipses_16383(seed=1)
    prob = P.Problem(g, f, ph)
    try:
        prob.assemble(prec)
        assert prob.solve(rtol=1e-14).converged
        om = prob.omega.clone()
        b = torch.empty(g.N, dtype=torch.float64, device="cuda")
        P.bie_rhs(prob.ctx, prob.phit, b)
        y = torch.empty_like(b)
        rng = np.random.default_rng(11)
        for scale in (3e-3, 1e-3, 3e-4, 1e-4):
            noise = torch.as_tensor(rng.standard_normal(g.N), device="cuda")
            prob.omega.copy_(om * (1.0 + scale * noise))
            info = prob.solve(rtol=1e-14, x0=1)
            assert info.converged and info.rel_resid <= 1e-14, (scale, info.rel_resid)
            P.bie_matvec(prob.ctx, 1, prob.omega, y)
            true = ((b - y).norm() / b.norm()).item()
            assert true <= 1.2e-14 and abs(true - info.rel_resid) <= 2e-16, (scale, true,
                                                                              info.rel_resid)
    finally:
        prob.close()
