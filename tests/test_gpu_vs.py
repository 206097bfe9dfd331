"""Vortex-sheet route (bie_vs_normal_velocity, Sec. 4) vs the oracle.

The oracle's vortex-sheet path (dense solve of eq. lin:sys2, U from eq.
U:from:gam:j) is pinned on the CPU against the velocity-potential path; here
the GPU's vortex-sheet U must match it (relative 2-norm 1e-11, the bound of
the single-problem U parity), and, with gamma_0 = -omega_0' of a GPU
velocity-potential solve, reproduce that solve's U and omega_j'.
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


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _cases():
    return {"one_ellipse_640": W.one_ellipse_640(), "ragged": W.random_geometry(np.random.default_rng(3), 1001),
            "problem3": W.paper_problem(3)}


@pytest.mark.parametrize("prec", ["fp64", "fp32_ir"])
@pytest.mark.parametrize("case", ["one_ellipse_640", "ragged", "problem3"])
def test_vs_matches_oracle(P, prec, case):
    import torch
    g, f, ph = _cases()[case]
    gamma0 = W.filtered_noise(np.random.default_rng(21), g.M[0], 0.5, 24)
    ref = O.vs_normal_velocity(g, f, gamma0)
    prob = P.Problem(g, f, ph)
    try:
        U = torch.empty(g.M[0], dtype=torch.float64, device="cuda")
        info = P.bie_vs_normal_velocity(prob.ctx, torch.as_tensor(gamma0, device="cuda"), U,
                                        precision=prec)
        assert info.converged
        assert _rel(U.cpu().numpy(), ref) <= 1e-11
    finally:
        prob.close()


def test_vs_reproduces_velocity_potential_solve(P):
    import torch
    g, f, ph = W.random_geometry(np.random.default_rng(5), 1500)
    prob = P.Problem(g, f, ph)
    try:
        prob.assemble("fp32_ir")
        assert prob.solve().converged
        om = prob.omega.cpu().numpy()
        w = O.split(om, g.M)
        gamma0 = -O.d_alpha(w[0])
        U = torch.empty(g.M[0], dtype=torch.float64, device="cuda")
        gs = torch.empty(g.N - g.M[0], dtype=torch.float64, device="cuda")
        P.bie_vs_normal_velocity(prob.ctx, torch.as_tensor(gamma0, device="cuda"), U, gs)
        assert _rel(U.cpu().numpy(), prob.U.cpu().numpy()) <= 1e-11
        wp = np.concatenate([O.d_alpha(x) for x in w[1:]])
        assert _rel(gs.cpu().numpy(), wp) <= 1e-10
        # the velocity-potential storage is untouched: the next solve still works
        assert prob.solve().converged
    finally:
        prob.close()


def test_vs_channel_without_obstacles(P):
    import torch
    g = W.simple_channel(M0=300, M1=200, h=1.1)
    f = W.Flow(V1=0.6, a=np.array([]))
    gamma0 = W.filtered_noise(np.random.default_rng(8), 300, 0.5, 20)
    ref = O.vs_normal_velocity(g, f, gamma0)
    prob = P.Problem(g, f, np.zeros(300))
    try:
        U = torch.empty(300, dtype=torch.float64, device="cuda")
        P.bie_vs_normal_velocity(prob.ctx, torch.as_tensor(gamma0, device="cuda"), U)
        assert _rel(U.cpu().numpy(), ref) <= 1e-11
    finally:
        prob.close()
