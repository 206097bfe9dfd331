"""Auxiliary Dirichlet problem for Phi_t - C (Sec. 4, eq. pressure:d:prob) on
the GPU vs the oracle: the right-hand side b^aux from a solved state, and its
solve on the same matrix (single bie_solve_b, and several states at once with
bie_solve_multi on raw right-hand sides).

b^aux_0 is an O(M_0) FP64 formula of the state's geometry, phi~ and U, so it
agrees with the oracle's to the accuracy of U (relative 1e-11 in the solve
tests); omega^aux then carries the solve's own 1e-11 parity bound.
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
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


CASES = [("one_ellipse_640", lambda: W.one_ellipse_640()),
         ("ragged1001", lambda: W.random_geometry(np.random.default_rng(5), 1001)),
         ("paper3", lambda: W.paper_problem(3))]


@pytest.mark.parametrize("name,make", CASES)
def test_pressure_rhs_matches_oracle(P, name, make):
    import torch
    g, f, ph = make()
    tau, grav = 0.07, 9.81
    om_ref, U_ref, _ = O.solve(g, f, ph)
    b_ref = O.pressure_rhs(g, f, ph, U_ref, tau=tau, g=grav)
    prob = P.Problem(g, f, ph)
    try:
        prob.assemble("fp32_ir")
        prob.solve()
        b = torch.full((g.N,), np.nan, dtype=torch.float64, device="cuda")
        P.bie_pressure_rhs(prob.ctx, prob.phit, prob.U, b, tau=tau, g=grav)
        bh = b.cpu().numpy()
        assert np.all(bh[g.M[0]:] == 0.0)
        assert np.abs(bh - b_ref).max() <= 1e-10 * np.abs(b_ref).max(), name
        # the same data with the oracle's own U: only the O(M_0) formula differs
        Ud = torch.as_tensor(U_ref, device="cuda")
        P.bie_pressure_rhs(prob.ctx, prob.phit, Ud, b, tau=tau, g=grav)
        assert np.abs(b.cpu().numpy() - b_ref).max() <= 1e-13 * np.abs(b_ref).max(), name
    finally:
        prob.close()


def test_aux_solve_single(P):
    import torch
    g, f, ph = W.one_ellipse_640()
    om_ref, U_ref, b_ref, omx_ref = O.solve_aux(g, f, ph, tau=0.07, g=9.81)
    prob = P.Problem(g, f, ph)
    try:
        prob.assemble("fp32_ir")
        prob.solve()
        b = torch.empty(g.N, dtype=torch.float64, device="cuda")
        P.bie_pressure_rhs(prob.ctx, prob.phit, prob.U, b, tau=0.07, g=9.81)
        omx = torch.empty(g.N, dtype=torch.float64, device="cuda")
        info = P.bie_solve_b(prob.ctx, b, omx)
        assert info.converged and info.rel_resid <= 1e-14
        assert _rel(omx.cpu().numpy(), omx_ref) <= 1e-10
        # bie_solve_b with the eq. Awb right-hand side reproduces bie_solve
        om2 = torch.empty(g.N, dtype=torch.float64, device="cuda")
        P.bie_solve_b(prob.ctx, torch.as_tensor(O.rhs(g, f, ph), device="cuda"), om2)
        assert _rel(om2.cpu().numpy(), prob.omega.cpu().numpy()) <= 1e-12
    finally:
        prob.close()


@pytest.mark.parametrize("prec", ["fp16_ir", "bf16_ir"])
def test_aux_solve_several_states(P, prec):
    """Six states on one geometry: their omega and U in one bie_solve_multi,
    then the six auxiliary systems in a second one on raw right-hand sides."""
    import torch
    g, f, ph0 = W.random_geometry(np.random.default_rng(8), 1001)
    rng = np.random.default_rng(1)
    PH = np.stack([W.filtered_noise(rng, g.M[0], 0.05 * (k + 1), 8 + 4 * k) for k in range(6)])
    prob = P.Problem(g, f, ph0)
    try:
        prob.assemble(prec)
        phd = torch.as_tensor(PH, device="cuda").contiguous()
        om = torch.empty((6, g.N), dtype=torch.float64, device="cuda")
        U = torch.empty((6, g.M[0]), dtype=torch.float64, device="cuda")
        infos = P.bie_solve_multi(prob.ctx, phd, om, U)
        assert all(i.converged for i in infos)
        B = torch.empty((6, g.N), dtype=torch.float64, device="cuda")
        for r in range(6):
            P.bie_pressure_rhs(prob.ctx, phd[r], U[r], B[r], tau=0.05, g=1.0)
        omx = torch.empty((6, g.N), dtype=torch.float64, device="cuda")
        infos = P.bie_solve_multi(prob.ctx, B, omx, None, kind="b")
        assert all(i.converged and i.rel_resid <= 1e-14 for i in infos)
        A = O.assemble(g)
        for r in range(6):
            _, U_ref, b_ref, omx_ref = O.solve_aux(g, f, PH[r], tau=0.05, g=1.0)
            assert _rel(U[r].cpu().numpy(), U_ref) <= 1e-11
            assert _rel(B[r].cpu().numpy(), b_ref) <= 1e-10
            assert _rel(omx[r].cpu().numpy(), omx_ref) <= 1e-10, r
            # and omega^aux solves the system for the GPU's own b^aux to the solve's bound
            x = np.linalg.solve(A, B[r].cpu().numpy())
            assert _rel(omx[r].cpu().numpy(), x) <= 1e-11, r
    finally:
        prob.close()


def test_pressure_rhs_errors(P):
    import torch
    g, f, ph = W.one_ellipse_640()
    ctx = P.bie_create(0, torch.cuda.current_stream())
    try:
        x = torch.zeros(g.M[0], dtype=torch.float64, device="cuda")
        b = torch.zeros(g.N, dtype=torch.float64, device="cuda")
        with pytest.raises(P.BieError) as e:
            P.bie_pressure_rhs(ctx, x, x, b)
        assert e.value.status == P.BIE_ERR_STATE
        with pytest.raises(P.BieError) as e:
            P.bie_solve_b(ctx, b, b)
        assert e.value.status == P.BIE_ERR_STATE
    finally:
        P.bie_destroy(ctx)


@pytest.mark.parametrize("name,make,prec", [
    ("one_ellipse_640", lambda: W.one_ellipse_640(), "fp32_ir"),
    ("one_ellipse_640", lambda: W.one_ellipse_640(), "fp64"),
    ("ragged1001", lambda: W.random_geometry(np.random.default_rng(5), 1001), "fp16_ir"),
    ("paper3", lambda: W.paper_problem(3), "fp32_ir")])
def test_boundary_potential_matches_oracle(P, name, make, prec):
    """Phi~ of eq. w123 on every boundary from the fluid side (Plemelj, Sec. 4)
    for the oracle's omega: real and imaginary parts on the surface (phi~ and
    the energy's psi) and on the solid boundaries (the new real part and the
    operator's imaginary part)."""
    import torch
    g, f, ph = make()
    om_ref = O.solve(g, f, ph)[0]
    ref = np.concatenate(O.phi_tilde_boundary(g, om_ref))
    prob = P.Problem(g, f, ph)
    try:
        prob.assemble(prec)
        out = torch.full((g.N,), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
        P.bie_boundary_potential(prob.ctx, torch.as_tensor(om_ref, device="cuda"), out)
        got = out.cpu().numpy()
        scale = np.abs(ref).max()
        M0 = g.M[0]
        assert np.abs(got.real[M0:] - ref.real[M0:]).max() <= 1e-12 * scale, name   # new part
        assert np.abs(got - ref).max() <= 1e-11 * scale, name
    finally:
        prob.close()


def test_pressure_on_the_solids_matches_oracle(P):
    """Phi_t - C on the bottom and the obstacle, end to end: state solve, b^aux,
    auxiliary solve, Plemelj evaluation (the real part of Phi~ for omega^aux)."""
    import torch
    g, f, ph = W.one_ellipse_640()
    om_ref, U_ref, b_ref, omx_ref = O.solve_aux(g, f, ph, tau=0.07, g=9.81)
    ref = np.concatenate(O.phi_tilde_boundary(g, omx_ref)[1:]).real
    prob = P.Problem(g, f, ph)
    try:
        prob.assemble("fp32_ir")
        prob.solve()
        b = torch.empty(g.N, dtype=torch.float64, device="cuda")
        P.bie_pressure_rhs(prob.ctx, prob.phit, prob.U, b, tau=0.07, g=9.81)
        omx = torch.empty(g.N, dtype=torch.float64, device="cuda")
        P.bie_solve_b(prob.ctx, b, omx)
        out = torch.empty(g.N, dtype=torch.complex128, device="cuda")
        P.bie_boundary_potential(prob.ctx, omx, out)
        got = out.cpu().numpy().real[g.M[0]:]
        assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()
        # on the surface the real part is the Dirichlet data itself
        assert np.abs(out.cpu().numpy().real[:g.M[0]] - b_ref[:g.M[0]]).max() <= 1e-10 * np.abs(b_ref).max()
    finally:
        prob.close()


@pytest.mark.parametrize("name,make", [("one_ellipse_640", lambda: W.one_ellipse_640()),
                                       ("paper3", lambda: W.paper_problem(3))])
def test_potential_at_targets_matches_oracle(P, name, make):
    """Phi~(z) inside the fluid: grid points well inside against the plain
    trapezoidal sums of eq. w123 (an independent formula), points within two
    node spacings of a boundary against the oracle's Helsing-Ojala ratio with
    its Plemelj boundary values; a target on a node returns that node's value."""
    import torch
    g, f, ph = make()
    om_ref = O.solve(g, f, ph)[0]
    zg = W.fluid_grid(g, 40, 30, margin=0.25)
    zn = W.near_boundary_targets(g, 300, seed=3, max_spacings=2.0)
    zs = g.zeta[[3, g.M[0] + 5]]   # one node of the surface, one of the bottom
    z = np.concatenate([zg, zn, zs])
    prob = P.Problem(g, f, ph)
    try:
        prob.assemble("fp32_ir")
        out = torch.empty(len(z), dtype=torch.complex128, device="cuda")
        P.bie_eval_potential(prob.ctx, torch.as_tensor(om_ref, device="cuda"),
                             torch.as_tensor(z, device="cuda"), out)
        got = out.cpu().numpy()
        far = O.phi_tilde_at(g, om_ref, zg)
        bnd = O.phi_tilde_boundary(g, om_ref)
        near = O.helsing_eval(g, bnd, zn)
        scale = np.abs(far).max()
        ng, nn = len(zg), len(zn)
        assert np.abs(got[:ng] - far).max() <= 1e-11 * scale, name
        assert np.abs(got[ng:ng + nn] - near).max() <= 1e-10 * scale, name
        allb = np.concatenate(bnd)
        assert np.abs(got[ng + nn:] - allb[[3, g.M[0] + 5]]).max() <= 1e-11 * scale, name
    finally:
        prob.close()


def test_boundary_and_interior_potential_channel_closed_form(P):
    """Phi~ = sum c_k cos(k(z + ih)) over the flat bottom y = -h (psi~ = 0 there):
    the GPU's Plemelj boundary values and its values inside the fluid equal the
    closed form."""
    import torch
    h = 1.3
    c = {1: 0.3, 2: -0.1, 3: 0.05}
    Phit = lambda z: sum(ck * np.cos(k * (z + 1j * h)) for k, ck in c.items())
    g = W.simple_channel(M0=128, M1=128, h=h)
    f = W.Flow(V1=0.0, a=np.array([]))
    z0 = g.block(0)[0]
    prob = P.Problem(g, f, np.real(Phit(z0)))
    try:
        prob.assemble("fp32_ir")
        prob.solve(rtol=1e-13)
        out = torch.empty(g.N, dtype=torch.complex128, device="cuda")
        P.bie_boundary_potential(prob.ctx, prob.omega, out)
        assert np.abs(out.cpu().numpy() - Phit(g.zeta)).max() < 1e-11
        zt = np.concatenate([W.fluid_grid(g, 30, 20, margin=0.1),
                             W.near_boundary_targets(g, 200, seed=1, max_spacings=2.0)])
        pz = torch.empty(len(zt), dtype=torch.complex128, device="cuda")
        P.bie_eval_potential(prob.ctx, prob.omega, torch.as_tensor(zt, device="cuda"), pz)
        assert np.abs(pz.cpu().numpy() - Phit(zt)).max() < 1e-10
    finally:
        prob.close()
