"""Time evolution of the graph formulation on the GPU vs the oracle (Sec. 2,
eqs. graph:eta:t and phitileq; filter of eq. filter; energy of eq. E:formula).

The right-hand side is an FP64 formula of the solved state, so it carries the
solve's parity bound (relative 1e-11 on U) amplified at most by the spectral
derivatives: the test allows 1e-10 of the largest entry.  The energy is an
FP64 trapezoidal sum over FP64 node-pair terms: 1e-12 relative.  After a few
RK4 steps the state differs from the oracle's by the accumulated per-stage
errors: 1e-10 relative.
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


def _eta(M0, amp=0.03):
    a = 2 * np.pi * np.arange(M0) / M0
    return amp * np.cos(a) + 0.3 * amp * np.sin(2 * a) - 0.1 * amp * np.cos(5 * a)


CASES = [("paper1", lambda: W.paper_problem(1)), ("one_ellipse_640", lambda: W.one_ellipse_640()),
         ("ragged1001", lambda: W.random_geometry(np.random.default_rng(2), 1001))]


@pytest.mark.parametrize("name,make", CASES)
def test_graph_rhs_matches_oracle(P, name, make):
    import torch
    g, f, ph = make()
    M0 = g.M[0]
    eta = _eta(M0)
    et_ref, pt_ref, om_ref, gs = O.graph_rhs(g, f, eta, ph, tau=0.1, g=1.0)
    prob = P.Problem(g, f, ph)
    try:
        ed = torch.as_tensor(eta, device="cuda")
        et = torch.empty(M0, dtype=torch.float64, device="cuda")
        pt = torch.empty_like(et)
        om = torch.empty(g.N, dtype=torch.float64, device="cuda")
        P.bie_graph_rhs(prob.ctx, ed, prob.phit, et, pt, tau=0.1, g=1.0, omega=om)
        assert np.abs(et.cpu().numpy() - et_ref).max() <= 1e-10 * np.abs(et_ref).max(), name
        assert np.abs(pt.cpu().numpy() - pt_ref).max() <= 1e-10 * np.abs(pt_ref).max(), name
        assert np.linalg.norm(om.cpu().numpy() - om_ref) <= 1e-11 * np.linalg.norm(om_ref)
    finally:
        prob.close()


@pytest.mark.parametrize("name,make", CASES + [("paper3", lambda: W.paper_problem(3))])
def test_energy_matches_oracle(P, name, make):
    g, f, ph = make()
    om_ref, _, _ = O.solve(g, f, ph)
    E_ref = O.energy(g, f, ph, om_ref, tau=0.1, g=1.0)
    prob = P.Problem(g, f, ph)
    try:
        prob.assemble("fp32_ir")
        prob.solve()
        E = P.bie_energy(prob.ctx, prob.phit, prob.omega, tau=0.1, g=1.0)
        assert abs(E - E_ref) <= 1e-12 * abs(E_ref), (name, E, E_ref)
        # with the oracle's omega the only difference is the FP64 evaluation order
        import torch
        E2 = P.bie_energy(prob.ctx, prob.phit, torch.as_tensor(om_ref, device="cuda"), 0.1, 1.0)
        assert abs(E2 - E_ref) <= 1e-13 * abs(E_ref), name
    finally:
        prob.close()


@pytest.mark.parametrize("M0", [256, 384])
def test_filter_matches_oracle(P, M0):
    import torch
    g = W.simple_channel(M0=M0, M1=96, h=1.0)
    f = W.Flow(V1=0.0, a=np.array([]))
    x = np.random.default_rng(M0).standard_normal(M0)
    prob = P.Problem(g, f, np.zeros(M0))
    try:
        xd = torch.as_tensor(x, device="cuda").contiguous()
        P.bie_filter(prob.ctx, xd)
        ref = O.filter36(x)
        assert np.abs(xd.cpu().numpy() - ref).max() <= 1e-13 * np.abs(x).max()
    finally:
        prob.close()


@pytest.mark.parametrize("filt,prec", [(False, "fp32_ir"), (True, "fp32_ir"), (True, "fp16_ir")])
def test_evolve_matches_oracle(P, filt, prec):
    """Problem 1 of Sec. 7 from rest (eta = 0): 4 RK4 steps of dt = 0.005."""
    import torch
    g, f, ph = W.paper_problem(1)
    M0 = g.M[0]
    eta_ref, ph_ref, E_ref = O.evolve_graph(g, f, np.zeros(M0), ph, 0.005, 4, filt=filt)
    prob = P.Problem(g, f, ph)
    try:
        eta = torch.zeros(M0, dtype=torch.float64, device="cuda")
        phit = prob.phit.clone()
        E, info = P.bie_graph_evolve(prob.ctx, eta, phit, 0.005, 4, tau=0.1, g=1.0, filter=filt,
                                     precision=prec)
        assert info.steps == 4 and info.solves == 17 and info.max_rel_resid <= 1e-14
        assert np.abs(eta.cpu().numpy() - eta_ref).max() <= 1e-10 * np.abs(eta_ref).max()
        assert np.abs(phit.cpu().numpy() - ph_ref).max() <= 1e-10 * np.abs(ph_ref).max()
        assert np.abs(E - E_ref).max() <= 1e-12 * abs(E_ref[0])
        assert np.abs(E - E[0]).max() <= 1e-11 * abs(E[0])
    finally:
        prob.close()


def test_evolve_longer_run_conserves_energy(P):
    """40 steps of dt = 0.0015 (inside the capillary step limit, which scales as
    M_0^(-3/2)) on problem 1 at M_0 = 512 with the filter: E stays within 1e-10
    of its initial value (the oracle is not run at this length)."""
    import torch
    g, f, ph = W.paper_problem(1, M0=512, M1=192, Me=256)
    prob = P.Problem(g, f, ph)
    try:
        eta = torch.zeros(g.M[0], dtype=torch.float64, device="cuda")
        phit = prob.phit.clone()
        E, info = P.bie_graph_evolve(prob.ctx, eta, phit, 0.0015, 40, filter=True)
        assert info.steps == 40
        assert np.abs(E - E[0]).max() <= 1e-10 * abs(E[0])
        assert float(eta.abs().max()) > 1e-4           # the surface did move
    finally:
        prob.close()


def test_evolve_errors(P):
    import torch
    g, f, ph = W.paper_problem(1)
    prob = P.Problem(g, f, ph)
    try:
        eta = torch.zeros(g.M[0], dtype=torch.float64, device="cuda")
        for dt, n in ((0.0, 1), (0.01, -1), (float("nan"), 1)):
            with pytest.raises(P.BieError) as e:
                P.bie_graph_evolve(prob.ctx, eta, prob.phit.clone(), dt, n)
            assert e.value.status == P.BIE_ERR_ARG
        with pytest.raises(P.BieError) as e:   # a surface that is not finite
            bad = eta.clone()
            bad[3] = float("nan")
            P.bie_graph_evolve(prob.ctx, bad, prob.phit.clone(), 0.005, 1, energies=False)
        assert e.value.status == P.BIE_ERR_GEOM
    finally:
        prob.close()


# ---------------------------------------------------------------------------
# HLS formulation with P theta reconstruction
# ---------------------------------------------------------------------------

def _ptheta(M0, amp=0.3):
    a = 2 * np.pi * np.arange(M0) / M0
    return amp * np.cos(a) + 0.6 * amp * np.cos(2 * a) + 0.3 * amp * np.sin(3 * a)


def test_hls_curve_matches_oracle(P):
    import torch
    g, f, ph = W.paper_problem(1)
    M0 = g.M[0]
    Pth = _ptheta(M0, 0.1)
    z_ref, dz_ref, d2z_ref, _, _ = O.hls_curve(Pth)
    prob = P.Problem(g, f, ph)
    try:
        z = torch.empty(M0, dtype=torch.complex128, device="cuda")
        dz, d2z = torch.empty_like(z), torch.empty_like(z)
        P.bie_hls_curve(prob.ctx, torch.as_tensor(Pth, device="cuda"), z, dz, d2z)
        assert np.abs(z.cpu().numpy() - z_ref).max() <= 1e-13
        assert np.abs(dz.cpu().numpy() - dz_ref).max() <= 1e-14
        assert np.abs(d2z.cpu().numpy() - d2z_ref).max() <= 1e-12
    finally:
        prob.close()


@pytest.mark.parametrize("name,make", CASES[:2])
def test_hls_rhs_matches_oracle(P, name, make):
    import torch
    g, f, ph = make()
    M0 = g.M[0]
    Pth = _ptheta(M0, 0.05)
    tt_ref, pt_ref, om_ref, _ = O.hls_rhs(g, f, Pth, ph, tau=0.1, g=1.0)
    prob = P.Problem(g, f, ph)
    try:
        tt = torch.empty(M0, dtype=torch.float64, device="cuda")
        pt = torch.empty_like(tt)
        om = torch.empty(g.N, dtype=torch.float64, device="cuda")
        P.bie_hls_rhs(prob.ctx, torch.as_tensor(Pth, device="cuda"), prob.phit, tt, pt, omega=om)
        assert np.abs(tt.cpu().numpy() - tt_ref).max() <= 1e-10 * np.abs(tt_ref).max(), name
        assert np.abs(pt.cpu().numpy() - pt_ref).max() <= 1e-10 * np.abs(pt_ref).max(), name
        assert np.linalg.norm(om.cpu().numpy() - om_ref) <= 1e-11 * np.linalg.norm(om_ref)
    finally:
        prob.close()


@pytest.mark.parametrize("filt", [False, True])
def test_hls_evolve_matches_oracle(P, filt):
    """Problem 1 from rest (P theta = 0): 4 RK4 steps of dt = 0.005."""
    import torch
    g, f, ph = W.paper_problem(1)
    M0 = g.M[0]
    th_ref, ph_ref, E_ref = O.evolve_hls(g, f, np.zeros(M0), ph, 0.005, 4, filt=filt)
    prob = P.Problem(g, f, ph)
    try:
        th = torch.zeros(M0, dtype=torch.float64, device="cuda")
        phit = prob.phit.clone()
        E, info = P.bie_hls_evolve(prob.ctx, th, phit, 0.005, 4, filter=filt)
        assert info.steps == 4 and info.solves == 17
        assert np.abs(th.cpu().numpy() - th_ref).max() <= 1e-10 * np.abs(th_ref).max()
        assert np.abs(phit.cpu().numpy() - ph_ref).max() <= 1e-10 * np.abs(ph_ref).max()
        assert np.abs(E - E_ref).max() <= 1e-12 * abs(E_ref[0])
    finally:
        prob.close()


@pytest.mark.parametrize("form", ["graph", "hls"])
def test_gbs8_evolve_matches_oracle(P, form):
    """Problem 1 from rest: two eighth-order GBS steps of dt = 0.01 (17
    right-hand sides each) in either formulation, with the filter."""
    import torch
    g, f, ph = W.paper_problem(1)
    M0 = g.M[0]
    y_ref, ph_ref, E_ref = O.evolve_gbs8(g, f, np.zeros(M0), ph, 0.01, 2, filt=True,
                                         formulation=form)
    prob = P.Problem(g, f, ph)
    try:
        y = torch.zeros(M0, dtype=torch.float64, device="cuda")
        phit = prob.phit.clone()
        E, info = P.bie_evolve(prob.ctx, y, phit, 0.01, 2, formulation=form, integrator="gbs8",
                               filter=True)
        assert info.steps == 2 and info.solves == 2 * 17 + 1
        assert np.abs(y.cpu().numpy() - y_ref).max() <= 1e-10 * np.abs(y_ref).max()
        assert np.abs(phit.cpu().numpy() - ph_ref).max() <= 1e-10 * np.abs(ph_ref).max()
        assert np.abs(E - E_ref).max() <= 1e-12 * abs(E_ref[0])
    finally:
        prob.close()


@pytest.mark.parametrize("form", ["graph", "hls"])
def test_dp8_evolve_matches_oracle(P, form):
    """Problem 1 from rest: two steps of dt = 0.01 of the paper's
    eighth-order Dormand-Prince scheme (12 right-hand sides each) in either
    formulation, with the filter, against the oracle's."""
    import torch
    g, f, ph = W.paper_problem(1)
    M0 = g.M[0]
    y_ref, ph_ref, E_ref = O.evolve_dp8(g, f, np.zeros(M0), ph, 0.01, 2, filt=True,
                                        formulation=form)
    prob = P.Problem(g, f, ph)
    try:
        y = torch.zeros(M0, dtype=torch.float64, device="cuda")
        phit = prob.phit.clone()
        E, info = P.bie_evolve(prob.ctx, y, phit, 0.01, 2, formulation=form, integrator="dp8",
                               filter=True)
        assert info.steps == 2 and info.solves == 2 * 12 + 1
        assert np.abs(y.cpu().numpy() - y_ref).max() <= 1e-10 * np.abs(y_ref).max()
        assert np.abs(phit.cpu().numpy() - ph_ref).max() <= 1e-10 * np.abs(ph_ref).max()
        assert np.abs(E - E_ref).max() <= 1e-12 * abs(E_ref[0])
    finally:
        prob.close()


def test_dp8_evolve_with_obstacle_circulation_matches_oracle(P):
    """The 640-unknown geometry (ellipse with circulation, curved surface and
    flat bottom): two DP8 steps of dt = 0.005, FP32-IR, against the oracle."""
    import torch
    g, f, ph = W.one_ellipse_640()
    M0 = g.M[0]
    eta0 = g.zeta[:M0].imag.copy()
    y_ref, ph_ref, E_ref = O.evolve_dp8(g, f, eta0, ph, 0.005, 2)
    prob = P.Problem(g, f, ph)
    try:
        y = torch.as_tensor(eta0, device="cuda").clone()
        phit = prob.phit.clone()
        E, info = P.bie_evolve(prob.ctx, y, phit, 0.005, 2, integrator="dp8", precision="fp32_ir")
        assert info.steps == 2
        assert np.abs(y.cpu().numpy() - y_ref).max() <= 1e-10 * np.abs(y_ref).max()
        assert np.abs(phit.cpu().numpy() - ph_ref).max() <= 1e-10 * np.abs(ph_ref).max()
        assert np.abs(E - E_ref).max() <= 1e-12 * abs(E_ref[0])
    finally:
        prob.close()


def test_dp8_vs_evolution_matches_oracle(P):
    """Vortex-sheet formulation (eta, gamma_0) under DP8: two steps of dt =
    0.005 from problem 1 at rest (24 stages, two solves each)."""
    import torch
    g, f, ph = W.paper_problem(1)
    M0 = g.M[0]
    om, _, _ = O.solve(g, f, ph)
    gam0 = -O.d_alpha(om[:M0])
    e_ref, gm_ref = O.evolve_vs_graph(g, f, np.zeros(M0), gam0, 0.005, 2, step=O.dp8_step)
    prob = P.Problem(g, f, ph)
    try:
        eta = torch.zeros(M0, dtype=torch.float64, device="cuda")
        gm = torch.as_tensor(gam0, device="cuda").clone()
        _, info = P.bie_evolve(prob.ctx, eta, gm, 0.005, 2, formulation="vs_graph",
                               integrator="dp8", energies=False)
        assert info.steps == 2 and info.solves == 2 * 12 * 2
        assert np.abs(eta.cpu().numpy() - e_ref).max() <= 1e-10 * np.abs(e_ref).max()
        assert np.abs(gm.cpu().numpy() - gm_ref).max() <= 1e-9 * np.abs(gm_ref).max()
    finally:
        prob.close()


def test_evolve_entry_errors(P):
    import torch
    g, f, ph = W.paper_problem(1)
    prob = P.Problem(g, f, ph)
    try:
        y = torch.zeros(g.M[0], dtype=torch.float64, device="cuda")
        with pytest.raises(KeyError):
            P.bie_evolve(prob.ctx, y, prob.phit.clone(), 0.01, 1, integrator="dp5")
        import ctypes
        st = P.lib().bie_evolve(prob.ctx, 0, 7, P._dptr(y), P._dptr(prob.phit.clone()), 0.01, 1,
                                0.1, 1.0, 0, P.BIE_FP32_IR, ctypes.byref(P.bie_default_opts()),
                                None, None)
        assert st == P.BIE_ERR_ARG
    finally:
        prob.close()


# ---------------------------------------------------------------------------
# vortex-sheet formulation: gamma_0,t
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name,make", CASES)
def test_vs_graph_rhs_matches_oracle(P, name, make):
    """(eta_t, gamma_0,t) of eqs. gam:t:final / gam:t:aux against the oracle;
    gamma_0 is -omega_0' of the state's velocity-potential solve."""
    import torch
    g, f, ph = make()
    M0 = g.M[0]
    eta = _eta(M0)
    gs = O.surface_replaced(g, eta)
    om, _, _ = O.solve(gs, f, ph)
    gam0 = -O.d_alpha(om[:M0])
    et_ref, gt_ref, U_ref, _ = O.vs_graph_rhs(g, f, eta, gam0, tau=0.1, g=1.0)
    prob = P.Problem(g, f, ph)
    try:
        et = torch.empty(M0, dtype=torch.float64, device="cuda")
        gt, U = torch.empty_like(et), torch.empty_like(et)
        P.bie_vs_graph_rhs(prob.ctx, torch.as_tensor(eta, device="cuda"),
                           torch.as_tensor(gam0, device="cuda"), et, gt, U=U)
        assert np.abs(U.cpu().numpy() - U_ref).max() <= 1e-10 * np.abs(U_ref).max(), name
        assert np.abs(et.cpu().numpy() - et_ref).max() <= 1e-10 * np.abs(et_ref).max(), name
        assert np.abs(gt.cpu().numpy() - gt_ref).max() <= 1e-9 * np.abs(gt_ref).max(), name
    finally:
        prob.close()


def test_vs_evolution_matches_oracle_and_the_vp_evolution(P):
    """Problem 1 from rest, 3 RK4 steps of dt = 0.005 in the vortex-sheet
    formulation: equal to the oracle's, and the surface equals the GPU's
    velocity-potential evolution to the two systems' truncation difference."""
    import torch
    g, f, ph = W.paper_problem(1)
    M0 = g.M[0]
    om, _, _ = O.solve(g, f, ph)
    gam0 = -O.d_alpha(om[:M0])
    e_ref, gm_ref = O.evolve_vs_graph(g, f, np.zeros(M0), gam0, 0.005, 3)
    prob = P.Problem(g, f, ph)
    try:
        eta = torch.zeros(M0, dtype=torch.float64, device="cuda")
        gm = torch.as_tensor(gam0, device="cuda").clone()
        _, info = P.bie_evolve(prob.ctx, eta, gm, 0.005, 3, formulation="vs_graph", energies=False)
        assert info.steps == 3 and info.solves == 2 * 12
        assert np.abs(eta.cpu().numpy() - e_ref).max() <= 1e-10 * np.abs(e_ref).max()
        assert np.abs(gm.cpu().numpy() - gm_ref).max() <= 1e-9 * np.abs(gm_ref).max()
        eta2 = torch.zeros(M0, dtype=torch.float64, device="cuda")
        phit = prob.phit.clone()
        P.bie_evolve(prob.ctx, eta2, phit, 0.005, 3, formulation="graph", energies=False)
        assert np.abs(eta.cpu().numpy() - eta2.cpu().numpy()).max() <= 1e-8 * np.abs(e_ref).max()
        with pytest.raises(P.BieError) as e:      # no energy monitor for gamma_0 states
            P.bie_evolve(prob.ctx, eta, gm, 0.005, 1, formulation="vs_graph")
        assert e.value.status == P.BIE_ERR_ARG
    finally:
        prob.close()


@pytest.mark.parametrize("prec", ["fp16_ir", "fp64"])
def test_stage_assembly_keeps_solid_pairs(P, prec):
    """A stage moves only the free surface, so its assembly recomputes the tile
    pairs that touch the surface and keeps the solid-solid entries of the
    previous assembly of the same storage.  Every stored entry (inner storage
    and full-accuracy storage) equals that of a context assembling the same
    stage geometry in full, bit for bit; and after bie_set_geometry (solids
    possibly moved) the next assembly is in full again."""
    import torch
    g, f, ph = W.random_geometry(np.random.default_rng(2), 1001)   # ragged tiles
    M0, N = g.M[0], g.N
    ed = torch.as_tensor(_eta(M0), device="cuda")
    rows = torch.arange(N, device="cuda").repeat_interleave(N)
    cols = torch.arange(N, device="cuda").repeat(N)
    outs = []
    for warm in (True, False):
        prob = P.Problem(g, f, ph)
        try:
            if warm:   # an assembly of the initial geometry is already stored
                prob.assemble(prec)
            et = torch.empty(M0, dtype=torch.float64, device="cuda")
            pt = torch.empty_like(et)
            P.bie_graph_rhs(prob.ctx, ed, prob.phit, et, pt, precision=prec)
            ent = []
            for which in ((0, 1) if prec != "fp64" else (0,)):
                o = torch.empty(N * N, dtype=torch.float64, device="cuda")
                P.bie_sample_entries(prob.ctx, which, rows, cols, o)
                ent.append(o.cpu().numpy())
            outs.append((ent, et.cpu().numpy(), pt.cpu().numpy()))
            if warm:   # new solids: a full assembly again, equal to a fresh context's
                g2, f2, ph2 = W.random_geometry(np.random.default_rng(3), 1001)
                zt = lambda a: torch.as_tensor(a, dtype=torch.complex128, device="cuda")
                P.bie_set_geometry(prob.ctx, g2.M, zt(g2.zeta), zt(g2.dzeta), zt(g2.d2zeta), g2.zc)
                prob.assemble(prec)
                o = torch.empty(N * N, dtype=torch.float64, device="cuda")
                P.bie_sample_entries(prob.ctx, 1 if prec != "fp64" else 0, rows, cols, o)
                A2 = O.assemble(g2)   # full-accuracy storage against the oracle
                assert np.abs(o.cpu().numpy().reshape(N, N) - A2).max() <= 1e-13
        finally:
            prob.close()
    (e1, et1, pt1), (e2, et2, pt2) = outs
    for a, b in zip(e1, e2):
        assert np.array_equal(a, b)
    assert np.array_equal(et1, et2) and np.array_equal(pt1, pt2)
