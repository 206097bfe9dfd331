"""Pins of the FP64 oracle against values the paper prints and closed forms.

Each test ties the oracle to something other than itself:
  * printed worked values (E(0) of problems 1-3; the problem-4 basin depth),
  * closed forms from the theory (constant-density potentials eq. Phij:w:const,
    the residue identity eq. res:thm, exact uniform flow, an exact DtN pair),
  * invariants (zero net flux, phi_n = 0 on solids, VP == VS at equal grids),
  * and mutation checks: a plausible mistake planted in the oracle (CPU only)
    must break at least one pin.
"""
import os

import numpy as np
import pytest

import workloads as W
from oracle import bie as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([float(t) for t in line.split()])
    return np.array(rows)


def _blocks(A, M):
    o = O.offsets(M)
    return lambda k, j: A[o[k]:o[k + 1], o[j]:o[j + 1]]


# ---------------------------------------------------------------- printed values

def test_energy_t0_matches_paper_table():
    """E(0) of problems 1-3 (Sec. 7.3) to the 5 printed decimals."""
    ref = _load_golden("energy_t0_problems_1_3.txt")
    for p, e_ref in ref:
        g, f, ph = W.paper_problem(int(p))
        om, U, ps = O.solve(g, f, ph)
        E = O.energy(g, f, ph, om)
        assert abs(E - e_ref) <= 5e-6, (p, E, e_ref)


def test_problem4_basin_depth():
    """eta_1(pi) = -2.072774 (Sec. 7.2)."""
    a, eta = _load_golden("problem4_bottom.txt")[0]
    assert abs(W.problem4_bottom_eta(np.array([a]))[0] - eta) <= 5e-7


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("which", ["one_ellipse_640", "problem1"])
def test_constant_density_row_sums(which):
    """eq. Phij:w:const: B 1_m = 0 for m >= 2 and the block row sums of Sec. 6.1:
    K_00 1 = 0, G_k0 1 = 0; G_01 1 = 0, K_11 1 = 0, K_k1 1 = 1/2 (k >= 2);
    K_mm 1 = -1/2, K_km 1 = 0 (k != m), G_0m 1 = 0 (m >= 2)."""
    g = W.one_ellipse_640()[0] if which == "one_ellipse_640" else W.paper_problem(1)[0]
    A = O.assemble(g)
    blk = _blocks(A, g.M)
    nb = g.nb
    for k in range(nb):
        for j in range(nb):
            B = blk(k, j).copy()
            if k == j:
                B -= np.diag(np.full(g.M[k], -0.5 if k == 0 else 0.5))
                if k >= 2:
                    B += 1.0 / g.M[k]
            s = B.sum(axis=1)
            if j >= 2 and k == j:
                expect = -0.5
            elif j == 1 and k >= 2:
                expect = 0.5
            else:
                expect = 0.0
            assert np.abs(s - expect).max() < 1e-12, (k, j, s.min(), s.max())
    # hence A 1_m = -1_m for obstacles (the finite-rank correction, eq. AB:cor)
    o = O.offsets(g.M)
    for m in range(2, nb):
        one = np.zeros(g.N)
        one[o[m]:o[m + 1]] = 1.0
        assert np.abs(A @ one + one).max() < 1e-12


@pytest.mark.parametrize("which", ["one_ellipse_640", "problem1"])
def test_obstacle_right_preconditioner_spectrum(which):
    """The refined solvers' inner GMRES runs on A P, P = I - 3/2 sum_k 1_k 1_k^T / M_k
    over the obstacles k >= 2.  With A 1_k = -1_k (eq. AB:cor, pinned above), A P
    has 1_k as eigenvector with eigenvalue 1/2 in place of -1, and every
    eigenvalue of D A P (surface rows negated) has positive real part; D A itself
    has nb - 2 eigenvalues at -1."""
    g = W.one_ellipse_640()[0] if which == "one_ellipse_640" else W.paper_problem(1)[0]
    A = O.assemble(g)
    o = O.offsets(g.M)
    P = np.eye(g.N)
    for m in range(2, g.nb):
        one = np.zeros(g.N)
        one[o[m]:o[m + 1]] = 1.0
        P -= 1.5 * np.outer(one, one) / g.M[m]
    AP = A @ P
    for m in range(2, g.nb):
        one = np.zeros(g.N)
        one[o[m]:o[m + 1]] = 1.0
        assert np.abs(AP @ one - 0.5 * one).max() < 1e-12
    Dm = np.ones(g.N)
    Dm[o[0]:o[1]] = -1.0
    ev_a = np.linalg.eigvals(Dm[:, None] * A)
    ev_p = np.linalg.eigvals(Dm[:, None] * AP)
    assert np.sum(np.abs(ev_a + 1.0) < 1e-9) == g.nb - 2
    assert ev_p.real.min() > 0.05
    # each eigenvalue -1 moved to 1/2: the trace grows by 3/2 per obstacle
    tr_a = np.trace(Dm[:, None] * A)
    tr_p = np.trace(Dm[:, None] * AP)
    assert abs(tr_p - tr_a - 1.5 * (g.nb - 2)) < 1e-10


def test_solid_system_preconditioner_spectrum():
    """The vortex-sheet solid system of eq. lin:sys2 (bottom and obstacles):
    1_k is a left eigenvector for -1 on every obstacle (the transposed-kernel
    blocks annihilate constants from the left), while the rest of the spectrum
    clusters at -1/2; P = I - 1/2 sum_k 1_k 1_k^T / M_k moves those eigenvalues
    to -1/2 (the trace grows by 1/2 per obstacle) and leaves none near -1."""
    g = W.one_ellipse_640()[0]
    M = list(g.M)
    nb = len(M)
    ns = sum(M[1:])
    os_ = O.offsets(M[1:])
    E = np.zeros((ns, ns))
    for kk, k in enumerate(range(1, nb)):
        for jj, j in enumerate(range(1, nb)):
            c = O.vs_kernel_block(g, j, k)
            blk = np.imag(c) / M[j]
            if j == k:
                blk = blk - 0.5 * np.eye(M[k])
            E[os_[kk]:os_[kk + 1], os_[jj]:os_[jj + 1]] = blk
    P = np.eye(ns)
    for kk in range(1, nb - 1):
        one = np.zeros(ns)
        one[os_[kk]:os_[kk + 1]] = 1.0
        assert np.abs(one @ E + one).max() < 1e-12
        P -= 0.5 * np.outer(one, one) / M[kk + 1]
    ev = np.linalg.eigvals(E)
    ev_p = np.linalg.eigvals(E @ P)
    assert np.sum(np.abs(ev + 1.0) < 1e-9) == nb - 2
    assert np.sum(np.abs(ev_p + 1.0) < 1e-6) == 0
    assert abs(np.trace(E @ P) - np.trace(E) - 0.5 * (nb - 2)) < 1e-10


def test_uniform_flow_exact():
    """Flat bottom y = -h, graph surface, no obstacles, phi~ = 0: the exact
    potential is V1 z + i V1 h, so omega_0 = 0, omega_1 = 2 V1 h (eq.
    Phij:w:const for the bottom) and U = -V1 eta'/s_alpha (eq. d:phi:mv)."""
    h, V1 = 1.3, 0.7
    g = W.simple_channel(M0=128, M1=96, h=h)
    f = W.Flow(V1=V1, a=np.array([]))
    om, U, _ = O.solve(g, f, np.zeros(128))
    z0, dz0, _ = g.block(0)
    assert np.abs(om[:128]).max() < 1e-14
    assert np.abs(om[128:] - 2 * V1 * h).max() < 1e-13
    assert np.abs(U + V1 * dz0.imag / np.abs(dz0)).max() < 1e-13


@pytest.mark.parametrize("M0", [64, 128])
def test_dtn_closed_form(M0):
    """Exact Dirichlet-to-Neumann pair over a flat bottom: Phi~ = sum c_k cos(k(z + ih))
    has psi~ = 0 on y = -h; with b_0 = Re Phi~(zeta_0) the solve must return
    U = Re{(Phi~' + V1) i zeta_0'}/s_alpha (eqs. Awb, d:phi:mv, d:phi:j, d:phi:0)."""
    h = 1.3
    c = {1: 0.3, 2: -0.1, 3: 0.05}
    Phit = lambda z: sum(ck * np.cos(k * (z + 1j * h)) for k, ck in c.items())
    dPhit = lambda z: sum(-ck * k * np.sin(k * (z + 1j * h)) for k, ck in c.items())
    f = W.Flow(V1=0.7, a=np.array([]))
    g = W.simple_channel(M0=M0, M1=M0, h=h)
    z0, dz0, _ = g.block(0)
    om, U, _ = O.solve(g, f, np.real(Phit(z0)))
    Uex = np.real((dPhit(z0) + f.V1) * 1j * dz0) / np.abs(dz0)
    assert np.abs(U - Uex).max() < 1e-12 * np.abs(Uex).max() * 10


def test_velocity_at_targets_exact_field():
    """The DtN pair above has the exact field Phi'(z) = Phi~'(z) + V1: the oracle's
    far sums (eqs. Phi:j:prime, Phi:0:prime), its boundary values (eqs. phi:prime,
    dphij:dnk, dphij:dsk) and its Helsing quadrature (eq. helsing:quad) must
    reproduce it."""
    h = 1.3
    c = {1: 0.3, 2: -0.1, 3: 0.05}
    Phit = lambda z: sum(ck * np.cos(k * (z + 1j * h)) for k, ck in c.items())
    dPhit = lambda z: sum(-ck * k * np.sin(k * (z + 1j * h)) for k, ck in c.items())
    f = W.Flow(V1=0.7, a=np.array([]))
    g = W.simple_channel(M0=128, M1=128, h=h)
    z0, dz0, _ = g.block(0)
    om, U, _ = O.solve(g, f, np.real(Phit(z0)))
    # interior points away from the boundaries
    x = np.linspace(0.3, 6.0, 9)
    zi = x - 0.6j
    assert np.abs(O.velocity_far(g, f, om, zi) - (dPhit(zi) + f.V1)).max() < 1e-11
    fb = O.boundary_dphi(g, f, om)
    zb = np.concatenate([z0, g.zeta[128:]])
    assert np.abs(np.concatenate(fb) - (dPhit(zb) + f.V1)).max() < 1e-11
    # points one node spacing under the surface
    zn = z0[::9] - 1j * 0.05
    assert np.abs(O.helsing_eval(g, fb, zn) - (dPhit(zn) + f.V1)).max() < 1e-11


def test_cauchy_identity_inside_outside():
    """eq. res:thm: the trapezoidal Cauchy integral over the positively oriented
    boundary reproduces f inside Omega and gives 0 outside (f = e^{inz})."""
    g = W.one_ellipse_640()[0]
    o = O.offsets(g.M)
    zin = np.array([1.0 - 0.3j, 3.0 - 0.8j, 0.5 - 0.5j])
    zout = np.array([1 + 0.5j, np.pi - 0.5 + 0.02j, 2.0 - 1.5j])
    for n in range(-3, 4):
        fv = [np.exp(1j * n * g.zeta[o[k]:o[k + 1]]) for k in range(g.nb)]
        assert np.abs(O.cauchy_sum(g, fv, zin) - np.exp(1j * n * zin)).max() < 1e-13
        assert np.abs(O.cauchy_sum(g, fv, zout)).max() < 1e-11


def test_helsing_near_boundary():
    """eq. helsing:quad keeps spectral accuracy 1e-3 away from an obstacle, where
    the plain trapezoidal Cauchy sum loses all digits."""
    g = W.one_ellipse_640()[0]
    o = O.offsets(g.M)
    zk = g.zeta[o[2]:o[3]]
    dzk = g.dzeta[o[2]:o[3]]
    ztg = zk[::7] + 1e-3 * (1j * dzk[::7] / np.abs(dzk[::7]))
    fun = lambda z: np.exp(2j * z) + 0.5 * O.half_cot(z - (np.pi - 0.5j))
    fv = [fun(g.zeta[o[k]:o[k + 1]]) for k in range(g.nb)]
    assert np.abs(O.helsing_eval(g, fv, ztg) - fun(ztg)).max() < 1e-12
    assert np.abs(O.cauchy_sum(g, fv, ztg) - fun(ztg)).max() > 1e-2
    # a target on a node returns the node value
    assert np.abs(O.helsing_eval(g, fv, zk[:3]) - fv[2][:3]).max() == 0.0


# ---------------------------------------------------------------- invariants

@pytest.mark.parametrize("which", ["one_ellipse_640", "problem3"])
def test_zero_net_flux(which):
    """int_Gamma U ds = 0 (App. A, divergence theorem)."""
    g, f, ph = W.one_ellipse_640() if which == "one_ellipse_640" else W.paper_problem(3)
    om, U, _ = O.solve(g, f, ph)
    dz0 = g.block(0)[1]
    assert abs(np.mean(U * np.abs(dz0))) < 1e-13


def test_solid_normal_velocity_vanishes():
    """psi = const on solids (eq. psi:k) means phi_n = 0 there: evaluate
    s_k phi_n with eqs. dphij:dnk from the VP densities."""
    g, f, ph = W.one_ellipse_640()
    om, U, _ = O.solve(g, f, ph)
    bd = O.boundary_dphi(g, f, om)
    o = O.offsets(g.M)
    for k in range(1, g.nb):
        dzk = g.dzeta[o[k]:o[k + 1]]
        assert np.abs(np.real(bd[k] * 1j * dzk)).max() < 1e-11
    # and on the surface phi_n from eq. phi:prime equals U
    dz0 = g.dzeta[: g.M[0]]
    assert np.abs(np.real(bd[0] * 1j * dz0) / np.abs(dz0) - U).max() < 1e-12


def test_vortex_sheet_matches_velocity_potential():
    """Sec. 4.1: U from gamma_0 = -omega_0' through eq. lin:sys2 / eq. U:from:gam:j
    (an independent system) equals the VP normal velocity."""
    g, f, ph = W.one_ellipse_640()
    om, U, _ = O.solve(g, f, ph)
    Uvs = O.vs_normal_velocity(g, f, -O.d_alpha(om[: g.M[0]]))
    assert np.abs(Uvs - U).max() < 1e-12


def test_spectral_self_convergence():
    """Refining every boundary by 3/2 changes U by ~ rounding only (Sec. 7.3)."""
    g1, f, ph = W.paper_problem(3, M0=256, M1=96, Me=128)
    g2, _, _ = W.paper_problem(3, M0=384, M1=144, Me=192)
    _, U1, p1 = O.solve(g1, f, np.zeros(256))
    _, U2, p2 = O.solve(g2, f, np.zeros(384))
    # compare on the common nodes (every 2nd of 256 <-> every 3rd of 384)
    assert np.abs(U1[::2] - U2[::3]).max() < 1e-11
    assert np.abs(p1 - p2).max() < 1e-11


def test_dense_solve_residual():
    g, f, ph = W.one_ellipse_640()
    A = O.assemble(g)
    b = O.rhs(g, f, ph)
    om = O.solve_dense(A, b)
    r = b - A @ om
    assert np.linalg.norm(r) <= 1e-14 * np.linalg.norm(A, 2) * np.linalg.norm(om)


# ---------------------------------------------------------------- planted mistakes

def _pins_hold():
    try:
        test_energy_t0_matches_paper_table()
        test_constant_density_row_sums("one_ellipse_640")
        test_dtn_closed_form(64)
        test_zero_net_flux("one_ellipse_640")
        test_vortex_sheet_matches_velocity_potential()
    except AssertionError:
        return False
    return True


@pytest.mark.parametrize("mutation", ["diag_limit_sign", "block_sign", "drop_hilbert",
                                      "ccw_ellipse", "psi_cyl_sign", "transpose_U"])
def test_planted_mistakes_break_a_pin(monkeypatch, mutation):
    """Each plausible mistake, planted in the oracle on the CPU, fails a pin."""
    if mutation == "diag_limit_sign":
        orig = O.kernel_rows

        def bad(geom, rows):
            A = orig(geom, rows)
            rows = np.asarray(rows)
            bid = O.block_ids(geom.M)
            Mj = np.asarray(geom.M, float)[bid[rows]]
            d = (geom.d2zeta[rows] / (2 * geom.dzeta[rows])).imag / Mj
            A[np.arange(len(rows)), rows] -= 2 * d
            return A
        monkeypatch.setattr(O, "kernel_rows", bad)
    elif mutation == "block_sign":
        orig = O.kernel_rows

        def bad(geom, rows):
            A = orig(geom, rows)
            bid = O.block_ids(geom.M)
            rows = np.asarray(rows)
            mask = (bid[rows][:, None] >= 1) & (bid[None, :] == 0)
            A[mask] *= -1.0          # +G_k0 instead of -G_k0
            return A
        monkeypatch.setattr(O, "kernel_rows", bad)
    elif mutation == "drop_hilbert":
        monkeypatch.setattr(O, "hilbert", lambda f: 0 * f)
    elif mutation == "ccw_ellipse":
        orig = W.ellipse

        def bad(M, x, y, q, b, th):
            z, dz, d2z = orig(M, x, y, q, -b, th)
            return z, dz, d2z
        monkeypatch.setattr(W, "ellipse", bad)
    elif mutation == "psi_cyl_sign":
        monkeypatch.setattr(O, "psi_cyl", lambda z: np.log(np.abs(1.0 - np.exp(1j * z))))
    elif mutation == "transpose_U":
        orig = O.normal_velocity

        def bad(geom, flow, omega):
            # use the source derivative zeta_j'(beta) instead of zeta_0'(alpha)
            M = list(geom.M)
            z0, dz0, d2z0 = geom.block(0)
            w = O.split(omega, M)
            wp = [O.d_alpha(x) for x in w]
            U = orig(geom, flow, omega) * np.abs(dz0)
            o = O.offsets(M)
            for j in range(1, len(M)):
                zj = geom.zeta[o[j]:o[j + 1]]
                dzj = geom.dzeta[o[j]:o[j + 1]]
                good = np.imag(dz0[:, None] * O.half_cot(z0[:, None] - zj[None, :]))
                badk = np.imag(-dzj[None, :] * O.half_cot(zj[None, :] - z0[:, None]))
                U += (badk - good) @ wp[j] / M[j]
            return U / np.abs(dz0)
        monkeypatch.setattr(O, "normal_velocity", bad)
    assert not _pins_hold(), mutation


# ---------------------------------------------------------------- directional derivatives

def _U_at(g, f, ph):
    return O.solve(g, f, ph)[1]


def test_directional_derivative_matches_central_differences():
    """Forward-mode dU (hand-differentiated chain) vs central differences of
    the oracle's own forward map: O(h^2) truncation, h = 1e-5."""
    g, f, ph = W.one_ellipse_640()
    d = W.adjoint_direction(g, seed=0)
    U, dU = O.directional_U(g, f, ph, *d)
    h = 1e-5
    Up = _U_at(W.perturbed(g, d, h), f, ph + h * d[4])
    Um = _U_at(W.perturbed(g, d, -h), f, ph - h * d[4])
    fd = (Up - Um) / (2 * h)
    assert np.abs(dU - fd).max() <= 1e-6 * np.abs(dU).max()
    dJ = O.directional_objective(g, f, ph, *d)
    assert abs(dJ - 2 * 2 * np.pi / g.M[0] * np.sum(U * fd)) <= 1e-6 * abs(dJ)


def test_directional_derivative_phitilde_exact():
    """U is affine in phi~ (A omega = b, b_0 = phi~): the derivative along phi~
    alone equals the finite difference for any step, to rounding."""
    g, f, ph = W.one_ellipse_640()
    dphit = W.filtered_noise(np.random.default_rng(5), g.M[0], 0.3, 12)
    z = np.zeros(g.N, complex)
    _, dU = O.directional_U(g, f, ph, z, z, z, np.zeros(len(g.zc), complex), dphit)
    diff = _U_at(g, f, ph + dphit) - _U_at(g, f, ph)
    assert np.abs(dU - diff).max() <= 1e-11 * np.abs(diff).max()


def test_directional_derivative_horizontal_translation():
    """Moving every node and centre by the same real shift leaves U unchanged
    (the kernel and Phi_mv depend on differences, psi_mv's V1 Im z does not see
    a real shift): dU = 0."""
    g, f, ph = W.one_ellipse_640()
    one = np.ones(g.N, complex)
    z = np.zeros(g.N, complex)
    U, dU = O.directional_U(g, f, ph, one, z, z, np.ones(len(g.zc), complex), np.zeros(g.M[0]))
    assert np.abs(dU).max() <= 1e-11 * np.abs(U).max()


@pytest.mark.parametrize("mutation", ["drop_kernel_derivative", "drop_centre_motion"])
def test_planted_derivative_mistakes_break_a_pin(monkeypatch, mutation):
    if mutation == "drop_kernel_derivative":
        monkeypatch.setattr(O, "d_half_cot", lambda z: 0.0 * z)
    else:
        orig = O.directional_U

        def bad(geom, flow, ph, dz, ddz, dd2z, dzc, dphit):
            return orig(geom, flow, ph, dz, ddz, dd2z, 0 * dzc, dphit)
        monkeypatch.setattr(O, "directional_U", bad)
    with pytest.raises(AssertionError):
        test_directional_derivative_matches_central_differences()


# ---------------------------------------------------------------- energy conservation

def _energy_drift(nsteps, dt=0.005):
    g, f, ph = W.paper_problem(1)
    E = O.evolve_energy(g, f, np.zeros(g.M[0]), ph, dt, nsteps)
    return np.abs(E - E[0]).max() / abs(E[0])


def test_energy_conserved_by_graph_evolution():
    """E of eq. E:formula is conserved by eqs. graph:eta:t and phitileq (Sec.
    5.2): problem 1 of Sec. 7 (flat surface at rest, circulation and current
    driving it), classical RK4 at dt = 0.005 (inside the capillary step limit
    for tau = 0.1, M_0 = 256) to t = 0.1.  Measured drift 1.3e-14."""
    assert _energy_drift(20) <= 1e-11


@pytest.mark.parametrize("mutation", ["drop_hilbert", "scale_U", "drop_psi_k"])
def test_planted_mistakes_break_energy_conservation(monkeypatch, mutation):
    if mutation == "drop_hilbert":
        monkeypatch.setattr(O, "hilbert", lambda x: 0 * x)
    elif mutation == "scale_U":
        orig = O.normal_velocity
        monkeypatch.setattr(O, "normal_velocity",
                            lambda geom, flow, om, targets=None: orig(geom, flow, om, targets) * (1 + 1e-3))
    else:
        orig = O.psi_k
        monkeypatch.setattr(O, "psi_k", lambda geom, om: 0 * orig(geom, om))
    assert _energy_drift(6) > 1e-9


# ---------------------------------------------------------------------------
# auxiliary Dirichlet data for Phi_t - C (Sec. 4, eq. pressure:d:prob)
# ---------------------------------------------------------------------------

def _reparam_graph(M, f, df, d2f, eps=0.2):
    """The graph y = f(x) traced with x = xi(alpha) = alpha + eps sin(alpha):
    zeta = xi + i f(xi), zeta' = xi' (1 + i f'), zeta'' = xi'' (1 + i f') + i xi'^2 f''."""
    a = 2 * np.pi * np.arange(M) / M
    xi, dxi, d2xi = a + eps * np.sin(a), 1 + eps * np.cos(a), -eps * np.sin(a)
    z = xi + 1j * f(xi)
    dz = dxi * (1 + 1j * df(xi))
    d2z = d2xi * (1 + 1j * df(xi)) + 1j * dxi ** 2 * d2f(xi)
    return (z, dz, d2z), xi


def test_curvature_closed_form():
    """kappa of a graph y = f(x) is f''/(1 + f'^2)^(3/2) however the curve is
    parametrized (uniform or stretched alpha)."""
    f = lambda x: 0.1 * np.cos(x) + 0.03 * np.sin(2 * x)
    df = lambda x: -0.1 * np.sin(x) + 0.06 * np.cos(2 * x)
    d2f = lambda x: -0.1 * np.cos(x) - 0.12 * np.sin(2 * x)
    for eps in (0.0, 0.2):
        surf, xi = _reparam_graph(128, f, df, d2f, eps)
        bot = W.graph_curve(96, lambda a: -1.0 + 0 * a, lambda a: 0 * a, lambda a: 0 * a)
        g = W.assemble_geometry([surf, bot], [])
        exact = d2f(xi) / (1 + df(xi) ** 2) ** 1.5
        assert np.abs(O.curvature_surface(g) - exact).max() < 1e-14


def test_pressure_rhs_exact_field():
    """For the exact flat-bottom field Phi = Phi~ + V1 z of the DtN pin,
    |grad phi|^2 = |Phi'(zeta_0)|^2 on the surface, so b^aux_0 must equal
    tau kappa - |Phi~'(zeta_0) + V1|^2 / 2 - g eta with U from the solve, and
    b^aux is 0 on the bottom."""
    h, tau, grav = 1.3, 0.07, 9.81
    c = {1: 0.3, 2: -0.1, 3: 0.05}
    Phit = lambda z: sum(ck * np.cos(k * (z + 1j * h)) for k, ck in c.items())
    dPhit = lambda z: sum(-ck * k * np.sin(k * (z + 1j * h)) for k, ck in c.items())
    f = W.Flow(V1=0.7, a=np.array([]))
    g = W.simple_channel(M0=128, M1=128, h=h)
    z0, dz0, d2z0 = g.block(0)
    ph = np.real(Phit(z0))
    om, U, _ = O.solve(g, f, ph)
    b = O.pressure_rhs(g, f, ph, U, tau=tau, g=grav)
    eta = z0.imag
    kap = (d2z0.imag) / (1 + dz0.imag ** 2) ** 1.5          # graph: xi = alpha
    exact = tau * kap - 0.5 * np.abs(dPhit(z0) + f.V1) ** 2 - grav * eta
    assert np.abs(b[:128] - exact).max() < 1e-11
    assert np.all(b[128:] == 0.0)
    # planted mistakes: tangential part dropped, curvature sign flipped
    s = np.abs(dz0)
    bad1 = exact + 0.5 * (O.phi_alpha_surface(g, f, ph) / s) ** 2
    bad2 = exact - 2 * tau * kap
    assert np.abs(bad1 - exact).max() > 1e-3 and np.abs(bad2 - exact).max() > 1e-3


def test_pressure_rhs_with_obstacle_current():
    """A uniform stream V1 over a flat surface and bottom, no obstacles: phi = V1 x,
    U = 0, so b^aux_0 = -V1^2/2 exactly; adding a circulation a_2 around an
    obstacle changes |grad phi|^2 by the multi-valued part of eq. d:phi:cyl,
    which the oracle must take from Phi_mv' (checked against the solve's own
    tangential velocity from the boundary values of Phi')."""
    g = W.simple_channel(M0=64, M1=64, h=1.0, surface=W.graph_curve(
        64, lambda a: 0 * a, lambda a: 0 * a, lambda a: 0 * a))
    f = W.Flow(V1=0.8, a=np.array([]))
    om, U, _ = O.solve(g, f, np.zeros(64))
    b = O.pressure_rhs(g, f, np.zeros(64), U, tau=0.3, g=2.0)
    assert np.abs(b[:64] + 0.5 * 0.8 ** 2).max() < 1e-13
    g2, f2, ph2 = W.one_ellipse_640()
    om2, U2, _ = O.solve(g2, f2, ph2)
    fb = O.boundary_dphi(g2, f2, om2)[0]                    # Phi' on the surface (from the fluid)
    grad2 = np.abs(fb) ** 2
    b2 = O.pressure_rhs(g2, f2, ph2, U2, tau=0.0, g=0.0)
    assert np.abs(b2[:256] + 0.5 * grad2).max() < 1e-9 * grad2.max()


# ---------------------------------------------------------------------------
# filter of eq. filter and the filtered graph evolution
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("M", [64, 96])
def test_filter36_closed_form(M):
    """cos(k alpha) and sin(k alpha) are eigenfunctions: the filter multiplies
    them by exp(-36 (k / (M/2))^36); a constant is kept; the Nyquist mode
    cos(M alpha / 2) (even M) is multiplied by exp(-36)."""
    a = 2 * np.pi * np.arange(M) / M
    for k in (0, 1, 5, M // 4, M // 2 - 1):
        rho = np.exp(-36.0 * (k / (M / 2)) ** 36)
        assert np.abs(O.filter36(np.cos(k * a)) - rho * np.cos(k * a)).max() < 1e-13
        assert np.abs(O.filter36(np.sin(k * a)) - rho * np.sin(k * a)).max() < 1e-13
    nyq = np.cos(M // 2 * a)
    assert np.abs(O.filter36(nyq) - np.exp(-36.0) * nyq).max() < 1e-13
    # a planted mistake (k_max = M instead of M/2) is caught
    k = M // 2 - 1
    wrong = np.exp(-36.0 * (k / M) ** 36) * np.cos(k * a)
    assert np.abs(O.filter36(np.cos(k * a)) - wrong).max() > 1e-3


def test_evolve_graph_matches_unfiltered_and_filter_is_tiny_on_resolved_data():
    """Without the filter the evolution is evolve_energy's (same energies); on a
    well-resolved state the filter changes the result by far less than the
    step's own truncation error, and energy stays conserved."""
    g, f, ph = W.paper_problem(1)
    z = np.zeros(g.M[0])
    E = O.evolve_energy(g, f, z, ph, 0.005, 4)
    eta1, ph1, E1 = O.evolve_graph(g, f, z, ph, 0.005, 4)
    assert np.array_equal(E, E1)
    eta2, ph2, E2 = O.evolve_graph(g, f, z, ph, 0.005, 4, filt=True)
    assert np.abs(eta2 - eta1).max() < 1e-10 and np.abs(ph2 - ph1).max() < 1e-10
    assert np.abs(E2 - E2[0]).max() / abs(E2[0]) < 1e-11


# ---------------------------------------------------------------------------
# App. B: psi prescribed on the solids, circulations unknown
# ---------------------------------------------------------------------------

def _alt_data_from_standard(g, f, ph):
    """The App. B data of the flow that the standard solve describes:
    phi - V1 xi = phi~ + sum a_j phi_cyl(zeta_0 - z_j) on the surface, psi = 0 on
    the bottom and psi|_k = <1_k, omega> on obstacle k (eqs. psi:k, Awb)."""
    om, U, psik = O.solve(g, f, ph)
    M0 = g.M[0]
    o = O.offsets(g.M)
    phic = ph + sum(aj * O.phi_cyl(g.zeta[:M0] - zj) for aj, zj in zip(f.a, g.zc))
    psi_s = np.zeros(g.N - M0)
    for k in range(2, len(g.M)):
        psi_s[o[k] - M0:o[k + 1] - M0] = psik[k - 2]
    return om, U, psik, phic, psi_s


@pytest.mark.parametrize("case", ["one_ellipse_640", "paper3"])
def test_psi_prescribed_reproduces_standard_flow(case):
    """Both formulations describe the same Phi (App. B): the App. B solve on the
    standard solution's boundary data returns its circulations a_j and normal
    velocity, and omega differs from the standard one by a constant on each
    obstacle (a_k - psi|_k: the kernel of B) and not at all elsewhere."""
    g, f, ph = W.one_ellipse_640() if case == "one_ellipse_640" else W.paper_problem(3)
    om, U, psik, phic, psi_s = _alt_data_from_standard(g, f, ph)
    om2, U2, a2 = O.solve_alt(g, f.V1, phic, psi_s)
    o = O.offsets(g.M)
    assert np.abs(a2 - f.a).max() < 1e-12
    assert np.abs(U2 - U).max() < 1e-12 * np.abs(U).max()
    assert np.abs(om2[:o[2]] - om[:o[2]]).max() < 1e-12 * np.abs(om).max()
    for k in range(2, len(g.M)):
        d = om2[o[k]:o[k + 1]] - om[o[k]:o[k + 1]]
        assert np.abs(d - (f.a[k - 2] - psik[k - 2])).max() < 1e-12 * np.abs(om).max()


def test_psi_prescribed_planted_mistakes():
    """Wrong-part mistakes in the rank-(N-1) column (psi_cyl on the surface rows,
    or phi_cyl's sign flipped) break the reproduction of a_j."""
    g, f, ph = W.one_ellipse_640()
    om, U, psik, phic, psi_s = _alt_data_from_standard(g, f, ph)
    orig = O.phi_cyl
    for bad in (O.psi_cyl, lambda z: -orig(z)):
        O.phi_cyl = bad
        try:
            _, _, a2 = O.solve_alt(g, f.V1, phic, psi_s)
        finally:
            O.phi_cyl = orig
        assert np.abs(a2 - f.a).max() > 1e-6


def test_phi_cyl_is_the_conjugate_of_psi_cyl():
    """Phi_cyl = phi_cyl + i psi_cyl is analytic with derivative
    e^{iz}/(e^{iz} - 1) (eq. d:phi:cyl): central differences in x of phi_cyl
    and in y of psi_cyl agree (Cauchy-Riemann) and match Re of the derivative."""
    z = np.array([0.3 + 0.4j, 2.0 + 1.1j, 5.5 + 0.2j])
    h = 1e-5
    dphi_dx = (O.phi_cyl(z + h) - O.phi_cyl(z - h)) / (2 * h)
    dpsi_dy = (O.psi_cyl(z + 1j * h) - O.psi_cyl(z - 1j * h)) / (2 * h)
    d = np.exp(1j * z) / (np.exp(1j * z) - 1.0)
    assert np.abs(dphi_dx - d.real).max() < 1e-9
    assert np.abs(dpsi_dy - d.real).max() < 1e-9


# ---------------------------------------------------------------------------
# HLS formulation with P theta reconstruction (Sec. 2)
# ---------------------------------------------------------------------------

def _trig_eval(samples, x):
    """The trigonometric interpolant of periodic samples at arbitrary x."""
    M = len(samples)
    F = np.fft.fft(samples) / M
    k = np.fft.fftfreq(M, d=1.0 / M)
    if M % 2 == 0:
        F[M // 2] = 0
    return np.real(np.exp(1j * np.outer(x, k)) @ F)


def test_hls_curve_reconstruction():
    """eq. CS:th / eq. xi:eta:recon: xi(0) = 0, <eta> = P0[eta xi_alpha] = 0,
    |zeta'| = s_alpha, the reconstructed curve is periodic (its spectral
    derivative is s_alpha e^{i theta}) and returns theta; P theta = 0 gives
    the flat line zeta = alpha.  A sign slip in P0 theta breaks periodicity."""
    M = 256
    a = 2 * np.pi * np.arange(M) / M
    Pth = 0.8 * np.cos(a) + 0.6 * np.cos(2 * a) + 0.1 * np.sin(3 * a)   # P0[sin] = -0.043
    z, dz, d2z, th, s = O.hls_curve(Pth)
    assert abs(z[0].real) < 1e-15 and abs(np.mean(z.imag * dz.real)) < 1e-15
    assert np.abs(np.abs(dz) - s).max() < 1e-14
    dxi = O.d_alpha(z.real - a) + 1.0
    deta = O.d_alpha(z.imag)
    assert np.abs(dxi - dz.real).max() < 1e-12 and np.abs(deta - dz.imag).max() < 1e-12
    assert np.abs(np.angle(dxi + 1j * deta) - th).max() < 1e-12
    assert np.abs(O.d_alpha(dz.real) + 1j * O.d_alpha(dz.imag) - d2z).max() < 1e-11
    z0, dz0, d2z0, _, s0 = O.hls_curve(np.zeros(M))
    assert np.abs(z0 - a).max() < 1e-15 and s0 == 1.0 and np.all(d2z0 == 0)
    # planted: P0 theta = arg(C + iS)
    C, S = np.mean(np.cos(Pth)), np.mean(np.sin(Pth))
    dzb = s * np.exp(1j * (Pth + np.angle(C + 1j * S)))
    assert abs(np.mean(dzb) - 1.0) > 1e-3          # the period would not close


def test_hls_and_graph_give_the_same_surface():
    """Problem 1 from rest to t = 0.05 (dt = 0.005, RK4) in both formulations:
    the HLS curve lies on the graph surface y = eta(x) to the time-stepping
    error (4.7e-12; 3.0e-13 at dt/2, the RK4 ratio 16), and both conserve E."""
    g, f, ph = W.paper_problem(1)
    M0 = g.M[0]
    eg, _, Eg = O.evolve_graph(g, f, np.zeros(M0), ph, 0.005, 10)
    th, _, Eh = O.evolve_hls(g, f, np.zeros(M0), ph, 0.005, 10)
    z, _, _, _, _ = O.hls_curve(th)
    assert np.abs(z.imag - _trig_eval(eg, z.real)).max() < 1e-10
    assert np.abs(Eh - Eh[0]).max() < 1e-11 * abs(Eh[0])
    assert abs(Eh[-1] - Eg[-1]) < 1e-11 * abs(Eg[-1])


@pytest.mark.parametrize("mutation", ["V0_zero", "drop_V_theta", "V_mean_kept"])
def test_hls_planted_mistakes(monkeypatch, mutation):
    orig_V, orig_t = O.hls_tangential_velocity, O.hls_theta_t
    if mutation == "V0_zero":
        monkeypatch.setattr(O, "hls_tangential_velocity",
                            lambda ta, U, dz0: orig_V(ta, U, dz0) - orig_V(ta, U, dz0)[0])
    elif mutation == "drop_V_theta":
        monkeypatch.setattr(O, "hls_theta_t", lambda U, V, ta, s: orig_t(U, 0 * V, ta, s))
    else:
        monkeypatch.setattr(O, "hls_tangential_velocity",
                            lambda ta, U, dz0: O.antiderivative(ta * U) + U[0] * dz0[0].imag / dz0[0].real)
    with pytest.raises(AssertionError):
        test_hls_and_graph_give_the_same_surface()


# ---------------------------------------------------------------------------
# eighth-order extrapolation step
# ---------------------------------------------------------------------------

def _rotation_error(h, n, step=None):
    step = step or O.gbs8_step
    f = lambda y: np.array([-y[1], y[0]])
    y = np.array([1.0, 0.0])
    for _ in range(n):
        y = step(f, y, h)
    t = h * n
    return np.abs(y - np.array([np.cos(t), np.sin(t)])).max()


def test_gbs8_is_eighth_order():
    """y' = (-y_1, y_0) to t = 2: halving h divides the error by 2^8 = 256
    (measured 261) and h = 0.25 is within 1e-10 of (cos 2, sin 2)."""
    e1, e2 = _rotation_error(0.5, 4), _rotation_error(0.25, 8)
    assert e2 < 1e-10
    assert 180 < e1 / e2 < 360


def test_gbs8_planted_mistake_lowers_the_order(monkeypatch):
    """The sequence (1, 2, 3, 4) contains odd n, for which the midpoint rule has
    no even-power expansion: the order drops and the pin above fails."""
    monkeypatch.setattr(O, "GBS_SEQUENCE", (1, 2, 3, 4))
    with pytest.raises(AssertionError):
        test_gbs8_is_eighth_order()


def test_gbs8_water_waves_agree_with_rk4_and_conserve_energy():
    """Problem 1 from rest to t = 0.02.  GBS8 with dt = 0.01 and 0.005 agree to
    7.6e-13 of max|eta| (eighth order); RK4 with dt = 0.00125 is within its own
    error (2.7e-11); the HLS formulation under GBS8 gives the same surface; E is
    conserved."""
    g, f, ph = W.paper_problem(1)
    M0 = g.M[0]
    e8, p8, E8 = O.evolve_gbs8(g, f, np.zeros(M0), ph, 0.01, 2)
    e8h, _, _ = O.evolve_gbs8(g, f, np.zeros(M0), ph, 0.005, 4)
    e4, p4, _ = O.evolve_graph(g, f, np.zeros(M0), ph, 0.00125, 16)
    sc = np.abs(e8h).max()
    assert np.abs(e8 - e8h).max() < 5e-12 * sc
    assert np.abs(e8h - e4).max() < 1e-10 * sc
    assert np.abs(p8 - p4).max() < 1e-9 * np.abs(p4).max()
    assert np.abs(E8 - E8[0]).max() < 1e-11 * abs(E8[0])
    t8, q8, _ = O.evolve_gbs8(g, f, np.zeros(M0), ph, 0.01, 2, formulation="hls")
    z, _, _, _, _ = O.hls_curve(t8)
    assert np.abs(z.imag - _trig_eval(e8, z.real)).max() < 1e-11


# ---------------------------------------------------------------------------
# the paper's eighth-order Dormand-Prince step (Sec. 7.1)
# ---------------------------------------------------------------------------

def _rooted_trees(max_order):
    """All rooted trees up to max_order, each as a canonical nested tuple of
    its subtrees (a leaf is ()), grown by attaching one leaf at every node of
    every tree of the previous order."""
    def canon(t):
        return tuple(sorted(canon(c) for c in t))

    def grow(t):
        out = [canon(t + ((),))]
        for i, c in enumerate(t):
            for g in grow(c):
                out.append(canon(t[:i] + (g,) + t[i + 1:]))
        return out

    levels = [[()]]
    for _ in range(max_order - 1):
        levels.append(sorted(set(g for t in levels[-1] for g in grow(t))))
    return levels


def _order_and_density(t):
    n, gam = 1, 1
    for c in t:
        nc, gc = _order_and_density(c)
        n += nc
        gam *= gc
    return n, gam * n


def _stage_weights(A, t):
    """The stage vector of the elementary weight: prod over the subtrees of
    A times their stage vectors (1 for a leaf)."""
    v = np.ones(A.shape[0])
    for c in t:
        v = v * (A @ _stage_weights(A, c))
    return v


def _order_defects(A, b, max_order=8):
    """|b . Phi(t) - 1/gamma(t)| for every rooted tree t up to max_order."""
    out = []
    for level in _rooted_trees(max_order):
        for t in level:
            _, gam = _order_and_density(t)
            out.append(abs(b @ _stage_weights(A, t) - 1.0 / gam))
    return np.array(out)


def test_rooted_tree_counts():
    """1, 1, 2, 4, 9, 20, 48, 115 rooted trees of orders 1..8 (200 in all)."""
    assert [len(l) for l in _rooted_trees(8)] == [1, 1, 2, 4, 9, 20, 48, 115]


def test_dp8_tableau_meets_every_order_condition_to_order_8():
    """All 200 order conditions b . Phi(t) = 1/gamma(t) of orders 1..8 hold to
    rounding; the abscissae are the row sums with their closed forms; at least
    one order-9 condition fails (the method is of order exactly 8)."""
    A, b, c = O.DP8_A, O.DP8_B, O.DP8_C
    assert np.abs(A.sum(axis=1) - c).max() < 1e-15
    r6 = np.sqrt(6.0)
    assert abs(c[3] - (6 - r6) / 30) < 1e-16 and abs(c[4] - (6 + r6) / 30) < 1e-16
    assert abs(c[2] - 2 * c[3] / 3) < 1e-16 and abs(c[1] - 2 * c[2] / 3) < 1e-16
    assert np.allclose(np.triu(A), 0.0)
    d = _order_defects(A, b, 8)
    assert len(d) == 200 and d.max() < 2e-14, d.max()
    d9 = _order_defects(A, b, 9)[200:]
    assert d9.max() > 1e-6


@pytest.mark.parametrize("where", [(8, 5), (11, 10)])
def test_dp8_planted_coefficient_error_breaks_an_order_condition(where):
    """A relative change of 1e-9 in one coefficient leaves the row sums to
    rounding-level c changes but breaks order conditions well above rounding."""
    A = O.DP8_A.copy()
    A[where] *= 1 + 1e-9
    assert _order_defects(A, O.DP8_B, 8).max() > 1e-11


def _kepler(t, e=0.5):
    """Kepler orbit of eccentricity e, period 2 pi, from perihelion: (x, y, x', y')."""
    E = t
    for _ in range(60):
        E = E - (E - e * np.sin(E) - t) / (1 - e * np.cos(E))
    r = 1 - e * np.cos(E)
    w = np.sqrt(1 - e * e)
    return np.array([np.cos(E) - e, w * np.sin(E), -np.sin(E) / r, w * np.cos(E) / r])


def _kepler_f(y):
    r3 = (y[0] ** 2 + y[1] ** 2) ** 1.5
    return np.array([y[2], y[3], -y[0] / r3, -y[1] / r3])


def test_dp8_step_equals_library_dop853_fixed_step():
    """scipy's DOP853 (the same published method) held to a fixed step h =
    2^-5 on the Kepler problem gives the same 64 steps to rounding."""
    from scipy.integrate import solve_ivp
    h, n = 2.0 ** -5, 64
    y = _kepler(0.0)
    for _ in range(n):
        y = O.dp8_step(_kepler_f, y, h)
    sol = solve_ivp(lambda t, x: _kepler_f(x), (0.0, n * h), _kepler(0.0), method="DOP853",
                    first_step=h, max_step=h, rtol=1e3, atol=1e3)
    assert len(sol.t) == n + 1 and np.allclose(np.diff(sol.t), h, rtol=0, atol=1e-15)
    assert np.abs(sol.y[:, -1] - y).max() < 1e-14 * np.abs(y).max()


def test_dp8_is_eighth_order_on_kepler():
    """Kepler (e = 0.5) to t = 2: halving h from 0.1 divides the error by
    2^8 (measured 250; 1.3e-9 and 5.3e-12)."""
    errs = []
    for h in (0.1, 0.05):
        y = _kepler(0.0)
        for _ in range(int(round(2.0 / h))):
            y = O.dp8_step(_kepler_f, y, h)
        errs.append(np.abs(y - _kepler(2.0)).max())
    assert errs[1] < 1e-10
    assert 180 < errs[0] / errs[1] < 360, errs


def test_dp8_planted_weight_error_lowers_the_order(monkeypatch):
    """A weight b_8 off by 1e-6 (so sum b != 1) makes the step first order:
    the order pin above fails."""
    b = O.DP8_B.copy()
    b[7] += 1e-6
    monkeypatch.setattr(O, "DP8_B", b)
    with pytest.raises(AssertionError):
        test_dp8_is_eighth_order_on_kepler()


def test_dp8_water_waves_self_converge_and_agree_with_gbs8():
    """Problem 1 from rest to t = 0.02 with the paper's integrator: dt = 0.01
    and 0.005 agree to eighth-order accuracy; GBS8 and fine RK4 give the same
    surface within their own errors; E is conserved; the HLS formulation under
    DP8 gives the same surface."""
    g, f, ph = W.paper_problem(1)
    M0 = g.M[0]
    e8, p8, E8 = O.evolve_dp8(g, f, np.zeros(M0), ph, 0.01, 2)
    e8h, p8h, _ = O.evolve_dp8(g, f, np.zeros(M0), ph, 0.005, 4)
    eg, pg, _ = O.evolve_gbs8(g, f, np.zeros(M0), ph, 0.005, 4)
    e4, p4, _ = O.evolve_graph(g, f, np.zeros(M0), ph, 0.00125, 16)
    sc = np.abs(e8h).max()
    assert np.abs(e8 - e8h).max() < 5e-12 * sc
    assert np.abs(e8h - eg).max() < 5e-12 * sc
    assert np.abs(p8h - pg).max() < 5e-11 * np.abs(pg).max()
    assert np.abs(e8h - e4).max() < 1e-10 * sc
    assert np.abs(E8 - E8[0]).max() < 1e-11 * abs(E8[0])
    t8, _, _ = O.evolve_dp8(g, f, np.zeros(M0), ph, 0.01, 2, formulation="hls")
    z, _, _, _, _ = O.hls_curve(t8)
    assert np.abs(z.imag - _trig_eval(e8, z.real)).max() < 1e-11


# ---------------------------------------------------------------------------
# vortex-sheet evolution: gamma_0,t (eqs. gam:t:final, gam:t:aux)
# ---------------------------------------------------------------------------

def _gamma_t_vs_fd(case):
    """gamma_0,t from the vortex-sheet system against the time derivative of
    gamma_0 = -omega_0' along the velocity-potential flow (eq. gam:def), by
    central differences in time with h = 1e-3 and 5e-4, Richardson-extrapolated
    (O(h^4)).  Returns the relative difference."""
    g, f, ph = W.paper_problem(1) if case == "paper1" else W.one_ellipse_640()
    M0 = g.M[0]
    eta0 = np.zeros(M0) if case == "paper1" else g.zeta[:M0].imag.copy()
    om, _, _ = O.solve(O.surface_replaced(g, eta0), f, ph)
    gam0 = -O.d_alpha(om[:M0])
    _, gt, _, _ = O.vs_graph_rhs(g, f, eta0, gam0)
    et, pt, _, _ = O.graph_rhs(g, f, eta0, ph)

    def fd(h):
        o1, _, _ = O.solve(O.surface_replaced(g, eta0 + h * et), f, ph + h * pt)
        o2, _, _ = O.solve(O.surface_replaced(g, eta0 - h * et), f, ph - h * pt)
        return (O.d_alpha(o2[:M0]) - O.d_alpha(o1[:M0])) / (2 * h)

    a, b = fd(1e-3), fd(5e-4)
    ref = (4 * b - a) / 3
    return np.abs(gt - ref).max() / np.abs(ref).max()


@pytest.mark.parametrize("case", ["paper1", "one_ellipse_640"])
def test_gamma_t_is_the_time_derivative_of_gamma0(case):
    """Measured 2.3e-11 (problem 1 at rest) and 1.6e-10 (640 unknowns: moving surface,
    obstacle with circulation)."""
    assert _gamma_t_vs_fd(case) < 1e-9


@pytest.mark.parametrize("mutation", ["drop_gamma_sq", "W_without_jump", "F00_sign"])
def test_gamma_t_planted_mistakes(monkeypatch, mutation):
    orig_W, orig_B = O.vs_surface_W, O.vs_bernoulli
    if mutation == "drop_gamma_sq":
        monkeypatch.setattr(O, "vs_bernoulli", lambda Wx, Wy, t, V, g0, s, fo, F:
                            orig_B(Wx, Wy, t, V, g0, s, fo, F) + g0 ** 2 / (8 * s * s))
    elif mutation == "W_without_jump":
        monkeypatch.setattr(O, "vs_surface_W", lambda fb, g0, s, t: orig_W(fb, 0 * g0, s, t))
    else:
        monkeypatch.setattr(O, "vs_bernoulli", lambda Wx, Wy, t, V, g0, s, fo, F:
                            orig_B(Wx, Wy, t, V, g0, s, fo, -F))
    assert _gamma_t_vs_fd("one_ellipse_640") > 1e-6


def test_vs_evolution_matches_velocity_potential_evolution():
    """Problem 1 from rest, 3 RK4 steps of dt = 0.005 in both formulations: the
    surfaces agree to 9.5e-10 of max|eta| (the two ODE systems have different
    RK4 truncation errors) and gamma_0 = -omega_0' of the final VP state to 1e-9."""
    g, f, ph = W.paper_problem(1)
    M0 = g.M[0]
    om, _, _ = O.solve(g, f, ph)
    gam0 = -O.d_alpha(om[:M0])
    e_vp, p_vp, _ = O.evolve_graph(g, f, np.zeros(M0), ph, 0.005, 3)
    e_vs, gm = O.evolve_vs_graph(g, f, np.zeros(M0), gam0, 0.005, 3)
    om3, _, _ = O.solve(O.surface_replaced(g, e_vp), f, p_vp)
    assert np.abs(e_vp - e_vs).max() < 1e-8 * np.abs(e_vp).max()
    assert np.abs(gm + O.d_alpha(om3[:M0])).max() < 1e-8 * np.abs(gm).max()


# ---------------------------------------------------------------------------
# Phi~ in the fluid and on the boundaries (eq. w123; Sec. 4, Phi_t - C)
# ---------------------------------------------------------------------------

# points of Omega at least 0.15 from every boundary of both geometries below
_INTERIOR = np.array([0.5 - 0.3j, 1.0 - 0.3j, 1.5 - 0.3j, 4.5 - 0.35j, 1.0 - 0.75j, 5.5 - 0.7j])


def _phi_case(name):
    if name == "one_ellipse_640":
        return W.one_ellipse_640()
    return W.random_geometry(np.random.default_rng(2), 1001)


@pytest.mark.parametrize("name", ["one_ellipse_640", "random1001"])
def test_phi_tilde_at_derivative_is_the_velocity(name):
    """d/dz of the trapezoidal Cauchy integrals (central difference along x)
    equals the velocity sums of eqs. Phi:j:prime and Phi:0:prime, which are
    written with omega' after an integration by parts."""
    from types import SimpleNamespace
    g, f, ph = _phi_case(name)
    om = O.solve(g, f, ph)[0]
    zero = SimpleNamespace(V1=0.0, a=np.zeros(len(g.M) - 2))
    h = 1e-5
    d = (O.phi_tilde_at(g, om, _INTERIOR + h) - O.phi_tilde_at(g, om, _INTERIOR - h)) / (2 * h)
    v = O.velocity_far(g, zero, om, _INTERIOR)
    assert np.abs(d - v).max() < 1e-8 * np.abs(v).max()


@pytest.mark.parametrize("name", ["one_ellipse_640", "random1001"])
def test_phi_tilde_boundary_is_the_trace_of_phi_tilde(name):
    """Cauchy's formula over the positively oriented boundary (the free surface
    right to left, bottom and clockwise obstacles as given; eq. res:thm) applied
    to the boundary values reproduces Phi~ inside Omega: real and imaginary
    parts on every boundary form the trace of the analytic function of eq.
    w123.  The real part on the free surface is the Dirichlet data phi~."""
    g, f, ph = _phi_case(name)
    om = O.solve(g, f, ph)[0]
    gb = O.phi_tilde_boundary(g, om)
    ref = O.phi_tilde_at(g, om, _INTERIOR)
    assert np.abs(O.cauchy_sum(g, gb, _INTERIOR) - ref).max() < 1e-12 * np.abs(ref).max()
    assert np.abs(gb[0].real - ph).max() < 1e-12 * np.abs(ph).max()


@pytest.mark.parametrize("mutation", ["hilbert_sign", "no_hilbert"])
def test_phi_tilde_boundary_planted_mistakes(monkeypatch, mutation):
    orig = O.hilbert
    if mutation == "hilbert_sign":
        monkeypatch.setattr(O, "hilbert", lambda f: -orig(f))
    else:
        monkeypatch.setattr(O, "hilbert", lambda f: 0.0 * f)
    with pytest.raises(AssertionError):
        test_phi_tilde_boundary_is_the_trace_of_phi_tilde("one_ellipse_640")


@pytest.mark.parametrize("name", ["one_ellipse_640", "random1001"])
def test_helsing_ratio_of_the_plemelj_values_is_phi_tilde(name):
    """The Helsing-Ojala ratio (eq. helsing:quad) fed with the Plemelj boundary
    values of Phi~ reproduces the direct sums of eq. w123 inside the fluid: the
    interior pressure path (Phi_t - C at targets) rests on this."""
    g, f, ph = _phi_case(name)
    om = O.solve(g, f, ph)[0]
    ref = O.phi_tilde_at(g, om, _INTERIOR)
    got = O.helsing_eval(g, O.phi_tilde_boundary(g, om), _INTERIOR)
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


def test_phi_tilde_boundary_channel_closed_form():
    """Over a flat bottom y = -h, Phi~ = sum c_k cos(k(z + ih)) has psi~ = 0 on the
    bottom; solving with b_0 = Re Phi~(zeta_0), the Plemelj boundary values must
    be Phi~ itself on the surface and on the bottom (real part cos(kx)/cosh(kh)
    terms: the part of eq. w123 that the Plemelj formula adds)."""
    h = 1.3
    c = {1: 0.3, 2: -0.1, 3: 0.05}
    Phit = lambda z: sum(ck * np.cos(k * (z + 1j * h)) for k, ck in c.items())
    g = W.simple_channel(M0=128, M1=128, h=h)
    z0 = g.block(0)[0]
    om = O.solve(g, W.Flow(V1=0.0, a=np.array([])), np.real(Phit(z0)))[0]
    gb = O.phi_tilde_boundary(g, om)
    assert np.abs(gb[0] - Phit(z0)).max() < 1e-13
    assert np.abs(gb[1] - Phit(g.zeta[128:])).max() < 1e-13


@pytest.mark.parametrize("name", ["one_ellipse_640", "paper_problem1"])
def test_residual_update_error_model(name):
    """The refined solvers update late residuals as r - A_s d with a rounded copy
    A_s of the integral part K of the operator (the +-1/2 I applied exactly).
    The thresholds rest on this model: for independent roundings with unit
    roundoff u, ||(K - K_s) d|| is about u/sqrt(3) max_l ||K e_l|| ||d|| and never
    above u sqrt(sum_m (sum_l |K_ml| |d_l|)^2).  Checked here with FP32 and
    FP16 copies of the oracle's own matrix (K's column norms are the
    0.14-0.18 quoted for these systems)."""
    g, f, ph = W.paper_problem(1) if name == "paper_problem1" else W.one_ellipse_640()
    A = O.kernel_rows(g, np.arange(g.N))
    K = A - np.diag(np.diag(A))
    cmax = np.linalg.norm(K, axis=0).max()
    assert 0.1 < cmax < 0.2
    d = np.random.default_rng(3).standard_normal(g.N)
    for dt, u in ((np.float32, 2.0 ** -24), (np.float16, 2.0 ** -11)):
        Ks = K.astype(dt).astype(np.float64)
        err = np.linalg.norm((K - Ks) @ d)
        worst = u * np.linalg.norm(np.abs(K) @ np.abs(d))
        model = u / np.sqrt(3.0) * cmax * np.linalg.norm(d)
        assert err <= worst
        assert 0.1 * model < err < 3.0 * model, (dt, err / model)
