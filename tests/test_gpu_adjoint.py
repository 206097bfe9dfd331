"""Backward pass (bie_backward, solve_u) vs the oracle's forward-mode derivatives.

The oracle differentiates the forward map along a direction v of the inputs
(node data, centres, phi~) by hand and returns dU(v); the GPU returns the
cotangents g of J = gU . U.  For every v the two sides must agree on
  gU . dU(v)  =  <g, v>  =  sum Re(conj(g_n) v_n) + g_phit . dphit.
Directions: seeded band-limited vectors in all inputs (raw cotangents), the
five parameters of every ellipse (g_shape, analytic derivatives of the
ellipse), and surface-node moves with zeta', zeta'' following spectrally
(g_node).  Errors are measured against ||gU|| ||dU(v)||, the size of the
terms of the inner product.

Tolerance 1e-11 of that scale: the gradient carries the conditioning of U
itself (spectral derivatives amplify mode k by k; the forward U parity at these
sizes is held to the same 1e-11), through one more solve at rtol 1e-14.
Measured: <= 1.4e-13 for the raw and node pairings, <= 8.3e-13 for the
ellipse parameters (FP64 and FP32-IR storage, 640 to 4096 unknowns).
"""
import numpy as np
import pytest

import workloads as W
from oracle import bie as O

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-11, "fp32_ir": 1e-11}


@pytest.fixture(scope="module")
def P():
    import paper_2108_01786_gb300 as P
    from paper_2108_01786_gb300 import _build
    _build.build()
    return P


def _ragged():
    return W.random_geometry(np.random.default_rng(3), 1001)


def ellipse_directions(g):
    """One direction per (x, y, q, b, theta) of every ellipse: the analytic
    derivatives of zeta = z_j + e^{i theta}(q cos a - i b sin a) and of its
    first two alpha-derivatives; x and y also move the centre in Phi_mv."""
    o = O.offsets(g.M)
    dirs = []
    for j, (x, y, q, b, th) in enumerate(g.ellipses):
        k = j + 2
        sl = slice(o[k], o[k + 1])
        a = W.alphas(g.M[k])
        r = np.exp(1j * th)
        ca, sa = np.cos(a), np.sin(a)
        for p in range(5):
            dz = np.zeros(g.N, complex)
            ddz = np.zeros(g.N, complex)
            dd2z = np.zeros(g.N, complex)
            dzc = np.zeros(len(g.zc), complex)
            if p == 0:
                dz[sl], dzc[j] = 1.0, 1.0
            elif p == 1:
                dz[sl], dzc[j] = 1j, 1j
            elif p == 2:
                dz[sl], ddz[sl], dd2z[sl] = r * ca, -r * sa, -r * ca
            elif p == 3:
                dz[sl], ddz[sl], dd2z[sl] = -1j * r * sa, -1j * r * ca, 1j * r * sa
            else:
                dz[sl] = 1j * (g.zeta[sl] - g.zc[j])
                ddz[sl], dd2z[sl] = 1j * g.dzeta[sl], 1j * g.d2zeta[sl]
            dirs.append((dz, ddz, dd2z, dzc, np.zeros(g.M[0])))
    return dirs


def surface_node_directions(g, n, seed):
    """Moves of the surface nodes with zeta', zeta'' their spectral derivatives."""
    rng = np.random.default_rng(seed)
    M0 = g.M[0]
    dirs = []
    for _ in range(n):
        v = W.filtered_noise(rng, M0, 1e-2, 16) + 1j * W.filtered_noise(rng, M0, 1e-2, 16)
        dv = O.d_alpha(v.real) + 1j * O.d_alpha(v.imag)
        d2v = O.d_alpha(dv.real) + 1j * O.d_alpha(dv.imag)
        z = np.zeros(g.N, complex)
        dz, ddz, dd2z = z.copy(), z.copy(), z.copy()
        dz[:M0], ddz[:M0], dd2z[:M0] = v, dv, d2v
        dirs.append((dz, ddz, dd2z, np.zeros(len(g.zc), complex), np.zeros(M0)))
    return dirs


def _ip(a, b):
    return float(np.sum(a.real * b.real + a.imag * b.imag))


def _run_backward(P, g, f, ph, prec, gU, with_shape=True):
    import torch
    prob = P.Problem(g, f, ph)
    try:
        prob.assemble(prec)
        info = prob.solve()
        assert info.converged
        dev = prob.omega.device
        out = {k: torch.empty(g.N, dtype=torch.complex128, device=dev)
               for k in ("g_zeta", "g_dzeta", "g_d2zeta", "g_node")}
        nobs = len(g.M) - 2
        out["g_zc"] = torch.empty(max(nobs, 1), dtype=torch.complex128, device=dev)
        out["g_phit"] = torch.empty(g.M[0], dtype=torch.float64, device=dev)
        out["g_shape"] = torch.empty(max(5 * nobs, 1), dtype=torch.float64, device=dev)
        out["lam"] = torch.empty(g.N, dtype=torch.float64, device=dev)
        ell = np.array(g.ellipses, dtype=np.float64) if nobs else None
        binfo = P.bie_backward(prob.ctx, prob.omega, torch.as_tensor(gU, device=dev), ell, **out)
        assert binfo.converged
        res = {k: v.cpu().numpy() for k, v in out.items()}
        res["g_zc"] = res["g_zc"][:nobs]
        res["g_shape"] = res["g_shape"][: 5 * nobs]
        res["omega"] = prob.omega.cpu().numpy()
        return res
    finally:
        prob.close()


def _raw_pairing(res, d):
    dz, ddz, dd2z, dzc, dphit = d
    return (_ip(res["g_zeta"], dz) + _ip(res["g_dzeta"], ddz) + _ip(res["g_d2zeta"], dd2z)
            + _ip(res["g_zc"], dzc) + float(res["g_phit"] @ dphit))


@pytest.mark.parametrize("prec", ["fp64", "fp32_ir"])
@pytest.mark.parametrize("case", ["one_ellipse_640", "ragged"])
def test_raw_cotangents_match_oracle(P, prec, case):
    g, f, ph = W.one_ellipse_640() if case == "one_ellipse_640" else _ragged()
    gU = W.filtered_noise(np.random.default_rng(11), g.M[0], 1.0, 40)
    res = _run_backward(P, g, f, ph, prec, gU)
    dirs = [W.adjoint_direction(g, seed=s) for s in range(8)]
    U, dUs = O.directional_U_many(g, f, ph, dirs)
    for d, dU in zip(dirs, dUs):
        want = float(gU @ dU)
        got = _raw_pairing(res, d)
        scale = np.linalg.norm(gU) * np.linalg.norm(dU)
        assert abs(got - want) <= TOL[prec] * scale, (got, want, scale)


@pytest.mark.parametrize("prec", ["fp64", "fp32_ir"])
def test_shape_and_node_gradients_match_oracle(P, prec):
    g, f, ph = _ragged()
    om, U, _ = O.solve(g, f, ph)
    gU = 2 * 2 * np.pi / g.M[0] * U          # J = (2 pi/M_0) sum U^2
    res = _run_backward(P, g, f, ph, prec, gU)
    edirs = ellipse_directions(g)
    ndirs = surface_node_directions(g, 4, seed=21)
    _, dUs = O.directional_U_many(g, f, ph, edirs + ndirs)
    for i, dU in enumerate(dUs[: len(edirs)]):
        want = float(gU @ dU)
        scale = np.linalg.norm(gU) * np.linalg.norm(dU)
        assert abs(res["g_shape"][i] - want) <= TOL[prec] * scale, (i, res["g_shape"][i], want)
    for d, dU in zip(ndirs, dUs[len(edirs):]):
        want = float(gU @ dU)
        got = _ip(res["g_node"], d[0])
        scale = np.linalg.norm(gU) * np.linalg.norm(dU)
        assert abs(got - want) <= TOL[prec] * scale, (got, want)


def test_phitilde_gradient_is_adjoint_density(P):
    """dJ/dphi~ = lambda on the surface, and lambda solves A^T lambda = omegabar:
    checked against the oracle's dense transpose solve."""
    g, f, ph = W.one_ellipse_640()
    gU = W.filtered_noise(np.random.default_rng(12), g.M[0], 1.0, 30)
    res = _run_backward(P, g, f, ph, "fp64", gU)
    A = O.assemble(g)
    # omegabar = (dU/domega)^T gU column by column from the oracle's U map (linear in omega)
    om = res["omega"]
    z = np.zeros(g.N)
    U0 = O.normal_velocity(g, f, z)
    J = np.stack([O.normal_velocity(g, f, np.eye(g.N)[i]) - U0 for i in range(g.N)], axis=1)
    lam = np.linalg.solve(A.T, J.T @ gU)
    assert np.abs(res["lam"] - lam).max() <= 1e-10 * np.abs(lam).max()
    assert np.abs(res["g_phit"] - lam[: g.M[0]]).max() <= 1e-10 * np.abs(lam).max()
    assert np.isfinite(om).all()


def test_autograd_solve_u(P):
    """J = (2 pi/M_0) sum U^2 through torch autograd: the gradients of the node
    data equal bie_backward's, and match the oracle along a direction."""
    import torch
    g, f, ph = W.one_ellipse_640()
    dev = torch.device("cuda", 0)
    zeta = torch.tensor(g.zeta, dtype=torch.complex128, device=dev, requires_grad=True)
    dzeta = torch.tensor(g.dzeta, dtype=torch.complex128, device=dev, requires_grad=True)
    d2zeta = torch.tensor(g.d2zeta, dtype=torch.complex128, device=dev, requires_grad=True)
    zc = torch.tensor(g.zc, dtype=torch.complex128, requires_grad=True)
    phit = torch.tensor(ph, dtype=torch.float64, device=dev, requires_grad=True)
    solver = P.Solver(g.M, f.V1, f.a, precision="fp32_ir")
    try:
        U = P.solve_u(zeta, dzeta, d2zeta, zc, phit, solver)
        J = 2 * np.pi / g.M[0] * (U * U).sum()
        J.backward()
        d = W.adjoint_direction(g, seed=4)
        dJ = O.directional_objective(g, f, ph, *d)
        got = (_ip(zeta.grad.cpu().numpy(), d[0]) + _ip(dzeta.grad.cpu().numpy(), d[1])
               + _ip(d2zeta.grad.cpu().numpy(), d[2]) + _ip(zc.grad.numpy(), d[3])
               + float(phit.grad.cpu().numpy() @ d[4]))
        Uo = O.solve(g, f, ph)[1]
        _, dU = O.directional_U(g, f, ph, *d)
        scale = 2 * 2 * np.pi / g.M[0] * np.linalg.norm(Uo) * np.linalg.norm(dU)
        assert abs(got - dJ) <= 1e-11 * scale
    finally:
        solver.close()


def test_state_after_backward(P):
    """After a backward pass the storage holds the adjoint operator: solve and
    matvec refuse until the next assemble; normal velocity still works."""
    import torch
    g, f, ph = W.one_ellipse_640()
    prob = P.Problem(g, f, ph)
    try:
        prob.assemble("fp32_ir")
        prob.solve()
        gU = torch.ones(g.M[0], dtype=torch.float64, device="cuda")
        P.bie_backward(prob.ctx, prob.omega, gU)
        with pytest.raises(P.BieError) as e:
            prob.solve()
        assert e.value.status == P.BIE_ERR_STATE
        with pytest.raises(P.BieError):
            P.bie_matvec(prob.ctx, 0, prob.omega, torch.empty_like(prob.omega))
        U = torch.empty(g.M[0], dtype=torch.float64, device="cuda")
        P.bie_normal_velocity(prob.ctx, prob.omega, U)
        assert np.abs(U.cpu().numpy() - prob.U.cpu().numpy()).max() <= 1e-13
        prob.assemble("fp32_ir")
        assert prob.solve().converged
        with pytest.raises(P.BieError) as e2:
            P.bie_backward(prob.ctx, prob.omega, gU, None,
                           g_shape=torch.empty(5, dtype=torch.float64, device="cuda"))
        assert e2.value.status == P.BIE_ERR_ARG
    finally:
        prob.close()


def test_backward_without_obstacles(P):
    """Surface and bottom only: no centres, no shape gradient; the raw
    cotangents still match the oracle."""
    g = W.simple_channel(M0=200, M1=136, h=1.1)
    f = W.Flow(V1=0.8, a=np.array([]))
    ph = W.filtered_noise(np.random.default_rng(2), 200, 0.1, 12)
    gU = W.filtered_noise(np.random.default_rng(13), 200, 1.0, 30)
    res = _run_backward(P, g, f, ph, "fp64", gU)
    dirs = [W.adjoint_direction(g, seed=s) for s in range(3)]
    _, dUs = O.directional_U_many(g, f, ph, dirs)
    for d, dU in zip(dirs, dUs):
        want = float(gU @ dU)
        scale = np.linalg.norm(gU) * np.linalg.norm(dU)
        assert abs(_raw_pairing(res, d) - want) <= 1e-11 * scale


def surface_node_coordinate_directions(g, n_nodes, seed):
    """Moves of single surface nodes, x or y, with zeta' and zeta'' following
    as the spectral derivatives of zeta - alpha (the node parametrisation of
    the gradient g_node): 2 n_nodes directions at seeded nodes."""
    rng = np.random.default_rng(seed)
    M0 = g.M[0]
    nodes = np.sort(rng.choice(M0, n_nodes, replace=False))
    dirs, picks = [], []
    for n in nodes:
        e = np.zeros(M0)
        e[n] = 1.0
        De = O.d_alpha(e)
        D2e = O.d_alpha(De)
        for c in (1.0, 1j):
            dz = np.zeros(g.N, complex)
            ddz, dd2z = dz.copy(), dz.copy()
            dz[:M0], ddz[:M0], dd2z[:M0] = c * e, c * De, c * D2e
            dirs.append((dz, ddz, dd2z, np.zeros(len(g.zc), complex), np.zeros(M0)))
            picks.append((int(n), c))
    return dirs, picks


@pytest.fixture(scope="module")
def config4():
    """two_ellipses_4096 (2048 + 1024 + 512 + 512 unknowns) with the oracle's
    forward-mode derivatives of U along the 10 ellipse parameters and 64
    single surface-node coordinates, and gU = dJ/dU for J = (2 pi/M_0) sum U^2."""
    g, f, ph = W.two_ellipses_4096()
    om, U, _ = O.solve(g, f, ph)
    gU = 2 * 2 * np.pi / g.M[0] * U
    edirs = ellipse_directions(g)
    ndirs, picks = surface_node_coordinate_directions(g, 32, seed=40)
    _, dUs = O.directional_U_many(g, f, ph, edirs + ndirs)
    want = np.array([float(gU @ dU) for dU in dUs])
    scale = np.array([np.linalg.norm(gU) * np.linalg.norm(dU) for dU in dUs])
    return dict(g=g, f=f, ph=ph, gU=gU, picks=picks,
                want_shape=want[:10], scale_shape=scale[:10],
                want_node=want[10:], scale_node=scale[10:])


def _node_values(g_node, picks):
    return np.array([g_node[n].real if c == 1.0 else g_node[n].imag for n, c in picks])


@pytest.mark.parametrize("prec", ["fp64", "fp32_ir"])
def test_config4_gradient_matches_oracle(P, config4, prec):
    """Config 4 at its own size: g_shape (x, y, q, b, theta of both ellipses)
    and g_node at 64 seeded surface-node coordinates against the oracle's
    forward-mode derivatives, within 1e-11 of ||gU|| ||dU(v)|| as above."""
    c = config4
    res = _run_backward(P, c["g"], c["f"], c["ph"], prec, c["gU"])
    err_s = np.abs(res["g_shape"] - c["want_shape"]) / c["scale_shape"]
    assert err_s.max() <= TOL[prec], (err_s, res["g_shape"], c["want_shape"])
    got_n = _node_values(res["g_node"], c["picks"])
    err_n = np.abs(got_n - c["want_node"]) / c["scale_node"]
    assert err_n.max() <= TOL[prec], (err_n.max(), int(err_n.argmax()))


def test_config4_gradient_matches_central_differences(P, config4):
    """Config 4: g_shape (10 parameters) and g_node (64 surface-node
    coordinates) against central differences of the GPU's own J = (2 pi/M_0)
    sum U^2 at h = 1e-6, FP64 storage.  A moved ellipse is rebuilt
    analytically; a moved surface node takes its zeta' and zeta'' as spectral
    derivatives of zeta - alpha.

    Bound: the truncation error h^2 J'''/6 is ~1e-12 relative here; the
    differences are limited by the non-smooth rounding of J itself, at most
    ~1e-13 |J| per evaluation (the solve stops at rtol 1e-14 and U amplifies
    the error of omega by its highest mode), so |FD - g| <= 4e-13 |J| / h
    (two evaluations, a factor 2 margin) plus 1e-6 |g|."""
    import torch
    c = config4
    g, f, ph = c["g"], c["f"], c["ph"]
    M0 = g.M[0]
    o = O.offsets(g.M)
    h = 1e-6
    base = [(g.zeta[o[k]:o[k + 1]], g.dzeta[o[k]:o[k + 1]], g.d2zeta[o[k]:o[k + 1]]) for k in (0, 1)]
    ells = [tuple(e) for e in g.ellipses]

    def J_of(gg):
        prob = P.Problem(gg, f, ph)
        try:
            prob.assemble("fp64")
            assert prob.solve().converged
            U = prob.U.cpu().numpy()
            return 2 * np.pi / M0 * float(U @ U)
        finally:
            prob.close()

    def shape_moved(j, p, t):
        e = [list(x) for x in ells]
        e[j][p] += t
        return W.assemble_geometry(base + [W.ellipse(g.M[2 + k], *x) for k, x in enumerate(e)],
                                   [tuple(x) for x in e])

    def node_moved(n, cc, t):
        a = W.alphas(M0)
        r = (g.zeta[:M0] - a).copy()
        r[n] += t * cc
        dr = O.d_alpha(r.real) + 1j * O.d_alpha(r.imag)
        d2r = O.d_alpha(dr.real) + 1j * O.d_alpha(dr.imag)
        return W.assemble_geometry([(a + r, 1.0 + dr, d2r), base[1]]
                                   + [W.ellipse(g.M[2 + k], *x) for k, x in enumerate(ells)], ells)

    prob = P.Problem(g, f, ph)
    try:
        prob.assemble("fp64")
        assert prob.solve().converged
        U = prob.U.cpu().numpy()
        J0 = 2 * np.pi / M0 * float(U @ U)
        dev = prob.omega.device
        gU = torch.as_tensor(2 * 2 * np.pi / M0 * U, device=dev)
        gs = torch.empty(10, dtype=torch.float64, device=dev)
        gn = torch.empty(g.N, dtype=torch.complex128, device=dev)
        P.bie_backward(prob.ctx, prob.omega, gU, np.array(ells), g_shape=gs, g_node=gn)
        grad_s = gs.cpu().numpy()
        grad_n = _node_values(gn.cpu().numpy(), c["picks"])
    finally:
        prob.close()
    bound = 4e-13 * abs(J0) / h
    fd_s = np.array([(J_of(shape_moved(j, p, h)) - J_of(shape_moved(j, p, -h))) / (2 * h)
                     for j in range(2) for p in range(5)])
    err_s = np.abs(grad_s - fd_s)
    assert np.all(err_s <= bound + 1e-6 * np.abs(grad_s)), (err_s, bound)
    fd_n = np.array([(J_of(node_moved(n, cc, h)) - J_of(node_moved(n, cc, -h))) / (2 * h)
                     for n, cc in c["picks"]])
    err_n = np.abs(grad_n - fd_n)
    assert np.all(err_n <= bound + 1e-6 * np.abs(grad_n)), (err_n.max(), bound)
