"""Velocity on the boundaries and at targets (Sec. 5.1, eq. helsing:quad) vs the oracle.

Tolerances: boundary values are double-float sums (the same accuracy class as
U): 1e-11 relative.  Far targets use FP32 sums: 2e-5 relative to max|Phi'|.
Helsing targets use double-float sums over the boundary values: 1e-10
relative to max|Phi'| (the boundary values themselves carry ~1e-12).
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


def _ct(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.complex128, device="cuda")


def _near_targets(g, rng, n_per, dist_spacings):
    """Points at `dist_spacings` local node spacings from each boundary, on the fluid side."""
    o = O.offsets(g.M)
    pts = []
    for k in range(g.nb):
        zk, dzk = g.zeta[o[k]:o[k + 1]], g.dzeta[o[k]:o[k + 1]]
        idx = rng.choice(g.M[k], n_per, replace=False)
        h = np.abs(dzk[idx]) * 2 * np.pi / g.M[k]
        nrm = 1j * dzk[idx] / np.abs(dzk[idx])        # left normal
        side = -1.0 if k == 0 else 1.0                 # fluid below the surface, left of solids
        pts.append(zk[idx] + side * dist_spacings * h * nrm
                   + 0.3 * h * dzk[idx] / np.abs(dzk[idx]))
    return np.concatenate(pts)


def _interior_grid(g, n, clearance):
    """Uniform grid points of the fluid at least `clearance` from every node:
    below the surface, above the bottom, outside every ellipse."""
    xs = np.linspace(0.05, 2 * np.pi - 0.05, n)
    ys = np.linspace(-1.2, 0.2, n)
    Z = (xs[None, :] + 1j * ys[:, None]).ravel()
    o = O.offsets(g.M)

    def height(k, x):
        zk = g.zeta[o[k]:o[k + 1]]
        return np.interp(x, np.concatenate([zk.real, [zk.real[0] + 2 * np.pi]]),
                         np.concatenate([zk.imag, [zk.imag[0]]]))

    ok = (Z.imag < height(0, Z.real)) & (Z.imag > height(1, Z.real))
    for (x, y, q, b, th) in g.ellipses:
        w = (Z - (x + 1j * y)) * np.exp(-1j * th)
        ok &= (w.real / q) ** 2 + (w.imag / b) ** 2 > 1.0
    d_all = np.abs(Z[:, None] - g.zeta[None, :]).min(axis=1)
    return Z[ok & (d_all > clearance)]


@pytest.mark.parametrize("cfg", ["one_ellipse_640", "problem3"])
def test_boundary_velocity_matches_oracle(P, cfg):
    g, f, ph = W.one_ellipse_640() if cfg == "one_ellipse_640" else W.paper_problem(3)
    om, U, _ = O.solve(g, f, ph)
    ref = np.concatenate(O.boundary_dphi(g, f, om))
    prob = P.Problem(g, f, ph)
    try:
        import torch
        out = torch.empty(g.N, dtype=torch.complex128, device="cuda")
        P.bie_boundary_velocity(prob.ctx, torch.as_tensor(om, device="cuda"), out)
        got = out.cpu().numpy()
        assert np.linalg.norm(got - ref) <= 1e-11 * np.linalg.norm(ref)
        # on the surface the normal component is U (eq. phi:prime)
        dz0 = g.dzeta[: g.M[0]]
        assert np.abs(np.real(got[: g.M[0]] * 1j * dz0) / np.abs(dz0) - U).max() <= 1e-11
    finally:
        prob.close()


def test_far_and_helsing_targets_match_oracle(P):
    import torch
    g, f, ph = W.one_ellipse_640()
    om, _, _ = O.solve(g, f, ph)
    fb = O.boundary_dphi(g, f, om)
    rng = np.random.default_rng(2)
    zf = _interior_grid(g, 40, clearance=0.12)
    zn = _near_targets(g, rng, 12, 1.5)
    ref_far = O.velocity_far(g, f, om, zf)
    ref_near = O.helsing_eval(g, fb, zn)
    prob = P.Problem(g, f, ph)
    try:
        omt = torch.as_tensor(om, device="cuda")
        uv = torch.empty(len(zf), dtype=torch.complex128, device="cuda")
        P.bie_eval_velocity(prob.ctx, omt, _ct(zf), uv, mode=P.VEL_FAR)
        scale = np.abs(ref_far).max()
        assert np.abs(uv.cpu().numpy() - ref_far).max() <= 2e-5 * scale
        uvn = torch.empty(len(zn), dtype=torch.complex128, device="cuda")
        P.bie_eval_velocity(prob.ctx, omt, _ct(zn), uvn, mode=P.VEL_HELSING)
        assert np.abs(uvn.cpu().numpy() - ref_near).max() <= 1e-10 * np.abs(ref_near).max()
        # a target on a node returns the node value
        on = g.zeta[[3, 300, 600]]
        uvo = torch.empty(3, dtype=torch.complex128, device="cuda")
        P.bie_eval_velocity(prob.ctx, omt, _ct(on), uvo, mode=P.VEL_HELSING)
        fall = np.concatenate(fb)[[3, 300, 600]]
        assert np.abs(uvo.cpu().numpy() - fall).max() <= 1e-10 * np.abs(fall).max()
    finally:
        prob.close()


def test_exact_field_dtn_pair(P):
    """Flat bottom y = -h, Phi~ = sum c_k cos(k(z + ih)): the exact velocity is
    Phi'(z) = Phi~'(z) + V1 everywhere in the fluid (eq. uv:phi:phi:t)."""
    import torch
    h = 1.3
    c = {1: 0.3, 2: -0.1, 3: 0.05}
    Phit = lambda z: sum(ck * np.cos(k * (z + 1j * h)) for k, ck in c.items())
    dPhit = lambda z: sum(-ck * k * np.sin(k * (z + 1j * h)) for k, ck in c.items())
    f = W.Flow(V1=0.7, a=np.array([]))
    g = W.simple_channel(M0=256, M1=256, h=h)
    z0 = g.zeta[:256]
    prob = P.Problem(g, f, np.real(Phit(z0)))
    try:
        prob.assemble("fp32_ir")
        prob.solve(rtol=1e-14)
        rng = np.random.default_rng(3)
        x = rng.uniform(0, 2 * np.pi, 400)
        surf = np.interp(x, np.concatenate([z0.real, [2 * np.pi]]), np.concatenate([z0.imag, [z0.imag[0]]]))
        y = -h + (surf + h) * rng.uniform(0.15, 0.85, 400)
        zi = x + 1j * y
        zn = _near_targets(g, rng, 20, 1.0)
        exact_i = dPhit(zi) + f.V1
        exact_n = dPhit(zn) + f.V1
        uv = torch.empty(len(zi), dtype=torch.complex128, device="cuda")
        P.bie_eval_velocity(prob.ctx, prob.omega, _ct(zi), uv, mode=P.VEL_FAR)
        assert np.abs(uv.cpu().numpy() - exact_i).max() <= 2e-5 * np.abs(exact_i).max()
        uvh = torch.empty(len(zi), dtype=torch.complex128, device="cuda")
        P.bie_eval_velocity(prob.ctx, prob.omega, _ct(zi), uvh, mode=P.VEL_HELSING)
        assert np.abs(uvh.cpu().numpy() - exact_i).max() <= 1e-10 * np.abs(exact_i).max()
        uvn = torch.empty(len(zn), dtype=torch.complex128, device="cuda")
        P.bie_eval_velocity(prob.ctx, prob.omega, _ct(zn), uvn, mode=P.VEL_HELSING)
        assert np.abs(uvn.cpu().numpy() - exact_n).max() <= 1e-10 * np.abs(exact_n).max()
    finally:
        prob.close()


def test_auto_mode_classifies_by_spacing(P):
    import torch
    g, f, ph = W.one_ellipse_640()
    om, _, _ = O.solve(g, f, ph)
    rng = np.random.default_rng(4)
    zf = _interior_grid(g, 30, clearance=0.15)
    zn = _near_targets(g, rng, 10, 1.2)
    z = np.concatenate([zf, zn])
    # expected near set: nearest node closer than 4 local spacings
    h = np.abs(g.dzeta) * 2 * np.pi / np.asarray(g.M, float)[O.block_ids(g.M)]
    dn = (np.abs(z[:, None] - g.zeta[None, :]) / h[None, :]).min(axis=1)
    expect = int((dn < 4.0).sum())
    prob = P.Problem(g, f, ph)
    try:
        uv = torch.empty(len(z), dtype=torch.complex128, device="cuda")
        nn = P.bie_eval_velocity(prob.ctx, torch.as_tensor(om, device="cuda"), _ct(z), uv,
                                 mode=P.VEL_AUTO, near_spacings=4.0, count_near=True)
        assert abs(nn - expect) <= max(2, expect // 50)   # FP32 distance test at the threshold
        fb = O.boundary_dphi(g, f, om)
        got = uv.cpu().numpy()
        ref_n = O.helsing_eval(g, fb, zn)
        assert np.abs(got[len(zf):] - ref_n).max() <= 1e-10 * np.abs(ref_n).max()
        ref_f = O.velocity_far(g, f, om, zf)
        assert np.abs(got[: len(zf)] - ref_f).max() <= 2e-5 * np.abs(ref_f).max()
    finally:
        prob.close()
