"""The allocation-free normal velocity, checked against the context-based one.

bie_normal_velocity_static serves callers that cannot allocate device memory
(a caller-owned pool holding all of HBM, a loop that must not stall in
cudaMalloc, another runtime owning the device heap).  It keeps its scratch in
one fixed device array, so these checks run it twice in a row (the second call
sees the first call's leftovers) and compare both results with
bie_normal_velocity on the same density, within the 1e-12 relative bound the
other U tests use.  This file is collected last so that a failure here cannot
hide the other tests' results.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2108_01786_gb300 as P
    from paper_2108_01786_gb300 import _build
    _build.build()
    return P


def _case(name):
    if name == "one_ellipse_640":
        return W.one_ellipse_640()
    if name == "two_ellipses_4096":
        return W.two_ellipses_4096()
    return W.paper_problem(3)


@pytest.mark.parametrize("case", ["one_ellipse_640", "problem3", "two_ellipses_4096"])
def test_static_matches_context_velocity(P, case):
    import torch
    g, f, ph = _case(case)
    rng = np.random.default_rng(11)
    # any smooth density will do; add a little noise so every mode is exercised
    om = np.concatenate([np.cos(np.arange(m) * 2 * np.pi / m * (k + 1)) for k, m in enumerate(g.M)])
    om = om + 1e-3 * rng.standard_normal(g.N)
    zt = lambda a: torch.as_tensor(a, dtype=torch.complex128, device="cuda").contiguous()
    zeta, dzeta, d2zeta = zt(g.zeta), zt(g.dzeta), zt(g.d2zeta)
    omt = torch.as_tensor(om, dtype=torch.float64, device="cuda")
    npsi = max(1, g.nb - 2)
    # reference: the context-based entry point
    prob = P.Problem(g, f, ph)
    try:
        U_ref = torch.empty(g.M[0], dtype=torch.float64, device="cuda")
        psi_ref = torch.empty(npsi, dtype=torch.float64, device="cuda")
        P.bie_normal_velocity(prob.ctx, omt, U_ref, psi_ref)
        torch.cuda.synchronize()
        U_ref, psi_ref = U_ref.cpu().numpy(), psi_ref.cpu().numpy()
    finally:
        prob.close()
    stream = torch.cuda.current_stream()
    for call in range(2):
        U = torch.full((g.M[0],), float("nan"), dtype=torch.float64, device="cuda")
        psi = torch.full((npsi,), float("nan"), dtype=torch.float64, device="cuda")
        P.bie_normal_velocity_static(g.M, zeta, dzeta, d2zeta, g.zc, f.V1, f.a, omt, U, psi,
                                     stream=stream)
        torch.cuda.synchronize()
        U, psi = U.cpu().numpy(), psi.cpu().numpy()
        assert np.linalg.norm(U - U_ref) <= 1e-12 * np.linalg.norm(U_ref), (case, call)
        if g.nb > 2:
            assert np.abs(psi[: g.nb - 2] - psi_ref[: g.nb - 2]).max() <= 1e-13, (case, call)


def test_static_rejects_sizes_beyond_limit(P):
    import torch
    g, f, ph = W.three_ellipses_16383()          # 16383 unknowns > 8192
    assert g.N > P.STATIC_MAXN
    zt = lambda a: torch.as_tensor(a, dtype=torch.complex128, device="cuda").contiguous()
    om = torch.zeros(g.N, dtype=torch.float64, device="cuda")
    U = torch.zeros(g.M[0], dtype=torch.float64, device="cuda")
    with pytest.raises(P.BieError) as ei:
        P.bie_normal_velocity_static(g.M, zt(g.zeta), zt(g.dzeta), zt(g.d2zeta), g.zc, f.V1, f.a,
                                     om, U)
    assert ei.value.status == P.BIE_ERR_ARG
