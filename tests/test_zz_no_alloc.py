"""The allocation-free normal velocity, checked against the context-based one
and the FP64 oracle.

bie_normal_velocity_static serves callers that cannot allocate device memory
(a caller-owned pool holding all of HBM, a loop that must not stall in
cudaMalloc, another runtime owning the device heap).  It keeps its scratch in
one fixed device array, so these checks run it twice in a row (the second call
sees the first call's leftovers) and compare both results with
bie_normal_velocity on the same density, within the 1e-12 relative bound the
other U tests use, and with the oracle's U.  A call after the first must leave
the device's free memory and torch's allocation count unchanged.  This file is
collected last so that a failure here cannot hide the other tests' results.
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
    if case == "one_ellipse_640":
        # against the oracle: the same density through eqs. d:phi:mv, d:phi:j, d:phi:0
        U_or = O.normal_velocity(g, f, om)
        assert np.linalg.norm(U - U_or) <= 1e-12 * np.linalg.norm(U_or)
        assert np.abs(psi[: g.nb - 2] - O.psi_k(g, om)).max() <= 1e-13


def test_static_call_allocates_nothing(P):
    """After a first call (which may load the module), a call changes neither
    the device's free memory nor torch's allocated bytes."""
    import torch
    g, f, ph = W.one_ellipse_640()
    zt = lambda a: torch.as_tensor(a, dtype=torch.complex128, device="cuda").contiguous()
    zeta, dzeta, d2zeta = zt(g.zeta), zt(g.dzeta), zt(g.d2zeta)
    om = torch.as_tensor(W.smooth_density(g), dtype=torch.float64, device="cuda")
    U = torch.empty(g.M[0], dtype=torch.float64, device="cuda")
    psi = torch.empty(g.nb - 2, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    P.bie_normal_velocity_static(g.M, zeta, dzeta, d2zeta, g.zc, f.V1, f.a, om, U, psi,
                                 stream=stream)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(3):
        P.bie_normal_velocity_static(g.M, zeta, dzeta, d2zeta, g.zc, f.V1, f.a, om, U, psi,
                                     stream=stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0


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
