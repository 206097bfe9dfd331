"""App. B variant on the GPU (psi prescribed on the solids, circulations a_j
unknown; eq. A:alt) vs the oracle.

Each system is an ordinary dense second-kind system, so the parity bounds are
those of the standard solve: omega and U within relative 1e-11 of the oracle's
dense LU solution; the a_j (means of omega) within 1e-11 of their size.
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


def _alt_data(g, f, ph):
    om, U, psik = O.solve(g, f, ph)
    M0 = g.M[0]
    o = O.offsets(g.M)
    phic = ph + sum(aj * O.phi_cyl(g.zeta[:M0] - zj) for aj, zj in zip(f.a, g.zc))
    psi_s = np.zeros(g.N - M0)
    for k in range(2, len(g.M)):
        psi_s[o[k] - M0:o[k + 1] - M0] = psik[k - 2]
    return om, U, phic, psi_s


CASES = [("one_ellipse_640", lambda: W.one_ellipse_640()), ("paper3", lambda: W.paper_problem(3)),
         ("ragged1001", lambda: W.random_geometry(np.random.default_rng(4), 1001))]


@pytest.mark.parametrize("prec", ["fp64", "fp32_ir", "fp16_ir"])
@pytest.mark.parametrize("name,make", CASES)
def test_psi_prescribed_matches_oracle(P, name, make, prec):
    import torch
    g, f, ph = make()
    om_std, U_std, phic, psi_s = _alt_data(g, f, ph)
    om_ref, U_ref, a_ref = O.solve_alt(g, f.V1, phic, psi_s)
    prob = P.Problem(g, f, ph)
    try:
        P.bie_assemble_psi(prob.ctx, prec)
        om = torch.empty(g.N, dtype=torch.float64, device="cuda")
        U = torch.empty(g.M[0], dtype=torch.float64, device="cuda")
        a, info = P.bie_solve_psi(prob.ctx, torch.as_tensor(phic, device="cuda"),
                                  torch.as_tensor(psi_s, device="cuda"), om, U, nobs=len(g.zc))
        assert info.converged
        assert _rel(om.cpu().numpy(), om_ref) <= 1e-11, (name, prec)
        assert _rel(U.cpu().numpy(), U_ref) <= 1e-11, (name, prec)
        assert np.abs(a - a_ref).max() <= 1e-11 * max(1.0, np.abs(a_ref).max())
        # the flow it describes is the standard solve's: same a_j and U
        assert np.abs(a - f.a).max() <= 1e-10 * max(1.0, np.abs(f.a).max())
        assert _rel(U.cpu().numpy(), U_std) <= 1e-11
    finally:
        prob.close()


def test_psi_prescribed_state_rules(P):
    """The App. B storage refuses the phi~-based solves; bie_assemble restores
    the standard operator (and its solve gives the standard answer)."""
    import torch
    g, f, ph = W.one_ellipse_640()
    om_std, U_std, phic, psi_s = _alt_data(g, f, ph)
    prob = P.Problem(g, f, ph)
    try:
        with pytest.raises(P.BieError) as e:      # not assembled for App. B
            P.bie_solve_psi(prob.ctx, torch.as_tensor(phic, device="cuda"),
                            torch.as_tensor(psi_s, device="cuda"), prob.omega)
        assert e.value.status == P.BIE_ERR_STATE
        P.bie_assemble_psi(prob.ctx, "fp32_ir")
        with pytest.raises(P.BieError) as e:
            prob.solve()
        assert e.value.status == P.BIE_ERR_STATE
        prob.assemble("fp32_ir")
        prob.solve()
        assert _rel(prob.U.cpu().numpy(), U_std) <= 1e-11
        with pytest.raises(P.BieError) as e:      # the standard storage refuses App. B
            P.bie_solve_psi(prob.ctx, torch.as_tensor(phic, device="cuda"),
                            torch.as_tensor(psi_s, device="cuda"), prob.omega)
        assert e.value.status == P.BIE_ERR_STATE
    finally:
        prob.close()
