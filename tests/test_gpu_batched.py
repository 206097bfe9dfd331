"""Batched solves (bie_batch_run) vs the oracle and vs single-problem solves.

Every problem of a batch is an ordinary system of eq. lin:sys, so the bounds
are those of the single-problem parity tests: relative 2-norm error of omega
and U within 1e-11 for the refined schemes (the oracle is dense FP64 LU).
The batch mixes sizes (ragged tails of the GEMV and vector units), obstacle
counts (0 to 4) and a problem of the paper's worked examples.
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


def _problems():
    rng = np.random.default_rng(17)
    probs = [W.one_ellipse_640()]
    for n in (701, 1001, 1536, 2049):
        probs.append(W.random_geometry(rng, n))
    g = W.simple_channel(M0=256, M1=144, h=1.2)
    probs.append((g, W.Flow(V1=0.9, a=np.array([])),
                  W.filtered_noise(np.random.default_rng(3), 256, 0.05, 16)))
    probs.append(W.paper_problem(3))
    return probs


@pytest.fixture(scope="module")
def refs():
    return [O.solve(g, f, ph) for g, f, ph in _problems()]


class Batch:
    def __init__(self, P, probs):
        import torch
        self.P = P
        self.probs = probs
        self.b = P.bie_batch_create(0, torch.cuda.current_stream())
        self.set_all(probs)

    def set_all(self, probs):
        import torch
        self.probs = probs
        zt = lambda a: torch.as_tensor(a, dtype=torch.complex128, device="cuda").contiguous()
        for p, (g, f, ph) in enumerate(probs):
            self.P.bie_batch_set_problem(self.b, p, g.M, zt(g.zeta), zt(g.dzeta), zt(g.d2zeta),
                                         g.zc, f.V1, f.a)
        self.phit = torch.as_tensor(np.concatenate([ph for _, _, ph in probs]), device="cuda")
        self.omega = torch.empty(sum(g.N for g, _, _ in probs), dtype=torch.float64, device="cuda")
        self.U = torch.empty(sum(g.M[0] for g, _, _ in probs), dtype=torch.float64, device="cuda")

    def run(self, prec="fp32_ir", **kw):
        o = self.P.bie_default_opts(**kw)
        return self.P.bie_batch_run(self.b, len(self.probs), self.phit, self.omega, self.U, prec, o)

    def split(self):
        om, U = self.omega.cpu().numpy(), self.U.cpu().numpy()
        out, i, j = [], 0, 0
        for g, _, _ in self.probs:
            out.append((om[i:i + g.N], U[j:j + g.M[0]]))
            i += g.N
            j += g.M[0]
        return out

    def close(self):
        self.P.bie_batch_destroy(self.b)


@pytest.mark.parametrize("prec", ["fp32_ir", "fp16_ir", "bf16_ir"])
def test_batch_matches_oracle(P, refs, prec):
    bt = Batch(P, _problems())
    try:
        infos = bt.run(prec)
        for k, ((om, U), (om_ref, U_ref, _), info) in enumerate(zip(bt.split(), refs, infos)):
            assert info.converged, k
            assert info.rel_resid <= 1e-14, (k, info.rel_resid)
            assert _rel(om, om_ref) <= 1e-11, (k, _rel(om, om_ref))
            assert _rel(U, U_ref) <= 1e-11, (k, _rel(U, U_ref))
    finally:
        bt.close()


@pytest.mark.parametrize("restart,itol", [(2, 0.0), (12, 1e-12)])
def test_batch_recycled_space_grows_and_caps(P, refs, restart, itol):
    """Short cycles grow each problem's recycled subspace a little at a time;
    full twelve-step cycles reach the 32-column cap, after which cycles keep
    the space; every problem still matches the oracle."""
    bt = Batch(P, _problems())
    try:
        infos = bt.run("fp32_ir", restart=restart, max_cycles=200, inner_tol=itol)
        for k, ((om, U), (om_ref, U_ref, _), info) in enumerate(zip(bt.split(), refs, infos)):
            assert info.converged and info.cycles >= 2, (k, info.as_dict())
            assert _rel(om, om_ref) <= 1e-11, (k, _rel(om, om_ref))
            assert _rel(U, U_ref) <= 1e-11, (k, _rel(U, U_ref))
    finally:
        bt.close()


def test_batch_matches_single_solves_and_replays_exactly(P):
    probs = _problems()
    bt = Batch(P, probs)
    try:
        bt.run("fp32_ir")
        first = [(om.copy(), U.copy()) for om, U in bt.split()]
        bt.run("fp32_ir")          # graph replay
        for (om1, U1), (om2, U2) in zip(first, bt.split()):
            assert np.array_equal(om1, om2) and np.array_equal(U1, U2)
        for (g, f, ph), (om, U) in zip(probs, first):
            prob = P.Problem(g, f, ph)
            try:
                prob.assemble("fp32_ir")
                prob.solve()
                assert _rel(om, prob.omega.cpu().numpy()) <= 1e-12
                assert _rel(U, prob.U.cpu().numpy()) <= 1e-11
            finally:
                prob.close()
    finally:
        bt.close()


def test_batch_geometry_update_recaptures(P):
    """Same sizes, moved obstacle and new flow: the run uses the new values."""
    probs = _problems()
    bt = Batch(P, probs)
    try:
        bt.run("fp32_ir")
        g, f, ph = probs[0]
        x, y, q, b, th = g.ellipses[0]
        e = (x + 0.2, y + 0.05, q, b, th + 0.3)
        surf = (g.zeta[: g.M[0]], g.dzeta[: g.M[0]], g.d2zeta[: g.M[0]])
        o = O.offsets(g.M)
        bot = (g.zeta[o[1]:o[2]], g.dzeta[o[1]:o[2]], g.d2zeta[o[1]:o[2]])
        g2 = W.assemble_geometry([surf, bot, W.ellipse(g.M[2], *e)], [e])
        f2 = W.Flow(V1=0.7, a=np.array([-0.4]))
        probs2 = [(g2, f2, ph)] + probs[1:]
        bt.set_all(probs2)
        infos = bt.run("fp32_ir")
        om_ref, U_ref, _ = O.solve(g2, f2, ph)
        om, U = bt.split()[0]
        assert infos[0].converged
        assert _rel(om, om_ref) <= 1e-11 and _rel(U, U_ref) <= 1e-11
    finally:
        bt.close()


def test_batch_autotuner_choice(P):
    """The first run times every GEMV unit size and keeps the fastest; the
    choice is reused (no retuning) while the problem sizes stay the same."""
    bt = Batch(P, _problems())
    try:
        assert P.bie_batch_tuning(bt.b)[0] == 0
        bt.run("fp32_ir")
        ub, ms = P.bie_batch_tuning(bt.b)
        cands = [256 << 10, 512 << 10, 1 << 20, 2 << 20, 4 << 20]
        assert ub in cands and all(t > 0 for t in ms)
        assert ms[cands.index(ub)] == min(ms)
        bt.run("fp32_ir")
        assert P.bie_batch_tuning(bt.b) == (ub, ms)
    finally:
        bt.close()


def test_batch_of_one(P, refs):
    g, f, ph = _problems()[0]
    bt = Batch(P, [(g, f, ph)])
    try:
        infos = bt.run("fp32_ir")
        om, U = bt.split()[0]
        assert infos[0].converged
        assert _rel(om, refs[0][0]) <= 1e-11 and _rel(U, refs[0][1]) <= 1e-11
    finally:
        bt.close()


def test_batch_errors(P):
    import torch
    probs = _problems()[:2]
    bt = Batch(P, probs)
    try:
        with pytest.raises(P.BieError) as e:
            bt.run("fp32_ir", restart=64)
        assert e.value.status == P.BIE_ERR_ARG
        with pytest.raises(P.BieError) as e:
            bt.run("fp64")
        assert e.value.status == P.BIE_ERR_ARG
        with pytest.raises(P.BieError) as e:
            P.bie_batch_run(bt.b, 3, bt.phit, bt.omega, bt.U, "fp32_ir")
        assert e.value.status == P.BIE_ERR_ARG
        big = W.simple_channel(M0=12288, M1=4104, h=1.0)
        zt = lambda a: torch.as_tensor(a, dtype=torch.complex128, device="cuda")
        with pytest.raises(P.BieError) as e:
            P.bie_batch_set_problem(bt.b, 2, big.M, zt(big.zeta), zt(big.dzeta), zt(big.d2zeta),
                                    big.zc, 1.0, [])
        assert e.value.status == P.BIE_ERR_ARG
        with pytest.raises(P.BieError) as e:   # problem 2 is not set
            P.bie_batch_run(bt.b, 3, bt.phit, bt.omega, bt.U, "fp32_ir")
        assert e.value.status == P.BIE_ERR_STATE
    finally:
        bt.close()


def test_grid_barrier_bounded_wait(P):
    """Without a stalled CTA every barrier is passed; with one CTA that never
    arrives, the others give up after their poll limit and report it."""
    import torch
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    st, passed, err = P.bie_test_grid_barrier(0, 1 << 16, -1)
    assert st == P.BIE_OK and err == 0 and passed == 3 * nsm
    st, passed, err = P.bie_test_grid_barrier(0, 1 << 14, 5)
    assert st == P.BIE_ERR_TIMEOUT and err == 1 and passed == 0
    # the device is still usable
    x = torch.ones(1000, device="cuda")
    assert float(x.sum()) == 1000.0


def test_random_batch_full(P):
    """The 96-problem workload (N ~ U{1024..12288}): every problem converges
    and solves the oracle's system on sampled rows (rows assembled by the
    oracle, residual relative to ||b||_inf), for the smallest, a middle and the
    largest problem."""
    probs = W.random_batch(seed=0)
    bt = Batch(P, probs)
    try:
        infos = bt.run("fp32_ir")
        assert all(i.converged for i in infos)
        sols = bt.split()
        Ns = np.array([g.N for g, _, _ in probs])
        for k in (int(np.argmin(Ns)), int(np.argsort(Ns)[len(Ns) // 2]), int(np.argmax(Ns))):
            g, f, ph = probs[k]
            b = O.rhs(g, f, ph)
            rows = np.random.default_rng(k).choice(g.N, 32, replace=False)
            rows = np.unique(np.concatenate([rows, g.offsets()[:-1], g.offsets()[1:] - 1]))
            r = b[rows] - O.kernel_rows(g, rows) @ sols[k][0]
            assert np.abs(r).max() <= 1e-12 * np.abs(b).max(), k
            tg = np.sort(np.random.default_rng(k + 1).choice(g.M[0], 16, replace=False))
            Uref = O.normal_velocity(g, f, sols[k][0], targets=tg)
            assert np.abs(sols[k][1][tg] - Uref).max() <= 1e-11 * np.abs(Uref).max(), k
    finally:
        bt.close()


@pytest.mark.parametrize("prec", ["fp16_ir", "fp32_ir", "bf16_ir"])
def test_batch_reported_residual_is_the_true_one(P, prec):
    """The batched solver's last residuals are updated from each problem's last
    increment (FP32 part, then the inner storage) once the residual allows it;
    what it reports must be the residual of the omega it returns, against the
    oracle's own FP64 matrix and right-hand side (relative 2-norm).  The GPU
    operator is assembled in double-float (about 2^-48 per entry), so the two
    operators' residuals of one omega differ by a few 1e-15 here; a residual
    updated from a wrong start would differ by orders of magnitude more."""
    probs = _problems()
    bt = Batch(P, probs)
    try:
        infos = bt.run(prec)
        for k, ((om, _), (g, f, ph), info) in enumerate(zip(bt.split(), probs, infos)):
            b = O.rhs(g, f, ph)
            A = O.kernel_rows(g, np.arange(g.N))
            true = float(np.linalg.norm(b - A @ om) / np.linalg.norm(b))
            assert info.converged and true <= 2e-14, (k, true, info.rel_resid)
            assert abs(true - info.rel_resid) <= 5e-15, (k, true, info.rel_resid)
        # one residual product per cycle, each reading 2 (inner FP16 / BF16 storage)
        # to 8 (hi + lo) bytes per stored entry
        ent = [i.cycles * g.N * (-(-g.N // 64) * 64) for (g, _, _), i in zip(probs, infos)]
        rb = P.bie_batch_resid_bytes(bt.b)
        lo = 4 if prec == "fp32_ir" else 2
        assert lo * sum(ent) <= rb <= 8 * sum(ent), (rb, sum(ent))
    finally:
        bt.close()
