"""Row-partitioned operator (bie_set_partition) on one GPU: the parts run as
separate contexts driven by separate host threads, and their exchange is an
in-process allgather / allreduce between the parts' staging buffers with host
barriers (no kernel waits on another; each part synchronises its own stream
before a barrier).  Checks: every product of the partitioned storage equals
the unpartitioned one bit for bit (each row is summed in the same order), the
parts agree with each other exactly, and the partitioned solve matches the
unpartitioned solve and the FP64 oracle."""
import threading

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


class ThreadExchange:
    """Allgather / allreduce among `n` contexts of one process, one host
    thread each."""

    def __init__(self, n):
        self.n = n
        self.barrier = threading.Barrier(n, timeout=120)
        self.stages = [None] * n
        self.streams = [None] * n

    def member(self, p, stage, stream):
        import torch
        self.stages[p], self.streams[p] = stage, stream

        def exchange(op, count, elem_bytes, _stream):
            st = self.streams[p]
            st.synchronize()                       # own segment in place
            self.barrier.wait()
            if op == 0:
                dt = torch.float32 if elem_bytes == 4 else torch.float64
                mine = self.stages[p].view(dt)
                with torch.cuda.stream(st):
                    for q in range(self.n):
                        if q != p:
                            mine[q * count:(q + 1) * count].copy_(
                                self.stages[q].view(dt)[q * count:(q + 1) * count])
                st.synchronize()
                self.barrier.wait()               # nobody overwrites a stage still being read
            else:
                with torch.cuda.stream(st):
                    tot = sum(self.stages[q].view(torch.float64)[:count].clone()
                              for q in range(self.n))
                st.synchronize()
                self.barrier.wait()
                with torch.cuda.stream(st):
                    self.stages[p].view(torch.float64)[:count].copy_(tot)
                st.synchronize()
                self.barrier.wait()
            return 0
        return exchange


def _run_part(P, g, f, ph, prec, nparts, p, ex, x, out, errs):
    import torch
    try:
        dev = torch.device("cuda", 0)
        st = torch.cuda.Stream(dev)
        with torch.cuda.stream(st):
            zt = lambda a: torch.as_tensor(a, dtype=torch.complex128, device=dev).contiguous()
            zeta, dzeta, d2zeta = zt(g.zeta), zt(g.dzeta), zt(g.d2zeta)
            ctx = P.bie_create(0, st)
            try:
                P.bie_set_geometry(ctx, g.M, zeta, dzeta, d2zeta, g.zc)
                P.bie_set_flow(ctx, f.V1, f.a)
                if nparts > 1:
                    stage = torch.empty(P.partition_stage_bytes(g.N, nparts), dtype=torch.uint8,
                                        device=dev)
                    P.bie_set_partition(ctx, nparts, p, stage, ex.member(p, stage, st))
                out["rows"] = P.bie_partition_rows(ctx)
                P.bie_assemble(ctx, P.PRECISIONS[prec])
                xt = torch.as_tensor(x, device=dev)
                for which in (0, 1):
                    y = torch.empty(g.N, dtype=torch.float64, device=dev)
                    P.bie_matvec(ctx, which, xt, y)
                    st.synchronize()
                    out[f"mv{which}"] = y.cpu().numpy()
                omega = torch.zeros(g.N, dtype=torch.float64, device=dev)
                U = torch.zeros(g.M[0], dtype=torch.float64, device=dev)
                psi = torch.zeros(max(1, g.nb - 2), dtype=torch.float64, device=dev)
                info = P.bie_solve(ctx, torch.as_tensor(ph, device=dev), omega, U, psi)
                st.synchronize()
                out.update(omega=omega.cpu().numpy(), U=U.cpu().numpy(),
                           psi=psi.cpu().numpy()[: max(0, g.nb - 2)], iters=info.iters,
                           resid=info.rel_resid)
                # backward pass of J = (2 pi/M_0) sum U^2: the local rows of S^T and the
                # parts' V^T Nbar added by the allreduce
                gU = torch.as_tensor(2 * 2 * np.pi / g.M[0] * out["U"], device=dev)
                gn = torch.empty(g.N, dtype=torch.complex128, device=dev)
                nobs = g.nb - 2
                gs = torch.empty(max(1, 5 * nobs), dtype=torch.float64, device=dev)
                ell = np.array(g.ellipses, dtype=np.float64) if nobs else None
                P.bie_backward(ctx, omega, gU, ell, g_node=gn, g_shape=gs if nobs else None)
                st.synchronize()
                out.update(g_node=gn.cpu().numpy(), g_shape=gs.cpu().numpy()[: 5 * nobs])
                if nparts > 1:   # entry points that do not follow the partition refuse
                    with pytest.raises(P.BieError) as e:
                        P.bie_assemble_psi(ctx, P.BIE_FP32_IR)
                    out["refused"] = e.value.status
            finally:
                P.bie_destroy(ctx)
    except BaseException as e:   # reported by the main thread
        errs.append(e)
        if nparts > 1:
            ex.barrier.abort()


def _partitioned(P, g, f, ph, prec, nparts, x):
    ex = ThreadExchange(nparts)
    outs = [dict() for _ in range(nparts)]
    errs = []
    th = [threading.Thread(target=_run_part, args=(P, g, f, ph, prec, nparts, p, ex, x, outs[p], errs))
          for p in range(nparts)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=300)
    assert not errs, errs
    return outs


@pytest.mark.parametrize("case,prec,nparts", [("one_ellipse_640", "fp16_ir", 2),
                                              ("one_ellipse_640", "fp64", 2),
                                              ("ragged", "fp32_ir", 3)])
def test_partitioned_products_and_solve(P, case, prec, nparts):
    g, f, ph = (W.one_ellipse_640() if case == "one_ellipse_640"
                else W.random_geometry(np.random.default_rng(3), 1001))
    x = W.smooth_density(g, seed=5)
    ref = {}
    _run_part(P, g, f, ph, prec, 1, 0, None, x, ref, [])
    outs = _partitioned(P, g, f, ph, prec, nparts, x)
    # every part holds its own rows, all rows once
    rows = [o["rows"] for o in outs]
    assert [r[:2] for r in rows] == [P.partition_rows(g.N, nparts, p)[:2] for p in range(nparts)]
    assert rows[0][0] == 0 and rows[-1][1] == g.N
    assert all(rows[p][1] == rows[p + 1][0] for p in range(nparts - 1))
    for o in outs:
        # products: the same per-row arithmetic as the unpartitioned storage
        assert np.array_equal(o["mv1"], ref["mv1"])
        assert np.array_equal(o["mv0"], ref["mv0"])
        # every part follows the same iteration
        assert np.array_equal(o["omega"], outs[0]["omega"]) and np.array_equal(o["U"], outs[0]["U"])
        assert o["refused"] == P.BIE_ERR_STATE
    om_o, U_o, psi_o = O.solve(g, f, ph)
    o = outs[0]
    assert np.linalg.norm(o["omega"] - ref["omega"]) <= 1e-12 * np.linalg.norm(ref["omega"])
    assert np.linalg.norm(o["U"] - ref["U"]) <= 1e-11 * np.linalg.norm(ref["U"])
    assert np.linalg.norm(o["omega"] - om_o) <= 1e-11 * np.linalg.norm(om_o)
    assert np.linalg.norm(o["U"] - U_o) <= 1e-11 * np.linalg.norm(U_o)
    if g.nb > 2:
        assert np.abs(o["psi"] - psi_o).max() <= 1e-12
    assert o["resid"] <= 1e-14
    # gradients: the same on every part, and the unpartitioned ones to the
    # solver's accuracy (the gradient carries U's conditioning)
    for q in outs:
        assert np.array_equal(q["g_node"], o["g_node"]) and np.array_equal(q["g_shape"], o["g_shape"])
    sc = np.abs(ref["g_node"]).max()
    assert np.abs(o["g_node"] - ref["g_node"]).max() <= 1e-9 * sc
    if g.nb > 2:
        assert np.abs(o["g_shape"] - ref["g_shape"]).max() <= 1e-9 * np.abs(ref["g_shape"]).max()


def test_partition_arguments(P):
    import torch
    g, f, ph = W.one_ellipse_640()
    prob = P.Problem(g, f, ph)
    try:
        small = torch.empty(16, dtype=torch.uint8, device="cuda")
        with pytest.raises(P.BieError) as e:
            P.bie_set_partition(prob.ctx, 2, 0, small, lambda *a: 0)
        assert e.value.status == P.BIE_ERR_ARG
        with pytest.raises(P.BieError) as e:
            P.bie_set_partition(prob.ctx, 2, 2, small, lambda *a: 0)
        assert e.value.status == P.BIE_ERR_ARG
        assert P.bie_partition_rows(prob.ctx) == (0, g.N, g.N)
        # a failing exchange is reported, not hidden
        stage = torch.empty(P.partition_stage_bytes(g.N, 2), dtype=torch.uint8, device="cuda")
        P.bie_set_partition(prob.ctx, 2, 0, stage, lambda *a: 1)
        assert P.bie_partition_rows(prob.ctx) == P.partition_rows(g.N, 2, 0)
        prob.assemble("fp32_ir")
        with pytest.raises(P.BieError) as e:
            prob.solve()
        assert e.value.status == P.BIE_ERR_CUDA
        P.bie_set_partition(prob.ctx, 1, 0)
        prob.assemble("fp32_ir")
        assert prob.solve().converged
    finally:
        prob.close()
