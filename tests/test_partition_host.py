"""Host side of the row partition on CPU: the row ranges, and the
torch.distributed exchange (DistExchange) between two gloo ranks on CPU
tensors (the same calls run over NCCL between GPUs)."""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_partition_rows_cover_every_row_once():
    from paper_2108_01786_gb300 import partition_rows, partition_stage_bytes
    for N in (640, 1001, 16383, 32768, 96, 33):
        for P in (1, 2, 3, 4, 8):
            spans = [partition_rows(N, P, p) for p in range(P)]
            R = spans[0][2]
            assert all(s[2] == R for s in spans)
            if P > 1:
                assert R % 32 == 0 and P * R >= N and (P - 1) * R < N + 32 * P
            assert spans[0][0] == 0 and spans[-1][1] == N
            assert all(spans[p][1] == spans[p + 1][0] for p in range(P - 1))
            assert all(s[0] <= s[1] for s in spans)
            assert partition_stage_bytes(N, P) == 8 * P * R


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from paper_2108_01786_gb300 import DistExchange, BIE_EXCH_ALLGATHER, BIE_EXCH_ALLREDUCE_SUM
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        R = 5
        stage = torch.zeros(8 * world * R, dtype=torch.uint8)
        ex = DistExchange(stage, world, rank)
        # FP64 allgather: rank p's segment holds 100 p + i
        v = stage.view(torch.float64)
        v[rank * R:(rank + 1) * R] = torch.arange(R, dtype=torch.float64) + 100 * rank
        assert ex(BIE_EXCH_ALLGATHER, R, 8, 0) == 0
        got64 = v[: world * R].clone()
        # FP32 allgather on the same buffer
        w = stage.view(torch.float32)
        w.zero_()
        w[rank * R:(rank + 1) * R] = torch.arange(R, dtype=torch.float32) - 10 * rank
        assert ex(BIE_EXCH_ALLGATHER, R, 4, 0) == 0
        got32 = w[: world * R].clone()
        # allreduce of the first 3 doubles
        v[:3] = torch.tensor([1.0, 2.0, 3.0]) * (rank + 1)
        assert ex(BIE_EXCH_ALLREDUCE_SUM, 3, 8, 0) == 0
        red = v[:3].clone()
        assert ex(7, 3, 8, 0) != 0          # an unknown operation is refused
        q.put((rank, got64.tolist(), got32.tolist(), red.tolist()))
    finally:
        dist.destroy_process_group()


def test_dist_exchange_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    R = 5
    want64 = [float(i + 100 * p) for p in range(2) for i in range(R)]
    want32 = [float(i - 10 * p) for p in range(2) for i in range(R)]
    for rank, g64, g32, red in res:
        assert g64 == want64 and g32 == want32
        assert red == pytest.approx([3.0, 6.0, 9.0])
