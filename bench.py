#!/usr/bin/env python3
"""Benchmark: boundary-integral solves per second on the 16383-unknown workload.

One step = one full solve of the hot path on one geometry, through the C ABI:
node preparation (set_geometry), assembly of the dense matrix of eq. lin:sys,
the right-hand side, GMRES / GMRES-IR to rtol, and the normal velocity U.

Workload (synthetic, seeded): free surface 8192 nodes (random smooth profile,
amplitude 0.15, |k| <= 64, k^-2 spectrum), Gaussian-bump bottom 4096 nodes,
three random ellipses of 1365 nodes, N = 16383 unknowns.  Every step rewrites
the 1.1-2.7 GB matrix storage, far larger than the 129 MB L2, so no step reads
another step's data from L2.

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]

Under torchrun (N > 1) each rank solves its own instance (seed = rank): the
problems are independent, there is no collective on the data path, and the
reported value is the total over ranks ("scaling": "weak").
The reference arm (--impl reference) times the FP64 CPU oracle on the host
cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BIE solves/sec at N=16384 (to 1e-11 vs FP64 oracle); matvec HBM GB/s vs peak"
WORKLOAD = "three ellipses: surface 8192 + Gaussian-bump bottom 4096 + 3 ellipses x 1365 = 16383 unknowns"
PRECISIONS = ["fp16_ir", "fp32_ir", "bf16_ir", "fp64"]


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# the source files that define each profiled kernel
KERNEL_SOURCES = {
    "k_gemv_lowp": ("gemv.cu", "gemv_dot.cuh", "common.cuh"),
    "k_targets_far": ("targets.cu", "pair_kernel.cuh", "df2.cuh", "common.cuh"),
    "k_targets_helsing": ("targets.cu", "pair_kernel.cuh", "df2.cuh", "common.cuh"),
    "k_assemble_pairs": ("assemble.cu", "pair_kernel.cuh", "df2.cuh", "common.cuh"),
}
# FP32 issue peak: 152 SMs x 4 schedulers x 1 warp instruction per cycle
ISSUE_SLOTS_PER_CYCLE = 152 * 4
# FP64 FMA throughput measured on this machine's GB300: eight independent DFMA
# chains per thread, 4 x 152 CTAs of 512 threads, CUDA events (1.181-1.196
# TFLOP/s over three runs; nominal 1.25; the FP32 FMA rate measured the same way
# is 74.6 TFLOP/s, 62x)
FP64_FMA_TFLOPS = 1.196
# FP64 flops of one matrix entry in the separable form (a complex product for
# d = P Q - 1, a complex reciprocal, a product with zeta'): about 30
ASM_FLOPS_PER_ENTRY = 30


def _peak_clock_mhz():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return float(json.load(f).get("sm_max_mhz", 2070.0))
    return 2070.0


def _code_text(text):
    """C/CUDA source with comments and blank lines removed.  String and
    character literals (inline PTX included) are kept whole, so a '//' or
    '/*' inside one is code, not a comment."""
    out = []
    i, n = 0, len(text)
    while i < n:
        c = text[i]
        if c in "\"'":
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    return "\n".join(line.rstrip() for line in "".join(out).splitlines() if line.strip())


def _src_hash(kernel_key):
    """Hash of the code (comments and blank lines left out) of the files that
    define a kernel: the stored counters are valid while it is unchanged."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2108_01786_gb300", "csrc")
    for fn in KERNEL_SOURCES[kernel_key.split("<")[0]]:
        with open(os.path.join(csrc, fn)) as f:
            code = _code_text(f.read())
        h.update(fn.encode())
        h.update(code.encode())
    return h.hexdigest()[:16]


def _counters(kernel_key, field):
    """A per-launch ncu counter from the committed summary (profiles/traffic.json),
    if it was taken on the current sources of that kernel; else None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(kernel_key)
    if not e or kernel_key.split("<")[0] not in KERNEL_SOURCES or e.get("source_hash") != _src_hash(kernel_key):
        return None
    return e.get(field)


def _traffic(kernel_key):
    return _counters(kernel_key, "dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 100 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.tmp = None

    def __enter__(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.tmp, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.tmp is None:
            return None
        try:
            with open(self.tmp.name) as f:
                rows = [r.strip().split(", ") for r in f if r.strip()]
            os.unlink(self.tmp.name)
        except Exception:
            return None
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for n, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------------------
# multi-rank host logic (one process per GPU; independent problems per rank)
# ---------------------------------------------------------------------------

def barrier(world):
    """Barrier over the default process group (no-op for one rank)."""
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(value, world, device):
    """The largest of each rank's host float (the job ends with its slowest rank)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world, seconds):
    """Units all ranks processed divided by the (max-over-ranks) time: weak scaling."""
    return world * units_per_rank / seconds


def rank_seed(rank):
    """Each rank solves its own seeded instance of the workload."""
    return int(rank)


# ---------------------------------------------------------------------------
# oracle timing on the host cores (cpu_baseline leg and the reference arm)
# ---------------------------------------------------------------------------

_OG = _OF = None


def _oracle_worker_init(g, f):
    global _OG, _OF
    _OG, _OF = g, f


def _oracle_rows(r0, r1):
    """Rows r0..r1-1 of the oracle's matrix (in a spawned worker)."""
    import numpy as np
    from oracle import bie as O
    return r0, O.kernel_rows(_OG, np.arange(r0, r1))


def _oracle_velocity(t0, t1, omega):
    """U at surface nodes t0..t1-1 by the oracle (in a spawned worker)."""
    import numpy as np
    from oracle import bie as O
    return t0, O.normal_velocity(_OG, _OF, omega, targets=np.arange(t0, t1))


class OracleSolve:
    """One full FP64 oracle solve of a workload, the steps of oracle.bie.solve
    in their order: the dense matrix of eq. lin:sys (oracle.bie.kernel_rows,
    row blocks spread over a pool of spawned processes, one per host core),
    the right-hand side, the dense LU solve (LAPACK gesv, multithreaded) and U
    (oracle.bie.normal_velocity, surface-node blocks over the pool) with
    psi|_k.  parts(k) cuts the solve into k consecutive pieces so that it can
    be timed as k steps; the pieces together are exactly one solve."""

    def __init__(self, g, f, ph, workers=None):
        import multiprocessing as mp
        import numpy as np
        self.g, self.f, self.ph = g, f, ph
        self.workers = workers or _cores()
        self.pool = mp.get_context("spawn").Pool(self.workers, initializer=_oracle_worker_init,
                                                 initargs=(g, f))
        self.A = np.empty((g.N, g.N))
        self.omega = self.U = self.psi = None

    def close(self):
        self.pool.terminate()
        self.pool.join()

    def warm(self):
        """Start every worker (imports) on a few rows; untimed."""
        n = self.workers
        self.pool.starmap(_oracle_rows, [(i, i + 1) for i in range(n)])

    def _assemble(self, r0, r1):
        step = max(8, (r1 - r0 + 4 * self.workers - 1) // (4 * self.workers))
        for a, rows in self.pool.starmap(_oracle_rows, [(r, min(r1, r + step))
                                                        for r in range(r0, r1, step)]):
            self.A[a:a + len(rows)] = rows

    def _lu(self):
        from oracle import bie as O
        b = O.rhs(self.g, self.f, self.ph)
        self.omega = O.solve_dense(self.A, b)

    def _velocity(self):
        import numpy as np
        from oracle import bie as O
        M0 = self.g.M[0]
        step = max(8, (M0 + 4 * self.workers - 1) // (4 * self.workers))
        out = self.pool.starmap(_oracle_velocity, [(t, min(M0, t + step), self.omega)
                                                   for t in range(0, M0, step)])
        self.U = np.concatenate([u for _, u in sorted(out, key=lambda x: x[0])])
        self.psi = O.psi_k(self.g, self.omega)

    def parts(self, k):
        """k callables (k >= 1) that run one solve in order: for k >= 3,
        k - 2 row blocks of the assembly, the LU solve, U; fewer parts merge."""
        N = self.g.N
        if k == 1:
            return [lambda: (self._assemble(0, N), self._lu(), self._velocity())]
        if k == 2:
            return [lambda: self._assemble(0, N), lambda: (self._lu(), self._velocity())]
        edges = [N * i // (k - 2) for i in range(k - 1)]
        asm = [(lambda a=a, b=b: self._assemble(a, b)) for a, b in zip(edges[:-1], edges[1:])]
        return asm + [self._lu, self._velocity]


def time_oracle_solve(g, f, ph, nparts, warm=1):
    """Time one full oracle solve as nparts consecutive pieces.  Returns
    (seconds per piece, OracleSolve with omega, U, psi, phase seconds)."""
    o = OracleSolve(g, f, ph)
    try:
        for _ in range(max(1, warm)):
            o.warm()
        per = []
        for part in o.parts(nparts):
            t0 = time.perf_counter()
            part()
            per.append(time.perf_counter() - t0)
    finally:
        o.close()
    k = len(per)
    phases = ({"assembly_s": sum(per[:-2]), "lu_s": per[-2], "u_s": per[-1]} if k >= 3
              else {"total_s": sum(per)})
    return per, o, phases


def oracle_description(g, workers, nparts):
    return (f"one full solve of the {g.N}-unknown workload by the FP64 oracle (numpy/LAPACK): "
            f"assembly row blocks over {workers} spawned processes, LAPACK gesv on the "
            f"assembled matrix, U over the same processes; timed as {nparts} consecutive "
            f"pieces that together are the whole solve")


def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


def run_reference(args):
    """The oracle on the host cores: one full solve of the workload, cut into
    args.steps consecutive pieces (assembly row blocks, LU, U), each timed as a
    step; the value is one over the whole solve's time."""
    ws, rank, local = _dist()
    if rank != 0:
        return 0
    import workloads as W
    g, f, ph = W.three_ellipses_16383(seed=0)
    K = max(1, args.steps)
    per, o, phases = time_oracle_solve(g, f, ph, K, warm=args.warmup)
    total = sum(per)
    value = 1.0 / total
    desc = oracle_description(g, o.workers, K)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
        "n_gpus": args.gpus, "steps": K, "warmup": args.warmup,
        "ms_per_step": total * 1e3 / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _config(args, g),
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": o.workers, "kind": "oracle",
                         "sample": desc, "phases_s": phases, "full_solve_s": total},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def _config(args, g):
    return {"workload": WORKLOAD, "N": g.N, "precision": args.precision, "rtol": args.rtol,
            "restart": 50, "row_flip": True,
            "l2": "no flush needed: each step rewrites >= 1.1 GB of matrix storage (L2 129 MB)",
            "parallelism": f"independent problems x{args.gpus}"}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_ours(args):
    import numpy as np
    import torch

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2108_01786_gb300 import _build
    _build.build()
    import paper_2108_01786_gb300 as P
    import workloads as W

    g, f, ph = W.three_ellipses_16383(seed=rank_seed(rank))
    N, M0 = g.N, g.M[0]
    stream = torch.cuda.current_stream(dev)
    zt = lambda a: torch.as_tensor(a, dtype=torch.complex128, device=dev).contiguous()
    zeta, dzeta, d2zeta = zt(g.zeta), zt(g.dzeta), zt(g.d2zeta)
    phit = torch.as_tensor(ph, dtype=torch.float64, device=dev)
    omega = torch.zeros(N, dtype=torch.float64, device=dev)
    U = torch.zeros(M0, dtype=torch.float64, device=dev)
    psi = torch.zeros(g.nb - 2, dtype=torch.float64, device=dev)
    ctx = P.bie_create(local, stream)
    opts = P.bie_default_opts(rtol=args.rtol)

    def step(prec):
        P.bie_set_geometry(ctx, g.M, zeta, dzeta, d2zeta, g.zc)
        P.bie_set_flow(ctx, f.V1, f.a)
        P.bie_assemble(ctx, prec)
        return P.bie_solve(ctx, phit, omega, U, psi, opts)

    def timed(prec, K, W_, profile=False, clocks=None):
        for _ in range(W_):
            step(prec)
        torch.cuda.synchronize(dev)
        if profile:
            P.bie_set_profiling(ctx, True)
        barrier(ws)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        infos = []
        cm = clocks if clocks is not None else _Null()
        with cm:
            e0.record(stream)
            for _ in range(K):
                infos.append(step(prec))
            e1.record(stream)
            torch.cuda.synchronize(dev)
        barrier(ws)
        ms = e0.elapsed_time(e1)
        prof = P.bie_get_profile(ctx).as_dict() if profile else None
        if profile:
            P.bie_set_profiling(ctx, False)
        ms = max_over_ranks(ms, ws, dev)
        return ms, infos, prof

    # --- every storage scheme, briefly, for the variant table
    variants = {}
    for prec in ([] if args.headline_only else PRECISIONS):
        K = max(2, min(args.steps, 5)) if prec != args.precision else 0
        if K == 0:
            continue
        ms, infos, vprof = timed(prec, K, 1, profile=(prec == "fp64"))
        variants[prec] = _variant_entry(ms, K, infos, ws)
        variants[prec]["U_checksum"] = float(U.double().sum().item())
        if prec == "fp64":
            # FP64 storage: 2 N^2 flops per product against the FP64 pipe: the
            # DFMA rate measured on this machine's GB300 (independent FMA chains at
            # full occupancy) and the nominal 1.25 TFLOP/s
            gms = vprof["ms_gemv_inner"] / max(1, vprof["n_gemv_inner"])
            fl = 2.0 * N * N / (gms * 1e-3)
            variants[prec]["gemv_f64"] = {"avg_ms": gms, "launches": vprof["n_gemv_inner"],
                                          "TFLOPs": fl / 1e12,
                                          "peak_TFLOPs_measured": FP64_FMA_TFLOPS,
                                          "frac_of_measured": fl / (FP64_FMA_TFLOPS * 1e12),
                                          "peak_TFLOPs_nominal": 1.25,
                                          "frac_of_nominal": fl / 1.25e12,
                                          "GBps": 8.0 * N * N / (gms * 1e-3) / 1e9}

    # --- the headline: the chosen scheme, K timed steps with nothing but the work
    hb_peak, peak_kind = _peaks()
    sampler = ClockSampler(local) if rank == 0 else None
    ms, infos, _ = timed(args.precision, args.steps, args.warmup, profile=False, clocks=sampler)
    variants[args.precision] = _variant_entry(ms, args.steps, infos, ws)
    value = job_throughput(args.steps, ws, ms / 1e3)
    # --- the same K steps again with CUDA events around every hot launch on the
    # library's stream (kernel shares, roofline, launch count); the events add
    # ~2% to a step, so the headline pass above runs without them
    ms_prof, _, prof = timed(args.precision, args.steps, 1, profile=True)
    om_head = omega.cpu().numpy().copy()
    U_head = U.cpu().numpy().copy()

    # agreement between the headline scheme and the plain FP64 scheme
    diff = None
    if not args.headline_only:
        step("fp64")
        torch.cuda.synchronize(dev)
        om64, U64 = omega.cpu().numpy(), U.cpu().numpy()
        diff = {"omega_rel": float(np.linalg.norm(om_head - om64) / np.linalg.norm(om64)),
                "U_rel": float(np.linalg.norm(U_head - U64) / np.linalg.norm(U64))}

    # --- end to end through the host-buffer entry point (pinned buffers)
    pin = lambda a: torch.as_tensor(a).pin_memory()
    hz, hdz, hd2z = (pin(torch.view_as_real(torch.as_tensor(x)).reshape(-1).contiguous())
                     for x in (g.zeta, g.dzeta, g.d2zeta))
    hph = pin(torch.as_tensor(ph, dtype=torch.float64))
    hom = torch.zeros(N, dtype=torch.float64).pin_memory()
    hU = torch.zeros(M0, dtype=torch.float64).pin_memory()
    hpsi = torch.zeros(g.nb - 2, dtype=torch.float64).pin_memory()
    ke = max(3, min(args.steps, 10))
    for _ in range(2):
        P.bie_solve_host(ctx, g.M, hz, hdz, hd2z, g.zc, f.V1, f.a, hph, args.precision, hom, hU,
                         hpsi, opts)
    barrier(ws)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(ke):
        P.bie_solve_host(ctx, g.M, hz, hdz, hd2z, g.zc, f.V1, f.a, hph, args.precision, hom, hU,
                         hpsi, opts)
    torch.cuda.synchronize(dev)
    e2e_s = time.perf_counter() - t0
    barrier(ws)
    e2e_s = max_over_ranks(e2e_s, ws, dev)
    e2e = {"value": job_throughput(ke, ws, e2e_s), "unit": "solves/s",
           "h2d_bytes_per_step": int(3 * 16 * N + 8 * M0),
           "d2h_bytes_per_step": int(8 * N + 8 * M0 + 8 * (g.nb - 2))}

    P.bie_destroy(ctx)

    # the other hot-path rows, measured briefly on their own workloads
    rows = {} if args.headline_only else {
            "a9_targets": row_targets(P, W, dev, stream),
            "a8_adjoint": row_adjoint(P, W, dev, stream),
            "a7_batched": row_batched(P, W, dev, stream),
            "f1_vortex_sheet": row_vortex_sheet(P, W, dev, stream),
            "f2_multi_rhs": row_multi_rhs(P, W, dev, stream),
            "f3_graph_evolution": row_graph_evolution(P, W, dev, stream),
            "f4_psi_prescribed": row_psi_prescribed(P, W, dev, stream)}
    if rank != 0:
        return 0

    # --- roofline of the dominant kernel (by accumulated time)
    kinds = {
        "gemv_inner": (prof["ms_gemv_inner"], prof["n_gemv_inner"], prof["bytes_gemv_inner"]),
        "gemv_full": (prof["ms_gemv_full"], prof["n_gemv_full"], prof["bytes_gemv_full"]),
        "gemv_hi": (prof["ms_gemv_hi"], prof["n_gemv_hi"], prof["bytes_gemv_hi"]),
        "assemble": (prof["ms_assemble"], prof["n_assemble"], None),
        "velocity": (prof["ms_velocity"], prof["n_velocity"], None),
    }
    step_ms = ms_prof / args.steps
    shares = {k: (v[0] / args.steps) / step_ms for k, v in kinds.items()}
    gemv_key = {"fp32_ir": "k_gemv_lowp<float>", "fp16_ir": "k_gemv_lowp<__half>",
                "bf16_ir": "k_gemv_lowp<__nv_bfloat16>", "fp64": "k_gemv_f64"}[args.precision]
    avg_ms = prof["ms_gemv_inner"] / max(1, prof["n_gemv_inner"])
    achieved = prof["bytes_gemv_inner"] / (avg_ms * 1e-3) / 1e9
    full_avg = prof["ms_gemv_full"] / max(1, prof["n_gemv_full"])
    roofline = {"bound": "hbm", "kernel": gemv_key, "achieved": achieved, "peak": hb_peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / hb_peak,
                "traffic": _traffic(gemv_key), "avg_launch_ms": avg_ms,
                "launches": prof["n_gemv_inner"],
                "algorithmic_bytes_per_launch": prof["bytes_gemv_inner"],
                "timed_pass": "the K headline steps repeated with an event pair around each launch"}
    if args.precision != "fp64":
        # the library's Gram-Schmidt kernels fetch the first quarter-L2 of the
        # stored matrix into L2 while HBM is otherwise idle; that part of each
        # launch's stream comes from L2, the rest from HBM
        l2 = int(getattr(torch.cuda.get_device_properties(0), "L2_cache_size", 0))
        pf = min(l2 // 4, int(prof["bytes_gemv_inner"])) // 16 * 16
        roofline["l2_prefetched_bytes_per_launch"] = pf
        roofline["frac_hbm_part"] = ((prof["bytes_gemv_inner"] - pf) / (avg_ms * 1e-3) / 1e9
                                     / hb_peak)
    asm_avg_ms = prof["ms_assemble"] / max(1, prof["n_assemble"])
    asm_inst = _counters("k_assemble_pairs<dfl>", "warp_instructions_per_launch")
    asm_peak = ISSUE_SLOTS_PER_CYCLE * _peak_clock_mhz() * 1e6
    roofline_asm = {"bound": "alu", "kernel": "k_assemble_pairs<dfl>",
                    "achieved": (asm_inst / (asm_avg_ms * 1e-3)) if asm_inst else None,
                    "peak": asm_peak, "unit": "warp-instructions/s",
                    "frac": (asm_inst / (asm_avg_ms * 1e-3) / asm_peak) if asm_inst else None,
                    "instructions_per_launch": asm_inst, "avg_launch_ms": asm_avg_ms,
                    "entries_per_s": N * N / (asm_avg_ms * 1e-3),
                    # algorithmic work: the separable-form kernel evaluation costs
                    # ~30 FP64 flops per entry (one complex product, one complex
                    # reciprocal, one product with zeta'); done here in double-float
                    # on the FP32 pipes, against the measured FP64 FMA rate
                    "algorithmic_fp64_flops_per_entry": ASM_FLOPS_PER_ENTRY,
                    "algorithmic_fp64_tflops": N * N * ASM_FLOPS_PER_ENTRY / (asm_avg_ms * 1e-3) / 1e12,
                    "algorithmic_vs_fp64_peak": (N * N * ASM_FLOPS_PER_ENTRY / (asm_avg_ms * 1e-3)
                                                 / (FP64_FMA_TFLOPS * 1e12)),
                    "fma_pipe_frac_ncu": _counters("k_assemble_pairs<dfl>", "fma_pipe_frac"),
                    # the stores alone (A hi/lo/16 + surface U-matrix hi/lo) at the HBM peak
                    "hbm_write_ms_at_peak": (N * N * 10.0 + M0 * N * 8.0) / (hb_peak * 1e9) * 1e3}
    kernels = {
        "gemv_inner": {"ms_per_step": kinds["gemv_inner"][0] / args.steps, "share": shares["gemv_inner"],
                       "launches_per_step": prof["n_gemv_inner"] / args.steps, "avg_ms": avg_ms,
                       "GBps": achieved},
        "gemv_full_hilo": {"ms_per_step": kinds["gemv_full"][0] / args.steps,
                           "share": shares["gemv_full"],
                           "launches_per_step": prof["n_gemv_full"] / args.steps,
                           "avg_ms": full_avg,
                           "GBps": (prof["bytes_gemv_full"] / (full_avg * 1e-3) / 1e9) if full_avg > 0 else None},
        "gemv_resid_hi_only": {"ms_per_step": kinds["gemv_hi"][0] / args.steps,
                               "share": shares["gemv_hi"],
                               "launches_per_step": prof["n_gemv_hi"] / args.steps},
        "assemble": {"ms_per_step": kinds["assemble"][0] / args.steps, "share": shares["assemble"],
                     "entries_per_s": N * N / (kinds["assemble"][0] / max(1, prof["n_assemble"]) * 1e-3)},
        "velocity": {"ms_per_step": kinds["velocity"][0] / args.steps, "share": shares["velocity"]},
        "profiled_pass_ms_per_step": step_ms,
    }

    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        per, o, phases = time_oracle_solve(g, f, ph, 3)
        cpu = {"value": 1.0 / sum(per), "unit": "solves/s", "cores": o.workers, "kind": "oracle",
               "sample": oracle_description(g, o.workers, 3), "phases_s": phases,
               "full_solve_s": sum(per),
               # the headline scheme's answer against this full oracle solve
               "gpu_vs_oracle": {
                   "omega_rel": float(np.linalg.norm(om_head - o.omega) / np.linalg.norm(o.omega)),
                   "U_rel": float(np.linalg.norm(U_head - o.U) / np.linalg.norm(o.U))}}

    clocks = sampler.summary() if sampler is not None else None
    dtype = {"fp32_ir": "f32+df64", "fp16_ir": "f16/f32+df64", "bf16_ir": "bf16/f32+df64",
             "fp64": "f64"}[args.precision]
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
        "data": "synthetic",
        "config": _config(args, g),
        "roofline": roofline,
        "roofline_assembly": roofline_asm,
        "kernels": kernels,
        "variants": variants,
        "accuracy": {"rel_resid": infos[-1].rel_resid, "vs_fp64_scheme": diff,
                     "iters": infos[-1].iters, "cycles": infos[-1].cycles},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(prof["kernel_launches"]),
        "clocks": clocks,
        "rows": rows,
    }
    print(json.dumps(line))
    return 0


def _events_ms(stream, fn, reps, warm=1):
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps, out


def row_targets(P, W, dev, stream, reps=2):
    """Velocity at targets (four ellipses): 32768 unknowns, ~10^6 grid targets plus
    10^5 targets within 2 node spacings (Helsing)."""
    import numpy as np
    import torch
    g, f, ph = W.four_ellipses_32768(seed=0)
    zg, zn = W.targets_32768(g)
    z = torch.as_tensor(np.concatenate([zg, zn]), dtype=torch.complex128, device=dev)
    zt = lambda a: torch.as_tensor(a, dtype=torch.complex128, device=dev).contiguous()
    zeta, dzeta, d2zeta = zt(g.zeta), zt(g.dzeta), zt(g.d2zeta)
    phit = torch.as_tensor(ph, dtype=torch.float64, device=dev)
    omega = torch.zeros(g.N, dtype=torch.float64, device=dev)
    U = torch.zeros(g.M[0], dtype=torch.float64, device=dev)
    uv = torch.empty(z.numel(), dtype=torch.complex128, device=dev)
    ctx = P.bie_create(dev.index, stream)
    try:
        opts = P.bie_default_opts()

        def solve():
            P.bie_set_geometry(ctx, g.M, zeta, dzeta, d2zeta, g.zc)
            P.bie_set_flow(ctx, f.V1, f.a)
            P.bie_assemble(ctx, "fp32_ir")
            return P.bie_solve(ctx, phit, omega, U, None, opts)

        ms_solve, info = _events_ms(stream, solve, reps)
        ms_t, _ = _events_ms(stream, lambda: P.bie_eval_velocity(
            ctx, omega, z, uv, mode=P.VEL_AUTO, near_spacings=2.0), reps)
        nn = P.bie_eval_velocity(ctx, omega, z, uv, mode=P.VEL_AUTO, near_spacings=2.0,
                                 count_near=True)
        nz = z.numel()
        # the two kernels alone: far sums on the grid targets, Helsing-Ojala on
        # the near ones; issue fractions from their ncu instruction counts
        zgt = torch.as_tensor(zg, dtype=torch.complex128, device=dev)
        znt = torch.as_tensor(zn, dtype=torch.complex128, device=dev)
        ug = torch.empty_like(zgt)
        un = torch.empty_like(znt)
        ms_far, _ = _events_ms(stream, lambda: P.bie_eval_velocity(ctx, omega, zgt, ug, mode=P.VEL_FAR),
                               reps)
        ms_hel, _ = _events_ms(stream, lambda: P.bie_eval_velocity(ctx, omega, znt, un,
                                                                   mode=P.VEL_HELSING), reps)
        peak = ISSUE_SLOTS_PER_CYCLE * _peak_clock_mhz() * 1e6

        def issue(kernel, pairs, ms):
            ipp = _counters(kernel, "thread_instructions_per_pair")
            if not ipp:
                return {"pairs_per_s": pairs / (ms * 1e-3), "ms": ms}
            ach = pairs / (ms * 1e-3) * ipp / 32.0
            return {"pairs_per_s": pairs / (ms * 1e-3), "ms": ms, "bound": "alu",
                    "thread_instructions_per_pair": ipp, "achieved": ach, "peak": peak,
                    "unit": "warp-instructions/s", "frac": ach / peak,
                    "fma_pipe_frac_ncu": _counters(kernel, "fma_pipe_frac")}

        return {"workload": "four_ellipses_32768: surface 16384 + bottom 8192 + 4 ellipses x 2048 = 32768 "
                            "unknowns; grid + near-boundary targets",
                "N": g.N, "targets": nz, "helsing_targets": int(nn),
                "ms_solve_fp32_ir": ms_solve, "solve_iters": info.iters,
                "solve_rel_resid": info.rel_resid, "ms_targets": ms_t,
                "target_pairs_per_s": nz * g.N / (ms_t * 1e-3),
                "far_alone": issue("k_targets_far", len(zg) * g.N, ms_far),
                "helsing_alone": issue("k_targets_helsing", len(zn) * g.N, ms_hel)}
    finally:
        P.bie_destroy(ctx)


def row_batched(P, W, dev, stream, reps=3):
    """96 independent problems of N ~ U{1024..12288} (random geometries) per call of
    bie_batch_run: node tables, assembly, right-hand side, one cooperative
    GMRES-IR kernel for all problems and U, replayed from a CUDA graph."""
    import numpy as np
    import torch
    probs = W.random_batch(seed=0)
    zt = lambda a: torch.as_tensor(a, dtype=torch.complex128, device=dev).contiguous()
    b = P.bie_batch_create(dev.index, stream)
    Ns = np.array([g.N for g, _, _ in probs], dtype=np.float64)
    out = {"workload": "random_batch: 96 random problems, N ~ U{1024..12288}, "
                       f"sum N = {int(Ns.sum())}, sum N^2 = {Ns @ Ns:.3e}",
           "problems": len(probs)}
    try:
        for p, (g, f, ph) in enumerate(probs):
            P.bie_batch_set_problem(b, p, g.M, zt(g.zeta), zt(g.dzeta), zt(g.d2zeta), g.zc,
                                    f.V1, f.a)
        phit = torch.as_tensor(np.concatenate([ph for _, _, ph in probs]), device=dev)
        omega = torch.empty(int(Ns.sum()), dtype=torch.float64, device=dev)
        U = torch.empty(sum(g.M[0] for g, _, _ in probs), dtype=torch.float64, device=dev)
        for prec in ("fp32_ir", "fp16_ir"):
            run = lambda: P.bie_batch_run(b, len(probs), phit, omega, U, prec)
            ms, infos = _events_ms(stream, run, reps, warm=1)
            ub0, cand0 = P.bie_batch_tuning(b)
            kern_ms = min(cand0)
            # matrix bytes of the whole batch: the inner storage read once per
            # Arnoldi step of each problem, and the residual products (counted by
            # the solver kernel: hi + lo, FP32 part or inner storage, per residual)
            es = 4 if prec == "fp32_ir" else 2
            ld = [int(np.ceil(g.N / 64) * 64) for g, _, _ in probs]
            inner_bytes = sum(i.iters * g.N * l * es for i, (g, _, _), l in zip(infos, probs, ld))
            resid_bytes = P.bie_batch_resid_bytes(b)
            hb, _ = _peaks()
            ub, cand = P.bie_batch_tuning(b)
            gbps = (inner_bytes + resid_bytes) / (kern_ms * 1e-3) / 1e9
            out[prec] = {"ms_per_batch": ms, "solves_per_s": len(probs) / (ms * 1e-3),
                         "tuned_gemv_unit_bytes": ub,
                         "tuning_kernel_ms": {str(c): round(t, 3) for c, t in
                                              zip([256 << 10, 512 << 10, 1 << 20, 2 << 20, 4 << 20], cand)},
                         "converged": int(sum(i.converged for i in infos)),
                         "max_iters": int(max(i.iters for i in infos)),
                         "max_cycles": int(max(i.cycles for i in infos)),
                         "max_rel_resid": float(max(i.rel_resid for i in infos)),
                         "solver_kernel_ms": kern_ms,
                         "matrix_bytes": {"arnoldi": inner_bytes, "residuals": resid_bytes},
                         "solver_kernel_GBps": gbps,
                         "solver_kernel_frac_of_measured_hbm": gbps / hb}
        return out
    finally:
        P.bie_batch_destroy(b)


def row_vortex_sheet(P, W, dev, stream, reps=5):
    """Vortex-sheet route on the 16383-unknown workload: gamma_0 -> solid system
    of eq. lin:sys2 (8191 unknowns) -> U; first call (assembles the solid
    system) and repeated calls on the same geometry."""
    import numpy as np
    import torch
    g, f, ph = W.three_ellipses_16383(seed=0)
    zt = lambda a: torch.as_tensor(a, dtype=torch.complex128, device=dev).contiguous()
    ctx = P.bie_create(dev.index, stream)
    out = {"workload": "three_ellipses_16383 geometry; gamma_0 band-limited (|k| <= 64); solid system "
                       f"{g.N - g.M[0]} unknowns", "N_solid": g.N - g.M[0]}
    try:
        P.bie_set_geometry(ctx, g.M, zt(g.zeta), zt(g.dzeta), zt(g.d2zeta), g.zc)
        P.bie_set_flow(ctx, f.V1, f.a)
        gamma0 = torch.as_tensor(W.filtered_noise(np.random.default_rng(1), g.M[0], 0.5, 64),
                                 device=dev)
        U = torch.empty(g.M[0], dtype=torch.float64, device=dev)
        for prec in ("fp32_ir", "fp16_ir"):
            P.bie_set_geometry(ctx, g.M, zt(g.zeta), zt(g.dzeta), zt(g.d2zeta), g.zc)
            ms_first, _ = _events_ms(stream, lambda: P.bie_vs_normal_velocity(
                ctx, gamma0, U, precision=prec), 1, warm=0)
            ms, info = _events_ms(stream, lambda: P.bie_vs_normal_velocity(
                ctx, gamma0, U, precision=prec), reps, warm=1)
            out[prec] = {"ms_first_call": ms_first, "ms_per_call": ms,
                         "calls_per_s": 1e3 / ms, "iters": info.iters, "cycles": info.cycles,
                         "rel_resid": info.rel_resid}
        return out
    finally:
        P.bie_destroy(ctx)


def row_multi_rhs(P, W, dev, stream, reps=3):
    """Several right-hand sides on the 16383-unknown matrix (FP16 storage):
    bie_solve_multi with 1..64 columns against one bie_solve per column
    (omega and U of every column, matrix assembled once, outside the timing)."""
    import numpy as np
    import torch
    g, f, ph = W.three_ellipses_16383(seed=0)
    rng = np.random.default_rng(4)
    PH = np.stack([W.filtered_noise(rng, g.M[0], 0.05, 20) for _ in range(64)])
    prob = P.Problem(g, f, ph, device=dev.index, stream=stream)
    out = {"workload": f"three_ellipses_16383 geometry, N={g.N}; phi~ band-limited noise per column",
           "storage": "fp16_ir"}
    try:
        prob.assemble("fp16_ir")
        ms1, info = _events_ms(stream, lambda: prob.solve(), reps, warm=1)
        out["single_ms_per_solve"] = ms1
        out["single_iters"] = info.iters
        for nrhs in (1, 8, 16, 32, 64):
            phd = torch.as_tensor(PH[:nrhs], device=dev).contiguous()
            om = torch.empty((nrhs, g.N), dtype=torch.float64, device=dev)
            U = torch.empty((nrhs, g.M[0]), dtype=torch.float64, device=dev)
            ms, infos = _events_ms(stream, lambda: P.bie_solve_multi(prob.ctx, phd, om, U),
                                   reps, warm=1)
            out[f"nrhs{nrhs}"] = {"ms_per_call": ms, "solves_per_s": 1e3 * nrhs / ms,
                                  "vs_single_solves": ms1 * nrhs / ms,
                                  "max_iters": max(i.iters for i in infos),
                                  "max_cycles": max(i.cycles for i in infos)}
        # Phi_t - C of 16 states (eq. pressure:d:prob): state solves, b^aux, auxiliary solves
        nst = 16
        phd = torch.as_tensor(PH[:nst], device=dev).contiguous()
        om = torch.empty((nst, g.N), dtype=torch.float64, device=dev)
        U = torch.empty((nst, g.M[0]), dtype=torch.float64, device=dev)
        B = torch.empty((nst, g.N), dtype=torch.float64, device=dev)
        omx = torch.empty((nst, g.N), dtype=torch.float64, device=dev)

        def multi_pipeline():
            P.bie_solve_multi(prob.ctx, phd, om, U)
            for r in range(nst):
                P.bie_pressure_rhs(prob.ctx, phd[r], U[r], B[r], tau=0.1, g=1.0)
            return P.bie_solve_multi(prob.ctx, B, omx, None, kind="b")

        def single_pipeline():
            for r in range(nst):
                P.bie_solve(prob.ctx, phd[r], om[r], U[r])
                P.bie_pressure_rhs(prob.ctx, phd[r], U[r], B[r], tau=0.1, g=1.0)
                info = P.bie_solve_b(prob.ctx, B[r], omx[r])
            return [info]

        ms_m, infos = _events_ms(stream, multi_pipeline, reps, warm=1)
        ms_s, _ = _events_ms(stream, single_pipeline, 1, warm=1)
        # Phi_t - C on every boundary node of one state (Plemelj evaluation of
        # omega^aux): with the solids' velocities it gives their pressure
        phib = torch.empty(g.N, dtype=torch.complex128, device=dev)
        ms_b, _ = _events_ms(stream, lambda: P.bie_boundary_potential(prob.ctx, omx[0], phib),
                             reps, warm=1)
        out["pressure_aux_16_states"] = {"ms_multi": ms_m, "ms_single_solves": ms_s,
                                         "speedup": ms_s / ms_m,
                                         "aux_max_iters": max(i.iters for i in infos),
                                         "ms_boundary_potential_one_state": ms_b}
        return out
    finally:
        prob.close()


def row_graph_evolution(P, W, dev, stream, nsteps=4):
    """RK4 steps of the graph formulation (eqs. graph:eta:t, phitileq) and of the
    HLS formulation (P theta reconstruction) with the filter, on problem 1 of
    Sec. 7 at M_0 = 4096 (N = 11776): every stage rebuilds the surface,
    assembles and solves; energy monitored each step."""
    import numpy as np
    import torch
    g, f, ph = W.paper_problem(1, M0=4096, M1=1536, Me=2048)
    prob = P.Problem(g, f, ph, device=dev.index, stream=stream)
    out = {"workload": f"paper problem 1 geometry, M0={g.M[0]}, N={g.N}; eta0 = 0, "
                       "phi~0 of the problem; dt = 1e-4, tau = 0.1, g = 1",
           "N": g.N, "steps": nsteps}
    try:
        for prec in ("fp32_ir", "fp16_ir"):
            eta = torch.zeros(g.M[0], dtype=torch.float64, device=dev)
            phit = prob.phit.clone()
            P.bie_graph_evolve(prob.ctx, eta, phit, 1e-4, 1, filter=True, precision=prec,
                               energies=False)
            eta.zero_()
            phit.copy_(prob.phit)
            ms, (E, info) = _events_ms(stream, lambda: P.bie_graph_evolve(
                prob.ctx, eta, phit, 1e-4, nsteps, filter=True, precision=prec), 1, warm=0)
            out[prec] = {"ms_per_step": ms / nsteps, "steps_per_s": 1e3 * nsteps / ms,
                         "solves": info.solves, "gmres_iters": int(info.gmres_iters),
                         "energy_rel_drift": float(np.abs(E - E[0]).max() / abs(E[0]))}
        # the HLS formulation (P theta reconstruction) on the same workload
        th = torch.zeros(g.M[0], dtype=torch.float64, device=dev)
        phit = prob.phit.clone()
        P.bie_hls_evolve(prob.ctx, th, phit, 1e-4, 1, filter=True, precision="fp16_ir",
                         energies=False)
        th.zero_()
        phit.copy_(prob.phit)
        ms, (E, info) = _events_ms(stream, lambda: P.bie_hls_evolve(
            prob.ctx, th, phit, 1e-4, nsteps, filter=True, precision="fp16_ir"), 1, warm=0)
        out["hls_fp16_ir"] = {"ms_per_step": ms / nsteps, "steps_per_s": 1e3 * nsteps / ms,
                              "solves": info.solves, "gmres_iters": int(info.gmres_iters),
                              "energy_rel_drift": float(np.abs(E - E[0]).max() / abs(E[0]))}
        # one step of the paper's eighth-order Dormand-Prince scheme (12 right-hand
        # sides) of the graph and HLS formulations
        for form in ("graph", "hls"):
            y1 = torch.zeros(g.M[0], dtype=torch.float64, device=dev)
            phit.copy_(prob.phit)
            ms, (E, info) = _events_ms(stream, lambda: P.bie_evolve(
                prob.ctx, y1, phit, 4e-4, 1, formulation=form, integrator="dp8", filter=True,
                precision="fp16_ir"), 1, warm=0)
            out[f"{form}_dp8_fp16_ir"] = {
                "ms_per_step": ms, "dt": 4e-4, "solves": info.solves,
                "energy_rel_drift": float(np.abs(E - E[0]).max() / abs(E[0]))}
        # one eighth-order GBS step (17 right-hand sides) of the HLS formulation
        th.zero_()
        phit.copy_(prob.phit)
        ms, (E, info) = _events_ms(stream, lambda: P.bie_evolve(
            prob.ctx, th, phit, 4e-4, 1, formulation="hls", integrator="gbs8", filter=True,
            precision="fp16_ir"), 1, warm=0)
        out["hls_gbs8_fp16_ir"] = {"ms_per_step": ms, "dt": 4e-4, "solves": info.solves,
                                   "energy_rel_drift": float(np.abs(E - E[0]).max() / abs(E[0]))}
        # the vortex-sheet formulation (state eta, gamma_0 = -omega_0' of the first solve)
        eta = torch.zeros(g.M[0], dtype=torch.float64, device=dev)
        om = torch.empty(g.N, dtype=torch.float64, device=dev)
        et = torch.empty(g.M[0], dtype=torch.float64, device=dev)
        pt = torch.empty_like(et)
        P.bie_graph_rhs(prob.ctx, eta, prob.phit, et, pt, omega=om)
        gm = -torch.as_tensor(np.fft.ifft(1j * np.fft.fftfreq(g.M[0], 1.0 / g.M[0]) *
                                          np.fft.fft(om[:g.M[0]].cpu().numpy())).real, device=dev)
        P.bie_evolve(prob.ctx, eta, gm.clone(), 1e-4, 1, formulation="vs_graph",
                     precision="fp16_ir", energies=False)
        eta.zero_()
        ms, (_, info) = _events_ms(stream, lambda: P.bie_evolve(
            prob.ctx, eta, gm.clone(), 1e-4, nsteps, formulation="vs_graph", precision="fp16_ir",
            energies=False), 1, warm=0)
        out["vortex_sheet_fp16_ir"] = {"ms_per_step": ms / nsteps, "steps_per_s": 1e3 * nsteps / ms,
                                       "solves": info.solves, "gmres_iters": int(info.gmres_iters)}
        return out
    finally:
        prob.close()


def row_psi_prescribed(P, W, dev, stream, reps=5):
    """App. B variant on the 16383-unknown workload: assembly of eq. A:alt and
    the solve for omega, a_j and U, against the standard assembly and solve."""
    import numpy as np
    import torch
    g, f, ph = W.three_ellipses_16383(seed=0)
    M0 = g.M[0]
    prob = P.Problem(g, f, ph, device=dev.index, stream=stream)
    out = {"workload": f"three_ellipses_16383 geometry, N={g.N}; phi - V1 xi = phi~ + sum a_j phi_cyl, "
                       "psi = 0 on the bottom and 0.1 j on obstacle j"}
    try:
        psi_s = np.zeros(g.N - M0)
        o = g.offsets()
        for k in range(2, len(g.M)):
            psi_s[o[k] - M0:o[k + 1] - M0] = 0.1 * k
        phic = torch.as_tensor(ph, device=dev)
        psid = torch.as_tensor(psi_s, device=dev)
        om = torch.empty(g.N, dtype=torch.float64, device=dev)
        U = torch.empty(M0, dtype=torch.float64, device=dev)
        zt = lambda a: torch.as_tensor(a, dtype=torch.complex128, device=dev).contiguous()
        zeta, dzeta, d2zeta = zt(g.zeta), zt(g.dzeta), zt(g.d2zeta)

        def fresh_assembly_ms(assemble):
            # each timed assembly follows bie_set_geometry (untimed), so it
            # recomputes every entry: the library keeps the solid-solid entries
            # of an unchanged geometry otherwise
            tot = 0.0
            for r in range(reps + 1):
                P.bie_set_geometry(prob.ctx, g.M, zeta, dzeta, d2zeta, g.zc)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                assemble()
                e1.record(stream)
                torch.cuda.synchronize(dev)
                if r > 0:
                    tot += e0.elapsed_time(e1)
            return tot / reps

        for prec in ("fp32_ir", "fp16_ir"):
            ms_a = fresh_assembly_ms(lambda: P.bie_assemble_psi(prob.ctx, prec))
            ms_s, (a, info) = _events_ms(stream, lambda: P.bie_solve_psi(
                prob.ctx, phic, psid, om, U, nobs=len(g.zc)), reps, warm=1)
            ms_a0 = fresh_assembly_ms(lambda: prob.assemble(prec))
            ms_s0, _ = _events_ms(stream, lambda: prob.solve(), reps, warm=1)
            out[prec] = {"assemble_ms": ms_a, "solve_ms": ms_s, "iters": info.iters,
                         "standard_assemble_ms": ms_a0, "standard_solve_ms": ms_s0,
                         "a": [float(x) for x in a]}
        return out
    finally:
        prob.close()


def row_adjoint(P, W, dev, stream, reps=5):
    """Gradient of J = (2 pi/M_0) sum U^2 (two ellipses: 4096 unknowns) with respect
    to the 10 ellipse parameters and the 2 x 2048 surface-node coordinates:
    backward time against the forward (assemble + solve) time."""
    import numpy as np
    import torch
    g, f, ph = W.two_ellipses_4096(seed=0)
    zt = lambda a: torch.as_tensor(a, dtype=torch.complex128, device=dev).contiguous()
    zeta, dzeta, d2zeta = zt(g.zeta), zt(g.dzeta), zt(g.d2zeta)
    phit = torch.as_tensor(ph, dtype=torch.float64, device=dev)
    omega = torch.zeros(g.N, dtype=torch.float64, device=dev)
    U = torch.zeros(g.M[0], dtype=torch.float64, device=dev)
    gU = torch.empty(g.M[0], dtype=torch.float64, device=dev)
    g_node = torch.empty(g.N, dtype=torch.complex128, device=dev)
    g_shape = torch.empty(10, dtype=torch.float64, device=dev)
    g_phit = torch.empty(g.M[0], dtype=torch.float64, device=dev)
    ell = np.array(g.ellipses, dtype=np.float64)
    ctx = P.bie_create(dev.index, stream)
    out = {"workload": "two_ellipses_4096: surface 2048 + bottom 1024 + 2 ellipses x 512 = 4096 unknowns; "
                       "J = (2 pi/M_0) sum U^2; gradient w.r.t. 10 ellipse parameters + "
                       "2048 surface nodes (and phi~)", "N": g.N}
    try:
        P.bie_set_geometry(ctx, g.M, zeta, dzeta, d2zeta, g.zc)
        P.bie_set_flow(ctx, f.V1, f.a)
        for prec in ("fp32_ir", "fp64"):
            opts = P.bie_default_opts()

            def forward():
                P.bie_assemble(ctx, prec)
                return P.bie_solve(ctx, phit, omega, U, None, opts)

            def backward():
                torch.mul(U, 2 * 2 * np.pi / g.M[0], out=gU)
                return P.bie_backward(ctx, omega, gU, ell, g_node=g_node, g_shape=g_shape,
                                      g_phit=g_phit, opts=opts)

            ms_f, ms_b = 0.0, 0.0
            for _ in range(2):          # warm-up
                forward()
                backward()
            for _ in range(reps):
                ms, info_f = _events_ms(stream, forward, 1, warm=0)
                ms_f += ms / reps
                ms, info_b = _events_ms(stream, backward, 1, warm=0)
                ms_b += ms / reps
            out[prec] = {"ms_forward": ms_f, "ms_backward": ms_b, "ratio": ms_b / ms_f,
                         "forward_iters": info_f.iters, "adjoint_iters": info_b.iters,
                         "adjoint_rel_resid": info_b.rel_resid}
        return out
    finally:
        P.bie_destroy(ctx)


def _variant_entry(ms, K, infos, ws):
    return {"solves_per_s": ws * K / (ms / 1e3), "ms_per_solve": ms / K,
            "iters": infos[-1].iters, "cycles": infos[-1].cycles,
            "rel_resid": infos[-1].rel_resid, "converged": bool(infos[-1].converged)}


class _Null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


def profile_case(name):
    """Small cases of each hot kernel for ncu captures (a few GB on the device,
    inputs larger than L2); each runs twice and prints one line."""
    import numpy as np
    import torch
    import paper_2108_01786_gb300 as P
    import workloads as W
    from paper_2108_01786_gb300 import _build
    _build.build()
    dev = torch.device("cuda", 0)
    zt = lambda a: torch.as_tensor(a, dtype=torch.complex128, device=dev).contiguous()
    if name == "solve":            # 16383 unknowns, fp16-IR: assembly, GEMVs, CGS, U
        g, f, ph = W.three_ellipses_16383()
        prob = P.Problem(g, f, ph)
        for _ in range(2):         # a full step each time, as in the headline
            P.bie_set_geometry(prob.ctx, g.M, zt(g.zeta), zt(g.dzeta), zt(g.d2zeta), g.zc)
            prob.assemble("fp16_ir")
            info = prob.solve()
        prob.close()
        print("solve", info.iters, info.cycles, info.rel_resid)
    elif name == "batch":          # 12 problems, N ~ U{3000..6000}, fp32-IR
        rng = np.random.default_rng(5)
        probs = [W.random_geometry(rng, int(n)) for n in rng.integers(3000, 6001, size=12)]
        b = P.bie_batch_create(0, torch.cuda.current_stream())
        for p, (g, f, ph) in enumerate(probs):
            P.bie_batch_set_problem(b, p, g.M, zt(g.zeta), zt(g.dzeta), zt(g.d2zeta), g.zc, f.V1, f.a)
        phit = torch.as_tensor(np.concatenate([ph for _, _, ph in probs]), device=dev)
        om = torch.empty(sum(g.N for g, _, _ in probs), dtype=torch.float64, device=dev)
        U = torch.empty(sum(g.M[0] for g, _, _ in probs), dtype=torch.float64, device=dev)
        for _ in range(2):
            infos = P.bie_batch_run(b, len(probs), phit, om, U, "fp32_ir")
        P.bie_batch_destroy(b)
        print("batch", max(i.iters for i in infos), max(i.rel_resid for i in infos))
    elif name == "adjoint":        # 4096 unknowns, fp32-IR: forward + backward
        g, f, ph = W.two_ellipses_4096()
        prob = P.Problem(g, f, ph)
        gU = torch.ones(g.M[0], dtype=torch.float64, device=dev)
        gn = torch.empty(g.N, dtype=torch.complex128, device=dev)
        gs = torch.empty(10, dtype=torch.float64, device=dev)
        for _ in range(2):
            prob.assemble("fp32_ir")
            prob.solve()
            info = P.bie_backward(prob.ctx, prob.omega, gU, np.array(g.ellipses), g_node=gn, g_shape=gs)
        prob.close()
        print("adjoint", info.iters, info.rel_resid)
    elif name == "targets":        # 8192 unknowns, 2e5 grid + 2e4 near targets
        g, f, ph = W.random_geometry(np.random.default_rng(9), 8192)
        zg = W.fluid_grid(g, 500, 400, margin=0.02)
        zn = W.near_boundary_targets(g, 20000, seed=1, max_spacings=2.0)
        prob = P.Problem(g, f, ph)
        prob.assemble("fp32_ir")
        prob.solve()
        # far sums on the grid, then Helsing-Ojala on the near set, twice
        zgt, znt = zt(zg), zt(zn)
        ug, un = torch.empty_like(zgt), torch.empty_like(znt)
        for _ in range(2):
            P.bie_eval_velocity(prob.ctx, prob.omega, zgt, ug, mode=P.VEL_FAR)
            P.bie_eval_velocity(prob.ctx, prob.omega, znt, un, mode=P.VEL_HELSING)
        torch.cuda.synchronize()
        prob.close()
        print("targets", len(zg), len(zn), g.N)
    elif name == "multi":          # 8192 unknowns, fp16-IR, 16 right-hand sides
        g, f, ph = W.random_geometry(np.random.default_rng(9), 8192)
        rng = np.random.default_rng(3)
        PH = torch.as_tensor(np.stack([W.filtered_noise(rng, g.M[0], 0.05, 20)
                                       for _ in range(16)]), device=dev).contiguous()
        prob = P.Problem(g, f, ph)
        prob.assemble("fp16_ir")
        om = torch.empty((16, g.N), dtype=torch.float64, device=dev)
        U = torch.empty((16, g.M[0]), dtype=torch.float64, device=dev)
        for _ in range(2):
            infos = P.bie_solve_multi(prob.ctx, PH, om, U)
        prob.close()
        print("multi", max(i.iters for i in infos), max(i.rel_resid for i in infos))
    elif name == "evolve":         # problem 1 at M_0 = 2048: two RK4 steps with energies
        g, f, ph = W.paper_problem(1, M0=2048, M1=768, Me=1024)
        prob = P.Problem(g, f, ph)
        eta = torch.zeros(g.M[0], dtype=torch.float64, device=dev)
        phit = prob.phit.clone()
        E, info = P.bie_graph_evolve(prob.ctx, eta, phit, 2e-4, 2, filter=True)
        prob.close()
        print("evolve", info.solves, float(abs(E[-1] - E[0]) / abs(E[0])))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--profile-case", choices=["solve", "batch", "adjoint", "targets", "multi",
                                               "evolve"],
                    help="run one small case of a hot kernel (for ncu) and exit")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp16_ir", choices=PRECISIONS)
    ap.add_argument("--rtol", type=float, default=1e-14)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--headline-only", action="store_true",
                    help="time the headline scheme only (no variant table, no other rows); "
                         "for a launch list whose shares match the timed region")
    args = ap.parse_args()
    if args.profile_case:
        return profile_case(args.profile_case)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
