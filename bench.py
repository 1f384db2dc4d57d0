#!/usr/bin/env python
"""Benchmark: FP64-accurate symmetric eigensolves per second at n = 4096 with
the mixed precision Jacobi method (libmpjacobi on one GB300), the plain FP64
Jacobi on the same GPU for the ratio, and the CPU oracle as a baseline.

One step = one mixed solve (validation and norms, FP32 stage, Newton-Schulz,
A_cond, FP64 sweeps, sorted W and Q = Q_d V) of the synthetic n = 4096 matrix
with |eigenvalues| geometric in [1e-6, 1] and random signs, input resident in
HBM, workspace preallocated.  L2 is flushed (a 256 MiB write) between steps;
the solve's working set (0.5 GiB) is larger than L2 anyway.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun: one independent replica per GPU (the single solve
does not shard), weak scaling, value = solves of all ranks / max rank time.
Prints ONE JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "n=4096 FP64-accurate eig solves/s, mixed vs plain FP64 Jacobi, same GB300"
UNIT = "solves/s"
U_D = 2.0 ** -53
FP64_PEAK_TFLOPS = 1.25  # nominal GB300 FP64 (152 SMs x 2 FP64 FMA/clk x 2 flop x ~2.07 GHz)
# DRAM bytes of one FP64 round at n = 4096 come from the committed ncu summary
# of the sweep kernels (a "traffic_bytes_per_round:" line), taken on the kernel
# versions the summary names; see traffic_per_round().
TRAFFIC_PROFILE = os.path.join(ROOT, "profiles", "rr_step64_geo4096.md")
BLOCK_TRAFFIC_PROFILE = os.path.join(ROOT, "profiles", "blk_rmul_geo4096.md")
# Sweep counts of the GPU arm on this input (FP32 stage, FP64 sweeps), used by
# the reference arm only while no full oracle run is recorded.
GPU_ARM_SWEEPS = (9, 11)
WORKLOAD = "geo4096: one symmetric FP64 matrix n=4096, |lam| geometric in [1e-6,1] (condition 1e6), random signs, Haar eigenvectors, seed 0"


def traffic_per_round(path: str = TRAFFIC_PROFILE) -> float | None:
    """dram__bytes_read.sum + dram__bytes_write.sum of one round from an ncu
    summary in profiles/ (its "traffic_bytes_per_round:" line)."""
    try:
        for line in open(path):
            if line.strip().startswith("traffic_bytes_per_round:"):
                return float(line.split(":", 1)[1].split()[0])
    except OSError:
        return None
    return None


def hbm_peak_gbs() -> tuple[float, str]:
    """Measured HBM copy bandwidth (MEASURED_PEAKS.json), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback 6.8 TB/s"


def oracle_record(which: str, workload: str = "geo4096") -> dict | None:
    """The oracle's full run on a recorded workload (oracle/record_geo4096.py)."""
    path = os.path.join(ROOT, "oracle", f"{workload}_{which}.json")
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return None


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.rows: list[list[str]] = []
        self.proc = None
        self.thread = None

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ---------------------------------------------------------------- multi-rank aggregation
def aggregate(value_ms: float, world: int, steps: int, dist=None, device=None) -> tuple[float, float]:
    """Replicas-only scaling: every rank solves its own matrices; the job's time
    is the slowest rank's.  Returns (max_ms over ranks, whole-job solves/s =
    world * steps / max_seconds).  With world == 1 no collective is used."""
    if world > 1 and dist is not None:
        import torch
        t = torch.tensor([value_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        value_ms = float(t.item())
    return value_ms, world * steps / (value_ms / 1000.0)


# ---------------------------------------------------------------- CPU oracle baseline
def cpu_baseline_estimate(A: np.ndarray, sweeps32: int, sweeps64: int, budget_s: float = 15.0) -> dict:
    """Time the oracle (as it stands, one core) on a bounded sample of the n=4096
    workload and extrapolate one full mixed solve:
      T = sweeps32 * N_pairs * t_rot32 + sweeps64 * N_pairs * t_rot64 + 14 n^3 * t_flop,
    t_rot* = seconds per rotation of the oracle's FP32/FP64 cyclic sweep loop
    (first rotations of a sweep on this matrix), t_flop = seconds per flop of
    the oracle's triple-loop product (A times a 16-column slice), 14 n^3 = the
    flops of the oracle's full (non-symmetric) products: Newton-Schulz 2 x 4n^3,
    A_cond 4n^3, Q_d V 2n^3."""
    import oracle
    n = A.shape[0]
    npairs = n * (n - 1) / 2
    per = budget_s / 3.0
    # calibrate counts from a short probe, then run about `per` seconds each
    t = oracle.sample_rotations(A, 50, np.float32)
    k32 = max(50, int(50 * per / max(t, 1e-6)))
    t32 = oracle.sample_rotations(A, k32, np.float32) / k32
    t = oracle.sample_rotations(A, 50, np.float64)
    k64 = max(50, int(50 * per / max(t, 1e-6)))
    t64 = oracle.sample_rotations(A, k64, np.float64) / k64
    cols = 16
    B = np.asfortranarray(np.random.default_rng(0).standard_normal((n, cols)))
    tg = oracle.sample_gemm(A, B)
    tflop = tg / (2.0 * n * n * cols)
    T = sweeps32 * npairs * t32 + sweeps64 * npairs * t64 + 14.0 * n ** 3 * tflop
    return {"value": 1.0 / T, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"oracle on the n={n} input: {k32} FP32 + {k64} FP64 cyclic rotations and one "
                       f"{n}x{n}x{cols} product, extrapolated to {sweeps32}+{sweeps64} sweeps and 14n^3 product "
                       f"flops (seconds per solve {T:.4g})"),
            "seconds_per_solve": T, "t_rot32_s": t32, "t_rot64_s": t64, "t_flop_s": tflop}


def oracle_sweep_counts(fallback: tuple[int, int] | None = None) -> tuple[int, int, str]:
    """The oracle's own sweep counts on the n = 4096 input (FP32 cyclic stage,
    FP64 cyclic sweeps), from its full run recorded by oracle/record_geo4096.py;
    without that record, `fallback` (labelled as such)."""
    rec = oracle_record("mixed")
    if rec is not None:
        return int(rec["sweeps32"]), int(rec["sweeps64"]), "the oracle's full n=4096 run (oracle/geo4096_mixed.json)"
    if fallback is None:
        raise SystemExit("oracle/geo4096_mixed.json missing: run oracle/record_geo4096.py mixed")
    return fallback[0], fallback[1], "GPU arm's sweep counts (no full oracle run recorded)"


def run_reference(args) -> None:
    """--impl reference: the CPU oracle as it stands, timed on the host."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2509_00495_gb300 import inputs
    A, lam = inputs.geo_4096(seed=0)
    s32, s64, _src = oracle_sweep_counts(GPU_ARM_SWEEPS)
    for _ in range(args.warmup):
        cpu_baseline_estimate(A, s32, s64, budget_s=2.0)
    vals, t0 = [], time.perf_counter()
    est = None
    for _ in range(args.steps):
        est = cpu_baseline_estimate(A, s32, s64, budget_s=args.ref_step_seconds)
        vals.append(est["value"])
    wall = time.perf_counter() - t0
    value = statistics.median(vals)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * wall / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": 4096, "method": "oracle mixed (FP32 cyclic stage, "
                       "Newton-Schulz, FP64 cyclic sweeps), extrapolated from bounded samples"},
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": est["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def oracle_full_runs() -> dict:
    """The oracle run in full: the n = 96 solve of the small geometric case,
    timed here on one host core, and the recorded full n = 4096 runs."""
    import oracle
    from paper_2509_00495_gb300 import inputs
    A, lam = inputs.small_geo(seed=0)
    t0 = time.perf_counter()
    reps = 0
    while True:
        W, Q, info = oracle.syev_mixed(A)
        reps += 1
        if time.perf_counter() - t0 > 1.0:
            break
    t96 = (time.perf_counter() - t0) / reps
    out = {"n96_mixed": {"seconds_per_solve": t96, "solves_per_s": 1.0 / t96, "sweeps32": info.sweeps32,
                         "sweeps64": info.sweeps64, "cores": 1}}
    # the differentiation workload (64 x n = 512): the oracle's adjoint on two
    # of its matrices (eigenvectors from LAPACK as inputs), scaled to 64
    mats, lams, dWs, dQs = inputs.backward_batch(count=2)
    tb = 0.0
    for Ab, dWb, dQb in zip(mats, dWs, dQs):
        w, q = np.linalg.eigh(Ab)
        t0 = time.perf_counter()
        oracle.eigh_backward(w, np.asfortranarray(q), dWb, dQb)
        tb += time.perf_counter() - t0
    out["backward_64x512"] = {"seconds": tb * 32, "batches_per_s": 1.0 / (tb * 32), "cores": 1,
                              "sample": "the oracle adjoint on 2 of the 64 matrices, scaled to 64"}
    for which in ("mixed", "plain"):
        rec = oracle_record(which)
        if rec is not None:
            out[f"n4096_{which}_recorded"] = {k: rec[k] for k in ("sweeps32", "sweeps64", "wall_seconds", "machine")
                                              if k in rec}
    for which in ("mixed", "plain"):
        rec = oracle_record(which, "clustered1024")
        if rec is not None:
            out[f"n1024_{which}_recorded"] = {k: rec[k] for k in ("sweeps32", "sweeps64", "wall_seconds", "machine")
                                              if k in rec}
    return out


# ---------------------------------------------------------------- GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 Jacobi timing")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched and backward workloads")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end timing")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-step-seconds", type=float, default=8.0)
    ap.add_argument("--plain-solves", type=int, default=3)
    ap.add_argument("--sweep-only", choices=["round_robin", "block", "cyclic"], default=None,
                    help="time FP64 sweeps (mpj_jacobi64) of one ordering on a nearly diagonal n x n matrix; "
                         "for profiling")
    ap.add_argument("--product-only", action="store_true",
                    help="time only the FP64-accurate tensor-core product (n x n x n, mpj_dgemm_tc); for profiling")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2509_00495_gb300 import build as mpj_build
    mpj_build.build()
    from paper_2509_00495_gb300 import inputs, mpj

    n = args.n
    if args.product_only:
        product_only(mpj, torch, dev, n, args)
        return
    if args.sweep_only:
        sweep_only(mpj, torch, dev, inputs, n, args)
        return
    A_np, lam = inputs.geo_4096(seed=0, n=n) if n == 4096 else inputs.geo_matrix(n, 1e6, seed=0)
    A = torch.from_numpy(A_np).to(dev)
    ws = torch.empty(mpj.syev_workspace(n), dtype=torch.uint8, device=dev)
    ws2 = None if args.no_extras else torch.empty(mpj.syev_workspace(n, precond_passes=2), dtype=torch.uint8,
                                                  device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    # warm-up
    infos = []
    for _ in range(args.warmup):
        r = mpj.syev_ex(A, workspace=ws)
        infos.append(r.info)
    torch.cuda.synchronize()

    # timed region: exactly K steps
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        uuid = None
    sampler = ClockSampler(uuid)
    sampler.start()
    time.sleep(0.3)
    launches0 = mpj.lib().mpj_kernel_launches()
    step_ms, step_info = [], []
    barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record()
    for k in range(args.steps):
        if k:
            flush.zero_()
        e_a = torch.cuda.Event(enable_timing=True)
        e_b = torch.cuda.Event(enable_timing=True)
        e_a.record()
        r = mpj.syev_ex(A, workspace=ws)
        e_b.record()
        e_b.synchronize()
        step_ms.append(e_a.elapsed_time(e_b))
        step_info.append(r.info)
    ev1.record()
    torch.cuda.synchronize()
    barrier()
    total_ms = ev0.elapsed_time(ev1)
    launches = mpj.lib().mpj_kernel_launches() - launches0
    clocks = sampler.stop()
    total_ms, value = aggregate(total_ms, world, args.steps, dist if world > 1 else None, dev)
    W_last, Q_last = r.W, r.Q

    # accuracy of the timed result (outside the timed region)
    with torch.no_grad():
        be = (torch.linalg.norm(A - (Q_last * W_last) @ Q_last.T) / torch.linalg.norm(A)).item() / (n * U_D)
        orF = torch.linalg.norm(Q_last.T @ Q_last - torch.eye(n, dtype=torch.float64, device=dev)).item() / (n * U_D)
        ew = (W_last - torch.from_numpy(np.sort(lam)).to(dev)).abs().max().item() / float(np.abs(lam).max())
    accuracy = {"backward_err_over_nu": be, "orth_fro_over_nu": orF, "eig_err_over_normA": ew,
                "bound_over_nu": 4.0}

    # end to end through the public API with host buffers
    A_host = torch.from_numpy(A_np).pin_memory()
    W_host = torch.empty(n, dtype=torch.float64).pin_memory()
    Q_host = torch.empty(n, n, dtype=torch.float64).pin_memory()
    A_e2e = torch.empty_like(A)
    e2e_steps = 0 if args.no_e2e else max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        A_e2e.copy_(A_host, non_blocking=True)
        re = mpj.syev_ex(A_e2e, workspace=ws)
        W_host.copy_(re.W, non_blocking=True)
        Q_host.copy_(re.Q, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    if e2e_steps:
        e2e_ms, e2e_value = aggregate(e2e_s * 1000.0, world, e2e_steps, dist if world > 1 else None, dev)
    else:
        e2e_value = None
    e2e = {"value": e2e_value, "unit": UNIT,
           "h2d_bytes_per_step": n * n * 8, "d2h_bytes_per_step": n * 8 + n * n * 8}

    info = step_info[-1]
    ms_mixed = statistics.median(step_ms)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
           "config": {"workload": WORKLOAD, "n": n, "method": "mixed (Algorithm 9): FP32 block round-robin "
                      "Jacobi, 2 Newton-Schulz steps and Q_d^T A Q_d as FP64-accurate tensor-core products, FP64 "
                      "Jacobi sweeps in block round-robin order with tensor-core block updates",
                      "tol": "n 2^-53 ||A||_F", "l2": "flushed between steps (256 MiB write); working set 0.5 GiB",
                      "parallelism": f"replicas x{world}"},
           "clocks": clocks, "gpu_launches": launches, "e2e": e2e, "accuracy": accuracy,
           "sweeps": {"stage1_fp32": info["sweeps32"], "fp64": info["sweeps64"], "paper_claim": "< 10"},
           "stage_ms": dict(zip(["stage1_fp32", "newton_schulz", "transform", "fp64_sweeps", "finalize", "total"],
                                [round(x, 3) for x in info["ms_stage"]]))}

    # roofline of the dominant kernel, per round of the FP64 sweeps
    sweeps64 = info["sweeps64"]
    st = info["ms_stage"]
    if sweeps64 > 0:
        N32 = (n + 31) // 32 * 32
        npairs = N32 // 32
        rounds = sweeps64 * (N32 // 16 - 1)
        round_s = st[3] / 1000.0 / rounds
        # one outer round of the block ordering: blk_solve (FP64 subproblems), then three
        # block-diagonal right multiplications on the tensor cores (V U~, A U~ into B, B^T U~
        # into A).  Algorithmic bytes: a round must read and write the column panels of A and
        # V that its rotations change, 32 n^2 bytes when every block pair rotates (one pass
        # over A and V, the fused lower bound); block pairs without rotations need nothing,
        # so the bytes are 32 n^2 x (rotated block pairs / block pairs), summed over rounds.
        rb = int(info.get("rotated_blocks64") or 0)
        bytes_total = 32.0 * n * n * rb / npairs
        bytes_round = bytes_total / rounds
        peak, peak_src = hbm_peak_gbs()
        achieved = bytes_total / (st[3] / 1000.0) / 1e9
        out["roofline"] = {"kernel": "blk_rmul x3 + blk_solve (one outer round of the block ordering)",
                           "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                           "frac": achieved / peak,
                           "traffic": traffic_per_round(BLOCK_TRAFFIC_PROFILE) if n == 4096 else None,
                           "peak_source": peak_src, "algorithmic_bytes_per_round": bytes_round,
                           "rotated_block_fraction": rb / (rounds * npairs),
                           "avg_round_ms": round_s * 1e3, "rounds": rounds, "dominant_stage": "fp64_sweeps",
                           "share_of_step": st[3] / st[5] if st[5] else None,
                           "note": "integer-ALU and latency bound (digit slicing and the exact epilogue); "
                                   "see profiles/blk_rmul_geo4096.md"}
    # GEMM stage rate (Newton-Schulz + transform: 6n^3 + 3n^3 algorithmic FP64 flops), on the
    # tensor cores from exact bf16 slices unless MPJ_GEMM_TC=0 selects the FP64 DMMA kernel
    if st[1] + st[2] > 0:
        tc = os.environ.get("MPJ_GEMM_TC", "1") != "0"
        out["gemm_fp64"] = {"achieved_tflops": 9.0 * n ** 3 / ((st[1] + st[2]) / 1000.0) / 1e12,
                            "unit": "FP64-equivalent TFLOP/s (algorithmic FP64 flops / time)",
                            "engine": "tcgen05 bf16 exact slices" if tc else "FP64 DMMA",
                            "fp64_pipe_peak": FP64_PEAK_TFLOPS, "stages": "newton_schulz + transform"}

    if rank == 0 and not args.no_plain:
        # the metric's denominator: plain FP64 Jacobi from V = I on the same input and
        # sweep kernels, timed like the mixed arm (L2 flushed before each solve), median of 3
        ms_p = []
        for _ in range(args.plain_solves):
            flush.zero_()
            torch.cuda.synchronize()
            e_a = torch.cuda.Event(enable_timing=True)
            e_b = torch.cuda.Event(enable_timing=True)
            e_a.record()
            rp = mpj.syev_ex(A, workspace=ws, method="plain")
            e_b.record()
            e_b.synchronize()
            ms_p.append(e_a.elapsed_time(e_b))
        ms_plain = statistics.median(ms_p)
        with torch.no_grad():
            bep = (torch.linalg.norm(A - (rp.Q * rp.W) @ rp.Q.T) / torch.linalg.norm(A)).item() / (n * U_D)
            orp = torch.linalg.norm(rp.Q.T @ rp.Q - torch.eye(n, dtype=torch.float64, device=dev)).item() / (n * U_D)
        out["plain"] = {"ms_per_solve": ms_plain, "solves": len(ms_p), "ms_all": [round(x, 1) for x in ms_p],
                        "sweeps64": rp.info["sweeps64"], "status": rp.status,
                        "backward_err_over_nu": bep, "orth_fro_over_nu": orp}
        out["speedup_vs_plain"] = ms_plain / ms_mixed

    if rank == 0 and not args.no_extras:
        # the same workload with the optional second preconditioning pass (not in the paper)
        r2 = mpj.syev_ex(A, workspace=ws2, precond_passes=2)
        torch.cuda.synchronize()
        ms2 = []
        for _ in range(2):
            flush.zero_()
            e_a = torch.cuda.Event(enable_timing=True)
            e_b = torch.cuda.Event(enable_timing=True)
            e_a.record()
            r2 = mpj.syev_ex(A, workspace=ws2, precond_passes=2)
            e_b.record()
            e_b.synchronize()
            ms2.append(e_a.elapsed_time(e_b))
        with torch.no_grad():
            be2 = (torch.linalg.norm(A - (r2.Q * r2.W) @ r2.Q.T) / torch.linalg.norm(A)).item() / (n * U_D)
            or2 = torch.linalg.norm(r2.Q.T @ r2.Q - torch.eye(n, dtype=torch.float64, device=dev)).item() / (n * U_D)
        out["mixed_2pass"] = {"ms_per_solve": min(ms2), "solves_per_s": 1000.0 / min(ms2),
                              "sweeps": {"stage1_fp32": r2.info["sweeps32"], "stage1_pass2": r2.info["sweeps32_pass2"],
                                         "fp64": r2.info["sweeps64"]},
                              "stage_ms": [round(x, 3) for x in r2.info["ms_stage"]],
                              "backward_err_over_nu": be2, "orth_fro_over_nu": or2}
        if "plain" in out:
            out["mixed_2pass"]["speedup_vs_plain"] = out["plain"]["ms_per_solve"] / min(ms2)
        # the paper's own ordering (cyclic-by-row, Sec. 3.3) for the FP64 sweeps, one solve
        ws_c = ws
        flush.zero_()
        torch.cuda.synchronize()
        e_a = torch.cuda.Event(enable_timing=True)
        e_b = torch.cuda.Event(enable_timing=True)
        e_a.record()
        rc = mpj.syev_ex(A, workspace=ws_c, ordering="cyclic")
        e_b.record()
        e_b.synchronize()
        with torch.no_grad():
            bec = (torch.linalg.norm(A - (rc.Q * rc.W) @ rc.Q.T) / torch.linalg.norm(A)).item() / (n * U_D)
            orc = torch.linalg.norm(rc.Q.T @ rc.Q - torch.eye(n, dtype=torch.float64, device=dev)).item() / (n * U_D)
        out["mixed_cyclic"] = {"ms_per_solve": e_a.elapsed_time(e_b), "status": rc.status,
                               "sweeps": {"stage1_fp32": rc.info["sweeps32"], "fp64": rc.info["sweeps64"]},
                               "stage_ms": [round(x, 3) for x in rc.info["ms_stage"]],
                               "backward_err_over_nu": bec, "orth_fro_over_nu": orc,
                               "ordering": "cyclic-by-row (the paper's), run as wavefronts of pairs with equal p+q"}
        # the same solve with the scalar round-robin FP64 sweeps (rr_step64 + v_apply_rounds)
        ws_r = torch.empty(mpj.syev_workspace(n, ordering="round_robin"), dtype=torch.uint8, device=dev)
        flush.zero_()
        torch.cuda.synchronize()
        e_a = torch.cuda.Event(enable_timing=True)
        e_b = torch.cuda.Event(enable_timing=True)
        e_a.record()
        rr = mpj.syev_ex(A, workspace=ws_r, ordering="round_robin")
        e_b.record()
        e_b.synchronize()
        del ws_r
        strr = rr.info["ms_stage"]
        rounds_rr = rr.info["sweeps64"] * (n - 1)
        out["mixed_round_robin"] = {
            "ms_per_solve": e_a.elapsed_time(e_b), "status": rr.status,
            "sweeps": {"stage1_fp32": rr.info["sweeps32"], "fp64": rr.info["sweeps64"]},
            "stage_ms": [round(x, 3) for x in strr],
            "fp64_round": {"kernel": "rr_step64+v_apply_rounds", "bound": "alu",
                           "achieved_tflops": 4.0 * n * n / (strr[3] / 1000.0 / rounds_rr) / 1e12 if rounds_rr else None,
                           "peak_tflops": FP64_PEAK_TFLOPS,
                           "traffic_per_round": traffic_per_round() if n == 4096 else None}}
        out["extras"] = extras(mpj, torch, dev, inputs)

    if rank == 0 and world == 1 and not args.no_cpu:
        s32, s64, _src = oracle_sweep_counts(GPU_ARM_SWEEPS)
        out["cpu_baseline"] = cpu_baseline_estimate(A_np, s32, s64, args.cpu_seconds)
        out["cpu_baseline"]["note"] = "a baseline, not the target"
        out["cpu_baseline"]["full_runs"] = oracle_full_runs()

    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def sweep_only(mpj, torch, dev, inputs, n: int, args) -> None:
    """`--warmup` then `--steps` single FP64 sweeps (mpj_jacobi64, max_sweeps 1)
    of the chosen ordering on A = Q diag(lam) Q^T, Q within 1e-4 of I, lam
    uniform in [-1, 1] (like the matrix the sweeps receive after
    preconditioning), each on a fresh copy; CUDA-event timed; one JSON line."""
    rng = np.random.default_rng(0)
    lam = np.sort(rng.uniform(-1.0, 1.0, n))
    A0 = torch.from_numpy(inputs.near_diagonal(n, lam, 1e-4, seed=0)).to(dev)
    tol = float(n * U_D * torch.linalg.norm(A0).item())
    ms = []
    for i in range(args.warmup + args.steps):
        A = A0.clone()
        torch.cuda.synchronize()
        e_a = torch.cuda.Event(enable_timing=True)
        e_b = torch.cuda.Event(enable_timing=True)
        e_a.record()
        _, _, sw, off, st = mpj.jacobi64(A, tol=tol, ordering=args.sweep_only, max_sweeps=1)
        e_b.record()
        e_b.synchronize()
        if i >= args.warmup:
            ms.append(e_a.elapsed_time(e_b))
    t = statistics.median(ms) if ms else float("nan")
    print(json.dumps({"kernel": f"FP64 sweep ({args.sweep_only})", "n": n, "ms_per_sweep": t, "sweeps": sw,
                      "off_after": off, "status": st}), flush=True)


def product_only(mpj, torch, dev, n: int, args) -> None:
    """`--warmup` then `--steps` products C = A B of n x n FP64 matrices on the
    tensor-core exact-slice engine (mpj_dgemm_tc: slicing of both operands and
    the product kernel), CUDA-event timed; prints one JSON line."""
    g = torch.Generator(device="cpu").manual_seed(0)
    A = torch.randn(n, n, dtype=torch.float64, generator=g).to(dev)
    B = torch.randn(n, n, dtype=torch.float64, generator=g).to(dev)
    for _ in range(args.warmup):
        mpj.dgemm_tc("N", "N", 1.0, A, B)
    torch.cuda.synchronize()
    ms = []
    for _ in range(args.steps):
        e_a = torch.cuda.Event(enable_timing=True)
        e_b = torch.cuda.Event(enable_timing=True)
        e_a.record()
        C = mpj.dgemm_tc("N", "N", 1.0, A, B)
        e_b.record()
        e_b.synchronize()
        ms.append(e_a.elapsed_time(e_b))
    err = ((C - A @ B).abs().max() / (A.abs() @ B.abs()).max()).item()
    t = statistics.median(ms) if ms else float("nan")
    print(json.dumps({"kernel": "mpj_dgemm_tc", "n": n, "ms_per_product": t,
                      "fp64_equiv_tflops": 2.0 * n ** 3 / (t / 1000.0) / 1e12,
                      "bf16_tensor_tflops": 36 * 2.0 * n ** 3 / (t / 1000.0) / 1e12,
                      "max_err_over_abs_product": err}), flush=True)


def extras(mpj, torch, dev, inputs) -> dict:
    """The batched workload (2048 matrices, n uniform in [8, 256]) and the
    backward workload (64 matrices n = 512), each timed once after a warm-up."""
    res = {}
    sizes, mats = inputs.batch_goe(2048, 8, 256, seed=0)
    dmats = [torch.from_numpy(a).to(dev) for a in mats]
    solver = mpj.BatchedSolver(sizes, device=dev)
    t0 = time.perf_counter()
    solver.solve(dmats)  # first call: plan, autotune the group size, capture the graph
    torch.cuda.synchronize()
    t_plan = time.perf_counter() - t0
    reps = []
    for _ in range(2):  # graph replays (inputs already in the solver's buffers)
        e_a = torch.cuda.Event(enable_timing=True)
        e_b = torch.cuda.Event(enable_timing=True)
        e_a.record()
        Ws, Qs, sw, st = solver.solve()
        e_b.record()
        e_b.synchronize()
        reps.append(e_a.elapsed_time(e_b) / 1000.0)
    dt = min(reps)
    res["batched"] = {"matrices": len(dmats), "seconds": dt, "matrices_per_s": len(dmats) / dt,
                      "first_call_s_incl_planning": t_plan, "group_size": solver.group_size(),
                      "sum_n3": float(np.sum(sizes.astype(np.float64) ** 3)), "max_sweeps64": int(max(sw)),
                      "mean_sweeps64": float(np.mean(sw)), "status": st}
    mats5, lams5, dW5, dQ5 = inputs.backward_batch(64, 512, seed=0, grad_seed=1)
    Wb, Qb = [], []
    for a in mats5:
        r = mpj.syev_ex(torch.from_numpy(a).to(dev))
        Wb.append(r.W)
        Qb.append(r.Q)
    W = torch.stack(Wb)
    Q = torch.stack(Qb)
    dW = torch.from_numpy(np.stack(dW5)).to(dev)
    dQ = torch.from_numpy(np.stack(dQ5)).to(dev)
    mpj.syev_backward(W, Q, dW, dQ)
    torch.cuda.synchronize()
    e_a = torch.cuda.Event(enable_timing=True)
    e_b = torch.cuda.Event(enable_timing=True)
    e_a.record()
    mpj.syev_backward(W, Q, dW, dQ)
    e_b.record()
    e_b.synchronize()
    ms = e_a.elapsed_time(e_b)
    res["backward"] = {"matrices": 64, "n": 512, "ms": ms, "batches_per_s": 1000.0 / ms,
                       "achieved_tflops": 64 * 5.0 * 512 ** 3 / (ms / 1000.0) / 1e12}
    return res


if __name__ == "__main__":
    main()
