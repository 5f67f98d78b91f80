"""Benchmark of the dose calculation hot path on GB300.

One step = one dose evaluation d = A x (dose_spmv) plus one dose+gradient
evaluation of the quadratic objective (dose_pg_step: fused d, f, A^T r and the
projected-gradient update) on the clinical-size pencil-beam matrix
(256x256x160 voxels x 4000 spots, ~1.5e8 entries, uint16 values + one FP32
scale, uint32 indices).  Inputs are resident in HBM when the timed region
starts; A (~1 GB) is larger than the 129 MB L2, so every step streams it from
HBM.  Prints one JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
    python bench.py --workload batched [--steps K]   # 27 scenario matrices x 16 vectors
    python bench.py --workload precision             # u16 / BF16 / FP8 / F16 / F32, plain and compensated
    python bench.py --workload halfdouble            # the paper's Half/double: F16 values, FP64 x and d
    python bench.py --workload robust                # 3-beam plan x 9 setup shifts: robust objective + PG step
    python bench.py --workload sell                  # dose eval on SELL-32-sigma copies, sigma sweep, vs CSR
    python bench.py --workload liver1                # the paper's Liver 1 shape (2.97e6 x 6.8e4, 1.48e9 entries)

--impl reference times the FP64 CPU oracle (the reference arm of this
project) on the same workload and metric.  Under torchrun (N > 1) every rank
runs an independent replica on its own GPU (weak scaling; no collective on the
data path) and rank 0 reports the whole-job throughput.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import dosegen  # noqa: E402

METRIC = "dose SpMV effective HBM GB/s (% of GB300 peak) and ms per dose+gradient eval"
WORKLOAD = "clinical pencil beam 256x256x160 voxels x 4000 spots, 1.5e8 entries, u16+scale, u32 indices"
GPU_STEP = ("dose eval d = A x, then dose+gradient eval: d, FP64 f = sum w (d-p)^2, g = A^T[2w(d-p)] and the "
            "projected-gradient update x <- max(0, x - eta g)")
REF_STEP = "FP64 d = A x, then FP64 f and g = A^T[2w(d-p)] on a row block (no projected-gradient update)"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


def max_over_ranks(ms: float, device=None) -> float:
    """The slowest rank's time (all ranks get it); the value itself with one rank."""
    import torch
    import torch.distributed as td

    if not (td.is_available() and td.is_initialized()) or td.get_world_size() == 1:
        return ms
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    td.all_reduce(t, op=td.ReduceOp.MAX)
    return float(t.item())


def whole_job_gbs(bytes_per_step: int, steps: int, world_size: int, max_ms: float) -> float:
    """Whole-job throughput of `world_size` replicas, each doing `steps` steps of
    `bytes_per_step` algorithmic bytes, timed by the slowest rank."""
    return world_size * bytes_per_step * steps / (max_ms * 1e-3) / 1e9


def _pinned_like(t):
    """A page-locked host copy of t, allocated page-locked from the start (on the
    Grace host, device-to-host copies into buffers pinned after allocation,
    Tensor.pin_memory(), ran at about half the link rate)."""
    import torch
    h = torch.empty(t.shape, dtype=t.dtype, pin_memory=True)
    h.copy_(t)
    return h


AUTOTUNE_CACHE = os.path.join(ROOT, "paper_2103_09683_gb300", "tuning", "autotune_gb300.json")


def _autotune(A, x, args, purposes):
    """Knobs for this handle from the autotune cache (dose_autotune_cached),
    outside any timed region; with --tuning the given knobs are kept as they are."""
    if args.tuning or args.autotune == "off":
        return {"source": "off"}
    r = A.autotune(x, mode=args.autotune, purposes=purposes, cache=args.autotune_cache)
    return {"source": r["source"], "purposes": list(purposes),
            "cache": os.path.relpath(args.autotune_cache, ROOT), "fingerprint": f"{r['fingerprint']:016x}",
            "sweep_ms": {"forward": round(r["ms_forward"], 4), "fused": round(r["ms_fused"], 4),
                         "batched": round(r["ms_batched"], 4)}}


def _traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if the sources the
    kernel depends on are the ones it was captured from."""
    try:
        import paper_2103_09683_gb300._build as b
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            tab = json.load(f)
        ent = tab.get(kernel)
        if ent and ent.get("inputs_sha256") == b._inputs_digest(ent.get("sources")):
            return float(ent["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


def _tuning_kv(args) -> dict:
    """--tuning "k=v,k=v" as a dict of schedule knobs."""
    return {k: int(v) for k, v in (kv.split("=") for kv in args.tuning.split(","))} if args.tuning else {}


def setup_workload(device):
    """Clinical beam on the device: handle, x, p, w and the PG step size."""
    import torch

    import paper_2103_09683_gb300 as dose

    beam = dosegen.CLINICAL
    csr = dosegen.generate(beam)
    A = dose.DoseMatrix.from_csr(csr.row_ptr, csr.col, ncols=csr.ncols, fmt="u16", values_f64=csr.val)
    p, w = dosegen.ellipsoid_target(beam, semi_axes=(30.0, 20.0, 16.0))
    x = dosegen.spot_weights(csr.ncols, dosegen.weight_seed(beam))
    # step size 1/L with L = 2 max(w) ||A||_1 ||A||_inf >= the gradient's Lipschitz constant
    cs = np.concatenate([[0.0], np.cumsum(csr.val)])
    rp = csr.row_ptr.astype(np.int64)
    absrow = cs[rp[1:]] - cs[rp[:-1]]
    del cs
    abscol = np.bincount(csr.col, weights=csr.val, minlength=csr.ncols)
    eta = 1.0 / (2.0 * float(w.max()) * float(absrow.max()) * float(abscol.max()))
    t = lambda a: torch.from_numpy(a).to(device)
    return csr, A, t(x), t(p), t(w), eta


def run_gpu(args):
    import torch

    import paper_2103_09683_gb300 as dose

    ws, rank, local = _dist()
    dose.build()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as td
        td.init_process_group("nccl", device_id=device)
    csr, A, x, p, w, eta = setup_workload(device)
    if args.tuning:
        A.set_tuning(**_tuning_kv(args))
    tuned = _autotune(A, x, args, ("forward", "fused"))
    info = A.info()
    stream = torch.cuda.current_stream()
    d = torch.empty(A.nrows, dtype=torch.float32, device=device)
    f = torch.empty(1, dtype=torch.float64, device=device)
    x0 = x.clone()

    def step():
        A.spmv(x, d)
        A.pg_step(x, p, w, eta, f=f)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    x.copy_(x0)
    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    e_start, e_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    e_start.record(stream)
    for k in range(K):
        ev[k][0].record(stream)
        A.spmv(x, d)
        ev[k][1].record(stream)
        A.pg_step(x, p, w, eta, f=f)
        ev[k][2].record(stream)
    e_end.record(stream)
    torch.cuda.synchronize()
    time.sleep(0.2)
    clk = clocks.stop()
    total_ms = e_start.elapsed_time(e_end)
    spmv_all = [ev[k][0].elapsed_time(ev[k][1]) for k in range(K)]
    grad_all = [ev[k][1].elapsed_time(ev[k][2]) for k in range(K)]
    spmv_ms, grad_ms = sum(spmv_all) / K, sum(grad_all) / K
    total_ms = max_over_ranks(total_ms, device)
    A.device_status()

    # End to end through the public API with host buffers: every step copies x in
    # from pinned host memory, runs both calls, and copies its dose d and
    # objective f out to pinned host memory.  The read-back of step k runs on a
    # copy stream while step k + 1 computes (d and f double-buffered; a buffer
    # is reused only after its copy has landed); the timed region ends when the
    # last copy has landed.
    xh = _pinned_like(x0)
    d_dev = [d, torch.empty_like(d)]
    f_dev = [f, torch.empty_like(f)]
    dh = [torch.empty(A.nrows, dtype=torch.float32, pin_memory=True) for _ in range(2)]
    fh = [torch.empty(1, dtype=torch.float64, pin_memory=True) for _ in range(2)]
    copy_stream = torch.cuda.Stream(device=device)
    ready = [torch.cuda.Event() for _ in range(2)]
    landed = [torch.cuda.Event() for _ in range(2)]
    ke = max(3, min(K, 50))

    def e2e_steps(n):
        for k in range(n):
            b = k & 1
            if k >= 2:
                stream.wait_event(landed[b])
            x.copy_(xh, non_blocking=True)
            A.spmv(x, d_dev[b])
            A.pg_step(x, p, w, eta, f=f_dev[b])
            ready[b].record(stream)
            copy_stream.wait_event(ready[b])
            with torch.cuda.stream(copy_stream):
                dh[b].copy_(d_dev[b], non_blocking=True)
                fh[b].copy_(f_dev[b], non_blocking=True)
            landed[b].record(copy_stream)
        stream.wait_stream(copy_stream)

    e2e_steps(4)
    torch.cuda.synchronize()
    e2 = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    e2[0].record(stream)
    e2e_steps(ke)
    e2[1].record(stream)
    torch.cuda.synchronize()
    e2e_ms = e2[0].elapsed_time(e2[1]) / ke

    # Algorithmic bytes of the fused pass: the CSR byte model of the measurement
    # plan (stored values and 32-bit indices once, row pointers, p and w, x in,
    # g out, the CTA partials written and read once).  On the row-group layout
    # the kernel moves fewer bytes (its own model is reported beside it).
    fused_csr = csr_fused_bytes(info)
    step_bytes = info["spmv_bytes"] + fused_csr
    value = whole_job_gbs(step_bytes, K, ws, total_ms)
    peak, peak_kind = _peaks()
    spmv_gbs = info["spmv_bytes"] / (spmv_ms * 1e-3) / 1e9
    grad_gbs = fused_csr / (grad_ms * 1e-3) / 1e9
    rg = info["adj_layout_fused"] == 2
    fused_name = "rg_kernel+rg_finalize" if rg else "adjoint_kernel+finalize"
    fwd_rg = info["spmv_layout"] == 2
    spmv_name = "rg_spmv_kernel" if fwd_rg else "spmv_kernel"
    spmv_entry = {"ms": round(spmv_ms, 5), "bytes": info["spmv_bytes"],
                  "achieved_gbs": round(spmv_gbs, 1), "frac": round(spmv_gbs / peak, 4),
                  "layout": "row groups" if fwd_rg else "CSR", "traffic": _traffic(spmv_name)}
    if fwd_rg:
        own = info["rg_spmv_bytes"]
        spmv_entry.update({"own_bytes": own, "own_gbs": round(own / (spmv_ms * 1e-3) / 1e9, 1),
                           "own_frac": round(own / (spmv_ms * 1e-3) / 1e9 / peak, 4)})
    kernels = {
        spmv_name: spmv_entry,
        fused_name: {"ms": round(grad_ms, 5), "bytes": fused_csr, "achieved_gbs": round(grad_gbs, 1),
                     "frac": round(grad_gbs / peak, 4),
                     "layout": "row groups" if rg else "CSR",
                     "own_bytes": info["fused_bytes"],
                     "own_gbs": round(info["fused_bytes"] / (grad_ms * 1e-3) / 1e9, 1),
                     "own_frac": round(info["fused_bytes"] / (grad_ms * 1e-3) / 1e9 / peak, 4),
                     "traffic": _traffic("rg_kernel" if rg else "adjoint_kernel")},
    }
    dom = max(kernels, key=lambda k: kernels[k]["ms"])
    roof = {"bound": "hbm", "kernel": dom, "achieved": kernels[dom]["achieved_gbs"], "peak": peak,
            "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
            else "fallback 6.8 TB/s", "unit": "GB/s", "frac": kernels[dom]["frac"],
            "traffic": kernels[dom]["traffic"]}
    if "own_bytes" in kernels[dom]:
        roof.update({"note": "achieved = the CSR byte model of the call / its time (the paper's effective "
                             "bandwidth); the row-group layout reads own_bytes, of which own_frac is the "
                             "fraction of the measured peak",
                     "own_bytes": kernels[dom]["own_bytes"], "own_frac": kernels[dom]["own_frac"]})
    out = {
        "metric": METRIC, "value": round(value, 1), "unit": "GB/s", "n_gpus": ws, "steps": K,
        "warmup": args.warmup, "ms_per_step": round(total_ms / K, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "nrows": A.nrows, "ncols": A.ncols, "nnz": A.nnz,
                   "format": "u16+scale", "bytes_per_step": step_bytes, "step": GPU_STEP,
                   "l2": "inputs larger than L2 (A streams ~1 GB per call; L2 129 MB)",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
        "ms_per_dose_eval": round(spmv_ms, 5),
        "ms_per_dose_grad_eval": round(grad_ms, 5),
        "ms_stats": {"dose_eval": {"mean": round(spmv_ms, 5), "median": round(statistics.median(spmv_all), 5),
                                   "min": round(min(spmv_all), 5)},
                     "dose_grad_eval": {"mean": round(grad_ms, 5), "median": round(statistics.median(grad_all), 5),
                                        "min": round(min(grad_all), 5)}},
        "pct_of_nominal_8tbs": round(100 * spmv_gbs / 8000.0, 1),
        "kernels": kernels,
        "roofline": roof,
        "e2e": {"value": round(step_bytes / (e2e_ms * 1e-3) / 1e9, 1), "unit": "GB/s",
                "ms_per_step": round(e2e_ms, 4), "h2d_bytes_per_step": 4 * A.ncols,
                "d2h_bytes_per_step": 4 * A.nrows + 8,
                "note": "pinned host buffers; step k's d and f copied out while step k+1 computes"},
        "gpu_launches": 3 * K,
        "clocks": clk,
        "tuning": info["tuning"],
        "autotuned": tuned["source"] != "off",
        "autotune": tuned,
        "fused_layout": {"name": "row groups" if rg else "CSR", "groups": info["rg_groups"],
                         "union_entries": info["rg_union_entries"], "window": info["rg_window"],
                         "workers": info["rg_warps_fused"], "index_bytes": info["rg_index_bytes"],
                         "bytes_per_entry": round(info["fused_bytes"] / A.nnz, 3),
                         "csr_bytes_per_entry": round(fused_csr / A.nnz, 3)},
    }
    if rank == 0 and not args.no_extras:
        # other forms of the same evaluation on this GPU (outside the timed region)
        del d
        out["precision_variants"] = precision_variants(csr, A, x0, p, w, eta, min(K, 100), args.warmup)
        out["batched_subset"] = batched_subset(min(K, 20), args.warmup, args)
        out["half_double"] = half_double_extra(csr, x0, min(K, 100), args.warmup)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        hx, hp, hw = x0.cpu().numpy(), p.cpu().numpy(), w.cpu().numpy()
        out["cpu_baseline"] = cpu_baseline(csr, hx, hp, hw)
        out["cpu_baseline_all_cores"] = cpu_baseline_all_cores(csr, hx, hp, hw)
    if ws > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


def _oracle_block(csr, enc, frac):
    """Contiguous block of rows from the middle of the matrix holding about
    frac of its entries, as a standalone CSR (rebased row pointers)."""
    rp = enc.row_ptr.astype(np.int64)
    nnz = int(rp[-1])
    want = max(1, int(frac * nnz))
    mid = int(np.searchsorted(rp, nnz // 2))
    r0 = int(np.searchsorted(rp, max(0, int(rp[mid]) - want // 2)))
    r1 = int(np.searchsorted(rp, min(nnz, int(rp[r0]) + want)))
    r1 = max(r1, r0 + 1)
    k0, k1 = int(rp[r0]), int(rp[r1])
    sub_rp = (rp[r0:r1 + 1] - k0).astype(np.uint32)
    return r0, r1, sub_rp, enc.col[k0:k1], enc.decoded[k0:k1]


def oracle_step(csr, enc, x, p, w, frac):
    """One oracle step (FP64 SpMV + f and A^T r) on a row block holding frac of
    the entries: returns (algorithmic bytes of that block, seconds)."""
    import oracle

    r0, r1, rp, col, a = _oracle_block(csr, enc, frac)
    nr, nc, nz = r1 - r0, csr.ncols, int(rp[-1])
    t0 = time.perf_counter()
    oracle.spmv(nr, rp, col, a, x)
    oracle.fgrad(nr, nc, rp, col, a, x, p[r0:r1], w[r0:r1])
    dt = time.perf_counter() - t0
    return oracle_step_bytes(nr, nc, nz), dt


def oracle_step_bytes(nr, nc, nz) -> int:
    """Bytes of one oracle step's arrays: the SpMV (values and indices, row
    pointers, x, d) and the f and A^T r pass (the same matrix again, p and w, x,
    g, f)."""
    return (6 * nz + 4 * (nr + 1) + 4 * nr + 4 * nc) + (6 * nz + 4 * (nr + 1) + 8 * nr + 8 * nc + 8)


def cpu_baseline(csr, x, p, w, budget_s=10.0):
    """The FP64 oracle, as it stands, on one host core: full-matrix steps
    (dose evaluation + dose+gradient evaluation) repeated for about budget_s."""
    import oracle

    enc = oracle.encode(csr, oracle.U16_SCALE)
    tot_b, tot_t, reps = 0, 0.0, 0
    while tot_t < budget_s and reps < 50:
        b, t = oracle_step(csr, enc, x, p, w, 1.0)
        tot_b, tot_t, reps = tot_b + b, tot_t + t, reps + 1
    return {"value": round(tot_b / tot_t / 1e9, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
            "ms_per_step": round(1e3 * tot_t / reps, 1),
            "sample": f"{reps} full-matrix step(s) of the clinical beam ({csr.nnz} entries): "
                      f"FP64 SpMV + f and A^T r, single thread"}


def oracle_row_blocks(row_ptr, col, a, p, w, n):
    """The rows cut into n contiguous blocks of about nnz / n entries each, as
    standalone CSR pieces (nr, rebased row_ptr, col, a, p, w)."""
    rp = np.asarray(row_ptr).astype(np.int64)
    nrows, nnz = rp.size - 1, int(rp[-1])
    cuts = [min(int(np.searchsorted(rp, nnz * t // n)), nrows) for t in range(n)] + [nrows]
    cuts[0] = 0
    out = []
    for t in range(n):
        r0, r1 = cuts[t], max(cuts[t], cuts[t + 1])
        k0, k1 = int(rp[r0]), int(rp[r1])
        out.append((r1 - r0, (rp[r0:r1 + 1] - k0).astype(np.uint32), col[k0:k1], a[k0:k1], p[r0:r1], w[r0:r1]))
    return out


def cpu_baseline_all_cores(csr, x, p, w, budget_s=10.0):
    """The same oracle calls on every host core: the rows cut into one
    contiguous block per core with equal entry counts (a static partition), one
    thread per block (the oracle's C calls release the interpreter lock); each
    block's f and A^T r are added in block order.  Full-matrix steps repeated
    for about budget_s."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle

    n = max(1, os.cpu_count() or 1)
    enc = oracle.encode(csr, oracle.U16_SCALE)
    blocks = oracle_row_blocks(enc.row_ptr, enc.col, enc.decoded, p, w, n)
    nc = csr.ncols

    def block_step(b):
        nr, brp, bcol, ba, bp, bw = b
        oracle.spmv(nr, brp, bcol, ba, x)
        return oracle.fgrad(nr, nc, brp, bcol, ba, x, bp, bw)

    step_bytes = oracle_step_bytes(csr.nrows, nc, csr.nnz)
    tot_t, reps = 0.0, 0
    with ThreadPoolExecutor(max_workers=n) as pool:
        list(pool.map(block_step, blocks))  # threads started, pages touched
        while tot_t < budget_s and reps < 200:
            t0 = time.perf_counter()
            parts = list(pool.map(block_step, blocks))
            f = sum(fb for fb, _ in parts)
            g = parts[0][1].copy()
            for _, gb in parts[1:]:
                g += gb
            tot_t += time.perf_counter() - t0
            reps += 1
    return {"value": round(reps * step_bytes / tot_t / 1e9, 3), "unit": "GB/s", "cores": n, "kind": "oracle",
            "ms_per_step": round(1e3 * tot_t / reps, 1), "cpu": f"{os.uname().machine}, {n} threads",
            "sample": f"{reps} full-matrix step(s) of the clinical beam ({csr.nnz} entries): FP64 SpMV + f "
                      f"and A^T r, rows in {n} equal-entry blocks, one thread each, partials added in block order"}


def csr_fused_bytes(info) -> int:
    """Byte model of one fused dose+gradient pass over the CSR arrays: stored
    values and 32-bit column indices once, row pointers, p and w, x in and g
    out, and the per-CTA gradient partials written and read once."""
    vb = {0: 2, 1: 2, 2: 1, 3: 2, 4: 4}[info["fmt"]]
    nz, nr, nc, P = info["nnz"], info["nrows"], info["ncols"], info["grid"]
    rs = 4 * nr if info["fmt"] == 2 else 0
    return (vb + 4) * nz + 4 * (nr + 1) + rs + 8 * nr + 8 * nc + 2 * P * nc * 4 + 8


def _time_calls(fn, steps, warmup):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def precision_variants(csr, A_u16, x, p, w, eta, steps, warmup):
    """The clinical beam in the other stored forms on the same GPU: FP8-E4M3
    with row scales, BF16, and u16 with 16-bit column indices for the dose
    SpMV; per form the dose eval and the dose+gradient eval times and the dose's
    relative error on 20000 sampled rows against the FP64 dose of the
    generator's values (fp64_dose_rows), next to the u16 baseline."""
    import torch

    import paper_2103_09683_gb300 as dose

    xh = x.cpu().numpy()
    rng = np.random.default_rng(7)
    lens = np.diff(csr.row_ptr.astype(np.int64))
    rows = np.unique(rng.choice(np.nonzero(lens > 0)[0], 20000, replace=False))
    exact = fp64_dose_rows(csr.row_ptr, csr.col, csr.val, xh, rows)
    nz = exact != 0
    f = torch.empty(1, dtype=torch.float64, device=x.device)
    g = torch.empty(csr.ncols, dtype=torch.float32, device=x.device)
    out = []
    for fmt, idx16 in (("u16", False), ("u16", True), ("bf16", False), ("fp8", False)):
        if fmt == "u16" and not idx16:
            A = A_u16
        else:
            codes, scales = dose.encode_host(fmt, csr.row_ptr, csr.val)
            A = dose.DoseMatrix.from_csr(csr.row_ptr, csr.col, ncols=csr.ncols, fmt=fmt, values=codes,
                                         scales=scales, index16=idx16)
            del codes, scales
        inf = A.info()
        d = torch.empty(A.nrows, dtype=torch.float32, device=x.device)
        ms_d = _time_calls(lambda: A.spmv(x, d), steps, warmup)
        dv = d.cpu().numpy()[rows].astype(np.float64)
        rel = np.abs(dv[nz] - exact[nz]) / np.abs(exact[nz])
        ms_g = _time_calls(lambda: A.fwd_adj_quadratic(x, p, w, f=f, g=g), steps, warmup)
        rg_fwd = inf["spmv_layout"] == 2
        csr_form = {}
        if rg_fwd:
            # the same dose evaluation on the CSR arrays, for comparison
            A.set_tuning(fwd_layout=1)
            ms_c = _time_calls(lambda: A.spmv(x, d), steps, warmup)
            A.set_tuning(fwd_layout=2)
            csr_form = {"ms_per_dose_eval_csr": round(ms_c, 5),
                        "dose_eval_gbs_csr": round(inf["spmv_bytes"] / (ms_c * 1e-3) / 1e9, 1)}
        A.device_status()
        out.append({"format": fmt, "spmv_index_bytes": 2 if idx16 else 4,
                    "spmv_layout": "row groups" if rg_fwd else "CSR",
                    "ms_per_dose_eval": round(ms_d, 5),
                    "dose_eval_gbs": round(inf["spmv_bytes"] / (ms_d * 1e-3) / 1e9, 1),
                    "dose_eval_own_bytes": inf["rg_spmv_bytes"] if rg_fwd else inf["spmv_bytes"],
                    **csr_form,
                    "ms_per_dose_grad_eval": round(ms_g, 5),
                    "dose_grad_eval_gbs_csr_model": round(csr_fused_bytes(inf) / (ms_g * 1e-3) / 1e9, 1),
                    "dose_grad_eval_own_bytes": inf["fused_bytes"],
                    "rel_err_vs_fp64_values": {"max": float(rel.max()), "mean": float(rel.mean())}})
        del d
        if A is not A_u16:
            A.close()
    return {"rows_sampled": int(len(rows)), "steps": steps, "variants": out}


def half_double_extra(csr, x, steps, warmup):
    """The paper's own configuration (Sec. IV, Half/double) on the clinical beam
    beside the plain form: IEEE half values, FP64 spot weights (the same weights
    as the plain form's) and FP64 dose through dose_spmv_f64, both
    accumulations; time, GB/s of the paper's byte model, and the dose's relative
    error on 20000 sampled rows against the FP64 dose of the generator's values."""
    import torch

    import paper_2103_09683_gb300 as dose

    xd = x.to(torch.float64)
    xh = xd.cpu().numpy()
    rng = np.random.default_rng(7)
    lens = np.diff(csr.row_ptr.astype(np.int64))
    rows = np.unique(rng.choice(np.nonzero(lens > 0)[0], 20000, replace=False))
    exact = fp64_dose_rows(csr.row_ptr, csr.col, csr.val, xh, rows)
    nz = exact != 0
    codes, _ = dose.encode_host("f16", csr.row_ptr, csr.val)
    A = dose.DoseMatrix.from_csr(csr.row_ptr, csr.col, ncols=csr.ncols, fmt="f16", values=codes)
    del codes
    nbytes = A.info()["spmv_f64_bytes"]
    d = torch.empty(A.nrows, dtype=torch.float64, device=x.device)
    peak, _ = _peaks()
    out = []
    for native in (False, True):
        ms = _time_calls(lambda: A.spmv_f64(xd, d, native=native), steps, warmup)
        dv = d.cpu().numpy()[rows]
        rel = np.abs(dv[nz] - exact[nz]) / np.abs(exact[nz])
        gbs = nbytes / (ms * 1e-3) / 1e9
        out.append({"accumulation": "fp64_fma" if native else "double_float", "ms_per_dose_eval": round(ms, 5),
                    "gbs_paper_model": round(gbs, 1), "frac": round(gbs / peak, 4),
                    "rel_err_vs_fp64_values": {"max": float(rel.max()), "mean": float(rel.mean())}})
    A.device_status()
    A.close()
    return {"format": "f16 values, f64 x and d (32-bit indices, CSR)", "bytes": nbytes, "rows_sampled": int(len(rows)),
            "variants": out}


def batched_subset(steps, warmup, args, pick=(4, 13, 22)):
    """Three of the 27 scenario matrices (one per beam shape, unshifted) x 16
    spot-weight vectors in one graph-captured dose_spmv_batched launch, against
    the same three as single-vector dose evaluations 16 times over."""
    import torch

    import paper_2103_09683_gb300 as dose

    nvec = 16
    mats, Xs, nbytes, nnz = [], [], 0, 0
    beams = dosegen.batched_beams()
    for i in pick:
        csr = dosegen.generate(beams[i])
        mats.append(dose.DoseMatrix.from_csr(csr.row_ptr, csr.col, ncols=csr.ncols, fmt="u16", values_f64=csr.val))
        Xs.append(torch.from_numpy(dosegen.spot_weights(csr.ncols, 300 + i, nvec=nvec).reshape(csr.ncols, nvec))
                  .cuda())
        nbytes += 6 * csr.nnz + 4 * (csr.nrows + 1) + 4 * nvec * (csr.nrows + csr.ncols)
        nnz += csr.nnz
        del csr
    sources = [_autotune(A, None, args, ("batched",))["source"] for A in mats]
    Ds = [torch.empty((A.nrows, nvec), dtype=torch.float32, device="cuda") for A in mats]
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        for _ in range(2):
            dose.spmv_batched(mats, Xs, Ds, stream=stream)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            dose.spmv_batched(mats, Xs, Ds, stream=stream)
        ms = _time_calls(graph.replay, steps, warmup)
    torch.cuda.synchronize()
    x1 = [X[:, 0].contiguous() for X in Xs]
    d1 = [torch.empty(A.nrows, dtype=torch.float32, device="cuda") for A in mats]
    ms_single = _time_calls(lambda: [A.spmv(x, d) for A, x, d in zip(mats, x1, d1)], steps, warmup)
    for A in mats:
        A.device_status()
    peak, _ = _peaks()
    return {"matrices": list(pick), "nvec": nvec, "nnz": nnz, "ms_per_step": round(ms, 4),
            "gbs": round(nbytes / (ms * 1e-3) / 1e9, 1), "frac": round(nbytes / (ms * 1e-3) / 1e9 / peak, 4),
            "bytes_per_step": nbytes, "ms_three_single_vector_evals": round(ms_single, 4),
            "ms_per_vector_batched": round(ms / nvec, 4),
            "layout": "row groups" if dose.spmv_batched_plan(mats, nvec)[0] == 2 else "CSR",
            "autotune_sources": sources}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle

    beam = dosegen.CLINICAL
    csr = dosegen.generate(beam)
    enc = oracle.encode(csr, oracle.U16_SCALE)
    p, w = dosegen.ellipsoid_target(beam, semi_axes=(30.0, 20.0, 16.0))
    x = dosegen.spot_weights(csr.ncols, dosegen.weight_seed(beam))
    # size each step's row block so that warmup + steps take about two minutes
    _, t_full = oracle_step(csr, enc, x, p, w, 1.0)
    frac = min(1.0, 120.0 / max(args.steps + args.warmup, 1) / max(t_full, 1e-6))
    for _ in range(args.warmup):
        oracle_step(csr, enc, x, p, w, frac)
    tot_b, tot_t = 0, 0.0
    for _ in range(args.steps):
        b, t = oracle_step(csr, enc, x, p, w, frac)
        tot_b, tot_t = tot_b + b, tot_t + t
    v = round(tot_b / tot_t / 1e9, 3)
    sample = (f"each step: a contiguous row block with {frac:.3%} of the clinical matrix's entries "
              f"(FP64 SpMV + f and A^T r), single thread")
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GB/s", "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * tot_t / args.steps, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": WORKLOAD, "nrows": csr.nrows, "ncols": csr.ncols,
                                           "nnz": csr.nnz, "format": "u16+scale",
                                           "bytes_per_step": oracle_step_bytes(csr.nrows, csr.ncols, csr.nnz),
                                           "step": REF_STEP, "sample_fraction": round(frac, 6),
                                           "l2": "host memory (the oracle on the CPU)",
                                           "parallelism": "single CPU thread"},
           "cpu_baseline": {"value": v, "unit": "GB/s", "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


BATCH_METRIC = "batched dose SpMM effective HBM GB/s (27 matrices x 16 vectors, one graph-captured launch)"
BATCH_WORKLOAD = ("batched uncertainty scenarios: 3 pencil beams (160x160x80 / 1000 spots, 200x200x120 / 2500, "
                  "256x256x120 / 4000) x 9 lateral setup shifts {-3,0,+3}^2 voxels = 27 CSR matrices "
                  "(1.84e9 entries, u16 + scale, u32 indices), each times 16 FP32 spot-weight vectors")


def run_batched(args):
    """D_m = A_m X_m for the 27 scenario matrices, 16 vectors each, in one
    graph-captured dose_spmv_batched launch per step."""
    import torch

    import paper_2103_09683_gb300 as dose

    ws, rank, local = _dist()
    dose.build()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as td
        td.init_process_group("nccl", device_id=device)
    nvec = 16
    mats, Xs, nbytes, nnz, nrows = [], [], 0, 0, 0
    sample = None
    pick = set(range(27)) if not args.matrices else {int(m) for m in args.matrices.split(",")}
    for i, beam in enumerate(dosegen.batched_beams()):
        if i not in pick:
            continue
        csr = dosegen.generate(beam)
        mats.append(dose.DoseMatrix.from_csr(csr.row_ptr, csr.col, ncols=csr.ncols, fmt="u16", values_f64=csr.val))
        Xs.append(torch.from_numpy(dosegen.spot_weights(csr.ncols, 300 + i, nvec=nvec).reshape(csr.ncols, nvec))
                  .to(device))
        nbytes += 6 * csr.nnz + 4 * (csr.nrows + 1) + 4 * nvec * (csr.nrows + csr.ncols)
        nnz += csr.nnz
        nrows += csr.nrows
        if i == max(pick) and rank == 0 and ws == 1 and not args.no_cpu_baseline:
            sample = (csr, Xs[-1].cpu().numpy())
        del csr
    sources = [_autotune(A, None, args, ("batched",))["source"] for A in mats]
    Ds = [torch.empty((A.nrows, nvec), dtype=torch.float32, device=device) for A in mats]
    layout, launches = dose.spmv_batched_plan(mats, nvec)
    kname = "rg_spmm_kernel" if layout == 2 else "spmm_staged_kernel"
    stream = torch.cuda.Stream(device)
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        for _ in range(2):
            dose.spmv_batched(mats, Xs, Ds, stream=stream)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            dose.spmv_batched(mats, Xs, Ds, stream=stream)
        for _ in range(args.warmup):
            graph.replay()
    torch.cuda.synchronize()
    K = args.steps
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(K):
            graph.replay()
        e1.record(stream)
    torch.cuda.synchronize()
    time.sleep(0.2)
    clk = clocks.stop()
    total_ms = max_over_ranks(e0.elapsed_time(e1), device)
    for A in mats:
        A.device_status()
    ms = total_ms / K
    gbs = whole_job_gbs(nbytes, K, 1, total_ms)
    peak, peak_kind = _peaks()
    # end to end: X from pinned host memory in, the graph, all of D out to
    # pinned host memory, every step on one stream.  The read-back (8.47 GB at
    # the host link's rate) is ten times the compute, so overlapping the two
    # saves little; copies issued right behind the kernel that wrote D ran at
    # the link rate, copies beside the next step's kernel at half of it.
    Xh = [_pinned_like(X) for X in Xs]
    Dh = [torch.empty(D.shape, dtype=torch.float32, pin_memory=True) for D in Ds]

    def e2e_steps(n):
        for _ in range(n):
            for X, H in zip(Xs, Xh):
                X.copy_(H, non_blocking=True)
            graph.replay()
            for D, H in zip(Ds, Dh):
                H.copy_(D, non_blocking=True)

    ke = max(3, min(K, 5))
    with torch.cuda.stream(stream):
        # untimed: the first copies into freshly pinned buffers map them for the GPU
        e2e_steps(2)
        torch.cuda.synchronize()
        ee0, ee1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ee0.record(stream)
        e2e_steps(ke)
        ee1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = ee0.elapsed_time(ee1) / ke
    h2d = sum(X.numel() * 4 for X in Xs)
    d2h = sum(D.numel() * 4 for D in Ds)
    out = {
        "metric": BATCH_METRIC, "value": round(ws * gbs, 1), "unit": "GB/s", "n_gpus": ws, "steps": K,
        "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": BATCH_WORKLOAD if len(mats) == 27 else
                   f"{len(mats)} of the scenario matrices ({sorted(pick)}) x 16 FP32 spot-weight vectors",
                   "matrices": len(mats), "nvec": nvec, "nnz": nnz, "nrows": nrows,
                   "bytes_per_step": nbytes, "l2": "inputs larger than L2 (A streams ~11 GB per step)",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "kernel": kname,
                     "achieved": round(gbs, 1), "peak": peak,
                     "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"
                     if peak_kind == "measured" else "fallback 6.8 TB/s",
                     "unit": "GB/s", "frac": round(gbs / peak, 4), "traffic": _traffic(kname)},
        "layout": "row groups" if layout == 2 else "CSR",
        "e2e": {"value": round(nbytes / (e2e_ms * 1e-3) / 1e9, 1), "unit": "GB/s", "ms_per_step": round(e2e_ms, 3),
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "note": "pinned host buffers; X in, the graph, D out, one stream"},
        "gpu_launches": K * launches,
        "clocks": clk,
        "autotuned": all(src != "off" for src in sources),
        "autotune": {"sources": {k: sources.count(k) for k in sorted(set(sources))}, "purposes": ["batched"],
                     "cache": os.path.relpath(args.autotune_cache, ROOT)},
    }
    if sample is not None:
        out["cpu_baseline"] = batched_cpu_baseline(*sample)
    if ws > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


PREC_METRIC = ("dose SpMV effective HBM GB/s per stored format (plain, compensated, 16-bit indices), with each "
               "result's relative error against the FP64 dose of the generator's values")


def fp64_dose_rows(row_ptr, col, val, x, rows):
    """d_i = sum_k val_k x[col_k] in FP64 (numpy) for the listed rows: the
    exact-values dose that a stored format's result is compared with."""
    rp = np.asarray(row_ptr).astype(np.int64)
    rows = np.asarray(rows, dtype=np.int64)
    lens = rp[rows + 1] - rp[rows]
    starts = np.zeros(len(rows) + 1, dtype=np.int64)
    np.cumsum(lens, out=starts[1:])
    idx = np.repeat(rp[rows] - starts[:-1], lens) + np.arange(int(starts[-1]))
    prod = np.asarray(val, dtype=np.float64)[idx] * np.asarray(x, dtype=np.float64)[np.asarray(col)[idx]]
    out = np.zeros(len(rows))
    ne = lens > 0
    out[ne] = np.add.reduceat(prod, starts[:-1][ne]) if prod.size else 0.0
    return out


def run_precision(args):
    """The clinical beam stored as u16 + scale (the baseline), BF16, FP8-E4M3
    with per-row scales, F16 and F32, each plain, with compensated (Dot2) rows,
    and with 16-bit column indices: time per dose evaluation, effective GB/s
    of the format's own bytes, and each result's relative error on sampled rows
    against the FP64 dose of the generator's own values (the format's rounding
    plus the FP32 accumulation).  The library encodes the generator's FP64
    values (dose_encode_host, once per format); parity with the FP64 oracle on
    the same decoded values is the full-size GPU tests' job."""
    import torch

    import paper_2103_09683_gb300 as dose

    dose.build()
    torch.cuda.set_device(0)
    beam = dosegen.CLINICAL
    csr = dosegen.generate(beam)
    x = dosegen.spot_weights(csr.ncols, dosegen.weight_seed(beam))
    xd = torch.from_numpy(x).cuda()
    rng = np.random.default_rng(7)
    lens = np.diff(csr.row_ptr.astype(np.int64))
    rows = np.unique(rng.choice(np.nonzero(lens > 0)[0], 20000, replace=False))
    exact = fp64_dose_rows(csr.row_ptr, csr.col, csr.val, x, rows)
    nz = exact != 0
    peak, _ = _peaks()
    K = max(3, min(args.steps, 200))
    variants = []
    for fmt in ("u16", "bf16", "fp8", "f16", "f32"):
        codes, scales = dose.encode_host(fmt, csr.row_ptr, csr.val)
        for comp, idx16 in ((False, False), (True, False), (False, True)):
            A = dose.DoseMatrix.from_csr(csr.row_ptr, csr.col, ncols=csr.ncols, fmt=fmt, values=codes,
                                         scales=scales, compensated=comp, index16=idx16)
            d = torch.empty(A.nrows, dtype=torch.float32, device="cuda")
            for _ in range(args.warmup):
                A.spmv(xd, d)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(K):
                A.spmv(xd, d)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / K
            A.device_status()
            inf = A.info()
            nbytes = inf["spmv_bytes"]
            rg = inf["spmv_layout"] == 2
            own = inf["rg_spmv_bytes"] if rg else nbytes
            dv = d.cpu().numpy()[rows].astype(np.float64)
            rel = np.abs(dv[nz] - exact[nz]) / np.abs(exact[nz])
            variants.append({"format": fmt, "compensated": comp, "index_bytes": 2 if idx16 else 4,
                             "spmv_layout": "row groups" if rg else "CSR", "ms": round(ms, 5),
                             "achieved_gbs": round(nbytes / (ms * 1e-3) / 1e9, 1),
                             "frac": round(nbytes / (ms * 1e-3) / 1e9 / peak, 4), "bytes": nbytes,
                             "bytes_per_entry": round(nbytes / csr.nnz, 3),
                             "own_bytes": own, "own_frac": round(own / (ms * 1e-3) / 1e9 / peak, 4),
                             "rel_err_vs_fp64_values": {"max": float(rel.max()), "mean": float(rel.mean())}})
            del A, d
        del codes, scales
    base = variants[0]
    out = {"metric": PREC_METRIC, "value": base["achieved_gbs"], "unit": "GB/s", "n_gpus": 1, "steps": K,
           "warmup": args.warmup, "ms_per_step": base["ms"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": WORKLOAD.split("; step")[0] + "; dose eval d = A x per stored format",
                      "error_rows": int(len(rows))},
           "gpu_launches": len(variants) * K, "variants": variants}
    print(json.dumps(out), flush=True)


HD_METRIC = ("Half/double dose SpMV (F16 values, FP64 x and d): effective HBM GB/s of the 6 nnz + 12 nr + 8 nc "
             "traffic model and GFLOP/s")


def run_halfdouble(args):
    """The paper's own configuration (Sec. IV, "Half/double") at the clinical
    size: IEEE half values, FP64 spot weights and dose, with 32-bit indices (the
    paper's byte model) and 16-bit indices; double-float accumulation (default)
    and FP64-FMA accumulation (the paper's arithmetic).  A step is one
    dose_spmv_f64 call (the x split and the SpMV kernel)."""
    import torch

    import paper_2103_09683_gb300 as dose

    dose.build()
    torch.cuda.set_device(0)
    beam = dosegen.CLINICAL
    csr = dosegen.generate(beam)
    x = dosegen.spot_weights_f64(csr.ncols, dosegen.weight_seed(beam))
    xd = torch.from_numpy(x).cuda()
    codes, _ = dose.encode_host("f16", csr.row_ptr, csr.val)
    peak, _ = _peaks()
    K = max(3, min(args.steps, 200))
    clocks = ClockSampler(0)
    variants = []
    clocks.start()
    for idx16 in (False, True):
        A = dose.DoseMatrix.from_csr(csr.row_ptr, csr.col, ncols=csr.ncols, fmt="f16", values=codes,
                                     index16=idx16)
        if args.tuning:
            A.set_tuning(**_tuning_kv(args))
        nbytes = A.info()["spmv_f64_bytes"]
        for native in (False, True):
            d = torch.empty(A.nrows, dtype=torch.float64, device="cuda")
            for _ in range(args.warmup):
                A.spmv_f64(xd, d, native=native)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(K):
                A.spmv_f64(xd, d, native=native)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / K
            A.device_status()
            gbs = nbytes / (ms * 1e-3) / 1e9
            variants.append({"accumulation": "fp64_fma" if native else "double_float", "index_bytes": 2 if idx16 else 4,
                             "ms": round(ms, 5), "achieved_gbs": round(gbs, 1), "frac": round(gbs / peak, 4),
                             "gflops": round(2 * csr.nnz / (ms * 1e-3) / 1e9, 1), "bytes": nbytes})
            del d
        del A
    clk = clocks.stop()
    base = variants[0]
    out = {"metric": HD_METRIC, "value": base["achieved_gbs"], "unit": "GB/s", "n_gpus": 1, "steps": K,
           "warmup": args.warmup, "ms_per_step": base["ms"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f16 values, f64 vectors", "data": "synthetic",
           "config": {"workload": "clinical pencil beam 256x256x160 voxels x 4000 spots, ~1.5e8 entries; "
                                  "F16 values; step = one dose_spmv_f64 (x split + SpMV)",
                      "tuning": _tuning_kv(args),
                      "l2": "A (~0.9 GB) > L2: streamed from HBM every step",
                      "peak_gbs": peak},
           "clocks": clk, "variants": variants}
    print(json.dumps(out), flush=True)


ROBUST_METRIC = ("robust dose+gradient evaluation over 9 setup-shift scenarios of a 3-beam plan: ms per "
                 "evaluation and effective HBM GB/s of its algorithmic bytes")


def run_robust(args):
    """A three-beam plan on a 160x160x100 grid (beams entering along +z, +x, +y,
    1000 spots each) under the nine lateral setup shifts: nine merged scenario
    handles (u16 + scale), one projected-gradient step of the expected and of
    the worst-case robust quadratic objective per timed step (nine fused passes
    and one combine kernel each), captured in a CUDA graph."""
    import torch

    import paper_2103_09683_gb300 as dose

    dose.build()
    torch.cuda.set_device(0)
    plan = dosegen.robust_plan()
    mats, abs_row, abs_col, nnz = [], None, None, 0
    for s, beams in enumerate(plan):
        csrs = [dosegen.generate_along(b, ax) for b, ax in beams]
        mats.append(dose.DoseMatrix.from_multibeam([(c.row_ptr, c.col, c.ncols, c.val) for c in csrs], fmt="u16",
                                                   tuning=_tuning_kv(args) or None))
        # ||A_s||_1 ||A_s||_inf bounds ||A_s||_2^2, hence the Lipschitz constant of every scenario's gradient
        rs = sum(np.add.reduceat(np.concatenate([c.val, [0.0]]), c.row_ptr.astype(np.int64)[:-1])
                 * (np.diff(c.row_ptr.astype(np.int64)) > 0) for c in csrs)
        cs = np.concatenate([np.bincount(c.col, weights=c.val, minlength=c.ncols) for c in csrs])
        abs_row = rs.max() if abs_row is None else max(abs_row, rs.max())
        abs_col = cs.max() if abs_col is None else max(abs_col, cs.max())
        nnz += sum(c.nnz for c in csrs)
        del csrs
    nrows, ncols = mats[0].nrows, mats[0].ncols
    grid_beam = plan[0][0][0]
    p, w = dosegen.ellipsoid_target(grid_beam, semi_axes=(20.0, 16.0, 12.0), depth_frac=0.5)
    eta = 1.0 / (2.0 * float(w.max()) * float(abs_row) * float(abs_col))
    x0 = np.concatenate([dosegen.spot_weights(1000, dosegen.weight_seed(b) & 0xFFFF) for b, _ in plan[4]])
    dev = torch.device("cuda", 0)
    pt, wt, x0t = (torch.from_numpy(a).to(dev) for a in (p, w, x0))
    S = dose.ScenarioSet(mats)
    step_bytes = sum(A.info()["fused_bytes"] for A in mats) + 9 * (ncols * 4) + ncols * 12 + 9 * 8
    peak, _ = _peaks()
    K = max(3, min(args.steps, 100))
    stream = torch.cuda.Stream()
    clocks = ClockSampler(0)
    variants = []
    clocks.start()
    for mode in ("expected", "worst"):
        x = x0t.clone()
        f = torch.empty(1, dtype=torch.float64, device=dev)
        g = torch.empty(ncols, dtype=torch.float32, device=dev)
        stream.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                S.pg_step(x, pt, wt, eta, mode=mode, f=f, g=g, stream=stream)
        stream.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            S.pg_step(x, pt, wt, eta, mode=mode, f=f, g=g, stream=stream)
        x.copy_(x0t)
        torch.cuda.synchronize()
        f_first = None
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            graph.replay()
            stream.synchronize()
            f_first = float(f.item())
            e0.record(stream)
            for _ in range(K):
                graph.replay()
            e1.record(stream)
        stream.synchronize()
        ms = e0.elapsed_time(e1) / K
        f_last = float(f.item())
        for A in mats:
            A.device_status()
        gbs = step_bytes / (ms * 1e-3) / 1e9
        variants.append({"mode": mode, "ms": round(ms, 4), "ms_per_scenario": round(ms / 9, 4),
                         "achieved_gbs": round(gbs, 1), "frac": round(gbs / peak, 4),
                         "f_first": f_first, "f_after": f_last, "launches_per_step": 2 * 9 + 1})
    clk = clocks.stop()
    S.close()
    base = variants[0]
    out = {"metric": ROBUST_METRIC, "value": base["achieved_gbs"], "unit": "GB/s", "n_gpus": 1, "steps": K,
           "warmup": args.warmup, "ms_per_step": base["ms"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": f"3-beam plan on 160x160x100 voxels (beams along +z, +x, +y, 1000 spots each) "
                                  f"x 9 setup shifts; {nnz} entries in all, u16 + scale; step = one robust PG step "
                                  f"(9 fused passes + combine) in a CUDA graph",
                      "nrows": nrows, "ncols": ncols, "step_bytes": step_bytes, "tuning": _tuning_kv(args),
                      "adj_window": max(A.info()["adj_window"] for A in mats),
                      "adj_block_fused": mats[0].info()["adj_block_fused"],
                      "l2": "9 scenario matrices (~5 GB) > L2: streamed from HBM every step", "peak_gbs": peak},
           "clocks": clk, "gpu_launches": 19 * K, "variants": variants}
    print(json.dumps(out), flush=True)


SELL_METRIC = ("dose SpMV on SELL-32-sigma storage (the paper's future-work format) against the CSR kernel: "
               "effective HBM GB/s of each layout's own bytes, ms per dose eval, padding")


def run_sell(args):
    """The clinical beam (u16 + scale) stored as SELL-32-sigma for several sigma,
    with 32- and 16-bit indices, next to the CSR kernel on the same matrix; a
    step is one dose_spmv.  The SELL dose at this size is checked against the
    FP64 oracle by the full-size GPU tests."""
    import torch

    import paper_2103_09683_gb300 as dose

    dose.build()
    torch.cuda.set_device(0)
    beam = dosegen.CLINICAL
    csr = dosegen.generate(beam)
    codes, scales = dose.encode_host("u16", csr.row_ptr, csr.val)
    x = dosegen.spot_weights(csr.ncols, dosegen.weight_seed(beam))
    xd = torch.from_numpy(x).cuda()
    peak, _ = _peaks()
    K = max(3, min(args.steps, 200))
    clocks = ClockSampler(0)
    variants = []
    clocks.start()
    # sigma 0: the CSR kernel; -1: the row-group kernel (dose_spmv's default form,
    # whose union indices are 16-bit here whatever the CSR index width)
    for idx16 in (False, True):
        for sigma in ((-1,) if not idx16 else ()) + (0, 1, 32, 256, 1024, 8192, 1 << 20):
            tuning = dict(sell_sigma=sigma) if sigma > 0 else (dict(fwd_layout=1) if sigma == 0 else None)
            A = dose.DoseMatrix.from_csr(csr.row_ptr, csr.col, ncols=csr.ncols, fmt="u16", values=codes,
                                         scales=scales, index16=idx16, sell=sigma > 0, tuning=tuning)
            inf = A.info()
            d = torch.empty(A.nrows, dtype=torch.float32, device="cuda")
            for _ in range(args.warmup):
                A.spmv(xd, d)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(K):
                A.spmv(xd, d)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / K
            A.device_status()
            gbs = inf["spmv_bytes"] / (ms * 1e-3) / 1e9
            name = f"sell-32-{sigma}" if sigma > 0 else ("csr" if sigma == 0 else "row-groups")
            v = {"layout": name, "index_bytes": 2 if (idx16 or sigma < 0) else 4,
                 "ms": round(ms, 5), "bytes": inf["spmv_bytes"], "achieved_gbs": round(gbs, 1),
                 "frac": round(gbs / peak, 4),
                 "stored_entries": inf["sell_entries"] if sigma > 0 else csr.nnz,
                 "padding": round(inf["sell_entries"] / csr.nnz - 1, 4) if sigma > 0 else 0.0}
            if sigma < 0:
                own = inf["rg_spmv_bytes"]
                v.update({"note": "bytes = the CSR byte model; the layout's own bytes are own_bytes",
                          "own_bytes": own, "own_frac": round(own / (ms * 1e-3) / 1e9 / peak, 4)})
            variants.append(v)
            del A, d
    clk = clocks.stop()
    base = next(v for v in variants if v["layout"] == "sell-32-1048576" and v["index_bytes"] == 4)
    out = {"metric": SELL_METRIC, "value": base["achieved_gbs"], "unit": "GB/s", "n_gpus": 1, "steps": K,
           "warmup": args.warmup, "ms_per_step": base["ms"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "clinical pencil beam 256x256x160 voxels x 4000 spots, ~1.5e8 entries; u16 + scale; "
                                  "step = one dose_spmv", "peak_gbs": peak},
           "clocks": clk, "variants": variants}
    print(json.dumps(out), flush=True)


LIVER_METRIC = ("dose SpMV on a matrix shaped like the paper's liver beam 1 (Table I): effective HBM GB/s "
                "of each call's algorithmic bytes and GFLOP/s, Half/double and FP32 forms")


def run_liver1(args):
    """The paper's own headline matrix shape: 2.97e6 voxels x 6.8e4 spots,
    1.48e9 entries, ~75 % empty rows, most non-empty rows longer than 1024
    entries (whole-CTA reduction), x too large for shared memory (gathered from
    L2).  Variants: the paper's Half/double (F16 values, FP64 x and d; the
    paper's 6 nnz + 12 nr + 8 nc bytes) with double-float and FP64-FMA
    accumulation, and the FP32-vector dose_spmv on u16 + scale.  The dose at
    this size is checked against the FP64 oracle on sampled rows by the
    full-size GPU tests."""
    import torch

    import paper_2103_09683_gb300 as dose

    dose.build()
    torch.cuda.set_device(0)
    beam = dosegen.LIVER1_SHAPED
    csr = dosegen.generate(beam)
    tun = _tuning_kv(args) or None
    A16 = dose.DoseMatrix.from_csr(csr.row_ptr, csr.col, ncols=csr.ncols, fmt="f16", values_f64=csr.val, tuning=tun)
    Au = dose.DoseMatrix.from_csr(csr.row_ptr, csr.col, ncols=csr.ncols, fmt="u16", values_f64=csr.val, tuning=tun)
    nrows, ncols, nnz = csr.nrows, csr.ncols, csr.nnz
    del csr
    x64 = dosegen.spot_weights_f64(ncols, dosegen.weight_seed(beam))
    x32 = dosegen.spot_weights(ncols, dosegen.weight_seed(beam))
    xd64, xd32 = torch.from_numpy(x64).cuda(), torch.from_numpy(x32).cuda()
    peak, _ = _peaks()
    K = max(3, min(args.steps, 50))

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(K):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / K

    clocks = ClockSampler(0)
    clocks.start()
    variants = []
    d64 = torch.empty(nrows, dtype=torch.float64, device="cuda")
    b64 = A16.info()["spmv_f64_bytes"]
    for native in (False, True):
        ms = timed(lambda: A16.spmv_f64(xd64, d64, native=native))
        gbs = b64 / (ms * 1e-3) / 1e9
        variants.append({"form": "half_double", "accumulation": "fp64_fma" if native else "double_float",
                         "ms": round(ms, 4), "bytes": b64, "achieved_gbs": round(gbs, 1), "frac": round(gbs / peak, 4),
                         "gflops": round(2 * nnz / (ms * 1e-3) / 1e9, 1)})
    del d64
    d32 = torch.empty(nrows, dtype=torch.float32, device="cuda")
    bu = Au.info()["spmv_bytes"]
    ms = timed(lambda: Au.spmv(xd32, d32))
    gbs = bu / (ms * 1e-3) / 1e9
    variants.append({"form": "u16+scale, FP32 vectors", "accumulation": "fp32", "ms": round(ms, 4), "bytes": bu,
                     "achieved_gbs": round(gbs, 1), "frac": round(gbs / peak, 4),
                     "gflops": round(2 * nnz / (ms * 1e-3) / 1e9, 1)})
    clk = clocks.stop()
    A16.device_status()
    Au.device_status()
    base = variants[0]
    out = {"metric": LIVER_METRIC, "value": base["achieved_gbs"], "unit": "GB/s", "n_gpus": 1, "steps": K,
           "warmup": args.warmup, "ms_per_step": base["ms"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f16 values, f64 vectors", "data": "synthetic",
           "config": {"workload": f"liver-beam-1-shaped pencil beam: {nrows} voxels x {ncols} spots, {nnz} entries "
                                  f"(Table I: 2.97e6 x 6.80e4, 1.48e9); step = one dose evaluation",
                      "peak_gbs": peak, "tuning": _tuning_kv(args),
                      "info": {k: Au.info()[k] for k in ("n_stages", "n_coop_rows", "lanes_hist", "adj_window")},
                      "paper_a100_half_double": "1250-1350 GB/s, up to 420 GFLOP/s on the liver beams (context)"},
           "clocks": clk, "variants": variants}
    print(json.dumps(out), flush=True)


def batched_cpu_baseline(csr, X, budget_s=10.0):
    """The oracle's FP64 SpMM on row blocks of one scenario matrix (about
    budget_s of single-core work), as GB/s of the same byte model."""
    import oracle

    enc = oracle.encode(csr, oracle.U16_SCALE)
    Xd = X.astype(np.float64)
    frac, spent, nb, blocks = 0.05, 0.0, 0, 0
    while spent < budget_s and blocks < 100:
        r0, r1, rp, col, a = _oracle_block(csr, enc, frac)
        t0 = time.perf_counter()
        oracle.spmm(r1 - r0, rp, col, a, Xd)
        spent += time.perf_counter() - t0
        nz = int(rp[-1])
        nb += 6 * nz + 4 * (r1 - r0 + 1) + 4 * X.shape[1] * ((r1 - r0) + X.shape[0])
        blocks += 1
    return {"value": round(nb / spent / 1e9, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": f"{blocks} row block(s) of ~5% of one scenario matrix ({csr.nnz} entries) x {X.shape[1]} "
                      f"vectors: FP64 SpMM, single thread, {spent:.1f} s"}


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the precision variants and the batched subset of the default line")
    ap.add_argument("--autotune", default="cached", choices=["off", "cached", "full"],
                    help="schedule knobs: off = defaults; cached = from the autotune cache, sweeping on a miss "
                         "(default); full = sweep and store")
    ap.add_argument("--autotune-cache", default=AUTOTUNE_CACHE,
                    help="the autotune cache file (default: the committed GB300 cache)")
    ap.add_argument("--tuning", default="", help="schedule knobs, e.g. tile_nnz=8192,adj_scatter_warps=4")
    ap.add_argument("--matrices", default="", help="batched: subset of the 27 scenario matrices, e.g. 4,13,22")
    ap.add_argument("--workload", default="clinical",
                    choices=["clinical", "batched", "precision", "halfdouble", "robust", "sell", "liver1"],
                    help="clinical: the dose + dose-gradient step (default); batched: 27 matrices x 16 vectors; "
                         "precision: dose eval per stored format with its error vs the FP64 oracle; "
                         "halfdouble: F16 values with FP64 x and d; robust: 3-beam plan x 9 scenarios")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "precision":
        run_precision(args)
    elif args.workload == "halfdouble":
        run_halfdouble(args)
    elif args.workload == "robust":
        run_robust(args)
    elif args.workload == "sell":
        run_sell(args)
    elif args.workload == "liver1":
        run_liver1(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
