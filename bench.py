#!/usr/bin/env python
"""Benchmark of the CI hot path on GB300 (prints one JSON line).

Workload: the 4p+4n problem in HO shells N <= 4 (70 states per species,
two-word bit strings) with Nmax = 4 and 2M = 0: dimension 172,684,
1.026e8 stored nonzeros, seeded FP32 TBMEs (synthetic, ``synth`` preset
c1).  One step is one pass of the whole hot path over it: stage the
interaction from the device-resident flat tables, enumerate the basis,
species filter, count, scan, fill H (FP32), and block Lanczos (b = 8,
FP64 reorthogonalisation) for the lowest 5 eigenvalues, whose SpMMs apply
H.  ``value`` = H nonzeros built per second of whole step time.

Also measured in the same run: the standalone SpMM (H X, 8 vectors, full
and half storage) as a fraction of the HBM roofline, per-kernel live
durations (CUDA events on the launch stream, one launch in 8 of each kernel
timed, every launch counted), the end-to-end time through the public API
with host buffers, and the FP64 oracle on the host cores (``cpu_baseline``);
then, each skippable with its flag: the count benchmark of Sec. 2.1
(``--no-count``), observables and transition elements (``--no-observables``),
the eigensolvers with FP64 Ritz refinement (``--no-eigensolvers``), the motif
benchmarks of Sec. 2.2-2.4 (``--no-motifs``), the Nmax = 6 precision study
(``--no-c2``), the 256-problem batch (``--no-batch``) and the served stream
(``--no-serve``).

``--impl reference`` times the oracle (the plain FP64 CPU program) on a
bounded sample of the same workload instead.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "H nonzeros built/s + SpMM % HBM peak; served solves/s, p50/p99 latency"
WORKLOAD = ("4p+4n HO shells N<=4 (70 m-states/species), Nmax=4, 2M=0: dim 172684, nnz 102601752; "
            "FP32 H, block Lanczos k=5 b=8, FP64-exact reorth on tensor cores")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=16.0, help="oracle sample budget (build part)")
    ap.add_argument("--cpu-sample", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--cpu-row0", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--spmm-reps", type=int, default=20)
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--batch-n", type=int, default=256)
    ap.add_argument("--fp64-sample", type=int, default=12, help="problems solved one by one in FP64")
    ap.add_argument("--no-count", action="store_true", help="skip the count-benchmark leg")
    ap.add_argument("--count-n", type=int, default=131072, help="states of the count benchmark")
    ap.add_argument("--no-observables", action="store_true", help="skip the observables leg")
    ap.add_argument("--no-c2", action="store_true", help="skip the Nmax=6 precision-study leg")
    ap.add_argument("--no-eigensolvers", action="store_true", help="skip the Lanczos / LOBPCG comparison leg")
    ap.add_argument("--no-motifs", action="store_true", help="skip the scan / fill / array-reduction motif leg")
    ap.add_argument("--no-products", action="store_true", help="skip the reorthogonalisation-product leg")
    ap.add_argument("--products-only", action="store_true",
                    help="run only the reorthogonalisation-product leg and print its JSON (a small profiling case)")
    ap.add_argument("--obs-m", type=int, default=16, help="operators of the observables leg")
    return ap.parse_args()


# ---------------------------------------------------------------- helpers

def dist_info():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def max_over_ranks(x, world, device=None):
    """The largest value of x over all ranks (all_reduce MAX); x for one rank.
    Ranks are independent replicas: this is the only exchange of a run."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, max_ms):
    """Units processed by all ranks per second of the slowest rank's time."""
    return units_per_rank * world / (max_ms * 1e-3)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured", d
    return 6800.0, "fallback", {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.flush()
        rows = []
        with open(self.out.name) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), power=float(parts[3]),
                                     hw=parts[5], hwt=parts[6], swt=parts[7], pcap=parts[8]))
                except ValueError:
                    continue
        os.unlink(self.out.name)
        if not rows:
            return None
        loaded = [r for r in rows if r["power"] > 200.0] or rows
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("pcap", "sw_power_cap")):
                if r[key].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in loaded), "sm_max_mhz": max(r["smax"] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows), "samples_under_load": len(loaded),
                "power_w_max": max(r["power"] for r in rows)}


# ---------------------------------------------------------------- workload

def workload_inputs():
    import numpy as np

    import synth
    p = synth.preset("c1")
    sp = synth.ho_sp_table(p.n_shell_max)
    eps = synth.sp_energies(sp, p.hbar_omega)
    T = synth.tbme_tables(sp, p.seed, np.float32)
    return p, sp, eps, T


TRACE_SAMPLE = 8

# DRAM bytes (read + write) per launch of a kernel, from one ncu capture
# summarised in profiles/dram_traffic_c1.txt; each line names the source
# file of the kernel and the SHA-256 prefix of that file when it was
# captured.  A kernel whose source has changed since reports null traffic.
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic_c1.txt")


def _source_digest(rel):
    import hashlib
    path = os.path.join(ROOT, rel)
    if not os.path.exists(path):
        return None
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def ncu_traffic():
    """kernel -> DRAM bytes per launch, for the kernels whose source still
    matches the capture."""
    out = {}
    if not os.path.exists(TRAFFIC_FILE):
        return out
    with open(TRAFFIC_FILE) as f:
        for line in f:
            parts = line.split()
            if len(parts) < 4 or line.startswith("#"):
                continue
            name, nbytes, src, digest = parts[:4]
            if _source_digest(src) == digest:
                out[name] = float(nbytes)
    return out


def algorithmic_bytes(kernel, dim, nnz, nvec=8, y_bytes=4):
    """Algorithmic DRAM bytes of one launch of the kernels with a byte roofline
    (y_bytes: 4 for the standalone FP32 product, 8 inside the solve, where the
    SpMM writes the Lanczos block W in FP64)."""
    if kernel == "k_fill_rows":      # col i32 + val f32 written, row_ptr read
        return 8 * nnz + 8 * (dim + 1)
    if kernel == "build_H":          # col + val written, row counts written and read, row_ptr written
        return 8 * nnz + 12 * dim + 8
    if kernel == "k_spmm":           # CSR streamed once, X (FP32) read once, Y written
        return 8 * nnz + 8 * (dim + 1) + 4 * nvec * dim + y_bytes * nvec * dim
    if kernel == "k_spmm16":         # the same with 16-vector X and Y rows
        return 8 * nnz + 8 * (dim + 1) + 2 * 4 * 16 * dim
    return None   # k_count_rows walks per-row segment tables: latency-bound, no byte roofline


def run_ours(args):
    import numpy as np
    import torch

    import paper_2110_10765_gb300 as ci

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    p, sp, eps, T = workload_inputs()
    dtab = {k: torch.from_numpy(v).to(dev) for k, v in T.items()}   # inputs resident in HBM
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)
    stream = torch.cuda.current_stream()

    def step(tables):
        prob = ci.Problem(sp, p.Z, p.N, p.nmax, p.twoM, eps, tables=tables)
        prob.enumerate_basis()
        M = prob.build_H("f32")
        ev, info = M.lowest_eigs(k=p.k, block=p.block)
        return prob, M, ev, info

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step(dtab)
    barrier()

    clocks = ClockSampler(local)
    clocks.start()
    # every launch counted; CUDA events on one launch in TRACE_SAMPLE of each
    # kernel (the per-launch means come from those, on their launch streams)
    ci.trace_enable(True, sample=TRACE_SAMPLE)
    ci.trace_read(reset=True)
    ev_s = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_h = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_b = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_e = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier()
    t_wall = time.perf_counter()
    nnz = dim = None
    evals = None
    infos = []
    for i in range(args.steps):
        flush.fill_(float(i))                       # L2 flush between steps (not timed)
        ev_s[i].record(stream)
        prob = ci.Problem(sp, p.Z, p.N, p.nmax, p.twoM, eps, tables=dtab)
        dim = prob.enumerate_basis()
        ev_h[i].record(stream)
        M = prob.build_H("f32")
        ev_b[i].record(stream)
        evals, info = M.lowest_eigs(k=p.k, block=p.block)
        ev_e[i].record(stream)
        nnz = M.nnz
        infos.append(info)
        del M, prob
    barrier()
    t_wall = time.perf_counter() - t_wall
    kern = ci.trace_read(reset=True)
    ci.trace_enable(False)
    clk = clocks.stop()
    hbm, peak_kind, peaks = load_peaks()
    step_ms = [ev_s[i].elapsed_time(ev_e[i]) for i in range(args.steps)]
    build_ms = [ev_s[i].elapsed_time(ev_b[i]) for i in range(args.steps)]
    buildH_ms = [ev_h[i].elapsed_time(ev_b[i]) for i in range(args.steps)]
    solve_ms = [ev_b[i].elapsed_time(ev_e[i]) for i in range(args.steps)]
    total_ms = sum(step_ms)
    total_ms = max_over_ranks(total_ms, world, dev)

    # ---- standalone SpMM (Y = H X, 8 vectors): fraction of the HBM roofline
    prob = ci.Problem(sp, p.Z, p.N, p.nmax, p.twoM, eps, tables=dtab)
    M = prob.build_H("f32")
    X = torch.randn(M.dim, 8, device=dev, dtype=torch.float32)
    Y = torch.empty_like(X)
    for _ in range(3):
        M.apply_H(X, Y)
    sp_ms = []
    for i in range(args.spmm_reps):
        flush.fill_(float(i))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        M.apply_H(X, Y)
        b.record(stream)
        b.synchronize()
        sp_ms.append(a.elapsed_time(b))
    spmm_ms = statistics.median(sp_ms)
    spmm_bytes = algorithmic_bytes("k_spmm", M.dim, M.nnz)
    spmm_gbs = spmm_bytes / (spmm_ms * 1e-3) / 1e9
    # the same product from the half-stored H (upper triangle, atomic updates)
    U = M.upper()
    for _ in range(3):
        U.apply_H(X, Y)
    up_ms = []
    for i in range(args.spmm_reps):
        flush.fill_(float(i))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        U.apply_H(X, Y)
        b.record(stream)
        b.synchronize()
        up_ms.append(a.elapsed_time(b))
    upper_ms = statistics.median(up_ms)
    upper_nnz = U.nnz
    del U

    # ---- kernels: shares and the dominant kernel's roofline
    tot_k = sum(v[1] for v in kern.values()) or 1.0
    kernels = {k: {"launches": int(v[0]), "total_ms": round(v[1], 4), "ms_per_launch": round(v[1] / max(v[0], 1), 5),
                   "share": round(v[1] / tot_k, 4)} for k, v in sorted(kern.items(), key=lambda kv: -kv[1][1])}
    gpu_launches = int(sum(v[0] for v in kern.values()))
    roofs = []
    traffic_of = ncu_traffic() if nnz == 102601752 else {}
    for name, v in kern.items():
        b = algorithmic_bytes(name, dim, nnz, y_bytes=8)
        if b is None:
            continue
        avg_s = v[1] / max(v[0], 1) * 1e-3
        # inside the solve the SpMM runs on the 8-vector blocks (Y in FP64),
        # once per solve on the final residual block
        traffic = traffic_of.get(name)
        roofs.append({"kernel": name, "bound": "hbm", "achieved": round(b / avg_s / 1e9, 1), "peak": hbm,
                      "unit": "GB/s", "frac": round(b / avg_s / 1e9 / hbm, 4), "traffic": traffic,
                      "bytes_per_launch": b, "ms_per_launch": round(avg_s * 1e3, 5)})
    dominant = max(kern.items(), key=lambda kv: kv[1][1])[0] if kern else None
    # the whole ci_build_H call (species filter, count, scan, fill): CUDA
    # events on the launch stream around it in every timed step
    bh_ms = statistics.median(buildH_ms)
    bh_bytes = algorithmic_bytes("build_H", dim, nnz)
    roofs.append({"kernel": "build_H", "bound": "hbm", "achieved": round(bh_bytes / (bh_ms * 1e-3) / 1e9, 1),
                  "peak": hbm, "unit": "GB/s", "frac": round(bh_bytes / (bh_ms * 1e-3) / 1e9 / hbm, 4),
                  "traffic": None, "bytes_per_launch": bh_bytes, "ms_per_launch": round(bh_ms, 5),
                  "scope": "ci_build_H: species filter (tables staged), count, scan, fill"})

    rec = {
        "metric": METRIC, "value": None, "unit": "nnz/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 (H, SpMM); f64 (Lanczos)", "data": "synthetic",
        "config": {"workload": WORKLOAD, "dim": dim, "nnz": nnz, "k": p.k, "block": p.block,
                   "l2": "inputs (288 MB flat TBME tables) and outputs (0.82 GB CSR) exceed L2; "
                         "512 MB L2 flush between steps, outside the step events",
                   "kernel_timing": "every launch counted; CUDA events on every %dth launch of each kernel "
                                    "inside the timed steps" % TRACE_SAMPLE,
                   "parallelism": "replicas" if world > 1 else "single GPU"},
    }
    per_rank_nnz = nnz * args.steps
    rec["value"] = whole_job_rate(per_rank_nnz, world, total_ms)
    rec["ms_per_step"] = total_ms / args.steps
    rec["phases_ms"] = {"build_median": statistics.median(build_ms), "build_H_median": bh_ms,
                        "solve_median": statistics.median(solve_ms),
                        "step_median": statistics.median(step_ms), "wall_total_s": t_wall}
    rec["build_nnz_per_s"] = nnz / (bh_ms * 1e-3)
    rec["solve"] = {"iterations": infos[-1]["iterations"], "restarts": infos[-1]["restarts"],
                    "lowest": [round(float(x), 9) for x in evals], "residual_max": max(infos[-1]["residual"]),
                    "hnorm_est": infos[-1]["hnorm_est"]}
    rec["spmm"] = {"ms": spmm_ms, "achieved_gbs": round(spmm_gbs, 1), "peak_gbs": hbm, "frac": round(spmm_gbs / hbm, 4),
                   "bytes": spmm_bytes, "peak_kind": peak_kind, "nvec": 8,
                   "half_storage": {"ms": round(upper_ms, 4), "stored_nnz": upper_nnz,
                                    "csr_bytes": 8 * upper_nnz + 8 * M.dim,
                                    "vs_full": round(upper_ms / spmm_ms, 3)}}
    rec["kernels"] = kernels
    rec["rooflines"] = roofs
    dom_roof = next((r for r in roofs if r["kernel"] == dominant), None)
    rec["roofline"] = dom_roof or {"kernel": dominant, "bound": "alu", "achieved": None, "peak": None,
                                   "unit": None, "frac": None, "traffic": None}
    rec["gpu_launches"] = gpu_launches
    rec["clocks"] = clk
    rec["peaks"] = {"hbm_gbs": hbm, "kind": peak_kind}
    del M, prob, X, Y

    # ---- end to end through the public API with host buffers
    if not args.no_e2e:
        host = {k: torch.from_numpy(v).pin_memory() for k, v in T.items()}
        step(host)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            prob, M, ev, info = step(host)   # H2D of the tables inside; evals come back to the host
            del M, prob
        barrier()
        e2e_s = time.perf_counter() - t0
        h2d = sum(v.numel() * v.element_size() for v in host.values()) + 3 * 4 * len(sp["N"]) + 8 * len(sp["N"])
        rec["e2e"] = {"value": nnz * args.steps * world / e2e_s, "unit": "nnz/s", "h2d_bytes_per_step": int(h2d),
                      "d2h_bytes_per_step": int(8 * p.k + 8), "ms_per_step": e2e_s / args.steps * 1e3}
    # the auxiliary legs: an error in one is recorded in its key and does not
    # void the measurement above
    def aux(key, fn, *a, **kw):
        try:
            rec[key] = fn(*a, **kw)
        except Exception as e:   # noqa: BLE001
            rec[key] = {"error": "%s: %s" % (type(e).__name__, e)}
            print("bench: %s leg failed: %s" % (key, e), file=sys.stderr)
    if not args.no_count:
        aux("count", run_count_leg, args.count_n, clock_mhz=(clk or {}).get("sm_mhz"))
    if not args.no_observables:
        aux("observables", run_observables_leg, sp, p, eps, dtab, args.obs_m)
    if not args.no_eigensolvers:
        aux("eigensolvers", run_eigensolver_leg, sp, p, eps, dtab)
    if not args.no_motifs:
        aux("motifs", run_motifs_leg, hbm, (clk or {}).get("sm_mhz"))
    if not args.no_products:
        aux("products", run_products_leg, hbm)
    if not args.no_c2:
        aux("c2_precision", run_c2_leg, hbm)
    if not args.no_batch:
        rec["batch"], pool = run_batch_leg(args)
        if not args.no_serve:
            rec["serve"] = run_serve_leg(pool)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rec["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    # the headline figures once more at the end of the line (kept by tails)
    bh = next(r for r in roofs if r["kernel"] == "build_H")
    rec["summary"] = {"step_ms": rec["ms_per_step"], "build_H_ms": round(bh_ms, 4),
                      "build_nnz_per_s": rec["build_nnz_per_s"], "build_H_frac_hbm": bh["frac"],
                      "solve_ms": statistics.median(solve_ms), "spmm_ms": round(spmm_ms, 4),
                      "spmm_frac_hbm": rec["spmm"]["frac"],
                      "dominant": {k: rec["roofline"].get(k) for k in ("kernel", "frac")},
                      "cpu_build_nnz_per_s": (rec.get("cpu_baseline") or {}).get("build_nnz_per_s")}
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(rec))


# ---------------------------------------------------------------- precision study

def run_c2_leg(hbm):
    """The same generator at Nmax = 6 (dim 2,680,018, 3.2e9 nonzeros): build
    and SpMM in FP32, lowest 10 eigenvalues with the FP32 H and with the FP64
    H (the FP64 GPU run is the reference at this size)."""
    import numpy as np
    import torch

    import synth
    import paper_2110_10765_gb300 as ci
    p = synth.preset("c2")
    sp = synth.ho_sp_table(p.n_shell_max)
    eps = synth.sp_energies(sp, p.hbar_omega)
    T = {k: torch.from_numpy(v).cuda() for k, v in synth.tbme_tables(sp, p.seed, np.float32).items()}
    stream = torch.cuda.current_stream()

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        out = fn()
        b.record(stream)
        b.synchronize()
        return out, a.elapsed_time(b)

    prob = ci.Problem(sp, p.Z, p.N, p.nmax, p.twoM, eps, tables=T)
    prob.enumerate_basis()
    M, build_ms = timed(lambda: prob.build_H("f32"))
    X = torch.randn(M.dim, 8, device="cuda")
    Y = torch.empty_like(X)
    M.apply_H(X, Y)
    sp_ms = min(timed(lambda: M.apply_H(X, Y))[1] for _ in range(3))
    b = algorithmic_bytes("k_spmm", M.dim, M.nnz)
    del X, Y
    E32 = torch.zeros((M.dim, p.k), dtype=torch.float64, device="cuda")
    (ev32, info32), s32 = timed(lambda: M.lowest_eigs(k=p.k, evecs=E32))
    dim, nnz = M.dim, M.nnz
    del M
    # the FP32 Ritz pairs refined with the FP64 H applied on the fly
    (evr, rnr), sr = timed(lambda: prob.refine_eigs(E32, iters=1))
    del E32
    # BF16 values with a per-row FP32 scale (6 bytes per nonzero)
    Mb = prob.build_H("bf16")
    X = torch.randn(dim, 8, device="cuda")
    Y = torch.empty_like(X)
    Mb.apply_H(X, Y)
    spb_ms = min(timed(lambda: Mb.apply_H(X, Y))[1] for _ in range(3))
    del X, Y
    (evb, infob), sb = timed(lambda: Mb.lowest_eigs(k=p.k, allow_unconverged=True))
    del Mb
    M64 = prob.build_H("f64")
    (ev64, info64), s64 = timed(lambda: M64.lowest_eigs(k=p.k))
    del M64
    return {"workload": "4p+4n N<=4 Nmax=6 (dim %d, nnz %d), k=%d" % (dim, nnz, p.k), "dim": dim, "nnz": nnz,
            "build_f32_ms": build_ms, "build_nnz_per_s": nnz / (build_ms * 1e-3),
            "spmm_f32_ms": sp_ms, "spmm_gbs": b / (sp_ms * 1e-3) / 1e9, "spmm_frac": b / (sp_ms * 1e-3) / 1e9 / hbm,
            "solve_f32_s": s32 * 1e-3, "solve_f32_iterations": info32["iterations"],
            "solve_f64_s": s64 * 1e-3, "solve_f64_iterations": info64["iterations"],
            "lowest_f64": [round(float(x), 7) for x in ev64],
            "max_abs_diff_f32_vs_f64": float(np.max(np.abs(ev32 - ev64))),
            "max_rel_diff_f32_vs_f64": float(np.max(np.abs(ev32 - ev64) / np.abs(ev64))),
            "refined_f32": {"s": sr * 1e-3, "iters": 1, "max_abs_diff_vs_f64": float(np.max(np.abs(evr - ev64))),
                            "max_rel_diff_vs_f64": float(np.max(np.abs(evr - ev64) / np.abs(ev64))),
                            "max_residual_f64": float(np.max(rnr))},
            "bf16_rowscale": {"spmm_ms": spb_ms, "solve_s": sb * 1e-3, "iterations": infob["iterations"],
                              "max_abs_diff_vs_f64": float(np.max(np.abs(evb - ev64))),
                              "max_rel_diff_vs_f64": float(np.max(np.abs(evb - ev64) / np.abs(ev64)))}}


# ---------------------------------------------------------------- motifs

# FP32 FMAs per clock per SM (CUDA arithmetic-throughput table): the ALU
# roofline of the array-reduction motif
FMA32_PER_CLK_SM = 128


def run_products_leg(hbm, dim=172684, widths=(8, 16, 32, 64), reps=10):
    """The block Lanczos reorthogonalisation products through ci_basis_product
    at the c1 dimension: Q^T W and W - Q C for a basis of `na` columns (row
    stride 64, as in the solver) and an 8-vector block, on the tensor cores
    (FP64-exact digit planes) and on the FP64 CUDA cores.  Kernel time from
    CUDA events on the launch stream; algorithmic bytes: the na columns of the
    basis (the tensor-core form reads its 8-byte fixed-point shadow) plus W
    (read, and for W - Q C written)."""
    import numpy as np
    import torch
    import paper_2110_10765_gb300 as ci
    rng = np.random.default_rng(5)
    A = torch.from_numpy(rng.uniform(-1, 1, (dim, 64)) / np.sqrt(dim)).cuda()
    B = torch.from_numpy(rng.standard_normal((dim, 8))).cuda()
    Cm = torch.from_numpy(rng.standard_normal((64, 8)) * 1e-3).cuda()
    out = {"dim": dim, "forms": {}}
    names = {"tc": ("k_oz_tn", "k_oz_nn"), "fp64": ("k_tn_partial", "k_nn_update")}
    for method in ("tc", "fp64"):
        rows = []
        for na in widths:
            C = torch.zeros((na, 8), dtype=torch.float64, device="cuda")
            for _ in range(2):
                ci.basis_product("tn", A[:, :na], B, C, method=method)
            ci.trace_enable(True)
            ci.trace_read(True)
            for _ in range(reps):
                ci.basis_product("tn", A[:, :na], B, C, method=method)
                ci.basis_product("nn", A[:, :na], B, Cm[:na], alpha=-1.0, beta=1.0, method=method)
            t = ci.trace_read(True)
            ci.trace_enable(False)
            kt, kn = names[method]
            tn_us = t[kt][1] / t[kt][0] * 1e3
            nn_us = t[kn][1] / t[kn][0] * 1e3
            btn, bnn = dim * (8 * na + 64), dim * (8 * na + 128)
            rows.append({"na": na, "tn_us": round(tn_us, 2), "nn_us": round(nn_us, 2),
                         "tn_frac_hbm": round(btn / (tn_us * 1e-6) / 1e9 / hbm, 4),
                         "nn_frac_hbm": round(bnn / (nn_us * 1e-6) / 1e9 / hbm, 4)})
        out["forms"][method] = rows
    del A, B, Cm
    return out


def run_motifs_leg(hbm, clock_mhz=None, reps=5):
    """The paper's motif benchmarks (Sec. 2.2-2.4): serial vs parallel scan of
    2^24 counts (Fig. 5), the shared-array fill of Listing 7 with m = 512,
    p = 1 over 2^20 rows (Fig. 6), and the small-array reduction with m = 64
    over n = 2^14 columns, n^2 pairs (Fig. 7)."""
    import torch

    import paper_2110_10765_gb300 as ci
    stream = torch.cuda.current_stream()

    def best(fn, r=reps):
        fn()
        ms = []
        for _ in range(r):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        return min(ms)

    g = torch.Generator(device="cuda").manual_seed(5)
    out = {}
    n = 1 << 24
    c = torch.randint(0, 10, (n,), dtype=torch.int32, device="cuda", generator=g)
    off = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    par = best(lambda: ci.exclusive_scan(c, off))
    ser = best(lambda: ci.scan_serial(c, off), r=1)
    out["scan"] = {"n": n, "parallel_ms": par, "serial_ms": ser, "speedup": ser / par,
                   "parallel_gbs": (4 * n + 8 * (n + 1)) / (par * 1e-3) / 1e9,
                   "parallel_frac_hbm": (4 * n + 8 * (n + 1)) / (par * 1e-3) / 1e9 / hbm}
    del c, off
    rows, m, p = 1 << 20, 512, 1
    offset = torch.arange(rows, dtype=torch.int64, device="cuda") * (m // p)
    arr = torch.empty(rows * (m // p), dtype=torch.int32, device="cuda")
    fm = best(lambda: ci.fill_shared(offset, m, p, arr))
    fb = 4 * rows * (m // p) + 8 * rows
    out["fill"] = {"rows": rows, "m": m, "p": p, "ms": fm, "gbs": fb / (fm * 1e-3) / 1e9,
                   "frac_hbm": fb / (fm * 1e-3) / 1e9 / hbm}
    del offset, arr
    nr, mr = 1 << 14, 64
    x = torch.randn((nr, mr), device="cuda", generator=g)
    y = torch.randn((nr, mr), device="cuda", generator=g)
    rm = best(lambda: ci.array_reduction(x, y))
    rate = nr * nr * mr / (rm * 1e-3)
    peak = FMA32_PER_CLK_SM * SMS * (clock_mhz or 2070.0) * 1e6
    out["array_reduction"] = {"n": nr, "m": mr, "ms": rm, "updates_per_s": rate, "bound": "alu",
                              "peak_updates_per_s": peak, "frac": rate / peak,
                              "peak_basis": "%d FP32 FMA/clk/SM x %d SMs x clock" % (FMA32_PER_CLK_SM, SMS)}
    return out


# ---------------------------------------------------------------- eigensolvers

def run_eigensolver_leg(sp, p, eps, tables):
    """Fig. 1, eigensolve on the benchmark workload (FP32 H): block Lanczos
    against LOBPCG with the diagonal and with the many-body-orbital
    block-diagonal preconditioner (Sec. 2), each timed with CUDA events
    around the whole solve (the orbital grouping, the block inversions and
    their applications included)."""
    import torch

    import synth
    import paper_2110_10765_gb300 as ci
    prob = ci.Problem(sp, p.Z, p.N, p.nmax, p.twoM, eps, tables=tables)
    M = prob.build_H("f32")
    stream = torch.cuda.current_stream()
    labels = synth.sp_orbitals(sp)
    out = {}
    for name in ("lanczos", "lobpcg_diagonal", "lobpcg_orbital_blocks"):
        def solve():
            if name == "lanczos":
                return M.lowest_eigs(k=p.k, block=p.block)
            blocks = prob.orbital_blocks(labels) if name == "lobpcg_orbital_blocks" else None
            return M.lowest_eigs(k=p.k, block=p.block, method="lobpcg", blocks=blocks)
        solve()                                            # warm-up
        ci.trace_enable(True)
        ci.trace_read(reset=True)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ev, info = solve()
        b.record(stream)
        b.synchronize()
        kern = ci.trace_read(reset=True)
        ci.trace_enable(False)
        rec = {"ms": round(a.elapsed_time(b), 3), "iterations": info["iterations"],
               "max_residual": max(info["residual"]), "evals": [round(float(x), 6) for x in ev]}
        for kname in ("k_block_inv", "k_block_apply"):
            if kname in kern:
                n_l, ms = kern[kname]
                rec[kname] = {"launches": int(n_l), "ms_per_launch": round(ms / max(n_l, 1), 4)}
        out[name] = rec
    # FP32 Lanczos pairs refined with the FP64 H on the fly, against the FP64 solve
    import numpy as np
    E = torch.zeros((M.dim, p.k), dtype=torch.float64, device="cuda")
    ev32, _ = M.lowest_eigs(k=p.k, block=p.block, evecs=E)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    evr, rnr = prob.refine_eigs(E, iters=1)
    b.record(stream)
    b.synchronize()
    M64 = prob.build_H("f64")
    a2, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a2.record(stream)
    ev64, info64 = M64.lowest_eigs(k=p.k, block=p.block)
    b2.record(stream)
    b2.synchronize()
    del M64
    out["refine_fp64"] = {"ms": round(a.elapsed_time(b), 3), "iters": 1,
                          "fp32_max_abs_diff_vs_fp64_solve": float(np.max(np.abs(ev32 - ev64))),
                          "refined_max_abs_diff_vs_fp64_solve": float(np.max(np.abs(evr - ev64))),
                          "max_residual_f64": float(np.max(rnr)),
                          "fp64_solve_ms": round(a2.elapsed_time(b2), 3), "fp64_iterations": info64["iterations"]}
    blk, nb = prob.orbital_blocks(labels)
    sizes = torch.bincount(blk.long(), minlength=nb).cpu()
    out["orbital_groups"] = {"groups": nb, "largest": int(sizes.max()), "mean": round(float(sizes.float().mean()), 2)}
    return out


# ---------------------------------------------------------------- observables

def run_observables_leg(sp, p, eps, tables, m, reps=2):
    """Fig. 1, observables step on the benchmark workload: expectation values of m
    seeded two-body operators in the k = 5 lowest eigenvectors, elements
    evaluated on the fly (never stored)."""
    import torch

    import paper_2110_10765_gb300 as ci
    prob = ci.Problem(sp, p.Z, p.N, p.nmax, p.twoM, eps, tables=tables)
    M = prob.build_H("f32")
    E = torch.zeros((M.dim, p.k), dtype=torch.float64, device="cuda")
    M.lowest_eigs(k=p.k, block=p.block, evecs=E)
    seeds = [7000 + i for i in range(m)]
    prob.observables(seeds[:1], E)           # builds the FP64 connectivity once
    stream = torch.cuda.current_stream()
    ms = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        vals = prob.observables(seeds, E)
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    t = min(ms)
    # transition elements x_v^T O_k y_v for 16 seeded vector pairs (two
    # passes of eight vectors per operator)
    g = torch.Generator(device="cuda").manual_seed(11)
    X = torch.randn((M.dim, 16), dtype=torch.float64, device="cuda", generator=g)
    Y = torch.randn((M.dim, 16), dtype=torch.float64, device="cuda", generator=g)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    prob.observables(seeds, X, Y)
    b.record(stream)
    b.synchronize()
    t16 = a.elapsed_time(b)
    return {"operators": m, "vectors": p.k, "ms": t, "ms_per_operator": t / m,
            "elements_per_s": M.nnz * m / (t * 1e-3), "nnz": M.nnz,
            "first_values": [round(float(x), 9) for x in vals[0]],
            "transition_16_vectors": {"ms": t16, "ms_per_operator": t16 / m}}


# ---------------------------------------------------------------- count benchmark

# 32-bit population counts per clock per SM (CUDA arithmetic-throughput
# table) and the GB300's SM count: the ALU roofline of the count kernels,
# whose pairs cost one 32-bit popcount (the XOR folded to 32 bits rejects
# all but the rare near pairs).
POPC_PER_CLK_SM = 16
SMS = 152


def run_count_leg(n, N=8, S=128, reps=5, clock_mhz=None):
    """The paper's nonzero-count benchmark (Sec. 2.1, Figs. 3-4): n random
    8-particle states over 128 s.p. states biased to low states; rate =
    n^2 / time for the three forms of the pair test."""
    import numpy as np
    import torch

    import synth
    import paper_2110_10765_gb300 as ci
    mbs = synth.e1_states(n, N=N, S=S, seed=1)
    d = torch.from_numpy(mbs.view(np.int16)).cuda()
    stream = torch.cuda.current_stream()
    out = {"n": n, "N": N, "S": S, "bias_ratio": synth.E1_RATIO, "variants": {}}
    for v in ("hybrid", "bits", "mbs"):
        r = reps if v != "mbs" else 2
        total = ci.count_pairs(d, S, v)
        ms = []
        for _ in range(r):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            total = ci.count_pairs(d, S, v)
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        t = statistics.median(ms)
        out["variants"][v] = {"ms": t, "pairs_per_s": n * n / (t * 1e-3), "total": total}
    tot = out["variants"]["hybrid"]["total"]
    out["density_offdiag"] = (tot - n) / (n * n - n)
    out["forms_agree"] = len({x["total"] for x in out["variants"].values()}) == 1
    f = (clock_mhz or 2070.0) * 1e6
    peak = POPC_PER_CLK_SM * SMS * f               # one 32-bit popcount per pair
    ach = out["variants"]["hybrid"]["pairs_per_s"]
    out["roofline"] = {"kernel": "k_count_hybrid", "bound": "alu", "achieved": ach, "peak": peak,
                       "unit": "pairs/s", "frac": ach / peak,
                       "peak_basis": "%d popc/clk/SM x %d SMs x %.0f MHz, 1 popc per pair" % (
                           POPC_PER_CLK_SM, SMS, f / 1e6)}
    return out


# ---------------------------------------------------------------- batched solves

def batch_problems(n, seed=3):
    """The batched mix: Z, N in 2..6, Nmax in 0..4, shells N <= 3, per-problem
    TBME seeds; draws whose dimension is outside [1e2, 1e5] are rejected."""
    import synth
    import paper_2110_10765_gb300 as ci
    sp = synth.ho_sp_table(3)
    eps = synth.sp_energies(sp, 20.0)
    out = []
    for c in synth.batch_candidates(seed, 20 * n):
        p = ci.Problem(sp, c["Z"], c["N"], c["nmax"], (c["Z"] + c["N"]) % 2, eps, seed=c["seed"])
        d = p.enumerate_basis()
        if 100 <= d <= 100000:
            out.append((c, p, d))
        if len(out) == n:
            break
    return sp, eps, out


def run_batch_leg(args):
    """256 problems built and solved in one batch (FP32 H, FP64 Lanczos, k=5)
    against the plain single-solve FP64 form on a sample of the same problems."""
    import numpy as np
    import torch

    import paper_2110_10765_gb300 as ci
    sp, eps, items = batch_problems(args.batch_n)
    probs = [p for _, p, _ in items]
    dims = [d for _, _, d in items]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b = ci.Batch(probs, k=5)
    b.run()
    t_batch = time.perf_counter() - t0
    st = b.stats()
    evs = []
    nconv = 0
    for i in range(len(probs)):
        ev, info = b.result(i, allow_unconverged=True)
        evs.append(ev)
        nconv += info["status"] == 0
    # plain FP64 form: one problem per call, FP64 H and Lanczos, no graph
    rng = np.random.default_rng(0)
    sample = sorted(rng.choice(len(items), size=min(args.fp64_sample, len(items)), replace=False).tolist())
    t_single = 0.0
    max_rel = 0.0
    for i in sample:
        c, _, _ = items[i]
        p = ci.Problem(sp, c["Z"], c["N"], c["nmax"], (c["Z"] + c["N"]) % 2, eps, seed=c["seed"])
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        p.enumerate_basis()
        M = p.build_H("f64")
        ev64, _ = M.lowest_eigs(k=5)
        t_single += time.perf_counter() - t1
        max_rel = max(max_rel, float(np.max(np.abs(evs[i] - ev64) / np.maximum(np.abs(ev64), 1))))
    # the sample's share of the batch rows, to compare like with like
    frac = sum(dims[i] for i in sample) / sum(dims)
    single_rate = len(sample) / t_single
    return {"problems": len(probs), "converged": int(nconv), "rows": int(sum(dims)), "nnz": st["nnz"],
            "dim_min": int(min(dims)), "dim_median": float(np.median(dims)), "dim_max": int(max(dims)),
            "build_s": st["build_s"], "solve_s": st["solve_s"], "steps": st["steps"], "wall_s": t_batch,
            "autotuned_launch": b.tuning(),
            "solves_per_s": len(probs) / t_batch,
            "fp64_single": {"sample": len(sample), "rows_fraction": frac, "seconds": t_single,
                            "solves_per_s": single_rate,
                            "max_rel_diff_vs_batch": max_rel},
            "k": 5, "precision": "batch: FP32 H + FP64 Lanczos; single: FP64 H + FP64 Lanczos"}, \
        [c for c, _, _ in items]


def _serve(reqs, paced):
    """Submit reqs to a fresh queue (at their arrival times when paced, all
    at once otherwise) and wait for every result."""
    import synth
    import paper_2110_10765_gb300 as ci
    sps = {n: synth.ho_sp_table(n) for n in (3, 4)}
    epss = {n: synth.sp_energies(sps[n], 20.0) for n in (3, 4)}
    q = ci.Queue(mem_budget=96 << 30, max_slots=256)
    t0 = time.perf_counter()
    tickets = []
    for r in reqs:
        dt = t0 + r["t_arrival"] - time.perf_counter()
        if paced and dt > 0:
            time.sleep(dt)
        n = r["n_shell_max"]
        tickets.append(q.submit(sps[n], r["Z"], r["N"], r["nmax"], (r["Z"] + r["N"]) % 2, epss[n], r["k"],
                                seed=r["seed"]))
    results = {}
    while len(results) < len(tickets):
        for t in tickets:
            if t not in results:
                st, res = q.poll(t)
                if st != 6:
                    results[t] = (st, res)
        time.sleep(0.001)
    stats = q.stats()
    q.close()
    ok = [res for st, res in results.values() if st == 0]
    span = max(res["t_done"] for _, res in results.values()) - min(res["t_submit"] for _, res in results.values())
    return ok, span, stats


def run_serve_leg(pool, n_requests=400, n_capacity=300, seed=4):
    """Continuous-batching solve queue.  Its capacity is measured first
    (n_capacity requests submitted at once, completions per second); then
    Poisson arrivals at 80 % of that rate, drawn from the batched mix plus
    5 % requests of the benchmark size (4p+4n, N<=4, Nmax=4), each with its
    own TBME seed and 1..10 wanted eigenvalues."""
    import numpy as np

    import synth
    cap_reqs = synth.serve_requests(1.0, n_capacity, seed=seed + 100, small_pool=pool)
    ok_c, span_c, _ = _serve(cap_reqs, paced=False)
    capacity = len(ok_c) / span_c
    rate = 0.8 * capacity
    reqs = synth.serve_requests(rate, n_requests, seed=seed, small_pool=pool)
    ok, span, stats = _serve(reqs, paced=True)
    lat = np.array([res["latency_s"] for res in ok]) * 1e3
    big = [res["latency_s"] * 1e3 for res in ok if res["dim"] > 100000]
    return {"requests": len(reqs), "completed_ok": len(ok), "failed": len(reqs) - len(ok),
            "capacity_per_s": capacity, "capacity_requests": n_capacity,
            "offered_rate_per_s": rate, "solves_per_s": len(ok) / span, "span_s": span,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "mean": float(lat.mean()), "max": float(lat.max())},
            "big_requests": len(big), "big_latency_ms_p50": float(np.median(big)) if big else None,
            "engine_steps": stats["steps"],
            "mix": "batched mix (Z,N in 2..6, Nmax 0..4, shells N<=3) + 5% 4p4n N<=4 Nmax=4; k in 1..10"}


# ---------------------------------------------------------------- the oracle

def _golden_c1():
    with open(os.path.join(ROOT, "tests", "golden", "golden.json")) as f:
        return json.load(f)["c1"]


def oracle_step_sample(o, i0, build_seconds, matvecs, ncv, chunk=256):
    """One bounded step of the oracle on rows i0, i0+1, ... of the workload:
    build rows (Fig. 1 count, scan and fill, the oracle's OpenMP row loops)
    chunk by chunk until build_seconds have passed, then the per-row work of
    the oracle's eigensolve on those rows: `matvecs` products of the row slab
    with a full-length vector (scipy's CSR product, the operator ARPACK
    applies) each followed by two classical Gram-Schmidt passes against
    `ncv` basis columns restricted to the slab (ARPACK's
    reorthogonalisation).  Returns (rows, nnz, build_s, solve_s)."""
    import numpy as np
    import scipy.sparse as sps
    t0 = time.perf_counter()
    parts = []
    i = i0
    while time.perf_counter() - t0 < build_seconds:
        a = i % o.dim
        b = min(a + chunk, o.dim)
        parts.append(o.csr_rows(a, b))
        i = a + (b - a)
    t_build = time.perf_counter() - t0
    rows = sum(len(rp) - 1 for rp, _, _ in parts)
    nnz = sum(int(rp[-1]) for rp, _, _ in parts)
    rp = np.concatenate([[0]] + [p[0][1:] + off for p, off in
                                 zip(parts, np.cumsum([0] + [int(q[0][-1]) for q in parts[:-1]]))])
    H = sps.csr_matrix((np.concatenate([p[2] for p in parts]), np.concatenate([p[1] for p in parts]), rp),
                       shape=(rows, o.dim))
    rng = np.random.default_rng(0)
    x = rng.standard_normal(o.dim)
    V = np.linalg.qr(rng.standard_normal((rows, ncv)))[0]
    t1 = time.perf_counter()
    for k in range(matvecs):
        y = H @ x
        for _ in range(2):
            y -= V @ (V.T @ y)
        V[:, k % ncv] = y / (np.linalg.norm(y) + 1e-300)
    t_solve = time.perf_counter() - t1
    return rows, nnz, t_build, t_solve


def _oracle_for_workload():
    import oracle
    p, sp, eps, T = workload_inputs()
    return oracle.OracleProblem(sp, p.Z, p.N, p.nmax, p.twoM, eps, T)


def cpu_sample_main(threads, seconds, i0):
    """Child process of the CPU baseline: one oracle step sample on
    `threads` OpenMP threads, printed as one JSON line."""
    import oracle
    used = oracle.set_threads(threads)
    g = _golden_c1()
    o = _oracle_for_workload()
    rows, nnz, tb, ts = oracle_step_sample(o, i0, seconds, g["arpack_matvecs"], g["arpack_ncv"])
    print(json.dumps({"threads": used, "rows": rows, "nnz": nnz, "build_s": tb, "solve_s": ts}))


def _cpu_sample(threads, seconds, i0):
    env = dict(os.environ)
    if threads == 1:
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            env[k] = "1"
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-sample", str(threads),
                          "--cpu-seconds", str(seconds), "--cpu-row0", str(i0)],
                         capture_output=True, text=True, env=env, timeout=600)
    if out.returncode != 0:
        raise RuntimeError("CPU sample failed: " + out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def _phase(r):
    return {"threads": r["threads"], "rows": r["rows"], "nnz": r["nnz"],
            "build_nnz_per_s": r["nnz"] / r["build_s"],
            "solve_nnz_per_s": r["nnz"] / r["solve_s"],
            "step_nnz_per_s": r["nnz"] / (r["build_s"] + r["solve_s"]),
            "build_s": round(r["build_s"], 3), "solve_s": round(r["solve_s"], 3)}


def cpu_baseline(seconds):
    """The oracle timed on the host cores, once on one thread and once on
    all of them, each a bounded sample of the workload's rows (about
    `seconds` of building, then the eigensolve's per-row work on the same
    rows).  value: H nonzeros per second of that build + solve sample on all
    cores, the unit of the GPU value."""
    nproc = os.cpu_count() or 1
    one = _phase(_cpu_sample(1, seconds * 0.5, 20000))
    allc = _phase(_cpu_sample(nproc, seconds * 0.5, 60000))
    g = _golden_c1()
    return {"value": allc["step_nnz_per_s"], "unit": "nnz/s", "cores": allc["threads"], "nproc": nproc,
            "kind": "oracle",
            "sample": "rows of the same H: FP64 Slater-Condon build (count, scan, fill; OpenMP over rows) "
                      "of ~%.0f s, then the oracle eigensolve's per-row work on those rows (%d CSR products "
                      "+ 2x Gram-Schmidt against %d columns, ARPACK's count for the whole H)"
                      % (seconds * 0.5, g["arpack_matvecs"], g["arpack_ncv"]),
            "phases": {"one_thread": one, "all_cores": allc},
            "build_nnz_per_s": allc["build_nnz_per_s"], "build_nnz_per_s_one_thread": one["build_nnz_per_s"]}


def run_reference(args):
    """The oracle, timed as it stands on all host cores: each step is one
    bounded sample of the workload (rows built, then the eigensolve's work on
    them), the unit of the GPU arm (H nonzeros per second of build + solve)."""
    rank, world, local = dist_info()
    if rank != 0:
        return
    import oracle
    nproc = os.cpu_count() or 1
    used = oracle.set_threads(nproc)
    g = _golden_c1()
    o = _oracle_for_workload()
    per_step = max(1.0, min(10.0, 60.0 / max(args.steps + args.warmup, 1)))
    for w in range(args.warmup):
        oracle_step_sample(o, 3000 * w, min(per_step, 1.0), g["arpack_matvecs"], g["arpack_ncv"])
    tot_nnz, tot_t, tot_rows, tb, ts = 0, 0.0, 0, 0.0, 0.0
    for s in range(args.steps):
        rows, nnz, b, sv = oracle_step_sample(o, 7919 * (s + 1), per_step, g["arpack_matvecs"], g["arpack_ncv"])
        tot_nnz += nnz
        tot_rows += rows
        tb += b
        ts += sv
    tot_t = tb + ts
    v = tot_nnz / tot_t
    rec = {"impl": "reference", "metric": METRIC, "value": v, "unit": "nnz/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": tot_t / args.steps * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD,
                      "sample": "each step: ~%.0f s of row builds on %d threads, then %d CSR products of those rows "
                                "with Gram-Schmidt against %d columns" % (per_step, used, g["arpack_matvecs"],
                                                                          g["arpack_ncv"])},
           "cpu_baseline": {"value": v, "unit": "nnz/s", "cores": used, "nproc": nproc, "kind": "oracle",
                            "sample": "%d rows, %d nonzeros over %d steps" % (tot_rows, tot_nnz, args.steps),
                            "build_nnz_per_s": tot_nnz / tb, "solve_nnz_per_s": tot_nnz / ts},
           "e2e": {"value": v, "unit": "nnz/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(rec))


def main():
    args = parse()
    if args.cpu_sample:
        cpu_sample_main(args.cpu_sample, args.cpu_seconds, args.cpu_row0)
    elif args.products_only:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps({"products": run_products_leg(load_peaks()[0])}))
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
