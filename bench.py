#!/usr/bin/env python
"""HAPOD throughput on one GB300: snapshot columns/s and algorithmic GB/s.

Workload (synthetic, seeded): n = 2^20 rows, 64 leaves x 256 snapshot columns of
the advection-diffusion trajectory u(x, t) = sum_k a_k exp(-nu k^2 t) sin(k(x - c t))
(32 harmonics, a_k ~ N(0, k^-2), nu = 1e-3, c = 1, t ~ U[0, 1]), balanced binary
tree of edge depth 6 (L_T = 7), eps = 1e-5 relative (sum_s ||s - P s||^2 <=
(1e-5 ||X||_F)^2), omega = 0.5.  The inputs (137 GB in FP64, 69 GB in FP32) are
generated on the device before timing and are larger than L2, so no flush is
needed between steps.

A step is one full HAPOD through the C ABI: create, push every leaf, result,
destroy.  The headline is the digit-slice FP64 form (FP64 data and results; Gram
and X V from exact integer digit products on the tensor cores) at the workload's
tolerance eps = 1e-5 rel; the FP64 ALU form runs at the same tolerance for
comparison.  The mixed form (FP32 snapshots, TF32 tensor-core Gram) resolves
singular values only down to its measured Gram error (noise eigenvalues summing
to ~6e-8 of the trace), so it is run at eps = 1e-2 rel, and the FP64 ALU form is
run at that tolerance too for a same-accuracy comparison; all appear under
"forms".

The end-to-end figure ("e2e") repeats the headline HAPOD from pinned host buffers
right after the headline form: the 64 leaf uploads (137 GB) are queued on a copy
stream and the context processes leaves in batches of 4 as they land, so the
host-to-device link (~210 GB/s measured) bounds it; "h2d_gbs" is the upload rate
seen during that step.

--impl reference times the CPU FP64 oracle on the host cores on a bounded sample
of the same workload (there is no other reference implementation of the method).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_ROWS = 1 << 20
LEAVES = 64
COLS = 256
SEED = 1607052102
EPS_REL = 1e-5
MIXED_EPS_REL = 1e-2
OMEGA = 0.5
TREE_DEPTH = 6
METRIC = "HAPOD snapshot columns/s at stated error (eps = 1e-5 rel, omega = 0.5)"
UNIT = "columns/s"
WORKLOAD = ("advection-diffusion HAPOD, n=2^20 rows, 64 leaves x 256 snapshots (16384 columns), "
            "balanced binary tree L_T=7, eps=1e-5 rel, omega=0.5")
ORACLE_SAMPLE_ROWS = N_ROWS // 16


def _peaks():
    """(HBM GB/s, bf16 TFLOP/s sustained, source).  The tensor-core kernels run inside a
    step of seconds, so the sustained bf16 figure is their denominator."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p.get("bf16_tflops_sustained", p["bf16_tflops"])), "measured"
    except Exception:
        return 6800.0, 1700.0, "fallback"


FP64_PEAK_TFLOPS = 1.25  # nominal FP64 rate of GB300 (CUDA cores and tensor cores alike)


# ----------------------------------------------------------------- clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.QUERY}",
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------- inputs
def make_inputs(dtype, device):
    import numpy as np
    import torch

    from paper_1607_05210_gb300 import synth

    B = torch.from_numpy(synth.fourier_basis(N_ROWS)).to(device)  # n x 64
    C = synth.advection_diffusion_coeffs(LEAVES * COLS, SEED)     # 64 x |S|
    bufs, fro2 = [], 0.0
    for j in range(LEAVES):
        Ct = torch.from_numpy(np.ascontiguousarray(C[:, j * COLS:(j + 1) * COLS].T)).to(device)
        Xt = (Ct @ B.T).to(dtype)  # COLS x n: row i = snapshot i (column-major n x COLS)
        fro2 += float(torch.sum(Xt.double() ** 2))
        bufs.append(Xt)
        del Ct
    del B
    torch.cuda.synchronize()
    return bufs, fro2


def tree():
    from paper_1607_05210_gb300 import synth

    parent = synth.balanced_tree(2, TREE_DEPTH)
    leaves = synth.leaves_of(parent)
    cols = [0] * len(parent)
    for a in leaves:
        cols[a] = COLS
    return parent, leaves, cols


# ----------------------------------------------------------------- our arm
def run_form(H, precision, bufs, fro2, steps, warmup, stream, dist_ctx, eps_rel=EPS_REL, shape=None,
             omega=OMEGA, n_rows=N_ROWS):
    import torch

    parent, leaves, cols = shape if shape is not None else tree()
    eps = eps_rel * math.sqrt(fro2)
    launches = [0]
    info = {}

    def step(profile):
        ctx = H.hapod_create(parent, cols, eps, omega, n_rows, precision, stream=stream,
                             flags=H.HAPOD_FLAG_PROFILE if profile else 0)
        for i, a in enumerate(leaves):
            H.hapod_push(ctx, a, bufs[i].t())
        s, U, st = H.hapod_result(ctx, device=bufs[0].device)
        if profile:
            prof = H.hapod_profile(ctx)
            for k, v in prof.items():
                d = info.setdefault(k, {"ms": 0.0, "launches": 0, "bytes": 0.0, "flops": 0.0})
                for f in d:
                    d[f] += v[f]
            launches[0] += sum(v["launches"] for v in prof.values())
            info["_nodes"] = [H.hapod_node_stats(ctx, a) for a in range(len(parent))]
            info["_k"] = int(s.numel())
            info["_status"] = int(st)
        H.hapod_destroy(ctx)
        return s

    for _ in range(warmup):
        step(False)
    torch.cuda.synchronize()
    dist_ctx.barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        ev0.record(stream)
        for _ in range(steps):
            step(True)
        ev1.record(stream)
    torch.cuda.synchronize()
    dist_ctx.barrier()
    ms = ev0.elapsed_time(ev1) / steps
    ms = dist_ctx.max(ms)
    # algorithmic bytes of the whole HAPOD (b n (2 m + k) per node)
    es = 4 if precision == H.HAPOD_MIXED_TF32X3 else 8
    alg_bytes = sum(es * n_rows * (2 * st_["m"] + max(0, st_["k"])) for st_ in info["_nodes"] if st_["m"] > 0)
    per = {k: {f: v[f] / steps for f in v} for k, v in info.items() if not k.startswith("_")}
    return {"ms": ms, "alg_bytes": alg_bytes, "steps": per, "launches_per_step": launches[0] // steps,
            "k": info["_k"], "status": info["_status"],
            "max_inner_k": max([st_["k"] for a, st_ in enumerate(info["_nodes"])
                                if st_["level"] > 1 and parent[a] >= 0] or [0]),
            "max_intermediate_k": max([st_["k"] for a, st_ in enumerate(info["_nodes"]) if parent[a] >= 0] or [0]),
            "leaf_k": max(st_["k"] for st_ in info["_nodes"] if st_["level"] == 1)}


E2E_PENDING = 4  # leaves per processing batch in the end-to-end run (max_pending_leaves)


def run_e2e(H, precision, host_bufs, dev_bufs, fro2, steps, stream):
    """Same HAPOD through the public API from pinned host buffers: H2D of every leaf and
    D2H of the result (sigma, modes) inside the timed region.  The leaf copies are
    queued up front on a copy stream; each push waits for its leaf's copy, and the
    context processes leaves in batches of E2E_PENDING (max_pending_leaves, Sec. 3.4)
    so that the copies of later leaves overlap the processing of earlier ones."""
    import torch

    parent, leaves, cols = tree()
    eps = EPS_REL * math.sqrt(fro2)
    h2d = sum(b.numel() * b.element_size() for b in host_bufs)
    d2h = [0]
    copy_stream = torch.cuda.Stream(dev_bufs[0].device)
    cev = [torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)]

    def step():
        ctx = H.hapod_create(parent, cols, eps, OMEGA, N_ROWS, precision, stream=stream,
                             max_pending_leaves=E2E_PENDING)
        copy_stream.wait_stream(stream)
        done = []
        with torch.cuda.stream(copy_stream):
            cev[0].record(copy_stream)
            for i in range(len(leaves)):
                dev_bufs[i].copy_(host_bufs[i], non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(copy_stream)
                done.append(ev)
            cev[1].record(copy_stream)
        for i, a in enumerate(leaves):
            stream.wait_event(done[i])
            H.hapod_push(ctx, a, dev_bufs[i].t())
        s, U, st = H.hapod_result(ctx, device=dev_bufs[0].device)
        Uh = U.cpu()
        d2h[0] = Uh.numel() * Uh.element_size() + s.numel() * 8
        H.hapod_destroy(ctx)

    step()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        ev0.record(stream)
        for _ in range(steps):
            step()
        ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / steps
    copy_ms = cev[0].elapsed_time(cev[1])  # the last step's leaf uploads alone
    return {"value": LEAVES * COLS / (ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h[0],
            "ms_per_step": ms, "h2d_ms": copy_ms, "h2d_gbs": h2d / (copy_ms / 1e3) / 1e9}


# DRAM traffic of the dominant kernels, from one ncu capture per kernel
# (dram__bytes_read.sum + dram__bytes_write.sum of a single launch), stored in
# profiles/traffic.json with the SHA-256 of the kernel's source file at capture
# time.  A kernel whose source changed since then reports traffic = null.
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")


def kernel_traffic(kernel: str):
    """(bytes per launch, note) of the last capture of `kernel`, or (None, why)."""
    import hashlib

    try:
        with open(TRAFFIC_FILE) as f:
            rec = json.load(f)[kernel]
    except (OSError, KeyError, ValueError):
        return None, "no capture recorded"
    src = rec["source"] if os.path.isabs(rec["source"]) else os.path.join(ROOT, rec["source"])
    try:
        with open(src, "rb") as f:
            digest = hashlib.sha256(f.read()).hexdigest()
    except OSError:
        return None, "kernel source missing"
    if digest != rec["sha256"]:
        return None, f"{rec['source']} changed since the capture"
    return float(rec["bytes_per_launch"]), rec["note"]


def f64_alu(precision, H):
    """Steps that run on the FP64 FMA pipe: every FP64-ALU step, the X V of the digit-slice form."""
    return precision in (H.HAPOD_FP64, H.HAPOD_FP64_OZAKI)


def roofline(res, precision, H, hbm, bf16, dom=None):
    steps = res["steps"]
    if dom is None:
        dom = max((k for k in steps if steps[k]["launches"] > 0), key=lambda k: steps[k]["ms"])
    d = steps[dom]
    if precision == H.HAPOD_FP64_OZAKI and dom == "gram":
        # the method's bytes: one pass over the FP64 snapshots, b n m per node (the
        # library's step accounting); the digit-pair tensor work (28 fp16 products per
        # FP64 product of the upper triangle) is reported beside it
        ach = d["bytes"] / (d["ms"] / 1e3) / 1e9
        traffic, note = kernel_traffic("gram_oz_kernel")
        return dom, {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                     "traffic": traffic, "traffic_note": note,
                     "digit_tflops": 28.0 * d["flops"] / (d["ms"] / 1e3) / 1e12,
                     "kernel": "gram_oz_kernel + oz_reduce_kernel (tcgen05 fp16 digit-pair MMAs); achieved = "
                               "8 n m algorithmic bytes per node over the step's CUDA-event time; digit_tflops = "
                               "28 fp16 pair products per FP64 product of the upper triangle over the same time"}
    if f64_alu(precision, H) and dom in ("gram", "modes"):
        ach = d["flops"] / (d["ms"] / 1e3) / 1e12
        return dom, {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": ach / FP64_PEAK_TFLOPS, "traffic": None,
                     "kernel": f"{dom} (FP64 FMA pipe; peak = nominal GB300 FP64 rate)"}
    if dom in ("gram", "modes"):
        ach = d["bytes"] / (d["ms"] / 1e3) / 1e9
        return dom, {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                     "traffic": None, "kernel": dom}
    return dom, {"bound": "alu", "achieved": None, "peak": None, "unit": None, "frac": None, "traffic": None,
                 "kernel": dom}


# ----------------------------------------------------------------- oracle
def oracle_sample():
    """A 256-column leaf of the same trajectory type at n/16 rows, FP64, with the leaf
    tolerance of the tree (Thm. cor:hapod_bound) computed from the sample's own RMS
    snapshot norm."""
    import oracle
    from paper_1607_05210_gb300 import synth

    X = synth.advection_diffusion(ORACLE_SAMPLE_ROWS, COLS, SEED)
    parent, leaves, cols = tree()
    eps_star = EPS_REL * math.sqrt(float((X * X).sum()) / COLS)
    return X, oracle.tolerances(parent, cols, eps_star, OMEGA)[leaves[0]]


def time_oracle(steps: int, warmup: int):
    import oracle

    X, eps_leaf = oracle_sample()
    for _ in range(warmup):
        oracle.pod(X, eps_leaf)
    t = []
    for _ in range(steps):
        t0 = time.perf_counter()
        oracle.pod(X, eps_leaf)
        t.append(time.perf_counter() - t0)
    sec = statistics.median(t)
    # cols/s of a full-length leaf: the oracle's cost is linear in the rows (QR + n-length reflectors)
    value = COLS / (sec * (N_ROWS / ORACLE_SAMPLE_ROWS))
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return value, sec, cores


# ----------------------------------------------------------------- distributed
class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist

            dist.init_process_group("nccl" if self._cuda() else "gloo")
            self.pg = dist

    @staticmethod
    def _cuda():
        import torch

        return torch.cuda.is_available()

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, v: float) -> float:
        if not self.pg:
            return v
        import torch

        t = torch.tensor([v], dtype=torch.float64, device="cuda" if self._cuda() else "cpu")
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


SWEEP_OMEGAS = (0.1, 0.25, 0.5, 0.75, 0.9, 0.95, 0.99, 0.999)
SWEEP_PARTITIONS = ((10, 1000), (40, 250), (100, 100), (400, 25), (1000, 10))  # blocks x columns (10^4)
SWEEP_DEPTHS = (2, 3, 4, 5)


def direct_pod_rank(sigma, eps):
    """N of POD(S, eps) (Def. truncated POD) from all singular values of S."""
    tail = 0.0
    for j in range(len(sigma) - 1, -1, -1):
        if tail + sigma[j] ** 2 > eps * eps:
            return j + 1
        tail += sigma[j] ** 2
    return 0


def run_sweep(kind, H, device, dist_ctx):
    """Sec. 4.3 (omega) and Sec. 4.2 (tree shape) on the digit-slice FP64 form: one
    JSON line per configuration (1 warm-up + 2 timed HAPODs).  The direct POD's
    rank comes from the closed form sigma(X) = sqrt(n/2) sigma(C) of the
    advection-diffusion snapshots X = B C."""
    import numpy as np
    import torch

    from paper_1607_05210_gb300 import synth

    stream = torch.cuda.Stream(device)
    prec = H.HAPOD_FP64_OZAKI
    if kind == "omega":
        bufs, fro2 = make_inputs(torch.float64, device)
        sig = math.sqrt(N_ROWS / 2.0) * np.linalg.svd(synth.advection_diffusion_coeffs(LEAVES * COLS, SEED),
                                                     compute_uv=False)
        k_pod = direct_pod_rank(sig, EPS_REL * math.sqrt(fro2))
        for w in SWEEP_OMEGAS:
            r = run_form(H, prec, bufs, fro2, 2, 1, stream, dist_ctx, EPS_REL, omega=w)
            print(json.dumps({"sweep": "omega", "omega": w, "workload": WORKLOAD.replace("omega=0.5", f"omega={w}"),
                              "value": LEAVES * COLS / (r["ms"] / 1e3), "unit": UNIT, "ms_per_step": r["ms"],
                              "k_root": r["k"], "direct_pod_k": k_pod, "additional_modes": r["k"] - k_pod,
                              "max_intermediate_k": r["max_intermediate_k"], "status": r["status"]}), flush=True)
        return
    total = 10_000
    Xt = synth.advection_diffusion_device(N_ROWS, total, SEED, torch.float64, device)  # total x n
    fro2 = sum(float(torch.sum(Xt[i:i + 500] ** 2)) for i in range(0, total, 500))
    sig = math.sqrt(N_ROWS / 2.0) * np.linalg.svd(synth.advection_diffusion_coeffs(total, SEED), compute_uv=False)
    k_pod = direct_pod_rank(sig, EPS_REL * math.sqrt(fro2))
    for s_blocks, c in SWEEP_PARTITIONS:
        bufs = [Xt[i * c:(i + 1) * c] for i in range(s_blocks)]
        for d in SWEEP_DEPTHS:
            parent = synth.nary_tree(s_blocks, d)
            leaves = synth.leaves_of(parent)
            cols = [0] * len(parent)
            for a in leaves:
                cols[a] = c
            r = run_form(H, prec, bufs, fro2, 2, 1, stream, dist_ctx, EPS_REL, shape=(parent, leaves, cols))
            arity = 1
            while arity ** d < s_blocks:
                arity += 1
            print(json.dumps({"sweep": "trees", "blocks": s_blocks, "block_cols": c, "edge_depth": d,
                              "levels": d + 1, "arity": arity, "nodes": len(parent),
                              "value": total / (r["ms"] / 1e3), "unit": UNIT, "ms_per_step": r["ms"],
                              "k_root": r["k"], "direct_pod_k": k_pod, "max_intermediate_k": r["max_intermediate_k"],
                              "status": r["status"], "n": N_ROWS, "eps_rel": EPS_REL, "omega": OMEGA}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--forms", default="mixed,fp64,oz",
                    help="comma list of forms: 'oz' (digit-slice FP64, the headline when present), "
                         "'fp64' (FP64 ALU), 'mixed' (FP32 snapshots at eps = 1e-2)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--profile-leaf", action="store_true",
                    help="run two digit-slice Gram + X V calls on one 2^20 x 256 FP64 leaf (k = 19) and exit: "
                         "the small case for ncu captures of oz_split / gram_oz / modes_oz")
    ap.add_argument("--profile-form", choices=["oz", "fp64", "mixed"], default="oz",
                    help="with --profile-leaf: 'fp64' runs three FP64 Gram calls on a 2^20 x 64 "
                         "advection-diffusion leaf (gram_f64_tiles), 'mixed' three mixed-form Gram calls on a "
                         "2^20 x 256 FP32 one (gram_tc_kernel)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sweep", choices=["omega", "trees"],
                    help="print one JSON line per configuration and exit: 'omega' runs the benchmark "
                         "workload for omega in 0.1 .. 0.999 (Sec. 4.3); 'trees' runs 10^4 advection-diffusion "
                         "columns in 10 x 1000 .. 1000 x 10 blocks on balanced trees of edge depth 2..5 (Sec. 4.2)")
    args = ap.parse_args()
    os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1))
    dist_ctx = Dist()

    if args.impl == "reference":
        if dist_ctx.rank != 0:
            dist_ctx.close()
            return
        value, sec, cores = time_oracle(args.steps, args.warmup)
        sample = (f"oracle POD (Householder QR + one-sided Jacobi, FP64) of one 256-column leaf at n/16 = "
                  f"{ORACLE_SAMPLE_ROWS} rows per step, {sec:.2f} s; columns/s scaled to full-length leaves")
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic", "config": {"workload": WORKLOAD, "form": "cpu oracle"},
                          "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                                           "sample": sample},
                          "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        dist_ctx.close()
        return

    import torch

    torch.cuda.set_device(dist_ctx.local)
    device = torch.device("cuda", dist_ctx.local)
    from paper_1607_05210_gb300 import hapod as H

    if args.profile_leaf and args.profile_form != "oz":
        from paper_1607_05210_gb300 import synth

        cols, dtype, prec = ((64, torch.float64, H.HAPOD_FP64) if args.profile_form == "fp64"
                             else (COLS, torch.float32, H.HAPOD_MIXED_TF32X3))
        X = synth.advection_diffusion_device(N_ROWS, cols, SEED, dtype, device).t()  # column-major n x cols
        for _ in range(3):
            G = H.hapod_gram(X, prec)
        torch.cuda.synchronize()
        print(json.dumps({"profile_leaf": True, "form": args.profile_form, "G00": float(G[0, 0])}))
        dist_ctx.close()
        return
    if args.profile_leaf:
        torch.manual_seed(SEED)
        X = torch.randn((COLS, N_ROWS), dtype=torch.float64, device=device).t()  # column-major n x m
        V = torch.randn((19, COLS), dtype=torch.float64, device=device).t() / 16.0
        for _ in range(2):
            G = H.hapod_gram(X, H.HAPOD_FP64_OZAKI)
            Y = H.hapod_modes(X, V, 19, None, H.HAPOD_FP64_OZAKI)
        torch.cuda.synchronize()
        print(json.dumps({"profile_leaf": True, "G00": float(G[0, 0]), "Y00": float(Y[0, 0])}))
        dist_ctx.close()
        return

    if args.sweep:
        if dist_ctx.rank == 0:
            run_sweep(args.sweep, H, device, dist_ctx)
        dist_ctx.close()
        return

    hbm, bf16, peak_src = _peaks()
    stream = torch.cuda.Stream(device)
    total_cols = LEAVES * COLS * dist_ctx.world

    def summarise(r, precision, eps_rel, dom=None):
        d, roof = roofline(r, precision, H, hbm, bf16, dom)
        roof["peak_source"] = peak_src if roof["bound"] in ("hbm", "tensor") else "nominal"
        return {"eps_rel": eps_rel, "value": total_cols / (r["ms"] / 1e3), "unit": UNIT, "ms_per_step": r["ms"],
                "gb_per_s": r["alg_bytes"] / (r["ms"] / 1e3) / 1e9 * dist_ctx.world,
                "k_root": r["k"], "max_leaf_k": r["leaf_k"], "max_inner_k": r["max_inner_k"],
                "step_ms": {k: v["ms"] for k, v in r["steps"].items()}, "roofline": roof}

    forms = {}
    # pinned host buffers for the end-to-end leg, allocated before any device work
    host = None
    if not args.no_e2e:
        try:
            host = [torch.empty((COLS, N_ROWS), dtype=torch.float64, pin_memory=True) for _ in range(LEAVES)]
        except (RuntimeError, MemoryError) as ex:
            host = str(ex)[:120]
    # mixed form at the tolerance its precision floor supports
    if "mixed" in args.forms:
        bufs, fro2 = make_inputs(torch.float32, device)
        try:
            rm = run_form(H, H.HAPOD_MIXED_TF32X3, bufs, fro2, args.steps, args.warmup, stream, dist_ctx,
                          MIXED_EPS_REL)
            forms[f"mixed@{MIXED_EPS_REL:g}"] = summarise(rm, H.HAPOD_MIXED_TF32X3, MIXED_EPS_REL, "gram")
            forms[f"mixed@{MIXED_EPS_REL:g}"]["launches_per_step"] = rm["launches_per_step"]
        except H.HapodError as e:
            forms[f"mixed@{MIXED_EPS_REL:g}"] = {"unavailable": str(e)}
        del bufs
        torch.cuda.empty_cache()
    # FP64 snapshots: the digit-slice form (headline) and the FP64 ALU form at the
    # workload tolerance, then the FP64 ALU form at the mixed tolerance
    bufs, fro2 = make_inputs(torch.float64, device)
    head = head_prec = clocks = None
    if "oz" in args.forms:
        sampler = ClockSampler(dist_ctx.local)
        head = run_form(H, H.HAPOD_FP64_OZAKI, bufs, fro2, args.steps, args.warmup, stream, dist_ctx, EPS_REL)
        clocks = sampler.stop()
        head_prec = H.HAPOD_FP64_OZAKI
        forms[f"fp64_ozaki@{EPS_REL:g}"] = summarise(head, H.HAPOD_FP64_OZAKI, EPS_REL)
    e2e = None

    steps_e2e = args.steps

    def measure_e2e(prec, key):
        # right after the headline form, with the pool's cached blocks returned first
        if not isinstance(host, list):
            return {"value": None, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0,
                    "note": f"pinned host buffers unavailable: {host}"}
        H.hapod_trim_pool(stream)
        for h_, b in zip(host, bufs):
            h_.copy_(b)
        # the link alone: one upload of every leaf with nothing else running
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            c0.record(stream)
            for h_, b in zip(host, bufs):
                b.copy_(h_, non_blocking=True)
            c1.record(stream)
        torch.cuda.synchronize()
        idle_gbs = sum(h_.numel() * 8 for h_ in host) / (c0.elapsed_time(c1) / 1e3) / 1e9
        r = run_e2e(H, prec, host, bufs, fro2, steps_e2e, stream)
        r["form"] = key
        r["max_pending_leaves"] = E2E_PENDING
        r["h2d_gbs_alone"] = idle_gbs
        return r

    if not args.no_e2e and head is not None:
        e2e = measure_e2e(head_prec, f"fp64_ozaki@{EPS_REL:g}")
    if "fp64" in args.forms or head is None:
        sampler = ClockSampler(dist_ctx.local)
        alu = run_form(H, H.HAPOD_FP64, bufs, fro2, args.steps, args.warmup, stream, dist_ctx, EPS_REL)
        alu_clocks = sampler.stop()
        forms[f"fp64@{EPS_REL:g}"] = summarise(alu, H.HAPOD_FP64, EPS_REL)
        if head is None:
            head, head_prec, clocks = alu, H.HAPOD_FP64, alu_clocks
            if not args.no_e2e:
                e2e = measure_e2e(head_prec, f"fp64@{EPS_REL:g}")
        else:
            forms[f"fp64_ozaki@{EPS_REL:g}"]["speedup_vs_fp64_alu"] = alu["ms"] / head["ms"]
    head_key = f"fp64_ozaki@{EPS_REL:g}" if head_prec == H.HAPOD_FP64_OZAKI else f"fp64@{EPS_REL:g}"
    if "mixed" in args.forms:
        r2 = run_form(H, H.HAPOD_FP64, bufs, fro2, max(1, min(args.steps, 2)), 1, stream, dist_ctx, MIXED_EPS_REL)
        forms[f"fp64@{MIXED_EPS_REL:g}"] = summarise(r2, H.HAPOD_FP64, MIXED_EPS_REL)
        mk = f"mixed@{MIXED_EPS_REL:g}"
        if "value" in forms.get(mk, {}):
            forms[mk]["speedup_vs_fp64_same_eps"] = forms[mk]["value"] / forms[f"fp64@{MIXED_EPS_REL:g}"]["value"]
    del bufs
    host = None
    torch.cuda.empty_cache()

    value = total_cols / (head["ms"] / 1e3)
    hs = forms[head_key]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist_ctx.world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "form": head_key.split("@")[0], "parallelism": f"replicas x{dist_ctx.world}",
                   "l2": "inputs larger than L2 (no flush needed)"},
        "gb_per_s": hs["gb_per_s"],
        "roofline": hs["roofline"],
        "gpu_launches": head["launches_per_step"] * args.steps,
        "clocks": clocks,
        "e2e": e2e,
        "result": {"k_root": head["k"], "max_leaf_k": head["leaf_k"], "max_inner_k": head["max_inner_k"],
                   "status": head["status"]},
        "step_ms": hs["step_ms"],
        "forms": forms,
    }
    if dist_ctx.rank == 0 and dist_ctx.world == 1 and not args.no_cpu_baseline:
        v, sec, cores = time_oracle(1, 0)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"one 256-column leaf at n/16 rows ({sec:.2f} s), scaled to full leaves"}
    if dist_ctx.rank == 0:
        print(json.dumps(line))
    dist_ctx.close()


if __name__ == "__main__":
    main()
