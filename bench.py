#!/usr/bin/env python
"""HAPOD throughput on one GB300: snapshot columns/s and algorithmic GB/s at the
stated error, mixed/batched form beside the FP64-accurate form.

Headline workload (precision form): n = 2^22 rows, 256 leaves x 128 FP32 snapshot
columns (32,768 columns, 512 GiB) of the travelling-pulse trajectory -- the
advection-diffusion field u = sum_k a_k exp(-nu k^2 t) sin(k(x - c t)) (32
harmonics, a_k ~ N(0, k^-2), nu = 1e-3, c = 1) plus 64 Gaussian pulses of width 0.01
with amplitudes 1/p moving at speed c, snapshot times from Philox4x32-10 -- on a
balanced quaternary tree of edge depth 4 (L_T = 5), eps = 1e-4 relative, omega =
0.5.  The snapshots are generated on the device by the library's generator
(hapod_synth_snapshots) in waves of 16 leaves (one level-3 subtree, 32 GiB FP32):
512 GiB never fit HBM at once.  The context processes each wave as it is pushed
(max_pending_leaves = 16), so a wave's leaves, its four level-2 nodes and its
level-3 node run before the next wave is generated; the root levels run with the
last wave.  Timed region: the sum over waves of the CUDA-event interval around the
wave's pushes (plus hapod_result after the last), so inputs are resident in HBM when
each interval starts and generation is reported separately.  Every wave's leaves
(2 GiB each) are larger than L2, so no flush is needed.

Forms: the mixed fixed-point form (HAPOD_MIXED_FX3: FP32 snapshots, Gram from exact
8-bit digit products on the tensor cores with int64 sums, tensor-core X V, FP64
eigensolve/tails, CholQR2 at the root) is the headline; the digit-slice FP64 form
(HAPOD_FP64_OZAKI: the same values in FP64) runs at the same eps beside it.

Other workloads ("workloads"): the FP64 advection-diffusion workload at n = 2^20,
64 leaves x 256 columns, eps = 1e-5 rel, on the balanced binary tree (L_T = 7) and
on the two-level star, resident in HBM (137 GB), digit-slice and FP64 ALU forms.

End to end ("e2e"): the headline HAPOD through the public API from pinned host
buffers.  Per wave the 16 generated leaves are first copied to pinned host memory
(untimed); the timed interval then holds their host-to-device copies (a copy
stream, each push waiting for its leaf) and the wave's processing.

--impl reference and cpu_baseline time the CPU FP64 oracle (Householder QR +
one-sided Jacobi per node) on a bounded sample: one leaf and one level-2 node of
the headline tree at two reduced row counts; each node kind's time is fitted
linearly in n and the whole tree (256 leaves + 85 inner nodes) is extrapolated to
n = 2^22.
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

UNIT = "columns/s"
METRIC = "HAPOD snapshot columns/s at stated error (mixed/batched form vs FP64 form)"

# precision workload: quaternary tree, device-generated travelling pulses
C3 = {"name": "c3", "n": 1 << 22, "leaves": 256, "cols": 128, "arity": 4, "depth": 4, "eps_rel": 1e-4,
      "omega": 0.5, "wave": 16, "seed": 1607052103}
C3_WORKLOAD = ("travelling-pulse HAPOD (precision form), n=2^22 FP32 rows, 256 leaves x 128 snapshots "
               "(32768 columns, 512 GiB generated on the device in waves of 16 leaves), quaternary tree L_T=5, "
               "eps=1e-4 rel, omega=0.5")

# streamed incremental workload: 64 chunks of 64 columns, never all resident, on a
# left-deep chain of four depth-4 binary subtrees (Sec. 3.2, skinny tree)
C5 = {"name": "c5", "n": 1 << 23, "leaves": 64, "cols": 64, "subtrees": 4, "depth": 4, "eps_rel": 1e-4,
      "omega": 0.5, "wave": 8, "seed": 1607052105}
C5_WORKLOAD = ("streamed incremental HAPOD, n=2^23 FP32 rows, 4096 snapshots generated on the device in chunks of 64 "
               "(2 GiB each, 8 chunks resident at a time), left-deep chain of 4 binary subtrees of depth 4 (L_T=8), "
               "eps=1e-4 rel, omega=0.5")

# batched uneven leaves: 1000 prescribed-spectrum leaves with m ~ U{16..512}
C4 = {"name": "c4", "n": 1 << 18, "leaves": 1000, "lo": 16, "hi": 512, "rank": 200, "arity": 4, "depth": 5,
      "eps_rel": 1e-5, "omega": 0.5, "wave": 64, "seed": 1607052104}
C4_WORKLOAD = ("batched uneven leaves, n=2^18 FP32 rows, 1000 leaves with m ~ U{16..512} (265336 columns, 278 GB, "
               "generated on the device in waves of 64 leaves), shared rank-200 basis, sigma_j = 10^(-delta j) with "
               "delta ~ U[1/40, 1/10] per leaf, + 1e-10 N(0,1), quaternary tree L_T=6 (first 1000 of 1024 slots), "
               "eps=1e-5 rel, omega=0.5")

# FP64 advection-diffusion workload, resident
N_ROWS = 1 << 20
LEAVES = 64
COLS = 256
SEED = 1607052102
EPS_REL = 1e-5
OMEGA = 0.5
TREE_DEPTH = 6
C2_WORKLOAD = ("advection-diffusion HAPOD, n=2^20 FP64 rows, 64 leaves x 256 snapshots (16384 columns), "
               "eps=1e-5 rel, omega=0.5")


def _peaks():
    """(HBM GB/s, bf16 TFLOP/s sustained, source).  The kernels run inside a step of
    seconds, so the sustained bf16 figure is the tensor denominator."""
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


# ----------------------------------------------------------------- precision workload (device-generated)
def c3_tree(wl=C3):
    """(parent, leaves in push order, cols): leaf i of the push order holds global
    columns i * cols .. (i + 1) * cols - 1 of the trajectory."""
    from paper_1607_05210_gb300 import synth

    if wl["name"] == "c4":
        parent = synth.balanced_tree(wl["arity"], wl["depth"], wl["leaves"])
        leaves = synth.leaves_of(parent)
        m = synth.uneven_leaf_cols(wl["seed"], wl["leaves"], wl["lo"], wl["hi"])
        cols = [0] * len(parent)
        for i, a in enumerate(leaves):
            cols[a] = int(m[i])
        return parent, leaves, cols
    if wl["name"] == "c5":
        parent = synth.chain_of_subtrees(wl["subtrees"], wl["depth"])
        leaves = synth.leaves_of(parent)
        # stream order: subtree 1 (deepest in the chain) first, then 2, 3, 4, so that each
        # chain node can run as soon as its subtree has arrived
        per = len(leaves) // wl["subtrees"]
        blocks = [leaves[i:i + per] for i in range(0, len(leaves), per)]
        leaves = [a for b in reversed(blocks) for a in b]
    else:
        parent = synth.balanced_tree(wl["arity"], wl["depth"])
        leaves = synth.leaves_of(parent)
    cols = [0] * len(parent)
    for a in leaves:
        cols[a] = wl["cols"]
    return parent, leaves, cols


def c3_params(H, wl=C3):
    from paper_1607_05210_gb300 import synth

    return H.synth_params(**synth.pulse_workload(wl["seed"]))


class PulseGenerator:
    """Leaf i of the travelling-pulse workloads = global columns i * cols .. (i + 1) *
    cols - 1, written by the library's device generator."""

    def __init__(self, H, wl, dtype, device, nbuf):
        import torch

        self.H, self.wl, self.dtype = H, wl, dtype
        self.params = c3_params(H, wl)
        self.bufs = [torch.empty((wl["cols"], wl["n"]), dtype=dtype, device=device) for _ in range(nbuf)]

    def gen(self, leaf_index, slot, stream):
        """Leaf `leaf_index` into buffer `slot` (on `stream`); returns the cols x n view."""
        wl = self.wl
        self.H.hapod_synth_snapshots(self.params, wl["n"], leaf_index * wl["cols"], wl["cols"],
                                     self.bufs[slot].t(), stream=stream)
        return self.bufs[slot]


class UnevenGenerator:
    """Leaf i of the batched workload: Q[:, :r] diag(sigma_i) W_i^T + 1e-10 N(0, 1) formed
    on the device in FP32 (the FP64 form receives the same FP32 values).  Q (n x 200) and
    the W_i are drawn on the host once (synth.shared_basis, synth.leaf_factors); the noise
    comes from torch's device generator seeded per leaf."""

    _cache = {}

    def __init__(self, H, wl, dtype, device, nbuf):
        import numpy as np
        import torch

        from paper_1607_05210_gb300 import synth

        self.wl, self.dtype, self.device = wl, dtype, device
        key = (wl["seed"], wl["n"], wl["leaves"], str(device))
        if key not in UnevenGenerator._cache:
            m = synth.uneven_leaf_cols(wl["seed"], wl["leaves"], wl["lo"], wl["hi"])
            delta = synth.uneven_decays(wl["seed"], wl["leaves"])
            Q = torch.from_numpy(synth.shared_basis(wl["seed"], wl["n"], wl["rank"]).astype(np.float32)).to(device)
            WS = []
            for i in range(wl["leaves"]):
                W, sg = synth.leaf_factors(wl["seed"], i, int(m[i]), wl["rank"], float(delta[i]))
                WS.append(torch.from_numpy((W * sg).astype(np.float32)).to(device))  # m x r
            UnevenGenerator._cache[key] = (m, Q, WS)
        self.m, self.Q, self.WS = UnevenGenerator._cache[key]
        mmax = int(self.m.max())
        self.bufs = [torch.empty((mmax, wl["n"]), dtype=dtype, device=device) for _ in range(nbuf)]
        self.g = torch.Generator(device=device)

    def gen(self, leaf_index, slot, stream):
        import torch

        m = int(self.m[leaf_index])
        with torch.cuda.stream(stream):
            WS = self.WS[leaf_index]
            Xt = WS @ self.Q[:, :WS.shape[1]].t()  # m x n: row j = snapshot j
            self.g.manual_seed(self.wl["seed"] * 4096 + leaf_index)
            Xt += 1e-10 * torch.randn(Xt.shape, generator=self.g, device=self.device, dtype=torch.float32)
            out = self.bufs[slot][:m]
            out.copy_(Xt)
            del Xt
        return out


def make_generator(H, wl, dtype, device, nbuf):
    return UnevenGenerator(H, wl, dtype, device, nbuf) if wl["name"] == "c4" else PulseGenerator(H, wl, dtype,
                                                                                                  device, nbuf)


Generator = make_generator


def c3_fro2(H, wl, device, stream):
    """||X||_F^2 of the whole workload (FP64 sum of the FP32 snapshots), untimed."""
    import torch

    g = make_generator(H, wl, torch.float32, device, 1)
    tot = 0.0
    with torch.cuda.stream(stream):
        for i in range(wl["leaves"]):
            b = g.gen(i, 0, stream)
            tot += float(torch.linalg.vector_norm(b, dtype=torch.float64) ** 2)
    del g
    return tot


def run_waves(H, precision, wl, fro2, steps, warmup, stream, dist_ctx, host=None, batch=None, copy_streams=1):
    """The headline HAPOD: per wave, generate its leaves (untimed), then push them
    (timed).  With ``host`` (pinned host buffers, one wave), the generated leaves are
    first copied to the host (untimed) and the timed interval holds their uploads:
    each leaf in ``copy_streams`` column slices on as many copy streams, and with
    ``batch`` (max_pending_leaves, default the wave) the context processes every
    ``batch`` pushed leaves while the next leaves are still uploading."""
    import torch

    parent, leaves, cols = c3_tree(wl)
    dtype = H.DTYPE[precision]
    device = torch.device("cuda", torch.cuda.current_device())
    W = wl["wave"]
    B = batch or W
    gen = make_generator(H, wl, dtype, device, W)
    eps = wl["eps_rel"] * math.sqrt(fro2)
    copy_ss = [torch.cuda.Stream(device) for _ in range(max(1, copy_streams))] if host is not None else None
    info = {}
    launches = [0]
    gen_ms = [0.0]

    def step(profile, timed):
        ctx = H.hapod_create(parent, cols, eps, wl["omega"], wl["n"], precision, stream=stream,
                             max_pending_leaves=B, flags=H.HAPOD_FLAG_PROFILE if profile else 0)
        ms = 0.0
        d2h = 0
        for w0 in range(0, len(leaves), W):
            g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            views = {}
            with torch.cuda.stream(stream):
                g0.record(stream)
                for i in range(w0, min(len(leaves), w0 + W)):
                    views[i] = gen.gen(i, i - w0, stream)
                g1.record(stream)
            if host is not None:  # untimed: the wave's leaves to pinned host memory
                with torch.cuda.stream(stream):
                    for i in range(w0, min(len(leaves), w0 + W)):
                        host[i - w0][:views[i].shape[0]].copy_(views[i], non_blocking=True)
                stream.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if host is not None:
                done = []
                for cs in copy_ss:
                    cs.wait_event(e0)
                for i in range(w0, min(len(leaves), w0 + W)):
                    mi = views[i].shape[0]
                    cuts = [mi * q // len(copy_ss) for q in range(len(copy_ss) + 1)]
                    evs = []
                    for q, cs in enumerate(copy_ss):
                        with torch.cuda.stream(cs):
                            views[i][cuts[q]:cuts[q + 1]].copy_(host[i - w0][cuts[q]:cuts[q + 1]], non_blocking=True)
                            ev = torch.cuda.Event()
                            ev.record(cs)
                            evs.append(ev)
                    done.append(evs)
            for i in range(w0, min(len(leaves), w0 + W)):
                if host is not None:
                    for ev in done[i - w0]:
                        stream.wait_event(ev)
                H.hapod_push(ctx, leaves[i], views[i].t())
            if w0 + W >= len(leaves):
                s, U, st = H.hapod_result(ctx, device=device)
                if host is not None:
                    Uh = U.cpu()
                    d2h = Uh.numel() * Uh.element_size() + s.numel() * 8
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            if timed:
                gen_ms[0] += g0.elapsed_time(g1)
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
            info["_sigma"] = s.numpy().tolist()
        H.hapod_destroy(ctx)
        return ms, d2h

    for _ in range(warmup):
        step(False, False)
    dist_ctx.barrier()
    tot, d2h = 0.0, 0
    for _ in range(steps):
        ms, d2h = step(True, True)
        tot += ms
    dist_ctx.barrier()
    ms = dist_ctx.max(tot / steps)
    es = 4 if dtype == torch.float32 else 8
    alg_bytes = sum(es * wl["n"] * (2 * st_["m"] + max(0, st_["k"])) for st_ in info["_nodes"] if st_["m"] > 0)
    per = {k: {f: v[f] / steps for f in v} for k, v in info.items() if not k.startswith("_")}
    res = {"ms": ms, "alg_bytes": alg_bytes, "steps": per, "launches_per_step": launches[0] // steps,
           "k": info["_k"], "status": info["_status"], "sigma": info["_sigma"], "nodes": info["_nodes"],
           "gen_ms": gen_ms[0] / steps, "parent": parent, **_rank_summary(parent, info["_nodes"])}
    if host is not None:
        res["h2d_bytes"] = sum(cols) * wl["n"] * es
        res["d2h_bytes"] = d2h
    del gen
    torch.cuda.empty_cache()
    return res



def run_waves_e2e(H, precision, wl, fro2, steps, warmup, stream, dist_ctx, host):
    """End-to-end leg of the headline: the snapshots come from pinned host memory and
    every upload lies inside a timed interval.  ``host``: two wave buffers of pinned
    host memory.  Wave w is pushed (and processed: max_pending_leaves = the wave)
    while wave w + 1 uploads on a copy stream into the other device wave buffer; an
    interval ends when both are done.  Between intervals (untimed) the device
    generator writes wave w + 2 and it is copied to the host buffer wave w used --
    the stand-in for snapshots that are already in host memory.  The first wave's
    upload is timed on its own; the last interval holds hapod_result and the read
    back of the root's modes and sigma."""
    import torch

    parent, leaves, cols = c3_tree(wl)
    dtype = H.DTYPE[precision]
    device = torch.device("cuda", torch.cuda.current_device())
    W = wl["wave"]
    gen = make_generator(H, wl, dtype, device, 2 * W)
    eps = wl["eps_rel"] * math.sqrt(fro2)
    cstream = torch.cuda.Stream(device)
    waves = list(range(0, len(leaves), W))

    def stage(wi):  # untimed: generate wave wi into device buffers (wi % 2), copy to host buffers (wi % 2)
        w0 = waves[wi]
        views = {}
        with torch.cuda.stream(stream):
            for i in range(w0, min(len(leaves), w0 + W)):
                views[i] = gen.gen(i, (i - w0) + W * (wi % 2), stream)
                host[wi % 2][i - w0][:views[i].shape[0]].copy_(views[i], non_blocking=True)
                views[i].fill_(float("nan"))  # only the upload brings the snapshots back
        stream.synchronize()
        return views

    def upload(wi, views):  # on the copy stream, after `stream`'s work so far; one event per leaf
        w0 = waves[wi]
        cstream.wait_stream(stream)
        evs = []
        with torch.cuda.stream(cstream):
            for i in range(w0, min(len(leaves), w0 + W)):
                views[i].copy_(host[wi % 2][i - w0][:views[i].shape[0]], non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(cstream)
                evs.append(ev)
        return evs

    def step():
        ctx = H.hapod_create(parent, cols, eps, wl["omega"], wl["n"], precision, stream=stream,
                             max_pending_leaves=W, flags=0)
        ms, d2h, st = 0.0, 0, -1
        views = {0: stage(0)}
        if len(waves) > 1:
            views[1] = stage(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        evs = upload(0, views[0])
        for ev in evs:
            stream.wait_event(ev)
        e1.record(stream)
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
        for wi in range(len(waves)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            nxt = upload(wi + 1, views[wi + 1]) if wi + 1 < len(waves) else []
            for i, v in views[wi].items():
                H.hapod_push(ctx, leaves[i], v.t())
            if wi + 1 == len(waves):
                s_, U, st = H.hapod_result(ctx, device=device)
                st = int(st)
                Uh = U.cpu()
                d2h = Uh.numel() * Uh.element_size() + s_.numel() * 8
            for ev in nxt:
                stream.wait_event(ev)
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            del views[wi]
            if wi + 2 < len(waves):
                views[wi + 2] = stage(wi + 2)
        H.hapod_destroy(ctx)
        return ms, d2h, st

    for _ in range(warmup):
        step()
    dist_ctx.barrier()
    tot, d2h, st = 0.0, 0, -1
    for _ in range(steps):
        ms, d2h, st = step()
        tot += ms
    dist_ctx.barrier()
    es = 4 if dtype == torch.float32 else 8
    res = {"ms": dist_ctx.max(tot / steps), "h2d_bytes": sum(cols) * wl["n"] * es, "d2h_bytes": d2h, "status": st}
    del gen
    torch.cuda.empty_cache()
    return res

def _rank_summary(parent, nodes):
    return {"max_inner_k": max([st_["k"] for a, st_ in enumerate(nodes) if st_["level"] > 1 and parent[a] >= 0]
                               or [0]),
            "max_intermediate_k": max([st_["k"] for a, st_ in enumerate(nodes) if parent[a] >= 0] or [0]),
            "leaf_k": max(st_["k"] for st_ in nodes if st_["level"] == 1)}


# ----------------------------------------------------------------- FP64 workload (resident)
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


def tree(kind="binary"):
    from paper_1607_05210_gb300 import synth

    parent = synth.balanced_tree(2, TREE_DEPTH) if kind == "binary" else synth.star_tree(LEAVES)
    leaves = synth.leaves_of(parent)
    cols = [0] * len(parent)
    for a in leaves:
        cols[a] = COLS
    return parent, leaves, cols


def run_form(H, precision, bufs, fro2, steps, warmup, stream, dist_ctx, eps_rel=EPS_REL, shape=None,
             omega=OMEGA, n_rows=N_ROWS):
    """One HAPOD per step over resident leaves: create, push every leaf, result, destroy."""
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
    es = 4 if H.DTYPE[precision] == torch.float32 else 8
    alg_bytes = sum(es * n_rows * (2 * st_["m"] + max(0, st_["k"])) for st_ in info["_nodes"] if st_["m"] > 0)
    per = {k: {f: v[f] / steps for f in v} for k, v in info.items() if not k.startswith("_")}
    return {"ms": ms, "alg_bytes": alg_bytes, "steps": per, "launches_per_step": launches[0] // steps,
            "k": info["_k"], "status": info["_status"], **_rank_summary(parent, info["_nodes"])}


# ----------------------------------------------------------------- roofline
# DRAM traffic of the dominant kernels, from one ncu capture per kernel
# (dram__bytes_read.sum + dram__bytes_write.sum of a single launch, scaled to the
# workload's launch where stated), stored with the SHA-256 of the kernel's source
# file at capture time.  A kernel whose source changed since then reports null.
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")


def kernel_traffic(kernel: str, alg_bytes: float = None):
    """(DRAM bytes, note) of the last capture of `kernel`, or (None, why).  A record
    with the capture's algorithmic bytes gives the traffic of `alg_bytes` algorithmic
    bytes at the captured ratio (the traffic grows in proportion to the units)."""
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
    if alg_bytes is not None and rec.get("alg_bytes_per_launch"):
        return float(rec["bytes_per_launch"]) / float(rec["alg_bytes_per_launch"]) * alg_bytes, rec["note"]
    return float(rec["bytes_per_launch"]), rec["note"]


GRAM_KERNEL = {2: "gram_oz_kernel", 4: "gram_fx3_kernel", 3: "gram_bf3_kernel", 1: "gram_tc_kernel",
               0: "gram_f64_tiles"}


def roofline(res, precision, H, hbm, dom=None):
    """Roofline of the dominant step on the method's algorithmic bytes: the Gram pass
    reads b n m bytes per node (the library's step accounting); achieved = those bytes
    over the step's CUDA-event time."""
    steps = res["steps"]
    if dom is None:
        dom = max((k for k in steps if steps[k]["launches"] > 0), key=lambda k: steps[k]["ms"])
    d = steps[dom]
    if precision == H.HAPOD_FP64 and dom in ("gram", "modes"):
        ach = d["flops"] / (d["ms"] / 1e3) / 1e12
        return dom, {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": ach / FP64_PEAK_TFLOPS, "traffic": None,
                     "kernel": f"{dom} (FP64 FMA pipe; peak = nominal GB300 FP64 rate)"}
    if dom in ("gram", "modes"):
        ach = d["bytes"] / (d["ms"] / 1e3) / 1e9
        kern = GRAM_KERNEL.get(precision, dom) if dom == "gram" else dom
        traffic, note = kernel_traffic(kern, d["bytes"])
        out = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm, "traffic": traffic,
               "traffic_note": note, "kernel": kern,
               "definition": f"achieved = b n m algorithmic bytes per node summed over the {dom} step's nodes, over "
                             "that step's CUDA-event time (launches on the context stream); traffic = DRAM bytes "
                             "of the same step at the ratio of an ncu capture",
               "launches_per_step": d["launches"], "bytes_per_step": d["bytes"], "ms_per_step": d["ms"]}
        if precision == H.HAPOD_FP64_OZAKI and dom == "gram":
            out["digit_tflops"] = 28.0 * d["flops"] / (d["ms"] / 1e3) / 1e12
        return dom, out
    return dom, {"bound": "alu", "achieved": None, "peak": None, "unit": None, "frac": None, "traffic": None,
                 "kernel": dom}


def summarise(r, precision, H, eps_rel, total_cols, hbm, peak_src, world, dom=None):
    d, roof = roofline(r, precision, H, hbm, dom)
    roof["peak_source"] = peak_src if roof["bound"] in ("hbm", "tensor") else "nominal"
    out = {"eps_rel": eps_rel, "value": total_cols / (r["ms"] / 1e3), "unit": UNIT, "ms_per_step": r["ms"],
           "gb_per_s": r["alg_bytes"] / (r["ms"] / 1e3) / 1e9 * world,
           "hbm_frac": r["alg_bytes"] / (r["ms"] / 1e3) / 1e9 / hbm,
           "k_root": r["k"], "max_leaf_k": r["leaf_k"], "max_inner_k": r["max_inner_k"], "status": r["status"],
           "launches_per_step": r["launches_per_step"],
           "step_ms": {k: v["ms"] for k, v in r["steps"].items()}, "roofline": roof}
    if "gen_ms" in r:
        out["generation_ms_per_step"] = r["gen_ms"]
    return out


# ----------------------------------------------------------------- autotuner
def run_autotune(H, device):
    """hapod_autotune for the fixed-point Gram on the node widths of the headline and
    streamed workloads (untimed): a generated leaf and a generated matrix as wide as
    their inner nodes, each in its (m, n) bucket."""
    import torch

    out = {}
    for wl, m, what in ((C3, C3["cols"], "leaves"), (C3, 384, "inner nodes (257..512 columns)"),
                        (C5, C5["cols"], "leaves"), (C5, 192, "inner nodes (129..256 columns)")):
        X = H.colmajor_empty(wl["n"], m, torch.float32, device)
        H.hapod_synth_snapshots(c3_params(H, wl), wl["n"], 0, m, X)
        pct, ms = H.hapod_autotune(X, H.HAPOD_MIXED_FX3)
        out[f"{wl['name']} {what}: n=2^{wl['n'].bit_length() - 1}, m={m}"] = {
            "split_factor_pct": pct, "ms_at_50_100_200_400_pct": [round(v, 3) for v in ms]}
        del X
    torch.cuda.empty_cache()
    return out


# ----------------------------------------------------------------- oracle (CPU baseline)
ORACLE_ROWS = (4096, 8192)


def time_oracle(reps: int = 1):
    """Whole-tree oracle time of the headline workload, extrapolated: the oracle POD of
    leaf 0 (128 columns) and of its level-2 parent (the four leaves' outputs) at two
    reduced row counts, fitted as a + b n per node kind and summed over the tree's
    256 leaves and 85 inner nodes at n = 2^22."""
    import numpy as np

    import oracle
    from paper_1607_05210_gb300 import synth

    parent, leaves, cols = c3_tree()
    S = sum(cols)
    P = synth.pulse_workload(C3["seed"])
    kids0 = [a for a in range(len(parent)) if parent[a] == parent[leaves[0]]]
    t_leaf, t_inner, wall = [], [], 0.0
    for n in ORACLE_ROWS:
        data = {a: synth.pulse_snapshots(n, leaves.index(a) * C3["cols"], C3["cols"], P, np.float32).astype(np.float64)
                for a in kids0}
        fro2_est = sum(float(np.sum(x * x)) for x in data.values()) * (C3["leaves"] / len(kids0))
        eps_nodes = oracle.tolerances(parent, cols, C3["eps_rel"] * math.sqrt(fro2_est) / math.sqrt(S), C3["omega"])
        tl, ti = [], []
        for _ in range(reps):
            outs = []
            t0 = time.perf_counter()
            for a in kids0:
                outs.append(oracle.pod(data[a], eps_nodes[a]).Y)
            t1 = time.perf_counter()
            oracle.pod(np.asfortranarray(np.concatenate(outs, axis=1)), eps_nodes[parent[kids0[0]]])
            t2 = time.perf_counter()
            tl.append((t1 - t0) / len(kids0))
            ti.append(t2 - t1)
            wall += t2 - t0
        t_leaf.append(min(tl))
        t_inner.append(min(ti))
    n0, n1 = ORACLE_ROWS
    N = C3["n"]

    def extrap(t):
        b = max(0.0, (t[1] - t[0]) / (n1 - n0))
        return t[1] + b * (N - n1)

    inner = sum(1 for a in range(len(parent)) if cols[a] == 0)
    total = len(leaves) * extrap(t_leaf) + inner * extrap(t_inner)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = (f"oracle POD of leaf 0 and of its level-2 parent at n = {n0} and {n1} rows ({wall:.1f} s of CPU time "
              f"over {reps} repetition(s)); per node kind time fitted as a + b n and summed over {len(leaves)} "
              f"leaves + {inner} inner nodes at n = 2^22: {total:.0f} s per HAPOD")
    return S / total, total, wall, cores, sample


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


# ----------------------------------------------------------------- sweeps (Sec. 4.2, 4.3)
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
            print(json.dumps({"sweep": "omega", "omega": w, "workload": C2_WORKLOAD.replace("omega=0.5", f"omega={w}"),
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


# ----------------------------------------------------------------- profiling cases
def profile_case(args, H, device):
    """Small cases for ncu captures: three Gram calls (and X V where named) on one leaf."""
    import torch

    from paper_1607_05210_gb300 import synth

    form = args.profile_form
    if form in ("fx3-node", "oz-node"):
        return profile_node(H, device, H.HAPOD_MIXED_FX3 if form == "fx3-node" else H.HAPOD_FP64_OZAKI)
    if form in ("fx3", "bf3"):
        prec = H.HAPOD_MIXED_FX3 if form == "fx3" else H.HAPOD_MIXED_BF16X3
        X = H.colmajor_empty(C3["n"], C3["cols"], torch.float32, device)
        H.hapod_synth_snapshots(c3_params(H), C3["n"], 0, C3["cols"], X)
        V = torch.randn((90, C3["cols"]), dtype=torch.float64, device=device).t() / 16.0
        for _ in range(3):
            G = H.hapod_gram(X, prec)
            Y = H.hapod_modes(X, V, 90, None, prec)
        torch.cuda.synchronize()
        return {"G00": float(G[0, 0]), "Y00": float(Y[0, 0])}
    if form in ("fp64", "mixed"):
        cols, dtype, prec = ((64, torch.float64, H.HAPOD_FP64) if form == "fp64"
                             else (COLS, torch.float32, H.HAPOD_MIXED_TF32X3))
        X = synth.advection_diffusion_device(N_ROWS, cols, SEED, dtype, device).t()
        for _ in range(3):
            G = H.hapod_gram(X, prec)
        torch.cuda.synchronize()
        return {"G00": float(G[0, 0])}
    torch.manual_seed(SEED)
    X = torch.randn((COLS, N_ROWS), dtype=torch.float64, device=device).t()
    V = torch.randn((19, COLS), dtype=torch.float64, device=device).t() / 16.0
    for _ in range(2):
        G = H.hapod_gram(X, H.HAPOD_FP64_OZAKI)
        Y = H.hapod_modes(X, V, 19, None, H.HAPOD_FP64_OZAKI)
    torch.cuda.synchronize()
    return {"G00": float(G[0, 0]), "Y00": float(Y[0, 0])}


def profile_node(H, device, precision):
    """One level-2 node of the headline workload and its four leaves: the leaves' PODs
    (generated on the device, leaf tolerance of the tree) and the POD of the node on
    their concatenated outputs, each step timed with CUDA events (2 repetitions)."""
    import torch

    wl = C3
    parent, leaves, cols = c3_tree(wl)
    dtype = H.DTYPE[precision]
    params = c3_params(H, wl)
    Xs = []
    for i in range(4):
        X = H.colmajor_empty(wl["n"], wl["cols"], dtype, device)
        H.hapod_synth_snapshots(params, wl["n"], i * wl["cols"], wl["cols"], X)
        Xs.append(X)
    fro2_cols = sum(float(torch.linalg.vector_norm(X, dtype=torch.float64) ** 2) for X in Xs) / (4 * wl["cols"])
    eps_star = wl["eps_rel"] * math.sqrt(fro2_cols)
    eps_leaf = math.sqrt(wl["cols"] / (wl["depth"]) * (1 - wl["omega"] ** 2)) * eps_star
    eps_l2 = math.sqrt(4 * wl["cols"] / (wl["depth"]) * (1 - wl["omega"] ** 2)) * eps_star
    out = {}

    def timed(name, f):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = f()
        e1.record()
        torch.cuda.synchronize()
        out.setdefault(name, []).append(round(e0.elapsed_time(e1), 3))
        return r

    for rep in range(2):
        Ys = []
        for i, X in enumerate(Xs):
            timed("leaf_gram", lambda: H.hapod_gram(X, precision))
            N, s, Y, tail, st = timed("leaf_pod", lambda: H.hapod_pod(X, eps_leaf, precision))
            Ys.append(Y)
        Xin = H.colmajor_empty(wl["n"], sum(Y.shape[1] for Y in Ys), dtype, device)
        off = 0
        for Y in Ys:
            Xin[:, off:off + Y.shape[1]].copy_(Y)
            off += Y.shape[1]
        G = timed("node_gram", lambda: H.hapod_gram(Xin, precision))
        lam, V, sw, st = timed("node_eig", lambda: H.hapod_eig(G, precision))
        N, tail = H.hapod_truncate(lam, eps_l2)
        timed("node_modes", lambda: H.hapod_modes(Xin, V, N, None, precision))
        Nn, s, Y, tail, st = timed("node_pod", lambda: H.hapod_pod(Xin, eps_l2, precision))
        out["node_m"] = Xin.shape[1]
        out["node_k"] = Nn
        out["node_sweeps"] = sw
        out["leaf_k"] = [Y.shape[1] for Y in Ys]
        del Xin, Ys
    return out


# ----------------------------------------------------------------- main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workloads", default="c4,c5,c2",
                    help="comma list of extra workloads beside the headline: 'c4' (1000 uneven prescribed-spectrum "
                         "leaves, device-generated; 'c4-fp64' adds its digit-slice FP64 form), 'c5' (streamed "
                         "incremental chain, "
                         "device-generated chunks), 'c2' (FP64 advection-diffusion, binary tree and star, "
                         "resident), 'none'")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64-form", action="store_true", help="skip the digit-slice FP64 form of the headline")
    ap.add_argument("--profile-leaf", action="store_true",
                    help="run the small per-leaf case named by --profile-form and exit (for ncu captures)")
    ap.add_argument("--profile-form", choices=["oz", "fp64", "mixed", "fx3", "bf3", "fx3-node", "oz-node"],
                    default="fx3",
                    help="with --profile-leaf: 'fx3'/'bf3' three Gram + X V calls on one 2^22 x 128 FP32 leaf of "
                         "the headline workload; 'oz' two digit-slice Gram + X V calls on a 2^20 x 256 FP64 leaf; "
                         "'fp64' three FP64 Gram calls on 2^20 x 64; 'mixed' three TF32 Gram calls on 2^20 x 256; "
                         "'fx3-node' / 'oz-node' the PODs of four headline leaves and of their level-2 parent, "
                         "each step timed")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the Gram planners' own split counts")
    ap.add_argument("--sweep", choices=["omega", "trees"],
                    help="print one JSON line per configuration and exit: 'omega' runs the FP64 workload for "
                         "omega in 0.1 .. 0.999 (Sec. 4.3); 'trees' runs 10^4 advection-diffusion columns in "
                         "10 x 1000 .. 1000 x 10 blocks on balanced trees of edge depth 2..5 (Sec. 4.2)")
    args = ap.parse_args()
    os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1))
    dist_ctx = Dist()

    if args.impl == "reference":
        if dist_ctx.rank != 0:
            dist_ctx.close()
            return
        vals = []
        for _ in range(args.warmup):
            time_oracle()
        sample = cores = None
        for _ in range(args.steps):
            v, total, wall, cores, sample = time_oracle()
            vals.append(v)
        value = statistics.median(vals)
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": C3["leaves"] * C3["cols"] / value * 1e3,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic", "config": {"workload": C3_WORKLOAD, "form": "cpu oracle"},
                          "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                                           "sample": sample},
                          "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        dist_ctx.close()
        return

    import torch

    torch.cuda.set_device(dist_ctx.local)
    device = torch.device("cuda", dist_ctx.local)
    from paper_1607_05210_gb300 import hapod as H

    if args.profile_leaf:
        print(json.dumps({"profile_leaf": True, "form": args.profile_form, **profile_case(args, H, device)}))
        dist_ctx.close()
        return
    if args.sweep:
        if dist_ctx.rank == 0:
            run_sweep(args.sweep, H, device, dist_ctx)
        dist_ctx.close()
        return

    hbm, _, peak_src = _peaks()
    stream = torch.cuda.Stream(device)
    world = dist_ctx.world
    total_c3 = C3["leaves"] * C3["cols"] * world
    forms = {}

    # pinned host buffers for two waves (end-to-end leg), before device work; every
    # rank runs the leg only if every rank got its buffers (the leg has barriers)
    host = None
    if not args.no_e2e:
        need = 2 * C3["wave"] * C3["cols"] * C3["n"] * 4 * dist_ctx.world
        try:
            phys = os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES")
        except (ValueError, OSError, AttributeError):
            phys = 0
        if dist_ctx.world > 1 and phys and need > phys // 2:
            host = (f"skipped: {dist_ctx.world} rank(s) x {need // dist_ctx.world >> 30} GiB of pinned host memory "
                    f"exceed half of the host's {phys >> 30} GiB")
        else:
            try:
                host = [[torch.empty((C3["cols"], C3["n"]), dtype=torch.float32, pin_memory=True)
                         for _ in range(C3["wave"])] for _ in range(2)]
            except (RuntimeError, MemoryError) as ex:
                host = str(ex)[:120]
        if dist_ctx.max(0.0 if isinstance(host, list) else 1.0) > 0.0 and isinstance(host, list):
            host = "pinned host buffers unavailable on another rank"

    fro2 = c3_fro2(H, C3, device, stream)
    autotune = {} if args.no_autotune else run_autotune(H, device)
    sampler = ClockSampler(dist_ctx.local)
    head = run_waves(H, H.HAPOD_MIXED_FX3, C3, fro2, args.steps, args.warmup, stream, dist_ctx)
    clocks = sampler.stop()
    head_key = f"mixed_fx3@{C3['eps_rel']:g}"
    forms[head_key] = summarise(head, H.HAPOD_MIXED_FX3, H, C3["eps_rel"], total_c3, hbm, peak_src, world, "gram")
    e2e = None
    if not args.no_e2e:
        if isinstance(host, list):
            r = run_waves_e2e(H, H.HAPOD_MIXED_FX3, C3, fro2, args.steps, 1, stream, dist_ctx, host)
            e2e = {"value": total_c3 / (r["ms"] / 1e3), "unit": UNIT, "h2d_bytes_per_step": r["h2d_bytes"],
                   "d2h_bytes_per_step": r["d2h_bytes"], "ms_per_step": r["ms"], "form": head_key,
                   "steps": args.steps, "status": r["status"],
                   "note": "snapshots from pinned host memory (device wave buffers NaN-filled after their copy "
                           "to the host, so only the uploads restore them), two wave buffers: wave w + 1 (16 leaves, "
                           "32 GiB) uploads on a copy stream while wave w "
                           "is pushed and processed, each interval ending when both are done; the first upload "
                           "timed alone; generating the next wave on the device and copying it to the host between "
                           "intervals is untimed; the root's modes and sigma read back"}
        else:
            e2e = {"value": None, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0,
                   "note": f"pinned host buffers unavailable: {host}"}
        host = None
    if not args.no_fp64_form:
        r64 = run_waves(H, H.HAPOD_FP64_OZAKI, C3, fro2, args.steps, 1, stream, dist_ctx)
        k64 = f"fp64_ozaki@{C3['eps_rel']:g}"
        forms[k64] = summarise(r64, H.HAPOD_FP64_OZAKI, H, C3["eps_rel"], total_c3, hbm, peak_src, world, "gram")
        forms[head_key]["speedup_vs_fp64_form_same_eps"] = r64["ms"] / head["ms"]
        s1, s2 = head["sigma"], r64["sigma"]
        k = min(len(s1), len(s2))
        forms[head_key]["vs_fp64_form"] = {
            "k_root": [len(s1), len(s2)],
            "max_rel_sigma_diff_above_1e-5": max([abs(s1[j] - s2[j]) / s2[j] for j in range(k)
                                                  if s2[j] >= 1e-5 * s2[0]] or [0.0])}

    workloads = {}
    if "c4" in args.workloads:
        fro2_c4 = c3_fro2(H, C4, device, stream)
        total_c4 = int(sum(c3_tree(C4)[2])) * world
        st4 = max(1, min(args.steps, 2))
        r4 = run_waves(H, H.HAPOD_MIXED_FX3, C4, fro2_c4, st4, 1, stream, dist_ctx)
        k1 = f"c4/mixed_fx3@{C4['eps_rel']:g}"
        workloads[k1] = summarise(r4, H.HAPOD_MIXED_FX3, H, C4["eps_rel"], total_c4, hbm, peak_src, world, "gram")
        if "c4-fp64" in args.workloads:
            r4b = run_waves(H, H.HAPOD_FP64_OZAKI, C4, fro2_c4, st4, 1, stream, dist_ctx)
            workloads[f"c4/fp64_ozaki@{C4['eps_rel']:g}"] = summarise(r4b, H.HAPOD_FP64_OZAKI, H, C4["eps_rel"],
                                                                     total_c4, hbm, peak_src, world, "gram")
            workloads[k1]["speedup_vs_fp64_form_same_eps"] = r4b["ms"] / r4["ms"]
        workloads["c4_workload"] = C4_WORKLOAD
    if "c5" in args.workloads:
        fro2_c5 = c3_fro2(H, C5, device, stream)
        total_c5 = C5["leaves"] * C5["cols"] * world
        st5 = max(1, min(args.steps, 2))
        r5 = run_waves(H, H.HAPOD_MIXED_FX3, C5, fro2_c5, st5, 1, stream, dist_ctx)
        r5b = run_waves(H, H.HAPOD_FP64_OZAKI, C5, fro2_c5, st5, 1, stream, dist_ctx)
        k1 = f"c5/mixed_fx3@{C5['eps_rel']:g}"
        workloads[k1] = summarise(r5, H.HAPOD_MIXED_FX3, H, C5["eps_rel"], total_c5, hbm, peak_src, world, "gram")
        workloads[f"c5/fp64_ozaki@{C5['eps_rel']:g}"] = summarise(r5b, H.HAPOD_FP64_OZAKI, H, C5["eps_rel"], total_c5,
                                                                 hbm, peak_src, world, "gram")
        workloads[k1]["speedup_vs_fp64_form_same_eps"] = r5b["ms"] / r5["ms"]
        workloads["c5_workload"] = C5_WORKLOAD
    if "c2" in args.workloads:
        bufs, fro2_c2 = make_inputs(torch.float64, device)
        total_c2 = LEAVES * COLS * world
        for kind in ("binary", "star"):
            shape = tree(kind)
            r = run_form(H, H.HAPOD_FP64_OZAKI, bufs, fro2_c2, max(1, min(args.steps, 3)), 1, stream, dist_ctx,
                         EPS_REL, shape=shape)
            workloads[f"c2_{kind}/fp64_ozaki@{EPS_REL:g}"] = summarise(r, H.HAPOD_FP64_OZAKI, H, EPS_REL, total_c2,
                                                                      hbm, peak_src, world)
        r = run_form(H, H.HAPOD_FP64, bufs, fro2_c2, 1, 1, stream, dist_ctx, EPS_REL, shape=tree("binary"))
        workloads[f"c2_binary/fp64@{EPS_REL:g}"] = summarise(r, H.HAPOD_FP64, H, EPS_REL, total_c2, hbm, peak_src,
                                                            world)
        workloads["c2_workload"] = C2_WORKLOAD + "; binary = balanced binary tree L_T=7, star = two-level (L_T=2)"
        del bufs
        torch.cuda.empty_cache()

    hs = forms[head_key]
    line = {
        "metric": METRIC, "value": hs["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": C3_WORKLOAD, "form": "mixed_fx3", "parallelism": f"replicas x{world}",
                   "l2": "every leaf (2 GiB) larger than L2; no flush needed",
                   "timed": "sum over waves of the push-to-processed interval (generation between waves untimed, "
                            "reported as generation_ms_per_step)", "seed": C3["seed"]},
        "gb_per_s": hs["gb_per_s"],
        "roofline": hs["roofline"],
        "gpu_launches": head["launches_per_step"] * args.steps,
        "clocks": clocks,
        "e2e": e2e,
        "result": {"k_root": head["k"], "max_leaf_k": head["leaf_k"], "max_inner_k": head["max_inner_k"],
                   "status": head["status"]},
        "step_ms": hs["step_ms"],
        "forms": forms,
        "workloads": workloads,
        "autotune": autotune,
    }
    if dist_ctx.rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, total, wall, cores, sample = time_oracle()
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}
    if dist_ctx.rank == 0:
        print(json.dumps(line))
    dist_ctx.close()


if __name__ == "__main__":
    main()
