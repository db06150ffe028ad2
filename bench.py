"""Benchmark: edge-based median-dual nabla operators on O1280 x 137 levels.

One step = the whole operator path on one synthetic batch: gradient of a
scalar, divergence and curl of a wind, and the Laplacian of the scalar
(gradient pass + divergence pass), FP32 storage and arithmetic with
compensated accumulation, FP64 geometry.  Throughput is node-levels per
second summed over the four operators.  Inputs (3.7 GB scalar, 7.4 GB wind)
are far larger than the 126 MB L2, so no L2 flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample (a few levels of the same grid) with the same metric.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

OPS = ("grad", "div", "curl", "lap")
# one step: grad(f) -> g; lap(f) = div(g), the divergence of the step's own
# gradient (as nb_nabla_gradlap computes it); div and curl of uv in one pass
PARTS = ("grad", "lap_from_grad", "divcurl")
# Nominal dense FP64 rate of a B300 (TFLOP/s), reported beside the measured
# rate of the FMA-chain probe that the FP64 path's roofline uses.
FP64_PEAK_TFLOPS = 1.25
METRIC = "Gnode-levels/s per nabla op (O1280x137, fp32 vs fp64), % HBM roofline; p99 ms"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--grid", type=int, default=1280)
    p.add_argument("--nlev", type=int, default=137)
    p.add_argument("--lmax", type=int, default=40)
    p.add_argument("--e2e-steps", type=int, default=4)
    p.add_argument("--fp64-steps", type=int, default=3)
    p.add_argument("--cpu-levels", type=int, default=32,
                   help="levels of the oracle's bounded CPU sample (also the levels of the error figures)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--single-op-reps", type=int, default=3,
                   help="timed single-operator div, curl and Laplacian calls after the timed region (0 = none)")
    p.add_argument("--variant", type=int, default=0, help="kernel variant (0 auto, 1 direct, 2 tiled)")
    p.add_argument("--tile", type=int, default=0)
    p.add_argument("--batch-fields", type=int, default=64, help="0 skips the batched section")
    p.add_argument("--serve-seconds", type=float, default=2.0, help="0 skips the serving section")
    p.add_argument("--serve-rate", type=float, default=2000.0)
    p.add_argument("--no-serve-baseline", action="store_true", help="skip the sequential FP64 serving baseline")
    p.add_argument("--serve-streams", type=int, default=8)
    p.add_argument("--serve-inflight", type=int, default=32)
    p.add_argument("--lap-route", default="two_pass", choices=["two_pass", "fused"],
                   help="Laplacian of the step: two passes (default) or the single-pass kernel")
    p.add_argument("--stages", type=int, default=0)
    p.add_argument("--stage-kb", type=int, default=0)
    return p.parse_args()


# ------------------------------------------------------------------ helpers

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max(x: float, world: int, device=None) -> float:
    """Maximum of x over all ranks (identity for one rank).  Works with the
    gloo (CPU tensors) and nccl (device tensors) backends."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for ln in open(self.path):
                c = [x.strip() for x in ln.split(",")]
                if len(c) < 9:
                    continue
                try:
                    sm.append(float(c[1]))
                    mx.append(float(c[2]))
                except ValueError:
                    continue
                for n, v in zip(names, c[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
            os.remove(self.path)
        except Exception:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_traffic(op, V, L):
    """DRAM bytes of one launch of `op` from the ncu capture recorded in
    profiles/dram_traffic.json (per node-level, scaled to V x L), or None when
    the staged kernels' sources have changed since that capture."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as fh:
            d = json.load(fh)
        blob = b"".join(open(os.path.join(ROOT, f), "rb").read() for f in d["kernel_sources"])
        if hashlib.sha256(blob).hexdigest() != d["kernel_sources_sha256"]:
            return None
        return int(d["dram_bytes_per_node_level"][op] * V * L)
    except Exception:
        return None


def algorithmic_bytes(op, V, E, L, elem):
    """Bytes a launch must move at minimum: each input value read once, each
    output written once, the connectivity and weights read once per node."""
    P = 2 * E
    if op == "grad":
        return V * L * elem * (1 + 2) + (V + 1) * 4 + P * (4 + 2 * elem)
    if op == "divcurl":  # one wind in, two scalars out, both weight sets
        return V * L * elem * (2 + 2) + (V + 1) * 4 + P * (4 + 4 * elem) + V * 4 * elem
    if op == "gradlap_fused":  # f in, g and lap out; gradient and divergence weights
        return V * L * elem * (1 + 2 + 1) + (V + 1) * 4 + 2 * P * (4 + 2 * elem) + V * 2 * elem
    # div / curl: vector in, scalar out, plus per-node self weights
    return V * L * elem * (2 + 1) + (V + 1) * 4 + P * (4 + 2 * elem) + V * 2 * elem


# ------------------------------------------------------------- our arm

def make_inputs(nabla, synth, grid, mesh, method, nlev, lmax, dtype, device):
    import torch
    ll = torch.as_tensor(grid.lonlat(), device=device)
    perm = torch.as_tensor(mesh.permutation().astype("int64"), device=device)
    lat, lon = ll[perm, 1].contiguous(), ll[perm, 0].contiguous()
    fs = nabla.NodeColumns(method, nlev, dtype)
    f = fs.create_field(device=device)
    uv = fs.create_field(nvar=2, device=device)
    basis = synth.scalar_basis(lat, lon, lmax, synth.BASE_SEED, device=device)
    w = torch.as_tensor(synth.level_weights(nlev, synth.BASE_SEED + 1), device=device)
    wb = synth.wind_basis(lat, lon, lmax, synth.BASE_SEED, method.radius, device=device)
    ww = torch.as_tensor(synth.level_weights(nlev, synth.BASE_SEED + 2), device=device)
    for k0 in range(0, nlev, 16):
        k1 = min(nlev, k0 + 16)
        f[:, k0:k1].copy_(basis @ w[k0:k1].T)
        uv[:, k0:k1].copy_(torch.einsum("vbc,kb->vkc", wb, ww[k0:k1]))
    del basis, wb
    return fs, f, uv


def run_step(nabla, method, f, uv, outs, scratch, stream, ev=None, fused=False):
    """One step of the hot path: g = grad(f); lap(f) = div(g), the Laplacian's
    second pass on the gradient just computed (the two launches of
    nb_nabla_gradlap, issued separately so that each is timed); div(uv) and
    curl(uv) in one fused pass.  ev[0..3] bracket the three launches.  With
    fused, g and lap(f) come from one single-pass nb_nabla_gradlap launch
    (the method's Laplacian route set to NB_LAP_FUSED) and ev[0..2] bracket
    the two launches."""
    g, d, z, l = outs

    def rec(i):
        if ev is not None:
            ev[i].record(stream)
    rec(0)
    if fused:
        nabla.gradlap(method, f, g, l, stream=stream)
        rec(1)
    else:
        nabla.apply(method, "grad", f, g, stream=stream)
        rec(1)
        nabla.apply(method, "div", g, l, stream=stream)
        rec(2)
    nabla.divcurl(method, uv, d, z, stream=stream)
    rec(2 if fused else 3)


def bench_ours(a):
    import torch
    import torch.distributed as dist
    from paper_1908_06091_b300 import nabla, synth

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    device = f"cuda:{local}"
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device(device))

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    t0 = time.time()
    grid = nabla.Grid(a.grid)
    mesh = nabla.Mesh(grid, 1)
    method = nabla.Method(mesh)
    method.set_kernel(a.variant, a.tile)
    if a.stages:
        method.set_staging(a.stages, a.stage_kb)
    fused = a.lap_route == "fused"
    method.set_laplacian_route(nabla.LAP_FUSED if fused else nabla.LAP_TWO_PASS)
    parts = ("gradlap", "divcurl") if fused else PARTS
    setup_s = time.time() - t0
    V, E, L = mesh.V, mesh.E, a.nlev
    fs, f, uv = make_inputs(nabla, synth, grid, mesh, method, L, a.lmax, torch.float32, device)
    outs = (fs.create_field(nvar=2, device=device), fs.create_field(device=device),
            fs.create_field(device=device), fs.create_field(device=device))
    scratch = fs.create_field(nvar=2, device=device)
    stream = torch.cuda.Stream(device=device)
    with torch.cuda.stream(stream):
        for _ in range(max(a.warmup, 3)):
            run_step(nabla, method, f, uv, outs, scratch, stream, fused=fused)
    stream.synchronize()

    # timed region: K steps, per-op CUDA events on the launching stream
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(a.steps)]
    launches0 = nabla.launch_count()
    barrier()
    with Clocks(local) as clk:
        start = torch.cuda.Event(enable_timing=True)
        stop = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        with torch.cuda.stream(stream):
            for k in range(a.steps):
                run_step(nabla, method, f, uv, outs, scratch, stream, evs[k], fused=fused)
        stop.record(stream)
        stream.synchronize()
    barrier()
    launches = nabla.launch_count() - launches0
    ms_total = reduce_max(start.elapsed_time(stop), world, device)
    ms_step = ms_total / a.steps
    per_op_ms = {op: statistics.median(evs[k][i].elapsed_time(evs[k][i + 1]) for k in range(a.steps))
                 for i, op in enumerate(parts)}
    nl = V * L
    value = world * 4 * nl * a.steps / (ms_total * 1e-3) / 1e9
    hbm, peak_kind = peaks()
    elem = 4
    # kernels of a step, one launch each: gradient, divergence (the
    # Laplacian's second pass), fused div+curl
    kern = {"grad": "grad", "lap_from_grad": "div", "divcurl": "divcurl", "gradlap": "gradlap_fused"}
    kern_ms = {kern[p]: per_op_ms[p] for p in parts}
    dom = max(kern_ms, key=kern_ms.get)
    algo = algorithmic_bytes(dom, V, E, L, elem)
    achieved = algo / (kern_ms[dom] * 1e-3) / 1e9
    per_op = {}
    for op in parts:
        b = algorithmic_bytes(kern[op], V, E, L, elem)
        per_op[op] = {"ms": round(per_op_ms[op], 4),
                      "gnl_s": round((2 if op in ("divcurl", "gradlap") else 1) * nl / per_op_ms[op] / 1e6, 1),
                      "algo_GBs": round(b / per_op_ms[op] / 1e6, 1),
                      "frac_hbm": round(b / per_op_ms[op] / 1e6 / hbm, 3)}
    # a level sample of this run's own inputs and outputs (grid order, host),
    # for the oracle comparison of the CPU-baseline leg
    sample = None
    if rank == 0 and not a.no_cpu_baseline:
        sample = take_sample(mesh, f, uv, outs, a.cpu_levels)
    # the single-operator passes, outside the timed region (for reference)
    single = {}
    with torch.cuda.stream(stream):
        singles = (("div", uv, outs[1]), ("curl", uv, outs[2]), ("lap", f, outs[3]))
        for op, xin, o in singles if a.single_op_reps > 0 else ():
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            sc = scratch if op == "lap" else None
            nabla.apply(method, op, xin, o, scratch=sc, stream=stream)
            e0.record(stream)
            for _ in range(a.single_op_reps):
                nabla.apply(method, op, xin, o, scratch=sc, stream=stream)
            e1.record(stream)
            stream.synchronize()
            single[op] = round(e0.elapsed_time(e1) / a.single_op_reps, 4)
        # the single-pass Laplacian (NB_LAP_FUSED), bit-identical to the
        # two-pass route timed above
        if a.single_op_reps > 0:
            method.set_laplacian_route(nabla.LAP_FUSED)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            nabla.apply(method, "lap", f, outs[3], stream=stream)
            e0.record(stream)
            for _ in range(a.single_op_reps):
                nabla.apply(method, "lap", f, outs[3], stream=stream)
            e1.record(stream)
            stream.synchronize()
            method.set_laplacian_route(nabla.LAP_TWO_PASS)
            single["lap_fused_single_pass"] = round(e0.elapsed_time(e1) / a.single_op_reps, 4)
    # the edge-based baseline (per-edge differences, then a node reduction)
    edge_ms = {}
    if a.single_op_reps > 0:
        method.set_kernel(nabla.KERNEL_EDGE, 0)
        with torch.cuda.stream(stream):
            for op, xin, o in (("grad", f, outs[0]), ("div", uv, outs[1])):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                nabla.apply(method, op, xin, o, stream=stream)
                e0.record(stream)
                for _ in range(a.single_op_reps):
                    nabla.apply(method, op, xin, o, stream=stream)
                e1.record(stream)
                stream.synchronize()
                edge_ms[op] = round(e0.elapsed_time(e1) / a.single_op_reps, 4)
        method.set_kernel(a.variant, a.tile)
        torch.cuda.empty_cache()

    # FP64 GPU path on the same workload (the plain reference GPU path)
    fp64 = None
    if a.fp64_steps > 0:
        fs64 = nabla.NodeColumns(method, L, torch.float64)
        f64 = fs64.create_field(device=device)
        uv64 = fs64.create_field(nvar=2, device=device)
        f64.copy_(f)
        uv64.copy_(uv)
        outs64 = (fs64.create_field(nvar=2, device=device), fs64.create_field(device=device),
                  fs64.create_field(device=device), fs64.create_field(device=device))
        scr64 = fs64.create_field(nvar=2, device=device)
        with torch.cuda.stream(stream):
            run_step(nabla, method, f64, uv64, outs64, scr64, stream)
            ev64 = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(a.fp64_steps)]
            for k in range(a.fp64_steps):
                run_step(nabla, method, f64, uv64, outs64, scr64, stream, ev64[k])
        stream.synchronize()
        ms64 = {op: statistics.median(ev64[k][i].elapsed_time(ev64[k][i + 1]) for k in range(a.fp64_steps))
                for i, op in enumerate(PARTS)}
        # The FP64 path is bound by B300's FP64 ALUs, not by HBM.  FP64
        # flops per node-level of a six-neighbour node, as the direct kernels
        # issue them: grad 6 x (1 sub + 2 fma) = 30; div (and curl) 6 x
        # (2 sub + 2 fma) + 2 fma of the self term = 40; div+curl = 80.
        flops = {"grad": 30, "lap_from_grad": 40, "divcurl": 80}
        dom64 = max(ms64, key=ms64.get)
        tf = flops[dom64] * nl / (ms64[dom64] * 1e-3) / 1e12
        # the FP64 units' rate on this GPU, measured by an FMA-chain probe
        # (median of three launches)
        probes = [nabla.probe_fp64_rate(40000, stream=stream) for _ in range(3)]
        fp64_peak = statistics.median(p[0] for p in probes)
        fp64 = {"ms_per_step": round(sum(ms64.values()), 3),
                "value": round(4 * nl / (sum(ms64.values()) * 1e-3) / 1e9, 2),
                "per_op": {op: {"ms": round(ms64[op], 3),
                                "gnl_s": round((2 if op == "divcurl" else 1) * nl / ms64[op] / 1e6, 1),
                                "tflops": round(flops[op] * nl / (ms64[op] * 1e-3) / 1e12, 3)}
                           for op in PARTS},
                "roofline": {"bound": "alu", "kernel": dom64, "achieved": round(tf, 3),
                             "peak": round(fp64_peak, 4), "unit": "TFLOP/s",
                             "frac": round(tf / fp64_peak, 3),
                             "peak_kind": "measured: FP64 FMA-chain probe on this GPU (nb_probe_fp64_rate, "
                                          "median of 3)",
                             "nominal_peak": FP64_PEAK_TFLOPS,
                             "flops_per_node_level": flops[dom64]}}
        if sample is not None:
            sample["out64"] = sample_outputs(mesh, outs64, sample["levels"])
        del f64, uv64, outs64, scr64
        torch.cuda.empty_cache()

    # end to end through the C ABI with host buffers (copies inside the timed region)
    e2e = None
    if a.e2e_steps > 0:
        # end to end through the C ABI: each step uploads its inputs (f once,
        # uv once) from pinned host memory, runs gradlap and divcurl, and
        # downloads all four results.  Uploads, operators and downloads sit
        # on three streams ordered by events, and device buffers alternate
        # between two sets, so step k+1's uploads overlap step k's downloads
        # and both copy directions stay busy.
        hf = f._base.cpu().pin_memory()
        huv = uv._base.cpu().pin_memory()
        hout = [torch.empty_like(o._base, device="cpu").pin_memory() for o in outs]
        nvars = (2, 1, 1, 1)
        h2d = sum(t.numel() * t.element_size() for t in (hf, huv))
        d2h = sum(t.numel() * t.element_size() for t in hout)
        s_up = torch.cuda.Stream(device=device)
        s_down = torch.cuda.Stream(device=device)
        sets = [(f, uv, outs)]
        f2, uv2 = fs.create_field(device=device), fs.create_field(nvar=2, device=device)  # filled by uploads
        sets.append((f2, uv2, (fs.create_field(nvar=2, device=device), fs.create_field(device=device),
                               fs.create_field(device=device), fs.create_field(device=device))))
        done = [None, None]  # per set: event after its downloads

        def e2e_step(k):
            fk, uvk, (g, d, z, l) = sets[k % 2]
            if done[k % 2] is not None:  # the set's previous downloads have read its outputs
                s_up.wait_event(done[k % 2])
            ev = [torch.cuda.Event() for _ in range(5)]
            nabla.upload(fk, hf, 1, stream=s_up)
            ev[0].record(s_up)
            nabla.upload(uvk, huv, 2, stream=s_up)
            ev[1].record(s_up)
            stream.wait_event(ev[0])
            nabla.gradlap(method, fk, g, l, stream=stream)
            ev[2].record(stream)
            stream.wait_event(ev[1])
            nabla.divcurl(method, uvk, d, z, stream=stream)
            ev[3].record(stream)
            for j, (o, h, nv) in enumerate(zip((g, d, z, l), hout, nvars)):
                s_down.wait_event(ev[2] if j in (0, 3) else ev[3])
                nabla.download(h, o, nv, stream=s_down)
            ev[4].record(s_down)
            done[k % 2] = ev[4]

        for k in range(2):
            e2e_step(k)
        s_down.synchronize()
        barrier()
        t1 = time.perf_counter()
        for k in range(a.e2e_steps):
            e2e_step(k)
        s_down.synchronize()  # every step's results are on the host
        barrier()
        dt = time.perf_counter() - t1
        e2e = {"value": round(world * 4 * nl * a.e2e_steps / dt / 1e9, 3), "unit": "Gnode-levels/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "steps": a.e2e_steps,
               "path": "nb_field_upload, gradlap, divcurl, nb_field_download on three streams, "
                       "two device buffer sets (step k+1 uploads while step k downloads)"}
        del sets, f2, uv2
        torch.cuda.empty_cache()

    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "Gnode-levels/s",
        "n_gpus": world, "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(ms_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic: seeded spherical-harmonic fields (degree<=40), levels mixed from 8 bases",
        "config": {"workload": f"O{a.grid}x{L} grad+div+curl+lap FP32, compensated accumulation, FP64 geometry",
                   "grid": f"O{a.grid}", "nodes": V, "edges": E, "levels": L, "level_stride": fs.lp,
                   "ops_per_step": list(OPS), "step": ("grad(f) and lap(f) in one single-pass kernel; " if fused else
                            "grad(f); lap(f) as the divergence of that gradient; ")
                           + "div(uv) and curl(uv) in one fused pass",
                   "l2": "inputs larger than L2 (no flush)",
                   "parallelism": f"replicas x{world} (independent fields per GPU)",
                   "setup_s": round(setup_s, 2)},
        "per_op": per_op,
        "single_op_ms": single,
        "edge_variant_ms": edge_ms,
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1),
                     "peak": hbm, "unit": "GB/s", "frac": round(achieved / hbm, 4),
                     "peak_kind": peak_kind, "algorithmic_bytes": int(algo),
                     "traffic": measured_traffic(dom, V, L) if a.variant != 1 else None},
        "fp64": fp64,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
    }
    if a.batch_fields > 0:
        line["batched"] = bench_batched(a, nabla, synth, stream)
    if a.serve_seconds > 0:
        line["served"] = bench_served(a, nabla, synth)
    if sample is not None:
        line["cpu_baseline"], line["errors"] = cpu_baseline(a, sample)
    if world > 1:
        dist.destroy_process_group()
    return line if rank == 0 else None


# ------------------------------------------------------ batched and served

def _grid_bases(nabla, synth, N, lmax, radius):
    """Scalar / wind bases of O<N> in functionspace order (float64 numpy)."""
    g = nabla.Grid(N)
    m = nabla.Mesh(g, 1)
    meth = nabla.Method(m, radius)
    ll = g.lonlat()[m.permutation()]
    sb = synth.scalar_basis(ll[:, 1], ll[:, 0], lmax, synth.BASE_SEED + N).numpy()
    wb = synth.wind_basis(ll[:, 1], ll[:, 0], lmax, synth.BASE_SEED + N, radius).numpy()
    return meth, sb, wb


def bench_batched(a, nabla, synth, stream):
    """64 fields in one persistent captured-graph launch over O48..O400 with
    levels from {1, 37, 91, 137} and ops drawn uniformly (seeded)."""
    import numpy as np
    import torch
    rng = np.random.default_rng(synth.BASE_SEED + 3)
    grids = {N: _grid_bases(nabla, synth, N, 30, 6.37122e6) for N in (48, 96, 200, 400)}
    ops = ["grad", "div", "curl", "lap"]
    items32, items64, nl = [], [], 0
    for k in range(a.batch_fields):
        N = int(rng.choice(list(grids)))
        L = int(rng.choice([1, 37, 91, 137]))
        op = ops[int(rng.integers(4))]
        meth, sb, wb = grids[N]
        w = (rng.standard_normal((L, 8)) / np.sqrt(8)) * (1 + np.arange(L) / L)[:, None]
        x = sb @ w.T if op in ("grad", "lap") else np.einsum("vbc,kb->vkc", wb, w)
        for dt, items in ((torch.float32, items32), (torch.float64, items64)):
            fs = nabla.NodeColumns(meth, L, dt)
            xin = fs.create_field(nvar=1 if op in ("grad", "lap") else 2)
            xin.copy_(torch.as_tensor(x).to(xin.device))
            out = fs.create_field(nvar=2 if op == "grad" else 1)
            items.append((op, meth, xin, out))
        nl += meth.mesh.V * L
    b = nabla.Batch(items32)
    t = time.perf_counter()
    b.tune(stream)
    tune_s = time.perf_counter() - t
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    with torch.cuda.stream(stream):
        for _ in range(3):
            b.run(stream)
        ev[0].record(stream)
        reps = 20
        for _ in range(reps):
            b.run(stream)
        ev[1].record(stream)
    stream.synchronize()
    t_graph = ev[0].elapsed_time(ev[1]) / reps

    def single_sum(items):
        """Sum of the single operations' own kernel times, and the time of
        the whole sequence of single calls on the stream (launch gaps in)."""
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in items]
        with torch.cuda.stream(stream):
            for (op, meth, xin, out) in items:  # warm
                nabla.apply(meth, op, xin, out, stream=stream)
            for (op, meth, xin, out), (e0, e1) in zip(items, evs):
                e0.record(stream)
                nabla.apply(meth, op, xin, out, stream=stream)
                e1.record(stream)
        stream.synchronize()
        return sum(e0.elapsed_time(e1) for e0, e1 in evs), evs[0][0].elapsed_time(evs[-1][1])

    t_single, t_seq = single_sum(items32)
    t_f64, _ = single_sum(items64)
    info = b.info()
    staged = sum(1 for v in info["levels_per_block"] if v == 0)
    return {"workload": f"{a.batch_fields} fields, grids O48/O96/O200/O400, levels {{1,37,91,137}}, "
                        "ops uniform, SH degree<=30, FP32; one CUDA graph: persistent launches for "
                        "small items, staged launches for large ones (tuned routes)",
            "node_levels": int(nl), "graph_ms": round(t_graph, 4),
            "value": round(nl / (t_graph * 1e-3) / 1e9, 2), "unit": "Gnode-levels/s",
            "staged_route_items": staged,
            "single_op_sum_ms": round(t_single, 4),
            "single_op_sequence_ms": round(t_seq, 4),
            "speedup_vs_single_op_sequence": round(t_seq / t_graph, 3),
            "single_op_value": round(nl / (t_single * 1e-3) / 1e9, 2),
            "fp64_single_op_sum_ms": round(t_f64, 4),
            "fp64_value": round(nl / (t_f64 * 1e-3) / 1e9, 2),
            "speedup_vs_single_op": round(t_single / t_graph, 3),
            "speedup_vs_fp64": round(t_f64 / t_graph, 3),
            "units": int(info["units"]), "tune_s": round(tune_s, 2),
            "graph_nodes": int(info["graph_nodes"]), "graph_kernel_nodes": int(info["graph_kernels"]),
            "nodes_per_warp": sorted(set(int(v) for v in info["nodes_per_warp"])),
            "levels_per_block": sorted(set(int(v) for v in info["levels_per_block"]))}


def bench_served(a, nabla, synth):
    """Seeded Poisson arrivals; op in {grad, div, curl, lap}, grid in
    {O80, O160, O320, O640}, levels in {1, 37, 91, 137}, 1-8 fields; meshes
    resident, 60 GB admission budget; vs the same trace as sequential plain
    FP64 solves."""
    import numpy as np
    rng = np.random.default_rng(synth.BASE_SEED + 4)
    grids = {N: _grid_bases(nabla, synth, N, 30, 6.37122e6) for N in (80, 160, 320, 640)}
    ops = ["grad", "div", "curl", "lap"]
    n = int(a.serve_rate * a.serve_seconds)
    arrivals = np.cumsum(rng.exponential(1.0 / a.serve_rate, n))
    spec = [(ops[int(rng.integers(4))], int(rng.choice(list(grids))), int(rng.choice([1, 37, 91, 137])),
             int(rng.integers(1, 9))) for _ in range(n)]

    def run(dtype, nstreams, inflight, count=n, stretch=1.0):
        """The first `count` requests of the trace, arrival times x stretch."""
        srv = nabla.Server(int(60e9), nstreams=nstreams, max_inflight=inflight)
        for N, (meth, sb, wb) in grids.items():
            srv.add_grid(meth, sb, wb)
        # warm: every (op, grid, levels) once, so tile plans and pools exist
        warm = [nabla.Server.request(op, N, L, 1, dtype, seed=1)
                for op in ops for N in grids for L in (1, 37, 91, 137)]
        srv.run_trace(warm, np.zeros(len(warm)))
        reqs = [nabla.Server.request(op, N, L, f, dtype, seed=k) for k, (op, N, L, f) in enumerate(spec[:count])]
        res = srv.run_trace(reqs, arrivals[:count] * stretch)
        lat = np.array([r.done_s - r.arrival_s for r in res]) * 1e3
        span = max(r.done_s for r in res) - min(r.arrival_s for r in res)
        nl = sum(r.node_levels for r in res)
        bad = sum(r.status != 0 for r in res)
        st = srv.stats()
        return {"requests": count, "offered_req_per_s": round(a.serve_rate / stretch, 1),
                "failed": int(bad), "wall_s": round(span, 3),
                "req_per_s": round(count / span, 1), "gnl_s": round(nl / span / 1e9, 2),
                "p50_ms": round(float(np.percentile(lat, 50)), 3), "p99_ms": round(float(np.percentile(lat, 99)), 3),
                "mean_ms": round(float(lat.mean()), 3), "peak_budget_GB": round(st["peak_used"] / 1e9, 2)}

    ns, nf = a.serve_streams, a.serve_inflight
    ours = run(nabla.NB_F32, ns, nf)
    # the same trace at a fifth of the rate (first fifth of the requests):
    # latency below saturation
    light = run(nabla.NB_F32, ns, nf, count=max(1, n // 5), stretch=5.0)
    base = None if a.no_serve_baseline else run(nabla.NB_F64, 1, 1)
    return {"workload": f"Poisson {a.serve_rate:.0f} req/s for {a.serve_seconds:.0f} s (seeded), op in "
                        "{grad,div,curl,lap}, O80/O160/O320/O640, levels {1,37,91,137}, 1-8 fields, "
                        f"60 GB budget, {ns} streams, {nf} in flight, FP32 compensated",
            "continuous_batching_fp32": ours, "continuous_batching_fp32_fifth_rate": light,
            "sequential_plain_fp64": base}


# ---------------------------------------------------------- oracle timing

def take_sample(mesh, f, uv, outs, nlev_sample):
    """Levels of this run's FP32 inputs and step outputs, copied to the host
    in grid order: nlev_sample levels spread over the column (first and last
    included).  Inputs are kept as FP64 (their exact FP32 values)."""
    import numpy as np
    L = f.shape[1]
    levels = sorted(set(int(round(x)) for x in np.linspace(0, L - 1, max(1, min(nlev_sample, L)))))
    perm = mesh.permutation()

    def host(t):
        x = t[:, levels].detach().cpu().numpy()
        out = np.empty(x.shape, dtype=np.float64)
        out[perm] = x
        return out
    return {"levels": levels, "f": host(f), "uv": host(uv), "out32": sample_outputs(mesh, outs, levels)}


def sample_outputs(mesh, outs, levels):
    """Step outputs (grad, div, curl, lap) at `levels`, grid order, host."""
    import numpy as np
    perm = mesh.permutation()
    res = {}
    for name, t in zip(("grad", "div", "curl", "lap"), outs):
        x = t[:, levels].detach().cpu().numpy()
        out = np.empty(x.shape, dtype=x.dtype)
        out[perm] = x
        res[name] = out
    return res


def _omp_threads():
    """OpenMP threads the oracle runs on: the libgomp runtime's setting, else
    the CPUs this process may run on."""
    try:
        import ctypes
        return int(ctypes.CDLL("libgomp.so.1").omp_get_max_threads())
    except OSError:
        return len(os.sched_getaffinity(0))


def cpu_baseline(a, sample):
    """The FP64 oracle (as it stands) on the host cores, on a level sample of
    this run's own inputs: all four operators.  Its outputs are also the
    reference of the per-op error figures of the FP32 and FP64 GPU paths on
    the same levels (relative L2, per-node maximum, pole rows alone)."""
    import numpy as np
    import oracle
    m = oracle.build_mesh(a.grid, oracle.EARTH_RADIUS_M)
    f, uv = sample["f"], sample["uv"]
    L = f.shape[1]
    ts = []
    for _ in range(3):  # median of three runs of the sample
        t = time.perf_counter()
        ref = {"grad": oracle.grad(m, f), "div": oracle.div(m, uv), "curl": oracle.curl(m, uv),
               "lap": oracle.lap(m, f)}
        ts.append(time.perf_counter() - t)
    dt = statistics.median(ts)
    cores = _omp_threads()
    out = {"value": round(4 * m.V * L / dt / 1e9, 5), "unit": "Gnode-levels/s", "cores": cores,
           "kind": "oracle", "seconds": round(dt, 2),
           "sample": f"O{a.grid}, {L} of {a.nlev} levels (spread over the column) of the run's own "
                     "inputs, grad+div+curl+lap, FP64 C + OpenMP, median of 3 runs"}
    # the same oracle on one thread (OpenMP runtime of this process set to
    # one thread, then restored), median of three runs on two levels
    L1 = min(2, L)
    try:
        import ctypes
        gomp = ctypes.CDLL("libgomp.so.1")
        prev = gomp.omp_get_max_threads()
        gomp.omp_set_num_threads(1)
        ts = []
        try:
            f1, uv1 = np.ascontiguousarray(f[:, :L1]), np.ascontiguousarray(uv[:, :L1])
            for _ in range(3):
                t = time.perf_counter()
                oracle.grad(m, f1)
                oracle.div(m, uv1)
                oracle.curl(m, uv1)
                oracle.lap(m, f1)
                ts.append(time.perf_counter() - t)
        finally:
            gomp.omp_set_num_threads(prev)
        dt1 = statistics.median(ts)
        out["single_core"] = {"value": round(4 * m.V * L1 / dt1 / 1e9, 5), "seconds": round(dt1, 2),
                              "sample": f"O{a.grid}, {L1} levels, one thread, median of 3"}
    except OSError:
        out["single_core"] = None
    # error figures of the GPU paths against these oracle outputs
    nx0 = int(np.argmax(m.lat != m.lat[0]))
    nx1 = int(np.argmax(m.lat[::-1] != m.lat[-1]))
    pole = np.zeros(m.V, dtype=bool)
    pole[:nx0] = True
    pole[m.V - nx1:] = True

    def stats(x, r):
        if x.ndim == 3:
            parts = [stats(x[..., c], r[..., c]) for c in range(x.shape[-1])]
            return {k: max(p[k] for p in parts) for k in parts[0]}
        d = x.astype(np.float64) - r
        return {"rel_l2": float(np.linalg.norm(d.ravel()) / np.linalg.norm(r.ravel())),
                "max_rel": float(np.abs(d).max() / np.abs(r).max()),
                "max_abs": float(np.abs(d).max()),
                "pole_rel_l2": float(np.linalg.norm(d[pole].ravel()) / np.linalg.norm(r[pole].ravel()))}
    errors = {"reference": "FP64 oracle on the same inputs", "levels": sample["levels"],
              "definitions": {"rel_l2": "||x-ref||/||ref|| over all nodes of the sampled levels",
                              "max_rel": "max|x-ref| / max|ref|", "max_abs": "max|x-ref|",
                              "pole_rel_l2": "relative L2 over the first and last grid rows"}}
    for key, name in (("out32", "f32"), ("out64", "f64")):
        if key in sample:
            errors[name] = {op: {k: float(f"{v:.3e}") for k, v in stats(sample[key][op], ref[op]).items()}
                            for op in ("grad", "div", "curl", "lap")}
    return out, errors


def bench_reference(a):
    rank, world, local = dist_env()
    if rank != 0:
        return None
    steps = []
    import numpy as np
    import oracle
    from paper_1908_06091_b300 import synth
    m = oracle.build_mesh(a.grid, oracle.EARTH_RADIUS_M)
    L = max(1, min(a.cpu_levels, 8))
    f = synth.scalar_field(m.lat, m.lon, L, a.lmax).numpy()
    uv = synth.wind_field(m.lat, m.lon, L, a.lmax, m.R).numpy()

    def step():
        oracle.grad(m, f)
        oracle.div(m, uv)
        oracle.curl(m, uv)
        oracle.lap(m, f)
    for _ in range(a.warmup):
        step()
    t = time.perf_counter()
    for _ in range(a.steps):
        step()
    dt = time.perf_counter() - t
    value = 4 * m.V * L * a.steps / dt / 1e9
    cores = _omp_threads()
    sample = f"O{a.grid}, {L} of {a.nlev} levels per step, grad+div+curl+lap, FP64 C + OpenMP"
    return {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": "Gnode-levels/s",
            "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": round(dt / a.steps * 1e3, 2), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"O{a.grid}x{a.nlev} grad+div+curl+lap (oracle sample: {L} levels)",
                       "grid": f"O{a.grid}", "levels": a.nlev},
            "cpu_baseline": {"value": round(value, 5), "unit": "Gnode-levels/s", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 5), "unit": "Gnode-levels/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    a = parse()
    line = bench_reference(a) if a.impl == "reference" else bench_ours(a)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
