#!/usr/bin/env python3
"""Throughput of the point-cloud Fresnel hologram on one GB300 (or N replicas).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload (default): a 1920x1080 hologram of 10,000 seeded synthetic points
(z ~ U[0.3, 1.0] m, A ~ U[0.5, 1.0], lambda = 532 nm, p = 8 um), the
display-size case of the paper's direct-calculation experiments.  One step is
one pass of the hot path over that cloud: point preparation, the direct
kernel (SFU cosine; the CTAs take equal shares of the (pixel tile, point)
pairs and sum each tile's parts in the kernel), and the 8-bit quantiser.
Inputs and outputs are far below L2, so a 256 MiB buffer is written between
timed steps to flush L2; the flush is not timed.

Metric: G point-pixel evaluations per second (W*H*N per hologram), with
holograms/s beside it.  Rank 0 prints one JSON line.  Under torchrun every
rank computes its own replica (no collective on the data path; weak scaling),
and the time is the maximum over ranks.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "G point-pixel evals/s and holograms/s, direct FP32 vs tensor GEMM, at stated NRMS error"
UNIT = "Gevals/s"
MUFU_PER_SM_PER_CLK = 16        # MUFU (hardware sine / cosine) operations per SM per clock
FMA_PER_SM_PER_CLK = 128        # FP32 FMA-pipe operations per SM per clock


def direct_ops(form, width, height, n_points):
    """The direct kernel's work per launch in FMA-pipe operations, as the kernel does it: a CTA covers a 128 x 64
    tile (256 x 32 where that pads a fifth fewer pixels); per point it takes the sine and cosine of the tile's
    columns and rows once (the SFU form: one FFMA and the sine's range multiply per entry, and the amplitude's two
    multiplies per row entry; the accurate form: two polynomials of 8 FMA-pipe operations per entry), then every
    pixel costs two FMAs (one packed two-lane FMA per pair of columns).  Returns (operations, pipe, peak operations per SM per clock, operations per
    evaluation); the MUFU operations of the SFU form (two per entry, 0.05 per evaluation) bound nothing."""
    def padded(tw, th):
        return -(-width // tw) * tw * (-(-height // th) * th)
    tw, th = (256, 32) if padded(256, 32) * 6 < padded(128, 64) * 5 else (128, 64)
    tiles = padded(tw, th) // (tw * th)
    per_col, per_row = (2, 4) if form == "direct_sfu" else (16, 18)
    per_point_tile = 2 * tw * th + tw * per_col + th * per_row
    ops = n_points * tiles * per_point_tile
    return ops, "FMA", FMA_PER_SM_PER_CLK, ops / (n_points * width * height)


# DRAM bytes per launch of the dominant kernel from ncu (dram__bytes_read.sum +
# dram__bytes_write.sum), keyed by the SHA-1 of the kernel's sources they were
# taken on; a changed source reports null until it is profiled again.
NCU_TRAFFIC = [
    # profiles/direct_sfu-1920x1080-n10000.md (api.cu holds the launch's CTA count)
    {"kernel": "direct_sfu", "form": "direct_sfu", "workload": "direct-1920x1080-n10000",
     "src": ["direct.cu", "direct_dev.cuh", "device_util.cuh", "api.cu"],
     "sha1": "9b424be116a5758083538cced11cb2c3dd771817", "bytes_per_launch": 365056},
    # profiles/gemm_f16-1920x1080-n50000.md: 600.731 MB read + 3.053 MB written per launch
    {"kernel": "gemm_tcgen05", "form": "gemm_f16", "workload": "gemm-1920x1080-n50000",
     "src": ["gemm.cu", "gemm_dev.cuh", "tcgen05.cuh", "device_util.cuh"],
     "sha1": "1b3da24ffb355250d6467758d091b4a7b91d7b3a", "bytes_per_launch": 603784192},
]


def ncu_traffic(kernel, form, workload):
    """DRAM bytes per launch from the committed ncu summary, if the kernel source is unchanged since."""
    for t in NCU_TRAFFIC:
        if (t["kernel"], t["form"], t["workload"]) == (kernel, form, workload):
            srcs = [os.path.join(ROOT, "paper_1309_2734_gb300", "csrc", f) for f in t["src"]]
            return t["bytes_per_launch"] if _sha1(srcs) == t["sha1"] else None
    return None


def _sha1(paths):
    """SHA-1 of the kernel's source files, concatenated in the order given."""
    h = hashlib.sha1()
    for path in paths:
        with open(path, "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while it runs."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clk", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def stop(self):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
            os.unlink(self.path)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"], "samples": 0}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max((num(r[3]) or 0.0) for r in rows)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def cpu_baseline(cloud, target_s: float = 12.0, gpu_field=None):
    """The FP64 oracle, as it stands, on a window of rows of the same workload (host cores)."""
    import numpy as np
    import oracle
    cores = oracle.threads()
    W, H = cloud.width, cloud.height
    t0 = time.perf_counter()
    probe_rows = max(1, min(H, cores))
    oracle.field(cloud.pitch_m, cloud.lambda_m, cloud.xyz, cloud.amp, W, H, window=(0, 0, probe_rows, W))
    per_row = (time.perf_counter() - t0) / probe_rows
    rows = int(max(cores, min(H, target_s / max(per_row, 1e-9))))
    rows = max(cores, rows // cores * cores) if rows >= cores else rows
    rows = min(rows, H)
    r0 = (H - rows) // 2
    t0 = time.perf_counter()
    ref = oracle.field(cloud.pitch_m, cloud.lambda_m, cloud.xyz, cloud.amp, W, H, window=(r0, 0, rows, W))
    dt = time.perf_counter() - t0
    evals = rows * W * cloud.n_points
    out = {"value": evals / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"rows {r0}..{r0 + rows - 1} (all {W} columns, all {cloud.n_points} points) of the "
                     f"{W}x{H} hologram; {evals:.3e} FP64 evals in {dt:.1f} s",
           "seconds": dt}
    nrms = None
    if gpu_field is not None:
        got = gpu_field[r0:r0 + rows].astype(np.float64)
        nrms = oracle.nrms(got, ref)
        out["max_abs_err_over_rms"] = float(np.max(np.abs(got - ref)) / np.sqrt(np.mean(ref * ref)))
    return out, nrms, (r0, rows, ref)


def nrms_of_forms(samples, cloud, rows_ref):
    """NRMS of each compared form: on the oracle rows of the timed cloud, or on 256 sampled
    pixels (FP64 oracle) of the other clouds."""
    import numpy as np
    import oracle
    r0, rows, ref = rows_ref
    out = {}
    cache = {}
    for key, (wc, field) in samples.items():
        if wc is cloud:
            out[key] = oracle.nrms(field[r0:r0 + rows], ref)
            continue
        if wc.evals <= 2e8:   # small clouds: the whole field
            if wc.name not in cache:
                cache[wc.name] = oracle.field(wc.pitch_m, wc.lambda_m, wc.xyz, wc.amp, wc.width, wc.height)
            out[key] = oracle.nrms(field, cache[wc.name])
            continue
        if wc.name not in cache:
            rng = np.random.default_rng(20260)
            cols = rng.integers(0, wc.width, 256)
            rws = rng.integers(0, wc.height, 256)
            cache[wc.name] = (cols, rws, oracle.field_at(wc.pitch_m, wc.lambda_m, wc.xyz, wc.amp, cols, rws))
        cols, rws, pix = cache[wc.name]
        out[key] = oracle.nrms(field[rws, cols], pix)
    return out


def _r3(v):
    """v rounded to three significant digits (None stays None)."""
    if v is None:
        return None
    return float(f"{v:.3g}")


def compact_summary(forms, large, vbatch, cloud_name):
    """The figures the comparison rests on, short enough for the end of the printed line: per form and
    workload the time, throughput, roofline fraction, DRAM traffic and NRMS against the FP64 oracle; the
    GEMM-versus-direct comparison at 1920x1080; the large case and the batch."""
    short = {"direct-256x256-n1024": "256x256n1024", "direct-1920x1080-n10000": "1080p-n10k",
             "gemm-1920x1080-n50000": "1080p-n50k"}
    fs = {"cols": ["ms", "Gevals/s", "kernel roofline frac", "hologram tensor frac", "nrms vs oracle",
                   "ncu DRAM bytes/launch"]}
    for key, rec in forms.items():
        form, wl = key.split("@")
        roof = rec.get("roofline") or {}
        fs[f"{form}@{short.get(wl, wl)}"] = [
            _r3(rec["ms_per_hologram"]), _r3(rec["gevals_per_s"]), _r3(roof.get("frac")),
            _r3(rec.get("e2e_tensor_frac")), _r3(rec.get("nrms_vs_oracle")), roof.get("traffic")]
    # GEMM against direct at 1920x1080: the fastest form within each accuracy class
    versus = {}
    for wl in ("direct-1920x1080-n10000", "gemm-1920x1080-n50000"):
        d = forms.get(f"direct_sfu@{wl}")
        for g, cls in (("gemm_split16", "1e-5"), ("gemm_f16", "2e-3"), ("gemm_bf16", "1e-2")):
            r = forms.get(f"{g}@{wl}")
            if d is not None and r is not None:
                versus[f"{short[wl]} {g} (NRMS<={cls})"] = [
                    _r3(r["ms_per_hologram"]), _r3(d["ms_per_hologram"]),
                    _r3(d["ms_per_hologram"] / r["ms_per_hologram"]),
                    _r3(r.get("nrms_vs_oracle")), _r3(d.get("nrms_vs_oracle"))]
    if versus:
        versus["cols"] = ["gemm ms", "direct_sfu ms", "speedup", "gemm nrms", "direct nrms"]
    lg = {k: {"ms": _r3(v.get("ms_per_hologram")), "frac": _r3((v.get("roofline") or {}).get("frac")),
              "nrms": _r3(v.get("nrms_vs_oracle"))} for k, v in large.items()}
    vb = {k: {"ms": _r3(v.get("ms_per_batch")), "holo_s": _r3(v.get("holograms_per_s")),
              "tc_frac": _r3(v.get("tensor_frac")), "nrms": _r3(v.get("nrms_vs_oracle")),
              "kernel_ms": {kk: _r3(vv) for kk, vv in (v.get("kernel_ms") or {}).items()}}
          for k, v in vbatch.items() if k.startswith("nrms_")}
    return {"forms": fs, "gemm_vs_direct": versus, "layered_4096": lg, "video_batch_64": vb}


def run_reference(args):
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    from paper_1309_2734_gb300 import workloads
    import oracle
    cloud = workloads.WORKLOADS[args.workload]()
    if world > 1:   # the launcher caps each rank at one OpenMP thread; rank 0 is the only one at work here
        oracle.set_threads(len(os.sched_getaffinity(0)))
    cores = oracle.threads()
    W, H = cloud.width, cloud.height
    # size one step so that the whole --steps/--warmup run takes about two minutes of host work
    t0 = time.perf_counter()
    oracle.field(cloud.pitch_m, cloud.lambda_m, cloud.xyz, cloud.amp, W, H, window=(0, 0, cores, W))
    per_row = (time.perf_counter() - t0) / cores
    step_s = min(6.0, max(0.3, 120.0 / (args.steps + args.warmup)))
    rows = max(1, min(H, int(step_s / max(per_row, 1e-9))))
    times = []
    for i in range(args.warmup + args.steps):
        r0 = (i * rows) % max(1, H - rows + 1)
        t0 = time.perf_counter()
        oracle.field(cloud.pitch_m, cloud.lambda_m, cloud.xyz, cloud.amp, W, H, window=(r0, 0, rows, W))
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    evals = rows * W * cloud.n_points
    value = evals * len(times) / sum(times) / 1e9
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": cloud.name, "width": W, "height": H, "n_points": cloud.n_points,
                       "step": f"{rows} rows x {W} columns of the hologram (bounded sample)"},
            "holograms_per_s": value * 1e9 / cloud.evals,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{rows} of {H} rows per step, all {cloud.n_points} points"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_ours(args):
    import numpy as np
    import torch
    rank, world, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl", init_method="env://")
    from paper_1309_2734_gb300 import Hologram, workloads
    from paper_1309_2734_gb300.build import build
    if rank == 0:
        build()
    if dist is not None:
        dist.barrier()

    cloud = workloads.WORKLOADS[args.workload]()
    W, H, N = cloud.width, cloud.height, cloud.n_points
    stream = torch.cuda.current_stream()
    xyz = torch.from_numpy(cloud.xyz).cuda()
    amp = torch.from_numpy(cloud.amp).cuda()
    out = torch.empty((H, W), dtype=torch.float32, device="cuda")
    q = torch.empty((H, W), dtype=torch.uint8, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    h = Hologram(W, H, cloud.pitch_m, cloud.lambda_m, form=args.form, stream=stream)

    def step():
        h.point_cloud(xyz, amp, out)
        h.quantize8(out, q)

    for _ in range(args.warmup):
        step()
    h.sync()
    h.profile(True)
    h.profile_read(reset=True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local).start()
    for a, b in ev:
        flush.fill_(1)
        a.record(stream)
        step()
        b.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clocks = clk.stop()
    h.sync()
    prof = h.profile_read(reset=True)
    h.profile(False)
    total_ms = sum(a.elapsed_time(b) for a, b in ev)
    if dist is not None:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    launches = sum(v[0] for v in prof.values())

    # end to end through the C ABI with host buffers (copies inside the timed region)
    hx = torch.from_numpy(cloud.xyz).pin_memory()
    ha = torch.from_numpy(cloud.amp).pin_memory()
    ho = torch.empty((H, W), dtype=torch.float32).pin_memory()
    for _ in range(2):
        h.point_cloud_host(hx, ha, ho)
    e2e_s = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        h.point_cloud_host(hx, ha, ho)
        e2e_s.append(time.perf_counter() - t0)
    e2e_total = sum(e2e_s)
    if dist is not None:
        t = torch.tensor([e2e_total], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_total = float(t.item())

    # other forms, for the comparison the metric names: every form on this cloud, and the
    # GEMM forms also on the 1920x1080, 50,000-point cloud they are meant for
    forms = {}
    samples = {}
    # every compared form on the headline cloud; the GEMM forms (and the direct kernel, for the comparison the
    # metric names) on the 1920x1080, 50,000-point cloud they are meant for; every form on the 256x256,
    # 1,024-point cloud (the small direct case)
    gemm_forms = [f for f in args.compare if f.startswith("gemm")]
    extra_clouds = []
    if gemm_forms:
        extra_clouds.append((workloads.display_gemm(), gemm_forms + ["direct_sfu"]))
    if not args.no_small:
        extra_clouds.append((workloads.small_direct(), ["direct_sfu", "direct_accurate"] + gemm_forms))
    runs = [(cloud, xyz, amp, h, f) for f in args.compare]
    for wc, flist in extra_clouds:
        dev = (torch.from_numpy(wc.xyz).cuda(), torch.from_numpy(wc.amp).cuda(),
               Hologram(wc.width, wc.height, wc.pitch_m, wc.lambda_m, stream=stream))
        runs += [(wc, dev[0], dev[1], dev[2], f) for f in flist]
    for wc, cx, ca, hh, extra in runs:
        hh.set_form(extra)
        o = torch.empty((wc.height, wc.width), dtype=torch.float32, device="cuda")
        for _ in range(2):
            hh.point_cloud(cx, ca, o)
        hh.sync()
        hh.profile(True)
        hh.profile_read(reset=True)
        reps = max(3, args.steps // 4) if wc.evals > 1e9 else max(20, args.steps)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            hh.point_cloud(cx, ca, o)
        e1.record(stream)
        torch.cuda.synchronize()
        hh.sync()
        kp = hh.profile_read(reset=True)
        hh.profile(False)
        ms = e0.elapsed_time(e1) / reps
        rec = {"gevals_per_s": wc.evals / ms / 1e6, "ms_per_hologram": ms,
               "kernel_ms": {k: v[1] / reps for k, v in kp.items()}}
        if extra.startswith("gemm") and "gemm_tcgen05" in kp:
            passes = 3 if extra == "gemm_split16" else 1
            gl, gms = kp["gemm_tcgen05"]   # one launch per chunk of points: time per hologram
            tflops = 4.0 * wc.evals * passes / (gms / reps * 1e-3) / 1e12
            peak_tc = _peaks().get("bf16_tflops") or 1939.7
            rec["roofline"] = {"kernel": "gemm_tcgen05", "bound": "tensor", "achieved": tflops,
                               "peak": peak_tc, "unit": "TFLOP/s", "frac": tflops / peak_tc,
                               "flops_per_eval": 4 * passes,
                               "traffic": ncu_traffic("gemm_tcgen05", extra, wc.name),
                               "peak_basis": "measured dense bf16 burst (fp16 nominal rate is the same)"}
            # the whole hologram (prep, factors, GEMM, reduction) against the same tensor peak
            rec["e2e_tensor_frac"] = 4.0 * wc.evals * passes / (ms * 1e-3) / 1e12 / peak_tc
        elif extra in kp:
            ops, pipe, per_clk, per_eval = direct_ops(extra, wc.width, wc.height, wc.n_points)
            pk = per_clk * torch.cuda.get_device_properties(local).multi_processor_count * \
                (_peaks().get("sm_max_mhz") or 2070.0) * 1e6
            dms = kp[extra][1] / max(kp[extra][0], 1)
            rec["roofline"] = {"kernel": extra, "bound": "alu", "achieved": ops / (dms * 1e-3) / 1e9,
                               "peak": pk / 1e9, "unit": f"G {pipe} op/s", "ops_per_eval": round(per_eval, 4),
                               "frac": ops / (dms * 1e-3) / pk,
                               "traffic": ncu_traffic(extra, extra, wc.name)}
        key = f"{extra}@{wc.name}"
        forms[key] = rec
        samples[key] = (wc, o.cpu().numpy())
    for wc, cx, ca, hh, extra in runs:
        if hh is not h:
            hh.close()
    # the paper's own timed workload (Tables 3-4): phase-only CGH of 1920x1080 holograms with
    # 10^3, 10^4 and 10^5 points (complex wave + kinoform quantisation), beside the Tesla K20's
    # published times for the direct calculation (context only: other hardware, fast math)
    paper = {}
    if not args.no_paper_workload:
        k20 = {1000: 0.016, 10000: 0.168, 100000: 1.68}
        for n_pts, t_k20 in k20.items():
            pc = workloads.random_cloud(13092734100 + n_pts, 1920, 1080, n_pts)
            px, pa = torch.from_numpy(pc.xyz).cuda(), torch.from_numpy(pc.amp).cuda()
            wbuf = torch.empty((2, 1080, 1920), dtype=torch.float32, device="cuda")
            kbuf = torch.empty((1080, 1920), dtype=torch.uint8, device="cuda")
            entry = {"k20_direct_s": t_k20}
            with Hologram(1920, 1080, pc.pitch_m, pc.lambda_m, stream=stream) as hp:
                for pform in ("direct_sfu", "gemm_f16", "gemm_split16"):
                    hp.set_form(pform)
                    hp.wave(px, pa, wbuf)
                    hp.kinoform8(wbuf, kbuf)
                    hp.sync()
                    reps = 3 if n_pts <= 10000 or pform != "direct_sfu" else 1
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    for _ in range(reps):
                        hp.wave(px, pa, wbuf)
                        hp.kinoform8(wbuf, kbuf)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    hp.sync()
                    sec = e0.elapsed_time(e1) / reps * 1e-3
                    entry[pform] = {"s_per_hologram": sec, "gevals_per_s": pc.evals / sec / 1e9,
                                    "speedup_vs_k20": t_k20 / sec}
            paper[f"n{n_pts}"] = entry

    # the large depth-layered case: 4096x4096, 10^6 points on 16 planes; the GEMM forms group
    # the points by plane and column (automatic rule), beside the ungrouped split form and the
    # direct kernel; NRMS on 256 sampled pixels against the FP64 oracle (CPU leg)
    large = {}
    if not args.no_large:
        from paper_1309_2734_gb300 import _lib
        lc = workloads.large_layered()
        lx, la = torch.from_numpy(lc.xyz).cuda(), torch.from_numpy(lc.amp).cuda()
        lbuf = torch.empty((lc.height, lc.width), dtype=torch.float32, device="cuda")
        n_groups = int(np.unique(lc.xyz[:, [0, 2]], axis=0).shape[0])
        rng = np.random.default_rng(4096)
        lcols, lrows = rng.integers(0, lc.width, 256), rng.integers(0, lc.height, 256)
        with Hologram(lc.width, lc.height, lc.pitch_m, lc.lambda_m, stream=stream, timeout_ms=60000) as hl:
            for lform, group, reps in (("gemm_split16", 0, 5), ("gemm_f16", 0, 5), ("gemm_split16", 1, 1),
                                       ("direct_sfu", 0, 1)):
                hl.set_form(lform)
                hl.set_option(_lib.CGH_OPT_GEMM_GROUP, group)
                hl.point_cloud(lx, la, lbuf)
                hl.sync()
                hl.profile(True)
                hl.profile_read(reset=True)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(reps):
                    hl.point_cloud(lx, la, lbuf)
                e1.record(stream)
                torch.cuda.synchronize()
                hl.sync()
                kp = hl.profile_read(reset=True)
                hl.profile(False)
                ms = e0.elapsed_time(e1) / reps
                grouped = "group_factors" in kp
                rec = {"ms_per_hologram": ms, "gevals_per_s": lc.evals / ms / 1e6, "grouped": grouped,
                       "kernel_ms": {k: v[1] / max(v[0], 1) for k, v in kp.items()}}
                if lform.startswith("gemm") and "gemm_tcgen05" in kp:
                    passes = 3 if lform == "gemm_split16" else 1
                    k_units = n_groups if grouped else lc.n_points
                    gl, gms = kp["gemm_tcgen05"]   # one launch per chunk of K units: time per hologram
                    tflops = 4.0 * lc.width * lc.height * k_units * passes / (gms / reps * 1e-3) / 1e12
                    peak_tc = _peaks().get("bf16_tflops") or 1939.7
                    rec["gemm_k"] = 2 * k_units
                    rec["roofline"] = {"kernel": "gemm_tcgen05", "bound": "tensor", "achieved": tflops,
                                       "peak": peak_tc, "unit": "TFLOP/s", "frac": tflops / peak_tc}
                rec["_sample"] = lbuf[torch.from_numpy(lrows).cuda(), torch.from_numpy(lcols).cuda()].cpu().numpy()
                large[f"{lform}{'' if group == 0 else '/ungrouped'}"] = rec
        if not args.no_cpu_baseline:
            import oracle
            lref = oracle.field_at(lc.pitch_m, lc.lambda_m, lc.xyz, lc.amp, lcols, lrows)
            for rec in large.values():
                rec["nrms_vs_oracle"] = oracle.nrms(rec["_sample"], lref)
        for rec in large.values():
            rec.pop("_sample", None)
        del lx, la, lbuf

    # the paper's Fresnel diffraction (Table 5: N x N planes, lambda = 633 nm, z = 1 m as in its listing)
    # and wavefront-recording method (Table 6: 10^3..10^5 points; here a 2048 x 2048 hologram with the
    # plane 0.5 m away and the points 2-10 mm behind it), beside the paper's times (other hardware)
    fresnel_t, wrp_t = {}, {}
    if not args.no_fresnel:
        def _ms(fn, reps):
            fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps
        table5 = {1024: (0.17, 0.32, 0.011), 2048: (0.60, 0.41, 0.027), 4096: (2.06, 0.87, 0.125),
                  8192: (9.00, 3.80, None)}
        for side, (t_cpu, t_phi, t_k20) in table5.items():
            plane = torch.from_numpy(workloads.complex_plane(5, side, side)).cuda()
            with Hologram(side, side, 8e-6, 633e-9, stream=stream) as hf:
                dst = torch.empty_like(plane)
                ms = _ms(lambda: hf.fresnel(plane, 1.0, dst), 5)
                hf.profile(True)
                hf.profile_read(reset=True)
                hf.fresnel(plane, 1.0, dst)
                hf.sync()
                kp = hf.profile_read(reset=True)
            fresnel_t[f"{side}x{side}"] = {"ms": ms, "paper_s": {"cpu": t_cpu, "xeon_phi": t_phi, "k20": t_k20},
                                     "speedup_vs_k20": (t_k20 * 1e3 / ms) if t_k20 else None,
                                     "kernel_ms": {k: v[1] for k, v in kp.items()}}
            del plane, dst
        table6 = {1000: (1.02, 0.68, 0.029), 10000: (3.04, 0.70, 0.030), 100000: (9.34, 0.72, 0.035)}
        for n_pts, (t_cpu, t_phi, t_k20) in table6.items():
            wc = workloads.wrp_cloud(6, 2048, 2048, n_pts)
            wx, wa = torch.from_numpy(wc.xyz).cuda(), torch.from_numpy(wc.amp).cuda()
            obuf = torch.empty((2, 2048, 2048), dtype=torch.float32, device="cuda")
            kbuf = torch.empty((2048, 2048), dtype=torch.uint8, device="cuda")
            with Hologram(2048, 2048, wc.pitch_m, wc.lambda_m, stream=stream) as hw:
                hw.set_phase_model("fresnel_piston")
                step_w = lambda: (hw.wrp(wx, wa, 0.5, obuf), hw.kinoform8(obuf, kbuf))
                ms = _ms(step_w, 5)
                hw.profile(True)
                hw.profile_read(reset=True)
                step_w()
                hw.sync()
                kp = hw.profile_read(reset=True)
            wrp_t[f"n{n_pts}"] = {"ms": ms, "paper_s": {"cpu": t_cpu, "xeon_phi": t_phi, "k20": t_k20},
                                  "speedup_vs_k20": t_k20 * 1e3 / ms, "kernel_ms": {k: v[1] for k, v in kp.items()},
                                  "step": "WRP record + Fresnel diffraction (2 FFTs, cached chirp spectrum) + kinoform8"}

    # the batched workload: 64 frames of uneven size and point count in one cgh_batch call (persistent
    # launches per form kind, captured in a CUDA graph and replayed), forms and tiles per frame from the
    # autotuner at each accuracy class; NRMS on sampled pixels of every frame (CPU leg)
    vbatch = {}
    if not args.no_batch:
        from paper_1309_2734_gb300 import _lib, batch as run_batch
        from paper_1309_2734_gb300.shard import shard_instances
        all_frames = workloads.video_batch()
        if args.batch_frames:   # a subset of the frames (a small case for profilers)
            all_frames = [all_frames[int(i)] for i in args.batch_frames.split(",")]
        # under torchrun every rank takes its share of the frames (largest W*H*N first to the least-loaded rank;
        # no collective on the data path) and the batch time is the slowest rank's
        mine = shard_instances([c.evals for c in all_frames], rank, world) if world > 1 else range(len(all_frames))
        frames = [all_frames[i] for i in mine]
        fdev = [(torch.from_numpy(c.xyz).cuda(), torch.from_numpy(c.amp).cuda(), c.width, c.height, c.pitch_m,
                 c.lambda_m) for c in frames]
        fouts = [torch.empty((c.height, c.width), dtype=torch.float32, device="cuda") for c in frames]
        evals = sum(c.evals for c in frames)
        rng = np.random.default_rng(6464)
        picks = [(rng.integers(0, c.width, 16), rng.integers(0, c.height, 16)) for c in frames]
        for tol in [float(t) for t in args.batch_tols.split(",")]:
            with Hologram(8, 8, 8e-6, 532e-9, form="auto", stream=stream, timeout_ms=20000) as hb:
                hb.set_option(_lib.CGH_OPT_TOLERANCE_E9, int(round(tol * 1e9)))
                _lib.check(_lib.cgh_autotune(hb.ctx, 0), "cgh_autotune")
                run_batch(hb, fdev, fouts)   # plan and graph, untimed
                hb.sync()
                forms_b = _lib.cgh_batch_forms(hb.ctx)
                hb.profile(True)
                hb.profile_read(reset=True)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                reps = 3
                e0.record(stream)
                for _ in range(reps):
                    run_batch(hb, fdev, fouts)
                e1.record(stream)
                torch.cuda.synchronize()
                hb.sync()
                kp = hb.profile_read(reset=True)
                hb.profile(False)
                ms = e0.elapsed_time(e1) / reps
                if dist is not None:
                    t_ms = torch.tensor([ms], device="cuda")
                    dist.all_reduce(t_ms, op=dist.ReduceOp.MAX)
                    ms = float(t_ms.item())
                picked = [o[torch.from_numpy(r).cuda(), torch.from_numpy(c).cuda()].cpu().numpy()
                          for o, (c, r) in zip(fouts, picks)]
            names = {_lib.CGH_DIRECT_SFU: "direct_sfu", _lib.CGH_DIRECT_ACCURATE: "direct_accurate",
                     _lib.CGH_GEMM_F16: "gemm_f16", _lib.CGH_GEMM_BF16: "gemm_bf16",
                     _lib.CGH_GEMM_SPLIT16: "gemm_split16"}
            flops = sum(4.0 * c.evals * (3 if f == _lib.CGH_GEMM_SPLIT16 else 1)
                        for c, f in zip(frames, forms_b) if f >= _lib.CGH_GEMM_F16)
            peak_tc = _peaks().get("bf16_tflops") or 1939.7
            if dist is not None:   # the whole batch's work and GEMM flops over the slowest rank's time
                tot = torch.tensor([float(evals), flops], device="cuda", dtype=torch.float64)
                dist.all_reduce(tot)
                evals_all, flops = float(tot[0].item()), float(tot[1].item())
            else:
                evals_all = evals
            vbatch[f"nrms_{tol:g}"] = {
                "ms_per_batch": ms, "holograms_per_s": len(all_frames) / (ms * 1e-3),
                "gevals_per_s": evals_all / (ms * 1e-3) / 1e9, "_samples": picked,
                "forms": {v: sum(1 for f in forms_b if f == k) for k, v in names.items()
                          if any(f == k for f in forms_b)},
                # one persistent launch per batch (and the memset of its counters), timed with CUDA events
                "kernel_ms": {k: v[1] / reps for k, v in kp.items()},
                "gemm_tflops": flops / (ms * 1e-3) / 1e12,
                "tensor_frac": flops / (ms * 1e-3) / 1e12 / peak_tc}
        vbatch["frames"] = len(all_frames)
        vbatch["frames_this_rank"] = len(frames)
        vbatch["sharding"] = f"frames split over {world} ranks (shard_instances)" if world > 1 else "one GPU"
        vbatch["evals_per_batch"] = sum(c.evals for c in all_frames)
        vbatch["sizes"] = sorted({f"{c.width}x{c.height}" for c in all_frames})
        vbatch["points"] = [int(min(c.n_points for c in all_frames)), int(max(c.n_points for c in all_frames))]
        if not args.no_cpu_baseline:
            import oracle
            refs = [oracle.field_at(c.pitch_m, c.lambda_m, c.xyz, c.amp, cc, rr) for c, (cc, rr) in zip(frames, picks)]
            for key in [k for k in vbatch if k.startswith("nrms_")]:
                got = np.concatenate(vbatch[key]["_samples"])
                vbatch[key]["nrms_vs_oracle"] = oracle.nrms(got, np.concatenate(refs))
        for key in [k for k in vbatch if k.startswith("nrms_")]:
            vbatch[key].pop("_samples", None)
        del fdev, fouts

    h.set_form(args.form)
    h.point_cloud(xyz, amp, out)
    h.sync()
    field = out.cpu().numpy()

    if rank != 0:
        h.close()
        if dist is not None:
            dist.destroy_process_group()
        return 0

    evals_all = cloud.evals * args.steps * world
    value = evals_all / (total_ms * 1e-3) / 1e9
    props = torch.cuda.get_device_properties(local)
    peaks = _peaks()
    sm_max = peaks.get("sm_max_mhz") or clocks.get("sm_max_mhz") or 2070.0
    if args.form.startswith("gemm"):
        # tensor-bound: 4 flop per evaluation per product (3 products for split FP16)
        dom = "gemm_tcgen05"
        src = "gemm.cu"
        dom_launches, dom_ms = prof.get(dom, (0, 0.0))
        passes = 3 if args.form == "gemm_split16" else 1
        peak = peaks.get("bf16_tflops") or 1939.7
        # the GEMM's K: 2 per point, or 2 per (plane, column) group when the grouped form ran; the flops of all
        # timed steps over the kernel's total time = flops per launch over the average launch (chunks included)
        grouped = "group_factors" in prof
        k_units = int(np.unique(cloud.xyz[:, [0, 2]], axis=0).shape[0]) if grouped else N
        achieved = (4.0 * W * H * k_units * passes * args.steps / (dom_ms * 1e-3) / 1e12) if dom_ms > 0 else None
        roof = {"bound": "tensor", "unit": "TFLOP/s", "gemm_k": 2 * k_units,
                "peak_basis": "measured dense bf16 burst (fp16 nominal rate is the same)"}
    else:
        # the FMA pipe of the implemented evaluation, see direct_ops
        dom = args.form
        src = "direct.cu"
        dom_launches, dom_ms = prof.get(dom, (0, 0.0))
        ops, pipe, per_clk, per_eval = direct_ops(args.form, W, H, N)
        peak = per_clk * props.multi_processor_count * sm_max * 1e6 / 1e9
        achieved = ops / (dom_ms / max(dom_launches, 1) * 1e-3) / 1e9 if dom_ms > 0 else None
        roof = {"bound": "alu", "unit": f"G {pipe} op/s",
                "peak_basis": f"{per_clk} {pipe} op/clk/SM x {props.multi_processor_count} SMs x {sm_max:.0f} MHz "
                              f"(sm_max_mhz of measured peaks); {per_eval:.4f} {pipe} op per evaluation "
                              "(two FMAs a pixel and point, and per point the sines and cosines of the CTA's "
                              "tile columns and rows)"}
        if pipe == "MUFU":
            # the same pipe measured in this run: independent hardware sines on every SM (cgh_measure_mufu)
            from paper_1309_2734_gb300 import _lib
            probe = _lib.cgh_measure_mufu(h.ctx) / 1e9
            roof["peak_probe"] = probe
            roof["frac_of_probe"] = achieved / probe if achieved else None
    traffic = ncu_traffic(dom, args.form, cloud.name)

    cpu, nrms = (None, None)
    if not args.no_cpu_baseline:
        cpu, nrms, rows_ref = cpu_baseline(cloud, gpu_field=field)
        form_nrms = nrms_of_forms(samples, cloud, rows_ref)
        for k, v in form_nrms.items():
            forms[k]["nrms_vs_oracle"] = v

    # the headline form on its own cloud, beside the compared forms
    forms = {f"{args.form}@{cloud.name}": {
        "ms_per_hologram": total_ms / args.steps, "gevals_per_s": value / world,
        "nrms_vs_oracle": nrms,
        "roofline": {"frac": (achieved / peak) if achieved else None, "traffic": traffic}}, **forms}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"gemm_f16": "f16", "gemm_bf16": "bf16", "gemm_split16": "f16x2 (hi+lo)"}.get(args.form, "f32"),
        "data": "synthetic",
        "config": {"workload": cloud.name, "width": W, "height": H, "n_points": N, "form": args.form,
                   "step": ("prep + factors + tcgen05 GEMM (+ split reduction) + quantize8"
                            if args.form.startswith("gemm") else
                            "prep + direct kernel (equal shares of the (tile, point) pairs, each tile's parts "
                            "summed in the kernel) + quantize8" if args.form == "direct_sfu" else
                            "prep + direct kernel (+ chunk reduction) + quantize8"),
                   "l2": "flushed between timed steps (256 MiB write, untimed)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "holograms_per_s": args.steps * world / (total_ms * 1e-3),
        "nrms_vs_oracle": nrms,
        "nrms_sample": "the cpu_baseline rows" if nrms is not None else None,
        "gpu_launches": launches,
        "kernel_ms": {k: v[1] / max(v[0], 1) for k, v in prof.items()},
        "roofline": {"kernel": dom, "bound": roof["bound"], "achieved": achieved, "peak": peak,
                     "unit": roof["unit"], "frac": (achieved / peak) if achieved else None,
                     "traffic": traffic, "peak_basis": roof["peak_basis"],
                     **({"peak_probe": roof["peak_probe"], "frac_of_probe": roof["frac_of_probe"]}
                        if "peak_probe" in roof else {})},
        "clocks": clocks,
        "e2e": {"value": cloud.evals * args.steps * world / e2e_total / 1e9, "unit": UNIT,
                "h2d_bytes_per_step": int(cloud.xyz.nbytes + cloud.amp.nbytes),
                "d2h_bytes_per_step": int(W * H * 4),
                "path": "cgh_point_cloud_host (pinned host buffers, copies and sync inside)"},
        "forms": forms,
        "paper_kinoform_1920x1080": paper,
        "layered_4096x4096_n1000000": large,
        "video_batch_64": vbatch,
        "paper_fresnel_diffraction": fresnel_t,
        "paper_wrp_2048x2048": wrp_t,
        "cpu_baseline": cpu,
        "summary": compact_summary(forms, large, vbatch, cloud.name),
    }
    assert line["config"]["n_points"] == cloud.n_points and line["config"]["workload"] == cloud.name
    print(json.dumps(line))
    h.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_layout_sweep(args):
    """Every GEMM launch shape (orientation, tile width, K splits, one-CTA or two-SM form) timed on a few hologram
    shapes, against the one cgh_gemm_layout picks: the evidence behind the layout model.  Prints one JSON line."""
    import torch
    from paper_1309_2734_gb300 import Hologram, workloads, _lib
    from paper_1309_2734_gb300.build import build
    build()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    shapes = [tuple(int(v) for v in t.split("x")) for t in args.layout_sweep.split(",")]
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    result = {"sweep": "gemm layouts", "form": args.form, "unit": "ms (GEMM kernel + split reduction, CUDA events)",
              "shapes": {}}

    def timed(hg, xyz, amp, out):
        hg.point_cloud(xyz, amp, out)
        hg.sync()
        hg.profile(True)
        hg.profile_read(reset=True)
        for _ in range(3):
            hg.point_cloud(xyz, amp, out)
        hg.sync()
        kp = hg.profile_read(reset=True)
        hg.profile(False)
        return (kp["gemm_tcgen05"][1] + kp.get("reduce_slices", (0, 0.0))[1]) / 3

    for (w, h, n) in shapes:
        c = workloads.random_cloud(777 + n, w, h, n)
        xyz, amp = torch.from_numpy(c.xyz).cuda(), torch.from_numpy(c.amp).cuda()
        out = torch.empty((h, w), device="cuda")
        kb = (2 * n + 63) // 64
        rows = []
        with Hologram(w, h, c.pitch_m, c.lambda_m, form=args.form, stream=stream) as hg:
            hg.set_option(_lib.CGH_OPT_GEMM_GROUP, 1)
            for pair in (2, 1):
                for tr in (1, 2):
                    for bn in (128, 192, 224, 240, 256):
                        for sp in range(1, 17):
                            if sp * 4 > kb or (pair == 1 and bn == 240):
                                continue
                            for key, v in ((_lib.CGH_OPT_GEMM_PAIR, pair), (_lib.CGH_OPT_GEMM_TRANSPOSE, tr),
                                           (_lib.CGH_OPT_GEMM_BN, bn), (_lib.CGH_OPT_GEMM_SPLITK, sp)):
                                hg.set_option(key, v)
                            rows.append(((pair == 1, tr == 2, bn, sp), timed(hg, xyz, amp, out)))
            for key in (_lib.CGH_OPT_GEMM_PAIR, _lib.CGH_OPT_GEMM_TRANSPOSE, _lib.CGH_OPT_GEMM_BN,
                        _lib.CGH_OPT_GEMM_SPLITK):
                hg.set_option(key, 0)
            auto_ms = timed(hg, xyz, amp, out)
        lay = _lib.cgh_gemm_layout(w, h, n, _lib.FORMS[args.form], sms)
        best = min(rows, key=lambda r: r[1])
        same = [t for k, t in rows if k == (lay["pair"], lay["transposed"], lay["bn"], lay["splits"])]
        result["shapes"][f"{w}x{h}-n{n}"] = {
            "layouts_timed": len(rows),
            "best": {"pair": best[0][0], "transposed": best[0][1], "bn": best[0][2], "splits": best[0][3],
                     "ms": round(best[1], 4)},
            "chosen": dict(lay, ms=round(auto_ms, 4), ms_in_sweep=round(same[0], 4) if same else None),
            "chosen_over_best": round((same[0] if same else auto_ms) / best[1], 3)}
        print(json.dumps({f"{w}x{h}-n{n}": result["shapes"][f"{w}x{h}-n{n}"]}), file=sys.stderr, flush=True)
    print(json.dumps(result))
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", default="direct-1920x1080-n10000")
    ap.add_argument("--form", default="direct_sfu")
    ap.add_argument("--compare", nargs="*",
                    default=["direct_accurate", "gemm_f16", "gemm_bf16", "gemm_split16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-frame batched workload")
    ap.add_argument("--batch-frames", default="",
                    help="comma-separated indices of the video batch's frames to run instead of all 64")
    ap.add_argument("--batch-tols", default="1e-5,2e-3", help="NRMS classes at which the batch is timed")
    ap.add_argument("--no-fresnel", action="store_true",
                    help="skip the Fresnel diffraction and wavefront-recording workloads of Tables 5-6")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the 4096x4096, 10^6-point depth-layered case")
    ap.add_argument("--no-small", action="store_true", help="skip the 256x256, 1,024-point cloud")
    ap.add_argument("--no-paper-workload", action="store_true",
                    help="skip the phase-only 1920x1080 workload of the paper's Tables 3-4")
    ap.add_argument("--layout-sweep", default="",
                    help="instead of the bench line: time every GEMM launch shape of --form on these hologram "
                         "shapes (WxHxN,...) against the chosen one")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.layout_sweep:
        return run_layout_sweep(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
