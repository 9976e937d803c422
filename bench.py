#!/usr/bin/env python3
"""Benchmark of the surfel rendering hot path on GB300.

Workload (the configuration the headline metric is quoted on): 3M surfels on a
synthetic 60 m street (ground + two facades), a 32-frame trajectory of
1920x1080 pinhole views (f=960, y from 5 m to 55 m), D=128 features stored in
BF16, Top-K Hard Selection with K=8, EXACT ellipse-vs-tile binning, Q=100 BF16
queries. One step = one frame through every step of the path: project,
intersect, sort, Top-K render, tensor-core decode, and the hand-written
adjoint with seeded N(0,1) upstream gradients. Each stage of each frame is a
captured CUDA graph; frames are timed with CUDA events on the launching
stream. The plain FP32 form (SPHERE bounds, dense FP32 features) is measured
beside it, and the CPU oracle on a bounded pixel sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl psi|reference]

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "frames/s at 1080p, 3M surfels, D=128 (fwd; fwd+bwd ms) vs plain FP32, 1×GB300"
PAPER_CONTEXT = ("Table 3 of the paper: Full Method 22 ms / 45 FPS, Baseline 46 ms / 22 FPS, on an RTX A6000, "
                 "resolution / surfel count / D / K not stated (different hardware and data: context only)")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=256)
    ap.add_argument("--warmup", type=int, default=4)
    ap.add_argument("--impl", default="psi", choices=["psi", "reference"])
    ap.add_argument("--surfels", type=int, default=3_000_000)
    ap.add_argument("--frames", type=int, default=32)
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="keep the default launch shapes (no autotuning)")
    ap.add_argument("--plain-steps", type=int, default=6)
    ap.add_argument("--ablation-frames", type=int, default=6, help="frames per Table-3 row (0: skip)")
    ap.add_argument("--label-frames", type=int, default=8, help="frames of the instance-label path (0: skip)")
    ap.add_argument("--e2e-steps", type=int, default=64)
    ap.add_argument("--batch-reps", type=int, default=10, help="replays of the 16-view batch graph (0: skip)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- helpers
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def frame_index(k: int, rank: int, n_frames: int) -> int:
    """Frame of the trajectory that rank `rank` renders at step k. Weak
    scaling: every rank renders its own K frames (no data-path collective:
    frames are independent given the replicated scene), ranks start at
    different points of the trajectory."""
    return (k + rank * 7) % n_frames


def max_over_ranks(value: float, world: int, device=None) -> float:
    """Max of a per-rank timing over all ranks (the job's time)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(steps_per_rank: int, world: int, max_ms: float) -> float:
    """Units all ranks processed divided by the slowest rank's time."""
    return world * steps_per_rank / (max_ms / 1000.0)


def roofline_traffic(kernel: str, pairs: float, view: str):
    """DRAM bytes (read + write) of one launch of `kernel` on a frame with
    `pairs` (tile, surfel) pairs, from the committed small-case ncu captures
    (profiles/roofline_traffic.json): one launch captured at two surfel counts
    of the same view gives a line, bytes = fixed + per_pair x pairs (the
    per-pixel buffers make the fixed part, the records and list entries the
    part that grows with the pairs), evaluated at this frame's pair count.
    Returns (bytes, note), or (None, reason) unless the captures were taken on
    the current sources of that kernel (its .cu file and the headers it
    includes, hashed together in the listed order) and on a view of this size."""
    path = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    try:
        d = json.load(open(path))
    except (OSError, ValueError):
        return None, "no committed captures"
    e = d.get(kernel)
    if not e:
        return None, f"no capture of {kernel}"
    h = hashlib.sha256()
    try:
        for name in e["sources"]:
            h.update(open(os.path.join(ROOT, "paper_2604_10982_gb300", "csrc", name), "rb").read())
    except (OSError, KeyError):
        return None, "sources missing"
    if h.hexdigest()[:16] != e.get("sha256_16"):
        return None, f"{kernel} changed since its capture"
    if e.get("view") != view:
        return None, f"captured on a {e.get('view')} view"
    (p1, b1), (p2, b2) = [(pt["pairs"], pt["dram_read"] + pt["dram_write"]) for pt in e["points"][:2]]
    per_pair = (b2 - b1) / (p2 - p1)
    fixed = b1 - per_pair * p1
    return fixed + per_pair * pairs, (f"ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch at "
                                      f"{p1} and {p2} pairs ({e['view']}), fixed {fixed / 1e6:.1f} MB + "
                                      f"{per_pair:.1f} B per pair at this frame's {pairs:.0f} pairs")


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# ---------------------------------------------------------------- CPU oracle
def oracle_frame_sample(w, cam, q_bf16_deq, Qm, gC_fn, target_s, opts_kw, max_pixels=4096):
    """Time the CPU oracle on one frame: the per-frame setup (binning of all
    surfels, canonical order) plus a pixel sample of the per-pixel work
    (forward, gradient, decode), extrapolated to the whole frame."""
    from oracle import oracle as orc
    o = orc.Opts(**opts_kw)
    t0 = time.perf_counter()
    b = orc.bin_view(w.surfels, cam, o)
    orc.canonical_order(b)
    t_fixed = time.perf_counter() - t0
    P = cam.width * cam.height
    rng = np.random.default_rng(0)
    n_pix = 8
    t_pix = None
    while True:
        pix = orc.all_pixels(cam)[rng.choice(P, n_pix, replace=False)]
        t1 = time.perf_counter()
        out = orc.render(w.surfels, cam, o, feat=q_bf16_deq, pixels=pix, b=b)
        gC, gF, gT = gC_fn(n_pix)
        orc.render_grad(w.surfels, cam, o, gC, feat=q_bf16_deq, gF=gF, gT=gT, pixels=pix, b=b)
        orc.decode(out["F"], Qm, out["T"])
        dt = time.perf_counter() - t1
        t_pix = dt / n_pix
        if dt >= 0.25 * target_s or n_pix >= max_pixels:
            break
        n_pix = min(max_pixels, max(n_pix * 2, int(n_pix * 0.5 * target_s / max(dt, 1e-3))))
    frame_s = t_fixed + t_pix * P
    return dict(frame_s=frame_s, t_fixed=t_fixed, t_pix=t_pix, sample_pixels=n_pix,
                threads=orc.num_threads(), out=out, pixels=pix)


def parity_of_sample(out, pix, cam, rgb, T, F, topk):
    """The GPU frame against the oracle's forward on the CPU leg's pixel sample:
    pixels whose result is fixed to float32 rounding (no threshold straddle,
    well conditioned) must match colour and T to 1e-4, the BF16 feature map to
    2e-2 relative and the Top-K id set exactly (except near ties); the excused
    shares and the largest error over them are reported."""
    W = cam.width
    p = pix[:, 1].astype(np.int64) * W + pix[:, 0].astype(np.int64)
    d = out["diag"]
    dp = 2.0 ** -24 * max(cam.width, cam.height)
    straddle = (d[:, 0] < 1e-5) | (d[:, 1] < 1e-5) | (d[:, 2] < 1e-5)
    ill = (d[:, 4] * dp > 1e-4) & ~straddle
    near = d[:, 3] < 1e-6
    strict = ~(straddle | ill)
    e = np.maximum(np.abs(rgb[:, p].T - out["rgb"]).max(1), np.abs(T[p] - out["T"]))
    relF = np.abs(F[p] - out["F"]).max(1) / (np.abs(out["F"]).max(1) + 1e-3)
    same = np.array([set(topk[q][topk[q] >= 0].tolist()) == set(out["topk"][i][out["topk"][i] >= 0].tolist())
                     for i, q in enumerate(p)])
    ok = strict & ~near
    return {"frame": 0, "pixels": int(len(p)),
            "excused_share": {"straddle": float(straddle.mean()), "ill_conditioned": float(ill.mean()),
                              "near_tie": float(near.mean())},
            "max_abs_err_strict": float(e[strict].max(initial=0)),
            "max_abs_err_excused": float(e[~strict].max(initial=0)),
            "max_rel_err_F_bf16_strict": float(relF[ok].max(initial=0)),
            "topk_set_mismatch_strict": int((ok & ~same).sum()),
            "topk_set_mismatch_excused": int((~ok & ~same).sum()),
            "pass": bool(e[strict].max(initial=0) < 1e-4 and relF[ok].max(initial=0) < 2e-2 and
                         (ok & ~same).sum() == 0),
            "bars": "strict pixels: |rgb|,|T| err < 1e-4, BF16 F rel err < 2e-2, Top-K sets equal (near ties "
                    "excused); straddles: a surfel within 1e-5 of a threshold; ill-conditioned: 1 ulp of the pixel "
                    "position moves the value by > 1e-4"}


def run_reference(args):
    """The oracle, timed on the host cores, as the reference arm."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_2604_10982_gb300 import scenegen as sg
    w = sg.panoptic_scene(n=args.surfels, frames=args.frames, with_features=True)
    deq = bf16_round(w.features).astype(np.float64)
    Qm = bf16_round(w.queries).astype(np.float64)
    D = w.features.shape[1]
    gfn = lambda n: (sg.make_upstream(3 * n, 3, 0).reshape(n, 3), sg.make_upstream(D * n, 3, 1).reshape(n, D),
                     sg.make_upstream(n, 3, 2))
    kw = dict(mode=2, top_k=8, opacity_radius=True)
    times = []
    info = None
    for k in range(args.warmup + args.steps):
        cam = w.cameras[k % len(w.cameras)]
        info = oracle_frame_sample(w, cam, deq, Qm, gfn, args.cpu_seconds / max(args.steps + args.warmup, 1), kw,
                                   max_pixels=64)
        if k >= args.warmup:
            times.append(info["frame_s"])
    fps = 1.0 / float(np.mean(times))
    line = {"impl": "reference", "metric": METRIC, "value": fps, "unit": "frames/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / fps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args, graph=False),
            "cpu_baseline": {"value": fps, "unit": "frames/s", "cores": info["threads"], "kind": "oracle",
                             "sample": f"per step: binning of all {args.surfels} surfels + forward, gradient and "
                                       f"decode of {info['sample_pixels']} random pixels of one 1920x1080 frame, "
                                       f"extrapolated to the frame's {1920 * 1080} pixels"},
            "e2e": {"value": fps, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round float32 to the nearest BF16 value (ties to even), as float32."""
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def workload_config(args, graph=True):
    return {"workload": f"panoptic street: {args.surfels} surfels, {args.frames}-frame trajectory of 1920x1080 views "
                        f"(f=960), D=128 BF16 features, Top-K K=8, EXACT tiles, Q=100 BF16 queries",
            "surfels": args.surfels, "resolution": "1920x1080", "feat_dim": 128, "feat_storage": "bf16",
            "top_k": 8, "queries": 100, "isect": "exact+opacity-radius", "frames": args.frames,
            "step": "project+intersect+sort+render+decode+backward (with gradient zeroing) of one frame",
            "streams": "forward and adjoint on one stream; gradient zeroing and decode on a second, overlapped",
            "cuda_graph": graph,
            "l2": "inputs larger than L2 (surfels 180 MB + BF16 features 768 MB read per frame; 129 MB L2)"}


# ---------------------------------------------------------------- main arm
def run_psi(args):
    import torch

    from paper_2604_10982_gb300 import pipeline as pl, psi, scenegen as sg

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    t_setup = time.time()
    w = sg.panoptic_scene(n=args.surfels, frames=args.frames, with_features=True)
    cams = w.cameras
    D, K, nq = 128, 8, 100
    ctx = psi.Context(local)
    scene = pl.DeviceScene(w.surfels, w.features, feat_dtype=psi.BF16, device=dev)
    Qd = torch.from_numpy(w.queries).to(dev).to(torch.bfloat16).contiguous()
    P = cams[0].width * cams[0].height
    gC_h = torch.from_numpy(sg.make_upstream(3 * P, 3, 0).reshape(3, P)).pin_memory()
    gF_h = torch.from_numpy(sg.make_upstream(D * P, 3, 1).reshape(P, D)).pin_memory()
    gT_h = torch.from_numpy(sg.make_upstream(P, 3, 2)).pin_memory()
    gC, gF, gT = gC_h.to(dev), gF_h.to(dev), gT_h.to(dev)

    opts = psi.default_opts(mode=psi.EXACT, top_k=K, opacity_radius=1)
    grads = dict(mu=torch.zeros(scene.n, 3, device=dev), tu=torch.zeros(scene.n, 3, device=dev),
                 tv=torch.zeros(scene.n, 3, device=dev), scale=torch.zeros(scene.n, 2, device=dev),
                 opacity=torch.zeros(scene.n, device=dev), rgb=torch.zeros(scene.n, 3, device=dev),
                 feat=torch.zeros(scene.n, D, device=dev))
    grads_struct = psi.PsiGrads(*(psi._ptr(grads[k]) for k in ("mu", "tu", "tv", "scale", "opacity", "rgb", "feat")))
    # the tile shape (16x16 or 16x8) of the autotuner: a whole frame with each, on frame 0
    tile_ms = None
    if not args.no_tune:
        opts, tile_ms = pl.tune_tile_height(ctx, scene, [cams[0]], opts, D=D, F_dtype=psi.BF16, g_rgb=gC, g_F=gF,
                                            g_T=gT, grads=grads)
        torch.cuda.synchronize()
    r = pl.Renderer(ctx, scene.n, [cams[0]], opts, 1024, D=D, F_dtype=psi.BF16, device=dev)
    need = 0
    for c in cams:
        r.set_cameras([c])
        need = max(need, r.required_pairs(scene))
    r.set_capacity(int(need * 1.15) + 1024)
    ids = torch.empty(r.n_pix, dtype=torch.int32, device=dev)

    def stage_fns(f):
        def proj():
            r.set_cameras([cams[f]])
            r.project(scene)

        def isect():
            r.set_cameras([cams[f]])
            r.intersect()

        def srt():
            r.sort()

        def rend():
            r.set_cameras([cams[f]])
            r.render(scene)

        def dec():
            psi.psi_decode_queries(ctx, r.F, r.n_pix, D, Qd, nq, r.T, ids)

        def zero():
            psi.psi_grads_zero(ctx, grads_struct, scene.n, D)

        def bwd():
            r.set_cameras([cams[f]])
            r.backward(scene, gC, gF, gT, grads=grads)

        return [proj, isect, srt, rend, dec, zero, bwd]

    names = ["project", "intersect", "sort", "render_fwd", "decode", "zero_grads", "render_bwd"]
    # the adjoint call launches three kernels (features, list walk, chain); it
    # runs eagerly so that the library can bracket its kernels with the
    # per-step timing events below (a graph replay cannot record them)
    EAGER = {"render_bwd"}
    # warm every code path once (lazy buffers, function attributes), let the
    # library pick the compositing kernels' launch shapes on frame 0, then
    # capture (the graphs keep the tuned shapes)
    for fn in stage_fns(0):
        fn()
    torch.cuda.synchronize()
    tuned = None
    if not args.no_tune:
        tr = r.tune(scene, gC, gF, gT, grads=grads, reps=3)
        tuned = {"tile": f"16x{int(opts.tile_h)}", "frame_ms_per_tile_height": tile_ms,
                 "forward": {"ms_per_shape": [round(x, 4) for x in tr["fwd"][0]], "shape": tr["fwd"][1]},
                 "adjoint": {"ms_per_shape": [round(x, 4) for x in tr["bwd"][0]], "shape": tr["bwd"][1]},
                 "shapes": "bit 0: the other CTAs-per-SM build (K<=8: forward 3->4, adjoint from saved state 4->3, else 2->1); "
                           "bit 1: dense 16-channel passes; bit 2: persistent launch (tile counter); bit 3: adjoint "
                           "walk with two pixels per lane instead of one (saved state, K>0); -1: shape does not apply; "
                           "tile height and shapes timed on frame 0 before the graphs are captured"}
    torch.cuda.synchronize()
    use_graph = not args.no_graph
    graphs = None
    if use_graph:
        cap_stream = torch.cuda.Stream(device=dev)
        graphs = []
        for f in range(len(cams)):
            gs = []
            for name, fn in zip(names, stage_fns(f)):
                if name in EAGER:
                    gs.append(None)
                    continue
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=cap_stream, capture_error_mode="relaxed"):
                    fn()
                gs.append(g)
            graphs.append(gs)
        torch.cuda.synchronize()

    # Two streams: the forward and the adjoint run in order on the main
    # stream; gradient zeroing (needs nothing of the frame; started beside
    # the forward compositing) and the decode (reads only forward outputs, as
    # the adjoint does) run on a side stream and overlap them. The frame ends
    # when both streams are done.
    main_s = torch.cuda.current_stream(dev)
    side = torch.cuda.Stream(device=dev)
    zero_done = torch.cuda.Event()
    STAGE = {n: i for i, n in enumerate(names)}

    def run_stage(f, n, fns):
        i = STAGE[n]
        if use_graph and graphs[f][i] is not None:
            graphs[f][i].replay()
        else:
            fns[i]()

    def run_frame(f, evs=None, kev=None, before_bwd=None):
        """evs: per-stage events (dict) or None; kev: the adjoint's kernel events;
        before_bwd: called just before the adjoint (the end-to-end loop waits
        there for the frame's upstream gradients, which only the adjoint reads)."""
        fns = stage_fns(f)
        rec = (lambda name, s: evs[name].record(s)) if evs is not None else (lambda name, s: None)
        rec("start", main_s)
        for n in ("project", "intersect", "sort"):
            run_stage(f, n, fns)
            rec(n, main_s)
        # the zeroing (1.7 GB of gradient buffers) overlaps the compositing,
        # which is issue-bound, rather than the HBM-bound binning and sort
        side.wait_stream(main_s)  # also: the previous frame's adjoint is done with the gradients
        with torch.cuda.stream(side):
            rec("zero0", side)
            run_stage(f, "zero_grads", fns)
            rec("zero1", side)
            zero_done.record(side)
        run_stage(f, "render_fwd", fns)
        rec("render_fwd", main_s)
        side.wait_stream(main_s)  # decode after the forward
        with torch.cuda.stream(side):
            rec("dec0", side)
            run_stage(f, "decode", fns)
            rec("dec1", side)
        main_s.wait_event(zero_done)
        if before_bwd is not None:
            before_bwd()
        if kev is not None:
            psi.psi_ctx_time_kernel(ctx, psi.KERNEL_BWD_FEAT, kev[0], kev[1])
            psi.psi_ctx_time_kernel(ctx, psi.KERNEL_BWD_WALK, kev[2], kev[3])
        run_stage(f, "render_bwd", fns)
        rec("bwd", main_s)
        main_s.wait_stream(side)
        rec("end", main_s)

    def fidx(k):
        return frame_index(k, rank, len(cams))

    for k in range(args.warmup):
        run_frame(fidx(k))
    torch.cuda.synchronize()
    st, req = ctx.status_fetch()
    assert st == 0, f"device status {st} (required pairs {req})"
    setup_s = time.time() - t_setup

    # ---- timed region
    EV = ("start", "zero0", "zero1", "project", "intersect", "sort", "render_fwd", "dec0", "dec1", "bwd", "end")
    evs = [{e: torch.cuda.Event(enable_timing=True) for e in EV} for _ in range(args.steps)]
    # per-step events around the adjoint's feature kernel and list walk
    kevs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    for kv in kevs:
        for e in kv:
            e.record()  # creates the CUDA event the library records into
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    t_start.record()
    for k in range(args.steps):
        run_frame(fidx(k), evs[k], kevs[k])
    t_end.record()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    def stage_times(e):
        return [e["start"].elapsed_time(e["project"]), e["project"].elapsed_time(e["intersect"]),
                e["intersect"].elapsed_time(e["sort"]), e["sort"].elapsed_time(e["render_fwd"]),
                e["dec0"].elapsed_time(e["dec1"]), e["zero0"].elapsed_time(e["zero1"]),
                e["render_fwd"].elapsed_time(e["bwd"])]
    stage = np.array([stage_times(evs[k]) for k in range(args.steps)])  # columns in `names` order
    frame_wall = np.array([evs[k]["start"].elapsed_time(evs[k]["end"]) for k in range(args.steps)])
    st, req = ctx.status_fetch()
    assert st == 0, f"device status {st}"
    total_ms = max_over_ranks(total_ms, world, dev)
    kern = np.array([[kevs[k][0].elapsed_time(kevs[k][1]), kevs[k][2].elapsed_time(kevs[k][3])]
                     for k in range(args.steps)])
    frame_ms = frame_wall  # both streams, overlapped
    fwd_ms = stage[:, :5].sum(1)  # a1-a4 + decode run one after another
    value = job_throughput(args.steps, world, total_ms)

    # ---- the forward alone (a1-a4 and the decode in order on one stream, as
    # an inference-only caller runs it), timed over the same frames
    fwd_loop = max(8, min(args.steps, 64))
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(main_s)
    for k in range(fwd_loop):
        fns = stage_fns(fidx(k))
        for n in ("project", "intersect", "sort", "render_fwd", "decode"):
            run_stage(fidx(k), n, fns)
    f1.record(main_s)
    torch.cuda.synchronize()
    fwd_only_ms = f0.elapsed_time(f1) / fwd_loop

    # ---- per-frame statistics (outside the timed region)
    pairs, nlast_sum, nonempty, uniq_sel = [], [], [], []
    for f in sorted(set(fidx(k) for k in range(args.steps))):
        run_frame(f)
        torch.cuda.synchronize()
        pairs.append(int(r.num_pairs.item()))
        nlast_sum.append(float(r.n_last.to(torch.float64).sum().item()))
        nonempty.append(int(((1.0 - r.T) >= 1e-4).sum().item()))
        ids_sel = r.topk_ids.reshape(-1)
        uniq_sel.append(int(torch.unique(ids_sel[ids_sel >= 0]).numel()))
    n_tiles = r.n_tiles

    # ---- roofline of the dominant kernel
    mean_stage = stage.mean(0)
    # the feature kernel: the register-resident form for K <= 8 and D <= 128
    feat_name = "feat_bwd_reg_kernel" if (K <= 8 and D <= 128) else "feat_bwd_kernel"
    # the list walk's kernel: the paired form if the tuned adjoint shape has bit 3
    walk_name = ("render_bwd_pair_kernel" if psi.psi_ctx_get_render_shape(ctx, 1, r.opts, psi.BF16, 1) & 8
                 else "render_bwd_kernel")
    kernel_ms = {"render_fwd_kernel": float(mean_stage[names.index("render_fwd")]),
                 "decode_kernel": float(mean_stage[names.index("decode")]),
                 feat_name: float(kern[:, 0].mean()),
                 walk_name: float(kern[:, 1].mean())}
    dom = max(kernel_ms, key=kernel_ms.get)
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = n_sm * 128 * 2 * sm_max * 1e6 / 1e12  # TFLOP/s: SMs x FP32 lanes x FMA x clock
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    launch_s = kernel_ms[dom] / 1000.0
    if dom == "render_fwd_kernel":
        flop = 20.0 * np.mean(nlast_sum) + 2.0 * K * D * np.mean(nonempty)
        roof = {"bound": "alu", "achieved": flop / launch_s / 1e12, "peak": fp32_peak, "unit": "TFLOP/s",
                "work": "20 FP32 flop per (pixel, list entry up to its last composited surfel) + 2KD per pixel"}
    elif dom == walk_name:
        flop = 40.0 * np.mean(nlast_sum)
        roof = {"bound": "alu", "achieved": flop / launch_s / 1e12, "peak": fp32_peak, "unit": "TFLOP/s",
                "work": "40 FP32 flop per (pixel, list entry up to its last composited surfel): twice the "
                        "forward's 20 (the adjoint of the alpha evaluation and blend)"}
    elif dom == feat_name:
        byts = r.n_pix * (4.0 * D + 12.0 * K) + np.mean(uniq_sel) * (2.0 * D + 8.0 * D)
        roof = {"bound": "hbm", "achieved": byts / launch_s / 1e9, "peak": hbm_peak, "unit": "GB/s",
                "work": "per pixel gF row + K ids, weights, dots; per selected surfel its BF16 row and dL/df row read+write"}
    else:
        byts = r.n_pix * (2.0 * D + 8.0)
        roof = {"bound": "hbm", "achieved": byts / launch_s / 1e9, "peak": hbm_peak, "unit": "GB/s",
                "work": "per pixel its BF16 feature row, T and id"}
    roof = {"kernel": dom, **roof}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["peak_source"] = ("measured HBM copy bandwidth (MEASURED_PEAKS.json)" if roof["bound"] == "hbm" else
                           f"derived: {n_sm} SMs (device) x 128 FP32 lanes x 2 flop x {sm_max:.0f} MHz")
    roof["traffic"], roof["traffic_source"] = roofline_traffic(dom, float(np.mean(pairs)),
                                                              f"{cams[0].width}x{cams[0].height}")
    roof["launch_ms"] = kernel_ms[dom]

    # ---- end to end through the public API with host buffers: each step's
    # upstream gradients come from pinned host memory (double-buffered on the
    # device, copied on a side stream while the previous step computes), ids
    # and RGB go back to pinned host memory after the step
    e2e = None
    if args.e2e_steps > 0:
        ids_h = torch.empty(r.n_pix, dtype=torch.int32).pin_memory()
        rgb_h = torch.empty(3, r.n_pix, dtype=torch.float32).pin_memory()
        main = torch.cuda.current_stream(dev)
        copy_stream = torch.cuda.Stream(device=dev)
        # three device buffers, copies issued two steps ahead: the copy stream
        # never waits for the step that is still reading the previous buffer
        NB = 3
        bufs = [(gC, gF, gT)] + [(torch.empty_like(gC), torch.empty_like(gF), torch.empty_like(gT))
                                 for _ in range(NB - 1)]
        ev_ready = [torch.cuda.Event() for _ in range(NB)]
        ev_used = [torch.cuda.Event() for _ in range(NB)]

        def h2d(k):
            b = k % NB
            if k >= NB:
                copy_stream.wait_event(ev_used[b])  # step k-NB is done with this buffer
            with torch.cuda.stream(copy_stream):
                for dst, src in zip(bufs[b], (gC_h, gF_h, gT_h)):
                    dst.copy_(src, non_blocking=True)
                ev_ready[b].record(copy_stream)

        # the copy alone, for reference (outside the timed region; the first
        # copies from freshly pinned pages are slower and are not the ones timed)
        h2d(0)
        h2d(1)
        torch.cuda.synchronize()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(copy_stream)
        h2d(0)
        c1.record(copy_stream)
        torch.cuda.synchronize()
        h2d_ms = c0.elapsed_time(c1)

        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        e0.record(main)
        copy_stream.wait_event(e0)
        h2d(0)
        if args.e2e_steps > 1:
            h2d(1)
        for k in range(args.e2e_steps):
            b = k % NB
            if k + 2 < args.e2e_steps:
                h2d(k + 2)
            gC, gF, gT = bufs[b]  # the adjoint stage reads these names
            run_frame(fidx(k), before_bwd=lambda ev=ev_ready[b]: main.wait_event(ev))
            ev_used[b].record(main)
            ids_h.copy_(ids, non_blocking=True)
            rgb_h.copy_(r.rgb, non_blocking=True)
        e1.record(main)
        torch.cuda.synchronize()
        gC, gF, gT = bufs[0]
        e2e_ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
        e2e = {"value": job_throughput(args.e2e_steps, world, e2e_ms), "unit": "frames/s",
               "h2d_bytes_per_step": int(gC_h.numel() * 4 + gF_h.numel() * 4 + gT_h.numel() * 4),
               "d2h_bytes_per_step": int(ids_h.numel() * 4 + rgb_h.numel() * 4),
               "h2d_ms_per_step": float(h2d_ms), "steps": int(args.e2e_steps),
               "what": "per step: upstream gradients copied from pinned host memory (side stream, three device "
                       "buffers, issued two steps ahead; the frame waits for them before its adjoint), the frame (all "
                       "stages), ids and RGB read back to pinned host memory"}

    # ---- plain FP32 form (paper's Baseline row): SPHERE bounds, dense FP32 features
    plain = None
    if args.plain_steps > 0:
        del graphs
        torch.cuda.empty_cache()
        scene32 = pl.DeviceScene(w.surfels, w.features, feat_dtype=psi.F32, device=dev)
        po = psi.default_opts(mode=psi.SPHERE, top_k=0, opacity_radius=0)
        rp = pl.Renderer(ctx, scene.n, [cams[0]], po, 1024, D=D, F_dtype=psi.F32, device=dev)
        need = 0
        for f in range(min(args.plain_steps + 1, len(cams))):
            rp.set_cameras([cams[fidx(f)]])
            need = max(need, rp.required_pairs(scene32))
        rp.set_capacity(int(need * 1.15) + 1024)
        pt = []
        for k in range(args.plain_steps + 1):
            f = fidx(k)
            rp.set_cameras([cams[f]])
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record()
            rp.frame(scene32)
            e[1].record()
            psi.psi_grads_zero(ctx, grads_struct, scene.n, D)
            rp.backward(scene32, gC, gF, gT, grads=grads)
            e[2].record()
            torch.cuda.synchronize()
            if k > 0:
                pt.append((e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2]), int(rp.num_pairs.item())))
        pt = np.array(pt)
        plain = {"fwd_ms": float(np.median(pt[:, 0])), "fwd_bwd_ms": float(np.median(pt[:, 0] + pt[:, 1])),
                 "fwd_frames_per_s": float(1000.0 / np.median(pt[:, 0])),
                 "frames_per_s": float(1000.0 / np.median(pt[:, 0] + pt[:, 1])),
                 "statistic": "median over frames after one warm-up frame",
                 "pairs_per_frame": float(pt[:, 2].mean()), "frames": int(len(pt)),
                 "form": "SPHERE tiles, dense FP32 features (no Top-K), single view per launch, no graph, no decode"}
        del scene32, rp

    # ---- tables rendered like features (once per map, then per frame):
    # instance labels (Sec. 4.1, Eqs. 4-8) and the plain query logits (the
    # decode fused into compositing by linearity); per frame the table is
    # composited with Top-K and the fused per-pixel argmax, no feature map
    labels = None
    if args.label_frames > 0:
        q_mu, q_cov = sg.make_query_gaussians(nq, 9, (-8, 0, 0), (8, 60, 12))
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        for rep in range(2):  # the second pass is timed
            ev[0].record()
            Lt = pl.surfel_labels(ctx, scene, Qd, q_mu, q_cov, dtype=psi.BF16)
            ev[1].record()
            Gt = pl.surfel_logits(ctx, scene, Qd, dtype=psi.BF16)
            ev[2].record()
            torch.cuda.synchronize()
        lab_ms, logit_ms = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
        out = {}
        for name, table in (("labels", Lt), ("decode_fused", Gt)):
            ts = pl.label_scene(scene, table)
            rl = pl.Renderer(ctx, scene.n, [cams[0]], opts, r.capacity, D=ts.D, F_dtype=psi.BF16, device=dev)
            rt, ft = [], []
            for k in range(args.label_frames + 1):
                rl.set_cameras([cams[fidx(k)]])
                ev[0].record()
                rl.project(ts)
                rl.intersect()
                rl.sort()
                ev[1].record()
                rl.render(ts, want_F=False, argmax=True)
                ev[2].record()
                torch.cuda.synchronize()
                if k > 0:
                    rt.append(ev[1].elapsed_time(ev[2]))
                    ft.append(ev[0].elapsed_time(ev[2]))
            out[name] = {"render_ms": float(np.median(rt)), "frame_ms": float(np.median(ft)),
                         "table": f"[{scene.n}, {ts.D}] BF16"}
            del rl, ts
        # the unfused forward on the same frames, timed the same way: the
        # feature map composited and written, then the tensor-core decode
        ut = []
        for k in range(args.label_frames + 1):
            r.set_cameras([cams[fidx(k)]])
            r.project(scene)
            r.intersect()
            r.sort()
            ev[1].record()
            r.render(scene)
            psi.psi_decode_queries(ctx, r.F, r.n_pix, D, Qd, nq, r.T, ids)
            ev[2].record()
            torch.cuda.synchronize()
            if k > 0:
                ut.append(ev[1].elapsed_time(ev[2]))
        out["unfused_render_plus_decode_ms"] = float(np.median(ut))
        st, _ = ctx.status_fetch()
        assert st == 0, f"device status {st}"
        lab_bytes = scene.n * (2.0 * D + 12.0 + 2.0 * Lt.shape[1])  # features + centres read, table written
        labels = {"labels_table_ms": float(lab_ms), "logits_table_ms": float(logit_ms), "queries": nq,
                  "labels_table_hbm_frac": lab_bytes / (lab_ms / 1000.0) / 1e9 / float(peaks.get("hbm_gbs", 6800.0)),
                  **out,
                  "form": "tables once per map on the tensor cores (labels: sigmoid x query-Gaussian density ratio, "
                          "softmax; logits: f_q^T f_g); per frame: project+intersect+sort (eager) and the compositing "
                          "of the table (K=8, EXACT) with the fused per-pixel argmax (render_ms)"}
        del Lt, Gt

    # ---- geometric and anisotropy regularisers (Sec. 4.2) over all surfels,
    # against 4096 synthetic planar priors (every surfel assigned)
    regs = None
    if args.label_frames > 0:
        rng = np.random.default_rng(5)
        n_nodes = 4096
        nm = torch.from_numpy(rng.normal(size=(n_nodes, 3)).astype(np.float32) * 10).to(dev)
        nn_ = torch.from_numpy(rng.normal(size=(n_nodes, 3)).astype(np.float32)).to(dev)
        nn_ = (nn_ / nn_.norm(dim=1, keepdim=True)).contiguous()
        node_of = torch.from_numpy(rng.integers(0, n_nodes, scene.n).astype(np.int32)).to(dev)
        losses = torch.empty(2, dtype=torch.float64, device=dev)
        gs = psi.PsiGrads(*(psi._ptr(grads[k]) for k in ("mu", "tu", "tv", "scale")), None, None, None)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        for rep in range(3):
            ev[0].record()
            psi.psi_surfel_regularisers(ctx, scene.surfels_struct(), node_of, nm, nn_, n_nodes, 0.5, 1.0, 1.0, losses, gs)
            ev[1].record()
            torch.cuda.synchronize()
        reg_ms = ev[0].elapsed_time(ev[1])
        reg_bytes = scene.n * (4.0 * (3 + 3 + 3 + 2) + 4.0 + 2 * 4.0 * (3 + 3 + 3 + 2))  # read + gradient read/write
        regs = {"ms": float(reg_ms), "surfels": scene.n, "priors": n_nodes,
                "hbm_frac": reg_bytes / (reg_ms / 1000.0) / 1e9 / float(peaks.get("hbm_gbs", 6800.0))}

    # ---- 2DGS compatibility over all surfels, one 1080p view: quaternion
    # tangent frames and their adjoint; the depth/normal table, its dense
    # composite (K = 0), the composite's adjoint and the table's adjoint
    geo = None
    if args.label_frames > 0:
        def timed(fn, reps=3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            fn()
            torch.cuda.synchronize()
            e0.record()
            for _ in range(reps):
                fn()
            e1.record()
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps
        rng = np.random.default_rng(7)
        qd = torch.from_numpy(rng.normal(size=(scene.n, 4)).astype(np.float32)).to(dev)
        tu_o, tv_o = torch.empty(scene.n, 3, device=dev), torch.empty(scene.n, 3, device=dev)
        gq = torch.zeros(scene.n, 4, device=dev)
        fr_ms = timed(lambda: psi.psi_quat_frames(ctx, qd, scene.n, tu_o, tv_o))
        frb_ms = timed(lambda: psi.psi_quat_frames_bwd(ctx, qd, scene.n, grads["tu"], grads["tv"], gq))
        cam_arr = psi.cameras([cams[0]])
        Gt = pl.surfel_geometry(ctx, scene, cams[0])
        gsc = pl.label_scene(scene, Gt)
        go = psi.default_opts(mode=psi.EXACT, top_k=0, opacity_radius=1)
        rg = pl.Renderer(ctx, scene.n, [cams[0]], go, r.capacity, D=16, F_dtype=psi.F32, device=dev)
        rg.project(gsc)
        rg.intersect()
        rg.sort()
        tab_ms = timed(lambda: psi.psi_surfel_geometry(ctx, scene.surfels_struct(), cam_arr, Gt, 16))
        ren_ms = timed(lambda: rg.render(gsc))
        gFg = torch.randn(rg.n_pix, 16, device=dev)
        gg = {k: torch.zeros_like(v) for k, v in grads.items() if k != "feat"}
        gg["feat"] = torch.zeros(scene.n, 16, device=dev)
        bwd_ms = timed(lambda: rg.backward(gsc, gC, gFg, gT, grads=gg))
        gsg = psi.PsiGrads(psi._ptr(gg["mu"]), psi._ptr(gg["tu"]), psi._ptr(gg["tv"]), None, None, None, None)
        tbwd_ms = timed(lambda: psi.psi_surfel_geometry_bwd(ctx, scene.surfels_struct(), cam_arr, gg["feat"], 16, gsg))
        geo = {"quat_frames_ms": float(fr_ms), "quat_frames_bwd_ms": float(frb_ms),
               "depth_normal_table_ms": float(tab_ms), "depth_normal_render_ms": float(ren_ms),
               "depth_normal_render_bwd_ms": float(bwd_ms), "depth_normal_table_bwd_ms": float(tbwd_ms),
               "form": "3M surfels, one 1920x1080 view; the [N, 16] FP32 depth/normal table composited densely "
                       "(K = 0, EXACT) by the compositing kernels; adjoint of that composite (saved state) and of "
                       "the table"}
        del rg, gg, Gt

    # ---- precision plus batching: 1M surfels, 16 views of uneven resolution
    # (640x360 .. 1920x1080) in one launch per stage, the frame captured as one
    # CUDA graph; features in BF16, then FP8-E4M3 with per-channel scales;
    # tile height and launch shapes from the autotuner
    batch = None
    batch_frames = {}
    batch_world = None
    if args.batch_reps > 0:
        wb = sg.batch_scene()
        batch = {"surfels": wb.surfels.n, "views": len(wb.cameras),
                 "pixels": int(sum(c.width * c.height for c in wb.cameras)), "top_k": 8, "feat_dim": 128}
        for name, fdt in (("bf16", psi.BF16), ("fp8_e4m3", psi.FP8_E4M3)):
            sb = pl.DeviceScene(wb.surfels, wb.features, feat_dtype=fdt, device=dev)
            ob = psi.default_opts(mode=psi.EXACT, top_k=8, opacity_radius=1)
            ob, tms = pl.tune_tile_height(ctx, sb, wb.cameras, ob, D=D, F_dtype=psi.BF16)
            rb = pl.make_renderer(ctx, sb, wb.cameras, ob, D=D, F_dtype=psi.BF16)
            rb.frame(sb)
            tr = rb.tune(sb, torch.zeros(3, rb.n_pix, device=dev), reps=2)
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            cs = torch.cuda.Stream(device=dev)
            with torch.cuda.graph(g, stream=cs, capture_error_mode="relaxed"):
                rb.frame(sb)
            for _ in range(3):
                g.replay()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(args.batch_reps):
                g.replay()
            e1.record()
            torch.cuda.synchronize()
            st, _ = ctx.status_fetch()
            assert st == 0, f"device status {st}"
            ms = e0.elapsed_time(e1) / args.batch_reps
            batch[name] = {"ms_per_batch": ms, "views_per_s": len(wb.cameras) * 1000.0 / ms,
                           "batches_per_s": 1000.0 / ms, "tile": f"16x{int(ob.tile_h)}",
                           "frame_ms_per_tile_height": tms, "forward_shape": tr["fwd"][1],
                           "forward_ms_per_shape": [round(x, 4) for x in tr["fwd"][0]],
                           "pairs": int(rb.num_pairs.item()), "launches_per_batch": rb.kernel_launches()}
            # 24 sampled pixels of views 2 and 9 for the oracle comparison on the CPU leg
            rng = np.random.default_rng(2)
            samp = []
            for v in (2, 9):
                cam = wb.cameras[v]
                idx = rng.choice(cam.width * cam.height, 24, replace=False)
                p = torch.from_numpy(int(rb.pix_base[v]) + idx).to(dev)
                samp.append((v, idx, rb.rgb[:, p].T.double().cpu().numpy(), rb.F[p].float().double().cpu().numpy()))
            batch_frames[name] = (samp, pl.dequantize(sb.q, sb.qscale, fdt))
            del g, rb, sb
        batch["form"] = ("project+intersect+sort+render of all 16 views, one launch per stage, replayed as one CUDA "
                         "graph; EXACT tiles, K=8, FP32 accumulation; ms per batch of 16 views")
        batch_world = wb

    # ---- frustum-constrained cross-attention (Sec. 4.1) over all surfels
    # for one view: 100 queries, C = d = 128, BF16 features; forward and adjoint
    attn = None
    if args.label_frames > 0:
        rng = np.random.default_rng(6)
        Wa = [torch.from_numpy((rng.normal(size=(D, D)) / np.sqrt(D)).astype(np.float32)).to(dev) for _ in range(3)]
        Qa = torch.from_numpy(rng.normal(size=(nq, D)).astype(np.float32)).to(dev)
        Ga = torch.from_numpy(rng.normal(size=(nq, D)).astype(np.float32)).to(dev)
        outa = torch.empty(nq, D, device=dev)
        gQa, gW = torch.empty(nq, D, device=dev), [torch.empty(D, D, device=dev) for _ in range(3)]
        wsa = torch.empty(psi.attention_workspace_size(scene.n, D, D, nq), dtype=torch.uint8, device=dev)
        gsa = psi.PsiGrads(psi._ptr(grads["mu"]), None, None, None, None, None, psi._ptr(grads["feat"]))
        ca = psi.cameras([cams[0]])
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        fw, bw = [], []
        for rep in range(4):
            ev[0].record()
            psi.psi_frustum_attention(ctx, scene.surfels_struct(), scene.features_struct(), ca[0], 0.2, Qa, nq,
                                      Wa[0], Wa[1], Wa[2], D, outa, wsa)
            ev[1].record()
            psi.psi_frustum_attention_bwd(ctx, scene.surfels_struct(), scene.features_struct(), Qa, nq, Wa[0], Wa[1],
                                          Wa[2], D, Ga, gQa, gW[0], gW[1], gW[2], gsa, wsa)
            ev[2].record()
            torch.cuda.synchronize()
            if rep > 0:
                fw.append(ev[0].elapsed_time(ev[1]))
                bw.append(ev[1].elapsed_time(ev[2]))
        st, _ = ctx.status_fetch()
        assert st == 0, f"device status {st}"
        fms, bms = float(np.median(fw)), float(np.median(bw))
        flops = 4.0 * nq * scene.n * D  # scores and the weighted sum over the surfels (folded form)
        fbytes = scene.n * (2.0 * D + 20.0)  # BF16 feature row, centre and scales per surfel
        bf16_peak = float(peaks.get("bf16_tflops", 1900.0))
        attn = {"fwd_ms": fms, "bwd_ms": bms, "surfels": scene.n, "queries": nq, "C": D, "d": D,
                "fwd_tflops": flops / (fms / 1000.0) / 1e12,
                "fwd_tflops_frac_of_bf16": flops / (fms / 1000.0) / 1e12 / bf16_peak,
                "fwd_hbm_frac": fbytes / (fms / 1000.0) / 1e9 / hbm_peak,
                "form": "tcgen05 kernels, BF16 operands / FP32 accumulation: per 128-surfel tile S = qh [f|psi]^T, "
                        "online masked softmax, O += P f; queries folded qh = (Q W_Q) W_K^T / sqrt(d), output O W_V. "
                        "Adjoint: P recomputed per tile, dqh, dK, dV on the tensor cores"}
        del wsa

    # ---- the paper's Table 3 rows on this GPU: tile test x feature selection,
    # same BF16 features, forward of one frame (project, intersect, sort,
    # render), eager launches, median over frames
    ablation = None
    if args.ablation_frames > 0:
        rows = [("baseline", psi.SPHERE, 0, 0), ("precise_tile_aabb", psi.AABB, 0, 0),
                ("precise_tile_exact", psi.EXACT, 0, 0), ("topk", psi.SPHERE, K, 0), ("full_aabb", psi.AABB, K, 0),
                ("full_exact", psi.EXACT, K, 0), ("full_exact_lowpass", psi.EXACT, K, 1)]
        ablation = {}
        for name, mode, kk, lp in rows:
            ao = psi.default_opts(mode=mode, top_k=kk, opacity_radius=1 if mode == psi.EXACT else 0, lowpass=lp)
            ra = pl.Renderer(ctx, scene.n, [cams[0]], ao, 1024, D=D, F_dtype=psi.BF16, device=dev)
            nf = min(args.ablation_frames, len(cams))
            need = 0
            for k in range(nf):
                ra.set_cameras([cams[fidx(k)]])
                need = max(need, ra.required_pairs(scene))
            ra.set_capacity(int(need * 1.15) + 1024)
            ts, prs = [], []
            for k in range(nf + 1):
                ra.set_cameras([cams[fidx(k)]])
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                ra.frame(scene)
                e1.record()
                torch.cuda.synchronize()
                if k > 0:
                    ts.append(e0.elapsed_time(e1))
                    prs.append(int(ra.num_pairs.item()))
            ablation[name] = {"fwd_ms": float(np.median(ts)), "pairs_per_frame": float(np.mean(prs)),
                              "pairs_per_tile": float(np.mean(prs)) / ra.n_tiles,
                              "tiles": {0: "sphere", 1: "aabb", 2: "exact+opacity-radius"}[mode], "top_k": kk,
                              "lowpass": bool(lp)}
            del ra
        ablation["form"] = ("forward (project+intersect+sort+render) of one 1920x1080 frame, BF16 features, "
                            "K=0 dense / K=8 Top-K, median over %d frames" % min(args.ablation_frames, len(cams)))

    # ---- CPU oracle on a bounded sample (rank 0); the same sample checks
    # frame 0 of the GPU path against the oracle (parity)
    cpu = None
    parity = None
    if rank == 0 and not args.no_cpu_baseline:
        r.set_cameras([cams[0]])
        r.frame(scene)
        torch.cuda.synchronize()
        g_rgb, g_T = r.rgb.cpu().numpy().astype(np.float64), r.T.cpu().numpy().astype(np.float64)
        g_F, g_tk = r.F.float().cpu().numpy().astype(np.float64), r.topk_ids.cpu().numpy()
        deq = bf16_round(w.features).astype(np.float64)
        Qm = bf16_round(w.queries).astype(np.float64)
        gfn = lambda n: (gC_h.numpy()[:, :n].T.astype(np.float64), gF_h.numpy()[:n].astype(np.float64),
                         gT_h.numpy()[:n].astype(np.float64))
        info = oracle_frame_sample(w, cams[0], deq, Qm, gfn, args.cpu_seconds,
                                   dict(mode=2, top_k=K, opacity_radius=True))
        cpu = {"value": 1.0 / info["frame_s"], "unit": "frames/s", "cores": info["threads"], "kind": "oracle",
               "sample": f"frame 0: binning + canonical order of all {args.surfels} surfels ({info['t_fixed']:.2f} s) "
                         f"and forward+gradient+decode of {info['sample_pixels']} random pixels "
                         f"({info['t_pix'] * 1e3:.1f} ms/pixel), extrapolated to {P} pixels"}
        parity = parity_of_sample(info["out"], info["pixels"], cams[0], g_rgb, g_T, g_F, g_tk)
        if batch is not None:
            # storage precision of the batch against the FP64 oracle: 24 pixels
            # of views 2 and 9, the oracle fed the unquantised features (the
            # storage error) and the stored ones (the arithmetic)
            from oracle import oracle as orc
            wb = batch_world
            ob = orc.Opts(mode=orc.EXACT, top_k=8, opacity_radius=True)
            f64 = wb.features.astype(np.float64)
            for name, (samp, deq) in batch_frames.items():
                e_rgb, e_st, e_q = 0.0, 0.0, 0.0
                for v, idx, b_rgb, b_F in samp:
                    cam = wb.cameras[v]
                    pix = orc.all_pixels(cam)[idx]
                    ref = orc.render(wb.surfels, cam, ob, feat=f64, pixels=pix)
                    refq = orc.render(wb.surfels, cam, ob, feat=deq, pixels=pix)
                    e_rgb = max(e_rgb, float(np.abs(b_rgb - ref["rgb"]).max()))
                    m = ref["sumw"] > 0.5
                    e_st = max(e_st, float(np.linalg.norm(b_F[m] - ref["F"][m]) / max(np.linalg.norm(ref["F"][m]), 1e-30)))
                    e_q = max(e_q, float(np.linalg.norm(b_F[m] - refq["F"][m]) / max(np.linalg.norm(refq["F"][m]), 1e-30)))
                batch[name]["oracle"] = {"max_abs_err_rgb": e_rgb, "rel_l2_F_vs_unquantised": e_st,
                                         "rel_l2_F_vs_stored_values": e_q, "pixels": 48}

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": workload_config(args, use_graph),
        "fwd_frames_per_s": float(1000.0 / fwd_only_ms), "fwd_bwd_ms": float(frame_ms.mean()),
        "frame_ms_p50": float(np.percentile(frame_ms, 50)), "frame_ms_p99": float(np.percentile(frame_ms, 99)),
        "stage_ms": {n: float(v) for n, v in zip(names, mean_stage)}, "kernel_ms": kernel_ms,
        "pairs_per_frame": float(np.mean(pairs)), "pairs_per_tile": float(np.mean(pairs) / n_tiles),
        "autotune": tuned, "plain_fp32": plain, "ablation": ablation, "labels": labels, "regularisers": regs, "compat_2dgs": geo, "attention": attn, "roofline": roof, "cpu_baseline": cpu, "parity": parity, "batch16": batch, "e2e": e2e,
        "gpu_launches": int(args.steps * r.kernel_launches(with_decode=True, with_bwd=True)),
        "clocks": clk, "paper_context": PAPER_CONTEXT, "setup_s": setup_s,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    run_psi(args)


if __name__ == "__main__":
    main()
