"""Benchmark of the guiding hot path on GB300.

One step = one pass of the whole path over the workload: grid build (Morton
codes, radix sort, adaptive split, leaf assignment) -> splat -> CNN
reconstruction -> normalisation + CDFs -> guided sampling of Q queries -> pdf
evaluation of Q (position, direction) pairs.  Default workload: 4,194,304
photons (64 blobs), depth 10, split threshold 2000, 64x64 maps, U-Net
32-64-128-256, BF16 tensor-core CNN, 8,388,608 queries.  `--progressive`
times instead one later iteration of the progressive form (a photon batch
binned into the fixed grid, maps rebuilt where photons arrived, tables,
sampling, evaluation); `--mis` samples and evaluates the BSDF/guide mixture.

Prints one JSON line.  `value` = guided samples per second over whole steps
(Q x steps / device time of the steps, inputs resident in HBM); `e2e` = the
same through the C ABI with inputs in pinned host memory and results read
back, copies inside the timed region.  `--impl reference` times the CPU
oracle (FP64, host cores) on a bounded sample of the same workload.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "guided samples/s + leaf tables/s, FP32 vs BF16/FP8 at KL≤1e-3; p50/p99 latency"
LO, HI = [0.0, 0.0, 0.0], [1.0, 1.0, 1.0]

# DRAM bytes (read + write) of one reconstruct call per active leaf, from one
# ncu capture of every kernel of a reconstruct (dram__bytes_read.sum +
# dram__bytes_write.sum; profiles/k_conv_tc_scale-mid.md), keyed by (H, W,
# precision).  The traffic of a reconstruct grows in proportion to its leaves.
CNN_DRAM_BYTES_PER_LEAF = {(64, 64, "bf16"): 7149.4e6 / 1322}


def unet_flops_per_leaf(H, W, widths, arch):
    """2 * MACs of the network per map (zero padding counted as work)."""
    from paper_2010_01775_gb300 import synth
    f, h, w = 0, H, W
    layers = synth.net_layers(arch, widths)
    res = {0: (H, W)}
    if arch == synth.ARCH_TINY3:
        return sum(2 * H * W * k * k * cin * cout for cout, cin, k, s, a in layers)
    if arch == synth.ARCH_PAPER:
        sizes = [(H, W), (H, W), (H // 2, W // 2), (H // 2, W // 2), (H // 4, W // 4), (H // 4, W // 4),
                 (H // 4, W // 4), (H // 2, W // 2), (H // 2, W // 2), (H, W), (H, W), (H, W)]
        return sum(2 * ho * wo * k * k * cin * cout for (cout, cin, k, s, a), (ho, wo) in zip(layers, sizes))
    sizes = [(H, W), (H, W), (H // 2, W // 2), (H // 2, W // 2), (H // 4, W // 4), (H // 4, W // 4),
             (H // 8, W // 8), (H // 8, W // 8), (H // 4, W // 4), (H // 4, W // 4), (H // 2, W // 2),
             (H // 2, W // 2), (H, W), (H, W), (H, W)]
    for (cout, cin, k, s, a), (ho, wo) in zip(layers, sizes):
        f += 2 * ho * wo * k * k * cin * cout
    return f


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during timing."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.skip = 0
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "50"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        # Wait (up to 3 s) until sampling is live, so that the timed region that
        # follows is covered; samples taken before it are dropped in stop().
        t_end = time.time() + 3.0
        while self.p is not None and time.time() < t_end:
            self.f.flush()
            n = len(open(self.f.name).read().strip().splitlines())
            if n:
                self.skip = n
                break
            time.sleep(0.02)

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = [r.split(", ") for r in open(self.f.name).read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        if len(rows) > self.skip:
            rows = rows[self.skip:]  # the samples taken during the timed region
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def run_pg(args, wl, prec):
    import torch

    from paper_2010_01775_gb300 import pg, synth

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    ph, pos, dirs, blob = synth.workload_inputs(wl)
    n, q, H, W = wl.n_photons, wl.n_queries, wl.H, wl.W
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = pg.Context(stream.cuda_stream)
    net = pg.pg_net_load(ctx, blob)
    # Optional mixture of experts (Sec. 8): experts 1.. are the same
    # architecture with other seeded weights.
    experts = [net] + [pg.pg_net_load(ctx, synth.net_blob(wl.arch, wl.widths, wl.seed + 1000 + e))
                       for e in range(1, args.experts)] if args.experts > 1 else []

    def recon(h, pr):
        if experts:
            return pg.pg_reconstruct_experts(ctx, h, experts, synth.EXPERT_BOUNDS[:len(experts) - 1], pr)
        return pg.pg_reconstruct(ctx, h, net, pr)
    d_ph = torch.from_numpy(ph).cuda()
    d_pos = torch.from_numpy(pos).cuda()
    d_dir = torch.from_numpy(dirs).cuda()
    outs = (torch.empty(q, 3, device="cuda"), torch.empty(q, device="cuda"),
            torch.empty(q, dtype=torch.int32, device="cuda"), torch.empty(q, dtype=torch.int32, device="cuda"),
            torch.empty(q, device="cuda"), torch.empty(q, dtype=torch.uint8, device="cuda"))
    # The paper's grid rule needs the surface normal at every photon.
    ph_nrm = synth.wall_normals(ph) if args.grid == "kd" else None
    d_nrm = torch.from_numpy(ph_nrm).cuda() if ph_nrm is not None else None
    # One-sample MIS (Sec. 7.3): vertex normals and bounce contributions.
    nrm, con = synth.vertex_records(q, wl.seed) if args.mis else (None, None)
    d_vtx = (torch.from_numpy(nrm).cuda(), torch.from_numpy(con).cuda()) if args.mis else None
    mis = None
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > 129 MB L2
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def build_grid(p_ph, p_nrm=None):
        if args.grid == "kd":  # the paper's rule: 100^3 voxels, trees of depth 8, M_thr = 500, V_thr = 0.5
            return pg.pg_build_grid_kd(ctx, p_ph, p_nrm if p_nrm is not None else d_nrm, n, LO, HI, KD_R, KD_DEPTH,
                                       KD_THR, KD_VTHR)
        return pg.pg_build_grid(ctx, p_ph, n, LO, HI, wl.max_depth, wl.min_depth, wl.split_threshold)

    def step(p_ph, p_pos, p_dir, outs, pr, marks=None, keep_tables=False, vtx=None, p_nrm=None):
        o_d, o_p, o_l, o_b, o_e, o_s = outs
        vtx = vtx if vtx is not None else d_vtx
        rec = (lambda i: marks[i].record(stream)) if marks is not None else (lambda i: None)
        rec(0)
        g = build_grid(p_ph, p_nrm)
        rec(1)
        h = pg.pg_splat_photons(ctx, g, p_ph, n, wl.n_prev, H, W, wl.frac_bits)
        rec(2)
        m = recon(h, pr)
        rec(3)
        t = pg.pg_build_cdf(ctx, m)
        rec(4)
        if mis is None:
            pg.pg_sample_dirs(ctx, g, t, p_pos, q, 20101775, 0, o_d, o_p, o_l, o_b)
            rec(5)
            pg.pg_eval_pdf(ctx, g, t, p_pos, p_dir, q, o_e)
        else:
            # Sample and evaluate the mixture, then fold this pass's bounces
            # into the statistics and update alpha for the next pass.
            pg.pg_mis_sample(ctx, g, t, mis, p_pos, vtx[0], q, 20101775, 0, o_d, o_p, o_s)
            rec(5)
            pg.pg_mis_eval(ctx, g, t, mis, p_pos, vtx[0], p_dir, q, o_e)
            pg.pg_mis_accumulate(ctx, mis, g, p_pos, o_s, vtx[1], q)
            pg.pg_mis_update(ctx, mis)
        rec(6)
        A = g.info(pg.PG_INFO_N_ACTIVE)
        L = g.info(pg.PG_INFO_N_LEAVES)
        P = pg.export_tables(t)["P"] if keep_tables else None
        for hd in (t, m, h, g):
            hd.free()
        return A, L, P

    # Launch shapes of the tensor-core convolutions are tuned once, untimed.
    g0 = build_grid(d_ph)
    h0 = pg.pg_splat_photons(ctx, g0, d_ph, n, wl.n_prev, H, W, wl.frac_bits)
    if args.load_tuning:
        pg.pg_net_set_tuning(net, np.load(args.load_tuning))
    elif args.autotune:
        lp = ({pg.PG_BF16, pg.PG_FP8_E4M3, pg.PG_FP8_MIXED} if args.arch == "unet"
              else {pg.PG_BF16})  # the paper-style net: BF16
        for pr in {prec} | (lp if args.sweep else set()):
            pg.pg_autotune(ctx, h0, net, pr)
    for ex in experts[1:]:  # same layer shapes: the first net's launch shapes fit every expert
        pg.pg_net_set_tuning(ex, pg.pg_net_get_tuning(net))
    if args.save_tuning:
        np.save(args.save_tuning, pg.pg_net_get_tuning(net))
    if args.mis:  # the grid is rebuilt from the same photons each step: same leaves
        mis = pg.pg_mis_create(ctx, g0)
    ctx.sync()

    def measure(pr, steps, warmup, clocks_on=False):
        for _ in range(warmup):
            A, L, _ = step(d_ph, d_pos, d_dir, outs, pr)
        ctx.sync()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        clocks = Clocks(local) if clocks_on else None
        launches0 = ctx.launch_count()
        times, stage = [], np.zeros(6)
        for _ in range(steps):
            flush.zero_()
            marks = [ev() for _ in range(7)]
            A, L, _ = step(d_ph, d_pos, d_dir, outs, pr, marks)
            marks[6].synchronize()
            times.append(marks[0].elapsed_time(marks[6]))
            stage += [marks[i].elapsed_time(marks[i + 1]) for i in range(6)]
        ctx.sync()
        torch.cuda.synchronize()
        launches = (ctx.launch_count() - launches0) // steps
        clk = clocks.stop() if clocks is not None else None
        total_ms = max_over_ranks(float(sum(times)), world)
        if world > 1:
            torch.distributed.barrier()
        stage_ms = dict(zip(["grid", "splat", "cnn", "cdf", "sample", "eval"], (stage / steps).round(4).tolist()))
        return dict(A=A, L=L, times=times, total_ms=total_ms, stage_ms=stage_ms, clocks=clk, launches=launches)

    main = measure(prec, args.steps, args.warmup, clocks_on=True)
    A, L, total_ms, stage_ms = main["A"], main["L"], main["total_ms"], main["stage_ms"]

    # End to end through the C ABI with pinned host buffers: photons are
    # copied once per step, query arrays are passed as host pointers (the
    # library stages them), results land in pinned host memory.
    h_ph = torch.from_numpy(ph).pin_memory()
    h_pos = torch.from_numpy(pos).pin_memory()
    h_dir = torch.from_numpy(dirs).pin_memory()
    h_outs = (torch.empty(q, 3).pin_memory(), torch.empty(q).pin_memory(),
              torch.empty(q, dtype=torch.int32).pin_memory(), torch.empty(q, dtype=torch.int32).pin_memory(),
              torch.empty(q).pin_memory(), torch.empty(q, dtype=torch.uint8).pin_memory())
    h_vtx = (torch.from_numpy(nrm).pin_memory(), torch.from_numpy(con).pin_memory()) if args.mis else None
    h_nrm = torch.from_numpy(ph_nrm).pin_memory() if ph_nrm is not None else None
    e2e_steps = max(1, min(args.steps, 3))

    def e2e_step():
        dph = torch.empty_like(d_ph)
        dph.copy_(h_ph, non_blocking=True)
        step(dph, h_pos, h_dir, h_outs, prec, vtx=h_vtx, p_nrm=h_nrm)
        ctx.sync()

    e2e_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    # The same through the C ABI with device pointers, the copies made by the
    # caller and pipelined on a second stream: step k+1's inputs go up and
    # step k-1's results come down while step k computes (double buffers).
    ins_h = [h_ph, h_pos, h_dir] + ([h_nrm] if h_nrm is not None else []) + (list(h_vtx) if h_vtx else [])
    ins_d = [[torch.empty(x.shape, dtype=x.dtype, device="cuda") for x in ins_h] for _ in range(2)]
    outs_d = [tuple(torch.empty_like(o) for o in outs) for _ in range(2)]
    outs_h = [tuple(torch.empty(o.shape, dtype=o.dtype).pin_memory() for o in outs) for _ in range(2)]
    cs, cs_down = torch.cuda.Stream(), torch.cuda.Stream()  # uploads and downloads overlap each other too
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_done = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]

    def copy_up(k):
        b = k % 2
        with torch.cuda.stream(cs):
            if k >= 2:
                cs.wait_event(ev_done[b])
            for d, hx in zip(ins_d[b], ins_h):
                d.copy_(hx, non_blocking=True)
            ev_in[b].record(cs)

    def compute(k):
        b = k % 2
        stream.wait_event(ev_in[b])
        if k >= 2:
            stream.wait_event(ev_out[b])
        x = ins_d[b]
        nx = 3 + (1 if h_nrm is not None else 0)
        step(x[0], x[1], x[2], outs_d[b], prec, vtx=(x[nx], x[nx + 1]) if h_vtx else None,
             p_nrm=x[3] if h_nrm is not None else None)
        ev_done[b].record(stream)

    def copy_down(k):
        b = k % 2
        with torch.cuda.stream(cs_down):
            cs_down.wait_event(ev_done[b])
            for hx, d in zip(outs_h[b], outs_d[b]):
                hx.copy_(d, non_blocking=True)
            ev_out[b].record(cs_down)

    def pipelined(K):
        copy_up(0)
        for k in range(K):
            if k + 1 < K:
                copy_up(k + 1)
            compute(k)
            copy_down(k)
        cs.synchronize()
        cs_down.synchronize()
        torch.cuda.synchronize()

    pipelined(2)
    K = max(3, min(args.steps, 10))
    t0 = time.perf_counter()
    pipelined(K)
    e2e_pipe_s = (time.perf_counter() - t0) / K

    if args.mis:  # positions, normals, eval directions, contributions in; dirs, pdfs, strategies out
        h2d = ph.nbytes + pos.nbytes + dirs.nbytes + nrm.nbytes + con.nbytes
        d2h = q * (12 + 4 + 4 + 1)
    else:
        h2d = ph.nbytes + pos.nbytes + dirs.nbytes
        d2h = q * (12 + 4 + 4 + 4 + 4)
    if ph_nrm is not None:
        h2d += ph_nrm.nbytes

    # Dominant kernel family: the CNN convolutions of one reconstruct call,
    # timed with events on the launching stream.
    flops_leaf = unet_flops_per_leaf(H, W, wl.widths, wl.arch)
    cnn_ms = []
    for _ in range(max(2, min(args.steps, 5))):
        a, b = ev(), ev()
        a.record(stream)
        m = recon(h0, prec)
        b.record(stream)
        b.synchronize()
        cnn_ms.append(a.elapsed_time(b))
        m.free()
    cnn_s = statistics.median(cnn_ms) / 1e3
    peaks, peak_src = load_peaks()
    if prec == pg.PG_FP32:
        sm_mhz = peaks.get("sm_max_mhz", 2070.0)
        peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
        bound, unit = "alu", "TFLOP/s"
    else:
        peak = peaks["bf16_tflops"] * (2.0 if prec == pg.PG_FP8_E4M3 else 1.0)
        bound, unit = "tensor", "TFLOP/s"
    achieved = flops_leaf * A / cnn_s / 1e12

    # The other precisions of the same workload (shorter runs), and their
    # sampling maps on a few leaves for the CPU-baseline leg's KL check.
    names = {pg.PG_FP32: "fp32", pg.PG_BF16: "bf16", pg.PG_FP8_E4M3: "fp8", pg.PG_FP8_MIXED: "fp8mix"}
    sweep, maps = {}, {}
    check = None
    if args.sweep and world == 1:
        for pr in ((pg.PG_FP32, pg.PG_BF16, pg.PG_FP8_E4M3, pg.PG_FP8_MIXED) if args.arch == "unet"
                   else (pg.PG_FP32, pg.PG_BF16)):
            r = main if pr == prec else measure(pr, max(1, min(args.steps, 3)), 1)
            sweep[names[pr]] = {"value": q * len(r["times"]) / (r["total_ms"] / 1e3),
                                "ms_per_step": r["total_ms"] / len(r["times"]),
                                "leaf_tables_per_s": r["A"] * len(r["times"]) / (r["total_ms"] / 1e3),
                                "cnn_ms": r["stage_ms"]["cnn"]}
            _, _, P = step(d_ph, d_pos, d_dir, outs, pr, keep_tables=True)
            if check is None:
                check = np.linspace(0, P.shape[0] - 1, args.cpu_sample_leaves).astype(np.int64)
            if not experts:  # the oracle leg runs the single net
                maps[names[pr]] = P[check].astype(np.float64)
    mis_alpha = None
    if mis is not None:
        e = pg.export_mis(mis)
        mis_alpha = {"mean": float(e["alpha"].mean()), "updated_leaves": int(np.sum(e["alpha"] != 0.5)),
                     "leaves": int(e["alpha"].size)}
        mis.free()
    for hd in (h0, g0):
        hd.free()
    ctx.destroy()

    value = whole_job_rate(q, args.steps, world, total_ms)
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": {0: "f32", 1: "bf16", 2: "fp8e4m3", 3: "fp8e4m3+bf16"}[prec],
            "data": "synthetic (seeded photon blobs on room walls, vMF directions, lognormal power; random He-init U-Net)",
            "config": {"workload": wl.name + (" (paper's grid rule)" if args.grid == "kd" else ""), "photons": n,
                       "queries": q, "H": H, "W": W,
                       "max_depth": KD_DEPTH if args.grid == "kd" else wl.max_depth,
                       "split_threshold": KD_THR if args.grid == "kd" else wl.split_threshold,
                       "leaves": L, "active_leaves": A,
                       "precision": args.precision, "parallelism": f"replicas x{world}",
                       "experts": args.experts or 1,
                       "sampling": ("one-sample MIS: Lambertian BSDF stand-in + guide, per-leaf alpha"
                                    if args.mis else "guide"),
                       "grid": (f"paper's rule: {KD_R}^3 voxels, binary trees of depth <= {KD_DEPTH}, "
                                f"M_thr {KD_THR}, V_thr {KD_VTHR}, wall normals" if args.grid == "kd"
                                else f"octree, depth {wl.max_depth}, split {wl.split_threshold}"),
                       "l2": "flushed between steps (256 MB write); inputs also exceed L2"},
            "leaf_tables_per_s": A * args.steps * world / (total_ms / 1e3),
            "stage_ms": stage_ms,
            "stage_throughput": {"leaf_tables_per_s_build": A / (sum(list(stage_ms.values())[:4]) / 1e3),
                                 "guided_samples_per_s_sample_eval": q / ((stage_ms["sample"] + stage_ms["eval"]) / 1e3)},
            "latency_ms": {"p50": float(np.percentile(main["times"], 50)),
                           "p99": float(np.percentile(main["times"], 99))},
            "e2e": {"value": q / e2e_pipe_s, "unit": "samples/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h),
                    "how": "C ABI on device pointers; every step's inputs copied up from pinned host memory and "
                           "all its results copied back inside the timed region, on an upload and a download "
                           "stream pipelined against the neighbouring steps' compute"},
            "e2e_serial": {"value": q / e2e_s, "unit": "samples/s",
                           "how": "host pointers passed to the C ABI (the library stages them), one step at a time"},
            "gpu_launches": main["launches"],
            "roofline": {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
                         "traffic": (CNN_DRAM_BYTES_PER_LEAF[(H, W, args.precision)] * A
                                     if (H, W, args.precision) in CNN_DRAM_BYTES_PER_LEAF and args.arch == "unet"
                                     else None),
                         "kernel": "CNN convolutions (all layers of one reconstruct call)",
                         "peak_source": ("of " + peak_src) if prec != pg.PG_FP32 else
                         "derived: 152 SM x 128 FP32 FMA/clk x 2 x max SM clock"},
            "clocks": main["clocks"],
        }
        if sweep:
            out["precisions"] = sweep
        if mis_alpha is not None:
            out["mis_alpha"] = mis_alpha
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(wl, args.cpu_sample_leaves, check, maps, out.get("precisions"),
                                               mis=args.mis, kd=args.grid == "kd")
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_batch(args, bw, prec):
    """Scene-batch workload: one batched grid build, then splat -> CNN -> CDF
    -> sample -> eval over all scenes, the post-grid part captured once as a
    CUDA graph and replayed."""
    import torch

    from paper_2010_01775_gb300 import pg, synth

    torch.cuda.set_device(0)
    ph, begin, pos, dirs, qbegin, blob = synth.batch_inputs(bw)
    S, n, Q = bw.n_scenes, int(begin[-1]), int(qbegin[-1])
    los, his = [[0.0, 0.0, 0.0]] * S, [[1.0, 1.0, 1.0]] * S
    n_prev = ((begin[1:] - begin[:-1]) // 2).astype(np.uint32)
    streams = np.arange(S, dtype=np.uint32)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = pg.Context(stream.cuda_stream)
    net = pg.pg_net_load(ctx, blob)
    d_ph = torch.from_numpy(ph).cuda()
    d_pos = torch.from_numpy(pos).cuda()
    d_dir = torch.from_numpy(dirs).cuda()
    d_begin = torch.from_numpy(begin.view(np.int32)).cuda()
    d_qbegin = torch.from_numpy(qbegin.view(np.int32)).cuda()
    d_nprev = torch.from_numpy(n_prev.view(np.int32)).cuda()
    d_streams = torch.from_numpy(streams.view(np.int32)).cuda()
    o = (torch.empty(Q, 3, device="cuda"), torch.empty(Q, device="cuda"), torch.empty(Q, dtype=torch.int32, device="cuda"),
         torch.empty(Q, dtype=torch.int32, device="cuda"), torch.empty(Q, device="cuda"))
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def grid():
        return pg.pg_build_grid_batched(ctx, d_ph, n, d_begin, los, his, bw.max_depth, bw.min_depth,
                                        bw.split_threshold)

    def post(g):
        h = pg.pg_splat_photons_batched(ctx, g, d_ph, n, d_nprev, bw.H, bw.W, bw.frac_bits)
        m = pg.pg_reconstruct(ctx, h, net, prec)
        t = pg.pg_build_cdf(ctx, m)
        pg.pg_sample_dirs_batched(ctx, g, t, d_pos, d_qbegin, Q, 20101775, d_streams, o[0], o[1], o[2], o[3])
        pg.pg_eval_pdf_batched(ctx, g, t, d_pos, d_dir, d_qbegin, Q, o[4])
        for hd in (t, m, h):
            hd.free()

    g = grid()
    A, L = g.info(pg.PG_INFO_N_ACTIVE), g.info(pg.PG_INFO_N_LEAVES)
    h0 = pg.pg_splat_photons_batched(ctx, g, d_ph, n, d_nprev, bw.H, bw.W, bw.frac_bits)
    if args.autotune:
        pg.pg_autotune(ctx, h0, net, prec)
    h0.free()
    for _ in range(args.warmup):
        post(g)
    ctx.sync()
    # Eager steps: grid + post, events around each part.
    eager, grid_ms = [], []
    launches0 = ctx.launch_count()
    for _ in range(args.steps):
        e0, e1, e2 = ev(), ev(), ev()
        e0.record(stream)
        g2 = grid()
        e1.record(stream)
        post(g2)
        e2.record(stream)
        e2.synchronize()
        grid_ms.append(e0.elapsed_time(e1))
        eager.append(e0.elapsed_time(e2))
        g2.free()
    launches = (ctx.launch_count() - launches0) // args.steps
    # CUDA graph of the post-grid pipeline (allocations become graph memory nodes).
    graph = torch.cuda.CUDAGraph()
    ctx.sync()
    torch.cuda.synchronize()
    with torch.cuda.graph(graph, stream=stream, capture_error_mode="relaxed"):
        post(g)
    replays = []
    for _ in range(args.steps):
        e0, e1 = ev(), ev()
        e0.record(stream)
        graph.replay()
        e1.record(stream)
        e1.synchronize()
        replays.append(e0.elapsed_time(e1))
    ctx.sync()
    graph_ms = statistics.median(replays) + statistics.median(grid_ms)
    eager_ms = statistics.median(eager)
    out = {
        "metric": METRIC, "value": Q / (graph_ms / 1e3), "unit": "samples/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": graph_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {0: "f32", 1: "bf16", 2: "fp8e4m3", 3: "fp8e4m3+bf16"}[prec], "data": "synthetic",
        "config": {"workload": bw.name, "scenes": S, "photons": n, "queries": Q, "leaves": L, "active_leaves": A,
                   "H": bw.H, "W": bw.W, "precision": args.precision,
                   "scene_photons_min_max": [int(np.min(np.diff(begin))), int(np.max(np.diff(begin)))]},
        "leaf_tables_per_s": A / (graph_ms / 1e3),
        "eager_ms_per_step": eager_ms, "graph_ms_per_step": graph_ms, "grid_ms": statistics.median(grid_ms),
        "graph_replay_ms": statistics.median(replays), "gpu_launches": launches,
    }
    graph.reset()
    g.free()
    ctx.destroy()
    print(json.dumps(out), flush=True)


def run_serve(args, tr):
    """Serving loop: open-loop Poisson trace at the trace's rate and at a
    sustainable rate, closed-loop capacity, and plain FP32 one-request-at-a-
    time execution of the same requests for comparison."""
    import torch

    from paper_2010_01775_gb300 import pg, serve, synth

    torch.cuda.set_device(0)
    trace = synth.serve_trace(tr, duration=args.serve_seconds)
    n_pool = max(max(r["n"] for r in trace), 1 << 20)
    ph = torch.from_numpy(synth.photons(n_pool, 64, tr.seed)).pin_memory()
    pmax = np.maximum.accumulate(ph[:, 6].numpy().astype(np.float64))
    qpos = torch.from_numpy(synth.query_positions(tr.q_max, tr.seed)).pin_memory()
    qdir = torch.from_numpy(synth.query_directions(tr.q_max, tr.seed)).pin_memory()
    blob = synth.net_blob(synth.ARCH_UNET4, (32, 64, 128, 256), tr.seed + 77)

    def make(spec, prec=None):
        n, q, o = spec["n"], spec["q"], spec["q_offset"]
        # Largest fixed-point scale (<= 2^32) that keeps every sum below 2^63.
        frac = int(min(32, np.floor(np.log2(2.0 ** 63 / (n * max(pmax[n - 1], 1e-30)))) - 1))
        return serve.Request(ph[:n], qpos[o:o + q], qdir[o:o + q], spec["H"], spec["W"],
                             pg.PRECISIONS[prec or spec["precision"]], max_depth=tr.max_depth,
                             split_threshold=tr.split_threshold, frac_bits=frac, stream_id=spec["stream_id"])

    def warm_requests(precs):
        return [serve.Request(ph[:1 << 20], qpos[:65536], qdir[:65536], s, s, pg.PRECISIONS[p], max_depth=tr.max_depth,
                              split_threshold=tr.split_threshold, stream_id=1 << 30)
                for p in precs for s in tr.sizes]

    def replay(srv, specs, rate_scale=1.0, closed=False):
        t0 = time.perf_counter()
        rs = []
        for spec in specs:
            if not closed:
                dt = t0 + spec["arrival"] * rate_scale - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
            rs.append(srv.submit(make(spec, "fp32" if srv.fp32 else None)))
        for r in rs:
            r.wait()
        return rs

    out = {}
    srv = serve.Server(blob, workers=args.serve_workers, hbm_budget=120 << 30)
    srv.fp32 = False
    t = time.perf_counter()
    srv.warmup(warm_requests(tr.precisions), autotune=args.autotune)
    warm_s = time.perf_counter() - t
    k = min(args.serve_closed, len(trace))
    replay(srv, trace[:8], closed=True)  # first touches of the pools and staging buffers
    closed = serve.latency_summary(replay(srv, trace[:k], closed=True))
    spec_rate = serve.latency_summary(replay(srv, trace))
    sustain = 0.7 * closed["requests_per_s"]
    scale = tr.rate / sustain
    sub = [r for r in trace if r["arrival"] * scale <= args.serve_seconds]
    sustained = serve.latency_summary(replay(srv, sub, rate_scale=scale))
    srv.close()
    # Plain FP32, one request at a time, no batching: the same first requests.
    k32 = min(args.serve_fp32, k)
    base = serve.Server(blob, workers=1, hbm_budget=120 << 30, batching=False)
    base.fp32 = True
    replay(base, trace[:2], closed=True)
    fp32 = serve.latency_summary(replay(base, trace[:k32], closed=True))
    base.close()
    srv2 = serve.Server(blob, workers=args.serve_workers, hbm_budget=120 << 30)
    srv2.fp32 = False
    srv2.warmup(warm_requests(tr.precisions), autotune=args.autotune)
    same = serve.latency_summary(replay(srv2, trace[:k32], closed=True))
    srv2.close()
    out = {
        "metric": METRIC, "value": spec_rate["samples_per_s"], "unit": "samples/s", "n_gpus": 1,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16+fp8e4m3",
        "data": "synthetic",
        "config": {"workload": tr.name, "requests": len(trace), "rate_per_s": tr.rate,
                   "arrival_seconds": args.serve_seconds, "workers": args.serve_workers, "hbm_budget_gb": 120,
                   "batching": "continuous, same map size/precision, <=64 scenes, <=8M photons"},
        "latency_ms": {"p50": spec_rate.get("p50_ms"), "p99": spec_rate.get("p99_ms")},
        "open_loop_at_trace_rate": spec_rate,
        "open_loop_at_70pct_capacity": dict(sustained, rate_per_s=sustain, requests=len(sub)),
        "closed_loop_capacity": dict(closed, requests=k),
        "fp32_one_at_a_time": dict(fp32, requests=k32),
        "served_same_requests": dict(same, requests=k32),
        "speedup_vs_fp32_one_at_a_time": same["samples_per_s"] / fp32["samples_per_s"],
        "warmup_s": warm_s,
    }
    print(json.dumps(out), flush=True)


KD_R, KD_DEPTH, KD_THR, KD_VTHR = 100, 8, 500, 0.5  # Sec. 8 (M_thr = c sqrt(2^t) at t = 0, c = 500)
PROGRESS_FRAC_BITS = 24  # fixed point of the progressive sums: room for ~60M photons of power <= 500


def run_progressive(args, wl, prec):
    """One step = one later iteration of the progressive form (Sec. 7.2;
    Algorithm 1): a batch of wl.n_photons photons binned into the fixed grid
    and merged, the maps of the leaves that received photons reconstructed,
    the tables rebuilt, then Q guided samples and Q pdf evaluations.  The
    grid is refined beforehand, untimed, by two iterations of N_p and 2 N_p
    photons (N_p = wl.n_photons / 4, so that the timed batch is iteration
    2's, 2^2 N_p) with threshold 500 sqrt(2^t) (Sec. 8)."""
    import torch

    from paper_2010_01775_gb300 import pg, synth

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    n, q, H, W = wl.n_photons, wl.n_queries, wl.H, wl.W
    n_p = n // 4
    pool = synth.photons(3 * n_p + 2 * n, wl.n_blobs, wl.seed)
    refine = [pool[:n_p], pool[n_p:3 * n_p]]
    batches = [pool[3 * n_p:3 * n_p + n], pool[3 * n_p + n:]]  # timed steps alternate between two batches
    _, pos, dirs, blob = synth.workload_inputs(wl)
    steps_total = args.warmup + args.steps + 8
    max_photons = 3 * n_p + n * steps_total
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = pg.Context(stream.cuda_stream)
    net = pg.pg_net_load(ctx, blob)
    kd = args.grid == "kd"  # refinement by the paper's rule (100^3 voxels, trees of depth 8, wall normals)
    st = pg.pg_progress_create(ctx, LO, HI, KD_DEPTH if kd else wl.max_depth, wl.min_depth, H, W, max_photons,
                               split_c=500.0, refine_iterations=2, frac_bits=PROGRESS_FRAC_BITS,
                               grid_rule=1 if kd else 0, resolution=KD_R, normal_variance_threshold=KD_VTHR)
    for b in refine:
        pg.pg_progress_add_photons(ctx, st, torch.from_numpy(b).cuda(), len(b),
                                   torch.from_numpy(synth.wall_normals(b)).cuda() if kd else None)
    d_b = [torch.from_numpy(b).cuda() for b in batches]
    d_pos = torch.from_numpy(pos).cuda()
    d_dir = torch.from_numpy(dirs).cuda()
    o_d, o_p = torch.empty(q, 3, device="cuda"), torch.empty(q, device="cuda")
    o_l, o_e = torch.empty(q, dtype=torch.int32, device="cuda"), torch.empty(q, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ev = lambda: torch.cuda.Event(enable_timing=True)
    _, h0, _, _ = pg.pg_progress_view(st)
    if args.load_tuning:
        pg.pg_net_set_tuning(net, np.load(args.load_tuning))
    elif args.autotune:
        pg.pg_autotune(ctx, h0, net, prec)
    pg.pg_progress_reconstruct(ctx, st, net, prec)
    ctx.sync()
    counter = [0]

    def step(marks=None, batch=None, p_pos=d_pos, p_dir=d_dir, outs=(o_d, o_p, o_l, o_e)):
        rec = (lambda i: marks[i].record(stream)) if marks is not None else (lambda i: None)
        b = batch if batch is not None else d_b[counter[0] % 2]
        counter[0] += 1
        rec(0)
        pg.pg_progress_add_photons(ctx, st, b, n)
        rec(1)
        pg.pg_progress_reconstruct(ctx, st, net, prec)
        rec(2)
        g, _, _, t = pg.pg_progress_view(st)
        pg.pg_sample_dirs(ctx, g, t, p_pos, q, 20101775, 0, outs[0], outs[1], outs[2])
        rec(3)
        pg.pg_eval_pdf(ctx, g, t, p_pos, p_dir, q, outs[3])
        rec(4)
        return st.info(pg.PG_INFO_N_UPDATED), g.info(pg.PG_INFO_N_LEAVES)

    for _ in range(args.warmup):
        step()
    ctx.sync()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    launches0 = ctx.launch_count()
    times, stage, upd = [], np.zeros(4), []
    for _ in range(args.steps):
        flush.zero_()
        marks = [ev() for _ in range(5)]
        A, L = step(marks)
        marks[4].synchronize()
        times.append(marks[0].elapsed_time(marks[4]))
        stage += [marks[i].elapsed_time(marks[i + 1]) for i in range(4)]
        upd.append(A)
    ctx.sync()
    torch.cuda.synchronize()
    launches = (ctx.launch_count() - launches0) // args.steps
    clk = clocks.stop()
    total_ms = max_over_ranks(float(sum(times)), world)
    if world > 1:
        torch.distributed.barrier()
    stage_ms = dict(zip(["bin_merge", "reconstruct_cdf", "sample", "eval"], (stage / args.steps).round(4).tolist()))

    # End to end: the batch and the queries from pinned host memory, results back.
    h_b = torch.from_numpy(batches[0]).pin_memory()
    h_pos, h_dir = torch.from_numpy(pos).pin_memory(), torch.from_numpy(dirs).pin_memory()
    h_outs = (torch.empty(q, 3).pin_memory(), torch.empty(q).pin_memory(),
              torch.empty(q, dtype=torch.int32).pin_memory(), torch.empty(q).pin_memory())
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        step(batch=h_b, p_pos=h_pos, p_dir=h_dir, outs=h_outs)
        ctx.sync()
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps

    # Dominant kernels: the CNN of one reconstruct of the updated leaves.
    flops_leaf = unet_flops_per_leaf(H, W, wl.widths, wl.arch)
    peaks, peak_src = load_peaks()
    A_mean = float(np.mean(upd))
    cnn_ms = stage_ms["reconstruct_cdf"]
    peak = peaks["bf16_tflops"] * (2.0 if prec == pg.PG_FP8_E4M3 else 1.0)
    achieved = flops_leaf * A_mean / (cnn_ms / 1e3) / 1e12
    st.free()
    ctx.destroy()
    value = whole_job_rate(q, args.steps, world, total_ms)
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": {0: "f32", 1: "bf16", 2: "fp8e4m3", 3: "fp8e4m3+bf16"}[prec],
            "data": "synthetic (seeded photon blobs on room walls, vMF directions, lognormal power; random He-init U-Net)",
            "config": {"workload": "progressive iteration, " + wl.name, "photons_per_iteration": n,
                       "refine": f"2 iterations of {n_p} and {2 * n_p} photons, threshold 500 sqrt(2^t)",
                       "grid": (f"paper's rule: {KD_R}^3 voxels, trees of depth <= {KD_DEPTH}, V_thr {KD_VTHR}, "
                                "wall normals" if kd else f"octree, depth {wl.max_depth}"),
                       "queries": q, "H": H, "W": W, "max_depth": KD_DEPTH if kd else wl.max_depth, "leaves": L,
                       "updated_leaves_per_step": A_mean, "frac_bits": PROGRESS_FRAC_BITS,
                       "precision": args.precision, "parallelism": f"replicas x{world}",
                       "l2": "flushed between steps (256 MB write); inputs also exceed L2"},
            "leaf_tables_per_s": A_mean * args.steps * world / (total_ms / 1e3),
            "stage_ms": stage_ms,
            "e2e": {"value": q / e2e_s, "unit": "samples/s", "h2d_bytes_per_step": int(batches[0].nbytes + pos.nbytes + dirs.nbytes),
                    "d2h_bytes_per_step": int(q * (12 + 4 + 4 + 4))},
            "gpu_launches": launches,
            "roofline": {"bound": "tensor" if prec != pg.PG_FP32 else "alu", "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                         "kernel": "CNN convolutions + CDF of one progressive reconstruct (stage time)",
                         "peak_source": "of " + peak_src},
            "clocks": clk,
        }
        if world == 1 and not args.no_cpu_baseline and kd:
            # The oracle keeps leaf-indexed planes: 10^6 leaves x 4096 bins do not fit host memory.
            out["cpu_baseline"] = {"value": None, "unit": "samples/s", "kind": "oracle", "cores": 1,
                                   "sample": "not run: the oracle's progressive form holds leaf-indexed planes, "
                                             "about 100 GB for a 100^3-voxel grid of 64x64 maps"}
        elif world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = progressive_cpu_baseline(wl, args.cpu_sample_leaves)
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def progressive_cpu_baseline(wl, n_leaves, n_batch=262_144, n_queries=262_144):
    """The oracle's later iteration on a bounded sample: refinement on the
    same N_p and 2 N_p photons (untimed), then a batch of n_batch photons
    binned and merged, n_leaves of the updated leaves reconstructed, the
    tables built, n_queries sampled and evaluated; per-stage times scaled to
    the full step."""
    from oracle import oracle as O
    from paper_2010_01775_gb300 import synth
    n = wl.n_photons
    n_p = n // 4
    n_batch, n_queries = min(n_batch, n), min(n_queries, wl.n_queries)
    pool = synth.photons(3 * n_p + 2 * n, wl.n_blobs, wl.seed)
    _, pos, dirs, blob = synth.workload_inputs(wl)
    pr = O.Progressive(LO, HI, wl.max_depth, wl.min_depth, wl.H, wl.W, 3 * n_p + n, split_c=500.0,
                       refine_iterations=2, F=PROGRESS_FRAC_BITS)
    pr.add_photons(pool[:n_p])
    pr.add_photons(pool[n_p:3 * n_p])
    net = O.parse_net(blob)
    t0 = time.perf_counter()
    pr.add_photons(pool[3 * n_p:3 * n_p + n_batch])
    t1 = time.perf_counter()
    upd = pr.updated
    keep = upd[np.linspace(0, upd.size - 1, n_leaves).astype(np.int64)]
    y = O.cnn_forward(O.assemble_inputs(pr.planes(keep)), net)
    t2 = time.perf_counter()
    tabs = O.tables_from_map(y)
    t3 = time.perf_counter()
    slot = np.full(pr.grid["L"], -1, np.int32)
    slot[keep] = np.arange(keep.size, dtype=np.int32)
    O.sample(pr.grid, slot, tabs, pos[:n_queries], 20101775)
    O.eval_pdf(pr.grid, slot, tabs, pos[:n_queries], dirs[:n_queries])
    t4 = time.perf_counter()
    full_leaf, _ = O.leaf_of_positions(pr.grid, pool[3 * n_p:3 * n_p + n, :3])
    A_full = np.unique(full_leaf).size  # leaves a full batch updates
    step_s = (t1 - t0) * n / n_batch + (t3 - t1) * A_full / keep.size + (t4 - t3) * wl.n_queries / n_queries
    return {"value": wl.n_queries / step_s, "unit": "samples/s", "cores": 1, "kind": "oracle",
            "sample": (f"FP64 oracle, single thread, progressive later iteration: {n_batch} of {n} photons binned "
                       f"and merged, CNN+CDF on {keep.size} of ~{int(A_full)} updated leaves, sample+eval on "
                       f"{n_queries} of {wl.n_queries} queries; per-stage times scaled to the full step "
                       f"({step_s:.1f} s); wall {t4 - t0:.1f} s")}


def oracle_sample_run(wl, n_leaves, n_queries, check=None, mis=False, kd=False):
    """The FP64 oracle on a bounded sample; returns per-stage seconds and the
    throughput extrapolated to the full workload."""
    from oracle import oracle as O
    from paper_2010_01775_gb300 import synth
    ph, pos, dirs, blob = synth.workload_inputs(wl)
    t0 = time.perf_counter()
    if kd:
        g = O.build_kd_grid(ph, synth.wall_normals(ph), LO, HI, KD_R, KD_DEPTH, KD_THR, KD_VTHR)
    else:
        g = O.build_grid(ph, LO, HI, wl.max_depth, wl.min_depth, wl.split_threshold)
    act, slot = O.active_leaves(g)
    t1 = time.perf_counter()
    keep = act[check] if check is not None else act[np.linspace(0, act.size - 1, n_leaves).astype(np.int64)]
    gsub = dict(g)
    if kd:  # ~10^6 leaves: splat the kept leaves only and scale by their share of the photons
        sub = dict(g, L=keep.size, leaf_begin=g["leaf_begin"][keep], leaf_end=g["leaf_end"][keep])
        hs = O.splat(ph, sub, wl.n_prev, wl.H, wl.W, wl.frac_bits)
        hs = {k: v for k, v in hs.items() if k != "status"}
        share = float((g["leaf_end"][keep] - g["leaf_begin"][keep]).sum()) / max(1, ph.shape[0])
        t2 = time.perf_counter()
        splat_s = (t2 - t1) / max(share, 1e-9)
    else:
        h = O.splat(ph, g, wl.n_prev, wl.H, wl.W, wl.frac_bits)
        t2 = time.perf_counter()
        splat_s = t2 - t1
        hs = O.hist_for_active(h, keep)
    y = O.cnn_forward(O.assemble_inputs(hs), O.parse_net(blob))
    t3 = time.perf_counter()
    tabs = O.tables_from_map(y)
    t4 = time.perf_counter()
    slot2 = np.full(g["L"], -1, np.int32)
    slot2[keep] = np.arange(keep.size, dtype=np.int32)
    if mis:
        nrm, con = synth.vertex_records(wl.n_queries, wl.seed)
        p, nq = pos[:n_queries], nrm[:n_queries].astype(np.float64)
        alpha = np.full(g["L"], 0.5)
        s = O.mis_sample(gsub, slot2, tabs, alpha, p, nq, 20101775)
        O.mis_eval(gsub, slot2, tabs, alpha, p, nq, dirs[:n_queries])
        leaf, _ = O.leaf_of_positions(gsub, p)
        O.mis_alpha(O.mis_accumulate(g["L"], leaf, s["strategy"], con[:n_queries].astype(np.float64)), alpha)
    else:
        s = O.sample(gsub, slot2, tabs, pos[:n_queries], 20101775)
        O.eval_pdf(gsub, slot2, tabs, pos[:n_queries], dirs[:n_queries])
    t5 = time.perf_counter()
    A = act.size
    step_s = (t1 - t0) + splat_s + (t3 - t2) * A / keep.size + (t4 - t3) * A / keep.size + \
        (t5 - t4) * wl.n_queries / n_queries
    return dict(step_s=step_s, samples_per_s=wl.n_queries / step_s, wall_s=t5 - t0, leaves=int(keep.size),
                A=int(A), queries=n_queries, P=tabs["P"])


def cpu_baseline(wl, n_leaves, check=None, maps=None, precisions=None, mis=False, kd=False):
    r = oracle_sample_run(wl, n_leaves, 65_536 if mis else 262_144, check, mis, kd)
    out = {"value": r["samples_per_s"], "unit": "samples/s", "cores": 1, "kind": "oracle",
           "sample": (f"FP64 oracle, single thread: grid+splat on all {wl.n_photons} photons"
                      f"{' (the splat on the sampled leaves, scaled by their photon share)' if kd else ''}, CNN+CDF on "
                      f"{r['leaves']} of {r['A']} active leaves, {'MIS ' if mis else ''}sample+eval on "
                      f"{r['queries']} of {wl.n_queries} "
                      f"queries; per-stage times scaled to the full step ({r['step_s']:.1f} s); "
                      f"wall {r['wall_s']:.1f} s")}
    if maps and precisions is not None:
        Pr = r["P"]
        for name, P in maps.items():
            kl, l1 = [], []
            for a in range(P.shape[0]):
                p, qq = Pr[a].ravel(), np.maximum(P[a].ravel(), 1e-38)
                nz = p > 0
                kl.append(float(np.sum(p[nz] * np.log(p[nz] / qq[nz]))))
                l1.append(float(np.abs(p - P[a].ravel()).sum()))
            precisions[name]["kl_vs_fp64_oracle"] = {"mean": float(np.mean(kl)), "max": float(np.max(kl)),
                                                     "leaves": len(kl)}
            precisions[name]["l1_vs_fp64_oracle_mean"] = float(np.mean(l1))
    return out


def max_over_ranks(ms, world, device="cuda"):
    """Time of a step replicated over `world` ranks: the slowest rank's time,
    returned on every rank (one all-reduce; no data-path collective)."""
    if world <= 1:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank_step, steps, world, job_ms):
    """Units all ranks processed per second of job time (weak scaling)."""
    return units_per_rank_step * steps * world / (job_ms / 1e3)


def run_reference(args, wl):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    steps = []
    for i in range(args.warmup + args.steps):
        r = oracle_sample_run(wl, 2, 65_536)
        if i >= args.warmup:
            steps.append(r)
    step_s = statistics.mean(r["step_s"] for r in steps)
    value = wl.n_queries / step_s
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "precision": "fp64 oracle"},
        "cpu_baseline": {"value": value, "unit": "samples/s", "cores": 1, "kind": "oracle",
                         "sample": "per step: grid+splat on all photons, CNN+CDF on 2 active leaves, sample+eval on "
                                   "65536 queries, scaled to the full step"},
        "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="pg", choices=["pg", "reference"])
    ap.add_argument("--workload", default="scale")
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16", "fp8", "fp8mix"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--experts", type=int, default=0,
                    help="reconstruct with a mixture of this many experts routed by leaf photon count (Sec. 8)")
    ap.add_argument("--arch", default="unet", choices=["unet", "paper"],
                    help="the workload's U-Net, or the paper-style masked U-Net (partial convolutions, residual "
                         "links, dilated bottleneck, 32-64 channels; BF16 or FP32)")
    ap.add_argument("--grid", default="octree", choices=["octree", "kd"],
                    help="octree grid, or the paper's rule (100^3 voxels refined by binary trees)")
    ap.add_argument("--progressive", action="store_true",
                    help="time one later iteration of the progressive form (Sec. 7.2) instead of a single-shot step")
    ap.add_argument("--mis", action="store_true",
                    help="sample and evaluate one-sample MIS of a Lambertian BSDF and the guide (Sec. 7.3), "
                         "with the per-leaf statistics and alpha update in every step")
    ap.add_argument("--save-tuning", default=None, help="write the autotuned launch shapes (.npy)")
    ap.add_argument("--load-tuning", default=None, help="use launch shapes from --save-tuning instead of tuning")
    ap.add_argument("--serve-seconds", type=float, default=2.0, help="serving trace: seconds of arrivals")
    ap.add_argument("--serve-workers", type=int, default=4)
    ap.add_argument("--serve-closed", type=int, default=64, help="requests in the closed-loop capacity run")
    ap.add_argument("--serve-fp32", type=int, default=12, help="requests in the FP32 one-at-a-time run")
    ap.add_argument("--cpu-sample-leaves", type=int, default=4)
    ap.add_argument("--autotune", action=argparse.BooleanOptionalAction, default=True,
                    help="tune the tensor-core launch shapes before timing (untimed)")
    ap.add_argument("--sweep", action=argparse.BooleanOptionalAction, default=True,
                    help="also time the other CNN precisions and report their KL against the oracle")
    args = ap.parse_args()
    from paper_2010_01775_gb300 import synth
    if args.workload in synth.SERVE_TRACES:
        import __graft_entry__
        __graft_entry__.build()
        run_serve(args, synth.SERVE_TRACES[args.workload])
        return
    if args.workload in synth.BATCH_WORKLOADS:
        import __graft_entry__
        __graft_entry__.build()
        from paper_2010_01775_gb300 import pg
        run_batch(args, synth.BATCH_WORKLOADS[args.workload], pg.PRECISIONS[args.precision])
        return
    wl = synth.WORKLOADS[args.workload]
    if args.arch == "paper":
        import dataclasses
        wl = dataclasses.replace(wl, arch=synth.ARCH_PAPER, widths=(32, 64),
                                 name=wl.name + " (paper-style masked U-Net 32-64)")
    if args.impl == "reference":
        run_reference(args, wl)
        return
    import __graft_entry__
    __graft_entry__.build()
    from paper_2010_01775_gb300 import pg
    if args.progressive:
        run_progressive(args, wl, pg.PRECISIONS[args.precision])
    else:
        run_pg(args, wl, pg.PRECISIONS[args.precision])


if __name__ == "__main__":
    main()
