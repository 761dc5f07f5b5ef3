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
CNN_DRAM_BYTES_PER_LEAF = {(64, 64, "bf16"): 5703.2e6 / 1322}


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


def unet_executed_flops_per_leaf(H, W, widths, arch, precision):
    """The FLOPs the tensor cores execute per map.  In BF16 the U-Net's
    decoder layers over [upsample2(U), S] whose half-resolution grid is at
    least 32 wide run in the phase form: U's part is four 2x2 convolutions at
    half resolution, one per output phase, instead of a 3x3 convolution of
    the upsampled map, so each output pixel takes 4 instead of 9 taps of U's
    channels.  The network computes the same function, and the algorithmic
    count (unet_flops_per_leaf) stays the dense one."""
    from paper_2010_01775_gb300 import synth
    f = unet_flops_per_leaf(H, W, widths, arch)
    if arch != synth.ARCH_UNET4 or precision != "bf16":
        return f
    c = list(widths)
    for lev, (cu, cout) in enumerate(((c[1], c[0]), (c[2], c[1]), (c[3], c[2]))):
        hl, wl = H >> lev, W >> lev
        if wl // 2 >= 32 and 2 * (wl // 2 + 2) <= 256 and hl % 2 == 0 and wl % 2 == 0:
            f -= 2 * hl * wl * cout * 5 * cu
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

    def step(p_ph, p_pos, p_dir, outs, pr, marks=None, probe=None, vtx=None, p_nrm=None):
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
        got = probe(g, t) if probe is not None else None
        for hd in (t, m, h, g):
            hd.free()
        return A, L, got

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
    executed = unet_executed_flops_per_leaf(H, W, wl.widths, wl.arch, args.precision) * A / cnn_s / 1e12

    # The other precisions of the same workload (shorter runs).  For the
    # reduced-precision check each one's sampling map is kept on the leaves
    # the oracle recomputes (stratified by photon count), and guided samples
    # drawn at the centres of a few of them for the chi-square test.
    names = {pg.PG_FP32: "fp32", pg.PG_BF16: "bf16", pg.PG_FP8_E4M3: "fp8", pg.PG_FP8_MIXED: "fp8mix"}
    sweep, maps, chi_bins = {}, {}, {}
    ocheck = None
    if args.sweep and world == 1:
        ocheck = OracleCheck(wl) if (not args.no_cpu_baseline and not experts and args.grid == "octree") else None
        probe = ocheck.gpu_probe(ctx, pg, torch) if ocheck is not None else None
        for pr in ((pg.PG_FP32, pg.PG_BF16, pg.PG_FP8_E4M3, pg.PG_FP8_MIXED) if args.arch == "unet"
                   else (pg.PG_FP32, pg.PG_BF16)):
            r = main if pr == prec else measure(pr, max(1, min(args.steps, 3)), 1)
            sweep[names[pr]] = {"value": q * len(r["times"]) / (r["total_ms"] / 1e3),
                                "ms_per_step": r["total_ms"] / len(r["times"]),
                                "leaf_tables_per_s": r["A"] * len(r["times"]) / (r["total_ms"] / 1e3),
                                "cnn_ms": r["stage_ms"]["cnn"]}
            if probe is not None:
                _, _, got = step(d_ph, d_pos, d_dir, outs, pr, probe=probe)
                maps[names[pr]], chi_bins[names[pr]] = got
    mis_alpha = None
    if mis is not None:
        e = pg.export_mis(mis)
        mis_alpha = {"mean": float(e["alpha"].mean()), "updated_leaves": int(np.sum(e["alpha"] != 0.5)),
                     "leaves": int(e["alpha"].size)}
        mis.free()
    for hd in (h0, g0):
        hd.free()
    ctx.destroy()
    # The precision workload (128x128 maps, the same photons, U-Net and
    # queries) as its own table: every form's step rate and its check
    # against the oracle.
    prec_block, ocheck3, maps3, chi3 = None, None, None, None
    if (args.precision_config and world == 1 and args.sweep and args.arch == "unet" and not experts
            and args.grid == "octree" and not args.mis and wl.H == 64 and wl.n_photons == synth.SCALE.n_photons):
        prec_block, ocheck3, maps3, chi3 = run_precision_config(args, synth.PRECISION,
                                                                with_oracle=not args.no_cpu_baseline)

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
                         "derived: 152 SM x 128 FP32 FMA/clk x 2 x max SM clock",
                         "flops_per_leaf": flops_leaf,
                         "executed_flops_per_leaf": unet_executed_flops_per_leaf(H, W, wl.widths, wl.arch,
                                                                                 args.precision),
                         "executed_achieved": executed, "executed_frac": executed / peak},
            "clocks": main["clocks"],
        }
        if sweep:
            out["precisions"] = sweep
        if mis_alpha is not None:
            out["mis_alpha"] = mis_alpha
        if prec_block is not None:
            out["configs"] = {"precision": prec_block}
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(wl, args.cpu_sample_leaves, ocheck, maps, chi_bins,
                                               out.get("precisions"), mis=args.mis, kd=args.grid == "kd")
        if prec_block is not None and ocheck3 is not None:
            t0 = time.perf_counter()
            tm = ocheck3.run(threads=0)
            ocheck3.attach(prec_block["precisions"], maps3, chi3)
            prec_block["oracle"] = {"threads": tm["threads"], "leaves": int(len(ocheck3.slots)),
                                    "wall_s": round(time.perf_counter() - t0 + ocheck3.grid_s, 1),
                                    "what": "FP64 grid + splat of all photons, CNN + tables of the checked leaves"}
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_precision_config(args, wl, with_oracle=True):
    """Every CNN form (FP32, BF16, FP8 E4M3, FP8 inside / BF16 outside) on
    the precision workload (128x128 maps): the whole step timed as in the
    main line, and each form's sampling map on the checked leaves plus guided
    samples for the chi-square, kept for the comparison with the FP64
    oracle."""
    import torch

    from paper_2010_01775_gb300 import pg, synth
    ph, pos, dirs, blob = synth.workload_inputs(wl)
    n, q, H, W = wl.n_photons, wl.n_queries, wl.H, wl.W
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = pg.Context(stream.cuda_stream)
    net = pg.pg_net_load(ctx, blob)
    d_ph, d_pos, d_dir = (torch.from_numpy(a).cuda() for a in (ph, pos, dirs))
    o_d, o_p = torch.empty(q, 3, device="cuda"), torch.empty(q, device="cuda")
    o_l, o_b = torch.empty(q, dtype=torch.int32, device="cuda"), torch.empty(q, dtype=torch.int32, device="cuda")
    o_e = torch.empty(q, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ocheck = OracleCheck(wl) if with_oracle else None
    probe = ocheck.gpu_probe(ctx, pg, torch) if ocheck is not None else None

    def step(pr, marks=None, probe=None):
        rec = (lambda i: marks[i].record(stream)) if marks is not None else (lambda i: None)
        rec(0)
        g = pg.pg_build_grid(ctx, d_ph, n, LO, HI, wl.max_depth, wl.min_depth, wl.split_threshold)
        h = pg.pg_splat_photons(ctx, g, d_ph, n, wl.n_prev, H, W, wl.frac_bits)
        rec(1)
        m = pg.pg_reconstruct(ctx, h, net, pr)
        rec(2)
        t = pg.pg_build_cdf(ctx, m)
        pg.pg_sample_dirs(ctx, g, t, d_pos, q, 20101775, 0, o_d, o_p, o_l, o_b)
        pg.pg_eval_pdf(ctx, g, t, d_pos, d_dir, q, o_e)
        rec(3)
        A = g.info(pg.PG_INFO_N_ACTIVE)
        got = probe(g, t) if probe is not None else None
        for hd in (t, m, h, g):
            hd.free()
        return A, got

    g0 = pg.pg_build_grid(ctx, d_ph, n, LO, HI, wl.max_depth, wl.min_depth, wl.split_threshold)
    h0 = pg.pg_splat_photons(ctx, g0, d_ph, n, wl.n_prev, H, W, wl.frac_bits)
    if args.autotune:
        for pr in (pg.PG_BF16, pg.PG_FP8_E4M3, pg.PG_FP8_MIXED):
            pg.pg_autotune(ctx, h0, net, pr)
    h0.free()
    g0.free()
    names = {pg.PG_FP32: "fp32", pg.PG_BF16: "bf16", pg.PG_FP8_E4M3: "fp8", pg.PG_FP8_MIXED: "fp8mix"}
    ev = lambda: torch.cuda.Event(enable_timing=True)
    table, maps, bins = {}, {}, {}
    A = 0
    for pr in (pg.PG_FP32, pg.PG_BF16, pg.PG_FP8_E4M3, pg.PG_FP8_MIXED):
        steps = 2 if pr == pg.PG_FP32 else max(2, min(args.steps, 5))
        step(pr)
        ctx.sync()
        times, cnn = [], []
        for _ in range(steps):
            flush.zero_()
            marks = [ev() for _ in range(4)]
            A, _ = step(pr, marks)
            marks[3].synchronize()
            times.append(marks[0].elapsed_time(marks[3]))
            cnn.append(marks[1].elapsed_time(marks[2]))
        ms = float(np.mean(times))
        flops = unet_flops_per_leaf(H, W, wl.widths, wl.arch) * A
        table[names[pr]] = {"ms_per_step": ms, "value": q / (ms / 1e3), "unit": "samples/s",
                            "leaf_tables_per_s": A / (ms / 1e3), "cnn_ms": float(np.mean(cnn)),
                            "cnn_tflops": flops / (float(np.mean(cnn)) / 1e3) / 1e12}
        if probe is not None:
            _, got = step(pr, probe=probe)
            maps[names[pr]], bins[names[pr]] = got
    ctx.destroy()
    block = {"workload": wl.name, "H": H, "W": W, "active_leaves": int(A), "queries": q,
             "l2": "flushed between steps (256 MB write)", "precisions": table}
    return block, ocheck, maps, bins


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
            rs.append(srv.submit(make(spec, "fp32" if srv.fp32 else override)))
        for r in rs:
            r.wait()
        return rs

    # The served form: BF16 by default, the reduced-precision form that meets
    # KL <= 1e-3 against the oracle ("trace": the trace's own BF16/FP8 mix).
    override = None if args.serve_precision == "trace" else args.serve_precision
    precs = (override,) if override else tr.precisions
    out = {}
    srv = serve.Server(blob, workers=args.serve_workers, hbm_budget=120 << 30)
    srv.fp32 = False
    t = time.perf_counter()
    srv.warmup(warm_requests(precs), autotune=args.autotune)
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
    srv2.warmup(warm_requests(precs), autotune=args.autotune)
    same = serve.latency_summary(replay(srv2, trace[:k32], closed=True))
    srv2.close()
    out = {
        "metric": METRIC, "value": spec_rate["samples_per_s"], "unit": "samples/s", "n_gpus": 1,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"bf16": "bf16", "fp8": "fp8e4m3", "fp8mix": "fp8e4m3+bf16", "fp32": "f32"}.get(override, "bf16+fp8e4m3"),
        "data": "synthetic",
        "config": {"workload": tr.name, "requests": len(trace), "rate_per_s": tr.rate,
                   "served_precision": override or "the trace's BF16/FP8 alternation",
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


N_CHECK_LEAVES = 64    # leaves of the reduced-precision KL / L1 check, stratified by photon count
N_CHI_LEAVES = 8       # leaves of the sample chi-square check (a stratified subset of those)
CHI_SAMPLES = 65_536   # guided samples per chi-square leaf
KL_GATE = 1e-3         # mean-over-leaves KL(P_oracle || P_gpu) a reduced-precision form must meet
CHI_SEED = 20101775 ^ 0xC1


def host_cpu():
    """Core count and CPU model of this host (for the oracle's timings)."""
    model = None
    try:
        for line in subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return os.cpu_count() or 1, model


def stratified(counts, n):
    """n indices spread evenly over the ascending order of counts (every
    photon-count stratum from the emptiest leaf to the fullest)."""
    order = np.argsort(np.asarray(counts), kind="stable")
    k = np.unique(np.linspace(0, len(order) - 1, min(n, len(order))).round().astype(np.int64))
    return np.sort(order[k])


def leaf_centres(g, leaves):
    """Centre of each octree leaf: its first cell at full depth D (the Morton
    code's de-interleaved bits) plus half the leaf's edge, in the domain."""
    D = g["D"]
    codes = g["leaf_code"][leaves].astype(np.uint64)
    q = np.zeros((len(leaves), 3))
    for b in range(D):
        for a in range(3):
            q[:, a] += ((codes >> np.uint64(3 * b + a)) & np.uint64(1)).astype(np.float64) * float(1 << b)
    edge = 2.0 ** (D - g["leaf_depth"][leaves].astype(np.float64))
    lo, hi = np.asarray(g["lo"], np.float64), np.asarray(g["hi"], np.float64)
    return ((q + edge[:, None] / 2.0) / 2.0 ** D * (hi - lo) + lo).astype(np.float32)


def kl_l1(P_ref, P):
    """Per leaf KL(P_ref || P) and L1 = sum |P_ref - P| of maps [n][HW]."""
    kl, l1 = [], []
    for a in range(P_ref.shape[0]):
        p, qq = P_ref[a].ravel(), P[a].ravel().astype(np.float64)
        nz = p > 0
        kl.append(float(np.sum(p[nz] * np.log(p[nz] / np.maximum(qq[nz], 1e-300)))))
        l1.append(float(np.abs(p - qq).sum()))
    return np.array(kl), np.array(l1)


def chi_square(bins, P_ref, n_per_leaf):
    """Pearson chi-square of guided-sample bins against the oracle's map, per
    leaf: expected counts n P_k, bins with expectation below 5 pooled into one
    cell; returns (chi2 / dof per leaf, p-values)."""
    from scipy.stats import chi2 as chi2_dist
    red, pv = [], []
    for a in range(P_ref.shape[0]):
        b = bins[a * n_per_leaf:(a + 1) * n_per_leaf].astype(np.int64)
        obs = np.bincount(b[(b >= 0) & (b < P_ref.shape[1])], minlength=P_ref.shape[1]).astype(np.float64)
        exp = n_per_leaf * P_ref[a].ravel()
        big = exp >= 5.0
        o = np.append(obs[big], obs[~big].sum())
        e = np.append(exp[big], exp[~big].sum())
        keep = e > 0
        o, e = o[keep], e[keep]
        c2, dof = float(np.sum((o - e) ** 2 / e)), max(1, int(keep.sum()) - 1)
        red.append(c2 / dof)
        pv.append(float(chi2_dist.sf(c2, dof)))
    return np.array(red), np.array(pv)


class OracleCheck:
    """The FP64 oracle's sampling maps on leaves stratified by photon count,
    for the reduced-precision check of every GPU form: KL and L1 of its map
    against the oracle's (mean, p99, max over the leaves) and a chi-square of
    its guided samples, drawn at the centres of a subset of the leaves,
    against the oracle's pdf.  Which leaves are checked is decided here, from
    the oracle's own grid (bit-identical to the GPU's)."""

    def __init__(self, wl, n_leaves=N_CHECK_LEAVES, n_chi=N_CHI_LEAVES):
        from oracle import oracle as O
        from paper_2010_01775_gb300 import synth
        self.O, self.wl = O, wl
        self.ph, _, _, self.blob = _inputs(wl)
        t0 = time.perf_counter()
        self.g = O.build_grid(self.ph, LO, HI, wl.max_depth, wl.min_depth, wl.split_threshold)
        self.grid_s = time.perf_counter() - t0
        self.act, _ = O.active_leaves(self.g)
        counts = (self.g["leaf_end"].astype(np.int64) - self.g["leaf_begin"])[self.act]
        self.slots = stratified(counts, n_leaves)
        self.chi_idx = stratified(counts[self.slots], n_chi)  # rows of self.slots
        self.counts = counts[self.slots]
        self.chi_pos = np.ascontiguousarray(np.repeat(leaf_centres(self.g, self.act[self.slots[self.chi_idx]]),
                                                      CHI_SAMPLES, axis=0))
        self.P = None
        self.times = {}

    def gpu_probe(self, ctx, pg, torch):
        """A step hook: the GPU map on the checked leaves (slots) and the bins
        of CHI_SAMPLES guided samples at each chi-square leaf's centre."""
        d_pos = torch.from_numpy(self.chi_pos).cuda()
        qn = self.chi_pos.shape[0]
        o = (torch.empty(qn, 3, device="cuda"), torch.empty(qn, device="cuda"),
             torch.empty(qn, dtype=torch.int32, device="cuda"), torch.empty(qn, dtype=torch.int32, device="cuda"))
        slots = self.slots

        def probe(g, t):
            A, H, W = t.info(pg.PG_INFO_N_ACTIVE), t.info(pg.PG_INFO_H), t.info(pg.PG_INFO_W)
            P = t.export(pg.PG_TAB_P, np.float32, A * H * W).reshape(A, H * W)
            pg.pg_sample_dirs(ctx, g, t, d_pos, qn, CHI_SEED, 0, o[0], o[1], o[2], o[3])
            ctx.sync()
            return np.ascontiguousarray(P[slots]), o[3].cpu().numpy()
        return probe

    def run(self, threads=0):
        """The oracle's splat of every photon, then CNN and tables on the
        checked leaves; stage seconds in self.times."""
        O, wl = self.O, self.wl
        used = O.set_threads(threads)
        t0 = time.perf_counter()
        h = O.splat(self.ph, self.g, wl.n_prev, wl.H, wl.W, wl.frac_bits)
        t1 = time.perf_counter()
        y = O.cnn_forward(O.assemble_inputs(O.hist_for_active(h, self.act[self.slots])), O.parse_net(self.blob))
        t2 = time.perf_counter()
        self.P = O.tables_from_map(y)["P"].reshape(len(self.slots), -1)
        t3 = time.perf_counter()
        O.set_threads(0)
        self.times = dict(grid=self.grid_s, splat=t1 - t0, cnn=t2 - t1, cdf=t3 - t2, threads=used)
        return self.times

    def stats(self, P_gpu, bins=None):
        kl, l1 = kl_l1(self.P, P_gpu)
        out = {"kl_vs_fp64_oracle": {"mean": float(kl.mean()), "p99": float(np.percentile(kl, 99)),
                                     "max": float(kl.max()), "leaves": int(kl.size),
                                     "leaf_photons": [int(self.counts.min()), int(self.counts.max())],
                                     "selection": "stratified by leaf photon count"},
               "l1_vs_fp64_oracle": {"mean": float(l1.mean()), "p99": float(np.percentile(l1, 99)),
                                     "max": float(l1.max())},
               "kl_gate": KL_GATE, "meets_kl_gate": bool(kl.mean() <= KL_GATE)}
        if bins is not None:
            red, pv = chi_square(bins, self.P[self.chi_idx], CHI_SAMPLES)
            out["sample_chi2_vs_fp64_oracle"] = {
                "chi2_per_dof_mean": float(red.mean()), "chi2_per_dof_max": float(red.max()),
                "p_min": float(pv.min()), "leaves_p_above_0.01": int(np.sum(pv > 0.01)), "leaves": int(pv.size),
                "samples_per_leaf": CHI_SAMPLES}
        return out

    def attach(self, precisions, maps, bins):
        """Adds each form's check to its entry of the precision table."""
        for name, P in maps.items():
            precisions[name].update(self.stats(P, bins.get(name)))


_INPUTS = {}


def _inputs(wl):
    """The workload's seeded inputs, generated once per process (input
    generation is not part of any timed oracle stage)."""
    from paper_2010_01775_gb300 import synth
    if wl.name not in _INPUTS:
        _INPUTS[wl.name] = synth.workload_inputs(wl)
    return _INPUTS[wl.name]


def oracle_sample_run(wl, n_leaves, n_queries, check=None, mis=False, kd=False, threads=0):
    """The FP64 oracle on a bounded sample; returns per-stage seconds and the
    throughput extrapolated to the full workload.  check: an OracleCheck whose
    grid and leaves are reused (its maps are computed here)."""
    from oracle import oracle as O
    from paper_2010_01775_gb300 import synth
    used = O.set_threads(threads)
    ph, pos, dirs, blob = _inputs(wl)
    t0 = time.perf_counter()
    if check is not None:
        g, grid_s = check.g, check.grid_s
    elif kd:
        g = O.build_kd_grid(ph, synth.wall_normals(ph), LO, HI, KD_R, KD_DEPTH, KD_THR, KD_VTHR)
    else:
        g = O.build_grid(ph, LO, HI, wl.max_depth, wl.min_depth, wl.split_threshold)
    act, slot = O.active_leaves(g)
    t1 = time.perf_counter()
    if check is None:
        grid_s = t1 - t0
    keep = act[check.slots] if check is not None else act[np.linspace(0, act.size - 1, n_leaves).astype(np.int64)]
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
    if check is not None:
        check.P = tabs["P"].reshape(keep.size, -1)
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
    O.set_threads(0)
    A = act.size
    step_s = grid_s + splat_s + (t3 - t2) * A / keep.size + (t4 - t3) * A / keep.size + \
        (t5 - t4) * wl.n_queries / n_queries
    return dict(step_s=step_s, samples_per_s=wl.n_queries / step_s, wall_s=t5 - t0 + (grid_s if check else 0.0),
                leaves=int(keep.size), A=int(A), queries=n_queries, P=tabs["P"], threads=used,
                stage_s=dict(grid=grid_s, splat=splat_s, cnn=(t3 - t2) * A / keep.size,
                             cdf=(t4 - t3) * A / keep.size, sample_eval=(t5 - t4) * wl.n_queries / n_queries))


def cpu_baseline(wl, n_leaves, check=None, maps=None, bins=None, precisions=None, mis=False, kd=False):
    """The oracle timed on this host: single-threaded on a small sample, and
    on all cores (OpenMP over the convolution, sampling and evaluation loops;
    the grid and the splat stay sequential) on the checked leaves, whose maps
    then serve the reduced-precision check."""
    cores, model = host_cpu()
    nq = 65_536 if mis else 262_144
    r1 = oracle_sample_run(wl, n_leaves, nq, None, mis, kd, threads=1)
    rN = oracle_sample_run(wl, n_leaves, nq, check, mis, kd, threads=0)
    out = {"value": rN["samples_per_s"], "unit": "samples/s", "cores": rN["threads"], "kind": "oracle",
           "cpu": model, "nproc": cores,
           "value_1_thread": r1["samples_per_s"],
           "stage_s_full_step": {k: round(v, 3) for k, v in rN["stage_s"].items()},
           "sample": (f"FP64 oracle on {rN['threads']} threads (OpenMP over the convolution, sampling and "
                      f"evaluation loops; grid and splat sequential): grid+splat on all {wl.n_photons} photons"
                      f"{' (the splat on the sampled leaves, scaled by their photon share)' if kd else ''}, CNN+CDF on "
                      f"{rN['leaves']} of {rN['A']} active leaves"
                      f"{' (stratified by photon count)' if check is not None else ''}, "
                      f"{'MIS ' if mis else ''}sample+eval on {rN['queries']} of {wl.n_queries} queries; per-stage "
                      f"times scaled to the full step ({rN['step_s']:.1f} s; {r1['step_s']:.1f} s on one thread, "
                      f"from {r1['leaves']} leaves); wall {rN['wall_s'] + r1['wall_s']:.1f} s")}
    if check is not None and maps and precisions is not None:
        check.attach(precisions, maps, bins or {})
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
    """The oracle as it stands (FP64, this host's cores) on the main line's
    workload: every step is one bounded sample of it (grid + splat of every
    photon, CNN + tables on a few leaves, sample + eval on a slice of the
    queries), timed for real; `value` is the full step's rate extrapolated
    from that step's per-stage times."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    cores, model = host_cpu()
    runs = []
    for i in range(args.warmup + args.steps):
        r = oracle_sample_run(wl, REF_LEAVES, REF_QUERIES, threads=0)
        r["wall"] = r["wall_s"]  # the oracle's own stages, inputs already generated
        if i >= args.warmup:
            runs.append(r)
    value = wl.n_queries / statistics.mean(r["step_s"] for r in runs)
    wall_ms = statistics.mean(r["wall"] for r in runs) * 1e3
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "precision": "fp64 oracle"},
        "cpu_baseline": {"value": value, "unit": "samples/s", "cores": runs[0]["threads"], "kind": "oracle",
                         "cpu": model, "nproc": cores,
                         "sample": (f"per step (ms_per_step is its wall time): grid+splat on all {wl.n_photons} "
                                    f"photons (sequential), CNN+CDF on {REF_LEAVES} active leaves and sample+eval on "
                                    f"{REF_QUERIES} queries (OpenMP, {runs[0]['threads']} threads); value = "
                                    f"{wl.n_queries} queries / the full step extrapolated from the per-stage times")},
        "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


REF_LEAVES, REF_QUERIES = 8, 65_536


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
    ap.add_argument("--serve-precision", default="bf16", choices=["bf16", "fp8", "fp8mix", "trace"],
                    help="CNN form of the served requests (default BF16, the form within KL <= 1e-3 of the oracle; "
                         "'trace': the trace's own BF16/FP8 alternation)")
    ap.add_argument("--cpu-sample-leaves", type=int, default=4,
                    help="leaves of the single-thread oracle timing sample")
    ap.add_argument("--precision-config", action=argparse.BooleanOptionalAction, default=True,
                    help="also run every CNN form on the precision workload (128x128 maps) with its oracle check")
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
