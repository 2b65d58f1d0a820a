#!/usr/bin/env python
"""Benchmark of the NeuralVDB hot path on B300: decoded voxels/s (and training samples/s).

Workload (default "union1024"): narrow-band SDF (half-width 3) of the union of
32 spheres + 32 tori (seed 2) in a 1024^3 grid; three networks of 4 hidden
layers x 64 (ReLU), Fourier features n = 64, sigma = 10 cycles per 1024 voxels;
trained on the GPU (tensor-core BF16 step by default, --train-prec; batch 65536,
lr 1e-3 decayed 0.975 / 100 steps),
then decoded in full.

One timed step = one nvdb_decompress of the whole model: level-1 node origins
from the level-2 masks, level-1 classification of every leaf slot, patch XOR,
compaction to the leaf list, level-0 classification of every voxel of every
leaf, patch XOR, compaction to the voxel list, regression of every active voxel
(all kernels of the library).  Inputs (the model) are resident in HBM; the
output (16 B per voxel, > L2) is written every step and L2 is flushed between
steps.  `value` is measured at the precision --prec (default fp16: FP16 operands on
the tensor cores meet the 2e-2 x half-width error bar at one MMA per K step;
plain BF16 misses it, compensated BF16 (bf16x3) meets it at two to three MMAs
per K step); every precision's throughput and its decoded-SDF error against
the FP64 oracle on sampled voxels are reported under "by_precision".

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

PRECS = {"fp32": 0, "bf16": 1, "fp8": 2, "fp16": 3, "bf16x3": 4}
WORKLOAD_DESC = ("union of 32 spheres + 32 tori (seed 2), 1024^3, half-band 3; 3 nets 4x64 ReLU, "
                 "FFM n=64 sigma=10/1024vox; full decompress")
NET_WIDTH, NET_LAYERS, FFM = [64, 64, 64], [4, 4, 4], [64, 64]
TRAIN_KERNELS = ("train_fwd_bwd", "train_tc_bf16", "adam_reduce")


def aggregate_replicas(local_ms: float, units_per_rank: int, dist=None, device="cpu"):
    """Replicas (one process per GPU, the same work on each): the step time is the maximum
    over ranks and the value counts every rank's units -> (max ms per step, units/s)."""
    ms, world = local_ms, 1
    if dist is not None:
        t = torch.tensor([local_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms, world = float(t.item()), dist.get_world_size()
    return ms, world * units_per_rank / (ms / 1e3)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--prec", choices=list(PRECS), default="fp16")
    ap.add_argument("--train-steps", type=int, default=2500)
    ap.add_argument("--train-batch", type=int, default=65536)
    ap.add_argument("--train-prec", choices=["fp32", "bf16"], default="bf16")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=["union1024", "water2048"], default="union1024")
    ap.add_argument("--frames", type=int, default=48)
    return ap.parse_args()


def flops_per_eval(n_in: int, w: int, layers: int) -> int:
    """Algorithmic FLOPs of one network evaluation: 2(n w + (L-1) w^2 + w)."""
    return 2 * (n_in * w + (layers - 1) * w * w + w)


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        d["source"] = "measured"
        return d
    return dict(hbm_gbs=6400.0, bf16_tflops=1800.0, bf16_tflops_sustained=1400.0, source="fallback")


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        cvd = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        ids = [x.strip() for x in cvd.split(",") if x.strip()]
        self.index = ids[index] if index < len(ids) else str(index)
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        if not self.out:
            return None
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return dict(sm_mhz=statistics.median(sm), sm_max_mhz=mx, reasons=sorted(reasons), samples=len(sm))


# ----------------------------------------------------------------------------- oracle sample (CPU)
def oracle_decode_sample(ijk: np.ndarray, val: np.ndarray, model_from_blob, n_nodes: int, seed: int,
                         time_budget: float | None = None):
    """Full oracle decode of a seeded sample of level-1 nodes of the workload.

    Returns (active voxels decoded, seconds, nodes, threads).  The sample model keeps
    the networks of `model_from_blob` (or the oracle's initial networks if None) and
    the explicit upper tree restricted to the sampled level-1 nodes; its patches are
    computed by the oracle for those nodes (untimed).
    """
    from oracle import codec, vdb
    node = ijk.astype(np.int64) >> 7
    key = (node[:, 0] << 28) | (node[:, 1] << 14) | node[:, 2]
    uk = np.unique(key)
    rng = np.random.default_rng(seed)
    done_vox, secs, nodes = 0, 0.0, 0
    order = rng.permutation(len(uk))
    for i in order[: max(1, n_nodes)]:
        sel = key == uk[i]
        g = vdb.build(ijk[sel], val[sel])
        if model_from_blob is not None:
            m = dict(model_from_blob)
        else:
            m = codec.init_model(g, 0, 3.0, codec.default_opts(width=NET_WIDTH, layers=NET_LAYERS, ffm_size=FFM,
                                                               sigma=10.0, seed=1))
            o, l2e = vdb.domain(ijk)
            m["origin"], m["log2_extent"] = o, l2e
        m.update(l2_origin=g["l2_origin"], l2_mask=g["l2_mask"], n_l2=g["l2_origin"].shape[0],
                 n_l1=g["l1_origin"].shape[0], n_leaf=g["leaf_origin"].shape[0], n_active=g["n"], patches={})
        codec.make_patches(g, m, 0)
        t0 = time.perf_counter()
        dijk, _ = codec.decompress(m, 0)
        secs += time.perf_counter() - t0
        done_vox += len(dijk)
        nodes += 1
        if time_budget is not None and secs >= time_budget:
            break
    return done_vox, secs, nodes


def level_bytes(om: dict, prec: int) -> dict:
    """Bytes of the two lower levels, explicit against learned (the analogue of the paper's
    per-level memory table, Section 3.3): explicit level-1 child masks (512 B per node), leaf
    active masks (64 B per leaf) and voxel values (4 B per voxel), against the networks that
    replace each (FP32 parameters, every expert) plus the patch lists of precision `prec`
    (4 B offsets per node or leaf, 2 B per patch)."""
    n_l1, n_leaf, n = om["n_l1"], om["n_leaf"], om["n_active"]
    nets = om["nets"]
    par = [4 * sum(int(sum(np.size(w) for w in nets[k]["W"]) + sum(np.size(b) for b in nets[k]["b"]) +
                       np.size(nets[k]["wh"]) + 1) for k in range(j, len(nets), 3)) for j in range(3)]
    p = om["patches"][prec]
    n1, n0 = int(p["l1_off"][-1]), int(p["l0_off"][-1])
    explicit = dict(level1_child_masks=512 * n_l1, leaf_active_masks=64 * n_leaf, voxel_values=4 * n)
    learned = dict(level1_classifier=par[0] + 4 * (n_l1 + 1) + 2 * n1, level0_classifier=par[1] + 4 * (n_leaf + 1) + 2 * n0,
                   regressor=par[2], patches_level1=n1, patches_level0=n0)
    return dict(explicit=explicit, learned=learned,
                topology_ratio=(learned["level1_classifier"] + learned["level0_classifier"]) /
                (explicit["level1_child_masks"] + explicit["leaf_active_masks"]))


def sampling_error(nv, train_steps: int, n: int = 128, points: int = 1 << 20) -> dict:
    """Random-sampling error at equal in-memory footprint (Section 4.4): a dense 128^3 fBm
    density lattice encoded as [Hash,5,4,NN(3)] (explicit topology, regressor network)
    against an explicit grid of the same noise on a coarser lattice whose values and
    topology take about the same bytes, sampled with order 0, 1 and 3; RMSE against the
    continuous noise at 2^20 uniform points."""
    from fixtures import fbm_noise
    a = torch.arange(n, device="cuda")
    fine = torch.stack(torch.meshgrid(a, a, a, indexing="ij"), -1).reshape(-1, 3)
    fv = fbm_noise(fine).to(torch.float32)
    g = nv.build(fine.to(torch.int32).contiguous(), fv.contiguous(), 1, 0.0)
    info = g.info()
    m = nv.compress(g, seed=7, width=[32, 32, 64], layers=[3, 3, 4], ffm_size=[32, 64], ffm_sigma=6.0,
                    steps=train_steps, batch=65536, train_prec=1, patch_precs=(1 << 0) | (1 << 3))
    from oracle import blob
    om = blob.read(m.export())
    params = sum(int(sum(np.size(w) for w in net["W"]) + sum(np.size(b) for b in net["b"]) + np.size(net["wh"]) + 1)
                 for net in om["nets"][2:3])
    neural = 64 * info["n_leaf"] + 512 * info["n_l1"] + 4096 * info["n_l2"] + 4 * params

    def explicit_bytes(c):
        return 4 * c ** 3 + 64 * (-(-c // 8)) ** 3 + 512 * (-(-c // 128)) ** 3 + 4096
    c = max(c for c in range(4, n + 1) if explicit_bytes(c) <= neural)
    b = torch.arange(c, device="cuda")
    coarse = torch.stack(torch.meshgrid(b, b, b, indexing="ij"), -1).reshape(-1, 3)
    cv = fbm_noise(coarse.to(torch.float64) * ((n - 1) / (c - 1))).to(torch.float32)
    gc = nv.build(coarse.to(torch.int32).contiguous(), cv.contiguous(), 1, 0.0)
    r = torch.Generator(device="cuda").manual_seed(11)
    p = 2.0 + (n - 5.0) * torch.rand((points, 3), generator=r, device="cuda", dtype=torch.float64)
    truth = fbm_noise(p)
    pf = p.to(torch.float32).contiguous()
    pc = (p * ((c - 1) / (n - 1))).to(torch.float32).contiguous()
    out = dict(fine_lattice=n, coarse_lattice=c, neural_bytes=neural, explicit_bytes=explicit_bytes(c), points=points)
    for order in (0, 1, 3):
        v = nv.grid_sample(gc, pc, order).to(torch.float64)
        out[f"explicit_order{order}_rmse"] = float(torch.sqrt(torch.mean((v - truth) ** 2)))
    for name, prec in (("fp32", 0), ("fp16", 3)):
        v = nv.query(m, pf, prec).to(torch.float64)
        out[f"neural_{name}_rmse"] = float(torch.sqrt(torch.mean((v - truth) ** 2)))
    # the ray marcher on the same model: 512 x 512 pixels, 256 samples per ray (nvdb_render)
    cam = dict(eye=[-80.0, 150.0, -120.0], target=[64.0, 64.0, 64.0], up=[0.0, 1.0, 0.0], fov_deg=40.0, width=512,
               height=512, step=0.75, max_steps=256, sigma=0.05, prec=3)
    img = nv.render(m, **cam)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    nv.render(m, out=img, **cam)
    torch.cuda.synchronize()
    out["render"] = dict(pixels="512x512", samples_per_ray=256, precision="fp16", ms=1e3 * (time.perf_counter() - t0),
                         mean_transmittance=float(img[..., 1].mean()))
    return out


def blas_threads() -> int:
    try:
        from threadpoolctl import threadpool_info
        n = [d.get("num_threads", 1) for d in threadpool_info() if d.get("user_api") == "blas"]
        return int(max(n)) if n else 1
    except Exception:
        return os.cpu_count() or 1


# ----------------------------------------------------------------------------- reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from fixtures import workload
    # input generation only (torch elementwise ops, none of the library); then CPU oracle work
    ijk, val, _ = workload("union1024", device="cuda" if torch.cuda.is_available() else "cpu")
    ijk, val = ijk.cpu().numpy(), val.cpu().numpy()
    times, voxels = [], []
    for s in range(args.warmup + args.steps):
        v, t, _ = oracle_decode_sample(ijk, val, None, 1, seed=1000 + s)
        if s >= args.warmup:
            times.append(t)
            voxels.append(v)
    value = sum(voxels) / sum(times)
    thr = blas_threads()
    sample = f"per step: full oracle decode of 1 seeded level-1 node (mean {np.mean(voxels):.0f} voxels); initial weights"
    line = dict(impl="reference", metric="decoded voxels/s", value=value, unit="voxels/s", n_gpus=args.gpus,
                steps=args.steps, warmup=args.warmup, ms_per_step=1000.0 * float(np.mean(times)),
                higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(workload=WORKLOAD_DESC),
                cpu_baseline=dict(value=value, unit="voxels/s", cores=thr, kind="oracle", sample=sample),
                e2e=dict(value=value, unit="voxels/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line))
    return 0



# ----------------------------------------------------------------------------- animated workload
def run_water(args):
    """Config 'animated batching': 48 frames of a 2048x256x2048 water surface (8 seeded
    waves), each frame warm-started from the previous one (Section 3.6) with an early
    stop at frame 0's final loss; one graph-captured plan decodes all frames per step."""
    import paper_2208_04448_b300 as nv
    from fixtures import water_frame
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    shape = dict(width=NET_WIDTH, layers=NET_LAYERS, ffm_size=FFM, batch=args.train_batch, patch_precs=0b11111,
                 train_prec=PRECS[args.train_prec])
    grids, n_total = [], 0
    for f in range(args.frames):
        ijk, val = water_frame(f, device="cuda")
        grids.append(nv.build(ijk.contiguous(), val.contiguous(), 0, 3.0))
        n_total += grids[-1].info()["n_active"]
        del ijk, val
    sigma = 10.0 * (1 << grids[0].info()["log2_extent"]) / 1024.0
    # nvdb_compress_sequence: frame 0 cold (lr 1e-3), refined 500 steps at lr 1e-4, later frames
    # warm-started at 1e-4 with the early stop at frame 0's final loss (Section 3.6)
    nv.profile_read()
    nv.profile_enable(True)
    models = nv.compress_sequence(grids, refine_lr_scale=0.1, refine_steps=500, warm_steps=500, seed=1,
                                  ffm_sigma=sigma, steps=args.train_steps, lr=1e-3, stop_window=50, **shape)
    prof = nv.profile_read()
    nv.profile_enable(False)
    train_ms = sum(v[1] for k, v in prof.items() if k in TRAIN_KERNELS)
    del grids
    steps = np.array([[len(m.losses(k)) for k in range(3)] for m in models])
    steps[0] += args.train_steps   # frame 0: the cold steps before its refinement
    prec = PRECS[args.prec]
    plan = nv.decompress_plan(models, prec)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        plan.launch()
    plan.check()
    ms = []
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        for _ in range(args.steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            plan.launch()
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
    plan.check()
    mean_ms = float(np.mean(ms))
    cold = int(steps[0].sum())
    warm = steps[1:].sum(1) if len(steps) > 1 else np.array([cold])
    line = dict(metric="decoded voxels/s", value=n_total / (mean_ms / 1e3), unit="voxels/s", n_gpus=1,
                steps=args.steps, warmup=args.warmup, ms_per_step=mean_ms, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype=args.prec, data="synthetic",
                config=dict(workload=f"water surface 2048x256x2048, 8 seeded waves, {args.frames} frames, half-band 3; "
                                     "3 nets 4x64, FFM 64, sigma 10/1024vox; all frames decoded by one plan",
                            n_active_total=n_total, frames=args.frames, plan=plan.info()),
                warm_start=dict(cold_steps=cold, refine_steps=3 * 500, warm_steps_mean=float(warm.mean()),
                                step_speedup=cold / float(max(warm.mean(), 1)), steps_per_frame=steps.tolist()),
                train_samples_per_s=float(steps.sum() * args.train_batch / (train_ms / 1e3)) if train_ms else None,
                clocks=clk.summary())
    print(json.dumps(line))
    return 0

# ----------------------------------------------------------------------------- our arm
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "water2048":
        return run_water(args)

    import paper_2208_04448_b300 as nv
    from fixtures import workload
    from oracle import blob, codec

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    # ---- setup (untimed): volume, tree, training
    ijk, val, _ = workload("union1024", device="cuda")
    ijk, val = ijk.contiguous(), val.contiguous()
    g = nv.build(ijk, val, 0, 3.0)
    info = g.info()
    n_active, n_leaf, n_l1 = info["n_active"], info["n_leaf"], info["n_l1"]
    opts = dict(seed=1, width=NET_WIDTH, layers=NET_LAYERS, ffm_size=FFM,
                ffm_sigma=10.0 * (1 << info["log2_extent"]) / 1024.0, steps=args.train_steps,
                batch=args.train_batch, lr=1e-3, lr_decay=0.975, lr_interval=100, patch_precs=0b11111,
                train_prec=PRECS[args.train_prec])
    # training, end to end: compress with all steps minus compress with none (the same
    # setup and patch generation), unprofiled, so that chunks of steps replay as CUDA graphs
    def compress_wall(**kw):
        torch.cuda.synchronize()
        t = time.perf_counter()
        mdl = nv.compress(g, **dict(opts, **kw))
        torch.cuda.synchronize()
        return mdl, time.perf_counter() - t
    _, base_wall = compress_wall(steps=0)
    model, full_wall = compress_wall()
    train_wall = max(full_wall - base_wall, 1e-9)
    train_samples = 3 * args.train_steps * args.train_batch
    # per-kernel breakdown from a profiled run (every step launched, events per launch)
    prof_steps = min(args.train_steps, 200)
    nv.profile_read()
    nv.profile_enable(True)
    compress_wall(steps=prof_steps, patch_precs=1 << PRECS["fp16"])
    prof = nv.profile_read()
    nv.profile_enable(False)
    train_kern = {k: dict(launches=v[0], us_per_launch=1e3 * v[1] / max(v[0], 1)) for k, v in prof.items()
                  if k in TRAIN_KERNELS}
    train_ms = sum(v[1] for k, v in prof.items() if k in TRAIN_KERNELS)
    n_in, w_, L_ = FFM[1], NET_WIDTH[1], NET_LAYERS[1]
    f_net = 2 * (n_in * w_ + (L_ - 1) * w_ * w_ + w_)
    train_flops_per_sample = 3 * f_net - 2 * n_in * w_          # forward, dW, delta (not into the encoding)
    train_tflops = 3 * prof_steps * args.train_batch * train_flops_per_sample / (train_ms / 1e3) / 1e12 if train_ms else None
    blob_bytes = model.export()

    out_ijk = torch.empty((n_active, 3), dtype=torch.int32, device="cuda")
    out_val = torch.empty(n_active, dtype=torch.float32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # 256 MB > 126 MB L2
    stream = torch.cuda.current_stream()

    def decode(prec):
        nv.decompress(model, prec, out=(out_ijk, out_val))

    def timed(prec, steps, profile=False):
        for _ in range(args.warmup):
            decode(prec)
        torch.cuda.synchronize()
        if profile:
            nv.profile_read()
            nv.profile_enable(True)
        ms = []
        l0 = nv.launch_count()
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            decode(prec)
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        launches = nv.launch_count() - l0
        kern = None
        if profile:
            kern = nv.profile_read()
            nv.profile_enable(False)
        return ms, launches, kern

    # decoded-value error against the oracle on sampled voxels, per precision
    om = blob.read(blob_bytes)
    rs = np.random.default_rng(7)

    def decode_error(prec):
        decode(prec)
        torch.cuda.synchronize()
        idx = rs.choice(n_active, size=min(4096, n_active), replace=False)
        pi = out_ijk[torch.from_numpy(idx).cuda()].cpu().numpy()
        pv = out_val[torch.from_numpy(idx).cuda()].cpu().numpy().astype(np.float64)
        want = codec.evaluate(om, codec.REG, pi) * 3.0
        return float(np.abs(pv - want).max())

    by_prec = {}
    head_prec = PRECS[args.prec]
    kern_by_prec = {}
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for name, p in PRECS.items():
            ms, launches, kern = timed(p, args.steps, profile=True)
            by_prec[name] = dict(ms_per_step=float(np.mean(ms)), voxels_per_s=n_active / (np.mean(ms) / 1e3),
                                 launches_per_step=launches / args.steps)
            kern_by_prec[name] = kern
            if p == head_prec:
                head_ms, head_launches, head_kern = ms, launches, kern
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    for name, p in PRECS.items():
        by_prec[name]["max_abs_err_vs_oracle"] = decode_error(p)
        by_prec[name]["err_bound"] = 0.02 * 3.0
        by_prec[name]["meets_bar"] = by_prec[name]["max_abs_err_vs_oracle"] <= by_prec[name]["err_bound"]

    # ---- point queries (Section 3.5 random access): 2^22 points uniform in occupied level-1 nodes
    from fixtures import query_points
    qpts = query_points(ijk, 1 << 22, seed=5).cuda().contiguous()
    qout = torch.empty(qpts.shape[0], dtype=torch.float32, device="cuda")
    query = {}
    for name, p in PRECS.items():
        for _ in range(2):
            nv.query(model, qpts, p, out=qout)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(5):
            nv.query(model, qpts, p, out=qout)
        b.record(stream)
        b.synchronize()
        query[name] = dict(points_per_s=5 * qpts.shape[0] / (a.elapsed_time(b) / 1e3))

    mean_ms, value = aggregate_replicas(float(np.mean(head_ms)), n_active, dist, "cuda")

    # ---- roofline of the dominant network kernel (live CUDA events on the launching stream)
    peaks = measured_peaks()

    def roofline(kern):
        mlp = {k: v for k, v in kern.items() if k.startswith("mlp_") and "." in k}
        name, (nl, tms) = max(mlp.items(), key=lambda kv: kv[1][1])
        per = {"L0": n_leaf * 512 * flops_per_eval(FFM[1], NET_WIDTH[1], NET_LAYERS[1]),
               "L1": n_l1 * 4096 * flops_per_eval(FFM[0], NET_WIDTH[0], NET_LAYERS[0]),
               "list": n_active * flops_per_eval(FFM[1], NET_WIDTH[2], NET_LAYERS[2])}[name.split(".")[1]]
        ach = per / (tms / nl / 1e3) / 1e12
        if name.startswith("mlp_f32"):
            pk = 148 * 128 * 2 * peaks.get("sm_max_mhz", 2032.0) * 1e6 / 1e12
            bd, src = "alu", "derived: 148 SMs x 128 FFMA/clk x 2 x max SM clock"
        elif name.startswith("mlp_fp8"):
            # first layer on kind::f16, hidden layers on kind::f8f6f4 at the nominal 2x rate: the
            # peak is the rate at which these FLOPs would run with every MMA at its own peak
            lev = name.split(".")[1]
            nin, w, L = (FFM[0], NET_WIDTH[0], NET_LAYERS[0]) if lev == "L1" else (FFM[1], NET_WIDTH[1], NET_LAYERS[1])
            f_first, f_hidden = 2 * nin * w, 2 * (L - 1) * w * w
            pk = peaks["bf16_tflops"] * (f_first + f_hidden) / (f_first + f_hidden / 2.0)
            bd, src = "tensor", (f"{peaks['source']} bf16 burst; hidden layers at the nominal 2x kind::f8f6f4 rate "
                                 f"(weighted by their FLOPs)")
        else:
            pk = peaks["bf16_tflops"]
            bd, src = "tensor", f"{peaks['source']} bf16 burst (16-bit kind::f16 rate)"
        return dict(kernel=name, bound=bd, achieved=ach, peak=pk, unit="TFLOP/s", frac=ach / pk,
                    flops_per_launch=per, avg_launch_ms=tms / nl, peak_source=src)

    rl = roofline(head_kern)
    dname = rl["kernel"]

    # ---- compaction against the measured HBM copy bandwidth: the level-0 single-pass kernel
    # (patches, counts, look-back scan and the voxel coordinates in one launch); algorithmic
    # bytes per launch: leaf words 64 B read and 64 B written, origin 16 B, patch offset 4 B and
    # voxel offset 8 B per leaf, 2 B per patch, 12 B written per voxel
    n0_patches = int(om["patches"][head_prec]["l0_off"][-1])
    comp_bytes = {"patch_scan_l0": 12 * n_active + 156 * n_leaf + 2 * n0_patches}
    compaction = {}
    for kname, nbytes in comp_bytes.items():
        if kname in head_kern:
            nl, tms = head_kern[kname]
            gbs = nbytes / (tms / nl / 1e3) / 1e9
            compaction[kname] = dict(bytes_per_launch=nbytes, avg_launch_us=1e3 * tms / nl, achieved_gbs=gbs,
                                     frac_of_hbm=gbs / peaks["hbm_gbs"])
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tfile):
        with open(tfile) as f:
            traffic = json.load(f).get(dname)

    # ---- bytes per level (explicit vs learned), undecomposed and with 512^3 subdomains
    # (Section 3.4: one expert per occupied subdomain, 8-voxel halo), whose decode is also timed
    bytes_levels = level_bytes(om, head_prec)
    moe_model = nv.compress(g, **dict(opts, subdomain=512, halo=8, patch_precs=1 << head_prec))
    om_moe = blob.read(moe_model.export())
    for _ in range(args.warmup):
        nv.decompress(moe_model, head_prec, out=(out_ijk, out_val))
    torch.cuda.synchronize()
    moe_ms = []
    for _ in range(max(3, args.steps // 2)):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        nv.decompress(moe_model, head_prec, out=(out_ijk, out_val))
        b.record(stream)
        b.synchronize()
        moe_ms.append(a.elapsed_time(b))
    idx = rs.choice(n_active, size=min(4096, n_active), replace=False)
    pi = out_ijk[torch.from_numpy(idx).cuda()].cpu().numpy()
    pv = out_val[torch.from_numpy(idx).cuda()].cpu().numpy().astype(np.float64)
    moe_err = float(np.abs(pv - codec.evaluate(om_moe, codec.REG, pi) * 3.0).max())
    decomposed = dict(subdomain=512, halo=8, experts=moe_model.info()["n_experts"], precision=args.prec,
                      ms_per_step=float(np.mean(moe_ms)), voxels_per_s=n_active / (np.mean(moe_ms) / 1e3),
                      max_abs_err_vs_oracle=moe_err, bytes_per_level=level_bytes(om_moe, head_prec),
                      final_loss=[float(np.mean(np.concatenate([moe_model.losses(3 * e + j)[-50:]
                                                                 for e in range(moe_model.info()["n_experts"])])))
                                  for j in range(3)] if args.train_steps else None)

    # ---- random-sampling error at equal footprint (Section 4.4), and the ray marcher
    samp_err = sampling_error(nv, args.train_steps)

    # ---- end to end through the C ABI with host buffers
    # input: the compressed model as shipped for this precision (the same deterministic
    # training, only this precision's patch set) in pinned host memory; output: the
    # voxels and values in pinned host memory (nvdb_decompress_host: the voxel copy
    # overlaps the regression)
    e2e_blob = nv.compress(g, **dict(opts, patch_precs=1 << head_prec)).export()
    blob_pinned = torch.frombuffer(bytearray(e2e_blob), dtype=torch.uint8).pin_memory()
    h_ijk = torch.empty((n_active, 3), dtype=torch.int32, pin_memory=True)
    h_val = torch.empty(n_active, dtype=torch.float32, pin_memory=True)
    e2e_ms = []
    for s in range(args.warmup + max(3, args.steps // 5)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m2 = nv.model_import(blob_pinned)
        nv.decompress_host(m2, head_prec, host=(h_ijk, h_val), out=(out_ijk, out_val))
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        del m2
        if s >= args.warmup:
            e2e_ms.append(dt * 1e3)
    e2e_value = world * n_active / (np.mean(e2e_ms) / 1e3)

    # ---- CPU baseline: the oracle on a bounded sample (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        hi, hv = ijk.cpu().numpy(), val.cpu().numpy()
        v, secs, nodes = oracle_decode_sample(hi, hv, om, 64, seed=11, time_budget=args.cpu_seconds)
        cpu = dict(value=v / secs, unit="voxels/s", cores=blas_threads(), kind="oracle",
                   sample=f"full FP64 oracle decode of {nodes} seeded level-1 nodes ({v} voxels, {secs:.1f} s)")

    clocks = clk.summary()
    line = dict(
        metric="decoded voxels/s", value=value, unit="voxels/s", n_gpus=world, steps=args.steps,
        warmup=args.warmup, ms_per_step=mean_ms, higher_is_better=True, scaling="weak", vs_baseline=None,
        dtype=args.prec, data="synthetic",
        config=dict(workload=WORKLOAD_DESC, n_active=n_active, n_leaf=n_leaf, n_l1=n_l1,
                    precision=args.prec, l2="flushed (256 MB write) between timed steps; output 16 B/voxel",
                    parallelism="replicas only" if world > 1 else "1 GPU"),
        roofline=dict(rl, traffic=traffic),
        roofline_by_precision={k: roofline(v) for k, v in kern_by_prec.items()},
        query=query,
        cpu_baseline=cpu,
        e2e=dict(value=e2e_value, unit="voxels/s", h2d_bytes_per_step=len(e2e_blob),
                 d2h_bytes_per_step=16 * n_active),
        gpu_launches=int(head_launches),
        clocks=clocks,
        train_samples_per_s=train_samples / train_wall if args.train_steps else None,
        train=dict(steps=args.train_steps, batch=args.train_batch, wall_s=train_wall, precision=args.train_prec,
                   samples_per_s="end to end: (compress wall - compress wall with 0 steps), chunks of 50 steps "
                                 "replayed as CUDA graphs",
                   kernels=train_kern, kernel_tflops=train_tflops,
                   kernel_frac_of_peak=(train_tflops / peaks["bf16_tflops"]) if train_tflops else None,
                   flops_per_sample=train_flops_per_sample,
                   final_loss=[float(np.mean(model.losses(k)[-50:])) for k in range(3)] if args.train_steps else None),
        by_precision=by_prec,
        bytes_per_level=bytes_levels,
        sampling_error=samp_err,
        decomposed=decomposed,
        kernels={k: dict(launches=v[0], ms=v[1]) for k, v in sorted(head_kern.items(), key=lambda kv: -kv[1][1])},
        compaction=compaction,
    )
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
