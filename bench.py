"""Benchmark of the fV-SRN render / fit path on GB300.

Workload (N = 1): the config-2 scene.  A 256^3 fractal-noise volume, an
fV-SRN with a 32^3 x 16 FP16 latent grid, 14 Fourier features and 4 SnakeAlt
layers of width 32, fitted to the volume by the library's own fit kernels,
rendered at 1024 x 1024 with step 1/512, an 8-point TF and early termination
at 0.99.  One step = one 1024^2 frame (views cycle over 8 orbit cameras).

Headline metric: network samples/s (device-counted network evaluations /
device time).  Also reported: ms/frame of fV-SRN vs dense-grid DVR of the
same volume with the PSNR between them, and fit steps/s (config 3).

--impl reference times the FP64 CPU oracle (the only reference there is) on
a bounded sample of the same workload, on the host cores.
"""
from __future__ import annotations

import argparse
import collections
import csv
import json
import math
import os
import platform
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "network samples/s and ms/frame @1024² (fV-SRN vs dense DVR, PSNR stated); fit steps/s"
W_IMG = H_IMG = 1024
STEP = 1.0 / 512
ET = 0.99
N_VIEWS = 8
FIT_STEPS = 2000
FIT_POINTS = 1 << 18
WORKLOAD = "cfg2: 256^3 fractal noise; fV-SRN 32^3x16 fp16 grid, m=14, 4x32 SnakeAlt; 1024^2, step 1/512, 8-pt TF, ET 0.99"


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def rank_views(k, rank, world, n_views=N_VIEWS):
    """View of timed frame k on a rank: ranks walk the orbit with disjoint
    offsets, so N replicas render N different frames per step (weak scaling;
    no data crosses ranks)."""
    return (k * world + rank) % n_views


def aggregate(t_seconds, samples, world, device):
    """Whole-job timing over ranks: the slowest rank's time and the sum of
    the samples all ranks took (a max and a sum all-reduce, nothing else)."""
    if world <= 1:
        return t_seconds, samples
    import torch
    import torch.distributed as dist
    t = torch.tensor([t_seconds], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    n = torch.tensor([float(samples)], device=device, dtype=torch.float64)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), int(n.item())


def seeded_params(seed=0):
    """The config-2 network with seeded weights (Xavier-uniform weights, zero
    biases, latent grid N(0, 0.01^2)), rounded to FP16: the network both
    bench arms render for the headline line."""
    from paper_2112_01579_gb300 import synth
    return synth.to_half_exact(synth.init_params(R=32, F=16, m=14, layers=4, width=32, out_dim=1,
                                                 act=synth.ACT_SNAKEALT, seed=seed))


def setup_scene(device="cuda", fit_steps=FIT_STEPS, seed=0):
    """Volume, fitted network (FP16 render copy), TF and cameras of config 2."""
    import torch
    from paper_2112_01579_gb300 import srn, synth
    vol = synth.noise_volume(256, seed=seed, device=device).contiguous()
    p = synth.init_params(R=32, F=16, m=14, layers=4, width=32, out_dim=1, act=synth.ACT_SNAKEALT, seed=seed)
    net = srn.Network(p, precision=srn.SRN_PREC_FP16, max_fit_points=FIT_POINTS, adam=True)
    fit_info = {"steps": 0}
    loss = torch.zeros(1, device=device)
    try:
        t0 = time.time()
        srn.srn_fit_steps(net.ctx, vol, FIT_POINTS, seed + 1, 0, fit_steps, loss, lr_grid=1e-2, lr_net=5e-3)
        torch.cuda.synchronize()
        fit_info = {"steps": fit_steps, "final_loss": float(loss.item()), "wall_s": time.time() - t0}
    except srn.SrnError as e:
        fit_info = {"steps": 0, "unavailable": str(e)}
    srn.srn_sync_half(net.ctx)
    return vol, net, synth.tf_preset(8), synth.orbit_cameras(N_VIEWS), fit_info


def vertex_points(n, device="cuda"):
    """Positions of the n^3 grid vertices, x fastest (the volume's layout)."""
    import torch
    x = torch.linspace(0.0, 1.0, n, device=device)
    Z, Y, X = torch.meshgrid(x, x, x, indexing="ij")
    return torch.stack([X.reshape(-1), Y.reshape(-1), Z.reshape(-1)], dim=1).contiguous()


def density_psnr_network(net, vol, pts):
    """PSNR of the network's density at every vertex of the volume."""
    import torch
    from paper_2112_01579_gb300 import srn
    out = torch.empty((pts.shape[0], net.out_dim), device=vol.device)
    srn.srn_eval(net.ctx, pts, out)
    mse = torch.zeros(1, dtype=torch.float64, device=vol.device)
    srn.srn_density_mse(out[:, 0].contiguous(), vol.reshape(-1), mse)
    torch.cuda.synchronize()
    return 10 * math.log10(1.0 / max(mse.item(), 1e-30))


def lowpass_baseline(vol, R, F):
    """Equal-memory density grid (Section 6.2 'off' row): M = round(cbrt(R^3 F)),
    returned with its density PSNR at the volume's vertices."""
    import torch
    from paper_2112_01579_gb300 import srn
    M = int(round((R ** 3 * F) ** (1.0 / 3.0)))
    tmp = torch.empty(2 * vol.numel(), device=vol.device)
    grid = torch.empty((M, M, M), device=vol.device)
    srn.srn_lowpass_resample(vol, M, tmp, grid)
    back = torch.empty_like(vol)
    srn.srn_resample(grid, back)
    mse = torch.zeros(1, dtype=torch.float64, device=vol.device)
    srn.srn_density_mse(back, vol, mse)
    torch.cuda.synchronize()
    return M, grid, 10 * math.log10(1.0 / max(mse.item(), 1e-30))


def fit_cfg3(vol, pts, steps=FIT_STEPS, seed=0):
    """Config 3: the plain-workload network (8^3 x 8 grid, m = 12, 2 sine
    layers) fitted to the volume, 2^18 points per step.  The same fit runs
    twice from the same initial state: one srn_fit_step call per step, then
    srn_fit_steps (one captured step replayed as a CUDA graph), whose final
    state must equal the first's bit for bit.  Returns steps/s of both (device
    time of all steps), final loss and density PSNR."""
    import torch
    from paper_2112_01579_gb300 import srn, synth
    p = synth.init_params(R=8, F=8, m=12, layers=2, width=32, act=synth.ACT_SINE, seed=seed)
    net = srn.Network(p, precision=srn.SRN_PREC_FP32, max_fit_points=FIT_POINTS, adam=True)
    loss = torch.zeros(1, device=vol.device)
    init = [t.clone() for t in (net.grid, net.weights, net.biases)]

    def reset():
        for t, t0 in zip((net.grid, net.weights, net.biases), init):
            t.copy_(t0)
        net.adam_m.zero_()
        net.adam_v.zero_()
        torch.cuda.synchronize()

    # warm-up with the timed arguments (this also captures the graph), then back to the initial state
    for s in range(3):
        srn.srn_fit_step(net.ctx, vol, FIT_POINTS, seed + 1, s, loss, lr_grid=1e-2, lr_net=5e-3)
    srn.srn_fit_steps(net.ctx, vol, FIT_POINTS, seed + 1, 0, 3, loss, lr_grid=1e-2, lr_net=5e-3)
    reset()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for s in range(steps):
        srn.srn_fit_step(net.ctx, vol, FIT_POINTS, seed + 1, s, loss, lr_grid=1e-2, lr_net=5e-3)
    e1.record()
    torch.cuda.synchronize()
    single_sps = steps / (e0.elapsed_time(e1) / 1e3)
    single = [t.clone() for t in (net.grid, net.weights, net.biases, loss)]
    reset()
    e0.record()
    srn.srn_fit_steps(net.ctx, vol, FIT_POINTS, seed + 1, 0, steps, loss, lr_grid=1e-2, lr_net=5e-3)
    e1.record()
    torch.cuda.synchronize()
    st, msg = srn.srn_sync_status(net.ctx)
    sps = steps / (e0.elapsed_time(e1) / 1e3)
    same = all(torch.equal(a, b) for a, b in zip(single, (net.grid, net.weights, net.biases, loss)))
    M, _, lp_psnr = lowpass_baseline(vol, 8, 8)
    res = {"steps": steps, "points_per_step": FIT_POINTS, "steps_per_s": sps, "api": "srn_fit_steps (graph replay)",
           "steps_per_s_single_calls": single_sps, "graph_equals_single_calls": same,
           "final_loss": float(loss.item()), "density_psnr_db": density_psnr_network(net, vol, pts),
           "lowpass_grid": M, "lowpass_density_psnr_db": lp_psnr, "status": st}
    pk = peaks()
    tf_ach = sps * FIT_POINTS * FIT_FLOP_PER_POINT / 1e12
    gb_ach = sps * FIT_POINTS * FIT_GATHER_BYTES_PER_POINT / 1e9
    res["roofline"] = {"bound": "latency", "tensor": {"achieved": tf_ach, "peak": pk.get("bf16_tflops"),
                                                      "unit": "TFLOP/s", "flop_per_point": FIT_FLOP_PER_POINT,
                                                      "frac": tf_ach / pk["bf16_tflops"] if pk.get("bf16_tflops") else None},
                       "gather": {"achieved": gb_ach, "unit": "GB/s", "bytes_per_point": FIT_GATHER_BYTES_PER_POINT,
                                  "hbm_frac": gb_ach / pk["hbm_gbs"] if pk.get("hbm_gbs") else None},
                       "note": "eight short dependent kernels per step (2-15 us each): launch and tail latency, "
                               "not a unit's throughput, set the rate"}
    net.close()
    return res


def point_eval(net, vol, n=1 << 20, seed=0):
    """Random-access reconstruction (the paper's evaluation of 10^6 random
    locations): 2^20 uniform points of the fitted render network, FP16
    tensor-core eval, FP32 eval, and FP32 density + adjoint gradient; ms per
    call (L2 flushed) and the density PSNR at the points against the
    trilinear volume."""
    import torch
    from paper_2112_01579_gb300 import srn
    g = torch.Generator(device=vol.device).manual_seed(seed)
    pts = torch.rand((n, 3), device=vol.device, generator=g)
    ref = torch.nn.functional.grid_sample(vol[None, None], (pts * 2 - 1).view(1, 1, 1, n, 3),
                                          align_corners=True).view(-1).contiguous()
    out = torch.empty((n, 1), device=vol.device)
    grad = torch.empty((n, 3), device=vol.device)
    rho = torch.empty(n, device=vol.device)
    n32 = srn.Network(net.unpack(), precision=srn.SRN_PREC_FP32)
    mse = torch.zeros(1, dtype=torch.float64, device=vol.device)
    res = {"workload": f"{n} uniform random points of the fitted cfg2 network"}
    for name, fn, o in (("eval_fp16_tensor", lambda: srn.srn_eval(net.ctx, pts, out), out),
                        ("eval_fp32", lambda: srn.srn_eval(n32.ctx, pts, out), out),
                        ("density_grad_fp32", lambda: srn.srn_density_grad(n32.ctx, pts, rho, grad), rho)):
        ms = _time_frames(fn, n=5)
        fn()
        srn.srn_density_mse(o.reshape(-1).contiguous(), ref, mse)
        torch.cuda.synchronize()
        res[name] = {"ms": ms, "points_per_s": n / (ms / 1e3),
                     "density_psnr_db": 10 * math.log10(1.0 / max(mse.item(), 1e-30))}
    n32.close()
    return res


def fit_adaptive(vol, pts, steps=FIT_STEPS, seed=0, every=50, res=128, spv=8):
    """Section 6.2 adaptive resampling on the config-2 fit: the render
    network fitted with uniform points and with points drawn in proportion
    to the error grid (res^3 voxels, spv positions each, recomputed every
    `every` steps; the first `every` steps are uniform).  Reports density
    PSNR, the mean and 99th percentile of the final error grid, and the time
    of the fit with the error-grid passes included."""
    import torch
    from paper_2112_01579_gb300 import srn, synth
    out = {"workload": f"cfg2 fit, {steps} steps x {FIT_POINTS} points; error grid {res}^3 x {spv}, every {every}"}
    E = torch.zeros(res ** 3, device=vol.device)
    for mode in ("uniform", "adaptive"):
        p = synth.init_params(R=32, F=16, m=14, layers=4, width=32, out_dim=1, act=synth.ACT_SNAKEALT, seed=seed)
        net = srn.Network(p, precision=srn.SRN_PREC_FP16, max_fit_points=FIT_POINTS, adam=True)
        loss = torch.zeros(1, device=vol.device)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        grid_ms = []
        e0.record()
        for s in range(0, steps, every):
            if mode == "adaptive" and s > 0:
                g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                g0.record()
                srn.srn_error_grid(net.ctx, vol, res, spv, seed + s, E)
                srn.srn_fit_set_sampling(net.ctx, E, res)
                g1.record()
                grid_ms.append((g0, g1))
            srn.srn_fit_steps(net.ctx, vol, FIT_POINTS, seed + 1, s, min(every, steps - s), loss, lr_grid=1e-2,
                              lr_net=5e-3)
        e1.record()
        torch.cuda.synchronize()
        srn.srn_error_grid(net.ctx, vol, res, spv, seed + 99991, E)
        torch.cuda.synchronize()
        e_np = E.cpu().numpy()
        srn.srn_sync_half(net.ctx)
        out[mode] = {"fit_ms": e0.elapsed_time(e1), "final_loss": float(loss.item()),
                     "density_psnr_db": density_psnr_network(net, vol, pts),
                     "error_grid_mean": float(e_np.mean()), "error_grid_p99": float(np.percentile(e_np, 99)),
                     "error_grid_max": float(e_np.max())}
        if grid_ms:
            out[mode]["error_grid_and_cdf_ms"] = float(np.median([a.elapsed_time(b) for a, b in grid_ms]))
        net.close()
    return out


def run_ours(args, rank, world):
    import torch
    from paper_2112_01579_gb300 import srn
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    vol, net, tf, cams, fit_info = setup_scene(fit_steps=args.fit_steps)
    # the headline renders the seeded network (the one the reference arm's
    # oracle renders); the fitted network's figures are reported beside it
    seeded = srn.Network(seeded_params(), precision=srn.SRN_PREC_FP16)
    prec_name = "fp16-mma"
    desc = srn.render_desc(W_IMG, H_IMG, STEP, ET)
    out = torch.zeros((1, 1, H_IMG, W_IMG, 4), device=dev)
    ctr = torch.zeros(1, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()
    # no fallback: the tensor-core kernel must cover the workload
    srn.srn_render(seeded.ctx, cams[:1], tf, desc, out, samples=ctr)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MiB > L2

    def frame(k, samples=None, which=seeded):
        srn.srn_render(which.ctx, [cams[rank_views(k, rank, world)]], tf, desc, out, samples=samples)

    for k in range(args.warmup):
        frame(k)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ctr.zero_()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clk:
        for k in range(args.steps):
            flush.zero_()
            evs[k][0].record(stream)
            frame(k, ctr)
            evs[k][1].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms = [a.elapsed_time(b) for a, b in evs]
    t_total = sum(ms) / 1e3
    samples = int(ctr.item())
    t_total, samples = aggregate(t_total, samples, world, dev)
    value = samples / t_total
    ms_frame = t_total * 1e3 / args.steps

    # the same frames with the network fitted to the volume
    fctr = torch.zeros(1, dtype=torch.int64, device=dev)
    f_ms = []
    for k in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        frame(k, fctr, which=net)
        b.record(stream)
        torch.cuda.synchronize()
        f_ms.append(a.elapsed_time(b))
    fitted_frames = {"ms_per_frame": float(np.mean(f_ms)),
                     "samples_per_s": int(fctr.item()) / (sum(f_ms) / 1e3),
                     "samples_per_frame": int(fctr.item()) / args.steps}

    # dense-grid DVR of the same volume and PSNR between the two renderers
    dense = torch.zeros_like(out[0])
    dctr = torch.zeros(1, dtype=torch.int64, device=dev)
    srn.srn_dvr_dense(vol, cams[:1], tf, desc, dense)
    torch.cuda.synchronize()
    d_ms = []
    for k in range(max(3, args.steps // 2)):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        srn.srn_dvr_dense(vol, [cams[k % N_VIEWS]], tf, desc, dense, samples=dctr)
        b.record(stream)
        torch.cuda.synchronize()
        d_ms.append(a.elapsed_time(b))
    # learned vs plain at equal memory (Section 6.2): the fitted fV-SRN and
    # the low-pass density grid of the latent grid's memory, both against
    # dense DVR of the full volume
    M, lp_grid, lp_dpsnr = lowpass_baseline(vol, 32, 16)
    lp_img = torch.zeros_like(out[0])
    psnrs, lp_psnrs, ssims, lp_ssims = [], [], [], []
    mse = torch.zeros(1, dtype=torch.float64, device=dev)
    ssim = torch.zeros(1, dtype=torch.float64, device=dev)
    for v in range(N_VIEWS):
        srn.srn_render(net.ctx, [cams[v]], tf, desc, out)
        srn.srn_dvr_dense(vol, [cams[v]], tf, desc, dense)
        srn.srn_image_mse(out, dense, mse)
        srn.srn_image_ssim(out[0, 0], dense[0], ssim)
        torch.cuda.synchronize()
        psnrs.append(10 * math.log10(1.0 / max(mse.item(), 1e-30)))
        ssims.append(ssim.item())
        srn.srn_dvr_dense(lp_grid, [cams[v]], tf, desc, lp_img)
        srn.srn_image_mse(lp_img, dense, mse)
        srn.srn_image_ssim(lp_img[0], dense[0], ssim)
        torch.cuda.synchronize()
        lp_psnrs.append(10 * math.log10(1.0 / max(mse.item(), 1e-30)))
        lp_ssims.append(ssim.item())
    pts = vertex_points(vol.shape[0])
    fvsrn_dpsnr = density_psnr_network(net, vol, pts)
    # the paper's 8-bit latent grid (Section 4.2) on the same fitted network
    n8 = srn.Network(net.unpack(), precision=srn.SRN_PREC_FP16, grid_u8=True)
    c8 = torch.zeros(1, dtype=torch.int64, device=dev)
    ms8 = _time_frames(lambda: srn.srn_render(n8.ctx, cams[:1], tf, desc, out, samples=c8), n=5)
    c8.zero_()
    srn.srn_render(n8.ctx, cams[:1], tf, desc, out, samples=c8)
    srn.srn_dvr_dense(vol, cams[:1], tf, desc, dense)
    u8 = {"ms_per_frame": ms8, "samples_per_s": int(c8.item()) / (ms8 / 1e3),
          "psnr_vs_dense_db": _psnr_imgs(srn, out[0], dense), "density_psnr_db": density_psnr_network(n8, vol, pts),
          "grid_bytes": n8.grid_q.numel()}
    n8.close()
    # the FP32 CUDA-core path on the same fitted network and frame, and how far
    # the FP16 tensor-core image is from it
    n32 = srn.Network(net.unpack(), precision=srn.SRN_PREC_FP32)
    c32 = torch.zeros(1, dtype=torch.int64, device=dev)
    ms32 = _time_frames(lambda: srn.srn_render(n32.ctx, cams[:1], tf, desc, out, samples=c32), n=3)
    c32.zero_()
    srn.srn_render(n32.ctx, cams[:1], tf, desc, out, samples=c32)
    img32 = out.clone()
    srn.srn_render(net.ctx, cams[:1], tf, desc, out)
    torch.cuda.synchronize()
    fp32_path = {"ms_per_frame": ms32, "samples_per_s": int(c32.item()) / (ms32 / 1e3),
                 "psnr_vs_dense_db": _psnr_imgs(srn, img32[0], dense),
                 "fp16_vs_fp32_max_abs": float((out - img32).abs().max().item()),
                 "fp32_over_fp16_time": ms32 / fitted_frames["ms_per_frame"]}
    del img32
    n32.close()
    cfg3 = fit_cfg3(vol, pts, steps=args.fit_steps) if fit_info.get("steps") else None
    del pts

    # end-to-end through the C ABI with host buffers: parameters uploaded from
    # pinned host memory and the image read back, every step
    e2e = run_e2e(seeded, tf, cams, desc, dev, args.steps)
    seeded.close()

    res = {
        "metric": METRIC, "value": value, "unit": "network samples/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_frame, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f16" if prec_name == "fp16-mma" else "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "network": "seeded weights (Xavier-uniform, zero biases, grid "
                   "N(0, 0.01^2), seed 0, FP16-rounded); the same network the reference arm renders",
                   "precision": prec_name, "width": W_IMG, "height": H_IMG,
                   "step": STEP, "et": ET, "l2": "flushed (256 MiB write) between timed frames",
                   "samples_per_frame": samples / args.steps / world,
                   "fvsrn_ms_per_frame": ms_frame, "fitted_network_frames": fitted_frames,
                   "dense_dvr_ms_per_frame": float(np.median(d_ms)),
                   "dense_dvr_roofline": dense_roofline(int(dctr.item()), float(np.sum(d_ms)), len(d_ms),
                                                        vol.numel() * 4),
                   "psnr_fvsrn_vs_dense_db": float(np.mean(psnrs)),
                   "psnr_lowpass_grid_vs_dense_db": float(np.mean(lp_psnrs)), "lowpass_grid": M,
                   "ssim_fvsrn_vs_dense": float(np.mean(ssims)), "ssim_lowpass_grid_vs_dense": float(np.mean(lp_ssims)),
                   "density_psnr_fvsrn_db": fvsrn_dpsnr, "density_psnr_lowpass_db": lp_dpsnr, "u8_grid": u8,
                   "fp32_path": fp32_path, "fit_render_network": fit_info,
                   "fit_steps_per_s": cfg3["steps_per_s"] if cfg3 else None, "fit_cfg3": cfg3,
                   "parallelism": f"replicas x{world} (views split across ranks)"},
        "e2e": e2e, "gpu_launches": args.steps,
        "clocks": clk.summary(),
    }
    return res, net, vol, tf, cams


def run_e2e(net, tf, cams, desc, dev, steps):
    import torch
    from paper_2112_01579_gb300 import srn
    host_grid = net.grid_h.cpu().pin_memory()
    host_w = net.weights_h.cpu().pin_memory()
    host_b = net.biases.cpu().pin_memory()
    host_img = torch.empty((1, 1, H_IMG, W_IMG, 4), dtype=torch.float32).pin_memory()
    out = torch.empty((1, 1, H_IMG, W_IMG, 4), device=dev)
    ctr = torch.zeros(1, dtype=torch.int64, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(steps):
        net.grid_h.copy_(host_grid, non_blocking=True)
        net.weights_h.copy_(host_w, non_blocking=True)
        net.biases.copy_(host_b, non_blocking=True)
        srn.srn_render(net.ctx, [cams[k % N_VIEWS]], tf, desc, out, samples=ctr)
        host_img.copy_(out, non_blocking=True)
        torch.cuda.current_stream().synchronize()
    dt = time.perf_counter() - t0
    h2d = host_grid.numel() * 2 + host_w.numel() * 2 + host_b.numel() * 4
    return {"value": int(ctr.item()) / dt, "unit": "network samples/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(host_img.numel() * 4)}


def _time_frames(fn, n=3):
    """Median device time of fn() over n calls after one warm-up (L2 flushed)."""
    import torch
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    fn()
    ms = []
    for _ in range(n):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    return float(np.median(ms))


def _psnr_imgs(S, a, b):
    import torch
    mse = torch.zeros(1, dtype=torch.float64, device="cuda")
    S.srn_image_mse(a.contiguous(), b.contiguous(), mse)
    torch.cuda.synchronize()
    return 10 * math.log10(1.0 / max(mse.item(), 1e-30))


def shaded_workload(fit_steps=FIT_STEPS, seed=0):
    """Config 4: 512^3 anisotropic blobs + noise; 64^3 x 16 FP16 grid, 4
    SnakeAlt layers; 1024^2 at step 1/1024 with headlight shading from the
    adjoint gradient (FP32 kernels, and backward MMAs on the FP16 tensor
    cores), central differences (FP16 tensor cores, 6 extra evaluations) and
    the 4-output head (FP16 tensor cores),
    against dense DVR of the volume with one-voxel central differences."""
    import torch
    from paper_2112_01579_gb300 import srn, synth
    vol = synth.aniso_blobs_volume(512, 64, seed=seed, device="cuda").contiguous()
    tf, cams = synth.tf_preset(8), synth.orbit_cameras(N_VIEWS)
    res = {"workload": "cfg4: 512^3 aniso blobs; 64^3x16 fp16 grid, 4x32 SnakeAlt; 1024^2, step 1/1024, Blinn-Phong"}
    nets = {}
    for D, gw in [(1, 0.0), (4, 1.0)]:
        p = synth.init_params(R=64, F=16, m=14, layers=4, width=32, out_dim=D, act=synth.ACT_SNAKEALT, seed=seed)
        net = srn.Network(p, precision=srn.SRN_PREC_FP16, max_fit_points=FIT_POINTS, adam=True)
        loss = torch.zeros(1, device="cuda")
        # head targets: central differences of the volume scaled by 1/100 (|grad V| reaches ~100 per unit)
        srn.srn_fit_steps(net.ctx, vol, FIT_POINTS, seed + 11, 0, fit_steps, loss, grad_weight=gw, grad_scale=0.01)
        srn.srn_sync_half(net.ctx)
        nets[D] = net
    out = torch.zeros((1, 1, H_IMG, W_IMG, 4), device="cuda")
    ref = torch.zeros((1, H_IMG, W_IMG, 4), device="cuda")
    n32 = srn.Network(nets[1].unpack(), precision=srn.SRN_PREC_FP32)
    modes = [("none_fp16", nets[1], srn.SRN_SHADE_NONE), ("adjoint_fp32", n32, srn.SRN_SHADE_ADJOINT),
             ("adjoint_fp16", nets[1], srn.SRN_SHADE_ADJOINT),
             ("fd_fp16", nets[1], srn.SRN_SHADE_FD), ("head_fp16", nets[4], srn.SRN_SHADE_HEAD)]
    for name, net, sh in modes:
        desc = srn.render_desc(W_IMG, H_IMG, 1 / 1024, ET, sh, 1 / 511)
        ms = _time_frames(lambda: srn.srn_render(net.ctx, cams[:1], tf, desc, out), n=3)
        srn.srn_dvr_dense(vol, cams[:1], tf, srn.render_desc(W_IMG, H_IMG, 1 / 1024, ET,
                                                             srn.SRN_SHADE_FD if sh else 0), ref)
        res[name] = {"ms_per_frame": ms, "psnr_vs_dense_db": _psnr_imgs(srn, out[0], ref)}
    desc = srn.render_desc(W_IMG, H_IMG, 1 / 1024, ET, srn.SRN_SHADE_FD)
    res["dense_fd_ms_per_frame"] = _time_frames(lambda: srn.srn_dvr_dense(vol, cams[:1], tf, desc, ref), n=3)
    res["ratio_fd_over_head"] = res["fd_fp16"]["ms_per_frame"] / res["head_fp16"]["ms_per_frame"]
    res["ratio_adjoint_over_head"] = res["adjoint_fp16"]["ms_per_frame"] / res["head_fp16"]["ms_per_frame"]
    res["ratio_adjoint_fp32_over_head"] = res["adjoint_fp32"]["ms_per_frame"] / res["head_fp16"]["ms_per_frame"]
    for n in list(nets.values()) + [n32]:
        n.close()
    del vol
    return res


def time_workload(fit_steps=FIT_STEPS, seed=0, time_input=0, vols=None):
    """Config 5: 16 timesteps of 256^3 moving blobs; five 32^3 x 16 keyframe
    grids at t = 0, 4, 8, 12, 15 with a shared 4-layer network, fitted on
    the even timesteps and t = 15; the batch of 16 times x 4 views at 1024^2
    rendered in one launch; PSNR per timestep against dense DVR.
    time_input = 1: the "direct" encoding (time as one more input, Section 7)
    instead of latent interpolation only."""
    import torch
    from paper_2112_01579_gb300 import srn, synth
    if vols is None:
        vols = synth.moving_blobs_volumes(256, 16, 32, seed=seed, device="cuda")
    keys = [0.0, 4.0, 8.0, 12.0, 15.0]
    p = synth.init_params(R=32, F=16, m=14, layers=4, width=32, act=synth.ACT_SNAKEALT, seed=seed, n_keyframes=5,
                          key_times=keys, time_input=time_input)
    net = srn.Network(p, precision=srn.SRN_PREC_FP16, max_fit_points=FIT_POINTS, adam=True)
    train_t = [0, 2, 4, 6, 8, 10, 12, 14, 15]
    loss = torch.zeros(1, device="cuda")
    for st in range(fit_steps):
        t = train_t[st % len(train_t)]
        srn.srn_fit_step(net.ctx, vols[t].contiguous(), FIT_POINTS, seed + 21, st, loss, time=float(t))
    srn.srn_sync_half(net.ctx)
    tf, cams = synth.tf_preset(8), synth.orbit_cameras(4)
    times = list(range(16))
    out = torch.zeros((16, 4, H_IMG, W_IMG, 4), device="cuda")
    desc = srn.render_desc(W_IMG, H_IMG, STEP, ET)
    ctr = torch.zeros(1, dtype=torch.int64, device="cuda")
    ms = _time_frames(lambda: srn.srn_render(net.ctx, cams, tf, desc, out, times=times), n=3)
    ctr.zero_()
    srn.srn_render(net.ctx, cams, tf, desc, out, times=times, samples=ctr)
    torch.cuda.synchronize()
    ref = torch.zeros((4, H_IMG, W_IMG, 4), device="cuda")
    psnr = []
    for t in times:
        srn.srn_dvr_dense(vols[t].contiguous(), cams, tf, desc, ref)
        psnr.append(_psnr_imgs(srn, out[t], ref))
    net.close()
    return {"workload": "cfg5: 16 x 256^3 moving blobs; 5 keyframe 32^3x16 fp16 grids; 16 times x 4 views @1024^2 in one launch",
            "ms_per_batch": ms, "frames": 64, "ms_per_frame": ms / 64,
            "samples_per_s": int(ctr.item()) / (ms / 1e3), "psnr_per_timestep_db": psnr,
            "trained_timesteps": train_t}


def width_sweep(seed=0, size=1024, step=1 / 256):
    """Width / layer sweep of the network render (Section 4.1 performance
    figure): hidden width c in {32, 48, 64} x l in {2, 4, 6} layers, 32^3 x 16
    latent grid, m Fourier rows so the input is c + 16 wide, random
    parameters, one size^2 view with early termination off (every ray
    marches the whole box, so all points take the same samples).  FP16
    tensor-core path against the FP32 CUDA-core path: ms per frame, ns per
    sample, and the network's algorithmic FLOP rate."""
    import torch
    from paper_2112_01579_gb300 import srn, synth
    tf, cams = synth.tf_preset(8), synth.orbit_cameras(1)
    out = torch.zeros((1, 1, size, size, 4), device="cuda")
    desc = srn.render_desc(size, size, step, 2.0)
    ctr = torch.zeros(1, dtype=torch.int64, device="cuda")
    rows = []
    for c in (32, 48, 64):
        m = synth.fourier_rows_for_width(c)
        for l in (2, 4, 6):
            p = synth.to_half_exact(synth.random_params(R=32, F=16, m=m, layers=l, width=c, act=synth.ACT_SNAKEALT,
                                                        seed=seed + c + l, grid_std=0.5, bias_std=0.2))
            d0 = 3 + 2 * m + 16
            flops = 2 * (d0 * c + (l - 2) * c * c + c)  # multiply-adds x 2 per sample
            row = {"width": c, "layers": l, "fourier_rows": m, "net_flops_per_sample": flops}
            for name, prec in (("fp16_tensor", srn.SRN_PREC_FP16), ("fp32_cuda_cores", srn.SRN_PREC_FP32)):
                net = srn.Network(p, precision=prec)
                ms = _time_frames(lambda: srn.srn_render(net.ctx, cams, tf, desc, out), n=3)
                ctr.zero_()
                srn.srn_render(net.ctx, cams, tf, desc, out, samples=ctr)
                torch.cuda.synchronize()
                ns = int(ctr.item())
                row[name] = {"ms_per_frame": ms, "ns_per_sample": ms * 1e6 / ns,
                             "net_tflops": flops * ns / (ms * 1e-3) / 1e12}
                net.close()
            row["fp32_over_fp16"] = row["fp32_cuda_cores"]["ms_per_frame"] / row["fp16_tensor"]["ms_per_frame"]
            rows.append(row)
    return {"workload": f"width/layer sweep: 32^3x16 grid, SnakeAlt, {size}^2, step 1/{round(1 / step)}, no early "
                        "termination, random parameters", "samples_per_frame": ns, "points": rows}


def cpu_baseline(params, vol_np, tf, cams, budget_rows=256, single_thread=True):
    """The FP64 oracle on a bounded sample: every (H / budget_rows)-th row of
    one 1024^2 frame of the same scene (256 rows: about 10-15 s on 16 cores)."""
    import oracle
    on = oracle.OracleNet(params)
    otf = oracle.OracleTF(tf["pos"], tf["rgba"], tf["opacity_scale"])
    rows = np.arange(0, H_IMG, H_IMG // budget_rows)
    pix = (rows[:, None] * W_IMG + np.arange(W_IMG)[None, :]).reshape(-1)
    t0 = time.perf_counter()
    _, _, ns = oracle.render(on, cams[:1], otf, W_IMG, H_IMG, STEP, ET, pixels=pix)
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    res = {"value": ns / dt, "unit": "network samples/s", "cores": cores, "kind": "oracle",
           "sample": f"{len(rows)} of {H_IMG} rows of one {W_IMG}x{H_IMG} frame ({ns} samples, {dt:.1f} s)",
           "samples": ns, "seconds": dt,
           "frame_ms_extrapolated": 1e3 * dt * H_IMG / len(rows), "cpu": _cpu_model()}
    if not single_thread:
        return res
    # one thread on two of those rows (OpenMP team size set through the runtime the oracle links)
    try:
        import ctypes
        gomp = ctypes.CDLL("libgomp.so.1")
        gomp.omp_set_num_threads(1)
        t0 = time.perf_counter()
        _, _, ns1 = oracle.render(on, cams[:1], otf, W_IMG, H_IMG, STEP, ET, pixels=pix[:2 * W_IMG])
        res["single_thread_value"] = ns1 / (time.perf_counter() - t0)
        gomp.omp_set_num_threads(cores)
    except OSError:
        res["single_thread_value"] = None
    return res


def _cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "hardware", "cpu part"):
                    return f"{platform.machine()} {line.split(':', 1)[1].strip()}"
    except OSError:
        pass
    return platform.machine()


# Algorithmic work of one network sample of the render network (47 -> 32 ->
# 32 -> 32 -> 1, SnakeAlt): MMA FLOPs 2 * sum(d_in * d_out) and transcendental
# evaluations (3 x 32 activation sines, 2 x 14 Fourier sin/cos, 1 exp).
MMA_FLOP_PER_SAMPLE = 2 * (47 * 32 + 32 * 32 + 32 * 32 + 32 * 1)
TRANSC_PER_SAMPLE = 3 * 32 + 2 * 14 + 1
SMS, MUFU_PER_SM_CLK, FP32_PER_SM_CLK, MAX_SM_GHZ = 152, 16, 128, 2.07
# DRAM bytes (read + write) of one 1024^2 frame of the render kernel and of
# the dense DVR, from the ncu captures summarised in profiles/ (None when the
# kernel changed after the capture).
RENDER_DRAM_BYTES = 1174272 + 10240
# Warp instructions per network sample of the render kernel from the same
# capture (smsp__inst_executed.sum 8.19375e9 over 2.08797e8 samples).
WARP_INST_PER_SAMPLE = 8.19375e9 / 2.08797e8
# Algorithmic work of one plain-workload fit step per point: forward 2 (35 x 32
# + 32) FLOP, weight gradients the same again, the backward through the
# output layer (2 x 32), the latent-input gradient (2 x 32 x 8) and its
# trilinear scatter (8 corners x 8 channels x 2); gathers: the volume's eight
# 4-byte corners.
FIT_FLOP_PER_POINT = 2 * (35 * 32 + 32) * 2 + 2 * 32 + 2 * 32 * 8 + 8 * 8 * 2
FIT_GATHER_BYTES_PER_POINT = 32
DENSE_DRAM_BYTES = 67166208 + 9174016
DENSE_L1_WAVEFRONT_PCT = 88.3  # l1tex__data_pipe_lsu_wavefronts, % of peak, same capture
# L1 load bandwidth of one SM (bytes per clock) for the gather roofline of
# dense DVR (unit count; the peak is derived, not measured).
L1_BYTES_PER_SM_CLK = 128
DENSE_GATHER_BYTES = 32  # 8 corners x 4 B per dense sample


def dense_roofline(samples, ms_total, frames, vol_bytes):
    """Dense DVR against the L1 gather roofline (8 x 4 B per sample, all SMs
    at the maximum clock) and, beside it, the HBM floor of reading the
    volume once per frame against the measured copy bandwidth."""
    secs = ms_total / 1e3
    achieved = samples * DENSE_GATHER_BYTES / secs / 1e9
    peak = SMS * L1_BYTES_PER_SM_CLK * MAX_SM_GHZ
    hbm = peaks().get("hbm_gbs")
    vol_gbs = vol_bytes * frames / secs / 1e9
    return {"bound": "l1", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": DENSE_DRAM_BYTES, "kernel": "dvr_dense_kernel", "per_sample_bytes": DENSE_GATHER_BYTES,
            "peak_source": "152 SMs x 128 B/clk x 2.07 GHz (unit counts)",
            "l1_data_wavefronts_pct": DENSE_L1_WAVEFRONT_PCT,
            "l1_note": "ncu: the L1 data pipe is 88 % busy with the wavefronts of the scattered 4-byte corner "
                       "gathers (several cache lines per warp load), which is what bounds the kernel",
            "hbm_floor": {"achieved": vol_gbs, "peak": hbm, "unit": "GB/s",
                          "frac": vol_gbs / hbm if hbm else None,
                          "note": "the volume read once per frame, against MEASURED_PEAKS.json hbm_gbs"}}


def roofline(res):
    """The render kernel against the XU (MUFU) transcendental roofline, which
    is the unit it uses the largest fraction of; the tensor-pipe fraction
    rides along.  peak = 16 MUFU lanes/SM x 152 SMs x 2.07 GHz."""
    if res["config"]["precision"] != "fp16-mma":
        return None
    sps = res["value"] / res["n_gpus"]  # per-GPU samples/s (kernel time only)
    peak_xu = SMS * MUFU_PER_SM_CLK * MAX_SM_GHZ * 1e9 / 1e12
    achieved_xu = sps * TRANSC_PER_SAMPLE / 1e12
    pk = peaks()
    peak_tc = pk.get("bf16_tflops", 1900.0)
    achieved_tc = sps * MMA_FLOP_PER_SAMPLE / 1e12
    return {"bound": "alu", "achieved": achieved_xu, "peak": peak_xu, "unit": "Top/s (transcendentals)",
            "frac": achieved_xu / peak_xu, "traffic": RENDER_DRAM_BYTES,
            "kernel": "render_mma_kernel (tcgen05)", "per_sample": {"transcendentals": TRANSC_PER_SAMPLE,
                                                                    "mma_flop": MMA_FLOP_PER_SAMPLE},
            "tensor": {"achieved": achieved_tc, "peak": peak_tc, "unit": "TFLOP/s", "frac": achieved_tc / peak_tc,
                       "peak_source": "MEASURED_PEAKS.json bf16_tflops (fp16 dense rate equal)"},
            "issue": {"achieved": sps * WARP_INST_PER_SAMPLE / 1e12, "peak": SMS * 4 * MAX_SM_GHZ * 1e9 / 1e12,
                      "unit": "T warp instructions/s", "frac": sps * WARP_INST_PER_SAMPLE / (SMS * 4 * MAX_SM_GHZ * 1e9),
                      "per_sample": WARP_INST_PER_SAMPLE,
                      "note": "warp instructions per sample from the ncu capture; 4 issue slots per SM per clock"},
            "peak_source": "unit counts x max SM clock; probe measured 15.1 sin/clk/SM"}


def run_reference(args, rank, world):
    """The FP64 oracle on the host cores, on the network and scene of the
    headline line; one step = a bounded sample of one frame (4 of its 1024
    rows).  value = samples / wall time of the timed steps."""
    if rank != 0:
        return None
    p = seeded_params()
    from paper_2112_01579_gb300 import synth
    tf, cams = synth.tf_preset(8), synth.orbit_cameras(N_VIEWS)
    for _ in range(args.warmup):
        cpu_baseline(p, None, tf, cams, budget_rows=4, single_thread=False)
    samples, secs, frame_ms = 0, 0.0, []
    cb = None
    for _ in range(args.steps):
        cb = cpu_baseline(p, None, tf, cams, budget_rows=4, single_thread=False)
        samples += cb["samples"]
        secs += cb["seconds"]
        frame_ms.append(cb["frame_ms_extrapolated"])
    value = samples / secs
    cb["value"] = value
    cb["sample"] = f"{args.steps} steps x 4 of 1024 rows of one 1024x1024 frame ({samples} samples, {secs:.1f} s)"
    return {"metric": METRIC, "value": value, "unit": "network samples/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD + " (bounded row sample per step)",
                       "network": "seeded weights (Xavier-uniform, zero biases, grid N(0, 0.01^2), seed 0, "
                                  "FP16-rounded); the same network the headline line renders",
                       "step_unit": "4 rows (4096 rays) of one 1024x1024 frame",
                       "frame_ms_extrapolated": float(np.mean(frame_ms))},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "network samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ---------------------------------------------------------------- ncu launch list


def short(name):
    name = re.sub(r"\(.*", "", name)
    name = re.sub(r"^void ", "", name)
    name = re.sub(r"<.*", "", name) if "srn::" not in name else name
    for k in ["render_mma_kernel", "render_fp32_kernel", "dvr_dense_kernel", "eval_fp32_kernel", "fit_point_kernel",
              "sort_hist_kernel", "sort_scatter_kernel", "scan_kernel", "digit_scan_kernel", "cell_start_kernel",
              "adam_kernel", "to_half_kernel", "gauss_pass_kernel", "resample_kernel"]:
        if re.search(r"(?<![A-Za-z0-9_])" + k + r"\b", name):
            return "srn::" + k
    return name[:60]


def summarize_launches(path):
    """Per kernel: launches, total device time, share (ncu launch-list CSV)."""
    rows = [r for r in csv.DictReader(l for l in open(path) if not l.startswith("=="))
            if r["Metric Name"] == "gpu__time_duration.sum"]
    agg = collections.defaultdict(lambda: [0, 0.0])
    for r in rows:
        v = float(r["Metric Value"].replace(",", ""))
        unit = r["Metric Unit"]
        ns = v * {"nsecond": 1, "usecond": 1e3, "msecond": 1e6, "second": 1e9}.get(unit, 1)
        a = agg[short(r["Kernel Name"])]
        a[0] += 1
        a[1] += ns
    tot = sum(v[1] for v in agg.values())
    print(f"{'kernel':44s} {'launches':>8s} {'total ms':>10s} {'share':>7s}")
    for k, (n, t) in sorted(agg.items(), key=lambda kv: -kv[1][1]):
        print(f"{k:44s} {n:8d} {t / 1e6:10.3f} {100 * t / tot:6.2f}%")
    print(f"{'all':44s} {sum(v[0] for v in agg.values()):8d} {tot / 1e6:10.3f}")



def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fit-steps", type=int, default=FIT_STEPS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the shaded and time-varying workloads")
    ap.add_argument("--summarize-launches", metavar="CSV",
                    help="print per-kernel launches / time / share of an ncu gpu__time_duration.sum CSV and exit")
    args = ap.parse_args()
    if args.summarize_launches:
        summarize_launches(args.summarize_launches)
        return
    args.warmup = max(args.warmup, 3)
    world = int(os.environ.get("WORLD_SIZE", 1))
    rank = int(os.environ.get("RANK", 0))
    if world > 1:
        import torch
        import torch.distributed as dist
        if args.impl == "ours":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
            dist.init_process_group("nccl")
    if args.impl == "reference":
        res = run_reference(args, rank, world)
        if res is not None:
            print(json.dumps(res))
        return
    import __graft_entry__
    __graft_entry__.build()
    res, net, vol, tf, cams = run_ours(args, rank, world)
    res["roofline"] = roofline(res)
    if rank == 0 and not args.no_extras:
        res["config"]["shaded_cfg4"] = shaded_workload(fit_steps=args.fit_steps)
        from paper_2112_01579_gb300 import synth
        vols = synth.moving_blobs_volumes(256, 16, 32, seed=0, device="cuda")
        res["config"]["time_cfg5"] = time_workload(fit_steps=args.fit_steps, vols=vols)
        direct = time_workload(fit_steps=args.fit_steps, vols=vols, time_input=1)
        res["config"]["time_cfg5"]["direct_encoding"] = {k: direct[k] for k in
                                                         ("ms_per_frame", "psnr_per_timestep_db")}
        del vols
        res["config"]["point_eval"] = point_eval(net, vol)
        res["config"]["width_sweep"] = width_sweep()
        pts = vertex_points(vol.shape[0])
        res["config"]["adaptive_resampling"] = fit_adaptive(vol, pts, steps=args.fit_steps)
        del pts
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(seeded_params(), None, tf, cams)
    if rank == 0:
        print(json.dumps(res))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
