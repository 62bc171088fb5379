#!/usr/bin/env python
"""Throughput of the BioEM scoring hot path on GB300: parameter-set x image evaluations per second.

One step = the whole path over one batch: prepare the images (moments + spectra), project the
model for every parameter set (rotate, project, PSF), and score every image against every
parameter set over every displacement (fused product / pruned inverse transform / likelihood /
log-sum-exp) down to log P per image.

Workload (per GPU): the "throughput" configuration — 2048 images of 128 x 128 px at 1.1 A, a
5000-atom model, 36,864 Hopf-grid orientations x 4 defocus x 2 B-factors = 294,912 parameter
sets, shifts within +-16 px (1089 displacements).  Images are synthesised on the GPU from the
model through the library's synthetic-map entry point plus seeded shifts, normalisation, offset
and noise.  Under torchrun every rank scores its own 2048 images against the full grid (weak
scaling, no data-path collective).

The scoring form is the FP32 one (pruned FFT on the CUDA cores); `--precision fp16x2_fft` times the
same path with its column transforms on the tensor cores.  Other workloads: `--workload precision`
(split-precision tensor-core forms at +-4 px), `shifts` (the shift-window sweep), `batched`
(models x mixed-size stacks in one graph launch) and `proposal` (the learned proposal, judged on
every image against the full fine grid).

`--impl reference` times the FP64 CPU oracle instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import tempfile
import time

NCORES = os.cpu_count() or 1
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, str(NCORES))

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "parameter-set×image evals/sec (all shifts) at stated |Δlog P| vs FP64 oracle"
# The scoring form the throughput line reports (both hold |d log P| <= 1e-3 at the posterior peak).
HEADLINE_PRECISION = "fp32"
UNIT = "evals/s"
CSRC = os.path.join(ROOT, "paper_1609_06634_gb300", "csrc")

# Identity of a kernel's source: the sha256 of the code (comments removed) between two markers of
# its file plus the shared headers it includes, so a stored DRAM figure stays valid while that
# kernel's code is unchanged.
KERNEL_SOURCES = {
    "k_score": (os.path.join(CSRC, "score.cu"), "template <int N_, int SMAX_",
                "// ---------------------------------------------------------------------------- reductions (float64)",
                [os.path.join(CSRC, "bioem_internal.cuh"), os.path.join(CSRC, "rdft16.cuh")]),
    "k_score_gemm": (os.path.join(CSRC, "gemm.cu"), "struct GemmArgs {", "bool mode_fp16(int mode)",
                     [os.path.join(CSRC, "tc_util.cuh"), os.path.join(CSRC, "bioem_internal.cuh")]),
    "k_score_tc": (os.path.join(CSRC, "score_tc.cu"), "namespace tcs {", "int bioem_tc_supported(",
                   [os.path.join(CSRC, "tc_util.cuh"), os.path.join(CSRC, "rdft16.cuh"),
                    os.path.join(CSRC, "bioem_internal.cuh")]),
}


def _code_only(txt: str) -> str:
    """C/C++ text with its comments and trailing blanks removed (the kernels hold no string literal
    with a comment marker), so that editing a comment keeps a kernel's identity."""
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    txt = re.sub(r"//[^\n]*", "", txt)
    return "\n".join(line.rstrip() for line in txt.splitlines() if line.strip())


def kernel_source_sha(kernel: str) -> str:
    path, begin, end, extra = KERNEL_SOURCES[kernel]
    txt = open(path).read()
    h = hashlib.sha256(_code_only(txt[txt.index(begin):txt.index(end)]).encode())
    for e in extra:
        h.update(_code_only(open(e).read()).encode())
    return h.hexdigest()


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum, one-pass ncu captures), valid only for
# the kernel source they were taken on (kernel_source_sha).
#   k_score: per evaluated pair, from one launch of 2048 images x 4608 sets (above L2), scaled by
#            pairs to the bench's launches (profiles/k_score_throughput.md).
#   k_score_gemm: per launch of the precision workloads (64 images x 6912 sets, +-4 px).
K_SCORE_TRAFFIC = {"source_sha256": "f1d1c96b7a9aaf909575e174927254a9a99fd620c601fec5e301c2ca40fd73c8", "bytes_per_pair": (1553334016 + 118952960) / (2048 * 4608)}
K_SCORE_GEMM_TRAFFIC = {"source_sha256": "083bf58cd6cd1f4630508bfac27c7d80488b5d30f742979416b2b4b648b51731", "bytes_per_launch": {
    '128/bf16x2': 3528212224, '128/fp16x2': 3795020800, '128/bf16x2_real': 3479105792, '128/fp16x2_real': 4123705344,
    '64/bf16x2': 895100672, '64/fp16x2': 895214592, '64/bf16x2_real': 868046336, '64/fp16x2_real': 867884544}}
K_SCORE_TC_TRAFFIC = {"source_sha256": "", "bytes_per_pair": None}


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="throughput")
    ap.add_argument("--n-img", type=int, default=None, help="images per GPU (default: the workload's)")
    ap.add_argument("--n-quat", type=int, default=None, help="use only the first n orientations (testing)")
    ap.add_argument("--cpu-images", type=int, default=16, help="images in the CPU-oracle sample")
    ap.add_argument("--cpu-quats", type=int, default=128, help="orientations in the CPU-oracle sample")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle leg")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--epochs", type=int, default=16, help="proposal workload: training epochs")
    ap.add_argument("--precision", default=None,
                    help="throughput workload: scoring form (fp32: pruned FFT on CUDA cores; fp16x2_fft: its "
                         "column transforms as split-FP16 tensor-core products); default: the form the bench "
                         "reports as its headline")
    return ap.parse_args()


def flops_per_eval(npix: int, max_shift: int) -> float:
    """Algorithmic FP32 work of one (image, parameter set) evaluation over all shifts:
    conjugate product 6 H + a full complex-to-real inverse FFT 2.5 n log2 n + the likelihood 4 S
    (log1p and exp not counted)."""
    n = npix * npix
    h = npix * (npix // 2 + 1)
    s = (2 * max_shift + 1) ** 2
    return 6.0 * h + 2.5 * n * math.log2(n) + 4.0 * s


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples every 200 ms while running."""

    FIELDS = ("index,pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id: str | None):
        self.bus_id = bus_id
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return None
        allrows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 10:
                allrows.append(parts)
        os.remove(self.path)
        rows = [r for r in allrows if self.bus_id and self.bus_id.lower() in r[1].lower()] or allrows
        if not rows:
            return None
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[6 + k].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def synth_images(bioem, ctx, cfg, atoms_d, first: int, n: int):
    """Observed images N I1(r + d) - mu + lambda z for images first..first+n of the workload."""
    import torch
    dev = ctx.device
    truths = [workloads.image_truth(cfg, i) for i in range(first, first + n)]
    quats = torch.from_numpy(np.stack([t["quat"] for t in truths]).astype(np.float32)).to(dev)
    ctfs = [(t["defocus_A"], t["amp_contrast"], t["bfactor"], t["voltage_kV"]) for t in truths]
    out = torch.empty((n, cfg.npix, cfg.npix), dtype=torch.float32, device=dev)
    chunk = 1024
    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        maps = bioem.synthetic_maps(ctx, atoms_d, cfg.sigma_A, quats[c0:c1], ctfs[c0:c1], cfg.npix, cfg.pixel_A)
        z = torch.from_numpy(np.stack([workloads.standard_normal_noise(cfg, first + i)
                                       for i in range(c0, c1)]).astype(np.float32)).to(dev)
        for k in range(c1 - c0):
            t = truths[c0 + k]
            sig = torch.roll(maps[k], shifts=(-t["dy"], -t["dx"]), dims=(0, 1)) * t["norm"]
            lam = torch.sqrt(sig.double().var(unbiased=False) / cfg.snr).float()
            out[c0 + k] = sig - t["offset"] + lam * z[k]
    return out


def run_cpu_oracle(images: np.ndarray, atoms, quats, ctfs, cfg):
    import oracle
    t0 = time.perf_counter()
    r = oracle.score(images, atoms, quats, ctfs, cfg.sigma_A, cfg.pixel_A, cfg.max_shift)
    dt = time.perf_counter() - t0
    return r, dt


def run_cpu_fft_context(images, projs, max_shift: int, reps: int = 5):
    """Context only: the paper's FP32 Fourier variant (Sec. 3.3, Eqs. 11-12) on the host cores.

    Per pair: the conjugate product of the zero-mean, unit-norm spectra, a full inverse real FFT
    (torch CPU FFT in float32 on all host threads), the displacement window, t = ln(1 - rho^2) and
    the closed form; per image the float64 log-sum-exp over the grid.  images [n_img, N, N] and
    projs [n_ps, N, N] are real arrays (projections with their PSF applied).  Returns
    (log P [n_img], median seconds of `reps` timed runs after one warm-up, threads used).
    """
    import torch
    import oracle
    npix = images.shape[-1]
    n = npix * npix
    c1 = 0.5 * (3 - n)
    side = 2 * max_shift + 1

    def unit(x):
        x = torch.from_numpy(np.asarray(x, dtype=np.float64))
        d = x - x.mean(dim=(-2, -1), keepdim=True)
        ss = (d * d).sum(dim=(-2, -1))
        return (d / ss.sqrt()[:, None, None]).float(), n * ss   # n sum (x - mean)^2 = n C_xx - C_x^2

    a, big_a = unit(images)
    b, big_b = unit(projs)
    k_a = 0.5 * (3 - n) * torch.log(big_a) + oracle.log_norm_constant(n)
    k_b = -0.5 * torch.log(big_b)
    idx = torch.arange(-max_shift, max_shift + 1) % npix
    blk = 256

    def once():
        fa = torch.fft.rfft2(a)
        fb = torch.fft.rfft2(b)
        out = torch.empty(len(a), dtype=torch.float64)
        for w in range(len(a)):
            parts = []
            for p0 in range(0, len(b), blk):
                rho = torch.fft.irfft2(fa[w].conj()[None] * fb[p0:p0 + blk], s=(npix, npix))
                win = rho[:, idx][:, :, idx]
                t = torch.log1p(-win * win).double()
                parts.append(torch.logsumexp((k_b[p0:p0 + blk, None, None] + c1 * t).reshape(-1), 0))
            out[w] = torch.logsumexp(torch.stack(parts), 0) + k_a[w]
        return (out - math.log(len(b) * side * side)).numpy()

    once()
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        logp = once()
        times.append(time.perf_counter() - t0)
    return logp, float(np.median(times)), torch.get_num_threads()


def measure_fma_peaks(bioem, ctx, bus_id):
    """CUDA-core FP32 / FP64 multiply-add throughput of this GPU (the FP32 form's roofline peak),
    measured by the library's microbenchmark with the SM clock sampled meanwhile."""
    with ClockSampler(bus_id) as clk:
        f32 = bioem.fma_peak(ctx, "fp32", reps=5)
        f32x2 = bioem.fma_peak(ctx, "fp32x2", reps=5)
        f64 = bioem.fma_peak(ctx, "fp64", reps=3)
    c = clk.summary() or {}
    best = max(f32, f32x2)
    return {"fp32_tflops": best / 1e12, "fp32_form": "packed FFMA2" if f32x2 >= f32 else "FFMA",
            "fp32_ffma_tflops": f32 / 1e12, "fp32_ffma2_tflops": f32x2 / 1e12, "fp64_tflops": f64 / 1e12,
            "sm_mhz": c.get("sm_mhz")}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def bench_reference(args):
    """The FP64 oracle on the host cores, each step a bounded sample of the workload."""
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return 0
    import oracle
    cfg = workloads.get_config(args.workload)
    n_img = max(1, min(4, args.cpu_images))
    nq = max(1, min(64, args.cpu_quats))
    wl = workloads.workload(cfg, n_img=n_img)
    imgs = oracle.synthesize_images(wl)
    quats = wl["quats"][:nq]
    evals = n_img * nq * len(wl["ctfs"])
    # the workload the GPU arm runs (its config); each step here is the bounded sample above
    full_img = args.n_img or cfg.n_img
    full_q = len(wl["quats"]) if args.n_quat is None else min(args.n_quat, len(wl["quats"]))
    for _ in range(args.warmup):
        run_cpu_oracle(imgs, wl["atoms"], quats, wl["ctfs"], cfg)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        run_cpu_oracle(imgs, wl["atoms"], quats, wl["ctfs"], cfg)
    dt = (time.perf_counter() - t0) / max(1, args.steps)
    value = evals / dt
    sample = (f"{n_img} images x {nq} orientations x {len(wl['ctfs'])} PSFs x {cfg.n_shift} shifts of the "
              f"{cfg.name} workload ({cfg.npix}x{cfg.npix} px); per step: projections, PSFs, direct-sum "
              "correlations, closed-form likelihoods, log-sum-exp")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(cfg, full_img, full_q * len(wl["ctfs"])),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": NCORES, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def workload_config(cfg, n_img, n_ps):
    return {"workload": f"{cfg.name}: {n_img} images {cfg.npix}x{cfg.npix} px @ {cfg.pixel_A} A, {cfg.n_atoms}-atom "
                        f"model, {n_ps} parameter sets ({cfg.orient} orientations x {cfg.n_defocus} defocus x "
                        f"{len(cfg.bfactors)} B), shifts +-{cfg.max_shift} ({cfg.n_shift} per pair)",
            "n_img": n_img, "n_ps": n_ps, "npix": cfg.npix, "max_shift": cfg.max_shift,
            "l2": "inputs larger than L2 (projection spectra and image stack exceed the 126 MB L2)",
            "step": "prepare_images + project_model + score"}


def bench_ours(args):
    import torch
    import torch.distributed as tdist

    import paper_1609_06634_gb300 as bioem
    from paper_1609_06634_gb300 import build

    world, rank, local = dist_setup(args)
    if world > 1:
        tdist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    cfg = workloads.get_config(args.workload)
    n_img = args.n_img or cfg.n_img
    wl = workloads.workload(cfg, n_img=0)
    quats_np = wl["quats"] if args.n_quat is None else wl["quats"][:args.n_quat]
    ctfs = wl["ctfs"]
    n_ps = len(quats_np) * len(ctfs)

    ctx = bioem.Context(local)
    precision = args.precision or HEADLINE_PRECISION
    atoms_d = torch.from_numpy(wl["atoms"]).to(dev)
    quats_d = torch.from_numpy(np.ascontiguousarray(quats_np)).to(dev)
    images_d = synth_images(bioem, ctx, cfg, atoms_d, rank * n_img, n_img)
    logp = torch.empty(n_img, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    if ctx.status() != 0:
        raise RuntimeError("device status error during input synthesis")

    def step(imgs, atoms, quats):
        im = bioem.prepare_images(ctx, imgs, cfg.pixel_A)
        ps = bioem.project_model(ctx, atoms, cfg.sigma_A, quats, ctfs, cfg.npix, cfg.pixel_A)
        bioem.score(ctx, im, ps, cfg.max_shift, out=logp)
        im.close()
        ps.close()

    def barrier():
        if world > 1:
            tdist.barrier()

    ctx.set_precision(precision)
    score_kernel = "k_score_tc" if precision == "fp16x2_fft" else "k_score"
    for _ in range(args.warmup):
        step(images_d, atoms_d, quats_d)
    torch.cuda.synchronize()
    if ctx.status() != 0:
        raise RuntimeError("device status error in warm-up")

    props = torch.cuda.get_device_properties(dev)
    bus = getattr(props, "pci_bus_id", None)
    bus_id = None
    if bus is not None:
        bus_id = f"{getattr(props, 'pci_domain_id', 0):08X}:{bus:02X}:{getattr(props, 'pci_device_id', 0):02X}"
    stream = torch.cuda.current_stream(dev)
    peaks = measure_fma_peaks(bioem, ctx, bus_id)
    ctx.reset_kernel_stats()
    ctx.set_kernel_timing(True)
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(bus_id) as clocks:
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            step(images_d, atoms_d, quats_d)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms = ev0.elapsed_time(ev1)
    launches = ctx.launch_count()
    k_ms, k_n = ctx.kernel_time(score_kernel)
    kernel_ms = {name: ctx.kernel_time(name)[0] for name in
                 ("k_prepare_images", "k_ctf_table", "k_project", "k_psf_spectra", score_kernel, "k_reduce_wave",
                  "k_finalize")}
    ctx.set_kernel_timing(False)
    if ctx.status() != 0:
        raise RuntimeError("device status error in the timed steps")
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    if world > 1:
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    ms_max = float(t.item())
    evals = world * n_img * n_ps * args.steps
    value = evals / (ms_max / 1e3)

    # end to end through the public API: pinned host inputs in, log P out, copies inside the region
    e2e = None
    if not args.no_e2e:
        img_h = images_d.cpu().pin_memory()
        atoms_h = atoms_d.cpu().pin_memory()
        quats_h = quats_d.cpu().pin_memory()
        logp_h = torch.empty(n_img, dtype=torch.float64).pin_memory()

        def e2e_step():
            step(img_h.to(dev, non_blocking=True), atoms_h.to(dev, non_blocking=True),
                 quats_h.to(dev, non_blocking=True))
            logp_h.copy_(logp, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        te = torch.tensor([e0.elapsed_time(e1)], dtype=torch.float64, device=dev)
        if world > 1:
            tdist.all_reduce(te, op=tdist.ReduceOp.MAX)
        h2d = img_h.numel() * 4 + atoms_h.numel() * 4 + quats_h.numel() * 4
        e2e = {"value": evals / (float(te.item()) / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(n_img * 8)}

    result = None
    if rank == 0:
        # roofline of the dominant kernel: FP32 ALU bound (pruned transforms + epilogue on CUDA cores)
        fpe = flops_per_eval(cfg.npix, cfg.max_shift)
        achieved = fpe * n_img * n_ps * args.steps / (k_ms / 1e3) / 1e12
        clk = clocks.summary()
        peak_mhz = 2070.0
        try:
            peak_mhz = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("sm_max_mhz", peak_mhz)
        except (OSError, ValueError):
            pass
        nominal = props.multi_processor_count * 128 * 2 * peak_mhz * 1e6 / 1e12
        peak = peaks["fp32_tflops"]
        traffic = None
        table = K_SCORE_TC_TRAFFIC if score_kernel == "k_score_tc" else K_SCORE_TRAFFIC
        if table["source_sha256"] == kernel_source_sha(score_kernel) and table["bytes_per_pair"]:
            traffic = table["bytes_per_pair"] * n_img * n_ps / max(1, k_n / args.steps)
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": score_kernel,
                "peak_basis": (f"measured: FP32 multiply-add microbenchmark (bioem_fma_peak, {peaks['fp32_form']}) "
                               f"on this GPU in this run, median SM clock {peaks['sm_mhz']} MHz during it"),
                "peak_nominal": nominal,
                "peak_nominal_basis": f"{props.multi_processor_count} SMs x 128 lanes x 2 flop x {peak_mhz:.0f} MHz",
                "fp32_ffma_measured_tflops": peaks["fp32_ffma_tflops"],
                "fp32_ffma2_measured_tflops": peaks["fp32_ffma2_tflops"],
                "fp64_peak_measured_tflops": peaks["fp64_tflops"],
                "flops_per_eval": fpe, "kernel_ms_per_step": k_ms / args.steps, "launches_per_step": k_n / args.steps}
        if clk and clk.get("sm_mhz") and peaks.get("sm_mhz"):
            # the peak rescaled from the microbenchmark's clock to the clock seen in the timed steps
            roof["frac_at_observed_clock"] = achieved / (peak * clk["sm_mhz"] / peaks["sm_mhz"])
        if score_kernel == "k_score_tc":
            # the column transforms' tensor-core products: per pair 2 MMA terms x 128 rows x 64 columns
            # x 256 K x 2 flop = 8.39 Mflop, against the measured dense 16-bit rate (FP16 = BF16 rate)
            tflop = 2 * 128 * 64 * 256 * 2 * n_img * n_ps * args.steps / (k_ms / 1e3) / 1e12
            bf16 = None
            try:
                bf16 = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("bf16_tflops")
            except (OSError, ValueError):
                pass
            roof["tensor"] = {"achieved": tflop, "peak": bf16 or 1900.0, "unit": "TFLOP/s",
                              "frac": tflop / (bf16 or 1900.0),
                              "peak_basis": "measured" if bf16 else "fallback",
                              "work": "stage-A products, 8.39 Mflop per pair (two split terms, stacked hi/lo rows)"}
        dtype = "f32 (column transforms: fp16x2 tensor cores)" if precision == "fp16x2_fft" else "f32"
        result = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                  "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                  "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic", "precision": precision,
                  "config": workload_config(cfg, n_img, n_ps), "roofline": roof, "e2e": e2e,
                  "gpu_launches": int(launches), "clocks": clk,
                  "kernel_ms_per_step": {k: v / args.steps for k, v in kernel_ms.items()}}

        # CPU oracle on a bounded sample of the same workload, and the GPU's |d log P| on it (N = 1 only)
        if not args.no_cpu and world == 1:
            ni = min(args.cpu_images, n_img)
            # orientations: each sampled image's truth neighbourhood (its nearest grid orientations),
            # so the error is measured at the posterior peak, where rho is largest
            per = max(1, min(args.cpu_quats, len(quats_np)) // ni)
            sample_q = []
            for i in range(ni):
                t = workloads.image_truth(cfg, rank * n_img + i)
                for q in workloads.nearest_orientations(quats_np, t["quat"], per):
                    if q not in sample_q:
                        sample_q.append(int(q))
            sample_q = np.array(sample_q)
            nq = len(sample_q)
            q_sample = np.ascontiguousarray(quats_np[sample_q])
            sample_imgs = images_d[:ni].cpu().numpy()
            ref, dt = run_cpu_oracle(sample_imgs, wl["atoms"], q_sample, ctfs, cfg)
            im = bioem.prepare_images(ctx, images_d[:ni].contiguous(), cfg.pixel_A)
            ps = bioem.project_model(ctx, atoms_d, cfg.sigma_A, torch.from_numpy(q_sample).to(dev), ctfs, cfg.npix,
                                     cfg.pixel_A)
            out_s = bioem.score_all(ctx, im, ps, cfg.max_shift, per_orient=True)
            got = out_s["logP"].cpu().numpy()
            got_o = out_s["logP_orient"].cpu().numpy()
            sample = (f"{ni} images x {nq} orientations x {len(ctfs)} PSFs x {cfg.n_shift} shifts of this workload "
                      f"(the images the GPU scored; the orientations are the union of each image's {per} grid "
                      f"orientations nearest its true orientation, i.e. the posterior peak)")
            result["cpu_baseline"] = {
                "value": ni * nq * len(ctfs) / dt, "unit": UNIT, "cores": NCORES, "kind": "oracle",
                "sample": sample + f"; FP64 numpy oracle, {dt:.1f} s"}
            result["dlogP_max_vs_oracle"] = float(np.max(np.abs(got - ref["logP"])))
            result["dlogP_orient_max_vs_oracle"] = float(np.max(np.abs(got_o - ref["logP_orient"])))
            result["dlogP_sample"] = sample
            # context only: the paper's own FP32 Fourier variant on the same host cores and sample
            try:
                import oracle
                projs = oracle.projections(wl["atoms"], q_sample, ctfs, cfg.sigma_A, cfg.npix, cfg.pixel_A)
                lp_fft, t_fft, threads = run_cpu_fft_context(sample_imgs, projs, cfg.max_shift)
                result["cpu_fft_context"] = {
                    "value": ni * nq * len(ctfs) / t_fft, "unit": UNIT, "cores": threads,
                    "kind": "the paper's FP32 Fourier variant (torch CPU FFT), context only",
                    "sample": "the oracle's sample; median of 5 timed runs after one warm-up",
                    "dlogP_max_vs_oracle": float(np.max(np.abs(lp_fft - ref["logP"])))}
            except Exception as e:   # context only: it never costs the bench line
                result["cpu_fft_context"] = {"unavailable": f"{type(e).__name__}: {e}"}
        print(json.dumps(result), flush=True)
    if world > 1:
        tdist.barrier()
        tdist.destroy_process_group()
    return 0


def bench_batched(args):
    """Batched uneven workload, capped: 8 models x 4 stacks (64/96/128/192 px) x 256 images, each stack
    scored on Hopf level 2 (4608 orientations) x 2 defocus x 2 B, shifts N/8; one graph replay per step."""
    import torch

    import paper_1609_06634_gb300 as bioem
    from paper_1609_06634_gb300 import build

    build.build()
    dev = torch.device("cuda", 0)
    n_models = 8
    stacks_spec = tuple(workloads.StackSpec(n, args.n_img or 256, 2, 2) for n in (64, 96, 128, 192))
    cfg = workloads.BatchedConfig(n_models=n_models, stacks=stacks_spec)
    wl = workloads.batched_workload(cfg)
    ctx = bioem.Context(0)
    t0 = time.perf_counter()
    atoms_d = [torch.from_numpy(a).to(dev) for a in wl["atoms"]]
    stacks, projsets = [], [[] for _ in range(n_models)]
    for k, st in enumerate(wl["stacks"]):
        sc = st["config"]
        n = len(st["truth"])
        imgs = torch.empty((n, sc.npix, sc.npix), dtype=torch.float32, device=dev)
        for m in range(n_models):
            idx = [i for i in range(n) if st["models"][i] == m]
            if not idx:
                continue
            t = [st["truth"][i] for i in idx]
            q = torch.from_numpy(np.stack([x["quat"] for x in t]).astype(np.float32)).to(dev)
            maps = bioem.synthetic_maps(ctx, atoms_d[m], sc.sigma_A, q,
                                        [(x["defocus_A"], x["amp_contrast"], x["bfactor"], x["voltage_kV"]) for x in t],
                                        sc.npix, sc.pixel_A)
            for j, i in enumerate(idx):
                x = st["truth"][i]
                sig = torch.roll(maps[j], shifts=(-x["dy"], -x["dx"]), dims=(0, 1)) * x["norm"]
                lam = torch.sqrt(sig.double().var(unbiased=False) / sc.snr).float()
                imgs[i] = sig - x["offset"] + lam * torch.from_numpy(st["noise"][i].astype(np.float32)).to(dev)
        stacks.append(bioem.prepare_images(ctx, imgs, sc.pixel_A))
        q_d = torch.from_numpy(st["quats"]).to(dev)
        for m in range(n_models):
            projsets[m].append(bioem.project_model(ctx, atoms_d[m], sc.sigma_A, q_d, st["ctfs"], sc.npix, sc.pixel_A))
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    t1 = time.perf_counter()
    chunks = {sc["config"].npix: bioem.autotune(ctx, stacks[k], projsets[0][k], sc["config"].max_shift)
              for k, sc in enumerate(wl["stacks"])}
    t_tune = time.perf_counter() - t1
    shifts = [st["config"].max_shift for st in wl["stacks"]]
    batch = bioem.Batch(ctx, stacks, projsets, shifts)
    for _ in range(args.warmup):
        batch.run()
    torch.cuda.synchronize()
    if ctx.status() != 0:
        raise RuntimeError("device status error")
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(None) as clocks:
        e0.record(stream)
        for _ in range(args.steps):
            batch.run()
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    out = batch.out.cpu().numpy()
    # which model explains each image best (images were drawn from seeded-random models)
    truth = np.concatenate([st["models"] for st in wl["stacks"]])
    acc = float(np.mean(np.argmax(out, axis=0) == truth))
    # ensemble posterior of the 8 models over all images (Eq. 10), weights by EM
    ens = bioem.ensemble(ctx, batch.out, n_iter=50)
    ens_w = ens["weights"].cpu().numpy()
    true_frac = np.bincount(truth, minlength=n_models) / len(truth)
    line = {"metric": METRIC, "value": batch.evals * args.steps / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batched uneven (capped): 8 models (500-20000 atoms) x 4 stacks of 256 images "
                                   "(64/96/128/192 px, 140.8 A field), Hopf level 2 x 2 defocus x 2 B per stack, "
                                   "shifts N/8; one graph replay (persistent scoring launch + reduction) per step",
                       "evals_per_step": batch.evals, "setup_s": t_setup, "autotune_s": t_tune, "chunks": chunks},
            "model_recovery": acc,
            "ensemble": {"log_post_uniform_weights": None, "log_post_em": float(ens["log_post"]),
                         "em_weights": [round(float(x), 4) for x in ens_w],
                         "true_model_fractions": [round(float(x), 4) for x in true_frac],
                         "model_rank_by_log_post": [int(i) for i in
                                                    np.argsort(-ens["model_log_post"].cpu().numpy())]},
            "clocks": clocks.summary()}
    line["ensemble"]["log_post_uniform_weights"] = float(bioem.ensemble(ctx, batch.out)["log_post"])
    print(json.dumps(line), flush=True)
    batch.close()
    return 0


def bench_proposal(args):
    """Learned proposal at the configuration's scale: train on 200k forward-model projections of 10
    models, propose the top-32 joint (coarse Hopf cell, defocus) bins for 10,000 images, score them on
    their fine parameter sets; judge every image against the full fine grid (2.36M parameter sets)."""
    import torch

    import paper_1609_06634_gb300 as bioem
    from paper_1609_06634_gb300 import build, proposal

    build.build()
    dev = torch.device("cuda", 0)
    cfg = workloads.ProposalConfig()
    if args.n_img:
        cfg = workloads.ProposalConfig(n_infer=args.n_img)
    ctx = bioem.Context(0)
    gen = torch.Generator(device=dev).manual_seed(5)
    t0 = time.perf_counter()
    atoms = [torch.from_numpy(a).to(dev) for a in workloads.proposal_models(cfg)]
    tr = workloads.proposal_draws(cfg, cfg.n_train, 8)
    imgs = proposal.compose(ctx, atoms, tr, cfg, gen)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    net = bioem.CNN(ctx, image_px=cfg.npix, downsample=cfg.downsample, channels=cfg.channels, n_qbins=cfg.n_coarse,
                    n_dbins=cfg.n_defocus, max_batch=256, seed=11)
    t0 = time.perf_counter()
    epochs = args.epochs
    # every epoch re-composes the 200k training projections with new displacements, scales, offsets
    # and noise (a fixed set is memorised after ~3 epochs: validation recall falls while the loss
    # goes to 0.5)
    losses = proposal.train_redrawn(ctx, net, atoms, tr, cfg, epochs=epochs, batch=256, lr=1e-3, gen=gen,
                                    rng=np.random.default_rng(77), images=imgs)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del imgs
    inf = workloads.proposal_draws(cfg, cfg.n_infer, 9, models=False)
    x = proposal.compose(ctx, [atoms[0]], inf, cfg, gen)
    im = bioem.prepare_images(ctx, x, cfg.pixel_A)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    bins, _ = net.propose(x, cfg.top_k)
    bins = bins.cpu().numpy().astype(np.int64)
    t_prop = time.perf_counter() - t0
    res = proposal.score_cells(ctx, im, atoms[0], bins, cfg)
    truth = inf["label_q"].astype(np.int64) * cfg.n_defocus + inf["label_d"]
    recall = float(np.mean([t in b for t, b in zip(truth, bins)]))
    recall_k = {}
    for k in (32, 256, 1024):
        bk = net.propose(x, k)[0].cpu().numpy()
        recall_k[k] = float(np.mean([t in b for t, b in zip(truth, bk)]))
    # two-stage: the network's top K1 joint bins re-ranked by the exact likelihood at the coarse grid
    # points (2 K1 parameter sets per image), the best top_k expanded to the fine grid; K1 = every
    # joint bin is the exact coarse scan without the network
    n_joint = cfg.n_coarse * cfg.n_defocus
    two_stage = {}
    # (network top K1, re-rank grid level, bins kept for the fine grid)
    variants = ((4096, cfg.coarse_level, cfg.top_k), (n_joint, cfg.coarse_level, cfg.top_k),
                (1024, cfg.coarse_level + 1, cfg.top_k), (4096, cfg.coarse_level + 1, cfg.top_k),
                (8192, cfg.coarse_level + 1, cfg.top_k))
    for k1, level, keep in variants:
        t0 = time.perf_counter()
        if k1 < n_joint:
            big = net.propose(x, k1)[0].cpu().numpy().astype(np.int64)
        else:
            big = proposal.all_bins(cfg.n_infer, cfg)
        rr = proposal.rerank_coarse(ctx, im, atoms[0], big, cfg, keep, level=level)
        t_rr = time.perf_counter() - t0
        res_rr = proposal.score_cells(ctx, im, atoms[0], rr["bins"], cfg)
        two_stage[(k1, level, keep)] = (rr, t_rr, res_rr,
                                        float(np.mean([t in b for t, b in zip(truth, rr["bins"])])))
    # judge: the full fine grid (294,912 orientations x 8 PSFs) for every inference image, scanned in
    # chunks of orientations (project, score, fold into per-image accumulators); random proposals
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    from paper_1609_06634_gb300 import driver
    fine_q = workloads.hopf_grid(cfg.fine_level).astype(np.float32)
    scan = driver.OrientationScan(ctx, im, atoms[0], cfg.sigma_A, fine_q, [tuple(r) for r in cfg.ctf_rows()], cfg.npix,
                                  cfg.pixel_A, cfg.max_shift, chunk=18432)
    scan.run()
    full_logP = scan.log_p().cpu().numpy()
    torch.cuda.synchronize()
    t_full = time.perf_counter() - t0
    n_judge = cfg.n_infer
    rng = np.random.default_rng(3)
    rand = np.stack([rng.choice(n_joint, cfg.top_k, replace=False) for _ in range(cfg.n_infer)])
    rnd = proposal.score_cells(ctx, im, atoms[0], rand, cfg)
    kept = res["logP"] - full_logP
    kept_rand = rnd["logP"] - full_logP
    per_img_prop = (t_prop + res["seconds"]) / cfg.n_infer
    per_img_full = t_full / cfg.n_infer
    reranked = []
    for (k1, level, keep), (rr, t_rr, res_rr, recall_rr) in two_stage.items():
        kept_rr = res_rr["logP"] - full_logP
        per_img_rr = (t_prop + t_rr + res_rr["seconds"]) / cfg.n_infer
        reranked.append({"network_top": k1 if k1 < n_joint else "all (no network)", "rerank_level": level,
                         "rerank_orientations_per_bin": 8 ** (level - cfg.coarse_level), "fine_bins": keep,
                         "recall_of_true_bin": recall_rr,
                         "coarse_evals_per_image": rr["evals"] / cfg.n_infer,
                         "fine_evals_per_image": res_rr["evals"] / cfg.n_infer, "rerank_s": t_rr,
                         "kept_log_mass_median": float(np.median(kept_rr)),
                         "kept_log_mass_mean": float(np.mean(kept_rr)),
                         "frac_images_within_1e-2": float(np.mean(np.abs(kept_rr) <= 1e-2)),
                         "frac_images_within_1e-1": float(np.mean(np.abs(kept_rr) <= 1e-1)),
                         "dlogP_max_vs_full": float(np.max(np.abs(kept_rr))),
                         "seconds_per_image": per_img_rr, "speedup_vs_full_grid": per_img_full / per_img_rr})
    line = {"metric": METRIC, "value": res["evals"] / res["seconds"], "unit": UNIT, "n_gpus": 1, "steps": 1,
            "warmup": 0, "ms_per_step": res["seconds"] * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "learned proposal: 10 models (2000-10000 atoms), 200k training projections "
                                   "(128 px, SNR 0.1; displacement, scale, offset and noise redrawn every epoch), "
                                   "10,000 inference images of model 0, top-32 of 4608 coarse "
                                   "Hopf cells x 4 defocus bins, each expanded to 64 fine orientations (Hopf level 4, "
                                   "294,912) x 2 B; judged on every image against the full fine grid",
                       "n_infer": cfg.n_infer, "n_judge": n_judge,
                       "epochs": epochs, "train_images": cfg.n_train},
            "proposal": {"train_loss_per_epoch": losses, "data_s": t_data, "train_s": t_train, "propose_s": t_prop,
                         "recall_at_k_true_joint_bin": recall, "random_recall": cfg.top_k / (cfg.n_coarse * cfg.n_defocus),
                         "recall_at": recall_k,
                         "evals_per_image": res["evals"] / cfg.n_infer,
                         "full_evals_per_image": len(fine_q) * len(cfg.ctf_rows()), "full_grid_s": t_full,
                         "kept_log_mass_median": float(np.median(kept)), "kept_log_mass_mean": float(np.mean(kept)),
                         "dlogP_max_vs_full": float(np.max(np.abs(kept))),
                         "random_kept_log_mass_mean": float(np.mean(kept_rand)),
                         "frac_images_within_1e-2": float(np.mean(np.abs(kept) <= 1e-2)),
                         "seconds_per_image_proposal": per_img_prop, "seconds_per_image_full": per_img_full,
                         "speedup_vs_full_grid": per_img_full / per_img_prop, "cells_projected": res["cells"]},
            "proposal_reranked": reranked}
    print(json.dumps(line), flush=True)
    net.close()
    return 0


def bench_precision(args):
    """Split-precision forms against the FP32 form on the precision workloads: the tiny grid (1152
    random orientations x 3 defocus x 2 B = 6912 parameter sets), shifts +-4, 64 images of the
    throughput model at 128 x 128 px (1.1 A) and at 64 x 64 px (2.2 A).  One step = one bioem_score
    pass over the resident images and projection set; the split-precision operand copies are built
    once per handle (in warm-up; their build time is reported separately).  |d log P| of each form
    against the FP64 oracle on these inputs is measured by tests/test_gpu_precision.py."""
    import torch

    import paper_1609_06634_gb300 as bioem
    from paper_1609_06634_gb300 import build

    build.build()
    dev = torch.device("cuda", 0)
    ctx = bioem.Context(0)
    stream = torch.cuda.current_stream(dev)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    peak_tf = peaks.get("bf16_tflops", 1900.0)
    sizes = {}
    launches = 0
    with ClockSampler(None) as clocks:
        for name in ("precision128", "precision64"):
            cfg = workloads.get_config(name)
            n_img = args.n_img or cfg.n_img
            wl = workloads.workload(cfg, n_img=0)
            quats_np = wl["quats"] if args.n_quat is None else wl["quats"][:args.n_quat]
            n_ps = len(quats_np) * len(wl["ctfs"])
            atoms_d = torch.from_numpy(wl["atoms"]).to(dev)
            imgs = synth_images(bioem, ctx, cfg, atoms_d, 0, n_img)
            im = bioem.prepare_images(ctx, imgs, cfg.pixel_A)
            ps = bioem.project_model(ctx, atoms_d, cfg.sigma_A, torch.from_numpy(np.ascontiguousarray(quats_np)).to(dev),
                                     wl["ctfs"], cfg.npix, cfg.pixel_A)
            logp = torch.empty(n_img, dtype=torch.float64, device=dev)
            forms = {}
            for mode in ("fp32", "bf16x2", "fp16x2", "bf16x2_real", "fp16x2_real"):
                ctx.set_precision(mode)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                bioem.score(ctx, im, ps, cfg.max_shift, out=logp)   # builds the operands in a tensor form
                torch.cuda.synchronize()
                first_s = time.perf_counter() - t0
                for _ in range(args.warmup):
                    bioem.score(ctx, im, ps, cfg.max_shift, out=logp)
                torch.cuda.synchronize()
                kname = "k_score" if mode == "fp32" else "k_score_gemm"
                ctx.reset_kernel_stats()
                ctx.set_kernel_timing(True)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(args.steps):
                    bioem.score(ctx, im, ps, cfg.max_shift, out=logp)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / args.steps
                k_ms, k_n = ctx.kernel_time(kname)
                launches += ctx.launch_count()
                ctx.set_kernel_timing(False)
                if ctx.status() != 0:
                    raise RuntimeError(f"device status error ({name}, {mode})")
                evals = n_img * n_ps
                f = {"evals_per_s": evals / (ms / 1e3), "ms_per_step": ms, "kernel": kname,
                     "kernel_ms_per_step": k_ms / args.steps, "launches_per_step": k_n / args.steps,
                     "first_call_s": first_s}
                if mode != "fp32":
                    # dense contraction per launch: 3 products (hi hi, hi lo, lo hi) x 2 flop x K per
                    # (parameter set, image, displacement), K = 2 N (N/2 + 1) real terms (N^2 in real space)
                    K = cfg.npix * cfg.npix if mode.endswith("_real") else cfg.npix * (cfg.npix + 2)
                    alg = 6.0 * K * evals * cfg.n_shift
                    ipt = 256 // cfg.n_shift
                    executed = 6.0 * K * (-(-n_ps // 128) * 128) * (-(-n_img // ipt) * 256)
                    per_launch_ms = k_ms / max(1, k_n)
                    achieved = alg / max(1, k_n / args.steps) / (per_launch_ms / 1e3) / 1e12
                    gsha = kernel_source_sha("k_score_gemm")
                    traffic = (K_SCORE_GEMM_TRAFFIC["bytes_per_launch"].get(f"{cfg.npix}/{mode}")
                               if K_SCORE_GEMM_TRAFFIC["source_sha256"] == gsha and n_img == 64 and n_ps == 6912 else None)
                    f["roofline"] = {"bound": "tensor", "achieved": achieved, "peak": peak_tf, "unit": "TFLOP/s",
                                     "frac": achieved / peak_tf, "traffic": traffic,
                                     "peak_basis": "measured cuBLAS bf16 burst (FP16 has the same dense rate)",
                                     "executed_tflops_incl_padding": executed / max(1, k_n / args.steps)
                                     / (per_launch_ms / 1e3) / 1e12}
                    f["operand_build_s"] = max(0.0, first_s - ms / 1e3)
                forms[mode] = f
            ctx.set_precision("fp32")
            sizes[str(cfg.npix)] = {"config": workload_config(cfg, n_img, n_ps), "forms": forms}
            im.close()
            ps.close()
    head = sizes["128"]["forms"]["fp16x2"]
    line = {"metric": METRIC, "value": head["evals_per_s"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f16x2 (split FP16 operands, FP32 accumulation)", "data": "synthetic",
            "config": {"workload": "precision: 64 images x 6912 parameter sets, shifts +-4, at 128 px and 64 px; "
                                   "value = the FP16 two-term form at 128 px",
                       "step": "bioem_score over resident images and projections"},
            "roofline": head["roofline"], "sizes": sizes, "gpu_launches": int(launches), "clocks": clocks.summary()}
    print(json.dumps(line), flush=True)
    return 0


def bench_shifts(args):
    """Where one back-transformation beats one correlation per displacement (Sec. 3.3, Fig. shifts),
    reproduced on synthetic data: evals/s of the FP32 pruned-FFT form and of the tensor-core forms
    (Fourier and real-space operands, BF16 two-term) against the shift half-width s, on the
    precision workloads (64 images x 6912 parameter sets at 128 px and 64 px)."""
    import torch

    import paper_1609_06634_gb300 as bioem
    from paper_1609_06634_gb300 import build

    build.build()
    dev = torch.device("cuda", 0)
    ctx = bioem.Context(0)
    stream = torch.cuda.current_stream(dev)
    sweep, crossover = {}, {}
    with ClockSampler(None) as clocks:
        for name in ("precision128", "precision64"):
            cfg = workloads.get_config(name)
            n_img = args.n_img or cfg.n_img
            wl = workloads.workload(cfg, n_img=0)
            quats_np = wl["quats"] if args.n_quat is None else wl["quats"][:args.n_quat]
            n_ps = len(quats_np) * len(wl["ctfs"])
            atoms_d = torch.from_numpy(wl["atoms"]).to(dev)
            im = bioem.prepare_images(ctx, synth_images(bioem, ctx, cfg, atoms_d, 0, n_img), cfg.pixel_A)
            ps = bioem.project_model(ctx, atoms_d, cfg.sigma_A, torch.from_numpy(np.ascontiguousarray(quats_np)).to(dev),
                                     wl["ctfs"], cfg.npix, cfg.pixel_A)
            logp = torch.empty(n_img, dtype=torch.float64, device=dev)
            fp32_max = {64: 8, 128: 16}[cfg.npix]
            res = {}
            for mode, shifts in [("fp32", sorted(set(list(range(0, 8)) + [8, 12, 16]))),
                                 ("bf16x2", list(range(0, 8))), ("bf16x2_real", list(range(0, 8)))]:
                res[mode] = {}
                ctx.set_precision(mode)
                for sh in shifts:
                    if mode == "fp32" and sh > fp32_max:
                        continue
                    for _ in range(max(1, args.warmup)):
                        bioem.score(ctx, im, ps, sh, out=logp)
                    torch.cuda.synchronize()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    for _ in range(args.steps):
                        bioem.score(ctx, im, ps, sh, out=logp)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ms = e0.elapsed_time(e1) / args.steps
                    res[mode][sh] = n_img * n_ps / (ms / 1e3)
                if ctx.status() != 0:
                    raise RuntimeError(f"device status error ({name}, {mode})")
            ctx.set_precision("fp32")
            # smallest s at which the FFT form is at least as fast as the per-displacement forms
            cross = next((sh for sh in range(0, 8) if res["fp32"][sh] >= max(res["bf16x2"][sh],
                                                                                res["bf16x2_real"][sh])), None)
            sweep[str(cfg.npix)] = {m: {str(k): v for k, v in r.items()} for m, r in res.items()}
            crossover[str(cfg.npix)] = cross if cross is not None else "beyond s = 7 (tensor-core forms faster)"
            im.close()
            ps.close()
    head = sweep["128"]["bf16x2"]["4"]
    line = {"metric": METRIC, "value": head, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (FFT form) / bf16x2 (tensor-core forms)", "data": "synthetic",
            "config": {"workload": "shift-window sweep: 64 images x 6912 parameter sets at 128 px and 64 px, "
                                   "s = 0..16; value = BF16 two-term form at 128 px, s = 4",
                       "step": "bioem_score over resident images and projections"},
            "sweep_evals_per_s": sweep, "fft_form_first_as_fast_at_s": crossover, "clocks": clocks.summary()}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse_args()
    if args.workload == "proposal":
        return bench_proposal(args)
    if args.impl == "reference":
        return bench_reference(args)
    if args.workload == "batched":
        return bench_batched(args)
    if args.workload == "precision":
        return bench_precision(args)
    if args.workload == "shifts":
        return bench_shifts(args)
    return bench_ours(args)


if __name__ == "__main__":
    sys.exit(main())
