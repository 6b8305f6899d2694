#!/usr/bin/env python
"""Benchmark of the demagnetizing operator applied as a sum of Kronecker products.

Metric: demag potential applications per second.  One step is one complete
application of the operator (all 3 components, all M = (R-1)/2 folded nodes,
summed output) to a full-format magnetization on a 256^3 grid (R = 41, the
vortex state with 5% noise); the same line reports the structured path on a
batch of CP magnetizations with n = 4096 per mode (CP rank 4 per component,
R = 61), where one application produces the CP output of rank 30*3*4.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints ONE JSON line on rank 0.  Under torchrun (N > 1) every rank runs the
same workload independently (the operator does not shard across GPUs here:
replicas only) and `value` is the total over ranks divided by the slowest
rank's time.  `--impl reference` times the FP64 CPU oracle on bounded samples
of the same workload.
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

METRIC = "demag potential apps/s at 256³ full & n=4096 CP; rel L2 err vs FP64 oracle"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
# DRAM bytes (read + write) per unit of work from ncu captures of smaller cases
# of the same kernels (traffic grows in proportion to the units processed), each
# keyed by a digest of the kernel's sources at capture time: a kernel changed
# since its capture reports traffic null.  The capture commands and their
# figures are summarised under profiles/.
NCU_TRAFFIC = {
    # the three tcgen05 mode-product stages of one application, BF16x3, R = 41,
    # per cell of the grid (captured at 192^3, folded axes)
    "tc_gemm_kernel": {"sources": ("full_tc.cu", "tc_ptx.cuh"), "sha": "05c5be55af52d644",
                       "bytes_per_cell": 5.73263e9 / 192 ** 3},
    # the fused schedule: tc_s12_kernel and the mode-3 tc_gemm_kernel launch of
    # one application, BF16x3, R = 41, per cell (captured at 192^3)
    "tc_fused": {"sources": ("full_tc.cu", "tc_ptx.cuh"), "sha": "05c5be55af52d644",
                 "bytes_per_cell": 2.36666e9 / 192 ** 3},
    # the Toeplitz FFT launch of a CP batch, n = 4096, r = 4, R = 61, per application
    "toeplitz_fft_kernel": {"sources": ("structured.cu", "fft.cuh"), "sha": "d08396a13974c222",
                            "bytes_per_app": 550.296e6 / 32},
}


def sources_sha(names):
    """Digest of the named CUDA sources of the package (the kernel as it stands)."""
    import hashlib
    hsh = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_1212_3509_gb300", "csrc", name), "rb") as f:
            hsh.update(f.read())
    return hsh.hexdigest()[:16]


def ncu_traffic(kernel, units, unit_key):
    """Captured DRAM bytes for `units` units, or None when the kernel changed since the capture."""
    rec = NCU_TRAFFIC[kernel]
    if rec["sha"] is None or rec.get(unit_key) is None or sources_sha(rec["sources"]) != rec["sha"]:
        return None
    return rec[unit_key] * units


# FP32 CUDA-core peak of a GB300: 152 SMs x 128 FP32 lanes x 2 flops (FMA) x 2.07 GHz
FP32_SIMT_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=256, help="full-format grid edge")
    ap.add_argument("--form", default="auto", help="auto | fp32 | fp64 | tf32x3 | bf16x3")
    ap.add_argument("--cp-n", type=int, default=4096)
    ap.add_argument("--cp-batch", type=int, default=256)
    ap.add_argument("--batch-grids", type=int, default=64, help="uneven full-format batch size (0: skip)")
    ap.add_argument("--c4-batch", type=int, default=128, help="Tucker / TT n=1024 batch (0: skip)")
    ap.add_argument("--no-oracle", action="store_true", help="skip the oracle error check and CPU baseline")
    ap.add_argument("--no-fig2", dest="fig2", action="store_false",
                    help="skip the uniform-cube energy study (Tucker format, n = 64..4096)")
    ap.add_argument("--no-tune", dest="tune", action="store_false",
                    help="default launch shapes (no autotuning before the timed region; for profiler runs)")
    ap.add_argument("--schedule", choices=("auto", "fused", "chain"), default="auto",
                    help="full-format forward schedule on tensor cores: the tuned choice (auto), the fused "
                         "mode-1/mode-2 kernel, or the three-stage chain")
    ap.add_argument("--cpu-table", action="store_true",
                    help="time the FP64 oracle on every configuration with 1 and with all host threads "
                         "(bounded samples) and print one JSON object; no GPU work")
    ap.add_argument("--cpu-one", default=None, help=argparse.SUPPRESS)
    return ap.parse_args()


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return dict(PEAKS_FALLBACK), "fallback"


class ClockSampler:
    """nvidia-smi clocks sampled every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def __enter__(self):
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        self.file.flush()

    def summary(self):
        rows = []
        try:
            with open(self.file.name) as f:
                for line in f:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
        finally:
            os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    """Largest per-rank time: the slowest replica sets the whole-job rate."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    device = "cpu" if dist.get_backend() == "gloo" else "cuda"
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, ms_max: float, world: int) -> float:
    """Units per second of all replicas together (weak scaling: every rank
    processes the same units; the slowest rank's time counts)."""
    return world * units_per_rank * 1e3 / ms_max


# ------------------------------------------------------------------ workloads

def bench_config(args, form, world):
    """The workload the headline value is quoted on (both arms report it)."""
    n, ncp, B = args.n, args.cp_n, args.cp_batch
    return {"workload": f"full format {n}^3, R=41 (M=20), form {form}; "
                        f"CP n={ncp} rank 4/component, R=61 (M=30), batch {B}",
            "grid": [n] * 3, "R": 41, "form": form, "cp_n": ncp, "cp_rank": 4, "cp_R": 61, "cp_batch": B,
            "parallelism": f"replicas x{world}",
            "l2": "inputs larger than L2 (m = 201 MB at 256^3; CP batch outputs 4.5 GB)"}


def full_config(n):
    return (n, n, n), (1.0 / n,) * 3, 41


def cp_config(n):
    return (n, n, n), (1.0 / n,) * 3, 61, 4


def make_cp_batch(n, r, batch, seed0):
    import numpy as np
    import synth
    lam = np.empty((batch, 3, r), dtype=np.float32)
    U = np.empty((batch, 3 * 3 * r * n), dtype=np.float32)
    for b in range(batch):
        l, u = synth.cp_inputs((n, n, n), r, seed0 + b)
        lam[b] = l
        U[b] = u.ravel()
    return lam, U


def time_region(fn, steps, stream):
    import torch
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(steps):
        fn()
    stop.record(stream)
    stop.synchronize()
    return start.elapsed_time(stop) / steps


def run_ours(args, world, rank, local):
    import numpy as np
    import torch
    import paper_1212_3509_gb300 as D
    import synth

    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    peaks, peak_src = load_peaks()

    # ---------------- full format, 256^3
    n3, h, R = full_config(args.n)
    form = args.form
    P = D.demag_build_factors(n3, h, R)
    # the autotuner times its candidates when the tensor-core state is created
    # (below, or on the first application), before the timed region
    if args.tune:
        D.demag_autotune(P, True)
    if args.schedule != "auto":
        D.demag_set_fused(P, args.schedule == "fused")
    if form == "auto":
        form = "fp32"
        for cand in ("bf16x3",):
            try:
                D.demag_reserve_workspace(P, cand)
                form = cand
                break
            except D.DemagError:
                pass
    D.demag_reserve_workspace(P, form)
    m_host = synth.vortex_m(n3, 1213)
    m = torch.from_numpy(m_host).cuda()
    phi = torch.empty(n3[2], n3[1], n3[0], device="cuda")
    full_fn = lambda: D.demag_apply_full(P, m, phi, form)  # noqa: E731
    for _ in range(args.warmup):
        full_fn()
    torch.cuda.synchronize()
    launches0 = D.demag_launch_count(P)
    D.demag_profile(P, True)
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ms_full = time_region(full_fn, args.steps, stream)
    torch.cuda.synchronize()
    barrier(world)
    D.demag_profile(P, False)
    launches_full = (D.demag_launch_count(P) - launches0) // args.steps
    fam = "gemm_tc" if form in ("bf16x3", "tf32x3") else "gemm_simt"
    gemm_ms, gemm_n = D.demag_profile_read(P, fam)
    split_ms, split_n = D.demag_profile_read(P, "split")
    misc_ms, _ = D.demag_profile_read(P, "misc")
    recs = [D.demag_profile_launch(P, i) for i in range(D.demag_profile_count(P))]
    gemm_recs = [t for f, t in recs if f == fam]
    per_app = max(1, len(gemm_recs) // args.steps)
    stage_ms = [sum(gemm_recs[j::per_app]) / args.steps for j in range(per_app)]
    ms_full_max = max_over_ranks(ms_full, world)

    M = P.M
    N1 = args.n
    # algorithmic work per application (Eq. kron_operator contracted densely by
    # Eq. modemul): 9 mode products of 2 n^4 flop per node; with the 8-GEMM
    # sharing of the chain 16 n^4 per node
    flops_app = 18.0 * (N1 ** 4) * M
    flops_app_8 = 16.0 * (N1 ** 4) * M
    gemm_ms_app = gemm_ms / args.steps
    achieved_tflops = flops_app / (gemm_ms_app * 1e-3) / 1e12
    hbm = peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"])
    hbm_note = f"{peak_src} STREAM copy (HBM)"
    # two tensor-core launches per application: the fused schedule (mode-1 and
    # mode-2 products in tc_s12_kernel, mode 3 in tc_gemm_kernel); three: the chain
    fused_sched = fam == "gemm_tc" and per_app == 2
    if fam == "gemm_tc":
        tpeak = peaks.get("bf16_tflops", PEAKS_FALLBACK["bf16_tflops"])
        if form == "tf32x3":
            tpeak = tpeak / 2.0  # TF32 dense rate is half the BF16 rate
        tpeak_note = f"{peak_src} dense {'bf16' if form == 'bf16x3' else 'tf32 (bf16/2)'} burst"
        # algorithmic DRAM bytes of the mode-product launches (folded layout,
        # the axis extents padded to 2 hq): the split input (3 fields), the
        # stage-1 intermediates (3M fields, written and read; not in the fused
        # schedule, where they stay on chip), the stage-2 intermediates (2M
        # fields, written and read), each as a hi and a lo plane, and the FP32
        # node-sum partial fields
        pair = 4 if form == "bf16x3" else 8
        al = 8 if form == "bf16x3" else 4
        hq = -(-((N1 + 1) // 2) // al) * al
        ext = 2 * hq if N1 > 16 else N1
        Nc = ext ** 3
        kb3 = -(-((N1 + 1) // 2 if N1 > 16 else N1) // (32 if form == "bf16x3" else 16))
        pp3 = max(1, (400 if form == "bf16x3" else 200) // (kb3 * 6))
        groups = -(-2 * M // pp3)
        gemm_bytes_app = pair * Nc * (3 + (4 if fused_sched else 10) * M) + 4.0 * groups * Nc
        achieved_gbs = gemm_bytes_app / (gemm_ms_app * 1e-3) / 1e9
        # the folded chain contracts h = n/2 entries per output (half the dense
        # MACs); the split forms issue 3 tensor-core products per product
        issued_tflops = flops_app_8 / 2.0 * 3.0 / (gemm_ms_app * 1e-3) / 1e12
        traffic = (ncu_traffic("tc_fused" if fused_sched else "tc_gemm_kernel", N1 ** 3, "bytes_per_cell")
                   if form == "bf16x3" else None)
        kname = ("tc_s12_kernel (tcgen05 mode-1 and mode-2 products, fused) and tc_gemm_kernel (mode 3 with "
                 "the node sum), the two launches of one application" if fused_sched else
                 "tc_gemm_kernel (tcgen05 mode products), the three stage launches of one application")
        roofline = {"kernel": kname, "schedule": "fused" if fused_sched else "chain",
                    "bound": "tensor", "achieved": achieved_tflops, "peak": tpeak, "unit": "TFLOP/s",
                    "frac": achieved_tflops / tpeak, "traffic": traffic,
                    "peak_source": tpeak_note,
                    "algorithmic_flops_per_app": flops_app,
                    "achieved_8gemm": flops_app_8 / (gemm_ms_app * 1e-3) / 1e12,
                    "frac_8gemm": flops_app_8 / (gemm_ms_app * 1e-3) / 1e12 / tpeak,
                    "algorithmic_flops_per_app_8gemm": flops_app_8,
                    "issued_tflops": issued_tflops, "issued_frac": issued_tflops / tpeak,
                    "hbm": {"achieved": achieved_gbs, "peak": hbm, "unit": "GB/s", "frac": achieved_gbs / hbm,
                            "algorithmic_bytes_per_app": gemm_bytes_app, "peak_source": hbm_note},
                    "launches_per_app": gemm_n / args.steps, "kernel_ms_per_app": gemm_ms_app,
                    "stage_ms_per_app": stage_ms,
                    "split_ms_per_app": split_ms / args.steps,
                    "reduce_ms_per_app": misc_ms / args.steps}
    else:
        tpeak = FP32_SIMT_PEAK_TFLOPS
        tpeak_note = "FP32 FMA peak from unit counts and max clock (152 SMs x 128 lanes x 2 x 2.07 GHz)"
        roofline = {"kernel": "gemm_tn_kernel (CUDA-core mode products), all stages of one application",
                    "bound": "alu", "achieved": achieved_tflops, "peak": tpeak, "unit": "TFLOP/s",
                    "frac": achieved_tflops / tpeak, "traffic": None, "peak_source": tpeak_note,
                    "algorithmic_flops_per_app": flops_app, "launches_per_app": gemm_n / args.steps,
                    "kernel_ms_per_app": gemm_ms_app, "stage_ms_per_app": stage_ms}

    # e2e through the public API with pinned host buffers: every step copies its
    # m from pinned host memory, applies the operator and reads phi back; steps
    # are double-buffered so step i+1's upload overlaps step i's compute
    m_pin = [torch.from_numpy(m_host).pin_memory() for _ in range(2)]
    phi_pin = [torch.empty(phi.shape, dtype=torch.float32).pin_memory() for _ in range(2)]
    m_dev = [torch.empty_like(m) for _ in range(2)]
    phi_dev = [torch.empty_like(phi) for _ in range(2)]
    up = torch.cuda.Stream()
    down = torch.cuda.Stream()
    ev_up = [torch.cuda.Event() for _ in range(2)]
    ev_done = [torch.cuda.Event() for _ in range(2)]
    ev_free = [torch.cuda.Event() for _ in range(2)]
    ev_read = [torch.cuda.Event() for _ in range(2)]

    def e2e_run(steps):
        for i in range(steps):
            b = i % 2
            with torch.cuda.stream(up):
                up.wait_event(ev_free[b])            # compute of step i-2 has consumed m_dev[b]
                m_dev[b].copy_(m_pin[b], non_blocking=True)
                ev_up[b].record(up)
            stream.wait_event(ev_up[b])
            stream.wait_event(ev_read[b])            # phi of step i-2 has been read back
            D.demag_apply_full(P, m_dev[b], phi_dev[b], form, stream=stream)
            ev_free[b].record(stream)
            ev_done[b].record(stream)
            with torch.cuda.stream(down):
                down.wait_event(ev_done[b])
                phi_pin[b].copy_(phi_dev[b], non_blocking=True)
                ev_read[b].record(down)

    e2e_run(max(2, args.warmup))
    torch.cuda.synchronize()
    barrier(world)
    t_start = torch.cuda.Event(enable_timing=True)
    t_stop = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    up.wait_stream(stream)
    down.wait_stream(stream)
    e2e_run(args.steps)
    stream.wait_stream(up)
    stream.wait_stream(down)
    t_stop.record(stream)
    t_stop.synchronize()
    ms_e2e = max_over_ranks(t_start.elapsed_time(t_stop) / args.steps, world)

    # ---------------- CP, n = 4096, batched
    ncp = args.cp_n
    cn3, ch, cR, r = cp_config(ncp)
    B = args.cp_batch
    PC = D.demag_build_factors(cn3, ch, cR)
    lam_h, U_h = make_cp_batch(ncp, r, B, 1214)
    lam = torch.from_numpy(lam_h).cuda()
    U = torch.from_numpy(U_h).cuda()
    Mc = PC.M
    out_w = torch.empty(B * Mc * 3 * r, device="cuda")
    out_U = torch.empty(B * Mc * 3 * r * 3 * ncp, device="cuda")
    if args.tune:
        D.demag_autotune(PC, True)
    cp_fn = lambda: D.demag_apply_cp_batched(PC, B, r, lam, U, out_w, out_U)  # noqa: E731
    for _ in range(args.warmup):
        cp_fn()
    torch.cuda.synchronize()
    cl0 = D.demag_launch_count(PC)
    D.demag_profile(PC, True)
    barrier(world)
    with ClockSampler(local) as clk_cp:
        ms_cp = time_region(cp_fn, args.steps, stream)
    D.demag_profile(PC, False)
    launches_cp = (D.demag_launch_count(PC) - cl0) // args.steps
    fft_ms, fft_n = D.demag_profile_read(PC, "fft")
    ms_cp_max = max_over_ranks(ms_cp, world)
    bytes_app = 4.0 * (9 * r * ncp + 3 * r) + 4.0 * (Mc * 3 * r * 3 * ncp + Mc * 3 * r)
    sym_bytes = 4.0 * Mc * 2 * (ncp + 1)  # symbol pairs of one axis (read once per axis)
    # all three modes run in one launch per batch (they share the FFT length)
    fft_batch_ms = fft_ms / args.steps
    fft_batch_bytes = B * bytes_app + 3 * sym_bytes
    fft_gbs = fft_batch_bytes / (fft_batch_ms * 1e-3) / 1e9
    hbm = peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"])
    # algorithmic FFT flops per application: 2.5 L log2 L per real transform of
    # length L = 2n (36 forward, 30*36 inverse), plus 2 flops per symbol product bin
    import math
    Lc = 2 * ncp
    fft_flops_app = (9 * r + Mc * 9 * r) * 2.5 * Lc * math.log2(Lc) + Mc * 9 * r * 2 * (Lc // 2 + 1)
    fft_tflops = B * fft_flops_app / (fft_batch_ms * 1e-3) / 1e12

    # ---------------- Tucker and TT, n = 1024, ranks 8, R = 61, batched, CUDA graph
    c4 = None
    if args.c4_batch > 0:
        c4 = run_c4(args, D, world, local, stream, peaks)

    # ---------------- energy study after Alg. 2: uniform cube in Tucker form, n = 64..4096
    fig2 = run_fig2(args, D, stream) if args.fig2 else None

    # ---------------- uneven batch: 64 grids of mixed shape, BF16x3, CUDA graph
    batch = None
    if args.batch_grids > 0:
        batch = run_uneven_batch(args, D, world, local, stream, form="bf16x3")

    result = {
        "metric": METRIC,
        "value": whole_job_rate(1, ms_full_max, world),
        "unit": "apps/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_full_max,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp64": "f64", "tf32x3": "tf32x3 (f32 accumulate)",
                  "bf16x3": "bf16x3 (f32 accumulate)"}[form],
        "data": "synthetic (seeded vortex state + 5% noise; smooth random CP factors)",
        "config": bench_config(args, form, world),
        "roofline": roofline,
        "cp": {"value": world * B * 1e3 / ms_cp_max, "unit": "apps/s", "ms_per_batch": ms_cp_max,
               "batch": B,
               "roofline": {"kernel": "toeplitz_fft_kernel", "bound": "hbm", "achieved": fft_gbs, "peak": hbm,
                            "unit": "GB/s", "frac": fft_gbs / hbm,
                            "traffic": (ncu_traffic("toeplitz_fft_kernel", B, "bytes_per_app")
                                        if ncp == 4096 else None),
                            "algorithmic_bytes_per_app": bytes_app, "launches_per_batch": fft_n / args.steps,
                            "kernel_ms_per_batch": fft_ms / args.steps, "peak_source": hbm_note,
                            "alu": {"achieved": fft_tflops, "peak": FP32_SIMT_PEAK_TFLOPS, "unit": "TFLOP/s",
                                    "frac": fft_tflops / FP32_SIMT_PEAK_TFLOPS,
                                    "algorithmic_flops_per_app": fft_flops_app,
                                    "peak_source": "FP32 FMA peak from unit counts and max clock"}},
               "gpu_launches": launches_cp,
               "clocks": clk_cp.summary()},
        "e2e": {"value": world * 1e3 / ms_e2e, "unit": "apps/s",
                "h2d_bytes_per_step": int(m.numel() * 4), "d2h_bytes_per_step": int(phi.numel() * 4)},
        "gpu_launches": int(launches_full),
        "clocks": clk.summary(),
        "autotune": {"full": [D.demag_autotune_entry(P, i) for i in range(D.demag_autotune_count(P))],
                     "cp": [D.demag_autotune_entry(PC, i) for i in range(D.demag_autotune_count(PC))],
                     "note": "chosen per stage program before the timed region; ms = chosen, "
                             "ms_default = the default setting, per launch"},
    }

    # ---------------- every full-format form on the same input (C2: error per form)
    phis = {}
    forms = {}
    for f in ("fp64", "fp32", "tf32x3", "bf16x3"):
        try:
            D.demag_reserve_workspace(P, f)
        except D.DemagError:
            continue
        out = torch.empty_like(phi)
        fn = lambda: D.demag_apply_full(P, m, out, f)  # noqa: E731
        fn()
        torch.cuda.synchronize()
        ms_f = time_region(fn, 2 if f == "fp64" else max(2, args.steps // 3), stream)
        forms[f] = {"apps_per_s": 1e3 / ms_f, "ms_per_app": ms_f}
        phis[f] = out

    # ---------------- the 128^3 point of the same configuration, every form
    c2_128 = run_c2_128(args, D, stream) if args.n == 256 else None

    # ---------------- the same operator by one 3D FFT convolution (Eq. fft_pot, node-summed kernel)
    fft3d = run_fft3d(args, D, world, local, stream, P, m, phi, peaks, n3)
    fibres = run_fibres(args, D, world, local, stream, P, m, phi, peaks, n3)

    # ---------------- the FFT path at 1024^3 (1.07 G cells; the cost does not depend on R)
    fft1024 = run_fft3d_1024(args, D, world, local, stream) if args.n == 256 else None

    # ---------------- the same application on a graded (non-uniform) 256^3 grid, BF16x3
    nonuni = run_nonuniform(args, D, world, local, stream, m, n3) if form == "bf16x3" else None

    # ---------------- demag energy and its gradient (forward, adjoint, FD stencils), 256^3 BF16x3
    energy = None
    if form in ("bf16x3", "tf32x3"):
        e_out = torch.empty(1, dtype=torch.float64, device="cuda")
        grad = torch.empty_like(m)
        efn = lambda: D.demag_energy(P, m, e_out, grad, form)  # noqa: E731
        efn()
        torch.cuda.synchronize()
        ms_e = time_region(efn, max(3, args.steps // 2), stream)
        energy = {"value": whole_job_rate(1, max_over_ranks(ms_e, world), world), "unit": "energy+gradient evals/s",
                  "ms_per_eval": ms_e, "form": form,
                  "work": "phi = P m, h_d = -D phi, E = -1/2 h^3 sum m.h_d, grad = 1/2 h^3 (D P m + P^T D^T m)"}
        # analytic stray field: the three derivative chains (eight stage launches)
        hd = torch.empty_like(m)
        ffn = lambda: D.demag_stray_field_exact(P, m, hd, form)  # noqa: E731
        ffn()
        torch.cuda.synchronize()
        ms_f = time_region(ffn, max(3, args.steps // 2), stream)
        energy["exact_stray_field"] = {"value": whole_job_rate(1, max_over_ranks(ms_f, world), world),
                                       "unit": "fields/s", "ms_per_field": ms_f, "form": form,
                                       "work": "h_d = -grad phi from derivative Kronecker factors, 3 directions"}
        # the same field by one 3D FFT convolution with the six node-summed derivative kernels
        hf = torch.empty_like(m)
        gfn = lambda: D.demag_stray_field_fft(P, m, hf)  # noqa: E731
        gfn()
        torch.cuda.synchronize()
        ms_g = time_region(gfn, max(3, args.steps // 2), stream)
        torch.cuda.synchronize()
        den = float(torch.linalg.vector_norm(hd.double()))
        energy["stray_field_fft"] = {"value": whole_job_rate(1, max_over_ranks(ms_g, world), world),
                                     "unit": "fields/s", "ms_per_field": ms_g, "form": "fp32 FFT",
                                     "rel_l2_vs_exact_stray_field": float(torch.linalg.vector_norm(
                                         (hf - hd).double())) / (den if den > 0 else 1.0),
                                     "work": "h_d[p] = IDFT(sum_q K_pq . DFT(m^(q))), K_pq the node-summed "
                                             "derivative kernels; five FFT passes"}
        ee = torch.empty(1, dtype=torch.float64, device="cuda")
        gg = torch.empty_like(m)
        efn2 = lambda: D.demag_energy_field_fft(P, m, ee, gg)  # noqa: E731
        efn2()
        torch.cuda.synchronize()
        ms_e2 = time_region(efn2, max(3, args.steps // 2), stream)
        energy["energy_field_fft"] = {"value": whole_job_rate(1, max_over_ranks(ms_e2, world), world),
                                      "unit": "energy+gradient evals/s", "ms_per_eval": ms_e2,
                                      "work": "E = -1/2 V sum m.h_d and dE/dm = -V h_d with h_d the analytic "
                                              "collocation field by one 3D FFT convolution"}

    # ---------------- parity against the oracle (sampled) and CPU baseline
    if not args.no_oracle and rank == 0:
        from oracle import full as ofull, structured as ost
        lines = [(0, 0), (n3[2] // 2, n3[1] // 3), (n3[2] - 1, n3[1] - 1), (n3[2] // 4, n3[1] - 7)]
        ref = ofull.apply_full_lines(m_host, n3, h, R, lines)

        def sampled_err(field):
            got = field.cpu().numpy()
            num = sum(float(((got[i3, i2] - ref[j]) ** 2).sum()) for j, (i3, i2) in enumerate(lines))
            den = sum(float((ref[j] ** 2).sum()) for j in range(len(lines)))
            return (num / den) ** 0.5

        result["rel_l2_full"] = sampled_err(phi)
        result["rel_l2_full_sample"] = f"{len(lines)} output lines phi[i3,i2,:] vs the FP64 oracle"
        for f, field in phis.items():
            forms[f]["rel_l2"] = sampled_err(field)
        if fft3d is not None:
            fft3d["rel_l2"] = sampled_err(fft3d.pop("_phi"))
        if fibres is not None:
            fibres["rel_l2"] = sampled_err(fibres.pop("_phi"))
        if nonuni is not None:
            from oracle import nonuniform as onu
            ref_nu = onu.apply_full_lines(m_host, nonuni.pop("_edges"), R, lines)
            got_nu = nonuni.pop("_phi").cpu().numpy()
            num = sum(float(((got_nu[i3, i2] - ref_nu[j]) ** 2).sum()) for j, (i3, i2) in enumerate(lines))
            den = sum(float((ref_nu[j] ** 2).sum()) for j in range(len(lines)))
            nonuni["rel_l2"] = (num / den) ** 0.5
        rw, rU = ost.apply_cp(lam_h[0], U_h[0], cn3, ch, cR)
        ref_cp = np.concatenate([rU[p].ravel() for p in range(3)])
        got_cp = out_U[: Mc * 3 * r * 3 * ncp].cpu().numpy()
        result["cp"]["rel_l2"] = float(np.linalg.norm(got_cp - ref_cp) / np.linalg.norm(ref_cp))
        result["cpu_baseline"] = cpu_baseline(n3, h, R, m_host, budget_s=20.0)
    result["forms_full"] = forms
    if c2_128 is not None:
        if not args.no_oracle and rank == 0:
            from oracle import full as ofull
            n128, h128, R128 = full_config(128)
            lines = [(0, 0), (64, 42), (127, 127), (32, 121)]
            ref = ofull.apply_full_lines(c2_128["_m"], n128, h128, R128, lines)
            for f, field in c2_128["_phi"].items():
                got = field.cpu().numpy()
                g = np.stack([got[i3, i2] for i3, i2 in lines])
                c2_128["forms"][f]["rel_l2"] = float(np.linalg.norm(g - ref) / np.linalg.norm(ref))
            c2_128["rel_l2_sample"] = f"{len(lines)} output lines phi[i3,i2,:] vs the FP64 oracle"
        c2_128.pop("_m")
        c2_128.pop("_phi")
        result["full_128"] = c2_128
    if fft3d is not None:
        fft3d.pop("_phi", None)
        result["full_fft3d"] = fft3d
    if fibres is not None:
        fibres.pop("_phi", None)
        result["full_fibres"] = fibres
    if nonuni is not None:
        nonuni.pop("_phi", None)
        nonuni.pop("_edges", None)
        result["full_nonuniform"] = nonuni
    if fft1024 is not None:
        result["full_fft3d_1024"] = fft1024
    if energy is not None:
        result["energy_gradient"] = energy
    if c4 is not None:
        if not args.no_oracle and rank == 0:
            from oracle import structured as ost
            n3, h, R = c4.pop("_cfg")
            core, Vh = c4.pop("_tucker_in")
            rw, rV = ost.apply_tucker(core, Vh, n3, (8, 8, 8), h, R)
            got = c4.pop("_tucker_out").cpu().numpy()
            ref = np.concatenate([rV[p].ravel() for p in range(3)])
            c4["tucker"]["rel_l2"] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
            G1, G2, G3 = c4.pop("_tt_in")
            rw, r1, r2, r3 = ost.apply_tt(G1, G2, G3, n3, (8, 8), h, R)
            outs = c4.pop("_tt_out")
            num = sum(float(np.linalg.norm(o.cpu().numpy() - rr.ravel()) ** 2) for o, rr in zip(outs, (r1, r2, r3)))
            den = sum(float(np.linalg.norm(rr) ** 2) for rr in (r1, r2, r3))
            c4["tt"]["rel_l2"] = (num / den) ** 0.5
            c4["rel_l2_sample"] = "the first batch item of each format in full vs the FP64 oracle"
        for k in [k for k in c4 if k.startswith("_")]:
            del c4[k]
        result["tucker_tt"] = c4
    if fig2 is not None:
        result["energy_study_uniform_cube"] = fig2
    if batch is not None:
        if not args.no_oracle and rank == 0:
            from oracle import full as ofull
            errs = []
            for i in batch.pop("_check"):
                sn, sh, sR = batch["_shapes"][i], batch["_h"][i], 41
                lines = [(0, 0), (sn[2] // 2, sn[1] - 1)]
                ref = ofull.apply_full_lines(batch["_m"][i], sn, sh, sR, lines)
                g = batch["_phi"][i].cpu().numpy()
                got = np.stack([g[i3, i2] for i3, i2 in lines])
                errs.append(float(np.linalg.norm(got - ref) / np.linalg.norm(ref)))
            batch["rel_l2_sampled_max"] = max(errs)
            batch["rel_l2_sample"] = "2 output lines of the first cube and the first 512x512x4 film vs the FP64 oracle"
        for k in [k for k in batch if k.startswith("_")]:
            del batch[k]
        result["uneven_batch"] = batch
    print(json.dumps(result), flush=True)


def run_c2_128(args, D, stream):
    """The 128^3 point of the full-format configuration (R = 41, vortex + 5% noise), every form."""
    import torch
    import synth
    n3, h, R = full_config(128)
    P = D.demag_build_factors(n3, h, R)
    m_host = synth.vortex_m(n3, 1213)
    m = torch.from_numpy(m_host).cuda()
    forms, phis = {}, {}
    for f in ("fp64", "fp32", "tf32x3", "bf16x3"):
        out = torch.empty(128, 128, 128, device="cuda")
        fn = lambda: D.demag_apply_full(P, m, out, f)  # noqa: E731
        fn()
        torch.cuda.synchronize()
        ms_f = time_region(fn, 3 if f == "fp64" else max(3, args.steps), stream)
        forms[f] = {"apps_per_s": 1e3 / ms_f, "ms_per_app": ms_f}
        phis[f] = out
    D.demag_sync_status(P)
    return {"grid": "128^3", "R": R, "forms": forms, "_m": m_host, "_phi": phis}


def fig2_terms(n, c0=2.15):
    """R for the n^3 uniform cube of the energy study: the sinc rule is not uniform
    in h (Remark after Lemma 2), so the largest node tau_max = sinh(c0 ln M) must
    grow with the cells per edge; the smallest M of 64, 128, 256 with
    tau_max >= 8 n (tau_max h >= 8 on the unit cube)."""
    import math
    for M in (64, 128, 256):
        if math.sinh(c0 * math.log(M)) >= 8 * n:
            return 2 * M + 1
    return 513


def run_fig2(args, D, stream, sizes=(64, 128, 256, 512, 1024, 2048, 4096), tol=1e-6):
    """The energy study after Alg. 2: the uniformly magnetized unit cube (m = z, a rank-1 Tucker
    tensor) on n^3 grids, its potential in Tucker form and the second-order energy without forming
    a full tensor.  Per n (R growing with n, fig2_terms): the relative energy error against the
    continuum value 1/6 and the time of one application plus energy (CUDA events, plain operator);
    and Alg. 2 proper (kernels compressed at tol, compressed application, approximate summation at
    tol, energy of the single Tucker potential) at R = 129, the largest R its compression takes:
    its ranks, energy error and wall time."""
    import math
    import time as _t
    import torch
    out = {"tol": tol, "sizes": list(sizes), "R_rule": "smallest M in {64, 128, 256} with sinh(c0 ln M) >= 8 n",
           "rows": [],
           "work": "demag_apply_tucker + demag_energy_tucker (rank 1, FP32 factors); fp64: "
                   "demag_energy_tucker_fp64 (FP64 Tucker application and energy); Alg. 2: demag_compress_kernel, "
                   "demag_apply_tucker_compressed, demag_recompress_tucker, demag_energy_tucker_phi (R = 129)"}
    ranks = (1, 1, 1)
    for n in sizes:
        R = fig2_terms(n)
        core = torch.zeros(3, device="cuda")
        core[2] = 1.0
        V = torch.ones(9 * n, device="cuda")
        E = torch.empty((), dtype=torch.float64, device="cuda")
        P = D.demag_build_factors((n, n, n), (1.0 / n,) * 3, R)
        w = torch.empty(P.M * 3, device="cuda")
        oV = torch.empty(P.M * 9 * n, device="cuda")

        def fn():
            D.demag_apply_tucker(P, ranks, V, w, oV)
            D.demag_energy_tucker(P, ranks, core, V, w, oV, E)
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        ms = time_region(fn, 20, stream)
        e = float(E.item())
        row = {"n": n, "R": R, "energy": e, "rel_err": abs(e - 1.0 / 6.0) * 6.0, "ms_apply_energy": ms}
        # the same energy with the Tucker application in FP64 (direct Toeplitz sums)
        core64, V64 = core.double(), V.double()

        def fn64():
            D.demag_energy_tucker_fp64(P, ranks, core64, V64, E)
        fn64()
        torch.cuda.synchronize()
        ms64 = time_region(fn64, 3, stream)
        e64 = float(E.item())
        row["fp64"] = {"energy": e64, "rel_err": abs(e64 - 1.0 / 6.0) * 6.0, "ms_apply_energy": ms64}
        del P
        try:
            P2 = D.demag_build_factors((n, n, n), (1.0 / n,) * 3, 129)
            D.demag_compress_kernel(P2, tol)
            rho = D.demag_compressed_ranks(P2)
            out_V = torch.empty(sum(3 * rho[p] * n for p in range(3)), device="cuda")
            torch.cuda.synchronize()
            t0 = _t.perf_counter()
            D.demag_apply_tucker_compressed(P2, 1, ranks, core, V, None, out_V)
            rk, C, Us, _ = D.demag_recompress_tucker(P2, ranks, core, out_V, tol)
            D.demag_energy_tucker_phi(P2, ranks, core, V, rk, C.contiguous().view(-1),
                                      torch.cat([u.reshape(-1) for u in Us]), E)
            ea = float(E.item())
            row["alg2"] = {"R": 129, "kernel_ranks": list(rho), "phi_ranks": list(rk), "energy": ea,
                           "rel_err": abs(ea - 1.0 / 6.0) * 6.0, "seconds": _t.perf_counter() - t0}
            del P2
        except D.DemagError as ex:
            row["alg2"] = {"unavailable": str(ex)}
        out["rows"].append(row)
    errs = [r["rel_err"] for r in out["rows"]]
    out["order_per_doubling"] = [math.log2(errs[i] / errs[i + 1]) if errs[i + 1] > 0 else None
                                 for i in range(len(errs) - 1)]
    e64 = [r["fp64"]["rel_err"] for r in out["rows"]]
    out["fp64_order_per_doubling"] = [math.log2(e64[i] / e64[i + 1]) if e64[i + 1] > 0 else None
                                      for i in range(len(e64) - 1)]
    # the same energies by the FP64 oracle's one-dimensional sums (after the timed work): what
    # the method gives without the FP32 factors, and how far the GPU values are from it
    from oracle import energy as oen
    oerr = []
    for r in out["rows"]:
        eo = oen.uniform_cube_energy(r["n"], r["R"])
        r["oracle_fp64"] = {"energy": eo, "rel_err": abs(eo - 1.0 / 6.0) * 6.0,
                            "gpu_minus_oracle_rel": (r["energy"] - eo) / eo,
                            "fp64_minus_oracle_rel": (r["fp64"]["energy"] - eo) / eo}
        oerr.append(r["oracle_fp64"]["rel_err"])
    out["oracle_order_per_doubling"] = [math.log2(oerr[i] / oerr[i + 1]) for i in range(len(oerr) - 1)]
    a2 = [r["alg2"].get("rel_err") for r in out["rows"]]
    out["alg2_order_per_doubling"] = [math.log2(a2[i] / a2[i + 1]) if a2[i] and a2[i + 1] else None
                                      for i in range(len(a2) - 1)]
    return out


def fft3d_pass_bytes(n):
    """Algorithmic DRAM bytes of the five passes of one 3D FFT convolution (read + write, FP32 data,
    complex spectra of 8 bytes, the kernel octant read once)."""
    def pow2(v):
        L = 1
        while L < 2 * v - 1:
            L *= 2
        return max(L, 2)
    n1, n2, n3 = n
    L1, L2, L3 = pow2(n1), pow2(n2), pow2(n3)
    H1, H2, H3 = L1 // 2 + 1, L2 // 2 + 1, L3 // 2 + 1
    s1 = 3 * H1 * n3 * n2 * 8
    s2 = 3 * L2 * H1 * n3 * 8
    s3 = n3 * H1 * L2 * 8
    s4 = n2 * n3 * H1 * 8
    return [3 * n1 * n2 * n3 * 4 + s1, s1 + s2, s2 + 3 * H1 * H2 * H3 * 4 + s3, s3 + s4, s4 + n1 * n2 * n3 * 4]


def run_fft3d(args, D, world, local, stream, P, m, phi, peaks, n3):
    """demag_apply_full_fft on the headline grid: throughput, per-pass times and the HBM roofline."""
    import torch
    out = torch.empty_like(phi)
    fn = lambda: D.demag_apply_full_fft(P, m, out)  # noqa: E731
    try:
        fn()
    except D.DemagError:
        return None
    for _ in range(args.warmup):
        fn()
    torch.cuda.synchronize()
    steps = max(5, args.steps)
    barrier(world)
    with ClockSampler(local) as clk:
        ms = time_region(fn, steps, stream)
    ms_max = max_over_ranks(ms, world)
    # per-pass device times (CUDA events around each launch, a separate run)
    D.demag_profile(P, True)
    reps = 5
    for _ in range(reps):
        fn()
    torch.cuda.synchronize()
    per = [0.0] * 5
    for i in range(D.demag_profile_count(P)):
        fam, t = D.demag_profile_launch(P, i)
        per[i % 5] += t / reps
    D.demag_profile(P, False)
    pb = fft3d_pass_bytes(n3)
    hbm = peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"])
    top = max(range(5), key=lambda i: per[i])
    ach = sum(pb) / (sum(per) * 1e-3) / 1e9
    return {"value": whole_job_rate(1, ms_max, world), "unit": "apps/s", "ms_per_app": ms_max,
            "work": "phi = IDFT(sum_q K^(q) . DFT(m^(q))) on the padded grid; five FP32 FFT passes; "
                    "kernel K summed over the R nodes once per plan (setup, not timed)",
            "launches_per_app": 5,
            "pass_ms": per, "pass_algorithmic_bytes": pb,
            "roofline": {"kernel": "fft3d passes (all five)", "bound": "hbm", "achieved": ach, "peak": hbm,
                         "unit": "GB/s", "frac": ach / hbm,
                         "top_pass": {"pass": top + 1, "ms": per[top], "achieved": pb[top] / (per[top] * 1e-3) / 1e9,
                                      "frac": pb[top] / (per[top] * 1e-3) / 1e9 / hbm},
                         "traffic": None},
            "clocks": clk.summary(), "_phi": out}


def run_fibres(args, D, world, local, stream, P, m, phi, peaks, n3):
    """demag_apply_full_fibres on the headline grid: per-fibre 1D Toeplitz FFTs along each axis
    (all nodes along axis 1, node by node along axes 2 and 3), transposes between, weighted sum."""
    import torch
    out = torch.empty_like(phi)
    fn = lambda: D.demag_apply_full_fibres(P, m, out)  # noqa: E731
    try:
        fn()
    except D.DemagError:
        return None
    for _ in range(args.warmup):
        fn()
    torch.cuda.synchronize()
    barrier(world)
    with ClockSampler(local) as clk:
        ms = time_region(fn, max(3, args.steps), stream)
    ms_max = max_over_ranks(ms, world)
    N = n3[0] * n3[1] * n3[2]
    M = P.M
    # m in, 3M fields out of each of the three Toeplitz stages and the two transposes (read + write
    # between), the sum reads 3M fields and writes phi
    bytes_app = 4.0 * (4 * N + 30 * M * N)
    hbm = peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"])
    ach = bytes_app / (ms_max * 1e-3) / 1e9
    launches = 6
    return {"value": whole_job_rate(1, ms_max, world), "unit": "apps/s", "ms_per_app": ms_max,
            "work": "Toeplitz FFTs of the axis-1 fibres for all M nodes, then of the axis-2 and axis-3 fibres "
                    "of each (node, component) volume; two batched transposes; weighted sum over (k, q)",
            "launches_per_app": launches,
            "roofline": {"kernel": "per-fibre chain (all six launches)", "bound": "hbm", "achieved": ach,
                         "peak": hbm, "unit": "GB/s", "frac": ach / hbm, "algorithmic_bytes_per_app": bytes_app,
                         "traffic": None},
            "clocks": clk.summary(), "_phi": out}


def run_fft3d_1024(args, D, world, local, stream):
    """demag_apply_full_fft on 1024^3, R = 41 (random unit m): about 110 GB of device memory for the
    input, output, spectra and kernel; skipped when that much is not free."""
    import gc
    import torch
    free, _ = torch.cuda.mem_get_info()
    if free < 160e9:
        return {"skipped": f"needs ~110 GB free device memory, {free / 1e9:.0f} GB free"}
    n3 = (1024, 1024, 1024)
    P = D.demag_build_factors(n3, (1.0 / 1024,) * 3, 41)
    # random unit vectors drawn on the device (a host copy would take 13 GB); the
    # cost of this path does not depend on the values
    g = torch.Generator(device="cuda").manual_seed(1212)
    m = torch.randn(3, 1024, 1024, 1024, device="cuda", generator=g)
    m /= torch.linalg.vector_norm(m, dim=0, keepdim=True)
    phi = torch.empty(1024, 1024, 1024, device="cuda")
    fn = lambda: D.demag_apply_full_fft(P, m, phi)  # noqa: E731
    fn()
    torch.cuda.synchronize()
    fn()
    barrier(world)
    with ClockSampler(local) as clk:
        ms = time_region(fn, 3, stream)
    ms = max_over_ranks(ms, world)
    pb = sum(fft3d_pass_bytes(n3))
    out = {"value": whole_job_rate(1, ms, world), "unit": "apps/s", "ms_per_app": ms, "cells": 1024 ** 3,
           "algorithmic_bytes_per_app": pb, "hbm_achieved_gbs": pb / (ms * 1e-3) / 1e9,
           "work": "the 256^3 FFT path at 1024^3 (FFT length 2048 per axis); one GPU", "clocks": clk.summary()}
    del P, m, phi
    gc.collect()
    torch.cuda.empty_cache()
    return out


def graded_edges(n, ratio):
    """n cells on [0, 1] whose widths grow geometrically by `ratio` from the first cell."""
    import numpy as np
    w = ratio ** np.arange(n, dtype=np.float64)
    return np.concatenate([[0.0], np.cumsum(w)]) / w.sum()


def run_nonuniform(args, D, world, local, stream, m, n3):
    """demag_apply_full (BF16x3) on a graded grid of the headline size: widths growing 0.5%/1%/0.2% per
    cell along the three axes (factor 3.6 / 13 / 1.7 from the first to the last cell)."""
    import torch
    edges = [graded_edges(n3[p], r) for p, r in enumerate((1.005, 1.01, 1.002))]
    P = D.demag_build_factors_nonuniform(edges, 41)
    out = torch.empty(n3[2], n3[1], n3[0], device="cuda")
    fn = lambda: D.demag_apply_full(P, m, out, "bf16x3")  # noqa: E731
    fn()
    for _ in range(args.warmup):
        fn()
    torch.cuda.synchronize()
    barrier(world)
    with ClockSampler(local) as clk:
        ms = time_region(fn, max(5, args.steps), stream)
    ms_max = max_over_ranks(ms, world)
    return {"value": whole_job_rate(1, ms_max, world), "unit": "apps/s", "ms_per_app": ms_max, "form": "bf16x3",
            "grid": "256^3 on [0,1]^3, cell widths growing geometrically by 1.005 / 1.01 / 1.002 per cell",
            "work": "the same tensor-core chain with dense (non-Toeplitz) factor matrices from the true cell limits",
            "clocks": clk.summary(), "_phi": out, "_edges": edges}


def run_c4(args, D, world, local, stream, peaks):
    """Tucker (multilinear ranks 8, 8, 8) and TT (ranks 8, 8) inputs on n = 1024
    per axis, R = 61: batched calls (one Toeplitz-FFT launch for all axes,
    nodes, components and items) captured in a CUDA graph and replayed."""
    import torch
    import synth
    n, B = 1024, args.c4_batch
    n3, h, R = (n,) * 3, (1.0 / n,) * 3, 61
    P = D.demag_build_factors(n3, h, R)
    M = P.M
    rt, rr = (8, 8, 8), (8, 8)
    tot = sum(rt)
    tucker_in = synth.tucker_inputs(n3, rt, 1500)
    V = torch.cat([torch.from_numpy(synth.tucker_inputs(n3, rt, 1500 + b)[1].ravel()) for b in range(B)]).cuda()
    tw = torch.empty(B * M * 3, device="cuda")
    tV = torch.empty(B * M * 3 * tot * n, device="cuda")
    tt_in = synth.tt_inputs(n3, rr, 1600)
    tts = [tt_in] + [synth.tt_inputs(n3, rr, 1600 + b) for b in range(1, B)]
    G = [torch.cat([torch.from_numpy(t[i].ravel()) for t in tts]).cuda() for i in range(3)]
    sizes = [8 * n, 64 * n, 8 * n]
    ww = torch.empty(B * M * 3, device="cuda")
    tO = [torch.empty(B * M * 3 * sz, device="cuda") for sz in sizes]
    hbm = peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"])
    out = {"n": n, "R": R, "batch": B, "_cfg": (n3, h, R)}
    sym_bytes = 3 * 4.0 * M * 2 * (n + 1)
    legs = {
        "tucker": (lambda st: D.demag_apply_tucker_batched(P, B, rt, V, tw, tV, st),
                   4.0 * (3 * tot * n) + 4.0 * (M * 3 * tot * n + M * 3)),
        "tt": (lambda st: D.demag_apply_tt_batched(P, B, rr, G[0], G[1], G[2], ww, *tO, stream=st),
               4.0 * 3 * sum(sizes) + 4.0 * (M * 3 * sum(sizes) + M * 3)),
    }
    for name, (call, bytes_app) in legs.items():
        fn = lambda: call(stream)  # noqa: E731
        fn()  # warm-up outside the capture (plan-level setup, kernel attributes)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            with torch.cuda.graph(g, stream=side):
                call(side)
        stream.wait_stream(side)
        replay = lambda: g.replay()  # noqa: E731
        for _ in range(args.warmup):
            replay()
        torch.cuda.synchronize()
        l0 = D.demag_launch_count(P)
        D.demag_profile(P, True)
        fn()
        D.demag_profile(P, False)
        fft_ms, fft_n = D.demag_profile_read(P, "fft")
        launches = D.demag_launch_count(P) - l0
        barrier(world)
        with ClockSampler(local) as clk:
            ms = time_region(replay, max(3, args.steps), stream)
        ms = max_over_ranks(ms, world)
        gbs = (B * bytes_app + sym_bytes) / (fft_ms * 1e-3) / 1e9
        out[name] = {"value": whole_job_rate(B, ms, world), "unit": "apps/s", "ms_per_batch": ms,
                     "kernel_ms_per_batch": fft_ms, "fft_launches_per_batch": fft_n, "gpu_launches": int(launches),
                     "roofline": {"kernel": "toeplitz_fft_kernel", "bound": "hbm", "achieved": gbs, "peak": hbm,
                                  "unit": "GB/s", "frac": gbs / hbm, "traffic": None,
                                  "algorithmic_bytes_per_app": bytes_app},
                     "clocks": clk.summary(), "timing": "CUDA-graph replays of the batched call"}
    out["tucker_compressed"] = run_tucker_compressed(args, D, world, local, stream, P, n3, rt, B, V, tw, tV, hbm)
    out["tt_rounded"] = run_tt_round(D, P, n3)
    out["tucker_energy"] = run_tucker_energy(D, P, n3, rt, tucker_in, stream)
    out["tt_energy"] = run_tt_energy(D, P, n3, rr, tt_in, stream)
    out["_tucker_in"] = tucker_in
    out["_tucker_out"] = tV[:M * 3 * tot * n]
    out["_tt_in"] = tt_in
    out["_tt_out"] = [o[:M * 3 * sz] for o, sz in zip(tO, sizes)]
    return out


def run_tucker_energy(D, P, n3, rt, tucker_in, stream):
    """Demag energy of one rank-(8, 8, 8) Tucker magnetization on the 1024^3 grid without forming a
    full tensor: demag_apply_tucker + demag_energy_tucker, CUDA events over 10 calls."""
    import torch
    core, Vh = tucker_in
    n, M = n3[0], P.M
    tot = sum(rt)
    cd = torch.from_numpy(core.ravel()).cuda()
    Vd = torch.from_numpy(Vh.ravel()).cuda()
    w = torch.empty(M * 3, device="cuda")
    oV = torch.empty(M * 3 * tot * n, device="cuda")
    E = torch.empty((), dtype=torch.float64, device="cuda")

    def fn():
        D.demag_apply_tucker(P, rt, Vd, w, oV)
        D.demag_energy_tucker(P, rt, cd, Vd, w, oV, E)
    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    ms = time_region(fn, 10, stream)
    return {"value": 1e3 / ms, "unit": "energy evals/s", "ms_per_eval": ms, "energy": float(E.item()),
            "work": "Tucker application (3M terms) and the energy from factor Grams and core contractions; "
                    "the 1024^3 magnetization and potential are never formed"}


def run_tt_energy(D, P, n3, rr, tt_in, stream):
    """Demag energy of one rank-(8, 8) TT magnetization on the 1024^3 grid without forming a full
    tensor: demag_apply_tt + demag_energy_tt, CUDA events over 10 calls."""
    import torch
    n, M = n3[0], P.M
    G = [torch.from_numpy(x.ravel()).cuda() for x in tt_in]
    w = torch.empty(M * 3, device="cuda")
    o = [torch.empty(M * 3 * s, device="cuda") for s in (rr[0] * n, rr[0] * rr[1] * n, rr[1] * n)]
    E = torch.empty((), dtype=torch.float64, device="cuda")

    def fn():
        D.demag_apply_tt(P, rr, G[0], G[1], G[2], w, *o)
        D.demag_energy_tt(P, rr, G[0], G[1], G[2], w, *o, E)
    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    ms = time_region(fn, 10, stream)
    return {"value": 1e3 / ms, "unit": "energy evals/s", "ms_per_eval": ms, "energy": float(E.item()),
            "work": "TT application (3M trains) and the energy from the Grams of first, middle and last cores"}


def run_tt_round(D, P, n3, tol=1e-5, rr=(8, 8)):
    """TT rounding (App. C) of the potential of one smooth rank-(8, 8) TT magnetization on the
    1024^3 grid: the 3M output trains of demag_apply_tt rounded to one train with relative
    error <= tol (second call timed; host-driven and synchronous)."""
    import torch
    import synth
    n, M = n3[0], P.M
    G = [torch.from_numpy(x.ravel()).cuda() for x in synth.tt_smooth_inputs(n3, rr, 1700)]
    w = torch.empty(M * 3, device="cuda")
    o = [torch.empty(M * 3 * sz, device="cuda") for sz in (rr[0] * n, rr[0] * rr[1] * n, rr[1] * n)]
    D.demag_apply_tt(P, rr, G[0], G[1], G[2], w, *o)
    torch.cuda.synchronize()
    try:
        D.demag_round_tt(P, rr, w, *o, tol)
        t0 = time.perf_counter()
        rk, _, _, _, err = D.demag_round_tt(P, rr, w, *o, tol)
        secs = time.perf_counter() - t0
    except D.DemagError as e:
        return {"tol": tol, "unavailable": str(e)}
    return {"tol": tol, "input_ranks": list(rr), "ranks": list(rk), "error": err, "seconds": secs,
            "ranks_before": [3 * M * rr[0], 3 * M * rr[1]],
            "floats_before": 3 * M * (rr[0] * n + rr[0] * rr[1] * n + rr[1] * n) + 3 * M,
            "floats_after": rk[0] * n + rk[0] * rk[1] * n + rk[1] * n,
            "work": "randomized TT rounding in FP64: exact ||phi|| from the term Grams, Khatri-Rao sketches "
                    "of both unfoldings, TT-SVD truncation of the projected train, last core by projection"}


def run_tucker_compressed(args, D, world, local, stream, P, n3, rt, B, V, tw, tV, hbm, tol=1e-6):
    """Alg. 2 with HOOI-compressed kernels on the Tucker workload (same inputs as the uncompressed leg):
    setup time, ranks, batched application rate, and the error against the uncompressed result at
    sampled points of item 0."""
    import time
    import numpy as np
    import torch
    import synth
    n = n3[0]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    D.demag_compress_kernel(P, tol)
    setup_s = time.perf_counter() - t0
    rho = D.demag_compressed_ranks(P)
    cores = torch.cat([torch.from_numpy(synth.tucker_inputs(n3, rt, 1500 + b)[0].ravel()) for b in range(B)]).cuda()
    per_V = sum(3 * rho[p] * rt[p] * n for p in range(3))
    out_V = torch.empty(B * per_V, device="cuda")
    # output cores C^(q) (x) G^(q) kept implicit (they have prod_p rho_p r_p entries each)
    fn = lambda: D.demag_apply_tucker_compressed(P, B, rt, None, V, None, out_V)  # noqa: E731
    fn()
    for _ in range(args.warmup):
        fn()
    torch.cuda.synchronize()
    barrier(world)
    with ClockSampler(local) as clk:
        ms = time_region(fn, max(3, args.steps), stream)
    ms = max_over_ranks(ms, world)
    bytes_app = 4.0 * 3 * sum(rt) * n + 4.0 * per_V
    gbs = B * bytes_app / (ms * 1e-3) / 1e9
    # error against the uncompressed application at sampled points of item 0
    M = P.M
    w = tw[: M * 3].cpu().numpy().reshape(M, 3).astype(np.float64)
    oU = tV[: M * 3 * sum(rt) * n].cpu().numpy()
    ublk, off = [], 0
    for p in range(3):
        size = M * 3 * rt[p] * n
        ublk.append(oU[off:off + size].reshape(M, 3, rt[p], n).astype(np.float64))
        off += size
    cV = out_V[:per_V].cpu().numpy()
    cblk, off = [], 0
    for p in range(3):
        size = 3 * rho[p] * rt[p] * n
        cblk.append(cV[off:off + size].reshape(rho[p], 3, rt[p], n).astype(np.float64))
        off += size
    ccore = torch.empty(3 * rho[0] * rho[1] * rho[2], device="cuda")
    D.demag_copy_compressed(P, None, ccore)
    C = ccore.cpu().numpy().reshape(3, rho[2], rho[1], rho[0]).astype(np.float64)
    G = cores[: 3 * rt[0] * rt[1] * rt[2]].cpu().numpy().reshape(3, rt[2], rt[1], rt[0]).astype(np.float64)
    pts = np.random.default_rng(0).integers(0, n, size=(32, 3))
    num = den = 0.0
    for i1, i2, i3 in pts:
        # [[C (x) G; W]] at one point: W rows reshaped [rho_p, r_p] ((i, l) order)
        a = sum(np.einsum("cba,fed,ad,be,cf->", C[q], G[q], cblk[0][:, q, :, i1], cblk[1][:, q, :, i2],
                          cblk[2][:, q, :, i3]) for q in range(3))
        b = sum(w[k, q] * np.einsum("cba,a,b,c->", G[q], ublk[0][k, q, :, i1], ublk[1][k, q, :, i2],
                                    ublk[2][k, q, :, i3]) for k in range(M) for q in range(3))
        num += (a - b) ** 2
        den += b ** 2
    # Alg. 2's approximate summation of item 0's potential (tolerance 1e-5)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rk, _, _, rc_err = D.demag_recompress_tucker(P, rt, cores[: 3 * rt[0] * rt[1] * rt[2]], out_V[:per_V], 1e-5)
    torch.cuda.synchronize()
    rc_s = time.perf_counter() - t0
    recompressed = {"tol": 1e-5, "ranks": list(rk), "error_bound": rc_err, "seconds": rc_s,
                    "ranks_before": [3 * rho[p] * rt[p] for p in range(3)],
                    "floats_before": per_V + 3 * ncore_implicit(rho, rt),
                    "floats_after": rk[0] * rk[1] * rk[2] + sum(rk[p] * n for p in range(3))}
    return {"value": whole_job_rate(B, ms, world), "unit": "apps/s", "ms_per_batch": ms, "tol": tol,
            "ranks": list(rho), "M": M, "setup_s": setup_s, "recompressed_item0": recompressed,
            "work": "Alg. 2: kernels compressed once (device QR, HOSVD ranks, 4 HOOI sweeps); per application "
                    "Toeplitz FFT matvecs of the rho_p compressed generators; output cores C^(q) (x) G^(q) implicit",
            "rel_err_vs_uncompressed": (num / den) ** 0.5,
            "rel_err_sample": "phi at 32 random points of item 0 from both Tucker outputs",
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                         "algorithmic_bytes_per_app": bytes_app, "traffic": None},
            "clocks": clk.summary()}


def ncore_implicit(rho, rt):
    """Entries of one component's Kronecker core C^(q) (x) G^(q) if it were formed."""
    return rho[0] * rt[0] * rho[1] * rt[1] * rho[2] * rt[2]


def run_uneven_batch(args, D, world, local, stream, form):
    """64 full-format grids of mixed shape (cubes 32^3..192^3, 512x512x4 and
    256x64x8 films), R = 41, replayed as a CUDA graph of five launches (split;
    the fused mode-1 / mode-2 products of the grids with the fused schedule;
    one persistent launch over their mode-3 stages and the other grids'
    tensor-core stages; the films' thin last stages on CUDA cores; reduction);
    compared with one call per grid."""
    import numpy as np
    import torch
    import synth
    shapes = synth.uneven_batch_shapes(args.batch_grids, 1215)
    plans, ms, phis, ms_host, hs = [], [], [], [], []
    for i, sn in enumerate(shapes):
        sh = (1.0 / max(sn),) * 3
        P = D.demag_build_factors(sn, sh, 41)
        D.demag_reserve_workspace(P, form)
        mh = synth.random_unit_m(sn, 1216 + i)
        plans.append(P)
        ms_host.append(mh)
        hs.append(sh)
        ms.append(torch.from_numpy(mh).cuda())
        phis.append(torch.empty(sn[2], sn[1], sn[0], device="cuda"))
    M = plans[0].M
    flops = sum(2.0 * M * (a * b * c) * (3 * a + 3 * b + 2 * c) for a, b, c in shapes)

    def grid_bytes(a, b, c, fused):  # algorithmic DRAM bytes of one grid's BF16x3 mode products
        pp3 = max(1, 400 // (-(-c // 32) * 6))
        return 4.0 * a * b * c * (3 + (4 if fused else 10) * M) + 4.0 * (-(-2 * M // pp3)) * a * b * c
    sched = [D.demag_forward_schedule(P, form) for P in plans]
    batch_bytes = sum(grid_bytes(*sh, sc == 1) for sh, sc in zip(shapes, sched))
    G = D.demag_graph_create_batched(plans, ms, phis, form)
    graph_fn = lambda: G.launch(stream)  # noqa: E731
    seq_fn = lambda: [D.demag_apply_full(P, m, f, form) for P, m, f in zip(plans, ms, phis)]  # noqa: E731
    for _ in range(args.warmup):
        graph_fn()
        seq_fn()
    torch.cuda.synchronize()
    steps = max(3, args.steps)
    l0 = D.demag_launch_count(plans[0])
    barrier(world)
    with ClockSampler(local) as clk:
        ms_graph = time_region(graph_fn, steps, stream)
    launches = (D.demag_launch_count(plans[0]) - l0) // steps
    ms_seq = time_region(seq_fn, steps, stream)
    graph_fn()
    torch.cuda.synchronize()
    for P in plans:
        D.demag_sync_status(P)
    ms_graph = max_over_ranks(ms_graph, world)
    check = [0, next(i for i, s in enumerate(shapes) if s == (512, 512, 4))]
    return {"grids": len(shapes), "form": form, "value": world * len(shapes) * 1e3 / ms_graph,
            "unit": "grids/s", "ms_per_batch": ms_graph, "ms_per_batch_one_call_per_grid": ms_seq,
            "algorithmic_tflops": flops / (ms_graph * 1e-3) / 1e12, "algorithmic_flops_per_batch": flops,
            "hbm_achieved_gbs": batch_bytes / (ms_graph * 1e-3) / 1e9, "algorithmic_bytes_per_batch": batch_bytes,
            "cells": int(sum(a * b * c for a, b, c in shapes)),
            "shapes": {f"{a}x{b}x{c}": shapes.count((a, b, c)) for a, b, c in sorted(set(shapes))},
            "gpu_launches": int(launches), "graph_kernels": G.kernels, "clocks": clk.summary(),
            "fused_grids": int(sum(1 for sc in sched if sc == 1)),
            "_check": check, "_shapes": shapes, "_h": hs, "_m": ms_host, "_phi": phis}


def cpu_baseline(n3, h, R, m_host, budget_s):
    """The FP64 oracle on the host cores, on a bounded number of nodes (scaled)."""
    from oracle import full as ofull
    M = (R - 1) // 2
    t0 = time.perf_counter()
    done = 0
    while done < M and (time.perf_counter() - t0) < budget_s:
        ofull.apply_full(m_host, n3, h, R, nodes=[done])
        done += 1
    dt = time.perf_counter() - t0
    return {"value": (done / M) / dt, "unit": "apps/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"full format {n3[0]}^3, {done} of {M} nodes (all 3 components), scaled to one app; "
                      f"numpy float64 with its default BLAS threads"}


def run_reference(args, world, rank, local):
    """The FP64 CPU oracle as it stands, timed on bounded samples (rank 0 only)."""
    if rank != 0:
        return
    import synth
    from oracle import full as ofull
    n3, h, R = full_config(args.n)
    M = (R - 1) // 2
    m_host = synth.vortex_m(n3, 1213)
    step = lambda: ofull.apply_full(m_host, n3, h, R, nodes=[0])  # noqa: E731
    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    value = (1.0 / M) / dt
    # a step is the bounded sample (one node of M), timed as it runs; the rate
    # counts it as 1/M of an application
    out = {"metric": METRIC, "value": value, "unit": "apps/s", "impl": "reference", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "app_fraction_per_step": 1.0 / M,
           "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded vortex state)",
           "config": dict(bench_config(args, "fp64 CPU oracle", world), parallelism="host cores"),
           "cpu_baseline": {"value": value, "unit": "apps/s", "cores": os.cpu_count(), "kind": "oracle",
                            "sample": f"each step: 1 of {M} nodes of the {args.n}^3 full-format application "
                                      "(numpy float64, default BLAS threads), counted as 1/M app"},
           "e2e": {"value": value, "unit": "apps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


CPU_CONFIGS = ("c1_16", "c2_128", "c2_256", "c3_cp4096", "c4_tucker1024", "c4_tt1024", "c5_batch64")


def cpu_one(cfg):
    """One bounded oracle sample of configuration `cfg`: (apps per second, what was sampled)."""
    import numpy as np
    import synth
    from oracle import full as ofull, structured as ost

    def timed(fn):
        t0 = time.perf_counter()
        fn()
        return time.perf_counter() - t0

    if cfg in ("c1_16", "c2_128", "c2_256"):
        n = {"c1_16": 16, "c2_128": 128, "c2_256": 256}[cfg]
        n3, h, R = full_config(n)
        M = (R - 1) // 2
        m = synth.vortex_m(n3, 1213) if n > 16 else synth.random_unit_m(n3, 1212)
        done, t = 0, 0.0
        while done < M and t < 10.0:
            t += timed(lambda: ofull.apply_full(m, n3, h, R, nodes=[done]))
            done += 1
        return (done / M) / t, f"full format {n}^3, R = {R}: {done} of {M} nodes, counted as {done}/{M} app"
    if cfg == "c3_cp4096":
        n3, h, R, r = cp_config(4096)
        lam, U = synth.cp_inputs(n3, r, 1214)
        t = timed(lambda: ost.apply_cp(lam, U, n3, h, R))
        return 1.0 / t, "one CP application, n = 4096, rank 4, R = 61 (dense O(n^2) Toeplitz matvecs)"
    if cfg == "c4_tucker1024":
        n3, h = (1024,) * 3, (1 / 1024,) * 3
        core, V = synth.tucker_inputs(n3, (8, 8, 8), 1219)
        t = timed(lambda: ost.apply_tucker(core, V, n3, (8, 8, 8), h, 61))
        return 1.0 / t, "one Tucker application, n = 1024, ranks (8, 8, 8), R = 61"
    if cfg == "c4_tt1024":
        n3, h = (1024,) * 3, (1 / 1024,) * 3
        G1, G2, G3 = synth.tt_inputs(n3, (8, 8), 1220)
        t = timed(lambda: ost.apply_tt(G1, G2, G3, n3, (8, 8), h, 61))
        return 1.0 / t, "one TT application, n = 1024, TT ranks (8, 8), R = 61"
    if cfg == "c5_batch64":
        shapes = synth.uneven_batch_shapes(64, 1215)
        total = 0.0
        for sn in sorted(set(shapes)):
            h = (1.0 / max(sn),) * 3
            m = synth.random_unit_m(sn, 1216)
            # one node of each distinct shape, scaled by the node count and its multiplicity
            total += shapes.count(sn) * 20 * timed(lambda: ofull.apply_full(m, sn, h, 41, nodes=[0]))
        return 64.0 / total, ("64-grid batch: one of 20 nodes of each of its 13 distinct shapes, "
                              "scaled by 20 and by the shape's count; grids/s")
    raise ValueError(cfg)


def cpu_table():
    """Oracle throughput per configuration with 1 host thread and with all of them."""
    import platform
    ncpu = os.cpu_count() or 1
    model = platform.processor() or platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part", "hardware")):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    rows = {}
    for threads in (1, ncpu):
        env = dict(os.environ)
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
            env[k] = str(threads)
        for cfg in CPU_CONFIGS:
            r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-one", cfg], env=env,
                               capture_output=True, text=True)
            try:
                rec = json.loads(r.stdout.strip().splitlines()[-1])
            except (ValueError, IndexError):
                rec = {"error": (r.stderr or r.stdout)[-300:]}
            rows.setdefault(cfg, {})[f"threads_{threads}"] = rec
    print(json.dumps({"cpu_table": rows, "cores": ncpu, "cpu_model": model, "machine": platform.machine()}),
          flush=True)


def main():
    args = parse()
    if args.cpu_one:
        v, what = cpu_one(args.cpu_one)
        print(json.dumps({"value": v, "sample": what}), flush=True)
        return
    if args.cpu_table:
        cpu_table()
        return
    world, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, world, rank, local)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    try:
        run_ours(args, world, rank, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
