#!/usr/bin/env python
"""Benchmark of the exact-exchange hot path: pair Poisson solves per second.

Workload (one "step"): 96^3 box at h = 0.2 bohr (padded 192^3), 16 orthonormal
occupied orbitals on 12 random Gaussian centres and 32 trial functions (seed 0):
  exchange apply Vx[Phi] Psi      512 pair solves
  ACE build from Phi              136 unique pair solves (rho_ij = rho_ji) + FP64 Cholesky
  ACE apply to Psi                two skinny contractions
= 648 pair Poisson solves per step.  value = solves/s over all GPUs (weak scaling: every
rank solves its own problem of this shape, seeded by its rank, on its own GPU).

Also reported on the same JSON line: the end-to-end rate through the public API with
host copies, the FP64 plain form of the same step, FP32-vs-FP64 accuracy, the
roofline of the dominant kernel from CUDA events recorded by the library around every
launch in the timed region, SM clocks sampled during it, and the CPU oracle baseline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl rsx|reference]
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2405_01522_gb300 import inputs  # noqa: E402

NOCC, NPSI, EDGE, H = 16, 32, 96, 0.2
SOLVES_EXCHANGE = NOCC * NPSI
SOLVES_ACE = NOCC * (NOCC + 1) // 2
SOLVES_PER_STEP = SOLVES_EXCHANGE + SOLVES_ACE
WORKLOAD = ("exchange apply + ACE build + ACE apply, 96^3 box at h=0.2 bohr padded to 192^3, "
            "16 orthonormal orbitals on 12 Gaussian centres (exponents U[0.3,3]), 32 trial functions, "
            "seed 0: 512 + 136 pair Poisson solves per step")
METRIC = "pair Poisson solves/s"
UNIT = "solves/s"


def env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.proc = None
        self.path = None
        try:
            bus = torch.cuda.get_device_properties(device).pci_bus_id
        except Exception:
            bus = None
        self.sel = ["-i", bus] if bus else []

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"]
                + self.sel, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[4:8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i].lower().startswith("active")})
        return {"sm_mhz": float(np.median([r[0] for r in rows])), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------- workload
def make_inputs(seed=0, edge=EDGE):
    """The exchange workload of one rank.  Ranks solve independent problems of the same
    shape (seed = rank): the path shards by problem, with no data exchange between ranks."""
    s = inputs.batched_system(n=edge, h=H, nocc=NOCC, ncentres=12, alpha=(0.3, 3.0), radius=3.0,
                              npsi=NPSI, seed=seed)
    return s


def max_over_ranks(x, dist, device):
    """Largest value of x over all ranks (the slowest rank's time); x itself when single."""
    if dist is None:
        return x
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def aggregate_rate(world, units_per_step, steps, ms_max):
    """Whole-job rate: units every rank processed over the slowest rank's time."""
    return world * units_per_step * steps / (ms_max / 1e3)


# Real flops of the register DFTs as implemented (adds + multiplies, a fused multiply-add
# counting 2; odd primes by the symmetric split, 6/10/12/14/24 by Good-Thomas, 8/16 by
# radix 2/4; a rotation by +-i is a swap, no flops).  tests/test_flop_model.py counts the
# codelets' operations on the host and checks these figures and the pruned forms below.
DFT_FLOPS = {1: 0, 2: 4, 3: 18, 4: 16, 5: 52, 6: 48, 7: 102, 8: 60, 10: 124, 12: 120, 14: 232, 16: 176,
             24: 3 * 60 + 8 * 18}
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12     # SMs x FP32 lanes x FMA x max SM clock

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) from ncu captures of the same
# kernels: pass 2 on the full 512-pair launch at 96^3 (a one-pass metric set), per line
# split and CTA size (8 lanes x 2A at 256 threads: 3.669 + 3.602 GB); the SYRK on a small
# case scaled by the panel bytes it reads
PASS2_DRAM_BYTES_PER_PAIR_96 = {(8, 256): 7.271e9 / 512}
SYRK_DRAM_PER_PANEL_BYTE = 1.938e9 / 1.850e9    # DRAM bytes per byte of the two bf16 panels


def _modinv(a, m):
    return next(i for i in range(1, m + 1) if (a * i) % m == 1 % m)


_PFA = {6: (2, 3), 10: (2, 5), 12: (3, 4), 14: (2, 7), 24: (3, 8)}


def _pfa_maps(A):
    P, Q = _PFA[A]
    qinv, pinv = _modinv(Q % P, P), _modinv(P % Q, Q)
    return P, Q, (lambda n1, n2: (Q * n1 + P * n2) % A), (lambda k1, k2: (Q * qinv * k1 + P * pinv * k2) % A)


def _small_in(m):
    """P-point DFT (P = 2, 3) with the inputs flagged False zero (all outputs formed)."""
    n = sum(m)
    if len(m) == 2:
        return 4 if n == 2 else 0
    return DFT_FLOPS[3] if n == 3 else 12 if n == 2 else (0 if m[0] else 8)


def _small_out(w):
    """P-point DFT (P = 2, 3) forming only the outputs flagged True."""
    n = sum(w)
    if len(w) == 2:
        return 4 if n == 2 else 2 * n
    if n == 0:
        return 0
    return 4 if (w[0] and n == 1) else 10 + 2 * n


def _half_in(A):
    """A-point DFT whose inputs A/2 .. A are zero."""
    if A % 2:
        return DFT_FLOPS[A]
    if A in _PFA:   # zero-skipping P-point DFTs, then P complete Q-point DFTs
        P, Q, fin, _ = _pfa_maps(A)
        return sum(_small_in([fin(n1, n2) < A // 2 for n1 in range(P)]) for n2 in range(Q)) + P * DFT_FLOPS[Q]
    return 2 * DFT_FLOPS[A // 2] + max(A // 2 - 2, 0) * 6   # radix 2, the rotation by i free


def _half_out(A):
    """A-point DFT of which outputs 0 .. A/2 are formed."""
    if A % 2:
        return DFT_FLOPS[A]
    if A in _PFA:   # P complete Q-point DFTs, then P-point DFTs forming the kept outputs
        P, Q, _, fout = _pfa_maps(A)
        return P * DFT_FLOPS[Q] + sum(_small_out([fout(k1, k2) < A // 2 for k1 in range(P)]) for k2 in range(Q))
    if A == 16:     # radix 4, second 4-point DFTs forming two outputs each
        return 4 * 16 + 8 * 6 + 4 * 12
    return 2 * DFT_FLOPS[A // 2] + max(A // 2 - 2, 0) * 6 + A


def line_flops(A, kind):
    """Flops of one line of length 16 A: two register stages + twiddles (6 per cmul)."""
    tw = 16 * (A - 1) * 6
    if kind == "fwd_pruned":        # forward, inputs beyond n are zero
        return 16 * _half_in(A) + tw + A * DFT_FLOPS[16]
    if kind == "inv_keep_half":     # inverse, only outputs below n kept (stage 2 pruned)
        return 16 * DFT_FLOPS[A] + tw + A * (_half_out(16) if A % 2 == 0 else DFT_FLOPS[16])
    if kind == "z_inverse":         # inverse z after the multiply (stage-1 outputs pruned);
        # even A: twiddles after the transpose, 16 lanes x (A - 1); odd A: A lanes x 16
        ztw = 16 * (A - 1) * 6 if A % 2 == 0 else A * 16 * 6
        return A * DFT_FLOPS[16] + ztw + 16 * (_half_out(A) if A % 2 == 0 else DFT_FLOPS[A])
    raise ValueError(kind)


def line_flops_l8(A, kind):
    """Flops of one line of length 16 A split 8 lanes x 2A: 2A-point DFTs (pruned halves)
    on 8 lanes, 8 x (2A - 1) twiddles, 2A 8-point DFTs."""
    tw = 8 * (2 * A - 1) * 6
    if kind == "fwd_pruned":
        return 8 * _half_in(2 * A) + tw + 2 * A * DFT_FLOPS[8]
    if kind in ("inv_keep_half", "z_inverse"):
        return 2 * A * DFT_FLOPS[8] + tw + 8 * _half_out(2 * A)
    raise ValueError(kind)


def algorithmic_flops(kernel, shape, nq, npsi_out, lanes=16):
    """Implemented FP32 flops of one launch over nq pairs (npsi_out outputs for pass 3);
    lanes: the line split of pass 2 (16 x A or 8 x 2A)."""
    nz, ny, nx = shape
    Ax, Ay, Az = nx // 8, ny // 8, nz // 8
    Hx = nx + 1
    if kernel == "pass2_yz_kernel":
        Ly = 16 * Ay
        lf = line_flops_l8 if lanes == 8 else line_flops
        plane = (nz * lf(Ay, "fwd_pruned")
                 + Ly * (lf(Az, "fwd_pruned") + 2 * 16 * Az + lf(Az, "z_inverse"))
                 + nz * lf(Ay, "inv_keep_half"))
        return nq * Hx * plane
    if kernel == "pass1_x_forward":
        return nq * nz * (ny // 2) * (line_flops(Ax, "fwd_pruned") + 8 * Hx)
    if kernel == "pass3_x_inverse_accumulate":
        return nq * nz * (ny // 2) * (line_flops(Ax, "inv_keep_half") + 2 * 16 * Ax + 4 * nx)
    return None


def algorithmic_bytes(kernel, shape, nq, nocc, npsi, elem=4):
    """Compulsory HBM bytes of one launch over nq pairs: each pair's x-transformed
    intermediate ((Mx/2 + 1) x nz x ny complex, M = 2n) is written once by pass 1, read and
    written once by pass 2 and read once by pass 3; passes 1 and 3 also read (and pass 3
    writes) the orbitals, pass 2 reads the (M/2 + 1)^3 kernel table once."""
    nz, ny, nx = shape
    N = nz * ny * nx
    inter = (nx + 1) * nz * ny * 2 * elem          # (Mx/2 + 1) * nz * ny complex per pair
    table = (nx + 1) * (ny + 1) * (nz + 1) * elem   # kernel table (M/2 + 1)^3
    if kernel == "pass1_x_forward":
        return nq * inter + (nocc + npsi) * N * elem
    if kernel == "pass2_yz_kernel":
        return 2 * nq * inter + table
    if kernel == "pass3_x_inverse_accumulate":
        return nq * inter + (nocc + npsi) * N * elem
    return None


def run_rsx(args, rank, local_rank, world):
    from paper_2405_01522_gb300 import rsx
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    s = make_inputs(seed=rank)
    shape = s.shape
    ctx = rsx.Context(shape, H, "fp32", device=local_rank)
    phi = torch.from_numpy(s.phi).float().to(dev)
    psi = torch.from_numpy(s.psi).float().to(dev)
    vx = torch.empty_like(psi)
    xi = torch.empty_like(phi)
    va = torch.empty_like(psi)
    stream = torch.cuda.current_stream()

    def step():
        ctx.exchange_apply(phi, psi, out=vx)
        ctx.ace_build(phi, xi=xi)
        ctx.ace_apply(xi, psi, out=va)

    tuning = ctx.autotune(NOCC, NPSI) if not args.no_tune else None   # outside the timed region
    for _ in range(args.warmup):
        step()
    ctx.sync()

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- timed region (device-resident inputs)
    clocks = ClockSampler(local_rank)
    ctx.profile_reset()
    ctx.profile(True)
    clocks.start()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    ctx.profile(False)
    ctx.sync()
    ms = e0.elapsed_time(e1)
    prof = ctx.profile_read()
    ms_max = max_over_ranks(ms, dist, dev)
    ms_step = ms_max / args.steps
    value = aggregate_rate(world, SOLVES_PER_STEP, args.steps, ms_max)

    # ---- per-kernel shares and the dominant kernel's roofline
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    total_kernel_ms = sum(v[0] for v in prof.values())
    kernels = {k: {"ms_per_launch": v[0] / v[1], "launches": v[1], "share": v[0] / total_kernel_ms}
               for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0])}
    launches = sum(v[1] for v in prof.values())
    # pair counts per launch of each pass in one step: exchange (512 pairs) and ACE (136)
    per_launch_pairs = {"pass1_x_forward": [SOLVES_EXCHANGE, SOLVES_ACE],
                        "pass2_yz_kernel": [SOLVES_EXCHANGE, SOLVES_ACE],
                        "pass3_x_inverse_accumulate": [SOLVES_EXCHANGE, SOLVES_ACE]}
    top = next(iter(kernels))
    roof = None
    if top in per_launch_pairs:
        # the FFT passes are instruction-issue / FP32 bound (ncu: DRAM ~7%, issue ~60%):
        # report the ALU roofline, with the HBM view alongside
        byts = [algorithmic_bytes(top, shape, nq, NOCC, NPSI if nq == SOLVES_EXCHANGE else 0)
                for nq in per_launch_pairs[top]]
        lanes = (tuning or {}).get("p2_lanes", 8 if os.environ.get("RSX_PASS2_LANES") == "8" else 16)
        p2_threads = (tuning or {}).get("p2_threads", int(os.environ.get("RSX_PASS2_THREADS", "256")))
        flops = [algorithmic_flops(top, shape, nq, 0, lanes) for nq in per_launch_pairs[top]]
        avg_bytes = sum(byts) / len(byts)
        avg_flops = sum(flops) / len(flops)
        avg_ms = kernels[top]["ms_per_launch"]
        ach_f = avg_flops / (avg_ms / 1e3) / 1e12
        ach_b = avg_bytes / (avg_ms / 1e3) / 1e9
        traffic = None
        per_pair = PASS2_DRAM_BYTES_PER_PAIR_96.get((lanes, p2_threads))
        if top == "pass2_yz_kernel" and tuple(shape) == (96, 96, 96) and per_pair:
            traffic = per_pair * sum(per_launch_pairs[top]) / len(per_launch_pairs[top])
        split = "8 lanes x 2A" if lanes == 8 else "16 lanes x A"
        roof = {"kernel": f"{top} ({split}, {p2_threads} threads)", "bound": "alu", "achieved": round(ach_f, 2),
                "peak": round(FP32_PEAK_TFLOPS, 2),
                "unit": "TFLOP/s", "frac": round(ach_f / FP32_PEAK_TFLOPS, 4), "traffic": traffic,
                "traffic_source": (f"ncu DRAM bytes of the 512-pair launch ({per_pair / 1e6:.1f} MB per pair) times "
                                   "the average pairs per launch") if traffic else
                                  "none: no capture of this kernel build yet",
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 (FMA) x 2.07 GHz",
                "algorithmic_flops_per_launch": avg_flops,
                "hbm_view": {"achieved_gbs": round(ach_b, 1), "peak_gbs": hbm_peak, "frac": round(ach_b / hbm_peak, 4),
                             "peak_source": peak_src, "algorithmic_bytes_per_launch": avg_bytes}}

    # ---- end to end through the public API: pinned host inputs -> device -> results -> host.
    # Two buffer sets: step i computes on one set while the inputs of step i + 1 are copied
    # in (copy stream) and the results of step i - 1 are copied out (second copy stream).
    phi_h = torch.from_numpy(s.phi).float().pin_memory()
    psi_h = torch.from_numpy(s.psi).float().pin_memory()
    h2d_s, d2h_s = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    sets = [dict(phi=torch.empty_like(phi), psi=torch.empty_like(psi), vx=torch.empty_like(psi),
                 xi=torch.empty_like(phi), va=torch.empty_like(psi),
                 vx_h=torch.empty(vx.shape, dtype=torch.float32).pin_memory(),
                 va_h=torch.empty(va.shape, dtype=torch.float32).pin_memory(),
                 h2d=torch.cuda.Event(), done=torch.cuda.Event(), d2h=torch.cuda.Event()) for _ in range(2)]

    def h2d(i):
        b = sets[i % 2]
        with torch.cuda.stream(h2d_s):
            if i >= 2:
                h2d_s.wait_event(sets[i % 2]["d2h"])      # step i - 2 has released this set
            b["phi"].copy_(phi_h, non_blocking=True)
            b["psi"].copy_(psi_h, non_blocking=True)
            b["h2d"].record(h2d_s)

    def e2e_run(nsteps, start_ev=None, end_ev=None):
        if start_ev is not None:
            start_ev.record(h2d_s)
        h2d(0)
        for i in range(nsteps):
            b = sets[i % 2]
            if i + 1 < nsteps:
                h2d(i + 1)
            stream.wait_event(b["h2d"])
            ctx.exchange_apply(b["phi"], b["psi"], out=b["vx"], stream=stream)
            ctx.ace_build(b["phi"], xi=b["xi"], stream=stream)
            ctx.ace_apply(b["xi"], b["psi"], out=b["va"], stream=stream)
            b["done"].record(stream)
            with torch.cuda.stream(d2h_s):
                d2h_s.wait_event(b["done"])
                b["vx_h"].copy_(b["vx"], non_blocking=True)
                b["va_h"].copy_(b["va"], non_blocking=True)
                b["d2h"].record(d2h_s)
        if end_ev is not None:
            stream.wait_event(sets[(nsteps - 1) % 2]["d2h"])   # the copy-out stream is in order
            end_ev.record(stream)

    e2e_run(2)
    barrier()
    e2 = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ne2e = max(3, args.steps)   # as many steps as the device-resident timing
    e2e_run(ne2e, e2[0], e2[1])
    barrier()
    ms_e2e = max_over_ranks(e2[0].elapsed_time(e2[1]), dist, dev)
    e2e = {"value": aggregate_rate(world, SOLVES_PER_STEP, ne2e, ms_e2e), "unit": UNIT,
           "h2d_bytes_per_step": phi_h.numel() * 4 + psi_h.numel() * 4,
           "d2h_bytes_per_step": sets[0]["vx_h"].numel() * 4 + sets[0]["va_h"].numel() * 4, "steps": ne2e,
           "pipelining": "inputs of step i+1 copied in and results of step i-1 copied out while step i computes"}

    # ---- ACE build time alone (FP32)
    ctx.sync()
    ea = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ea[0].record(stream)
    for _ in range(5):
        ctx.ace_build(phi, xi=xi)
    ea[1].record(stream)
    torch.cuda.synchronize()
    ace_ms = ea[0].elapsed_time(ea[1]) / 5

    # ---- the Gram kernel alone per ACE shape (launch profiler: kernel time only)
    gram_us = {}
    for label, (ga, gb) in (("16x16 <phi, W>", (phi, xi)), ("16x32 <xi, psi>", (xi, psi))):
        ctx.sync()
        ctx.profile_reset()
        ctx.profile(True)
        for _ in range(10):
            ctx.gram(ga, gb)
        ctx.profile(False)
        ctx.sync()
        g = ctx.profile_read().get("gram")
        gram_us[label] = round(g[0] / g[1] * 1e3, 1) if g else None

    # step-level HBM view against the per-solve byte model of a plane-pass design (orbital
    # rows read in the first and last pass, the 2x-padded-in-y intermediate written and read
    # twice: 3.54 + 4 x 14.30 + 3.54 MB at 96^3); this design moves fewer bytes per solve
    nz_, ny_, nx_ = shape
    model_bytes = 2 * nz_ * ny_ * nx_ * 4 + 4 * (nx_ + 1) * nz_ * (2 * ny_) * 8
    model_gbs = value * model_bytes / 1e9
    step_model = {"bytes_per_solve": model_bytes, "effective_gbs": round(model_gbs, 1),
                  "frac_of_measured_hbm": round(model_gbs / hbm_peak, 4),
                  "what": "solves/s x the per-solve HBM bytes of a plane-pass design (orbital rows read twice, "
                          "four passes over a (Mx/2 + 1) x nz x 2 ny complex intermediate)"}
    logical = SOLVES_EXCHANGE + NOCC * NOCC   # the ACE build's rho_ij and rho_ji counted separately
    out = {"metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(ms_step, 4), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": bench_config(shape, world),
           "tuning": tuning, "roofline": roof, "kernels": kernels, "gpu_launches": launches, "clocks": clk, "e2e": e2e,
           "ace_build_ms": round(ace_ms, 4), "gram_kernel_us": gram_us, "step_model_hbm": step_model,
           "solves_logical": {"per_step": logical, "per_s": round(value * logical / SOLVES_PER_STEP, 1),
                              "what": "the ACE build's 16 x 16 pair potentials counted as 256 (136 unique)"}}

    # ---- FP64 plain form of the same step, and FP32 accuracy against it
    if not args.skip_fp64 and rank == 0:
        ctx64 = rsx.Context(shape, H, "fp64", device=local_rank)
        phi64 = torch.from_numpy(s.phi).to(dev)
        psi64 = torch.from_numpy(s.psi).to(dev)
        vx64 = torch.empty_like(psi64)
        xi64 = torch.empty_like(phi64)
        va64 = torch.empty_like(psi64)

        def step64():
            ctx64.exchange_apply(phi64, psi64, out=vx64)
            ctx64.ace_build(phi64, xi=xi64)
            ctx64.ace_apply(xi64, psi64, out=va64)

        step64()
        ctx64.sync()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        step64()
        f1.record(stream)
        torch.cuda.synchronize()
        ms64 = f0.elapsed_time(f1)
        step()
        ctx.sync()
        h3 = H ** 3
        e32 = (psi.double() * vx.double()).sum(dim=(1, 2, 3)) * h3
        e64 = (psi64 * vx64).sum(dim=(1, 2, 3)) * h3
        ex32 = 0.5 * h3 * (phi.double() * ctx.exchange_apply(phi, phi).double()).sum().item()
        ex64 = 0.5 * h3 * (phi64 * ctx64.exchange_apply(phi64, phi64)).sum().item()
        out["fp64_plain"] = {"value": round(SOLVES_PER_STEP / (ms64 / 1e3), 1), "unit": UNIT,
                             "ms_per_step": round(ms64, 3), "speedup_fp32_over_fp64": round(ms64 / ms_step, 2)}
        out["accuracy"] = {
            "ref": "FP64 GPU path (parity-tested against the FP64 CPU oracle to 1e-11)",
            "vx_energy_rel_err_max": float(((e32 - e64).abs() / e64.abs()).max()),
            "exchange_energy_rel_err": abs(ex32 - ex64) / abs(ex64),
            "vx_rel_max_err": float((vx.double() - vx64).abs().max() / vx64.abs().max()),
            "ace_apply_rel_max_err": float((va.double() - va64).abs().max() / va64.abs().max()),
            "tolerance_energy": 1e-6}
        ctx64.close()

    # ---- Casida coupling (config with 512 transitions), rank 0
    if rank == 0 and not args.skip_casida:
        out["casida"] = casida_bench(args, dev, local_rank, peaks)

    # ---- uneven molecule batch, rank 0
    if rank == 0 and not args.skip_batch:
        out["batch"] = batch_bench(args, dev, local_rank, peaks)

    # ---- learned eigensolver preconditioner, rank 0
    if rank == 0 and not args.skip_precond:
        out["learned_precond"] = precond_bench(args, dev, local_rank)

    # ---- plain eigensolver step and HF SCF time per iteration with and without ACE, rank 0
    if rank == 0 and not args.skip_scf:
        out["eigensolver"] = eig_bench(args, dev)
        out["scf"] = scf_bench(args, dev)

    # ---- CPU oracle baseline (rank 0, N = 1 only)
    if rank == 0 and world == 1 and not args.skip_cpu:
        out["cpu_baseline"] = cpu_baseline(s, nsolve=args.cpu_solves)

    if rank == 0:
        print(json.dumps(out), flush=True)
    ctx.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def casida_bench(args, dev, local_rank, peaks):
    """Casida coupling K (80^3 at 0.25 bohr, 8 occupied + 64 virtual, 512 transitions):
    split-BF16 tensor-core K vs the FP64 plain form, TDA roots, tensor roofline of the
    K contraction kernel."""
    from paper_2405_01522_gb300 import rsx
    s = inputs.casida_system(n=args.casida_edge, h=0.25, nocc=8, nvirt=64)
    nt = 8 * 64
    ng = 2 * (s.shape[2] + 1) * (2 * s.shape[1]) * (2 * s.shape[0])
    c32 = rsx.Context(s.shape, s.h, "fp32", device=local_rank)
    po = torch.from_numpy(s.phi).float().to(dev)
    pv = torch.from_numpy(s.phi_virt).float().to(dev)
    K = torch.empty((nt, nt), dtype=torch.float64, device=dev)
    eo = torch.from_numpy(s.eps_occ).to(dev)
    ev = torch.from_numpy(s.eps_virt).to(dev)
    c32.casida_K(po, pv, K=K)
    c32.sync()
    reps = 3
    c32.profile_reset()
    c32.profile(True)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    e[0].record()
    for _ in range(reps):
        c32.casida_K(po, pv, K=K)
    e[1].record()
    torch.cuda.synchronize()
    c32.profile(False)
    prof = c32.profile_read()
    k_ms = e[0].elapsed_time(e[1]) / reps
    gemm_ms = prof["k_gemm_tcgen05"][0] / prof["k_gemm_tcgen05"][1]
    useful = 2.0 * nt * nt * ng                      # one product, full nt x nt
    method = 3 * nt * (nt + 1) * ng                  # three split products of the SYRK half (upper triangle)
    nbk = (nt + 127) // 128
    executed = 3 * (nbk * (nbk + 1) // 2) * 2.0 * 128 * 128 * ng   # three products, upper-triangle tiles
    peak = peaks.get("bf16_tflops", 1900.0)
    es = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    es[0].record()
    w32 = c32.casida_solve(eo, ev, K, None, 1.0, 10)
    es[1].record()
    torch.cuda.synchronize()
    solve_ms = es[0].elapsed_time(es[1])
    # absorption spectrum of the lowest 10 roots (Eqs. 8-10) and the full TDHF roots (Eqs. 3-5)
    w32v, X32 = c32.casida_solve(eo, ev, K, None, 1.0, 10, vectors=True)
    # untimed first calls: position table, full-TDHF workspace, first-launch module loading
    f0 = c32.oscillator_strengths(w32v, X32, c32.casida_dipoles(po, pv))
    c32.strength_function(w32v, f0, 0.001, torch.zeros(8, dtype=torch.float64, device=dev))
    c32.casida_solve_full(eo, ev, K, None, 1.0, 10)
    torch.cuda.synchronize()
    grid = torch.linspace(0.0, 1.0, 4001, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    ef = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ef[0].record()
    dip = c32.casida_dipoles(po, pv)
    f32 = c32.oscillator_strengths(w32v, X32, dip)
    S = c32.strength_function(w32v, f32, 0.0136 / 27.211386245988, grid)
    ef[1].record()
    ef[2].record()
    wfull = c32.casida_solve_full(eo, ev, K, None, 1.0, 10)
    ef[3].record()
    torch.cuda.synchronize()
    spectrum_ms = ef[0].elapsed_time(ef[1])
    full_ms = ef[2].elapsed_time(ef[3])
    # spin-polarised form: alpha 8 occupied + 64 virtual, beta the first 7 occupied + the
    # same virtuals (one electron removed), 960 transitions in one panel
    nta, ntb = 8 * 64, 7 * 64
    Ku = torch.empty((nta + ntb, nta + ntb), dtype=torch.float64, device=dev)
    pob = po[:7].contiguous()
    c32.casida_K_uhf(po, pv, pob, pv, K=Ku)
    Kda, Kdb = c32.casida_Kd(po, pv), c32.casida_Kd(pob, pv)
    c32.casida_solve_uhf(eo, ev, eo[:7].contiguous(), ev, Ku, Kda, Kdb, nroots=10)
    torch.cuda.synchronize()
    eu = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    eu[0].record()
    c32.casida_K_uhf(po, pv, pob, pv, K=Ku)
    eu[1].record()
    eu[2].record()
    wu = c32.casida_solve_uhf(eo, ev, eo[:7].contiguous(), ev, Ku, Kda, Kdb, nroots=10)
    eu[3].record()
    torch.cuda.synchronize()
    nbu = (nta + ntb + 127) // 128
    exec_u = 3 * (nbu * (nbu + 1) // 2) * 2.0 * 128 * 128 * ng
    uhf = {"what": "spin-polarised TDA (Eqs. 4-5): alpha 8 occ + 64 virt, beta 7 occ + 64 virt, 960 transitions; "
                   "K over both spins from one split-BF16 panel, A = diag + K - blockdiag(K_d), lowest 10 roots",
           "K_ms": round(eu[0].elapsed_time(eu[1]), 3), "eigensolve_ms": round(eu[2].elapsed_time(eu[3]), 3),
           "executed_tflop": round(exec_u / 1e12, 3),
           "omega_ev": [round(float(x) * 27.211386245988, 6) for x in wu]}
    out = {"workload": "TDA coupling K, 80^3 box at h=0.25 bohr padded to 160^3, 8 occupied + 64 virtual "
                       "orthonormal Gaussian-sum orbitals, 512 transitions, K via split-BF16 tcgen05 "
                       "(hi.hi + hi.lo + lo.hi), lowest 10 roots of diag(de) + K",
           "casida_K_ms": round(k_ms, 3), "gemm_ms": round(gemm_ms, 3), "eigensolve_ms": round(solve_ms, 3),
           "spectrum": {"ms": round(spectrum_ms, 3), "what": "dipoles <i|r|a>, oscillator strengths f_k (Eq. 9) of "
                        "the 10 TDA roots, Lorentzian strength function (half-width 0.0136 eV) on 4001 points",
                        "f": [round(float(x), 6) for x in f32], "S_max": round(float(S.max()), 3)},
           "full_tdhf": {"ms": round(full_ms, 3), "omega_ev": [round(float(x) * 27.211386245988, 6) for x in wfull],
                         "what": "A and B (Eqs. 3-5), half-size form by FP64 Cholesky, lowest 10 roots"},
           "uhf": uhf,
           "useful_tflops": round(useful / (gemm_ms / 1e3) / 1e12, 1),
           "method_work": {"what": "3 split products of the SYRK half, 3 nt (nt + 1) N_G flops",
                           "tflops": round(method / (gemm_ms / 1e3) / 1e12, 1),
                           "frac_of_peak": round(method / (gemm_ms / 1e3) / 1e12 / peaks.get("bf16_tflops", 1900.0), 4)},
           "kernels": {k: {"ms_per_launch": round(v[0] / v[1], 4), "launches": v[1]} for k, v in prof.items()},
           "roofline": {"kernel": "k_syrk_bf16x3 (tcgen05)", "bound": "tensor",
                        "achieved": round(executed / (gemm_ms / 1e3) / 1e12, 1), "peak": peak, "unit": "TFLOP/s",
                        "frac": round(executed / (gemm_ms / 1e3) / 1e12 / peak, 4),
                        "traffic": SYRK_DRAM_PER_PANEL_BYTE * 2 * 2 * ((nt + 127) // 128 * 128) * ((ng + 63) // 64 * 64),
                        "traffic_source": "ncu DRAM bytes per panel byte at 48^3 x 512 times the two bf16 panels here",
                        "peak_source": "measured" if "bf16_tflops" in peaks else "fallback",
                        "algorithmic_flops_per_launch": executed}}
    if not args.skip_fp64:
        c64 = rsx.Context(s.shape, s.h, "fp64", device=local_rank)
        K64 = c64.casida_K(po.double(), pv.double())
        c64.sync()
        f = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        f[0].record()
        c64.casida_K(po.double(), pv.double(), K=K64)
        f[1].record()
        torch.cuda.synchronize()
        w64 = c64.casida_solve(eo, ev, K64, None, 1.0, 10)
        c64.sync()
        out["fp64_plain_K_ms"] = round(f[0].elapsed_time(f[1]), 2)
        out["omega_err_ev_max"] = float((w32 - w64).abs().max()) * 27.211386245988
        out["omega_ev"] = [round(float(x) * 27.211386245988, 6) for x in w64]
        out["tolerance_ev"] = 1e-5
        c64.close()
    c32.close()
    return out


def batch_bench(args, dev, local_rank, peaks):
    """Uneven batch: 64 molecules, edges from {48,64,80,96,112}, N_occ ~ U{2..24}, h 0.2;
    exchange apply (psi = phi) + ACE build of every molecule in persistent launches
    replayed from a CUDA graph."""
    from paper_2405_01522_gb300 import rsx
    desc = inputs.uneven_batch(nmol=args.batch_mols)
    t0 = time.perf_counter()
    mols = [inputs.batched_system(n=e, h=0.2, nocc=k, npsi=0, seed=sd) for e, k, sd in desc]
    gen_s = time.perf_counter() - t0
    b = rsx.Batch([e for e, _, _ in desc], [k for _, k, _ in desc], 0.2, device=local_rank)
    phi = [torch.from_numpy(m.phi).float().to(dev) for m in mols]
    W = [torch.empty_like(p) for p in phi]
    xi = [torch.empty_like(p) for p in phi]
    b.bind(phi, W, xi)
    b.run()
    b.sync()
    reps = 3
    e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    e[0].record()
    for _ in range(reps):
        b.run()
    e[1].record()
    torch.cuda.synchronize()
    ms = e[0].elapsed_time(e[1]) / reps
    solves = sum(k * (k + 1) // 2 for _, k, _ in desc)
    # algorithmic bytes of the three passes (intermediates written once, read/written by
    # pass 2, read by pass 3; orbitals read, W written)
    byts = 0
    for ed, k, _ in desc:
        inter = (ed + 1) * ed * ed * 8
        npairs = k * (k + 1) // 2
        byts += 4 * npairs * inter + 3 * k * ed ** 3 * 4
    hbm = peaks.get("hbm_gbs", 6800.0)
    ach = byts / (ms / 1e3) / 1e9
    b.close()
    return {"workload": f"{len(desc)} molecules, edges from {{48,64,80,96,112}}, N_occ U{{2..24}}, h=0.2: "
                        "exchange apply (psi = phi) + ACE build each; per box edge one launch of each FFT pass over "
                        "all that edge's pairs, ACE per molecule, one CUDA graph",
            "solves_per_batch": solves, "ms_per_batch": round(ms, 3), "solves_per_s": round(solves / (ms / 1e3), 1),
            "hbm_model_gbs": round(ach, 1), "hbm_frac": round(ach / hbm, 4), "input_generation_s": round(gen_s, 1)}


def precond_bench(args, dev, local_rank):
    """Learned eigensolver preconditioner on 96^3 systems with 16 bands (h 0.2, 4 model
    atoms): training pairs from plain-solver runs on several systems, Adam training on the
    GPU, then iterations and wall time to |dE| < 1e-6 Ha on an unseen system, plain vs
    plain + learned directions."""
    from paper_2405_01522_gb300 import precond, rsx
    n, h, nb = args.precond_edge, 0.2, 16
    t_all = time.perf_counter()
    pots = [inputs.model_potential(n=n, h=h, natoms=4, Z=4.0, rc=0.6, radius=2.5, seed=s) for s in (11, 12, 13, 14, 21)]
    Vs = [torch.from_numpy(v).float().to(dev) for v in pots]
    vscale = float(1.0 / max(float(v.abs().max()) for v in Vs))
    psi0s = [torch.from_numpy(inputs.starting_orbitals(n=n, h=h, nband=nb, radius=2.5, seed=100 + s)).float().to(dev)
             for s in range(5)]
    Xs, Ys = [], []
    target = args.precond_pairs
    plain_iters = []
    for i in range(4):
        res = precond.solve(Vs[i], h, psi0s[i], nb, tol=1e-6, vscale=vscale, record_every=2, max_iter=600)
        plain_iters.append(res["iters"])
        per = max(1, target // (4 * max(1, len(res["records"])) * nb))
        X, Y = precond.make_pairs(Vs[i], h, res, vscale, crop=32, crops_per_sample=per, seed=i)
        Xs.append(X)
        Ys.append(Y)
        del res
    X = torch.cat(Xs)[:target].contiguous()
    Y = torch.cat(Ys)[:target].contiguous()
    del Xs, Ys
    net = rsx.Net(precond.init_params(seed=0), device=local_rank)
    t0 = time.perf_counter()
    losses = precond.train(net, X, Y, epochs=args.precond_epochs, batch=32, lr=1e-3, border=3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    # conv throughput: one training step and one full-grid forward
    xb, yb = X[:32].contiguous(), Y[:32].contiguous()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    e[0].record()
    for _ in range(5):
        net.train_step(xb, yb, 1e-12, border=3)
    e[1].record()
    xf = torch.zeros((nb, 2, n, n, n), dtype=torch.float32, device=dev)
    net.forward(xf)
    e[2].record()
    for _ in range(3):
        net.forward(xf)
    e[3].record()
    torch.cuda.synchronize()
    step_ms = e[0].elapsed_time(e[1]) / 5
    fwd_ms = e[2].elapsed_time(e[3]) / 3
    flop_vox = 2 * 27 * (2 * 16 + 16 * 16 + 16 * 1)
    fwd_tflops = flop_vox * nb * n ** 3 / (fwd_ms / 1e3) / 1e12
    train_tflops = 3 * flop_vox * 32 * 32 ** 3 / (step_ms / 1e3) / 1e12
    del X, Y, xf
    # evaluation on an unseen system, every energy evaluated in FP64 after each step
    # (rsx_eig_energy64, outside the timed solver steps): the reference is an independent
    # plain run converged to |dE| < 1e-10 Ha; then the iterations and solver time each
    # method needs to come (and stay) within 1e-6 Ha of it
    ref = precond.solve(Vs[4], h, psi0s[4], nb, tol=1e-10, vscale=vscale, max_iter=3000, energy64=True)
    plain = precond.solve(Vs[4], h, psi0s[4], nb, tol=1e-9, vscale=vscale, max_iter=1500, energy64=True)
    learned = precond.solve(Vs[4], h, psi0s[4], nb, net=net, tol=1e-9, vscale=vscale, max_iter=1500,
                            energy64=True)
    net.close()
    e_ref = ref["energy"]
    ip, tp = precond.time_to_target(plain, e_ref)
    il, tl = precond.time_to_target(learned, e_ref)
    ip5, tp5 = precond.time_to_target(plain, e_ref, tol=1e-5)
    il5, tl5 = precond.time_to_target(learned, e_ref, tol=1e-5)
    return {"workload": f"{n}^3 box at h=0.2, 16 bands of H = -1/2 Lap(FD4) + V (4 model atoms, Z=4); "
                        "training pairs from plain runs on 4 systems, evaluation on a 5th",
            "pairs": int(target), "epochs": args.precond_epochs, "loss_first_last": [losses[0], losses[-1]],
            "train_s": round(train_s, 2), "plain_train_iters": plain_iters,
            "reference_energy_ha": e_ref, "reference_iters": ref["iters"],
            "target": "|E - E_ref| < 1e-6 Ha (and 1e-5 Ha) from that iteration on; E the FP64 block energy, "
                      "E_ref an independent plain run to |dE| < 1e-10 Ha",
            "plain": {"iters_to_target": ip, "time_to_target_s": None if tp is None else round(tp, 3),
                      "iters_to_1e-5": ip5, "time_to_1e-5_s": None if tp5 is None else round(tp5, 3),
                      "final_energy_ha": plain["energy"], "min_energy_ha": min(plain["trace"]),
                      "iters": plain["iters"], "s_per_iter": round(plain["time_s"] / plain["iters"], 5)},
            "learned": {"iters_to_target": il, "time_to_target_s": None if tl is None else round(tl, 3),
                        "iters_to_1e-5": il5, "time_to_1e-5_s": None if tl5 is None else round(tl5, 3),
                        "final_energy_ha": learned["energy"], "min_energy_ha": min(learned["trace"]),
                        "iters": learned["iters"], "s_per_iter": round(learned["time_s"] / learned["iters"], 5),
                        "fell_back_at": learned["fell_back_at"]},
            "final_energy_diff_ha": abs(learned["energy"] - plain["energy"]),
            "conv_forward_tflops": round(fwd_tflops, 2), "conv_train_step_tflops": round(train_tflops, 2),
            "total_s": round(time.perf_counter() - t_all, 1)}


def eig_bench(args, dev, warm=4, steps=10):
    """Plain block eigensolver step (LOBPCG with the kinetic-energy preconditioner) on a 96^3
    box at h = 0.2 with 16 bands of -1/2 Lap(FD4) + V (8 model atoms, Z = 4): time per step
    and the per-kernel split of one step."""
    from paper_2405_01522_gb300 import rsx
    n, h, nb = args.scf_edge, 0.2, 16
    v = torch.from_numpy(inputs.model_potential(n=n, h=h, natoms=8, Z=4.0, rc=0.6, radius=3.0, seed=41)).float().to(dev)
    psi0 = torch.from_numpy(inputs.starting_orbitals(n=n, h=h, nband=nb, radius=3.0, seed=42)).float().to(dev)
    es = rsx.Eigensolver(v, h, nb, device=dev.index or 0)
    es.init(psi0)
    for _ in range(warm):
        es.step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        th = es.step()
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) / steps * 1e3
    es.close()
    # the same in a spherical domain (Sec. 3.4) of radius 0.45 n h around the box centre
    ax = (torch.arange(n, device=dev, dtype=torch.float32) - n / 2) * h
    r2 = ax[:, None, None] ** 2 + ax[None, :, None] ** 2 + ax[None, None, :] ** 2
    mask = (r2 <= (0.45 * n * h) ** 2).float().contiguous()
    es = rsx.Eigensolver(v, h, nb, device=dev.index or 0)
    es.set_mask(mask)
    es.init(psi0)
    for _ in range(warm):
        es.step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        ths = es.step()
    torch.cuda.synchronize()
    ms_s = (time.perf_counter() - t0) / steps * 1e3
    es.close()
    return {"workload": f"{n}^3 box at h=0.2, 16 bands, LOBPCG [Psi | W | P] with 3 damped-Jacobi sweeps of "
                        "(K + T)^-1, one-CTA FP64 Rayleigh-Ritz", "ms_per_step": round(ms, 3),
            "energy_ha": float(sum(th)), "steps_timed": steps,
            "sphere": {"radius_bohr": round(0.45 * n * h, 3), "points": int(mask.sum().item()),
                       "ms_per_step": round(ms_s, 3), "energy_ha": float(sum(ths))}}


def scf_bench(args, dev, iters=10, inner=2, max_iter=300):
    """Closed-shell HF SCF on a 96^3 box at h = 0.2 with 16 doubly occupied orbitals (16 model
    atoms, Z = 4, r_c = 0.35, in a 5.5-bohr ball): wall time per SCF iteration over the first `iters` iterations with the
    exact exchange in every Fock application and with ACE (Sec. 3.1 compares the two the
    same way), both from the same start; then ACE cycles run towards a relative density
    error (Eq. 15) below 1e-6 with density mixing and with state mixing (Sec. 3.2)."""
    from paper_2405_01522_gb300 import rsx
    n, h, nocc = args.scf_edge, 0.2, 16
    v = torch.from_numpy(inputs.model_potential(n=n, h=h, natoms=16, Z=4.0, rc=0.35, radius=5.5, seed=43)).float().to(dev)
    psi0 = torch.from_numpy(inputs.starting_orbitals(n=n, h=h, nband=nocc, radius=5.5, seed=42)).float().to(dev)
    ctx = rsx.Context((n, n, n), h, "fp32", device=dev.index or 0)
    res = {}
    for name, ace in (("exact", False), ("ace", True)):
        scf = rsx.SCF(ctx, v, nocc, ace=ace, alpha=0.3)
        scf.init(psi0)
        scf.step(inner=inner)                       # first iteration: module loading, workspace growth
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hist = [scf.step(inner=inner) for _ in range(iters)]
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / iters
        res[name] = {"s_per_iteration": round(dt, 5), "energy_after_ha": hist[-1]["energy"],
                     "reldens_after": hist[-1]["reldens"], "exchange_ha": hist[-1]["exchange"]}
        scf.close()
    res["speedup_ace"] = round(res["exact"]["s_per_iteration"] / res["ace"]["s_per_iteration"], 2)
    for mix in ("density", "states"):
        scf = rsx.SCF(ctx, v, nocc, ace=True, alpha=0.3, mix=mix)
        scf.init(psi0)
        t0 = time.perf_counter()
        hist, first = [], {}
        while len(hist) < max_iter:
            hist.append(scf.step(inner=inner))
            r = hist[-1]["reldens"]
            for tol in (1e-4, 1e-5, 1e-6):
                if len(hist) > 1 and r < tol and tol not in first:
                    first[tol] = len(hist)
            if len(hist) > 1 and r < 1e-6:
                break
        last = hist[-1]
        res[f"ace_{mix}_mixing"] = {
            "iterations": len(hist), "iterations_to": {f"{t:g}": first.get(t) for t in (1e-4, 1e-5, 1e-6)},
            "reldens": last["reldens"], "energy_ha": last["energy"], "one_body_ha": last["one_body"],
            "hartree_ha": last["hartree"], "exchange_ha": last["exchange"], "s": round(time.perf_counter() - t0, 3)}
        scf.close()
    ctx.close()
    res["workload"] = (f"{n}^3 box at h=0.2, 16 occupied orbitals (16 model atoms, Z=4, r_c=0.35, 5.5-bohr ball), "
                       f"mixing parameter 0.3, "
                       f"{inner} block eigensolver steps per SCF iteration; time per iteration averaged over "
                       f"iterations 2..{iters + 1}; convergence runs capped at {max_iter} iterations")
    return res


# ----------------------------------------------------------------------------- CPU oracle
# The oracle as it stands, timed on the host cores: its exchange loop runs unchanged in
# each worker process, the pairs of a sample are split across the workers by output
# function (all orbitals j for one psi_p, or a slice of them), and the inputs are shared
# with the workers through shared memory.  Workers are started with "spawn" so that no
# process forks after the CUDA context exists.
_POOL_ARRAYS = {}


def _pool_init(specs):
    from multiprocessing import shared_memory
    import oracle  # noqa: F401  (imported once per worker, outside the timed region)
    for name, (shm_name, shape) in specs.items():
        shm = shared_memory.SharedMemory(name=shm_name)
        _POOL_ARRAYS[name] = (shm, np.ndarray(shape, dtype=np.float64, buffer=shm.buf))


def _pool_task(task):
    """Vx[phi_j0..j1] psi_p by the oracle (its own loop over j), returned as FP64."""
    import oracle
    p, j0, j1, h = task
    phi = _POOL_ARRAYS["phi"][1]
    psi = _POOL_ARRAYS["psi"][1]
    return oracle.exchange_apply(phi[j0:j1], psi[p:p + 1], h)


def _pool_ready(_):
    return os.getpid()


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class OraclePool:
    """A spawn-started process pool with the step's inputs in shared memory."""

    def __init__(self, s, workers):
        import multiprocessing as mp
        from multiprocessing import shared_memory
        self.workers = workers
        self.h = s.h
        self.shm = []
        specs = {}
        for name, arr in (("phi", s.phi), ("psi", s.psi)):
            a = np.ascontiguousarray(arr, dtype=np.float64)
            shm = shared_memory.SharedMemory(create=True, size=a.nbytes)
            np.ndarray(a.shape, dtype=np.float64, buffer=shm.buf)[...] = a
            self.shm.append(shm)
            specs[name] = (shm.name, a.shape)
        self.pool = mp.get_context("spawn").Pool(workers, initializer=_pool_init, initargs=(specs,))
        self.pool.map(_pool_ready, range(workers), chunksize=1)     # every worker started

    def run(self, tasks):
        return self.pool.map(_pool_task, [t + (self.h,) for t in tasks], chunksize=1)

    def close(self):
        self.pool.close()
        self.pool.join()
        for shm in self.shm:
            shm.close()
            shm.unlink()


def cpu_baseline(s, nsolve=16, npsi_all=None):
    """The FP64 oracle as it stands, on the host: (1) the whole exchange apply of the step
    (Vx on every trial function from all orbitals, NOCC x NPSI pair solves) split by output
    function over one worker per host core; (2) the same oracle on one core for `nsolve`
    solves, for comparison."""
    import oracle
    cores = host_cores()
    npsi_all = s.psi.shape[0] if npsi_all is None else npsi_all
    t0 = time.perf_counter()
    oracle.exchange_apply(s.phi[:nsolve], s.psi[:1], s.h)
    dt1 = time.perf_counter() - t0
    pool = OraclePool(s, cores)
    try:
        nj = s.phi.shape[0]
        split = max(1, min(nj, -(-cores // npsi_all)))         # at least one task per core
        bounds = [nj * c // split for c in range(split + 1)]
        tasks = [(p, bounds[c], bounds[c + 1]) for p in range(npsi_all) for c in range(split)]
        t0 = time.perf_counter()
        out = pool.run(tasks)
        dt = time.perf_counter() - t0
    finally:
        pool.close()
    nsolves = s.phi.shape[0] * npsi_all
    assert len(out) == len(tasks)
    return {"value": round(nsolves / dt, 3), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"the step's exchange apply: Vx on all {npsi_all} trial functions from all "
                      f"{s.phi.shape[0]} orbitals ({nsolves} pair solves) of the 96^3 workload, numpy "
                      f"pocketfft FP64, split by trial function over {cores} spawn-started worker processes "
                      f"(one per host core); {dt:.1f} s",
            "single_core": {"value": round(nsolve / dt1, 3), "cores": 1,
                            "sample": f"{nsolve} pair solves (Vx on trial 0 from orbitals 0..{nsolve - 1}) in this "
                                      f"process; {dt1:.1f} s"}}


def bench_config(shape, world):
    """The `config` object of both arms (the same workload, the same keys)."""
    return {"workload": WORKLOAD, "grid": list(shape), "padded": [2 * x for x in shape], "h_bohr": H,
            "nocc": NOCC, "npsi": NPSI, "solves_per_step": SOLVES_PER_STEP,
            "l2": "no flush: inputs (170 MB) and FFT intermediates (3.7 GB) exceed the 129 MB L2",
            "parallelism": f"independent problems x{world} (seed = rank)"}


def run_reference(args, rank, world):
    """The oracle as the reference arm: same metric, workload and config; each step is a
    bounded sample of the step's pair solves, one per host core, run in parallel."""
    if rank != 0:
        return
    s = make_inputs()
    cores = host_cores()
    pool = OraclePool(s, cores)

    def tasks(k):
        # pair solves (j, p) of the exchange apply, in order, `cores` per step
        out = []
        for u in range(cores):
            q = (k * cores + u) % (NOCC * NPSI)
            p, j = divmod(q, NOCC)
            out.append((p, j, j + 1))
        return out

    try:
        for k in range(args.warmup):
            pool.run(tasks(k))
        t0 = time.perf_counter()
        for k in range(args.steps):
            pool.run(tasks(args.warmup + k))
        dt = time.perf_counter() - t0
    finally:
        pool.close()
    value = cores * args.steps / dt
    out = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(1e3 * dt / args.steps, 2), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": bench_config(s.shape, world),
           "impl": "reference",
           "cpu_baseline": {"value": round(value, 3), "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"{cores} pair solves of the step's exchange apply per step, one per "
                                      f"spawn-started worker process (one per host core), FP64 numpy oracle"},
           "e2e": {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="rsx", choices=["rsx", "reference"])
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--cpu-solves", type=int, default=16)
    ap.add_argument("--skip-casida", action="store_true")
    ap.add_argument("--skip-batch", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (default knobs)")
    ap.add_argument("--skip-precond", action="store_true")
    ap.add_argument("--skip-scf", action="store_true")
    ap.add_argument("--eig-only", action="store_true", help="only the plain eigensolver step (profiling captures)")
    ap.add_argument("--scf-only", action="store_true", help="only the SCF section")
    ap.add_argument("--scf-edge", type=int, default=96)
    ap.add_argument("--precond-only", action="store_true")
    ap.add_argument("--precond-edge", type=int, default=96)
    ap.add_argument("--precond-pairs", type=int, default=20000)
    ap.add_argument("--precond-epochs", type=int, default=4)
    ap.add_argument("--batch-mols", type=int, default=64)
    ap.add_argument("--casida-only", action="store_true", help="only the Casida section (profiling captures)")
    ap.add_argument("--batch-only", action="store_true", help="only the uneven-batch section (profiling captures)")
    ap.add_argument("--casida-edge", type=int, default=80, help="box edge of the Casida case")
    ap.add_argument("--nocc", type=int, default=16, help="smaller cases for profiling captures only")
    ap.add_argument("--npsi", type=int, default=32, help="smaller cases for profiling captures only")
    args = ap.parse_args()
    global NOCC, NPSI, SOLVES_EXCHANGE, SOLVES_ACE, SOLVES_PER_STEP
    NOCC, NPSI = args.nocc, args.npsi
    SOLVES_EXCHANGE = NOCC * NPSI
    SOLVES_ACE = NOCC * (NOCC + 1) // 2
    SOLVES_PER_STEP = SOLVES_EXCHANGE + SOLVES_ACE
    if args.warmup < 3:
        args.warmup = 3
    rank, local_rank, world = env_rank()
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.precond_only:
        dev = torch.device("cuda", local_rank)
        torch.cuda.set_device(dev)
        print(json.dumps({"learned_precond": precond_bench(args, dev, local_rank)}), flush=True)
    elif args.eig_only:
        dev = torch.device("cuda", local_rank)
        torch.cuda.set_device(dev)
        print(json.dumps({"eigensolver": eig_bench(args, dev)}), flush=True)
    elif args.scf_only:
        dev = torch.device("cuda", local_rank)
        torch.cuda.set_device(dev)
        print(json.dumps({"scf": scf_bench(args, dev)}), flush=True)
    elif args.batch_only:
        dev = torch.device("cuda", local_rank)
        torch.cuda.set_device(dev)
        peaks = {}
        try:
            peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        except Exception:
            pass
        print(json.dumps({"batch": batch_bench(args, dev, local_rank, peaks)}), flush=True)
    elif args.casida_only:
        dev = torch.device("cuda", local_rank)
        torch.cuda.set_device(dev)
        peaks = {}
        try:
            peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        except Exception:
            pass
        print(json.dumps({"casida": casida_bench(args, dev, local_rank, peaks)}), flush=True)
    else:
        run_rsx(args, rank, local_rank, world)


if __name__ == "__main__":
    main()
