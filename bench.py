#!/usr/bin/env python3
"""Benchmark of the GB300 ionising-MD hot path.

One step = one full timestep of the method on the whole sample: kick/drift,
stochastic charge update and free-electron reduction, cell-list rebuild
(when the Verlet-buffered list is used up), screened pair forces.  The
default workload is the largest single-GPU one: the 2,000,000-atom water
droplet (vacuum) irradiated by an 8 keV, 20 fs, 1e13 ph/um^2 pulse, 800
steps of 50 as from -1 FWHM.  The timed window of K steps sits at the middle
of that run, on the pulse peak: the state is advanced there by untimed steps
and checkpointed, and every timed arm (mixed, FP64, end-to-end) restores the
checkpoint, runs W warm-up steps and times K.  Mixed precision: FP32 pairs
with 64-bit fixed-point sums, FP64 integrator and charge update.

Prints ONE JSON line (rank 0).  Multi-GPU (torchrun): every rank runs an
independent replica of the workload (weak scaling, no collective on the data
path; the barrier and the max-over-ranks timing use torch.distributed).

--impl reference runs the FP64 CPU oracle on the host cores instead (the
reference arm for this build; a deliberately slow, obviously correct program).
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "atom-steps/s (pair forces + ionisation) on 1 GB300, mixed vs FP64 at stated error"
UNIT = "atom-steps/s"
FLOPS_PER_PAIR = 41          # FP32 operations per in-cutoff pair in the pair kernel (FMA = 2)
L2_FLUSH_BYTES = 256 << 20   # > 129 MB L2
SKIN_NM = 0.12               # Verlet buffer of the pair list (measured: best at the pulse peak of the droplet and the water box)
SKIN_MODE = "fixed"          # "adaptive": the device drops the buffer while lists live under 4 steps


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--steps-per-launch", type=int, default=1,
                    help="steps per timed md_step_async call (the L2 is flushed between calls); "
                         "md_step runs eight steps per graph launch")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="c5_droplet_2m")
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--fp64-steps", type=int, default=30)
    ap.add_argument("--window", default="centre", choices=["centre", "start"],
                    help="where the timed steps sit in the configured run: its middle (the pulse peak; "
                         "reached by untimed steps) or its first steps")
    ap.add_argument("--no-peaks", action="store_true", help="skip the FMA-pipe peak measurement")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--profile-case", action="store_true",
                    help="minimal run for ncu: default launch shape, W + K steps, no baselines")
    ap.add_argument("--profile-resume", action="store_true",
                    help="with --profile-case and --skin > 0: end with a checkpoint round trip, whose "
                         "last force launch runs outside the step graph over the trimmed list")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--screening", default="debye", choices=["debye", "hybrid"],
                    help="Coulomb screening: Debye (Eq. 2) or hybrid ion sphere / Debye (Eqs. 4-7)")
    ap.add_argument("--langevin", type=float, default=0.0,
                    help="electron-ion coupling g (nm^3/ps) of every species, Eqs. 13-14; 0: off")
    ap.add_argument("--charge-table", action="store_true",
                    help="charges from per-step CR charge-state fractions (a synthetic table) instead of the rates")
    ap.add_argument("--bonded", action="store_true",
                    help="add the Morse bonds and harmonic angles of the water/methane molecules (Eqs. 9-10)")
    ap.add_argument("--probe", action="store_true",
                    help="record the per-species charge and displacement series of Eq. 17 every step")
    ap.add_argument("--skin", type=float, default=SKIN_NM,
                    help="Verlet buffer of the cluster-pair list (nm); 0 rebuilds every step")
    ap.add_argument("--skin-mode", default=SKIN_MODE, choices=["fixed", "adaptive"],
                    help="adaptive: unbuffered lists while buffered ones live fewer than 4 steps")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# inputs
# ---------------------------------------------------------------------------
def make_workload(name, scale, rank):
    from paper_2401_03180_gb300 import workloads as W
    wl = W.workload(name, scale=scale)
    if rank:   # an independent replica per rank: its own RNG key
        wl.sample.seed[:] = wl.sample.seed + np.uint64(7919 * rank)
    atom = W.atomic_data(wl.photon_kev)
    return wl, atom


def max_over_ranks(ms, dist, device):
    """The slowest rank's time: the job is done when its last rank is."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, n_atoms, steps, ms):
    """Whole-job atom-steps/s: each of the `world` ranks advances its own
    replica of n_atoms atoms by `steps` steps in `ms` milliseconds."""
    return world * n_atoms * steps / (ms / 1e3)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        rows = [l.strip().split(", ") for l in open(self.path) if l.strip()]
        os.unlink(self.path)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1])); smax.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].strip().lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "samples": len(sm),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def kernel_source_digest():
    src = os.path.join(ROOT, "paper_2401_03180_gb300", "csrc", "k_pair.cu")
    return hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]


def profiled_traffic(workload):
    """DRAM bytes per pair-kernel launch of this workload from the committed
    ncu summary, if the kernel source is unchanged since the capture."""
    path = os.path.join(ROOT, "profiles", f"k_pair_{workload}.md") if workload else None
    if not path or not os.path.exists(path):
        return None, None
    txt = open(path).read()
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    h = re.search(r"k_pair_source_sha256_16:\s*([0-9a-f]+)", txt)
    if not m or not h or h.group(1) != kernel_source_digest():
        return None, (h.group(1) if h else None)
    return float(m.group(1)), h.group(1)


def step_calls(k_steps, per_call):
    """Sizes of the timed md_step calls: k_steps in calls of per_call steps,
    the last one shorter when per_call does not divide k_steps."""
    n = max(1, int(per_call))
    return [min(n, k_steps - k) for k in range(0, k_steps, n)]


def sms_count(torch):
    return torch.cuda.get_device_properties(0).multi_processor_count


def fp32_peak_tflops(torch):
    """FP32 peak from unit counts: SMs x 128 FP32 lanes x 2 x the maximum SM clock."""
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    max_mhz = 2070.0
    try:
        mp = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        max_mhz = float(mp.get("sm_max_mhz", max_mhz))
    except Exception:
        pass
    return sms * 128 * 2 * max_mhz * 1e6 / 1e12, sms, max_mhz


def measured_fma_peaks(M, local):
    """FP32 and FP64 FMA-pipe throughput of this device (md_fma_peak, an FMA
    counted as two operations), in TFLOP/s: burst = best of three ~50 ms
    launches; sustained = one ~1 s launch, with the SM clocks sampled during it."""
    out = {}
    for name, prec in (("fp32", M.MD_PREC_MIXED), ("fp64", M.MD_PREC_FP64)):
        M.md_fma_peak(prec, 64)                              # load the kernel
        f, sec = M.md_fma_peak(prec, 256)
        it50 = max(int(256 * 0.05 / max(sec, 1e-6)), 1)      # ~50 ms per launch
        burst = max(M.md_fma_peak(prec, it50)[0] for _ in range(3))
        with ClockSampler(local) as clk:
            sus, sec_s = M.md_fma_peak(prec, it50 * 20)
        out[name] = {"burst_tflops": burst / 1e12, "sustained_tflops": sus / 1e12,
                     "sustained_s": sec_s, "clocks_sustained": clk.summary()}
    return out


CKPT_KEYS = ("x", "v", "q", "h", "n_e", "e_gas_mev", "event_counts", "x_list")


def window_start(n_steps, steps, warmup, where):
    """Untimed steps before the warm-up: the timed window then sits at the
    middle of the configured run (the pulse peak of every workload)."""
    if where == "start":
        return 0
    return max(0, (n_steps - steps) // 2 - warmup)


def run_gpu(args, rank, world, local):
    import torch
    from paper_2401_03180_gb300 import build as B
    from paper_2401_03180_gb300 import md as M
    from paper_2401_03180_gb300 import workloads as W

    B.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    wl, atom = make_workload(args.workload, args.scale, rank)
    if args.bonded:
        wl.sample = W.with_topology(wl.sample)
    s = wl.sample
    n_atoms = s.n_atoms
    W_, K = args.warmup, args.steps
    s0 = window_start(wl.n_steps, K, W_, args.window)
    max_steps = max(wl.n_steps, s0 + W_ + K + 1)
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    peaks = None if args.no_peaks else measured_fma_peaks(M, local)

    def make(prec, profile, autotune=None):
        g = M.IonisingMD(s, atom, precision=prec, r_cut=1.2, dt_ps=5e-5, max_steps=max_steps,
                         t_start_fs=wl.t_start_fs, autotune=(prec == "mixed") if autotune is None else autotune,
                         profile=profile, list_skin_nm=args.skin, screening=args.screening,
                         list_skin_adaptive=args.skin_mode == "adaptive",
                         langevin_g=args.langevin if args.langevin > 0 else None,
                         charge_mode="table" if args.charge_table else "rates", probe_record=args.probe)
        for r in range(s.n_replicas):
            g.set_pulse(wl.pulses[r], replica=r)
            if args.charge_table:
                g.set_charge_table(W.charge_fraction_table(wl.pulses[r], wl.t_start_fs, 5e-5 * 1000.0, max_steps + 1),
                                   replica=r)
        return g

    # ---- untimed advance to the window, one checkpoint for every arm ----
    ckpt = None
    if s0 > 0:
        g0 = make("mixed", profile=False, autotune=False)
        g0.step(s0)
        ckpt = g0.get_state(M.MD_FIELD_ALL)
        g0.close()

    def start(prec, profile):
        g = make(prec, profile)
        if ckpt is not None:
            g.set_state(M.MD_FIELD_ALL, **{k: ckpt[k] for k in CKPT_KEYS}, step=ckpt["step"])
        return g

    def timed_steps(g, k_steps):
        # steps are enqueued without a host round trip (their status is read
        # once at the end), so the events bracket the device work of each call
        # of steps_per_launch steps
        calls = step_calls(k_steps, args.steps_per_launch)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in calls]
        for k, n in enumerate(calls):
            flush.zero_()                       # evict the 129 MB L2 between calls
            ev[k][0].record(stream)
            g.step(n, wait=False)
            ev[k][1].record(stream)
        g.sync()
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev)

    # ---- mixed path, device-timed: the step graph without event nodes ----
    g = start("mixed", profile=False)
    for _ in range(W_):
        g.step(1)
    _, _, pairs0 = g.energies()
    g.reset_timing()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ms = timed_steps(g, K)
    torch.cuda.synchronize()
    ms = max_over_ranks(ms, dist, "cuda")
    tim = g.timing()
    _, _, pairs1 = g.energies()
    state = g.get_state(M.MD_FIELD_PLASMA | M.MD_FIELD_COUNTS | M.MD_FIELD_Q | M.MD_FIELD_X | M.MD_FIELD_F)
    g.close()
    # the force kernel's own time: the same steps again, with event nodes around
    # it in the step graph (they add inter-kernel gaps, so they stay out of `value`)
    gp = start("mixed", profile=True)
    for _ in range(W_):
        gp.step(1)
    gp.reset_timing()
    timed_steps(gp, K)
    ptim = gp.timing()
    gp.close()
    pair_ms = ptim.pair_ms / max(ptim.pair_launches, 1)
    pairs = 0.5 * (pairs0 + pairs1)
    value = job_throughput(world, n_atoms, K, ms)
    peak_units, sms, max_mhz = fp32_peak_tflops(torch)
    if peaks is not None:
        peak = peaks["fp32"]["burst_tflops"]
        peak_basis = (f"measured: FP32 FMA-pipe throughput of this GB300 (md_fma_peak, best of three ~50 ms "
                      f"launches); {peaks['fp32']['sustained_tflops']:.1f} TFLOP/s sustained over "
                      f"{peaks['fp32']['sustained_s']:.1f} s; {peak_units:.1f} from unit counts at {max_mhz:.0f} MHz")
    else:
        peak = peak_units
        peak_basis = f"{sms} SMs x 128 FP32 lanes x 2 x {max_mhz:.0f} MHz (max SM clock)"
    achieved = FLOPS_PER_PAIR * pairs / (pair_ms / 1e3) / 1e12
    traffic, _ = profiled_traffic(args.workload if args.scale == 1.0 else None)

    # ---- FP64 path on the same inputs and window ----
    k64 = min(args.fp64_steps, K)
    g64 = start("fp64", profile=False)
    for _ in range(W_):
        g64.step(1)
    ms64 = timed_steps(g64, k64)
    state64 = g64.get_state(M.MD_FIELD_PLASMA | M.MD_FIELD_Q | M.MD_FIELD_X | M.MD_FIELD_F)
    g64.close()
    value64 = world * n_atoms * k64 / (ms64 / 1e3)
    # the FP64 force kernel's own time: a short run with event nodes around it
    g64p = start("fp64", profile=True)
    for _ in range(W_):
        g64p.step(1)
    g64p.reset_timing()
    timed_steps(g64p, min(k64, 10))
    t64 = g64p.timing()
    g64p.close()
    pair_ms64 = t64.pair_ms / max(t64.pair_launches, 1)
    if peaks is not None:
        peak64 = peaks["fp64"]["burst_tflops"]
        peak64_basis = "measured: FP64 FMA-pipe throughput of this GB300 (md_fma_peak, best of three ~50 ms launches)"
    else:
        peak64 = sms * 2 * 2 * max_mhz * 1e6 / 1e12   # 2 FP64 lanes per SM, FMA = 2
        peak64_basis = ("SMs x 2 FP64 lanes x 2 x max SM clock (GB300 issues FP64 at 2 lanes per SM per clock)")
    achieved64 = FLOPS_PER_PAIR * pairs / (pair_ms64 / 1e3) / 1e12

    # ---- end to end through the C ABI, host buffers ----
    e2e = None
    if not args.no_e2e:
        from paper_2401_03180_gb300 import md as M2
        ge = start("mixed", profile=False)
        # each replica's own pulse train, streamed one step at a time
        dF_tab = np.stack([M2.md_pulse_table([p for p in wl.pulses[r]], wl.t_start_fs, 5e-5 * 1000.0, max_steps)
                           for r in range(s.n_replicas)])
        h_in = torch.empty(s.n_replicas, dtype=torch.float64, pin_memory=True).numpy()
        h_q = torch.empty(n_atoms, dtype=torch.uint8, pin_memory=True).numpy()
        outs = {"q": h_q, "n_e": np.empty(s.n_replicas, np.int64), "e_gas_mev": np.empty(s.n_replicas, np.int64),
                "te_ev": np.empty(s.n_replicas), "kappa": np.empty(s.n_replicas)}
        for _ in range(W_):
            ge.step(1)
        tot = 0.0
        for k in range(K):
            flush.zero_()
            torch.cuda.synchronize()
            step = s0 + W_ + k
            h_in[:] = dF_tab[:, step]
            t0 = time.perf_counter()
            M2.md_set_fluence_at(ge.h, step, h_in)                  # H2D: this step's fluence, per replica
            ge.step(1, wait=False)                                   # the step's graph, enqueued
            ge.get_state(M2.MD_FIELD_Q | M2.MD_FIELD_PLASMA, out=outs)  # D2H: charges + plasma + status
            tot += time.perf_counter() - t0
        ge.close()
        e2e = {"value": world * n_atoms * K / tot, "unit": UNIT,
               "h2d_bytes_per_step": int(8 * s.n_replicas),
               # charges, each replica's 104-byte state record, the 4-byte error flags
               "d2h_bytes_per_step": int(n_atoms + 104 * s.n_replicas + 4)}

    dt_fs = 5e-5 * 1000.0
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W_,
        "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+i64 pairs, f64 integrator/charge update",
        "data": "synthetic (seeded generators; no paper sample or atomic data available)",
        "config": {"workload": args.workload if args.scale == 1.0 else f"{args.workload}@{args.scale}",
                   "n_atoms": n_atoms, "replicas_per_gpu": s.n_replicas,
                   "box_nm": float(s.box[0, 0]) if s.box[0, 0] > 0 else None, "r_cut_nm": 1.2, "dt_as": 50,
                   "pulse": [vars(p) for p in wl.pulses[0]], "t_start_fs": wl.t_start_fs,
                   "configured_steps": wl.n_steps,
                   "timed_window": {"first_step": s0 + W_, "t_fs": [wl.t_start_fs + (s0 + W_) * dt_fs,
                                                                     wl.t_start_fs + (s0 + W_ + K) * dt_fs],
                                    "untimed_steps_before": s0, "placement": args.window},
                   "l2": ("flushed between steps (256 MB write, untimed)" if args.steps_per_launch <= 1 else
                          f"flushed between calls of {args.steps_per_launch} steps (256 MB write, untimed)"),
                   "steps_per_launch": max(1, args.steps_per_launch),
                   "pair_tile": {"warps": tim.tile_warps, "blocks_per_sm": tim.tile_blocks_per_sm},
                   "build_shape": {"sort_threads": tim.sort_threads, "list_blocks_per_sm": tim.list_blocks_per_sm,
                                   "kernels_per_build": tim.build_kernels},
                   "list_skin_nm": args.skin, "list_skin_mode": args.skin_mode, "screening": args.screening,
                   "langevin_g": args.langevin,
                   "charges": "table" if args.charge_table else "rates",
                   "bonded": ({"bonds": int(len(s.topology.bonds)), "angles": int(len(s.topology.angles))}
                              if s.topology is not None else None),
                   "probe_record": bool(args.probe),
                   "parallelism": f"replicas{world}"},
        "pair_interactions_per_s": world * pairs * K / (ms / 1e3),
        "pairs_per_step": pairs,
        "fp64_gpu": {"value": value64, "unit": UNIT, "steps": k64, "ms_per_step": ms64 / k64,
                     "speedup_mixed_vs_fp64": value / value64,
                     "roofline": {"bound": "fp64", "kernel": "k_pair (FP64 path)", "achieved": achieved64,
                                  "peak": peak64, "unit": "TFLOP/s", "frac": achieved64 / peak64,
                                  "peak_basis": peak64_basis, "pair_kernel_ms": pair_ms64}},
        "roofline": {"bound": "alu", "kernel": "k_pair (FP32 FMA pipe)", "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                     "peak_basis": peak_basis, "frac_of_unit_count_peak": achieved / peak_units,
                     "flops_per_pair": FLOPS_PER_PAIR, "pair_kernel_ms": pair_ms,
                     "pair_kernel_share": pair_ms / (ms / K)},
        "fma_peaks": peaks,
        "e2e": e2e,
        # per step: step kernel + force kernel (the bonded terms run inside it) (+ the
        # probe kernel; + the warp-per-replica reduction above 4 replicas, the step
        # kernel's inline limit), and the build's kernels (cells + list, 5 to 12 by
        # grid size) in the steps whose list is rebuilt
        "gpu_launches": (2 + bool(args.probe) + (s.n_replicas > 4)) * K + tim.build_kernels * int(tim.list_builds),
        "pair_list": {"skin_nm": args.skin, "skin_mode": args.skin_mode, "builds": int(tim.list_builds),
                      "unbuffered_builds": int(tim.list_unbuffered_builds), "steps": K,
                      "steps_per_build": (K / tim.list_builds) if tim.list_builds else None,
                      "entries_last_build": int(tim.list_entries), "capacity": int(tim.list_capacity)},
        "clocks": clk.summary(),
        "charge_state": ({"n_e": [int(v) for v in state["n_e"]], "te_ev": [float(v) for v in state["te_ev"]],
                          "events_pi_auger_ci_rec": [int(v) for v in state["event_counts"][0]]}
                         if s.n_replicas <= 8 else
                         {"n_e_total": int(state["n_e"].sum()),
                          "events_pi_auger_ci_rec": [int(v) for v in state["event_counts"].sum(0)]}),
    }
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"], out["force_error_vs_oracle"] = cpu_baseline(args, wl, atom)
        out["force_error_vs_oracle_ionised"] = ionised_force_errors(
            wl, atom, {"mixed": (state, s0 + W_ + K), "fp64": (state64, s0 + W_ + k64)}, args.screening)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return out


# ---------------------------------------------------------------------------
# CPU oracle: baseline leg and reference arm
# ---------------------------------------------------------------------------
def _oracle_run(wl, atom, seconds, max_steps_cap=50, screening="debye"):
    from oracle import oracle as O
    threads = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(threads))
    s = wl.sample
    t0 = time.perf_counter()
    md = O.OracleMD(s, atom, r_cut=1.2, t_start_fs=wl.t_start_fs, pulses=wl.pulses,
                    n_steps_max=max(wl.n_steps, max_steps_cap + 1), screening=screening)
    t_init = time.perf_counter() - t0
    md.F0 = md.F.copy()
    steps = 0
    t0 = time.perf_counter()
    while steps < max_steps_cap and (time.perf_counter() - t0) < seconds:
        md.step()
        steps += 1
    dt = time.perf_counter() - t0
    return md, steps, dt, t_init, int(os.environ["OMP_NUM_THREADS"])


SAMPLED_ABOVE = 60_000   # atoms: above this, the oracle is timed and compared on a sample


def cpu_baseline_sampled(args, wl, atom, compare_gpu=True):
    """Large systems: the oracle's all-pairs forces for m random atoms (m x N
    pair terms, about 1e9), timed per atom, and the GPU forces of both paths
    on the same atoms at the initial state."""
    from oracle import oracle as O
    O.build()
    threads = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(threads))
    s = wl.sample
    m = int(min(s.n_atoms, max(64, 1.0e9 // s.n_atoms)))
    idx = np.sort(np.random.default_rng(12).choice(s.n_atoms, m, replace=False))
    t0 = time.perf_counter()
    F_ref = O.forces_of_atoms(s, atom, idx, r_cut=1.2, kappa=0.0)
    dt = time.perf_counter() - t0
    base = {"value": m / dt, "unit": UNIT, "cores": int(os.environ["OMP_NUM_THREADS"]), "kind": "oracle",
            "sample": f"all-pairs FP64 forces of {m} random atoms of {args.workload} ({s.n_atoms} atoms) "
                      f"against all atoms of their replica ({dt:.1f} s), per atom; the O(N) charge update "
                      f"and integrator are left out (they cost < 1e-4 of the pair terms)"}
    if not compare_gpu:
        return base, None
    from paper_2401_03180_gb300 import md as M
    err = {}
    try:
        for prec in ("mixed", "fp64"):
            g = M.IonisingMD(s, atom, precision=prec, r_cut=1.2, max_steps=wl.n_steps, t_start_fs=wl.t_start_fs,
                             screening=args.screening)
            F = g.get_state(M.MD_FIELD_F)["f"][idx]
            g.close()
            err[prec] = force_error_stats(F, F_ref)
        err["state"] = f"initial state (neutral sample, kappa = 0), {m} sampled atoms"
    except Exception as e:
        err = {"error": str(e)[:200]}
    return base, err


def force_error_stats(F, F_ref):
    """RMS relative error, max error over RMS|F|, and the max relative error
    over atoms whose reference force exceeds a tenth of the RMS."""
    d = F - F_ref
    fn = np.linalg.norm(F_ref, axis=1)
    rms_f = float(np.sqrt((fn ** 2).mean()))
    big = fn > 0.1 * rms_f
    return {"rms_rel": float(np.linalg.norm(d) / np.linalg.norm(F_ref)),
            "max_abs_over_rms": float(np.abs(d).max() / rms_f),
            "max_rel_big": float((np.linalg.norm(d[big], axis=1) / fn[big]).max()) if big.any() else None}


def ionised_force_errors(wl, atom, states, screening):
    """Forces of the GPU paths at the end of their timed runs (ionised, with
    free electrons and kappa > 0, so the screened Coulomb term is exercised)
    against the oracle's all-pairs forces at the same positions, charges and
    kappa: every atom up to 60,000 atoms, else a random sample of about 1e9
    pair terms."""
    import dataclasses
    from oracle import oracle as O
    O.build()
    if screening != "debye":
        return {"skipped": "hybrid screening: the sampled check covers the Debye path"}
    s = wl.sample
    n = s.n_atoms
    m = n if n <= SAMPLED_ABOVE else int(min(n, max(64, 1.0e9 // n)))
    idx = np.arange(n) if m == n else np.sort(np.random.default_rng(13).choice(n, m, replace=False))
    out = {}
    for prec, (st, steps) in states.items():
        ss = dataclasses.replace(s, x=st["x"], q0=st["q"].astype(np.uint8))
        t0 = time.perf_counter()
        F_ref = O.forces_of_atoms(ss, atom, idx, r_cut=1.2, kappa=st["kappa"])
        ne, kap = np.asarray(st["n_e"]), np.asarray(st["kappa"])
        plasma = ({"n_e": [int(v) for v in ne], "kappa": [float(v) for v in kap]} if len(ne) <= 8 else
                  {"n_e_total": int(ne.sum()), "kappa_min": float(kap.min()), "kappa_max": float(kap.max())})
        out[prec] = dict(force_error_stats(st["f"][idx], F_ref), steps=int(steps), **plasma,
                         atoms=int(m), oracle_s=round(time.perf_counter() - t0, 2))
    return out


def cpu_baseline(args, wl, atom):
    if wl.sample.n_atoms > SAMPLED_ABOVE:
        return cpu_baseline_sampled(args, wl, atom)
    md, steps, dt, t_init, cores = _oracle_run(wl, atom, args.cpu_seconds, screening=args.screening)
    s = wl.sample
    val = s.n_atoms * steps / dt
    base = {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{steps} steps of {args.workload} ({s.n_atoms} atoms), all-pairs FP64, "
                      f"after an untimed initial force evaluation ({t_init:.1f} s)"}
    # force error of the GPU paths vs the oracle on the initial state (same inputs)
    err = None
    try:
        from paper_2401_03180_gb300 import md as M
        F_ref = md.F0
        err = {}
        for prec in ("mixed", "fp64"):
            g = M.IonisingMD(s, atom, precision=prec, r_cut=1.2, max_steps=wl.n_steps, t_start_fs=wl.t_start_fs,
                             screening=args.screening)
            F = g.get_state(M.MD_FIELD_F)["f"]
            g.close()
            err[prec] = force_error_stats(F, F_ref)
        err["state"] = "initial state (neutral sample, kappa = 0), all atoms"
    except Exception as e:  # the baseline number stands even if the comparison fails
        err = {"error": str(e)[:200]}
    return base, err


REF_BUDGET_S = 120.0   # host seconds for the reference arm's warm-up and timed steps together


def run_reference(args, rank, world):
    """The oracle as the reference arm: W warm-up and K timed steps, each a
    bounded piece of the workload so that the whole run takes about
    REF_BUDGET_S.  A system whose full oracle steps fit runs them (forces,
    charge update, integration); a larger one times, per step, the all-pairs
    forces of a fresh random sample of atoms, sized from a short calibration,
    and reports atom-steps/s over the sampled atoms."""
    if rank != 0:
        return None
    from oracle import oracle as O
    O.build()
    wl, atom = make_workload(args.workload, args.scale, 0)
    if args.bonded:
        from paper_2401_03180_gb300 import workloads as W
        wl.sample = W.with_topology(wl.sample)
    s = wl.sample
    k, w = max(1, args.steps), max(0, args.warmup)
    os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1))
    cores = int(os.environ["OMP_NUM_THREADS"])
    per_step = REF_BUDGET_S / (k + w)
    md = None
    if s.n_atoms <= SAMPLED_ABOVE:
        md = O.OracleMD(s, atom, r_cut=1.2, t_start_fs=wl.t_start_fs, pulses=wl.pulses,
                        n_steps_max=max(wl.n_steps, k + w + 2), screening=args.screening)
        t0 = time.perf_counter()
        md.step()                                   # calibration, untimed
        if time.perf_counter() - t0 > per_step:
            md = None
    if md is not None:
        for _ in range(w):
            md.step()
        t0 = time.perf_counter()
        for _ in range(k):
            md.step()
        dt = time.perf_counter() - t0
        val = s.n_atoms * k / dt
        sample = f"{k} timed oracle steps (after {w} warm-up) of {args.workload} ({s.n_atoms} atoms)"
    else:
        rng = np.random.default_rng(13)
        t0 = time.perf_counter()
        O.forces_of_atoms(s, atom, rng.choice(s.n_atoms, 16, replace=False), r_cut=1.2, kappa=0.0)
        per_atom = (time.perf_counter() - t0) / 16
        m = int(min(s.n_atoms, max(8, per_step / per_atom)))
        for _ in range(w):
            O.forces_of_atoms(s, atom, rng.choice(s.n_atoms, m, replace=False), r_cut=1.2, kappa=0.0)
        dt = 0.0
        for _ in range(k):
            idx = rng.choice(s.n_atoms, m, replace=False)
            t0 = time.perf_counter()
            O.forces_of_atoms(s, atom, idx, r_cut=1.2, kappa=0.0)
            dt += time.perf_counter() - t0
        val = m * k / dt
        sample = (f"{k} timed steps (after {w} warm-up), each the all-pairs FP64 forces of {m} random atoms of "
                  f"{args.workload} ({s.n_atoms} atoms) against all atoms of their replica; atom-steps/s over "
                  f"the sampled atoms, ms_per_step extrapolated to all atoms (the O(N) charge update and "
                  f"integrator cost < 1e-4 of the pair terms)")
    return {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world, "steps": k,
            "warmup": w, "ms_per_step": 1e3 * s.n_atoms / val, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "n_atoms": s.n_atoms, "r_cut_nm": 1.2, "dt_as": 50},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_profile_case(args):
    """Kernels launched: init 10 (step kernel, 5 cell kernels, 3 list kernels,
    forces), then per step the step kernel and the forces, plus 8 when the list
    is rebuilt; --profile-resume adds the checkpoint round trip (step kernel, 5
    cell kernels, 3 list kernels, two force launches, refresh)."""
    import torch
    from paper_2401_03180_gb300 import build as B
    from paper_2401_03180_gb300 import md as M
    B.build()
    wl, atom = make_workload(args.workload, args.scale, 0)
    if args.bonded:
        from paper_2401_03180_gb300 import workloads as W
        wl.sample = W.with_topology(wl.sample)
    s = wl.sample
    g = M.IonisingMD(s, atom, precision=args.precision, r_cut=1.2, max_steps=max(wl.n_steps, args.warmup + args.steps + 1),
                     t_start_fs=wl.t_start_fs, autotune=False, list_skin_nm=args.skin, screening=args.screening,
                     list_skin_adaptive=args.skin_mode == "adaptive",
                     langevin_g=args.langevin if args.langevin > 0 else None)
    g.set_pulse(wl.pulses[0])
    g.step(args.warmup)
    g.step(args.steps)
    if args.profile_resume:
        # set_state rebuilds the list at the checkpoint's list positions, trims it
        # (one force launch) and evaluates the forces at the current positions (a
        # second one): the same kernel as a step between builds, launched on its own
        st = g.get_state(M.MD_FIELD_ALL)
        g.set_state(M.MD_FIELD_ALL, **{k: st[k] for k in ("x", "v", "q", "h", "n_e", "e_gas_mev",
                                                         "event_counts", "x_list")}, step=st["step"])
    torch.cuda.synchronize()
    t = g.timing()
    g.close()
    return {"profile_case": args.workload, "n_atoms": s.n_atoms, "precision": args.precision,
            "warmup": args.warmup, "steps": args.steps, "tile_warps": t.tile_warps,
            "tile_blocks_per_sm": t.tile_blocks_per_sm, "skin_nm": args.skin, "skin_mode": args.skin_mode,
            "list_builds": t.list_builds, "unbuffered_builds": t.list_unbuffered_builds}


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.profile_case:
        print(json.dumps(run_profile_case(args)), flush=True)
        return
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        out = run_gpu(args, rank, world, local)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
