#!/usr/bin/env python
"""Constant-potential electrostatics benchmark: one JSON line.

A step is one whole pass of the per-timestep CPM electrostatics (cpm_step: cell list, b from
real-space pairs + SPME, q = S(b + dpsi v) with the neutrality projection, SPME + real-space
forces on all electrolyte sites, float64 energies); with --workload paper-md it is one time step
of the whole MD loop (cpm_md_run).  Default: the paper-scale finite-field cell:
3,024 graphite electrode sites (9 x 14 cells x 3 layers x 2 electrodes, 38.34 x 34.44 x 168 A),
500 coarse-grained ion pairs (2,000 sites), SPME mesh 40 x 36 x 168 (1 A), order 5, alpha 0.25,
r_c 12 A, eta 1.979.  ns/day assumes one step per 2 fs timestep (Appendix A of the paper).

  python bench.py [--gpus N --steps K --warmup W --precision mixed|fp64 --impl gb300|reference]

N > 1 runs under torchrun: every rank steps an independent replica (different seed) on its own
GPU; there is no collective on the data path (replicas only), value is the aggregate.
--impl reference times the FP64 CPU oracle (the correctness reference) on this host's cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CPM MD ns/day and replica-steps/s on 1 GB300 vs plain FP64 GPU at |dq|<=1e-5 e"
NS_PER_DAY_PER_STEP_PER_S = 2.0e-6 * 86400.0        # 2 fs per step -> ns/day per (step/s)
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-baseline-child", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--oracle-out", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--seed", type=int, default=None)
    ap.add_argument("--kernels", default="auto",
                    help="auto (cpm_autotune picks) or 'S-apply,transform,assignment' names, e.g. "
                         "sym,library,sites, to run a fixed kernel choice (profiling captures)")
    ap.add_argument("--pair-variant", default="auto", choices=["auto", "cell", "warp-elec", "warp-elyt", "warp"],
                    help="real-space pair kernels: one block per cell, or one warp per target for electrode "
                         "targets, electrolyte targets or both (default: autotuned)")
    ap.add_argument("--pair-group", type=int, default=0,
                    help="z cells per block of the real-space pair kernels (default: the autotuner's choice)")
    ap.add_argument("--charge-every", type=int, default=5,
                    help="MD workloads: re-solve the electrode charges every k steps (Appendix B: 5)")
    ap.add_argument("--workload", default="paper", choices=["paper", "paper-dc", "paper-slab", "paper-proximal", "large",
                                                            "dc-large", "paper-md", "paper-dc-md"],
                    help="paper: the paper-scale cell (default); paper-dc / paper-slab: the same cell as a doubled "
                         "cell (6,048 sites, mirror blocks) or a slab (3x z padding); paper-proximal: only the "
                         "1,008 proximal-layer sites charged; large: the 10,080-site cell; "
                         "dc-large: the 40,320-site doubled cell (mirror blocks, mesh-operator A); paper-md / "
                         "paper-dc-md: the whole MD loop (velocity-Verlet, Nose-Hoover, Lennard-Jones, charges "
                         "re-solved every --charge-every steps) on point-ion versions of the paper cells")
    return ap.parse_args()


def replica_seed(base, rank):
    """Each rank steps its own independent replica (replicas only, no data-path collective)."""
    return base + 2 * rank


def reduce_max(x, device="cpu"):
    """Maximum of x over all ranks (the slowest rank's time sets the aggregate rate)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_steps_per_s(total_ms_max, steps, world):
    """Whole-job throughput: all ranks' steps over the slowest rank's timed region."""
    return world * steps / (total_ms_max / 1e3)


WORKLOADS = {
    "paper": ("paper-scale finite-field cell: 3,024 electrode sites (3-layer graphite x 2), 500 CG ion "
              "pairs (2,000 sites), 38.34x34.44x168 A, SPME 40x36x168 order 5, alpha 0.25, r_c 12 A", 2000),
    "paper-dc": ("paper-scale doubled cell: the 3,024-site cell and its z-mirror image (6,048 electrode sites, "
                 "S as two 3,024^2 mirror blocks), 500 CG ion pairs per sub-cell (4,000 sites), 38.34x34.44x336 A, "
                 "SPME 40x36x336 order 5, alpha 0.25, r_c 12 A", 2000),
    "paper-slab": ("paper-scale slab: the 3,024-site cell with z padded 3x (38.34x34.44x504 A Ewald box) and the "
                   "Yeh-Berkowitz dipole correction, 500 CG ion pairs, SPME 40x36x504 order 5, alpha 0.25, r_c 12 A",
                   2000),
    "paper-proximal": ("paper-scale finite-field cell with only the proximal electrode layers charged (1,008 "
                       "sites; the further layers are neutral), 500 CG ion pairs, 38.34x34.44x168 A, SPME 40x36x168 "
                       "order 5, alpha 0.25, r_c 12 A", 2000),
    "large": ("scaled finite-field cell: 10,080 electrode sites (3-layer graphite x 2), 5,000 point-ion pairs "
              "(10,000 sites), 63.90x68.88x154 A, SPME 64x70x160 order 5, alpha 0.25, r_c 12 A", 4000),
    "dc-large": ("large doubled cell: 40,320 electrode sites (two mirrored 125x123x100 A sub-cells, 3-layer "
                 "60x56 rectangular-lattice electrodes), 25,000 CG ion pairs (100,000 sites), 125x123x200 A, "
                 "SPME 128x128x200 order 5, alpha 0.25, r_c 12 A; S stored as two 20,160^2 mirror blocks, "
                 "A's reciprocal part as the SPME mesh operator", 5000),
    "paper-md": ("MD on the paper-scale finite-field cell: 3,024 electrode sites (3-layer graphite x 2), 1,000 "
                 "point-ion pairs +-0.78 e (2,000 Lennard-Jones sites, the site count of the CG cell), "
                 "38.34x34.44x168 A, SPME 40x36x168 order 5, alpha 0.25, r_c 12 A; velocity-Verlet 2 fs, "
                 "Nose-Hoover 400 K / 100 fs, force-shifted LJ 12 A, charges re-solved every k steps", 6000),
    "paper-dc-md": ("MD on the paper-scale doubled cell: 6,048 electrode sites (S as two 3,024^2 mirror blocks), "
                    "1,000 point-ion pairs per sub-cell (4,000 LJ sites), 38.34x34.44x336 A, SPME 40x36x336 order 5; "
                    "velocity-Verlet 2 fs, one Nose-Hoover thermostat per sub-cell (400 K / 100 fs), LJ 12 A, "
                    "charges re-solved every k steps", 6000),
}
GEOMETRY_NAME = {"paper": "finite field", "paper-dc": "doubled cell", "paper-slab": "slab",
                 "paper-proximal": "finite field", "large": "finite field",
                 "dc-large": "doubled cell", "paper-md": "finite field", "paper-dc-md": "doubled cell"}
MD_WORKLOADS = ("paper-md", "paper-dc-md")


def workload(seed, kind="paper"):
    import synth
    if kind == "large":
        return synth.config_large_ff(seed=seed)
    if kind == "dc-large":
        return synth.config_large_dc(seed=seed)
    if kind == "paper-dc":
        return synth.config_paper_cell(seed=seed, geometry="dc")
    if kind == "paper-slab":
        return synth.config_paper_cell(seed=seed, geometry="slab")
    if kind == "paper-proximal":
        return synth.proximal_only(synth.config_paper_cell(seed=seed))
    if kind == "paper-md":
        return synth.md_cell(seed=seed)
    if kind == "paper-dc-md":
        return synth.md_cell(seed=seed, geometry="dc")
    return synth.config_paper_cell(seed=seed)


def system_options(kind):
    """Build options of each workload: the doubled cell is built with mirror blocks and the mesh
    form of A's reciprocal part (the direct Ewald sum over ~10^6 k-vectors is out of reach in
    float64 at 40,320 sites)."""
    if kind == "dc-large":
        return {"matrix_kspace": "mesh", "dc_blocks": "mirror"}
    return {}


# ----------------------------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------------------------
# roofline models per phase: algorithmic bytes (HBM-bound kernels) or FP32 flops (ALU-bound pair
# kernels) per launch.  Phases made of one kernel of this library are the candidates for the
# dominant kernel; the FFT phases are mostly cuFFT.
# ----------------------------------------------------------------------------------------------
PAIR_FLOPS = 40            # FP32 flops per pair interaction within r_c (distance 8, erfc/exp 20, force 12)
# DRAM bytes (read + write) per launch from one ncu capture of the current kernels, keyed by workload
# and "phase:kernel variant" (the autotuner may pick another S-apply kernel, whose traffic was not
# captured: then traffic is null).  Summaries: profiles/dram_k_sapply32_k_pair_cell_paper-cell-ff-mixed.md,
# profiles/dram_k_sapply_sym_k_pair_cell_large-cell-ff-mixed.md (the S-apply phase there is the packed
# kernel plus its finishing kernel, so its traffic is the sum of both).  Set an entry to None whenever its kernel changes.
NCU_TRAFFIC_MIXED = {"paper": {"s_apply:rows": 36.74e6, "f_pair_elyt": 0.21248e6, "b_real": 0.1157e6},
                     "paper-dc": {}, "paper-slab": {}, "paper-proximal": {}, "paper-md": {}, "paper-dc-md": {},
                     "large": {"s_apply:sym": 212.28e6, "f_pair_elyt": 0.7493e6},
                     "dc-large": {}}
SINGLE_KERNEL_PHASES = ("b_real", "b_spread", "b_gather", "s_apply", "project", "f_gather", "f_pair_elyt",
                        "f_pair_elec", "energy")


def pair_counts(w):
    """Ordered (target, source) pairs within r_c for the workload: electrolyte targets with
    electrolyte and electrode sources (forces), electrode targets with electrolyte sources (b)."""
    from scipy.spatial import cKDTree
    import numpy as np
    box = np.asarray(w.box, float)
    R = np.mod(w.elyt_xyz[0], box)
    E = np.mod(w.elec_xyz, box)
    tl, te = cKDTree(R, boxsize=box), cKDTree(E, boxsize=box)
    ll = int(tl.count_neighbors(tl, w.rcut)) - len(R)       # ordered pairs, self excluded
    le = int(tl.count_neighbors(te, w.rcut))
    return {"f_pair_elyt": ll + le, "b_real": le}


def phase_model(phase, s, w, pairs):
    """(bound, algorithmic amount per launch, unit, description) for one profiled phase."""
    ne = s.ne
    mixed = s.params.precision == 1
    fb = 4 if mixed else 8
    if phase == "s_apply":
        import paper_2201_12963_gb300 as g
        mirror, s_bytes = g.cpm_matrix_layout(s.ctx)
        byt = s_bytes + 8 * ne * 3                # S once, b in, q out, S v
        what = f"two mirror blocks S+- ({ne // 2}^2 each)" if mirror else f"S ({ne}^2)"
        if s_bytes < (ne // 2 if mirror else ne) ** 2 * fb * (2 if mirror else 1) * 3 // 4:
            what = "upper-triangle tiles of " + what
        return "hbm", byt, "GB/s", f"{what} x {fb} B + b, Sv, q (float64)"
    if phase in pairs:
        return "alu", PAIR_FLOPS * pairs[phase], "TFLOP/s", f"{pairs[phase]} pairs within r_c x {PAIR_FLOPS} FP32 flops"
    return None


def alu_peak_tflops(sm_mhz):
    """FP32 (non-tensor) peak: 152 SMs x 128 FP32 lanes x 2 flops per FMA x SM clock."""
    return 152 * 128 * 2 * (sm_mhz or 2070.0) * 1e6 / 1e12


def setup_ranks():
    """(world, rank, local rank, device); one process per GPU, NCCL only for the barrier and max."""
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    return world, rank, local, torch.device("cuda", local)


def build_system(args, w, dev):
    """Build the context (timed) and pick the kernels (autotuned or fixed by --kernels)."""
    import torch
    import paper_2201_12963_gb300 as g
    from paper_2201_12963_gb300.driver import System
    tb = time.perf_counter()
    s = System(w, args.precision, device=dev, **system_options(args.workload))
    torch.cuda.synchronize(dev)
    build_s = time.perf_counter() - tb
    if args.kernels == "auto":
        variants = g.cpm_autotune(s.ctx, s.offsets, s.xyzq, s.dpsi, s.q)
    else:
        variants = tuple(args.kernels.split(","))
        g.cpm_set_sapply_variant(s.ctx, variants[0])
        g.cpm_set_fft_variant(s.ctx, variants[1])
        g.cpm_set_mesh_variant(s.ctx, variants[2])
    if args.pair_group > 0:
        g.cpm_set_pair_group(s.ctx, args.pair_group)
    if args.pair_variant != "auto":
        g.cpm_set_pair_variant(s.ctx, args.pair_variant)
    return s, build_s, variants


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def roofline(args, s, w, phase_ms, clk, sapply_variant):
    """Roofline objects of the dominant single-kernel phase and of the S-apply (per launch, from the
    library's per-phase CUDA events)."""
    peaks = load_peaks()
    pairs = pair_counts(w)
    mixed_prec = args.precision == "mixed"

    def roof_for(p):
        bound, amount, unit, desc = phase_model(p, s, w, pairs)
        sec = phase_ms[p] / 1e3
        if bound == "hbm":
            achieved, peak = amount / sec / 1e9, float(peaks.get("hbm_gbs", 6800.0))
            src = "measured (MEASURED_PEAKS.json hbm_gbs)" if "hbm_gbs" in peaks else "fallback"
        else:
            achieved, peak = amount / sec / 1e12, alu_peak_tflops(clk.get("sm_mhz"))
            src = "derived: 152 SMs x 128 FP32 lanes x 2 x median SM clock"
        key = f"{p}:{sapply_variant}" if p == "s_apply" else p
        traffic = NCU_TRAFFIC_MIXED[args.workload].get(key) if mixed_prec else None
        return {"bound": bound, "kernel": p, "achieved": round(achieved, 3), "peak": round(peak, 1), "unit": unit,
                "frac": round(achieved / peak, 4), "traffic": traffic, "algorithmic_per_launch": amount,
                "launch_ms": round(phase_ms[p], 5), "peak_source": src, "model": desc}

    mine = [p for p in SINGLE_KERNEL_PHASES if p in phase_ms]
    dom = max(mine, key=phase_ms.get)
    roof = roof_for(dom) if phase_model(dom, s, w, pairs) else None
    if roof is not None:
        roof["dominant_phase_overall"] = max(phase_ms, key=phase_ms.get)
    roof_s = roof_for("s_apply") if "s_apply" in phase_ms else None
    return roof, roof_s


def run_gb300(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    import paper_2201_12963_gb300 as g

    if args.workload in MD_WORKLOADS:
        return run_md(args)
    world, rank, local, dev = setup_ranks()
    w = workload(replica_seed(args.seed, rank), args.workload)
    s, build_s, (sapply_variant, fft_variant, mesh_variant) = build_system(args, w, dev)

    # the whole step captured once into a CUDA graph
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(side):
        for _ in range(3):
            s.step(elec=False, energy=True)
    torch.cuda.current_stream(dev).wait_stream(side)
    torch.cuda.synchronize(dev)
    st = g.cpm_status(s.ctx)
    if st != 0:
        raise RuntimeError(f"device status after warm-up: {g.cpm_strerror(st)}")
    l0 = g.cpm_counters(s.ctx)
    s.step(elec=False, energy=True)
    torch.cuda.synchronize(dev)
    launches_per_step = g.cpm_counters(s.ctx) - l0
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        s.step(elec=False, energy=True)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    for _ in range(max(3, args.warmup)):
        graph.replay()
    torch.cuda.synchronize(dev)

    K = args.steps
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    wall0 = time.perf_counter()
    for k in range(K):
        flush.zero_()
        ev0[k].record()
        graph.replay()
        ev1[k].record()
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - wall0
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    tot_ms = reduce_max(sum(step_ms), dev)
    ms_per_step = tot_ms / K
    steps_per_s = aggregate_steps_per_s(tot_ms, K, world)
    value = steps_per_s * NS_PER_DAY_PER_STEP_PER_S
    st = g.cpm_status(s.ctx)
    if st != 0:
        raise RuntimeError(f"device status after the timed region: {g.cpm_strerror(st)}")

    # ---- end to end through the public API with host buffers ----
    Ke = min(K, 50)
    off, xyzq = __import__("paper_2201_12963_gb300.driver", fromlist=["pack"]).pack(w)
    h_xyzq = torch.from_numpy(xyzq).pin_memory()
    nl = int(off[-1])
    h_f = torch.empty(3 * nl, dtype=torch.float64).pin_memory()
    h_e = torch.empty(4, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record()
    for _ in range(Ke):
        s.xyzq.copy_(h_xyzq, non_blocking=True)
        graph.replay()
        h_f.copy_(s.f_elyt[: 3 * nl], non_blocking=True)
        h_e.copy_(s.energy[:4], non_blocking=True)
        torch.cuda.current_stream(dev).synchronize()
    e1.record()
    torch.cuda.synchronize(dev)
    e2e_s = reduce_max(max(time.perf_counter() - t0, e0.elapsed_time(e1) / 1e3), dev)
    e2e_value = world * Ke / e2e_s * NS_PER_DAY_PER_STEP_PER_S

    # ---- per-phase profile of the same step (events inside the library), L2 flushed per step ----
    Kp = min(K, 50)
    g.cpm_profile_enable(s.ctx, 16 * Kp + 16)
    for _ in range(Kp):
        flush.zero_()
        s.step(elec=False, energy=True)
    prof = g.cpm_profile_read(s.ctx)
    g.cpm_profile_enable(s.ctx, 0)
    phase_ms = {k: v[0] / max(1, v[1]) for k, v in prof.items() if v[1] > 0}
    roof, roof_s = roofline(args, s, w, phase_ms, clk, sapply_variant)

    out = {"metric": METRIC, "value": round(value, 2), "unit": "ns/day", "n_gpus": world, "steps": K,
           "warmup": max(3, args.warmup), "ms_per_step": round(ms_per_step, 5), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == "mixed" else "f64",
           "data": "synthetic",
           "config": {"workload": WORKLOADS[args.workload][0], "geometry": GEOMETRY_NAME[args.workload],
                      "precision": args.precision, "build_s": round(build_s, 2),
                      "s_apply_variant": sapply_variant, "mesh_transform": fft_variant,
                      "charge_assignment": mesh_variant, "pair_group_z": g.cpm_get_pair_group(s.ctx),
                      "pair_kernel": g.cpm_get_pair_variant(s.ctx),
                      "kernel_choice": "autotuned" if args.kernels == "auto" else "fixed by --kernels",
                      "replicas_per_gpu": 1, "parallelism": f"replicas x{world} (no collective)",
                      "data_ns_per_day": round(value * (2 if GEOMETRY_NAME[args.workload] == "doubled cell" else 1), 2),
                      "l2": "flushed between steps (256 MiB write); per-step CUDA-event time",
                      "graph": "whole step captured in one CUDA graph", "steps_per_s": round(steps_per_s, 1),
                      "replica_steps_per_s": round(steps_per_s, 1), "wall_s": round(wall, 3)},
           "clocks": clk,
           "e2e": {"value": round(e2e_value, 2), "unit": "ns/day",
                   "h2d_bytes_per_step": int(xyzq.nbytes), "d2h_bytes_per_step": int(8 * 3 * nl + 32),
                   "steps": Ke},
           "gpu_launches": int(launches_per_step * K),
           "phase_ms": {k: round(v, 5) for k, v in phase_ms.items()},
           "roofline": roof, "roofline_s_apply": roof_s}
    q_batched = None
    if args.workload == "paper":
        out["batched"], q_batched = batched_replicas(args, dev, flush)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        if args.workload == "paper":
            out["cpu_baseline"], ref = cpu_baseline(args)
            if ref is not None:
                torch.cuda.synchronize(dev)
                out["accuracy"] = accuracy_against(ref, s.q.cpu().numpy(), s.f_elyt.cpu().numpy(),
                                                   s.energy[:4].cpu().numpy())
                if q_batched is not None and "q_batched" in ref:
                    try:
                        out["batched"]["accuracy"] = batched_accuracy(ref["q_batched"], q_batched)
                    except Exception as e:      # the line is printed whatever this comparison does
                        out["batched"]["accuracy"] = {"error": f"{type(e).__name__}: {e}"[:300]}
        else:
            out["cpu_baseline"] = {
                "value": None, "unit": "ns/day", "kind": "oracle", "cores": os.cpu_count(),
                "sample": f"not run: the oracle's dense A for {w.n_elec:,} sites takes hours on the host"}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_md(args):
    """MD workloads: a timed step is one velocity-Verlet time step of the whole MD loop (thermostat,
    kicks, drift, CPM electrostatics with charges re-solved every k steps and held in between,
    Lennard-Jones).  The loop runs as a CUDA graph of one k-step block (one charge re-solve and
    k - 1 fixed-charge force evaluations), replayed; L2 is flushed between replays."""
    import numpy as np
    import torch
    import torch.distributed as dist
    import synth
    import paper_2201_12963_gb300 as g
    from paper_2201_12963_gb300.driver import MD

    world, rank, local, dev = setup_ranks()
    w = workload(replica_seed(args.seed, rank), args.workload)
    mi = synth.md_inputs(w, seed=replica_seed(args.seed, rank) + 1)
    s, build_s, (sapply_variant, fft_variant, mesh_variant) = build_system(args, w, dev)
    k = max(1, args.charge_every)
    m = MD(s, mi, dt=synth.PAPER_TIMESTEP_FS, charge_every=k, lj_cut=w.rcut)
    m.run(0, energy=True)
    e_start = m.energies()[0]
    # untimed warm-up, ending on a block boundary (step index a multiple of k)
    warm = max(3, args.warmup)
    m.run(warm + (-warm) % k, energy=False)
    torch.cuda.synchronize(dev)
    st = g.cpm_status(s.ctx)
    if st != 0:
        raise RuntimeError(f"device status after warm-up: {g.cpm_strerror(st)}")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    if args.pair_variant == "auto" and args.pair_group == 0:
        m.tune()                                  # pair-kernel form and z group on the MD block itself
    l0 = g.cpm_counters(s.ctx)
    m.run(k, energy=True)
    torch.cuda.synchronize(dev)
    launches_per_block = g.cpm_counters(s.ctx) - l0
    replay = m.capture(k, energy=True)
    replay(2)
    torch.cuda.synchronize(dev)

    blocks = max(1, -(-args.steps // k))
    K = blocks * k
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(blocks)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(blocks)]
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    wall0 = time.perf_counter()
    for b in range(blocks):
        flush.zero_()
        ev0[b].record()
        replay.graph.replay()
        ev1[b].record()
    torch.cuda.synchronize(dev)
    g.cpm_md_advance(m.md, K)
    wall = time.perf_counter() - wall0
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    tot_ms = reduce_max(sum(a.elapsed_time(b) for a, b in zip(ev0, ev1)), dev)
    ms_per_step = tot_ms / K
    steps_per_s = aggregate_steps_per_s(tot_ms, K, world)
    value = steps_per_s * NS_PER_DAY_PER_STEP_PER_S
    st = g.cpm_status(s.ctx)
    if st != 0:
        raise RuntimeError(f"device status after the timed region: {g.cpm_strerror(st)}")
    e_end = m.energies()[0]

    # ---- end to end: per block, the state (positions, velocities) from pinned host memory, the
    # block, and the new state plus the energy record back to the host ----
    Ke = min(blocks, 20)
    h_x = s.xyzq.cpu().pin_memory()
    h_v = m.vel.cpu().pin_memory()
    o_x = torch.empty_like(h_x).pin_memory()
    o_v = torch.empty_like(h_v).pin_memory()
    o_e = torch.empty(8, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(Ke):
        s.xyzq.copy_(h_x, non_blocking=True)
        m.vel.copy_(h_v, non_blocking=True)
        replay.graph.replay()
        o_x.copy_(s.xyzq, non_blocking=True)
        o_v.copy_(m.vel, non_blocking=True)
        o_e.copy_(m.energy[:8], non_blocking=True)
        torch.cuda.current_stream(dev).synchronize()
    e2e_s = reduce_max(time.perf_counter() - t0, dev)
    g.cpm_md_advance(m.md, Ke * k)
    e2e_value = world * Ke * k / e2e_s * NS_PER_DAY_PER_STEP_PER_S
    h2d = int(h_x.numel() * 8 + h_v.numel() * 8)
    d2h = int(h2d + 64)

    # ---- per-phase profile of the electrostatics inside the loop (direct calls, no graph) ----
    g.cpm_profile_enable(s.ctx, 16 * 10 * k + 16)
    for _ in range(10):
        flush.zero_()
        m.run(k, energy=False)
    prof = g.cpm_profile_read(s.ctx)
    g.cpm_profile_enable(s.ctx, 0)
    g.cpm_status(s.ctx)
    phase_ms = {kk: v[0] / max(1, v[1]) for kk, v in prof.items() if v[1] > 0}
    roof, roof_s = roofline(args, s, w, phase_ms, clk, sapply_variant)

    out = {"metric": METRIC, "value": round(value, 2), "unit": "ns/day", "n_gpus": world, "steps": K,
           "warmup": warm, "ms_per_step": round(ms_per_step, 5), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == "mixed" else "f64",
           "data": "synthetic",
           "config": {"workload": WORKLOADS[args.workload][0], "geometry": GEOMETRY_NAME[args.workload],
                      "precision": args.precision, "build_s": round(build_s, 2), "charge_every": k,
                      "timestep_fs": synth.PAPER_TIMESTEP_FS, "thermostat": "Nose-Hoover 400 K, 100 fs",
                      "s_apply_variant": sapply_variant, "mesh_transform": fft_variant,
                      "charge_assignment": mesh_variant, "pair_group_z": g.cpm_get_pair_group(s.ctx),
                      "pair_kernel": g.cpm_get_pair_variant(s.ctx),
                      "kernel_choice": "autotuned" if args.kernels == "auto" else "fixed by --kernels",
                      "replicas_per_gpu": 1, "parallelism": f"replicas x{world} (no collective)",
                      "data_ns_per_day": round(value * (2 if GEOMETRY_NAME[args.workload] == "doubled cell" else 1), 2),
                      "l2": f"flushed between replays of the {k}-step block (256 MiB write); CUDA-event time per block",
                      "graph": f"one CUDA graph per {k}-step block (energy record at its end)",
                      "steps_per_s": round(steps_per_s, 1), "wall_s": round(wall, 3),
                      "temperature_K": [round(e_start["T"], 1), round(e_end["T"], 1)],
                      "steps_before_timing": warm + (-warm) % k + 3 * k + (28 * k if args.pair_variant == "auto" and args.pair_group == 0 else 0)},
           "clocks": clk,
           "e2e": {"value": round(e2e_value, 2), "unit": "ns/day", "h2d_bytes_per_step": h2d // k,
                   "d2h_bytes_per_step": d2h // k, "steps": Ke * k,
                   "note": f"per {k}-step block: state in, block, state and energy record out"},
           "gpu_launches": int(launches_per_block * blocks),
           "phase_ms": {kk: round(v, 5) for kk, v in phase_ms.items()},
           "roofline": roof, "roofline_s_apply": roof_s}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args)[0] if args.workload == "paper-md" else {
            "value": None, "unit": "ns/day", "kind": "oracle", "cores": os.cpu_count(),
            "sample": "not run for this workload (see the paper-md line)"}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def graph_step_ms(s, flush, steps, dev):
    """Capture one cpm_step of System s in a CUDA graph; mean CUDA-event time per replay with L2
    flushed before every replay."""
    import torch
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(side):
        for _ in range(3):
            s.step(elec=False, energy=True)
    torch.cuda.current_stream(dev).wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        s.step(elec=False, energy=True)
    for _ in range(3):
        graph.replay()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize(dev)
    for a, b in ev:
        flush.zero_()
        a.record()
        graph.replay()
        b.record()
    torch.cuda.synchronize(dev)
    return sum(a.elapsed_time(b) for a, b in ev) / steps


def batched_replicas(args, dev, flush):
    """Replica throughput: 64 replicas of the 672-site plain cell (400-600 point-ion pairs each,
    dpsi 0-4 V) in one batched step (mixed precision, tensor-core S-apply), against the plain
    float64 path stepping one replica of the same cell.  Returns the line's object and the
    batched step's charges [64, 672]."""
    import synth
    import paper_2201_12963_gb300 as g
    from paper_2201_12963_gb300.driver import System
    steps = max(10, min(args.steps, 100))
    wb = synth.config_batched(n_rep=64)
    sb = System(wb, "mixed", device=dev)
    ms_b = graph_step_ms(sb, flush, steps, dev)
    st = g.cpm_status(sb.ctx)
    q_b = sb.results()["q"]
    w1 = wb.replica(0)
    s1 = System(w1, "fp64", device=dev)
    ms_1 = graph_step_ms(s1, flush, steps, dev)
    return {"workload": "64 replicas x 672-site plain cell (17.04x17.22x60 A), 400-600 point-ion pairs each, "
                        "mesh 18x18x60 order 5", "replicas": 64, "precision": "mixed, tcgen05 split-TF32 S-apply",
            "ms_per_step": round(ms_b, 5), "replica_steps_per_s": round(64 * 1e3 / ms_b, 1),
            "plain_fp64_one_replica": {"ms_per_step": round(ms_1, 5), "steps_per_s": round(1e3 / ms_1, 1)},
            "speedup_replica_steps": round((64 / ms_b) / (1 / ms_1), 2), "status": st}, q_b


def batched_oracle_charges(n_rep=64):
    """The oracle's charges [n_rep, 672] for every replica of the batched workload (one A and
    Cholesky factor for the shared electrode, one b and KKT solve per replica)."""
    import numpy as np
    import synth
    from oracle import cpm as ocpm
    wb = synth.config_batched(n_rep=n_rep)
    ref = ocpm.Reference(wb.replica(0))
    out = np.zeros((n_rep, wb.n_elec))
    for r in range(n_rep):
        out[r] = ref.charges(wb.elyt_xyz[r], wb.elyt_q[r], float(wb.dpsi[r]))[0]
    return out


def batched_accuracy(q_ref, q):
    """Per-replica max |dq| (e) of the batched step's charges against the oracle's."""
    import numpy as np
    q_ref = np.asarray(q_ref)
    q = np.asarray(q).reshape(q_ref.shape[0], -1)[:, : q_ref.shape[1]]
    dq = np.abs(q - q_ref).max(axis=1)
    return {"dq_max_e": float(dq.max()), "dq_max_e_per_replica": [float(f"{x:.3g}") for x in dq],
            "replicas_within_1e-5_e": int((dq <= 1e-5).sum()), "replicas": int(dq.size),
            "reference": "FP64 CPU oracle (direct Ewald b, KKT solve) per replica on the same input"}


# ----------------------------------------------------------------------------------------------
# CPU oracle timings
# ----------------------------------------------------------------------------------------------
def cpu_baseline(args):
    """One full oracle step of the same workload on this host, timed in a child process
    (the oracle's A and its Cholesky factor are built first, untimed).  The child also leaves its
    charges, electrolyte forces and energies in a scratch file: the GPU run's errors against them
    are the line's `accuracy`."""
    import tempfile
    fd, path = tempfile.mkstemp(suffix=".npz")
    os.close(fd)
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-baseline-child", "--seed", str(args.seed),
           "--workload", args.workload, "--oracle-out", path]
    try:
        r = subprocess.run(cmd, capture_output=True, text=True, timeout=900)
        if r.returncode != 0:
            return {"value": None, "unit": "ns/day", "kind": "oracle", "error": r.stderr[-300:]}, None
        import numpy as np
        with np.load(path) as z:
            ref = {k: z[k] for k in z.files}
        return json.loads(r.stdout.strip().splitlines()[-1]), ref
    finally:
        if os.path.exists(path):
            os.remove(path)


def accuracy_against(ref, q, f_elyt, energy):
    """Errors of one GPU step against the oracle's step on the same input: max |dq| (e), RMS
    relative force error on the electrolyte, relative error of U and of H."""
    import numpy as np
    q = np.asarray(q).reshape(-1)[: ref["q"].size]
    F = np.asarray(f_elyt).reshape(-1, 3)[: ref["F_elyt"].shape[0]]
    Fo = ref["F_elyt"]
    return {"dq_max_e": float(np.abs(q - ref["q"]).max()),
            "force_rms_rel": float(np.sqrt(((F - Fo) ** 2).sum() / (Fo ** 2).sum())),
            "energy_U_rel": float(abs(energy[0] - ref["U"]) / abs(ref["U"])),
            "energy_H_rel": float(abs(energy[1] - ref["H"]) / abs(ref["H"])),
            "reference": "FP64 CPU oracle (direct Ewald sums, KKT solve) on the same input"}


def cpu_baseline_child(args):
    from oracle import cpm as ocpm
    w = workload(args.seed, args.workload)
    ref = ocpm.Reference(w)
    t0 = time.perf_counter()
    out = ref.step(0)
    dt = time.perf_counter() - t0
    if args.oracle_out:
        import numpy as np
        extra = {}
        if args.workload == "paper":       # untimed: the batched line's per-replica accuracy
            extra["q_batched"] = batched_oracle_charges()
        np.savez(args.oracle_out, q=out["q"], F_elyt=out["F_elyt"], U=out["U"], H=out["H"], **extra)
    print(json.dumps({"value": round(NS_PER_DAY_PER_STEP_PER_S / dt, 6), "unit": "ns/day", "cores": os.cpu_count(),
                      "kind": "oracle", "seconds_per_step": round(dt, 3),
                      "sample": "one full FP64 oracle step (direct Ewald b, KKT solve with a prebuilt Cholesky "
                                "factor, full-Ewald energy and forces) of the benchmark workload; numpy, "
                                "BLAS threads = all cores, elementwise work single-threaded"
                                + ("; for the MD workload this is the charge re-solve step, an upper bound of the "
                                   "oracle's MD step (its Lennard-Jones and integration cost are not added)"
                                   if args.workload in MD_WORKLOADS else "")}))


def run_reference(args):
    """The reference arm: the FP64 oracle, each step a bounded sample (a random fraction f of the
    real-space targets and of the k-vectors), scaled to a full step through a two-point fit
    t(f) = a + b f made during the warm-up."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    from oracle import cpm as ocpm
    w = workload(args.seed, args.workload)
    ref = ocpm.Reference(w)
    f1, f2 = 0.03, 0.12
    t = time.perf_counter(); ref.sampled_step(0, f1, 1); t1 = time.perf_counter() - t
    t = time.perf_counter(); ref.sampled_step(0, f2, 2); t2 = time.perf_counter() - t
    b = max(1e-9, (t2 - t1) / (f2 - f1))
    a = max(0.0, t1 - b * f1)
    budget = 150.0 / max(1, args.steps + args.warmup)      # keep the whole run within a few minutes
    f = min(0.5, max(0.01, (budget - a) / b))
    for k in range(max(0, args.warmup - 2)):
        ref.sampled_step(0, f, 10 + k)
    ts = []
    for k in range(args.steps):
        t = time.perf_counter()
        ref.sampled_step(0, f, 100 + k)
        ts.append(time.perf_counter() - t)
    tmean = sum(ts) / len(ts)
    t_full = a + (tmean - a) / f
    value = NS_PER_DAY_PER_STEP_PER_S / t_full
    sample = (f"per step: real-space sums over a random {f:.3f} of the target sites and reciprocal sums "
              f"over a random {f:.3f} of the k-vectors, KKT solve in full; full-step time estimated as "
              f"a + (t - a)/f with a = {a:.3f} s from a two-point fit (t(f) = a + b f)")
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "ns/day", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_full * 1e3, 1),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOADS[args.workload][0], "geometry": GEOMETRY_NAME[args.workload],
                      "precision": "fp64 oracle"},
           "cpu_baseline": {"value": round(value, 6), "unit": "ns/day", "cores": os.cpu_count(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": round(value, 6), "unit": "ns/day", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.seed is None:
        args.seed = WORKLOADS[args.workload][1]
    if args.cpu_baseline_child:
        cpu_baseline_child(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gb300(args)


if __name__ == "__main__":
    main()
