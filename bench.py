#!/usr/bin/env python
"""Constant-potential electrostatics benchmark: one JSON line.

A step is one whole pass of the per-timestep CPM electrostatics (cpm_step: cell list, b from
real-space pairs + SPME, q = S(b + dpsi v) with the neutrality projection, SPME + real-space
forces on all sites -- electrolyte and electrode --, float64 energies), captured in one CUDA graph;
with --workload paper-md it is one time step of the whole MD loop (cpm_md_run).

Default workload: the large doubled cell -- 40,320 electrode sites (two mirrored 125 x 123 x 100 A
sub-cells with three-layer electrodes), 25,000 coarse-grained ion pairs (100,000 sites), SPME mesh
128 x 128 x 200 order 5, alpha 0.25, r_c 12 A, eta 1.979; S stored as two 20,160^2 mirror blocks.
ns/day assumes one step per 2 fs timestep (Appendix A of the paper); a doubled cell simulates two
cells, so its data ns/day is twice that.

The line also carries, on one GPU: the same workload on the plain float64 path (`plain_fp64`), the
errors of the timed step against the float64 path and against the FP64 oracle (`accuracy`), the
paper-scale cell (`paper_cell`), 64 batched replicas on the tensor-core S-apply (`batched`) and the
oracle timed on the host's cores (`cpu_baseline`).

  python bench.py [--gpus N --steps K --warmup W --workload W --precision mixed|fp64 --impl gb300|reference]

N > 1 runs under torchrun: every rank steps an independent replica (different seed) on its own
GPU; there is no collective on the data path (replicas only), value is the aggregate.
--impl reference times the FP64 CPU oracle (the correctness reference) on this host's cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import pickle
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CPM MD ns/day and replica-steps/s on 1 GB300 vs plain FP64 GPU at |dq|<=1e-5 e"
NS_PER_DAY_PER_STEP_PER_S = 2.0e-6 * 86400.0        # 2 fs per step -> ns/day per (step/s)
L2_FLUSH_BYTES = 256 << 20


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="only the main line: no float64 comparison, accuracy, paper-cell, batched or CPU objects")
    ap.add_argument("--child", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--workload-file", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--child-out", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--child-in", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--seed", type=int, default=None)
    ap.add_argument("--kernels", default="auto",
                    help="auto (cpm_autotune picks) or 'S-apply,transform,assignment' names, e.g. "
                         "sym,library,sites, to run a fixed kernel choice (profiling captures)")
    ap.add_argument("--pair-variant", default="auto",
                    choices=["auto", "cell", "warp-elec", "warp-elyt", "warp", "n3", "n3-warp-elec"],
                    help="real-space pair kernels: one block per cell, or one warp per target for electrode "
                         "targets, electrolyte targets or both (default: autotuned)")
    ap.add_argument("--pair-group", type=int, default=0,
                    help="z cells per block of the real-space pair kernels (default: the autotuner's choice)")
    ap.add_argument("--charge-every", type=int, default=5,
                    help="MD workloads: re-solve the electrode charges every k steps (Appendix B: 5)")
    ap.add_argument("--workload", default="dc-large",
                    choices=["paper", "paper-dc", "paper-slab", "paper-proximal", "large", "dc-large", "paper-md",
                             "paper-dc-md", "batched"],
                    help="dc-large (default): the 40,320-site doubled cell (mirror blocks, mesh-operator A); "
                         "paper: the paper-scale cell; paper-dc / paper-slab: the same cell as a doubled "
                         "cell (6,048 sites, mirror blocks) or a slab (3x z padding); paper-proximal: only the "
                         "1,008 proximal-layer sites charged; large: the 10,080-site cell; paper-md / "
                         "paper-dc-md: the whole MD loop (velocity-Verlet, Nose-Hoover, Lennard-Jones, charges "
                         "re-solved every --charge-every steps) on point-ion versions of the paper cells; batched: "
                         "64 replicas of the 672-site plain cell in one batched step (replica-steps/s)")
    return ap.parse_args(argv)


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
    "batched": ("64 replicas x 672-site plain cell (17.04x17.22x60 A), 400-600 point-ion pairs each, dpsi 0-4 V, "
                "mesh 18x18x60 order 5, one batched step with the tcgen05 split-TF32 S-apply", 3000),
    "paper-dc-md": ("MD on the paper-scale doubled cell: 6,048 electrode sites (S as two 3,024^2 mirror blocks), "
                    "1,000 point-ion pairs per sub-cell (4,000 LJ sites), 38.34x34.44x336 A, SPME 40x36x336 order 5; "
                    "velocity-Verlet 2 fs, one Nose-Hoover thermostat per sub-cell (400 K / 100 fs), LJ 12 A, "
                    "charges re-solved every k steps", 6000),
}
GEOMETRY_NAME = {"paper": "finite field", "paper-dc": "doubled cell", "paper-slab": "slab",
                 "paper-proximal": "finite field", "large": "finite field",
                 "dc-large": "doubled cell", "paper-md": "finite field", "paper-dc-md": "doubled cell",
                 "batched": "finite field"}
MD_WORKLOADS = ("paper-md", "paper-dc-md")
# workloads whose oracle step fits the host in seconds to a minute (dense A and its Cholesky factor);
# the others are checked and timed through sampled sums
DENSE_ORACLE = ("paper", "paper-dc", "paper-slab", "paper-proximal", "paper-md", "paper-dc-md")


def workload(seed, kind="paper"):
    import synth
    if kind == "batched":
        return synth.config_batched(n_rep=64)
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


def load_workload(args):
    """The workload of a child process: from the parent's pickle (config 5 takes ~20 s to draw)."""
    if args.workload_file:
        with open(args.workload_file, "rb") as f:
            return pickle.load(f)
    return workload(args.seed, args.workload)


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
# roofline models per phase: algorithmic bytes (HBM-bound kernels), FP32 flops (ALU-bound pair
# kernels) or tensor flops (the batched tcgen05 S-apply) per launch.  Phases made of one kernel of
# this library are the candidates for the dominant kernel; the FFT phases are mostly cuFFT.
# ----------------------------------------------------------------------------------------------
PAIR_FLOPS = 40            # FP32 flops per pair interaction within r_c (distance 8, erfc/exp 20, force 12)
TF32_OVER_BF16 = 1.1 / 2.25   # nominal dense tf32 / bf16 tensor rate of GB300
# DRAM bytes (read + write) per launch from one ncu capture of the current kernels, keyed by workload
# and "phase:kernel variant" (the autotuner may pick another S-apply kernel, whose traffic was not
# captured: then traffic is null).  Set an entry to None whenever its kernel changes.
# The packed S-apply kernels (sym, sym-tma) changed after their capture (the projection sums and
# the split epilogue; the tile reads are the same), so their entries are None until the next
# capture; the capture before the change measured 19.894 MB (paper) and 1,649.7 MB (dc-large: the
# two packed applies and the two finishes) against 19.73 MB and 1,647.4 MB algorithmic.
# profiles/dram_dc-large-and-paper-cell-mixed.md.
NCU_TRAFFIC_MIXED = {"paper": {"s_apply:sym": None, "s_apply:sym-tma": None, "f_pair_elyt:cell": 214_000,
                               "f_pair_elec": 6_720_000},
                     "paper-dc": {}, "paper-slab": {}, "paper-proximal": {}, "paper-md": {},
                     "paper-dc-md": {}, "large": {},
                     "dc-large": {"s_apply:sym-tma": None, "f_pair_elyt:cell": 5_580_000, "f_pair_elyt:n3": 4_340_000,
                                  "f_pair_elec": 51_420_000},
                     "batched": {}}
SINGLE_KERNEL_PHASES = ("b_real", "b_spread", "b_gather", "s_apply", "project", "f_gather", "f_pair_elyt",
                        "f_pair_elec", "energy")


def pair_counts(w):
    """Ordered (target, source) pairs within r_c for the workload: electrolyte targets with
    electrolyte and electrode sources (forces), electrode targets with electrolyte sources (b and,
    in the same pass, the field for the electrode forces) and electrode targets with electrode
    sources (the electrode-electrode forces)."""
    from scipy.spatial import cKDTree
    import numpy as np
    box = np.asarray(w.box, float)
    R = np.mod(w.elyt_xyz[0], box)
    E = np.mod(w.elec_xyz, box)
    tl, te = cKDTree(R, boxsize=box), cKDTree(E, boxsize=box)
    ll = int(tl.count_neighbors(tl, w.rcut)) - len(R)       # ordered pairs, self excluded
    le = int(tl.count_neighbors(te, w.rcut))
    ee = int(te.count_neighbors(te, w.rcut)) - len(E)
    return {"f_pair_elyt": ll + le, "b_real": le, "f_pair_elec": ee}


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
    if phase == "f_pair_elec" and mixed:
        # the frozen electrode's precomputed pair list, streamed once
        import paper_2201_12963_gb300 as g
        npairs, table = g.cpm_pair_list_layout(s.ctx)
        if npairs:
            eb = 4 if table else 16
            byt = npairs * eb + 4 * (ne + 1) + ne * (4 + 48)
            form = "compressed list: j and an index into a table of distinct G" if table else "full list: G and j"
            return ("hbm", byt, "GB/s", f"{npairs} electrode pairs x {eb} B ({form}) + row starts, charges and "
                    f"forces (float64, read and written)")
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


def build_system(args, w, dev, precision=None, image=None, tune=True):
    """Build the context (timed) and pick the kernels (autotuned or fixed by --kernels)."""
    import torch
    import paper_2201_12963_gb300 as g
    from paper_2201_12963_gb300.driver import System
    tb = time.perf_counter()
    s = System(w, precision or args.precision, device=dev, image=image, **system_options(args.workload))
    torch.cuda.synchronize(dev)
    build_s = time.perf_counter() - tb
    variants = ("default", "default", "default")
    if args.kernels == "auto":
        if tune:
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


def roofline(workload_kind, s, w, phase_ms, clk):
    """Roofline objects of the dominant single-kernel phase and of the S-apply (per launch, from the
    library's per-phase CUDA events)."""
    peaks = load_peaks()
    pairs = pair_counts(w)
    mixed_prec = s.params.precision == 1
    sapply_variant = s.sapply_variant
    import paper_2201_12963_gb300 as g
    pair_variant = g.cpm_get_pair_variant(s.ctx)

    def roof_for(p):
        bound, amount, unit, desc = phase_model(p, s, w, pairs)
        sec = phase_ms[p] / 1e3
        if bound == "hbm":
            achieved, peak = amount / sec / 1e9, float(peaks.get("hbm_gbs", 6800.0))
            src = ("of measured (MEASURED_PEAKS.json hbm_gbs, burst copy)" if "hbm_gbs" in peaks
                   else "of fallback (6.8 TB/s)")
        else:
            achieved, peak = amount / sec / 1e12, alu_peak_tflops(clk.get("sm_mhz"))
            src = "derived: 152 SMs x 128 FP32 lanes x 2 x median SM clock under load"
        key = (f"{p}:{sapply_variant}" if p == "s_apply" else
               f"{p}:{pair_variant}" if p in ("f_pair_elyt", "b_real") else p)
        traffic = NCU_TRAFFIC_MIXED.get(workload_kind, {}).get(key) if mixed_prec else None
        return {"bound": bound, "kernel": p, "achieved": round(achieved, 3), "peak": round(peak, 1), "unit": unit,
                "frac": round(achieved / peak, 4), "traffic": traffic, "algorithmic_per_launch": amount,
                "launch_ms": round(phase_ms[p], 5), "peak_source": src, "model": desc}

    mine = [p for p in SINGLE_KERNEL_PHASES if p in phase_ms]
    dom = max(mine, key=phase_ms.get)
    roof = roof_for(dom) if phase_model(dom, s, w, pairs) else None
    if roof is not None:
        roof["dominant_phase_overall"] = max(phase_ms, key=phase_ms.get)
    roof_s = roof_for("s_apply") if "s_apply" in phase_ms else None
    roof_pair = roof_for("f_pair_elyt") if "f_pair_elyt" in phase_ms else None
    # the electrode pair list (HBM model), where the step uses it
    roof_ee = None
    if "f_pair_elec" in phase_ms and (phase_model("f_pair_elec", s, w, pairs) or ("",))[0] == "hbm":
        roof_ee = roof_for("f_pair_elec")
    return roof, roof_s, roof_pair, roof_ee


# ----------------------------------------------------------------------------------------------
# timing helpers
# ----------------------------------------------------------------------------------------------
def capture_step(s, elec, dev):
    """Warm the step up on a side stream, then capture one cpm_step in a CUDA graph."""
    import torch
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(side):
        for _ in range(3):
            s.step(elec=elec, energy=True)
    torch.cuda.current_stream(dev).wait_stream(side)
    torch.cuda.synchronize(dev)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        s.step(elec=elec, energy=True)
    return graph


def time_replays(graph, flush, K, dev, warmup=3, world=1, clocks=None):
    """Replays of graph with L2 flushed before each, CUDA events around each replay on the launching
    stream; (total ms, per-step ms list, host wall seconds)."""
    import torch
    import torch.distributed as dist
    for _ in range(max(3, warmup)):
        graph.replay()
    torch.cuda.synchronize(dev)
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    if clocks is not None:
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
    step_ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    return sum(step_ms), step_ms, wall


def profile_phases(s, flush, K, elec):
    """Per-phase device times (ms per launch) of K direct calls, L2 flushed before each call."""
    import paper_2201_12963_gb300 as g
    g.cpm_profile_enable(s.ctx, 16 * K + 16)
    for _ in range(K):
        flush.zero_()
        s.step(elec=elec, energy=True)
    prof = g.cpm_profile_read(s.ctx)
    g.cpm_profile_enable(s.ctx, 0)
    return {k: v[0] / max(1, v[1]) for k, v in prof.items() if v[1] > 0}


def end_to_end(s, w, graph, dev, steps, world, elec):
    """The same step through the public API with host buffers: every step copies the electrolyte
    positions and charges in from pinned host memory and the electrode charges, forces and energies
    back; (ns/day, bytes in, bytes out)."""
    import torch
    from paper_2201_12963_gb300.driver import pack
    off, xyzq = pack(w)
    h_xyzq = torch.from_numpy(xyzq).pin_memory()
    nl, ne = int(off[-1]), s.ne
    h_q = torch.empty(ne, dtype=torch.float64).pin_memory()
    h_f = torch.empty(3 * nl, dtype=torch.float64).pin_memory()
    h_fe = torch.empty(3 * ne, dtype=torch.float64).pin_memory()
    h_e = torch.empty(4, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record()
    for _ in range(steps):
        s.xyzq.copy_(h_xyzq, non_blocking=True)
        graph.replay()
        h_q.copy_(s.q[:ne], non_blocking=True)
        h_f.copy_(s.f_elyt[: 3 * nl], non_blocking=True)
        if elec:
            h_fe.copy_(s.f_elec[: 3 * ne], non_blocking=True)
        h_e.copy_(s.energy[:4], non_blocking=True)
        torch.cuda.current_stream(dev).synchronize()
    e1.record()
    torch.cuda.synchronize(dev)
    e2e_s = reduce_max(max(time.perf_counter() - t0, e0.elapsed_time(e1) / 1e3), dev)
    d2h = 8 * (ne + 3 * nl + (3 * ne if elec else 0) + 4)
    return world * steps / e2e_s * NS_PER_DAY_PER_STEP_PER_S, int(xyzq.nbytes), int(d2h)


def step_results(s, elec):
    """q, electrolyte forces, electrode forces and energies of the last step (host copies)."""
    r = s.results()
    return {"q": r["q"][0], "F_elyt": r["F_elyt"][0], "F_elec": r["F_elec"][0] if elec else None,
            "energy": r["energy"][0]}


def precision_errors(mixed, fp64):
    """The timed (mixed-precision) step against the float64 GPU path on the same input and mesh:
    the float32 error, apart from the mesh discretisation that both share."""
    import numpy as np

    def rms(a, b):
        return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))
    out = {"dq_max_e": float(np.abs(mixed["q"] - fp64["q"]).max()),
           "force_rms_rel_elyt": rms(mixed["F_elyt"], fp64["F_elyt"]),
           "energy_U_rel": float(abs(mixed["energy"][0] - fp64["energy"][0]) / abs(fp64["energy"][0])),
           "energy_H_rel": float(abs(mixed["energy"][1] - fp64["energy"][1]) / abs(fp64["energy"][1]))}
    if mixed["F_elec"] is not None and fp64["F_elec"] is not None:
        out["force_rms_rel_elec"] = rms(mixed["F_elec"], fp64["F_elec"])
    return out


# ----------------------------------------------------------------------------------------------
# the GPU arm
# ----------------------------------------------------------------------------------------------
def run_gb300(args):
    import torch
    import torch.distributed as dist
    import paper_2201_12963_gb300 as g

    if args.workload in MD_WORKLOADS:
        return run_md(args)
    if args.workload == "batched":
        return run_batched(args)
    world, rank, local, dev = setup_ranks()
    w = workload(replica_seed(args.seed, rank), args.workload)
    s, build_s, (sapply_variant, fft_variant, mesh_variant) = build_system(args, w, dev)
    s.sapply_variant = sapply_variant
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    # ---- the timed step: charges, forces on all sites, energies; one CUDA graph ----
    graph = capture_step(s, True, dev)
    st = g.cpm_status(s.ctx)
    if st != 0:
        raise RuntimeError(f"device status after warm-up: {g.cpm_strerror(st)}")
    l0 = g.cpm_counters(s.ctx)
    s.step(elec=True, energy=True)
    torch.cuda.synchronize(dev)
    launches_per_step = g.cpm_counters(s.ctx) - l0
    K = args.steps
    clocks = ClockSampler(local)
    tot_ms, step_ms, wall = time_replays(graph, flush, K, dev, args.warmup, world, clocks)
    clk = clocks.stop()
    tot_ms = reduce_max(tot_ms, dev)
    ms_per_step = tot_ms / K
    steps_per_s = aggregate_steps_per_s(tot_ms, K, world)
    value = steps_per_s * NS_PER_DAY_PER_STEP_PER_S
    st = g.cpm_status(s.ctx)
    if st != 0:
        raise RuntimeError(f"device status after the timed region: {g.cpm_strerror(st)}")
    mixed_res = step_results(s, True)

    # the same step without electrode forces (a frozen electrode in MD needs none)
    graph_fe = capture_step(s, False, dev)
    Kf = min(K, 300)
    tot_fe, _, _ = time_replays(graph_fe, flush, Kf, dev, 3, world)
    tot_fe = reduce_max(tot_fe, dev)
    del graph_fe

    e2e_value, h2d, d2h = end_to_end(s, w, graph, dev, min(K, 50), world, True)
    phase_ms = profile_phases(s, flush, min(K, 50), True)
    roof, roof_s, roof_pair, roof_ee = roofline(args.workload, s, w, phase_ms, clk)
    geo = GEOMETRY_NAME[args.workload]
    out = {"metric": METRIC, "value": round(value, 2), "unit": "ns/day", "n_gpus": world, "steps": K,
           "warmup": max(3, args.warmup), "ms_per_step": round(ms_per_step, 5), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == "mixed" else "f64",
           "data": "synthetic",
           "config": {"workload": WORKLOADS[args.workload][0], "geometry": geo, "precision": args.precision,
                      "precision_detail": ("float32 pair, mesh and S-apply arithmetic with compensated sums; "
                                           "float64 A, factorisation, projection and energy accumulation"
                                           if args.precision == "mixed" else "float64 throughout"),
                      "forces": "all sites (electrolyte and electrode)", "build_s": round(build_s, 2),
                      "s_apply_variant": sapply_variant, "mesh_transform": fft_variant,
                      "charge_assignment": mesh_variant, "pair_group_z": g.cpm_get_pair_group(s.ctx),
                      "pair_kernel": g.cpm_get_pair_variant(s.ctx),
                      "kernel_choice": "autotuned" if args.kernels == "auto" else "fixed by --kernels",
                      "replicas_per_gpu": 1, "parallelism": f"replicas x{world} (no collective)",
                      "data_ns_per_day": round(value * (2 if geo == "doubled cell" else 1), 2),
                      "l2": "flushed between steps (256 MiB write); per-step CUDA-event time",
                      "graph": "whole step captured in one CUDA graph", "steps_per_s": round(steps_per_s, 1),
                      "replica_steps_per_s": round(steps_per_s, 1), "wall_s": round(wall, 3)},
           "clocks": clk,
           "e2e": {"value": round(e2e_value, 2), "unit": "ns/day", "h2d_bytes_per_step": h2d,
                   "d2h_bytes_per_step": d2h, "steps": min(K, 50),
                   "note": "per step: electrolyte xyzq in from pinned host memory; electrode charges, "
                           "electrolyte and electrode forces and energies out"},
           "gpu_launches": int(launches_per_step * K),
           "frozen_electrode": {"ms_per_step": round(tot_fe / Kf, 5),
                                "value": round(world * Kf / (tot_fe / 1e3) * NS_PER_DAY_PER_STEP_PER_S, 2),
                                "unit": "ns/day", "steps": Kf,
                                "note": "the same step without electrode forces (forces on electrolyte sites only)"},
           "phase_ms": {k: round(v, 5) for k, v in phase_ms.items()},
           "roofline": roof, "roofline_s_apply": roof_s, "roofline_pair_elyt": roof_pair,
           "roofline_pair_list": roof_ee}
    del graph
    if rank == 0 and world == 1 and not args.no_extras:
        extras(args, w, s, mixed_res, dev, flush, out)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def extras(args, w, s, mixed_res, dev, flush, out):
    """Everything beside the main line (rank 0, one GPU).  The GPU sub-runs come first; the CPU
    oracle work runs afterwards in child processes (two at a time at most), so that host load does
    not disturb any GPU timing."""
    import numpy as np
    import torch
    tmp = tempfile.mkdtemp(prefix="cpm-bench-")
    wfile = os.path.join(tmp, "workload.pkl")
    with open(wfile, "wb") as f:
        pickle.dump(w, f)
    # charges, b and offsets of one charge update: the inputs of the oracle comparison
    s.charges()
    r = s.results()
    np.savez(os.path.join(tmp, "gpu.npz"), q=mixed_res["q"], F_elyt=mixed_res["F_elyt"], energy=mixed_res["energy"],
             q_c=r["q"][0], b_c=r["b"][0], psibar_c=r["psibar"][0])
    # ---- GPU: the same workload on the plain float64 path ----
    try:
        out["plain_fp64"], fp64_res = plain_fp64(args, w, s, dev, flush)
        prec = precision_errors(mixed_res, fp64_res)
    except Exception as e:                # the line is printed whatever this sub-run does
        out["plain_fp64"], prec = {"error": f"{type(e).__name__}: {e}"[:300]}, None
    torch.cuda.empty_cache()
    # ---- GPU: the paper-scale cell and the batched replicas ----
    paper_pending = None
    if args.workload == "dc-large":
        try:
            out["paper_cell"], paper_pending = paper_cell(args, dev, flush, tmp)
        except Exception as e:
            out["paper_cell"] = {"error": f"{type(e).__name__}: {e}"[:300]}
    torch.cuda.empty_cache()
    q_batched = None
    try:
        out["batched"], q_batched = batched_replicas(args, dev, flush)
    except Exception as e:
        out["batched"] = {"error": f"{type(e).__name__}: {e}"[:300]}
    torch.cuda.empty_cache()
    plain_pending = None
    if args.workload == "dc-large":
        try:
            out["plain_cell"], plain_pending = plain_cell(args, dev, flush, tmp)
        except Exception as e:
            out["plain_cell"] = {"error": f"{type(e).__name__}: {e}"[:300]}
    # ---- CPU: the oracle ----
    acc = {"vs_plain_fp64_gpu": prec}
    first = []
    if args.workload in DENSE_ORACLE:
        first.append(("oracle", spawn_child(args, "oracle-step", wfile, os.path.join(tmp, "oracle.npz"),
                                            batched=args.workload == "paper")))
    else:
        first.append(("accuracy", spawn_child(args, "accuracy-large", wfile, os.path.join(tmp, "acc.json"),
                                              os.path.join(tmp, "gpu.npz"))))
    if paper_pending is not None:
        a2, pwfile = paper_pending[2], paper_pending[3]
        first.append(("paper", spawn_child(a2, "oracle-step", pwfile, os.path.join(tmp, "paper_oracle.npz"),
                                           batched=True)))
    done = {name: finish_child(c) for name, c in first}
    if "oracle" in done:
        ok, ref = done["oracle"]
        if ok:
            acc["vs_oracle"] = accuracy_against(ref, mixed_res)
            out["cpu_baseline"] = ref["cpu_baseline"]
            if args.workload == "paper" and q_batched is not None and "q_batched" in ref:
                out["batched"]["accuracy"] = batched_accuracy(ref["q_batched"], q_batched)
                if "batched_step_s" in ref:
                    out["batched"]["cpu_baseline"] = batched_cpu_baseline(float(ref["batched_step_s"]),
                                                                          ref["cpu_baseline"].get("cores"))
        else:
            acc["vs_oracle"] = {"error": ref}
    if "accuracy" in done:
        ok, res = done["accuracy"]
        acc["vs_oracle"] = res if ok else {"error": res}
    out["accuracy"] = acc
    if paper_pending is not None:
        finish_paper_cell(out["paper_cell"], done["paper"], paper_pending[1], out.get("batched"), q_batched,
                          paper_pending[4])
    if plain_pending is not None:
        try:
            finish_plain_cell(out["plain_cell"], plain_pending[0], plain_pending[1], tmp)
        except Exception as e:
            out["plain_cell"]["accuracy"] = {"error": f"{type(e).__name__}: {e}"[:300]}
    if not args.no_cpu_baseline and args.workload not in DENSE_ORACLE:
        ok, res = finish_child(spawn_child(args, "oracle-sample", wfile, os.path.join(tmp, "cpu_all.json"),
                                           cores=os.cpu_count() or 1))
        base = res if ok else {"value": None, "unit": "ns/day", "kind": "oracle", "error": res}
        ok1, res1 = finish_child(spawn_child(args, "oracle-sample", wfile, os.path.join(tmp, "cpu_1.json"), cores=1))
        base["one_core"] = res1 if ok1 else {"error": res1}
        out["cpu_baseline"] = base


def plain_fp64(args, w, s_mixed, dev, flush):
    """The same workload and mesh on the float64 path: S from the mixed context's matrix image
    (no second assembly and factorisation of A), the float64 kernels, the same graph timing."""
    import torch
    import paper_2201_12963_gb300 as g
    t0 = time.perf_counter()
    image = g.cpm_matrix_image(s_mixed.ctx)
    s, build_s, _ = build_system(args, w, dev, precision="fp64", image=image, tune=False)
    del image
    graph = capture_step(s, True, dev)
    K = min(args.steps, 100)
    tot, _, _ = time_replays(graph, flush, K, dev, 3)
    res = step_results(s, True)
    st = g.cpm_status(s.ctx)
    ms = tot / K
    obj = {"ms_per_step": round(ms, 5), "value": round(1e3 / ms * NS_PER_DAY_PER_STEP_PER_S, 3), "unit": "ns/day",
           "steps": K, "status": st, "build_from_image_s": round(time.perf_counter() - t0, 2),
           "note": "float64 pair, mesh, S-apply and energies; same mesh and kernels' structure, default variants"}
    del graph, s
    return obj, res


def spawn_child(args, mode, wfile, out_path, in_path=None, cores=None, batched=False):
    """Start `bench.py --child mode` (CPU oracle work) in the background; batched: the oracle step
    child also solves the batched replicas' charges (untimed)."""
    cmd = [sys.executable, os.path.abspath(__file__), "--child", mode, "--workload", args.workload,
           "--seed", str(args.seed), "--workload-file", wfile, "--child-out", out_path]
    if in_path:
        cmd += ["--child-in", in_path]
    env = dict(os.environ)
    env["CUDA_VISIBLE_DEVICES"] = ""            # host work only
    if cores is not None:
        n = str(cores)
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
            env[k] = n
        env["CPM_ORACLE_PROCS"] = n
    if batched:
        env["CPM_BENCH_BATCHED"] = "1"
    p = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env)
    return p, out_path


def finish_child(child, timeout=900):
    """(ok, result): a child's output file, or its error."""
    p, out_path = child
    try:
        so, se = p.communicate(timeout=timeout)
    except subprocess.TimeoutExpired:
        p.kill()
        return False, "timed out"
    if p.returncode != 0 or not os.path.exists(out_path):
        return False, (se or so or f"exit {p.returncode}")[-300:]
    if out_path.endswith(".npz"):
        import numpy as np
        with np.load(out_path, allow_pickle=False) as z:
            ref = {k: z[k] for k in z.files}
        ref["cpu_baseline"] = json.loads(str(ref.pop("cpu_baseline_json")))
        return True, ref
    with open(out_path) as f:
        return True, json.load(f)


def paper_cell(args, dev, flush, tmp):
    """The paper-scale finite-field cell (3,024 sites) beside the default workload: mixed step
    timing with its rooflines and the float64 path; the oracle step (one full FP64 step, also the
    batched replicas' charges) runs later in a child, and finish_paper_cell adds its results."""
    import torch
    import paper_2201_12963_gb300 as g
    a2 = argparse.Namespace(**vars(args))
    a2.workload, a2.seed = "paper", WORKLOADS["paper"][1]
    w = workload(a2.seed, "paper")
    wfile = os.path.join(tmp, "paper.pkl")
    with open(wfile, "wb") as f:
        pickle.dump(w, f)
    s, build_s, (sv, fv, mv) = build_system(a2, w, dev)
    s.sapply_variant = sv
    graph = capture_step(s, True, dev)
    K = min(args.steps, 500)
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    tot, _, _ = time_replays(graph, flush, K, dev, 3, 1, clocks)
    clk = clocks.stop()
    mixed_res = step_results(s, True)
    st = g.cpm_status(s.ctx)
    graph_fe = capture_step(s, False, dev)
    tot_fe, _, _ = time_replays(graph_fe, flush, K, dev, 3)
    del graph_fe
    phase_ms = profile_phases(s, flush, min(K, 50), True)
    roof, roof_s, roof_pair, roof_ee = roofline("paper", s, w, phase_ms, clk)
    ms = tot / K
    obj = {"workload": WORKLOADS["paper"][0], "precision": a2.precision, "ms_per_step": round(ms, 5),
           "value": round(1e3 / ms * NS_PER_DAY_PER_STEP_PER_S, 2), "unit": "ns/day", "steps": K, "status": st,
           "frozen_electrode_ms_per_step": round(tot_fe / K, 5),
           "kernels": {"s_apply": sv, "transform": fv, "assignment": mv, "pair": g.cpm_get_pair_variant(s.ctx),
                       "pair_group_z": g.cpm_get_pair_group(s.ctx)},
           "phase_ms": {k: round(v, 5) for k, v in phase_ms.items()},
           "roofline": roof, "roofline_s_apply": roof_s, "roofline_pair_elyt": roof_pair,
           "roofline_pair_list": roof_ee, "clocks": clk}
    del graph
    fp64_res = None
    try:
        obj["plain_fp64"], fp64_res = plain_fp64(a2, w, s, dev, flush)
        obj["accuracy"] = {"vs_plain_fp64_gpu": precision_errors(mixed_res, fp64_res)}
    except Exception as e:
        obj["plain_fp64"] = {"error": f"{type(e).__name__}: {e}"[:300]}
        obj["accuracy"] = {}
    return obj, (None, mixed_res, a2, wfile, fp64_res)


def finish_paper_cell(obj, done, mixed_res, batched_obj, q_batched, fp64_res=None):
    """The paper cell's oracle comparison (the timed mixed step, and the float64 GPU path on the
    same mesh: the mesh's own error) and CPU time, and the batched replicas' accuracy."""
    ok, ref = done
    if not ok:
        obj["accuracy"]["vs_oracle"] = {"error": ref}
        return
    obj["accuracy"]["vs_oracle"] = accuracy_against(ref, mixed_res)
    if fp64_res is not None:
        obj["accuracy"]["plain_fp64_vs_oracle"] = accuracy_against(ref, fp64_res)
    obj["cpu_baseline"] = ref["cpu_baseline"]
    if batched_obj is not None and q_batched is not None and "q_batched" in ref:
        try:
            batched_obj["accuracy"] = batched_accuracy(ref["q_batched"], q_batched)
        except Exception as e:
            batched_obj["accuracy"] = {"error": f"{type(e).__name__}: {e}"[:300]}
    if batched_obj is not None and "batched_step_s" in ref:
        try:
            batched_obj["cpu_baseline"] = batched_cpu_baseline(float(ref["batched_step_s"]),
                                                               ref["cpu_baseline"].get("cores"))
        except Exception as e:
            batched_obj["cpu_baseline"] = {"error": f"{type(e).__name__}: {e}"[:300]}


def graph_step_ms(s, flush, steps, dev, elec=True):
    """Mean CUDA-event time per replay of one captured cpm_step, L2 flushed before every replay."""
    graph = capture_step(s, elec, dev)
    tot, _, _ = time_replays(graph, flush, steps, dev, 3)
    return tot / steps


def batched_replicas(args, dev, flush):
    """Replica throughput: 64 replicas of the 672-site plain cell (400-600 point-ion pairs each,
    dpsi 0-4 V) in one batched step (mixed precision, tensor-core S-apply), against the plain
    float64 path stepping one replica of the same cell.  Returns the line's object and the
    batched step's charges [64, 672]."""
    import synth
    import paper_2201_12963_gb300 as g
    from paper_2201_12963_gb300.driver import System
    steps = max(10, min(args.steps, 200))
    wb = synth.config_batched(n_rep=64)
    sb = System(wb, "mixed", device=dev)
    ms_b = graph_step_ms(sb, flush, steps, dev)
    st = g.cpm_status(sb.ctx)
    q_b = sb.results()["q"]
    phase_ms = profile_phases(sb, flush, 20, True)
    peaks = load_peaks()
    ne, R = sb.ne, 64
    flops = 2 * 3 * ne * ne * R                   # three tf32 products (hi.hi + hi.lo + lo.hi) of S Y
    t_s = phase_ms.get("s_apply")
    peak = float(peaks.get("bf16_tflops", 1900.0)) * TF32_OVER_BF16
    roof = None
    if t_s:
        ach = flops / (t_s / 1e3) / 1e12
        roof = {"bound": "tensor", "kernel": "s_apply (k_sapply_tc + float64 epilogue)", "achieved": round(ach, 3),
                "peak": round(peak, 1), "unit": "TFLOP/s", "frac": round(ach / peak, 5), "traffic": None,
                "algorithmic_per_launch": flops, "launch_ms": round(t_s, 5),
                "peak_source": "measured bf16 burst (MEASURED_PEAKS.json) x nominal tf32/bf16 ratio 1.1/2.25",
                "model": f"2 x 3 x {ne} x {ne} x {R} flops (split-TF32: three products)"}
    w1 = wb.replica(0)
    s1 = System(w1, "fp64", device=dev)
    ms_1 = graph_step_ms(s1, flush, steps, dev)
    return {"workload": "64 replicas x 672-site plain cell (17.04x17.22x60 A), 400-600 point-ion pairs each, "
                        "mesh 18x18x60 order 5, forces on all sites",
            "replicas": 64, "precision": "mixed, tcgen05 split-TF32 S-apply",
            "ms_per_step": round(ms_b, 5), "replica_steps_per_s": round(64 * 1e3 / ms_b, 1),
            "plain_fp64_one_replica": {"ms_per_step": round(ms_1, 5), "steps_per_s": round(1e3 / ms_1, 1)},
            "speedup_replica_steps": round((64 / ms_b) / (1 / ms_1), 2), "status": st,
            "phase_ms": {k: round(v, 5) for k, v in phase_ms.items()}, "roofline": roof}, q_b


def plain_cell(args, dev, flush, tmp):
    """The 672-site plain finite-field cell (17.04 x 17.22 x 60 A, 100 + 100 point ions, dpsi 2 V,
    mesh 18 x 18 x 60 order 5) on the float64 path: one step with forces on all sites, timed as
    graph replays (latency-bound: its S is 3.6 MB).  Returns the object and (its results, the
    workload file for the oracle children)."""
    import synth
    import paper_2201_12963_gb300 as g
    from paper_2201_12963_gb300.driver import System
    w = synth.config_plain_ff()
    wfile = os.path.join(tmp, "plain.pkl")
    with open(wfile, "wb") as f:
        pickle.dump(w, f)
    s = System(w, "fp64", device=dev)
    steps = max(10, min(args.steps, 200))
    ms = graph_step_ms(s, flush, steps, dev)
    res = step_results(s, True)
    obj = {"workload": "672-site plain finite-field cell (17.04x17.22x60 A), 100 + 100 point ions "
                       "+-0.78 e, dpsi 2 V, mesh 18x18x60 order 5, forces on all sites",
           "precision": "fp64", "ms_per_step": round(ms, 5), "steps_per_s": round(1e3 / ms, 1),
           "value": round(NS_PER_DAY_PER_STEP_PER_S * 1e3 / ms, 2), "unit": "ns/day", "steps": steps,
           "status": g.cpm_status(s.ctx)}
    return obj, (res, wfile)


def finish_plain_cell(obj, res, wfile, tmp):
    """The plain cell's oracle comparison and the oracle's step time on all cores and on one core
    (one child after the other)."""
    a1 = argparse.Namespace(workload="paper", seed=WORKLOADS["paper"][1])
    ok, ref = finish_child(spawn_child(a1, "oracle-step", wfile, os.path.join(tmp, "plain_all.npz"),
                                       cores=os.cpu_count() or 1))
    if not ok:
        obj["accuracy"] = {"vs_oracle": {"error": ref}}
        return
    obj["accuracy"] = {"vs_oracle": accuracy_against(ref, res)}
    base = dict(ref["cpu_baseline"])
    ok1, ref1 = finish_child(spawn_child(a1, "oracle-step", wfile, os.path.join(tmp, "plain_1.npz"), cores=1))
    base["one_core"] = ref1["cpu_baseline"] if ok1 else {"error": ref1}
    if ok1:
        base["one_core"]["cores"] = 1
        base["one_core"]["sample"] = "the same oracle step with BLAS threads = 1"
    obj["cpu_baseline"] = base


def batched_oracle_charges(n_rep=64):
    """The oracle's charges [n_rep, 672] for every replica of the batched workload (one A and
    Cholesky factor for the shared electrode, one b and KKT solve per replica), and the time of
    one full oracle step of replica 0 (charges, full-Ewald energy and forces; seconds)."""
    import numpy as np
    import synth
    from oracle import cpm as ocpm
    wb = synth.config_batched(n_rep=n_rep)
    ref = ocpm.Reference(wb.replica(0))
    out = np.zeros((n_rep, wb.n_elec))
    for r in range(n_rep):
        out[r] = ref.charges(wb.elyt_xyz[r], wb.elyt_q[r], float(wb.dpsi[r]))[0]
    t0 = time.perf_counter()
    ref.step(0)
    return out, time.perf_counter() - t0


def batched_cpu_baseline(step_s, cores):
    """cpu_baseline of the batched line: the oracle steps independent replicas one after another,
    so its replica-steps/s is the inverse of one replica's full step."""
    return {"value": round(1.0 / step_s, 4), "unit": "replica-steps/s", "cores": cores, "kind": "oracle",
            "seconds_per_step": round(step_s, 3),
            "sample": "one full FP64 oracle step of replica 0 of the batched workload (672 sites: direct "
                      "Ewald b, KKT solve with a prebuilt Cholesky factor, full-Ewald energy and forces); "
                      "replicas are independent and the oracle runs them one after another; numpy, BLAS "
                      "threads = all cores, elementwise work single-threaded"}


def batched_accuracy(q_ref, q):
    """Per-replica max |dq| (e) of the batched step's charges against the oracle's."""
    import numpy as np
    q_ref = np.asarray(q_ref)
    q = np.asarray(q).reshape(q_ref.shape[0], -1)[:, : q_ref.shape[1]]
    dq = np.abs(q - q_ref).max(axis=1)
    return {"dq_max_e": float(dq.max()), "dq_max_e_per_replica": [float(f"{x:.3g}") for x in dq],
            "replicas_within_1e-5_e": int((dq <= 1e-5).sum()), "replicas": int(dq.size),
            "reference": "FP64 CPU oracle (direct Ewald b, KKT solve) per replica on the same input"}


def accuracy_against(ref, res):
    """Errors of one GPU step against the oracle's step on the same input: max |dq| (e), RMS
    relative force error on the electrolyte, relative error of U and of H."""
    import numpy as np
    q = np.asarray(res["q"]).reshape(-1)[: ref["q"].size]
    F = np.asarray(res["F_elyt"]).reshape(-1, 3)[: ref["F_elyt"].shape[0]]
    Fo = ref["F_elyt"]
    e = res["energy"]
    return {"dq_max_e": float(np.abs(q - ref["q"]).max()),
            "force_rms_rel": float(np.sqrt(((F - Fo) ** 2).sum() / (Fo ** 2).sum())),
            "energy_U_rel": float(abs(e[0] - ref["U"]) / abs(ref["U"])),
            "energy_H_rel": float(abs(e[1] - ref["H"]) / abs(ref["H"])),
            "reference": "FP64 CPU oracle (direct Ewald sums, dense KKT solve) on the same input"}


# ----------------------------------------------------------------------------------------------
# CPU oracle children
# ----------------------------------------------------------------------------------------------
def child_oracle_step(args):
    """One full oracle step (dense A and its Cholesky factor built first, untimed): its results
    and its time, as an .npz."""
    import numpy as np
    from oracle import cpm as ocpm
    w = load_workload(args)
    ref = ocpm.Reference(w)
    t0 = time.perf_counter()
    out = ref.step(0)
    dt = time.perf_counter() - t0
    extra = {}
    if os.environ.get("CPM_BENCH_BATCHED") == "1":        # untimed: the batched line's per-replica accuracy
        extra["q_batched"], extra["batched_step_s"] = batched_oracle_charges()
    base = {"value": round(NS_PER_DAY_PER_STEP_PER_S / dt, 6), "unit": "ns/day", "cores": os.cpu_count(),
            "kind": "oracle", "seconds_per_step": round(dt, 3),
            "sample": "one full FP64 oracle step (direct Ewald b, KKT solve with a prebuilt Cholesky factor, "
                      "full-Ewald energy and forces) of the workload; numpy, BLAS threads = all cores, "
                      "elementwise work single-threaded"}
    np.savez(args.child_out, q=out["q"], F_elyt=out["F_elyt"], U=out["U"], H=out["H"], psibar=out["psibar"],
             b=out["b"], cpu_baseline_json=json.dumps(base), **extra)


def child_accuracy_large(args):
    """The timed step of a workload too large for a dense oracle solve, against the oracle at
    sampled sites (reciprocal sums through the per-axis plane-wave tables): b at 64 electrode sites,
    electrolyte forces at 64 sites from the GPU's charges, and the KKT residual
    A q - b - dpsi v - C psibar at 256 electrode sites from the GPU's charges, b and offsets."""
    import numpy as np
    from oracle import cpm as ocpm
    w = load_workload(args)
    with np.load(args.child_in) as z:
        gpu = {k: z[k] for k in z.files}
    R, Q, dpsi = w.elyt_xyz[0], w.elyt_q[0], float(w.dpsi[0])
    rng = np.random.default_rng(7)
    ie = np.sort(rng.choice(w.n_elec, 64, replace=False))
    il = np.sort(rng.choice(len(Q), 64, replace=False))
    ik = np.sort(rng.choice(w.n_elec, 256, replace=False))
    t0 = time.perf_counter()
    b_ref = ocpm.b_at(w, R, Q, ie, kspace="separable")
    F_ref = ocpm.electrolyte_forces_at(w, R, Q, gpu["q"], dpsi, il, kspace="separable")
    Aq = ocpm.elastance_apply(w, gpu["q_c"], idx=ik, kspace="separable")
    C = ocpm.constraints(w)[ik]
    v = ocpm.geometry_vector(w)[ik]
    resid = Aq - gpu["b_c"][ik] - dpsi * v - C @ gpu["psibar_c"]
    fit = np.linalg.lstsq(C, resid, rcond=None)[0]
    F = gpu["F_elyt"][il]
    out = {"b_max_abs_V": float(np.abs(gpu["b_c"][ie] - b_ref).max()),
           "b_rms_V": float(np.sqrt(np.mean(gpu["b_c"] ** 2))),
           "b_max_rel_to_rms": float(np.abs(gpu["b_c"][ie] - b_ref).max() / np.sqrt(np.mean(gpu["b_c"] ** 2))),
           "force_rms_rel_elyt": float(np.sqrt(((F - F_ref) ** 2).sum() / (F_ref ** 2).sum())),
           "kkt_residual_max_V": float(np.abs(resid).max()),
           "kkt_residual_offset_fit_V": [float(x) for x in fit],
           "kkt_residual_after_offsets_max_V": float(np.abs(resid - C @ fit).max()),
           "sites": {"b": 64, "forces": 64, "kkt": 256}, "seconds": round(time.perf_counter() - t0, 1),
           "reference": "FP64 oracle at sampled sites: direct real-space sums and the direct reciprocal sum "
                        "(per-axis plane-wave tables, pinned to the cos/sin sum), alpha 0.25, r_c 12 A; the "
                        "GPU's A is the mesh operator of its own SPME (the direct sum is out of reach at this "
                        "size), so the residual also carries the mesh error of A; the full Ewald energy at this "
                        "size is not evaluated (all-pairs real-space sums over 1.4e5 sites)"}
    with open(args.child_out, "w") as f:
        json.dump(out, f)


def _sample_worker(payload):
    """One sampled oracle step in a worker process: (seconds)."""
    wfile, frac, seed = payload
    import numpy as np
    from oracle import cpm as ocpm
    with open(wfile, "rb") as f:
        w = pickle.load(f)
    q = np.zeros(w.n_elec)
    t0 = time.perf_counter()
    ocpm.sampled_step_sums(w, w.elyt_xyz[0], w.elyt_q[0], frac, seed, q=q)
    return time.perf_counter() - t0


class SampledOracle:
    """The oracle's per-step sums of a workload too large for its dense A (b, energies and forces
    at given electrode charges; the KKT solve is left out because A cannot be formed), run as
    bounded samples (a fraction f of the real-space targets and of the k-vectors) on `procs`
    worker processes at once.  With every worker taking fraction f, a sample costs
    T(f) = a + b f; a full step on `procs` cores, one worker per 1/procs of the work, costs
    a + b / procs."""

    def __init__(self, wfile, procs):
        import multiprocessing as mp
        self.wfile, self.procs = wfile, max(1, procs)
        self.pool = mp.get_context("spawn").Pool(self.procs) if self.procs > 1 else None
        self.seed = 0

    def sample(self, frac):
        self.seed += self.procs
        jobs = [(self.wfile, frac, self.seed + k) for k in range(self.procs)]
        t0 = time.perf_counter()
        if self.pool is None:
            _sample_worker(jobs[0])
        else:
            self.pool.map(_sample_worker, jobs)
        return time.perf_counter() - t0

    def fit(self, f1, f2):
        t1, t2 = self.sample(f1), self.sample(f2)
        b = max(1e-9, (t2 - t1) / (f2 - f1))
        return max(0.0, t1 - b * f1), b

    def calibrate(self, work_s=10.0):
        """(a, b, fractions, times): two short samples for a first T(f), a third whose f-part is
        about work_s seconds, and the least-squares line through the three."""
        import numpy as np
        fs = [2e-5, 8e-5]
        ts = [self.sample(f) for f in fs]
        b0 = max(1e-9, (ts[1] - ts[0]) / (fs[1] - fs[0]))
        fs.append(min(0.5, work_s / b0))
        ts.append(self.sample(fs[2]))
        b, a = np.polyfit(fs, ts, 1)
        return max(0.0, float(a)), max(1e-9, float(b)), fs, ts

    def close(self):
        if self.pool is not None:
            self.pool.close()
            self.pool.join()


def oracle_procs():
    """Worker processes for the sampled oracle: the cores asked for, bounded by host memory
    (about 3 GB per worker at 10^5 sources)."""
    want = int(os.environ.get("CPM_ORACLE_PROCS", str(os.cpu_count() or 1)))
    try:
        mem_gb = os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES") / 2 ** 30
        want = min(want, max(1, int(mem_gb // 6)))
    except (ValueError, OSError):
        pass
    return max(1, want)


def child_oracle_sample(args):
    """cpu_baseline of a large workload: the sampled oracle on the cores given (one worker each),
    scaled to a full step through the two-point fit."""
    procs = oracle_procs()
    so = SampledOracle(args.workload_file, procs)
    try:
        a, b, fs, ts = so.calibrate()
        t_full = a + b / procs
    finally:
        so.close()
    w = load_workload(args)
    base = {"value": round(NS_PER_DAY_PER_STEP_PER_S / t_full, 8), "unit": "ns/day", "cores": procs,
            "kind": "oracle", "seconds_per_step": round(t_full, 1),
            "sample": (f"{procs} worker process(es), one core each (BLAS threads {os.environ.get('OMP_NUM_THREADS', 'default')}); "
                       f"each sample restricts every real-space sum to a random fraction f of its target sites and "
                       f"every reciprocal sum to a fraction f of the k-vectors, all workers at once; samples at "
                       f"f = {', '.join(f'{x:.2e}' for x in fs)} ({', '.join(f'{x:.1f}' for x in ts)} s) give "
                       f"T(f) = {a:.2f} s + {b:.0f} s x f; a full step is "
                       f"a + b/{procs}. The KKT solve is not included: the oracle's dense A for "
                       f"{w.n_elec:,} sites cannot be formed on the host (its reciprocal part alone is "
                       f"~10^16 flops), so the electrode charges are held fixed")}
    with open(args.child_out, "w") as f:
        json.dump(base, f)


def run_batched(args):
    """--workload batched: the 64-replica step as the line itself (replica-steps/s), for profiling and
    for a batched-only run; the default line carries the same object as `batched`."""
    import torch
    import torch.distributed as dist
    world, rank, local, dev = setup_ranks()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    clocks = ClockSampler(local)
    clocks.start()
    obj, _ = batched_replicas(args, dev, flush)
    clk = clocks.stop()
    ms = reduce_max(obj["ms_per_step"], dev)
    value = world * 64 * 1e3 / ms
    out = {"metric": METRIC, "value": round(value, 1), "unit": "replica-steps/s", "n_gpus": world,
           "steps": max(10, min(args.steps, 200)), "warmup": 3, "ms_per_step": round(ms, 5), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": WORKLOADS["batched"][0], "geometry": "finite field", "precision": "mixed",
                      "forces": "all sites (electrolyte and electrode)", "replicas_per_gpu": 64,
                      "parallelism": f"replicas x{world} (no collective)",
                      "l2": "flushed between steps (256 MiB write); per-step CUDA-event time",
                      "graph": "whole step captured in one CUDA graph"},
           "clocks": clk, "batched": obj, "roofline": obj.get("roofline")}
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
    s.sapply_variant = sapply_variant
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
    roof, roof_s, roof_pair, roof_ee = roofline(args.workload, s, w, phase_ms, clk)

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
           "roofline": roof, "roofline_s_apply": roof_s, "roofline_pair_elyt": roof_pair}
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.no_extras:
        tmp = tempfile.mkdtemp(prefix="cpm-bench-")
        wfile = os.path.join(tmp, "workload.pkl")
        with open(wfile, "wb") as f:
            pickle.dump(w, f)
        ok, ref = finish_child(spawn_child(args, "oracle-step", wfile, os.path.join(tmp, "oracle.npz")))
        if ok:
            base = ref["cpu_baseline"]
            base["sample"] += ("; for the MD workload this is the charge re-solve step, an upper bound of the "
                               "oracle's MD step (its Lennard-Jones and integration cost are not added)")
            out["cpu_baseline"] = base
        else:
            out["cpu_baseline"] = {"value": None, "unit": "ns/day", "kind": "oracle", "error": ref}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()



# ----------------------------------------------------------------------------------------------
# the reference arm: the FP64 oracle on the host's cores
# ----------------------------------------------------------------------------------------------
def run_reference(args):
    """The oracle timed on this host, on the GPU arm's workload, metric and unit.  Workloads with
    a dense oracle: one full step (its A and Cholesky factor built first, untimed) gives the value,
    and each timed step is a bounded sample of it (a random fraction f of the real-space targets
    and of the k-vectors, KKT solve in full).  Larger workloads: the sampled oracle on all cores
    (SampledOracle), the value from its two-point fit, each timed step one sample of it.
    ms_per_step is the measured time of the timed (sampled) steps."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    from oracle import cpm as ocpm
    w = workload(args.seed, args.workload)
    K, W = max(1, args.steps), max(0, args.warmup)
    budget = 120.0                                     # seconds for the warm-up and timed samples
    if args.workload in DENSE_ORACLE:
        ref = ocpm.Reference(w)
        t0 = time.perf_counter()
        ref.step(0)
        t_full = time.perf_counter() - t0
        procs = os.cpu_count() or 1
        sampler = lambda f, seed: ref.sampled_step(0, f, seed)   # noqa: E731
        f_step = min(1.0, max(1e-4, budget / (K + W) / t_full))
        how = (f"value: one full FP64 oracle step ({t_full:.2f} s: direct Ewald b, KKT solve with a prebuilt "
               f"Cholesky factor, full-Ewald energy and forces; numpy, BLAS threads = all cores, elementwise work "
               f"single-threaded); each timed step: a sample with a random fraction f = {f_step:.4f} of the "
               f"real-space targets and of the k-vectors, KKT solve in full")
        so = None
    else:
        tmp = tempfile.mkdtemp(prefix="cpm-ref-")
        wfile = os.path.join(tmp, "workload.pkl")
        with open(wfile, "wb") as f:
            pickle.dump(w, f)
        procs = oracle_procs()
        so = SampledOracle(wfile, procs)
        a, b, fs, ts = so.calibrate()
        t_full = a + b / procs
        f_step = max(1e-7, (budget / (K + W) - a) / b)
        sampler = lambda f, seed: so.sample(f)       # noqa: E731
        how = (f"value: {procs} worker processes (one core each) of the oracle's per-step sums, samples at "
               f"f = {', '.join(f'{x:.2e}' for x in fs)} (a random fraction f of the real-space targets and of the "
               f"k-vectors per worker) fit T(f) = {a:.2f} s + {b:.0f} s x f, full step = a + b/{procs}; the KKT "
               f"solve is left out (the dense A for {w.n_elec:,} sites cannot be formed on the host); each "
               f"timed step: one sample at f = {f_step:.2e}")
    for k in range(W):
        sampler(f_step, 10 + k)
    ts = []
    for k in range(K):
        t = time.perf_counter()
        sampler(f_step, 1000 + k)
        ts.append(time.perf_counter() - t)
    if so is not None:
        so.close()
    value = NS_PER_DAY_PER_STEP_PER_S / t_full
    ms_sample = 1e3 * sum(ts) / len(ts)
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 8), "unit": "ns/day", "n_gpus": world,
           "steps": K, "warmup": W, "ms_per_step": round(ms_sample, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOADS[args.workload][0], "geometry": GEOMETRY_NAME[args.workload],
                      "precision": "fp64 oracle", "full_step_ms": round(t_full * 1e3, 1),
                      "ms_per_step_is": "the measured time of the timed sampled steps"},
           "cpu_baseline": {"value": round(value, 8), "unit": "ns/day", "cores": procs, "kind": "oracle",
                            "sample": how},
           "e2e": {"value": round(value, 8), "unit": "ns/day", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.seed is None:
        args.seed = WORKLOADS[args.workload][1]
    if args.child == "oracle-step":
        child_oracle_step(args)
    elif args.child == "accuracy-large":
        child_accuracy_large(args)
    elif args.child == "oracle-sample":
        child_oracle_sample(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gb300(args)


if __name__ == "__main__":
    main()
