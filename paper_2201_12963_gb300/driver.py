"""Convenience wrapper: run a whole system description through the C ABI.

`System` holds device copies of one electrolyte batch and the output buffers, and calls the entry
points of the library; no arithmetic happens here.  The system description is any object with the
attributes box, eta, alpha, rcut, grid, order, geometry, slab_factor, elec_xyz, elec_side,
elec_cell, elyt_xyz (list per replica), elyt_q (list per replica) and dpsi (per replica).
"""
from __future__ import annotations

import numpy as np
import torch

import os

from . import (CPMError, Context, cpm_build_matrix, cpm_build_matrix_from_image, cpm_energy, cpm_forces,
               cpm_matrix_image, cpm_matrix_key, cpm_step, cpm_step_charges, make_params)


def params_for(w, precision="fp64", grid=None, order=None, max_replicas=None, max_elyt=None, kmax_build=0.0,
               matrix_kspace="ewald", dc_blocks="auto"):
    counts = [len(q) for q in w.elyt_q]
    return make_params(w.box, w.eta, w.alpha, w.rcut, grid or w.grid, order or w.order, w.geometry, precision,
                       max_replicas=max_replicas or max(1, len(counts)),
                       max_elyt=max_elyt or max(1, max(counts) if counts else 1),
                       slab_factor=w.slab_factor, kmax_build=kmax_build, matrix_kspace=matrix_kspace,
                       dc_blocks=dc_blocks)


def pack(w):
    """Replica-major (offsets [R+1] int32, xyzq [N,4] float64) host arrays."""
    counts = [len(q) for q in w.elyt_q]
    offsets = np.zeros(len(counts) + 1, dtype=np.int32)
    offsets[1:] = np.cumsum(counts)
    xyzq = np.zeros((max(1, int(offsets[-1])), 4), dtype=np.float64)   # >= 1 row: never a null pointer
    for r in range(len(counts)):
        xyzq[offsets[r]:offsets[r + 1], :3] = w.elyt_xyz[r]
        xyzq[offsets[r]:offsets[r + 1], 3] = w.elyt_q[r]
    return offsets, xyzq


def build_context(params, w, cache_dir=None):
    """cpm_build_matrix, or, with cache_dir, a context from the matrix image cached there under the
    key of its inputs (written after a fresh build; an image the library refuses is rebuilt)."""
    if cache_dir is None:
        return cpm_build_matrix(params, w.elec_xyz, w.elec_side, w.elec_cell), False
    key = cpm_matrix_key(params, w.elec_xyz, w.elec_side, w.elec_cell)
    path = os.path.join(cache_dir, f"cpm-matrix-{key:016x}.img")
    if os.path.exists(path):
        try:
            with open(path, "rb") as f:
                image = np.frombuffer(f.read(), dtype=np.uint8)
            return cpm_build_matrix_from_image(params, w.elec_xyz, w.elec_side, w.elec_cell, image), True
        except CPMError:
            pass
    ctx = cpm_build_matrix(params, w.elec_xyz, w.elec_side, w.elec_cell)
    os.makedirs(cache_dir, exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "wb") as f:
        f.write(cpm_matrix_image(ctx).tobytes())
    os.replace(tmp, path)
    return ctx, False


class System:
    def __init__(self, w, precision="fp64", grid=None, order=None, device="cuda", kmax_build=0.0,
                 max_replicas=None, max_elyt=None, matrix_kspace="ewald", dc_blocks="auto", cache_dir=None,
                 image=None):
        """image: a matrix image (cpm_matrix_image of a context with the same electrode and build
        parameters, of either precision) to build from instead of assembling and factorising A."""
        self.w = w
        self.device = torch.device(device)
        self.params = params_for(w, precision, grid, order, max_replicas, max_elyt, kmax_build, matrix_kspace,
                                 dc_blocks)
        with torch.cuda.device(self.device):
            if image is not None:
                self.ctx = cpm_build_matrix_from_image(self.params, w.elec_xyz, w.elec_side, w.elec_cell, image)
                self.from_cache = True
            else:
                self.ctx, self.from_cache = build_context(self.params, w, cache_dir)
        self.ne = self.ctx.n_elec
        self.load(w)

    def load(self, w):
        """Copy a (new) electrolyte batch to the device and size the outputs."""
        off, xyzq = pack(w)
        d = self.device
        self.n_rep = len(w.elyt_q)
        self.offsets = torch.from_numpy(off).to(d)
        self.xyzq = torch.from_numpy(xyzq).to(d)
        self.dpsi = torch.as_tensor(np.asarray(w.dpsi, dtype=np.float64)).to(d)
        n = int(off[-1])
        f64 = dict(dtype=torch.float64, device=d)
        self.q = torch.zeros(self.n_rep * self.ne, **f64)
        self.b = torch.zeros(self.n_rep * self.ne, **f64)
        self.psibar = torch.zeros(self.n_rep * self.ctx.ncons, **f64)
        self.f_elyt = torch.zeros(max(1, n) * 3, **f64)
        self.f_elec = torch.zeros(self.n_rep * self.ne * 3, **f64)
        self.energy = torch.zeros(4 * self.n_rep, **f64)       # U, H, dH/d(dpsi), Q_+ per replica

    def charges(self):
        cpm_step_charges(self.ctx, self.n_rep, self.offsets, self.xyzq, self.dpsi, self.q, self.b, self.psibar)

    def forces(self, elec=True, energy=True):
        cpm_forces(self.ctx, self.n_rep, self.offsets, self.xyzq, self.dpsi, self.q, self.f_elyt,
                   self.f_elec if elec else None, self.energy if energy else None)

    def energies(self):
        cpm_energy(self.ctx, self.n_rep, self.offsets, self.xyzq, self.dpsi, self.q, self.energy)

    def step(self, elec=False, energy=True):
        cpm_step(self.ctx, self.n_rep, self.offsets, self.xyzq, self.dpsi, self.q, self.psibar, self.f_elyt,
                 self.f_elec if elec else None, self.energy if energy else None)

    def results(self) -> dict:
        torch.cuda.synchronize(self.device)
        R, ne = self.n_rep, self.ne
        off = self.offsets.cpu().numpy()
        fl = self.f_elyt.cpu().numpy()[: 3 * int(off[-1])].reshape(-1, 3)
        return {"q": self.q.cpu().numpy().reshape(R, ne), "b": self.b.cpu().numpy().reshape(R, ne),
                "psibar": self.psibar.cpu().numpy().reshape(R, -1),
                "F_elyt": [fl[off[r]:off[r + 1]] for r in range(R)],
                "F_elec": self.f_elec.cpu().numpy().reshape(R, ne, 3),
                "energy": self.energy.cpu().numpy().reshape(R, 4)}


class MD:
    """The MD loop of a System through cpm_md_*: velocities, energies and forces on the device,
    positions and charges in the System's buffers.  `inputs` is one synth.MDInputs-like object per
    replica (types, groups, vel, mass, sigma, eps, elec_type, temperature, t_damp)."""

    def __init__(self, system: System, inputs, dt=2.0, charge_every=5, lj_cut=None, t_damp=None,
                 temperature=None, n_groups=None):
        from . import cpm_md_create, make_md_params
        self.s = system
        inputs = list(inputs) if isinstance(inputs, (list, tuple)) else [inputs]
        if len(inputs) != system.n_rep:
            raise ValueError("one MD input per replica required")
        mi = inputs[0]
        types = np.concatenate([np.asarray(m.types, np.int32) for m in inputs])
        groups = np.concatenate([np.asarray(m.groups, np.int32) for m in inputs])
        vel = np.concatenate([np.asarray(m.vel, np.float64).reshape(-1, 3) for m in inputs])
        self.n_groups = int(n_groups or (groups.max() + 1 if groups.size else 1))
        self.params = make_md_params(dt=dt, charge_every=charge_every, mass=mi.mass, sigma=mi.sigma, eps=mi.eps,
                                     elec_type=mi.elec_type, n_groups=self.n_groups,
                                     lj_cut=system.w.rcut if lj_cut is None else lj_cut,
                                     temperature=mi.temperature if temperature is None else temperature,
                                     t_damp=mi.t_damp if t_damp is None else t_damp)
        off = system.offsets.cpu().numpy()
        with torch.cuda.device(system.device):
            self.md = cpm_md_create(system.ctx, self.params, off, types, groups)
        f64 = dict(dtype=torch.float64, device=system.device)
        n = int(off[-1])
        self.vel = torch.from_numpy(vel.reshape(-1)).to(system.device) if n else torch.zeros(3, **f64)
        self.energy = torch.zeros(8 * system.n_rep, **f64)
        self.force = torch.zeros(max(1, n) * 3, **f64)

    def run(self, n_steps, energy=True, force=False, stream=None):
        from . import cpm_md_run
        s = self.s
        cpm_md_run(self.md, n_steps, s.xyzq, self.vel, s.dpsi, s.q, s.psibar, self.energy if energy else None,
                   self.force if force else None, stream=stream)

    def energies(self) -> list:
        """Per replica {U, H, U_lj, KE, E_nh, E_total, T, Q_plus} of the last run with energy=True."""
        from . import MD_ENERGY_KEYS
        e = self.energy.cpu().numpy().reshape(-1, 8)
        return [dict(zip(MD_ENERGY_KEYS, map(float, row))) for row in e]

    def checkpoint(self) -> dict:
        """Everything needed to continue the trajectory (host copies)."""
        from . import cpm_md_get_state
        step, thermo = cpm_md_get_state(self.md)
        s = self.s
        return {"step": step, "thermo": thermo, "xyzq": s.xyzq.cpu().numpy().copy(), "vel": self.vel.cpu().numpy().copy(),
                "q": s.q.cpu().numpy().copy()}

    def restore(self, ck: dict):
        from . import cpm_md_set_state
        s = self.s
        s.xyzq.copy_(torch.from_numpy(ck["xyzq"]))
        self.vel.copy_(torch.from_numpy(ck["vel"]))
        s.q.copy_(torch.from_numpy(ck["q"]))
        torch.cuda.synchronize(s.device)
        cpm_md_set_state(self.md, ck["step"], ck["thermo"])

    def tune(self, flush_bytes=256 << 20, replays=5):
        """Choose the real-space pair-kernel form and z group for this MD loop (the step autotuner
        times a charge re-solve without the Lennard-Jones term; here most steps keep their
        charges): graph replays of one charge_every-step block per candidate, a buffer larger than
        L2 written before each, median of `replays`.  Returns (variant, z group)."""
        from . import cpm_md_advance, cpm_set_pair_group, cpm_set_pair_variant
        k = self.params.charge_every
        flush = torch.empty(flush_bytes, dtype=torch.uint8, device=self.s.device)
        best = None
        for pv, gz in (("cell", 1), ("cell", 2), ("warp-elyt", 1), ("warp", 1)):
            cpm_set_pair_variant(self.s.ctx, pv)
            cpm_set_pair_group(self.s.ctx, gz)
            replay = self.capture(k, energy=False)
            replay(2)
            ts = []
            for _ in range(replays):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                replay.graph.replay()
                e1.record()
                torch.cuda.synchronize(self.s.device)
                ts.append(e0.elapsed_time(e1))
            cpm_md_advance(self.md, replays * k)
            med = sorted(ts)[len(ts) // 2]
            if best is None or med < best[0]:
                best = (med, pv, gz)
        cpm_set_pair_variant(self.s.ctx, best[1])
        cpm_set_pair_group(self.s.ctx, best[2])
        return best[1], best[2]

    def capture(self, n_steps, energy=False):
        """A CUDA graph of one cpm_md_run of n_steps (capture on a side stream).  Replaying it
        advances n_steps; call `replay` to keep the library's step index in step."""
        from . import cpm_md_advance
        st = torch.cuda.Stream(self.s.device)
        st.wait_stream(torch.cuda.current_stream(self.s.device))
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(st):
            with torch.cuda.graph(g, stream=st):
                self.run(n_steps, energy=energy, stream=st)
        torch.cuda.current_stream(self.s.device).wait_stream(st)

        def replay(times=1):
            for _ in range(times):
                g.replay()
            cpm_md_advance(self.md, n_steps * times)
        replay.graph = g
        return replay
