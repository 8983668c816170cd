"""Convenience wrapper: run a whole system description through the C ABI.

`System` holds device copies of one electrolyte batch and the output buffers, and calls the entry
points of the library; no arithmetic happens here.  The system description is any object with the
attributes box, eta, alpha, rcut, grid, order, geometry, slab_factor, elec_xyz, elec_side,
elec_cell, elyt_xyz (list per replica), elyt_q (list per replica) and dpsi (per replica).
"""
from __future__ import annotations

import numpy as np
import torch

from . import (Context, cpm_build_matrix, cpm_energy, cpm_forces, cpm_step, cpm_step_charges, make_params)


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


class System:
    def __init__(self, w, precision="fp64", grid=None, order=None, device="cuda", kmax_build=0.0,
                 max_replicas=None, max_elyt=None, matrix_kspace="ewald", dc_blocks="auto"):
        self.w = w
        self.device = torch.device(device)
        self.params = params_for(w, precision, grid, order, max_replicas, max_elyt, kmax_build, matrix_kspace,
                                 dc_blocks)
        with torch.cuda.device(self.device):
            self.ctx: Context = cpm_build_matrix(self.params, w.elec_xyz, w.elec_side, w.elec_cell)
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
