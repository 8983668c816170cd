"""The 10,080-site differentiation workload over its 50 seeded configurations (GPU).

One electrode (15 x 28 graphene cells x 3 layers x 2, 63.90 x 68.88 x 154 A) and one float64 and
one mixed-precision context, built once; the 50 electrolytes (5,000 point-ion pairs each, seeds
4000-4049) are loaded in turn.  alpha 0.45 / A and r_c 13.5 A keep the truncated real-space sum
smooth (erfc(alpha r_c) ~ 1e-17), A's reciprocal part is the mesh operator (H is then the exact
minimum of the discrete energy), SPME order 8 on the 1 A mesh.  For every configuration:

* the mixed path against float64: |dq| <= 1e-5 e per site, RMS force error <= 1e-5 on the
  electrolyte and on the electrode sites, the energy within the float32 rounding of its mesh
  transform (3e-7 of the charges' mesh self-energy, about 1e-5 of H);
* the autograd gradient (-forces, from cpm_forces) against the forces of the step.

On every tenth configuration also: central finite differences of the float64 energy (h = 1e-4 A at
12 sampled coordinates, h = 1e-3 V for dH/d dpsi and dQ_+/d dpsi), and the oracle's gradient at 32
sampled electrolyte sites (direct Ewald sums at the GPU's charges, reciprocal part through the
per-axis plane-wave tables).  The oracle's dense A at this size is out of reach on the host, so
its gradient is evaluated at the GPU's float64 charges; the difference is then the mesh error of
the forces.
"""
import dataclasses
import multiprocessing as mp
import os

import numpy as np
import pytest

import synth
from oracle import cpm as ocpm

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SEEDS = list(range(4000, 4050))


def _rms_rel(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))


def test_fifty_seeded_configurations():
    # the electrolytes first, drawn in spawned workers (no process is forked once CUDA is up; the
    # workers import only synth)
    with mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1))) as pool:
        elyts = [(w.elyt_xyz[0], w.elyt_q[0]) for w in pool.map(synth.config_large_ff, SEEDS)]
    import __graft_entry__
    __graft_entry__.build()
    import paper_2201_12963_gb300 as g
    from paper_2201_12963_gb300.autograd import electrode_charge, energy
    from paper_2201_12963_gb300.driver import System
    w0 = dataclasses.replace(synth.config_large_ff(seed=SEEDS[0]), alpha=0.45, rcut=13.5)
    s64 = System(w0, "fp64", matrix_kspace="mesh", order=8)
    s32 = System(w0, "mixed", matrix_kspace="mesh", order=8)
    worst = {"dq": 0.0, "f_elyt": 0.0, "f_elec": 0.0, "e": 0.0, "fd": 0.0, "oracle": 0.0}
    for k, (R_np, Q_np) in enumerate(elyts):
        w = dataclasses.replace(w0, elyt_xyz=[R_np], elyt_q=[Q_np])
        res = {}
        for name, s in (("fp64", s64), ("mixed", s32)):
            s.load(w)
            s.step(elec=True, energy=True)
            res[name] = s.results()
            assert g.cpm_status(s.ctx) == 0
        r64, r32 = res["fp64"], res["mixed"]
        dq = float(np.max(np.abs(r32["q"][0] - r64["q"][0])))
        fe = _rms_rel(r32["F_elyt"][0], r64["F_elyt"][0])
        fc = _rms_rel(r32["F_elec"][0], r64["F_elec"][0])
        de = abs(r32["energy"][0, 1] - r64["energy"][0, 1]) / abs(r64["energy"][0, 1])
        # the mesh self-energy of the charges, KE alpha/sqrt(pi) sum Q^2 (cancelled exactly by the
        # float64 self term): the float32 transform's rounding is a fraction of it
        e_self = ocpm.KE * w.alpha / np.sqrt(np.pi) * float(np.sum(Q_np ** 2))
        assert dq <= 1e-5, (SEEDS[k], dq)
        assert fe <= 1e-5, (SEEDS[k], fe)
        assert fc <= 1e-5, (SEEDS[k], fc)
        # float32 mesh: its transform rounds at ~1e-7 of the mesh energy, which at alpha 0.45 is
        # dominated by the charges' self-interaction (22,000 eV here, about 40 |H|)
        assert abs(r32["energy"][0, 1] - r64["energy"][0, 1]) <= 3e-7 * e_self, (SEEDS[k], de)
        for key, v in (("dq", dq), ("f_elyt", fe), ("f_elec", fc), ("e", de)):
            worst[key] = max(worst[key], v)
        # autograd: the backward pass returns minus the step's forces
        R = torch.tensor(R_np, dtype=torch.float64, device="cuda", requires_grad=True)
        dpsi = torch.tensor(w.dpsi, dtype=torch.float64, device="cuda", requires_grad=True)
        H = energy(R, dpsi, s64)
        H.sum().backward()
        grad = R.grad.cpu().numpy()
        assert _rms_rel(-grad, r64["F_elyt"][0]) <= 1e-12
        # the same float64 step evaluated again: its mesh spread adds with atomics in no fixed
        # order, so H repeats to float64 rounding of the mesh energy (self-energy included)
        assert abs(H.item() - r64["energy"][0, 1]) <= 1e-13 * e_self
        if k % 10:
            continue
        # finite differences of the float64 energy
        rng = np.random.default_rng(SEEDS[k])
        R0 = R.detach().clone()
        gmax = np.abs(grad).max()
        h = 1e-4
        for p in rng.choice(R0.shape[0] * 3, size=12, replace=False):
            j, c = divmod(int(p), 3)
            Rp, Rm = R0.clone(), R0.clone()
            Rp[j, c] += h
            Rm[j, c] -= h
            fd = (energy(Rp, dpsi.detach(), s64) - energy(Rm, dpsi.detach(), s64)).item() / (2 * h)
            assert abs(fd - grad[j, c]) <= 2e-6 * gmax
            worst["fd"] = max(worst["fd"], abs(fd - grad[j, c]) / gmax)
        hv = 1e-3
        d0 = dpsi.detach()
        fdv = (energy(R0, d0 + hv, s64) - energy(R0, d0 - hv, s64)).item() / (2 * hv)
        assert abs(fdv - float(dpsi.grad)) <= 1e-7 * max(1.0, abs(float(dpsi.grad)))
        d = d0.clone().requires_grad_(True)
        Qp = electrode_charge(d, s64)
        Qp.backward()
        fdq = (electrode_charge(d0 + hv, s64) - electrode_charge(d0 - hv, s64)).item() / (2 * hv)
        assert abs(fdq - float(d.grad)) <= 1e-9 * abs(float(d.grad))
        # the oracle's gradient at sampled electrolyte sites, at the GPU's float64 charges
        s64.step(elec=False, energy=True)
        q64 = s64.results()["q"][0]
        il = np.sort(rng.choice(len(Q_np), 32, replace=False))
        F_or = ocpm.electrolyte_forces_at(w, R_np, Q_np, q64, float(w.dpsi[0]), il, kspace="separable")
        err = _rms_rel(r64["F_elyt"][0][il], F_or)
        worst["oracle"] = max(worst["oracle"], err)
        # the SPME mesh error of the forces at alpha 0.45 / A on the 1 A mesh (order 8): 2.6e-5
        assert err <= 5e-5, (SEEDS[k], err)
    print("worst over 50 configurations:", {k: f"{v:.2e}" for k, v in worst.items()})
