"""Differentiable energy: backward (forces from the library) against central finite differences
of the GPU energy itself, against the oracle's analytic gradient, and dQ_+/d dpsi against the
capacitance (GPU)."""
import dataclasses

import numpy as np
import pytest

import synth
from oracle import cpm as ocpm

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _system(w, prec="fp64", **kw):
    import __graft_entry__
    __graft_entry__.build()
    from paper_2201_12963_gb300.driver import System
    return System(w, prec, **kw)


def _smooth_cell():
    """Small cell where erfc(alpha r_c) < 1e-16, so the truncated sums are smooth in R."""
    w = synth.tiny_cell(seed=12, n_pairs=3)
    return dataclasses.replace(w, alpha=0.45, rcut=13.5, grid=(24, 20, 96))


def test_energy_gradient_matches_finite_differences():
    from paper_2201_12963_gb300.autograd import energy
    w = _smooth_cell()
    s = _system(w, order=8)
    R = torch.tensor(w.elyt_xyz[0], dtype=torch.float64, device="cuda", requires_grad=True)
    dpsi = torch.tensor(w.dpsi, dtype=torch.float64, device="cuda", requires_grad=True)
    H = energy(R, dpsi, s)
    H.sum().backward()
    g = R.grad.cpu().numpy()
    gd = float(dpsi.grad.cpu())
    h = 1e-4
    R0 = R.detach().clone()
    for j in range(R0.shape[0]):
        for c in range(3):
            Rp, Rm = R0.clone(), R0.clone()
            Rp[j, c] += h
            Rm[j, c] -= h
            fd = (energy(Rp, dpsi.detach(), s) - energy(Rm, dpsi.detach(), s)).item() / (2 * h)
            assert abs(fd - g[j, c]) <= 2e-6 * np.abs(g).max()
    hv = 1e-3
    d0 = dpsi.detach()
    fdv = (energy(R0, d0 + hv, s) - energy(R0, d0 - hv, s)).item() / (2 * hv)
    assert abs(fdv - gd) <= 1e-8 * max(1.0, abs(gd))


def test_energy_gradient_matches_oracle_forces():
    from paper_2201_12963_gb300.autograd import energy
    w = _smooth_cell()
    out = ocpm.Reference(w).step()
    s = _system(w, order=8)
    R = torch.tensor(w.elyt_xyz[0], dtype=torch.float64, device="cuda", requires_grad=True)
    dpsi = torch.tensor(w.dpsi, dtype=torch.float64, device="cuda", requires_grad=True)
    H = energy(R, dpsi, s)
    H.sum().backward()
    F = -R.grad.cpu().numpy()
    Fo = out["F_elyt"]
    assert np.sqrt(((F - Fo) ** 2).sum() / (Fo ** 2).sum()) <= 1e-5
    assert abs(H.item() - out["H"]) <= 1e-7 * abs(out["H"])
    assert abs(float(dpsi.grad) - out["dH_ddpsi"]) <= 1e-6


def test_capacitance_is_charge_derivative():
    from paper_2201_12963_gb300.autograd import electrode_charge
    import paper_2201_12963_gb300 as g
    w = synth.config_plain_ff()
    s = _system(w, order=5)
    d = torch.tensor([2.0], dtype=torch.float64, device="cuda", requires_grad=True)
    Q = electrode_charge(d, s)
    Q.backward()
    cap = g.cpm_capacitance(s.ctx)
    assert abs(float(d.grad) - cap) <= 1e-14
    h = 1e-3
    fd = (electrode_charge(d.detach() + h, s) - electrode_charge(d.detach() - h, s)).item() / (2 * h)
    assert abs(fd - cap) <= 1e-9 * abs(cap)
    ref = ocpm.Reference(w)
    So = ocpm.paper_projected_inverse(ref.A, ref.C)
    assert abs(cap - (So @ ref.v)[w.elec_side > 0].sum()) <= 1e-12


def test_differentiation_at_the_10080_site_cell():
    """The 10,080-site, 5,000-ion-pair finite-field cell: autograd forces against central finite
    differences (h = 1e-4 A) of the GPU float64 energy at 64 sampled coordinates, dH/d dpsi and
    dQ_+/d dpsi against h = 1e-3 V differences, and the mixed path against float64 (charges and
    forces).  alpha 0.45 A^-1 and r_c 13.5 A make the truncated real-space sum smooth
    (erfc(alpha r_c) ~ 1e-17), so differences across the cutoff do not spoil the quotients; A's
    reciprocal part is the mesh operator, so H is the exact minimum of the discrete energy.  The
    oracle's dense A at this size is out of reach on the host; the oracle gradient is checked on the
    small cells above."""
    from paper_2201_12963_gb300.autograd import electrode_charge, energy
    import paper_2201_12963_gb300 as g
    w = dataclasses.replace(synth.config_large_ff(), alpha=0.45, rcut=13.5)
    s = _system(w, "fp64", matrix_kspace="mesh")
    R = torch.tensor(w.elyt_xyz[0], dtype=torch.float64, device="cuda", requires_grad=True)
    dpsi = torch.tensor(w.dpsi, dtype=torch.float64, device="cuda", requires_grad=True)
    H = energy(R, dpsi, s)
    H.sum().backward()
    grad = R.grad.cpu().numpy()
    gd = float(dpsi.grad)
    q64 = s.q.cpu().numpy().copy()
    rng = np.random.default_rng(4000)
    picks = rng.choice(R.shape[0] * 3, size=64, replace=False)
    h = 1e-4
    R0 = R.detach().clone()
    gmax = np.abs(grad).max()
    for p in picks:
        j, c = divmod(int(p), 3)
        Rp, Rm = R0.clone(), R0.clone()
        Rp[j, c] += h
        Rm[j, c] -= h
        fd = (energy(Rp, dpsi.detach(), s) - energy(Rm, dpsi.detach(), s)).item() / (2 * h)
        assert abs(fd - grad[j, c]) <= 2e-6 * gmax
    hv = 1e-3
    d0 = dpsi.detach()
    fdv = (energy(R0, d0 + hv, s) - energy(R0, d0 - hv, s)).item() / (2 * hv)
    assert abs(fdv - gd) <= 1e-7 * max(1.0, abs(gd))
    d = d0.clone().requires_grad_(True)
    Q = electrode_charge(d, s)
    Q.backward()
    fdq = (electrode_charge(d0 + hv, s) - electrode_charge(d0 - hv, s)).item() / (2 * hv)
    assert abs(fdq - float(d.grad)) <= 1e-9 * abs(float(d.grad))
    # the mixed path at full size against float64 (the |dq| <= 1e-5 e bar and 1e-5 RMS forces)
    sm = _system(w, "mixed", matrix_kspace="mesh")
    Rm_ = R0.clone().requires_grad_(True)
    Hm = energy(Rm_, d0, sm)
    Hm.sum().backward()
    assert np.max(np.abs(sm.q.cpu().numpy() - q64)) <= 1e-5
    gm = Rm_.grad.cpu().numpy()
    assert np.sqrt(((gm - grad) ** 2).sum() / (grad ** 2).sum()) <= 1e-5
    assert abs(Hm.item() - H.item()) <= 2e-6 * abs(H.item())
    assert g.cpm_status(s.ctx) == 0 and g.cpm_status(sm.ctx) == 0
