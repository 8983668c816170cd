"""Charge density and potential profiles across the cell (Sec. II.C) and proximal-layer-only
charging (Appendix B) on the GPU.

cpm_density_z is compared with the oracle's binned density for the same electrode charges (the
GPU's own charges, so only the binning and the Gaussian integration are tested), cpm_potential_z
with the oracle's finite-difference matrix inverse, in the finite-field, doubled-cell and slab
geometries; repeated density calls accumulate.  A proximal-only cell (one third of the sites
charged) is held to the oracle at the usual charge bar.
"""
import dataclasses

import numpy as np
import pytest

import synth
from oracle import cpm as ocpm
from oracle import profile as oprof

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2201_12963_gb300 as g
    from paper_2201_12963_gb300.driver import System
    return g, System


def _cell(kind):
    if kind == "ff":
        return synth.config_plain_ff()
    base = synth.tiny_cell(seed=4, n_pairs=4)
    if kind == "dc":
        w = synth.mirror_to_doubled(base, "independent", seed=40)
        w.grid = (18, 16, 144)
        return w
    return dataclasses.replace(base, geometry="slab", grid=(18, 16, 216))


@pytest.mark.parametrize("kind", ["ff", "dc", "slab"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_density_and_potential_profiles_match_oracle(kind, prec):
    g, System = _lib()
    w = _cell(kind)
    s = System(w, prec)
    s.charges()
    nb = 400
    rho = torch.zeros(nb, dtype=torch.float64, device="cuda")
    g.cpm_density_z(s.ctx, 1, s.offsets, s.xyzq, s.q, nb, rho)
    psi = torch.zeros(nb, dtype=torch.float64, device="cuda")
    g.cpm_potential_z(s.ctx, 1, nb, rho, 1.0, s.dpsi, psi)
    assert g.cpm_status(s.ctx) == 0
    q = s.q.cpu().numpy()
    lx, ly, lz = w.box
    bz = lz * (w.slab_factor if kind == "slab" else 1.0)
    ro = oprof.charge_density_z(bz, lx * ly, nb, w.elyt_xyz[0][:, 2], w.elyt_q[0], w.elec_xyz[:, 2], q, w.eta)
    r = rho.cpu().numpy()
    assert np.max(np.abs(r - ro)) <= 1e-12 * np.max(np.abs(ro))
    po = oprof.potential_z(r, bz, geometry=w.geometry, dpsi=float(w.dpsi[0]))
    p = psi.cpu().numpy()
    assert np.max(np.abs(p - po)) <= 1e-9 * np.max(np.abs(po))
    # accumulation: two samples averaged give the same profile
    g.cpm_density_z(s.ctx, 1, s.offsets, s.xyzq, s.q, nb, rho)
    psi2 = torch.zeros_like(psi)
    g.cpm_potential_z(s.ctx, 1, nb, rho, 0.5, s.dpsi, psi2)
    assert torch.max(torch.abs(psi2 - psi)).item() <= 1e-12 * np.max(np.abs(po))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_proximal_only_charging_matches_oracle(prec):
    g, System = _lib()
    w = synth.proximal_only(synth.config_plain_ff())
    out = ocpm.Reference(w).step()
    s = System(w, prec, order=8)
    s.charges()
    s.forces(elec=True, energy=True)
    assert g.cpm_status(s.ctx) == 0
    res = s.results()
    assert np.max(np.abs(res["q"][0] - out["q"])) <= 1e-5
    F, Fo = res["F_elyt"][0], out["F_elyt"]
    assert np.sqrt(((F - Fo) ** 2).sum() / (Fo ** 2).sum()) <= 1e-5
