"""Doubled-cell mirror blocks and the mesh form of A's reciprocal part (GPU).

Mirror blocks: for a doubled cell whose sub-cell-1 electrode is the z-mirror image of sub-cell 0,
A = [[P, Q], [Q, P]] and the library stores the two singly-constrained half-size projected
inverses S+- of P +- Q instead of the full S (the reduction is pinned on the oracle's A in
test_oracle_pins.test_doubled_cell_two_mirror_blocks_equal_full_solve).  Here the GPU mirror form
is compared with the GPU full form built from the same electrode (matrices, charges, offsets,
forces, energies) and with the oracle.

Mesh form of A: the reciprocal part of A as the SPME operator W^T Phi W of the per-step calls.
At the constrained optimum the closed-form energy of cpm_step, U_elyt - q^T b / 2 + dpsi q^T v / 2,
then equals the full sum of cpm_energy (real-space pairs + mesh energy of all charges + self terms)
to rounding, because both evaluate the same discrete quadratic form; with the Ewald-sum A they
differ by the mesh error.  This pins the mesh A (constants, stencil convention, normalisation)
against kernels that share no code with its build.
"""
import dataclasses

import numpy as np
import pytest

import synth
from kkt_checks import check_psibar
from oracle import cpm as ocpm

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2201_12963_gb300 as g
    from paper_2201_12963_gb300.driver import System
    return g, System


def _dc_cell(seed=4):
    w = synth.mirror_to_doubled(synth.tiny_cell(seed=seed, n_pairs=4), "independent", seed=40)
    w.grid = (18, 16, 144)
    return w


def _run(System, w, prec, **kw):
    s = System(w, prec, **kw)
    s.charges()
    s.forces(elec=True, energy=True)
    return s, s.results()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_mirror_blocks_equal_full_matrix(prec):
    g, System = _lib()
    w = _dc_cell()
    sf, rf = _run(System, w, prec, order=8, dc_blocks="full")
    sm, rm = _run(System, w, prec, order=8, dc_blocks="mirror")
    assert g.cpm_status(sf.ctx) == 0 and g.cpm_status(sm.ctx) == 0
    mf, bytes_f = g.cpm_matrix_layout(sf.ctx)
    mm, bytes_m = g.cpm_matrix_layout(sm.ctx)
    assert not mf and mm
    assert bytes_m * 2 <= bytes_f + 16 * w.n_elec * 8           # two half blocks: half the S bytes
    for which in (0, 1, 2):
        a, b = g.cpm_copy_matrix(sf.ctx, which), g.cpm_copy_matrix(sm.ctx, which)
        assert np.max(np.abs(a - b)) <= 1e-11 * np.max(np.abs(a))
    assert abs(g.cpm_capacitance(sf.ctx) - g.cpm_capacitance(sm.ctx)) <= 1e-11 * abs(g.cpm_capacitance(sf.ctx))
    qtol = 1e-11 if prec == "fp64" else 1e-6                     # float32 S: different rounding of S vs S+-
    q_f, q_m = rf["q"][0], rm["q"][0]
    assert np.max(np.abs(q_f - q_m)) <= qtol
    n = w.n_elec // 2
    assert abs(q_m.sum()) <= 1e-12 and abs(q_m[n:].sum()) <= 1e-12
    assert np.max(np.abs(rf["psibar"][0] - rm["psibar"][0])) <= (1e-9 if prec == "fp64" else 1e-5)
    for key in ("F_elyt", "F_elec"):
        a, b = rf[key][0], rm[key][0]
        assert np.sqrt(((a - b) ** 2).sum() / (a ** 2).sum()) <= (1e-10 if prec == "fp64" else 1e-5)
    assert np.max(np.abs(rf["energy"][0] - rm["energy"][0]) / np.maximum(1.0, np.abs(rf["energy"][0]))) <= 1e-6


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_mirror_blocks_against_oracle(prec):
    """Charges, offsets, forces and energies of the mirror form against the oracle's full KKT
    solve, with an electrolyte that is not mirrored (both the sum and the difference modes)."""
    g, System = _lib()
    w = _dc_cell(seed=6)
    oracle = ocpm.Reference(w)
    ref = oracle.step()
    s, res = _run(System, w, prec, order=8, dc_blocks="mirror")
    assert g.cpm_status(s.ctx) == 0
    q = res["q"][0]
    assert np.max(np.abs(q - ref["q"])) <= 1e-5
    check_psibar(res["psibar"][0], res["b"][0], float(w.dpsi[0]), oracle, ref["psibar"], ref["b"])
    F, Fo = res["F_elyt"][0], ref["F_elyt"]
    assert np.sqrt(((F - Fo) ** 2).sum() / (Fo ** 2).sum()) <= 1e-5
    U = res["energy"][0][0]
    assert abs(U - ref["U"]) <= (1e-7 if prec == "fp64" else 2e-6) * abs(ref["U"])


def test_mirror_blocks_need_a_mirror_symmetric_electrode():
    g, System = _lib()
    w = _dc_cell()
    xyz = w.elec_xyz.copy()
    xyz[w.n_elec - 1, 0] += 0.01                                # one image site off its mirror position
    wa = dataclasses.replace(w, elec_xyz=xyz)
    with pytest.raises(g.CPMError) as ei:
        System(wa, "fp64", order=8, dc_blocks="mirror")
    assert ei.value.status == -1
    s = System(wa, "fp64", order=8, dc_blocks="auto")           # falls back to the full matrix
    assert g.cpm_matrix_layout(s.ctx)[0] is False
    s2 = System(w, "fp64", order=8, dc_blocks="auto")
    assert g.cpm_matrix_layout(s2.ctx)[0] is True


@pytest.mark.parametrize("geometry", ["ff", "dc"])
def test_mesh_matrix_closed_form_energy_equals_full_sum(plain_ff, geometry):
    g, System = _lib()
    if geometry == "ff":
        w = plain_ff[0]
    else:
        w = _dc_cell()
    gaps = {}
    for kspace in ("mesh", "ewald"):
        s = System(w, "fp64", matrix_kspace=kspace)
        s.step(elec=False, energy=True)
        U_closed = s.energy[0].item()
        s.energies()                                             # full sum at the same charges
        U_full = s.energy[0].item()
        assert g.cpm_status(s.ctx) == 0
        gaps[kspace] = abs(U_closed - U_full) / abs(U_full)
    assert gaps["mesh"] <= 1e-10
    assert gaps["ewald"] > 10 * gaps["mesh"]                     # the Ewald-sum A differs by the mesh error


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_mesh_matrix_against_oracle(plain_ff, prec):
    """The mesh form of A differs from the oracle's converged Ewald A by the mesh discretisation
    error: at an order-8 mesh the charges stay within the 1e-5 e bar."""
    g, System = _lib()
    w, ref, out = plain_ff
    s, res = _run(System, w, prec, order=8, matrix_kspace="mesh")
    assert g.cpm_status(s.ctx) == 0
    assert np.max(np.abs(res["q"][0] - out["q"])) <= 1e-5
    F, Fo = res["F_elyt"][0], out["F_elyt"]
    assert np.sqrt(((F - Fo) ** 2).sum() / (Fo ** 2).sum()) <= 1e-5
    S = g.cpm_copy_matrix(s.ctx, 0)
    So = ocpm.paper_projected_inverse(ref.A, ref.C)
    assert np.max(np.abs(S - So)) <= 1e-4 * np.max(np.abs(So))


def test_mesh_matrix_mirror_blocks_against_oracle():
    """The large doubled-cell configuration's build (mesh A, mirror blocks), small cell."""
    g, System = _lib()
    w = _dc_cell(seed=8)
    ref = ocpm.Reference(w).step()
    s, res = _run(System, w, "mixed", order=8, matrix_kspace="mesh", dc_blocks="mirror")
    assert g.cpm_status(s.ctx) == 0
    assert np.max(np.abs(res["q"][0] - ref["q"])) <= 1e-5
    F, Fo = res["F_elyt"][0], ref["F_elyt"]
    assert np.sqrt(((F - Fo) ** 2).sum() / (Fo ** 2).sum()) <= 1e-5
