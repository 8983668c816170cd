"""GPU path against the FP64 oracle, element by element, on the same seeded inputs.

Tolerances (spec bars): |dq| <= 1e-5 e per site, RMS relative force error <= 1e-5, relative
energy error <= 1e-7.  The float64 path is held to them with an SPME mesh fine enough that the
mesh discretisation error sits below them (order 8 at ~1 A or finer); the mixed path (float32
pair and mesh work) is held to the charge bar and to its float32 error level for forces (1e-5)
and energies (2e-6).  The paper's own mesh (1 A, order 5) is checked at its measured
discretisation error in test_paper_mesh_errors.
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


TOL = {"fp64": dict(q=1e-5, f=1e-5, e=1e-7, b=1e-6),
       "mixed": dict(q=1e-5, f=1e-5, e=2e-6, b=5e-5)}


def _check(res, ref, prec, r=0, tol=None, oracle=None):
    """Element-wise comparison of a GPU result with the oracle's step `ref`; `oracle` (the
    oracle.cpm.Reference that produced it) enables the offset-potential checks."""
    t = dict(TOL[prec])
    if tol:
        t.update(tol)
    q, qo = res["q"][r], ref["q"]
    assert np.max(np.abs(q - qo)) <= t["q"]
    assert abs(q.sum()) <= 1e-12 * max(1.0, np.abs(q).sum())
    assert np.max(np.abs(res["b"][r] - ref["b"])) <= t["b"] * np.sqrt(np.mean(ref["b"] ** 2))
    if oracle is not None:
        # the oracle holds the single-replica view of replica r
        check_psibar(res["psibar"][r], res["b"][r], float(oracle.w.dpsi[0]), oracle, ref["psibar"], ref["b"])
    F, Fo = res["F_elyt"][r], ref["F_elyt"]
    assert np.sqrt(((F - Fo) ** 2).sum() / (Fo ** 2).sum()) <= t["f"]
    Fe, Feo = res["F_elec"][r], ref["F_elec"]
    assert np.sqrt(((Fe - Feo) ** 2).sum() / (Feo ** 2).sum()) <= 3 * t["f"]
    U, H, dH, Qp = res["energy"][r]
    assert abs(U - ref["U"]) <= t["e"] * abs(ref["U"])
    assert abs(H - ref["H"]) <= t["e"] * abs(ref["H"])
    assert abs(Qp - ref["Q_plus"]) <= t["q"] * len(qo)
    assert abs(dH - ref["dH_ddpsi"]) <= t["b"] * max(1.0, abs(ref["dH_ddpsi"]))


def _run(w, prec, **kw):
    g, System = _lib()
    s = System(w, prec, **kw)
    s.charges()
    s.forces(elec=True, energy=True)
    assert g.cpm_status(s.ctx) == 0
    return s, s.results()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_plain_finite_field_cell(plain_ff, prec):
    w, ref, out = plain_ff
    s, res = _run(w, prec, order=8)
    _check(res, out, prec, oracle=ref)


def test_projected_inverse_and_capacitance(plain_ff):
    g, System = _lib()
    w, ref, out = plain_ff
    s = System(w, "fp64")
    S = g.cpm_copy_matrix(s.ctx, 0)
    So = ocpm.paper_projected_inverse(ref.A, ref.C)
    assert np.max(np.abs(S - So)) <= 1e-12 * np.max(np.abs(So))
    Sv = g.cpm_copy_matrix(s.ctx, 1)
    assert np.max(np.abs(Sv - So @ ref.v)) <= 1e-12 * np.max(np.abs(So @ ref.v))
    assert abs(g.cpm_capacitance(s.ctx) - (So @ ref.v)[w.elec_side > 0].sum()) <= 1e-12


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("geometry", ["dc", "slab"])
def test_doubled_cell_and_slab(prec, geometry):
    base = synth.tiny_cell(seed=4, n_pairs=4)
    if geometry == "dc":
        w = synth.mirror_to_doubled(base, "independent", seed=40)
        w.grid = (18, 16, 144)
    else:
        w = dataclasses.replace(base, geometry="slab", grid=(18, 16, 216))
    oracle = ocpm.Reference(w)
    ref = oracle.step()
    s, res = _run(w, prec, order=8)
    _check(res, ref, prec, oracle=oracle)
    if geometry == "dc":
        n = w.n_elec // 2
        assert abs(res["q"][0][n:].sum()) <= 1e-12      # sub-cell 1 neutral on its own (Eq. 12)


def test_mirror_symmetric_doubled_cell_gives_mirror_charges():
    w = synth.tiny_cell(seed=4, n_pairs=4, geometry="dc")
    w.grid = (18, 16, 144)
    s, res = _run(w, "fp64", order=8)
    n = w.n_elec // 2
    q = res["q"][0]
    assert np.max(np.abs(q[:n] - q[n:])) <= 1e-9


def test_batched_ragged_replicas_match_per_replica_oracle():
    w = synth.config_batched(n_rep=3)
    s, res = _run(w, "mixed")
    ref = None
    for r in range(w.n_rep):
        wr = w.replica(r)
        if ref is None:
            ref = ocpm.Reference(wr)
        ref.w = wr
        out = ref.step()
        # the paper's 1 A, order-5 mesh on a dense point-ion electrolyte
        _check(res, out, "mixed", r=r, tol=dict(f=5e-5, e=1e-4, b=2e-5), oracle=ref)


def test_fused_step_equals_separate_calls(plain_ff):
    """cpm_step equals cpm_step_charges + cpm_forces; its closed-form energy (exact A) agrees with
    the full Ewald sum of cpm_forces / cpm_energy (mesh for the electrode-electrode part) to the
    mesh error, and both agree with the oracle."""
    g, System = _lib()
    w, _, out = plain_ff
    a = System(w, "fp64", order=8)
    a.charges()
    a.forces(elec=False, energy=True)
    ra = a.results()
    b = System(w, "fp64", order=8)
    b.step(elec=False, energy=True)
    rb = b.results()
    assert np.max(np.abs(ra["q"] - rb["q"])) <= 1e-14
    assert np.max(np.abs(ra["F_elyt"][0] - rb["F_elyt"][0])) <= 1e-12
    for k in (0, 1):
        assert abs(ra["energy"][0, k] - rb["energy"][0, k]) <= 1e-7 * abs(rb["energy"][0, k])
        assert abs(rb["energy"][0, k] - (out["U"], out["H"])[k]) <= 1e-7 * abs(out["U"])
    assert np.max(np.abs(ra["energy"][0, 2:] - rb["energy"][0, 2:])) <= 1e-12
    c = System(w, "fp64", order=8)
    c.q.copy_(b.q)
    c.energies()
    assert np.max(np.abs(c.results()["energy"] - ra["energy"])) <= 1e-10 * abs(out["U"])


def test_empty_electrolyte_gives_capacitor_charges():
    g, System = _lib()
    w = synth.config_plain_ff()
    w = dataclasses.replace(w, elyt_xyz=[np.zeros((0, 3))], elyt_q=[np.zeros(0)])
    ref = ocpm.Reference(w)
    qo, lam, _ = ref.charges(np.zeros((0, 3)), np.zeros(0), float(w.dpsi[0]))
    s = System(w, "fp64", max_elyt=8)
    s.step(elec=True, energy=True)
    r = s.results()
    assert np.max(np.abs(r["q"][0] - qo)) <= 1e-12
    assert np.max(np.abs(r["q"][0] - w.dpsi[0] * g.cpm_copy_matrix(s.ctx, 1))) <= 1e-12


def test_device_errors_are_latched():
    g, System = _lib()
    w = synth.tiny_cell(seed=2, n_pairs=2)
    s = System(w, "fp64", grid=(20, 16, 72), order=6)
    s.xyzq[0, 2] = w.box[2] + 5.0          # outside [0, L_z)
    s.charges()
    assert g.cpm_status(s.ctx) == -6
    s.xyzq[0, 2] = float("nan")
    s.charges()
    assert g.cpm_status(s.ctx) == -4
    s.load(w)
    s.charges()
    assert g.cpm_status(s.ctx) == 0
    off2 = torch.tensor([0, 2, 4], dtype=torch.int32, device=s.xyzq.device)
    dp2 = torch.zeros(2, dtype=torch.float64, device=s.xyzq.device)
    q2 = torch.zeros(2 * s.ne, dtype=torch.float64, device=s.xyzq.device)
    with pytest.raises(g.CPMError) as ei:
        g.cpm_step_charges(s.ctx, 2, off2, s.xyzq, dp2, q2)   # n_rep above capacity 1
    assert ei.value.status == -5


def test_paper_mesh_errors(plain_ff):
    """The paper's mesh (1 A, order 5): charges within 1e-5 e, discretisation errors as measured."""
    w, ref, out = plain_ff
    for prec in ("fp64", "mixed"):
        s, res = _run(w, prec)
        _check(res, out, prec, tol=dict(f=5e-5, e=3e-5, b=1e-5), oracle=ref)


def test_batched_tensor_core_s_apply_matches_float64_path():
    """16 replicas with the mixed path take the tcgen05 split-TF32 S-apply; charges must agree with
    the float64 path (same mesh) and with the oracle to the charge bar |dq| <= 1e-5 e (measured
    about 4e-6 e on this dense 400-600-pair electrolyte: three TF32 products keep ~21 bits)."""
    g, System = _lib()
    w = synth.config_batched(n_rep=16)
    mixed = System(w, "mixed")
    mixed.charges()
    assert g.cpm_status(mixed.ctx) == 0
    r32 = mixed.results()
    ref64 = System(w, "fp64")
    ref64.charges()
    r64 = ref64.results()
    assert np.max(np.abs(r32["q"] - r64["q"])) <= 1e-5
    assert np.max(np.abs(r32["q"].sum(axis=1))) <= 1e-12
    assert np.max(np.abs(r32["psibar"] - r64["psibar"])) <= 1e-4
    ref = None
    for r in (0, 15):
        wr = w.replica(r)
        if ref is None:
            ref = ocpm.Reference(wr)
        ref.w = wr
        q, lam, _ = ref.charges(wr.elyt_xyz[0], wr.elyt_q[0], float(wr.dpsi[0]))
        assert np.max(np.abs(r32["q"][r] - q)) <= 1e-5



def _indefinite_cell():
    """The tiny cell with alpha = 0.01 / A and r_c = 2 A: the Ewald split is truncated so hard
    (no reciprocal vector below 2 alpha sqrt(27.6), real space cut at 2 A) that A is indefinite
    (its smallest eigenvalue is -7.2 V/e on the oracle: test_oracle_pins)."""
    return dataclasses.replace(synth.tiny_cell(seed=1, n_pairs=2), alpha=0.01, rcut=2.0, grid=(20, 16, 72))


@pytest.mark.parametrize("blocks", ["full", "mirror"])
def test_indefinite_elastance_is_refused(blocks):
    """The build's Cholesky factorisation refuses an A that is not positive definite with
    CPM_ERR_NOT_SPD (also for the two mirror blocks of a doubled cell), and the library stays
    usable: a normal build afterwards succeeds."""
    g, System = _lib()
    w = _indefinite_cell()
    if blocks == "mirror":
        w = synth.mirror_to_doubled(w, "mirror")
        w.grid = (20, 16, 144)
    with pytest.raises(g.CPMError) as ei:
        System(w, "fp64", dc_blocks=blocks if w.geometry == "dc" else "auto")
    assert ei.value.status == -3
    s = System(synth.tiny_cell(seed=1, n_pairs=2), "fp64", grid=(20, 16, 72))
    s.charges()
    assert g.cpm_status(s.ctx) == 0


def _rms_rel(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))


@pytest.mark.parametrize("case", ["plain", "jittered", "dc", "batched"])
def test_electrode_forces_from_the_precomputed_pair_list(plain_ff, case):
    """cpm_step with electrode forces (closed-form energy) in mixed precision takes the
    Gaussian-Gaussian forces of the frozen electrode from the pair list precomputed at build, and
    the electrolyte's real-space force on the electrode sites from the field of the b pass;
    cpm_forces with the full energy computes both in the pair kernels.  Both must agree, and
    with the oracle's electrode forces.  The lattice electrodes take the compressed list (a table
    of distinct G vectors); `jittered` moves every electrode site by up to 0.02 A, so that the G
    vectors no longer repeat and the full list is used."""
    g, System = _lib()
    if case == "plain":
        w, _, out = plain_ff
    elif case == "jittered":
        w = dataclasses.replace(plain_ff[0])
        rng = np.random.Generator(np.random.PCG64(91))
        w.elec_xyz = np.asarray(w.elec_xyz, float) + rng.uniform(-0.02, 0.02, size=np.shape(w.elec_xyz))
        out = ocpm.Reference(w).step()
    elif case == "dc":
        w = synth.mirror_to_doubled(synth.tiny_cell(seed=4, n_pairs=4), "independent", seed=40)
        w.grid = (18, 16, 144)
        out = ocpm.Reference(w).step()
    else:
        w = synth.config_batched(n_rep=3)
        out = None
    a = System(w, "mixed", order=8)
    pairs, table = g.cpm_pair_list_layout(a.ctx)
    assert pairs > 0
    assert (table == 0) if case == "jittered" else (0 < table < 4096)
    a.step(elec=True, energy=True)
    ra = a.results()
    assert g.cpm_status(a.ctx) == 0
    b = System(w, "mixed", order=8)
    b.q.copy_(a.q)
    b.forces(elec=True, energy=True)
    rb = b.results()
    for r in range(w.n_rep):
        assert _rms_rel(ra["F_elec"][r], rb["F_elec"][r]) <= 3e-6
        assert _rms_rel(ra["F_elyt"][r], rb["F_elyt"][r]) <= 1e-6
    if out is not None:
        assert _rms_rel(ra["F_elec"][0], out["F_elec"]) <= 3e-5


@pytest.mark.parametrize("case", ["plain", "dc", "batched", "large"])
def test_third_law_pair_kernel_matches_the_cell_kernel(plain_ff, case):
    """CPM_PAIR_N3_ELYT: the electrolyte-electrolyte pairs taken once (half stencil, each periodic
    image pair once: the 17 x 17 A plain cell spans fewer cells than the stencil, so every
    neighbour cell appears at several images), the reaction added to the source.  Forces and
    energies must equal the cell kernel's to float32 rounding, and the forces the oracle's."""
    g, System = _lib()
    out = None
    if case == "plain":
        w, _, out = plain_ff
    elif case == "dc":
        w = synth.mirror_to_doubled(synth.tiny_cell(seed=4, n_pairs=4), "independent", seed=40)
        w.grid = (18, 16, 144)
        out = ocpm.Reference(w).step()
    elif case == "batched":
        w = synth.config_batched(n_rep=3)
    else:
        w = synth.config_large_ff()
    s = System(w, "mixed", order=8) if case != "large" else System(w, "mixed", matrix_kspace="mesh")
    res = {}
    for v, gz in (("cell", 1), ("n3", 1), ("n3-warp-elec", 1), ("n3", 2)):
        g.cpm_set_pair_variant(s.ctx, v)
        assert g.cpm_get_pair_variant(s.ctx) == v
        g.cpm_set_pair_group(s.ctx, gz)                  # z groups of cells: the ordering rule
        s.step(elec=True, energy=True)
        res[(v, gz)] = s.results()
        assert g.cpm_status(s.ctx) == 0
    ra = res[("cell", 1)]
    for v in (("n3", 1), ("n3-warp-elec", 1), ("n3", 2)):
        rb = res[v]
        for r in range(w.n_rep):
            assert np.max(np.abs(rb["q"][r] - ra["q"][r])) <= 1e-6
            assert _rms_rel(rb["F_elyt"][r], ra["F_elyt"][r]) <= 2e-6
            assert _rms_rel(rb["F_elec"][r], ra["F_elec"][r]) <= 2e-6
            # the pair energies are float32 terms summed in another order: on the dense batched
            # electrolyte (sites 1.5 A apart, terms of several eV) their rounding reaches 1e-6 of H
            etol = 1e-5 if case == "batched" else 1e-6
            if case != "batched":
                # per site: a pair within r_c taken twice or missed would move two sites by at
                # least the pair force at r_c, 2.7e-5 eV/A for these +-0.78 e ions (1.5e-5 in its
                # largest component), above float32 rounding of the sums (up to 5e-6 measured)
                assert np.max(np.abs(rb["F_elyt"][r] - ra["F_elyt"][r])) <= 1e-5
            assert abs(rb["energy"][r, 1] - ra["energy"][r, 1]) <= etol * abs(ra["energy"][r, 1])
        if out is not None:
            assert _rms_rel(rb["F_elyt"][0], out["F_elyt"]) <= 3e-5
    with pytest.raises(g.CPMError):
        g.cpm_set_pair_variant(s.ctx, 6)                 # third law with warp-per-target electrolyte
