"""S-apply kernel variants and the autotuner (GPU).

The single-replica mixed-precision S-apply has several kernels: one warp per row of S, streaming
kernels (persistent CTAs with the right-hand side in shared memory, equal contiguous spans of S per
warp, float64 row partial sums), and the packed upper-triangle tiles read with plain loads or with
bulk asynchronous copies into shared memory.  All must give the same charges to float32 rounding
and match the oracle at the charge bar, in the full and the mirror-block layouts; cpm_autotune must
keep one of them and leave the context's results unchanged.
"""
import numpy as np
import pytest

import synth
from oracle import cpm as ocpm

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2201_12963_gb300 as g
    from paper_2201_12963_gb300.driver import System
    return g, System


def _cases(plain_ff):
    w_dc = synth.mirror_to_doubled(synth.tiny_cell(seed=4, n_pairs=4), "independent", seed=40)
    w_dc.grid = (18, 16, 144)
    return {"ff": (plain_ff[0], plain_ff[2]), "dc": (w_dc, None)}


@pytest.mark.parametrize("case", ["ff", "dc"])
def test_sapply_variants_agree_and_match_oracle(plain_ff, case):
    g, System = _lib()
    w, out = _cases(plain_ff)[case]
    if out is None:
        out = ocpm.Reference(w).step(want_forces=False, want_energy=False)
    s = System(w, "mixed", order=8)
    qs, pb = {}, {}
    for v in ("rows", "stream", "stream16", "sym", "sym-tma"):
        g.cpm_set_sapply_variant(s.ctx, v)
        for _ in range(2):                          # the second call checks the cleared partial sums
            s.charges()
        assert g.cpm_status(s.ctx) == 0
        qs[v] = s.q.cpu().numpy().copy()
        pb[v] = s.psibar.cpu().numpy().copy()
        assert np.max(np.abs(qs[v] - out["q"])) <= 1e-5
        assert abs(qs[v].sum()) <= 1e-12
        # the packed kernels form the offsets' sums (A^-1 C)^T b in their own epilogue (Eq. 9;
        # Eqs. 13-15 per mirror block): the same offsets as the finish pass of the other kernels,
        # up to the run-to-run float32 rounding of b (mesh atomics in no fixed order)
        assert np.max(np.abs(pb[v] - pb["rows"])) <= 1e-5
    assert np.max(np.abs(qs["rows"] - qs["stream"])) <= 1e-6
    assert np.max(np.abs(qs["rows"] - qs["stream16"])) <= 1e-6
    assert np.max(np.abs(qs["rows"] - qs["sym"])) <= 1e-6
    assert np.max(np.abs(qs["rows"] - qs["sym-tma"])) <= 1e-6
    choice, transform, assign = g.cpm_autotune(s.ctx, s.offsets, s.xyzq, s.dpsi, s.q)
    assert choice in ("rows", "stream", "stream16", "sym", "sym-tma") and transform in ("library", "own")
    assert assign in ("sites", "brick")
    s.charges()
    # float32 mesh spreading adds with atomics in no fixed order: repeated mixed-precision runs
    # differ at float32 rounding
    assert np.max(np.abs(s.q.cpu().numpy() - qs[choice])) <= 1e-6


def test_stream_variant_needs_mixed_precision(plain_ff):
    g, System = _lib()
    s = System(plain_ff[0], "fp64")
    with pytest.raises(g.CPMError):
        g.cpm_set_sapply_variant(s.ctx, "stream")
    g.cpm_set_sapply_variant(s.ctx, "rows")


@pytest.mark.parametrize("case", ["ff", "dc", "slab"])
def test_own_mesh_transform_matches_library_and_oracle(plain_ff, case):
    """The library's own float32 mesh convolution (five launches, four-step line transforms) against
    cuFFT in the same context: charges, forces and energies to float32 rounding, and both against
    the oracle at the charge and force bars."""
    import dataclasses
    g, System = _lib()
    if case == "ff":
        w, out = plain_ff[0], plain_ff[2]
    elif case == "dc":
        w = _cases(plain_ff)["dc"][0]
        out = ocpm.Reference(w).step()
    else:
        base = synth.tiny_cell(seed=4, n_pairs=4)
        w = dataclasses.replace(base, geometry="slab", grid=(18, 16, 216))
        out = ocpm.Reference(w).step()
    s = System(w, "mixed", order=8)
    res = {}
    for v in ("library", "own"):
        g.cpm_set_fft_variant(s.ctx, v)
        s.charges()
        s.forces(elec=True, energy=True)
        assert g.cpm_status(s.ctx) == 0
        res[v] = s.results()
        r = res[v]
        assert np.max(np.abs(r["q"][0] - out["q"])) <= 1e-5
        F, Fo = r["F_elyt"][0], out["F_elyt"]
        assert np.sqrt(((F - Fo) ** 2).sum() / (Fo ** 2).sum()) <= 1e-5
        assert abs(r["energy"][0][0] - out["U"]) <= 2e-6 * abs(out["U"])
    a, b = res["library"], res["own"]
    assert np.max(np.abs(a["q"][0] - b["q"][0])) <= 1e-6
    Fa, Fb = a["F_elyt"][0], b["F_elyt"][0]
    assert np.sqrt(((Fa - Fb) ** 2).sum() / (Fa ** 2).sum()) <= 2e-6
    assert abs(a["energy"][0][0] - b["energy"][0][0]) <= 1e-6 * abs(a["energy"][0][0])


def test_own_mesh_transform_needs_mixed_precision(plain_ff):
    g, System = _lib()
    s = System(plain_ff[0], "fp64")
    with pytest.raises(g.CPMError):
        g.cpm_set_fft_variant(s.ctx, "own")


@pytest.mark.parametrize("case", ["ff", "dc", "slab"])
def test_brick_charge_assignment_matches_sites_and_oracle(plain_ff, case):
    """Charge assignment and force interpolation through shared-memory bricks moved by TMA (halo-
    padded mesh, fold, halo fill) against the per-site atomics in the same context, and both against
    the oracle: charges, forces (electrolyte and electrode) and energies."""
    import dataclasses
    g, System = _lib()
    if case == "ff":
        w, out = plain_ff[0], plain_ff[2]
    elif case == "dc":
        w = _cases(plain_ff)["dc"][0]
        out = ocpm.Reference(w).step()
    else:
        base = synth.tiny_cell(seed=4, n_pairs=4)
        w = dataclasses.replace(base, geometry="slab", grid=(18, 16, 216))
        out = ocpm.Reference(w).step()
    s = System(w, "mixed", order=8)
    res = {}
    for v in ("sites", "brick"):
        g.cpm_set_mesh_variant(s.ctx, v)
        for _ in range(2):                       # the second call checks the cleared padded mesh
            s.charges()
            s.forces(elec=True, energy=True)
        assert g.cpm_status(s.ctx) == 0
        res[v] = s.results()
        r = res[v]
        assert np.max(np.abs(r["q"][0] - out["q"])) <= 1e-5
        F, Fo = r["F_elyt"][0], out["F_elyt"]
        assert np.sqrt(((F - Fo) ** 2).sum() / (Fo ** 2).sum()) <= 1e-5
        Fe, Feo = r["F_elec"][0], out["F_elec"]
        assert np.sqrt(((Fe - Feo) ** 2).sum() / (Feo ** 2).sum()) <= 3e-5
        assert abs(r["energy"][0][0] - out["U"]) <= 2e-6 * abs(out["U"])
    a, b = res["sites"], res["brick"]
    assert np.max(np.abs(a["q"][0] - b["q"][0])) <= 1e-6
    Fa, Fb = a["F_elyt"][0], b["F_elyt"][0]
    assert np.sqrt(((Fa - Fb) ** 2).sum() / (Fa ** 2).sum()) <= 2e-6
    # the fused step (charges and forces in one call) through the bricks as well
    s.step(elec=False, energy=True)
    assert g.cpm_status(s.ctx) == 0
    assert np.max(np.abs(s.q.cpu().numpy()[: w.n_elec] - b["q"][0])) <= 1e-6


def test_brick_charge_assignment_needs_mixed_precision(plain_ff):
    g, System = _lib()
    s = System(plain_ff[0], "fp64")
    with pytest.raises(g.CPMError):
        g.cpm_set_mesh_variant(s.ctx, "brick")


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ["ff", "dc", "slab"])
def test_pair_kernel_z_groups_match_single_cells_and_oracle(plain_ff, case, prec):
    """Blocks of 1, 2, 4 and 3 cells along z (3 leaves a shorter last group) and the
    warp-per-target kernels give the same b, charges, forces on both site kinds and energies: only
    the order of the sums changes."""
    g, System = _lib()
    if case == "ff":
        w, out = plain_ff[0], plain_ff[2]
    elif case == "dc":
        w, out = _cases(plain_ff)["dc"][0], None
    else:
        w = synth.tiny_cell(seed=9, n_pairs=4, geometry="slab")
        w.grid = (18, 16, 216)
        out = None
    if out is None:
        out = ocpm.Reference(w).step()
    s = System(w, prec, order=8)
    res = {}
    for gz in (1, 2, 3, 4, "warp", "warp-elec"):
        if isinstance(gz, str):
            g.cpm_set_pair_group(s.ctx, 1)
            g.cpm_set_pair_variant(s.ctx, gz)
            assert g.cpm_get_pair_variant(s.ctx) == gz
        else:
            g.cpm_set_pair_group(s.ctx, gz)
            assert g.cpm_get_pair_group(s.ctx) == gz
        s.step(elec=True, energy=True)
        s.energies()
        r = s.results()
        assert g.cpm_status(s.ctx) == 0
        res[gz] = r
        assert np.max(np.abs(r["q"][0] - out["q"])) <= 1e-5
        F, Fo = r["F_elyt"][0], out["F_elyt"]
        assert np.sqrt(((F - Fo) ** 2).sum() / (Fo ** 2).sum()) <= 1e-5
    tol = 1e-12 if prec == "fp64" else 2e-6
    for gz in (2, 3, 4, "warp", "warp-elec"):
        a, b = res[gz], res[1]
        assert np.max(np.abs(a["b"] - b["b"])) <= tol * np.max(np.abs(b["b"]))
        assert np.max(np.abs(a["q"] - b["q"])) <= tol
        for key in ("F_elyt", "F_elec"):
            x, y = np.asarray(a[key]).reshape(-1, 3), np.asarray(b[key]).reshape(-1, 3)
            assert np.sqrt(((x - y) ** 2).sum() / (y ** 2).sum()) <= tol
        assert np.max(np.abs(a["energy"] - b["energy"])) <= tol * np.max(np.abs(b["energy"]))
    with pytest.raises(g.CPMError):
        g.cpm_set_pair_group(s.ctx, 0)


@pytest.mark.parametrize("case", ["ff", "dc", "large"])
def test_packed_variants_at_full_size(case):
    """The packed kernels at the paper-scale cell (3,024 sites: 24 tile rows, 300 tiles, about two
    per CTA, a ragged last tile row; the doubled cell: two mirror blocks of the same size), where
    they form the projection sums in their own epilogue, and at the 10,080-site cell (79 tile rows,
    about 21 tiles per CTA), where a finish pass forms them, give the charges and offsets of the row
    kernel, whose charges the full-size tests check against the oracle.  The charge sum stays
    neutral to float64 rounding either way; b differs between calls at float32 rounding (mesh
    atomics), which bounds the comparisons (about 2e-6 e in q at the paper-scale cell)."""
    g, System = _lib()
    w = synth.config_large_ff() if case == "large" else synth.config_paper_cell(geometry=case)
    s = System(w, "mixed")
    res = {}
    for v in ("rows", "sym", "sym-tma", "sym"):
        g.cpm_set_sapply_variant(s.ctx, v)
        for _ in range(2):                          # the second call checks the cleared partial sums
            s.charges()
        assert g.cpm_status(s.ctx) == 0
        q, pb = s.q.cpu().numpy().copy(), s.psibar.cpu().numpy().copy()
        assert abs(q.sum()) <= 1e-12
        if v in res:
            assert np.max(np.abs(q - res[v][0])) <= 1e-5
        res[v] = (q, pb)
    for v in ("sym", "sym-tma"):
        assert np.max(np.abs(res[v][0] - res["rows"][0])) <= 1e-5
        assert np.max(np.abs(res[v][1] - res["rows"][1])) <= 1e-5
