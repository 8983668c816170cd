"""Matrix images (cpm_matrix_key / cpm_matrix_image / cpm_build_matrix_from_image).

CPU: the key changes with every input that determines A and with nothing else.
GPU: a context built from an image holds the same S, A^-1 C and S v as a fresh build and steps
identically; images whose key or layout differ are refused; the driver's file cache round-trips.
"""
import dataclasses

import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def g():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2201_12963_gb300 as pkg
    return pkg


def _key(g, w, **kw):
    args = dict(box=w.box, eta=w.eta, alpha=w.alpha, rcut=w.rcut, grid=w.grid, order=4, geometry=w.geometry,
                precision="mixed")
    args.update(kw)
    p = g.make_params(**args)
    return g.cpm_matrix_key(p, w.elec_xyz, w.elec_side, w.elec_cell)


def test_key_tracks_exactly_the_inputs_of_A(g):
    w = synth.tiny_cell()
    k0 = _key(g, w)
    assert _key(g, w, precision="fp64") == k0
    assert _key(g, w, max_replicas=7, max_elyt=1234) == k0
    assert _key(g, w, grid=(16, 16, 40)) == k0                     # Ewald form: the per-step mesh does not enter A
    for kw in (dict(alpha=0.26), dict(eta=1.9), dict(rcut=11.0), dict(box=w.box + [0, 0, 1e-9]),
               dict(matrix_kspace="mesh"), dict(kmax_build=3.0), dict(geometry="slab")):
        assert _key(g, w, **kw) != k0, kw
    assert _key(g, w, matrix_kspace="mesh", grid=(16, 16, 40)) != _key(g, w, matrix_kspace="mesh")
    xyz = w.elec_xyz.copy()
    xyz[5, 2] = np.nextafter(xyz[5, 2], 1e9)
    assert _key(g, dataclasses.replace(w, elec_xyz=xyz)) != k0
    side = w.elec_side.copy()
    side[[0, -1]] = side[[-1, 0]]
    assert _key(g, dataclasses.replace(w, elec_side=side)) != k0
    wd = synth.tiny_cell(geometry="dc")
    kd = _key(g, wd)
    cell = wd.elec_cell.copy()
    cell[[0, -1]] = cell[[-1, 0]]
    assert _key(g, dataclasses.replace(wd, elec_cell=cell)) != kd
    assert _key(g, wd, dc_blocks="full") != kd


def _cell(geometry="ff", n_pairs=4):
    """The tiny cell with a mesh fine enough for order 8 (K >= 16)."""
    w = synth.tiny_cell(n_pairs=n_pairs, geometry=geometry)
    return dataclasses.replace(w, grid=tuple(2 * k for k in w.grid))


def _results(s):
    s.step(elec=True, energy=True)
    return s.results()


@pytest.mark.gpu
@pytest.mark.parametrize("geometry,prec", [("ff", "fp64"), ("ff", "mixed"), ("dc", "fp64"), ("dc", "mixed")])
def test_context_from_image_equals_fresh_build(g, geometry, prec):
    from paper_2201_12963_gb300.driver import System
    w = _cell(geometry)
    a = System(w, prec, order=8)
    img = g.cpm_matrix_image(a.ctx)
    ctx_b = g.cpm_build_matrix_from_image(a.params, w.elec_xyz, w.elec_side, w.elec_cell, img)
    assert g.cpm_matrix_layout(ctx_b) == g.cpm_matrix_layout(a.ctx)
    assert g.cpm_capacitance(ctx_b) == g.cpm_capacitance(a.ctx)
    for which in (0, 1, 2):
        assert np.array_equal(g.cpm_copy_matrix(ctx_b, which), g.cpm_copy_matrix(a.ctx, which))
    b = System(w, prec, order=8)
    b.ctx = ctx_b
    ra, rb = _results(a), _results(b)
    tol = 1e-13 if prec == "fp64" else 1e-6                 # float atomics in the mesh spread
    assert np.max(np.abs(ra["q"] - rb["q"])) <= tol
    assert np.max(np.abs(ra["energy"] - rb["energy"])) <= tol * np.max(np.abs(ra["energy"]))
    assert g.cpm_status(b.ctx) == 0


@pytest.mark.gpu
def test_foreign_or_damaged_images_are_refused(g):
    from paper_2201_12963_gb300.driver import System
    w = _cell()
    a = System(w, "fp64", order=8)
    img = g.cpm_matrix_image(a.ctx)
    other = g.make_params(w.box, w.eta, 0.3, w.rcut, w.grid, 8, "ff", "fp64")
    for params, image in ((other, img), (a.params, img[:-8]), (a.params, np.concatenate([img, img[:8]]))):
        with pytest.raises(g.CPMError) as ei:
            g.cpm_build_matrix_from_image(params, w.elec_xyz, w.elec_side, None, image)
        assert ei.value.status == -1
    bad = img.copy()
    bad[0] ^= 1                                             # magic
    with pytest.raises(g.CPMError):
        g.cpm_build_matrix_from_image(a.params, w.elec_xyz, w.elec_side, None, bad)


@pytest.mark.gpu
def test_driver_file_cache_round_trips(g, tmp_path):
    from paper_2201_12963_gb300.driver import System
    w = _cell("dc")
    a = System(w, "mixed", order=8, cache_dir=str(tmp_path))
    assert not a.from_cache and len(list(tmp_path.iterdir())) == 1
    b = System(w, "mixed", order=8, cache_dir=str(tmp_path))
    assert b.from_cache
    assert np.array_equal(g.cpm_copy_matrix(a.ctx, 0), g.cpm_copy_matrix(b.ctx, 0))
    ra, rb = _results(a), _results(b)
    assert np.max(np.abs(ra["q"] - rb["q"])) <= 1e-6
    # a damaged file is rebuilt, not used
    f = next(tmp_path.iterdir())
    f.write_bytes(f.read_bytes()[:-16])
    c = System(w, "mixed", order=8, cache_dir=str(tmp_path))
    assert not c.from_cache


@pytest.mark.gpu
def test_slab_mesh_form_image_round_trips(g):
    """The slab geometry with the mesh form of A (whose key includes the mesh and order)."""
    from paper_2201_12963_gb300.driver import System
    w = synth.tiny_cell(n_pairs=4, geometry="slab")
    w = dataclasses.replace(w, grid=(20, 16, 216))
    a = System(w, "mixed", order=8, matrix_kspace="mesh")
    img = g.cpm_matrix_image(a.ctx)
    ctx_b = g.cpm_build_matrix_from_image(a.params, w.elec_xyz, w.elec_side, None, img)
    assert np.array_equal(g.cpm_copy_matrix(ctx_b, 0), g.cpm_copy_matrix(a.ctx, 0))
    other = g.make_params(w.box, w.eta, w.alpha, w.rcut, (20, 16, 224), 8, "slab", "mixed", matrix_kspace="mesh")
    with pytest.raises(g.CPMError):
        g.cpm_build_matrix_from_image(other, w.elec_xyz, w.elec_side, None, img)
