"""Seeded input generator: shapes, neutrality, separations and determinism (CPU only)."""
import numpy as np

import synth


def _min_sep_xy_periodic(x, box):
    d = x[:, None, :] - x[None, :, :]
    d[..., :2] -= box[:2] * np.round(d[..., :2] / box[:2])
    r = np.sqrt((d * d).sum(-1))
    r[np.diag_indices_from(r)] = np.inf
    return r.min()


def test_plain_cell_shapes_and_placement():
    w = synth.config_plain_ff()
    assert w.n_elec == 672
    assert np.allclose(w.box, [17.04, 17.22, 60.0])
    zs = sorted(set(np.round(w.elec_xyz[:, 2], 6)))
    assert np.allclose(zs, [3.30, 6.65, 10.00, 50.00, 53.35, 56.70])
    R, Q = w.elyt_xyz[0], w.elyt_q[0]
    assert R.shape == (200, 3) and abs(Q.sum()) < 1e-12
    assert np.all((R[:, 2] >= 13.0) & (R[:, 2] <= 47.0))
    assert _min_sep_xy_periodic(R, w.box) >= 3.0
    assert np.all(w.elec_side[w.elec_xyz[:, 2] > 30] == 1)


def test_generator_is_deterministic():
    a = synth.config_plain_ff(seed=1000)
    b = synth.config_plain_ff(seed=1000)
    c = synth.config_plain_ff(seed=1001)
    assert np.array_equal(a.elyt_xyz[0], b.elyt_xyz[0])
    assert not np.array_equal(a.elyt_xyz[0], c.elyt_xyz[0])


def test_paper_cell_coarse_grained_electrolyte():
    w = synth.config_paper_cell()
    assert w.n_elec == 3024
    Q = w.elyt_q[0]
    assert len(Q) == 2000 and abs(Q.sum()) < 1e-9
    assert np.isclose(Q[Q > 0].sum(), 500 * 0.78)
    assert w.grid == (40, 36, 168)


def test_doubled_cell_mirror_layout():
    w = synth.mirror_to_doubled(synth.config_plain_ff(), "mirror")
    n = w.n_elec // 2
    assert np.allclose(w.elec_xyz[n:, 2], 120.0 - w.elec_xyz[:n, 2])
    assert np.array_equal(w.elec_side[n:], w.elec_side[:n])
    assert w.elec_cell[:n].sum() == 0 and w.elec_cell[n:].sum() == n
    assert np.allclose(w.box, [17.04, 17.22, 120.0])


def test_batched_replicas():
    w = synth.config_batched(n_rep=4)
    assert w.n_rep == 4
    counts = [len(q) for q in w.elyt_q]
    assert all(800 <= c <= 1200 for c in counts)
    offs, xyzq = w.packed_electrolyte()
    assert offs[-1] == sum(counts) and xyzq.shape == (sum(counts), 4)
    assert np.allclose(w.dpsi, [0, 4 / 3, 8 / 3, 4])


def test_plain_cell_grid():
    assert synth.config_plain_ff().grid == (18, 18, 60)


def test_md_cell_point_ions_and_inputs():
    w = synth.md_cell()
    assert w.n_elec == 3024 and np.allclose(w.box, [38.34, 34.44, 168.0])
    R, Q = w.elyt_xyz[0], w.elyt_q[0]
    assert R.shape == (2000, 3) and abs(Q.sum()) < 1e-12
    assert np.all(np.abs(np.abs(Q) - synth.ION_CHARGE) < 1e-12)
    assert np.all((R[:, 2] >= 13.0) & (R[:, 2] <= 155.0))
    assert _min_sep_xy_periodic(R, w.box) >= 3.0
    mi = synth.md_inputs(w, seed=5)
    assert np.array_equal(mi.types, np.where(Q > 0, 0, 1)) and not np.any(mi.groups)
    # Maxwell-Boltzmann: <m v_d^2> = k_B T per component (2,000 x 3 samples: ~2 % spread)
    m = np.asarray(mi.mass)[mi.types]
    kt = (m[:, None] * mi.vel ** 2).mean() * synth.AMU_A2_FS2_EV
    assert abs(kt / (synth.KB_EV * mi.temperature) - 1.0) < 0.06
    assert abs(mi.vel.mean()) < 5 * mi.vel.std() / np.sqrt(mi.vel.size)


def test_md_doubled_cell_thermostat_groups():
    w = synth.md_cell(geometry="dc")
    mi = synth.md_inputs(w)
    z = w.elyt_xyz[0][:, 2]
    assert w.n_elec == 6048 and len(z) == 4000
    assert np.array_equal(mi.groups, (z >= 0.5 * w.box[2]).astype(np.int32))
    assert mi.groups.sum() == 2000
    # every ion stays inside its own sub-cell's electrolyte region (the electrodes separate them)
    assert np.all((z[mi.groups == 0] > 13.0) & (z[mi.groups == 0] < 155.0))
    assert np.all((z[mi.groups == 1] > 181.0) & (z[mi.groups == 1] < 323.0))


def test_md_inputs_refuse_molecular_electrolytes():
    import pytest
    with pytest.raises(ValueError):
        synth.md_inputs(synth.config_paper_cell())


def _paper_parameters():
    import os
    vals = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                key, value = line.split()[:2]
                vals[key] = float(value)
    return vals


def test_generators_and_defaults_use_the_parameters_the_paper_fixes(monkeypatch):
    """tests/golden/paper_parameters.txt holds the values the paper prints (each with its section);
    the paper-scale cell, the MD settings and the geometry vector must use them."""
    import dataclasses
    import inspect
    import sys
    from oracle import cpm
    from oracle.md import MDParams
    p = _paper_parameters()
    w = synth.config_paper_cell()
    assert w.eta == p["gaussian_eta_per_A"]
    Q = w.elyt_q[0]
    n_pairs = int((Q < 0).sum())
    assert n_pairs == 500 and np.allclose(Q[Q < 0], -p["ion_charge_e"])
    assert abs(Q[Q > 0].sum() / n_pairs - p["ion_charge_e"]) < 1e-12     # three sites per cation
    zs = np.unique(np.round(w.elec_xyz[:, 2], 9))
    assert np.allclose(np.diff(zs[:3]), p["interlayer_spacing_A"])
    assert np.allclose(np.diff(zs[-3:]), p["interlayer_spacing_A"])
    layer = w.elec_xyz[np.isclose(w.elec_xyz[:, 2], zs[0])]
    assert abs(_min_sep_xy_periodic(layer, w.box) - p["cc_bond_A"]) < 1e-9
    # ion-pair number density in the accessible slab against 1.267 g/cm^3 of BMIm-PF6 (284.18 g/mol)
    rho_paper = p["bulk_density_g_cm3"] / 284.18 * 6.02214076e23 / 1e24
    lx, ly, lz = w.box
    rho = n_pairs / (lx * ly * (lz - 2 * synth.ELECTROLYTE_MARGIN))
    assert abs(rho / rho_paper - 1.0) < 0.01
    # the MD loop: 2 fs steps, charges re-solved every 5 steps (oracle, library driver, benchmark)
    assert synth.PAPER_TIMESTEP_FS == p["timestep_fs"] == MDParams().dt
    assert MDParams().charge_every == p["charge_update_every"]
    import __graft_entry__
    __graft_entry__.build()                     # the driver module loads the library
    from paper_2201_12963_gb300.driver import MD
    sig = inspect.signature(MD.__init__).parameters
    assert sig["dt"].default == p["timestep_fs"] and sig["charge_every"].default == p["charge_update_every"]
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    assert bench.parse().charge_every == p["charge_update_every"]
    # d = +-1/2 on the two electrodes (Eq. 5)
    v = cpm.geometry_vector(dataclasses.replace(w, geometry="slab"))
    assert np.allclose(np.abs(v), p["d_entry_magnitude"])
