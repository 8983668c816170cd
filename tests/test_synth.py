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
