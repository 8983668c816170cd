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
