"""The MD loop (cpm_md_*) against the FP64 oracle's integrator and against invariants (GPU).

* Lennard-Jones forces and energy of the library's cell-list kernel against the oracle's direct
  sum over images (the difference of runs with and without LJ isolates them exactly).
* Trajectories: positions, velocities, charges, thermostat state and energies after a few steps
  of velocity-Verlet with Nose-Hoover thermostats and charges re-solved every k steps, against
  oracle.md.Integrator on the same seeded inputs (finite field one thermostat, doubled cell one per
  sub-cell).  The library's k-space is SPME, the oracle's a direct Ewald sum: an order-8 mesh at
  about 0.45 A spacing keeps the force difference small enough for the stated bounds.
* NVE with charges re-solved every step conserves the total energy with a fluctuation that shrinks
  as dt^2 (the SPME forces are the exact gradient of the SPME energy).
* A run interrupted by a checkpoint and restored into a fresh integrator continues the trajectory;
  a captured CUDA graph of k steps replays the same trajectory as direct calls.
"""
import dataclasses

import numpy as np
import pytest

import synth
from oracle import md as omd

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2201_12963_gb300 as g
    from paper_2201_12963_gb300.driver import MD, System
    return g, System, MD


def _cell(geometry="ff", seed=7, n_pairs=4):
    w = synth.tiny_cell(seed=seed, n_pairs=n_pairs, geometry=geometry)
    # alpha 0.35: no visible energy jumps at the real-space cutoff; fine order-8 mesh: SPME close to Ewald
    lx, ly, lz = w.box
    if geometry == "slab":
        lz = lz * w.slab_factor                        # the mesh spans the padded Ewald box
    grid = tuple(int(2 * round(L / 0.45 / 2)) for L in (lx, ly, lz))
    return dataclasses.replace(w, alpha=0.35, grid=grid, order=8)


def _oracle(w, mi, k, dt, t_damp, lj_cut):
    p = omd.MDParams(dt=dt, charge_every=k, mass=mi.mass, sigma=mi.sigma, eps=mi.eps, elec_type=mi.elec_type,
                     lj_cut=lj_cut, temperature=mi.temperature, t_damp=t_damp)
    integ = omd.Integrator(w, mi.types, mi.groups, p)
    st = omd.initial_state(w.elyt_xyz[0], mi.vel, w.n_elec, integ.n_groups)
    return integ, st


def _wrapdiff(a, b, box):
    d = a - b
    d[:, :2] -= box[:2] * np.round(d[:, :2] / box[:2])
    return d


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_lennard_jones_forces_and_energy_against_oracle(prec):
    g, System, MD = _lib()
    w = _cell(n_pairs=6)
    mi = synth.md_inputs(w, seed=3)
    res = {}
    for cut in (0.0, 7.0):
        s = System(w, prec, order=8)
        m = MD(s, mi, dt=2.0, charge_every=1, lj_cut=cut, t_damp=0.0)
        m.run(0, energy=True, force=True)
        assert g.cpm_status(s.ctx) == 0
        res[cut] = (m.force.cpu().numpy().reshape(-1, 3).copy(), m.energies()[0])
    U, F = omd.lj_energy_forces(w.elyt_xyz[0], mi.types, w.elec_xyz, mi.elec_type, mi.sigma, mi.eps, 7.0,
                                np.asarray(w.box))
    F_lj = res[7.0][0] - res[0.0][0]
    tol = 1e-10 if prec == "fp64" else 2e-5
    assert np.sqrt(((F_lj - F) ** 2).sum() / (F ** 2).sum()) <= tol
    assert abs(res[7.0][1]["U_lj"] - U) <= tol * max(1.0, abs(U))
    assert res[0.0][1]["U_lj"] == 0.0


@pytest.mark.parametrize("geometry,k,t_damp", [("ff", 1, 0.0), ("ff", 3, 50.0), ("dc", 2, 50.0), ("slab", 2, 50.0)])
def test_trajectory_against_oracle(geometry, k, t_damp):
    g, System, MD = _lib()
    w = _cell(geometry)
    mi = synth.md_inputs(w, seed=5)
    dt, n, cut = 2.0, 9, 7.0
    s = System(w, "fp64", order=8)
    m = MD(s, mi, dt=dt, charge_every=k, lj_cut=cut, t_damp=t_damp)
    m.run(n, energy=True)
    assert g.cpm_status(s.ctx) == 0
    integ, st = _oracle(w, mi, k, dt, t_damp, cut)
    integ.run(st, n)
    box = np.asarray(w.box)
    R = s.xyzq.cpu().numpy()[:, :3]
    V = m.vel.cpu().numpy().reshape(-1, 3)
    assert np.max(np.abs(_wrapdiff(R, st.R, box))) <= 1e-6
    assert np.max(np.abs(V - st.V)) <= 1e-6 * np.max(np.abs(st.V))
    assert np.max(np.abs(s.q.cpu().numpy() - st.q)) <= 1e-5
    step, thermo = g.cpm_md_get_state(m.md)
    assert step == n
    if t_damp > 0:
        assert np.max(np.abs(thermo[:, 0] - st.xi)) <= 1e-6 * max(1.0, np.max(np.abs(st.xi)))
        assert np.max(np.abs(thermo[:, 1] - st.vxi)) <= 1e-6 * max(1e-3, np.max(np.abs(st.vxi)))
    e, eo = m.energies()[0], integ.conserved(st)
    assert abs(e["KE"] - eo["KE"]) <= 1e-6 * eo["KE"]
    assert abs(e["U_lj"] - eo["U_lj"]) <= 1e-9 * max(1.0, abs(eo["U_lj"]))
    assert abs(e["H"] - eo["H"]) <= 1e-6 * abs(eo["H"])
    assert abs(e["E_nh"] - eo["E_nh"]) <= 1e-6 * max(1e-3, abs(eo["E_nh"]))
    assert abs(e["T"] - eo["T"]) <= 1e-6 * eo["T"]


def test_nve_energy_conservation_is_second_order():
    g, System, MD = _lib()
    w = _cell(n_pairs=4)                  # 8 ions: stays near 600 K (12 ions in this cell heat to ~2,500 K)
    mi = synth.md_inputs(w, seed=3)
    spread = []
    for dt, n in ((2.0, 25), (1.0, 50)):
        s = System(w, "fp64", order=8)
        m = MD(s, mi, dt=dt, charge_every=1, lj_cut=7.0, t_damp=0.0)
        m.run(0, energy=True)
        e = [m.energies()[0]["E_total"]]
        for _ in range(n):
            m.run(1, energy=True)
            e.append(m.energies()[0]["E_total"])
        assert g.cpm_status(s.ctx) == 0
        spread.append(max(e) - min(e))
        assert spread[-1] <= 5e-5 * m.energies()[0]["KE"]
    assert 2.5 <= spread[0] / spread[1] <= 6.0


def test_thermostat_energy_is_conserved():
    """With the thermostat on, KE + H + U_LJ + E_thermostat stays constant (charges re-solved every
    step), while KE + H + U_LJ alone does not."""
    g, System, MD = _lib()
    w = _cell(n_pairs=6)
    mi = synth.md_inputs(w, seed=13, temperature=900.0)     # start hot: the thermostat removes energy
    s = System(w, "fp64", order=8)
    m = MD(s, mi, dt=1.0, charge_every=1, lj_cut=7.0, t_damp=20.0, temperature=300.0)
    tot, phys = [], []
    for _ in range(40):
        m.run(1, energy=True)
        e = m.energies()[0]
        tot.append(e["E_total"])
        phys.append(e["E_total"] - e["E_nh"])
    assert g.cpm_status(s.ctx) == 0
    assert max(tot) - min(tot) <= 0.02 * (max(phys) - min(phys))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_checkpoint_restore_continues_the_trajectory(prec):
    g, System, MD = _lib()
    w = _cell(n_pairs=6)
    mi = synth.md_inputs(w, seed=17)
    s1 = System(w, prec, order=8)
    m1 = MD(s1, mi, dt=2.0, charge_every=3, lj_cut=7.0, t_damp=40.0)
    m1.run(10, energy=True)
    ref = m1.checkpoint()
    s2 = System(w, prec, order=8)
    m2 = MD(s2, mi, dt=2.0, charge_every=3, lj_cut=7.0, t_damp=40.0)
    m2.run(4)
    ck = m2.checkpoint()
    assert ck["step"] == 4
    s3 = System(w, prec, order=8)
    m3 = MD(s3, mi, dt=2.0, charge_every=3, lj_cut=7.0, t_damp=40.0)
    m3.restore(ck)
    m3.run(6, energy=True)
    out = m3.checkpoint()
    assert out["step"] == 10
    tol = 1e-9 if prec == "fp64" else 1e-5
    box = np.asarray(w.box)
    assert np.max(np.abs(_wrapdiff(out["xyzq"][:, :3], ref["xyzq"][:, :3], box))) <= tol
    assert np.max(np.abs(out["vel"] - ref["vel"])) <= tol * np.max(np.abs(ref["vel"]))
    assert np.max(np.abs(out["q"] - ref["q"])) <= tol
    assert np.max(np.abs(out["thermo"] - ref["thermo"])) <= tol * max(1.0, np.max(np.abs(ref["thermo"])))


def test_graph_replay_equals_direct_calls():
    g, System, MD = _lib()
    w = _cell(n_pairs=6)
    mi = synth.md_inputs(w, seed=19)
    k = 3
    sd = System(w, "fp64", order=8)
    md_direct = MD(sd, mi, dt=2.0, charge_every=k, lj_cut=7.0, t_damp=40.0)
    md_direct.run(0)
    md_direct.run(4 * k)
    sg = System(w, "fp64", order=8)
    md_graph = MD(sg, mi, dt=2.0, charge_every=k, lj_cut=7.0, t_damp=40.0)
    md_graph.run(0)
    replay = md_graph.capture(k)
    assert g.cpm_md_get_state(md_graph.md)[0] == 0
    replay(4)
    torch.cuda.synchronize()
    assert g.cpm_md_get_state(md_graph.md)[0] == 4 * k
    a, b = md_direct.checkpoint(), md_graph.checkpoint()
    assert np.max(np.abs(_wrapdiff(a["xyzq"][:, :3], b["xyzq"][:, :3], np.asarray(w.box)))) <= 1e-9
    assert np.max(np.abs(a["vel"] - b["vel"])) <= 1e-9 * np.max(np.abs(a["vel"]))
    assert np.max(np.abs(a["q"] - b["q"])) <= 1e-9


def test_mixed_precision_trajectory_stays_close():
    g, System, MD = _lib()
    w = _cell(n_pairs=6)
    mi = synth.md_inputs(w, seed=23)
    out = {}
    for prec in ("fp64", "mixed"):
        s = System(w, prec, order=8)
        m = MD(s, mi, dt=2.0, charge_every=5, lj_cut=7.0, t_damp=100.0)
        m.run(10, energy=True)
        assert g.cpm_status(s.ctx) == 0
        out[prec] = (s.xyzq.cpu().numpy()[:, :3], s.q.cpu().numpy(), m.energies()[0])
    d = _wrapdiff(out["mixed"][0], out["fp64"][0], np.asarray(w.box))
    assert np.max(np.abs(d)) <= 1e-4
    assert np.max(np.abs(out["mixed"][1] - out["fp64"][1])) <= 1e-5
    assert abs(out["mixed"][2]["E_total"] - out["fp64"][2]["E_total"]) <= 1e-4 * abs(out["fp64"][2]["E_total"])


def test_md_create_rejects_bad_input():
    g, System, MD = _lib()
    w = _cell()
    s = System(w, "fp64", order=8)
    mi = synth.md_inputs(w)
    off = s.offsets.cpu().numpy()
    bad = [dict(dt=-1.0), dict(charge_every=0), dict(lj_cut=w.rcut + 1.0), dict(elec_type=5),
           dict(t_damp=10.0, temperature=0.0)]
    for kw in bad:
        args = dict(dt=2.0, charge_every=1, mass=mi.mass, sigma=mi.sigma, eps=mi.eps, elec_type=2, lj_cut=7.0)
        args.update(kw)
        with pytest.raises(g.CPMError) as ei:
            g.cpm_md_create(s.ctx, g.make_md_params(**args), off, mi.types)
        assert ei.value.status == -1
    p = g.make_md_params(dt=2.0, mass=mi.mass, sigma=mi.sigma, eps=mi.eps, elec_type=2, lj_cut=7.0)
    with pytest.raises(g.CPMError):
        g.cpm_md_create(s.ctx, p, off, np.full(len(mi.types), 2))      # type 2 has no mass
    with pytest.raises(g.CPMError):
        g.cpm_md_create(s.ctx, p, off, mi.types, np.full(len(mi.types), 3))   # group outside n_groups


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_lennard_jones_warp_kernel_against_oracle(prec):
    """The warp-per-target pair kernel with the fused Lennard-Jones term."""
    g, System, MD = _lib()
    w = _cell(n_pairs=6)
    mi = synth.md_inputs(w, seed=3)
    res = {}
    for cut in (0.0, 7.0):
        s = System(w, prec, order=8)
        g.cpm_set_pair_variant(s.ctx, "warp")
        m = MD(s, mi, dt=2.0, charge_every=1, lj_cut=cut, t_damp=0.0)
        m.run(0, energy=True, force=True)
        assert g.cpm_status(s.ctx) == 0
        res[cut] = (m.force.cpu().numpy().reshape(-1, 3).copy(), m.energies()[0])
    U, F = omd.lj_energy_forces(w.elyt_xyz[0], mi.types, w.elec_xyz, mi.elec_type, mi.sigma, mi.eps, 7.0,
                                np.asarray(w.box))
    F_lj = res[7.0][0] - res[0.0][0]
    tol = 1e-10 if prec == "fp64" else 2e-5
    assert np.sqrt(((F_lj - F) ** 2).sum() / (F ** 2).sum()) <= tol
    assert abs(res[7.0][1]["U_lj"] - U) <= tol * max(1.0, abs(U))


def test_replica_batch_equals_replicas_alone():
    """Two replicas (different electrolytes and potential differences) in one integrator: each
    follows the trajectory it has when run alone (thermostat slots and offsets per replica)."""
    g, System, MD = _lib()
    w0 = _cell(n_pairs=4, seed=7)
    w1 = _cell(n_pairs=5, seed=11)
    wb = dataclasses.replace(w0, elyt_xyz=[w0.elyt_xyz[0], w1.elyt_xyz[0]], elyt_q=[w0.elyt_q[0], w1.elyt_q[0]],
                             dpsi=np.array([1.0, 2.5]))
    mis = [synth.md_inputs(wb, seed=31, r=0), synth.md_inputs(wb, seed=32, r=1)]
    s = System(wb, "fp64", order=8)
    m = MD(s, mis, dt=2.0, charge_every=2, lj_cut=7.0, t_damp=40.0)
    m.run(6, energy=True)
    assert g.cpm_status(s.ctx) == 0
    ck = m.checkpoint()
    off = s.offsets.cpu().numpy()
    e_b = m.energies()
    for r in range(2):
        wr = wb.replica(r)
        sr = System(wr, "fp64", order=8)
        mr = MD(sr, [mis[r]], dt=2.0, charge_every=2, lj_cut=7.0, t_damp=40.0)
        mr.run(6, energy=True)
        cr = mr.checkpoint()
        box = np.asarray(wb.box)
        xb = ck["xyzq"][off[r]:off[r + 1], :3]
        assert np.max(np.abs(_wrapdiff(xb, cr["xyzq"][:, :3], box))) <= 1e-9
        vb = ck["vel"].reshape(-1, 3)[off[r]:off[r + 1]]
        assert np.max(np.abs(vb - cr["vel"].reshape(-1, 3))) <= 1e-9 * np.max(np.abs(vb))
        ne = w0.n_elec
        assert np.max(np.abs(ck["q"][r * ne:(r + 1) * ne] - cr["q"])) <= 1e-9
        assert np.max(np.abs(ck["thermo"][r] - cr["thermo"][0])) <= 1e-9 * max(1.0, np.max(np.abs(cr["thermo"])))
        er = mr.energies()[0]
        for key in ("KE", "H", "U_lj", "E_total"):
            assert abs(e_b[r][key] - er[key]) <= 1e-8 * max(1.0, abs(er[key])), key


def test_replica_without_electrolyte():
    """A replica with no electrolyte sites runs beside a populated one: its thermostat slot has no
    degrees of freedom (left untouched), its charges follow its potential difference alone, and
    the populated replica is unaffected."""
    g, System, MD = _lib()
    w0 = _cell(n_pairs=4, seed=7)
    empty = np.zeros((0, 3))
    wb = dataclasses.replace(w0, elyt_xyz=[w0.elyt_xyz[0], empty], elyt_q=[w0.elyt_q[0], np.zeros(0)],
                             dpsi=np.array([1.0, 2.0]))
    mi0 = synth.md_inputs(wb, seed=41, r=0)
    mi1 = synth.md_inputs(wb, seed=42, r=1)
    s = System(wb, "fp64", order=8)
    m = MD(s, [mi0, mi1], dt=2.0, charge_every=2, lj_cut=7.0, t_damp=40.0)
    m.run(4, energy=True)
    assert g.cpm_status(s.ctx) == 0
    ck = m.checkpoint()
    assert np.all(ck["thermo"][1] == 0.0)
    e = m.energies()
    assert e[1]["KE"] == 0.0 and e[1]["T"] == 0.0 and np.isfinite(e[1]["H"])
    sr = System(wb.replica(0), "fp64", order=8)
    mr = MD(sr, [mi0], dt=2.0, charge_every=2, lj_cut=7.0, t_damp=40.0)
    mr.run(4, energy=True)
    cr = mr.checkpoint()
    n0 = len(w0.elyt_q[0])
    assert np.max(np.abs(_wrapdiff(ck["xyzq"][:n0, :3], cr["xyzq"][:, :3], np.asarray(wb.box)))) <= 1e-9
    # the empty replica's charges: the response to its potential difference alone (b = 0)
    ne = w0.n_elec
    sv = g.cpm_copy_matrix(s.ctx, 1)
    assert np.max(np.abs(ck["q"][ne:] - 2.0 * sv)) <= 1e-9
