"""Pins of the MD-loop oracle (oracle.md) against closed forms and invariants (CPU).

* Lennard-Jones: the textbook values U(sigma) = 0, U(2^(1/6) sigma) = -eps with zero force there
  (cutoff far away), Lorentz-Berthelot mixing seen through the position and depth of the minimum,
  energy and force vanishing at the cutoff, force = -gradient (finite differences), Newton's third
  law, and images beyond the nearest counted when the cell is shorter than the cutoff.
* Velocity-Verlet on a harmonic oscillator obeys the Stormer recurrence
  x_{n+1} - 2 x_n + x_{n-1} = -(omega dt)^2 x_n exactly, so x_n = x_0 cos(n theta) + B sin(n theta)
  with cos(theta) = 1 - (omega dt)^2 / 2.
* The Nose-Hoover equations of motion (dx/dt = v, dv/dt = F/m - v_xi v, dxi/dt = v_xi,
  dv_xi/dt = (2K - g k_B T)/Q) integrated by an adaptive Runge-Kutta solver: the Trotter scheme
  converges to that solution at second order in dt.  Thermostat groups are independent.
* CPM + LJ with charges re-solved every step: the total energy KE + H + U_LJ is conserved with a
  fluctuation that shrinks as dt^2 (forces are minus the gradient of that energy), the dynamics is
  time-reversible, and with k > 1 the charges change only at multiples of k.
"""
import math

import numpy as np
import pytest
from scipy.integrate import solve_ivp

import synth
from oracle import md


def _lj2(r, sig=(3.0, 3.0), eps=(0.02, 0.02), cut=1000.0, box=4000.0):
    """Energy and force on site 0 of two electrolyte sites at distance r along x."""
    R = np.array([[100.0, 100.0, 100.0], [100.0 + r, 100.0, 100.0]])
    U, F = md.lj_energy_forces(R, [0, 1], np.zeros((0, 3)), 2, list(sig) + [1.0], list(eps) + [0.0], cut,
                               np.array([box, box, box]))
    return U, F


def test_lj_textbook_values():
    s, e = 3.4, 0.0104
    U, F = _lj2(s, (s, s), (e, e))
    assert abs(U) <= 1e-12
    rmin = 2 ** (1 / 6) * s
    U, F = _lj2(rmin, (s, s), (e, e))
    assert abs(U + e) <= 1e-12 * e * 1e3
    assert np.max(np.abs(F)) <= 1e-12
    # repulsive inside the minimum: site 0 pushed towards -x
    U, F = _lj2(3.0, (s, s), (e, e))
    assert F[0, 0] < 0 and abs(F[0, 0] + F[1, 0]) <= 1e-15 * abs(F[0, 0]) + 1e-18


def test_lorentz_berthelot_mixing_sets_the_minimum():
    sa, sb, ea, eb = 3.0, 4.2, 0.02, 0.005
    r = np.linspace(3.0, 6.0, 30001)
    U = np.array([_lj2(x, (sa, sb), (ea, eb))[0] for x in r[::100]])
    i = int(np.argmin(U)) * 100
    fine = r[max(0, i - 100):i + 100]
    Uf = np.array([_lj2(x, (sa, sb), (ea, eb))[0] for x in fine])
    rmin = fine[int(np.argmin(Uf))]
    assert abs(rmin - 2 ** (1 / 6) * 0.5 * (sa + sb)) <= 2e-4
    assert abs(Uf.min() + math.sqrt(ea * eb)) <= 1e-9


def test_lj_vanishes_continuously_at_the_cutoff():
    cut = 9.0
    for r in (cut - 1e-7, cut + 1e-7):
        U, F = _lj2(r, cut=cut, box=100.0)
        assert abs(U) <= 1e-12 and np.max(np.abs(F)) <= 1e-9


def test_lj_force_is_minus_gradient_and_obeys_newton():
    rng = np.random.default_rng(5)
    box = np.array([14.0, 13.0, 30.0])
    R = rng.uniform(0, 1, size=(12, 3)) * box
    E = np.stack([rng.uniform(0, box[0], 20), rng.uniform(0, box[1], 20), np.full(20, 2.0)], axis=1)
    types = rng.integers(0, 2, size=12)
    sig, eps = [3.0, 3.6, 3.37], [0.02, 0.01, 0.0024]
    U, F = md.lj_energy_forces(R, types, np.zeros((0, 3)), 2, sig, eps, 8.0, box)
    assert np.max(np.abs(F.sum(0))) <= 1e-10 * np.max(np.abs(F))
    U, F = md.lj_energy_forces(R, types, E, 2, sig, eps, 8.0, box)
    h = 1e-5
    for i in (0, 5, 11):
        for c in range(3):
            Rp, Rm = R.copy(), R.copy()
            Rp[i, c] += h
            Rm[i, c] -= h
            fd = -(md.lj_energy_forces(Rp, types, E, 2, sig, eps, 8.0, box)[0]
                   - md.lj_energy_forces(Rm, types, E, 2, sig, eps, 8.0, box)[0]) / (2 * h)
            assert abs(fd - F[i, c]) <= 1e-6 * max(1.0, abs(F[i, c]))


def test_lj_counts_every_image_within_the_cutoff():
    """One site alone in a cubic cell of edge L < cut: its periodic images sit at L, sqrt(2) L, ...;
    the energy is half the sum of the pair energy over all lattice vectors within the cutoff."""
    L, cut = 4.0, 9.0
    U, F = md.lj_energy_forces(np.array([[1.0, 2.0, 3.0]]), [0], np.zeros((0, 3)), 2, [3.0, 3.0, 3.37],
                               [0.02, 0.02, 0.0], cut, np.array([L, L, L]))
    n = np.arange(-3, 4)
    g = np.stack(np.meshgrid(n, n, n, indexing="ij"), -1).reshape(-1, 3) * L
    r = np.sqrt((g * g).sum(1))
    r = r[(r > 0) & (r < cut)]
    s6 = (3.0 / r) ** 6
    sc6 = (3.0 / cut) ** 6
    fc = 24 * 0.02 * (2 * sc6 * sc6 - sc6) / cut
    u = 4 * 0.02 * (s6 * s6 - s6) - 4 * 0.02 * (sc6 * sc6 - sc6) + (r - cut) * fc
    assert abs(U - 0.5 * u.sum()) <= 1e-12 * abs(u).sum()
    assert np.max(np.abs(F)) <= 1e-12


def _harmonic(k_spring, centre):
    def f(R, q, step):
        d = R - centre
        return -k_spring * d, q, {"H": 0.5 * k_spring * float((d * d).sum()), "U_lj": 0.0}
    return f


def _toy(n, p, groups=None, kspring=0.05, seed=1):
    w = synth.tiny_cell()
    centre = 0.5 * np.asarray(w.box)[None, :] * np.ones((n, 1))
    rng = np.random.default_rng(seed)
    R = centre + rng.normal(size=(n, 3)) * 0.3
    V = rng.normal(size=(n, 3)) * 2e-3
    types = np.arange(n) % 2
    groups = np.zeros(n, int) if groups is None else np.asarray(groups)
    w = synth.dataclasses.replace(w, elyt_xyz=[R], elyt_q=[np.zeros(n)])
    integ = md.Integrator(w, types, groups, p, force_fn=_harmonic(kspring, centre))
    st = md.initial_state(R, V, w.n_elec, integ.n_groups)
    return integ, st, centre


def test_velocity_verlet_matches_the_stormer_recurrence_solution():
    p = md.MDParams(dt=2.0, t_damp=0.0, mass=(100.0, 100.0))
    integ, st, centre = _toy(1, p)
    k = 0.05
    omega2 = k / (100.0 * md.MVV2E)
    x0 = st.R[0] - centre[0]
    v0 = st.V[0].copy()
    integ.run(st, 1000)
    c = 1 - 0.5 * omega2 * p.dt ** 2
    th = math.acos(c)
    x1 = x0 + p.dt * v0 - 0.5 * p.dt ** 2 * omega2 * x0
    B = (x1 - x0 * c) / math.sin(th)
    expect = x0 * math.cos(1000 * th) + B * math.sin(1000 * th)
    assert np.max(np.abs((st.R[0] - centre[0]) - expect)) <= 1e-10


def _nh_rhs(n, m, k, centre, gkt, Qm):
    def rhs(t, y):
        x = y[:3 * n].reshape(n, 3)
        v = y[3 * n:6 * n].reshape(n, 3)
        xi, vxi = y[6 * n], y[6 * n + 1]
        a = (-k * (x - centre)) / (m[:, None] * md.MVV2E) - vxi * v
        K = 0.5 * md.MVV2E * float((m[:, None] * v * v).sum())
        return np.concatenate([v.ravel(), a.ravel(), [vxi, (2 * K - gkt) / Qm]])
    return rhs


def test_nose_hoover_trotter_converges_to_the_equations_of_motion():
    n, T, tau = 4, 400.0, 20.0
    errs = []
    for dt in (0.5, 0.25):
        p = md.MDParams(dt=dt, t_damp=tau, temperature=T, mass=(100.0, 120.0))
        integ, st, centre = _toy(n, p, kspring=0.02)
        y0 = np.concatenate([st.R.ravel(), st.V.ravel(), [0.0, 0.0]])
        steps = int(round(200.0 / dt))
        integ.run(st, steps)
        gkt = 3 * n * md.KB * T
        sol = solve_ivp(_nh_rhs(n, integ.m, 0.02, centre, gkt, gkt * tau * tau), (0.0, 200.0), y0,
                        rtol=1e-11, atol=1e-13, method="DOP853")
        yT = sol.y[:, -1]
        errs.append(max(np.max(np.abs(st.R.ravel() - yT[:3 * n])), abs(st.xi[0] - yT[6 * n])))
        assert abs(st.vxi[0] - yT[6 * n + 1]) <= 1e-3 * max(1e-6, abs(yT[6 * n + 1])) + 1e-7
    assert errs[1] <= 1e-4
    assert 3.0 <= errs[0] / errs[1] <= 5.0          # second order in dt


def test_thermostat_groups_are_independent():
    """Two uncoupled groups: running them together equals running each alone."""
    p = md.MDParams(dt=1.0, t_damp=30.0)
    groups = np.array([0, 0, 0, 1, 1])
    integ, st, _ = _toy(5, p, groups=groups)
    R0, V0 = st.R.copy(), st.V.copy()
    integ.run(st, 300)
    for g in (0, 1):
        sel = groups == g
        solo, st1, centre = _toy(int(sel.sum()), p)
        st1.R, st1.V = R0[sel].copy(), V0[sel].copy()
        solo.types = integ.types[sel]
        solo.m = integ.m[sel]
        solo.run(st1, 300)
        assert np.max(np.abs(st1.R - st.R[sel])) <= 1e-12
        assert abs(st1.xi[0] - st.xi[g]) <= 1e-12


def _cpm_md(k, dt, t_damp=0.0, n_pairs=4, seed=7):
    # alpha = 0.35: erfc(alpha r_c) ~ 3e-9, so pairs crossing the real-space cutoff make no visible
    # energy jumps (at alpha = 0.25 they are ~1e-5 eV, as large as the integration error)
    w = synth.dataclasses.replace(synth.tiny_cell(seed=seed, n_pairs=n_pairs), alpha=0.35)
    mi = synth.md_inputs(w, seed=3)
    p = md.MDParams(dt=dt, charge_every=k, mass=mi.mass, sigma=mi.sigma, eps=mi.eps, elec_type=mi.elec_type,
                    lj_cut=7.0, temperature=mi.temperature, t_damp=t_damp)
    integ = md.Integrator(w, mi.types, mi.groups, p)
    st = md.initial_state(w.elyt_xyz[0], mi.vel, w.n_elec, integ.n_groups)
    return integ, st


def test_cpm_md_energy_conservation_is_second_order():
    spread = []
    for dt, n in ((2.0, 10), (1.0, 20)):
        integ, st = _cpm_md(1, dt)
        integ.start(st)
        e = [integ.conserved(st)["E_total"]]
        for _ in range(n):
            integ.run(st, 1)
            e.append(integ.conserved(st)["E_total"])
        spread.append(max(e) - min(e))
        assert spread[-1] <= 5e-5 * integ.conserved(st)["KE"]
    assert 2.5 <= spread[0] / spread[1] <= 6.0


def test_cpm_md_is_time_reversible():
    integ, st = _cpm_md(1, 2.0)
    R0, V0 = st.R.copy(), st.V.copy()
    integ.run(st, 8)
    st.V *= -1.0
    integ.run(st, 8)
    d = st.R - R0
    d[:, :2] -= np.asarray(integ.w.box)[:2] * np.round(d[:, :2] / np.asarray(integ.w.box)[:2])
    assert np.max(np.abs(d)) <= 1e-9
    assert np.max(np.abs(st.V + V0)) <= 1e-11


def test_charges_change_only_every_k_steps():
    integ, st = _cpm_md(3, 2.0, t_damp=100.0)
    integ.start(st)
    qs = [st.q.copy()]
    for _ in range(6):
        integ.run(st, 1)
        qs.append(st.q.copy())
    for n in range(1, 7):
        same = np.array_equal(qs[n], qs[n - 1])
        assert same == (n % 3 != 0)
