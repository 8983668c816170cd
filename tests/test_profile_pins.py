"""Pins of the rho(z) / psi(z) oracle (Sec. II.C) against closed forms (CPU).

* The periodic second difference has the eigenfunctions sin(2 pi m z / L) with eigenvalue
  -(2 - 2 cos(2 pi m h / L)) / h^2, so the discrete solution of psi'' = -4 pi k_e rho for a
  sinusoidal rho is known exactly.
* Two opposite charge sheets +-sigma a distance d apart in a periodic cell of length L: the
  periodic potential is piecewise linear and drops by 4 pi k_e sigma d (L - d) / L from the
  positive to the negative sheet (sign and 4 pi k_e).
* The binned density conserves charge, and the z-projection of an electrode's Gaussian (Eq. 2)
  has second moment 1 / (2 eta^2) (plus h^2 / 12 from binning).
* The finite-field potential rises by dpsi across the cell (continuous ramp, jump at the boundary).
"""
import math

import numpy as np

import synth
from oracle import profile
from oracle.ewald import KE


def test_sinusoid_is_an_exact_discrete_eigenfunction():
    L, n = 136.0, 400
    h = L / n
    z = (np.arange(n) + 0.5) * h
    for m in (1, 3, 17):
        rho = 1e-3 * np.sin(2 * math.pi * m * z / L)
        psi = profile.potential_z(rho, L, geometry="dc")
        expect = 4 * math.pi * KE * rho * h * h / (2 - 2 * math.cos(2 * math.pi * m * h / L))
        assert np.max(np.abs(psi - expect)) <= 1e-10 * np.max(np.abs(expect))


def test_two_charge_sheets_give_the_capacitor_drop():
    L, n = 100.0, 500
    h = L / n
    i1, i2 = 120, 370
    sigma = 2e-3                                      # e / A^2
    rho = np.zeros(n)
    rho[i1] = sigma / h
    rho[i2] = -sigma / h
    psi = profile.potential_z(rho, L, geometry="dc")
    d = (i2 - i1) * h
    drop = 4 * math.pi * KE * sigma * d * (L - d) / L
    assert abs((psi[i1] - psi[i2]) - drop) <= 1e-10 * drop
    # linear between the sheets: constant field
    mid = np.diff(psi[i1 + 1:i2])
    assert np.max(np.abs(mid - mid.mean())) <= 1e-10 * abs(mid.mean())


def test_binned_density_conserves_charge_and_resolves_the_gaussian():
    w = synth.config_plain_ff()
    lx, ly, lz = w.box
    n = 400
    q = np.random.default_rng(3).normal(size=w.n_elec) * 0.01
    rho = profile.charge_density_z(lz, lx * ly, n, w.elyt_xyz[0][:, 2], w.elyt_q[0], w.elec_xyz[:, 2], q, w.eta)
    total = rho.sum() * lx * ly * lz / n
    assert abs(total - (w.elyt_q[0].sum() + q.sum())) <= 1e-12 * max(1.0, np.abs(q).sum())
    # one Gaussian site in the middle of the cell
    zc, eta = 30.123, w.eta
    r1 = profile.charge_density_z(lz, 1.0, 2000, [], [], [zc], [1.0], eta)
    h = lz / 2000
    zb = (np.arange(2000) + 0.5) * h
    wgt = r1 * h
    assert abs(wgt.sum() - 1.0) <= 1e-12
    mean = (wgt * zb).sum()
    var = (wgt * (zb - mean) ** 2).sum()
    assert abs(mean - zc) <= 1e-6
    assert abs(var - (1.0 / (2 * eta * eta) + h * h / 12)) <= 1e-6


def test_finite_field_ramp_jumps_by_dpsi_across_the_boundary():
    L, n = 60.0, 300
    psi = profile.potential_z(np.zeros(n), L, geometry="ff", dpsi=2.0)
    step = psi[1] - psi[0]
    assert abs((psi[-1] - psi[0]) - 2.0 * (n - 1) / n) <= 1e-12
    assert abs(step - 2.0 / n) <= 1e-12
    assert abs((psi[0] + 2.0 - psi[-1]) - step) <= 1e-12   # periodic image one cell up: +dpsi


def test_all_layer_charging_puts_most_charge_on_the_proximal_layers():
    """With all three layers charged (the snapshot re-run of Appendix B), the proximal layers carry
    more than 90 % of each electrode's induced charge (Sec. IV.C), and charging only the proximal
    layers gives each electrode nearly the same total charge."""
    from oracle import cpm
    w = synth.config_plain_ff()
    out = cpm.Reference(w).step(want_forces=False, want_energy=False)
    q = out["q"]
    for side in (+1, -1):
        on = w.elec_side == side
        total = q[on].sum()
        prox = q[on & (w.elec_layer == 0)].sum()
        assert abs(total) > 1e-3
        assert prox / total > 0.9
    wp = synth.proximal_only(w)
    assert wp.n_elec * 3 == w.n_elec
    outp = cpm.Reference(wp).step(want_forces=False, want_energy=False)
    qp = outp["q"]
    for side in (+1, -1):
        full = q[w.elec_side == side].sum()
        assert abs(qp[wp.elec_side == side].sum() - full) <= 0.1 * abs(full)
