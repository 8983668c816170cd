"""Pins of the FP64 oracle to facts fixed outside the oracle itself (CPU only).

The paper prints no worked numeric example, so each part of the oracle is tied to a closed form,
a textbook lattice sum, an independent route to the same number, or an invariant that a dropped
term, a wrong sign or a transposed index would break:

* point-charge Ewald core          -> NaCl and CsCl Madelung constants (1e-8)
* Gaussian kernels and self terms  -> radial / angular quadrature of Eq. 2 densities
* A (incl. Gaussian self term) and b -> pure reciprocal-space sums of the Gaussian densities,
                                       a route with no real-space split and no alpha at all
* Ewald split                      -> alpha-invariance of A, b and the energy
* charges                          -> KKT residual, neutrality, optimality under perturbation,
                                      the paper's projector closed forms (Eqs. 8-9, 13-15)
* geometries                       -> empty capacitor: finite field, doubled cell and a
                                      large-vacuum slab agree; parallel-plate capacitance
* forces                           -> central finite differences of the energy, envelope theorem
* energy                           -> closed form at the optimum
"""
import dataclasses
import math
import os

import numpy as np
import pytest
from scipy import integrate
from scipy.special import erf

import synth
from oracle import cpm, ewald
from oracle.ewald import KE

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _madelung():
    vals = {}
    with open(os.path.join(GOLDEN, "madelung.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


def _point_energy(P, c, box, alpha, rcut):
    phi = ewald.real_space(P, P, c, box, rcut, alpha, None, same=True)
    phi += ewald.recip_space(P, P, c, box, alpha)
    return 0.5 * c @ phi - alpha / math.sqrt(math.pi) * c @ c


@pytest.mark.parametrize("alpha", [0.5, 0.8])
def test_madelung_nacl(alpha):
    a = 5.64
    box = np.array([a, a, a])
    fcc = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]]) * a
    P = np.vstack([fcc, fcc + np.array([0.5 * a, 0, 0])])
    c = np.array([1.0] * 4 + [-1.0] * 4)
    E = _point_energy(P, c, box, alpha, 12.0)
    M = -E / 4.0 * (a / 2.0)
    assert abs(M - _madelung()["NaCl"]) < 1e-8


def test_madelung_cscl():
    a = 4.12
    box = np.array([a, a, a])
    P = np.array([[0, 0, 0], [0.5 * a, 0.5 * a, 0.5 * a]])
    c = np.array([1.0, -1.0])
    E = _point_energy(P, c, box, 0.6, 11.0)
    r0 = a * math.sqrt(3.0) / 2.0
    assert abs(-E * r0 - _madelung()["CsCl"]) < 1e-8


def _gauss_density(s, eta):
    return eta ** 3 * math.pi ** -1.5 * np.exp(-(eta * s) ** 2)


def _gauss_potential_quad(r, eta):
    """Potential of a unit Gaussian (Eq. 2) at distance r by the shell theorem."""
    inner = integrate.quad(lambda s: _gauss_density(s, eta) * s * s, 0, r, epsabs=1e-15)[0]
    outer = integrate.quad(lambda s: _gauss_density(s, eta) * s, r, np.inf, epsabs=1e-15)[0]
    return 4 * math.pi * (inner / r + outer)


@pytest.mark.parametrize("r", [0.3, 1.0, 2.7, 6.0])
def test_gaussian_point_kernel_quadrature(r):
    eta, alpha = synth.PAPER_ETA, 0.25
    quad = _gauss_potential_quad(r, eta)
    split = ewald.screened(r, alpha, eta) + erf(alpha * r) / r   # real + reciprocal pieces
    assert abs(split - quad) < 1e-11


@pytest.mark.parametrize("r", [0.5, 1.5, 4.0])
def test_gaussian_gaussian_kernel_quadrature(r):
    """Interaction of two unit Gaussians: integrate one density against the other's potential."""
    eta, alpha = synth.PAPER_ETA, 0.25

    def pot(d):
        return erf(eta * d) / d if d > 1e-12 else 2 * eta / math.sqrt(math.pi)

    def integrand(ct, s):
        d = math.sqrt(max(s * s + r * r - 2 * s * r * ct, 0.0))
        return _gauss_density(s, eta) * pot(d) * 2 * math.pi * s * s

    quad = integrate.dblquad(integrand, 0, 8.0 / eta, -1, 1, epsabs=1e-13, epsrel=1e-12)[0]
    split = ewald.screened(r, alpha, eta / math.sqrt(2)) + erf(alpha * r) / r
    assert abs(split - quad) < 1e-9


def test_gaussian_self_energy_quadrature():
    """Half the self-interaction of a unit Gaussian equals eta/sqrt(2 pi), the oracle's self term
    (which enters A's diagonal doubled, together with -2 alpha/sqrt(pi))."""
    eta = synth.PAPER_ETA
    quad = 0.5 * integrate.quad(lambda s: _gauss_density(s, eta) * erf(eta * s) / s * 4 * math.pi * s * s,
                                0, np.inf, epsabs=1e-15)[0]
    assert abs(quad - eta / math.sqrt(2 * math.pi)) < 1e-12


def _tiny_mixed_cell(seed=11):
    rng = np.random.default_rng(seed)
    box = np.array([6.0, 7.0, 8.0])
    E = rng.uniform(0, 1, (4, 3)) * box
    R = rng.uniform(0, 1, (4, 3)) * box
    q = rng.normal(size=4)
    q -= q.mean()
    Q = rng.normal(size=4)
    Q -= Q.mean()
    w = synth.Workload("pin", box, E, np.array([1, 1, -1, -1]), None, np.zeros(4, np.int32), [R], [Q],
                       np.array([0.0]), "dc", eta=synth.PAPER_ETA, alpha=0.5, rcut=12.0)
    return w, E, R, q, Q


def _full_kspace_sum(box, kmax):
    m = [np.arange(-int(kmax * L / (2 * math.pi)) - 1, int(kmax * L / (2 * math.pi)) + 2) for L in box]
    mm = np.stack(np.meshgrid(*m, indexing="ij"), -1).reshape(-1, 3)
    mm = mm[np.any(mm != 0, axis=1)]
    k = 2 * math.pi * mm / box
    k2 = (k * k).sum(1)
    keep = k2 <= kmax * kmax
    return k[keep], k2[keep]


def test_pure_reciprocal_gaussian_energy_and_b():
    """Neutral Gaussian charges: 1/2 q^T A q is the tin-foil energy of the smooth density
    sum_i q_i n_i(r), which in Fourier space is (2 pi / V) sum_k exp(-k^2/2 eta^2)/k^2 |S_q(k)|^2.
    b_i is minus the potential of the point charges smeared by site i's Gaussian:
    (4 pi / V) sum_k exp(-k^2/4 eta^2)/k^2 sum_j Q_j cos(k.(r_i - R_j)).  No alpha enters."""
    w, E, R, q, Q = _tiny_mixed_cell()
    V = float(np.prod(w.box))
    eta = w.eta
    k, k2 = _full_kspace_sum(w.box, 2 * eta * 6.2)
    sq = np.exp(1j * (E @ k.T)).T @ q
    e_gg = KE * (2 * math.pi / V) * np.sum(np.exp(-k2 / (2 * eta ** 2)) / k2 * np.abs(sq) ** 2)
    A = cpm.elastance(w)
    assert abs(0.5 * q @ A @ q - e_gg) < 1e-10 * abs(e_gg)
    wgt = np.exp(-k2 / (4 * eta ** 2)) / k2
    phase = E @ k.T
    sQ = np.exp(1j * (R @ k.T)).T @ Q
    pot = (4 * math.pi / V) * np.real(np.exp(-1j * phase) @ (wgt * sQ))
    b = cpm.b_vector(w, R, Q)
    assert np.max(np.abs(b + KE * pot)) < 1e-10 * np.max(np.abs(b))


@pytest.mark.parametrize("box", [(10.0, 10.0, 10.0), (9.0, 10.5, 12.0)])
def test_mixed_energy_equals_direct_lattice_sum(box):
    """U of Eq. 3 for Gaussian (Eq. 2) and point charges against a plain sum over whole periodic
    images, with no Ewald split: pair kernels erf(eta r / sqrt 2) / r (Gaussian-Gaussian),
    erf(eta r) / r (Gaussian-point), 1 / r (point-point), plus the Gaussian self-energy
    q^2 eta / sqrt(2 pi).  The cell (a point charge +1 with six Gaussians of -1/6 at +-1 A along each
    axis) is neutral with no dipole and no quadrupole, so the image sum over growing boxes
    converges absolutely to the tin-foil lattice energy; eta = 1 A^-1 keeps every intra-cell
    kernel 5-16 % away from 1 / r."""
    box = np.asarray(box)
    eta, d = 1.0, 1.0
    c0 = np.array([4.7, 5.1, 5.3])
    E = c0 + d * np.vstack([np.eye(3), -np.eye(3)])
    q = np.full(6, -1.0 / 6.0)
    R, Q = c0[None, :], np.array([1.0])
    w = synth.Workload("pin", box, E, np.array([1, 1, 1, -1, -1, -1]), None, np.zeros(6, np.int32), [R], [Q],
                       np.array([0.0]), "dc", eta=eta, alpha=0.6, rcut=9.5)
    U = cpm.energies(w, R, Q, q, 0.0)["U"]
    P, c, gauss = np.vstack([E, R]), np.concatenate([q, Q]), [True] * 6 + [False]
    m = np.arange(-6, 7)
    shifts = np.stack(np.meshgrid(m, m, m, indexing="ij"), -1).reshape(-1, 3) * box
    total = eta / math.sqrt(2 * math.pi) * float(q @ q)
    for a in range(7):
        for b in range(7):
            r = np.linalg.norm(P[a] - P[b] + shifts, axis=1)
            if a == b:
                r = r[r > 0]
            if gauss[a] and gauss[b]:
                kern = erf(eta * r / math.sqrt(2)) / r
            elif gauss[a] or gauss[b]:
                kern = erf(eta * r) / r
            else:
                kern = 1.0 / r
            total += 0.5 * c[a] * c[b] * kern.sum()
    assert abs(KE * total - U) <= 1e-10 * abs(U)


def test_alpha_invariance():
    """A (on neutral charge vectors), b and U are physical: they may not depend on the Ewald
    splitting parameter alpha.  A itself carries an alpha-dependent multiple of e e^T (the
    neutralising-background constant of a non-neutral Ewald sum), which neutral q never see."""
    base = synth.tiny_cell(seed=5, n_pairs=3)
    R, Q = base.elyt_xyz[0], base.elyt_q[0]
    res = []
    for alpha in (0.2, 0.25, 0.35):
        w = dataclasses.replace(base, alpha=alpha, rcut=5.9 / alpha)
        kmax = 2 * alpha * 6.1
        A = cpm.elastance(w, kmax)
        b = cpm.b_vector(w, R, Q, kmax)
        q, _ = cpm.solve_charges(cpm.factorize(A), b, cpm.geometry_vector(w), 1.0, cpm.constraints(w))
        U = cpm.energies(w, R, Q, q, 1.0, kmax)["U"]
        res.append((A, b, q, U))
    A0, b0, q0, U0 = res[0]
    n = A0.shape[0]
    P = np.eye(n) - np.ones((n, n)) / n
    for A, b, q, U in res[1:]:
        assert np.max(np.abs(P @ (A - A0) @ P)) < 1e-10 * np.max(np.abs(A0))
        assert np.max(np.abs(b - b0)) < 1e-10 * np.max(np.abs(b0))
        assert np.max(np.abs(q - q0)) < 1e-9 * np.max(np.abs(q0))
        assert abs(U - U0) < 1e-10 * abs(U0)


@pytest.mark.parametrize("geometry", ["ff", "dc", "slab"])
def test_elastance_symmetric_positive_definite(geometry):
    w = synth.tiny_cell(seed=3, geometry=geometry)
    A = cpm.elastance(w)
    assert np.max(np.abs(A - A.T)) <= 1e-15 * np.max(np.abs(A))
    cpm.factorize(A)
    assert np.linalg.eigvalsh(A).min() > 0
    rng = np.random.default_rng(0)
    for _ in range(5):
        x = rng.normal(size=w.n_elec)
        assert x @ A @ x > 0


def test_kkt_residual_neutrality_and_optimality(plain_ff):
    w, ref, out = plain_ff
    q, lam, b = out["q"], out["psibar"], out["b"]
    v = ref.v
    dpsi = float(w.dpsi[0])
    psi = ref.A @ q - b                               # Eq. 4
    assert np.max(np.abs(psi - dpsi * v - lam[0])) < 1e-10   # Eq. 5 (finite-field form, Eq. 11)
    assert abs(q.sum()) < 10 * w.n_elec * np.finfo(float).eps * np.max(np.abs(q))
    F = lambda x: 0.5 * x @ ref.A @ x - x @ (b + dpsi * v)
    f0 = F(q)
    rng = np.random.default_rng(1)
    for _ in range(10):
        d = rng.normal(size=w.n_elec) * 1e-3
        d -= d.mean()
        assert F(q + d) > f0
    # the legacy non-neutral update (Eq. 6 with psibar = 0) is not neutral
    assert abs(cpm.legacy_charges(ref.cho, b, v, dpsi).sum()) > 1e-3


def test_paper_projector_closed_forms_ff(plain_ff):
    w, ref, out = plain_ff
    S = cpm.paper_projected_inverse(ref.A, ref.C)       # O A^-1 (Eqs. 8-9)
    y = out["b"] + float(w.dpsi[0]) * ref.v
    assert np.max(np.abs(S @ y - out["q"])) < 1e-12 * max(1.0, np.max(np.abs(out["q"])))
    assert np.max(np.abs(S - S.T)) < 1e-12 * np.max(np.abs(S))


def test_paper_projector_closed_forms_doubled_cell():
    w = synth.mirror_to_doubled(synth.tiny_cell(seed=9, n_pairs=3), "independent", seed=99)
    ref = cpm.Reference(w)
    out = ref.step(want_forces=False, want_energy=False)
    q = out["q"]
    e1 = (w.elec_cell == 1)
    assert abs(q.sum()) < 1e-12 and abs(q[e1].sum()) < 1e-12          # both sub-cells neutral
    S = cpm.paper_projected_inverse(ref.A, ref.C)                     # O_1 O A^-1 (Eqs. 13-15)
    y = out["b"] + float(w.dpsi[0]) * ref.v
    assert np.max(np.abs(S @ y - q)) < 1e-12 * max(1.0, np.max(np.abs(q)))
    psi = ref.A @ q - out["b"] - float(w.dpsi[0]) * ref.v
    lam = out["psibar"]
    assert np.max(np.abs(psi - lam[0] - lam[1] * e1)) < 1e-10          # Eq. 12


def test_charges_linear_in_dpsi(plain_ff):
    w, ref, out = plain_ff
    R, Q = w.elyt_xyz[0], w.elyt_q[0]
    q0, _, _ = ref.charges(R, Q, 0.0)
    q1, _, _ = ref.charges(R, Q, 1.0)
    q2, _, _ = ref.charges(R, Q, 2.0)
    assert np.max(np.abs(q2 - 2 * q1 + q0)) < 1e-13
    assert np.max(np.abs(out["q"] - q2)) < 1e-13


def test_doubled_cell_mirror_symmetry():
    w = synth.tiny_cell(seed=4, n_pairs=4, geometry="dc")        # electrolyte mirrored as well
    ref = cpm.Reference(w)
    n = w.n_elec // 2
    A = ref.A
    assert np.max(np.abs(A[:n, :n] - A[n:, n:])) < 1e-12 * np.max(np.abs(A))
    assert np.max(np.abs(A[:n, n:] - A[:n, n:].T)) < 1e-12 * np.max(np.abs(A))
    out = ref.step(want_forces=False, want_energy=False)
    q = out["q"]
    assert np.max(np.abs(q[:n] - q[n:])) < 1e-12


def test_doubled_cell_two_mirror_blocks_equal_full_solve():
    """A mirror-symmetric doubled cell has A = [[P, Q], [Q, P]] (sites ordered sub-cell 0, then
    images).  With y+- = y_0 +- y_1 the constrained problem separates: q+- minimises
    1/2 x^T (P +- Q) x - x^T y+- subject to 1^T x = 0, q_0 = (q+ + q-)/2, q_1 = (q+ - q-)/2, and the
    offsets of Eq. 12 are psibar = (mu+ + mu-)/2, psibar_1 = -mu- (A+- q+- = y+- + mu+- 1).  The
    GPU stores the doubled cell this way; this pins the reduction on the oracle's own A, with an
    electrolyte that is not mirrored (q- != 0)."""
    w = synth.mirror_to_doubled(synth.tiny_cell(seed=9, n_pairs=3), "independent", seed=99)
    ref = cpm.Reference(w)
    out = ref.step(want_forces=False, want_energy=False)
    n = w.n_elec // 2
    A = ref.A
    P, Q = A[:n, :n], A[:n, n:]
    y = out["b"] + float(w.dpsi[0]) * ref.v
    one = np.ones((n, 1))
    qpm, mu = [], []
    for sgn in (+1.0, -1.0):
        Ab = P + sgn * Q
        yb = y[:n] + sgn * y[n:]
        x, lam = cpm.solve_charges(cpm.factorize(Ab), yb, np.zeros(n), 0.0, one)
        qpm.append(x)
        mu.append(float(lam[0]))
    q0 = 0.5 * (qpm[0] + qpm[1])
    q1 = 0.5 * (qpm[0] - qpm[1])
    q = out["q"]
    scale = max(1.0, np.max(np.abs(q)))
    assert np.max(np.abs(np.concatenate([q0, q1]) - q)) < 1e-12 * scale
    assert np.max(np.abs(qpm[1])) > 1e-4                               # the difference mode is exercised
    lam = out["psibar"]
    assert abs(0.5 * (mu[0] + mu[1]) - lam[0]) < 1e-10
    assert abs(-mu[1] - lam[1]) < 1e-10


def _empty(w):
    return dataclasses.replace(w, elyt_xyz=[np.zeros((0, 3))], elyt_q=[np.zeros(0)])


def test_empty_capacitor_geometries_agree():
    """Finite field, doubled cell and a 10x-vacuum slab give the same electrode charge for the
    same potential difference (Sec. II.B, Sec. IV.A), and it is close to the parallel-plate value;
    the high-z electrode (d = +1/2) charges positively."""
    w = _empty(synth.config_plain_ff())
    res = {}
    for name, ww in (("ff", w), ("dc", synth.mirror_to_doubled(w, "mirror")),
                     ("slab", dataclasses.replace(w, geometry="slab", slab_factor=10.0))):
        ref = cpm.Reference(ww)
        q, _, _ = ref.charges(np.zeros((0, 3)), np.zeros(0), 1.0)
        sel = ww.elec_side > 0
        if ww.elec_cell is not None:
            sel &= ww.elec_cell == 0
        res[name] = q[sel].sum()
    assert res["ff"] > 0
    assert abs(res["ff"] - res["slab"]) < 1e-3 * res["slab"]
    assert abs(res["dc"] - res["slab"]) < 1e-6 * res["slab"]
    lx, ly, _ = w.box
    plate = lx * ly / (4 * math.pi * KE * 40.0)     # eps0 A / d, 40 A between proximal planes
    assert abs(res["slab"] / plate - 1.0) < 0.05


def test_slab_correction_converges_with_padding():
    w = synth.tiny_cell(seed=8, n_pairs=3)
    out = {}
    for f in (3.0, 6.0):
        ww = dataclasses.replace(w, geometry="slab", slab_factor=f)
        out[f] = cpm.Reference(ww).step(want_forces=False)
    assert np.max(np.abs(out[3.0]["q"] - out[6.0]["q"])) < 2e-3 * np.max(np.abs(out[6.0]["q"]))
    assert abs(out[3.0]["U"] - out[6.0]["U"]) < 1e-3 * abs(out[6.0]["U"])


def test_energy_closed_form_at_optimum(plain_ff):
    """At q*: U = U_elyt - 1/2 q^T b + 1/2 dpsi q^T v (since A q = b + dpsi v + C lam, C^T q = 0)."""
    w, ref, out = plain_ff
    R, Q = w.elyt_xyz[0], w.elyt_q[0]
    q, b = out["q"], out["b"]
    dpsi = float(w.dpsi[0])
    closed = cpm.electrolyte_energy(w, R, Q) - 0.5 * q @ b + 0.5 * dpsi * q @ ref.v
    assert abs(out["U"] - closed) < 1e-12 * abs(out["U"])
    direct = cpm.electrolyte_energy(w, R, Q) - q @ b + 0.5 * q @ ref.A @ q
    assert abs(out["U"] - direct) < 1e-12 * abs(out["U"])


@pytest.mark.parametrize("geometry", ["ff", "dc", "slab"])
def test_forces_are_minus_energy_gradient(geometry):
    """Central differences of H against the analytic forces.  r_c is raised so that erfc(alpha r_c)
    is below 1e-16: the truncated real-space sum jumps where a pair crosses r_c, which a
    finite difference would otherwise pick up."""
    w = synth.tiny_cell(seed=6, n_pairs=3, geometry=geometry)
    if geometry == "dc":
        w = synth.mirror_to_doubled(synth.tiny_cell(seed=6, n_pairs=3), "independent", seed=60)
    w = dataclasses.replace(w, rcut=24.0)
    ref = cpm.Reference(w)
    R, Q = w.elyt_xyz[0].copy(), w.elyt_q[0]
    dpsi = float(w.dpsi[0])
    out = ref.step()
    q, F_l, F_e = out["q"], out["F_elyt"], out["F_elec"]
    h = 1e-4
    scale = np.max(np.abs(F_l))
    for j in range(R.shape[0]):
        for c in range(3):
            Rp, Rm = R.copy(), R.copy()
            Rp[j, c] += h
            Rm[j, c] -= h
            # fixed charges
            fd = -(cpm.energies(w, Rp, Q, q, dpsi)["H"] - cpm.energies(w, Rm, Q, q, dpsi)["H"]) / (2 * h)
            assert abs(fd - F_l[j, c]) < 1e-6 * scale
            if c == 2 and j < 2:
                # charges re-solved at each displaced configuration (envelope theorem)
                qp = ref.charges(Rp, Q, dpsi)[0]
                qm = ref.charges(Rm, Q, dpsi)[0]
                fd2 = -(cpm.energies(w, Rp, Q, qp, dpsi)["H"] - cpm.energies(w, Rm, Q, qm, dpsi)["H"]) / (2 * h)
                assert abs(fd2 - F_l[j, c]) < 1e-6 * scale
    E0 = w.elec_xyz.copy()
    for i in (0, 7, w.n_elec - 1):
        for c in range(3):
            Wp = dataclasses.replace(w, elec_xyz=E0.copy())
            Wm = dataclasses.replace(w, elec_xyz=E0.copy())
            Wp.elec_xyz[i, c] += h
            Wm.elec_xyz[i, c] -= h
            fd = -(cpm.energies(Wp, R, Q, q, dpsi)["H"] - cpm.energies(Wm, R, Q, q, dpsi)["H"]) / (2 * h)
            assert abs(fd - F_e[i, c]) < 1e-6 * max(scale, np.max(np.abs(F_e)))
    total = F_l.sum(0) + F_e.sum(0)
    assert np.max(np.abs(total)) < 1e-9 * scale


@pytest.mark.parametrize("kspace", ["direct", "separable"])
@pytest.mark.parametrize("geometry", ["ff", "dc", "slab"])
def test_sampled_checkers_equal_the_dense_oracle(geometry, kspace):
    """The matrix-free and sampled helpers that check the full-size GPU runs (elastance_apply,
    b_at, electrolyte_forces_at, with either form of the reciprocal sum) against the dense oracle
    they restate (Eq. 3 for A and b, the fixed-charge forces of Sec. II.A), which the pins above
    tie to the paper and to physics: a dropped slab or finite-field term, a wrong target index or
    a missing self term fails here."""
    base = synth.tiny_cell(seed=4, n_pairs=4)
    if geometry == "dc":
        w = synth.mirror_to_doubled(base, "independent", seed=40)
    elif geometry == "slab":
        w = dataclasses.replace(base, geometry="slab")
    else:
        w = base
    R, Q, dpsi = w.elyt_xyz[0], w.elyt_q[0], float(w.dpsi[0])
    rng = np.random.default_rng(11)
    # a charge vector that is neither neutral nor mirror-symmetric, so every column of A counts
    q = 0.02 * rng.standard_normal(w.n_elec)
    A = cpm.elastance(w)
    Aq = A @ q
    assert np.max(np.abs(cpm.elastance_apply(w, q, kspace=kspace) - Aq)) <= 1e-12 * np.max(np.abs(Aq))
    ie = rng.choice(w.n_elec, 19, replace=False)
    assert np.max(np.abs(cpm.elastance_apply(w, q, idx=ie, kspace=kspace) - Aq[ie])) <= 1e-12 * np.max(np.abs(Aq))
    b = cpm.b_vector(w, R, Q)
    assert np.max(np.abs(cpm.b_at(w, R, Q, ie, kspace=kspace) - b[ie])) <= 1e-12 * np.max(np.abs(b))
    F_l, _ = cpm.forces(w, R, Q, q, dpsi)
    il = rng.choice(len(Q), 5, replace=False)
    F_at = cpm.electrolyte_forces_at(w, R, Q, q, dpsi, il, kspace=kspace)
    assert np.max(np.abs(F_at - F_l[il])) <= 1e-12 * np.max(np.abs(F_l))


@pytest.mark.parametrize("box", [(17.04, 17.22, 60.0), (38.34, 34.44, 336.0), (12.0, 13.0, 9.0)])
def test_separable_reciprocal_sum_equals_direct_sum(box):
    """recip_space_separable (per-axis plane-wave tables) is the same sum as recip_space
    (cos/sin per site and k-vector): potentials and gradients agree to rounding."""
    rng = np.random.default_rng(5)
    box = np.asarray(box)
    src = rng.random((300, 3)) * box
    c = rng.standard_normal(300)
    tgt = rng.random((40, 3)) * box
    p1, g1 = ewald.recip_space(tgt, src, c, box, 0.3, want_grad=True)
    p2, g2 = ewald.recip_space_separable(tgt, src, c, box, 0.3, want_grad=True)
    assert np.max(np.abs(p1 - p2)) <= 1e-13 * np.max(np.abs(p1))
    assert np.max(np.abs(g1 - g2)) <= 1e-13 * np.max(np.abs(g1))


def test_hard_truncated_ewald_split_gives_an_indefinite_elastance():
    """The premise of the GPU build's CPM_ERR_NOT_SPD test: with alpha = 0.01 / A and r_c = 2 A
    the truncated sums no longer represent the positive Coulomb energy of Gaussians, and A has
    negative eigenvalues (in the single cell and, z-mirrored, in both mirror blocks P +- Q)."""
    w = dataclasses.replace(synth.tiny_cell(seed=1, n_pairs=2), alpha=0.01, rcut=2.0)
    assert np.linalg.eigvalsh(cpm.elastance(w))[0] < -1.0
    wd = synth.mirror_to_doubled(w, "mirror")
    A = cpm.elastance(wd)
    n = w.n_elec
    P, Q = A[:n, :n], A[:n, n:]
    assert np.linalg.eigvalsh(P + Q)[0] < -1.0 and np.linalg.eigvalsh(P - Q)[0] < -1.0
