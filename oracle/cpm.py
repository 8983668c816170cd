"""FP64 constant-potential-method (CPM) oracle: elastance A, vector b, charges q, energy, forces.

Test infrastructure: only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg use this
module; the GPU library does not.  It follows Sec. II of the paper step by step in FP64:

* Eq. 3: U = U_elyt - q^T b + 1/2 q^T A q.  A (electrode-electrode) and b (electrolyte-electrode)
  come from the Ewald pieces of oracle.ewald; b is minus the electrolyte potential at each
  electrode site, so that Eq. 4 reads Psi = A q - b.
* Eqs. 5-9: each electrode sits at its set potential Psi = psibar e + dpsi d, with the total
  charge constrained to zero.  Eqs. 12-15 add a second offset and constraint for the doubled cell.
  These closed forms all describe the unique minimiser of 1/2 q^T A q - q^T (b + dpsi v) subject
  to C^T q = 0 (A is symmetric positive definite), which solve_charges computes directly by a
  dense Cholesky factorisation and the KKT system; psibar is the constraint multiplier.
* Geometry (Sec. II.B): finite field (Eqs. 10-11, v = d - z/L_z with the electrode z unwrapped so
  that the electrolyte lies between the electrodes, d = +1/2 on the high-z electrode; constant
  shifts of v along e are removed by the neutrality constraint), doubled cell (Eqs. 12-15,
  v = d, C = [e, e_1]) and slab with the Yeh-Berkowitz dipole correction (Sec. II.B, v = d).

Energies returned: U, the Coulomb energy of Eq. 3 (plus the slab correction), and
H = U - dpsi q^T v (+ dpsi/L_z sum_j Q_j Z_j for the finite field), the constant-potential
energy whose gradient at the constrained optimum is minus the force (dH/dq is parallel to the
constraints there, so the charge response drops out).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.linalg import cho_factor, cho_solve

from .ewald import (KE, SQRT2, SQRT_PI, default_kmax, image_shifts, real_space, recip_matrix,
                    recip_space, screened, recip_space_separable)


# ----------------------------------------------------------------------------------------------
# geometry helpers (Sec. II.B)
# ----------------------------------------------------------------------------------------------
def ewald_box(w) -> np.ndarray:
    """Periodic box used by the Ewald sums: the slab geometry pads z by slab_factor.
    Sec. II.B (slab comparison geometry: vacuum padding in z)."""
    box = np.asarray(w.box, np.float64).copy()
    if w.geometry == "slab":
        box[2] *= w.slab_factor
    return box


def geometry_vector(w) -> np.ndarray:
    """v such that the electrode target potentials are psibar-terms + dpsi v.

    d = +1/2 on side +1 and -1/2 on side -1 (Eq. 5).  Finite field (Eq. 11): v = d - z/L_z.
    """
    d = 0.5 * np.asarray(w.elec_side, np.float64)
    if w.geometry == "ff":
        return d - w.elec_xyz[:, 2] / float(w.box[2])
    return d


def constraints(w) -> np.ndarray:
    """Constraint matrix C: [e] (Eq. 7) or, for the doubled cell, [e, e_1] (Eq. 12)."""
    e = np.ones((w.n_elec, 1))
    if w.geometry == "dc":
        e1 = (np.asarray(w.elec_cell) == 1).astype(np.float64)[:, None]
        return np.hstack([e, e1])
    return e


# ----------------------------------------------------------------------------------------------
# A and b (Eq. 3)
# ----------------------------------------------------------------------------------------------
def real_space_matrix(pa, pb, box, rcut, alpha, beta, same=False, chunk=512) -> np.ndarray:
    """Sum over periodic images within r_c of the real-space kernel between every pair (a, b).
    Sec. II.B: the real-space part of the Ewald split of Eq. 3's pair terms."""
    box = np.asarray(box, np.float64)
    na, nb = pa.shape[0], pb.shape[0]
    M = np.zeros((na, nb))
    rc2 = rcut * rcut
    for a in range(0, na, chunk):
        b = min(na, a + chunk)
        d0 = pa[a:b, None, :] - pb[None, :, :]
        d0 -= box * np.round(d0 / box)
        for s in image_shifts(box, rcut):
            d = d0 + s
            r2 = np.einsum("ijk,ijk->ij", d, d)
            m = r2 < rc2
            if same and not np.any(s):
                ii = np.arange(b - a)
                m[ii, a + ii] = False
            r = np.sqrt(np.where(m, r2, 1.0))
            M[a:b] += np.where(m, screened(r, alpha, beta), 0.0)
    return M


def elastance(w, kmax=None) -> np.ndarray:
    """A_ii' = KE [ sum_images gg-kernel + reciprocal + delta_ii' (sqrt2 eta - 2 alpha)/sqrt pi ]
    (+ KE 4 pi/V z z^T for the slab correction).  The diagonal term is the Gaussian self-energy
    (eta/sqrt(2 pi) per unit charge squared, doubled by the 1/2 of Eq. 3) minus the Ewald point
    self-term (alpha/sqrt pi, doubled likewise)."""
    box = ewald_box(w)
    E = np.asarray(w.elec_xyz, np.float64)
    A = real_space_matrix(E, E, box, w.rcut, w.alpha, w.eta / SQRT2, same=True)
    A += recip_matrix(E, box, w.alpha, kmax)
    A[np.diag_indices_from(A)] += (SQRT2 * w.eta - 2.0 * w.alpha) / SQRT_PI
    A *= KE
    if w.geometry == "slab":
        V = float(np.prod(box))
        z = E[:, 2]
        A += KE * (4.0 * math.pi / V) * np.outer(z, z)
    return A


def elastance_apply(w, q, kmax=None, idx=None, kspace="direct") -> np.ndarray:
    """A q without forming A: the potential (V) at each electrode site (or at the sites idx only)
    due to the Gaussian charges q (used for residual checks where N_e is too large for a dense A).
    kspace="separable" evaluates the reciprocal sum through recip_space_separable (the same sum).
    Eq. 3 (A), Eq. 4 (Psi = A q - b)."""
    box = ewald_box(w)
    E = np.asarray(w.elec_xyz, np.float64)
    T = E if idx is None else E[idx]
    rec = _recip(kspace)
    phi = real_space(T, E, q, box, w.rcut, w.alpha, w.eta / SQRT2, same=True, target_index=idx)
    phi += rec(T, E, q, box, w.alpha, kmax)
    qt = q if idx is None else q[idx]
    phi += (SQRT2 * w.eta - 2.0 * w.alpha) / SQRT_PI * qt
    phi *= KE
    if w.geometry == "slab":
        V = float(np.prod(box))
        phi += KE * (4.0 * math.pi / V) * T[:, 2] * float(E[:, 2] @ q)
    return phi


def _recip(kspace):
    """The reciprocal-sum routine: the direct cos/sin sum or its per-axis factorised form."""
    if kspace == "direct":
        return recip_space
    if kspace == "separable":
        return recip_space_separable
    raise ValueError(f"kspace must be 'direct' or 'separable', got {kspace!r}")


def b_vector(w, R, Q, kmax=None) -> np.ndarray:
    """b_i = -(potential at electrode site i due to the electrolyte point charges), Eq. 3."""
    box = ewald_box(w)
    E = np.asarray(w.elec_xyz, np.float64)
    phi = real_space(E, R, Q, box, w.rcut, w.alpha, w.eta)
    phi += recip_space(E, R, Q, box, w.alpha, kmax)
    b = -KE * phi
    if w.geometry == "slab":
        V = float(np.prod(box))
        b -= KE * (4.0 * math.pi / V) * E[:, 2] * float(np.dot(Q, R[:, 2]))
    return b


# ----------------------------------------------------------------------------------------------
# charges (Eqs. 5-15, as the constrained minimiser)
# ----------------------------------------------------------------------------------------------
def factorize(A):
    """Dense Cholesky factor of A (raises numpy.linalg.LinAlgError if A is not SPD).
    Eq. 3: A is the matrix of a positive electrostatic self-energy of the Gaussians (Sec. II.A)."""
    return cho_factor(A, lower=True, check_finite=True)


def solve_charges(cho, b, v, dpsi, C):
    """Minimise 1/2 q^T A q - q^T y, y = b + dpsi v, subject to C^T q = 0.

    Stationarity: A q - y = C lam, so q = A^-1 (y + C lam) and
    lam = -(C^T A^-1 C)^-1 C^T A^-1 y.  lam holds the offset potentials (psibar[, psibar_1]).
    Eqs. 4-7 (one constraint), Eq. 12 (doubled cell: the second offset).
    """
    y = b + dpsi * v
    ainv_y = cho_solve(cho, y)
    ainv_c = cho_solve(cho, C)
    lam = -np.linalg.solve(C.T @ ainv_c, C.T @ ainv_y)
    q = ainv_y + ainv_c @ lam
    return q, lam


def paper_projected_inverse(A, C):
    """The paper's closed forms: O A^-1 (Eqs. 8-9) or, with a second column e_1, O_1 O A^-1
    (Eqs. 13-15).  Independent algebraic route used to cross-check solve_charges."""
    n = A.shape[0]
    Ainv = np.linalg.inv(A)
    e = C[:, :1]
    O = np.eye(n) - (Ainv @ e @ e.T) / (e.T @ Ainv @ e).item()
    OA = O @ Ainv
    if C.shape[1] == 1:
        return OA
    e1 = C[:, 1:2]
    O1 = np.eye(n) - (OA @ e1 @ e1.T) / (e1.T @ OA @ e1).item()
    return O1 @ OA


def legacy_charges(cho, b, v, dpsi):
    """Eq. 6 with psibar = 0 (the non-neutral legacy update); used only as a negative check."""
    return cho_solve(cho, b + dpsi * v)


# ----------------------------------------------------------------------------------------------
# energy and forces
# ----------------------------------------------------------------------------------------------
def _site_potentials(w, R, Q, q, want_grad, kmax=None):
    """Potential (and gradient) at every electrode and electrolyte site due to all other charges,
    kind-dependent real space plus reciprocal space over all charges as points.  No KE."""
    box = ewald_box(w)
    E = np.asarray(w.elec_xyz, np.float64)
    a, eta, rc = w.alpha, w.eta, w.rcut
    out = {}
    out["ee"] = real_space(E, E, q, box, rc, a, eta / SQRT2, same=True, want_grad=want_grad)
    out["el"] = real_space(E, R, Q, box, rc, a, eta, want_grad=want_grad)
    out["le"] = real_space(R, E, q, box, rc, a, eta, want_grad=want_grad)
    out["ll"] = real_space(R, R, Q, box, rc, a, None, same=True, want_grad=want_grad)
    P = np.vstack([E, R])
    c = np.concatenate([q, Q])
    out["k"] = recip_space(P, P, c, box, a, kmax, want_grad=want_grad)
    return out


def energies(w, R, Q, q, dpsi, kmax=None) -> dict:
    """Full Ewald energy of electrode Gaussians q and electrolyte points Q (eV).

    U = KE [ 1/2 sum_a c_a phi_real,a + 1/2 sum_a c_a phi_k,a - alpha/sqrt pi sum c^2
             + eta/sqrt(2 pi) sum q^2 ] (+ KE 2 pi/V M_z^2 for the slab),
    H = U - dpsi q^T v (+ dpsi/L_z sum_j Q_j Z_j for the finite field); also the explicit
    derivative dH/d(dpsi) at fixed charges and the total charge Q_+ of the side +1 electrode.
    Eqs. 1 and 3; finite field: the field term of Sec. II.B (Eqs. 10-11, with the sign that Eq. 11
    implies); slab: the Yeh-Berkowitz term.
    """
    box = ewald_box(w)
    E = np.asarray(w.elec_xyz, np.float64)
    p = _site_potentials(w, R, Q, q, want_grad=False, kmax=kmax)
    c = np.concatenate([q, Q])
    e_real = 0.5 * q @ p["ee"] + q @ p["el"] + 0.5 * Q @ p["ll"]
    e_recip = 0.5 * c @ p["k"]
    e_self = -(w.alpha / SQRT_PI) * float(c @ c) + (w.eta / math.sqrt(2.0 * math.pi)) * float(q @ q)
    U = KE * (e_real + e_recip + e_self)
    if w.geometry == "slab":
        V = float(np.prod(box))
        mz = float(q @ E[:, 2] + Q @ R[:, 2])
        U += KE * (2.0 * math.pi / V) * mz * mz
    v = geometry_vector(w)
    dH = -float(q @ v)
    if w.geometry == "ff":
        dH += float(Q @ R[:, 2]) / float(w.box[2])
    H = U + dpsi * dH
    return {"U": U, "H": H, "dH_ddpsi": dH, "Q_plus": float(q[np.asarray(w.elec_side) > 0].sum())}


def electrolyte_energy(w, R, Q, kmax=None) -> float:
    """U_elyt of Eq. 3: the Ewald energy of the electrolyte point charges alone (eV)."""
    box = ewald_box(w)
    phi = real_space(R, R, Q, box, w.rcut, w.alpha, None, same=True)
    phi += recip_space(R, R, Q, box, w.alpha, kmax)
    U = KE * (0.5 * Q @ phi - (w.alpha / SQRT_PI) * float(Q @ Q))
    if w.geometry == "slab":
        V = float(np.prod(box))
        mz = float(Q @ R[:, 2])
        U += KE * (2.0 * math.pi / V) * mz * mz
    return U


def forces(w, R, Q, q, dpsi, kmax=None):
    """Forces (eV/A) on electrolyte and electrode sites at fixed charges: F = -dH/dr.

    Electrostatic part -c_a grad phi_a; slab correction -KE 4 pi/V c_a M_z z-hat; finite field
    -c_a dpsi/L_z z-hat (the applied field E_z = -dpsi/L_z of Sec. II.B.1).
    """
    box = ewald_box(w)
    E = np.asarray(w.elec_xyz, np.float64)
    p = _site_potentials(w, R, Q, q, want_grad=True, kmax=kmax)
    ne = E.shape[0]
    gk = p["k"][1]
    g_e = p["ee"][1] + p["el"][1] + gk[:ne]
    g_l = p["le"][1] + p["ll"][1] + gk[ne:]
    F_e = -KE * q[:, None] * g_e
    F_l = -KE * Q[:, None] * g_l
    if w.geometry == "slab":
        V = float(np.prod(box))
        mz = float(q @ E[:, 2] + Q @ R[:, 2])
        F_e[:, 2] -= KE * (4.0 * math.pi / V) * q * mz
        F_l[:, 2] -= KE * (4.0 * math.pi / V) * Q * mz
    if w.geometry == "ff":
        F_e[:, 2] -= q * dpsi / float(w.box[2])
        F_l[:, 2] -= Q * dpsi / float(w.box[2])
    return F_l, F_e


# ----------------------------------------------------------------------------------------------
# one full step
# ----------------------------------------------------------------------------------------------
class Reference:
    """Caches A and its Cholesky factor for one electrode geometry (Sec. II.A: A is constant for
    fixed electrodes and its inverse is precomputed once)."""

    def __init__(self, w, kmax=None):
        self.w = w
        self.kmax = kmax
        self.A = elastance(w, kmax)
        self.cho = factorize(self.A)
        self.C = constraints(w)
        self.v = geometry_vector(w)

    def charges(self, R, Q, dpsi):
        """b (Eq. 3) for the electrolyte (R, Q) and the constrained charges (Eqs. 4-7, 12)."""
        b = b_vector(self.w, R, Q, self.kmax)
        q, lam = solve_charges(self.cho, b, self.v, dpsi, self.C)
        return q, lam, b

    def step(self, r=0, want_forces=True, want_energy=True) -> dict:
        """Charges, offsets, b, energies and forces for replica r.  Sec. II.A-B: one full step of the method."""
        w = self.w
        R, Q, dpsi = w.elyt_xyz[r], w.elyt_q[r], float(w.dpsi[r])
        q, lam, b = self.charges(R, Q, dpsi)
        out = {"q": q, "psibar": lam, "b": b}
        if want_energy:
            out.update(energies(w, R, Q, q, dpsi, self.kmax))
        if want_forces:
            out["F_elyt"], out["F_elec"] = forces(w, R, Q, q, dpsi, self.kmax)
        return out

    def sampled_step(self, r=0, frac=0.1, seed=0):
        """A bounded timing sample of step(r): every real-space sum restricted to a random fraction
        `frac` of its target sites and every reciprocal sum to a random fraction `frac` of the
        k-vectors, with the KKT solve in full.  Its cost is close to `frac` times that of a full
        step; the values it produces are partial sums and are not returned.
        Sec. II.A-B (the sums of step(), partially)."""
        w = self.w
        R, Q, dpsi = w.elyt_xyz[r], w.elyt_q[r], float(w.dpsi[r])
        sampled_step_sums(w, R, Q, frac, seed, self.kmax,
                          solve=lambda b: solve_charges(self.cho, b, self.v, dpsi, self.C)[0])


def sampled_step_sums(w, R, Q, frac, seed, kmax=None, solve=None, q=None):
    """The sums of one step (b; then, at the electrode charges, the energy and force sums) with
    every real-space sum restricted to a random fraction `frac` of its target sites and every
    reciprocal sum to a random fraction `frac` of the k-vectors: a bounded timing sample whose
    cost is close to `frac` times that of the full sums.  The charges come from solve(b) (the KKT
    solve, Reference.sampled_step) or are given as q where the dense A cannot be formed (tens of
    thousands of sites).  The values are partial sums and are not returned.
    Sec. II.A-B (the sums of a step, partially)."""
    rng = np.random.default_rng(seed)
    box = ewald_box(w)
    E = np.asarray(w.elec_xyz, np.float64)
    a, eta, rc = w.alpha, w.eta, w.rcut
    te = np.flatnonzero(rng.random(E.shape[0]) < frac)
    tl = np.flatnonzero(rng.random(R.shape[0]) < frac)

    def ksub(n):
        return rng.random(n) < frac

    b = np.zeros(E.shape[0])
    b[te] = -KE * real_space(E[te], R, Q, box, rc, a, eta)
    b -= KE * recip_space(E, R, Q, box, a, kmax, ksub=ksub)
    if solve is not None:
        q = solve(b)
    P = np.vstack([E, R])
    c = np.concatenate([q, Q])
    for grad in (False, True):       # a step evaluates energies, then forces
        real_space(E[te], E, q, box, rc, a, eta / SQRT2, same=True, want_grad=grad, target_index=te)
        real_space(E[te], R, Q, box, rc, a, eta, want_grad=grad)
        real_space(R[tl], E, q, box, rc, a, eta, want_grad=grad)
        real_space(R[tl], R, Q, box, rc, a, None, same=True, want_grad=grad, target_index=tl)
        recip_space(P, P, c, box, a, kmax, want_grad=grad, ksub=ksub)


# ----------------------------------------------------------------------------------------------
# sampled checks for workloads too large for a dense oracle solve
# ----------------------------------------------------------------------------------------------
def b_at(w, R, Q, idx, kmax=None, kspace="direct") -> np.ndarray:
    """b_i (Eq. 3) at the electrode sites idx only (kspace as in elastance_apply)."""
    box = ewald_box(w)
    E = np.asarray(w.elec_xyz, np.float64)[idx]
    phi = real_space(E, R, Q, box, w.rcut, w.alpha, w.eta)
    phi += _recip(kspace)(E, R, Q, box, w.alpha, kmax)
    b = -KE * phi
    if w.geometry == "slab":
        V = float(np.prod(box))
        b -= KE * (4.0 * math.pi / V) * E[:, 2] * float(np.dot(Q, R[:, 2]))
    return b


def electrolyte_forces_at(w, R, Q, q, dpsi, idx, kmax=None, kspace="direct") -> np.ndarray:
    """Forces on the electrolyte sites idx for given electrode charges q (as in forces()):
    minus the gradient of Eq. 3 at fixed q (Sec. II.A); kspace as in elastance_apply."""
    box = ewald_box(w)
    E = np.asarray(w.elec_xyz, np.float64)
    T = R[idx]
    _, g_le = real_space(T, E, q, box, w.rcut, w.alpha, w.eta, want_grad=True)
    _, g_ll = real_space(T, R, Q, box, w.rcut, w.alpha, None, same=True, want_grad=True, target_index=idx)
    P = np.vstack([E, R])
    c = np.concatenate([q, Q])
    _, g_k = _recip(kspace)(T, P, c, box, w.alpha, kmax, want_grad=True)
    F = -KE * Q[idx, None] * (g_le + g_ll + g_k)
    if w.geometry == "slab":
        V = float(np.prod(box))
        mz = float(q @ E[:, 2] + Q @ R[:, 2])
        F[:, 2] -= KE * (4.0 * math.pi / V) * Q[idx] * mz
    if w.geometry == "ff":
        F[:, 2] -= Q[idx] * dpsi / float(w.box[2])
    return F
