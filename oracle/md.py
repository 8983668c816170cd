"""FP64 oracle for the molecular-dynamics loop around the CPM step (test infrastructure only).

Only tests/ import this module; the GPU library does not, and the two share no code.

Appendix A of the paper integrates the electrolyte with velocity-Verlet at a 2 fs step under a
Nose-Hoover thermostat (400 K, 100 fs damping) acting on the electrolyte only, with one thermostat
per sub-cell in the doubled cell (Sec. II.B.2); Appendix B re-solves the electrode charges every
5 steps and keeps them in between.  The electrode sites are frozen.  Where the paper is silent this
oracle takes these readings:

* Thermostat discretisation.  One Nose-Hoover thermostat per group (no chain), propagated by the
  symmetric Trotter splitting of Martyna, Tuckerman, Tobias and Klein (Mol. Phys. 87, 1117, 1996):
  a thermostat half step, a velocity half kick, a full drift, the force evaluation, a velocity half
  kick and a thermostat half step.  The thermostat half step is itself split into a quarter-step
  update of the thermostat velocity v_xi, the velocity scaling exp(-v_xi dt / 2), the thermostat
  position update xi += v_xi dt / 2 and a second quarter-step update of v_xi, where
  dv_xi/dt = (2 K_g - g_g k_B T) / Q_g, Q_g = g_g k_B T tau^2, g_g = 3 N_g (the frozen electrode
  breaks momentum conservation, so no degree of freedom is removed) and tau is the damping time.
  The conserved quantity is KE + H + U_LJ + sum_g (Q_g v_xi,g^2 / 2 + g_g k_B T xi_g), with H the
  constant-potential energy of the CPM step (oracle.cpm.energies).
* Non-Coulomb forces.  The paper's force fields are not available.  A synthetic Lennard-Jones
  interaction with Lorentz-Berthelot mixing (sigma_ab = (sigma_a + sigma_b) / 2,
  eps_ab = sqrt(eps_a eps_b)) acts between electrolyte sites and between electrolyte and electrode
  sites, summed over every periodic image within the cutoff r_LJ and force-shifted there:
  U(r) = U_LJ(r) - U_LJ(r_LJ) + (r - r_LJ) F_LJ(r_LJ), so that energy and force vanish
  continuously at r_LJ.
* Charge schedule.  Step n (n counts force evaluations, the initial one is n = 0) re-solves the
  charges at the new positions when n is a multiple of k (Eqs. 8-15); otherwise the previous
  charges are kept and the forces are those of H at fixed charges.
* x and y are wrapped into [0, L) after every drift (a relabelling of periodic images).

Units: A, fs, amu, eV, e, K.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import cpm
from .ewald import image_shifts

KB = 8.617333262e-5                 # Boltzmann constant, eV / K
MVV2E = 103.64269652680505          # 1 amu A^2 / fs^2 in eV (amu 1.66053906660e-27 kg, e 1.602176634e-19 C)


# ----------------------------------------------------------------------------------------------
# synthetic Lennard-Jones
# ----------------------------------------------------------------------------------------------
def lj_pair(r, sigma, eps, cut):
    """Force-shifted LJ energy and force magnitude (eV, eV/A; positive = repulsive) at distance r.
    Appendix A (non-Coulomb pair term; synthetic Lennard-Jones stand-in)."""
    def u(x):
        s6 = (sigma / x) ** 6
        return 4.0 * eps * (s6 * s6 - s6)

    def f(x):
        s6 = (sigma / x) ** 6
        return 24.0 * eps * (2.0 * s6 * s6 - s6) / x

    fc = f(cut)
    return u(r) - u(cut) + (r - cut) * fc, f(r) - fc


def lj_energy_forces(R, types, E, elec_type, sigma, eps, cut, box):
    """U_LJ (eV) and the forces on the electrolyte sites (eV/A) by a direct sum over all pairs and
    all periodic images within `cut` (electrolyte-electrolyte pairs once, electrolyte-electrode
    pairs once; electrode sites carry type `elec_type` and feel no force, being frozen).
    Appendix A (non-Coulomb pair term; synthetic Lennard-Jones stand-in)."""
    R = np.asarray(R, np.float64)
    E = np.asarray(E, np.float64)
    box = np.asarray(box, np.float64)
    types = np.asarray(types, int)
    sigma = np.asarray(sigma, np.float64)
    eps = np.asarray(eps, np.float64)
    n = R.shape[0]
    F = np.zeros((n, 3))
    U = 0.0
    shifts = image_shifts(box, cut)
    sources = [(R, types, True), (E, np.full(E.shape[0], elec_type), False)]
    for i in range(n):
        for S, st, same in sources:
            if S.shape[0] == 0:
                continue
            sig = 0.5 * (sigma[types[i]] + sigma[st])
            ep = np.sqrt(eps[types[i]] * eps[st])
            d0 = R[i] - S
            d0 -= box * np.round(d0 / box)
            for s in shifts:
                d = d0 + s
                r = np.sqrt((d * d).sum(1))
                m = (r < cut) & (ep > 0)
                if same and not np.any(s):
                    m[i] = False
                if not np.any(m):
                    continue
                u, fmag = lj_pair(r[m], sig[m], ep[m], cut)
                U += (0.5 if same else 1.0) * u.sum()
                F[i] += ((fmag / r[m])[:, None] * d[m]).sum(0)
    return U, F


# ----------------------------------------------------------------------------------------------
# the integrator
# ----------------------------------------------------------------------------------------------
@dataclasses.dataclass
class MDParams:
    """Integrator settings: step, charge schedule, masses, Lennard-Jones, thermostat (Appendices A-B)."""
    dt: float = 2.0                  # fs
    charge_every: int = 5            # k
    mass: tuple = (139.2, 144.96)    # amu per type
    sigma: tuple = (3.0, 3.0)        # A per type
    eps: tuple = (0.02, 0.02)        # eV per type
    elec_type: int = 2
    lj_cut: float = 10.0             # A; 0 = no LJ
    temperature: float = 400.0       # K
    t_damp: float = 100.0            # fs; <= 0: no thermostat (NVE)


@dataclasses.dataclass
class MDState:
    """Positions, velocities, charges, forces, thermostat variables and step index (Appendix A)."""
    R: np.ndarray                    # [N, 3] electrolyte positions
    V: np.ndarray                    # [N, 3] velocities, A / fs
    q: np.ndarray                    # [N_e] electrode charges
    xi: np.ndarray                   # [G] thermostat positions
    vxi: np.ndarray                  # [G] thermostat velocities, 1 / fs
    step: int = 0


class Integrator:
    """Velocity-Verlet with per-group Nose-Hoover thermostats around the oracle CPM step.

    `force_fn(R, q, step)` may replace the CPM + LJ forces (returning (F, q, energies)); the
    thermostat and integration steps are the same either way."""

    def __init__(self, w, types, groups, p: MDParams, force_fn=None, kmax=None):
        self.w = w
        self.p = p
        self.types = np.asarray(types, int)
        self.groups = np.asarray(groups, int)
        self.n_groups = int(self.groups.max()) + 1 if self.groups.size else 1
        masses = np.asarray(p.mass, np.float64)
        self.m = masses[self.types]
        self.ndof = np.array([3.0 * np.count_nonzero(self.groups == g) for g in range(self.n_groups)])
        self.Qm = self.ndof * KB * p.temperature * p.t_damp ** 2 if p.t_damp > 0 else np.zeros(self.n_groups)
        self.force_fn = force_fn
        self.ref = None if force_fn is not None else cpm.Reference(w, kmax)
        self.kmax = kmax
        self.Q = np.asarray(w.elyt_q[0], np.float64)
        self.F = None
        self.energies = None

    # -- forces ------------------------------------------------------------------------------
    def _forces(self, R, q, step):
        if self.force_fn is not None:
            return self.force_fn(R, q, step)
        w, p = self.w, self.p
        dpsi = float(w.dpsi[0])
        if step % p.charge_every == 0:
            q, _, _ = self.ref.charges(R, self.Q, dpsi)
        F, _ = cpm.forces(w, R, self.Q, q, dpsi, self.kmax)
        en = cpm.energies(w, R, self.Q, q, dpsi, self.kmax)
        U_lj = 0.0
        if p.lj_cut > 0:
            U_lj, F_lj = lj_energy_forces(R, self.types, w.elec_xyz, p.elec_type, p.sigma, p.eps, p.lj_cut,
                                          cpm.ewald_box(w))
            F = F + F_lj
        en = dict(en, U_lj=U_lj)
        return F, q, en

    def kinetic(self, V):
        """Per-group kinetic energy (eV).  Appendix A (thermostat input)."""
        k = 0.5 * MVV2E * self.m * (V * V).sum(1)
        return np.array([k[self.groups == g].sum() for g in range(self.n_groups)])

    def _thermostat_half(self, st, K):
        """Half a time step of every group's thermostat; returns the velocity scale per group."""
        p = self.p
        s = np.ones(self.n_groups)
        if p.t_damp <= 0:
            return s
        dt = p.dt
        for g in range(self.n_groups):
            gkt = self.ndof[g] * KB * p.temperature
            st.vxi[g] += 0.25 * dt * (2.0 * K[g] - gkt) / self.Qm[g]
            s[g] = math.exp(-0.5 * dt * st.vxi[g])
            K[g] *= s[g] * s[g]
            st.xi[g] += 0.5 * dt * st.vxi[g]
            st.vxi[g] += 0.25 * dt * (2.0 * K[g] - gkt) / self.Qm[g]
        return s

    def _wrap_xy(self, R):
        box = np.asarray(self.w.box, np.float64)
        R[:, :2] -= box[:2] * np.floor(R[:, :2] / box[:2])

    def start(self, st: MDState):
        """Forces at the current positions (charges re-solved if the step index is a multiple of k).
        Appendix B (charge update schedule)."""
        self.F, st.q, self.energies = self._forces(st.R, st.q, st.step)

    def run(self, st: MDState, n_steps: int):
        """Advance n velocity-Verlet steps with the thermostat half steps around them (Appendices A-B)."""
        if self.F is None:
            self.start(st)
        dt, acc = self.p.dt, (1.0 / MVV2E) / self.m[:, None]
        for _ in range(n_steps):
            s = self._thermostat_half(st, self.kinetic(st.V))
            st.V *= s[self.groups][:, None]
            st.V += 0.5 * dt * acc * self.F
            st.R += dt * st.V
            self._wrap_xy(st.R)
            st.step += 1
            self.F, st.q, self.energies = self._forces(st.R, st.q, st.step)
            st.V += 0.5 * dt * acc * self.F
            s = self._thermostat_half(st, self.kinetic(st.V))
            st.V *= s[self.groups][:, None]
        return st

    def conserved(self, st: MDState) -> dict:
        """Energy terms at the current state: KE, H, U_LJ, thermostat energy and their total.
        Appendix A (Nose-Hoover extended energy)."""
        K = self.kinetic(st.V)
        e_nh = 0.0
        if self.p.t_damp > 0:
            kt = KB * self.p.temperature
            e_nh = float((0.5 * self.Qm * st.vxi ** 2 + self.ndof * kt * st.xi).sum())
        H = self.energies.get("H", 0.0)
        U_lj = self.energies.get("U_lj", 0.0)
        KE = float(K.sum())
        return {"KE": KE, "H": H, "U_lj": U_lj, "E_nh": e_nh, "E_total": KE + H + U_lj + e_nh,
                "T": 2.0 * KE / (self.ndof.sum() * KB)}


def initial_state(R, V, n_elec, n_groups, step=0) -> MDState:
    """State at step 0 from positions and velocities, thermostats at rest (Appendix A)."""
    return MDState(np.array(R, np.float64), np.array(V, np.float64), np.zeros(n_elec), np.zeros(n_groups),
                   np.zeros(n_groups), step)
