"""FP64 Ewald sums for Gaussian electrode charges and point electrolyte charges.

Test infrastructure: this oracle is a plain, slow, CPU-only statement of the electrostatics of
Sec. II.A (Eqs. 1-3). It is imported only by tests/, by __graft_entry__.smoke() and by bench.py's
cpu_baseline leg; the GPU library never links, imports or calls it, and it shares no code with it.

Model (Eqs. 1-2): electrolyte charges Q_j are points; electrode charges q_i are Gaussians
rho_i(r) = q_i eta^3 pi^-3/2 exp(-eta^2 |r - r_i|^2).  The interaction energy of two such
distributions at distance r follows from convolving the densities:

    point-point        1/r
    Gaussian-point     erf(eta r)/r
    Gaussian-Gaussian  erf(eta r / sqrt 2)/r          (two width-eta Gaussians)
    Gaussian self      q^2 eta / sqrt(2 pi)            (half the r -> 0 limit of the line above)

The cell is orthorhombic and 3-D periodic with tin-foil boundary conditions (Sec. II.B).  Each
1/r is split Ewald-wise as erfc(alpha r)/r + erf(alpha r)/r: the smooth erf(alpha r)/r part of
every pair (Gaussians included, treated as points) goes to a direct reciprocal-space sum, the
rest is summed in real space over every periodic image within r_c (no minimum-image
shortcut, so cells shorter than 2 r_c are handled).  Real-space kernels:

    point-point        erfc(alpha r)/r
    Gaussian-point     (erfc(alpha r) - erfc(eta r))/r
    Gaussian-Gaussian  (erfc(alpha r) - erfc(eta r / sqrt 2))/r

and the reciprocal sum, for the potential at r from charges c_a at r_a,

    phi_k(r) = (4 pi / V) sum_{k != 0} exp(-k^2 / 4 alpha^2) / k^2  Re[S(k) exp(-i k.r)],
    S(k) = sum_a c_a exp(i k.r_a),

with the point self-energy correction -(alpha/sqrt pi) c_a^2.  Energies carry the Coulomb
constant KE so that potentials are in V, charges in e, lengths in A and energies in eV.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erfc

KE = 14.3996454784          # e^2 / (4 pi eps0) in eV A (CODATA 2018)
SQRT_PI = math.sqrt(math.pi)
SQRT2 = math.sqrt(2.0)
KMAX_EXPONENT = 27.6        # reciprocal terms below exp(-27.6) ~ 1e-12 of the leading one are dropped


def default_kmax(alpha: float) -> float:
    """Reciprocal cutoff |k| <= 2 alpha sqrt(27.6): exp(-k^2/4 alpha^2) <= 1e-12.
    Sec. II.B (Ewald summation, reciprocal part)."""
    return 2.0 * alpha * math.sqrt(KMAX_EXPONENT)


def screened(r, alpha, beta):
    """(erfc(alpha r) - erfc(beta r)) / r; beta=None means a point charge (erfc(beta r) = 0).
    Eqs. 1-2 under the Ewald split (Sec. II.B)."""
    f = erfc(alpha * r)
    if beta is not None:
        f = f - erfc(beta * r)
    return f / r


def screened_dr(r, alpha, beta):
    """d/dr of screened(r, alpha, beta).  Eqs. 1-2 under the Ewald split (Sec. II.B)."""
    g = -erfc(alpha * r) / (r * r) - (2.0 * alpha / SQRT_PI) * np.exp(-(alpha * r) ** 2) / r
    if beta is not None:
        g = g + erfc(beta * r) / (r * r) + (2.0 * beta / SQRT_PI) * np.exp(-(beta * r) ** 2) / r
    return g


def image_shifts(box, rcut) -> np.ndarray:
    """Lattice vectors n*L that can bring a minimum-image difference within rcut.

    A wrapped difference has |d| <= L/2 per axis, so image n matters only if |n| L - L/2 < r_c.
    Sec. II.B: the cell is periodic in x, y and z.
    """
    nmax = [int(math.floor(rcut / L + 0.5)) for L in box]
    rng = [np.arange(-n, n + 1) for n in nmax]
    n = np.stack(np.meshgrid(*rng, indexing="ij"), axis=-1).reshape(-1, 3)
    # put the zero shift first so the self-exclusion below is easy to read
    order = np.argsort((n * n).sum(1), kind="stable")
    return n[order] * np.asarray(box)[None, :]


def real_space(targets, sources, charges, box, rcut, alpha, beta, same=False, want_grad=False,
               chunk=256, target_index=None):
    """Real-space Ewald potential (and its gradient) at `targets` from all images of `sources`.

    beta selects the kernel (see module docstring).  same=True means the targets are members of the
    source set (target i is source target_index[i], default i) and each target's own zero-shift
    term is excluded.
    Returns phi [nt] (without KE) and, if want_grad, grad [nt, 3] = d phi / d r_target.
    Eqs. 1-2 under the Ewald split (Sec. II.B).
    """
    targets = np.asarray(targets, np.float64)
    sources = np.asarray(sources, np.float64)
    charges = np.asarray(charges, np.float64)
    box = np.asarray(box, np.float64)
    nt = targets.shape[0]
    phi = np.zeros(nt)
    grad = np.zeros((nt, 3)) if want_grad else None
    if nt == 0 or sources.shape[0] == 0:
        return (phi, grad) if want_grad else phi
    shifts = image_shifts(box, rcut)
    rc2 = rcut * rcut
    for a in range(0, nt, chunk):
        b = min(nt, a + chunk)
        d0 = targets[a:b, None, :] - sources[None, :, :]
        d0 -= box * np.round(d0 / box)
        for si, s in enumerate(shifts):
            d = d0 + s
            r2 = np.einsum("ijk,ijk->ij", d, d)
            m = r2 < rc2
            if same and not np.any(s):
                ii = np.arange(b - a)
                own = a + ii if target_index is None else np.asarray(target_index)[a:b]
                m[ii, own] = False
            ti, sj = np.nonzero(m)
            if ti.size == 0:
                continue
            r = np.sqrt(r2[ti, sj])
            f = screened(r, alpha, beta) * charges[sj]
            phi[a:b] += np.bincount(ti, weights=f, minlength=b - a)
            if want_grad:
                g = screened_dr(r, alpha, beta) * charges[sj] / r
                for c in range(3):
                    grad[a:b, c] += np.bincount(ti, weights=g * d[ti, sj, c], minlength=b - a)
    return (phi, grad) if want_grad else phi


def kvectors(box, kmax) -> np.ndarray:
    """Half-space set of nonzero reciprocal vectors k = 2 pi m / L with |k| <= kmax.
    Sec. II.B (Ewald summation, reciprocal part)."""
    box = np.asarray(box, np.float64)
    mmax = [int(math.floor(kmax * L / (2 * math.pi))) for L in box]
    rng = [np.arange(-n, n + 1) for n in mmax]
    m = np.stack(np.meshgrid(*rng, indexing="ij"), axis=-1).reshape(-1, 3)
    half = (m[:, 0] > 0) | ((m[:, 0] == 0) & (m[:, 1] > 0)) | ((m[:, 0] == 0) & (m[:, 1] == 0) & (m[:, 2] > 0))
    k = 2 * math.pi * m[half] / box[None, :]
    k2 = (k * k).sum(1)
    return k[k2 <= kmax * kmax]


def recip_weights(k, box, alpha):
    """Per half-space vector: 2 * (4 pi / V) exp(-k^2/4 alpha^2) / k^2 (factor 2 for -k).
    Sec. II.B (Ewald summation, reciprocal part)."""
    V = float(np.prod(box))
    k2 = (k * k).sum(1)
    return 2.0 * (4.0 * math.pi / V) * np.exp(-k2 / (4.0 * alpha * alpha)) / k2


def recip_space(targets, sources, charges, box, alpha, kmax=None, want_grad=False, kchunk=2048, ksub=None):
    """Reciprocal-space potential (and gradient) at `targets` from point charges at `sources`.

    phi(r) = sum_{k half} w_k [Re S(k) cos(k.r) + Im S(k) sin(k.r)],
    grad   = sum_{k half} w_k k [Im S(k) cos(k.r) - Re S(k) sin(k.r)],  w_k from recip_weights.
    ksub (timing samples only) maps the number of k-vectors to a selection of them.
    Sec. II.B (Ewald summation, reciprocal part).
    """
    targets = np.asarray(targets, np.float64)
    sources = np.asarray(sources, np.float64)
    charges = np.asarray(charges, np.float64)
    kmax = default_kmax(alpha) if kmax is None else kmax
    k_all = kvectors(box, kmax)
    if ksub is not None:
        k_all = k_all[ksub(k_all.shape[0])]
    w_all = recip_weights(k_all, box, alpha)
    phi = np.zeros(targets.shape[0])
    grad = np.zeros((targets.shape[0], 3)) if want_grad else None
    for a in range(0, k_all.shape[0], kchunk):
        k = k_all[a:a + kchunk]
        w = w_all[a:a + kchunk]
        ps = sources @ k.T
        s_re = np.cos(ps).T @ charges
        s_im = np.sin(ps).T @ charges
        pt = targets @ k.T
        ct, st = np.cos(pt), np.sin(pt)
        phi += ct @ (w * s_re) + st @ (w * s_im)
        if want_grad:
            grad += (ct * (w * s_im) - st * (w * s_re)) @ k
    return (phi, grad) if want_grad else phi


def recip_matrix(positions, box, alpha, kmax=None, kchunk=2048):
    """Reciprocal-space interaction matrix M_ab = sum_{k half} w_k cos(k.(r_a - r_b))
    = C diag(w) C^T + S diag(w) S^T with C = cos(r k^T), S = sin(r k^T).
    Sec. II.B; the reciprocal part of A in Eq. 3."""
    positions = np.asarray(positions, np.float64)
    kmax = default_kmax(alpha) if kmax is None else kmax
    k_all = kvectors(box, kmax)
    w_all = recip_weights(k_all, box, alpha)
    n = positions.shape[0]
    M = np.zeros((n, n))
    for a in range(0, k_all.shape[0], kchunk):
        k = k_all[a:a + kchunk]
        sw = np.sqrt(w_all[a:a + kchunk])
        p = positions @ k.T
        c = np.cos(p) * sw
        s = np.sin(p) * sw
        M += c @ c.T + s @ s.T
    return M


def recip_space_separable(targets, sources, charges, box, alpha, kmax=None, want_grad=False, schunk=4096,
                          tchunk=4096):
    """The sum of recip_space (same half-space k-vectors, weights and cutoff), evaluated through the
    factorisation exp(i k.r) = exp(i k_x x) exp(i k_y y) exp(i k_z z) of every plane wave with
    k = 2 pi (m_x/L_x, m_y/L_y, m_z/L_z): one table of exp(2 pi i m x / L) per axis and site, the
    structure factor S(m) = sum_a c_a X_a(m_x) Y_a(m_y) Z_a(m_z) as matrix products over the
    sources, and the potential sum_k w_k Re[S(k) exp(-i k.r)] likewise over the targets.  Used
    where recip_space's cos/sin per (site, k) is out of reach (10^5 sites x 10^5-10^6 k-vectors);
    equal to recip_space to rounding (pinned in the tests).  Sec. II.B (Ewald summation,
    reciprocal part)."""
    targets = np.asarray(targets, np.float64)
    sources = np.asarray(sources, np.float64)
    charges = np.asarray(charges, np.float64)
    box = np.asarray(box, np.float64)
    kmax = default_kmax(alpha) if kmax is None else kmax
    mmax = [int(math.floor(kmax * L / (2 * math.pi))) for L in box]
    mx = np.arange(0, mmax[0] + 1)
    my = np.arange(-mmax[1], mmax[1] + 1)
    mz = np.arange(-mmax[2], mmax[2] + 1)
    # the half-space set and weights of kvectors() / recip_weights() on the (m_x, m_y, m_z) block
    MX, MY, MZ = np.meshgrid(mx, my, mz, indexing="ij")
    half = (MX > 0) | ((MX == 0) & (MY > 0)) | ((MX == 0) & (MY == 0) & (MZ > 0))
    kx, ky, kz = (2 * math.pi * MX / box[0], 2 * math.pi * MY / box[1], 2 * math.pi * MZ / box[2])
    k2 = kx * kx + ky * ky + kz * kz
    keep = half & (k2 <= kmax * kmax)
    wk = np.zeros(MX.shape)
    V = float(np.prod(box))
    wk[keep] = 2.0 * (4.0 * math.pi / V) * np.exp(-k2[keep] / (4.0 * alpha * alpha)) / k2[keep]

    def tables(p):
        ph = 2 * math.pi * p / box[None, :]
        return (np.exp(1j * ph[:, 0:1] * mx[None, :]), np.exp(1j * ph[:, 1:2] * my[None, :]),
                np.exp(1j * ph[:, 2:3] * mz[None, :]))

    S = np.zeros(MX.shape, complex)
    for a in range(0, sources.shape[0], schunk):
        X, Y, Z = tables(sources[a:a + schunk])
        cX = charges[a:a + schunk, None] * X
        for i in range(mx.size):
            S[i] += (cX[:, i:i + 1] * Y).T @ Z
    G = wk * S
    nt = targets.shape[0]
    phi = np.zeros(nt)
    grad = np.zeros((nt, 3)) if want_grad else None
    Gs = [G] + ([G * MY, G * MZ] if want_grad else [])
    for a in range(0, nt, tchunk):
        X, Y, Z = tables(targets[a:a + tchunk])
        Xc, Yc, Zc = np.conj(X), np.conj(Y), np.conj(Z)
        acc = [np.zeros(Xc.shape[0], complex) for _ in range(4 if want_grad else 1)]
        for i in range(mx.size):
            part = [((Gi[i] @ Zc.T).T * Yc).sum(axis=1) * Xc[:, i] for Gi in Gs]
            acc[0] += part[0]
            if want_grad:
                acc[1] += mx[i] * part[0]
                acc[2] += part[1]
                acc[3] += part[2]
        phi[a:a + tchunk] = acc[0].real
        if want_grad:
            for d in range(3):
                grad[a:a + tchunk, d] = (2 * math.pi / box[d]) * acc[d + 1].imag
    return (phi, grad) if want_grad else phi
