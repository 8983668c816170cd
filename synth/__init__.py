"""Seeded synthetic inputs for fully periodic constant-potential electrostatics.

This module builds geometry and random placements only: graphite electrode stacks, point-ion and
coarse-grained ionic-liquid electrolytes, doubled (z-mirrored) cells and replica batches. It holds
no electrostatics. Both the FP64 oracle and the GPU library consume what it returns.

The paper (Sec. III and Appendix) simulates a coarse-grained BMIm-PF6 ionic liquid (cation: three
sites, anion: one site, ion charges +-0.78 e) between two three-layer graphene electrodes with
0.335 nm interlayer spacing and A-B stacking. Its force-field parameters and trajectories are not
available, so the inputs here stand in for them with the same shapes, densities and charges:

* graphite layers are built from the 4-atom rectangular graphene cell 4.26 x 2.46 A
  (C-C bond 1.42 A), alternate layers shifted by 1.42 A in x, 3.35 A apart;
* the low-z electrode has its proximal plane at z = 10.00 A and the high-z electrode at
  z = L_z - 10.00 A, so that the two electrodes face each other across the periodic boundary
  through a 6.6 A empty gap (the finite-field arrangement of Sec. II.B.1);
* electrolyte sites are drawn uniformly (PCG64, fixed seed) in the accessible slab
  z in [13, L_z - 13] A by rejection sampling with a minimum site separation between molecules
  (minimum image in x, y);
* the coarse-grained cation is a rigid triangle of three +0.26 e sites with 2.5-3.0 A bonds,
  the anion a single -0.78 e site (synthetic, not the Roy-Maroncelli parameters).

Electrode side labels: +1 marks the high-z electrode (it receives d = +1/2), -1 the low-z one.
For the doubled cell the second sub-cell is the mirror image z -> 2 L_z - z of the first, so the
two +1/2 electrodes meet at the mirror plane and the two -1/2 electrodes across the periodic
boundary (Sec. II.B.2).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

GRAPHENE_CELL = (4.26, 2.46)          # rectangular 4-atom graphene cell (A)
GRAPHENE_BASIS = ((0.00, 0.00), (0.71, 1.23), (2.13, 1.23), (2.84, 0.00))
LAYER_SPACING = 3.35                   # A, Sec. III / Appendix A
PROXIMAL_OFFSET = 10.00                # proximal electrode plane distance from the cell edge (A)
ELECTROLYTE_MARGIN = 13.00             # accessible electrolyte slab starts here (A)
ION_CHARGE = 0.78                      # e, charge-scaled coarse-grained ionic liquid
PAPER_ETA = 1.979                      # 1/A, Gaussian width (Appendix B)
PAPER_TIMESTEP_FS = 2.0                # fs (Appendix A)


@dataclasses.dataclass
class Workload:
    """One electrode geometry plus one or more electrolyte replicas.

    box           physical cell (Lx, Ly, Lz) in A; for the doubled cell Lz is the doubled length
    elec_xyz      [N_e, 3] float64 electrode (Gaussian) site positions, A
    elec_side     [N_e] int32, +1 high-z (d = +1/2) / -1 low-z electrode
    elec_cell     [N_e] int32 sub-cell label (0/1) for the doubled cell, else None
    elec_layer    [N_e] int32, 0 = proximal layer
    elyt_xyz      list (one per replica) of [N_l, 3] float64 point-charge positions, A
    elyt_q        list of [N_l] float64 charges, e
    dpsi          [R] float64 potential differences, V
    geometry      'ff' (finite field), 'dc' (doubled cell) or 'slab'
    """

    name: str
    box: np.ndarray
    elec_xyz: np.ndarray
    elec_side: np.ndarray
    elec_cell: np.ndarray | None
    elec_layer: np.ndarray
    elyt_xyz: list
    elyt_q: list
    dpsi: np.ndarray
    geometry: str = "ff"
    eta: float = PAPER_ETA
    alpha: float = 0.25
    rcut: float = 12.0
    grid: tuple = (0, 0, 0)
    order: int = 5
    slab_factor: float = 3.0
    min_sep: float = 3.0

    @property
    def n_elec(self) -> int:
        return int(self.elec_xyz.shape[0])

    @property
    def n_rep(self) -> int:
        return len(self.elyt_xyz)

    def replica(self, r: int) -> "Workload":
        """A single-replica view of replica r."""
        return dataclasses.replace(self, elyt_xyz=[self.elyt_xyz[r]], elyt_q=[self.elyt_q[r]],
                                   dpsi=np.array([self.dpsi[r]], dtype=np.float64))

    def packed_electrolyte(self):
        """(offsets [R+1] int32, xyzq [sum N_l, 4] float64) in replica-major order."""
        counts = [len(q) for q in self.elyt_q]
        offsets = np.zeros(len(counts) + 1, dtype=np.int32)
        offsets[1:] = np.cumsum(counts)
        xyzq = np.zeros((int(offsets[-1]), 4), dtype=np.float64)
        for r in range(len(counts)):
            xyzq[offsets[r]:offsets[r + 1], :3] = self.elyt_xyz[r]
            xyzq[offsets[r]:offsets[r + 1], 3] = self.elyt_q[r]
        return offsets, xyzq


def graphene_layer(nx: int, ny: int, z: float, shift_x: float = 0.0) -> np.ndarray:
    """Sites of one graphene sheet of nx x ny rectangular cells at height z."""
    ax, ay = GRAPHENE_CELL
    pts = []
    for i in range(nx):
        for j in range(ny):
            for bx, by in GRAPHENE_BASIS:
                x = (i * ax + bx + shift_x) % (nx * ax)
                pts.append((x, j * ay + by, z))
    return np.asarray(pts, dtype=np.float64)


def rect_layer(nx: int, ny: int, lx: float, ly: float, z: float, shift: float = 0.0) -> np.ndarray:
    """A rectangular nx x ny lattice filling lx x ly, optionally shifted by shift*(dx, dy)/2."""
    dx, dy = lx / nx, ly / ny
    gx, gy = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    x = ((gx.ravel() + 0.5 * shift) * dx) % lx
    y = ((gy.ravel() + 0.5 * shift) * dy) % ly
    return np.stack([x, y, np.full(x.shape, z)], axis=1)


def electrode_pair(nx: int, ny: int, lz: float, n_layers: int = 3, lattice: str = "graphite",
                   lxy=None):
    """Two n_layers electrodes in a cell of height lz (proximal planes at 10 A and lz - 10 A).

    Returns (xyz [N_e,3], side [N_e], layer [N_e], (Lx, Ly)).
    """
    if lattice == "graphite":
        lx, ly = nx * GRAPHENE_CELL[0], ny * GRAPHENE_CELL[1]
    else:
        lx, ly = lxy
    xyz, side, layer = [], [], []
    for s, sign in ((-1, -1.0), (+1, +1.0)):
        for k in range(n_layers):
            if s < 0:
                z = PROXIMAL_OFFSET - LAYER_SPACING * k
            else:
                z = lz - PROXIMAL_OFFSET + LAYER_SPACING * k
            if lattice == "graphite":
                pts = graphene_layer(nx, ny, z, shift_x=1.42 * (k % 2))
            else:
                pts = rect_layer(nx, ny, lx, ly, z, shift=float(k % 2))
            xyz.append(pts)
            side.append(np.full(len(pts), s, dtype=np.int32))
            layer.append(np.full(len(pts), k, dtype=np.int32))
    return np.concatenate(xyz), np.concatenate(side), np.concatenate(layer), (lx, ly)


class _SpatialHash:
    """Uniform-cell hash for minimum-separation rejection sampling (periodic in x, y only)."""

    def __init__(self, lx, ly, dmin):
        self.lx, self.ly, self.d = lx, ly, dmin
        self.nx = max(1, int(lx // dmin))
        self.ny = max(1, int(ly // dmin))
        self.cx, self.cy = lx / self.nx, ly / self.ny
        self.cells: dict = {}

    def _key(self, p):
        return (int(p[0] // self.cx) % self.nx, int(p[1] // self.cy) % self.ny, int(math.floor(p[2] / self.d)))

    def ok(self, p) -> bool:
        kx, ky, kz = self._key(p)
        d2 = self.d * self.d
        seen = set()
        for ix in (-1, 0, 1):
            for iy in (-1, 0, 1):
                cx = (kx + ix) % self.nx
                cy = (ky + iy) % self.ny
                for iz in (-1, 0, 1):
                    key = (cx, cy, kz + iz)
                    if key in seen:
                        continue
                    seen.add(key)
                    for q in self.cells.get(key, ()):
                        dx = p[0] - q[0]
                        dx -= self.lx * round(dx / self.lx)
                        dy = p[1] - q[1]
                        dy -= self.ly * round(dy / self.ly)
                        dz = p[2] - q[2]
                        if dx * dx + dy * dy + dz * dz < d2:
                            return False
        return True

    def add(self, p):
        self.cells.setdefault(self._key(p), []).append(tuple(p))


def _random_rotation(rng) -> np.ndarray:
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([[a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
                     [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
                     [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d]])


def place_electrolyte(rng, lx, ly, zlo, zhi, n_pairs, model="point", dmin=3.0, max_tries=200000):
    """Random non-overlapping electrolyte: n_pairs cations and n_pairs anions.

    model 'point': +-0.78 e single sites.  model 'cg': 3-site cation (+0.26 e each), 1-site anion.
    Returns (xyz [N_l,3], q [N_l]).  Molecules alternate cation/anion so partial fills stay neutral.
    """
    h = _SpatialHash(lx, ly, dmin)
    xyz, q = [], []
    for m in range(2 * n_pairs):
        cation = (m % 2 == 0)
        for _ in range(max_tries):
            c = np.array([rng.uniform(0, lx), rng.uniform(0, ly), rng.uniform(zlo, zhi)])
            if model == "cg" and cation:
                b1, b2 = rng.uniform(2.5, 3.0, size=2)
                ang = rng.uniform(math.radians(60.0), math.radians(120.0))
                local = np.array([[0.0, 0.0, 0.0], [b1, 0.0, 0.0],
                                  [b2 * math.cos(ang), b2 * math.sin(ang), 0.0]])
                local -= local.mean(axis=0)
                sites = local @ _random_rotation(rng).T + c
                charges = [ION_CHARGE / 3.0] * 3
            else:
                sites = c[None, :]
                charges = [ION_CHARGE if cation else -ION_CHARGE]
            if np.any(sites[:, 2] < zlo) or np.any(sites[:, 2] > zhi):
                continue
            sites[:, 0] %= lx
            sites[:, 1] %= ly
            if all(h.ok(s) for s in sites):
                for s in sites:
                    h.add(s)
                xyz.extend(sites.tolist())
                q.extend(charges)
                break
        else:
            raise RuntimeError("electrolyte placement failed: density too high for min separation")
    return np.asarray(xyz, dtype=np.float64), np.asarray(q, dtype=np.float64)


def _molecule_sites(rng, n, lx, ly, zlo, zhi, cation, model):
    """n random molecules (all cations or all anions): sites [n, k, 3] and charges [k]."""
    c = np.stack([rng.uniform(0, lx, n), rng.uniform(0, ly, n), rng.uniform(zlo, zhi, n)], axis=1)
    if model == "cg" and cation:
        b1 = rng.uniform(2.5, 3.0, n)
        b2 = rng.uniform(2.5, 3.0, n)
        ang = rng.uniform(math.radians(60.0), math.radians(120.0), n)
        local = np.zeros((n, 3, 3))
        local[:, 1, 0] = b1
        local[:, 2, 0] = b2 * np.cos(ang)
        local[:, 2, 1] = b2 * np.sin(ang)
        local -= local.mean(axis=1, keepdims=True)
        qn = rng.normal(size=(n, 4))
        qn /= np.linalg.norm(qn, axis=1, keepdims=True)
        a, b, cc, d = qn.T
        rot = np.stack([np.stack([a * a + b * b - cc * cc - d * d, 2 * (b * cc - a * d), 2 * (b * d + a * cc)], -1),
                        np.stack([2 * (b * cc + a * d), a * a - b * b + cc * cc - d * d, 2 * (cc * d - a * b)], -1),
                        np.stack([2 * (b * d - a * cc), 2 * (cc * d + a * b), a * a - b * b - cc * cc + d * d], -1)],
                       axis=1)
        sites = np.einsum("nkj,nij->nki", local, rot) + c[:, None, :]
        return sites, np.full(3, ION_CHARGE / 3.0)
    return c[:, None, :], np.array([ION_CHARGE if cation else -ION_CHARGE])


def place_electrolyte_batched(rng, lx, ly, zlo, zhi, n_pairs, model="point", dmin=3.0, batch=16384,
                              max_batches=10000):
    """Random non-overlapping electrolyte like place_electrolyte, drawn in vectorised batches for
    large systems: each batch of candidate molecules (cations and anions alternately in draw
    order) is checked against the placed sites with a k-d tree periodic in x, y, and conflicts
    inside the batch are resolved by dropping the later-drawn molecule of every conflicting pair.  Returns (xyz [N_l,3], q [N_l]),
    cations first, then anions."""
    from scipy.spatial import cKDTree
    zbox = zhi + dmin + 1.0                       # no wrap in z: the slab sits inside [0, zbox)
    placed = np.zeros((0, 3))
    kept = {True: [], False: []}
    need = {True: n_pairs, False: n_pairs}
    charges = {}
    for _ in range(max_batches):
        if need[True] == 0 and need[False] == 0:
            break
        parts = []
        for cation in (True, False):
            if need[cation] == 0:
                continue
            sites, ch = _molecule_sites(rng, batch, lx, ly, zlo, zhi, cation, model)
            charges[cation] = ch
            inside = np.all((sites[:, :, 2] >= zlo) & (sites[:, :, 2] <= zhi), axis=1)
            ids = 2 * np.arange(batch) + (0 if cation else 1)      # draw order
            sites = sites[inside]
            sites[:, :, 0] %= lx
            sites[:, :, 1] %= ly
            parts.append((cation, sites, ids[inside]))
        flat = np.concatenate([p[1].reshape(-1, 3) for p in parts])
        owner = np.concatenate([np.repeat(p[2], p[1].shape[1]) for p in parts])
        ok = np.zeros(2 * batch, dtype=bool)
        for p in parts:
            ok[p[2]] = True
        if len(placed):
            d, _ = cKDTree(placed, boxsize=(lx, ly, zbox)).query(flat, distance_upper_bound=dmin)
            ok[owner[d < dmin]] = False
        live = ok[owner]
        lsites, lowner = flat[live], owner[live]
        acc = ok.copy()
        if len(lsites):
            pairs = cKDTree(lsites, boxsize=(lx, ly, zbox)).query_pairs(dmin, output_type="ndarray")
            if len(pairs):
                # of every conflicting pair the later-drawn molecule is dropped
                oa, ob = lowner[pairs[:, 0]], lowner[pairs[:, 1]]
                diff = oa != ob
                acc[np.maximum(oa, ob)[diff]] = False
        new_sites = []
        for cation, sites, ids in parts:
            take = np.flatnonzero(acc[ids])[:need[cation]]
            need[cation] -= len(take)
            kept[cation].append(sites[take])
            new_sites.append(sites[take].reshape(-1, 3))
        placed = np.concatenate([placed] + new_sites)
    else:
        raise RuntimeError("electrolyte placement failed: density too high for min separation")
    xyz, q = [], []
    for cation in (True, False):
        s = np.concatenate(kept[cation])
        xyz.append(s.reshape(-1, 3))
        q.append(np.tile(charges[cation], len(s)))
    return np.concatenate(xyz).astype(np.float64), np.concatenate(q).astype(np.float64)


def mirror_to_doubled(w: Workload, electrolyte: str = "mirror", seed: int | None = None,
                      model: str = "point", n_pairs: int | None = None, placer=None) -> Workload:
    """Doubled cell: sub-cell 0 is w, sub-cell 1 its z-mirror image z -> 2 L_z - z.

    electrolyte='mirror' reflects the electrolyte as well (mirror-symmetric cell); 'independent'
    draws a fresh electrolyte for sub-cell 1 with `seed`.  Electrode order: sub-cell 0 sites, then
    their mirror images in the same order (site i + N_e maps to site i).
    """
    lx, ly, lz = w.box
    ez = w.elec_xyz.copy()
    mz = ez.copy()
    mz[:, 2] = 2 * lz - ez[:, 2]
    xyz = np.concatenate([ez, mz])
    side = np.concatenate([w.elec_side, w.elec_side])
    cell = np.concatenate([np.zeros(w.n_elec, np.int32), np.ones(w.n_elec, np.int32)])
    layer = np.concatenate([w.elec_layer, w.elec_layer])
    ex, eq = [], []
    for r in range(w.n_rep):
        a = w.elyt_xyz[r]
        if electrolyte == "mirror":
            b = a.copy()
            b[:, 2] = 2 * lz - a[:, 2]
            bq = w.elyt_q[r].copy()
        else:
            rng = np.random.Generator(np.random.PCG64(seed + r))
            npairs = n_pairs if n_pairs is not None else len(w.elyt_q[r]) // (4 if model == "cg" else 2)
            b, bq = (placer or place_electrolyte)(rng, lx, ly, lz + ELECTROLYTE_MARGIN,
                                                  2 * lz - ELECTROLYTE_MARGIN, npairs, model=model,
                                                  dmin=w.min_sep)
        ex.append(np.concatenate([a, b]))
        eq.append(np.concatenate([w.elyt_q[r], bq]))
    return dataclasses.replace(w, name=w.name + "-dc", box=np.array([lx, ly, 2 * lz]), elec_xyz=xyz,
                               elec_side=side, elec_cell=cell, elec_layer=layer, elyt_xyz=ex,
                               elyt_q=eq, geometry="dc")


def _nice(n: int) -> int:
    """Smallest even m >= n whose only prime factors are 2, 3, 5 and 7 (FFT-friendly)."""
    m = max(2, n + (n % 2))
    while True:
        k = m
        for p in (2, 3, 5, 7):
            while k % p == 0:
                k //= p
        if k == 1:
            return m
        m += 2


def _grid_for(box, spacing=1.0):
    """SPME mesh with spacing at most `spacing` per axis, rounded up to FFT-friendly sizes."""
    return tuple(_nice(int(math.ceil(L / spacing - 1e-9))) for L in box)


def config_plain_ff(seed: int = 1000, dpsi: float = 2.0) -> Workload:
    """Plain finite-field cell: 17.04 x 17.22 x 60 A, 672 electrode sites, 100 + 100 point ions.

    Layers at z = 3.30, 6.65, 10.00 and 50.00, 53.35, 56.70 A; ions uniform in z in [13, 47] A with
    >= 3 A separation; Gaussian width eta = 1.979 1/A; Ewald alpha 0.25 1/A, r_c 12 A.
    """
    lz = 60.0
    xyz, side, layer, (lx, ly) = electrode_pair(4, 7, lz)
    rng = np.random.Generator(np.random.PCG64(seed))
    ex, eq = place_electrolyte(rng, lx, ly, ELECTROLYTE_MARGIN, lz - ELECTROLYTE_MARGIN, 100, "point", 3.0)
    box = np.array([lx, ly, lz])
    return Workload("ff-672", box, xyz, side, None, layer, [ex], [eq], np.array([dpsi]),
                    "ff", grid=_grid_for(box), min_sep=3.0)


def config_paper_cell(seed: int = 2000, dpsi: float = 2.0, geometry: str = "ff") -> Workload:
    """Paper-scale cell: 3,024 electrode sites (9 x 14 graphene cells, 38.34 x 34.44 A, three layers
    per electrode), 500 coarse-grained ion pairs (2,000 sites) at the paper's bulk ion-pair density
    (2.687e-3 pairs/A^3, 1.267 g/cm^3, Appendix B), L_z = 168 A, SPME grid 1 A, order 5.
    geometry: 'ff', 'dc' (mirror stack, 6,048 sites, independent second electrolyte) or 'slab'.
    """
    lz = 168.0
    xyz, side, layer, (lx, ly) = electrode_pair(9, 14, lz)
    rng = np.random.Generator(np.random.PCG64(seed))
    ex, eq = place_electrolyte(rng, lx, ly, ELECTROLYTE_MARGIN, lz - ELECTROLYTE_MARGIN, 500, "cg", 2.5)
    box = np.array([lx, ly, lz])
    w = Workload("ff-3024", box, xyz, side, None, layer, [ex], [eq], np.array([dpsi]), "ff",
                 grid=_grid_for(box), min_sep=2.5)
    if geometry == "dc":
        w = mirror_to_doubled(w, "independent", seed=seed + 1, model="cg")
        w.grid = _grid_for(w.box)
        w.name = "dc-6048"
    elif geometry == "slab":
        w = dataclasses.replace(w, name="slab-3024", geometry="slab", slab_factor=3.0,
                                grid=_grid_for((lx, ly, 3.0 * lz)))
    return w


def config_batched(n_rep: int = 64, seed0: int = 3000, dmin: float = 1.5) -> Workload:
    """Replica batch sharing the 672-site plain cell electrode: dpsi_r = 4 r / (R - 1) V and
    400-600 point-ion pairs per replica (drawn uniformly, seed seed0 + r), min separation 1.5 A."""
    base = config_plain_ff()
    lx, ly, lz = base.box
    exs, eqs = [], []
    for r in range(n_rep):
        rng = np.random.Generator(np.random.PCG64(seed0 + r))
        npairs = int(rng.integers(400, 601))
        ex, eq = place_electrolyte(rng, lx, ly, ELECTROLYTE_MARGIN, lz - ELECTROLYTE_MARGIN, npairs,
                                   "point", dmin)
        exs.append(ex)
        eqs.append(eq)
    dpsi = np.array([4.0 * r / max(1, n_rep - 1) for r in range(n_rep)])
    return dataclasses.replace(base, name=f"batched-{n_rep}x672", elyt_xyz=exs, elyt_q=eqs, dpsi=dpsi,
                               min_sep=dmin)


def config_large_ff(seed: int = 4000, n_pairs: int = 5000, dpsi: float = 2.0) -> Workload:
    """Scaled finite-field cell: 10,080 electrode sites (15 x 28 graphene cells, 63.90 x 68.88 A),
    5,000 point-ion pairs at the 672-site cell's ion density, L_z = 154 A."""
    lz = 154.0
    xyz, side, layer, (lx, ly) = electrode_pair(15, 28, lz)
    rng = np.random.Generator(np.random.PCG64(seed))
    ex, eq = place_electrolyte(rng, lx, ly, ELECTROLYTE_MARGIN, lz - ELECTROLYTE_MARGIN, n_pairs, "point", 3.0)
    box = np.array([lx, ly, lz])
    return Workload("ff-10080", box, xyz, side, None, layer, [ex], [eq], np.array([dpsi]), "ff",
                    grid=_grid_for(box), min_sep=3.0)


def tiny_cell(seed: int = 7, n_pairs: int = 3, nx: int = 2, ny: int = 3, lz: float = 36.0,
              dpsi: float = 1.0, geometry: str = "ff") -> Workload:
    """A small cell (2 x 3 graphene cells per layer, 144 sites) for quick checks."""
    xyz, side, layer, (lx, ly) = electrode_pair(nx, ny, lz)
    rng = np.random.Generator(np.random.PCG64(seed))
    ex, eq = place_electrolyte(rng, lx, ly, ELECTROLYTE_MARGIN, lz - ELECTROLYTE_MARGIN, n_pairs, "point", 3.0)
    box = np.array([lx, ly, lz])
    w = Workload("tiny", box, xyz, side, None, layer, [ex], [eq], np.array([dpsi]), "ff",
                 grid=_grid_for(box), min_sep=3.0)
    if geometry == "dc":
        w = mirror_to_doubled(w, "mirror")
        w.grid = _grid_for(w.box)
    elif geometry == "slab":
        w = dataclasses.replace(w, geometry="slab", grid=_grid_for((lx, ly, 3.0 * lz)))
    return w


def config_large_dc(seed: int = 5000, n_pairs_per_cell: int = 12500, dpsi: float = 2.0,
                    electrolyte: str = "independent", dmin: float = 2.0) -> Workload:
    """Large doubled cell: a 125 x 123 x 100 A sub-cell with two three-layer electrodes of a
    60 x 56 rectangular lattice per layer (2.083 x 2.196 A, alternate layers offset by half a
    step), 20,160 sites, and its z-mirror image: 40,320 electrode sites in a 125 x 123 x 200 A
    doubled cell.  12,500 coarse-grained ion pairs per sub-cell (25,000 pairs, 100,000 sites),
    drawn independently in each sub-cell (seeds `seed`, `seed + 1`) or mirrored
    (electrolyte='mirror').  SPME mesh 128 x 128 x 200, order 5.

    50,000 sites per 74 A sub-cell gap cannot be placed by rejection sampling at a 2.5 A site
    separation (hard-sphere packing fraction ~0.36, near the random-sequential-addition limit),
    so the minimum site separation between molecules is 2.0 A (packing fraction ~0.18).  The
    sites are drawn with place_electrolyte_batched.
    """
    lz = 100.0
    xyz, side, layer, (lx, ly) = electrode_pair(60, 56, lz, lattice="rect", lxy=(125.0, 123.0))
    rng = np.random.Generator(np.random.PCG64(seed))
    ex, eq = place_electrolyte_batched(rng, lx, ly, ELECTROLYTE_MARGIN, lz - ELECTROLYTE_MARGIN,
                                       n_pairs_per_cell, "cg", dmin)
    box = np.array([lx, ly, lz])
    w = Workload("dc-sub-20160", box, xyz, side, None, layer, [ex], [eq], np.array([dpsi]), "ff",
                 grid=(128, 128, 100), min_sep=dmin)
    w = mirror_to_doubled(w, electrolyte, seed=seed + 1, model="cg", n_pairs=n_pairs_per_cell,
                          placer=place_electrolyte_batched)
    w.grid = (128, 128, 200)
    w.name = "dc-40320"
    return w


def proximal_only(w: Workload) -> Workload:
    """The same cell with only the electrode layer nearest the electrolyte (layer 0) charged: the
    further layers carry no charge, so they drop out of the electrostatics altogether (they would
    contribute Lennard-Jones interactions only), as in the paper's production runs (Appendix B)."""
    keep = np.asarray(w.elec_layer) == 0
    return dataclasses.replace(w, name=w.name + "-proximal", elec_xyz=w.elec_xyz[keep],
                               elec_side=w.elec_side[keep],
                               elec_cell=None if w.elec_cell is None else w.elec_cell[keep],
                               elec_layer=w.elec_layer[keep])


# ----------------------------------------------------------------------------------------------
# molecular-dynamics inputs (point ions; the rigid three-site cation needs constraints)
# ----------------------------------------------------------------------------------------------
KB_EV = 8.617333262e-5                 # Boltzmann constant, eV / K
AMU_A2_FS2_EV = 103.64269652680505     # 1 amu A^2 / fs^2 in eV
MD_MASS = (139.2, 144.96)              # amu: cation (BMIm+), anion (PF6-) formula masses
MD_SIGMA = (3.0, 3.0, 3.37)            # A: cation, anion, electrode carbon (synthetic LJ)
MD_EPS = (0.02, 0.02, 0.0024)          # eV
MD_TEMPERATURE = 400.0                 # K (Appendix A)
MD_DAMP_FS = 100.0                     # fs (Appendix A)


@dataclasses.dataclass
class MDInputs:
    """Per-site MD labels and initial velocities for replica 0 of a workload.

    types     [N_l] int32: 0 cation, 1 anion (by the sign of the charge); the electrode is type 2
    groups    [N_l] int32 thermostat group: the sub-cell (z >= L_z / 2) in the doubled cell, else 0
    vel       [N_l, 3] float64 Maxwell-Boltzmann velocities at `temperature` (A / fs)
    """
    types: np.ndarray
    groups: np.ndarray
    vel: np.ndarray
    mass: tuple = MD_MASS
    sigma: tuple = MD_SIGMA
    eps: tuple = MD_EPS
    elec_type: int = 2
    temperature: float = MD_TEMPERATURE
    t_damp: float = MD_DAMP_FS


def md_inputs(w: Workload, seed: int = 77, temperature: float = MD_TEMPERATURE, r: int = 0) -> MDInputs:
    q = np.asarray(w.elyt_q[r])
    if np.any(np.abs(np.abs(q) - ION_CHARGE) > 1e-12):
        raise ValueError("md_inputs: the MD loop takes single-site ions of charge +-0.78 e")
    types = np.where(q > 0, 0, 1).astype(np.int32)
    z = np.asarray(w.elyt_xyz[r])[:, 2]
    groups = ((z >= 0.5 * w.box[2]) if w.geometry == "dc" else np.zeros(len(q), bool)).astype(np.int32)
    m = np.asarray(MD_MASS)[types]
    rng = np.random.Generator(np.random.PCG64(seed))
    sd = np.sqrt(KB_EV * temperature / (m * AMU_A2_FS2_EV))
    vel = rng.normal(size=(len(q), 3)) * sd[:, None]
    return MDInputs(types, groups, vel, temperature=temperature)


def md_cell(seed: int = 6000, n_pairs: int = 1000, dpsi: float = 2.0, geometry: str = "ff",
            nx: int = 9, ny: int = 14, lz: float = 168.0, dmin: float = 3.0) -> Workload:
    """Point-ion cell for the MD loop: the paper-scale electrode (9 x 14 graphene cells, three
    layers per electrode, L_z = 168 A) with n_pairs +-0.78 e point-ion pairs (default 1,000 pairs:
    the 2,000 electrolyte sites of the coarse-grained paper cell, each a single Lennard-Jones site),
    >= dmin apart, SPME grid 1 A, order 5.  geometry 'ff' or 'dc' (mirror stack, independent
    second electrolyte)."""
    xyz, side, layer, (lx, ly) = electrode_pair(nx, ny, lz)
    rng = np.random.Generator(np.random.PCG64(seed))
    ex, eq = place_electrolyte(rng, lx, ly, ELECTROLYTE_MARGIN, lz - ELECTROLYTE_MARGIN, n_pairs, "point", dmin)
    box = np.array([lx, ly, lz])
    w = Workload(f"md-{len(xyz)}-{2 * n_pairs}", box, xyz, side, None, layer, [ex], [eq], np.array([dpsi]),
                 "ff", grid=_grid_for(box), min_sep=dmin)
    if geometry == "dc":
        w = mirror_to_doubled(w, "independent", seed=seed + 1)
        w.grid = _grid_for(w.box)
        w.name = f"md-dc-{len(w.elec_xyz)}-{len(w.elyt_q[0])}"
    return w
