"""The pair-counting rule of the third-law cell kernel (CPM_PAIR_N3_ELYT), on the host.

The kernel stages, for the block of cells (cx, cy, cz .. cz + gz - 1), the stencil cells at a
lexicographically positive offset (x, then y, then z) from the block's origin cell that pass the
cell-to-group distance test, and inside the block's own cells takes a pair only with the source
after the target in the cell-sorted order.  Here that rule is enumerated in plain Python over small
periodic boxes, including boxes narrower than the stencil (every neighbour cell then appears at
several images), and compared with brute force: every unordered pair (i, j, periodic image)
within r_c must be produced exactly once, and the plain rule (the full stencil, every source)
must produce every ordered pair exactly once.
"""
import itertools
import math

import numpy as np
import pytest


def _grid(box, rc):
    nc = [max(1, int(math.floor(b / (0.5 * rc)))) for b in box]
    edge = [b / n for b, n in zip(box, nc)]
    sten = [int(math.ceil(rc / e - 1e-12)) for e in edge]
    return nc, edge, sten


def _enumerate(x, box, rc, gz, third_law):
    """(target, source, image) triples the kernel's rule visits; image = integer box shifts."""
    nc, edge, sten = _grid(box, rc)
    cell = [tuple(int(math.floor(x[i, d] / edge[d])) % nc[d] for d in range(3)) for i in range(len(x))]
    order = sorted(range(len(x)), key=lambda i: ((cell[i][0] * nc[1] + cell[i][1]) * nc[2] + cell[i][2], i))
    gi = {i: k for k, i in enumerate(order)}                     # sorted position
    members = {}
    for i in order:
        members.setdefault(cell[i], []).append(i)
    out = []
    for cx, cy in itertools.product(range(nc[0]), range(nc[1])):
        for cz in range(0, nc[2], gz):
            gzb = min(gz, nc[2] - cz)
            targets = [i for k in range(gzb) for i in members.get((cx, cy, cz + k), [])]
            for dx in range(-sten[0], sten[0] + 1):
                for dy in range(-sten[1], sten[1] + 1):
                    for dz in range(-sten[2], gzb + sten[2]):
                        gapz = -dz - 1 if dz < 0 else max(0, dz - gzb)
                        gx, gy, g3 = max(0, abs(dx) - 1) * edge[0], max(0, abs(dy) - 1) * edge[1], gapz * edge[2]
                        if gx * gx + gy * gy + g3 * g3 >= rc * rc:
                            continue
                        half_ok = dx > 0 or (dx == 0 and (dy > 0 or (dy == 0 and dz >= 0)))
                        if third_law and not half_ok:
                            continue
                        own = dx == 0 and dy == 0 and 0 <= dz < gzb
                        u = (cx + dx, cy + dy, cz + dz)
                        w = tuple(u[d] % nc[d] for d in range(3))
                        img = tuple(u[d] // nc[d] for d in range(3))    # whole boxes crossed
                        for j in members.get(w, []):
                            for i in targets:
                                # source position of this stencil cell's image
                                d = x[i] - (x[j] + np.array(img) * box)
                                r2 = float(d @ d)
                                if r2 >= rc * rc or r2 == 0.0:
                                    continue
                                if third_law and own and not gi[j] > gi[i]:
                                    continue
                                out.append((i, j, img))
    return out


def _brute(x, box, rc):
    """Every ordered (i, j, image n) with 0 < |x_i - x_j - n box| < rc."""
    nmax = [int(math.ceil(rc / b)) + 1 for b in box]
    out = set()
    for i in range(len(x)):
        for j in range(len(x)):
            for n in itertools.product(*[range(-m, m + 1) for m in nmax]):
                d = x[i] - (x[j] + np.array(n) * box)
                r2 = float(d @ d)
                if 0.0 < r2 < rc * rc:
                    out.add((i, j, n))
    return out


@pytest.mark.parametrize("box, n, gz", [((17.0, 17.4, 30.0), 40, 1), ((17.0, 17.4, 30.0), 40, 2),
                                         ((26.0, 25.0, 37.0), 60, 3), ((40.0, 38.0, 50.0), 80, 2)])
def test_half_stencil_rule_counts_every_pair_once(box, n, gz):
    rng = np.random.default_rng(7 + n + gz)
    box = np.asarray(box)
    x = rng.uniform(0.0, 1.0, size=(n, 3)) * box
    rc = 12.0
    ordered = _brute(x, box, rc)
    plain = _enumerate(x, box, rc, gz, third_law=False)
    assert len(plain) == len(set(plain)) == len(ordered) and set(plain) == ordered
    n3 = _enumerate(x, box, rc, gz, third_law=True)
    unordered = {}
    for i, j, img in n3:
        key = min((i, j, img), (j, i, tuple(-v for v in img)))
        unordered[key] = unordered.get(key, 0) + 1
    assert all(v == 1 for v in unordered.values())
    assert 2 * len(n3) == len(ordered)
    # every unordered pair of the brute force is among them
    for i, j, img in ordered:
        key = min((i, j, img), (j, i, tuple(-v for v in img)))
        assert key in unordered
