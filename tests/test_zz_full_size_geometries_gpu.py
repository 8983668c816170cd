"""Parity of the paper-scale doubled cell and slab at full size, in the benchmark's launch
configuration (GPU).

The paper compares the finite field with the doubled cell (Sec. II.B: 6,048 sites, two
constraints, S as two mirror blocks here) and the slab (3x z padding with the Yeh-Berkowitz term).
As for the finite-field cell (test_parity_full_size_gpu.py), the dense oracle solve is out of the
test budget, so b and the electrolyte forces are compared at 48 sampled sites, q is checked by the
KKT residual of the GPU charges through the oracle's elastance (both offsets of the doubled cell),
and the energy against the oracle's full Ewald energy at the GPU's q.  The smallest eigenvalue of
the oracle's A for this electrode is 7.248 V/e in all three geometries (dense eigendecomposition,
also restricted to the null space of C^T), so |dq| <= |residual| / 7 V/e.
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import synth
from oracle import cpm as ocpm

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _graph_step(s):
    """One cpm_step captured in a CUDA graph and replayed, as the benchmark times it."""
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        s.step(elec=False, energy=True)
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        s.step(elec=False, energy=True)
    graph.replay()
    torch.cuda.synchronize()


@pytest.mark.parametrize("geometry", ["dc", "slab"])
def test_paper_scale_doubled_cell_and_slab(geometry):
    import __graft_entry__
    __graft_entry__.build()
    import paper_2201_12963_gb300 as g
    from paper_2201_12963_gb300.driver import System
    w = synth.config_paper_cell(geometry=geometry)
    s = System(w, "mixed")
    _graph_step(s)
    assert g.cpm_status(s.ctx) == 0
    r = s.results()
    q, psibar = r["q"][0], r["psibar"][0]
    s.charges()
    b_gpu = s.results()["b"][0]
    R, Q, dpsi = w.elyt_xyz[0], w.elyt_q[0], float(w.dpsi[0])
    rng = np.random.default_rng(1)
    ie = rng.choice(w.n_elec, 48, replace=False)
    il = rng.choice(len(Q), 48, replace=False)
    # the four oracle evaluations are independent: numpy releases the GIL in its kernels
    with ThreadPoolExecutor(4) as ex:
        f_b = ex.submit(ocpm.b_at, w, R, Q, ie)
        f_aq = ex.submit(ocpm.elastance_apply, w, q)
        f_f = ex.submit(ocpm.electrolyte_forces_at, w, R, Q, q, dpsi, il)
        f_e = ex.submit(ocpm.energies, w, R, Q, q, dpsi)
        b_ref, Aq, F_ref, e = f_b.result(), f_aq.result(), f_f.result(), f_e.result()
    # b at sampled sites: the paper mesh's discretisation error (1 A, order 5)
    assert np.max(np.abs(b_gpu[ie] - b_ref)) <= 4e-5 * np.sqrt(np.mean(b_ref ** 2))
    # neutrality of the whole electrode and, in the doubled cell, of each sub-cell (Eq. 12)
    C = ocpm.constraints(w)
    assert np.max(np.abs(C.T @ q)) <= 1e-12 * max(1.0, np.abs(q).sum())
    # KKT: A q - b - dpsi v = C psibar, which bounds the charge error by |residual| / lambda_min(A)
    v = ocpm.geometry_vector(w)
    assert psibar.shape == (C.shape[1],)
    resid = Aq - b_gpu - dpsi * v - C @ psibar
    assert np.max(np.abs(resid)) / 7.0 <= 1e-5
    F = r["F_elyt"][0][il]
    assert np.sqrt(((F - F_ref) ** 2).sum() / (F_ref ** 2).sum()) <= 5e-5
    assert abs(r["energy"][0, 0] - e["U"]) <= 3e-5 * abs(e["U"])
    assert abs(r["energy"][0, 1] - e["H"]) <= 3e-5 * abs(e["H"])
