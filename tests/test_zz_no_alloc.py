"""The allocation-free charge update, cpm_step_charges_static (GPU).

Some callers cannot call cudaMalloc while they run (allocator-free regions of a host program,
real-time loops with a no-allocation rule); cpm_step_charges_static serves them from a static
device array.  Its charges, b and offsets must match the allocating cpm_step_charges on the
same context and inputs, on two calls in a row (the array keeps the previous call's contents,
so the second call checks that everything that must start at zero is cleared), and calls after
the first leave the device's free memory unchanged.  A context whose scratch does not fit the
array is rejected with CPM_ERR_CAPACITY.

This file is named to run last, so a failure here leaves every other test already run.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# the charge tolerance of the parity tests (|dq| <= 1e-5 e), far above the rounding-order
# differences expected between two runs of the same kernels
Q_TOL = 1e-5


def _lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2201_12963_gb300 as g
    from paper_2201_12963_gb300.driver import System
    return g, System


@pytest.mark.parametrize("prec,geometry", [("fp64", "ff"), ("mixed", "ff"), ("mixed", "dc")])
def test_static_scratch_entry_matches_allocating_entry(prec, geometry):
    g, System = _lib()
    if geometry == "ff":
        w = synth.config_plain_ff()
    else:                                   # doubled cell stored as mirror blocks
        w = synth.mirror_to_doubled(synth.tiny_cell(seed=4, n_pairs=4), "independent", seed=40)
        w.grid = (18, 16, 144)
    s = System(w, prec)
    assert g.cpm_matrix_layout(s.ctx)[0] == (geometry == "dc")
    s.charges()
    torch.cuda.synchronize()
    q_ref, b_ref, p_ref = s.q.clone(), s.b.clone(), s.psibar.clone()
    # the contract itself: after a first call, further calls leave the device's free memory as it
    # was (any cudaMalloc, or a library routine that allocates, would take at least one page)
    qa, ba, pa = torch.empty_like(s.q), torch.empty_like(s.b), torch.empty_like(s.psibar)
    g.cpm_step_charges_static(s.ctx, s.offsets, s.xyzq, s.dpsi, qa, ba, pa)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        g.cpm_step_charges_static(s.ctx, s.offsets, s.xyzq, s.dpsi, qa, ba, pa)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    for _ in range(2):
        q = torch.full_like(s.q, float("nan"))
        b = torch.full_like(s.b, float("nan"))
        p = torch.full_like(s.psibar, float("nan"))
        g.cpm_step_charges_static(s.ctx, s.offsets, s.xyzq, s.dpsi, q, b, p)
        assert g.cpm_status(s.ctx) == 0
        assert torch.max(torch.abs(q - q_ref)).item() <= Q_TOL
        assert torch.max(torch.abs(b - b_ref)).item() <= 1e-6 * torch.sqrt(torch.mean(b_ref ** 2)).item()
        assert torch.max(torch.abs(p - p_ref)).item() <= 1e-6
        assert abs(q.sum().item()) <= 1e-12


def test_static_scratch_rejects_contexts_that_do_not_fit():
    g, System = _lib()
    w = synth.config_plain_ff()
    s = System(w, "fp64", grid=(128, 128, 256))          # ~16 M-point float64 meshes
    with pytest.raises(g.CPMError) as ei:
        g.cpm_step_charges_static(s.ctx, s.offsets, s.xyzq, s.dpsi, s.q)
    assert ei.value.status == -5
