"""Checks of the offset potentials psibar shared by the GPU parity tests (imported, not collected).

At the constrained optimum A q = b + dpsi v + C psibar and C^T q = 0 (Eqs. 4-7, 12), so
psibar = -M W^T (b + dpsi v) with W = A^-1 C and M = (C^T W)^-1 (Eqs. 8-9, 13-15).  Two checks
keep the offsets apart from the mesh error of b:

* consistency: the GPU's psibar against -M W^T (b_gpu + dpsi v), the oracle's W and M applied to
  the GPU's own b.  The GPU forms psibar from b in float64 in both precision modes, so this holds
  to float64 rounding whatever the mesh;
* against the oracle: psibar - psibar_oracle = -M W^T (b_gpu - b_oracle), bounded by the row
  sums of |M W^T| times max |b_gpu - b_oracle|.
"""
import numpy as np
from scipy.linalg import cho_solve


def offsets_operator(oracle):
    """M W^T ([ncons, N_e]) of an oracle.cpm.Reference (its Cholesky factor of A)."""
    W = cho_solve(oracle.cho, oracle.C)
    M = np.linalg.inv(oracle.C.T @ W)
    return M @ W.T


def check_psibar(psibar, b_gpu, dpsi, oracle, psibar_ref, b_ref, rel=1e-9):
    """Assert both offset checks; returns (consistency error, oracle error, oracle bound)."""
    P = offsets_operator(oracle)
    cons = -P @ (b_gpu + dpsi * oracle.v)
    scale = max(1.0, float(np.max(np.abs(psibar))))
    e_cons = float(np.max(np.abs(psibar - cons)))
    assert e_cons <= rel * scale, (e_cons, psibar, cons)
    bound = float(np.max(np.abs(P).sum(axis=1))) * float(np.max(np.abs(b_gpu - b_ref))) + rel * scale
    e_ref = float(np.max(np.abs(psibar - psibar_ref)))
    assert e_ref <= bound, (e_ref, bound)
    return e_cons, e_ref, bound
