"""The float32 erfc of the real-space pair kernels (CPU): the coefficient table in
csrc/cpm_step.cu (PairMath<float>::erfc_e) is the one erfc_fit.py fits, and evaluated in float32
in the kernel's operation order it stays within 4e-7 relative of scipy's erfc on the range the
kernels use (0 <= x <= 6.5), i.e. at float32 rounding level with no systematic term."""
import os
import re

import numpy as np
from scipy.special import erfc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _table():
    src = open(os.path.join(ROOT, "paper_2201_12963_gb300", "csrc", "cpm_step.cu")).read()
    body = src[src.index("static float erfc_e("):]
    body = body[:body.index("return t * poly * e;")]
    p = float(re.search(r"fmaf\(([0-9.eE+-]+)f, x, 1\.0f\)", body).group(1))
    lead = float(re.search(r"float poly = ([0-9.eE+-]+)f;", body).group(1))
    rest = [float(v) for v in re.findall(r"poly = fmaf\(poly, t, ([0-9.eE+-]+)f\);", body)]
    return p, [lead] + rest            # highest power first


def test_table_is_the_fit():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "erfc_fit", os.path.join(ROOT, "paper_2201_12963_gb300", "erfc_fit.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    c, err = mod.fit()
    p, table = _table()
    assert p == mod.P
    assert err < 4e-8
    assert np.allclose(table[::-1], c, rtol=0, atol=1e-8)


def test_float32_evaluation_is_within_rounding():
    p, table = _table()
    x = np.linspace(0.0, 6.5, 200001).astype(np.float32)
    e = np.exp(-(x.astype(np.float64) ** 2)).astype(np.float32)
    t = (np.float32(1.0) / (np.float32(p) * x + np.float32(1.0))).astype(np.float32)
    poly = np.full_like(x, np.float32(table[0]))
    for c in table[1:]:
        poly = (poly * t + np.float32(c)).astype(np.float32)
    val = (t * poly * e).astype(np.float64)
    ref = erfc(x.astype(np.float64))
    rel = np.abs(val - ref) / ref
    assert rel.max() < 4e-7
    # no systematic bias: the mean signed error is far below the float32 epsilon
    assert abs(np.mean((val - ref) / ref)) < 3e-8
