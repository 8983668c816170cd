"""Shared pytest setup: the `gpu` marker and cached oracle results for the small workloads."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU oracle cases")


_CACHE = {}


def cached(key, fn):
    """Memoise expensive oracle objects across test modules within one session."""
    if key not in _CACHE:
        _CACHE[key] = fn()
    return _CACHE[key]


@pytest.fixture(scope="session")
def plain_ff():
    import synth
    from oracle import cpm
    w = cached("w:plain_ff", synth.config_plain_ff)
    ref = cached("ref:plain_ff", lambda: cpm.Reference(w))
    out = cached("out:plain_ff", lambda: ref.step())
    return w, ref, out
