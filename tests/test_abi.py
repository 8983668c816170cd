"""The C-ABI library loads and exports every entry point that include/cpm.h declares (CPU only:
no call here touches a GPU)."""
import ctypes
import os
import re
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "cpm.h")).read()
    return sorted(set(re.findall(r"^(?:int|void|const char\*)\s+(cpm_\w+)\s*\(", txt, flags=re.M)))


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2201_12963_gb300 as g
    return g


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("cpm_build_matrix", "cpm_step_charges", "cpm_forces", "cpm_energy"):
        assert required in names


def test_library_exports_every_declared_symbol(pkg):
    lib = ctypes.CDLL(pkg.build.lib_path())
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(pkg.EXPORTED) == set(_declared())


def test_strerror_covers_every_status(pkg):
    for s in range(0, -10, -1):
        assert pkg.cpm_strerror(s) != "unknown status"
    assert pkg.cpm_strerror(-99) == "unknown status"


def test_invalid_parameters_rejected_before_any_device_work(pkg):
    xyz = np.array([[0, 0, 1.0], [1, 0, 1.0], [0, 0, 9.0], [1, 0, 9.0]])
    side = np.array([-1, -1, 1, 1])
    bad = [dict(order=9), dict(order=2), dict(alpha=2.0), dict(grid=(8, 8, 9)), dict(max_replicas=0)]
    for kw in bad:
        args = dict(box=(10, 10, 10), eta=1.979, alpha=0.25, rcut=5.0, grid=(16, 16, 16), order=5)
        args.update(kw)
        p = pkg.make_params(**args)
        with pytest.raises(pkg.CPMError) as ei:
            pkg.cpm_build_matrix(p, xyz, side, stream=0)
        assert ei.value.status == -1
    p = pkg.make_params((10, 10, 10), 1.979, 0.25, 5.0, (16, 16, 16))
    with pytest.raises(pkg.CPMError) as ei:
        pkg.cpm_build_matrix(p, xyz, np.array([-1, 2, 1, 1]), stream=0)
    assert ei.value.status == -1
    bad_xyz = xyz.copy()
    bad_xyz[0, 0] = np.nan
    with pytest.raises(pkg.CPMError) as ei:
        pkg.cpm_build_matrix(p, bad_xyz, side, stream=0)
    assert ei.value.status == -4
    pdc = pkg.make_params((10, 10, 10), 1.979, 0.25, 5.0, (16, 16, 16), geometry="dc")
    with pytest.raises(pkg.CPMError) as ei:
        pkg.cpm_build_matrix(pdc, xyz, side, None, stream=0)   # doubled cell needs sub-cell labels
    assert ei.value.status == -1


def test_host_tensors_are_rejected(pkg):
    """The entry points take device memory only: host tensors raise before any call, so there is
    no path on which the step runs anywhere but in the library's kernels."""
    torch = pytest.importorskip("torch")
    off = torch.tensor([0, 2], dtype=torch.int32)
    xyzq = torch.zeros(8, dtype=torch.float64)
    dpsi = torch.zeros(1, dtype=torch.float64)
    q = torch.zeros(4, dtype=torch.float64)
    for fn in (pkg.cpm_step_charges, pkg.cpm_step, pkg.cpm_forces):
        with pytest.raises(TypeError, match="CUDA"):
            fn(None, 1, off, xyzq, dpsi, q)
    with pytest.raises(TypeError, match="CUDA"):
        pkg.cpm_energy(None, 1, off, xyzq, dpsi, q, torch.zeros(4, dtype=torch.float64))


def test_import_fails_without_the_library(tmp_path):
    """Importing the package with the shared library absent raises ImportError (no fallback)."""
    code = (
        "import importlib.util, sys\n"
        f"spec = importlib.util.spec_from_file_location('paper_2201_12963_gb300.build', "
        f"{os.path.join(ROOT, 'paper_2201_12963_gb300', 'build.py')!r})\n"
        "mod = importlib.util.module_from_spec(spec)\n"
        "spec.loader.exec_module(mod)\n"
        f"mod.LIBDIR = {str(tmp_path)!r}\n"
        "sys.modules['paper_2201_12963_gb300.build'] = mod\n"
        "try:\n"
        "    import paper_2201_12963_gb300\n"
        "except ImportError as e:\n"
        "    print('ImportError:', e)\n"
        "    sys.exit(0)\n"
        "sys.exit(3)\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "not built" in r.stdout


def test_system_fails_loudly_without_a_gpu(pkg):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import synth
    from paper_2201_12963_gb300.driver import System
    with pytest.raises((RuntimeError, pkg.CPMError)):
        System(synth.tiny_cell(seed=7, n_pairs=2), "fp64")


def test_coincident_electrode_sites_are_rejected(pkg):
    """Two Gaussian sites at one point (also through a periodic image) make A's Gaussian-Gaussian
    kernel 0/0: the build refuses them before any device work."""
    xyz = np.array([[0.5, 0.5, 1.0], [1.5, 0.5, 1.0], [0.5, 0.5, 9.0], [1.5, 0.5, 9.0]])
    side = np.array([-1, -1, 1, 1])
    p = pkg.make_params((10, 10, 10), 1.979, 0.25, 5.0, (16, 16, 16))
    pkg.cpm_matrix_key(p, xyz, side)                        # distinct sites: accepted
    for j, shift in ((0, (0.0, 0.0, 0.0)), (0, (10.0, 0.0, 0.0)), (1, (0.0, -10.0, 0.0)), (2, (0.0, 0.0, 3e-7))):
        dup = np.vstack([xyz, xyz[j] + np.array(shift)])
        with pytest.raises(pkg.CPMError) as ei:
            pkg.cpm_matrix_key(p, dup, np.r_[side, side[j]])
        assert ei.value.status == -1
        with pytest.raises(pkg.CPMError) as ei:
            pkg.cpm_build_matrix(p, dup, np.r_[side, side[j]], stream=0)
        assert ei.value.status == -1
    near = np.vstack([xyz, xyz[0] + np.array([2e-6, 0.0, 0.0])])  # beyond the 1e-6 A tolerance
    pkg.cpm_matrix_key(p, near, np.r_[side, -1])
    big = pkg.make_params((1e12, 10, 10), 1.979, 0.25, 5.0, (16, 16, 16))    # hash grid capped per axis
    pkg.cpm_matrix_key(big, xyz, side)
    with pytest.raises(pkg.CPMError):
        pkg.cpm_matrix_key(big, np.vstack([xyz, xyz[3] + np.array([1e12, 0.0, 0.0])]), np.r_[side, 1])


def test_every_generated_electrode_passes_validation(pkg):
    """The coincidence check accepts the electrodes of every workload the tests and the benchmark
    build (the large cells with a token electrolyte: only the electrode matters here)."""
    import synth
    from paper_2201_12963_gb300.driver import params_for
    ws = [synth.config_plain_ff(), synth.config_paper_cell(), synth.config_paper_cell(geometry="dc"),
          synth.config_paper_cell(geometry="slab"), synth.proximal_only(synth.config_paper_cell()),
          synth.config_large_ff(n_pairs=10), synth.config_large_dc(n_pairs_per_cell=10), synth.md_cell(),
          synth.md_cell(geometry="dc")]
    for w in ws:
        pkg.cpm_matrix_key(params_for(w), w.elec_xyz, w.elec_side, w.elec_cell)
    # the small test cells, with the meshes their tests use
    w = synth.tiny_cell(seed=4, n_pairs=4)
    pkg.cpm_matrix_key(params_for(w, grid=(20, 16, 72), order=8), w.elec_xyz, w.elec_side, w.elec_cell)
    w = synth.mirror_to_doubled(w, "independent", seed=40)
    pkg.cpm_matrix_key(params_for(w, grid=(18, 16, 144), order=8), w.elec_xyz, w.elec_side, w.elec_cell)
