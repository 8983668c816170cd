"""GB300 constant-potential-method (CPM) electrostatics: thin Python binding of the C ABI.

Every function here marshals arguments (torch device tensors -> raw pointers, numpy host arrays
-> host pointers) and calls the entry point of the same name in libcpm_gb300.so; all arithmetic
runs in the library's CUDA kernels.  Importing the package loads the library and raises if it is
missing: there is no CPU fallback.  The C declarations and their contracts are in include/cpm.h.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

CPM_FF, CPM_DOUBLED, CPM_SLAB = 0, 1, 2
CPM_FP64, CPM_MIXED = 0, 1
GEOMETRY = {"ff": CPM_FF, "dc": CPM_DOUBLED, "slab": CPM_SLAB}
PRECISION = {"fp64": CPM_FP64, "mixed": CPM_MIXED}
MATRIX_KSPACE = {"ewald": 0, "mesh": 1}                 # enum cpm_matrix_kspace
DC_BLOCKS = {"auto": 0, "mirror": 1, "full": 2}        # enum cpm_dc_blocks

EXPORTED = ("cpm_build_matrix", "cpm_matrix_key", "cpm_matrix_image", "cpm_build_matrix_from_image", "cpm_step_charges", "cpm_forces", "cpm_energy", "cpm_step", "cpm_capacitance",
            "cpm_copy_matrix", "cpm_info", "cpm_status", "cpm_profile_enable", "cpm_profile_read", "cpm_counters",
            "cpm_step_charges_static", "cpm_matrix_layout", "cpm_pair_list_layout", "cpm_set_sapply_variant", "cpm_set_fft_variant", "cpm_set_mesh_variant",
            "cpm_set_pair_group", "cpm_get_pair_group", "cpm_set_pair_variant", "cpm_get_pair_variant",
            "cpm_set_wait_test",
            "cpm_autotune", "cpm_density_z", "cpm_potential_z",
            "cpm_md_create", "cpm_md_run", "cpm_md_advance", "cpm_md_get_state", "cpm_md_set_state", "cpm_md_info",
            "cpm_md_destroy", "cpm_destroy",
            "cpm_strerror", "cpm_last_error")
PHASES = ("cell_list", "b_real", "b_spread", "b_fft", "b_gather", "s_apply", "project", "f_spread", "f_fft",
          "f_gather", "f_pair_elyt", "f_pair_elec", "energy")


class CpmParams(ctypes.Structure):
    """Mirror of cpm_params in include/cpm.h."""
    _fields_ = [("box", ctypes.c_double * 3), ("eta", ctypes.c_double), ("alpha", ctypes.c_double),
                ("rcut", ctypes.c_double), ("slab_factor", ctypes.c_double), ("kmax_build", ctypes.c_double),
                ("grid", ctypes.c_int32 * 3), ("spme_order", ctypes.c_int32), ("geometry", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("max_replicas", ctypes.c_int32), ("max_elyt", ctypes.c_int32),
                ("matrix_kspace", ctypes.c_int32), ("dc_blocks", ctypes.c_int32)]


MD_MAX_TYPES = 8
MD_NENERGY = 8           # per replica: U, H, U_LJ, KE, E_thermostat, E_total, T, Q_+
MD_ENERGY_KEYS = ("U", "H", "U_lj", "KE", "E_nh", "E_total", "T", "Q_plus")


class CpmMdParams(ctypes.Structure):
    """Mirror of cpm_md_params in include/cpm.h."""
    _fields_ = [("dt", ctypes.c_double), ("charge_every", ctypes.c_int32), ("n_types", ctypes.c_int32),
                ("mass", ctypes.c_double * MD_MAX_TYPES), ("lj_sigma", ctypes.c_double * MD_MAX_TYPES),
                ("lj_epsilon", ctypes.c_double * MD_MAX_TYPES), ("elec_type", ctypes.c_int32),
                ("n_groups", ctypes.c_int32), ("lj_cut", ctypes.c_double), ("temperature", ctypes.c_double),
                ("t_damp", ctypes.c_double)]


class CPMError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = f"{where}: {_lib.cpm_strerror(status).decode()} ({status})"
        detail = _lib.cpm_last_error().decode()
        if detail:
            msg += f": {detail}"
        super().__init__(msg)


def _load():
    path = _build.lib_path()
    if not os.path.exists(path):
        raise ImportError(f"CPM CUDA library not built ({path}); run __graft_entry__.build() "
                          "or python -m paper_2201_12963_gb300.build")
    lib = ctypes.CDLL(path)
    vp, i32, pd, pi32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p
    lib.cpm_build_matrix.argtypes = [ctypes.POINTER(CpmParams), i32, pd, pi32, pi32, vp, ctypes.POINTER(vp)]
    lib.cpm_matrix_key.argtypes = [ctypes.POINTER(CpmParams), i32, pd, pi32, pi32, ctypes.POINTER(ctypes.c_uint64)]
    lib.cpm_matrix_image.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_int64)]
    lib.cpm_build_matrix_from_image.argtypes = [ctypes.POINTER(CpmParams), i32, pd, pi32, pi32, vp, ctypes.c_int64,
                                                vp, ctypes.POINTER(vp)]
    lib.cpm_step_charges.argtypes = [vp, i32, pi32, pd, pd, pd, pd, pd, vp]
    lib.cpm_forces.argtypes = [vp, i32, pi32, pd, pd, pd, pd, pd, pd, vp]
    lib.cpm_energy.argtypes = [vp, i32, pi32, pd, pd, pd, pd, vp]
    lib.cpm_step.argtypes = [vp, i32, pi32, pd, pd, pd, pd, pd, pd, pd, vp]
    lib.cpm_capacitance.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    lib.cpm_copy_matrix.argtypes = [vp, i32, pd]
    lib.cpm_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_int64),
                             ctypes.POINTER(i32)]
    lib.cpm_status.argtypes = [vp, vp]
    lib.cpm_profile_enable.argtypes = [vp, i32]
    lib.cpm_profile_read.argtypes = [vp, pd, pd]
    lib.cpm_counters.argtypes = [vp, ctypes.POINTER(ctypes.c_int64)]
    lib.cpm_step_charges_static.argtypes = [vp, pi32, pd, pd, pd, pd, pd, vp]
    lib.cpm_matrix_layout.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_int64)]
    lib.cpm_pair_list_layout.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(i32)]
    lib.cpm_set_sapply_variant.argtypes = [vp, i32]
    lib.cpm_set_fft_variant.argtypes = [vp, i32]
    lib.cpm_set_mesh_variant.argtypes = [vp, i32]
    lib.cpm_set_pair_group.argtypes = [vp, i32]
    lib.cpm_set_wait_test.argtypes = [vp, i32]
    lib.cpm_get_pair_group.argtypes = [vp, ctypes.POINTER(i32)]
    lib.cpm_set_pair_variant.argtypes = [vp, i32]
    lib.cpm_get_pair_variant.argtypes = [vp, ctypes.POINTER(i32)]
    lib.cpm_density_z.argtypes = [vp, i32, pi32, pd, pd, i32, pd, vp]
    lib.cpm_potential_z.argtypes = [vp, i32, i32, pd, ctypes.c_double, pd, pd, vp]
    lib.cpm_autotune.argtypes = [vp, pi32, pd, pd, pd, vp, pi32]
    lib.cpm_md_create.argtypes = [vp, ctypes.POINTER(CpmMdParams), i32, pi32, pi32, pi32, vp, ctypes.POINTER(vp)]
    lib.cpm_md_run.argtypes = [vp, i32, pd, pd, pd, pd, pd, pd, pd, vp]
    lib.cpm_md_advance.argtypes = [vp, ctypes.c_int64]
    lib.cpm_md_get_state.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), pd, vp]
    lib.cpm_md_set_state.argtypes = [vp, ctypes.c_int64, pd, vp]
    lib.cpm_md_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    lib.cpm_md_destroy.argtypes = [vp]
    lib.cpm_md_destroy.restype = None
    lib.cpm_destroy.argtypes = [vp]
    lib.cpm_destroy.restype = None
    lib.cpm_strerror.argtypes = [ctypes.c_int]
    lib.cpm_strerror.restype = ctypes.c_char_p
    lib.cpm_last_error.argtypes = []
    lib.cpm_last_error.restype = ctypes.c_char_p
    for name in EXPORTED:
        if name not in ("cpm_destroy", "cpm_md_destroy", "cpm_strerror", "cpm_last_error"):
            getattr(lib, name).restype = ctypes.c_int
    return lib


_lib = _load()


def library():
    """The loaded ctypes.CDLL (for symbol checks)."""
    return _lib


def _check(status: int, where: str):
    if status != 0:
        raise CPMError(status, where)


def make_params(box, eta, alpha, rcut, grid, order=5, geometry="ff", precision="fp64", max_replicas=1,
                max_elyt=1, slab_factor=3.0, kmax_build=0.0, matrix_kspace="ewald", dc_blocks="auto") -> CpmParams:
    p = CpmParams()
    for d in range(3):
        p.box[d] = float(box[d])
        p.grid[d] = int(grid[d])
    p.eta, p.alpha, p.rcut = float(eta), float(alpha), float(rcut)
    p.slab_factor, p.kmax_build = float(slab_factor), float(kmax_build)
    p.spme_order = int(order)
    p.geometry = GEOMETRY[geometry] if isinstance(geometry, str) else int(geometry)
    p.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
    p.max_replicas, p.max_elyt = int(max_replicas), int(max_elyt)
    p.matrix_kspace = MATRIX_KSPACE[matrix_kspace] if isinstance(matrix_kspace, str) else int(matrix_kspace)
    p.dc_blocks = DC_BLOCKS[dc_blocks] if isinstance(dc_blocks, str) else int(dc_blocks)
    return p


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _dev(t, dtype, name, numel=None, optional=False):
    """Raw pointer of a contiguous CUDA tensor of the given torch dtype (or None if optional)."""
    if t is None:
        if optional:
            return None
        raise ValueError(f"{name} is required")
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA torch.Tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{name} has {t.numel()} elements, needs {numel}")
    return t.data_ptr()


class Context:
    """Owning handle of a cpm_ctx (destroyed with the object)."""

    def __init__(self, handle, params: CpmParams):
        self.handle = handle
        self.params = params
        n, c, m, nc = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int32()
        _check(_lib.cpm_info(handle, ctypes.byref(n), ctypes.byref(c), ctypes.byref(m), ctypes.byref(nc)), "cpm_info")
        self.n_elec, self.ncons, self.mesh_points, self.n_cells = n.value, c.value, m.value, nc.value

    def close(self):
        h = getattr(self, "handle", None)
        if h:
            _lib.cpm_destroy(h)
            self.handle = None

    def __del__(self):
        self.close()


def cpm_build_matrix(params: CpmParams, elec_xyz, elec_side, elec_cell=None, stream=None) -> Context:
    xyz = np.ascontiguousarray(elec_xyz, dtype=np.float64)
    side = np.ascontiguousarray(elec_side, dtype=np.int32)
    cell = None if elec_cell is None else np.ascontiguousarray(elec_cell, dtype=np.int32)
    n = xyz.shape[0]
    if xyz.shape != (n, 3) or side.shape != (n,) or (cell is not None and cell.shape != (n,)):
        raise ValueError("electrode arrays have inconsistent shapes")
    out = ctypes.c_void_p()
    st = _stream_ptr(stream)
    s = _lib.cpm_build_matrix(ctypes.byref(params), n, xyz.ctypes.data, side.ctypes.data,
                              None if cell is None else cell.ctypes.data, st, ctypes.byref(out))
    _check(s, "cpm_build_matrix")
    return Context(out.value, params)


def _electrode_arrays(elec_xyz, elec_side, elec_cell):
    xyz = np.ascontiguousarray(elec_xyz, dtype=np.float64)
    side = np.ascontiguousarray(elec_side, dtype=np.int32)
    cell = None if elec_cell is None else np.ascontiguousarray(elec_cell, dtype=np.int32)
    n = xyz.shape[0]
    if xyz.shape != (n, 3) or side.shape != (n,) or (cell is not None and cell.shape != (n,)):
        raise ValueError("electrode arrays have inconsistent shapes")
    return xyz, side, cell, n


def cpm_matrix_key(params: CpmParams, elec_xyz, elec_side, elec_cell=None) -> int:
    """64-bit key of the inputs that determine A (names cached matrix images)."""
    xyz, side, cell, n = _electrode_arrays(elec_xyz, elec_side, elec_cell)
    key = ctypes.c_uint64()
    _check(_lib.cpm_matrix_key(ctypes.byref(params), n, xyz.ctypes.data, side.ctypes.data,
                               None if cell is None else cell.ctypes.data, ctypes.byref(key)), "cpm_matrix_key")
    return int(key.value)


def cpm_matrix_image(ctx: Context) -> bytes:
    """The context's matrix image (S, A^-1 C, S v and the projection scalars, with its key)."""
    nb = ctypes.c_int64()
    _check(_lib.cpm_matrix_image(ctx.handle, None, ctypes.byref(nb)), "cpm_matrix_image")
    buf = np.empty(int(nb.value), dtype=np.uint8)
    _check(_lib.cpm_matrix_image(ctx.handle, buf.ctypes.data, ctypes.byref(nb)), "cpm_matrix_image")
    return buf


def cpm_build_matrix_from_image(params: CpmParams, elec_xyz, elec_side, elec_cell, image, stream=None) -> Context:
    xyz, side, cell, n = _electrode_arrays(elec_xyz, elec_side, elec_cell)
    img = np.ascontiguousarray(np.frombuffer(image, dtype=np.uint8) if isinstance(image, (bytes, bytearray))
                               else image, dtype=np.uint8)
    out = ctypes.c_void_p()
    s = _lib.cpm_build_matrix_from_image(ctypes.byref(params), n, xyz.ctypes.data, side.ctypes.data,
                                         None if cell is None else cell.ctypes.data, img.ctypes.data, img.size,
                                         _stream_ptr(stream), ctypes.byref(out))
    _check(s, "cpm_build_matrix_from_image")
    return Context(out.value, params)


def _common(ctx, n_rep, offsets, xyzq, dpsi):
    import torch
    p_off = _dev(offsets, torch.int32, "offsets", n_rep + 1)
    p_x = _dev(xyzq, torch.float64, "xyzq")
    p_d = _dev(dpsi, torch.float64, "dpsi", n_rep)
    return p_off, p_x, p_d


def cpm_step_charges(ctx: Context, n_rep, offsets, xyzq, dpsi, q, b=None, psibar=None, stream=None):
    import torch
    p_off, p_x, p_d = _common(ctx, n_rep, offsets, xyzq, dpsi)
    ne = ctx.n_elec
    s = _lib.cpm_step_charges(ctx.handle, n_rep, p_off, p_x, p_d, _dev(q, torch.float64, "q", n_rep * ne),
                              _dev(b, torch.float64, "b", n_rep * ne, True),
                              _dev(psibar, torch.float64, "psibar", n_rep * ctx.ncons, True), _stream_ptr(stream))
    _check(s, "cpm_step_charges")


def cpm_forces(ctx: Context, n_rep, offsets, xyzq, dpsi, q, f_elyt=None, f_elec=None, energy=None, stream=None):
    import torch
    p_off, p_x, p_d = _common(ctx, n_rep, offsets, xyzq, dpsi)
    ne = ctx.n_elec
    s = _lib.cpm_forces(ctx.handle, n_rep, p_off, p_x, p_d, _dev(q, torch.float64, "q", n_rep * ne),
                        _dev(f_elyt, torch.float64, "f_elyt", None, True),
                        _dev(f_elec, torch.float64, "f_elec", n_rep * ne * 3, True),
                        _dev(energy, torch.float64, "energy", 4 * n_rep, True), _stream_ptr(stream))
    _check(s, "cpm_forces")


def cpm_energy(ctx: Context, n_rep, offsets, xyzq, dpsi, q, energy, stream=None):
    import torch
    p_off, p_x, p_d = _common(ctx, n_rep, offsets, xyzq, dpsi)
    s = _lib.cpm_energy(ctx.handle, n_rep, p_off, p_x, p_d, _dev(q, torch.float64, "q", n_rep * ctx.n_elec),
                        _dev(energy, torch.float64, "energy", 4 * n_rep), _stream_ptr(stream))
    _check(s, "cpm_energy")


def cpm_step(ctx: Context, n_rep, offsets, xyzq, dpsi, q, psibar=None, f_elyt=None, f_elec=None, energy=None,
             stream=None):
    import torch
    p_off, p_x, p_d = _common(ctx, n_rep, offsets, xyzq, dpsi)
    ne = ctx.n_elec
    s = _lib.cpm_step(ctx.handle, n_rep, p_off, p_x, p_d, _dev(q, torch.float64, "q", n_rep * ne),
                      _dev(psibar, torch.float64, "psibar", n_rep * ctx.ncons, True),
                      _dev(f_elyt, torch.float64, "f_elyt", None, True),
                      _dev(f_elec, torch.float64, "f_elec", n_rep * ne * 3, True),
                      _dev(energy, torch.float64, "energy", 4 * n_rep, True), _stream_ptr(stream))
    _check(s, "cpm_step")


def cpm_step_charges_static(ctx: Context, offsets, xyzq, dpsi, q, b=None, psibar=None, stream=None):
    """Single-replica charge update that allocates nothing (scratch in the library's static
    device array); see cpm_step_charges_static in include/cpm.h."""
    import torch
    p_off, p_x, p_d = _common(ctx, 1, offsets, xyzq, dpsi)
    ne = ctx.n_elec
    s = _lib.cpm_step_charges_static(ctx.handle, p_off, p_x, p_d, _dev(q, torch.float64, "q", ne),
                                     _dev(b, torch.float64, "b", ne, True),
                                     _dev(psibar, torch.float64, "psibar", ctx.ncons, True), _stream_ptr(stream))
    _check(s, "cpm_step_charges_static")


def cpm_capacitance(ctx: Context) -> float:
    v = ctypes.c_double()
    _check(_lib.cpm_capacitance(ctx.handle, ctypes.byref(v)), "cpm_capacitance")
    return v.value


def cpm_copy_matrix(ctx: Context, which: int) -> np.ndarray:
    n = ctx.n_elec
    shape = {0: (n, n), 1: (n,), 2: (n, ctx.ncons)}[which]
    out = np.zeros(shape, dtype=np.float64)
    _check(_lib.cpm_copy_matrix(ctx.handle, which, out.ctypes.data), "cpm_copy_matrix")
    return out


def cpm_matrix_layout(ctx: Context):
    """(mirror_blocks: bool, S bytes streamed per replica-step)."""
    m = ctypes.c_int32()
    nb = ctypes.c_int64()
    _check(_lib.cpm_matrix_layout(ctx.handle, ctypes.byref(m), ctypes.byref(nb)), "cpm_matrix_layout")
    return bool(m.value), int(nb.value)


def cpm_pair_list_layout(ctx: Context):
    """(ordered electrode pairs in the frozen-electrode force list, distinct G vectors of its
    compressed form or 0 for the full form)."""
    n = ctypes.c_int64()
    t = ctypes.c_int32()
    _check(_lib.cpm_pair_list_layout(ctx.handle, ctypes.byref(n), ctypes.byref(t)), "cpm_pair_list_layout")
    return int(n.value), int(t.value)


SAPPLY_VARIANTS = {"rows": 0, "stream": 1, "stream16": 2, "sym": 3, "sym-tma": 4}   # enum cpm_sapply_variant


def cpm_set_sapply_variant(ctx: Context, variant):
    v = SAPPLY_VARIANTS[variant] if isinstance(variant, str) else int(variant)
    _check(_lib.cpm_set_sapply_variant(ctx.handle, v), "cpm_set_sapply_variant")


FFT_VARIANTS = {"library": 0, "own": 1}               # enum cpm_fft_variant


def cpm_set_fft_variant(ctx: Context, variant):
    v = FFT_VARIANTS[variant] if isinstance(variant, str) else int(variant)
    _check(_lib.cpm_set_fft_variant(ctx.handle, v), "cpm_set_fft_variant")


MESH_VARIANTS = {"sites": 0, "brick": 1}              # enum cpm_mesh_variant


def cpm_set_mesh_variant(ctx: Context, variant):
    v = MESH_VARIANTS[variant] if isinstance(variant, str) else int(variant)
    _check(_lib.cpm_set_mesh_variant(ctx.handle, v), "cpm_set_mesh_variant")


def cpm_set_wait_test(ctx: Context, on: bool):
    """Test hook: the first bounded device waits give up at once (see include/cpm.h)."""
    _check(_lib.cpm_set_wait_test(ctx.handle, 1 if on else 0), "cpm_set_wait_test")


def cpm_set_pair_group(ctx: Context, gz: int):
    _check(_lib.cpm_set_pair_group(ctx.handle, int(gz)), "cpm_set_pair_group")


def cpm_get_pair_group(ctx: Context) -> int:
    v = ctypes.c_int32()
    _check(_lib.cpm_get_pair_group(ctx.handle, ctypes.byref(v)), "cpm_get_pair_group")
    return int(v.value)


PAIR_VARIANTS = {"cell": 0, "warp-elec": 1, "warp-elyt": 2, "warp": 3, "n3": 4, "n3-warp-elec": 5}   # enum cpm_pair_variant


def cpm_set_pair_variant(ctx: Context, variant):
    v = PAIR_VARIANTS[variant] if isinstance(variant, str) else int(variant)
    _check(_lib.cpm_set_pair_variant(ctx.handle, v), "cpm_set_pair_variant")


def cpm_get_pair_variant(ctx: Context) -> str:
    v = ctypes.c_int32()
    _check(_lib.cpm_get_pair_variant(ctx.handle, ctypes.byref(v)), "cpm_get_pair_variant")
    return {k: x for x, k in PAIR_VARIANTS.items()}[int(v.value)]


def cpm_autotune(ctx: Context, offsets, xyzq, dpsi, q, stream=None):
    """Time the available S-apply kernels, mesh convolutions and charge assignments on this input
    (one replica); keeps and returns the fastest as (S-apply, transform, assignment) names."""
    import torch
    ne = ctx.n_elec
    p_off = _dev(offsets, torch.int32, "offsets", 2)
    p_x = _dev(xyzq, torch.float64, "xyzq")
    p_d = _dev(dpsi, torch.float64, "dpsi", 1)
    out = (ctypes.c_int32 * 3)()
    _check(_lib.cpm_autotune(ctx.handle, p_off, p_x, p_d, _dev(q, torch.float64, "q", ne), _stream_ptr(stream),
                             out), "cpm_autotune")
    names_s = {v: k for k, v in SAPPLY_VARIANTS.items()}
    names_f = {v: k for k, v in FFT_VARIANTS.items()}
    names_m = {v: k for k, v in MESH_VARIANTS.items()}
    return names_s[out[0]], names_f[out[1]], names_m[out[2]]


def cpm_density_z(ctx: Context, n_rep: int, offsets, xyzq, q, nbins: int, rho, stream=None):
    """Adds the x-y averaged charge density of this configuration into rho [n_rep * nbins]."""
    import torch
    _check(_lib.cpm_density_z(ctx.handle, int(n_rep), _dev(offsets, torch.int32, "offsets", n_rep + 1),
                              _dev(xyzq, torch.float64, "xyzq"), _dev(q, torch.float64, "q", n_rep * ctx.n_elec),
                              int(nbins), _dev(rho, torch.float64, "rho", n_rep * nbins), _stream_ptr(stream)),
           "cpm_density_z")


def cpm_potential_z(ctx: Context, n_rep: int, nbins: int, rho, scale: float, dpsi, psi, stream=None):
    """psi [n_rep * nbins] (V) from the 1-D Poisson equation of rho * scale."""
    import torch
    _check(_lib.cpm_potential_z(ctx.handle, int(n_rep), int(nbins), _dev(rho, torch.float64, "rho", n_rep * nbins),
                                float(scale), _dev(dpsi, torch.float64, "dpsi", n_rep),
                                _dev(psi, torch.float64, "psi", n_rep * nbins), _stream_ptr(stream)),
           "cpm_potential_z")


def make_md_params(dt=2.0, charge_every=5, mass=(), sigma=(), eps=(), elec_type=-1, n_groups=1, lj_cut=0.0,
                   temperature=400.0, t_damp=100.0) -> CpmMdParams:
    p = CpmMdParams()
    n = max(len(mass), len(sigma), len(eps))
    if n < 1 or n > MD_MAX_TYPES:
        raise ValueError(f"between 1 and {MD_MAX_TYPES} types required")
    p.dt, p.charge_every, p.n_types = float(dt), int(charge_every), n
    for t in range(n):
        p.mass[t] = float(mass[t]) if t < len(mass) else 0.0
        p.lj_sigma[t] = float(sigma[t]) if t < len(sigma) else 0.0
        p.lj_epsilon[t] = float(eps[t]) if t < len(eps) else 0.0
    p.elec_type, p.n_groups = int(elec_type), int(n_groups)
    p.lj_cut, p.temperature, p.t_damp = float(lj_cut), float(temperature), float(t_damp)
    return p


class MDHandle:
    """Owning handle of a cpm_md integrator (destroyed with the object; keeps its context alive)."""

    def __init__(self, handle, ctx: Context, params: CpmMdParams, n_rep: int):
        self.handle, self.ctx, self.params, self.n_rep = handle, ctx, params, n_rep
        n, s = ctypes.c_int32(), ctypes.c_int32()
        _check(_lib.cpm_md_info(handle, ctypes.byref(n), ctypes.byref(s)), "cpm_md_info")
        self.n_sites, self.n_slots = n.value, s.value

    def close(self):
        h = getattr(self, "handle", None)
        if h:
            _lib.cpm_md_destroy(h)
            self.handle = None

    def __del__(self):
        self.close()


def cpm_md_create(ctx: Context, params: CpmMdParams, offsets, types, groups=None, stream=None) -> MDHandle:
    off = np.ascontiguousarray(offsets, dtype=np.int32)
    ty = np.ascontiguousarray(types, dtype=np.int32)
    gr = None if groups is None else np.ascontiguousarray(groups, dtype=np.int32)
    n_rep = len(off) - 1
    if n_rep < 1 or ty.shape != (int(off[-1]),) or (gr is not None and gr.shape != ty.shape):
        raise ValueError("offsets / types / groups have inconsistent shapes")
    out = ctypes.c_void_p()
    _check(_lib.cpm_md_create(ctx.handle, ctypes.byref(params), n_rep, off.ctypes.data, ty.ctypes.data,
                              None if gr is None else gr.ctypes.data, _stream_ptr(stream), ctypes.byref(out)),
           "cpm_md_create")
    return MDHandle(out.value, ctx, params, n_rep)


def cpm_md_run(md: MDHandle, n_steps: int, xyzq, vel, dpsi, q, psibar=None, energy=None, force=None, stream=None):
    import torch
    R, ne, n = md.n_rep, md.ctx.n_elec, md.n_sites
    _check(_lib.cpm_md_run(md.handle, int(n_steps), _dev(xyzq, torch.float64, "xyzq", 4 * n),
                           _dev(vel, torch.float64, "vel", 3 * n), _dev(dpsi, torch.float64, "dpsi", R),
                           _dev(q, torch.float64, "q", R * ne),
                           _dev(psibar, torch.float64, "psibar", R * md.ctx.ncons, True),
                           _dev(energy, torch.float64, "energy", R * MD_NENERGY, True),
                           _dev(force, torch.float64, "force", 3 * n, True), _stream_ptr(stream)),
           "cpm_md_run")


def cpm_md_advance(md: MDHandle, n_steps: int):
    _check(_lib.cpm_md_advance(md.handle, int(n_steps)), "cpm_md_advance")


def cpm_md_get_state(md: MDHandle, stream=None):
    """(step index, thermostat state [n_rep * n_groups, 2] of (xi, v_xi))."""
    step = ctypes.c_int64()
    th = np.zeros((md.n_slots, 2), dtype=np.float64)
    _check(_lib.cpm_md_get_state(md.handle, ctypes.byref(step), th.ctypes.data, _stream_ptr(stream)),
           "cpm_md_get_state")
    return int(step.value), th


def cpm_md_set_state(md: MDHandle, step: int, thermo=None, stream=None):
    th = None if thermo is None else np.ascontiguousarray(thermo, dtype=np.float64).reshape(-1)
    if th is not None and th.size != 2 * md.n_slots:
        raise ValueError(f"thermostat state needs {2 * md.n_slots} values")
    _check(_lib.cpm_md_set_state(md.handle, int(step), None if th is None else th.ctypes.data, _stream_ptr(stream)),
           "cpm_md_set_state")


def cpm_status(ctx: Context, stream=None) -> int:
    return int(_lib.cpm_status(ctx.handle, _stream_ptr(stream)))


def cpm_profile_enable(ctx: Context, capacity: int):
    _check(_lib.cpm_profile_enable(ctx.handle, int(capacity)), "cpm_profile_enable")


def cpm_profile_read(ctx: Context) -> dict:
    """{phase name: (milliseconds, intervals)} accumulated since the last read."""
    ms = np.zeros(len(PHASES), dtype=np.float64)
    cnt = np.zeros(len(PHASES), dtype=np.int64)
    _check(_lib.cpm_profile_read(ctx.handle, ms.ctypes.data, cnt.ctypes.data), "cpm_profile_read")
    return {name: (float(ms[k]), int(cnt[k])) for k, name in enumerate(PHASES)}


def cpm_counters(ctx: Context) -> int:
    """Kernel launches issued by the per-step calls of ctx so far."""
    v = ctypes.c_int64()
    _check(_lib.cpm_counters(ctx.handle, ctypes.byref(v)), "cpm_counters")
    return v.value


def cpm_strerror(status: int) -> str:
    return _lib.cpm_strerror(status).decode()
