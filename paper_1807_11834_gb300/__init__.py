"""Python binding of the GB300 particle <-> dual-grid coupling library.

A thin ctypes layer over the C ABI of ``include/cg.h``.  It marshals torch
CUDA tensors (``data_ptr()``) and the current CUDA stream, and checks
shapes and dtypes; every step of the coupling runs in the library's own
CUDA kernels.  There is no CPU fallback: if the shared library has not
been built, importing the binding succeeds but the first call raises.

The step follows Fig. 1 and Sec. 2 of Pozzetti et al., "A parallel
dual-grid multiscale approach to CFD-DEM couplings" (arXiv 1807.11834):
particles are binned on the coarse bulk grid, porosity and the reaction
source are deposited there, the fluid velocity is averaged from the fine
grid, drag is computed at the particles (Eq. DragLaw), and the source is
projected back to the fine grid.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libcg.so")

CG_OK = 0
STATUS_NAMES = {0: "CG_OK", 1: "CG_ERR_INVALID_ARG", 2: "CG_ERR_CUDA", 3: "CG_ERR_OOM",
                4: "CG_ERR_NOT_BINNED", 5: "CG_ERR_OUT_OF_RANGE", 6: "CG_ERR_TIMEOUT",
                7: "CG_ERR_NONFINITE"}
CG_FP32, CG_FP64 = 0, 1
CG_DRAG_DI_FELICE, CG_DRAG_ERGUN_WEN_YU = 0, 1
CG_INTERP_TRILINEAR, CG_INTERP_CELL = 0, 1
CG_DEP_VOLUME, CG_DEP_MOMENTUM = 0, 1
CG_FLAG_OUTSIDE, CG_FLAG_NONFINITE, CG_FLAG_EPS_CLAMPED, CG_FLAG_TIMEOUT = 1, 2, 4, 8
CG_NSUMS = 16
CG_NCOUNTS = 5
# binning sort choices (descriptor key "sort_digits"): automatic, per-cell
# sort, or 6..11 for the digit sort with digits of that many bits at most
CG_SORT_AUTO = 0
CG_SORT_CELLS = 1
CG_SORT_CELLS_AUTO_MAX = 1 << 23
CG_SORT_CELLS_AUTO_DENSITY = 32
# the drag's stencil reads (descriptor key "stencil")
CG_STENCIL_GATHER, CG_STENCIL_WINDOW = 0, 1
SUM_NAMES = ["vol_particles", "vol_deposited", "F_x", "F_y", "F_z", "SbVb_x", "SbVb_y", "SbVb_z",
             "SfVf_x", "SfVf_y", "SfVf_z", "F_abs", "mom_x", "mom_y", "mom_z", "n_clamped"]


class CgError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {STATUS_NAMES.get(code, code)}")


class GridDesc(C.Structure):
    _fields_ = [("origin", C.c_double * 3), ("extent", C.c_double * 3), ("fine_n", C.c_int32 * 3),
                ("ratio", C.c_int32), ("prec", C.c_int32), ("law", C.c_int32), ("interp", C.c_int32),
                ("sort_digits", C.c_int32), ("stencil", C.c_int32), ("rho_f", C.c_double), ("mu_f", C.c_double),
                ("rho_p", C.c_double), ("eps_switch", C.c_double), ("eps_min", C.c_double),
                ("gravity", C.c_double * 3)]


class Particles(C.Structure):
    _fields_ = [("n", C.c_int64), ("pos_d", C.c_void_p), ("vel", C.c_void_p)]


class StepOut(C.Structure):
    _fields_ = [("eps_bulk", C.c_void_p), ("u_bulk", C.c_void_p), ("var_bulk", C.c_void_p),
                ("S_bulk", C.c_void_p), ("force", C.c_void_p), ("S_fine", C.c_void_p),
                ("eps_fine", C.c_void_p), ("sums", C.c_void_p), ("cell", C.c_void_p),
                ("perm", C.c_void_p), ("cell_start", C.c_void_p), ("implicit_bulk", C.c_void_p),
                ("implicit_fine", C.c_void_p)]


class BoxGrid(C.Structure):
    _fields_ = [("origin", C.c_double * 3), ("extent", C.c_double * 3), ("n", C.c_int32 * 3),
                ("prec", C.c_int32)]


class BatchItem(C.Structure):
    _fields_ = [("desc", GridDesc), ("particles", Particles), ("u_fine", C.c_void_p), ("out", StepOut)]


class BatchConfig(C.Structure):
    _fields_ = [("digit_bits", C.c_int32), ("drag_items", C.c_int32), ("avg_items", C.c_int32),
                ("seg_chunks", C.c_int32), ("grid_mult", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lock = threading.Lock()
_lib = None

_SIGS = {
    "cg_status_string": (C.c_char_p, [C.c_int]),
    "cg_create_grids": (C.c_int, [C.POINTER(GridDesc), C.c_void_p, C.POINTER(C.c_void_p)]),
    "cg_destroy_grids": (C.c_int, [C.c_void_p]),
    "cg_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "cg_grid_dims": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "cg_bin_particles": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "cg_bin_particles_static": (C.c_int, [C.POINTER(GridDesc), C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                          C.c_void_p, C.c_void_p]),
    "cg_deposit": (C.c_int, [C.c_void_p, C.c_int32, C.c_int64, C.c_void_p, C.c_void_p]),
    "cg_average_fine_to_bulk": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "cg_drag": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                          C.c_void_p, C.c_void_p, C.c_void_p]),
    "cg_project_bulk_to_fine": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    "cg_step": (C.c_int, [C.c_void_p, C.POINTER(Particles), C.c_void_p, C.POINTER(StepOut), C.c_double]),
    "cg_step_host": (C.c_int, [C.c_void_p, C.POINTER(Particles), C.c_void_p, C.POINTER(StepOut), C.c_double]),
    "cg_step_sorted": (C.c_int, [C.c_void_p, C.POINTER(Particles), C.POINTER(Particles), C.c_void_p,
                                 C.POINTER(StepOut), C.c_double]),
    "cg_step_host_async": (C.c_int, [C.c_void_p, C.POINTER(Particles), C.c_void_p, C.POINTER(StepOut),
                                     C.c_double]),
    "cg_step_host_wait": (C.c_int, [C.c_void_p]),
    "cg_sync_status": (C.c_int, [C.c_void_p, C.POINTER(C.c_uint32), C.POINTER(C.c_int64)]),
    "cg_launch_count": (C.c_int64, [C.c_void_p]),
    "cg_profile_enable": (C.c_int, [C.c_void_p, C.c_int32]),
    "cg_profile_reset": (C.c_int, [C.c_void_p]),
    "cg_profile_read": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_char_p), C.POINTER(C.c_int64),
                                  C.POINTER(C.c_double), C.POINTER(C.c_int32)]),
    "cg_mlp_create": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p)]),
    "cg_mlp_destroy": (C.c_int, [C.c_void_p]),
    "cg_mlp_get_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "cg_mlp_set_params": (C.c_int, [C.c_void_p, C.c_void_p]),
    "cg_mlp_forward": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]),
    "cg_mlp_grads": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]),
    "cg_mlp_train_step": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_float, C.c_void_p]),
    "cg_mlp_sync_status": (C.c_int, [C.c_void_p, C.POINTER(C.c_uint32)]),
    "cg_mlp_save": (C.c_int, [C.c_void_p, C.c_char_p, C.c_char_p]),
    "cg_mlp_load": (C.c_int, [C.c_char_p, C.c_void_p, C.POINTER(C.c_void_p)]),
    "cg_mlp_checkpoint_write": (C.c_int, [C.c_char_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_char_p]),
    "cg_mlp_checkpoint_read": (C.c_int, [C.c_char_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "cg_mlp_set_activation": (C.c_int, [C.c_void_p, C.c_int32]),
    "cg_mlp_get_activation": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32)]),
    "cg_mlp_wait_selftest": (C.c_int, [C.c_void_p, C.c_uint32]),
    "cg_debug_fail_alloc_after": (C.c_int, [C.c_int64]),
    "cg_mlp_features": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "cg_mlp_bind": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]),
    "cg_step_learned": (C.c_int, [C.c_void_p, C.POINTER(Particles), C.c_void_p, C.POINTER(StepOut), C.c_double,
                                  C.c_void_p, C.c_int32]),
    "cg_batch_default_config": (C.c_int, [C.POINTER(BatchConfig)]),
    "cg_batch_create": (C.c_int, [C.POINTER(BatchItem), C.c_int32, C.c_void_p, C.POINTER(C.c_void_p)]),
    "cg_batch_destroy": (C.c_int, [C.c_void_p]),
    "cg_reorder_particles": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "cg_map_create": (C.c_int, [C.POINTER(BoxGrid), C.POINTER(BoxGrid), C.c_void_p, C.POINTER(C.c_void_p)]),
    "cg_map_destroy": (C.c_int, [C.c_void_p]),
    "cg_map_average": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    "cg_map_project": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    "cg_batch_set_config": (C.c_int, [C.c_void_p, C.POINTER(BatchConfig)]),
    "cg_batch_get_config": (C.c_int, [C.c_void_p, C.POINTER(BatchConfig)]),
    "cg_batch_use_graph": (C.c_int, [C.c_void_p, C.c_int32]),
    "cg_batch_step": (C.c_int, [C.c_void_p, C.c_double]),
    "cg_batch_step_each": (C.c_int, [C.c_void_p, C.c_double]),
    "cg_batch_tune": (C.c_int, [C.c_void_p, C.c_int32, C.c_char_p, C.POINTER(BatchConfig),
                                C.POINTER(C.c_double)]),
    "cg_batch_sync_status": (C.c_int, [C.c_void_p, C.POINTER(C.c_uint32), C.POINTER(C.c_int64)]),
    "cg_batch_instance": (C.c_void_p, [C.c_void_p, C.c_int32]),
    "cg_batch_launch_count": (C.c_int64, [C.c_void_p]),
    "cg_batch_launches_per_step": (C.c_int64, [C.c_void_p]),
}

MLP_NPARAM = 5313
MLP_NFEAT = 7
MLP_ACTIVATIONS = {"gelu": 0, "relu": 1}   # CG_MLP_GELU, CG_MLP_RELU


def lib():
    """The loaded shared library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA coupling library not built ({LIB_PATH}); "
                                   "run __graft_entry__.build() first")
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(code, where):
    if code != CG_OK:
        raise CgError(code, where)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def check_tensor(t, numel, dtype, on_device, name="tensor"):
    """The binding's check of a tensor before its pointer crosses the ABI:
    device memory for the device entries (host memory for the host-buffer
    ones), contiguous, and the dtype and element count the entry reads or
    writes.  A host pointer handed to a device entry would be dereferenced by
    a kernel; this stops it on the host."""
    if t.is_cuda != on_device or not t.is_contiguous() or t.dtype != dtype:
        where = "CUDA" if on_device else "host"
        raise ValueError(f"{name}: need a contiguous {where} {dtype} tensor")
    if numel is not None and t.numel() != int(numel):
        raise ValueError(f"{name}: need {numel} elements, got {t.numel()}")
    return t


# Components, cell set and dtype of each cg_step_out field ("T": the grids'
# precision); the counts the ABI documents for each pointer.
STEP_OUT_LAYOUT = {
    "eps_bulk": (1, "bulk", "f64"), "u_bulk": (3, "bulk", "T"), "var_bulk": (1, "bulk", "T"),
    "S_bulk": (3, "bulk", "T"), "force": (3, "particles", "T"), "S_fine": (3, "fine", "T"),
    "eps_fine": (1, "fine", "T"), "sums": (CG_NSUMS, "one", "f64"), "cell": (1, "particles", "i32"),
    "perm": (1, "particles", "i32"), "cell_start": (1, "bulk+1", "i32"), "implicit_bulk": (4, "bulk", "T"),
    "implicit_fine": (4, "fine", "T"),
}


def check_step_outputs(out, n, n_bulk, n_fine, dtype, on_device):
    """check_tensor for every output of one step that is not None (which
    combinations may be None is the library's to check)."""
    import torch
    count = {"bulk": n_bulk, "fine": n_fine, "particles": n, "bulk+1": n_bulk + 1, "one": 1}
    kinds = {"T": dtype, "f64": torch.float64, "i32": torch.int32}
    for name, (comps, cells, kind) in STEP_OUT_LAYOUT.items():
        t = out.get(name)
        if t is not None:
            check_tensor(t, comps * count[cells], kinds[kind], on_device, name)


def _stream_handle(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def make_desc(d: dict) -> GridDesc:
    g = GridDesc()
    g.origin[:] = d["origin"]
    g.extent[:] = d["extent"]
    g.fine_n[:] = d["fine_n"]
    g.ratio = d["ratio"]
    g.prec = CG_FP64 if d.get("fp64", False) else CG_FP32
    g.law = d["law"]
    g.interp = d.get("interp", CG_INTERP_TRILINEAR)
    g.rho_f, g.mu_f, g.rho_p = d["rho_f"], d["mu_f"], d["rho_p"]
    g.eps_switch, g.eps_min = d["eps_switch"], d["eps_min"]
    g.sort_digits = int(d.get("sort_digits", 0))
    g.stencil = int(d.get("stencil", CG_STENCIL_GATHER))
    g.gravity[:] = d.get("gravity", (0.0, 0.0, 0.0))
    return g


class Grids:
    """Owner of a ``cg_grids`` handle (one coupling instance on cuda:0).

    All tensors passed in must be contiguous CUDA tensors of the path
    dtype (float32 or float64; the bulk porosity is always float64)."""

    def __init__(self, desc: dict, stream=None):
        import torch
        self.desc = dict(desc)
        self.dtype = torch.float64 if desc.get("fp64", False) else torch.float32
        self._d = make_desc(desc)
        h = C.c_void_p()
        _check(lib().cg_create_grids(C.byref(self._d), _stream_handle(stream), C.byref(h)), "cg_create_grids")
        self.h = h
        nb = (C.c_int32 * 3)()
        nbulk, nfine = C.c_int64(), C.c_int64()
        _check(lib().cg_grid_dims(self.h, nb, C.byref(nbulk), C.byref(nfine)), "cg_grid_dims")
        self.bulk_n = tuple(nb)
        self.n_bulk = nbulk.value
        self.n_fine = nfine.value

    def close(self):
        if getattr(self, "h", None):
            lib().cg_destroy_grids(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- argument checks (marshalling only) ---------------------------------
    def _t(self, t, shape, dtype=None, name="tensor"):
        if t is None:
            return None
        return check_tensor(t, shape, dtype or self.dtype, True, name)

    def set_stream(self, stream=None):
        _check(lib().cg_set_stream(self.h, _stream_handle(stream)), "cg_set_stream")

    # -- the C ABI, one method per entry -----------------------------------
    def cg_bin_particles(self, pos_d, cell=None, perm=None, cell_start=None):
        import torch
        n = pos_d.shape[0]
        self._t(pos_d, 4 * n, name="pos_d")
        self._t(cell, n, torch.int32, "cell")
        self._t(perm, n, torch.int32, "perm")
        self._t(cell_start, self.n_bulk + 1, torch.int32, "cell_start")
        _check(lib().cg_bin_particles(self.h, n, _ptr(pos_d), _ptr(cell), _ptr(perm), _ptr(cell_start)),
               "cg_bin_particles")

    def cg_deposit(self, kind, n, per_particle, bulk_out):
        import torch
        if kind == CG_DEP_VOLUME:
            self._t(per_particle, 4 * n, name="pos_d")
            self._t(bulk_out, self.n_bulk, torch.float64, "eps_bulk")
        else:
            self._t(per_particle, 3 * n, name="force")
            self._t(bulk_out, 3 * self.n_bulk, name="S_bulk")
        _check(lib().cg_deposit(self.h, kind, n, _ptr(per_particle), _ptr(bulk_out)), "cg_deposit")

    def cg_average_fine_to_bulk(self, u_fine, u_bulk, var_bulk=None):
        self._t(u_fine, 3 * self.n_fine, name="u_fine")
        self._t(u_bulk, 3 * self.n_bulk, name="u_bulk")
        self._t(var_bulk, self.n_bulk, name="var_bulk")
        _check(lib().cg_average_fine_to_bulk(self.h, _ptr(u_fine), _ptr(u_bulk), _ptr(var_bulk)),
               "cg_average_fine_to_bulk")

    def cg_drag(self, pos_d, vel, eps_bulk, u_bulk, force, S_bulk=None, mlp=None):
        import torch
        n = pos_d.shape[0]
        self._t(pos_d, 4 * n, name="pos_d")
        self._t(vel, 4 * n, name="vel")
        self._t(eps_bulk, self.n_bulk, torch.float64, "eps_bulk")
        self._t(u_bulk, 3 * self.n_bulk, name="u_bulk")
        self._t(force, 3 * n, name="force")
        self._t(S_bulk, 3 * self.n_bulk, name="S_bulk")
        _check(lib().cg_drag(self.h, n, _ptr(pos_d), _ptr(vel), _ptr(eps_bulk), _ptr(u_bulk), _ptr(force),
                             _ptr(S_bulk), None if mlp is None else mlp.h), "cg_drag")

    def cg_project_bulk_to_fine(self, bulk, fine_out):
        ncomp = bulk.numel() // self.n_bulk
        self._t(bulk, ncomp * self.n_bulk, name="bulk")
        self._t(fine_out, ncomp * self.n_fine, name="fine_out")
        _check(lib().cg_project_bulk_to_fine(self.h, ncomp, _ptr(bulk), _ptr(fine_out)),
               "cg_project_bulk_to_fine")

    def alloc_outputs(self, n, var=True, eps_fine=False, bins=False, implicit=False, implicit_fine=False,
                      device="cuda"):
        """Output tensors of one step (device), by cg_step_out field name;
        implicit: the semi-implicit coefficients [4][n_b] (A, b), and with
        implicit_fine their projection [4][n_f]."""
        import torch
        kw = dict(device=device, dtype=self.dtype)
        o = dict(eps_bulk=torch.empty(self.n_bulk, device=device, dtype=torch.float64),
                 u_bulk=torch.empty(3, self.n_bulk, **kw),
                 var_bulk=torch.empty(self.n_bulk, **kw) if var else None,
                 S_bulk=torch.empty(3, self.n_bulk, **kw),
                 force=torch.empty(3, n, **kw),
                 S_fine=torch.empty(3, self.n_fine, **kw),
                 eps_fine=torch.empty(self.n_fine, **kw) if eps_fine else None,
                 sums=torch.empty(CG_NSUMS, device=device, dtype=torch.float64))
        if implicit or implicit_fine:
            o["implicit_bulk"] = torch.empty(4, self.n_bulk, **kw)
        if implicit_fine:
            o["implicit_fine"] = torch.empty(4, self.n_fine, **kw)
        if bins:
            o["cell"] = torch.empty(n, device=device, dtype=torch.int32)
            o["perm"] = torch.empty(n, device=device, dtype=torch.int32)
            o["cell_start"] = torch.empty(self.n_bulk + 1, device=device, dtype=torch.int32)
        return o

    @staticmethod
    def _out_struct(out):
        so = StepOut()
        for name, _ in StepOut._fields_:
            t = out.get(name)
            setattr(so, name, None if t is None else t.data_ptr())
        return so

    def cg_reorder_particles(self, pos_d, vel, pos_out, vel_out):
        """Gather the particle records into the order of the last binning
        of these n particles (vel / vel_out may both be None)."""
        n = pos_d.shape[0]
        self._t(pos_d, 4 * n, name="pos_d")
        self._t(pos_out, 4 * n, name="pos_out")
        if vel is not None:
            self._t(vel, 4 * n, name="vel")
            self._t(vel_out, 4 * n, name="vel_out")
        _check(lib().cg_reorder_particles(self.h, n, _ptr(pos_d), _ptr(vel), _ptr(pos_out), _ptr(vel_out)),
               "cg_reorder_particles")

    def cg_step(self, pos_d, vel, u_fine, out, dt=0.0):
        n = pos_d.shape[0]
        self._t(pos_d, 4 * n, name="pos_d")
        self._t(vel, 4 * n, name="vel")
        self._t(u_fine, 3 * self.n_fine, name="u_fine")
        check_step_outputs(out, n, self.n_bulk, self.n_fine, self.dtype, True)
        p = Particles(n, pos_d.data_ptr() if n else None, vel.data_ptr() if n else None)
        so = self._out_struct(out)
        _check(lib().cg_step(self.h, C.byref(p), _ptr(u_fine), C.byref(so), float(dt)), "cg_step")

    def cg_step_sorted(self, pos_d, vel, pos_out, vel_out, u_fine, out, dt=0.0):
        """cg_step that writes the (advanced) particles to pos_out / vel_out in
        this step's cell order (pos_out[s] = particle out["perm"][s]); pos_d
        and vel are not written.  Keep the particles this way from step to
        step (swap the two pairs of arrays) and each binning starts from the
        last one."""
        n = pos_d.shape[0]
        self._t(pos_d, 4 * n, name="pos_d")
        self._t(vel, 4 * n, name="vel")
        self._t(pos_out, 4 * n, name="pos_out")
        self._t(vel_out, 4 * n, name="vel_out")
        self._t(u_fine, 3 * self.n_fine, name="u_fine")
        check_step_outputs(out, n, self.n_bulk, self.n_fine, self.dtype, True)
        p = Particles(n, pos_d.data_ptr() if n else None, vel.data_ptr() if n else None)
        po = Particles(n, pos_out.data_ptr() if n else None, vel_out.data_ptr() if n else None)
        so = self._out_struct(out)
        _check(lib().cg_step_sorted(self.h, C.byref(p), C.byref(po), _ptr(u_fine), C.byref(so), float(dt)),
               "cg_step_sorted")

    def cg_step_learned(self, pos_d, vel, u_fine, out, mlp, age, dt=0.0):
        """cg_step with the learned closure: age 0 refreshes (cg_step);
        age >= 1 uses out["u_bulk"] and out["var_bulk"] as the stale record
        (inputs) of that age."""
        n = pos_d.shape[0]
        self._t(pos_d, 4 * n, name="pos_d")
        self._t(vel, 4 * n, name="vel")
        self._t(u_fine, 3 * self.n_fine, name="u_fine")
        check_step_outputs(out, n, self.n_bulk, self.n_fine, self.dtype, True)
        p = Particles(n, pos_d.data_ptr() if n else None, vel.data_ptr() if n else None)
        so = self._out_struct(out)
        _check(lib().cg_step_learned(self.h, C.byref(p), _ptr(u_fine), C.byref(so), float(dt), mlp.h,
                                     int(age)), "cg_step_learned")

    def cg_mlp_features(self, pos_d, vel, eps_bulk, u_stale, var_stale, u_fresh, features, target):
        """Closure features [n][8] float32 and targets [n] float32 at every particle."""
        import torch
        n = pos_d.shape[0]
        self._t(pos_d, 4 * n, name="pos_d")
        self._t(vel, 4 * n, name="vel")
        self._t(eps_bulk, self.n_bulk, torch.float64, "eps_bulk")
        self._t(u_stale, 3 * self.n_bulk, name="u_stale")
        self._t(var_stale, self.n_bulk, name="var_stale")
        self._t(u_fresh, 3 * self.n_bulk, name="u_fresh")
        self._t(features, 8 * n, torch.float32, "features")
        self._t(target, n, torch.float32, "target")
        _check(lib().cg_mlp_features(self.h, n, _ptr(pos_d), _ptr(vel), _ptr(eps_bulk), _ptr(u_stale),
                                     _ptr(var_stale), _ptr(u_fresh), _ptr(features), _ptr(target)),
               "cg_mlp_features")

    def _host_step_args(self, pos_d, vel, u_fine, out):
        n = pos_d.shape[0]
        check_tensor(pos_d, 4 * n, self.dtype, False, "pos_d")
        check_tensor(vel, 4 * n, self.dtype, False, "vel")
        check_tensor(u_fine, 3 * self.n_fine, self.dtype, False, "u_fine")
        check_step_outputs(out, n, self.n_bulk, self.n_fine, self.dtype, False)

    def cg_step_host(self, pos_d, vel, u_fine, out, dt=0.0):
        """Same as cg_step on host (CPU, ideally pinned) tensors; blocks."""
        n = pos_d.shape[0]
        self._host_step_args(pos_d, vel, u_fine, out)
        p = Particles(n, pos_d.data_ptr() if n else None, vel.data_ptr() if n else None)
        so = self._out_struct(out)
        _check(lib().cg_step_host(self.h, C.byref(p), _ptr(u_fine), C.byref(so), float(dt)), "cg_step_host")

    def cg_step_host_async(self, pos_d, vel, u_fine, out, dt=0.0):
        """cg_step_host without the final wait (call cg_step_host_wait before
        reading the outputs or changing the inputs)."""
        n = pos_d.shape[0]
        self._host_step_args(pos_d, vel, u_fine, out)
        p = Particles(n, pos_d.data_ptr() if n else None, vel.data_ptr() if n else None)
        so = self._out_struct(out)
        _check(lib().cg_step_host_async(self.h, C.byref(p), _ptr(u_fine), C.byref(so), float(dt)),
               "cg_step_host_async")

    def cg_step_host_wait(self):
        _check(lib().cg_step_host_wait(self.h), "cg_step_host_wait")

    def cg_sync_status(self):
        """(return code, flags, [outside, nonfinite, clamped, timeouts, fallbacks])."""
        flags = C.c_uint32()
        counts = (C.c_int64 * CG_NCOUNTS)()
        rc = lib().cg_sync_status(self.h, C.byref(flags), counts)
        return rc, flags.value, list(counts)

    def cg_launch_count(self):
        return int(lib().cg_launch_count(self.h))

    def cg_profile_enable(self, on=True):
        _check(lib().cg_profile_enable(self.h, 1 if on else 0), "cg_profile_enable")

    def cg_profile_reset(self):
        _check(lib().cg_profile_reset(self.h), "cg_profile_reset")

    def cg_profile_read(self):
        """{kernel name: (launches, total ms)} since the last reset."""
        count = C.c_int32()
        _check(lib().cg_profile_read(self.h, -1, None, None, None, C.byref(count)), "cg_profile_read")
        res = {}
        for k in range(count.value):
            name, launches, ms = C.c_char_p(), C.c_int64(), C.c_double()
            _check(lib().cg_profile_read(self.h, k, C.byref(name), C.byref(launches), C.byref(ms), None),
                   "cg_profile_read")
            res[name.value.decode()] = (launches.value, ms.value)
        return res


def cg_bin_particles_static(desc: dict, pos_d, perm, cell_start, cell=None, stream=None):
    """Binning without any device allocation (fixed scratch inside the
    library, at most 262,144 particles); same outputs as cg_bin_particles.
    Every tensor is checked as the handle entries check theirs: CUDA memory,
    contiguous, the descriptor's precision for pos_d ([n][4]) and int32
    perm / cell ([n]) and cell_start ([n_b + 1])."""
    import torch
    d = make_desc(desc)
    n = pos_d.shape[0]
    dtype = torch.float64 if desc.get("fp64", False) else torch.float32
    ratio = int(desc["ratio"])
    n_bulk = 1
    for f in desc["fine_n"]:
        n_bulk *= int(f) // ratio if ratio > 0 else 0
    check_tensor(pos_d, 4 * n, dtype, True, "pos_d")
    check_tensor(perm, n, torch.int32, True, "perm")
    check_tensor(cell_start, n_bulk + 1, torch.int32, True, "cell_start")
    if cell is not None:
        check_tensor(cell, n, torch.int32, True, "cell")
    _check(lib().cg_bin_particles_static(C.byref(d), n, _ptr(pos_d), _ptr(cell), _ptr(perm), _ptr(cell_start),
                                         _stream_handle(stream)), "cg_bin_particles_static")


def _activation_code(activation):
    if activation not in MLP_ACTIVATIONS:
        raise ValueError(f"activation must be one of {sorted(MLP_ACTIVATIONS)}")
    return MLP_ACTIVATIONS[activation]


def checkpoint_write(path, params, feat_lo, feat_hi, meta=None, activation="gelu"):
    """cg_mlp_checkpoint_write: a closure checkpoint from host arrays (no device)."""
    import json
    import numpy as np
    p = np.ascontiguousarray(params, dtype=np.float32)
    lo = np.ascontiguousarray(feat_lo, dtype=np.float32)
    hi = np.ascontiguousarray(feat_hi, dtype=np.float32)
    if p.size != MLP_NPARAM or lo.size != MLP_NFEAT or hi.size != MLP_NFEAT:
        raise ValueError("bad closure parameter or feature-box sizes")
    _check(lib().cg_mlp_checkpoint_write(os.fsencode(path), p.ctypes.data, lo.ctypes.data, hi.ctypes.data,
                                         _activation_code(activation), json.dumps(meta or {}).encode()),
           "cg_mlp_checkpoint_write")


def checkpoint_read(path):
    """cg_mlp_checkpoint_read: (params, feat_lo, feat_hi) float32 arrays of a
    checkpoint and its activation ("gelu" or "relu")."""
    import numpy as np
    p = np.zeros(MLP_NPARAM, np.float32)
    lo = np.zeros(MLP_NFEAT, np.float32)
    hi = np.zeros(MLP_NFEAT, np.float32)
    act = C.c_int32(-1)
    _check(lib().cg_mlp_checkpoint_read(os.fsencode(path), p.ctypes.data, lo.ctypes.data, hi.ctypes.data,
                                        C.addressof(act)), "cg_mlp_checkpoint_read")
    return p, lo, hi, {v: k for k, v in MLP_ACTIVATIONS.items()}[act.value]


class Mlp:
    """Owner of a ``cg_mlp`` closure handle (learned drag correction).
    Parameters are a flat float32 array of MLP_NPARAM (W1, b1, W2, b2, w3, b3)."""

    def __init__(self, params, feat_lo, feat_hi, stream=None, activation="gelu"):
        import numpy as np
        p = np.ascontiguousarray(params, dtype=np.float32)
        lo = np.ascontiguousarray(feat_lo, dtype=np.float32)
        hi = np.ascontiguousarray(feat_hi, dtype=np.float32)
        if p.size != MLP_NPARAM or lo.size != MLP_NFEAT or hi.size != MLP_NFEAT:
            raise ValueError("bad closure parameter or feature-box sizes")
        code = _activation_code(activation)
        h = C.c_void_p()
        _check(lib().cg_mlp_create(p.ctypes.data, lo.ctypes.data, hi.ctypes.data, _stream_handle(stream),
                                   C.byref(h)), "cg_mlp_create")
        self.h = h
        self.lo, self.hi = lo, hi
        _check(lib().cg_mlp_set_activation(self.h, code), "cg_mlp_set_activation")

    @property
    def activation(self):
        """The closure's activation, "gelu" or "relu" (cg_mlp_get_activation)."""
        a = C.c_int32(-1)
        _check(lib().cg_mlp_get_activation(self.h, C.byref(a)), "cg_mlp_get_activation")
        return {v: k for k, v in MLP_ACTIVATIONS.items()}[a.value]

    @classmethod
    def load(cls, path, stream=None):
        """The closure of a checkpoint (cg_mlp_load)."""
        import numpy as np
        m = cls.__new__(cls)
        h = C.c_void_p()
        _check(lib().cg_mlp_load(os.fsencode(path), _stream_handle(stream), C.byref(h)), "cg_mlp_load")
        m.h = h
        m.lo = np.zeros(MLP_NFEAT, np.float32)
        m.hi = np.zeros(MLP_NFEAT, np.float32)
        _check(lib().cg_mlp_checkpoint_read(os.fsencode(path), None, m.lo.ctypes.data, m.hi.ctypes.data, None),
               "cg_mlp_checkpoint_read")
        return m

    def save(self, path, meta=None):
        """Checkpoint of the current parameters, feature box and activation (cg_mlp_save);
        meta: a JSON-serialisable dict kept in the head."""
        import json
        _check(lib().cg_mlp_save(self.h, os.fsencode(path), json.dumps(meta or {}).encode()), "cg_mlp_save")

    def close(self):
        if getattr(self, "h", None):
            lib().cg_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self, grads=False):
        import numpy as np
        p = np.zeros(MLP_NPARAM, np.float32)
        g = np.zeros(MLP_NPARAM, np.float32) if grads else None
        _check(lib().cg_mlp_get_params(self.h, p.ctypes.data, None if g is None else g.ctypes.data),
               "cg_mlp_get_params")
        return (p, g) if grads else p

    def set_params(self, params):
        import numpy as np
        p = np.ascontiguousarray(params, dtype=np.float32)
        _check(lib().cg_mlp_set_params(self.h, p.ctypes.data), "cg_mlp_set_params")

    @staticmethod
    def _batch(features, targets=None, loss=None):
        """Rows of a feature batch ([n][8] float32 on the device) after the
        checks of its companions (targets [n], loss [1], both float32)."""
        import torch
        n = features.shape[0]
        check_tensor(features, 8 * n, torch.float32, True, "features")
        if targets is not None:
            check_tensor(targets, n, torch.float32, True, "targets")
        if loss is not None:
            check_tensor(loss, 1, torch.float32, True, "loss")
        return n

    def forward(self, features, c_out, in_range=None):
        import torch
        n = Mlp._batch(features)
        check_tensor(c_out, n, torch.float32, True, "c_out")
        if in_range is not None:
            check_tensor(in_range, n, torch.int32, True, "in_range")
        _check(lib().cg_mlp_forward(self.h, n, _ptr(features), _ptr(c_out), _ptr(in_range)), "cg_mlp_forward")

    def grads(self, features, targets, loss=None):
        n = Mlp._batch(features, targets, loss)
        _check(lib().cg_mlp_grads(self.h, n, _ptr(features), _ptr(targets), _ptr(loss)), "cg_mlp_grads")

    def train_step(self, features, targets, lr, loss=None):
        n = Mlp._batch(features, targets, loss)
        _check(lib().cg_mlp_train_step(self.h, n, _ptr(features), _ptr(targets), float(lr), _ptr(loss)),
               "cg_mlp_train_step")

    def sync_status(self):
        flags = C.c_uint32()
        rc = lib().cg_mlp_sync_status(self.h, C.byref(flags))
        return rc, flags.value

    def wait_selftest(self, polls):
        """Enqueue the bounded-wait check (cg_mlp_wait_selftest): the next
        sync_status reports CG_ERR_TIMEOUT."""
        _check(lib().cg_mlp_wait_selftest(self.h, int(polls)), "cg_mlp_wait_selftest")

    def bind(self, var_stale, u_fine, age=1):
        """Stale variance field, fine velocity and record age used by
        Grids.cg_drag(mlp=self) (float32 device tensors, kept alive by this
        object)."""
        import torch
        for name, t in (("var_stale", var_stale), ("u_fine", u_fine)):
            if t is not None:
                check_tensor(t, None, torch.float32, True, name)
        self._bound = (var_stale, u_fine)
        _check(lib().cg_mlp_bind(self.h, _ptr(var_stale), _ptr(u_fine), int(age)), "cg_mlp_bind")


class Batch:
    """Owner of a ``cg_batch``: many FP32 coupling instances stepped by one
    persistent launch per phase.  ``instances`` is a list of
    (desc dict, pos_d, vel, u_fine, out dict) with contiguous CUDA float32
    tensors (out as from Grids.alloc_outputs, bins=False); the tensors are
    kept alive by this object."""

    def __init__(self, instances, stream=None):
        items = (BatchItem * len(instances))()
        self._keep = []
        for k, (desc, pos, vel, uf, out) in enumerate(instances):
            # device memory only (a host pointer would reach a kernel); sizes,
            # precision and descriptors are the library's to check
            for t in [pos, vel, uf] + [v for v in out.values() if v is not None]:
                if not t.is_cuda or not t.is_contiguous():
                    raise ValueError(f"batch instance {k}: contiguous CUDA tensors expected")
            it = items[k]
            it.desc = make_desc(desc)
            it.particles = Particles(pos.shape[0], pos.data_ptr(), vel.data_ptr())
            it.u_fine = uf.data_ptr()
            it.out = Grids._out_struct(out)
            self._keep.append((pos, vel, uf, out))
        self._items = items
        h = C.c_void_p()
        _check(lib().cg_batch_create(items, len(instances), _stream_handle(stream), C.byref(h)), "cg_batch_create")
        self.h = h
        self.count = len(instances)

    def close(self):
        if getattr(self, "h", None):
            lib().cg_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, dt=0.0):
        _check(lib().cg_batch_step(self.h, float(dt)), "cg_batch_step")

    def step_each(self, dt=0.0):
        """cg_step of every instance in turn (the one-by-one reference)."""
        _check(lib().cg_batch_step_each(self.h, float(dt)), "cg_batch_step_each")

    def step_one(self, i, dt=0.0):
        """cg_step of instance i alone, on its own grids handle (same buffers)."""
        it = self._items[i]
        g = lib().cg_batch_instance(self.h, i)
        if not g:
            raise IndexError(i)
        _check(lib().cg_step(C.c_void_p(g), C.byref(it.particles), it.u_fine, C.byref(it.out), float(dt)),
               "cg_step")

    def use_graph(self, on=True):
        _check(lib().cg_batch_use_graph(self.h, 1 if on else 0), "cg_batch_use_graph")

    def config(self):
        c = BatchConfig()
        _check(lib().cg_batch_get_config(self.h, C.byref(c)), "cg_batch_get_config")
        return c.as_dict()

    def set_config(self, **kw):
        c = BatchConfig()
        _check(lib().cg_batch_get_config(self.h, C.byref(c)), "cg_batch_get_config")
        for k, v in kw.items():
            setattr(c, k, int(v))
        _check(lib().cg_batch_set_config(self.h, C.byref(c)), "cg_batch_set_config")

    def tune(self, reps=5, cache_path=None):
        c = BatchConfig()
        ms = C.c_double()
        _check(lib().cg_batch_tune(self.h, int(reps), None if cache_path is None else str(cache_path).encode(),
                                   C.byref(c), C.byref(ms)), "cg_batch_tune")
        return c.as_dict(), ms.value

    def sync_status(self):
        flags = C.c_uint32()
        counts = (C.c_int64 * CG_NCOUNTS)()
        rc = lib().cg_batch_sync_status(self.h, C.byref(flags), counts)
        return rc, flags.value, list(counts)

    def launch_count(self):
        return int(lib().cg_batch_launch_count(self.h))

    def launches_per_step(self):
        return int(lib().cg_batch_launches_per_step(self.h))

    def instance_launch_count(self, i):
        return int(lib().cg_launch_count(C.c_void_p(lib().cg_batch_instance(self.h, i))))


def mlp_pack(p: dict):
    """Flatten a parameter dict (W1, b1, W2, b2, w3, b3) in the ABI order."""
    import numpy as np
    return np.concatenate([np.asarray(p[k], np.float64).reshape(-1) for k in ("W1", "b1", "W2", "b2", "w3", "b3")]
                          ).astype(np.float32)


def mlp_unpack(flat, hidden=64, k0=16):
    import numpy as np
    f = np.asarray(flat, np.float64)
    out, o = {}, 0
    for k, shape in (("W1", (k0, hidden)), ("b1", (hidden,)), ("W2", (hidden, hidden)), ("b2", (hidden,)),
                     ("w3", (hidden,)), ("b3", (1,))):
        sz = int(np.prod(shape))
        out[k] = f[o:o + sz].reshape(shape)
        o += sz
    return out


def status_string(code: int) -> str:
    return lib().cg_status_string(code).decode()


class Map:
    """Owner of a ``cg_map``: the volume-weighted maps between a bulk and a
    fine uniform grid that are not nested.  bulk, fine: (origin, extent, n);
    fields are [ncomp][cells] tensors on the device."""

    def __init__(self, bulk, fine, fp64=False, stream=None):
        import torch
        self.dtype = torch.float64 if fp64 else torch.float32
        self.n_bulk = int(bulk[2][0]) * int(bulk[2][1]) * int(bulk[2][2])
        self.n_fine = int(fine[2][0]) * int(fine[2][1]) * int(fine[2][2])
        gb, gf = BoxGrid(), BoxGrid()
        for g, (o, e, n) in ((gb, bulk), (gf, fine)):
            g.origin[:] = [float(v) for v in o]
            g.extent[:] = [float(v) for v in e]
            g.n[:] = [int(v) for v in n]
            g.prec = CG_FP64 if fp64 else CG_FP32
        h = C.c_void_p()
        _check(lib().cg_map_create(C.byref(gb), C.byref(gf), _stream_handle(stream), C.byref(h)), "cg_map_create")
        self.h = h

    def _fields(self, t, cells, name):
        if not t.is_cuda or t.dtype != self.dtype or not t.is_contiguous() or t.numel() % cells != 0:
            raise ValueError(f"{name}: contiguous CUDA {self.dtype} tensor of [ncomp][{cells}] expected")
        return t.numel() // cells

    def average(self, fine_in, bulk_out):
        nc = self._fields(fine_in, self.n_fine, "fine_in")
        if self._fields(bulk_out, self.n_bulk, "bulk_out") != nc:
            raise ValueError("component counts differ")
        _check(lib().cg_map_average(self.h, nc, _ptr(fine_in), _ptr(bulk_out)), "cg_map_average")

    def project(self, bulk_in, fine_out):
        nc = self._fields(bulk_in, self.n_bulk, "bulk_in")
        if self._fields(fine_out, self.n_fine, "fine_out") != nc:
            raise ValueError("component counts differ")
        _check(lib().cg_map_project(self.h, nc, _ptr(bulk_in), _ptr(fine_out)), "cg_map_project")

    def close(self):
        if getattr(self, "h", None):
            lib().cg_map_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
