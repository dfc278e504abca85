"""ctypes binding of libamr_transfer.so (the C ABI in include/amr_transfer.h).

Argument marshalling only: every step of the transfer runs in the library's
CUDA kernels.  Importing this module does not load the library; the first
call that needs it does, and raises if the library has not been built (there
is no CPU fallback).
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libamr_transfer.so")

ABI_VERSION = 1
PREC_FP64, PREC_SPLIT, PREC_FIXED = 0, 1, 2
SCHEME_FD, SCHEME_LS = 0, 1
FLAG_CSR = 1
ORDER_DLINEAR, ORDER_TAYLOR2, ORDER_TAYLOR3 = 1, 2, 3
STATUS = {0: "ok", 1: "invalid argument", 2: "unsupported", 3: "out of memory", 4: "CUDA error",
          5: "timeout", 6: "internal error"}


class AmrError(RuntimeError):
    def __init__(self, status, where, detail=""):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}" + (f" ({detail})" if detail else ""))


class Item(ctypes.Structure):
    _fields_ = [("face", ctypes.c_int32), ("subface", ctypes.c_int32), ("patch_size", ctypes.c_int32),
                ("overlap", ctypes.c_int32), ("order", ctypes.c_int32), ("scheme", ctypes.c_int32),
                ("coarse_offset", ctypes.c_int64), ("fine_offset", ctypes.c_int64)]


class Desc(ctypes.Structure):
    _fields_ = [("abi_version", ctypes.c_int32), ("num_unknowns", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("flags", ctypes.c_int32), ("num_items", ctypes.c_int64),
                ("items", ctypes.c_void_p), ("coarse_elems", ctypes.c_int64), ("fine_elems", ctypes.c_int64)]


def diagonal_elems(items, num_unknowns):
    """float64 values of the diagonal-halo buffer: per item, per fine face
    array, k ghost layers of (p + 2k)^2 volumes of U unknowns."""
    total = 0
    for it in items:
        p, k = int(it["patch_size"]), int(it["overlap"])
        total += (9 if int(it["subface"]) < 0 else 1) * k * (p + 2 * k) ** 2 * int(num_unknowns)
    return total


class PlanInfo(ctypes.Structure):
    _fields_ = [("num_items", ctypes.c_int64), ("interp_outputs", ctypes.c_int64),
                ("restrict_outputs", ctypes.c_int64), ("interp_bytes", ctypes.c_int64),
                ("restrict_bytes", ctypes.c_int64), ("interp_launches", ctypes.c_int32),
                ("restrict_launches", ctypes.c_int32), ("increment_elems", ctypes.c_int64)]


class Tuning(ctypes.Structure):
    _fields_ = [("interp_threads", ctypes.c_int32), ("interp_smem_budget", ctypes.c_int32),
                ("restrict_threads", ctypes.c_int32), ("interp_addback", ctypes.c_int32),
                ("interp_lanes", ctypes.c_int32)]


ENTRY_POINTS = {
    "amr_transfer_plan_create": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "amr_transfer_plan_interpolate": ([ctypes.c_void_p] * 4, ctypes.c_int),
    "amr_transfer_plan_restrict": ([ctypes.c_void_p] * 4, ctypes.c_int),
    "amr_transfer_plan_interpolate_adjoint": ([ctypes.c_void_p] * 4, ctypes.c_int),
    "amr_transfer_plan_restrict_adjoint": ([ctypes.c_void_p] * 4, ctypes.c_int),
    "amr_transfer_plan_get_info": ([ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "amr_transfer_plan_interpolate_increments": ([ctypes.c_void_p] * 4, ctypes.c_int),
    "amr_transfer_plan_apply_increments": ([ctypes.c_void_p] * 5, ctypes.c_int),
    "amr_transfer_plan_interpolate_diagonal": ([ctypes.c_void_p] * 3 + [ctypes.c_int64, ctypes.c_void_p], ctypes.c_int),
    "amr_transfer_plan_get_tuning": ([ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "amr_transfer_plan_set_tuning": ([ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "amr_transfer_plan_autotune": ([ctypes.c_void_p] * 6, ctypes.c_int),
    "amr_transfer_plan_capture_step": ([ctypes.c_void_p] * 4, ctypes.c_int),
    "amr_transfer_plan_launch_step": ([ctypes.c_void_p] * 2, ctypes.c_int),
    "amr_transfer_plan_destroy": ([ctypes.c_void_p], ctypes.c_int),
    "amr_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "amr_last_cuda_error": ([], ctypes.c_char_p),
}

_lib = None


def lib():
    """The loaded library (loads it on first use; raises if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2504_15814_gb300.build_lib")
        handle = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in ENTRY_POINTS.items():
            fn = getattr(handle, name)
            fn.argtypes = args
            fn.restype = res
        _lib = handle
    return _lib


def _check(status, where):
    if status != 0:
        raise AmrError(status, where, lib().amr_last_cuda_error().decode(errors="replace"))


def _items_array(items):
    """Contiguous ctypes array of Item from a numpy structured array or a sequence of mappings."""
    n = len(items)
    arr = (Item * max(n, 1))()
    for i in range(n):
        it = items[i]
        try:
            scheme = int(it["scheme"])
        except (KeyError, ValueError, IndexError):
            scheme = 0
        arr[i] = Item(int(it["face"]), int(it["subface"]), int(it["patch_size"]), int(it["overlap"]),
                      int(it["order"]), scheme, int(it["coarse_offset"]), int(it["fine_offset"]))
    return arr, n


def _ptr(x):
    """Pointer of a contiguous float64 torch tensor in device memory or in
    pinned host memory (which the kernels read and write in place over the
    host link), or a raw int."""
    if isinstance(x, int) or x is None:
        return x
    import torch
    if not (isinstance(x, torch.Tensor) and (x.is_cuda or x.is_pinned()) and x.dtype == torch.float64
            and x.is_contiguous()):
        raise TypeError("buffers must be contiguous float64 tensors on the GPU or in pinned host memory")
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Plan:
    """A transfer plan over a fixed item list (amr_transfer_plan_create)."""

    def __init__(self, items, num_unknowns, coarse_elems, fine_elems, precision=PREC_FP64, flags=0):
        self._handle = None
        arr, n = _items_array(items)
        desc = Desc(ABI_VERSION, int(num_unknowns), int(precision), int(flags), n,
                    ctypes.cast(arr, ctypes.c_void_p), int(coarse_elems), int(fine_elems))
        h = ctypes.c_void_p()
        _check(lib().amr_transfer_plan_create(ctypes.byref(desc), ctypes.byref(h)), "amr_transfer_plan_create")
        self._handle = h
        import torch
        self.device = torch.cuda.current_device()  # the plan's tables live on this device
        self.num_unknowns = int(num_unknowns)
        self.coarse_elems = int(coarse_elems)
        self.fine_elems = int(fine_elems)
        self.precision = int(precision)
        self.diagonal_elems = diagonal_elems(items, num_unknowns)

    def _sized(self, x, n, name):
        if not isinstance(x, int) and x is not None:
            if x.numel() < n:
                raise ValueError(f"{name} holds {x.numel()} elements, the plan needs {n}")
            if x.is_cuda and x.device.index != self.device:
                raise ValueError(f"{name} is on cuda:{x.device.index}, the plan on cuda:{self.device}")
        return _ptr(x)

    def interpolate(self, coarse, fine, stream=None):
        _check(lib().amr_transfer_plan_interpolate(self._handle, self._sized(coarse, self.coarse_elems, "coarse"),
                                                   self._sized(fine, self.fine_elems, "fine"), _stream(stream)),
               "interpolate")
        return fine

    def restrict(self, fine, coarse, stream=None):
        _check(lib().amr_transfer_plan_restrict(self._handle, self._sized(fine, self.fine_elems, "fine"),
                                                self._sized(coarse, self.coarse_elems, "coarse"), _stream(stream)),
               "restrict")
        return coarse

    def _fptr(self, x, n, name):
        """Device pointer of a contiguous float32 CUDA tensor holding >= n values."""
        if isinstance(x, int):
            return x
        import torch
        if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float32 and x.is_contiguous()):
            raise TypeError(f"{name} must be a contiguous float32 CUDA tensor")
        if x.numel() < n:
            raise ValueError(f"{name} holds {x.numel()} elements, the plan needs {n}")
        return x.data_ptr()

    def interpolate_increments(self, coarse, increments, stream=None):
        """float32 increments (fine ghost value - nearest coarse centre value)."""
        _check(lib().amr_transfer_plan_interpolate_increments(
            self._handle, self._sized(coarse, self.coarse_elems, "coarse"),
            self._fptr(increments, self.info["increment_elems"], "increments"), _stream(stream)),
            "interpolate_increments")
        return increments

    def apply_increments(self, coarse, increments, fine, stream=None):
        _check(lib().amr_transfer_plan_apply_increments(
            self._handle, self._sized(coarse, self.coarse_elems, "coarse"),
            self._fptr(increments, self.info["increment_elems"], "increments"),
            self._sized(fine, self.fine_elems, "fine"), _stream(stream)), "apply_increments")
        return fine

    def interpolate_diagonal(self, coarse, diag, stream=None):
        """Widened ghost boxes of every subface (edge and vertex halos), float64;
        layout in amr_transfer_plan_interpolate_diagonal."""
        _check(lib().amr_transfer_plan_interpolate_diagonal(
            self._handle, self._sized(coarse, self.coarse_elems, "coarse"),
            self._sized(diag, self.diagonal_elems, "diag"), self.diagonal_elems, _stream(stream)),
            "interpolate_diagonal")
        return diag

    def interpolate_adjoint(self, g_fine, g_coarse, stream=None):
        _check(lib().amr_transfer_plan_interpolate_adjoint(
            self._handle, self._sized(g_fine, self.fine_elems, "g_fine"),
            self._sized(g_coarse, self.coarse_elems, "g_coarse"), _stream(stream)), "interpolate_adjoint")
        return g_coarse

    def restrict_adjoint(self, g_coarse, g_fine, stream=None):
        _check(lib().amr_transfer_plan_restrict_adjoint(
            self._handle, self._sized(g_coarse, self.coarse_elems, "g_coarse"),
            self._sized(g_fine, self.fine_elems, "g_fine"), _stream(stream)), "restrict_adjoint")
        return g_fine

    @property
    def tuning(self):
        out = Tuning()
        _check(lib().amr_transfer_plan_get_tuning(self._handle, ctypes.byref(out)), "get_tuning")
        return {name: getattr(out, name) for name, _ in Tuning._fields_}

    def set_tuning(self, interp_threads, interp_smem_budget, restrict_threads, interp_addback=2, interp_lanes=0):
        t = Tuning(int(interp_threads), int(interp_smem_budget), int(restrict_threads), int(interp_addback),
                   int(interp_lanes))
        _check(lib().amr_transfer_plan_set_tuning(self._handle, ctypes.byref(t)), "set_tuning")

    def autotune(self, coarse, fine, coarse_out, stream=None):
        """Time candidate launch shapes on these buffers and keep the fastest
        (overwrites fine's ghost halves and coarse_out's restricted volumes)."""
        out = Tuning()
        _check(lib().amr_transfer_plan_autotune(self._handle, self._sized(coarse, self.coarse_elems, "coarse"),
                                                self._sized(fine, self.fine_elems, "fine"),
                                                self._sized(coarse_out, self.coarse_elems, "coarse_out"),
                                                _stream(stream), ctypes.byref(out)), "autotune")
        return {name: getattr(out, name) for name, _ in Tuning._fields_}

    def capture_step(self, coarse, fine, coarse_out):
        """Capture interpolate(coarse -> fine) + restrict(fine -> coarse_out) as a CUDA graph."""
        _check(lib().amr_transfer_plan_capture_step(self._handle, self._sized(coarse, self.coarse_elems, "coarse"),
                                                    self._sized(fine, self.fine_elems, "fine"),
                                                    self._sized(coarse_out, self.coarse_elems, "coarse_out")),
               "capture_step")

    def launch_step(self, stream=None):
        _check(lib().amr_transfer_plan_launch_step(self._handle, _stream(stream)), "launch_step")

    @property
    def info(self):
        out = PlanInfo()
        _check(lib().amr_transfer_plan_get_info(self._handle, ctypes.byref(out)), "get_info")
        return {name: getattr(out, name) for name, _ in PlanInfo._fields_}

    def close(self):
        if self._handle is not None and _lib is not None:
            _lib.amr_transfer_plan_destroy(self._handle)
        self._handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
