"""ctypes binding of libtcbf.so (include/tcbf.h), same names as the C ABI.

Argument marshalling only: every step of the beamforming path runs in the
library's CUDA kernels.  Tensors are passed as raw device pointers with
``tensor.data_ptr()`` and the stream as ``torch.cuda.current_stream()``'s
handle; torch provides device memory and streams, nothing else.  There is
no fallback: if the library or a GPU is missing, calls raise.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libtcbf.so")

TCBF_OK = 0
STATUS_NAMES = {0: "TCBF_OK", 1: "TCBF_ERR_INVALID_ARG", 2: "TCBF_ERR_UNSUPPORTED",
                3: "TCBF_ERR_OOM", 4: "TCBF_ERR_BUDGET", 5: "TCBF_ERR_CUDA",
                6: "TCBF_ERR_TIMEOUT", 7: "TCBF_ERR_DEVICE"}
MODE_FP16, MODE_FP8SPLIT, MODE_1BIT, MODE_TF32 = 0, 1, 2, 3
SRC_CF16, SRC_CF32 = 0, 1
FLAG_STACKED_X = 1
FLAG_FP8_HI_ONLY = 2
FLAG_FP8_FOUR_PRODUCTS = 4
FLAG_INTERLEAVED_X = 8
FLAG_FP8_BLOCK_SCALES = 16
FLAG_AUTO_LAYOUT = 32

# every symbol include/tcbf.h declares
EXPORTED = [
    "tcbf_plan_create", "tcbf_plan_destroy", "tcbf_packed_size", "tcbf_workspace_size",
    "tcbf_transpose_pack", "tcbf_beamform_fp16", "tcbf_beamform_fp8split",
    "tcbf_beamform_1bit", "tcbf_weights_from_geometry", "tcbf_last_device_error",
    "tcbf_status_string", "tcbf_plan_num_configs", "tcbf_plan_get_config",
    "tcbf_plan_set_config", "tcbf_config_name", "tcbf_beamform_fp16_noalloc",
    "tcbf_plan_set_batch_rows", "tcbf_autotune", "tcbf_graph_capture", "tcbf_graph_launch",
    "tcbf_beamform_host", "tcbf_debug_drop_fill", "tcbf_unpack_bits", "tcbf_beamform_tf32",
    "tcbf_expand_1bit", "tcbf_beamform_1bit_expanded", "tcbf_transpose_pack_expanded",
    "tcbf_plan_flags", "tcbf_autotune_layout",
]


class TcbfError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}")


class Problem(ctypes.Structure):
    _fields_ = [("batch", ctypes.c_int64), ("M", ctypes.c_int64), ("N", ctypes.c_int64),
                ("K", ctypes.c_int64), ("w_batches", ctypes.c_int64),
                ("mode", ctypes.c_int32), ("flags", ctypes.c_uint32)]


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libtcbf.so (build it first with paper_2505_03269_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libtcbf.so is not built ({path}); run "
                           "python -c 'import __graft_entry__ as g; g.build()'")
    lib = ctypes.CDLL(path)
    vp, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint32
    sig = {
        "tcbf_plan_create": [ctypes.POINTER(vp), ctypes.POINTER(Problem), i32],
        "tcbf_plan_destroy": [vp],
        "tcbf_packed_size": [vp, i32, ctypes.POINTER(ctypes.c_size_t)],
        "tcbf_workspace_size": [vp, ctypes.POINTER(ctypes.c_size_t)],
        "tcbf_transpose_pack": [vp, i32, i32, vp, vp, vp],
        "tcbf_beamform_fp16": [vp, vp, vp, vp, vp],
        "tcbf_beamform_fp8split": [vp, vp, vp, vp, vp],
        "tcbf_beamform_1bit": [vp, vp, vp, vp, vp],
        "tcbf_expand_1bit": [vp, i32, vp, vp],
        "tcbf_beamform_1bit_expanded": [vp, vp, vp],
        "tcbf_transpose_pack_expanded": [vp, i32, i32, vp, vp],
        "tcbf_weights_from_geometry": [vp, vp, vp, i32, vp, ctypes.c_double, vp, vp],
        "tcbf_last_device_error": [vp],
        "tcbf_debug_drop_fill": [vp, ctypes.c_int64],
        "tcbf_unpack_bits": [vp, i32, vp, vp, i32, vp],
        "tcbf_beamform_tf32": [vp, vp, vp, vp, vp],
        "tcbf_plan_num_configs": [vp, ctypes.POINTER(i32)],
        "tcbf_plan_get_config": [vp, ctypes.POINTER(i32)],
        "tcbf_plan_flags": [vp, ctypes.POINTER(u32)],
        "tcbf_autotune_layout": [vp, vp, vp, i32, vp, i32, vp, ctypes.POINTER(u32), vp],
        "tcbf_plan_set_config": [vp, i32],
        "tcbf_beamform_fp16_noalloc": [ctypes.POINTER(Problem), i32, vp, vp, i32, vp, i32, vp],
        "tcbf_plan_set_batch_rows": [vp, vp],
        "tcbf_autotune": [vp, vp, vp, vp, i32, vp, ctypes.POINTER(i32), vp],
        "tcbf_graph_capture": [vp, vp, i32, vp, vp, vp],
        "tcbf_graph_launch": [vp, vp],
        "tcbf_beamform_host": [vp, vp, i32, vp, vp, i64, vp],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.tcbf_status_string.argtypes = [ctypes.c_int]
    lib.tcbf_status_string.restype = ctypes.c_char_p
    lib.tcbf_config_name.argtypes = [vp, ctypes.c_int]
    lib.tcbf_config_name.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(status: int, where: str):
    if status != TCBF_OK:
        raise TcbfError(status, where)


def _ptr(t):
    """Raw pointer of a torch tensor / int / None."""
    if t is None:
        return None
    if isinstance(t, int):
        return ctypes.c_void_p(t)
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class Plan:
    """A tcbf plan: one problem shape, mode and device."""

    def __init__(self, batch, M, N, K, mode=MODE_FP16, w_batches=0, device=0, flags=0):
        lib = load()
        self._lib = lib
        self.problem = Problem(batch, M, N, K, w_batches, mode, flags)
        h = ctypes.c_void_p()
        _check(lib.tcbf_plan_create(ctypes.byref(h), ctypes.byref(self.problem), device),
               "tcbf_plan_create")
        self.handle = h
        self.batch, self.M, self.N, self.K = batch, M, N, K
        self.w_batches = w_batches or batch
        self.mode = mode
        self.device = device
        # the plan's own flags: TCBF_FLAG_AUTO_LAYOUT resolved to a layout
        f = ctypes.c_uint32()
        _check(lib.tcbf_plan_flags(h, ctypes.byref(f)), "tcbf_plan_flags")
        self.flags = f.value

    def close(self):
        if getattr(self, "handle", None):
            self._lib.tcbf_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # --------------------------------------------------------------- sizes
    def packed_size(self, which: int) -> int:
        n = ctypes.c_size_t()
        _check(self._lib.tcbf_packed_size(self.handle, which, ctypes.byref(n)), "tcbf_packed_size")
        return n.value

    @property
    def Kp(self):
        return (self.K + 63) // 64 * 64

    @property
    def Kw(self):
        return (self.K + 127) // 128 * 4

    # ------------------------------------------------------------- kernels
    def transpose_pack(self, which, src, dst, src_type=SRC_CF16, stream=None):
        _check(self._lib.tcbf_transpose_pack(self.handle, which, src_type, _ptr(src), _ptr(dst),
                                             _stream(stream)), "tcbf_transpose_pack")

    def beamform_tf32(self, Wp, Xp, Y, stream=None):
        _check(self._lib.tcbf_beamform_tf32(self.handle, _ptr(Wp), _ptr(Xp), _ptr(Y),
                                            _stream(stream)), "tcbf_beamform_tf32")

    def unpack_bits(self, which, src, dst, dst_type=SRC_CF16, stream=None):
        """Packed 1-bit planes back to interleaved complex +-1 values (the
        inverse of transpose_pack on a 1-bit plan)."""
        _check(self._lib.tcbf_unpack_bits(self.handle, int(which), _ptr(src), _ptr(dst),
                                          int(dst_type), _stream(stream)), "tcbf_unpack_bits")

    def beamform_fp16(self, Wp, Xp, Y, stream=None):
        _check(self._lib.tcbf_beamform_fp16(self.handle, _ptr(Wp), _ptr(Xp), _ptr(Y),
                                            _stream(stream)), "tcbf_beamform_fp16")

    def beamform_fp8split(self, Wp, Xp, Y, stream=None):
        _check(self._lib.tcbf_beamform_fp8split(self.handle, _ptr(Wp), _ptr(Xp), _ptr(Y),
                                                _stream(stream)), "tcbf_beamform_fp8split")

    def beamform_1bit(self, Wb, Xb, Y, stream=None):
        _check(self._lib.tcbf_beamform_1bit(self.handle, _ptr(Wb), _ptr(Xb), _ptr(Y),
                                            _stream(stream)), "tcbf_beamform_1bit")

    def expand_1bit(self, which, bits, stream=None):
        """4-bit tensor path: expand packed bits of W (0) or X (1) into the
        plan's E2M1 planes."""
        _check(self._lib.tcbf_expand_1bit(self.handle, int(which), _ptr(bits), _stream(stream)),
               "tcbf_expand_1bit")

    def transpose_pack_expanded(self, which, src, src_type=SRC_CF16, stream=None):
        """4-bit tensor path: sign-quantise interleaved complex W (0) or X (1)
        straight into the plan's E2M1 planes (no packed bits)."""
        _check(self._lib.tcbf_transpose_pack_expanded(self.handle, int(which), int(src_type),
                                                      _ptr(src), _stream(stream)),
               "tcbf_transpose_pack_expanded")

    def beamform_1bit_expanded(self, Y, stream=None):
        """4-bit tensor path: the GEMM on the planes last expanded."""
        _check(self._lib.tcbf_beamform_1bit_expanded(self.handle, _ptr(Y), _stream(stream)),
               "tcbf_beamform_1bit_expanded")

    def weights_from_geometry(self, rx_pos, targets, near_field, freqs, c, Wp, stream=None):
        _check(self._lib.tcbf_weights_from_geometry(
            self.handle, _ptr(rx_pos), _ptr(targets), int(near_field), _ptr(freqs), float(c),
            _ptr(Wp), _stream(stream)), "tcbf_weights_from_geometry")

    def last_device_error(self) -> int:
        return self._lib.tcbf_last_device_error(self.handle)

    def debug_drop_fill(self, fill: int):
        """Test hook of the device failure path: the next beamform call leaves
        out operand load `fill` of the first CTA, so its bounded waits run out
        (TCBF_ERR_TIMEOUT from last_device_error).  fill < 0 clears it."""
        _check(self._lib.tcbf_debug_drop_fill(self.handle, int(fill)), "debug_drop_fill")

    # ------------------------------------------------------------- configs
    def num_configs(self) -> int:
        n = ctypes.c_int()
        _check(self._lib.tcbf_plan_num_configs(self.handle, ctypes.byref(n)), "num_configs")
        return n.value

    def get_config(self) -> int:
        n = ctypes.c_int()
        _check(self._lib.tcbf_plan_get_config(self.handle, ctypes.byref(n)), "get_config")
        return n.value

    def set_config(self, c: int):
        _check(self._lib.tcbf_plan_set_config(self.handle, int(c)), "set_config")

    def config_name(self, c: int) -> str:
        return self._lib.tcbf_config_name(self.handle, int(c)).decode()

    # ------------------------------------------- uneven batches, tuning, graphs
    def set_batch_rows(self, rows):
        """Per-batch beam counts (host sequence of ints), or None for uniform."""
        if rows is None:
            _check(self._lib.tcbf_plan_set_batch_rows(self.handle, None), "set_batch_rows")
            return
        arr = (ctypes.c_int64 * len(rows))(*[int(r) for r in rows])
        _check(self._lib.tcbf_plan_set_batch_rows(self.handle, ctypes.cast(arr, ctypes.c_void_p)),
               "set_batch_rows")

    def autotune(self, Wp, Xp, Y, reps=3, stream=None):
        """Time every valid configuration; the fastest stays set.  Returns
        (best, [ms per configuration, -1 where not valid])."""
        n = self.num_configs()
        ms = (ctypes.c_float * n)()
        best = ctypes.c_int()
        _check(self._lib.tcbf_autotune(self.handle, _ptr(Wp), _ptr(Xp), _ptr(Y), int(reps),
                                       _stream(stream), ctypes.byref(best),
                                       ctypes.cast(ms, ctypes.c_void_p)), "tcbf_autotune")
        return best.value, list(ms)

    def autotune_layout(self, Wp, X_src, Y, src_type=SRC_CF16, reps=3, stream=None):
        """tcbf_autotune_layout (plans made with FLAG_AUTO_LAYOUT): the fastest
        of the planar, stacked and interleaved layouts, by the timed pack +
        beamform step, with its best configuration.  Returns (flags,
        [planar_ms, stacked_ms, interleaved_ms]) (-1 for a layout not timed)
        and updates self.flags; packed X must be remade when it changed."""
        f = ctypes.c_uint32()
        ms = (ctypes.c_float * 3)()
        _check(self._lib.tcbf_autotune_layout(self.handle, _ptr(Wp), _ptr(X_src), int(src_type),
                                              _ptr(Y), int(reps), _stream(stream), ctypes.byref(f),
                                              ms), "tcbf_autotune_layout")
        self.flags = f.value
        return f.value, [ms[0], ms[1], ms[2]]

    def graph_capture(self, Xsrc, Xp, Wp, Y, src_type=SRC_CF16):
        _check(self._lib.tcbf_graph_capture(self.handle, _ptr(Xsrc), int(src_type), _ptr(Xp),
                                            _ptr(Wp), _ptr(Y)), "tcbf_graph_capture")

    def graph_launch(self, stream=None):
        _check(self._lib.tcbf_graph_launch(self.handle, _stream(stream)), "tcbf_graph_launch")

    # ------------------------------------------------------- host-resident data
    def beamform_host(self, X_host, Wp, Y_host, chunk=0, src_type=SRC_CF16, stream=None):
        """tcbf_beamform_host: X_host and Y_host are CPU tensors (pinned for
        overlap), Wp the packed weights on the device; stream-ordered."""
        _check(self._lib.tcbf_beamform_host(self.handle, _ptr(X_host), int(src_type), _ptr(Wp),
                                            _ptr(Y_host), int(chunk), _stream(stream)),
               "tcbf_beamform_host")


def beamform_fp16_noalloc(batch, M, N, K, Wp, X, Y, w_batches=0, device=0,
                          src_type=SRC_CF16, check=True, stream=None) -> int:
    """tcbf_beamform_fp16_noalloc: no plan, no packed-sample buffer, no
    device allocation; returns the raw status code."""
    lib = load()
    prob = Problem(batch, M, N, K, w_batches, MODE_FP16, 0)
    return lib.tcbf_beamform_fp16_noalloc(ctypes.byref(prob), device, _ptr(Wp), _ptr(X),
                                          src_type, _ptr(Y), int(bool(check)), _stream(stream))


def status_string(s: int) -> str:
    return load().tcbf_status_string(int(s)).decode()
