"""Thin ctypes binding of libsymphase (include/symphase.h).

Argument marshalling only: every step of building and sampling runs in the
library's CUDA kernels. PyTorch provides device memory and streams. The
library must have been built (``paper_2311_03906_gb300._build.build()`` or
``__graft_entry__.build()``); importing this module on a machine where it is
missing raises ImportError rather than falling back to anything."""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence, Tuple

import numpy as np

from . import _build

SP_OK = 0
STATUS_NAMES = {0: "SP_OK", 1: "SP_ERR_INVALID_ARG", 2: "SP_ERR_UNSUPPORTED_OP",
                3: "SP_ERR_NONDETERMINISTIC_DETECTOR", 4: "SP_ERR_OOM", 5: "SP_ERR_CUDA",
                6: "SP_ERR_TIMEOUT", 7: "SP_ERR_TOO_LARGE"}
OPCODES = {"H": 0, "S": 1, "CX": 2, "X": 3, "Y": 4, "Z": 5, "M": 6, "MR": 7, "R": 8,
           "X_ERROR": 9, "Y_ERROR": 10, "Z_ERROR": 11, "DEPOLARIZE1": 12, "DEPOLARIZE2": 13,
           "DETECTOR": 14, "OBSERVABLE_INCLUDE": 15, "TICK": 16, "X_IF": 17, "Y_IF": 18, "Z_IF": 19}
PATH_AUTO, PATH_SPARSE, PATH_DENSE, PATH_FUSED, PATH_TENSOR = 0, 1, 2, 3, 4

# every entry point declared in include/symphase.h
EXPORTS = ("sp_build", "sp_save", "sp_load", "sp_info", "sp_sample", "sp_sample_host", "sp_sample_static",
           "sp_sample_batch", "sp_expect", "sp_expect_sign",
           "sp_expect_grad", "sp_export_rows", "sp_export_channels", "sp_set_path", "sp_set_fused_config",
           "sp_set_chunk", "sp_set_stream", "sp_device_status", "sp_set_wait_limit",
           "sp_profile_enable", "sp_profile_read", "sp_batch_plans", "sp_debug_fail_alloc",
           "sp_debug_live_allocs", "sp_free", "sp_last_error")
KERNEL_CLASSES = ("draw", "product", "emit", "fused", "tensor", "consts")


class SymPhaseError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class sp_op(C.Structure):
    _fields_ = [("opcode", C.c_uint32), ("ntargets", C.c_uint32),
                ("targets", C.POINTER(C.c_uint32)), ("arg", C.c_double)]


class sp_circuit_desc(C.Structure):
    _fields_ = [("num_qubits", C.c_uint32), ("num_ops", C.c_uint32), ("ops", C.POINTER(sp_op))]


class sp_info_t(C.Structure):
    _fields_ = [("num_qubits", C.c_uint64), ("num_measurements", C.c_uint64),
                ("num_detectors", C.c_uint64), ("num_observables", C.c_uint64),
                ("num_symbols", C.c_uint64), ("num_channels", C.c_uint64),
                ("num_random", C.c_uint64), ("nnz_rows", C.c_uint64), ("nnz_delta", C.c_uint64),
                ("log_words", C.c_uint64), ("density", C.c_double), ("path", C.c_int32),
                ("fused_tile_shots", C.c_int32), ("fused_variant", C.c_int32),
                ("fused_ctas_per_sm", C.c_int32), ("autotune_launches", C.c_int32), ("stream", C.c_int32),
                ("chunk_shots", C.c_uint64), ("build_ms", C.c_double), ("path_probe_ms", C.c_double * 5),
                ("live_blocks", C.c_uint64)]


_lib = None


def lib_path() -> str:
    return _build.LIB


def load() -> C.CDLL:
    """Load the built library (raises ImportError if it was never built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise ImportError(f"libsymphase is not built ({path} missing); run __graft_entry__.build()")
    lib = C.CDLL(path)
    vp, u64, u32, i32 = C.c_void_p, C.c_uint64, C.c_uint32, C.c_int32
    lib.sp_build.argtypes = [C.POINTER(sp_circuit_desc), vp, C.POINTER(vp)]
    lib.sp_save.argtypes = [vp, vp, C.c_size_t, C.POINTER(C.c_size_t)]
    lib.sp_load.argtypes = [vp, C.c_size_t, vp, C.POINTER(vp)]
    lib.sp_info.argtypes = [vp, C.POINTER(sp_info_t)]
    lib.sp_sample.argtypes = [vp, u64, u64, u64, vp, vp, vp, vp]
    lib.sp_sample_host.argtypes = [vp, u64, u64, u64, vp, vp, vp, vp]
    lib.sp_sample_static.argtypes = [vp, u64, u64, u64, vp, vp, vp, vp]
    lib.sp_sample_batch.argtypes = [vp, u32, vp, vp, vp, vp, vp, vp]
    lib.sp_expect.argtypes = [vp, vp, vp, vp]
    lib.sp_expect_grad.argtypes = [vp, vp, vp, vp, vp]
    lib.sp_expect_sign.argtypes = [vp, vp, vp, vp]
    lib.sp_export_rows.argtypes = [vp, i32, vp, u64]
    lib.sp_export_channels.argtypes = [vp, vp, vp, vp]
    lib.sp_set_path.argtypes = [vp, i32]
    lib.sp_set_chunk.argtypes = [vp, u64]
    lib.sp_set_stream.argtypes = [vp, i32]
    lib.sp_device_status.argtypes = [vp, C.POINTER(C.c_int32)]
    lib.sp_set_wait_limit.argtypes = [vp, u64]
    lib.sp_set_fused_config.argtypes = [vp, i32, i32]
    lib.sp_profile_enable.argtypes = [vp, i32]
    lib.sp_profile_read.argtypes = [vp, vp, vp]
    lib.sp_batch_plans.argtypes = [vp, vp]
    lib.sp_debug_fail_alloc.argtypes = [C.c_int64]
    lib.sp_debug_live_allocs.argtypes = [vp, vp]
    lib.sp_free.argtypes = [vp]
    lib.sp_free.restype = None
    lib.sp_last_error.restype = C.c_char_p
    for name in EXPORTS:
        if name not in ("sp_free", "sp_last_error"):
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def _check(status: int) -> None:
    if status != SP_OK:
        msg = load().sp_last_error().decode(errors="replace")
        raise SymPhaseError(status, msg)


def _stream_handle(stream=None) -> int:
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return int(s.cuda_stream)


def _ptr(t) -> Optional[int]:
    return None if t is None else int(t.data_ptr())


def _circuit_struct(circuit):
    """Marshal a workloads.Circuit (or its text) into sp_circuit_desc."""
    if isinstance(circuit, str):
        from workloads import Circuit
        circuit = Circuit.from_text(circuit)
    keep = []
    ops = (sp_op * max(1, len(circuit.ops)))()
    p32 = C.POINTER(C.c_uint32)
    for i, op in enumerate(circuit.ops):
        arr = np.asarray(op.targets, dtype=np.uint32) if len(op.targets) else np.zeros(1, np.uint32)
        keep.append(arr)
        o = ops[i]
        o.opcode = OPCODES[op.name]
        o.ntargets = len(op.targets)
        o.targets = arr.ctypes.data_as(p32)
        o.arg = float(op.arg)
    desc = sp_circuit_desc(circuit.num_qubits, len(circuit.ops), C.cast(ops, C.POINTER(sp_op)))
    return desc, (ops, keep)


class Program:
    """A circuit built by ``sp_build`` on the current CUDA device."""

    def __init__(self, circuit=None, stream=None, saved: Optional[bytes] = None):
        import torch  # noqa: F401  (CUDA context through torch)
        lib = load()
        h = C.c_void_p()
        if saved is not None:
            buf = bytes(saved)
            _check(lib.sp_load(buf, len(buf), C.c_void_p(_stream_handle(stream)), C.byref(h)))
        else:
            desc, keep = _circuit_struct(circuit)
            _check(lib.sp_build(C.byref(desc), C.c_void_p(_stream_handle(stream)), C.byref(h)))
            del keep
        self._h = h
        self._lib = lib
        info = sp_info_t()
        _check(lib.sp_info(h, C.byref(info)))
        self.info = {f: (list(getattr(info, f)) if f == "path_probe_ms" else getattr(info, f))
                     for f, _ in sp_info_t._fields_}
        self.num_measurements = info.num_measurements
        self.num_detectors = info.num_detectors
        self.num_observables = info.num_observables
        self.num_symbols = info.num_symbols
        self.num_channels = info.num_channels

    @property
    def handle(self):
        return self._h

    def save(self, path: Optional[str] = None) -> bytes:
        """The program as sp_save's blob; also written to `path` if given."""
        size = C.c_size_t(0)
        _check(self._lib.sp_save(self._h, None, 0, C.byref(size)))
        buf = C.create_string_buffer(size.value)
        _check(self._lib.sp_save(self._h, buf, size.value, C.byref(size)))
        data = buf.raw[:size.value]
        if path is not None:
            with open(path, "wb") as f:
                f.write(data)
        return data

    def close(self):
        if getattr(self, "_h", None):
            self._lib.sp_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def refresh_info(self):
        info = sp_info_t()
        _check(self._lib.sp_info(self._h, C.byref(info)))
        self.info = {f: (list(getattr(info, f)) if f == "path_probe_ms" else getattr(info, f))
                     for f, _ in sp_info_t._fields_}
        return self.info

    # -------------------------------------------------------------- records
    def words(self) -> Tuple[int, int, int]:
        return ((self.num_measurements + 63) // 64, (self.num_detectors + 63) // 64,
                (self.num_observables + 63) // 64)

    def alloc_outputs(self, shots: int, device="cuda", pin_memory=False):
        import torch
        wm, wd, wo = self.words()
        kw = dict(dtype=torch.int64)
        if device == "cpu":
            kw["pin_memory"] = pin_memory
        else:
            kw["device"] = device
        return (torch.empty((shots, wm), **kw), torch.empty((shots, wd), **kw),
                torch.empty((shots, wo), **kw))

    def sample(self, shots: int, seed: int = 0, shot0: int = 0, out=None, stream=None,
               meas: bool = True, det: bool = True, obs: bool = True):
        """Records of shots shot0..shot0+shots-1 as int64 tensors on the GPU
        (bit-packed uint64 words, shot-major)."""
        m, d, o = out if out is not None else self.alloc_outputs(shots)
        _check(self._lib.sp_sample(self._h, seed, shot0, shots, _ptr(m) if meas else None,
                                   _ptr(d) if det else None, _ptr(o) if obs else None,
                                   C.c_void_p(_stream_handle(stream))))
        return m, d, o

    def sample_host(self, shots: int, seed: int = 0, shot0: int = 0, out=None, stream=None):
        """Records written straight into (pinned) host tensors."""
        m, d, o = out if out is not None else self.alloc_outputs(shots, device="cpu", pin_memory=True)
        _check(self._lib.sp_sample_host(self._h, seed, shot0, shots, _ptr(m), _ptr(d), _ptr(o),
                                        C.c_void_p(_stream_handle(stream))))
        return m, d, o

    def sample_static(self, shots: int, seed: int = 0, shot0: int = 0, out=None, stream=None):
        """Like sample(), but the library allocates nothing: it works in its
        fixed per-device scratch array (for callers that cannot allocate)."""
        m, d, o = out if out is not None else self.alloc_outputs(shots)
        _check(self._lib.sp_sample_static(self._h, seed, shot0, shots, _ptr(m), _ptr(d), _ptr(o),
                                          C.c_void_p(_stream_handle(stream))))
        return m, d, o

    def set_path(self, path: int):
        _check(self._lib.sp_set_path(self._h, path))
        self.refresh_info()

    def set_fused_config(self, tile_shots: int, variant: int = 1):
        _check(self._lib.sp_set_fused_config(self._h, tile_shots, variant))
        self.refresh_info()

    def set_stream(self, stream: int):
        """Fault-draw stream: 1 per-channel Philox (default), 2 grouped."""
        _check(self._lib.sp_set_stream(self._h, int(stream)))
        self.refresh_info()

    def set_chunk(self, chunk_shots: int):
        _check(self._lib.sp_set_chunk(self._h, chunk_shots))
        self.refresh_info()

    def device_status(self) -> int:
        """Waits for the device; 0 if every tensor-core tile since the last
        call completed, 1 if one gave up on a bounded wait (the library then
        also returns SP_ERR_TIMEOUT, which this method turns into the value)."""
        v = C.c_int32(0)
        st = self._lib.sp_device_status(self._h, C.byref(v))
        if st != 6:
            _check(st)
        return int(v.value)

    def set_wait_limit(self, ns: int):
        """Bound of the tensor-core kernel's stage waits (0 = default 2 s)."""
        _check(self._lib.sp_set_wait_limit(self._h, int(ns)))

    def profile(self, on: bool = True):
        _check(self._lib.sp_profile_enable(self._h, 1 if on else 0))

    def profile_read(self):
        """{kernel class: (milliseconds, launches)} since the last read."""
        ms = np.zeros(8, np.float64)
        n = np.zeros(8, np.uint64)
        _check(self._lib.sp_profile_read(self._h, ms.ctypes.data, n.ctypes.data))
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(KERNEL_CLASSES)}

    # ---------------------------------------------------------- expectation
    def expect_raw(self, p=None, out=None, stream=None):
        import torch
        n = self.num_detectors + self.num_observables
        out = torch.empty(n, dtype=torch.float32, device="cuda") if out is None else out
        _check(self._lib.sp_expect(self._h, _ptr(p), _ptr(out), C.c_void_p(_stream_handle(stream))))
        return out

    def expect_sign_raw(self, p=None, out=None, stream=None):
        """sign E_j (+1, -1, or 0 where E_j = 0) for detectors then observables."""
        import torch
        n = self.num_detectors + self.num_observables
        out = torch.empty(n, dtype=torch.float32, device="cuda") if out is None else out
        _check(self._lib.sp_expect_sign(self._h, _ptr(p), _ptr(out), C.c_void_p(_stream_handle(stream))))
        return out

    def expect_grad_raw(self, p, grad_logE, out=None, stream=None):
        import torch
        out = torch.empty(self.num_channels, dtype=torch.float32, device="cuda") if out is None else out
        _check(self._lib.sp_expect_grad(self._h, _ptr(p), _ptr(grad_logE), _ptr(out),
                                        C.c_void_p(_stream_handle(stream))))
        return out

    # -------------------------------------------------------------- exports
    def rows(self, which: str) -> np.ndarray:
        idx = {"meas": 0, "det": 1, "obs": 2}[which]
        cnt = {"meas": self.num_measurements, "det": self.num_detectors, "obs": self.num_observables}[which]
        rw = (self.num_symbols + 1 + 63) // 64
        out = np.zeros((max(cnt, 1), rw), dtype=np.uint64)
        _check(self._lib.sp_export_rows(self._h, idx, out.ctypes.data, rw))
        return out[:cnt]

    def channels(self):
        n = self.num_channels
        T = np.zeros(max(n, 1), np.uint32)
        kind = np.zeros(max(n, 1), np.uint8)
        s0 = np.zeros(max(n, 1), np.uint64)
        _check(self._lib.sp_export_channels(self._h, T.ctypes.data, kind.ctypes.data, s0.ctypes.data))
        return T[:n], kind[:n], s0[:n]


def build(circuit, stream=None) -> Program:
    return Program(circuit, stream=stream)


def load_program(saved, stream=None) -> Program:
    """Restore a program from sp_save's blob (bytes) or a file holding it."""
    if isinstance(saved, (str, os.PathLike)):
        with open(saved, "rb") as f:
            saved = f.read()
    return Program(saved=saved, stream=stream)


def sample_batch(progs: Sequence[Program], seeds: Sequence[int], shots: Sequence[int], outs=None,
                 stream=None):
    """Sample several programs in one call; returns [(meas, det, obs)]."""
    lib = load()
    n = len(progs)
    outs = outs if outs is not None else [p.alloc_outputs(s) for p, s in zip(progs, shots)]
    H = (C.c_void_p * n)(*[p.handle.value for p in progs])
    S = (C.c_uint64 * n)(*seeds)
    N = (C.c_uint64 * n)(*shots)
    M = (C.c_void_p * n)(*[_ptr(o[0]) for o in outs])
    D = (C.c_void_p * n)(*[_ptr(o[1]) for o in outs])
    O = (C.c_void_p * n)(*[_ptr(o[2]) for o in outs])
    _check(lib.sp_sample_batch(H, n, S, N, M, D, O, C.c_void_p(_stream_handle(stream))))
    return outs


def batch_plans() -> Tuple[int, int]:
    """(cached sp_sample_batch plans, cache capacity)."""
    lib = load()
    cnt, cap = C.c_uint32(0), C.c_uint32(0)
    _check(lib.sp_batch_plans(C.byref(cnt), C.byref(cap)))
    return int(cnt.value), int(cap.value)


def debug_fail_alloc(after: int) -> None:
    """Make the library's allocation number `after` (0 = the next) fail
    once; a negative value disarms the hook."""
    _check(load().sp_debug_fail_alloc(int(after)))


def debug_live_allocs() -> Tuple[int, int]:
    """(device allocations, programs) the library currently holds."""
    dev, host = C.c_int64(0), C.c_int64(0)
    _check(load().sp_debug_live_allocs(C.byref(dev), C.byref(host)))
    return int(dev.value), int(host.value)


def _expect_function():
    import torch

    class ExpectFunction(torch.autograd.Function):
        """log|E_j| of every detector/observable as a function of the
        per-channel probabilities; forward and backward are the library's
        FP32 kernels (sp_expect / sp_expect_grad)."""

        @staticmethod
        def forward(ctx, p, prog):
            p = p.contiguous()
            ctx.prog = prog
            ctx.save_for_backward(p)
            return prog.expect_raw(p)

        @staticmethod
        def backward(ctx, g):
            (p,) = ctx.saved_tensors
            return ctx.prog.expect_grad_raw(p, g.contiguous()), None

    return ExpectFunction


_EXPECT = None


def expect(prog: Program, p):
    """Differentiable log|E| (detectors then observables) at probabilities p
    (FP32 CUDA tensor, one per channel)."""
    global _EXPECT
    if _EXPECT is None:
        _EXPECT = _expect_function()
    return _EXPECT.apply(p, prog)


def unpack_bits(words, count: int) -> np.ndarray:
    """int64/uint64 packed records (tensor or array) -> 0/1 uint8 [shots, count]."""
    if hasattr(words, "cpu"):
        words = words.cpu().numpy()
    words = np.ascontiguousarray(words).view(np.uint64)
    bits = np.unpackbits(words.view(np.uint8).reshape(words.shape[0], -1), axis=1, bitorder="little")
    return bits[:, :count]
