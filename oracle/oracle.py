"""ctypes wrapper of the plain CPU oracle (``symphase_oracle.c``).

TEST INFRASTRUCTURE ONLY. The tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use it to check and time the CUDA library;
the library itself never imports it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "symphase_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

# op names -> the oracle's own op codes (the order of its enum)
_CODES = {"H": 0, "S": 1, "CX": 2, "X": 3, "Y": 4, "Z": 5, "M": 6, "MR": 7, "R": 8,
          "X_ERROR": 9, "Y_ERROR": 10, "Z_ERROR": 11, "DEPOLARIZE1": 12,
          "DEPOLARIZE2": 13, "DETECTOR": 14, "OBSERVABLE_INCLUDE": 15, "TICK": 16,
          "X_IF": 17, "Y_IF": 18, "Z_IF": 19}
CH_TYPES = ("X_ERROR", "Y_ERROR", "Z_ERROR", "DEPOLARIZE1", "DEPOLARIZE2", "RANDOM")
STATUS = {0: "ok", 1: "invalid argument", 2: "unsupported op", 3: "nondeterministic detector",
          4: "out of memory"}


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` with gcc."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        # a test may point the wrapper at a deliberately broken copy of the
        # oracle to check that the pins catch it
        lib = C.CDLL(os.environ.get("SYMPHASE_ORACLE_LIB") or build())
        P, I64, U64 = C.c_void_p, C.c_int64, C.c_uint64
        ptr = C.c_void_p
        lib.or_build.restype = P
        lib.or_build.argtypes = [I64, I64, ptr, ptr, ptr, ptr, I64]
        lib.or_free.argtypes = [P]
        lib.or_info.argtypes = [P, ptr]
        lib.or_rows.argtypes = [P, C.c_int32, ptr]
        lib.or_channels.argtypes = [P, ptr, ptr, ptr, ptr, ptr]
        lib.or_random_symbols.argtypes = [P, ptr]
        lib.or_tableau.argtypes = [P, ptr, ptr, ptr]
        lib.or_draw.argtypes = [P, U64, U64, ptr]
        lib.or_eval.argtypes = [P, ptr, ptr, ptr, ptr]
        lib.or_sample.argtypes = [P, U64, U64, I64, ptr, ptr, ptr]
        lib.or_sample_shots.argtypes = [P, U64, ptr, I64, ptr, ptr, ptr]
        lib.or_draw_grouped.argtypes = [P, U64, U64, ptr]
        lib.or_sample_grouped.argtypes = [P, U64, U64, I64, ptr, ptr, ptr]
        lib.or_expect.argtypes = [P, ptr, ptr, ptr]
        lib.or_expect_vjp.argtypes = [P, ptr, ptr, ptr]
        lib.or_philox.argtypes = [ptr, ptr, ptr]
        lib.or_threshold.restype = C.c_uint32
        lib.or_threshold.argtypes = [C.c_double]
        _lib = lib
        return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def circuit_arrays(circuit):
    """Flatten a ``workloads.Circuit`` into (code, offsets, targets, arg)."""
    code = np.array([_CODES[op.name] for op in circuit.ops], dtype=np.int32)
    lens = np.array([len(op.targets) for op in circuit.ops], dtype=np.int64)
    off = np.zeros(len(circuit.ops) + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    tg = np.array([t for op in circuit.ops for t in op.targets] or [0], dtype=np.int32)
    arg = np.array([op.arg for op in circuit.ops] or [0.0], dtype=np.float64)
    return code, off, tg, arg


def philox4x32_10(counter: Sequence[int], key: Sequence[int]) -> np.ndarray:
    lib = _load()
    ctr = np.array(counter, dtype=np.uint32)
    k = np.array(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.or_philox(_p(ctr), _p(k), _p(out))
    return out


def threshold(p: float) -> int:
    return int(_load().or_threshold(float(p)))


class OracleError(RuntimeError):
    pass


@dataclass
class Channels:
    type: np.ndarray   # index into CH_TYPES
    p: np.ndarray
    T: np.ndarray
    sym0: np.ndarray
    nsym: np.ndarray


class Program:
    """The oracle's result for one circuit: the affine forms of every
    measurement, detector and observable over the symbols."""

    def __init__(self, circuit, stop: Optional[int] = None, check: bool = True):
        lib = _load()
        self._lib = lib
        code, off, tg, arg = circuit_arrays(circuit)
        self._keep = (code, off, tg, arg)
        nops = len(circuit.ops)
        h = lib.or_build(circuit.num_qubits, nops, _p(code), _p(off), _p(tg), _p(arg),
                         nops if stop is None else int(stop))
        if not h:
            raise MemoryError("oracle build failed to allocate")
        self._h = h
        info = np.zeros(9, dtype=np.int64)
        lib.or_info(h, _p(info))
        (self.status, self.num_qubits, self.num_meas, self.num_det, self.num_obs,
         self.num_symbols, self.num_channels, self.pw, self.bad_row) = (int(v) for v in info)
        if check and self.status != 0:
            raise OracleError(f"oracle build: {STATUS.get(self.status, self.status)} (row {self.bad_row})")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.or_free(h)
            self._h = None

    # ------------------------------------------------------------ structure
    def rows(self, which: str) -> np.ndarray:
        """Bit rows (uint64, ``pw`` words each; bit 0 = the constant)."""
        idx = {"meas": 0, "det": 1, "obs": 2}[which]
        cnt = {"meas": self.num_meas, "det": self.num_det, "obs": self.num_obs}[which]
        out = np.zeros((cnt, self.pw), dtype=np.uint64)
        if cnt:
            self._lib.or_rows(self._h, idx, _p(out))
        return out

    def row_bits(self, which: str) -> np.ndarray:
        """Rows as a dense 0/1 matrix over symbols 0..num_symbols."""
        r = self.rows(which)
        bits = np.unpackbits(r.view(np.uint8), axis=1, bitorder="little")
        return bits[:, : self.num_symbols + 1]

    def channels(self) -> Channels:
        n = self.num_channels
        t = np.zeros(n, np.int32); p = np.zeros(n, np.float64); T = np.zeros(n, np.uint32)
        s0 = np.zeros(n, np.int64); ns = np.zeros(n, np.int32)
        if n:
            self._lib.or_channels(self._h, _p(t), _p(p), _p(T), _p(s0), _p(ns))
        return Channels(t, p, T, s0, ns)

    def random_symbols(self) -> np.ndarray:
        f = np.zeros(self.num_symbols + 1, np.uint8)
        self._lib.or_random_symbols(self._h, _p(f))
        return f.astype(bool)

    def tableau(self):
        """(x, z, phases) of rows 0..2n-1 (destabilizers, then stabilizers);
        phases as a 0/1 matrix over symbols 0..num_symbols."""
        n = self.num_qubits
        x = np.zeros((2 * n, n), np.uint8); z = np.zeros((2 * n, n), np.uint8)
        ph = np.zeros((2 * n, self.pw), np.uint64)
        self._lib.or_tableau(self._h, _p(x), _p(z), _p(ph))
        bits = np.unpackbits(ph.view(np.uint8), axis=1, bitorder="little")[:, : self.num_symbols + 1]
        return x, z, bits

    # ------------------------------------------------------------- sampling
    def _words(self):
        return (self.num_meas + 63) // 64, (self.num_det + 63) // 64, (self.num_obs + 63) // 64

    def draw(self, seed: int, shot: int) -> np.ndarray:
        b = np.zeros(self.pw, np.uint64)
        self._lib.or_draw(self._h, seed, shot, _p(b))
        return b

    def draw_bits(self, seed: int, shot: int) -> np.ndarray:
        b = self.draw(seed, shot)
        return np.unpackbits(b.view(np.uint8), bitorder="little")[: self.num_symbols + 1]

    def draw_grouped(self, seed: int, shot: int) -> np.ndarray:
        """b of one shot under the grouped draw (stream 2), packed."""
        b = np.zeros(self.pw, np.uint64)
        self._lib.or_draw_grouped(self._h, seed, shot, _p(b))
        return b

    def draw_grouped_bits(self, seed: int, shot: int) -> np.ndarray:
        b = self.draw_grouped(seed, shot)
        return np.unpackbits(b.view(np.uint8), bitorder="little")[: self.num_symbols + 1]

    def sample_grouped(self, seed: int, shot0: int, nshots: int):
        """Records of shots shot0.. under the grouped draw (stream 2)."""
        wm, wd, wo = self._words()
        m = np.zeros((nshots, max(wm, 1)), np.uint64)
        d = np.zeros((nshots, max(wd, 1)), np.uint64)
        o = np.zeros((nshots, max(wo, 1)), np.uint64)
        if nshots:
            self._lib.or_sample_grouped(self._h, seed, shot0, nshots, _p(m), _p(d), _p(o))
        return m[:, :wm], d[:, :wd], o[:, :wo]

    def evaluate(self, b_bits: np.ndarray):
        """Records for an explicit symbol assignment (b_bits[0] must be 1)."""
        b_bits = np.asarray(b_bits, dtype=np.uint8)
        pad = np.zeros(self.pw * 64, np.uint8)
        pad[: len(b_bits)] = b_bits
        b = np.packbits(pad, bitorder="little").view(np.uint64).copy()
        wm, wd, wo = self._words()
        m = np.zeros(max(wm, 1), np.uint64); d = np.zeros(max(wd, 1), np.uint64)
        o = np.zeros(max(wo, 1), np.uint64)
        self._lib.or_eval(self._h, _p(b), _p(m), _p(d), _p(o))
        return m[:wm], d[:wd], o[:wo]

    def sample(self, seed: int, shot0: int, nshots: int):
        """Shot-major packed records (meas, det, obs) of shots shot0..shot0+n-1."""
        wm, wd, wo = self._words()
        m = np.zeros((nshots, max(wm, 1)), np.uint64)
        d = np.zeros((nshots, max(wd, 1)), np.uint64)
        o = np.zeros((nshots, max(wo, 1)), np.uint64)
        if nshots:
            self._lib.or_sample(self._h, seed, shot0, nshots, _p(m), _p(d), _p(o))
        return m[:, :wm], d[:, :wd], o[:, :wo]

    def sample_parallel(self, seed: int, shot0: int, nshots: int, threads: Optional[int] = None,
                        piece: int = 256):
        """``sample`` split into contiguous pieces run on host threads (the C
        calls release the GIL); the records are the same as one call's."""
        import concurrent.futures as cf
        threads = threads or os.cpu_count() or 1
        wm, wd, wo = self._words()
        m = np.zeros((nshots, max(wm, 1)), np.uint64)
        d = np.zeros((nshots, max(wd, 1)), np.uint64)
        o = np.zeros((nshots, max(wo, 1)), np.uint64)

        def run(a):
            n = min(piece, nshots - a)
            self._lib.or_sample(self._h, seed, shot0 + a, n, _p(m[a:]), _p(d[a:]), _p(o[a:]))

        with cf.ThreadPoolExecutor(max_workers=threads) as ex:
            list(ex.map(run, range(0, nshots, piece)))
        return m[:, :wm], d[:, :wd], o[:, :wo]

    def sample_shots(self, seed: int, shots: Sequence[int]):
        shots = np.ascontiguousarray(np.asarray(shots, dtype=np.uint64))
        n = len(shots)
        wm, wd, wo = self._words()
        m = np.zeros((n, max(wm, 1)), np.uint64)
        d = np.zeros((n, max(wd, 1)), np.uint64)
        o = np.zeros((n, max(wo, 1)), np.uint64)
        if n:
            self._lib.or_sample_shots(self._h, seed, _p(shots), n, _p(m), _p(d), _p(o))
        return m[:, :wm], d[:, :wd], o[:, :wo]

    # ---------------------------------------------------------- expectation
    def expect(self, p: Optional[np.ndarray] = None):
        """(log|E_j|, sign_j) for detectors then observables, FP64."""
        p = self.channels().p if p is None else np.ascontiguousarray(p, dtype=np.float64)
        n = self.num_det + self.num_obs
        la = np.zeros(n, np.float64); sg = np.zeros(n, np.int8)
        self._lib.or_expect(self._h, _p(p), _p(la), _p(sg))
        return la, sg

    def expect_vjp(self, p: np.ndarray, g: np.ndarray) -> np.ndarray:
        p = np.ascontiguousarray(p, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        out = np.zeros(self.num_channels, np.float64)
        self._lib.or_expect_vjp(self._h, _p(p), _p(g), _p(out))
        return out


def unpack_records(words: np.ndarray, count: int) -> np.ndarray:
    """Shot-major packed uint64 records -> 0/1 matrix [shots, count]."""
    words = np.ascontiguousarray(words, dtype=np.uint64)
    bits = np.unpackbits(words.view(np.uint8).reshape(words.shape[0], -1), axis=1, bitorder="little")
    return bits[:, :count]
