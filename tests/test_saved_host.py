"""sp_load's host-side checks, without a GPU: a blob written here by hand
in the documented format (include/symphase.h, sp_save) for a two-
measurement circuit passes them, and each single corruption of it is
refused with SP_ERR_INVALID_ARG before any device call."""
import ctypes as C
import struct

import pytest

MAGIC = b"SYMPHASE"
LOOKBACK = 512


def _fnv1a(data: bytes) -> int:
    x = 0xcbf29ce484222325
    for b in data:
        x ^= b
        x = (x * 0x100000001b3) & 0xFFFFFFFFFFFFFFFF
    return x


def _pad8(b: bytes) -> bytes:
    return b + b"\0" * (-len(b) % 8)


def _threshold(p: float) -> int:
    t = int(p * 4294967296.0)   # floor for p >= 0
    return min(t, 4294967295) if p > 0 else 0


def _fields():
    """X_ERROR(0.1) on qubit 0, M 0, M 0, DETECTOR rec[-1] rec[-2]: one
    symbol; rows m0 = s1, m1 = s1 (parent m0, no own symbols), d0 = 0."""
    p = 0.1
    return {
        "n": 1, "n_meas": 2, "n_det": 1, "n_obs": 0, "n_sym": 1, "n_ch": 1, "log_len": 0,
        "nnz_rows": 2, "nnz_delta": 1,
        "chT": [_threshold(p)], "chKind": [0], "chP": [p], "chSym0": [1], "fault_p": [p],
        "xoff": [0, 2], "xrefs": [1, 0],
        "parent": [-1, 0, -1], "const": [0, 0, 0], "rowOff": [0, 1, 1, 1], "idx": [0],
    }


def _blob(f, *, magic=MAGIC, version=1, endian=0x01020304, header_bytes=128, lookback=LOOKBACK,
          payload_fix=None, checksum_fix=None):
    R = f["n_meas"] + f["n_det"] + f["n_obs"]
    secs = [struct.pack(f"<{len(f['chT'])}I", *f["chT"]),
            bytes(f["chKind"]),
            struct.pack(f"<{len(f['chP'])}f", *f["chP"]),
            struct.pack(f"<{len(f['chSym0'])}I", *f["chSym0"]),
            struct.pack(f"<{len(f['fault_p'])}d", *f["fault_p"]),
            struct.pack(f"<{len(f['xoff'])}I", *f["xoff"]),
            struct.pack(f"<{len(f['xrefs'])}I", *f["xrefs"]),
            struct.pack(f"<{R}i", *f["parent"]),
            bytes(f["const"]),
            struct.pack(f"<{R + 1}I", *f["rowOff"]),
            struct.pack(f"<{len(f['idx'])}I", *f["idx"])]
    payload = b"".join(_pad8(s) for s in secs)
    n_fault, n_xrefs = len(f["fault_p"]), len(f["xrefs"])
    plen = len(payload) if payload_fix is None else payload_fix
    ck = _fnv1a(payload) if checksum_fix is None else checksum_fix
    head = magic + struct.pack("<4I", version, endian, header_bytes, lookback) + struct.pack(
        "<13Q", f["n"], f["n_meas"], f["n_det"], f["n_obs"], f["n_sym"], f["n_ch"], f["log_len"],
        f["nnz_rows"], f["nnz_delta"], n_fault, n_xrefs, plen, ck)
    assert len(head) == 128
    return head + payload


@pytest.fixture(scope="module")
def lib():
    from paper_2311_03906_gb300 import _build
    _build.build()
    from paper_2311_03906_gb300 import binding
    return binding.load()


def _load(lib, data: bytes):
    h = C.c_void_p()
    st = lib.sp_load(data, len(data), None, C.byref(h))
    if st == 0:
        lib.sp_free(h)
    return st, lib.sp_last_error().decode()


def test_hand_written_blob_passes_the_host_checks(lib):
    st, msg = _load(lib, _blob(_fields()))
    # no GPU here: the load stops at its first device call (SP_ERR_CUDA); on
    # a machine with one it succeeds
    assert st in (0, 5), msg


def _mut(**kw):
    f = _fields()
    f.update(kw)
    return f


BAD = {
    "magic": lambda: _blob(_fields(), magic=b"SYMPHASF"),
    "version": lambda: _blob(_fields(), version=2),
    "byte order": lambda: _blob(_fields(), endian=0x04030201),
    "header size": lambda: _blob(_fields(), header_bytes=136),
    "parent bound": lambda: _blob(_fields(), lookback=256),
    "payload size": lambda: _blob(_fields(), payload_fix=8),
    "checksum": lambda: _blob(_fields(), checksum_fix=1),
    "truncated": lambda: _blob(_fields())[:-1],
    "trailing byte": lambda: _blob(_fields()) + b"\0",
    "too many qubits": lambda: _blob(_mut(n=1025)),
    "huge count": lambda: _blob(_mut(n_sym=1 << 31)),
    "unknown kind": lambda: _blob(_mut(chKind=[4])),
    "symbols out of order": lambda: _blob(_mut(chSym0=[2])),
    "symbols not covered": lambda: _blob(_mut(n_sym=2, idx=[1])),
    "threshold": lambda: _blob(_mut(chT=[_threshold(0.1) + 1])),
    "fp32 probability": lambda: _blob(_mut(chP=[0.2])),
    "probability range": lambda: _blob(_mut(fault_p=[1.5], chP=[1.5], chT=[4294967295])),
    "extra probability": lambda: _blob(_mut(fault_p=[0.1, 0.1])),
    "random outcome table": lambda: _blob(_mut(chKind=[3], fault_p=[])),
    "detector offsets": lambda: _blob(_mut(xoff=[0, 1])),
    "detector reference": lambda: _blob(_mut(xrefs=[2, 0])),
    "parent not earlier": lambda: _blob(_mut(parent=[-1, 1, -1])),
    "parent negative": lambda: _blob(_mut(parent=[-1, -2, -1])),
    "constant bit": lambda: _blob(_mut(const=[0, 2, 0])),
    "row offsets": lambda: _blob(_mut(rowOff=[0, 1, 1, 0])),
    "row offsets decrease": lambda: _blob(_mut(rowOff=[0, 1, 0, 1])),
    "symbol range": lambda: _blob(_mut(idx=[1])),
}


@pytest.mark.parametrize("name", sorted(BAD))
def test_corrupted_blob_is_refused_on_the_host(lib, name):
    st, msg = _load(lib, BAD[name]())
    assert st == 1, (name, st, msg)
    assert msg.startswith("saved program:"), msg


def test_parent_distance_is_bounded(lib):
    # 600 measurements of one symbol: row 599's parent 599 rows back is refused
    n_meas = 600
    f = _fields()
    f.update(n_meas=n_meas, n_det=0, xoff=[0], xrefs=[], nnz_rows=n_meas,
             parent=[-1] + [0] * (n_meas - 1), const=[0] * n_meas,
             rowOff=[0] + [1] * n_meas, idx=[0])
    st, msg = _load(lib, _blob(f))
    assert st == 1 and "parent" in msg, msg
    f["parent"] = [-1] + list(range(n_meas - 1))
    st, msg = _load(lib, _blob(f))
    assert st in (0, 5), msg


def test_null_and_size_queries(lib):
    h = C.c_void_p()
    assert lib.sp_load(None, 0, None, C.byref(h)) == 1
    assert lib.sp_load(b"x", 1, None, None) == 1
    size = C.c_size_t(0)
    assert lib.sp_save(None, None, 0, C.byref(size)) == 1
