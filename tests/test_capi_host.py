"""The C-ABI library without a GPU: it builds for sm_103a, loads, exports
every entry point include/symphase.h declares, and rejects bad arguments
on the host before touching CUDA."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2311_03906_gb300 import _build
    _build.build()
    from paper_2311_03906_gb300 import binding
    return binding.load()


def _declared():
    text = open(os.path.join(ROOT, "include", "symphase.h")).read()
    return sorted(set(re.findall(r"SP_API\s+[\w\s\*]*?\b(sp_\w+)\s*\(", text)))


def test_header_declares_entry_points():
    names = _declared()
    for n in ("sp_build", "sp_sample", "sp_expect", "sp_expect_grad", "sp_free", "sp_last_error"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2311_03906_gb300 import binding
    names = _declared()
    assert names, "no SP_API declarations found"
    for n in names:
        assert hasattr(lib, n), f"{n} declared in symphase.h but not exported"
    assert set(names) == set(binding.EXPORTS)


def _desc(binding, nq, ops):
    keep = []
    arr = (binding.sp_op * len(ops))()
    for i, (code, tg, arg) in enumerate(ops):
        t = (C.c_uint32 * max(1, len(tg)))(*tg)
        keep.append(t)
        arr[i].opcode, arr[i].ntargets = code, len(tg)
        arr[i].targets = C.cast(t, C.POINTER(C.c_uint32))
        arr[i].arg = arg
    return binding.sp_circuit_desc(nq, len(ops), C.cast(arr, C.POINTER(binding.sp_op))), (arr, keep)


@pytest.mark.parametrize("nq,ops,status", [
    (2, [(2, [0, 0], 0.0)], 1),              # CX on one qubit
    (2, [(0, [5], 0.0)], 1),                 # target out of range
    (2, [(9, [0], 1.5)], 1),                 # probability > 1
    (2, [(9, [0], -0.1)], 1),                # probability < 0
    (2, [(13, [0, 1, 1], 0.1)], 1),          # odd DEPOLARIZE2 targets
    (2, [(6, [0], 0.0), (14, [2], 0.0)], 1), # look-back beyond the records
    (2, [(42, [0], 0.0)], 2),                # unknown opcode
    (2000, [(0, [0], 0.0)], 7),              # too many qubits
    (2, [(13, [0, 0], 0.1)], 1),             # DEPOLARIZE2 on one qubit
    (2, [(6, [0], 0.0), (17, [1], 0.0)], 1),     # feed-forward needs (rec, qubit) pairs
    (2, [(6, [0], 0.0), (17, [2, 0], 0.0)], 1),  # feed-forward look-back beyond the records
    (2, [(6, [0], 0.0), (18, [1, 5], 0.0)], 1),  # feed-forward qubit out of range
    (2, [(19, [1, 0], 0.0)], 1),                 # feed-forward before any record
])
def test_build_rejects_on_host(lib, nq, ops, status):
    from paper_2311_03906_gb300 import binding
    desc, keep = _desc(binding, nq, ops)
    h = C.c_void_p()
    st = lib.sp_build(C.byref(desc), None, C.byref(h))
    assert st == status
    assert not h.value
    assert lib.sp_last_error()


def test_null_arguments(lib):
    h = C.c_void_p()
    assert lib.sp_build(None, None, C.byref(h)) == 1
    assert lib.sp_info(None, None) == 1
    assert lib.sp_sample(None, 0, 0, 10, None, None, None, None) == 1
    assert lib.sp_expect(None, None, None, None) == 1
    assert lib.sp_expect_grad(None, None, None, None, None) == 1
    assert lib.sp_export_rows(None, 0, None, 1) == 1
    assert lib.sp_set_chunk(None, 1024) == 1
    assert lib.sp_set_path(None, 0) == 1
    assert lib.sp_set_fused_config(None, 64, 1) == 1
    st = C.c_int32(7)
    assert lib.sp_device_status(None, C.byref(st)) == 1
    lib.sp_free(None)
    assert b"NULL" in lib.sp_last_error()


def test_failed_program_allocation_is_reported_without_a_leak(lib):
    """The allocation-failure hook on the host: sp_build's first allocation
    (the program object) fails before any CUDA call, so this runs without a
    GPU; the call returns SP_ERR_OOM and holds nothing afterwards."""
    from paper_2311_03906_gb300 import binding
    desc, keep = _desc(binding, 2, [(0, [0], 0.0), (6, [0, 1], 0.0)])
    dev0, host0 = C.c_int64(0), C.c_int64(0)
    assert lib.sp_debug_live_allocs(C.byref(dev0), C.byref(host0)) == 0
    assert lib.sp_debug_fail_alloc(0) == 0
    h = C.c_void_p()
    st = lib.sp_build(C.byref(desc), None, C.byref(h))
    assert st == 4 and not h.value
    assert b"allocation" in lib.sp_last_error()
    dev1, host1 = C.c_int64(0), C.c_int64(0)
    lib.sp_debug_live_allocs(C.byref(dev1), C.byref(host1))
    assert (dev1.value, host1.value) == (dev0.value, host0.value)
    # the hook fired once and disarmed itself: the next failure is the
    # missing GPU, not an injected one
    st = lib.sp_build(C.byref(desc), None, C.byref(h))
    assert st != 4


def test_batch_plan_cache_is_empty_and_bounded(lib):
    n, cap = C.c_uint32(7), C.c_uint32(0)
    assert lib.sp_batch_plans(C.byref(n), C.byref(cap)) == 0
    assert n.value == 0 and cap.value == 8


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes mirrors of sp_op, sp_circuit_desc and sp_info_t have the
    C header's size and field offsets (compiled with the host C compiler)."""
    import shutil
    import subprocess
    from paper_2311_03906_gb300 import binding
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    structs = {"sp_op": binding.sp_op, "sp_circuit_desc": binding.sp_circuit_desc, "sp_info_t": binding.sp_info_t}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "symphase.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "probe"
    r = subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            name, key, val = line.split()
            got[(name, key)] = int(val)
    for name, cls in structs.items():
        assert got[(name, "size")] == C.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)
