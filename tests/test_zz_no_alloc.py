"""sp_sample_static -- the sampling entry point that allocates nothing.

It is meant for callers that cannot call cudaMalloc (their GPU memory is
owned by another allocator, or an allocation's implicit synchronisation is
not acceptable on their path). It must give exactly the records of
sp_sample, also when called twice in a row on the same fixed scratch array,
and in a fresh process where its first call performs the per-device
set-up. Records are integer data, so the comparison is bit for bit."""
import numpy as np
import pytest

from workloads import repetition_code, surface_code

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2311_03906_gb300 as sp  # noqa: E402


@pytest.mark.parametrize("circuit,shots", [
    (surface_code(11, 11, 1e-3), 30_000),   # several chunks of the fixed scratch
    (repetition_code(5, 5, 0.01), 10_000),  # one chunk
])
def test_static_scratch_matches_sp_sample_twice(circuit, shots):
    prog = sp.build(circuit)
    for call, (seed, shot0) in enumerate([(11, 0), (12, 123_457)]):
        want = prog.sample(shots, seed=seed, shot0=shot0)
        got = prog.alloc_outputs(shots)
        for t in got:
            t.fill_(-1)  # stale contents must be overwritten
        prog.sample_static(shots, seed=seed, shot0=shot0, out=got)
        torch.cuda.synchronize()
        for name, a, b in zip(("meas", "det", "obs"), got, want):
            assert torch.equal(a, b), f"call {call}: {name} records differ from sp_sample"
    prog.close()


def test_static_scratch_rejects_misaligned_output():
    prog = sp.build(repetition_code(3, 2, 0.1))
    buf = torch.zeros(1000, dtype=torch.uint8, device="cuda")
    lib = sp.load()
    import ctypes as C
    st = lib.sp_sample_static(prog.handle, 1, 0, 10, C.c_void_p(buf.data_ptr() + 1), None, None, None)
    assert st == 1
    assert b"aligned" in lib.sp_last_error()


def test_static_scratch_rejects_a_program_of_another_device():
    """The scratch and the program's tables must be on one GPU: a program
    whose device field names another ordinal is refused before any launch
    (the field is forged here, since one GPU is all this test has)."""
    import ctypes as C
    prog = sp.build(repetition_code(3, 2, 0.1))
    lib = sp.load()
    dev = C.cast(prog.handle, C.POINTER(C.c_int))   # sp_program's first field: its device
    saved = dev[0]
    out = prog.alloc_outputs(10)
    try:
        dev[0] = saved + 7
        st = lib.sp_sample_static(prog.handle, 1, 0, 10, C.c_void_p(out[0].data_ptr()), None, None, None)
    finally:
        dev[0] = saved
    assert st == 1
    assert b"device" in lib.sp_last_error()
    prog.close()
