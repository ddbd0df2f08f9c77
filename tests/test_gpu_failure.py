"""Failure detection on the GPU without faulting it: the tensor-core
kernel's bounded waits are made to run out (a bound too short for any stage
to be ready), and allocations are made to fail through the library's host-
side hook. Each error must reach the caller as a status (SP_ERR_TIMEOUT,
SP_ERR_OOM), leak nothing, and leave the program usable: the next normal
call gives the oracle's records bit for bit."""
import numpy as np
import pytest

import oracle
from workloads import mirror_circuit, surface_code

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2311_03906_gb300 as sp  # noqa: E402

SP_ERR_OOM, SP_ERR_TIMEOUT = 4, 6


def _u64(t):
    return t.cpu().numpy().view(np.uint64)


def _same(prog, ref, shots, seed):
    m, d, o = prog.sample(shots, seed=seed)
    torch.cuda.synchronize()
    rm, rd, ro = ref.sample(seed, 0, shots)
    np.testing.assert_array_equal(_u64(m), rm)
    np.testing.assert_array_equal(_u64(d), rd)
    np.testing.assert_array_equal(_u64(o), ro)


def test_tensor_kernel_wait_bound_runs_out_and_recovers():
    c = mirror_circuit(128, 8, p=0.02, seed=2)
    prog, ref = sp.build(c), oracle.Program(c)
    prog.set_path(sp.PATH_TENSOR)
    assert prog.device_status() == 0
    # 1 ns: a stage's operands are never ready at the first check
    prog.set_wait_limit(1)
    prog.sample(4096, seed=3)
    lib = sp.load()
    import ctypes as C
    v = C.c_int32(0)
    assert lib.sp_device_status(prog.handle, C.byref(v)) == SP_ERR_TIMEOUT
    assert v.value == 1
    assert b"bounded wait" in lib.sp_last_error()
    # the status word was cleared by the read
    assert prog.device_status() == 0
    # the synchronous host-buffer entry point reports the same error itself
    with pytest.raises(sp.SymPhaseError) as e:
        prog.sample_host(4096, seed=3)
    assert e.value.status == SP_ERR_TIMEOUT
    # default bound again: every tile completes and the records are exact
    prog.set_wait_limit(0)
    _same(prog, ref, 4096, 3)
    assert prog.device_status() == 0


def test_every_build_allocation_can_fail_without_a_leak():
    """Fail allocation k of sp_build for k = 0, 1, ... until a build goes
    through: each failure is SP_ERR_OOM and releases everything it took."""
    import gc
    c = surface_code(3, 3, 1e-3)
    ref = oracle.Program(c)
    gc.collect()
    gc.disable()   # no program of another test may be released meanwhile
    base = sp.debug_live_allocs()
    failures = 0
    prog = None
    for k in range(500):
        sp.debug_fail_alloc(k)
        try:
            prog = sp.build(c)
        except sp.SymPhaseError as e:
            assert e.status == SP_ERR_OOM, (k, e)
            assert sp.debug_live_allocs() == base, f"allocation {k}: a failed build leaked"
            failures += 1
            continue
        finally:
            sp.debug_fail_alloc(-1)
        break
    gc.enable()
    assert prog is not None and failures >= 10
    _same(prog, ref, 1000, 7)


@pytest.mark.parametrize("call", ["staged", "host", "expect", "dense"])
def test_failed_allocation_in_a_call_leaves_the_program_usable(call):
    c = surface_code(5, 5, 2e-3) if call != "dense" else mirror_circuit(48, 4, p=0.02, seed=1)
    prog, ref = sp.build(c), oracle.Program(c)
    if call == "staged":
        prog.set_path(sp.PATH_SPARSE)
    if call == "dense":
        prog.set_path(sp.PATH_DENSE)
    shots = 40_000 if call == "dense" else 3000   # beyond the build probe's 32,768-shot buffers
    sp.debug_fail_alloc(0)
    try:
        with pytest.raises(sp.SymPhaseError) as e:
            if call in ("staged", "dense"):
                prog.sample(shots, seed=1)
            elif call == "host":
                prog.sample_host(3000, seed=1)
            else:
                prog.expect_raw()
        assert e.value.status == SP_ERR_OOM
    finally:
        sp.debug_fail_alloc(-1)
    torch.cuda.synchronize()
    _same(prog, ref, shots, 1)
    if call == "host":
        hm, hd, ho = prog.sample_host(3000, seed=1)
        rm, rd, _ = ref.sample(1, 0, 3000)
        np.testing.assert_array_equal(hm.numpy().view(np.uint64), rm)
    if call == "expect":
        la, _ = ref.expect(ref.channels().p.astype(np.float32).astype(np.float64))
        np.testing.assert_allclose(prog.expect_raw().cpu().numpy(), la, rtol=1e-4, atol=1e-6)
