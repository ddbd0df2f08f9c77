"""Saved programs (sp_save / sp_load): a program restored from its blob has
the same coefficient rows, channel table and sampler program as the one
that was built, and samples the same records for every seed (and the
oracle's on sampled shots). A corrupted blob is refused; an allocation
failure while loading leaves nothing behind."""
import numpy as np
import pytest

import oracle
from workloads import (mirror_circuit, random_feedforward_circuit, random_layered, repetition_code,
                       surface_code, surface_code_all_channels)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2311_03906_gb300 as sp  # noqa: E402

CASES = {
    "surface-d5": lambda: surface_code(5, 5, 1e-3),
    "all-channels-d3": lambda: surface_code_all_channels(3, 3, 2e-2),
    "repetition": lambda: repetition_code(5, 5, 0.01),
    "feed-forward": lambda: random_feedforward_circuit(12, 300, seed=5, p_noise=0.2),
    "random-layered-60": lambda: random_layered(60, 60, depolarize=0.01, seed=2),
    "mirror-dense": lambda: mirror_circuit(128, 6, p=0.02, seed=3),
}

INFO_KEYS = ("num_qubits", "num_measurements", "num_detectors", "num_observables", "num_symbols",
             "num_channels", "num_random", "nnz_rows", "nnz_delta", "log_words", "density")


def _u64(t):
    return t.cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("name", sorted(CASES))
def test_round_trip_is_exact(name):
    c = CASES[name]()
    a = sp.build(c)
    blob = a.save()
    b = sp.load_program(blob)
    for k in INFO_KEYS:
        assert a.info[k] == b.info[k], k
    for which in ("meas", "det", "obs"):
        np.testing.assert_array_equal(a.rows(which), b.rows(which))
    for x, y in zip(a.channels(), b.channels()):
        np.testing.assert_array_equal(x, y)
    # the restored program writes the same blob
    assert b.save() == blob
    # same records on every path either program takes, for two seeds
    for seed in (1, 2**40 + 7):
        ra, rb = a.sample(3000, seed=seed), b.sample(3000, seed=seed)
        torch.cuda.synchronize()
        for x, y in zip(ra, rb):
            assert torch.equal(x, y)
    b.set_path(sp.PATH_SPARSE)
    a.set_path(sp.PATH_SPARSE)
    ra, rb = a.sample(1000, seed=9), b.sample(1000, seed=9)
    torch.cuda.synchronize()
    for x, y in zip(ra, rb):
        assert torch.equal(x, y)
    # and the oracle's records on sampled shots
    ref = oracle.Program(c)
    pick = np.array([0, 517, 999])
    m, d, o = rb
    rm, rd, ro = ref.sample_shots(9, pick)
    idx = torch.as_tensor(pick, device="cuda")
    np.testing.assert_array_equal(_u64(m[idx]), rm)
    np.testing.assert_array_equal(_u64(d[idx]), rd)
    np.testing.assert_array_equal(_u64(o[idx]), ro)
    # expectations
    if b.num_detectors + b.num_observables:
        ea, eb = a.expect_raw(), b.expect_raw()
        torch.cuda.synchronize()
        assert torch.equal(ea, eb)


def test_file_round_trip_and_rejections(tmp_path):
    a = sp.build(surface_code(3, 3, 1e-3))
    path = tmp_path / "d3.symphase"
    blob = a.save(str(path))
    b = sp.load_program(str(path))
    ra, rb = a.sample(2048, seed=4), b.sample(2048, seed=4)
    torch.cuda.synchronize()
    for x, y in zip(ra, rb):
        assert torch.equal(x, y)
    dev0, host0 = sp.debug_live_allocs()
    bad = bytearray(blob)
    bad[len(bad) // 2] ^= 0x10
    for broken in (bytes(bad), blob[:-8], b"SYMPHASE" + blob[8:16]):
        with pytest.raises(sp.SymPhaseError) as e:
            sp.load_program(broken)
        assert e.value.status == 1
    assert sp.debug_live_allocs() == (dev0, host0)


def test_allocation_failure_while_loading_leaks_nothing():
    blob = sp.build(surface_code(3, 3, 1e-3)).save()
    import gc
    gc.collect()
    gc.disable()
    try:
        dev0, host0 = sp.debug_live_allocs()
        for k in (0, 3, 9):
            sp.debug_fail_alloc(k)
            with pytest.raises(sp.SymPhaseError) as e:
                sp.load_program(blob)
            assert e.value.status == 4
            assert sp.debug_live_allocs() == (dev0, host0)
        sp.debug_fail_alloc(-1)
        p = sp.load_program(blob)
        p.close()
        assert sp.debug_live_allocs() == (dev0, host0)
    finally:
        sp.debug_fail_alloc(-1)
        gc.enable()
