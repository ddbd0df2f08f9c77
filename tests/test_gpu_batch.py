"""Batched sampling (sp_sample_batch): many circuits of uneven size, shot
count and noise rate in one graph-captured enqueue of persistent kernels.
Records must be bit-identical to one sp_sample call per circuit (and to the
oracle on sampled shots), also when the captured graph is replayed."""
import numpy as np
import pytest

import oracle
from workloads import batch_suite, repetition_code, surface_code

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2311_03906_gb300 as sp  # noqa: E402


def _u64(t):
    return t.cpu().numpy().view(np.uint64)


def _suite():
    # uneven: tiny to d=15; the test sends one of them through the staged kernels
    specs = [(repetition_code(5, 5, 0.01), 1, 1000), (surface_code(3, 3, 2e-3), 2, 4097),
             (surface_code(5, 5, 1e-3), 3, 777), (surface_code(7, 7, 5e-4), 4, 3001),
             (surface_code(9, 9, 2e-3), 5, 2048), (surface_code(15, 15, 1e-3), 6, 1500),
             (surface_code(3, 3, 5e-4), 7, 31)]
    return specs


def test_batch_matches_separate_calls_and_replay():
    specs = _suite()
    progs = [sp.build(c) for c, _, _ in specs]
    assert progs[5].info["path"] == sp.PATH_FUSED
    progs[2].set_path(sp.PATH_SPARSE)   # one circuit through the staged kernels
    seeds = [s for _, s, _ in specs]
    shots = [n for _, _, n in specs]
    outs = [p.alloc_outputs(n) for p, n in zip(progs, shots)]
    for rep in range(2):
        for o in outs:
            for t in o:
                t.fill_(-1)
        sp.sample_batch(progs, seeds, shots, outs=outs)
        torch.cuda.synchronize()
        for p, s, n, o in zip(progs, seeds, shots, outs):
            want = p.sample(n, seed=s)
            torch.cuda.synchronize()
            for a, b in zip(o, want):
                assert torch.equal(a, b), f"replay {rep}: batch differs from sp_sample"


def test_batch_against_oracle_on_sampled_shots():
    specs = _suite()[:5]
    progs = [sp.build(c) for c, _, _ in specs]
    outs = sp.sample_batch(progs, [s for _, s, _ in specs], [n for _, _, n in specs])
    torch.cuda.synchronize()
    for (c, s, n), (m, d, o) in zip(specs, outs):
        ref = oracle.Program(c)
        pick = np.unique(np.array([0, n // 2, n - 1]))
        rm, rd, ro = ref.sample_shots(s, pick)
        idx = torch.as_tensor(pick, device="cuda")
        np.testing.assert_array_equal(_u64(m[idx]), rm)
        np.testing.assert_array_equal(_u64(d[idx]), rd)
        np.testing.assert_array_equal(_u64(o[idx]), ro)


def test_batch_plan_dropped_when_a_program_is_freed():
    c = surface_code(3, 3, 1e-3)
    p1, p2 = sp.build(c), sp.build(c)
    outs = sp.sample_batch([p1, p2], [1, 2], [500, 600])
    p1.close()
    p3 = sp.build(surface_code(5, 5, 1e-3))
    outs2 = sp.sample_batch([p3, p2], [1, 2], [500, 600])
    torch.cuda.synchronize()
    want = p3.sample(500, seed=1)
    torch.cuda.synchronize()
    assert torch.equal(outs2[0][1], want[1])


def test_config4_suite_builds_and_samples_a_slice():
    """The 64-circuit suite (d in 3..15, p in {5e-4, 1e-3, 2e-3}, seeds 0..63)
    batched at 256 shots per circuit, checked against separate calls."""
    suite = batch_suite(64)
    progs = [sp.build(c) for c, _ in suite]
    seeds = [s for _, s in suite]
    outs = sp.sample_batch(progs, seeds, [256] * len(progs))
    torch.cuda.synchronize()
    for p, s, o in zip(progs[::9], seeds[::9], outs[::9]):
        want = p.sample(256, seed=s)
        torch.cuda.synchronize()
        for a, b in zip(o, want):
            assert torch.equal(a, b)
