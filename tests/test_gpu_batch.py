"""Batched sampling (sp_sample_batch): many circuits of uneven size, shot
count and noise rate in one graph-captured enqueue of persistent kernels,
one per autotuned launch shape. Records must be bit-identical to one
sp_sample call per circuit (and to the oracle on sampled shots), also when
the captured graph is replayed with new seeds and new output buffers, and
after a member's configuration or scratch changed between two calls."""
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


def _check_members(progs, seeds, shots, outs):
    for p, s, n, o in zip(progs, seeds, shots, outs):
        want = p.sample(n, seed=s)
        torch.cuda.synchronize()
        for a, b in zip(o, want):
            assert torch.equal(a, b), "batch differs from sp_sample"


def test_plan_is_reused_for_new_seeds_and_outputs():
    """Seeds and output pointers are per-call data: 100 seed sets on new
    buffers replay one plan, and the cache stays within its bound when the
    shot counts change."""
    specs = _suite()[:4]
    progs = [sp.build(c) for c, _, _ in specs]
    shots = [n for _, _, n in specs]
    before, cap = sp.batch_plans()
    for k in range(100):
        seeds = [1000 * k + i for i in range(len(progs))]
        outs = sp.sample_batch(progs, seeds, shots)
        if k in (0, 57, 99):
            torch.cuda.synchronize()
            _check_members(progs, seeds, shots, outs)
    assert sp.batch_plans()[0] <= before + 1
    for k in range(3 * cap):
        sp.sample_batch(progs, [7] * len(progs), [n + 32 * k for n in shots])
    assert sp.batch_plans()[0] <= cap
    outs = sp.sample_batch(progs, [3, 4, 5, 6], shots)
    torch.cuda.synchronize()
    _check_members(progs, [3, 4, 5, 6], shots, outs)


def test_batch_after_member_scratch_and_config_change():
    """batch -> set_chunk and a larger sp_sample on a staged member (its
    scratch is reallocated) -> the same batch with new seeds: the records
    still equal separate calls and the oracle. Then a fused member is moved
    to other tile shapes and the staged one back to the fused path."""
    specs = _suite()[:5]
    progs = [sp.build(c) for c, _, _ in specs]
    progs[1].set_path(sp.PATH_SPARSE)
    shots = [n for _, _, n in specs]
    outs = sp.sample_batch(progs, [1, 2, 3, 4, 5], shots)
    torch.cuda.synchronize()
    _check_members(progs, [1, 2, 3, 4, 5], shots, outs)
    progs[1].set_chunk(65536)
    progs[1].sample(50_000, seed=9)       # the staged scratch is reallocated, larger
    progs[1].set_chunk(0)
    seeds = [11, 12, 13, 14, 15]
    outs = sp.sample_batch(progs, seeds, shots)
    torch.cuda.synchronize()
    _check_members(progs, seeds, shots, outs)
    for (c, _, n), s, (m, d, o) in zip(specs, seeds, outs):
        ref = oracle.Program(c)
        pick = np.unique(np.array([0, 1, n // 3, n - 1]))
        rm, rd, ro = ref.sample_shots(s, pick)
        idx = torch.as_tensor(pick, device="cuda")
        np.testing.assert_array_equal(_u64(m[idx]), rm)
        np.testing.assert_array_equal(_u64(d[idx]), rd)
        np.testing.assert_array_equal(_u64(o[idx]), ro)
    progs[1].set_path(sp.PATH_AUTO)
    progs[2].set_fused_config(128, 1)
    progs[3].set_fused_config(32, 1)
    progs[4].set_fused_config(64, 3)
    outs = sp.sample_batch(progs, seeds, shots)
    torch.cuda.synchronize()
    _check_members(progs, seeds, shots, outs)


def test_every_launch_shape_in_one_batch():
    """Members with every fused launch shape (32-, 64- and 128-shot tiles,
    each variant) in one call: one persistent launch per shape."""
    shapes = [(32, 1), (32, 2), (64, 1), (64, 2), (64, 3), (128, 1), (128, 2)]
    progs, seeds, shots = [], [], []
    for k, (tile, var) in enumerate(shapes):
        p = sp.build(surface_code(3 + 2 * (k % 3), 3, 2e-3))
        p.set_fused_config(tile, var)
        progs.append(p)
        seeds.append(40 + k)
        shots.append(1000 + 333 * k)
    outs = sp.sample_batch(progs, seeds, shots)
    torch.cuda.synchronize()
    _check_members(progs, seeds, shots, outs)


def test_same_program_twice_in_one_batch():
    """One program listed twice with different seeds (and a third entry of
    another program): each member's records equal its own sp_sample call.
    The repeated program's members share one launch-constant buffer, so
    they draw without it. With these shot counts the repeated program's
    members run as their own kernel nodes and the other one inside the
    persistent batch kernel; three calls with new seeds and new output
    buffers replay one plan."""
    a = sp.build(surface_code(7, 7, 1e-3))
    b = sp.build(surface_code(5, 5, 2e-3))
    progs, shots = [a, b, a], [50_000, 9_000, 40_000]
    before = sp.batch_plans()[0]
    for rep in range(3):
        seeds = [11 + 10 * rep, 12 + 10 * rep, 13 + 10 * rep]
        outs = sp.sample_batch(progs, seeds, shots)
        torch.cuda.synchronize()
        _check_members(progs, seeds, shots, outs)
    assert sp.batch_plans()[0] <= before + 1


def test_large_members_as_kernel_nodes_against_oracle():
    """Members with at least a full wave of tiles run as separate kernel
    nodes on parallel branches of the plan's graph (with their own launch
    constants); records equal sp_sample and the oracle on sampled shots,
    over two calls with new seeds."""
    specs = [surface_code(9, 9, 1e-3), surface_code(11, 11, 5e-4), repetition_code(5, 5, 0.01),
             surface_code(3, 3, 2e-3)]
    progs = [sp.build(c) for c in specs]
    shots = [120_000, 100_003, 150_000, 70_000]
    for rep in range(2):
        seeds = [100 * rep + k for k in range(len(progs))]
        outs = sp.sample_batch(progs, seeds, shots)
        torch.cuda.synchronize()
        _check_members(progs, seeds, shots, outs)
    for c, s, n, (m, d, o) in zip(specs, seeds, shots, outs):
        ref = oracle.Program(c)
        pick = np.array([0, n // 3, n - 1])
        rm, rd, ro = ref.sample_shots(s, pick)
        idx = torch.as_tensor(pick, device="cuda")
        np.testing.assert_array_equal(_u64(m[idx]), rm)
        np.testing.assert_array_equal(_u64(d[idx]), rd)
        np.testing.assert_array_equal(_u64(o[idx]), ro)
