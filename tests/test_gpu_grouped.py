"""The grouped fault draw (stream 2, sp_set_stream(prog, 2)) on the GPU
against the oracle's definition of the same stream: records bit for bit on
circuits with every channel kind, random outcomes, feed-forward and noise
up to p = 0.05; ragged shot counts and offsets, shots across 2^32, every
fused launch shape, the d=11 configuration at full size on sampled shots;
and detector rates within 5 sigma of the analytic expectation."""
import numpy as np
import pytest

import oracle
from workloads import (random_feedforward_circuit, random_layered, random_small_circuit, repetition_code,
                       surface_code, surface_code_all_channels)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2311_03906_gb300 as sp  # noqa: E402

CIRCUITS = {
    "rep5": lambda: repetition_code(5, 5, 0.01),
    "surf3": lambda: surface_code(3, 3, 1e-2),
    "surf5": lambda: surface_code(5, 5, 2e-3),
    "allkinds": lambda: surface_code_all_channels(3, 3, 1e-3),
    "noisy5": lambda: surface_code(5, 5, 0.05),
    "layered40": lambda: random_layered(40, 40, depolarize=0.01, seed=3),
    "rand6": lambda: random_small_circuit(45, 240, seed=906),
    "ff4": lambda: random_feedforward_circuit(27, 220, seed=804),
}


def _u64(t):
    return t.cpu().numpy().view(np.uint64)


def _grouped(c):
    prog, ref = sp.build(c), oracle.Program(c)
    prog.set_stream(2)
    assert prog.info["stream"] == 2 and prog.info["path"] == sp.PATH_FUSED
    return prog, ref


@pytest.mark.parametrize("name", sorted(CIRCUITS))
@pytest.mark.parametrize("shot0,shots", [(0, 1), (5, 31), (64, 33), (1 << 33, 1061), (7, 4101)])
def test_records_match_oracle(name, shot0, shots):
    prog, ref = _grouped(CIRCUITS[name]())
    m, d, o = prog.sample(shots, seed=17, shot0=shot0)
    torch.cuda.synchronize()
    rm, rd, ro = ref.sample_grouped(17, shot0, shots)
    np.testing.assert_array_equal(_u64(m), rm)
    np.testing.assert_array_equal(_u64(d), rd)
    np.testing.assert_array_equal(_u64(o), ro)


@pytest.mark.parametrize("tile,variant", [(32, 1), (32, 2), (64, 1), (64, 2), (64, 3), (128, 1), (128, 2)])
@pytest.mark.parametrize("name", ["surf5", "noisy5", "rand6"])
def test_every_launch_shape(name, tile, variant):
    prog, ref = _grouped(CIRCUITS[name]())
    prog.set_fused_config(tile, variant)
    shot0 = (1 << 32) - 77      # tiles whose shots have two high counter words
    m, d, o = prog.sample(2113, seed=5, shot0=shot0)
    torch.cuda.synchronize()
    rm, rd, ro = ref.sample_grouped(5, shot0, 2113)
    np.testing.assert_array_equal(_u64(m), rm)
    np.testing.assert_array_equal(_u64(d), rd)
    np.testing.assert_array_equal(_u64(o), ro)


def test_streams_switch_back_and_forth():
    c = surface_code(3, 3, 2e-2)
    prog, ref = sp.build(c), oracle.Program(c)
    for stream in (1, 2, 1, 2):
        prog.set_stream(stream)
        m, d, _ = prog.sample(500, seed=3)
        torch.cuda.synchronize()
        rm, rd, _ = (ref.sample if stream == 1 else ref.sample_grouped)(3, 0, 500)
        np.testing.assert_array_equal(_u64(d), rd)
    with pytest.raises(sp.SymPhaseError):
        prog.set_path(sp.PATH_SPARSE)       # the grouped draw runs on the fused path only
    with pytest.raises(sp.SymPhaseError):
        prog.sample_static(100, seed=1)     # the static-scratch entry point draws stream 1


def test_batch_with_a_grouped_member():
    specs = [(surface_code(3, 3, 2e-3), 1, 1000), (surface_code(5, 5, 1e-3), 2, 777), (repetition_code(5, 5, 0.01), 3, 64)]
    progs = [sp.build(c) for c, _, _ in specs]
    progs[1].set_stream(2)
    outs = sp.sample_batch(progs, [s for _, s, _ in specs], [n for _, _, n in specs])
    torch.cuda.synchronize()
    for (c, s, n), p, o in zip(specs, progs, outs):
        ref = oracle.Program(c)
        rm, rd, ro = (ref.sample_grouped if p.info["stream"] == 2 else ref.sample)(s, 0, n)
        np.testing.assert_array_equal(_u64(o[0]), rm)
        np.testing.assert_array_equal(_u64(o[1]), rd)


@pytest.fixture(scope="module")
def d11():
    c = surface_code(11, 11, 1e-3)
    prog, ref = _grouped(c)
    return c, prog, ref


def test_full_size_d11_sampled_shots(d11):
    c, prog, ref = d11
    shots = 1_000_000
    m, d, o = prog.sample(shots, seed=1, shot0=0)
    torch.cuda.synchronize()
    rng = np.random.default_rng(2)
    pick = np.unique(np.concatenate([rng.integers(0, shots, 124), [0, 63, 64, shots - 1]]))
    rows_m, rows_d, rows_o = [], [], []
    for t in pick:
        a, b, e = ref.sample_grouped(1, int(t), 1)
        rows_m.append(a[0]); rows_d.append(b[0]); rows_o.append(e[0])
    idx = torch.as_tensor(pick, device="cuda")
    np.testing.assert_array_equal(_u64(m[idx]), np.array(rows_m))
    np.testing.assert_array_equal(_u64(d[idx]), np.array(rows_d))
    np.testing.assert_array_equal(_u64(o[idx]), np.array(rows_o))


def test_full_size_d11_detector_rates(d11):
    """Monte-Carlo detector rates of 1e6 grouped-stream shots against the
    analytic expectation, within 5 sigma."""
    c, prog, ref = d11
    shots = 1_000_000
    _, d, _ = prog.sample(shots, seed=2, shot0=0, meas=False, obs=False)
    dd = d.view(torch.int64)
    bits = torch.stack([((dd[:, j // 64] >> (j % 64)) & 1).sum() for j in range(prog.num_detectors)]).double()
    rates = (bits / shots).cpu().numpy()
    la = prog.expect_raw().cpu().numpy()[: prog.num_detectors].astype(np.float64)
    r = (1 - np.exp(la)) / 2
    z = np.abs(rates - r) / np.sqrt(r * (1 - r) / shots)
    assert z.max() < 5.0, z.max()
