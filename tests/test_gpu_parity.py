"""CUDA path vs the CPU oracle, through the C ABI.

Integer/bit work (coefficient rows, channel tables, records) must be
bit-exact. FP32 expectations: relative error <= 1e-4 on log|E| against the
FP64 oracle; gradients <= 1e-4 against the oracle's analytic adjoint and
<= 1e-3 against FP64 central differences (h = 1e-6)."""
import numpy as np
import pytest

import oracle
from workloads import (Circuit, random_clifford_circuit, random_feedforward_circuit, random_layered,
                       random_small_circuit, repetition_code, surface_code, surface_code_all_channels)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2311_03906_gb300 as sp  # noqa: E402


def _fig1():
    c = Circuit(4)
    c.append("H", [0]); c.append("CX", [0, 1, 1, 2, 2, 3])
    c.append("Z_ERROR", [0], 0.1); c.append("X_ERROR", [1, 2, 3], 0.1)
    c.append("CX", [2, 3, 1, 2, 0, 1]); c.append("H", [0]); c.append("M", [0, 1, 2, 3])
    return c


def _sec31():
    c = Circuit(2)
    c.append("H", [0]); c.append("CX", [0, 1]); c.append("X_ERROR", [0], 0.1)
    c.append("X_ERROR", [1], 0.1); c.append("M", [0, 1])
    return c


CIRCUITS = {
    "fig1": _fig1,
    "sec31": _sec31,
    "rep5": lambda: repetition_code(5, 5, 0.01),
    "surf3": lambda: surface_code(3, 3, 1e-2),
    "surf5": lambda: surface_code(5, 5, 2e-3),
    # X/Y/Z_ERROR, DEPOLARIZE1 and DEPOLARIZE2 channels all reach the detectors
    "allkinds": lambda: surface_code_all_channels(3, 3, 1e-3),
    "layered40": lambda: random_layered(40, 40, depolarize=0.01, seed=3),
    "wide1000": lambda: random_layered(1000, 3, cnot_pairs=500, depolarize=0.001, seed=4),
    # depolarizing events in most (block, shot) pairs: the warps' event queues fill and drain
    "noisy5": lambda: surface_code(5, 5, 0.05),
    # 256 qubits or more: the replay splits each event's rows over eight warps
    "layered300": lambda: random_layered(300, 30, depolarize=0.01, seed=6),
    "ffwide": lambda: random_feedforward_circuit(260, 3000, seed=810),
    # more than 577 qubits: the traversal's tableau spreads over a cluster of
    # 8 CTAs (80 to 125 qubit columns each), with resets and feed-forward
    "rand640": lambda: random_small_circuit(640, 5000, seed=930),
    "ff700": lambda: random_feedforward_circuit(700, 6000, seed=820),
    "rand1000": lambda: random_small_circuit(1000, 6000, seed=931),
}
for _s in range(8):
    CIRCUITS[f"rand{_s}"] = (lambda s=_s: random_small_circuit(3 + 7 * s, 60 + 30 * s, seed=900 + s))
for _s in range(6):
    CIRCUITS[f"cliff{_s}"] = (lambda s=_s: random_clifford_circuit(2 + 3 * s, 80 + 40 * s, seed=700 + s))
for _s in range(6):
    CIRCUITS[f"ff{_s}"] = (lambda s=_s: random_feedforward_circuit(3 + 6 * s, 60 + 40 * s, seed=800 + s))


def _u64(t):
    return t.cpu().numpy().view(np.uint64)


@pytest.fixture(scope="module")
def d11():
    c = surface_code(11, 11, 1e-3)
    return c, sp.build(c), oracle.Program(c)


@pytest.mark.parametrize("name", sorted(CIRCUITS))
def test_rows_match_oracle(name):
    c = CIRCUITS[name]()
    prog, ref = sp.build(c), oracle.Program(c)
    assert (prog.num_measurements, prog.num_detectors, prog.num_observables) == \
        (ref.num_meas, ref.num_det, ref.num_obs)
    assert prog.num_symbols == ref.num_symbols and prog.num_channels == ref.num_channels
    w = (ref.num_symbols + 1 + 63) // 64
    for which in ("meas", "det", "obs"):
        np.testing.assert_array_equal(prog.rows(which)[:, :w], ref.rows(which)[:, :w], err_msg=which)
    T, kind, s0 = prog.channels()
    ch = ref.channels()
    np.testing.assert_array_equal(T, ch.T)
    np.testing.assert_array_equal(s0, ch.sym0)
    want_kind = np.select([ch.type == 3, ch.type == 4, ch.type == 5], [1, 2, 3], 0)
    np.testing.assert_array_equal(kind, want_kind)
    # the channel table keeps every threshold; the draws evaluate only the
    # 4-channel blocks holding a channel that can fire (T > 0) with a symbol
    # some measurement row holds (the oracle's rows): the others change no
    # record
    held = np.unpackbits(np.bitwise_or.reduce(ref.rows("meas"), axis=0).view(np.uint8),
                         bitorder="little")[: ref.num_symbols + 1].astype(bool)
    live = np.array([ch.T[i] > 0 and held[ch.sym0[i]: ch.sym0[i] + ch.nsym[i]].any() for i in range(len(ch.T))],
                    dtype=bool)
    blocks = np.zeros((len(live) + 3) // 4, dtype=bool)
    blocks[np.nonzero(live)[0] // 4] = True
    assert prog.info["live_blocks"] == int(blocks.sum())


@pytest.mark.parametrize("path", ["fused", "staged"])
@pytest.mark.parametrize("name", ["fig1", "rep5", "surf3", "surf5", "layered40", "wide1000", "rand3", "rand7",
                                  "cliff2", "cliff5", "ff1", "ff4", "layered300", "ffwide", "rand640", "ff700",
                                  "rand1000"])
@pytest.mark.parametrize("shot0,shots", [(0, 1), (5, 31), (64, 33), (1 << 33, 1061), (7, 4101)])
def test_records_match_oracle(name, shot0, shots, path):
    c = CIRCUITS[name]()
    prog, ref = sp.build(c), oracle.Program(c)
    if path == "staged":
        prog.set_path(sp.PATH_SPARSE)
    else:
        assert prog.info["path"] == sp.PATH_FUSED, "small circuits take the fused path"
    m, d, o = prog.sample(shots, seed=17, shot0=shot0)
    torch.cuda.synchronize()
    rm, rd, ro = ref.sample(17, shot0, shots)
    np.testing.assert_array_equal(_u64(m), rm)
    np.testing.assert_array_equal(_u64(d), rd)
    np.testing.assert_array_equal(_u64(o), ro)


@pytest.mark.parametrize("tile", [32, 64, 128])
@pytest.mark.parametrize("name", ["surf5", "layered40"])
def test_fused_tiles_straddling_2_pow_32_shots(name, tile):
    """shot0 just below 2^32: some tiles hold shots with two different high
    counter words, which the draw must not treat as one."""
    c = CIRCUITS[name]()
    prog, ref = sp.build(c), oracle.Program(c)
    prog.set_fused_config(tile, 1)
    shot0 = (1 << 32) - 77
    m, d, o = prog.sample(301, seed=11, shot0=shot0)
    torch.cuda.synchronize()
    rm, rd, ro = ref.sample(11, shot0, 301)
    np.testing.assert_array_equal(_u64(m), rm)
    np.testing.assert_array_equal(_u64(d), rd)
    np.testing.assert_array_equal(_u64(o), ro)


@pytest.mark.parametrize("tile,variant", [(32, 1), (32, 2), (64, 1), (64, 2), (64, 3), (128, 1), (128, 2)])
@pytest.mark.parametrize("name", ["rep5", "surf5", "layered40", "rand6", "noisy5"])
def test_every_fused_variant_matches_oracle(name, tile, variant):
    c = CIRCUITS[name]()
    prog, ref = sp.build(c), oracle.Program(c)
    prog.set_fused_config(tile, variant)
    assert prog.info["fused_tile_shots"] == tile and prog.info["fused_variant"] == variant
    m, d, o = prog.sample(2113, seed=5, shot0=77)
    torch.cuda.synchronize()
    rm, rd, ro = ref.sample(5, 77, 2113)
    np.testing.assert_array_equal(_u64(m), rm)
    np.testing.assert_array_equal(_u64(d), rd)
    np.testing.assert_array_equal(_u64(o), ro)


def test_teleportation_with_feedforward():
    """Teleporting |1> with X_IF / Z_IF corrections: the last record is 1 in
    every shot while both Bell-measurement records are uniformly random."""
    c = Circuit(3)
    c.append("X", [0]); c.append("H", [1]); c.append("CX", [1, 2]); c.append("CX", [0, 1]); c.append("H", [0])
    c.append("M", [0, 1]); c.append("X_IF", [1, 2]); c.append("Z_IF", [2, 2]); c.append("M", [2])
    prog, ref = sp.build(c), oracle.Program(c)
    m, _, _ = prog.sample(4096, seed=9)
    torch.cuda.synchronize()
    rec = oracle.unpack_records(_u64(m), 3)
    assert rec[:, 2].all()
    assert 0.45 < rec[:, 0].mean() < 0.55 and 0.45 < rec[:, 1].mean() < 0.55
    np.testing.assert_array_equal(_u64(m), ref.sample(9, 0, 4096)[0])


def test_chunking_and_host_path_give_identical_records():
    c = surface_code(5, 5, 5e-3)
    prog = sp.build(c)
    shots = 10_000
    m0, d0, o0 = prog.sample(shots, seed=3, shot0=11)
    prog.set_chunk(1024)
    m1, d1, o1 = prog.sample(shots, seed=3, shot0=11)
    hm, hd, ho = prog.sample_host(shots, seed=3, shot0=11)
    torch.cuda.synchronize()
    for a, b, h in ((m0, m1, hm), (d0, d1, hd), (o0, o1, ho)):
        assert torch.equal(a, b)
        assert torch.equal(a.cpu(), h)
    # a sub-range equals the matching rows of the full range
    m2, _, _ = prog.sample(100, seed=3, shot0=11 + 5000)
    assert torch.equal(m2, m0[5000:5100])


def test_fig3c_circuit_staged_forms_equal_fused():
    """The paper's Fig. 3c circuit at n = 300 (300 qubits x 300 layers,
    DEPOLARIZE1(0.01), 184,584 symbols): the staged product with few shots
    (fired symbols pushed into L2-resident records) and with many shots
    (a fault-bit table gathered row by row) equals the fused kernel's records
    bit for bit, and sampled shots equal the oracle's."""
    c = random_layered(300, 300, depolarize=0.01, seed=1)
    prog = sp.build(c)
    assert prog.info["path"] == sp.PATH_FUSED
    ref = oracle.Program(c)
    for shots, shot0 in ((5_001, 77), (650_000, 1 << 32)):
        prog.set_path(sp.PATH_FUSED)
        fm, fd, fo = prog.sample(shots, seed=9, shot0=shot0)
        prog.set_path(sp.PATH_SPARSE)
        m, d, o = prog.sample(shots, seed=9, shot0=shot0)
        torch.cuda.synchronize()
        for a, b in ((m, fm), (d, fd), (o, fo)):
            assert torch.equal(a, b)
        pick = np.array([0, 1, 31, 32, shots // 2, shots - 1])
        rm, rd, ro = ref.sample_shots(9, shot0 + pick)
        idx = torch.as_tensor(pick, device="cuda")
        np.testing.assert_array_equal(_u64(m[idx]), rm)
        np.testing.assert_array_equal(_u64(d[idx]), rd)
    prog.set_path(sp.PATH_AUTO)


def test_host_path_with_a_short_last_piece():
    """300,001 shots into host buffers: the records come back in pieces and
    the last piece is cut short (one wave of the fused kernel's tiles) so
    that its copy is brief; every record equals sp_sample's."""
    prog = sp.build(surface_code(5, 5, 2e-3))
    shots = 300_001
    m0, d0, o0 = prog.sample(shots, seed=4, shot0=7)
    hm, hd, ho = prog.sample_host(shots, seed=4, shot0=7)
    torch.cuda.synchronize()
    for a, h in ((m0, hm), (d0, hd), (o0, ho)):
        assert torch.equal(a.cpu(), h)


def test_full_size_d11_sampled_shots(d11):
    """The d=11 r=11 p=1e-3 configuration at 1e6 shots in the launch
    configuration the benchmark times; 300 shots spread over the range are
    recomputed one by one by the oracle."""
    c, prog, ref = d11
    shots = 1_000_000
    m, d, o = prog.sample(shots, seed=1, shot0=0)
    torch.cuda.synchronize()
    rng = np.random.default_rng(0)
    pick = np.unique(np.concatenate([rng.integers(0, shots, 296), [0, 31, 32, shots - 1]]))
    rm, rd, ro = ref.sample_shots(1, pick)
    idx = torch.as_tensor(pick, device="cuda")
    np.testing.assert_array_equal(_u64(m[idx]), rm)
    np.testing.assert_array_equal(_u64(d[idx]), rd)
    np.testing.assert_array_equal(_u64(o[idx]), ro)
    # pad bits beyond the last record are zero in every shot
    nm = prog.num_measurements
    pad_mask = np.uint64(~((1 << (nm % 64)) - 1) & 0xFFFFFFFFFFFFFFFF) if nm % 64 else np.uint64(0)
    last = _u64(m[:, -1])
    assert not np.any(last & pad_mask)


def test_config1_every_shot():
    """Repetition-code memory d=5, 5 rounds, X_ERROR(0.01): all 1e4 shots at
    seed 1 against the oracle, record for record."""
    c = repetition_code(5, 5, 0.01)
    prog, ref = sp.build(c), oracle.Program(c)
    m, d, o = prog.sample(10_000, seed=1, shot0=0)
    torch.cuda.synchronize()
    rm, rd, ro = ref.sample_parallel(1, 0, 10_000)
    np.testing.assert_array_equal(_u64(m), rm)
    np.testing.assert_array_equal(_u64(d), rd)
    np.testing.assert_array_equal(_u64(o), ro)


@pytest.mark.parametrize("path", ["fused", "staged"])
def test_full_size_d11_contiguous_range(d11, path):
    """One call of 1,100,000 shots of the d=11 configuration; 16,384
    consecutive shots from 1,040,000 on are recomputed by the oracle (on all
    host cores). The range spans the staged path's 1,048,576-shot chunk
    boundary and, on the fused path, the boundary of kernel waves of
    num_SMs x CTAs/SM tiles at 1,050,624 (54 waves of 304 x 64 shots)."""
    c, prog, ref = d11
    prog.set_path(sp.PATH_FUSED if path == "fused" else sp.PATH_SPARSE)
    try:
        assert prog.info["chunk_shots"] == 1 << 20
        m, d, o = prog.sample(1_100_000, seed=6, shot0=0)
        torch.cuda.synchronize()
        a, n = 1_040_000, 16_384
        rm, rd, ro = ref.sample_parallel(6, a, n)
        np.testing.assert_array_equal(_u64(m[a:a + n]), rm)
        np.testing.assert_array_equal(_u64(d[a:a + n]), rd)
        np.testing.assert_array_equal(_u64(o[a:a + n]), ro)
    finally:
        prog.set_path(sp.PATH_AUTO)


@pytest.mark.parametrize("path", ["fused", "staged"])
def test_full_size_d11_both_paths_agree(d11, path):
    c, prog, ref = d11
    prog.set_path(sp.PATH_FUSED if path == "fused" else sp.PATH_SPARSE)
    try:
        m, d, o = prog.sample(200_000, seed=4, shot0=999)
        torch.cuda.synchronize()
        pick = np.array([0, 1, 31, 32, 63, 64, 65, 1023, 1024, 99_999, 150_001, 199_999])
        rm, rd, ro = ref.sample_shots(4, pick + 999)
        idx = torch.as_tensor(pick, device="cuda")
        np.testing.assert_array_equal(_u64(m[idx]), rm)
        np.testing.assert_array_equal(_u64(d[idx]), rd)
        np.testing.assert_array_equal(_u64(o[idx]), ro)
    finally:
        prog.set_path(sp.PATH_AUTO)


@pytest.mark.parametrize("tile,variant", [(64, 1), (64, 3), (128, 1), (128, 2)])
def test_full_size_d11_fused_variants_agree(d11, tile, variant):
    """Every 64- and 128-shot launch shape gives the records of the
    autotuner's choice at d=11 (200,000 shots, ragged tail), and a few shots
    are recomputed by the oracle."""
    c, prog, ref = d11
    tuned = (prog.info["fused_tile_shots"], prog.info["fused_variant"])
    base = prog.sample(200_003, seed=8, shot0=5)
    prog.set_fused_config(tile, variant)
    try:
        assert prog.info["fused_tile_shots"] == tile and prog.info["fused_variant"] == variant
        out = prog.sample(200_003, seed=8, shot0=5)
        torch.cuda.synchronize()
        for a, b in zip(out, base):
            assert torch.equal(a, b)
        pick = np.array([0, 127, 128, 200_002])
        rm, rd, ro = ref.sample_shots(8, pick + 5)
        idx = torch.as_tensor(pick, device="cuda")
        np.testing.assert_array_equal(_u64(out[0][idx]), rm)
        np.testing.assert_array_equal(_u64(out[1][idx]), rd)
    finally:
        prog.set_fused_config(*tuned)


@pytest.mark.parametrize("name", ["rand640", "rand1000"])
def test_traversal_without_a_cluster(name, monkeypatch):
    """The one-CTA traversal with its tableau in global memory (the fallback
    when no thread-block cluster can be launched) gives the same rows and
    records as the oracle."""
    monkeypatch.setenv("SP_TRAVERSE_NO_CLUSTER", "1")
    c = CIRCUITS[name]()
    prog, ref = sp.build(c), oracle.Program(c)
    w = (ref.num_symbols + 1 + 63) // 64
    for which in ("meas", "det"):
        np.testing.assert_array_equal(prog.rows(which)[:, :w], ref.rows(which)[:, :w], err_msg=which)
    m, d, o = prog.sample(1061, seed=3, shot0=7)
    torch.cuda.synchronize()
    rm, rd, ro = ref.sample(3, 7, 1061)
    np.testing.assert_array_equal(_u64(m), rm)
    np.testing.assert_array_equal(_u64(d), rd)


def _long_repetition(rounds: int, noisy_every: int, p: float):
    """Distance-3 repetition memory with many rounds (about four record rows
    per round) and X_ERROR(p) on the data qubits only every noisy_every
    rounds, so the rows are many and the symbols few."""
    c = Circuit(5)
    c.append("R", [0, 1, 2, 3, 4])
    for r in range(rounds):
        if r % noisy_every == 0:
            c.append("X_ERROR", [0, 1, 2], p)
        c.append("CX", [0, 3, 1, 4])
        c.append("CX", [1, 3, 2, 4])
        c.append("MR", [3, 4])
        for i in range(2):
            c.append("DETECTOR", [2 - i] if r == 0 else [2 - i, 4 - i])
    c.append("M", [0, 1, 2])
    for i in range(2):
        # data i, data i+1 and ancilla i of the last round
        c.append("DETECTOR", [3 - i, 2 - i, 5 - i])
    c.append("OBSERVABLE_INCLUDE", [3], 0)
    return c


@pytest.mark.parametrize("rounds,tile", [(8000, 32), (15000, 0)])
def test_records_beyond_shared_memory(rounds, tile):
    """Maximum sizes of the fused tile: at 8,000 rounds (32k record rows) the
    records fit in shared memory only as 32-shot tiles; at 15,000 (60k rows)
    not at all, and the fused path is refused. The build's own choice, the
    staged path, both dense products and (where it fits) the fused path all
    give the oracle's records."""
    c = _long_repetition(rounds, 1000, 0.05)
    prog, ref = sp.build(c), oracle.Program(c)
    assert prog.num_measurements == 2 * rounds + 3
    assert prog.info["fused_tile_shots"] == tile
    if not tile:
        with pytest.raises(sp.SymPhaseError):
            prog.set_path(sp.PATH_FUSED)
    rm, rd, ro = ref.sample(6, 31, 301)
    assert rd.any()   # faults reach the detectors
    paths = [sp.PATH_AUTO, sp.PATH_SPARSE, sp.PATH_DENSE, sp.PATH_TENSOR] + ([sp.PATH_FUSED] if tile else [])
    for path in paths:
        prog.set_path(path)
        m, d, o = prog.sample(301, seed=6, shot0=31)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(_u64(m), rm, err_msg=f"path {path}")
        np.testing.assert_array_equal(_u64(d), rd, err_msg=f"path {path}")
        np.testing.assert_array_equal(_u64(o), ro, err_msg=f"path {path}")
    assert prog.device_status() == 0


@pytest.mark.parametrize("path", ["fused", "staged"])
def test_full_size_d17_in_64k_chunks(path):
    """d=17 r=17 p=2e-3 (about 100k symbols), 1e6 shots sampled in
    65536-shot chunks on the fused and the staged path; 48 shots spread over
    the range are recomputed by the oracle."""
    c = surface_code(17, 17, 2e-3)
    prog, ref = sp.build(c), oracle.Program(c)
    assert prog.info["path"] == sp.PATH_FUSED
    if path == "staged":
        prog.set_path(sp.PATH_SPARSE)
    prog.set_chunk(65536)
    shots = 1_000_000
    m, d, o = prog.sample(shots, seed=3, shot0=0)
    torch.cuda.synchronize()
    rng = np.random.default_rng(17)
    pick = np.unique(np.concatenate([rng.integers(0, shots, 44), [0, 65535, 65536, shots - 1]]))
    rm, rd, ro = ref.sample_shots(3, pick)
    idx = torch.as_tensor(pick, device="cuda")
    np.testing.assert_array_equal(_u64(m[idx]), rm)
    np.testing.assert_array_equal(_u64(d[idx]), rd)
    np.testing.assert_array_equal(_u64(o[idx]), ro)


def test_full_size_d11_detector_rates(d11):
    """Monte-Carlo detector rates of 1e6 GPU shots against the analytic
    expectation, within 5 sigma."""
    c, prog, ref = d11
    shots = 1_000_000
    _, d, _ = prog.sample(shots, seed=2, shot0=0, meas=False, obs=False)
    bits = torch.zeros(prog.num_detectors, dtype=torch.float64, device="cuda")
    dd = d.view(torch.int64)
    for j in range(prog.num_detectors):
        bits[j] = ((dd[:, j // 64] >> (j % 64)) & 1).sum()
    rates = (bits / shots).cpu().numpy()
    la = prog.expect_raw().cpu().numpy()[: prog.num_detectors].astype(np.float64)
    r = (1 - np.exp(la)) / 2
    z = np.abs(rates - r) / np.sqrt(r * (1 - r) / shots)
    assert z.max() < 5.0, z.max()


def _draw_p(rng, n, regime):
    """Per-channel probabilities: circuit-level noise, or large rates where
    factors 1 - 2 kappa p turn negative (X_ERROR above 1/2, DEPOLARIZE1 above
    3/4, DEPOLARIZE2 at 1) or vanish (X/Y/Z_ERROR at exactly 1/2)."""
    if regime == "small":
        return rng.uniform(5e-4, 2e-3, n).astype(np.float32)
    p = rng.uniform(5e-4, 2e-3, n)
    big = rng.random(n) < 0.05
    p[big] = rng.choice([0.3, 0.5, 0.6, 0.8, 1.0], big.sum())
    return p.astype(np.float32)


def _check_expect(prog, ref, p):
    pt = torch.as_tensor(p, device="cuda")
    got = prog.expect_raw(pt).cpu().numpy().astype(np.float64)
    sgn = prog.expect_sign_raw(pt).cpu().numpy()
    la, sa = ref.expect(p.astype(np.float64))
    zero = np.isneginf(la)
    np.testing.assert_array_equal(np.isneginf(got), zero)
    np.testing.assert_allclose(got[~zero], la[~zero], rtol=1e-4, atol=1e-6)
    np.testing.assert_array_equal(sgn[zero], 0.0)
    np.testing.assert_array_equal(sgn[~zero], sa[~zero].astype(np.float32))
    return zero


@pytest.mark.parametrize("regime", ["small", "large"])
@pytest.mark.parametrize("name", ["rep5", "surf3", "surf5", "allkinds"])
def test_expectation_matches_oracle(name, regime):
    """log|E| and sign E of every detector and observable against the FP64
    oracle, over channel probabilities up to 1 (negative and zero factors)."""
    c = CIRCUITS[name]()
    prog, ref = sp.build(c), oracle.Program(c)
    assert prog.num_detectors > 0
    rng = np.random.default_rng(1)
    p = _draw_p(rng, prog.num_channels, regime)
    if regime == "large":
        # every 37th one-symbol channel at exactly 1/2: its factor vanishes
        _, kind, _ = prog.channels()
        p[np.flatnonzero(kind == 0)[::37]] = 0.5
    zero = _check_expect(prog, ref, p)
    if regime == "large":
        _, sa = ref.expect(p.astype(np.float64))
        assert (sa[~zero] < 0).any(), "no negative expectation was exercised"
        assert zero.any(), "no vanishing expectation was exercised"


def _check_grad(prog, ref, p, g):
    """The adjoint against the FP64 oracle, element by element: relative 1e-4,
    with an absolute floor of 1e-5 times the element's own scale, the sum of
    the absolute values of its terms (what FP32 accumulation error is
    relative to)."""
    pt = torch.as_tensor(p, device="cuda")
    grad = prog.expect_grad_raw(pt, torch.as_tensor(g, device="cuda")).cpu().numpy().astype(np.float64)
    want = ref.expect_vjp(p.astype(np.float64), g.astype(np.float64))
    scale = np.abs(ref.expect_vjp(p.astype(np.float64), np.abs(g).astype(np.float64)))
    err = np.abs(grad - want)
    bad = err > 1e-4 * np.abs(want) + 1e-5 * scale
    assert not bad.any(), (np.flatnonzero(bad)[:5], grad[bad][:5], want[bad][:5])
    return grad, want


@pytest.mark.parametrize("regime", ["small", "large"])
def test_gradient_all_channel_kinds(regime):
    c = CIRCUITS["allkinds"]()
    prog, ref = sp.build(c), oracle.Program(c)
    rng = np.random.default_rng(3)
    p = _draw_p(rng, prog.num_channels, regime)
    # keep the gradient finite: no factor exactly zero
    _, kind, _ = prog.channels()
    p[(kind == 0) & (p == 0.5)] = 0.6
    g = rng.normal(size=prog.num_detectors + prog.num_observables).astype(np.float32)
    _check_grad(prog, ref, p, g)


def test_expectation_d11_and_gradient(d11):
    c, prog, ref = d11
    rng = np.random.default_rng(5)
    p = rng.uniform(5e-4, 2e-3, prog.num_channels).astype(np.float32)
    pt = torch.as_tensor(p, device="cuda")
    got = prog.expect_raw(pt).cpu().numpy().astype(np.float64)
    la, _ = ref.expect(p.astype(np.float64))
    np.testing.assert_allclose(got, la, rtol=1e-4)
    g = rng.normal(size=prog.num_detectors + prog.num_observables).astype(np.float32)
    grad, want = _check_grad(prog, ref, p, g)
    scale = np.abs(want).max()
    # central differences of the FP64 oracle on 64 channels
    h = 1e-6
    p64 = p.astype(np.float64)
    for ch in rng.choice(prog.num_channels, 64, replace=False):
        if want[ch] == 0:
            continue
        pp, pm = p64.copy(), p64.copy()
        pp[ch] += h
        pm[ch] -= h
        fd = (ref.expect(pp)[0] @ g - ref.expect(pm)[0] @ g) / (2 * h)
        assert abs(grad[ch] - fd) <= 1e-3 * abs(fd) + 1e-6 * scale, (ch, grad[ch], fd)


def test_autograd_function(d11):
    c, prog, ref = d11
    rng = np.random.default_rng(9)
    p = torch.tensor(rng.uniform(5e-4, 2e-3, prog.num_channels), dtype=torch.float32,
                     device="cuda", requires_grad=True)
    target = torch.rand(prog.num_detectors + prog.num_observables, device="cuda") * 0.02
    logE = sp.expect(prog, p)
    r = (1 - torch.exp(logE)) / 2
    loss = ((r - target) ** 2).sum()
    loss.backward()
    g = (2 * (r - target) * (-0.5) * torch.exp(logE)).detach().cpu().numpy().astype(np.float64)
    want = ref.expect_vjp(p.detach().cpu().numpy().astype(np.float64), g)
    got = p.grad.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(got, want, rtol=1e-3, atol=1e-4 * np.abs(want).max())


def test_nondeterministic_detector_is_rejected():
    c = Circuit(2)
    c.append("H", [0]); c.append("M", [0]); c.append("DETECTOR", [1])
    with pytest.raises(sp.SymPhaseError) as e:
        sp.build(c)
    assert e.value.status == 3


def test_noiseless_and_symbol_free_circuits():
    c = Circuit(3)
    c.append("X", [1]); c.append("CX", [1, 2]); c.append("M", [0, 1, 2])
    c.append("DETECTOR", [1, 2]); c.append("OBSERVABLE_INCLUDE", [1], 0)
    prog = sp.build(c)
    assert prog.num_symbols == 0
    m, d, o = prog.sample(100, seed=1)
    torch.cuda.synchronize()
    assert np.all(_u64(m)[:, 0] == 0b110)
    assert np.all(_u64(d)[:, 0] == 0)
    assert np.all(_u64(o)[:, 0] == 1)


def test_zero_shots_and_null_outputs():
    prog = sp.build(repetition_code(3, 2, 0.1))
    prog.sample(0, seed=1)
    m, d, o = prog.alloc_outputs(50)
    prog.sample(50, seed=1, out=(m, d, o), meas=False, obs=False)
    torch.cuda.synchronize()
    ref = oracle.Program(repetition_code(3, 2, 0.1))
    np.testing.assert_array_equal(_u64(d), ref.sample(1, 0, 50)[1])
