"""Host-side checks of the synthetic workload generators (no GPU): the mirror
circuit undoes its own Clifford layers, so every noiseless record is 0 and its
detectors are deterministic; its coefficient rows are dense; the paper's
random layered circuits are mostly random outcomes with sparse rows."""
import numpy as np

import oracle
from checkers import chp
from workloads import mirror_circuit, random_layered


def test_mirror_circuit_noiseless_records_are_zero():
    for n, layers, seed in [(6, 4, 0), (12, 8, 1), (30, 10, 2)]:
        prog = oracle.Program(mirror_circuit(n, layers, p=0.0, seed=seed))
        m, d, _ = prog.sample(seed=5, shot0=0, nshots=8)
        assert not m.any() and not d.any()
        assert prog.num_meas == n and prog.num_det == n


def test_mirror_circuit_is_an_identity_under_chp():
    """The concrete CHP tableau (independent of the oracle) measures 0 on
    every qubit of the noiseless mirror circuit."""
    c = mirror_circuit(10, 6, p=0.0, seed=3)
    m, d, _ = chp.simulate(c, np.array([1], np.uint8))
    assert not np.any(m) and not np.any(d)


def test_mirror_circuit_rows_are_dense():
    prog = oracle.Program(mirror_circuit(48, 16, p=0.01, seed=2))
    bits = prog.row_bits("meas")[:, 1:]
    assert bits.mean() > 0.2


def test_random_layered_rows_are_sparse():
    prog = oracle.Program(random_layered(60, 60, depolarize=0.01, seed=1))
    bits = prog.row_bits("meas")[:, 1:]
    assert bits.mean() < 0.01
    # most records are a fresh random-measurement symbol
    rnd = prog.random_symbols()
    assert rnd.sum() > 0.5 * prog.num_meas


def test_per_channel_probabilities_follow_channel_order():
    from workloads import channel_probabilities, surface_code, with_channel_probabilities
    base = surface_code(3, 3, 1e-3)
    p = channel_probabilities(base.num_fault_channels, seed=4)
    c = with_channel_probabilities(base, p)
    assert c.num_fault_channels == base.num_fault_channels
    prog, ref = oracle.Program(c), oracle.Program(base)
    ch = prog.channels()
    fault = ch.type != 5          # random-measurement channels keep 1/2
    np.testing.assert_allclose(ch.p[fault], p)
    # same symbols and coefficient rows: only the probabilities changed
    np.testing.assert_array_equal(prog.rows("det"), ref.rows("det"))
    np.testing.assert_array_equal(prog.channels().sym0, ref.channels().sym0)
