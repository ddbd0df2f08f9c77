"""The oracle's symbolic forms against an independent concrete CHP-style
tableau re-simulated shot by shot under the same symbol bits (<= 20 qubits).
By Fact 2 the branches taken do not depend on the phases, so for every
assignment b of the symbols the records of the concrete run must equal the
affine forms evaluated at b."""
import numpy as np
import pytest

import oracle
from checkers import chp
from workloads import (random_clifford_circuit, random_feedforward_circuit, random_small_circuit, repetition_code,
                       surface_code)


def _check(circuit, nassign, seed, density):
    prog = oracle.Program(circuit)
    rng = np.random.default_rng(seed)
    for _ in range(nassign):
        b = (rng.random(prog.num_symbols + 1) < density).astype(np.uint8)
        b[0] = 1
        m, d, o = prog.evaluate(b)
        cm, cd, co = chp.simulate(circuit, b)
        np.testing.assert_array_equal(oracle.unpack_records(m[None], prog.num_meas)[0], cm)
        np.testing.assert_array_equal(oracle.unpack_records(d[None], prog.num_det)[0], cd)
        np.testing.assert_array_equal(oracle.unpack_records(o[None], prog.num_obs)[0], co)


@pytest.mark.parametrize("seed", range(24))
def test_random_circuits(seed):
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(1, 21))
    circuit = random_small_circuit(n, int(rng.integers(10, 120)), seed=seed)
    _check(circuit, 6, seed, density=0.5)


@pytest.mark.parametrize("seed", range(48))
def test_clifford_heavy_circuits(seed):
    """Long H/S/CX sequences with few measurements: deterministic outcomes
    then depend on Y phases and on long products of stabilizer rows."""
    rng = np.random.default_rng(2000 + seed)
    circuit = random_clifford_circuit(int(rng.integers(2, 9)), int(rng.integers(20, 90)), seed=3000 + seed)
    _check(circuit, 4, seed, density=0.5)


@pytest.mark.parametrize("seed", range(32))
def test_feedforward_circuits(seed):
    """X_IF / Y_IF / Z_IF conditioned on earlier records (Sec. 6's
    conditional Paulis): the concrete run applies the Pauli when the record
    it reads is 1."""
    rng = np.random.default_rng(4000 + seed)
    circuit = random_feedforward_circuit(int(rng.integers(2, 12)), int(rng.integers(20, 90)), seed=5000 + seed)
    _check(circuit, 4, seed, density=0.5)


def test_repetition_code():
    _check(repetition_code(5, 5, 0.01), 20, 1, density=0.1)


@pytest.mark.parametrize("density", [0.02, 0.5])
def test_surface_code_d3(density):
    _check(surface_code(3, 3, 1e-3), 10, 2, density=density)


def test_noiseless_surface_code_detectors_are_zero():
    circuit = surface_code(3, 3, 0.0)
    prog = oracle.Program(circuit)
    m, d, o = prog.sample(seed=9, shot0=0, nshots=64)
    assert not d.any() and not o.any()
