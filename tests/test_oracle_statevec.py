"""The oracle against a dense state-vector simulator (<= 8 qubits): for a
fixed fault assignment, the measurement-record distribution obtained by
enumerating the 2^k random-measurement symbols (each assignment with
probability 2^-k) must equal the exact branching distribution."""
from collections import defaultdict

import numpy as np
import pytest

import oracle
from checkers import statevec
from workloads import random_clifford_circuit, random_feedforward_circuit, random_small_circuit


@pytest.mark.parametrize("seed", range(36))
def test_distribution_matches(seed):
    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(1, 8))
    if seed < 16:
        circuit = random_small_circuit(n, int(rng.integers(8, 40)), seed=100 + seed)
    elif seed < 24:
        circuit = random_clifford_circuit(max(n, 2), int(rng.integers(20, 60)), seed=200 + seed)
    else:
        circuit = random_feedforward_circuit(max(n, 2), int(rng.integers(10, 50)), seed=300 + seed)
    prog = oracle.Program(circuit)
    rnd = prog.random_symbols()
    rand_syms = [s for s in range(1, prog.num_symbols + 1) if rnd[s]]
    fault_syms = [s for s in range(1, prog.num_symbols + 1) if not rnd[s]]
    if len(rand_syms) > 12:
        pytest.skip("too many random measurements to enumerate")
    for trial in range(3):
        fault_bits = (rng.random(len(fault_syms)) < 0.5).astype(np.uint8)
        sv = statevec.distribution(circuit, fault_bits)
        sym = defaultdict(float)
        k = len(rand_syms)
        for mask in range(1 << k):
            b = np.zeros(prog.num_symbols + 1, np.uint8)
            b[0] = 1
            b[fault_syms] = fault_bits
            for i, s in enumerate(rand_syms):
                b[s] = (mask >> i) & 1
            m, _, _ = prog.evaluate(b)
            rec = tuple(int(v) for v in oracle.unpack_records(m[None], prog.num_meas)[0])
            sym[rec] += 2.0 ** -k
        assert set(sym) == set(sv), (sorted(sym), sorted(sv))
        for rec, pr in sym.items():
            assert abs(pr - sv[rec]) < 1e-9, (rec, pr, sv[rec])
