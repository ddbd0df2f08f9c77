"""The oracle against the paper's two worked examples (Fig. 1 and the
two-qubit example of Sec. 3.1), symbol for symbol and tableau for tableau."""
import numpy as np
import pytest

import oracle
from golden_fixtures import load


def _pad(v, n):
    out = np.zeros(n, np.uint8)
    out[: len(v)] = v[:n]
    return out


@pytest.mark.parametrize("fixture,nsym", [("fig1_four_qubit.txt", 4), ("sec31_two_qubit.txt", 3)])
def test_outcomes(fixture, nsym):
    circuit, outcomes, _ = load(fixture, nsym)
    prog = oracle.Program(circuit)
    assert prog.num_symbols == nsym
    rows = prog.row_bits("meas")
    assert rows.shape[0] == len(outcomes)
    for k, v in outcomes.items():
        np.testing.assert_array_equal(rows[k], v, err_msg=f"m{k + 1}")


@pytest.mark.parametrize("fixture,nsym", [("fig1_four_qubit.txt", 4), ("sec31_two_qubit.txt", 3)])
def test_intermediate_tableaux(fixture, nsym):
    circuit, _, tables = load(fixture, nsym)
    assert tables
    for (kind, after), rows in tables.items():
        prog = oracle.Program(circuit, stop=after)
        x, z, ph = prog.tableau()
        n = prog.num_qubits
        sel = range(n, 2 * n) if kind == "stabilizers" else range(2 * n)
        for want, r in zip(rows, sel):
            np.testing.assert_array_equal(x[r], want[0], err_msg=f"{kind} after {after}, row {r} x")
            np.testing.assert_array_equal(z[r], want[1], err_msg=f"{kind} after {after}, row {r} z")
            np.testing.assert_array_equal(_pad(ph[r], nsym + 1), want[2],
                                          err_msg=f"{kind} after {after}, row {r} phase")


def test_random_measurement_only_new_row_gets_symbol():
    """Reading of the random branch of Init-M: only the new stabilizer row
    carries the new symbol. Applying X^s to every row with z_a = 1 instead
    would give m2 = s1 + s2 in the Sec. 3.1 example; the printed tableau
    gives s1 + s2 + s3."""
    circuit, outcomes, _ = load("sec31_two_qubit.txt", 3)
    prog = oracle.Program(circuit)
    m2 = prog.row_bits("meas")[1]
    assert m2[3] == 1 and m2[1] == 1 and m2[2] == 1


@pytest.mark.parametrize("basis", ["Z", "X"])
def test_teleportation_with_feedforward_is_deterministic(basis):
    """Teleporting |1> (or |->) from qubit 0 to qubit 2 with the textbook
    corrections X_IF (from qubit 1's outcome) and Z_IF (from qubit 0's) makes
    the final record the constant 1: no random symbol survives in it,
    although both Bell-measurement outcomes are random."""
    from workloads import Circuit
    c = Circuit(3)
    c.append("X", [0])
    if basis == "X":
        c.append("H", [0])
    c.append("H", [1]); c.append("CX", [1, 2])        # Bell pair (1, 2)
    c.append("CX", [0, 1]); c.append("H", [0])        # Bell measurement of (0, 1)
    c.append("M", [0, 1])
    c.append("X_IF", [1, 2]); c.append("Z_IF", [2, 2])
    if basis == "X":
        c.append("H", [2])
    c.append("M", [2])
    prog = oracle.Program(c)
    rnd = prog.random_symbols()
    rows = prog.row_bits("meas")
    assert rnd.sum() == 2 and rows[0][1:].any() and rows[1][1:].any()   # Bell outcomes random
    assert rows[2][0] == 1 and not rows[2][1:].any()                   # teleported record = 1
    # without the corrections the record depends on the random outcomes
    c2 = Circuit(3, [op for op in c.ops if op.name not in ("X_IF", "Z_IF")])
    assert oracle.Program(c2).row_bits("meas")[2][1:].any()
