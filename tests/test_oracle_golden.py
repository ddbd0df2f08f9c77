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
