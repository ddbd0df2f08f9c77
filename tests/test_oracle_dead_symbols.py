"""Eq. sampling restricted to the symbols that matter: a symbol whose column
is zero in every measurement row changes no record, since detectors and
observables are XORs of measurement records.  The per-channel draw skips the
channel blocks made only of such symbols' channels; these tests pin, on the
oracle alone, that clearing those symbols' fault bits leaves every record
unchanged, that detector and observable rows hold no other symbols, and that
such symbols are common in the paper's random layered circuits (most of
their measurements are random and erase the faults before them)."""
import numpy as np
import pytest

import oracle
from workloads import random_layered, surface_code


def _held(ref):
    rows = ref.rows("meas")
    acc = np.bitwise_or.reduce(rows, axis=0) if len(rows) else np.zeros(ref.pw, np.uint64)
    return np.unpackbits(acc.view(np.uint8), bitorder="little")[: ref.num_symbols + 1].astype(bool)


def _bits(words, n):
    if len(words) == 0:
        return np.zeros(n, bool)
    acc = np.bitwise_or.reduce(words, axis=0)
    return np.unpackbits(acc.view(np.uint8), bitorder="little")[:n].astype(bool)


CASES = {
    "layered60": (lambda: random_layered(60, 60, depolarize=0.01, seed=1), 0.5),
    "surface3": (lambda: surface_code(3, 3, 2e-2), 0.0),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_symbols_outside_every_measurement_row_change_no_record(name):
    make, min_dead = CASES[name]
    ref = oracle.Program(make())
    held = _held(ref)
    dead = ~held
    dead[0] = False                      # the constant
    assert dead[1:].mean() >= min_dead, dead[1:].mean()
    # detector and observable rows only hold symbols of measurement rows
    n = ref.num_symbols + 1
    assert not (_bits(ref.rows("det"), n) & dead).any()
    assert not (_bits(ref.rows("obs"), n) & dead).any()
    seed = 77
    touched = 0
    for shot in range(24):
        b = ref.draw_bits(seed, shot)
        cleared = b.copy()
        cleared[dead] = 0
        touched += int((b != cleared).any())
        full = ref.evaluate(b)
        kept = ref.evaluate(cleared)
        sampled = ref.sample(seed, shot, 1)
        for x, y, z in zip(full, kept, sampled):
            np.testing.assert_array_equal(x, y)
            np.testing.assert_array_equal(x, z[0])
    # not vacuous: some shots drew faults on those symbols
    assert touched > 0 or not dead.any()
