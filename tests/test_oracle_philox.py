"""Pins of the oracle's fault draw: Philox4x32-10 against the published
known-answer vectors of the Random123 distribution (Salmon et al., SC'11),
the integer thresholds, and the channel distributions of Sec. 3.1
(X-error Bernoulli(p); depolarizing X^{s1}Z^{s2} with 00 w.p. 1-p and the
three others p/3 each) checked by chi-square tests."""
import numpy as np
import pytest

import oracle
from workloads import Circuit

# (counter, key, expected output) -- Random123 kat_vectors, philox4x32 10 rounds
KAT = [
    ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
    ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
    ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
     (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
]


@pytest.mark.parametrize("ctr,key,want", KAT)
def test_philox_known_answers(ctr, key, want):
    np.testing.assert_array_equal(oracle.philox4x32_10(ctr, key), np.array(want, np.uint32))


def test_thresholds():
    assert oracle.threshold(0.0) == 0
    assert oracle.threshold(1.0) == 2 ** 32 - 1
    assert oracle.threshold(0.5) == 2 ** 31
    assert oracle.threshold(1e-3) == 4294967          # floor(4294967.296)
    assert oracle.threshold(2.0 ** -32) == 1
    assert oracle.threshold(0.75) == 3 * 2 ** 30


def test_draw_uses_counter_layout():
    """channel c of shot t: counter (t lo, t hi, c // 4, 0), key (seed lo, seed
    hi), word c % 4, bit = word < T."""
    c = Circuit(1)
    c.append("X_ERROR", [0] * 9, 0.5)
    prog = oracle.Program(c)
    seed, shot = 0x1234_5678_9ABC_DEF0, (7 << 32) + 3
    bits = prog.draw_bits(seed, shot)
    assert bits[0] == 1
    for ch in range(9):
        w = oracle.philox4x32_10((shot & 0xFFFFFFFF, shot >> 32, ch // 4, 0),
                                 (seed & 0xFFFFFFFF, seed >> 32))[ch % 4]
        assert bits[1 + ch] == int(w < 2 ** 31)


def _chi2_ok(counts, probs, n):
    exp = n * np.asarray(probs)
    chi2 = float(((counts - exp) ** 2 / exp).sum())
    dof = len(probs) - 1
    # generous bound: mean + 6 sd of the chi-square distribution
    return chi2 < dof + 6 * np.sqrt(2 * dof), chi2


def _outcome_counts(prog, seed, nshots, sym0, k):
    counts = np.zeros(1 << k, np.int64)
    for t in range(nshots):
        b = prog.draw_bits(seed, t)
        v = sum(int(b[sym0 + i]) << i for i in range(k))
        counts[v] += 1
    return counts


def test_depolarize1_distribution():
    p, n = 0.6, 12000
    c = Circuit(1)
    c.append("DEPOLARIZE1", [0], p)
    prog = oracle.Program(c)
    counts = _outcome_counts(prog, 11, n, 1, 2)
    ok, chi2 = _chi2_ok(counts, [1 - p, p / 3, p / 3, p / 3], n)
    assert ok, (counts, chi2)


def test_depolarize2_distribution():
    p, n = 0.75, 16000
    c = Circuit(2)
    c.append("DEPOLARIZE2", [0, 1], p)
    prog = oracle.Program(c)
    counts = _outcome_counts(prog, 5, n, 1, 4)
    ok, chi2 = _chi2_ok(counts, [1 - p] + [p / 15] * 15, n)
    assert ok, (counts, chi2)


def test_bernoulli_and_random_measurement_rates():
    n = 12000
    c = Circuit(2)
    c.append("X_ERROR", [0], 0.3)
    c.append("H", [1])
    c.append("M", [1])           # random outcome -> fair-coin symbol
    prog = oracle.Program(c)
    assert prog.random_symbols().tolist() == [False, False, True]
    b = np.array([prog.draw_bits(3, t)[:3] for t in range(n)])
    for col, p in ((1, 0.3), (2, 0.5)):
        k = b[:, col].sum()
        assert abs(k - n * p) < 5 * np.sqrt(n * p * (1 - p)), (col, k)
