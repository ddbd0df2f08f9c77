"""Pins of the oracle's grouped draw (stream 2, opt-in): the same channel
distributions as the first stream (Sec. 3.1: X/Y/Z-error Bernoulli(p);
depolarizing X^{s1}Z^{s2} with each non-identity outcome p/3, two-qubit p/15;
a random outcome a fair coin), independent across channels, drawn through
a group test and a walk to the first fired channel. Checked by z-scores of
per-channel rates, chi-square tests of outcome frequencies, of the number of
channels fired per group (a Poisson-binomial law computed exactly) and of
the gap from a group's start to its first fired channel (a truncated
geometric law), pairwise joint rates, and the special cases p = 0 and 1."""
import numpy as np
import pytest
from scipy import stats

import oracle
from workloads import Circuit

SHOTS = 20_000


def _circuit():
    """One qubit and 184 noise channels: a group of 32 X_ERRORs whose first
    channel has p = 0.3 and the others 0.01, a group all at 0.01, then 80
    X_ERRORs at several rates (spanning groups, with zero and one), then
    DEPOLARIZE1 and DEPOLARIZE2, and four random measurements interleaved
    (H then M)."""
    c = Circuit(3)
    c.append("X_ERROR", [0], 0.3)
    for k in range(63):
        c.append("X_ERROR", [0], 0.01)
    rates = [1e-3, 0.01, 0.05, 0.2, 0.5, 0.8, 1.0, 0.0, 0.3, 0.02]
    for k in range(80):
        c.append("X_ERROR", [0], rates[k % len(rates)])
        if k % 20 == 19:
            c.append("H", [1]); c.append("M", [1])
    for k in range(20):
        c.append("DEPOLARIZE1", [0], 0.3)
    for k in range(20):
        c.append("DEPOLARIZE2", [0, 2], 0.6)
    c.append("M", [0])
    return c


@pytest.fixture(scope="module")
def draws():
    c = _circuit()
    ref = oracle.Program(c)
    bits = np.stack([ref.draw_grouped_bits(7, t) for t in range(SHOTS)])
    return ref, ref.channels(), bits


def _outcomes(ch, bits, c):
    s0, k = ch.sym0[c], ch.nsym[c]
    v = np.zeros(len(bits), np.int64)
    for i in range(k):
        v |= bits[:, s0 + i].astype(np.int64) << i
    return v


def test_constant_symbol_and_layout(draws):
    ref, ch, bits = draws
    assert bits[:, 0].all()
    assert (ch.type == 5).sum() == 4 and ref.num_channels == 188


def test_one_symbol_rates(draws):
    ref, ch, bits = draws
    for c in np.flatnonzero(ch.type == 0):
        p = ch.p[c]
        got = bits[:, ch.sym0[c]].mean()
        if p in (0.0, 1.0):
            assert got == p, (c, p, got)
            continue
        z = abs(got - p) / np.sqrt(p * (1 - p) / SHOTS)
        assert z < 5, (c, p, got, z)


def test_random_outcomes_are_fair_and_independent(draws):
    ref, ch, bits = draws
    rnd = np.flatnonzero(ch.type == 5)
    cols = bits[:, ch.sym0[rnd]].astype(np.float64)
    for j in range(len(rnd)):
        assert abs(cols[:, j].mean() - 0.5) / np.sqrt(0.25 / SHOTS) < 5
        for k in range(j + 1, len(rnd)):
            both = (cols[:, j] * cols[:, k]).mean()
            assert abs(both - 0.25) / np.sqrt(0.25 * 0.75 / SHOTS) < 5


@pytest.mark.parametrize("kind,m", [(3, 3), (4, 15)])
def test_depolarizing_outcome_frequencies(draws, kind, m):
    ref, ch, bits = draws
    counts = np.zeros(m + 1)
    n = 0
    for c in np.flatnonzero(ch.type == kind):
        v = _outcomes(ch, bits, c)
        counts += np.bincount(v, minlength=m + 1)
        n += len(v)
    p = ch.p[np.flatnonzero(ch.type == kind)[0]]
    want = np.array([1 - p] + [p / m] * m) * n
    chi2 = ((counts - want) ** 2 / want).sum()
    assert stats.chi2.sf(chi2, m) > 1e-4, (counts, want)


def _groups(ch):
    fault = np.flatnonzero(ch.type != 5)
    return [fault[i:i + 32] for i in range(0, len(fault), 32)]


def _fired(ch, bits, c):
    return _outcomes(ch, bits, c) != 0


def test_fired_per_group_is_poisson_binomial(draws):
    """The number of channels fired in a group has the law of a sum of
    independent Bernoulli(p_i): compared by chi-square over its values."""
    ref, ch, bits = draws
    for grp in _groups(ch):
        pmf = np.array([1.0])
        for c in grp:
            p = ch.p[c]
            pmf = np.convolve(pmf, [1 - p, p])
        n_fired = sum(_fired(ch, bits, c).astype(np.int64) for c in grp)
        counts = np.bincount(n_fired, minlength=len(pmf)).astype(np.float64)
        want = pmf * SHOTS
        keep = want > 5
        obs = np.append(counts[keep], counts[~keep].sum())
        exp = np.append(want[keep], want[~keep].sum())
        obs, exp = obs[exp > 0], exp[exp > 0]
        chi2 = ((obs - exp) ** 2 / exp).sum()
        assert stats.chi2.sf(chi2, max(len(obs) - 1, 1)) > 1e-4, (grp[0], obs, exp)


def test_gap_to_first_fired_channel(draws):
    """Given that a group fired, its first fired channel is i with
    probability prod_{j<i}(1-p_j) p_i / (1 - prod_j (1-p_j))."""
    ref, ch, bits = draws
    for grp in _groups(ch):
        p = ch.p[grp]
        none_before = np.concatenate([[1.0], np.cumprod(1 - p)[:-1]])
        law = none_before * p / (1 - np.prod(1 - p))
        fired = np.stack([_fired(ch, bits, c) for c in grp], axis=1)
        hit = fired.any(axis=1)
        first = np.argmax(fired[hit], axis=1)
        counts = np.bincount(first, minlength=len(grp)).astype(np.float64)
        want = law * hit.sum()
        keep = want > 5
        obs = np.append(counts[keep], counts[~keep].sum())
        exp = np.append(want[keep], want[~keep].sum())
        obs, exp = obs[exp > 0], exp[exp > 0]
        chi2 = ((obs - exp) ** 2 / exp).sum()
        assert stats.chi2.sf(chi2, max(len(obs) - 1, 1)) > 1e-4, (grp[0], obs, exp)
        # and the group fires as often as one minus the chance that none does
        pg = 1 - np.prod(1 - p)
        assert abs(hit.mean() - pg) / np.sqrt(pg * (1 - pg) / SHOTS + 1e-300) < 5 or pg in (0.0, 1.0)


def test_pairs_within_a_group_are_independent(draws):
    ref, ch, bits = draws
    grp = _groups(ch)[0]
    f = {c: _fired(ch, bits, c) for c in grp if 0.05 <= ch.p[c] <= 0.8}
    keys = sorted(f)
    for a in range(len(keys)):
        for b in range(a + 1, len(keys)):
            pa, pb = ch.p[keys[a]], ch.p[keys[b]]
            both = (f[keys[a]] & f[keys[b]]).mean()
            assert abs(both - pa * pb) / np.sqrt(pa * pb * (1 - pa * pb) / SHOTS) < 5


def test_records_follow_the_grouped_draw():
    """sample_grouped evaluates Eq. sampling on the grouped draw's b."""
    from workloads import surface_code
    ref = oracle.Program(surface_code(3, 3, 0.02))
    m, d, o = ref.sample_grouped(5, 100, 40)
    for t in range(40):
        em, ed, eo = ref.evaluate(ref.draw_grouped_bits(5, 100 + t))
        np.testing.assert_array_equal(m[t], em)
        np.testing.assert_array_equal(d[t], ed)


def test_streams_differ_but_agree_in_law():
    """The two streams give different bits for the same (seed, shot) but the
    same detector rates."""
    from workloads import surface_code
    ref = oracle.Program(surface_code(3, 3, 0.02))
    _, d1, _ = ref.sample(3, 0, 4000)
    _, d2, _ = ref.sample_grouped(3, 0, 4000)
    assert not np.array_equal(d1, d2)
    r1 = oracle.unpack_records(d1, ref.num_det).mean(0)
    r2 = oracle.unpack_records(d2, ref.num_det).mean(0)
    se = np.sqrt((r1 * (1 - r1) + r2 * (1 - r2)) / 4000 + 1e-12)
    assert (np.abs(r1 - r2) / se).max() < 5
