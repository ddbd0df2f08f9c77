"""Pins of the oracle's analytic expectations E_j = E[(-1)^{D_j}]:
  * closed form (-1)^{c_j} prod_{s in supp} (1 - 2 p_s) for independent
    single-symbol channels;
  * brute-force enumeration of every joint channel outcome on tiny circuits
    (DEPOLARIZE1/2 included);
  * central finite differences of log|E| for the gradient;
  * Monte-Carlo detector rates of the oracle's own sampler within 5 sigma;
  * the noiseless special case and the repetition code's textbook
    graph-like structure (every fault flips at most two detectors)."""
import itertools

import numpy as np
import pytest

import oracle
from workloads import Circuit, random_small_circuit, repetition_code, surface_code


def test_closed_form_independent_symbols():
    c = repetition_code(5, 5, 0.03)
    prog = oracle.Program(c)
    ch = prog.channels()
    p_sym = np.zeros(prog.num_symbols + 1)
    p_sym[ch.sym0] = ch.p
    rows = prog.row_bits("det")
    la, sg = prog.expect()
    for j in range(prog.num_det):
        supp = np.nonzero(rows[j, 1:])[0] + 1
        want = np.prod(1 - 2 * p_sym[supp]) * (-1.0) ** int(rows[j, 0])
        assert abs(np.exp(la[j]) * sg[j] - want) < 1e-12 * max(1, abs(want))


def _brute_expectation(prog, p):
    """E_j by summing over every joint outcome of every channel."""
    ch = prog.channels()
    rows = np.vstack([prog.row_bits("det"), prog.row_bits("obs")]).astype(np.int64)
    outs = []
    for c in range(prog.num_channels):
        m = {0: 1, 1: 1, 2: 1, 3: 3, 4: 15, 5: 1}[int(ch.type[c])]
        pc = 0.5 if ch.type[c] == 5 else p[c]
        outs.append([(0, 1 - pc)] + [(v, pc / m) for v in range(1, m + 1)])
    E = np.zeros(rows.shape[0])
    for combo in itertools.product(*outs):
        b = np.zeros(prog.num_symbols + 1, np.int64)
        b[0] = 1
        w = 1.0
        for c, (v, pv) in enumerate(combo):
            w *= pv
            for i in range(ch.nsym[c]):
                b[ch.sym0[c] + i] = (v >> i) & 1
        E += w * (-1.0) ** ((rows @ b) % 2)
    return E


@pytest.mark.parametrize("seed", range(6))
def test_brute_force_enumeration(seed):
    rng = np.random.default_rng(seed)
    c = Circuit(3)
    c.append("CX", [0, 1])
    c.append("DEPOLARIZE2", [0, 1], 0.3)
    c.append("DEPOLARIZE1", [2], 0.2)
    c.append("CX", [1, 2]); c.append("X_ERROR", [0], 0.1)
    c.append("H", [2]); c.append("Z_ERROR", [2], 0.05); c.append("H", [2])
    c.append("Y_ERROR", [1], 0.15)
    c.append("CX", [0, 1])
    c.append("M", [0, 1, 2])
    c.append("DETECTOR", [3]); c.append("DETECTOR", [2]); c.append("DETECTOR", [1, 2])
    c.append("OBSERVABLE_INCLUDE", [3, 1], 0)
    prog = oracle.Program(c)
    p = rng.uniform(0.01, 0.4, prog.num_channels)
    la, sg = prog.expect(p)
    E = _brute_expectation(prog, p)
    np.testing.assert_allclose(np.exp(la) * sg, E, rtol=1e-12, atol=1e-14)


def test_gradient_matches_central_differences():
    prog = oracle.Program(surface_code(3, 3, 1e-3))
    rng = np.random.default_rng(7)
    p = rng.uniform(5e-4, 2e-3, prog.num_channels)
    g = rng.normal(size=prog.num_det + prog.num_obs)
    grad = prog.expect_vjp(p, g)
    h = 1e-6
    for c in rng.choice(prog.num_channels, size=64, replace=False):
        pp, pm = p.copy(), p.copy()
        pp[c] += h
        pm[c] -= h
        fd = (prog.expect(pp)[0] @ g - prog.expect(pm)[0] @ g) / (2 * h)
        assert abs(fd - grad[c]) <= 1e-6 * max(1.0, abs(grad[c])), (c, fd, grad[c])


def test_monte_carlo_rates_within_5_sigma():
    prog = oracle.Program(surface_code(3, 3, 0.02))
    n = 20000
    _, d, o = prog.sample(seed=3, shot0=0, nshots=n)
    rates = oracle.unpack_records(d, prog.num_det).mean(axis=0)
    la, sg = prog.expect()
    r = (1 - np.exp(la[: prog.num_det]) * sg[: prog.num_det]) / 2
    sigma = np.sqrt(np.maximum(r * (1 - r), 1e-12) / n)
    z = np.abs(rates - r) / sigma
    assert z.max() < 5.0, z.max()


def test_noiseless_is_deterministic():
    prog = oracle.Program(surface_code(3, 3, 0.0))
    la, sg = prog.expect()
    assert np.all(la == 0) and np.all(sg == 1)


def test_repetition_code_is_graphlike():
    """X errors in a repetition code flip at most two detectors each, and an
    X error on a data qubit right before its final readout flips exactly the
    final-round checks that contain that qubit (and the observable iff it is
    data qubit 0)."""
    d = 5
    c = repetition_code(d, 5, 0.01)
    prog = oracle.Program(c)
    det = prog.row_bits("det")
    obs = prog.row_bits("obs")
    assert det[:, 1:].sum(axis=0).max() <= 2
    ch = prog.channels()
    # the last d fault channels are the pre-readout X_ERRORs on data 0..d-1
    final_checks = det[-(d - 1):]
    for q in range(d):
        s = int(ch.sym0[prog.num_channels - d + q])
        flips = set(np.nonzero(final_checks[:, s])[0].tolist())
        want = {i for i in (q - 1, q) if 0 <= i < d - 1}
        assert flips == want, (q, flips)
        assert obs[0, s] == (1 if q == 0 else 0)
