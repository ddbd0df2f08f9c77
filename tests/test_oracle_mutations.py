"""The pins are strong enough: each plausible mistake planted in a copy of
the oracle (compiled to a temporary library, CPU only) makes at least one
pin test fail. The real oracle is never modified."""
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "symphase_oracle.c")
PINS = ["test_oracle_golden.py", "test_oracle_chp.py", "test_oracle_statevec.py",
        "test_oracle_philox.py", "test_oracle_expect.py", "test_oracle_grouped.py"]

MUTANTS = {
    "cx-phase-rule": ("if (x[a] & z[b] & (x[b] ^ z[a] ^ 1)) flipb(PH(P, r), 0);",
                      "if (x[a] & z[b] & (x[b] ^ z[a])) flipb(PH(P, r), 0);"),
    "h-no-phase": ("        if (x[a] & z[a]) flipb(PH(P, r), 0);\n        uint8_t t = x[a]; x[a] = z[a]; z[a] = t;",
                   "        uint8_t t = x[a]; x[a] = z[a]; z[a] = t;"),
    "g-function-sign": ("if (x1 && !z1) return z2 * (2 * x2 - 1);", "if (x1 && !z1) return z2 * (1 - 2 * x2);"),
    "random-outcome-literal-reading": ("        memset(PH(P, p), 0, (size_t)P->pw * 8);\n        flipb(PH(P, p), s);",
                                       "        memset(PH(P, p), 0, (size_t)P->pw * 8);\n        pauli_column(P, a, 1, 0, s);"),
    "rowsum-skips-symbols": ("    for (int64_t w = 0; w < P->pw; w++) ph[w] ^= pi[w];\n    /* column 0",
                             "    for (int64_t w = 0; w < P->pw; w++) ph[w] ^= pi[w] & 1u;\n    /* column 0"),
    "dep1-symbol-order": ("                pauli_column(P, t[j], 1, 0, s);     /* X^{s}   */\n                pauli_column(P, t[j], 0, 1, s + 1); /* Z^{s+1} */",
                          "                pauli_column(P, t[j], 1, 0, s + 1);\n                pauli_column(P, t[j], 0, 1, s);"),
    "philox-weyl-constant": ("W1 = 0xBB67AE85u;", "W1 = 0xBB67AE86u;"),
    "threshold-ceil": ("double t = floor(p * 4294967296.0);", "double t = ceil(p * 4294967296.0);"),
    "dep2-categorical": ("(((uint64_t)u * 15u) / T) + 1u;", "(((uint64_t)u * 14u) / T) + 1u;"),
    "expect-kappa": ("for (int v = 1; v <= m; v++) odd +=", "for (int v = 1; v < m; v++) odd +="),
    "vjp-sign": ("grad_p[c] += g[j] * (-2.0 * dP / f);", "grad_p[c] += g[j] * (2.0 * dP / f);"),
    "deterministic-row-set": ("            if (X(P, i)[a]) rowsum(P, sc, i + n);", "            if (Z(P, i)[a]) rowsum(P, sc, i + n);"),
    "reset-row-set": ("if (c != OR_M) cond_pauli(P, t[j], 1, 0, e);", "if (c != OR_M) cond_pauli(P, t[j], 0, 1, e);"),
    "conditional-pauli-rows": ("if ((xb && Z(P, r)[a]) ^ (zb && X(P, r)[a])) {", "if ((xb && X(P, r)[a]) ^ (zb && Z(P, r)[a])) {"),
    "feedforward-lookback": ("P->meas + (P->nmeas - lb) * P->pw);", "P->meas + (P->nmeas - lb + 1) * P->pw);"),
    "feedforward-y-as-x": ("cond_pauli(P, t[j + 1], c != OR_ZIF, c != OR_XIF,", "cond_pauli(P, t[j + 1], c != OR_ZIF, c == OR_ZIF,"),
    "grouped-first-unconditioned": ("U = i == last ? 4294967295u : or_threshold(P->ch_p[c] / (1.0 - R[i]));",
                                    "U = i == last ? 4294967295u : or_threshold(P->ch_p[c]);"),
    "grouped-group-threshold": ("uint32_t G = or_threshold(1.0 - R[0]);", "uint32_t G = or_threshold(1.0 - R[1]);"),
    "grouped-after-threshold": ("                U = P->ch_T[c];\n", "                U = or_threshold(P->ch_p[c] / (1.0 - R[i]));\n"),
    "grouped-random-bit": ("if ((w >> (r % 32)) & 1u)", "if ((w >> (r % 2)) & 1u)"),
    "grouped-dep-category": ("uint64_t m = type == CH_DEP1 ? 3u : 15u;", "uint64_t m = type == CH_DEP1 ? 3u : 14u;"),
    "grouped-channel-counter": ("(uint32_t)(8 * g + i / 4), 2u", "(uint32_t)(8 * g + i / 8), 2u"),
    "counter-layout": ("uint32_t ctr[4] = {(uint32_t)shot, (uint32_t)(shot >> 32), (uint32_t)(c / 4), 0u};",
                       "uint32_t ctr[4] = {(uint32_t)shot, (uint32_t)(c / 4), (uint32_t)(shot >> 32), 0u};"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    mutant = tmp_path / "mutant.c"
    mutant.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", str(lib), str(mutant), "-lm"])
    env = dict(os.environ, SYMPHASE_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider"] +
                       [os.path.join(HERE, f) for f in PINS], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"no pin caught the planted mistake {name!r}:\n{r.stdout[-2000:]}"
