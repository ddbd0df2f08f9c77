"""Parser for the text fixtures under tests/golden/ (paper worked examples)."""
from __future__ import annotations

import os
import re

import numpy as np

from workloads import Circuit

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _expr(s: str, nsym: int) -> np.ndarray:
    """'s1 + s3' / '0' -> 0/1 vector over symbols 0..nsym (0 = constant)."""
    v = np.zeros(nsym + 1, np.uint8)
    s = s.strip()
    if s in ("0", ""):
        return v
    for term in s.split("+"):
        term = term.strip()
        if term == "1":
            v[0] ^= 1
        else:
            m = re.fullmatch(r"s(\d+)", term)
            assert m, term
            v[int(m.group(1))] ^= 1
    return v


def load(name: str, nsym: int):
    """-> (circuit, outcomes{index: vector}, tables{(kind, after): rows})"""
    text = open(os.path.join(GOLDEN, name)).read()
    sections, cur = {}, None
    for raw in text.splitlines():
        line = raw.split("#", 1)[0].rstrip()
        if not line.strip():
            continue
        m = re.fullmatch(r"\[(.+)\]", line.strip())
        if m:
            cur = m.group(1)
            sections[cur] = []
            continue
        sections[cur].append(line)
    circuit = Circuit.from_text("\n".join(sections.pop("circuit")))
    outcomes = {}
    for line in sections.pop("outcomes"):
        lhs, rhs = line.split("=")
        outcomes[int(lhs.strip()[1:]) - 1] = _expr(rhs, nsym)
    tables = {}
    for key, lines in sections.items():
        kind, _, after = key.split()
        rows = []
        for line in lines:
            xs, zs, ph = (p.strip() for p in line.split("|"))
            rows.append((np.array([int(c) for c in xs], np.uint8),
                         np.array([int(c) for c in zs], np.uint8), _expr(ph, nsym)))
        tables[(kind, int(after))] = rows
    return circuit, outcomes, tables
