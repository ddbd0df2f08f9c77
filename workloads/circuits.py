"""Seeded synthetic circuit workloads for the symbolic-phase sampler.

This module is the one place both the CPU oracle and the CUDA library take
their inputs from. It holds only circuit *descriptions* (which gates, faults,
measurements and detectors, in which order) and contains none of the method's
arithmetic: no tableau, no phase, no sampling.

Op vocabulary (a small Stim-like grammar written for this project):

    H a..            S a..            CX c t c t ..
    X a..  Y a..  Z a..               (deterministic Pauli gates, Fact 1)
    M a..  MR a..  R a..              (Z-basis measure / measure+reset / reset)
    X_ERROR(p) a..  Y_ERROR(p) a..  Z_ERROR(p) a..
    DEPOLARIZE1(p) a..                DEPOLARIZE2(p) a b a b ..
    DETECTOR rec[-k] ..               OBSERVABLE_INCLUDE(i) rec[-k] ..
    X_IF rec[-k] a ..  Y_IF rec[-k] a ..  Z_IF rec[-k] a ..
                                      (feed-forward: the Pauli on qubit a when
                                       record rec[-k] is 1; the conditional
                                       Paulis of Sec. 6)
    TICK

Generators:
  * ``repetition_code``   distance-d bit-flip repetition memory (X_ERROR only);
  * ``surface_code``      rotated surface-code Z-memory with circuit-level noise
                          (DEPOLARIZE1 after H, DEPOLARIZE2 after CX, X_ERROR on
                          reset and before measurement);
  * ``random_layered``    the layered random-interaction circuits of the
                          paper's benchmark section (Fig. 3 caption): n qubits,
                          n layers of random H/S/I, CNOT pairs, 5% measured.
"""
from __future__ import annotations

import dataclasses
import hashlib
import re
from typing import Iterable, List, Optional, Sequence, Tuple

import numpy as np

GATES_1Q = ("H", "S", "X", "Y", "Z")
GATES_2Q = ("CX",)
MEASURES = ("M", "MR", "R")
NOISE_1Q = ("X_ERROR", "Y_ERROR", "Z_ERROR", "DEPOLARIZE1")
NOISE_2Q = ("DEPOLARIZE2",)
ANNOTATIONS = ("DETECTOR", "OBSERVABLE_INCLUDE", "TICK")
FEEDFORWARD = ("X_IF", "Y_IF", "Z_IF")
ALL_OPS = GATES_1Q + GATES_2Q + MEASURES + NOISE_1Q + NOISE_2Q + ANNOTATIONS + FEEDFORWARD


@dataclasses.dataclass(frozen=True)
class Op:
    """One instruction. ``targets`` are qubit indices, except for DETECTOR and
    OBSERVABLE_INCLUDE where they are positive look-backs k of ``rec[-k]``,
    and X_IF/Y_IF/Z_IF where they are (k, qubit) pairs.
    ``arg`` is the probability of a noise op, the observable index of
    OBSERVABLE_INCLUDE, and 0 otherwise."""

    name: str
    targets: Tuple[int, ...]
    arg: float = 0.0


class Circuit:
    """An ordered list of ops over ``num_qubits`` qubits."""

    def __init__(self, num_qubits: int = 0, ops: Optional[Iterable[Op]] = None):
        self.ops: List[Op] = list(ops or [])
        self.num_qubits = num_qubits
        for op in self.ops:
            self._grow(op)

    def _grow(self, op: Op) -> None:
        if op.name in GATES_1Q + GATES_2Q + MEASURES + NOISE_1Q + NOISE_2Q and op.targets:
            self.num_qubits = max(self.num_qubits, max(op.targets) + 1)
        elif op.name in FEEDFORWARD and len(op.targets) >= 2:
            self.num_qubits = max(self.num_qubits, max(op.targets[1::2]) + 1)

    def append(self, name: str, targets: Sequence[int] = (), arg: float = 0.0) -> "Circuit":
        if name not in ALL_OPS:
            raise ValueError(f"unknown op {name!r}")
        op = Op(name, tuple(int(t) for t in targets), float(arg))
        self.ops.append(op)
        self._grow(op)
        return self

    # ------------------------------------------------------------------ counts
    @property
    def num_measurements(self) -> int:
        return sum(len(op.targets) for op in self.ops if op.name in ("M", "MR"))

    @property
    def num_detectors(self) -> int:
        return sum(1 for op in self.ops if op.name == "DETECTOR")

    @property
    def num_observables(self) -> int:
        idx = [int(op.arg) for op in self.ops if op.name == "OBSERVABLE_INCLUDE"]
        return (max(idx) + 1) if idx else 0

    @property
    def num_fault_channels(self) -> int:
        n = 0
        for op in self.ops:
            if op.name in NOISE_1Q:
                n += len(op.targets)
            elif op.name in NOISE_2Q:
                n += len(op.targets) // 2
        return n

    @property
    def num_fault_symbols(self) -> int:
        per = {"X_ERROR": 1, "Y_ERROR": 1, "Z_ERROR": 1, "DEPOLARIZE1": 2}
        n = 0
        for op in self.ops:
            if op.name in per:
                n += per[op.name] * len(op.targets)
            elif op.name == "DEPOLARIZE2":
                n += 4 * (len(op.targets) // 2)
        return n

    # ---------------------------------------------------------------- text I/O
    def to_text(self) -> str:
        lines = []
        for op in self.ops:
            head = op.name
            if op.name in NOISE_1Q + NOISE_2Q:
                head += f"({op.arg!r})"
            elif op.name == "OBSERVABLE_INCLUDE":
                head += f"({int(op.arg)})"
            if op.name in ("DETECTOR", "OBSERVABLE_INCLUDE"):
                tail = " ".join(f"rec[-{k}]" for k in op.targets)
            elif op.name in FEEDFORWARD:
                tail = " ".join(f"rec[-{k}] {q}" for k, q in zip(op.targets[::2], op.targets[1::2]))
            else:
                tail = " ".join(str(t) for t in op.targets)
            lines.append((head + " " + tail).rstrip())
        return "\n".join(lines) + "\n"

    @staticmethod
    def from_text(text: str) -> "Circuit":
        c = Circuit()
        pat = re.compile(r"^([A-Z_0-9]+)(?:\(([^)]*)\))?\s*(.*)$")
        for lineno, raw in enumerate(text.splitlines(), 1):
            line = raw.split("#", 1)[0].strip()
            if not line:
                continue
            m = pat.match(line)
            if not m:
                raise ValueError(f"line {lineno}: cannot parse {raw!r}")
            name, arg, rest = m.group(1), m.group(2), m.group(3).split()
            if name == "CNOT":
                name = "CX"
            if name not in ALL_OPS:
                raise ValueError(f"line {lineno}: unknown op {name!r}")
            if name in ("DETECTOR", "OBSERVABLE_INCLUDE"):
                tg = []
                for t in rest:
                    mm = re.fullmatch(r"rec\[-(\d+)\]", t)
                    if not mm:
                        raise ValueError(f"line {lineno}: bad record target {t!r}")
                    tg.append(int(mm.group(1)))
            elif name in FEEDFORWARD:
                if len(rest) % 2:
                    raise ValueError(f"line {lineno}: {name} takes rec[-k] qubit pairs")
                tg = []
                for rt, qt in zip(rest[::2], rest[1::2]):
                    mm = re.fullmatch(r"rec\[-(\d+)\]", rt)
                    if not mm:
                        raise ValueError(f"line {lineno}: bad record target {rt!r}")
                    tg += [int(mm.group(1)), int(qt)]
            else:
                tg = [int(t) for t in rest]
            c.append(name, tg, float(arg) if arg not in (None, "") else 0.0)
        return c

    def fingerprint(self) -> str:
        """sha256 of the text form; freezes a generated workload in tests."""
        return hashlib.sha256(self.to_text().encode()).hexdigest()

    def __repr__(self) -> str:
        return (f"Circuit(qubits={self.num_qubits}, ops={len(self.ops)}, "
                f"meas={self.num_measurements}, det={self.num_detectors}, "
                f"obs={self.num_observables}, channels={self.num_fault_channels})")


# ---------------------------------------------------------------------------
# Repetition code
# ---------------------------------------------------------------------------
def repetition_code(distance: int = 5, rounds: int = 5, p: float = 0.01) -> Circuit:
    """Bit-flip repetition-code memory: data qubits 0..d-1, ancillas d..2d-2
    (ancilla i checks data i and i+1). X_ERROR(p) after every reset, after
    every CNOT on both of its qubits, and before every measurement. One
    detector per ancilla per round (round 1 against the known +1), one per
    ancilla from the final data readout, and observable 0 = data qubit 0."""
    d = distance
    data = list(range(d))
    anc = list(range(d, 2 * d - 1))
    c = Circuit(2 * d - 1)
    allq = data + anc
    c.append("R", allq)
    c.append("X_ERROR", allq, p)
    for r in range(rounds):
        for layer in range(2):
            pairs = []
            for i, a in enumerate(anc):
                pairs += [data[i + layer], a]
            c.append("CX", pairs)
            c.append("X_ERROR", pairs, p)
        c.append("X_ERROR", anc, p)
        c.append("MR", anc)
        c.append("X_ERROR", anc, p)
        na = len(anc)
        for i in range(na):
            if r == 0:
                c.append("DETECTOR", [na - i])
            else:
                c.append("DETECTOR", [na - i, 2 * na - i])
    c.append("X_ERROR", data, p)
    c.append("M", data)
    na = len(anc)
    for i in range(na):
        # data i, data i+1 (just measured) and ancilla i of the last round
        c.append("DETECTOR", [d - i, d - i - 1, d + na - i])
    c.append("OBSERVABLE_INCLUDE", [d], 0)
    return c


# ---------------------------------------------------------------------------
# Rotated surface code, Z memory
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class _Plaquette:
    kind: str                     # "X" or "Z"
    corners: List[Optional[int]]  # data indices for NW, NE, SW, SE (None = absent)
    ancilla: int = -1


def _rotated_layout(d: int) -> List[_Plaquette]:
    """Plaquettes of the rotated distance-d code on a d x d data grid.

    Plaquette (i, j), i, j in -1..d-1, has corners (i, j), (i, j+1), (i+1, j),
    (i+1, j+1) clipped to the grid, and type X when i + j is even, Z when odd.
    All interior plaquettes are kept; weight-2 plaquettes are kept on the top
    and bottom edges when X-type and on the left and right edges when Z-type,
    which gives d^2 - 1 independent checks."""
    def q(a, b):
        return a * d + b if 0 <= a < d and 0 <= b < d else None

    out = []
    for i in range(-1, d):
        for j in range(-1, d):
            kind = "X" if (i + j) % 2 == 0 else "Z"
            corners = [q(i, j), q(i, j + 1), q(i + 1, j), q(i + 1, j + 1)]
            present = sum(x is not None for x in corners)
            interior = 0 <= i <= d - 2 and 0 <= j <= d - 2
            if interior:
                out.append(_Plaquette(kind, corners))
            elif present == 2:
                top_bottom = i in (-1, d - 1) and 0 <= j <= d - 2
                left_right = j in (-1, d - 1) and 0 <= i <= d - 2
                if (top_bottom and kind == "X") or (left_right and kind == "Z"):
                    out.append(_Plaquette(kind, corners))
    for k, pl in enumerate(out):
        pl.ancilla = d * d + k
    return out


def surface_code(distance: int = 11, rounds: Optional[int] = None, p: float = 1e-3) -> Circuit:
    """Rotated surface-code Z-memory with circuit-level noise.

    Qubits: data d*d (row-major), then one ancilla per plaquette. Each round:
    H on X-ancillas (+DEPOLARIZE1), four CX layers in the hook-avoiding order
    (X checks NW, NE, SW, SE with the ancilla as control; Z checks NW, SW, NE,
    SE with the ancilla as target), each CX followed by DEPOLARIZE2, H on
    X-ancillas (+DEPOLARIZE1), X_ERROR before the ancilla measurement, MR,
    X_ERROR after the reset. Detectors: Z checks in round 1, every check in
    later rounds (XOR with the previous round), and every Z check against the
    final data readout. Observable 0 is the Z parity of data row 0."""
    d = distance
    rounds = d if rounds is None else rounds
    plaq = _rotated_layout(d)
    nd = d * d
    anc = [pl.ancilla for pl in plaq]
    xanc = [pl.ancilla for pl in plaq if pl.kind == "X"]
    c = Circuit(nd + len(anc))
    allq = list(range(nd)) + anc
    c.append("R", allq)
    c.append("X_ERROR", allq, p)
    order = {"X": (0, 1, 2, 3), "Z": (0, 2, 1, 3)}
    na = len(anc)
    pos = {a: k for k, a in enumerate(anc)}
    for r in range(rounds):
        c.append("TICK")
        c.append("H", xanc)
        c.append("DEPOLARIZE1", xanc, p)
        for layer in range(4):
            pairs = []
            for pl in plaq:
                dq = pl.corners[order[pl.kind][layer]]
                if dq is None:
                    continue
                pairs += [pl.ancilla, dq] if pl.kind == "X" else [dq, pl.ancilla]
            c.append("CX", pairs)
            c.append("DEPOLARIZE2", pairs, p)
        c.append("H", xanc)
        c.append("DEPOLARIZE1", xanc, p)
        c.append("X_ERROR", anc, p)
        c.append("MR", anc)
        c.append("X_ERROR", anc, p)
        for pl in plaq:
            k = na - pos[pl.ancilla]
            if r == 0:
                if pl.kind == "Z":
                    c.append("DETECTOR", [k])
            else:
                c.append("DETECTOR", [k, k + na])
    c.append("X_ERROR", list(range(nd)), p)
    c.append("M", list(range(nd)))
    for pl in plaq:
        if pl.kind != "Z":
            continue
        lb = [nd - dq for dq in pl.corners if dq is not None]
        lb.append(nd + na - pos[pl.ancilla])
        c.append("DETECTOR", lb)
    c.append("OBSERVABLE_INCLUDE", [nd - b for b in range(d)], 0)
    return c


def surface_code_all_channels(distance: int = 3, rounds: Optional[int] = None, p: float = 1e-3) -> Circuit:
    """``surface_code`` with every channel kind reaching the detectors: at the
    start of each round, after the X-ancillas' H and DEPOLARIZE1, a Y_ERROR(p)
    on every data qubit and a Z_ERROR(p) on every X-ancilla (in |+>, where a
    Z flips its outcome), next to the DEPOLARIZE1, DEPOLARIZE2 and X_ERROR
    channels of the base circuit."""
    base = surface_code(distance, rounds, p)
    nd = distance * distance
    out = Circuit(base.num_qubits)
    after_tick = False
    for op in base.ops:
        out.append(op.name, op.targets, op.arg)
        if op.name == "TICK":
            after_tick = True
        elif op.name == "DEPOLARIZE1" and after_tick:
            out.append("Y_ERROR", list(range(nd)), p)
            out.append("Z_ERROR", list(op.targets), p)
            after_tick = False
    return out


# ---------------------------------------------------------------------------
# Random layered circuits (the paper's Fig. 3 benchmark family)
# ---------------------------------------------------------------------------
def random_layered(n: int, layers: Optional[int] = None, cnot_pairs: Optional[int] = None,
                   depolarize: float = 0.0, measure_fraction: float = 0.05,
                   seed: int = 0) -> Circuit:
    """n qubits, ``layers`` (default n) layers; each layer applies H, S or
    nothing to every qubit at random, then ``cnot_pairs`` random disjoint CX
    pairs (default floor(n/2)), then optionally DEPOLARIZE1(depolarize) on
    every qubit, then measures a random 5% of the qubits; finally every qubit
    is measured (Fig. 3 caption, benchmark section)."""
    rng = np.random.default_rng(seed)
    layers = n if layers is None else layers
    pairs = n // 2 if cnot_pairs is None else cnot_pairs
    c = Circuit(n)
    nmeas = max(1, int(round(measure_fraction * n)))
    for _ in range(layers):
        choice = rng.integers(0, 3, size=n)
        h = [q for q in range(n) if choice[q] == 0]
        s = [q for q in range(n) if choice[q] == 1]
        if h:
            c.append("H", h)
        if s:
            c.append("S", s)
        perm = rng.permutation(n)[: 2 * pairs]
        c.append("CX", [int(x) for x in perm])
        if depolarize > 0:
            c.append("DEPOLARIZE1", list(range(n)), depolarize)
        mq = sorted(int(x) for x in rng.choice(n, size=nmeas, replace=False))
        c.append("M", mq)
    c.append("M", list(range(n)))
    return c


def mirror_circuit(n: int, layers: int, p: float = 0.01, seed: int = 0) -> Circuit:
    """``layers`` random Clifford layers (H or S or nothing on every qubit,
    then floor(n/2) random disjoint CX pairs) followed by their inverse in
    reverse order, DEPOLARIZE1(p) on every qubit after every layer, then
    every qubit measured, with one detector per measurement (its noiseless
    value is 0).  Every outcome is deterministic and, once the light cones
    have spread, depends on faults all through the circuit: the coefficient
    rows are dense, the regime where the product is a real contraction."""
    rng = np.random.default_rng(seed)
    c = Circuit(n)
    fwd = []
    for _ in range(layers):
        choice = rng.integers(0, 3, size=n)
        h = [q for q in range(n) if choice[q] == 0]
        s_ = [q for q in range(n) if choice[q] == 1]
        pairs = [int(x) for x in rng.permutation(n)[: 2 * (n // 2)]]
        fwd.append((h, s_, pairs))
        if h:
            c.append("H", h)
        if s_:
            c.append("S", s_)
        c.append("CX", pairs)
        if p > 0:
            c.append("DEPOLARIZE1", list(range(n)), p)
    for h, s_, pairs in reversed(fwd):
        # inverse layer: CX pairs (self-inverse), then S^-1 = S^3, then H
        rev = [x for k in range(len(pairs) // 2 - 1, -1, -1) for x in pairs[2 * k: 2 * k + 2]]
        c.append("CX", rev)
        if s_:
            for _ in range(3):
                c.append("S", s_)
        if h:
            c.append("H", h)
        if p > 0:
            c.append("DEPOLARIZE1", list(range(n)), p)
    c.append("M", list(range(n)))
    for q in range(n):
        c.append("DETECTOR", [n - q])
    return c


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------
def batch_suite(count: int = 64) -> List[Tuple[Circuit, int]]:
    """Uneven batch: circuit i is a rotated surface code with d = 3 + 2*(i mod 7),
    rounds = d, p = (5e-4, 1e-3, 2e-3)[(i // 7) mod 3], seed i."""
    ps = (5e-4, 1e-3, 2e-3)
    out = []
    for i in range(count):
        d = 3 + 2 * (i % 7)
        out.append((surface_code(d, d, ps[(i // 7) % 3]), i))
    return out


def perturbed_probabilities(base: np.ndarray, seed: int = 1, rel: float = 0.2) -> np.ndarray:
    """p' = p * (1 + delta), delta ~ U(-rel, rel), seeded (the fitting target)."""
    rng = np.random.default_rng(seed)
    return base * (1.0 + rng.uniform(-rel, rel, size=base.shape))


def channel_probabilities(n_channels: int, lo: float = 5e-4, hi: float = 2e-3, seed: int = 0) -> np.ndarray:
    """Per-channel probabilities p_i ~ U(lo, hi), seeded."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=n_channels)


def with_channel_probabilities(circuit: Circuit, p: Sequence[float]) -> Circuit:
    """The same circuit with fault channel c (in op order: one per target of
    a one-qubit noise op, one per pair of DEPOLARIZE2) at probability p[c]:
    each noise op is split into one op per channel."""
    p = np.asarray(p, dtype=np.float64)
    if len(p) != circuit.num_fault_channels:
        raise ValueError(f"{len(p)} probabilities for {circuit.num_fault_channels} fault channels")
    out = Circuit(circuit.num_qubits)
    c = 0
    for op in circuit.ops:
        if op.name in NOISE_1Q:
            for t in op.targets:
                out.append(op.name, [t], float(p[c]))
                c += 1
        elif op.name in NOISE_2Q:
            for a, b in zip(op.targets[::2], op.targets[1::2]):
                out.append(op.name, [a, b], float(p[c]))
                c += 1
        else:
            out.append(op.name, op.targets, op.arg)
    return out


def random_clifford_circuit(num_qubits: int, num_ops: int, seed: int, p_noise: float = 0.2) -> Circuit:
    """Clifford-heavy random circuits: mostly H, S and CX (building Y
    components and long products of stabilizers), some faults, rare
    mid-circuit measurements, and a final measurement of every qubit."""
    rng = np.random.default_rng(seed)
    c = Circuit(num_qubits)
    kinds = ["H", "S", "CX", "X_ERROR", "DEPOLARIZE1", "DEPOLARIZE2", "M"]
    probs = [0.3, 0.3, 0.25, 0.04, 0.04, 0.03, 0.04]
    for _ in range(num_ops):
        k = kinds[rng.choice(len(kinds), p=probs)]
        if k in ("CX", "DEPOLARIZE2"):
            if num_qubits < 2:
                continue
            a, b = rng.choice(num_qubits, size=2, replace=False)
            c.append(k, [int(a), int(b)], p_noise if k == "DEPOLARIZE2" else 0.0)
        else:
            c.append(k, [int(rng.integers(num_qubits))], p_noise if k in NOISE_1Q else 0.0)
    c.append("M", list(range(num_qubits)))
    return c


def random_small_circuit(num_qubits: int, num_ops: int, seed: int, p_noise: float = 0.2,
                         allow_reset: bool = True) -> Circuit:
    """Small random circuits over the whole op vocabulary for cross-checks:
    Clifford gates, Pauli gates, every noise channel, M, MR and R."""
    rng = np.random.default_rng(seed)
    c = Circuit(num_qubits)
    kinds = ["H", "S", "CX", "X", "Y", "Z", "M", "X_ERROR", "Y_ERROR", "Z_ERROR",
             "DEPOLARIZE1", "DEPOLARIZE2"] + (["MR", "R"] if allow_reset else [])
    for _ in range(num_ops):
        k = kinds[rng.integers(len(kinds))]
        if k in ("CX", "DEPOLARIZE2"):
            if num_qubits < 2:
                continue
            a, b = rng.choice(num_qubits, size=2, replace=False)
            c.append(k, [int(a), int(b)], p_noise if k == "DEPOLARIZE2" else 0.0)
        else:
            q = int(rng.integers(num_qubits))
            c.append(k, [q], p_noise if k in NOISE_1Q else 0.0)
    c.append("M", list(range(num_qubits)))
    return c


def random_feedforward_circuit(num_qubits: int, num_ops: int, seed: int, p_noise: float = 0.2) -> Circuit:
    """Small random circuits with feed-forward: the vocabulary of
    ``random_small_circuit`` plus X_IF / Y_IF / Z_IF on a random qubit,
    conditioned on a random earlier record (rec[-k], k up to 6), and a
    teleportation-style correction after some measurements (X_IF rec[-1] on
    another qubit)."""
    rng = np.random.default_rng(seed)
    c = Circuit(num_qubits)
    kinds = ["H", "S", "CX", "X", "Y", "Z", "M", "MR", "R", "X_ERROR", "Y_ERROR", "Z_ERROR",
             "DEPOLARIZE1", "DEPOLARIZE2", "X_IF", "Y_IF", "Z_IF"]
    nrec = 0
    for _ in range(num_ops):
        k = kinds[rng.integers(len(kinds))]
        if k in ("CX", "DEPOLARIZE2"):
            if num_qubits < 2:
                continue
            a, b = rng.choice(num_qubits, size=2, replace=False)
            c.append(k, [int(a), int(b)], p_noise if k == "DEPOLARIZE2" else 0.0)
        elif k in FEEDFORWARD:
            if nrec == 0:
                continue
            back = int(rng.integers(1, min(nrec, 6) + 1))
            c.append(k, [back, int(rng.integers(num_qubits))])
        else:
            q = int(rng.integers(num_qubits))
            c.append(k, [q], p_noise if k in NOISE_1Q else 0.0)
            if k in ("M", "MR"):
                nrec += 1
                if num_qubits > 1 and rng.random() < 0.3:
                    c.append("X_IF", [1, int((q + 1 + rng.integers(num_qubits - 1)) % num_qubits)])
    c.append("M", list(range(num_qubits)))
    return c
