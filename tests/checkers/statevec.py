"""Dense state-vector simulator (<= ~12 qubits) used only to pin the oracle.

For a fixed assignment of the fault bits it returns the exact probability
distribution over the measurement-record vectors, branching at every
measurement. The symbolic forms, evaluated over all assignments of the
random-measurement symbols (each equally likely), must give the same
distribution."""
from __future__ import annotations

from collections import defaultdict

import numpy as np

_H = np.array([[1, 1], [1, -1]], dtype=complex) / np.sqrt(2)
_S = np.array([[1, 0], [0, 1j]], dtype=complex)
_X = np.array([[0, 1], [1, 0]], dtype=complex)
_Y = np.array([[0, -1j], [1j, 0]], dtype=complex)
_Z = np.array([[1, 0], [0, -1]], dtype=complex)


def _apply1(psi, n, a, U):
    t = psi.reshape((2,) * n)
    t = np.moveaxis(np.tensordot(U, t, axes=([1], [n - 1 - a])), 0, n - 1 - a)
    return t.reshape(-1)


def _apply_cx(psi, n, c, t):
    idx = np.arange(1 << n)
    src = np.where((idx >> c) & 1, idx ^ (1 << t), idx)
    return psi[src]


def _project(psi, n, a, v):
    idx = np.arange(1 << n)
    out = np.where(((idx >> a) & 1) == v, psi, 0)
    pr = float(np.vdot(out, out).real)
    return out, pr


def distribution(circuit, fault_bits) -> dict:
    """{tuple(meas records): probability} for one fixed assignment of the
    fault symbols (fault_bits[s] for fault symbol s, numbered in op order
    counting only faults here; random measurements take no symbol)."""
    n = circuit.num_qubits
    psi = np.zeros(1 << n, dtype=complex)
    psi[0] = 1.0
    branches = [(psi, 1.0, ())]
    k = 0

    def take(m):
        nonlocal k
        out = [int(fault_bits[k + i]) for i in range(m)]
        k += m
        return out

    def each(fn):
        return [(fn(p), pr, rec) for p, pr, rec in branches]

    for op in circuit.ops:
        t, name = op.targets, op.name
        if name in ("H", "S", "X", "Y", "Z"):
            U = {"H": _H, "S": _S, "X": _X, "Y": _Y, "Z": _Z}[name]
            for a in t:
                branches = each(lambda p, a=a: _apply1(p, n, a, U))
        elif name == "CX":
            for a, b in zip(t[::2], t[1::2]):
                branches = each(lambda p, a=a, b=b: _apply_cx(p, n, a, b))
        elif name in ("X_ERROR", "Y_ERROR", "Z_ERROR"):
            U = {"X_ERROR": _X, "Y_ERROR": _Y, "Z_ERROR": _Z}[name]
            for a in t:
                if take(1)[0]:
                    branches = each(lambda p, a=a: _apply1(p, n, a, U))
        elif name == "DEPOLARIZE1":
            for a in t:
                vx, vz = take(2)
                if vz:
                    branches = each(lambda p, a=a: _apply1(p, n, a, _Z))
                if vx:
                    branches = each(lambda p, a=a: _apply1(p, n, a, _X))
        elif name == "DEPOLARIZE2":
            for a, b in zip(t[::2], t[1::2]):
                xa, za, xb, zb = take(4)
                for q, vx, vz in ((a, xa, za), (b, xb, zb)):
                    if vz:
                        branches = each(lambda p, q=q: _apply1(p, n, q, _Z))
                    if vx:
                        branches = each(lambda p, q=q: _apply1(p, n, q, _X))
        elif name in ("X_IF", "Y_IF", "Z_IF"):
            U = {"X_IF": _X, "Y_IF": _Y, "Z_IF": _Z}[name]
            for lb, a in zip(t[::2], t[1::2]):
                branches = [(_apply1(p, n, a, U) if rec[-lb] else p, pr, rec) for p, pr, rec in branches]
        elif name in ("M", "MR", "R"):
            for a in t:
                nb = []
                for p, pr, rec in branches:
                    for v in (0, 1):
                        q, w = _project(p, n, a, v)
                        if w < 1e-12:
                            continue
                        q = q / np.sqrt(w)
                        if name != "M" and v:
                            q = _apply1(q, n, a, _X)
                        nb.append((q, pr * w, rec + ((v,) if name != "R" else ())))
                branches = nb
        elif name in ("DETECTOR", "OBSERVABLE_INCLUDE", "TICK"):
            pass
        else:
            raise ValueError(name)
    dist = defaultdict(float)
    for _, pr, rec in branches:
        dist[rec] += pr
    return dict(dist)
