"""Concrete (non-symbolic) CHP-style stabilizer simulator, written
independently of the oracle, used only to pin it.

One shot is simulated with every fault symbol and every random-measurement
symbol given a concrete bit: a fault applies its Pauli when its bits say so,
and a random measurement takes the value of its symbol as its outcome. By
Fact 2 the sequence of random/deterministic branches is the same as in the
symbolic run, so the records must equal the symbolic forms evaluated at the
same bits.

Rows are kept as boolean numpy arrays; the phase of a product of Paulis is
computed from the power of i that the product collects, via a lookup table
over the (left, right) single-qubit Pauli pairs."""
from __future__ import annotations

import numpy as np

# power of i collected by P_left * P_right for single-qubit Paulis encoded
# as 2*x + z  (0 = I, 1 = Z, 2 = X, 3 = Y)
_I_POWER = np.zeros((4, 4), dtype=np.int64)
for _l, _r, _k in [(2, 3, 1), (3, 1, 1), (1, 2, 1), (3, 2, -1), (1, 3, -1), (2, 1, -1)]:
    _I_POWER[_l, _r] = _k


def _product_phase(xl, zl, xr, zr) -> int:
    """sum over qubits of the i-power of left * right (integer)."""
    return int(_I_POWER[2 * xl.astype(np.int64) + zl, 2 * xr.astype(np.int64) + zr].sum())


class CHPState:
    def __init__(self, n: int):
        self.n = n
        self.x = np.zeros((2 * n, n), dtype=bool)
        self.z = np.zeros((2 * n, n), dtype=bool)
        self.r = np.zeros(2 * n, dtype=bool)
        for i in range(n):
            self.x[i, i] = True          # destabilizer X_i
            self.z[n + i, i] = True      # stabilizer Z_i

    # gates -----------------------------------------------------------------
    def h(self, a):
        self.r ^= self.x[:, a] & self.z[:, a]
        self.x[:, a], self.z[:, a] = self.z[:, a].copy(), self.x[:, a].copy()

    def s(self, a):
        self.r ^= self.x[:, a] & self.z[:, a]
        self.z[:, a] ^= self.x[:, a]

    def cx(self, a, b):
        self.r ^= self.x[:, a] & self.z[:, b] & ~(self.x[:, b] ^ self.z[:, a])
        self.x[:, b] ^= self.x[:, a]
        self.z[:, a] ^= self.z[:, b]

    def pauli(self, a, px: bool, pz: bool):
        self.r ^= (px & self.z[:, a]) ^ (pz & self.x[:, a])

    # row algebra -------------------------------------------------------------
    def _mul_into(self, h, i):
        """row h := row i * row h, with the sign from the i-power."""
        k = 2 * int(self.r[h]) + 2 * int(self.r[i]) + _product_phase(self.x[i], self.z[i], self.x[h], self.z[h])
        self.r[h] = (k % 4) == 2
        self.x[h] ^= self.x[i]
        self.z[h] ^= self.z[i]

    def is_random(self, a) -> bool:
        return bool(self.x[self.n:, a].any())

    def measure(self, a, forced_outcome: int) -> int:
        n = self.n
        stab_hits = np.nonzero(self.x[n:, a])[0]
        if len(stab_hits):
            p = n + int(stab_hits[0])
            for i in np.nonzero(self.x[:, a])[0]:
                if i != p:
                    self._mul_into(int(i), p)
            self.x[p - n], self.z[p - n], self.r[p - n] = self.x[p].copy(), self.z[p].copy(), self.r[p]
            self.x[p] = False
            self.z[p] = False
            self.z[p, a] = True
            self.r[p] = bool(forced_outcome)
            return int(forced_outcome)
        # deterministic: multiply the stabilizers paired with the
        # destabilizers that have an X on qubit a
        sx = np.zeros(n, bool); sz = np.zeros(n, bool); sk = 0
        for i in np.nonzero(self.x[:n, a])[0]:
            h = n + int(i)
            sk += 2 * int(self.r[h]) + _product_phase(self.x[h], self.z[h], sx, sz)
            sx ^= self.x[h]
            sz ^= self.z[h]
        assert sk % 2 == 0
        return int((sk % 4) == 2)


def simulate(circuit, bits) -> tuple:
    """Records (meas, det, obs as 0/1 numpy arrays) of one shot in which
    symbol s takes bits[s] (bits[0] ignored). Symbols are numbered in op
    order: a fault's symbols when it is reached, a random measurement's
    symbol when it happens."""
    st = CHPState(circuit.num_qubits)
    next_sym = 1
    meas, det = [], []
    obs = {}

    def take(k):
        nonlocal next_sym
        out = [int(bits[next_sym + i]) for i in range(k)]
        next_sym += k
        return out

    for op in circuit.ops:
        t = op.targets
        name = op.name
        if name == "H":
            for a in t: st.h(a)
        elif name == "S":
            for a in t: st.s(a)
        elif name == "CX":
            for a, b in zip(t[::2], t[1::2]): st.cx(a, b)
        elif name in ("X", "Y", "Z"):
            for a in t: st.pauli(a, name in "XY", name in "YZ")
        elif name in ("X_ERROR", "Y_ERROR", "Z_ERROR"):
            for a in t:
                (v,) = take(1)
                if v:
                    st.pauli(a, name[0] in "XY", name[0] in "YZ")
        elif name == "DEPOLARIZE1":
            for a in t:
                vx, vz = take(2)
                st.pauli(a, bool(vx), bool(vz))
        elif name == "DEPOLARIZE2":
            for a, b in zip(t[::2], t[1::2]):
                xa, za, xb, zb = take(4)
                st.pauli(a, bool(xa), bool(za))
                st.pauli(b, bool(xb), bool(zb))
        elif name in ("M", "MR", "R"):
            for a in t:
                forced = take(1)[0] if st.is_random(a) else 0
                m = st.measure(a, forced)
                if name != "R":
                    meas.append(m)
                if name != "M" and m:
                    st.pauli(a, True, False)
        elif name in ("X_IF", "Y_IF", "Z_IF"):
            for k, a in zip(t[::2], t[1::2]):
                if meas[-k]:
                    st.pauli(a, name[0] in "XY", name[0] in "YZ")
        elif name == "DETECTOR":
            det.append(int(np.bitwise_xor.reduce([meas[-k] for k in t])) if t else 0)
        elif name == "OBSERVABLE_INCLUDE":
            o = int(op.arg)
            v = int(np.bitwise_xor.reduce([meas[-k] for k in t])) if t else 0
            obs[o] = obs.get(o, 0) ^ v
        elif name == "TICK":
            pass
        else:
            raise ValueError(name)
    nobs = (max(obs) + 1) if obs else 0
    return (np.array(meas, np.uint8), np.array(det, np.uint8),
            np.array([obs.get(i, 0) for i in range(nobs)], np.uint8))
