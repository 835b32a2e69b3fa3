"""Host-side decoding of the memory experiment, off the timed path.

The paper decodes the syndromes with minimum-weight matching under an error
model built from the Pauli twirling approximation of the crosstalk (Sec. III C,
Eq. 6): a rotation exp(-i theta P) is replaced by the Pauli P applied with
probability sin^2 theta, and the circuit's Pauli noise (Eq. 2-3, Table I)
enters with its own rates.  This module builds that error model from the
library's compiled program (stn_compile_program, stn_compile_detectors) by
Pauli-frame propagation through the Clifford part of the circuit, and decodes
with a lookup table over all fault sets of up to two faults: each syndrome
maps to the logical flip of larger total probability among the fault sets
that produce it.

Everything here is integer bookkeeping on the host; the simulation itself
never calls it.
"""

from dataclasses import dataclass

import numpy as np

from . import compile_detectors, compile_program

OP_RESET_FLIP, OP_H, OP_NOISE1, OP_CNOT, OP_NOISE2, OP_ROT, OP_MEAS = 1, 2, 3, 4, 5, 6, 7


@dataclass
class FaultModel:
    """Independent fault locations of the circuit: fault f applies its Pauli
    with probability prob[f] and flips the detectors det[f] (bool, [F, n_det])
    and the logical observable obs[f]."""
    prob: np.ndarray
    det: np.ndarray
    obs: np.ndarray
    kind: list  # per fault: ("rot", op index, pair) or ("noise", op index, pauli label)


def _propagate(ops, n, n_meas, inject):
    """Record flips [F, n_meas] of F Pauli faults.  inject[i] lists the
    (fault row, x bits, z bits) applied right after op i (x, z: dicts qubit ->
    bit).  Clifford gates move the frame (H swaps X and Z; CNOT copies X from
    control to target and Z from target to control); a Z measurement records
    the frame's X on its qubit, and a reset clears the qubit's frame."""
    F = sum(len(v) for v in inject.values())
    x = np.zeros((F, n), dtype=bool)
    z = np.zeros((F, n), dtype=bool)
    flips = np.zeros((F, n_meas), dtype=bool)
    for i, (kind, a, b, pauli, _, idx) in enumerate(ops):
        if kind == OP_H:
            x[:, a], z[:, a] = z[:, a].copy(), x[:, a].copy()
        elif kind == OP_CNOT:
            x[:, b] ^= x[:, a]
            z[:, a] ^= z[:, b]
        elif kind == OP_MEAS:
            flips[:, idx] = x[:, a]
            if pauli == 1:  # measured ancilla reset to |0>: its frame is cleared
                x[:, a] = False
                z[:, a] = False
        for row, xs, zs in inject.get(i, ()):
            for q, v in xs.items():
                x[row, q] ^= v
            for q, v in zs.items():
                z[row, q] ^= v
    return flips


def _apply_tables(flips, det_table, logical):
    ext = np.concatenate([flips, np.zeros((flips.shape[0], 1), dtype=bool)], axis=1)  # index -1: zero
    det = np.bitwise_xor.reduce(ext[:, det_table], axis=2)
    obs = np.bitwise_xor.reduce(flips[:, logical], axis=1) if len(logical) else np.zeros(len(flips), bool)
    return det, obs


def build_fault_model(workload, theta, include_pauli_noise=True):
    """Fault model of `workload` with per-pair angles `theta` (radians): one
    PTA fault per crosstalk rotation (its pair's Pauli with probability
    sin^2 theta, Eq. 6), and, when the workload has Pauli noise and
    include_pauli_noise, every single-qubit Pauli after H (p1/3 each), every
    two-qubit Pauli after CNOT (p2/15 each), an X after each reset (pR) and a
    flipped record after each measurement (pM), as in Table I."""
    counts, ops, pairs = compile_program(workload)
    n, n_meas = int(counts[0]), int(counts[2])
    det_table, logical = compile_detectors(workload)
    theta = np.asarray(theta, dtype=np.float64)
    p = workload.p
    p1, p2 = p * workload.p1_scale, p * workload.p2_scale
    pR, pM = p * workload.pR_scale, p * workload.pM_scale
    inject, prob, kinds = {}, [], []
    meas_flip = []  # (fault row, record index)

    def add(i, xs, zs, pr, kind):
        inject.setdefault(i, []).append((len(prob), xs, zs))
        prob.append(pr)
        kinds.append(kind)

    letters = {"X": (1, 0), "Y": (1, 1), "Z": (0, 1)}
    for i, (kind, a, b, pauli, _, idx) in enumerate(ops):
        if kind == OP_ROT:
            q = float(np.sin(theta[idx]) ** 2)
            if q > 0:
                bit = {a: True, b: True}
                add(i, bit if pauli == 1 else {}, {} if pauli == 1 else bit, q, ("rot", i, int(idx)))
        elif not include_pauli_noise or p == 0:
            continue
        elif kind == OP_NOISE1 and p1 > 0:
            for lab, (xb, zb) in letters.items():
                add(i, {a: bool(xb)}, {a: bool(zb)}, p1 / 3, ("noise", i, lab))
        elif kind == OP_NOISE2 and p2 > 0:
            for k in range(1, 16):
                lc, lt = "IXYZ"[k // 4], "IXYZ"[k % 4]
                xs, zs = {}, {}
                for q, lab in ((a, lc), (b, lt)):
                    if lab != "I":
                        xs[q], zs[q] = bool(letters[lab][0]), bool(letters[lab][1])
                add(i, xs, zs, p2 / 15, ("noise", i, lc + lt))
        elif kind == OP_RESET_FLIP and pR > 0:
            add(i, {a: True}, {}, pR, ("noise", i, "reset"))
        elif kind == OP_MEAS:
            if pM > 0:
                meas_flip.append((len(prob), int(idx)))
                add(i, {}, {}, pM, ("noise", i, "record"))
            if pauli == 1 and pR > 0:
                add(i, {a: True}, {}, pR, ("noise", i, "reset"))
    flips = _propagate(ops, n, n_meas, inject)
    for row, rec in meas_flip:
        flips[row, rec] ^= True
    det, obs = _apply_tables(flips, det_table, logical)
    return FaultModel(np.array(prob), det, obs, kinds)


def _key(bits):
    return np.packbits(bits, bitorder="little").tobytes()


class LookupDecoder:
    """Syndrome -> predicted logical flip, from all fault sets of at most two
    faults of a FaultModel (the lookup-table decoder of the d = 3 workload).
    A syndrome outside the table is predicted as no flip and counted."""

    def __init__(self, model, max_faults=2):
        acc = {}

        def put(key, flip, w):
            e = acc.setdefault(key, [0.0, 0.0])
            e[int(flip)] += w

        q = model.prob
        q0 = float(np.prod(1.0 - q))
        put(_key(np.zeros(model.det.shape[1], dtype=bool)), False, q0)
        odds = q / (1.0 - q)
        for f in range(len(q)):
            put(_key(model.det[f]), model.obs[f], q0 * odds[f])
        if max_faults >= 2:
            F = len(q)
            for f in range(F):
                g = np.arange(f + 1, F)
                if len(g) == 0:
                    continue
                dets = model.det[f] ^ model.det[g]
                obs = model.obs[f] ^ model.obs[g]
                w = q0 * odds[f] * odds[g]
                keys = np.packbits(dets, axis=1, bitorder="little")
                for k, o, ww in zip(keys, obs, w):
                    put(k.tobytes(), o, float(ww))
        self.table = {k: int(v[1] > v[0]) for k, v in acc.items()}
        self.n_det = model.det.shape[1]
        self.unseen = 0

    def predict(self, det_bits):
        """Predicted logical flips of detector rows [shots, n_det] (0/1)."""
        det_bits = np.asarray(det_bits, dtype=bool)
        out = np.zeros(len(det_bits), dtype=np.uint8)
        for s, row in enumerate(det_bits):
            v = self.table.get(_key(row))
            if v is None:
                self.unseen += 1
                v = 0
            out[s] = v
        return out


class MatchingDecoder:
    """Minimum-weight perfect matching on the detector graph of a FaultModel
    (the paper decodes with MWPM under the PTA error model, Sec. III C).

    Graph: one node per detector plus a boundary node.  Each fault that flips
    one detector (an edge to the boundary) or two (an edge between them) gives
    an edge of weight log((1 - q) / q); parallel edges keep the likelier
    fault.  Faults that flip more detectors (a Y, or a two-qubit Pauli that
    acts on both check types) are products of such edges and add none.
    uniform=True gives every edge weight 1, which makes the decoder a
    nearest-explanation decoder: at distance d it corrects every set of
    fewer than d / 2 faults, the property the CPU tests pin.

    Decoding a syndrome: shortest paths between all nodes (Dijkstra) carry
    their logical parity.  The fired detectors are matched in pairs or to
    the boundary at least total path length: exactly by dynamic programming
    over subsets for up to dp_limit defects, else by the blossom algorithm
    (networkx.max_weight_matching, each defect with its own copy of the
    boundary).  The predicted flip is the XOR of the matched paths'
    parities.  Host-side and off the timed path."""

    def __init__(self, model, uniform=False, dp_limit=12):
        import scipy.sparse as sp
        from scipy.sparse.csgraph import dijkstra
        n = model.det.shape[1]
        self.n_det, self.boundary = n, n
        best = {}  # (a, b) -> (q, obs)
        for f in range(len(model.prob)):
            d = np.flatnonzero(model.det[f])
            if len(d) == 0 or len(d) > 2:
                continue
            key = (int(d[0]), int(d[1])) if len(d) == 2 else (int(d[0]), n)
            q = float(model.prob[f])
            if q <= 0.0:
                continue
            if key not in best or q > best[key][0]:
                best[key] = (q, bool(model.obs[f]))
        rows, cols, wts = [], [], []
        self._edge_obs = {}
        for (a, b), (q, o) in best.items():
            w = 1.0 if uniform else float(np.log((1.0 - q) / q)) if q < 0.5 else 1e-9
            rows.append(a)
            cols.append(b)
            wts.append(max(w, 1e-9))
            self._edge_obs[(a, b)] = self._edge_obs[(b, a)] = o
        g = sp.coo_matrix((wts, (rows, cols)), shape=(n + 1, n + 1)).tocsr()
        self.dist, pred = dijkstra(g, directed=False, return_predecessors=True)
        # logical parity of each shortest path, walking the predecessor tree
        par = np.zeros((n + 1, n + 1), dtype=bool)
        for src in range(n + 1):
            order = np.argsort(self.dist[src])
            for v in order:
                u = pred[src, v]
                if u >= 0:
                    par[src, v] = par[src, u] ^ self._edge_obs[(int(u), int(v))]
        self.parity = par
        self.dp_limit = int(dp_limit)
        self.unmatched = 0

    def _decode(self, defects):
        k = len(defects)
        if k == 0:
            return 0
        if k <= self.dp_limit:
            return self._decode_dp(defects)
        return self._decode_blossom(defects)

    def _decode_dp(self, defects):
        """Exact minimum-weight matching of a few defects by dynamic
        programming over subsets: the lowest remaining defect either goes to
        the boundary or pairs with one of the others."""
        from functools import lru_cache
        bd = [self.dist[a, self.boundary] for a in defects]
        bp = [int(self.parity[a, self.boundary]) for a in defects]

        @lru_cache(maxsize=None)
        def best(mask):
            if mask == 0:
                return 0.0, 0
            i = (mask & -mask).bit_length() - 1
            rest = mask & ~(1 << i)
            c, f = best(rest)
            cand = (bd[i] + c, f ^ bp[i])
            m2 = rest
            while m2:
                j = (m2 & -m2).bit_length() - 1
                m2 &= m2 - 1
                c2, f2 = best(rest & ~(1 << j))
                v = self.dist[defects[i], defects[j]] + c2
                if v < cand[0]:
                    cand = (v, f2 ^ int(self.parity[defects[i], defects[j]]))
            return cand

        cost, flip = best((1 << len(defects)) - 1)
        if not np.isfinite(cost):
            self.unmatched += 1
        return flip

    def _decode_blossom(self, defects):
        """The same matching for many defects: each defect with its own copy
        of the boundary, perfect matching of least total path length by the
        blossom algorithm (networkx)."""
        import networkx as nx
        k = len(defects)
        big = 1.0 + 2.0 * np.nanmax(np.where(np.isfinite(self.dist), self.dist, 0.0)) * max(k, 1)
        g = nx.Graph()
        for i in range(k):
            a = defects[i]
            db = self.dist[a, self.boundary]
            if np.isfinite(db):
                g.add_edge(("d", i), ("b", i), weight=big - db)
            for j in range(i + 1, k):
                dab = self.dist[a, defects[j]]
                if np.isfinite(dab):
                    g.add_edge(("d", i), ("d", j), weight=big - dab)
                g.add_edge(("b", i), ("b", j), weight=big)
        match = nx.max_weight_matching(g, maxcardinality=True)
        flip = 0
        covered = 0
        for u, v in match:
            if u[0] == "b" and v[0] == "b":
                continue
            if u[0] == "b":
                u, v = v, u
            a = defects[u[1]]
            b = self.boundary if v[0] == "b" else defects[v[1]]
            flip ^= int(self.parity[a, b])
            covered += 1 + (v[0] == "d")
        if covered < k:
            self.unmatched += 1
        return flip

    def predict(self, det_bits):
        """Predicted logical flips of detector rows [shots, n_det] (0/1)."""
        det_bits = np.asarray(det_bits, dtype=bool)
        return np.array([self._decode(np.flatnonzero(row)) for row in det_bits], dtype=np.uint8)


def logical_error_rate(decoder, det_bits, observed):
    """Fraction of shots whose predicted flip differs from the observed
    logical parity, and that count."""
    pred = decoder.predict(det_bits)
    fails = int(np.sum(pred != np.asarray(observed, dtype=np.uint8)))
    return fails / max(1, len(pred)), fails


def wilson_interval(k, n, z=1.959963984540054):
    """95% Wilson score interval of a binomial proportion k / n."""
    if n == 0:
        return 0.0, 1.0
    ph = k / n
    den = 1 + z * z / n
    c = (ph + z * z / (2 * n)) / den
    h = z * np.sqrt(ph * (1 - ph) / n + z * z / (4 * n * n)) / den
    lo = 0.0 if k == 0 else max(0.0, c - h)  # exact ends (no rounding residue)
    hi = 1.0 if k == n else min(1.0, c + h)
    return lo, hi


def eq1_estimate(expectations, corrections):
    """P_L of Sec. II, Eq. 1: the mean over the sampled syndromes of
    |sin(theta_i / 2)|, with sin^2(theta_i / 2) = (1 - (-1)^c_i <L>_i) / 2
    from the logical expectation <L>_i before the readout
    (stn_logical_expectation) and the decoder's correction c_i.  For Pauli
    errors <L>_i = +-1 and the estimate is the sampled failure rate."""
    e = np.asarray(expectations, dtype=np.float64)
    c = np.asarray(corrections, dtype=np.float64)
    q = np.clip(0.5 * (1.0 - (-1.0) ** c * e), 0.0, 1.0)
    return float(np.mean(np.sqrt(q)))
