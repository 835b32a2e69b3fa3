"""Rotated surface code layout and the syndrome-extraction program of one shot.

Test infrastructure only: the CUDA path never imports this module (the library
compiles the same program independently, in C++).

Sec. II and Fig. 1: d x d data qubits on the vertices, d^2 - 1 ancillas on the
faces, alternating X and Z faces, weight-2 faces on the boundary; a Z face
measures Z^4 with CNOTs data -> ancilla, an X face measures X^4 with H,
CNOTs ancilla -> data, H; repeated for d (here: `rounds`) rounds.
Sec. III A / Table I: depolarising noise after 1- and 2-qubit gates
(Eq. 2-3), an X flip after reset, a flipped record after measurement.
Sec. III B / Eq. 4 and the Fig. 1 caption: crosstalk after each CNOT layer.

Readings of what the paper leaves open:
  * Coordinates: data qubit (column i, row j) at (x, y) = (2i+1, 2j+1);
    face (i, j), 0 <= i, j <= d, at (2i, 2j), X type when i + j is odd.
    Interior faces are 1 <= i, j <= d-1; boundary X faces lie on the top
    and bottom rows (j = 0, d), boundary Z faces on the left and right
    columns (i = 0, d).  Qubit (= MPS site) index: all 2d^2-1 qubits sorted
    by (y, x).
  * CNOT order (offsets dx, dy of the data qubit from the face):
    Z faces NW, SW, NE, SE; X faces NW, NE, SW, SE.  Layer l uses the l-th
    offset; a face without that neighbour idles in layer l.
  * Crosstalk pairs: every (ancilla, neighbouring data) edge, ordered by
    ancilla index then layer.  An edge is gated in exactly one layer and
    receives exp(-i theta Z Z) after each of the other layers.  Optional
    next-nearest pairs (X X at the given angle) receive it after every layer.
  * Events (each consumes one Philox uniform, see `oracle.philox`) are numbered
    in program order: reset flip on every qubit at the start; per round
    H noise on X ancillas, CNOT noise in layer order, H noise again, then for
    each ancilla: Born draw, record flip, reset flip; at the end, for each data
    qubit: Born draw, record flip.
"""

from dataclasses import dataclass, field

Z_ORDER = ((-1, -1), (-1, 1), (1, -1), (1, 1))  # NW, SW, NE, SE
X_ORDER = ((-1, -1), (1, -1), (-1, 1), (1, 1))  # NW, NE, SW, SE


@dataclass
class Layout:
    d: int
    coords: list  # qubit index -> (x, y)
    data: list  # qubit indices of data qubits (ascending)
    ancillas: list  # qubit indices of ancillas (ascending)
    kind: dict  # ancilla -> 'X' or 'Z'
    slots: dict  # ancilla -> [data qubit or None] * 4 (layer order)
    index: dict = field(default_factory=dict)  # (x, y) -> qubit index

    @property
    def n(self):
        return len(self.coords)


def build_layout(d, schedule=None):
    """Qubits of the distance-d rotated code.  `schedule` (optional) replaces
    the CNOT order: one 4-tuple per ancilla, in ascending qubit order, of the
    data qubit each layer gates (or -1 / None for an idle layer)."""
    pts = []
    for j in range(d):
        for i in range(d):
            pts.append((2 * i + 1, 2 * j + 1, "D"))
    for j in range(d + 1):
        for i in range(d + 1):
            kind = "X" if (i + j) % 2 == 1 else "Z"
            interior = 1 <= i <= d - 1 and 1 <= j <= d - 1
            top_bottom = j in (0, d) and 1 <= i <= d - 1 and kind == "X"
            left_right = i in (0, d) and 1 <= j <= d - 1 and kind == "Z"
            if interior or top_bottom or left_right:
                pts.append((2 * i, 2 * j, kind))
    pts.sort(key=lambda t: (t[1], t[0]))
    coords = [(x, y) for x, y, _ in pts]
    index = {c: q for q, c in enumerate(coords)}
    data = [q for q, (x, y, k) in enumerate(pts) if k == "D"]
    ancillas = [q for q, (x, y, k) in enumerate(pts) if k != "D"]
    kind = {q: pts[q][2] for q in ancillas}
    slots = {}
    for a in ancillas:
        x, y = coords[a]
        order = X_ORDER if kind[a] == "X" else Z_ORDER
        slots[a] = [index.get((x + dx, y + dy)) for dx, dy in order]
    if schedule is not None:
        slots = schedule_slots(coords, index, ancillas, slots, schedule)
    return Layout(d, coords, data, ancillas, kind, slots, index)


def schedule_slots(coords, index, ancillas, default, schedule):
    """Validate a caller's CNOT schedule: every ancilla gates each of its
    face's data qubits in exactly one of the four layers, and no qubit takes
    part in two CNOTs of one layer (Fig. 1: four CNOT layers per round)."""
    if len(schedule) != len(ancillas):
        raise ValueError("one schedule row per ancilla")
    slots = {}
    busy = [set() for _ in range(4)]
    for a, row in zip(ancillas, schedule):
        if len(row) != 4:
            raise ValueError("four layers per ancilla")
        got = [None if (q is None or q < 0) else int(q) for q in row]
        face = sorted(q for q in default[a] if q is not None)
        if sorted(q for q in got if q is not None) != face:
            raise ValueError(f"ancilla {a} must gate each of its data qubits once")
        for l, q in enumerate(got):
            if q is not None:
                if q in busy[l] or a in busy[l]:
                    raise ValueError(f"qubit {q} or {a} gated twice in layer {l}")
                busy[l].update((q, a))
        slots[a] = got
    return slots


@dataclass
class Pair:
    a: int
    b: int
    pauli: str  # 'ZZ' or 'XX'
    layer_mask: int  # bit l: rotation after CNOT layer l


def adjacent_idle_pairs(layout):
    pairs = []
    for a in layout.ancillas:
        for l in range(4):
            dq = layout.slots[a][l]
            if dq is not None:
                pairs.append(Pair(a, dq, "ZZ", 0b1111 & ~(1 << l)))
    return pairs


def diagonal_xx_pairs(layout):
    """Next-nearest pairs: data-data and ancilla-ancilla at offset (2, 0) or
    (0, 2), each once, ordered by the lower index."""
    pairs = []
    for q, (x, y) in enumerate(layout.coords):
        for dx, dy in ((2, 0), (0, 2)):
            r = layout.index.get((x + dx, y + dy))
            if r is not None:
                pairs.append(Pair(q, r, "XX", 0b1111))
    return pairs


def idle_mask(layout, a, b):
    """Layers after which a pair (a, b) is idle: all layers except those in
    which a CNOT acts on exactly this pair (Sec. III B: crosstalk on coupled
    qubits that are not gated together)."""
    mask = 0b1111
    for anc in layout.ancillas:
        for l, dq in enumerate(layout.slots[anc]):
            if dq is not None and {anc, dq} == {a, b}:
                mask &= ~(1 << l)
    return mask


def build_pairs(layout, rule, explicit=None):
    """Crosstalk pairs: the rule's, or `explicit` = (a, b, pauli, mask) tuples
    with pauli 'ZZ' or 'XX' and mask the layers after which the pair rotates
    (None: the layers in which the pair is idle)."""
    if explicit is not None:
        pairs = []
        for a, b, pauli, mask in explicit:
            a, b = int(a), int(b)
            if a == b or not (0 <= a < layout.n and 0 <= b < layout.n) or pauli not in ("ZZ", "XX"):
                raise ValueError(f"bad pair {(a, b, pauli)}")
            pairs.append(Pair(a, b, pauli, idle_mask(layout, a, b) if mask is None else int(mask) & 0b1111))
        return pairs
    pairs = adjacent_idle_pairs(layout)
    if rule == "adjacent_idle+diag_xx":
        pairs += diagonal_xx_pairs(layout)
    elif rule != "adjacent_idle":
        raise ValueError(rule)
    return pairs


@dataclass
class Program:
    layout: Layout
    pairs: list
    rounds: int
    ops: list  # tuples, see build_program
    n_events: int
    n_meas: int
    meas_qubit: list  # record index -> qubit
    meas_round: list  # record index -> round (rounds for the final data readout)
    basis: str = "Z"  # memory basis: data prepared and read out in Z or X


def build_program(layout, pairs, rounds, basis="Z"):
    """Op tuples:
    ('RN', q, ev)              reset flip: X on q if u < pR
    ('H', q)                   Hadamard
    ('D1', q, ev)              1-qubit depolarising (Eq. 2) with p1
    ('CX', c, t)               CNOT
    ('D2', c, t, ev)           2-qubit depolarising (Eq. 3) with p2
    ('ROT', k)                 exp(-i theta_k P_k) on pair k
    ('M', q, ev_born, ev_flip, rec, reset, ev_reset)   Z measurement
    """
    ops = []
    ev = 0
    rec = 0
    meas_qubit, meas_round = [], []
    n = layout.n
    if basis not in ("Z", "X"):
        raise ValueError(basis)
    for q in range(n):
        ops.append(("RN", q, ev))
        ev += 1
    if basis == "X":  # data qubits start in |+>: H (with its Eq. 2 noise) after the reset
        for q in layout.data:
            ops.append(("H", q))
            ops.append(("D1", q, ev))
            ev += 1
    xanc = [a for a in layout.ancillas if layout.kind[a] == "X"]
    for r in range(rounds):
        for a in xanc:
            ops.append(("H", a))
            ops.append(("D1", a, ev))
            ev += 1
        for l in range(4):
            for a in layout.ancillas:
                dq = layout.slots[a][l]
                if dq is None:
                    continue
                c, t = (a, dq) if layout.kind[a] == "X" else (dq, a)
                ops.append(("CX", c, t))
                ops.append(("D2", c, t, ev))
                ev += 1
            for k, p in enumerate(pairs):
                if (p.layer_mask >> l) & 1:
                    ops.append(("ROT", k))
        for a in xanc:
            ops.append(("H", a))
            ops.append(("D1", a, ev))
            ev += 1
        for a in layout.ancillas:
            ops.append(("M", a, ev, ev + 1, rec, True, ev + 2))
            ev += 3
            meas_qubit.append(a)
            meas_round.append(r)
            rec += 1
    if basis == "X":  # X readout of the data: H (with its noise), then Z measurement
        for q in layout.data:
            ops.append(("H", q))
            ops.append(("D1", q, ev))
            ev += 1
    for q in layout.data:
        ops.append(("M", q, ev, ev + 1, rec, False, -1))
        ev += 2
        meas_qubit.append(q)
        meas_round.append(rounds)
        rec += 1
    return Program(layout, pairs, rounds, ops, ev, rec, meas_qubit, meas_round, basis)


def detectors(program, record):
    """Detector bits of a memory experiment in basis B (Z or X) from one
    shot's record bits: the B faces in round 0 (their stabilizers start in a
    definite state); every face from round 1 on (XOR with the previous
    round); each B face once more from the final data readout."""
    layout = program.layout
    anc = layout.ancillas
    na = len(anc)
    basis = program.basis
    out = []
    for r in range(program.rounds):
        for i, a in enumerate(anc):
            m = record[r * na + i]
            if r == 0:
                if layout.kind[a] == basis:
                    out.append(m)
            else:
                out.append(m ^ record[(r - 1) * na + i])
    base = program.rounds * na
    data_pos = {q: base + i for i, q in enumerate(layout.data)}
    for i, a in enumerate(anc):
        if layout.kind[a] != basis:
            continue
        par = record[(program.rounds - 1) * na + i]
        for dq in layout.slots[a]:
            if dq is not None:
                par ^= record[data_pos[dq]]
        out.append(par)
    return out


def logical_z(program, record):
    """Parity of the final readout along the logical operator of the memory
    basis: Z_L on the top data row (y = 1), which commutes with the X faces
    (the X boundary faces lie on the top and bottom rows); X_L on the left
    data column (x = 1) for an X-memory run, commuting with the Z faces."""
    layout = program.layout
    base = program.rounds * len(layout.ancillas)
    par = 0
    for i, q in enumerate(layout.data):
        x, y = layout.coords[q]
        if (y == 1 and program.basis == "Z") or (x == 1 and program.basis == "X"):
            par ^= record[base + i]
    return par
