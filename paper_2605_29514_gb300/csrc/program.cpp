// Rotated surface code layout, CNOT schedule, crosstalk pairs and the op
// program of one shot (Sec. II, Fig. 1; Sec. III A, Table I; Sec. III B).
//
// Readings of what the paper leaves open (the same ones the oracle takes):
//   * data qubit (column i, row j) at (2i+1, 2j+1); face (i, j) at (2i, 2j),
//     X type when i + j is odd; interior faces 1 <= i, j <= d-1, boundary X
//     faces on rows j = 0, d, boundary Z faces on columns i = 0, d; qubits
//     (= MPS sites) numbered in (y, x) row-major order;
//   * CNOT layers: Z faces visit NW, SW, NE, SE, X faces NW, NE, SW, SE;
//   * crosstalk: every (ancilla, neighbour) edge, gated in one layer, gets
//     exp(-i theta Z Z) after each of the other three layers; the optional
//     next-nearest pairs (offset (2,0) or (0,2)) get X X after every layer;
//     explicit pairs without a layer mask rotate after every layer in which
//     a CNOT does not act on exactly that pair;
//   * X-memory: the data qubits get H (with its Eq. 2 noise) after the
//     initial reset and again before the final Z readout;
//   * random events numbered in program order (see build_program).
#include "program.h"

#include <algorithm>
#include <initializer_list>
#include <map>
#include <tuple>

namespace stn {

namespace {
const int kZOrder[4][2] = {{-1, -1}, {-1, 1}, {1, -1}, {1, 1}};
const int kXOrder[4][2] = {{-1, -1}, {1, -1}, {-1, 1}, {1, 1}};

Op make_op(OpKind k, int a, int b, int pauli, int ev, int idx) {
  Op o{};
  o.kind = k;
  o.a = static_cast<uint16_t>(a);
  o.b = static_cast<uint16_t>(b);
  o.pauli = static_cast<uint8_t>(pauli);
  o.ev = ev;
  o.idx = idx;
  return o;
}
}  // namespace

std::string build_program(const ProgramSpec &spec, Program &P) {
  const int d = spec.d, rounds = spec.rounds, pair_rule = spec.pair_rule;
  if (d < 3 || d % 2 == 0 || d > 11) return "distance must be odd, 3..11";
  if (rounds < 1 || rounds > 1000) return "rounds must be 1..1000";
  if (pair_rule != 0 && pair_rule != 1) return "unknown pair_rule";
  if (spec.basis != 0 && spec.basis != 1) return "memory_basis must be 0 (Z) or 1 (X)";
  P = Program();
  P.d = d;
  P.rounds = rounds;
  P.basis = spec.basis;

  // (y, x, kind) of every qubit, sorted row-major.
  std::vector<std::tuple<int, int, char>> pts;
  for (int j = 0; j < d; ++j)
    for (int i = 0; i < d; ++i) pts.emplace_back(2 * j + 1, 2 * i + 1, 'D');
  for (int j = 0; j <= d; ++j) {
    for (int i = 0; i <= d; ++i) {
      char k = ((i + j) % 2 == 1) ? 'X' : 'Z';
      bool interior = i >= 1 && i <= d - 1 && j >= 1 && j <= d - 1;
      bool top_bottom = (j == 0 || j == d) && i >= 1 && i <= d - 1 && k == 'X';
      bool left_right = (i == 0 || i == d) && j >= 1 && j <= d - 1 && k == 'Z';
      if (interior || top_bottom || left_right) pts.emplace_back(2 * j, 2 * i, k);
    }
  }
  std::sort(pts.begin(), pts.end());
  P.n = static_cast<int>(pts.size());
  if (P.n != 2 * d * d - 1) return "internal: wrong qubit count";
  std::map<std::pair<int, int>, int> index;  // (x, y) -> qubit
  P.xy.resize(2 * P.n);
  P.kind.resize(P.n);
  for (int q = 0; q < P.n; ++q) {
    int y = std::get<0>(pts[q]), x = std::get<1>(pts[q]);
    P.xy[2 * q] = x;
    P.xy[2 * q + 1] = y;
    P.kind[q] = std::get<2>(pts[q]);
    index[{x, y}] = q;
    if (P.kind[q] == 'D') P.data.push_back(q); else P.anc.push_back(q);
  }
  auto at = [&](int x, int y) {
    auto it = index.find({x, y});
    return it == index.end() ? -1 : it->second;
  };
  P.slots.assign(4 * P.anc.size(), -1);
  for (size_t ai = 0; ai < P.anc.size(); ++ai) {
    int a = P.anc[ai];
    const int(*ord)[2] = P.kind[a] == 'X' ? kXOrder : kZOrder;
    for (int l = 0; l < 4; ++l)
      P.slots[4 * ai + l] = at(P.xy[2 * a] + ord[l][0], P.xy[2 * a + 1] + ord[l][1]);
  }
  if (!spec.schedule.empty()) {
    // a caller's schedule: each ancilla gates each of its face's data
    // qubits in exactly one layer, no qubit twice in one layer
    if (spec.schedule.size() != P.slots.size()) return "cnot_schedule needs 4 entries per ancilla";
    std::vector<std::vector<char>> busy(4, std::vector<char>(P.n, 0));
    for (size_t ai = 0; ai < P.anc.size(); ++ai) {
      std::vector<int> face, got;
      for (int l = 0; l < 4; ++l) {
        if (P.slots[4 * ai + l] >= 0) face.push_back(P.slots[4 * ai + l]);
        const int q = spec.schedule[4 * ai + l];
        if (q < -1 || q >= P.n) return "cnot_schedule entry out of range";
        if (q >= 0) got.push_back(q);
      }
      std::sort(face.begin(), face.end());
      std::sort(got.begin(), got.end());
      if (face != got) return "cnot_schedule: an ancilla must gate each of its data qubits once";
      for (int l = 0; l < 4; ++l) {
        const int q = spec.schedule[4 * ai + l];
        if (q < 0) continue;
        if (busy[l][q] || busy[l][P.anc[ai]]) return "cnot_schedule: a qubit is gated twice in one layer";
        busy[l][q] = busy[l][P.anc[ai]] = 1;
      }
    }
    P.slots = spec.schedule;
  }

  // Crosstalk pairs.
  if (spec.explicit_pairs) {
    for (const Pair &p : spec.pairs) {
      if (p.a < 0 || p.b < 0 || p.a >= P.n || p.b >= P.n || p.a == p.b) return "pair qubit out of range";
      if (p.pauli != 0 && p.pauli != 1) return "pair_pauli must be 0 (ZZ) or 1 (XX)";
      int mask = p.layer_mask;
      if (mask < 0) {  // idle rule: every layer in which no CNOT acts on exactly this pair
        mask = 0xF;
        for (size_t ai = 0; ai < P.anc.size(); ++ai)
          for (int l = 0; l < 4; ++l) {
            const int a = P.anc[ai], q = P.slots[4 * ai + l];
            if (q >= 0 && ((a == p.a && q == p.b) || (a == p.b && q == p.a))) mask &= ~(1 << l);
          }
      }
      P.pairs.push_back({p.a, p.b, p.pauli, mask & 0xF});
    }
  } else {
    for (size_t ai = 0; ai < P.anc.size(); ++ai)
      for (int l = 0; l < 4; ++l)
        if (P.slots[4 * ai + l] >= 0)
          P.pairs.push_back({P.anc[ai], P.slots[4 * ai + l], 0, 0xF & ~(1 << l)});
  }
  if (!spec.explicit_pairs && pair_rule == 1) {
    for (int q = 0; q < P.n; ++q) {
      const int off[2][2] = {{2, 0}, {0, 2}};
      for (auto &o : off) {
        int r = at(P.xy[2 * q] + o[0], P.xy[2 * q + 1] + o[1]);
        if (r >= 0) P.pairs.push_back({q, r, 1, 0xF});
      }
    }
  }

  // Program.  Events in program order.
  int ev = 0, rec = 0;
  P.seg_begin.push_back(0);
  P.step_begin.push_back(0);
  for (int q = 0; q < P.n; ++q) P.ops.push_back(make_op(OP_RESET_FLIP, q, 0, 0, ev++, 0));
  if (P.basis == 1) {  // X-memory: data qubits start in |+>
    for (int q : P.data) {
      P.ops.push_back(make_op(OP_H, q, 0, 0, 0, 0));
      P.ops.push_back(make_op(OP_NOISE1, q, 0, 0, ev++, 0));
    }
  }
  std::vector<int> xanc;
  for (int a : P.anc)
    if (P.kind[a] == 'X') xanc.push_back(a);
  for (int r = 0; r < rounds; ++r) {
    if (r > 0) {
      P.seg_begin.push_back(static_cast<int>(P.ops.size()));
      P.step_begin.push_back(static_cast<int>(P.ops.size()));
    }
    for (int a : xanc) {
      P.ops.push_back(make_op(OP_H, a, 0, 0, 0, 0));
      P.ops.push_back(make_op(OP_NOISE1, a, 0, 0, ev++, 0));
    }
    for (int l = 0; l < 4; ++l) {
      if (l > 0) P.step_begin.push_back(static_cast<int>(P.ops.size()));
      for (size_t ai = 0; ai < P.anc.size(); ++ai) {
        int a = P.anc[ai], dq = P.slots[4 * ai + l];
        if (dq < 0) continue;
        int c = P.kind[a] == 'X' ? a : dq;
        int t = P.kind[a] == 'X' ? dq : a;
        P.ops.push_back(make_op(OP_CNOT, c, t, 0, 0, 0));
        P.ops.push_back(make_op(OP_NOISE2, c, t, 0, ev++, 0));
      }
      for (size_t k = 0; k < P.pairs.size(); ++k)
        if ((P.pairs[k].layer_mask >> l) & 1)
          P.ops.push_back(make_op(OP_ROT, P.pairs[k].a, P.pairs[k].b, P.pairs[k].pauli, 0,
                                  static_cast<int>(k)));
    }
    for (int a : xanc) {
      P.ops.push_back(make_op(OP_H, a, 0, 0, 0, 0));
      P.ops.push_back(make_op(OP_NOISE1, a, 0, 0, ev++, 0));
    }
    for (int a : P.anc) {
      P.ops.push_back(make_op(OP_MEAS, a, 0, 1, ev, rec++));
      ev += 3;
    }
  }
  P.seg_begin.push_back(static_cast<int>(P.ops.size()));
  if (P.basis == 1) {  // X readout: H, then the Z measurement
    for (int q : P.data) {
      P.ops.push_back(make_op(OP_H, q, 0, 0, 0, 0));
      P.ops.push_back(make_op(OP_NOISE1, q, 0, 0, ev++, 0));
    }
  }
  for (int q : P.data) {
    P.ops.push_back(make_op(OP_MEAS, q, 0, 0, ev, rec++));
    ev += 2;
  }
  P.seg_begin.push_back(static_cast<int>(P.ops.size()));
  P.step_begin.push_back(static_cast<int>(P.ops.size()));
  P.n_events = ev;
  P.n_meas = rec;

  // Detectors (Sec. II) of a memory experiment in basis B: round 0 sees only
  // the B faces, which start in a definite state; from round 1 on every face
  // is compared with its previous outcome; the final data readout closes
  // each B face with its last round.
  const int na = static_cast<int>(P.anc.size());
  const char bkind = P.basis == 1 ? 'X' : 'Z';
  auto add_det = [&](std::initializer_list<int> idx, const std::vector<int> &more) {
    int k = 0;
    for (int i : idx) P.det.push_back(i), ++k;
    for (int i : more) P.det.push_back(i), ++k;
    for (; k < kDetWidth; ++k) P.det.push_back(-1);
    ++P.n_det;
  };
  const std::vector<int> none;
  for (int r = 0; r < rounds; ++r)
    for (int ai = 0; ai < na; ++ai) {
      if (r == 0) {
        if (P.kind[P.anc[ai]] == bkind) add_det({ai}, none);
      } else {
        add_det({r * na + ai, (r - 1) * na + ai}, none);
      }
    }
  std::vector<int> data_pos(P.n, -1);
  for (size_t i = 0; i < P.data.size(); ++i) data_pos[P.data[i]] = rounds * na + static_cast<int>(i);
  for (int ai = 0; ai < na; ++ai) {
    if (P.kind[P.anc[ai]] != bkind) continue;
    std::vector<int> dq;
    for (int l = 0; l < 4; ++l)
      if (P.slots[4 * ai + l] >= 0) dq.push_back(data_pos[P.slots[4 * ai + l]]);
    add_det({(rounds - 1) * na + ai}, dq);
  }
  // Z_L: the data qubits of the top row (y = 1); X_L: the left column (x = 1)
  for (int q : P.data)
    if ((P.basis == 0 && P.xy[2 * q + 1] == 1) || (P.basis == 1 && P.xy[2 * q] == 1))
      P.logical.push_back(data_pos[q]);
  return std::string();
}

}  // namespace stn
