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

std::string build_program(int d, int rounds, int pair_rule, Program &P) {
  if (d < 3 || d % 2 == 0 || d > 11) return "distance must be odd, 3..11";
  if (rounds < 1 || rounds > 1000) return "rounds must be 1..1000";
  if (pair_rule != 0 && pair_rule != 1) return "unknown pair_rule";
  P = Program();
  P.d = d;
  P.rounds = rounds;

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

  // Crosstalk pairs.
  for (size_t ai = 0; ai < P.anc.size(); ++ai)
    for (int l = 0; l < 4; ++l)
      if (P.slots[4 * ai + l] >= 0)
        P.pairs.push_back({P.anc[ai], P.slots[4 * ai + l], 0, 0xF & ~(1 << l)});
  if (pair_rule == 1) {
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
  for (int q = 0; q < P.n; ++q) P.ops.push_back(make_op(OP_RESET_FLIP, q, 0, 0, ev++, 0));
  std::vector<int> xanc;
  for (int a : P.anc)
    if (P.kind[a] == 'X') xanc.push_back(a);
  for (int r = 0; r < rounds; ++r) {
    if (r > 0) P.seg_begin.push_back(static_cast<int>(P.ops.size()));
    for (int a : xanc) {
      P.ops.push_back(make_op(OP_H, a, 0, 0, 0, 0));
      P.ops.push_back(make_op(OP_NOISE1, a, 0, 0, ev++, 0));
    }
    for (int l = 0; l < 4; ++l) {
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
  for (int q : P.data) {
    P.ops.push_back(make_op(OP_MEAS, q, 0, 0, ev, rec++));
    ev += 2;
  }
  P.seg_begin.push_back(static_cast<int>(P.ops.size()));
  P.n_events = ev;
  P.n_meas = rec;

  // Detectors (Sec. II): round 0 sees only the Z faces, which start in a
  // definite state; from round 1 on every face is compared with its previous
  // outcome; the final data readout closes each Z face with its last round.
  const int na = static_cast<int>(P.anc.size());
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
        if (P.kind[P.anc[ai]] == 'Z') add_det({ai}, none);
      } else {
        add_det({r * na + ai, (r - 1) * na + ai}, none);
      }
    }
  std::vector<int> data_pos(P.n, -1);
  for (size_t i = 0; i < P.data.size(); ++i) data_pos[P.data[i]] = rounds * na + static_cast<int>(i);
  for (int ai = 0; ai < na; ++ai) {
    if (P.kind[P.anc[ai]] != 'Z') continue;
    std::vector<int> dq;
    for (int l = 0; l < 4; ++l)
      if (P.slots[4 * ai + l] >= 0) dq.push_back(data_pos[P.slots[4 * ai + l]]);
    add_det({(rounds - 1) * na + ai}, dq);
  }
  // Z_L: the data qubits of the top row (y = 1)
  for (int q : P.data)
    if (P.xy[2 * q + 1] == 1) P.logical.push_back(data_pos[q]);
  return std::string();
}

}  // namespace stn
