// Compiled syndrome-extraction program shared by the host API and the kernels.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace stn {

enum OpKind : uint8_t {
  OP_RESET_FLIP = 1,  // X on qubit a when u < pR
  OP_H = 2,           // Hadamard on a
  OP_NOISE1 = 3,      // depolarising (Eq. 2) on a
  OP_CNOT = 4,        // control a, target b
  OP_NOISE2 = 5,      // depolarising (Eq. 3) on (a, b)
  OP_ROT = 6,         // exp(-i theta_idx P_a P_b), P = Z (pauli 0) or X (pauli 1)
  OP_MEAS = 7,        // Z measurement of a; record idx; pauli = 1: reset afterwards
};

// 16-byte op.  ev: first random event of the op (a measurement uses ev (Born
// draw), ev+1 (record flip) and, when it resets, ev+2 (reset flip)).
struct Op {
  uint8_t kind;
  uint8_t pauli;
  uint16_t a;
  uint16_t b;
  uint16_t pad;
  int32_t ev;
  int32_t idx;
};
static_assert(sizeof(Op) == 16, "Op must stay 16 bytes");

struct Pair {
  int32_t a, b, pauli, layer_mask;
};

// What the caller asks for (stn_config, deep-copied): code distance and
// rounds, memory basis (0 Z, 1 X), an optional CNOT schedule ([n_anc][4]
// data qubits or -1, ancillas in ascending qubit order; empty = the default
// order) and optional explicit crosstalk pairs (layer_mask < 0: the layers in
// which the pair is not gated; empty with explicit_pairs false = pair_rule).
struct ProgramSpec {
  int d = 0, rounds = 0, pair_rule = 0, basis = 0;
  std::vector<int32_t> schedule;
  bool explicit_pairs = false;
  std::vector<Pair> pairs;
};

struct Program {
  int d = 0, rounds = 0, n = 0, basis = 0;
  std::vector<int> xy;          // qubit -> x, y (2 ints)
  std::vector<int> data, anc;   // qubit indices
  std::vector<char> kind;       // qubit -> 'D', 'X', 'Z'
  std::vector<int> slots;       // ancilla (position in anc) -> 4 data qubits or -1
  std::vector<Pair> pairs;
  std::vector<Op> ops;
  std::vector<int> seg_begin;   // rounds + 2 entries: segment r = [seg_begin[r], seg_begin[r+1])
  // 4 rounds + 1 entries: layer step s = [step_begin[s], step_begin[s+1]) is
  // CNOT layer s % 4 of round s / 4 with its crosstalk rotations; the first
  // layer of a round also holds the round's opening H gates (and, in round
  // 0, the initial resets), the last one its closing H gates and ancilla
  // measurements, and the very last step the final data readout
  std::vector<int> step_begin;
  int n_events = 0, n_meas = 0;
  // Detectors of the Z-memory experiment: [n_det][kDetWidth] record indices
  // whose XOR is the detector bit (-1 pads); logical: record indices of the
  // final data readout whose XOR is the Z_L parity.
  std::vector<int32_t> det, logical;
  int n_det = 0;
};

constexpr int kDetWidth = 6;

// Builds the program; returns an empty string or the reason for failure.
std::string build_program(const ProgramSpec &spec, Program &out);

}  // namespace stn
