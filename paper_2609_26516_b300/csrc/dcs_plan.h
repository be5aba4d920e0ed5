// Host-side planning of a whole circuit for libdcs (dcs_run_circuit): reset lowering and
// the grouping of operations into chunks and measurement runs, each one launch.
#pragma once
#include <cstdint>
#include <cstring>
#include <vector>

#include "dcs_tables.h"

namespace dcs {

// One launch of a circuit: the compression of the chunk whose `n` sub-layers are layers
// idx .. idx + n - 1 (kind 0), or a run of `n` consecutive measurements starting at
// measurement `idx` (kind 1).
struct Step {
  int kind;
  int idx;
  int n;
};

// A chunk's gates cut into sub-layers: a two-qubit gate touching a qubit that carries a
// two-qubit gate of the current sub-layer starts the next one; single-qubit gates stay with
// the sub-layer they follow.  Each sub-layer is then one layer of disjoint blocks.
inline std::vector<std::vector<dcs_op>> split_sublayers(const dcs_op* gates, int n_gates, int n) {
  std::vector<std::vector<dcs_op>> out(1);
  std::vector<char> busy(n > 0 ? n : 1, 0);
  for (int i = 0; i < n_gates; ++i) {
    const dcs_op& o = gates[i];
    if (o.kind == DCS_OP_GATE2 && o.q0 >= 0 && o.q0 < n && o.q1 >= 0 && o.q1 < n &&
        (busy[o.q0] || busy[o.q1])) {
      out.emplace_back();
      std::fill(busy.begin(), busy.end(), 0);
    }
    out.back().push_back(o);
    if (o.kind == DCS_OP_GATE2 && o.q0 >= 0 && o.q0 < n && o.q1 >= 0 && o.q1 < n)
      busy[o.q0] = busy[o.q1] = 1;
  }
  return out;
}

// build_layer for each sub-layer of a chunk and the step that compresses them in one launch.
template <class Prog>
const char* add_chunk(Prog& P, int n, const dcs_op* gates, int n_gates) {
  const int first = (int)P.layers.size();
  const std::vector<std::vector<dcs_op>> subs = split_sublayers(gates, n_gates, n);
  for (const std::vector<dcs_op>& sub : subs)
    if (const char* e = build_layer(P, n, sub.data(), (int)sub.size())) return e;
  P.steps.push_back({0, first, (int)subs.size()});
  return nullptr;
}

// Appends the circuit ops[0 .. n_ops) to P (tables of every chunk, measurements, steps):
//  - a reset becomes a measurement into its bit followed by X conditioned on that bit
//    (Sec. "Reset operations");
//  - operations are grouped into chunks (Sec. "Handling unitary chunks in dynamic
//    circuits"): a chunk closes at a measurement, before its (chunk_k + 1)-th operation when
//    chunk_k > 0, and before a two-qubit gate touching a qubit that already carries a
//    two-qubit gate of the chunk's current sub-layer when the chunk holds chunk_layers
//    sub-layers (chunk_layers <= 1: one layer per chunk); otherwise that gate opens the next
//    sub-layer;
//  - consecutive measurements form one run; measurement ordinals (the sampler's counter)
//    count from meas_idx0 in circuit order.
// The ops must already be valid (qubits, bits, kinds).  Returns nullptr or an error message.
template <class Prog>
const char* plan_circuit(Prog& P, int n, int chunk_k, const dcs_op* ops, int n_ops,
                         uint64_t meas_idx0, int chunk_layers = 1) {
  std::vector<dcs_op> lo;
  lo.reserve(n_ops + 8);
  for (int i = 0; i < n_ops; ++i) {
    if (ops[i].kind != DCS_OP_RESET) {
      lo.push_back(ops[i]);
      continue;
    }
    dcs_op m = ops[i];
    m.kind = DCS_OP_MEASURE;
    lo.push_back(m);
    dcs_op x;
    std::memset(&x, 0, sizeof(x));
    x.kind = DCS_OP_GATE1;
    x.q0 = ops[i].q0;
    x.q1 = -1;
    x.m[2] = 1.0;  // X = [[0, 1], [1, 0]]
    x.m[4] = 1.0;
    x.cond.op = DCS_COND_XOR;
    x.cond.value = 1;
    x.cond.mask[ops[i].cbit >> 6] = 1ull << (ops[i].cbit & 63);
    lo.push_back(x);
  }
  std::vector<dcs_op> cur;
  std::vector<char> busy(n, 0);  // qubits carrying a two-qubit gate of the current sub-layer
  int nsub = 1;
  const int max_sub = chunk_layers > 1 ? chunk_layers : 1;
  auto close = [&]() -> const char* {
    const char* e = nullptr;
    if (!cur.empty()) e = add_chunk(P, n, cur.data(), (int)cur.size());
    cur.clear();
    std::fill(busy.begin(), busy.end(), 0);
    nsub = 1;
    return e;
  };
  uint64_t ord = meas_idx0;
  for (const dcs_op& o : lo) {
    if (o.kind == DCS_OP_MEASURE) {
      if (const char* e = close()) return e;
      if (!P.steps.empty() && P.steps.back().kind == 1) {
        P.steps.back().n++;
      } else {
        P.steps.push_back({1, (int)P.meas.size(), 1});
      }
      P.meas.push_back({o.q0, o.cbit, ord++});
      continue;
    }
    if (o.kind == DCS_OP_GATE2 && (busy[o.q0] || busy[o.q1])) {
      if (nsub < max_sub) {
        ++nsub;
        std::fill(busy.begin(), busy.end(), 0);
      } else if (const char* e = close()) {
        return e;
      }
    }
    if (chunk_k > 0 && (int)cur.size() >= chunk_k) {
      if (const char* e = close()) return e;
    }
    cur.push_back(o);
    if (o.kind == DCS_OP_GATE2) busy[o.q0] = busy[o.q1] = 1;
  }
  return close();
}

}  // namespace dcs
