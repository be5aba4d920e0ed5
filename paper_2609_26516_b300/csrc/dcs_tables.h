// Host-side construction of the per-chunk device tables of libdcs (shared by the context
// API and the allocation-free entry point): the FP64 operator-Schmidt split of each
// two-qubit gate and the per-site description of a chunk.
#pragma once
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>

#include "dcs_kernels.cuh"

namespace dcs {

using cd = std::complex<double>;

// ----------------------------------------------------------------------------- 4x4 SVD
// One-sided Jacobi SVD of a 4x4 complex matrix in FP64: M V = U Sigma.  Returns sigma
// (descending), the columns of M V (= U Sigma) and V, reordered accordingly.
inline void svd4(const cd M[16], double sig[4], cd MV[16], cd Vm[16]) {
  cd X[16], V[16];
  for (int i = 0; i < 16; ++i) {
    X[i] = M[i];
    V[i] = (i / 4 == i % 4) ? 1.0 : 0.0;
  }
  // X, V row-major [row][col]; rotate columns
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < 4; ++i)
      for (int j = i + 1; j < 4; ++j) {
        double a = 0, b = 0;
        cd g = 0;
        for (int r = 0; r < 4; ++r) {
          a += std::norm(X[r * 4 + i]);
          b += std::norm(X[r * 4 + j]);
          g += std::conj(X[r * 4 + i]) * X[r * 4 + j];
        }
        const double ag = std::abs(g);
        if (ag <= 1e-15 * std::sqrt(a * b) || ag == 0.0) continue;
        off = std::max(off, ag / std::sqrt(a * b));
        const double zeta = (b - a) / (2 * ag);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1 + zeta * zeta));
        const double c = 1 / std::sqrt(1 + t * t), s = c * t;
        const cd ph = std::conj(g) / ag;
        for (int r = 0; r < 4; ++r) {
          const cd xi = X[r * 4 + i], xj = ph * X[r * 4 + j];
          X[r * 4 + i] = c * xi - s * xj;
          X[r * 4 + j] = s * xi + c * xj;
          const cd vi = V[r * 4 + i], vj = ph * V[r * 4 + j];
          V[r * 4 + i] = c * vi - s * vj;
          V[r * 4 + j] = s * vi + c * vj;
        }
      }
    if (off < 1e-15) break;
  }
  double nrm[4];
  int idx[4] = {0, 1, 2, 3};
  for (int j = 0; j < 4; ++j) {
    double s = 0;
    for (int r = 0; r < 4; ++r) s += std::norm(X[r * 4 + j]);
    nrm[j] = std::sqrt(s);
  }
  std::stable_sort(idx, idx + 4, [&](int a, int b) { return nrm[a] > nrm[b]; });
  for (int k = 0; k < 4; ++k) {
    sig[k] = nrm[idx[k]];
    for (int r = 0; r < 4; ++r) {
      MV[r * 4 + k] = X[r * 4 + idx[k]];
      Vm[r * 4 + k] = V[r * 4 + idx[k]];
    }
  }
}

// A condition the device can evaluate: a known op, and at most 5 bits for a truth table.
inline bool cond_valid(const dcs_cond& c) {
  if (c.op == DCS_COND_NONE || c.op == DCS_COND_XOR || c.op == DCS_COND_AND ||
      c.op == DCS_COND_OR)
    return true;
  if (c.op != DCS_COND_TABLE) return false;
  int bits = 0;
  for (int w = 0; w < DCS_CWORDS; ++w) bits += __builtin_popcountll(c.mask[w]);
  return bits <= 5;
}

inline DCond to_dcond(const dcs_cond& c) {
  DCond d;
  std::memset(&d, 0, sizeof(d));
  for (int w = 0; w < DCS_CWORDS; ++w) d.mask[w] = c.mask[w];
  d.op = c.op;
  d.value = c.value;
  return d;
}

// Normalised gate: qubits ascending, matrix over |s_lo s_hi>.
inline void gate_matrix(const dcs_op& o, cd* m, int& lo) {
  if (o.kind == DCS_OP_GATE1) {
    lo = o.q0;
    for (int i = 0; i < 4; ++i) m[i] = cd(o.m[2 * i], o.m[2 * i + 1]);
    return;
  }
  cd g[16];
  for (int i = 0; i < 16; ++i) g[i] = cd(o.m[2 * i], o.m[2 * i + 1]);
  if (o.q0 < o.q1) {
    lo = o.q0;
    for (int i = 0; i < 16; ++i) m[i] = g[i];
  } else {
    lo = o.q1;
    // swap the two tensor factors on both the output and the input side
    for (int oa = 0; oa < 2; ++oa)
      for (int ob = 0; ob < 2; ++ob)
        for (int ia = 0; ia < 2; ++ia)
          for (int ib = 0; ib < 2; ++ib)
            m[(oa * 2 + ob) * 4 + (ia * 2 + ib)] = g[(ob * 2 + oa) * 4 + (ib * 2 + ia)];
  }
}

inline DGate1 to_dgate1(const cd* m, const dcs_cond& c) {
  DGate1 g;
  for (int i = 0; i < 4; ++i) g.u[i] = make_float2((float)m[i].real(), (float)m[i].imag());
  g.cond = to_dcond(c);
  return g;
}

// Tables of one chunk (gates[0 .. n_gates) in circuit order) appended to P.  Returns
// nullptr or an error message.  Uses no heap memory itself; P decides where tables live.
template <class Prog>
const char* build_layer(Prog& P, int n, const dcs_op* gates, int n_gates) {
  DLayer L;
  std::memset(&L, 0, sizeof(L));
  int pair_of[DCS_MAX_QUBITS];  // left qubit of the two-qubit gate touching q
  int two_pos[DCS_MAX_QUBITS];  // position of that gate in the chunk
  for (int q = 0; q < n; ++q) pair_of[q] = two_pos[q] = -1;
  for (int i = 0; i < n_gates; ++i) {
    const dcs_op& o = gates[i];
    if (o.kind != DCS_OP_GATE2) continue;
    const int lo = std::min(o.q0, o.q1), hi = std::max(o.q0, o.q1);
    if (lo < 0 || hi >= n || hi - lo != 1) return "two-qubit gates must act on neighbouring qubits";
    if (pair_of[lo] >= 0 || pair_of[hi] >= 0) return "a qubit carries two two-qubit gates in one chunk";
    pair_of[lo] = lo;
    pair_of[hi] = lo;
    two_pos[lo] = two_pos[hi] = (int)i;
  }
  L.uncond = 0;
  L.cond_off = (int)P.conds.size();
  for (int i = 0; i < n_gates; ++i) {
    const dcs_op& o = gates[i];
    if (o.cond.op == DCS_COND_NONE) L.uncond = 1;
    else P.conds.push_back(to_dcond(o.cond));
  }
  L.n_conds = (int)P.conds.size() - L.cond_off;
  L.blk_off = (int)P.blocks.size();
  // blocks in decreasing q
  int lefts[DCS_MAX_QUBITS];
  int n_lefts = 0;
  for (int q = n - 1; q >= 0; --q)
    if (pair_of[q] == q) lefts[n_lefts++] = q;
  for (int bi = 0; bi < n_lefts; ++bi) {
    const int q = lefts[bi];
    const dcs_op& o2 = gates[two_pos[q]];
    DBlock B;
    std::memset(&B, 0, sizeof(B));
    B.q = q;
    cd G[16];
    int lo;
    gate_matrix(o2, G, lo);
    for (int i = 0; i < 16; ++i) B.G[i] = make_float2((float)G[i].real(), (float)G[i].imag());
    B.cond = to_dcond(o2.cond);
    // operator-Schmidt split: M[(o0 i0), (o1 i1)] = G[(o0 o1), (i0 i1)]
    cd M[16], MV[16], Vm[16];
    double sig[4];
    for (int o0 = 0; o0 < 2; ++o0)
      for (int i0 = 0; i0 < 2; ++i0)
        for (int o1 = 0; o1 < 2; ++o1)
          for (int i1 = 0; i1 < 2; ++i1)
            M[(o0 * 2 + i0) * 4 + (o1 * 2 + i1)] = G[(o0 * 2 + o1) * 4 + (i0 * 2 + i1)];
    svd4(M, sig, MV, Vm);
    int D = 0;
    for (int k = 0; k < 4; ++k)
      if (sig[k] > 1e-14 * sig[0]) ++D;
    if (D < 1) D = 1;
    B.D = D;
    for (int d = 0; d < D; ++d) {
      const double sq = std::sqrt(sig[d]);
      for (int r = 0; r < 4; ++r) {
        const cd wl = MV[r * 4 + d] / sq;              // U sqrt(sigma)
        const cd wr = sq * std::conj(Vm[r * 4 + d]);   // sqrt(sigma) V^H
        B.WL[r * 4 + d] = make_float2((float)wl.real(), (float)wl.imag());
        B.WR[d * 4 + r] = make_float2((float)wr.real(), (float)wr.imag());
      }
    }
    // single-qubit gates on q (side 0) and q+1 (side 1), before / after the two-qubit gate
    for (int side = 0; side < 2; ++side) {
      const int qq = q + side;
      B.pre_off[side] = (int)P.g1.size();
      for (int i = 0; i < two_pos[q]; ++i)
        if (gates[i].kind == DCS_OP_GATE1 && gates[i].q0 == qq) {
          cd m[4];
          int l2;
          gate_matrix(gates[i], m, l2);
          P.g1.push_back(to_dgate1(m, gates[i].cond));
        }
      B.pre_n[side] = (int)P.g1.size() - B.pre_off[side];
      B.post_off[side] = (int)P.g1.size();
      for (int i = two_pos[q] + 1; i < n_gates; ++i)
        if (gates[i].kind == DCS_OP_GATE1 && gates[i].q0 == qq) {
          cd m[4];
          int l2;
          gate_matrix(gates[i], m, l2);
          P.g1.push_back(to_dgate1(m, gates[i].cond));
        }
      B.post_n[side] = (int)P.g1.size() - B.post_off[side];
    }
    // a block without conditional gates is the same on every slot: compose it here
    bool fixed = o2.cond.op == DCS_COND_NONE;
    for (int i = 0; i < n_gates && fixed; ++i)
      if (gates[i].kind == DCS_OP_GATE1 && (gates[i].q0 == q || gates[i].q0 == q + 1) &&
          gates[i].cond.op != DCS_COND_NONE)
        fixed = false;
    B.composed = fixed ? 1 : 0;
    if (fixed) {
      // one-qubit products, later gates on the left: pre[side], post[side]
      cd pre[2][4], post[2][4];
      for (int side = 0; side < 2; ++side) {
        const int qq = q + side;
        for (int part = 0; part < 2; ++part) {
          cd* U = part == 0 ? pre[side] : post[side];
          U[0] = 1.0; U[1] = 0.0; U[2] = 0.0; U[3] = 1.0;
          const int i0 = part == 0 ? 0 : two_pos[q] + 1, i1 = part == 0 ? two_pos[q] : n_gates;
          for (int i = i0; i < i1; ++i) {
            if (gates[i].kind != DCS_OP_GATE1 || gates[i].q0 != qq) continue;
            cd m[4], o[4];
            int l2;
            gate_matrix(gates[i], m, l2);
            for (int r = 0; r < 2; ++r)
              for (int k = 0; k < 2; ++k) o[r * 2 + k] = m[r * 2 + 0] * U[0 * 2 + k] + m[r * 2 + 1] * U[1 * 2 + k];
            for (int e = 0; e < 4; ++e) U[e] = o[e];
          }
        }
      }
      cd Mx[16];
      for (int oi = 0; oi < 4; ++oi)  // Mx = G2 (pre_q x pre_{q+1})
        for (int ii = 0; ii < 4; ++ii) {
          cd acc = 0.0;
          for (int k = 0; k < 4; ++k) acc += G[oi * 4 + k] * pre[0][(k >> 1) * 2 + (ii >> 1)] * pre[1][(k & 1) * 2 + (ii & 1)];
          Mx[oi * 4 + ii] = acc;
        }
      for (int oi = 0; oi < 4; ++oi)  // Gc = (post_q x post_{q+1}) Mx
        for (int ii = 0; ii < 4; ++ii) {
          cd acc = 0.0;
          for (int k = 0; k < 4; ++k) acc += post[0][(oi >> 1) * 2 + (k >> 1)] * post[1][(oi & 1) * 2 + (k & 1)] * Mx[k * 4 + ii];
          B.Gc[oi * 4 + ii] = make_float2((float)acc.real(), (float)acc.imag());
        }
    }
    L.site[q].kind = 2;
    L.site[q].blk = (int)bi;
    L.site[q + 1].kind = 3;
    L.site[q + 1].blk = (int)bi;
    P.blocks.push_back(B);
  }
  L.n_blocks = n_lefts;
  for (int q = 0; q < n; ++q) {
    if (pair_of[q] >= 0) continue;
    const int off = (int)P.g1.size();
    for (int i = 0; i < n_gates; ++i) {
      const dcs_op& o = gates[i];
      if (o.kind == DCS_OP_GATE1 && o.q0 == q) {
        cd m[4];
        int l2;
        gate_matrix(o, m, l2);
        P.g1.push_back(to_dgate1(m, o.cond));
      }
    }
    const int cnt = (int)P.g1.size() - off;
    if (cnt > 0) {
      L.site[q].kind = 1;
      L.site[q].g_off = off;
      L.site[q].g_n = cnt;
    }
  }
  P.layers.push_back(L);
  if (P.overflow()) return "chunk tables exceed their capacity";
  return nullptr;
}


}  // namespace dcs
