// Kernels of libdcs for sm_103a: one CTA per slot (shot or branch) runs a whole
// CompressionStep, measurement or branch update with the MPS tiles staged in shared memory
// (bond dimension up to DCS_MAX_CHI_FUSED).
//
// Compression step (Sec. "Simulating unitary quantum circuits with DMRG"): the bra starts
// as the chunk applied block by block to the ket in canonical form, each two-qubit block
// followed by a truncated SVD (keep the smallest rank whose discarded weight is
// <= tol * total, at most chi_max), the blocks taken from the end of the layer nearest the
// orthogonality centre so the centre crosses the layer once.  If no block discarded more
// than the tolerance the guess is the result (f = product of the kept weight fractions);
// otherwise `sweeps` one-site sweeps against the exact target W|A> follow: each site takes
// F / ||F|| (Sec. above: the optimum of max <T|F>), made orthonormal by Householder QR, and
// the last site gives f = ||F||^2 = |<B|W A>|^2.
//
// Right-to-left steps reuse the left-to-right code on the mirrored chain: a site tensor
// A[a][t][x] is read as A'[x][t][a], an MPO tensor W[d][s][t][e] as W'[e][s][t][d], and the
// right environment R[c][e][x] plays the role of the left one.  (Reversing the chain leaves
// the overlap network unchanged.)
//
// This header holds what the kernel translation units share: the helpers, the contraction
// loops, the working-set carving, the blocked QR and the gauge moves.  The kernels live in
// dcs_k_small.cu (shared-memory tiles), dcs_k_big.cu (global tiles) and dcs_k_ops.cu
// (measurement, initialisation, branches), compiled in parallel.
#pragma once
#include <cstdio>

// Whether this translation unit's kernels run the tensor-core GEMM (only the TF32X3 / BF16X3
// compression kernel does; keeping its code out of the others keeps their registers free).
#ifndef DCS_TU_TENSOR_CORES
#define DCS_TU_TENSOR_CORES 0
#endif

#include "dcs_device.cuh"
#include "dcs_gemm.cuh"
#include "dcs_kernels.cuh"

namespace dcs {

// ----------------------------------------------------------------------------- helpers

// Optional per-phase cycle counters of the compression and measurement kernels (built with
// -DDCS_PHASE_TIMERS; read back with dcs_debug_phase_cycles).  Off in normal builds.
// Slots 0-9: large-tile compression; 10-15: small-tile compression; 16-17: measurement.
#ifdef DCS_PHASE_TIMERS
static __device__ unsigned long long g_phase_cycles[24];
#define PHASE_START() long long _pt = clock64()
#define PHASE_MARK(i)                                                                     \
  do {                                                                                    \
    __syncthreads();                                                                      \
    if (threadIdx.x == 0) {                                                               \
      const long long _n = clock64();                                                     \
      atomicAdd(&g_phase_cycles[i], (unsigned long long)(_n - _pt));                      \
      _pt = _n;                                                                           \
    }                                                                                     \
  } while (0)
#else
#define PHASE_START()
#define PHASE_MARK(i)
#endif


__device__ __forceinline__ bool cond_holds(const DCond& cd, const uint64_t* c) {
  if (cd.op == DCS_COND_NONE) return true;
  if (cd.op == DCS_COND_XOR) {
    int par = 0;
#pragma unroll
    for (int w = 0; w < DCS_CWORDS; ++w) par ^= __popcll(c[w] & cd.mask[w]) & 1;
    return par == cd.value;
  }
  if (cd.op == DCS_COND_OR) {
    bool any = false;
#pragma unroll
    for (int w = 0; w < DCS_CWORDS; ++w) any = any || ((c[w] & cd.mask[w]) != 0ull);
    return (int)any == cd.value;
  }
  if (cd.op == DCS_COND_TABLE) {
    // the masked bits in ascending order form the index into the truth table
    uint32_t idx = 0;
    int k = 0;
    for (int w = 0; w < DCS_CWORDS; ++w) {
      uint64_t m = cd.mask[w];
      while (m != 0ull && k < 5) {
        const int b = __ffsll((long long)m) - 1;
        idx |= (uint32_t)((c[w] >> b) & 1ull) << k;
        ++k;
        m &= m - 1ull;
      }
    }
    return (((uint32_t)cd.value >> idx) & 1u) != 0u;
  }
  bool all = true;
#pragma unroll
  for (int w = 0; w < DCS_CWORDS; ++w) all = all && ((c[w] & cd.mask[w]) == cd.mask[w]);
  return (int)all == cd.value;
}

// U := product of the applicable single-qubit gates g[off .. off+n) (later gates on the left)
static __device__ __noinline__ void prod1q(const DGate1* g, int off, int n, const uint64_t* c, float2* U) {
  U[0] = make_float2(1.f, 0.f);
  U[1] = cz();
  U[2] = cz();
  U[3] = make_float2(1.f, 0.f);
  for (int i = 0; i < n; ++i) {
    const DGate1& G = g[off + i];
    if (!cond_holds(G.cond, c)) continue;
    float2 o[4];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        float2 a = cz();
        cfma(a, G.u[r * 2 + 0], U[0 * 2 + k]);
        cfma(a, G.u[r * 2 + 1], U[1 * 2 + k]);
        o[r * 2 + k] = a;
      }
#pragma unroll
    for (int i2 = 0; i2 < 4; ++i2) U[i2] = o[i2];
  }
}

// W of site j for register c into W[dl][s][t][dr] (row-major); returns dl, dr.  One thread.
static __device__ __noinline__ void build_W(int j, const DLayer* L, const DBlock* BK, const DGate1* G1,
                        const uint64_t* c, float2* W, int* dl_out, int* dr_out) {
  const DSite& st = L->site[j];
  if (st.kind == 0 || st.kind == 1) {
    float2 U[4];
    if (st.kind == 1) {
      prod1q(G1, st.g_off, st.g_n, c, U);
    } else {
      U[0] = make_float2(1.f, 0.f);
      U[1] = cz();
      U[2] = cz();
      U[3] = make_float2(1.f, 0.f);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) W[i] = U[i];
    *dl_out = 1;
    *dr_out = 1;
    return;
  }
  const DBlock& b = BK[L->blk_off + st.blk];
  const int side = (st.kind == 2) ? 0 : 1;
  float2 Pre[4], Post[4];
  prod1q(G1, b.pre_off[side], b.pre_n[side], c, Pre);
  prod1q(G1, b.post_off[side], b.post_n[side], c, Post);
  const bool on = cond_holds(b.cond, c);
  const int D = b.D;
  for (int d = 0; d < D; ++d)
    for (int so = 0; so < 2; ++so)
      for (int si = 0; si < 2; ++si) {
        float2 acc = cz();
        for (int u = 0; u < 2; ++u)
          for (int v = 0; v < 2; ++v) {
            float2 core;
            if (on) {
              core = side == 0 ? b.WL[(u * 2 + v) * 4 + d] : b.WR[(d * 2 + u) * 2 + v];
            } else {
              core = make_float2((u == v && d == 0) ? 1.f : 0.f, 0.f);
            }
            cfma(acc, cmul(Post[so * 2 + u], core), Pre[v * 2 + si]);
          }
        if (side == 0) W[(so * 2 + si) * D + d] = acc;   // [0][so][si][d]
        else W[(d * 2 + so) * 2 + si] = acc;             // [d][so][si][0]
      }
  *dl_out = side == 0 ? 1 : D;
  *dr_out = side == 0 ? D : 1;
}

// G_blk = (Post_q x Post_{q+1}) G2 (Pre_q x Pre_{q+1}), row-major 4x4.  One thread.
static __device__ __noinline__ void build_block(const DBlock& b, const DGate1* G1, const uint64_t* c, float2* G) {
  if (b.composed) {
    for (int i = 0; i < 16; ++i) G[i] = b.Gc[i];
    return;
  }
  float2 Pre0[4], Post0[4], Pre1[4], Post1[4];
  prod1q(G1, b.pre_off[0], b.pre_n[0], c, Pre0);
  prod1q(G1, b.post_off[0], b.post_n[0], c, Post0);
  prod1q(G1, b.pre_off[1], b.pre_n[1], c, Pre1);
  prod1q(G1, b.post_off[1], b.post_n[1], c, Post1);
  const bool on = cond_holds(b.cond, c);
  float2 M[16];
  // M = G2 (Pre0 x Pre1)
  for (int o = 0; o < 4; ++o)
    for (int i = 0; i < 4; ++i) {
      const int t0 = i >> 1, t1 = i & 1;
      float2 acc = cz();
      for (int k = 0; k < 4; ++k) {
        const int b0 = k >> 1, b1 = k & 1;
        const float2 g = on ? b.G[o * 4 + k] : make_float2(o == k ? 1.f : 0.f, 0.f);
        cfma(acc, g, cmul(Pre0[b0 * 2 + t0], Pre1[b1 * 2 + t1]));
      }
      M[o * 4 + i] = acc;
    }
  for (int o = 0; o < 4; ++o)
    for (int i = 0; i < 4; ++i) {
      const int s0 = o >> 1, s1 = o & 1;
      float2 acc = cz();
      for (int k = 0; k < 4; ++k) {
        const int a0 = k >> 1, a1 = k & 1;
        cfma(acc, cmul(Post0[s0 * 2 + a0], Post1[s1 * 2 + a1]), M[k * 4 + i]);
      }
      G[o * 4 + i] = acc;
    }
}

__device__ __forceinline__ float2* site_ptr(const DevCtx& c, int buf, int slot, int j) {
  return c.mps[buf] + (size_t)slot * c.mps_slot_stride + __ldg(c.site_off + j);
}
__device__ __forceinline__ float2* env_ptr(const DevCtx& c, int slot, int b) {
  return c.env + (size_t)slot * c.env_slot_stride + __ldg(c.env_off + b);
}
__device__ __forceinline__ int* bonds_ptr(const DevCtx& c, int slot, int buf) {
  return c.bonds + ((size_t)slot * 2 + buf) * (c.n + 1);
}

template <int NT>
__device__ __forceinline__ void gcopy(float2* dst, const float2* src, int n) {
  for (int i = threadIdx.x; i < n; i += NT) dst[i] = src[i];
}

// ----------------------------------------------------------------------------- contractions
// C1: T[b][d][t][x] = sum_a E[b][d][a] S[a][t][x]; T strides (2 Dm nx, 2 nx, nx, 1).
template <int NT>
static __device__ void c1_env_site(const float2* E, const float2* S, float2* T, int nb, int nd, int na,
                            int nx, int Dm) {
  const int tot = nb * nd * 2 * nx;
  for (int idx = threadIdx.x; idx < tot; idx += NT) {
    const int x = idx % nx;
    int r = idx / nx;
    const int t = r & 1;
    r >>= 1;
    const int d = r % nd, b = r / nd;
    const float2* e = E + (b * nd + d) * na;
    const float2* s = S + t * nx + x;
    float2 acc = cz();
    for (int a = 0; a < na; ++a) cfma(acc, e[a], s[a * 2 * nx]);
    T[b * 2 * Dm * nx + (d * 2 + t) * nx + x] = acc;
  }
  __syncthreads();
}

// C2 (in place): per fiber (b, x), T2[b][s][e][x] = sum_{d,t} T1[b][d][t][x] W[d][s][t][e].
template <int NT>
static __device__ void c2_mix(float2* T, const float2* W, int nb, int nd, int ne, int nx, int Dm) {
  for (int idx = threadIdx.x; idx < nb * nx; idx += NT) {
    const int x = idx % nx, b = idx / nx;
    float2* base = T + b * 2 * Dm * nx + x;
    float2 v[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = (m < 2 * nd) ? base[m * nx] : cz();
    float2 w[8];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        float2 acc = cz();
        if (e < ne) {
#pragma unroll
          for (int d = 0; d < 4; ++d)
#pragma unroll
            for (int t = 0; t < 2; ++t)
              if (d < nd) cfma(acc, v[d * 2 + t], W[((d * 2 + s) * 2 + t) * ne + e]);
        }
        w[s * 4 + e] = acc;
      }
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (e < ne) base[(s * ne + e) * nx] = w[s * 4 + e];
  }
  __syncthreads();
}

// C3: F[(b s) + c ldx] = sum_{e,x} T2[b][s][e][x] R[c][e][x]   (column-major, ldx = 2 nb)
template <int NT>
static __device__ void c3_site_env(const float2* T, const float2* R, float2* F, int nb, int ne, int nx,
                            int nc, int Dm) {
  const int K = ne * nx;
  const int tot = nb * 2 * nc;
  for (int idx = threadIdx.x; idx < tot; idx += NT) {
    const int row = idx % (2 * nb), col = idx / (2 * nb);
    const int b = row >> 1, s = row & 1;
    const float2* t = T + b * 2 * Dm * nx + s * ne * nx;
    const float2* r = R + col * K;
    float2 acc = cz();
    for (int k = 0; k < K; ++k) cfma(acc, t[k], r[k]);
    F[row + col * 2 * nb] = acc;
  }
  __syncthreads();
}

// C4: Enew[c][e][x] = sum_{b,s} conj(Q[(b s) + c ldq]) T2[b][s][e][x],  c < k
template <int NT>
static __device__ void c4_env_update(const float2* Q, int ldq, const float2* T, float2* En, int nb,
                              int ne, int nx, int k, int Dm) {
  const int tot = k * ne * nx;
  for (int idx = threadIdx.x; idx < tot; idx += NT) {
    const int x = idx % nx;
    const int r = idx / nx;
    const int e = r % ne, cc = r / ne;
    float2 acc = cz();
    for (int b = 0; b < nb; ++b)
#pragma unroll
      for (int s = 0; s < 2; ++s)
        cfmac(acc, Q[(b * 2 + s) + cc * ldq], T[b * 2 * Dm * nx + (s * ne + e) * nx + x]);
    En[idx] = acc;
  }
  __syncthreads();
}

// ----------------------------------------------------------------------------- working set
// Working set of one slot.  The small arrays always live in shared memory.  The five large
// tiles (E 4C^2, S 2C^2, T 8C^2, R 4C^2, F 2C^2 complex) live in shared memory for tile
// capacity C <= 32, and in the slot's global work area above that, where T2 (8C^2, the
// mixed T of the large-tile path) and the GEMM staging tiles are added.
struct Work {
  float2* E;   // environment (in / out)
  float2* S;   // site tensor
  float2* T;   // T1/T2 (small path), T1 (large path), or Theta + V
  float2* R;   // far environment, or Q
  float2* F;   // F (QR work)
  float2* T2;  // mixed T (large path)
  float2* Wc;  // composed MPO tensor of a chunk of several layers, then 3 x 64 factors
  float2* W;   // 64     MPO tensor of the site
  float2* W2;  // 64     mirrored MPO tensor
  float2* G;   // 16     block matrix / single-qubit gate
  float2* alph;
  float2* gA;  // GEMM staging tiles (large path)
  float2* gB;
  TcState tc;  // tensor-core GEMM state (large path with precision TF32X3)
  bool use_tc;
  float2* stage;       // large path: shared staging of the blocked SVD (aliases tc.stage)
  size_t stage_elems;  // its size in complex elements
  double* red;
  double* sig2;
  double* dv;  // scalar broadcast
  float* tau;
  float* sigf;  // singular values squared, FP32 (2C)
  int* perm;
  int* bnd;    // bonds being modified [n+1]
  int* abnd;   // bonds of the ket [n+1]
  int* iv;     // small ints
  uint64_t* creg;
  int C;       // tile capacity
};


__host__ __device__ inline size_t work_arrays_bytes(int C, bool big) {
  (void)big;
  return sizeof(float2) * (64 + 64 + 16 + 2 * C) +
         sizeof(double) * (32 + 2 * C + 8) + sizeof(float) * 4 * C +
         sizeof(int) * (2 * C + 2 * (DCS_MAX_QUBITS + 1) + 16) + sizeof(uint64_t) * DCS_CWORDS + 64;
}
// Large path: a 128-byte head (tensor-core barriers and counters) and a staging region that
// serves the tensor-core GEMM tiles, the SIMT GEMM tiles and the blocked SVD in turn, filling
// the CTA's shared memory up to 224 KB.
constexpr size_t BIG_SMEM_BYTES = 224 * 1024;
constexpr size_t BIG_HEAD_BYTES = 128;
static_assert(TC_HEAD_BYTES <= (int)BIG_HEAD_BYTES, "tensor-core barriers exceed the head");
__host__ __device__ inline size_t big_stage_bytes(int C) {
  const size_t rest = work_arrays_bytes(C, true) + BIG_HEAD_BYTES;
  return rest < BIG_SMEM_BYTES ? ((BIG_SMEM_BYTES - rest) & ~(size_t)127) : 0;
}
__host__ __device__ inline size_t work_small_bytes(int C, bool big, bool tc = false) {
  (void)tc;
  return work_arrays_bytes(C, big) + (big ? BIG_HEAD_BYTES + big_stage_bytes(C) : 0);
}
// Composed chunk MPO tensors (complex elements): the final one of bond <= dmax and the
// intermediates (at least one factor's 64).
__host__ __device__ inline size_t chunk_w_fin_elems(int dmax) { return 4 * (size_t)dmax * dmax; }
__host__ __device__ inline size_t chunk_w_mid_elems(int d) {
  const size_t e = 4 * (size_t)d * d;
  return e < 64 ? 64 : e;
}
// Large path: E dmax C^2, S 2 C^2, T 2 dmax C^2, R dmax C^2, F 2 C^2, T2 2 dmax C^2 and, for
// chunks of several layers, the composed MPO tensor, two intermediates and one 2 x 2 x 4 x 4
// factor per layer; with dmax = 4 the tiles are 28 C^2.
__host__ __device__ inline size_t work_tile_elems(int C, bool big, int dmax = 4) {
  if (!big) return (size_t)20 * C * C;
  return (size_t)(6 * dmax + 4) * C * C +
         (dmax > 4 ? chunk_w_fin_elems(dmax) + chunk_w_mid_elems(dmax / 4) +
                         chunk_w_mid_elems(dmax / 16) + 64 * DCS_MAX_CHUNK_LAYERS
                   : 0);
}

static __device__ void carve(Work& w, unsigned char* raw, int C, float2* big_area, bool tc = false,
                             int dmax = 4) {
  w.C = C;
  w.use_tc = tc;
  w.tc.bf16 = false;  // set by the tensor-core kernels after tc_setup; read by the gauge moves
  w.stage = nullptr;
  w.stage_elems = 0;
  if (big_area) {  // head (barriers, counters), then the 128-byte aligned staging region
    uint64_t* head = reinterpret_cast<uint64_t*>(raw);
    w.tc.mbar = head;
    w.tc.uses = reinterpret_cast<int*>(head + TC_NBAR);
    w.tc.tmem = reinterpret_cast<uint32_t*>(w.tc.uses + 2);
    w.tc.err = reinterpret_cast<int*>(w.tc.tmem + 1);
    raw += BIG_HEAD_BYTES;
    w.stage = reinterpret_cast<float2*>(raw);
    w.stage_elems = big_stage_bytes(C) / sizeof(float2);
    w.tc.stage = reinterpret_cast<float*>(raw);
    w.tc.stage_bytes = big_stage_bytes(C);
    raw += big_stage_bytes(C);
  }
  uint64_t* c64 = reinterpret_cast<uint64_t*>(raw);
  w.creg = c64;
  double* d = reinterpret_cast<double*>(c64 + DCS_CWORDS);
  w.red = d;
  w.sig2 = w.red + 32;
  w.dv = w.sig2 + 2 * C;
  float2* f2 = reinterpret_cast<float2*>(w.dv + 8);
  w.W = f2;
  w.W2 = w.W + 64;
  w.G = w.W2 + 64;
  w.alph = w.G + 16;
  float2* tiles = w.alph + 2 * C;
  if (big_area) {  // the SIMT GEMM tiles share the staging region
    w.gA = w.stage;
    w.gB = w.gA + GBM * GSA_LD;
  } else {
    w.gA = w.gB = nullptr;
  }
  float2* t = big_area ? big_area : tiles;
  const int dm = big_area ? dmax : 4;
  w.E = t;
  w.S = w.E + (size_t)dm * C * C;
  w.T = w.S + 2 * C * C;
  w.R = w.T + (size_t)2 * dm * C * C;
  w.F = w.R + (size_t)dm * C * C;
  w.T2 = big_area ? w.F + 2 * C * C : nullptr;
  w.Wc = (big_area && dm > 4) ? w.T2 + (size_t)2 * dm * C * C : nullptr;
  float2* after = big_area ? tiles : w.F + 2 * C * C;
  w.tau = reinterpret_cast<float*>(after);
  w.sigf = w.tau + 2 * C;
  w.perm = reinterpret_cast<int*>(w.sigf + 2 * C);
  w.bnd = w.perm + 2 * C;
  w.abnd = w.bnd + DCS_MAX_QUBITS + 1;
  w.iv = w.abnd + DCS_MAX_QUBITS + 1;
}

// Complex GEMM of the large tiles: tensor cores when enabled, the shape fills at least half
// an MMA tile in M and N and K spans 16 stages or more (shorter products, such as the panel
// updates of the blocked QR, cost more in pipeline set-up than they save), the SIMT tiles
// otherwise.
template <int NT>
__device__ __forceinline__ void wgemm(Work& sm, int M, int N, int K, const float2* A, int sam,
                                      int sak, bool conjA, const float2* B, int sbk, int sbn,
                                      bool conjB, float2* Cm, int scm, int scn) {
  if constexpr (NT >= 128) {
#if DCS_TU_TENSOR_CORES
    if (sm.use_tc && M >= 64 && N >= 64 && K >= 128) {
      cta_cgemm_tc<NT>(M, N, K, A, sam, sak, conjA, B, sbk, sbn, conjB, Cm, scm, scn, sm.tc);
      return;
    }
#endif
    cta_cgemm<NT>(M, N, K, A, sam, sak, conjA, B, sbk, sbn, conjB, Cm, scm, scn, sm.gA, sm.gB);
  }
}

// ----------------------------------------------------------------------------- blocked QR
constexpr int QR_PB = 64;  // panel width of the blocked QR

// Scratch (complex elements) of cta_qr_blocked for an m x n matrix.
__host__ __device__ inline size_t qr_blocked_scratch(int m, int n) {
  const int r = m < n ? m : n;
  const size_t panels = (size_t)(r + QR_PB - 1) / QR_PB;
  return panels * QR_PB * QR_PB + (size_t)m * QR_PB + 2 * (size_t)QR_PB * n + (size_t)m * n;
}

// Householder QR of F (m x n, column-major, ld m) with the explicit Q (m x r, r = min(m, n),
// column-major, ldq) and no R; the reflectors are those of cta_qr.  Blocked: panels of
// QR_PB columns are factored with house_columns; the panel's reflectors are gathered into
// U (zeros above each reflector) with the compact WY form H_0 ... H_{b-1} = I - U T U^H,
// T upper triangular (T_jj = tau_j, T[0:j, j] = -tau_j T[0:j, 0:j] U[:, 0:j]^H u_j); the
// columns right of the panel take F -= U T^H (U^H F) in three GEMMs, and Q is accumulated
// from the right, Q -= U T (U^H Q) per panel.  The GEMMs go through wgemm (tensor cores on
// the TF32X3 path).  ws: qr_blocked_scratch(m, n) complex in global memory.  With Q null
// only the factorisation runs: R is then F's strict upper triangle with the diagonal in
// sm.alph[0 .. r).
template <int NT>
static __device__ int cta_qr_blocked(Work& sm, float2* F, int m, int n, float2* Q, int ldq, float2* ws) {
  const int r = m < n ? m : n;
  const int npan = (r + QR_PB - 1) / QR_PB;
  float2* Tall = ws;                                   // npan x QR_PB x QR_PB, row-major
  float2* U = Tall + (size_t)npan * QR_PB * QR_PB;     // mu x pb, column-major (ld mu)
  float2* W = U + (size_t)m * QR_PB;                   // pb x cols, row-major
  float2* W2 = W + (size_t)QR_PB * n;                  // pb x cols, row-major
  float2* Y = W2 + (size_t)QR_PB * n;                  // mu x cols, column-major (ld mu)
  // U of panel p0 from the reflectors stored in F
  auto gather_u = [&](int p0, int pb) {
    const int mu = m - p0;
    for (int idx = threadIdx.x; idx < mu * pb; idx += NT) {
      const int i = idx % mu, j = idx / mu;
      U[idx] = (i >= j && sm.tau[p0 + j] != 0.f) ? F[(size_t)(p0 + i) + (size_t)(p0 + j) * m] : cz();
    }
    __syncthreads();
  };
  for (int p = 0; p < npan; ++p) {
    const int p0 = p * QR_PB, pb = (r - p0) < QR_PB ? (r - p0) : QR_PB, mu = m - p0;
    house_columns<NT>(F, m, m, p0, p0 + pb, p0 + pb, sm.tau, sm.alph, sm.red);
    __syncthreads();
    gather_u(p0, pb);
    // S = U^H U into W, then T column by column (one thread per row of T), both in the
    // staging area (free between GEMMs) when it holds them, T copied out for the GEMMs
    float2* T = Tall + (size_t)p * QR_PB * QR_PB;
    wgemm<NT>(sm, pb, pb, mu, U, mu, 1, true, U, 1, mu, false, W, pb, 1);
    const bool staged = sm.stage != nullptr && sm.stage_elems >= (size_t)2 * QR_PB * QR_PB;
    float2* sS = staged ? sm.stage : W;                       // S, ld pb
    float2* sT = staged ? sm.stage + QR_PB * QR_PB : T;       // T, ld QR_PB
    if (staged) {
      for (int idx = threadIdx.x; idx < pb * pb; idx += NT) sS[idx] = W[idx];
      __syncthreads();
    }
    for (int j = 0; j < pb; ++j) {
      const float tj = sm.tau[p0 + j];
      if ((int)threadIdx.x < pb) {
        const int i = threadIdx.x;
        float2 v = cz();
        if (i < j) {
          for (int l = i; l < j; ++l) cfma(v, sT[i * QR_PB + l], sS[l * pb + j]);
          v = cscale(v, -tj);
        } else if (i == j) {
          v = make_float2(tj, 0.f);
        }
        sT[i * QR_PB + j] = v;
      }
      __syncthreads();
    }
    if (staged) {
      for (int idx = threadIdx.x; idx < pb * QR_PB; idx += NT) {
        const int i = idx / QR_PB, j = idx % QR_PB;
        if (j < pb) T[idx] = sT[idx];
      }
      __syncthreads();
    }
    const int nt = n - p0 - pb;
    if (nt > 0) {
      float2* Ft = F + (size_t)p0 + (size_t)(p0 + pb) * m;
      wgemm<NT>(sm, pb, nt, mu, U, mu, 1, true, Ft, 1, m, false, W, nt, 1);
      wgemm<NT>(sm, pb, nt, pb, T, 1, QR_PB, true, W, nt, 1, false, W2, nt, 1);
      wgemm<NT>(sm, mu, nt, pb, U, 1, mu, false, W2, nt, 1, false, Y, 1, mu);
      for (int idx = threadIdx.x; idx < mu * nt; idx += NT) {
        const int i = idx % mu, j = idx / mu;
        float2& f = Ft[(size_t)i + (size_t)j * m];
        f = csub(f, Y[idx]);
      }
      __syncthreads();
    }
  }
  if (Q == nullptr) return r;
  // Q = H_0 ... H_{r-1} [I_r; 0], panels applied from the last one
  for (int idx = threadIdx.x; idx < m * r; idx += NT) {
    const int i = idx % m, j = idx / m;
    Q[(size_t)i + (size_t)j * ldq] = make_float2(i == j ? 1.f : 0.f, 0.f);
  }
  __syncthreads();
  for (int p = npan - 1; p >= 0; --p) {
    const int p0 = p * QR_PB, pb = (r - p0) < QR_PB ? (r - p0) : QR_PB, mu = m - p0;
    const int qc = r - p0;
    gather_u(p0, pb);
    const float2* T = Tall + (size_t)p * QR_PB * QR_PB;
    float2* Qs = Q + (size_t)p0 + (size_t)p0 * ldq;
    wgemm<NT>(sm, pb, qc, mu, U, mu, 1, true, Qs, 1, ldq, false, W, qc, 1);
    wgemm<NT>(sm, pb, qc, pb, T, QR_PB, 1, false, W, qc, 1, false, W2, qc, 1);
    wgemm<NT>(sm, mu, qc, pb, U, 1, mu, false, W2, qc, 1, false, Y, 1, mu);
    for (int idx = threadIdx.x; idx < mu * qc; idx += NT) {
      const int i = idx % mu, j = idx / mu;
      float2& q = Qs[(size_t)i + (size_t)j * ldq];
      q = csub(q, Y[idx]);
    }
    __syncthreads();
  }
  return r;
}

// QR of a sweep's F (m x n in the work area) into Q = sm.R: the blocked form when the panel
// pays off and its scratch fits the T tile (free at this point of a site update), else cta_qr.
template <int NT>
__device__ __forceinline__ int sweep_qr(Work& sm, int m, int n) {
  if (n >= 2 * QR_PB && m >= QR_PB && qr_blocked_scratch(m, n) <= (size_t)8 * sm.C * sm.C)
    return cta_qr_blocked<NT>(sm, sm.F, m, n, sm.R, m, sm.T);
  return cta_qr<NT>(sm.F, m, n, m, sm.R, m, nullptr, 0, sm.tau, sm.alph, sm.red);
}

// ----------------------------------------------------------------------------- gauge moves
// A gauge move of an m x n site matrix takes the blocked QR (panels + GEMMs) when the tiles
// are in the global work area, the panel pays off and its scratch fits the T tile.
template <int NT>
__device__ __forceinline__ bool hop_blocked(const Work& sm, int m, int n) {
  return NT >= 128 && sm.gA != nullptr && n >= 2 * QR_PB && m >= QR_PB &&
         qr_blocked_scratch(m, n) <= (size_t)8 * sm.C * sm.C;
}

// Move the orthogonality centre of MPS buffer `buf` of `slot` from j to j+1:
// T_j = Q R (as (2 b_j) x b_{j+1}), T_j := Q, T_{j+1} := R T_{j+1}.
template <int NT>
static __device__ void hop_right(const DevCtx& c, Work& sm, int buf, int slot, int j) {
  int* b = sm.bnd;
  const int bl = b[j], br = b[j + 1], bn = b[j + 2];
  const int m = 2 * bl;
  const float2* src = site_ptr(c, buf, slot, j);
  for (int idx = threadIdx.x; idx < m * br; idx += NT) {
    const int row = idx / br, x = idx % br;  // row = a*2 + s
    sm.F[row + x * m] = src[idx];
  }
  __syncthreads();
  float2* dst = site_ptr(c, buf, slot, j);
  int r;
  if (hop_blocked<NT>(sm, m, br)) {
    // large tiles: blocked Householder QR for Q, then R = Q^H T_j (one GEMM on the
    // untouched site), FP32-accurate products
    r = cta_qr_blocked<NT>(sm, sm.F, m, br, sm.R, m, sm.T);
    const bool tc = sm.use_tc;
    sm.use_tc = tc && !sm.tc.bf16;
    wgemm<NT>(sm, r, br, m, sm.R, m, 1, true, src, br, 1, false, sm.E, br, 1);
    sm.use_tc = tc;
    __syncthreads();
  } else {
    r = cta_qr<NT>(sm.F, m, br, m, sm.R, m, sm.E, br, sm.tau, sm.alph, sm.red);
  }
  for (int idx = threadIdx.x; idx < m * r; idx += NT) {
    const int row = idx / r, k = idx % r;
    dst[idx] = sm.R[row + k * m];
  }
  const float2* nx = site_ptr(c, buf, slot, j + 1);
  if (NT >= 128 && sm.gA) {  // large tiles: R (r x br) times T_{j+1} (br x 2 bn), tiled GEMM
    wgemm<NT>(sm, r, 2 * bn, br, sm.E, br, 1, false, nx, 2 * bn, 1, false, sm.T, 2 * bn, 1);
  } else {
    gcopy<NT>(sm.S, nx, br * 2 * bn);
    __syncthreads();
    for (int idx = threadIdx.x; idx < r * 2 * bn; idx += NT) {
      const int k = idx / (2 * bn), col = idx % (2 * bn);
      float2 acc = cz();
      for (int x = 0; x < br; ++x) cfma(acc, sm.E[k * br + x], sm.S[x * 2 * bn + col]);
      sm.T[idx] = acc;
    }
    __syncthreads();
  }
  gcopy<NT>(site_ptr(c, buf, slot, j + 1), sm.T, r * 2 * bn);
  __syncthreads();
  if (threadIdx.x == 0) b[j + 1] = r;
  __syncthreads();
}

// Move the centre from j to j-1 (mirrored hop): T_j[a][t][x] read as (x t) x a = Q' R',
// T_j[k][t][x] := Q'[(x t), k], T_{j-1}[a'][s][k] := sum_a T_{j-1}[a'][s][a] R'[k][a].
template <int NT>
static __device__ void hop_left(const DevCtx& c, Work& sm, int buf, int slot, int j) {
  int* b = sm.bnd;
  const int bl = b[j], br = b[j + 1], bp = b[j - 1];
  const int m = 2 * br;
  const float2* src = site_ptr(c, buf, slot, j);
  for (int idx = threadIdx.x; idx < bl * 2 * br; idx += NT) {
    const int x = idx % br, t = (idx / br) & 1, a = idx / (2 * br);
    sm.F[(x * 2 + t) + a * m] = src[idx];
  }
  __syncthreads();
  float2* dst = site_ptr(c, buf, slot, j);
  int r;
  if (hop_blocked<NT>(sm, m, bl)) {
    // large tiles: blocked QR for Q', then R' = Q'^H T_j' from a copy of T_j' ((x t) x a,
    // in the S tile, which the large path does not use otherwise)
    gcopy<NT>(sm.S, sm.F, m * bl);
    __syncthreads();
    r = cta_qr_blocked<NT>(sm, sm.F, m, bl, sm.R, m, sm.T);
    const bool tc = sm.use_tc;
    sm.use_tc = tc && !sm.tc.bf16;
    wgemm<NT>(sm, r, bl, m, sm.R, m, 1, true, sm.S, 1, m, false, sm.E, bl, 1);
    sm.use_tc = tc;
    __syncthreads();
  } else {
    r = cta_qr<NT>(sm.F, m, bl, m, sm.R, m, sm.E, bl, sm.tau, sm.alph, sm.red);
  }
  for (int idx = threadIdx.x; idx < r * 2 * br; idx += NT) {
    const int x = idx % br, t = (idx / br) & 1, k = idx / (2 * br);
    dst[idx] = sm.R[(x * 2 + t) + k * m];
  }
  if (NT >= 128 && sm.gA) {  // large tiles: T_{j-1} ((2 bp) x bl) times R'^T (bl x r)
    __syncthreads();
    wgemm<NT>(sm, 2 * bp, r, bl, site_ptr(c, buf, slot, j - 1), bl, 1, false, sm.E, 1, bl, false,
              sm.T, r, 1);
  } else {
    gcopy<NT>(sm.S, site_ptr(c, buf, slot, j - 1), bp * 2 * bl);
    __syncthreads();
    for (int idx = threadIdx.x; idx < bp * 2 * r; idx += NT) {
      const int k = idx % r, row = idx / r;
      float2 acc = cz();
      for (int a = 0; a < bl; ++a) cfma(acc, sm.S[row * bl + a], sm.E[k * bl + a]);
      sm.T[idx] = acc;
    }
    __syncthreads();
  }
  gcopy<NT>(site_ptr(c, buf, slot, j - 1), sm.T, bp * 2 * r);
  __syncthreads();
  if (threadIdx.x == 0) b[j] = r;
  __syncthreads();
}

// Every bond <= 4, one warp per slot: the orthogonality-centre tensor T_j rides in
// registers (warp layout of warp_qr8x4) through runs of centre moves and measurements.  In
// the right layout its matrix is rows (a s) = a * 2 + s, columns x; in the left layout rows
// (x s) = x * 2 + s, columns a.  Each hop is the same gauge move as hop_right / hop_left;
// only the hop's Q goes to memory, and the centre tensor when the run ends.
struct Roll {
  float2 x;    // T_j[a][s][x] in the current layout, zero outside
  int j;       // site
  int bl, br;  // its bonds
  bool right;  // layout
};

__device__ __forceinline__ int roll_lane_row() { return threadIdx.x & 7; }
__device__ __forceinline__ int roll_lane_col() { return (threadIdx.x & 31) >> 3; }

// element offset of this lane's entry inside the packed site [bl][2][br], or -1
__device__ __forceinline__ int roll_offset(const Roll& R) {
  const int row = roll_lane_row(), col = roll_lane_col();
  if (R.right) return (row < 2 * R.bl && col < R.br) ? row * R.br + col : -1;
  return (row < 2 * R.br && col < R.bl) ? (col * 2 + (row & 1)) * R.br + (row >> 1) : -1;
}

__device__ __forceinline__ void roll_load(const DevCtx& c, const Work& sm, int buf, int slot,
                                          int j, bool right, Roll& R) {
  R.j = j;
  R.bl = sm.bnd[j];
  R.br = sm.bnd[j + 1];
  R.right = right;
  const int off = roll_offset(R);
  R.x = off >= 0 ? site_ptr(c, buf, slot, j)[off] : cz();
}

__device__ __forceinline__ void roll_store(const DevCtx& c, int buf, int slot, const Roll& R) {
  const int off = roll_offset(R);
  if (off >= 0) site_ptr(c, buf, slot, R.j)[off] = R.x;
}

// switch layouts: lane (col u, row v * 2 + s) takes lane (col v, row u * 2 + s)
__device__ __forceinline__ void roll_flip(Roll& R) {
  const int row = roll_lane_row(), col = roll_lane_col();
  const float2 v = shfl2(R.x, (row >> 1) * 8 + col * 2 + (row & 1));
  const bool ok = R.right ? (col < R.bl && (row >> 1) < R.br) : (col < R.br && (row >> 1) < R.bl);
  R.x = ok ? v : cz();
  R.right = !R.right;
}

// centre j -> j+1 (right layout): T_j = Q R, T_j := Q, T_{j+1} := R T_{j+1}
__device__ __forceinline__ void roll_hop_right(const DevCtx& c, Work& sm, int buf, int slot, Roll& R) {
  const int lane = threadIdx.x & 31, row = roll_lane_row(), col = roll_lane_col();
  const int j = R.j, bl = R.bl, br = R.br, bn = sm.bnd[j + 2];
  float2 q;
  const int r = warp_qr8x4(R.x, 2 * bl, br, q);
  if (row < 2 * bl && col < r) site_ptr(c, buf, slot, j)[row * r + col] = q;
  const float2* nx = site_ptr(c, buf, slot, j + 1);
  const int k = row >> 1, sp = row & 1;
  const bool live = k < r && col < bn;
  float2 acc = cz();
  for (int y = 0; y < br; ++y) {
    const float2 ry = shfl2(R.x, y * 8 + k);
    if (live) cfma(acc, ry, nx[(y * 2 + sp) * bn + col]);
  }
  R.x = live ? acc : cz();
  if (lane == 0) sm.bnd[j + 1] = r;
  __syncwarp();
  R.j = j + 1;
  R.bl = r;
  R.br = bn;
}

// centre j -> j-1 (left layout): T_j read as (x t) x a = Q' R', T_j[k][t][x] := Q'[(x t)][k],
// T_{j-1}[a'][s][k] := sum_a T_{j-1}[a'][s][a] R'[k][a]
__device__ __forceinline__ void roll_hop_left(const DevCtx& c, Work& sm, int buf, int slot, Roll& R) {
  const int lane = threadIdx.x & 31, row = roll_lane_row(), col = roll_lane_col();
  const int j = R.j, bl = R.bl, br = R.br, bp = sm.bnd[j - 1];
  float2 q;
  const int r = warp_qr8x4(R.x, 2 * br, bl, q);
  if (row < 2 * br && col < r) site_ptr(c, buf, slot, j)[(col * 2 + (row & 1)) * br + (row >> 1)] = q;
  const float2* pv = site_ptr(c, buf, slot, j - 1);
  const int k = row >> 1, sp = row & 1;
  const bool live = k < r && col < bp;
  float2 acc = cz();
  for (int a = 0; a < bl; ++a) {
    const float2 ra = shfl2(R.x, a * 8 + k);
    if (live) cfma(acc, pv[(col * 2 + sp) * bl + a], ra);
  }
  R.x = live ? acc : cz();
  if (lane == 0) sm.bnd[j] = r;
  __syncwarp();
  R.j = j - 1;
  R.br = r;
  R.bl = bp;
}

__device__ __forceinline__ void roll_move(const DevCtx& c, Work& sm, int buf, int slot, Roll& R,
                                          int target) {
  if (target > R.j) {
    if (!R.right) roll_flip(R);
    while (R.j < target) roll_hop_right(c, sm, buf, slot, R);
  } else if (target < R.j) {
    if (R.right) roll_flip(R);
    while (R.j > target) roll_hop_left(c, sm, buf, slot, R);
  }
}

static __device__ void warp_move_centre4(const DevCtx& c, Work& sm, int buf, int slot, int& centre,
                                  int target) {
  if (centre == target) return;
  Roll R;
  roll_load(c, sm, buf, slot, centre, target > centre, R);
  roll_move(c, sm, buf, slot, R, target);
  roll_store(c, buf, slot, R);
  centre = target;
  __syncwarp();
}

// A run of measurements (Alg. 1 Measure / MeasureProb) with the centre tensor in registers:
// the same steps as the general path of k_measure, for every bond <= 4.
static __device__ void warp_measure_run4(const DevCtx& c, Work& sm, int kb, int slot, int centre,
                                  const DMeas* meas, int n_meas, int mode,
                                  const uint8_t* forced, double* p0_out) {
  const int lane = threadIdx.x & 31, row = lane & 7;
  Roll R;
  roll_load(c, sm, kb, slot, centre, n_meas == 0 || meas[0].q >= centre, R);
  for (int im = 0; im < n_meas; ++im) {
    const int q = meas[im].q;
    roll_move(c, sm, kb, slot, R, q);
    // slice weights r_s = sum |T_q[:, s, :]|^2 and p_0 = r_0 / (r_0 + r_1), all in float-float
    // (about 2^-44 relative, FP32 pipe); the slice is the row's low bit
    const ffloat w = ff_abs2(R.x);
    const ffloat z{0.f, 0.f};
    const ffloat r0 = ff_warp_sum((row & 1) ? z : w);
    const ffloat r1 = ff_warp_sum((row & 1) ? w : z);
    const ffloat p0 = ff_div(r0, ff_add(r0, r1));
    if (mode == MEAS_PROB) {
      if (lane == 0) {
        const double p0d = ff_to_double(p0);
        if (p0_out) p0_out[slot] = p0d;
        c.rr[2 * (size_t)slot] = ff_to_double(r0);
        c.rr[2 * (size_t)slot + 1] = ff_to_double(r1);
        if (!(p0d == p0d)) c.flags[slot] |= DCS_FLAG_NUMERICAL;
      }
      continue;
    }
    int m;
    if (mode == MEAS_SAMPLE) {
      // m = 0 iff u < p_0; u within 2^-48 of the FP64 uniform, so only draws far inside
      // the flagged window |u - p_0| < 1e-6 could be decided differently
      uint32_t hi27, lo26;
      philox_words(c.seed, c.shot[slot], meas[im].ordinal, hi27, lo26);
      const ffloat u = ff_uniform(hi27, lo26);
      m = ff_cmp(u, p0) < 0 ? 0 : 1;
      const ffloat d = ff_add(u, ff_neg(p0));
      if (lane == 0 && fabsf(d.hi) < 1e-6f) c.flags[slot] |= DCS_FLAG_DRAW_NEAR_THRESHOLD;
    } else {
      m = forced[slot] ? 1 : 0;
    }
    const ffloat one{1.f, 0.f};
    const ffloat pm = m ? ff_add(one, ff_neg(p0)) : p0;
    const ffloat rm = m ? r1 : r0;
    if (!(pm.hi > 1e-12f)) {
      if (lane == 0) c.flags[slot] |= (pm.hi == pm.hi) ? DCS_FLAG_ZERO_PROB : DCS_FLAG_NUMERICAL;
      continue;
    }
    const float sc = 1.f / sqrtf(rm.hi);
    R.x = (row & 1) == m ? cscale(R.x, sc) : cz();
    if (lane == 0) {
      c.p[slot] *= ff_to_double(pm);
      const int cb = meas[im].cbit;
      uint64_t& wd = c.creg[(size_t)slot * DCS_CWORDS + (cb >> 6)];
      wd = (wd & ~(1ull << (cb & 63))) | ((uint64_t)m << (cb & 63));
    }
  }
  roll_store(c, kb, slot, R);
  __syncwarp();
  int* kbonds = bonds_ptr(c, slot, kb);
  for (int i = lane; i <= c.n; i += 32) kbonds[i] = sm.bnd[i];
  if (lane == 0) c.centre[slot] = R.j;
}

// Sites [lo, hi] of buffer `from` copied to buffer `to`, bond dimensions `bd`; every bond
// <= 4: one thread per site.  16-byte accesses when both sites start on a 16-byte boundary
// (the site stride, 2 C^2 complex, is even, so the pair read past an odd end stays inside
// the site); 8-byte ones otherwise (a caller's buffer in dcs_compress_noalloc).
template <int NT>
__device__ __forceinline__ void copy_sites4(const DevCtx& c, int to, int from, int slot, int lo,
                                            int hi, const int* bd) {
  for (int j = lo + (int)threadIdx.x; j <= hi; j += NT) {
    const int len = bd[j] * 2 * bd[j + 1];
    const float2* s2 = site_ptr(c, from, slot, j);
    float2* d2 = site_ptr(c, to, slot, j);
    if (((reinterpret_cast<uintptr_t>(s2) | reinterpret_cast<uintptr_t>(d2)) & 15) == 0) {
      const float4* s = reinterpret_cast<const float4*>(s2);
      float4* d = reinterpret_cast<float4*>(d2);
      for (int e = 0; e < (len + 1) / 2; ++e) d[e] = s[e];
    } else {
      for (int e = 0; e < len; ++e) d2[e] = s2[e];
    }
  }
}

// The chunk's lone single-qubit gates (sites of kind 1), one thread per site.
template <int NT>
__device__ __forceinline__ void apply_lone_1q_threads(const DevCtx& c, Work& sm, int buf,
                                                      int slot, const DLayer* L,
                                                      const DGate1* G1) {
  for (int j = threadIdx.x; j < c.n; j += NT) {
    if (L->site[j].kind != 1) continue;
    float2 U[4];
    prod1q(G1, L->site[j].g_off, L->site[j].g_n, sm.creg, U);
    float2* p = site_ptr(c, buf, slot, j);
    const int bl = sm.bnd[j], br = sm.bnd[j + 1];
    for (int a = 0; a < bl; ++a)
      for (int x = 0; x < br; ++x) {
        const float2 v0 = p[(a * 2 + 0) * br + x], v1 = p[(a * 2 + 1) * br + x];
        float2 o0 = cz(), o1 = cz();
        cfma(o0, U[0], v0);
        cfma(o0, U[1], v1);
        cfma(o1, U[2], v0);
        cfma(o1, U[3], v1);
        p[(a * 2 + 0) * br + x] = o0;
        p[(a * 2 + 1) * br + x] = o1;
      }
  }
}

template <int NT>
static __device__ void move_centre(const DevCtx& c, Work& sm, int buf, int slot, int& centre,
                            int target) {
  if constexpr (NT == 32) {
    if (sm.C == 4) {
      warp_move_centre4(c, sm, buf, slot, centre, target);
      return;
    }
  }
  while (centre < target) {
    hop_right<NT>(c, sm, buf, slot, centre);
    ++centre;
  }
  while (centre > target) {
    hop_left<NT>(c, sm, buf, slot, centre);
    --centre;
  }
}

// ----------------------------------------------------------------------------- compression
// The sites the initial guess reads or writes form one interval [lo, hi]: the centre's path
// from where it stands through every block (q, q+1) of the chunk, plus every site a lone
// single-qubit gate acts on.  Only these sites are copied into the bra buffer up front; when
// the guess turns out exact they are copied back in place and the buffers are not swapped.
__device__ __forceinline__ void guess_range(const DLayer* L, const DBlock* BK, int n, int centre,
                                            int& lo, int& hi) {
  lo = hi = centre;
  for (int j = 0; j < n; ++j)
    if (L->site[j].kind == 1) {
      lo = j < lo ? j : lo;
      hi = j > hi ? j : hi;
    }
  for (int ib = 0; ib < L->n_blocks; ++ib) {
    const int q = BK[L->blk_off + ib].q;
    lo = q < lo ? q : lo;
    hi = q + 1 > hi ? q + 1 : hi;
  }
}

// Blocks (stored by decreasing q) are taken from the end of the layer nearest the centre:
// ascending when |centre - q_min| <= |centre - (q_max + 1)|.
__device__ __forceinline__ bool guess_ascending(const DLayer* L, const DBlock* BK, int centre) {
  const int nb = L->n_blocks;
  if (nb == 0) return true;
  const int qmin = BK[L->blk_off + nb - 1].q, qmax = BK[L->blk_off].q;
  const int dl = centre - qmin, dr = centre - (qmax + 1);
  return (dl < 0 ? -dl : dl) <= (dr < 0 ? -dr : dr);
}

// one warp per CTA for the small tiles: at most 64 registers so 32 CTAs fit an SM
template <int NT>
struct MinBlocks {
  static constexpr int value = NT == 32 ? 32 : (NT == 64 ? 16 : (NT == 128 ? 4 : 1));
};

// threads of the large-tile kernels
constexpr int BIG_NT = 512;

// launchers of the compression kernels (defined in dcs_k_small.cu / dcs_k_big.cu)
void launch_compress_big(const DevCtx& c, const DLayer* L, int nsub, const DBlock* B,
                         const DGate1* G1, const DCond* CD, double* fid_out, cudaStream_t s);

}  // namespace dcs
