// Data layout shared by the host API and the kernels of libdcs.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/dcs.h"

namespace dcs {

// A condition phi(c) (Sec. "Classically controlled operations").
struct DCond {
  uint64_t mask[DCS_CWORDS];
  int32_t op;     // dcs_cond_op
  int32_t value;  // 0 / 1
};

// A single-qubit gate U (row-major [out][in]) applied iff cond holds.
struct DGate1 {
  float2 u[4];
  DCond cond;
};

// A two-qubit block on (q, q+1): the chunk's only two-qubit gate on these qubits, G2, with
// its operator-Schmidt factors, and the single-qubit gates before / after it on q and q+1.
struct DBlock {
  int32_t q;
  int32_t D;        // operator-Schmidt rank of G2 (1..4)
  float2 G[16];     // G2, row-major over |s_q s_{q+1}>: G[(o0*2+o1)*4 + (i0*2+i1)]
  float2 WL[16];    // WL[(u*2+v)*4 + d]: left factor, out u, in v
  float2 WR[16];    // WR[(d*2+u)*2 + v]: right factor
  DCond cond;       // condition of G2 (op NONE: unconditional)
  int32_t pre_off[2], pre_n[2], post_off[2], post_n[2];  // into the DGate1 array
  int32_t composed;  // 1: no gate of the block is conditional and Gc holds the whole block
  float2 Gc[16];     // (Post_q x Post_{q+1}) G2 (Pre_q x Pre_{q+1}), composed in FP64
};

// Per-site description of a chunk.
struct DSite {
  int32_t kind;  // 0 untouched, 1 single-qubit gates only, 2 left of a block, 3 right of a block
  int32_t blk;   // block index (kind 2, 3)
  int32_t g_off, g_n;  // single-qubit gates (kind 1)
};

// One chunk (a layer of disjoint blocks).
struct DLayer {
  DSite site[DCS_MAX_QUBITS];
  int32_t n_blocks;
  int32_t blk_off;    // into the DBlock array; blocks sorted by decreasing q
  int32_t uncond;     // some gate is unconditional: never empty
  int32_t cond_off;   // all conditions of the chunk (for the empty test), into DCond array
  int32_t n_conds;
};

// One mid-circuit measurement of a run.
struct DMeas {
  int32_t q;
  int32_t cbit;
  uint64_t ordinal;
};

// Device view of a context (passed by value to every kernel).
struct DevCtx {
  int32_t n;         // sites
  int32_t chi_cap;   // bond capacity (>= chi_max); bond b holds at most bond_cap(b, n, chi_cap)
  int32_t dmax;      // MPO bond capacity of a chunk: 4 per layer of the chunk, multiplied
  int32_t n_slots;
  const size_t* site_off;    // [n+1] complex-element offset of site j in a slot's MPS buffer
  const size_t* env_off;     // [n+1] offset of the environment of bond b in a slot's cache
  size_t mps_slot_stride;    // complex elements per slot per MPS buffer
  size_t env_slot_stride;    // complex elements per slot of the environment cache
  float2* mps[2];            // MPS buffer pair
  float2* env;               // environment cache: bond b holds L_b or R_b, whichever the
                             // sweep reads next (a left-to-right step reads R_{j+1} before it
                             // writes L_{j+1} over it; right to left mirrored)
  int32_t* bonds;            // [slot][2][n+1]
  int32_t* centre;           // [slot]
  int32_t* ketbuf;           // [slot] which MPS buffer holds the ket
  double* p;                 // [slot] path probability p_gamma
  double* F;                 // [slot] estimated fidelity F~ (product of f)
  double* rr;                // [slot][2] slice weights r_0, r_1 of the last MeasureProb
  uint64_t* creg;            // [slot][DCS_CWORDS]
  uint32_t* flags;           // [slot]
  uint64_t* shot;            // [slot] sampler counter of the shot
  int32_t* order;            // [n_slots] list order of active slots
  int32_t* count;            // number of active slots
  int32_t* status;           // context-wide error bits
  int32_t* plan;             // branch plan scratch
  unsigned long long* counters;  // [0] compression steps run, [1] sweeps run (since init)
  float2* work;              // per-slot work area of the large-tile kernels (nullptr: small)
  int32_t use_tc;            // large-tile contractions on the tensor cores: 0 no,
                             // 1 3xTF32, 2 BF16x3
  size_t work_stride;        // complex elements per slot of `work`
  uint64_t seed;
  int32_t chi_max;
  double tol;
  int32_t sweeps;
};

// Capacity of bond b (0..n) of an n-site MPS whose bonds are capped at C: min(C,
// 2^min(b, n-b)), the largest Schmidt rank of a cut into b and n-b qubits (paragraph
// "Matrix Product States": the bond dimensions chi_b vary along the chain).
__host__ __device__ inline int bond_cap(int b, int n, int C) {
  const int e = b < n - b ? b : n - b;
  if (e >= 30) return C;
  return C < (1 << e) ? C : (1 << e);
}

// Bond-sized layout of one slot: site j ([chi_j][2][chi_{j+1}], complex) at site_off[j],
// the environment of bond b ([beta_b][D <= dmax][alpha_b]) at env_off[b]; every region
// starts on a 256-byte boundary.  Returns the per-slot sizes through mps_elems / env_elems.
__host__ __device__ inline void layout_offsets(int n, int C, int dmax, size_t* site_off,
                                               size_t* env_off, size_t* mps_elems,
                                               size_t* env_elems) {
  size_t s = 0, e = 0;
  for (int b = 0; b <= n; ++b) {
    const size_t cb = (size_t)bond_cap(b, n, C);
    if (site_off) site_off[b] = s;
    if (env_off) env_off[b] = e;
    if (b < n) s += ((cb * 2 * (size_t)bond_cap(b + 1, n, C)) + 31) / 32 * 32;
    e += ((size_t)dmax * cb * cb + 31) / 32 * 32;
  }
  *mps_elems = s;
  *env_elems = e;
}

// plan layout (int32 words): [0] n_copy, [1] n_coll, [2] new count,
// then copy pairs (src, dst) x n_slots, then collapse records (slot, m) x n_slots.
constexpr int PLAN_HDR = 4;

// two launches: the layout offset tables, then the initial state of every slot
void launch_init(const DevCtx& c, int n_active, int multipath, uint64_t shot0, cudaStream_t s);
// tile_chi: shared-memory tile (4, 8, 16 or 32), at least every bond the launch can meet
// L: the chunk's nsub sub-layers (nsub > 1 only on the large-tile path)
void launch_compress(const DevCtx& c, int tile_chi, const DLayer* L, int nsub, const DBlock* B,
                     const DGate1* G1, const DCond* C, double* fid_out, cudaStream_t s);
void launch_measure(const DevCtx& c, int tile_chi, const DMeas* meas, int n_meas, int mode,
                    const uint8_t* forced, double* p0_out, cudaStream_t s);
// pmin > 0: adaptive pruning, children with p < pmin are dropped (the first of the key
// order stays)
void launch_branch_split(const DevCtx& c, int q, int cbit, double eps, int M, double pmin,
                         cudaStream_t s, int* launches);
void launch_branch_topk(const DevCtx& c, int M, cudaStream_t s);
void launch_branch_keep(const DevCtx& c, const uint8_t* keep, int n, cudaStream_t s);
void launch_fork_shots(const DevCtx& c, int n_active, cudaStream_t s);
int fused_chi(int chi_max);          // shared-memory tile for chi_max (0 if above 32)
int big_chi(int chi_max);            // slot capacity per bond of the large-tile path
size_t big_work_elems(int chi_cap, int dmax);  // complex elements of one slot's work area
// MPO bond capacity of chunks of up to `layers` layers: 4^layers
inline int chunk_dmax(int layers) { return layers <= 1 ? 4 : 1 << (2 * layers); }

// measurement modes
constexpr int MEAS_SAMPLE = 0;
constexpr int MEAS_FORCED = 1;
constexpr int MEAS_PROB = 2;

}  // namespace dcs
