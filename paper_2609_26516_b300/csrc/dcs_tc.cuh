// Tensor-core complex GEMM for sm_103a: tcgen05.mma (kind::tf32) with the accumulators in
// tensor memory (TMEM), issued by one thread of the CTA, completion signalled on mbarriers.
//
// C[m, n] = sum_k opA(m, k) opB(k, n) in complex64 with FP32 accumulators in TMEM (each MMA's
// rounding into the accumulator adds an error that grows with K, above CUDA-core FP32 for
// long products):
//  * real embedding: A_r[m][2k] = Re a, A_r[m][2k+1] = Im a;
//    B_r[2k][2n] = Re b, B_r[2k+1][2n] = -Im b, B_r[2k][2n+1] = Im b, B_r[2k+1][2n+1] = Re b,
//    so that (A_r B_r)[m][2n] = Re c and [m][2n+1] = Im c;
//  * 3xTF32: every operand x = hi + lo with hi = x with the low 13 mantissa bits cleared and
//    lo = x - hi; A B ~ hi_A hi_B + hi_A lo_B + lo_A hi_B (the dropped lo lo term is
//    ~2^-22 relative);
//  * or BF16x3 (kind::f16 with BF16 operands): hi = x rounded to BF16, lo = x - hi rounded
//    to BF16, the same three products; each MMA covers K = 16 where TF32 takes two of K = 8,
//    at about 2^-16 relative accuracy (the dropped lo lo term and the rounding of lo).
// Tile: 128 complex rows x 128 complex columns (MMA M = 128, N = 256 real), K in stages of
// 8 complex (16 real).  The CTA's warps are specialised: warp 0 issues the MMAs (one
// thread), the other warps load the complex operands of the coming stages from global
// memory, split them (hi / lo) and write them in the canonical K-major layout without
// swizzle (8-row x 16-byte core matrices, core matrices along K 128 bytes apart: the
// leading-dimension offset; 8-row groups 512 bytes apart for TF32, 256 for BF16: the stride
// offset) into a ring of stage buffers.  Per stage a "full" mbarrier collects one arrival per
// loader warp and an "empty" one the MMAs' completion (tcgen05.commit), so the loaders run up
// to a ring's length ahead of the tensor core and no CTA barrier sits in the K loop.  After a
// tile's last stage a "done" commit releases the epilogue (TMEM -> registers -> C, all
// warps).  Every mbarrier wait is bounded and flags *err when it gives up.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "dcs_device.cuh"

namespace dcs {

constexpr int TC_M = 128;   // complex rows per tile (= MMA M)
constexpr int TC_N = 128;   // complex columns per tile (MMA N = 256 real)
constexpr int TC_K = 8;     // complex K per stage (16 real)
constexpr int TC_A_FLOATS = TC_M * 2 * TC_K;        // one A copy (hi or lo): 128 x 16
constexpr int TC_B_FLOATS = 2 * TC_N * 2 * TC_K;    // one B copy: 256 x 16
constexpr int TC_STAGE_FLOATS = 2 * (TC_A_FLOATS + TC_B_FLOATS);  // 48 KB (TF32)
constexpr int TC_STAGE16_BYTES = TC_STAGE_FLOATS * 2;              // 24 KB (BF16)
constexpr int TC_MAX_PIPE = 6;        // stage buffers at most
constexpr int TC_MIN_PIPE = 2;
constexpr int TC_RAW = 3;             // raw operand stages in flight per loader thread
constexpr int TC_RAW_MIN = 2;         // (two where shared memory is short)
// one raw stage of a 512-thread CTA: 480 loader threads x 8 elements (30 KB); the
// 512-thread kernels are the ones that run the tensor-core GEMM
constexpr int TC_RAW_STAGE_FLOATS = 8 * 480 * 2;
// the smallest staging region the tensor-core GEMM runs in: two TF32 stages and two raw ones
constexpr int TC_SMEM_FLOATS = TC_MIN_PIPE * TC_STAGE_FLOATS + TC_RAW_MIN * TC_RAW_STAGE_FLOATS;
constexpr int TC_NBAR = 2 * TC_MAX_PIPE + 1;  // full[], empty[], done
constexpr int TC_TMEM_COLS = 256;
constexpr long long TC_WAIT_LIMIT = 1ll << 26;      // bounded mbarrier spins

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start >> 4 (bits 0-13), leading-dimension byte offset
// >> 4 (16-29), stride byte offset >> 4 (32-45), version 1 (bit 46), no swizzle (61-63 = 0).
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::tf32: D = F32 (bits 4-5 = 1), A = B = TF32 (bits 7-9,
// 10-12 = 2), both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// The same for kind::f16 with A = B = BF16 (bits 7-9, 10-12 = 1), D = F32.
__host__ __device__ constexpr uint32_t tc_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                       uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
      :
      : "r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tc_mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                            uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      :
      : "r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               :
               : "r"(smem_addr(mbar))
               : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" : : "r"(smem_addr(mbar)), "r"(count) : "memory");
}

// Wait for the completion of the phase with parity `parity`; false if the bounded spin ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity) {
  for (long long it = 0; it < TC_WAIT_LIMIT; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(mbar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// TMEM allocation / release by one whole warp.
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
               :
               : "r"(smem_addr(dst_smem)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" : : "r"(taddr), "r"(ncols) : "memory");
}

// 32 lanes x 32 consecutive columns of 32-bit data into v[0..31] (this warp's lane quadrant).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tf32_split(float x, float& hi, float& lo) {
  hi = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
  lo = x - hi;
}

// float index of element (row, kr) of a K-major 16-column operand in the canonical layout
__device__ __forceinline__ int tc_off(int row, int kr) {
  return (((row >> 3) * 4 + (kr >> 2)) * 32) + (row & 7) * 4 + (kr & 3);
}

// The BF16 operands: 16-bit index of element (row, kr), core matrices of 8 rows x 8 values
// (16 bytes a row), the two along K 128 bytes apart, 8-row groups 256 bytes apart.
__device__ __forceinline__ int tc_off16(int row, int kr) {
  return (((row >> 3) * 2 + (kr >> 3)) * 64) + (row & 7) * 8 + (kr & 7);
}

// x = hi + lo in BF16 (round to nearest), packed with the next real column: (a, b) -> two
// 32-bit words (hi_a | hi_b << 16) and (lo_a | lo_b << 16).
__device__ __forceinline__ void bf16_split2(float a, float b, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat16 ha = __float2bfloat16_rn(a), hb = __float2bfloat16_rn(b);
  const __nv_bfloat16 la = __float2bfloat16_rn(a - __bfloat162float(ha));
  const __nv_bfloat16 lb = __float2bfloat16_rn(b - __bfloat162float(hb));
  hi = (uint32_t)__bfloat16_as_ushort(ha) | ((uint32_t)__bfloat16_as_ushort(hb) << 16);
  lo = (uint32_t)__bfloat16_as_ushort(la) | ((uint32_t)__bfloat16_as_ushort(lb) << 16);
}

// Per-CTA state of the tensor-core GEMM (in shared memory).
struct TcState {
  float* stage;        // stage ring, 16-byte aligned
  size_t stage_bytes;  // its size
  uint64_t* mbar;      // TC_NBAR mbarriers: full[TC_MAX_PIPE], empty[TC_MAX_PIPE], done
  int* uses;           // [0] stages and [1] tiles run since tc_setup (the barriers' phases)
  uint32_t* tmem;      // TMEM base address (written by tmem_alloc)
  int* err;            // set to 1 if a bounded wait gave up
  bool bf16;           // BF16x3 products instead of 3xTF32; fixed for the whole kernel: the
                       // stage size, hence the pipeline depth behind the barrier phases,
                       // depends on it
};

// Bytes of the smem head tc_setup needs: the mbarriers, the two counters, TMEM base, error.
constexpr int TC_HEAD_BYTES = 8 * TC_NBAR + 4 * 4;

// One thread initialises the barriers; warp 0 allocates TMEM.  All threads call.
__device__ __forceinline__ void tc_setup(TcState& t) {
  if (threadIdx.x == 0) {
    for (int i = 0; i < TC_MAX_PIPE; ++i) {
      mbar_init(&t.mbar[i], (uint32_t)(blockDim.x / 32 - 1));  // full: one per loader warp
      mbar_init(&t.mbar[TC_MAX_PIPE + i], 1);                 // empty: the MMAs' commit
    }
    mbar_init(&t.mbar[2 * TC_MAX_PIPE], 1);                    // done
    t.uses[0] = t.uses[1] = 0;
    *t.err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  t.bf16 = false;
  if (threadIdx.x < 32) tmem_alloc(t.tmem, TC_TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
}

__device__ __forceinline__ void tc_teardown(TcState& t) {
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (threadIdx.x < 32) tmem_dealloc(*t.tmem, TC_TMEM_COLS);
}

__device__ __forceinline__ void cp_async8(uint32_t saddr, const void* g, int bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" : : "r"(saddr), "l"(g), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N_PENDING>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" : : "n"(N_PENDING) : "memory");
}

// Element e of a K-step in the staging order: a warp covers 8 consecutive rows (bits 2-4 of
// e) by 4 consecutive complex k (bits 0-1), so its 8-byte (re, im) stores fill whole core
// matrices without bank conflicts.
__device__ __forceinline__ void tc_elem(int e, int& row, int& kk) {
  kk = (e & 3) | (((e >> 5) & 1) << 2);
  row = ((e >> 2) & 7) | ((e >> 6) << 3);
}

// One operand element of a stage, loaded from global memory (zero outside the matrices):
// A element e of the stage (TC_M x TC_K complex) and B element e (2 TC_N real rows x TC_K:
// row 2n holds (Re b, -Im b), row 2n+1 (Im b, Re b) of B's column n).
__device__ __forceinline__ float2 tc_load_a(int e, int m0, int k0, int M, int K, const float2* A,
                                            int sam, int sak, bool conjA) {
  int mm, kk;
  tc_elem(e, mm, kk);
  const int gm = m0 + mm, gk = k0 + kk;
  // plain loads: the operands may have been written earlier in the same kernel
  float2 v = (gm < M && gk < K) ? A[(size_t)gm * sam + (size_t)gk * sak] : cz();
  if (conjA) v.y = -v.y;
  return v;
}
__device__ __forceinline__ float2 tc_load_b(int e, int n0, int k0, int N, int K, const float2* B,
                                            int sbk, int sbn, bool conjB) {
  int nr, kk;
  tc_elem(e, nr, kk);
  const int gn = n0 + (nr >> 1), gk = k0 + kk;
  float2 v = (gn < N && gk < K) ? B[(size_t)gk * sbk + (size_t)gn * sbn] : cz();
  if (conjB) v.y = -v.y;
  return (nr & 1) ? make_float2(v.y, v.x) : make_float2(v.x, -v.y);
}

// Element e's hi / lo parts into the canonical stage st (A: which = 0, B: which = 1).
__device__ __forceinline__ void tc_store(float* st, bool bf, int which, int e, float2 v) {
  int row, kk;
  tc_elem(e, row, kk);
  if (bf) {
    uint16_t* base = reinterpret_cast<uint16_t*>(st);
    uint16_t* hi = which == 0 ? base : base + 2 * TC_M * 16;
    uint16_t* lo = which == 0 ? base + TC_M * 16 : base + 2 * TC_M * 16 + 2 * TC_N * 16;
    uint32_t h, l;
    bf16_split2(v.x, v.y, h, l);
    const int o = tc_off16(row, 2 * kk);
    *reinterpret_cast<uint32_t*>(hi + o) = h;
    *reinterpret_cast<uint32_t*>(lo + o) = l;
  } else {
    float* hi = which == 0 ? st : st + 2 * TC_A_FLOATS;
    float* lo = which == 0 ? st + TC_A_FLOATS : st + 2 * TC_A_FLOATS + TC_B_FLOATS;
    float2 h, l;
    tf32_split(v.x, h.x, l.x);
    tf32_split(v.y, h.y, l.y);
    const int o = tc_off(row, 2 * kk);
    *reinterpret_cast<float2*>(hi + o) = h;
    *reinterpret_cast<float2*>(lo + o) = l;
  }
}

// The three products of one stage (issued by one thread).
__device__ __forceinline__ void tc_issue_stage(uint32_t tbase, const float* st, bool bf,
                                               bool first) {
  constexpr uint32_t IDESC = tc_idesc(128, 256);
  constexpr uint32_t IDESC16 = tc_idesc_bf16(128, 256);
  const uint32_t a0 = smem_addr(st);
  if (bf) {
    // A hi / lo 4 KB each, B hi / lo 8 KB each; one MMA of K = 16 per product
    const uint32_t b0 = a0 + 2 * 4096;
    const uint32_t as[3] = {a0, a0, a0 + 4096};
    const uint32_t bs[3] = {b0, b0 + 8192, b0};
#pragma unroll
    for (int p = 0; p < 3; ++p)
      tc_mma_bf16(tbase, tc_desc(as[p], 128, 256), tc_desc(bs[p], 128, 256), IDESC16,
                  (!first || p > 0) ? 1u : 0u);
  } else {
    const uint32_t b0 = a0 + 2 * TC_A_FLOATS * 4;
    const uint32_t as[3] = {a0, a0, a0 + TC_A_FLOATS * 4};
    const uint32_t bs[3] = {b0, b0 + TC_B_FLOATS * 4, b0};
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int h = 0; h < 2; ++h)  // K-chunks 2h, 2h+1: two core matrices (256 B) further
        tc_mma(tbase, tc_desc(as[p] + h * 256, 128, 512), tc_desc(bs[p] + h * 256, 128, 512),
               IDESC, (!first || p > 0 || h > 0) ? 1u : 0u);
  }
}

__device__ __forceinline__ void mbar_arrive(uint64_t* mbar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.release.cta.shared::cta.b64 st, [%0];\n\t}"
               :
               : "r"(smem_addr(mbar))
               : "memory");
}

template <int NT>
__device__ void cta_cgemm_tc(int M, int N, int K, const float2* A, int sam, int sak, bool conjA,
                             const float2* B, int sbk, int sbn, bool conjB, float2* Cm, int scm,
                             int scn, TcState& t) {
  static_assert(NT % 128 == 0, "the epilogue needs whole warp quadrants");
  static_assert(TC_K == 8, "the element mapping covers 8 complex k per step");
  constexpr int NL = NT - 32;  // loader threads (warps 1 ..)
  constexpr int PA = (TC_M * TC_K + NL - 1) / NL;
  constexpr int PB = (2 * TC_N * TC_K + NL - 1) / NL;
  const bool bf = t.bf16;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t tbase = *t.tmem;
  const size_t sstride = bf ? (size_t)TC_STAGE16_BYTES : (size_t)TC_STAGE_FLOATS * 4;
  // the raw ring (rawd stages of every loader thread's elements) sits at the end of the
  // staging region, the stage buffers before it: three raw stages when two stage buffers
  // still fit beside them, else two
  constexpr size_t RAW_STAGE = (size_t)(PA + PB) * NL * sizeof(float2);
  const int rawd = t.stage_bytes >= TC_RAW * RAW_STAGE + TC_MIN_PIPE * sstride ? TC_RAW : TC_RAW_MIN;
  int pipe = (int)((t.stage_bytes - rawd * RAW_STAGE) / sstride);
  pipe = pipe > TC_MAX_PIPE ? TC_MAX_PIPE : pipe;
  float2* raw = reinterpret_cast<float2*>(reinterpret_cast<char*>(t.stage) + t.stage_bytes -
                                          rawd * RAW_STAGE);
  const int ksteps = (K + TC_K - 1) / TC_K;
  uint64_t* full = t.mbar;
  uint64_t* empty = t.mbar + TC_MAX_PIPE;
  uint64_t* done = t.mbar + 2 * TC_MAX_PIPE;
  __syncthreads();  // earlier writes of the operands; the counters below are settled
  const int g0 = t.uses[0], tile0 = t.uses[1];
  int ntile = 0;
  for (int m0 = 0; m0 < M; m0 += TC_M)
    for (int n0 = 0; n0 < N; n0 += TC_N) {
      const int gbase = g0 + ntile * ksteps;
      if (warp == 0) {
        if (lane == 0) {
          for (int s = 0; s < ksteps; ++s) {
            const int g = gbase + s, slot = g % pipe;
            if (!mbar_wait(&full[slot], (uint32_t)((g / pipe) & 1))) *t.err = 1;
            tc_fence_after();
            tc_issue_stage(tbase, reinterpret_cast<const float*>(
                                      reinterpret_cast<const char*>(t.stage) + slot * sstride),
                           bf, s == 0);
            tc_commit(&empty[slot]);
          }
          tc_commit(done);
          if (!mbar_wait(done, (uint32_t)((tile0 + ntile) & 1))) *t.err = 1;
        }
        __syncwarp();
      } else {
        // loader warps: each thread copies its own elements of stage s + TC_RAW - 1 into its
        // own slots of the raw ring (cp.async, zero fill outside the matrices), then splits
        // its elements of stage s from there into the canonical stage buffer
        const int lt = tid - 32;
        // per element: the global offset at k = 0 (-1 outside the matrix) and the packed
        // stage index e (bits 0-15), k within the stage (16-18) and odd real row (19)
        int ga[PA], gb[PB], ma[PA], mb[PB];
#pragma unroll
        for (int i = 0; i < PA; ++i) {
          const int e = lt + i * NL;
          int mm, kk;
          tc_elem(e < TC_M * TC_K ? e : 0, mm, kk);
          const bool ok = e < TC_M * TC_K && m0 + mm < M;
          ga[i] = ok ? (m0 + mm) * sam + kk * sak : -1;
          ma[i] = e < TC_M * TC_K ? (e | (kk << 16)) : -1;
        }
#pragma unroll
        for (int i = 0; i < PB; ++i) {
          const int e = lt + i * NL;
          int nr, kk;
          tc_elem(e < 2 * TC_N * TC_K ? e : 0, nr, kk);
          const bool ok = e < 2 * TC_N * TC_K && n0 + (nr >> 1) < N;
          gb[i] = ok ? kk * sbk + (n0 + (nr >> 1)) * sbn : -1;
          mb[i] = e < 2 * TC_N * TC_K ? (e | (kk << 16) | ((nr & 1) << 19)) : -1;
        }
        const int adv_a = TC_K * sak, adv_b = TC_K * sbk;
        auto raw_slot = [&](int s, int i) {  // this thread's slot i of raw stage s
          return raw + ((size_t)((s % rawd) * (PA + PB) + i) * NL + lt);
        };
        auto issue = [&](int s) {
          if (s < ksteps) {
            const int k0 = s * TC_K;
#pragma unroll
            for (int i = 0; i < PA; ++i) {
              const bool in = ga[i] >= 0 && k0 + ((ma[i] >> 16) & 7) < K;
              cp_async8(smem_addr(raw_slot(s, i)), in ? A + ((size_t)ga[i] + (size_t)s * adv_a) : A,
                        in ? 8 : 0);
            }
#pragma unroll
            for (int i = 0; i < PB; ++i) {
              const bool in = gb[i] >= 0 && k0 + ((mb[i] >> 16) & 7) < K;
              cp_async8(smem_addr(raw_slot(s, PA + i)),
                        in ? B + ((size_t)gb[i] + (size_t)s * adv_b) : B, in ? 8 : 0);
            }
          }
          cp_async_commit();
        };
        for (int r = 0; r < rawd - 1; ++r) issue(r);
        for (int s = 0; s < ksteps; ++s) {
          issue(s + rawd - 1);
          // this thread's copies of stage s have landed
          if (rawd == TC_RAW) cp_async_wait<TC_RAW - 1>();
          else cp_async_wait<TC_RAW_MIN - 1>();
          const int g = gbase + s, slot = g % pipe;
          // the MMAs that last read this buffer (stage g - pipe) must have completed
          if (g >= pipe && lane == 0) {
            if (!mbar_wait(&empty[slot], (uint32_t)(((g / pipe) - 1) & 1))) *t.err = 1;
          }
          __syncwarp();
          float* st = reinterpret_cast<float*>(reinterpret_cast<char*>(t.stage) + slot * sstride);
#pragma unroll
          for (int i = 0; i < PA; ++i) {
            if (ma[i] < 0) continue;
            float2 v = *raw_slot(s, i);
            if (conjA) v.y = -v.y;
            tc_store(st, bf, 0, ma[i] & 0xFFFF, v);
          }
#pragma unroll
          for (int i = 0; i < PB; ++i) {
            if (mb[i] < 0) continue;
            float2 v = *raw_slot(s, PA + i);
            if (conjB) v.y = -v.y;
            v = ((mb[i] >> 19) & 1) ? make_float2(v.y, v.x) : make_float2(v.x, -v.y);
            tc_store(st, bf, 1, mb[i] & 0xFFFF, v);
          }
          fence_async_smem();
          __syncwarp();
          if (lane == 0) mbar_arrive(&full[slot]);
        }
        cp_async_wait<0>();
      }
      // epilogue: the tile's accumulators are complete (done) once thread 0 passes
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
      for (int wq = warp; wq < 16; wq += NT / 32) {
        const int quad = wq & 3, cg = wq >> 2;  // lanes 32 quad.., real columns 64 cg..
        const int row = quad * 32 + lane;
        for (int half = 0; half < 2; ++half) {
          float v[32];
          tmem_ld32(tbase + ((uint32_t)(quad * 32) << 16) + (uint32_t)(cg * 64 + half * 32), v);
          const int gm = m0 + row;
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int gn = n0 + cg * 32 + half * 16 + j;
            if (gm < M && gn < N) Cm[(size_t)gm * scm + (size_t)gn * scn] = make_float2(v[2 * j], v[2 * j + 1]);
          }
        }
      }
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
      ++ntile;
    }
  if (tid == 0) {
    t.uses[0] = g0 + ntile * ksteps;
    t.uses[1] = tile0 + ntile;
  }
  __syncthreads();
}

}  // namespace dcs
