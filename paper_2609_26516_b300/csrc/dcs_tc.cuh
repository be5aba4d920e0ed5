// Tensor-core complex GEMM for sm_103a: tcgen05.mma (kind::tf32) with the accumulators in
// tensor memory (TMEM), issued by one thread of the CTA, completion signalled on mbarriers.
//
// C[m, n] = sum_k opA(m, k) opB(k, n) in complex64 with FP32 accuracy:
//  * real embedding: A_r[m][2k] = Re a, A_r[m][2k+1] = Im a;
//    B_r[2k][2n] = Re b, B_r[2k+1][2n] = -Im b, B_r[2k][2n+1] = Im b, B_r[2k+1][2n+1] = Re b,
//    so that (A_r B_r)[m][2n] = Re c and [m][2n+1] = Im c;
//  * 3xTF32: every operand x = hi + lo with hi = x with the low 13 mantissa bits cleared and
//    lo = x - hi; A B ~ hi_A hi_B + hi_A lo_B + lo_A hi_B (the dropped lo lo term is
//    ~2^-22 relative);
//  * or BF16x3 (kind::f16 with BF16 operands): hi = x rounded to BF16, lo = x - hi rounded
//    to BF16, the same three products; each MMA covers K = 16 where TF32 takes two of K = 8,
//    at about 2^-16 relative accuracy (the dropped lo lo term and the rounding of lo).
// Tile: 128 complex rows x 128 complex columns (MMA M = 128, N = 256 real), K in steps of 8
// complex (16 real = two MMAs of K = 8).  The raw complex operand tiles of the next K-steps
// stream into a 4-deep shared-memory ring with cp.async (zero fill outside the matrices), so
// global latency stays off the critical path.  From there all threads split them into hi/lo
// TF32 in the canonical K-major layout without swizzle: 8-row x 16-byte core matrices, core
// matrices along K 128 bytes apart (leading-dimension offset), 8-row groups 512 bytes apart
// (stride offset).  Two canonical buffers alternate; the MMAs of one stage run while the
// other is filled.
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
constexpr int TC_STAGE_FLOATS = 2 * (TC_A_FLOATS + TC_B_FLOATS);
constexpr int TC_RAW = 4;                            // raw operand ring depth (K-steps)
constexpr int TC_RAW_ELEMS = TC_M * TC_K + TC_K * TC_N;  // complex elements per raw step
// two canonical stages (96 KB) and the raw ring (64 KB)
constexpr int TC_SMEM_FLOATS = 2 * TC_STAGE_FLOATS + TC_RAW * 2 * TC_RAW_ELEMS;
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
  float* stage;        // TC_SMEM_FLOATS, 16-byte aligned
  uint64_t* mbar;      // 2 mbarriers
  int* uses;           // 2 commit counters
  uint32_t* tmem;      // TMEM base address (written by tmem_alloc)
  int* err;            // set to 1 if a bounded wait gave up
  bool bf16;           // BF16x3 products instead of 3xTF32
};

// One thread initialises the barriers; warp 0 allocates TMEM.  All threads call.
__device__ __forceinline__ void tc_setup(TcState& t) {
  if (threadIdx.x == 0) {
    mbar_init(&t.mbar[0], 1);
    mbar_init(&t.mbar[1], 1);
    t.uses[0] = t.uses[1] = 0;
    *t.err = 0;
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

// Raw tiles of K-step s into ring slot `raw` (A as [mm][kk], B as [kk][nn], complex), one
// 8-byte cp.async per element; consecutive threads follow the contiguous global index.
template <int NT>
__device__ __forceinline__ void tc_raw_issue(float2* raw, int s, int m0, int n0, int M, int N,
                                             int K, const float2* A, int sam, int sak,
                                             const float2* B, int sbk, int sbn) {
  const int k0 = s * TC_K;
  float2* rA = raw;
  float2* rB = raw + TC_M * TC_K;
#pragma unroll
  for (int e = threadIdx.x; e < TC_M * TC_K; e += NT) {
    const int mm = sak == 1 ? e / TC_K : e % TC_M;
    const int kk = sak == 1 ? e % TC_K : e / TC_M;
    const int gm = m0 + mm, gk = k0 + kk;
    const bool in = gm < M && gk < K;
    cp_async8(smem_addr(rA + mm * TC_K + kk), in ? A + ((size_t)gm * sam + (size_t)gk * sak) : A,
              in ? 8 : 0);
  }
#pragma unroll
  for (int e = threadIdx.x; e < TC_K * TC_N; e += NT) {
    const int kk = sbn == 1 ? e / TC_N : e % TC_K;
    const int nn = sbn == 1 ? e % TC_N : e / TC_K;
    const int gk = k0 + kk, gn = n0 + nn;
    const bool in = gk < K && gn < N;
    cp_async8(smem_addr(rB + kk * TC_N + nn), in ? B + ((size_t)gk * sbk + (size_t)gn * sbn) : B,
              in ? 8 : 0);
  }
}

// Element e of a K-step in the staging order: a warp covers 8 consecutive rows (bits 2-4 of
// e) by 4 consecutive complex k (bits 0-1), so its 8-byte (re, im) stores fill whole core
// matrices without bank conflicts.
__device__ __forceinline__ void tc_elem(int e, int& row, int& kk) {
  kk = (e & 3) | (((e >> 5) & 1) << 2);
  row = ((e >> 2) & 7) | ((e >> 6) << 3);
}

// Raw slot -> canonical hi / lo stage.  A per complex element (TC_M x TC_K); B per real row
// of B_r^T (2 TC_N x TC_K: row 2n holds (Re b, -Im b), row 2n+1 holds (Im b, Re b)).
template <int NT>
__device__ __forceinline__ void tc_stage_from_raw_bf16(const float2* raw, float* st, bool conjA,
                                                       bool conjB) {
  const float2* rA = raw;
  const float2* rB = raw + TC_M * TC_K;
  // per copy: A 128 x 16 and B 256 x 16 BF16 values
  uint16_t* Ahi = reinterpret_cast<uint16_t*>(st);
  uint16_t* Alo = Ahi + TC_M * 16;
  uint16_t* Bhi = Alo + TC_M * 16;
  uint16_t* Blo = Bhi + 2 * TC_N * 16;
#pragma unroll
  for (int e = threadIdx.x; e < TC_M * TC_K; e += NT) {
    int mm, kk;
    tc_elem(e, mm, kk);
    float2 v = rA[mm * TC_K + kk];
    if (conjA) v.y = -v.y;
    uint32_t h, l;
    bf16_split2(v.x, v.y, h, l);
    const int o = tc_off16(mm, 2 * kk);
    *reinterpret_cast<uint32_t*>(Ahi + o) = h;
    *reinterpret_cast<uint32_t*>(Alo + o) = l;
  }
#pragma unroll
  for (int e = threadIdx.x; e < 2 * TC_N * TC_K; e += NT) {
    int nr, kk;
    tc_elem(e, nr, kk);
    float2 v = rB[kk * TC_N + (nr >> 1)];
    if (conjB) v.y = -v.y;
    v = (nr & 1) ? make_float2(v.y, v.x) : make_float2(v.x, -v.y);
    uint32_t h, l;
    bf16_split2(v.x, v.y, h, l);
    const int o = tc_off16(nr, 2 * kk);
    *reinterpret_cast<uint32_t*>(Bhi + o) = h;
    *reinterpret_cast<uint32_t*>(Blo + o) = l;
  }
}

template <int NT>
__device__ __forceinline__ void tc_stage_from_raw(const float2* raw, float* st, bool conjA,
                                                  bool conjB) {
  const float2* rA = raw;
  const float2* rB = raw + TC_M * TC_K;
  float* Ahi = st;
  float* Alo = Ahi + TC_A_FLOATS;
  float* Bhi = Alo + TC_A_FLOATS;
  float* Blo = Bhi + TC_B_FLOATS;
#pragma unroll
  for (int e = threadIdx.x; e < TC_M * TC_K; e += NT) {
    int mm, kk;
    tc_elem(e, mm, kk);
    float2 v = rA[mm * TC_K + kk];
    if (conjA) v.y = -v.y;
    float2 h, l;
    tf32_split(v.x, h.x, l.x);
    tf32_split(v.y, h.y, l.y);
    const int o = tc_off(mm, 2 * kk);
    *reinterpret_cast<float2*>(Ahi + o) = h;
    *reinterpret_cast<float2*>(Alo + o) = l;
  }
#pragma unroll
  for (int e = threadIdx.x; e < 2 * TC_N * TC_K; e += NT) {
    int nr, kk;
    tc_elem(e, nr, kk);
    float2 v = rB[kk * TC_N + (nr >> 1)];
    if (conjB) v.y = -v.y;
    v = (nr & 1) ? make_float2(v.y, v.x) : make_float2(v.x, -v.y);
    float2 h, l;
    tf32_split(v.x, h.x, l.x);
    tf32_split(v.y, h.y, l.y);
    const int o = tc_off(nr, 2 * kk);
    *reinterpret_cast<float2*>(Bhi + o) = h;
    *reinterpret_cast<float2*>(Blo + o) = l;
  }
}

template <int NT>
__device__ void cta_cgemm_tc(int M, int N, int K, const float2* A, int sam, int sak, bool conjA,
                             const float2* B, int sbk, int sbn, bool conjB, float2* Cm, int scm,
                             int scn, TcState& t) {
  static_assert(NT % 128 == 0, "the epilogue needs whole warp quadrants");
  static_assert(TC_K == 8, "the element mapping covers 8 complex k per step");
  constexpr uint32_t IDESC = tc_idesc(128, 256);
  constexpr uint32_t IDESC16 = tc_idesc_bf16(128, 256);
  const bool bf = t.bf16;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t tbase = *t.tmem;
  const int ksteps = (K + TC_K - 1) / TC_K;
  float2* ring = reinterpret_cast<float2*>(t.stage + 2 * TC_STAGE_FLOATS);
  for (int m0 = 0; m0 < M; m0 += TC_M)
    for (int n0 = 0; n0 < N; n0 += TC_N) {
      __syncthreads();  // the ring's last reads (previous tile) are done
#pragma unroll
      for (int r = 0; r < TC_RAW - 1; ++r) {
        if (r < ksteps)
          tc_raw_issue<NT>(ring + r * TC_RAW_ELEMS, r, m0, n0, M, N, K, A, sam, sak, B, sbk, sbn);
        cp_async_commit();
      }
      for (int s = 0; s < ksteps; ++s) {
        const int b = s & 1;
        float* st = t.stage + b * TC_STAGE_FLOATS;
        float* Ahi = st;
        float* Alo = Ahi + TC_A_FLOATS;
        float* Bhi = Alo + TC_A_FLOATS;
        float* Blo = Bhi + TC_B_FLOATS;
        // refill the slot read in the previous step with step s + TC_RAW - 1
        const int ahead = s + TC_RAW - 1;
        if (ahead < ksteps)
          tc_raw_issue<NT>(ring + (ahead % TC_RAW) * TC_RAW_ELEMS, ahead, m0, n0, M, N, K, A,
                           sam, sak, B, sbk, sbn);
        cp_async_commit();
        cp_async_wait<TC_RAW - 1>();  // this thread's copies of step s have landed
        // the MMAs that last read this canonical buffer must be done before it is overwritten
        if (tid == 0 && t.uses[b] > 0) {
          if (!mbar_wait(&t.mbar[b], (uint32_t)((t.uses[b] - 1) & 1))) *t.err = 1;
        }
        __syncthreads();
        if (bf) tc_stage_from_raw_bf16<NT>(ring + (s % TC_RAW) * TC_RAW_ELEMS, st, conjA, conjB);
        else tc_stage_from_raw<NT>(ring + (s % TC_RAW) * TC_RAW_ELEMS, st, conjA, conjB);
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
          tc_fence_after();
          if (bf) {
            // BF16 copies: A hi / lo 4 KB each, B hi / lo 8 KB each; one MMA of K = 16 per
            // product (both K core matrices of the stage)
            const uint32_t a0 = smem_addr(st), b0 = a0 + 2 * 4096;
            const uint32_t as[3] = {a0, a0, a0 + 4096};
            const uint32_t bs[3] = {b0, b0 + 8192, b0};
#pragma unroll
            for (int p = 0; p < 3; ++p)
              tc_mma_bf16(tbase, tc_desc(as[p], 128, 256), tc_desc(bs[p], 128, 256), IDESC16,
                          (s > 0 || p > 0) ? 1u : 0u);
          } else {
            const float* As[3] = {Ahi, Ahi, Alo};
            const float* Bs[3] = {Bhi, Blo, Bhi};
#pragma unroll
            for (int p = 0; p < 3; ++p)
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                // K-chunks 2h, 2h+1 of this stage: start two core matrices (256 B) further
                const uint64_t ad = tc_desc(smem_addr(As[p]) + h * 256, 128, 512);
                const uint64_t bd = tc_desc(smem_addr(Bs[p]) + h * 256, 128, 512);
                tc_mma(tbase, ad, bd, IDESC, (s > 0 || p > 0 || h > 0) ? 1u : 0u);
              }
          }
          tc_commit(&t.mbar[b]);
          t.uses[b] += 1;
        }
      }
      cp_async_wait<0>();
      // epilogue: wait for the last stage (and the one before), read TMEM, write C
      if (tid == 0) {
        for (int b = 0; b < 2; ++b)
          if (t.uses[b] > 0 && !mbar_wait(&t.mbar[b], (uint32_t)((t.uses[b] - 1) & 1))) *t.err = 1;
      }
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
    }
}

}  // namespace dcs
