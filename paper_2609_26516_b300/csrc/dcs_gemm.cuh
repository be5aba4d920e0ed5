// CTA-level complex GEMMs of libdcs: a shared-memory-tiled FP32 SIMT version and the
// tensor-core version of dcs_tc.cuh.
#pragma once
#include "dcs_device.cuh"
#include "dcs_tc.cuh"

namespace dcs {

constexpr int GBM = 64, GBN = 64, GBK = 16;  // SIMT CTA GEMM tile
// padded leading dimensions of the staged tiles (fewer bank conflicts on the transposing
// stores; the B rows stay 16-byte aligned)
constexpr int GSA_LD = GBK + 1, GSB_LD = GBN + 2;
constexpr int GEMM_SIMT_SMEM_ELEMS = GBM * GSA_LD + GBK * GSB_LD;

// ----------------------------------------------------------------------------- CTA GEMM
// C[m, n] = sum_k opA(m, k) opB(k, n) with opA(m, k) = A[m sam + k sak] (conjugated if
// conjA), opB(k, n) = B[k sbk + n sbn] (conjugated if conjB), C[m scm + n scn].  FP32 SIMT
// with 64 x 64 x 16 shared-memory tiles (sA, sB: GEMM_SIMT_SMEM_ELEMS complex); each thread
// owns an 8-element micro tile, 2 rows x 4 columns at 512 threads, so a k step costs two
// broadcast loads of A and two 16-byte loads of B for eight complex FMAs.  The next k tile's
// elements are loaded into registers while the current one is multiplied.
template <int NT>
__device__ void cta_cgemm(int M, int N, int K, const float2* A, int sam, int sak, bool conjA,
                          const float2* B, int sbk, int sbn, bool conjB, float2* Cm, int scm,
                          int scn, float2* sA, float2* sB, bool accumulate = false) {
  static_assert((GBM * GBN) % NT == 0, "tile / threads");
  constexpr int PER = GBM * GBN / NT;  // outputs per thread
  constexpr int LA = (GBM * GBK + NT - 1) / NT, LB = (GBK * GBN + NT - 1) / NT;
  const int tid = threadIdx.x;
  for (int m0 = 0; m0 < M; m0 += GBM)
    for (int n0 = 0; n0 < N; n0 += GBN) {
      float2 acc[PER];
#pragma unroll
      for (int i = 0; i < PER; ++i) acc[i] = cz();
      // element r of this thread in the A tile (GBM x GBK, stored sA[m][k]) and the B tile
      // (GBK x GBN, stored sB[k][n]), in the order that keeps the global loads coalesced
      auto a_pos = [&](int idx, int& mm, int& kk) {
        if (sak == 1) {
          mm = idx / GBK;
          kk = idx % GBK;
        } else {
          kk = idx / GBM;
          mm = idx % GBM;
        }
      };
      auto b_pos = [&](int idx, int& kk, int& nn) {
        if (sbn == 1) {
          kk = idx / GBN;
          nn = idx % GBN;
        } else {
          nn = idx / GBK;
          kk = idx % GBK;
        }
      };
      float2 ra[LA], rb[LB];
      auto load_tile = [&](int k0) {
#pragma unroll
        for (int r = 0; r < LA; ++r) {
          const int idx = tid + r * NT;
          int mm, kk;
          a_pos(idx, mm, kk);
          const int gm = m0 + mm, gk = k0 + kk;
          float2 v = cz();
          if (idx < GBM * GBK && gm < M && gk < K) {
            v = A[(size_t)gm * sam + (size_t)gk * sak];
            if (conjA) v.y = -v.y;
          }
          ra[r] = v;
        }
#pragma unroll
        for (int r = 0; r < LB; ++r) {
          const int idx = tid + r * NT;
          int kk, nn;
          b_pos(idx, kk, nn);
          const int gk = k0 + kk, gn = n0 + nn;
          float2 v = cz();
          if (idx < GBK * GBN && gk < K && gn < N) {
            v = B[(size_t)gk * sbk + (size_t)gn * sbn];
            if (conjB) v.y = -v.y;
          }
          rb[r] = v;
        }
      };
      load_tile(0);
      for (int k0 = 0; k0 < K; k0 += GBK) {
#pragma unroll
        for (int r = 0; r < LA; ++r) {
          const int idx = tid + r * NT;
          int mm, kk;
          a_pos(idx, mm, kk);
          if (idx < GBM * GBK) sA[mm * GSA_LD + kk] = ra[r];
        }
#pragma unroll
        for (int r = 0; r < LB; ++r) {
          const int idx = tid + r * NT;
          int kk, nn;
          b_pos(idx, kk, nn);
          if (idx < GBK * GBN) sB[kk * GSB_LD + nn] = rb[r];
        }
        __syncthreads();
        if (k0 + GBK < K) load_tile(k0 + GBK);
        if constexpr (NT == 512) {
          // rows 2 ty, 2 ty + 1 and columns 4 tx .. 4 tx + 3, tx = tid mod 16
          const int tx = tid & 15, ty = tid >> 4;
#pragma unroll 4
          for (int kk = 0; kk < GBK; ++kk) {
            const float2 a0 = sA[(2 * ty) * GSA_LD + kk], a1 = sA[(2 * ty + 1) * GSA_LD + kk];
            const float4 b01 = *reinterpret_cast<const float4*>(sB + kk * GSB_LD + 4 * tx);
            const float4 b23 = *reinterpret_cast<const float4*>(sB + kk * GSB_LD + 4 * tx + 2);
            const float2 bv[4] = {make_float2(b01.x, b01.y), make_float2(b01.z, b01.w),
                                  make_float2(b23.x, b23.y), make_float2(b23.z, b23.w)};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              cfma(acc[i], a0, bv[i]);
              cfma(acc[4 + i], a1, bv[i]);
            }
          }
        } else {
          // PER outputs in one row
          const int row = tid / (GBN / PER);
          const int col0 = (tid % (GBN / PER)) * PER;
#pragma unroll 4
          for (int kk = 0; kk < GBK; ++kk) {
            const float2 a = sA[row * GSA_LD + kk];
#pragma unroll
            for (int i = 0; i < PER; ++i) cfma(acc[i], a, sB[kk * GSB_LD + col0 + i]);
          }
        }
        __syncthreads();
      }
#pragma unroll
      for (int i = 0; i < PER; ++i) {
        int row, col;
        if constexpr (NT == 512) {
          row = 2 * (tid >> 4) + (i >> 2);
          col = 4 * (tid & 15) + (i & 3);
        } else {
          row = tid / (GBN / PER);
          col = (tid % (GBN / PER)) * PER + i;
        }
        const int gm = m0 + row, gn = n0 + col;
        if (gm < M && gn < N) {
          float2* dst = Cm + (size_t)gm * scm + (size_t)gn * scn;
          *dst = accumulate ? cadd(*dst, acc[i]) : acc[i];
        }
      }
    }
  __syncthreads();
}

}  // namespace dcs
