// CTA-level complex GEMMs of libdcs: a shared-memory-tiled FP32 SIMT version and the
// tensor-core version of dcs_tc.cuh.
#pragma once
#include "dcs_device.cuh"
#include "dcs_tc.cuh"

namespace dcs {

constexpr int GBM = 64, GBN = 64, GBK = 16;  // SIMT CTA GEMM tile

// ----------------------------------------------------------------------------- CTA GEMM
// C[m, n] = sum_k opA(m, k) opB(k, n) with opA(m, k) = A[m sam + k sak] (conjugated if
// conjA), opB(k, n) = B[k sbk + n sbn] (conjugated if conjB), C[m scm + n scn].  FP32 SIMT
// with 64 x 64 x 16 shared-memory tiles; each thread owns an 8-element micro tile.
template <int NT>
__device__ void cta_cgemm(int M, int N, int K, const float2* A, int sam, int sak, bool conjA,
                          const float2* B, int sbk, int sbn, bool conjB, float2* Cm, int scm,
                          int scn, float2* sA, float2* sB, bool accumulate = false) {
  static_assert((GBM * GBN) % NT == 0, "tile / threads");
  constexpr int PER = GBM * GBN / NT;  // outputs per thread
  const int tid = threadIdx.x;
  for (int m0 = 0; m0 < M; m0 += GBM)
    for (int n0 = 0; n0 < N; n0 += GBN) {
      float2 acc[PER];
#pragma unroll
      for (int i = 0; i < PER; ++i) acc[i] = cz();
      for (int k0 = 0; k0 < K; k0 += GBK) {
        // stage A tile (GBM x GBK) as sA[m][k] and B tile (GBK x GBN) as sB[k][n]
        for (int idx = tid; idx < GBM * GBK; idx += NT) {
          int mm, kk;
          if (sak == 1) {
            mm = idx / GBK;
            kk = idx % GBK;
          } else {
            kk = idx / GBM;
            mm = idx % GBM;
          }
          const int gm = m0 + mm, gk = k0 + kk;
          float2 v = cz();
          if (gm < M && gk < K) {
            v = A[(size_t)gm * sam + (size_t)gk * sak];
            if (conjA) v.y = -v.y;
          }
          sA[mm * GBK + kk] = v;
        }
        for (int idx = tid; idx < GBK * GBN; idx += NT) {
          int kk, nn;
          if (sbn == 1) {
            kk = idx / GBN;
            nn = idx % GBN;
          } else {
            nn = idx / GBK;
            kk = idx % GBK;
          }
          const int gk = k0 + kk, gn = n0 + nn;
          float2 v = cz();
          if (gk < K && gn < N) {
            v = B[(size_t)gk * sbk + (size_t)gn * sbn];
            if (conjB) v.y = -v.y;
          }
          sB[kk * GBN + nn] = v;
        }
        __syncthreads();
        // thread tid owns rows (tid / (GBN / 2)) * ... : PER outputs in one row, PER columns
        const int row = tid / (GBN / PER);
        const int col0 = (tid % (GBN / PER)) * PER;
#pragma unroll 4
        for (int kk = 0; kk < GBK; ++kk) {
          const float2 a = sA[row * GBK + kk];
#pragma unroll
          for (int i = 0; i < PER; ++i) cfma(acc[i], a, sB[kk * GBN + col0 + i]);
        }
        __syncthreads();
      }
      const int row = tid / (GBN / PER);
      const int col0 = (tid % (GBN / PER)) * PER;
      const int gm = m0 + row;
      if (gm < M) {
#pragma unroll
        for (int i = 0; i < PER; ++i) {
          const int gn = n0 + col0 + i;
          if (gn < N) {
            float2* dst = Cm + (size_t)gm * scm + (size_t)gn * scn;
            *dst = accumulate ? cadd(*dst, acc[i]) : acc[i];
          }
        }
      }
    }
  __syncthreads();
}

}  // namespace dcs
