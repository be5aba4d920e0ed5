// dcs_cgemm: the contraction primitive of the large-bond kernels (every environment and site
// product of Sec. "Simulating unitary quantum circuits with DMRG" is a complex GEMM) exposed
// on its own, one CTA per problem of a batch.
#include <cuda_runtime.h>

#include "dcs_gemm.cuh"
#include "dcs_kernels.cuh"

namespace {

using namespace dcs;

constexpr int GEMM_NT = 512;
// staging of the tensor-core mode: three raw stages and two TF32 stage buffers (four BF16)
constexpr size_t GEMM_TC_STAGE_BYTES =
    (size_t)(TC_RAW * TC_RAW_STAGE_FLOATS + TC_MIN_PIPE * TC_STAGE_FLOATS) * sizeof(float);

struct GemmArgs {
  int M, N, K;
  const float2* A;
  long long sam, sak, sab;
  int conjA;
  const float2* B;
  long long sbk, sbn, sbb;
  int conjB;
  float2* C;
  long long scm, scn, scb;
};

__global__ void __launch_bounds__(GEMM_NT, 1) k_cgemm(GemmArgs g, int mode, int* err) {
  extern __shared__ __align__(128) unsigned char raw[];
  const int b = blockIdx.x;
  const float2* A = g.A + (size_t)b * g.sab;
  const float2* B = g.B + (size_t)b * g.sbb;
  float2* C = g.C + (size_t)b * g.scb;
  if (mode == DCS_GEMM_TENSOR || mode == DCS_GEMM_TENSOR_BF16X3) {
    TcState t;
    t.stage = reinterpret_cast<float*>(raw);
    t.stage_bytes = GEMM_TC_STAGE_BYTES;
    uint64_t* tail = reinterpret_cast<uint64_t*>(raw + GEMM_TC_STAGE_BYTES);
    t.mbar = tail;
    t.uses = reinterpret_cast<int*>(tail + TC_NBAR);
    t.tmem = reinterpret_cast<uint32_t*>(t.uses + 2);
    t.err = reinterpret_cast<int*>(t.tmem + 1);
    tc_setup(t);
    t.bf16 = mode == DCS_GEMM_TENSOR_BF16X3;
    cta_cgemm_tc<GEMM_NT>(g.M, g.N, g.K, A, (int)g.sam, (int)g.sak, g.conjA, B, (int)g.sbk,
                          (int)g.sbn, g.conjB, C, (int)g.scm, (int)g.scn, t);
    if (threadIdx.x == 0 && *t.err) atomicOr(err, 1);
    tc_teardown(t);
  } else {
    float2* sA = reinterpret_cast<float2*>(raw);
    float2* sB = sA + GBM * GSA_LD;
    cta_cgemm<GEMM_NT>(g.M, g.N, g.K, A, (int)g.sam, (int)g.sak, g.conjA, B, (int)g.sbk,
                       (int)g.sbn, g.conjB, C, (int)g.scm, (int)g.scn, sA, sB);
  }
}

}  // namespace

extern "C" dcs_status_t dcs_cgemm(int32_t mode, int32_t batch, int32_t M, int32_t N, int32_t K,
                                 const void* A, int64_t sam, int64_t sak, int64_t sab,
                                 int32_t conjA, const void* B, int64_t sbk, int64_t sbn,
                                 int64_t sbb, int32_t conjB, void* C, int64_t scm, int64_t scn,
                                 int64_t scb, int32_t* err_dev, dcs_stream_t stream) {
  const bool tensor = mode == DCS_GEMM_TENSOR || mode == DCS_GEMM_TENSOR_BF16X3;
  if (batch < 0 || M < 0 || N < 0 || K < 0 || (mode != DCS_GEMM_SIMT && !tensor))
    return DCS_ERR_INVALID;
  if (batch == 0 || M == 0 || N == 0) return DCS_OK;
  if (!A || !B || !C || (tensor && !err_dev)) return DCS_ERR_INVALID;
  const long long lim = 1ll << 31;
  if (sam >= lim || sak >= lim || sbk >= lim || sbn >= lim || scm >= lim || scn >= lim)
    return DCS_ERR_UNSUPPORTED;
  GemmArgs g{M, N, K, static_cast<const float2*>(A), sam, sak, sab, conjA,
             static_cast<const float2*>(B), sbk, sbn, sbb, conjB, static_cast<float2*>(C),
             scm, scn, scb};
  const size_t smem = tensor
                          ? GEMM_TC_STAGE_BYTES + 256
                          : sizeof(float2) * GEMM_SIMT_SMEM_ELEMS;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaFuncSetAttribute(k_cgemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return DCS_ERR_CUDA;
  k_cgemm<<<batch, GEMM_NT, smem, s>>>(g, mode, err_dev);
  return cudaGetLastError() == cudaSuccess ? DCS_OK : DCS_ERR_CUDA;
}
