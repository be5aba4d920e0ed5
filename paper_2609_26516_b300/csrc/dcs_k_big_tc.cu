// The large-tile compression kernel with tcgen05 tensor-core contractions (TF32X3).
#define DCS_TU_TENSOR_CORES 1
#include "dcs_k_big.cuh"

namespace dcs {

void launch_compress_big_tc(const DevCtx& c, const DLayer* L, int nsub, const DBlock* B,
                            const DGate1* G1, const DCond* CD, double* fid_out, cudaStream_t s) {
  const size_t sm = work_small_bytes(c.chi_cap, true, true);
  cudaFuncSetAttribute(k_compress_big<BIG_NT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_compress_big<BIG_NT, true><<<c.n_slots, BIG_NT, sm, s>>>(c, c.chi_cap, L, nsub, B, G1, CD, fid_out);
}

}  // namespace dcs
