// The large-tile compression kernel with FP32 CUDA-core contractions, and the launcher of
// both large-tile variants (the tensor-core one is compiled in dcs_k_big_tc.cu).
#include "dcs_k_big.cuh"

namespace dcs {

void launch_compress_big_tc(const DevCtx& c, const DLayer* L, int nsub, const DBlock* B,
                            const DGate1* G1, const DCond* CD, double* fid_out, cudaStream_t s);

void launch_compress_big(const DevCtx& c, const DLayer* L, int nsub, const DBlock* B,
                         const DGate1* G1, const DCond* CD, double* fid_out, cudaStream_t s) {
  // the tensor-core tiles live in the staging region; the bond cap keeps it large enough
  if (c.use_tc && big_stage_bytes(c.chi_cap) >= sizeof(float) * TC_SMEM_FLOATS) {
    launch_compress_big_tc(c, L, nsub, B, G1, CD, fid_out, s);
    return;
  }
  const size_t sm = work_small_bytes(c.chi_cap, true, false);
  cudaFuncSetAttribute(k_compress_big<BIG_NT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_compress_big<BIG_NT, false><<<c.n_slots, BIG_NT, sm, s>>>(c, c.chi_cap, L, nsub, B, G1, CD, fid_out);
}

}  // namespace dcs


#ifdef DCS_PHASE_TIMERS
// Debug builds only: the large-tile kernel's per-phase cycle sums, 24 slots (not part of
// the ABI).
extern "C" int dcs_debug_phase_cycles(unsigned long long* out, int reset) {
  if (cudaMemcpyFromSymbol(out, dcs::g_phase_cycles, sizeof(unsigned long long) * 24) != cudaSuccess)
    return 1;
  if (reset) {
    unsigned long long z[24] = {0};
    cudaMemcpyToSymbol(dcs::g_phase_cycles, z, sizeof(z));
  }
  return 0;
}
#endif
