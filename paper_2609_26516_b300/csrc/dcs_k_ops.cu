// Measurement, initialisation and branch kernels of libdcs and their launchers.
#include "dcs_common.cuh"

namespace dcs {

// ----------------------------------------------------------------------------- measurement
// mode MEAS_SAMPLE: u = Philox(seed, shot, ordinal), m = 0 iff u < p_0 (Alg. 1 Measure);
// MEAS_FORCED: m = forced[slot]; MEAS_PROB: only p_0 (MeasureProb) and the slice weights.
// p_m = <psi|P_m|psi> is evaluated at the orthogonality centre moved to q; Collapse zeroes
// the other slice of the centre tensor and rescales by 1/sqrt(r_m) (Sec. "Mid-circuit
// measurements").
template <int NT, bool BIG>
__global__ void __launch_bounds__(NT, MinBlocks<NT>::value) k_measure(DevCtx c, int C,
                                                const DMeas* __restrict__ meas,
                                                int n_meas, int mode,
                                                const uint8_t* __restrict__ forced,
                                                double* p0_out) {
  const int pos = blockIdx.x;
  if (pos >= *c.count) return;
  const int slot = c.order[pos];
  extern __shared__ __align__(16) unsigned char smraw[];
  Work sm;
  carve(sm, smraw, C, BIG ? c.work + (size_t)slot * c.work_stride : nullptr, false, c.dmax);
  const int n = c.n;
  const int kb = c.ketbuf[slot];
  int* kbonds = bonds_ptr(c, slot, kb);
  for (int i = threadIdx.x; i <= n; i += NT) sm.bnd[i] = kbonds[i];
  __syncthreads();
  int centre = c.centre[slot];
  if constexpr (NT == 32 && !BIG) {
    if (C == 4) {
      warp_measure_run4(c, sm, kb, slot, centre, meas, n_meas, mode, forced, p0_out);
      return;
    }
  }
  PHASE_START();
  for (int im = 0; im < n_meas; ++im) {
    const int q = meas[im].q;
    PHASE_MARK(17);
    move_centre<NT>(c, sm, kb, slot, centre, q);
    PHASE_MARK(16);
    const int bl = sm.bnd[q], br = sm.bnd[q + 1];
    float2* A = site_ptr(c, kb, slot, q);
    double s0 = 0.0, s1 = 0.0;
    if constexpr (NT == 32) {  // one warp: float-float sums (FP64 accuracy, FP32 pipe)
      ffloat a0{0.f, 0.f}, a1{0.f, 0.f};
      for (int idx = threadIdx.x; idx < bl * 2 * br; idx += NT) {
        const ffloat w = ff_abs2(A[idx]);
        if ((idx / br) & 1) a1 = ff_add(a1, w);
        else a0 = ff_add(a0, w);
      }
      s0 = ff_to_double(ff_warp_sum(a0));
      s1 = ff_to_double(ff_warp_sum(a1));
    } else {
      for (int idx = threadIdx.x; idx < bl * 2 * br; idx += NT) {
        const double w = cabs2d(A[idx]);
        if ((idx / br) & 1) s1 += w;
        else s0 += w;
      }
      s0 = block_sum<NT>(s0, sm.red);
      s1 = block_sum<NT>(s1, sm.red);
    }
    const double tot = s0 + s1;
    const double p0 = s0 / tot;
    if (mode == MEAS_PROB) {
      if (threadIdx.x == 0) {
        if (p0_out) p0_out[slot] = p0;
        c.rr[2 * (size_t)slot] = s0;
        c.rr[2 * (size_t)slot + 1] = s1;
        if (!(p0 == p0)) c.flags[slot] |= DCS_FLAG_NUMERICAL;
      }
      continue;
    }
    int m;
    if (mode == MEAS_SAMPLE) {
      const double u = philox_uniform(c.seed, c.shot[slot], meas[im].ordinal);
      m = (u < p0) ? 0 : 1;
      if (threadIdx.x == 0 && fabs(u - p0) < 1e-6) c.flags[slot] |= DCS_FLAG_DRAW_NEAR_THRESHOLD;
    } else {
      m = forced[slot] ? 1 : 0;
    }
    const double pm = m ? (1.0 - p0) : p0;
    const double rm = m ? s1 : s0;
    if (!(pm > 1e-12)) {
      if (threadIdx.x == 0) c.flags[slot] |= (pm == pm) ? DCS_FLAG_ZERO_PROB : DCS_FLAG_NUMERICAL;
      __syncthreads();
      continue;
    }
    const float sc = NT == 32 ? 1.f / sqrtf((float)rm) : (float)(1.0 / sqrt(rm));
    for (int idx = threadIdx.x; idx < bl * 2 * br; idx += NT) {
      const int s = (idx / br) & 1;
      A[idx] = (s == m) ? cscale(A[idx], sc) : cz();
    }
    if (threadIdx.x == 0) {
      c.p[slot] *= pm;
      const int cb = meas[im].cbit;
      uint64_t& w = c.creg[(size_t)slot * DCS_CWORDS + (cb >> 6)];
      w = (w & ~(1ull << (cb & 63))) | ((uint64_t)m << (cb & 63));
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i <= n; i += NT) kbonds[i] = sm.bnd[i];
  if (threadIdx.x == 0) c.centre[slot] = centre;
}

// ----------------------------------------------------------------------------- init
// The bond-sized layout offsets (layout_offsets) written to the arena's offset tables.
__global__ void k_layout(DevCtx c) {
  if (threadIdx.x == 0) {
    size_t me = 0, ee = 0;
    layout_offsets(c.n, c.chi_cap, c.dmax, const_cast<size_t*>(c.site_off),
                   const_cast<size_t*>(c.env_off), &me, &ee);
  }
}

__global__ void k_init(DevCtx c, int n_active, int multipath, uint64_t shot0) {
  const int slot = blockIdx.x;
  const int n = c.n;
  if (slot >= c.n_slots) return;
  if (slot == 0 && threadIdx.x == 0) {
    *c.count = multipath ? 1 : n_active;
    *c.status = 0;
    if (c.counters) c.counters[0] = c.counters[1] = 0ull;
  }
  if (threadIdx.x == 0) c.order[slot] = slot;
  const bool active = multipath ? (slot == 0) : (slot < n_active);
  if (!active) return;
  for (int i = threadIdx.x; i <= n; i += blockDim.x) {
    bonds_ptr(c, slot, 0)[i] = 1;
    bonds_ptr(c, slot, 1)[i] = 1;
  }
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    float2* p = site_ptr(c, 0, slot, j);
    p[0] = make_float2(1.f, 0.f);
    p[1] = cz();
  }
  if (threadIdx.x < DCS_CWORDS) c.creg[(size_t)slot * DCS_CWORDS + threadIdx.x] = 0ull;
  if (threadIdx.x == 0) {
    c.centre[slot] = 0;
    c.ketbuf[slot] = 0;
    c.p[slot] = 1.0;
    c.F[slot] = 1.0;
    c.flags[slot] = 0u;
    c.shot[slot] = shot0 + (uint64_t)slot;
    c.rr[2 * (size_t)slot] = 1.0;
    c.rr[2 * (size_t)slot + 1] = 0.0;
  }
}

// ----------------------------------------------------------------------------- branches
// TopK selection key (Alg. 2 "keep the M branches with largest p", ties read as list order):
// key = round(p / (1e-5 * max p)); a larger key wins, equal keys keep the earlier position.
__device__ __forceinline__ long long topk_key(double p, double pmax) {
  return (long long)floor(p / (1e-5 * pmax) + 0.5);
}

// One CTA.  Children of the current list (parent positions in order, m = 0 before m = 1,
// kept when p_m > eps), optionally pruned to M, assigned to slots: the first kept child of a
// parent inherits the parent's slot, a second one takes a free slot (copied from the
// parent before the collapses run).
__global__ void k_branch_plan(DevCtx c, double eps, int M, int cbit, double pmin) {
  __shared__ int s_nchild[1024];
  __shared__ int s_start[1025];
  __shared__ double s_cp[2048];
  __shared__ int s_keep[2048];
  __shared__ int s_slot[2048];
  __shared__ int s_free[1024];
  __shared__ int s_err;
  __shared__ double s_pmax;
  const int cnt = *c.count;
  const int ns = c.n_slots;
  if (threadIdx.x == 0) {
    s_err = 0;
    if (ns > 1024) s_err = 1;
  }
  __syncthreads();
  if (s_err) {
    if (threadIdx.x == 0) *c.status |= 1 << DCS_ERR_UNSUPPORTED;
    return;
  }
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    const int slot = c.order[i];
    const double r0 = c.rr[2 * (size_t)slot], r1 = c.rr[2 * (size_t)slot + 1];
    const double p0 = r0 / (r0 + r1), p1 = 1.0 - p0;
    s_nchild[i] = (p0 > eps) + (p1 > eps);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    s_start[0] = 0;
    for (int i = 0; i < cnt; ++i) s_start[i + 1] = s_start[i] + s_nchild[i];
  }
  __syncthreads();
  const int nch = s_start[cnt];
  if (nch > ns || nch > 2048) {
    if (threadIdx.x == 0) {
      *c.status |= 1 << DCS_ERR_OOM;
      c.plan[0] = 0;
      c.plan[1] = 0;
      c.plan[2] = cnt;
    }
    return;
  }
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    const int slot = c.order[i];
    const double r0 = c.rr[2 * (size_t)slot], r1 = c.rr[2 * (size_t)slot + 1];
    const double p0 = r0 / (r0 + r1), p1 = 1.0 - p0;
    int k = s_start[i];
    if (p0 > eps) s_cp[k++] = c.p[slot] * p0;
    if (p1 > eps) s_cp[k++] = c.p[slot] * p1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double pm = 0.0;
    for (int i = 0; i < nch; ++i) pm = fmax(pm, s_cp[i]);
    s_pmax = pm;
  }
  __syncthreads();
  // kept: the top M by key (all when M = 0 or no more than M), then, with adaptive pruning,
  // only those with p >= pmin (the first of the key order always stays)
  const bool topm = M > 0 && nch > M;
  for (int i = threadIdx.x; i < nch; i += blockDim.x) {
    int keep = 1;
    if (topm || pmin > 0.0) {
      const long long ki = topk_key(s_cp[i], s_pmax);
      int rank = 0;
      for (int j = 0; j < nch; ++j) {
        const long long kj = topk_key(s_cp[j], s_pmax);
        rank += (kj > ki) || (kj == ki && j < i);
      }
      keep = topm ? rank < M : 1;
      if (pmin > 0.0 && rank > 0 && !(s_cp[i] >= pmin)) keep = 0;
    }
    s_keep[i] = keep;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // free slots: not used by any parent, or by a parent none of whose children is kept
    int used_mark[1];
    (void)used_mark;
    for (int s = 0; s < ns; ++s) s_free[s] = 1;
    for (int i = 0; i < cnt; ++i) {
      bool any = false;
      for (int k = s_start[i]; k < s_start[i + 1]; ++k) any = any || s_keep[k];
      if (any) s_free[c.order[i]] = 0;
    }
    int nf = 0;
    for (int s = 0; s < ns; ++s)
      if (s_free[s]) s_free[nf++] = s;
    int* copy = c.plan + PLAN_HDR;
    int* coll = c.plan + PLAN_HDR + 2 * ns;
    int ncopy = 0, ncoll = 0, newc = 0;
    int fi = 0;
    for (int i = 0; i < cnt; ++i) {
      const int slot = c.order[i];
      const double r0 = c.rr[2 * (size_t)slot], r1 = c.rr[2 * (size_t)slot + 1];
      const double p0 = r0 / (r0 + r1), p1 = 1.0 - p0;
      int k = s_start[i];
      bool parent_taken = false;
      for (int m = 0; m < 2; ++m) {
        const double pmv = m ? p1 : p0;
        if (!(pmv > eps)) continue;
        if (s_keep[k]) {
          int dst;
          if (!parent_taken) {
            dst = slot;
            parent_taken = true;
          } else {
            dst = s_free[fi++];
            copy[2 * ncopy] = slot;
            copy[2 * ncopy + 1] = dst;
            ++ncopy;
          }
          coll[2 * ncoll] = dst;
          coll[2 * ncoll + 1] = m;
          ++ncoll;
          s_slot[newc++] = dst;
        }
        ++k;
      }
    }
    c.plan[0] = ncopy;
    c.plan[1] = ncoll;
    c.plan[2] = newc;
    for (int i = 0; i < newc; ++i) c.order[i] = s_slot[i];
    *c.count = newc;
    (void)cbit;
  }
}

// Copy a whole branch (ket MPS, bonds, centre, register, p, F, rr, flags) src -> dst.
__global__ void k_branch_copy(DevCtx c) {
  const int i = blockIdx.x;
  if (i >= c.plan[0]) return;
  const int src = c.plan[PLAN_HDR + 2 * i], dst = c.plan[PLAN_HDR + 2 * i + 1];
  const int n = c.n;
  const int kb = c.ketbuf[src];
  const int* sb = bonds_ptr(c, src, kb);
  for (int j = 0; j < n; ++j) {
    const int len = sb[j] * 2 * sb[j + 1];
    const float2* s = site_ptr(c, kb, src, j);
    float2* d = site_ptr(c, kb, dst, j);
    for (int e = threadIdx.x; e < len; e += blockDim.x) d[e] = s[e];
  }
  int* db = bonds_ptr(c, dst, kb);
  for (int j = threadIdx.x; j <= n; j += blockDim.x) db[j] = sb[j];
  if (threadIdx.x < DCS_CWORDS)
    c.creg[(size_t)dst * DCS_CWORDS + threadIdx.x] = c.creg[(size_t)src * DCS_CWORDS + threadIdx.x];
  if (threadIdx.x == 0) {
    c.ketbuf[dst] = kb;
    c.centre[dst] = c.centre[src];
    c.p[dst] = c.p[src];
    c.F[dst] = c.F[src];
    c.rr[2 * (size_t)dst] = c.rr[2 * (size_t)src];
    c.rr[2 * (size_t)dst + 1] = c.rr[2 * (size_t)src + 1];
    c.flags[dst] = c.flags[src];
    c.shot[dst] = c.shot[src];
  }
}

// Collapse each planned child onto its outcome (centre already at q from MeasureProb).
__global__ void k_branch_collapse(DevCtx c, int q, int cbit) {
  const int i = blockIdx.x;
  if (i >= c.plan[1]) return;
  const int ns = c.n_slots;
  const int slot = c.plan[PLAN_HDR + 2 * ns + 2 * i], m = c.plan[PLAN_HDR + 2 * ns + 2 * i + 1];
  const int kb = c.ketbuf[slot];
  const int* b = bonds_ptr(c, slot, kb);
  const int bl = b[q], br = b[q + 1];
  const double r0 = c.rr[2 * (size_t)slot], r1 = c.rr[2 * (size_t)slot + 1];
  const double rm = m ? r1 : r0;
  const double pm = rm / (r0 + r1);
  const float sc = (float)(1.0 / sqrt(rm));
  float2* A = site_ptr(c, kb, slot, q);
  for (int idx = threadIdx.x; idx < bl * 2 * br; idx += blockDim.x) {
    const int s = (idx / br) & 1;
    A[idx] = (s == m) ? cscale(A[idx], sc) : cz();
  }
  if (threadIdx.x == 0) {
    c.p[slot] *= pm;
    uint64_t& w = c.creg[(size_t)slot * DCS_CWORDS + (cbit >> 6)];
    w = (w & ~(1ull << (cbit & 63))) | ((uint64_t)m << (cbit & 63));
  }
}

// TopK on the current list (one CTA).
__global__ void k_branch_topk(DevCtx c, int M) {
  __shared__ int s_keep[1024];
  __shared__ int s_ord[1024];
  __shared__ double s_pmax;
  const int cnt = *c.count;
  if (cnt <= M || cnt > 1024) return;
  if (threadIdx.x == 0) {
    double pm = 0.0;
    for (int i = 0; i < cnt; ++i) pm = fmax(pm, c.p[c.order[i]]);
    s_pmax = pm;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    const long long ki = topk_key(c.p[c.order[i]], s_pmax);
    int rank = 0;
    for (int j = 0; j < cnt; ++j) {
      const long long kj = topk_key(c.p[c.order[j]], s_pmax);
      rank += (kj > ki) || (kj == ki && j < i);
    }
    s_keep[i] = rank < M;
    s_ord[i] = c.order[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int k = 0;
    for (int i = 0; i < cnt; ++i)
      if (s_keep[i]) c.order[k++] = s_ord[i];
    *c.count = k;
  }
}

// Compaction of the current list by a caller's keep mask (one thread): entry i of the list
// stays iff keep[i] != 0, the kept entries in their relative order; the dropped slots become
// free for the next split.  A mask whose length n differs from the active count leaves the
// list as it is and raises DCS_ERR_INVALID in the status word.
__global__ void k_branch_keep(DevCtx c, const uint8_t* keep, int n) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int cnt = *c.count;
  if (cnt != n) {
    *c.status |= 1 << DCS_ERR_INVALID;
    return;
  }
  int k = 0;
  for (int i = 0; i < cnt; ++i)
    if (keep[i]) c.order[k++] = c.order[i];
  *c.count = k;
}

// Hybrid single-path start (one CTA per slot): the common prefix of every shot, computed once
// on slot 0, is copied into slots 1 .. n_active - 1, each keeping its own sampler counter
// shot0 + slot.  Nothing happens unless the list holds exactly one shot; k_fork_count then
// sets the list to n_active shots (a separate launch, so that no block reads the count after
// it changed).
__global__ void k_fork_shots(DevCtx c, int n_active) {
  const int dst = blockIdx.x;
  if (*c.count != 1 || dst == 0 || dst >= n_active || dst >= c.n_slots) return;
  const int src = 0;
  const int n = c.n;
  const int kb = c.ketbuf[src];
  const int* sb = bonds_ptr(c, src, kb);
  for (int j = 0; j < n; ++j) {
    const int len = sb[j] * 2 * sb[j + 1];
    const float2* s = site_ptr(c, kb, src, j);
    float2* d = site_ptr(c, kb, dst, j);
    for (int e = threadIdx.x; e < len; e += blockDim.x) d[e] = s[e];
  }
  int* db = bonds_ptr(c, dst, kb);
  for (int j = threadIdx.x; j <= n; j += blockDim.x) db[j] = sb[j];
  if (threadIdx.x < DCS_CWORDS)
    c.creg[(size_t)dst * DCS_CWORDS + threadIdx.x] = c.creg[(size_t)src * DCS_CWORDS + threadIdx.x];
  if (threadIdx.x == 0) {
    c.ketbuf[dst] = kb;
    c.centre[dst] = c.centre[src];
    c.p[dst] = c.p[src];
    c.F[dst] = c.F[src];
    c.rr[2 * (size_t)dst] = c.rr[2 * (size_t)src];
    c.rr[2 * (size_t)dst + 1] = c.rr[2 * (size_t)src + 1];
    c.flags[dst] = c.flags[src];
    c.shot[dst] = c.shot[src] + (uint64_t)dst;
  }
}

// The list after k_fork_shots: n_active shots, or DCS_ERR_INVALID in the status word when it
// did not hold exactly one.
__global__ void k_fork_count(DevCtx c, int n_active) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (*c.count != 1)
    *c.status |= 1 << DCS_ERR_INVALID;
  else
    *c.count = n_active;
}

// ----------------------------------------------------------------------------- launchers
int fused_chi(int chi_max) {
  if (chi_max <= 4) return 4;
  if (chi_max <= 8) return 8;
  if (chi_max <= 16) return 16;
  if (chi_max <= 32) return 32;
  return 0;
}

int big_chi(int chi_max) { return (chi_max + 7) / 8 * 8; }

size_t big_work_elems(int chi_cap, int dmax) { return work_tile_elems(chi_cap, true, dmax); }

template <int NT, bool BIG>
static void measure_c(const DevCtx& c, int C, const DMeas* meas, int n_meas, int mode,
                      const uint8_t* forced, double* p0_out, cudaStream_t s) {
  const size_t sm = work_small_bytes(C, BIG) + (BIG ? 0 : sizeof(float2) * work_tile_elems(C, false));
  cudaFuncSetAttribute(k_measure<NT, BIG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_measure<NT, BIG><<<c.n_slots, NT, sm, s>>>(c, C, meas, n_meas, mode, forced, p0_out);
}

void launch_init(const DevCtx& c, int n_active, int multipath, uint64_t shot0, cudaStream_t s) {
  k_layout<<<1, 32, 0, s>>>(c);
  k_init<<<c.n_slots, 64, 0, s>>>(c, n_active, multipath, shot0);
}

void launch_measure(const DevCtx& c, int tile_chi, const DMeas* meas, int n_meas, int mode,
                    const uint8_t* forced, double* p0_out, cudaStream_t s) {
  if (c.work) {
    measure_c<BIG_NT, true>(c, c.chi_cap, meas, n_meas, mode, forced, p0_out, s);
    return;
  }
  switch (tile_chi) {
    case 4: measure_c<32, false>(c, 4, meas, n_meas, mode, forced, p0_out, s); break;
    case 8: measure_c<32, false>(c, 8, meas, n_meas, mode, forced, p0_out, s); break;
    case 16: measure_c<64, false>(c, 16, meas, n_meas, mode, forced, p0_out, s); break;
    case 32: measure_c<128, false>(c, 32, meas, n_meas, mode, forced, p0_out, s); break;
    default: break;
  }
}

void launch_branch_split(const DevCtx& c, int q, int cbit, double eps, int M, double pmin,
                         cudaStream_t s, int* launches) {
  k_branch_plan<<<1, 256, 0, s>>>(c, eps, M, cbit, pmin);
  k_branch_copy<<<c.n_slots, 128, 0, s>>>(c);
  k_branch_collapse<<<c.n_slots, 128, 0, s>>>(c, q, cbit);
  *launches += 3;
}

void launch_branch_topk(const DevCtx& c, int M, cudaStream_t s) {
  k_branch_topk<<<1, 256, 0, s>>>(c, M);
}

void launch_branch_keep(const DevCtx& c, const uint8_t* keep, int n, cudaStream_t s) {
  k_branch_keep<<<1, 32, 0, s>>>(c, keep, n);
}

void launch_fork_shots(const DevCtx& c, int n_active, cudaStream_t s) {
  k_fork_shots<<<c.n_slots, 128, 0, s>>>(c, n_active);
  k_fork_count<<<1, 32, 0, s>>>(c, n_active);
}

}  // namespace dcs

