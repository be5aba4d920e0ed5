// Compression step with every tile in shared memory (bond dimension up to
// DCS_MAX_CHI_FUSED): one CTA per slot.
#include "dcs_common.cuh"

namespace dcs {

template <int NT>
__global__ void __launch_bounds__(NT, MinBlocks<NT>::value) k_compress(DevCtx c, int C,
                                                 const DLayer* __restrict__ L,
                                                 const DBlock* __restrict__ BK,
                                                 const DGate1* __restrict__ G1,
                                                 const DCond* __restrict__ CD, double* fid_out) {
  const int pos = blockIdx.x;
  if (pos >= *c.count) return;
  const int slot = c.order[pos];
  extern __shared__ __align__(16) unsigned char smraw[];
  Work sm;
  carve(sm, smraw, C, nullptr);
  const int n = c.n;
  if (threadIdx.x < DCS_CWORDS) sm.creg[threadIdx.x] = c.creg[(size_t)slot * DCS_CWORDS + threadIdx.x];
  __syncthreads();
  // a slot on which every gate of the chunk is skipped is left unchanged
  if (!L->uncond) {
    if (threadIdx.x == 0) {
      int any = 0;
      for (int i = 0; i < L->n_conds && !any; ++i) any = cond_holds(CD[L->cond_off + i], sm.creg);
      sm.iv[4] = any;
    }
    __syncthreads();
    if (!sm.iv[4]) {
      if (threadIdx.x == 0 && fid_out) fid_out[slot] = 1.0;
      return;
    }
  }
  const int kb = c.ketbuf[slot], bb = 1 - kb;
  const int* kbonds = bonds_ptr(c, slot, kb);
  for (int i = threadIdx.x; i <= n; i += NT) {
    sm.abnd[i] = kbonds[i];
    sm.bnd[i] = kbonds[i];
  }
  __syncthreads();
  int centre = c.centre[slot];
  if (threadIdx.x == 0) {
    sm.iv[7] = 1;    // the guess is exact (no truncation beyond the tolerance) so far
    sm.dv[1] = 1.0;  // product of the kept weight fractions
  }
  PHASE_START();
  // ---- initial guess: copy the sites it touches, then apply the chunk block by block
  int lo, hi;
  guess_range(L, BK, n, centre, lo, hi);
  if (C == 4) {
    copy_sites4<NT>(c, bb, kb, slot, lo, hi, sm.abnd);
    __syncthreads();
    apply_lone_1q_threads<NT>(c, sm, bb, slot, L, G1);
  } else {
    for (int j = lo; j <= hi; ++j)
      gcopy<NT>(site_ptr(c, bb, slot, j), site_ptr(c, kb, slot, j), sm.abnd[j] * 2 * sm.abnd[j + 1]);
  }
  __syncthreads();
  for (int j = 0; j < n && C != 4; ++j) {
    if (L->site[j].kind != 1) continue;
    if (threadIdx.x == 0) prod1q(G1, L->site[j].g_off, L->site[j].g_n, sm.creg, sm.G);
    __syncthreads();
    float2* p = site_ptr(c, bb, slot, j);
    const int bl = sm.bnd[j], br = sm.bnd[j + 1];
    for (int idx = threadIdx.x; idx < bl * br; idx += NT) {
      const int a = idx / br, x = idx % br;
      const float2 v0 = p[(a * 2 + 0) * br + x], v1 = p[(a * 2 + 1) * br + x];
      float2 o0 = cz(), o1 = cz();
      cfma(o0, sm.G[0], v0);
      cfma(o0, sm.G[1], v1);
      cfma(o1, sm.G[2], v0);
      cfma(o1, sm.G[3], v1);
      p[(a * 2 + 0) * br + x] = o0;
      p[(a * 2 + 1) * br + x] = o1;
    }
    __syncthreads();
  }
  const bool asc = guess_ascending(L, BK, centre);
  for (int t = 0; t < L->n_blocks; ++t) {
    const DBlock& blk = BK[L->blk_off + (asc ? L->n_blocks - 1 - t : t)];
    const int q = blk.q;
    PHASE_MARK(10);
    move_centre<NT>(c, sm, bb, slot, centre, centre <= q ? q : q + 1);
    PHASE_MARK(11);
    const int b0 = sm.bnd[q], b1 = sm.bnd[q + 1], b2 = sm.bnd[q + 2];
    gcopy<NT>(sm.S, site_ptr(c, bb, slot, q), b0 * 2 * b1);
    gcopy<NT>(sm.F, site_ptr(c, bb, slot, q + 1), b1 * 2 * b2);
    if (blk.composed) {
      if (threadIdx.x < 16) sm.G[threadIdx.x] = blk.Gc[threadIdx.x];
    } else if (threadIdx.x == 0) {
      build_block(blk, G1, sm.creg, sm.G);
    }
    __syncthreads();
    const int m = 2 * b0, nn = 2 * b2;
    // X = Theta, column-major with leading dimension ldx (8 when every bond <= 4: the row
    // and column of an entry then come from shifts)
    const int ldx = C == 4 ? 8 : m;
    float2* X = sm.T;
    float2* V = sm.T + 4 * C * C;
    // P[(a t), (v b)] = sum_x B_q[a][t][x] B_{q+1}[x][v][b]
    if (C == 4) {
      for (int idx = threadIdx.x; idx < 64; idx += NT) {
        const int row = idx & 7, col = idx >> 3;
        if (row < m && col < nn) {
          float2 acc = cz();
          for (int x = 0; x < b1; ++x) cfma(acc, sm.S[row * b1 + x], sm.F[x * nn + col]);
          X[row + col * 8] = acc;
        }
      }
    } else {
      for (int idx = threadIdx.x; idx < m * nn; idx += NT) {
        const int row = idx % m, col = idx / m;
        float2 acc = cz();
        for (int x = 0; x < b1; ++x) cfma(acc, sm.S[row * b1 + x], sm.F[x * nn + col]);
        X[row + col * m] = acc;
      }
    }
    __syncthreads();
    // Theta[(a s), (u b)] = sum_{t v} G[(s u), (t v)] P[(a t), (v b)]  (in place per (a, b))
    for (int idx = threadIdx.x; idx < b0 * b2; idx += NT) {
      const int a = idx / b2, bcol = idx % b2;
      float2 in[4], out[4];
#pragma unroll
      for (int t = 0; t < 2; ++t)
#pragma unroll
        for (int v = 0; v < 2; ++v) in[t * 2 + v] = X[(a * 2 + t) + (v * b2 + bcol) * ldx];
#pragma unroll
      for (int o = 0; o < 4; ++o) {
        float2 acc = cz();
#pragma unroll
        for (int i = 0; i < 4; ++i) cfma(acc, sm.G[o * 4 + i], in[i]);
        out[o] = acc;
      }
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int u = 0; u < 2; ++u) X[(a * 2 + s) + (u * b2 + bcol) * ldx] = out[s * 2 + u];
    }
    __syncthreads();
    PHASE_MARK(12);
    const int svd_sweeps =
        cta_jacobi_svd<NT>(X, m, nn, ldx, V, nn, sm.sig2, sm.sigf, sm.perm, &sm.iv[5], sm.red);
    (void)svd_sweeps;
#ifdef DCS_PHASE_TIMERS
    if (threadIdx.x == 0) {
      atomicAdd(&g_phase_cycles[22], (unsigned long long)svd_sweeps);
      atomicAdd(&g_phase_cycles[23], 1ull);
    }
#endif
    PHASE_MARK(13);
    int k;
    float inv;
    if constexpr (NT == 32) {  // one warp: lane-parallel rank decision, FP32
      float kept, disc;
      k = warp_trunc_rank(sm.sigf, sm.perm, nn, c.chi_max, c.tol, kept, disc);
      const float tot = kept + disc;
      inv = 1.f / sqrtf(kept);
      if (threadIdx.x == 0) {
        // exact unless the rank was capped by chi_max above the tolerance
        if (disc > (float)c.tol * tot) sm.iv[7] = 0;
        if (tot > 0.f && disc > 0.f) sm.dv[1] *= 1.0 - (double)(disc / tot);
      }
    } else {
      if (threadIdx.x == 0) {
        const int kk = trunc_rank(sm.sig2, sm.perm, nn, c.chi_max, c.tol);
        double w = 0.0, tot = 0.0;
        for (int i = 0; i < nn; ++i) tot += sm.sig2[i];
        for (int i = 0; i < kk; ++i) w += sm.sig2[sm.perm[i]];
        sm.iv[6] = kk;
        sm.dv[0] = w;
        // exact unless the rank was capped by chi_max above the tolerance
        if (tot - w > c.tol * tot) sm.iv[7] = 0;
        if (tot > 0.0) sm.dv[1] *= w / tot;
      }
      __syncthreads();
      k = sm.iv[6];
      inv = (float)(1.0 / sqrt(sm.dv[0]));
    }
    // the singular values go to the site facing the next block: B_q = U S, B_{q+1} = Vh
    // (descending, centre q) or B_q = U, B_{q+1} = S Vh (ascending, centre q+1); X = U S
    float2* pq = site_ptr(c, bb, slot, q);
    for (int idx = threadIdx.x; idx < m * k; idx += NT) {
      const int row = idx / k, kk = idx % k;
      const float sg = sm.sigf[sm.perm[kk]];
      const float sc = asc ? (sg > 0.f ? 1.f / sqrtf(sg) : 0.f) : inv;
      pq[idx] = cscale(X[row + sm.perm[kk] * ldx], sc);
    }
    float2* pq1 = site_ptr(c, bb, slot, q + 1);
    for (int idx = threadIdx.x; idx < k * nn; idx += NT) {
      const int kk = idx / nn, col = idx % nn;
      const float2 v = cconj(V[col + sm.perm[kk] * nn]);
      pq1[idx] = asc ? cscale(v, sqrtf(sm.sigf[sm.perm[kk]]) * inv) : v;
    }
    __syncthreads();
    if (threadIdx.x == 0) sm.bnd[q + 1] = k;
    centre = asc ? q + 1 : q;
    __syncthreads();
    PHASE_MARK(14);
  }
  PHASE_MARK(10);
  int* bt = sm.bnd;
  int* at = sm.abnd;
  double fval = 0.0;
  // An exact guess is the target W|A> itself, already the optimum of every one-site update:
  // the sweeps would return it unchanged (f = 1 up to the tolerance), so they are skipped and
  // the touched sites go back into the ket buffer, the centre staying where the guess left it.
  const bool exact = sm.iv[7] != 0;
  if (exact) {
    if (C == 4) {
      copy_sites4<NT>(c, kb, bb, slot, lo, hi, bt);
    } else {
      for (int j = lo; j <= hi; ++j)
        gcopy<NT>(site_ptr(c, kb, slot, j), site_ptr(c, bb, slot, j), bt[j] * 2 * bt[j + 1]);
    }
    fval = sm.dv[1];
  } else {
  for (int j = 0; j < n; ++j)
    if (j < lo || j > hi) gcopy<NT>(site_ptr(c, bb, slot, j), site_ptr(c, kb, slot, j), at[j] * 2 * at[j + 1]);
  __syncthreads();
  // the sweeps start at the end of the chain nearest the centre the guess left
  const int first = centre <= n - 1 - centre ? 0 : 1;  // 0: left to right first
  move_centre<NT>(c, sm, bb, slot, centre, first == 0 ? 0 : n - 1);
  if (threadIdx.x == 0) sm.E[0] = make_float2(1.f, 0.f);
  __syncthreads();
  // ---- left environments of the guess: L_j for j = 1 .. n-1 (first sweep right to left)
  for (int j = 0; first == 1 && j < n - 1; ++j) {
    if (threadIdx.x == 0) build_W(j, L, BK, G1, sm.creg, sm.W, &sm.iv[0], &sm.iv[1]);
    __syncthreads();
    const int dl = sm.iv[0], dr = sm.iv[1], Dm = dl > dr ? dl : dr;
    const int nb = bt[j], nc = bt[j + 1], na = at[j], nx = at[j + 1];
    const int m = 2 * nb;
    gcopy<NT>(sm.S, site_ptr(c, kb, slot, j), na * 2 * nx);
    const float2* Bj = site_ptr(c, bb, slot, j);
    for (int idx = threadIdx.x; idx < m * nc; idx += NT) {  // Q[(b s), c] = B[b][s][c]
      const int row = idx / nc, cc = idx % nc;
      sm.R[row + cc * m] = Bj[idx];
    }
    __syncthreads();
    c1_env_site<NT>(sm.E, sm.S, sm.T, nb, dl, na, nx, Dm);
    c2_mix<NT>(sm.T, sm.W, nb, dl, dr, nx, Dm);
    c4_env_update<NT>(sm.R, m, sm.T, sm.E, nb, dr, nx, nc, Dm);
    gcopy<NT>(env_ptr(c, slot, j + 1), sm.E, nc * dr * nx);
    __syncthreads();
  }
  // ---- right environments of the guess: R_j for j = n-1 .. 1 (mirrored env updates)
  for (int j = n - 1; first == 0 && j >= 1; --j) {
    if (threadIdx.x == 0) build_W(j, L, BK, G1, sm.creg, sm.W, &sm.iv[0], &sm.iv[1]);
    __syncthreads();
    const int dl = sm.iv[0], dr = sm.iv[1], Dm = dl > dr ? dl : dr;
    for (int i = threadIdx.x; i < dr * 4 * dl; i += NT) {  // W'[e][s][t][d] = W[d][s][t][e]
      const int d = i % dl, st = (i / dl) % 4, e = i / (4 * dl);
      sm.W2[i] = sm.W[(d * 4 + st) * dr + e];
    }
    const float2* A = site_ptr(c, kb, slot, j);
    const int al = at[j], ar = at[j + 1];
    for (int idx = threadIdx.x; idx < al * 2 * ar; idx += NT) {  // S'[x][t][a] = A[a][t][x]
      const int x = idx % ar, t = (idx / ar) & 1, a = idx / (2 * ar);
      sm.S[(x * 2 + t) * al + a] = A[idx];
    }
    const float2* Bj = site_ptr(c, bb, slot, j);
    const int bl = bt[j], br = bt[j + 1];
    const int ldq = 2 * br;
    for (int idx = threadIdx.x; idx < bl * 2 * br; idx += NT) {  // Q'[(c s), b] = B[b][s][c]
      const int x = idx % br, s = (idx / br) & 1, bq = idx / (2 * br);
      sm.R[(x * 2 + s) + bq * ldq] = Bj[idx];
    }
    __syncthreads();
    c1_env_site<NT>(sm.E, sm.S, sm.T, br, dr, ar, al, Dm);
    c2_mix<NT>(sm.T, sm.W2, br, dr, dl, al, Dm);
    c4_env_update<NT>(sm.R, ldq, sm.T, sm.E, br, dl, al, bl, Dm);
    gcopy<NT>(env_ptr(c, slot, j), sm.E, bl * dl * al);
    __syncthreads();
  }
  // ---- one-site sweeps
  for (int sw = 0; sw < c.sweeps; ++sw) {
    if (threadIdx.x == 0) sm.E[0] = make_float2(1.f, 0.f);
    __syncthreads();
    if (((sw + first) & 1) == 0) {  // left to right
      for (int j = 0; j < n; ++j) {
        if (threadIdx.x == 0) build_W(j, L, BK, G1, sm.creg, sm.W, &sm.iv[0], &sm.iv[1]);
        __syncthreads();
        const int dl = sm.iv[0], dr = sm.iv[1], Dm = dl > dr ? dl : dr;
        const int nb = bt[j], nc = bt[j + 1], na = at[j], nx = at[j + 1];
        gcopy<NT>(sm.S, site_ptr(c, kb, slot, j), na * 2 * nx);
        if (j < n - 1) gcopy<NT>(sm.R, env_ptr(c, slot, j + 1), nc * dr * nx);
        else if (threadIdx.x == 0) sm.R[0] = make_float2(1.f, 0.f);
        __syncthreads();
        c1_env_site<NT>(sm.E, sm.S, sm.T, nb, dl, na, nx, Dm);
        c2_mix<NT>(sm.T, sm.W, nb, dl, dr, nx, Dm);
        c3_site_env<NT>(sm.T, sm.R, sm.F, nb, dr, nx, nc, Dm);
        const int m = 2 * nb;
        float2* dst = site_ptr(c, bb, slot, j);
        if (j < n - 1) {
          const int r = cta_qr<NT>(sm.F, m, nc, m, sm.R, m, nullptr, 0, sm.tau, sm.alph, sm.red);
          for (int idx = threadIdx.x; idx < m * r; idx += NT) {
            const int row = idx / r, k = idx % r;
            dst[idx] = sm.R[row + k * m];
          }
          c4_env_update<NT>(sm.R, m, sm.T, sm.E, nb, dr, nx, r, Dm);
          gcopy<NT>(env_ptr(c, slot, j + 1), sm.E, r * dr * nx);
          __syncthreads();
          if (threadIdx.x == 0) bt[j + 1] = r;
          __syncthreads();
        } else {
          double s2 = 0.0;
          for (int i = threadIdx.x; i < m; i += NT) s2 += cabs2d(sm.F[i]);
          s2 = block_sum<NT>(s2, sm.red);
          const float inv = (float)(1.0 / sqrt(s2));
          for (int i = threadIdx.x; i < m; i += NT) dst[i] = cscale(sm.F[i], inv);
          fval = s2;
          __syncthreads();
        }
      }
      centre = n - 1;
    } else {  // right to left, mirrored
      for (int j = n - 1; j >= 0; --j) {
        if (threadIdx.x == 0) build_W(j, L, BK, G1, sm.creg, sm.W, &sm.iv[0], &sm.iv[1]);
        __syncthreads();
        const int dl = sm.iv[0], dr = sm.iv[1], Dm = dl > dr ? dl : dr;
        for (int i = threadIdx.x; i < dr * 4 * dl; i += NT) {
          const int d = i % dl, st = (i / dl) % 4, e = i / (4 * dl);
          sm.W2[i] = sm.W[(d * 4 + st) * dr + e];
        }
        const int nb = bt[j + 1], nc = bt[j], na = at[j + 1], nx = at[j];
        const float2* A = site_ptr(c, kb, slot, j);
        for (int idx = threadIdx.x; idx < nx * 2 * na; idx += NT) {
          const int x = idx % na, t = (idx / na) & 1, a = idx / (2 * na);
          sm.S[(x * 2 + t) * nx + a] = A[idx];
        }
        if (j > 0) gcopy<NT>(sm.R, env_ptr(c, slot, j), nc * dl * nx);
        else if (threadIdx.x == 0) sm.R[0] = make_float2(1.f, 0.f);
        __syncthreads();
        c1_env_site<NT>(sm.E, sm.S, sm.T, nb, dr, na, nx, Dm);
        c2_mix<NT>(sm.T, sm.W2, nb, dr, dl, nx, Dm);
        c3_site_env<NT>(sm.T, sm.R, sm.F, nb, dl, nx, nc, Dm);
        const int m = 2 * nb;
        float2* dst = site_ptr(c, bb, slot, j);
        if (j > 0) {
          const int r = cta_qr<NT>(sm.F, m, nc, m, sm.R, m, nullptr, 0, sm.tau, sm.alph, sm.red);
          // B_j[k][s][c] = Q'[(c s), k]
          for (int idx = threadIdx.x; idx < r * 2 * nb; idx += NT) {
            const int cc = idx % nb, s = (idx / nb) & 1, k = idx / (2 * nb);
            dst[idx] = sm.R[(cc * 2 + s) + k * m];
          }
          c4_env_update<NT>(sm.R, m, sm.T, sm.E, nb, dl, nx, r, Dm);
          gcopy<NT>(env_ptr(c, slot, j), sm.E, r * dl * nx);
          __syncthreads();
          if (threadIdx.x == 0) bt[j] = r;
          __syncthreads();
        } else {
          double s2 = 0.0;
          for (int i = threadIdx.x; i < m; i += NT) s2 += cabs2d(sm.F[i]);
          s2 = block_sum<NT>(s2, sm.red);
          const float inv = (float)(1.0 / sqrt(s2));
          for (int idx = threadIdx.x; idx < m; idx += NT) {  // B_0[0][s][c] = F'[(c s), 0]
            const int cc = idx % nb, s = idx / nb;
            dst[idx] = cscale(sm.F[cc * 2 + s], inv);
          }
          fval = s2;
          __syncthreads();
        }
      }
      centre = 0;
    }
  }
  }  // not exact
  PHASE_MARK(15);
  // ---- the bra becomes the ket (an exact guess was written back into the ket buffer)
  const int nb_ = exact ? kb : bb;
  int* obonds = bonds_ptr(c, slot, nb_);
  for (int i = threadIdx.x; i <= n; i += NT) obonds[i] = bt[i];
  if (threadIdx.x == 0) {
    c.centre[slot] = centre;
    c.ketbuf[slot] = nb_;
    if (!(fval == fval) || fval > 1e300) c.flags[slot] |= DCS_FLAG_NUMERICAL;
    c.F[slot] *= fval;
    if (fid_out) fid_out[slot] = fval;
    if (c.counters) {
      atomicAdd(&c.counters[0], 1ull);
      atomicAdd(&c.counters[1], exact ? 0ull : (unsigned long long)c.sweeps);
    }
  }
}


template <int NT>
static void compress_c(const DevCtx& c, int C, const DLayer* L, const DBlock* B, const DGate1* G1,
                       const DCond* CD, double* fid_out, cudaStream_t s) {
  const size_t sm = work_small_bytes(C, false) + sizeof(float2) * work_tile_elems(C, false);
  cudaFuncSetAttribute(k_compress<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_compress<NT><<<c.n_slots, NT, sm, s>>>(c, C, L, B, G1, CD, fid_out);
}

void launch_compress(const DevCtx& c, int tile_chi, const DLayer* L, int nsub, const DBlock* B,
                     const DGate1* G1, const DCond* CD, double* fid_out, cudaStream_t s) {
  if (c.work) {
    launch_compress_big(c, L, nsub, B, G1, CD, fid_out, s);
    return;
  }
  if (nsub != 1) return;  // chunks of several layers take the large-tile path
  switch (tile_chi) {
    case 4: compress_c<32>(c, 4, L, B, G1, CD, fid_out, s); break;
    case 8: compress_c<32>(c, 8, L, B, G1, CD, fid_out, s); break;
    case 16: compress_c<64>(c, 16, L, B, G1, CD, fid_out, s); break;
    case 32: compress_c<128>(c, 32, L, B, G1, CD, fid_out, s); break;
    default: break;
  }
}

}  // namespace dcs
