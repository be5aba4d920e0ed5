// Compression step with the large tiles in the slot's global work area (bond dimension
// above DCS_MAX_CHI_FUSED, or DCS_PATH_GLOBAL): one CTA per slot, every contraction a
// tiled complex GEMM (CUDA cores, or tcgen05 tensor cores on the TF32X3 path).
#pragma once
#include "dcs_common.cuh"

namespace dcs {

// ----------------------------------------------------------------------------- large tiles
// The guess SVD of a two-site tensor with at most 512 rows runs cta_jacobi_svd_regs with
// DCS_SVD_CPW columns per warp in registers (DCS_SVD_REGS 0: cta_jacobi_svd_staged).
#ifndef DCS_SVD_REGS
#define DCS_SVD_REGS 1
#endif
#ifndef DCS_SVD_CPW
#define DCS_SVD_CPW 2
#endif
// Blocks of at least 128 x 128 are preconditioned by a norm-sorted QR before the Jacobi
// sweeps (DCS_SVD_QRPRE 0: Jacobi on the two-site tensor itself).
#ifndef DCS_SVD_QRPRE
#define DCS_SVD_QRPRE 1
#endif


// T2[b][s][e][x] = sum_{d,t} T1(b, d, t, x) W(d, s, t, e) with T1 at
// b*ib + d*id + t*it + x*ix and T2 natural (b-stride 2 ne nx); mirrored: the coefficient is
// W[e][s][t][d] (the MPO read right to left).
// W of site j for the chunk's sub-layers L[0 .. nsub): one layer -> build_W into sm.W; more
// -> each layer's factor (build_W, thread 0) composed in order into sm.Wc, bonds grouped
// (earlier layer's, later layer's) on both sides:
//   W[(a, d)][s][v][(f, e)] = sum_u Wlater[d][s][u][e] Wearlier[a][u][v][f].
// Sets sm.iv[0], sm.iv[1] to the composed bond dimensions.  All threads call.
template <int NT>
__device__ const float2* chunk_W(int j, const DLayer* L, int nsub, const DBlock* BK,
                                 const DGate1* G1, Work& sm, int dmax) {
  if (nsub <= 1) {
    if (threadIdx.x == 0) build_W(j, L, BK, G1, sm.creg, sm.W, &sm.iv[0], &sm.iv[1]);
    __syncthreads();
    return sm.W;
  }
  // the composed tensor and two intermediates used in turn, the last product landing in fin:
  // after sub-layer l the bond is at most 4^(l+1) = dmax / 4^(nsub-1-l)
  float2* fin = sm.Wc;                                      // 4 dmax^2
  float2* midA = fin + chunk_w_fin_elems(dmax);             // 4 (dmax/4)^2: product nsub-2
  float2* midB = midA + chunk_w_mid_elems(dmax / 4);        // 4 (dmax/16)^2: product nsub-3
  float2* fac = midB + chunk_w_mid_elems(dmax / 16);        // DCS_MAX_CHUNK_LAYERS x 64
  if (threadIdx.x == 0)
    for (int l = 0; l < nsub; ++l)
      build_W(j, L + l, BK, G1, sm.creg, fac + 64 * l, &sm.iv[8 + 2 * l], &sm.iv[9 + 2 * l]);
  __syncthreads();
  const float2* cur = fac;
  int cd = sm.iv[8], ce = sm.iv[9];
  for (int l = 1; l < nsub; ++l) {
    const float2* nx = fac + 64 * l;
    const int nd = sm.iv[8 + 2 * l], ne = sm.iv[9 + 2 * l];
    float2* out = (l == nsub - 1) ? fin : ((nsub - 1 - l) & 1 ? midA : midB);
    const int od = cd * nd, oe = ce * ne;
    for (int idx = threadIdx.x; idx < od * 4 * oe; idx += NT) {
      const int oei = idx % oe, v = (idx / oe) & 1, s = (idx / (2 * oe)) & 1, odi = idx / (4 * oe);
      const int a = odi / nd, d = odi % nd, f = oei / ne, e = oei % ne;
      float2 acc = cz();
#pragma unroll
      for (int u = 0; u < 2; ++u)
        cfma(acc, nx[((d * 2 + s) * 2 + u) * ne + e], cur[((a * 2 + u) * 2 + v) * ce + f]);
      out[idx] = acc;
    }
    __syncthreads();
    cur = out;
    cd = od;
    ce = oe;
  }
  if (threadIdx.x == 0) {
    sm.iv[0] = cd;
    sm.iv[1] = ce;
  }
  __syncthreads();
  return fin;
}

template <int NT>
__device__ void mix_big(const float2* T1, int ib, int id, int it, int ix, float2* T2, const float2* W,
                        int nb, int nd, int ne, int nx, bool mirrored) {
  if (nd > 4 || ne > 4) {  // MPO bonds of a chunk of several layers: plain loops
    for (int idx = threadIdx.x; idx < nb * nx * 2 * ne; idx += NT) {
      const int x = idx % nx, e = (idx / nx) % ne, sv = (idx / (nx * ne)) & 1,
                b = idx / (nx * ne * 2);
      float2 acc = cz();
      for (int d = 0; d < nd; ++d)
#pragma unroll
        for (int t = 0; t < 2; ++t) {
          const float2 w = mirrored ? W[((e * 2 + sv) * 2 + t) * nd + d] : W[((d * 2 + sv) * 2 + t) * ne + e];
          cfma(acc, T1[(size_t)b * ib + d * id + t * it + (size_t)x * ix], w);
        }
      T2[(size_t)b * 2 * ne * nx + (sv * ne + e) * nx + x] = acc;
    }
    __syncthreads();
    return;
  }
  for (int idx = threadIdx.x; idx < nb * nx; idx += NT) {
    const int x = idx % nx, b = idx / nx;
    float2 v[8];
#pragma unroll
    for (int d = 0; d < 4; ++d)
#pragma unroll
      for (int t = 0; t < 2; ++t)
        v[d * 2 + t] = d < nd ? T1[(size_t)b * ib + d * id + t * it + (size_t)x * ix] : cz();
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        if (e >= ne) continue;
        float2 acc = cz();
#pragma unroll
        for (int d = 0; d < 4; ++d)
#pragma unroll
          for (int t = 0; t < 2; ++t) {
            if (d >= nd) continue;
            const float2 w = mirrored ? W[((e * 2 + s) * 2 + t) * nd + d] : W[((d * 2 + s) * 2 + t) * ne + e];
            cfma(acc, v[d * 2 + t], w);
          }
        T2[(size_t)b * 2 * ne * nx + (s * ne + e) * nx + x] = acc;
      }
  }
  __syncthreads();
}

// The compression step of k_compress with the large tiles in the slot's global work area
// and every contraction a tiled CTA GEMM on natural layouts:
//   T1[(b d),(t x)] = E[(b d), a] A[a, (t x)],  T2 = mix(T1, W),
//   F[(b s), c] = T2[(b s), (e x)] R[c, (e x)]^T,  E'[c, (e x)] = Q^H[c, (b s)] T2[(b s), (e x)];
// right-to-left steps read the same products on the mirrored chain.
template <int NT, bool TC>
__global__ void __launch_bounds__(NT, 1) k_compress_big(DevCtx c, int C, const DLayer* __restrict__ L,
                                                        int nsub, const DBlock* __restrict__ BK,
                                                        const DGate1* __restrict__ G1,
                                                        const DCond* __restrict__ CD, double* fid_out) {
  const int pos = blockIdx.x;
  if (pos >= *c.count) return;
  const int slot = c.order[pos];
  extern __shared__ __align__(16) unsigned char smraw[];
  Work sm;
  carve(sm, smraw, C, c.work + (size_t)slot * c.work_stride, TC, c.dmax);
  const int n = c.n;
  if (threadIdx.x < DCS_CWORDS) sm.creg[threadIdx.x] = c.creg[(size_t)slot * DCS_CWORDS + threadIdx.x];
  __syncthreads();
  bool uncond = false;
  for (int l = 0; l < nsub; ++l) uncond = uncond || L[l].uncond;
  if (!uncond) {
    if (threadIdx.x == 0) {
      int any = 0;
      for (int l = 0; l < nsub && !any; ++l)
        for (int i = 0; i < L[l].n_conds && !any; ++i)
          any = cond_holds(CD[L[l].cond_off + i], sm.creg);
      sm.iv[4] = any;
    }
    __syncthreads();
    if (!sm.iv[4]) {
      if (threadIdx.x == 0 && fid_out) fid_out[slot] = 1.0;
      return;
    }
  }
  if (TC) {
    tc_setup(sm.tc);
    sm.tc.bf16 = c.use_tc == 2;
  }
  const int kb = c.ketbuf[slot], bb = 1 - kb;
  const int* kbonds = bonds_ptr(c, slot, kb);
  for (int i = threadIdx.x; i <= n; i += NT) {
    sm.abnd[i] = kbonds[i];
    sm.bnd[i] = kbonds[i];
  }
  __syncthreads();
  int centre = c.centre[slot];
  int* bt = sm.bnd;
  int* at = sm.abnd;
  if (threadIdx.x == 0) {
    sm.iv[7] = 1;
    sm.dv[1] = 1.0;
  }
  PHASE_START();
  // ---- initial guess: the chunk applied block by block to a copy of the sites it touches
  int lo, hi;
  guess_range(L, BK, n, centre, lo, hi);
  for (int l = 1; l < nsub; ++l) {  // the sites any sub-layer touches
    int lo2, hi2;
    guess_range(L + l, BK, n, centre, lo2, hi2);
    lo = lo2 < lo ? lo2 : lo;
    hi = hi2 > hi ? hi2 : hi;
  }
  for (int j = lo; j <= hi; ++j)
    gcopy<NT>(site_ptr(c, bb, slot, j), site_ptr(c, kb, slot, j), at[j] * 2 * at[j + 1]);
  __syncthreads();
  // the sub-layers in order: each one's single-qubit sites, then its blocks
  for (int l = 0; l < nsub; ++l) {
  const DLayer* Ll = L + l;
  for (int j = 0; j < n; ++j) {
    if (Ll->site[j].kind != 1) continue;
    if (threadIdx.x == 0) prod1q(G1, Ll->site[j].g_off, Ll->site[j].g_n, sm.creg, sm.G);
    __syncthreads();
    float2* p = site_ptr(c, bb, slot, j);
    const int bl = bt[j], br = bt[j + 1];
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
  PHASE_MARK(0);
  const bool asc = guess_ascending(Ll, BK, centre);
  for (int t = 0; t < Ll->n_blocks; ++t) {
    const DBlock& blk = BK[Ll->blk_off + (asc ? Ll->n_blocks - 1 - t : t)];
    const int q = blk.q;
    move_centre<NT>(c, sm, bb, slot, centre, centre <= q ? q : q + 1);
    PHASE_MARK(1);
    const int b0 = bt[q], b1 = bt[q + 1], b2 = bt[q + 2];
    if (threadIdx.x == 0) build_block(blk, G1, sm.creg, sm.G);
    const int m = 2 * b0, nn = 2 * b2;
    float2* X = sm.T;           // m x nn, column-major (fits in T: 4 C^2)
    // P[(a t), (v b)] = B_q[(a t), x] B_{q+1}[x, (v b)]
    wgemm<NT>(sm, m, nn, b1, site_ptr(c, bb, slot, q), b1, 1, false, site_ptr(c, bb, slot, q + 1),
                  nn, 1, false, X, 1, m);
    for (int idx = threadIdx.x; idx < b0 * b2; idx += NT) {
      const int a = idx / b2, bcol = idx % b2;
      float2 in[4], out[4];
#pragma unroll
      for (int t = 0; t < 2; ++t)
#pragma unroll
        for (int v = 0; v < 2; ++v) in[t * 2 + v] = X[(a * 2 + t) + (size_t)(v * b2 + bcol) * m];
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
        for (int u = 0; u < 2; ++u) X[(a * 2 + s) + (size_t)(u * b2 + bcol) * m] = out[s * 2 + u];
    }
    __syncthreads();
    PHASE_MARK(2);
    // Truncated SVD of Theta = U S V^H, one side only: the one-sided Jacobi method
    // orthogonalises the columns of Theta (ascending: they become U S) or of Theta^H
    // (descending: V S) without accumulating the rotations, and the factor on the other
    // side comes from one GEMM with an untouched copy of Theta: S_k V_k^H = U_k^H Theta
    // (ascending), U_k S_k = Theta V_k (descending).  Neither needs S^-1.
    //
    // Large blocks are preconditioned first (Drmac-Veselic: QR with the columns in order of
    // decreasing norm, then Jacobi on R^H, which is far closer to orthogonal columns and
    // converges in fewer sweeps).  P = Theta^H (ascending) or Theta (descending) has its
    // columns sorted by norm (permutation pi), P pi = Q R (blocked Householder, GEMMs on the
    // tensor cores in the TF32X3 / BF16X3 kernels), and Z = R^H satisfies
    // pi^T P^H = Z Q^H: Z has the column space and singular values of Theta (ascending) or
    // Theta^H (descending) with its rows permuted by pi, so the orthogonalised columns of Z
    // are U (or V) with row i standing for row pi(i).  Q is not formed.
    float2* Y = sm.T2;  // ascending: a copy of Theta; descending: Theta^H (nn x m) or Z
    const int rp = asc ? nn : m, cp = asc ? m : nn;  // P: rp x cp
    const bool pre = DCS_SVD_QRPRE && rp >= 128 && cp >= 128 &&
                     qr_blocked_scratch(rp, cp) <= (size_t)(c.dmax + 2) * C * C;
    for (int idx = threadIdx.x; idx < m * nn; idx += NT) {
      if (asc) {
        Y[idx] = X[idx];
      } else if (!pre) {
        const int row = idx % m, col = idx / m;
        Y[col + (size_t)row * nn] = cconj(X[idx]);
      }
    }
    __syncthreads();
    float2* Z = asc ? X : Y;
    int zr = asc ? m : nn, zc = asc ? nn : m;
    const int* piv = nullptr;  // row i of Z stands for row piv[i] of U (V)
    if (pre) {
      int* pv = reinterpret_cast<int*>(sm.F);  // the F tile is free during the guess
      float* nrm = sm.sigf;
      if (asc) {  // squared norms of Theta's rows
        for (int i = threadIdx.x; i < m; i += NT) {
          float a = 0.f;
          for (int j = 0; j < nn; ++j) a += cabs2(X[i + (size_t)j * m]);
          nrm[i] = a;
        }
      } else {    // of its columns, one warp per column
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int j = warp; j < nn; j += NT / 32) {
          float a = 0.f;
          for (int i = lane; i < m; i += 32) a += cabs2(X[i + (size_t)j * m]);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(FULL_MASK, a, o);
          if (lane == 0) nrm[j] = a;
        }
      }
      __syncthreads();
      for (int j = threadIdx.x; j < cp; j += NT) {  // decreasing norm, ties by index
        const float v = nrm[j];
        int rank = 0;
        for (int k = 0; k < cp; ++k) {
          const float w = nrm[k];
          rank += (w > v) || (w == v && k < j);
        }
        pv[rank] = j;
      }
      __syncthreads();
      float2* Fq = sm.R;  // P pi, rp x cp column-major
      for (int idx = threadIdx.x; idx < rp * cp; idx += NT) {
        const int i = idx % rp, j = idx / rp;
        Fq[idx] = asc ? cconj(X[pv[j] + (size_t)i * m]) : X[i + (size_t)pv[j] * m];
      }
      __syncthreads();
      const int r = cta_qr_blocked<NT>(sm, Fq, rp, cp, nullptr, 0, sm.E);
      // Z = R^H (cp x r, lower triangular): ascending over Theta in X (its copy is in Y),
      // descending in Y (X keeps Theta)
      for (int idx = threadIdx.x; idx < cp * r; idx += NT) {
        const int i = idx % cp, j = idx / cp;
        Z[idx] = j < i ? cconj(Fq[j + (size_t)i * rp]) : (j == i ? cconj(sm.alph[j]) : cz());
      }
      __syncthreads();
      zr = cp;
      zc = r;
      piv = pv;
    }
    // columns of up to 512 rows: the register-resident variant
    const int svd_sweeps =
        (DCS_SVD_REGS && zr <= 512 && zc >= 2 * (NT / 32))
            ? cta_jacobi_svd_regs<NT, 16, DCS_SVD_CPW>(Z, zr, zc, zr, sm.sig2, sm.sigf, sm.perm, &sm.iv[5],
                                          sm.red, sm.stage, sm.stage_elems)
            : cta_jacobi_svd_staged<NT>(Z, zr, zc, zr, nullptr, 0, sm.sig2, sm.sigf, sm.perm,
                                        &sm.iv[5], sm.red, sm.stage, sm.stage_elems);
    (void)svd_sweeps;
#ifdef DCS_PHASE_TIMERS
    if (threadIdx.x == 0 && zc >= 64) {
      atomicAdd(&g_phase_cycles[20], (unsigned long long)svd_sweeps);
      atomicAdd(&g_phase_cycles[21], 1ull);
    }
#endif
    PHASE_MARK(3);
    if (threadIdx.x == 0) {
      const int kk = trunc_rank(sm.sig2, sm.perm, zc, c.chi_max, c.tol);
      double w = 0.0, tot = 0.0;
      for (int i = 0; i < zc; ++i) tot += sm.sig2[i];
      for (int i = 0; i < kk; ++i) w += sm.sig2[sm.perm[i]];
      sm.iv[6] = kk;
      sm.dv[0] = w;
      if (tot - w > c.tol * tot) sm.iv[7] = 0;
      if (tot > 0.0) sm.dv[1] *= w / tot;
    }
    __syncthreads();
    const int kk = sm.iv[6];
    const float inv = (float)(1.0 / sqrt(sm.dv[0]));
    float2* pq = site_ptr(c, bb, slot, q);  // singular values placed as in k_compress
    float2* pq1 = site_ptr(c, bb, slot, q + 1);
    if (asc) {
      // B_q = U_k (the kept columns, normalised), B_{q+1} = U_k^H Theta / ||S_k||
      for (int idx = threadIdx.x; idx < m * kk; idx += NT) {
        const int row = idx / kk, k2 = idx % kk;
        const float sg = sm.sigf[sm.perm[k2]];
        const int dst = piv ? piv[row] * kk + k2 : idx;
        pq[dst] = cscale(Z[row + (size_t)sm.perm[k2] * zr], sg > 0.f ? 1.f / sqrtf(sg) : 0.f);
      }
      __syncthreads();
      wgemm<NT>(sm, kk, nn, m, pq, 1, kk, true, Y, 1, m, false, pq1, nn, 1);
      __syncthreads();
      for (int idx = threadIdx.x; idx < kk * nn; idx += NT) pq1[idx] = cscale(pq1[idx], inv);
    } else {
      // B_{q+1} = V_k^H (rows: the kept columns of Theta^H, normalised and conjugated),
      // B_q = Theta V_k / ||S_k||
      for (int idx = threadIdx.x; idx < kk * nn; idx += NT) {
        const int k2 = idx / nn, col = idx % nn;
        const float sg = sm.sigf[sm.perm[k2]];
        const int dst = piv ? k2 * nn + piv[col] : idx;
        pq1[dst] = cscale(cconj(Z[col + (size_t)sm.perm[k2] * zr]), sg > 0.f ? 1.f / sqrtf(sg) : 0.f);
      }
      __syncthreads();
      wgemm<NT>(sm, m, kk, nn, X, 1, m, false, pq1, 1, nn, true, pq, kk, 1);
      __syncthreads();
      for (int idx = threadIdx.x; idx < m * kk; idx += NT) pq[idx] = cscale(pq[idx], inv);
    }
    __syncthreads();
    if (threadIdx.x == 0) bt[q + 1] = kk;
    centre = asc ? q + 1 : q;
    __syncthreads();
    PHASE_MARK(4);
  }
  }  // sub-layers
  double fval = 0.0;
  const bool exact = sm.iv[7] != 0;  // exact guess: the sweeps are skipped (see k_compress)
  if (exact) {
    for (int j = lo; j <= hi; ++j)
      gcopy<NT>(site_ptr(c, kb, slot, j), site_ptr(c, bb, slot, j), bt[j] * 2 * bt[j + 1]);
    fval = sm.dv[1];
  } else {
  for (int j = 0; j < n; ++j)
    if (j < lo || j > hi) gcopy<NT>(site_ptr(c, bb, slot, j), site_ptr(c, kb, slot, j), at[j] * 2 * at[j + 1]);
  __syncthreads();
  // the sweeps start at the end of the chain nearest the centre the guess left
  const int first = centre <= n - 1 - centre ? 0 : 1;  // 0: left to right first
  move_centre<NT>(c, sm, bb, slot, centre, first == 0 ? 0 : n - 1);
  PHASE_MARK(5);
  if (threadIdx.x == 0) sm.E[0] = make_float2(1.f, 0.f);
  __syncthreads();
  // ---- left environments of the guess (env updates with B given; first sweep right to left)
  for (int j = 0; first == 1 && j < n - 1; ++j) {
    const float2* Wj = chunk_W<NT>(j, L, nsub, BK, G1, sm, c.dmax);
    const int dl = sm.iv[0], dr = sm.iv[1];
    const int nb = bt[j], nc = bt[j + 1], na = at[j], nx = at[j + 1];
    const float2* A = site_ptr(c, kb, slot, j);
    const float2* Bj = site_ptr(c, bb, slot, j);
    wgemm<NT>(sm, nb * dl, 2 * nx, na, sm.E, na, 1, false, A, 2 * nx, 1, false, sm.T, 2 * nx, 1);
    mix_big<NT>(sm.T, dl * 2 * nx, 2 * nx, nx, 1, sm.T2, Wj, nb, dl, dr, nx, false);
    // L_{j+1}[c, (e x)] = sum_{(b s)} conj(B_j[(b s), c]) T2[(b s), (e x)]
    wgemm<NT>(sm, nc, dr * nx, 2 * nb, Bj, 1, nc, true, sm.T2, dr * nx, 1, false, sm.E, dr * nx, 1);
    gcopy<NT>(env_ptr(c, slot, j + 1), sm.E, nc * dr * nx);
    __syncthreads();
  }
  // ---- right environments of the guess (mirrored env updates with B given)
  for (int j = n - 1; first == 0 && j >= 1; --j) {
    const float2* Wj = chunk_W<NT>(j, L, nsub, BK, G1, sm, c.dmax);
    const int dl = sm.iv[0], dr = sm.iv[1];
    const float2* A = site_ptr(c, kb, slot, j);
    const int al = at[j], ar = at[j + 1];
    const float2* Bj = site_ptr(c, bb, slot, j);
    const int bl = bt[j], br = bt[j + 1];
    const int ldq = 2 * br;
    for (int idx = threadIdx.x; idx < bl * 2 * br; idx += NT) {  // Q'[(c s), b] = B[b][s][c]
      const int x = idx % br, s = (idx / br) & 1, bq = idx / (2 * br);
      sm.R[(x * 2 + s) + (size_t)bq * ldq] = Bj[idx];
    }
    // T1[(c e), (a t)] = sum_x E[(c e), x] A[(a t), x]
    wgemm<NT>(sm, br * dr, 2 * al, ar, sm.E, ar, 1, false, A, 1, ar, false, sm.T, 2 * al, 1);
    // T2[c][s][d][a] from T1[c][e][a][t]: fibre (c, a), incoming MPO index e, outgoing d
    mix_big<NT>(sm.T, dr * 2 * al, 2 * al, 1, 2, sm.T2, Wj, br, dr, dl, al, true);
    // R_j[b, (d a)] = sum_{(c s)} conj(Q'[(c s), b]) T2[(c s), (d a)]
    wgemm<NT>(sm, bl, dl * al, 2 * br, sm.R, ldq, 1, true, sm.T2, dl * al, 1, false, sm.E, dl * al,
                  1);
    gcopy<NT>(env_ptr(c, slot, j), sm.E, bl * dl * al);
    __syncthreads();
  }
  PHASE_MARK(6);
  // ---- one-site sweeps
  for (int sw = 0; sw < c.sweeps; ++sw) {
    // reduced-precision contractions, then the last sweep in FP32 as refinement (its f is
    // the reported fidelity)
    sm.use_tc = TC && (sw < c.sweeps - 1);
    if (threadIdx.x == 0) sm.E[0] = make_float2(1.f, 0.f);
    __syncthreads();
    if (((sw + first) & 1) == 0) {  // left to right
      for (int j = 0; j < n; ++j) {
        const float2* Wj = chunk_W<NT>(j, L, nsub, BK, G1, sm, c.dmax);
        const int dl = sm.iv[0], dr = sm.iv[1];
        const int nb = bt[j], nc = bt[j + 1], na = at[j], nx = at[j + 1];
        const float2* A = site_ptr(c, kb, slot, j);
        const float2* Rn = sm.R;
        if (j < n - 1) Rn = env_ptr(c, slot, j + 1);
        else if (threadIdx.x == 0) sm.R[0] = make_float2(1.f, 0.f);
        __syncthreads();
        wgemm<NT>(sm, nb * dl, 2 * nx, na, sm.E, na, 1, false, A, 2 * nx, 1, false, sm.T, 2 * nx, 1);
        mix_big<NT>(sm.T, dl * 2 * nx, 2 * nx, nx, 1, sm.T2, Wj, nb, dl, dr, nx, false);
        const int m = 2 * nb;
        wgemm<NT>(sm, m, nc, dr * nx, sm.T2, dr * nx, 1, false, Rn, 1, dr * nx, false, sm.F, 1, m);
        PHASE_MARK(7);
        float2* dst = site_ptr(c, bb, slot, j);
        if (j < n - 1) {
          const int r = sweep_qr<NT>(sm, m, nc);
          PHASE_MARK(8);
          for (int idx = threadIdx.x; idx < m * r; idx += NT) {
            const int row = idx / r, k2 = idx % r;
            dst[idx] = sm.R[row + (size_t)k2 * m];
          }
          wgemm<NT>(sm, r, dr * nx, m, sm.R, m, 1, true, sm.T2, dr * nx, 1, false, sm.E, dr * nx, 1);
          gcopy<NT>(env_ptr(c, slot, j + 1), sm.E, r * dr * nx);
          __syncthreads();
          if (threadIdx.x == 0) bt[j + 1] = r;
          __syncthreads();
          PHASE_MARK(9);
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
        const float2* Wj = chunk_W<NT>(j, L, nsub, BK, G1, sm, c.dmax);
        const int dl = sm.iv[0], dr = sm.iv[1];
        const int nb = bt[j + 1], nc = bt[j], na = at[j + 1], nx = at[j];
        const float2* A = site_ptr(c, kb, slot, j);
        const float2* Ln = sm.R;
        if (j > 0) Ln = env_ptr(c, slot, j);
        else if (threadIdx.x == 0) sm.R[0] = make_float2(1.f, 0.f);
        __syncthreads();
        // T1[(c e), (a t)] = sum_x E[(c e), x] A[(a t), x]
        wgemm<NT>(sm, nb * dr, 2 * nx, na, sm.E, na, 1, false, A, 1, na, false, sm.T, 2 * nx, 1);
        mix_big<NT>(sm.T, dr * 2 * nx, 2 * nx, 1, 2, sm.T2, Wj, nb, dr, dl, nx, true);
        const int m = 2 * nb;
        // F'[(c s), b] = sum_{(d a)} T2[(c s), (d a)] L[b, (d a)]
        wgemm<NT>(sm, m, nc, dl * nx, sm.T2, dl * nx, 1, false, Ln, 1, dl * nx, false, sm.F, 1, m);
        PHASE_MARK(7);
        float2* dst = site_ptr(c, bb, slot, j);
        if (j > 0) {
          const int r = sweep_qr<NT>(sm, m, nc);
          PHASE_MARK(8);
          for (int idx = threadIdx.x; idx < r * 2 * nb; idx += NT) {
            const int cc = idx % nb, s = (idx / nb) & 1, k2 = idx / (2 * nb);
            dst[idx] = sm.R[(cc * 2 + s) + (size_t)k2 * m];
          }
          wgemm<NT>(sm, r, dl * nx, m, sm.R, m, 1, true, sm.T2, dl * nx, 1, false, sm.E, dl * nx, 1);
          gcopy<NT>(env_ptr(c, slot, j), sm.E, r * dl * nx);
          __syncthreads();
          if (threadIdx.x == 0) bt[j] = r;
          __syncthreads();
          PHASE_MARK(9);
        } else {
          double s2 = 0.0;
          for (int i = threadIdx.x; i < m; i += NT) s2 += cabs2d(sm.F[i]);
          s2 = block_sum<NT>(s2, sm.red);
          const float inv = (float)(1.0 / sqrt(s2));
          for (int idx = threadIdx.x; idx < m; idx += NT) {
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
  if (TC) {
    if (threadIdx.x == 0 && *sm.tc.err) atomicOr(c.status, 1 << DCS_ERR_TIMEOUT);
    tc_teardown(sm.tc);
  }
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


}  // namespace dcs
