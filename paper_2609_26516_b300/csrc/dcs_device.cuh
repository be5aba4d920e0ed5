// Device building blocks of libdcs (sm_103a): complex arithmetic, the counter-based
// outcome sampler, CTA-level linear algebra on shared-memory tiles (Householder QR,
// one-sided Jacobi SVD) and the four contractions of a site update.
//
// Every routine here is executed by all NT threads of a CTA and ends with a __syncthreads()
// unless stated otherwise.  Matrices in shared memory are column-major with a leading
// dimension `ld` unless stated otherwise; complex numbers are float2 (x = re, y = im).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace dcs {

// ----------------------------------------------------------------------------- complex
__device__ __forceinline__ float2 cz() { return make_float2(0.f, 0.f); }
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float cabs2(float2 a) { return a.x * a.x + a.y * a.y; }
// |a|^2 with the squares taken in FP64 (no FP32 underflow for tiny entries)
__device__ __forceinline__ double cabs2d(float2 a) {
  return (double)a.x * (double)a.x + (double)a.y * (double)a.y;
}
// acc += a * b
__device__ __forceinline__ void cfma(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}
// acc += conj(a) * b
__device__ __forceinline__ void cfmac(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(-a.y, b.x, acc.y);
}

// ----------------------------------------------------------------------------- sampler
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): multipliers 0xD2511F53, 0xCD9E8D57,
// Weyl increments 0x9E3779B9, 0xBB67AE85.  Counter (ordinal, 0, shot lo, shot hi), key
// (seed lo, seed hi); the uniform is ((w0 >> 5) * 2^26 + (w1 >> 6)) * 2^-53.
// The two words that make the uniform: hi27 = w0 >> 5, lo26 = w1 >> 6.
__device__ __forceinline__ void philox_words(uint64_t seed, uint64_t shot, uint64_t ordinal,
                                             uint32_t& hi27, uint32_t& lo26) {
  uint32_t c0 = (uint32_t)ordinal, c1 = 0u, c2 = (uint32_t)shot, c3 = (uint32_t)(shot >> 32);
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  hi27 = c0 >> 5;
  lo26 = c1 >> 6;
}
__device__ __forceinline__ double philox_uniform(uint64_t seed, uint64_t shot, uint64_t ordinal) {
  uint32_t hi, lo;
  philox_words(seed, shot, ordinal, hi, lo);
  return (double)((uint64_t)hi * 67108864ull + lo) * (1.0 / 9007199254740992.0);
}

// ----------------------------------------------------------------------------- reductions
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (NT > 32) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    v = 0.0;
#pragma unroll
    for (int i = 0; i < NT / 32; ++i) v += red[i];
  }
  __syncthreads();
  return v;
}

template <int NT>
__device__ __forceinline__ float block_sumf(float v, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (NT > 32) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    v = 0.f;
#pragma unroll
    for (int i = 0; i < NT / 32; ++i) v += red[i];
  }
  __syncthreads();
  return v;
}

// ----------------------------------------------------------------------------- QR
// Householder QR of X (m x n, column-major, ld >= m) in place: Q (m x r, column-major, ldq)
// is formed explicitly (r = min(m, n)), and if R != nullptr the factor R (r x n, row-major,
// ldr) is written.  Reflector k is H_k = I - 2 u_k u_k^H with the unit vector
// u_k = (x - alpha_k e_1) / ||x - alpha_k e_1|| stored in X[k:, k], where x is the current
// column below the diagonal and alpha_k = -(x_0/|x_0|) ||x||, so H_k x = alpha_k e_1.
// The reflector is normalised explicitly, so H_k stays unitary to FP32 rounding whatever
// the column's magnitude; a column whose FP32 squared norm is below 1e-30 (a column of
// rounding noise, where FP32 squares can underflow) is normalised from FP64 squares.
// Scratch: tau[r] (2 or 0), alpha[r], red[NT/32] (double).
// Householder reflectors of columns k0 .. k1-1 of X (m rows, ld), each applied to the
// columns up to napply-1: the column loop of cta_qr (and of its blocked form, one panel at a
// time).  Reflector k is left in X[k:, k] (unit vector), tau[k] = 2 (0: H_k = I), alpha[k]
// the new diagonal entry.
template <int NT>
__device__ void house_columns(float2* X, int m, int ld, int k0, int k1, int napply, float* tau,
                              float2* alpha, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = NT / 32;
  for (int k = k0; k < k1; ++k) {
    // FP32 norm; a column whose squared norm is below 1e-30 (where FP32 squares of its
    // entries may underflow) is redone from FP64 squares
    float s32 = 0.f;
    for (int i = k + threadIdx.x; i < m; i += NT) s32 += cabs2(X[i + k * ld]);
    s32 = block_sumf<NT>(s32, reinterpret_cast<float*>(red));
    const float2 x0 = X[k + k * ld];
    bool skip;
    if (s32 > 1e-30f) {
      const float nrm = sqrtf(s32);
      // |x_0| without underflow: alpha = -(x_0/|x_0|) nrm must have modulus nrm exactly
      const float a0 = hypotf(x0.x, x0.y);
      const float vn = sqrtf(2.f * nrm * (nrm + a0));  // ||x - alpha e_1||
      const float inv = 1.f / vn;
      float ar, ai;
      if (a0 > 0.f) {
        ar = -x0.x / a0 * nrm;
        ai = -x0.y / a0 * nrm;
      } else {
        ar = -nrm;
        ai = 0.f;
      }
      __syncthreads();
      for (int i = k + threadIdx.x; i < m; i += NT) {
        float2 v = X[i + k * ld];
        if (i == k) {
          v.x -= ar;
          v.y -= ai;
        }
        X[i + k * ld] = make_float2(v.x * inv, v.y * inv);
      }
      if (threadIdx.x == 0) {
        tau[k] = 2.f;
        alpha[k] = make_float2(ar, ai);
      }
      skip = false;
    } else {
      double s = 0.0;
      for (int i = k + threadIdx.x; i < m; i += NT) s += cabs2d(X[i + k * ld]);
      s = block_sum<NT>(s, red);
      const double nrm = sqrt(s);
      const double a0 = sqrt(cabs2d(x0));
      // v = x - alpha e_1, ||v||^2 = 2 nrm (nrm + |x_0|); u = v / ||v||
      const double vn = sqrt(2.0 * nrm * (nrm + a0));
      skip = !(vn > 0.0);
      __syncthreads();
      if (!skip) {
        double ar, ai;
        if (a0 > 0.0) {
          ar = -(double)x0.x / a0 * nrm;
          ai = -(double)x0.y / a0 * nrm;
        } else {
          ar = -nrm;
          ai = 0.0;
        }
        for (int i = k + threadIdx.x; i < m; i += NT) {
          const float2 xi = X[i + k * ld];
          double vr = xi.x, vi = xi.y;
          if (i == k) {
            vr -= ar;
            vi -= ai;
          }
          X[i + k * ld] = make_float2((float)(vr / vn), (float)(vi / vn));
        }
        if (threadIdx.x == 0) {
          tau[k] = 2.f;
          alpha[k] = make_float2((float)ar, (float)ai);
        }
      } else if (threadIdx.x == 0) {
        tau[k] = 0.f;
        alpha[k] = cz();
      }
    }
    __syncthreads();
    if (!skip) {
      // rows in chunks of 32 HC per warp, each chunk's loads issued together (X may sit in
      // global memory, where one dependent load per row would serialise the latencies); the
      // sums run in row order as a plain loop would
      constexpr int HC = 8;
      for (int j = k + 1 + warp; j < napply; j += NW) {
        float2 d = cz();
        for (int i0 = k + lane; i0 < m; i0 += 32 * HC) {
          float2 u[HC], x[HC];
#pragma unroll
          for (int t = 0; t < HC; ++t) {
            const int i = i0 + 32 * t;
            u[t] = i < m ? X[i + k * ld] : cz();
            x[t] = i < m ? X[i + j * ld] : cz();
          }
#pragma unroll
          for (int t = 0; t < HC; ++t) cfmac(d, u[t], x[t]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          d.x += __shfl_xor_sync(0xffffffffu, d.x, o);
          d.y += __shfl_xor_sync(0xffffffffu, d.y, o);
        }
        d = cscale(d, 2.f);
        for (int i0 = k + lane; i0 < m; i0 += 32 * HC) {
          float2 u[HC], x[HC];
#pragma unroll
          for (int t = 0; t < HC; ++t) {
            const int i = i0 + 32 * t;
            u[t] = i < m ? X[i + k * ld] : cz();
            x[t] = i < m ? X[i + j * ld] : cz();
          }
#pragma unroll
          for (int t = 0; t < HC; ++t) {
            const int i = i0 + 32 * t;
            float2 a = x[t];
            a.x -= u[t].x * d.x - u[t].y * d.y;
            a.y -= u[t].x * d.y + u[t].y * d.x;
            if (i < m) X[i + j * ld] = a;
          }
        }
      }
    }
    __syncthreads();
  }
}

template <int NT>
__device__ int cta_qr(float2* X, int m, int n, int ld, float2* Q, int ldq, float2* R, int ldr,
                      float* tau, float2* alpha, double* red) {
  const int r = m < n ? m : n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = NT / 32;
  house_columns<NT>(X, m, ld, 0, r, n, tau, alpha, red);
  if (R != nullptr) {
    for (int idx = threadIdx.x; idx < r * n; idx += NT) {
      const int i = idx / n, j = idx % n;
      float2 v;
      if (j < i) v = cz();
      else if (j == i) v = tau[i] != 0.f ? alpha[i] : X[i + i * ld];
      else v = X[i + j * ld];
      R[i * ldr + j] = v;
    }
  }
  // Q = H_0 ... H_{r-1} [I_r; 0]
  for (int idx = threadIdx.x; idx < m * r; idx += NT) {
    const int i = idx % m, j = idx / m;
    Q[i + j * ldq] = make_float2(i == j ? 1.f : 0.f, 0.f);
  }
  __syncthreads();
  for (int k = r - 1; k >= 0; --k) {
    if (tau[k] != 0.f) {
      for (int j = k + warp; j < r; j += NW) {
        float2 d = cz();
        for (int i = k + lane; i < m; i += 32) cfmac(d, X[i + k * ld], Q[i + j * ldq]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          d.x += __shfl_xor_sync(0xffffffffu, d.x, o);
          d.y += __shfl_xor_sync(0xffffffffu, d.y, o);
        }
        d = cscale(d, 2.f);
        for (int i = k + lane; i < m; i += 32) {
          float2 v = X[i + k * ld];
          float2 a = Q[i + j * ldq];
          a.x -= v.x * d.x - v.y * d.y;
          a.y -= v.x * d.y + v.y * d.x;
          Q[i + j * ldq] = a;
        }
      }
    }
    __syncthreads();
  }
  return r;
}

// ----------------------------------------------------------------------------- warp QR
// Bond dimensions <= 4: the (m x n) matrix of a centre move (m <= 8 rows, n <= 4 columns)
// lives in one warp's registers, one complex entry per lane at lane = col * 8 + row and
// zero outside the matrix; a column sum is a butterfly over the three row bits.
constexpr unsigned FULL_MASK = 0xffffffffu;

__device__ __forceinline__ float2 shfl2(float2 v, int src) {
  return make_float2(__shfl_sync(FULL_MASK, v.x, src), __shfl_sync(FULL_MASK, v.y, src));
}
__device__ __forceinline__ float colsum8(float v) {
  v += __shfl_xor_sync(FULL_MASK, v, 1);
  v += __shfl_xor_sync(FULL_MASK, v, 2);
  v += __shfl_xor_sync(FULL_MASK, v, 4);
  return v;
}
__device__ __forceinline__ double colsum8d(double v) {
  v += __shfl_xor_sync(FULL_MASK, v, 1);
  v += __shfl_xor_sync(FULL_MASK, v, 2);
  v += __shfl_xor_sync(FULL_MASK, v, 4);
  return v;
}
__device__ __forceinline__ float2 colsum8c(float2 v) {
  return make_float2(colsum8(v.x), colsum8(v.y));
}

// Householder QR of the warp matrix x (m x n, m <= 8, n <= 4): the same reflectors as
// cta_qr (unit vectors u_k = (x - alpha_k e_k) / ||x - alpha_k e_k||, alpha_k of modulus
// ||x|| and phase opposite to x_k; FP32 norms, redone in FP64 below 1e-30; a zero column
// gets H_k = I).  On return x holds R (r x n, upper triangular, rows >= r zero) and q holds
// the explicit Q = H_0 ... H_{r-1} [I_r; 0] (m x r), r = min(m, n), both in the warp layout.
// Every lane of the warp must call it with the same m and n.
__device__ __forceinline__ int warp_qr8x4(float2& x, int m, int n, float2& q) {
  const int lane = threadIdx.x & 31, row = lane & 7, col = lane >> 3;
  const int r = m < n ? m : n;
  float2 U = cz();  // reflector `col` at this lane's row
  for (int k = 0; k < r; ++k) {
    const bool in_k = col == k && row >= k && row < m;
    const float s32 = __shfl_sync(FULL_MASK, colsum8(in_k ? cabs2(x) : 0.f), k * 8);
    const float2 x0 = shfl2(x, k * 8 + k);
    const float2 xk = shfl2(x, k * 8 + row);  // X[row][k]
    float2 u = cz(), alpha = cz();
    bool skip = false;
    if (s32 > 1e-30f) {
      const float nrm = sqrtf(s32);
      // |x_0|, exact for a real or imaginary x_0 (then x_0 / |x_0| is exactly +-1 or +-i and
      // alpha has modulus nrm exactly); otherwise a plain square root unless the squares
      // could underflow
      const float ax = fabsf(x0.x), ay = fabsf(x0.y);
      const float a0 = ay == 0.f ? ax
                       : ax == 0.f ? ay
                       : (fmaxf(ax, ay) > 1e-18f ? sqrtf(fmaf(x0.x, x0.x, x0.y * x0.y))
                                                 : hypotf(x0.x, x0.y));
      const float inv = 1.f / sqrtf(2.f * nrm * (nrm + a0));
      alpha = a0 > 0.f ? make_float2(-x0.x / a0 * nrm, -x0.y / a0 * nrm) : make_float2(-nrm, 0.f);
      if (row >= k && row < m) {
        u = xk;
        if (row == k) u = csub(u, alpha);
        u = cscale(u, inv);
      }
    } else if (!__any_sync(FULL_MASK, in_k && (x.x != 0.f || x.y != 0.f))) {
      skip = true;  // an exactly zero column (common after a collapse): H_k = I, no FP64
    } else {
      const double sd = __shfl_sync(FULL_MASK, colsum8d(in_k ? cabs2d(x) : 0.0), k * 8);
      const double nrm = sqrt(sd);
      const double a0 = sqrt(cabs2d(x0));
      const double vn = sqrt(2.0 * nrm * (nrm + a0));
      skip = !(vn > 0.0);
      if (!skip) {
        double ar = -nrm, ai = 0.0;
        if (a0 > 0.0) {
          ar = -(double)x0.x / a0 * nrm;
          ai = -(double)x0.y / a0 * nrm;
        }
        alpha = make_float2((float)ar, (float)ai);
        if (row >= k && row < m) {
          double vr = xk.x, vi = xk.y;
          if (row == k) {
            vr -= ar;
            vi -= ai;
          }
          u = make_float2((float)(vr / vn), (float)(vi / vn));
        }
      }
    }
    if (!skip) {
      float2 d = cz();
      if (col > k && col < n) cfmac(d, u, x);
      d = colsum8c(d);
      if (col > k && col < n) {
        x.x -= 2.f * (u.x * d.x - u.y * d.y);
        x.y -= 2.f * (u.x * d.y + u.y * d.x);
      }
      if (col == k && row >= k) x = row == k ? alpha : cz();
    }
    if (col == k) U = u;
  }
  float2 qv = make_float2(row == col && col < r ? 1.f : 0.f, 0.f);
  for (int k = r - 1; k >= 0; --k) {
    const float2 uk = shfl2(U, k * 8 + row);
    float2 d = cz();
    if (col < r) cfmac(d, uk, qv);
    d = colsum8c(d);
    if (col < r) {
      qv.x -= 2.f * (uk.x * d.x - uk.y * d.y);
      qv.y -= 2.f * (uk.x * d.y + uk.y * d.x);
    }
  }
  q = qv;
  return r;
}

// ----------------------------------------------------------------------------- SVD
// Absolute rotation floor of the Jacobi SVDs: 2^-40 ||X||_F^2 (FP32 sum, block reduction).
template <int NT>
__device__ float jacobi_floor(const float2* X, int m, int n, int ld, double* red) {
  float s = 0.f;
  for (int j = 0; j < n; ++j)
    for (int i = threadIdx.x; i < m; i += NT) s += cabs2(X[i + (size_t)j * ld]);
  s = block_sumf<NT>(s, reinterpret_cast<float*>(red));
  return s * 9.09494702e-13f;
}

// One-sided (Hestenes) Jacobi SVD of X (m x n, column-major, ld): rotates pairs of columns
// until they are mutually orthogonal, X V = U Sigma, accumulating the unitary V (n x n,
// column-major, ldv; not accumulated when V is null).  Pairs follow the circle-method tournament so each round rotates
// disjoint pairs in parallel, one group of G lanes per pair.  A pair (i, j) with
// Gram [[a, g], [conj g, b]] is rotated when |g| > 2 sqrt(m) eps sqrt(a b):
// zeta = (b - a) / (2|g|), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), c = 1/sqrt(1+t^2),
// s = c t, x_i' = c x_i - s e^{-i phi} x_j, x_j' = s x_i + c e^{-i phi} x_j, g = |g| e^{i phi}.
// Afterwards sig2[j] = sigf[j] = ||x_j||^2 (FP32 sum) and perm[0..n) lists columns by
// decreasing norm (ties: lower index first).  Scratch: red[NT/32], flag (int).
template <int NT>
__device__ void svd_finish(const float2* X, int m, int n, int ld, double* sig2, float* sigf,
                           int* perm);

template <int NT>
__device__ int cta_jacobi_svd(float2* X, int m, int n, int ld, float2* V, int ldv,
                              double* sig2, float* sigf, int* perm, int* flag, double* red) {
  for (int idx = threadIdx.x; V != nullptr && idx < n * n; idx += NT) {
    const int i = idx % n, j = idx / n;
    V[i + j * ldv] = make_float2(i == j ? 1.f : 0.f, 0.f);
  }
  __syncthreads();
  const int N = (n + 1) & ~1;  // players, padded to even
  const int npairs = N / 2;
  int G = 32;
  while (G > 1 && (NT / G) < npairs) G >>= 1;
  const int ngroups = NT / G;
  const int grp = threadIdx.x / G, gl = threadIdx.x % G;
  // convergence: |g| <= 2 sqrt(m) eps32 sqrt(a b), the FP32 rounding level of the computed
  // inner product (the column-orthogonality test of one-sided Jacobi codes), or |g| below
  // 2^-40 of the squared Frobenius norm: pairs of columns at the FP32 noise level, which
  // rounding otherwise keeps rotating up to the sweep cap.  The floor sits two orders of
  // magnitude under the truncation tolerances used (1e-10 of the weight)
  const float thr = 2.f * sqrtf((float)m) * 5.96e-8f;
  // (small matrices converge in a few sweeps without the floor; it is not worth its pass)
  const float floor_g = n > 16 ? jacobi_floor<NT>(X, m, n, ld, red) : 0.f;
  int sweep = 0;
  for (; sweep < 30 && N >= 2; ++sweep) {
    if (threadIdx.x == 0) *flag = 0;
    __syncthreads();
    for (int rnd = 0; rnd < N - 1; ++rnd) {
      for (int pbase = 0; pbase < npairs; pbase += ngroups) {
        const int p = pbase + grp;
        int ci = -1, cj = -1;
        if (p < npairs) {
          if (p == 0) {
            ci = rnd;
            cj = N - 1;
          } else {
            ci = (rnd + p) % (N - 1);
            cj = (rnd - p + (N - 1)) % (N - 1);
          }
          if (ci > cj) {
            const int t = ci;
            ci = cj;
            cj = t;
          }
        }
        const bool valid = (p < npairs) && (cj < n);
        float a = 0.f, b = 0.f;
        float2 g = cz();
        if (valid) {
          for (int i = gl; i < m; i += G) {
            const float2 xi = X[i + ci * ld], xj = X[i + cj * ld];
            a += cabs2(xi);
            b += cabs2(xj);
            cfmac(g, xi, xj);
          }
        }
        // reduce within the group of G lanes (all lanes take part in the shuffles)
        for (int o = G / 2; o > 0; o >>= 1) {
          a += __shfl_xor_sync(0xffffffffu, a, o);
          b += __shfl_xor_sync(0xffffffffu, b, o);
          g.x += __shfl_xor_sync(0xffffffffu, g.x, o);
          g.y += __shfl_xor_sync(0xffffffffu, g.y, o);
        }
        const float ag = hypotf(g.x, g.y);  // the phase g/|g| must have modulus 1
        if (valid && ag > thr * sqrtf(a * b) && ag > floor_g && ag > 0.f) {
          const float zeta = (b - a) / (2.f * ag);
          const float t = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
          const float c = rsqrtf(1.f + t * t);
          const float s = c * t;
          const float2 ph = make_float2(g.x / ag, -g.y / ag);  // e^{-i phi}
          for (int i = gl; i < m; i += G) {
            const float2 xi = X[i + ci * ld];
            const float2 xj = cmul(ph, X[i + cj * ld]);
            X[i + ci * ld] = make_float2(c * xi.x - s * xj.x, c * xi.y - s * xj.y);
            X[i + cj * ld] = make_float2(s * xi.x + c * xj.x, s * xi.y + c * xj.y);
          }
          for (int i = gl; V != nullptr && i < n; i += G) {
            const float2 vi = V[i + ci * ldv];
            const float2 vj = cmul(ph, V[i + cj * ldv]);
            V[i + ci * ldv] = make_float2(c * vi.x - s * vj.x, c * vi.y - s * vj.y);
            V[i + cj * ldv] = make_float2(s * vi.x + c * vj.x, s * vi.y + c * vj.y);
          }
          if (gl == 0) *flag = 1;
        }
      }
      __syncthreads();
    }
    if (*flag == 0) break;
    __syncthreads();
  }
  svd_finish<NT>(X, m, n, ld, sig2, sigf, perm);
  return sweep;
}

// Column norms of the rotated X (FP32 sums, also handed out in FP64) and their ordering.
template <int NT>
__device__ void svd_finish(const float2* X, int m, int n, int ld, double* sig2, float* sigf,
                           int* perm) {
  for (int j = threadIdx.x; j < n; j += NT) {
    float s = 0.f;
    for (int i = 0; i < m; ++i) s += cabs2(X[i + j * ld]);
    sigf[j] = s;
    sig2[j] = (double)s;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += NT) {
    int rank = 0;
    const float sj = sigf[j];
    for (int i = 0; i < n; ++i) {
      const float si = sigf[i];
      rank += (si > sj) || (si == sj && i < j);
    }
    perm[rank] = j;
  }
  __syncthreads();
}

// One pair rotation of the one-sided Jacobi method on two staged columns ci, cj of length
// cs, whose first m entries are X and the rest V, by one warp (same rotation and threshold
// as cta_jacobi_svd).  Returns whether it rotated.
__device__ __forceinline__ bool warp_jacobi_pair(float2* ci, float2* cj, int m, int cs, float thr,
                                                 float floor_g) {
  const int lane = threadIdx.x & 31;
  float a = 0.f, b = 0.f;
  float2 g = cz();
  for (int i = lane; i < m; i += 32) {
    const float2 xi = ci[i], xj = cj[i];
    a += cabs2(xi);
    b += cabs2(xj);
    cfmac(g, xi, xj);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(FULL_MASK, a, o);
    b += __shfl_xor_sync(FULL_MASK, b, o);
    g.x += __shfl_xor_sync(FULL_MASK, g.x, o);
    g.y += __shfl_xor_sync(FULL_MASK, g.y, o);
  }
  const float ag = hypotf(g.x, g.y);
  if (!(ag > thr * sqrtf(a * b) && ag > floor_g && ag > 0.f)) return false;
  const float zeta = (b - a) / (2.f * ag);
  const float t = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
  const float c = rsqrtf(1.f + t * t);
  const float s = c * t;
  const float2 ph = make_float2(g.x / ag, -g.y / ag);  // e^{-i phi}
  for (int i = lane; i < cs; i += 32) {
    const float2 xi = ci[i];
    const float2 xj = cmul(ph, cj[i]);
    ci[i] = make_float2(c * xi.x - s * xj.x, c * xi.y - s * xj.y);
    cj[i] = make_float2(s * xi.x + c * xj.x, s * xi.y + c * xj.y);
  }
  return true;
}

// Columns [c0, c0 + w) of X (m rows) and V (n rows; n = 0 without V) to or from the staging
// area, one staged column of m + n entries each.
template <int NT>
__device__ __forceinline__ void stage_cols(float2* S, float2* X, int m, int ld, float2* V,
                                           int n, int ldv, int c0, int w, bool in) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cs = m + n;
  for (int col = warp; col < w; col += NT / 32) {
    float2* sc = S + (size_t)col * cs;
    float2* xc = X + (size_t)(c0 + col) * ld;
    float2* vc = n > 0 ? V + (size_t)(c0 + col) * ldv : nullptr;
    for (int i = lane; i < m; i += 32) {
      if (in) sc[i] = xc[i];
      else xc[i] = sc[i];
    }
    for (int i = lane; i < n; i += 32) {
      if (in) sc[m + i] = vc[i];
      else vc[i] = sc[m + i];
    }
  }
}

// Blocked one-sided Jacobi SVD for matrices too large for shared memory, with the rotations,
// threshold and outputs of cta_jacobi_svd.  The n columns are cut into blocks of w.  Each
// sweep rotates every pair of columns once, with both columns staged in shared memory
// together with the matching columns of V.  Block I stays staged while the blocks J > I pass
// through.  The pairs inside I come first (circle method on its columns), then for each J
// its cross pairs in w rounds of disjoint pairs (a, (a + r) mod w).  Per sweep X and V
// cross HBM about n / w times instead of about n times.  Without V (null) only X is staged,
// which doubles w.
template <int NT>
__device__ int cta_jacobi_svd_staged(float2* X, int m, int n, int ld, float2* V, int ldv,
                                      double* sig2, float* sigf, int* perm, int* flag,
                                      double* red, float2* stage, size_t stage_elems) {
  const int nv = V != nullptr ? n : 0;  // V rows staged with each column (none without V)
  const int cs = m + nv;
  int w = (int)(stage_elems / (2 * (size_t)cs));
  if (w > n) w = n;
  if (w < 2) return cta_jacobi_svd<NT>(X, m, n, ld, V, ldv, sig2, sigf, perm, flag, red);
  constexpr int NW = NT / 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int idx = threadIdx.x; V != nullptr && idx < n * n; idx += NT) {
    const int i = idx % n, j = idx / n;
    V[i + (size_t)j * ldv] = make_float2(i == j ? 1.f : 0.f, 0.f);
  }
  __syncthreads();
  const int nb = (n + w - 1) / w;
  const float thr = 2.f * sqrtf((float)m) * 5.96e-8f;  // as cta_jacobi_svd
  const float floor_g = jacobi_floor<NT>(X, m, n, ld, red);
  float2* SI = stage;
  float2* SJ = stage + (size_t)w * cs;
  if (threadIdx.x == 0) *flag = 0;
  int sweep = 0;
  for (; sweep < 30; ++sweep) {
    int rotated = 0;
    for (int I = 0; I < nb; ++I) {
      const int i0 = I * w, wi = (n - i0) < w ? (n - i0) : w;
      __syncthreads();
      stage_cols<NT>(SI, X, m, ld, V, nv, ldv, i0, wi, true);
      __syncthreads();
      // pairs inside block I: circle method
      const int N = (wi + 1) & ~1;
      for (int rnd = 0; rnd < N - 1; ++rnd) {
        for (int p = warp; p < N / 2; p += NW) {
          int ci, cj;
          if (p == 0) {
            ci = rnd;
            cj = N - 1;
          } else {
            ci = (rnd + p) % (N - 1);
            cj = (rnd - p + (N - 1)) % (N - 1);
          }
          if (ci < wi && cj < wi && ci != cj)
            rotated |= warp_jacobi_pair(SI + (size_t)ci * cs, SI + (size_t)cj * cs, m, cs, thr, floor_g);
        }
        __syncthreads();
      }
      for (int J = I + 1; J < nb; ++J) {
        const int j0 = J * w, wj = (n - j0) < w ? (n - j0) : w;
        stage_cols<NT>(SJ, X, m, ld, V, nv, ldv, j0, wj, true);
        __syncthreads();
        for (int r = 0; r < w; ++r) {
          for (int a = warp; a < wi; a += NW) {
            const int bcol = (a + r) % w;
            if (bcol < wj)
              rotated |= warp_jacobi_pair(SI + (size_t)a * cs, SJ + (size_t)bcol * cs, m, cs, thr, floor_g);
          }
          __syncthreads();
        }
        stage_cols<NT>(SJ, X, m, ld, V, nv, ldv, j0, wj, false);
        __syncthreads();
      }
      stage_cols<NT>(SI, X, m, ld, V, nv, ldv, i0, wi, false);
    }
    if (lane == 0 && rotated) *flag = 1;
    __syncthreads();
    const int any = *flag;
    __syncthreads();
    if (threadIdx.x == 0) *flag = 0;
    if (!any) break;
  }
  __syncthreads();
  svd_finish<NT>(X, m, n, ld, sig2, sigf, perm);
  return sweep + 1;
}

// The rotation of one pair (x_i held by this warp in registers, x_j given in registers too),
// as warp_jacobi_pair, with the squared norms a = ||x_i||^2, b = ||x_j||^2 kept from the
// columns' last change instead of re-read: the same threshold, angle and phase; the new
// norms are summed while the rotated columns are formed.  Returns whether it rotated.
template <int MR>
__device__ __forceinline__ bool reg_jacobi_pair(float2 (&xi)[MR], float2 (&xj)[MR], float& a,
                                                float& b, float thr, float floor_g) {
  float2 g = cz();
#pragma unroll
  for (int k = 0; k < MR; ++k) cfmac(g, xi[k], xj[k]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    g.x += __shfl_xor_sync(FULL_MASK, g.x, o);
    g.y += __shfl_xor_sync(FULL_MASK, g.y, o);
  }
  const float ag = hypotf(g.x, g.y);
  if (!(ag > thr * sqrtf(a * b) && ag > floor_g && ag > 0.f)) return false;
  const float zeta = (b - a) / (2.f * ag);
  const float t = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
  const float c = rsqrtf(1.f + t * t);
  const float s = c * t;
  const float2 ph = make_float2(g.x / ag, -g.y / ag);  // e^{-i phi}
  float na = 0.f, nb = 0.f;
#pragma unroll
  for (int k = 0; k < MR; ++k) {
    const float2 u = xi[k];
    const float2 v = cmul(ph, xj[k]);
    xi[k] = make_float2(c * u.x - s * v.x, c * u.y - s * v.y);
    xj[k] = make_float2(s * u.x + c * v.x, s * u.y + c * v.y);
    na += cabs2(xi[k]);
    nb += cabs2(xj[k]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    na += __shfl_xor_sync(FULL_MASK, na, o);
    nb += __shfl_xor_sync(FULL_MASK, nb, o);
  }
  a = na;
  b = nb;
  return true;
}

// cta_jacobi_svd_staged without V for m <= 32 MR rows, with less shared-memory traffic: the
// columns are taken in blocks I of CPW NW (CPW per warp).  The pairs inside I are rotated in
// shared memory (circle method, warp_jacobi_pair); then each warp holds its CPW columns of
// I in registers while the columns after I stream through the staging area in blocks J,
// round r pairing column a of I with column (a + r) mod R of J (R = max(|I|, |J|): disjoint
// pairs within a round), so a pair moves one column through shared memory instead of three
// reads and two writes.  Every pair of columns is still rotated once per sweep, with the
// rotation, threshold and stopping rule of cta_jacobi_svd_staged.
template <int NT, int MR, int CPW>
__device__ __noinline__ int cta_jacobi_svd_regs(float2* X, int m, int n, int ld, double* sig2,
                                                float* sigf, int* perm, int* flag, double* red,
                                                float2* stage, size_t stage_elems) {
  constexpr int NW = NT / 32;
  constexpr int W = CPW * NW;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // staged J columns (m complex each) and their squared norms behind them
  int wjcap = (int)((stage_elems * sizeof(float2)) / ((size_t)m * sizeof(float2) + sizeof(float)));
  if (wjcap > n) wjcap = n;
  float* bnorm = reinterpret_cast<float*>(stage + (size_t)wjcap * m);
  const float thr = 2.f * sqrtf((float)m) * 5.96e-8f;  // as cta_jacobi_svd
  const float floor_g = jacobi_floor<NT>(X, m, n, ld, red);
  if (threadIdx.x == 0) *flag = 0;
  int sweep = 0;
  for (; sweep < 30; ++sweep) {
    int rotated = 0;
    for (int i0 = 0; i0 < n; i0 += W) {
      const int wi = (n - i0) < W ? (n - i0) : W;
      __syncthreads();
      stage_cols<NT>(stage, X, m, ld, nullptr, 0, 0, i0, wi, true);
      __syncthreads();
      // pairs inside I: circle method in shared memory
      const int N = (wi + 1) & ~1;
      for (int rnd = 0; rnd < N - 1; ++rnd) {
        for (int p = warp; p < N / 2; p += NW) {
          int ci, cj;
          if (p == 0) {
            ci = rnd;
            cj = N - 1;
          } else {
            ci = (rnd + p) % (N - 1);
            cj = (rnd - p + (N - 1)) % (N - 1);
          }
          if (ci < wi && cj < wi && ci != cj)
            rotated |= warp_jacobi_pair(stage + (size_t)ci * m, stage + (size_t)cj * m, m, m, thr, floor_g);
        }
        __syncthreads();
      }
      // this warp's columns of I into registers, with their squared norms
      float2 xr[CPW][MR];
      float an[CPW];
#pragma unroll
      for (int c = 0; c < CPW; ++c) {
        const int col = warp + c * NW;
        float sacc = 0.f;
#pragma unroll
        for (int k = 0; k < MR; ++k) {
          const int row = lane + 32 * k;
          xr[c][k] = (col < wi && row < m) ? stage[(size_t)col * m + row] : cz();
          sacc += cabs2(xr[c][k]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sacc += __shfl_xor_sync(FULL_MASK, sacc, o);
        an[c] = sacc;
      }
      __syncthreads();  // the staging area now serves the J blocks
      for (int j0 = i0 + wi; j0 < n; j0 += wjcap) {
        const int wj = (n - j0) < wjcap ? (n - j0) : wjcap;
        stage_cols<NT>(stage, X, m, ld, nullptr, 0, 0, j0, wj, true);
        __syncthreads();
        for (int col = warp; col < wj; col += NW) {
          float sacc = 0.f;
          for (int row = lane; row < m; row += 32) sacc += cabs2(stage[(size_t)col * m + row]);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) sacc += __shfl_xor_sync(FULL_MASK, sacc, o);
          if (lane == 0) bnorm[col] = sacc;
        }
        __syncthreads();
        const int R = wi > wj ? wi : wj;
        for (int r = 0; r < R; ++r) {
#pragma unroll
          for (int c = 0; c < CPW; ++c) {
            const int a = warp + c * NW;
            const int bcol = (a + r) % R;
            if (a < wi && bcol < wj) {
              float2* sc = stage + (size_t)bcol * m;
              float2 xj[MR];
#pragma unroll
              for (int k = 0; k < MR; ++k) {
                const int row = lane + 32 * k;
                xj[k] = row < m ? sc[row] : cz();
              }
              float bb = bnorm[bcol];
              if (reg_jacobi_pair<MR>(xr[c], xj, an[c], bb, thr, floor_g)) {
                rotated = 1;
#pragma unroll
                for (int k = 0; k < MR; ++k) {
                  const int row = lane + 32 * k;
                  if (row < m) sc[row] = xj[k];
                }
                __syncwarp();
                if (lane == 0) bnorm[bcol] = bb;
              }
            }
          }
          __syncthreads();
        }
        stage_cols<NT>(stage, X, m, ld, nullptr, 0, 0, j0, wj, false);
        __syncthreads();
      }
      // this warp's columns of I back to X
#pragma unroll
      for (int c = 0; c < CPW; ++c) {
        const int col = warp + c * NW;
        if (col < wi) {
#pragma unroll
          for (int k = 0; k < MR; ++k) {
            const int row = lane + 32 * k;
            if (row < m) X[(size_t)(i0 + col) * ld + row] = xr[c][k];
          }
        }
      }
    }
    if (lane == 0 && rotated) *flag = 1;
    __syncthreads();
    const int any = *flag;
    __syncthreads();
    if (threadIdx.x == 0) *flag = 0;
    if (!any) break;
  }
  __syncthreads();
  svd_finish<NT>(X, m, n, ld, sig2, sigf, perm);
  return sweep + 1;
}

// ----------------------------------------------------------------------------- float-float
// Sums of squares to about FP64 accuracy on the FP32 pipe (an FP64 instruction costs a
// whole warp dozens of cycles on this part): a value is an unevaluated sum hi + lo, squares
// are split exactly with an FMA, additions use Knuth's TwoSum.  The _rn intrinsics keep
// the compiler from contracting the error terms.
struct ffloat {
  float hi, lo;
};
__device__ __forceinline__ ffloat ff_add(ffloat a, ffloat b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  const float t = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  const float hi = __fadd_rn(s, t);
  return {hi, __fsub_rn(t, __fsub_rn(hi, s))};
}
__device__ __forceinline__ ffloat ff_abs2(float2 x) {
  const float p = __fmul_rn(x.x, x.x), q = __fmul_rn(x.y, x.y);
  const ffloat a{p, fmaf(x.x, x.x, -p)}, b{q, fmaf(x.y, x.y, -q)};
  return ff_add(a, b);
}
__device__ __forceinline__ ffloat ff_warp_sum(ffloat a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const ffloat b{__shfl_xor_sync(FULL_MASK, a.hi, o), __shfl_xor_sync(FULL_MASK, a.lo, o)};
    a = ff_add(a, b);
  }
  return a;
}
__device__ __forceinline__ double ff_to_double(ffloat a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ ffloat ff_neg(ffloat a) { return {-a.hi, -a.lo}; }
// a / b to about 2^-44 relative (one correction step of the FP32 quotient)
__device__ __forceinline__ ffloat ff_div(ffloat a, ffloat b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const float ph = __fmul_rn(q1, b.hi);
  const float pl = fmaf(q1, b.hi, -ph);
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, ph), pl), __fsub_rn(a.lo, __fmul_rn(q1, b.lo)));
  const float q2 = __fdiv_rn(r, b.hi);
  const float hi = __fadd_rn(q1, q2);
  return {hi, __fsub_rn(q2, __fsub_rn(hi, q1))};
}
// sign of a - b: -1, 0, +1
__device__ __forceinline__ int ff_cmp(ffloat a, ffloat b) {
  const ffloat d = ff_add(a, ff_neg(b));
  return d.hi < 0.f ? -1 : (d.hi > 0.f ? 1 : (d.lo < 0.f ? -1 : (d.lo > 0.f ? 1 : 0)));
}
// The uniform u = hi27 2^-27 + lo26 2^-53 as a float-float, within 2^-48 of u.
__device__ __forceinline__ ffloat ff_uniform(uint32_t hi27, uint32_t lo26) {
  const float a = __fmul_rn((float)(hi27 >> 3), 5.9604644775390625e-08f);          // 2^-24
  const float b = __fmul_rn((float)(((hi27 & 7u) << 26) | lo26), 1.1102230246251565e-16f);  // 2^-53
  const float hi = __fadd_rn(a, b);
  return {hi, __fsub_rn(b, __fsub_rn(hi, a))};
}

// Warp version of trunc_rank for n <= 32 values, FP32: lane i takes the i-th largest value
// w_(i) = sigf[perm[i]]; returns k and sets kept = sum_{i<k} w_(i), disc = sum_{i>=k} w_(i).
__device__ __forceinline__ int warp_trunc_rank(const float* sigf, const int* perm, int n, int cap,
                                               double tol, float& kept, float& disc) {
  const int lane = threadIdx.x & 31;
  const float v = lane < n ? sigf[perm[lane]] : 0.f;
  float S = v;  // suffix sums S_i = sum_{j >= i} w_(j)
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float t = __shfl_down_sync(FULL_MASK, S, o);
    if (lane + o < 32) S += t;
  }
  const float tot = __shfl_sync(FULL_MASK, S, 0);
  const float lim = (float)tol * tot;
  const unsigned keep = __ballot_sync(FULL_MASK, lane >= 1 && lane < n && S > lim);
  int k = keep ? 32 - __clz(keep) : 1;
  if (k > cap) k = cap;
  if (k > n) k = n;
  if (k < 1) k = 1;
  disc = k < 32 ? __shfl_sync(FULL_MASK, S, k & 31) : 0.f;
  if (k >= n) disc = 0.f;
  float w = lane < k ? v : 0.f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(FULL_MASK, w, o);
  kept = w;
  return k;
}

// Smallest k >= 1 with sum_{i >= k} w_(i) <= tol * sum_i w_i, w_(i) the values in
// decreasing order (through perm), capped at cap and n.  Suffix sums are accumulated from
// the smallest value up.  Evaluated by one thread in FP64.
static __device__ __noinline__ int trunc_rank(const double* w, const int* perm, int n, int cap,
                                          double tol) {
  double total = 0.0;
  for (int i = 0; i < n; ++i) total += w[i];
  int k = 1;
  double s = 0.0;
  for (int i = n - 1; i >= 1; --i) {
    s += w[perm[i]];
    if (s > tol * total) {
      k = i + 1;
      break;
    }
  }
  if (k > cap) k = cap;
  if (k > n) k = n;
  if (k < 1) k = 1;
  return k;
}

}  // namespace dcs
