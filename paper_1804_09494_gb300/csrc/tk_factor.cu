// New factor F~_n = leading K_n left singular vectors of Z_(n) (Fig. 1, "SVD").
//
//   W = Z^T Z            Gram over the R_n compact rows (split over rows, FP64 reduction in fixed order)
//   W V = V Lambda       top-K eigenpairs in one CTA: Lanczos with full re-orthogonalisation,
//                        eigenvalues of the tridiagonal by multisection (Sturm counts), eigenvectors by
//                        inverse iteration + modified Gram-Schmidt; the FP32 context polishes the top-K
//                        subspace in FP64 (one subspace step + Rayleigh-Ritz)
//   U = Z V Sigma^-1     back-projection
//   U <- U R^-1 twice    CholeskyQR2 (Gram reductions, Cholesky and inverses in FP64)
//   signs                column's entry of largest magnitude (lowest slice id on a tie) made positive
//   F_n[row_map[r]] = U[r] (row_map: slice ids, or the context's popularity labels), other rows zero
#include <algorithm>
#include <type_traits>

#include "tk_common.cuh"

namespace {

// ------------------------------------------------------------------ Gram
// Thread (tx, ty) of a 16 x 16 grid owns rows ty + 16 i and columns tx + 16 j of
// a TM x TM output tile, so shared-memory reads are conflict free.
template <typename T, int TM>
__global__ void __launch_bounds__(256) k_gram(const T* __restrict__ Z, int R, int Khat, const int2* __restrict__ tiles,
                                              int ntiles, int rows_per_split, T* __restrict__ Wpart) {
  constexpr int RT = TM / 16;
  constexpr int BR = 16;
  __shared__ T As[BR][TM];
  __shared__ T Bs[BR][TM];
  const int t = blockIdx.x, sp = blockIdx.y;
  const int ti = tiles[t].x, tj = tiles[t].y;
  const int r0 = sp * rows_per_split, r1 = min(R, r0 + rows_per_split);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  // batch sums (acc) are folded into a compensated (Kahan) running sum (tot, cmp)
  T acc[RT][RT], tot[RT][RT], cmp[RT][RT];
#pragma unroll
  for (int i = 0; i < RT; ++i)
#pragma unroll
    for (int j = 0; j < RT; ++j) acc[i][j] = tot[i][j] = cmp[i][j] = T(0);
  for (int rb = r0; rb < r1; rb += BR) {
    for (int i = threadIdx.x; i < BR * TM; i += 256) {
      const int r = i / TM, cc = i - r * TM;
      const int row = rb + r, ca = ti * TM + cc, cb = tj * TM + cc;
      const bool rv = row < r1;
      As[r][cc] = (rv && ca < Khat) ? Z[(int64_t)row * Khat + ca] : T(0);
      Bs[r][cc] = (rv && cb < Khat) ? Z[(int64_t)row * Khat + cb] : T(0);
    }
    __syncthreads();
#pragma unroll 4
    for (int r = 0; r < BR; ++r) {
      T a[RT], b[RT];
#pragma unroll
      for (int i = 0; i < RT; ++i) a[i] = As[r][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < RT; ++j) b[j] = Bs[r][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < RT; ++i)
#pragma unroll
        for (int j = 0; j < RT; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < RT; ++i)
#pragma unroll
      for (int j = 0; j < RT; ++j) {
        const T y = acc[i][j] - cmp[i][j];
        const T t2 = tot[i][j] + y;
        cmp[i][j] = (t2 - tot[i][j]) - y;
        tot[i][j] = t2;
        acc[i][j] = T(0);
      }
  }
  T* out = Wpart + ((int64_t)sp * ntiles + t) * TM * TM;
#pragma unroll
  for (int i = 0; i < RT; ++i)
#pragma unroll
    for (int j = 0; j < RT; ++j) out[(ty + 16 * i) * TM + tx + 16 * j] = tot[i][j];
}

// W (FP64, both triangles) from the split partials: 8 lanes per entry, each
// summing every 8th split in order, combined by a fixed shuffle tree.
template <typename T>
__global__ void k_gram_reduce(const T* __restrict__ Wpart, int nsplit, int ntiles, int tpd, int TM, int Khat,
                              double* __restrict__ W) {
  const int64_t total = (int64_t)Khat * Khat;
  const int part = threadIdx.x & 7;
  const int64_t per_pass = ((int64_t)gridDim.x * blockDim.x) >> 3;
  for (int64_t base = 0; base < total; base += per_pass) {  // uniform trip count for every lane
    const int64_t idx0 = base + (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3);
    const bool live = idx0 < total;
    const int64_t idx = live ? idx0 : 0;
    int i = (int)(idx / Khat), j = (int)(idx - (int64_t)i * Khat);
    int ti = i / TM, tj = j / TM, ii = i - ti * TM, jj = j - tj * TM;
    if (ti > tj) {
      int x = ti; ti = tj; tj = x;
      x = ii; ii = jj; jj = x;
    }
    const int t = ti * tpd - ti * (ti - 1) / 2 + (tj - ti);
    double s = 0.0;
    if (live)
      for (int sp = part; sp < nsplit; sp += 8) s += (double)Wpart[((int64_t)sp * ntiles + t) * TM * TM + ii * TM + jj];
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    s += __shfl_xor_sync(0xffffffffu, s, 4);
    if (part == 0 && live) W[idx] = s;
  }
}

template <typename T>
struct EigArgs {
  const double* W;
  int n, K;
  T* gA;         // n x n (global) when A is not kept in shared memory
  T* gQ;         // n x n Lanczos basis (global) when not in shared memory
  int use_smem;
  int polish;
  double* X;     // n x K scratch (FP64)
  double* Y;     // n x K scratch (FP64)
  double* ab;    // 2n: Lanczos alpha, beta
  T* tri;        // K x 6n: pivoted LU of T - lambda I and the inverse-iteration vector
  double* Vout;  // n x K
  double* sigma; // K
  T* Vs;         // n x K: Vout[:,k] / sigma_k
  int* err;
  unsigned long long* clk;  // optional: clock64() at phase boundaries (profiling; NULL in normal use)
};

__device__ __forceinline__ uint32_t mix32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352dU;
  x ^= x >> 15;
  x *= 0x846ca68bU;
  x ^= x >> 16;
  return x;
}
// deterministic pseudo-random entries in [-0.5, 0.5) for start vectors
template <typename T>
__device__ __forceinline__ T hash_unit(uint32_t seed, uint32_t i) {
  return (T)(int)(mix32(seed * 0x9E3779B9u + i * 0x85EBCA6Bu + 0x165667B1u) >> 8) * (T)(1.0 / 16777216.0) - (T)0.5;
}

template <typename T>
__device__ __forceinline__ T warp_allsum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block sum (blockDim multiple of 32): warp sums, then warp 0 adds the 32
// partials; red needs 33 slots.  Two barriers; the same value for all threads.
template <typename T>
__device__ T block_sum(T v, T* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_allsum(v);
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    T s = lane < nw ? red[lane] : T(0);
    s = warp_allsum(s);
    if (lane == 0) red[32] = s;
  }
  __syncthreads();
  return red[32];
}

// h[k] = q_k . w for k <= j (warp per k); then w -= sum_k h[k] q_k with 8
// threads per row, each over a stride-8 subset of k, combined by shuffles.
template <typename T>
__device__ void reorth_pass(const T* Q, int n, int j, T* w, T* h) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int k = wid; k <= j; k += nw) {
    const T* q = Q + (size_t)k * n;
    T d = T(0);
    for (int i = lane; i < n; i += 32) d = fma(q[i], w[i], d);
    d = warp_allsum(d);
    if (lane == 0) h[k] = d;
  }
  __syncthreads();
  const int part = threadIdx.x & 7;
  const int rows_per_pass = blockDim.x >> 3;
  for (int i0 = 0; i0 < n; i0 += rows_per_pass) {
    const int i = i0 + (threadIdx.x >> 3);
    T acc = T(0);
    if (i < n)
      for (int k = part; k <= j; k += 8) acc = fma(h[k], Q[(size_t)k * n + i], acc);
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    acc += __shfl_xor_sync(0xffffffffu, acc, 4);
    if (i < n && part == 0) w[i] -= acc;
  }
  __syncthreads();
}

// FP32 variant with 16-byte shared-memory reads (n % 4 == 0): warp per q_k for
// the dots; for the update, warp per quad of rows with lanes over k.
__device__ void reorth_pass_v4(const float* Q, int n, int j, float* w, float* h) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int n4 = n >> 2;
  const float4* w4 = reinterpret_cast<const float4*>(w);
  for (int k = wid; k <= j; k += nw) {
    const float4* q4 = reinterpret_cast<const float4*>(Q + (size_t)k * n);
    float d = 0.f;
    for (int i = lane; i < n4; i += 32) {
      const float4 a = q4[i], b = w4[i];
      d = fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, fmaf(a.w, b.w, d))));
    }
    d = warp_allsum(d);
    if (lane == 0) h[k] = d;
  }
  __syncthreads();
  float4* wv = reinterpret_cast<float4*>(w);
  for (int qd = wid; qd < n4; qd += nw) {
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int k = lane; k <= j; k += 32) {
      const float hk = h[k];
      const float4 q = reinterpret_cast<const float4*>(Q + (size_t)k * n)[qd];
      acc.x = fmaf(hk, q.x, acc.x);
      acc.y = fmaf(hk, q.y, acc.y);
      acc.z = fmaf(hk, q.z, acc.z);
      acc.w = fmaf(hk, q.w, acc.w);
    }
    acc.x = warp_allsum(acc.x);
    acc.y = warp_allsum(acc.y);
    acc.z = warp_allsum(acc.z);
    acc.w = warp_allsum(acc.w);
    if (lane == 0) {
      float4 x = wv[qd];
      x.x -= acc.x;
      x.y -= acc.y;
      x.z -= acc.z;
      x.w -= acc.w;
      wv[qd] = x;
    }
  }
  __syncthreads();
}

template <typename T>
__device__ __forceinline__ void reorth(const T* Q, int n, int j, T* w, T* h) {
  if constexpr (sizeof(T) == 4) {
    if ((n & 3) == 0) {
      reorth_pass_v4(Q, n, j, w, h);
      return;
    }
  }
  reorth_pass<T>(Q, n, j, w, h);
}

// number of eigenvalues of the symmetric tridiagonal (a, b2 = off-diagonal^2) below x
template <typename T>
__device__ int sturm_count(const T* a, const T* b2, int m, T x, T pivmin) {
  int cnt = 0;
  T d = a[0] - x;
  if (fabs(d) < pivmin) d = -pivmin;
  cnt += d < T(0);
  for (int i = 1; i < m; ++i) {
    d = (a[i] - x) - b2[i - 1] / d;
    if (fabs(d) < pivmin) d = -pivmin;
    cnt += d < T(0);
  }
  return cnt;
}

// One thread: factor T - lam I (symmetric tridiagonal: diagonal a, off-diagonal
// b) by Gaussian elimination with partial pivoting; the upper factor has two
// superdiagonals.  `lu` holds 5m values.
template <typename T>
__device__ void tri_factor(const T* a, const T* b, int m, T lam, T tiny, T* lu) {
  T* u0 = lu;
  T* u1 = lu + m;
  T* u2 = lu + 2 * m;
  T* l = lu + 3 * m;
  T* pv = lu + 4 * m;
  T p = a[0] - lam, q = m > 1 ? b[0] : T(0), r = T(0);
  for (int i = 0; i < m - 1; ++i) {
    const T s = b[i], t = a[i + 1] - lam, u = (i + 2 < m) ? b[i + 1] : T(0);
    if (fabs(p) >= fabs(s)) {
      const T piv = (p == T(0)) ? tiny : p;
      u0[i] = piv;
      u1[i] = q;
      u2[i] = r;
      const T mult = s / piv;
      l[i] = mult;
      pv[i] = T(0);
      p = t - mult * q;
      q = u - mult * r;
      r = T(0);
    } else {
      u0[i] = s;
      u1[i] = t;
      u2[i] = u;
      const T mult = p / s;
      l[i] = mult;
      pv[i] = T(1);
      p = q - mult * t;
      q = r - mult * u;
      r = T(0);
    }
  }
  u0[m - 1] = (fabs(p) < tiny) ? (p < T(0) ? -tiny : tiny) : p;
  u1[m - 1] = T(0);
  u2[m - 1] = T(0);
}

// Solves with the factor of tri_factor; x holds the right-hand side on entry.
template <typename T>
__device__ void tri_solve(const T* lu, int m, T* x) {
  const T* u0 = lu;
  const T* u1 = lu + m;
  const T* u2 = lu + 2 * m;
  const T* l = lu + 3 * m;
  const T* pv = lu + 4 * m;
  T top = x[0];
  for (int i = 0; i < m - 1; ++i) {
    const T bot = x[i + 1];
    if (pv[i] == T(0)) {
      x[i] = top;
      top = bot - l[i] * top;
    } else {
      x[i] = bot;
      top = top - l[i] * bot;
    }
  }
  x[m - 1] = top;
  for (int i = m - 1; i >= 0; --i) {
    T v = x[i];
    if (i + 1 < m) v -= u1[i] * x[i + 1];
    if (i + 2 < m) v -= u2[i] * x[i + 2];
    x[i] = v / u0[i];
  }
}

constexpr int kEigSmallThreads = 128;

// Shared phases of the compact eigensolvers (128 threads): the top-K
// eigenpairs of the m x m tridiagonal (ta, tb) -- Gershgorin interval,
// multisection, inverse iteration into tri -- and, after the caller's
// back-transformation into Xs, modified Gram-Schmidt, the FP64 refinement and
// the scaled output Vs.
template <typename T>
struct EigSmem {
  T* red;
  double* lo_s;
  double* hi_s;
  T* lam_s;
  T* inv_sig;
  int* cnt_s;
  T* mn_s;
  T* mx_s;
  T* b2_s;
};

template <typename T, int NT = kEigSmallThreads>
__device__ void eig_tridiag_topk(const EigArgs<T>& a, const EigSmem<T>& sh, int m, T* ta, T* tb, T* tb2, T* tri,
                                 T fro, T eps) {
  const int K = a.K, tid = threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5;
  constexpr int NW = NT / 32;
  T* red = sh.red;
  double* lo_s = sh.lo_s;
  double* hi_s = sh.hi_s;
  T* lam_s = sh.lam_s;
  int* cnt_s = sh.cnt_s;
  T* mn_s = sh.mn_s;
  T* mx_s = sh.mx_s;
  T* b2_s = sh.b2_s;
  // ---- Gershgorin interval and pivot threshold
  {
    T mn = T(INFINITY), mx = T(-INFINITY), b2m = T(0);
    for (int i = tid; i < m; i += NT) {
      const T bb = tb[i];
      tb2[i] = bb * bb;
      const T r = (i > 0 ? fabs(tb[i - 1]) : T(0)) + fabs(bb);
      mn = fmin(mn, ta[i] - r);
      mx = fmax(mx, ta[i] + r);
      b2m = fmax(b2m, bb * bb);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
      mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      b2m = fmax(b2m, __shfl_xor_sync(0xffffffffu, b2m, o));
    }
    if (lane == 0) {
      mn_s[wid] = mn;
      mx_s[wid] = mx;
      b2_s[wid] = b2m;
    }
    __syncthreads();
    if (tid < K) {
      T lo = T(INFINITY), hi = T(-INFINITY);
      for (int i = 0; i < NW; ++i) {
        lo = fmin(lo, mn_s[i]);
        hi = fmax(hi, mx_s[i]);
      }
      const T pad = T(1e-6) * (hi - lo) + T(10) * eps * fabs(hi) + T(1e-30);
      lo_s[tid] = (double)(lo - pad);
      hi_s[tid] = (double)(hi + pad);
    }
    if (tid == 0) {
      T b2 = T(0);
      for (int i = 0; i < NW; ++i) b2 = fmax(b2, b2_s[i]);
      red[0] = (sizeof(T) == 4 ? T(1e-30) : T(1e-290)) * fmax(T(1), b2);
    }
    __syncthreads();
  }
  const T pivmin = red[0];
  __syncthreads();
  // ---- multisection for the K largest eigenvalues of T (NT / K sections each)
  {
    const int S = NT / K;
    const double inv_s1 = 1.0 / (double)(S + 1);
    // shrink by (S + 1) per round down to FP rounding of the interval width
    const int rounds = (int)ceil((sizeof(T) == 4 ? 24.0 : 53.0) * 0.6931471805599453 / log((double)(S + 1))) + 1;
    for (int rd = 0; rd < rounds; ++rd) {
      const int k = tid / S, sidx = tid - k * S;
      if (k < K) {
        const double step = (hi_s[k] - lo_s[k]) * inv_s1;
        cnt_s[tid] = sturm_count<T>(ta, tb2, m, (T)(lo_s[k] + step * (double)(sidx + 1)), pivmin);
      }
      __syncthreads();
      if (tid < K) {
        const int target = m - 1 - tid;  // ascending index of the (tid+1)-th largest eigenvalue
        const double l0 = lo_s[tid], step = (hi_s[tid] - l0) * inv_s1;
        double nlo = l0, nhi = hi_s[tid];
        for (int s2 = 0; s2 < S; ++s2) {
          if (cnt_s[tid * S + s2] <= target) {
            nlo = l0 + step * (double)(s2 + 1);
          } else {
            nhi = l0 + step * (double)(s2 + 1);
            break;
          }
        }
        lo_s[tid] = nlo;
        hi_s[tid] = nhi;
      }
      __syncthreads();
    }
  }
  if (tid < K) lam_s[tid] = (T)(0.5 * (lo_s[tid] + hi_s[tid]));
  __syncthreads();
  if (a.clk && tid == 0) a.clk[2] = clock64();
  // ---- inverse iteration, one thread per eigenvalue, factors in shared memory
  for (int k = tid; k < K; k += NT) {
    T* lu = tri + (size_t)k * 6 * m;
    T* x = lu + 5 * m;
    const T tiny = eps * fro + T(1e-30);
    tri_factor<T>(ta, tb, m, lam_s[k], tiny, lu);
    for (int i = 0; i < m; ++i) x[i] = hash_unit<T>(101 + k, i);
    for (int it = 0; it < 3; ++it) {
      tri_solve<T>(lu, m, x);
      T nn = T(0);
      for (int i = 0; i < m; ++i) nn = fma(x[i], x[i], nn);
      const T inv = nn > T(0) ? T(1) / sqrt(nn) : T(0);
      for (int i = 0; i < m; ++i) x[i] *= inv;
    }
  }
  __syncthreads();
  if (a.clk && tid == 0) a.clk[3] = clock64();
}

// Early stop of the Lanczos process: after m steps (T_m = tridiag(ta, tb) with
// tb[m-1] = 0, next coefficient beta) the top-K Ritz pairs of W have residual
// norms ||W y_k - theta_k y_k|| = beta |s_k[m-1]|, s_k the k-th eigenvector of
// T_m (into `tri`, K x 6m).  True, for the whole block, when every residual is
// <= tol * theta_max: the Ritz vectors are then within tol * theta_max / gap
// of W's eigenvectors, and the FP64 refinement that follows shrinks the rest.
// Checked from step kLanczosFirstCheck(K) on, every kLanczosCheckEvery steps.
constexpr int kLanczosCheckEvery = 8;
__host__ __device__ inline int kLanczosFirstCheck(int K) { return 2 * K + 4; }

template <typename T, int NT>
__device__ bool lanczos_converged(const EigArgs<T>& a, const EigSmem<T>& sh, int m, T* ta, T* tb, T* tb2, T* tri,
                                  T beta, T fro, T eps, int* flag) {
  eig_tridiag_topk<T, NT>(a, sh, m, ta, tb, tb2, tri, fro, eps);
  if (threadIdx.x == 0) *flag = 1;
  __syncthreads();
  const T tol = (sizeof(T) == 4 ? T(2e-6) : T(1e-13)) * fabs(sh.lam_s[0]);
  if (threadIdx.x < a.K) {
    const T* x = tri + (size_t)threadIdx.x * 6 * m + 5 * m;
    if (!(beta * fabs(x[m - 1]) <= tol)) *flag = 0;
  }
  __syncthreads();
  const bool ok = *flag != 0;
  __syncthreads();
  return ok;
}

// Top-K eigenpairs of the symmetric n x n Gram matrix W in one CTA, in the
// context precision T:
//   Lanczos tridiagonalisation T = Q^T W Q with full re-orthogonalisation
//   (classical Gram-Schmidt, twice); multisection (parallel Sturm counts) for
//   the K largest eigenvalues of T; inverse iteration (pivoted tridiagonal LU)
//   for their eigenvectors; back-transformation X = Q S and modified
//   Gram-Schmidt.  With `polish` (FP32 context) the basis is refined in FP64:
//   Y = W X, then CholeskyQR of Y gives the basis X' = Y R^-1 and R_kk ~ lambda_k.
template <typename T>
__global__ void __launch_bounds__(1024) k_eig(const EigArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ T red[33];
  __shared__ double lo_s[TK_MAXK], hi_s[TK_MAXK];
  __shared__ T lam_s[TK_MAXK], inv_sig[TK_MAXK];
  __shared__ double C[TK_MAXK][TK_MAXK + 1];
  __shared__ double Ri[TK_MAXK][TK_MAXK + 1];
  __shared__ int cnt_s[1024];
  __shared__ T mn_s[32], mx_s[32], b2_s[32];
  const int n = a.n, K = a.K, tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  int m = n;  // Lanczos steps taken (early stop at convergence)
  unsigned char* p = smem;
  T* A;
  T* Q;
  if (a.use_smem) {
    A = (T*)p;
    p += (size_t)n * n * sizeof(T);
    Q = (T*)p;
    p += (size_t)n * m * sizeof(T);
  } else {
    A = a.gA;
    Q = a.gQ;
  }
  T* w = (T*)p;
  p += (size_t)n * sizeof(T);
  T* h = (T*)p;
  p += (size_t)m * sizeof(T);
  T* ta = (T*)p;
  p += (size_t)m * sizeof(T);
  T* tb = (T*)p;
  p += (size_t)m * sizeof(T);
  T* tb2 = (T*)p;

  T fro2 = T(0);
  for (int idx = tid; idx < n * n; idx += nt) {
    const T v = (T)a.W[idx];
    A[idx] = v;
    fro2 = fma(v, v, fro2);
  }
  const T fro = sqrt(block_sum<T>(fro2, red));
  const T eps = sizeof(T) == 4 ? T(1.2e-7) : T(2.3e-16);
  const EigSmem<T> sh_ck{red, lo_s, hi_s, lam_s, inv_sig, cnt_s, mn_s, mx_s, b2_s};
  __shared__ int conv_flag;
  bool conv = false;  // the Lanczos run stopped at a successful check
  if (a.clk && tid == 0) a.clk[0] = clock64();

  // ---- Lanczos
  for (int i = tid; i < n; i += nt) w[i] = hash_unit<T>(1, i);
  {
    T nn = T(0);
    for (int i = tid; i < n; i += nt) nn = fma(w[i], w[i], nn);
    const T inv = T(1) / sqrt(block_sum<T>(nn, red));
    for (int i = tid; i < n; i += nt) Q[i] = w[i] * inv;
    __syncthreads();
  }
  for (int j = 0; j < m; ++j) {
    const T* qj = Q + (size_t)j * n;
    bool vec_done = false;
    if constexpr (sizeof(T) == 4) {
      if ((n & 3) == 0) {  // w = A q_j, warp per row, 16-byte reads
        const int n4 = n >> 2;
        const float4* q4 = reinterpret_cast<const float4*>(qj);
        for (int r = wid; r < n; r += nw) {
          const float4* a4 = reinterpret_cast<const float4*>(A + (size_t)r * n);
          float sacc = 0.f;
          for (int i = lane; i < n4; i += 32) {
            const float4 x = a4[i], y = q4[i];
            sacc = fmaf(x.x, y.x, fmaf(x.y, y.y, fmaf(x.z, y.z, fmaf(x.w, y.w, sacc))));
          }
          sacc = warp_allsum(sacc);
          if (lane == 0) w[r] = sacc;
        }
        vec_done = true;
      }
    }
    if (!vec_done) {
      for (int r = wid; r < n; r += nw) {  // w = A q_j, warp per row
        const T* ar = A + (size_t)r * n;
        T sacc = T(0);
        for (int cidx = lane; cidx < n; cidx += 32) sacc = fma(ar[cidx], qj[cidx], sacc);
        sacc = warp_allsum(sacc);
        if (lane == 0) w[r] = sacc;
      }
    }
    __syncthreads();
    reorth<T>(Q, n, j, w, h);
    T al = h[j];
    reorth<T>(Q, n, j, w, h);
    al += h[j];
    if (tid == 0) ta[j] = al;
    T nn = T(0);
    for (int i = tid; i < n; i += nt) nn = fma(w[i], w[i], nn);
    const T bnorm = sqrt(block_sum<T>(nn, red));
    if (j == m - 1) break;
    if (j + 1 >= kLanczosFirstCheck(K) && (j + 1 - kLanczosFirstCheck(K)) % kLanczosCheckEvery == 0) {
      // early stop once the top-K Ritz pairs have converged
      if (tid == 0) tb[j] = T(0);
      __syncthreads();
      if (lanczos_converged<T, 1024>(a, sh_ck, j + 1, ta, tb, tb2, a.tri, bnorm, fro, eps, &conv_flag)) {
        m = j + 1;
        conv = true;
        break;
      }
    }
    T* qn = Q + (size_t)(j + 1) * n;
    if (bnorm > T(100) * eps * fro) {
      if (tid == 0) tb[j] = bnorm;
      const T inv = T(1) / bnorm;
      for (int i = tid; i < n; i += nt) qn[i] = w[i] * inv;
    } else {
      // invariant subspace found: restart with a fresh vector orthogonal to q_0..q_j
      if (tid == 0) tb[j] = T(0);
      for (int i = tid; i < n; i += nt) w[i] = hash_unit<T>(j + 2, i);
      __syncthreads();
      reorth<T>(Q, n, j, w, h);
      reorth<T>(Q, n, j, w, h);
      T n2 = T(0);
      for (int i = tid; i < n; i += nt) n2 = fma(w[i], w[i], n2);
      n2 = block_sum<T>(n2, red);
      const T inv = n2 > T(0) ? T(1) / sqrt(n2) : T(0);
      for (int i = tid; i < n; i += nt) qn[i] = w[i] * inv;
    }
    __syncthreads();
  }
  if (tid == 0) tb[m - 1] = T(0);
  __syncthreads();
  if (a.clk && tid == 0) a.clk[1] = clock64();

  // a successful early-stop check has solved this very T_m into a.tri already
  if (!conv) eig_tridiag_topk<T, 1024>(a, sh_ck, m, ta, tb, tb2, a.tri, fro, eps);
  if (a.clk && tid == 0) a.clk[3] = clock64();
  // ---- X = Q S, then modified Gram-Schmidt (separates clustered eigenvalues)
  for (int idx = tid; idx < n * K; idx += nt) {
    const int i = idx / K, k = idx - i * K;
    const T* x = a.tri + (size_t)k * 6 * m + 5 * m;
    T s2 = T(0);
    for (int j = 0; j < m; ++j) s2 = fma(Q[(size_t)j * n + i], x[j], s2);
    a.X[idx] = (double)s2;
  }
  __syncthreads();
  if (a.clk && tid == 0) a.clk[4] = clock64();
  for (int k = 0; k < K; ++k) {
    for (int j = 0; j < k; ++j) {
      T d = T(0);
      for (int i = tid; i < n; i += nt) d = fma((T)a.X[i * K + j], (T)a.X[i * K + k], d);
      d = block_sum<T>(d, red);
      for (int i = tid; i < n; i += nt) a.X[i * K + k] = (double)((T)a.X[i * K + k] - d * (T)a.X[i * K + j]);
      __syncthreads();
    }
    T nn = T(0);
    for (int i = tid; i < n; i += nt) nn = fma((T)a.X[i * K + k], (T)a.X[i * K + k], nn);
    nn = block_sum<T>(nn, red);
    const T inv = nn > T(0) ? T(1) / sqrt(nn) : T(0);
    for (int i = tid; i < n; i += nt) a.X[i * K + k] = (double)((T)a.X[i * K + k] * inv);
    __syncthreads();
  }
  if (a.clk && tid == 0) a.clk[5] = clock64();
  if (a.polish) {
    // FP64 refinement: Y = W X, C = Y^T Y, C = R^T R, X' = Y R^-1, sigma_k^2 ~ R_kk
    for (int idx = tid; idx < n * K; idx += nt) {
      const int i = idx / K, k = idx - i * K;
      double s2 = 0.0;
      const double* wr = a.W + (int64_t)i * n;
      for (int cc = 0; cc < n; ++cc) s2 = fma(wr[cc], a.X[cc * K + k], s2);
      a.Y[idx] = s2;
    }
    __syncthreads();
    if (a.clk && tid == 0) a.clk[6] = clock64();
    for (int pr = tid; pr < K * K; pr += nt) {
      const int r = pr / K, cc = pr - r * K;
      if (r <= cc) {
        double s2 = 0.0;
        for (int i = 0; i < n; ++i) s2 = fma(a.Y[i * K + r], a.Y[i * K + cc], s2);
        C[r][cc] = s2;
        C[cc][r] = s2;
      }
    }
    __syncthreads();
    if (wid == 0) {  // Cholesky C = L L^T (lower, in place) and Ri = L^-T (upper), one warp
      bool bad = false;
      for (int j = 0; j < K; ++j) {
        double d = C[j][j];
        if (!(d > 0.0)) bad = true;
        d = d > 0.0 ? sqrt(d) : 1.0;
        __syncwarp();
        if (lane == j) C[j][j] = d;
        if (lane > j && lane < K) C[lane][j] /= d;
        __syncwarp();
        if (lane > j && lane < K)
          for (int k2 = j + 1; k2 <= lane; ++k2) C[lane][k2] -= C[lane][j] * C[k2][j];
        __syncwarp();
      }
      if (bad && lane == 0) atomicOr(a.err, TK_DEV_ERR_NUMERIC);
      if (lane < K) {
        for (int i = K - 1; i >= 0; --i) {
          double s2 = (i == lane) ? 1.0 : 0.0;
          for (int k2 = i + 1; k2 < K; ++k2) s2 -= C[k2][i] * Ri[k2][lane];
          Ri[i][lane] = (i <= lane) ? s2 / C[i][i] : 0.0;
        }
        a.sigma[lane] = sqrt(fabs(C[lane][lane]));  // R_kk ~ lambda_k, sigma_k = sqrt(lambda_k)
      }
    }
    __syncthreads();
    for (int idx = tid; idx < n * K; idx += nt) {
      const int i = idx / K, k = idx - i * K;
      double s2 = 0.0;
      for (int j = 0; j <= k; ++j) s2 = fma(a.Y[i * K + j], Ri[j][k], s2);
      a.Vout[idx] = s2;
    }
  } else {
    for (int idx = tid; idx < n * K; idx += nt) a.Vout[idx] = a.X[idx];
    for (int k = tid; k < K; k += nt) a.sigma[k] = sqrt(fmax((double)lam_s[k], 0.0));
  }
  __syncthreads();
  if (tid < K) {
    const double sg = a.sigma[tid];
    const bool ok = sg > 0.0 && isfinite(sg);
    if (!ok) atomicOr(a.err, TK_DEV_ERR_NUMERIC);
    inv_sig[tid] = ok ? (T)(1.0 / sg) : T(0);
  }
  __syncthreads();
  for (int idx = tid; idx < n * K; idx += nt) a.Vs[idx] = (T)a.Vout[idx] * inv_sig[idx % K];
  if (a.clk && tid == 0) a.clk[7] = clock64();
}

// Compact form of the same eigensolver for Gram matrices that fit in shared
// memory with their Lanczos basis (Khat up to about 150 in FP32): 128 threads,
// thread r owning rows r, r + 128 of every Lanczos vector, so that a step needs
// no cross-warp shuffles -- only seven short barriers:
//   w = A q_j           thread r: dot of column-major A's row r with q_j
//   h = Q^T w, w -= Q h thread k forms h_k, thread r its row of Q h (twice)
//   beta = ||w||        block sum
// Q is stored row-major with an odd leading dimension (ldq), conflict-free for
// both the per-k and the per-r sweeps.  The tridiagonal phases and the modified
// Gram-Schmidt of the eigenvectors work in shared memory; the FP64 refinement
// is the same as in k_eig.

template <typename T>
__host__ __device__ inline int eig_small_ldq(int n) {
  return n | 1;
}
// dynamic shared memory: A (n*n; reused for the inverse-iteration factors when
// 6*K*n <= n*n), Q (n*ldq), X (n*K), 6 vectors of n, the factors (if not reused)
// (after two K x (K+1) FP64 matrices for the refinement's Cholesky factor)
template <typename T>
__host__ __device__ inline size_t eig_small_smem(int n, int K) {
  const size_t tri = (size_t)6 * K * n;
  size_t e = (size_t)n * n + (size_t)n * eig_small_ldq<T>(n) + (size_t)n * K + (size_t)6 * n;
  if (tri > (size_t)n * n) e += tri;
  return (size_t)2 * K * (K + 1) * sizeof(double) + e * sizeof(T);
}

template <typename T>
__device__ void eig_finish(const EigArgs<T>& a, const EigSmem<T>& sh, int n, T* Xs, double* Cm, double* Rm) {
  const int K = a.K, tid = threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5;
  constexpr int NT = kEigSmallThreads;
  T* lam_s = sh.lam_s;
  T* inv_sig = sh.inv_sig;
  // ---- modified Gram-Schmidt on one warp (separates clustered eigenvalues)
  if (wid == 0) {
    for (int k = 0; k < K; ++k) {
      for (int j = 0; j < k; ++j) {
        T d = T(0);
        for (int r = lane; r < n; r += 32) d = fma(Xs[r * K + j], Xs[r * K + k], d);
        d = warp_allsum(d);
        for (int r = lane; r < n; r += 32) Xs[r * K + k] -= d * Xs[r * K + j];
        __syncwarp();
      }
      T nn = T(0);
      for (int r = lane; r < n; r += 32) nn = fma(Xs[r * K + k], Xs[r * K + k], nn);
      nn = warp_allsum(nn);
      const T inv = nn > T(0) ? T(1) / sqrt(nn) : T(0);
      for (int r = lane; r < n; r += 32) Xs[r * K + k] *= inv;
      __syncwarp();
    }
  }
  __syncthreads();
  if (a.clk && tid == 0) a.clk[5] = clock64();
  if (a.polish) {
    // FP64 refinement: Y = W X, C = Y^T Y, C = R^T R, X' = Y R^-1, sigma_k^2 ~ R_kk
    for (int idx = tid; idx < n * K; idx += NT) {
      const int i = idx / K, k = idx - i * K;
      double s2 = 0.0;
      const double* wr = a.W + (int64_t)i * n;
      for (int cc = 0; cc < n; ++cc) s2 = fma(wr[cc], (double)Xs[cc * K + k], s2);
      a.Y[idx] = s2;
    }
    __syncthreads();
    if (a.clk && tid == 0) a.clk[6] = clock64();
    for (int pr = tid; pr < K * K; pr += NT) {
      const int r = pr / K, cc = pr - r * K;
      if (r <= cc) {
        double s2 = 0.0;
        for (int i = 0; i < n; ++i) s2 = fma(a.Y[i * K + r], a.Y[i * K + cc], s2);
        Cm[(r) * (K + 1) + (cc)] = s2;
        Cm[(cc) * (K + 1) + (r)] = s2;
      }
    }
    __syncthreads();
    if (wid == 0) {  // Cholesky C = L L^T (lower, in place) and Ri = L^-T (upper), one warp
      bool bad = false;
      for (int j = 0; j < K; ++j) {
        double d = Cm[(j) * (K + 1) + (j)];
        if (!(d > 0.0)) bad = true;
        d = d > 0.0 ? sqrt(d) : 1.0;
        __syncwarp();
        if (lane == j) Cm[(j) * (K + 1) + (j)] = d;
        if (lane > j && lane < K) Cm[(lane) * (K + 1) + (j)] /= d;
        __syncwarp();
        if (lane > j && lane < K)
          for (int k2 = j + 1; k2 <= lane; ++k2) Cm[(lane) * (K + 1) + (k2)] -= Cm[(lane) * (K + 1) + (j)] * Cm[(k2) * (K + 1) + (j)];
        __syncwarp();
      }
      if (bad && lane == 0) atomicOr(a.err, TK_DEV_ERR_NUMERIC);
      if (lane < K) {
        for (int i = K - 1; i >= 0; --i) {
          double s2 = (i == lane) ? 1.0 : 0.0;
          for (int k2 = i + 1; k2 < K; ++k2) s2 -= Cm[(k2) * (K + 1) + (i)] * Rm[(k2) * (K + 1) + (lane)];
          Rm[(i) * (K + 1) + (lane)] = (i <= lane) ? s2 / Cm[(i) * (K + 1) + (i)] : 0.0;
        }
        a.sigma[lane] = sqrt(fabs(Cm[(lane) * (K + 1) + (lane)]));
      }
    }
    __syncthreads();
    for (int idx = tid; idx < n * K; idx += NT) {
      const int i = idx / K, k = idx - i * K;
      double s2 = 0.0;
      for (int j = 0; j <= k; ++j) s2 = fma(a.Y[i * K + j], Rm[(j) * (K + 1) + (k)], s2);
      a.Vout[idx] = s2;
    }
  } else {
    for (int idx = tid; idx < n * K; idx += NT) a.Vout[idx] = (double)Xs[idx];
    for (int k = tid; k < K; k += NT) a.sigma[k] = sqrt(fmax((double)lam_s[k], 0.0));
  }
  __syncthreads();
  if (tid < K) {
    const double sg = a.sigma[tid];
    const bool ok = sg > 0.0 && isfinite(sg);
    if (!ok) atomicOr(a.err, TK_DEV_ERR_NUMERIC);
    inv_sig[tid] = ok ? (T)(1.0 / sg) : T(0);
  }
  __syncthreads();
  for (int idx = tid; idx < n * K; idx += NT) a.Vs[idx] = (T)a.Vout[idx] * inv_sig[idx % K];
  if (a.clk && tid == 0) a.clk[7] = clock64();
}

template <typename T>
__global__ void __launch_bounds__(kEigSmallThreads) k_eig_small(const EigArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ T red[33];
  __shared__ double lo_s[TK_MAXK], hi_s[TK_MAXK];
  __shared__ T lam_s[TK_MAXK], inv_sig[TK_MAXK];
  __shared__ int cnt_s[kEigSmallThreads];
  __shared__ T mn_s[4], mx_s[4], b2_s[4];
  const int n = a.n, K = a.K, tid = threadIdx.x;
  constexpr int NT = kEigSmallThreads;
  int m = n;  // Lanczos steps taken (early stop at convergence)
  const int ldq = eig_small_ldq<T>(n);
  // Cholesky factor C and its inverse Ri (refinement), K x (K + 1) row-major
  double* Cm = (double*)smem;
  double* Rm = Cm + K * (K + 1);
  T* A = (T*)(Rm + K * (K + 1));
  T* Q = A + (size_t)n * n;
  T* Xs = Q + (size_t)n * ldq;
  T* ws = Xs + (size_t)n * K;
  T* hs = ws + n;
  T* ta = hs + n;
  T* tb = ta + n;
  T* tb2 = tb + n;
  T* tri = ((size_t)6 * K * n <= (size_t)n * n) ? A : tb2 + n;

  T fro2 = T(0);
  for (int idx = tid; idx < n * n; idx += NT) {
    const T v = (T)a.W[idx];  // W symmetric: row-major = column-major
    A[idx] = v;
    fro2 = fma(v, v, fro2);
  }
  const T fro = sqrt(block_sum<T>(fro2, red));
  const T eps = sizeof(T) == 4 ? T(1.2e-7) : T(2.3e-16);
  const EigSmem<T> sh_ck{red, lo_s, hi_s, lam_s, inv_sig, cnt_s, mn_s, mx_s, b2_s};
  __shared__ int conv_flag;
  bool conv = false;  // the Lanczos run stopped at a successful check
  if (a.clk && tid == 0) a.clk[0] = clock64();

  // rows owned by this thread (n <= 2 * NT)
  const int r0 = tid, r1 = tid + NT;
  const bool h0 = r0 < n, h1 = r1 < n;
  T w0 = T(0), w1 = T(0);
  // start vector
  {
    if (h0) w0 = hash_unit<T>(1, r0);
    if (h1) w1 = hash_unit<T>(1, r1);
    const T inv = T(1) / sqrt(block_sum<T>(w0 * w0 + w1 * w1, red));
    if (h0) Q[(size_t)r0 * ldq] = w0 * inv;
    if (h1) Q[(size_t)r1 * ldq] = w1 * inv;
    __syncthreads();
  }
  // one classical Gram-Schmidt pass of (w0, w1) against q_0..q_j; returns h_j
  auto cgs = [&](int j) -> T {
    if (h0) ws[r0] = w0;
    if (h1) ws[r1] = w1;
    __syncthreads();
    for (int k = tid; k <= j; k += NT) {
      T s0 = T(0), s1 = T(0);
      int r = 0;
      for (; r + 1 < n; r += 2) {
        s0 = fma(Q[(size_t)r * ldq + k], ws[r], s0);
        s1 = fma(Q[(size_t)(r + 1) * ldq + k], ws[r + 1], s1);
      }
      if (r < n) s0 = fma(Q[(size_t)r * ldq + k], ws[r], s0);
      hs[k] = s0 + s1;
    }
    __syncthreads();
    if (h0) {
      const T* qr = Q + (size_t)r0 * ldq;
      T s0 = T(0), s1 = T(0);
      int k = 0;
      for (; k + 1 <= j; k += 2) {
        s0 = fma(qr[k], hs[k], s0);
        s1 = fma(qr[k + 1], hs[k + 1], s1);
      }
      if (k <= j) s0 = fma(qr[k], hs[k], s0);
      w0 -= s0 + s1;
    }
    if (h1) {
      const T* qr = Q + (size_t)r1 * ldq;
      T s0 = T(0), s1 = T(0);
      int k = 0;
      for (; k + 1 <= j; k += 2) {
        s0 = fma(qr[k], hs[k], s0);
        s1 = fma(qr[k + 1], hs[k + 1], s1);
      }
      if (k <= j) s0 = fma(qr[k], hs[k], s0);
      w1 -= s0 + s1;
    }
    return hs[j];
  };

  for (int j = 0; j < m; ++j) {
    // w = A q_j
    {
      T s0 = T(0), s1 = T(0), u0 = T(0), u1 = T(0);
      int cc = 0;
      for (; cc + 1 < n; cc += 2) {
        const T q0 = Q[(size_t)cc * ldq + j], q1 = Q[(size_t)(cc + 1) * ldq + j];
        if (h0) {
          s0 = fma(A[(size_t)cc * n + r0], q0, s0);
          s1 = fma(A[(size_t)(cc + 1) * n + r0], q1, s1);
        }
        if (h1) {
          u0 = fma(A[(size_t)cc * n + r1], q0, u0);
          u1 = fma(A[(size_t)(cc + 1) * n + r1], q1, u1);
        }
      }
      if (cc < n) {
        const T q0 = Q[(size_t)cc * ldq + j];
        if (h0) s0 = fma(A[(size_t)cc * n + r0], q0, s0);
        if (h1) u0 = fma(A[(size_t)cc * n + r1], q0, u0);
      }
      w0 = s0 + s1;
      w1 = u0 + u1;
    }
    T al = cgs(j);
    __syncthreads();  // hs is rewritten by the second pass
    al += cgs(j);
    if (tid == 0) ta[j] = al;
    const T bnorm = sqrt(block_sum<T>(w0 * w0 + w1 * w1, red));
    if (j == m - 1) break;
    if (j + 1 >= kLanczosFirstCheck(K) && (j + 1 - kLanczosFirstCheck(K)) % kLanczosCheckEvery == 0) {
      // early stop once the top-K Ritz pairs have converged
      if (tid == 0) tb[j] = T(0);
      __syncthreads();
      if (lanczos_converged<T, 128>(a, sh_ck, j + 1, ta, tb, tb2, a.tri, bnorm, fro, eps, &conv_flag)) {
        m = j + 1;
        conv = true;
        break;
      }
    }
    if (bnorm > T(100) * eps * fro) {
      if (tid == 0) tb[j] = bnorm;
      const T inv = T(1) / bnorm;
      if (h0) Q[(size_t)r0 * ldq + j + 1] = w0 * inv;
      if (h1) Q[(size_t)r1 * ldq + j + 1] = w1 * inv;
    } else {
      // invariant subspace: continue with a fresh vector orthogonal to q_0..q_j
      if (tid == 0) tb[j] = T(0);
      w0 = h0 ? hash_unit<T>(j + 2, r0) : T(0);
      w1 = h1 ? hash_unit<T>(j + 2, r1) : T(0);
      cgs(j);
      __syncthreads();
      cgs(j);
      const T n2 = block_sum<T>(w0 * w0 + w1 * w1, red);
      const T inv = n2 > T(0) ? T(1) / sqrt(n2) : T(0);
      if (h0) Q[(size_t)r0 * ldq + j + 1] = w0 * inv;
      if (h1) Q[(size_t)r1 * ldq + j + 1] = w1 * inv;
    }
    __syncthreads();
  }
  if (tid == 0) tb[m - 1] = T(0);
  __syncthreads();
  if (a.clk && tid == 0) a.clk[1] = clock64();

  const EigSmem<T> sh{red, lo_s, hi_s, lam_s, inv_sig, cnt_s, mn_s, mx_s, b2_s};
  // a successful early-stop check has solved this very T_m into a.tri already
  const T* trix = conv ? a.tri : tri;
  if (!conv) eig_tridiag_topk<T>(a, sh, m, ta, tb, tb2, tri, fro, eps);
  // ---- X = Q S (row r of X from row r of Q)
  for (int idx = tid; idx < n * K; idx += NT) {
    const int r = idx / K, k = idx - r * K;
    const T* x = trix + (size_t)k * 6 * m + 5 * m;
    const T* qr = Q + (size_t)r * ldq;
    T s0 = T(0), s1 = T(0);
    int j = 0;
    for (; j + 1 < m; j += 2) {
      s0 = fma(qr[j], x[j], s0);
      s1 = fma(qr[j + 1], x[j + 1], s1);
    }
    if (j < m) s0 = fma(qr[j], x[j], s0);
    Xs[idx] = s0 + s1;
  }
  __syncthreads();
  if (a.clk && tid == 0) a.clk[4] = clock64();
  eig_finish<T>(a, sh, n, Xs, Cm, Rm);
}

// FP32 form with 16-byte shared-memory traffic, for Khat <= 128 (thread r owns
// row r): W row-major and the Lanczos basis twice, component-major Q[r][k] for
// the update w -= Q h and vector-major QT[k][r] for the projections h = Q^T w,
// so that every inner product reads float4 from its own row and a float4
// broadcast of the other operand; leading dimensions are odd multiples of 4
// floats (eight lanes' 16-byte reads fall on distinct banks).  Vectors are
// padded to a multiple of 4 with zeros, which the Krylov space never touches
// (W's padding is zero).  The tridiagonal phases, Gram-Schmidt and the FP64
// refinement are shared with k_eig_small.
constexpr int kEigV4MaxN = 128;

__host__ __device__ inline int eig_v4_ld(int n) {
  int l = (n + 3) & ~3;
  while (l % 8 != 4) l += 4;
  return l;
}
__host__ __device__ inline size_t eig_v4_smem(int n, int K) {
  const int ld = eig_v4_ld(n), np = (n + 3) & ~3;
  // the n x K block is padded to whole float4s: the vectors after it are read as float4
  size_t e = (size_t)3 * n * ld + (((size_t)n * K + 3) & ~(size_t)3) + (size_t)5 * np;
  if ((size_t)6 * K * n > (size_t)n * ld) e += (size_t)6 * K * n;
  return (size_t)2 * K * (K + 1) * sizeof(double) + e * sizeof(float);
}

__global__ void __launch_bounds__(kEigSmallThreads) k_eig_v4(const EigArgs<float> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ float red[33];
  __shared__ double lo_s[TK_MAXK], hi_s[TK_MAXK];
  __shared__ float lam_s[TK_MAXK], inv_sig[TK_MAXK];
  __shared__ int cnt_s[kEigSmallThreads];
  __shared__ float mn_s[4], mx_s[4], b2_s[4];
  const int n = a.n, K = a.K, tid = threadIdx.x;
  constexpr int NT = kEigSmallThreads;
  int m = n;  // Lanczos steps taken (early stop at convergence)
  const int ld = eig_v4_ld(n), np = (n + 3) & ~3, np4 = np / 4;
  double* Cm = (double*)smem;
  double* Rm = Cm + K * (K + 1);
  float* A = (float*)(Rm + K * (K + 1));  // n x ld, row r = W[r][:]
  float* Q = A + (size_t)n * ld;          // n x ld, Q[r][k]
  float* QT = Q + (size_t)n * ld;         // m x ld, QT[k][r]
  float* Xs = QT + (size_t)m * ld;
  float* ws = Xs + (((size_t)n * K + 3) & ~(size_t)3);  // 16-byte aligned (float4 reads)
  float* hs = ws + np;
  float* ta = hs + np;
  float* tb = ta + np;
  float* tb2 = tb + np;
  float* tri = ((size_t)6 * K * n <= (size_t)n * ld) ? A : tb2 + np;

  float fro2 = 0.f;
  for (int idx = tid; idx < n * ld; idx += NT) {
    const int r = idx / ld, c = idx - r * ld;
    const float v = c < n ? (float)a.W[(int64_t)r * n + c] : 0.f;
    A[idx] = v;
    fro2 = fmaf(v, v, fro2);
    Q[idx] = 0.f;
    QT[idx] = 0.f;  // m == n rows
  }
  for (int i = tid; i < 2 * np; i += NT) ws[i] = 0.f;  // ws and hs, including padding
  const float fro = sqrtf(block_sum<float>(fro2, red));
  const float eps = 1.2e-7f;
  const EigSmem<float> sh_ck{red, lo_s, hi_s, lam_s, inv_sig, cnt_s, mn_s, mx_s, b2_s};
  __shared__ int conv_flag;
  bool conv = false;  // the Lanczos run stopped at a successful check
  if (a.clk && tid == 0) a.clk[0] = clock64();

  const int r = tid;
  const bool own = r < n;
  float w = own ? hash_unit<float>(1, r) : 0.f;
  {
    const float inv = 1.f / sqrtf(block_sum<float>(w * w, red));
    if (own) {
      QT[r] = w * inv;
      Q[(size_t)r * ld] = w * inv;
    }
    __syncthreads();
  }
  // one classical Gram-Schmidt pass of w against q_0..q_j; returns h_j
  auto cgs = [&](int j) -> float {
    if (own) ws[r] = w;
    __syncthreads();
    const int jr = (j + 4) & ~3;  // q_0..q_j rounded up to whole float4s
    if (tid <= j) {
      const float4* qk = reinterpret_cast<const float4*>(QT + (size_t)tid * ld);
      const float4* wv = reinterpret_cast<const float4*>(ws);
      float s0 = 0.f, s1 = 0.f;
      for (int c4 = 0; c4 < np4; ++c4) {
        const float4 x = qk[c4], y = wv[c4];
        s0 = fmaf(x.x, y.x, fmaf(x.y, y.y, s0));
        s1 = fmaf(x.z, y.z, fmaf(x.w, y.w, s1));
      }
      hs[tid] = s0 + s1;
    } else if (tid < jr) {
      hs[tid] = 0.f;
    }
    __syncthreads();
    if (own) {
      const float4* qr = reinterpret_cast<const float4*>(Q + (size_t)r * ld);
      const float4* hv = reinterpret_cast<const float4*>(hs);
      float s0 = 0.f, s1 = 0.f;
      for (int k4 = 0; k4 < jr / 4; ++k4) {
        const float4 x = qr[k4], y = hv[k4];
        s0 = fmaf(x.x, y.x, fmaf(x.y, y.y, s0));
        s1 = fmaf(x.z, y.z, fmaf(x.w, y.w, s1));
      }
      w -= s0 + s1;
    }
    return hs[j];
  };

  for (int j = 0; j < m; ++j) {
    // w = A q_j
    if (own) {
      const float4* ar = reinterpret_cast<const float4*>(A + (size_t)r * ld);
      const float4* qj = reinterpret_cast<const float4*>(QT + (size_t)j * ld);
      float s0 = 0.f, s1 = 0.f;
      for (int c4 = 0; c4 < np4; ++c4) {
        const float4 x = ar[c4], y = qj[c4];
        s0 = fmaf(x.x, y.x, fmaf(x.y, y.y, s0));
        s1 = fmaf(x.z, y.z, fmaf(x.w, y.w, s1));
      }
      w = s0 + s1;
    }
    float al = cgs(j);
    __syncthreads();  // hs is rewritten by the second pass
    al += cgs(j);
    if (tid == 0) ta[j] = al;
    const float bnorm = sqrtf(block_sum<float>(w * w, red));
    if (j == m - 1) break;
    if (j + 1 >= kLanczosFirstCheck(K) && (j + 1 - kLanczosFirstCheck(K)) % kLanczosCheckEvery == 0) {
      // early stop once the top-K Ritz pairs have converged
      if (tid == 0) tb[j] = float(0);
      __syncthreads();
      if (lanczos_converged<float, 128>(a, sh_ck, j + 1, ta, tb, tb2, a.tri, bnorm, fro, eps, &conv_flag)) {
        m = j + 1;
        conv = true;
        break;
      }
    }
    if (bnorm > 100.f * eps * fro) {
      if (tid == 0) tb[j] = bnorm;
      const float inv = 1.f / bnorm;
      if (own) {
        QT[(size_t)(j + 1) * ld + r] = w * inv;
        Q[(size_t)r * ld + j + 1] = w * inv;
      }
    } else {
      // invariant subspace: continue with a fresh vector orthogonal to q_0..q_j
      if (tid == 0) tb[j] = 0.f;
      w = own ? hash_unit<float>(j + 2, r) : 0.f;
      cgs(j);
      __syncthreads();
      cgs(j);
      const float n2 = block_sum<float>(w * w, red);
      const float inv = n2 > 0.f ? 1.f / sqrtf(n2) : 0.f;
      if (own) {
        QT[(size_t)(j + 1) * ld + r] = w * inv;
        Q[(size_t)r * ld + j + 1] = w * inv;
      }
    }
    __syncthreads();
  }
  if (tid == 0) tb[m - 1] = 0.f;
  __syncthreads();
  if (a.clk && tid == 0) a.clk[1] = clock64();

  const EigSmem<float> sh{red, lo_s, hi_s, lam_s, inv_sig, cnt_s, mn_s, mx_s, b2_s};
  // a successful early-stop check has solved this very T_m into a.tri already
  const float* trix = conv ? a.tri : tri;
  if (!conv) eig_tridiag_topk<float>(a, sh, m, ta, tb, tb2, tri, fro, eps);
  // ---- X = Q S (row r of X from row r of Q)
  for (int idx = tid; idx < n * K; idx += NT) {
    const int rr = idx / K, k = idx - rr * K;
    const float* x = trix + (size_t)k * 6 * m + 5 * m;
    const float* qr = Q + (size_t)rr * ld;
    float s0 = 0.f, s1 = 0.f;
    int j = 0;
    for (; j + 1 < m; j += 2) {
      s0 = fmaf(qr[j], x[j], s0);
      s1 = fmaf(qr[j + 1], x[j + 1], s1);
    }
    if (j < m) s0 = fmaf(qr[j], x[j], s0);
    Xs[idx] = s0 + s1;
  }
  __syncthreads();
  if (a.clk && tid == 0) a.clk[4] = clock64();
  eig_finish<float>(a, sh, n, Xs, Cm, Rm);
}

// ------------------------------------------------------------------ back-projection
template <typename T, int KM>
__global__ void __launch_bounds__(256) k_backproj(const T* __restrict__ Z, int R, int Khat, const T* __restrict__ Vs,
                                                  int K, T* __restrict__ U) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x) {
    T acc[KM];
#pragma unroll
    for (int k = 0; k < KM; ++k) acc[k] = T(0);
    const T* z = Z + (int64_t)r * Khat;
    for (int c = 0; c < Khat; ++c) {
      const T zc = z[c];
      const T* vr = Vs + (int64_t)c * K;
#pragma unroll
      for (int k = 0; k < KM; ++k)
        if (k < K) acc[k] = fma(zc, __ldg(vr + k), acc[k]);
    }
#pragma unroll
    for (int k = 0; k < KM; ++k)
      if (k < K) U[(int64_t)r * K + k] = acc[k];
  }
}

// Tiled back-projection: a tile of 128 rows of Z is copied with coalesced
// 16-byte loads into shared memory (row stride Khat+1 words, so the per-thread
// row reads are conflict free), V Sigma^-1 sits in shared memory with rows
// padded to 16 bytes (vector reads), and each thread forms one row of U = Z Vs.
// With GRAM the thread also accumulates u u^T (upper triangle) over its rows
// and each block writes an FP64 partial of U^T U (the first CholeskyQR Gram).
template <typename T, int KM, bool GRAM>
__global__ void __launch_bounds__(128) k_backproj_tile(const T* __restrict__ Z, int R, int Khat,
                                                       const T* __restrict__ Vs, int K, T* __restrict__ U,
                                                       double* __restrict__ Cpart) {
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int NP = GRAM ? KM * (KM + 1) / 2 : 1;
  constexpr int W = 16 / sizeof(T);
  constexpr int KP = (KM + W - 1) / W * W;  // padded row of Vs
  using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  __shared__ T wsum[4][NP];
  T* vs = (T*)smraw;             // Khat x KP
  T* tile = vs + Khat * KP;      // 128 x (Khat + 1)
  const int ld = Khat + 1;
  const int tid = threadIdx.x;
  for (int i = tid; i < Khat * KP; i += 128) {
    const int cc = i / KP, k = i - cc * KP;
    vs[i] = k < K ? Vs[cc * K + k] : T(0);
  }
  T g[NP];
#pragma unroll
  for (int q = 0; q < NP; ++q) g[q] = T(0);
  for (int r0 = blockIdx.x * 128; r0 < R; r0 += gridDim.x * 128) {
    __syncthreads();
    const int nr = min(128, R - r0);
    const T* src = Z + (int64_t)r0 * Khat;
    const int total = nr * Khat;
    if (Khat % W == 0) {
      const V* s4 = reinterpret_cast<const V*>(src);
      for (int e = tid; e < total / W; e += 128) {
        const V x = s4[e];
        const int f = e * W, r = f / Khat, cc = f - r * Khat;
        T* d = tile + r * ld + cc;
        if constexpr (sizeof(T) == 4) {
          d[0] = x.x; d[1] = x.y; d[2] = x.z; d[3] = x.w;
        } else {
          d[0] = x.x; d[1] = x.y;
        }
      }
    } else {
      for (int e = tid; e < total; e += 128) {
        const int r = e / Khat, cc = e - r * Khat;
        tile[r * ld + cc] = src[e];
      }
    }
    __syncthreads();
    if (tid < nr) {
      T u[KP];
#pragma unroll
      for (int k = 0; k < KP; ++k) u[k] = T(0);
      const T* zr = tile + tid * ld;
#pragma unroll 4
      for (int cc = 0; cc < Khat; ++cc) {
        const T z = zr[cc];
        const V* v = reinterpret_cast<const V*>(vs + cc * KP);
#pragma unroll
        for (int q = 0; q < KP / W; ++q) {
          const V x = v[q];
          if constexpr (sizeof(T) == 4) {
            u[4 * q + 0] = fma(z, x.x, u[4 * q + 0]);
            u[4 * q + 1] = fma(z, x.y, u[4 * q + 1]);
            u[4 * q + 2] = fma(z, x.z, u[4 * q + 2]);
            u[4 * q + 3] = fma(z, x.w, u[4 * q + 3]);
          } else {
            u[2 * q + 0] = fma(z, x.x, u[2 * q + 0]);
            u[2 * q + 1] = fma(z, x.y, u[2 * q + 1]);
          }
        }
      }
      T* ur = U + (int64_t)(r0 + tid) * K;
#pragma unroll
      for (int k = 0; k < KM; ++k)
        if (k < K) ur[k] = u[k];
      if (GRAM) {
        int q = 0;
#pragma unroll
        for (int x = 0; x < KM; ++x)
#pragma unroll
          for (int y = x; y < KM; ++y) {
            g[q] = fma(u[x], u[y], g[q]);
            ++q;
          }
      }
    }
  }
  if (GRAM) {
    const int lane = tid & 31, w = tid >> 5;
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      T v = g[q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) wsum[w][q] = v;
    }
    __syncthreads();
    for (int q = tid; q < NP; q += 128) {
      int x = 0, rem = q;
      while (rem >= KM - x) {
        rem -= KM - x;
        ++x;
      }
      const int y = x + rem;
      if (x < K && y < K) {
        const double sum = (double)wsum[0][q] + (double)wsum[1][q] + (double)wsum[2][q] + (double)wsum[3][q];
        Cpart[(int64_t)blockIdx.x * K * K + x * K + y] = sum;
        Cpart[(int64_t)blockIdx.x * K * K + y * K + x] = sum;
      }
    }
  }
}

// FP32 back-projection U = Z Vs (Vs = V Sigma^-1) fused with the first
// CholeskyQR Gram, with the tile stream in flight: each CTA walks 128-row tiles
// of Z (one contiguous span each), loaded by bulk async copies into two
// buffers while the other is consumed.  Thread r computes row r of the tile
// from 16-byte reads of its row (the unpadded 4 * Khat-byte stride keeps the
// eight lanes of each read phase on distinct banks) and broadcast reads of Vs.
// Waits are bounded; a timeout sets TK_DEV_ERR_TIMEOUT.
template <int KM>
__global__ void __launch_bounds__(128) k_backproj_bulk(const float* __restrict__ Z, int R, int Khat,
                                                       const float* __restrict__ Vs, int K, float* __restrict__ U,
                                                       double* __restrict__ Cpart, int* err, int cap) {
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int NP = KM * (KM + 1) / 2;
  constexpr int KP = (KM + 3) / 4 * 4;
  __shared__ float wsum[4][NP];
  __shared__ __align__(8) uint64_t full[2];
  __shared__ int s_fail;
  float* vs = (float*)smraw;        // Khat x KP
  float* tiles = vs + Khat * KP;    // 2 x 128 x Khat
  const int tid = threadIdx.x;
  const int ntile = (R + 127) / 128;
  for (int i = tid; i < Khat * KP; i += 128) {
    const int cc = i / KP, k = i - cc * KP;
    vs[i] = k < K ? Vs[cc * K + k] : 0.f;
  }
  if (tid == 0) {
    s_fail = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(&full[0])), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(&full[1])), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  __syncthreads();
  int issued = 0;  // thread 0: tiles issued
  auto issue = [&](int i) {
    const int t = blockIdx.x + i * gridDim.x;
    if (t >= ntile) return;
    const int rows = min(128, R - t * 128);
    const unsigned bar = (unsigned)__cvta_generic_to_shared(&full[i & 1]);
    const unsigned bytes = (unsigned)(rows * Khat * 4);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     (unsigned)__cvta_generic_to_shared(tiles + (size_t)(i & 1) * 128 * Khat)),
                 "l"(Z + (int64_t)t * 128 * Khat), "r"(bytes), "r"(bar)
                 : "memory");
    issued = i + 1;
  };
  // bounded by ~4e9 cycles and, if pcap > 0, by pcap polls; pcap < 0 abandons
  // the wait at once (fault injection)
  auto wait_full = [&](int i, int pcap) -> bool {
    if (pcap < 0) return false;
    const unsigned bar = (unsigned)__cvta_generic_to_shared(&full[i & 1]);
    const unsigned par = (unsigned)((i >> 1) & 1);
    uint32_t done = 0;
    const long long t0 = clock64();
    for (int polls = 1; !done; ++polls) {
      asm volatile(
          "{\n .reg .pred P1;\n mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n selp.b32 %0, 1, 0, P1;\n}\n"
          : "=r"(done)
          : "r"(bar), "r"(par)
          : "memory");
      if (!done && (clock64() - t0 > 4000000000LL || (pcap > 0 && polls >= pcap))) return false;
    }
    return true;
  };
  if (tid == 0) {
    issue(0);
    issue(1);
  }
  float g[NP];
#pragma unroll
  for (int q = 0; q < NP; ++q) g[q] = 0.f;
  int i = 0;
  for (; blockIdx.x + i * gridDim.x < ntile; ++i) {
    const int t = blockIdx.x + i * gridDim.x;
    if (!wait_full(i, cap)) atomicOr(&s_fail, 1);
    __syncthreads();
    if (s_fail) break;
    const int nr = min(128, R - t * 128);
    if (tid < nr) {
      float u[KP];
#pragma unroll
      for (int k = 0; k < KP; ++k) u[k] = 0.f;
      const float4* zr = reinterpret_cast<const float4*>(tiles + (size_t)(i & 1) * 128 * Khat + (size_t)tid * Khat);
#pragma unroll 2
      for (int c4 = 0; c4 < Khat / 4; ++c4) {
        const float4 z = zr[c4];
        const float zz[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float4* v = reinterpret_cast<const float4*>(vs + (size_t)(4 * c4 + e) * KP);
#pragma unroll
          for (int q = 0; q < KP / 4; ++q) {
            const float4 x = v[q];
            u[4 * q + 0] = fmaf(zz[e], x.x, u[4 * q + 0]);
            u[4 * q + 1] = fmaf(zz[e], x.y, u[4 * q + 1]);
            u[4 * q + 2] = fmaf(zz[e], x.z, u[4 * q + 2]);
            u[4 * q + 3] = fmaf(zz[e], x.w, u[4 * q + 3]);
          }
        }
      }
      float* ur = U + ((int64_t)t * 128 + tid) * K;
#pragma unroll
      for (int k = 0; k < KM; ++k)
        if (k < K) ur[k] = u[k];
      int q = 0;
#pragma unroll
      for (int x = 0; x < KM; ++x)
#pragma unroll
        for (int y = x; y < KM; ++y) {
          g[q] = fmaf(u[x], u[y], g[q]);
          ++q;
        }
    }
    __syncthreads();  // buffer i & 1 is free
    if (tid == 0) issue(i + 2);
  }
  if (s_fail && tid == 0) {
    for (int x = i; x < issued; ++x) wait_full(x, 0);  // copies in flight land before the CTA exits
    atomicOr(err, TK_DEV_ERR_TIMEOUT);
  }
  const int lane = tid & 31, w = tid >> 5;
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    float v = g[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) wsum[w][q] = v;
  }
  __syncthreads();
  for (int q = tid; q < NP; q += 128) {
    int x = 0, rem = q;
    while (rem >= KM - x) {
      rem -= KM - x;
      ++x;
    }
    const int y = x + rem;
    if (x < K && y < K) {
      const double sum = (double)wsum[0][q] + (double)wsum[1][q] + (double)wsum[2][q] + (double)wsum[3][q];
      Cpart[(int64_t)blockIdx.x * K * K + x * K + y] = sum;
      Cpart[(int64_t)blockIdx.x * K * K + y * K + x] = sum;
    }
  }
}

// ------------------------------------------------------------------ CholeskyQR2
// Per-block partial of (U M)^T (U M): batches of 64 rows are transformed into
// shared memory, each thread sums its (a,b) pairs over a batch in T and adds
// the batch sum into an FP64 accumulator.
template <typename T>
__global__ void __launch_bounds__(256) k_small_gram(const T* __restrict__ U, int R, int K, const double* __restrict__ M,
                                                    double* __restrict__ Cpart) {
  __shared__ T rows[64][TK_MAXK + 1];
  __shared__ T raw[64][TK_MAXK + 1];
  __shared__ T Ms[TK_MAXK][TK_MAXK];
  __shared__ unsigned char pa[TK_MAXK * (TK_MAXK + 1) / 2], pb[TK_MAXK * (TK_MAXK + 1) / 2];
  const int tid = threadIdx.x;
  const int npairs = K * (K + 1) / 2;
  if (tid == 0) {
    int q = 0;
    for (int x = 0; x < K; ++x)
      for (int y = x; y < K; ++y) {
        pa[q] = (unsigned char)x;
        pb[q] = (unsigned char)y;
        ++q;
      }
  }
  if (M)
    for (int i = tid; i < K * K; i += 256) Ms[i / K][i % K] = (T)M[i];
  double acc[3] = {0.0, 0.0, 0.0};
  const int nbatch = (int)tk_ceil_div(R, 64);
  __syncthreads();
  for (int b = blockIdx.x; b < nbatch; b += gridDim.x) {
    const int r0 = b * 64;
    for (int i = tid; i < 64 * K; i += 256) {  // raw rows, coalesced
      const int r = i / K, k = i - r * K;
      raw[r][k] = (r0 + r < R) ? U[(int64_t)r0 * K + i] : T(0);
    }
    __syncthreads();
    for (int i = tid; i < 64 * K; i += 256) {
      const int r = i / K, k = i - r * K;
      T v;
      if (M) {
        v = T(0);
        for (int j = 0; j <= k; ++j) v = fma(raw[r][j], Ms[j][k], v);  // M upper triangular
      } else {
        v = raw[r][k];
      }
      rows[r][k] = v;
    }
    __syncthreads();
    for (int u = 0; u < 3; ++u) {
      const int pi = tid + 256 * u;
      if (pi >= npairs) break;
      const int x = pa[pi], y = pb[pi];
      T s = T(0);
#pragma unroll 8
      for (int r = 0; r < 64; ++r) s = fma(rows[r][x], rows[r][y], s);
      acc[u] += (double)s;
    }
    __syncthreads();
  }
  for (int u = 0; u < 3; ++u) {
    const int pi = tid + 256 * u;
    if (pi >= npairs) break;
    const int x = pa[pi], y = pb[pi];
    Cpart[(int64_t)blockIdx.x * K * K + x * K + y] = acc[u];
    Cpart[(int64_t)blockIdx.x * K * K + y * K + x] = acc[u];
  }
}

// Second CholeskyQR Gram, thread per row: v = u M (M upper triangular),
// v v^T accumulated in registers over the thread's rows; warp sums, then one
// FP64 partial per block.
template <typename T, int KM>
__global__ void __launch_bounds__(256) k_row_gram(const T* __restrict__ U, int R, int K, const double* __restrict__ M,
                                                  double* __restrict__ Cpart) {
  constexpr int NP = KM * (KM + 1) / 2;
  __shared__ T Ms[KM][KM];
  __shared__ T wsum[8][NP];
  const int tid = threadIdx.x;
  for (int i = tid; i < KM * KM; i += 256) {
    const int r = i / KM, cc = i - r * KM;
    Ms[r][cc] = (r < K && cc < K) ? (T)M[r * K + cc] : T(0);
  }
  __syncthreads();
  T g[NP];
#pragma unroll
  for (int q = 0; q < NP; ++q) g[q] = T(0);
  for (int r = blockIdx.x * 256 + tid; r < R; r += gridDim.x * 256) {
    T u[KM], v[KM];
#pragma unroll
    for (int k = 0; k < KM; ++k) u[k] = k < K ? U[(int64_t)r * K + k] : T(0);
#pragma unroll
    for (int k = 0; k < KM; ++k) {
      T acc = T(0);
#pragma unroll
      for (int j = 0; j <= k; ++j) acc = fma(u[j], Ms[j][k], acc);
      v[k] = acc;
    }
    int q = 0;
#pragma unroll
    for (int x = 0; x < KM; ++x)
#pragma unroll
      for (int y = x; y < KM; ++y) {
        g[q] = fma(v[x], v[y], g[q]);
        ++q;
      }
  }
  const int lane = tid & 31, w = tid >> 5;
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    T x = g[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) wsum[w][q] = x;
  }
  __syncthreads();
  for (int q = tid; q < NP; q += 256) {
    int x = 0, rem = q;
    while (rem >= KM - x) {
      rem -= KM - x;
      ++x;
    }
    const int y = x + rem;
    if (x < K && y < K) {
      double sum = 0.0;
      for (int ww = 0; ww < 8; ++ww) sum += (double)wsum[ww][q];
      Cpart[(int64_t)blockIdx.x * K * K + x * K + y] = sum;
      Cpart[(int64_t)blockIdx.x * K * K + y * K + x] = sum;
    }
  }
}

// C = sum of the block partials (8 lanes per entry, fixed shuffle tree);
// C = R^T R; out = prev * R^-1.  The factorisation runs on warp 0.
__global__ void __launch_bounds__(1024) k_chol_inv(const double* __restrict__ Cpart, int nblk, int K,
                                                   const double* prev, double* out, int* err) {
  __shared__ double C[TK_MAXK][TK_MAXK + 1];
  __shared__ double Ri[TK_MAXK][TK_MAXK + 1];
  const int tid = threadIdx.x, lane = tid & 31;
  const int part = tid & 7;
  for (int base = 0; base < K * K; base += 1024 >> 3) {  // uniform trip count for every lane
    const int e = base + (tid >> 3);
    double s = 0.0;
    if (e < K * K)
      for (int b = part; b < nblk; b += 8) s += Cpart[(int64_t)b * K * K + e];
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    s += __shfl_xor_sync(0xffffffffu, s, 4);
    if (part == 0 && e < K * K) C[e / K][e % K] = s;
  }
  __syncthreads();
  if (tid >= 32) return;
  // Cholesky C = L L^T in place (lower); R = L^T
  bool bad = false;
  for (int j = 0; j < K; ++j) {
    double d = C[j][j];
    if (!(d > 0.0) || !isfinite(d)) bad = true;
    d = (d > 0.0 && isfinite(d)) ? sqrt(d) : 1.0;
    __syncwarp();
    if (lane == j) C[j][j] = d;
    if (lane > j && lane < K) C[lane][j] /= d;
    __syncwarp();
    if (lane > j && lane < K)
      for (int k = j + 1; k <= lane; ++k) C[lane][k] -= C[lane][j] * C[k][j];
    __syncwarp();
  }
  if (bad && lane == 0) atomicOr(err, TK_DEV_ERR_NUMERIC);
  // Ri = R^-1 (upper): column `lane` solves R x = e_lane by back substitution, R[i][k] = C[k][i]
  if (lane < K) {
    for (int i = K - 1; i >= 0; --i) {
      double s = (i == lane) ? 1.0 : 0.0;
      for (int k = i + 1; k < K; ++k) s -= C[k][i] * Ri[k][lane];
      Ri[i][lane] = (i <= lane) ? s / C[i][i] : 0.0;
    }
  }
  __syncwarp();
  for (int i = lane; i < K * K; i += 32) {
    const int r = i / K, cc = i % K;
    double s;
    if (prev) {
      s = 0.0;
      for (int k = 0; k < K; ++k) s = fma(prev[r * K + k], Ri[k][cc], s);
    } else {
      s = Ri[r][cc];
    }
    out[i] = s;
  }
}

template <typename T>
struct Cand {
  T a;    // |value|
  int r;  // compact row (increasing slice id)
  T v;    // signed value
};
template <typename T>
__device__ __forceinline__ bool better(const Cand<T>& x, const Cand<T>& y) {
  return x.a > y.a || (x.a == y.a && x.r < y.r);
}

// U <- U M (row by row) and per-block best (|value|, lowest row) per column;
// KM >= K is the compile-time bound that keeps the row in registers.
template <typename T, int KM>
__global__ void __launch_bounds__(256) k_apply(T* __restrict__ U, int R, int K, const double* __restrict__ M,
                                               double* __restrict__ colbest) {
  __shared__ T Ms[KM][KM];
  __shared__ Cand<T> wbest[8][KM];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  for (int i = tid; i < KM * KM; i += 256) {
    const int r = i / KM, cc = i - r * KM;
    Ms[r][cc] = (r < K && cc < K) ? (T)M[r * K + cc] : T(0);
  }
  __syncthreads();
  Cand<T> best[KM];
#pragma unroll
  for (int k = 0; k < KM; ++k) best[k] = Cand<T>{T(-1), 0x7fffffff, T(0)};
  for (int r = blockIdx.x * 256 + tid; r < R; r += gridDim.x * 256) {
    T u[KM];
#pragma unroll
    for (int k = 0; k < KM; ++k) u[k] = k < K ? U[(int64_t)r * K + k] : T(0);
#pragma unroll
    for (int k = 0; k < KM; ++k) {
      T s = T(0);
#pragma unroll
      for (int j = 0; j <= k; ++j) s = fma(u[j], Ms[j][k], s);  // M upper triangular
      if (k < K) {
        U[(int64_t)r * K + k] = s;
        const Cand<T> c{fabs(s), r, s};
        if (better(c, best[k])) best[k] = c;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < KM; ++k) {
    Cand<T> c = best[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      Cand<T> d;
      d.a = __shfl_down_sync(0xffffffffu, c.a, o);
      d.r = __shfl_down_sync(0xffffffffu, c.r, o);
      d.v = __shfl_down_sync(0xffffffffu, c.v, o);
      if (better(d, c)) c = d;
    }
    if (lane == 0) wbest[w][k] = c;
  }
  __syncthreads();
  if (tid < K) {
    Cand<T> c = wbest[0][tid];
    for (int ww = 1; ww < 8; ++ww)
      if (better(wbest[ww][tid], c)) c = wbest[ww][tid];
    double* o = colbest + ((int64_t)blockIdx.x * K + tid) * 3;
    o[0] = (double)c.a;
    o[1] = (double)c.r;
    o[2] = (double)c.v;
  }
}

__global__ void k_signs(const double* colbest, int nblk, int K, double* sign) {
  const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (k >= K) return;
  Cand<double> c{-1.0, 0x7fffffff, 0.0};
  for (int b = lane; b < nblk; b += 32) {
    const double* o = colbest + ((int64_t)b * K + k) * 3;
    const Cand<double> d{o[0], (int)o[1], o[2]};
    if (better(d, c)) c = d;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Cand<double> d;
    d.a = __shfl_xor_sync(0xffffffffu, c.a, o);
    d.r = __shfl_xor_sync(0xffffffffu, c.r, o);
    d.v = __shfl_xor_sync(0xffffffffu, c.v, o);
    if (better(d, c)) c = d;
  }
  if (lane == 0) sign[k] = c.v < 0.0 ? -1.0 : 1.0;
}

// F[row_id[r]][k] = sign[k] * U[r][k], thread per row (KM >= K).
template <typename T, int KM>
__global__ void k_scatter_rows(const T* __restrict__ U, int R, int K, const int32_t* __restrict__ row_id,
                               const double* __restrict__ sign, T* __restrict__ F, int ldF) {
  T sg[KM];
#pragma unroll
  for (int k = 0; k < KM; ++k) sg[k] = k < K ? (T)sign[k] : T(0);
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x) {
    const T* u = U + (int64_t)r * K;
    T* f = F + (int64_t)row_id[r] * ldF;
#pragma unroll
    for (int k = 0; k < KM; ++k)
      if (k < K) f[k] = sg[k] * u[k];
  }
}

template <typename Kern>
void set_tile_attr(Kern k, size_t bytes) {
  TK_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max<size_t>(bytes, 48 * 1024)));
}

constexpr size_t kEigSmallSmemMax = 200 * 1024;

template <typename T>
void setup_eig_attr() {
  static bool done = false;
  if (!done) {
    TK_CUDA(cudaFuncSetAttribute(k_eig<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024));
    TK_CUDA(cudaFuncSetAttribute(k_eig_small<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEigSmallSmemMax));
    TK_CUDA(cudaFuncSetAttribute(k_eig_v4, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEigSmallSmemMax));
    done = true;
  }
}

template <typename T>
void factor_impl(tucker_ctx* c, int n, const void* Zv, void* F_out, int ldF_out, const int32_t* row_map,
                 double* sigma_out, cudaStream_t s) {
  const tk_mode& md = c->mode[n];
  tk_fuws* ws = &c->fu[n];
  const int R = md.R, Khat = md.Khat, K = c->K[n];
  const T* Z = (const T*)Zv;
  const int sms = c->sm_count;

  // ---- Gram W = Z^T Z (exact route), or the Lanczos bidiagonalisation of Z
  // with W = B^T B of its m x m bidiagonal (the paper's route)
  int eig_n = Khat;
  tk_phase_begin(c, PH_GRAM, s);
  bool gram_done = false;
  if (c->svd_lanczos) {
    eig_n = tk_lanczos_bidiag(c, n, Z, s);
    gram_done = true;
  }
  if constexpr (sizeof(T) == 4) {
    if (gram_done) {
    } else if (!c->gram_bf16 && tk_gram_tc_supported(Khat) && ((uintptr_t)Z % 16 == 0)) {
      // tensor cores: per-CTA partials, reduced and symmetrised in FP64
      tk_gram_tc(c, (const float*)Z, R, Khat, (float*)ws->Wpart, ws->Wpart_elems, ws->W, s);
      tk_launched(c, PH_GRAM, 2);
      gram_done = true;
    } else if ((Khat > 128 || c->gram_bf16) && tk_gram_tiles_supported(Khat) && ((uintptr_t)Z % 16 == 0) &&
               (size_t)tk_gram_tiles_splits(c, Khat, R) * tk_gram_tiles_pairs(Khat) * 128 * 128 <= ws->Wpart_elems &&
               tk_gram_tiles_pairs(Khat) <= ws->gram_tiles_cap) {
      // tensor cores, 128 x 128 blocks of W
      tk_gram_tiles(c, (const float*)Z, R, Khat, (float*)ws->Wpart, ws->gram_tiles, ws->W, c->gram_bf16, s);
      tk_launched(c, PH_GRAM, 2);
      gram_done = true;
    }
  }
  if (!gram_done) {
    const int TM = (sizeof(T) == 4 && Khat > 64) ? 128 : 64;
    const int tpd = (int)tk_ceil_div(Khat, TM);
    const int ntiles = tpd * (tpd + 1) / 2;
    int nsplit = (int)std::max<int64_t>(1, std::min<int64_t>(tk_ceil_div(R, 64), tk_ceil_div(2 * sms, ntiles)));
    while ((size_t)nsplit * ntiles * TM * TM > ws->Wpart_elems && nsplit > 1) --nsplit;
    const int rps = (int)tk_ceil_div(R, nsplit);
    std::vector<int2> tl;
    for (int i = 0; i < tpd; ++i)
      for (int j = i; j < tpd; ++j) tl.push_back(make_int2(i, j));
    if ((int)tl.size() > ws->gram_tiles_cap) tk_throw(TUCKER_ERR_STATE, "internal: Gram tile list too long");
    int2* dtiles = ws->gram_tiles;
    TK_CUDA(cudaMemcpyAsync(dtiles, tl.data(), tl.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
    dim3 grid(ntiles, nsplit);
    if constexpr (sizeof(T) == 4) {
      if (TM == 128) k_gram<T, 128><<<grid, 256, 0, s>>>(Z, R, Khat, dtiles, ntiles, rps, (T*)ws->Wpart);
      else k_gram<T, 64><<<grid, 256, 0, s>>>(Z, R, Khat, dtiles, ntiles, rps, (T*)ws->Wpart);
    } else {
      k_gram<T, 64><<<grid, 256, 0, s>>>(Z, R, Khat, dtiles, ntiles, rps, (T*)ws->Wpart);
    }
    TK_CUDA(cudaGetLastError());
    const unsigned g2 = (unsigned)std::min<int64_t>(tk_ceil_div((int64_t)Khat * Khat * 8, 256), 8192);
    k_gram_reduce<T><<<g2, 256, 0, s>>>((const T*)ws->Wpart, nsplit, ntiles, tpd, TM, Khat, ws->W);
    TK_CUDA(cudaGetLastError());
    tk_launched(c, PH_GRAM, 2);
  }
  tk_phase_end(c, s);

  // ---- eigensolve
  tk_phase_begin(c, PH_EIG, s);
  {
    setup_eig_attr<T>();
    EigArgs<T> a{};
    a.W = ws->W;
    a.n = eig_n;
    a.K = K;
    a.gA = (T*)ws->eigA;
    a.gQ = (T*)ws->eigV;
    const size_t mat = (size_t)2 * eig_n * eig_n * sizeof(T);
    const size_t work = (size_t)5 * eig_n * sizeof(T) + 64;
    a.use_smem = (mat + work) <= 150 * 1024;
    const size_t shm = (a.use_smem ? mat : 0) + work;
    const size_t shm_small = eig_small_smem<T>(eig_n, K);
    const bool small = eig_n <= 2 * kEigSmallThreads && shm_small <= kEigSmallSmemMax;
    a.polish = c->prec == TUCKER_FP32;
    a.X = ws->eigX;
    a.Y = ws->eigX + (size_t)Khat * K;
    a.ab = ws->eigAB;
    a.tri = (T*)ws->eigTri;
    a.Vout = ws->V;
    a.sigma = ws->sigma;
    a.Vs = (T*)ws->Vs;
    a.err = c->err;
    bool v4 = false;
    if constexpr (sizeof(T) == 4) {
      const size_t shm_v4 = eig_v4_smem(eig_n, K);
      if (eig_n <= kEigV4MaxN && shm_v4 <= kEigSmallSmemMax) {
        k_eig_v4<<<1, kEigSmallThreads, shm_v4, s>>>(a);
        v4 = true;
      }
    }
    if (v4) {
    } else if (small) k_eig_small<T><<<1, kEigSmallThreads, shm_small, s>>>(a);
    else k_eig<T><<<1, 1024, shm, s>>>(a);
    TK_CUDA(cudaGetLastError());
    tk_launched(c, PH_EIG);
    // Lanczos route: the eigenvectors of B^T B are B's right singular vectors Q;
    // the right singular vectors of Z are V_K = V_lanczos Q_K
    if (c->svd_lanczos) {
      tk_lanczos_vk(c, n, eig_n, s);
      tk_launched(c, PH_EIG);
    }
  }
  tk_phase_end(c, s);

  // ---- back-projection + CholeskyQR2 + signs + scatter
  tk_phase_begin(c, PH_BACKPROJ, s);
  {
    const T* Vs = (const T*)ws->Vs;
    T* U = (T*)ws->U;
    double* R1 = ws->Rinv;
    double* R2 = ws->Rinv + TK_MAXK * TK_MAXK;
    double* sign = ws->Rinv + 2 * TK_MAXK * TK_MAXK;
    const size_t tshm = ((size_t)Khat * 16 + (size_t)128 * (Khat + 1)) * sizeof(T);
    int nblk = (int)std::max<int64_t>(1, std::min<int64_t>(tk_ceil_div(R, 128), 4 * sms));
    const size_t bshm = ((size_t)Khat * 12 + (size_t)2 * 128 * Khat) * 4;
    bool bulk = false;
    if constexpr (sizeof(T) == 4) {
      bulk = K <= 12 && Khat % 4 == 0 && ((uintptr_t)Z % 16) == 0 && bshm <= 110 * 1024;
    }
    if (bulk) {
      if constexpr (sizeof(T) == 4) {
        nblk = (int)std::max<int64_t>(1, std::min<int64_t>(tk_ceil_div(R, 128), 2 * sms));
        if (K <= 8) {
          set_tile_attr(k_backproj_bulk<8>, bshm);
          k_backproj_bulk<8><<<nblk, 128, bshm, s>>>(Z, R, Khat, Vs, K, U, ws->Cpart, c->err, c->wait_cap);
        } else {
          set_tile_attr(k_backproj_bulk<12>, bshm);
          k_backproj_bulk<12><<<nblk, 128, bshm, s>>>(Z, R, Khat, Vs, K, U, ws->Cpart, c->err, c->wait_cap);
        }
        TK_CUDA(cudaGetLastError());
      }
    } else if (K <= (sizeof(T) == 4 ? 16 : 12) && tshm <= 200 * 1024) {
      // tiled back-projection fused with the first CholeskyQR Gram
      if (K <= 8) {
        set_tile_attr(k_backproj_tile<T, 8, true>, tshm);
        k_backproj_tile<T, 8, true><<<nblk, 128, tshm, s>>>(Z, R, Khat, Vs, K, U, ws->Cpart);
      } else if (K <= 12) {
        set_tile_attr(k_backproj_tile<T, 12, true>, tshm);
        k_backproj_tile<T, 12, true><<<nblk, 128, tshm, s>>>(Z, R, Khat, Vs, K, U, ws->Cpart);
      } else if constexpr (sizeof(T) == 4) {
        set_tile_attr(k_backproj_tile<T, 16, true>, tshm);
        k_backproj_tile<T, 16, true><<<nblk, 128, tshm, s>>>(Z, R, Khat, Vs, K, U, ws->Cpart);
      }
      TK_CUDA(cudaGetLastError());
    } else {
      const unsigned gb = (unsigned)std::max<int64_t>(1, std::min<int64_t>(tk_ceil_div(R, 256), 8 * sms));
      if (K <= 8) k_backproj<T, 8><<<gb, 256, 0, s>>>(Z, R, Khat, Vs, K, U);
      else if (K <= 16) k_backproj<T, 16><<<gb, 256, 0, s>>>(Z, R, Khat, Vs, K, U);
      else k_backproj<T, 32><<<gb, 256, 0, s>>>(Z, R, Khat, Vs, K, U);
      TK_CUDA(cudaGetLastError());
      nblk = (int)std::max<int64_t>(1, std::min<int64_t>(tk_ceil_div(R, 64), 2 * sms));
      k_small_gram<T><<<nblk, 256, 0, s>>>(U, R, K, nullptr, ws->Cpart);
    }
    k_chol_inv<<<1, 1024, 0, s>>>(ws->Cpart, nblk, K, nullptr, R1, c->err);
    nblk = (int)std::max<int64_t>(1, std::min<int64_t>(tk_ceil_div(R, 64), 2 * sms));
    if (K <= (sizeof(T) == 4 ? 12 : 8)) {
      nblk = (int)std::max<int64_t>(1, std::min<int64_t>(tk_ceil_div(R, 256), 4 * sms));
      if (K <= 8) k_row_gram<T, 8><<<nblk, 256, 0, s>>>(U, R, K, R1, ws->Cpart);
      else if constexpr (sizeof(T) == 4) k_row_gram<T, 12><<<nblk, 256, 0, s>>>(U, R, K, R1, ws->Cpart);
    } else {
      k_small_gram<T><<<nblk, 256, 0, s>>>(U, R, K, R1, ws->Cpart);
    }
    k_chol_inv<<<1, 1024, 0, s>>>(ws->Cpart, nblk, K, R1, R2, c->err);
    const int nab = (int)std::max<int64_t>(1, std::min<int64_t>(tk_ceil_div(R, 256), 2 * sms));
    const unsigned gs = (unsigned)std::max<int64_t>(1, std::min<int64_t>(tk_ceil_div(R, 256), 8 * sms));
    auto tail = [&](auto km) {
      constexpr int KM = decltype(km)::value;
      k_apply<T, KM><<<nab, 256, 0, s>>>(U, R, K, R2, ws->colbest);
      k_signs<<<1, 32 * K, 0, s>>>(ws->colbest, nab, K, sign);
      TK_CUDA(cudaMemsetAsync(F_out, 0, (size_t)c->L[n] * ldF_out * sizeof(T), s));
      k_scatter_rows<T, KM><<<gs, 256, 0, s>>>(U, R, K, row_map, sign, (T*)F_out, ldF_out);
    };
    if (K <= 8) tail(std::integral_constant<int, 8>());
    else if (K <= 12) tail(std::integral_constant<int, 12>());
    else if (K <= 16) tail(std::integral_constant<int, 16>());
    else tail(std::integral_constant<int, 32>());
    TK_CUDA(cudaGetLastError());
    tk_launched(c, PH_BACKPROJ, 8);
    if (sigma_out) TK_CUDA(cudaMemcpyAsync(sigma_out, ws->sigma, K * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  tk_phase_end(c, s);
}

}  // namespace

void tk_factor_update(tucker_ctx* c, int n, const void* Z, void* F_out, int ldF_out, const int32_t* row_map,
                      double* sigma_out, cudaStream_t s) {
  if (c->prec == TUCKER_FP32) factor_impl<float>(c, n, Z, F_out, ldF_out, row_map, sigma_out, s);
  else factor_impl<double>(c, n, Z, F_out, ldF_out, row_map, sigma_out, s);
}

// Per-mode factor-update workspace, sized for that mode.
void tk_alloc_fuws(tucker_ctx* c, int n) {
  const tk_mode& md = c->mode[n];
  tk_fuws& w = c->fu[n];
  const size_t esz = c->esz;
  const int Khat = md.Khat, K = c->K[n], sms = c->sm_count;
  const int TM = (esz == 4 && Khat > 64) ? 128 : 64;
  const int tpd = (int)tk_ceil_div(Khat, TM);
  const int ntiles = tpd * (tpd + 1) / 2;
  w.Wpart_elems = (size_t)(2 * sms + ntiles) * TM * TM;
  w.gram_tiles_cap = ntiles;
  if (esz == 4 && tk_gram_tiles_supported(Khat) && (Khat > 128 || c->gram_bf16)) {
    // tensor-core blocks: one 128 x 128 tile per (split, block pair)
    const size_t need = (size_t)tk_gram_tiles_splits(c, Khat, md.R) * tk_gram_tiles_pairs(Khat) * 128 * 128;
    w.Wpart_elems = std::max(w.Wpart_elems, need);
    w.gram_tiles_cap = std::max(ntiles, tk_gram_tiles_pairs(Khat));
  }
  w.Wpart = tk_alloc(c, w.Wpart_elems * esz);
  w.gram_tiles = (int2*)tk_alloc(c, (size_t)w.gram_tiles_cap * sizeof(int2));
  w.W = (double*)tk_alloc(c, (size_t)Khat * Khat * 8);
  w.eigA = tk_alloc(c, (size_t)Khat * Khat * esz);
  w.eigV = tk_alloc(c, (size_t)Khat * Khat * esz);
  w.eigX = (double*)tk_alloc(c, (size_t)2 * Khat * K * 8);
  w.eigAB = (double*)tk_alloc(c, (size_t)2 * Khat * 8);
  w.eigTri = tk_alloc(c, (size_t)6 * K * Khat * esz);
  w.Vs = tk_alloc(c, (size_t)Khat * K * esz);
  w.V = (double*)tk_alloc(c, (size_t)Khat * K * 8);
  w.sigma = (double*)tk_alloc(c, (size_t)TK_MAXK * 8);
  w.U = tk_alloc(c, (size_t)std::max(md.R, 1) * K * esz);
  w.Cpart = (double*)tk_alloc(c, (size_t)4 * sms * TK_MAXK * TK_MAXK * 8);
  w.Rinv = (double*)tk_alloc(c, (size_t)3 * TK_MAXK * TK_MAXK * 8);
  w.colbest = (double*)tk_alloc(c, (size_t)2 * sms * TK_MAXK * 3 * 8);
}
