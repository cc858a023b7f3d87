// New factor F~_n = leading K_n left singular vectors of Z_(n) (Fig. 1, "SVD").
//
//   W = Z^T Z            Gram over the R_n compact rows (split over rows, FP64 reduction in fixed order)
//   W V = V Lambda       cyclic-by-rounds Jacobi (Golub & Van Loan 8.5) in one CTA; the FP32
//                        context polishes the top-K subspace in FP64 (one subspace step + Rayleigh-Ritz)
//   U = Z V Sigma^-1     back-projection
//   U <- U R^-1 twice    CholeskyQR2 (Gram reductions, Cholesky and inverses in FP64)
//   signs                column's entry of largest magnitude (lowest slice id on a tie) made positive
//   F_n[row_id[r]] = U[r], rows of empty slices zero
#include <algorithm>

#include "tk_common.cuh"

namespace {

// ------------------------------------------------------------------ block sums
__device__ double block_sum_d(double v, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < nw; ++i) s += red[i];  // every thread, same order
  __syncthreads();
  return s;
}

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
  T acc[RT][RT];
#pragma unroll
  for (int i = 0; i < RT; ++i)
#pragma unroll
    for (int j = 0; j < RT; ++j) acc[i][j] = T(0);
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
  }
  T* out = Wpart + ((int64_t)sp * ntiles + t) * TM * TM;
#pragma unroll
  for (int i = 0; i < RT; ++i)
#pragma unroll
    for (int j = 0; j < RT; ++j) out[(ty + 16 * i) * TM + tx + 16 * j] = acc[i][j];
}

template <typename T>
__global__ void k_gram_reduce(const T* __restrict__ Wpart, int nsplit, int ntiles, int tpd, int TM, int Khat,
                              double* __restrict__ W) {
  const int64_t total = (int64_t)Khat * Khat;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(idx / Khat), j = (int)(idx - (int64_t)i * Khat);
    int ti = i / TM, tj = j / TM, ii = i - ti * TM, jj = j - tj * TM;
    if (ti > tj) {
      int x = ti; ti = tj; tj = x;
      x = ii; ii = jj; jj = x;
    }
    const int t = ti * tpd - ti * (ti - 1) / 2 + (tj - ti);
    double s = 0.0;
    for (int sp = 0; sp < nsplit; ++sp) s += (double)Wpart[((int64_t)sp * ntiles + t) * TM * TM + ii * TM + jj];
    W[idx] = s;
  }
}

// ------------------------------------------------------------------ Jacobi
template <typename T>
struct JacobiWork {
  T* cs;
  T* sn;
  int* pp;
  int* qq;
};

// Cyclic Jacobi by rounds: the round-robin ("circle") ordering pairs every
// index with every other once per sweep, n/2 disjoint rotations per round.
template <typename T>
__device__ void jacobi_block(T* A, T* V, int n, int max_sweeps, double tol, JacobiWork<T> wk, double* red) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int np = n + (n & 1), half = np / 2;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int idx = tid; idx < n * n; idx += nt) {
      const double v = (double)A[idx] * (double)A[idx];
      tot += v;
      if (idx / n != idx % n) off += v;
    }
    off = block_sum_d(off, red);
    tot = block_sum_d(tot, red);
    if (off <= tol * tol * tot) break;
    for (int r = 0; r < np - 1; ++r) {
      for (int k = tid; k < half; k += nt) {
        int p = k == 0 ? 0 : ((k - 1 + r) % (np - 1)) + 1;
        int q = ((np - 2 - k + r) % (np - 1)) + 1;
        if (p > q) {
          const int x = p; p = q; q = x;
        }
        T c = T(1), s = T(0);
        if (q < n) {
          const T apq = A[p * n + q];
          if (apq != T(0)) {
            const T app = A[p * n + p], aqq = A[q * n + q];
            const T tau = (aqq - app) / (T(2) * apq);
            const T tt = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + sqrt(T(1) + tau * tau));
            c = T(1) / sqrt(T(1) + tt * tt);
            s = tt * c;
          }
        }
        wk.cs[k] = c;
        wk.sn[k] = s;
        wk.pp[k] = p;
        wk.qq[k] = q < n ? q : p;
      }
      __syncthreads();
      for (int idx = tid; idx < half * n; idx += nt) {
        const int k = idx / n, j = idx - k * n;
        const T s = wk.sn[k];
        if (s == T(0)) continue;
        const T c = wk.cs[k];
        const int p = wk.pp[k], q = wk.qq[k];
        const T ap = A[p * n + j], aq = A[q * n + j];
        A[p * n + j] = c * ap - s * aq;
        A[q * n + j] = s * ap + c * aq;
      }
      __syncthreads();
      for (int idx = tid; idx < n * half; idx += nt) {
        const int i = idx / half, k = idx - i * half;
        const T s = wk.sn[k];
        if (s == T(0)) continue;
        const T c = wk.cs[k];
        const int p = wk.pp[k], q = wk.qq[k];
        const T ap = A[i * n + p], aq = A[i * n + q];
        A[i * n + p] = c * ap - s * aq;
        A[i * n + q] = s * ap + c * aq;
        const T vp = V[i * n + p], vq = V[i * n + q];
        V[i * n + p] = c * vp - s * vq;
        V[i * n + q] = s * vp + c * vq;
      }
      __syncthreads();
    }
  }
}

// Index of the largest diagonal entry not yet taken (lowest index on a tie).
template <typename T>
__device__ int block_argmax_diag(const T* A, int n, const unsigned char* taken, double* redv, int* redi) {
  double best = -INFINITY;
  int bi = n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    if (taken[i]) continue;
    const double v = (double)A[i * n + i];
    if (v > best || (v == best && i < bi)) {
      best = v;
      bi = i;
    }
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_down_sync(0xffffffffu, best, o);
    const int oi = __shfl_down_sync(0xffffffffu, bi, o);
    if (ov > best || (ov == best && oi < bi)) {
      best = ov;
      bi = oi;
    }
  }
  __syncthreads();
  if (lane == 0) {
    redv[w] = best;
    redi[w] = bi;
  }
  __syncthreads();
  double b = -INFINITY;
  int r = n;
  for (int i = 0; i < nw; ++i)
    if (redv[i] > b || (redv[i] == b && redi[i] < r)) {
      b = redv[i];
      r = redi[i];
    }
  __syncthreads();
  return r;
}

template <typename T>
struct EigArgs {
  const double* W;
  int n, K;
  T* gA;
  T* gV;
  int use_smem;
  int polish;
  int max_sweeps;
  double tol;
  double* X;     // n x K scratch
  double* Y;     // n x K scratch
  double* Vout;  // n x K
  double* sigma; // K
  T* Vs;         // n x K: Vout[:,k] / sigma_k in T
  int* err;
};

template <typename T>
__global__ void __launch_bounds__(1024) k_eig(const EigArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[32];
  __shared__ int redi[32];
  __shared__ double H[TK_MAXK * TK_MAXK];
  __shared__ double HV[TK_MAXK * TK_MAXK];
  __shared__ double hcs[TK_MAXK / 2 + 1], hsn[TK_MAXK / 2 + 1];
  __shared__ int hpp[TK_MAXK / 2 + 1], hqq[TK_MAXK / 2 + 1];
  __shared__ int sel[TK_MAXK];
  __shared__ unsigned char taken[TK_MAXKHAT];
  const int n = a.n, K = a.K, tid = threadIdx.x, nt = blockDim.x;
  const int half = (n + 1) / 2;
  unsigned char* p = smem;
  T* A;
  T* V;
  if (a.use_smem) {
    A = (T*)p;
    p += (size_t)n * n * sizeof(T);
    V = (T*)p;
    p += (size_t)n * n * sizeof(T);
  } else {
    A = a.gA;
    V = a.gV;
  }
  JacobiWork<T> wk;
  wk.cs = (T*)p;
  p += (size_t)half * sizeof(T);
  wk.sn = (T*)p;
  p += (size_t)half * sizeof(T);
  wk.pp = (int*)p;
  p += (size_t)half * sizeof(int);
  wk.qq = (int*)p;
  for (int idx = tid; idx < n * n; idx += nt) {
    A[idx] = (T)a.W[idx];
    V[idx] = (idx / n == idx % n) ? T(1) : T(0);
  }
  for (int i = tid; i < n; i += nt) taken[i] = 0;
  __syncthreads();
  jacobi_block<T>(A, V, n, a.max_sweeps, a.tol, wk, red);
  __syncthreads();
  for (int kk = 0; kk < K; ++kk) {
    const int i = block_argmax_diag<T>(A, n, taken, red, redi);
    if (tid == 0) {
      sel[kk] = i < n ? i : 0;
      taken[i < n ? i : 0] = 1;
    }
    __syncthreads();
  }
  // X = selected eigenvectors (FP64)
  for (int idx = tid; idx < n * K; idx += nt) {
    const int i = idx / K, k = idx - i * K;
    a.X[idx] = (double)V[i * n + sel[k]];
  }
  __syncthreads();
  if (a.polish) {
    // modified Gram-Schmidt in FP64
    for (int k = 0; k < K; ++k) {
      for (int j = 0; j < k; ++j) {
        double d = 0.0;
        for (int i = tid; i < n; i += nt) d += a.X[i * K + j] * a.X[i * K + k];
        d = block_sum_d(d, red);
        for (int i = tid; i < n; i += nt) a.X[i * K + k] -= d * a.X[i * K + j];
        __syncthreads();
      }
      double nn = 0.0;
      for (int i = tid; i < n; i += nt) nn += a.X[i * K + k] * a.X[i * K + k];
      nn = block_sum_d(nn, red);
      const double inv = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
      for (int i = tid; i < n; i += nt) a.X[i * K + k] *= inv;
      __syncthreads();
    }
    // one subspace step Y = W X, then Rayleigh-Ritz on span(Y)
    for (int idx = tid; idx < n * K; idx += nt) {
      const int i = idx / K, k = idx - i * K;
      double s = 0.0;
      const double* wr = a.W + (int64_t)i * n;
      for (int cc = 0; cc < n; ++cc) s = fma(wr[cc], a.X[cc * K + k], s);
      a.Y[idx] = s;
    }
    __syncthreads();
    for (int k = 0; k < K; ++k) {  // orthonormalise Y (MGS) -> new basis X
      for (int j = 0; j < k; ++j) {
        double d = 0.0;
        for (int i = tid; i < n; i += nt) d += a.Y[i * K + j] * a.Y[i * K + k];
        d = block_sum_d(d, red);
        for (int i = tid; i < n; i += nt) a.Y[i * K + k] -= d * a.Y[i * K + j];
        __syncthreads();
      }
      double nn = 0.0;
      for (int i = tid; i < n; i += nt) nn += a.Y[i * K + k] * a.Y[i * K + k];
      nn = block_sum_d(nn, red);
      const double inv = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
      for (int i = tid; i < n; i += nt) {
        a.Y[i * K + k] *= inv;
        a.X[i * K + k] = a.Y[i * K + k];
      }
      __syncthreads();
    }
    // Y = W X ; H = X^T Y
    for (int idx = tid; idx < n * K; idx += nt) {
      const int i = idx / K, k = idx - i * K;
      double s = 0.0;
      const double* wr = a.W + (int64_t)i * n;
      for (int cc = 0; cc < n; ++cc) s = fma(wr[cc], a.X[cc * K + k], s);
      a.Y[idx] = s;
    }
    __syncthreads();
    for (int idx = tid; idx < K * K; idx += nt) {
      const int r = idx / K, cidx = idx - r * K;
      double s = 0.0;
      for (int i = 0; i < n; ++i) s = fma(a.X[i * K + r], a.Y[i * K + cidx], s);
      H[idx] = s;
    }
    __syncthreads();
    for (int idx = tid; idx < K * K; idx += nt) {
      const int r = idx / K, cidx = idx - r * K;
      HV[idx] = (r == cidx) ? 1.0 : 0.0;
      if (r < cidx) {
        const double m = 0.5 * (H[idx] + H[cidx * K + r]);
        H[idx] = m;
        H[cidx * K + r] = m;
      }
    }
    __syncthreads();
    JacobiWork<double> hw{hcs, hsn, hpp, hqq};
    jacobi_block<double>(H, HV, K, 40, 1e-15, hw, red);
    for (int i = tid; i < K; i += nt) taken[i] = 0;
    __syncthreads();
    for (int kk = 0; kk < K; ++kk) {
      const int i = block_argmax_diag<double>(H, K, taken, red, redi);
      if (tid == 0) {
        sel[kk] = i < K ? i : 0;
        taken[i < K ? i : 0] = 1;
      }
      __syncthreads();
    }
    for (int idx = tid; idx < n * K; idx += nt) {
      const int i = idx / K, k = idx - i * K;
      double s = 0.0;
      for (int j = 0; j < K; ++j) s = fma(a.X[i * K + j], HV[j * K + sel[k]], s);
      a.Vout[idx] = s;
    }
    for (int k = tid; k < K; k += nt) a.sigma[k] = sqrt(fmax(H[sel[k] * K + sel[k]], 0.0));
  } else {
    for (int idx = tid; idx < n * K; idx += nt) a.Vout[idx] = a.X[idx];
    for (int k = tid; k < K; k += nt) a.sigma[k] = sqrt(fmax((double)A[sel[k] * n + sel[k]], 0.0));
  }
  __syncthreads();
  for (int idx = tid; idx < n * K; idx += nt) {
    const int k = idx % K;
    const double sg = a.sigma[k];
    if (!(sg > 0.0) || !isfinite(sg)) {
      if (idx < K) atomicOr(a.err, TK_DEV_ERR_NUMERIC);
      a.Vs[idx] = T(0);
    } else {
      a.Vs[idx] = (T)(a.Vout[idx] / sg);
    }
  }
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

// ------------------------------------------------------------------ CholeskyQR2
// Per-block partial of (U M)^T (U M): batches of 64 rows are transformed into
// shared memory, each thread sums its (a,b) pairs over a batch in T and adds
// the batch sum into an FP64 accumulator.
template <typename T>
__global__ void __launch_bounds__(256) k_small_gram(const T* __restrict__ U, int R, int K, const double* __restrict__ M,
                                                    double* __restrict__ Cpart) {
  __shared__ T rows[64][TK_MAXK + 1];
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
    for (int i = tid; i < 64 * K; i += 256) {
      const int r = i / K, k = i - r * K;
      const int row = r0 + r;
      T v = T(0);
      if (row < R) {
        if (M) {
          for (int j = 0; j <= k; ++j) v = fma(U[(int64_t)row * K + j], Ms[j][k], v);  // M upper triangular
        } else {
          v = U[(int64_t)row * K + k];
        }
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

// C = sum of the block partials (fixed order); C = R^T R; out = prev * R^-1.
// One warp: lanes over rows / columns.
__global__ void k_chol_inv(const double* __restrict__ Cpart, int nblk, int K, const double* prev, double* out, int* err) {
  __shared__ double C[TK_MAXK][TK_MAXK + 1];
  __shared__ double Ri[TK_MAXK][TK_MAXK + 1];
  const int lane = threadIdx.x;
  for (int i = lane; i < K * K; i += 32) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += Cpart[(int64_t)b * K * K + i];
    C[i / K][i % K] = s;
  }
  __syncwarp();
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

struct Cand {
  double a;  // |value|
  int r;     // compact row (increasing slice id)
  double v;  // signed value
};
__device__ __forceinline__ bool better(const Cand& x, const Cand& y) { return x.a > y.a || (x.a == y.a && x.r < y.r); }

// U <- U M (row by row) and per-block best (|value|, lowest row) per column.
template <typename T>
__global__ void __launch_bounds__(256) k_apply(T* __restrict__ U, int R, int K, const double* __restrict__ M,
                                               double* __restrict__ colbest) {
  __shared__ T Ms[TK_MAXK][TK_MAXK];
  __shared__ Cand wbest[8][TK_MAXK];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  for (int i = tid; i < K * K; i += 256) Ms[i / K][i % K] = (T)M[i];
  __syncthreads();
  Cand best[TK_MAXK];
  for (int k = 0; k < K; ++k) best[k] = Cand{-1.0, 0x7fffffff, 0.0};
  for (int r = blockIdx.x * 256 + tid; r < R; r += gridDim.x * 256) {
    T u[TK_MAXK], v[TK_MAXK];
    for (int k = 0; k < K; ++k) u[k] = U[(int64_t)r * K + k];
    for (int k = 0; k < K; ++k) {
      T s = T(0);
      for (int j = 0; j <= k; ++j) s = fma(u[j], Ms[j][k], s);
      v[k] = s;
    }
    for (int k = 0; k < K; ++k) {
      U[(int64_t)r * K + k] = v[k];
      const Cand c{fabs((double)v[k]), r, (double)v[k]};
      if (better(c, best[k])) best[k] = c;
    }
  }
  for (int k = 0; k < K; ++k) {
    Cand c = best[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      Cand d;
      d.a = __shfl_down_sync(0xffffffffu, c.a, o);
      d.r = __shfl_down_sync(0xffffffffu, c.r, o);
      d.v = __shfl_down_sync(0xffffffffu, c.v, o);
      if (better(d, c)) c = d;
    }
    if (lane == 0) wbest[w][k] = c;
  }
  __syncthreads();
  if (tid < K) {
    Cand c = wbest[0][tid];
    for (int ww = 1; ww < 8; ++ww)
      if (better(wbest[ww][tid], c)) c = wbest[ww][tid];
    double* o = colbest + ((int64_t)blockIdx.x * K + tid) * 3;
    o[0] = c.a;
    o[1] = (double)c.r;
    o[2] = c.v;
  }
}

__global__ void k_signs(const double* colbest, int nblk, int K, double* sign) {
  const int k = threadIdx.x;
  if (k >= K) return;
  Cand c{-1.0, 0x7fffffff, 0.0};
  for (int b = 0; b < nblk; ++b) {
    const double* o = colbest + ((int64_t)b * K + k) * 3;
    const Cand d{o[0], (int)o[1], o[2]};
    if (better(d, c)) c = d;
  }
  sign[k] = c.v < 0.0 ? -1.0 : 1.0;
}

template <typename T>
__global__ void k_scatter_rows(const T* __restrict__ U, int R, int K, const int32_t* __restrict__ row_id,
                               const double* __restrict__ sign, T* __restrict__ F, int ldF) {
  const int64_t total = (int64_t)R * K;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(i / K), k = (int)(i - (int64_t)r * K);
    F[(int64_t)row_id[r] * ldF + k] = (T)(sign[k] * (double)U[i]);
  }
}

template <typename T>
void setup_eig_attr() {
  static bool done = false;
  if (!done) {
    TK_CUDA(cudaFuncSetAttribute(k_eig<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024));
    done = true;
  }
}

template <typename T>
void factor_impl(tucker_ctx* c, int n, const void* Zv, void* F_out, int ldF_out, double* sigma_out, cudaStream_t s) {
  const tk_mode& md = c->mode[n];
  const int R = md.R, Khat = md.Khat, K = c->K[n];
  const T* Z = (const T*)Zv;
  const int sms = c->sm_count;

  // ---- Gram W = Z^T Z
  tk_phase_begin(c, PH_GRAM, s);
  {
    const int TM = (sizeof(T) == 4 && Khat > 64) ? 128 : 64;
    const int tpd = (int)tk_ceil_div(Khat, TM);
    const int ntiles = tpd * (tpd + 1) / 2;
    int nsplit = (int)std::max<int64_t>(1, std::min<int64_t>(tk_ceil_div(R, 64), tk_ceil_div(2 * sms, ntiles)));
    while ((size_t)nsplit * ntiles * TM * TM > c->Wpart_elems && nsplit > 1) --nsplit;
    const int rps = (int)tk_ceil_div(R, nsplit);
    std::vector<int2> tl;
    for (int i = 0; i < tpd; ++i)
      for (int j = i; j < tpd; ++j) tl.push_back(make_int2(i, j));
    if ((int)tl.size() > c->gram_tiles_cap) tk_throw(TUCKER_ERR_STATE, "internal: Gram tile list too long");
    int2* dtiles = c->gram_tiles;
    TK_CUDA(cudaMemcpyAsync(dtiles, tl.data(), tl.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
    dim3 grid(ntiles, nsplit);
    if (TM == 128) k_gram<T, 128><<<grid, 256, 0, s>>>(Z, R, Khat, dtiles, ntiles, rps, (T*)c->Wpart);
    else k_gram<T, 64><<<grid, 256, 0, s>>>(Z, R, Khat, dtiles, ntiles, rps, (T*)c->Wpart);
    TK_CUDA(cudaGetLastError());
    const unsigned g2 = (unsigned)std::min<int64_t>(tk_ceil_div((int64_t)Khat * Khat, 256), 4096);
    k_gram_reduce<T><<<g2, 256, 0, s>>>((const T*)c->Wpart, nsplit, ntiles, tpd, TM, Khat, c->W);
    TK_CUDA(cudaGetLastError());
    tk_launched(c, PH_GRAM, 2);
  }
  tk_phase_end(c, s);

  // ---- eigensolve
  tk_phase_begin(c, PH_EIG, s);
  {
    setup_eig_attr<T>();
    EigArgs<T> a{};
    a.W = c->W;
    a.n = Khat;
    a.K = K;
    a.gA = (T*)c->eigA;
    a.gV = (T*)c->eigV;
    const size_t mat = (size_t)2 * Khat * Khat * sizeof(T);
    const int half = (Khat + 1) / 2;
    const size_t work = (size_t)half * (2 * sizeof(T) + 2 * sizeof(int)) + 64;
    a.use_smem = (mat + work) <= 140 * 1024;
    const size_t shm = (a.use_smem ? mat : 0) + work;
    a.polish = c->prec == TUCKER_FP32;
    a.max_sweeps = sizeof(T) == 4 ? 20 : 40;
    a.tol = sizeof(T) == 4 ? 1e-6 : 1e-13;
    a.X = c->eigX;
    a.Y = c->eigX + (size_t)Khat * K;
    a.Vout = c->V;
    a.sigma = c->sigma;
    a.Vs = (T*)c->Vs;
    a.err = c->err;
    k_eig<T><<<1, 1024, shm, s>>>(a);
    TK_CUDA(cudaGetLastError());
    tk_launched(c, PH_EIG);
  }
  tk_phase_end(c, s);

  // ---- back-projection + CholeskyQR2 + signs + scatter
  tk_phase_begin(c, PH_BACKPROJ, s);
  {
    const T* Vs = (const T*)c->Vs;
    T* U = (T*)c->U;
    const unsigned gb = (unsigned)std::max<int64_t>(1, std::min<int64_t>(tk_ceil_div(R, 256), 8 * sms));
    if (K <= 8) k_backproj<T, 8><<<gb, 256, 0, s>>>(Z, R, Khat, Vs, K, U);
    else if (K <= 16) k_backproj<T, 16><<<gb, 256, 0, s>>>(Z, R, Khat, Vs, K, U);
    else k_backproj<T, 32><<<gb, 256, 0, s>>>(Z, R, Khat, Vs, K, U);
    TK_CUDA(cudaGetLastError());
    const int nblk = (int)std::max<int64_t>(1, std::min<int64_t>(tk_ceil_div(R, 64), 2 * sms));
    double* R1 = c->Rinv;
    double* R2 = c->Rinv + TK_MAXK * TK_MAXK;
    double* sign = c->Rinv + 2 * TK_MAXK * TK_MAXK;
    k_small_gram<T><<<nblk, 256, 0, s>>>(U, R, K, nullptr, c->Cpart);
    k_chol_inv<<<1, 32, 0, s>>>(c->Cpart, nblk, K, nullptr, R1, c->err);
    k_small_gram<T><<<nblk, 256, 0, s>>>(U, R, K, R1, c->Cpart);
    k_chol_inv<<<1, 32, 0, s>>>(c->Cpart, nblk, K, R1, R2, c->err);
    const int nab = (int)std::max<int64_t>(1, std::min<int64_t>(tk_ceil_div(R, 256), 2 * sms));
    k_apply<T><<<nab, 256, 0, s>>>(U, R, K, R2, c->colbest);
    k_signs<<<1, 32, 0, s>>>(c->colbest, nab, K, sign);
    TK_CUDA(cudaMemsetAsync(F_out, 0, (size_t)c->L[n] * ldF_out * sizeof(T), s));
    const unsigned gs = (unsigned)std::max<int64_t>(1, std::min<int64_t>(tk_ceil_div((int64_t)R * K, 256), 8 * sms));
    k_scatter_rows<T><<<gs, 256, 0, s>>>(U, R, K, md.row_id, sign, (T*)F_out, ldF_out);
    TK_CUDA(cudaGetLastError());
    tk_launched(c, PH_BACKPROJ, 8);
    if (sigma_out) TK_CUDA(cudaMemcpyAsync(sigma_out, c->sigma, K * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  tk_phase_end(c, s);
}

}  // namespace

void tk_factor_update(tucker_ctx* c, int n, const void* Z, void* F_out, int ldF_out, double* sigma_out, cudaStream_t s) {
  if (c->prec == TUCKER_FP32) factor_impl<float>(c, n, Z, F_out, ldF_out, sigma_out, s);
  else factor_impl<double>(c, n, Z, F_out, ldF_out, sigma_out, s);
}
