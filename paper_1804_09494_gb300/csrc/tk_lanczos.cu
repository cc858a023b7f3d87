// The paper's SVD route for the factor update (Section 3, "SVD component";
// Section 7: 2K iterations): a Golub-Kahan-Lanczos bidiagonalisation of the
// compact penultimate matrix Z (R x Khat), matrix-free -- each step asks for
// one product Z v and one product u^T Z -- with both bases re-orthogonalised
// in full (classical Gram-Schmidt, twice).  After m = min(2K, Khat, R) steps,
// Z V = U B with B upper bidiagonal (alpha on the diagonal, beta above it);
// the right singular vectors Q_K of B (eigenvectors of the tridiagonal B^T B,
// through the context's eigensolver) give V_K = V Q_K and sigma_K, written
// where the exact route's eigensolver writes them, so the back-projection,
// CholeskyQR2, signs and scatter are shared.
//
// The start vector is the all-ones vector.  Products with Z run in the
// working precision in chunks of 32 terms, summed in FP64; the Lanczos
// vectors and every reduction are FP64, in a fixed order.  Per step: the
// product Z v (a thread per row), two rounds of (dots with the previous u,
// subtraction), the norm, the scaling; the product u^T Z (column partials per
// row block, reduced in order); the v-side orthogonalisation in one CTA.
#include <algorithm>

#include "tk_common.cuh"

namespace {

constexpr int kLzThreads = 256;
constexpr int kLzMaxM = 64;  // steps at most (2 K with K <= 32)

unsigned lz_blocks(const tucker_ctx* c, int64_t R) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(tk_ceil_div(R, kLzThreads), 2 * c->sm_count));
}

// p[r] = sum_c Z[r][c] v[c] - beta_prev u_prev[r]
template <typename T>
__global__ void __launch_bounds__(kLzThreads) k_lz_zv(const T* __restrict__ Z, int64_t R, int Khat,
                                                      const double* __restrict__ v, const double* __restrict__ beta_prev,
                                                      const double* __restrict__ uprev, double* __restrict__ p) {
  extern __shared__ unsigned char lz_sm[];
  T* vs = (T*)lz_sm;
  for (int i = threadIdx.x; i < Khat; i += blockDim.x) vs[i] = (T)v[i];
  __syncthreads();
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < R; r += (int64_t)gridDim.x * blockDim.x) {
    const T* zr = Z + r * Khat;
    double acc = 0.0;
    for (int c0 = 0; c0 < Khat; c0 += 32) {
      const int c1 = min(Khat, c0 + 32);
      T part = T(0);
      for (int cc = c0; cc < c1; ++cc) part = fma(zr[cc], vs[cc], part);
      acc += (double)part;
    }
    if (uprev) acc -= beta_prev[0] * uprev[r];
    p[r] = acc;
  }
}

// part[b][i] = sum over block b's rows of U[i][r] p[r], i < j (fixed order)
__global__ void __launch_bounds__(kLzThreads) k_lz_dots(const double* __restrict__ U, const double* __restrict__ p,
                                                        int64_t R, int j, double* __restrict__ part) {
  __shared__ double red[kLzThreads];
  const int64_t per = tk_ceil_div(R, gridDim.x);
  const int64_t r0 = blockIdx.x * per, r1 = min(R, r0 + per);
  for (int i = 0; i < j; ++i) {
    double s = 0.0;
    for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) s = fma(U[(int64_t)i * R + r], p[r], s);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
      if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[(int64_t)blockIdx.x * kLzMaxM + i] = red[0];
    __syncthreads();
  }
}

// out[i] = sum_b part[b][i] in order (one CTA); with scale: out[0] = sqrt(sum)
__global__ void k_lz_sum(const double* __restrict__ part, int nb, int j, double* __restrict__ out, int as_norm) {
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[(int64_t)b * kLzMaxM + i];
    out[i] = as_norm ? sqrt(fmax(s, 0.0)) : s;
  }
}

// p[r] -= sum_{i<j} c[i] U[i][r]; with norm: part[b][0] = sum over block b of p[r]^2
__global__ void __launch_bounds__(kLzThreads) k_lz_axpy(const double* __restrict__ U, const double* __restrict__ cf,
                                                        int64_t R, int j, double* __restrict__ p, int norm,
                                                        double* __restrict__ part) {
  __shared__ double red[kLzThreads];
  __shared__ double cs[kLzMaxM];
  for (int i = threadIdx.x; i < j; i += blockDim.x) cs[i] = cf[i];
  __syncthreads();
  const int64_t per = tk_ceil_div(R, gridDim.x);
  const int64_t r0 = blockIdx.x * per, r1 = min(R, r0 + per);
  double s = 0.0;
  for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
    double x = p[r];
    for (int i = 0; i < j; ++i) x = fma(-cs[i], U[(int64_t)i * R + r], x);
    p[r] = x;
    s = fma(x, x, s);
  }
  if (!norm) return;
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(int64_t)blockIdx.x * kLzMaxM] = red[0];
}

// U[j][r] = p[r] / alpha (0 if alpha is 0)
__global__ void k_lz_scale(const double* __restrict__ p, const double* __restrict__ alpha, int64_t R,
                           double* __restrict__ u) {
  const double a = alpha[0];
  const double inv = a > 0.0 ? 1.0 / a : 0.0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < R; r += (int64_t)gridDim.x * blockDim.x)
    u[r] = p[r] * inv;
}

// part[b][c] = sum over block b's rows of Z[r][c] u[r]
template <typename T>
__global__ void __launch_bounds__(kLzThreads) k_lz_ztu(const T* __restrict__ Z, int64_t R, int Khat,
                                                       const double* __restrict__ u, double* __restrict__ part) {
  __shared__ T us[32];
  const int64_t per = tk_ceil_div(R, gridDim.x);
  const int64_t r0 = blockIdx.x * per, r1 = min(R, r0 + per);
  for (int c0 = 0; c0 < Khat; c0 += blockDim.x) {
    const int c = c0 + threadIdx.x;
    double acc = 0.0;
    for (int64_t rb = r0; rb < r1; rb += 32) {
      __syncthreads();
      if (threadIdx.x < 32) us[threadIdx.x] = rb + threadIdx.x < r1 ? (T)u[rb + threadIdx.x] : T(0);
      __syncthreads();
      if (c < Khat) {
        T partial = T(0);
        const int nr = (int)min((int64_t)32, r1 - rb);
        for (int q = 0; q < nr; ++q) partial = fma(Z[(rb + q) * Khat + c], us[q], partial);
        acc += (double)partial;
      }
    }
    if (c < Khat) part[(int64_t)blockIdx.x * Khat + c] = acc;
  }
}

// The v side of step j, one CTA: q = sum_b part[b] (in order); r = q - alpha v_j;
// two rounds of r -= V (V^T r) over v_0..v_j; beta = ||r||; v_{j+1} = r / beta.
__global__ void __launch_bounds__(1024) k_lz_vside(const double* __restrict__ part, int nb, int Khat, int j,
                                                   const double* __restrict__ alpha, double* __restrict__ V,
                                                   double* __restrict__ beta) {
  extern __shared__ unsigned char lz_sm[];
  double* r = (double*)lz_sm;       // Khat
  double* cf = r + Khat;            // kLzMaxM + 1
  __shared__ double red[1024];
  const double a = alpha[0];
  for (int c = threadIdx.x; c < Khat; c += blockDim.x) {
    double q = 0.0;
    for (int b = 0; b < nb; ++b) q += part[(int64_t)b * Khat + c];
    r[c] = q - a * V[(int64_t)j * Khat + c];
  }
  __syncthreads();
  for (int round = 0; round < 2; ++round) {
    for (int i = 0; i <= j; ++i) {
      double s = 0.0;
      for (int c = threadIdx.x; c < Khat; c += blockDim.x) s = fma(V[(int64_t)i * Khat + c], r[c], s);
      red[threadIdx.x] = s;
      __syncthreads();
      for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
      }
      if (threadIdx.x == 0) cf[i] = red[0];
      __syncthreads();
    }
    for (int c = threadIdx.x; c < Khat; c += blockDim.x) {
      double x = r[c];
      for (int i = 0; i <= j; ++i) x = fma(-cf[i], V[(int64_t)i * Khat + c], x);
      r[c] = x;
    }
    __syncthreads();
  }
  double s = 0.0;
  for (int c = threadIdx.x; c < Khat; c += blockDim.x) s = fma(r[c], r[c], s);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  const double b = sqrt(fmax(red[0], 0.0));
  const double inv = b > 0.0 ? 1.0 / b : 0.0;
  for (int c = threadIdx.x; c < Khat; c += blockDim.x) V[(int64_t)(j + 1) * Khat + c] = r[c] * inv;
  if (threadIdx.x == 0) beta[j] = b;
}

__global__ void k_lz_start(double* __restrict__ V, int Khat) {
  const double x = 1.0 / sqrt((double)Khat);
  for (int c = threadIdx.x; c < Khat; c += blockDim.x) V[c] = x;
}

// W = B^T B (m x m, FP64, tridiagonal), B = diag(alpha) + superdiag(beta[0..m-2])
__global__ void k_lz_btb(const double* __restrict__ alpha, const double* __restrict__ beta, int m,
                         double* __restrict__ W) {
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    const int k = idx / m, l = idx % m;
    double w = 0.0;
    if (k == l) w = alpha[k] * alpha[k] + (k > 0 ? beta[k - 1] * beta[k - 1] : 0.0);
    else if (l == k + 1) w = alpha[k] * beta[k];
    else if (k == l + 1) w = alpha[l] * beta[l];
    W[idx] = w;
  }
}

// V_K = V Q_K (Khat x K) from the m x K eigenvectors Q of B^T B held in Vout;
// Vs = V_K / sigma in the working precision (one CTA)
template <typename T>
__global__ void __launch_bounds__(1024) k_lz_vk(const double* __restrict__ V, int Khat, int m, int K,
                                                double* __restrict__ Vout, const double* __restrict__ sigma,
                                                T* __restrict__ Vs) {
  extern __shared__ unsigned char lz_sm[];
  double* Q = (double*)lz_sm;  // m x K
  for (int i = threadIdx.x; i < m * K; i += blockDim.x) Q[i] = Vout[i];
  __syncthreads();
  for (int idx = threadIdx.x; idx < Khat * K; idx += blockDim.x) {
    const int c = idx / K, k = idx % K;
    double s = 0.0;
    for (int jj = 0; jj < m; ++jj) s = fma(V[(int64_t)jj * Khat + c], Q[jj * K + k], s);
    Vout[idx] = s;
    const double sg = sigma[k];
    Vs[idx] = (T)(sg > 0.0 ? s / sg : 0.0);
  }
}

template <typename T>
int lanczos_impl(tucker_ctx* c, int n, const T* Z, cudaStream_t s) {
  tk_mode& md = c->mode[n];
  tk_fuws* ws = &c->fu[n];
  const int64_t R = md.R;
  const int Khat = md.Khat, K = c->K[n];
  const int m = (int)std::min<int64_t>(std::min<int64_t>(2 * K, Khat), R);
  tk_lzws& lw = ws->lz;
  const unsigned nb = lz_blocks(c, R);
  const unsigned nbc = nb;  // row blocks of the u^T Z partials
  k_lz_start<<<1, 256, 0, s>>>(lw.V, Khat);
  for (int j = 0; j < m; ++j) {
    double* p = lw.p;
    const size_t zshm = (size_t)Khat * sizeof(T);
    k_lz_zv<T><<<nb, kLzThreads, zshm, s>>>(Z, R, Khat, lw.V + (int64_t)j * Khat, j > 0 ? lw.beta + j - 1 : nullptr,
                                            j > 0 ? lw.U + (int64_t)(j - 1) * R : nullptr, p);
    if (j > 0) {
      for (int round = 0; round < 2; ++round) {
        k_lz_dots<<<nb, kLzThreads, 0, s>>>(lw.U, p, R, j, lw.part);
        k_lz_sum<<<1, 64, 0, s>>>(lw.part, (int)nb, j, lw.cf, 0);
        k_lz_axpy<<<nb, kLzThreads, 0, s>>>(lw.U, lw.cf, R, j, p, round == 1, lw.part);
      }
    } else {
      k_lz_axpy<<<nb, kLzThreads, 0, s>>>(lw.U, lw.cf, R, 0, p, 1, lw.part);
    }
    k_lz_sum<<<1, 64, 0, s>>>(lw.part, (int)nb, 1, lw.alpha + j, 1);
    k_lz_scale<<<nb, kLzThreads, 0, s>>>(p, lw.alpha + j, R, lw.U + (int64_t)j * R);
    k_lz_ztu<T><<<nbc, kLzThreads, 0, s>>>(Z, R, Khat, lw.U + (int64_t)j * R, lw.part_c);
    const size_t vshm = ((size_t)Khat + kLzMaxM + 1) * sizeof(double);
    k_lz_vside<<<1, 1024, vshm, s>>>(lw.part_c, (int)nbc, Khat, j, lw.alpha + j, lw.V, lw.beta);
    TK_CUDA(cudaGetLastError());
  }
  k_lz_btb<<<1, 256, 0, s>>>(lw.alpha, lw.beta, m, ws->W);
  TK_CUDA(cudaGetLastError());
  tk_launched(c, PH_EIG, 2 + m * 10);
  return m;
}

}  // namespace

size_t tk_lanczos_shared_bytes(int Khat) {
  return std::max((size_t)Khat * 8, ((size_t)Khat + kLzMaxM + 1) * sizeof(double));
}

void tk_lanczos_alloc(tucker_ctx* c, int n) {
  const tk_mode& md = c->mode[n];
  tk_lzws& lw = c->fu[n].lz;
  const int64_t R = std::max(md.R, 1);
  const int Khat = md.Khat;
  const unsigned nb = lz_blocks(c, R);
  const int m = (int)std::min<int64_t>(std::min<int64_t>(2 * c->K[n], Khat), R);
  lw.U = (double*)tk_alloc(c, (size_t)R * m * 8);
  lw.p = (double*)tk_alloc(c, (size_t)R * 8);
  lw.V = (double*)tk_alloc(c, (size_t)Khat * (kLzMaxM + 1) * 8);
  lw.part = (double*)tk_alloc(c, (size_t)nb * kLzMaxM * 8);
  lw.part_c = (double*)tk_alloc(c, (size_t)nb * Khat * 8);
  lw.cf = (double*)tk_alloc(c, (size_t)kLzMaxM * 8);
  lw.alpha = (double*)tk_alloc(c, (size_t)kLzMaxM * 8);
  lw.beta = (double*)tk_alloc(c, (size_t)kLzMaxM * 8);
}

int tk_lanczos_bidiag(tucker_ctx* c, int n, const void* Z, cudaStream_t s) {
  if (c->prec == TUCKER_FP32) return lanczos_impl<float>(c, n, (const float*)Z, s);
  return lanczos_impl<double>(c, n, (const double*)Z, s);
}

void tk_lanczos_vk(tucker_ctx* c, int n, int m, cudaStream_t s) {
  tk_fuws* ws = &c->fu[n];
  const int Khat = c->mode[n].Khat, K = c->K[n];
  const size_t shm = (size_t)m * K * sizeof(double);
  if (c->prec == TUCKER_FP32)
    k_lz_vk<float><<<1, 1024, shm, s>>>(ws->lz.V, Khat, m, K, ws->V, ws->sigma, (float*)ws->Vs);
  else
    k_lz_vk<double><<<1, 1024, shm, s>>>(ws->lz.V, Khat, m, K, ws->V, ws->sigma, (double*)ws->Vs);
  TK_CUDA(cudaGetLastError());
}
