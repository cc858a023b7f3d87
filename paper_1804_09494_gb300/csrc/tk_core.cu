// New core G = T x_1 F_1^T ... x_N F_N^T (Fig. 1), computed as
// G_(n*) = F_n*^T Z_(n*) from the compact penultimate matrix of one mode, then
// folded to the first-mode-fastest layout; ||G||^2 and the fit in FP64.
#include <algorithm>

#include "tk_common.cuh"

namespace {

// Deterministic block sum: fixed shuffle tree per warp, warp 0 adds the warp
// sums in order (FP64 work stays on one warp; red needs 33 slots).
__device__ double block_sum_fixed(double v, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    double s = lane < nw ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) red[32] = s;
  }
  __syncthreads();
  return red[32];
}

// Gpart[split][k][c] = sum over the split's rows r of F[frow[r]][k] * Z[r][c] (F is one of the
// context's factor buffers, whose rows are popularity labels: frow[r] = label of compact row r).
// Thread owns column c; rows in batches of 32 (factor rows staged in shared
// memory), batch sums in T added into FP64 accumulators.
template <typename T, int KM>
__global__ void __launch_bounds__(128) k_core_partial(const T* __restrict__ Z, int R, int Khat,
                                                      const int32_t* __restrict__ frow, const T* __restrict__ F,
                                                      int ldF, int K, int rows_per_split, double* __restrict__ Gpart) {
  __shared__ T fr[32][KM];
  const int c = blockIdx.x * 128 + threadIdx.x;
  const int sp = blockIdx.y;
  const int r0 = sp * rows_per_split, r1 = min(R, r0 + rows_per_split);
  double dacc[KM];
#pragma unroll
  for (int k = 0; k < KM; ++k) dacc[k] = 0.0;
  for (int rb = r0; rb < r1; rb += 32) {
    for (int i = threadIdx.x; i < 32 * KM; i += 128) {
      const int r = i / KM, k = i - r * KM;
      fr[r][k] = (rb + r < r1 && k < K) ? F[(int64_t)frow[rb + r] * ldF + k] : T(0);
    }
    __syncthreads();
    if (c < Khat) {
      T acc[KM];
#pragma unroll
      for (int k = 0; k < KM; ++k) acc[k] = T(0);
      const int nr = min(32, r1 - rb);
      for (int r = 0; r < nr; ++r) {
        const T z = Z[(int64_t)(rb + r) * Khat + c];
#pragma unroll
        for (int k = 0; k < KM; ++k) acc[k] = fma(fr[r][k], z, acc[k]);
      }
#pragma unroll
      for (int k = 0; k < KM; ++k) dacc[k] += (double)acc[k];
    }
    __syncthreads();
  }
  if (c < Khat)
    for (int k = 0; k < K; ++k) Gpart[((int64_t)sp * K + k) * Khat + c] = dacc[k];
}

struct FoldInfo {
  int N, n, Kn, Khat;
  int K[TK_MAXN];
};

// G (first mode fastest) from the split partials: 8 lanes per entry, each
// summing every 8th split in order, combined by a fixed shuffle tree; the
// entry is written at its folded position.
template <typename T>
__global__ void __launch_bounds__(256) k_core_fold(const double* __restrict__ Gpart, int nsplit, FoldInfo fi,
                                                   double* __restrict__ Gd, T* __restrict__ Gout) {
  int stride[TK_MAXN];
  {
    int s = 1;
    for (int m = 0; m < fi.N; ++m) {
      stride[m] = s;
      s *= fi.K[m];
    }
  }
  const int total = fi.Kn * fi.Khat;
  const int part = threadIdx.x & 7;
  const int per_pass = (gridDim.x * blockDim.x) >> 3;
  for (int base = 0; base < total; base += per_pass) {  // uniform trip count for every lane
    const int idx0 = base + ((blockIdx.x * blockDim.x + threadIdx.x) >> 3);
    const bool live = idx0 < total;
    const int idx = live ? idx0 : 0;
    const int k = idx / fi.Khat, c = idx - k * fi.Khat;
    double s = 0.0;
    if (live)
      for (int sp = part; sp < nsplit; sp += 8) s += Gpart[((int64_t)sp * fi.Kn + k) * fi.Khat + c];
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    s += __shfl_xor_sync(0xffffffffu, s, 4);
    if (part == 0 && live) {
      int lin = k * stride[fi.n];
      int rem = c;
      for (int m = 0; m < fi.N; ++m) {
        if (m == fi.n) continue;
        lin += (rem % fi.K[m]) * stride[m];
        rem /= fi.K[m];
      }
      Gd[lin] = s;
      if (Gout) Gout[lin] = (T)s;
    }
  }
}

// ||G||^2 (fixed order) and the fit, one CTA.
__global__ void __launch_bounds__(256) k_core_fit(const double* __restrict__ Gd, int size, double normT2,
                                                  double* __restrict__ fit_out) {
  __shared__ double red[33];
  double g2 = 0.0;
  for (int i = threadIdx.x; i < size; i += blockDim.x) g2 = fma(Gd[i], Gd[i], g2);
  g2 = block_sum_fixed(g2, red);
  if (threadIdx.x == 0) {
    fit_out[0] = g2;
    fit_out[1] = 1.0 - sqrt(fmax(0.0, normT2 - g2)) / sqrt(normT2);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_norm2_partial(const T* __restrict__ v, int64_t n, double* part, int* err) {
  __shared__ double red[33];
  double s = 0.0;
  bool bad = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = (double)v[i];
    if (!isfinite(x)) bad = true;
    s = fma(x, x, s);
  }
  if (bad) atomicOr(err, TK_DEV_ERR_NONFINITE);
  s = block_sum_fixed(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_sum_final(const double* part, int n, double* out) {
  __shared__ double red[33];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
  s = block_sum_fixed(s, red);
  if (threadIdx.x == 0) *out = s;
}

template <typename T>
void core_impl(tucker_ctx* c, void* const* F, const int* ldF, void* G_out, cudaStream_t s, cudaEvent_t before_Fn) {
  const int n = tk_core_mode(c);
  const tk_mode& md = c->mode[n];
  // the TTM-chain of mode n does not read F_n: the producer of F_n may still run
  tk_ttmc_forward(c, n, F, ldF, nullptr, c->Zcore, s);
  if (before_Fn) TK_CUDA(cudaStreamWaitEvent(s, before_Fn, 0));
  tk_phase_begin(c, PH_CORE, s);
  const int K = c->K[n], Khat = md.Khat, R = md.R;
  const int cb = (int)tk_ceil_div(Khat, 128);
  int nsplit = (int)std::max<int64_t>(1, std::min<int64_t>(tk_ceil_div(R, 64), tk_ceil_div(4 * c->sm_count, cb)));
  const int rps = (int)tk_ceil_div(R, nsplit);
  dim3 grid(cb, nsplit);
  const T* Z = (const T*)c->Zcore;
  const T* Fn = (const T*)F[n];
  if (K <= 8) k_core_partial<T, 8><<<grid, 128, 0, s>>>(Z, R, Khat, md.frow, Fn, ldF[n], K, rps, c->Gpart);
  else if (K <= 16) k_core_partial<T, 16><<<grid, 128, 0, s>>>(Z, R, Khat, md.frow, Fn, ldF[n], K, rps, c->Gpart);
  else k_core_partial<T, 32><<<grid, 128, 0, s>>>(Z, R, Khat, md.frow, Fn, ldF[n], K, rps, c->Gpart);
  TK_CUDA(cudaGetLastError());
  FoldInfo fi{};
  fi.N = c->N;
  fi.n = n;
  fi.Kn = K;
  fi.Khat = Khat;
  for (int m = 0; m < c->N; ++m) fi.K[m] = c->K[m];
  const unsigned gf = (unsigned)std::max<int64_t>(1, std::min<int64_t>(tk_ceil_div((int64_t)K * Khat * 8, 256), 4 * c->sm_count));
  k_core_fold<T><<<gf, 256, 0, s>>>(c->Gpart, nsplit, fi, c->Gd, (T*)G_out);
  TK_CUDA(cudaGetLastError());
  k_core_fit<<<1, 256, 0, s>>>(c->Gd, (int)c->Gsize, c->normT2, c->fit_d);
  TK_CUDA(cudaGetLastError());
  tk_launched(c, PH_CORE, 3);
  tk_phase_end(c, s);
}

}  // namespace

// the mode with the smallest TTM-chain work (nnz * Khat) and then the fewest rows
int tk_core_mode(const tucker_ctx* c) {
  int best = 0;
  for (int n = 1; n < c->N; ++n) {
    const tk_mode& a = c->mode[n];
    const tk_mode& b = c->mode[best];
    if (a.Khat < b.Khat || (a.Khat == b.Khat && a.R < b.R)) best = n;
  }
  return best;
}

void tk_core(tucker_ctx* c, void* const* F, const int* ldF, void* G_out, cudaStream_t s, cudaEvent_t before_Fn) {
  if (c->prec == TUCKER_FP32) core_impl<float>(c, F, ldF, G_out, s, before_Fn);
  else core_impl<double>(c, F, ldF, G_out, s, before_Fn);
}

double tk_norm2(tucker_ctx* c, const void* vals, int64_t n, cudaStream_t s) {
  const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(tk_ceil_div(n, 256), 4 * c->sm_count));
  double* part = (double*)tk_dev_alloc(c, (size_t)(nb + 1) * sizeof(double));
  if (c->prec == TUCKER_FP32) k_norm2_partial<float><<<nb, 256, 0, s>>>((const float*)vals, n, part, c->err);
  else k_norm2_partial<double><<<nb, 256, 0, s>>>((const double*)vals, n, part, c->err);
  k_sum_final<<<1, 256, 0, s>>>(part, nb, part + nb);
  double out = 0.0;
  TK_CUDA(cudaMemcpyAsync(&out, part + nb, sizeof(double), cudaMemcpyDeviceToHost, s));
  TK_CUDA(cudaStreamSynchronize(s));
  tk_dev_free(c, part, (size_t)(nb + 1) * sizeof(double));
  return out;
}
