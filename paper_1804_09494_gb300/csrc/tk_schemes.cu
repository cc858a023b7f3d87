// Section 4.1 metrics of the prior distribution schemes the paper compares
// Lite with (Section 5), on the device, from a mode's permuted copy.
//
// CoarseG (multi-policy): along mode n every slice goes whole to one
// processor; in the random order pos_n (position of each slice), the slice at
// position t with H_t elements before it goes to processor floor(P H_t / nnz)
// -- contiguous blocks balanced by elements.
//
// MediumG (uni-policy): P = q_1 x ... x q_N (the prime factors of P, largest
// first, each to the mode with the largest L_m / q_m so far, the lowest m on a
// tie); mode m's permuted positions pos_m[l] are cut into q_m contiguous
// ranges (position x in range floor(x q_m / L_m)); the element goes to the
// processor of its cell, b_1 + q_1 (b_2 + q_2 (...)).
//
// Metrics per processor p: E^p = elements, R^p = distinct mode-n slices among
// them; E_max, R_sum, R_max over p.
#include <algorithm>
#include <vector>

#include "tk_common.cuh"

namespace {

struct CopyView {
  const uint32_t* rowcode;
  const int32_t* oidx[TK_MAXN - 1];
  const int32_t* bin_len;
  const int32_t* row_id;
  int Pa, limit;
  int64_t cap;
};

// slice sizes from the copy: a thread per bin adds each run of one row code
// (a whole slice or a split piece) once
__global__ void k_slice_sizes(const CopyView v, int64_t* __restrict__ cnt) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= v.Pa) return;
  const int len = v.bin_len[p];
  const int64_t base = (int64_t)(p >> 5) * v.limit * 32 + (p & 31);
  uint32_t prev = 0;
  int64_t run = 0;
  for (int k = 0; k < len; ++k) {
    const uint32_t cd = v.rowcode[base + 32 * (int64_t)k] & TK_ROW_MASK;
    if (k > 0 && cd != prev) {
      atomicAdd((unsigned long long*)&cnt[v.row_id[prev]], (unsigned long long)run);
      run = 0;
    }
    prev = cd;
    ++run;
  }
  if (len > 0) atomicAdd((unsigned long long*)&cnt[v.row_id[prev]], (unsigned long long)run);
}

// by_pos[pos[l]] = cnt[l] (by_pos and seen zeroed before); an entry outside
// [0, L) or a position given twice (pos not a permutation) is reported
__global__ void k_by_position(const int64_t* __restrict__ cnt, const int32_t* __restrict__ pos, int64_t L,
                              int64_t* __restrict__ by_pos, int32_t* __restrict__ seen, int* err) {
  for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < L; l += (int64_t)gridDim.x * blockDim.x) {
    const int32_t t = pos[l];
    if (t < 0 || t >= L || atomicAdd(&seen[t], 1) != 0) {
      atomicOr(err, TK_DEV_ERR_INDEX);
      continue;
    }
    by_pos[t] = cnt[l];
  }
}

// CoarseG: slice l (non-empty) -> processor floor(P H[pos[l]] / nnz)
__global__ void k_coarseg(const int64_t* __restrict__ cnt, const int32_t* __restrict__ pos,
                          const int64_t* __restrict__ H, int64_t L, int P, int64_t nnz, unsigned long long* __restrict__ E,
                          unsigned long long* __restrict__ R) {
  for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < L; l += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = cnt[l];
    if (c == 0) continue;
    const int32_t t = pos[l];
    if (t < 0 || t >= L) continue;  // reported by k_by_position
    const int p = (int)min((int64_t)P - 1, (int64_t)P * H[t] / nnz);  // P H < 2^62; < P unless pos is invalid
    atomicAdd(&E[p], (unsigned long long)c);
    atomicAdd(&R[p], 1ull);
  }
}

struct GridInfo {
  int N, n;
  int q[TK_MAXN];
  int64_t L[TK_MAXN];
  int64_t stride[TK_MAXN];   // of the processor index
  int64_t rstride[TK_MAXN];  // of the other modes' cell index r (mode n excluded)
  int64_t Rn;                // P / q_n
  const int32_t* pos[TK_MAXN];
  const int32_t* unlabel[TK_MAXN];
  int others[TK_MAXN - 1];
};

// MediumG, one pass over the copy: E^p (shared-memory histogram when P is
// small, global atomics otherwise) and the (slice, other cell) presence bits
__global__ void k_mediumg_elems(const CopyView v, const GridInfo gi, int P, unsigned long long* __restrict__ E,
                                uint32_t* __restrict__ bits, int* err) {
  extern __shared__ unsigned long long Es[];
  const bool priv = P <= 4096;
  if (priv)
    for (int i = threadIdx.x; i < P; i += blockDim.x) Es[i] = 0;
  __syncthreads();
  for (int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; slot < v.cap;
       slot += (int64_t)gridDim.x * blockDim.x) {
    const int lane = (int)(slot & 31);
    const int64_t rest = slot >> 5;
    const int64_t k = rest % v.limit;
    const int bin = (int)((rest / v.limit) * 32 + lane);
    if (k >= v.bin_len[bin]) continue;
    const int32_t ln = v.row_id[v.rowcode[slot] & TK_ROW_MASK];
    int64_t p = 0, r = 0;
    bool bad = false;
    {
      const int64_t x = gi.pos[gi.n][ln];
      bad |= x < 0 || x >= gi.L[gi.n];
      p += (x * gi.q[gi.n] / gi.L[gi.n]) * gi.stride[gi.n];
    }
    for (int q = 0; q < gi.N - 1; ++q) {
      const int m = gi.others[q];
      const int32_t l = gi.unlabel[m][v.oidx[q][slot]];
      const int64_t x = gi.pos[m][l];
      bad |= x < 0 || x >= gi.L[m];
      const int64_t b = x * gi.q[m] / gi.L[m];
      p += b * gi.stride[m];
      r += b * gi.rstride[m];
    }
    if (bad) {
      atomicOr(err, TK_DEV_ERR_INDEX);
      continue;
    }
    if (priv) atomicAdd(&Es[p], 1ull);
    else atomicAdd(&E[p], 1ull);
    const int64_t bit = (int64_t)ln * gi.Rn + r;
    atomicOr(&bits[bit >> 5], 1u << (bit & 31));
  }
  __syncthreads();
  if (priv)
    for (int i = threadIdx.x; i < P; i += blockDim.x)
      if (Es[i]) atomicAdd(&E[i], Es[i]);
}

// MediumG: every present (slice, other cell) pair adds one to R of its processor
__global__ void k_mediumg_count(const uint32_t* __restrict__ bits, int64_t nwords, const GridInfo gi,
                                unsigned long long* __restrict__ R) {
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nwords; w += (int64_t)gridDim.x * blockDim.x) {
    uint32_t word = bits[w];
    while (word) {
      const int b = __ffs(word) - 1;
      word &= word - 1;
      const int64_t bit = w * 32 + b;
      const int64_t ln = bit / gi.Rn;
      int64_t r = bit - ln * gi.Rn;
      int64_t p = (gi.pos[gi.n][ln] * gi.q[gi.n] / gi.L[gi.n]) * gi.stride[gi.n];
      for (int q = gi.N - 2; q >= 0; --q) {
        const int m = gi.others[q];
        const int64_t bm = r / gi.rstride[m];
        r -= bm * gi.rstride[m];
        p += bm * gi.stride[m];
      }
      atomicAdd(&R[p], 1ull);
    }
  }
}

// E_max, R_sum, R_max over the P processors (one CTA, fixed order)
__global__ void k_scheme_reduce(const unsigned long long* __restrict__ E, const unsigned long long* __restrict__ R, int P,
                                int64_t* __restrict__ out) {
  __shared__ unsigned long long se[256], sr[256], sm[256];
  unsigned long long emax = 0, rsum = 0, rmax = 0;
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    emax = max(emax, E[i]);
    rsum += R[i];
    rmax = max(rmax, R[i]);
  }
  se[threadIdx.x] = emax;
  sr[threadIdx.x] = rsum;
  sm[threadIdx.x] = rmax;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      se[threadIdx.x] = max(se[threadIdx.x], se[threadIdx.x + s]);
      sr[threadIdx.x] += sr[threadIdx.x + s];
      sm[threadIdx.x] = max(sm[threadIdx.x], sm[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = (int64_t)se[0];
    out[1] = (int64_t)sr[0];
    out[2] = (int64_t)sm[0];
  }
}

unsigned grid_for(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>(tk_ceil_div(n, 256), 8 * 1024)); }

CopyView view_of(const tucker_ctx* c, int n) {
  const tk_mode& md = c->mode[n];
  CopyView v{};
  v.rowcode = md.rowcode;
  for (int q = 0; q < c->N - 1; ++q) v.oidx[q] = md.oidx[q];
  v.bin_len = md.bin_len;
  v.row_id = md.row_id;
  v.Pa = md.Pa;
  v.limit = md.limit;
  v.cap = md.cap;
  return v;
}

}  // namespace

std::vector<int> tk_mediumg_grid(const int64_t* L, int N, int P) {
  std::vector<int> f;
  int x = P;
  for (int d = 2; (int64_t)d * d <= x; ++d)
    while (x % d == 0) {
      f.push_back(d);
      x /= d;
    }
  if (x > 1) f.push_back(x);
  std::sort(f.rbegin(), f.rend());
  std::vector<int> q(N, 1);
  for (int fac : f) {
    int best = 0;
    for (int m = 1; m < N; ++m)
      if (L[m] * q[best] > L[best] * q[m]) best = m;  // L_m / q_m > L_best / q_best (products < 2^62)
    q[best] *= fac;
  }
  return q;
}

void tk_scheme_metrics(tucker_ctx* c, int n, int scheme, int P, const int32_t* const* d_pos, int64_t* out3,
                       int64_t* d_E, int64_t* d_R, cudaStream_t s) {
  if (scheme != 1 && scheme != 2) tk_throw(TUCKER_ERR_ARG, "scheme must be 1 (CoarseG) or 2 (MediumG)");
  if (P < 1) tk_throw(TUCKER_ERR_ARG, "P must be >= 1");
  if (!d_pos) tk_throw(TUCKER_ERR_ARG, "NULL permutation array");
  for (int m = 0; m < c->N; ++m)
    if ((scheme == 2 || m == n) && !d_pos[m]) tk_throw(TUCKER_ERR_ARG, "NULL permutation array");
  c->alloc_stream = s;
  const CopyView v = view_of(c, n);
  const int64_t Ln = c->L[n];
  unsigned long long* E = (unsigned long long*)tk_dev_alloc(c, (size_t)P * 8);
  unsigned long long* R = (unsigned long long*)tk_dev_alloc(c, (size_t)P * 8);
  int64_t* o = (int64_t*)tk_dev_alloc(c, 3 * 8);
  TK_CUDA(cudaMemsetAsync(E, 0, (size_t)P * 8, s));
  TK_CUDA(cudaMemsetAsync(R, 0, (size_t)P * 8, s));
  std::vector<std::pair<void*, size_t>> tmp;
  if (scheme == 1) {
    int64_t* cnt = (int64_t*)tk_dev_alloc(c, (size_t)Ln * 8);
    int64_t* bp = (int64_t*)tk_dev_alloc(c, (size_t)(Ln + 1) * 8);
    int64_t* H = (int64_t*)tk_dev_alloc(c, (size_t)(Ln + 1) * 8);
    const size_t tb = std::max<size_t>(tk_scan_tmp_bytes(Ln + 1, 8), 16);
    void* st = tk_dev_alloc(c, tb);
    int32_t* seen = (int32_t*)tk_dev_alloc(c, (size_t)Ln * 4);
    tmp = {{cnt, (size_t)Ln * 8}, {bp, (size_t)(Ln + 1) * 8}, {H, (size_t)(Ln + 1) * 8}, {st, tb}, {seen, (size_t)Ln * 4}};
    TK_CUDA(cudaMemsetAsync(cnt, 0, (size_t)Ln * 8, s));
    TK_CUDA(cudaMemsetAsync(bp, 0, (size_t)(Ln + 1) * 8, s));
    TK_CUDA(cudaMemsetAsync(seen, 0, (size_t)Ln * 4, s));
    k_slice_sizes<<<(unsigned)tk_ceil_div(v.Pa, 128), 128, 0, s>>>(v, cnt);
    k_by_position<<<grid_for(Ln), 256, 0, s>>>(cnt, d_pos[n], Ln, bp, seen, c->err);
    tk_exclusive_scan_i64(bp, H, Ln + 1, st, s);
    k_coarseg<<<grid_for(Ln), 256, 0, s>>>(cnt, d_pos[n], H, Ln, P, c->nnz, E, R);
    TK_CUDA(cudaGetLastError());
  } else {
    const std::vector<int> q = tk_mediumg_grid(c->L, c->N, P);
    GridInfo gi{};
    gi.N = c->N;
    gi.n = n;
    int64_t st = 1;
    for (int m = 0; m < c->N; ++m) {
      gi.q[m] = q[m];
      gi.L[m] = c->L[m];
      gi.stride[m] = st;
      st *= q[m];
      gi.pos[m] = d_pos[m];
      gi.unlabel[m] = c->unlabel[m];
    }
    int64_t rs = 1;
    int no = 0;
    for (int m = 0; m < c->N; ++m) {
      if (m == n) continue;
      gi.others[no++] = m;
      gi.rstride[m] = rs;
      rs *= q[m];
    }
    gi.Rn = rs;
    const int64_t nbits = Ln * gi.Rn;
    if (nbits > ((int64_t)1 << 35)) tk_throw(TUCKER_ERR_ARG, "MediumG presence map too large (L_n x P / q_n > 2^35)");
    const int64_t nwords = tk_ceil_div(nbits, 32);
    uint32_t* bits = (uint32_t*)tk_dev_alloc(c, (size_t)nwords * 4);
    tmp = {{bits, (size_t)nwords * 4}};
    TK_CUDA(cudaMemsetAsync(bits, 0, (size_t)nwords * 4, s));
    const size_t shm = P <= 4096 ? (size_t)P * 8 : 0;
    k_mediumg_elems<<<grid_for(v.cap), 256, shm, s>>>(v, gi, P, E, bits, c->err);
    k_mediumg_count<<<grid_for(nwords), 256, 0, s>>>(bits, nwords, gi, R);
    TK_CUDA(cudaGetLastError());
  }
  k_scheme_reduce<<<1, 256, 0, s>>>(E, R, P, o);
  TK_CUDA(cudaGetLastError());
  if (d_E) TK_CUDA(cudaMemcpyAsync(d_E, E, (size_t)P * 8, cudaMemcpyDeviceToDevice, s));
  if (d_R) TK_CUDA(cudaMemcpyAsync(d_R, R, (size_t)P * 8, cudaMemcpyDeviceToDevice, s));
  TK_CUDA(cudaMemcpyAsync(out3, o, 3 * 8, cudaMemcpyDeviceToHost, s));
  TK_CUDA(cudaStreamSynchronize(s));
  for (auto& t : tmp) tk_dev_free(c, t.first, t.second);
  tk_dev_free(c, o, 3 * 8);
  tk_dev_free(c, R, (size_t)P * 8);
  tk_dev_free(c, E, (size_t)P * 8);
}
