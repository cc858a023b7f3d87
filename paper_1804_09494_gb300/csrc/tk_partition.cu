// Lite distribution along one mode (Section 6.1, Fig. 7) as a device pass,
// with one bin per TTM-chain thread, and the permuted ("multi-policy",
// Section 3) copy of the tensor that the TTM-chain kernels stream.
//
// The sequential pseudocode is evaluated in closed form:
//  * Stage 1 sends sorted slice t (0-based) to bin t mod P while the bin stays
//    within limit = ceil(nnz/P).  With H_t = sum of the sizes of the earlier
//    slices of the same residue class, the first violation is
//    t_hat = min{ t : H_t + s_t > limit }, and h(p) = sum_{t<t_hat, t = p mod P} s_t.
//  * Stage 2 walks bins in order and fills each to the limit with the
//    remaining slices laid end to end, so bin p receives exactly the stream
//    range [G_p, G_p + g(p)), G = exclusive scan of the gaps g(p) = limit - h(p).
//    Stream position x therefore belongs to bin max{p : G_p <= x}, which
//    automatically has g(p) > 0.
// Tie-breaks: empty slices dropped; sort by (size, slice id); inside a slice
// the elements are listed by the popularity label of their coordinate along
// the fiber mode f(n) (the other mode with the smallest length), then in
// original COO order, and a stage-2 piece takes the slice's next ones in that
// order.  The copy stores every other coordinate as its popularity label.
#include <algorithm>

#include "tk_common.cuh"

namespace {

struct IdxPtrs {
  const int32_t* p[TK_MAXN];
};

__global__ void k_hist_validate(const int32_t* __restrict__ idx, int64_t nnz, int64_t Ln, int32_t* cnt, int* err) {
  // the whole warp iterates together (stride is a multiple of 32) so the
  // full-mask match below is always executed by all 32 lanes
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  for (int64_t e0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); e0 < nnz; e0 += stride) {
    const int64_t e = e0 + lane;
    const bool in = e < nnz;
    const int32_t l = in ? idx[e] : 0;
    const bool ok = in && l >= 0 && (int64_t)l < Ln;
    if (in && !ok) atomicOr(err, TK_DEV_ERR_INDEX);
    // warp-aggregated increment: one atomic per distinct slice id in the warp
    const int key = ok ? l : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const int leader = __ffs(peers) - 1;
    if (ok && lane == leader) atomicAdd(&cnt[l], __popc(peers));
  }
}

// Popularity sort input: key = nnz - cnt (ascending key = decreasing
// cardinality), value = slice id (id order, so the stable sort breaks ties
// by lower id and lists empty slices last).
__global__ void k_popularity_keys(const int32_t* cnt, int64_t Ln, int64_t nnz, uint32_t* keys, int32_t* vals) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < Ln; l += stride) {
    keys[l] = (uint32_t)(nnz - cnt[l]);
    vals[l] = (int32_t)l;
  }
}

__global__ void k_labels(const int32_t* order, int64_t Ln, int32_t* relabel, int32_t* unlabel) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < Ln; i += stride) {
    relabel[order[i]] = (int32_t)i;
    unlabel[i] = order[i];
  }
}

// Listing order inside a slice, first key: the popularity label of the
// element's fiber-mode coordinate (value = element id, so ties keep COO order).
__global__ void k_fiber_keys(const int32_t* __restrict__ idx_f, const int32_t* __restrict__ relabel_f, int64_t nnz,
                             uint32_t* keys, int32_t* vals) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride) {
    keys[e] = (uint32_t)relabel_f[idx_f[e]];
    vals[e] = (int32_t)e;
  }
}

// Second (major) key: the slice id of each element in the current order.
__global__ void k_slice_keys(const int32_t* __restrict__ idx_n, const int32_t* __restrict__ elem, int64_t nnz,
                             uint32_t* keys) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += stride) keys[i] = (uint32_t)idx_n[elem[i]];
}

__global__ void k_frow(const int32_t* row_id, int R, const int32_t* relabel_n, int32_t* frow) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x) frow[r] = relabel_n[row_id[r]];
}

__global__ void k_nonempty_flags(const int32_t* cnt, int64_t Ln, int32_t* flag) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < Ln; l += stride) flag[l] = cnt[l] > 0;
}

// rowidx[l] = compact row (exclusive scan of the flags), -1 for empty slices;
// row_id[r] = l; slice-sort input keys = cnt, vals = slice id (in id order).
__global__ void k_compact_rows(const int32_t* cnt, int64_t Ln, int32_t* rowidx, int32_t* row_id, uint32_t* skeys,
                               int32_t* svals) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < Ln; l += stride) {
    if (cnt[l] > 0) {
      const int32_t r = rowidx[l];
      row_id[r] = (int32_t)l;
      skeys[r] = (uint32_t)cnt[l];
      svals[r] = (int32_t)l;
    } else {
      rowidx[l] = -1;
    }
  }
}

__global__ void k_t_of(const int32_t* order, int R, int32_t* t_of) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < R; t += gridDim.x * blockDim.x) t_of[order[t]] = t;
}

// Stage 1, first violation per residue class p; the global t_hat is the minimum.
__global__ void k_stage1_violation(const uint32_t* s, int R, int P, int64_t limit, int* t_hat) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  int64_t H = 0;
  for (int64_t t = p; t < R; t += P) {
    if (H + (int64_t)s[t] > limit) {
      atomicMin(t_hat, (int)t);
      return;
    }
    H += s[t];
  }
}

// Offsets of stage-1 slices inside their bin and the stage-1 loads h(p).
__global__ void k_stage1_offsets(const uint32_t* s, int t_hat, int P, int32_t* off1, int64_t* hhat) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  int64_t H = 0;
  for (int64_t t = p; t < t_hat; t += P) {
    off1[t] = (int32_t)H;
    H += s[t];
  }
  hhat[p] = H;
}

__global__ void k_gaps(const int64_t* hhat, int P, int64_t limit, int64_t* gap) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < P) gap[p] = limit - hhat[p];
}

__global__ void k_stage2_sizes(const uint32_t* s, int t_hat, int nsplit, int64_t* sz) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nsplit) sz[k] = s[t_hat + k];
}

__device__ __forceinline__ int upper_bound_i64(const int64_t* a, int n, int64_t x) {
  int lo = 0, hi = n;  // first index with a[i] > x
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] <= x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__global__ void k_bins(const int64_t* hhat, const int64_t* gap, const int64_t* Gp, int P, int64_t S2, int64_t limit,
                       int32_t* bin_len, int32_t* gap2, int* err) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const int64_t take = max((int64_t)0, min(S2 - Gp[p], gap[p]));
  const int64_t len = hhat[p] + take;
  if (len > limit) atomicOr(err, TK_DEV_ERR_LIMIT);
  bin_len[p] = (int32_t)len;
  gap2[p] = (int32_t)gap[p];
}

__global__ void k_split_tables(const int32_t* order, const uint32_t* s, const int32_t* rowidx, const int64_t* X,
                               const int64_t* Gp, int P, int t_hat, int nsplit, int32_t* split_row, int32_t* bhead,
                               int32_t* blast) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nsplit) return;
  const int t = t_hat + k;
  split_row[k] = rowidx[order[t]];
  bhead[k] = upper_bound_i64(Gp, P, X[k]) - 1;
  blast[k] = upper_bound_i64(Gp, P, X[k] + (int64_t)s[t] - 1) - 1;
}

template <typename T>
struct ScatterArgs {
  const uint32_t* skey;  // slice id of sorted position i
  const int32_t* sval;   // element id of sorted position i
  const int32_t* slice_start;
  const int32_t* t_of;
  const int32_t* rowidx;
  const int32_t* off1;
  const int64_t* hhat;
  const int64_t* Gp;
  const int64_t* X;
  const int32_t* bhead;
  IdxPtrs idx;
  IdxPtrs relabel;
  const T* val;
  int N, n, P, t_hat;
  int64_t limit, nnz;
  uint32_t* rowcode;
  int32_t* oidx[TK_MAXN - 1];
  T* oval;
  int32_t* perm;
};

template <typename T>
__global__ void k_scatter(const ScatterArgs<T> a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.nnz; i += stride) {
    const int32_t l = (int32_t)a.skey[i];
    const int32_t e = a.sval[i];
    const int64_t j = i - a.slice_start[l];
    const int t = a.t_of[l];
    uint32_t code = (uint32_t)a.rowidx[l];
    int p;
    int64_t k;
    if (t < a.t_hat) {
      p = t % a.P;
      k = a.off1[t] + j;
    } else {
      const int kk = t - a.t_hat;
      const int64_t x = a.X[kk] + j;
      p = upper_bound_i64(a.Gp, a.P, x) - 1;
      k = a.hhat[p] + (x - a.Gp[p]);
      code |= TK_SPLIT_BIT;
      if (p == a.bhead[kk]) code |= TK_HEAD_BIT;
    }
    const int64_t dest = ((int64_t)(p >> 5) * a.limit + k) * 32 + (p & 31);
    a.rowcode[dest] = code;
    int q = 0;
    for (int m = 0; m < a.N; ++m) {
      if (m == a.n) continue;
      a.oidx[q++][dest] = a.relabel.p[m][a.idx.p[m][e]];
    }
    a.oval[dest] = a.val[e];
    a.perm[dest] = e;
  }
}

__global__ void k_stats(const int32_t* bin_len, const int64_t* Gp, const int64_t* gap, const int64_t* X, int nsplit,
                        int64_t S2, int P, int t_hat, unsigned long long* out /* Emax, Rsum, Rmax */) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  int64_t r = t_hat > p ? (int64_t)(t_hat - 1 - p) / P + 1 : 0;
  const int64_t first = Gp[p];
  const int64_t last = min(Gp[p] + gap[p], S2) - 1;
  if (first <= last) {
    const int kf = upper_bound_i64(X, nsplit, first) - 1;
    const int kl = upper_bound_i64(X, nsplit, last) - 1;
    r += kl - kf + 1;
  }
  atomicMax(&out[0], (unsigned long long)bin_len[p]);
  atomicAdd(&out[1], (unsigned long long)r);
  atomicMax(&out[2], (unsigned long long)r);
}

__global__ void k_export(const int32_t* perm, const int32_t* bin_len, const int64_t* bin_ptr, int P, int Pa,
                         int64_t limit, int32_t* out) {
  const int64_t cap = (int64_t)Pa * limit;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; slot < cap; slot += stride) {
    const int lane = (int)(slot & 31);
    const int64_t rest = slot >> 5;
    const int64_t k = rest % limit;
    const int p = (int)((rest / limit) * 32 + lane);
    if (p < P && k < bin_len[p]) out[bin_ptr[p] + k] = perm[slot];
  }
}

__global__ void k_i32_to_i64(const int32_t* in, int64_t* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = in[i];
  if (i == n) out[n] = 0;
}

int bitlen(uint64_t x) {
  int b = 0;
  while (x) {
    ++b;
    x >>= 1;
  }
  return b;
}

// Temporaries of one partition pass, returned when the pass (which ends with a
// stream synchronisation) goes out of scope.
struct TmpPool {
  tucker_ctx* c;
  std::vector<std::pair<void*, size_t>> ptrs;
  explicit TmpPool(tucker_ctx* ctx) : c(ctx) {}
  void* get(size_t bytes) {
    void* p = tk_dev_alloc(c, bytes);
    ptrs.emplace_back(p, bytes);
    return p;
  }
  ~TmpPool() {
    for (auto& q : ptrs) tk_dev_free(c, q.first, q.second);
  }
};

unsigned grid_for(int64_t n, int threads = 256) {
  int64_t b = tk_ceil_div(n > 0 ? n : 1, threads);
  return (unsigned)std::min<int64_t>(b, 1 << 20);
}

template <typename T>
void launch_scatter(ScatterArgs<T>& a, cudaStream_t s) {
  k_scatter<T><<<grid_for(a.nnz), 256, 0, s>>>(a);
  TK_CUDA(cudaGetLastError());
}

}  // namespace

void tk_relabel_modes(tucker_ctx* c, const int32_t* const* d_idx, cudaStream_t s) {
  const int64_t nnz = c->nnz;
  for (int n = 0; n < c->N; ++n) {
    int f = -1;
    for (int m = 0; m < c->N; ++m)
      if (m != n && (f < 0 || c->L[m] < c->L[f])) f = m;
    c->fiber[n] = f;
  }
  for (int m = 0; m < c->N; ++m) {
    const int64_t Lm = c->L[m];
    TmpPool tmp(c);
    int32_t* cnt = (int32_t*)tmp.get(Lm * 4);
    uint32_t* keys[2] = {(uint32_t*)tmp.get(Lm * 4), (uint32_t*)tmp.get(Lm * 4)};
    int32_t* vals[2] = {(int32_t*)tmp.get(Lm * 4), (int32_t*)tmp.get(Lm * 4)};
    void* sort_tmp = tmp.get(tk_sort_tmp_bytes(Lm));
    TK_CUDA(cudaMemsetAsync(cnt, 0, Lm * 4, s));
    TK_CUDA(cudaMemsetAsync(c->err, 0, sizeof(int), s));
    k_hist_validate<<<grid_for(nnz), 256, 0, s>>>(d_idx[m], nnz, Lm, cnt, c->err);
    TK_CUDA(cudaGetLastError());
    int herr = 0;
    TK_CUDA(cudaMemcpyAsync(&herr, c->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    TK_CUDA(cudaStreamSynchronize(s));
    if (herr & TK_DEV_ERR_INDEX) tk_throw(TUCKER_ERR_INDEX, "a coordinate of mode " + std::to_string(m) + " is outside [0, L)");
    k_popularity_keys<<<grid_for(Lm), 256, 0, s>>>(cnt, Lm, nnz, keys[0], vals[0]);
    TK_CUDA(cudaGetLastError());
    uint32_t* ko;
    int32_t* vo;
    tk_radix_sort_pairs(keys[0], vals[0], keys[1], vals[1], Lm, bitlen((uint64_t)nnz), sort_tmp, s, &ko, &vo);
    c->relabel[m] = (int32_t*)tk_alloc(c, (size_t)Lm * 4);
    c->unlabel[m] = (int32_t*)tk_alloc(c, (size_t)Lm * 4);
    k_labels<<<grid_for(Lm), 256, 0, s>>>(vo, Lm, c->relabel[m], c->unlabel[m]);
    TK_CUDA(cudaGetLastError());
    TK_CUDA(cudaStreamSynchronize(s));  // temporaries go out of scope
  }
}

void tk_partition_mode(tucker_ctx* c, int n, const int32_t* const* d_idx, const void* d_val, int P, cudaStream_t s) {
  tk_mode& md = c->mode[n];
  const int64_t nnz = c->nnz;
  const int64_t Ln = c->L[n];
  md.n = n;
  md.P = P;
  md.Pa = (int)tk_ceil_div(P, 32) * 32;
  md.limit = (int)tk_ceil_div(nnz, P);
  md.cap = (int64_t)md.Pa * md.limit;
  if (md.cap >= ((int64_t)1 << 31) - 32) tk_throw(TUCKER_ERR_ARG, "nnz too large for int32 slot indices");

  TmpPool tmp(c);
  int32_t* cnt = (int32_t*)tmp.get(Ln * 4);
  uint32_t* ekey[2] = {(uint32_t*)tmp.get(nnz * 4), (uint32_t*)tmp.get(nnz * 4)};
  int32_t* eval_[2] = {(int32_t*)tmp.get(nnz * 4), (int32_t*)tmp.get(nnz * 4)};
  int32_t* rowidx = (int32_t*)tmp.get(Ln * 4);
  int32_t* slice_start = (int32_t*)tmp.get(Ln * 4);
  int32_t* t_of = (int32_t*)tmp.get(Ln * 4);
  const size_t scan_bytes = std::max(tk_scan_tmp_bytes(Ln, 8), tk_scan_tmp_bytes(P + 1, 8));
  void* scan_tmp = tmp.get(std::max(scan_bytes, tk_sort_tmp_bytes(std::max<int64_t>(nnz, Ln))));
  int* d_scalar = (int*)tmp.get(64);

  TK_CUDA(cudaMemsetAsync(cnt, 0, Ln * 4, s));
  TK_CUDA(cudaMemsetAsync(c->err, 0, sizeof(int), s));
  k_hist_validate<<<grid_for(nnz), 256, 0, s>>>(d_idx[n], nnz, Ln, cnt, c->err);
  TK_CUDA(cudaGetLastError());
  int herr = 0;
  TK_CUDA(cudaMemcpyAsync(&herr, c->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  TK_CUDA(cudaStreamSynchronize(s));
  if (herr & TK_DEV_ERR_INDEX) tk_throw(TUCKER_ERR_INDEX, "a coordinate of mode " + std::to_string(n) + " is outside [0, L)");

  // compact rows: rowidx = exclusive scan of (cnt > 0)
  k_nonempty_flags<<<grid_for(Ln), 256, 0, s>>>(cnt, Ln, rowidx);
  int32_t last_flag = 0;
  TK_CUDA(cudaMemcpyAsync(&last_flag, rowidx + Ln - 1, 4, cudaMemcpyDeviceToHost, s));
  tk_exclusive_scan_i32(rowidx, rowidx, Ln, scan_tmp, s);
  int32_t last_row = 0;
  TK_CUDA(cudaMemcpyAsync(&last_row, rowidx + Ln - 1, 4, cudaMemcpyDeviceToHost, s));
  TK_CUDA(cudaStreamSynchronize(s));
  const int R = last_row + last_flag;
  md.R = R;
  md.row_id = (int32_t*)tk_alloc(c, (size_t)std::max(R, 1) * 4);
  uint32_t* skey[2] = {(uint32_t*)tmp.get((size_t)R * 4), (uint32_t*)tmp.get((size_t)R * 4)};
  int32_t* sval[2] = {(int32_t*)tmp.get((size_t)R * 4), (int32_t*)tmp.get((size_t)R * 4)};
  k_compact_rows<<<grid_for(Ln), 256, 0, s>>>(cnt, Ln, rowidx, md.row_id, skey[0], sval[0]);
  TK_CUDA(cudaGetLastError());
  md.frow = (int32_t*)tk_alloc(c, (size_t)std::max(R, 1) * 4);
  k_frow<<<grid_for(R), 256, 0, s>>>(md.row_id, R, c->relabel[n], md.frow);
  TK_CUDA(cudaGetLastError());
  tk_exclusive_scan_i32(cnt, slice_start, Ln, scan_tmp, s);

  // elements in listing order: by slice id, inside a slice by the popularity
  // label of the fiber-mode coordinate, then by element id (two stable passes,
  // the minor key first)
  const int f = c->fiber[n];
  k_fiber_keys<<<grid_for(nnz), 256, 0, s>>>(d_idx[f], c->relabel[f], nnz, ekey[0], eval_[0]);
  TK_CUDA(cudaGetLastError());
  uint32_t* f_key;
  int32_t* f_val;
  tk_radix_sort_pairs(ekey[0], eval_[0], ekey[1], eval_[1], nnz, bitlen((uint64_t)(c->L[f] - 1)), scan_tmp, s, &f_key,
                      &f_val);
  k_slice_keys<<<grid_for(nnz), 256, 0, s>>>(d_idx[n], f_val, nnz, f_key);
  TK_CUDA(cudaGetLastError());
  uint32_t* es_key;
  int32_t* es_val;
  {
    uint32_t* k_alt = f_key == ekey[0] ? ekey[1] : ekey[0];
    int32_t* v_alt = f_val == eval_[0] ? eval_[1] : eval_[0];
    tk_radix_sort_pairs(f_key, f_val, k_alt, v_alt, nnz, bitlen((uint64_t)(Ln - 1)), scan_tmp, s, &es_key, &es_val);
  }
  // non-empty slices sorted by (cardinality, slice id): the input is in id order and the sort is stable
  uint32_t* ss_key;
  int32_t* ss_val;
  tk_radix_sort_pairs(skey[0], sval[0], skey[1], sval[1], R, bitlen((uint64_t)nnz), scan_tmp, s, &ss_key, &ss_val);
  k_t_of<<<grid_for(R), 256, 0, s>>>(ss_val, R, t_of);

  // stage 1
  int h_that = R;
  TK_CUDA(cudaMemcpyAsync(d_scalar, &h_that, 4, cudaMemcpyHostToDevice, s));
  k_stage1_violation<<<grid_for(P), 256, 0, s>>>(ss_key, R, P, md.limit, d_scalar);
  TK_CUDA(cudaMemcpyAsync(&h_that, d_scalar, 4, cudaMemcpyDeviceToHost, s));
  TK_CUDA(cudaStreamSynchronize(s));
  md.t_hat = h_that;
  const int nsplit = R - h_that;
  md.nsplit = nsplit;
  int32_t* off1 = (int32_t*)tmp.get((size_t)std::max(h_that, 1) * 4);
  int64_t* hhat = (int64_t*)tmp.get((size_t)P * 8);
  int64_t* gap = (int64_t*)tmp.get((size_t)P * 8);
  int64_t* Gp = (int64_t*)tmp.get((size_t)(P + 1) * 8);
  int64_t* X = (int64_t*)tmp.get((size_t)(nsplit + 1) * 8);
  k_stage1_offsets<<<grid_for(P), 256, 0, s>>>(ss_key, h_that, P, off1, hhat);
  k_gaps<<<grid_for(P), 256, 0, s>>>(hhat, P, md.limit, gap);
  tk_exclusive_scan_i64(gap, Gp, P, scan_tmp, s);
  // stage-2 stream offsets X_k of slice t_hat + k
  int64_t S2 = 0;
  if (nsplit > 0) {
    k_stage2_sizes<<<grid_for(nsplit), 256, 0, s>>>(ss_key, h_that, nsplit, X);
    int64_t last_sz = 0;
    TK_CUDA(cudaMemcpyAsync(&last_sz, X + nsplit - 1, 8, cudaMemcpyDeviceToHost, s));
    tk_exclusive_scan_i64(X, X, nsplit, scan_tmp, s);
    int64_t last_x = 0;
    TK_CUDA(cudaMemcpyAsync(&last_x, X + nsplit - 1, 8, cudaMemcpyDeviceToHost, s));
    TK_CUDA(cudaStreamSynchronize(s));
    S2 = last_x + last_sz;
  }

  // permuted copy
  md.bin_len = (int32_t*)tk_alloc(c, (size_t)md.Pa * 4);
  md.gap2 = (int32_t*)tk_alloc(c, (size_t)md.Pa * 4);
  TK_CUDA(cudaMemsetAsync(md.bin_len, 0, (size_t)md.Pa * 4, s));
  TK_CUDA(cudaMemsetAsync(md.gap2, 0, (size_t)md.Pa * 4, s));
  // every slot of the copy holds valid values: padding slots (past a bin's
  // length) stay zero -- row 0, coordinate 0, value 0, element 0 -- so the
  // TTM-chain may read them ahead of use without checks
  md.rowcode = (uint32_t*)tk_alloc(c, (size_t)md.cap * 4);
  TK_CUDA(cudaMemsetAsync(md.rowcode, 0, (size_t)md.cap * 4, s));
  for (int q = 0; q < c->N - 1; ++q) {
    md.oidx[q] = (int32_t*)tk_alloc(c, (size_t)md.cap * 4);
    TK_CUDA(cudaMemsetAsync(md.oidx[q], 0, (size_t)md.cap * 4, s));
  }
  md.val = tk_alloc(c, (size_t)md.cap * c->esz);
  TK_CUDA(cudaMemsetAsync(md.val, 0, (size_t)md.cap * c->esz, s));
  md.perm = (int32_t*)tk_alloc(c, (size_t)md.cap * 4);
  TK_CUDA(cudaMemsetAsync(md.perm, 0, (size_t)md.cap * 4, s));
  TK_CUDA(cudaMemsetAsync(c->err, 0, sizeof(int), s));
  k_bins<<<grid_for(P), 256, 0, s>>>(hhat, gap, Gp, P, S2, md.limit, md.bin_len, md.gap2, c->err);
  TK_CUDA(cudaGetLastError());

  md.split_row = (int32_t*)tk_alloc(c, (size_t)std::max(nsplit, 1) * 4);
  md.split_bhead = (int32_t*)tk_alloc(c, (size_t)std::max(nsplit, 1) * 4);
  int32_t* blast = (int32_t*)tmp.get((size_t)std::max(nsplit, 1) * 4);
  if (nsplit > 0) {
    k_split_tables<<<grid_for(nsplit), 256, 0, s>>>(ss_val, ss_key, rowidx, X, Gp, P, h_that, nsplit, md.split_row,
                                                    md.split_bhead, blast);
    TK_CUDA(cudaGetLastError());
  }

  {
    IdxPtrs ip{}, rl{};
    for (int m = 0; m < c->N; ++m) {
      ip.p[m] = d_idx[m];
      rl.p[m] = c->relabel[m];
    }
    if (c->prec == TUCKER_FP32) {
      ScatterArgs<float> a{};
      a.skey = es_key; a.sval = es_val; a.slice_start = slice_start; a.t_of = t_of; a.rowidx = rowidx;
      a.off1 = off1; a.hhat = hhat; a.Gp = Gp; a.X = X; a.bhead = md.split_bhead; a.idx = ip; a.relabel = rl;
      a.val = (const float*)d_val; a.N = c->N; a.n = n; a.P = P; a.t_hat = h_that; a.limit = md.limit; a.nnz = nnz;
      a.rowcode = md.rowcode; for (int q = 0; q < c->N - 1; ++q) a.oidx[q] = md.oidx[q];
      a.oval = (float*)md.val; a.perm = md.perm;
      launch_scatter(a, s);
    } else {
      ScatterArgs<double> a{};
      a.skey = es_key; a.sval = es_val; a.slice_start = slice_start; a.t_of = t_of; a.rowidx = rowidx;
      a.off1 = off1; a.hhat = hhat; a.Gp = Gp; a.X = X; a.bhead = md.split_bhead; a.idx = ip; a.relabel = rl;
      a.val = (const double*)d_val; a.N = c->N; a.n = n; a.P = P; a.t_hat = h_that; a.limit = md.limit; a.nnz = nnz;
      a.rowcode = md.rowcode; for (int q = 0; q < c->N - 1; ++q) a.oidx[q] = md.oidx[q];
      a.oval = (double*)md.val; a.perm = md.perm;
      launch_scatter(a, s);
    }
  }

  // Section 4.1 metrics
  unsigned long long* d_stats = (unsigned long long*)tmp.get(3 * 8);
  TK_CUDA(cudaMemsetAsync(d_stats, 0, 3 * 8, s));
  k_stats<<<grid_for(P), 256, 0, s>>>(md.bin_len, Gp, gap, X, nsplit, S2, P, h_that, d_stats);
  unsigned long long hs[3];
  TK_CUDA(cudaMemcpyAsync(hs, d_stats, 3 * 8, cudaMemcpyDeviceToHost, s));
  TK_CUDA(cudaMemcpyAsync(&herr, c->err, sizeof(int), cudaMemcpyDeviceToHost, s));

  // fix-up chunks: split slice k spans bins [bhead, blast]; chunks of <= 256 bins
  std::vector<int32_t> hb(std::max(nsplit, 1)), hl(std::max(nsplit, 1));
  if (nsplit > 0) {
    TK_CUDA(cudaMemcpyAsync(hb.data(), md.split_bhead, (size_t)nsplit * 4, cudaMemcpyDeviceToHost, s));
    TK_CUDA(cudaMemcpyAsync(hl.data(), blast, (size_t)nsplit * 4, cudaMemcpyDeviceToHost, s));
  }
  TK_CUDA(cudaStreamSynchronize(s));
  if (herr & TK_DEV_ERR_LIMIT) tk_throw(TUCKER_ERR_STATE, "internal: a Lite bin exceeds the limit");
  md.E_max = (int64_t)hs[0];
  md.R_sum = (int64_t)hs[1];
  md.R_max = (int64_t)hs[2];
  std::vector<int32_t> cs, c0, c1, sc0(nsplit + 1);
  const int CH = 256;
  for (int k = 0; k < nsplit; ++k) {
    sc0[k] = (int)cs.size();
    for (int b = hb[k]; b <= hl[k]; b += CH) {
      cs.push_back(k);
      c0.push_back(b);
      c1.push_back(std::min(hl[k] + 1, b + CH));
    }
  }
  sc0[nsplit] = (int)cs.size();
  md.nchunks = (int)cs.size();
  md.chunk_split = (int32_t*)tk_alloc(c, std::max<size_t>(cs.size(), 1) * 4);
  md.chunk_b0 = (int32_t*)tk_alloc(c, std::max<size_t>(cs.size(), 1) * 4);
  md.chunk_b1 = (int32_t*)tk_alloc(c, std::max<size_t>(cs.size(), 1) * 4);
  md.split_chunk0 = (int32_t*)tk_alloc(c, sc0.size() * 4);
  if (!cs.empty()) {
    TK_CUDA(cudaMemcpyAsync(md.chunk_split, cs.data(), cs.size() * 4, cudaMemcpyHostToDevice, s));
    TK_CUDA(cudaMemcpyAsync(md.chunk_b0, c0.data(), c0.size() * 4, cudaMemcpyHostToDevice, s));
    TK_CUDA(cudaMemcpyAsync(md.chunk_b1, c1.data(), c1.size() * 4, cudaMemcpyHostToDevice, s));
  }
  TK_CUDA(cudaMemcpyAsync(md.split_chunk0, sc0.data(), sc0.size() * 4, cudaMemcpyHostToDevice, s));
  TK_CUDA(cudaStreamSynchronize(s));  // host vectors and temporaries go out of scope
}

void tk_partition_export(tucker_ctx* c, int n, int64_t* d_bin_ptr, int32_t* d_perm, cudaStream_t s) {
  tk_mode& md = c->mode[n];
  c->alloc_stream = s;
  TmpPool tmp(c);
  void* scan_tmp = tmp.get(tk_scan_tmp_bytes(md.P + 1, 8));
  k_i32_to_i64<<<grid_for(md.P + 1), 256, 0, s>>>(md.bin_len, d_bin_ptr, md.P);
  tk_exclusive_scan_i64(d_bin_ptr, d_bin_ptr, md.P + 1, scan_tmp, s);
  k_export<<<grid_for(md.cap), 256, 0, s>>>(md.perm, md.bin_len, d_bin_ptr, md.P, md.Pa, md.limit, d_perm);
  TK_CUDA(cudaGetLastError());
  TK_CUDA(cudaStreamSynchronize(s));
}

// Same export as tk_partition_export, with the scan's temporary supplied by
// the caller (at least tk_scan_tmp_bytes(P + 1, 8) bytes) and no host sync.
void tk_partition_export_into(tucker_ctx* c, int n, int64_t* d_bin_ptr, int32_t* d_perm, void* scan_tmp,
                              cudaStream_t s) {
  tk_mode& md = c->mode[n];
  k_i32_to_i64<<<grid_for(md.P + 1), 256, 0, s>>>(md.bin_len, d_bin_ptr, md.P);
  TK_CUDA(cudaGetLastError());
  tk_exclusive_scan_i64(d_bin_ptr, d_bin_ptr, md.P + 1, scan_tmp, s);
  k_export<<<grid_for(md.cap), 256, 0, s>>>(md.perm, md.bin_len, d_bin_ptr, md.P, md.Pa, md.limit, d_perm);
  TK_CUDA(cudaGetLastError());
}
