// Device-wide exclusive scan and stable LSD radix sort used by the Lite
// partitioner (slice histogram -> slice order -> element placement).
// No spin-waits: every scan is the classic reduce-then-scan in separate launches.
#include "tk_common.cuh"

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

template <typename T>
__device__ T block_exclusive_scan(T v, T* total) {
  __shared__ T warp_sums[kScanThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[w] = x;
  __syncthreads();
  if (w == 0) {
    T s = lane < kScanThreads / 32 ? warp_sums[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < kScanThreads / 32) warp_sums[lane] = s;  // inclusive over warps
  }
  __syncthreads();
  T warp_prefix = w ? warp_sums[w - 1] : T(0);
  *total = warp_sums[kScanThreads / 32 - 1];
  __syncthreads();
  return warp_prefix + x - v;
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_scan_block(const T* in, T* out, int64_t n, T* block_sums) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  T v[kScanItems];
  T local = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = (base + i < n) ? in[base + i] : T(0);
    local += v[i];
  }
  T total;
  T run = block_exclusive_scan<T>(local, &total);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) out[base + i] = run;
    run += v[i];
  }
  if (threadIdx.x == 0 && block_sums) block_sums[blockIdx.x] = total;
}

template <typename T>
__global__ void k_scan_add(T* out, int64_t n, const T* offs) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  const T o = offs[blockIdx.x];
  for (int i = threadIdx.x; i < kScanTile; i += blockDim.x) {
    const int64_t j = base + i;
    if (j < n) out[j] += o;
  }
}

template <typename T>
void scan_impl(const T* in, T* out, int64_t n, T* tmp, cudaStream_t s) {
  if (n <= 0) return;
  const int64_t nb = tk_ceil_div(n, kScanTile);
  k_scan_block<T><<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, nb > 1 ? tmp : nullptr);
  TK_CUDA(cudaGetLastError());
  if (nb > 1) {
    scan_impl<T>(tmp, tmp, nb, tmp + nb, s);
    k_scan_add<T><<<(unsigned)nb, 256, 0, s>>>(out, n, tmp);
    TK_CUDA(cudaGetLastError());
  }
}

// ---------------------------------------------------------------- radix sort
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 8;  // 32-element chunks per warp
constexpr int kSortTile = kSortThreads * kSortItems;

__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint32_t* keys, int64_t n, int shift,
                                                              int32_t* hist, int nb) {
  __shared__ int h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  for (int i = threadIdx.x; i < kSortTile; i += kSortThreads) {
    const int64_t j = base + i;
    if (j < n) atomicAdd(&h[(keys[j] >> shift) & 255u], 1);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: warp w owns the tile's elements [w*256, (w+1)*256), visited in
// order 32 at a time; ranks among equal digits come from __match_any_sync.
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(const uint32_t* keys, const int32_t* vals,
                                                                 uint32_t* okeys, int32_t* ovals, int64_t n,
                                                                 int shift, const int32_t* offs, int nb) {
  __shared__ int whist[kSortWarps][256];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kSortWarps * 256; i += kSortThreads) (&whist[0][0])[i] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSortTile + (int64_t)w * (32 * kSortItems);
  uint32_t k[kSortItems];
  int32_t v[kSortItems];
  int rank[kSortItems], dig[kSortItems];
#pragma unroll
  for (int c = 0; c < kSortItems; ++c) {
    const int64_t i = base + c * 32 + lane;
    const bool ok = i < n;
    k[c] = ok ? keys[i] : 0u;
    v[c] = ok ? vals[i] : 0;
    const int d = ok ? (int)((k[c] >> shift) & 255u) : 256;
    dig[c] = d;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int r = __popc(peers & ((1u << lane) - 1u));
    const int before = d < 256 ? whist[w][d] : 0;
    __syncwarp();
    if (d < 256 && r == 0) whist[w][d] += __popc(peers);
    __syncwarp();
    rank[c] = before + r;
  }
  __syncthreads();
  {
    const int d = threadIdx.x;
    int run = offs[(int64_t)d * nb + blockIdx.x];
    for (int ww = 0; ww < kSortWarps; ++ww) {
      const int t = whist[ww][d];
      whist[ww][d] = run;
      run += t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < kSortItems; ++c) {
    if (dig[c] < 256) {
      const int pos = whist[w][dig[c]] + rank[c];
      okeys[pos] = k[c];
      ovals[pos] = v[c];
    }
  }
}

}  // namespace

size_t tk_scan_tmp_bytes(int64_t n, size_t esz) {
  size_t total = 0;
  int64_t m = n;
  while (m > 1) {
    m = tk_ceil_div(m, kScanTile);
    total += (size_t)m * esz;
  }
  return total + 256;
}

void tk_exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, void* tmp, cudaStream_t s) {
  scan_impl<int32_t>(in, out, n, (int32_t*)tmp, s);
}

void tk_exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, void* tmp, cudaStream_t s) {
  scan_impl<int64_t>(in, out, n, (int64_t*)tmp, s);
}

size_t tk_sort_tmp_bytes(int64_t n) {
  const int64_t nb = tk_ceil_div(n > 0 ? n : 1, kSortTile);
  const int64_t h = 256 * nb;
  return (size_t)h * 4 + tk_scan_tmp_bytes(h, 4) + 256;
}

void tk_radix_sort_pairs(uint32_t* keys, int32_t* vals, uint32_t* keys_alt, int32_t* vals_alt, int64_t n,
                         int bits, void* tmp, cudaStream_t s, uint32_t** keys_out, int32_t** vals_out) {
  uint32_t* kin = keys;
  int32_t* vin = vals;
  uint32_t* kout = keys_alt;
  int32_t* vout = vals_alt;
  if (n > 0) {
    const int nb = (int)tk_ceil_div(n, kSortTile);
    int32_t* hist = (int32_t*)tmp;
    void* scan_tmp = (char*)tmp + (size_t)256 * nb * 4;
    for (int shift = 0; shift < bits; shift += 8) {
      k_radix_hist<<<nb, kSortThreads, 0, s>>>(kin, n, shift, hist, nb);
      TK_CUDA(cudaGetLastError());
      tk_exclusive_scan_i32(hist, hist, (int64_t)256 * nb, scan_tmp, s);
      k_radix_scatter<<<nb, kSortThreads, 0, s>>>(kin, vin, kout, vout, n, shift, hist, nb);
      TK_CUDA(cudaGetLastError());
      std::swap(kin, kout);
      std::swap(vin, vout);
    }
  }
  *keys_out = kin;
  *vals_out = vin;
}
