// Gram matrix W = Z^T Z of the compact penultimate matrix on the 5th-generation
// tensor cores (tcgen05, kind::tf32) -- the FP32 context's first factor-update
// step.  Z is R x Khat (row-major FP32, Khat <= 128, Khat % 4 == 0).
//
// Each value is split into hi = TF32(z) (mantissa truncated) and lo = z - hi
// (exact in FP32).  Since hi^T hi is symmetric,
//     W = hi^T hi + hi^T lo + lo^T hi = sym(D),  D = hi^T hi + hi^T (2 lo),
// with sym(D) = (D + D^T) / 2: two MMAs per K-step instead of three, the
// symmetrisation done in the final FP64 reduction (lo^T lo, below FP32
// resolution, is dropped).
//
// One persistent CTA per SM takes a contiguous range of rows.  Per batch of 32
// rows:
//   * the rows (one contiguous span) arrive by a bulk async copy into one of 8
//     raw stages (mbarrier with transaction count), issued 8 batches ahead;
//   * 256 threads transpose them into the K-major, 128-byte-swizzled operand
//     layout (M = Z's column index padded to 128, K = the batch's rows) as hi
//     and 2 lo;
//   * one thread issues 4 K-steps x 2 MMAs into one of two 128-column FP32
//     accumulators in tensor memory and commits them to the operand stage's
//     mbarrier.
// The accumulators alternate every 8 batches (256 rows): while the tensor core
// fills one, the threads read the other back (tcgen05.ld) and add it with
// Kahan compensation into per-thread register sums -- each thread's fragment
// is exactly the 64 entries it owns -- so every FP32 sum inside the tensor
// core covers at most 256 rows.  Partials are reduced in FP64 in a fixed
// order.  Every mbarrier wait is bounded; a timeout sets TK_DEV_ERR_TIMEOUT and
// the CTA waits (bounded) for its copies and MMAs in flight, releases its
// tensor memory and returns.
#include <algorithm>

#include "tk_common.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kBatch = 32;        // rows of Z per MMA batch (one 128-byte swizzle atom of K)
constexpr int kDrainEvery = 8;    // batches per accumulator group
constexpr int kRaw = 8;           // raw-row stages (bulk copies in flight)
constexpr int kOpBytes = 128 * kBatch * 4;  // one 128 x 32 FP32 operand tile (16 KB)
constexpr int kTmemCols = 256;    // two 128-column accumulators
constexpr long long kWaitCycles = 4000000000LL;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (m, k) in a K-major tile with 128-byte swizzle (8-row atoms of 1 KB)
__device__ __forceinline__ uint32_t sw128_off(int m, int k) {
  const int r8 = m & 7;
  return (m >> 3) * 1024 + r8 * 128 + (((k >> 2) ^ r8) << 4) + (k & 3) * 4;
}

__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;            // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset between 8-row atoms
  d |= (uint64_t)1 << 46;            // descriptor version
  d |= (uint64_t)2 << 61;            // 128-byte swizzle
  return d;
}

// kind::tf32 instruction descriptor: D FP32, A and B TF32 K-major, M = 128, N = n
__host__ __device__ constexpr uint32_t idesc_tf32(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar)));
}

__device__ __forceinline__ uint32_t mbar_try(uint32_t addr, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred P1;\n mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n selp.b32 %0, 1, 0, P1;\n}\n"
      : "=r"(done)
      : "r"(addr), "r"(parity)
      : "memory");
  return done;
}

// One thread: wait for the phase with the given parity, bounded by kWaitCycles.
__device__ __forceinline__ bool mbar_wait(const uint64_t* bar, uint32_t parity) {
  const uint32_t addr = smem_u32(bar);
  const long long t0 = clock64();
  while (!mbar_try(addr, parity))
    if (clock64() - t0 > kWaitCycles) return false;
  return true;
}

// Whole warp (converged): the same wait with an outcome common to all lanes,
// so that the warp-collective tcgen05 instructions after it are executed by
// every lane or by none.  Bounded by kWaitCycles and, if cap > 0, by cap polls;
// cap < 0 abandons the wait at once (fault injection).
__device__ __forceinline__ bool mbar_wait_warp(const uint64_t* bar, uint32_t parity, int cap) {
  if (cap < 0) return false;
  const uint32_t addr = smem_u32(bar);
  const long long t0 = clock64();
  for (int polls = 1;; ++polls) {
    const uint32_t done = mbar_try(addr, parity);
    if (__all_sync(0xffffffffu, done)) return true;
    const bool out = clock64() - t0 > kWaitCycles || (cap > 0 && polls >= cap);
    if (__any_sync(0xffffffffu, out)) return false;
  }
}

// bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned) into
// shared memory, completing on `bar`
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

struct GramTcArgs {
  const float* Z;
  int R, Khat;
  int rows_per_cta;
  float* Wpart;  // gridDim.x x 128 x 128: D of each CTA
  int* err;
  int cap;       // polls per wait (0: time bound only)
};

__global__ void __launch_bounds__(kThreads, 1) k_gram_tc(const GramTcArgs a) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* sm = smraw + ((1024 - (smem_u32(smraw) & 1023)) & 1023);
  const int Khat = a.Khat;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // layout: operands [2 stages][hi, 2 lo] | raw [kRaw][kBatch][Khat] | barriers | TMEM slot
  unsigned char* ops = sm;
  float* raw = (float*)(sm + 4 * kOpBytes);
  const int rawStage = kBatch * Khat;  // floats
  uint64_t* raw_full = (uint64_t*)(raw + kRaw * rawStage);
  uint64_t* op_free = raw_full + kRaw;
  uint64_t* acc_done = op_free + 2;
  uint32_t* tslot = (uint32_t*)(acc_done + 2);
  __shared__ int s_fail;

  const int64_t r0 = (int64_t)blockIdx.x * a.rows_per_cta;
  const int64_t r1 = min((int64_t)a.R, r0 + a.rows_per_cta);
  const int nrows = (int)max((int64_t)0, r1 - r0);
  const int nb = (nrows + kBatch - 1) / kBatch;
  const int ncols = (Khat + 15) & ~15;  // MMA N
  const uint32_t idesc = idesc_tf32(ncols);

  // zero the operand tiles once: padding rows m >= Khat stay zero
  for (int i = tid; i < 4 * kOpBytes / 16; i += kThreads) reinterpret_cast<float4*>(ops)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (tid == 0) {
    s_fail = 0;
    for (int i = 0; i < kRaw + 4; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&raw_full[i])), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;

  // thread 0 only
  int issued = 0;   // raw batches issued
  int mma_last = -1;  // last batch whose MMAs were issued
  auto issue_raw = [&](int b) {
    const int rows = min(kBatch, nrows - b * kBatch);
    bulk_load(raw + (b % kRaw) * rawStage, a.Z + (r0 + (int64_t)b * kBatch) * Khat, (uint32_t)(rows * Khat * 4),
              &raw_full[b % kRaw]);
    issued = b + 1;
  };
  if (tid == 0)
    for (int b = 0; b < min(kRaw, nb); ++b) issue_raw(b);

  // Kahan sums of the 64 accumulator entries this thread reads back:
  // D row 32 * (warp % 4) + lane, columns 64 * (warp / 4) + [0, 64)
  float sacc[64], scmp[64];
#pragma unroll
  for (int j = 0; j < 64; ++j) {
    sacc[j] = 0.f;
    scmp[j] = 0.f;
  }
  auto drain = [&](int G) -> bool {
    if (!mbar_wait_warp(&acc_done[G & 1], (uint32_t)((G >> 1) & 1), a.cap)) return false;
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t base = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((G & 1) * 128 + 64 * (warp >> 2));
#pragma unroll
    for (int cc = 0; cc < 64; cc += 16) {
      uint32_t v[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(base + (uint32_t)cc));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float y = __uint_as_float(v[j]) - scmp[cc + j];
        const float t = sacc[cc + j] + y;
        scmp[cc + j] = (t - sacc[cc + j]) - y;
        sacc[cc + j] = t;
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    return true;
  };

  // Warp 0 only issues copies and MMAs (an MMA issue blocks while the tensor
  // core is busy, ~0.8 k cycles per batch); warps 1-7 transpose and split.
  // This thread's (column m, 4-row chunk) pairs of the transposition, the same
  // for every batch: at most kPairs per thread (Khat * kBatch / 4 <= 1024).
  constexpr int kXT = kThreads - 32;
  constexpr int kPairs = (128 * (kBatch / 4) + kXT - 1) / kXT;
  int pm[kPairs], pc[kPairs];
  uint32_t poff[kPairs];
#pragma unroll
  for (int i = 0; i < kPairs; ++i) {
    const int pidx = (tid - 32) + i * kXT;
    pm[i] = (warp > 0 && pidx < Khat * (kBatch / 4)) ? pidx % Khat : -1;
    pc[i] = pm[i] >= 0 ? pidx / Khat : 0;
    poff[i] = pm[i] >= 0 ? sw128_off(pm[i], 4 * pc[i]) : 0u;
  }

  int b = 0;
  for (; b < nb; ++b) {
    const int slot = b % kRaw, st = b & 1;
    bool okb = true;
    if (warp > 0) {
      okb = mbar_wait_warp(&raw_full[slot], (uint32_t)((b / kRaw) & 1), a.cap);
      // operand stage st is free once the MMAs of batch b - 2 are done
      if (okb && b >= 2) okb = mbar_wait_warp(&op_free[st], (uint32_t)(((b - 2) >> 1) & 1), a.cap);
    }
    if (!okb) {
      atomicOr(&s_fail, 1);
    } else if (warp > 0) {
      const int rows = min(kBatch, nrows - b * kBatch);
      const float* rw = raw + slot * rawStage;
      unsigned char* hi = ops + st * 2 * kOpBytes;
      unsigned char* lo = hi + kOpBytes;
      float zv[kPairs][4];
#pragma unroll
      for (int i = 0; i < kPairs; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int r = 4 * pc[i] + q;
          zv[i][q] = (pm[i] >= 0 && r < rows) ? rw[r * Khat + pm[i]] : 0.f;
        }
#pragma unroll
      for (int i = 0; i < kPairs; ++i) {
        if (pm[i] < 0) continue;
        float h4[4], l4[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float h = __uint_as_float(__float_as_uint(zv[i][q]) & 0xFFFFE000u);
          h4[q] = h;
          l4[q] = 2.f * (zv[i][q] - h);
        }
        *reinterpret_cast<float4*>(hi + poff[i]) = make_float4(h4[0], h4[1], h4[2], h4[3]);
        *reinterpret_cast<float4*>(lo + poff[i]) = make_float4(l4[0], l4[1], l4[2], l4[3]);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (s_fail) break;
    if (tid == 0) {
      // raw stage `slot` is free: every thread has passed its reads
      if (b + kRaw < nb) issue_raw(b + kRaw);
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int G = b / kDrainEvery;
      const uint32_t dacc = tmem + (uint32_t)((G & 1) * 128);
      const uint64_t dh = sdesc_sw128(smem_u32(ops + st * 2 * kOpBytes));
      const uint64_t dl = sdesc_sw128(smem_u32(ops + st * 2 * kOpBytes + kOpBytes));
      const bool first = (b % kDrainEvery) == 0;
#pragma unroll
      for (int s = 0; s < kBatch / 8; ++s) {
        const uint64_t k = (uint64_t)(2 * s);  // +32 bytes per K-step of 8
        mma_tf32(dacc, dh + k, dh + k, idesc, (first && s == 0) ? 0u : 1u);
        mma_tf32(dacc, dh + k, dl + k, idesc, 1u);
      }
      mma_commit(&op_free[st]);
      if ((b % kDrainEvery) == kDrainEvery - 1 || b == nb - 1) mma_commit(&acc_done[G & 1]);
      mma_last = b;
    }
    // read back the previous group while this group's first MMAs run
    if ((b % kDrainEvery) == 0 && b > 0)
      if (!drain(b / kDrainEvery - 1)) atomicOr(&s_fail, 1);
  }
  if (!s_fail && nb > 0)
    if (!drain((nb - 1) / kDrainEvery)) atomicOr(&s_fail, 1);
  __syncthreads();
  const bool failed = s_fail != 0;
  if (tid == 0 && failed) {
    // let the copies and MMAs in flight finish (bounded) before the memory goes away
    for (int x = max(0, b); x < issued; ++x) mbar_wait(&raw_full[x % kRaw], (uint32_t)((x / kRaw) & 1));
    if (mma_last >= 0) mbar_wait(&op_free[mma_last & 1], (uint32_t)((mma_last >> 1) & 1));
    atomicOr(a.err, TK_DEV_ERR_TIMEOUT);
  }
  float* out = a.Wpart + (int64_t)blockIdx.x * 128 * 128;
  {
    const int row = 32 * (warp & 3) + lane, c0 = 64 * (warp >> 2);
#pragma unroll
    for (int j = 0; j < 64; j += 4) {
      float4 v = make_float4(sacc[j], sacc[j + 1], sacc[j + 2], sacc[j + 3]);
      if (failed) v = make_float4(0.f, 0.f, 0.f, 0.f);
      *reinterpret_cast<float4*>(out + row * 128 + c0 + j) = v;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

// W[i][j] = (S[i][j] + S[j][i]) / 2 with S = sum of the CTA partials in split
// order (FP64); 8 lanes per entry, each over every 8th split, combined by a
// fixed shuffle tree.
__global__ void k_gram_tc_reduce(const float* __restrict__ Wpart, int nsplit, int Khat, double* __restrict__ W) {
  const int64_t total = (int64_t)Khat * Khat;
  const int part = threadIdx.x & 7;
  const int64_t per_pass = ((int64_t)gridDim.x * blockDim.x) >> 3;
  for (int64_t base = 0; base < total; base += per_pass) {  // uniform trip count for every lane
    const int64_t idx0 = base + (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3);
    const bool live = idx0 < total;
    const int64_t idx = live ? idx0 : 0;
    const int i = (int)(idx / Khat), j = (int)(idx - (int64_t)i * Khat);
    double s = 0.0, t = 0.0;
    if (live)
      for (int sp = part; sp < nsplit; sp += 8) {
        s += (double)Wpart[(int64_t)sp * 128 * 128 + i * 128 + j];
        t += (double)Wpart[(int64_t)sp * 128 * 128 + j * 128 + i];
      }
    s += t;
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    s += __shfl_xor_sync(0xffffffffu, s, 4);
    if (part == 0 && live) W[idx] = 0.5 * s;
  }
}

size_t smem_bytes(int Khat) {
  return 1024 + (size_t)4 * kOpBytes + (size_t)kRaw * kBatch * Khat * 4 + (size_t)8 * (kRaw + 4) + 16;
}

}  // namespace

bool tk_gram_tc_supported(int Khat) {
  return Khat >= 8 && Khat <= 128 && Khat % 4 == 0 && smem_bytes(Khat) <= 225 * 1024;
}

// W (Khat x Khat FP64) = Z^T Z; Wpart holds the per-CTA partials (128 x 128 FP32 each).
void tk_gram_tc(tucker_ctx* c, const float* Z, int R, int Khat, float* Wpart, size_t Wpart_elems, double* W,
                cudaStream_t s) {
  int nblk = std::max(1, std::min(c->sm_count, (int)tk_ceil_div(R, 1024)));
  while ((size_t)nblk * 128 * 128 > Wpart_elems && nblk > 1) --nblk;
  GramTcArgs a{};
  a.Z = Z;
  a.R = R;
  a.Khat = Khat;
  a.rows_per_cta = (int)tk_ceil_div(tk_ceil_div(R, nblk), kBatch) * kBatch;
  nblk = (int)std::max<int64_t>(1, tk_ceil_div(R, a.rows_per_cta));
  a.Wpart = Wpart;
  a.err = c->err;
  a.cap = c->wait_cap;
  const size_t shm = smem_bytes(Khat);
  static bool attr = false;
  if (!attr) {
    TK_CUDA(cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 225 * 1024));
    attr = true;
  }
  k_gram_tc<<<nblk, kThreads, shm, s>>>(a);
  TK_CUDA(cudaGetLastError());
  const unsigned g2 = (unsigned)std::min<int64_t>(tk_ceil_div((int64_t)Khat * Khat * 8, 256), 8192);
  k_gram_tc_reduce<<<g2, 256, 0, s>>>(Wpart, nblk, Khat, W);
  TK_CUDA(cudaGetLastError());
}
