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
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "tk_common.cuh"
#include "tk_tc.cuh"

namespace {

using namespace tk_tc;

constexpr int kThreads = 256;
constexpr int kBatch = 32;        // rows of Z per MMA batch (one 128-byte swizzle atom of K)
constexpr int kDrainEvery = 8;    // batches per accumulator group
constexpr int kRaw = 8;           // raw-row stages (bulk copies in flight)
constexpr int kOpBytes = 128 * kBatch * 4;  // one 128 x 32 FP32 operand tile (16 KB)
constexpr int kTmemCols = 256;    // two 128-column accumulators

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

// ---------------------------------------------------------------- tiled form
// For Khat > 128, W is tiled into 128 x 128 blocks (I, J), I <= J.  CTA
// (split s, pair p) forms block (I, J) from the rows of split s:
//   D_IJ = sum_rows hi_I hi_J^T + hi_I lo_J^T + lo_I hi_J^T      (I != J)
//   D_II = sum_rows hi_I hi_I^T + hi_I (2 lo_I)^T                  (I == J, symmetrised when reduced)
// A batch of 32 rows arrives as one or two 32 x 128 boxes of a 2D tensor map
// (columns past Khat and rows past R read as zero); warps 1-7 split and
// transpose them into the K-major operand tiles, thread 0 issues the copies
// and the MMAs; accumulators, drains and waits as in the single-tile form.
constexpr int kTileRaw = 2;                 // raw stages (two boxes each)
constexpr int kBoxBytes = kBatch * 128 * 4;  // one 32 x 128 FP32 box (16 KB)

struct GramTileArgs {
  int R, Khat;
  int npairs;
  int rows_per_split;
  const int2* pairs;  // (I, J), I <= J, in units of 128 columns
  float* Wpart;       // per CTA a 128 x 128 tile
  int* err;
  int cap;
};

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// BF: every value as three BF16 terms z = b0 + b1 + b2 (round to nearest each,
// z - b0 - b1 - b2 = O(2^-27 z)) and W from the six products of order up to
// 2^-18, b0b0 + b0b1 + b1b0 + b0b2 + b2b0 + b1b1, as kind::f16 MMAs (K = 16 per
// instruction, twice the TF32 rate) on 64-byte swizzled tiles; diagonal blocks
// take the same six products.  Otherwise split TF32 as described above.
template <bool BF>
__global__ void __launch_bounds__(kThreads, 1) k_gram_tiles(const __grid_constant__ CUtensorMap tz, const GramTileArgs a) {
  constexpr int kOp = BF ? 128 * kBatch * 2 : kOpBytes;  // one operand tile (8 or 16 KB)
  constexpr int kRowsPer = BF ? 8 : 4;                  // consecutive K (rows) per 16-byte chunk
  constexpr int NT = BF ? 3 : 2;                        // operand tiles per box
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* sm = smraw + ((1024 - (smem_u32(smraw) & 1023)) & 1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int pair = blockIdx.x % a.npairs, split = blockIdx.x / a.npairs;
  const int I = a.pairs[pair].x, J = a.pairs[pair].y;
  const bool diag = I == J;
  const int nstrips = diag ? 1 : 2;
  // layout: operands [2 stages][NT tiles of box I, NT of box J] | raw [kTileRaw][2 boxes] | barriers | TMEM slot
  unsigned char* ops = sm;
  unsigned char* raw = sm + 2 * 2 * NT * kOp;
  uint64_t* raw_full = (uint64_t*)(raw + kTileRaw * 2 * kBoxBytes);
  uint64_t* op_free = raw_full + kTileRaw;
  uint64_t* acc_done = op_free + 2;
  uint32_t* tslot = (uint32_t*)(acc_done + 2);
  __shared__ int s_fail;

  const int64_t r0 = (int64_t)split * a.rows_per_split;
  const int64_t r1 = min((int64_t)a.R, r0 + a.rows_per_split);
  const int nrows = (int)max((int64_t)0, r1 - r0);
  const int nb = (nrows + kBatch - 1) / kBatch;
  const uint32_t idesc = BF ? idesc_bf16(128) : idesc_tf32(128);

  if (tid == 0) {
    s_fail = 0;
    for (int i = 0; i < kTileRaw + 4; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&raw_full[i])), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;

  int issued = 0, mma_last = -1;  // thread 0 only
  auto issue_raw = [&](int b) {
    const int slot = b % kTileRaw;
    uint64_t* bar = &raw_full[slot];
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"((uint32_t)(nstrips * kBoxBytes))
                 : "memory");
    const int y = (int)(r0 + (int64_t)b * kBatch);
    tma_load_2d(raw + slot * 2 * kBoxBytes, &tz, 128 * I, y, bar);
    if (!diag) tma_load_2d(raw + slot * 2 * kBoxBytes + kBoxBytes, &tz, 128 * J, y, bar);
    issued = b + 1;
  };
  if (tid == 0)
    for (int b = 0; b < min(kTileRaw, nb); ++b) issue_raw(b);

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

  // this thread's (box, column m, chunk of kRowsPer rows) triples of the transposition
  constexpr int kXT = kThreads - 32;
  constexpr int kChunks = kBatch / kRowsPer;
  constexpr int kTP = (2 * 128 * kChunks + kXT - 1) / kXT;
  int pbox[kTP], pm[kTP], pc[kTP];
  uint32_t poff[kTP];
#pragma unroll
  for (int i = 0; i < kTP; ++i) {
    const int pidx = (tid - 32) + i * kXT;
    const int bx = pidx / (128 * kChunks), rem = pidx % (128 * kChunks);
    const bool live = warp > 0 && bx < nstrips;
    pbox[i] = bx;
    pm[i] = live ? rem % 128 : -1;
    pc[i] = live ? rem / 128 : 0;
    poff[i] = live ? (BF ? sw64_off(pm[i], kRowsPer * pc[i]) : sw128_off(pm[i], kRowsPer * pc[i])) : 0u;
  }

  int b = 0;
  for (; b < nb; ++b) {
    const int slot = b % kTileRaw, st = b & 1;
    bool okb = true;
    if (warp > 0) {
      okb = mbar_wait_warp(&raw_full[slot], (uint32_t)((b / kTileRaw) & 1), a.cap);
      if (okb && b >= 2) okb = mbar_wait_warp(&op_free[st], (uint32_t)(((b - 2) >> 1) & 1), a.cap);
    }
    if (!okb) {
      atomicOr(&s_fail, 1);
    } else if (warp > 0) {
      const int rows = min(kBatch, nrows - b * kBatch);
      const float* rw = (const float*)(raw + slot * 2 * kBoxBytes);
      float zv[kTP][kRowsPer];
#pragma unroll
      for (int i = 0; i < kTP; ++i)
#pragma unroll
        for (int q = 0; q < kRowsPer; ++q) {
          const int r = kRowsPer * pc[i] + q;
          zv[i][q] = (pm[i] >= 0 && r < rows) ? rw[pbox[i] * (kBoxBytes / 4) + r * 128 + pm[i]] : 0.f;
        }
#pragma unroll
      for (int i = 0; i < kTP; ++i) {
        if (pm[i] < 0) continue;
        unsigned char* hi = ops + (st * 2 * NT + NT * pbox[i]) * kOp;
        unsigned char* lo = hi + kOp;
        if constexpr (BF) {
          uint32_t t2[3][4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            uint32_t t0[3], t1[3];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const float z = zv[i][2 * q + h];
              const __nv_bfloat16 b0 = __float2bfloat16_rn(z);
              const float r1 = z - __bfloat162float(b0);
              const __nv_bfloat16 b1 = __float2bfloat16_rn(r1);
              const __nv_bfloat16 b2 = __float2bfloat16_rn(r1 - __bfloat162float(b1));
              uint32_t* t = h ? t1 : t0;
              t[0] = __bfloat16_as_ushort(b0);
              t[1] = __bfloat16_as_ushort(b1);
              t[2] = __bfloat16_as_ushort(b2);
            }
#pragma unroll
            for (int u = 0; u < 3; ++u) t2[u][q] = t0[u] | (t1[u] << 16);
          }
#pragma unroll
          for (int u = 0; u < 3; ++u)
            *reinterpret_cast<uint4*>(hi + u * kOp + poff[i]) = make_uint4(t2[u][0], t2[u][1], t2[u][2], t2[u][3]);
        } else {
          float h4[4], l4[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float h = __uint_as_float(__float_as_uint(zv[i][q]) & 0xFFFFE000u);
            h4[q] = h;
            l4[q] = diag ? 2.f * (zv[i][q] - h) : zv[i][q] - h;
          }
          *reinterpret_cast<float4*>(hi + poff[i]) = make_float4(h4[0], h4[1], h4[2], h4[3]);
          *reinterpret_cast<float4*>(lo + poff[i]) = make_float4(l4[0], l4[1], l4[2], l4[3]);
        }
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (s_fail) break;
    if (tid == 0) {
      if (b + kTileRaw < nb) issue_raw(b + kTileRaw);
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int G = b / kDrainEvery;
      const uint32_t dacc = tmem + (uint32_t)((G & 1) * 128);
      auto desc = [&](int t) {
        return BF ? sdesc_sw64(smem_u32(ops + (st * 2 * NT + t) * kOp)) : sdesc_sw128(smem_u32(ops + (st * 2 * NT + t) * kOp));
      };
      const uint64_t aI0 = desc(0), aI1 = desc(1), aI2 = BF ? desc(2) : 0;
      const uint64_t aJ0 = diag ? aI0 : desc(NT), aJ1 = diag ? aI1 : desc(NT + 1), aJ2 = BF ? (diag ? aI2 : desc(NT + 2)) : 0;
      const bool first = (b % kDrainEvery) == 0;
      // 32 bytes of K per instruction: 8 TF32 or 16 BF16 values
      constexpr int kSteps = BF ? kBatch / 16 : kBatch / 8;
#pragma unroll
      for (int s2 = 0; s2 < kSteps; ++s2) {
        const uint64_t k = (uint64_t)(2 * s2);
        if constexpr (BF) {
          mma_bf16(dacc, aI0 + k, aJ0 + k, idesc, (first && s2 == 0) ? 0u : 1u);
          mma_bf16(dacc, aI0 + k, aJ1 + k, idesc, 1u);
          mma_bf16(dacc, aI1 + k, aJ0 + k, idesc, 1u);
          mma_bf16(dacc, aI0 + k, aJ2 + k, idesc, 1u);
          mma_bf16(dacc, aI2 + k, aJ0 + k, idesc, 1u);
          mma_bf16(dacc, aI1 + k, aJ1 + k, idesc, 1u);
        } else {
          mma_tf32(dacc, aI0 + k, aJ0 + k, idesc, (first && s2 == 0) ? 0u : 1u);
          mma_tf32(dacc, aI0 + k, aJ1 + k, idesc, 1u);
          if (!diag) mma_tf32(dacc, aI1 + k, aJ0 + k, idesc, 1u);
        }
      }
      mma_commit(&op_free[st]);
      if ((b % kDrainEvery) == kDrainEvery - 1 || b == nb - 1) mma_commit(&acc_done[G & 1]);
      mma_last = b;
    }
    if ((b % kDrainEvery) == 0 && b > 0)
      if (!drain(b / kDrainEvery - 1)) atomicOr(&s_fail, 1);
  }
  if (!s_fail && nb > 0)
    if (!drain((nb - 1) / kDrainEvery)) atomicOr(&s_fail, 1);
  __syncthreads();
  const bool failed = s_fail != 0;
  if (tid == 0 && failed) {
    for (int x = max(0, b); x < issued; ++x) mbar_wait(&raw_full[x % kTileRaw], (uint32_t)((x / kTileRaw) & 1));
    if (mma_last >= 0) mbar_wait(&op_free[mma_last & 1], (uint32_t)((mma_last >> 1) & 1));
    atomicOr(a.err, TK_DEV_ERR_TIMEOUT);
  }
  float* out = a.Wpart + (int64_t)blockIdx.x * 128 * 128;
  {
    const int row = 32 * (warp & 3) + lane, c0 = 64 * (warp >> 2);
#pragma unroll
    for (int j = 0; j < 64; j += 4) {
      float4 v = make_float4(sacc[j], sacc[j + 1], sacc[j + 2], sacc[j + 3]);
      if (failed || nb == 0) v = make_float4(0.f, 0.f, 0.f, 0.f);
      *reinterpret_cast<float4*>(out + row * 128 + c0 + j) = v;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

// Block (I, J) of W from the per-split tiles, summed in split order in FP64:
// W_IJ = S and W_JI = S^T off the diagonal, W_II = (S + S^T) / 2.
__global__ void k_gram_tiles_reduce(const float* __restrict__ Wpart, int npairs, int nsplit, const int2* __restrict__ pairs,
                                    int Khat, double* __restrict__ W) {
  const int p = blockIdx.y;
  const int I = pairs[p].x, J = pairs[p].y;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 128 * 128; e += gridDim.x * blockDim.x) {
    const int m = e >> 7, n = e & 127;
    const int i = 128 * I + m, j = 128 * J + n;
    if (i >= Khat || j >= Khat) continue;
    double s = 0.0, t = 0.0;
    for (int sp = 0; sp < nsplit; ++sp) {
      const float* tile = Wpart + ((int64_t)sp * npairs + p) * 128 * 128;
      s += (double)tile[m * 128 + n];
      if (I == J) t += (double)tile[n * 128 + m];
    }
    if (I == J) {
      W[(int64_t)i * Khat + j] = 0.5 * (s + t);
    } else {
      W[(int64_t)i * Khat + j] = s;
      W[(int64_t)j * Khat + i] = s;
    }
  }
}

size_t tiles_smem_bytes(bool bf) {
  // operands: 2 stages x 2 boxes x (3 BF16 tiles of 8 KB | 2 TF32 tiles of 16 KB)
  return 1024 + (size_t)4 * (bf ? 3 * kOpBytes / 2 : 2 * kOpBytes) + (size_t)kTileRaw * 2 * kBoxBytes +
         (size_t)8 * (kTileRaw + 4) + 16;
}

size_t smem_bytes(int Khat) {
  return 1024 + (size_t)4 * kOpBytes + (size_t)kRaw * kBatch * Khat * 4 + (size_t)8 * (kRaw + 4) + 16;
}

}  // namespace

bool tk_gram_tc_supported(int Khat) {
  return Khat >= 8 && Khat <= 128 && Khat % 4 == 0 && smem_bytes(Khat) <= 225 * 1024;
}

bool tk_gram_tiles_supported(int Khat) { return Khat >= 8 && Khat <= TK_MAXKHAT && Khat % 4 == 0; }

int tk_gram_tiles_pairs(int Khat) {
  const int nt = (int)tk_ceil_div(Khat, 128);
  return nt * (nt + 1) / 2;
}

int tk_gram_tiles_splits(const tucker_ctx* c, int Khat, int R) {
  const int np = tk_gram_tiles_pairs(Khat);
  const int by_sms = std::max(1, c->sm_count / np);
  return std::max(1, std::min(by_sms, (int)tk_ceil_div(R, 4 * kBatch)));
}

namespace {
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    TK_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !p) tk_throw(TUCKER_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    fn = (EncodeTiledFn)p;
  }
  return fn;
}
}  // namespace

// W (FP64) = Z^T Z for Khat > 128 by 128 x 128 blocks; Wpart holds
// tk_gram_tiles_splits x tk_gram_tiles_pairs tiles of 128 x 128 floats, pairs
// the (I, J) block list (device, filled here once).
void tk_gram_tiles(tucker_ctx* c, const float* Z, int R, int Khat, float* Wpart, int2* pairs, double* W, bool bf16,
                   cudaStream_t s) {
  const int nt = (int)tk_ceil_div(Khat, 128);
  const int np = tk_gram_tiles_pairs(Khat);
  std::vector<int2> hp;
  for (int i = 0; i < nt; ++i)
    for (int j = i; j < nt; ++j) hp.push_back(make_int2(i, j));
  TK_CUDA(cudaMemcpyAsync(pairs, hp.data(), hp.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
  const int nsplit = tk_gram_tiles_splits(c, Khat, R);
  CUtensorMap tm;
  const cuuint64_t dims[2] = {(cuuint64_t)Khat, (cuuint64_t)std::max(R, 1)};
  const cuuint64_t strides[1] = {(cuuint64_t)Khat * 4};
  const cuuint32_t box[2] = {128, (cuuint32_t)kBatch};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult cr = encode_fn()(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)Z, dims, strides, box, estr,
                                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) tk_throw(TUCKER_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)cr) + ")");
  GramTileArgs a{};
  a.R = R;
  a.Khat = Khat;
  a.npairs = np;
  a.rows_per_split = (int)(tk_ceil_div(tk_ceil_div(R, nsplit), kBatch) * kBatch);
  a.pairs = pairs;
  a.Wpart = Wpart;
  a.err = c->err;
  a.cap = c->wait_cap;
  static bool attr = false;
  if (!attr) {
    TK_CUDA(cudaFuncSetAttribute(k_gram_tiles<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tiles_smem_bytes(false)));
    TK_CUDA(cudaFuncSetAttribute(k_gram_tiles<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tiles_smem_bytes(true)));
    attr = true;
  }
  if (bf16) k_gram_tiles<true><<<nsplit * np, kThreads, tiles_smem_bytes(true), s>>>(tm, a);
  else k_gram_tiles<false><<<nsplit * np, kThreads, tiles_smem_bytes(false), s>>>(tm, a);
  TK_CUDA(cudaGetLastError());
  dim3 g2(16, np);
  k_gram_tiles_reduce<<<g2, 256, 0, s>>>(Wpart, np, nsplit, pairs, Khat, W);
  TK_CUDA(cudaGetLastError());
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
