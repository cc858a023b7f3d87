// Gram matrix W = Z^T Z of the compact penultimate matrix on the 5th-generation
// tensor cores (tcgen05, kind::tf32) -- the FP32 context's first factor-update
// step.  Z is R x Khat (row-major FP32, Khat <= 128, Khat % 4 == 0).
//
// One persistent CTA per SM takes a contiguous range of rows.  Per batch of 32
// rows:
//   * the raw rows (one contiguous span) arrive in shared memory through a
//     4-deep cp.async pipeline;
//   * 256 threads transpose them into the K-major, 128-byte-swizzled operand
//     layout (M = Z's column index padded to 128, K = the batch's 32 rows),
//     splitting each value into hi = TF32(z) (mantissa truncated) and
//     lo = z - hi (exact in FP32);
//   * one thread issues 4 K-steps x 3 MMAs, D += hi hi^T + hi lo^T + lo hi^T,
//     into a 128 x 128 FP32 accumulator in tensor memory, and commits them to
//     the stage's mbarrier (which also frees the operand stage for reuse).
// Every 8 batches (256 rows) the accumulator is read back (tcgen05.ld) and
// added with Kahan compensation into per-CTA sums in shared memory, so each
// FP32 sum inside the tensor core covers at most 256 rows.  The CTA finally
// writes its partial W; partials are reduced in FP64 in a fixed order.
// Every mbarrier wait is bounded; a timeout sets TK_DEV_ERR_TIMEOUT and the
// kernel releases its tensor memory and returns.
#include <algorithm>

#include "tk_common.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kBatch = 32;        // rows of Z per MMA batch (one 128-byte swizzle atom of K)
constexpr int kDrainEvery = 8;    // batches per TMEM drain
constexpr int kRaw = 4;           // raw-row pipeline depth
constexpr int kOpBytes = 128 * kBatch * 4;  // one 128 x 32 FP32 operand tile (16 KB)
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

// kind::tf32 instruction descriptor: D FP32, A and B TF32 K-major, M = 128, N = 128
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc));
}

__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity) {
  uint32_t done = 0;
  const long long t0 = clock64();
  while (!done) {
    asm volatile(
        "{\n .reg .pred P1;\n mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n selp.b32 %0, 1, 0, P1;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (!done && clock64() - t0 > kWaitCycles) return false;
  }
  return true;
}

__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(sdst)), "l"(gsrc) : "memory");
}

struct GramTcArgs {
  const float* Z;
  int R, Khat;
  int rows_per_cta;
  float* Wpart;  // gridDim.x x 128 x 128
  int* err;
};

__global__ void __launch_bounds__(kThreads, 1) k_gram_tc(const GramTcArgs a) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* sm = smraw + ((1024 - (smem_u32(smraw) & 1023)) & 1023);
  const int Khat = a.Khat;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // layout: operands [2 stages][hi, lo] | raw [kRaw][kBatch][Khat] | acc, cmp [Khat][Khat+1] | barriers
  unsigned char* ops = sm;
  float* raw = (float*)(sm + 4 * kOpBytes);
  const int rawStage = kBatch * Khat;  // floats
  float* acc = raw + kRaw * rawStage;
  const int ldA = Khat + 1;
  float* cmp = acc + Khat * ldA;
  uint64_t* mbar = (uint64_t*)(((uintptr_t)(cmp + Khat * ldA) + 15) & ~(uintptr_t)15);
  uint32_t* tslot = (uint32_t*)(mbar + 2);
  __shared__ int s_fail;

  const int64_t r0 = (int64_t)blockIdx.x * a.rows_per_cta;
  const int64_t r1 = min((int64_t)a.R, r0 + a.rows_per_cta);
  const int nrows = (int)max((int64_t)0, r1 - r0);
  const int nb = (nrows + kBatch - 1) / kBatch;

  for (int i = tid; i < Khat * ldA; i += kThreads) {
    acc[i] = 0.f;
    cmp[i] = 0.f;
  }
  // zero the operand tiles once: padding columns (m >= Khat) stay zero
  for (int i = tid; i < 4 * kOpBytes / 16; i += kThreads) reinterpret_cast<float4*>(ops)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (tid == 0) {
    s_fail = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[0])), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[1])), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)), "r"(128));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;

  auto issue_raw = [&](int b) {
    if (b < nb) {
      const int rows = min(kBatch, nrows - b * kBatch);
      const float* src = a.Z + (r0 + (int64_t)b * kBatch) * Khat;
      float* dst = raw + (b % kRaw) * rawStage;
      const int n16 = rows * Khat / 4;
      for (int q = tid; q < n16; q += kThreads) cp_async16(dst + 4 * q, src + 4 * q);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  for (int b = 0; b < kRaw - 1; ++b) issue_raw(b);

  bool ok = true;
  for (int b = 0; b < nb && ok; ++b) {
    issue_raw(b + kRaw - 1);
    asm volatile("cp.async.wait_group %0;\n" ::"n"(kRaw - 1) : "memory");
    __syncthreads();
    const int st = b & 1;
    if (b >= 2 && !mbar_wait(smem_u32(&mbar[st]), ((b - 2) >> 1) & 1)) ok = false;
    if (!ok) {
      atomicOr(&s_fail, 1);
    } else {
      // transpose + split: thread handles (column m, 4-row chunk c)
      const int rows = min(kBatch, nrows - b * kBatch);
      const float* rw = raw + (b % kRaw) * rawStage;
      unsigned char* hi = ops + st * 2 * kOpBytes;
      unsigned char* lo = hi + kOpBytes;
      for (int pidx = tid; pidx < Khat * (kBatch / 4); pidx += kThreads) {
        const int m = pidx % Khat, cch = pidx / Khat;
        float h4[4], l4[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int r = 4 * cch + q;
          const float z = r < rows ? rw[r * Khat + m] : 0.f;
          const float h = __uint_as_float(__float_as_uint(z) & 0xFFFFE000u);
          h4[q] = h;
          l4[q] = z - h;
        }
        const uint32_t off = sw128_off(m, 4 * cch);
        *reinterpret_cast<float4*>(hi + off) = make_float4(h4[0], h4[1], h4[2], h4[3]);
        *reinterpret_cast<float4*>(lo + off) = make_float4(l4[0], l4[1], l4[2], l4[3]);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (s_fail) {
      ok = false;
      break;
    }
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint64_t dh = sdesc_sw128(smem_u32(ops + st * 2 * kOpBytes));
      const uint64_t dl = sdesc_sw128(smem_u32(ops + st * 2 * kOpBytes + kOpBytes));
      const bool first = (b % kDrainEvery) == 0;
#pragma unroll
      for (int s = 0; s < kBatch / 8; ++s) {
        const uint64_t k = (uint64_t)(2 * s);  // +32 bytes per K-step of 8
        mma_tf32(tmem, dh + k, dh + k, (first && s == 0) ? 0u : 1u);
        mma_tf32(tmem, dh + k, dl + k, 1u);
        mma_tf32(tmem, dl + k, dh + k, 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(&mbar[st])));
    }
    if ((b % kDrainEvery) == kDrainEvery - 1 || b == nb - 1) {
      if (!mbar_wait(smem_u32(&mbar[st]), (b >> 1) & 1)) atomicOr(&s_fail, 1);
      asm volatile("tcgen05.fence::after_thread_sync;");
      __syncthreads();
      if (!s_fail) {
        // warp w reads TMEM lanes 32*(w%4).. and columns 64*(w/4)..; lane = row of D
        const int row = 32 * (warp & 3) + lane;
        const int c0 = 64 * (warp >> 2);
#pragma unroll
        for (int cc = 0; cc < 64; cc += 16) {
          uint32_t v[16];
          const uint32_t taddr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(c0 + cc);
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
              "[%16];"
              : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                "=r"(v[15])
              : "r"(taddr));
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          if (row < Khat) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int col = c0 + cc + j;
              if (col < Khat) {
                float* sp = acc + row * ldA + col;
                float* cp = cmp + row * ldA + col;
                const float y = __uint_as_float(v[j]) - *cp;
                const float t = *sp + y;
                *cp = (t - *sp) - y;
                *sp = t;
              }
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();
      if (s_fail) {
        ok = false;
        break;
      }
    }
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
  if (!ok || s_fail) {
    if (tid == 0) atomicOr(a.err, TK_DEV_ERR_TIMEOUT);
  }
  float* out = a.Wpart + (int64_t)blockIdx.x * 128 * 128;
  for (int i = tid; i < 128 * 128; i += kThreads) {
    const int r = i >> 7, cc = i & 127;
    out[i] = (r < Khat && cc < Khat) ? acc[r * ldA + cc] : 0.f;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128));
}

size_t smem_bytes(int Khat) {
  return 1024 + (size_t)4 * kOpBytes + (size_t)kRaw * kBatch * Khat * 4 + (size_t)2 * Khat * (Khat + 1) * 4 + 64;
}

}  // namespace

bool tk_gram_tc_supported(int Khat) {
  return Khat >= 8 && Khat <= 128 && Khat % 4 == 0 && smem_bytes(Khat) <= 225 * 1024;
}

// Writes gridDim partials of W (128 x 128 FP32 tiles) into Wpart; returns the number of partials.
int tk_gram_tc(tucker_ctx* c, const float* Z, int R, int Khat, float* Wpart, size_t Wpart_elems, cudaStream_t s) {
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
  const size_t shm = smem_bytes(Khat);
  static bool attr = false;
  if (!attr) {
    TK_CUDA(cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 225 * 1024));
    attr = true;
  }
  k_gram_tc<<<nblk, kThreads, shm, s>>>(a);
  TK_CUDA(cudaGetLastError());
  return nblk;
}
