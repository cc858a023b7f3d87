// TTM-chain of a 4-mode FP32 tensor with a large Khat on the 5th-generation
// tensor cores (Section 3, eq. (1); Appendix A; tcgen05 kind::tf32).
//
// With a < b < c the remaining modes of mode n, the row of slice l of the
// unfolding, read as a (K_a K_b) x K_c matrix (column i + K_a j + K_a K_b k is
// entry (i + K_a j, k): the first remaining mode fastest), is
//     Z[l] = sum_{e in slice l} x_e y_e^T,
//     x_e = val_e F_a[l_a(e)] (x) F_b[l_b(e)]   (M = K_a K_b <= 128 entries),
//     y_e = F_c[l_c(e)]                          (N = K_c <= 48, padded to 16),
// a product A B^T whose contraction runs over the slice's elements.  Each
// block of 8 elements is one MMA step (M = 128, N = 16..48, K = 8).  In FP32
// accuracy: x = xh + xl and y = yh + yl with xh, yh the TF32-truncated values
// and xl, yl the exact FP32 rests, and Z[l] += xh yh^T + xh yl^T + xl yh^T
// (xl yl^T is below FP32 resolution).  The yh and yl tiles lie one after the
// other in shared memory, so the first two terms are one MMA of twice the
// width, xh [yh | yl]^T, into an accumulator of 2N columns, and xl yh^T adds
// into its first N columns: two MMAs per block, whose issue cost does not
// grow with N.
//
// Layout: a second copy of the mode's elements, made at init from the Lite
// copy: every bin's elements contiguous, every segment of a bin (a whole
// slice, or the piece of a split slice) padded with zero-valued elements to a
// multiple of 8, so that each block belongs to one segment.  Per block: the
// destination of its segment (compact row, or the split piece's partial slot
// bin * 2 + head) and three flags: an accumulator starts at the block, one
// ends there, the segment ends there.  An accumulator covers at most 32
// blocks (256 elements): the tensor core's FP32 accumulation truncates, so a
// long segment is summed as pieces, added in round-to-nearest FP32 in a
// per-thread running sum (shared memory) in order, the row stored once.
//
// One CTA takes a contiguous range of bins (balanced by blocks) and streams
// it in chunks of 32 elements (4 blocks) through a ring of shared-memory
// stages, with three roles:
//   * warps 4-7 load: per chunk, warp 4 the values and F_a rows (as val F_a,
//     transposed), warp 5 the F_b rows, warp 6 the F_c rows as the TF32
//     hi / lo B operands (K-major, 128-byte swizzle), warp 7 the block table;
//     the loads of a group of chunks are all in flight before any is stored;
//   * warps 0-3 (thread t = tensor-memory lane t = row t of A) form the
//     chunk's A operand x_e[t] for its 32 elements, split it, store hi and lo
//     into tensor memory (tcgen05.st; two buffers) and hand the buffer over;
//     one chunk later they read each finished accumulator back (tcgen05.ld),
//     add it to the segment's running sum, and at the segment's end store its
//     row of Z (or the split piece's partial, added by the fix-up in bin
//     order, as for the CUDA-core kernel), then release the slot;
//   * warp 8 issues the MMAs: per block, the accumulator slot of its piece (up
//     to 8 slots of 2N columns, round robin, a slot reused only once it has
//     been read back) and two MMAs; where a piece ends, a commit to the slot's
//     mbarrier.  The drain adds the slot's two halves.
// A tcgen05.mma of this shape (M = 128, N = 16..96, K = 8) occupies its
// issuing thread for far longer than the tensor core computes it (about 50-70
// cycles, whatever N): two CTAs share an SM (256 tensor-memory columns each)
// to run two issuers side by side.
// Every mbarrier wait is bounded (clock and the context's poll cap); a
// timeout sets TK_DEV_ERR_TIMEOUT, every role leaves its loop, the CTA waits
// (bounded) for its MMAs in flight and releases its tensor memory.
#include <algorithm>

#include "tk_common.cuh"
#include "tk_tc.cuh"

namespace {

using namespace tk_tc;

constexpr int kTcThreads = 288;  // warps 0-3 build and drain, 4-7 load, 8 issues the MMAs
constexpr int kChunk = 32;       // elements per stage: 4 blocks of 8
constexpr int kStages = 8;
constexpr int kNacc = 8;         // accumulator slots at most
constexpr int kRowStride = 36;   // floats per staged F_a / F_b row (144 B: rows on different banks)
constexpr uint32_t kCodeSplit = 0x80000000u;
constexpr uint8_t kStart = 1, kEnd = 2, kFinal = 4;
constexpr int kPiece = 32;       // blocks per tensor-memory accumulation at most
constexpr uint32_t kTf32Mask = 0xFFFFE000u;

struct TcArgs {
  const uint32_t* code;    // nblk
  const uint8_t* flag;     // nblk
  const int64_t* blk_ptr;  // Pa + 1
  const int32_t* oidx[3];  // 8 nblk each
  const float* val;
  const int32_t* perm;
  const float* vals_override;
  const float* F[3];
  int ld[3];
  int K[3];
  int nv[3];  // float4 vectors per row
  int Pa;
  int64_t nblk;
  int Mu, Nu, NP;
  int Khat;
  int stage_bytes;   // multiple of 1024
  int off_va, off_bb, off_info;
  int tmem_cols;
  int nacc;  // accumulator slots of 2 NP columns after the 128 columns of A
  float* Z;
  float* Zpart;
  int* err;
  int cap;
};

// stream loads: read once, not kept in L1, first out of L2
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ int32_t ld_stream_i32(const int32_t* p, uint64_t pol) {
  int32_t v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ float ld_stream_f32(const float* p, uint64_t pol) {
  float v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
  return v;
}

// Whole-warp bounded wait that also gives up once another role has failed.
__device__ __forceinline__ bool wait_warp(const uint64_t* bar, uint32_t parity, int cap, const volatile int* fail) {
  if (cap < 0) return false;
  const uint32_t addr = smem_u32(bar);
  const long long t0 = clock64();
  for (int polls = 1;; ++polls) {
    const uint32_t done = mbar_try(addr, parity);
    if (__all_sync(0xffffffffu, done)) return true;
    const bool out = *fail != 0 || clock64() - t0 > kWaitCycles || (cap > 0 && polls >= cap);
    if (__any_sync(0xffffffffu, out)) return false;
  }
}

// One thread's bounded wait (the MMA issuer works alone), with the same limits.
__device__ __forceinline__ bool wait_one(const uint64_t* bar, uint32_t parity, int cap, const volatile int* fail) {
  if (cap < 0) return false;
  const uint32_t addr = smem_u32(bar);
  const long long t0 = clock64();
  for (int polls = 1;; ++polls) {
    if (mbar_try(addr, parity)) return true;
    if (*fail != 0 || clock64() - t0 > kWaitCycles || (cap > 0 && polls >= cap)) return false;
  }
}

__device__ __forceinline__ void mma_tf32_ts(uint32_t d, uint32_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
      "r"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
      "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]),
      "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]),
      "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & kTf32Mask); }

// first index p in [0, n] with a[p] >= x (a non-decreasing, a[n] is the total)
__device__ __forceinline__ int lower_bound_i64(const int64_t* a, int n, int64_t x) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// NVR: float4 vectors per factor row at most; kU: chunks per producer load group
template <int kNVR, int kU>
__global__ void __launch_bounds__(kTcThreads, 2) k_ttmc_tc(const TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* sm = smraw + ((1024 - (smem_u32(smraw) & 1023)) & 1023);
  uint64_t* full = (uint64_t*)(sm + kStages * a.stage_bytes);
  uint64_t* empty = full + kStages;
  // empty[s] also frees the A buffer of the stage's chunk: its MMAs are done
  uint64_t* afull = empty + kStages;  // 2: A buffer written (4 builder warps)
  uint64_t* accf = afull + 2;        // kNacc: accumulator of the slot complete
  uint64_t* acce = accf + kNacc;     // kNacc: slot read back (4 builder warps)
  uint64_t* fin = acce + kNacc;
  uint32_t* tslot = (uint32_t*)(fin + 1);
  float* run = (float*)(fin + 2);    // NP x 128: running sums of the open segment, [n][lane]
  __shared__ int s_fail;
  __shared__ int64_t s_range[2];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int NP = a.NP;

  // zero the B operand tiles of every stage once: rows n >= K_c stay zero
  for (int s = 0; s < kStages; ++s) {
    float4* b = reinterpret_cast<float4*>(sm + s * a.stage_bytes);
    for (int i = tid; i < 2 * NP * 128 / 16; i += kTcThreads) b[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  if (tid == 0) {
    s_fail = 0;
    for (int i = 0; i < kStages; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[i])), "r"(128));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&empty[i])), "r"(1));
    }
    for (int i = 0; i < 2; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&afull[i])), "r"(4));
    for (int i = 0; i < kNacc; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&accf[i])), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&acce[i])), "r"(4));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(fin)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
    const int64_t t0 = a.nblk * blockIdx.x / gridDim.x, t1 = a.nblk * (blockIdx.x + 1) / gridDim.x;
    s_range[0] = a.blk_ptr[lower_bound_i64(a.blk_ptr, a.Pa, t0)];
    s_range[1] = a.blk_ptr[lower_bound_i64(a.blk_ptr, a.Pa, t1)];
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(a.tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;
  const int64_t B0 = s_range[0], B1 = s_range[1];
  const int nchunks = (int)((B1 - B0 + 3) / 4);
  const int64_t e0 = 8 * B0, e1 = 8 * B1;
  volatile int* fail = &s_fail;

  if (warp >= 4 && warp < 8) {
    // ------------------------------------------------------------ loaders
    const int q = warp - 4;
    const uint64_t pol = policy_evict_first();
    int id_c[kU], id_n[kU];
    float v_c[kU], v_n[kU];
    uint32_t code_c = 0, code_n = 0;
    uint32_t flag_c = 0, flag_n = 0;
    auto load_group = [&](int g, int (&id)[kU], float (&v)[kU], uint32_t& cd, uint32_t& fl) {
      if (q < 3) {
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const int64_t slot = e0 + (int64_t)(g * kU + u) * kChunk + lane;
          const bool ok = slot < e1;
          id[u] = ok ? ld_stream_i32(a.oidx[q] + slot, pol) : 0;
          v[u] = 0.f;
          if (q == 0 && ok) {
            if (a.vals_override) {
              const int32_t pe = ld_stream_i32(a.perm + slot, pol);
              v[u] = pe >= 0 ? __ldg(a.vals_override + pe) : 0.f;
            } else {
              v[u] = ld_stream_f32(a.val + slot, pol);
            }
          }
        }
      } else {
        // lane l: block l of the group (4 chunks x 4 blocks)
        const int64_t blk = B0 + (int64_t)g * kU * 4 + (lane & 15);
        const bool ok = lane < 16 && blk < B1;
        cd = ok ? __ldg(a.code + blk) : 0u;
        fl = ok ? (uint32_t)__ldg(a.flag + blk) : 0u;
      }
    };
    const int ngroups = (nchunks + kU - 1) / kU;
    if (ngroups > 0) load_group(0, id_c, v_c, code_c, flag_c);
    for (int g = 0; g < ngroups; ++g) {
      float4 row[kU][kNVR];
      if (q < 3) {
        const float* Fq = a.F[q];
        const int ldq = a.ld[q], nvq = a.nv[q];
#pragma unroll
        for (int u = 0; u < kU; ++u)
#pragma unroll
          for (int v = 0; v < kNVR; ++v)
            row[u][v] = v < nvq ? __ldg(reinterpret_cast<const float4*>(Fq + (int64_t)id_c[u] * ldq) + v)
                                : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      if (g + 1 < ngroups) load_group(g + 1, id_n, v_n, code_n, flag_n);
      bool ok = true;
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int c = g * kU + u;
        if (c >= nchunks) break;
        const int s = c % kStages;
        if (c >= kStages && !wait_warp(&empty[s], (uint32_t)(((c / kStages) - 1) & 1), a.cap, fail)) {
          ok = false;
          break;
        }
        unsigned char* st = sm + s * a.stage_bytes;
        if (q == 0) {
          float* va = (float*)(st + a.off_va);
#pragma unroll
          for (int v = 0; v < kNVR; ++v) {
            const float r4[4] = {row[u][v].x, row[u][v].y, row[u][v].z, row[u][v].w};
#pragma unroll
            for (int t = 0; t < 4; ++t)
              if (4 * v + t < a.K[0]) va[(4 * v + t) * kRowStride + lane] = v_c[u] * r4[t];
          }
        } else if (q == 1) {
          float* bb = (float*)(st + a.off_bb);
#pragma unroll
          for (int v = 0; v < kNVR; ++v) {
            const float r4[4] = {row[u][v].x, row[u][v].y, row[u][v].z, row[u][v].w};
#pragma unroll
            for (int t = 0; t < 4; ++t)
              if (4 * v + t < a.K[1]) bb[(4 * v + t) * kRowStride + lane] = r4[t];
          }
        } else if (q == 2) {
          unsigned char* bh = st;
          unsigned char* bl = st + NP * 128;
#pragma unroll
          for (int v = 0; v < kNVR; ++v) {
            const float r4[4] = {row[u][v].x, row[u][v].y, row[u][v].z, row[u][v].w};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
              const int nn = 4 * v + t;
              if (nn < a.K[2]) {
                const float h = tf32_hi(r4[t]);
                *(float*)(bh + sw128_off(nn, lane)) = h;
                *(float*)(bl + sw128_off(nn, lane)) = r4[t] - h;
              }
            }
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        } else {
          // lanes 4u .. 4u + 3 hold this chunk's blocks
          const uint32_t cd = __shfl_sync(0xffffffffu, code_c, (4 * u + (lane & 3)) & 31);
          const uint32_t fl = __shfl_sync(0xffffffffu, flag_c, (4 * u + (lane & 3)) & 31);
          if (lane < 4) {
            uint32_t* info = (uint32_t*)(st + a.off_info);
            info[lane] = cd;
            info[4 + lane] = fl;
          }
        }
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&full[s])) : "memory");
      }
      if (!ok) {
        atomicOr((int*)&s_fail, 1);
        break;
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        id_c[u] = id_n[u];
        v_c[u] = v_n[u];
      }
      code_c = code_n;
      flag_c = flag_n;
    }
  } else if (warp == 8) {
    // ------------------------------------------------------------ MMA issuer
    // Per chunk, once the builders have written its A: the slot of each
    // block's accumulator (a new one where a piece starts, after the builders
    // have read back its previous piece), two MMAs per block, a commit to
    // the slot's barrier where a piece ends, then one commit releases the
    // stage and the A buffer.
    // Lane 0 alone: MMAs and commits are issued by one thread.
    if (lane == 0) {
      const uint32_t idesc = idesc_tf32(NP), idesc2 = idesc_tf32(2 * NP);
      const uint32_t dcol0 = 128;
      int segc = 0, cur_slot = 0;
      uint32_t used = 0, epar = 0;
      for (int c = 0; c < nchunks; ++c) {
        const int s = c % kStages;
        unsigned char* st = sm + s * a.stage_bytes;
        bool ok = wait_one(&afull[c & 1], (uint32_t)((c >> 1) & 1), a.cap, fail);
        if (ok) {
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t* info = (const uint32_t*)(st + a.off_info);
          const int nvb = (int)min((int64_t)4, B1 - B0 - 4 * (int64_t)c);
          const uint32_t acol = (uint32_t)((c & 1) * 64);
          const uint64_t dh = sdesc_sw128(smem_u32(st));  // yh rows, then yl rows
          for (int kb = 0; kb < nvb; ++kb) {
            const uint32_t fl = info[4 + kb];
            if (fl & kStart) {
              cur_slot = segc % a.nacc;
              ++segc;
              if (used & (1u << cur_slot)) {
                if (!wait_one(&acce[cur_slot], (epar >> cur_slot) & 1u, a.cap, fail)) {
                  ok = false;
                  break;
                }
                epar ^= 1u << cur_slot;
                asm volatile("tcgen05.fence::after_thread_sync;");
              }
              used |= 1u << cur_slot;
            }
            const uint32_t d = tmem + dcol0 + (uint32_t)(cur_slot * 2 * NP);
            const uint32_t ah = tmem + acol + 8 * kb, al = ah + 32;
            const uint64_t k = (uint64_t)(2 * kb);  // +32 bytes per K-step of 8
            const uint32_t en = (fl & kStart) ? 0u : 1u;
            mma_tf32_ts(d, ah, dh + k, idesc2, en);  // [xh yh | xh yl]
            mma_tf32_ts(d, al, dh + k, idesc, 1u);   // + xl yh in the first half
            if (fl & kEnd) mma_commit(&accf[cur_slot]);
          }
          if (ok) mma_commit(&empty[s]);
        }
        if (!ok) {
          atomicOr((int*)&s_fail, 1);
          break;
        }
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------- A operand, drain
    const int m = tid;  // tensor-memory lane = row of A
    const bool act = m < a.Mu;
    const int ii = act ? m % a.K[0] : 0, jj = act ? m / a.K[0] : 0;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * warp) << 16);
    const uint32_t dcol0 = 128;
    uint32_t accpar = 0;
    int segc = 0, cur_slot = 0;
    int npend = 0;
    bool has_run = false;
    uint32_t pend_code[4];
    int pend_slot[4];
    bool pend_final[4];
    // reads back the pieces that ended in the previous chunk (in order), adds
    // each to the segment's running sum, stores the row at the segment's end,
    // and releases the slot to the issuer
    auto drain = [&]() -> bool {
      for (int p = 0; p < npend; ++p) {
        const int sl = pend_slot[p];
        if (!wait_warp(&accf[sl], (accpar >> sl) & 1u, a.cap, fail)) return false;
        accpar ^= 1u << sl;
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t cd = pend_code[p];
        const bool fin_p = pend_final[p];
        float* dst = (cd & kCodeSplit) ? a.Zpart + (int64_t)(cd & ~kCodeSplit) * a.Khat : a.Z + (int64_t)cd * a.Khat;
        for (int n0 = 0; n0 < NP; n0 += 8) {
          uint32_t r[8], r2[8];
          tmem_ld8(lane_base + dcol0 + (uint32_t)(sl * 2 * NP + n0), r);
          tmem_ld8(lane_base + dcol0 + (uint32_t)(sl * 2 * NP + NP + n0), r2);
          if (act) {
#pragma unroll
            for (int t = 0; t < 8; ++t) {
              const int nn = n0 + t;
              if (nn < a.Nu) {
                float x = __uint_as_float(r[t]) + __uint_as_float(r2[t]);
                if (has_run) x += run[nn * 128 + m];
                if (fin_p) dst[m + (int64_t)a.Mu * nn] = x;
                else run[nn * 128 + m] = x;
              }
            }
          }
        }
        has_run = !fin_p;
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acce[sl])) : "memory");
      }
      npend = 0;
      return true;
    };
    for (int c = 0; c < nchunks; ++c) {
      const int s = c % kStages;
      unsigned char* st = sm + s * a.stage_bytes;
      bool ok = wait_warp(&full[s], (uint32_t)((c / kStages) & 1), a.cap, fail);
      // A buffer c & 1 is free once the MMAs of chunk c - 2 are done
      if (ok && c >= 2) ok = wait_warp(&empty[(c - 2) % kStages], (uint32_t)(((c - 2) / kStages) & 1), a.cap, fail);
      if (!ok) {
        atomicOr((int*)&s_fail, 1);
        break;
      }
      uint32_t cds[4], fls[4];
      const int nvb = (int)min((int64_t)4, B1 - B0 - 4 * (int64_t)c);
      {
        const uint32_t* info = (const uint32_t*)(st + a.off_info);
#pragma unroll
        for (int kb = 0; kb < 4; ++kb) {
          cds[kb] = info[kb];
          fls[kb] = kb < nvb ? info[4 + kb] : 0u;
        }
        const float4* va = reinterpret_cast<const float4*>((const float*)(st + a.off_va) + ii * kRowStride);
        const float4* bb = reinterpret_cast<const float4*>((const float*)(st + a.off_bb) + jj * kRowStride);
        uint32_t h[32], l[32];
#pragma unroll
        for (int e4 = 0; e4 < 8; ++e4) {
          const float4 x4 = va[e4], y4 = bb[e4];
          const float xs[4] = {x4.x * y4.x, x4.y * y4.y, x4.z * y4.z, x4.w * y4.w};
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const float x = act ? xs[t] : 0.f;
            const float hx = tf32_hi(x);
            h[4 * e4 + t] = __float_as_uint(hx);
            l[4 * e4 + t] = __float_as_uint(x - hx);
          }
        }
        const uint32_t acol = (uint32_t)((c & 1) * 64);
        tmem_st32(lane_base + acol, h);
        tmem_st32(lane_base + acol + 32, l);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&afull[c & 1])) : "memory");
      }
      // the pieces that ended in the previous chunk, while the issuer works on this one
      if (!drain()) {
        atomicOr((int*)&s_fail, 1);
        break;
      }
      // this chunk's pieces: slot per block, and the ones ending here
#pragma unroll
      for (int kb = 0; kb < 4; ++kb) {
        if (fls[kb] & kStart) {
          cur_slot = segc % a.nacc;
          ++segc;
        }
        if (fls[kb] & kEnd) {
          pend_code[npend] = cds[kb];
          pend_slot[npend] = cur_slot;
          pend_final[npend] = (fls[kb] & kFinal) != 0;
          ++npend;
        }
      }
    }
    if (!*fail)
      if (!drain()) atomicOr((int*)&s_fail, 1);
  }

  // no MMA may be in flight when the tensor memory is released
  if (tid == 8 * 32) {
    mma_commit(fin);
    if (!mbar_wait(fin, 0)) atomicOr((int*)&s_fail, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (tid == 0 && s_fail) atomicOr(a.err, TK_DEV_ERR_TIMEOUT);
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols));
  }
}

// ---------------------------------------------------------------- the copy

// blocks of bin p: its segments (maximal runs of one row code) padded to 8
__global__ void k_tc_count(const uint32_t* __restrict__ rowcode, const int32_t* __restrict__ bin_len, int Pa,
                           int limit, int64_t* __restrict__ nblk) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= Pa) return;
  const int len = bin_len[p];
  const int64_t base = (int64_t)(p >> 5) * limit * 32 + (p & 31);
  int64_t cnt = 0;
  int run = 0;
  uint32_t prev = 0;
  for (int k = 0; k < len; ++k) {
    const uint32_t cd = rowcode[base + 32 * (int64_t)k];
    if (k == 0 || cd != prev) {
      cnt += (run + 7) / 8;
      run = 0;
      prev = cd;
    }
    ++run;
  }
  nblk[p] = cnt + (run + 7) / 8;
}

struct TcFillArgs {
  const uint32_t* rowcode;
  const int32_t* oidx[3];
  const float* val;
  const int32_t* perm;
  const int32_t* bin_len;
  const int64_t* blk_ptr;
  int Pa, limit;
  uint32_t* code;
  uint8_t* flag;
  int32_t* t_oidx[3];
  float* t_val;
  int32_t* t_perm;
};

__device__ __forceinline__ void tc_pad(const TcFillArgs& a, int64_t b, int from) {
  for (int j = from; j < 8; ++j) {
    const int64_t d = 8 * b + j;
    for (int q = 0; q < 3; ++q) a.t_oidx[q][d] = 0;
    a.t_val[d] = 0.f;
    a.t_perm[d] = -1;
  }
}

__global__ void k_tc_fill(const TcFillArgs a) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.Pa) return;
  const int len = a.bin_len[p];
  if (len == 0) return;
  const int64_t base = (int64_t)(p >> 5) * a.limit * 32 + (p & 31);
  int64_t b = a.blk_ptr[p] - 1;
  int pos = 8;  // element position inside block b
  int j = 0;    // index of block b inside its segment
  uint32_t prev = 0, dest = 0;
  for (int k = 0; k < len; ++k) {
    const int64_t sl = base + 32 * (int64_t)k;
    const uint32_t cd = a.rowcode[sl];
    const bool seg_start = k == 0 || cd != prev;
    if (seg_start || pos == 8) {
      if (seg_start && k > 0) {
        tc_pad(a, b, pos);
        a.flag[b] |= kEnd | kFinal;
      }
      if (seg_start) {
        prev = cd;
        dest = (cd & TK_SPLIT_BIT) ? (kCodeSplit | (uint32_t)(2 * p + ((cd & TK_HEAD_BIT) ? 1 : 0)))
                                   : (cd & TK_ROW_MASK);
        j = 0;
      } else {
        ++j;
      }
      ++b;
      pos = 0;
      a.code[b] = dest;
      a.flag[b] = (uint8_t)(((j % kPiece) == 0 ? kStart : 0) | ((j % kPiece) == kPiece - 1 ? kEnd : 0));
    }
    const int64_t d = 8 * b + pos;
    for (int q = 0; q < 3; ++q) a.t_oidx[q][d] = a.oidx[q][sl];
    a.t_val[d] = a.val[sl];
    a.t_perm[d] = a.perm[sl];
    ++pos;
  }
  tc_pad(a, b, pos);
  a.flag[b] |= kEnd | kFinal;
}

constexpr int kTcStageAlign = 1024;

int stage_bytes_for(int K0, int K1, int NP, int* off_va, int* off_bb, int* off_info) {
  int off = 2 * NP * 128;
  *off_va = off;
  off += K0 * kRowStride * 4;
  *off_bb = off;
  off += K1 * kRowStride * 4;
  *off_info = off;
  off += 32;
  return (off + kTcStageAlign - 1) / kTcStageAlign * kTcStageAlign;
}

// A buffers in columns [0, 128), then at least four accumulator slots of
// 2 NP columns (NP = 16: 256 columns, two CTAs per SM)
int tmem_cols_for(int NP) {
  const int need = 128 + 4 * 2 * NP;
  int c = 32;
  while (c < need) c *= 2;
  return c;
}
int nacc_for(int NP, int cols) { return std::min(kNacc, (cols - 128) / (2 * NP)); }

void others_of(const tucker_ctx* c, int n, int* o) {
  int k = 0;
  for (int m = 0; m < c->N; ++m)
    if (m != n) o[k++] = m;
}

}  // namespace

bool tk_ttmc_tc_eligible(const tucker_ctx* c, int n) {
  if (c->prec != TUCKER_FP32 || c->N != 4) return false;
  int o[3];
  others_of(c, n, o);
  const int Mu = c->K[o[0]] * c->K[o[1]], Nu = c->K[o[2]];
  return Mu >= 32 && Mu <= 128 && Nu <= 48 && Mu * Nu >= 256;
}

void tk_ttmc_tc_build(tucker_ctx* c, int n, cudaStream_t s) {
  tk_mode& md = c->mode[n];
  int o[3];
  others_of(c, n, o);
  int64_t* cnt = (int64_t*)tk_dev_alloc(c, (size_t)(md.Pa + 1) * 8);
  md.tc_blk_ptr = (int64_t*)tk_alloc(c, (size_t)(md.Pa + 1) * 8);
  k_tc_count<<<(unsigned)tk_ceil_div(md.Pa, 256), 256, 0, s>>>(md.rowcode, md.bin_len, md.Pa, md.limit, cnt);
  TK_CUDA(cudaGetLastError());
  TK_CUDA(cudaMemsetAsync(cnt + md.Pa, 0, 8, s));
  const size_t tb = tk_scan_tmp_bytes(md.Pa + 1, 8);
  void* tmp = tk_dev_alloc(c, std::max<size_t>(tb, 16));
  tk_exclusive_scan_i64(cnt, md.tc_blk_ptr, md.Pa + 1, tmp, s);
  int64_t nblk = 0;
  TK_CUDA(cudaMemcpyAsync(&nblk, md.tc_blk_ptr + md.Pa, 8, cudaMemcpyDeviceToHost, s));
  TK_CUDA(cudaStreamSynchronize(s));
  tk_dev_free(c, tmp, std::max<size_t>(tb, 16));
  tk_dev_free(c, cnt, (size_t)(md.Pa + 1) * 8);
  md.tc_nblk = nblk;
  const size_t ne = (size_t)std::max<int64_t>(nblk, 1) * 8;
  md.tc_code = (uint32_t*)tk_alloc(c, ne / 8 * 4);
  md.tc_flag = (uint8_t*)tk_alloc(c, ne / 8);
  for (int q = 0; q < 3; ++q) md.tc_oidx[q] = (int32_t*)tk_alloc(c, ne * 4);
  md.tc_val = (float*)tk_alloc(c, ne * 4);
  md.tc_perm = (int32_t*)tk_alloc(c, ne * 4);
  TcFillArgs f{};
  f.rowcode = md.rowcode;
  for (int q = 0; q < 3; ++q) {
    f.oidx[q] = md.oidx[q];
    f.t_oidx[q] = md.tc_oidx[q];
  }
  f.val = (const float*)md.val;
  f.perm = md.perm;
  f.bin_len = md.bin_len;
  f.blk_ptr = md.tc_blk_ptr;
  f.Pa = md.Pa;
  f.limit = md.limit;
  f.code = md.tc_code;
  f.flag = md.tc_flag;
  f.t_val = md.tc_val;
  f.t_perm = md.tc_perm;
  k_tc_fill<<<(unsigned)tk_ceil_div(md.Pa, 128), 128, 0, s>>>(f);
  TK_CUDA(cudaGetLastError());
  md.tc_Mu = c->K[o[0]] * c->K[o[1]];
  md.tc_Nu = c->K[o[2]];
  md.tc = true;
}

void tk_ttmc_tc_launch(tucker_ctx* c, int n, void* const* F, const int* ldF, const void* vals_override, void* Z,
                       cudaStream_t s) {
  const tk_mode& md = c->mode[n];
  int o[3];
  others_of(c, n, o);
  TcArgs a{};
  a.code = md.tc_code;
  a.flag = md.tc_flag;
  a.blk_ptr = md.tc_blk_ptr;
  for (int q = 0; q < 3; ++q) {
    a.oidx[q] = md.tc_oidx[q];
    a.F[q] = (const float*)F[o[q]];
    a.ld[q] = ldF[o[q]];
    a.K[q] = c->K[o[q]];
    a.nv[q] = (a.K[q] + 3) / 4;
    if ((uintptr_t)F[o[q]] % 16 != 0 || ldF[o[q]] % 4 != 0)
      tk_throw(TUCKER_ERR_ARG, "tensor-core TTM-chain needs 16-byte aligned factor rows");
  }
  a.val = md.tc_val;
  a.perm = md.tc_perm;
  a.vals_override = (const float*)vals_override;
  a.Pa = md.Pa;
  a.nblk = md.tc_nblk;
  a.Mu = md.tc_Mu;
  a.Nu = md.tc_Nu;
  a.NP = (md.tc_Nu + 15) / 16 * 16;
  a.Khat = md.Khat;
  a.stage_bytes = stage_bytes_for(a.K[0], a.K[1], a.NP, &a.off_va, &a.off_bb, &a.off_info);
  a.tmem_cols = tmem_cols_for(a.NP);
  a.nacc = nacc_for(a.NP, a.tmem_cols);
  a.Z = (float*)Z;
  a.Zpart = (float*)c->Zpart;
  a.err = c->err;
  a.cap = c->wait_cap;
  // stages | barriers (2 kStages + 2 + 2 kNacc + 1) | TMEM slot (8 B) | running sums (NP x 128 floats)
  const size_t smem = 1024 + (size_t)kStages * a.stage_bytes + (2 * kStages + 2 + 2 * kNacc + 2) * 8 +
                      (size_t)a.NP * 128 * 4;
  const int nvr = std::max(a.nv[0], std::max(a.nv[1], a.nv[2]));
  // loader registers: kU chunks' rows of kNVR vectors within the 96 registers of two CTAs per SM
  void (*kern)(const TcArgs) = nvr <= 2 ? k_ttmc_tc<2, 4> : nvr <= 3 ? k_ttmc_tc<3, 4> : nvr <= 4 ? k_ttmc_tc<4, 2>
                                                                                                   : k_ttmc_tc<8, 1>;
  TK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  // two CTAs per SM when their tensor memory fits (N = 16): each CTA has one
  // MMA-issuing thread, and a tcgen05.mma of this size costs its issuer far
  // more cycles than the tensor core needs for it, so issuers run side by side
  const int per_sm = a.tmem_cols <= 256 ? 2 : 1;
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((int64_t)per_sm * c->sm_count, md.tc_nblk));
  kern<<<(unsigned)grid, kTcThreads, smem, s>>>(a);
  TK_CUDA(cudaGetLastError());
}
