// TTM-chain along mode n (Section 3, eq. (1); Appendix A) and its adjoint.
//
// One Lite bin per thread.  A bin's elements are a run of whole slices
// (stage 1) followed by at most one tail and one head piece of split slices
// (stage 2, Theorem 1), stored warp-interleaved so that the 32 bins of a warp
// read each stream array as one 128-byte line per step.  A thread keeps the
// Kronecker accumulator of its current slice in registers:
//     acc[i + MA*j] += val * F_a[l_a][i] * F_b[l_b][j0+j] * prod_outer F_q[l_q][c_q]
// where a and b are the first two remaining modes (a varies fastest, as in
// Appendix A) and the remaining ("outer") modes' columns, together with the
// block j0 of b, are fixed per column group g.  A whole slice is written to its
// compact Z row once; a split piece goes to a per-bin partial slot and the
// fix-up adds the pieces in bin order (deterministic, FP64 sums).
//
// The forward kernel is bound by the two gathered factor rows per element
// (their L1 misses and the latency behind them), so it keeps as many rows in
// flight as the registers allow: the rows of the next D elements are requested
// before the current element is used, and the stream (row code, coordinates,
// value) is read straight from memory 2D elements ahead, not cached in L1 and
// marked evict-first in L2.  The F_a row comes through the LSU path, the F_b
// block through the texture path; factor rows carry an evict-last hint.  The
// coordinates in the copy are popularity labels and each slice lists its
// elements by the label of the fiber-mode coordinate, so all threads sweep the
// hot factor rows together.
//
// Fiber-factored form (an option): when the fiber mode is b, consecutive
// elements of a slice that share F_b's row form a fiber, and
//     sum_fiber val F_a (x) F_b = (sum_fiber val F_a) (x) F_b,
// so each element adds val F_a into a fiber sum (K_a FMAs) and the F_b row is
// gathered, and the sum expanded into the slice tile, once per fiber.  The
// fiber ends differ between the threads of a warp, so the expansion is taken
// by the whole warp almost every step; the form saves gathers, not FMAs.
#include <algorithm>

#include "tk_common.cuh"

#ifndef TK_TTMC_NE
#define TK_TTMC_NE 2  // elements in flight per thread (exact FP32 3-mode tiles)
#endif


namespace {

template <typename T>
struct VecT;
template <>
struct VecT<float> {
  using type = float4;
  static constexpr int W = 4;
};
template <>
struct VecT<double> {
  using type = double2;
  static constexpr int W = 2;
};

template <typename T>
struct TtmcArgs {
  const uint32_t* rowcode;
  const int32_t* oidx[TK_MAXN - 1];
  const T* val;
  const int32_t* perm;
  const int32_t* bin_len;
  const T* vals_override;
  const T* F[TK_MAXN - 1];  // factors of the other modes, increasing mode order
  cudaTextureObject_t texB; // texture over the second remaining factor (0: plain loads)
  int ld[TK_MAXN - 1];      // their (padded) leading dimensions
  int Kf[TK_MAXN - 1];
  int nother;
  int P, limit;
  int G, NB, TB;
  int KA, KB;
  int Khat;
  int store_vec;
  int tile_vec;  // adjoint: the cotangent block rows can be read as 16-byte vectors
  T* Z;
  T* Zpart;
  // adjoint
  const T* dZ;
  T* dval;
};

__device__ __forceinline__ void unpack(const float4& x, float* o) {
  o[0] = x.x;
  o[1] = x.y;
  o[2] = x.z;
  o[3] = x.w;
}
__device__ __forceinline__ void unpack(const double2& x, double* o) {
  o[0] = x.x;
  o[1] = x.y;
}

template <typename T, int M>
struct Row {
  static constexpr int W = VecT<T>::W;
  static constexpr int NV = (M + W - 1) / W;
};

__device__ __forceinline__ float4 tex_v4_ordered(cudaTextureObject_t t, int i) {
  float4 v;
  asm volatile("tex.1d.v4.f32.s32 {%0, %1, %2, %3}, [%4, {%5}];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(t), "r"(i));
  return v;
}

// The element stream and the Z rows are touched once per launch: they are
// marked evict-first in L2 so that they do not displace the factor rows, which
// are gathered again and again.
__device__ __forceinline__ uint64_t l2_evict_first() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_evict_last() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
// element stream: read once per launch, no L1 allocation, evict-first in L2
__device__ __forceinline__ uint32_t ld_stream(const uint32_t* p, uint64_t pol) {
  uint32_t v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ int32_t ld_stream(const int32_t* p, uint64_t pol) {
  return (int32_t)ld_stream((const uint32_t*)p, pol);
}
__device__ __forceinline__ float ld_stream(const float* p, uint64_t pol) {
  float v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ double ld_stream(const double* p, uint64_t pol) {
  double v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ float2 ld_row2(const float* p, uint64_t pol) {
  float2 v;
  asm volatile("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(p), "l"(pol));
  return v;
}
// gathered factor rows (16-byte vectors), evict-last in L2
__device__ __forceinline__ float4 ld_row(const float* p, uint64_t pol) {
  float4 v;
  asm volatile("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ double2 ld_row(const double* p, uint64_t pol) {
  double2 v;
  asm volatile("ld.global.nc.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;" : "=d"(v.x), "=d"(v.y) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ float4 tex_row_vec(cudaTextureObject_t t, int i, float) { return tex_v4_ordered(t, i); }
__device__ __forceinline__ double2 tex_row_vec(cudaTextureObject_t t, int i, double) {
  int4 v;
  asm volatile("tex.1d.v4.s32.s32 {%0, %1, %2, %3}, [%4, {%5}];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(t), "r"(i));
  return make_double2(__hiloint2double(v.y, v.x), __hiloint2double(v.w, v.z));
}

// Store-and-clear of accumulator registers in one asm block: the store is
// predicated on `on` and the registers are zeroed in place, so that the slice
// change inside the software-pipelined loop stays a real branch the compiler
// cannot turn into selects over a second copy of the accumulator.
__device__ __forceinline__ void st_clear(float* p, float& x, float& y, float& z, float& w, int on, uint64_t pol) {
  asm volatile(
      "{\n .reg .pred q;\n setp.ne.s32 q, %5, 0;\n"
      " @q st.global.L2::cache_hint.v4.f32 [%4], {%0, %1, %2, %3}, %6;\n"
      " mov.b32 %0, 0;\n mov.b32 %1, 0;\n mov.b32 %2, 0;\n mov.b32 %3, 0;\n}"
      : "+f"(x), "+f"(y), "+f"(z), "+f"(w)
      : "l"(p), "r"(on), "l"(pol)
      : "memory");
}
__device__ __forceinline__ void st_clear(double* p, double& x, double& y, int on, uint64_t pol) {
  asm volatile(
      "{\n .reg .pred q;\n setp.ne.s32 q, %3, 0;\n"
      " @q st.global.L2::cache_hint.v2.f64 [%2], {%0, %1}, %4;\n"
      " mov.b64 %0, 0;\n mov.b64 %1, 0;\n}"
      : "+d"(x), "+d"(y)
      : "l"(p), "r"(on), "l"(pol)
      : "memory");
}
__device__ __forceinline__ void st_clear1(float* p, float& x, int on) {
  asm volatile("{\n .reg .pred q;\n setp.ne.s32 q, %2, 0;\n @q st.global.f32 [%1], %0;\n mov.b32 %0, 0;\n}"
               : "+f"(x) : "l"(p), "r"(on) : "memory");
}
__device__ __forceinline__ void st_clear1(double* p, double& x, int on) {
  asm volatile("{\n .reg .pred q;\n setp.ne.s32 q, %2, 0;\n @q st.global.f64 [%1], %0;\n mov.b64 %0, 0;\n}"
               : "+d"(x) : "l"(p), "r"(on) : "memory");
}

constexpr uint32_t kNoCode = 0xFFFFFFFFu;  // no slice yet (row codes stay below 2^31 + 2^30 + 2^30)

// D elements' rows in flight per thread; OUTER: the tensor has outer modes
// (more than two other modes), whose scalings are gathered with the rows;
// OVR: values come from a caller's array (by original element id).
template <typename T, int MA, int MB, bool EA, bool EB, int D, bool OUTER, bool OVR, bool FIB = false>
__global__ void __launch_bounds__(128, 1) k_ttmc_fwd(const TtmcArgs<T> a) {
  using V = typename VecT<T>::type;
  constexpr int W = VecT<T>::W;
  constexpr int NA = Row<T, MA>::NV, NB = Row<T, MB>::NV;
  constexpr int NQ = OUTER ? TK_MAXN - 3 : 1;
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int g = (int)(gw % a.G);
  const int64_t bw = gw / a.G;
  if (bw * 32 >= a.P) return;
  const int bin = (int)(bw * 32 + lane);
  const int len = a.bin_len[bin];
  const int wlen = __reduce_max_sync(0xffffffffu, len);
  const int ka = EA ? MA : a.KA;
  const int jb = g % a.NB, o = g / a.NB;
  const int j0 = jb * a.TB;
  const int tb = EB ? MB : min(a.TB, a.KB - j0);
  // outer modes: loops run to the compile-time bound NQ with a runtime guard,
  // so that every per-mode array stays in registers
  const int nq_rt = a.nother - 2;
  int oc[NQ];
  if (OUTER) {
    int t = o;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      oc[q] = q < nq_rt ? t % a.Kf[q + 2] : 0;
      if (q < nq_rt) t /= a.Kf[q + 2];
    }
  }
  const int colbase = a.KA * j0 + a.KA * a.KB * o;
  const int64_t base = bw * a.limit * 32 + lane;  // slot of element k: base + 32 k
  const uint64_t pf = l2_evict_first(), pl = l2_evict_last();
  const bool twob = a.nother >= 2;

  T acc[MA * MB];
#pragma unroll
  for (int i = 0; i < MA * MB; ++i) acc[i] = T(0);
  uint32_t cur = kNoCode;
  T sf[FIB ? MA : 1], Bf[FIB ? MB : 1];
  int cur_lb = -1;
  if constexpr (FIB) {
#pragma unroll
    for (int i = 0; i < MA; ++i) sf[i] = T(0);
  }

  // writes the accumulator to the row (or split slot) of `code` when `on`, and
  // clears it either way
  auto flush_clear = [&](uint32_t code, int on) __attribute__((always_inline)) {
    T* dst = (code & TK_SPLIT_BIT) ? a.Zpart + ((int64_t)bin * 2 + ((code & TK_HEAD_BIT) ? 1 : 0)) * a.Khat
                                   : a.Z + (int64_t)(code & TK_ROW_MASK) * a.Khat;
    dst += colbase;
    if (EA && EB && (MA * MB) % W == 0 && a.store_vec) {
#pragma unroll
      for (int v = 0; v < MA * MB / W; ++v) {
        if constexpr (sizeof(T) == 4)
          st_clear(dst + v * W, acc[v * W], acc[v * W + 1], acc[v * W + 2], acc[v * W + 3], on, pf);
        else
          st_clear(dst + v * W, acc[v * W], acc[v * W + 1], on, pf);
      }
    } else {
#pragma unroll
      for (int jj = 0; jj < MB; ++jj)
#pragma unroll
        for (int i = 0; i < MA; ++i)
          st_clear1(dst + i + a.KA * jj, acc[i + MA * jj], on && (EB || jj < tb) && (EA || i < ka));
    }
  };

  // coordinates of element k, 2D ahead of use (the row gathers need them
  // first).  Slot min(k, limit-1) of the bin always holds valid values: an
  // element, or a padding slot zeroed at init (row 0, value 0, element 0), so
  // the loads need no select on their results and stay in flight; elements
  // past the bin's length are never accumulated.
  int nla[D], nlb[D], nq[D][NQ];
  auto slot = [&](int k) __attribute__((always_inline)) { return base + (int64_t)min(k, a.limit - 1) * 32; };
  auto fetch = [&](int d, int k) __attribute__((always_inline)) {
    const int64_t sl = slot(k);
    nla[d] = ld_stream(a.oidx[0] + sl, pf);
    nlb[d] = twob ? ld_stream(a.oidx[1] + sl, pf) : 0;
    if (OUTER) {
#pragma unroll
      for (int q = 0; q < NQ; ++q) nq[d][q] = q < nq_rt ? ld_stream(a.oidx[q + 2] + sl, pf) : 0;
    }
  };
  // rows of the element whose stream sits in slot d (D ahead of use); an
  // exact FP32 row whose length is 2 mod 4 ends with an 8-byte load
  constexpr int RA = (EA && sizeof(T) == 4 && MA % 4 == 2) ? MA : NA * W;
  constexpr int RB = (EB && sizeof(T) == 4 && MB % 4 == 2) ? MB : NB * W;
  T A[D][RA], B[D][RB];
  T v[D], fq[D][NQ];
  uint32_t code[D];
  int lbk[FIB ? D : 1];
  int prev_lb = -1;
  auto issue = [&](int d, int k) __attribute__((always_inline)) {
    // row code and value of element k, D ahead of use, with its rows
    {
      const int64_t sl = slot(k);
      code[d] = ld_stream(a.rowcode + sl, pf);
      if (OVR) v[d] = __ldg(a.vals_override + ld_stream(a.perm + sl, pf));
      else v[d] = ld_stream(a.val + sl, pf);
    }
    const T* ra = a.F[0] + (int64_t)nla[d] * a.ld[0];
#pragma unroll
    for (int u = 0; u < NA; ++u) {
      if (u * W + W <= RA) {
        if (EA || u * W < ka) unpack(ld_row(ra + u * W, pl), &A[d][u * W]);
        else for (int w = 0; w < W; ++w) A[d][u * W + w] = T(0);
      } else if constexpr (sizeof(T) == 4) {
        const float2 t = ld_row2((const float*)ra + u * W, pl);
        A[d][u * W] = t.x;
        A[d][u * W + 1] = t.y;
      }
    }
    bool needB = true;
    if constexpr (FIB) {
      lbk[d] = nlb[d];
      needB = nlb[d] != prev_lb;
      prev_lb = nlb[d];
    }
    if (twob && needB) {
      const int64_t rb = (int64_t)nlb[d] * a.ld[1] + j0;
#pragma unroll
      for (int u = 0; u < NB; ++u) {
        if (u * W + W <= RB) {
          if (EB || u * W < tb) unpack(a.texB && RB == NB * W ? tex_row_vec(a.texB, (int)(rb / W) + u, T(0)) : ld_row(a.F[1] + rb + u * W, pl), &B[d][u * W]);
          else for (int w = 0; w < W; ++w) B[d][u * W + w] = T(0);
        } else if constexpr (sizeof(T) == 4) {
          const float2 t = ld_row2((const float*)a.F[1] + rb + u * W, pl);
          B[d][u * W] = t.x;
          B[d][u * W + 1] = t.y;
        }
      }
    }
    if (OUTER) {
#pragma unroll
      for (int q = 0; q < NQ; ++q)
        fq[d][q] = q < nq_rt ? __ldg(a.F[q + 2] + (int64_t)nq[d][q] * a.ld[q + 2] + oc[q]) : T(1);
    }
  };

#pragma unroll
  for (int d = 0; d < D; ++d) fetch(d, d);
#pragma unroll
  for (int d = 0; d < D; ++d) {
    issue(d, d);
    fetch(d, d + D);
  }
#pragma unroll 1
  for (int j = 0; j < wlen; j += D) {
#pragma unroll
    for (int d = 0; d < D; ++d) {
      // element j+d sits in slot d: close the previous slice if it starts a
      // new one, use the element straight from the slot's registers, then
      // refill the slot with element j+d+D's rows and element j+d+2D's
      // coordinates (the other D-1 slots stay in flight meanwhile; no copies,
      // so the loop carries every slot in the same registers)
      if (FIB && j + d < len) {
        const uint32_t cd = code[d];
        const int lb = lbk[FIB ? d : 0];
        if (cd != cur || lb != cur_lb) {
          if (cur != kNoCode) {
#pragma unroll
            for (int jj = 0; jj < MB; ++jj)
#pragma unroll
              for (int i = 0; i < MA; ++i) acc[i + MA * jj] = fma(sf[i], Bf[jj], acc[i + MA * jj]);
          }
#pragma unroll
          for (int i = 0; i < MA; ++i) sf[i] = T(0);
          if (cd != cur) {
            flush_clear(cur == kNoCode ? 0u : cur, cur != kNoCode);
            cur = cd;
          }
          if (lb != cur_lb) {
#pragma unroll
            for (int jj = 0; jj < MB; ++jj) Bf[jj] = B[d][jj];
            cur_lb = lb;
          }
        }
        const T vcf = v[d];
#pragma unroll
        for (int i = 0; i < MA; ++i) sf[i] = fma(A[d][i], vcf, sf[i]);
      } else if (!FIB && j + d < len) {
        const uint32_t cd = code[d];
        if (cd != cur) {
          flush_clear(cur == kNoCode ? 0u : cur, cur != kNoCode);
          cur = cd;
        }
        T vc = v[d];
        if (OUTER) {
#pragma unroll
          for (int q = 0; q < NQ; ++q) vc *= fq[d][q];
        }
#pragma unroll
        for (int jj = 0; jj < MB; ++jj) {
          const T t = vc * (twob ? B[d][jj] : T(jj == 0));
#pragma unroll
          for (int i = 0; i < MA; ++i) acc[i + MA * jj] = fma(A[d][i], t, acc[i + MA * jj]);
        }
      }
      issue(d, j + d + D);
      fetch(d, j + d + 2 * D);
    }
  }
  if constexpr (FIB) {
    if (len > 0) {
#pragma unroll
      for (int jj = 0; jj < MB; ++jj)
#pragma unroll
        for (int i = 0; i < MA; ++i) acc[i + MA * jj] = fma(sf[i], Bf[jj], acc[i + MA * jj]);
    }
  }
  if (len > 0) flush_clear(cur, 1);
}

// Outputs of one element pass of the adjoint, all in the slot order of mode
// n's copy (slot s = the element's position in that copy):
//   dv[s]           dval of the element (scattered to original order at the end)
//   X[q][s * K_q]   its contribution to dF of the q-th other mode
// A null pointer skips that output; first != 0: the pass writes, else adds.
template <typename T>
struct BwdOut {
  T* dv;
  int first_dv;
  T* X[TK_MAXN - 1];
  int first[TK_MAXN - 1];
};

// Adjoint, element pass over mode n's copy for one column group g (groups are
// launched one after another, in order).  A thread walks its bin, stages the
// cotangent row dZ[row] of each slice once, and for every element computes
//     dv(e) (+)= so * <fa, D fb>                     (so: outer-mode scalings)
// and the element's contributions to dF of the other modes:
//     mode a:     X_a[s][i]        (+)= w so sum_j D[i,j] fb[j]
//     mode b:     X_b[s][j0 + j]   (+)= w so sum_i D[i,j] fa[i]
//     outer q:    X_q[s][oc_q]      += w <fa, D fb> prod_{q2 != q} F_q2[l_q2][oc_q2]
// Every slot is written by exactly one thread per launch, the 32 threads of a
// warp write consecutive slots (coalesced rows), there are no atomics and the
// order of the sums is fixed; the reduction to dF_m gathers X by slot.
template <typename T, int MA, int MB, bool EA, bool EB, int D, bool OUTER, bool OVR>
__global__ void __launch_bounds__(128, 1) k_bwd_elem(const TtmcArgs<T> a, int g, const BwdOut<T> out) {
  constexpr int W = VecT<T>::W;
  constexpr int NA = Row<T, MA>::NV, NB = Row<T, MB>::NV;
  constexpr int NQ = OUTER ? TK_MAXN - 3 : 1;
  const int lane = threadIdx.x & 31;
  const int64_t bw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (bw * 32 >= a.P) return;
  const int bin = (int)(bw * 32 + lane);
  const int len = a.bin_len[bin];
  const int wlen = __reduce_max_sync(0xffffffffu, len);
  const int ka = EA ? MA : a.KA;
  const int jb = g % a.NB, o = g / a.NB;
  const int j0 = jb * a.TB;
  const int tb = EB ? MB : min(a.TB, a.KB - j0);
  const int nq_rt = a.nother - 2;
  int oc[NQ];
  if (OUTER) {
    int t = o;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      oc[q] = q < nq_rt ? t % a.Kf[q + 2] : 0;
      if (q < nq_rt) t /= a.Kf[q + 2];
    }
  }
  const int colbase = a.KA * j0 + a.KA * a.KB * o;
  const int64_t base = bw * a.limit * 32 + lane;  // slot of element k: base + 32 k
  const uint64_t pf = l2_evict_first(), pl = l2_evict_last();
  const bool twob = a.nother >= 2;

  T Dt[MA * MB];  // the cotangent block of the current slice
  uint32_t cur = kNoCode;

  // the element pipeline of the forward kernel: coordinates 2D ahead, rows D
  // ahead, padding slots valid (zeroed at init)
  int nla[D], nlb[D], nq[D][NQ];
  auto slot = [&](int k) __attribute__((always_inline)) { return base + (int64_t)min(k, a.limit - 1) * 32; };
  auto fetch = [&](int d, int k) __attribute__((always_inline)) {
    const int64_t sl = slot(k);
    nla[d] = ld_stream(a.oidx[0] + sl, pf);
    nlb[d] = twob ? ld_stream(a.oidx[1] + sl, pf) : 0;
    if (OUTER) {
#pragma unroll
      for (int q = 0; q < NQ; ++q) nq[d][q] = q < nq_rt ? ld_stream(a.oidx[q + 2] + sl, pf) : 0;
    }
  };
  constexpr int RA = (EA && sizeof(T) == 4 && MA % 4 == 2) ? MA : NA * W;
  constexpr int RB = (EB && sizeof(T) == 4 && MB % 4 == 2) ? MB : NB * W;
  T A[D][RA], B[D][RB];
  T v[D], fq[D][NQ];
  uint32_t code[D];
  auto issue = [&](int d, int k) __attribute__((always_inline)) {
    {
      const int64_t sl = slot(k);
      code[d] = ld_stream(a.rowcode + sl, pf);
      if (OVR) v[d] = __ldg(a.vals_override + ld_stream(a.perm + sl, pf));
      else v[d] = ld_stream(a.val + sl, pf);
    }
    const T* ra = a.F[0] + (int64_t)nla[d] * a.ld[0];
#pragma unroll
    for (int u = 0; u < NA; ++u) {
      if (u * W + W <= RA) {
        if (EA || u * W < ka) unpack(ld_row(ra + u * W, pl), &A[d][u * W]);
        else for (int w = 0; w < W; ++w) A[d][u * W + w] = T(0);
      } else if constexpr (sizeof(T) == 4) {
        const float2 t = ld_row2((const float*)ra + u * W, pl);
        A[d][u * W] = t.x;
        A[d][u * W + 1] = t.y;
      }
    }
    if (twob) {
      const T* rb = a.F[1] + (int64_t)nlb[d] * a.ld[1] + j0;
#pragma unroll
      for (int u = 0; u < NB; ++u) {
        if (u * W + W <= RB) {
          if (EB || u * W < tb) unpack(ld_row(rb + u * W, pl), &B[d][u * W]);
          else for (int w = 0; w < W; ++w) B[d][u * W + w] = T(0);
        } else if constexpr (sizeof(T) == 4) {
          const float2 t = ld_row2((const float*)rb + u * W, pl);
          B[d][u * W] = t.x;
          B[d][u * W + 1] = t.y;
        }
      }
    } else {
#pragma unroll
      for (int u = 0; u < RB; ++u) B[d][u] = T(u == 0);
    }
    if (OUTER) {
#pragma unroll
      for (int q = 0; q < NQ; ++q)
        fq[d][q] = q < nq_rt ? __ldg(a.F[q + 2] + (int64_t)nq[d][q] * a.ld[q + 2] + oc[q]) : T(1);
    }
  };

#pragma unroll
  for (int d = 0; d < D; ++d) fetch(d, d);
#pragma unroll
  for (int d = 0; d < D; ++d) {
    issue(d, d);
    fetch(d, d + D);
  }
#pragma unroll 1
  for (int j = 0; j < wlen; j += D) {
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const int k = j + d;
      if (k < len) {
        const uint32_t cd = code[d];
        if (cd != cur) {
          const T* src = a.dZ + (int64_t)(cd & TK_ROW_MASK) * a.Khat + colbase;
          bool done = false;
          if constexpr (EA && MA % W == 0) {
            if (a.tile_vec) {
              using V = typename VecT<T>::type;
#pragma unroll
              for (int jj = 0; jj < MB; ++jj) {
#pragma unroll
                for (int u = 0; u < MA / W; ++u) {
                  if (EB || jj < tb) unpack(__ldg(reinterpret_cast<const V*>(src + a.KA * jj) + u), &Dt[MA * jj + u * W]);
                  else
#pragma unroll
                    for (int w = 0; w < W; ++w) Dt[MA * jj + u * W + w] = T(0);
                }
              }
              done = true;
            }
          }
          if (!done) {
#pragma unroll
            for (int jj = 0; jj < MB; ++jj)
#pragma unroll
              for (int i = 0; i < MA; ++i)
                Dt[i + MA * jj] = ((EB || jj < tb) && (EA || i < ka)) ? __ldg(src + i + a.KA * jj) : T(0);
          }
          cur = cd;
        }
        T so = T(1);
        if (OUTER) {
#pragma unroll
          for (int q = 0; q < NQ; ++q) so *= fq[d][q];
        }
        T x[MA], y[MB];
#pragma unroll
        for (int i = 0; i < MA; ++i) x[i] = T(0);
#pragma unroll
        for (int jj = 0; jj < MB; ++jj) {
          T yy = T(0);
#pragma unroll
          for (int i = 0; i < MA; ++i) {
            x[i] = fma(Dt[i + MA * jj], B[d][jj], x[i]);
            yy = fma(Dt[i + MA * jj], A[d][i], yy);
          }
          y[jj] = yy;
        }
        T dot = T(0);
#pragma unroll
        for (int i = 0; i < MA; ++i) dot = fma(A[d][i], x[i], dot);
        const int64_t sl = base + (int64_t)k * 32;
        if (out.dv) {
          T* dv = out.dv + sl;
          *dv = out.first_dv ? so * dot : *dv + so * dot;
        }
        const T w = v[d];
        const T ws = w * so;
        if (out.X[0]) {
          T* xr = out.X[0] + sl * a.KA;
          const bool f = out.first[0] != 0;
#pragma unroll
          for (int i = 0; i < MA; ++i)
            if (EA || i < ka) xr[i] = f ? ws * x[i] : xr[i] + ws * x[i];
        }
        if (twob && out.X[1]) {
          T* xr = out.X[1] + sl * a.KB + j0;
          const bool f = out.first[1] != 0;
#pragma unroll
          for (int jj = 0; jj < MB; ++jj)
            if (EB || jj < tb) xr[jj] = f ? ws * y[jj] : xr[jj] + ws * y[jj];
        }
        if (OUTER) {
#pragma unroll
          for (int q = 0; q < NQ; ++q) {
            if (q >= nq_rt || !out.X[q + 2]) continue;
            T prod = w * dot;
#pragma unroll
            for (int q2 = 0; q2 < NQ; ++q2)
              if (q2 != q && q2 < nq_rt) prod *= fq[d][q2];
            out.X[q + 2][sl * a.Kf[q + 2] + oc[q]] += prod;
          }
        }
      }
      issue(d, j + d + D);
      fetch(d, j + d + 2 * D);
    }
  }
}

// Adjoint, reduction over mode m's copy: every slice of mode m sums the
// contributions of its elements in the order of its copy (a thread per Lite
// bin, registers).  The contributions were written in the slot order of mode
// n's copy, so element e = perm_m[slot] reads row pos_n[e] of X.  Whole slices
// write their compact row of Zc, split pieces the bin's partial slots, which
// the fix-up adds in bin order.  A bin is one thread's chain of dependent
// gathers (perm -> pos -> row), so the loop keeps PD elements' rows and the
// next PD elements' row indices in flight: slot d holds element j + d's row and
// element j + d + PD's index, refilled right after the element is added.
template <typename T, int KM, int PD>
__global__ void __launch_bounds__(128) k_bwd_reduce(const T* __restrict__ X, int Km, const int32_t* __restrict__ perm,
                                                    const int32_t* __restrict__ pos_n,
                                                    const uint32_t* __restrict__ rowcode,
                                                    const int32_t* __restrict__ bin_len, int Pa, int limit,
                                                    T* __restrict__ Zc, T* __restrict__ Zpart) {
  const int bin = blockIdx.x * blockDim.x + threadIdx.x;
  if (bin >= Pa) return;
  const int len = bin_len[bin];
  if (len == 0) return;
  const int64_t base = (int64_t)(bin >> 5) * limit * 32 + (bin & 31);
  T acc[KM];
#pragma unroll
  for (int k = 0; k < KM; ++k) acc[k] = T(0);
  uint32_t cur = 0xFFFFFFFFu;
  auto flush = [&](uint32_t code) {
    T* dst = (code & TK_SPLIT_BIT) ? Zpart + ((int64_t)bin * 2 + ((code & TK_HEAD_BIT) ? 1 : 0)) * Km
                                   : Zc + (int64_t)(code & TK_ROW_MASK) * Km;
#pragma unroll
    for (int k = 0; k < KM; ++k)
      if (k < Km) dst[k] = acc[k];
  };
  // element k's slot; past the bin's end the last element is read again (never added)
  auto slot = [&](int k) __attribute__((always_inline)) { return base + (int64_t)min(k, len - 1) * 32; };
  auto index_of = [&](int k) __attribute__((always_inline)) { return __ldg(pos_n + __ldg(perm + slot(k))); };
  T xr[PD][KM];
  uint32_t cc[PD];
  int nx[PD];
  auto fetch_row = [&](int d, int k, int p) __attribute__((always_inline)) {
    cc[d] = __ldg(rowcode + slot(k));
    const T* r = X + (int64_t)p * Km;
#pragma unroll
    for (int q = 0; q < KM; ++q) xr[d][q] = q < Km ? __ldg(r + q) : T(0);
  };
#pragma unroll
  for (int d = 0; d < PD; ++d) fetch_row(d, d, index_of(d));
#pragma unroll
  for (int d = 0; d < PD; ++d) nx[d] = index_of(d + PD);
#pragma unroll 1
  for (int j = 0; j < len; j += PD) {
#pragma unroll
    for (int d = 0; d < PD; ++d) {
      if (j + d < len) {
        if (cc[d] != cur) {
          if (cur != 0xFFFFFFFFu) flush(cur);
#pragma unroll
          for (int q = 0; q < KM; ++q) acc[q] = T(0);
          cur = cc[d];
        }
#pragma unroll
        for (int q = 0; q < KM; ++q) acc[q] += xr[d][q];
      }
      fetch_row(d, j + d + PD, nx[d]);
      nx[d] = index_of(j + d + 2 * PD);
    }
  }
  flush(cur);
}

// dF[row_id[r]][k] += Zc[r][k]
template <typename T>
__global__ void k_add_rows(const T* __restrict__ Zc, int R, int Km, const int32_t* __restrict__ row_id, T* __restrict__ dF) {
  const int64_t total = (int64_t)R * Km;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    const int64_t r = i / Km;
    const int k = (int)(i - r * Km);
    dF[(int64_t)row_id[r] * Km + k] += Zc[i];
  }
}

// dval[perm[slot]] = dv[slot] for the occupied slots of mode n's copy
template <typename T>
__global__ void k_dv_scatter(const T* __restrict__ dv, const int32_t* __restrict__ perm,
                             const int32_t* __restrict__ bin_len, int Pa, int limit, T* __restrict__ dval) {
  const int64_t cap = (int64_t)Pa * limit;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; slot < cap; slot += stride) {
    const int lane = (int)(slot & 31);
    const int64_t rest = slot >> 5;
    const int64_t k = rest % limit;
    const int p = (int)((rest / limit) * 32 + lane);
    if (k < bin_len[p]) dval[perm[slot]] = dv[slot];
  }
}

// pos[perm[slot]] = slot for the occupied slots of a mode's copy
__global__ void k_inv_pos(const int32_t* __restrict__ perm, const int32_t* __restrict__ bin_len, int Pa, int limit,
                          int32_t* __restrict__ pos) {
  const int64_t cap = (int64_t)Pa * limit;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; slot < cap; slot += stride) {
    const int lane = (int)(slot & 31);
    const int64_t rest = slot >> 5;
    const int64_t k = rest % limit;
    const int p = (int)((rest / limit) * 32 + lane);
    if (k < bin_len[p]) pos[perm[slot]] = (int32_t)slot;
  }
}

// Split-slice fix-up, level 1: one CTA per (chunk of <= 256 bins of one split
// slice, 32 columns).  Warp w adds bins b0+w, b0+w+8, ... in order; the 8 warp
// sums are combined in order.  Bin bhead holds the slice's head piece in slot
// 1; later bins with a stage-2 gap hold a tail piece in slot 0.
template <typename T>
__global__ void __launch_bounds__(256) k_fixup_chunks(const T* __restrict__ Zpart, int Khat,
                                                      const int32_t* chunk_split, const int32_t* chunk_b0,
                                                      const int32_t* chunk_b1, const int32_t* split_bhead,
                                                      const int32_t* gap2, const int32_t* split_chunk0,
                                                      const int32_t* split_row, T* Z, double* Zchunk) {
  __shared__ double part[8][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int chunk = blockIdx.x;
  const int col = blockIdx.y * 32 + lane;
  const int k = chunk_split[chunk], b0 = chunk_b0[chunk], b1 = chunk_b1[chunk], bh = split_bhead[k];
  double acc = 0.0;
  if (col < Khat) {
    for (int b = b0 + w; b < b1; b += 8) {
      const int slot = (b == bh) ? 1 : (gap2[b] > 0 ? 0 : -1);
      if (slot >= 0) acc += (double)Zpart[((int64_t)b * 2 + slot) * Khat + col];
    }
  }
  part[w][lane] = acc;
  __syncthreads();
  if (w == 0 && col < Khat) {
    double s = 0.0;
#pragma unroll
    for (int ww = 0; ww < 8; ++ww) s += part[ww][lane];
    if (split_chunk0[k + 1] - split_chunk0[k] == 1) Z[(int64_t)split_row[k] * Khat + col] = (T)s;
    else Zchunk[(int64_t)chunk * Khat + col] = s;
  }
}

// Level 2: slices with several chunks add their chunk sums in order.
template <typename T>
__global__ void k_fixup_final(int Khat, const int32_t* split_chunk0, const int32_t* split_row, const double* Zchunk,
                              T* Z) {
  const int k = blockIdx.x;
  const int col = blockIdx.y * blockDim.x + threadIdx.x;
  if (col >= Khat) return;
  const int c0 = split_chunk0[k], c1 = split_chunk0[k + 1];
  if (c1 - c0 <= 1) return;
  double s = 0.0;
  for (int c = c0; c < c1; ++c) s += Zchunk[(int64_t)c * Khat + col];
  Z[(int64_t)split_row[k] * Khat + col] = (T)s;
}

// dst[dst_map ? dst_map[r] : r][:] = src[src_map ? src_map[r] : r][:cols], zero padded to ldd
template <typename T>
__global__ void k_copy_factor(const T* __restrict__ src, int lds, T* __restrict__ dst, int ldd, int64_t rows, int cols,
                              const int32_t* __restrict__ dst_map, const int32_t* __restrict__ src_map) {
  const int64_t total = rows * ldd;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    const int64_t r = i / ldd;
    const int cc = (int)(i - r * ldd);
    const int64_t dr = dst_map ? dst_map[r] : r;
    const int64_t sr = src_map ? src_map[r] : r;
    dst[dr * ldd + cc] = cc < cols ? src[sr * lds + cc] : T(0);
  }
}

struct Tile {
  int MA, MB;
  bool EA, EB;
};
constexpr Tile kTilesF[] = {{10, 10, true, true}, {8, 8, true, true}, {16, 8, true, true}, {16, 8, false, false},
                            {32, 4, false, false}};
constexpr Tile kTilesD[] = {{10, 4, true, false}, {8, 4, true, true}, {16, 4, true, true}, {16, 4, false, false},
                            {32, 2, false, false}};
constexpr int kNumTiles = 5;

template <typename T>
using KernelT = void (*)(TtmcArgs<T>);

// Rows in flight per thread for each tile (register budget: the accumulator
// plus D elements' rows must stay within 255 registers).
#define TK_FWD_PICK(T, MA, MB, EA, EB, D)                                                        \
  (outer ? (ovr ? k_ttmc_fwd<T, MA, MB, EA, EB, D, true, true> : k_ttmc_fwd<T, MA, MB, EA, EB, D, true, false>) \
         : (ovr ? k_ttmc_fwd<T, MA, MB, EA, EB, D, false, true> : k_ttmc_fwd<T, MA, MB, EA, EB, D, false, false>))
template <typename T>
KernelT<T> fwd_kernel(int id, bool outer, bool ovr);
template <>
KernelT<float> fwd_kernel<float>(int id, bool outer, bool ovr) {
  switch (id) {
    case 0: return TK_FWD_PICK(float, 10, 10, true, true, 4);
    case 1: return TK_FWD_PICK(float, 8, 8, true, true, 4);
    case 2: return TK_FWD_PICK(float, 16, 8, true, true, 2);
    case 3: return TK_FWD_PICK(float, 16, 8, false, false, 2);
    default: return TK_FWD_PICK(float, 32, 4, false, false, 2);
  }
}
template <>
KernelT<double> fwd_kernel<double>(int id, bool outer, bool ovr) {
  switch (id) {
    case 0: return TK_FWD_PICK(double, 10, 4, true, false, 3);
    case 1: return TK_FWD_PICK(double, 8, 4, true, true, 3);
    case 2: return TK_FWD_PICK(double, 16, 4, true, true, 2);
    case 3: return TK_FWD_PICK(double, 16, 4, false, false, 2);
    default: return TK_FWD_PICK(double, 32, 2, false, false, 1);
  }
}
#undef TK_FWD_PICK
// Fiber-factored forms (FP32, exact tiles, two remaining modes): one element
// fewer in flight for the fiber sum and the current fiber's row
KernelT<float> fib_kernel(int id, bool ovr) {
  switch (id) {
    case 0: return ovr ? k_ttmc_fwd<float, 10, 10, true, true, 3, false, true, true>
                       : k_ttmc_fwd<float, 10, 10, true, true, 3, false, false, true>;
    case 1: return ovr ? k_ttmc_fwd<float, 8, 8, true, true, 3, false, true, true>
                       : k_ttmc_fwd<float, 8, 8, true, true, 3, false, false, true>;
    case 2: return ovr ? k_ttmc_fwd<float, 16, 8, true, true, 2, false, true, true>
                       : k_ttmc_fwd<float, 16, 8, true, true, 2, false, false, true>;
    default: return nullptr;
  }
}

template <typename T>
using BwdKernelT = void (*)(TtmcArgs<T>, int, BwdOut<T>);
// rows in flight per thread for the adjoint: the cotangent block plus D
// elements' rows within the register budget
#define TK_BWD_PICK(T, MA, MB, EA, EB, D)                                                                \
  (outer ? (ovr ? k_bwd_elem<T, MA, MB, EA, EB, D, true, true> : k_bwd_elem<T, MA, MB, EA, EB, D, true, false>) \
         : (ovr ? k_bwd_elem<T, MA, MB, EA, EB, D, false, true> : k_bwd_elem<T, MA, MB, EA, EB, D, false, false>))
template <typename T>
BwdKernelT<T> bwd_kernel(int id, bool outer, bool ovr);
template <>
BwdKernelT<float> bwd_kernel<float>(int id, bool outer, bool ovr) {
  switch (id) {
    case 0: return TK_BWD_PICK(float, 10, 10, true, true, 3);
    case 1: return TK_BWD_PICK(float, 8, 8, true, true, 4);
    case 2: return TK_BWD_PICK(float, 16, 8, true, true, 2);
    case 3: return TK_BWD_PICK(float, 16, 8, false, false, 2);
    default: return TK_BWD_PICK(float, 32, 4, false, false, 1);
  }
}
template <>
BwdKernelT<double> bwd_kernel<double>(int id, bool outer, bool ovr) {
  switch (id) {
    case 0: return TK_BWD_PICK(double, 10, 4, true, false, 2);
    case 1: return TK_BWD_PICK(double, 8, 4, true, true, 2);
    case 2: return TK_BWD_PICK(double, 16, 4, true, true, 1);
    case 3: return TK_BWD_PICK(double, 16, 4, false, false, 1);
    default: return TK_BWD_PICK(double, 32, 2, false, false, 1);
  }
}
#undef TK_BWD_PICK

struct Plan {
  int tile_id;
  Tile tile;
  int KA, KB, NB, G;
  int others[TK_MAXN - 1];
  int nother;
};

Plan make_plan(const tucker_ctx* c, int n) {
  Plan p{};
  p.nother = 0;
  for (int m = 0; m < c->N; ++m)
    if (m != n) p.others[p.nother++] = m;
  p.KA = c->K[p.others[0]];
  p.KB = p.nother >= 2 ? c->K[p.others[1]] : 1;
  const Tile* tiles = c->prec == TUCKER_FP32 ? kTilesF : kTilesD;
  p.tile_id = -1;
  for (int i = 0; i < kNumTiles; ++i) {
    const Tile& t = tiles[i];
    const bool okA = t.EA ? p.KA == t.MA : p.KA <= t.MA;
    // an exact b block must start on a vector boundary of the padded rows
    const bool okB = t.EB ? (p.KB % t.MB == 0 && (p.KB == t.MB || t.MB % (16 / c->esz) == 0)) : true;
    if (okA && okB) {
      p.tile_id = i;
      p.tile = t;
      break;
    }
  }
  if (p.tile_id < 0) tk_throw(TUCKER_ERR_ARG, "core length of the first remaining mode exceeds 32");
  p.NB = (int)tk_ceil_div(p.KB, p.tile.MB);
  p.G = p.NB;
  for (int q = 2; q < p.nother; ++q) p.G *= c->K[p.others[q]];
  return p;
}

template <typename T>
TtmcArgs<T> make_args(tucker_ctx* c, int n, const Plan& pl, void* const* F, const int* ldF, const void* vals_override) {
  const tk_mode& md = c->mode[n];
  TtmcArgs<T> a{};
  a.rowcode = md.rowcode;
  for (int q = 0; q < pl.nother; ++q) {
    a.oidx[q] = md.oidx[q];
    a.F[q] = (const T*)F[pl.others[q]];
    a.ld[q] = ldF[pl.others[q]];
    a.Kf[q] = c->K[pl.others[q]];
  }
  a.val = (const T*)md.val;
  a.perm = md.perm;
  a.bin_len = md.bin_len;
  a.vals_override = (const T*)vals_override;
  a.nother = pl.nother;
  a.P = md.Pa;  // padded bins have length 0
  a.limit = md.limit;
  a.G = pl.G;
  a.NB = pl.NB;
  a.TB = pl.tile.MB;
  a.KA = pl.KA;
  a.KB = pl.KB;
  a.Khat = md.Khat;
  return a;
}


unsigned blocks_for(const tk_mode& md, int G) {
  const int64_t warps = (int64_t)(md.Pa / 32) * G;
  return (unsigned)tk_ceil_div(warps, 4);
}

template <typename T>
void forward_impl(tucker_ctx* c, int n, void* const* F, const int* ldF, const void* vals_override, void* Z,
                  cudaStream_t s) {
  tk_mode& md = c->mode[n];
  const Plan pl = make_plan(c, n);
  TtmcArgs<T> a = make_args<T>(c, n, pl, F, ldF, vals_override);
  a.Z = (T*)Z;
  a.Zpart = (T*)c->Zpart;
  a.store_vec = ((uintptr_t)Z % 16 == 0) && (md.Khat % VecT<T>::W == 0) &&
                ((pl.KA * pl.tile.MB) % VecT<T>::W == 0);
  a.texB = pl.nother >= 2 ? tk_factor_tex(c, F[pl.others[1]]) : 0;
  tk_phase_begin(c, PH_TTM, s);
  if (md.tc) {
    tk_ttmc_tc_launch(c, n, F, ldF, vals_override, Z, s);
  } else {
    KernelT<T> kern = fwd_kernel<T>(pl.tile_id, pl.nother > 2, vals_override != nullptr);
    if constexpr (sizeof(T) == 4) {
      // the fiber-factored form where it applies (tucker_opts.ttm_path = 2)
      if (c->ttm_path == 2 && pl.nother == 2 && c->fiber[n] == pl.others[1]) {
        KernelT<float> f = fib_kernel(pl.tile_id, vals_override != nullptr);
        if (f) kern = f;
      }
    }
    kern<<<blocks_for(md, pl.G), 128, 0, s>>>(a);
    TK_CUDA(cudaGetLastError());
  }
  tk_phase_end(c, s);
  tk_launched(c, PH_TTM);
  if (md.nsplit > 0) {
    tk_phase_begin(c, PH_FIXUP, s);
    dim3 g1(md.nchunks, (unsigned)tk_ceil_div(md.Khat, 32));
    k_fixup_chunks<T><<<g1, 256, 0, s>>>((const T*)c->Zpart, md.Khat, md.chunk_split, md.chunk_b0, md.chunk_b1,
                                         md.split_bhead, md.gap2, md.split_chunk0, md.split_row, (T*)Z, c->Zchunk);
    TK_CUDA(cudaGetLastError());
    dim3 g2(md.nsplit, (unsigned)tk_ceil_div(md.Khat, 128));
    k_fixup_final<T><<<g2, 128, 0, s>>>(md.Khat, md.split_chunk0, md.split_row, c->Zchunk, (T*)Z);
    TK_CUDA(cudaGetLastError());
    tk_phase_end(c, s);
    tk_launched(c, PH_FIXUP, 2);
  }
}

// Sets of other modes whose dF contributions one element pass produces
// together: both for a 3-mode tensor, one at a time above (the per-slot
// contribution buffers grow with the number of targets).
int bwd_sets(int nother, int (*sets)[TK_MAXN - 1], int* sizes) {
  if (nother <= 2) {
    for (int q = 0; q < nother; ++q) sets[0][q] = q;
    sizes[0] = nother;
    return 1;
  }
  for (int q = 0; q < nother; ++q) {
    sets[q][0] = q;
    sizes[q] = 1;
  }
  return nother;
}

// Adjoint workspace, allocated by the first backward call of a context:
// element slots of every mode's copy, the per-slot dval and contribution
// buffers (slot order of the TTM-chain mode's copy), the compact reduction
// result and the fix-up scratch.
void ensure_bwd_workspace(tucker_ctx* c, cudaStream_t s) {
  if (c->bwd_ready) return;
  c->alloc_stream = s;
  int64_t xcap = 0, dvcap = 0, zc = 0, zp = 0, zch = 0;
  for (int n = 0; n < c->N; ++n) {
    const tk_mode& md = c->mode[n];
    int others[TK_MAXN - 1], no = 0;
    for (int m = 0; m < c->N; ++m)
      if (m != n) others[no++] = m;
    int sets[TK_MAXN - 1][TK_MAXN - 1], sizes[TK_MAXN - 1];
    const int ns = bwd_sets(no, sets, sizes);
    for (int t = 0; t < ns; ++t) {
      int64_t k = 0;
      for (int i = 0; i < sizes[t]; ++i) k += c->K[others[sets[t][i]]];
      xcap = std::max(xcap, md.cap * k);
    }
    dvcap = std::max(dvcap, md.cap);
    zc = std::max(zc, (int64_t)md.R * c->K[n]);
    zp = std::max(zp, (int64_t)2 * md.Pa * c->K[n]);
    zch = std::max(zch, (int64_t)md.nchunks * c->K[n]);
  }
  for (int m = 0; m < c->N; ++m) {
    const tk_mode& md = c->mode[m];
    c->bwd_pos[m] = (int32_t*)tk_alloc(c, (size_t)c->nnz * 4);
    k_inv_pos<<<(unsigned)std::min<int64_t>(tk_ceil_div(md.cap, 256), 1 << 20), 256, 0, s>>>(md.perm, md.bin_len, md.Pa,
                                                                                         md.limit, c->bwd_pos[m]);
    TK_CUDA(cudaGetLastError());
  }
  c->bwd_X = tk_alloc(c, (size_t)std::max<int64_t>(xcap, 1) * c->esz);
  c->bwd_dv = tk_alloc(c, (size_t)std::max<int64_t>(dvcap, 1) * c->esz);
  c->bwd_Zc = tk_alloc(c, (size_t)std::max<int64_t>(zc, 1) * c->esz);
  c->bwd_Zp = tk_alloc(c, (size_t)std::max<int64_t>(zp, 1) * c->esz);
  c->bwd_Zch = (double*)tk_alloc(c, (size_t)std::max<int64_t>(zch, 1) * 8);
  c->bwd_ready = true;
}

// dF_m += the contributions X (slot order of mode n's copy, rows of K_m)
template <typename T>
void reduce_into(tucker_ctx* c, int m, int n, const T* X, T* dF, cudaStream_t s) {
  tk_mode& md = c->mode[m];
  const int Km = c->K[m];
  const int32_t* pos_n = c->bwd_pos[n];
  T* Zc = (T*)c->bwd_Zc;
  T* Zp = (T*)c->bwd_Zp;
  const unsigned grid = (unsigned)tk_ceil_div(md.Pa, 128);
  // rows in flight per thread: 128 registers' worth
  constexpr int R = 128 * 4 / (int)sizeof(T);
  if (Km <= 8)
    k_bwd_reduce<T, 8, R / 8 < 8 ? R / 8 : 8><<<grid, 128, 0, s>>>(X, Km, md.perm, pos_n, md.rowcode, md.bin_len,
                                                                    md.Pa, md.limit, Zc, Zp);
  else if (Km <= 16)
    k_bwd_reduce<T, 16, R / 16><<<grid, 128, 0, s>>>(X, Km, md.perm, pos_n, md.rowcode, md.bin_len, md.Pa, md.limit,
                                                    Zc, Zp);
  else
    k_bwd_reduce<T, 32, R / 32><<<grid, 128, 0, s>>>(X, Km, md.perm, pos_n, md.rowcode, md.bin_len, md.Pa, md.limit,
                                                    Zc, Zp);
  TK_CUDA(cudaGetLastError());
  if (md.nsplit > 0) {
    dim3 g1(md.nchunks, (unsigned)tk_ceil_div(Km, 32));
    k_fixup_chunks<T><<<g1, 256, 0, s>>>(Zp, Km, md.chunk_split, md.chunk_b0, md.chunk_b1, md.split_bhead, md.gap2,
                                         md.split_chunk0, md.split_row, Zc, c->bwd_Zch);
    TK_CUDA(cudaGetLastError());
    dim3 g2(md.nsplit, (unsigned)tk_ceil_div(Km, 128));
    k_fixup_final<T><<<g2, 128, 0, s>>>(Km, md.split_chunk0, md.split_row, c->bwd_Zch, Zc);
    TK_CUDA(cudaGetLastError());
  }
  const int64_t total = (int64_t)md.R * Km;
  k_add_rows<T><<<(unsigned)std::min<int64_t>(tk_ceil_div(total > 0 ? total : 1, 256), 8192), 256, 0, s>>>(
      Zc, md.R, Km, md.row_id, dF);
  TK_CUDA(cudaGetLastError());
  tk_launched(c, PH_BWD, md.nsplit > 0 ? 4 : 2);
}

template <typename T>
void backward_impl(tucker_ctx* c, int n, void* const* F, const int* ldF, const void* dZ, const void* vals_override,
                   void* const* dF, void* dval, cudaStream_t s) {
  tk_mode& md = c->mode[n];
  const Plan pl = make_plan(c, n);
  TtmcArgs<T> a = make_args<T>(c, n, pl, F, ldF, vals_override);
  a.dZ = (const T*)dZ;
  {
    const int W = 16 / (int)sizeof(T);
    a.tile_vec = ((uintptr_t)dZ % 16 == 0) && md.Khat % W == 0 && pl.KA % W == 0;
  }
  BwdKernelT<T> kern = bwd_kernel<T>(pl.tile_id, pl.nother > 2, vals_override != nullptr);
  const unsigned grid = blocks_for(md, 1);
  tk_phase_begin(c, PH_BWD, s);
  ensure_bwd_workspace(c, s);
  T* Xbase = (T*)c->bwd_X;
  T* dv = (T*)c->bwd_dv;
  bool dval_pending = dval != nullptr;
  auto element_passes = [&](BwdOut<T> o) {
    for (int g = 0; g < pl.G; ++g) {
      // X of mode a: every group adds to all K_a columns (the first writes);
      // of mode b: group g owns the column block jb = g % NB (the first outer
      // combination writes); of an outer mode: zeroed before, always added
      o.first_dv = g == 0;
      o.first[0] = g == 0;
      o.first[1] = g < pl.NB;
      kern<<<grid, 128, 0, s>>>(a, g, o);
      TK_CUDA(cudaGetLastError());
    }
    tk_launched(c, PH_BWD, pl.G);
    if (o.dv) {
      k_dv_scatter<T><<<(unsigned)std::min<int64_t>(tk_ceil_div(md.cap, 256), 1 << 20), 256, 0, s>>>(
          dv, md.perm, md.bin_len, md.Pa, md.limit, (T*)dval);
      TK_CUDA(cudaGetLastError());
      tk_launched(c, PH_BWD, 1);
    }
  };
  int sets[TK_MAXN - 1][TK_MAXN - 1], sizes[TK_MAXN - 1];
  const int nsets = bwd_sets(pl.nother, sets, sizes);
  for (int t = 0; t < nsets; ++t) {
    BwdOut<T> o{};
    T* X[TK_MAXN - 1] = {};
    int64_t off = 0;
    bool any = false;
    for (int i = 0; i < sizes[t]; ++i) {
      const int q = sets[t][i], m = pl.others[q];
      if (!dF || !dF[m]) continue;
      X[q] = Xbase + off;
      off += md.cap * c->K[m];
      if (q >= 2) TK_CUDA(cudaMemsetAsync(X[q], 0, (size_t)md.cap * c->K[m] * sizeof(T), s));
      o.X[q] = X[q];
      any = true;
    }
    if (!any) continue;
    o.dv = dval_pending ? dv : nullptr;
    element_passes(o);
    dval_pending = false;
    for (int q = 0; q < pl.nother; ++q)
      if (X[q]) reduce_into<T>(c, pl.others[q], n, X[q], (T*)dF[pl.others[q]], s);
  }
  if (dval_pending) {
    BwdOut<T> o{};
    o.dv = dv;
    element_passes(o);
  }
  tk_phase_end(c, s);
}

}  // namespace

int tk_ttmc_groups(const tucker_ctx* c, int n) { return make_plan(c, n).G; }

int tk_ttmc_threads_per_sm(const tucker_ctx* c, int n) {
  const Plan pl = make_plan(c, n);
  int nb = 0;
  if (c->prec == TUCKER_FP32)
    TK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fwd_kernel<float>(pl.tile_id, pl.nother > 2, false), 128, 0));
  else
    TK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fwd_kernel<double>(pl.tile_id, pl.nother > 2, false), 128, 0));
  return std::max(1, nb) * 128;
}

void tk_ttmc_forward(tucker_ctx* c, int n, void* const* F, const int* ldF, const void* vals_override, void* Z,
                     cudaStream_t s) {
  if (c->prec == TUCKER_FP32) forward_impl<float>(c, n, F, ldF, vals_override, Z, s);
  else forward_impl<double>(c, n, F, ldF, vals_override, Z, s);
}

void tk_ttmc_backward(tucker_ctx* c, int n, void* const* F, const int* ldF, const void* dZ, const void* vals_override,
                      void* const* dF, void* dval, cudaStream_t s) {
  if (c->prec == TUCKER_FP32) backward_impl<float>(c, n, F, ldF, dZ, vals_override, dF, dval, s);
  else backward_impl<double>(c, n, F, ldF, dZ, vals_override, dF, dval, s);
}

void tk_copy_factor(tucker_ctx* c, const void* src, int lds, void* dst, int ldd, int64_t rows, int cols,
                    const int32_t* dst_map, const int32_t* src_map, cudaStream_t s) {
  const int64_t total = rows * ldd;
  const unsigned grid = (unsigned)std::min<int64_t>(tk_ceil_div(total > 0 ? total : 1, 256), 8192);
  if (c->prec == TUCKER_FP32)
    k_copy_factor<float><<<grid, 256, 0, s>>>((const float*)src, lds, (float*)dst, ldd, rows, cols, dst_map, src_map);
  else
    k_copy_factor<double><<<grid, 256, 0, s>>>((const double*)src, lds, (double*)dst, ldd, rows, cols, dst_map, src_map);
  TK_CUDA(cudaGetLastError());
  tk_launched(c, PH_OTHER);
}
