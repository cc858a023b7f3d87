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
// The kernel is bound by the latency of the two row gathers per element: the
// F_a row is read through the LSU path and the F_b block through the texture
// path (two L1 pipelines), the exact FP32 tiles of 3-mode tensors take two
// elements per step with all four rows requested before either is used (more
// loads in flight per SM at 8 warps than one element at 12), and the element
// stream and the Z rows carry an L2 evict-first policy so that the reused
// factor rows stay in L2.
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
  int chunk;  // staged steps per buffer
  T* Z;
  T* Zpart;
  // adjoint
  const T* dZ;
  T* dF[TK_MAXN - 1];
  int ldd[TK_MAXN - 1];
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
__device__ __forceinline__ float4 pack(const float* i) { return make_float4(i[0], i[1], i[2], i[3]); }
__device__ __forceinline__ double2 pack(const double* i) { return make_double2(i[0], i[1]); }

template <typename T, int M>
struct Row {
  static constexpr int W = VecT<T>::W;
  static constexpr int NV = (M + W - 1) / W;
  static constexpr int R = NV * W;
};

// Loads the first `valid` entries of a 16-byte aligned row (whole vectors);
// entries past `valid` inside a loaded vector are the row's zero padding.
template <typename T, int M>
__device__ __forceinline__ void load_row(const T* __restrict__ row, int valid, T (&out)[Row<T, M>::R]) {
  using V = typename VecT<T>::type;
  constexpr int W = VecT<T>::W;
#pragma unroll
  for (int v = 0; v < Row<T, M>::NV; ++v) {
    if (v * W < valid) {
      unpack(__ldg(reinterpret_cast<const V*>(row) + v), &out[v * W]);
    } else {
#pragma unroll
      for (int u = 0; u < W; ++u) out[v * W + u] = T(0);
    }
  }
}

// The same through the texture path (texel = one 16-byte vector), so that the
// two gathered rows of an element use the LSU and the texture pipelines.
__device__ __forceinline__ void tex_vec(cudaTextureObject_t t, int i, float* o) {
  unpack(tex1Dfetch<float4>(t, i), o);
}
__device__ __forceinline__ void tex_vec(cudaTextureObject_t t, int i, double* o) {
  const int4 v = tex1Dfetch<int4>(t, i);
  o[0] = __hiloint2double(v.y, v.x);
  o[1] = __hiloint2double(v.w, v.z);
}
template <typename T, int M>
__device__ __forceinline__ void tex_row(cudaTextureObject_t t, int64_t first, int valid, T (&out)[Row<T, M>::R]) {
  constexpr int W = VecT<T>::W;
#pragma unroll
  for (int v = 0; v < Row<T, M>::NV; ++v) {
    if (v * W < valid) {
      tex_vec(t, (int)(first / W) + v, &out[v * W]);
    } else {
#pragma unroll
      for (int u = 0; u < W; ++u) out[v * W + u] = T(0);
    }
  }
}

// Loads issued in program order (volatile), so that the rows of two elements
// are all requested before either is used.
__device__ __forceinline__ float4 ldg_v4_ordered(const float* p) {
  float4 v;
  asm volatile("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
  return v;
}
__device__ __forceinline__ float4 tex_v4_ordered(cudaTextureObject_t t, int i) {
  float4 v;
  asm volatile("tex.1d.v4.f32.s32 {%0, %1, %2, %3}, [%4, {%5}];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(t), "r"(i));
  return v;
}

// ---------------------------------------------------------------- staging
// Each warp streams the element arrays of its 32 bins through shared memory:
// steps [k0, k0+C) of a warp occupy one contiguous span per array (the
// warp-interleaved layout), copied with 16-byte cp.async into one of two
// buffers while the other buffer is being consumed.
// The element stream and the Z rows are touched once per launch: they are
// marked evict-first in L2 so that they do not displace the factor rows, which
// are gathered again and again.
__device__ __forceinline__ uint64_t l2_evict_first() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gsrc),
               "l"(l2_evict_first())
               : "memory");
}
__device__ __forceinline__ void st_stream(float4* p, const float4& v) {
  asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z),
               "f"(v.w), "l"(l2_evict_first())
               : "memory");
}
__device__ __forceinline__ void st_stream(double2* p, const double2& v) {
  asm volatile("st.global.L2::cache_hint.v2.f64 [%0], {%1, %2}, %3;" ::"l"(p), "d"(v.x), "d"(v.y),
               "l"(l2_evict_first())
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__device__ __forceinline__ void stage_span(void* sdst, const void* gsrc, int bytes, int lane) {
#pragma unroll 1
  for (int off = lane * 16; off < bytes; off += 32 * 16) cp_async16((char*)sdst + off, (const char*)gsrc + off);
}

// One staging buffer of C steps: code[C*32], oidx_q[C*32] (q < nother),
// then val[C*32] (type T, if staged) and perm[C*32] (if staged).
template <typename T>
__host__ __device__ inline int stage_bytes(int C, int nother, bool val, bool perm) {
  return C * 32 * (4 * (1 + nother) + (val ? (int)sizeof(T) : 0) + (perm ? 4 : 0));
}

template <typename T>
__device__ __forceinline__ void issue_chunk(const TtmcArgs<T>& a, char* buf, int CW, int64_t wbase, int k0, int ns,
                                            int lane, bool val, bool perm) {
  const int64_t off = (wbase + k0) * 32;
  const int b4 = ns * 32 * 4;
  uint32_t* w = (uint32_t*)buf;
  stage_span(w, a.rowcode + off, b4, lane);
#pragma unroll 1
  for (int q = 0; q < a.nother; ++q) stage_span(w + (1 + q) * CW, a.oidx[q] + off, b4, lane);
  char* vb = (char*)(w + (1 + a.nother) * CW);
  if (val) {
    stage_span(vb, a.val + off, ns * 32 * (int)sizeof(T), lane);
    vb += (size_t)CW * sizeof(T);
  }
  if (perm) stage_span(vb, a.perm + off, b4, lane);
}

template <typename T, int MA, int MB, bool EA, bool EB>
__global__ void __launch_bounds__(128) k_ttmc_fwd(const TtmcArgs<T> a) {
  extern __shared__ __align__(16) char smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
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
  int oc[TK_MAXN - 3];
  {
    int t = o;
    for (int q = 2; q < a.nother; ++q) {
      oc[q - 2] = t % a.Kf[q];
      t /= a.Kf[q];
    }
  }
  const int colbase = a.KA * j0 + a.KA * a.KB * o;
  const int64_t wbase = bw * a.limit;
  const int C = a.chunk;
  const bool sval = a.vals_override == nullptr, sperm = !sval;
  const int sb = stage_bytes<T>(C, a.nother, sval, sperm);
  const int CW = C * 32;
  char* wsm = smem + (size_t)wib * 2 * sb;

  T acc[MA * MB];
#pragma unroll
  for (int i = 0; i < MA * MB; ++i) acc[i] = T(0);

  auto flush = [&](uint32_t code) {
    T* dst = (code & TK_SPLIT_BIT) ? a.Zpart + ((int64_t)bin * 2 + ((code & TK_HEAD_BIT) ? 1 : 0)) * a.Khat
                                   : a.Z + (int64_t)(code & TK_ROW_MASK) * a.Khat;
    dst += colbase;
    if (EA && EB && (MA * MB) % VecT<T>::W == 0 && a.store_vec) {
      using V = typename VecT<T>::type;
      V* d = reinterpret_cast<V*>(dst);
#pragma unroll
      for (int v = 0; v < MA * MB / VecT<T>::W; ++v) st_stream(d + v, pack(&acc[v * VecT<T>::W]));
    } else {
#pragma unroll
      for (int jj = 0; jj < MB; ++jj)
#pragma unroll
        for (int i = 0; i < MA; ++i)
          if ((EB || jj < tb) && (EA || i < ka)) dst[i + a.KA * jj] = acc[i + MA * jj];
    }
  };

  const int nch = (wlen + C - 1) / C;
  if (nch > 0) issue_chunk(a, wsm, CW, wbase, 0, min(C, wlen), lane, sval, sperm);
  cp_commit();
  if (nch > 1) issue_chunk(a, wsm + sb, CW, wbase, C, min(C, wlen - C), lane, sval, sperm);
  cp_commit();
  uint32_t cur = len > 0 ? a.rowcode[wbase * 32 + lane] : 0u;
  // gathers element sj's rows and its outer-mode scaling into v, fa, fb
  auto gather = [&](const uint32_t* sw, int CW_, int sj, T& v, T (&fa)[Row<T, MA>::R], T (&fb)[Row<T, MB>::R]) {
    for (int q = 2; q < a.nother; ++q) v *= __ldg(a.F[q] + (int64_t)(int32_t)sw[(1 + q) * CW_ + sj] * a.ld[q] + oc[q - 2]);
    load_row<T, MA>(a.F[0] + (int64_t)(int32_t)sw[CW_ + sj] * a.ld[0], ka, fa);
    if (a.nother >= 2) {
      const int64_t rb = (int64_t)(int32_t)sw[2 * CW_ + sj] * a.ld[1] + j0;
      if (a.texB) tex_row<T, MB>(a.texB, rb, tb, fb);
      else load_row<T, MB>(a.F[1] + rb, tb, fb);
    } else {
#pragma unroll
      for (int u = 0; u < Row<T, MB>::R; ++u) fb[u] = T(u == 0);
    }
  };
  auto accumulate = [&](uint32_t code, T v, const T (&fa)[Row<T, MA>::R], const T (&fb)[Row<T, MB>::R]) {
    if (code != cur) {
      flush(cur);
#pragma unroll
      for (int i = 0; i < MA * MB; ++i) acc[i] = T(0);
      cur = code;
    }
#pragma unroll
    for (int jj = 0; jj < MB; ++jj) {
      const T t = v * fb[jj];
#pragma unroll
      for (int i = 0; i < MA; ++i) acc[i + MA * jj] = fma(fa[i], t, acc[i + MA * jj]);
    }
  };
  for (int c = 0; c < nch; ++c) {
    cp_wait_1();
    __syncwarp();
    const uint32_t* sw = (const uint32_t*)(wsm + (c & 1) * sb);
    const T* sv = (const T*)(sw + (1 + a.nother) * CW);
    const int32_t* sp = (const int32_t*)((const char*)sv + (sval ? (size_t)CW * sizeof(T) : 0));
    // this lane's steps in the chunk
    const int ns = min(C, len - c * C);
    if constexpr (sizeof(T) == 4 && EA && EB) {
      if (a.nother == 2 && a.texB && sval) {
        // NE elements per step, all their rows requested before the first is used
        constexpr int NA = Row<T, MA>::NV, NB = Row<T, MB>::NV, NE = TK_TTMC_NE;
#pragma unroll 1
        for (int j = 0; j < ns; j += NE) {
          int sjs[NE];
          bool has[NE];
#pragma unroll
          for (int e = 0; e < NE; ++e) {
            has[e] = j + e < ns;
            sjs[e] = (j + (has[e] ? e : 0)) * 32 + lane;
          }
          float4 A[NE][NA], B[NE][NB];
#pragma unroll
          for (int e = 0; e < NE; ++e) {
            const T* ra = a.F[0] + (int64_t)(int32_t)sw[CW + sjs[e]] * a.ld[0];
            const int tb = (int)(((int64_t)(int32_t)sw[2 * CW + sjs[e]] * a.ld[1] + j0) / 4);
#pragma unroll
            for (int u = 0; u < NA; ++u) A[e][u] = ldg_v4_ordered(ra + 4 * u);
#pragma unroll
            for (int u = 0; u < NB; ++u) B[e][u] = tex_v4_ordered(a.texB, tb + u);
          }
          T v[NE];
          uint32_t code[NE];
          bool same = true;
#pragma unroll
          for (int e = 0; e < NE; ++e) {
            v[e] = has[e] ? sv[sjs[e]] : T(0);
            code[e] = sw[sjs[e]];
            same = same && code[e] == cur;
          }
          if (same) {
#pragma unroll
            for (int jj = 0; jj < MB; ++jj) {
              T t[NE];
#pragma unroll
              for (int e = 0; e < NE; ++e) t[e] = v[e] * (&B[e][jj / 4].x)[jj % 4];
#pragma unroll
              for (int i = 0; i < MA; ++i) {
                T x = acc[i + MA * jj];
#pragma unroll
                for (int e = 0; e < NE; ++e) x = fma((&A[e][i / 4].x)[i % 4], t[e], x);
                acc[i + MA * jj] = x;
              }
            }
          } else {
#pragma unroll
            for (int e = 0; e < NE; ++e) {
              if (!has[e]) break;
              T fa[NA * 4], fb[NB * 4];
#pragma unroll
              for (int u = 0; u < NA; ++u) unpack(A[e][u], &fa[4 * u]);
#pragma unroll
              for (int u = 0; u < NB; ++u) unpack(B[e][u], &fb[4 * u]);
              accumulate(code[e], v[e], fa, fb);
            }
          }
        }
        goto chunk_done;
      }
    }
#pragma unroll 1
    for (int j = 0; j < ns; ++j) {
      const int sj = j * 32 + lane;
      T v = sval ? sv[sj] : a.vals_override[sp[sj]];
      T fa[Row<T, MA>::R], fb[Row<T, MB>::R];
      gather(sw, CW, sj, v, fa, fb);
      accumulate(sw[sj], v, fa, fb);
    }
  chunk_done:
    __syncwarp();
    if (c + 2 < nch) issue_chunk(a, wsm + (c & 1) * sb, CW, wbase, (c + 2) * C, min(C, wlen - (c + 2) * C), lane, sval, sperm);
    cp_commit();
  }
  cp_wait_0();
  if (len > 0) flush(cur);
}

template <typename T, int MA, int MB, bool EA, bool EB>
__global__ void __launch_bounds__(128) k_ttmc_bwd(const TtmcArgs<T> a) {
  extern __shared__ __align__(16) char smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
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
  int oc[TK_MAXN - 3];
  {
    int t = o;
    for (int q = 2; q < a.nother; ++q) {
      oc[q - 2] = t % a.Kf[q];
      t /= a.Kf[q];
    }
  }
  const int colbase = a.KA * j0 + a.KA * a.KB * o;
  const int64_t wbase = bw * a.limit;
  const int C = a.chunk;
  const bool sval = a.vals_override == nullptr;
  const int sb = stage_bytes<T>(C, a.nother, sval, true);
  const int CW = C * 32;
  char* wsm = smem + (size_t)wib * 2 * sb;

  T D[MA * MB];
  uint32_t cur = 0xFFFFFFFFu;
  const int nch = (wlen + C - 1) / C;
  if (nch > 0) issue_chunk(a, wsm, CW, wbase, 0, min(C, wlen), lane, sval, true);
  cp_commit();
  if (nch > 1) issue_chunk(a, wsm + sb, CW, wbase, C, min(C, wlen - C), lane, sval, true);
  cp_commit();
  for (int c = 0; c < nch; ++c) {
    cp_wait_1();
    __syncwarp();
    const uint32_t* sw = (const uint32_t*)(wsm + (c & 1) * sb);
    const T* sv = (const T*)(sw + (1 + a.nother) * CW);
    const int32_t* sp = (const int32_t*)((const char*)sv + (sval ? (size_t)CW * sizeof(T) : 0));
    const int ns = min(C, wlen - c * C);
#pragma unroll 1
    for (int j = 0; j < ns; ++j) {
      if (c * C + j >= len) break;
      const int sj = j * 32 + lane;
      const uint32_t code = sw[sj];
      if (code != cur) {
        const T* src = a.dZ + (int64_t)(code & TK_ROW_MASK) * a.Khat + colbase;
#pragma unroll
        for (int jj = 0; jj < MB; ++jj)
#pragma unroll
          for (int i = 0; i < MA; ++i)
            D[i + MA * jj] = ((EB || jj < tb) && (EA || i < ka)) ? __ldg(src + i + a.KA * jj) : T(0);
        cur = code;
      }
      const int32_t e = sp[sj];
      const T w = sval ? sv[sj] : a.vals_override[e];
      T fq[TK_MAXN - 3];
      T so = T(1);
      for (int q = 2; q < a.nother; ++q) {
        fq[q - 2] = __ldg(a.F[q] + (int64_t)(int32_t)sw[(1 + q) * CW + sj] * a.ld[q] + oc[q - 2]);
        so *= fq[q - 2];
      }
      const int ia = (int32_t)sw[CW + sj];
      T fa[Row<T, MA>::R];
      load_row<T, MA>(a.F[0] + (int64_t)ia * a.ld[0], ka, fa);
      T fb[Row<T, MB>::R];
      int ib = 0;
      if (a.nother >= 2) {
        ib = (int32_t)sw[2 * CW + sj];
        load_row<T, MB>(a.F[1] + (int64_t)ib * a.ld[1] + j0, tb, fb);
      } else {
#pragma unroll
        for (int u = 0; u < Row<T, MB>::R; ++u) fb[u] = T(u == 0);
      }
      T x[MA], y[MB];
#pragma unroll
      for (int i = 0; i < MA; ++i) x[i] = T(0);
#pragma unroll
      for (int jj = 0; jj < MB; ++jj) {
        T yy = T(0);
#pragma unroll
        for (int i = 0; i < MA; ++i) {
          x[i] = fma(D[i + MA * jj], fb[jj], x[i]);
          yy = fma(D[i + MA * jj], fa[i], yy);
        }
        y[jj] = yy;
      }
      T dot = T(0);
#pragma unroll
      for (int i = 0; i < MA; ++i) dot = fma(fa[i], x[i], dot);
      if (a.dval) {
        if (a.G == 1) a.dval[e] = so * dot;
        else atomicAdd(a.dval + e, so * dot);
      }
      const T ws = w * so;
      if (a.dF[0]) {
        T* d = a.dF[0] + (int64_t)ia * a.ldd[0];
#pragma unroll
        for (int i = 0; i < MA; ++i)
          if (EA || i < ka) atomicAdd(d + i, ws * x[i]);
      }
      if (a.nother >= 2 && a.dF[1]) {
        T* d = a.dF[1] + (int64_t)ib * a.ldd[1] + j0;
#pragma unroll
        for (int jj = 0; jj < MB; ++jj)
          if (EB || jj < tb) atomicAdd(d + jj, ws * y[jj]);
      }
      for (int q = 2; q < a.nother; ++q) {
        if (!a.dF[q]) continue;
        T prod = w * dot;
        for (int q2 = 2; q2 < a.nother; ++q2)
          if (q2 != q) prod *= fq[q2 - 2];
        atomicAdd(a.dF[q] + (int64_t)(int32_t)sw[(1 + q) * CW + sj] * a.ldd[q] + oc[q - 2], prod);
      }
    }
    __syncwarp();
    if (c + 2 < nch) issue_chunk(a, wsm + (c & 1) * sb, CW, wbase, (c + 2) * C, min(C, wlen - (c + 2) * C), lane, sval, true);
    cp_commit();
  }
  cp_wait_0();
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

template <typename T>
__global__ void k_copy_factor(const T* __restrict__ src, int lds, T* __restrict__ dst, int ldd, int64_t rows, int cols) {
  const int64_t total = rows * ldd;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    const int64_t r = i / ldd;
    const int cc = (int)(i - r * ldd);
    dst[i] = cc < cols ? src[r * lds + cc] : T(0);
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

template <typename T>
KernelT<T> fwd_kernel(int id);
template <>
KernelT<float> fwd_kernel<float>(int id) {
  switch (id) {
    case 0: return k_ttmc_fwd<float, 10, 10, true, true>;
    case 1: return k_ttmc_fwd<float, 8, 8, true, true>;
    case 2: return k_ttmc_fwd<float, 16, 8, true, true>;
    case 3: return k_ttmc_fwd<float, 16, 8, false, false>;
    default: return k_ttmc_fwd<float, 32, 4, false, false>;
  }
}
template <>
KernelT<double> fwd_kernel<double>(int id) {
  switch (id) {
    case 0: return k_ttmc_fwd<double, 10, 4, true, false>;
    case 1: return k_ttmc_fwd<double, 8, 4, true, true>;
    case 2: return k_ttmc_fwd<double, 16, 4, true, true>;
    case 3: return k_ttmc_fwd<double, 16, 4, false, false>;
    default: return k_ttmc_fwd<double, 32, 2, false, false>;
  }
}
template <typename T>
KernelT<T> bwd_kernel(int id);
template <>
KernelT<float> bwd_kernel<float>(int id) {
  switch (id) {
    case 0: return k_ttmc_bwd<float, 10, 10, true, true>;
    case 1: return k_ttmc_bwd<float, 8, 8, true, true>;
    case 2: return k_ttmc_bwd<float, 16, 8, true, true>;
    case 3: return k_ttmc_bwd<float, 16, 8, false, false>;
    default: return k_ttmc_bwd<float, 32, 4, false, false>;
  }
}
template <>
KernelT<double> bwd_kernel<double>(int id) {
  switch (id) {
    case 0: return k_ttmc_bwd<double, 10, 4, true, false>;
    case 1: return k_ttmc_bwd<double, 8, 4, true, true>;
    case 2: return k_ttmc_bwd<double, 16, 4, true, true>;
    case 3: return k_ttmc_bwd<double, 16, 4, false, false>;
    default: return k_ttmc_bwd<double, 32, 2, false, false>;
  }
}

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

// Staged steps per buffer: 16 for 3-mode FP32, 8 otherwise (keeps a CTA of
// 4 warps, double-buffered, within 64 KB of shared memory).
template <typename T>
int stage_chunk(int nother) {
  return (sizeof(T) == 4 && nother <= 2) ? 16 : 8;
}

template <typename K>
void set_smem_attr(K kernel, int bytes) {
  TK_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, std::max(bytes, 48 * 1024)));
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
  a.chunk = stage_chunk<T>(pl.nother);
  const int shm = 4 * 2 * stage_bytes<T>(a.chunk, pl.nother, vals_override == nullptr, vals_override != nullptr);
  set_smem_attr(fwd_kernel<T>(pl.tile_id), shm);
  tk_phase_begin(c, PH_TTM, s);
  fwd_kernel<T>(pl.tile_id)<<<blocks_for(md, pl.G), 128, shm, s>>>(a);
  TK_CUDA(cudaGetLastError());
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

template <typename T>
void backward_impl(tucker_ctx* c, int n, void* const* F, const int* ldF, const void* dZ, const void* vals_override,
                   void* const* dF, void* dval, cudaStream_t s) {
  tk_mode& md = c->mode[n];
  const Plan pl = make_plan(c, n);
  TtmcArgs<T> a = make_args<T>(c, n, pl, F, ldF, vals_override);
  a.dZ = (const T*)dZ;
  for (int q = 0; q < pl.nother; ++q) {
    a.dF[q] = dF ? (T*)dF[pl.others[q]] : nullptr;
    a.ldd[q] = c->K[pl.others[q]];
  }
  a.dval = (T*)dval;
  tk_phase_begin(c, PH_BWD, s);
  if (dval && pl.G > 1) TK_CUDA(cudaMemsetAsync(dval, 0, (size_t)c->nnz * sizeof(T), s));
  a.chunk = stage_chunk<T>(pl.nother);
  const int shm = 4 * 2 * stage_bytes<T>(a.chunk, pl.nother, vals_override == nullptr, true);
  set_smem_attr(bwd_kernel<T>(pl.tile_id), shm);
  bwd_kernel<T>(pl.tile_id)<<<blocks_for(md, pl.G), 128, shm, s>>>(a);
  TK_CUDA(cudaGetLastError());
  tk_phase_end(c, s);
  tk_launched(c, PH_BWD);
}

}  // namespace

int tk_ttmc_groups(const tucker_ctx* c, int n) { return make_plan(c, n).G; }

int tk_ttmc_threads_per_sm(const tucker_ctx* c, int n) {
  const Plan pl = make_plan(c, n);
  int nb = 0;
  if (c->prec == TUCKER_FP32) {
    const int shm = 4 * 2 * stage_bytes<float>(stage_chunk<float>(pl.nother), pl.nother, true, false);
    set_smem_attr(fwd_kernel<float>(pl.tile_id), shm);
    TK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fwd_kernel<float>(pl.tile_id), 128, shm));
  } else {
    const int shm = 4 * 2 * stage_bytes<double>(stage_chunk<double>(pl.nother), pl.nother, true, false);
    set_smem_attr(fwd_kernel<double>(pl.tile_id), shm);
    TK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fwd_kernel<double>(pl.tile_id), 128, shm));
  }
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
                    cudaStream_t s) {
  const int64_t total = rows * ldd;
  const unsigned grid = (unsigned)std::min<int64_t>(tk_ceil_div(total > 0 ? total : 1, 256), 8192);
  if (c->prec == TUCKER_FP32) k_copy_factor<float><<<grid, 256, 0, s>>>((const float*)src, lds, (float*)dst, ldd, rows, cols);
  else k_copy_factor<double><<<grid, 256, 0, s>>>((const double*)src, lds, (double*)dst, ldd, rows, cols);
  TK_CUDA(cudaGetLastError());
  tk_launched(c, PH_OTHER);
}
