// C ABI of libtucker (declared in include/tucker.h): argument checks,
// workspace, and the per-call orchestration of the device passes.
#include <algorithm>
#include <cstring>
#include <exception>

#include "tk_common.cuh"

namespace {

struct tk_exception {
  tucker_status code;
  std::string msg;
};

thread_local std::string g_init_error;

constexpr int kEvPairs = 1024;

int pad_ld(int K, int prec) { return prec == TUCKER_FP32 ? (K + 3) / 4 * 4 : (K + 1) / 2 * 2; }

void accumulate_events(tucker_ctx* c) {
  if (!c->timing || c->ev_used == 0) return;
  TK_CUDA(cudaEventSynchronize(c->ev[2 * (c->ev_used - 1) + 1]));
  for (int i = 0; i < c->ev_used; ++i) {
    float ms = 0.f;
    TK_CUDA(cudaEventElapsedTime(&ms, c->ev[2 * i], c->ev[2 * i + 1]));
    c->ms[c->ev_phase[i]] += ms;
  }
  c->ev_used = 0;
}

void check_device_error(tucker_ctx* c, cudaStream_t s) {
  int h = 0;
  TK_CUDA(cudaMemcpyAsync(&h, c->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  TK_CUDA(cudaStreamSynchronize(s));
  if (h) {
    TK_CUDA(cudaMemsetAsync(c->err, 0, sizeof(int), s));
    TK_CUDA(cudaStreamSynchronize(s));
    // a timed-out wait leaves partial results behind, so it is reported first
    if (h & TK_DEV_ERR_TIMEOUT) tk_throw(TUCKER_ERR_TIMEOUT, "a bounded device wait ran out");
    if (h & TK_DEV_ERR_NUMERIC) tk_throw(TUCKER_ERR_NUMERIC, "numeric breakdown (rank-deficient factor update)");
    if (h & TK_DEV_ERR_NONFINITE) tk_throw(TUCKER_ERR_ARG, "non-finite tensor value");
    if (h & TK_DEV_ERR_INDEX) tk_throw(TUCKER_ERR_INDEX, "coordinate out of range");
    tk_throw(TUCKER_ERR_STATE, "device error word " + std::to_string(h));
  }
}

void release(tucker_ctx* c) {
  if (!c) return;
  cudaDeviceSynchronize();
  for (int n = 0; n < TK_MAXN; ++n) {
    if (c->aux[n]) cudaStreamDestroy(c->aux[n]);
    if (c->ev_ttm[n]) cudaEventDestroy(c->ev_ttm[n]);
    if (c->ev_fu[n]) cudaEventDestroy(c->ev_fu[n]);
  }
  for (int m = 0; m < TK_MAXN; ++m) {
    if (c->texFa[m]) cudaDestroyTextureObject(c->texFa[m]);
    if (c->texFb[m]) cudaDestroyTextureObject(c->texFb[m]);
  }
  for (auto& a : c->allocs) tk_dev_free(c, a.first, a.second);
  c->allocs.clear();
  if (c->timing)
    for (int i = 0; i < 2 * kEvPairs; ++i) cudaEventDestroy(c->ev[i]);
  delete c;
}

// Linear textures over the padded factor buffers (16-byte texels: float4 or
// two doubles as int4); a factor wider than the device's linear texture limit
// keeps texture 0 and is gathered with plain loads.
void make_factor_tex(tucker_ctx* c, int m) {
  int dev = 0, maxw = 0;
  TK_CUDA(cudaGetDevice(&dev));
  TK_CUDA(cudaDeviceGetAttribute(&maxw, cudaDevAttrMaxTexture1DLinearWidth, dev));
  const size_t bytes = (size_t)c->L[m] * c->ldF[m] * c->esz;
  if (bytes / 16 > (size_t)maxw || bytes / 16 > (size_t)INT32_MAX) return;
  for (int w = 0; w < 2; ++w) {
    cudaResourceDesc rd{};
    rd.resType = cudaResourceTypeLinear;
    rd.res.linear.devPtr = w ? c->Fb[m] : c->Fa[m];
    rd.res.linear.desc = c->prec == TUCKER_FP32 ? cudaCreateChannelDesc<float4>() : cudaCreateChannelDesc<int4>();
    rd.res.linear.sizeInBytes = bytes;
    cudaTextureDesc td{};
    td.readMode = cudaReadModeElementType;
    TK_CUDA(cudaCreateTextureObject(w ? &c->texFb[m] : &c->texFa[m], &rd, &td, nullptr));
  }
}

void copy_in_factors(tucker_ctx* c, const void* const* d_F, int skip, cudaStream_t s) {
  for (int m = 0; m < c->N; ++m) {
    if (m == skip) continue;
    if (!d_F || !d_F[m]) tk_throw(TUCKER_ERR_ARG, "factor pointer for mode " + std::to_string(m) + " is NULL");
    tk_copy_factor(c, d_F[m], c->K[m], c->Fa[m], c->ldF[m], c->L[m], c->K[m], c->relabel[m], nullptr, s);
  }
}

template <typename F>
tucker_status guarded(tucker_ctx* c, F&& body) {
  try {
    body();
    return TUCKER_OK;
  } catch (const tk_exception& ex) {
    if (c) c->last_error = ex.msg;
    else g_init_error = ex.msg;
    return ex.code;
  } catch (const std::exception& ex) {
    if (c) c->last_error = ex.what();
    else g_init_error = ex.what();
    return TUCKER_ERR_STATE;
  }
}

void check_ctx(tucker_t t) {
  if (!t) throw tk_exception{TUCKER_ERR_ARG, "NULL context"};
}
void check_mode(tucker_t t, int mode) {
  if (mode < 0 || mode >= t->N) tk_throw(TUCKER_ERR_ARG, "mode out of range");
}

}  // namespace

// ------------------------------------------------------------ shared helpers
// Runs body(arg) with the C-ABI error handling (status code + last-error text).
tucker_status tk_guarded_call(tucker_ctx* c, void (*body)(void*), void* arg) {
  return guarded(c, [&] { body(arg); });
}

void tk_throw(tucker_status code, const std::string& msg) { throw tk_exception{code, msg}; }

void tk_check_cuda(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw tk_exception{e == cudaErrorMemoryAllocation ? TUCKER_ERR_OOM : TUCKER_ERR_CUDA,
                       std::string(what) + ": " + cudaGetErrorString(e)};
  }
}

void* tk_dev_alloc(tucker_ctx* c, size_t bytes) {
  if (bytes == 0) bytes = 16;
  void* p = nullptr;
  if (c->alloc_fn) {
    p = c->alloc_fn(bytes, (void*)c->alloc_stream, c->alloc_user);
    if (!p) tk_throw(TUCKER_ERR_OOM, "the caller's allocator returned NULL for " + std::to_string(bytes) + " bytes");
    if ((uintptr_t)p % 256 != 0) {
      c->free_fn(p, bytes, (void*)c->alloc_stream, c->alloc_user);
      tk_throw(TUCKER_ERR_ARG, "the caller's allocator returned memory that is not 256-byte aligned");
    }
    return p;
  }
  const cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    tk_throw(TUCKER_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
  }
  return p;
}

void tk_dev_free(tucker_ctx* c, void* p, size_t bytes) {
  if (!p) return;
  if (bytes == 0) bytes = 16;
  if (c->free_fn) c->free_fn(p, bytes, (void*)c->alloc_stream, c->alloc_user);
  else cudaFree(p);
}

void* tk_alloc(tucker_ctx* c, size_t bytes) {
  void* p = tk_dev_alloc(c, bytes);
  c->allocs.emplace_back(p, bytes == 0 ? 16 : bytes);
  c->bytes += (int64_t)bytes;
  return p;
}

void tk_phase_begin(tucker_ctx* c, int phase, cudaStream_t s) {
  if (!c->timing) return;
  if (c->ev_used >= kEvPairs) accumulate_events(c);
  c->ev_phase[c->ev_used] = phase;
  TK_CUDA(cudaEventRecord(c->ev[2 * c->ev_used], s));
}

void tk_phase_end(tucker_ctx* c, cudaStream_t s) {
  if (!c->timing) return;
  TK_CUDA(cudaEventRecord(c->ev[2 * c->ev_used + 1], s));
  ++c->ev_used;
}

void tk_launched(tucker_ctx* c, int phase, int n) { c->launches[phase] += n; }

int tk_sm_count() {
  int dev = 0, sms = 0;
  TK_CUDA(cudaGetDevice(&dev));
  TK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  return sms;
}

// ------------------------------------------------------------ C ABI
extern "C" {

void tucker_default_opts(tucker_opts* opts) {
  if (!opts) return;
  std::memset(opts, 0, sizeof(*opts));
  opts->prec = TUCKER_FP32;
}

const char* tucker_last_error(tucker_t t) { return t ? t->last_error.c_str() : g_init_error.c_str(); }

void tucker_destroy(tucker_t t) { release(t); }

tucker_status tucker_init(tucker_t* out, int N, const int64_t* L, const int32_t* K, int64_t nnz,
                          const int32_t* const* d_idx, const void* d_val, const tucker_opts* opts, void* stream) {
  tucker_ctx* c = nullptr;
  const tucker_status st = guarded(nullptr, [&] {
    if (!out) tk_throw(TUCKER_ERR_ARG, "out is NULL");
    *out = nullptr;
    tucker_opts o;
    tucker_default_opts(&o);
    if (opts) o = *opts;
    if (N < 2 || N > TK_MAXN) tk_throw(TUCKER_ERR_ARG, "N must be in [2, 6]");
    if (!L || !K || !d_idx || !d_val) tk_throw(TUCKER_ERR_ARG, "NULL array argument");
    if (nnz < 1 || nnz >= ((int64_t)1 << 31) - 1) tk_throw(TUCKER_ERR_ARG, "nnz must be in [1, 2^31 - 1)");
    if (o.prec != TUCKER_FP32 && o.prec != TUCKER_FP64 && o.prec != TUCKER_BF16X3)
      tk_throw(TUCKER_ERR_ARG, "unknown precision");
    if (o.P_bins < 0) tk_throw(TUCKER_ERR_ARG, "P_bins must be >= 0");
    if (o.wait_cap < -1) tk_throw(TUCKER_ERR_ARG, "wait_cap must be >= -1");
    if (o.ttm_path < 0 || o.ttm_path > 2) tk_throw(TUCKER_ERR_ARG, "ttm_path must be 0, 1 or 2");
    for (int i = 0; i < 3; ++i)
      if (o.reserved[i]) tk_throw(TUCKER_ERR_ARG, "reserved option fields must be zero");
    if (o.svd != 0 && o.svd != 1) tk_throw(TUCKER_ERR_ARG, "svd must be 0 or 1");
    if ((o.alloc == nullptr) != (o.free == nullptr)) tk_throw(TUCKER_ERR_ARG, "alloc and free must be set together");
    for (int m = 0; m < N; ++m) {
      if (L[m] < 1 || L[m] >= ((int64_t)1 << 31) - 1) tk_throw(TUCKER_ERR_ARG, "mode length out of range");
      if (K[m] < 1 || K[m] > TK_MAXK || (int64_t)K[m] > L[m])
        tk_throw(TUCKER_ERR_ARG, "core length must satisfy 1 <= K_n <= min(L_n, 32)");
      if (!d_idx[m]) tk_throw(TUCKER_ERR_ARG, "NULL index array");
    }
    c = new tucker_ctx();
    c->N = N;
    c->nnz = nnz;
    c->prec = o.prec == TUCKER_FP64 ? TUCKER_FP64 : TUCKER_FP32;
    c->gram_bf16 = o.prec == TUCKER_BF16X3;
    c->esz = c->prec == TUCKER_FP32 ? 4 : 8;
    c->gauss_seidel = o.gauss_seidel != 0;
    c->ttm_path = o.ttm_path;
    c->svd_lanczos = o.svd;
    c->timing = o.timing != 0;
    c->wait_cap = o.wait_cap;
    c->sm_count = tk_sm_count();
    c->alloc_fn = o.alloc;
    c->free_fn = o.free;
    c->alloc_user = o.alloc_user;
    c->alloc_stream = (cudaStream_t)stream;
    for (int m = 0; m < N; ++m) {
      c->L[m] = L[m];
      c->K[m] = K[m];
      c->Kmax = std::max(c->Kmax, (int)K[m]);
      c->Gsize *= K[m];
    }
    for (int n = 0; n < N; ++n) {
      int64_t kh = 1;
      for (int m = 0; m < N; ++m)
        if (m != n) kh *= K[m];
      if (kh > TK_MAXKHAT) tk_throw(TUCKER_ERR_ARG, "prod_{m != n} K_m must be <= 4096");
      c->mode[n].Khat = (int)kh;
      c->maxKhat = std::max(c->maxKhat, (int)kh);
    }
    if (c->timing)
      for (int i = 0; i < 2 * kEvPairs; ++i) TK_CUDA(cudaEventCreate(&c->ev[i]));
    cudaStream_t s = (cudaStream_t)stream;
    c->err = (int*)tk_alloc(c, 64);
    TK_CUDA(cudaMemsetAsync(c->err, 0, 64, s));
    c->normT2 = tk_norm2(c, d_val, nnz, s);
    check_device_error(c, s);
    if (!(c->normT2 > 0.0)) tk_throw(TUCKER_ERR_ARG, "the tensor has zero norm");
    tk_relabel_modes(c, d_idx, s);

    for (int n = 0; n < N; ++n) {
      const int G = tk_ttmc_groups(c, n);
      c->mode[n].G = G;
      int P = o.P_bins;
      if (P == 0) {
        const int64_t tpsm = tk_ttmc_threads_per_sm(c, n);
        // one CTA slot short of a full wave, so that a one-CTA kernel of a
        // concurrent factor update finds room beside the TTM-chain
        int64_t p = ((int64_t)c->sm_count * tpsm - 128) / G;
        p = std::min<int64_t>(p, tk_ceil_div(tk_ceil_div(nnz, 16), 32) * 32);
        p = std::max<int64_t>(32, p / 32 * 32);
        P = (int)p;
      }
      tk_partition_mode(c, n, d_idx, d_val, P, s);
      if (c->ttm_path == 0 && tk_ttmc_tc_eligible(c, n)) tk_ttmc_tc_build(c, n, s);
      const tk_mode& md = c->mode[n];
      if (K[n] > md.R || K[n] > md.Khat)
        tk_throw(TUCKER_ERR_ARG, "K_" + std::to_string(n) + " exceeds min(non-empty slices, prod of the other K)");
      c->maxR = std::max(c->maxR, md.R);
    }

    // workspace (sized for the largest mode)
    size_t zc = 0, zp = 0, zch = 0, wp = 0, gp = 0;
    int tiles_cap = 1;
    for (int n = 0; n < N; ++n) {
      const tk_mode& md = c->mode[n];
      zc = std::max(zc, (size_t)md.R * md.Khat);
      zp = std::max(zp, (size_t)2 * md.Pa * md.Khat);
      zch = std::max(zch, (size_t)md.nchunks * md.Khat);
      const int TM = (c->esz == 4 && md.Khat > 64) ? 128 : 64;
      const int tpd = (int)tk_ceil_div(md.Khat, TM);
      const int ntiles = tpd * (tpd + 1) / 2;
      tiles_cap = std::max(tiles_cap, ntiles);
      wp = std::max(wp, (size_t)(2 * c->sm_count + ntiles) * TM * TM);
      const int cb = (int)tk_ceil_div(md.Khat, 128);
      const int64_t ns = std::max<int64_t>(1, std::min<int64_t>(tk_ceil_div(md.R, 64), tk_ceil_div(4 * c->sm_count, cb)));
      gp = std::max(gp, (size_t)ns * c->K[n] * md.Khat);
    }
    const size_t esz = c->esz;
    for (int n = 0; n < N; ++n) {
      c->Zm[n] = tk_alloc(c, (size_t)std::max(c->mode[n].R, 1) * c->mode[n].Khat * esz);
      tk_alloc_fuws(c, n);
      if (c->svd_lanczos) tk_lanczos_alloc(c, n);
      TK_CUDA(cudaStreamCreateWithFlags(&c->aux[n], cudaStreamNonBlocking));
      TK_CUDA(cudaEventCreateWithFlags(&c->ev_ttm[n], cudaEventDisableTiming));
      TK_CUDA(cudaEventCreateWithFlags(&c->ev_fu[n], cudaEventDisableTiming));
    }
    {
      const tk_mode& mc = c->mode[tk_core_mode(c)];
      c->Zcore = tk_alloc(c, (size_t)std::max(mc.R, 1) * mc.Khat * esz);
    }
    (void)zc;
    (void)wp;
    (void)tiles_cap;
    c->Zpart = tk_alloc(c, zp * esz);
    c->Zchunk = (double*)tk_alloc(c, std::max<size_t>(zch, 1) * 8);
    c->Gpart = (double*)tk_alloc(c, gp * 8);
    c->Gd = (double*)tk_alloc(c, (size_t)c->Gsize * 8);
    c->fit_d = (double*)tk_alloc(c, 4 * 8);
    for (int m = 0; m < N; ++m) {
      c->ldF[m] = pad_ld(K[m], c->prec);
      c->Fa[m] = tk_alloc(c, (size_t)L[m] * c->ldF[m] * esz);
      c->Fb[m] = tk_alloc(c, (size_t)L[m] * c->ldF[m] * esz);
      TK_CUDA(cudaMemsetAsync(c->Fa[m], 0, (size_t)L[m] * c->ldF[m] * esz, s));
      TK_CUDA(cudaMemsetAsync(c->Fb[m], 0, (size_t)L[m] * c->ldF[m] * esz, s));
      make_factor_tex(c, m);
    }
    TK_CUDA(cudaStreamSynchronize(s));
    *out = c;
  });
  if (st != TUCKER_OK && c) release(c);
  return st;
}

tucker_status tucker_stats(tucker_t t, int mode, int64_t* E_max, int64_t* R_sum, int64_t* R_max, int64_t* R_n,
                           int64_t* P) {
  return guarded(t, [&] {
    check_ctx(t);
    check_mode(t, mode);
    const tk_mode& md = t->mode[mode];
    if (E_max) *E_max = md.E_max;
    if (R_sum) *R_sum = md.R_sum;
    if (R_max) *R_max = md.R_max;
    if (R_n) *R_n = md.R;
    if (P) *P = md.P;
  });
}

tucker_status tucker_scheme_metrics(tucker_t t, int mode, int scheme, int P, const int32_t* const* d_pos,
                                    int64_t* E_max, int64_t* R_sum, int64_t* R_max, int64_t* d_E, int64_t* d_R,
                                    void* stream) {
  return guarded(t, [&] {
    check_ctx(t);
    check_mode(t, mode);
    int64_t o[3] = {0, 0, 0};
    tk_scheme_metrics(t, mode, scheme, P, d_pos, o, d_E, d_R, (cudaStream_t)stream);
    check_device_error(t, (cudaStream_t)stream);
    if (E_max) *E_max = o[0];
    if (R_sum) *R_sum = o[1];
    if (R_max) *R_max = o[2];
  });
}

tucker_status tucker_ttm_form(tucker_t t, int mode, int32_t* tensor_cores, int64_t* blocks) {
  return guarded(t, [&] {
    check_ctx(t);
    check_mode(t, mode);
    const tk_mode& md = t->mode[mode];
    if (tensor_cores) *tensor_cores = md.tc ? 1 : 0;
    if (blocks) *blocks = md.tc ? md.tc_nblk : 0;
  });
}

tucker_status tucker_partition(tucker_t t, int mode, int64_t* d_bin_ptr, int32_t* d_perm, void* stream) {
  return guarded(t, [&] {
    check_ctx(t);
    check_mode(t, mode);
    if (!d_bin_ptr || !d_perm) tk_throw(TUCKER_ERR_ARG, "NULL output");
    tk_partition_export(t, mode, d_bin_ptr, d_perm, (cudaStream_t)stream);
  });
}

tucker_status ttm_chain(tucker_t t, int mode, const void* const* d_F, const void* d_vals, void* d_Z, int32_t* d_row_id,
                        void* stream) {
  return guarded(t, [&] {
    check_ctx(t);
    check_mode(t, mode);
    if (!d_Z) tk_throw(TUCKER_ERR_ARG, "d_Z is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    copy_in_factors(t, d_F, mode, s);
    tk_ttmc_forward(t, mode, t->Fa, t->ldF, d_vals, d_Z, s);
    if (d_row_id)
      TK_CUDA(cudaMemcpyAsync(d_row_id, t->mode[mode].row_id, (size_t)t->mode[mode].R * 4, cudaMemcpyDeviceToDevice, s));
  });
}

tucker_status factor_update(tucker_t t, int mode, const void* d_Z, void* d_F_out, double* d_sigma, void* stream) {
  return guarded(t, [&] {
    check_ctx(t);
    check_mode(t, mode);
    if (!d_Z || !d_F_out) tk_throw(TUCKER_ERR_ARG, "NULL buffer");
    tk_factor_update(t, mode, d_Z, d_F_out, t->K[mode], t->mode[mode].row_id, d_sigma, (cudaStream_t)stream);
  });
}

tucker_status core(tucker_t t, const void* const* d_F, void* d_G, void* stream) {
  return guarded(t, [&] {
    check_ctx(t);
    if (!d_G) tk_throw(TUCKER_ERR_ARG, "d_G is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    copy_in_factors(t, d_F, -1, s);
    tk_core(t, t->Fa, t->ldF, d_G, s);
  });
}

tucker_status hooi_iter(tucker_t t, void* const* d_F, void* d_G, double* h_fit, void* stream) {
  return guarded(t, [&] {
    check_ctx(t);
    cudaStream_t s = (cudaStream_t)stream;
    copy_in_factors(t, (const void* const*)d_F, -1, s);
    if (t->gauss_seidel) {
      // each mode sees the factors refined so far: strictly sequential
      for (int n = 0; n < t->N; ++n) {
        void* src[TK_MAXN];
        for (int m = 0; m < t->N; ++m) src[m] = m < n ? t->Fb[m] : t->Fa[m];
        tk_ttmc_forward(t, n, src, t->ldF, nullptr, t->Zm[n], s);
        tk_factor_update(t, n, t->Zm[n], t->Fb[n], t->ldF[n], t->mode[n].frow, nullptr, s);
      }
    } else {
      // Fig. 1 as printed: every TTM-chain reads the input factors, so the
      // factor update of mode n (side stream n) overlaps the TTM-chains of the
      // later modes on the caller's stream.  The mode whose TTM-chain forms the
      // core goes last: its factor update overlaps that TTM-chain, which does
      // not read it.
      const int nc = tk_core_mode(t);
      for (int i = 0; i < t->N; ++i) {
        const int n = i < t->N - 1 ? (i < nc ? i : i + 1) : nc;
        tk_ttmc_forward(t, n, t->Fa, t->ldF, nullptr, t->Zm[n], s);
        TK_CUDA(cudaEventRecord(t->ev_ttm[n], s));
        TK_CUDA(cudaStreamWaitEvent(t->aux[n], t->ev_ttm[n], 0));
        tk_factor_update(t, n, t->Zm[n], t->Fb[n], t->ldF[n], t->mode[n].frow, nullptr, t->aux[n]);
        TK_CUDA(cudaEventRecord(t->ev_fu[n], t->aux[n]));
      }
      for (int n = 0; n < t->N; ++n)
        if (n != nc) TK_CUDA(cudaStreamWaitEvent(s, t->ev_fu[n], 0));
      tk_core(t, t->Fb, t->ldF, d_G, s, t->ev_fu[nc]);
    }
    if (t->gauss_seidel) tk_core(t, t->Fb, t->ldF, d_G, s);
    for (int m = 0; m < t->N; ++m)
      tk_copy_factor(t, t->Fb[m], t->ldF[m], d_F[m], t->K[m], t->L[m], t->K[m], nullptr, t->relabel[m], s);
    if (h_fit) {
      TK_CUDA(cudaMemcpyAsync(h_fit, t->fit_d + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
      check_device_error(t, s);
    }
  });
}

tucker_status ttm_chain_backward(tucker_t t, int mode, const void* const* d_F, const void* d_dZ, const void* d_vals,
                                 void* const* d_dF, void* d_dval, void* stream) {
  return guarded(t, [&] {
    check_ctx(t);
    check_mode(t, mode);
    if (!d_dZ) tk_throw(TUCKER_ERR_ARG, "d_dZ is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    copy_in_factors(t, d_F, mode, s);
    tk_ttmc_backward(t, mode, t->Fa, t->ldF, d_dZ, d_vals, d_dF, d_dval, s);
  });
}

tucker_status tucker_timings(tucker_t t, double* ms, int64_t* launches, int reset, void* stream) {
  return guarded(t, [&] {
    check_ctx(t);
    TK_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    accumulate_events(t);
    for (int i = 0; i < PH_COUNT; ++i) {
      if (ms) ms[i] = t->ms[i];
      if (launches) launches[i] = t->launches[i];
    }
    if (reset) {
      for (int i = 0; i < PH_COUNT; ++i) {
        t->ms[i] = 0.0;
        t->launches[i] = 0;
      }
    }
  });
}

tucker_status tucker_memory(tucker_t t, int64_t* bytes) {
  return guarded(t, [&] {
    check_ctx(t);
    if (bytes) *bytes = t->bytes;
  });
}

}  // extern "C"

cudaTextureObject_t tk_factor_tex(const tucker_ctx* c, const void* F) {
  for (int m = 0; m < c->N; ++m) {
    if (F == c->Fa[m]) return c->texFa[m];
    if (F == c->Fb[m]) return c->texFb[m];
  }
  return 0;
}
