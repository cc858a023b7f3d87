// Internal declarations shared by the libtucker translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/tucker.h"

#define TK_MAXN 6     // modes
#define TK_MAXK 32    // core length per mode
#define TK_MAXKHAT 4096

// Row code stored per element of a mode-n copy: the compact row of its slice,
// plus two flags for slices Lite splits over bins (Section 6.2: head / tail).
#define TK_ROW_MASK 0x3FFFFFFFu
#define TK_SPLIT_BIT 0x80000000u
#define TK_HEAD_BIT 0x40000000u

// Device error word bits.
#define TK_DEV_ERR_INDEX 1
#define TK_DEV_ERR_NUMERIC 2
#define TK_DEV_ERR_NONFINITE 4
#define TK_DEV_ERR_LIMIT 8
#define TK_DEV_ERR_TIMEOUT 16

enum tk_phase { PH_TTM = 0, PH_FIXUP, PH_GRAM, PH_EIG, PH_BACKPROJ, PH_CORE, PH_BWD, PH_OTHER, PH_COUNT };

struct tk_status_error {
  tucker_status code;
  std::string msg;
};

// One mode's Lite partition and permuted copy, laid out "warp-interleaved":
// bin p's k-th element lives at ((p / 32) * limit + k) * 32 + p % 32, so the
// 32 bins of a warp read one contiguous 128-byte line per step.
struct tk_mode {
  int n = 0;
  int P = 0;            // Lite bins
  int Pa = 0;           // bins allocated: P rounded up to a multiple of 32 (extra bins empty)
  int limit = 0;        // ceil(nnz / P)
  int64_t cap = 0;      // Pa * limit slots per array
  int R = 0;            // non-empty slices (compact rows)
  int t_hat = 0;        // first stage-2 slice in sorted order
  int nsplit = 0;       // stage-2 (split) slices
  int Khat = 0;
  int G = 1;            // column groups of the TTM-chain tile
  int64_t E_max = 0, R_sum = 0, R_max = 0;
  // permuted copy
  uint32_t* rowcode = nullptr;
  int32_t* oidx[TK_MAXN - 1] = {};
  void* val = nullptr;
  int32_t* perm = nullptr;
  int32_t* bin_len = nullptr;
  int32_t* row_id = nullptr;    // R slice ids
  int32_t* frow = nullptr;      // R internal factor rows: relabel[n][row_id[r]]
  // split-slice fix-up tables
  int32_t* split_row = nullptr;   // nsplit compact rows
  int32_t* split_bhead = nullptr; // nsplit
  int32_t* gap2 = nullptr;        // P stage-2 gap per bin
  int nchunks = 0;
  int32_t* chunk_split = nullptr;  // nchunks
  int32_t* chunk_b0 = nullptr;     // nchunks (inclusive)
  int32_t* chunk_b1 = nullptr;     // nchunks (exclusive)
  int32_t* split_chunk0 = nullptr; // nsplit + 1
  // tensor-core TTM-chain copy (4-mode FP32 contexts with a large Khat, tk_ttmc_tc.cu):
  // bins contiguous, each segment padded to 8-element blocks
  bool tc = false;
  int tc_Mu = 0, tc_Nu = 0;        // A rows K_a K_b, B rows K_c
  int64_t tc_nblk = 0;
  int64_t* tc_blk_ptr = nullptr;   // Pa + 1: first block of each bin
  uint32_t* tc_code = nullptr;     // nblk: compact row, or 2^31 | (2 bin + head) for a split piece
  uint8_t* tc_flag = nullptr;      // nblk: 1 = first block of its segment, 2 = last
  int32_t* tc_oidx[3] = {};        // 8 nblk each
  float* tc_val = nullptr;         // 8 nblk (0 on padding)
  int32_t* tc_perm = nullptr;      // 8 nblk (-1 on padding)
};

struct tk_buf {
  void* p = nullptr;
  size_t bytes = 0;
};

// Scratch of the Lanczos bidiagonalisation route of one mode (tk_lanczos.cu)
struct tk_lzws {
  double* U = nullptr;       // R x m, column-major: the left Lanczos vectors
  double* p = nullptr;       // R
  double* V = nullptr;       // Khat x (m + 1), column-major: the right Lanczos vectors
  double* part = nullptr;    // row-block partial sums (blocks x 64)
  double* part_c = nullptr;  // row-block partials of u^T Z (blocks x Khat)
  double* cf = nullptr;      // Gram-Schmidt coefficients
  double* alpha = nullptr;   // diagonal of B
  double* beta = nullptr;    // superdiagonal of B
};

// Scratch of one factor update (Gram, eigensolve, back-projection, CholeskyQR2).
struct tk_fuws {
  void* Wpart = nullptr;    // Gram split partials
  size_t Wpart_elems = 0;
  double* W = nullptr;      // Khat x Khat
  int2* gram_tiles = nullptr;
  int gram_tiles_cap = 0;
  double* eigX = nullptr;   // 2 x Khat x K
  double* eigAB = nullptr;  // 2 x Khat
  void* eigTri = nullptr;   // K x 6 x Khat (T)
  void* Vs = nullptr;       // Khat x K (T)
  double* V = nullptr;      // Khat x K
  double* sigma = nullptr;  // TK_MAXK
  void* eigA = nullptr;     // Khat x Khat (T)
  void* eigV = nullptr;     // Khat x Khat (T)
  void* U = nullptr;        // R x K (T)
  double* Cpart = nullptr;  // 4 * SMs x TK_MAXK^2
  double* Rinv = nullptr;   // 3 x TK_MAXK^2
  double* colbest = nullptr;// 2 * SMs x TK_MAXK x 3
  tk_lzws lz;               // Lanczos route only
};

struct tucker_ctx {
  int N = 0;
  int64_t L[TK_MAXN] = {};
  int32_t K[TK_MAXN] = {};
  int64_t nnz = 0;
  int prec = TUCKER_FP32;   // data precision: TUCKER_FP32 or TUCKER_FP64
  bool gram_bf16 = false;   // TUCKER_BF16X3: the Gram in split BF16
  size_t esz = 4;
  int gauss_seidel = 0;
  int ttm_path = 0;         // 0: tensor-core TTM-chain where eligible, 1: CUDA cores only,
                            // 2: CUDA cores, fiber-factored where it applies
  int svd_lanczos = 0;      // factor update: 0 exact leading subspace (Gram), 1 Lanczos bidiagonalisation
  int timing = 0;
  int sm_count = 0;
  double normT2 = 0.0;
  tk_mode mode[TK_MAXN];
  // library-owned device memory (everything allocated at init, plus the
  // adjoint's workspace on its first use), from the caller's callbacks or cudaMalloc
  std::vector<std::pair<void*, size_t>> allocs;
  int64_t bytes = 0;
  tucker_alloc_fn alloc_fn = nullptr;
  tucker_free_fn free_fn = nullptr;
  void* alloc_user = nullptr;
  cudaStream_t alloc_stream = nullptr;
  // Row labels.  Every mode's slices are relabelled by popularity: relabel[m][l]
  // = rank of slice l when the slices of mode m are listed by decreasing
  // cardinality (ties by lower id, empty slices last); unlabel[m] is the
  // inverse.  The permuted copies store relabelled coordinates and the factor
  // buffers Fa/Fb hold row relabel[m][l] = row l of the caller's factor, so
  // the most gathered rows sit together at the start of each buffer.
  int32_t* relabel[TK_MAXN] = {};
  int32_t* unlabel[TK_MAXN] = {};
  int fiber[TK_MAXN] = {};  // f(n): the other mode with the smallest length (lowest index on a tie)
  // factor buffers, padded leading dimension ldF[m]
  int ldF[TK_MAXN] = {};
  void* Fa[TK_MAXN] = {};   // current factors
  void* Fb[TK_MAXN] = {};   // new factors
  // linear textures over Fa / Fb (one texel = 16 bytes; 0 where the factor
  // exceeds the device's linear texture width)
  cudaTextureObject_t texFa[TK_MAXN] = {};
  cudaTextureObject_t texFb[TK_MAXN] = {};
  // workspace
  void* Z = nullptr;        // max_n R_n * Khat_n
  void* Zpart = nullptr;    // max_n 2 * P_n * Khat_n
  double* Zchunk = nullptr; // max_n nchunks * Khat_n
  tk_fuws fu[TK_MAXN];      // factor-update workspace, one per mode (modes overlap on side streams)
  void* Zm[TK_MAXN] = {};   // per-mode penultimate matrices (R_n x Khat_n)
  int wait_cap = 0;         // polls per device wait (0: time bound only, -1: abandon at once)
  void* Zcore = nullptr;    // the core's penultimate matrix (mode tk_core_mode), apart from
                            // Zm so that it can be formed while that mode's update reads Zm
  cudaStream_t aux[TK_MAXN] = {};
  cudaEvent_t ev_ttm[TK_MAXN] = {};
  cudaEvent_t ev_fu[TK_MAXN] = {};
  // adjoint workspace (allocated by the first ttm_chain_backward call)
  bool bwd_ready = false;
  int32_t* bwd_pos[TK_MAXN] = {};  // nnz: slot of element e in mode m's copy
  void* bwd_X = nullptr;           // per-slot contributions to dF of the targets of one element pass
                                   // (slot order of the TTM-chain mode's copy)
  void* bwd_dv = nullptr;          // max_n cap_n: dval in slot order
  void* bwd_Zc = nullptr;          // max_m R_m * K_m: compact dF_m
  void* bwd_Zp = nullptr;          // max_m 2 * Pa_m * K_m: split-piece partials
  double* bwd_Zch = nullptr;       // max_m nchunks_m * K_m: fix-up chunk sums
  double* Gpart = nullptr;  // core partials
  double* Gd = nullptr;     // core (double) prod K
  double* fit_d = nullptr;  // [0] = ||G||^2, [1] = fit
  int* err = nullptr;       // device error word
  int maxR = 0, maxKhat = 0, Kmax = 0;
  int64_t Gsize = 1;
  // timing
  cudaEvent_t ev[2 * 1024];
  int ev_used = 0;
  int ev_phase[1024];
  double ms[PH_COUNT] = {};
  int64_t launches[PH_COUNT] = {};
  std::string last_error;
};

// ---- helpers implemented in tk_api.cu ----
void tk_throw(tucker_status code, const std::string& msg);
void tk_check_cuda(cudaError_t e, const char* what);
void* tk_alloc(tucker_ctx* c, size_t bytes);
// temporary device memory through the context's callbacks (or cudaMalloc);
// tk_dev_free only after the work using it has completed
void* tk_dev_alloc(tucker_ctx* c, size_t bytes);
void tk_dev_free(tucker_ctx* c, void* p, size_t bytes);
void tk_phase_begin(tucker_ctx* c, int phase, cudaStream_t s);
void tk_phase_end(tucker_ctx* c, cudaStream_t s);
void tk_launched(tucker_ctx* c, int phase, int n = 1);
int tk_sm_count();

// ---- scan / sort (tk_scan_sort.cu) ----
// exclusive prefix sum of n values; out may alias in. tmp is scratch from tk_scan_tmp_bytes.
size_t tk_scan_tmp_bytes(int64_t n, size_t esz);
void tk_exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, void* tmp, cudaStream_t s);
void tk_exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, void* tmp, cudaStream_t s);
// stable LSD radix sort of (key, value) pairs on the low `bits` bits of the keys.
size_t tk_sort_tmp_bytes(int64_t n);
void tk_radix_sort_pairs(uint32_t* keys, int32_t* vals, uint32_t* keys_alt, int32_t* vals_alt, int64_t n,
                         int bits, void* tmp, cudaStream_t s, uint32_t** keys_out, int32_t** vals_out);

// ---- partition (tk_partition.cu) ----
// Histograms (with coordinate validation) and popularity labels of every mode;
// fills c->relabel / c->unlabel / c->fiber.  Throws TUCKER_ERR_INDEX on an
// out-of-range coordinate.
void tk_relabel_modes(tucker_ctx* c, const int32_t* const* d_idx, cudaStream_t s);
void tk_partition_mode(tucker_ctx* c, int n, const int32_t* const* d_idx, const void* d_val, int P,
                       cudaStream_t s);
void tk_partition_export(tucker_ctx* c, int n, int64_t* d_bin_ptr, int32_t* d_perm, cudaStream_t s);
void tk_partition_export_into(tucker_ctx* c, int n, int64_t* d_bin_ptr, int32_t* d_perm, void* scan_tmp,
                              cudaStream_t s);
tucker_status tk_guarded_call(tucker_ctx* c, void (*body)(void*), void* arg);

// ---- TTM-chain (tk_ttmc.cu) ----
int tk_ttmc_groups(const tucker_ctx* c, int n);
int tk_ttmc_threads_per_sm(const tucker_ctx* c, int n);
void tk_ttmc_forward(tucker_ctx* c, int n, void* const* F, const int* ldF, const void* vals_override, void* Z,
                     cudaStream_t s);
// tensor-core form (tk_ttmc_tc.cu): 4-mode FP32 contexts with 32 <= K_a K_b <= 128,
// K_c <= 48 and Khat >= 256 (a < b < c the modes other than n)
bool tk_ttmc_tc_eligible(const tucker_ctx* c, int n);
void tk_ttmc_tc_build(tucker_ctx* c, int n, cudaStream_t s);
void tk_ttmc_tc_launch(tucker_ctx* c, int n, void* const* F, const int* ldF, const void* vals_override, void* Z,
                       cudaStream_t s);
void tk_ttmc_backward(tucker_ctx* c, int n, void* const* F, const int* ldF, const void* dZ,
                      const void* vals_override, void* const* dF, void* dval, cudaStream_t s);

// ---- Gram on the tensor cores (tk_gram_tc.cu) ----
bool tk_gram_tc_supported(int Khat);
// tiled form for 8 <= Khat <= 4096 (Khat % 4 == 0; used above 128, and at every
// Khat for the BF16 split): pairs of 128-column blocks x row splits
bool tk_gram_tiles_supported(int Khat);
int tk_gram_tiles_pairs(int Khat);
int tk_gram_tiles_splits(const tucker_ctx* c, int Khat, int R);
void tk_gram_tiles(tucker_ctx* c, const float* Z, int R, int Khat, float* Wpart, int2* pairs, double* W, bool bf16,
                   cudaStream_t s);
// W (FP64, Khat x Khat) = Z^T Z via per-CTA partials in Wpart (>= sm_count 128 x 128 tiles)
void tk_gram_tc(tucker_ctx* c, const float* Z, int R, int Khat, float* Wpart, size_t Wpart_elems, double* W,
                cudaStream_t s);

// ---- factor update (tk_factor.cu) ----
// F_out[row_map[r]] = U[r] (row_map = row_id for a caller's buffer, frow for
// the context's relabelled factor buffers); other rows zero.
void tk_factor_update(tucker_ctx* c, int n, const void* Z, void* F_out, int ldF_out, const int32_t* row_map,
                      double* sigma_out, cudaStream_t s);
void tk_alloc_fuws(tucker_ctx* c, int n);

// ---- prior distribution schemes (tk_schemes.cu) ----
// Section 4.1 metrics of CoarseG (scheme 1) or MediumG (scheme 2) along mode n:
// out3 = {E_max, R_sum, R_max} on the host; d_E / d_R (P int64 each, may be
// NULL) receive E^p and R^p.  Synchronises s.
void tk_scheme_metrics(tucker_ctx* c, int n, int scheme, int P, const int32_t* const* d_pos, int64_t* out3,
                       int64_t* d_E, int64_t* d_R, cudaStream_t s);

// ---- the Lanczos route of the factor update (tk_lanczos.cu) ----
void tk_lanczos_alloc(tucker_ctx* c, int n);
// runs the bidiagonalisation of Z, writes W = B^T B (m x m) into the mode's
// factor-update workspace and returns m
int tk_lanczos_bidiag(tucker_ctx* c, int n, const void* Z, cudaStream_t s);
// after the eigensolve of B^T B: V (m x K) -> V_K = V_lanczos Q (Khat x K), Vs
void tk_lanczos_vk(tucker_ctx* c, int n, int m, cudaStream_t s);

// ---- core / fit (tk_core.cu) ----
// New core from the TTM-chain of mode tk_core_mode(c); with before_Fn, the
// stream waits on that event after the TTM-chain, before F_n is first read.
int tk_core_mode(const tucker_ctx* c);
void tk_core(tucker_ctx* c, void* const* F, const int* ldF, void* G_out, cudaStream_t s, cudaEvent_t before_Fn = nullptr);
// texture object over one of the context's factor buffers (0 if none)
cudaTextureObject_t tk_factor_tex(const tucker_ctx* c, const void* F);
double tk_norm2(tucker_ctx* c, const void* vals, int64_t n, cudaStream_t s);

// ---- small device utilities ----
// dst[dst_map ? dst_map[r] : r][0..ldd) = src[src_map ? src_map[r] : r][0..cols), zero padded
void tk_copy_factor(tucker_ctx* c, const void* src, int lds, void* dst, int ldd, int64_t rows, int cols,
                    const int32_t* dst_map, const int32_t* src_map, cudaStream_t s);

#define TK_CUDA(x) tk_check_cuda((x), #x)

static inline __host__ __device__ int64_t tk_ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
