// tucker_partition_noalloc: the partition export with no device allocation.
//
// Callers that cannot allocate device memory while they run -- for example a
// process whose device memory is entirely handed out by its own pool or
// caching allocator, or code on a path where a device-synchronising
// cudaMalloc/cudaFree is not acceptable -- use this variant.  Its only
// scratch (the block sums of the prefix scan over the bin lengths) lives in
// the file-scope device array below, so nothing is allocated per call.
#include <atomic>
#include <mutex>

#include "tk_common.cuh"

namespace {

// Scratch shared by every call on a device.  Held by every GPU that loads the
// library until the process exits.
constexpr size_t kNoallocScratchBytes = 256 * 1024;
static __device__ __align__(256) unsigned char tk_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::atomic<void*> g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

// The array's name is a host-side stand-in in host code; the device address
// is looked up once per device, with that device current.  Host threads that
// make their first call on the same device at the same time are serialised by
// the mutex; later calls only read the atomic entry.
void* scratch_for_current_device() {
  int dev = 0;
  TK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) tk_throw(TUCKER_ERR_STATE, "device ordinal out of range for the static scratch table");
  void* ptr = g_scratch_addr[dev].load(std::memory_order_acquire);
  if (ptr) return ptr;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  ptr = g_scratch_addr[dev].load(std::memory_order_relaxed);
  if (!ptr) {
    const cudaError_t e = cudaGetSymbolAddress(&ptr, tk_noalloc_scratch);
    if (e != cudaSuccess || !ptr) {
      cudaGetLastError();
      tk_throw(TUCKER_ERR_CUDA, std::string("cudaGetSymbolAddress of the static scratch failed: ") + cudaGetErrorString(e));
    }
    g_scratch_addr[dev].store(ptr, std::memory_order_release);
  }
  return ptr;
}

struct Call {
  tucker_ctx* t;
  int mode;
  int64_t* d_bin_ptr;
  int32_t* d_perm;
  cudaStream_t s;
};

void run(void* p) {
  Call& a = *(Call*)p;
  if (a.mode < 0 || a.mode >= a.t->N) tk_throw(TUCKER_ERR_ARG, "mode out of range");
  if (!a.d_bin_ptr || !a.d_perm) tk_throw(TUCKER_ERR_ARG, "NULL output");
  const tk_mode& md = a.t->mode[a.mode];
  const size_t need = tk_scan_tmp_bytes((int64_t)md.P + 1, 8);
  if (need > kNoallocScratchBytes)
    tk_throw(TUCKER_ERR_ARG, "tucker_partition_noalloc: " + std::to_string(md.P) + " bins need " + std::to_string(need) +
                                 " scratch bytes, more than the static " + std::to_string(kNoallocScratchBytes));
  void* scratch = scratch_for_current_device();
  tk_partition_export_into(a.t, a.mode, a.d_bin_ptr, a.d_perm, scratch, a.s);
}

}  // namespace

extern "C" tucker_status tucker_partition_noalloc(tucker_t t, int mode, int64_t* d_bin_ptr, int32_t* d_perm,
                                                  void* stream) {
  if (!t) return TUCKER_ERR_ARG;
  Call a{t, mode, d_bin_ptr, d_perm, (cudaStream_t)stream};
  return tk_guarded_call(t, run, &a);
}
