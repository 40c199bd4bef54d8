// Allocation-free population evaluation: ebic_eval_population_noalloc.
//
// Some callers cannot allocate device memory when they evaluate. Examples: a serving loop that
// must never take the allocator's lock or risk an out-of-memory error in the middle of a
// request; and a process whose device memory is already carved up by another framework's
// caching allocator, so that a cudaMalloc of ours could fail or fragment its pool. The regular
// entry point allocates small stream-ordered scratch on every call (a status word, plus device
// copies of host inputs). This entry point uses a fixed scratch area compiled into the library
// instead.
//
// The scratch is a file-scope __device__ array of kNoAllocScratchBytes (1 MiB). Every GPU that
// loads this library holds it until the process exits. Host code cannot use the array's name as
// a device address: in host code the symbol is only a host-side stand-in, and a kernel given it
// would fault, or on a system where the GPU can reach host memory it would silently use the
// wrong memory. So the first call on each device (with that device current) fetches the real
// device address once with cudaGetSymbolAddress, checks it, caches it per device and passes it
// to the kernels. The same first call also loads, on that device, the code of every kernel this
// entry point can launch (every evaluator variant and the list check), so that no later call
// makes the CUDA runtime load code. Make that first call before any stream capture.
//
// All calls share the one array, and it keeps the previous call's contents: the status word is
// cleared at the start of every call. Calls that overlap on the GPU (different streams, or
// different host threads, at the same time) race on the array and must not be issued.
#include <mutex>
#include <string>

#include "ebic.h"
#include "ebic_internal.h"

namespace ebic {
namespace {

constexpr size_t kNoAllocScratchBytes = 1u << 20;
constexpr size_t kNoAllocListsOffset = 256;  // [0, 4): per-call status word; lists from here

static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
uint8_t* g_scratch_ptr[kMaxDevices] = {};

// One-time set-up on `dev` (the current device): the scratch array's device address, and the
// code of every kernel this entry point launches loaded (evaluator shared-memory limits raised).
int scratch_address(int dev, uint8_t** out) {
  if (dev < 0 || dev >= kMaxDevices) return set_last_error(EBIC_ERR_UNSUPPORTED, "device index");
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      (void)cudaGetLastError();
      return set_last_error(EBIC_ERR_CUDA,
                            (std::string("cudaGetSymbolAddress(no-allocation scratch): ") +
                             cudaGetErrorString(e)).c_str());
    }
    e = ready_eval_w8v4();
    if (e == cudaSuccess) e = ready_eval_w16v4();
    if (e == cudaSuccess) e = ready_eval_w16v2();
    if (e == cudaSuccess) e = ready_eval_w16v1();
    if (e == cudaSuccess) e = ready_prepare();
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      return set_last_error(EBIC_ERR_CUDA, (std::string("loading the evaluator kernels: ") +
                                            cudaGetErrorString(e)).c_str());
    }
    g_scratch_ptr[dev] = static_cast<uint8_t*>(p);
  }
  *out = g_scratch_ptr[dev];
  return EBIC_OK;
}

// Where a caller's pointer lives, relative to device `dev`, from one attribute query.
enum class Place { kHost, kDevice, kForeign };

Place place_of(const void* p, int dev) {
  cudaPointerAttributes at;
  if (!p || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return Place::kHost;
  }
  if (at.type == cudaMemoryTypeManaged) return Place::kDevice;
  if (at.type == cudaMemoryTypeDevice) return at.device == dev ? Place::kDevice : Place::kForeign;
  return Place::kHost;
}

int cuda_error(cudaError_t e, const char* what) {
  (void)cudaGetLastError();
  return set_last_error(e == cudaErrorMemoryAllocation ? EBIC_ERR_OOM : EBIC_ERR_CUDA,
                        (std::string(what) + ": " + cudaGetErrorString(e)).c_str());
}

}  // namespace
}  // namespace ebic

using namespace ebic;

extern "C" int ebic_eval_population_noalloc(const ebic_matrix* m, const uint16_t* cols,
                                            const uint32_t* offsets, uint32_t n_cand,
                                            uint32_t flags, uint32_t* counts, uint32_t* bitmaps,
                                            void* stream) {
  if (!m) return set_last_error(EBIC_ERR_INVALID_ARG, "matrix is NULL");
  if (flags & ~EBIC_NEGATIVE_TRENDS) return set_last_error(EBIC_ERR_INVALID_ARG, "unknown flag");
  if (n_cand == 0) return EBIC_OK;
  if (!cols || !offsets || !counts) return set_last_error(EBIC_ERR_INVALID_ARG, "NULL argument");
  MatrixView v;
  matrix_view(m, &v);
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) {
    (void)cudaGetLastError();
    prev = -1;
  }
  if (prev != v.device) {
    cudaError_t e = cudaSetDevice(v.device);
    if (e != cudaSuccess) return cuda_error(e, "cudaSetDevice");
  }
  struct Restore {
    int prev, dev;
    ~Restore() {
      if (prev >= 0 && prev != dev) (void)cudaSetDevice(prev);
    }
  } restore{prev, v.device};
  const int dev = v.device;
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  // Every pointer's placement, before anything is dereferenced on the host: memory of another
  // device is rejected (the host could not read it, and the kernels must not).
  const Place p_counts = place_of(counts, dev);
  const Place p_bitmaps = bitmaps ? place_of(bitmaps, dev) : Place::kDevice;
  const Place p_cols = place_of(cols, dev), p_offs = place_of(offsets, dev);
  if (p_counts == Place::kForeign || p_bitmaps == Place::kForeign || p_cols == Place::kForeign ||
      p_offs == Place::kForeign)
    return set_last_error(EBIC_ERR_INVALID_ARG,
                          "ebic_eval_population_noalloc: buffer on another device");
  // Outputs cannot be staged without an allocation: they must already be device memory.
  if (p_counts != Place::kDevice || p_bitmaps != Place::kDevice)
    return set_last_error(EBIC_ERR_INVALID_ARG,
                          "ebic_eval_population_noalloc: counts and bitmaps must be device "
                          "memory of the matrix's device");
  uint8_t* scratch = nullptr;
  int rc = scratch_address(dev, &scratch);
  if (rc != EBIC_OK) return rc;
  uint32_t* err = reinterpret_cast<uint32_t*>(scratch);

  const bool cols_dev = p_cols == Place::kDevice, offs_dev = p_offs == Place::kDevice;
  if (cols_dev != offs_dev)
    return set_last_error(EBIC_ERR_INVALID_ARG,
                          "cols and offsets must both be host memory or both device memory");
  const uint16_t* dcols = cols;
  const uint32_t* doffs = offsets;
  int64_t total_hint = 0;
  if (!cols_dev) {
    // host lists: checked here, then staged into the fixed scratch if they fit
    const char* why = check_candidates_host_c(cols, offsets, n_cand, v.L.cols);
    if (why[0]) return set_last_error(EBIC_ERR_INVALID_ARG, why);
    total_hint = offsets[n_cand];
    const size_t off_bytes = ((size_t)n_cand + 1) * sizeof(uint32_t);
    const size_t col_off = kNoAllocListsOffset + ((off_bytes + 255) / 256) * 256;
    const size_t need = col_off + (size_t)total_hint * sizeof(uint16_t);
    if (need > kNoAllocScratchBytes)
      return set_last_error(
          EBIC_ERR_UNSUPPORTED,
          ("ebic_eval_population_noalloc: a host-resident population needs " +
           std::to_string(need) + " bytes of scratch, more than the fixed " +
           std::to_string(kNoAllocScratchBytes) +
           " bytes; pass the population in device memory or use ebic_eval_population")
              .c_str());
    cudaError_t e = cudaMemcpyAsync(scratch + kNoAllocListsOffset, offsets, off_bytes,
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(scratch + col_off, cols, (size_t)total_hint * sizeof(uint16_t),
                          cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_error(e, "staging the population into the scratch");
    doffs = reinterpret_cast<const uint32_t*>(scratch + kNoAllocListsOffset);
    dcols = reinterpret_cast<const uint16_t*>(scratch + col_off);
  }

  EvalArgs a;
  EvalConfig cfg;
  const CUtensorMap* tmap = nullptr;
  rc = matrix_eval_plan(m, n_cand, total_hint, &a, &cfg, &tmap);
  if (rc != EBIC_OK) return rc;

  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(uint32_t), s);  // the status word starts at 0
  if (e != cudaSuccess) return cuda_error(e, "clearing the scratch status word");
  PrepareArgs pa;
  pa.cols[0] = dcols;
  pa.offsets[0] = doffs;
  pa.n[0] = cols_dev ? n_cand : 0;  // host lists were checked above
  pa.ncols = v.L.cols;
  pa.zero = counts;
  pa.n_zero = n_cand;
  pa.err = err;
  pa.status = v.status;
  e = launch_prepare(pa, s);
  if (e != cudaSuccess) return cuda_error(e, "prepare launch");
  a.n_cand = n_cand;
  a.cand_cols = dcols;
  a.cand_offsets = doffs;
  a.counts = counts;
  a.bitmaps = bitmaps;
  a.err = err;
  a.err_out = err;
  a.status = v.status;
  cfg.negative = (flags & EBIC_NEGATIVE_TRENDS) != 0;
  cfg.bitmaps = bitmaps != nullptr;
  e = launch_eval(cfg, tmap, a, s);
  if (e != cudaSuccess) return cuda_error(e, "evaluator launch");
  return EBIC_OK;
}
