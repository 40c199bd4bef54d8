// Host runtime and C ABI of the EBIC GB300 library: argument checks, placement of host/device
// buffers, stream-ordered scratch, tensor-map setup, launch planning and error reporting.
// Every computational step runs in this library's CUDA kernels; this file only moves data and
// launches them.
#include <cudaTypedefs.h>

#include <algorithm>
#include <climits>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "ebic.h"
#include "ebic_internal.h"

using namespace ebic;

struct ebic_matrix {
  int device = 0;
  Layout L;
  uint32_t flags = 0;
  float fill = 0.f;
  uint32_t* ranks = nullptr;   // device rank matrix
  uint32_t* status = nullptr;  // device deferred-status word
  int num_sms = 0;
  std::mutex mu;
  CUtensorMap tmap[3];         // one per tile height TS = 1, 2, 4
  bool tmap_ok[3] = {false, false, false};
  int tile = 0;                // 0: built-in tile choice; else the TS every evaluation uses
  int chunk = 0;               // 0: built-in chunk size; else candidate columns per chunk
  uint32_t* pairs = nullptr;   // pair table [cols*cols][pair_stride], padding zero, or null
  uint32_t pair_stride = 0;
  size_t pair_bytes = 0;
  int64_t row_offset = 0;      // a row shard: its first row in the whole matrix (a multiple of 32)
  int64_t total_rows = 0;      // and the whole matrix's rows (rows when not a shard)
};

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  int code = EBIC_ERR_CUDA;
  if (e == cudaErrorMemoryAllocation) code = EBIC_ERR_OOM;
  if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) code = EBIC_ERR_NO_DEVICE;
  (void)cudaGetLastError();
  return fail(code, std::string(what) + ": " + cudaGetErrorString(e));
}

#define EBIC_CUDA(expr)                                      \
  do {                                                       \
    cudaError_t e_ = (expr);                                 \
    if (e_ != cudaSuccess) return cuda_fail(e_, #expr);      \
  } while (0)

// Current device switched for the duration of a call.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) { prev = -1; (void)cudaGetLastError(); }
    if (prev != dev) (void)cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) (void)cudaSetDevice(prev);
  }
};

// Stream-ordered scratch freed on the same stream when the call ends.
struct Scratch {
  cudaStream_t s;
  std::vector<void*> ptrs;
  explicit Scratch(cudaStream_t st) : s(st) {}
  cudaError_t alloc(void** p, size_t bytes) {
    cudaError_t e = cudaMallocAsync(p, bytes ? bytes : 16, s);
    if (e == cudaSuccess) ptrs.push_back(*p);
    return e;
  }
  ~Scratch() {
    for (void* p : ptrs) (void)cudaFreeAsync(p, s);
  }
};

// true: device (or managed) memory of `dev`; false: host memory (pageable or pinned)
bool on_device(const void* p, int dev) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

bool foreign_device(const void* p, int dev) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice && at.device != dev;
}

// A pointer's placement relative to device `dev`, from one attribute query.
struct Where {
  bool dev = false;      // device memory of `dev`, or managed
  bool foreign = false;  // device memory of another device
  void* mapped = nullptr;  // pinned host memory: the address kernels use for it
};

Where where(const void* p, int dev) {
  Where w;
  if (!p) return w;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return w;
  }
  w.dev = at.type == cudaMemoryTypeManaged || (at.type == cudaMemoryTypeDevice && at.device == dev);
  w.foreign = at.type == cudaMemoryTypeDevice && at.device != dev;
  if (at.type == cudaMemoryTypeHost) w.mapped = at.devicePointer;
  return w;
}

// A host word that kernels can write directly (pinned, mapped), one per host thread: the error
// word of a call whose outputs are on the host reaches the host through it without a copy.
struct MappedWord {
  uint32_t* host = nullptr;
  uint32_t* dev = nullptr;
  ~MappedWord() {
    if (host) (void)cudaFreeHost(host);
  }
  uint32_t* get() {
    if (!dev) {
      void* h = nullptr;
      if (cudaHostAlloc(&h, 64, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
      }
      void* d = nullptr;
      if (cudaHostGetDevicePointer(&d, h, 0) != cudaSuccess) {
        (void)cudaGetLastError();
        (void)cudaFreeHost(h);
        return nullptr;
      }
      host = static_cast<uint32_t*>(h);
      dev = static_cast<uint32_t*>(d);
    }
    return dev;
  }
};
thread_local MappedWord t_err_word;

// A host input read in place by the kernels when it is pinned, else copied.
template <class T>
cudaError_t input_at(const T* p, size_t n, const Where& w, Scratch& sc, const T** out) {
  if (!w.dev && w.mapped) {
    *out = static_cast<const T*>(w.mapped);
    return cudaSuccess;
  }
  return to_device_at(p, n, w.dev, sc, out);
}

// to_device / out_buffer with the placement already known.
template <class T>
cudaError_t to_device_at(const T* p, size_t n, bool is_dev, Scratch& sc, const T** out) {
  if (is_dev) { *out = p; return cudaSuccess; }
  void* d = nullptr;
  cudaError_t e = sc.alloc(&d, n * sizeof(T));
  if (e != cudaSuccess) return e;
  if (n) e = cudaMemcpyAsync(d, p, n * sizeof(T), cudaMemcpyHostToDevice, sc.s);
  *out = static_cast<const T*>(d);
  return e;
}

template <class T>
cudaError_t out_buffer_at(T* p, size_t n, bool is_dev, Scratch& sc, T** out, bool* host) {
  if (is_dev) { *out = p; *host = false; return cudaSuccess; }
  void* d = nullptr;
  cudaError_t e = sc.alloc(&d, n * sizeof(T));
  *out = static_cast<T*>(d);
  *host = true;
  return e;
}

template <class T>
cudaError_t to_device(const T* p, size_t n, int dev, Scratch& sc, const T** out) {
  if (on_device(p, dev)) { *out = p; return cudaSuccess; }
  void* d = nullptr;
  cudaError_t e = sc.alloc(&d, n * sizeof(T));
  if (e != cudaSuccess) return e;
  if (n) e = cudaMemcpyAsync(d, p, n * sizeof(T), cudaMemcpyHostToDevice, sc.s);
  *out = static_cast<const T*>(d);
  return e;
}

template <class T>
cudaError_t out_buffer(T* p, size_t n, int dev, Scratch& sc, T** out, bool* host) {
  if (on_device(p, dev)) { *out = p; *host = false; return cudaSuccess; }
  void* d = nullptr;
  cudaError_t e = sc.alloc(&d, n * sizeof(T));
  *out = static_cast<T*>(d);
  *host = true;
  return e;
}

std::once_flag g_pool_once[64];
void init_pool(int dev) {
  if (dev < 0 || dev >= 64) return;
  std::call_once(g_pool_once[dev], [dev] {
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t keep = UINT64_MAX;  // keep freed scratch in the pool instead of the OS
      (void)cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    (void)cudaGetLastError();
  });
}

// Host-side check of a CSR candidate list: offsets[0] == 0, lengths in [1, 64], columns in
// range and distinct. Returns an empty string when valid.
// The offsets of a host-resident CSR list: offsets[0] == 0 and every length in [1, 64], so
// offsets[n] bounds the columns a copy reads.
std::string check_offsets_host(const uint32_t* offsets, uint32_t n) {
  if (offsets[0] != 0) return "offsets[0] must be 0";
  for (uint32_t i = 0; i < n; ++i) {
    const uint32_t a = offsets[i], b = offsets[i + 1];
    if (b <= a || b - a > (uint32_t)kMaxLen)
      return "candidate " + std::to_string(i) + " has length outside [1, 64]";
  }
  return "";
}

// The columns of a host-resident CSR list whose offsets passed check_offsets_host: each below
// ncols and distinct within its candidate.
std::string check_columns_host(const uint16_t* cols, const uint32_t* offsets, uint32_t n,
                               int32_t ncols) {
  std::vector<uint32_t> seen((size_t)ncols, 0xFFFFFFFFu);
  for (uint32_t i = 0; i < n; ++i) {
    const uint32_t a = offsets[i], b = offsets[i + 1];
    for (uint32_t j = a; j < b; ++j) {
      const uint16_t c = cols[j];
      if (c >= (uint32_t)ncols)
        return "candidate " + std::to_string(i) + " has column " + std::to_string(c) +
               " >= cols";
      if (seen[c] == i) return "candidate " + std::to_string(i) + " repeats column " +
                               std::to_string(c);
      seen[c] = i;
    }
  }
  return "";
}

std::string check_candidates_host(const uint16_t* cols, const uint32_t* offsets, uint32_t n,
                                  int32_t ncols) {
  std::string why = check_offsets_host(offsets, n);
  return why.empty() ? check_columns_host(cols, offsets, n, ncols) : why;
}

// Tensor map over the rank matrix: dims {32*VEC words, Q slabs, C columns}, box
// {32*VEC, TS, col_box}. Built once per (matrix, TS) and cached.
int get_tmap(ebic_matrix* m, int ts, int col_box, const CUtensorMap** out) {
  const int idx = ts == 1 ? 0 : ts == 2 ? 1 : 2;
  std::lock_guard<std::mutex> lk(m->mu);
  if (!m->tmap_ok[idx]) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
      cudaDriverEntryPointQueryResult q;
      void* fn = nullptr;
      cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                       cudaEnableDefault, &q);
      if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
        return fail(EBIC_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
      encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const Layout& L = m->L;
    const cuuint64_t wps = 32ull * (cuuint64_t)L.vec;
    cuuint64_t dims[3] = {wps, (cuuint64_t)L.slabs, (cuuint64_t)L.cols};
    cuuint64_t strides[2] = {wps * 4ull, (cuuint64_t)L.slabs * wps * 4ull};
    cuuint32_t box[3] = {(cuuint32_t)wps, (cuuint32_t)ts, (cuuint32_t)col_box};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = encode(&m->tmap[idx], CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, m->ranks, dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
      return fail(EBIC_ERR_CUDA, "cuTensorMapEncodeTiled failed with code " + std::to_string(r));
    m->tmap_ok[idx] = true;
  }
  *out = &m->tmap[idx];
  return EBIC_OK;
}

// ---- diagnostics: launch counter and per-kernel CUDA-event timing --------------------------
std::atomic<int64_t> g_launches{0};
std::atomic<bool> g_timing{false};
std::mutex g_timing_mu;
std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_timed[EBIC_TIMING_KINDS];
std::vector<cudaEvent_t> g_event_pool;

cudaEvent_t take_event() {
  std::lock_guard<std::mutex> lk(g_timing_mu);
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) { (void)cudaGetLastError(); return nullptr; }
  return e;
}

// Records a start event before and an end event after the launches in its scope, on the
// stream they are launched on, when timing is enabled.
// Kernels of a call are chained with programmatic dependent launch unless per-kernel timing is
// on (an event recorded between two kernels would separate them anyway).
bool timing_on() { return g_timing.load(std::memory_order_relaxed); }

struct Timed {
  int kind;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  Timed(int k, cudaStream_t st) : kind(k), s(st) {
    if (g_timing.load(std::memory_order_relaxed)) {
      a = take_event();
      if (a && cudaEventRecord(a, s) != cudaSuccess) { (void)cudaGetLastError(); a = nullptr; }
    }
  }
  ~Timed() {
    if (!a) return;
    cudaEvent_t b = take_event();
    if (!b || cudaEventRecord(b, s) != cudaSuccess) { (void)cudaGetLastError(); return; }
    std::lock_guard<std::mutex> lk(g_timing_mu);
    g_timed[kind].emplace_back(a, b);
  }
};

int status_code(uint32_t bits, const char* where) {
  if (bits & kErrTimeout)
    return fail(EBIC_ERR_DEVICE_TIMEOUT, std::string(where) + ": a bounded device wait expired");
  if (bits & kErrInvalid)
    return fail(EBIC_ERR_INVALID_ARG,
                std::string(where) + ": the device-side check rejected a candidate list");
  return EBIC_OK;
}

}  // namespace

namespace ebic {

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

Layout make_layout(int64_t rows, int32_t cols) {
  Layout L;
  L.rows = rows;
  L.cols = cols;
  L.words = (rows + 31) / 32;
  if (cols <= 127) {
    L.width = 8;
    L.vec = 4;
  } else {
    L.width = 16;
    L.vec = (int64_t)cols * 512 <= kStageMax ? 4 : (int64_t)cols * 256 <= kStageMax ? 2 : 1;
  }
  L.rows_per_group = L.width == 8 ? 128 : 64;
  L.words_per_group = L.rows_per_group / 32;
  const int64_t g = (rows + L.rows_per_group - 1) / L.rows_per_group;
  L.slabs = (g + L.vec - 1) / L.vec;
  L.groups = L.slabs * L.vec;
  return L;
}

static void col_boxes(int32_t cols, int* nb, int* cb) {
  *nb = (cols + 255) / 256;
  *cb = (cols + *nb - 1) / *nb;
}

int default_tile_slabs(const Layout& L) {
  int nb, cb;
  col_boxes(L.cols, &nb, &cb);
  for (int ts = 4; ts >= 1; ts >>= 1) {
    if (ts > L.slabs && ts > 1) continue;
    if ((int64_t)nb * cb * ts * 128 * L.vec <= kStageMax) return ts;
  }
  return 1;
}

bool plan_eval(const Layout& L, int ts, uint32_t n_cand, int64_t total_cols_hint, int grid,
               EvalArgs* a, int32_t chunk_override) {
  int nb, cb;
  col_boxes(L.cols, &nb, &cb);
  const int64_t col_stride = (int64_t)ts * 128 * L.vec;
  const int64_t stage = (int64_t)nb * cb * col_stride;
  // chunk buffers: (CC + slack) column slots and (CC + 1) offsets, 2 bytes each
  const int64_t left = kSmemDynMax - 2 * stage - 2 * (kChunkSlack + 1) - 256;
  int64_t cc_max = std::min<int64_t>(kMaxChunkCols, left / 4);
  cc_max = cc_max / 64 * 64;
  if (cc_max < 64) return false;
  const int64_t n_tiles = (L.slabs + ts - 1) / ts;
  const int64_t total = total_cols_hint > 0 ? total_cols_hint : (int64_t)n_cand * 16;
  const int64_t want_chunks = std::max<int64_t>(1, (2 * (int64_t)grid + n_tiles - 1) / n_tiles);
  int64_t cc = (total + want_chunks - 1) / want_chunks;
  if (chunk_override > 0) cc = chunk_override;
  cc = (cc + 63) / 64 * 64;
  cc = std::max<int64_t>(64, std::min(cc, cc_max));
  a->cols = L.cols;
  a->slabs = L.slabs;
  a->groups = L.groups;
  a->words = L.words;
  a->bitmap_stride = L.words;
  a->chunk_cols = (int32_t)cc;
  a->col_box = cb;
  a->n_col_boxes = nb;
  a->stage_bytes = (uint32_t)stage;
  a->smem_bytes =
      (uint32_t)((2 * stage + 2 * (cc + kChunkSlack) + 2 * (cc + 1) + 15) / 16 * 16);
  return true;
}

void matrix_view(const ebic_matrix* m, MatrixView* v) {
  v->device = m->device;
  v->L = m->L;
  v->status = m->status;
  v->num_sms = m->num_sms;
  v->pairs = m->pairs;
  v->pair_stride = m->pair_stride;
  v->row_offset = m->row_offset;
  v->total_rows = m->total_rows;
}

int matrix_eval_plan(const ebic_matrix* cm, uint32_t n_cand, int64_t total_cols_hint,
                     EvalArgs* a, EvalConfig* cfg, const CUtensorMap** tmap, int ts_cap) {
  ebic_matrix* m = const_cast<ebic_matrix*>(cm);
  const Layout& L = m->L;
  int ts = m->tile ? m->tile : default_tile_slabs(L);
  while (ts > 1 && ts > L.slabs) ts >>= 1;
  while (ts_cap > 0 && ts > ts_cap) ts >>= 1;
  if (!plan_eval(L, ts, n_cand, total_cols_hint, m->num_sms, a, m->chunk))
    return fail(EBIC_ERR_UNSUPPORTED, "no shared-memory plan for this matrix shape");
  int rc = get_tmap(m, ts, a->col_box, tmap);
  if (rc != EBIC_OK) return rc;
  cfg->width = L.width;
  cfg->vec = L.vec;
  cfg->ts = ts;
  cfg->grid = m->num_sms;
  return EBIC_OK;
}

int set_last_error(int code, const char* msg) { return fail(code, msg); }

const char* check_candidates_host_c(const uint16_t* cols, const uint32_t* offsets, uint32_t n,
                                    int32_t ncols) {
  thread_local std::string why;
  why = check_candidates_host(cols, offsets, n, ncols);
  return why.c_str();
}

cudaError_t launch_eval(const EvalConfig& cfg, const CUtensorMap* tmap, const EvalArgs& a,
                        cudaStream_t s) {
  if (cfg.width == 8) return launch_eval_w8v4(cfg, tmap, a, s);
  switch (cfg.vec) {
    case 4: return launch_eval_w16v4(cfg, tmap, a, s);
    case 2: return launch_eval_w16v2(cfg, tmap, a, s);
    case 1: return launch_eval_w16v1(cfg, tmap, a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ebic

// ebic_eval_population with the candidates' bitmaps `bitmap_stride` words apart (the pair table
// is built through this with its padded stride).
static int eval_population_impl(ebic_matrix* m, const uint16_t* cols, const uint32_t* offsets,
                         uint32_t n_cand, uint32_t flags, uint32_t* counts, uint32_t* bitmaps,
                         int64_t bitmap_stride, void* stream) {
  if (!m) return fail(EBIC_ERR_INVALID_ARG, "matrix is NULL");
  if (flags & ~(EBIC_NEGATIVE_TRENDS | EBIC_EVAL_DIRECT))
    return fail(EBIC_ERR_INVALID_ARG, "unknown eval flag");
  if (n_cand == 0) return EBIC_OK;
  if (!cols || !offsets || !counts) return fail(EBIC_ERR_INVALID_ARG, "NULL argument");
  DeviceGuard g(m->device);
  const int dev = m->device;
  const Layout& L = m->L;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (const void* p : {(const void*)cols, (const void*)offsets, (const void*)counts,
                        (const void*)bitmaps})
    if (foreign_device(p, dev)) return fail(EBIC_ERR_INVALID_ARG, "buffer on another device");

  const bool host_lists = !on_device(cols, dev) && !on_device(offsets, dev);
  int64_t total_hint = 0;
  if (host_lists) {
    std::string why = check_candidates_host(cols, offsets, n_cand, L.cols);
    if (!why.empty()) return fail(EBIC_ERR_INVALID_ARG, why);
    total_hint = offsets[n_cand];
  }

  int ts = m->tile ? m->tile : default_tile_slabs(L);
  while (ts > 1 && ts > L.slabs) ts >>= 1;
  EvalArgs a;
  if (!plan_eval(L, ts, n_cand, total_hint, m->num_sms, &a, m->chunk))
    return fail(EBIC_ERR_UNSUPPORTED, "no shared-memory plan for this matrix shape");
  const CUtensorMap* tmap = nullptr;
  int rc = get_tmap(m, ts, a.col_box, &tmap);
  if (rc != EBIC_OK) return rc;

  Scratch sc(s);
  uint32_t* err = nullptr;
  EBIC_CUDA(sc.alloc(reinterpret_cast<void**>(&err), sizeof(uint32_t)));
  EBIC_CUDA(cudaMemsetAsync(err, 0, sizeof(uint32_t), s));
  const uint16_t* dcols = nullptr;
  const uint32_t* doffs = nullptr;
  EBIC_CUDA(to_device(offsets, (size_t)n_cand + 1, dev, sc, &doffs));
  // the column count is only known from the offsets; device lists are read by the kernels
  const size_t ncols_total = host_lists ? offsets[n_cand] : 0;
  if (on_device(cols, dev)) {
    dcols = cols;
  } else {
    size_t n = ncols_total;
    if (!host_lists) {  // host columns with device offsets: fetch the total first
      uint32_t t = 0;
      EBIC_CUDA(cudaMemcpyAsync(&t, offsets + n_cand, 4, cudaMemcpyDeviceToHost, s));
      EBIC_CUDA(cudaStreamSynchronize(s));
      n = t;
    }
    EBIC_CUDA(to_device(cols, n, dev, sc, &dcols));
  }
  bool counts_host = false, bitmaps_host = false;
  uint32_t* dcounts = nullptr;
  uint32_t* dbitmaps = nullptr;
  EBIC_CUDA(out_buffer(counts, n_cand, dev, sc, &dcounts, &counts_host));
  if (bitmaps)
    EBIC_CUDA(out_buffer(bitmaps, (size_t)n_cand * bitmap_stride, dev, sc, &dbitmaps,
                         &bitmaps_host));

  const bool use_pairs = m->pairs && !(flags & EBIC_EVAL_DIRECT) && bitmap_stride == L.words;
  const bool neg = (flags & EBIC_NEGATIVE_TRENDS) != 0;
  uint32_t* dterms = nullptr;  // the pair-table term lists, built by the preparation kernel
  if (use_pairs)
    EBIC_CUDA(sc.alloc(reinterpret_cast<void**>(&dterms),
                       (size_t)n_cand * term_slots(neg) * sizeof(uint32_t)));
  {
    Timed t(EBIC_TIMING_PREPARE, s);
    PrepareArgs pa;
    pa.cols[0] = dcols;
    pa.offsets[0] = doffs;
    pa.n[0] = host_lists ? 0 : n_cand;  // host lists were checked on the host
    pa.ncols = L.cols;
    pa.zero = dcounts;
    pa.n_zero = n_cand;
    pa.err = err;
    pa.status = m->status;
    pa.terms = dterms;
    pa.n_terms_cand = use_pairs ? n_cand : 0;
    pa.pair_cols = L.cols;
    pa.pair_stride = m->pair_stride;
    pa.negative = neg;
    EBIC_CUDA(launch_prepare(pa, s));
  }
  if (use_pairs) {
    Timed t(EBIC_TIMING_PAIR_EVALUATE, s);
    PairArgs p;
    p.table = m->pairs;
    p.stride = m->pair_stride;
    p.C = L.cols;
    p.W = L.words;
    p.terms = dterms;
    p.n_cand = n_cand;
    p.counts = dcounts;
    p.bitmaps = dbitmaps;
    p.err = err;
    p.err_out = err;
    p.status = m->status;
    EBIC_CUDA(launch_pair_eval(p, neg, m->num_sms, !timing_on(), s));
  } else {
  a.n_cand = n_cand;
  a.cand_cols = dcols;
  a.cand_offsets = doffs;
  a.counts = dcounts;
  a.bitmaps = dbitmaps;
  a.bitmap_stride = bitmap_stride;
  a.err = err;
  a.err_out = err;
  a.status = m->status;
  EvalConfig cfg;
  cfg.width = L.width;
  cfg.vec = L.vec;
  cfg.ts = ts;
  cfg.negative = (flags & EBIC_NEGATIVE_TRENDS) != 0;
  cfg.bitmaps = dbitmaps != nullptr;
  cfg.grid = m->num_sms;
  {
    Timed t(EBIC_TIMING_EVALUATE, s);
    EBIC_CUDA(launch_eval(cfg, tmap, a, s));
  }
  }

  if (counts_host || bitmaps_host) {
    if (counts_host)
      EBIC_CUDA(cudaMemcpyAsync(counts, dcounts, (size_t)n_cand * 4, cudaMemcpyDeviceToHost, s));
    if (bitmaps_host)
      EBIC_CUDA(cudaMemcpyAsync(bitmaps, dbitmaps, (size_t)n_cand * bitmap_stride * 4,
                                cudaMemcpyDeviceToHost, s));
    uint32_t bits = 0;
    EBIC_CUDA(cudaMemcpyAsync(&bits, err, 4, cudaMemcpyDeviceToHost, s));
    EBIC_CUDA(cudaStreamSynchronize(s));
    return status_code(bits, "ebic_eval_population");
  }
  return EBIC_OK;
}


extern "C" {

int ebic_version(void) { return (1 << 16) | 0; }

const char* ebic_last_error(void) { return g_last_error.c_str(); }

int ebic_load_matrix(const float* x, int64_t rows, int32_t cols, int64_t ld, uint32_t flags,
                     float fill_value, void* stream, ebic_matrix** out) {
  if (!out) return fail(EBIC_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!x) return fail(EBIC_ERR_INVALID_ARG, "x is NULL");
  if (rows < 1 || rows > 2147483647LL)
    return fail(EBIC_ERR_INVALID_ARG, "rows must be in [1, 2^31-1]");
  if (cols < 1) return fail(EBIC_ERR_INVALID_ARG, "cols must be >= 1");
  if (cols > kMaxCols)
    return fail(EBIC_ERR_UNSUPPORTED, "cols > " + std::to_string(kMaxCols) +
                                          " is outside this build's limits");
  if (ld < cols) return fail(EBIC_ERR_INVALID_ARG, "ld must be >= cols");
  if (flags & ~EBIC_EXCLUDE_MISSING) return fail(EBIC_ERR_INVALID_ARG, "unknown load flag");
  if (std::isnan(fill_value)) return fail(EBIC_ERR_INVALID_ARG, "fill_value must not be NaN");

  int dev = 0;
  EBIC_CUDA(cudaGetDevice(&dev));
  init_pool(dev);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (foreign_device(x, dev)) return fail(EBIC_ERR_INVALID_ARG, "x is on another device");

  ebic_matrix* m = new ebic_matrix();
  m->device = dev;
  m->L = make_layout(rows, cols);
  m->flags = flags;
  m->fill = fill_value;
  m->total_rows = rows;
  auto cleanup = [&](int code) {
    if (m->ranks) cudaFree(m->ranks);
    if (m->status) cudaFree(m->status);
    delete m;
    return code;
  };
  cudaError_t e = cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "cudaDeviceGetAttribute"));
  e = cudaMalloc(&m->ranks, m->L.rank_words() * 4);
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "cudaMalloc(rank matrix)"));
  e = cudaMalloc(&m->status, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemsetAsync(m->status, 0, sizeof(uint32_t), s);
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "status word"));

  {
    Scratch sc(s);
    const float* dx = x;
    int64_t dld = ld;
    if (!on_device(x, dev)) {
      void* d = nullptr;
      e = sc.alloc(&d, (size_t)rows * cols * sizeof(float));
      if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(d, (size_t)cols * sizeof(float), x, (size_t)ld * sizeof(float),
                              (size_t)cols * sizeof(float), (size_t)rows, cudaMemcpyHostToDevice,
                              s);
      if (e != cudaSuccess) return cleanup(cuda_fail(e, "copy of x to the device"));
      dx = static_cast<const float*>(d);
      dld = cols;
    }
    {
      Timed t(EBIC_TIMING_RANK_TRANSFORM, s);
      e = launch_rank_transform(m->L, dx, dld, (flags & EBIC_EXCLUDE_MISSING) ? 1 : 0,
                                fill_value, m->ranks, m->status, m->num_sms, s);
    }
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "rank transform launch"));
  }
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "rank transform"));
  {  // a bounded wait of the transform that expired leaves the matrix unusable
    uint32_t bits = 0;
    e = cudaMemcpy(&bits, m->status, sizeof(uint32_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "rank transform status"));
    if (bits & kErrTimeout)
      return cleanup(fail(EBIC_ERR_DEVICE_TIMEOUT, "rank transform: a bounded device wait expired"));
  }
  *out = m;
  return EBIC_OK;
}

int ebic_free_matrix(ebic_matrix* m) {
  if (!m) return EBIC_OK;
  DeviceGuard g(m->device);
  if (m->pairs) cudaFree(m->pairs);
  cudaError_t e1 = cudaFree(m->ranks);
  cudaError_t e2 = cudaFree(m->status);
  delete m;
  if (e1 != cudaSuccess) return cuda_fail(e1, "cudaFree(rank matrix)");
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaFree(status)");
  return EBIC_OK;
}

int ebic_matrix_info(const ebic_matrix* m, int64_t* rows, int32_t* cols, int64_t* words,
                     int32_t* rank_bits) {
  if (!m) return fail(EBIC_ERR_INVALID_ARG, "matrix is NULL");
  if (rows) *rows = m->L.rows;
  if (cols) *cols = m->L.cols;
  if (words) *words = m->L.words;
  if (rank_bits) *rank_bits = m->L.width;
  return EBIC_OK;
}

int ebic_matrix_ranks(const ebic_matrix* m, uint16_t* out, void* stream) {
  if (!m || !out) return fail(EBIC_ERR_INVALID_ARG, "NULL argument");
  DeviceGuard g(m->device);
  const Layout& L = m->L;
  std::vector<uint32_t> raw(L.rank_words());
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  EBIC_CUDA(cudaMemcpyAsync(raw.data(), m->ranks, raw.size() * 4, cudaMemcpyDeviceToHost, s));
  EBIC_CUDA(cudaStreamSynchronize(s));
  const uint32_t mask = L.width == 8 ? 0xFFu : 0xFFFFu;
  for (int64_t r = 0; r < L.rows; ++r) {
    const int64_t g = r / L.rows_per_group, rr = r % L.rows_per_group;
    const int64_t lane = rr & 31, k = rr >> 5, q = g / L.vec, j = g % L.vec;
    for (int32_t c = 0; c < L.cols; ++c) {
      const size_t w = (((size_t)c * L.slabs + q) * 32 + lane) * L.vec + j;
      const uint32_t v = (raw[w] >> (L.width * k)) & mask;  // code 0 = missing, else rank + 1
      out[r * L.cols + c] = v == 0 ? 0xFFFFu : (uint16_t)(v - 1);
    }
  }
  return EBIC_OK;
}

int ebic_eval_population(const ebic_matrix* cm, const uint16_t* cols, const uint32_t* offsets,
                         uint32_t n_cand, uint32_t flags, uint32_t* counts, uint32_t* bitmaps,
                         void* stream) {
  ebic_matrix* m = const_cast<ebic_matrix*>(cm);
  if (!m) return fail(EBIC_ERR_INVALID_ARG, "matrix is NULL");
  return eval_population_impl(m, cols, offsets, n_cand, flags, counts, bitmaps, m->L.words,
                              stream);
}

}  // extern "C"

// ebic_fitness, and also the archive members' row counts into `arch_counts_out` (when not
// null; [n_arch], device or host).
static int fitness_impl(const ebic_matrix* cm, const uint16_t* cols, const uint32_t* offsets,
                        uint32_t n_cand, const uint32_t* counts, const uint32_t* bitmaps,
                        const uint16_t* arch_cols, const uint32_t* arch_offsets,
                        const uint32_t* arch_bitmaps, uint32_t n_arch, uint32_t flags,
                        uint64_t* fitness, uint32_t* overlaps, uint32_t* arch_counts_out,
                        void* stream) {
  ebic_matrix* m = const_cast<ebic_matrix*>(cm);
  if (!m) return fail(EBIC_ERR_INVALID_ARG, "matrix is NULL");
  if (flags != 0) return fail(EBIC_ERR_INVALID_ARG, "flags is reserved (pass 0)");
  if (n_cand == 0) return EBIC_OK;
  if (!cols || !offsets || !counts || !bitmaps || !fitness)
    return fail(EBIC_ERR_INVALID_ARG, "NULL argument");
  if (n_arch > 0 && (!arch_cols || !arch_offsets || !arch_bitmaps))
    return fail(EBIC_ERR_INVALID_ARG, "NULL archive argument");
  DeviceGuard g(m->device);
  const int dev = m->device;
  const Layout& L = m->L;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (const void* p : {(const void*)cols, (const void*)offsets, (const void*)counts,
                        (const void*)bitmaps, (const void*)arch_cols, (const void*)arch_offsets,
                        (const void*)arch_bitmaps, (const void*)fitness, (const void*)overlaps,
                        (const void*)arch_counts_out})
    if (foreign_device(p, dev)) return fail(EBIC_ERR_INVALID_ARG, "buffer on another device");

  const bool host_c = !on_device(cols, dev) && !on_device(offsets, dev);
  if (host_c) {
    std::string why = check_candidates_host(cols, offsets, n_cand, L.cols);
    if (!why.empty()) return fail(EBIC_ERR_INVALID_ARG, why);
  }
  const bool host_a = n_arch == 0 || (!on_device(arch_cols, dev) && !on_device(arch_offsets, dev));
  if (n_arch > 0 && host_a) {
    std::string why = check_candidates_host(arch_cols, arch_offsets, n_arch, L.cols);
    if (!why.empty()) return fail(EBIC_ERR_INVALID_ARG, "archive: " + why);
  }
  if ((!host_c && !on_device(cols, dev)) || (!host_c && !on_device(offsets, dev)) ||
      (n_arch > 0 && !host_a && (!on_device(arch_cols, dev) || !on_device(arch_offsets, dev))))
    return fail(EBIC_ERR_INVALID_ARG,
                "a candidate list must have its columns and offsets in the same memory");

  Scratch sc(s);
  uint32_t* err = nullptr;
  EBIC_CUDA(sc.alloc(reinterpret_cast<void**>(&err), sizeof(uint32_t)));
  EBIC_CUDA(cudaMemsetAsync(err, 0, sizeof(uint32_t), s));
  const uint16_t *dcols = nullptr, *dacols = nullptr;
  const uint32_t *doffs = nullptr, *daoffs = nullptr, *dcounts = nullptr, *dbm = nullptr,
                 *dabm = nullptr;
  EBIC_CUDA(to_device(offsets, (size_t)n_cand + 1, dev, sc, &doffs));
  EBIC_CUDA(to_device(cols, host_c ? (size_t)offsets[n_cand] : 0, dev, sc, &dcols));
  EBIC_CUDA(to_device(counts, n_cand, dev, sc, &dcounts));
  EBIC_CUDA(to_device(bitmaps, (size_t)n_cand * L.words, dev, sc, &dbm));
  if (n_arch > 0) {
    EBIC_CUDA(to_device(arch_offsets, (size_t)n_arch + 1, dev, sc, &daoffs));
    EBIC_CUDA(to_device(arch_cols, host_a ? (size_t)arch_offsets[n_arch] : 0, dev, sc, &dacols));
    EBIC_CUDA(to_device(arch_bitmaps, (size_t)n_arch * L.words, dev, sc, &dabm));
  }
  bool fit_host = false, ov_host = false;
  uint64_t* dfit = nullptr;
  uint32_t* dov = nullptr;
  EBIC_CUDA(out_buffer(fitness, n_cand, dev, sc, &dfit, &fit_host));
  const size_t n_ov = (size_t)n_cand * n_arch;
  uint32_t* darch_counts = nullptr;  // the archive members' row counts (computed on the device)
  if (n_arch > 0) {
    if (overlaps) {
      EBIC_CUDA(out_buffer(overlaps, n_ov, dev, sc, &dov, &ov_host));
    } else {
      EBIC_CUDA(sc.alloc(reinterpret_cast<void**>(&dov), n_ov * sizeof(uint32_t)));
    }
    EBIC_CUDA(sc.alloc(reinterpret_cast<void**>(&darch_counts), n_arch * sizeof(uint32_t)));
  }
  {
    Timed t(EBIC_TIMING_PREPARE, s);
    PrepareArgs pa;
    pa.cols[0] = dcols;
    pa.offsets[0] = doffs;
    pa.n[0] = host_c ? 0 : n_cand;
    pa.cols[1] = dacols;
    pa.offsets[1] = daoffs;
    pa.n[1] = host_a ? 0 : n_arch;
    pa.ncols = L.cols;
    pa.zero = dov;
    pa.n_zero = n_ov;
    pa.zero2 = darch_counts;
    pa.n_zero2 = darch_counts ? n_arch : 0;
    pa.err = err;
    pa.status = m->status;
    EBIC_CUDA(launch_prepare(pa, s));
  }
  {
    Timed t(EBIC_TIMING_OVERLAP, s);
    EBIC_CUDA(launch_overlap(dbm, n_cand, dabm, n_arch, L.words, dov, darch_counts, err,
                             m->num_sms, s));
  }
  {
    Timed t(EBIC_TIMING_FITNESS, s);
    EBIC_CUDA(launch_fitness_finalize(dcols, doffs, n_cand, dcounts, dacols, daoffs, n_arch, dov,
                                      darch_counts, dfit, err, s));
  }
  const bool ac_host = arch_counts_out && n_arch > 0 && !on_device(arch_counts_out, dev);
  if (arch_counts_out && n_arch > 0)
    EBIC_CUDA(cudaMemcpyAsync(arch_counts_out, darch_counts, (size_t)n_arch * 4,
                              ac_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
  if (fit_host || ov_host || ac_host) {
    if (fit_host)
      EBIC_CUDA(cudaMemcpyAsync(fitness, dfit, (size_t)n_cand * 8, cudaMemcpyDeviceToHost, s));
    if (ov_host)
      EBIC_CUDA(cudaMemcpyAsync(overlaps, dov, n_ov * 4, cudaMemcpyDeviceToHost, s));
    uint32_t bits = 0;
    EBIC_CUDA(cudaMemcpyAsync(&bits, err, 4, cudaMemcpyDeviceToHost, s));
    EBIC_CUDA(cudaStreamSynchronize(s));
    return status_code(bits, "ebic_fitness");
  }
  return EBIC_OK;
}

extern "C" int ebic_fitness(const ebic_matrix* cm, const uint16_t* cols, const uint32_t* offsets,
                            uint32_t n_cand, const uint32_t* counts, const uint32_t* bitmaps,
                            const uint16_t* arch_cols, const uint32_t* arch_offsets,
                            const uint32_t* arch_bitmaps, uint32_t n_arch, uint32_t flags,
                            uint64_t* fitness, uint32_t* overlaps, void* stream) {
  return fitness_impl(cm, cols, offsets, n_cand, counts, bitmaps, arch_cols, arch_offsets,
                      arch_bitmaps, n_arch, flags, fitness, overlaps, nullptr, stream);
}

// The fused route's outputs: the caller's overlaps from the paired layout, host copies, and
// (when an output is on the host, so the call synchronizes) the call's error word.
// `sync`: an output is on the host, so the call waits for the device and reports its error
// word, which the finalize kernel mirrored into `err_mirror` (host) when it is not null;
// counts_host / fit_host: those outputs still need a copy.
static int finish_fitness(uint32_t n_cand, uint32_t n_arch, uint32_t ov_stride,
                          uint32_t* dcounts, uint32_t* dbm, uint64_t* dfit, uint32_t* dov,
                          uint32_t* err, uint32_t* counts, uint32_t* bitmaps, uint64_t* fitness,
                          uint32_t* overlaps, bool counts_host, bool bm_host, bool fit_host,
                          int64_t words, bool ov_dev, bool sync,
                          const volatile uint32_t* err_mirror, cudaStream_t s) {
  const bool ov_host = overlaps && n_arch > 0 && !ov_dev;
  if (overlaps && n_arch > 0)  // the caller's [n_cand][n_arch] from the paired layout
    EBIC_CUDA(cudaMemcpy2DAsync(overlaps, (size_t)n_arch * 4, dov, (size_t)ov_stride * 4,
                                (size_t)n_arch * 4, n_cand,
                                ov_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
  if (sync && err_mirror && !counts_host && !bm_host && !fit_host && !ov_host) {
    EBIC_CUDA(cudaStreamSynchronize(s));
    return status_code(*err_mirror, "ebic_eval_fitness");
  }
  if (sync || counts_host || bm_host || fit_host || ov_host) {
    if (counts_host)
      EBIC_CUDA(cudaMemcpyAsync(counts, dcounts, (size_t)n_cand * 4, cudaMemcpyDeviceToHost, s));
    if (bm_host)
      EBIC_CUDA(cudaMemcpyAsync(bitmaps, dbm, (size_t)n_cand * words * 4,
                                cudaMemcpyDeviceToHost, s));
    if (fit_host)
      EBIC_CUDA(cudaMemcpyAsync(fitness, dfit, (size_t)n_cand * 8, cudaMemcpyDeviceToHost, s));
    uint32_t bits = 0;
    EBIC_CUDA(cudaMemcpyAsync(&bits, err, 4, cudaMemcpyDeviceToHost, s));
    EBIC_CUDA(cudaStreamSynchronize(s));
    return status_code(bits, "ebic_eval_fitness");
  }
  return EBIC_OK;
}


// ebic_eval_fitness, and also the archive members' row counts into `arch_counts_out` (when not
// null). `sharing_only`: with `overlaps` asked for, the fused route may skip the members that
// share no column with a candidate (their entries are then 0); the other route computes them.
static int eval_fitness_impl(const ebic_matrix* cm, const uint16_t* cols, const uint32_t* offsets,
                             uint32_t n_cand, uint32_t flags, const uint16_t* arch_cols,
                             const uint32_t* arch_offsets, const uint32_t* arch_bitmaps,
                             uint32_t n_arch, uint32_t* counts, uint32_t* bitmaps,
                             uint64_t* fitness, uint32_t* overlaps, uint32_t* arch_counts_out,
                             bool sharing_only, void* stream) {
  ebic_matrix* m = const_cast<ebic_matrix*>(cm);
  if (!m) return fail(EBIC_ERR_INVALID_ARG, "matrix is NULL");
  if (flags & ~(EBIC_NEGATIVE_TRENDS | EBIC_EVAL_DIRECT))
    return fail(EBIC_ERR_INVALID_ARG, "unknown eval flag");
  if (n_cand == 0) return EBIC_OK;
  if (!cols || !offsets || !counts || !fitness) return fail(EBIC_ERR_INVALID_ARG, "NULL argument");
  if (n_arch > 0 && (!arch_cols || !arch_offsets || !arch_bitmaps))
    return fail(EBIC_ERR_INVALID_ARG, "NULL archive argument");
  DeviceGuard g(m->device);
  const int dev = m->device;
  const Layout& L = m->L;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // each pointer's placement, queried once
  const Where w_cols = where(cols, dev), w_offs = where(offsets, dev), w_cnt = where(counts, dev),
              w_bm = where(bitmaps, dev), w_acols = where(arch_cols, dev),
              w_aoffs = where(arch_offsets, dev), w_abm = where(arch_bitmaps, dev),
              w_fit = where(fitness, dev), w_ov = where(overlaps, dev),
              w_ac = where(arch_counts_out, dev);
  for (const Where& w : {w_cols, w_offs, w_cnt, w_bm, w_acols, w_aoffs, w_abm, w_fit, w_ov, w_ac})
    if (w.foreign) return fail(EBIC_ERR_INVALID_ARG, "buffer on another device");

  const bool fused = m->pairs && !(flags & EBIC_EVAL_DIRECT) && n_arch <= (uint32_t)kPairMaxArch;
  if (!fused) {
    // the two calls in sequence; the bitmaps go through scratch when the caller wants none
    Scratch sc(s);
    uint32_t* bm = bitmaps;
    if (!bm) EBIC_CUDA(sc.alloc(reinterpret_cast<void**>(&bm), (size_t)n_cand * L.words * 4));
    int rc = ebic_eval_population(m, cols, offsets, n_cand, flags, counts, bm, stream);
    if (rc != EBIC_OK) return rc;
    return fitness_impl(m, cols, offsets, n_cand, counts, bm, arch_cols, arch_offsets,
                        arch_bitmaps, n_arch, 0, fitness, overlaps, arch_counts_out, stream);
  }

  const bool host_c = !w_cols.dev && !w_offs.dev;
  const bool host_a = n_arch == 0 || (!w_acols.dev && !w_aoffs.dev);
  if ((!host_c && (!w_cols.dev || !w_offs.dev)) ||
      (n_arch > 0 && !host_a && (!w_acols.dev || !w_aoffs.dev)))
    return fail(EBIC_ERR_INVALID_ARG,
                "a candidate list must have its columns and offsets in the same memory");
  // host lists: the offsets (they bound what the copies read) before any launch, the columns
  // while the kernels run (the device preparation checks them as well, without recording a
  // deferred status for a host list, so a bad host list leaves every kernel a no-op and the call
  // returns the host check's verdict)
  if (host_c) {
    std::string why = check_offsets_host(offsets, n_cand);
    if (!why.empty()) return fail(EBIC_ERR_INVALID_ARG, why);
  }
  if (n_arch > 0 && host_a) {
    std::string why = check_offsets_host(arch_offsets, n_arch);
    if (!why.empty()) return fail(EBIC_ERR_INVALID_ARG, "archive: " + why);
  }
  auto deferred_host_check = [&]() -> int {
    if (host_c) {
      std::string why = check_columns_host(cols, offsets, n_cand, L.cols);
      if (!why.empty()) return fail(EBIC_ERR_INVALID_ARG, why);
    }
    if (n_arch > 0 && host_a) {
      std::string why = check_columns_host(arch_cols, arch_offsets, n_arch, L.cols);
      if (!why.empty()) return fail(EBIC_ERR_INVALID_ARG, "archive: " + why);
    }
    return EBIC_OK;
  };

  Scratch sc(s);
  const uint16_t *dcols = nullptr, *dacols = nullptr;
  const uint32_t *doffs = nullptr, *daoffs = nullptr, *dabm = nullptr;
  // pinned host inputs are read in place by the kernels (over the host link), other host inputs
  // are copied
  EBIC_CUDA(input_at(offsets, (size_t)n_cand + 1, w_offs, sc, &doffs));
  EBIC_CUDA(input_at(cols, host_c ? (size_t)offsets[n_cand] : 0, w_cols, sc, &dcols));
  if (n_arch > 0) {
    EBIC_CUDA(input_at(arch_offsets, (size_t)n_arch + 1, w_aoffs, sc, &daoffs));
    EBIC_CUDA(input_at(arch_cols, host_a ? (size_t)arch_offsets[n_arch] : 0, w_acols, sc,
                       &dacols));
    EBIC_CUDA(input_at(arch_bitmaps, (size_t)n_arch * L.words, w_abm, sc, &dabm));
  }
  // outputs: pinned host counts are written by the finalize kernel from the device accumulator,
  // pinned host fitness in place; other host outputs go through scratch and a copy
  bool counts_host = false, bm_host = false, fit_host = false;
  uint32_t *dcounts = nullptr, *dbm = nullptr, *counts_mirror = nullptr;
  uint64_t* dfit = nullptr;
  if (!w_cnt.dev && w_cnt.mapped) {
    EBIC_CUDA(sc.alloc(reinterpret_cast<void**>(&dcounts), (size_t)n_cand * 4));
    counts_mirror = static_cast<uint32_t*>(w_cnt.mapped);
  } else {
    EBIC_CUDA(out_buffer_at(counts, n_cand, w_cnt.dev, sc, &dcounts, &counts_host));
  }
  if (bitmaps)
    EBIC_CUDA(out_buffer_at(bitmaps, (size_t)n_cand * L.words, w_bm.dev, sc, &dbm, &bm_host));
  if (!w_fit.dev && w_fit.mapped)
    dfit = static_cast<uint64_t*>(w_fit.mapped);
  else
    EBIC_CUDA(out_buffer_at(fitness, n_cand, w_fit.dev, sc, &dfit, &fit_host));
  // an output on the host: the call waits for the device and reports its error word, mirrored to
  // the host by the finalize kernel
  const bool sync = !w_cnt.dev || !w_fit.dev || (bitmaps && !w_bm.dev) ||
                    (overlaps && n_arch > 0 && !w_ov.dev) ||
                    (arch_counts_out && n_arch > 0 && !w_ac.dev);
  uint32_t* err_mirror = sync ? t_err_word.get() : nullptr;

  const bool neg = (flags & EBIC_NEGATIVE_TRENDS) != 0;
  // overlaps are accumulated in pairs of adjacent counters: rows of an even number of members
  const uint32_t ov_stride = (n_arch + 1u) & ~1u;
  const uint32_t stride = m->pair_stride;
  size_t total = 0;
  auto carve = [&total](size_t bytes) {
    const size_t off = total;
    total += (bytes + 255) & ~(size_t)255;
    return off;
  };
  // the call's working buffers, carved from one stream-ordered allocation; none needs zeroing
  // before the preparation kernel (it writes every word the later kernels read)
  const uint32_t prep_blocks = fused_prepare_blocks(n_cand, n_arch, stride, m->num_sms);
  const size_t o_err = carve(sizeof(uint32_t));
  const size_t o_flags = carve((size_t)prep_blocks * 4);
  const size_t o_terms = carve((size_t)n_cand * term_slots(neg) * 4);
  const size_t o_ov = carve(n_arch ? (size_t)n_cand * ov_stride * 4 : 0);
  const size_t o_pad = carve(n_arch ? (size_t)ov_stride * stride * 4 : 0);
  const size_t o_acnt = carve((size_t)n_arch * 4);
  const size_t o_share = carve(n_arch ? (size_t)n_cand * 8 : 0);
  char* work = nullptr;
  EBIC_CUDA(sc.alloc(reinterpret_cast<void**>(&work), total));
  uint32_t* err = reinterpret_cast<uint32_t*>(work + o_err);
  uint32_t* dflags = reinterpret_cast<uint32_t*>(work + o_flags);
  uint32_t* dterms = reinterpret_cast<uint32_t*>(work + o_terms);
  uint32_t* dov = n_arch ? reinterpret_cast<uint32_t*>(work + o_ov) : nullptr;
  uint32_t* dpad = n_arch ? reinterpret_cast<uint32_t*>(work + o_pad) : nullptr;
  uint32_t* darch_counts = n_arch ? reinterpret_cast<uint32_t*>(work + o_acnt) : nullptr;
  uint64_t* dshare = n_arch ? reinterpret_cast<uint64_t*>(work + o_share) : nullptr;
  {
    Timed t(EBIC_TIMING_PREPARE, s);
    FusedPrepareArgs pa;
    pa.cols = dcols;
    pa.offsets = doffs;
    pa.n_cand = n_cand;
    pa.acols = dacols;
    pa.aoffsets = daoffs;
    pa.n_arch = n_arch;
    pa.check_arch = !host_a;
    pa.ncols = L.cols;
    pa.W = L.words;
    pa.stride = stride;
    pa.arch_src = dabm;
    pa.arch_pad = dpad;
    pa.counts = dcounts;
    pa.overlaps = dov;
    pa.ov_stride = ov_stride;
    pa.arch_counts = darch_counts;
    pa.share = dshare;
    pa.terms = dterms;
    pa.negative = neg;
    pa.flags = dflags;
    pa.status_cand = host_c ? nullptr : m->status;  // host lists: the host check reports
    pa.status_arch = host_a ? nullptr : m->status;
    pa.table = m->pairs;
    EBIC_CUDA(launch_fused_prepare(pa, prep_blocks, s));
  }
  {
    Timed t(EBIC_TIMING_PAIR_EVALUATE, s);
    PairArgs p;
    p.table = m->pairs;
    p.stride = stride;
    p.C = L.cols;
    p.W = L.words;
    p.terms = dterms;
    p.n_cand = n_cand;
    p.counts = dcounts;
    p.bitmaps = dbm;
    p.arch = n_arch > 0 ? dpad : nullptr;
    p.n_arch = n_arch;
    // all members only when the caller reads all their overlaps
    p.score = overlaps && !sharing_only ? nullptr : dshare;
    p.overlaps = dov;
    p.ov_stride = ov_stride;
    p.arch_counts = darch_counts;
    p.flags = dflags;
    p.n_flags = prep_blocks;
    p.err_out = err;  // CTA 0 stores the OR of the flags here for the finalize and the host
    p.status = m->status;
    EBIC_CUDA(launch_pair_eval(p, neg, m->num_sms, !timing_on(), s));
  }
  {
    Timed t(EBIC_TIMING_FITNESS, s);
    EBIC_CUDA(launch_fused_finalize(doffs, n_cand, dcounts, daoffs, n_arch, dov, ov_stride,
                                    darch_counts, dshare, dfit, err, counts_mirror, err_mirror,
                                    !timing_on(), s));
  }
  const int hc = deferred_host_check();
  if (hc != EBIC_OK) {
    // the kernels (no-ops on these lists) may still write the caller's pinned outputs and this
    // thread's error word: let them finish first
    if (sync) (void)cudaStreamSynchronize(s);
    return hc;
  }
  // the archive members' counts (a host destination makes the call synchronous above, so the
  // synchronisation in finish_fitness also covers this copy)
  if (arch_counts_out && n_arch > 0)
    EBIC_CUDA(cudaMemcpyAsync(arch_counts_out, darch_counts, (size_t)n_arch * 4,
                              w_ac.dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  return finish_fitness(n_cand, n_arch, ov_stride, dcounts, dbm, dfit, dov, err, counts,
                        bitmaps, fitness, overlaps, counts_host, bm_host, fit_host, L.words,
                        w_ov.dev, sync, err_mirror ? t_err_word.host : nullptr, s);
}

extern "C" {

int ebic_eval_fitness(const ebic_matrix* cm, const uint16_t* cols, const uint32_t* offsets,
                      uint32_t n_cand, uint32_t flags, const uint16_t* arch_cols,
                      const uint32_t* arch_offsets, const uint32_t* arch_bitmaps,
                      uint32_t n_arch, uint32_t* counts, uint32_t* bitmaps, uint64_t* fitness,
                      uint32_t* overlaps, void* stream) {
  return eval_fitness_impl(cm, cols, offsets, n_cand, flags, arch_cols, arch_offsets,
                           arch_bitmaps, n_arch, counts, bitmaps, fitness, overlaps, nullptr,
                           false, stream);
}

int ebic_matrix_status(ebic_matrix* m, void* stream) {
  if (!m) return fail(EBIC_ERR_INVALID_ARG, "matrix is NULL");
  DeviceGuard g(m->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint32_t bits = 0;
  EBIC_CUDA(cudaStreamSynchronize(s));
  EBIC_CUDA(cudaMemcpy(&bits, m->status, 4, cudaMemcpyDeviceToHost));
  EBIC_CUDA(cudaMemset(m->status, 0, 4));
  return status_code(bits, "deferred device status");
}

int ebic_copy_async(void* dst, const void* src, size_t bytes, void* stream) {
  if (bytes == 0) return EBIC_OK;
  if (!dst || !src) return fail(EBIC_ERR_INVALID_ARG, "copy: NULL buffer");
  EBIC_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault,
                            static_cast<cudaStream_t>(stream)));
  return EBIC_OK;
}

int64_t ebic_launch_count(void) { return g_launches.load(); }

int ebic_timing_enable(int on) {
  std::lock_guard<std::mutex> lk(g_timing_mu);
  for (auto& v : g_timed)
    for (auto& pr : v) {
      g_event_pool.push_back(pr.first);
      g_event_pool.push_back(pr.second);
    }
  for (auto& v : g_timed) v.clear();
  g_timing.store(on != 0);
  return EBIC_OK;
}

int ebic_timing_read(int kind, double* total_ms, int64_t* launches) {
  if (kind < 0 || kind >= EBIC_TIMING_KINDS || !total_ms || !launches)
    return fail(EBIC_ERR_INVALID_ARG, "bad timing kind or NULL output");
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> v;
  {
    std::lock_guard<std::mutex> lk(g_timing_mu);
    v = g_timed[kind];
  }
  double tot = 0;
  for (auto& pr : v) {
    EBIC_CUDA(cudaEventSynchronize(pr.second));
    float ms = 0;
    EBIC_CUDA(cudaEventElapsedTime(&ms, pr.first, pr.second));
    tot += ms;
  }
  *total_ms = tot;
  *launches = (int64_t)v.size();
  return EBIC_OK;
}

int ebic_matrix_set_tile(ebic_matrix* m, int32_t tile_slabs) {
  if (!m) return fail(EBIC_ERR_INVALID_ARG, "matrix is NULL");
  if (tile_slabs != 0 && tile_slabs != 1 && tile_slabs != 2 && tile_slabs != 4)
    return fail(EBIC_ERR_INVALID_ARG, "tile_slabs must be 0, 1, 2 or 4");
  if (tile_slabs != 0) {
    int nb = (m->L.cols + 255) / 256, cb = (m->L.cols + nb - 1) / nb;
    if ((int64_t)nb * cb * tile_slabs * 128 * m->L.vec > kStageMax)
      return fail(EBIC_ERR_UNSUPPORTED, "tile does not fit in shared memory for this matrix");
  }
  m->tile = tile_slabs;
  return EBIC_OK;
}

int ebic_matrix_build_pairs(ebic_matrix* m, uint64_t max_bytes, void* stream, uint64_t* bytes) {
  if (!m) return fail(EBIC_ERR_INVALID_ARG, "matrix is NULL");
  const Layout& L = m->L;
  const int64_t stride = pair_stride(L.words);
  const uint64_t rows = (uint64_t)L.cols * (uint64_t)L.cols * (uint64_t)stride * 4ull;
  const uint64_t need = rows + (uint64_t)kOnesWords * 4ull;
  if (bytes) *bytes = need;
  if (need > max_bytes)
    return fail(EBIC_ERR_UNSUPPORTED, "the pair table needs " + std::to_string(need) +
                                          " bytes, more than max_bytes");
  if (rows / 4ull > 0xFFFFFFFFull)  // table rows are addressed with 32-bit word offsets
    return fail(EBIC_ERR_UNSUPPORTED, "the pair table would exceed 2^32 words");
  DeviceGuard g(m->device);
  if (m->pairs) return EBIC_OK;
  // the population of all ordered pairs (a, b), a != b, and of all singles (a), in table order
  const uint32_t C = (uint32_t)L.cols, n = C * C;
  std::vector<uint16_t> cols;
  std::vector<uint32_t> offs(1, 0u);
  cols.reserve((size_t)2 * n);
  for (uint32_t a = 0; a < C; ++a)
    for (uint32_t b = 0; b < C; ++b) {
      cols.push_back((uint16_t)a);
      if (b != a) cols.push_back((uint16_t)b);
      offs.push_back((uint32_t)cols.size());
    }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint32_t* table = nullptr;
  uint32_t* counts = nullptr;
  cudaError_t e = cudaMalloc(&table, need);
  if (e == cudaSuccess) e = cudaMalloc(&counts, (size_t)n * 4);
  if (e == cudaSuccess) e = cudaMemsetAsync(table, 0, rows, s);  // the rows' padding words
  if (e == cudaSuccess)  // the all-ones row after the table
    e = cudaMemsetAsync(reinterpret_cast<char*>(table) + rows, 0xFF, (size_t)kOnesWords * 4, s);
  if (e != cudaSuccess) {
    if (table) cudaFree(table);
    if (counts) cudaFree(counts);
    return cuda_fail(e, "pair table allocation");
  }
  int rc = eval_population_impl(m, cols.data(), offs.data(), n, EBIC_EVAL_DIRECT, counts, table,
                                stride, stream);
  cudaError_t e2 = cudaStreamSynchronize(s);
  cudaFree(counts);
  if (rc == EBIC_OK && e2 != cudaSuccess) rc = cuda_fail(e2, "pair table build");
  if (rc != EBIC_OK) {
    cudaFree(table);
    return rc;
  }
  m->pairs = table;
  m->pair_stride = (uint32_t)stride;
  m->pair_bytes = need;
  return EBIC_OK;
}

int ebic_matrix_drop_pairs(ebic_matrix* m) {
  if (!m) return fail(EBIC_ERR_INVALID_ARG, "matrix is NULL");
  if (m->pairs) {
    DeviceGuard g(m->device);
    EBIC_CUDA(cudaFree(m->pairs));
    m->pairs = nullptr;
    m->pair_stride = 0;
    m->pair_bytes = 0;
  }
  return EBIC_OK;
}

int ebic_matrix_set_chunk_cols(ebic_matrix* m, int32_t chunk_cols) {
  if (!m) return fail(EBIC_ERR_INVALID_ARG, "matrix is NULL");
  if (chunk_cols < 0 || chunk_cols > kMaxChunkCols)
    return fail(EBIC_ERR_INVALID_ARG, "chunk_cols must be in [0, 16384]");
  m->chunk = chunk_cols;
  return EBIC_OK;
}

int ebic_matrix_get_tile(const ebic_matrix* m, int32_t* tile_slabs, int32_t* rows_per_slab) {
  if (!m) return fail(EBIC_ERR_INVALID_ARG, "matrix is NULL");
  int ts = m->tile ? m->tile : default_tile_slabs(m->L);
  while (ts > 1 && ts > m->L.slabs) ts >>= 1;
  if (tile_slabs) *tile_slabs = ts;
  if (rows_per_slab) *rows_per_slab = (int32_t)m->L.rows_per_slab();
  return EBIC_OK;
}


// ---- row shards (the paper's multi-GPU layout: rows spread over GPUs, Methods, "Support for Big
// Data"; Abstract) ------------------------------------------------------------------------------

int ebic_load_matrix_shard(const float* x, int64_t rows, int32_t cols, int64_t ld,
                           int64_t row_offset, int64_t total_rows, uint32_t flags,
                           float fill_value, void* stream, ebic_matrix** out) {
  if (!out) return fail(EBIC_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (total_rows < 1 || total_rows > 2147483647LL)
    return fail(EBIC_ERR_INVALID_ARG, "total_rows must be in [1, 2^31-1]");
  if (row_offset < 0 || row_offset % 32 != 0)
    return fail(EBIC_ERR_INVALID_ARG, "row_offset must be a non-negative multiple of 32");
  if (rows < 1 || row_offset + rows > total_rows)
    return fail(EBIC_ERR_INVALID_ARG, "the shard must lie inside the whole matrix");
  if (row_offset + rows != total_rows && rows % 32 != 0)
    return fail(EBIC_ERR_INVALID_ARG,
                "a shard that does not end the matrix must hold a multiple of 32 rows");
  int rc = ebic_load_matrix(x, rows, cols, ld, flags, fill_value, stream, out);
  if (rc != EBIC_OK) return rc;
  (*out)->row_offset = row_offset;
  (*out)->total_rows = total_rows;
  return EBIC_OK;
}

int ebic_matrix_shard(const ebic_matrix* m, int64_t* row_offset, int64_t* total_rows,
                      int64_t* word_offset) {
  if (!m) return fail(EBIC_ERR_INVALID_ARG, "matrix is NULL");
  if (row_offset) *row_offset = m->row_offset;
  if (total_rows) *total_rows = m->total_rows;
  if (word_offset) *word_offset = m->row_offset / 32;
  return EBIC_OK;
}

int ebic_eval_partials(const ebic_matrix* m, const uint16_t* cols, const uint32_t* offsets,
                       uint32_t n_cand, uint32_t flags, const uint16_t* arch_cols,
                       const uint32_t* arch_offsets, const uint32_t* arch_bitmaps,
                       uint32_t n_arch, uint32_t* counts, uint32_t* overlaps,
                       uint32_t* arch_counts, uint32_t* bitmaps, void* stream) {
  if (!m) return fail(EBIC_ERR_INVALID_ARG, "matrix is NULL");
  if (n_cand == 0) return EBIC_OK;
  if (n_arch > 0 && (!overlaps || !arch_counts))
    return fail(EBIC_ERR_INVALID_ARG, "overlaps and arch_counts are needed with an archive");
  DeviceGuard g(m->device);
  // the shard's own fitness is of no use before the sum: it goes to scratch
  Scratch sc(static_cast<cudaStream_t>(stream));
  uint64_t* fit = nullptr;
  EBIC_CUDA(sc.alloc(reinterpret_cast<void**>(&fit), (size_t)n_cand * 8));
  return eval_fitness_impl(m, cols, offsets, n_cand, flags, arch_cols, arch_offsets,
                           arch_bitmaps, n_arch, counts, bitmaps, fit,
                           n_arch ? overlaps : nullptr, n_arch ? arch_counts : nullptr, true,
                           stream);
}

int ebic_fitness_reduced(const ebic_matrix* cm, const uint16_t* cols, const uint32_t* offsets,
                         uint32_t n_cand, const uint32_t* counts, const uint32_t* overlaps,
                         const uint16_t* arch_cols, const uint32_t* arch_offsets,
                         const uint32_t* arch_counts, uint32_t n_arch, uint32_t flags,
                         uint64_t* fitness, void* stream) {
  ebic_matrix* m = const_cast<ebic_matrix*>(cm);
  if (!m) return fail(EBIC_ERR_INVALID_ARG, "matrix is NULL");
  if (flags != 0) return fail(EBIC_ERR_INVALID_ARG, "flags is reserved (pass 0)");
  if (n_cand == 0) return EBIC_OK;
  if (!cols || !offsets || !counts || !fitness) return fail(EBIC_ERR_INVALID_ARG, "NULL argument");
  if (n_arch > 0 && (!arch_cols || !arch_offsets || !arch_counts || !overlaps))
    return fail(EBIC_ERR_INVALID_ARG, "NULL archive argument");
  DeviceGuard g(m->device);
  const int dev = m->device;
  const Layout& L = m->L;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (const void* p : {(const void*)cols, (const void*)offsets, (const void*)counts,
                        (const void*)overlaps, (const void*)arch_cols, (const void*)arch_offsets,
                        (const void*)arch_counts, (const void*)fitness})
    if (foreign_device(p, dev)) return fail(EBIC_ERR_INVALID_ARG, "buffer on another device");
  const bool host_c = !on_device(cols, dev) && !on_device(offsets, dev);
  if (!host_c && (!on_device(cols, dev) || !on_device(offsets, dev)))
    return fail(EBIC_ERR_INVALID_ARG,
                "a candidate list must have its columns and offsets in the same memory");
  if (host_c) {
    std::string why = check_candidates_host(cols, offsets, n_cand, L.cols);
    if (!why.empty()) return fail(EBIC_ERR_INVALID_ARG, why);
  }
  const bool host_a = n_arch == 0 || (!on_device(arch_cols, dev) && !on_device(arch_offsets, dev));
  if (n_arch > 0 && !host_a && (!on_device(arch_cols, dev) || !on_device(arch_offsets, dev)))
    return fail(EBIC_ERR_INVALID_ARG,
                "a candidate list must have its columns and offsets in the same memory");
  if (n_arch > 0 && host_a) {
    std::string why = check_candidates_host(arch_cols, arch_offsets, n_arch, L.cols);
    if (!why.empty()) return fail(EBIC_ERR_INVALID_ARG, "archive: " + why);
  }
  Scratch sc(s);
  uint32_t* err = nullptr;
  EBIC_CUDA(sc.alloc(reinterpret_cast<void**>(&err), sizeof(uint32_t)));
  EBIC_CUDA(cudaMemsetAsync(err, 0, sizeof(uint32_t), s));
  const uint16_t *dcols = nullptr, *dacols = nullptr;
  const uint32_t *doffs = nullptr, *daoffs = nullptr, *dcounts = nullptr, *dov = nullptr,
                 *dacnt = nullptr;
  EBIC_CUDA(to_device(offsets, (size_t)n_cand + 1, dev, sc, &doffs));
  EBIC_CUDA(to_device(cols, host_c ? (size_t)offsets[n_cand] : 0, dev, sc, &dcols));
  EBIC_CUDA(to_device(counts, n_cand, dev, sc, &dcounts));
  if (n_arch > 0) {
    EBIC_CUDA(to_device(arch_offsets, (size_t)n_arch + 1, dev, sc, &daoffs));
    EBIC_CUDA(to_device(arch_cols, host_a ? (size_t)arch_offsets[n_arch] : 0, dev, sc, &dacols));
    EBIC_CUDA(to_device(arch_counts, n_arch, dev, sc, &dacnt));
    EBIC_CUDA(to_device(overlaps, (size_t)n_cand * n_arch, dev, sc, &dov));
  }
  bool fit_host = false;
  uint64_t* dfit = nullptr;
  EBIC_CUDA(out_buffer(fitness, n_cand, dev, sc, &dfit, &fit_host));
  {
    Timed t(EBIC_TIMING_PREPARE, s);
    PrepareArgs pa;  // device-resident lists are checked here; nothing to zero
    pa.cols[0] = dcols;
    pa.offsets[0] = doffs;
    pa.n[0] = host_c ? 0 : n_cand;
    pa.cols[1] = dacols;
    pa.offsets[1] = daoffs;
    pa.n[1] = host_a ? 0 : n_arch;
    pa.ncols = L.cols;
    pa.err = err;
    pa.status = m->status;
    EBIC_CUDA(launch_prepare(pa, s));
  }
  {
    Timed t(EBIC_TIMING_FITNESS, s);
    EBIC_CUDA(launch_fitness_finalize(dcols, doffs, n_cand, dcounts, dacols, daoffs, n_arch, dov,
                                      dacnt, dfit, err, s));
  }
  if (fit_host) {
    EBIC_CUDA(cudaMemcpyAsync(fitness, dfit, (size_t)n_cand * 8, cudaMemcpyDeviceToHost, s));
    uint32_t bits = 0;
    EBIC_CUDA(cudaMemcpyAsync(&bits, err, 4, cudaMemcpyDeviceToHost, s));
    EBIC_CUDA(cudaStreamSynchronize(s));
    return status_code(bits, "ebic_fitness_reduced");
  }
  return EBIC_OK;
}

}  // extern "C"
