// Internal definitions shared by the TT-IGA CUDA sources: context, device
// buffers, error propagation and small launch helpers.
#pragma once
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <map>
#include <memory>
#include <stdexcept>
#include <string>
#include <functional>
#include <vector>

#include "../../include/tt_iga.h"

namespace ttiga {

// An error carrying a tt_iga_status, thrown inside the library and turned
// into a return code at the C boundary.
struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string &m) : std::runtime_error(m), code(c) {}
};

[[noreturn]] inline void fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  throw Error(code, buf);
}

#define TTI_CUDA(call)                                                                       \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      ::ttiga::fail(e_ == cudaErrorMemoryAllocation ? TT_IGA_ERR_OOM : TT_IGA_ERR_CUDA,      \
                    "%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_));      \
  } while (0)

// Kernel launches issued by the library (process-wide), for launch accounting.
extern std::atomic<unsigned long long> g_launches;
// Contexts created by tt_iga_ctx_create and not yet destroyed (helpers not counted).
extern std::atomic<int> g_live_contexts;
#define TTI_LAUNCH()                                                 \
  do {                                                               \
    ::ttiga::g_launches.fetch_add(1, std::memory_order_relaxed);     \
    TTI_CUDA(cudaGetLastError());                                    \
  } while (0)

#define TTI_CHECK_ARG(cond, ...)                          \
  do {                                                    \
    if (!(cond)) ::ttiga::fail(TT_IGA_ERR_ARG, __VA_ARGS__); \
  } while (0)

struct Ctx;

// Stream-ordered device allocation owned by a context.
class DBuf {
 public:
  DBuf() = default;
  DBuf(Ctx *c, size_t bytes);
  ~DBuf() { release(); }
  DBuf(const DBuf &) = delete;
  DBuf &operator=(const DBuf &) = delete;
  DBuf(DBuf &&o) noexcept : ctx_(o.ctx_), p_(o.p_), bytes_(o.bytes_) { o.p_ = nullptr; o.bytes_ = 0; }
  DBuf &operator=(DBuf &&o) noexcept {
    if (this != &o) {
      release();
      ctx_ = o.ctx_; p_ = o.p_; bytes_ = o.bytes_;
      o.p_ = nullptr; o.bytes_ = 0;
    }
    return *this;
  }
  void release();
  // Hand the allocation to another context (same device): it is freed on that
  // context's stream.  The caller orders that stream after every use so far.
  void rehome(Ctx *to);
  void *get() const { return p_; }
  size_t bytes() const { return bytes_; }
  template <typename T> T *as() const { return static_cast<T *>(p_); }
  double *d() const { return static_cast<double *>(p_); }
  void *detach() { void *q = p_; p_ = nullptr; bytes_ = 0; return q; }

 private:
  Ctx *ctx_ = nullptr;
  void *p_ = nullptr;
  size_t bytes_ = 0;
};

struct Ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  void *(*alloc_fn)(size_t, void *, void *) = nullptr;
  void (*free_fn)(void *, void *, void *) = nullptr;
  void *alloc_user = nullptr;
  std::string last_error;
  size_t in_use = 0, peak = 0;
  int num_sms = 0;
  // SMs' worth of CTAs the context's cooperative kernels (the fused local PCG) may
  // take (0: the whole GPU), so that concurrent contexts share the GPU.
  int coop_sms = 0;
  // Run the independent parts of a call (coefficient fields, operator and loads) on helper
  // streams and host threads (run_concurrent).  Off for the lanes of a batch, whose contexts
  // already overlap: there the extra host threads compete for the CPU with the lanes.
  bool use_helpers = true;
  // small pinned host scratch for scalar read-backs
  void *pinned = nullptr;
  size_t pinned_bytes = 0;
  // device status word written by kernels that detect errors (0 = fine)
  int *dstatus = nullptr;
  // persistent device scratch for reductions (kScratchDoubles doubles)
  double *dscratch = nullptr;
  static constexpr int kScratchDoubles = 8192;

  // Helper contexts for independent work run concurrently (own stream and
  // scratch, the parent's status word); created on first use, see concurrent.cu.
  bool is_sub = false;
  std::vector<std::unique_ptr<Ctx>> subs;
  Ctx *sub(int i);
  void release_subs();
  // Host worker threads of run_concurrent, created on first use and kept for the
  // context's lifetime (a new thread's first CUDA call costs a few hundred microseconds).
  std::shared_ptr<struct WorkerPool> pool;

  // Live CUDA-event timing of one kernel family (0 = off), for roofline reporting.
  int prof_family = 0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_events;
  std::vector<double> prof_work;
  size_t prof_used = 0;

  void *alloc(size_t bytes) {
    if (bytes == 0) bytes = 16;
    void *p = nullptr;
    if (alloc_fn) {
      p = alloc_fn(bytes, stream, alloc_user);
      if (!p) fail(TT_IGA_ERR_OOM, "allocator callback failed for %zu bytes", bytes);
      if (reinterpret_cast<uintptr_t>(p) & 255) {
        free_fn(p, stream, alloc_user);
        fail(TT_IGA_ERR_ARG, "allocator callback returned a pointer that is not 256-byte aligned");
      }
    } else {
      cudaError_t e = cudaMallocAsync(&p, bytes, stream);
      if (e != cudaSuccess) fail(TT_IGA_ERR_OOM, "cudaMallocAsync(%zu): %s", bytes, cudaGetErrorString(e));
    }
    in_use += bytes;
    if (in_use > peak) peak = in_use;
    return p;
  }
  void free(void *p, size_t bytes) {
    if (!p) return;
    if (free_fn) free_fn(p, stream, alloc_user);
    else cudaFreeAsync(p, stream);
    in_use -= bytes;
  }
  void sync() { TTI_CUDA(cudaStreamSynchronize(stream)); }
  void *host_scratch(size_t bytes) {
    if (bytes > pinned_bytes) {
      if (pinned) cudaFreeHost(pinned);
      pinned = nullptr;
      TTI_CUDA(cudaMallocHost(&pinned, bytes));
      pinned_bytes = bytes;
    }
    return pinned;
  }
  // Copy device -> host synchronously.  Small read-backs (ranks, pivots, norms, singular
  // values: the host decisions of every call) go through the context's pinned scratch,
  // which a pageable destination would otherwise make the driver stage on every call.
  static constexpr size_t kPinnedSmall = 256 * 1024;
  void d2h(void *dst, const void *src, size_t bytes) {
    if (bytes <= kPinnedSmall) {
      void *h = host_scratch(kPinnedSmall);
      TTI_CUDA(cudaMemcpyAsync(h, src, bytes, cudaMemcpyDeviceToHost, stream));
      sync();
      memcpy(dst, h, bytes);
      return;
    }
    TTI_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, stream));
    sync();
  }
  void h2d(void *dst, const void *src, size_t bytes) {
    TTI_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, stream));
  }
  void zero(void *dst, size_t bytes) { TTI_CUDA(cudaMemsetAsync(dst, 0, bytes, stream)); }
};

inline DBuf::DBuf(Ctx *c, size_t bytes) : ctx_(c), p_(c->alloc(bytes)), bytes_(bytes ? bytes : 16) {}
inline void DBuf::rehome(Ctx *to) {
  if (!p_ || ctx_ == to) return;
  ctx_->in_use -= bytes_;
  to->in_use += bytes_;
  if (to->in_use > to->peak) to->peak = to->in_use;
  ctx_ = to;
}

// Run f(i, ctx_i) for i < n concurrently, each on its own helper context and
// host thread, ordered after the work already queued on c and before the work
// queued on c afterwards.  Sequential on c itself when n <= 1 or when c uses a
// caller-supplied allocator (whose streams the helpers must not touch).  The
// first exception of any task is rethrown after all have finished.
void run_concurrent(Ctx *c, int n, const std::function<void(int, Ctx *)> &f);

// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) once per (kernel, device), thread-safe.
void set_smem_limit_once(const void *kernel, int bytes);

inline void DBuf::release() {
  if (p_ && ctx_) ctx_->free(p_, bytes_);
  p_ = nullptr;
  bytes_ = 0;
}

// Kernel families that can be timed live (tt_iga_profile_enable).
enum ProfFamily { PROF_OFF = 0, PROF_LOCAL_BAND = 1, PROF_GEMM64 = 2, PROF_QR = 3, PROF_PRECOND = 4, PROF_CROSS = 5,
                  PROF_PCG_FUSED = 6 };

// Records a CUDA event pair around the launches in its scope when the
// context times this kernel family; `work` is the launch's algorithmic work
// (FLOPs or bytes, per family).
struct ProfScope {
  Ctx *c;
  long idx = -1;
  ProfScope(Ctx *c_, int family, double work) : c(c_) {
    if (c->prof_family != family) return;
    if (c->prof_used == c->prof_events.size()) {
      cudaEvent_t a, b;
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      c->prof_events.push_back({a, b});
    }
    idx = (long)c->prof_used++;
    c->prof_work.push_back(work);
    cudaEventRecord(c->prof_events[idx].first, c->stream);
  }
  ~ProfScope() {
    if (idx >= 0) cudaEventRecord(c->prof_events[idx].second, c->stream);
  }
};

// Set the work of the most recent timed launch of `family` (when the work is
// only known after the launch, e.g. an iteration count read back by the host).
inline void prof_set_last_work(Ctx *c, int family, double work) {
  if (c->prof_family == family && !c->prof_work.empty()) c->prof_work.back() = work;
}

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }
inline unsigned grid1d(long long n, int threads, int cap = 152 * 16) {
  long long g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (unsigned)g;
}

// Device status codes written by kernels into Ctx::dstatus.
enum DeviceStatus { DS_OK = 0, DS_BAD_GEOMETRY = 1, DS_NONFINITE = 2, DS_BOUNDS = 3, DS_BREAKDOWN = 4 };

// ----------------------------------------------------------------- TT types

// TT tensor of order 3 with cores [r_{k-1}][m_k][r_k] (FP64, device).
struct TT3 {
  int m[3] = {0, 0, 0};
  int r[4] = {1, 0, 0, 1};
  DBuf core[3];
  size_t core_elems(int k) const { return (size_t)r[k] * m[k] * r[k + 1]; }
  void alloc(Ctx *c) {
    for (int k = 0; k < 3; ++k) core[k] = DBuf(c, core_elems(k) * sizeof(double));
  }
};

}  // namespace ttiga

// Opaque handle definitions visible to every translation unit.
struct tt_iga_ctx : ttiga::Ctx {};
