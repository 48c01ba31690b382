// Concurrent execution of independent parts of one call (the six coefficient
// fields of the geometry, the operator and the load vectors of the assembly):
// each part runs on a host thread with a helper context of its own stream, so
// the host read-backs inside one part (ranks, pivots, validation maxima) no
// longer serialise the others.  Ordering with the parent stream uses events.
#include <exception>
#include <mutex>
#include <set>
#include <thread>
#include <utility>

#include "common.cuh"

namespace ttiga {

Ctx *Ctx::sub(int i) {
  while ((int)subs.size() <= i) {
    auto s = std::make_unique<Ctx>();
    s->device = device;
    s->num_sms = num_sms;
    s->coop_sms = coop_sms;
    s->use_helpers = use_helpers;
    s->is_sub = true;
    s->dstatus = dstatus;  // shared: kernels of every helper report into the parent's word
    TTI_CUDA(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
    s->own_stream = true;
    TTI_CUDA(cudaMalloc(&s->dscratch, Ctx::kScratchDoubles * sizeof(double)));
    subs.push_back(std::move(s));
  }
  return subs[i].get();
}

void Ctx::release_subs() {
  for (auto &s : subs) {
    s->release_subs();
    if (s->stream) cudaStreamSynchronize(s->stream);
    if (s->dscratch) cudaFree(s->dscratch);
    if (s->pinned) cudaFreeHost(s->pinned);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
  }
  subs.clear();
}

void run_concurrent(Ctx *c, int n, const std::function<void(int, Ctx *)> &f) {
  if (n <= 1 || c->alloc_fn || !c->use_helpers) {
    for (int i = 0; i < n; ++i) f(i, c);
    return;
  }
  std::vector<Ctx *> h(n);
  for (int i = 0; i < n; ++i) h[i] = c->sub(i);
  cudaEvent_t start;
  TTI_CUDA(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
  TTI_CUDA(cudaEventRecord(start, c->stream));
  for (int i = 0; i < n; ++i) TTI_CUDA(cudaStreamWaitEvent(h[i]->stream, start, 0));
  cudaEventDestroy(start);
  std::vector<std::exception_ptr> err(n);
  std::vector<std::thread> th;
  th.reserve(n);
  for (int i = 0; i < n; ++i)
    th.emplace_back([&, i] {
      try {
        TTI_CUDA(cudaSetDevice(c->device));
        f(i, h[i]);
      } catch (...) {
        err[i] = std::current_exception();
      }
    });
  for (auto &t : th) t.join();
  for (int i = 0; i < n; ++i) {
    cudaEvent_t done;
    TTI_CUDA(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
    TTI_CUDA(cudaEventRecord(done, h[i]->stream));
    TTI_CUDA(cudaStreamWaitEvent(c->stream, done, 0));
    cudaEventDestroy(done);
  }
  for (int i = 0; i < n; ++i)
    if (err[i]) std::rethrow_exception(err[i]);
}

void set_smem_limit_once(const void *kernel, int bytes) {
  static std::mutex mu;
  static std::set<std::pair<const void *, int>> done;
  int dev = 0;
  TTI_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  if (done.count({kernel, dev})) return;
  TTI_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  done.insert({kernel, dev});
}

}  // namespace ttiga
