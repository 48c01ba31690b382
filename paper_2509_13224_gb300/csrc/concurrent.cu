// Concurrent execution of independent parts of one call (the six coefficient
// fields of the geometry, the operator and the load vectors of the assembly):
// each part runs on a host thread with a helper context of its own stream, so
// the host read-backs inside one part (ranks, pivots, validation maxima) no
// longer serialise the others.  Ordering with the parent stream uses events.
#include <condition_variable>
#include <deque>
#include <exception>
#include <mutex>
#include <set>
#include <thread>
#include <utility>

#include "common.cuh"

namespace ttiga {

// Persistent host threads for run_concurrent: each sets the device once, then runs tasks
// from a queue until the pool is destroyed.
struct WorkerPool {
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<std::function<void()>> tasks;
  std::vector<std::thread> threads;
  bool stop = false;

  explicit WorkerPool(int dev) : device(dev) {}
  ~WorkerPool() {
    {
      std::lock_guard<std::mutex> lk(mu);
      stop = true;
    }
    cv.notify_all();
    for (auto &t : threads) t.join();
  }
  void ensure(int n) {
    while ((int)threads.size() < n)
      threads.emplace_back([this] {
        cudaSetDevice(device);
        for (;;) {
          std::function<void()> task;
          {
            std::unique_lock<std::mutex> lk(mu);
            cv.wait(lk, [this] { return stop || !tasks.empty(); });
            if (tasks.empty()) return;  // stop requested and nothing left
            task = std::move(tasks.front());
            tasks.pop_front();
          }
          task();
        }
      });
  }
  // Run the n tasks concurrently (the pool has at least n threads) and wait for all.
  void run(std::vector<std::function<void()>> &batch) {
    ensure((int)batch.size());
    std::mutex dmu;
    std::condition_variable dcv;
    int left = (int)batch.size();
    {
      std::lock_guard<std::mutex> lk(mu);
      for (auto &f : batch)
        tasks.emplace_back([&f, &dmu, &dcv, &left] {
          f();
          std::lock_guard<std::mutex> l2(dmu);
          if (--left == 0) dcv.notify_all();
        });
    }
    cv.notify_all();
    std::unique_lock<std::mutex> lk(dmu);
    dcv.wait(lk, [&] { return left == 0; });
  }
};

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
  pool.reset();  // joins the worker threads (no task is running: every run_concurrent waited for its own)
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
  std::vector<std::function<void()>> batch;
  batch.reserve(n);
  for (int i = 0; i < n; ++i)
    batch.emplace_back([&, i] {
      try {
        f(i, h[i]);
      } catch (...) {
        err[i] = std::current_exception();
      }
    });
  if (!c->pool) c->pool = std::make_shared<WorkerPool>(c->device);
  c->pool->run(batch);
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
