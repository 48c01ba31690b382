// Batched solves: many independent TT-IGA instances of uneven size and rank
// on one GPU.  A host work queue feeds `lanes` contexts, each with its own
// non-blocking stream and host thread, so the small kernels of different
// instances overlap on the device.  Instances are started largest first
// (by n1 n2 n3 times the number of right-hand sides) to shorten the tail.
// The right-hand sides of an instance are solved as one block-TT solve
// (tt_iga_solve_block) or one by one, as the item asks.
// Each instance's arithmetic is independent of the others: no cross-instance
// reductions or atomics, so a result is the same alone and in a batch.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <thread>
#include <vector>

#include "handles.cuh"

extern "C" {

int tt_iga_batch_solve(int device, int count, const tt_iga_batch_item *items, int lanes, tt_iga_batch_result *results,
                       double *wall_ms) {
  if (count < 0 || (count > 0 && (!items || !results)) || lanes < 1 || lanes > 64) return TT_IGA_ERR_ARG;
  for (int i = 0; i < count; ++i)
    if (items[i].n_rhs < 1 || items[i].n_rhs > 8 || !items[i].rhs ||
        (items[i].rhs_solve != TT_IGA_RHS_BLOCK && items[i].rhs_solve != TT_IGA_RHS_EACH))
      return TT_IGA_ERR_ARG;
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  auto cost = [&](int i) {
    const tt_iga_geom_desc &g = items[i].geom;
    return (double)g.n[0] * g.n[1] * g.n[2] * items[i].n_rhs;
  };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
  std::atomic<int> next{0};
  std::atomic<int> first_error{0};
  const auto t0 = std::chrono::steady_clock::now();
  auto worker = [&]() {
    if (cudaSetDevice(device) != cudaSuccess) {
      first_error.store(TT_IGA_ERR_CUDA);
      return;
    }
    tt_iga_ctx_opts o{};
    o.device = device;
    tt_iga_ctx *ctx = nullptr;
    int rc = tt_iga_ctx_create(&ctx, &o);
    if (rc != TT_IGA_OK) {
      first_error.store(rc);
      return;
    }
    for (;;) {
      const int slot = next.fetch_add(1);
      if (slot >= count) break;
      const int i = order[slot];
      const tt_iga_batch_item &it = items[i];
      tt_iga_batch_result &res = results[i];
      res = tt_iga_batch_result{};
      res.dofs = (long long)it.geom.n[0] * it.geom.n[1] * it.geom.n[2] * it.n_rhs;
      auto ta = std::chrono::steady_clock::now();
      tt_iga_geom *g = nullptr;
      tt_iga_system *s = nullptr;
      int st = tt_iga_geometry(ctx, &it.geom, &g);
      auto tb = std::chrono::steady_clock::now();
      if (st == TT_IGA_OK) st = tt_iga_assemble(ctx, g, it.rhs, it.n_rhs, it.round_tol, &s);
      auto tc = std::chrono::steady_clock::now();
      double worst = 0.0;
      if (st == TT_IGA_OK && it.n_rhs > 1 && it.rhs_solve == TT_IGA_RHS_BLOCK) {
        tt_iga_solution *us[8] = {};
        double rr[8];
        tt_iga_stats stats{};
        st = tt_iga_solve_block(ctx, s, &it.opts, -1, us, &stats, rr);
        for (int k = 0; k < it.n_rhs; ++k) {
          worst = (worst < 0.0 || rr[k] < 0.0) ? -1.0 : std::max(worst, rr[k]);
          tt_iga_solution_destroy(us[k]);
        }
        res.ranks[0] = stats.ranks[0];
        res.ranks[1] = stats.ranks[1];
        res.sweeps = stats.sweeps;
      }
      for (int k = 0; k < it.n_rhs && st == TT_IGA_OK && !(it.n_rhs > 1 && it.rhs_solve == TT_IGA_RHS_BLOCK); ++k) {
        tt_iga_solve_opts so = it.opts;
        so.rhs_index = k;
        tt_iga_solution *u = nullptr;
        tt_iga_stats stats{};
        st = tt_iga_solve(ctx, s, &so, &u, &stats);
        worst = std::max(worst, stats.rel_residual);
        res.ranks[0] = stats.ranks[0];
        res.ranks[1] = stats.ranks[1];
        res.sweeps += stats.sweeps;
        tt_iga_solution_destroy(u);
      }
      auto td = std::chrono::steady_clock::now();
      res.status = st;
      res.rel_residual_max = worst;
      res.ms_geometry = std::chrono::duration<double, std::milli>(tb - ta).count();
      res.ms_assemble = std::chrono::duration<double, std::milli>(tc - tb).count();
      res.ms_solve = std::chrono::duration<double, std::milli>(td - tc).count();
      res.t_start_ms = std::chrono::duration<double, std::milli>(ta - t0).count();
      res.t_end_ms = std::chrono::duration<double, std::milli>(td - t0).count();
      tt_iga_system_destroy(s);
      tt_iga_geom_destroy(g);
    }
    tt_iga_ctx_destroy(ctx);
  };
  std::vector<std::thread> pool;
  const int nl = std::min(lanes, std::max(1, count));
  for (int l = 0; l < nl; ++l) pool.emplace_back(worker);
  for (auto &t : pool) t.join();
  if (wall_ms) *wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (first_error.load() != 0) return first_error.load();
  for (int i = 0; i < count; ++i)
    if (results[i].status != TT_IGA_OK) return results[i].status;
  return TT_IGA_OK;
}

int tt_iga_batch_autotune(int device, int count, const tt_iga_batch_item *items, const int *candidates,
                          int n_candidates, tt_iga_batch_result *results, int *best_lanes, double *best_ms) {
  if (!candidates || n_candidates < 1 || !best_lanes) return TT_IGA_ERR_ARG;
  double best = 1e300;
  int pick = candidates[0];
  for (int c = 0; c < n_candidates; ++c) {
    double ms = 0.0;
    const int rc = tt_iga_batch_solve(device, count, items, candidates[c], results, &ms);
    if (rc != TT_IGA_OK && rc != TT_IGA_ERR_NOT_CONVERGED) return rc;
    if (ms < best) {
      best = ms;
      pick = candidates[c];
    }
  }
  *best_lanes = pick;
  if (best_ms) *best_ms = best;
  return TT_IGA_OK;
}

}  // extern "C"
