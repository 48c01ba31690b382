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

int tt_iga_batch_solve(int device, int count, const tt_iga_batch_item *items, int lanes, int sm_per_lane,
                       tt_iga_batch_result *results, double *wall_ms) {
  if (count < 0 || (count > 0 && (!items || !results)) || lanes < 1 || lanes > 64 || sm_per_lane < -1)
    return TT_IGA_ERR_ARG;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return TT_IGA_ERR_CUDA;
  // -1: an equal share of the SMs per lane, so the lanes' cooperative PCG kernels fit side by side.
  // The share follows from `lanes` alone (not from how many instances there are), so an instance
  // gets the same grids, and the same bits, alone and in a batch run with the same lanes.
  const int share = sm_per_lane == -1 ? (lanes > 1 ? std::max(1, sms / lanes) : 0) : sm_per_lane;
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
    if (rc == TT_IGA_OK) rc = tt_iga_ctx_set_sm_limit(ctx, share);
    // the lanes overlap each other; helper threads inside a lane would only compete with them
    if (rc == TT_IGA_OK && lanes > 1) ctx->use_helpers = false;
    if (rc != TT_IGA_OK) {
      first_error.store(rc);
      if (ctx) tt_iga_ctx_destroy(ctx);
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
      size_t cores_off = 0;
      // the solution cores of right-hand side k, back to back, when the item asks for them
      auto keep_cores = [&](int k, const tt_iga_solution *u) {
        if (!it.cores_out || !u) return;
        int modes[3], ranks[4];
        if (tt_iga_solution_cores(ctx, u, nullptr, 0, modes, ranks) != TT_IGA_OK) return;
        const size_t need = (size_t)ranks[1] * modes[0] + (size_t)ranks[1] * modes[1] * ranks[2] +
                            (size_t)ranks[2] * modes[2];
        if (cores_off + need > it.cores_cap) {
          if (st == TT_IGA_OK) st = TT_IGA_ERR_TOO_LARGE;
          return;
        }
        tt_iga_solution_cores(ctx, u, it.cores_out + cores_off, it.cores_cap - cores_off, modes, ranks);
        res.rhs_ranks[k][0] = ranks[1];
        res.rhs_ranks[k][1] = ranks[2];
        cores_off += need;
      };
      if (st == TT_IGA_OK && it.n_rhs > 1 && it.rhs_solve == TT_IGA_RHS_BLOCK) {
        tt_iga_solution *us[8] = {};
        double rr[8];
        tt_iga_stats stats{};
        st = tt_iga_solve_block(ctx, s, &it.opts, -1, us, &stats, rr);
        for (int k = 0; k < it.n_rhs; ++k) {
          worst = (worst < 0.0 || rr[k] < 0.0) ? -1.0 : std::max(worst, rr[k]);
          keep_cores(k, us[k]);
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
        worst = (worst < 0.0 || stats.rel_residual < 0.0) ? -1.0 : std::max(worst, stats.rel_residual);
        res.ranks[0] = stats.ranks[0];
        res.ranks[1] = stats.ranks[1];
        res.sweeps += stats.sweeps;
        keep_cores(k, u);
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

int tt_iga_batch_autotune(int device, int count, const tt_iga_batch_item *items, const int *lane_candidates,
                          int n_lane_candidates, const int *share_candidates, int n_share_candidates,
                          tt_iga_batch_result *results, int *best_lanes, int *best_sm_per_lane, double *best_ms) {
  if (!lane_candidates || n_lane_candidates < 1 || !best_lanes || (n_share_candidates > 0 && !share_candidates))
    return TT_IGA_ERR_ARG;
  const int default_share = -1;
  const int *shares = n_share_candidates > 0 ? share_candidates : &default_share;
  const int ns = n_share_candidates > 0 ? n_share_candidates : 1;
  double best = 1e300;
  int pick = lane_candidates[0], pick_share = shares[0];
  for (int c = 0; c < n_lane_candidates; ++c)
    for (int q = 0; q < ns; ++q) {
      double ms = 0.0;
      const int rc = tt_iga_batch_solve(device, count, items, lane_candidates[c], shares[q], results, &ms);
      if (rc != TT_IGA_OK && rc != TT_IGA_ERR_NOT_CONVERGED) return rc;
      if (ms < best) {
        best = ms;
        pick = lane_candidates[c];
        pick_share = shares[q];
      }
    }
  *best_lanes = pick;
  if (best_sm_per_lane) *best_sm_per_lane = pick_share;
  if (best_ms) *best_ms = best;
  return TT_IGA_OK;
}

}  // extern "C"
