// Launch-shape autotuner: times the candidate values of each shape on the
// caller's input and keeps the fastest in the plan. The shapes only spread
// the same work differently over the GPU, so every candidate gives the same
// results bit for bit.
#include <algorithm>
#include <vector>

#include "hpm_internal.cuh"

using namespace hpm;

namespace {

bool valid_tuning(const hpm_tuning &t) {
  return t.level_blocks_per_sm >= 0 && t.level_blocks_per_sm <= 4 &&
         (t.gridlet_warps == 0 || t.gridlet_warps == 2 || t.gridlet_warps == 4 || t.gridlet_warps == 8) &&
         t.m2l_ctas_per_sm >= 0 && t.m2l_ctas_per_sm <= 2 && t.m2l_block_order >= 0 && t.m2l_block_order <= 2 &&
         (t.m2l_tile_parents == 0 || t.m2l_tile_parents == 256 || t.m2l_tile_parents == 224 ||
          t.m2l_tile_parents == 208 || t.m2l_tile_parents == 192);
}

// One build + solve; the device time of the stages `stage` selects (0 tree,
// 1 child-to-parent + parent-to-child, 2 source-to-target).
hpm_status run_once(hpm_plan_t pl, const double *pos, const double *mass, int64_t n, cudaStream_t st, float *phi,
                    float *acc, int stage, float *ms) {
  HPM_TRY(hpm_build_tree(pl, pos, n, st));
  HPM_TRY(hpm_solve(pl, pos, mass, phi, acc, st));
  hpm_stats s{};
  HPM_TRY(hpm_get_stats(pl, &s));
  *ms = stage == 0 ? s.ms_tree : (stage == 1 ? s.ms_m2m + s.ms_l2l : s.ms_m2l);
  return HPM_OK;
}

// Best of three runs of the current shapes.
hpm_status best_of(hpm_plan_t pl, const double *pos, const double *mass, int64_t n, cudaStream_t st, float *phi,
                   float *acc, int stage, float *best) {
  *best = 1e30f;
  for (int r = 0; r < 3; ++r) {
    float ms = 0.f;
    HPM_TRY(run_once(pl, pos, mass, n, st, phi, acc, stage, &ms));
    *best = std::min(*best, ms);
  }
  return HPM_OK;
}

// Tries each candidate value of *knob, keeps the fastest.
hpm_status tune_knob(hpm_plan_t pl, int *knob, const std::vector<int> &cands, const double *pos,
                     const double *mass, int64_t n, cudaStream_t st, float *phi, float *acc, int stage) {
  int best_v = *knob;
  float best_ms = 1e30f;
  for (int v : cands) {
    *knob = v;
    float ms = 0.f;
    HPM_TRY(best_of(pl, pos, mass, n, st, phi, acc, stage, &ms));
    if (ms < best_ms) {
      best_ms = ms;
      best_v = v;
    }
  }
  *knob = best_v;
  return HPM_OK;
}

}  // namespace

extern "C" {

hpm_status hpm_set_tuning(hpm_plan_t plan, const hpm_tuning *tuning) {
  if (!plan || !tuning || !valid_tuning(*tuning)) return HPM_ERR_INVALID_ARG;
  plan->tuning = *tuning;
  return HPM_OK;
}

hpm_status hpm_test_stall(hpm_plan_t plan, int on, long long wait_limit_cycles) {
  if (!plan || wait_limit_cycles < 0) return HPM_ERR_INVALID_ARG;
  plan->test_stall = on ? 1 : 0;
  plan->test_wait_limit = wait_limit_cycles;
  return HPM_OK;
}

hpm_status hpm_get_tuning(hpm_plan_t plan, hpm_tuning *tuning) {
  if (!plan || !tuning) return HPM_ERR_INVALID_ARG;
  *tuning = plan->tuning;
  return HPM_OK;
}

hpm_status hpm_tune(hpm_plan_t plan, const double *d_pos, const double *d_mass, int64_t n, void *stream,
                    hpm_tuning *out) {
  if (!plan || n < 0 || (n > 0 && (!d_pos || !d_mass))) return HPM_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  // stage timings need the plan's events
  const bool had_events = plan->events_ready;
  if (!had_events) {
    for (auto &ev : plan->ev)
      if (!ev) HPM_CUDA(cudaEventCreate(&ev));
    plan->events_ready = true;
  }
  hpm_status s = HPM_OK;
  DevBuf phi, acc;
  if (n > 0) {
    s = phi.ensure(sizeof(float) * n, st);
    if (s == HPM_OK) s = acc.ensure(sizeof(float) * 3 * n, st);
  }
  if (s == HPM_OK && n > 0) {
    hpm_tuning &t = plan->tuning;
    if (t.level_blocks_per_sm == 0) t.level_blocks_per_sm = 2;
    s = tune_knob(plan, &t.level_blocks_per_sm, {1, 2, 3, 4}, d_pos, d_mass, n, st, phi.as<float>(),
                  acc.as<float>(), 0);
    if (s == HPM_OK && plan->ng == 4) {
      if (t.gridlet_warps == 0) t.gridlet_warps = 8;
      s = tune_knob(plan, &t.gridlet_warps, {2, 4, 8}, d_pos, d_mass, n, st, phi.as<float>(), acc.as<float>(), 1);
    }
    if (s == HPM_OK && use_tc_m2l(plan)) {
      if (t.m2l_block_order == 0) t.m2l_block_order = 1;
      s = tune_knob(plan, &t.m2l_block_order, {1, 2}, d_pos, d_mass, n, st, phi.as<float>(), acc.as<float>(), 2);
    }
    if (s == HPM_OK && use_tc_m2l(plan) && plan->ng == 4) {
      if (t.m2l_tile_parents == 0) t.m2l_tile_parents = 256;
      s = tune_knob(plan, &t.m2l_tile_parents, {256, 224, 208, 192}, d_pos, d_mass, n, st, phi.as<float>(),
                    acc.as<float>(), 2);
    }
    if (s == HPM_OK && !use_tc_m2l(plan) && !(plan->opts.flags & HPM_FLAG_GENERIC_M2L)) {
      if (t.m2l_ctas_per_sm == 0) t.m2l_ctas_per_sm = 2;
      s = tune_knob(plan, &t.m2l_ctas_per_sm, {1, 2}, d_pos, d_mass, n, st, phi.as<float>(), acc.as<float>(), 2);
    }
    // leave the plan built for this input with the chosen shapes
    if (s == HPM_OK) {
      float ms = 0.f;
      s = run_once(plan, d_pos, d_mass, n, st, phi.as<float>(), acc.as<float>(), 0, &ms);
    }
  }
  if (s == HPM_OK) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      set_cuda_error(e);
      s = HPM_ERR_CUDA;
    }
  }
  phi.release(st);
  acc.release(st);
  if (!had_events) {
    cudaStreamSynchronize(st);
    for (auto &ev : plan->ev)
      if (ev) {
        cudaEventDestroy(ev);
        ev = nullptr;
      }
    plan->events_ready = false;
    cudaGetLastError();
  }
  if (s == HPM_OK && out) *out = plan->tuning;
  return s;
}

}  // extern "C"
