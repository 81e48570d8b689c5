// tune.cu -- the autotuner: times one loop over the data of the last calls
// for each candidate work distribution and keeps the fastest. Every loop is
// deterministic given its inputs, so re-running it rewrites the same outputs.
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"

namespace sg {

static int run_density(Ctx* c, cudaStream_t s) {
  return density_impl(c, c->last_pos_in, c->last_vel_in, c->last_active, c->last_h_out, c->last_rho4, c->last_cd,
                      c->last_ngb, s);
}

static int run_loop(Ctx* c, int loop, cudaStream_t s) {
  if (loop == 0) return run_density(c, s);
  if (loop == 1) return gradient_impl(c, c->last_grad_out, s);
  if (loop == 3) return grad_force_impl(c, c->last_grad_out, c->last_force_out, c->last_dhdt, nullptr, s);
  if (loop == 4) {  // the whole step after the cell build: density, ghost, gradient + force
    int rc = run_density(c, s);
    if (rc == SWIFT_GPU_OK) rc = ghost_impl(c, c->last_u, c->last_alpha_v, c->last_alpha_c, s);
    if (rc == SWIFT_GPU_OK)
      rc = grad_force_impl(c, c->last_grad_out, c->last_force_out, c->last_dhdt, nullptr, s);
    return rc;
  }
  return force_impl(c, c->last_force_out, c->last_dhdt, nullptr, s);
}

// The ghost arrays the loop reads: the force loops those of the force call, gradient those of the gradient call.
static int run_ghost(Ctx* c, int loop, cudaStream_t s) {
  return loop != 1 ? ghost_impl(c, c->last_u, c->last_alpha_v, c->last_alpha_c, s)
                   : ghost_impl(c, c->last_u, nullptr, nullptr, s);
}

// The tuning picks the engine too (one lane a particle: the lane-per-particle
// path, whose lists the density call writes), so a gradient or force
// candidate first re-runs the density call and the ghost step, untimed.
static int prepare(Ctx* c, int loop, cudaStream_t s) {
  if (loop == 0 || loop == 4) return SWIFT_GPU_OK;
  int rc = run_density(c, s);
  if (rc == SWIFT_GPU_OK) rc = run_ghost(c, loop, s);
  return rc;
}

int autotune_impl(Ctx* c, int loop, cudaStream_t s) {
  if ((loop == 1 || loop == 3 || loop == 4) && !c->last_grad_out) return SWIFT_GPU_ERR_ORDER;
  // lanes per particle (1 twice: the shared-row and the windowed collect) x blocks per SM
  const int cand_l[7] = {1, 1, 2, 4, 8, 16, 32};
  const int cand_c[7] = {SWIFT_GPU_COLLECT_ROWS, SWIFT_GPU_COLLECT_WINDOWS, SWIFT_GPU_COLLECT_ROWS,
                         SWIFT_GPU_COLLECT_ROWS, SWIFT_GPU_COLLECT_ROWS, SWIFT_GPU_COLLECT_ROWS,
                         SWIFT_GPU_COLLECT_ROWS};
  const int cand_b[3] = {0, 1, 2};
  swift_gpu_tuning best = c->tuning, orig = c->tuning;
  float best_ms = 1e30f;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return SWIFT_GPU_ERR_CUDA;
  int rc = SWIFT_GPU_OK;
  for (int bi = 0; bi < 3 && rc == SWIFT_GPU_OK; ++bi) {
    for (int li = 0; li < 7 && rc == SWIFT_GPU_OK; ++li) {
      c->tuning.max_lanes_per_particle = cand_l[li];
      c->tuning.group_collect = cand_c[li];
      c->tuning.blocks_per_sm = cand_b[bi];
      rc = prepare(c, loop, s);
      if (rc == SWIFT_GPU_OK) rc = run_loop(c, loop, s);  // warm-up
      float tot = 0.0f;
      for (int r = 0; r < 3 && rc == SWIFT_GPU_OK; ++r) {
        cudaEventRecord(e0, s);
        rc = run_loop(c, loop, s);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = SWIFT_GPU_ERR_CUDA;
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        tot += ms;
      }
      if (rc == SWIFT_GPU_OK && tot < best_ms) {
        best_ms = tot;
        best = c->tuning;
      }
    }
  }
  c->tuning = rc == SWIFT_GPU_OK ? best : orig;
  // the loop's outputs (and, for density, the kept candidate lists) from the chosen setting
  if (rc == SWIFT_GPU_OK) rc = prepare(c, loop, s);
  if (rc == SWIFT_GPU_OK) rc = run_loop(c, loop, s);
  // leave the ghost arrays as the last force call left them
  ghost_impl(c, c->last_u, c->last_alpha_v, c->last_alpha_c, s);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

}  // namespace sg
