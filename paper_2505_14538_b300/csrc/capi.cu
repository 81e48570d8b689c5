// capi.cu -- the extern "C" entry points declared in include/swift_gpu.h:
// argument checks, the context and its device arena, call-order state, the
// status word and statistics.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <new>

#include "common.cuh"
#include "internal.h"
#include "lpp.cuh"

struct swift_gpu_ctx {
  sg::Ctx c;
};

namespace sg {

Ctx* from(swift_gpu_ctx* c) { return c ? &c->c : nullptr; }

static bool aligned(const void* p, size_t a) { return p && ((uintptr_t)p % a) == 0; }

int phys_from(const swift_gpu_params* p, Phys* ph) {
  for (int a = 0; a < 3; ++a)
    if (!(p->box[a] > 0.0f) || !isfinite(p->box[a])) return SWIFT_GPU_ERR_ARG;
  if (!(p->kernel_gamma > 0.0f) || !(p->eta > 0.0f) || !(p->gamma_eos > 1.0f)) return SWIFT_GPU_ERR_ARG;
  if (p->max_iter < 1 || !(p->h_tol >= 0.0f) || p->h_max < 0.0f || p->cell_margin < 0.0f)
    return SWIFT_GPU_ERR_ARG;
  if (p->kernel < SWIFT_GPU_KERNEL_CUBIC || p->kernel > SWIFT_GPU_KERNEL_WENDLAND_C4) return SWIFT_GPU_ERR_ARG;
  if ((p->flags & SWIFT_GPU_ADAPTIVE) &&
      ((p->flags & SWIFT_GPU_PLAIN) || p->leaf_max < 8 || p->leaf_max > 1024 || !(p->leaf_margin >= 0.01f) ||
       !isfinite(p->leaf_margin)))
    return SWIFT_GPU_ERR_ARG;
  for (int a = 0; a < 3; ++a) ph->L[a] = p->box[a];
  ph->kg = p->kernel_gamma;
  ph->gamma_eos = p->gamma_eos;
  ph->alpha_v = p->alpha_v;
  ph->beta_v = p->beta_v;
  ph->alpha_c = p->alpha_c;
  ph->eta3 = (double)p->eta * (double)p->eta * (double)p->eta;
  ph->h_tol = (double)p->h_tol;
  ph->max_iter = p->max_iter < kMaxPasses ? p->max_iter : kMaxPasses;
  ph->h_max = p->h_max;
  ph->compensated = (p->flags & SWIFT_GPU_NO_COMPENSATION) ? 0 : 1;
  ph->kernel = p->kernel;
  ph->knorm = kernel_norm(p->kernel);
  return SWIFT_GPU_OK;
}

template <class T>
static bool dalloc(T** p, size_t count) {
  if (count == 0) count = 1;
  return cudaMalloc((void**)p, sizeof(T) * count) == cudaSuccess;
}

static void free_all(Ctx* c) {
  void* ptrs[] = {c->d_status, c->d_grid, c->d_hmax_bits, c->d_keys[0], c->d_keys[1], c->d_vals[0], c->d_vals[1],
                  c->d_hist, c->d_scan_tmp, c->d_cell_start, c->d_pos, c->d_vel, c->d_rho4, c->d_cd, c->d_h,
                  c->d_bracket, c->d_ngb, c->d_ga, c->d_gb, c->d_act, c->d_items0, c->d_plist0, c->d_items[0],
                  c->d_items[1], c->d_plist[0], c->d_plist[1], c->d_counters, c->d_stats, c->d_red_partial,
                  c->d_scratch4[0], c->d_scratch1[0], c->d_scratch1[1], c->d_plain_act, c->d_aux[0], c->d_aux[1],
                  c->d_node_range, c->d_node, c->d_node_link, c->d_node_parent, c->d_node_done, c->d_node_flag,
                  c->d_leaf_range, c->d_leaf_hcap, c->d_leaf_node, c->d_nbr_span, c->d_nbr, c->d_tree_ctr,
                  c->d_nlist, c->d_item_nl, c->d_rep, c->d_lcnt, c->d_gc};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (c->h_status) cudaFreeHost(c->h_status);
  if (c->h_stats) cudaFreeHost(c->h_stats);
}

}  // namespace sg

using namespace sg;

extern "C" {

void swift_gpu_default_params(swift_gpu_params* p) {
  if (!p) return;
  p->box[0] = p->box[1] = p->box[2] = 1.0f;
  p->gamma_eos = 5.0f / 3.0f;
  p->eta = 1.2348f;
  p->kernel_gamma = 1.825742f;
  p->alpha_v = 1.0f;
  p->beta_v = 3.0f;
  p->alpha_c = 1.0f;
  p->h_tol = 1e-4f;
  p->max_iter = 30;
  p->h_max = 0.0f;
  p->cell_margin = 0.05f;
  p->flags = 0;
  p->leaf_max = 32;
  p->leaf_margin = 0.1f;
  p->kernel = SWIFT_GPU_KERNEL_CUBIC;
}

int swift_gpu_create(swift_gpu_ctx** out, const swift_gpu_params* p, int64_t n_max) {
  if (!out || !p || n_max < 1 || n_max > (int64_t)kIndexMask) return SWIFT_GPU_ERR_ARG;
  *out = nullptr;
  swift_gpu_ctx* h = new (std::nothrow) swift_gpu_ctx();
  if (!h) return SWIFT_GPU_ERR_NOMEM;
  Ctx* c = &h->c;
  if (phys_from(p, &c->phys) != SWIFT_GPU_OK) {
    delete h;
    return SWIFT_GPU_ERR_ARG;
  }
  c->params = *p;
  c->n_max = n_max;
  if (cudaGetDevice(&c->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
    delete h;
    return SWIFT_GPU_ERR_CUDA;
  }
  c->tuning.threads_per_block = 256;
  c->tuning.max_lanes_per_particle = 32;  // one lane a particle below, where that path exists
  c->tuning.blocks_per_sm = 0;
  c->tuning.group_collect = SWIFT_GPU_COLLECT_ROWS;
  int nc_cap = (int)floor(cbrt(2.0 * (double)n_max));
  if (nc_cap < 3) nc_cap = 3;
  if (nc_cap > 1024) nc_cap = 1024;
  c->nc_cap = nc_cap;
  const int64_t ncells_max = (int64_t)nc_cap * nc_cap * nc_cap;
  int bits = 0;
  while (((int64_t)1 << bits) < ncells_max) ++bits;
  c->max_key_bits = bits;
  c->max_passes = kMaxPasses;
  const int64_t n = n_max;
  const int64_t nb = (n + kRadixTile - 1) / kRadixTile;  // radix tiles: 256 histogram entries each
  int64_t scan_m = 256 * nb > ncells_max + 1 ? 256 * nb : ncells_max + 1;
  // adaptive tree: cells (at most kAdaptiveNcCap^3 of them) plus 2 nodes per
  // particle, all addressable with kIndexBits; leaves are disjoint and non-empty
  const int64_t acells = ncells_max < (int64_t)kAdaptiveNcCap * kAdaptiveNcCap * kAdaptiveNcCap
                             ? ncells_max
                             : (int64_t)kAdaptiveNcCap * kAdaptiveNcCap * kAdaptiveNcCap;
  const int64_t node_cap = acells + 2 * n < (int64_t)kIndexMask ? acells + 2 * n : (int64_t)kIndexMask;
  c->node_cap = (int)node_cap;
  c->leaf_cap = (int)n;
  if (scan_m < node_cap + 1) scan_m = node_cap + 1;  // leaf flags of the tree nodes
  // Kept candidate lists (uniform grid only; adaptive leaves never keep them): a fixed span of W
  // entries a lane for every group of 32 particles (lpp_width_of: W = 92 for the cubic spline's
  // about 56 candidates, more for the shapes with more neighbours). A context created for
  // adaptive leaves holds the tree arrays instead; one created for the uniform grid holds none.
  const bool adaptive = (p->flags & SWIFT_GPU_ADAPTIVE) != 0;
  const bool lpp = !adaptive && (p->flags & SWIFT_GPU_PLAIN) == 0;
  const int64_t lpp_need = (int64_t)lpp_width_of(p->kernel) * 32 * ((n + 31) / 32);
  c->nl_cap = lpp ? lpp_need : 0;  // every index into the store is 64-bit
  const bool lpp_fits = c->nl_cap > 0;
  const int64_t ngroups = (n + 31) / 32 + 1;
  int64_t nbr_cap = 48 * n > ((int64_t)1 << 22) ? 48 * n : ((int64_t)1 << 22);  // at least 16 MB of lists
  c->nbr_cap = (int)(nbr_cap < (int64_t)INT32_MAX ? nbr_cap : (int64_t)INT32_MAX);
  c->red_blocks = c->num_sms * 32;
  bool ok = dalloc(&c->d_status, 1) && dalloc(&c->d_grid, 1) && dalloc(&c->d_hmax_bits, kHmaxWords) &&
            dalloc(&c->d_keys[0], n) && dalloc(&c->d_keys[1], n) && dalloc(&c->d_vals[0], n) &&
            dalloc(&c->d_vals[1], n) && dalloc(&c->d_hist, 256 * nb) &&
            dalloc(&c->d_scan_tmp, scan_tiles_needed(scan_m) + 1) && dalloc(&c->d_cell_start, ncells_max + 1) &&
            dalloc(&c->d_pos, n) && dalloc(&c->d_vel, n) && dalloc(&c->d_rho4, n) && dalloc(&c->d_cd, n) &&
            dalloc(&c->d_h, n) && dalloc(&c->d_bracket, n) && dalloc(&c->d_ngb, n) && dalloc(&c->d_ga, n) &&
            dalloc(&c->d_gb, n) && dalloc(&c->d_act, n) && dalloc(&c->d_items0, n) && dalloc(&c->d_plist0, n) &&
            dalloc(&c->d_items[0], n) && dalloc(&c->d_items[1], n) && dalloc(&c->d_plist[0], n) &&
            dalloc(&c->d_plist[1], n) && dalloc(&c->d_counters, kCtrCount(kMaxPasses)) &&
            dalloc(&c->d_stats, kStatCount) && dalloc(&c->d_red_partial, 8 * (size_t)c->red_blocks) &&
            dalloc(&c->d_scratch4[0], 4 * n) && dalloc(&c->d_scratch1[0], n) && dalloc(&c->d_scratch1[1], n) &&
            dalloc(&c->d_plain_act, n) && dalloc(&c->d_tree_ctr, kTreeCtrCount) &&
            (!adaptive ||
             (dalloc(&c->d_aux[0], n) && dalloc(&c->d_aux[1], n) && dalloc(&c->d_node_range, node_cap) &&
              dalloc(&c->d_node, 2 * node_cap) && dalloc(&c->d_node_link, node_cap) &&
              dalloc(&c->d_node_parent, node_cap) && dalloc(&c->d_node_done, node_cap) &&
              dalloc(&c->d_node_flag, node_cap + 1) && dalloc(&c->d_leaf_range, n) && dalloc(&c->d_leaf_hcap, n) &&
              dalloc(&c->d_leaf_node, n) && dalloc(&c->d_nbr_span, n) && dalloc(&c->d_nbr, (size_t)c->nbr_cap))) &&
            (c->nl_cap == 0 || dalloc(&c->d_nlist, (size_t)c->nl_cap)) && dalloc(&c->d_item_nl, ngroups) &&
            (!lpp_fits || (dalloc(&c->d_rep, (size_t)kAxes * n) && dalloc(&c->d_lcnt, n) && dalloc(&c->d_gc, n))) &&
            cudaMallocHost((void**)&c->h_status, sizeof(Status)) == cudaSuccess &&
            cudaMallocHost((void**)&c->h_stats, sizeof(unsigned long long) * kStatCount) == cudaSuccess;
  if (ok)
    for (int q = 1; q < 4; ++q) c->d_scratch4[q] = c->d_scratch4[0] + q * n;

  if (!ok) {
    cudaGetLastError();
    free_all(c);
    delete h;
    return SWIFT_GPU_ERR_NOMEM;
  }
  cudaMemset(c->d_status, 0, sizeof(Status));
  cudaMemset(c->d_stats, 0, sizeof(unsigned long long) * kStatCount);
  cudaMemset(c->d_counters, 0, sizeof(int) * kCtrCount(kMaxPasses));
  cudaMemset(c->d_hmax_bits, 0, sizeof(unsigned) * kHmaxWords);  // k_scan_h leaves them zero after each call
  cudaMemset(c->d_tree_ctr, 0, sizeof(int) * kTreeCtrCount);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    free_all(c);
    delete h;
    return SWIFT_GPU_ERR_CUDA;
  }
  *out = h;
  return SWIFT_GPU_OK;
}

int swift_gpu_destroy(swift_gpu_ctx* h) {
  if (!h) return SWIFT_GPU_OK;
  cudaDeviceSynchronize();
  free_all(&h->c);
  delete h;
  return SWIFT_GPU_OK;
}

int swift_gpu_set_params(swift_gpu_ctx* h, const swift_gpu_params* p) {
  Ctx* c = from(h);
  if (!c || !p) return SWIFT_GPU_ERR_ARG;
  // adaptive leaves need the tree arrays, which only a context created with the flag holds
  if ((p->flags & SWIFT_GPU_ADAPTIVE) && c->d_node == nullptr) return SWIFT_GPU_ERR_ARG;
  Phys ph;
  if (phys_from(p, &ph) != SWIFT_GPU_OK) return SWIFT_GPU_ERR_ARG;
  c->params = *p;
  c->phys = ph;
  return SWIFT_GPU_OK;
}

int swift_gpu_build_cells(swift_gpu_ctx* h, const float* pos_h, int64_t n, float min_cell_width, void* stream) {
  Ctx* c = from(h);
  if (!c || n < 0 || !(min_cell_width >= 0.0f)) return SWIFT_GPU_ERR_ARG;
  if (n > c->n_max) return SWIFT_GPU_ERR_CAPACITY;
  if (n > 0 && !aligned(pos_h, 16)) return SWIFT_GPU_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  int rc = build_cells_impl(c, reinterpret_cast<const float4*>(pos_h), (int)n, min_cell_width, s);
  c->state = rc == SWIFT_GPU_OK ? 1 : 0;
  return rc;
}

int swift_gpu_density(swift_gpu_ctx* h, const float* pos_h_in, const float* vel_m, const uint8_t* active,
                      float* h_out, float* rho4, float* curl_div, uint32_t* ngb_count, void* stream) {
  Ctx* c = from(h);
  if (!c) return SWIFT_GPU_ERR_ARG;
  if (!(c->state & 1)) return SWIFT_GPU_ERR_ORDER;
  if (c->n > 0 && (!aligned(pos_h_in, 16) || !aligned(vel_m, 16) || !aligned(h_out, 4) || !aligned(rho4, 16) ||
                   !aligned(curl_div, 16) || (ngb_count && !aligned(ngb_count, 4))))
    return SWIFT_GPU_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  int (*impl)(Ctx*, const float4*, const float4*, const uint8_t*, float*, float4*, float4*, uint32_t*,
              cudaStream_t) = (c->params.flags & SWIFT_GPU_PLAIN) ? plain_density_impl : density_impl;
  int rc = impl(c, reinterpret_cast<const float4*>(pos_h_in), reinterpret_cast<const float4*>(vel_m), active, h_out,
                reinterpret_cast<float4*>(rho4), reinterpret_cast<float4*>(curl_div), ngb_count, s);
  c->state = rc == SWIFT_GPU_OK ? 3 : 1;
  c->last_pos_in = reinterpret_cast<const float4*>(pos_h_in);
  c->last_vel_in = reinterpret_cast<const float4*>(vel_m);
  c->last_active = active;
  c->last_h_out = h_out;
  c->last_rho4 = reinterpret_cast<float4*>(rho4);
  c->last_cd = reinterpret_cast<float4*>(curl_div);
  c->last_ngb = ngb_count;
  return rc;
}

int swift_gpu_gradient(swift_gpu_ctx* h, const float* u, float* vsig_lapu, void* stream) {
  Ctx* c = from(h);
  if (!c) return SWIFT_GPU_ERR_ARG;
  if (!(c->state & 2)) return SWIFT_GPU_ERR_ORDER;
  if (c->n > 0 && (!aligned(u, 4) || !aligned(vsig_lapu, 8))) return SWIFT_GPU_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  int rc = ghost_impl(c, u, nullptr, nullptr, s);
  if (rc == SWIFT_GPU_OK)
    rc = (c->params.flags & SWIFT_GPU_PLAIN) ? plain_gradient_impl(c, reinterpret_cast<float2*>(vsig_lapu), s)
                                             : gradient_impl(c, reinterpret_cast<float2*>(vsig_lapu), s);
  c->last_grad_out = reinterpret_cast<float2*>(vsig_lapu);
  if (rc == SWIFT_GPU_OK) c->state |= 4;
  return rc;
}

int swift_gpu_force(swift_gpu_ctx* h, const float* u, const float* alpha_v_i, const float* alpha_c_i,
                    float* accel_dudt, float* dh_dt, double* reductions, void* stream) {
  Ctx* c = from(h);
  if (!c) return SWIFT_GPU_ERR_ARG;
  if (!(c->state & 2)) return SWIFT_GPU_ERR_ORDER;
  if (c->n > 0 && (!aligned(u, 4) || !aligned(accel_dudt, 16) || (dh_dt && !aligned(dh_dt, 4)) ||
                   (alpha_v_i && !aligned(alpha_v_i, 4)) || (alpha_c_i && !aligned(alpha_c_i, 4))))
    return SWIFT_GPU_ERR_ARG;
  if (reductions && !aligned(reductions, 8)) return SWIFT_GPU_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  int rc = ghost_impl(c, u, alpha_v_i, alpha_c_i, s);
  if (rc == SWIFT_GPU_OK)
    rc = (c->params.flags & SWIFT_GPU_PLAIN)
             ? plain_force_impl(c, reinterpret_cast<float4*>(accel_dudt), dh_dt, reductions, s)
             : force_impl(c, reinterpret_cast<float4*>(accel_dudt), dh_dt, reductions, s);
  if (rc == SWIFT_GPU_OK) {
    c->state |= 8;
    c->last_u = u;
    c->last_alpha_v = alpha_v_i;
    c->last_alpha_c = alpha_c_i;
    c->last_force_out = reinterpret_cast<float4*>(accel_dudt);
    c->last_dhdt = dh_dt;
  }
  return rc;
}

int swift_gpu_gradient_force(swift_gpu_ctx* h, const float* u, const float* alpha_v_i, const float* alpha_c_i,
                             float* vsig_lapu, float* accel_dudt, float* dh_dt, double* reductions, void* stream) {
  Ctx* c = from(h);
  if (!c) return SWIFT_GPU_ERR_ARG;
  if (!(c->state & 2)) return SWIFT_GPU_ERR_ORDER;
  if (c->n > 0 && (!aligned(u, 4) || !aligned(vsig_lapu, 8) || !aligned(accel_dudt, 16) ||
                   (dh_dt && !aligned(dh_dt, 4)) || (alpha_v_i && !aligned(alpha_v_i, 4)) ||
                   (alpha_c_i && !aligned(alpha_c_i, 4))))
    return SWIFT_GPU_ERR_ARG;
  if (reductions && !aligned(reductions, 8)) return SWIFT_GPU_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  int rc = ghost_impl(c, u, alpha_v_i, alpha_c_i, s);
  if (rc == SWIFT_GPU_OK) {
    if (c->params.flags & SWIFT_GPU_PLAIN) {
      rc = plain_gradient_impl(c, reinterpret_cast<float2*>(vsig_lapu), s);
      if (rc == SWIFT_GPU_OK)
        rc = plain_force_impl(c, reinterpret_cast<float4*>(accel_dudt), dh_dt, reductions, s);
    } else {
      rc = grad_force_impl(c, reinterpret_cast<float2*>(vsig_lapu), reinterpret_cast<float4*>(accel_dudt), dh_dt,
                           reductions, s);
    }
  }
  if (rc == SWIFT_GPU_OK) {
    c->state |= 4 | 8;
    c->last_u = u;
    c->last_alpha_v = alpha_v_i;
    c->last_alpha_c = alpha_c_i;
    c->last_grad_out = reinterpret_cast<float2*>(vsig_lapu);
    c->last_force_out = reinterpret_cast<float4*>(accel_dudt);
    c->last_dhdt = dh_dt;
  }
  return rc;
}

int swift_gpu_force_backward(swift_gpu_ctx* h, const float* grad_accel_dudt, float* grad_x, float* grad_v,
                             float* grad_u, int h_mode, void* stream) {
  Ctx* c = from(h);
  if (!c || (h_mode != 0 && h_mode != 1)) return SWIFT_GPU_ERR_ARG;
  if (!(c->state & 8)) return SWIFT_GPU_ERR_ORDER;
  if (!c->all_active || (c->params.flags & SWIFT_GPU_PLAIN)) return SWIFT_GPU_ERR_ARG;
  if (c->n > 0 && (!aligned(grad_accel_dudt, 16) || !aligned(grad_x, 16) || !aligned(grad_v, 16) ||
                   !aligned(grad_u, 4)))
    return SWIFT_GPU_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  return backward_impl(c, reinterpret_cast<const float4*>(grad_accel_dudt), reinterpret_cast<float4*>(grad_x),
                       reinterpret_cast<float4*>(grad_v), grad_u, h_mode, s);
}

int swift_gpu_set_inactive(swift_gpu_ctx* h, const uint8_t* mask, const float* h_in, const float* rho4,
                           const float* curl_div, void* stream) {
  Ctx* c = from(h);
  if (!c) return SWIFT_GPU_ERR_ARG;
  if (!(c->state & 2) || (c->params.flags & SWIFT_GPU_PLAIN)) return SWIFT_GPU_ERR_ORDER;
  if (c->n > 0 && (!aligned(mask, 1) || !aligned(h_in, 4) || !aligned(rho4, 16) || !aligned(curl_div, 16)))
    return SWIFT_GPU_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  return set_inactive_impl(c, mask, h_in, reinterpret_cast<const float4*>(rho4),
                           reinterpret_cast<const float4*>(curl_div), s);
}

int swift_gpu_sync_status(swift_gpu_ctx* h, int* status, int64_t* detail) {
  Ctx* c = from(h);
  if (!c) return SWIFT_GPU_ERR_ARG;
  // The whole device, not one stream: the calls may have been captured in a
  // CUDA graph and replayed on a stream the library never saw.
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(c->h_status, c->d_status, sizeof(Status), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return SWIFT_GPU_ERR_CUDA;
  if (status) *status = c->h_status->code;
  if (detail) *detail = (int64_t)c->h_status->detail;
  return cudaMemset(c->d_status, 0, sizeof(Status)) == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess
             ? SWIFT_GPU_OK
             : SWIFT_GPU_ERR_CUDA;
}

int swift_gpu_get_info(swift_gpu_ctx* h, swift_gpu_info* info) {
  Ctx* c = from(h);
  if (!c || !info) return SWIFT_GPU_ERR_ARG;
  Grid g;
  if (cudaDeviceSynchronize() != cudaSuccess || cudaMemcpy(&g, c->d_grid, sizeof(Grid), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(c->h_stats, c->d_stats, sizeof(unsigned long long) * kStatCount, cudaMemcpyDeviceToHost) !=
          cudaSuccess)
    return SWIFT_GPU_ERR_CUDA;
  memset(info, 0, sizeof(*info));
  info->n = c->n;
  for (int a = 0; a < 3; ++a) {
    info->nc[a] = (c->state & 1) ? g.nc[a] : 0;
    info->cell_width[a] = (c->state & 1) ? g.width[a] : 0.0f;
  }
  info->h_cap = (c->state & 1) ? g.hcap : 0.0f;
  info->n_cells = (c->state & 1) ? g.ncells : 0;
  info->n_items = (int64_t)c->h_stats[kStatItems];
  info->density_passes = (int32_t)c->h_stats[kStatPasses];
  info->interactions[0] = c->h_stats[kStatInterDens];
  info->interactions[1] = c->h_stats[kStatInterGrad];
  info->interactions[2] = c->h_stats[kStatInterForce];
  info->candidates[0] = c->h_stats[kStatCandDens];
  info->candidates[1] = c->h_stats[kStatCandGrad];
  info->candidates[2] = c->h_stats[kStatCandForce];
  info->launches = c->launches;
  info->h_iteration_pairs = c->h_stats[kStatInterHiter];
  if ((c->state & 1) && c->tree_built) {
    int tc[kTreeCtrCount];
    if (cudaMemcpy(tc, c->d_tree_ctr, sizeof(tc), cudaMemcpyDeviceToHost) != cudaSuccess) return SWIFT_GPU_ERR_CUDA;
    info->n_leaves = tc[kTreeLeaves];
    info->leaf_pairs = tc[kTreeEntries];
    info->tree_depth = tc[kTreeDepth];
  }
  return SWIFT_GPU_OK;
}

int swift_gpu_get_leaves(swift_gpu_ctx* h, int32_t* range, float* h_cap, int32_t* nbr_count, int64_t max_leaves,
                         void* stream) {
  Ctx* c = from(h);
  if (!c || max_leaves < 0) return SWIFT_GPU_ERR_ARG;
  if (!(c->state & 1) || !c->tree_built) return SWIFT_GPU_ERR_ORDER;
  if ((range && !aligned(range, 4)) || (h_cap && !aligned(h_cap, 4)) || (nbr_count && !aligned(nbr_count, 4)))
    return SWIFT_GPU_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  return leaves_export_impl(c, range, h_cap, nbr_count, max_leaves, s);
}

int swift_gpu_get_cells(swift_gpu_ctx* h, uint32_t* cell_id, uint32_t* perm, void* stream) {
  Ctx* c = from(h);
  if (!c) return SWIFT_GPU_ERR_ARG;
  if (!(c->state & 1)) return SWIFT_GPU_ERR_ORDER;
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  return cells_export_impl(c, cell_id, perm, s);
}

int swift_gpu_get_tuning(swift_gpu_ctx* h, swift_gpu_tuning* t) {
  Ctx* c = from(h);
  if (!c || !t) return SWIFT_GPU_ERR_ARG;
  *t = c->tuning;
  return SWIFT_GPU_OK;
}

int swift_gpu_set_tuning(swift_gpu_ctx* h, const swift_gpu_tuning* t) {
  Ctx* c = from(h);
  if (!c || !t) return SWIFT_GPU_ERR_ARG;
  const int l = t->max_lanes_per_particle;
  if (t->threads_per_block != 256 || !(l == 1 || l == 2 || l == 4 || l == 8 || l == 16 || l == 32) ||
      t->blocks_per_sm < 0 ||
      !(t->group_collect == SWIFT_GPU_COLLECT_ROWS || t->group_collect == SWIFT_GPU_COLLECT_WINDOWS))
    return SWIFT_GPU_ERR_ARG;
  c->tuning = *t;
  return SWIFT_GPU_OK;
}

int swift_gpu_autotune(swift_gpu_ctx* h, int loop, void* stream) {
  Ctx* c = from(h);
  if (!c || loop < 0 || loop > 4 || (c->params.flags & SWIFT_GPU_PLAIN)) return SWIFT_GPU_ERR_ARG;
  if (!(c->state & 8)) return SWIFT_GPU_ERR_ORDER;
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  return autotune_impl(c, loop, s);
}

}  // extern "C"
