// integrate.cu -- leapfrog kick and drift (Sec. 2.2.2) and the evolution of
// the viscosity and conduction coefficients (Sec. 2.1.3, Eqs. 12-15; Sec.
// 2.1.4, Eqs. 21, 23, 24), as O(N) grid-stride kernels over the caller's
// particle arrays. The readings of the paper these follow are listed in
// include/swift_gpu_time.h.
//
// Each kernel streams its particle arrays once (float4 loads and stores,
// coalesced); the step size is read from and written to the caller's device
// clock so a whole step needs no host synchronisation.
#include <cuda_runtime.h>

#include "internal.h"
#include "../../include/swift_gpu_time.h"

namespace sg {
namespace {

constexpr int kIntThreads = 256;
constexpr unsigned kNoBoundBits = 0x7f7f7f7fu;  // 3.39e38: dt_next when no particle bounds the step

// Step of the step in progress: dt_next capped by dt_max and by t_end - t, >= 0.
__device__ __forceinline__ float step_size(const swift_gpu_clock* ck, float dt_max) {
  double dt = (double)ck->dt_next;
  if (dt_max > 0.0f) dt = fmin(dt, (double)dt_max);
  if (ck->t_end > 0.0) dt = fmin(dt, fmax(ck->t_end - ck->t, 0.0));
  return (float)fmax(dt, 0.0);
}

// u + (du/dt) dt/2, never below frac * u.
__device__ __forceinline__ float half_kick_u(float u, float dudt, float hdt, float frac) {
  return fmaxf(fmaf(dudt, hdt, u), frac * u);
}

// Periodic wrap into [0, L): the FP64 wrap of the library, and L itself (a
// rounding of a tiny negative x) maps to 0.
__device__ __forceinline__ float wrap_strict(float x, float L) {
  const float y = wrap_coord(x, L);
  return y < L ? y : 0.0f;
}

__global__ void __launch_bounds__(kIntThreads) k_kick_drift(swift_gpu_time_params tp, swift_gpu_clock* ck, int n,
                                                             float Lx, float Ly, float Lz, float4* __restrict__ pos_h,
                                                             float4* __restrict__ vel_m, float* __restrict__ u,
                                                             const float4* __restrict__ accel_dudt,
                                                             const float* __restrict__ dh_dt,
                                                             float4* __restrict__ vel_pred,
                                                             float* __restrict__ u_pred) {
  pdl_wait();
  // every thread derives dt from fields this kernel does not write
  const float dt = step_size(ck, tp.dt_max);
  if (blockIdx.x == 0 && threadIdx.x == 0) ck->dt = dt;
  const float hdt = 0.5f * dt;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float4 a = accel_dudt[i];
    float4 v = vel_m[i];
    float4 p = pos_h[i];
    v.x = fmaf(a.x, hdt, v.x);
    v.y = fmaf(a.y, hdt, v.y);
    v.z = fmaf(a.z, hdt, v.z);
    const float uh = half_kick_u(u[i], a.w, hdt, tp.u_min_frac);
    p.x = wrap_strict(fmaf(v.x, dt, p.x), Lx);
    p.y = wrap_strict(fmaf(v.y, dt, p.y), Ly);
    p.z = wrap_strict(fmaf(v.z, dt, p.z), Lz);
    if (dh_dt) p.w = p.w * expf(dh_dt[i] * dt / p.w);
    pos_h[i] = p;
    vel_m[i] = v;
    u[i] = uh;
    vel_pred[i] = make_float4(fmaf(a.x, hdt, v.x), fmaf(a.y, hdt, v.y), fmaf(a.z, hdt, v.z), v.w);
    u_pred[i] = half_kick_u(uh, a.w, hdt, tp.u_min_frac);
  }
}

__global__ void __launch_bounds__(kIntThreads) k_viscosity_switch(swift_gpu_time_params tp, float gamma_eos,
                                                                   float kg, const swift_gpu_clock* ck, int n,
                                                                   const float* __restrict__ h,
                                                                   const float* __restrict__ u,
                                                                   const float4* __restrict__ curl_div,
                                                                   const float2* __restrict__ vsig_lapu,
                                                                   float* __restrict__ div_prev,
                                                                   float* __restrict__ alpha_v) {
  pdl_wait();
  const float dt = ck->dt;
  const float c2 = gamma_eos * (gamma_eos - 1.0f);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float div = curl_div[i].w;
    if (dt > 0.0f) {
      const float H = kg * h[i];
      const float c = sqrtf(c2 * fmaxf(u[i], 0.0f));
      const float ddiv = (div - div_prev[i]) / dt;        // Eq. 15
      const float S = H * H * fmaxf(0.0f, -ddiv);         // Eq. 14
      const float vs = vsig_lapu[i].x;
      const float den = fmaf(vs, vs, S);
      const float a_loc = den > 0.0f ? tp.alpha_v_max * S / den : 0.0f;  // Eq. 13
      float a = alpha_v[i];
      a = a_loc >= a ? a_loc : a_loc + (a - a_loc) * expf(-tp.visc_length * c * dt / H);  // Eq. 12
      alpha_v[i] = fminf(fmaxf(a, tp.alpha_v_min), tp.alpha_v_max);
    }
    div_prev[i] = div;
  }
}

__global__ void __launch_bounds__(kIntThreads) k_kick_finish(swift_gpu_time_params tp, float kg, float alpha_v_const,
                                                              swift_gpu_clock* ck, int n, const float* __restrict__ h,
                                                              float4* __restrict__ pos_h, float4* __restrict__ vel_m,
                                                              float* __restrict__ u,
                                                              const float4* __restrict__ accel_dudt,
                                                              const float2* __restrict__ vsig_lapu,
                                                              const float* __restrict__ alpha_v,
                                                              float* __restrict__ alpha_c) {
  pdl_wait();
  __shared__ float s_min[kIntThreads / 32];
  const float dt = ck->dt;
  const float hdt = 0.5f * dt;
  const float two_cfl = 2.0f * tp.cfl;
  float dt_min = __uint_as_float(kNoBoundBits);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float4 a = accel_dudt[i];
    float4 v = vel_m[i];
    v.x = fmaf(a.x, hdt, v.x);
    v.y = fmaf(a.y, hdt, v.y);
    v.z = fmaf(a.z, hdt, v.z);
    vel_m[i] = v;
    const float ui = half_kick_u(u[i], a.w, hdt, tp.u_min_frac);
    u[i] = ui;
    const float hi = h[i];
    float4 p = pos_h[i];
    p.w = hi;
    pos_h[i] = p;
    const float H = kg * hi;
    const float2 g = vsig_lapu[i];
    if (alpha_c) {
      float ac = alpha_c[i];
      const float src = ui > 0.0f ? tp.beta_c * H * g.y * ac / sqrtf(ui) : 0.0f;
      const float dec = (ac - tp.alpha_c_min) * g.x / H;
      ac = fmaf(dt, src - dec, ac);                                           // Eq. 21
      const float av = alpha_v ? alpha_v[i] : alpha_v_const;
      ac = fminf(ac, tp.alpha_c_max * (1.0f - av / tp.alpha_v_max));          // Eqs. 24, 23
      alpha_c[i] = fmaxf(ac, tp.alpha_c_min);
    }
    if (g.x > 0.0f) dt_min = fminf(dt_min, two_cfl * H / g.x);
  }
  for (int o = 16; o > 0; o >>= 1) dt_min = fminf(dt_min, __shfl_xor_sync(0xffffffffu, dt_min, o));
  if ((threadIdx.x & 31) == 0) s_min[threadIdx.x >> 5] = dt_min;
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = s_min[0];
    for (int w = 1; w < kIntThreads / 32; ++w) m = fminf(m, s_min[w]);
    // non-negative floats order as their bit patterns
    if (__float_as_uint(m) < kNoBoundBits) atomicMin(reinterpret_cast<unsigned*>(&ck->dt_next), __float_as_uint(m));
    if (blockIdx.x == 0 && dt > 0.0f) {
      ck->t += (double)dt;
      ck->step += 1;
    }
  }
}

// One wave of resident blocks (grid-stride loops cover the rest).
int blocks_for(const Ctx* c, const void* kern, int64_t n) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kIntThreads, 0);
  if (per_sm < 1) per_sm = 1;
  const int64_t want = (n + kIntThreads - 1) / kIntThreads;
  const int64_t cap = (int64_t)c->num_sms * per_sm;
  return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

bool aligned_to(const void* p, size_t a) { return p && ((uintptr_t)p % a) == 0; }

bool valid(const swift_gpu_time_params* tp) {
  return tp && tp->cfl > 0.0f && tp->dt_max >= 0.0f && tp->alpha_v_max > 0.0f &&
         tp->alpha_v_min >= 0.0f && tp->alpha_v_min <= tp->alpha_v_max && tp->visc_length >= 0.0f &&
         tp->alpha_c_min >= 0.0f && tp->alpha_c_min <= tp->alpha_c_max && tp->beta_c >= 0.0f &&
         tp->u_min_frac >= 0.0f && tp->u_min_frac <= 1.0f;
}

int check_common(Ctx* c, const swift_gpu_time_params* tp, const void* clock, int64_t n) {
  if (!c || !valid(tp) || !aligned_to(clock, 8) || n < 0) return SWIFT_GPU_ERR_ARG;
  if (n > c->n_max) return SWIFT_GPU_ERR_CAPACITY;
  return SWIFT_GPU_OK;
}

int launched(Ctx* c) {
  c->launches++;
  return cudaGetLastError() == cudaSuccess ? SWIFT_GPU_OK : SWIFT_GPU_ERR_CUDA;
}

}  // namespace
}  // namespace sg

using namespace sg;

extern "C" {

void swift_gpu_default_time_params(swift_gpu_time_params* tp) {
  if (!tp) return;
  tp->cfl = 0.1f;
  tp->dt_max = 0.0f;
  tp->alpha_v_max = 2.0f;
  tp->alpha_v_min = 0.0f;
  tp->visc_length = 0.05f;
  tp->alpha_c_max = 1.0f;
  tp->alpha_c_min = 0.0f;
  tp->beta_c = 1.0f;
  tp->u_min_frac = 0.5f;
}

int swift_gpu_kick_drift(swift_gpu_ctx* h, const swift_gpu_time_params* tp, swift_gpu_clock* clock, int64_t n,
                         float* pos_h, float* vel_m, float* u, const float* accel_dudt, const float* dh_dt,
                         float* vel_pred, float* u_pred, void* stream) {
  Ctx* c = from(h);
  int rc = check_common(c, tp, clock, n);
  if (rc != SWIFT_GPU_OK) return rc;
  if (n > 0 && (!aligned_to(pos_h, 16) || !aligned_to(vel_m, 16) || !aligned_to(u, 4) ||
                !aligned_to(accel_dudt, 16) || (dh_dt && !aligned_to(dh_dt, 4)) || !aligned_to(vel_pred, 16) ||
                !aligned_to(u_pred, 4)))
    return SWIFT_GPU_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  launch_pdl(k_kick_drift, blocks_for(c, (const void*)k_kick_drift, n), kIntThreads, 0, s,
      *tp, clock, (int)n, c->phys.L[0], c->phys.L[1], c->phys.L[2], reinterpret_cast<float4*>(pos_h),
      reinterpret_cast<float4*>(vel_m), u, reinterpret_cast<const float4*>(accel_dudt), dh_dt,
      reinterpret_cast<float4*>(vel_pred), u_pred);
  return launched(c);
}

int swift_gpu_viscosity_switch(swift_gpu_ctx* h, const swift_gpu_time_params* tp, const swift_gpu_clock* clock,
                               int64_t n, const float* hh, const float* u, const float* curl_div,
                               const float* vsig_lapu, float* div_prev, float* alpha_v, void* stream) {
  Ctx* c = from(h);
  int rc = check_common(c, tp, clock, n);
  if (rc != SWIFT_GPU_OK) return rc;
  if (n > 0 && (!aligned_to(hh, 4) || !aligned_to(u, 4) || !aligned_to(curl_div, 16) ||
                !aligned_to(vsig_lapu, 8) || !aligned_to(div_prev, 4) || !aligned_to(alpha_v, 4)))
    return SWIFT_GPU_ERR_ARG;
  if (n == 0) return SWIFT_GPU_OK;
  cudaStream_t s = (cudaStream_t)stream;
  launch_pdl(k_viscosity_switch, blocks_for(c, (const void*)k_viscosity_switch, n), kIntThreads, 0, s,
      *tp, c->phys.gamma_eos, c->phys.kg, clock, (int)n, hh, u, reinterpret_cast<const float4*>(curl_div),
      reinterpret_cast<const float2*>(vsig_lapu), div_prev, alpha_v);
  return launched(c);
}

int swift_gpu_kick_finish(swift_gpu_ctx* h, const swift_gpu_time_params* tp, swift_gpu_clock* clock, int64_t n,
                          const float* hh, float* pos_h, float* vel_m, float* u, const float* accel_dudt,
                          const float* vsig_lapu, const float* alpha_v, float* alpha_c, void* stream) {
  Ctx* c = from(h);
  int rc = check_common(c, tp, clock, n);
  if (rc != SWIFT_GPU_OK) return rc;
  if (n > 0 && (!aligned_to(hh, 4) || !aligned_to(pos_h, 16) || !aligned_to(vel_m, 16) || !aligned_to(u, 4) ||
                !aligned_to(accel_dudt, 16) || !aligned_to(vsig_lapu, 8) || (alpha_v && !aligned_to(alpha_v, 4)) ||
                (alpha_c && !aligned_to(alpha_c, 4))))
    return SWIFT_GPU_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(&clock->dt_next, 0x7f, sizeof(float), s) != cudaSuccess) return SWIFT_GPU_ERR_CUDA;
  launch_pdl(k_kick_finish, blocks_for(c, (const void*)k_kick_finish, n), kIntThreads, 0, s,
      *tp, c->phys.kg, c->phys.alpha_v, clock, (int)n, hh, reinterpret_cast<float4*>(pos_h),
      reinterpret_cast<float4*>(vel_m), u, reinterpret_cast<const float4*>(accel_dudt),
      reinterpret_cast<const float2*>(vsig_lapu), alpha_v, alpha_c);
  return launched(c);
}

}  // extern "C"
