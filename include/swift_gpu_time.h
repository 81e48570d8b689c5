/*
 * swift_gpu_time.h -- time integration and switch evolution of the SPH
 * library (C ABI), on top of swift_gpu.h.
 *
 * The paper's solver advances the particles with "kick" and "drift" tasks
 * (Sec. 2.2.2) and evolves the artificial viscosity and conduction
 * coefficients between steps (Sec. 2.1.3, Eqs. 12-15; Sec. 2.1.4, Eqs. 21,
 * 23, 24). These are O(N) per-particle kernels, one grid-stride pass each,
 * in the caller's particle order; they read the outputs of the pair loops of
 * swift_gpu.h.
 *
 * One step of the kick-drift-kick leapfrog with a global time step:
 *   swift_gpu_kick_drift        half kick, drift, prediction (the step's dt is fixed here)
 *   swift_gpu_build_cells, swift_gpu_density     at the drifted positions, predicted velocities
 *   swift_gpu_viscosity_switch  alpha_v from the change of div v (Eqs. 12-15)
 *   swift_gpu_gradient_force    with the predicted u and the new alpha_v
 *   swift_gpu_kick_finish       second half kick, alpha_c (Eqs. 21, 23, 24), next dt
 * The step size lives in a caller-owned device clock, so the whole sequence
 * can be captured in a CUDA graph and replayed without host synchronisation.
 *
 * Readings of the paper (it fixes neither the integrator nor the step):
 *  - half kick: v += a dt/2, u += (du/dt) dt/2 but never below u_min_frac u;
 *    drift: x += v dt wrapped into [0, L), h *= exp((dh/dt) dt / h); the loops
 *    of the step see the predicted v + a dt/2 and u + (du/dt) dt/2 (the same
 *    floor), the second half kick uses the new rates;
 *  - dt = min over particles of cfl * 2 H_i / v_sig,i (H = kernel_gamma h,
 *    v_sig from the gradient loop; particles with v_sig = 0 set no bound),
 *    capped by dt_max and by the time left to t_end;
 *  - Eq. 15: d(div v)/dt = (div v now - div v at the previous step) / dt;
 *    Eq. 14: S = H^2 max(0, -d(div v)/dt);
 *    Eq. 13: alpha_loc = alpha_v_max S / (v_sig^2 + S) with the particle's
 *    v_sig of the previous gradient loop (the printed trailing dt dropped);
 *    Eq. 12: alpha_v = alpha_loc when alpha_loc >= alpha_v, else
 *    alpha_loc + (alpha_v - alpha_loc) exp(-visc_length c dt / H), kept in
 *    [alpha_v_min, alpha_v_max]; c = sqrt(gamma (gamma - 1) u);
 *  - Eq. 21 as printed, one forward-Euler step:
 *    alpha_c += dt (beta_c H lap(u) alpha_c / sqrt(u) - (alpha_c - alpha_c_min) v_sig / H),
 *    source term only where u > 0 (u after the second half kick);
 *    Eq. 24: cap = alpha_c_max (1 - alpha_v / alpha_v_max); Eq. 23: alpha_c <= cap;
 *    then alpha_c >= alpha_c_min.
 *
 * Conventions as in swift_gpu.h: caller-owned DEVICE pointers aligned to their
 * element size, the stream as void*, a negative SWIFT_GPU_ERR_* on a host-side
 * error (ERR_ARG: null or misaligned pointer, n < 0 or n > the context's
 * n_max, invalid parameters). All n particles are integrated (global step).
 */
#ifndef SWIFT_GPU_TIME_H
#define SWIFT_GPU_TIME_H

#include "swift_gpu.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  float cfl;           /* dt_i = cfl * 2 H_i / v_sig,i (0.1) */
  float dt_max;        /* upper bound on dt; 0 = none */
  float alpha_v_max;   /* Eqs. 13, 24 (2.0) */
  float alpha_v_min;   /* lower bound of alpha_v (0.0) */
  float visc_length;   /* l of Eq. 12 (0.05) */
  float alpha_c_max;   /* Eqs. 23, 24 (1.0) */
  float alpha_c_min;   /* Eq. 21 (0.0) */
  float beta_c;        /* Eq. 21 (1.0) */
  float u_min_frac;    /* a half kick keeps u >= u_min_frac u (0.5) */
} swift_gpu_time_params;

/* Device-resident integration clock, 32 bytes, owned by the caller (e.g. a
 * 32-byte device buffer). The caller writes it once (t = 0, t_end, dt = 0,
 * dt_next = 0, step = 0); a first swift_gpu_kick_finish with dt = 0 after
 * the loops at the initial state fills dt_next, and the calls below keep it
 * up to date on the device. */
typedef struct {
  double t;        /* time reached by the completed steps */
  double t_end;    /* > 0: the step is cut so that t never passes t_end (dt = 0 once there) */
  float dt;        /* step size of the step in progress (written by swift_gpu_kick_drift) */
  float dt_next;   /* minimum of cfl 2 H_i / v_sig,i of the last swift_gpu_kick_finish
                      (3.39e38 when no particle bounds it) */
  int64_t step;    /* completed steps with dt > 0 */
} swift_gpu_clock;

/* Fill *tp with the defaults listed above. Host only; never fails. */
void swift_gpu_default_time_params(swift_gpu_time_params* tp);

/* First half of a leapfrog step (Sec. 2.2.2 "kick" and "drift").
 * dt = min(clock->dt_next, tp->dt_max if > 0, clock->t_end - clock->t if
 * t_end > 0), at least 0; written to clock->dt. Per particle i < n:
 *   vel_m.xyz += a dt/2; u <- max(u + (du/dt) dt/2, u_min_frac u);
 *   pos_h.xyz += vel_m.xyz dt, wrapped into [0, L) of the context's box;
 *   pos_h.w *= exp(dh_dt dt / pos_h.w) (dh_dt may be NULL: h unchanged);
 *   vel_pred = (vel_m.xyz + a dt/2, m); u_pred = max(u + (du/dt) dt/2, u_min_frac u)
 * with a, du/dt from accel_dudt (float4, the last force loop). pos_h, vel_m,
 * u are updated in place; vel_pred (float4) and u_pred are outputs that the
 * step's density and gradient/force calls take as vel_m and u. */
int swift_gpu_kick_drift(swift_gpu_ctx* ctx, const swift_gpu_time_params* tp, swift_gpu_clock* clock, int64_t n,
                         float* pos_h, float* vel_m, float* u, const float* accel_dudt, const float* dh_dt,
                         float* vel_pred, float* u_pred, void* stream);

/* Viscosity switch (Eqs. 12-15) with dt = clock->dt, per particle i < n:
 * h[i] the final smoothing length of the step's density call, u[i] the
 * internal energy the loops see (u_pred), curl_div[i].w the new div v,
 * vsig_lapu[i].x the v_sig of the previous gradient loop; div_prev[i] holds
 * div v of the previous step on entry and the new div v on return;
 * alpha_v[i] is updated in place. With dt = 0 only div_prev is written. */
int swift_gpu_viscosity_switch(swift_gpu_ctx* ctx, const swift_gpu_time_params* tp, const swift_gpu_clock* clock,
                               int64_t n, const float* h, const float* u, const float* curl_div,
                               const float* vsig_lapu, float* div_prev, float* alpha_v, void* stream);

/* Second half of the step with dt = clock->dt, per particle i < n:
 *   vel_m.xyz += a dt/2; u <- max(u + (du/dt) dt/2, u_min_frac u);
 *   pos_h.w = h[i] (the step's final smoothing length);
 *   alpha_c (may be NULL: not evolved): Eqs. 21, 24, 23 with lap(u) and
 *   v_sig from vsig_lapu (this step's gradient loop) and alpha_v[i] (NULL:
 *   the context's constant alpha_v);
 * then clock->dt_next = min_i cfl 2 kernel_gamma h[i] / v_sig,i, clock->t +=
 * dt and clock->step += 1 when dt > 0. With dt = 0 (clock->dt = 0) it only
 * sets pos_h.w and dt_next: the call that starts an integration. */
int swift_gpu_kick_finish(swift_gpu_ctx* ctx, const swift_gpu_time_params* tp, swift_gpu_clock* clock, int64_t n,
                          const float* h, float* pos_h, float* vel_m, float* u, const float* accel_dudt,
                          const float* vsig_lapu, const float* alpha_v, float* alpha_c, void* stream);

#ifdef __cplusplus
}
#endif

#endif
