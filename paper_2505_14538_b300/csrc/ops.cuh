// ops.cuh -- the pair interactions of the three loops (Sec. 2.1) and the
// Newton step on h, shared by the persistent kernels (loops.cu) and the
// per-task kernels (plain.cu), so both paths do the same arithmetic.
//
// Each op has: I (the particle's state and accumulators), stage_w (what a
// staged candidate carries in .w), candidate (the cheap neighbour test with
// the guard band) and interact (the full pair term, with the exact FP64
// neighbour decision inside the guard band).
#pragma once

#include <math.h>

#include "common.cuh"

namespace sg {

struct DensOp {
  struct I {
    float x, y, z, h, H2lo, H2hi, invH, c3, c4;
    float vx, vy, vz;
    float ns, nc, rs, rc, dn, dr, div, cx, cy, cz;
    unsigned count;
    int k;
  };
  const float4* __restrict__ pos;
  const float4* __restrict__ vel;
  float L[3];
  float kg;
  int compensated;
  int kernel;
  float knorm;

  __device__ __forceinline__ float stage_w(float) const { return 0.0f; }
  __device__ __forceinline__ bool candidate(const I& i, float r2, float) const { return r2 < i.H2hi; }
  // j's two records, for loops that load several entries ahead of the arithmetic
  // (named apart from the force loops' Rec: the cell-item flush takes one entry at a time here)
  struct DRec {
    float4 pj, vj;
  };
  __device__ __forceinline__ void load_rec(int j, DRec& r) const {
    r.pj = pos[j];
    r.vj = vel[j];
  }
  __device__ __forceinline__ void interact(I& i, int j, unsigned code) const {
    DRec r;
    load_rec(j, r);
    interact(i, j, code, r);
  }
  __device__ __forceinline__ void interact(I& i, int j, unsigned code, const DRec& rec) const {
    const float4 pj = rec.pj;
    const float4 vj = rec.vj;
    float xj = pj.x, yj = pj.y, zj = pj.z;
    shift_j(code, L, xj, yj, zj);
    const float dx = i.x - xj, dy = i.y - yj, dz = i.z - zj;
    const float r2 = r2_of(dx, dy, dz);
    // j is in N_i: below the guard band in FP32, or by the exact FP64
    // decision inside it; out-of-set pairs add exact zeros (W = dW = 0)
    bool in = r2 < i.H2lo;
    if (!in && r2 < i.H2hi)
      in = exact_r2(i.x, i.y, i.z, pj.x, pj.y, pj.z, L[0], L[1], L[2]) < exact_H2(kg, i.h);
    const float invr = r2 > 0.0f ? rsqrtf(r2) : 0.0f;
    const float r = r2 * invr;
    float w, dw;
    kshape(kernel, r * i.invH, w, dw);
    const float W = in ? i.c3 * w : 0.0f;
    const float dW = in ? i.c4 * dw : 0.0f;
    const float mj = vj.w;
    if (compensated) {
      two_sum_acc(i.ns, i.nc, W);
      two_sum_acc(i.rs, i.rc, mj * W);
    } else {
      i.ns += W;
      i.rs = fmaf(mj, W, i.rs);
    }
    const float t = fmaf(r, dW, 3.0f * W);
    i.dn += t;
    i.dr = fmaf(mj, t, i.dr);
    const float g = mj * dW * invr;
    const float dvx = vj.x - i.vx, dvy = vj.y - i.vy, dvz = vj.z - i.vz;
    i.div = fmaf(g, fmaf(dvz, dz, fmaf(dvy, dy, dvx * dx)), i.div);
    i.cx = fmaf(-g, fmaf(dvy, dz, -dvz * dy), i.cx);
    i.cy = fmaf(-g, fmaf(dvz, dx, -dvx * dz), i.cy);
    i.cz = fmaf(-g, fmaf(dvx, dy, -dvy * dx), i.cz);
    i.count += (in && j != i.k) ? 1u : 0u;
  }
};

__device__ __forceinline__ void dens_set_h(DensOp::I& I, float h, float kg, float knorm, float Lmax) {
  I.h = h;
  const float H = kg * h;
  const float b = band_of(H, Lmax);
  I.H2lo = H * H - b;
  I.H2hi = H * H + b;
  I.invH = 1.0f / H;
  I.c3 = knorm * I.invH * I.invH * I.invH;
  I.c4 = I.c3 * I.invH;
}

// One step of the Newton iteration on F(h) = n - (eta/h)^3 (Sec. 2.1.2) from
// the compensated sum n = ns + nc and dn_acc = sum(3W + r dW/dr) at h.
// Convergence |n h^3 - eta^3| <= h_tol eta^3 is decided as in FP64 (no division);
// the step itself, F' = dn/dh + 3 eta^3 / h^4 clamped to [h/2, 2h] with
// bisection on the bracket [lo, hi], is FP32. h never exceeds hcap (the cell
// or leaf cap); a particle that needs more is finished with flag cap_flag.
// Returns true with hn set when another evaluation is needed; false when the
// particle is finished (flag 0: converged; otherwise not converged / capped).
__device__ __forceinline__ bool newton_step(float h, float ns, float nc, float dn_acc, float& lo, float& hi,
                                            float hcap, int cap_flag, const Phys& ph, bool last, float& hn,
                                            int& flag) {
  flag = 0;
  // G = (ns + nc) h^3 - eta^3 in FP32 first: its error is below 8 ulp of
  // max(n h^3, eta^3), so outside that margin around the tolerance both the
  // convergence decision and the sign of G are those of the FP64 value;
  // inside it (rare) G is taken in FP64.
  const float e3 = (float)ph.eta3;
  const float n32 = ns + nc;
  const float h3f = h * h * h;
  const float Gf = fmaf(n32, h3f, -e3);
  const float tol = (float)(ph.h_tol * ph.eta3);
  const float margin = 4.76837158203125e-7f * fmaxf(n32 * h3f, e3);  // 8 * 2^-24
  bool conv, neg;
  if (fabsf(Gf) + margin <= tol) {
    conv = true;
    neg = false;
  } else if (fabsf(Gf) - margin > tol) {
    conv = false;
    neg = Gf < 0.0f;
  } else {
    const double hd = (double)h;
    const double h3 = hd * hd * hd;
    const double G = fma((double)ns, h3, fma((double)nc, h3, -ph.eta3));
    conv = fabs(G) <= ph.h_tol * ph.eta3;
    neg = G < 0.0;
  }
  if (conv) return false;
  if (last) {
    flag = SWIFT_GPU_ERR_H_NOT_CONVERGED;
    return false;
  }
  if (neg) lo = fmaxf(lo, h);
  else hi = fminf(hi, h);
  if (neg && h >= hcap) {
    flag = cap_flag;
    return false;
  }
  const float ih = 1.0f / h;
  const float target = (float)ph.eta3 * ih * ih * ih;
  const float F = (ns + nc) - target;
  const float Fp = fmaf(-dn_acc, ih, 3.0f * target * ih);
  hn = Fp > 0.0f ? h - F / Fp : __int_as_float(0x7fc00000);
  if (hn == hn) hn = fminf(fmaxf(hn, 0.5f * h), 2.0f * h);
  if (!(hn == hn) || !(hn > lo) || !(hn < hi)) {
    if (isfinite(hi) && lo > 0.0f) hn = 0.5f * (lo + hi);
    else if (!isfinite(hi)) hn = 2.0f * h;
    else hn = 0.5f * h;
  }
  hn = fminf(hn, hcap);
  return hn != h;  // a float h that cannot move is as converged as FP32 allows
}

struct GradOp {
  struct I {
    float x, y, z, h, H2lo, H2hi, invH, c4;
    float vx, vy, vz, c, u;
    float vsig, lap;
    unsigned count;
    int k;
  };
  const float4* __restrict__ pos;
  const float4* __restrict__ vel;
  const float4* __restrict__ ga;
  const float4* __restrict__ gb;
  float L[3];
  float kg, beta;
  int kernel;
  float knorm;

  __device__ __forceinline__ float stage_w(float) const { return 0.0f; }
  __device__ __forceinline__ bool candidate(const I& i, float r2, float) const { return r2 < i.H2hi; }
  __device__ __forceinline__ void interact(I& i, int j, unsigned code) const {
    const float4 pj = pos[j];
    float xj = pj.x, yj = pj.y, zj = pj.z;
    shift_j(code, L, xj, yj, zj);
    const float dx = i.x - xj, dy = i.y - yj, dz = i.z - zj;
    const float r2 = r2_of(dx, dy, dz);
    if (!(r2 > 0.0f)) return;  // the particle itself: its v_sig term is added at load
    if (r2 >= i.H2lo) {
      if (r2 >= i.H2hi) return;  // outside the support (entries of a stored list may be)
      if (!(exact_r2(i.x, i.y, i.z, pj.x, pj.y, pj.z, L[0], L[1], L[2]) < exact_H2(kg, i.h))) return;
    }
    const float4 vj = vel[j];
    const float4 aj = ga[j];
    const float uj = gb[j].w;
    const float invr = rsqrtf(r2);
    const float r = r2 * invr;
    const float dW = i.c4 * dkshape(kernel, r * i.invH);
    const float dvx = i.vx - vj.x, dvy = i.vy - vj.y, dvz = i.vz - vj.z;
    const float vr = fmaf(dvz, dz, fmaf(dvy, dy, dvx * dx)) * invr;
    const float mu = fminf(vr, 0.0f);
    i.vsig = fmaxf(i.vsig, fmaf(-beta, mu, i.c + aj.w));
    i.lap = fmaf(__fdividef(vj.w, aj.z) * (i.u - uj), dW * invr, i.lap);
    i.count += 1u;
  }
};

struct ForceOp {
  struct I {
    float x, y, z, h, H2lo, H2hi, invH, c4;
    float vx, vy, vz;
    float A, f, rho, c, B, av, acP, u, P;
    float axs, axc, ays, ayc, azs, azc, dus, duc, dh;
    unsigned count;
    int k;
  };
  const float4* __restrict__ pos;
  const float4* __restrict__ vel;
  const float4* __restrict__ ga;
  const float4* __restrict__ gb;
  float L[3];
  float kg, beta, gm1, Lmax;
  int compensated;
  int kernel;
  float knorm;

  // staged w: the j support squared plus its guard band
  __device__ __forceinline__ float stage_w(float hj) const {
    const float H = kg * hj;
    return H * H + band_of(H, Lmax);
  }
  __device__ __forceinline__ bool candidate(const I& i, float r2, float H2j_hi) const {
    return r2 < fmaxf(i.H2hi, H2j_hi);
  }
  __device__ __forceinline__ void interact(I& i, int j, unsigned code) const {
    const float4 pj = pos[j];
    float xj = pj.x, yj = pj.y, zj = pj.z;
    shift_j(code, L, xj, yj, zj);
    const float dx = i.x - xj, dy = i.y - yj, dz = i.z - zj;
    const float r2 = r2_of(dx, dy, dz);
    if (!(r2 > 0.0f)) return;  // the particle itself
    const float Hj = kg * pj.w;
    const float bj_band = band_of(Hj, Lmax);
    if (r2 >= fmaxf(i.H2lo, Hj * Hj - bj_band)) {
      if (r2 >= fmaxf(i.H2hi, Hj * Hj + bj_band)) return;  // outside both supports
      const double e = exact_r2(i.x, i.y, i.z, pj.x, pj.y, pj.z, L[0], L[1], L[2]);
      if (!(e < exact_H2(kg, i.h)) && !(e < exact_H2(kg, pj.w))) return;
    }
    const float4 vj = vel[j];
    const float4 aj = ga[j];  // (A, f, rho, c)
    const float4 bj = gb[j];  // (B, alpha_v, alpha_c P, u)
    const float invr = rsqrtf(r2);
    const float r = r2 * invr;
    const float ex = dx * invr, ey = dy * invr, ez = dz * invr;
    const float dWi = i.c4 * dkshape(kernel, r * i.invH);
    const float invHj = __fdividef(1.0f, Hj);
    const float ih2 = invHj * invHj;
    const float dWj = (knorm * ih2 * ih2) * dkshape(kernel, r * invHj);
    const float dvx = i.vx - vj.x, dvy = i.vy - vj.y, dvz = i.vz - vj.z;
    const float vr = fmaf(dvz, ez, fmaf(dvy, ey, dvx * ex));
    const float mj = vj.w;
    const float fsum = fmaf(i.f, dWi, aj.y * dWj);
    // pressure (Eq. 17) and its work (Eq. 18)
    const float ps = mj * fmaf(i.A, dWi, aj.x * dWj);
    float du = mj * i.A * dWi * vr;
    // artificial viscosity (Eqs. 7, 9-11, 16) and its heating
    const float mu = fminf(vr, 0.0f);
    const float vsig = fmaf(-beta, mu, i.c + aj.w);
    const float alpha = 0.25f * (i.av + bj.y) * (i.B + bj.x);
    const float irs = __fdividef(1.0f, i.rho + aj.z);
    const float nu = -alpha * mu * vsig * irs;
    const float vs = 0.5f * mj * nu * fsum;
    du = fmaf(0.5f * vs, vr, du);
    // artificial conduction (Eqs. 19, 20, 22)
    const float Pj = gm1 * aj.z * bj.w;
    const float Ps = i.P + Pj;
    const float ac = Ps > 0.0f ? __fdividef(i.acP + bj.z, Ps) : 0.0f;
    const float dP = 2.0f * fabsf(i.P - Pj) * irs;
    const float vc = fabsf(vr) + (dP > 0.0f ? dP * rsqrtf(dP) : 0.0f);
    du = fmaf(ac * vc * mj * (i.u - bj.w), fsum * irs, du);
    const float as = ps + vs;
    if (compensated) {
      two_sum_acc(i.axs, i.axc, -as * ex);
      two_sum_acc(i.ays, i.ayc, -as * ey);
      two_sum_acc(i.azs, i.azc, -as * ez);
      two_sum_acc(i.dus, i.duc, du);
    } else {
      i.axs = fmaf(-as, ex, i.axs);
      i.ays = fmaf(-as, ey, i.ays);
      i.azs = fmaf(-as, ez, i.azs);
      i.dus += du;
    }
    i.dh = fmaf(mj * dWi, vr, i.dh);
    i.count += 1u;
  }
};

// The gradient and force loops in one pass over the same pairs: the force
// pair set (r < max(H_i, H_j)) is a superset of the gradient's (r < H_i), so
// one interaction evaluates the force terms and, for r < H_i, the gradient
// terms with the gradient loop's own expressions (identical results to the
// two loops run one after the other).
struct GradForceOp : ForceOp {
  struct I : ForceOp::I {
    float vsig, lap;
    unsigned gcount;
  };
  __device__ __forceinline__ bool candidate(const I& i, float r2, float H2j_hi) const {
    return ForceOp::candidate(i, r2, H2j_hi);
  }
  // The four records of particle j, loaded ahead of the arithmetic.
  struct Rec {
    float4 pj, vj, aj, bj;
  };
  __device__ __forceinline__ void load(int j, Rec& r) const {
    r.pj = pos[j];
    r.vj = vel[j];
    r.aj = ga[j];
    r.bj = gb[j];
  }
  __device__ __forceinline__ void interact(I& i, int j, unsigned code) const {
    Rec r;
    load(j, r);
    interact(i, j, code, r);
  }
  __device__ __forceinline__ void interact(I& i, int j, unsigned code, const Rec& rec) const {
    float t[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    interact_acc(i, j, code, rec, t);
    commit(i, t);
  }
  // The pair term with its momentum and energy terms added to t (a_x, a_y,
  // a_z, du/dt) instead of the compensated sums, which commit() then takes.
  // 1/r is folded into the scalar factors, and the gradient terms are masked
  // by r < H_i instead of taken in a branch.
  __device__ __forceinline__ void interact_acc(I& i, int j, unsigned code, const Rec& rec, float (&t)[4]) const {
    const float4 pj = rec.pj;
    float xj = pj.x, yj = pj.y, zj = pj.z;
    shift_j(code, L, xj, yj, zj);
    const float dx = i.x - xj, dy = i.y - yj, dz = i.z - zj;
    const float r2 = r2_of(dx, dy, dz);
    if (!(r2 > 0.0f)) return;  // the particle itself
    const float Hj = kg * pj.w;
    const float bj_band = band_of(Hj, Lmax);
    // membership in i's support (gradient) and in either support (force),
    // in FP32 where the guard band allows, else in FP64 from the same floats
    bool in_i = r2 < i.H2lo;
    bool in_f = in_i || r2 < Hj * Hj - bj_band;
    if (!in_f) {
      if (r2 >= fmaxf(i.H2hi, Hj * Hj + bj_band)) return;  // outside both supports
      const double e = exact_r2(i.x, i.y, i.z, pj.x, pj.y, pj.z, L[0], L[1], L[2]);
      in_i = e < exact_H2(kg, i.h);
      in_f = in_i || e < exact_H2(kg, pj.w);
      if (!in_f) return;
    } else if (!in_i && r2 < i.H2hi) {
      in_i = exact_r2(i.x, i.y, i.z, pj.x, pj.y, pj.z, L[0], L[1], L[2]) < exact_H2(kg, i.h);
    }
    const float4 vj = rec.vj;
    const float4 aj = rec.aj;  // (A, f, rho, c)
    const float4 bj = rec.bj;  // (B, alpha_v, alpha_c P, u)
    const float invr = rsqrtf(r2);
    const float r = r2 * invr;
    const float dWi = i.c4 * dkshape(kernel, r * i.invH);
    const float dvx = i.vx - vj.x, dvy = i.vy - vj.y, dvz = i.vz - vj.z;
    const float vr = fmaf(dvz, dz, fmaf(dvy, dy, dvx * dx)) * invr;
    const float mu = fminf(vr, 0.0f);
    const float vsig = fmaf(-beta, mu, i.c + aj.w);
    // gradient loop (as GradOp), for r < H_i
    i.vsig = in_i ? fmaxf(i.vsig, vsig) : i.vsig;
    const float lt = __fdividef(vj.w, aj.z) * (i.u - bj.w) * (dWi * invr);
    i.lap += in_i ? lt : 0.0f;
    i.gcount += in_i ? 1u : 0u;
    const float invHj = __fdividef(1.0f, Hj);
    const float ih2 = invHj * invHj;
    const float dWj = (knorm * ih2 * ih2) * dkshape(kernel, r * invHj);
    const float mj = vj.w;
    const float fsum = fmaf(i.f, dWi, aj.y * dWj);
    // pressure (Eq. 17) and its work (Eq. 18)
    const float ps = mj * fmaf(i.A, dWi, aj.x * dWj);
    // artificial viscosity (Eqs. 7, 9-11, 16) and its heating: the viscous term is
    // vs = 0.5 m_j nu fsum with nu = -(1/4)(alpha_i + alpha_j)(B_i + B_j) mu v_sig / (rho_i + rho_j);
    // vsh = vs / 2 folds the constants into one factor, -1/16
    const float a16 = -0.0625f * (i.av + bj.y) * (i.B + bj.x);
    const float irs = __fdividef(1.0f, i.rho + aj.z);
    const float vsh = mj * fsum * (a16 * mu * vsig * irs);
    float du = vr * fmaf(mj * i.A, dWi, vsh);
    // artificial conduction (Eqs. 19, 20, 22)
    const float Pj = gm1 * aj.z * bj.w;
    const float Ps = i.P + Pj;
    const float ac = Ps > 0.0f ? __fdividef(i.acP + bj.z, Ps) : 0.0f;
    const float dP = 2.0f * fabsf(i.P - Pj) * irs;
    const float vc = fabsf(vr) + sqrt_approx(dP);  // exact at dP = 0
    du = fmaf(ac * vc * mj * (i.u - bj.w), fsum * irs, du);
    const float asr = fmaf(2.0f, vsh, ps) * invr;
    t[0] = fmaf(-asr, dx, t[0]);
    t[1] = fmaf(-asr, dy, t[1]);
    t[2] = fmaf(-asr, dz, t[2]);
    t[3] += du;
    i.dh = fmaf(mj * dWi, vr, i.dh);
    i.count += 1u;
  }
  __device__ __forceinline__ void commit(I& i, const float (&t)[4]) const {
    if (compensated) {
      two_sum_acc(i.axs, i.axc, t[0]);
      two_sum_acc(i.ays, i.ayc, t[1]);
      two_sum_acc(i.azs, i.azc, t[2]);
      two_sum_acc(i.dus, i.duc, t[3]);
    } else {
      i.axs += t[0];
      i.ays += t[1];
      i.azs += t[2];
      i.dus += t[3];
    }
  }
};

}  // namespace sg
