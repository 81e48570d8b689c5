// force_lpp.cuh -- the force pair term (Sec. 2.1.4: Eqs. 7, 9-11, 16-20, 22,
// with the gradient loop's Eqs. 10-11 and Laplacian of u fused in) for the
// lane-per-particle loop over kept lists, written for instruction count:
//
//  - four 16-byte records a neighbour: the ghost step writes each particle's
//    position with 1/H in place of h, and a pair derives C/H_j^4 and the two
//    bounds of H_j^2's guard band from 1/H_j (a few FP32 operations cost less
//    than a fifth record's gather); h_j itself is read only inside the guard
//    band, where the decision is taken in FP64;
//  - 1/r is folded into the scalar factors (a_i -= (as/r) dx instead of
//    as * (dx/r));
//  - the gradient terms are masked by the exact r < H_i decision instead of
//    taken in a branch;
//  - compensation is blocked: the loop adds the terms of four entries in FP32
//    and carries that sum into the running TwoSum (Knuth) pair, which bounds
//    the error of a sum by a few times 2^-24 times the sum of the terms'
//    magnitudes, far below the 1e-4-of-the-force-scale tolerance.
//
// Same pair set and the same exact neighbour decisions as ForceOp and
// GradForceOp (ops.cuh): FP32 where the guard band allows, FP64 inside it.
#pragma once

#include "common.cuh"

namespace sg {

// The four records of neighbour j.
struct LeanRec {
  float4 p;   // (x, y, z, 1/H): the ghost step's position record
  float4 v;   // (vx, vy, vz, m)
  float4 ga;  // (A = f P / rho^2, f, rho, c)
  float4 gb;  // (B, alpha_v, alpha_c P, u)
};

__device__ __forceinline__ void lean_load(const float4* __restrict__ xih, const float4* __restrict__ vel,
                                          const float4* __restrict__ ga, const float4* __restrict__ gb, int j,
                                          LeanRec& r) {
  r.p = xih[j];
  r.v = vel[j];
  r.ga = ga[j];
  r.gb = gb[j];
}

// The particle's state and sums.
struct LeanI {
  float x, y, z, h, H2lo, H2hi, invH, c4;
  float vx, vy, vz;
  float A, f, rho, c, B, av, acP, u, P;
  float axs, axc, ays, ayc, azs, azc, dus, duc, dh;
  float vsig, lap;
  unsigned gcount, count;
};

// The run's constants, read from the kernel's parameters (constant bank) where
// used; pos: the sorted (x, y, z, h) records, for h_j inside the guard band.
struct LeanConst {
  const Phys& ph;
  float Lmax;
  const float4* __restrict__ pos;
  __device__ __forceinline__ float gm1() const { return ph.gamma_eos - 1.0f; }
};

// One kept-list entry (j with shift code) of particle I: the pair terms go
// into the block sums (tax, tay, taz, tdu); the rest straight into I.
template <int K, bool kGrad>
__device__ __forceinline__ void lean_pair(LeanI& I, const LeanRec& R, int j, unsigned code, const LeanConst& k,
                                          float& tax, float& tay, float& taz, float& tdu) {
  float xj = R.p.x, yj = R.p.y, zj = R.p.z;
  // j's support from 1/H_j: the band bounds need H_j^2 only to within a small
  // part of the band (2^-16 H^2), so an approximate reciprocal serves
  const float iHj = R.p.w;
  const float Hj = __fdividef(1.0f, iHj);
  // band_of(Hj, Lmax) as Hj (2^-16 Hj + 2^-20 Lmax): the same band to rounding, two operations
  const float bdj = Hj * fmaf(Hj, 1.52587890625e-05f, k.Lmax * 9.5367431640625e-07f);
  const float H2lo_j = fmaf(Hj, Hj, -bdj), H2hi_j = fmaf(Hj, Hj, bdj);
  shift_j(code, k.ph.L, xj, yj, zj);
  const float dx = I.x - xj, dy = I.y - yj, dz = I.z - zj;
  const float r2 = r2_of(dx, dy, dz);
  // membership in i's support (gradient) and in either support (force): FP32
  // outside the guard bands, the FP64 definition from the same floats inside
  bool in_i = r2 < I.H2lo;
  bool in_f = in_i || r2 < H2lo_j;
  const bool band_f = !in_f && r2 < fmaxf(I.H2hi, H2hi_j);
  const bool band_i = kGrad && in_f && !in_i && r2 < I.H2hi;
  if (band_f || band_i) {
    const double e = exact_r2(I.x, I.y, I.z, R.p.x, R.p.y, R.p.z, k.ph.L[0], k.ph.L[1], k.ph.L[2]);
    const bool ei = e < exact_H2(k.ph.kg, I.h);
    in_i = ei;
    in_f = in_f || ei || e < exact_H2(k.ph.kg, k.pos[j].w);
  }
  if (!(r2 > 0.0f) || !in_f) return;  // the particle itself, or outside both supports
  const float invr = rsqrtf(r2);
  const float r = r2 * invr;
  const float dWi = I.c4 * dkshape(K, r * I.invH);
  const float i2j = iHj * iHj;
  const float dWj = k.ph.knorm * (i2j * i2j) * dkshape(K, r * iHj);
  const float dvx = I.vx - R.v.x, dvy = I.vy - R.v.y, dvz = I.vz - R.v.z;
  const float vr = fmaf(dvz, dz, fmaf(dvy, dy, dvx * dx)) * invr;
  const float mj = R.v.w;
  const float fsum = fmaf(I.f, dWi, R.ga.y * dWj);
  const float mu = fminf(vr, 0.0f);
  const float vsig = fmaf(-k.ph.beta_v, mu, I.c + R.ga.w);
  if constexpr (kGrad) {  // gradient loop: v_sig,max and the Laplacian of u (r < H_i)
    I.vsig = in_i ? fmaxf(I.vsig, vsig) : I.vsig;
    const float lt = __fdividef(mj, R.ga.z) * (I.u - R.gb.w) * (dWi * invr);
    I.lap += in_i ? lt : 0.0f;
    I.gcount += in_i ? 1u : 0u;
  }
  // pressure (Eq. 17) and its work (Eq. 18)
  const float ps = mj * fmaf(I.A, dWi, R.ga.x * dWj);
  // artificial viscosity (Eqs. 7, 9-11, 16) and its heating: the viscous term is
  // vs = 0.5 m_j nu fsum with nu = -(1/4)(alpha_i + alpha_j)(B_i + B_j) mu v_sig / (rho_i + rho_j);
  // vsh = vs / 2 folds the constants into one factor, -1/16
  const float irs = __fdividef(1.0f, I.rho + R.ga.z);
  const float a16 = -0.0625f * (I.av + R.gb.y) * (I.B + R.gb.x);
  const float vsh = mj * fsum * (a16 * mu * vsig * irs);
  float du = vr * fmaf(mj * I.A, dWi, vsh);
  // artificial conduction (Eqs. 19, 20, 22)
  const float Pj = k.gm1() * R.ga.z * R.gb.w;
  const float Ps = I.P + Pj;
  const float ac = Ps > 0.0f ? __fdividef(I.acP + R.gb.z, Ps) : 0.0f;
  const float dP = 2.0f * fabsf(I.P - Pj) * irs;
  const float vc = fabsf(vr) + sqrt_approx(dP);  // exact at dP = 0
  du = fmaf(ac * vc * mj * (I.u - R.gb.w), fsum * irs, du);
  const float asr = fmaf(2.0f, vsh, ps) * invr;
  tax = fmaf(-asr, dx, tax);
  tay = fmaf(-asr, dy, tay);
  taz = fmaf(-asr, dz, taz);
  tdu += du;
  I.dh = fmaf(mj * dWi, vr, I.dh);
  I.count += 1u;
}

}  // namespace sg
