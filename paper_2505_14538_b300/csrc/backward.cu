// backward.cu -- adjoint of the density + ghost + force loops (not in the
// paper): for a loss L = sum_i w_i . a_i + c_i du_i/dt of the last force call,
// the gradients dL/dx, dL/dv, dL/du at fixed smoothing lengths (h_mode 0), or
// with each h_i the root of the h iteration (h_mode 1, Sec. 2.1.2).
//
// Two gather passes, each scanning the 27 neighbour cells of the forward
// call's cell items again (no atomics, and no pair list of the forward call
// is read: the candidates are recomputed; the per-particle density sums of
// the forward call are reused):
//   k_force_adj  for particle k and every force pair (r < max(H_k, H_j)), the
//                pair term is evaluated forward and then in reverse in both
//                orientations: k as the first particle (weights w_k, c_k) and
//                k as the second particle of j's sum (weights w_j, c_j). This
//                gives the direct dL/dx_k, dL/dv_k, dL/du_k and the adjoints
//                of k's per-particle inputs (A, f, rho, c, B, P, alpha_c P, u);
//                the ghost step (Eq. 8, EOS, Balsara) is then reversed per
//                particle into adjoints of rho, D = sum m (3W + r dW/dr),
//                S = rho div v and C = rho curl v.
//   k_dens_adj   for particle k and every pair in k's or j's density sums,
//                the adjoints of rho, D, S, C of both particles are carried to
//                dL/dx_k and dL/dv_k, and the totals go to caller order.
// With h_mode 1 the same two passes also collect dL/dh_k at fixed x: through
// dW(r, h_k) in the force pairs (both orientations), the 1/h_k of the
// Balsara switch, and the h-derivatives of k's own sums rho, D, S, C. Since
// F_k = n_k(x, h_k) - (eta/h_k)^3 = 0 defines h_k and n_k depends on h_k
// alone, the implicit function theorem gives the extra term
//   dL/dx_k -= sum_j (lambda_k dW(r,h_k)/dr + lambda_j dW(r,h_j)/dr) e_kj,
//   lambda = (dL/dh) / F',  F' = dn/dh + 3 eta^3 / h^4,
// gathered by a third pass, k_ift_adj.
#include <cuda_runtime.h>
#include <math.h>

#include "common.cuh"
#include "engine.cuh"
#include "internal.h"

namespace sg {

constexpr int kAdjThreads = 128;
constexpr size_t kAdjSmemBytes = sizeof(WarpSmem) * (kAdjThreads / 32);

__device__ __forceinline__ WarpSmem& adj_smem(unsigned char* smem) {
  return reinterpret_cast<WarpSmem*>(smem)[threadIdx.x >> 5];
}

struct AdjArgs {
  int hmode;           // 1: h = h(x), collect dL/dh and lambda
  Grid* grid;
  Nbr nb;
  const unsigned* perm;
  Phys ph;
  int lmax;
  const float4* pos;   // sorted (x, h)
  const float4* vel;   // sorted (v, m)
  const float4* rho4;  // sorted (rho, drho/dh, n, dn/dh)
  const float4* cd;    // sorted (curl, div)
  const float4* ga;    // sorted (A, f, rho, c)
  const float4* gb;    // sorted (B, alpha_v, alpha_c P, u)
  const float4* g4;    // sorted loss weights (w, c)
  float4* xb;          // sorted: dL/dx direct (xyz), dL/du total (w)
  float4* vb;          // sorted: dL/dv direct
  float4* qb;          // sorted: adjoints of (rho, D, S, C_x)
  float* cby;          // sorted: adjoint of C_y
  float* lam;          // sorted: lambda = (dL/dh) / F' (h_mode 1)
  float* cbz;          // sorted: adjoint of C_z
  const Item* items;
  const int* plist;
  const int* ctr;
  int* ticket;
  float4* grad_x;      // caller order
  float4* grad_v;
  float* grad_u;
};

// One side of a force pair: the per-particle inputs and, after the reverse
// sweep, their adjoints.
struct Side {
  float A, f, rho, c, B, av, acP, u, P;
};
struct SideBar {
  float A, f, rho, c, B, acP, u, P;
};

// Forward and reverse of one force pair term for the loss lw . a + lc du of
// the FIRST particle: a_first -= as e, du_first += du1 + du2 + du3 (the same
// arithmetic as the force loop, Eqs. 7, 9-11, 16-20, 22). Outputs: adjoints
// w.r.t. d = x_first - x_second, v = v_first - v_second, and both sides.
__device__ __forceinline__ void pair_reverse(const Side& I, const Side& J, float mj, float r, const float e[3],
                                             float dWi, float dWj, float d2Wi, float d2Wj, const float v[3],
                                             const float lw[3], float lc, float beta, float dbar[3], float vbar[3],
                                             SideBar& Ib, SideBar& Jb, float& dWib_out, float& dWjb_out) {
  // forward values needed by the reverse sweep
  const float vr = fmaf(v[2], e[2], fmaf(v[1], e[1], v[0] * e[0]));
  const float fsum = fmaf(I.f, dWi, J.f * dWj);
  const float ps = mj * fmaf(I.A, dWi, J.A * dWj);
  const float mu = fminf(vr, 0.0f);
  const float vsig = fmaf(-beta, mu, I.c + J.c);
  const float al = 0.25f * (I.av + J.av) * (I.B + J.B);
  const float irs = 1.0f / (I.rho + J.rho);
  const float nu = -al * mu * vsig * irs;
  const float vs = 0.5f * mj * nu * fsum;
  const float Ps = I.P + J.P;
  const float ac = Ps > 0.0f ? (I.acP + J.acP) / Ps : 0.0f;
  const float dPa = I.P - J.P;
  const float dP = 2.0f * fabsf(dPa) * irs;
  const float sdP = dP > 0.0f ? sqrtf(dP) : 0.0f;
  const float vc = fabsf(vr) + sdP;
  const float duu = I.u - J.u;
  const float as = ps + vs;
  // reverse
  const float we = fmaf(lw[2], e[2], fmaf(lw[1], e[1], lw[0] * e[0]));
  float eb[3] = {-as * lw[0], -as * lw[1], -as * lw[2]};
  const float asb = -we;
  const float psb = asb;
  float vsb = asb;
  const float k3 = lc * mj;
  const float acb = k3 * vc * duu * fsum * irs;
  const float vcb = k3 * ac * duu * fsum * irs;
  const float duub = k3 * ac * vc * fsum * irs;
  float fsumb = k3 * ac * vc * duu * irs;
  float irsb = k3 * ac * vc * duu * fsum;
  vsb += 0.5f * lc * vr;
  float vrb = 0.5f * lc * vs;
  Ib.A = lc * mj * dWi * vr;
  float dWib = lc * mj * I.A * vr;
  vrb += lc * mj * I.A * dWi;
  vrb += vcb * (float)((vr > 0.0f) - (vr < 0.0f));
  const float dPb = sdP > 0.0f ? vcb * 0.5f / sdP : 0.0f;
  const float sgnP = (float)((dPa > 0.0f) - (dPa < 0.0f));
  Ib.P = dPb * 2.0f * sgnP * irs;
  Jb.P = -Ib.P;
  irsb += dPb * 2.0f * fabsf(dPa);
  Ib.acP = Jb.acP = 0.0f;
  if (Ps > 0.0f) {
    Ib.acP = acb / Ps;
    Jb.acP = Ib.acP;
    const float Psb = -acb * ac / Ps;
    Ib.P += Psb;
    Jb.P += Psb;
  }
  const float nub = vsb * 0.5f * mj * fsum;
  fsumb += vsb * 0.5f * mj * nu;
  const float alb = -nub * mu * vsig * irs;
  float mub = -nub * al * vsig * irs;
  const float vsigb = -nub * al * mu * irs;
  irsb += -nub * al * mu * vsig;
  const float rsb = -irsb * irs * irs;
  Ib.rho = rsb;
  Jb.rho = rsb;
  Ib.B = alb * 0.25f * (I.av + J.av);
  Jb.B = Ib.B;
  Ib.c = vsigb;
  Jb.c = vsigb;
  mub += -beta * vsigb;
  if (vr < 0.0f) vrb += mub;
  Ib.A += psb * mj * dWi;
  Jb.A = psb * mj * dWj;
  dWib += psb * mj * I.A;
  float dWjb = psb * mj * J.A;
  Ib.f = fsumb * dWi;
  Jb.f = fsumb * dWj;
  dWib += fsumb * I.f;
  dWjb += fsumb * J.f;
  Ib.u = duub;
  Jb.u = -duub;
  vbar[0] = vrb * e[0];
  vbar[1] = vrb * e[1];
  vbar[2] = vrb * e[2];
  eb[0] = fmaf(vrb, v[0], eb[0]);
  eb[1] = fmaf(vrb, v[1], eb[1]);
  eb[2] = fmaf(vrb, v[2], eb[2]);
  dWib_out = dWib;
  dWjb_out = dWjb;
  const float rb = fmaf(dWib, d2Wi, dWjb * d2Wj);
  const float ebe = fmaf(eb[2], e[2], fmaf(eb[1], e[1], eb[0] * e[0]));
  const float ir = 1.0f / r;
  dbar[0] = fmaf(eb[0] - ebe * e[0], ir, rb * e[0]);
  dbar[1] = fmaf(eb[1] - ebe * e[1], ir, rb * e[1]);
  dbar[2] = fmaf(eb[2] - ebe * e[2], ir, rb * e[2]);
}

// ------------------------------------------------------- force adjoint op
struct ForceAdjOp {
  struct I {
    float x, y, z, h, H2lo, H2hi, invH, c4, c5;
    float vx, vy, vz, m;
    Side s;
    float lw[3], lc;
    float xb[3], vb[3];
    SideBar sb;
    float hb, ih;  // dL/dh_k through dW(r, h_k) in the force pairs; 1/h_k
    int k;
  };
  const float4* __restrict__ pos;
  const float4* __restrict__ vel;
  const float4* __restrict__ ga;
  const float4* __restrict__ gb;
  const float4* __restrict__ g4;
  float L[3];
  float kg, beta, gm1, Lmax;
  int kernel;
  float knorm;

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
    const float d[3] = {i.x - xj, i.y - yj, i.z - zj};
    const float r2 = r2_of(d[0], d[1], d[2]);
    if (!(r2 > 0.0f)) return;
    const float Hj = kg * pj.w;
    const float bj_band = band_of(Hj, Lmax);
    if (r2 >= fmaxf(i.H2lo, Hj * Hj - bj_band)) {
      if (r2 >= fmaxf(i.H2hi, Hj * Hj + bj_band)) return;  // outside both supports
      const double ex = exact_r2(i.x, i.y, i.z, pj.x, pj.y, pj.z, L[0], L[1], L[2]);
      if (!(ex < exact_H2(kg, i.h)) && !(ex < exact_H2(kg, pj.w))) return;
    }
    const float4 vj = vel[j];
    const float4 aj = ga[j];
    const float4 bj = gb[j];
    const float4 wj = g4[j];
    const float r = sqrtf(r2);
    const float ir = 1.0f / r;
    const float e[3] = {d[0] * ir, d[1] * ir, d[2] * ir};
    float dwi, d2wi, dwj, d2wj;
    kshape_d12(kernel, r * i.invH, dwi, d2wi);
    const float invHj = 1.0f / Hj;
    kshape_d12(kernel, r * invHj, dwj, d2wj);
    const float c4j = knorm * invHj * invHj * invHj * invHj;
    const float dWk = i.c4 * dwi, d2Wk = i.c5 * d2wi;
    const float dWj = c4j * dwj, d2Wj = c4j * invHj * d2wj;
    Side sj;
    sj.A = aj.x; sj.f = aj.y; sj.rho = aj.z; sj.c = aj.w;
    sj.B = bj.x; sj.av = bj.y; sj.acP = bj.z; sj.u = bj.w;
    sj.P = gm1 * aj.z * bj.w;
    const float vkj[3] = {i.vx - vj.x, i.vy - vj.y, i.vz - vj.z};
    float db[3], vbv[3];
    SideBar Ib, Jb;
    float dWkb1, dWjb1, dWjb2, dWkb2;
    // k first: k's own sum, weights of k
    pair_reverse(i.s, sj, vj.w, r, e, dWk, dWj, d2Wk, d2Wj, vkj, i.lw, i.lc, beta, db, vbv, Ib, Jb, dWkb1, dWjb1);
    i.xb[0] += db[0]; i.xb[1] += db[1]; i.xb[2] += db[2];
    i.vb[0] += vbv[0]; i.vb[1] += vbv[1]; i.vb[2] += vbv[2];
    i.sb.A += Ib.A; i.sb.f += Ib.f; i.sb.rho += Ib.rho; i.sb.c += Ib.c; i.sb.B += Ib.B;
    i.sb.acP += Ib.acP; i.sb.u += Ib.u; i.sb.P += Ib.P;
    // k second: j's sum, weights of j (d and v change sign)
    const float en[3] = {-e[0], -e[1], -e[2]};
    const float vjk[3] = {-vkj[0], -vkj[1], -vkj[2]};
    const float lwj[3] = {wj.x, wj.y, wj.z};
    pair_reverse(sj, i.s, i.m, r, en, dWj, dWk, d2Wj, d2Wk, vjk, lwj, wj.w, beta, db, vbv, Jb, Ib, dWjb2, dWkb2);
    i.xb[0] -= db[0]; i.xb[1] -= db[1]; i.xb[2] -= db[2];
    i.vb[0] -= vbv[0]; i.vb[1] -= vbv[1]; i.vb[2] -= vbv[2];
    i.sb.A += Ib.A; i.sb.f += Ib.f; i.sb.rho += Ib.rho; i.sb.c += Ib.c; i.sb.B += Ib.B;
    i.sb.acP += Ib.acP; i.sb.u += Ib.u; i.sb.P += Ib.P;
    // dW(r, h)/dh = -(4 dW/dr + r d2W/dr2) / h, for both terms that hold dW(r, h_k)
    i.hb = fmaf(-(dWkb1 + dWkb2) * i.ih, fmaf(r, d2Wk, 4.0f * dWk), i.hb);
  }
};

__device__ __forceinline__ void force_adj_item(const AdjArgs& a, const ForceAdjOp& op, const Grid& g, WarpSmem& w,
                                               const Item& it, int t) {
  const int lsh = lanes_shift(it.cnt, a.lmax);
  const unsigned lane = lane_id();
  const int slot = (int)(lane & ((32u >> lsh) - 1u)), s = (int)(lane >> (5 - lsh));
  const bool live = slot < it.cnt;
  const int k = a.plist[it.off + (live ? slot : 0)];
  ForceAdjOp::I I;
  const float4 p = a.pos[k];
  const float4 v = a.vel[k];
  const float4 gi = a.ga[k];
  const float4 bi = a.gb[k];
  const float4 wk = a.g4[k];
  I.x = p.x; I.y = p.y; I.z = p.z; I.h = p.w;
  const float H = a.ph.kg * p.w;
  const float b = band_of(H, op.Lmax);
  I.H2lo = H * H - b;
  I.H2hi = H * H + b;
  I.invH = 1.0f / H;
  I.c4 = a.ph.knorm * I.invH * I.invH * I.invH * I.invH;
  I.c5 = I.c4 * I.invH;
  I.vx = v.x; I.vy = v.y; I.vz = v.z; I.m = v.w;
  I.s.A = gi.x; I.s.f = gi.y; I.s.rho = gi.z; I.s.c = gi.w;
  I.s.B = bi.x; I.s.av = bi.y; I.s.acP = bi.z; I.s.u = bi.w;
  I.s.P = op.gm1 * gi.z * bi.w;
  I.lw[0] = wk.x; I.lw[1] = wk.y; I.lw[2] = wk.z; I.lc = wk.w;
  I.xb[0] = I.xb[1] = I.xb[2] = I.vb[0] = I.vb[1] = I.vb[2] = 0.0f;
  I.sb = SideBar{0, 0, 0, 0, 0, 0, 0, 0};
  I.hb = 0.0f;
  I.ih = 1.0f / p.w;
  I.k = k;
  unsigned ncand = 0;
  scan_item(op, I, g, a.nb, a.pos, it.cell, lsh, s, live, w, ncand);
  for (int q = 0; q < 3; ++q) {
    I.xb[q] = lsum(I.xb[q], lsh);
    I.vb[q] = lsum(I.vb[q], lsh);
  }
  I.sb.A = lsum(I.sb.A, lsh);
  I.sb.f = lsum(I.sb.f, lsh);
  I.sb.rho = lsum(I.sb.rho, lsh);
  I.sb.c = lsum(I.sb.c, lsh);
  I.sb.B = lsum(I.sb.B, lsh);
  I.sb.acP = lsum(I.sb.acP, lsh);
  I.sb.u = lsum(I.sb.u, lsh);
  I.sb.P = lsum(I.sb.P, lsh);
  I.hb = lsum(I.hb, lsh);
  if (!(live && s == 0)) return;
  // reverse of the ghost step of particle k
  const float gam = a.ph.gamma_eos, gm1 = gam - 1.0f;
  const float4 r4 = a.rho4[k];
  const float4 c4v = a.cd[k];
  const float rho = r4.x, h = p.w, u = bi.w, f = gi.y, c = gi.w;
  const float D = -h * r4.y;                      // sum m (3W + r dW/dr)
  const float P = gm1 * rho * u;
  const float alpha_c = P != 0.0f ? bi.z / P : a.ph.alpha_c;
  float Pb = I.sb.P + I.sb.acP * alpha_c;         // acP = alpha_c P
  float fb = I.sb.f + I.sb.A * P / (rho * rho);   // A = f P / rho^2
  Pb += I.sb.A * f / (rho * rho);
  float rhob = I.sb.rho - 2.0f * I.sb.A * f * P / (rho * rho * rho);
  rhob += Pb * gm1 * u;                            // P = (gamma-1) rho u
  float ub = I.sb.u + Pb * gm1 * rho;
  // Balsara B = |div| / (|div| + |curl| + 1e-4 c / h)
  const float dv = c4v.w;
  const float cx = c4v.x, cy = c4v.y, cz = c4v.z;
  const float ad = fabsf(dv), acurl = sqrtf(cx * cx + cy * cy + cz * cz);
  const float eps = 1e-4f * c / h;
  float divb = 0.0f, curlb[3] = {0.0f, 0.0f, 0.0f}, cb = I.sb.c;
  if (ad > 0.0f) {
    const float den = ad + acurl + eps;
    const float iden2 = 1.0f / (den * den);
    const float adb = I.sb.B * (acurl + eps) * iden2;
    const float acb = -I.sb.B * ad * iden2;
    const float epsb = -I.sb.B * ad * iden2;
    divb = adb * (dv > 0.0f ? 1.0f : -1.0f);
    if (acurl > 0.0f) {
      curlb[0] = acb * cx / acurl;
      curlb[1] = acb * cy / acurl;
      curlb[2] = acb * cz / acurl;
    }
    cb += epsb * 1e-4f / h;
    I.hb -= epsb * 1e-4f * c / (h * h);  // eps = 1e-4 c / h
  }
  if (c > 0.0f) ub += cb * gam * gm1 / (2.0f * c);  // c = sqrt(gamma (gamma-1) u)
  // f = 1/Omega, Omega = 1 - D / (3 rho)
  const float omb = -fb * f * f;
  const float Db = -omb / (3.0f * rho);
  rhob += omb * D / (3.0f * rho * rho);
  // div = S / rho, curl = C / rho
  const float ir = 1.0f / rho;
  rhob -= (divb * dv + curlb[0] * cx + curlb[1] * cy + curlb[2] * cz) * ir;
  a.qb[k] = make_float4(rhob, Db, divb * ir, curlb[0] * ir);
  a.cby[k] = curlb[1] * ir;
  a.cbz[k] = curlb[2] * ir;
  a.xb[k] = make_float4(I.xb[0], I.xb[1], I.xb[2], ub);
  a.vb[k] = make_float4(I.vb[0], I.vb[1], I.vb[2], I.hb);  // .w: dL/dh_k so far (h_mode 1)
}

__global__ void __launch_bounds__(kAdjThreads, 5) k_force_adj(AdjArgs a) {
  pdl_wait();
  extern __shared__ __align__(16) unsigned char smem[];
  const Grid g = *a.grid;
  WarpSmem& w = adj_smem(smem);
  ForceAdjOp op;
  op.pos = a.pos; op.vel = a.vel; op.ga = a.ga; op.gb = a.gb; op.g4 = a.g4;
  op.L[0] = g.L[0]; op.L[1] = g.L[1]; op.L[2] = g.L[2];
  op.Lmax = fmaxf(g.L[0], fmaxf(g.L[1], g.L[2]));
  op.kg = a.ph.kg;
  op.kernel = a.ph.kernel;
  op.knorm = a.ph.knorm;
  op.beta = a.ph.beta_v;
  op.gm1 = a.ph.gamma_eos - 1.0f;
  const int n_items = a.ctr[0];
  for (;;) {
    const int t = take_ticket(a.ticket);
    if (t >= n_items) break;
    force_adj_item(a, op, g, w, a.items[t], t);
  }
}

// ----------------------------------------------------- density adjoint op
struct DensAdjOp {
  struct I {
    float x, y, z, h, H2lo, H2hi, invH, c4, c5;
    float vx, vy, vz, m;
    float rb, Db, Sb, Cb[3];
    float xb[3], vb[3];
    float hE, hS, hC[3];  // h_mode 1: sums of k's own pairs for dD/dh, dS/dh, dC/dh
  };
  const float4* __restrict__ pos;
  const float4* __restrict__ vel;
  const float4* __restrict__ qb;
  const float* __restrict__ cby;
  const float* __restrict__ cbz;
  float L[3];
  float kg, Lmax;
  int kernel;
  float knorm;
  int hmode;

  __device__ __forceinline__ float stage_w(float hj) const {
    const float H = kg * hj;
    return H * H + band_of(H, Lmax);
  }
  __device__ __forceinline__ bool candidate(const I& i, float r2, float H2j_hi) const {
    return r2 < fmaxf(i.H2hi, H2j_hi);
  }
  // Adjoint of one particle's density sums (rho, D, S, C) over the pair, at
  // support 1/invH: adds the x-gradient (along e, scaled) and v-gradient of
  // the particle k. sgn = +1 when the sum is k's own, -1 when it is j's.
  __device__ __forceinline__ void add_sum(I& i, float r, const float e[3], const float d[3], const float vjk[3],
                                          float invH, float c4, float c5, float mass, float rb, float Db, float Sb,
                                          const float Cb[3], bool own) const {
    float dw, d2w;
    kshape_d12(kernel, r * invH, dw, d2w);
    const float W1 = c4 * dw, W2 = c5 * d2w;
    const float g = W1 / r;
    const float gp = (W2 - g) / r;
    // rho and D: radial functions of |x_k - x_j|, same gradient either way
    const float radial = mass * (rb * W1 + Db * fmaf(r, W2, 4.0f * W1));
    // velocity difference seen by the sum: v_other - v_owner
    const float sv = own ? 1.0f : -1.0f;  // own: v_j - v_k; j's sum: v_k - v_j
    const float va[3] = {sv * vjk[0], sv * vjk[1], sv * vjk[2]};
    const float sd = fmaf(va[2], d[2], fmaf(va[1], d[1], va[0] * d[0]));
    // C.(va x d) with va x d
    const float vxd[3] = {va[1] * d[2] - va[2] * d[1], va[2] * d[0] - va[0] * d[2], va[0] * d[1] - va[1] * d[0]};
    const float cv = Cb[0] * vxd[0] + Cb[1] * vxd[1] + Cb[2] * vxd[2];
    const float Cxv[3] = {Cb[1] * va[2] - Cb[2] * va[1], Cb[2] * va[0] - Cb[0] * va[2],
                          Cb[0] * va[1] - Cb[1] * va[0]};
    const float dxC[3] = {d[1] * Cb[2] - d[2] * Cb[1], d[2] * Cb[0] - d[0] * Cb[2], d[0] * Cb[1] - d[1] * Cb[0]};
    // own sum: +[S: gp e sd + g va] - [C: gp e cv + g C x va];  j's sum: the negated forms
    const float so = own ? 1.0f : -1.0f;
    const float es = radial + so * mass * (Sb * gp * sd - gp * cv);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      i.xb[q] = fmaf(es, e[q], i.xb[q]);
      i.xb[q] = fmaf(so * mass * g, Sb * va[q] - Cxv[q], i.xb[q]);
      i.vb[q] = fmaf(mass * g, -Sb * d[q] + dxC[q], i.vb[q]);
    }
    if (own && hmode) {
      // h-derivatives of k's own sums (times -h or h): D: 9W + 7 r W' + r^2 W'';
      // S and C: (4 W' + r W'') / r times the pair's (v_j - v_k).d and (v_j - v_k) x d
      float w0, dw0;
      kshape(kernel, r * invH, w0, dw0);
      const float W0 = c4 * w0 / invH;
      i.hE = fmaf(mass, fmaf(r, fmaf(r, W2, 7.0f * W1), 9.0f * W0), i.hE);
      const float gh = mass * fmaf(r, W2, 4.0f * W1) / r;
      i.hS = fmaf(gh, sd, i.hS);
      i.hC[0] = fmaf(gh, vxd[0], i.hC[0]);
      i.hC[1] = fmaf(gh, vxd[1], i.hC[1]);
      i.hC[2] = fmaf(gh, vxd[2], i.hC[2]);
    }
  }
  __device__ __forceinline__ void interact(I& i, int j, unsigned code) const {
    const float4 pj = pos[j];
    float xj = pj.x, yj = pj.y, zj = pj.z;
    shift_j(code, L, xj, yj, zj);
    const float d[3] = {i.x - xj, i.y - yj, i.z - zj};
    const float r2 = r2_of(d[0], d[1], d[2]);
    if (!(r2 > 0.0f)) return;
    const float Hj = kg * pj.w;
    const float H2j = Hj * Hj;
    const float bj_band = band_of(Hj, Lmax);
    if (r2 >= fmaxf(i.H2hi, H2j + bj_band)) return;  // outside both supports
    // membership in each support: in FP32 outside its guard band, in FP64
    // (from the same floats) only inside it
    bool in_k = r2 < i.H2lo;
    bool in_j = r2 < H2j - bj_band;
    const bool band_k = !in_k && r2 < i.H2hi;
    const bool band_j = !in_j && r2 < H2j + bj_band;
    if (band_k || band_j) {
      const double ex = exact_r2(i.x, i.y, i.z, pj.x, pj.y, pj.z, L[0], L[1], L[2]);
      if (band_k) in_k = ex < exact_H2(kg, i.h);
      if (band_j) in_j = ex < exact_H2(kg, pj.w);
    }
    if (!in_k && !in_j) return;
    const float4 vj = vel[j];
    const float r = sqrtf(r2);
    const float ir = 1.0f / r;
    const float e[3] = {d[0] * ir, d[1] * ir, d[2] * ir};
    const float vjk[3] = {vj.x - i.vx, vj.y - i.vy, vj.z - i.vz};
    if (in_k) add_sum(i, r, e, d, vjk, i.invH, i.c4, i.c5, vj.w, i.rb, i.Db, i.Sb, i.Cb, true);
    if (in_j) {
      const float4 q = qb[j];
      const float Cj[3] = {q.w, cby[j], cbz[j]};
      const float invHj = 1.0f / Hj;
      const float c4j = knorm * invHj * invHj * invHj * invHj;
      add_sum(i, r, e, d, vjk, invHj, c4j, c4j * invHj, i.m, q.x, q.y, q.z, Cj, false);
    }
  }
};

__global__ void __launch_bounds__(kAdjThreads, 5) k_dens_adj(AdjArgs a) {
  pdl_wait();
  extern __shared__ __align__(16) unsigned char smem[];
  const Grid g = *a.grid;
  WarpSmem& w = adj_smem(smem);
  DensAdjOp op;
  op.pos = a.pos; op.vel = a.vel; op.qb = a.qb; op.cby = a.cby; op.cbz = a.cbz;
  op.L[0] = g.L[0]; op.L[1] = g.L[1]; op.L[2] = g.L[2];
  op.Lmax = fmaxf(g.L[0], fmaxf(g.L[1], g.L[2]));
  op.kg = a.ph.kg;
  op.kernel = a.ph.kernel;
  op.knorm = a.ph.knorm;
  op.hmode = a.hmode;
  const int n_items = a.ctr[0];
  const unsigned lane = lane_id();
  for (;;) {
    const int t = take_ticket(a.ticket);
    if (t >= n_items) break;
    const Item it = a.items[t];
    const int lsh = lanes_shift(it.cnt, a.lmax);
    const int slot = (int)(lane & ((32u >> lsh) - 1u)), s = (int)(lane >> (5 - lsh));
    const bool live = slot < it.cnt;
    const int k = a.plist[it.off + (live ? slot : 0)];
    DensAdjOp::I I;
    const float4 p = a.pos[k];
    const float4 v = a.vel[k];
    const float4 q = a.qb[k];
    I.x = p.x; I.y = p.y; I.z = p.z; I.h = p.w;
    const float H = a.ph.kg * p.w;
    const float b = band_of(H, op.Lmax);
    I.H2lo = H * H - b;
    I.H2hi = H * H + b;
    I.invH = 1.0f / H;
    I.c4 = a.ph.knorm * I.invH * I.invH * I.invH * I.invH;
    I.c5 = I.c4 * I.invH;
    I.vx = v.x; I.vy = v.y; I.vz = v.z; I.m = v.w;
    I.rb = q.x; I.Db = q.y; I.Sb = q.z;
    I.Cb[0] = q.w; I.Cb[1] = a.cby[k]; I.Cb[2] = a.cbz[k];
    I.xb[0] = I.xb[1] = I.xb[2] = I.vb[0] = I.vb[1] = I.vb[2] = 0.0f;
    I.hE = I.hS = I.hC[0] = I.hC[1] = I.hC[2] = 0.0f;
    unsigned ncand = 0;
    scan_item(op, I, g, a.nb, a.pos, it.cell, lsh, s, live, w, ncand);
    for (int c = 0; c < 3; ++c) {
      I.xb[c] = lsum(I.xb[c], lsh);
      I.vb[c] = lsum(I.vb[c], lsh);
    }
    if (a.hmode) {
      I.hE = lsum(I.hE, lsh);
      I.hS = lsum(I.hS, lsh);
      for (int c = 0; c < 3; ++c) I.hC[c] = lsum(I.hC[c], lsh);
    }
    if (live && s == 0) {
      const float4 xd = a.xb[k];
      const float4 vd = a.vb[k];
      const unsigned dst = a.perm[k];
      if (a.hmode) {
        // dL/dh_k = (force and Balsara part) + rho_b drho/dh + D_b dD/dh + S_b dS/dh + C_b . dC/dh,
        // then lambda_k = (dL/dh_k) / F'_k
        const float4 r4 = a.rho4[k];
        const float h = p.w, ih = 1.0f / h;
        const float D = -h * r4.y;
        const float W00 = I.c4 / I.invH;  // W(0, h_k): every shape has w(0) = 1
        const float dD = -(I.hE + 9.0f * I.m * W00) * ih;
        float hb = vd.w - I.rb * D * ih + I.Db * dD - I.Sb * I.hS * ih;
        hb += (I.Cb[0] * I.hC[0] + I.Cb[1] * I.hC[1] + I.Cb[2] * I.hC[2]) * ih;
        const float Fp = r4.w + (float)(3.0 * a.ph.eta3) * ih * ih * ih * ih;
        a.lam[k] = hb / Fp;
      }
      a.grad_x[dst] = make_float4(xd.x + I.xb[0], xd.y + I.xb[1], xd.z + I.xb[2], 0.0f);
      a.grad_v[dst] = make_float4(vd.x + I.vb[0], vd.y + I.vb[1], vd.z + I.vb[2], 0.0f);
      a.grad_u[dst] = xd.w;
    }
  }
}

// ------------------------------------------------ implicit-function term
struct IftAdjOp {
  struct I {
    float x, y, z, h, H2lo, H2hi, invH, c4, lam;
    float xb[3];
  };
  const float4* __restrict__ pos;
  const float* __restrict__ lam;
  float L[3];
  float kg, Lmax;
  int kernel;
  float knorm;

  __device__ __forceinline__ float stage_w(float hj) const {
    const float H = kg * hj;
    return H * H + band_of(H, Lmax);
  }
  __device__ __forceinline__ bool candidate(const I& i, float r2, float H2j_hi) const {
    return r2 < fmaxf(i.H2hi, H2j_hi);
  }
  // -(lambda_k dW(r,h_k)/dr + lambda_j dW(r,h_j)/dr) e_kj: the x-derivative of
  // lambda_k n_k and of lambda_j n_j for the pair (each zero beyond its support)
  __device__ __forceinline__ void interact(I& i, int j, unsigned code) const {
    const float4 pj = pos[j];
    float xj = pj.x, yj = pj.y, zj = pj.z;
    shift_j(code, L, xj, yj, zj);
    const float d[3] = {i.x - xj, i.y - yj, i.z - zj};
    const float r2 = r2_of(d[0], d[1], d[2]);
    if (!(r2 > 0.0f)) return;
    const float Hj = kg * pj.w;
    const float H2j = Hj * Hj;
    const float bj_band = band_of(Hj, Lmax);
    if (r2 >= fmaxf(i.H2hi, H2j + bj_band)) return;  // outside both supports
    // membership in each support: in FP32 outside its guard band, in FP64
    // (from the same floats) only inside it
    bool in_k = r2 < i.H2lo;
    bool in_j = r2 < H2j - bj_band;
    const bool band_k = !in_k && r2 < i.H2hi;
    const bool band_j = !in_j && r2 < H2j + bj_band;
    if (band_k || band_j) {
      const double ex = exact_r2(i.x, i.y, i.z, pj.x, pj.y, pj.z, L[0], L[1], L[2]);
      if (band_k) in_k = ex < exact_H2(kg, i.h);
      if (band_j) in_j = ex < exact_H2(kg, pj.w);
    }
    if (!in_k && !in_j) return;
    const float r = sqrtf(r2);
    float t = 0.0f;
    if (in_k) t = i.lam * i.c4 * dkshape(kernel, r * i.invH);
    if (in_j) {
      const float invHj = 1.0f / Hj;
      t = fmaf(lam[j] * knorm * (invHj * invHj) * (invHj * invHj), dkshape(kernel, r * invHj), t);
    }
    const float tr = t / r;
    i.xb[0] = fmaf(-tr, d[0], i.xb[0]);
    i.xb[1] = fmaf(-tr, d[1], i.xb[1]);
    i.xb[2] = fmaf(-tr, d[2], i.xb[2]);
  }
};

__global__ void __launch_bounds__(kAdjThreads) k_ift_adj(AdjArgs a) {
  pdl_wait();
  extern __shared__ __align__(16) unsigned char smem[];
  const Grid g = *a.grid;
  WarpSmem& w = adj_smem(smem);
  IftAdjOp op;
  op.pos = a.pos; op.lam = a.lam;
  op.L[0] = g.L[0]; op.L[1] = g.L[1]; op.L[2] = g.L[2];
  op.Lmax = fmaxf(g.L[0], fmaxf(g.L[1], g.L[2]));
  op.kg = a.ph.kg;
  op.kernel = a.ph.kernel;
  op.knorm = a.ph.knorm;
  const int n_items = a.ctr[0];
  const unsigned lane = lane_id();
  for (;;) {
    const int t = take_ticket(a.ticket);
    if (t >= n_items) break;
    const Item it = a.items[t];
    const int lsh = lanes_shift(it.cnt, a.lmax);
    const int slot = (int)(lane & ((32u >> lsh) - 1u)), s = (int)(lane >> (5 - lsh));
    const bool live = slot < it.cnt;
    const int k = a.plist[it.off + (live ? slot : 0)];
    IftAdjOp::I I;
    const float4 p = a.pos[k];
    I.x = p.x; I.y = p.y; I.z = p.z; I.h = p.w;
    const float H = a.ph.kg * p.w;
    const float b = band_of(H, op.Lmax);
    I.H2lo = H * H - b;
    I.H2hi = H * H + b;
    I.invH = 1.0f / H;
    I.c4 = a.ph.knorm * (I.invH * I.invH) * (I.invH * I.invH);
    I.lam = a.lam[k];
    I.xb[0] = I.xb[1] = I.xb[2] = 0.0f;
    unsigned ncand = 0;
    scan_item(op, I, g, a.nb, a.pos, it.cell, lsh, s, live, w, ncand);
    for (int c = 0; c < 3; ++c) I.xb[c] = lsum(I.xb[c], lsh);
    if (live && s == 0) {
      const unsigned dst = a.perm[k];
      float4 gx = a.grad_x[dst];
      gx.x += I.xb[0];
      gx.y += I.xb[1];
      gx.z += I.xb[2];
      a.grad_x[dst] = gx;
    }
  }
}

__global__ void k_gather_weights(int n, const unsigned* __restrict__ perm, const float4* __restrict__ in,
                                 float4* __restrict__ out) {
  pdl_wait();
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) out[k] = in[perm[k]];
}

int backward_impl(Ctx* c, const float4* grad_ad, float4* grad_x, float4* grad_v, float* grad_u, int h_mode,
                  cudaStream_t s) {
  // h = h(x) needs the h iteration's root: not with a density call at fixed h
  if (h_mode == 1 && (c->params.flags & SWIFT_GPU_NO_H_ITER)) return SWIFT_GPU_ERR_ARG;
  if (c->n == 0) return SWIFT_GPU_OK;
  // function attributes belong to the current device's context: set them on every call (cheap, and
  // allowed while a stream is captured)
  cudaFuncSetAttribute(k_force_adj, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kAdjSmemBytes);
  cudaFuncSetAttribute(k_dens_adj, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kAdjSmemBytes);
  cudaFuncSetAttribute(k_ift_adj, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kAdjSmemBytes);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)k_force_adj, kAdjThreads, kAdjSmemBytes);
  int per_sm2 = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, (const void*)k_dens_adj, kAdjThreads, kAdjSmemBytes);
  const int nb1 = (per_sm > 0 ? per_sm : 1) * c->num_sms;
  const int nb2 = (per_sm2 > 0 ? per_sm2 : 1) * c->num_sms;
  int* tickets = c->d_counters + kCtrPerPass * (c->max_passes + 1) + 2;
  cudaMemsetAsync(tickets, 0, 2 * sizeof(int), s);
  const int nbg = min((c->n + 255) / 256, c->num_sms * 8);
  launch_pdl(k_gather_weights, nbg, 256, 0, s, c->n, (const unsigned*)c->d_vals[c->sorted_buf], grad_ad,
             c->d_scratch4[0]);
  AdjArgs a;
  a.hmode = h_mode;
  a.grid = c->d_grid;
  a.nb = nbr_of(c);
  // the gathers rescan the cells: the forward call's kept lists are laid out for
  // the lane-per-particle loops, not for these cell items
  a.perm = c->d_vals[c->sorted_buf];
  a.ph = c->phys;
  a.lmax = cell_lanes(c);
  a.pos = c->d_pos;
  a.vel = c->d_vel;
  a.rho4 = c->d_rho4;
  a.cd = c->d_cd;
  a.ga = c->d_ga;
  a.gb = c->d_gb;
  a.g4 = c->d_scratch4[0];
  a.xb = c->d_scratch4[1];
  a.vb = c->d_scratch4[2];
  a.qb = c->d_scratch4[3];
  a.cby = c->d_scratch1[0];
  a.cbz = c->d_scratch1[1];
  // lambda reuses the loss weights' array: only k_force_adj reads those
  a.lam = reinterpret_cast<float*>(c->d_scratch4[0]);
  a.items = c->d_items0;
  a.plist = c->d_plist0;
  a.ctr = c->d_counters;
  a.grad_x = grad_x;
  a.grad_v = grad_v;
  a.grad_u = grad_u;
  a.ticket = tickets;
  launch_pdl(k_force_adj, nb1, kAdjThreads, kAdjSmemBytes, s, a);
  a.ticket = tickets + 1;
  launch_pdl(k_dens_adj, nb2, kAdjThreads, kAdjSmemBytes, s, a);
  c->launches += 4;
  if (h_mode == 1) {
    cudaMemsetAsync(tickets, 0, sizeof(int), s);  // k_force_adj's ticket, free again
    a.ticket = tickets;
    launch_pdl(k_ift_adj, nb2, kAdjThreads, kAdjSmemBytes, s, a);
    c->launches += 2;
  }
  return cudaGetLastError() == cudaSuccess ? SWIFT_GPU_OK : SWIFT_GPU_ERR_CUDA;
}

}  // namespace sg
