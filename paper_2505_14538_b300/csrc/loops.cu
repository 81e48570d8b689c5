// loops.cu -- the SPH pair loops of Sec. 2.1 as persistent work-queue
// kernels for sm_103a (neighbour scan in engine.cuh):
//
//   k_density   Eqs. 2-6 (+ div/curl, Eqs. 3-4) and the Newton iteration on
//               h (Sec. 2.1.2): ONE cooperative launch runs every pass; after
//               each pass the unconverged particles of an item form one item
//               of the next pass, and a bounded grid barrier separates passes.
//   k_ghost     per particle: f = 1/Omega (Eq. 8), P, c, Balsara B.
//   k_gradient  v_sig,max (Eqs. 10-11) and the Laplacian of u.
//   k_force     Eqs. 7, 9-11, 16-20, 22 and dh/dt, with FP64 block partials of
//               the momentum / energy sums.
//
// Pairs whose FP32 r^2 falls in the guard band of the support re-take the
// neighbour decision in FP64 from the same float inputs, so the neighbour
// sets equal those of the FP64 definition exactly.
#include <cuda_runtime.h>
#include <math.h>

#include <type_traits>

#include "common.cuh"
#include "engine.cuh"
#include "force_lpp.cuh"
#include "internal.h"
#include "lpp.cuh"
#include "ops.cuh"

namespace sg {

constexpr int kLoopThreads = 128;
constexpr int kWarpsPerBlock = kLoopThreads / 32;
constexpr size_t kLoopSmemBytes = sizeof(WarpSmem) * kWarpsPerBlock;

__device__ __forceinline__ WarpSmem& warp_smem(unsigned char* smem) {
  return reinterpret_cast<WarpSmem*>(smem)[threadIdx.x >> 5];
}

// Lane layout of an item: L = 2^lsh lanes per particle, slot = lane % (32/L),
// sub-lane s = lane / (32/L).
struct LaneMap {
  int lsh, slot, s;
  bool live;
};
__device__ __forceinline__ LaneMap lane_map(int cnt, int lmax) {
  LaneMap m;
  m.lsh = lanes_shift(cnt, lmax);
  const unsigned lane = lane_id();
  m.slot = (int)(lane & ((32u >> m.lsh) - 1u));
  m.s = (int)(lane >> (5 - m.lsh));
  m.live = m.slot < cnt;
  return m;
}

// ============================================================ density loop
// Predicted convergence of the h iteration: a Newton step from a relative
// residual below kPredict sqrt(h_tol) is taken as the last (dens_item).
constexpr float kPredict = 0.8f;

struct DensArgs {
  Grid* grid;
  Nbr nb;
  const unsigned* perm;   // sorted -> caller index
  int n;
  Phys ph;
  int lmax;
  int single_pass;
  // caller arrays
  const float4* pos_in;
  const float4* vel_in;
  const uint8_t* active;
  float* h_out;
  float4* rho4_io;
  float4* cd_io;
  unsigned* ngb_out;
  // sorted arrays
  float4* pos;
  float4* vel;
  float* h;
  float2* bracket;
  float4* rho4;
  float4* cd;
  unsigned* ngb;
  uint8_t* act;
  // work lists
  Item* items0;
  int* plist0;
  Item* items[2];
  int* plist[2];
  int* ctr;
  unsigned* barrier;  // [count, generation]
  unsigned long long wait_ns;  // limit of each bounded grid barrier (0: give up at once)
  Status* st;
  unsigned long long* stats;
  // candidate lists kept for the gradient and force loops (NULL: none), per group of
  // 32 pass-0 particles: W entries a lane, item_nl[group] = (0 or -1 without a list, longest list)
  unsigned* nlist;
  int2* item_nl;
  // lane-per-particle pass 0 (uniform grid): axis-sorted cell replicas and the
  // per-lane candidate counts of each group's kept list
  float4* rep;
  long long rep_stride;
  int* lcnt;
  int lpp_w;  // entries a lane of a group's kept list holds
  int* missing;  // set when a group is left without a kept list
};

__device__ __forceinline__ void dens_load(DensOp::I& I, const DensArgs& a, float Lmax, int k) {
  const float4 p = a.pos[k];
  const float4 v = a.vel[k];
  I.x = p.x; I.y = p.y; I.z = p.z;
  dens_set_h(I, a.h[k], a.ph.kg, a.ph.knorm, Lmax);
  I.vx = v.x; I.vy = v.y; I.vz = v.z;
  I.ns = I.nc = I.rs = I.rc = I.dn = I.dr = I.div = I.cx = I.cy = I.cz = 0.0f;
  I.count = 0;
  I.k = k;
}

// Eqs. 5-6 at the lane particle's current h over its list (one step of the
// h iteration). Entries go four at a time: the four position loads are issued
// before any of them is used, so a warp keeps four loads in flight. The four
// shape values are summed in FP32 and scaled once, and the block goes into
// the compensated pair as one term: the running sum then carries at most
// about 4 ulp of n of rounding, far inside h_tol (the final sums at the last
// h, flush, compensate every term).
__device__ __forceinline__ void number_walk(const DensOp& op, const DensOp::I& I, const WarpSmem& w, int cnt,
                                            float& ns, float& nc, float& dn, unsigned& npairs) {
  const unsigned lane = lane_id();
  const int m = __reduce_max_sync(kFull, cnt);
  for (int t0 = 0; t0 < m; t0 += 4) {
    unsigned e[4];
    float4 pj[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int t = t0 + q;
      e[q] = t < cnt ? w.list[t * 32 + lane] : (unsigned)I.k;  // past the end: the particle itself (r = 0)
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) pj[q] = op.pos[e[q] & kIndexMask];
    float ws = 0.0f, ds = 0.0f;  // the block's sums of w(q) and r dw/dq
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      // branch-free: W and dW/dr vanish beyond the support (so entries of
      // the list outside H add exact zeros), and padding is masked
      const bool valid = t0 + q < cnt;
      float xj = pj[q].x, yj = pj[q].y, zj = pj[q].z;
      shift_j(e[q] >> kIndexBits, op.L, xj, yj, zj);
      const float dx = I.x - xj, dy = I.y - yj, dz = I.z - zj;
      const float r = sqrt_approx(r2_of(dx, dy, dz));
      float wq, dwq;
      kshape(op.kernel, r * I.invH, wq, dwq);
      ws += valid ? wq : 0.0f;
      ds = fmaf(r, valid ? dwq : 0.0f, ds);
      npairs += (valid && wq > 0.0f) ? 1u : 0u;  // r < H, the particle itself included
    }
    // W = c3 w(q), dn term = r dW/dr + 3 W (Eq. 6 summed as -h dn/dh)
    const float W = I.c3 * ws;
    if (op.compensated) two_sum_acc(ns, nc, W);
    else ns += W;
    dn += fmaf(I.c4, ds, 3.0f * W);
  }
}

// The candidates a pass-0 item collects (every j within the cap's support,
// a superset of every pair the later loops need, since no h exceeds its cap)
// are kept in HBM for the gradient and force loops, in the layout of the
// lane-per-particle groups: the particle at pass-0 list position idx owns
// lane idx % 32 of group idx / 32, entry t at t * 32 + lane of the group's
// span of W entries a lane, and lcnt[idx] its count. The sub-lanes of a
// particle write their shares one after the other (an exclusive prefix of
// their counts). A group is left without a list (item_nl[group].x = -1) when
// one of its particles has more than W candidates, or took the multi-pass
// route, or when some h may exceed the cap (`ok` false).
__device__ __forceinline__ void keep_list(const DensArgs& a, const WarpSmem& w, const Item& it, const LaneMap& lm,
                                          bool ok, int cnt) {
  const unsigned lane = lane_id();
  const int A = 32 >> lm.lsh;
  const int c = lm.live ? cnt : 0;
  int incl = c, tot = c;
  for (int o = A; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, incl, o);
    if ((int)lane >= o) incl += y;
    tot += __shfl_xor_sync(kFull, tot, o);
  }
  const bool all_ok = __all_sync(kFull, ok);
  if (!lm.live) return;
  const int idx = it.off + lm.slot;
  const int grp = idx >> 5;
  if (!all_ok || tot > a.lpp_w) {
    if (lm.s == 0) {
      a.item_nl[grp].x = -1;
      *a.missing = 1;
    }
    return;
  }
  unsigned* dst = a.nlist + (long long)grp * (a.lpp_w * 32) + (idx & 31);
  const int pre = incl - c;
  for (int t = 0; t < c; ++t) dst[(pre + t) * 32] = w.list[t * 32 + lane];
  if (lm.s == 0) {
    a.lcnt[idx] = tot;
    atomicMax(&a.item_nl[grp].y, tot);
  }
}

// A pass-0 item whose particles' lists are not kept: their groups have none.
__device__ __forceinline__ void drop_lists(const DensArgs& a, const Item& it, const LaneMap& lm) {
  if (lm.live && lm.s == 0) {
    a.item_nl[(it.off + lm.slot) >> 5].x = -1;
    *a.missing = 1;
  }
}

// kFixedH: the density at the given h (no h iteration), a kernel of its own
// so that the iterating one carries none of its branches.
template <bool kFixedH>
__device__ __forceinline__ void dens_item(const DensArgs& a, const DensOp& op, const Grid& g, WarpSmem& w,
                                          const Item& it, const int* __restrict__ plist, bool list_mode,
                                          bool last, Item* items_next, int* plist_next, int* ctr_next, float Lmax,
                                          unsigned& ninter, unsigned& nhiter, unsigned& ncand, int item_idx) {
  const unsigned lane = lane_id();
  const LaneMap lm = lane_map(it.cnt, a.lmax);
  const int k = plist[it.off + (lm.live ? lm.slot : 0)];
  DensOp::I I;
  dens_load(I, a, Lmax, k);
  bool retry = false;  // take the multi-pass route from the starting h
  int flag = 0;
  bool step_again = false;
  float hn = I.h;
  // h cap of the item: the cell's, or its leaf's with adaptive leaves
  float hcap = g.hcap;
  int cap_flag = cell_cap_flag(g);
  if (a.nb.adaptive) {
    hcap = a.nb.leaf_hcap[it.cell];
    if (hcap < g.hcap) cap_flag = SWIFT_GPU_ERR_H_EXCEEDS_CELL;
  }
  // Newton bracket of the list mode, and whether its last step was taken on
  // the prediction that it converges: the final sums then verify it
  float lo = 0.0f, hi = __int_as_float(0x7f800000);
  bool prov = false;
  bool scan = false;  // fixed h: the item's sums from a scan of the cells instead of its lists
  if (list_mode) {
    const float Hc = a.ph.kg * hcap;
    const float R2 = Hc * Hc + band_of(Hc, Lmax);
    bool ovf = false;
    int cnt = collect_item(g, a.nb, a.pos, it.cell, I.x, I.y, I.z, R2, lm.lsh, lm.s, lm.live, w, ncand, ovf);
    retry = lsum_u(ovf ? 1u : 0u, lm.lsh) != 0;
    // even lists shorten the Newton walks and the final sums here, and the
    // kept lists' width (the trips of the gradient and force loops)
    cnt = balance_lists(w, cnt, lm.lsh);
    // kept only where every h (active or not) is within this item's cap: the
    // uniform grid with the cell-derived cap (leaves have caps of their own,
    // and a user h_max may lie below an inactive particle's h)
    if (a.item_nl && item_idx >= 0) keep_list(a, w, it, lm, !retry && !a.nb.adaptive && g.hcap_from_cells, cnt);
    // at fixed h (no h iteration) there is no later pass: an item with a
    // list that overflowed scans the cells below, all its particles (the
    // scan and the flush are warp-wide, so the choice is the whole warp's)
    if constexpr (kFixedH) {
      scan = __any_sync(kFull, retry);
      if (scan) retry = false;
    }
    bool done = !lm.live || retry || kFixedH;
    // a step whose relative residual G = |n h^3 - eta^3| / eta^3 is below
    // this leaves, by Newton's quadratic convergence, a residual inside
    // h_tol: the walk that would only confirm it is skipped. With n nearly
    // constant in h the next residual is about c G^2 with c = 2/3 (0.72-0.84
    // on a jittered lattice), so 0.8 sqrt(h_tol) leaves at most 0.64 c h_tol
    // (any c below 1.56 converges); a miss only costs the particle another
    // pass, the final sums verify it
    const float e3 = (float)a.ph.eta3;
    const float pred = kPredict * sqrtf((float)a.ph.h_tol);
    for (int iter = 0;; ++iter) {
      float ns = 0.0f, nc = 0.0f, dn = 0.0f;
      unsigned np = 0;
      number_walk(op, I, w, done ? 0 : cnt, ns, nc, dn, np);
      lsum2(ns, nc, lm.lsh);
      dn = lsum(dn, lm.lsh);
      np = lsum_u(np, lm.lsh);
      if (!done) {
        if (lm.s == 0 && np > 0) nhiter += np - 1;  // the walk counted the particle itself once
        float h1;
        const float h0 = I.h;
        if (newton_step(h0, ns, nc, dn, lo, hi, hcap, cap_flag, a.ph, iter == a.ph.max_iter - 1, h1, flag)) {
          dens_set_h(I, h1, a.ph.kg, a.ph.knorm, Lmax);
          if (fabsf(fmaf(ns + nc, h0 * h0 * h0, -e3)) < pred * e3 && iter + 2 < a.ph.max_iter) {
            done = true;
            prov = true;
          }
        } else {
          done = true;
        }
      }
      if (!__any_sync(kFull, !done)) break;
    }
    if (!scan) flush(op, I, w, (lm.live && !retry) ? cnt : 0);  // full sums at the final h
  } else {
    if (a.item_nl && item_idx >= 0) drop_lists(a, it, lm);
    scan_item(op, I, g, a.nb, a.pos, it.cell, lm.lsh, lm.s, lm.live, w, ncand);
  }
  if constexpr (kFixedH) {
    if (list_mode && scan) {
      if (a.item_nl && item_idx >= 0) drop_lists(a, it, lm);
      scan_item(op, I, g, a.nb, a.pos, it.cell, lm.lsh, lm.s, lm.live, w, ncand);
    }
  }
  lsum2(I.ns, I.nc, lm.lsh);
  lsum2(I.rs, I.rc, lm.lsh);
  I.dn = lsum(I.dn, lm.lsh);
  I.dr = lsum(I.dr, lm.lsh);
  I.div = lsum(I.div, lm.lsh);
  I.cx = lsum(I.cx, lm.lsh);
  I.cy = lsum(I.cy, lm.lsh);
  I.cz = lsum(I.cz, lm.lsh);
  I.count = lsum_u(I.count, lm.lsh);
  bool again = false;
  if (lm.live && lm.s == 0) {
    if (retry) {
      again = true;
    } else {
      ninter += I.count;
      if (prov) {
        // the predicted step, verified on the final sums (n at the new h);
        // a particle that is not converged after all continues next pass
        float2 br = make_float2(lo, hi);
        if (newton_step(I.h, I.ns, I.nc, I.dn, br.x, br.y, hcap, cap_flag, a.ph, last, hn, flag)) {
          a.h[k] = hn;
          a.bracket[k] = br;
          again = true;
        }
      } else if (!list_mode && !a.single_pass) {  // NO_H_ITER: the sums at the given h, no Newton step
        float2 br = a.bracket[k];
        step_again = newton_step(I.h, I.ns, I.nc, I.dn, br.x, br.y, hcap, cap_flag, a.ph, last, hn, flag);
        if (step_again) {
          a.h[k] = hn;
          a.bracket[k] = br;
          again = true;
        }
      }
      if (!again) {
        a.h[k] = I.h;
        const float rho = I.rs + I.rc;
        const float invh = 1.0f / I.h;
        a.rho4[k] = make_float4(rho, -I.dr * invh, I.ns + I.nc, -I.dn * invh);
        const float ir = 1.0f / rho;
        a.cd[k] = make_float4(I.cx * ir, I.cy * ir, I.cz * ir, I.div * ir);
        a.ngb[k] = I.count;
        if (flag) set_error(a.st, flag);
      }
    }
  }
  const unsigned am = __ballot_sync(kFull, again);
  if (am) {
    const int nu = __popc(am);
    int pbase = 0, ibase = 0;
    if (lane == 0) {
      pbase = atomicAdd(&ctr_next[1], nu);
      ibase = atomicAdd(&ctr_next[0], 1);
    }
    pbase = __shfl_sync(kFull, pbase, 0);
    ibase = __shfl_sync(kFull, ibase, 0);
    if (again) plist_next[pbase + __popc(am & ((1u << lane) - 1u))] = k;
    if (lane == 0) items_next[ibase] = Item{it.cell, pbase, nu, 0};
  }
}

// ================================================ lane-per-particle pass 0
template <int K>
__host__ __device__ constexpr int lpp_width() {
  return lpp_width_of(K);
}
// Shared memory a warp of the density kernel uses: the cell-item lanes' lists,
// or a lane-per-particle group's squared distances (W per lane).
__host__ __device__ constexpr size_t lpp_warp_bytes(int kind) {
  return (size_t)lpp_width_of(kind) * 32 * 4;
}
// With the shared-row collect (lpp 2) the warp's staging area follows the
// squared distances; later passes use the same memory as cell items.
__host__ __device__ constexpr size_t dens_warp_bytes(int kind, int lpp) {
  return lpp == 2 ? (lpp_warp_bytes(kind) + sizeof(RowStage) > sizeof(WarpSmem)
                         ? lpp_warp_bytes(kind) + sizeof(RowStage)
                         : sizeof(WarpSmem))
         : lpp && lpp_warp_bytes(kind) > sizeof(WarpSmem) ? lpp_warp_bytes(kind)
                                                          : sizeof(WarpSmem);
}

// Eqs. 5-6 at the lane particle's current h over its stored squared
// distances (one step of the h iteration): no neighbour records are read.
// Four entries at a time; the sums are taken in list order.
template <int K>
__device__ __forceinline__ void walk_r2(const DensOp::I& I, const float* r2s, int cnt, bool compensated, float& ns,
                                        float& nc, float& dn, unsigned& npairs) {
  const int m = __reduce_max_sync(kFull, cnt);
  for (int t0 = 0; t0 < m; t0 += 4) {
    float r2[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) r2[q] = t0 + q < cnt ? r2s[(t0 + q) * 32] : -1.0f;
    float ws = 0.0f, ds = 0.0f;  // the block's sums, as number_walk
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const bool valid = r2[q] >= 0.0f;
      const float rr = fmaxf(r2[q], 0.0f);
      const float r = sqrt_approx(rr);
      float wq, dwq;
      kshape(K, r * I.invH, wq, dwq);
      ws += valid ? wq : 0.0f;
      ds = fmaf(r, valid ? dwq : 0.0f, ds);
      npairs += (valid && rr > 0.0f && rr < I.H2hi) ? 1u : 0u;
    }
    const float W = I.c3 * ws;
    if (compensated) two_sum_acc(ns, nc, W);
    else ns += W;
    dn += fmaf(I.c4, ds, 3.0f * W);
  }
}

// Pass 0 of the density loop for group `grp` (pass-0 particle list entries
// [32 grp, 32 grp + 32), one lane each): the collect (lpp.cuh: kLPP 1 the
// windows along the pair axes, 2 the shared rows of cells) into
// the group's kept list and the lane's squared distances, the Newton
// iteration on those distances, and the full sums at the final h over the
// kept list. Particles whose candidates do not fit in W, and predicted
// convergences that the final sums refute, continue as one-particle cell
// items of the next pass. At fixed h (kFixedH) a particle whose candidates do
// not fit scans its 27 cells instead.
template <int K, bool kFixedH, int kLPP>
__device__ __forceinline__ void dens_group(const DensArgs& a, const DensOp& op, const Grid& g, float* r2w, int grp,
                                           int P, bool last, Item* items_next, int* plist_next, int* ctr_next,
                                           float Lmax, unsigned& ninter, unsigned& nhiter, unsigned& ncand) {
  constexpr int W = lpp_width<K>();
  const unsigned lane = lane_id();
  const int idx = grp * 32 + (int)lane;
  const bool live = idx < P;
  const int k = a.plist0[live ? idx : grp * 32];
  DensOp::I I;
  dens_load(I, a, Lmax, k);
  const float hcap = g.hcap;
  const int cap_flag = cell_cap_flag(g);
  const float Hc = a.ph.kg * hcap;
  const float R2 = Hc * Hc + band_of(Hc, Lmax);
  unsigned* lst = a.nlist + (long long)grp * (W * 32) + lane;
  float* r2s = r2w + lane;
  const int cell = (int)a.nb.skeys[k];
  bool ovf = false;
  int cnt;
  if constexpr (kLPP == 2)
    cnt = rows_collect<W>(g, a.nb.cell_start, a.pos, I.x, I.y, I.z, cell, R2, live, lst, r2s,
                          *reinterpret_cast<RowStage*>(r2w + W * 32), ovf, ncand);
  else
    cnt = lpp_collect<W>(g, a.nb.cell_start, a.pos, a.rep, a.rep_stride, I.x, I.y, I.z, cell, R2, Lmax, live, lst,
                         r2s, ovf, ncand);
  if (!live) cnt = 0;
  cnt = min(cnt, W);
  // the group's kept list serves the later loops when every lane's candidates
  // fit and every h (active or not) is within the cell cap
  const bool keep = __all_sync(kFull, !ovf) && g.hcap_from_cells;
  const int mw = __reduce_max_sync(kFull, cnt);
  if (lane == 0) {
    a.item_nl[grp] = make_int2(keep ? 0 : -1, mw);
    if (!keep) *a.missing = 1;
  }
  if (live) a.lcnt[idx] = cnt;
  bool retry = ovf;  // the multi-pass route from the starting h
  bool scan = false; // fixed h: the particle's sums from a scan of its cells
  int flag = 0;
  float hn = I.h;
  float lo = 0.0f, hi = __int_as_float(0x7f800000);
  bool prov = false;
  if constexpr (kFixedH) {
    scan = ovf && live;
    retry = false;
  } else {
    bool done = !live || retry;
    // the predicted-convergence skip of dens_item: a relative residual below
    // kPredict sqrt(h_tol) leaves, by Newton's quadratic convergence, a
    // residual inside h_tol, and the final sums verify it
    const float e3 = (float)a.ph.eta3;
    const float pred = kPredict * sqrtf((float)a.ph.h_tol);
    for (int iter = 0;; ++iter) {
      float ns = 0.0f, nc = 0.0f, dn = 0.0f;
      unsigned np = 0;
      walk_r2<K>(I, r2s, done ? 0 : cnt, a.ph.compensated, ns, nc, dn, np);
      if (!done) {
        nhiter += np;
        float h1;
        const float h0 = I.h;
        if (newton_step(h0, ns, nc, dn, lo, hi, hcap, cap_flag, a.ph, iter == a.ph.max_iter - 1, h1, flag)) {
          dens_set_h(I, h1, a.ph.kg, a.ph.knorm, Lmax);
          if (fabsf(fmaf(ns + nc, h0 * h0 * h0, -e3)) < pred * e3 && iter + 2 < a.ph.max_iter) {
            done = true;
            prov = true;
          }
        } else {
          done = true;
        }
      }
      if (!__any_sync(kFull, !done)) break;
    }
  }
  // full sums at the final h over the kept list, four entries at a time: the
  // entries, then all eight records, are loaded before any arithmetic; the
  // sums are taken in list order
  {
    const int fc = (live && !retry && !scan) ? cnt : 0;
    const int m = __reduce_max_sync(kFull, fc);
    // the next batch's entries are read while the current batch's records load
    unsigned e[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) e[q] = q < fc ? lst[q * 32] : (unsigned)k;
    for (int t0 = 0; t0 < m; t0 += 4) {
      DensOp::DRec r[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) op.load_rec((int)(e[q] & kIndexMask), r[q]);
      unsigned nx[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) nx[q] = t0 + 4 + q < fc ? lst[(t0 + 4 + q) * 32] : (unsigned)k;
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (t0 + q < fc) op.interact(I, (int)(e[q] & kIndexMask), e[q] >> kIndexBits, r[q]);
#pragma unroll
      for (int q = 0; q < 4; ++q) e[q] = nx[q];
    }
  }
  if constexpr (kFixedH) {
    if (__any_sync(kFull, scan)) lpp_scan(op, I, g, a.nb.cell_start, cell, scan, ncand);
  }
  bool again = false;
  if (live) {
    if (retry) {
      again = true;
    } else {
      ninter += I.count;
      if (prov) {
        float2 br = make_float2(lo, hi);
        if (newton_step(I.h, I.ns, I.nc, I.dn, br.x, br.y, hcap, cap_flag, a.ph, last, hn, flag)) {
          a.h[k] = hn;
          a.bracket[k] = br;
          again = true;
        }
      }
      if (!again) {
        a.h[k] = I.h;
        const float rho = I.rs + I.rc;
        const float invh = 1.0f / I.h;
        a.rho4[k] = make_float4(rho, -I.dr * invh, I.ns + I.nc, -I.dn * invh);
        const float ir = 1.0f / rho;
        a.cd[k] = make_float4(I.cx * ir, I.cy * ir, I.cz * ir, I.div * ir);
        a.ngb[k] = I.count;
        if (flag) set_error(a.st, flag);
      }
    }
  }
  // particles that continue: one cell item each (all lanes of the next pass on it)
  const unsigned am = __ballot_sync(kFull, again);
  if (am) {
    const int nu = __popc(am);
    int pbase = 0, ibase = 0;
    if (lane == 0) {
      pbase = atomicAdd(&ctr_next[1], nu);
      ibase = atomicAdd(&ctr_next[0], nu);
    }
    pbase = __shfl_sync(kFull, pbase, 0);
    ibase = __shfl_sync(kFull, ibase, 0);
    if (again) {
      const int r = __popc(am & ((1u << lane) - 1u));
      plist_next[pbase + r] = k;
      items_next[ibase + r] = Item{cell, pbase + r, 1, 0};
    }
  }
}

// The loop kernels are instantiated per kernel shape K (kKernelCubic,
// kKernelWendlandC2, kKernelWendlandC4), so the shape is fixed at compile time.
// kLPP: pass 0 runs cell items (0) or lane per particle over groups
// (dens_group) with the windowed collect (1, the replicas of every cell built
// in the prologue) or the shared-row collect (2); later passes run cell items.
// With the shared rows and every particle active, the pass-0 list is the
// sorted order itself, so that a group is 32 consecutive particles, a few
// cells of one row.
template <int K, bool kFixedH, int kLPP>
__global__ void __launch_bounds__(kLoopThreads, kLPP ? 4 : 5) k_density(DensArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const unsigned lane = lane_id();
  const Grid g = *a.grid;
  const float Lmax = fmaxf(g.L[0], fmaxf(g.L[1], g.L[2]));
  constexpr size_t kWarpBytes = dens_warp_bytes(K, kLPP);
  WarpSmem& w = *reinterpret_cast<WarpSmem*>(smem + (threadIdx.x >> 5) * kWarpBytes);

  // ---- prologue: gather into cell order, inputs of inactive particles
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < a.n; k += gridDim.x * blockDim.x) {
    const unsigned src = a.perm[k];
    const float4 p = wrap_pos(a.pos_in[src], a.ph.L);
    a.pos[k] = p;
    a.vel[k] = a.vel_in[src];
    a.h[k] = p.w;
    const uint8_t act = a.active ? (a.active[src] != 0) : 1;
    a.act[k] = act;
    a.bracket[k] = make_float2(0.0f, __int_as_float(0x7f800000));
    if (!act) {
      a.rho4[k] = a.rho4_io[src];
      a.cd[k] = a.cd_io[src];
      a.ngb[k] = a.ngb_out ? a.ngb_out[src] : 0u;
    }
  }
  // ---- active work items (runs of <= kItemMax active particles of a cell or
  // leaf). In round r, warp w of block b takes cell r * 4G + 4b + w (G blocks,
  // 4 warps a block); the block reserves its share of the round with one
  // atomic per counter. Rounds run nearly in step across the grid, so the
  // work queue comes out close to ascending cell order: the warps that later
  // take neighbouring tickets work on neighbouring cells (or leaves) and share
  // their neighbours in cache.
  {
    __shared__ int s_tot[kWarpsPerBlock], s_nit[kWarpsPerBlock], s_base[2];
    const int nunits = a.nb.adaptive ? *a.nb.n_leaves : g.ncells;
    const int wib = (int)(threadIdx.x >> 5);
    const int stride = kWarpsPerBlock * (int)gridDim.x;
    for (int r0 = 0; r0 < nunits; r0 += stride) {  // the same trip count for every warp of the block
      const int c = r0 + (int)blockIdx.x * kWarpsPerBlock + wib;
      int cs = 0, ce = 0;
      if (c < nunits) {
        if (a.nb.adaptive) {
          const int2 r = a.nb.leaf_range[c];
          cs = r.x;
          ce = r.y;
        } else {
          cs = a.nb.cell_start[c];
          ce = a.nb.cell_start[c + 1];
        }
      }
      int total = 0;
      for (int b = cs; b < ce; b += 32) {
        const int k = b + (int)lane;
        const bool on = k < ce && (a.active ? a.active[a.perm[k]] != 0 : true);
        total += __popc(__ballot_sync(kFull, on));
      }
      const int nit = (total + kItemMax - 1) / kItemMax;
      if (lane == 0) {
        s_tot[wib] = total;
        s_nit[wib] = nit;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        int pt = 0, it = 0;
        for (int q = 0; q < kWarpsPerBlock; ++q) {
          const int tq = s_tot[q], nq = s_nit[q];
          s_tot[q] = pt;
          s_nit[q] = it;
          pt += tq;
          it += nq;
        }
        s_base[0] = pt ? atomicAdd(&a.ctr[ctr_index(0, 1)], pt) : 0;
        s_base[1] = it ? atomicAdd(&a.ctr[ctr_index(0, 0)], it) : 0;
      }
      __syncthreads();
      const int pbase = (kLPP == 2 && a.active == nullptr) ? cs : s_base[0] + s_tot[wib];
      const int ibase = s_base[1] + s_nit[wib];
      int wc = 0;
      for (int b = cs; b < ce; b += 32) {
        const int k = b + (int)lane;
        const bool on = k < ce && (a.active ? a.active[a.perm[k]] != 0 : true);
        const unsigned m = __ballot_sync(kFull, on);
        if (on) a.plist0[pbase + wc + __popc(m & ((1u << lane) - 1u))] = k;
        wc += __popc(m);
      }
      for (int t = (int)lane; t < nit; t += 32)
        a.items0[ibase + t] = Item{c, pbase + t * kItemMax, min(kItemMax, wc - t * kItemMax), 0};
      __syncthreads();  // s_tot, s_nit and s_base are reused by the next round
    }
  }
  // ---- replicas of every cell along the 13 pair axes (one warp a cell), from
  // the same wrapped positions the gather above writes
  if constexpr (kLPP == 1) {
    const int nw = (int)((gridDim.x * blockDim.x) >> 5);
    for (int c = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); c < g.ncells; c += nw) {
      const int cs = a.nb.cell_start[c], m = a.nb.cell_start[c + 1] - cs;
      if (m == 0 || m > kRepMax) continue;
      float4 p = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      if ((int)lane < m) p = wrap_pos(a.pos_in[a.perm[cs + (int)lane]], a.ph.L);
      build_replicas_cell(a.rep, a.rep_stride, cs, m, p);
    }
  }
  if (!grid_barrier(&a.barrier[0], &a.barrier[1], a.st, a.wait_ns)) return;

  DensOp op;
  op.pos = a.pos;
  op.vel = a.vel;
  op.L[0] = g.L[0]; op.L[1] = g.L[1]; op.L[2] = g.L[2];
  op.kg = a.ph.kg;
  op.kernel = K;
  op.knorm = a.ph.knorm;
  op.compensated = a.ph.compensated;
  unsigned ninter = 0, nhiter = 0, ncand = 0;
  const int max_pass = a.single_pass ? 1 : a.ph.max_iter;
  int pass = 0;
  for (; pass < max_pass; ++pass) {
    const int n_items = *((volatile int*)&a.ctr[ctr_index(pass, 0)]);
    if (n_items == 0) break;
    const Item* items = pass == 0 ? a.items0 : a.items[pass & 1];
    const int* plist = pass == 0 ? a.plist0 : a.plist[pass & 1];
    Item* items_next = a.items[(pass + 1) & 1];
    int* plist_next = a.plist[(pass + 1) & 1];
    int* ctr_next = &a.ctr[ctr_index(pass + 1, 0)];
    const bool last = pass == max_pass - 1;
    if (kLPP && pass == 0) {
      const int P = *((volatile int*)&a.ctr[ctr_index(0, 1)]);
      const int ng = (P + 31) >> 5;
      float* r2w = reinterpret_cast<float*>(smem + (threadIdx.x >> 5) * kWarpBytes);
      for (;;) {
        const int t = take_ticket(&a.ctr[ctr_index(0, 2)]);
        if (t >= ng) break;
        dens_group<K, kFixedH, kLPP>(a, op, g, r2w, t, P, last, items_next, plist_next, ctr_next, Lmax, ninter,
                                     nhiter, ncand);
      }
    } else {
      for (;;) {
        const int t = take_ticket(&a.ctr[ctr_index(pass, 2)]);
        if (t >= n_items) break;
        const Item it = items[t];
        dens_item<kFixedH>(a, op, g, w, it, plist, !kLPP && pass == 0 && (kFixedH || !a.single_pass), last,
                           items_next, plist_next, ctr_next, Lmax, ninter, nhiter, ncand,
                           !kLPP && pass == 0 ? t : -1);
      }
    }
    if (!grid_barrier(&a.barrier[0], &a.barrier[1], a.st, a.wait_ns)) return;
  }
  // ---- epilogue: h into the sorted positions, outputs to caller order
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < a.n; k += gridDim.x * blockDim.x) {
    const unsigned dst = a.perm[k];
    const float h = a.h[k];
    a.pos[k].w = h;
    a.h_out[dst] = h;
    if (a.act[k]) {
      a.rho4_io[dst] = a.rho4[k];
      a.cd_io[dst] = a.cd[k];
      if (a.ngb_out) a.ngb_out[dst] = a.ngb[k];
    }
  }
  ninter = warp_sum(ninter);
  nhiter = warp_sum(nhiter);
  ncand = warp_sum(ncand);
  if (lane == 0) {
    atomicAdd(&a.stats[kStatInterDens], (unsigned long long)ninter);
    atomicAdd(&a.stats[kStatInterHiter], (unsigned long long)nhiter);
    atomicAdd(&a.stats[kStatCandDens], (unsigned long long)ncand);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    atomicExch(&a.stats[kStatPasses], (unsigned long long)pass);
    atomicExch(&a.stats[kStatItems], (unsigned long long)a.ctr[ctr_index(0, 0)]);
  }
}

// ============================================================== ghost step
// Per particle (Eq. 8, equation of state, sound speed, Balsara switch):
// ga = (A = f P / rho^2, f, rho, c), gb = (B, alpha_v, alpha_c P, u).
// gc (may be NULL) = (x, y, z, 1/H): the particle's position record for the
// lane-per-particle force term (force_lpp.cuh), which derives its kernel
// constants and guard band from 1/H.
__global__ void k_ghost(int n, const unsigned* __restrict__ perm, const float4* __restrict__ pos,
                        const float4* __restrict__ rho4, const float4* __restrict__ cd, const float* __restrict__ u,
                        const float* __restrict__ alpha_v, const float* __restrict__ alpha_c, Phys ph,
                        float4* __restrict__ ga, float4* __restrict__ gb, float4* __restrict__ gc) {
  pdl_wait();
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const unsigned src = perm[k];
    const float h = pos[k].w;
    const float4 r = rho4[k];
    const float4 c4 = cd[k];
    const float uk = u[src];
    const float rho = r.x;
    const float omega = 1.0f + h / (3.0f * rho) * r.y;
    const float f = 1.0f / omega;
    const float P = (ph.gamma_eos - 1.0f) * rho * uk;
    const float c = sqrtf(ph.gamma_eos * (ph.gamma_eos - 1.0f) * uk);
    const float A = f * P / (rho * rho);
    const float ad = fabsf(c4.w);
    const float ac = sqrtf(c4.x * c4.x + c4.y * c4.y + c4.z * c4.z);
    const float B = ad > 0.0f ? ad / (ad + ac + 1e-4f * c / h) : 0.0f;
    const float av = alpha_v ? alpha_v[src] : ph.alpha_v;
    const float acoef = alpha_c ? alpha_c[src] : ph.alpha_c;
    ga[k] = make_float4(A, f, rho, c);
    gb[k] = make_float4(B, av, acoef * P, uk);
    if (gc) {
      const float4 p = pos[k];
      gc[k] = make_float4(p.x, p.y, p.z, 1.0f / (ph.kg * h));
    }
  }
}

// ============================================================ gradient loop
struct LoopArgs {
  Grid* grid;
  Nbr nb;
  const unsigned* perm;
  Phys ph;
  int lmax;
  const float4* pos;
  const float4* vel;
  const float4* ga;
  const float4* gb;
  const Item* items;
  const int* plist;
  const int* ctr;   // item count at ctr[0]
  int* ticket;
  int* done;             // finished blocks; the last one zeroes ticket and done (release_ticket)
  void* out;        // caller order: float2 (gradient) / float4 (force)
  float2* out2;     // fused gradient + force: the gradient's float2 output
  float* dhdt;      // force: caller order, may be NULL
  double* red_partial;  // force: [gridDim.x][8]
  Status* st;
  unsigned long long* stats;
  const unsigned* nlist;  // candidate lists kept by the density call, per group (NULL: scan)
  const int2* item_nl;    // per group: (0 or -1 without a list, longest list)
  const int* lcnt;  // lane-per-particle path: candidates of each group lane's kept list
  const int* missing;    // set by the density call when some group has no kept list
  int only_unlisted;     // cell-item kernels: only particles whose group has no kept list
  int red_offset;        // first block slot of this launch's partial sums
  const float4* gc; // sorted (x, y, z, 1/H) from the ghost step (force_lpp.cuh)
};

// The end of a persistent loop launch: the last block to finish sets the
// launch's ticket, and this count, back to zero, so the next launch on the
// ticket needs no memset node between it and the kernel before it (a memset
// ends a programmatic-launch chain). Every block reaches this once its warps
// have taken their last ticket; a launch whose blocks all return before
// taking one (nothing to do) touches neither counter.
__device__ __forceinline__ void release_ticket(int* ticket, int* done) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(done, 1) == (int)gridDim.x - 1) {
      atomicExch(ticket, 0);
      atomicExch(done, 0);
    }
  }
}

__device__ __forceinline__ void grad_item(const LoopArgs& a, const GradOp& op, const Grid& g, WarpSmem& w,
                                          const Item& it, int t, float Lmax, unsigned& ninter, unsigned& ncand) {
  LaneMap lm = lane_map(it.cnt, a.lmax);
  const int k = a.plist[it.off + (lm.live ? lm.slot : 0)];
  if (a.only_unlisted) lm.live = lm.live && a.item_nl[(it.off + lm.slot) >> 5].x < 0;
  GradOp::I I;
  const float4 p = a.pos[k];
  const float4 v = a.vel[k];
  const float4 gi = a.ga[k];
  I.x = p.x; I.y = p.y; I.z = p.z; I.h = p.w;
  const float H = a.ph.kg * p.w;
  const float b = band_of(H, Lmax);
  I.H2lo = H * H - b;
  I.H2hi = H * H + b;
  I.invH = 1.0f / H;
  I.c4 = a.ph.knorm * I.invH * I.invH * I.invH * I.invH;
  I.vx = v.x; I.vy = v.y; I.vz = v.z;
  I.c = gi.w;
  I.u = a.gb[k].w;
  I.vsig = 2.0f * gi.w;
  I.lap = 0.0f;
  I.count = 0;
  I.k = k;
  scan_item(op, I, g, a.nb, a.pos, it.cell, lm.lsh, lm.s, lm.live, w, ncand);
  I.vsig = lmax(I.vsig, lm.lsh);
  I.lap = lsum(I.lap, lm.lsh);
  I.count = lsum_u(I.count, lm.lsh);
  if (lm.live && lm.s == 0) {
    ninter += I.count;
    reinterpret_cast<float2*>(a.out)[a.perm[k]] = make_float2(I.vsig, 2.0f * I.lap);
  }
}

template <int K>
__global__ void __launch_bounds__(kLoopThreads, 5) k_gradient(LoopArgs a) {
  pdl_wait();
  extern __shared__ __align__(16) unsigned char smem[];
  const unsigned lane = lane_id();
  const Grid g = *a.grid;
  const float Lmax = fmaxf(g.L[0], fmaxf(g.L[1], g.L[2]));
  WarpSmem& w = warp_smem(smem);
  GradOp op;
  op.pos = a.pos; op.vel = a.vel; op.ga = a.ga; op.gb = a.gb;
  op.L[0] = g.L[0]; op.L[1] = g.L[1]; op.L[2] = g.L[2];
  op.kg = a.ph.kg;
  op.kernel = K;
  op.knorm = a.ph.knorm;
  op.beta = a.ph.beta_v;
  // after a lane-per-particle launch, only the particles whose group has no kept list (none: no work)
  if (a.only_unlisted && *a.missing == 0) return;
  const int n_items = a.ctr[0];
  unsigned ninter = 0, ncand = 0;
  for (;;) {
    const int t = take_ticket(a.ticket);
    if (t >= n_items) break;
    const Item it = a.items[t];
    if (a.only_unlisted && !__any_sync(kFull, (int)lane < it.cnt && a.item_nl[(it.off + (int)lane) >> 5].x < 0))
      continue;
    grad_item(a, op, g, w, it, t, Lmax, ninter, ncand);
  }
  ninter = warp_sum(ninter);
  ncand = warp_sum(ncand);
  if (lane == 0) {
    atomicAdd(&a.stats[kStatInterGrad], (unsigned long long)ninter);
    atomicAdd(&a.stats[kStatCandGrad], (unsigned long long)ncand);
  }
  release_ticket(a.ticket, a.done);
}

// =============================================================== force loop
// kGrad: the gradient loop fused in (GradForceOp), writing both outputs.
template <bool kGrad>
__device__ __forceinline__ void force_item(const LoopArgs& a,
                                           const typename std::conditional<kGrad, GradForceOp, ForceOp>::type& op,
                                           const Grid& g, WarpSmem& w, const Item& it, int t, unsigned& ninter,
                                           unsigned& nginter, unsigned& ncand, float* acc, float* accc) {
  using Op = typename std::conditional<kGrad, GradForceOp, ForceOp>::type;
  LaneMap lm = lane_map(it.cnt, a.lmax);
  const int k = a.plist[it.off + (lm.live ? lm.slot : 0)];
  if (a.only_unlisted) lm.live = lm.live && a.item_nl[(it.off + lm.slot) >> 5].x < 0;
  typename Op::I I;
  const float4 p = a.pos[k];
  const float4 v = a.vel[k];
  const float4 gi = a.ga[k];
  const float4 bi = a.gb[k];
  I.x = p.x; I.y = p.y; I.z = p.z; I.h = p.w;
  const float H = a.ph.kg * p.w;
  const float b = band_of(H, op.Lmax);
  I.H2lo = H * H - b;
  I.H2hi = H * H + b;
  I.invH = 1.0f / H;
  I.c4 = a.ph.knorm * I.invH * I.invH * I.invH * I.invH;
  I.vx = v.x; I.vy = v.y; I.vz = v.z;
  I.A = gi.x; I.f = gi.y; I.rho = gi.z; I.c = gi.w;
  I.B = bi.x; I.av = bi.y; I.acP = bi.z; I.u = bi.w;
  I.P = op.gm1 * gi.z * bi.w;
  I.axs = I.axc = I.ays = I.ayc = I.azs = I.azc = I.dus = I.duc = I.dh = 0.0f;
  I.count = 0;
  I.k = k;
  if constexpr (kGrad) {
    I.vsig = 2.0f * gi.w;  // the j = i term of v_sig,max
    I.lap = 0.0f;
    I.gcount = 0;
  }
  scan_item(op, I, g, a.nb, a.pos, it.cell, lm.lsh, lm.s, lm.live, w, ncand);
  lsum2(I.axs, I.axc, lm.lsh);
  lsum2(I.ays, I.ayc, lm.lsh);
  lsum2(I.azs, I.azc, lm.lsh);
  lsum2(I.dus, I.duc, lm.lsh);
  I.dh = lsum(I.dh, lm.lsh);
  I.count = lsum_u(I.count, lm.lsh);
  if constexpr (kGrad) {
    I.vsig = lmax(I.vsig, lm.lsh);
    I.lap = lsum(I.lap, lm.lsh);
    I.gcount = lsum_u(I.gcount, lm.lsh);
  }
  if (lm.live && lm.s == 0) {
    ninter += I.count;
    const float ax = I.axs + I.axc, ay = I.ays + I.ayc, az = I.azs + I.azc, du = I.dus + I.duc;
    const unsigned dst = a.perm[k];
    reinterpret_cast<float4*>(a.out)[dst] = make_float4(ax, ay, az, du);
    if (a.dhdt) a.dhdt[dst] = -(I.h / (3.0f * I.rho)) * I.f * I.dh;
    if constexpr (kGrad) {
      nginter += I.gcount;
      a.out2[dst] = make_float2(I.vsig, 2.0f * I.lap);
    }
    // compensated per-thread sums of the FP32 per-particle terms (FP64 beyond the thread)
    const float m = v.w;
    const float mx = m * ax, my = m * ay, mz = m * az;
    const float va = fmaf(v.z, az, fmaf(v.y, ay, v.x * ax));
    two_sum_acc(acc[0], accc[0], mx);
    two_sum_acc(acc[1], accc[1], my);
    two_sum_acc(acc[2], accc[2], mz);
    two_sum_acc(acc[3], accc[3], m * va);
    two_sum_acc(acc[3], accc[3], m * du);
    two_sum_acc(acc[4], accc[4], sqrtf(fmaf(mz, mz, fmaf(my, my, mx * mx))));
    two_sum_acc(acc[5], accc[5], m * fabsf(va));
    two_sum_acc(acc[5], accc[5], m * fabsf(du));
    two_sum_acc(acc[6], accc[6], m * du);
    acc[7] += (float)I.count;  // exact: counts stay far below 2^24 per thread
  }
}

// The block's partial of the eight global sums from its threads' FP32 TwoSum
// pairs (sum, error): each warp combines its lanes' pairs in FP32 (TwoSum of
// the sums, the errors added), and only the warps' pairs are carried into
// FP64 and added in warp order. Lane-level FP64 shuffles would cost more:
// FP64 issues at a small fraction of the FP32 rate on this part.
__device__ __forceinline__ void block_partial(float (&acc)[8], float (&accc)[8], double (&red)[kWarpsPerBlock][8],
                                              double* out) {
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    lsum2(acc[q], accc[q], 5);
    if (lane_id() == 0) red[threadIdx.x >> 5][q] = (double)acc[q] + (double)accc[q];
  }
  __syncthreads();
  if (threadIdx.x < 8) {
    double x = 0.0;
    for (int ww = 0; ww < kWarpsPerBlock; ++ww) x += red[ww][threadIdx.x];
    out[threadIdx.x] = x;
  }
}

template <bool kGrad, int K>
__device__ __forceinline__ void force_kernel_body(const LoopArgs& a) {
  pdl_wait();
  using Op = typename std::conditional<kGrad, GradForceOp, ForceOp>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[kWarpsPerBlock][8];
  const unsigned lane = lane_id();
  const Grid g = *a.grid;
  WarpSmem& w = warp_smem(smem);
  Op op;
  op.pos = a.pos; op.vel = a.vel; op.ga = a.ga; op.gb = a.gb;
  op.L[0] = g.L[0]; op.L[1] = g.L[1]; op.L[2] = g.L[2];
  op.Lmax = fmaxf(g.L[0], fmaxf(g.L[1], g.L[2]));
  op.kg = a.ph.kg;
  op.kernel = K;
  op.knorm = a.ph.knorm;
  op.beta = a.ph.beta_v;
  op.gm1 = a.ph.gamma_eos - 1.0f;
  op.compensated = a.ph.compensated;
  // after a lane-per-particle launch, only the particles whose group has no kept list; none: the
  // block's slots of the global sums are zero and there is nothing else to do
  if (a.only_unlisted && *a.missing == 0) {
    if (threadIdx.x < 8) a.red_partial[(a.red_offset + blockIdx.x) * 8 + threadIdx.x] = 0.0;
    return;
  }
  const int n_items = a.ctr[0];
  unsigned ninter = 0, nginter = 0, ncand = 0;
  // per-thread partials of the global sums: FP32 TwoSum pairs (sum, error),
  // carried into FP64 for the block and global sums
  float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0}, accc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (;;) {
    const int t = take_ticket(a.ticket);
    if (t >= n_items) break;
    const Item it = a.items[t];
    if (a.only_unlisted && !__any_sync(kFull, (int)lane < it.cnt && a.item_nl[(it.off + (int)lane) >> 5].x < 0))
      continue;
    force_item<kGrad>(a, op, g, w, it, t, ninter, nginter, ncand, acc, accc);
  }
  // block partial of the FP64 sums (summed in block order by k_reduce_partials)
  block_partial(acc, accc, red, a.red_partial + (long long)(a.red_offset + blockIdx.x) * 8);
  ninter = warp_sum(ninter);
  ncand = warp_sum(ncand);
  if (lane == 0) {
    atomicAdd(&a.stats[kStatInterForce], (unsigned long long)ninter);
    atomicAdd(&a.stats[kStatCandForce], (unsigned long long)ncand);
  }
  if constexpr (kGrad) {
    nginter = warp_sum(nginter);
    if (lane == 0) {
      atomicAdd(&a.stats[kStatInterGrad], (unsigned long long)nginter);
      atomicAdd(&a.stats[kStatCandGrad], (unsigned long long)ncand);
    }
  }
  release_ticket(a.ticket, a.done);
}

template <int K>
__global__ void __launch_bounds__(kLoopThreads, 4) k_force(LoopArgs a) { force_kernel_body<false, K>(a); }

// Gradient (Eqs. 10-11, Laplacian of u) and force in one pass over the pairs.
template <int K>
// 4 blocks a SM (128 registers): at 5 (96 registers) the fused pair term spilled
// 296 bytes a thread, and the adaptive plummer2M step's gradient + force took
// 2.27 ms against 1.72 ms (zeldovich256: 40.9 against 35.2 ms).
__global__ void __launch_bounds__(kLoopThreads, 4) k_grad_force(LoopArgs a) { force_kernel_body<true, K>(a); }

// ================================== lane-per-particle gradient / force loops
// One lane per particle over the kept list of its group (written by the
// density call; entry t of lane l at t * 32 + l of the group's span, so the
// 32 lanes read entry t in one coalesced access). A group without a kept list
// (a particle with more candidates than a list holds: clustered sets on the
// uniform grid) is left to the cell-item kernel launched after this one,
// which scans the cells of those particles only (LoopArgs::only_unlisted). kMode: 0 gradient, 1 force, 2 gradient + force
// (one pass over the pairs). The force modes take the pair term of
// force_lpp.cuh, kLppBatch entries at a time: the batch's records are loaded
// first, the next batch's list entries are read meanwhile, and the batch's
// terms are summed in FP32 before the compensated sums take them. Four
// entries a batch at 3 blocks a SM (168 registers) keep 16 record loads in
// flight a lane; on sedov64 that beat two entries at 4 blocks a SM (0.2043 ->
// 0.2003 ms) and three or five entries, or eight at 2 blocks a SM.
constexpr int kLppBatch = 4;
template <int kMode, int K>
__global__ void __launch_bounds__(kLoopThreads, 3) k_loop_lpp(const __grid_constant__ LoopArgs a) {
  pdl_wait();
  constexpr int W = lpp_width<K>();
  constexpr bool kGrad = kMode != 1;
  __shared__ double red[kWarpsPerBlock][8];
  const unsigned lane = lane_id();
  const Grid g = *a.grid;
  const float Lmax = fmaxf(g.L[0], fmaxf(g.L[1], g.L[2]));
  const int P = a.ctr[ctr_index(0, 1)];
  const int ng = (P + 31) >> 5;
  unsigned ninter = 0, nginter = 0, ncand = 0;
  // per-thread partials of the global sums as FP32 TwoSum pairs (sum, error), kept in shared
  // memory (column per thread) so that they take no registers in the pair loop
  __shared__ float s_acc[16][kLoopThreads];
  if constexpr (kMode != 0)
    for (int q = 0; q < 16; ++q) s_acc[q][threadIdx.x] = 0.0f;
  // the gradient loop's pair function (gradient alone)
  GradOp gop;
  gop.pos = a.pos;
  gop.vel = a.vel;
  gop.ga = a.ga;
  gop.gb = a.gb;
  for (int q = 0; q < 3; ++q) gop.L[q] = g.L[q];
  gop.kg = a.ph.kg;
  gop.kernel = K;
  gop.knorm = a.ph.knorm;
  gop.beta = a.ph.beta_v;
  const LeanConst kc{a.ph, Lmax, a.pos};
  for (;;) {
    const int t = take_ticket(a.ticket);
    if (t >= ng) break;
    const int idx = t * 32 + (int)lane;
    const bool live = idx < P;
    const int k = a.plist[live ? idx : t * 32];
    const bool has = a.nlist != nullptr && a.item_nl[t].x >= 0;
    if (!has) continue;  // the cell-item launch that follows takes this group's particles
    const int cnt = live ? a.lcnt[idx] : 0;
    const unsigned* lst = a.nlist + (long long)t * (W * 32) + lane;
    const unsigned dst = live ? a.perm[k] : 0u;
    const float4 p = a.pos[k];
    const float4 v = a.vel[k];
    const float4 gi = a.ga[k];
    const float H = a.ph.kg * p.w;
    const float b = band_of(H, Lmax);
    if constexpr (kMode == 0) {
      GradOp::I I;
      I.x = p.x; I.y = p.y; I.z = p.z; I.h = p.w;
      I.H2lo = H * H - b;
      I.H2hi = H * H + b;
      I.invH = 1.0f / H;
      I.c4 = a.ph.knorm * I.invH * I.invH * I.invH * I.invH;
      I.vx = v.x; I.vy = v.y; I.vz = v.z;
      I.c = gi.w;
      I.u = a.gb[k].w;
      I.vsig = 2.0f * gi.w;
      I.lap = 0.0f;
      I.count = 0;
      I.k = k;
      const int m = __reduce_max_sync(kFull, cnt);
      for (int u = 0; u < m; ++u) {
        if (u < cnt) {
          const unsigned e = lst[u * 32];
          gop.interact(I, (int)(e & kIndexMask), e >> kIndexBits);
        }
      }
      ncand += (unsigned)cnt;
      if (live) {
        ninter += I.count;
        reinterpret_cast<float2*>(a.out)[dst] = make_float2(I.vsig, 2.0f * I.lap);
      }
    } else {
      const float4 bi = a.gb[k];
      LeanI I;
      I.x = p.x; I.y = p.y; I.z = p.z; I.h = p.w;
      I.H2lo = H * H - b;
      I.H2hi = H * H + b;
      I.invH = 1.0f / H;
      I.c4 = a.ph.knorm * I.invH * I.invH * I.invH * I.invH;
      I.vx = v.x; I.vy = v.y; I.vz = v.z;
      I.A = gi.x; I.f = gi.y; I.rho = gi.z; I.c = gi.w;
      I.B = bi.x; I.av = bi.y; I.acP = bi.z; I.u = bi.w;
      I.P = kc.gm1() * gi.z * bi.w;
      I.axs = I.axc = I.ays = I.ayc = I.azs = I.azc = I.dus = I.duc = I.dh = 0.0f;
      I.vsig = 2.0f * gi.w;  // the j = i term of v_sig,max
      I.lap = 0.0f;
      I.gcount = I.count = 0;
      const int m = __reduce_max_sync(kFull, cnt);
      constexpr int B = kLppBatch;
      unsigned e[B];  // the batch's list entries (the particle itself past the list's end)
#pragma unroll
      for (int q = 0; q < B; ++q) e[q] = q < cnt ? lst[q * 32] : (unsigned)k;
      for (int u = 0; u < m; u += B) {
        LeanRec r[B];
#pragma unroll
        for (int q = 0; q < B; ++q) lean_load(a.gc, a.vel, a.ga, a.gb, (int)(e[q] & kIndexMask), r[q]);
        unsigned nx[B];
#pragma unroll
        for (int q = 0; q < B; ++q) nx[q] = u + B + q < cnt ? lst[(u + B + q) * 32] : (unsigned)k;
        float tax = 0.0f, tay = 0.0f, taz = 0.0f, tdu = 0.0f;
#pragma unroll
        for (int q = 0; q < B; ++q)
          if (u + q < cnt)
            lean_pair<K, kGrad>(I, r[q], (int)(e[q] & kIndexMask), e[q] >> kIndexBits, kc, tax, tay, taz, tdu);
        if (a.ph.compensated) {
          two_sum_acc(I.axs, I.axc, tax);
          two_sum_acc(I.ays, I.ayc, tay);
          two_sum_acc(I.azs, I.azc, taz);
          two_sum_acc(I.dus, I.duc, tdu);
        } else {
          I.axs += tax;
          I.ays += tay;
          I.azs += taz;
          I.dus += tdu;
        }
#pragma unroll
        for (int q = 0; q < B; ++q) e[q] = nx[q];
      }
      ncand += (unsigned)cnt;
      if (live) {
        ninter += I.count;
        const float ax = I.axs + I.axc, ay = I.ays + I.ayc, az = I.azs + I.azc, du = I.dus + I.duc;
        reinterpret_cast<float4*>(a.out)[dst] = make_float4(ax, ay, az, du);
        if (a.dhdt) a.dhdt[dst] = -(I.h / (3.0f * I.rho)) * I.f * I.dh;
        if constexpr (kMode == 2) {
          nginter += I.gcount;
          a.out2[dst] = make_float2(I.vsig, 2.0f * I.lap);
        }
        const float m = v.w;
        const float mx = m * ax, my = m * ay, mz = m * az;
        const float va = fmaf(v.z, az, fmaf(v.y, ay, v.x * ax));
        float acc[8], accc[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          acc[q] = s_acc[q][threadIdx.x];
          accc[q] = s_acc[8 + q][threadIdx.x];
        }
        two_sum_acc(acc[0], accc[0], mx);
        two_sum_acc(acc[1], accc[1], my);
        two_sum_acc(acc[2], accc[2], mz);
        two_sum_acc(acc[3], accc[3], m * va);
        two_sum_acc(acc[3], accc[3], m * du);
        two_sum_acc(acc[4], accc[4], sqrtf(fmaf(mz, mz, fmaf(my, my, mx * mx))));
        two_sum_acc(acc[5], accc[5], m * fabsf(va));
        two_sum_acc(acc[5], accc[5], m * fabsf(du));
        two_sum_acc(acc[6], accc[6], m * du);
        acc[7] += (float)I.count;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          s_acc[q][threadIdx.x] = acc[q];
          s_acc[8 + q][threadIdx.x] = accc[q];
        }
      }
    }
  }
  if constexpr (kMode != 0) {
    float acc[8], accc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      acc[q] = s_acc[q][threadIdx.x];
      accc[q] = s_acc[8 + q][threadIdx.x];
    }
    block_partial(acc, accc, red, a.red_partial + (long long)(a.red_offset + blockIdx.x) * 8);
  }
  ninter = warp_sum(ninter);
  ncand = warp_sum(ncand);
  if (lane == 0) {
    atomicAdd(&a.stats[kMode == 0 ? kStatInterGrad : kStatInterForce], (unsigned long long)ninter);
    atomicAdd(&a.stats[kMode == 0 ? kStatCandGrad : kStatCandForce], (unsigned long long)ncand);
  }
  if constexpr (kMode == 2) {
    nginter = warp_sum(nginter);
    if (lane == 0) {
      atomicAdd(&a.stats[kStatInterGrad], (unsigned long long)nginter);
      atomicAdd(&a.stats[kStatCandGrad], (unsigned long long)ncand);
    }
  }
  release_ticket(a.ticket, a.done);
}

// One warp per quantity; lane l sums blocks l, l+32, ... and the warp then
// combines the lanes in a fixed order, so the result does not depend on timing.
// The unrolled loop issues eight loads before their adds (the order of the
// adds is unchanged), so the lane's chain waits on one load latency per eight
// blocks instead of per block.
__global__ void k_reduce_partials(const double* __restrict__ part, int nblocks, double* __restrict__ out) {
  pdl_wait();
  const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double x = 0.0;
#pragma unroll 8
  for (int b = lane; b < nblocks; b += 32) x += part[b * 8 + q];
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  if (lane == 0) out[q] = x;
}

// =================================================================== hosts
static int persistent_blocks(Ctx* c, const void* kern, size_t smem) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kLoopThreads, smem);
  if (per_sm < 1) per_sm = 1;
  if (c->tuning.blocks_per_sm > 0 && c->tuning.blocks_per_sm < per_sm) per_sm = c->tuning.blocks_per_sm;
  int nb = per_sm * c->num_sms;
  return nb < c->red_blocks ? nb : c->red_blocks;
}

// The instantiation of each loop kernel for kernel shape `kind`.
template <int K>
static const void* density_kernel_k(bool fixed_h, int lpp) {
  if (lpp == 2) return fixed_h ? (const void*)k_density<K, true, 2> : (const void*)k_density<K, false, 2>;
  if (lpp == 1) return fixed_h ? (const void*)k_density<K, true, 1> : (const void*)k_density<K, false, 1>;
  return fixed_h ? (const void*)k_density<K, true, 0> : (const void*)k_density<K, false, 0>;
}
static const void* density_kernel(int kind, bool fixed_h, int lpp) {
  return kind == kKernelWendlandC2   ? density_kernel_k<kKernelWendlandC2>(fixed_h, lpp)
         : kind == kKernelWendlandC4 ? density_kernel_k<kKernelWendlandC4>(fixed_h, lpp)
                                     : density_kernel_k<kKernelCubic>(fixed_h, lpp);
}
static const void* gradient_kernel(int kind) {
  return kind == kKernelWendlandC2 ? (const void*)k_gradient<kKernelWendlandC2>
         : kind == kKernelWendlandC4 ? (const void*)k_gradient<kKernelWendlandC4>
                                     : (const void*)k_gradient<kKernelCubic>;
}
static const void* force_kernel(int kind) {
  return kind == kKernelWendlandC2 ? (const void*)k_force<kKernelWendlandC2>
         : kind == kKernelWendlandC4 ? (const void*)k_force<kKernelWendlandC4>
                                     : (const void*)k_force<kKernelCubic>;
}
static const void* grad_force_kernel(int kind) {
  return kind == kKernelWendlandC2 ? (const void*)k_grad_force<kKernelWendlandC2>
         : kind == kKernelWendlandC4 ? (const void*)k_grad_force<kKernelWendlandC4>
                                     : (const void*)k_grad_force<kKernelCubic>;
}
// Lane-per-particle loop kernel of `mode` (0 gradient, 1 force, 2 both).
template <int M>
static const void* lpp_loop_kernel_m(int kind) {
  return kind == kKernelWendlandC2 ? (const void*)k_loop_lpp<M, kKernelWendlandC2>
         : kind == kKernelWendlandC4 ? (const void*)k_loop_lpp<M, kKernelWendlandC4>
                                     : (const void*)k_loop_lpp<M, kKernelCubic>;
}
static const void* lpp_loop_kernel(int mode, int kind) {
  return mode == 0 ? lpp_loop_kernel_m<0>(kind) : mode == 1 ? lpp_loop_kernel_m<1>(kind) : lpp_loop_kernel_m<2>(kind);
}

static size_t dens_smem(int kind, int lpp) { return dens_warp_bytes(kind, lpp) * kWarpsPerBlock; }

// Raise the dynamic shared-memory limit of every loop kernel, once per device
// (function attributes belong to the device's context).
constexpr int kMaxAttrDevices = 64;
static int g_attr_done[kMaxAttrDevices] = {0};
static void ensure_attrs(const Ctx* c) {
  const int dev = c->device;
  if (dev >= 0 && dev < kMaxAttrDevices && __atomic_load_n(&g_attr_done[dev], __ATOMIC_ACQUIRE)) return;
  for (int kind = kKernelCubic; kind <= kKernelWendlandC4; ++kind) {
    for (int fh = 0; fh < 2; ++fh)
      for (int lpp = 0; lpp < 3; ++lpp)
        cudaFuncSetAttribute(density_kernel(kind, fh != 0, lpp), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)dens_smem(kind, lpp));
    for (const void* f : {gradient_kernel(kind), force_kernel(kind), grad_force_kernel(kind)})
      cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLoopSmemBytes);
  }
  if (dev >= 0 && dev < kMaxAttrDevices) __atomic_store_n(&g_attr_done[dev], 1, __ATOMIC_RELEASE);
}

// The loop kernels start with pdl_wait(): launched with programmatic stream
// serialization, they may be scheduled while the kernel before them drains.
static cudaError_t launch_loop(const void* f, int nblk, LoopArgs& a, cudaStream_t s, size_t smem = kLoopSmemBytes) {
  void* args[] = {&a};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nblk);
  cfg.blockDim = dim3(kLoopThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, f, args);
}

void reduce_partials(Ctx* c, int nblocks, double* out, cudaStream_t s) {
  launch_pdl(k_reduce_partials, 1, 256, 0, s, (const double*)c->d_red_partial, nblocks, out);
  c->launches++;
}

// Whether the kept-list store holds a span of W entries a lane (W of the
// current kernel shape, which swift_gpu_set_params may have changed since the
// store was sized) for every group of the current particles.
static bool lpp_store_fits(const Ctx* c) {
  return c->d_nlist != nullptr && c->d_lcnt != nullptr &&
         (int64_t)lpp_width_of(c->phys.kernel) * 32 * (((int64_t)c->n + 31) / 32) <= c->nl_cap;
}

// The lane-per-particle path runs the persistent density call on the uniform
// grid when the tuning asks for one lane a particle and the context holds the
// kept-list store (and, for the windowed collect, the replicas): 0 the cell
// items, 1 the windowed collect, 2 the shared-row collect.
static int use_lpp(const Ctx* c) {
  if (c->tuning.max_lanes_per_particle != 1 || !lpp_store_fits(c) ||
      (c->params.flags & (SWIFT_GPU_ADAPTIVE | SWIFT_GPU_PLAIN)))
    return 0;
  if (c->tuning.group_collect == SWIFT_GPU_COLLECT_WINDOWS) return c->d_rep != nullptr ? 1 : 0;
  return 2;
}

int density_impl(Ctx* c, const float4* pos_in, const float4* vel_in, const uint8_t* active, float* h_out,
                 float4* rho4, float4* cd, uint32_t* ngb, cudaStream_t s) {
  ensure_attrs(c);
  const int lpp = use_lpp(c);
  const void* kern = density_kernel(c->phys.kernel, (c->params.flags & SWIFT_GPU_NO_H_ITER) != 0, lpp);
  const size_t smem = dens_smem(c->phys.kernel, lpp);
  const int nblk = persistent_blocks(c, kern, smem);
  cudaMemsetAsync(c->d_counters, 0, sizeof(int) * (size_t)kCtrCount(c->max_passes), s);
  DensArgs a;
  a.grid = c->d_grid;
  a.nb = nbr_of(c);
  a.perm = c->d_vals[c->sorted_buf];
  a.n = c->n;
  a.ph = c->phys;
  // the cell items of later passes (one particle each on this path) take all lanes of a warp
  a.lmax = cell_lanes(c);
  a.single_pass = (c->params.flags & SWIFT_GPU_NO_H_ITER) ? 1 : 0;
  a.pos_in = pos_in;
  a.vel_in = vel_in;
  a.active = active;
  a.h_out = h_out;
  a.rho4_io = rho4;
  a.cd_io = cd;
  a.ngb_out = ngb;
  a.pos = c->d_pos;
  a.vel = c->d_vel;
  a.h = c->d_h;
  a.bracket = c->d_bracket;
  a.rho4 = c->d_rho4;
  a.cd = c->d_cd;
  a.ngb = c->d_ngb;
  a.act = c->d_act;
  a.items0 = c->d_items0;
  a.plist0 = c->d_plist0;
  a.items[0] = c->d_items[0];
  a.items[1] = c->d_items[1];
  a.plist[0] = c->d_plist[0];
  a.plist[1] = c->d_plist[1];
  a.ctr = c->d_counters;
  a.barrier = reinterpret_cast<unsigned*>(c->d_counters + kCtrPerPass * (c->max_passes + 2));
  a.wait_ns = wait_limit_ns(c);
  a.st = c->d_status;
  a.stats = c->d_stats;
  // kept lists in the groups' layout (either engine), where the context holds the store for it
  const bool keep = lpp_store_fits(c) && !(c->params.flags & SWIFT_GPU_ADAPTIVE);
  a.nlist = keep ? c->d_nlist : nullptr;
  a.item_nl = keep ? c->d_item_nl : nullptr;
  a.rep = c->d_rep;
  a.rep_stride = c->n;
  a.lcnt = c->d_lcnt;
  a.lpp_w = lpp_width_of(c->phys.kernel);
  a.missing = c->d_counters + kCtrMissing(c->max_passes);  // zeroed with the counters above
  if (keep && !lpp && c->n > 0) cudaMemsetAsync(c->d_item_nl, 0, sizeof(int2) * (size_t)((c->n + 31) / 32), s);
  void* args[] = {&a};
  cudaError_t e = cudaLaunchCooperativeKernel(kern, dim3(nblk), dim3(kLoopThreads), args, smem, s);
  c->launches += 2;
  c->all_active = active == nullptr;
  // the kept lists are per group of the pass-0 list, whichever engine wrote them
  c->lpp_lists = keep ? 1 : 0;
  return e == cudaSuccess ? SWIFT_GPU_OK : SWIFT_GPU_ERR_CUDA;
}

int ghost_impl(Ctx* c, const float* u, const float* alpha_v, const float* alpha_c, cudaStream_t s) {
  if (c->n == 0) return SWIFT_GPU_OK;
  const int nb = min((c->n + 255) / 256, c->num_sms * 8);
  launch_pdl(k_ghost, nb, 256, 0, s, c->n, (const unsigned*)c->d_vals[c->sorted_buf], c->d_pos, c->d_rho4, c->d_cd,
             u, alpha_v, alpha_c, c->phys, c->d_ga, c->d_gb, c->d_gc);
  c->launches++;
  return cudaGetLastError() == cudaSuccess ? SWIFT_GPU_OK : SWIFT_GPU_ERR_CUDA;
}

// The density results of the particles marked in mask (caller order) replaced
// by values computed elsewhere: h (into the sorted positions), rho4, curl_div.
// An h beyond the cell cap cannot be served by the kept lists or the cells:
// ERR_H_EXCEEDS_CELL.
__global__ void k_set_inactive(int n, const unsigned* __restrict__ perm, const Grid* __restrict__ g,
                               const uint8_t* __restrict__ mask, const float* __restrict__ h,
                               const float4* __restrict__ rho4_in, const float4* __restrict__ cd_in, float4* pos,
                               float4* __restrict__ rho4, float4* __restrict__ cd, Status* st) {
  const float hcap = g->hcap;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const unsigned src = perm[k];
    if (!mask[src]) continue;
    const float hk = h[src];
    if (!(hk > 0.0f) || hk > hcap) set_error(st, cell_cap_flag(*g));
    pos[k].w = hk;
    rho4[k] = rho4_in[src];
    cd[k] = cd_in[src];
  }
}

int set_inactive_impl(Ctx* c, const uint8_t* mask, const float* h, const float4* rho4, const float4* cd,
                      cudaStream_t s) {
  if (c->n == 0) return SWIFT_GPU_OK;
  const int nb = min((c->n + 255) / 256, c->num_sms * 8);
  k_set_inactive<<<nb, 256, 0, s>>>(c->n, c->d_vals[c->sorted_buf], c->d_grid, mask, h, rho4, cd, c->d_pos,
                                    c->d_rho4, c->d_cd, c->d_status);
  c->launches++;
  return cudaGetLastError() == cudaSuccess ? SWIFT_GPU_OK : SWIFT_GPU_ERR_CUDA;
}

static LoopArgs loop_args(Ctx* c, int* ticket, int* done, void* out) {
  LoopArgs a;
  a.done = done;
  a.grid = c->d_grid;
  a.nb = nbr_of(c);
  a.perm = c->d_vals[c->sorted_buf];
  a.ph = c->phys;
  a.lmax = cell_lanes(c);
  a.pos = c->d_pos;
  a.vel = c->d_vel;
  a.ga = c->d_ga;
  a.gb = c->d_gb;
  a.items = c->d_items0;
  a.plist = c->d_plist0;
  a.ctr = c->d_counters;  // pass-0 item count
  a.ticket = ticket;
  a.out = out;
  a.out2 = nullptr;
  a.dhdt = nullptr;
  a.red_partial = c->d_red_partial;
  a.st = c->d_status;
  a.stats = c->d_stats;
  // the lane-per-particle loops read the density call's kept lists; the cell-item
  // kernels (no kept lists: adaptive leaves) scan the cells
  a.nlist = c->lpp_lists ? c->d_nlist : nullptr;
  a.item_nl = c->lpp_lists ? c->d_item_nl : nullptr;
  a.lcnt = c->d_lcnt;
  a.gc = c->d_gc;
  a.missing = c->d_counters + kCtrMissing(c->max_passes);
  a.only_unlisted = 0;
  a.red_offset = 0;
  return a;
}

// One gradient / force / both pass (mode 0 / 1 / 2). Over kept lists: the
// lane-per-particle kernel, then the cell-item kernel for the particles of
// groups without a kept list (it returns at once when the density call left
// every group a list); without kept lists: the cell-item kernel alone. The
// launches' block partials of the global sums are slots [0, *nblk_out).
static int loop_launch(Ctx* c, int mode, LoopArgs& a, cudaStream_t s, int* nblk_out) {
  ensure_attrs(c);
  const void* cell_kern = mode == 0   ? gradient_kernel(c->phys.kernel)
                          : mode == 1 ? force_kernel(c->phys.kernel)
                                      : grad_force_kernel(c->phys.kernel);
  int total = 0;
  cudaError_t e = cudaSuccess;
  if (c->lpp_lists) {
    const void* kern = lpp_loop_kernel(mode, c->phys.kernel);
    const int nblk = persistent_blocks(c, kern, 0);
    e = launch_loop(kern, nblk, a, s, 0);
    c->launches += 1;
    total = nblk;
    LoopArgs b = a;
    b.only_unlisted = 1;
    b.red_offset = nblk;
    b.ticket = c->d_counters + kCtrUnlistedTicket(c->max_passes);
    b.done = c->d_counters + kCtrLoopDone(c->max_passes, 2);
    const int nblk2 = min(persistent_blocks(c, cell_kern, kLoopSmemBytes), c->red_blocks - nblk);
    if (e == cudaSuccess) e = launch_loop(cell_kern, nblk2, b, s, kLoopSmemBytes);
    c->launches += 2;
    total += nblk2;
  } else {
    const int nblk = persistent_blocks(c, cell_kern, kLoopSmemBytes);
    e = launch_loop(cell_kern, nblk, a, s, kLoopSmemBytes);
    c->launches += 2;
    total = nblk;
  }
  if (nblk_out) *nblk_out = total;
  return e == cudaSuccess ? SWIFT_GPU_OK : SWIFT_GPU_ERR_CUDA;
}

int gradient_impl(Ctx* c, float2* out, cudaStream_t s) {
  int* ticket = c->d_counters + kCtrPerPass * (c->max_passes + 1) + 0;
  LoopArgs a = loop_args(c, ticket, c->d_counters + kCtrLoopDone(c->max_passes, 0), out);
  return loop_launch(c, 0, a, s, nullptr);
}

int force_impl(Ctx* c, float4* out, float* dhdt, double* reductions, cudaStream_t s) {
  int* ticket = c->d_counters + kCtrPerPass * (c->max_passes + 1) + 1;
  LoopArgs a = loop_args(c, ticket, c->d_counters + kCtrLoopDone(c->max_passes, 1), out);
  a.dhdt = dhdt;
  int nblk = 0;
  const int rc = loop_launch(c, 1, a, s, &nblk);
  if (rc != SWIFT_GPU_OK) return rc;
  if (reductions) {
    launch_pdl(k_reduce_partials, 1, 256, 0, s, (const double*)c->d_red_partial, nblk, reductions);
    c->launches++;
  }
  return cudaGetLastError() == cudaSuccess ? SWIFT_GPU_OK : SWIFT_GPU_ERR_CUDA;
}

int grad_force_impl(Ctx* c, float2* grad_out, float4* out, float* dhdt, double* reductions, cudaStream_t s) {
  int* ticket = c->d_counters + kCtrPerPass * (c->max_passes + 1) + 1;
  LoopArgs a = loop_args(c, ticket, c->d_counters + kCtrLoopDone(c->max_passes, 1), out);
  a.out2 = grad_out;
  a.dhdt = dhdt;
  int nblk = 0;
  const int rc = loop_launch(c, 2, a, s, &nblk);
  if (rc != SWIFT_GPU_OK) return rc;
  if (reductions) {
    launch_pdl(k_reduce_partials, 1, 256, 0, s, (const double*)c->d_red_partial, nblk, reductions);
    c->launches++;
  }
  return cudaGetLastError() == cudaSuccess ? SWIFT_GPU_OK : SWIFT_GPU_ERR_CUDA;
}

}  // namespace sg
