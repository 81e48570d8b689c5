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
#include "internal.h"
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
  // candidate lists kept for the gradient / force / adjoint loops (NULL: none)
  unsigned* nlist;
  long long nl_cap;
  unsigned long long* nl_ctr;
  int2* item_nl;       // per pass-0 item: (first entry, entries per lane) or (-1, 0)
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
// before any of them is used, so a warp keeps four loads in flight; the sums
// are taken in list order, as one at a time would.
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
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      // branch-free: W and dW/dr vanish beyond the support (so entries of
      // the list outside H add exact zeros), and padding is masked
      const bool valid = t0 + q < cnt;
      const int j = (int)(e[q] & kIndexMask);
      float xj = pj[q].x, yj = pj[q].y, zj = pj[q].z;
      shift_j(e[q] >> kIndexBits, op.L, xj, yj, zj);
      const float dx = I.x - xj, dy = I.y - yj, dz = I.z - zj;
      const float r2 = r2_of(dx, dy, dz);
      const float invr = r2 > 0.0f ? rsqrtf(r2) : 0.0f;
      const float r = r2 * invr;
      float wq, dwq;
      kshape(op.kernel, r * I.invH, wq, dwq);
      const float W = valid ? I.c3 * wq : 0.0f;
      const float D = valid ? fmaf(r, I.c4 * dwq, 3.0f * W) : 0.0f;
      if (op.compensated) two_sum_acc(ns, nc, W);
      else ns += W;
      dn += D;
      npairs += (valid && r2 < I.H2hi && j != I.k) ? 1u : 0u;
    }
  }
}

// The candidates a pass-0 item collects (every j within the cap's support,
// a superset of every pair the later loops need, since no h exceeds its cap)
// are kept in HBM, lane-interleaved as in shared memory and padded with
// kNoEntry, so the gradient, force and adjoint loops need not scan again.
__device__ __forceinline__ void keep_list(const DensArgs& a, const WarpSmem& w, int item_idx, bool ok, int cnt,
                                          bool live) {
  const unsigned lane = lane_id();
  int2 span = make_int2(-1, 0);
  if (__all_sync(kFull, ok)) {
    const int m = __reduce_max_sync(kFull, live ? cnt : 0);
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(a.nl_ctr, (unsigned long long)m * 32ull);
    base = __shfl_sync(kFull, base, 0);
    if (base + (unsigned long long)m * 32ull <= (unsigned long long)a.nl_cap) {
      for (int t = 0; t < m; ++t)
        a.nlist[base + (unsigned long long)(t * 32 + (int)lane)] =
            (live && t < cnt) ? w.list[t * 32 + lane] : kNoEntry;
      span = make_int2((int)base, m);
    }
  }
  if (lane == 0) a.item_nl[item_idx] = span;
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
    if (a.item_nl && item_idx >= 0)
      keep_list(a, w, item_idx, !retry && !a.nb.adaptive && g.hcap_from_cells, cnt, lm.live);
    // at fixed h (no h iteration) there is no later pass: an item with a
    // list that overflowed scans the cells below, all its particles (the
    // scan and the flush are warp-wide, so the choice is the whole warp's)
    if constexpr (kFixedH) {
      scan = __any_sync(kFull, retry);
      if (scan) retry = false;
    }
    bool done = !lm.live || retry || kFixedH;
    // a step whose relative residual G = |n h^3 - eta^3| / eta^3 is below
    // this leaves, by Newton's quadratic convergence, a residual well inside
    // h_tol: the walk that would only confirm it is skipped. With n nearly
    // constant in h the next residual is about (2/3) G^2 (0.72-0.84 G^2 on a
    // jittered lattice), so 0.6 sqrt(h_tol) leaves at most 0.36 c h_tol; a
    // miss only costs the particle another pass, the final sums verify it
    const float e3 = (float)a.ph.eta3;
    const float pred = 0.6f * sqrtf((float)a.ph.h_tol);
    for (int iter = 0;; ++iter) {
      float ns = 0.0f, nc = 0.0f, dn = 0.0f;
      unsigned np = 0;
      number_walk(op, I, w, done ? 0 : cnt, ns, nc, dn, np);
      lsum2(ns, nc, lm.lsh);
      dn = lsum(dn, lm.lsh);
      np = lsum_u(np, lm.lsh);
      if (!done) {
        if (lm.s == 0) nhiter += np;
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
    if (a.item_nl && item_idx >= 0 && lane == 0) a.item_nl[item_idx] = make_int2(-1, 0);
    scan_item(op, I, g, a.nb, a.pos, it.cell, lm.lsh, lm.s, lm.live, w, ncand);
  }
  if constexpr (kFixedH) {
    if (list_mode && scan) {
      if (a.item_nl && item_idx >= 0 && lane == 0) a.item_nl[item_idx] = make_int2(-1, 0);
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

// The loop kernels are instantiated per kernel shape K (kKernelCubic,
// kKernelWendlandC2, kKernelWendlandC4), so the shape is fixed at compile time.
template <int K, bool kFixedH>
__global__ void __launch_bounds__(kLoopThreads, 5) k_density(DensArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const unsigned lane = lane_id();
  const Grid g = *a.grid;
  const float Lmax = fmaxf(g.L[0], fmaxf(g.L[1], g.L[2]));
  WarpSmem& w = warp_smem(smem);

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
      const int pbase = s_base[0] + s_tot[wib], ibase = s_base[1] + s_nit[wib];
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
    for (;;) {
      const int t = take_ticket(&a.ctr[ctr_index(pass, 2)]);
      if (t >= n_items) break;
      const Item it = items[t];
      dens_item<kFixedH>(a, op, g, w, it, plist, pass == 0 && (kFixedH || !a.single_pass), last, items_next,
                         plist_next, ctr_next,
                Lmax, ninter, nhiter, ncand, pass == 0 ? t : -1);
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
__global__ void k_ghost(int n, const unsigned* __restrict__ perm, const float4* __restrict__ pos,
                        const float4* __restrict__ rho4, const float4* __restrict__ cd, const float* __restrict__ u,
                        const float* __restrict__ alpha_v, const float* __restrict__ alpha_c, Phys ph,
                        float4* __restrict__ ga, float4* __restrict__ gb) {
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
  void* out;        // caller order: float2 (gradient) / float4 (force)
  float2* out2;     // fused gradient + force: the gradient's float2 output
  float* dhdt;      // force: caller order, may be NULL
  double* red_partial;  // force: [gridDim.x][8]
  Status* st;
  unsigned long long* stats;
  const unsigned* nlist;  // candidate lists kept by the density call (NULL: scan)
  const int2* item_nl;
  const unsigned long long* nl_ctr;  // space the items asked for (above nl_cap: the lists are not used)
  long long nl_cap;
};


__device__ __forceinline__ void grad_item(const LoopArgs& a, const GradOp& op, const Grid& g, WarpSmem& w,
                                          const Item& it, int t, float Lmax, unsigned& ninter, unsigned& ncand) {
  const LaneMap lm = lane_map(it.cnt, a.lmax);
  const int k = a.plist[it.off + (lm.live ? lm.slot : 0)];
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
  int sm;
  const unsigned* sl = kept_list(a.nlist, a.item_nl, t, sm, a.nl_ctr, a.nl_cap);
  scan_item(op, I, g, a.nb, a.pos, it.cell, lm.lsh, lm.s, lm.live, w, ncand, sl, sm);
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
  const int n_items = a.ctr[0];
  unsigned ninter = 0, ncand = 0;
  for (;;) {
    const int t = take_ticket(a.ticket);
    if (t >= n_items) break;
    const Item it = a.items[t];
    grad_item(a, op, g, w, it, t, Lmax, ninter, ncand);
  }
  ninter = warp_sum(ninter);
  ncand = warp_sum(ncand);
  if (lane == 0) {
    atomicAdd(&a.stats[kStatInterGrad], (unsigned long long)ninter);
    atomicAdd(&a.stats[kStatCandGrad], (unsigned long long)ncand);
  }
}

// =============================================================== force loop
// kGrad: the gradient loop fused in (GradForceOp), writing both outputs.
template <bool kGrad>
__device__ __forceinline__ void force_item(const LoopArgs& a,
                                           const typename std::conditional<kGrad, GradForceOp, ForceOp>::type& op,
                                           const Grid& g, WarpSmem& w, const Item& it, int t, unsigned& ninter,
                                           unsigned& nginter, unsigned& ncand, float* acc, float* accc) {
  using Op = typename std::conditional<kGrad, GradForceOp, ForceOp>::type;
  const LaneMap lm = lane_map(it.cnt, a.lmax);
  const int k = a.plist[it.off + (lm.live ? lm.slot : 0)];
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
  int sm;
  const unsigned* sl = kept_list(a.nlist, a.item_nl, t, sm, a.nl_ctr, a.nl_cap);
  scan_item(op, I, g, a.nb, a.pos, it.cell, lm.lsh, lm.s, lm.live, w, ncand, sl, sm);
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

template <bool kGrad, int K>
__device__ __forceinline__ void force_kernel_body(const LoopArgs& a) {
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
  const int n_items = a.ctr[0];
  unsigned ninter = 0, nginter = 0, ncand = 0;
  // per-thread partials of the global sums: FP32 TwoSum pairs (sum, error),
  // carried into FP64 for the block and global sums
  float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0}, accc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (;;) {
    const int t = take_ticket(a.ticket);
    if (t >= n_items) break;
    const Item it = a.items[t];
    force_item<kGrad>(a, op, g, w, it, t, ninter, nginter, ncand, acc, accc);
  }
  // block partial of the FP64 sums (summed in block order by k_reduce_partials)
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    double x = (double)acc[q] + (double)accc[q];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    if (lane == 0) red[threadIdx.x >> 5][q] = x;
  }
  __syncthreads();
  if (threadIdx.x < 8) {
    double x = 0.0;
    for (int ww = 0; ww < kWarpsPerBlock; ++ww) x += red[ww][threadIdx.x];
    a.red_partial[blockIdx.x * 8 + threadIdx.x] = x;
  }
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
}

template <int K>
__global__ void __launch_bounds__(kLoopThreads, 4) k_force(LoopArgs a) { force_kernel_body<false, K>(a); }

// Gradient (Eqs. 10-11, Laplacian of u) and force in one pass over the pairs.
template <int K>
__global__ void __launch_bounds__(kLoopThreads, 5) k_grad_force(LoopArgs a) { force_kernel_body<true, K>(a); }

// One warp per quantity; lane l sums blocks l, l+32, ... and the warp then
// combines the lanes in a fixed order, so the result does not depend on timing.
__global__ void k_reduce_partials(const double* __restrict__ part, int nblocks, double* __restrict__ out) {
  const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double x = 0.0;
  for (int b = lane; b < nblocks; b += 32) x += part[b * 8 + q];
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  if (lane == 0) out[q] = x;
}

// =================================================================== hosts
static int persistent_blocks(Ctx* c, const void* kern) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kLoopThreads, kLoopSmemBytes);
  if (per_sm < 1) per_sm = 1;
  if (c->tuning.blocks_per_sm > 0 && c->tuning.blocks_per_sm < per_sm) per_sm = c->tuning.blocks_per_sm;
  int nb = per_sm * c->num_sms;
  return nb < c->red_blocks ? nb : c->red_blocks;
}

// The instantiation of each loop kernel for kernel shape `kind`.
static const void* density_kernel(int kind, bool fixed_h) {
  if (fixed_h)
    return kind == kKernelWendlandC2 ? (const void*)k_density<kKernelWendlandC2, true>
           : kind == kKernelWendlandC4 ? (const void*)k_density<kKernelWendlandC4, true>
                                       : (const void*)k_density<kKernelCubic, true>;
  return kind == kKernelWendlandC2 ? (const void*)k_density<kKernelWendlandC2, false>
         : kind == kKernelWendlandC4 ? (const void*)k_density<kKernelWendlandC4, false>
                                     : (const void*)k_density<kKernelCubic, false>;
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

static bool g_attr_done = false;
static void ensure_attrs() {
  if (g_attr_done) return;
  for (int kind = kKernelCubic; kind <= kKernelWendlandC4; ++kind)
    for (const void* f : {density_kernel(kind, false), density_kernel(kind, true), gradient_kernel(kind),
                          force_kernel(kind), grad_force_kernel(kind)})
      cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLoopSmemBytes);
  g_attr_done = true;
}

static cudaError_t launch_loop(const void* f, int nblk, LoopArgs& a, cudaStream_t s) {
  void* args[] = {&a};
  return cudaLaunchKernel(f, dim3(nblk), dim3(kLoopThreads), args, kLoopSmemBytes, s);
}

void reduce_partials(Ctx* c, int nblocks, double* out, cudaStream_t s) {
  k_reduce_partials<<<1, 256, 0, s>>>(c->d_red_partial, nblocks, out);
  c->launches++;
}

int density_impl(Ctx* c, const float4* pos_in, const float4* vel_in, const uint8_t* active, float* h_out,
                 float4* rho4, float4* cd, uint32_t* ngb, cudaStream_t s) {
  ensure_attrs();
  const void* kern = density_kernel(c->phys.kernel, (c->params.flags & SWIFT_GPU_NO_H_ITER) != 0);
  const int nblk = persistent_blocks(c, kern);
  cudaMemsetAsync(c->d_counters, 0, sizeof(int) * (size_t)(kCtrPerPass * (c->max_passes + 2) + 2), s);
  DensArgs a;
  a.grid = c->d_grid;
  a.nb = nbr_of(c);
  a.perm = c->d_vals[c->sorted_buf];
  a.n = c->n;
  a.ph = c->phys;
  a.lmax = c->tuning.max_lanes_per_particle;
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
  a.nlist = c->d_nlist;
  a.nl_cap = c->nl_cap;
  a.nl_ctr = c->d_nl_ctr;
  a.item_nl = c->d_nlist ? c->d_item_nl : nullptr;
  if (c->d_nl_ctr) cudaMemsetAsync(c->d_nl_ctr, 0, sizeof(unsigned long long), s);
  void* args[] = {&a};
  cudaError_t e = cudaLaunchCooperativeKernel(kern, dim3(nblk), dim3(kLoopThreads), args, kLoopSmemBytes, s);
  c->launches += 2;
  c->all_active = active == nullptr;
  c->nl_lmax = a.item_nl ? c->tuning.max_lanes_per_particle : 0;  // lists follow this lane layout
  return e == cudaSuccess ? SWIFT_GPU_OK : SWIFT_GPU_ERR_CUDA;
}

int ghost_impl(Ctx* c, const float* u, const float* alpha_v, const float* alpha_c, cudaStream_t s) {
  if (c->n == 0) return SWIFT_GPU_OK;
  const int nb = min((c->n + 255) / 256, c->num_sms * 8);
  k_ghost<<<nb, 256, 0, s>>>(c->n, c->d_vals[c->sorted_buf], c->d_pos, c->d_rho4, c->d_cd, u, alpha_v, alpha_c,
                             c->phys, c->d_ga, c->d_gb);
  c->launches++;
  return cudaGetLastError() == cudaSuccess ? SWIFT_GPU_OK : SWIFT_GPU_ERR_CUDA;
}

static LoopArgs loop_args(Ctx* c, int* ticket, void* out) {
  LoopArgs a;
  a.grid = c->d_grid;
  a.nb = nbr_of(c);
  a.perm = c->d_vals[c->sorted_buf];
  a.ph = c->phys;
  a.lmax = c->tuning.max_lanes_per_particle;
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
  const bool lists = kept_lists_usable(c);
  a.nlist = lists ? c->d_nlist : nullptr;
  a.item_nl = lists ? c->d_item_nl : nullptr;
  a.nl_ctr = c->d_nl_ctr;
  a.nl_cap = c->nl_cap;
  return a;
}

int gradient_impl(Ctx* c, float2* out, cudaStream_t s) {
  ensure_attrs();
  const void* kern = gradient_kernel(c->phys.kernel);
  const int nblk = persistent_blocks(c, kern);
  int* ticket = c->d_counters + kCtrPerPass * (c->max_passes + 1) + 0;
  cudaMemsetAsync(ticket, 0, sizeof(int), s);
  LoopArgs a = loop_args(c, ticket, out);
  const cudaError_t e = launch_loop(kern, nblk, a, s);
  c->launches += 2;
  return e == cudaSuccess ? SWIFT_GPU_OK : SWIFT_GPU_ERR_CUDA;
}

int force_impl(Ctx* c, float4* out, float* dhdt, double* reductions, cudaStream_t s) {
  ensure_attrs();
  const void* kern = force_kernel(c->phys.kernel);
  const int nblk = persistent_blocks(c, kern);
  int* ticket = c->d_counters + kCtrPerPass * (c->max_passes + 1) + 1;
  cudaMemsetAsync(ticket, 0, sizeof(int), s);
  LoopArgs a = loop_args(c, ticket, out);
  a.dhdt = dhdt;
  if (launch_loop(kern, nblk, a, s) != cudaSuccess) return SWIFT_GPU_ERR_CUDA;
  c->launches += 2;
  if (reductions) {
    k_reduce_partials<<<1, 256, 0, s>>>(c->d_red_partial, nblk, reductions);
    c->launches++;
  }
  return cudaGetLastError() == cudaSuccess ? SWIFT_GPU_OK : SWIFT_GPU_ERR_CUDA;
}

int grad_force_impl(Ctx* c, float2* grad_out, float4* out, float* dhdt, double* reductions, cudaStream_t s) {
  ensure_attrs();
  const void* kern = grad_force_kernel(c->phys.kernel);
  const int nblk = persistent_blocks(c, kern);
  int* ticket = c->d_counters + kCtrPerPass * (c->max_passes + 1) + 1;
  cudaMemsetAsync(ticket, 0, sizeof(int), s);
  LoopArgs a = loop_args(c, ticket, out);
  a.out2 = grad_out;
  a.dhdt = dhdt;
  if (launch_loop(kern, nblk, a, s) != cudaSuccess) return SWIFT_GPU_ERR_CUDA;
  c->launches += 2;
  if (reductions) {
    k_reduce_partials<<<1, 256, 0, s>>>(c->d_red_partial, nblk, reductions);
    c->launches++;
  }
  return cudaGetLastError() == cudaSuccess ? SWIFT_GPU_OK : SWIFT_GPU_ERR_CUDA;
}

}  // namespace sg
