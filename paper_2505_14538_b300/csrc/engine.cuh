// engine.cuh -- the warp-level neighbour scan shared by every pair loop.
//
// A work item is a run of <= 16 active particles of one cell (Sec. 2.2:
// self and pair interactions of a cell with its 26 neighbours) or, with
// adaptive leaves, of one leaf. One warp handles one item:
//
//   segments  lanes 0..26 each look up one of the 27 neighbour cells (with
//             its periodic image), or up to 32 lanes one entry each of the
//             leaf's neighbour list, and a warp scan concatenates them into
//             one candidate sequence, so candidates are taken in full chunks
//             of 32 whatever the cell or leaf occupancies;
//   phase 1   a chunk of 32 candidates is staged in shared memory by one
//             coalesced float4 load per lane; each lane tests its particle
//             against its share of the chunk (r^2 < support^2 + guard band)
//             and appends hits to a lane-private list in shared memory;
//   phase 2   when a list could overflow, and at the end, each lane walks its
//             own list and evaluates the full pair interaction, so the costly
//             arithmetic runs on converged lanes instead of diverging on the
//             ~15 % hit rate of a 27-cell scan.
//
// With few particles in an item, L = 2, 4, 8, 16 or 32 lanes share one
// particle and split its candidates.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace sg {

constexpr int kCap = 64;  // list entries per lane before a flush
constexpr unsigned kFull = 0xffffffffu;

struct WarpSmem {
  // lane-private lists, entry t of lane l at [t * 32 + l]; row kCap takes the
  // stores of collect_item's tests that miss once a list is full
  unsigned list[(kCap + 1) * 32];
  float4 stage[32];          // current chunk: shifted position + per-loop w
  unsigned stage_idx[32];    // current chunk: j | shift code << kIndexBits
  int seg_start[32];
  unsigned seg_code[32];
  int seg_pref[33];
};

// log2 of the lanes per particle for an item of cnt particles (L = 2^lsh <= lmax).
__device__ __forceinline__ int lanes_shift(int cnt, int lmax) {
  int lsh = cnt <= 1 ? 5 : cnt <= 2 ? 4 : cnt <= 4 ? 3 : cnt <= 8 ? 2 : cnt <= 16 ? 1 : 0;
  while ((1 << lsh) > lmax) --lsh;
  return lsh;
}

// The candidate segments of an item: the 27 neighbour cells of `cell`, or
// nseg entries of a leaf list from list_off.
struct Segs {
  int cell;
  int list_off;
  int nseg;
  bool list;
};

__device__ __forceinline__ Segs item_segments(const Nbr& nb, int item_cell) {
  Segs q;
  q.cell = item_cell;
  q.list_off = 0;
  q.nseg = 27;
  q.list = false;
  if (nb.adaptive) {
    const int2 sp = nb.nbr_span[item_cell];
    if (sp.y <= nb.nbr_cap - sp.x) {
      q.list_off = sp.x;
      q.nseg = sp.y;
      q.list = true;
    } else {
      q.cell = (int)nb.skeys[nb.leaf_range[item_cell].x];
    }
  }
  return q;
}

// Segments sb .. sb + bn - 1 (bn = min(32, nseg - sb) >= 1) of an item, one
// per lane, concatenated by a warp scan; returns their candidate count.
__device__ __forceinline__ int setup_segments(const Grid& g, const Nbr& nb, const Segs& q, int sb, WarpSmem& w,
                                              int& bn) {
  const unsigned lane = lane_id();
  bn = min(32, q.nseg - sb);
  int len = 0;
  if ((int)lane < bn) {
    int b;
    unsigned code;
    if (q.list) {
      const unsigned e = nb.nbr[q.list_off + sb + (int)lane];
      const int2 r = nb.leaf_range[e & kIndexMask];
      b = r.x;
      len = r.y - r.x;
      code = e >> kIndexBits;
    } else {
      const int nx = g.nc[0], ny = g.nc[1], nz = g.nc[2];
      const int cell = q.cell;
      const int cx = cell % nx, cy = (cell / nx) % ny, cz = cell / (nx * ny);
      int x = cx + (int)(lane % 3u) - 1, y = cy + (int)((lane / 3u) % 3u) - 1, z = cz + (int)(lane / 9u) - 1;
      code = 0;
      if (x < 0) { x += nx; code |= 2u; } else if (x >= nx) { x -= nx; code |= 1u; }
      if (y < 0) { y += ny; code |= 8u; } else if (y >= ny) { y -= ny; code |= 4u; }
      if (z < 0) { z += nz; code |= 32u; } else if (z >= nz) { z -= nz; code |= 16u; }
      const int c = x + nx * (y + ny * z);
      b = nb.cell_start[c];
      len = nb.cell_start[c + 1] - b;
    }
    w.seg_start[lane] = b;
    w.seg_code[lane] = code;
  }
  int incl = len;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(kFull, incl, o);
    if ((int)lane >= o) incl += y;
  }
  if ((int)lane < bn) w.seg_pref[lane + 1] = incl;
  if (lane == 0) w.seg_pref[0] = 0;
  __syncwarp();
  return __shfl_sync(kFull, incl, bn - 1);
}

// Stage candidate `p` (< the batch total) of the current segment batch: its
// position with the periodic shift applied, and its list entry.
__device__ __forceinline__ void stage_candidate(const Grid& g, const float4* __restrict__ pos, const WarpSmem& w,
                                                int bn, int p, float4& pj, unsigned& entry) {
  int q = 0;
#pragma unroll
  for (int step = 16; step > 0; step >>= 1)
    if (q + step < bn && w.seg_pref[q + step] <= p) q += step;
  const int j = w.seg_start[q] + (p - w.seg_pref[q]);
  const unsigned code = w.seg_code[q];
  pj = pos[j];
  shift_j(code, g.L, pj.x, pj.y, pj.z);
  entry = (unsigned)j | (code << kIndexBits);
}

// Evens out the list lengths of the L = 2^lsh lanes that share one particle
// (lanes slot + k A, A = 32 >> lsh, sub-lane k = lane / A): a particle with T
// entries ends with T / L entries in each of its lanes, plus one in the first
// T % L of them. Entries past a lane's new length move, in order, to the ends
// of the lanes that are short. Which lane takes an entry changes a sum only by
// rounding, and a phase over the lists then runs as many trips as the
// particle's T / L needs instead of its longest lane. Every lane of the warp
// calls it (lsh is the same for the whole item); returns the lane's new count.
__device__ __forceinline__ int balance_lists(WarpSmem& w, int cnt, int lsh) {
  if (lsh == 0) return cnt;
  const unsigned lane = lane_id();
  const int A = 32 >> lsh, L = 1 << lsh;
  int T = cnt;
  for (int o = A; o < 32; o <<= 1) T += __shfl_xor_sync(kFull, T, o);
  const int sub = (int)lane >> (5 - lsh);
  const int target = (T >> lsh) + (sub < (T & (L - 1)) ? 1 : 0);
  const int sur = cnt > target ? cnt - target : 0;
  const int def = target > cnt ? target - cnt : 0;
  if (!__any_sync(kFull, sur > 0)) return cnt;
  int ps = sur, pd = def;  // inclusive prefixes over the particle's sub-lanes
  for (int o = A; o < 32; o <<= 1) {
    const int ys = __shfl_up_sync(kFull, ps, o);
    const int yd = __shfl_up_sync(kFull, pd, o);
    if ((int)lane >= o) {
      ps += ys;
      pd += yd;
    }
  }
  const int es = ps - sur, ed = pd - def;  // this lane's surplus units [es, ps), wanted units [ed, pd)
  const int slot = (int)lane & (A - 1);
  __syncwarp();
  for (int k = 0; k < L; ++k) {
    const int src = slot + k * A;
    const int es_k = __shfl_sync(kFull, es, src);
    const int ps_k = __shfl_sync(kFull, ps, src);
    const int tg_k = __shfl_sync(kFull, target, src);
    const int lo = max(ed, es_k), hi = min(pd, ps_k);
    for (int u = lo; u < hi; ++u)
      w.list[(cnt + (u - ed)) * 32 + (int)lane] = w.list[(tg_k + (u - es_k)) * 32 + src];
  }
  __syncwarp();
  return target;
}

// Phase 2: each lane evaluates the interactions in its list.
template <class Op>
__device__ __forceinline__ void flush(const Op& op, typename Op::I& I, const WarpSmem& w, int cnt) {
  const unsigned lane = lane_id();
  const int m = __reduce_max_sync(kFull, cnt);
  for (int t = 0; t < m; ++t) {
    if (t < cnt) {
      const unsigned e = w.list[t * 32 + lane];
      op.interact(I, (int)(e & kIndexMask), e >> kIndexBits);
    }
  }
}

// Phase 2 for an Op with a record type (Op::Rec, Op::load): each entry's
// records are loaded by every lane, past the end of its list its own particle's,
// before the branch, and the interaction follows. Against the loads inside the
// branch (flush): adaptive zeldovich256 gradient + force 37.6 -> 35.2 ms. Two
// entries' records at a time spilled at the fused kernel's 128 registers.
template <class Op>
__device__ __forceinline__ void flush_loaded(const Op& op, typename Op::I& I, const WarpSmem& w, int cnt) {
  const unsigned lane = lane_id();
  const int m = __reduce_max_sync(kFull, cnt);
  for (int t = 0; t < m; ++t) {
    const unsigned e = t < cnt ? w.list[t * 32 + lane] : (unsigned)I.k;
    typename Op::Rec r;
    op.load((int)(e & kIndexMask), r);
    if (t < cnt) op.interact(I, (int)(e & kIndexMask), e >> kIndexBits, r);
  }
}

template <class Op, class = void>
struct has_load : std::false_type {};
template <class Op>
struct has_load<Op, decltype((void)sizeof(typename Op::Rec))> : std::true_type {};

template <class Op>
__device__ __forceinline__ void flush_any(const Op& op, typename Op::I& I, const WarpSmem& w, int cnt) {
  if constexpr (has_load<Op>::value) flush_loaded(op, I, w, cnt);
  else flush(op, I, w, cnt);
}

// Next chunk of an item's candidates: moves `base` past the current chunk
// (to the next batch of segments when the batch is used up) and returns the
// chunk's length, 0 at the end.
__device__ __forceinline__ int next_chunk(const Grid& g, const Nbr& nb, const Segs& q, WarpSmem& w, int& sb,
                                          int& bn, int& total, int& base) {
  base += 32;
  while (base >= total && sb + 32 < q.nseg) {
    sb += 32;
    base = 0;
    __syncwarp();
    total = setup_segments(g, nb, q, sb, w, bn);
  }
  return base < total ? min(32, total - base) : 0;
}

// Full neighbour scan of one item for lane particle I (sub-lane s of the
// 2^lsh lanes that share the particle). Segments come in batches of up to
// 32; candidates are taken in chunks of 32 within a batch. The loads of the
// next chunk are issued before the current one is tested (software
// pipelining: the test hides their latency). One flush site keeps the
// inlined interaction code in a single copy.
template <class Op>
__device__ __forceinline__ void scan_item(const Op& op, typename Op::I& I, const Grid& g, const Nbr& nb,
                                          const float4* __restrict__ pos, int cell, int lsh, int s, bool live,
                                          WarpSmem& w, unsigned& ncand) {
  const unsigned lane = lane_id();
  int cnt = 0;
  int bn = 0, sb = 0, base = -32, total = 0;
  const Segs q = item_segments(nb, cell);
  if (q.nseg > 0) total = setup_segments(g, nb, q, 0, w, bn);
  int len = next_chunk(g, nb, q, w, sb, bn, total, base);
  float4 pj = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  unsigned ej = 0;
  if ((int)lane < len) stage_candidate(g, pos, w, bn, base + (int)lane, pj, ej);
  const int per = 32 >> lsh;  // candidates a lane tests per chunk (at most)
  for (;;) {
    const bool done = len == 0;
    if (done || __any_sync(kFull, cnt > kCap - per)) {
      flush_any(op, I, w, cnt);
      cnt = 0;
      if (done) break;
    }
    __syncwarp();
    if ((int)lane < len) {
      w.stage[lane] = make_float4(pj.x, pj.y, pj.z, op.stage_w(pj.w));
      w.stage_idx[lane] = ej;
    }
    const int cur = len;
    __syncwarp();
    len = next_chunk(g, nb, q, w, sb, bn, total, base);
    if ((int)lane < len) stage_candidate(g, pos, w, bn, base + (int)lane, pj, ej);
    if (live) {
      const int nk = cur > s ? ((cur - s - 1) >> lsh) + 1 : 0;
#pragma unroll 4
      for (int kk = 0; kk < nk; ++kk) {
        const int k = (kk << lsh) + s;
        const float4 c = w.stage[k];
        const float dx = I.x - c.x, dy = I.y - c.y, dz = I.z - c.z;
        if (op.candidate(I, r2_of(dx, dy, dz), c.w)) {
          w.list[cnt * 32 + lane] = w.stage_idx[k];
          ++cnt;
        }
      }
      ncand += (unsigned)nk;
    }
  }
}

// Phase 1 only, for the h iteration: every candidate with r^2 < R2 (the
// largest support any h may reach) goes into the lane's list, which is never
// flushed; `ovf` is set when the list is full (the particle then takes the
// multi-pass route). Pipelined like scan_item.
__device__ __forceinline__ int collect_item(const Grid& g, const Nbr& nb, const float4* __restrict__ pos, int cell,
                                            float xi, float yi, float zi, float R2, int lsh, int s, bool live,
                                            WarpSmem& w, unsigned& ncand, bool& ovf) {
  const unsigned lane = lane_id();
  const Segs q = item_segments(nb, cell);
  int bn = 0, sb = 0, base = -32, total = 0;
  if (q.nseg > 0) total = setup_segments(g, nb, q, 0, w, bn);
  int len = next_chunk(g, nb, q, w, sb, bn, total, base);
  float4 pj = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  unsigned ej = 0;
  if ((int)lane < len) stage_candidate(g, pos, w, bn, base + (int)lane, pj, ej);
  int cnt = 0;
  while (len > 0) {
    __syncwarp();
    if ((int)lane < len) {
      w.stage[lane] = pj;
      w.stage_idx[lane] = ej;
    }
    const int cur = len;
    __syncwarp();
    len = next_chunk(g, nb, q, w, sb, bn, total, base);
    if ((int)lane < len) stage_candidate(g, pos, w, bn, base + (int)lane, pj, ej);
    if (live) {
      const int nk = cur > s ? ((cur - s - 1) >> lsh) + 1 : 0;
#pragma unroll 4
      for (int kk = 0; kk < nk; ++kk) {
        const int k = (kk << lsh) + s;
        // branch-free: every test stores its entry at the list's end, and
        // a hit keeps it (a miss is overwritten by the next store)
        const float4 c = w.stage[k];
        const unsigned ix = w.stage_idx[k];
        const float dx = xi - c.x, dy = yi - c.y, dz = zi - c.z;
        const bool hit = r2_of(dx, dy, dz) < R2;
        w.list[min(cnt, kCap) * 32 + lane] = ix;
        ovf = ovf || (hit && cnt >= kCap);
        cnt += (hit && cnt < kCap) ? 1 : 0;
      }
      ncand += (unsigned)nk;
    }
  }
  __syncwarp();
  return cnt;
}

// Combination of the sub-lanes of one particle (lanes a, a + A, a + 2A, ...
// with A = 32 >> lsh).
__device__ __forceinline__ float lsum(float v, int lsh) {
  for (int o = 32 >> lsh; o < 32; o <<= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
__device__ __forceinline__ float lmax(float v, int lsh) {
  for (int o = 32 >> lsh; o < 32; o <<= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
  return v;
}
__device__ __forceinline__ unsigned lsum_u(unsigned v, int lsh) {
  for (int o = 32 >> lsh; o < 32; o <<= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
// Compensated pair (s, c): TwoSum of the partial sums, errors carried in c.
__device__ __forceinline__ void lsum2(float& s, float& c, int lsh) {
  for (int o = 32 >> lsh; o < 32; o <<= 1) {
    const float so = __shfl_xor_sync(kFull, s, o);
    const float co = __shfl_xor_sync(kFull, c, o);
    const float t = s + so;
    const float bp = t - s;
    const float e = (s - (t - bp)) + (so - bp);
    s = t;
    c = c + co + e;
  }
}

__device__ __forceinline__ int take_ticket(int* ticket) {
  int t = 0;
  if (lane_id() == 0) t = atomicAdd(ticket, 1);
  return __shfl_sync(kFull, t, 0);
}

}  // namespace sg
