// lpp.cuh -- the lane-per-particle neighbour search of the uniform grid.
//
// A warp takes 32 consecutive active particles (a "group", several cells
// wide) and each lane works on its own particle from start to end: no lanes
// share a particle, none is idle while the group is full, and no sub-lane
// sums are combined.
//
// Candidates come from the 27 cells around the lane's own cell (Sec. 2.2:
// self and pair interactions of cells no narrower than the support), found
// in one of two ways: the shared rows (rows_collect, below: the group's lanes
// test, in step, every particle of the rows of cells their neighbourhoods
// share), or per lane through windows on sorted replicas, as follows. For a
// neighbour cell at offset o (one of 26), the cell's particles are read in
// the order of their projection on o (SWIFT's sorted pair interactions,
// Sec. 2.2.2: cells sorted along the 13 pair axes), and the lane stops at the
// first particle whose projection passes the lane's own projection by more
// than |o| times the support: every particle after it is farther than the
// support along o, so farther in space too (|o . d| <= |o| |d|). On a
// lattice-like set this tests about 80 candidates a particle instead of the
// 27 cells' ~360.
//
// The sorted orders are "replicas": for each of the 13 axes, every cell's
// particles as (x, y, z, sorted index) in ascending projection, stored
// cell-major with the same cell starts as the sorted arrays. They are built
// per cell by one warp (a rank sort, cells of at most kRepMax particles);
// larger cells have no replica and are read whole, in sorted order.
#pragma once

#include "common.cuh"

namespace sg {

constexpr int kAxes = 13;
constexpr int kRepMax = 32;  // largest cell with replicas (one particle a lane)

// Width W of a lane's candidate list, per kernel shape: above the most
// candidates within the cell cap's support (57 to about 75 on a jittered
// lattice at the cubic spline's eta, about 90 and 110 with the Wendland
// shapes' wider supports); a particle with more takes the multi-pass route.
// The cubic spline's 92 lets four blocks of the density kernel share an SM.
__host__ __device__ constexpr int lpp_width_of(int kind) {
  return kind == kKernelCubic ? 92 : kind == kKernelWendlandC2 ? 128 : 160;
}

// Canonical pair axes: the 13 offsets o in {-1,0,1}^3 whose first nonzero
// component (x, then y, then z) is positive. Axis a: 0..8 -> (1, a%3-1, a/3-1),
// 9..11 -> (0, 1, a-10), 12 -> (0, 0, 1).
__host__ __device__ __forceinline__ void axis_vec(int a, int& ox, int& oy, int& oz) {
  if (a < 9) {
    ox = 1;
    oy = a % 3 - 1;
    oz = a / 3 - 1;
  } else if (a < 12) {
    ox = 0;
    oy = 1;
    oz = a - 10;
  } else {
    ox = 0;
    oy = 0;
    oz = 1;
  }
}

// Axis and direction of offset o != 0: o = s * axis(a).
__host__ __device__ __forceinline__ void axis_of(int ox, int oy, int oz, int& a, int& s) {
  s = (ox > 0 || (ox == 0 && (oy > 0 || (oy == 0 && oz > 0)))) ? 1 : -1;
  const int px = s * ox, py = s * oy, pz = s * oz;
  a = px == 1 ? (py + 1) + 3 * (pz + 1) : py == 1 ? 10 + pz : 12;
}

// Projection of a position on an integer offset, one fixed expression (two
// roundings) everywhere: the replicas are sorted by it and the windows
// compare it.
__device__ __forceinline__ float proj(float ox, float oy, float oz, float x, float y, float z) {
  return fmaf(oz, z, fmaf(oy, y, ox * x));
}

// Total order key of a float (negative values flipped): orders like the
// values, NaN included somewhere, so a rank sort by (key, index) is a
// permutation whatever the inputs.
__device__ __forceinline__ unsigned order_key(float d) {
  const unsigned b = __float_as_uint(d);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// One warp writes the 13 replicas of cell [cs, ce) (ce - cs <= kRepMax):
// rep[a * stride + cs + rank] = (x, y, z, sorted index) with rank the place
// of the particle in ascending projection on axis a (ties by index).
// p is the lane's particle (lane < ce - cs), already wrapped into the box.
// The ranks of all 13 axes are counted in one pass over the cell's
// particles (13 independent shuffles per particle).
__device__ __forceinline__ void build_replicas_cell(float4* __restrict__ rep, long long stride, int cs, int m,
                                                    float4 p) {
  const unsigned lane = lane_id();
  unsigned key[kAxes];
  int rank[kAxes];
#pragma unroll
  for (int a = 0; a < kAxes; ++a) {
    int ox, oy, oz;
    axis_vec(a, ox, oy, oz);
    key[a] = order_key(proj((float)ox, (float)oy, (float)oz, p.x, p.y, p.z));
    rank[a] = 0;
  }
  for (int u = 0; u < m; ++u) {
    const bool before = u < (int)lane;
#pragma unroll
    for (int a = 0; a < kAxes; ++a) {
      const unsigned ku = __shfl_sync(0xffffffffu, key[a], u);
      rank[a] += (ku < key[a] || (ku == key[a] && before)) ? 1 : 0;
    }
  }
  if ((int)lane < m) {
    const float4 e = make_float4(p.x, p.y, p.z, __uint_as_float((unsigned)(cs + (int)lane)));
#pragma unroll
    for (int a = 0; a < kAxes; ++a) rep[a * stride + cs + rank[a]] = e;
  }
}

// The neighbour cell of offset q (0..26; q = 13 is the own cell) of cell
// (cx, cy, cz), its periodic shift code (as shift_j reads it) and the shift
// S that the image of its particles carries.
struct NbrCell {
  int c;
  unsigned code;
  float sx, sy, sz;
  int ox, oy, oz;
};

__device__ __forceinline__ NbrCell nbr_cell(const Grid& g, int cx, int cy, int cz, int q) {
  NbrCell r;
  r.ox = q % 3 - 1;
  r.oy = (q / 3) % 3 - 1;
  r.oz = q / 9 - 1;
  const int nx = g.nc[0], ny = g.nc[1], nz = g.nc[2];
  int x = cx + r.ox, y = cy + r.oy, z = cz + r.oz;
  r.code = 0;
  r.sx = r.sy = r.sz = 0.0f;
  if (x < 0) { x += nx; r.code |= 2u; r.sx = -g.L[0]; } else if (x >= nx) { x -= nx; r.code |= 1u; r.sx = g.L[0]; }
  if (y < 0) { y += ny; r.code |= 8u; r.sy = -g.L[1]; } else if (y >= ny) { y -= ny; r.code |= 4u; r.sy = g.L[1]; }
  if (z < 0) { z += nz; r.code |= 32u; r.sz = -g.L[2]; } else if (z >= nz) { z -= nz; r.code |= 16u; r.sz = g.L[2]; }
  r.c = x + nx * (y + ny * z);
  return r;
}

// Collect, for the lane's particle at (xi, yi, zi) in cell `cell`, every
// candidate j (itself included) with FP32 r^2 < R2 from the 27 cells, reading
// each neighbour cell through its window. Entry t goes to lst[t * 32]
// (j | shift code << kIndexBits) and its r^2 to r2s[t * 32], for t < W;
// more candidates set ovf. Returns the count.
//
// The window of neighbour offset o: the particles with proj(o, x_j) <
// proj(o, x_i - S) + |o| Rc + margin (Rc = sqrt(R2)), read in ascending
// proj(o, .) (the replica of o's axis, forwards or backwards). Rounding: both
// projections carry at most about 2^-20 L of error with coordinates within
// [-L, 2L), and the margin is 2^-17 L, so the window keeps every candidate the
// FP32 test would accept.
//
// Latency: the candidates are read four at a time, all four loads issued
// first; the next offset's cell bounds are loaded, and its entries prefetched
// into L1, while the current offset's window is read.
__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

template <int W>
__device__ __forceinline__ int lpp_collect(const Grid& g, const int* __restrict__ cell_start,
                                           const float4* __restrict__ pos, const float4* __restrict__ rep,
                                           long long stride, float xi, float yi, float zi, int cell, float R2,
                                           float Lmax, bool live, unsigned* __restrict__ lst, float* r2s, bool& ovf,
                                           unsigned& ncand) {
  const int nx = g.nc[0], ny = g.nc[1];
  const int cx = cell % nx, cy = (cell / nx) % ny, cz = cell / (nx * ny);
  const float Rc = sqrtf(R2);
  const float margin = 7.62939453125e-06f * Lmax;  // 2^-17 L
  int cnt = 0;
  NbrCell nxt = nbr_cell(g, cx, cy, cz, 0);
  int nxt_cs = cell_start[nxt.c], nxt_ce = cell_start[nxt.c + 1];
#pragma unroll 1
  for (int q = 0; q < 27; ++q) {
    const NbrCell nbc = nxt;
    const int cs = nxt_cs, m = nxt_ce - nxt_cs;
    const bool rep_ok = m <= kRepMax;  // the cell has replicas
    const bool self = q == 13;
    const bool win = !self && rep_ok;
    int a = 0, s = 1;
    if (!self) axis_of(nbc.ox, nbc.oy, nbc.oz, a, s);
    const float4* base = rep_ok ? rep + (long long)a * stride + cs : pos + cs;
    int step = 1;
    if (win && s < 0) {
      base += m - 1;
      step = -1;
    }
    if (q + 1 < 27) {
      nxt = nbr_cell(g, cx, cy, cz, q + 1);
      nxt_cs = cell_start[nxt.c];
      nxt_ce = cell_start[nxt.c + 1];
    }
    const float xs = xi - nbc.sx, ys = yi - nbc.sy, zs = zi - nbc.sz;
    const float fx = (float)nbc.ox, fy = (float)nbc.oy, fz = (float)nbc.oz;
    float lim = 0.0f;
    if (win) {
      const int l1 = abs(nbc.ox) + abs(nbc.oy) + abs(nbc.oz);
      const float norm = l1 == 1 ? 1.0f : l1 == 2 ? 1.41421356f : 1.73205081f;
      lim = proj(fx, fy, fz, xs, ys, zs) + fmaf(norm * 1.0000002f, Rc, margin);
    }
    // four candidates at a time, all four loaded first; a lane stops at the
    // first candidate outside its window (the rest of the batch is dropped)
    bool on = live && m > 0;
    int u = 0;
    bool pf = q + 1 < 27 && live;
    while (__any_sync(0xffffffffu, on)) {
      float4 c[4];
#pragma unroll
      for (int b = 0; b < 4; ++b)
        c[b] = (on && u + b < m) ? base[step * (u + b)] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      if (pf) {
        // the next offset's cell entries into L1 (its whole cell: at most kRepMax entries, 4 lines)
        pf = false;
        const int mn = nxt_ce - nxt_cs;
        int an = 0, sn = 1;
        if (q + 1 != 13) axis_of(nxt.ox, nxt.oy, nxt.oz, an, sn);
        const float4* bn = mn <= kRepMax ? rep + (long long)an * stride + nxt_cs : pos + nxt_cs;
        const int lines = mn <= kRepMax ? (mn + 7) >> 3 : 0;
        for (int t = 0; t <= lines && mn > 0; ++t) prefetch_l1(bn + min(t * 8, mn - 1));
      }
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        if (on) {
          if (u < m && (!win || proj(fx, fy, fz, c[b].x, c[b].y, c[b].z) < lim)) {
            const float dx = xs - c[b].x, dy = ys - c[b].y, dz = zs - c[b].z;
            const float r2 = r2_of(dx, dy, dz);
            ++ncand;
            if (r2 < R2) {
              const unsigned j = rep_ok ? __float_as_uint(c[b].w) : (unsigned)(cs + u);
              if (cnt < W) {
                lst[cnt * 32] = j | (nbc.code << kIndexBits);
                r2s[cnt * 32] = r2;
              } else {
                ovf = true;
              }
              ++cnt;
            }
            ++u;
          } else {
            on = false;
          }
        }
      }
      on = on && u < m;
    }
  }
  return cnt;
}

// Plain per-lane collect over the 27 cells around `cell`, no windows: every
// candidate j (itself included) with FP32 r^2 < R2 is appended to the lane's
// list from position cnt on, the cells taken in the order q = 0..26 (x
// fastest) and each cell in sorted order. Lanes with live = false take no
// part. The fallback of rows_collect for lanes no shared row run covers.
template <int W>
__device__ __forceinline__ int cells_collect(const Grid& g, const int* __restrict__ cell_start,
                                             const float4* __restrict__ pos, float xi, float yi, float zi, int cell,
                                             float R2, bool live, unsigned* __restrict__ lst, float* r2s, int cnt,
                                             bool& ovf, unsigned& ncand) {
  if (!live) return cnt;
  const int nx = g.nc[0], ny = g.nc[1];
  const int cx = cell % nx, cy = (cell / nx) % ny, cz = cell / (nx * ny);
#pragma unroll 1
  for (int q = 0; q < 27; ++q) {
    const NbrCell nbc = nbr_cell(g, cx, cy, cz, q);
    const int cs = cell_start[nbc.c], ce = cell_start[nbc.c + 1];
    const float xs = xi - nbc.sx, ys = yi - nbc.sy, zs = zi - nbc.sz;
    const unsigned eb = nbc.code << kIndexBits;
    for (int j = cs; j < ce; ++j) {
      const float4 c = pos[j];
      const float r2 = r2_of(xs - c.x, ys - c.y, zs - c.z);
      if (r2 < R2) {
        if (cnt < W) {
          lst[cnt * 32] = (unsigned)j | eb;
          r2s[cnt * 32] = r2;
        } else {
          ovf = true;
        }
        ++cnt;
      }
    }
    ncand += (unsigned)(ce - cs);
  }
  return cnt;
}

// Shared rows (the uniform grid's lane-per-particle collect). The lanes of a
// group whose particles lie in one row of cells (same y and z cell index),
// within kRowSpan cells of each other in x, form a run. The union of their
// 27-cell neighbourhoods is 9 rows of consecutive cells: x from the run's
// smallest x - 1 to its largest x + 1, at y - 1..y + 1 and z - 1..z + 1, each
// row a contiguous range of the sorted particles (cell ids run x fastest).
// x - 1 below 0 and x + 1 past the last cell are the periodic images (shift
// codes as shift_j reads them), so a row has up to three segments and every
// (cell, image) pair of a lane's neighbourhood is read exactly once, in the
// order cells_collect reads it: z, then y, then x ascending.
//
// Every lane of the run tests every candidate of those segments, in step.
// The segments' records are staged in shared memory in chunks of up to 32
// (one 16-byte cp.async a lane), kRowDepth - 1 chunks ahead of the chunk
// being tested, so the tests read broadcast shared-memory values instead of
// waiting on a load from L2 per batch. A chunk holds records of one segment
// only, so the lane's shifted position is set once a chunk.
//
// A lane's list is therefore the one cells_collect writes, except that
// candidates of cells two or more cells away in x that pass the FP32 test
// are kept as well (the test's guard band admits a thin shell beyond a cell
// width); they lie outside every support, which the exact decisions of the
// later sums reject. At most kRowRuns runs are taken; lanes left over
// (groups spread over many rows, as an active subset gives) go to
// cells_collect. Dead lanes (live = false) take no part.
constexpr int kRowSpan = 6;   // largest x extent of a run, in cells
constexpr int kRowRuns = 2;   // shared runs a group takes before the per-lane fallback
constexpr int kRowDepth = 3;  // staged chunks of a warp (kRowDepth - 1 in flight while one is tested)

// A warp's staging area: the chunk ring and the run's segments (at most 27).
struct RowStage {
  float4 ring[kRowDepth][32];
  int seg_start[32];
  int seg_end[32];
  unsigned seg_code[32];
  int chunk_pref[33];  // chunks of the run before segment q
  int pad[3];
};
static_assert(sizeof(RowStage) % 16 == 0, "the next warp's ring starts 16-byte aligned");

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// every group of this thread but the kRowDepth - 1 newest has landed
__device__ __forceinline__ void cp_async_wait_older() {
  asm volatile("cp.async.wait_group %0;" ::"n"(kRowDepth - 1) : "memory");
}

// Segment of chunk c (binary search over the chunk prefix; nseg >= 1).
__device__ __forceinline__ int row_chunk_seg(const RowStage& rs, int nseg, int c) {
  int q = 0;
#pragma unroll
  for (int step = 16; step > 0; step >>= 1)
    if (q + step < nseg && rs.chunk_pref[q + step] <= c) q += step;
  return q;
}

// Chunk c (< nch) into ring slot c % kRowDepth: lane l copies record l of
// the chunk, if the chunk has one. Every lane commits one group a call, so
// the groups of all lanes count alike.
__device__ __forceinline__ void row_stage(const float4* __restrict__ pos, RowStage& rs, int nseg, int nch, int c) {
  if (c < nch) {
    const int q = row_chunk_seg(rs, nseg, c);
    const int j = rs.seg_start[q] + (c - rs.chunk_pref[q]) * 32 + (int)lane_id();
    if (j < rs.seg_end[q]) cp_async16(&rs.ring[c % kRowDepth][lane_id()], pos + j);
  }
  cp_async_commit();
}

template <int W>
__device__ __forceinline__ int rows_collect(const Grid& g, const int* __restrict__ cell_start,
                                            const float4* __restrict__ pos, float xi, float yi, float zi, int cell,
                                            float R2, bool live, unsigned* __restrict__ lst, float* r2s,
                                            RowStage& rs, bool& ovf, unsigned& ncand) {
  const unsigned lane = lane_id();
  const int nx = g.nc[0], ny = g.nc[1], nz = g.nc[2];
  const int cx = cell % nx, rw = cell / nx;  // rw = cy + ny cz
  int cnt = 0;
  unsigned pending = __ballot_sync(0xffffffffu, live);
#pragma unroll 1
  for (int run = 0; run < kRowRuns && pending != 0u; ++run) {
    const int lead = __ffs(pending) - 1;
    const int rrow = __shfl_sync(0xffffffffu, rw, lead);
    const bool same = ((pending >> lane) & 1u) && rw == rrow;
    const int x0 = __reduce_min_sync(0xffffffffu, same ? cx : 0x7fffffff);
    const bool in = same && cx <= x0 + kRowSpan;
    const int x1 = __reduce_max_sync(0xffffffffu, in ? cx : -1);
    pending &= ~__ballot_sync(0xffffffffu, in);
    const float R2in = in ? R2 : -1.0f;
    // segment of lane l < 27: row l / 3 (y fastest, then z), part l % 3 (the
    // image at x = -1, the cells inside the box, the image at x = nx)
    int len = 0;
    if (lane < 27u) {
      const int ry = rrow % ny, rz = rrow / ny;
      const int rq = (int)lane / 3, part = (int)lane % 3;
      int y = ry + rq % 3 - 1, z = rz + rq / 3 - 1;
      unsigned code = 0;
      if (y < 0) { y += ny; code |= 8u; } else if (y >= ny) { y -= ny; code |= 4u; }
      if (z < 0) { z += nz; code |= 32u; } else if (z >= nz) { z -= nz; code |= 16u; }
      const int base = nx * (y + ny * z);
      int xa = 0, xb = -1;
      if (part == 0) {
        if (x0 == 0) { xa = xb = nx - 1; code |= 2u; }
      } else if (part == 1) {
        xa = max(x0 - 1, 0);
        xb = min(x1 + 1, nx - 1);
      } else {
        if (x1 == nx - 1) { xa = xb = 0; code |= 1u; }
      }
      int js = 0, je = 0;
      if (xb >= xa) {
        js = cell_start[base + xa];
        je = cell_start[base + xb + 1];
      }
      rs.seg_start[lane] = js;
      rs.seg_end[lane] = je;
      rs.seg_code[lane] = code;
      len = je - js;
    }
    int incl = (len + 31) >> 5;  // chunks of the segment
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if ((int)lane >= o) incl += y;
    }
    if (lane < 27u) rs.chunk_pref[lane + 1] = incl;
    if (lane == 0) rs.chunk_pref[0] = 0;
    const int nch = __shfl_sync(0xffffffffu, incl, 26);
    const unsigned tested = (unsigned)__reduce_add_sync(0xffffffffu, (unsigned)len);
    __syncwarp();
#pragma unroll
    for (int c = 0; c < kRowDepth - 1; ++c) row_stage(pos, rs, 27, nch, c);
#pragma unroll 1
    for (int c = 0; c < nch; ++c) {
      row_stage(pos, rs, 27, nch, c + kRowDepth - 1);
      cp_async_wait_older();
      __syncwarp();  // every lane's copies of chunk c have landed
      const int q = row_chunk_seg(rs, 27, c);
      const int j0 = rs.seg_start[q] + (c - rs.chunk_pref[q]) * 32;
      const int m = min(32, rs.seg_end[q] - j0);
      const unsigned code = rs.seg_code[q];
      // the lane's position less the segment's image shift S (as cells_collect takes it)
      const float xs = xi - ((code & 1u) ? g.L[0] : (code & 2u) ? -g.L[0] : 0.0f);
      const float ys = yi - ((code & 4u) ? g.L[1] : (code & 8u) ? -g.L[1] : 0.0f);
      const float zs = zi - ((code & 16u) ? g.L[2] : (code & 32u) ? -g.L[2] : 0.0f);
      const unsigned e0 = (unsigned)j0 | (code << kIndexBits);  // entry of the chunk's first record
      const float4* ch = rs.ring[c % kRowDepth];
      if (__all_sync(0xffffffffu, cnt + m <= W)) {
        // no list can fill in this chunk. Eight tests at a time: the hit mask
        // first (lanes outside the run test against -1: no hits), then each
        // hit's place from a popcount of the hits before it, so that the
        // stores do not wait on one another. Slots past m hold stale records
        // and are masked out.
        for (int b0 = 0; b0 < m; b0 += 8) {
          float r2v[8];
          unsigned hm = 0;
#pragma unroll
          for (int b = 0; b < 8; ++b) {
            const float4 cj = ch[b0 + b];
            r2v[b] = r2_of(xs - cj.x, ys - cj.y, zs - cj.z);
            hm |= (r2v[b] < R2in && b0 + b < m) ? (1u << b) : 0u;
          }
          unsigned* lp = lst + cnt * 32;
          float* rp = r2s + cnt * 32;
#pragma unroll
          for (int b = 0; b < 8; ++b) {
            if (hm & (1u << b)) {
              const int at = __popc(hm & ((1u << b) - 1u)) * 32;
              lp[at] = e0 + (unsigned)(b0 + b);
              rp[at] = r2v[b];
            }
          }
          cnt += __popc(hm);
        }
      } else {
        for (int b = 0; b < m; ++b) {
          const float4 cj = ch[b];
          const float r2 = r2_of(xs - cj.x, ys - cj.y, zs - cj.z);
          if (r2 < R2in) {
            if (cnt < W) {
              lst[cnt * 32] = e0 + (unsigned)b;
              r2s[cnt * 32] = r2;
            } else {
              ovf = true;
            }
            ++cnt;
          }
        }
      }
      __syncwarp();  // chunk c's slot is restaged by the next iteration
    }
    if (in) ncand += tested;
  }
  const bool rest = (pending >> lane) & 1u;
  if (__any_sync(0xffffffffu, rest))
    cnt = cells_collect<W>(g, cell_start, pos, xi, yi, zi, cell, R2, rest, lst, r2s, cnt, ovf, ncand);
  return cnt;
}

// Per-lane scan of the 27 cells around `cell` without windows or lists: every
// particle of every neighbour cell is handed to op.interact (which takes the
// exact neighbour decision itself). The fallback of a group that has no kept
// list. Lanes with live = false take no part.
template <class Op>
__device__ __forceinline__ void lpp_scan(const Op& op, typename Op::I& I, const Grid& g,
                                         const int* __restrict__ cell_start, int cell, bool live, unsigned& ncand) {
  const int nx = g.nc[0], ny = g.nc[1];
  const int cx = cell % nx, cy = (cell / nx) % ny, cz = cell / (nx * ny);
#pragma unroll 1
  for (int q = 0; q < 27; ++q) {
    const NbrCell nbc = nbr_cell(g, cx, cy, cz, q);
    const int cs = cell_start[nbc.c], ce = cell_start[nbc.c + 1];
    if (live)
      for (int j = cs; j < ce; ++j) op.interact(I, j, nbc.code);
    if (live) ncand += (unsigned)(ce - cs);
  }
}

}  // namespace sg
