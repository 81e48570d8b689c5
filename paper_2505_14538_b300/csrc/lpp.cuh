// lpp.cuh -- the lane-per-particle neighbour search of the uniform grid.
//
// A warp takes 32 consecutive active particles (a "group", several cells
// wide) and each lane works on its own particle from start to end: no lanes
// share a particle, none is idle while the group is full, and no sub-lane
// sums are combined.
//
// Candidates come from the 27 cells around the lane's own cell (Sec. 2.2:
// self and pair interactions of cells no narrower than the support). For a
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
