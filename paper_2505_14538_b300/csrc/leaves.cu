// leaves.cu -- adaptive leaves for clustered particle sets: the cell tree
// of Sec. 2.2.2 (Fig. 3c), which the paper's GPU path lacks (Sec. 4.4.4),
// built on the device after the cell sort has left every cell in Morton
// order:
//
//   k_tree_gather  sorted positions and Morton codes
//   k_tree_level   one launch per level (cells are level 0, at most
//                  kTreeLevels below): one warp per node reduces its
//                  particles' bounding box and largest h; a node with more
//                  than leaf_max particles is split into its non-empty
//                  octants (binary search of the level's Morton digit inside
//                  the node's range), any other node is a leaf
//   k_leaf_walk    one warp per leaf walks the trees of the 27 neighbour
//                  cells (periodic images included) with a shared-memory
//                  stack, descends into nodes whose bounding box comes within
//                  the larger reach (kernel_gamma * h_cap) of the two sides,
//                  and counts (pass 0) or writes (pass 1) its neighbour leaves
//
// Every pair that any loop may need is covered: a pair (i, j) is a candidate
// only when its FP32 r^2 is below max(H_i, H_j)^2 plus the guard band, and
// the bounding-box gap of the two leaves, evaluated with the same rounded
// operations on the same shifted coordinates, is no larger than r_ij, while
// H_i, H_j never exceed their leaves' reach.
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"

namespace sg {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kTreeThreads = 256;
constexpr int kWalkThreads = 128;
constexpr int kWalkWarps = kWalkThreads / 32;
// Walk stack per warp: 27 roots plus at most 32 * 8 children pushed per step
// for each of the kTreeLevels + 1 depths that can lie on the stack at once.
constexpr int kStack = 3072;
static_assert(27 + (kTreeLevels + 1) * 256 <= kStack, "walk stack too small");

__global__ void k_tree_gather(const float4* __restrict__ pos_h, const unsigned* __restrict__ perm,
                              const unsigned* __restrict__ morton, int n, float4* __restrict__ pos,
                              unsigned* __restrict__ mk) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const unsigned src = perm[k];
    pos[k] = pos_h[src];
    mk[k] = morton[src];
  }
}

struct TreeArgs {
  const Grid* grid;
  const float4* pos;       // sorted (x, y, z, h)
  const unsigned* mk;      // sorted Morton codes inside the cell
  const int* cell_start;
  int2* node_range;
  int2* node_kids;
  float4* node_lo;
  float4* node_hi;
  int* node_leaf;
  int2* leaf_range;
  float* leaf_hcap;
  int* leaf_node;
  int* tctr;
  int node_cap;
  int leaf_max;
  float margin;
  float kg;
};

__global__ void __launch_bounds__(kTreeThreads) k_tree_level(TreeArgs a, int level) {
  const unsigned lane = lane_id();
  const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const Grid& g = *a.grid;
  const float hcap_cell = g.hcap;
  int begin = 0;
  for (int m = 0; m < level; ++m) begin += m == 0 ? g.ncells : a.tctr[kTreeNodes + m];
  int size = level == 0 ? g.ncells : a.tctr[kTreeNodes + level];
  size = min(size, a.node_cap - begin);  // nodes past the capacity were never created
  const int next_begin = begin + size;
  const float inf = __int_as_float(0x7f800000);
  for (int i = gwarp; i < size; i += nwarps) {
    const int v = begin + i;
    int s, e;
    if (level == 0) {
      s = a.cell_start[v];
      e = a.cell_start[v + 1];
      if (lane == 0) a.node_range[v] = make_int2(s, e);
    } else {
      const int2 r = a.node_range[v];
      s = r.x;
      e = r.y;
    }
    if (e == s) {  // empty cell (children are never empty)
      if (lane == 0) {
        a.node_lo[v] = make_float4(inf, inf, inf, 0.0f);
        a.node_hi[v] = make_float4(-inf, -inf, -inf, 0.0f);
        a.node_kids[v] = make_int2(0, 0);
        a.node_leaf[v] = -1;
      }
      continue;
    }
    float lx = inf, ly = inf, lz = inf, hx = -inf, hy = -inf, hz = -inf, hm = 0.0f;
    for (int k = s + (int)lane; k < e; k += 32) {
      const float4 p = a.pos[k];
      lx = fminf(lx, p.x); ly = fminf(ly, p.y); lz = fminf(lz, p.z);
      hx = fmaxf(hx, p.x); hy = fmaxf(hy, p.y); hz = fmaxf(hz, p.z);
      hm = fmaxf(hm, p.w);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lx = fminf(lx, __shfl_xor_sync(kFull, lx, o));
      ly = fminf(ly, __shfl_xor_sync(kFull, ly, o));
      lz = fminf(lz, __shfl_xor_sync(kFull, lz, o));
      hx = fmaxf(hx, __shfl_xor_sync(kFull, hx, o));
      hy = fmaxf(hy, __shfl_xor_sync(kFull, hy, o));
      hz = fmaxf(hz, __shfl_xor_sync(kFull, hz, o));
      hm = fmaxf(hm, __shfl_xor_sync(kFull, hm, o));
    }
    const float hcap = fminf(hcap_cell, (1.0f + a.margin) * hm);
    const float reach = a.kg * hcap;
    bool split = (e - s) > a.leaf_max && level < kTreeLevels;
    int cbase = 0, nch = 0;
    if (split) {
      // octant o of this node: the particles whose Morton digit of this level is o
      const int sh = 3 * (kTreeLevels - 1 - level);
      int lb = e;
      if (lane < 8) {
        int lo = s, hi = e;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if ((int)((a.mk[mid] >> sh) & 7u) < (int)lane) lo = mid + 1;
          else hi = mid;
        }
        lb = lo;
      }
      const int nxt = __shfl_down_sync(kFull, lb, 1);  // lane o: start of octant o + 1 (lane 7: e)
      const bool nonempty = lane < 8 && nxt > lb;
      const unsigned m = __ballot_sync(kFull, nonempty);
      nch = __popc(m);
      if (lane == 0) cbase = atomicAdd(&a.tctr[kTreeNodes + level + 1], nch);
      cbase = __shfl_sync(kFull, cbase, 0) + next_begin;
      if (cbase + nch > a.node_cap) {
        // out of node capacity: this node stays a leaf; the slots it took
        // inside the capacity become empty nodes
        split = false;
        for (int t = (int)lane; t < nch; t += 32)
          if (cbase + t < a.node_cap) a.node_range[cbase + t] = make_int2(s, s);
      } else if (nonempty) {
        a.node_range[cbase + __popc(m & ((1u << lane) - 1u))] = make_int2(lb, nxt);
      }
    }
    if (lane == 0) {
      a.node_lo[v] = make_float4(lx, ly, lz, reach);
      a.node_hi[v] = make_float4(hx, hy, hz, hcap);
      if (split) {
        a.node_kids[v] = make_int2(cbase, nch);
        a.node_leaf[v] = -1;
      } else {
        const int li = atomicAdd(&a.tctr[kTreeLeaves], 1);  // leaves are disjoint and non-empty: li < n
        a.leaf_range[li] = make_int2(s, e);
        a.leaf_hcap[li] = hcap;
        a.leaf_node[li] = v;
        a.node_kids[v] = make_int2(0, 0);
        a.node_leaf[v] = li;
        atomicMax(&a.tctr[kTreeDepth], level);
      }
    }
  }
}

struct WalkArgs {
  const Grid* grid;
  const unsigned* skeys;   // sorted cell ids
  const int2* node_kids;
  const float4* node_lo;
  const float4* node_hi;
  const int* node_leaf;
  const int2* leaf_range;
  const int* leaf_node;
  const int* tctr;
  int* nbr_off;            // pass 0: counts out; pass 1: offsets in
  unsigned* nbr;
  int nbr_cap;
  Status* st;
};

__global__ void __launch_bounds__(kWalkThreads) k_leaf_walk(WalkArgs a, int fill) {
  __shared__ unsigned stack_all[kWalkWarps][kStack];
  unsigned* st = stack_all[threadIdx.x >> 5];
  const unsigned lane = lane_id();
  const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const Grid& g = *a.grid;
  const float L[3] = {g.L[0], g.L[1], g.L[2]};
  const float Lmax = fmaxf(L[0], fmaxf(L[1], L[2]));
  const int nx = g.nc[0], ny = g.nc[1], nz = g.nc[2];
  const int nleaves = a.tctr[kTreeLeaves];
  for (int li = gwarp; li < nleaves; li += nwarps) {
    const int va = a.leaf_node[li];
    const float4 la = a.node_lo[va], ha = a.node_hi[va];
    const int cell = (int)a.skeys[a.leaf_range[li].x];
    __syncwarp();
    if (lane < 27) {
      const int cx = cell % nx, cy = (cell / nx) % ny, cz = cell / (nx * ny);
      int x = cx + (int)(lane % 3u) - 1, y = cy + (int)((lane / 3u) % 3u) - 1, z = cz + (int)(lane / 9u) - 1;
      unsigned code = 0;
      if (x < 0) { x += nx; code |= 2u; } else if (x >= nx) { x -= nx; code |= 1u; }
      if (y < 0) { y += ny; code |= 8u; } else if (y >= ny) { y -= ny; code |= 4u; }
      if (z < 0) { z += nz; code |= 32u; } else if (z >= nz) { z -= nz; code |= 16u; }
      st[lane] = (unsigned)(x + nx * (y + ny * z)) | (code << kIndexBits);
    }
    int sp = 27;
    int count = 0;
    const int off = fill ? a.nbr_off[li] : 0;
    bool overflow = false;
    __syncwarp();
    while (sp > 0) {
      const int take = min(32, sp);
      unsigned e = 0;
      if ((int)lane < take) e = st[sp - take + (int)lane];
      sp -= take;
      __syncwarp();
      bool pass = false;
      int2 kids = make_int2(0, 0);
      int leaf = -1;
      const unsigned code = e >> kIndexBits;
      if ((int)lane < take) {
        const int b = (int)(e & kIndexMask);
        float4 lb = a.node_lo[b], hb = a.node_hi[b];
        shift_j(code, L, lb.x, lb.y, lb.z);
        shift_j(code, L, hb.x, hb.y, hb.z);
        const float gx = fmaxf(fmaxf(lb.x - ha.x, la.x - hb.x), 0.0f);
        const float gy = fmaxf(fmaxf(lb.y - ha.y, la.y - hb.y), 0.0f);
        const float gz = fmaxf(fmaxf(lb.z - ha.z, la.z - hb.z), 0.0f);
        const float R = fmaxf(la.w, lb.w);
        // the particle test is r2 < H^2 + band(H) with H <= R; 2^-12 extra slack
        pass = r2_of(gx, gy, gz) < (R * R + band_of(R, Lmax)) * 1.000244140625f;
        if (pass) {
          kids = a.node_kids[b];
          leaf = a.node_leaf[b];
        }
      }
      const bool is_leaf = pass && leaf >= 0;
      const unsigned lm = __ballot_sync(kFull, is_leaf);
      if (fill && is_leaf) {
        const int t = off + count + __popc(lm & ((1u << lane) - 1u));
        if (t < a.nbr_cap) a.nbr[t] = (unsigned)leaf | (code << kIndexBits);  // a list past the cap is unused
      }
      count += __popc(lm);
      int nk = (pass && leaf < 0) ? kids.y : 0;
      int incl = nk;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, incl, o);
        if ((int)lane >= o) incl += y;
      }
      const int tot = __shfl_sync(kFull, incl, 31);
      if (sp + tot > kStack) {
        overflow = true;  // cannot happen for trees of kTreeLevels levels; guards the stack
      } else {
        for (int t = 0; t < nk; ++t)
          st[sp + incl - nk + t] = (unsigned)(kids.x + t) | (code << kIndexBits);
        sp += tot;
      }
      __syncwarp();
    }
    if (lane == 0) {
      if (overflow) set_error(a.st, SWIFT_GPU_ERR_CAPACITY);
      if (!fill) a.nbr_off[li] = count;
    }
  }
}

// Total list length (lists past the capacity are replaced by cell scans).
__global__ void k_tree_finish(int* tctr, const int* nbr_off) { tctr[kTreeEntries] = nbr_off[tctr[kTreeLeaves]]; }

int leaves_build(Ctx* c, const float4* pos_h, cudaStream_t s) {
  const int n = c->n;
  cudaMemsetAsync(c->d_tree_ctr, 0, sizeof(int) * kTreeCtrCount, s);
  cudaMemsetAsync(c->d_nbr_off, 0, sizeof(int) * (size_t)(n + 1), s);
  if (n == 0) return cudaGetLastError() == cudaSuccess ? SWIFT_GPU_OK : SWIFT_GPU_ERR_CUDA;
  const int sm = c->num_sms;
  const unsigned* perm = c->d_vals[c->sorted_buf];
  unsigned* mk = c->d_keys[1 - c->sorted_buf];  // free after the sort
  k_tree_gather<<<min((n + 255) / 256, sm * 8), 256, 0, s>>>(pos_h, perm, c->d_aux[1], n, c->d_pos, mk);
  c->launches++;
  TreeArgs t;
  t.grid = c->d_grid;
  t.pos = c->d_pos;
  t.mk = mk;
  t.cell_start = c->d_cell_start;
  t.node_range = c->d_node_range;
  t.node_kids = c->d_node_kids;
  t.node_lo = c->d_node_lo;
  t.node_hi = c->d_node_hi;
  t.node_leaf = c->d_node_leaf;
  t.leaf_range = c->d_leaf_range;
  t.leaf_hcap = c->d_leaf_hcap;
  t.leaf_node = c->d_leaf_node;
  t.tctr = c->d_tree_ctr;
  t.node_cap = c->node_cap;
  t.leaf_max = c->params.leaf_max;
  t.margin = c->params.leaf_margin;
  t.kg = c->phys.kg;
  const int tree_blocks = sm * 4;
  for (int level = 0; level <= kTreeLevels; ++level) {
    k_tree_level<<<tree_blocks, kTreeThreads, 0, s>>>(t, level);
    c->launches++;
  }
  WalkArgs w;
  w.grid = c->d_grid;
  w.skeys = c->d_keys[c->sorted_buf];
  w.node_kids = c->d_node_kids;
  w.node_lo = c->d_node_lo;
  w.node_hi = c->d_node_hi;
  w.node_leaf = c->d_node_leaf;
  w.leaf_range = c->d_leaf_range;
  w.leaf_node = c->d_leaf_node;
  w.tctr = c->d_tree_ctr;
  w.nbr_off = c->d_nbr_off;
  w.nbr = c->d_nbr;
  w.nbr_cap = c->nbr_cap;
  w.st = c->d_status;
  const int walk_blocks = sm * 8;
  k_leaf_walk<<<walk_blocks, kWalkThreads, 0, s>>>(w, 0);
  exclusive_scan(c, reinterpret_cast<const unsigned*>(c->d_nbr_off), reinterpret_cast<unsigned*>(c->d_nbr_off),
                 n + 1, c->d_scan_tmp, s);
  k_leaf_walk<<<walk_blocks, kWalkThreads, 0, s>>>(w, 1);
  k_tree_finish<<<1, 1, 0, s>>>(c->d_tree_ctr, c->d_nbr_off);
  c->launches += 3;
  return cudaGetLastError() == cudaSuccess ? SWIFT_GPU_OK : SWIFT_GPU_ERR_CUDA;
}

Nbr nbr_of(Ctx* c) {
  Nbr b;
  b.cell_start = c->d_cell_start;
  b.skeys = c->d_keys[c->sorted_buf];
  b.leaf_range = c->d_leaf_range;
  b.nbr_off = c->d_nbr_off;
  b.nbr = c->d_nbr;
  b.leaf_hcap = c->d_leaf_hcap;
  b.n_leaves = c->d_tree_ctr ? c->d_tree_ctr + kTreeLeaves : nullptr;
  b.nbr_cap = c->nbr_cap;
  b.adaptive = c->tree_built;
  return b;
}

__global__ void k_leaves_export(const int2* __restrict__ range, const float* __restrict__ hcap,
                                const int* __restrict__ off, const int* __restrict__ tctr, int64_t max_leaves,
                                int32_t* __restrict__ out_range, float* __restrict__ out_hcap,
                                int32_t* __restrict__ out_cnt) {
  const int nl = tctr[kTreeLeaves];
  const int m = (int)min((int64_t)nl, max_leaves);
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < m; l += gridDim.x * blockDim.x) {
    const int2 r = range[l];
    if (out_range) {
      out_range[2 * l] = r.x;
      out_range[2 * l + 1] = r.y;
    }
    if (out_hcap) out_hcap[l] = hcap[l];
    if (out_cnt) out_cnt[l] = off[l + 1] - off[l];
  }
}

int leaves_export_impl(Ctx* c, int32_t* range, float* hcap, int32_t* nbr_count, int64_t max_leaves, cudaStream_t s) {
  if (max_leaves <= 0 || c->n == 0) return SWIFT_GPU_OK;
  const int64_t m = max_leaves < c->n ? max_leaves : c->n;
  const int nb = (int)((m + 255) / 256 < c->num_sms * 8 ? (m + 255) / 256 : c->num_sms * 8);
  k_leaves_export<<<nb, 256, 0, s>>>(c->d_leaf_range, c->d_leaf_hcap, c->d_nbr_off, c->d_tree_ctr, max_leaves, range,
                                     hcap, nbr_count);
  c->launches++;
  return cudaGetLastError() == cudaSuccess ? SWIFT_GPU_OK : SWIFT_GPU_ERR_CUDA;
}

}  // namespace sg
