// leaves.cu -- adaptive leaves for clustered particle sets: the cell tree
// of Sec. 2.2.2 (Fig. 3c), which the paper's GPU path lacks (Sec. 4.4.4),
// built on the device after the cell sort has left every cell in Morton
// order:
//
//   k_tree_gather  sorted positions and Morton codes
//   k_tree_split   one launch per level (cells are level 0, at most
//                  kTreeLevels below): a node with more than leaf_max
//                  particles is split into its non-empty octants (binary
//                  search of the level's Morton digit inside the node's
//                  range), any other node is a leaf
//   k_leaf_number  leaf indices from a scan of the leaf flags
//   k_leaf_finish  8 lanes per leaf reduce its particles' bounding box and
//                  largest h; the boxes and reaches of the inner nodes follow
//                  bottom-up (the last child to finish completes its parent)
//   k_leaf_walk    one warp per parent of leaves walks the trees of the 27
//                  neighbour cells (periodic images included) with a
//                  shared-memory stack, descends into nodes whose bounding box
//                  comes within the larger reach (kernel_gamma * h_cap) of the
//                  two sides, and filters that list for each of its leaves,
//                  which get their neighbour leaves as one contiguous list
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
// Walk stack per warp. A step pops P entries (one per lane) and pushes at
// most 8 children for each. With g = kStack - (entries on the stack): while
// g >= kDfsGap, P = min(32, (g - 80) / 7), so at least 80 entries stay free;
// below that P = 1, a depth-first walk, which adds at most 7 entries for
// each of the kTreeLevels levels (70 < 80) before it unwinds. The stack thus
// never overflows; the overflow guard below only backs that bound up.
constexpr int kStack = 1024;
constexpr int kDfsGap = 87;
static_assert(kStack >= 27 + kDfsGap, "walk stack too small for its roots");

__global__ void k_tree_gather(const float4* __restrict__ pos_h, const unsigned* __restrict__ perm,
                              const unsigned* __restrict__ morton, int n, const Grid* __restrict__ g,
                              float4* __restrict__ pos, unsigned* __restrict__ mk) {
  pdl_wait();
  const float L[3] = {g->L[0], g->L[1], g->L[2]};
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const unsigned src = perm[k];
    pos[k] = wrap_pos(pos_h[src], L);
    mk[k] = morton[src];
  }
}

struct TreeArgs {
  const Grid* grid;
  const float4* pos;       // sorted (x, y, z, h)
  const unsigned* mk;      // sorted Morton codes inside the cell
  const int* cell_start;
  int2* node_range;
  float4* node;            // 2 per node: (low corner, reach), (high corner, link)
  int* node_link;
  int* node_parent;
  int* node_done;
  unsigned* node_flag;     // 1 for a leaf (then its exclusive scan: the leaf index)
  int2* leaf_range;
  float* leaf_hcap;
  int* leaf_node;
  int* tctr;
  int node_cap;
  int leaf_max;
  float margin;
  float kg;
};

// Link word of a node (the w of its second float4, as int bits): child
// count << 27 | first child for an inner node, the leaf index for a leaf
// (child count 0); kEmptyLink for an empty cell.
constexpr int kLinkShift = 27;
constexpr int kLinkMask = (1 << kLinkShift) - 1;
constexpr int kEmptyLink = 0x7fffffff;
constexpr int kLeafMark = -1;
static_assert(kIndexBits <= kLinkShift, "node and leaf indices must fit the link word");

// Top-down, one launch per level: split decisions from the particle counts
// alone (no particle is read but the Morton codes of the binary searches).
__global__ void __launch_bounds__(kTreeThreads) k_tree_split(TreeArgs a, int level) {
  pdl_wait();
  const unsigned lane = lane_id();
  const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const Grid& g = *a.grid;
  int begin = 0;
  for (int m = 0; m < level; ++m) begin += m == 0 ? g.ncells : a.tctr[kTreeNodes + m];
  int size = level == 0 ? g.ncells : a.tctr[kTreeNodes + level];
  size = min(size, a.node_cap - begin);  // nodes past the capacity were never created
  const int next_begin = begin + size;
  const float inf = __int_as_float(0x7f800000);
  bool made_leaf = false;
  for (int i = gwarp; i < size; i += nwarps) {
    const int v = begin + i;
    int s, e;
    if (level == 0) {
      s = a.cell_start[v];
      e = a.cell_start[v + 1];
      if (lane == 0) {
        a.node_range[v] = make_int2(s, e);
        a.node_parent[v] = -1;
      }
    } else {
      const int2 r = a.node_range[v];
      s = r.x;
      e = r.y;
    }
    if (e == s) {  // empty cell, or a slot left by a node that ran out of capacity
      if (lane == 0) {
        a.node[2 * v] = make_float4(inf, inf, inf, 0.0f);
        a.node[2 * v + 1] = make_float4(-inf, -inf, -inf, __int_as_float(kEmptyLink));
        a.node_link[v] = kEmptyLink;
      }
      continue;
    }
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
        const int c = cbase + __popc(m & ((1u << lane) - 1u));
        a.node_range[c] = make_int2(lb, nxt);
        a.node_parent[c] = v;
      }
    }
    if (lane == 0) {
      a.node_link[v] = split ? ((nch << kLinkShift) | cbase) : kLeafMark;
      a.node_flag[v] = split ? 0u : 1u;
    }
    made_leaf |= !split;
  }
  if (lane == 0 && made_leaf && *((volatile int*)&a.tctr[kTreeDepth]) < level) atomicMax(&a.tctr[kTreeDepth], level);
}

// Leaf index of every leaf node from the exclusive scan of the leaf flags.
__global__ void k_leaf_number(const unsigned* __restrict__ scan, int node_cap, int* __restrict__ node_link,
                              int* __restrict__ leaf_node, int* __restrict__ tctr) {
  pdl_wait();
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < node_cap; v += gridDim.x * blockDim.x) {
    const unsigned li = scan[v];
    if (scan[v + 1] != li) {
      leaf_node[li] = v;
      node_link[v] = (int)li;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) tctr[kTreeLeaves] = (int)scan[node_cap];
}

// A group of 8 lanes per leaf (leaves hold about leaf_max / 4 particles on
// average, so a warp works on four at once): bounding box and largest h of
// its particles; then up the tree, the last child to finish writes its
// parent's box (the union of the children's, at most 8) and reach (the
// largest of theirs), and carries on. The groups of a warp run their loops
// independently; every shuffle names only its group's lanes.
constexpr int kFinishLanes = 8;
__global__ void __launch_bounds__(kTreeThreads) k_leaf_finish(TreeArgs a) {
  pdl_wait();
  const unsigned lane = lane_id();
  const unsigned gl = lane & (kFinishLanes - 1);
  const unsigned gmask = 0xffu << (lane & ~(unsigned)(kFinishLanes - 1));
  const int group = (int)((blockIdx.x * blockDim.x + threadIdx.x) / kFinishLanes);
  const int ngroups = (int)((gridDim.x * blockDim.x) / kFinishLanes);
  const float hcap_cell = a.grid->hcap;
  const float inf = __int_as_float(0x7f800000);
  const int nleaves = a.tctr[kTreeLeaves];
  for (int li = group; li < nleaves; li += ngroups) {
    int v = a.leaf_node[li];
    const int2 r = a.node_range[v];
    float lx = inf, ly = inf, lz = inf, hx = -inf, hy = -inf, hz = -inf, hm = 0.0f;
    for (int k = r.x + (int)gl; k < r.y; k += kFinishLanes) {
      const float4 p = a.pos[k];
      lx = fminf(lx, p.x); ly = fminf(ly, p.y); lz = fminf(lz, p.z);
      hx = fmaxf(hx, p.x); hy = fmaxf(hy, p.y); hz = fmaxf(hz, p.z);
      hm = fmaxf(hm, p.w);
    }
#pragma unroll
    for (int o = kFinishLanes / 2; o > 0; o >>= 1) {
      lx = fminf(lx, __shfl_xor_sync(gmask, lx, o, kFinishLanes));
      ly = fminf(ly, __shfl_xor_sync(gmask, ly, o, kFinishLanes));
      lz = fminf(lz, __shfl_xor_sync(gmask, lz, o, kFinishLanes));
      hx = fmaxf(hx, __shfl_xor_sync(gmask, hx, o, kFinishLanes));
      hy = fmaxf(hy, __shfl_xor_sync(gmask, hy, o, kFinishLanes));
      hz = fmaxf(hz, __shfl_xor_sync(gmask, hz, o, kFinishLanes));
      hm = fmaxf(hm, __shfl_xor_sync(gmask, hm, o, kFinishLanes));
    }
    const float hcap = fminf(hcap_cell, (1.0f + a.margin) * hm);
    if (gl == 0) {
      a.leaf_range[li] = r;
      a.leaf_hcap[li] = hcap;
      a.node[2 * v] = make_float4(lx, ly, lz, a.kg * hcap);
      a.node[2 * v + 1] = make_float4(hx, hy, hz, __int_as_float(li));
    }
    for (;;) {
      int p = -1, done = 0, link = 0;
      if (gl == 0) {
        p = a.node_parent[v];
        if (p >= 0) {
          __threadfence();  // this node's record before the count
          done = atomicAdd(&a.node_done[p], 1);
          link = a.node_link[p];
        }
      }
      p = __shfl_sync(gmask, p, 0, kFinishLanes);
      done = __shfl_sync(gmask, done, 0, kFinishLanes);
      link = __shfl_sync(gmask, link, 0, kFinishLanes);
      const int nch = link >> kLinkShift;
      if (p < 0 || done != nch - 1) break;  // a sibling is still running: it finishes the parent
      __threadfence();
      const int first = link & kLinkMask;
      float4 cl = make_float4(inf, inf, inf, 0.0f), ch = make_float4(-inf, -inf, -inf, 0.0f);
      if ((int)gl < nch) {
        cl = __ldcg(&a.node[2 * (first + (int)gl)]);  // from L2: written by other warps
        ch = __ldcg(&a.node[2 * (first + (int)gl) + 1]);
      }
#pragma unroll
      for (int o = kFinishLanes / 2; o > 0; o >>= 1) {
        cl.x = fminf(cl.x, __shfl_xor_sync(gmask, cl.x, o, kFinishLanes));
        cl.y = fminf(cl.y, __shfl_xor_sync(gmask, cl.y, o, kFinishLanes));
        cl.z = fminf(cl.z, __shfl_xor_sync(gmask, cl.z, o, kFinishLanes));
        cl.w = fmaxf(cl.w, __shfl_xor_sync(gmask, cl.w, o, kFinishLanes));
        ch.x = fmaxf(ch.x, __shfl_xor_sync(gmask, ch.x, o, kFinishLanes));
        ch.y = fmaxf(ch.y, __shfl_xor_sync(gmask, ch.y, o, kFinishLanes));
        ch.z = fmaxf(ch.z, __shfl_xor_sync(gmask, ch.z, o, kFinishLanes));
      }
      if (gl == 0) {
        a.node[2 * p] = cl;
        a.node[2 * p + 1] = make_float4(ch.x, ch.y, ch.z, __int_as_float(link));
      }
      v = p;
    }
  }
}

struct WalkArgs {
  const Grid* grid;
  const unsigned* skeys;   // sorted cell ids
  const float4* node;
  const int2* leaf_range;
  const int* leaf_node;
  const int* node_parent;
  int* tctr;               // list entries reserved so far at kTreeEntries, tickets at kTreeTicket
  int2* nbr_span;          // per leaf: (first entry, length)
  unsigned* nbr;
  int nbr_cap;
};

constexpr int kOutBuf = 512;      // list entries a warp keeps in shared memory before reserving
constexpr int kWalkChunk = 8;     // leaves per ticket
constexpr size_t kWalkSmemBytes = sizeof(unsigned) * kWalkWarps * (kStack + kOutBuf);
static_assert(kOutBuf / 32 * 8 + 16 * 4 <= kStack, "the stack holds the masks and boxes of a shared walk");
static_assert((kOutBuf / 32 * 8) % 4 == 0, "the siblings' boxes start 16-byte aligned");

// Whether node b's box (shifted by the periodic image `code`) comes within
// the larger reach of the box (la, ha) and b's own: the particle test is
// r2 < H^2 + band(H) with H <= reach, evaluated with the same rounded
// operations, and 2^-12 extra slack. The test is monotone: a box inside
// another, with no larger reach, never passes where the larger one fails.
__device__ __forceinline__ bool box_near(const float4& la, const float4& ha, float4 lb, float4 hb, unsigned code,
                                         const float* L, float Lmax) {
  shift_j(code, L, lb.x, lb.y, lb.z);
  shift_j(code, L, hb.x, hb.y, hb.z);
  const float gx = fmaxf(fmaxf(lb.x - ha.x, la.x - hb.x), 0.0f);
  const float gy = fmaxf(fmaxf(lb.y - ha.y, la.y - hb.y), 0.0f);
  const float gz = fmaxf(fmaxf(lb.z - ha.z, la.z - hb.z), 0.0f);
  const float R = fmaxf(la.w, lb.w);
  return r2_of(gx, gy, gz) < (R * R + band_of(R, Lmax)) * 1.000244140625f;
}

// Walk of the trees of the 27 cells around `cell` for the box (la, ha):
// every leaf (with periodic image) that passes box_near, and whose
// ancestors do; entry t of the list goes to out[t] when t < out_cap, as
// leaf index | code << kIndexBits, or with `as_node` as its node index
// instead. Returns the list length; `overflow` when the stack ran out.
__device__ __forceinline__ int walk_box(const WalkArgs& a, const Grid& g, int cell, const float4& la,
                                        const float4& ha, unsigned* st, unsigned* out, int out_cap, bool as_node,
                                        bool& overflow) {
  const unsigned lane = lane_id();
  const float L[3] = {g.L[0], g.L[1], g.L[2]};
  const float Lmax = fmaxf(L[0], fmaxf(L[1], L[2]));
  const int nx = g.nc[0], ny = g.nc[1], nz = g.nc[2];
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
  overflow = false;
  __syncwarp();
  while (sp > 0 && !overflow) {
    const int gap = kStack - sp;
    const int take = min(sp, gap >= kDfsGap ? min(32, (gap - 80) / 7) : 1);
    unsigned e = 0;
    if ((int)lane < take) e = st[sp - take + (int)lane];
    sp -= take;
    __syncwarp();
    bool pass = false;
    int link = 0;
    const unsigned code = e >> kIndexBits;
    const int b = (int)(e & kIndexMask);
    if ((int)lane < take) {
      const float4 lb = a.node[2 * b], hb = a.node[2 * b + 1];
      link = __float_as_int(hb.w);
      pass = box_near(la, ha, lb, hb, code, L, Lmax);
    }
    const int nch = link >> kLinkShift;  // empty cells never pass
    const bool is_leaf = pass && nch == 0;
    const unsigned lm = __ballot_sync(kFull, is_leaf);
    if (is_leaf) {
      const int t = count + __popc(lm & ((1u << lane) - 1u));
      if (t < out_cap) out[t] = (unsigned)(as_node ? b : (link & kLinkMask)) | (code << kIndexBits);
    }
    count += __popc(lm);
    const int nk = pass ? nch : 0;
    int incl = nk;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, incl, o);
      if ((int)lane >= o) incl += y;
    }
    const int tot = __shfl_sync(kFull, incl, 31);
    if (sp + tot > kStack) {
      overflow = true;  // (never, by the bound above) this leaf's items would scan the 27 cells
    } else {
      const int first = link & kLinkMask;
      for (int t = 0; t < nk; ++t) st[sp + incl - nk + t] = (unsigned)(first + t) | (code << kIndexBits);
      sp += tot;
    }
    __syncwarp();
  }
  return count;
}

// One leaf's own walk; the list is reserved with one atomic and copied out
// (a list longer than the buffer is walked a second time straight into its
// place). A leaf whose walk ran out of stack gets no list.
__device__ __forceinline__ void walk_one_leaf(const WalkArgs& a, const Grid& g, int li, int cell, unsigned* st,
                                              unsigned* buf) {
  const unsigned lane = lane_id();
  const int va = a.leaf_node[li];
  const float4 la = a.node[2 * va], ha = a.node[2 * va + 1];
  bool overflow = false;
  const int count = walk_box(a, g, cell, la, ha, st, buf, kOutBuf, false, overflow);
  int base = 0;
  if (lane == 0 && !overflow) base = atomicAdd(&a.tctr[kTreeEntries], count);
  base = __shfl_sync(kFull, base, 0);
  const int room = a.nbr_cap - base;  // entries of this list that fit (a list past the cap is unused)
  if (!overflow) {
    if (count <= kOutBuf) {
      for (int t = (int)lane; t < count && t < room; t += 32) a.nbr[base + t] = buf[t];
    } else if (room > 0) {
      walk_box(a, g, cell, la, ha, st, a.nbr + base, room, false, overflow);
    }
  }
  if (lane == 0) a.nbr_span[li] = overflow ? make_int2(0, 0x7fffffff) : make_int2(base, count);
}

// Warps take kWalkChunk leaves per ticket. The leaves of one parent node
// have consecutive indices (leaves are numbered in node order, and a node's
// children are consecutive nodes), and the first of them walks for all: one
// walk with the parent's box and reach, whose list (in shared memory) holds
// every leaf any sibling's own walk would find, since the parent's box
// contains theirs and its reach is no smaller, and box_near is monotone.
// Each sibling's list is that list filtered by box_near against its own box:
// the same set its own walk gives, in the parent walk's order. A parent list
// longer than the buffer falls back to a walk per leaf. Each list is
// contiguous; where the lists lie does not change any result.
__global__ void __launch_bounds__(kWalkThreads) k_leaf_walk(WalkArgs a) {
  pdl_wait();
  extern __shared__ __align__(16) unsigned wsmem[];
  unsigned* st = wsmem + (threadIdx.x >> 5) * (kStack + kOutBuf);
  unsigned* buf = st + kStack;
  const unsigned lane = lane_id();
  const Grid& g = *a.grid;
  const float L[3] = {g.L[0], g.L[1], g.L[2]};
  const float Lmax = fmaxf(L[0], fmaxf(L[1], L[2]));
  const int nleaves = a.tctr[kTreeLeaves];
  for (;;) {
    int l0 = 0;
    if (lane == 0) l0 = atomicAdd(&a.tctr[kTreeTicket], kWalkChunk);
    l0 = __shfl_sync(kFull, l0, 0);
    if (l0 >= nleaves) break;
    for (int li = l0; li < min(l0 + kWalkChunk, nleaves); ++li) {
      const int p = a.node_parent[a.leaf_node[li]];
      if (p >= 0 && li > 0 && a.node_parent[a.leaf_node[li - 1]] == p) continue;  // a sibling walks for it
      const int cell = (int)a.skeys[a.leaf_range[li].x];
      // siblings: the leaves li, li + 1, ... with parent p (at most 8)
      int m = 1;
      if (p >= 0) {
        const int lj = li + (int)lane;
        const bool sib = lane < 8 && lj < nleaves && a.node_parent[a.leaf_node[lj]] == p;
        m = __ffs(~__ballot_sync(kFull, sib)) - 1;
      }
      if (m == 1) {
        walk_one_leaf(a, g, li, cell, st, buf);
        continue;
      }
      bool overflow = false;
      const float4 lp = a.node[2 * p], hp = a.node[2 * p + 1];
      const int count = walk_box(a, g, cell, lp, hp, st, buf, kOutBuf, true, overflow);
      if (overflow || count > kOutBuf) {
        for (int c = 0; c < m; ++c) walk_one_leaf(a, g, li + c, cell, st, buf);
        continue;
      }
      // one pass over the parent's list: lane t tests entry t against every
      // sibling's box; the ballot of sibling c for chunk q goes to
      // st[q * 8 + c] (the stack is empty now), and entry t becomes the
      // leaf index | code it is written out as
      const int nq = (count + 31) / 32;
      float4* sib_box = reinterpret_cast<float4*>(st + kOutBuf / 32 * 8);  // the siblings' boxes
      if ((int)lane < 2 * m) sib_box[lane] = a.node[2 * a.leaf_node[li + (int)(lane >> 1)] + (int)(lane & 1u)];
      __syncwarp();
      for (int q = 0; q < nq; ++q) {
        const int t = q * 32 + (int)lane;
        unsigned outv = 0;
        float4 lb = make_float4(0.0f, 0.0f, 0.0f, 0.0f), hb = lb;
        unsigned code = 0;
        const bool on = t < count;
        if (on) {
          const unsigned e = buf[t];
          const int b = (int)(e & kIndexMask);
          code = e >> kIndexBits;
          lb = a.node[2 * b];
          hb = a.node[2 * b + 1];
          outv = (unsigned)(__float_as_int(hb.w) & kLinkMask) | (code << kIndexBits);
        }
        for (int c = 0; c < m; ++c) {
          const unsigned pm = __ballot_sync(kFull, on && box_near(sib_box[2 * c], sib_box[2 * c + 1], lb, hb, code,
                                                                  L, Lmax));
          if (lane == 0) st[q * 8 + c] = pm;
        }
        __syncwarp();
        if (on) buf[t] = outv;
      }
      __syncwarp();
      // list lengths, one reservation for the family, then the lists
      int len = 0;
      if ((int)lane < m)
        for (int q = 0; q < nq; ++q) len += __popc(st[q * 8 + (int)lane]);
      int incl = len;
#pragma unroll
      for (int o = 1; o < 8; o <<= 1) {
        const int y = __shfl_up_sync(kFull, incl, o);
        if ((int)lane >= o) incl += y;
      }
      const int total = __shfl_sync(kFull, incl, 7);
      int base = 0;
      if (lane == 0) base = atomicAdd(&a.tctr[kTreeEntries], total);
      base = __shfl_sync(kFull, base, 0);
      if ((int)lane < m) a.nbr_span[li + (int)lane] = make_int2(base + incl - len, len);
      const unsigned lt = (1u << lane) - 1u;
      for (int c = 0; c < m; ++c) {
        int o = base + __shfl_sync(kFull, incl - len, c);
        for (int q = 0; q < nq; ++q) {
          const unsigned pm = st[q * 8 + c];
          if ((pm >> lane) & 1u) {
            const int dst = o + __popc(pm & lt);
            if (dst < a.nbr_cap) a.nbr[dst] = buf[q * 32 + (int)lane];
          }
          o += __popc(pm);
        }
      }
      __syncwarp();
    }
  }
}

int leaves_build(Ctx* c, const float4* pos_h, cudaStream_t s) {
  const int n = c->n;
  cudaMemsetAsync(c->d_tree_ctr, 0, sizeof(int) * kTreeCtrCount, s);
  if (n == 0) return cudaGetLastError() == cudaSuccess ? SWIFT_GPU_OK : SWIFT_GPU_ERR_CUDA;
  // per call: function attributes belong to the current device's context
  cudaFuncSetAttribute(k_leaf_walk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWalkSmemBytes);
  cudaMemsetAsync(c->d_node_flag, 0, sizeof(unsigned) * ((size_t)c->node_cap + 1), s);
  cudaMemsetAsync(c->d_node_done, 0, sizeof(int) * (size_t)c->node_cap, s);
  const int sm = c->num_sms;
  const unsigned* perm = c->d_vals[c->sorted_buf];
  unsigned* mk = c->d_keys[1 - c->sorted_buf];  // free after the sort
  launch_pdl(k_tree_gather, min((n + 255) / 256, sm * 8), 256, 0, s, pos_h, perm, (const unsigned*)c->d_aux[1], n,
             (const Grid*)c->d_grid, c->d_pos, mk);
  c->launches++;
  TreeArgs t;
  t.grid = c->d_grid;
  t.pos = c->d_pos;
  t.mk = mk;
  t.cell_start = c->d_cell_start;
  t.node_range = c->d_node_range;
  t.node = c->d_node;
  t.node_link = c->d_node_link;
  t.node_parent = c->d_node_parent;
  t.node_done = c->d_node_done;
  t.node_flag = c->d_node_flag;
  t.leaf_range = c->d_leaf_range;
  t.leaf_hcap = c->d_leaf_hcap;
  t.leaf_node = c->d_leaf_node;
  t.tctr = c->d_tree_ctr;
  t.node_cap = c->node_cap;
  t.leaf_max = c->params.leaf_max;
  t.margin = c->params.leaf_margin;
  t.kg = c->phys.kg;
  const int tree_blocks = sm * 8;
  for (int level = 0; level <= kTreeLevels; ++level) {
    launch_pdl(k_tree_split, tree_blocks, kTreeThreads, 0, s, t, level);
    c->launches++;
  }
  exclusive_scan(c, c->d_node_flag, c->d_node_flag, c->node_cap + 1, c->d_scan_tmp, s);
  launch_pdl(k_leaf_number, min((c->node_cap + 255) / 256, sm * 16), 256, 0, s, (const unsigned*)c->d_node_flag,
             c->node_cap, c->d_node_link, c->d_leaf_node, c->d_tree_ctr);
  launch_pdl(k_leaf_finish, tree_blocks, kTreeThreads, 0, s, t);
  c->launches += 2;
  WalkArgs w;
  w.grid = c->d_grid;
  w.skeys = c->d_keys[c->sorted_buf];
  w.node = c->d_node;
  w.leaf_range = c->d_leaf_range;
  w.leaf_node = c->d_leaf_node;
  w.node_parent = c->d_node_parent;
  w.tctr = c->d_tree_ctr;
  w.nbr_span = c->d_nbr_span;
  w.nbr = c->d_nbr;
  w.nbr_cap = c->nbr_cap;
  launch_pdl(k_leaf_walk, sm * 8, kWalkThreads, kWalkSmemBytes, s, w);
  c->launches++;
  return cudaGetLastError() == cudaSuccess ? SWIFT_GPU_OK : SWIFT_GPU_ERR_CUDA;
}

Nbr nbr_of(Ctx* c) {
  Nbr b;
  b.cell_start = c->d_cell_start;
  b.skeys = c->d_keys[c->sorted_buf];
  b.leaf_range = c->d_leaf_range;
  b.nbr_span = c->d_nbr_span;
  b.nbr = c->d_nbr;
  b.leaf_hcap = c->d_leaf_hcap;
  b.n_leaves = c->d_tree_ctr ? c->d_tree_ctr + kTreeLeaves : nullptr;
  b.nbr_cap = c->nbr_cap;
  b.adaptive = c->tree_built;
  return b;
}

__global__ void k_leaves_export(const int2* __restrict__ range, const float* __restrict__ hcap,
                                const int2* __restrict__ span, const int* __restrict__ tctr, int nbr_cap,
                                int64_t max_leaves, int32_t* __restrict__ out_range, float* __restrict__ out_hcap,
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
    if (out_cnt) {
      const int2 sp = span[l];
      out_cnt[l] = sp.y <= nbr_cap - sp.x ? sp.y : -1;  // -1: no list, the leaf's items scan the cells
    }
  }
}

int leaves_export_impl(Ctx* c, int32_t* range, float* hcap, int32_t* nbr_count, int64_t max_leaves, cudaStream_t s) {
  if (max_leaves <= 0 || c->n == 0) return SWIFT_GPU_OK;
  const int64_t m = max_leaves < c->n ? max_leaves : c->n;
  const int nb = (int)((m + 255) / 256 < c->num_sms * 8 ? (m + 255) / 256 : c->num_sms * 8);
  k_leaves_export<<<nb, 256, 0, s>>>(c->d_leaf_range, c->d_leaf_hcap, c->d_nbr_span, c->d_tree_ctr, c->nbr_cap,
                                     max_leaves, range, hcap, nbr_count);
  c->launches++;
  return cudaGetLastError() == cudaSuccess ? SWIFT_GPU_OK : SWIFT_GPU_ERR_CUDA;
}

}  // namespace sg
