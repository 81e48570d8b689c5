// cells.cu -- device-side binning of particles into the periodic cell grid
// (Sec. 2.2, Fig. 3: cubic cells, self and pair interactions) and the stable
// sort of particles by cell id, all without host synchronisation.
//
//   k_scan_h       max of h, NaN / h <= 0 checks; its last block sets up the
//                  grid: nc, widths, h cap, key bits
//   k_cell_ids     FP64 cell id per particle (wrap, floor(x nc / L), clamp);
//                  with adaptive leaves also the Morton code inside the cell,
//                  sorted on first so that each cell ends in Morton order;
//                  per radix tile, the counts of the first pass
//   radix passes   LSD radix sort of (cell id, original index), 8-bit digits,
//                  stable, so ties keep the input order
//   k_cell_start   start offset of every cell (empty cells included)
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"

namespace sg {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;  // 2048

// ------------------------------------------------------------------ scans
// Exclusive scan of uint32, three phases: per-tile sums, scan of the sums in
// one block, then per-tile scans with the offsets.
__device__ __forceinline__ unsigned block_excl_scan(unsigned v, unsigned* smem, unsigned* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) smem[w] = x;
  __syncthreads();
  if (w == 0) {
    unsigned s = (lane < (int)(blockDim.x >> 5)) ? smem[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      unsigned y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    smem[lane] = s;  // inclusive per warp
  }
  __syncthreads();
  unsigned warp_off = (w > 0) ? smem[w - 1] : 0u;
  if (total) *total = smem[(blockDim.x >> 5) - 1];
  unsigned r = warp_off + x - v;
  __syncthreads();
  return r;
}

// `gate` (may be NULL): the scan is skipped when *gate == 0 (a radix pass
// over key bits the cells do not use).
__global__ void k_scan_tiles(const unsigned* __restrict__ in, int m, unsigned* __restrict__ tile_sums,
                             const int* __restrict__ gate) {
  pdl_wait();
  __shared__ unsigned sm[32];
  if (gate && *gate == 0) return;
  const int base = blockIdx.x * kScanTile;
  unsigned s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int i = base + threadIdx.x * kScanItems + k;
    s += (i < m) ? in[i] : 0u;
  }
  unsigned tot;
  block_excl_scan(s, sm, &tot);
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

__global__ void k_scan_top(unsigned* __restrict__ tile_sums, int ntiles, const int* __restrict__ gate) {
  pdl_wait();
  __shared__ unsigned sm[32];
  if (gate && *gate == 0) return;
  unsigned carry = 0;
  for (int base = 0; base < ntiles; base += kScanTile) {
    unsigned v[kScanItems];
    unsigned s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      int i = base + threadIdx.x * kScanItems + k;
      v[k] = (i < ntiles) ? tile_sums[i] : 0u;
      s += v[k];
    }
    unsigned tot;
    unsigned off = block_excl_scan(s, sm, &tot) + carry;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      int i = base + threadIdx.x * kScanItems + k;
      if (i < ntiles) tile_sums[i] = off;
      off += v[k];
    }
    carry += tot;
    __syncthreads();
  }
}

__global__ void k_scan_down(const unsigned* __restrict__ in, int m, const unsigned* __restrict__ tile_offs,
                            unsigned* __restrict__ out, const int* __restrict__ gate) {
  pdl_wait();
  __shared__ unsigned sm[32];
  if (gate && *gate == 0) return;
  const int base = blockIdx.x * kScanTile;
  unsigned v[kScanItems];
  unsigned s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int i = base + threadIdx.x * kScanItems + k;
    v[k] = (i < m) ? in[i] : 0u;
    s += v[k];
  }
  unsigned off = block_excl_scan(s, sm, nullptr) + tile_offs[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int i = base + threadIdx.x * kScanItems + k;
    if (i < m) out[i] = off;
    off += v[k];
  }
}

int scan_tiles_needed(int64_t m) { return (int)((m + kScanTile - 1) / kScanTile); }

// out may alias in. tile_tmp needs scan_tiles_needed(m) entries.
void exclusive_scan(Ctx* c, const unsigned* in, unsigned* out, int m, unsigned* tile_tmp, cudaStream_t s,
                    const int* gate) {
  if (m <= 0) return;
  int nt = scan_tiles_needed(m);
  launch_pdl(k_scan_tiles, nt, kScanThreads, 0, s, in, m, tile_tmp, gate);
  launch_pdl(k_scan_top, 1, kScanThreads, 0, s, tile_tmp, nt, gate);
  launch_pdl(k_scan_down, nt, kScanThreads, 0, s, in, m, tile_tmp, out, gate);
  c->launches += 3;
}

// ------------------------------------------------------------- grid setup
// Grid of the build from the largest h: nc per axis (cells no narrower than
// the support of the largest h, at least 3, at most nc_cap), widths, the h
// cap the cells allow, and the radix passes the cell ids need.
__device__ void grid_setup(float hmax, Grid* g, const Phys& ph, float margin, float min_width, int nc_cap,
                           int host_passes, Status* st) {
  float want = fmaxf(min_width, (1.0f + margin) * ph.kg * hmax);
  int nct = 1;
  for (int a = 0; a < 3; ++a) {
    int nc = want > 0.0f ? (int)floorf(ph.L[a] / want) : nc_cap;
    if (nc > nc_cap) nc = nc_cap;
    if (nc < 3) {
      nc = 3;
      if (want > ph.L[a] / 3.0f) set_error(st, SWIFT_GPU_ERR_H_EXCEEDS_CELL);
    }
    g->nc[a] = nc;
    g->L[a] = ph.L[a];
    g->width[a] = ph.L[a] / (float)nc;
    nct *= nc;
  }
  g->ncells = nct;
  float wmin = fminf(g->width[0], fminf(g->width[1], g->width[2]));
  // largest float h with kernel_gamma * h <= wmin in FP64 terms
  float hc = wmin * (1.0f - 9.5367432e-7f) / ph.kg;  // 2^-20 margin against FP64 rounding of cell ids
  while ((double)ph.kg * (double)hc > (double)wmin) hc = nextafterf(hc, 0.0f);
  g->hcap_from_cells = 1;
  if (ph.h_max > 0.0f && ph.h_max < hc) {
    hc = ph.h_max;
    g->hcap_from_cells = 0;
  }
  g->hcap = hc;
  int bits = 0;
  while ((1 << bits) < nct) ++bits;
  g->key_bits = bits;
  int live = 0;
  for (int q = 0; q < kMaxKeyPasses; ++q) {
    g->pass_live[q] = 8 * q < bits ? 1 : 0;
    live += g->pass_live[q];
  }
  // the host runs host_passes passes and reads the sort from buffer host_passes % 2; the
  // passes past the live ones do nothing, so the keys start where live passes end there
  g->sort_start = (host_passes & 1) ^ (live & 1);
}

// Largest h (NaN / h <= 0 rejected) into hm[0]; the last block to finish
// (counted in hm[1]) sets up the grid from it. hm starts zeroed.
__global__ void k_scan_h(const float4* __restrict__ pos_h, int n, unsigned* hm_words, Grid* g, Phys ph, float margin,
                         float min_width, int nc_cap, int host_passes, Status* st) {
  pdl_wait();
  __shared__ bool s_last;
  float hm = 0.0f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float4 p = pos_h[i];
    bool bad = !(isfinite(p.x) && isfinite(p.y) && isfinite(p.z) && isfinite(p.w)) || !(p.w > 0.0f);
    if (bad) set_error(st, SWIFT_GPU_ERR_ARG);
    else hm = fmaxf(hm, p.w);
  }
  for (int o = 16; o > 0; o >>= 1) hm = fmaxf(hm, __shfl_xor_sync(0xffffffffu, hm, o));
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&hm_words[0], __float_as_uint(hm));  // h > 0: bits order like values
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&hm_words[1], 1u) == gridDim.x - 1;
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
    __threadfence();
    const float hmax = __uint_as_float(atomicExch(&hm_words[0], 0u));
    atomicExch(&hm_words[1], 0u);  // both words zero again for the next call: no memset before it
    grid_setup(hmax, g, ph, margin, min_width, nc_cap, host_passes, st);
  }
}

// The grid alone (no particles).
__global__ void k_grid_setup(Grid* g, Phys ph, float margin, float min_width, int nc_cap, int host_passes,
                             Status* st) {
  grid_setup(0.0f, g, ph, margin, min_width, nc_cap, host_passes, st);
}

// Spread the 10 low bits of v to every third bit (bit b -> bit 3b).
__device__ __forceinline__ unsigned spread3(unsigned v) {
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000ffu;
  v = (v | (v << 8)) & 0x0300f00fu;
  v = (v | (v << 4)) & 0x030c30c3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

// 30-bit Morton code of a position inside its cell, from the fractions of
// the cell width along each axis, in units of 1/1024 of the width.
__device__ __forceinline__ unsigned morton_of(float fx, float fy, float fz) {
  const unsigned qx = (unsigned)fminf(fmaxf(fx * 1024.0f, 0.0f), 1023.0f);
  const unsigned qy = (unsigned)fminf(fmaxf(fy * 1024.0f, 0.0f), 1023.0f);
  const unsigned qz = (unsigned)fminf(fmaxf(fz * 1024.0f, 0.0f), 1023.0f);
  return spread3(qx) | (spread3(qy) << 1) | (spread3(qz) << 2);
}

// Cell id of every particle; with `cell_out` (adaptive leaves) the sort key
// is instead the 30-bit Morton code of the position inside the cell (10 bits
// per axis, x in the lowest bit of each 3-bit digit) and the cell id goes to
// cell_out, morton_out keeping a copy of the code. Blocks take the radix
// tiles, so each also writes its tile's histogram of the keys' lowest digit:
// the counts of the first radix pass.
__global__ void __launch_bounds__(kRadixThreads) k_cell_ids(const float4* __restrict__ pos_h, int n,
                                                            const Grid* __restrict__ g, KeyBufs kb,
                                                            unsigned* __restrict__ cell_out,
                                                            unsigned* __restrict__ morton_out,
                                                            unsigned* __restrict__ hist) {
  pdl_wait();
  __shared__ unsigned hcount[256];
  // uniform grid: buffer g->sort_start; adaptive leaves: buffer 0 (their passes are all live)
  const int b = cell_out ? 0 : g->sort_start;
  unsigned* __restrict__ keys = kb.k[b];
  unsigned* __restrict__ vals = kb.v[b];
  const int nx = g->nc[0], ny = g->nc[1], nz = g->nc[2];
  const double Lx = g->L[0], Ly = g->L[1], Lz = g->L[2];
  const float ncf[3] = {(float)nx, (float)ny, (float)nz};
  const float Lf[3] = {g->L[0], g->L[1], g->L[2]};
  hcount[threadIdx.x] = 0;
  float4 pt[kRadixItems];  // the tile's positions, all loads issued first
#pragma unroll
  for (int it = 0; it < kRadixItems; ++it) {
    const int i = blockIdx.x * kRadixTile + it * kRadixThreads + (int)threadIdx.x;
    pt[it] = i < n ? pos_h[i] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < kRadixItems; ++it) {
    const int i = blockIdx.x * kRadixTile + it * kRadixThreads + (int)threadIdx.x;
    if (i >= n) continue;
    unsigned key;
    const float4 p = pt[it];
    vals[i] = (unsigned)i;
    {
      // FP32 first: t = x nc / L carries at most 3 roundings (< 2^-22 t), so
      // a fraction of t farther than 8 ulps from an integer floors as the FP64
      // value does; closer ones, positions outside [0, L) and, for Morton
      // codes, box sides other than 1 take FP64.
      const float xs[3] = {p.x, p.y, p.z};
      int cf[3];
      float frs[3];
      bool ok = true;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const float t = Lf[q] == 1.0f ? xs[q] * ncf[q] : (xs[q] * ncf[q]) / Lf[q];
        const float fl = floorf(t);
        const float fr = t - fl;
        const float eta = 4.76837158203125e-7f * fmaxf(t, 1.0f);  // 8 * 2^-24
        ok = ok && xs[q] >= 0.0f && xs[q] < Lf[q] && fr > eta && fr < 1.0f - eta;
        cf[q] = min(max((int)fl, 0), (q == 0 ? nx : q == 1 ? ny : nz) - 1);
        // Morton fraction (L = 1): x nc = t + lo exactly, and t - fl is
        // exact, so one rounding gives the float of the exact fraction,
        // as the FP64 path's float(x nc - c)
        frs[q] = fr + fmaf(xs[q], ncf[q], -t);
        ok = ok && (cell_out == nullptr || Lf[q] == 1.0f);
      }
      if (ok) {
        const unsigned cell = (unsigned)(cf[0] + nx * (cf[1] + ny * cf[2]));
        if (cell_out) {
          const unsigned m = morton_of(frs[0], frs[1], frs[2]);
          keys[i] = key = m;
          morton_out[i] = m;
          cell_out[i] = cell;
        } else {
          keys[i] = key = cell;
        }
        atomicAdd(&hcount[key & 255u], 1u);
        continue;
      }
    }
    // wrap into [0, L) and floor(x nc / L), each FP64 operation rounded once.
    // A float x in [0, L) has floor(x / L) = 0, and x * nc is exact, so the
    // divisions (slow in FP64) are skipped only where they cannot change the result.
    double x = p.x, y = p.y, z = p.z;
    if (!(x >= 0.0 && x < Lx)) x = __dsub_rn(x, __dmul_rn(Lx, floor(__ddiv_rn(x, Lx))));
    if (!(y >= 0.0 && y < Ly)) y = __dsub_rn(y, __dmul_rn(Ly, floor(__ddiv_rn(y, Ly))));
    if (!(z >= 0.0 && z < Lz)) z = __dsub_rn(z, __dmul_rn(Lz, floor(__ddiv_rn(z, Lz))));
    const double tx0 = __dmul_rn(x, (double)nx), ty0 = __dmul_rn(y, (double)ny), tz0 = __dmul_rn(z, (double)nz);
    const double tx = Lx == 1.0 ? tx0 : __ddiv_rn(tx0, Lx);
    const double ty = Ly == 1.0 ? ty0 : __ddiv_rn(ty0, Ly);
    const double tz = Lz == 1.0 ? tz0 : __ddiv_rn(tz0, Lz);
    int cx = (int)floor(tx), cy = (int)floor(ty), cz = (int)floor(tz);
    cx = min(max(cx, 0), nx - 1);
    cy = min(max(cy, 0), ny - 1);
    cz = min(max(cz, 0), nz - 1);
    const unsigned cell = (unsigned)(cx + nx * (cy + ny * cz));
    if (cell_out) {
      // the fraction is exact in FP64; its FP32 rounding only orders particles
      const unsigned m = morton_of((float)(tx - cx), (float)(ty - cy), (float)(tz - cz));
      keys[i] = key = m;
      morton_out[i] = m;
      cell_out[i] = cell;
    } else {
      keys[i] = key = cell;
    }
    atomicAdd(&hcount[key & 255u], 1u);
  }
  __syncthreads();
  hist[threadIdx.x * gridDim.x + blockIdx.x] = hcount[threadIdx.x];
}

// keys[k] = src[idx[k]]
// Adaptive leaves: after the Morton passes (in buffer 0), the cell ids of the
// Morton-ordered particles become the keys of the cell-id passes, in buffer
// g->sort_start (with their values) like the uniform grid's keys.
__global__ void k_gather_keys(KeyBufs kb, const unsigned* __restrict__ cell_of, int n, const Grid* __restrict__ g) {
  pdl_wait();
  const int b = g->sort_start;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const unsigned v = kb.v[0][k];
    kb.k[b][k] = cell_of[v];
    if (b != 0) kb.v[b][k] = v;
  }
}

// ------------------------------------------------------------ radix sort
// Histogram layout: hist[d * nblocks + b].
// Radix pass `pass` over 8-bit digit `shift`. With bits >= 0 (the Morton keys of
// adaptive leaves) every pass is live and src is the host's buffer. With bits
// < 0 (cell ids) a pass over bits no cell uses does nothing, and the live
// passes read buffer g->sort_start ^ (pass & 1): they end in the buffer the
// host reads.
__device__ __forceinline__ int pass_src(const Grid* g, int bits, int pass, int host_src) {
  return bits >= 0 ? host_src : (g->sort_start ^ (pass & 1));
}

__global__ void k_radix_count(KeyBufs kb, int host_src, int pass, int n, int shift, const Grid* __restrict__ g,
                              int bits, unsigned* __restrict__ hist) {
  pdl_wait();
  __shared__ unsigned h[256];
  const bool live = shift < (bits >= 0 ? bits : g->key_bits);
  if (!live) return;  // its scan and scatter are skipped too
  const unsigned* __restrict__ keys = kb.k[pass_src(g, bits, pass, host_src)];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int base = blockIdx.x * kRadixTile;
  for (int k = 0; k < kRadixItems; ++k) {
    int i = base + k * kRadixThreads + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[threadIdx.x * gridDim.x + blockIdx.x] = h[threadIdx.x];
}

__global__ void k_radix_scatter(KeyBufs kb, int host_src, int pass, int n, int shift, const Grid* __restrict__ g,
                                int bits, const unsigned* __restrict__ offs) {
  pdl_wait();
  __shared__ unsigned run[256];
  __shared__ unsigned wcnt[kRadixThreads / 32][256];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool live = shift < (bits >= 0 ? bits : g->key_bits);
  if (!live) return;
  const int src = pass_src(g, bits, pass, host_src);
  const unsigned* __restrict__ kin = kb.k[src];
  const unsigned* __restrict__ vin = kb.v[src];
  unsigned* __restrict__ kout = kb.k[1 - src];
  unsigned* __restrict__ vout = kb.v[1 - src];
  run[threadIdx.x] = offs[threadIdx.x * gridDim.x + blockIdx.x];
  for (int ww = 0; ww < kRadixThreads / 32; ++ww) wcnt[ww][threadIdx.x] = 0;
  const int base = blockIdx.x * kRadixTile;
  unsigned keys[kRadixItems], vals[kRadixItems];  // the tile's keys, all loads issued first
#pragma unroll
  for (int k = 0; k < kRadixItems; ++k) {
    const int i = base + k * kRadixThreads + threadIdx.x;
    keys[k] = i < n ? kin[i] : 0u;
    vals[k] = i < n ? vin[i] : 0u;
  }
  __syncthreads();
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int k = 0; k < kRadixItems; ++k) {
    int i = base + k * kRadixThreads + threadIdx.x;
    bool valid = i < n;
    unsigned key = keys[k];
    unsigned val = vals[k];
    unsigned d = (key >> shift) & 255u;
    unsigned vmask = __ballot_sync(0xffffffffu, valid);
    unsigned peers = __match_any_sync(0xffffffffu, valid ? d : 0xffffffffu) & vmask;
    unsigned rank = __popc(peers & lt);
    if (valid && rank == 0) wcnt[w][d] = __popc(peers);
    __syncthreads();
    if (valid) {
      unsigned pos = run[d] + rank;
      for (int ww = 0; ww < w; ++ww) pos += wcnt[ww][d];
      kout[pos] = key;
      vout[pos] = val;
    }
    __syncthreads();
    unsigned add = 0;
    for (int ww = 0; ww < kRadixThreads / 32; ++ww) {
      add += wcnt[ww][threadIdx.x];
      wcnt[ww][threadIdx.x] = 0;
    }
    run[threadIdx.x] += add;
    __syncthreads();
  }
}

__global__ void k_cell_start(const unsigned* __restrict__ skeys, int n, const Grid* __restrict__ g,
                             int* __restrict__ cell_start) {
  pdl_wait();
  const int nct = g->ncells;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= n; k += gridDim.x * blockDim.x) {
    int lo = (k == 0) ? 0 : (int)skeys[k - 1] + 1;
    int hi = (k == n) ? nct : (int)skeys[k];
    for (int c = lo; c <= hi; ++c) cell_start[c] = k;
  }
}

int build_cells_impl(Ctx* c, const float4* pos_h, int n, float min_width, cudaStream_t s) {
  c->n = n;
  c->lpp_lists = 0;  // kept candidate lists belong to the previous build
  int sm = c->num_sms;
  const bool adaptive = (c->params.flags & SWIFT_GPU_ADAPTIVE) != 0;
  const int nc_cap = adaptive && c->nc_cap > kAdaptiveNcCap ? kAdaptiveNcCap : c->nc_cap;
  const int host_passes = (c->max_key_bits + 7) / 8;
  if (n > 0) {
    launch_pdl(k_scan_h, min((n + 255) / 256, sm * 8), 256, 0, s, pos_h, n, c->d_hmax_bits, c->d_grid, c->phys,
               c->params.cell_margin, min_width, nc_cap, host_passes, c->d_status);
  } else {
    k_grid_setup<<<1, 1, 0, s>>>(c->d_grid, c->phys, c->params.cell_margin, min_width, nc_cap, host_passes,
                                 c->d_status);
  }
  c->launches++;
  if (n > 0) {
    int gb = min((n + 255) / 256, sm * 8);
    const KeyBufs kb{{c->d_keys[0], c->d_keys[1]}, {c->d_vals[0], c->d_vals[1]}};
    const int nb = (n + kRadixTile - 1) / kRadixTile;
    // the keys, and the counts of the first pass (its digit 0 is always live)
    launch_pdl(k_cell_ids, nb, kRadixThreads, 0, s, pos_h, n, c->d_grid, kb, adaptive ? c->d_aux[0] : nullptr,
               adaptive ? c->d_aux[1] : nullptr, c->d_hist);
    c->launches++;
    int src = 0;  // host's view of the buffer a pass reads (as if every pass ran)
    bool counted = true;
    auto pass = [&](int p, int shift, int bits) {
      if (!counted) {
        launch_pdl(k_radix_count, nb, kRadixThreads, 0, s, kb, src, p, n, shift, c->d_grid, bits, c->d_hist);
        c->launches++;
      }
      counted = false;
      const int* gate = bits >= 0 ? nullptr : &c->d_grid->pass_live[shift / 8];
      exclusive_scan(c, c->d_hist, c->d_hist, 256 * nb, c->d_scan_tmp, s, gate);
      launch_pdl(k_radix_scatter, nb, kRadixThreads, 0, s, kb, src, p, n, shift, c->d_grid, bits, c->d_hist);
      c->launches++;
      src = 1 - src;
    };
    if (adaptive) {
      // least significant key first: the Morton code inside the cell (four passes, ending in
      // buffer 0), then the cell id
      for (int shift = 0, p = 0; shift < 30; shift += 8, ++p) pass(p, shift, 30);
      launch_pdl(k_gather_keys, gb, 256, 0, s, kb, c->d_aux[0], n, c->d_grid);
      c->launches++;
    }
    for (int shift = 0, p = 0; shift < c->max_key_bits; shift += 8, ++p) pass(p, shift, -1);
    // the live cell-id passes end in buffer host_passes % 2 (their start buffer was chosen for it)
    c->sorted_buf = host_passes & 1;
  }
  {
    int gb = min((n + 1 + 255) / 256, sm * 8);
    launch_pdl(k_cell_start, max(gb, 1), 256, 0, s, c->d_keys[c->sorted_buf], n, c->d_grid, c->d_cell_start);
    c->launches++;
  }
  c->tree_built = 0;
  if (adaptive) {
    const int rc = leaves_build(c, pos_h, s);
    if (rc != SWIFT_GPU_OK) return rc;
    c->tree_built = 1;
  }
  return cudaGetLastError() == cudaSuccess ? SWIFT_GPU_OK : SWIFT_GPU_ERR_CUDA;
}

}  // namespace sg

namespace sg {

__global__ void k_cells_export(const unsigned* __restrict__ skeys, const unsigned* __restrict__ svals, int n,
                               uint32_t* __restrict__ cell_id, uint32_t* __restrict__ perm) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const unsigned src = svals[k];
    if (cell_id) cell_id[src] = skeys[k];
    if (perm) perm[k] = src;
  }
}

int cells_export_impl(Ctx* c, uint32_t* cell_id, uint32_t* perm, cudaStream_t s) {
  if (c->n == 0) return SWIFT_GPU_OK;
  const int nb = min((c->n + 255) / 256, c->num_sms * 8);
  k_cells_export<<<nb, 256, 0, s>>>(c->d_keys[c->sorted_buf], c->d_vals[c->sorted_buf], c->n, cell_id, perm);
  c->launches++;
  return cudaGetLastError() == cudaSuccess ? SWIFT_GPU_OK : SWIFT_GPU_ERR_CUDA;
}

}  // namespace sg
