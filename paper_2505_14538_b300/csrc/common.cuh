// common.cuh -- device-side types and helpers shared by the sm_103a kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/swift_gpu.h"

namespace sg {

constexpr int kWarp = 32;
constexpr int kItemMax = 16;          // particles per work item (at least two lanes each)
constexpr int kIndexBits = 26;        // list entry: j index (26 bits) + shift code (6 bits)
constexpr uint32_t kIndexMask = (1u << kIndexBits) - 1u;
constexpr float kPi = 3.14159265358979323846f;

// Guard band around H^2 in which the FP32 neighbour decision is re-taken in
// FP64 from the same float inputs. A periodic image costs one FP32 rounding
// of a coordinate (at most 2^-24 L), so the band has a relative part (FP32
// rounding of r^2 and H^2) and a part proportional to H L.
// r from r^2 >= 0 with the hardware's approximate square root (one
// instruction, relative error about 2^-23, exact at 0).
__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Programmatic dependent launch: a kernel launched with launch_pdl (internal.h)
// may be scheduled while the kernel before it on the stream is finishing; it
// waits here, as its first statement, until that kernel has completed and its
// memory is visible, so only the launch latency overlaps, not the work. In a
// kernel launched without the attribute the wait returns at once.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__host__ __device__ __forceinline__ float band_of(float H, float Lmax) {
  return H * H * 1.52587890625e-05f + H * Lmax * 9.5367431640625e-07f;  // 2^-16 H^2 + 2^-20 H L
}

// Device status word (first error wins; detail accumulates).
struct Status {
  int code;
  int pad;
  unsigned long long detail;
};

// Cell grid descriptor, computed on the device by the build so that no host
// synchronisation is needed.
constexpr int kMaxKeyPasses = 4;  // 8-bit radix passes over a cell id (at most 2^30 cells)

struct Grid {
  int nc[3];
  int ncells;
  float L[3];
  float hcap;        // largest h with kernel_gamma*h <= cell width
  int hcap_from_cells;
  int key_bits;
  float width[3];
  int pass_live[kMaxKeyPasses];  // radix pass q sorts bits 8q.. of the cell id (0: all zero)
  int sort_start;    // uniform grid: key buffer the cell ids are written to, so that the live
                     // passes alone end in the buffer the host expects
};

// The two key/value buffers of the cell sort.
struct KeyBufs {
  unsigned* k[2];
  unsigned* v[2];
};

// Status a particle capped at the cell's h raises: a wider cell would help
// (ERR_H_EXCEEDS_CELL) unless the user's h_max set the cap.
__host__ __device__ __forceinline__ int cell_cap_flag(const Grid& g) {
  return g.hcap_from_cells ? SWIFT_GPU_ERR_H_EXCEEDS_CELL : SWIFT_GPU_ERR_H_NOT_CONVERGED;
}

// Physics constants for the kernels.
struct Phys {
  float L[3];
  float kg;          // kernel_gamma
  float gamma_eos;
  float alpha_v, beta_v, alpha_c;
  double eta3;       // eta^3
  double h_tol;
  int max_iter;
  float h_max;       // user cap (0 = none)
  int compensated;
  int kernel;        // kernel shape: 0 cubic spline, 1 Wendland C2, 2 Wendland C4
  float knorm;       // its 3-D normalisation C (W = C H^-3 w(r/H))
};

// Where the candidate segments of a work item come from: the 27 neighbour
// cells of the item's cell (uniform grid), or the neighbour-leaf list of the
// item's leaf (adaptive leaves; Item::cell is then a leaf index). A list
// entry is a leaf index (kIndexBits) plus the periodic shift code. A leaf
// whose list does not end within nbr_cap was never written in full; its
// items scan the 27 neighbour cells of the leaf's cell instead.
struct Nbr {
  const int* cell_start;
  const unsigned* skeys;    // sorted cell ids
  const int2* leaf_range;   // [first, end) sorted positions of each leaf
  const int2* nbr_span;     // (first entry, length) of each leaf's list
  const unsigned* nbr;      // leaf index | shift code << kIndexBits
  const float* leaf_hcap;   // largest h the particles of a leaf may take
  const int* n_leaves;      // device count of leaves
  int nbr_cap;
  int adaptive;
};

constexpr int kTreeLevels = 10;     // octree levels below a cell (10-bit Morton code per axis)
constexpr int kAdaptiveNcCap = 256;  // cells per axis with adaptive leaves (the tree refines below)

// Octree counters of an adaptive build (device ints).
enum TreeCtr {
  kTreeNodes = 0,                   // [0 .. kTreeLevels]: nodes created at each level
  kTreeLeaves = kTreeLevels + 1,    // leaf count
  kTreeDepth,                       // deepest level holding a leaf
  kTreeEntries,                     // total entries of the leaf lists (reserved by the walk)
  kTreeTicket,                      // walk work tickets
  kTreeCtrCount = 16
};

struct Item {
  int cell;
  int off;   // offset into the particle index list
  int cnt;   // 1..kItemMax
  int pad;
};

// Statistics counters (device, 64-bit).
enum StatSlot {
  kStatInterDens = 0, kStatInterGrad, kStatInterForce,
  kStatCandDens, kStatCandGrad, kStatCandForce,
  kStatPasses, kStatItems, kStatInterHiter,
  kStatCount = 16
};

__device__ __forceinline__ void set_error(Status* st, int code, unsigned long long add = 1) {
  atomicCAS(&st->code, 0, code);
  atomicAdd(&st->detail, add);
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// TwoSum (Knuth): s + c carries the exact running sum of the added terms.
__device__ __forceinline__ void two_sum_acc(float& s, float& c, float x) {
  float t = s + x;
  float bp = t - s;
  float e = (s - (t - bp)) + (x - bp);
  s = t;
  c += e;
}

// Cubic-spline shape w(q) and dw/dq for q >= 0 (zero beyond q = 1).
__device__ __forceinline__ void spline(float q, float& w, float& dw) {
  float s = fmaxf(1.0f - q, 0.0f);
  float wo = 2.0f * s * s * s;
  float dwo = -6.0f * s * s;
  float q2 = q * q;
  float wi = fmaf(q2, fmaf(6.0f, q, -6.0f), 1.0f);
  float dwi = q * fmaf(18.0f, q, -12.0f);
  bool in = q < 0.5f;
  w = in ? wi : wo;
  dw = in ? dwi : dwo;
}

__device__ __forceinline__ float dspline(float q) {
  float s = fmaxf(1.0f - q, 0.0f);
  float dwo = -6.0f * s * s;
  float dwi = q * fmaf(18.0f, q, -12.0f);
  return q < 0.5f ? dwi : dwo;
}

// Kernel shapes (Sec. 2.1.1 names the cubic spline and the Wendland kernels):
// 0 cubic spline, 1 Wendland C2 w = (1-q)^4 (1+4q), 2 Wendland C4
// w = (1-q)^6 (1+6q+35q^2/3); W = C H^-3 w(r/H) with C the 3-D normalisation.
constexpr int kKernelCubic = 0, kKernelWendlandC2 = 1, kKernelWendlandC4 = 2;

__host__ __device__ __forceinline__ float kernel_norm(int kind) {
  return kind == kKernelWendlandC2 ? 21.0f / (2.0f * kPi) : kind == kKernelWendlandC4 ? 495.0f / (32.0f * kPi)
                                                                                       : 8.0f / kPi;
}

// Wendland C2 (kind 1) or C4 (kind 2) shape and dw/dq, zero beyond q = 1.
__device__ __forceinline__ void wendland(int kind, float q, float& w, float& dw) {
  const float s = fmaxf(1.0f - q, 0.0f);
  const float s2 = s * s;
  if (kind == kKernelWendlandC2) {
    const float s3 = s2 * s;
    w = s3 * s * fmaf(4.0f, q, 1.0f);
    dw = -20.0f * q * s3;
  } else {
    const float s4 = s2 * s2;
    w = s4 * s2 * fmaf(q, fmaf(35.0f / 3.0f, q, 6.0f), 1.0f);
    dw = (-56.0f / 3.0f) * q * fmaf(5.0f, q, 1.0f) * s4 * s;
  }
}

// w(q) and dw/dq of the selected shape (the branch is the same for a whole launch).
__device__ __forceinline__ void kshape(int kind, float q, float& w, float& dw) {
  if (kind == kKernelCubic) spline(q, w, dw);
  else wendland(kind, q, w, dw);
}

__device__ __forceinline__ float dkshape(int kind, float q) {
  if (kind == kKernelCubic) return dspline(q);
  float w, dw;
  wendland(kind, q, w, dw);
  return dw;
}

// dw/dq and d2w/dq2 of the selected shape (the adjoint loops).
__device__ __forceinline__ void kshape_d12(int kind, float q, float& dw, float& d2w) {
  const float s = fmaxf(1.0f - q, 0.0f);
  if (kind == kKernelCubic) {
    const bool in = q < 0.5f;
    dw = in ? q * fmaf(18.0f, q, -12.0f) : -6.0f * s * s;
    d2w = in ? fmaf(36.0f, q, -12.0f) : 12.0f * s;
  } else if (kind == kKernelWendlandC2) {
    const float s2 = s * s;
    dw = -20.0f * q * s2 * s;
    d2w = 20.0f * s2 * fmaf(4.0f, q, -1.0f);
  } else {
    const float s4 = (s * s) * (s * s);
    dw = (-56.0f / 3.0f) * q * fmaf(5.0f, q, 1.0f) * s4 * s;
    d2w = (56.0f / 3.0f) * s4 * fmaf(q, fmaf(35.0f, q, -4.0f), -1.0f);
  }
}

__device__ __forceinline__ float r2_of(float dx, float dy, float dz) {
  return fmaf(dz, dz, fmaf(dy, dy, dx * dx));
}

// Periodic image of a j particle: bit 2a adds L on axis a, bit 2a+1
// subtracts L (the j cell was wrapped across the low / high face).
__device__ __forceinline__ void shift_j(unsigned code, const float L[3], float& xj, float& yj, float& zj) {
  if (code) {
    if (code & 1u) xj += L[0];
    if (code & 2u) xj -= L[0];
    if (code & 4u) yj += L[1];
    if (code & 8u) yj -= L[1];
    if (code & 16u) zj += L[2];
    if (code & 32u) zj -= L[2];
  }
}

// The neighbour predicate, re-taken in FP64 exactly as the definition states
// it: dx = x_i - x_j, dx -= L round(dx/L), r2 = (dx^2 + dy^2) + dz^2 and
// H = kernel_gamma * h, each operation rounded once (no contraction).
static __device__ __noinline__ double exact_r2(float xi, float yi, float zi, float xj, float yj, float zj,
                                        float Lx, float Ly, float Lz) {
  double L[3] = {(double)Lx, (double)Ly, (double)Lz};
  double d[3] = {__dsub_rn((double)xi, (double)xj), __dsub_rn((double)yi, (double)yj),
                 __dsub_rn((double)zi, (double)zj)};
#pragma unroll
  for (int a = 0; a < 3; ++a) d[a] = __dsub_rn(d[a], __dmul_rn(L[a], round(__ddiv_rn(d[a], L[a]))));
  return __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
}

__device__ __forceinline__ double exact_H2(float kg, float h) {
  double H = __dmul_rn((double)kg, (double)h);
  return __dmul_rn(H, H);
}

// A coordinate wrapped into the periodic box [0, L) with the same FP64
// operations as the cell ids (x - L floor(x / L), each rounded once); a float
// already in [0, L) is returned as is. The FP32 result may round up to L, which
// still lies on the face of the cell the FP64 id gives it.
__device__ __forceinline__ float wrap_coord(float x, float L) {
  if (x >= 0.0f && x < L) return x;
  const double Ld = (double)L;
  return (float)__dsub_rn((double)x, __dmul_rn(Ld, floor(__ddiv_rn((double)x, Ld))));
}

__device__ __forceinline__ float4 wrap_pos(float4 p, const float L[3]) {
  return make_float4(wrap_coord(p.x, L[0]), wrap_coord(p.y, L[1]), wrap_coord(p.z, L[2]), p.w);
}

// Warp-wide max of an int.
__device__ __forceinline__ unsigned warp_sum(unsigned v) { return __reduce_add_sync(0xffffffffu, v); }

// Nanosecond timer for bounded waits.
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier for cooperative (co-resident) launches. Bounded: gives up
// after `limit_ns` (0: at once, without waiting) and records
// SWIFT_GPU_ERR_TIMEOUT; returns false then.
__device__ __forceinline__ bool grid_barrier(unsigned* count, unsigned* gen, Status* st,
                                             unsigned long long limit_ns) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    unsigned nb = gridDim.x * gridDim.y * gridDim.z;
    volatile unsigned* vgen = gen;
    unsigned g = *vgen;
    __threadfence();
    unsigned arrived = atomicAdd(count, 1u);
    if (arrived == nb - 1) {
      atomicExch(count, 0u);
      __threadfence();
      atomicAdd(gen, 1u);
    } else if (limit_ns == 0) {
      set_error(st, SWIFT_GPU_ERR_TIMEOUT);
      ok = 0;
    } else {
      unsigned long long t0 = global_ns();
      while (*vgen == g) {
        __nanosleep(100);
        if (global_ns() - t0 > limit_ns) {
          set_error(st, SWIFT_GPU_ERR_TIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

}  // namespace sg
