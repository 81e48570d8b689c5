// internal.h -- host-side context shared by the .cu files of the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

struct swift_gpu_ctx;

namespace sg {

struct Ctx {
  int device = 0;
  int num_sms = 0;
  swift_gpu_params params{};
  swift_gpu_tuning tuning{};
  Phys phys{};
  int64_t n_max = 0;
  int nc_cap = 0;
  int max_key_bits = 0;
  int n = 0;
  int sorted_buf = 0;
  uint64_t launches = 0;
  int state = 0;  // bit 0 cells, 1 density, 2 ghost, 3 force
  int all_active = 1;
  int last_passes = 0;
  cudaStream_t last_stream = nullptr;
  // arguments of the last calls (autotune re-runs them; they are idempotent)
  const float4* last_pos_in = nullptr;
  const float4* last_vel_in = nullptr;
  const uint8_t* last_active = nullptr;
  float* last_h_out = nullptr;
  float4* last_rho4 = nullptr;
  float4* last_cd = nullptr;
  uint32_t* last_ngb = nullptr;
  const float* last_u = nullptr;
  const float* last_alpha_v = nullptr;
  const float* last_alpha_c = nullptr;
  float2* last_grad_out = nullptr;
  float4* last_force_out = nullptr;
  float* last_dhdt = nullptr;

  // device buffers (all allocated at create)
  Status* d_status = nullptr;
  Grid* d_grid = nullptr;
  unsigned* d_hmax_bits = nullptr;
  unsigned* d_keys[2] = {nullptr, nullptr};
  unsigned* d_vals[2] = {nullptr, nullptr};
  unsigned* d_hist = nullptr;
  unsigned* d_scan_tmp = nullptr;
  int* d_cell_start = nullptr;
  float4* d_pos = nullptr;    // sorted (x, y, z, h)
  float4* d_vel = nullptr;    // sorted (vx, vy, vz, m)
  float4* d_rho4 = nullptr;   // sorted (rho, drho/dh, n, dn/dh)
  float4* d_cd = nullptr;     // sorted (curl, div)
  float* d_h = nullptr;       // sorted h during the Newton iteration
  float2* d_bracket = nullptr;// sorted Newton bracket (lo, hi)
  unsigned* d_ngb = nullptr;  // sorted neighbour counts
  float4* d_ga = nullptr;     // sorted ghost (A = f P/rho^2, f, rho, c)
  float4* d_gb = nullptr;     // sorted ghost (B, alpha_v, alpha_c P, u)
  uint8_t* d_act = nullptr;   // sorted active flags
  Item* d_items0 = nullptr;   // active work items (kept for gradient/force)
  int* d_plist0 = nullptr;
  Item* d_items[2] = {nullptr, nullptr};
  int* d_plist[2] = {nullptr, nullptr};
  int* d_counters = nullptr;  // per pass: [item_count, plist_count, ticket] x (max passes + 1); + barrier
  unsigned long long* d_stats = nullptr;
  double* d_red_partial = nullptr;  // per block partial FP64 reductions
  float4* d_scratch4[4] = {nullptr, nullptr, nullptr, nullptr};  // work arrays (sorted), one block of 4 n_max
  uint8_t* d_plain_act = nullptr;  // active flags while the per-task path iterates
  float* d_scratch1[2] = {nullptr, nullptr};
  int red_blocks = 0;
  int max_passes = 0;

  // adaptive leaves (built when params.flags has SWIFT_GPU_ADAPTIVE)
  int tree_built = 0;            // the last build made leaves; the loops take their segments from them
  int node_cap = 0, leaf_cap = 0, nbr_cap = 0;
  unsigned* d_aux[2] = {nullptr, nullptr};  // caller order: cell id, Morton code inside the cell
  int2* d_node_range = nullptr;  // [first, end) sorted positions
  float4* d_node = nullptr;      // 2 per node: (box low corner, reach kernel_gamma * h_cap), (box high corner, link)
  int* d_node_link = nullptr;    // link word of each node while the tree is built
  int* d_node_parent = nullptr;  // parent node (-1 for cells)
  int* d_node_done = nullptr;    // children finished (bottom-up pass)
  unsigned* d_node_flag = nullptr;  // leaf flags, then their exclusive scan (node_cap + 1)
  int2* d_leaf_range = nullptr;
  float* d_leaf_hcap = nullptr;
  int* d_leaf_node = nullptr;
  int2* d_nbr_span = nullptr;    // per leaf: (first list entry, list length)
  unsigned* d_nbr = nullptr;     // leaf index | shift code << kIndexBits
  int* d_tree_ctr = nullptr;     // TreeCtr

  // candidate lists kept by the density call for the later loops
  unsigned* d_nlist = nullptr;
  long long nl_cap = 0;
  int2* d_item_nl = nullptr;
  // lane-per-particle path (uniform grid): the 13 axis-sorted replicas of the
  // cells (13 n_max float4), the per-lane candidate counts of the groups' kept
  // lists (n_max), and whether the last density call kept such lists
  float4* d_rep = nullptr;
  int* d_lcnt = nullptr;
  float4* d_gc = nullptr;  // sorted (x, y, z, 1/H) from the ghost step: the force term's position record

  int lpp_lists = 0;

  // host mirrors
  Status* h_status = nullptr;  // pinned
  unsigned long long* h_stats = nullptr;  // pinned
};

Ctx* from(swift_gpu_ctx* c);
int phys_from(const swift_gpu_params* p, Phys* ph);

int scan_tiles_needed(int64_t m);
void exclusive_scan(Ctx* c, const unsigned* in, unsigned* out, int m, unsigned* tile_tmp, cudaStream_t s,
                    const int* gate = nullptr);
int build_cells_impl(Ctx* c, const float4* pos_h, int n, float min_width, cudaStream_t s);
int density_impl(Ctx* c, const float4* pos_h_in, const float4* vel_m, const uint8_t* active, float* h_out,
                 float4* rho4, float4* curl_div, uint32_t* ngb, cudaStream_t s);
int ghost_impl(Ctx* c, const float* u, const float* alpha_v, const float* alpha_c, cudaStream_t s);
int set_inactive_impl(Ctx* c, const uint8_t* mask, const float* h, const float4* rho4, const float4* cd,
                      cudaStream_t s);
int gradient_impl(Ctx* c, float2* vsig_lapu, cudaStream_t s);
int force_impl(Ctx* c, float4* accel_dudt, float* dh_dt, double* reductions, cudaStream_t s);
int grad_force_impl(Ctx* c, float2* vsig_lapu, float4* accel_dudt, float* dh_dt, double* reductions,
                    cudaStream_t s);
int plain_density_impl(Ctx* c, const float4* pos_h_in, const float4* vel_m, const uint8_t* active, float* h_out,
                       float4* rho4, float4* curl_div, uint32_t* ngb, cudaStream_t s);
int plain_gradient_impl(Ctx* c, float2* vsig_lapu, cudaStream_t s);
int plain_force_impl(Ctx* c, float4* accel_dudt, float* dh_dt, double* reductions, cudaStream_t s);
void reduce_partials(Ctx* c, int nblocks, double* out, cudaStream_t s);
int leaves_build(Ctx* c, const float4* pos_h, cudaStream_t s);
int leaves_export_impl(Ctx* c, int32_t* range, float* hcap, int32_t* nbr_count, int64_t max_leaves, cudaStream_t s);
Nbr nbr_of(Ctx* c);
int cells_export_impl(Ctx* c, uint32_t* cell_id, uint32_t* perm, cudaStream_t s);
int autotune_impl(Ctx* c, int loop, cudaStream_t s);
int backward_impl(Ctx* c, const float4* grad_ad, float4* grad_x, float4* grad_v, float* grad_u, int h_mode,
                  cudaStream_t s);

// Lanes per particle of the cell-item kernels. A tuning of one lane a
// particle selects the lane-per-particle path where it exists; the cell-item
// kernels that still run there (the later density passes, the adjoint, the
// fallbacks) share a particle among up to 32 lanes.
inline int cell_lanes(const Ctx* c) {
  return c->tuning.max_lanes_per_particle == 1 && c->d_rep ? 32 : c->tuning.max_lanes_per_particle;
}

// Most Newton passes of one density call: the counters of the context and of
// the static entry point are laid out for this many.
constexpr int kMaxPasses = 64;

// Limit of each bounded device-side wait: tuning.wait_limit_us (0: 5 s;
// negative: give up at once, the fault-injection setting).
inline unsigned long long wait_limit_ns(const Ctx* c) {
  const int us = c->tuning.wait_limit_us;
  if (us < 0) return 0ull;
  if (us == 0) return 5000000000ull;
  return (unsigned long long)us * 1000ull;
}

// Radix sort of the cell ids: one block sorts a tile of kRadixTile keys, and
// the histogram holds 256 digits per tile (every allocation derives from these).
constexpr int kRadixThreads = 256;
constexpr int kRadixItems = 8;
constexpr int kRadixTile = kRadixThreads * kRadixItems;  // 2048
// The max-h buffer of the cell build: the bits of the largest h, and the
// count of k_scan_h blocks done (the last one sets up the grid).
constexpr int kHmaxWords = 2;

// counters layout helpers
constexpr int kCtrPerPass = 4;  // item_count, plist_count, ticket, spare
__host__ __device__ inline int ctr_index(int pass, int which) { return pass * kCtrPerPass + which; }
// After the passes' counters: the later loops' tickets (pass slot passes + 1: gradient, force, and the
// adjoint's two), the density launch's grid barrier (2), the ticket of the cell-item launch that follows
// a lane-per-particle one, and the flag the density call sets when a group has no kept list.
__host__ __device__ constexpr int kCtrUnlistedTicket(int passes) { return kCtrPerPass * (passes + 2) + 2; }
__host__ __device__ constexpr int kCtrMissing(int passes) { return kCtrPerPass * (passes + 2) + 3; }
// finished-block counts of the loop launches' tickets: 0 gradient, 1 force, 2 unlisted
__host__ __device__ constexpr int kCtrLoopDone(int passes, int which) { return kCtrPerPass * (passes + 2) + 4 + which; }
__host__ __device__ constexpr int kCtrCount(int passes) { return kCtrPerPass * (passes + 2) + 7; }

// Launch of a kernel whose first statement is pdl_wait() (common.cuh), with
// programmatic stream serialization: its blocks may be scheduled while the
// previous kernel on the stream drains, which hides the launch gap between the
// short kernels of a chain (the cell sort, the loop epilogues). Stream capture
// records the dependency as a programmatic edge.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

}  // namespace sg
