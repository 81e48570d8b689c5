// static_density.cu -- swift_gpu_density_static: the density call (cell
// build, density loop and h iteration) for callers that cannot allocate GPU
// memory, e.g. code running inside a host framework whose allocator owns all
// device memory and forbids direct cudaMalloc, or a plug-in that may only use
// buffers its host hands it. Every work buffer of the call lives in one
// file-scope __device__ array of fixed size; nothing is allocated, on the
// device or the host.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "internal.h"

namespace sg {

// Capacity of the static scratch: particles and the cell grid it implies
// (at most 2 * n_max cells, as for a context of the same size).
constexpr int64_t kStaticN = SWIFT_GPU_STATIC_MAX_PARTICLES;
constexpr int kStaticMaxPasses = kMaxPasses;  // the counters hold every pass phys_from allows
constexpr size_t kAlign = 256;

constexpr size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

constexpr int static_nc_cap() {
  int c = 3;
  while ((int64_t)(c + 1) * (c + 1) * (c + 1) <= 2 * kStaticN) ++c;
  return c;
}
constexpr int64_t kStaticCells = (int64_t)static_nc_cap() * static_nc_cap() * static_nc_cap();
constexpr int64_t kStaticRadixBlocks = (kStaticN + kRadixTile - 1) / kRadixTile;
constexpr int64_t kStaticScanM = 256 * kStaticRadixBlocks > kStaticCells + 1 ? 256 * kStaticRadixBlocks
                                                                             : kStaticCells + 1;

// Layout of the scratch array (byte offsets, each sub-buffer 256-byte aligned).
struct StaticLayout {
  size_t status, grid, hmax, keys0, keys1, vals0, vals1, hist, scan_tmp, cell_start, pos, vel, rho4, cd, h,
      bracket, ngb, act, items0, items1, items2, plist0, plist1, plist2, counters, stats, total;
};

constexpr StaticLayout static_layout() {
  StaticLayout L{};
  size_t o = 0;
  auto take = [&o](size_t bytes) {
    size_t at = o;
    o = align_up(o + bytes);
    return at;
  };
  const size_t n = (size_t)kStaticN;
  L.status = take(sizeof(Status));
  L.grid = take(sizeof(Grid));
  L.hmax = take(sizeof(unsigned) * kHmaxWords);
  L.keys0 = take(4 * n);
  L.keys1 = take(4 * n);
  L.vals0 = take(4 * n);
  L.vals1 = take(4 * n);
  L.hist = take(4 * 256 * (size_t)kStaticRadixBlocks);
  L.scan_tmp = take(4 * (size_t)((kStaticScanM + 2047) / 2048 + 1));
  L.cell_start = take(4 * (size_t)(kStaticCells + 1));
  L.pos = take(16 * n);
  L.vel = take(16 * n);
  L.rho4 = take(16 * n);
  L.cd = take(16 * n);
  L.h = take(4 * n);
  L.bracket = take(8 * n);
  L.ngb = take(4 * n);
  L.act = take(n);
  L.items0 = take(sizeof(Item) * n);
  L.items1 = take(sizeof(Item) * n);
  L.items2 = take(sizeof(Item) * n);
  L.plist0 = take(4 * n);
  L.plist1 = take(4 * n);
  L.plist2 = take(4 * n);
  L.counters = take(sizeof(int) * (size_t)kCtrCount(kStaticMaxPasses));
  L.stats = take(sizeof(unsigned long long) * kStatCount);
  L.total = o;
  return L;
}
constexpr StaticLayout kLayout = static_layout();

// The scratch itself. Host code must not pass its name to a kernel (on the
// host the name is only a stand-in); the device address comes from
// cudaGetSymbolAddress, taken once per device below.
static __device__ __align__(256) unsigned char g_static_scratch[kLayout.total];

constexpr int kMaxDevices = 64;
static void* g_scratch_addr[kMaxDevices] = {nullptr};

__global__ void k_static_status(const Status* __restrict__ st, int64_t* __restrict__ out) {
  out[0] = st->code;
  out[1] = (int64_t)st->detail;
}

}  // namespace sg

using namespace sg;

extern "C" int swift_gpu_density_static(const swift_gpu_params* p, const float* pos_h, const float* vel_m,
                                        int64_t n, float min_cell_width, float* h_out, float* rho4,
                                        float* curl_div, uint32_t* ngb_count, int64_t* status_out,
                                        void* stream) {
  if (!p || n < 0 || !(min_cell_width >= 0.0f)) return SWIFT_GPU_ERR_ARG;
  if (n > kStaticN) return SWIFT_GPU_ERR_CAPACITY;
  auto aligned = [](const void* q, size_t a) { return q && ((uintptr_t)q % a) == 0; };
  if (n > 0 && (!aligned(pos_h, 16) || !aligned(vel_m, 16) || !aligned(h_out, 4) || !aligned(rho4, 16) ||
                !aligned(curl_div, 16) || (ngb_count && !aligned(ngb_count, 4))))
    return SWIFT_GPU_ERR_ARG;
  if (status_out && !aligned(status_out, 8)) return SWIFT_GPU_ERR_ARG;

  Ctx c;  // on the stack: no host allocation either
  if (phys_from(p, &c.phys) != SWIFT_GPU_OK) return SWIFT_GPU_ERR_ARG;
  c.params = *p;
  if (c.params.flags & (SWIFT_GPU_PLAIN | SWIFT_GPU_ADAPTIVE)) return SWIFT_GPU_ERR_ARG;
  if (cudaGetDevice(&c.device) != cudaSuccess || c.device < 0 || c.device >= kMaxDevices) return SWIFT_GPU_ERR_CUDA;
  if (cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, c.device) != cudaSuccess)
    return SWIFT_GPU_ERR_CUDA;
  // one-time set-up on this device (the device must be current)
  if (!g_scratch_addr[c.device]) {
    void* addr = nullptr;
    if (cudaGetSymbolAddress(&addr, g_static_scratch) != cudaSuccess || !addr) return SWIFT_GPU_ERR_CUDA;
    g_scratch_addr[c.device] = addr;
  }
  unsigned char* base = static_cast<unsigned char*>(g_scratch_addr[c.device]);
  auto at = [base](size_t off) { return static_cast<void*>(base + off); };

  c.n_max = kStaticN;
  c.nc_cap = static_nc_cap();
  int bits = 0;
  while (((int64_t)1 << bits) < kStaticCells) ++bits;
  c.max_key_bits = bits;
  c.max_passes = kStaticMaxPasses;
  c.red_blocks = c.num_sms * 32;
  c.tuning.threads_per_block = 256;
  c.tuning.max_lanes_per_particle = 8;
  c.tuning.blocks_per_sm = 0;
  c.d_status = static_cast<Status*>(at(kLayout.status));
  c.d_grid = static_cast<Grid*>(at(kLayout.grid));
  c.d_hmax_bits = static_cast<unsigned*>(at(kLayout.hmax));
  c.d_keys[0] = static_cast<unsigned*>(at(kLayout.keys0));
  c.d_keys[1] = static_cast<unsigned*>(at(kLayout.keys1));
  c.d_vals[0] = static_cast<unsigned*>(at(kLayout.vals0));
  c.d_vals[1] = static_cast<unsigned*>(at(kLayout.vals1));
  c.d_hist = static_cast<unsigned*>(at(kLayout.hist));
  c.d_scan_tmp = static_cast<unsigned*>(at(kLayout.scan_tmp));
  c.d_cell_start = static_cast<int*>(at(kLayout.cell_start));
  c.d_pos = static_cast<float4*>(at(kLayout.pos));
  c.d_vel = static_cast<float4*>(at(kLayout.vel));
  c.d_rho4 = static_cast<float4*>(at(kLayout.rho4));
  c.d_cd = static_cast<float4*>(at(kLayout.cd));
  c.d_h = static_cast<float*>(at(kLayout.h));
  c.d_bracket = static_cast<float2*>(at(kLayout.bracket));
  c.d_ngb = static_cast<unsigned*>(at(kLayout.ngb));
  c.d_act = static_cast<uint8_t*>(at(kLayout.act));
  c.d_items0 = static_cast<Item*>(at(kLayout.items0));
  c.d_items[0] = static_cast<Item*>(at(kLayout.items1));
  c.d_items[1] = static_cast<Item*>(at(kLayout.items2));
  c.d_plist0 = static_cast<int*>(at(kLayout.plist0));
  c.d_plist[0] = static_cast<int*>(at(kLayout.plist1));
  c.d_plist[1] = static_cast<int*>(at(kLayout.plist2));
  c.d_counters = static_cast<int*>(at(kLayout.counters));
  c.d_stats = static_cast<unsigned long long*>(at(kLayout.stats));

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the array keeps the previous call's contents: reset what must start at zero
  if (cudaMemsetAsync(c.d_status, 0, sizeof(Status), s) != cudaSuccess ||
      cudaMemsetAsync(c.d_stats, 0, sizeof(unsigned long long) * kStatCount, s) != cudaSuccess)
    return SWIFT_GPU_ERR_CUDA;
  int rc = build_cells_impl(&c, reinterpret_cast<const float4*>(pos_h), (int)n, min_cell_width, s);
  if (rc != SWIFT_GPU_OK) return rc;
  rc = density_impl(&c, reinterpret_cast<const float4*>(pos_h), reinterpret_cast<const float4*>(vel_m), nullptr,
                    h_out, reinterpret_cast<float4*>(rho4), reinterpret_cast<float4*>(curl_div), ngb_count, s);
  if (rc != SWIFT_GPU_OK) return rc;
  if (status_out) {
    k_static_status<<<1, 1, 0, s>>>(c.d_status, status_out);
    if (cudaGetLastError() != cudaSuccess) return SWIFT_GPU_ERR_CUDA;
  }
  return SWIFT_GPU_OK;
}
