// plain.cu -- the task granularity of the paper (Sec. 2.2.2, Fig. 3): one
// kernel launch per self task (a cell with itself) and per pair task (a cell
// with one of its 13 half-space neighbours, updating both cells), with the
// h iteration driven pass by pass from the host (the paper's CPU ghost task).
// It is the baseline the persistent path is measured against
// (SWIFT_GPU_PLAIN) and uses the same pair arithmetic (ops.cuh).
//
// Per-particle partial sums live in the context's work arrays between task
// launches; launches on one stream run in order, so tasks that share a cell
// never overlap.
#include <cuda_runtime.h>

#include <vector>

#include "common.cuh"
#include "internal.h"
#include "ops.cuh"

namespace sg {

constexpr int kTaskThreads = 64;

// Accumulator field f of particle k in the context's work arrays (16 floats per particle).
struct Acc {
  float* base;
  int n;
  __device__ __forceinline__ float& at(int f, int k) const { return base[(size_t)f * n + k]; }
};

struct PlainArgs {
  const float4* pos;
  const float4* vel;
  const float4* ga;
  const float4* gb;
  const float* h;       // density: h during the iteration
  const uint8_t* need;  // particles still computed in this pass
  Acc acc;
  float Lmax;
  float kg, knorm;
  int kernel;
};

struct Task {
  int a0, a1, b0, b1;
  unsigned code_ab, code_ba;
  int self;
};

// --------------------------------------------------------------- density
__device__ __forceinline__ void dens_acc_load(DensOp::I& I, const Acc& A, int k) {
  I.ns = A.at(0, k); I.nc = A.at(1, k); I.rs = A.at(2, k); I.rc = A.at(3, k); I.dn = A.at(4, k);
  I.dr = A.at(5, k); I.div = A.at(6, k); I.cx = A.at(7, k); I.cy = A.at(8, k); I.cz = A.at(9, k);
  I.count = __float_as_uint(A.at(10, k));
}
__device__ __forceinline__ void dens_acc_store(const DensOp::I& I, const Acc& A, int k) {
  A.at(0, k) = I.ns; A.at(1, k) = I.nc; A.at(2, k) = I.rs; A.at(3, k) = I.rc; A.at(4, k) = I.dn;
  A.at(5, k) = I.dr; A.at(6, k) = I.div; A.at(7, k) = I.cx; A.at(8, k) = I.cy; A.at(9, k) = I.cz;
  A.at(10, k) = __uint_as_float(I.count);
}

template <class Op>
__device__ __forceinline__ void task_side(const Op& op, typename Op::I& I, const float4* __restrict__ pos, int j0,
                                          int j1, unsigned code) {
  for (int j = j0; j < j1; ++j) {
    const float4 pj = pos[j];
    float xj = pj.x, yj = pj.y, zj = pj.z;
    shift_j(code, op.L, xj, yj, zj);
    const float dx = I.x - xj, dy = I.y - yj, dz = I.z - zj;
    if (op.candidate(I, r2_of(dx, dy, dz), op.stage_w(pj.w))) op.interact(I, j, code);
  }
}

__global__ void k_plain_dens(PlainArgs a, DensOp op, Task t) {
  const int na = t.a1 - t.a0, nb = t.self ? 0 : t.b1 - t.b0;
  for (int q = threadIdx.x; q < na + nb; q += blockDim.x) {
    const bool sideA = q < na;
    const int k = sideA ? t.a0 + q : t.b0 + (q - na);
    if (!a.need[k]) continue;
    DensOp::I I;
    const float4 p = a.pos[k];
    const float4 v = a.vel[k];
    I.x = p.x; I.y = p.y; I.z = p.z;
    dens_set_h(I, a.h[k], a.kg, a.knorm, a.Lmax);
    I.vx = v.x; I.vy = v.y; I.vz = v.z;
    I.k = k;
    dens_acc_load(I, a.acc, k);
    if (t.self) task_side(op, I, a.pos, t.a0, t.a1, 0u);
    else if (sideA) task_side(op, I, a.pos, t.b0, t.b1, t.code_ab);
    else task_side(op, I, a.pos, t.a0, t.a1, t.code_ba);
    dens_acc_store(I, a.acc, k);
  }
}

struct PlainDensState {
  const unsigned* perm;
  int n;
  Phys ph;
  Grid* grid;
  const float4* pos_in;
  const float4* vel_in;
  const uint8_t* active;
  float* h_out;
  float4* rho4_io;
  float4* cd_io;
  unsigned* ngb_out;
  float4* pos;
  float4* vel;
  float* h;
  float2* bracket;
  float4* rho4;
  float4* cd;
  unsigned* ngb;
  uint8_t* act;
  uint8_t* need;
  int* remaining;
  Status* st;
  unsigned long long* stats;
  Acc acc;
};

__global__ void k_plain_dens_prologue(PlainDensState s) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < s.n; k += gridDim.x * blockDim.x) {
    const unsigned src = s.perm[k];
    const float4 p = wrap_pos(s.pos_in[src], s.ph.L);
    s.pos[k] = p;
    s.vel[k] = s.vel_in[src];
    s.h[k] = p.w;
    const uint8_t act = s.active ? (s.active[src] != 0) : 1;
    s.act[k] = act;
    s.need[k] = act;
    s.bracket[k] = make_float2(0.0f, __int_as_float(0x7f800000));
    if (!act) {
      s.rho4[k] = s.rho4_io[src];
      s.cd[k] = s.cd_io[src];
      s.ngb[k] = s.ngb_out ? s.ngb_out[src] : 0u;
    }
  }
}

// The host's ghost task for the h iteration: one Newton step per particle.
__global__ void k_plain_newton(PlainDensState s, int last, int fixed_h) {
  const Grid g = *s.grid;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < s.n; k += gridDim.x * blockDim.x) {
    if (!s.need[k]) continue;
    const Acc& A = s.acc;
    const float ns = A.at(0, k), nc = A.at(1, k), rs = A.at(2, k), rc = A.at(3, k), dn = A.at(4, k);
    const float dr = A.at(5, k), dv = A.at(6, k), cx = A.at(7, k), cy = A.at(8, k), cz = A.at(9, k);
    const unsigned count = __float_as_uint(A.at(10, k));
    atomicAdd(&s.stats[kStatInterDens], (unsigned long long)count);
    const float h = s.h[k];
    float2 br = s.bracket[k];
    float hn = h;
    int flag = 0;
    if (!fixed_h && newton_step(h, ns, nc, dn, br.x, br.y, g.hcap, cell_cap_flag(g), s.ph, last != 0, hn, flag)) {
      s.h[k] = hn;
      s.bracket[k] = br;
      atomicAdd(s.remaining, 1);
    } else {
      const float rho = rs + rc;
      const float invh = 1.0f / h;
      s.rho4[k] = make_float4(rho, -dr * invh, ns + nc, -dn * invh);
      const float ir = 1.0f / rho;
      s.cd[k] = make_float4(cx * ir, cy * ir, cz * ir, dv * ir);
      s.ngb[k] = count;
      s.need[k] = 0;
      if (flag) set_error(s.st, flag);
    }
  }
}

__global__ void k_plain_dens_epilogue(PlainDensState s) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < s.n; k += gridDim.x * blockDim.x) {
    const unsigned dst = s.perm[k];
    const float h = s.h[k];
    s.pos[k].w = h;
    s.h_out[dst] = h;
    if (s.act[k]) {
      s.rho4_io[dst] = s.rho4[k];
      s.cd_io[dst] = s.cd[k];
      if (s.ngb_out) s.ngb_out[dst] = s.ngb[k];
    }
  }
}

// -------------------------------------------------------- gradient, force
__global__ void k_plain_grad(PlainArgs a, GradOp op, Task t) {
  const int na = t.a1 - t.a0, nb = t.self ? 0 : t.b1 - t.b0;
  for (int q = threadIdx.x; q < na + nb; q += blockDim.x) {
    const bool sideA = q < na;
    const int k = sideA ? t.a0 + q : t.b0 + (q - na);
    if (!a.need[k]) continue;
    GradOp::I I;
    const float4 p = a.pos[k];
    const float4 v = a.vel[k];
    I.x = p.x; I.y = p.y; I.z = p.z; I.h = p.w;
    const float H = a.kg * p.w;
    const float b = band_of(H, a.Lmax);
    I.H2lo = H * H - b;
    I.H2hi = H * H + b;
    I.invH = 1.0f / H;
    I.c4 = a.knorm * I.invH * I.invH * I.invH * I.invH;
    I.vx = v.x; I.vy = v.y; I.vz = v.z;
    I.c = a.ga[k].w;
    I.u = a.gb[k].w;
    I.k = k;
    I.vsig = a.acc.at(0, k);
    I.lap = a.acc.at(1, k);
    I.count = __float_as_uint(a.acc.at(2, k));
    if (t.self) task_side(op, I, a.pos, t.a0, t.a1, 0u);
    else if (sideA) task_side(op, I, a.pos, t.b0, t.b1, t.code_ab);
    else task_side(op, I, a.pos, t.a0, t.a1, t.code_ba);
    a.acc.at(0, k) = I.vsig;
    a.acc.at(1, k) = I.lap;
    a.acc.at(2, k) = __uint_as_float(I.count);
  }
}

__global__ void k_plain_force(PlainArgs a, ForceOp op, Task t) {
  const int na = t.a1 - t.a0, nb = t.self ? 0 : t.b1 - t.b0;
  for (int q = threadIdx.x; q < na + nb; q += blockDim.x) {
    const bool sideA = q < na;
    const int k = sideA ? t.a0 + q : t.b0 + (q - na);
    if (!a.need[k]) continue;
    ForceOp::I I;
    const float4 p = a.pos[k];
    const float4 v = a.vel[k];
    const float4 gi = a.ga[k];
    const float4 bi = a.gb[k];
    I.x = p.x; I.y = p.y; I.z = p.z; I.h = p.w;
    const float H = a.kg * p.w;
    const float b = band_of(H, a.Lmax);
    I.H2lo = H * H - b;
    I.H2hi = H * H + b;
    I.invH = 1.0f / H;
    I.c4 = a.knorm * I.invH * I.invH * I.invH * I.invH;
    I.vx = v.x; I.vy = v.y; I.vz = v.z;
    I.A = gi.x; I.f = gi.y; I.rho = gi.z; I.c = gi.w;
    I.B = bi.x; I.av = bi.y; I.acP = bi.z; I.u = bi.w;
    I.P = op.gm1 * gi.z * bi.w;
    I.k = k;
    I.axs = a.acc.at(0, k); I.axc = a.acc.at(1, k); I.ays = a.acc.at(2, k); I.ayc = a.acc.at(3, k);
    I.azs = a.acc.at(4, k); I.azc = a.acc.at(5, k); I.dus = a.acc.at(6, k); I.duc = a.acc.at(7, k);
    I.dh = a.acc.at(8, k);
    I.count = __float_as_uint(a.acc.at(9, k));
    if (t.self) task_side(op, I, a.pos, t.a0, t.a1, 0u);
    else if (sideA) task_side(op, I, a.pos, t.b0, t.b1, t.code_ab);
    else task_side(op, I, a.pos, t.a0, t.a1, t.code_ba);
    a.acc.at(0, k) = I.axs; a.acc.at(1, k) = I.axc; a.acc.at(2, k) = I.ays; a.acc.at(3, k) = I.ayc;
    a.acc.at(4, k) = I.azs; a.acc.at(5, k) = I.azc; a.acc.at(6, k) = I.dus; a.acc.at(7, k) = I.duc;
    a.acc.at(8, k) = I.dh;
    a.acc.at(9, k) = __uint_as_float(I.count);
  }
}

__global__ void k_plain_grad_init(int n, const float4* __restrict__ ga, Acc acc) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    acc.at(0, k) = 2.0f * ga[k].w;  // the particle itself: mu = 0
    acc.at(1, k) = 0.0f;
    acc.at(2, k) = 0.0f;
  }
}

__global__ void k_plain_grad_out(int n, const uint8_t* __restrict__ need, const unsigned* __restrict__ perm, Acc acc,
                                 float2* __restrict__ out, unsigned long long* stats) {
  unsigned cnt = 0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    if (!need[k]) continue;
    out[perm[k]] = make_float2(acc.at(0, k), 2.0f * acc.at(1, k));
    cnt += __float_as_uint(acc.at(2, k));
  }
  atomicAdd(&stats[kStatInterGrad], (unsigned long long)cnt);
}

__global__ void k_plain_force_out(int n, const uint8_t* __restrict__ need, const unsigned* __restrict__ perm,
                                  const float4* __restrict__ vel, const float4* __restrict__ ga,
                                  const float4* __restrict__ pos, Acc acc, float4* __restrict__ out,
                                  float* __restrict__ dhdt, double* __restrict__ red_partial,
                                  unsigned long long* stats) {
  __shared__ double red[8][8];
  double s8[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    if (!need[k]) continue;
    const float ax = acc.at(0, k) + acc.at(1, k), ay = acc.at(2, k) + acc.at(3, k);
    const float az = acc.at(4, k) + acc.at(5, k), du = acc.at(6, k) + acc.at(7, k);
    const unsigned dst = perm[k];
    out[dst] = make_float4(ax, ay, az, du);
    const float4 gi = ga[k];
    const float h = pos[k].w;
    if (dhdt) dhdt[dst] = -(h / (3.0f * gi.z)) * gi.y * acc.at(8, k);
    const float4 v = vel[k];
    const float m = v.w;
    const float mx = m * ax, my = m * ay, mz = m * az;
    const float va = fmaf(v.z, az, fmaf(v.y, ay, v.x * ax));
    s8[0] += (double)mx;
    s8[1] += (double)my;
    s8[2] += (double)mz;
    s8[3] += (double)(m * va) + (double)(m * du);
    s8[4] += (double)sqrtf(fmaf(mz, mz, fmaf(my, my, mx * mx)));
    s8[5] += (double)(m * fabsf(va)) + (double)(m * fabsf(du));
    s8[6] += (double)(m * du);
    s8[7] += (double)__float_as_uint(acc.at(9, k));
  }
  const unsigned lane = threadIdx.x & 31u;
  for (int q = 0; q < 8; ++q) {
    double x = s8[q];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) red[threadIdx.x >> 5][q] = x;
  }
  __syncthreads();
  if (threadIdx.x < 8) {
    double x = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) x += red[w][threadIdx.x];
    red_partial[blockIdx.x * 8 + threadIdx.x] = x;
    if (threadIdx.x == 7) atomicAdd(&stats[kStatInterForce], (unsigned long long)x);
  }
}

// ----------------------------------------------------------------- hosts
// The self and pair tasks of the current grid (host copy of the cell starts).
static int make_tasks(Ctx* c, cudaStream_t s, std::vector<Task>& tasks) {
  Grid g;
  if (cudaMemcpyAsync(&g, c->d_grid, sizeof(Grid), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return SWIFT_GPU_ERR_CUDA;
  std::vector<int> cs((size_t)g.ncells + 1);
  if (cudaMemcpyAsync(cs.data(), c->d_cell_start, sizeof(int) * cs.size(), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return SWIFT_GPU_ERR_CUDA;
  const int nx = g.nc[0], ny = g.nc[1], nz = g.nc[2];
  tasks.clear();
  for (int cz = 0; cz < nz; ++cz)
    for (int cy = 0; cy < ny; ++cy)
      for (int cx = 0; cx < nx; ++cx) {
        const int a = cx + nx * (cy + ny * cz);
        if (cs[a + 1] == cs[a]) continue;
        tasks.push_back(Task{cs[a], cs[a + 1], 0, 0, 0u, 0u, 1});
        for (int dz = -1; dz <= 1; ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              // the 13 half-space neighbours: each unordered pair once
              if (dz < 0 || (dz == 0 && (dy < 0 || (dy == 0 && dx <= 0)))) continue;
              int x = cx + dx, y = cy + dy, z = cz + dz;
              unsigned ab = 0;
              if (x < 0) { x += nx; ab |= 2u; } else if (x >= nx) { x -= nx; ab |= 1u; }
              if (y < 0) { y += ny; ab |= 8u; } else if (y >= ny) { y -= ny; ab |= 4u; }
              if (z < 0) { z += nz; ab |= 32u; } else if (z >= nz) { z -= nz; ab |= 16u; }
              const int b = x + nx * (y + ny * z);
              if (cs[b + 1] == cs[b]) continue;
              // B's particles seen from A shift by ab; A's seen from B shift the opposite way
              const unsigned ba = ((ab & 0x15u) << 1) | ((ab & 0x2Au) >> 1);
              tasks.push_back(Task{cs[a], cs[a + 1], cs[b], cs[b + 1], ab, ba, 0});
            }
      }
  return SWIFT_GPU_OK;
}

static PlainArgs plain_args(Ctx* c, float Lmax) {
  PlainArgs a;
  a.pos = c->d_pos;
  a.vel = c->d_vel;
  a.ga = c->d_ga;
  a.gb = c->d_gb;
  a.h = c->d_h;
  a.need = c->d_act;
  a.acc = Acc{reinterpret_cast<float*>(c->d_scratch4[0]), (int)c->n_max};
  a.Lmax = Lmax;
  a.kg = c->phys.kg;
  a.knorm = c->phys.knorm;
  a.kernel = c->phys.kernel;
  return a;
}

static float lmax_of(const Phys& ph) { return fmaxf(ph.L[0], fmaxf(ph.L[1], ph.L[2])); }

// The work arrays d_scratch4[0..3] are one block of 4 n_max float4, viewed
// here as [16][n_max] floats: accumulator f of particle k at [f][k].
static void zero_acc(Ctx* c, cudaStream_t s) {
  cudaMemsetAsync(c->d_scratch4[0], 0, sizeof(float4) * 4 * (size_t)c->n_max, s);
}

int plain_density_impl(Ctx* c, const float4* pos_in, const float4* vel_in, const uint8_t* active, float* h_out,
                       float4* rho4, float4* cd, uint32_t* ngb, cudaStream_t s) {
  PlainDensState st;
  st.perm = c->d_vals[c->sorted_buf];
  st.n = c->n;
  st.ph = c->phys;
  st.grid = c->d_grid;
  st.pos_in = pos_in;
  st.vel_in = vel_in;
  st.active = active;
  st.h_out = h_out;
  st.rho4_io = rho4;
  st.cd_io = cd;
  st.ngb_out = ngb;
  st.pos = c->d_pos;
  st.vel = c->d_vel;
  st.h = c->d_h;
  st.bracket = c->d_bracket;
  st.rho4 = c->d_rho4;
  st.cd = c->d_cd;
  st.ngb = c->d_ngb;
  st.act = c->d_plain_act;
  st.need = c->d_act;
  st.remaining = c->d_counters + kCtrPerPass * (c->max_passes + 1) + 3;
  st.st = c->d_status;
  st.stats = c->d_stats;
  st.acc = Acc{reinterpret_cast<float*>(c->d_scratch4[0]), (int)c->n_max};
  c->all_active = active == nullptr;
  c->lpp_lists = 0;  // no kept candidate lists from this path
  if (c->n == 0) return SWIFT_GPU_OK;
  const int nb = min((c->n + 255) / 256, c->num_sms * 8);
  k_plain_dens_prologue<<<nb, 256, 0, s>>>(st);
  c->launches++;
  std::vector<Task> tasks;
  int rc = make_tasks(c, s, tasks);
  if (rc != SWIFT_GPU_OK) return rc;
  DensOp op;
  op.pos = c->d_pos;
  op.vel = c->d_vel;
  op.L[0] = c->phys.L[0]; op.L[1] = c->phys.L[1]; op.L[2] = c->phys.L[2];
  op.kg = c->phys.kg;
  op.kernel = c->phys.kernel;
  op.knorm = c->phys.knorm;
  op.compensated = c->phys.compensated;
  PlainArgs a = plain_args(c, lmax_of(c->phys));
  a.acc = st.acc;
  const int max_pass = (c->params.flags & SWIFT_GPU_NO_H_ITER) ? 1 : c->phys.max_iter;
  int pass = 0;
  int remaining = 0;
  for (; pass < max_pass; ++pass) {
    zero_acc(c, s);
    for (const Task& t : tasks) k_plain_dens<<<1, kTaskThreads, 0, s>>>(a, op, t);
    c->launches += tasks.size();
    cudaMemsetAsync(st.remaining, 0, sizeof(int), s);
    k_plain_newton<<<nb, 256, 0, s>>>(st, pass == max_pass - 1, (c->params.flags & SWIFT_GPU_NO_H_ITER) ? 1 : 0);
    c->launches++;
    if (cudaMemcpyAsync(&remaining, st.remaining, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return SWIFT_GPU_ERR_CUDA;
    if (remaining == 0) {
      ++pass;
      break;
    }
  }
  k_plain_dens_epilogue<<<nb, 256, 0, s>>>(st);
  c->launches++;
  // the active flags stay in d_act for gradient and force
  cudaMemcpyAsync(c->d_act, c->d_plain_act, (size_t)c->n, cudaMemcpyDeviceToDevice, s);
  unsigned long long p = (unsigned long long)pass;
  cudaMemcpyAsync(&c->d_stats[kStatPasses], &p, sizeof(p), cudaMemcpyHostToDevice, s);
  cudaStreamSynchronize(s);
  return cudaGetLastError() == cudaSuccess ? SWIFT_GPU_OK : SWIFT_GPU_ERR_CUDA;
}

int plain_gradient_impl(Ctx* c, float2* out, cudaStream_t s) {
  if (c->n == 0) return SWIFT_GPU_OK;
  std::vector<Task> tasks;
  int rc = make_tasks(c, s, tasks);
  if (rc != SWIFT_GPU_OK) return rc;
  GradOp op;
  op.pos = c->d_pos; op.vel = c->d_vel; op.ga = c->d_ga; op.gb = c->d_gb;
  op.L[0] = c->phys.L[0]; op.L[1] = c->phys.L[1]; op.L[2] = c->phys.L[2];
  op.kg = c->phys.kg;
  op.kernel = c->phys.kernel;
  op.knorm = c->phys.knorm;
  op.beta = c->phys.beta_v;
  PlainArgs a = plain_args(c, lmax_of(c->phys));
  a.acc = Acc{reinterpret_cast<float*>(c->d_scratch4[0]), (int)c->n_max};
  const int nb = min((c->n + 255) / 256, c->num_sms * 8);
  k_plain_grad_init<<<nb, 256, 0, s>>>(c->n, c->d_ga, a.acc);
  for (const Task& t : tasks) k_plain_grad<<<1, kTaskThreads, 0, s>>>(a, op, t);
  k_plain_grad_out<<<nb, 256, 0, s>>>(c->n, c->d_act, c->d_vals[c->sorted_buf], a.acc, out, c->d_stats);
  c->launches += tasks.size() + 2;
  return cudaGetLastError() == cudaSuccess ? SWIFT_GPU_OK : SWIFT_GPU_ERR_CUDA;
}

int plain_force_impl(Ctx* c, float4* out, float* dhdt, double* reductions, cudaStream_t s) {
  if (c->n == 0) return SWIFT_GPU_OK;
  std::vector<Task> tasks;
  int rc = make_tasks(c, s, tasks);
  if (rc != SWIFT_GPU_OK) return rc;
  ForceOp op;
  op.pos = c->d_pos; op.vel = c->d_vel; op.ga = c->d_ga; op.gb = c->d_gb;
  op.L[0] = c->phys.L[0]; op.L[1] = c->phys.L[1]; op.L[2] = c->phys.L[2];
  op.Lmax = lmax_of(c->phys);
  op.kg = c->phys.kg;
  op.kernel = c->phys.kernel;
  op.knorm = c->phys.knorm;
  op.beta = c->phys.beta_v;
  op.gm1 = c->phys.gamma_eos - 1.0f;
  op.compensated = c->phys.compensated;
  PlainArgs a = plain_args(c, op.Lmax);
  a.acc = Acc{reinterpret_cast<float*>(c->d_scratch4[0]), (int)c->n_max};
  zero_acc(c, s);
  for (const Task& t : tasks) k_plain_force<<<1, kTaskThreads, 0, s>>>(a, op, t);
  const int nb = min(min((c->n + 255) / 256, c->num_sms * 8), c->red_blocks);
  k_plain_force_out<<<nb, 256, 0, s>>>(c->n, c->d_act, c->d_vals[c->sorted_buf], c->d_vel, c->d_ga, c->d_pos, a.acc,
                                       out, dhdt, c->d_red_partial, c->d_stats);
  c->launches += tasks.size() + 1;
  if (reductions) reduce_partials(c, nb, reductions, s);
  return cudaGetLastError() == cudaSuccess ? SWIFT_GPU_OK : SWIFT_GPU_ERR_CUDA;
}

}  // namespace sg
