/*
 * swift_gpu.h -- C ABI of the B300 (sm_103a) SPH pair-interaction library.
 *
 * The library runs the hot path of the SWIFT SPH solver described in
 * "Task-parallelism in SWIFT for heterogeneous compute architectures"
 * (arXiv 2505.14538): the density loop with the Newton iteration on the
 * smoothing length (Sec. 2.1.2, Eqs. 2-6), the gradient loop (Sec. 2.1.3,
 * Eqs. 10-11) and the force loop (Sec. 2.1.4, Eqs. 7, 9-11, 16-20, 22), over
 * the self and pair interactions of a periodic grid of cubic cells no finer
 * than the kernel support (Sec. 2.2, Fig. 3). Everything runs as CUDA kernels
 * on one GPU; the caller owns every particle array, the library owns only the
 * opaque context (sorted copies, cell arrays, work lists, status word).
 *
 * Conventions shared by every call below:
 *  - All particle pointers are DEVICE pointers owned by the caller, contiguous,
 *    and aligned to their element size (16 bytes for float4, 8 for float2).
 *    They are indexed in the caller's particle order.
 *  - float4 layouts: pos_h = (x, y, z, h); vel_m = (vx, vy, vz, m). These
 *    mirror the packed particle records of Sec. 2.3.2.1 (float4 position and
 *    smoothing length, float4 velocity and mass) as structure-of-arrays.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream). Calls are asynchronous on that stream unless stated otherwise;
 *    device-side errors are recorded in the context's status word and read
 *    with swift_gpu_sync_status.
 *  - Return value: SWIFT_GPU_OK (0) or a negative SWIFT_GPU_ERR_* code for an
 *    error detected on the host (bad argument, call order, CUDA launch error).
 *    Nothing is thrown across the ABI.
 *  - Positions live in the periodic box [0, L)^3; positions outside are first
 *    wrapped into it in FP64 (x - L floor(x / L)), and everything (cell ids,
 *    distances by the minimum image) uses the wrapped position, rounded to FP32.
 */
#ifndef SWIFT_GPU_H
#define SWIFT_GPU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define SWIFT_GPU_OK 0
#define SWIFT_GPU_ERR_ARG (-1)               /* bad pointer, size, NaN/Inf position, h <= 0 */
#define SWIFT_GPU_ERR_ORDER (-2)             /* call before its prerequisite (see each call) */
#define SWIFT_GPU_ERR_CUDA (-3)              /* a CUDA runtime call failed */
#define SWIFT_GPU_ERR_H_NOT_CONVERGED (-4)   /* Newton on h hit max_iter; detail = count */
#define SWIFT_GPU_ERR_H_EXCEEDS_CELL (-5)    /* h wanted a support wider than a cell; detail = count */
#define SWIFT_GPU_ERR_TIMEOUT (-6)           /* a bounded device-side wait gave up */
#define SWIFT_GPU_ERR_NOMEM (-7)             /* device allocation failed */
#define SWIFT_GPU_ERR_CAPACITY (-8)          /* n exceeds the context's n_max */

/* swift_gpu_params.flags */
#define SWIFT_GPU_PLAIN 1         /* one kernel launch per self/pair cell task (the paper's task granularity,
                                     Sec. 2.2.2), h iteration driven from the host pass by pass; the baseline
                                     for the persistent path (no autotune, no force_backward) */
#define SWIFT_GPU_NO_H_ITER 2     /* density at the given h: no Newton iteration, no convergence status */
#define SWIFT_GPU_NO_COMPENSATION 4 /* plain FP32 sums instead of two-sum compensated rho, a, du/dt */
#define SWIFT_GPU_ADAPTIVE 8      /* adaptive leaves for clustered sets (the task recursion of Sec. 2.2.2 and
                                     Fig. 3c, which the paper's GPU path lacks, Sec. 4.4.4): each cell is split
                                     octree-wise into leaves of <= leaf_max particles and every loop scans, for
                                     the particles of a leaf, only the leaves whose bounding boxes come within
                                     the larger of the two leaves' supports (not with PLAIN) */

/* swift_gpu_params.kernel: the kernel shape W = C H^-3 w(r/H) (Sec. 2.1.1
 * names the cubic spline and the Wendland kernels). kernel_gamma should be
 * the shape's own H/h from the second-moment definition h = 2 sigma:
 * sqrt(30)/3 = 1.825742, sqrt(15)/2 = 1.936492, sqrt(78)/4 = 2.207940. */
#define SWIFT_GPU_KERNEL_CUBIC 0        /* cubic spline M4, C = 8/pi */
#define SWIFT_GPU_KERNEL_WENDLAND_C2 1  /* w = (1-q)^4 (1+4q), C = 21/(2 pi) */
#define SWIFT_GPU_KERNEL_WENDLAND_C4 2  /* w = (1-q)^6 (1+6q+35q^2/3), C = 495/(32 pi) */

typedef struct {
  float box[3];        /* periodic box edge lengths L (the box is [0,L)^3) */
  float gamma_eos;     /* adiabatic index gamma (Sec. 3.1: 5/3) */
  float eta;           /* resolution: the h iteration targets n = (eta/h)^3 (1.2348: ~48 neighbours) */
  float kernel_gamma;  /* H/h of the cubic-spline kernel (1.825742) */
  float alpha_v;       /* viscosity alpha, used when no per-particle array is given (Eq. 16) */
  float beta_v;        /* signal-velocity beta (Eq. 10; 3) */
  float alpha_c;       /* conduction alpha, used when no per-particle array is given (Eq. 20) */
  float h_tol;         /* Newton tolerance: |n - (eta/h)^3| <= h_tol (eta/h)^3 (Sec. 2.1.2: 1e-4) */
  int max_iter;        /* maximum Newton passes (>= 1) */
  float h_max;         /* cap on h; 0 = the largest h whose support fits in one cell */
  float cell_margin;   /* automatic cell width = (1 + cell_margin) * kernel_gamma * max h */
  int flags;           /* SWIFT_GPU_* flags above */
  int leaf_max;        /* ADAPTIVE: a node with more particles is split into its 8 octants (8..1024) */
  float leaf_margin;   /* ADAPTIVE: the h cap of a leaf is (1 + leaf_margin) * its largest h at the build;
                          >= 0.01, since a rebuild after a capped iteration lets h grow by this factor */
  int kernel;          /* SWIFT_GPU_KERNEL_*: kernel shape (every loop and the adjoint) */
} swift_gpu_params;

/* Work-distribution knobs (chosen by swift_gpu_autotune, or set by hand). */
typedef struct {
  int threads_per_block; /* must be 256 (reserved). The loop kernels run fixed blocks of 128
                            threads: four warps, each taking one cell or leaf item (or one group of
                            32 particles) at a time from the device queue, so four cells a block
                            are in flight; 64- and 256-thread blocks measured slower */
  int max_lanes_per_particle; /* 1, 2, 4, 8, 16 or 32: lanes that share one particle's neighbour scan;
                                 on the uniform grid 1 selects the lane-per-particle density call (a
                                 warp takes 32 particles, one a lane; group_collect says how they find
                                 their candidates) and 2..32 the cell items (a warp shares one cell's
                                 candidates); the gradient and force loops run one lane a particle
                                 over the density call's kept lists either way */
  int blocks_per_sm;     /* persistent blocks per SM (0 = occupancy maximum) */
  int wait_limit_us;     /* limit of each bounded device-side wait (the density launch's grid barrier):
                            0 = 5 s; negative = give up at once (fault injection: the call then reports
                            ERR_TIMEOUT, its outputs are undefined, the context stays usable) */
  int group_collect;     /* candidate search of the lane-per-particle density call:
                            SWIFT_GPU_COLLECT_ROWS (0): the warp's lanes test, in step, every particle of
                            the rows of cells their 27-cell neighbourhoods share (Sec. 2.2: self and pair
                            interactions of neighbouring cells), one broadcast load a candidate;
                            SWIFT_GPU_COLLECT_WINDOWS (1): each lane reads its own 26 neighbour cells
                            through windows along the 13 pair axes (sorted pair interactions, Sec. 2.2.2) */
} swift_gpu_tuning;

#define SWIFT_GPU_COLLECT_ROWS 0
#define SWIFT_GPU_COLLECT_WINDOWS 1

typedef struct {
  int64_t n;               /* particles of the last build */
  int32_t nc[3];           /* cells per axis */
  float cell_width[3];     /* cell edge lengths */
  float h_cap;             /* largest h whose support fits in a cell */
  int64_t n_cells;
  int64_t n_items;         /* work items (cell chunks of <= 32 active particles) */
  int32_t density_passes;  /* Newton passes run by the last density call */
  uint64_t interactions[3];/* pair interactions: density (full sums, every pass), gradient, force */
  uint64_t candidates[3];  /* candidate pairs tested by the neighbour scan, same loops */
  uint64_t launches;       /* kernel launches issued since the context was created */
  uint64_t h_iteration_pairs; /* pairs of the Newton steps on h that evaluate only Eqs. 5-6 */
  int64_t n_leaves;        /* ADAPTIVE: leaves of the last build (0 otherwise) */
  int64_t leaf_pairs;      /* ADAPTIVE: entries of the leaf neighbour lists (ordered leaf pairs) */
  int32_t tree_depth;      /* ADAPTIVE: deepest octree level holding a leaf (cells are level 0) */
} swift_gpu_info;

typedef struct swift_gpu_ctx swift_gpu_ctx;

/* Fill *p with the defaults (unit box, gamma 5/3, eta 1.2348, kernel_gamma
 * 1.825742, alpha_v 1, beta_v 3, alpha_c 1, h_tol 1e-4, max_iter 30, h_max 0,
 * cell_margin 0.05, flags 0, leaf_max 32, leaf_margin 0.1, kernel CUBIC). Host only; never fails. */
void swift_gpu_default_params(swift_gpu_params* p);

/* Create a context for up to n_max particles on the current CUDA device.
 * Allocates every device buffer the calls need, so no later call allocates:
 * about 0.3 KB per particle of sorted records, sums and work lists, plus the
 * cell arrays, and then by the grid it is created for:
 *   uniform grid (no ADAPTIVE): the store of the candidate lists the density
 *     call keeps for the gradient and force loops, W x 4 bytes a particle
 *     (W = 92 entries for the cubic spline, 128 Wendland C2, 160 Wendland C4),
 *     and the pair-axis replicas of the lane-per-particle density path, 208
 *     bytes a particle: 872 bytes a particle in all for the cubic spline;
 *   ADAPTIVE: the octree, the leaves and their neighbour lists instead, 719
 *     bytes a particle in all.
 * *ctx is owned by the caller and freed with swift_gpu_destroy. Errors:
 * ERR_ARG (null/invalid params, n_max < 1 or n_max >= 2^26: a list entry
 * holds a particle index in 26 bits), ERR_NOMEM, ERR_CUDA. */
int swift_gpu_create(swift_gpu_ctx** ctx, const swift_gpu_params* p, int64_t n_max);

/* Release every buffer of the context (synchronises the device). NULL is allowed. */
int swift_gpu_destroy(swift_gpu_ctx* ctx);

/* Replace the physics parameters (same rules as create). Host only. A
 * context created without ADAPTIVE holds no tree arrays: turning ADAPTIVE on
 * here is ERR_ARG. A kernel shape wider than the one the context was created
 * with leaves the kept-list store too small for its lists; the density call
 * then keeps none, and the gradient and force loops scan the cells. */
int swift_gpu_set_params(swift_gpu_ctx* ctx, const swift_gpu_params* p);

/* Build the cell grid and the particle order (paper Sec. 2.2: cubic cells,
 * self and pair tasks; the sort tasks of Sec. 2.2.2 left on the CPU there).
 * pos_h[n]: float4 (x, y, z, h), device. The cell width is the largest of
 * min_cell_width and (1 + cell_margin) * kernel_gamma * max_i h_i, rounded up
 * so an integer number nc >= 3 of cells spans each box edge; cell ids are
 * computed in FP64 (wrap into [0,L), floor(x nc / L), clamp) and particles are
 * stably sorted by cell id (ties keep the input order). Device-side errors:
 * ERR_ARG (NaN/Inf position, h <= 0), ERR_H_EXCEEDS_CELL (support wider than
 * L/3). Host errors: ERR_ARG, ERR_CAPACITY (n > n_max). n = 0 is allowed.
 * With SWIFT_GPU_ADAPTIVE the particles of a cell are ordered by the Morton
 * code of their position inside the cell (10 bits per axis, ties by input
 * order) and the cell tree of Sec. 2.2.2 is built on the device: a node with
 * more than leaf_max particles is split into its non-empty octants, down to
 * 10 levels below the cell; the rest are leaves. A leaf's h cap is
 * min(cell cap, (1 + leaf_margin) * its largest h); its neighbour list holds
 * every leaf (with periodic image) whose bounding box comes within the
 * larger of the two leaves' supports kernel_gamma * h_cap. Capacities:
 * 2 n_max tree nodes beyond the cells (a node that would exceed them stays a
 * leaf) and max(48 n_max, 2^22) list entries (a leaf whose list would end past them
 * scans the 27 neighbour cells of its cell instead); both keep results exact.
 * Where the lists lie in the store is unspecified; each list's order is
 * fixed by the tree, so results do not depend on it.
 * With ADAPTIVE at most 256 cells per axis are used. */
int swift_gpu_build_cells(swift_gpu_ctx* ctx, const float* pos_h, int64_t n, float min_cell_width,
                          void* stream);

/* Density loop with the Newton iteration on h (Sec. 2.1.2, Eqs. 2-6).
 * pos_h_in[n]: float4 (x, y, z, h) - the same positions as build_cells; h is
 *              the starting smoothing length.
 * vel_m[n]:    float4 (vx, vy, vz, m).
 * active[n]:   uint8, nonzero = compute this particle; NULL = all active.
 * Outputs (device, caller order):
 *   h_out[n]        final smoothing length (inactive: copied from pos_h_in.w)
 *   rho4[n]         float4 (rho, drho/dh, n, dn/dh) - the part_recv_d record of
 *                   Sec. 2.3.2.3 (Eq. 2, 5, 6)
 *   curl_div[n]     float4 (curl v x, y, z, div v) (Eqs. 3-4, differenced form)
 *   ngb_count[n]    uint32 neighbours j != i with r_ij < H_i (may be NULL)
 * For inactive particles rho4 and curl_div are INPUTS: they must hold that
 * particle's last values, which the gradient and force loops read.
 * Each active particle iterates h <- h - F/F' on F = n - (eta/h)^3 until
 * |F| <= h_tol (eta/h)^3, at most max_iter steps; all outputs belong to the
 * final h. Runs as ONE persistent cooperative launch: one neighbour scan
 * collects every candidate within the largest support a cell allows and the
 * steps run over those lists; particles whose candidates do not fit take
 * further scan passes. Device-side status:
 * ERR_H_NOT_CONVERGED / ERR_H_EXCEEDS_CELL with detail = number of particles
 * (outputs are still written at their last h), ERR_TIMEOUT.
 * Requires build_cells (ERR_ORDER otherwise). */
int swift_gpu_density(swift_gpu_ctx* ctx, const float* pos_h_in, const float* vel_m, const uint8_t* active,
                      float* h_out, float* rho4, float* curl_div, uint32_t* ngb_count, void* stream);

/* Gradient loop (Sec. 2.1.3): per active i, over j with r_ij < H_i,
 * v_sig,max = max_j (c_i + c_j - beta mu_ij) (Eqs. 10-11, j = i included) and
 * the Laplacian of u, 2 sum_j (m_j/rho_j)(u_i - u_j) (dW/dr)/r.
 * u[n]: internal energy (device, caller order). vsig_lapu[n]: float2 output.
 * Also evaluates the per-particle ghost step for all particles:
 * f = 1/Omega (Eq. 8), P = (gamma-1) rho u, c = sqrt(gamma (gamma-1) u),
 * Balsara B. Requires density (ERR_ORDER otherwise). */
int swift_gpu_gradient(swift_gpu_ctx* ctx, const float* u, float* vsig_lapu, void* stream);

/* Force loop (Sec. 2.1.4): per active i over j with r_ij < max(H_i, H_j):
 * pressure acceleration (Eq. 17), du/dt (Eq. 18), artificial viscosity
 * (Eqs. 7, 9-11, 16) with its heating term, artificial conduction
 * (Eqs. 19, 20, 22) and dh/dt = -(h/(3 rho)) f sum_j m_j v_ij . grad W(h_i).
 * u[n] internal energy; alpha_v_i[n], alpha_c_i[n]: per-particle coefficients
 * or NULL for the constants in the parameters.
 * accel_dudt[n]: float4 (a_x, a_y, a_z, du/dt) output; dh_dt[n] may be NULL.
 * reductions: NULL or a DEVICE array of 8 doubles receiving FP64 sums over
 * active particles: [0..2] sum m a, [3] sum m (v.a + du/dt), [4] sum |m a|,
 * [5] sum m (|v.a| + |du/dt|), [6] sum m du/dt, [7] number of interactions.
 * Requires density (ERR_ORDER otherwise); evaluates the ghost step itself. */
int swift_gpu_force(swift_gpu_ctx* ctx, const float* u, const float* alpha_v_i, const float* alpha_c_i,
                    float* accel_dudt, float* dh_dt, double* reductions, void* stream);

/* Gradient and force loops in one pass over the pairs (an optimisation, not
 * in the paper): the outputs of swift_gpu_gradient followed by
 * swift_gpu_force with the same u, alpha_v_i, alpha_c_i (the gradient loop
 * reads no alpha). The force pair set r < max(H_i, H_j) contains the
 * gradient's r < H_i, so each pair is evaluated once for both, in the same
 * order as the two calls: vsig_lapu is bitwise the same; accel_dudt and
 * dh_dt agree to a few FP32 roundings (multiply-adds may be fused
 * differently). Arguments as in the two calls; requires density (ERR_ORDER
 * otherwise). */
int swift_gpu_gradient_force(swift_gpu_ctx* ctx, const float* u, const float* alpha_v_i, const float* alpha_c_i,
                             float* vsig_lapu, float* accel_dudt, float* dh_dt, double* reductions, void* stream);

/* Adjoint of density + ghost + force (not in the paper): given
 * grad_accel_dudt[n] = float4 (dL/da_x, dL/da_y, dL/da_z, dL/d(du/dt)) for a
 * scalar loss L of the outputs of the last swift_gpu_force call, write
 * grad_x[n] (float4, w unused), grad_v[n] (float4, w unused), grad_u[n].
 * h_mode 0: h held at the values of the last density call.
 * h_mode 1: each h_i is the root of the h iteration, F_i = n_i(x, h_i) -
 * (eta/h_i)^3 = 0 (Sec. 2.1.2), so h moves with x: by the implicit function
 * theorem grad_x gains -sum_i lambda_i dn_i/dx with lambda_i = (dL/dh_i at
 * fixed x) / (dn_i/dh_i + 3 eta^3 / h_i^4); dL/dh comes from the same two
 * passes and a third gather adds the term. Exact at the root: the density
 * call should have converged (a tighter h_tol makes it closer); ERR_ARG with
 * SWIFT_GPU_NO_H_ITER (h is then an input, not a root).
 * Two gather passes, each scanning the neighbour cells (or leaves) as the
 * cell-item loops do: the force pair terms are reversed in both orientations
 * of every pair, the ghost step is reversed per particle, and the adjoints of
 * each particle's density sums are carried back through both particles' sums.
 * The candidates are found again by the scan, not read from a stored pair
 * list; the per-particle sums of the forward calls are reused. grad_x and
 * grad_v are float4 with w = 0. Requires force (ERR_ORDER otherwise); every
 * particle must have been active (ERR_ARG otherwise). */
int swift_gpu_force_backward(swift_gpu_ctx* ctx, const float* grad_accel_dudt, float* grad_x, float* grad_v,
                             float* grad_u, int h_mode, void* stream);

/* Replace the density results of the particles marked in mask[n] (uint8,
 * caller order, device) with values computed elsewhere: h_in[n] (also the h
 * the later loops take for them), rho4[n] and curl_div[n] (float4, as
 * swift_gpu_density writes them). For a domain decomposition over several
 * GPUs (SWIFT keeps its CPU code's domain decomposition over MPI ranks with
 * the GPU off-loading, Sec. 5): the ghost-layer particles of a rank are
 * inactive in its density call, their owners compute them, and this call puts
 * the owners' results in place before swift_gpu_gradient / swift_gpu_force /
 * swift_gpu_gradient_force. The marked
 * particles must have been inactive in the density call, and their h within
 * the cell cap (device-side ERR_H_EXCEEDS_CELL otherwise). Requires density
 * (ERR_ORDER otherwise; also with SWIFT_GPU_PLAIN). Asynchronous. */
int swift_gpu_set_inactive(swift_gpu_ctx* ctx, const uint8_t* mask, const float* h_in, const float* rho4,
                           const float* curl_div, void* stream);

/* Wait for all work on the device (the calls may have been captured in a CUDA
 * graph and replayed on any stream) and read the device status word:
 * *status = first device-side error code (0 = none), *detail = its count or
 * index. Clears the status word. Blocking. */
int swift_gpu_sync_status(swift_gpu_ctx* ctx, int* status, int64_t* detail);

/* Fill *info (blocking: waits for all work on the device first, as
 * swift_gpu_sync_status does). */
int swift_gpu_get_info(swift_gpu_ctx* ctx, swift_gpu_info* info);

/* Copy the cell id of every particle (caller order) and the sort permutation
 * (sorted position k -> caller index perm[k]) of the last build into device
 * arrays cell_id[n], perm[n] (either may be NULL). Asynchronous. */
int swift_gpu_get_cells(swift_gpu_ctx* ctx, uint32_t* cell_id, uint32_t* perm, void* stream);

/* ADAPTIVE only: copy the leaves of the last build into device arrays:
 * range[2 * l], range[2 * l + 1] = first and one-past-last SORTED position of
 * leaf l (sorted positions are those of swift_gpu_get_cells' perm),
 * h_cap[l] = the largest h its particles may take before the h iteration
 * reports ERR_H_EXCEEDS_CELL, nbr_count[l] = length of its neighbour-leaf
 * list (itself included), or -1 when the leaf has no list (the list store
 * was full, or the tree walk ran out of its stack) and its particles scan
 * the 27 neighbour cells of their cell instead. Any pointer may be NULL. Leaves l < max_leaves are
 * copied; the leaf count is swift_gpu_info.n_leaves. The order of the leaves
 * is unspecified. Errors: ERR_ORDER (no adaptive build), ERR_ARG. Asynchronous. */
int swift_gpu_get_leaves(swift_gpu_ctx* ctx, int32_t* range, float* h_cap, int32_t* nbr_count, int64_t max_leaves,
                         void* stream);

/* Read / set the work-distribution knobs. */
int swift_gpu_get_tuning(swift_gpu_ctx* ctx, swift_gpu_tuning* t);
int swift_gpu_set_tuning(swift_gpu_ctx* ctx, const swift_gpu_tuning* t);

/* Time the given loop (0 density, 1 gradient, 2 force, 3 gradient + force,
 * 4 the whole step after the cell build: density, then gradient + force)
 * on the data of the last calls for each candidate tuning (lanes per
 * particle 1..32, blocks per SM 0..2) and keep the fastest; the setting is
 * shared by all loops. The lanes per particle also choose the density
 * call's engine on the uniform grid (1: one lane a particle with pair-axis
 * windows; 2..32: cell items), whose kept lists the gradient and force loops
 * read, so for loops 1-3 each candidate first re-runs the density call
 * (untimed). Requires force (or gradient + force) to have run once; loops 1,
 * 3 and 4 require a gradient output of a previous call. Blocking. The loop is
 * run once more with the chosen setting, so its outputs (in the arrays of
 * the last calls) are those of that setting: the same sums as before up to
 * the FP32 summation order. */
int swift_gpu_autotune(swift_gpu_ctx* ctx, int loop, void* stream);

/* Largest particle count swift_gpu_density_static accepts. */
#define SWIFT_GPU_STATIC_MAX_PARTICLES 32768

/* The density call (cell build, then the density loop with the Newton
 * iteration on h, every particle active) with no context and no allocation
 * of any kind. The paper has no counterpart to this entry point. It is for
 * callers that cannot allocate GPU memory themselves: code whose host
 * framework owns every device allocation and forbids direct cudaMalloc, or a
 * plug-in that may only work in buffers it is handed.
 * Work memory: one fixed array of 5.4 MB (5.2 MiB) built into the library, which
 * every GPU that loads the library holds until the process exits. It fits
 * n <= SWIFT_GPU_STATIC_MAX_PARTICLES; a larger n returns
 * SWIFT_GPU_ERR_CAPACITY before any work is queued.
 * Arguments: *p the physics parameters (host); pos_h, vel_m, h_out, rho4,
 * curl_div, ngb_count as in swift_gpu_build_cells and swift_gpu_density
 * (device, caller order, ngb_count may be NULL); min_cell_width as in
 * swift_gpu_build_cells; status_out NULL or a device array of 2 int64 that
 * receives the device status code and its detail (what swift_gpu_sync_status
 * reports for a context). Asynchronous on `stream`.
 * The first call on a device looks up the array's device address, a one-time
 * set-up per device: make that first call before any stream capture.
 * Every call shares the one array and finds the previous call's contents in
 * it (the call resets what must start at zero). Calls that can overlap on the
 * GPU (other streams, other host threads) race and corrupt each other's
 * results: order them on one stream. Host-side errors as for
 * swift_gpu_density, plus ERR_CAPACITY. */
int swift_gpu_density_static(const swift_gpu_params* p, const float* pos_h, const float* vel_m, int64_t n,
                             float min_cell_width, float* h_out, float* rho4, float* curl_div, uint32_t* ngb_count,
                             int64_t* status_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SWIFT_GPU_H */
