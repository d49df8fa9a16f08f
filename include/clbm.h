/*
 * clbm.h -- C ABI of the GB300 cascaded D3Q19 lattice Boltzmann library for
 * power-law fluids.
 *
 * The method is the 3D cascaded (central-moment, multiple-relaxation-time)
 * LBM of Adam, Hajabdollahi & Premnath, "Cascaded lattice Boltzmann modeling
 * and simulations of three-dimensional non-Newtonian fluid flows":
 *   - D3Q19 velocity set, Eq. velocityd3qq19 (direction order as the paper's
 *     component vectors |e_x>, |e_y>, |e_z> of Sec. 3);
 *   - cascaded collision f~ = f + K g^, Eqs. cascadecollision1 and
 *     cascadedcollision1, with g^_4..g^_18 from Eqs. collisionkernelg4..g18;
 *   - second-order rates omega_4..8 set at every node from the shear rate,
 *     Eq. localvarationsrelaxationtimes with the power law of Eq. 6 and the
 *     strain rate of Eq. strainratetensor; omega_9..18 = 1 as in Sec. 3.1
 *     unless clbm_set_rates() sets others;
 *   - streaming, Eq. cascadedstreaming1, with halfway bounce-back walls, a
 *     moving lid with a momentum correction and periodic faces (Sec. 4).
 *
 * Conventions shared by every entry point:
 *   - Every function returns an int status: CLBM_OK (0) or a negative
 *     CLBM_ERR_* code.  No C++ exception crosses this interface.  The text of
 *     the last error of a handle is returned by clbm_last_error().
 *   - Field arrays use the unpadded layout [z][y][x], x fastest, N = nx*ny*nz
 *     entries.  Vector fields are 3 consecutive such arrays (x, then y, then z
 *     component).  Population arrays are 19 consecutive such arrays, in the
 *     direction order above, holding plain (unshifted) FP64 values f_alpha.
 *   - The caller owns every host and device buffer it passes in.  The library
 *     owns the device memory of a handle (populations, work buffers) and frees
 *     it in clbm_destroy(); it takes that memory from cudaMalloc, or from an
 *     allocator registered with clbm_set_allocator().
 *   - Work is queued on the handle's CUDA stream.  Calls that return data to
 *     the host synchronise that stream; clbm_step() does not.
 *   - A handle is not thread-safe: use one handle per thread, or serialise.
 *   - One GPU: the handle lives on the device that is current when
 *     clbm_create() is called; the library makes that device current again in
 *     every call on the handle.
 */
#ifndef CLBM_H
#define CLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define CLBM_OK 0
#define CLBM_ERR_ARG -1         /* invalid argument or handle */
#define CLBM_ERR_OOM -2         /* device memory allocation failed */
#define CLBM_ERR_CUDA -3        /* CUDA runtime error */
#define CLBM_ERR_DIVERGED -4    /* NaN/Inf or density outside [0.5, 2] seen */
#define CLBM_ERR_TIMEOUT -5     /* a bounded device wait gave up */
#define CLBM_ERR_UNSUPPORTED -6 /* valid request the library does not support */

/* Storage precision of the populations.
 *   CLBM_F64  : f - w rho0 stored in FP64, collision in FP64.
 *   CLBM_F32  : f - w rho0 stored in FP32, collision in FP32.
 *   CLBM_F16S : (f - w rho0) * 1024 stored in FP16 (round to nearest even,
 *               or stochastic rounding: clbm_set_rounding), collision in FP32.
 *   CLBM_F16R : (f - w [rho0 + drho + 3 (rho0 + drho)(e . u)]) * 1024 in
 *               FP16 with stochastic rounding, relative to the writing node's
 *               own (drho, 3 (rho0 + drho) u), which is stored beside the
 *               populations as four FP16 values (scaled by 1024); collision
 *               in FP32.  Removing
 *               the first-order equilibrium before rounding keeps steady
 *               states close to FP64.  16 more bytes per node update than
 *               F16S.  Not available to clbm_step_noalloc, to in-place
 *               streaming or to a batch's one-launch-per-lattice mode.
 * Residual and mass reductions accumulate in FP64 for every form. */
typedef enum { CLBM_F64 = 0, CLBM_F32 = 1, CLBM_F16S = 2, CLBM_F16R = 3 } clbm_dtype;

/* Face kinds, for faces ordered (-x, +x, -y, +y, -z, +z).
 *   CLBM_PERIODIC : both faces of the pair must be periodic.
 *   CLBM_WALL     : halfway bounce-back, no slip (Sec. 4.1, 4.2).
 *   CLBM_LID      : halfway bounce-back plus the momentum correction
 *                   6 w_alpha rho0 (e_alpha . U_lid) of a wall moving with
 *                   velocity U_lid (Sec. 4.3).  U_lid must be tangential to
 *                   every LID face.  Where a link crosses a lid and another
 *                   wall (edges, corners), the lid rule applies. */
typedef enum { CLBM_PERIODIC = 0, CLBM_WALL = 1, CLBM_LID = 2 } clbm_bc;

typedef struct {
  int nx, ny, nz;      /* lattice nodes per axis, each >= 1; ny, nz <= 65535
                        * (the launch grid has one row per y row and z plane) */
  int face[6];         /* clbm_bc of faces -x, +x, -y, +y, -z, +z */
  double rho0;         /* reference density (rest state, lid); 0 -> 1 */
  double nu_min;       /* kinematic-viscosity clamp; 0 -> 5e-4 */
  double nu_max;       /* 0 -> 10 */
  int check_interval;  /* steps between residual checks; 0 -> 100 */
  void* stream;        /* cudaStream_t to queue on; NULL -> library-owned */
  int in_place;        /* 1: one population buffer, streamed in place (not in
                        * the paper): half the memory, the same results and
                        * bytes per update; FP64, FP32 and F16S only; in a
                        * batch only with one launch per lattice
                        * (clbm_batch_set_lattice_launch); the server's
                        * lattices ignore it) */
} clbm_domain;

typedef struct clbm_ctx* clbm_handle;

/* Create a lattice in the rest state f = w rho0 (Sec. 3; initial state not
 * stated by the paper).
 *   K          consistency coefficient mu_p of Eq. 5, > 0.
 *   n          power-law index of Eq. 5, in (0, 3].
 *   U_lid      velocity of LID faces (3 doubles); may be NULL if no LID face;
 *              |U_lid| must be < 0.3.
 *   body_force force per unit volume (3 doubles), NULL -> 0; applied by a
 *              symmetric split, half before and half after the collision.
 *   dtype      storage precision.
 *   out        receives the handle.
 * Errors: CLBM_ERR_ARG (bad sizes or parameters), CLBM_ERR_OOM, CLBM_ERR_CUDA. */
int clbm_create(const clbm_domain* d, double K, double n, const double U_lid[3],
                const double body_force[3], clbm_dtype dtype,
                clbm_handle* out);

/* Queue nsteps time steps (pull-stream + collide, Eqs. cascadedstreaming1 and
 * cascadedcollision1) on the handle's stream and return.  Every step whose
 * global index is a multiple of check_interval also writes u and reduces the
 * residual, the mass and a divergence flag in FP64.
 * Returns CLBM_ERR_DIVERGED if an earlier, already completed check found a
 * non-finite value or a density outside [0.5, 2]; the queued steps still run. */
int clbm_step(clbm_handle h, int64_t nsteps);

/* Macroscopic fields of the current state (Eqs. hydrodynamicfields1/2,
 * shearrateexpression): rho (N), u (3N, the half-force velocity
 * (j + F/2)/rho) and |gamma_dot| (N), computed from the streamed
 * populations.  Host pointers; any may be NULL.  Synchronises the stream. */
int clbm_fields(clbm_handle h, double* rho, double* u, double* gamma_dot);

/* As clbm_fields, into device pointers on the handle's device. */
int clbm_fields_device(clbm_handle h, double* rho, double* u,
                       double* gamma_dot);

/* Last steady-state residual R = ||u - u_prev|| / (check_interval ||u||)
 * over all nodes (FP64); +Inf before the second check.  Synchronises.
 * Returns CLBM_ERR_DIVERGED (and still writes R) if divergence was seen. */
int clbm_residual(clbm_handle h, double* out);

/* Total mass sum(rho) at the last check step (FP64).  Synchronises. */
int clbm_mass(clbm_handle h, double* out);

/* Copy the stored populations to / from the host as plain FP64 f
 * (19 x N, layout above).  Synchronises. */
int clbm_get_state(clbm_handle h, double* f_host);
int clbm_set_state(clbm_handle h, const double* f_host);

/* Steps run so far. */
int clbm_steps_done(clbm_handle h, int64_t* out);

/* Wait for all queued work of the handle. */
int clbm_sync(clbm_handle h);

/* Free the handle and its device memory.  NULL is accepted. */
int clbm_destroy(clbm_handle h);

/* ---- External device allocator -------------------------------------------
 * Not in the paper.  A lattice's long-lived device buffers (populations,
 * F16R references, check-step velocities and sums) come from cudaMalloc
 * unless an allocator is registered here, e.g. PyTorch's caching allocator.
 * Lattices created after the call take their buffers from
 *   alloc_fn(bytes, device, stream, user) -> device pointer, or NULL when out
 *     of memory (clbm_create then fails with CLBM_ERR_OOM);
 * and return them, in clbm_destroy() after synchronising the lattice's
 * stream, through
 *   free_fn(ptr, bytes, device, stream, user);
 * where `stream` is the lattice's CUDA stream and `user` is passed through.
 * A pointer must be aligned to 256 bytes (the kernels' vector and TMA
 * accesses assume it): clbm_create returns CLBM_ERR_ARG for a misaligned one,
 * after handing it back to free_fn.  Each lattice frees through the allocator
 * it was created with.  NULL for both restores cudaMalloc.  Process-wide: call
 * it while no clbm_create or clbm_destroy runs.  Scratch buffers of single
 * calls (field and state transfer, autotuning) stay on the stream-ordered
 * cudaMallocAsync pool.  Errors: CLBM_ERR_ARG if exactly one function is NULL. */
typedef void* (*clbm_alloc_fn)(size_t bytes, int device, void* stream, void* user);
typedef void (*clbm_free_fn)(void* ptr, size_t bytes, int device, void* stream, void* user);
int clbm_set_allocator(clbm_alloc_fn alloc_fn, clbm_free_fn free_fn, void* user);

/* Pick the launch shape of h's step kernel by timing: thread-block shapes
 * from 32x1 to 256x1 (and, for a lattice narrower than a warp, blocks 8 or
 * 16 wide) and, for the FP32-math forms, one or two nodes per
 * thread (two nodes are collided together with packed FP32 instructions),
 * with and without a 64-register cap; for FP32 and F16S storage also the
 * TMA-staged kernel in each of its shapes (see clbm_set_launch).
 * Each candidate runs `steps` steps (<= 0 -> 10) after two warm-up steps,
 * timed with CUDA events on the handle's stream; the state is saved first
 * and restored afterwards, and the step counter does not move.  The choice
 * is cached per (dtype, nx, ny, nz, force, Newtonian) for the process, so
 * later handles of the same kind reuse it without timing.  Any output
 * pointer may be NULL.  Synchronises; temporarily needs one extra population
 * buffer of device memory. */
int clbm_autotune(clbm_handle h, int steps, int* block_x, int* block_y, int* npt,
                  double* us_per_step);

/* Set the launch shape of h's step kernel directly: block_x * block_y
 * threads (a multiple of 32, at most 256; at most 128 when npt = 2) and
 * npt = 1 or 2 nodes per thread (2 only for the FP32 and F16S forms), plus 4
 * for the register-capped variant.  FP32 and F16S storage also take
 * npt = 16 + 32 v, the kernel whose upwind populations are staged in shared
 * memory by TMA loads, in shape v (block, nodes per thread): v = 0: 64x4, 1;
 * v = 1: 128x2, 1; v = 2: 32x8, 1; v = 3: 64x4, 1 (three ring stages);
 * v = 4: 32x4, 1; v = 5: 64x2, 1; v = 6: 64x2, 2; v = 7: 32x4, 2; v = 8:
 * 64x2, 2 (four CTAs per SM); v = 9: 128x1, 2.  With two nodes a thread
 * collides rows 2y and 2y+1 as a packed FP32 pair.  block_x x block_y must
 * be that shape's.  Check steps run
 * the plain kernel with the same block.  If a pipeline wait of that kernel
 * gives up (about one second; never expected), the next check makes
 * clbm_step / clbm_residual return CLBM_ERR_CUDA. */
int clbm_set_launch(clbm_handle h, int block_x, int block_y, int npt);

/* Set the relaxation rates omega_9 .. omega_18 of h: the bulk rate (omega_9)
 * and the third- (omega_10..15) and fourth-order (omega_16..18) rates of the
 * cascaded collision (Sec. 3.1 sets all to 1; Sec. 5 notes that tuning them
 * can improve stability).  omega[k] is omega_(9+k); each must lie in (0, 2).
 * omega_9 also scales the isotropic part of the strain rate that sets
 * omega_nu.  Takes effect from the next step.  Not for a lattice in a batch
 * (CLBM_ERR_ARG: detach it first).  Errors: CLBM_ERR_ARG. */
int clbm_set_rates(clbm_handle h, const double omega[10]);

/* Rounding of the FP16 stores of an F16S lattice (not in the paper, which
 * computes in one precision).  CLBM_ROUND_NEAREST (the default) rounds each
 * stored value to the nearest FP16 value.  Near a steady state the per-step
 * change of a stored value falls below half an FP16 ulp and is rounded away,
 * so the state freezes short of the steady state.  CLBM_ROUND_STOCHASTIC
 * rounds up in magnitude with probability equal to the fraction of an ulp the
 * value carries, from random bits that depend only on the node and the
 * lattice's step count (the same bits alone and in any run); such changes
 * then survive on average.  The stored layout does not change.  Stochastic
 * rounding runs the one-node-per-thread step kernel only (npt 1 or 5);
 * clbm_set_rounding resets another launch shape to npt 1, and a batch does
 * not take such a lattice (clbm_batch_add: CLBM_ERR_UNSUPPORTED).  Errors:
 * CLBM_ERR_UNSUPPORTED for other storage forms (F16R always rounds
 * stochastically and accepts CLBM_ROUND_STOCHASTIC as a no-op; FP32 and FP64
 * accept CLBM_ROUND_NEAREST as a no-op) and for stochastic rounding of an
 * in-place lattice; CLBM_ERR_ARG for an invalid handle, an unknown mode or a
 * lattice in a batch (detach it first). */
typedef enum { CLBM_ROUND_NEAREST = 0, CLBM_ROUND_STOCHASTIC = 1 } clbm_rounding;
int clbm_set_rounding(clbm_handle h, clbm_rounding mode);

/* ---- Batched stepping of many lattices --------------------------------
 * Not in the paper: a batch steps up to `capacity` lattices of one storage
 * form (any of the four, F16R with its reference moments) together: per
 * time step one launch of a persistent kernel over the tiles of all
 * lattices without body force and one over those with it, the two on two
 * streams at once (tiles from a device-side table), with each whole
 * check interval queued as one CUDA graph (or, after
 * clbm_batch_set_lattice_launch, one launch per lattice within that graph).  Lattices join and leave between
 * clbm_batch_step() calls; each keeps its own buffers, parameters, step
 * count and residual.  While a lattice is in a batch, clbm_step() on it
 * fails; clbm_fields/get_state/residual/... on it first wait for the batch.
 * Destroying a lattice removes it from its batch. */
typedef struct clbm_batch_ctx* clbm_batch;

/* capacity: at most this many lattices at once (1..65536); check_interval:
 * even number of steps between residual checks (0 -> 100); stream: CUDA
 * stream for the batch's work (NULL -> library-owned). */
int clbm_batch_create(clbm_dtype dtype, int capacity, int check_interval, void* stream,
                      clbm_batch* out);
/* Attach h (same dtype and device, not in another batch, 19 x padded nodes
 * < 2^31; an in-place lattice only in the one-launch-per-lattice mode, an
 * F16S lattice with stochastic rounding only in the persistent mode, else
 * CLBM_ERR_UNSUPPORTED); its queued work is waited for; *slot receives its
 * slot. */
int clbm_batch_add(clbm_batch b, clbm_handle h, int* slot);
/* Detach the lattice in `slot` (waits for the batch's queued work). */
int clbm_batch_remove(clbm_batch b, int slot);
int clbm_batch_detach(clbm_batch b, clbm_handle h);
/* Queue nsteps steps of every attached lattice (Eqs. cascadedstreaming1,
 * cascadedcollision1).  Every step whose batch index is a multiple of the
 * check interval is a check step for all of them. */
int clbm_batch_step(clbm_batch b, int64_t nsteps);
/* Results of the last check of the lattice in `slot`: residual (as
 * clbm_residual; +Inf until it has had two checks in this batch), mass, the
 * divergence flag and its step count.  Any pointer may be NULL.  Syncs. */
int clbm_batch_stats(clbm_batch b, int slot, double* residual, double* mass, int* diverged,
                     int64_t* steps);
/* clbm_batch_stats of every slot at once: arrays of `capacity` entries
 * (empty slots give NaN, NaN, 0, -1).  Any pointer may be NULL.  Syncs once. */
int clbm_batch_stats_all(clbm_batch b, double* residual, double* mass, int* diverged,
                         int64_t* steps);
/* The persistent kernel with this launch shape: thread block (multiple of
 * 32 threads, <= 256), planes per tile zc >= 1, resident blocks per SM of
 * the persistent grid (negative: the same count with the register-capped
 * kernel variant).  CLBM_ERR_UNSUPPORTED while an in-place lattice is
 * attached. */
int clbm_batch_set_launch(clbm_batch b, int block_x, int block_y, int zc, int blocks_per_sm);
/* One launch per lattice instead of the persistent kernel (FP64, FP32,
 * F16S; CLBM_ERR_UNSUPPORTED for F16R and while an F16S lattice with
 * stochastic rounding is attached, whose rounding is seeded by the batch's
 * device-side step count): every step launches each attached lattice's own
 * step kernel (block_x x block_y threads, a multiple of 32 and <= 256; npt 1,
 * or 5 for the register-capped kernel), the lattices spread over `streams`
 * (1..16) streams, largest first onto the least-loaded one.  The streams fork
 * from the batch's stream and join it around each check interval, which is
 * still one CUDA graph; a change of membership recaptures it.  Results are
 * those of clbm_step on each lattice.  This mode also steps in-place
 * lattices.  clbm_batch_set_launch() returns to the persistent kernel. */
int clbm_batch_set_lattice_launch(clbm_batch b, int block_x, int block_y, int npt, int streams);
/* Time block shapes x zc x blocks-per-SM x register cap of the persistent
 * kernel and, except for F16R and stochastically rounding F16S lattices,
 * block shapes x kernel variant x streams of one
 * launch per lattice, on the attached lattices (states saved and restored),
 * and keep the fastest (only the latter while an in-place lattice is
 * attached).  Persistent kernel: *blocks_per_sm is negative when
 * the capped variant won.  One launch per lattice: *zc is 0, *block_x and
 * *block_y are the lattices' block, |*blocks_per_sm| is the stream count,
 * negative for the register-capped kernel. */
int clbm_batch_autotune(clbm_batch b, int steps, int* block_x, int* block_y, int* zc,
                        int* blocks_per_sm, double* us_per_step);
int clbm_batch_sync(clbm_batch b);
int clbm_batch_destroy(clbm_batch b);
const char* clbm_batch_last_error(clbm_batch b);

/* ---- Continuous-batching solve server -----------------------------------
 * Not in the paper: a worker thread owns a batch and repeatedly (1) admits
 * queued requests first come first served while a slot is free and the
 * request's device memory fits the HBM budget, (2) steps every admitted
 * lattice by one check interval in one graph launch, (3) retires lattices
 * whose residual (as clbm_residual) is <= tol, that diverged, that reached
 * max_steps, or whose residual has not fallen by 10 % for plateau_checks
 * checks.  Requests join only at check-interval boundaries, so a request's
 * step count and result do not depend on the other requests in the mix. */
typedef struct {
  clbm_domain dom;       /* lattice; dom.stream and dom.check_interval ignored */
  double K, n;           /* as clbm_create */
  double U_lid[3];
  double body_force[3];
  double tol;            /* residual target */
  int64_t max_steps;     /* step cap (0: none) */
  int plateau_checks;    /* 0: no plateau rule */
  int keep_fields;       /* copy rho, u, gamma_dot to host memory at the end */
} clbm_request;

enum {
  CLBM_SOLVE_CONVERGED = 0,
  CLBM_SOLVE_MAX_STEPS = 1,
  CLBM_SOLVE_PLATEAU = 2,
  CLBM_SOLVE_DIVERGED = 3,
  CLBM_SOLVE_REJECTED = 4,   /* larger than the whole budget */
  CLBM_SOLVE_CANCELLED = 5,  /* server destroyed first */
  CLBM_SOLVE_ERROR = 6
};

typedef struct {
  int64_t id;
  int status;                         /* CLBM_SOLVE_* */
  int64_t steps;
  double residual, mass;
  double t_submit, t_admit, t_done;   /* seconds on the server's clock */
  int64_t N;                          /* lattice nodes */
} clbm_result;

typedef struct {
  int64_t queued, active, done;
  double used_bytes;                  /* device memory held by admitted lattices */
  double lattice_updates;             /* node updates done so far */
  double busy_seconds;                /* time spent stepping */
  double clock;                       /* the server clock now */
} clbm_server_stats;

typedef struct clbm_server_ctx* clbm_server;

/* The server's lattices live on the device current at creation. */
int clbm_server_create(clbm_dtype dtype, double hbm_budget_bytes, int max_active,
                       int check_interval, clbm_server* out);
/* Store rounding of the lattices an F16S server admits from now on
 * (clbm_set_rounding; default CLBM_ROUND_NEAREST).  The same errors as
 * clbm_set_rounding for the server's storage form. */
int clbm_server_set_rounding(clbm_server s, clbm_rounding mode);
/* Queue a request (thread-safe); *id identifies it. */
int clbm_server_submit(clbm_server s, const clbm_request* req, int64_t* id);
/* Block until request id is finished (timeout_s < 0: no limit); returns
 * CLBM_ERR_TIMEOUT if it is not finished in time. */
int clbm_server_wait(clbm_server s, int64_t id, double timeout_s, clbm_result* out);
/* Up to max finished results (not yet released), in id order. */
int clbm_server_results(clbm_server s, clbm_result* out, int max, int* n);
/* Fields of a finished keep_fields request, layouts as clbm_fields. */
int clbm_server_fields(clbm_server s, int64_t id, double* rho, double* u, double* gamma_dot);
/* Forget a finished request and its fields. */
int clbm_server_release(clbm_server s, int64_t id);
int clbm_server_info(clbm_server s, clbm_server_stats* out);
/* Stop after the current interval; unfinished requests end CANCELLED. */
int clbm_server_destroy(clbm_server s);
const char* clbm_server_last_error(clbm_server s);

/* Text of the last error on h (never NULL); h may be NULL for errors of
 * clbm_create. */
const char* clbm_last_error(clbm_handle h);

/* Collide M independent nodes without streaming (Eqs. cascadecollision1,
 * cascadedcollision1): f_in and f_out are host arrays of 19 x M plain FP64
 * populations, [alpha][node].  The node states are stored in dtype first
 * (so F16S/F32 see their storage rounding), collided with the parameters
 * K, n, body_force, rho0, nu_min, nu_max (0 -> defaults) on the current
 * device, and returned.  rho, u (3 x M) and gamma_dot, if not NULL, receive
 * the per-node fields.  Synchronous. */
int clbm_collide_nodes(clbm_dtype dtype, double K, double n,
                       const double body_force[3], double rho0, double nu_min,
                       double nu_max, const double* f_in, double* f_out,
                       double* rho, double* u, double* gamma_dot, int64_t M);

/* The local relaxation rate omega_nu (Eq. localvarationsrelaxationtimes with
 * the power law of Eq. 6) and |gamma_dot| (Eqs. strainratetensor,
 * shearrateexpression) of M nodes, solved on the current device exactly as
 * the collision of storage form dtype solves them (FP64 for CLBM_F64, FP32
 * for the other forms), with omega_9..18 = 1 and the viscosity clamped to
 * [nu_min, nu_max] (0 -> 5e-4, 10).
 *   rho:   M densities (host, FP64);
 *   m:     host array of 6 x M non-equilibrium second moments
 *          m^(1)_4..m^(1)_9 of Sec. 3.2, [moment][node];
 *   omega, gamma_dot: M outputs each (host; gamma_dot may be NULL).
 * Synchronous.  Errors: CLBM_ERR_ARG, CLBM_ERR_OOM, CLBM_ERR_CUDA. */
int clbm_omega_nodes(clbm_dtype dtype, double K, double n, double nu_min, double nu_max,
                     const double* rho, const double* m, double* omega, double* gamma_dot,
                     int64_t M);

/* Fused multiply-add throughput of the current device, in FLOP/s (two per
 * FMA), for dtype CLBM_F64 or CLBM_F32: a measurement utility with no
 * counterpart in the paper.  It gives the arithmetic ceiling of a step form
 * bound by its arithmetic pipe instead of HBM (the FP64 form on GB300): one
 * grid of 8 blocks of 256 threads per SM, eight independent FMA chains per
 * thread, timed with CUDA events on the legacy default stream (about 0.1 s,
 * after a shorter warm-up launch).  Synchronous; allocates no device memory.
 * Errors: CLBM_ERR_ARG (other dtype, NULL out), CLBM_ERR_CUDA. */
int clbm_probe_fma_rate(clbm_dtype dtype, double* flops_per_s);

/* One check step between caller-owned device buffers, with no device memory
 * allocated by the library.  The paper has no counterpart: this entry point
 * exists for callers that cannot call cudaMalloc while they step -- a host
 * application that hands out a fixed device-memory pool reserved at start-up,
 * a framework that has already claimed the whole device, or code that must
 * not stall on the allocator's implicit synchronisation.  It allocates
 * nothing and calls no allocating library routine.
 *
 * It runs the same fused pull-stream + collide step as a check step of
 * clbm_step() (Eqs. cascadedstreaming1, cascadedcollision1) from src to dst:
 *   d, K, n, U_lid, body_force, dtype: as for clbm_create(); d->stream is the
 *          CUDA stream to queue on (NULL: the legacy default stream);
 *          d->check_interval is ignored.
 *   src, dst: device buffers of 19 x N stored values in the dtype's storage
 *          type (double, float, or FP16 bits), dense layout [q][z][y][x]
 *          with no padding, holding f - w rho0 (times 1024 for F16S); src is
 *          read, dst is written; they must not overlap.
 *   u_prev: device buffer of 3 x N velocities [component][z][y][x] in the
 *          math type (double for F64, float otherwise): read as the previous
 *          check's velocity, overwritten with this step's.
 *   stats:  device pointer to 4 doubles, written with sum |u - u_prev|^2,
 *          sum |u|^2, sum (rho - rho0) and a divergence flag (0 or 1).
 * The per-block partial sums of the reductions live in a fixed array of
 * 65536 x 4 doubles (2 MiB) inside the library, which every GPU that loads
 * the library holds until the process exits; a lattice needing more than
 * 65536 blocks of 32 x 4 nodes (about 8.4 million nodes) is rejected with
 * CLBM_ERR_ARG and a message from clbm_last_error(NULL).  Each call rewrites
 * all the partial sums it reads, so no state carries over between calls, but
 * calls that overlap on the GPU (on different streams, or on the same device
 * from different threads) share that array and race.  The first call on each
 * device looks up the array's device address (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture.
 * Queues two kernels and returns without synchronising.
 * Errors: CLBM_ERR_ARG (bad sizes or parameters, checked as for
 * clbm_create()), CLBM_ERR_UNSUPPORTED (dtype CLBM_F16R), CLBM_ERR_CUDA (a
 * failed launch, or a first call made inside a stream capture); the text is
 * in clbm_last_error(NULL). */
int clbm_step_noalloc(const clbm_domain* d, double K, double n, const double U_lid[3],
                      const double body_force[3], clbm_dtype dtype, const void* src,
                      void* dst, void* u_prev, double* stats);

#ifdef __cplusplus
}
#endif
#endif
