/*
 * liblbm: GB300 (sm_103a) implementation of the coupled D2Q9 flow / D2Q5
 * temperature multiple-relaxation-time lattice Boltzmann step for convection
 * heat transfer in porous media at the REV scale (Liu, He, Li, Tao,
 * arXiv:1308.2071, Section 3), with the cavity problem of Section 4.
 *
 * Conventions shared by every entry point
 *  - Every function returns an int status (LBM_OK = 0 or an LBM_ERR_* code);
 *    no C++ exception crosses this boundary.  lbm_last_error() describes the
 *    last failure of a handle.
 *  - Pointers named *_dev are CUDA device pointers on the device that was
 *    current when lbm_init() ran; pointers named *_host are host pointers.
 *  - Fields are dense row-major (ny, nx) arrays with x fastest; node (x, y)
 *    is element y * nx + x.  Walls lie on the perimeter nodes: x = 0 is the
 *    hot wall, x = nx - 1 the cold wall, y = 0 and y = ny - 1 the adiabatic
 *    walls of the side-heated cavity (Section 4.1), so L = nx - 1.
 *  - Work is enqueued on the stream given to lbm_init(); calls that return
 *    host values synchronise that stream, the others are stream-ordered.
 *  - The library owns its state buffers (allocated in lbm_init(), freed in
 *    lbm_destroy()); caller buffers are never retained past a call.
 *  - A handle is not thread-safe: one host thread at a time.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define LBM_OK 0
#define LBM_ERR_ARG 1      /* invalid argument: tau <= 1/2, phi outside (0, 1], n < 5, ... */
#define LBM_ERR_CUDA 2     /* a CUDA runtime call failed                                  */
#define LBM_ERR_DIVERGED 3 /* a non-finite value or |u| >= 1/2 was met on the lattice     */
#define LBM_ERR_TIMEOUT 4  /* a bounded device-side wait ran out                          */
#define LBM_ERR_STATE 5    /* call out of order (e.g. adjoint before any forward state)   */

/* Storage / arithmetic precision of the populations.  Populations are stored
 * as deviations from the rest state.  The FP32-arithmetic variants keep the
 * thermal populations relative to a per-node temperature frame (one more
 * plane: the node's T - T0 when it was last written), so that the stored
 * values stay small and FP32 keeps the slow late-time evolution of T (plain
 * FP32 deviations g_j - w~_j T0 of up to 0.3 lose changes below 3e-8 per
 * step).  LBM_F32 and LBM_F32_FRAMED collide in increments (f + M^-1 (m+ -
 * m), equal in exact arithmetic to Eq. 18), which keeps the rounded factors
 * of M^-1 from biasing the momentum step after step.  LBM_F32_STORE_F16
 * rounds the flow values to half precision with a threshold taken from other
 * populations' low bits (dithered) instead of to nearest, so the rounding
 * errors average out over the steps.  Bytes moved per node and step: 224,
 * 114, 78, 120. */
#define LBM_F64 0            /* FP64 storage, FP64 arithmetic                       */
#define LBM_F32 1            /* FP32 storage, 8-bit temperature frame (a power-of-
                                two quantum fq: F = k fq), FP32 arithmetic          */
#define LBM_F32_STORE_F16 2  /* FP16 flow storage, FP32 thermal storage with the
                                8-bit temperature frame, FP32 arithmetic            */
#define LBM_F32_FRAMED 3     /* FP32 storage, FP32 temperature frame, FP32
                                arithmetic                                          */

/* thermal boundary layouts */
#define LBM_BC_SIDE_HEATED 0 /* Section 4.1: left T_h, right T_c, top/bottom adiabatic */
#define LBM_BC_COOLED 1      /* Section 4.2: every wall at T_c                         */

/* collision operators */
#define LBM_MRT 0            /* Eq. 17 and Eq. 34 with the rates of Section 4        */
#define LBM_LBGK 1           /* every rate 1/tau (the reduction stated after Eq. 24) */

/* Parameters of one cavity.  Physical inputs follow Section 2 (Ra, Da, Pr, J,
 * porosity), the lattice set-up follows Section 4: rho0 = 1, delta_t = 1,
 * Eq. 37 (second occurrence) for tau_nu and tau_T, U = sqrt(g beta dT L) =
 * Ma c_s, K = Da L^2 (Da = INFINITY: no Darcy or Forchheimer drag), F_phi
 * from Ergun's relation (Eq. 5). */
typedef struct {
    int nx, ny;          /* nodes including the wall nodes, both >= 5                 */
    double Ra, Da, Pr, J;
    double phi;          /* porosity (mean porosity when a field is set), in (0, 1]   */
    double Ma;           /* Mach number (Section 4: 0.1)                               */
    double sigma, varpi; /* thermal capacity ratio, D2Q5 constant (Section 4: 1, -2) */
    double Th, Tc;       /* wall temperatures; T0 = (Th + Tc) / 2                      */
    double Qppp;         /* internal heat source Q''' in lattice units (Eq. 30, 33-36) */
    int precision;       /* LBM_F64, LBM_F32, LBM_F32_STORE_F16, LBM_F32_FRAMED         */
    int use_phi_field;   /* 0: uniform phi; 1: per-cell phi from lbm_set_porous_field  */
    int forchheimer;     /* 1: F_phi of Eq. 5; 0: F_phi = 0 (Brinkman model, Sect. 3.1)*/
    int thermal_bc;      /* LBM_BC_SIDE_HEATED or LBM_BC_COOLED                          */
    int adiabatic_order; /* 1: T_b = T_f on adiabatic walls; 2: T_b = (4T_f - T_ff)/3   */
    int collision;       /* LBM_MRT or LBM_LBGK                                          */
    int block_x, block_y;/* launch shape of the step kernel; 0 = library default        */
    int nodes_per_thread;/* 1: one node per thread; 2: two along y; 3: two side by side
                            along x (paired loads and stores); 0 = library default */
    double RaI;          /* internal Rayleigh number (Section 2); 0 = none.  With
                            LBM_BC_SIDE_HEATED: Q''' = (RaI/Ra) alpha_e (Th-Tc)/L^2
                            (Section 4.3); with LBM_BC_COOLED: tau_nu from RaI,
                            dT = Q''' L^2 / alpha_e := Th - Tc, T0 = Tc (Section 4.2) */
} lbm_params;

/* Observables of the post-stream state at the current time t (the state the
 * next collision reads).  Nusselt numbers follow Eq. 38 with a one-sided
 * fourth-order five-point derivative and the trapezoidal mean over the wall
 * nodes, accumulated in FP64. */
typedef struct {
    long t;              /* time steps taken since lbm_init                            */
    double nu_hot;       /* mean Nu of the wall x = 0                                  */
    double nu_cold;      /* mean Nu of the wall x = nx - 1                             */
    double residual;     /* max|u - u_prev| / max|u| since the previous observables call*/
    double umax;         /* max |u| over the lattice                                   */
    double mass;         /* sum over nodes of sum_i f_i (FP64)                         */
    double heat;         /* sum over nodes of T (FP64)                                 */
    int status;          /* LBM_OK or LBM_ERR_DIVERGED                                 */
} lbm_obs;

typedef struct lbm_handle_s* lbm_handle;

/* Fills p with the defaults of Section 4 for an nx-by-ny side-heated cavity:
 * Pr = 1, J = 1, Ma = 0.1, sigma = 1, varpi = -2, Th = 1, Tc = 0, Q''' = 0,
 * FP32, uniform porosity, Ergun F_phi, first-order adiabatic walls, MRT. */
void lbm_params_default(lbm_params* p, int nx, int ny, double Ra, double Da, double phi);

/* Creates a cavity (Section 4.1 set-up) on the current CUDA device.
 * stream: a cudaStream_t (NULL = legacy default stream) on which all work of
 * the handle is enqueued.  Initial state (a reading of Section 4, where the
 * paper says only "uniform"): u = 0, phi p = rho0 c_s^2, T = T0, then the
 * non-equilibrium extrapolation wall rule once.  Errors: LBM_ERR_ARG for an
 * invalid p (tau <= 1/2, phi outside (0, 1], nx or ny < 5, lattice too large
 * for 32-bit offsets), LBM_ERR_CUDA. *out is NULL on failure. */
int lbm_init(const lbm_params* p, void* stream, lbm_handle* out);

/* Sets a per-cell porosity field (extension of the homogeneous model of
 * Section 2: K(phi) and F_phi(phi) follow Eq. 5 per cell, with the particle
 * diameter fixed so that K(p->phi) = Da L^2).  phi_dev: device array of ny*nx
 * values in (0, 1), dtype LBM_F64 (double) or LBM_F32 (float); the caller
 * keeps ownership, the library copies it (to float for the FP32 and
 * FP16-storage paths, double for FP64).  Requires
 * use_phi_field = 1.  Resets the state to the initial state (t = 0).  The
 * values are checked on the device first (the call synchronises the stream):
 * a field with any value outside (0, 1), NaN included, is rejected with
 * LBM_ERR_ARG and leaves the handle as it was.
 * Errors: LBM_ERR_ARG, LBM_ERR_STATE (use_phi_field = 0), LBM_ERR_CUDA. */
int lbm_set_porous_field(lbm_handle h, const void* phi_dev, int dtype);

/* Bounds-checked build (the library compiled with LBM_BOUNDS_CHECK; no
 * counterpart in the paper): every population, frame and porosity access of
 * the step kernels' pull, wall rule and stores is checked against its plane
 * before it is made, and one outside is skipped and counted.  *enabled
 * (may be NULL) tells whether this library is such a build; *count (may be
 * NULL) receives the number of skipped accesses on the current device since
 * the previous call (0 in the normal build), which clears it.  Synchronises
 * the device.  Errors: LBM_ERR_CUDA. */
int lbm_bounds_check(int* enabled, long* count);

/* Restarts the cavity from the initial state of lbm_init (t = 0), keeping its
 * parameters, porosity field and launch shape; stream-ordered.  Clears the
 * divergence flag.  Errors: LBM_ERR_ARG (NULL), LBM_ERR_CUDA. */
int lbm_reset(lbm_handle h);

/* Autotuner of the step kernel: times candidate launch shapes (block_x x
 * block_y threads, nodes_per_thread 1, 2 or 3) on this lattice, keeps the
 * fastest and records it in a text cache at cache_path (NULL: no cache; one
 * line per device, precision, lattice size and porosity mode); a cached entry
 * is reused without timing.  Timing advances the lattice, so the handle is
 * reset to its initial state (t = 0) afterwards.  Outputs may be NULL. */
int lbm_tune(lbm_handle h, const char* cache_path, int* block_x, int* block_y, int* nodes_per_thread);

/* Advances nsteps time steps of Eq. 17-18 and Eq. 34-35 with the wall rule
 * (Section 4), asynchronously on the handle's stream.  Long runs replay a
 * captured CUDA graph.  Errors: LBM_ERR_ARG (nsteps < 0), LBM_ERR_CUDA. */
int lbm_step(lbm_handle h, long nsteps);

/* Computes the observables of the current state and, for each non-NULL
 * pointer, the field: ux_dev, uy_dev (Eq. 21), T_dev (Eq. 36), p_dev (Eq. 23),
 * each ny*nx device values of double (LBM_F64) or float (other precisions);
 * wall nodes report their imposed values (u = 0, wall T and p).
 * Synchronises the stream.  Returns LBM_ERR_DIVERGED (with *out filled) if
 * the divergence flag was raised by any step since lbm_init. */
int lbm_observables(lbm_handle h, lbm_obs* out, void* ux_dev, void* uy_dev, void* T_dev,
                    void* p_dev);

/* As lbm_nusselt, without waiting: enqueues the computation of (nu_hot,
 * nu_cold) into out2 (2 doubles) on the handle's stream.  When out2 is device
 * memory or pinned (mapped) host memory the kernel writes it directly;
 * otherwise a copy follows the kernel (pageable host memory makes that copy
 * synchronous).  The values are there once the stream reaches this point
 * (e.g. after cudaStreamSynchronize or lbm_query).  Lets a caller read the
 * result of every step without stalling.  Errors: LBM_ERR_ARG (NULL), LBM_ERR_CUDA. */
int lbm_nusselt_async(lbm_handle h, double* out2);

/* Advances nsteps time steps, as lbm_step (the same lattice, bit for bit),
 * and after step k (0-based) writes the mean Nusselt numbers (Eq. 38) of the
 * walls x = 0 and x = nx - 1 of the new state to out[2k] and out[2k + 1]: the
 * values lbm_nusselt would return there, bit for bit.  Each step stores the
 * temperatures of the five node columns next to each wall as it computes
 * them (10 doubles per row, double-buffered in the handle), so nothing is
 * pulled twice; a small kernel reduces them on a second, high-priority
 * stream of the handle (created on first use) while the next step runs.
 * out: 2 * nsteps doubles in device memory or page-locked host memory,
 * caller-owned, written by the GPU directly.  Asynchronous on the handle's
 * stream: the values are complete once the stream reaches this point.
 * Errors: LBM_ERR_ARG (NULL handle or out, nsteps < 0, out in pageable host
 * memory or not aligned for double), LBM_ERR_CUDA. */
int lbm_step_nusselt(lbm_handle h, long nsteps, double* out);

/* Discrete adjoint (no counterpart in the paper, which has no gradient).
 * Resets the handle to its initial state, runs nsteps steps forward keeping
 * one lattice every ckpt_every steps, evaluates J = mean Nu of the hot wall
 * (Eq. 38) at t = nsteps, then sweeps backwards, recomputing each segment of
 * ckpt_every states from its checkpoint, and writes dJ/dphi for every cell
 * (ny*nx dense device values, double for LBM_F64, float for the FP32
 * variants) to dJdphi_dev; *J (host, may be NULL) receives J.  The porosity
 * enters through the per-cell Ergun drag (Eq. 4-5) and the equilibria (Eq.
 * 14, 16, 19, 23).  The adjoint is taken at the plain deviations: the
 * temperature frames of the FP32 storage are an exact change of variables.
 * The recomputation of each segment runs on a stream of its own, beside the
 * reverse sweep of the segment after it.  The handle ends at t = nsteps.
 * Needs use_phi_field = 1, LBM_F64, LBM_F32 or LBM_F32_FRAMED, first-order
 * adiabatic walls.  Allocates (nsteps/ckpt_every + 2 ckpt_every + 1)
 * lattices of temporary device memory for the call.  Synchronises.
 * Errors: LBM_ERR_STATE (no porosity field), LBM_ERR_ARG, LBM_ERR_CUDA. */
int lbm_adjoint_step(lbm_handle h, long nsteps, long ckpt_every, double* J, void* dJdphi_dev);

/* Mean Nusselt numbers (Eq. 38) of the walls x = 0 and x = nx - 1 of the
 * current state, FP64; reads only the five node columns next to each wall.
 * Synchronises the stream. */
int lbm_nusselt(lbm_handle h, double* nu_hot, double* nu_cold);

/* Steady-state control loop run on the device: one CUDA graph whose
 * conditional while-node repeats {check_every steps (rounded up to even),
 * then a one-block check of both wall Nusselt numbers} until their relative
 * change between two checks falls below tol, the divergence flag is raised,
 * or max_steps is reached; the host waits once.  *steps_taken and *change
 * (host, may be NULL) report the steps run and the last relative change.
 * Returns LBM_ERR_DIVERGED if the flag was raised. */
int lbm_run_steady(lbm_handle h, double tol, long check_every, long max_steps, long* steps_taken, double* change);

/* Extrema for the validation tables: maximum temperature and the minimum and
 * maximum of the stream function psi(x, y) = integral_0^y u_x dy' (trapezoidal
 * along y, psi = 0 on the bottom wall; lattice units) of the current state.
 * Host outputs may be NULL.  Synchronises. */
int lbm_field_extrema(lbm_handle h, double* T_max, double* psi_min, double* psi_max);

/* Writes the full post-stream populations of the current state as FP64:
 * f_dev[9][ny][nx] and g_dev[5][ny][nx] (device, caller-owned), velocity
 * order of Eq. 8 (rest, E, N, W, S, NE, NW, SW, SE) and Eq. 26.  Used to
 * compare the lattice with a reference implementation.  Stream-ordered. */
int lbm_read_state(lbm_handle h, double* f_dev, double* g_dev);

/* Checkpoint / resume.  A checkpoint is a header (magic, version 3, nx, ny,
 * precision, t) and one state buffer, the post-collision lattice B_{n-1}
 * that the current post-stream state S_n is pulled from (Eq. 18, 35): every
 * observable at t_n comes from it, and lbm_load() rebuilds B_n from it with
 * one step, so a handle that loads it continues exactly as the handle that
 * saved it would, given the same launch shape (lbm_tune).  Version-1
 * checkpoints (B_{n-1} then B_n) and version 2 are still read for LBM_F64 and
 * LBM_F32_FRAMED, whose layout they share; LBM_F32 and LBM_F32_STORE_F16
 * lattices of those versions (stored without temperature frames) are
 * refused with LBM_ERR_ARG.  lbm_checkpoint_size() gives
 * the byte count; lbm_save() writes it into a caller-owned host buffer of at
 * least that size (synchronises the stream); lbm_load() restores it into a
 * handle created with the same nx, ny and precision (synchronises the
 * stream).  Errors: LBM_ERR_ARG (buffer too small, header mismatch),
 * LBM_ERR_CUDA. */
int lbm_checkpoint_size(lbm_handle h, size_t* bytes);
int lbm_save(lbm_handle h, void* host, size_t bytes);
int lbm_load(lbm_handle h, const void* host, size_t bytes);

/* Observables of a saved lattice, computed without allocating any memory.
 * For callers that may not allocate device memory on their call path: a
 * framework's custom operator whose device memory belongs to the framework's
 * own allocator or to a fixed budget, or a monitoring stage that runs between
 * latency-critical GPU work, where a cudaMalloc would synchronise the device.
 * The caller keeps a checkpoint (the bytes lbm_save writes: header, then the
 * state buffer) in its own device memory at ckpt_dev, `bytes` long, and
 * passes the lbm_params it was made with.  The function computes what
 * lbm_observables computes for that state, except the residual (reported as
 * 0), writes *out (host) and, for each non-NULL pointer, the field (ny*nx
 * device values, double for LBM_F64, float otherwise); the work is enqueued on
 * `stream` (a cudaStream_t, NULL = legacy default) and synchronised before
 * the call returns.  The paper has no counterpart to this call.
 * Scratch: one static device array of 38,984 bytes (the FP64 partial sums of
 * the fixed 1216-block reduction grid, the result, and a status word), which
 * every device that loads the library holds until the process exits; any
 * lattice that lbm_init accepts uses the same grid.  The first call on a
 * device looks up that array's device address once, with the device current:
 * make that first call before any stream capture.  All calls share the array
 * and it keeps the previous call's contents (the status word is cleared on
 * entry), so calls that overlap on the GPU race: serialise them.
 * A checkpoint carries no divergence flag of the steps that made it, so the
 * state itself is tested: a non-finite value anywhere (the maximum of |u|
 * keeps NaN) or |u| >= 1/2 sets out->status and returns LBM_ERR_DIVERGED,
 * with *out and the fields filled.
 * Errors: LBM_ERR_ARG (invalid parameters, use_phi_field set, a lattice
 * beyond 32-bit offsets, a buffer smaller than the lattice needs, a header
 * that does not match p, a checkpoint of an older storage layout),
 * LBM_ERR_DIVERGED, LBM_ERR_CUDA; lbm_last_error(NULL) describes it. */
int lbm_observables_noalloc(const lbm_params* p, const void* ckpt_dev, size_t bytes, void* stream,
                            lbm_obs* out, void* ux_dev, void* uy_dev, void* T_dev, void* p_dev);

/* ---- batched sweep ---------------------------------------------------------
 * Many independent cavities (each its own nx, ny, Ra, Da, porosity, ...; one
 * precision, LBM_F32, LBM_F32_FRAMED or LBM_F64, uniform porosity) advanced together: every
 * lbm_batch_step() is ONE persistent cooperative kernel launch that runs all
 * requested steps of all cavities (blocks walk a tile list that covers every
 * cavity; a bounded grid-wide barrier, or in the dataflow schedule bounded
 * per-cavity step counters, order the steps), captured into a CUDA graph on
 * first use and replayed.  Per node it runs the same code as lbm_step: with
 * one node per thread each cavity evolves bit for bit as it would alone with
 * one node per thread, with two it agrees to FP rounding. */
typedef struct lbm_batch_s* lbm_batch;

/* p: ncav parameter sets (host); same precision in all.  Initial state as in
 * lbm_init.  Errors: LBM_ERR_ARG (with the cavity index in the message),
 * LBM_ERR_CUDA. */
int lbm_batch_init(const lbm_params* p, int ncav, void* stream, lbm_batch* out);
/* Advances every cavity by nsteps (asynchronous, one launch). */
int lbm_batch_step(lbm_batch b, long nsteps);
/* Mean Nusselt numbers (Eq. 38) of every cavity into host arrays of ncav
 * doubles (either may be NULL); synchronises. */
int lbm_batch_nusselt(lbm_batch b, double* nu_hot, double* nu_cold);
/* Per-cavity divergence status into status[ncav] (may be NULL); returns
 * LBM_ERR_TIMEOUT if a bounded wait (grid barrier or step counter) ran out in any step since the last
 * lbm_batch_set_wait_limit (the lattice is then incomplete), LBM_ERR_DIVERGED
 * if any cavity diverged, else LBM_OK.  Synchronises. */
int lbm_batch_status(lbm_batch b, int* status);
/* FP64 post-stream populations of cavity cav (as lbm_read_state). */
int lbm_batch_read_state(lbm_batch b, int cav, double* f_dev, double* g_dev);
/* Upper bound on the polls (sleeps of 32 ns growing to 1 us between them) a
 * block spends at the grid barrier before it records LBM_ERR_TIMEOUT and
 * leaves the kernel; default 2e7.  Also clears a previous timeout. */
int lbm_batch_set_wait_limit(lbm_batch b, long long polls);
/* Autotuner: times candidate tile shapes (tile_w x tile_h nodes, or runs of
 * tile_w nodes with tile_h = 0), blocks per SM and the three schedules (see
 * lbm_batch_set_tiles) on this batch, keeps the fastest, and records it in a
 * text cache (one line per device, precision and batch shape) at cache_path
 * (NULL: no cache); a cached entry is reused without timing.  Tuning advances
 * the lattices, so the batch is reset to t = 0 afterwards.  Outputs may be
 * NULL. */
int lbm_batch_tune(lbm_batch b, const char* cache_path, int* tile_w, int* tile_h, int* blocks_per_sm);
/* Sets the tile shape (tile_w a power of two >= 32; tile_w x tile_h = 256 or
 * 512 nodes run on 256-thread blocks, 32 or 64 nodes on one-warp blocks; the
 * larger size of each pair is two nodes per thread; tile_h = 0: runs of
 * tile_w consecutive nodes in each cavity's row-major order, wrapping onto
 * the next row, so no lanes idle at a cavity's right edge; tile_h = -1: runs
 * of tile_w (32 to 256) pairs of nodes side by side along x, one pair per
 * thread; tile_h = -2: the same over each cavity's interior pairs, with the
 * wall nodes and their neighbours in tiles of their own, so that no warp of
 * the interior branches into the wall rule), blocks per SM (0 = as
 * many as fit) and the scheduling without timing: dynamic = 0, each block
 * owns a contiguous run of tiles and a grid barrier ends every step; 1, blocks
 * take chunks of 4 tiles from a per-step counter, same barrier; 2, dataflow:
 * blocks take (step, tile) items in order from one counter and an item of
 * step s waits (bounded, like the barrier) only for its own cavity's step
 * s - 1, so no grid-wide barrier.  Resets the batch to t = 0. */
int lbm_batch_set_tiles(lbm_batch b, int tile_w, int tile_h, int blocks_per_sm, int dynamic);
/* Steps taken, number of tiles and blocks of the persistent launch. */
int lbm_batch_query(lbm_batch b, long* t, int* ntiles, int* nblocks);
/* Releases every resource of the batch (synchronises its stream first);
 * NULL is a no-op. */
int lbm_batch_destroy(lbm_batch b);
/* Text of the last error of b, or of the last failed lbm_batch_init or
 * lbm_init when b is NULL; valid until the next call on b. */
const char* lbm_batch_last_error(lbm_batch b);

/* Current time step count and divergence status (synchronises the stream). */
int lbm_query(lbm_handle h, long* t, int* status);

/* Releases every resource of the handle (synchronises its stream). */
int lbm_destroy(lbm_handle h);

/* Text of the last error of h (or of the last failed lbm_init when h is
 * NULL); valid until the next call on h. */
const char* lbm_last_error(lbm_handle h);

#ifdef __cplusplus
}
#endif
#endif
