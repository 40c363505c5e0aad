/*
 * lbm.h -- C ABI of the GB300 library for the consistent two-phase lattice
 * Boltzmann method of Zelko & Duenweg (arXiv:1402.2920): the per-time-step
 * moments / interface force / implicit u-solve / collision / streaming update
 * on the D2Q21 and D3Q59 lattices (Tables I and II).
 *
 * Conventions shared by every entry point
 *   - Return value: 0 (LBM_OK) on success, a negative LBM_E_* code otherwise.
 *     An lbm_sim stays valid (and must still be destroyed) after any error.
 *   - Lattice units: time step h = 1 and lattice spacing a = 1 (captions of
 *     Tables I-III).
 *   - Scalar fields are C order [z][y][x] (x fastest), nx*ny*nz doubles;
 *     vector fields are component-major [d][z][y][x].  2D lattices use
 *     nz = 1 and d = 2.
 *   - Pointers the caller passes are borrowed for the duration of the call
 *     only.  on_device = 1 means the pointer is CUDA device memory of the
 *     device the simulation lives on; 0 means ordinary host memory.
 *   - All device work is issued on the stream given to lbm_create.  Calls
 *     that hand data back (lbm_fields, lbm_populations, lbm_stats_get,
 *     lbm_sync, lbm_save) synchronise that stream and report any error the
 *     device recorded since the previous such call.
 *   - The library owns all device memory it allocates; lbm_destroy frees it.
 *   - There is no CPU fallback: without a usable CUDA device every call that
 *     needs one returns LBM_E_CUDA.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_sim lbm_sim;

/* Velocity sets: Table II (D2Q21) and Table I (D3Q59). */
enum { LBM_D2Q21 = 0, LBM_D3Q59 = 1 };

/* Equation of state p(rho) (App. B; the van der Waals form is the workload's). */
enum { LBM_EOS_VDW = 0, LBM_EOS_PSI_SINE = 1 };

/* Population storage.  F32: n_i as float.  F32_DEV / F16_DEV / BF16_DEV: the
 * deviation n_i - w_i(rho0) rho0 as float / half / bfloat16, with FP32
 * arithmetic.  F64: n_i as double with FP64 arithmetic throughout.
 * F32_LOC / F16_LOC / BF16_LOC: the deviation n_i - w_i(c_s^2(rho_r)) rho_r from the
 * local equilibrium weight of the site r that sent the population (its last
 * collision), which keeps only the velocity and non-equilibrium parts of n_i for
 * rounding; the library keeps each site's w_k rho per shell (8 floats per site and
 * buffer in 3D, 6 in 2D).  These run the u-solve in FP32 (LBM_USOLVE_F64 is refused). */
enum { LBM_STORE_F32 = 0, LBM_STORE_F32_DEV = 1, LBM_STORE_F16_DEV = 2, LBM_STORE_BF16_DEV = 3,
       LBM_STORE_F64 = 4, LBM_STORE_F32_LOC = 5, LBM_STORE_F16_LOC = 6, LBM_STORE_BF16_LOC = 7 };

/* Arithmetic of the implicit u-solve (Sec. IX): the storage's arithmetic, or
 * FP64 sweeps also for the reduced-precision storages. */
enum { LBM_USOLVE_NATIVE = 0, LBM_USOLVE_F64 = 1 };

/* Error codes. */
enum {
    LBM_OK = 0,
    LBM_E_INVALID_ARG = -1,     /* bad pointer, size, enum or parameter                  */
    LBM_E_WEIGHTS = -2,         /* c_s^2 = p/rho left the positive-weight window (Sec. III)
                                   at some site, or a density became non-finite          */
    LBM_E_BULKVISC = -3,        /* EOS admissibility at create (App. B)                  */
    LBM_E_USOLVE_DIVERGED = -4, /* u-solve hit its sweep cap or produced non-finite j~   */
    LBM_E_OOM = -5,             /* device allocation failed                              */
    LBM_E_CUDA = -6,            /* a CUDA call failed or no device is usable             */
    LBM_E_TIMEOUT = -7,         /* a bounded device wait (on a tensor copy) ran out      */
    LBM_E_IO = -8               /* lbm_save / lbm_load file error or mismatched header   */
};

/* Equation of state.
 *   LBM_EOS_VDW:       p = rho T / (1 - b rho) - a rho^2          (uses a, b, T)
 *   LBM_EOS_PSI_SINE:  p = rho c_s^2(rho), c_s^2 = c_s^2(rho1) exp(int_{rho1}^{rho} psi),
 *                      psi = A sin(pi (rho - rho1)/(rho2 - rho1)) on (rho1, 2 rho2 - rho1),
 *                      0 elsewhere (App. B; uses rho1, rho2, A, cs2_rho1). */
typedef struct {
    int kind;
    double a, b, T;
    double rho1, rho2, A, cs2_rho1;
} lbm_eos;

typedef struct {
    double gamma;          /* BGK relaxation parameter, -1 < gamma < 1 (Sec. II)          */
    double kappa;          /* interfacial stiffness, f = kappa rho grad lap rho (Sec. VI) */
    double rho0;           /* reference density of Delta^int, Delta^corr (Secs. VI, VIII)
                              and of the deviation storages                               */
    int storage;           /* LBM_STORE_*                                                 */
    int usolve_precision;  /* LBM_USOLVE_*                                                */
    double usolve_tol;     /* stop when max|j~new - j~| of the plain iteration (S6) and, with
                              relaxation or Chebyshev acceleration, the largest update rho |du|
                              the sweep applied are both <= usolve_tol + usolve_rtol max|j~new|;
                              both <= 0 select the default: 1e-14 for an FP64 u-solve; else
                              5e-9 (32-bit storages) or 4e-8 (16-bit storages), below the
                              rounding noise the stored populations put into j0 each step   */
    double usolve_rtol;
    int usolve_max_iter;   /* sweep cap per u-solve; <= 0 selects 500                     */
    int usolve_warm_start; /* 1: start from the previous step's j~ (Sec. IX item 3); 0: from 0 (S1);
                              2: from j~_n + 0.75 (j~_n - j~_n-1), the last two steps' j~
                              extrapolated (one more 3-vector field on the device, read once
                              per step); other values are LBM_E_INVALID_ARG */
    double rho_check_min;  /* create-time EOS check over [rho_check_min, rho_check_max]:  */
    double rho_check_max;  /* c_s^2 window and positive bulk viscosity (App. B); both 0 skip it */
    double usolve_omega;   /* relaxation of each u-solve sweep, j~ += omega (J(j~) - j~), with J
                              the update of S3-S5.  1: the plain iteration of Sec. IX; any value
                              in (0, 2) converges to the same fixed point when the bulk viscosity
                              is positive (the iteration operator is then positive semidefinite
                              with spectral radius below 1).  0 selects 2/(2 - g), g the largest
                              frozen-coefficient eigenvalue over [rho_check_min, rho_check_max]
                              (1 when no range is given).                                   */
    int usolve_chebyshev;  /* 1: Chebyshev acceleration of the sweeps for the spectrum [0, g] of
                              the iteration (g as for usolve_omega; needs the density range),
                              about half the sweeps of the best plain relaxation; it falls
                              back to plain sweeps within a solve if the residual grows.  The
                              fixed point, and so the result up to the tolerance, is unchanged */
} lbm_params;

typedef struct {
    double mass;              /* sum over sites of rho, FP64                              */
    double mom[3];            /* sum over sites of sum_i n_i c_i, FP64                    */
    int64_t steps;            /* time steps taken since lbm_init / lbm_load               */
    int usolve_iters_last;    /* sweeps of the most recent u-solve                        */
    int usolve_iters_max;     /* largest sweep count since lbm_init                        */
    double usolve_resid;      /* final max|j~new - j~| of the most recent u-solve         */
    int status;               /* device-recorded error bits: 1 weights window, 2 non-finite
                                 density, 4 u-solve cap, 8 non-finite j~                   */
    int64_t usolve_sweeps_total; /* u-solve sweeps since lbm_init (each is two kernels)   */
    int usolve_tensor_copies; /* 1 when the most recent u-solve's sweeps loaded the planes of
                                 interior tiles with tensor copies (TMA), 0 when every tile
                                 copied per thread (2D, LBM_SWEEP_COPY=cp_async, or rows that
                                 are not a multiple of 16 bytes)                        */
} lbm_stats;

/* Create a simulation on the current CUDA device.
 *   lattice: LBM_D2Q21 or LBM_D3Q59.  dims[3] = {nx, ny, nz}, periodic in every
 *   direction; each of nx, ny (and nz in 3D) must be >= 4; nz must be 1 in 2D;
 *   nx*ny*nz < 2^31 sites and ny <= 524280.
 *   cuda_stream: a cudaStream_t (may be NULL for the legacy default stream).
 *   Fails with LBM_E_INVALID_ARG on bad arguments, LBM_E_BULKVISC or LBM_E_WEIGHTS
 *   when the EOS check over [rho_check_min, rho_check_max] fails, LBM_E_OOM when
 *   device memory is short.
 * Two environment variables, read here, select among launch forms that give bitwise the
 * same results: LBM_SWEEP_COPY=cp_async makes every tile of the u-solve sweep copy its
 * planes per thread instead of by tensor copies; LBM_TILE_Z=<n> sets the z-slab depth of
 * the tiled kernels (otherwise chosen from the lattice and the GPU's SM count). */
int lbm_create(int lattice, const int64_t dims[3], const lbm_eos* eos, const lbm_params* params,
               void* cuda_stream, lbm_sim** out);

/* Device bytes a simulation of this shape and storage holds (for admission). */
size_t lbm_footprint_bytes(int lattice, const int64_t dims[3], int storage);

/* Initial condition (the paper is silent; the library's choice): n_i = n_i^eq(rho, u)
 * of Eq. equilibrium with the local c_s^2 = p/rho, and j~ = 0.
 *   rho: N doubles; u: d*N doubles or NULL for u = 0. */
int lbm_init(lbm_sim* sim, const double* rho, const double* u, int on_device);

/* Advance nsteps >= 0 full time steps S1..S12 of the Supplemental Material:
 * moments and EOS (S1), interface force and j0' (S2), implicit u-solve (S3-S8),
 * derivative fields, Sigma and Xi' (S10-S11), collision with the bulk, interface
 * and correction operators (Eq. CollisionOperator) and push streaming
 * n_i(r + c_i) = n_i(r) + Delta_i (S11, S12).  Asynchronous on the stream: each
 * step is a CUDA graph whose u-solve loop runs on the device.  With the
 * environment variable LBM_LAUNCH=direct the same kernels are launched one by
 * one and the loop is driven from the host (for profilers that cannot see into
 * conditional graphs); results are identical. */
int lbm_step(lbm_sim* sim, int64_t nsteps);

/* Hydrodynamic fields of the current populations: S1-S8 without collision.
 *   rho: N doubles (may be NULL); u: d*N doubles (may be NULL), u = j/rho of S8.
 * Leaves the warm-start j~ of the simulation unchanged.  Synchronises. */
int lbm_fields(lbm_sim* sim, double* rho, double* u, int on_device);

/* The pre-collision populations n_i(r) as doubles, [Q][N], in the velocity order
 * of lbm_velocities.  Synchronises. */
int lbm_populations(lbm_sim* sim, double* out, int on_device);

/* Overwrite the populations ([Q][N] doubles, lbm_velocities order); j~ is reset to 0. */
int lbm_set_populations(lbm_sim* sim, const double* in, int on_device);

/* Velocity set in the library's order: writes Q*3 ints (c_x, c_y, c_z) to c_out
 * (may be NULL) and returns Q (21 or 59), or LBM_E_INVALID_ARG. */
int lbm_velocities(int lattice, int* c_out);

/* Conservation sums (FP64, fixed reduction order), step counter and u-solve
 * statistics.  Synchronises. */
int lbm_stats_get(lbm_sim* sim, lbm_stats* out);

/* Kernel timing (tracing aid).  Each kernel of the time step is launched reps >= 1
 * times back to back, after one untimed launch, between two CUDA events on the
 * simulation's stream; ms_out[k] receives the average milliseconds per launch of
 * kernel k for k < n, in the order 0 moments (S1), 1 force (S2), 2 one u-solve
 * sweep (S3-S6), 3 derivatives (S8-S11, site-local parts), 4 collision and
 * streaming (S11-S12).  Only per-step temporaries are written,
 * so the simulation's state is unchanged.  Synchronises. */
int lbm_profile(lbm_sim* sim, int reps, double* ms_out, int n);

/* Synchronise the stream; returns the first device-recorded error as an LBM_E_* code. */
int lbm_sync(lbm_sim* sim);

/* Checkpoint: populations in storage format (with the senders' references of the
 * local-reference storages), the warm-start j~, the step counter and
 * the parameters.  lbm_load requires a simulation created with the same lattice,
 * dims and storage; a loaded run continues bitwise like an uninterrupted one. */
int lbm_save(lbm_sim* sim, const char* path);
int lbm_load(lbm_sim* sim, const char* path);

/* Advance several independent simulations: sims[k] by nsteps[k] steps.  Their work is
 * issued on their own streams and may overlap on the device; each result is the same
 * as when that simulation is stepped alone. */
int lbm_step_batch(lbm_sim* const* sims, int n, const int64_t* nsteps);

/* ---------------------------------------------------------------------------
 * Serving: many independent simulations of mixed lattice and size, admitted as they
 * arrive (no counterpart in the paper; the physics of each request is lbm_step's).
 * ------------------------------------------------------------------------- */
typedef struct {
    int lattice;            /* LBM_D2Q21 or LBM_D3Q59                                  */
    int64_t dims[3];        /* as for lbm_create                                       */
    lbm_eos eos;
    lbm_params params;
    int64_t steps;          /* time steps to run (>= 0)                                */
    double arrival_s;       /* arrival time in seconds after lbm_serve starts (>= 0)   */
    const double* rho_init; /* host, N doubles [z][y][x]: initial density (required)   */
    const double* u_init;   /* host, d*N doubles or NULL (u = 0)                       */
    double* rho_out;        /* host, N doubles or NULL: rho after the last step (S1)   */
    double* u_out;          /* host, d*N doubles or NULL: u after the last step (S8)   */
} lbm_request;

typedef struct {
    double admit_s;         /* when the request got its slot (-1: never admitted)      */
    double finish_s;        /* when its result was in the host buffers                 */
    int status;             /* LBM_OK or the request's own error code                  */
    int64_t steps_done;
    size_t footprint;       /* device bytes it was admitted with                       */
} lbm_request_result;

typedef struct {
    size_t memory_budget;   /* device bytes for simulations; 0: 90 % of free memory     */
    int max_active;         /* simulations resident at once                             */
    int chunk_steps;        /* steps issued to a simulation per turn of the loop        */
    int batched;            /* 0: one stream and one graph launch per simulation; 1: the resident
                               simulations of each kernel combination (lattice, storage, u-solve
                               precision, gamma = 0 or not) and size class (sites within a factor
                               of 4) step together, one persistent launch per stage over all of
                               them, at most 32 per batch.  Both give the same results; on the
                               seeded serving workload the per-stream form serves more site
                               updates per second at lower latency                            */
} lbm_serve_config;

/* Run a stream of requests to completion on the current device (continuous batching).
 *   A request is admitted once it has arrived, a slot is free and its footprint
 *   (lbm_footprint_bytes) fits in the budget beside the running ones, in arrival order.
 *   Admitted simulations stay resident and advance chunk_steps at a time: with batched = 1
 *   in batched launches per kernel combination (a combination's batch takes its next chunk
 *   once the previous one has finished, admitting waiting requests in between; the
 *   combinations run on streams of their own), with batched = 0 each on its own stream.
 *   Finished ones hand their fields to rho_out / u_out, free their slot and memory, and
 *   the next arrivals take them.  Each result equals that of the same simulation stepped
 *   alone.  Blocks until every
 *   request is done; per-request times and statuses go to out[n].  A request that can
 *   never fit gets LBM_E_OOM, an invalid one LBM_E_INVALID_ARG; neither stops the
 *   others.  Returns LBM_E_INVALID_ARG for bad arguments, LBM_E_CUDA when streams or
 *   events cannot be made, LBM_OK otherwise.  Caller buffers are borrowed until the
 *   call returns. */
int lbm_serve(const lbm_request* reqs, int n, const lbm_serve_config* cfg, lbm_request_result* out);

/* Static description of an error code. */
const char* lbm_error_string(int code);

/* Mass and momentum of a population array, computed without allocating anything.
 *   The sums are those lbm_stats_get reports, rho = sum_i n_i and j = sum_i n_i c_i
 *   over all sites.  The paper has no counterpart of this entry point: it exists for
 *   callers that may not use the device allocator, such as a serving
 *   loop that has handed its whole memory budget to admitted simulations, or a monitor
 *   of running simulations that must not synchronise the device.
 *   lattice: LBM_D2Q21 or LBM_D3Q59.  pops: device pointer to FP64 populations
 *   [Q][n_sites], in the velocity order of lbm_velocities (the layout lbm_populations
 *   writes).  n_sites: 1 .. 67,108,864 (= 4096 blocks x 256 threads x 64 sites, the
 *   capacity of the library's fixed scratch array); larger counts return
 *   LBM_E_INVALID_ARG and launch nothing.  sums: device pointer to 4 doubles that
 *   receive (mass, j_x, j_y, j_z); j_z = 0 in 2D.  cuda_stream: the stream the two
 *   kernels run on (NULL: legacy default stream); the call does not synchronise.
 *   Caller memory is borrowed for the duration of the kernels.
 *   Scratch: one 128 KB device array per device, shared by all calls; its address is
 *   looked up (cudaGetSymbolAddress) on the first call made on each device, with that
 *   device current, so make that first call before any stream capture starts.  The
 *   address is kept for the life of the process: after cudaDeviceReset (or anything
 *   else that replaces the device's primary context) do not call this again.  Nothing
 *   in the scratch must start at zero.  Calls on one device whose kernels may overlap
 *   (different streams, or host threads) race on the scratch; calls ordered on one
 *   stream do not.  Errors: LBM_E_INVALID_ARG (lattice, NULL pointer, n_sites out of
 *   range), LBM_E_CUDA (no device, launch failure). */
int lbm_moment_sums_noalloc(int lattice, const double* pops, int64_t n_sites, double* sums, void* cuda_stream);

/* Tensor cores for the collision's polynomial map, measured against the scalar form.
 *   With gamma = 0 each post-collision population of D3Q59 is W_k P(c_i) + w_k(rho0) H(c_i)
 *   (S11; n^eq of Sec. III, Delta^int and Delta^corr of Secs. VI and VIII), P and H polynomials
 *   in c with 10 and 20 coefficients per site.  This times that map over n_sites synthetic
 *   sites two ways: the scalar per-pair form the collision kernel uses, and one tcgen05 matrix
 *   product per tile of 128 sites ([128 x 32] coefficients, split into two TF32 terms, times
 *   the [32 x 128] table of monomials, accumulator in tensor memory).  Each form reduces a
 *   site's 59 values to one weighted sum; the two sums are compared on the host.
 *   n_sites: a multiple of 128, at most 2^31.  reps >= 1 timed repetitions after one warm-up.
 *   Outputs (host): milliseconds per pass of each form, the largest difference of the two
 *   per-site sums and the largest sum.  Allocates and frees its own device buffers; runs on
 *   the legacy default stream and synchronises.  Errors: LBM_E_INVALID_ARG, LBM_E_OOM,
 *   LBM_E_CUDA, LBM_E_TIMEOUT (a tensor-core completion wait ran out). */
int lbm_collision_map_bench(int64_t n_sites, int reps, double* ms_scalar, double* ms_tensor, double* max_abs_diff,
                            double* max_abs_value);

/* Free a simulation and its device memory.  NULL is accepted. */
void lbm_destroy(lbm_sim* sim);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
