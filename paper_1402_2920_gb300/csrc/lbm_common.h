// Host/device shared declarations of the CUDA library: the parameter block
// every kernel receives by value, the device-resident u-solve control word,
// and the kernel table each lattice translation unit exports.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda.h>
#include <cuda_runtime.h>

namespace lbm {

enum Store { ST_F32 = 0, ST_F32_DEV = 1, ST_F16_DEV = 2, ST_BF16_DEV = 3, ST_F64 = 4, ST_F32_LOC = 5, ST_F16_LOC = 6,
             ST_BF16_LOC = 7 };

// Device-resident state of one implicit u-solve (Sec. IX): which of the two
// j~ buffers is current, the sweep counter and the residual reductions.
struct UsolveState {
    unsigned long long resid_bits;  // atomicMax over |j~new - j~| (non-negative double bits)
    unsigned long long jmax_bits;   // atomicMax over |j~new|
    int cur;                        // buffer holding the current j~
    int iter;                       // sweeps of the solve in progress
    int iters_last;                 // sweeps of the last finished solve
    int iters_max;                  // largest sweep count since init
    double resid_last;              // final residual of the last finished solve
    int converged;                  // 1 once the last solve met its tolerance
    int running;                    // 1 from k_us_begin until the control kernel stops the loop
    long long sweeps_total;         // sweeps since the last reset
    // the update of the next sweep: d = c1 d_prev + c2 (J(j~) - j~), j~ += d
    double c1, c2;
    double cheb_rho;                // Chebyshev recurrence variable
    double cheb_sigma, cheb_delta;  // this solve's spectrum [1 - g, 1] of I - A (theta = 1 - g/2)
    double gain;                    // this solve's bound g, from the density range of the state
    double resid_min;               // smallest residual of the solve so far (divergence guard)
    int mode;                       // 1: Chebyshev acceleration, 0: plain relaxation
    int wsel;                       // pair 0: the warm-start buffer holding the newest j~ (see jwp)
    int tma;                        // 1 once a sweep of this solve loaded planes by tensor copies
};

// planes ahead of the one in work whose per-site inputs the collision and derivative
// kernels prefetch into L2 (measured at 256^3)
constexpr int kCollideLead = 1;
constexpr int kDerivsLead = 1;

// slots of the density-range reduction (spread so that block atomics do not contend)
constexpr int kRangeSlots = 64;

// Launch shape of the FP64 conservation sums (fixed, so the reduction order is fixed).
constexpr int kRedBlock = 256;
constexpr int kRedGrid = 1024;

// Error bits recorded by kernels (read back by lbm_sync and friends).
enum StatusBits { STB_WEIGHTS = 1, STB_NONFINITE_RHO = 2, STB_USOLVE_CAP = 4, STB_USOLVE_NAN = 8, STB_TIMEOUT = 16 };

// Physical parameters and derived constants in the kernel arithmetic T, filled on the
// host so that device code neither converts from double nor divides per site.
template <typename T>
struct Phys {
    T rho0, cs0, gamma, kappa, omega;
    T a, b, Teos, bT, g0;                 // van der Waals; bT = b T, g0 = 1 - b rho0
    T F0, F0lo, b2T_g02;                  // slope of c_s^2 = p/rho at rho0, b T / g0^2 - a, as a pair
                                          // F0 + F0lo; and b^2 T / g0^2 (c_s^2 differences)
    T rho1, rho3, cs2_1, A, pi_D, A_pi_D, AD_pi, ph0;  // psi-sine: pi/D, A pi/D, A D/pi, phase at rho0
    T cs2_lo, cs2_hi;                     // positive-weight window
    T w0[8], off[8];                      // w_k(c_s^2(rho0)) and w_k rho0 per shell
    T isc[8];                             // 1 / w_k(c_s^2(rho0)): scale of the half storage
    T offc[8];                            // w_k rho0 (FP64) minus off[k] in this precision
    T k1, k2, k3;                         // prefactors of Sigma (two) and Xi' (Sec. VIII, S11)
    T cf_int, cf_jt, cf_h2, cf_h3, cj;    // (1+g)/(2 cs0), (g-1)/cs0, 1/(2 cs0^2), 1/(6 cs0^3), (1-g) cs0
};

// Everything a kernel needs, passed by value (lives in the kernel parameter space).
struct DevSim {
    int lattice, d, Q;
    int nx, ny, nz;
    long long N;          // sites
    // fields
    void* pop[2];         // populations, [Q][N] in the storage type
    void* pop0[2];        // float2 [N]: the rest population of the reduced storages as a float
                          // pair hi + lo; unused for FP64 storage
    void* rho_lo;         // float [N]: rho - rho0 minus its float rounding (reduced storages)
    void* rho;            // T [N]: rho - rho0 (exact differences; rho0 + it recovers rho)
    void* j0p;            // T [3][N]: j0 after S1, j0' = j0 + f/2 after S2
    void* f;              // T [3][N]: interface force
    void* uit[2][2];      // U [3][N]: u iterates of the u-solve, ping-pong, for pair 0 (the run)
                          // and pair 1 (lbm_fields); u = (j0' + j~)/rho (S3)
    void* jt_warm;        // U [nw][3][N]: j~ = rho u - j0' of the last step, the warm start (Sec. IX),
                          // and with the extrapolated start (warm = 2) that of the step before
    void* aux;            // T [26][N]: A, B_ab, C_a, the local part of Sigma_ab, Xi'_abc
    float* wref[2];       // [NSHELL][N] per population buffer (local-reference storages): w_k(c_s^2(rho)) rho
                          // of every site at the collision that sent the populations in that buffer
    UsolveState* us;      // [2]: pair 0 and pair 1
    unsigned* range;      // [2][2][kRangeSlots]: float bits of min and max density per pair
    int* status;          // error bits
    int aligned16;        // 1: every field array starts on a 16-byte boundary (vector copies allowed)
    double* red;          // reduction scratch
    // physics
    double gamma, kappa, rho0, cs0;  // cs0 = c_s^2(rho0)
    double w0[8];                    // w_k(c_s^2(rho0)) per shell
    double off[8];                   // w_k(c_s^2(rho0)) rho0: offsets of the deviation storages
    int eos_kind;
    double a, b, T;
    double rho1, rho2, A, cs2_1;
    double cs2_lo, cs2_hi;           // positive-weight window (Sec. III)
    double tol, rtol;
    double omega;                    // relaxation of the u-solve sweep (1 = the plain iteration);
                                     // 0: 2/(2 - g) with g the bound of each solve
    int cheb;                        // Chebyshev acceleration of the sweeps
    double s2max;                    // max over k of |s(k)|^2 of the first-derivative symbol (1D)
    void* dvec[2];                   // U [3][N]: previous update of the u-solve, pair 0 and 1
    int maxit;
    int warm;                        // u-solve start: 0 j~ = 0, 1 the last step's j~, 2 extrapolated
                                     // from the last two steps' j~ (see jwp)
    double wtheta;                   // warm = 2: j~ start = j~_n + wtheta (j~_n - j~_n-1)
    Phys<float> pf;                  // the same parameters for FP32 arithmetic
    Phys<double> pd;                 // and for FP64 arithmetic
    // Tensor maps of the sweep's plane loads (TMA) in device memory, valid when tma = 1.
    const struct SweepMaps* tmaps;
    // plane i of population buffer b, pop[b] + i N elements: the collision's stores address their
    // plane through this table (one parameter load instead of 64-bit index arithmetic per store)
    void* popp[2][59];
    // plane tables of the aux field (aux + c N) and of the 3-vector fields j0', f and the warm-start
    // j~ (field + a N), in the field's element type.  jwp[b]: warm-start buffer b.  The force kernel
    // starts the u-solve from jwp[wsel] (the newest j~) and, for warm = 2, jwp[wsel ^ 1] (the one
    // before); the run's k_us_begin flips wsel, and the collision writes the new j~ over the older
    // one.  With one buffer (warm < 2) both entries name it.
    void* auxp[26];
    void* j0pp[3];
    void* fpp[3];
    void* jwp[2][3];
    int tma;
    int zb;  // z planes per CTA of the tiled kernels (3D; 1 in 2D), chosen at creation
};

// The sweep's tensor maps: the u iterates uit[pair][buffer] as {nx, ny, nz, 3} and rho - rho0
// as {nx, ny, nz}, each loaded in boxes of 40 x 16 sites (the tile with its in-plane halo of 4)
// of one plane.
struct SweepMaps {
    CUtensorMap u[2][2];
    CUtensorMap rho;
};

// Batched launches: up to kBatchSlots simulations of one kernel combination take their time
// steps together, each stage one persistent launch whose blocks walk the work list of all of
// them (a tile or block of one simulation per pass).  The table lives in device memory.
constexpr int kBatchSlots = 32;
struct BatchWork {
    int nslot;                       // slots in use (0 .. kBatchSlots)
    int live[kBatchSlots];           // 1: the slot takes the current step
    int src[kBatchSlots];            // its current population buffer
    int todo[kBatchSlots];           // steps it still takes in the running chunk
    int tstart[kBatchSlots + 1];     // prefix sums of the tiled kernels' tile counts
    int mstart[kBatchSlots + 1];     // prefix sums of the moments kernel's block counts
    int tgx[kBatchSlots], tgy[kBatchSlots];  // tile grid extents in x and y
    int mgx[kBatchSlots], mgy[kBatchSlots];  // moments grid extents in x and y
};

// Kernels of one (lattice, arithmetic, storage, u-solve arithmetic) combination.
struct KernelTable {
    const void* moments;      // (DevSim, int src, int pair)
    const void* force;        // (DevSim, int pair): also the u-solve's starting u
    const void* us_begin;     // (DevSim, int pair)
    const void* sweep;        // (DevSim, int pair): one tiled u-solve sweep, planes copied per thread
    const void* sweep_tma;    // the same with tensor-copy (TMA) plane loads (3D; nullptr in 2D)
    const void* us_ctl;       // (DevSim, int pair, cudaGraphConditionalHandle, int use_cond)
    const void* derivs;       // (DevSim)
    const void* collide;      // (DevSim, int src)
    const void* init_eq;      // (DevSim, const double* rho, const double* u, int dst)
    const void* init_ref;     // (DevSim, const double* rho, int dst): local-reference storages only
    const void* pops_rho;     // (DevSim, const double* pops, double* rho): sum over i of FP64 populations
    const void* fields_out;   // (DevSim, int pair, double* rho, double* u)
    const void* pops_out;     // (DevSim, int src, double* out)
    const void* pops_in;      // (DevSim, const double* in, int dst)
    const void* red_partial;  // (DevSim, int src, double* partials)
    const void* red_final;    // (DevSim, const double* partials, int nparts, double* out)
    // batched forms (const DevSim* sims, BatchWork* work, ...): see BatchWork
    const void* kb_step_begin;  // (sims, work)
    const void* kb_moments;     // (sims, work, int pair)
    const void* kb_force;       // (sims, work, int pair)
    const void* kb_us_begin;    // (sims, work, int pair)
    const void* kb_sweep;       // (sims, work, int pair)
    const void* kb_us_ctl;      // (sims, work, int pair, cudaGraphConditionalHandle)
    const void* kb_derivs;      // (sims, work)
    const void* kb_collide;     // (sims, work)
    const void* kb_step_end;    // (sims, work)
    int block;                // threads per block of the per-site kernels
    int tile[2];              // TX, TY of the tiled kernels (the z-slab depth is DevSim::zb)
    int tile_threads;
    size_t smem_force, smem_sweep, smem_derivs, smem_collide;  // dynamic shared memory bytes
    size_t tsize, usize, ssize;  // bytes of T, U and the storage type
    size_t rsize;                // bytes of a rest-plane element (0: no separate plane)
    int sweep_box[2];            // in-plane box of the sweep's plane loads (tile plus halo 4)
    bool exact;                  // float-pair density bookkeeping (rho_lo is used)
    bool local_ref;              // the storage is relative to the sender's w_k rho (DevSim::wref)
};

// Exported by the lattice translation units.
// read_pops: the collision needs the pre-collision populations (gamma != 0).
bool get_kernels_d2q21(int storage, bool usolve_f64, bool read_pops, KernelTable* out);
bool get_kernels_d3q59(int storage, bool usolve_f64, bool read_pops, KernelTable* out);

}  // namespace lbm
