// Host side of the C ABI declared in include/lbm.h.
//
// A simulation owns its device buffers and four CUDA graphs: one time step
// and two time steps, each for either population buffer as the source.  A
// time step is the chain moments -> force -> u-solve -> derivatives ->
// collide; the u-solve is a WHILE conditional node whose body is one Jacobi
// sweep (q, j~new) followed by a one-thread control kernel that tests
// convergence on the device and sets the loop condition, so a step never
// returns to the host.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include <cudaTypedefs.h>

#include "lbm.h"
#include "lbm_batch.h"
#include "lbm_common.h"
#include "lbm_lattice.h"

using namespace lbm;

namespace {

constexpr int MAX_AUX = 26;
// extrapolation factor of the u-solve start j~_n + theta (j~_n - j~_n-1) (usolve_warm_start = 2):
// of 0.5, 0.75 and 1 measured on the 256^3 spinodal, 0.75 took the fewest sweeps over steps 6-25
// (5.95 against 6.35 and 6.4) at one sweep per step later on
constexpr double kWarmTheta = 0.75;

struct Graphs {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t x = nullptr;
};

}  // namespace

struct lbm_sim {
    int device = 0;
    cudaStream_t stream = nullptr;
    int lattice = 0, d = 0, Q = 0;
    int64_t dims[3] = {0, 0, 0};
    lbm_eos eos{};
    lbm_params prm{};
    KernelTable kt{};
    const void* sweep = nullptr;  // the sweep kernel in use: kt.sweep, or kt.sweep_tma when selected
    DevSim dev{};
    int cur = 0;  // population buffer holding the current pre-collision populations
    int64_t steps = 0;
    std::vector<void*> allocs;
    double* red_part = nullptr;
    double* red_out = nullptr;
    Graphs one[2], two[2];
    bool graphs = false;  // the step graphs are built on the first lbm_step
};

namespace {

#define LBM_CK(call)                                                  \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) {                                      \
            (void)cudaGetLastError();                                 \
            return e_ == cudaErrorMemoryAllocation ? LBM_E_OOM : LBM_E_CUDA; \
        }                                                             \
    } while (0)

int nblocks(long long N, int block) { return int((N + block - 1) / block); }

// grid of the tiled kernels: one CTA per TX x TY column tile and z-slab
dim3 tile_grid(const lbm_sim* s);
dim3 moments_grid(const lbm_sim* s);
int moments_block(const lbm_sim* s);
cudaError_t launch_moments(const lbm_sim* s, DevSim dv, int src, int pair);

void host_eos(const lbm_eos& e, double rho, double out[4])
{
    double p, dp, d2p;
    if (e.kind == LBM_EOS_VDW) {
        const double g = 1.0 - e.b * rho;
        p = rho * e.T / g - e.a * rho * rho;
        dp = e.T / (g * g) - 2.0 * e.a * rho;
        d2p = 2.0 * e.b * e.T / (g * g * g) - 2.0 * e.a;
    } else {
        const double D = e.rho2 - e.rho1, rho3 = 2.0 * e.rho2 - e.rho1;
        double psi = 0.0, dpsi = 0.0, integ = 0.0;
        if (rho > e.rho1 && rho < rho3) {
            const double ph = M_PI * (rho - e.rho1) / D;
            psi = e.A * std::sin(ph);
            dpsi = e.A * M_PI / D * std::cos(ph);
            integ = e.A * D / M_PI * (1.0 - std::cos(ph));
        }
        const double cs2 = e.cs2_rho1 * std::exp(integ);
        p = rho * cs2;
        dp = cs2 * (1.0 + rho * psi);
        d2p = cs2 * psi * (1.0 + rho * psi) + cs2 * (psi + rho * dpsi);
    }
    out[0] = p;
    out[1] = dp;
    out[2] = p - rho * dp;
    out[3] = rho * d2p;
}

template <int LAT>
double host_weight(int k, double s)
{
    using L = Lat<LAT>;
    return L::wc(k, 0) + s * (L::wc(k, 1) + s * (L::wc(k, 2) + s * L::wc(k, 3)));
}

template <int LAT>
double min_weight(double s)
{
    double m = 1e300;
    for (int k = 0; k < Lat<LAT>::NSHELL; ++k) m = std::fmin(m, host_weight<LAT>(k, s));
    return m;
}

// edges of the interval around s_in where every shell weight is positive
template <int LAT>
void weight_window(double& lo, double& hi)
{
    const double s_in = 0.6;  // inside the window of both lattices
    double a = 0.01, b = s_in;
    for (int it = 0; it < 200; ++it) {
        const double m = 0.5 * (a + b);
        (min_weight<LAT>(m) > 0.0 ? b : a) = m;
    }
    lo = b;
    a = s_in;
    b = 3.0;
    for (int it = 0; it < 200; ++it) {
        const double m = 0.5 * (a + b);
        (min_weight<LAT>(m) > 0.0 ? a : b) = m;
    }
    hi = a;
}

// The parameters and derived constants of the kernels in arithmetic T (see Phys).
template <typename T>
void fill_phys(Phys<T>& q, const DevSim& dv, const lbm_eos& e)
{
    const double g = dv.gamma, c0 = dv.cs0;
    q.rho0 = T(dv.rho0);
    q.cs0 = T(c0);
    q.gamma = T(g);
    q.kappa = T(dv.kappa);
    q.omega = T(dv.omega);
    q.a = T(e.a);
    q.b = T(e.b);
    q.Teos = T(e.T);
    q.bT = T(e.b * e.T);
    q.g0 = T(1.0 - e.b * dv.rho0);
    {
        const double g0 = 1.0 - e.b * dv.rho0;
        const double F0 = e.b * e.T / (g0 * g0) - e.a;
        q.F0 = T(F0);
        q.F0lo = T(F0 - double(T(F0)));
        q.b2T_g02 = T(e.b * e.b * e.T / (g0 * g0));
    }
    const double D = e.kind == LBM_EOS_PSI_SINE ? e.rho2 - e.rho1 : 1.0;
    q.rho1 = T(e.rho1);
    q.rho3 = T(2.0 * e.rho2 - e.rho1);
    q.cs2_1 = T(e.cs2_rho1);
    q.A = T(e.A);
    q.pi_D = T(M_PI / D);
    q.A_pi_D = T(e.A * M_PI / D);
    q.AD_pi = T(e.A * D / M_PI);
    q.ph0 = T(M_PI * (dv.rho0 - e.rho1) / D);
    q.cs2_lo = T(dv.cs2_lo);
    q.cs2_hi = T(dv.cs2_hi);
    for (int k = 0; k < 8; ++k) {
        q.w0[k] = T(dv.w0[k]);
        q.off[k] = T(dv.off[k]);
        q.offc[k] = T(dv.off[k] - double(T(dv.off[k])));
        q.isc[k] = dv.w0[k] > 0.0 ? T(1.0 / dv.w0[k]) : T(0);
    }
    q.k1 = T(-0.25 * (g + 1.0) * (g + 1.0) / (g - 1.0));
    q.k2 = T((1.0 / 6.0) * (g * g + 4.0 * g + 1.0) / (g - 1.0));
    q.k3 = T((1.0 / 3.0) * (g * g + 4.0 * g + 1.0) / (g + 1.0));
    q.cf_int = T(0.5 * (1.0 + g) / c0);
    q.cf_jt = T((g - 1.0) / c0);
    q.cf_h2 = T(0.5 / (c0 * c0));
    q.cf_h3 = T(1.0 / (6.0 * c0 * c0 * c0));
    q.cj = T((1.0 - g) * c0);
}

// warm-start j~ buffers: two for the start extrapolated from the last two steps
int warm_buffers(const DevSim& dv) { return dv.warm == 2 ? 2 : 1; }

bool is_local(int storage)
{
    return storage == LBM_STORE_F32_LOC || storage == LBM_STORE_F16_LOC || storage == LBM_STORE_BF16_LOC;
}

size_t bytes_per_site(int lattice, int storage, size_t* ssize_out = nullptr)
{
    const int Q = lattice == LBM_D3Q59 ? 59 : 21;
    const int naux = lattice == LBM_D3Q59 ? 26 : 13;
    size_t ssize = 4, tsize = 4;
    if (storage == LBM_STORE_F16_DEV || storage == LBM_STORE_BF16_DEV || storage == LBM_STORE_F16_LOC ||
        storage == LBM_STORE_BF16_LOC)
        ssize = 2;
    if (storage == LBM_STORE_F64) ssize = tsize = 8;
    if (ssize_out) *ssize_out = ssize;
    const size_t usize = 8;  // worst case: FP64 u-solve
    const size_t rest = storage == LBM_STORE_F64 ? 0 : 2 * 8 + 4;  // two float-pair rest planes, rho_lo
    // the senders' references of the local-reference storages, one set per population buffer
    const size_t wref = is_local(storage) ? 2 * (lattice == LBM_D3Q59 ? 8 : 6) * 4 : 0;
    // populations (two buffers), rest planes, rho - rho0, j0', f, aux; u iterates (2 x 2),
    // warm-start j~ (two buffers with the extrapolated start) and the two Chebyshev update vectors
    return 2 * Q * ssize + rest + wref + tsize * (1 + 3 + 3 + naux) + usize * (4 * 3 + 2 * 3 + 2 * 3);
}

int validate(int lattice, const int64_t dims[3], int storage)
{
    if (lattice != LBM_D2Q21 && lattice != LBM_D3Q59) return LBM_E_INVALID_ARG;
    if (!dims) return LBM_E_INVALID_ARG;
    if (storage < LBM_STORE_F32 || storage > LBM_STORE_BF16_LOC) return LBM_E_INVALID_ARG;
    if (dims[0] < 4 || dims[1] < 4) return LBM_E_INVALID_ARG;
    if (lattice == LBM_D2Q21 && dims[2] != 1) return LBM_E_INVALID_ARG;
    if (lattice == LBM_D3Q59 && dims[2] < 4) return LBM_E_INVALID_ARG;
    if (dims[0] > (1 << 20) || dims[1] > (1 << 20) || dims[2] > (1 << 20)) return LBM_E_INVALID_ARG;
    const double N = double(dims[0]) * double(dims[1]) * double(dims[2]);
    const int Q = lattice == LBM_D3Q59 ? 59 : 21;
    if (N * Q > 9.0e18 / 8.0) return LBM_E_INVALID_ARG;
    // site indices inside a plane stack are 32-bit in the streaming kernel; the tiled
    // kernels' grid has ceil(ny / 16) <= 65535 rows
    if (N >= 2147483648.0 || dims[1] > 65535 * 8) return LBM_E_INVALID_ARG;
    return LBM_OK;
}

cudaError_t add_kernel(cudaGraph_t g, cudaGraphNode_t* out, const void* fn, dim3 grid, int block, void** args,
                       const cudaGraphNode_t* deps, size_t ndeps, size_t smem = 0)
{
    cudaKernelNodeParams kp{};
    kp.func = const_cast<void*>(fn);
    kp.gridDim = grid;
    kp.blockDim = dim3(block);
    kp.sharedMemBytes = (unsigned)smem;
    kp.kernelParams = args;
    kp.extra = nullptr;
    return cudaGraphAddKernelNode(out, g, deps, ndeps, &kp);
}

// Append one time step (source buffer src) to graph g after dependency dep.
int add_step(lbm_sim* s, cudaGraph_t g, cudaGraphNode_t dep, int src, cudaGraphNode_t* last)
{
    DevSim& dv = s->dev;
    const int B = s->kt.block;
    const int G = nblocks(dv.N, B);
    int pair = 0, one = 1;
    cudaGraphNode_t n1, n2, n3, nc, n5, n6;
    const cudaGraphNode_t* d0 = dep ? &dep : nullptr;
    size_t nd0 = dep ? 1 : 0;
    {
        void* a[] = {&dv, &src, &pair};
        LBM_CK(add_kernel(g, &n1, s->kt.moments, moments_grid(s), moments_block(s), a, d0, nd0));
    }
    const dim3 TG = tile_grid(s);
    const int TB = s->kt.tile_threads;
    {
        void* a[] = {&dv, &pair};
        LBM_CK(add_kernel(g, &n2, s->kt.force, TG, TB, a, &n1, 1, s->kt.smem_force));
    }
    {
        void* a[] = {&dv, &pair};
        LBM_CK(add_kernel(g, &n3, s->kt.us_begin, dim3(1), 32, a, &n2, 1));
    }
    cudaGraphConditionalHandle h;
    LBM_CK(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    LBM_CK(cudaGraphAddNode(&nc, g, &n3, nullptr, 1, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    {
        cudaGraphNode_t b1, b3;
        void* a1[] = {&dv, &pair};
        LBM_CK(add_kernel(body, &b1, s->sweep, TG, TB, a1, nullptr, 0, s->kt.smem_sweep));
        void* a3[] = {&dv, &pair, &h, &one};
        LBM_CK(add_kernel(body, &b3, s->kt.us_ctl, dim3(1), 1, a3, &b1, 1));
    }
    {
        void* a[] = {&dv};
        LBM_CK(add_kernel(g, &n5, s->kt.derivs, TG, TB, a, &nc, 1, s->kt.smem_derivs));
    }
    {
        void* a[] = {&dv, &src};
        LBM_CK(add_kernel(g, &n6, s->kt.collide, TG, TB, a, &n5, 1, s->kt.smem_collide));
    }
    *last = n6;
    return LBM_OK;
}

int build_graphs(lbm_sim* s)
{
    for (int src = 0; src < 2; ++src) {
        LBM_CK(cudaGraphCreate(&s->one[src].g, 0));
        cudaGraphNode_t last;
        int rc = add_step(s, s->one[src].g, nullptr, src, &last);
        if (rc) return rc;
        LBM_CK(cudaGraphInstantiate(&s->one[src].x, s->one[src].g, 0));
        LBM_CK(cudaGraphCreate(&s->two[src].g, 0));
        cudaGraphNode_t mid;
        rc = add_step(s, s->two[src].g, nullptr, src, &mid);
        if (rc) return rc;
        rc = add_step(s, s->two[src].g, mid, src ^ 1, &last);
        if (rc) return rc;
        LBM_CK(cudaGraphInstantiate(&s->two[src].x, s->two[src].g, 0));
    }
    return LBM_OK;
}

// Device buffers come from the stream-ordered allocator on the simulation's stream:
// creating and destroying simulations (a serving loop does it per request) then
// neither synchronises the device nor stalls the other simulations' streams.
int dev_alloc(lbm_sim* s, void** p, size_t bytes)
{
    cudaError_t e = cudaMallocAsync(p, bytes, s->stream);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        *p = nullptr;
        return e == cudaErrorMemoryAllocation ? LBM_E_OOM : LBM_E_CUDA;
    }
    s->allocs.push_back(*p);
    return LBM_OK;
}

template <class... A>
cudaError_t launch(const lbm_sim* s, const void* fn, int grid, int block, A... args)
{
    void* a[] = {&args...};
    return cudaLaunchKernel(fn, dim3(grid), dim3(block), a, 0, s->stream);
}

template <class... A>
cudaError_t launch_tiled(const lbm_sim* s, const void* fn, size_t smem, A... args)
{
    void* a[] = {&args...};
    return cudaLaunchKernel(fn, tile_grid(s), dim3(s->kt.tile_threads), a, smem, s->stream);
}

int read_status(lbm_sim* s, int* bits)
{
    int st = 0;
    LBM_CK(cudaMemcpyAsync(&st, s->dev.status, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    LBM_CK(cudaStreamSynchronize(s->stream));
    if (st) {
        const int z = 0;
        LBM_CK(cudaMemcpyAsync(s->dev.status, &z, sizeof(int), cudaMemcpyHostToDevice, s->stream));
        LBM_CK(cudaStreamSynchronize(s->stream));
    }
    *bits = st;
    return LBM_OK;
}

int status_code(int bits)
{
    if (bits & STB_TIMEOUT) return LBM_E_TIMEOUT;
    if (bits & (STB_WEIGHTS | STB_NONFINITE_RHO)) return LBM_E_WEIGHTS;
    if (bits & (STB_USOLVE_CAP | STB_USOLVE_NAN)) return LBM_E_USOLVE_DIVERGED;
    return LBM_OK;
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
using EncodeTiledFn = PFN_cuTensorMapEncodeTiled_v12000;
EncodeTiledFn tensor_map_encoder()
{
    static const EncodeTiledFn fn = []() -> EncodeTiledFn {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
        return reinterpret_cast<EncodeTiledFn>(f);
    }();
    return fn;
}

// Tensor map of a field [ncomp][nz][ny][nx] (rank 3 when ncomp = 1) read in boxes of one plane of
// box_x x box_y sites, out-of-range elements read as zero.
bool encode_plane_map(CUtensorMap* m, void* base, int ncomp, size_t esize, const DevSim& dv, const int box[2])
{
    const EncodeTiledFn enc = tensor_map_encoder();
    if (!enc || !base) return false;
    const cuuint32_t rank = ncomp > 1 ? 4 : 3;
    const cuuint64_t dims[4] = {cuuint64_t(dv.nx), cuuint64_t(dv.ny), cuuint64_t(dv.nz), cuuint64_t(ncomp)};
    const cuuint64_t strides[3] = {cuuint64_t(dv.nx) * esize, cuuint64_t(dv.nx) * cuuint64_t(dv.ny) * esize,
                                   cuuint64_t(dv.N) * esize};
    const cuuint32_t boxd[4] = {cuuint32_t(box[0]), cuuint32_t(box[1]), 1, 1};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    const CUresult r = enc(m, esize == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank, base,
                           dims, strides, boxd, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// The sweep kernel: the tensor-copy (TMA) form, whose tensor maps need a 3D lattice with rows a
// multiple of 16 bytes, or per-thread plane copies (2D, other sizes, or LBM_SWEEP_COPY=cp_async in
// the environment).  The TMA form is the default: at three CTAs per SM it is the faster of the two
// (0.395 against 0.402 ms at 256^3), the copies no longer issued by every thread.
void setup_sweep_maps(lbm_sim* s)
{
    DevSim& dv = s->dev;
    dv.tma = 0;
    dv.tmaps = nullptr;
    s->sweep = s->kt.sweep;
    const char* sel = std::getenv("LBM_SWEEP_COPY");
    if ((sel && std::strcmp(sel, "cp_async") == 0) || !s->kt.sweep_tma) return;
    if (s->d != 3 || !dv.aligned16 || dv.nx % 4 != 0) return;
    SweepMaps m;
    bool ok = true;
    for (int pr = 0; pr < 2; ++pr)
        for (int b = 0; b < 2; ++b)
            ok = ok && encode_plane_map(&m.u[pr][b], dv.uit[pr][b], 3, s->kt.usize, dv, s->kt.sweep_box);
    ok = ok && encode_plane_map(&m.rho, dv.rho, 1, s->kt.tsize, dv, s->kt.sweep_box);
    void* dm = nullptr;
    ok = ok && dev_alloc(s, &dm, sizeof(SweepMaps)) == LBM_OK;
    ok = ok && cudaMemcpyAsync(dm, &m, sizeof(SweepMaps), cudaMemcpyHostToDevice, s->stream) == cudaSuccess &&
         cudaStreamSynchronize(s->stream) == cudaSuccess;  // m lives on this stack
    if (!ok) (void)cudaGetLastError();
    dv.tmaps = ok ? static_cast<const SweepMaps*>(dm) : nullptr;
    dv.tma = ok ? 1 : 0;
    if (ok) s->sweep = s->kt.sweep_tma;
}

int reset_usolve(lbm_sim* s)
{
    UsolveState z[2];
    std::memset(z, 0, sizeof(z));
    LBM_CK(cudaMemcpyAsync(s->dev.us, z, sizeof(z), cudaMemcpyHostToDevice, s->stream));
    std::vector<unsigned> rg(4 * kRangeSlots);
    for (int k = 0; k < 4 * kRangeSlots; ++k) rg[k] = ((k / kRangeSlots) % 2 == 0) ? 0x7f7fffffu : 0u;
    LBM_CK(cudaMemcpyAsync(s->dev.range, rg.data(), rg.size() * sizeof(unsigned), cudaMemcpyHostToDevice, s->stream));
    LBM_CK(cudaStreamSynchronize(s->stream));  // rg lives on this stack
    const size_t jbytes = 3 * size_t(s->dev.N) * s->kt.usize;
    for (int pr = 0; pr < 2; ++pr)
        for (int b = 0; b < 2; ++b) LBM_CK(cudaMemsetAsync(s->dev.uit[pr][b], 0, jbytes, s->stream));
    LBM_CK(cudaMemsetAsync(s->dev.jt_warm, 0, warm_buffers(s->dev) * jbytes, s->stream));
    const int zi = 0;
    LBM_CK(cudaMemcpyAsync(s->dev.status, &zi, sizeof(int), cudaMemcpyHostToDevice, s->stream));
    return LBM_OK;
}

// moments kernel: flat grid, or for the local-reference storages the row grid (x-blocks of
// kMomentsRowBlock threads, y, z), which gives each thread its coordinates
constexpr int kMomentsRowBlock = 128;
dim3 moments_grid(const lbm_sim* s)
{
    if (!s->kt.local_ref) return dim3(nblocks(s->dev.N, s->kt.block));
    return dim3((s->dev.nx + kMomentsRowBlock - 1) / kMomentsRowBlock, s->dev.ny, s->d == 3 ? s->dev.nz : 1);
}
int moments_block(const lbm_sim* s) { return s->kt.local_ref ? kMomentsRowBlock : s->kt.block; }

cudaError_t launch_moments(const lbm_sim* s, DevSim dv, int src, int pair)
{
    void* a[] = {&dv, &src, &pair};
    return cudaLaunchKernel(s->kt.moments, moments_grid(s), dim3(moments_block(s)), a, 0, s->stream);
}

dim3 tile_grid(const lbm_sim* s)
{
    const int* t = s->kt.tile;
    return dim3((s->dev.nx + t[0] - 1) / t[0], (s->dev.ny + t[1] - 1) / t[1],
                s->d == 3 ? (s->dev.nz + s->dev.zb - 1) / s->dev.zb : 1);
}

// z-slab depth of the tiled kernels.  A CTA marches zb planes plus its halo (4 planes; the sweep 9
// phases), and the grid's tiles_xy * ceil(nz / zb) CTAs run in waves of resident CTAs per SM x SMs.
// A last wave that fills the GPU only in part leaves SMs idle for a whole march, so on grids of two
// waves or more the depth in [24, 48] is taken that minimises the sum over the tiled kernels of
// waves x (zb + halo) x the kernel's time per CTA-plane (measured at 256^3 on GB300: force 1.9,
// sweep 2.0 x two sweeps per step, derivatives 2.6, collision 6.7 units).  At 256^3 on 152 SMs
// this gives 37 (1792 CTAs: four waves of the sweep's 456 resident CTAs, where 32 gave 2048 CTAs,
// 4.5 waves); measured, the step's tiled kernels ran 2 to 5 % faster.  Smaller grids keep 32.
// LBM_TILE_Z=<n> in the environment at lbm_create sets the depth (any depth gives the same
// results, bit for bit).
int choose_zb(const lbm_sim* s)
{
    if (s->d != 3) return 1;
    const int nz = s->dev.nz;
    if (const char* env = std::getenv("LBM_TILE_Z")) {
        const int v = std::atoi(env);
        if (v >= 1) return v < nz ? v : nz;
    }
    const int* t = s->kt.tile;
    const long long txy = (long long)((s->dev.nx + t[0] - 1) / t[0]) * ((s->dev.ny + t[1] - 1) / t[1]);
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess || nsm < 1) {
        (void)cudaGetLastError();
        return 32;
    }
    struct Kern {
        const void* fn;
        size_t smem;
        int halo;
        double w;
    } ks[4] = {{s->kt.force, s->kt.smem_force, 4, 1.9},
               {s->sweep, s->kt.smem_sweep, 9, 4.0},
               {s->kt.derivs, s->kt.smem_derivs, 4, 2.6},
               {s->kt.collide, s->kt.smem_collide, 4, 6.7}};
    long long slots[4];
    for (int k = 0; k < 4; ++k) {
        int r = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, ks[k].fn, s->kt.tile_threads, ks[k].smem) != cudaSuccess) {
            (void)cudaGetLastError();
            r = 1;
        }
        slots[k] = (long long)(r > 0 ? r : 1) * nsm;
    }
    auto cost = [&](int zb) {
        const long long ctas = txy * ((nz + zb - 1) / zb);
        double c = 0.0;
        for (int k = 0; k < 4; ++k) c += ks[k].w * double((ctas + slots[k] - 1) / slots[k]) * (zb + ks[k].halo);
        return c;
    };
    if (nz <= 32 || txy * ((nz + 31) / 32) < 2 * slots[1]) return nz < 32 ? nz : 32;
    int best = 32;
    double cbest = cost(32);
    for (int zb = 24; zb <= 48 && zb <= nz; ++zb) {
        const double c = cost(zb);
        if (c < cbest * (1.0 - 1e-9)) {
            best = zb;
            cbest = c;
        }
    }
    return best;
}

// S1-S8 on the current populations with the scratch j~ pair; host-driven loop.
int run_fields(lbm_sim* s)
{
    DevSim& dv = s->dev;
    const int B = s->kt.block, G = nblocks(dv.N, B);
    const int pair = 1;
    LBM_CK(launch_moments(s, dv, s->cur, pair));
    LBM_CK(launch_tiled(s, s->kt.force, s->kt.smem_force, dv, pair));
    LBM_CK(launch(s, s->kt.us_begin, 1, 32, dv, pair));
    cudaGraphConditionalHandle h{};
    const int no = 0;
    for (int it = 0; it < s->dev.maxit + 1; ++it) {
        LBM_CK(launch_tiled(s, s->sweep, s->kt.smem_sweep, dv, pair));
        LBM_CK(launch(s, s->kt.us_ctl, 1, 1, dv, pair, h, no));
        UsolveState u;
        LBM_CK(cudaMemcpyAsync(&u, &dv.us[1], sizeof(u), cudaMemcpyDeviceToHost, s->stream));
        LBM_CK(cudaStreamSynchronize(s->stream));
        if (!u.running) break;  // the control kernel recorded a stop
    }
    return LBM_OK;
}

}  // namespace

extern "C" {

const char* lbm_error_string(int code)
{
    switch (code) {
    case LBM_OK: return "ok";
    case LBM_E_INVALID_ARG: return "invalid argument";
    case LBM_E_WEIGHTS: return "c_s^2 left the positive-weight window or a density became non-finite";
    case LBM_E_BULKVISC: return "equation of state not admissible (bulk viscosity or weights)";
    case LBM_E_USOLVE_DIVERGED: return "u-solve did not converge within its sweep cap";
    case LBM_E_OOM: return "out of device memory";
    case LBM_E_CUDA: return "CUDA error or no usable device";
    case LBM_E_TIMEOUT: return "device wait timed out";
    case LBM_E_IO: return "checkpoint file error";
    default: return "unknown error";
    }
}

int lbm_velocities(int lattice, int* c_out)
{
    if (lattice == LBM_D2Q21) {
        using L = Lat<0>;
        if (c_out)
            for (int i = 0; i < L::Q; ++i) { c_out[3 * i] = L::cx(i); c_out[3 * i + 1] = L::cy(i); c_out[3 * i + 2] = 0; }
        return L::Q;
    }
    if (lattice == LBM_D3Q59) {
        using L = Lat<1>;
        if (c_out)
            for (int i = 0; i < L::Q; ++i) { c_out[3 * i] = L::cx(i); c_out[3 * i + 1] = L::cy(i); c_out[3 * i + 2] = L::cz(i); }
        return L::Q;
    }
    return LBM_E_INVALID_ARG;
}

size_t lbm_footprint_bytes(int lattice, const int64_t dims[3], int storage)
{
    if (validate(lattice, dims, storage) != LBM_OK) return 0;
    const size_t N = size_t(dims[0]) * size_t(dims[1]) * size_t(dims[2]);
    return N * bytes_per_site(lattice, storage) + 64 * 1024;
}

void lbm_destroy(lbm_sim* s)
{
    if (!s) return;
    cudaSetDevice(s->device);
    if (s->stream) cudaStreamSynchronize(s->stream);
    for (int k = 0; k < 2; ++k) {
        if (s->one[k].x) cudaGraphExecDestroy(s->one[k].x);
        if (s->one[k].g) cudaGraphDestroy(s->one[k].g);
        if (s->two[k].x) cudaGraphExecDestroy(s->two[k].x);
        if (s->two[k].g) cudaGraphDestroy(s->two[k].g);
    }
    for (void* p : s->allocs) cudaFreeAsync(p, s->stream);
    if (s->stream) cudaStreamSynchronize(s->stream);
    (void)cudaGetLastError();
    delete s;
}

int lbm_create(int lattice, const int64_t dims[3], const lbm_eos* eos, const lbm_params* params, void* cuda_stream,
               lbm_sim** out)
{
    if (!out || !eos || !params) return LBM_E_INVALID_ARG;
    *out = nullptr;
    int rc = validate(lattice, dims, params->storage);
    if (rc) return rc;
    if (!(params->gamma > -1.0 && params->gamma < 1.0)) return LBM_E_INVALID_ARG;
    if (!(params->kappa >= 0.0) || !(params->rho0 > 0.0)) return LBM_E_INVALID_ARG;
    if (eos->kind != LBM_EOS_VDW && eos->kind != LBM_EOS_PSI_SINE) return LBM_E_INVALID_ARG;
    if (eos->kind == LBM_EOS_PSI_SINE && !(eos->rho2 > eos->rho1 && eos->cs2_rho1 > 0.0)) return LBM_E_INVALID_ARG;
    if (params->usolve_precision != LBM_USOLVE_NATIVE && params->usolve_precision != LBM_USOLVE_F64)
        return LBM_E_INVALID_ARG;

    const int d = lattice == LBM_D3Q59 ? 3 : 2;
    double lo, hi;
    if (lattice == LBM_D3Q59) weight_window<1>(lo, hi); else weight_window<0>(lo, hi);

    // create-time admissibility of the EOS (App. B) over the density range of the run
    double e0[4];
    host_eos(*eos, params->rho0, e0);
    const double cs0 = e0[0] / params->rho0;
    if (!(cs0 > lo && cs0 < hi)) return LBM_E_WEIGHTS;
    if (params->rho_check_max > params->rho_check_min && params->rho_check_min > 0.0) {
        for (int k = 0; k <= 2000; ++k) {
            const double r = params->rho_check_min + (params->rho_check_max - params->rho_check_min) * k / 2000.0;
            double e[4];
            host_eos(*eos, r, e);
            const double cs2 = e[0] / r;
            if (!(cs2 > lo && cs2 < hi)) return LBM_E_WEIGHTS;
            if (!(r * e[1] / e[0] < 1.0 + 2.0 / d)) return LBM_E_BULKVISC;
        }
    }

    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        (void)cudaGetLastError();
        return LBM_E_CUDA;
    }
    lbm_sim* s = new (std::nothrow) lbm_sim();
    if (!s) return LBM_E_OOM;
    cudaGetDevice(&s->device);
    s->stream = static_cast<cudaStream_t>(cuda_stream);
    s->lattice = lattice;
    s->d = d;
    s->Q = lattice == LBM_D3Q59 ? 59 : 21;
    for (int k = 0; k < 3; ++k) s->dims[k] = dims[k];
    s->eos = *eos;
    s->prm = *params;

    const bool f64 = params->storage == LBM_STORE_F64;
    const bool us64 = f64 || params->usolve_precision == LBM_USOLVE_F64;
    const bool read_pops = params->gamma != 0.0;
    bool ok = lattice == LBM_D3Q59 ? get_kernels_d3q59(params->storage, us64, read_pops, &s->kt)
                                   : get_kernels_d2q21(params->storage, us64, read_pops, &s->kt);
    if (!ok) { delete s; return LBM_E_INVALID_ARG; }

    DevSim& dv = s->dev;
    dv.lattice = lattice;
    dv.d = d;
    dv.Q = s->Q;
    dv.nx = int(dims[0]);
    dv.ny = int(dims[1]);
    dv.nz = int(dims[2]);
    dv.N = (long long)dims[0] * dims[1] * dims[2];
    dv.gamma = params->gamma;
    dv.kappa = params->kappa;
    dv.rho0 = params->rho0;
    dv.cs0 = cs0;
    const int nshell = lattice == LBM_D3Q59 ? 8 : 6;
    for (int k = 0; k < 8; ++k) {
        dv.w0[k] = k < nshell ? (lattice == LBM_D3Q59 ? host_weight<1>(k, cs0) : host_weight<0>(k, cs0)) : 0.0;
        dv.off[k] = dv.w0[k] * params->rho0;
    }
    dv.eos_kind = eos->kind;
    dv.a = eos->a; dv.b = eos->b; dv.T = eos->T;
    dv.rho1 = eos->rho1; dv.rho2 = eos->rho2; dv.A = eos->A; dv.cs2_1 = eos->cs2_rho1;
    dv.cs2_lo = lo;
    dv.cs2_hi = hi;
    if (params->usolve_tol > 0.0 || params->usolve_rtol > 0.0) {
        dv.tol = params->usolve_tol > 0.0 ? params->usolve_tol : 0.0;
        dv.rtol = params->usolve_rtol > 0.0 ? params->usolve_rtol : 0.0;
    } else if (us64) {
        dv.tol = 1e-14;
        dv.rtol = 0.0;
    } else {
        // below the rounding noise the stored populations put into j0 each step: tighter
        // stops only chase that noise
        dv.tol = s->kt.ssize == 2 ? 4e-8 : 5e-9;
        dv.rtol = 0.0;
    }
    if (!(params->usolve_omega >= 0.0 && params->usolve_omega < 2.0)) { lbm_destroy(s); return LBM_E_INVALID_ARG; }
    dv.omega = params->usolve_omega;  // 0: 2/(2 - g) per solve
    dv.maxit = params->usolve_max_iter > 0 ? params->usolve_max_iter : 500;
    if (params->usolve_warm_start < 0 || params->usolve_warm_start > 2) { lbm_destroy(s); return LBM_E_INVALID_ARG; }
    dv.warm = params->usolve_warm_start;
    dv.wtheta = kWarmTheta;
    {
        double smax = 0.0;  // max_k |(4/3) sin k - (1/6) sin 2k|, the Sec. IV.B symbol
        for (int k = 0; k <= 20000; ++k) {
            const double x = M_PI * k / 20000.0;
            smax = std::fmax(smax, std::fabs(4.0 / 3.0 * std::sin(x) - std::sin(2.0 * x) / 6.0));
        }
        dv.s2max = smax * smax;
        dv.cheb = params->usolve_chebyshev ? 1 : 0;  // the bound of each solve comes from its density range
    }
    fill_phys<float>(dv.pf, dv, *eos);
    fill_phys<double>(dv.pd, dv, *eos);

    const size_t N = size_t(dv.N);
    const size_t T = s->kt.tsize, U = s->kt.usize, SS = s->kt.ssize;
    rc = LBM_OK;
    rc = rc ? rc : dev_alloc(s, &dv.pop[0], size_t(s->Q) * N * SS);
    rc = rc ? rc : dev_alloc(s, &dv.pop[1], size_t(s->Q) * N * SS);
    if (s->kt.rsize) {  // separate rest plane of the reduced storages
        rc = rc ? rc : dev_alloc(s, &dv.pop0[0], N * s->kt.rsize);
        rc = rc ? rc : dev_alloc(s, &dv.pop0[1], N * s->kt.rsize);
    }
    for (int b = 0; b < 2 && !rc; ++b)
        for (int i = 0; i < s->Q; ++i) dv.popp[b][i] = static_cast<char*>(dv.pop[b]) + size_t(i) * N * SS;
    if (s->kt.exact) rc = rc ? rc : dev_alloc(s, &dv.rho_lo, N * sizeof(float));
    rc = rc ? rc : dev_alloc(s, &dv.rho, N * T);
    rc = rc ? rc : dev_alloc(s, &dv.j0p, 3 * N * T);
    rc = rc ? rc : dev_alloc(s, &dv.f, 3 * N * T);
    for (int pr = 0; pr < 2; ++pr)
        for (int b = 0; b < 2; ++b) rc = rc ? rc : dev_alloc(s, &dv.uit[pr][b], 3 * N * U);
    rc = rc ? rc : dev_alloc(s, &dv.jt_warm, size_t(warm_buffers(dv)) * 3 * N * U);
    if (s->kt.local_ref) {
        const int nshell = lattice == LBM_D3Q59 ? 8 : 6;
        for (int b = 0; b < 2; ++b) {
            void* w = nullptr;
            rc = rc ? rc : dev_alloc(s, &w, size_t(nshell) * N * sizeof(float));
            dv.wref[b] = static_cast<float*>(w);
        }
    }
    if (dv.cheb) {
        rc = rc ? rc : dev_alloc(s, &dv.dvec[0], 3 * N * U);
        rc = rc ? rc : dev_alloc(s, &dv.dvec[1], 3 * N * U);
    }
    rc = rc ? rc : dev_alloc(s, &dv.aux, size_t(MAX_AUX) * N * T);
    if (!rc) {
        for (int c = 0; c < MAX_AUX; ++c) dv.auxp[c] = static_cast<char*>(dv.aux) + size_t(c) * N * T;
        for (int a = 0; a < 3; ++a) {
            dv.j0pp[a] = static_cast<char*>(dv.j0p) + size_t(a) * N * T;
            dv.fpp[a] = static_cast<char*>(dv.f) + size_t(a) * N * T;
            for (int b = 0; b < 2; ++b)
                dv.jwp[b][a] = static_cast<char*>(dv.jt_warm) + size_t((warm_buffers(dv) - 1) * b * 3 + a) * N * U;
        }
    }
    void* usp = nullptr;
    rc = rc ? rc : dev_alloc(s, &usp, 2 * sizeof(UsolveState));
    dv.us = static_cast<UsolveState*>(usp);
    void* rgp = nullptr;
    rc = rc ? rc : dev_alloc(s, &rgp, 4 * kRangeSlots * sizeof(unsigned));
    dv.range = static_cast<unsigned*>(rgp);
    void* stp = nullptr;
    rc = rc ? rc : dev_alloc(s, &stp, 256);
    dv.status = static_cast<int*>(stp);
    void* rp = nullptr;
    rc = rc ? rc : dev_alloc(s, &rp, (kRedGrid * 4 + 8) * sizeof(double));
    s->red_part = static_cast<double*>(rp);
    s->red_out = s->red_part + kRedGrid * 4;
    dv.red = s->red_part;
    if (rc) { lbm_destroy(s); return rc; }
    {  // vector (16-byte) copies of the tiled kernels need 16-byte aligned field arrays
        auto a16 = [](const void* q) { return q == nullptr || (reinterpret_cast<uintptr_t>(q) & 15u) == 0; };
        bool ok = a16(dv.rho) && a16(dv.j0p) && a16(dv.f) && a16(dv.aux) && a16(dv.jt_warm);
        for (int pr = 0; pr < 2; ++pr)
            for (int b = 0; b < 2; ++b) ok = ok && a16(dv.uit[pr][b]);
        dv.aligned16 = ok ? 1 : 0;
    }
    setup_sweep_maps(s);
    dv.zb = choose_zb(s);
    // well-defined contents before the first lbm_init
    for (int b = 0; b < 2; ++b) {
        const size_t wbytes = dv.wref[b] ? size_t(lattice == LBM_D3Q59 ? 8 : 6) * N * sizeof(float) : 0;
        if (cudaMemsetAsync(dv.pop[b], 0, size_t(s->Q) * N * SS, s->stream) != cudaSuccess ||
            (dv.pop0[b] && cudaMemsetAsync(dv.pop0[b], 0, N * s->kt.rsize, s->stream) != cudaSuccess) ||
            (wbytes && cudaMemsetAsync(dv.wref[b], 0, wbytes, s->stream) != cudaSuccess)) {
            lbm_destroy(s);
            return LBM_E_CUDA;
        }
    }
    rc = reset_usolve(s);
    if (!rc && cudaStreamSynchronize(s->stream) != cudaSuccess) rc = LBM_E_CUDA;
    if (rc) { lbm_destroy(s); return rc; }
    *out = s;
    return LBM_OK;
}

int lbm_init(lbm_sim* s, const double* rho, const double* u, int on_device)
{
    if (!s || !rho) return LBM_E_INVALID_ARG;
    LBM_CK(cudaSetDevice(s->device));
    const size_t N = size_t(s->dev.N);
    const double* drho = rho;
    const double* du = u;
    // staging buffer of host inputs, released on every return path (stream-ordered)
    struct Staging {
        double* p = nullptr;
        cudaStream_t st;
        ~Staging() { if (p) (void)cudaFreeAsync(p, st); }
    } stage{nullptr, s->stream};
    double*& tmp = stage.p;
    if (!on_device) {
        LBM_CK(cudaMallocAsync(&tmp, (1 + s->d) * N * sizeof(double), s->stream));
        LBM_CK(cudaMemcpyAsync(tmp, rho, N * sizeof(double), cudaMemcpyHostToDevice, s->stream));
        drho = tmp;
        if (u) {
            LBM_CK(cudaMemcpyAsync(tmp + N, u, s->d * N * sizeof(double), cudaMemcpyHostToDevice, s->stream));
            du = tmp + N;
        }
    }
    int rc = reset_usolve(s);
    if (rc) return rc;
    s->cur = 0;
    s->steps = 0;
    const int B = s->kt.block, G = nblocks(s->dev.N, B);
    if (s->kt.init_ref) LBM_CK(launch(s, s->kt.init_ref, G, B, s->dev, drho, 0));
    LBM_CK(launch(s, s->kt.init_eq, G, B, s->dev, drho, du, 0));
    if (tmp) {
        double* p = tmp;
        tmp = nullptr;
        LBM_CK(cudaFreeAsync(p, s->stream));
    }
    return LBM_OK;
}

}  // extern "C"

namespace {

bool trace_mode()
{
    const char* v = std::getenv("LBM_TRACE");
    return v && v[0] == '1';
}

// One step with every kernel launched on its own and the u-solve loop driven
// from the host (the same kernels and order as the graph).
int step_direct(lbm_sim* s)
{
    DevSim& dv = s->dev;
    const int B = s->kt.block, G = nblocks(dv.N, B);
    const int pair = 0, no = 0, src = s->cur;
    cudaGraphConditionalHandle h{};
    LBM_CK(launch_moments(s, dv, src, pair));
    LBM_CK(launch_tiled(s, s->kt.force, s->kt.smem_force, dv, pair));
    LBM_CK(launch(s, s->kt.us_begin, 1, 32, dv, pair));
    for (int it = 0; it < dv.maxit + 1; ++it) {
        LBM_CK(launch_tiled(s, s->sweep, s->kt.smem_sweep, dv, pair));
        LBM_CK(launch(s, s->kt.us_ctl, 1, 1, dv, pair, h, no));
        UsolveState u;
        LBM_CK(cudaMemcpyAsync(&u, &dv.us[0], sizeof(u), cudaMemcpyDeviceToHost, s->stream));
        LBM_CK(cudaStreamSynchronize(s->stream));
        if (trace_mode())  // the residual history of every u-solve, for tuning the solver
            std::fprintf(stderr, "lbm usolve step %lld sweep %d resid %.3e mode %d next c1 %.4f c2 %.4f\n",
                         (long long)s->steps, u.iter, u.running ? u.resid_min : u.resid_last, u.mode, u.c1, u.c2);
        if (!u.running) break;
    }
    LBM_CK(launch_tiled(s, s->kt.derivs, s->kt.smem_derivs, dv));
    LBM_CK(launch_tiled(s, s->kt.collide, s->kt.smem_collide, dv, src));
    s->cur ^= 1;
    return LBM_OK;
}

bool direct_mode()
{
    const char* v = std::getenv("LBM_LAUNCH");
    return v && std::strcmp(v, "direct") == 0;
}

}  // namespace

extern "C" {

int lbm_step(lbm_sim* s, int64_t nsteps)
{
    if (!s || nsteps < 0) return LBM_E_INVALID_ARG;
    LBM_CK(cudaSetDevice(s->device));
    if (direct_mode()) {
        for (int64_t k = 0; k < nsteps; ++k) {
            const int rc = step_direct(s);
            if (rc) return rc;
            s->steps += 1;
        }
        return LBM_OK;
    }
    if (!s->graphs && nsteps > 0) {  // built on first use: simulations stepped in batches never need them
        const int rc = build_graphs(s);
        if (rc) return rc;
        s->graphs = true;
    }
    int64_t n = nsteps;
    while (n >= 2) {
        LBM_CK(cudaGraphLaunch(s->two[s->cur].x, s->stream));
        n -= 2;
    }
    if (n == 1) {
        LBM_CK(cudaGraphLaunch(s->one[s->cur].x, s->stream));
        s->cur ^= 1;
    }
    s->steps += nsteps;
    return LBM_OK;
}

int lbm_sync(lbm_sim* s)
{
    if (!s) return LBM_E_INVALID_ARG;
    LBM_CK(cudaSetDevice(s->device));
    LBM_CK(cudaStreamSynchronize(s->stream));
    int bits = 0;
    int rc = read_status(s, &bits);
    if (rc) return rc;
    return status_code(bits);
}

int lbm_fields(lbm_sim* s, double* rho, double* u, int on_device)
{
    if (!s) return LBM_E_INVALID_ARG;
    LBM_CK(cudaSetDevice(s->device));
    int rc = run_fields(s);
    if (rc) return rc;
    const size_t N = size_t(s->dev.N);
    const int B = s->kt.block, G = nblocks(s->dev.N, B);
    double* drho = rho;
    double* du = u;
    double* tmp = nullptr;
    if (!on_device && (rho || u)) {
        LBM_CK(cudaMallocAsync(&tmp, (1 + s->d) * N * sizeof(double), s->stream));
        drho = rho ? tmp : nullptr;
        du = u ? tmp + N : nullptr;
    }
    LBM_CK(launch(s, s->kt.fields_out, G, B, s->dev, 1, drho, du));
    if (tmp) {
        if (rho) LBM_CK(cudaMemcpyAsync(rho, drho, N * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
        if (u) LBM_CK(cudaMemcpyAsync(u, du, s->d * N * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
        LBM_CK(cudaFreeAsync(tmp, s->stream));
    }
    LBM_CK(cudaStreamSynchronize(s->stream));
    int bits = 0;
    rc = read_status(s, &bits);
    if (rc) return rc;
    return status_code(bits);
}

int lbm_populations(lbm_sim* s, double* out, int on_device)
{
    if (!s || !out) return LBM_E_INVALID_ARG;
    LBM_CK(cudaSetDevice(s->device));
    const size_t bytes = size_t(s->Q) * size_t(s->dev.N) * sizeof(double);
    double* d = out;
    if (!on_device) LBM_CK(cudaMallocAsync(&d, bytes, s->stream));
    const int B = s->kt.block, G = nblocks(s->dev.N, B);
    LBM_CK(launch(s, s->kt.pops_out, G, B, s->dev, s->cur, d));
    if (!on_device) {
        LBM_CK(cudaMemcpyAsync(out, d, bytes, cudaMemcpyDeviceToHost, s->stream));
        LBM_CK(cudaFreeAsync(d, s->stream));
    }
    LBM_CK(cudaStreamSynchronize(s->stream));
    return LBM_OK;
}

int lbm_set_populations(lbm_sim* s, const double* in, int on_device)
{
    if (!s || !in) return LBM_E_INVALID_ARG;
    LBM_CK(cudaSetDevice(s->device));
    const size_t bytes = size_t(s->Q) * size_t(s->dev.N) * sizeof(double);
    const double* d = in;
    double* tmp = nullptr;
    if (!on_device) {
        LBM_CK(cudaMallocAsync(&tmp, bytes, s->stream));
        LBM_CK(cudaMemcpyAsync(tmp, in, bytes, cudaMemcpyHostToDevice, s->stream));
        d = tmp;
    }
    int rc = reset_usolve(s);
    if (rc) return rc;
    s->cur = 0;
    const int B = s->kt.block, G = nblocks(s->dev.N, B);
    double* rho = nullptr;
    if (s->kt.init_ref) {
        // local-reference storages: every site's references from the density of the given
        // populations, then the populations relative to their senders'
        LBM_CK(cudaMallocAsync(&rho, size_t(s->dev.N) * sizeof(double), s->stream));
        LBM_CK(launch(s, s->kt.pops_rho, G, B, s->dev, d, rho));
        LBM_CK(launch(s, s->kt.init_ref, G, B, s->dev, (const double*)rho, 0));
    }
    LBM_CK(launch(s, s->kt.pops_in, G, B, s->dev, d, 0));
    if (rho) LBM_CK(cudaFreeAsync(rho, s->stream));
    if (tmp) LBM_CK(cudaFreeAsync(tmp, s->stream));
    LBM_CK(cudaStreamSynchronize(s->stream));
    return LBM_OK;
}

int lbm_stats_get(lbm_sim* s, lbm_stats* out)
{
    if (!s || !out) return LBM_E_INVALID_ARG;
    LBM_CK(cudaSetDevice(s->device));
    LBM_CK(launch(s, s->kt.red_partial, kRedGrid, kRedBlock, s->dev, s->cur, s->red_part));
    LBM_CK(launch(s, s->kt.red_final, 1, kRedBlock, s->dev, (const double*)s->red_part, kRedGrid, s->red_out));
    double sums[4];
    UsolveState u;
    int st = 0;
    LBM_CK(cudaMemcpyAsync(sums, s->red_out, sizeof(sums), cudaMemcpyDeviceToHost, s->stream));
    LBM_CK(cudaMemcpyAsync(&u, &s->dev.us[0], sizeof(u), cudaMemcpyDeviceToHost, s->stream));
    LBM_CK(cudaMemcpyAsync(&st, s->dev.status, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    LBM_CK(cudaStreamSynchronize(s->stream));
    out->mass = sums[0];
    out->mom[0] = sums[1];
    out->mom[1] = sums[2];
    out->mom[2] = sums[3];
    out->steps = s->steps;
    out->usolve_iters_last = u.iters_last;
    out->usolve_iters_max = u.iters_max;
    out->usolve_resid = u.resid_last;
    out->status = st;
    out->usolve_sweeps_total = u.sweeps_total;
    out->usolve_tensor_copies = u.tma;
    return LBM_OK;
}

int lbm_profile(lbm_sim* s, int reps, double* ms_out, int n)
{
    if (!s || reps < 1 || !ms_out || n < 0) return LBM_E_INVALID_ARG;
    LBM_CK(cudaSetDevice(s->device));
    DevSim& dv = s->dev;
    const int B = s->kt.block, G = nblocks(dv.N, B);
    const int src = s->cur, pair = 1;
    // the collision kernel rewrites the warm-start j~: keep the run's copy aside
    const size_t jbytes = size_t(warm_buffers(dv)) * 3 * size_t(dv.N) * s->kt.usize;
    void* keep = nullptr;
    LBM_CK(cudaMallocAsync(&keep, jbytes, s->stream));
    LBM_CK(cudaMemcpyAsync(keep, dv.jt_warm, jbytes, cudaMemcpyDeviceToDevice, s->stream));
    cudaEvent_t e0, e1;
    LBM_CK(cudaEventCreate(&e0));
    LBM_CK(cudaEventCreate(&e1));
    // the scratch u-solve pair; the collision writes the spare population buffer
    LBM_CK(launch_moments(s, dv, src, pair));
    LBM_CK(launch_tiled(s, s->kt.force, s->kt.smem_force, dv, pair));
    LBM_CK(launch(s, s->kt.us_begin, 1, 32, dv, pair));
    int rc = LBM_OK;
    for (int k = 0; k < 5 && rc == LBM_OK; ++k) {
        for (int r = 0; r <= reps && rc == LBM_OK; ++r) {
            if (r == 1 && cudaEventRecord(e0, s->stream) != cudaSuccess) rc = LBM_E_CUDA;
            cudaError_t e = cudaSuccess;
            switch (k) {
            case 0: e = launch_moments(s, dv, src, pair); break;
            case 1: e = launch_tiled(s, s->kt.force, s->kt.smem_force, dv, pair); break;
            case 2: e = launch_tiled(s, s->sweep, s->kt.smem_sweep, dv, pair); break;
            case 3: e = launch_tiled(s, s->kt.derivs, s->kt.smem_derivs, dv); break;
            case 4: e = launch_tiled(s, s->kt.collide, s->kt.smem_collide, dv, src); break;
            }
            if (e != cudaSuccess) rc = LBM_E_CUDA;
        }
        if (rc == LBM_OK && cudaEventRecord(e1, s->stream) != cudaSuccess) rc = LBM_E_CUDA;
        if (rc == LBM_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = LBM_E_CUDA;
        float ms = 0.f;
        if (rc == LBM_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = LBM_E_CUDA;
        if (rc == LBM_OK && k < n) ms_out[k] = double(ms) / reps;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    (void)cudaGetLastError();
    // the scratch residual accumulators were left mid-loop: clear them; restore the warm start
    UsolveState u1{};
    if (rc == LBM_OK && cudaMemcpyAsync(&dv.us[1], &u1, sizeof(u1), cudaMemcpyHostToDevice, s->stream) != cudaSuccess)
        rc = LBM_E_CUDA;
    if (cudaMemcpyAsync(dv.jt_warm, keep, jbytes, cudaMemcpyDeviceToDevice, s->stream) != cudaSuccess) rc = LBM_E_CUDA;
    if (cudaFreeAsync(keep, s->stream) != cudaSuccess) rc = LBM_E_CUDA;
    if (rc == LBM_OK && cudaStreamSynchronize(s->stream) != cudaSuccess) rc = LBM_E_CUDA;
    return rc;
}

namespace {
struct CkptHeader {
    char magic[8];
    int32_t lattice, storage, usize, Q;
    int32_t warm_buffers, pad;
    int64_t dims[3];
    int64_t steps;
    double gamma, kappa, rho0;
};
}  // namespace

int lbm_save(lbm_sim* s, const char* path)
{
    if (!s || !path) return LBM_E_INVALID_ARG;
    LBM_CK(cudaSetDevice(s->device));
    LBM_CK(cudaStreamSynchronize(s->stream));
    const size_t N = size_t(s->dev.N);
    const size_t pbytes = size_t(s->Q) * N * s->kt.ssize;
    const size_t zbytes = N * s->kt.rsize;
    const size_t jbytes = size_t(warm_buffers(s->dev)) * 3 * N * s->kt.usize;
    const size_t wbytes = s->dev.wref[0] ? size_t(s->d == 3 ? 8 : 6) * N * sizeof(float) : 0;
    std::vector<char> buf(pbytes + zbytes + jbytes + wbytes);
    UsolveState us[2];
    LBM_CK(cudaMemcpy(us, s->dev.us, sizeof(us), cudaMemcpyDeviceToHost));
    LBM_CK(cudaMemcpy(buf.data(), s->dev.pop[s->cur], pbytes, cudaMemcpyDeviceToHost));
    if (zbytes) LBM_CK(cudaMemcpy(buf.data() + pbytes, s->dev.pop0[s->cur], zbytes, cudaMemcpyDeviceToHost));
    LBM_CK(cudaMemcpy(buf.data() + pbytes + zbytes, s->dev.jt_warm, jbytes, cudaMemcpyDeviceToHost));
    if (wbytes)  // the senders' references the stored populations are relative to
        LBM_CK(cudaMemcpy(buf.data() + pbytes + zbytes + jbytes, s->dev.wref[s->cur], wbytes, cudaMemcpyDeviceToHost));
    CkptHeader h{};
    std::memcpy(h.magic, "LBM2PH03", 8);
    h.lattice = s->lattice;
    h.storage = s->prm.storage;
    h.usize = int32_t(s->kt.usize);
    h.Q = s->Q;
    h.warm_buffers = warm_buffers(s->dev);
    for (int k = 0; k < 3; ++k) h.dims[k] = s->dims[k];
    h.steps = s->steps;
    h.gamma = s->prm.gamma;
    h.kappa = s->prm.kappa;
    h.rho0 = s->prm.rho0;
    FILE* fp = std::fopen(path, "wb");
    if (!fp) return LBM_E_IO;
    bool ok = std::fwrite(&h, sizeof(h), 1, fp) == 1 && std::fwrite(&us[0], sizeof(UsolveState), 1, fp) == 1 &&
              std::fwrite(buf.data(), 1, buf.size(), fp) == buf.size();
    ok = (std::fclose(fp) == 0) && ok;
    return ok ? LBM_OK : LBM_E_IO;
}

int lbm_load(lbm_sim* s, const char* path)
{
    if (!s || !path) return LBM_E_INVALID_ARG;
    LBM_CK(cudaSetDevice(s->device));
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return LBM_E_IO;
    CkptHeader h{};
    UsolveState u0{};
    bool ok = std::fread(&h, sizeof(h), 1, fp) == 1 && std::fread(&u0, sizeof(u0), 1, fp) == 1;
    ok = ok && std::memcmp(h.magic, "LBM2PH03", 8) == 0 && h.lattice == s->lattice && h.storage == s->prm.storage &&
         h.warm_buffers == warm_buffers(s->dev) &&
         h.usize == int32_t(s->kt.usize) && h.Q == s->Q && h.dims[0] == s->dims[0] && h.dims[1] == s->dims[1] &&
         h.dims[2] == s->dims[2];
    const size_t N = size_t(s->dev.N);
    const size_t pbytes = size_t(s->Q) * N * s->kt.ssize;
    const size_t zbytes = N * s->kt.rsize;
    const size_t jbytes = size_t(warm_buffers(s->dev)) * 3 * N * s->kt.usize;
    const size_t wbytes = s->dev.wref[0] ? size_t(s->d == 3 ? 8 : 6) * N * sizeof(float) : 0;
    std::vector<char> buf;
    if (ok) {
        buf.resize(pbytes + zbytes + jbytes + wbytes);
        ok = std::fread(buf.data(), 1, buf.size(), fp) == buf.size();
    }
    std::fclose(fp);
    if (!ok) return LBM_E_IO;
    LBM_CK(cudaStreamSynchronize(s->stream));
    int rc = reset_usolve(s);
    if (rc) return rc;
    s->cur = 0;
    u0.cur = 0;
    u0.resid_bits = 0;
    u0.jmax_bits = 0;
    LBM_CK(cudaMemcpy(s->dev.pop[0], buf.data(), pbytes, cudaMemcpyHostToDevice));
    if (zbytes) LBM_CK(cudaMemcpy(s->dev.pop0[0], buf.data() + pbytes, zbytes, cudaMemcpyHostToDevice));
    LBM_CK(cudaMemcpy(s->dev.jt_warm, buf.data() + pbytes + zbytes, jbytes, cudaMemcpyHostToDevice));
    if (wbytes) LBM_CK(cudaMemcpy(s->dev.wref[0], buf.data() + pbytes + zbytes + jbytes, wbytes, cudaMemcpyHostToDevice));
    LBM_CK(cudaMemcpy(&s->dev.us[0], &u0, sizeof(u0), cudaMemcpyHostToDevice));
    s->steps = h.steps;
    return LBM_OK;
}

int lbm_step_batch(lbm_sim* const* sims, int n, const int64_t* nsteps)
{
    if ((!sims || !nsteps) && n > 0) return LBM_E_INVALID_ARG;
    for (int k = 0; k < n; ++k)
        if (!sims[k] || nsteps[k] < 0) return LBM_E_INVALID_ARG;
    for (int k = 0; k < n; ++k) {
        int rc = lbm_step(sims[k], nsteps[k]);
        if (rc) return rc;
    }
    return LBM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched stepping (lbm_batch.h)
// ---------------------------------------------------------------------------
namespace lbm {

struct Batch {
    KernelTable kt{};
    int key = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    DevSim* d_sims = nullptr;    // [kBatchSlots] device table
    BatchWork* d_work = nullptr;
    DevSim* h_sims = nullptr;    // pinned mirrors of the table and the work list (copied from
    BatchWork* h_work = nullptr; // these asynchronously, so they change only between chunks)
    cudaEvent_t copied = nullptr; // the mirrors' last copy to the device has been done
    lbm_sim* slot[kBatchSlots] = {};
    cudaGraph_t g = nullptr;
    cudaGraphExec_t x = nullptr;
};

int batch_key(int lattice, const int64_t dims[3], const lbm_params& prm)
{
    const bool us64 = prm.storage == LBM_STORE_F64 || prm.usolve_precision == LBM_USOLVE_F64;
    const int combo = ((lattice * 16 + prm.storage) * 2 + (us64 ? 1 : 0)) * 2 + (prm.gamma != 0.0 ? 1 : 0);
    int64_t n = dims[0] * dims[1] * (lattice == LBM_D3Q59 ? dims[2] : 1);
    int size_class = 0;
    while (n >= 4) {
        n >>= 2;
        ++size_class;
    }
    return combo * 64 + size_class;
}

int batch_key_of(const lbm_sim* s) { return batch_key(s->lattice, s->dims, s->prm); }

namespace {

// persistent grid of a batched kernel: the blocks that fit on the device at once
int resident_grid(const void* fn, int threads, size_t smem)
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, smem) != cudaSuccess || per < 1) {
        (void)cudaGetLastError();
        per = 1;
    }
    return sms * per;
}

int build_batch_graph(Batch* b)
{
    LBM_CK(cudaGraphCreate(&b->g, 0));
    const KernelTable& kt = b->kt;
    DevSim* sims = b->d_sims;
    BatchWork* w = b->d_work;
    int pair = 0;
    const int TB = kt.tile_threads;
    const int MB = kt.local_ref ? kMomentsRowBlock : kt.block;
    cudaGraphNode_t n0, n1, n2, n3, nc, n5, n6, n7;
    {
        void* a[] = {&sims, &w};
        LBM_CK(add_kernel(b->g, &n0, kt.kb_step_begin, dim3(1), 32, a, nullptr, 0));
    }
    {
        void* a[] = {&sims, &w, &pair};
        LBM_CK(add_kernel(b->g, &n1, kt.kb_moments, dim3(resident_grid(kt.kb_moments, MB, 0)), MB, a, &n0, 1));
    }
    {
        void* a[] = {&sims, &w, &pair};
        LBM_CK(add_kernel(b->g, &n2, kt.kb_force, dim3(resident_grid(kt.kb_force, TB, kt.smem_force)), TB, a, &n1, 1,
                          kt.smem_force));
    }
    {
        void* a[] = {&sims, &w, &pair};
        LBM_CK(add_kernel(b->g, &n3, kt.kb_us_begin, dim3(1), 32 * kBatchSlots, a, &n2, 1));
    }
    cudaGraphConditionalHandle h;
    LBM_CK(cudaGraphConditionalHandleCreate(&h, b->g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    LBM_CK(cudaGraphAddNode(&nc, b->g, &n3, nullptr, 1, &cp));
    {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        cudaGraphNode_t b1, b2;
        void* a1[] = {&sims, &w, &pair};
        LBM_CK(add_kernel(body, &b1, kt.kb_sweep, dim3(resident_grid(kt.kb_sweep, TB, kt.smem_sweep)), TB, a1, nullptr, 0,
                          kt.smem_sweep));
        void* a2[] = {&sims, &w, &pair, &h};
        LBM_CK(add_kernel(body, &b2, kt.kb_us_ctl, dim3(1), 32, a2, &b1, 1));
    }
    {
        void* a[] = {&sims, &w};
        LBM_CK(add_kernel(b->g, &n5, kt.kb_derivs, dim3(resident_grid(kt.kb_derivs, TB, kt.smem_derivs)), TB, a, &nc, 1,
                          kt.smem_derivs));
    }
    {
        void* a[] = {&sims, &w};
        LBM_CK(add_kernel(b->g, &n6, kt.kb_collide, dim3(resident_grid(kt.kb_collide, TB, kt.smem_collide)), TB, a, &n5,
                          1, kt.smem_collide));
    }
    {
        void* a[] = {&sims, &w};
        LBM_CK(add_kernel(b->g, &n7, kt.kb_step_end, dim3(1), 32, a, &n6, 1));
    }
    LBM_CK(cudaGraphInstantiate(&b->x, b->g, 0));
    return LBM_OK;
}

}  // namespace

int batch_create(const lbm_sim* proto, cudaStream_t stream, Batch** out)
{
    if (!proto || !out) return LBM_E_INVALID_ARG;
    *out = nullptr;
    Batch* b = new (std::nothrow) Batch();
    if (!b) return LBM_E_OOM;
    b->kt = proto->kt;
    b->key = batch_key_of(proto);
    b->device = proto->device;
    b->stream = stream;
    int rc = LBM_OK;
    if (cudaSetDevice(b->device) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void**>(&b->d_sims), sizeof(DevSim) * kBatchSlots) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void**>(&b->d_work), sizeof(BatchWork)) != cudaSuccess ||
        cudaMallocHost(reinterpret_cast<void**>(&b->h_sims), sizeof(DevSim) * kBatchSlots) != cudaSuccess ||
        cudaMallocHost(reinterpret_cast<void**>(&b->h_work), sizeof(BatchWork)) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->copied, cudaEventDisableTiming) != cudaSuccess) {
        (void)cudaGetLastError();
        rc = LBM_E_OOM;
    }
    if (!rc) {
        std::memset(static_cast<void*>(b->h_sims), 0, sizeof(DevSim) * kBatchSlots);
        std::memset(static_cast<void*>(b->h_work), 0, sizeof(BatchWork));
        rc = build_batch_graph(b);
    }
    if (rc) {
        batch_destroy(b);
        return rc;
    }
    *out = b;
    return LBM_OK;
}

int batch_attach(Batch* b, int slot, lbm_sim* s)
{
    if (!b || !s || slot < 0 || slot >= kBatchSlots || b->slot[slot] || batch_key_of(s) != b->key) return LBM_E_INVALID_ARG;
    b->slot[slot] = s;
    return LBM_OK;
}

void batch_detach(Batch* b, int slot)
{
    if (b && slot >= 0 && slot < kBatchSlots) b->slot[slot] = nullptr;
}

int batch_launch(Batch* b, const int64_t* steps)
{
    if (!b || !steps) return LBM_E_INVALID_ARG;
    LBM_CK(cudaSetDevice(b->device));
    LBM_CK(cudaEventSynchronize(b->copied));  // the mirrors may be rewritten
    BatchWork& w = *b->h_work;
    int nslot = 0;
    int64_t most = 0;
    for (int k = 0; k < kBatchSlots; ++k)
        if (b->slot[k]) nslot = k + 1;
    w.nslot = nslot;
    w.tstart[0] = 0;
    w.mstart[0] = 0;
    for (int k = 0; k < kBatchSlots; ++k) {
        lbm_sim* s = b->slot[k];
        const int64_t n = s ? steps[k] : 0;
        if (n < 0) return LBM_E_INVALID_ARG;
        most = n > most ? n : most;
        w.live[k] = 0;
        w.todo[k] = int(n);
        w.src[k] = s ? s->cur : 0;
        int tiles = 0, mblocks = 0;
        w.tgx[k] = w.tgy[k] = w.mgx[k] = w.mgy[k] = 1;
        if (s) {
            b->h_sims[k] = s->dev;
            const dim3 tg = tile_grid(s), mg = moments_grid(s);
            w.tgx[k] = int(tg.x);
            w.tgy[k] = int(tg.y);
            w.mgx[k] = int(mg.x);
            w.mgy[k] = int(mg.y);
            tiles = int(tg.x * tg.y * tg.z);
            mblocks = int(mg.x * mg.y * mg.z);
        }
        w.tstart[k + 1] = w.tstart[k] + (k < nslot ? tiles : 0);
        w.mstart[k + 1] = w.mstart[k] + (k < nslot ? mblocks : 0);
    }
    if (most == 0) return LBM_OK;
    LBM_CK(cudaMemcpyAsync(b->d_sims, b->h_sims, sizeof(DevSim) * size_t(nslot), cudaMemcpyHostToDevice, b->stream));
    LBM_CK(cudaMemcpyAsync(b->d_work, b->h_work, sizeof(BatchWork), cudaMemcpyHostToDevice, b->stream));
    LBM_CK(cudaEventRecord(b->copied, b->stream));
    for (int64_t i = 0; i < most; ++i) LBM_CK(cudaGraphLaunch(b->x, b->stream));
    return LBM_OK;
}

void batch_account(Batch* b, const int64_t* steps)
{
    if (!b || !steps) return;
    for (int k = 0; k < kBatchSlots; ++k) {
        lbm_sim* s = b->slot[k];
        if (!s || steps[k] <= 0) continue;
        s->cur ^= int(steps[k] & 1);
        s->steps += steps[k];
    }
}

void batch_destroy(Batch* b)
{
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->x) cudaGraphExecDestroy(b->x);
    if (b->g) cudaGraphDestroy(b->g);
    if (b->d_sims) cudaFree(b->d_sims);
    if (b->d_work) cudaFree(b->d_work);
    if (b->h_sims) cudaFreeHost(b->h_sims);
    if (b->h_work) cudaFreeHost(b->h_work);
    if (b->copied) cudaEventDestroy(b->copied);
    (void)cudaGetLastError();
    delete b;
}

}  // namespace lbm
