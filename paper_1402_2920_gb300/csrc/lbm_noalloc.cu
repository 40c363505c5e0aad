// Mass and momentum sums of a population array that allocate nothing.
//
// The same reduction as lbm_stats_get (rho = sum_i n_i, j = sum_i n_i c_i summed
// over the lattice, Sec. II), but the per-block partial sums live in one
// file-scope device array instead of a buffer the simulation allocates.  It serves
// callers that may not touch the device allocator while they run: a serving loop
// that has promised the whole device-memory budget to admitted simulations by their
// footprint (an allocation would break the accounting it enforces), and loops
// that watch running simulations, where cudaMalloc / cudaFree may synchronise the
// device and stall the other streams.
#include <mutex>

#include "lbm.h"
#include "lbm_lattice.h"

namespace {

constexpr int kNaBlock = 256;            // threads per block
constexpr int kNaSitesPerThread = 64;    // sites each thread sums
constexpr int kNaMaxBlocks = 4096;       // capacity of the scratch array
constexpr long long kNaMaxSites = (long long)kNaMaxBlocks * kNaBlock * kNaSitesPerThread;  // 67,108,864
constexpr int kNaMaxDevices = 64;

// Per-block partials (mass, momentum x, y, z) of the call in flight on this device:
// 4096 x 4 doubles = 128 KB.  Every block overwrites its own four entries before the
// final kernel reads them, so nothing here has to start at zero.
static __device__ __align__(256) double g_na_scratch[kNaMaxBlocks * 4];

double* g_na_addr[kNaMaxDevices] = {};
std::mutex g_na_mutex;

// Block b sums sites b*256*64 + t + 256*k (k < 64) of a [Q][n] population array in a
// fixed order and writes its four partials.
template <int LAT>
__global__ void __launch_bounds__(kNaBlock) k_na_partial(const double* __restrict__ pops, long long n, double* part)
{
    using L = lbm::Lat<LAT>;
    __shared__ double sm[4][kNaBlock];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    const long long base = (long long)blockIdx.x * kNaBlock * kNaSitesPerThread + threadIdx.x;
    for (int k = 0; k < kNaSitesPerThread; ++k) {
        const long long s = base + (long long)k * kNaBlock;
        if (s >= n) break;
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            const double v = pops[(long long)i * n + s];
            acc[0] += v;
            if (L::cx(i)) acc[1] += L::cx(i) * v;
            if (L::cy(i)) acc[2] += L::cy(i) * v;
            if (L::cz(i)) acc[3] += L::cz(i) * v;
        }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) sm[c][threadIdx.x] = acc[c];
    __syncthreads();
    for (int w = kNaBlock / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
#pragma unroll
            for (int c = 0; c < 4; ++c) sm[c][threadIdx.x] += sm[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 4) part[blockIdx.x * 4 + threadIdx.x] = sm[threadIdx.x][0];
}

__global__ void __launch_bounds__(kNaBlock) k_na_final(const double* part, int nparts, double* out)
{
    __shared__ double sm[4][kNaBlock];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int k = threadIdx.x; k < nparts; k += kNaBlock)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[c] += part[k * 4 + c];
#pragma unroll
    for (int c = 0; c < 4; ++c) sm[c][threadIdx.x] = acc[c];
    __syncthreads();
    for (int w = kNaBlock / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
#pragma unroll
            for (int c = 0; c < 4; ++c) sm[c][threadIdx.x] += sm[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 4) out[threadIdx.x] = sm[threadIdx.x][0];
}

// Device address of the scratch array on the current device, looked up once per device.
double* na_scratch(int dev)
{
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_addr[dev]) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_na_scratch) != cudaSuccess) return nullptr;
        g_na_addr[dev] = static_cast<double*>(ptr);
    }
    return g_na_addr[dev];
}

}  // namespace

extern "C" int lbm_moment_sums_noalloc(int lattice, const double* pops, int64_t n_sites, double* sums, void* cuda_stream)
{
    if (lattice != LBM_D2Q21 && lattice != LBM_D3Q59) return LBM_E_INVALID_ARG;
    if (!pops || !sums || n_sites < 1) return LBM_E_INVALID_ARG;
    if (n_sites > kNaMaxSites) return LBM_E_INVALID_ARG;  // beyond the scratch capacity
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) return LBM_E_CUDA;
    double* part = na_scratch(dev);
    if (!part) return LBM_E_CUDA;
    const long long per_block = (long long)kNaBlock * kNaSitesPerThread;
    const int nblocks = int((n_sites + per_block - 1) / per_block);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (lattice == LBM_D2Q21) k_na_partial<0><<<nblocks, kNaBlock, 0, st>>>(pops, n_sites, part);
    else k_na_partial<1><<<nblocks, kNaBlock, 0, st>>>(pops, n_sites, part);
    k_na_final<<<1, kNaBlock, 0, st>>>(part, nblocks, sums);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_E_CUDA;
}
