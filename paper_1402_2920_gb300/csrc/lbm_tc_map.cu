// The collision's polynomial map on the tensor cores (tcgen05), measured against the scalar
// form that the collision kernel uses.
//
// With gamma = 0 every post-collision population of D3Q59 is
//   n*_i = W_k(i) P(c_i) + w_k(i)(rho0) H(c_i),                                 (S11)
//   P(c) = 1 + c.u/s + (c.u)^2/(2 s^2) - u.u/(2 s)                  (Sec. III, n^eq / (w rho))
//   H(c) = cf_int c.f + cf_jt c.j~ + cf_h2 (Sigma:cc - s0 tr Sigma)
//          + cf_h3 (Xi':ccc - 3 s0 (tr Xi').c)                                 (Secs. VI, VIII)
// with W_k = w_k(s) rho.  P and H are polynomials in c with 10 and 20 monomials, so for a tile
// of 128 sites the 2 x 59 values are one product [128 x 32] x [32 x 128] of per-site
// coefficients with the fixed table of monomials c_i^m (small integers, exact in TF32).  The
// tensor form issues that product as tcgen05.mma (kind::tf32, accumulator in tensor memory) on
// a two-term split of the coefficients (hi + lo, each TF32), which keeps the product to about
// 2^-21 of the coefficients; the scalar form evaluates it per pair of opposite velocities, as
// the collision kernel does.  Both read the same synthetic per-site inputs and reduce the 59
// populations of a site to one weighted sum, so the comparison times the map itself.
#include <cstdint>
#include <new>

#include "lbm.h"
#include "lbm_lattice.h"

namespace {

using L3 = lbm::Lat<1>;
constexpr int kQ = 59;
constexpr int kTile = 128;  // sites per tensor tile (MMA M)
constexpr int kK = 32;      // coefficient columns (10 + 20 used)
constexpr int kN = 128;     // output columns: P_i at i, H_i at 64 + i

struct MapConst {
    float s0, cf_int, cf_jt, cf_h2, cf_h3, rho0;
    float w0[8];   // w_k(s0)
    float wc[8][4];  // cubic coefficients of w_k(s)
    float r[kQ];     // weights of the per-site checksum
};

__device__ __forceinline__ unsigned hash32(unsigned x)
{
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}
// uniform in [-1, 1): one linear congruential step of the site's generator state per value
// (cheap, so that generating the inputs does not hide the cost of the map)
__device__ __forceinline__ float urand(unsigned& state)
{
    state = state * 1664525u + 1013904223u;
    return float(state) * (2.0f / 4294967296.0f) - 1.0f;
}

// Synthetic inputs of a site (magnitudes of a two-phase droplet: rho ~ 1 +- 0.1, u ~ 1e-2,
// Sigma and Xi' ~ 1e-4) and the monomial coefficients of P (a[0..9]) and H (a[10..29]).
// Monomial order: 1, x, y, z, xx, yy, zz, xy, xz, yz (P and H), then xxx, yyy, zzz, xxy, xxz,
// xyy, yyz, xzz, yzz, xyz (H).
__device__ __forceinline__ void site_coeffs(const MapConst& c, long long s, float (&a)[30], float& rho_out, float& sc)
{
    unsigned st = hash32(unsigned(s) ^ hash32(unsigned(s >> 32) + 0x632be5abu));
    const float rho = c.rho0 + 0.1f * urand(st);
    sc = c.s0 + 0.05f * urand(st);
    rho_out = rho;
    float u[3], f[3], jt[3], S[6], X[10];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        u[k] = 1e-2f * urand(st);
        f[k] = 1e-3f * urand(st);
        jt[k] = 1e-4f * urand(st);
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) S[k] = 1e-4f * urand(st);
#pragma unroll
    for (int k = 0; k < 10; ++k) X[k] = 1e-4f * urand(st);
    const float is = 1.0f / sc, uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    a[0] = 1.0f - 0.5f * uu * is;
    a[1] = u[0] * is;
    a[2] = u[1] * is;
    a[3] = u[2] * is;
    const float h = 0.5f * is * is;
    a[4] = h * u[0] * u[0];
    a[5] = h * u[1] * u[1];
    a[6] = h * u[2] * u[2];
    a[7] = 2.0f * h * u[0] * u[1];
    a[8] = 2.0f * h * u[0] * u[2];
    a[9] = 2.0f * h * u[1] * u[2];
    // Sigma: xx, yy, zz, xy, xz, yz; Xi': xxx, yyy, zzz, xxy, xxz, xyy, yyz, xzz, yzz, xyz
    const float trS = S[0] + S[1] + S[2];
    const float trX[3] = {X[0] + X[5] + X[7], X[3] + X[1] + X[8], X[4] + X[6] + X[2]};
    a[10] = -c.cf_h2 * c.s0 * trS;
#pragma unroll
    for (int k = 0; k < 3; ++k) a[11 + k] = c.cf_int * f[k] + c.cf_jt * jt[k] - 3.0f * c.cf_h3 * c.s0 * trX[k];
    a[14] = c.cf_h2 * S[0];
    a[15] = c.cf_h2 * S[1];
    a[16] = c.cf_h2 * S[2];
    a[17] = 2.0f * c.cf_h2 * S[3];
    a[18] = 2.0f * c.cf_h2 * S[4];
    a[19] = 2.0f * c.cf_h2 * S[5];
    a[20] = c.cf_h3 * X[0];
    a[21] = c.cf_h3 * X[1];
    a[22] = c.cf_h3 * X[2];
#pragma unroll
    for (int k = 3; k < 9; ++k) a[20 + k] = 3.0f * c.cf_h3 * X[k];
    a[29] = 6.0f * c.cf_h3 * X[9];
}

__device__ __forceinline__ float weight_of(const MapConst& c, int k, float s)
{
    return c.wc[k][0] + s * (c.wc[k][1] + s * (c.wc[k][2] + s * c.wc[k][3]));
}

// monomial m of velocity i (P part for m < 10, H part for 10 <= m < 30)
__host__ __device__ constexpr int monomial(int i, int m)
{
    const int x = L3::cx(i), y = L3::cy(i), z = L3::cz(i);
    const int mm = m < 10 ? m : m - 10;
    switch (mm) {
    case 0: return 1;
    case 1: return x;
    case 2: return y;
    case 3: return z;
    case 4: return x * x;
    case 5: return y * y;
    case 6: return z * z;
    case 7: return x * y;
    case 8: return x * z;
    case 9: return y * z;
    case 10: return x * x * x;
    case 11: return y * y * y;
    case 12: return z * z * z;
    case 13: return x * x * y;
    case 14: return x * x * z;
    case 15: return x * y * y;
    case 16: return y * y * z;
    case 17: return x * z * z;
    case 18: return y * z * z;
    default: return x * y * z;
    }
}

// ---------------------------------------------------------------------------------------------
// Scalar form: per pair of opposite velocities, the even and odd parts of P and H
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_map_scalar(MapConst c, long long n, float* out)
{
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        float a[30], rho, sc;
        site_coeffs(c, s, a, rho, sc);
        float Wk[8], w0[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            Wk[k] = weight_of(c, k, sc) * rho;
            w0[k] = c.w0[k];
        }
        float acc = c.r[0] * (Wk[0] * a[0] + w0[0] * a[10]);
#pragma unroll
        for (int i = 1; i < kQ; i += 2) {
            float Pe = 0.f, Po = 0.f, He = 0.f, Ho = 0.f;  // even and odd parts in c
#pragma unroll
            for (int m = 0; m < 10; ++m) {
                const int v = monomial(i, m);
                if (v == 0) continue;
                const bool odd = m >= 1 && m <= 3;
                if (odd) Po += float(v) * a[m];
                else Pe += float(v) * a[m];
            }
#pragma unroll
            for (int m = 0; m < 20; ++m) {
                const int v = monomial(i, m + 10);
                if (v == 0) continue;
                const bool odd = (m >= 1 && m <= 3) || m >= 10;
                if (odd) Ho += float(v) * a[10 + m];
                else He += float(v) * a[10 + m];
            }
            const int k = L3::shell(i);
            const float np = Wk[k] * (Pe + Po) + w0[k] * (He + Ho);
            const float nm = Wk[k] * (Pe - Po) + w0[k] * (He - Ho);
            acc += c.r[i] * np + c.r[i + 1] * nm;
        }
        out[s] = acc;
    }
}

// ---------------------------------------------------------------------------------------------
// Tensor form (tcgen05, one CTA of 128 threads per SM slot, persistent over tiles of 128 sites)
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned su32(const void* p) { return static_cast<unsigned>(__cvta_generic_to_shared(p)); }

// Byte offset of element (row r, column k) of a [rows][32] TF32 operand in the canonical K-major
// layout without swizzle: 8 x 16-byte core matrices, the 8 core matrices of a row group along K
// adjacent (128 bytes apart), row groups 1024 bytes apart.
__host__ __device__ constexpr unsigned op_offset(int r, int k) { return unsigned(((r >> 3) * 8 + (k >> 2)) * 128 + (r & 7) * 16 + (k & 3) * 4); }

// Shared-memory matrix descriptor (tcgen05): start address, leading-dimension byte offset (K
// direction, 128), stride byte offset (row groups, 1024), descriptor version 1, no swizzle.
__device__ __forceinline__ unsigned long long smem_desc(unsigned addr)
{
    return (unsigned long long)((addr & 0x3FFFFu) >> 4) | ((unsigned long long)(128u >> 4) << 16) |
           ((unsigned long long)(1024u >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both K-major, N = 128, M = 128.
constexpr unsigned kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned(kN) >> 3) << 17) | ((unsigned(kTile) >> 4) << 24);

__device__ __forceinline__ float tf32_round(float x)
{
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ bool mbar_wait_parity(unsigned bar, unsigned parity)
{
    const long long t0 = clock64();
    while (true) {
        unsigned ok;
        asm volatile("{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n selp.u32 %0, 1, 0, P;\n}\n"
                     : "=r"(ok)
                     : "r"(bar), "r"(parity)
                     : "memory");
        if (ok) return true;
        if (clock64() - t0 > (1ll << 31)) return false;
    }
}

#define TMEM_LD32(taddr, v)                                                                                            \
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "     \
                 "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "     \
                 "[%32];\n"                                                                                             \
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),    \
                   "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),           \
                   "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),         \
                   "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),         \
                   "=r"(v[29]), "=r"(v[30]), "=r"(v[31])                                                               \
                 : "r"(taddr))

constexpr int kOpBytes = kTile * kK * 4;  // one operand tile: 16 KB

// Four CTAs per SM (16 warps), each holding 128 tensor-memory columns: the SM's 512.
constexpr int kTcCtasPerSm = 4;

__global__ void __launch_bounds__(kTile, kTcCtasPerSm) k_map_tc(MapConst c, long long n, float* out, int* status)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char* Ahi = sm;                  // [128 sites][32] coefficients, high TF32 part
    unsigned char* Alo = sm + kOpBytes;       // low part
    unsigned char* Bm = sm + 2 * kOpBytes;    // [128 output columns][32] monomials
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ unsigned tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    // the monomial table, once per CTA
    for (int e = tid; e < kN * kK; e += kTile) {
        const int row = e / kK, k = e % kK;
        float v = 0.f;
        if (row < kQ && k < 10) v = float(monomial(row, k));
        else if (row >= 64 && row - 64 < kQ && k >= 10 && k < 30) v = float(monomial(row - 64, k));
        *reinterpret_cast<float*>(Bm + op_offset(row, k)) = v;
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(su32(&mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(&tmem_base)),
                     "r"(kN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const unsigned tmem = tmem_base;
    const unsigned lane_addr = tmem + ((unsigned(warp) * 32u) << 16);
    unsigned phase = 0;
    bool ok = true;
    const long long ntiles = n / kTile;
    for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const long long s = tile * kTile + tid;
        float a[30], rho, sc;
        site_coeffs(c, s, a, rho, sc);
#pragma unroll
        for (int k = 0; k < kK; ++k) {
            const float v = k < 30 ? a[k] : 0.f;
            const float hi = tf32_round(v);
            *reinterpret_cast<float*>(Ahi + op_offset(tid, k)) = hi;
            *reinterpret_cast<float*>(Alo + op_offset(tid, k)) = tf32_round(v - hi);
        }
        // the operands are visible to the tensor core; the previous tile's accumulator reads are done
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
            for (int part = 0; part < 2; ++part)
#pragma unroll
                for (int ks = 0; ks < kK / 8; ++ks) {
                    const unsigned long long ad = smem_desc(su32(part ? Alo : Ahi) + unsigned(ks) * 256u);
                    const unsigned long long bd = smem_desc(su32(Bm) + unsigned(ks) * 256u);
                    const unsigned acc = (part | ks) ? 1u : 0u;
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                        "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc)
                        : "memory");
                }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(su32(&mbar))
                         : "memory");
        }
        ok = mbar_wait_parity(su32(&mbar), phase);
        phase ^= 1u;
        ok = __syncthreads_and(ok);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        float Wk[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) Wk[k] = weight_of(c, k, sc) * rho;
        float acc = 0.f;
#pragma unroll
        for (int blk = 0; blk < 2; ++blk) {  // columns 0..63 hold P, 64..127 hold H
            unsigned P[32], H[32];
            TMEM_LD32(lane_addr + unsigned(blk * 32), P);
            TMEM_LD32(lane_addr + unsigned(64 + blk * 32), H);
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int i = blk * 32 + j;
                if (i < kQ) {
                    const int k = L3::shell(i);
                    acc += c.r[i] * (Wk[k] * __uint_as_float(P[j]) + c.w0[k] * __uint_as_float(H[j]));
                }
            }
        }
        out[s] = acc;
    }
    if (!ok && tid == 0) atomicOr(status, 1);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kN) : "memory");
}

}  // namespace

extern "C" int lbm_collision_map_bench(int64_t n_sites, int reps, double* ms_scalar, double* ms_tensor,
                                       double* max_abs_diff, double* max_abs_value)
{
    if (n_sites < kTile || n_sites % kTile != 0 || n_sites > (int64_t(1) << 31) || reps < 1 || !ms_scalar || !ms_tensor ||
        !max_abs_diff || !max_abs_value)
        return LBM_E_INVALID_ARG;
    MapConst c{};
    const double s0 = 0.5;
    c.s0 = float(s0);
    c.rho0 = 1.0f;
    c.cf_int = float(0.5 / s0);
    c.cf_jt = float(-1.0 / s0);
    c.cf_h2 = float(0.5 / (s0 * s0));
    c.cf_h3 = float(1.0 / (6.0 * s0 * s0 * s0));
    for (int k = 0; k < 8; ++k) {
        for (int q = 0; q < 4; ++q) c.wc[k][q] = float(L3::wc(k, q));
        c.w0[k] = float(L3::wc(k, 0) + s0 * (L3::wc(k, 1) + s0 * (L3::wc(k, 2) + s0 * L3::wc(k, 3))));
    }
    for (int i = 0; i < kQ; ++i) c.r[i] = float(1.0 + 0.01 * i);
    float *o1 = nullptr, *o2 = nullptr;
    int* st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = LBM_OK;
    const size_t bytes = size_t(n_sites) * sizeof(float);
    if (cudaMalloc(&o1, bytes) != cudaSuccess || cudaMalloc(&o2, bytes) != cudaSuccess ||
        cudaMalloc(&st, sizeof(int)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess)
        rc = LBM_E_OOM;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = 3 * size_t(kOpBytes);
    if (!rc && cudaFuncSetAttribute(k_map_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess)
        rc = LBM_E_CUDA;
    if (!rc && cudaMemset(st, 0, sizeof(int)) != cudaSuccess) rc = LBM_E_CUDA;
    float t1 = 0.f, t2 = 0.f;
    for (int pass = 0; pass < 2 && !rc; ++pass) {  // the first pass warms up
        if (cudaEventRecord(e0) != cudaSuccess) rc = LBM_E_CUDA;
        for (int r = 0; r < reps && !rc; ++r) k_map_scalar<<<sms * 8, 256>>>(c, n_sites, o1);
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = LBM_E_CUDA;
        cudaEventElapsedTime(&t1, e0, e1);
        cudaEventRecord(e0);
        for (int r = 0; r < reps && !rc; ++r) k_map_tc<<<sms * kTcCtasPerSm, kTile, smem>>>(c, n_sites, o2, st);
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = LBM_E_CUDA;
        cudaEventElapsedTime(&t2, e0, e1);
    }
    int flag = 0;
    if (!rc && cudaMemcpy(&flag, st, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) rc = LBM_E_CUDA;
    if (!rc && flag) rc = LBM_E_TIMEOUT;
    if (!rc) {
        // compare the two on the host (a sample of sites is enough; here every site)
        const size_t m = size_t(n_sites);
        float* h1 = new (std::nothrow) float[m];
        float* h2 = new (std::nothrow) float[m];
        if (!h1 || !h2 || cudaMemcpy(h1, o1, bytes, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(h2, o2, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) {
            rc = LBM_E_CUDA;
        } else {
            double dmax = 0.0, vmax = 0.0;
            for (size_t k = 0; k < m; ++k) {
                const double d = double(h1[k]) - double(h2[k]);
                dmax = d > dmax ? d : (-d > dmax ? -d : dmax);
                const double v = h1[k] < 0 ? -double(h1[k]) : double(h1[k]);
                vmax = v > vmax ? v : vmax;
            }
            *max_abs_diff = dmax;
            *max_abs_value = vmax;
        }
        delete[] h1;
        delete[] h2;
    }
    *ms_scalar = t1 / reps;
    *ms_tensor = t2 / reps;
    if (o1) cudaFree(o1);
    if (o2) cudaFree(o2);
    if (st) cudaFree(st);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    (void)cudaGetLastError();
    return rc;
}
