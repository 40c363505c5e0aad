// Device code of the two-phase lattice Boltzmann step (Zelko & Duenweg,
// arXiv:1402.2920): lattice traits, equation of state, storage codecs and the
// per-site kernels of the Supplemental Material's steps S1-S12.
//
// Kernel map (each is a full sweep, as the supplement requires between steps):
//   k_moments   S1      rho = sum n_i, j0 = sum n_i c_i, c_s^2 window check
//   k_force     S2      f = kappa rho d_a d_b d_b rho (Sec. IV.E), j0' = j0 + f/2
//   k_sweep     S3-S6   one Jacobi sweep of the u-solve, tiled: u = (j0' + j~)/rho,
//                       d_a u_b (Sec. IV.B), q_ab, j~new = -(1/12) d_b q_ab; the stop test
//                       takes max|j~new - j~| of the plain iteration (S6) and the size of the
//                       accelerated update
//   k_us_ctl    S6, S7  convergence test, buffer swap, graph loop condition
//   k_derivs    S8-S11  u, j; first derivatives (tiled); A, B, C; the site-local
//                       parts of Sigma and the whole Xi'
//   k_collide   S11,S12 nested derivatives (tiled), Sigma, per-velocity collision,
//                       push streaming n_i(r + c_i) = n_i + Delta_i
#pragma once

#include <climits>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>
#include <utility>

#include "lbm_common.h"
#include "lbm_lattice.h"

namespace lbm {

template <int LAT, typename T>
__device__ __forceinline__ T weight(int k, T s)
{
    using L = Lat<LAT>;
    return T(L::wc(k, 0)) + s * (T(L::wc(k, 1)) + s * (T(L::wc(k, 2)) + s * T(L::wc(k, 3))));
}

// ---------------------------------------------------------------------------
// Storage codecs.  raw() returns what is stored: n_i, or n_i - w_i(rho0) rho0
// for the deviation formats.  In the reduced storages (EXACT) the rest
// population (i = 0) lives in a plane of its own as an unevaluated float pair
// hi + lo, and the density sum is accumulated as a float pair with the
// error-free TwoSum: the collision gives the rest population the exact mass
// remainder, so the stored populations keep the pre-collision mass to about
// 2^-48 relative (in plain float the same rounding repeats at every
// stationary site and the mass drifts).
// ---------------------------------------------------------------------------

// s + e = a + b exactly (Knuth's TwoSum; the _rn intrinsics forbid contraction)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (hi, lo) += v with the rounding error of the leading sum kept in lo
__device__ __forceinline__ void acc2(float& hi, float& lo, float v)
{
    float e;
    two_sum(hi, v, hi, e);
    lo = __fadd_rn(lo, e);
}
template <int S>
struct Codec;
template <>
struct Codec<ST_F32> {
    using type = float;
    static constexpr bool DEV = false, SPLIT0 = true, EXACT = true, SCALED = false, LOC = false;
    template <typename T>
    __device__ static T raw(const type* p, long long k) { return T(p[k]); }
    // evict-first: the populations are read again only in the next step, long after L2 turned over
    template <typename T>
    __device__ static void put(type* p, long long k, T v) { __stcs(p + k, float(v)); }
    template <typename T>
    __device__ static T rounded(T v) { return T(float(v)); }
};
template <>
struct Codec<ST_F32_DEV> {
    using type = float;
    static constexpr bool DEV = true, SPLIT0 = true, EXACT = true, SCALED = false, LOC = false;
    template <typename T>
    __device__ static T raw(const type* p, long long k) { return T(p[k]); }
    template <typename T>
    __device__ static void put(type* p, long long k, T v) { __stcs(p + k, float(v)); }
    template <typename T>
    __device__ static T rounded(T v) { return T(float(v)); }
};
template <>
struct Codec<ST_F16_DEV> {
    using type = __half;
    // SCALED: the half holds (n_i - w_i rho0) / w_i(rho0), which keeps the small deviations of
    // the outer shells (weights down to ~1e-5) out of the subnormal range of half
    static constexpr bool DEV = true, SPLIT0 = true, EXACT = true, SCALED = true, LOC = false;
    template <typename T>
    __device__ static T raw(const type* p, long long k) { return T(__half2float(p[k])); }
    template <typename T>
    __device__ static void put(type* p, long long k, T v) { p[k] = __float2half_rn(float(v)); }
    template <typename T>
    __device__ static T rounded(T v) { return T(__half2float(__float2half_rn(float(v)))); }
};
template <>
struct Codec<ST_BF16_DEV> {
    using type = __nv_bfloat16;
    static constexpr bool DEV = true, SPLIT0 = true, EXACT = true, SCALED = false, LOC = false;
    template <typename T>
    __device__ static T raw(const type* p, long long k) { return T(__bfloat162float(p[k])); }
    template <typename T>
    __device__ static void put(type* p, long long k, T v) { p[k] = __float2bfloat16_rn(float(v)); }
    template <typename T>
    __device__ static T rounded(T v) { return T(__bfloat162float(__float2bfloat16_rn(float(v)))); }
};
template <>
struct Codec<ST_F64> {
    using type = double;
    static constexpr bool DEV = false, SPLIT0 = false, EXACT = false, SCALED = false, LOC = false;
    template <typename T>
    __device__ static T raw(const type* p, long long k) { return T(p[k]); }
    template <typename T>
    __device__ static void put(type* p, long long k, T v) { p[k] = double(v); }
    template <typename T>
    __device__ static T rounded(T v) { return T(double(v)); }
};

// Local-reference storages: the stored value is n_i - w_i(c_s^2(rho_r)) rho_r with r the site that
// sent the population (its last collision), so only the part of n_i that the local equilibrium
// weight does not carry is rounded: the velocity and non-equilibrium parts, ~1e-3 of n_i,
// instead of the 10-20 % of n_i by which a two-phase density field departs from w_i(rho0) rho0.
// The sender's references w_k rho_r per shell live in DevSim::wref.
template <>
struct Codec<ST_F32_LOC> : Codec<ST_F32_DEV> {
    static constexpr bool LOC = true;
};
template <>
struct Codec<ST_F16_LOC> : Codec<ST_F16_DEV> {
    static constexpr bool LOC = true;  // scaled by 1/w_i(rho0) as well: the values are small
};
template <>
struct Codec<ST_BF16_LOC> : Codec<ST_BF16_DEV> {
    static constexpr bool LOC = true;
};

template <typename T>
__device__ __forceinline__ const Phys<T>& phys(const DevSim& p);
template <>
__device__ __forceinline__ const Phys<float>& phys<float>(const DevSim& p) { return p.pf; }
template <>
__device__ __forceinline__ const Phys<double>& phys<double>(const DevSim& p) { return p.pd; }

// ---------------------------------------------------------------------------
// Equation of state (App. B; S1).  P = p, DP = dp/drho, PM = p - rho dp/drho,
// RPP = rho d2p/drho2.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void eos_full(const DevSim& p, T rho, T& P, T& DP, T& PM, T& RPP)
{
    const Phys<T>& q = phys<T>(p);
    if (p.eos_kind == 0) {
        const T ig = T(1) / (T(1) - q.b * rho);
        P = rho * q.Teos * ig - q.a * rho * rho;
        DP = q.Teos * ig * ig - T(2) * q.a * rho;
        RPP = rho * (T(2) * q.bT * ig * ig * ig - T(2) * q.a);
    } else {
        T psi = T(0), dpsi = T(0), integ = T(0);
        if (rho > q.rho1 && rho < q.rho3) {
            const T ph = q.pi_D * (rho - q.rho1);
            const T sn = sin(ph), cn = cos(ph);
            psi = q.A * sn;
            dpsi = q.A_pi_D * cn;
            integ = q.AD_pi * (T(1) - cn);
        }
        const T cs2 = q.cs2_1 * exp(integ);
        P = rho * cs2;
        DP = cs2 * (T(1) + rho * psi);
        RPP = rho * (cs2 * psi * (T(1) + rho * psi) + cs2 * (psi + rho * dpsi));
    }
    PM = P - rho * DP;
}

template <typename T>
__device__ __forceinline__ T eos_p(const DevSim& p, T rho)
{
    const Phys<T>& q = phys<T>(p);
    if (p.eos_kind == 0) return rho * q.Teos / (T(1) - q.b * rho) - q.a * rho * rho;
    T P, DP, PM, RPP;
    eos_full(p, rho, P, DP, PM, RPP);
    return P;
}

// c_s^2 = p/rho at rho = rho0 + drho, and its difference ds from c_s^2(rho0) = cs0,
// evaluated from drho directly so that ds keeps its relative precision when small.
template <typename T>
__device__ __forceinline__ void cs2_delta(const DevSim& p, T drho, T& s, T& ds)
{
    const Phys<T>& q = phys<T>(p);
    const T rho = q.rho0 + drho;
    if (p.eos_kind == 0) {
        // s = T/(1 - b rho) - a rho  =>  s - s0 = drho F(rho), F(rho) = b T / ((1 - b rho)(1 - b rho0)) - a
        // = F(rho0) + b^2 T drho / ((1 - b rho) (1 - b rho0)^2).  F(rho0) is a difference of O(1)
        // terms; it comes precomputed as an unevaluated pair F0 + F0lo, so that ds carries one
        // rounding of its own size instead of the cancellation of the O(1) terms (in FP32 that
        // cancellation biased the lattice pressure of the bulk phases at ~1e-7).
        const T g = q.g0 - q.b * drho;
        const T corr = q.b2T_g02 * drho / g;
        ds = fma(drho, q.F0, fma(drho, q.F0lo, drho * corr));
        s = q.cs0 + ds;
    } else {
        // s = cs2(rho1) exp(I), I = (A D / pi)(1 - cos phi), phi = pi (rho - rho1)/D clamped to [0, 2 pi]
        const T PI = T(3.14159265358979323846);
        const T ph_raw = q.pi_D * (rho - q.rho1);
        const T ph = fmin(fmax(ph_raw, T(0)), T(2) * PI), ph0 = fmin(fmax(q.ph0, T(0)), T(2) * PI);
        const bool inside = ph == ph_raw && ph0 == q.ph0;
        const T dph = inside ? q.pi_D * drho : ph - ph0;
        const T dI = q.AD_pi * T(2) * sin(T(0.5) * (ph + ph0)) * sin(T(0.5) * dph);
        ds = q.cs0 * expm1(dI);
        s = q.cs0 + ds;
    }
}

// ---------------------------------------------------------------------------
// Periodic neighbourhoods.  Every extent is >= 4, so one correction wraps any
// shift of at most 4.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int wrapc(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }
// v mod n in [0, n) for any v (tile halos of small lattices wrap more than once)
__device__ __forceinline__ int wrapm(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

struct Site {
    int x, y, z;
    long long s;
};

__device__ __forceinline__ Site site_of(const DevSim& p, long long s)
{
    Site r;
    r.s = s;
    r.x = int(s % p.nx);
    long long t = s / p.nx;
    r.y = int(t % p.ny);
    r.z = int(t / p.ny);
    return r;
}

__device__ __forceinline__ long long at(const DevSim& p, int x, int y, int z)
{
    return (long long)x + (long long)p.nx * ((long long)y + (long long)p.ny * z);
}

__device__ __forceinline__ long long shifted(const DevSim& p, const Site& r, int dx, int dy, int dz)
{
    return at(p, wrapc(r.x + dx, p.nx), wrapc(r.y + dy, p.ny), wrapc(r.z + dz, p.nz));
}

// Site that sent population i to site (x, y, z): (x, y, z) - c_i, periodic (|c| <= 4 <= n).
template <int LAT>
__device__ __forceinline__ long long sender(const DevSim& p, int x, int y, int z, int i)
{
    using L = Lat<LAT>;
    return at(p, wrapc(x - L::cx(i), p.nx), wrapc(y - L::cy(i), p.ny), L::D == 3 ? wrapc(z - L::cz(i), p.nz) : 0);
}

// Site indices of r - 2e_a, r - e_a, r + e_a, r + 2e_a for every axis a.
struct Axes {
    long long n[3][4];
};

template <int D>
__device__ __forceinline__ void make_axes(const DevSim& p, const Site& r, Axes& A)
{
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const int sh[4] = {-2, -1, 1, 2};
#pragma unroll
        for (int k = 0; k < 4; ++k)
            A.n[a][k] = shifted(p, r, a == 0 ? sh[k] : 0, a == 1 ? sh[k] : 0, a == 2 ? sh[k] : 0);
    }
}

// First derivative of Sec. IV.B along axis a: shells (1 0) with 2/3 and (2 0)
// with -1/24, i.e. (2/3)(g(+1) - g(-1)) - (1/12)(g(+2) - g(-2)).
template <typename T, class G>
__device__ __forceinline__ T d1(const Axes& A, int a, G g)
{
    return T(2.0 / 3.0) * (g(A.n[a][2]) - g(A.n[a][1])) - T(1.0 / 12.0) * (g(A.n[a][3]) - g(A.n[a][0]));
}

// symmetric-pair index in 2D (xx, yy, xy) and 3D (xx, yy, zz, xy, xz, yz)
template <int D>
__host__ __device__ __forceinline__ constexpr int sym2(int a, int b)
{
    if (a == b) return a;
    if (D == 2) return 2;
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    return lo == 0 ? (hi == 1 ? 3 : 4) : 5;
}
// fully symmetric 3-index: 2D (xxx, yyy, xxy, xyy); 3D (xxx, yyy, zzz, xxy, xxz, xyy, yyz, xzz, yzz, xyz)
template <int D>
__host__ __device__ __forceinline__ constexpr int sym3(int a, int b, int c)
{
    const int nx = (a == 0) + (b == 0) + (c == 0);
    const int ny = (a == 1) + (b == 1) + (c == 1);
    const int nz = (a == 2) + (b == 2) + (c == 2);
    if (D == 2) return nx == 3 ? 0 : ny == 3 ? 1 : nx == 2 ? 2 : 3;
    if (nx == 3) return 0;
    if (ny == 3) return 1;
    if (nz == 3) return 2;
    if (nx == 2) return ny == 1 ? 3 : 4;
    if (ny == 2) return nx == 1 ? 5 : 6;
    if (nz == 2) return nx == 1 ? 7 : 8;
    return 9;
}

// aux layout offsets
template <int D>
struct AuxLayout {
    static constexpr int NB = D == 2 ? 3 : 6;
    static constexpr int NX = D == 2 ? 4 : 10;
    static constexpr int A = 0, B = 1, C = 1 + NB, SIGL = 1 + NB + D, XI = 1 + NB + D + NB;
    static constexpr int N = XI + NX;
};

__device__ __forceinline__ long long gtid() { return blockIdx.x * (long long)blockDim.x + threadIdx.x; }

// Block coordinates of a kernel body: blockIdx for a launch over one simulation, or the block
// a batched launch assigned to this pass over its work list.
struct Blk {
    int x, y, z;
};
__device__ __forceinline__ Blk launch_blk() { return Blk{int(blockIdx.x), int(blockIdx.y), int(blockIdx.z)}; }

template <typename T>
__device__ __forceinline__ const T* cp(const void* v) { return static_cast<const T*>(v); }
template <typename T>
__device__ __forceinline__ T* mp(void* v) { return static_cast<T*>(v); }
// Plane c of the aux field and plane a of a 3-vector field, through the parameter block's tables
// (one parameter load per access instead of 64-bit index arithmetic)
template <typename T>
__device__ __forceinline__ T* auxp(const DevSim& p, int c) { return static_cast<T*>(p.auxp[c]); }
template <typename T>
__device__ __forceinline__ T* plane(void* const (&tab)[3], int a) { return static_cast<T*>(tab[a]); }

// Stored value of population i at site s of buffer b: n_i, or n_i - w_i(rho0) rho0.
// The 16-bit storages keep the rest population (i = 0) in FP32 so that the mass
// remainder below survives storage.
template <int LAT, int S, typename T>
__device__ __forceinline__ T pop_raw(const DevSim& p, int b, int i, long long s)
{
    using C = Codec<S>;
    if (C::SPLIT0 && i == 0) {
        const float2 r = cp<float2>(p.pop0[b])[s];
        return T(r.x) + T(r.y);
    }
    const auto* base = cp<typename C::type>(p.pop[b]);
    // scaled storage: the value is half * w_i(rho0), one float product (the same everywhere)
    if (C::SCALED) return T(__fmul_rn(C::template raw<float>(base, (long long)i * p.N + s), p.pf.w0[Lat<LAT>::shell(i)]));
    return C::template raw<T>(base, (long long)i * p.N + s);
}

// Store v (in the storage's convention) and return the value actually stored.
template <int LAT, int S, typename T>
__device__ __forceinline__ T pop_put(const DevSim& p, int b, int i, long long s, T v)
{
    using C = Codec<S>;
    if (C::SPLIT0 && i == 0) {
        const float hi = float(v);
        const float lo = float(v - T(hi));
        mp<float2>(p.pop0[b])[s] = make_float2(hi, lo);
        return T(hi) + T(lo);
    }
    auto* base = mp<typename C::type>(p.popp[b][i]);  // plane i of buffer b
    if (C::SCALED) {
        const int k = Lat<LAT>::shell(i);
        const float x = __fmul_rn(float(v), p.pf.isc[k]);
        C::template put<float>(base, s, x);
        return T(__fmul_rn(C::template rounded<float>(x), p.pf.w0[k]));
    }
    C::template put<T>(base, s, v);
    return C::template rounded<T>(v);
}

// block-wide maximum of two non-negative doubles, then atomicMax on their bit patterns
__device__ __forceinline__ void block_max2(double a, double b, unsigned long long* da, unsigned long long* db)
{
    __shared__ double sa[32], sb[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
        b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
    }
    // NaN must win: fmax drops it, so fold a NaN flag separately
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { sa[warp] = a; sb[warp] = b; }
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        a = lane < nw ? sa[lane] : 0.0;
        b = lane < nw ? sb[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
            b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
        }
        if (lane == 0) {
            atomicMax(da, (unsigned long long)__double_as_longlong(a));
            atomicMax(db, (unsigned long long)__double_as_longlong(b));
        }
    }
}

// ---------------------------------------------------------------------------
// S1: moments and the c_s^2 window check
// ---------------------------------------------------------------------------
template <int LAT, typename T, int S, typename U>
__device__ __forceinline__ void b_moments(const DevSim& p, int src, int pair, const Blk bid)
{
    using L = Lat<LAT>;
    using C = Codec<S>;
    // local-reference storages run on the row grid (x-blocks, y, z), which hands each thread its
    // coordinates; the others on a flat grid
    int x = 0, y = 0, z = 0;
    long long s0;
    if (C::LOC) {
        x = int(bid.x * blockDim.x + threadIdx.x);
        y = bid.y;
        z = bid.z;
        s0 = x < p.nx ? at(p, x, y, z) : p.N;
        x = min(x, p.nx - 1);
    } else {
        s0 = bid.x * (long long)blockDim.x + threadIdx.x;
    }
    const long long s = s0 < p.N ? s0 : (C::LOC ? at(p, x, y, z) : p.N - 1);  // tails recompute a site
    const bool own = s0 < p.N;
    T sum = T(0), j[3] = {T(0), T(0), T(0)};
    float hi = 0.f, lo = 0.f;
    if (C::EXACT) {
        const float2 r0 = cp<float2>(p.pop0[src])[s];
        hi = r0.x;
        lo = r0.y;
    }
    if (C::LOC) {
        // n_i = stored_i + the sender's reference w_k rho.  The mass sums the decoded floats
        // fl(stored + reference), the values the sending collision accounted for; j0 goes over
        // opposite pairs, where the references enter as differences of neighbouring values.
        int ox[7], oy[7], oz[7];  // wrapped site offsets for the shifts -4, -2, -1, 0, 1, 2, 4
#pragma unroll
        for (int k = 0; k < 7; ++k) {
            const int sh = k == 0 ? -4 : k == 6 ? 4 : k - 3;
            ox[k] = wrapc(x + sh, p.nx);
            oy[k] = wrapc(y + sh, p.ny) * p.nx;
            oz[k] = L::D == 3 ? wrapc(z + sh, p.nz) * p.nx * p.ny : 0;
        }
        auto sidx = [](int c) { return c == -4 ? 0 : c == 4 ? 6 : c + 3; };
        const float* wr = p.wref[src];
        acc2(hi, lo, wr[s]);  // the rest population's reference: its own site
#pragma unroll
        for (int i = 1; i < L::Q; i += 2) {
            const int k = L::shell(i);
            const int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
            const float va = float(pop_raw<LAT, S, T>(p, src, i, s)), vb = float(pop_raw<LAT, S, T>(p, src, i + 1, s));
            // population i came from the site at -c_i, its opposite from +c_i
            const float ra = wr[k * p.N + ox[sidx(-cx)] + oy[sidx(-cy)] + oz[sidx(-cz)]];
            const float rb = wr[k * p.N + ox[sidx(cx)] + oy[sidx(cy)] + oz[sidx(cz)]];
            acc2(hi, lo, __fadd_rn(va, ra));
            acc2(hi, lo, __fadd_rn(vb, rb));
            const T d = T(va - vb) + T(ra - rb);
            if (cx) j[0] += T(cx) * d;
            if (cy) j[1] += T(cy) * d;
            if (cz) j[2] += T(cz) * d;
        }
    } else {
        // all loads first, so that a warp keeps the whole column of Q planes in flight
        T v[L::Q];
#pragma unroll
        for (int i = C::EXACT ? 1 : 0; i < L::Q; ++i) v[i] = pop_raw<LAT, S, T>(p, src, i, s);
#pragma unroll
        for (int i = C::EXACT ? 1 : 0; i < L::Q; ++i) {
            if (C::EXACT) acc2(hi, lo, float(v[i]));
            else sum += v[i];
        }
        // j0 over opposite pairs: c_i (n_i - n_-i), whose difference is exact for nearly equal
        // populations and whose products with c in {1, 2, 4} are exact, so the partial sums stay
        // at the size of j0 instead of the size of the populations
#pragma unroll
        for (int i = 1; i < L::Q; i += 2) {
            const T d = v[i] - v[i + 1];
            if (L::cx(i)) j[0] += T(L::cx(i)) * d;
            if (L::cy(i)) j[1] += T(L::cy(i)) * d;
            if (L::cz(i)) j[2] += T(L::cz(i)) * d;
        }
    }
    // rho - rho0: the deviation sum itself (sum_i w_i(rho0) rho0 = rho0 and the
    // odd offsets cancel in j0), or sum - rho0
    T drho;
    if (C::EXACT) {
        if (!C::DEV || C::LOC) {  // the sum is rho itself
            float e;
            two_sum(hi, -p.pf.rho0, hi, e);
            lo = __fadd_rn(lo, e);
        }
        float e;
        two_sum(hi, lo, hi, e);  // renormalise: hi = the float nearest to the pair
        drho = T(hi);
        if (own) mp<float>(p.rho_lo)[s] = e;  // the part float drops
    } else {
        drho = C::DEV ? sum : sum - phys<T>(p).rho0;
    }
    const T r = phys<T>(p).rho0 + drho;
    if (own) mp<T>(p.rho)[s] = drho;
    if (own)
#pragma unroll
        for (int a = 0; a < L::D; ++a) mp<T>(p.j0p)[a * p.N + s] = j[a];
    {  // density range of the state (bounds the spectrum of the u-solve iteration): one atomic per block
        __shared__ float slo[32], shi[32];
        float lo = float(r), hi = float(r);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        if (lane == 0) { slo[warp] = lo; shi[warp] = hi; }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < int(blockDim.x >> 5); ++w) { lo = fminf(lo, slo[w]); hi = fmaxf(hi, shi[w]); }
            if (lo > 0.f) {
                unsigned* rg = p.range + pair * 2 * kRangeSlots;
                const int slot = (bid.x + bid.y + bid.z) % kRangeSlots;
                atomicMin(rg + slot, __float_as_uint(lo));
                atomicMax(rg + kRangeSlots + slot, __float_as_uint(hi));
            }
        }
    }
    const T cs2 = eos_p(p, r) / r;
    if (!isfinite(r)) atomicOr(p.status, STB_NONFINITE_RHO);
    else if (!(cs2 > phys<T>(p).cs2_lo && cs2 < phys<T>(p).cs2_hi)) atomicOr(p.status, STB_WEIGHTS);
}
template <int LAT, typename T, int S, typename U>
__global__ void __launch_bounds__(256, 3) k_moments(DevSim p, int src, int pair)
{
    b_moments<LAT, T, S, U>(p, src, pair, launch_blk());
}

// ---------------------------------------------------------------------------
// S3-S7: the implicit u-solve (Sec. IX)
// ---------------------------------------------------------------------------
// Frozen-coefficient largest eigenvalue of the iteration at density rho:
// (d s2max / 12) max(3 c_s^2 - p', c_s^2), s2max = max_k |s(k)|^2 of the Sec. IV.B symbol.
static __device__ double frozen_gain(const DevSim& p, double rho)
{
    double P, DP, PM, RPP;
    eos_full<double>(p, rho, P, DP, PM, RPP);
    const double cs2 = P / rho;
    return p.d * p.s2max / 12.0 * fmax(3.0 * cs2 - DP, cs2);
}

// One warp (lane 0..31) per solve: the reductions are spread over the lanes (one thread took
// 22 us per step, most of it in the 17 FP64 gain evaluations one after the other).
static __device__ void b_us_begin(const DevSim& p, int pair, int lane)
{
    UsolveState& u = p.us[pair];
    // spectrum bound g of this solve from the density range of the state, with 2 % margin (the
    // frozen-coefficient value is the largest eigenvalue of a uniform state; a bound the solve
    // outgrows shows as a growing residual, and the control kernel then falls back to plain sweeps)
    unsigned* rg = p.range + pair * 2 * kRangeSlots;
    float flo = 3.0e38f, fhi = 0.f;
    for (int k = lane; k < kRangeSlots; k += 32) {
        flo = fminf(flo, __uint_as_float(rg[k]));
        fhi = fmaxf(fhi, __uint_as_float(rg[kRangeSlots + k]));
        rg[k] = 0x7f7fffffu;  // reset for the next state
        rg[kRangeSlots + k] = 0u;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        flo = fminf(flo, __shfl_xor_sync(0xffffffffu, flo, o));
        fhi = fmaxf(fhi, __shfl_xor_sync(0xffffffffu, fhi, o));
    }
    double lo = flo, hi = fhi;
    if (!(lo > 0.0 && hi >= lo && hi < 1e30)) lo = hi = p.rho0;
    double g = lane <= 16 ? frozen_gain(p, lo + (hi - lo) * lane / 16.0) : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) g = fmax(g, __shfl_xor_sync(0xffffffffu, g, o));
    if (lane != 0) return;
    g = fmin(0.95, 1.02 * g);
    u.gain = g;
    if (pair == 0) u.wsel ^= 1;  // the run's collision writes this step's j~ over the older one
    u.cheb_delta = 0.5 * g;
    u.cheb_sigma = (1.0 - 0.5 * g) / (0.5 * g);
    u.iter = 0;
    u.resid_bits = 0ull;
    u.jmax_bits = 0ull;
    u.converged = 0;
    u.running = 1;
    u.tma = 0;
    u.resid_min = 1e300;
    if (p.cheb) {  // first Chebyshev step: x += r / theta
        u.mode = 1;
        u.cheb_rho = 1.0 / u.cheb_sigma;
        u.c1 = 0.0;
        u.c2 = 1.0 / (1.0 - 0.5 * g);
    } else {       // plain relaxation x += omega r (omega = 0: 2/(2 - g))
        u.mode = 0;
        u.c1 = 0.0;
        u.c2 = p.omega > 0.0 ? p.omega : 2.0 / (2.0 - g);
    }
}
static __global__ void k_us_begin(DevSim p, int pair) { b_us_begin(p, pair, threadIdx.x & 31); }  // one warp

// One thread: the S6 test, the S7 swap, and the loop condition of the graph.
// Returns whether the solve stopped.
static __device__ bool b_us_ctl(const DevSim& p, int pair)
{
    UsolveState& u = p.us[pair];
    const double r = __longlong_as_double((long long)u.resid_bits);
    const double jm = __longlong_as_double((long long)u.jmax_bits);
    u.iter += 1;
    u.sweeps_total += 1;
    u.cur ^= 1;
    const bool bad = !isfinite(r);
    const bool conv = !bad && r <= p.tol + p.rtol * jm;
    const bool stop = conv || bad || u.iter >= p.maxit;
    if (bad) atomicOr(p.status, STB_USOLVE_NAN);
    else if (stop && !conv) atomicOr(p.status, STB_USOLVE_CAP);
    u.resid_bits = 0ull;
    u.jmax_bits = 0ull;
    // coefficients of the next sweep (Chebyshev semi-iteration for the real spectrum
    // [1 - g, 1] of I - A); a residual four times above the best one so far means the
    // spectral bound was too small: continue with plain relaxation
    if (u.mode == 1 && !bad && r > 4.0 * u.resid_min) u.mode = 0;
    if (u.mode == 1) {
        const double rn = 1.0 / (2.0 * u.cheb_sigma - u.cheb_rho);
        u.c1 = rn * u.cheb_rho;
        u.c2 = 2.0 * rn / u.cheb_delta;
        u.cheb_rho = rn;
    } else if (p.cheb) {  // fell back from Chebyshev: plain sweeps
        u.c1 = 0.0;
        u.c2 = 1.0;
    }
    u.resid_min = r < u.resid_min ? r : u.resid_min;
    if (stop) {
        u.iters_last = u.iter;
        u.iters_max = u.iter > u.iters_max ? u.iter : u.iters_max;
        u.resid_last = r;
        u.converged = conv ? 1 : 0;
        u.running = 0;
    }
    return stop;
}
static __global__ void k_us_ctl(DevSim p, int pair, cudaGraphConditionalHandle h, int use_cond)
{
    const bool stop = b_us_ctl(p, pair);
    if (use_cond) cudaGraphSetConditional(h, stop ? 0u : 1u);
}

// ---------------------------------------------------------------------------
// Per-site tails shared by the tiled kernels below
// ---------------------------------------------------------------------------
template <int LAT, typename T>
__device__ __forceinline__ void collision_consts(const DevSim& p, T& k1, T& k2, T& k3)
{
    const Phys<T>& q = phys<T>(p);
    k1 = q.k1;  // -(h^2/4)(g+1)^2/(g-1)
    k2 = q.k2;  // (h^2/6)(g^2+4g+1)/(g-1)
    k3 = q.k3;  // (h/3)(g^2+4g+1)/(g+1)
}

// S10 results at one site -> A = (p - rho p') div u, B_ab = p(d_a u_b + d_b u_a),
// C_b = rho^-1 d_b p + u_g d_g u_b (the three bracketed S11 arguments), the
// site-local part of Sigma and the whole Xi' (S11), written to aux.
template <int LAT, typename T>
__device__ __forceinline__ void derivs_tail(const DevSim& p, long long s, const T (&du)[3][3], T divj,
                                            const T (&dp)[3], const T (&dpr)[3], const T (&dpuu)[3][3][3], T rs,
                                            const T (&u)[3], const T (&jtl)[3])
{
    constexpr int D = Lat<LAT>::D;
    using AL = AuxLayout<D>;
    T P, DP, PM, RPP;
    eos_full<T>(p, rs, P, DP, PM, RPP);
    T divu = T(0);
#pragma unroll
    for (int a = 0; a < D; ++a) divu += du[a][a];
    T k1, k2, k3;
    collision_consts<LAT, T>(p, k1, k2, k3);
    auxp<T>(p, AL::A)[s] = PM * divu;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = a; b < D; ++b) {
            const T sd = du[a][b] + du[b][a];
            auxp<T>(p, AL::B + sym2<D>(a, b))[s] = P * sd;
            auxp<T>(p, AL::SIGL + sym2<D>(a, b))[s] = k2 * (-DP * divj * sd + (a == b ? RPP * divu * divj : T(0)));
        }
#pragma unroll
    for (int b = 0; b < D; ++b) {
        T c = dp[b] / rs;
#pragma unroll
        for (int g = 0; g < D; ++g) c += u[g] * du[g][b];
        auxp<T>(p, AL::C + b)[s] = c;
    }
    // Xi'_abc = k3 [X(a,b;c) + X(a,c;b) + X(b,c;a)] + (1-gamma) cs0 (delta j~ sym),
    // X(a,b;c) = d_c(p u_a u_b) + delta_ab [p d_c(p/rho) + (p - rho p') u_c div u]
    auto PUU = [&](int c, int a, int b) { return a <= b ? dpuu[c][a][b] : dpuu[c][b][a]; };
    auto X = [&](int a, int b, int c) { return PUU(c, a, b) + (a == b ? P * dpr[c] + PM * u[c] * divu : T(0)); };
    const T cj = phys<T>(p).cj;  // (1 - gamma) c_s^2(rho0)
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = a; b < D; ++b)
#pragma unroll
            for (int c = b; c < D; ++c) {
                T v = k3 * (X(a, b, c) + X(a, c, b) + X(b, c, a));
                v += cj * ((a == b ? jtl[c] : T(0)) + (a == c ? jtl[b] : T(0)) + (b == c ? jtl[a] : T(0)));
                auxp<T>(p, AL::XI + sym3<D>(a, b, c))[s] = v;
            }
}

// Reference w_k rho of the local-reference storages, as the float nearest to
// w_k(rho0) rho0 + dw (dw = w_k rho - w_k(rho0) rho0 from the difference formula, accurate to
// its own size).  corr returns w_k rho - ref: the float rounding of w_k(rho0) rho0 and of the sum,
// which the stored deviation carries so that deviation + ref is w_k rho to FP32 accuracy of dw.
__device__ __forceinline__ float local_ref(const Phys<float>& q, int k, float dw, float& corr)
{
    float ref, e;
    two_sum(q.off[k], dw, ref, e);
    corr = __fadd_rn(q.offc[k], e);
    return ref;
}

// velocities in shell k (the rest velocity counts in shell 0)
template <int LAT>
__host__ __device__ constexpr int shell_count(int k)
{
    int m = 0;
    for (int i = 0; i < Lat<LAT>::Q; ++i) m += Lat<LAT>::shell(i) == k ? 1 : 0;
    return m;
}

// Pair (odd index) whose first velocity is +- m c_i: its index, negative when it is -m c_i; 0 if
// no pair has it.
template <int LAT>
__host__ __device__ constexpr int pair_multiple(int i, int m)
{
    using L = Lat<LAT>;
    for (int j = 1; j < L::Q; j += 2) {
        if (L::cx(j) == m * L::cx(i) && L::cy(j) == m * L::cy(i) && L::cz(j) == m * L::cz(i)) return j;
        if (L::cx(j) == -m * L::cx(i) && L::cy(j) == -m * L::cy(i) && L::cz(j) == -m * L::cz(i)) return -j;
    }
    return 0;
}

// Lowest pair index of shell k (0 for the rest shell).
template <int LAT>
__host__ __device__ constexpr int first_pair_of_shell(int k)
{
    for (int i = 1; i < Lat<LAT>::Q; i += 2)
        if (Lat<LAT>::shell(i) == k) return i;
    return 0;
}

// A pair is a base pair unless its velocity is 2 or 4 times another pair's.
template <int LAT>
__host__ __device__ constexpr bool pair_base(int i)
{
    using L = Lat<LAT>;
    for (int j = 1; j < L::Q; j += 2)
        for (int m = 2; m <= 4; m *= 2) {
            const int q = pair_multiple<LAT>(j, m);
            if (q == i || q == -i) return false;
        }
    return true;
}

// f(integral_constant<int, 0>), ..., f(integral_constant<int, N - 1>) at compile time
template <int... I, class F>
__device__ __forceinline__ void static_foreach_impl(std::integer_sequence<int, I...>, F&& f)
{
    (f(std::integral_constant<int, I>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void static_foreach(F&& f)
{
    static_foreach_impl(std::make_integer_sequence<int, N>{}, f);
}

// i and i + 1 are opposite velocities for every odd i (the tables' order)
template <int LAT>
__host__ __device__ constexpr bool pairs_opposite()
{
    using L = Lat<LAT>;
    for (int i = 1; i < L::Q; i += 2)
        if (L::cx(i + 1) != -L::cx(i) || L::cy(i + 1) != -L::cy(i) || L::cz(i + 1) != -L::cz(i) ||
            L::shell(i + 1) != L::shell(i))
            return false;
    return (L::Q & 1) == 1;
}

// Collision of one site with Sigma and Xi' known, and push streaming (S11, S12).
// For a pair c, -c every term of n*_i is even or odd in c:
//   n^eq   = w rho [1 + (c.u)/cs2 + (c.u)^2/(2 cs2^2) - u.u/(2 cs2)]   (Sec. III)
//   Delta^int + Delta^corr = w(rho0) [cf_int c.f + cf_jt c.j~ + cf_h2 h2 + cf_h3 h3]
//   h2 = Sigma : c c - cs0 tr Sigma,  h3 = Xi' : c c c - 3 cs0 (tr Xi')_b c_b     (Sec. VIII)
// so the pair costs one evaluation of the even part E and the odd part O: n*_{+-} = E +- O.
template <int LAT, typename T, int S, bool READ>
__device__ __forceinline__ void collide_tail(const DevSim& p, int src, const Site& r, T drs, const T (&u)[3],
                                             const T (&f)[3], const T (&jtl)[3], const T (&Sig)[3][3],
                                             const T (&Xi)[10])
{
    using L = Lat<LAT>;
    using C = Codec<S>;
    constexpr int D = L::D;
    static_assert(pairs_opposite<LAT>(), "velocity table must list opposite pairs");
    const long long s = r.s;
    const Phys<T>& q = phys<T>(p);
    const T rs = q.rho0 + drs;
    T cs2, dcs2;
    cs2_delta<T>(p, drs, cs2, dcs2);
    const T cs0 = q.cs0;
    T trS = T(0);
#pragma unroll
    for (int a = 0; a < D; ++a) trS += Sig[a][a];
    const T ics2 = T(1) / cs2;
    T uu = T(0);
#pragma unroll
    for (int a = 0; a < D; ++a) uu += u[a] * u[a];
    const T g = q.gamma, omg = T(1) - g;
    const T A1 = T(0.5) * ics2 * ics2, B1 = T(-0.5) * uu * ics2;
    const T h2c = -cs0 * trS;  // the c-independent part of h2
    // c.V gathers the odd terms linear in c: cf_int f + cf_jt j~ - 3 cs0 cf_h3 tr Xi'
    T V[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int b = 0; b < D; ++b) {
        T t = T(0);
#pragma unroll
        for (int a = 0; a < D; ++a) t += Xi[sym3<D>(a, a, b)];
        V[b] = q.cf_int * f[b] + q.cf_jt * jtl[b] - T(3) * cs0 * q.cf_h3 * t;
    }
    // wrapped destination offsets (site indices < 2^31) for the shifts -4, -2, -1, 0, 1, 2, 4
    // that the velocity components take
    int ox[7], oy[7], oz[7];
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        const int sh = k == 0 ? -4 : k == 6 ? 4 : k - 3;
        ox[k] = wrapc(r.x + sh, p.nx);
        oy[k] = wrapc(r.y + sh, p.ny) * p.nx;
        oz[k] = D == 3 ? wrapc(r.z + sh, p.nz) * p.nx * p.ny : 0;
    }
    auto sidx = [](int c) { return c == -4 ? 0 : c == 4 ? 6 : c + 3; };
    // Every population but the rest one; the rest population then takes the
    // remainder, so the stored populations sum to the pre-collision density
    // (sum_i Delta_i = 0 holds exactly for the method's collision operator).
    T stored_sum = T(0);
    float sh = 0.f, sl = 0.f;  // float-pair sum of the stored values (EXACT storages)
    // One pair of opposite velocities (i, i + 1) from its contractions c.u, c.V, Sigma:cc, Xi':ccc.
    auto emit = [&](auto ic, T uc, T lin, T h2, T h3) {
        constexpr int i = decltype(ic)::value;
        const int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
        const int k = L::shell(i);
        // shell constants (pure in k: shared by the shell's pairs).  w(s) = w(s0) + (s - s0) [c1 +
        // c2 (s + s0) + c3 (s^2 + s s0 + s0^2)]: the difference form keeps the relative accuracy of
        // the outer shells' small weights, which the cubic itself would lose to cancellation
        const T w0k = q.w0[k];
        const T dwk = dcs2 * (T(L::wc(k, 1)) + T(L::wc(k, 2)) * (cs2 + cs0) +
                              T(L::wc(k, 3)) * (cs2 * cs2 + cs2 * cs0 + cs0 * cs0));
        const T wl = w0k + dwk;
        const T wr = wl * rs;
        T even0;
        float lref = 0.f, lcorr = 0.f;  // this site's reference for shell k and w rho - reference
        if (C::LOC) {
            // n^eq - w rho = w rho X; the stored value is relative to the float reference
            const T dw0 = wl * drs + q.rho0 * dwk;
            lref = local_ref(p.pf, k, float(dw0), lcorr);
            even0 = omg * (wr * B1) + w0k * q.cf_h2 * h2c + T(lcorr);
            // the reference the decoder adds is this very value (one store per shell)
            if (i == first_pair_of_shell<LAT>(k)) p.wref[src ^ 1][k * p.N + s] = lref;
        } else if (C::DEV) {
            // n^eq - w(rho0) rho0 = w rho X + w drho + rho0 (w(s) - w(s0))
            const T dw0 = wl * drs + q.rho0 * dwk;
            even0 = omg * (wr * B1 + dw0) + w0k * q.cf_h2 * h2c;
        } else {
            even0 = omg * wr * (T(1) + B1) + w0k * q.cf_h2 * h2c;
        }
        const T E = omg * wr * A1 * uc * uc + w0k * q.cf_h2 * h2 + even0;
        const T O = omg * wr * ics2 * uc + w0k * (lin + q.cf_h3 * h3);
        T np = E + O, nm = E - O;
        if (READ) {
            np += g * pop_raw<LAT, S, T>(p, src, i, s);
            nm += g * pop_raw<LAT, S, T>(p, src, i + 1, s);
            if (C::LOC) {  // n - w rho: the stored part, the sender's reference minus this site's
                const float* wf = p.wref[src];
                np += g * (T(__fsub_rn(wf[k * p.N + sender<LAT>(p, r.x, r.y, r.z, i)], lref)) - T(lcorr));
                nm += g * (T(__fsub_rn(wf[k * p.N + sender<LAT>(p, r.x, r.y, r.z, i + 1)], lref)) - T(lcorr));
            }
        }
        const long long dp = ox[sidx(cx)] + oy[sidx(cy)] + oz[sidx(cz)];
        const long long dm = ox[sidx(-cx)] + oy[sidx(-cy)] + oz[sidx(-cz)];
        const T sp = pop_put<LAT, S, T>(p, src ^ 1, i, dp, np);
        const T sm = pop_put<LAT, S, T>(p, src ^ 1, i + 1, dm, nm);
        if (C::LOC) {
            // the decoded values the next moments kernel will sum: stored part plus this site's
            // reference, rounded to float the same way there
            acc2(sh, sl, __fadd_rn(float(sp), lref));
            acc2(sh, sl, __fadd_rn(float(sm), lref));
        } else if (C::EXACT) {
            acc2(sh, sl, float(sp));
            acc2(sh, sl, float(sm));
        } else {
            stored_sum += sp;
            stored_sum += sm;
        }
    };
    // The contractions of the base pairs; a pair whose velocity is m c of a base pair (m = 2, 4)
    // takes them scaled by m, m, m^2, m^3, which is exact in floating point (m a power of two).
    static_foreach<(L::Q - 1) / 2>([&](auto pc) {
        constexpr int i = 2 * decltype(pc)::value + 1;
        if constexpr (pair_base<LAT>(i)) {
            const int c[3] = {L::cx(i), L::cy(i), L::cz(i)};
            T uc = T(0), lin = T(0), h2 = T(0), h3 = T(0);
#pragma unroll
            for (int a = 0; a < D; ++a)
                if (c[a]) { uc += T(c[a]) * u[a]; lin += T(c[a]) * V[a]; }
#pragma unroll
            for (int a = 0; a < D; ++a)
#pragma unroll
                for (int b = a; b < D; ++b)
                    if (c[a] && c[b]) h2 += T((a == b ? 1 : 2) * c[a] * c[b]) * Sig[a][b];
#pragma unroll
            for (int a = 0; a < D; ++a)
#pragma unroll
                for (int b = a; b < D; ++b)
#pragma unroll
                    for (int e = b; e < D; ++e)
                        if (c[a] && c[b] && c[e]) {
                            const int mult = (a == b && b == e) ? 1 : (a == b || b == e) ? 3 : 6;
                            h3 += T(mult * c[a] * c[b] * c[e]) * Xi[sym3<D>(a, b, e)];
                        }
            emit(std::integral_constant<int, i>{}, uc, lin, h2, h3);
            constexpr int j2 = pair_multiple<LAT>(i, 2), j4 = pair_multiple<LAT>(i, 4);
            if constexpr (j2 != 0) {
                constexpr int jp = j2 > 0 ? j2 : -j2;
                const T sg = T(j2 > 0 ? 1 : -1);
                emit(std::integral_constant<int, jp>{}, sg * T(2) * uc, sg * T(2) * lin, T(4) * h2, sg * T(8) * h3);
            }
            if constexpr (j4 != 0) {
                constexpr int jp = j4 > 0 ? j4 : -j4;
                const T sg = T(j4 > 0 ? 1 : -1);
                emit(std::integral_constant<int, jp>{}, sg * T(4) * uc, sg * T(4) * lin, T(16) * h2, sg * T(64) * h3);
            }
        }
    });
    if (C::LOC) {
        // the rest population's reference (shell 0, no pair): it joins the float pair, the others
        // are inside the decoded values
        const T dwk = dcs2 * (T(L::wc(0, 1)) + T(L::wc(0, 2)) * (cs2 + cs0) +
                              T(L::wc(0, 3)) * (cs2 * cs2 + cs2 * cs0 + cs0 * cs0));
        const T dw0 = (q.w0[0] + dwk) * drs + q.rho0 * dwk;
        float corr;
        const float wk = local_ref(p.pf, 0, float(dw0), corr);
        p.wref[src ^ 1][s] = wk;
        acc2(sh, sl, wk);
    }
    // rest population: the stored convention sums to rho - rho0 (global deviations) or rho
    if (C::EXACT) {
        float th = float(drs), tl = cp<float>(p.rho_lo)[s];  // the exact pre-collision sum
        if (!C::DEV || C::LOC) {
            float e;
            two_sum(th, p.pf.rho0, th, e);
            tl = __fadd_rn(tl, e);
        }
        float rh, e;
        two_sum(th, -sh, rh, e);
        const float rl = __fadd_rn(e, __fsub_rn(tl, sl));
        float h2, l2;
        two_sum(rh, rl, h2, l2);
        mp<float2>(p.pop0[src ^ 1])[s] = make_float2(h2, l2);
    } else {
        pop_put<LAT, S, T>(p, src ^ 1, 0, s, (C::DEV ? drs : rs) - stored_sum);
    }
}

// ---------------------------------------------------------------------------
// Tiled kernels.  A CTA owns TX x TY columns of one z-slab of DevSim::zb planes and marches
// along z (2.5D blocking): each plane it loads is kept in a shared-memory ring that
// holds the 5 planes the Sec. IV.B first derivative reaches (2 on each side)
// plus those in flight, so x and y derivatives read the current plane and z
// derivatives the ring.  In 2D the ring is the single plane.
// ---------------------------------------------------------------------------
template <int D>
struct Tile {
    static constexpr int TX = 32, TY = D == 3 ? 8 : 16;
    static constexpr int THREADS = TX * TY;
};

// Ring of the derivative kernel: the 5 planes of the stencil, plus (FP32) one more, so that the
// slot written next never holds a plane the previous pass still reads (one barrier per plane).
template <int D, typename T>
struct DerivsPlan {
    static constexpr int R = D == 3 ? (sizeof(T) == 4 ? 6 : 5) : 1;
    static constexpr bool CLOSING_BARRIER = R < 6;
    __device__ static int slot(int z) { return D == 3 ? (z + 8 * R) % R : 0; }  // z >= -8
    __device__ static void planes(T* ring, int plane_elems, int z, const T* (&pl)[5])
    {
#pragma unroll
        for (int k = 0; k < 5; ++k) pl[k] = ring + slot(D == 3 ? z - 2 + k : 0) * plane_elems;
    }
};

// First derivative of Sec. IV.B along axis a, (2/3)(g(+1) - g(-1)) - (1/12)(g(+2) - g(-2)),
// of a field read by g(plane, index) at in-plane index i (row pitch PX) of the centre plane.
// The Sec. IV.B first derivative from the values at offsets -2, -1, +1, +2.
template <typename T>
__device__ __forceinline__ T d1v(T m2, T m1, T p1, T p2)
{
    return T(2.0 / 3.0) * (p1 - m1) - T(1.0 / 12.0) * (p2 - m2);
}

template <typename T, class G>
__device__ __forceinline__ T d1p(const T* const (&pl)[5], int a, int i, int PX, G g)
{
    if (a == 0)
        return T(2.0 / 3.0) * (g(pl[2], i + 1) - g(pl[2], i - 1)) - T(1.0 / 12.0) * (g(pl[2], i + 2) - g(pl[2], i - 2));
    if (a == 1)
        return T(2.0 / 3.0) * (g(pl[2], i + PX) - g(pl[2], i - PX)) -
               T(1.0 / 12.0) * (g(pl[2], i + 2 * PX) - g(pl[2], i - 2 * PX));
    return T(2.0 / 3.0) * (g(pl[3], i) - g(pl[1], i)) - T(1.0 / 12.0) * (g(pl[4], i) - g(pl[0], i));
}

// Asynchronous element copy global -> shared (cp.async); completion is tracked per thread in
// commit groups, and a barrier after cp.async.wait_group publishes the data to the CTA.
template <int B>
__device__ __forceinline__ void cp_async(void* sdst, const void* gsrc)
{
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(sdst));
    if (B == 16) asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
    else if (B == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gsrc) : "memory");
    else asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// Ask L2 to fetch the line holding p (no register, no completion to wait for).
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];\n" ::"l"(p)); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// ---------------------------------------------------------------------------
// Tensor-memory-access (TMA) plane loads completed on shared-memory mbarriers.
// One thread arms a ring slot's barrier with the bytes it expects and issues the
// tensor copies; every thread then waits on the barrier's phase.  The waits are
// bounded (about a second of clock), so a copy that never lands ends the kernel
// with an error bit instead of a hang.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* q) { return static_cast<unsigned>(__cvta_generic_to_shared(q)); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// the barrier initialisation visible to the tensor copies (async proxy)
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
// shared-memory accesses of the threads ordered before later tensor copies into the same bytes
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n"
        " .reg .pred P;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n"
        " selp.u32 %0, 1, 0, P;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for the phase of the given parity to complete; false after about 2^31 clocks.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > (1ll << 31)) return false;
    return true;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, unsigned long long* bar, int x, int y, int z)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];\n" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, unsigned long long* bar, int x, int y, int z,
                                            int w)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6}], [%2];\n" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z), "r"(w)
        : "memory");
}

// Two consecutive shared-memory elements in one access (the index must be even).
template <typename U>
struct Vec2;
template <>
struct Vec2<float> {
    using type = float2;
};
template <>
struct Vec2<double> {
    using type = double2;
};
template <typename U>
__device__ __forceinline__ typename Vec2<U>::type ld2(const U* p)
{
    return *reinterpret_cast<const typename Vec2<U>::type*>(p);
}
template <typename U>
__device__ __forceinline__ void st2(U* p, U a, U b)
{
    typename Vec2<U>::type v;
    v.x = a;
    v.y = b;
    *reinterpret_cast<typename Vec2<U>::type*>(p) = v;
}

// Shared-memory plan of the sweep: a ring of R planes of u (sweep precision) and rho - rho0
// (storage precision) with in-plane halo 4, PF of them in flight, and the q plane, which
// shares the row pitch UX of the ring so that a warp's stage-Q reads fall in distinct banks.
// One plane in flight and one q buffer keep the plan at 73 KB (FP32), so that three CTAs share
// an SM: at 256^3 that is 0.412 ms per sweep against 0.430 ms for two CTAs with two planes in
// flight and a double-buffered q (95 KB), whose single barrier per phase the second barrier
// here gives back.
template <int D, typename T, typename U>
struct SweepPlan {
    using TL = Tile<D>;
    static constexpr int UX = TL::TX + 8, UY = TL::TY + 8, UP = UX * UY;
    static constexpr int QX = TL::TX + 4, QY = TL::TY + 4, QP = QY * UX;
    static constexpr int NQ = D == 3 ? 6 : 3;
    static constexpr int PF = D == 3 ? 1 : 0;      // planes fetched ahead
    static constexpr int R = D == 3 ? 5 + PF : 1;  // ring planes
    static constexpr int NQB = 1;                  // q plane buffers
    static constexpr size_t OFF_Q = size_t(R) * D * UP * sizeof(U);
    // 128-byte aligned: the rho planes are tensor-copy destinations
    static constexpr size_t OFF_R = (OFF_Q + size_t(NQB) * NQ * QP * sizeof(U) + 127) / 128 * 128;
    // the dynamic shared memory starts after the static barriers, 16-byte aligned only: the kernel
    // moves its ring up to the next 128-byte boundary, within this slack
    static constexpr size_t BYTES = OFF_R + size_t(R) * UP * sizeof(T) + 128;
};

// S3-S6 fused: one sweep of the u-solve, iterated in u = (j0' + j~)/rho (the same iteration
// as in j~, which the paper uses).  The CTA marches along z; per phase zl (two barriers):
//   fetch    plane zl + PF of u and rho - rho0 (in-plane halo 4) into the ring, asynchronously;
//   stage J  at the thread's own site, for the plane zs = zq - 1 that the previous phase's
//            stage Q wrote: the in-plane part d_x q_ax + d_y q_ay of plane zs, and q_az(zs)
//            scattered into the z-derivative sums of planes zs-2 .. zs+2, which live in
//            registers.  Plane zs - 2 is then complete: j~new = -(1/12) d_b q_ab (S5),
//            J(u) = (j0' + j~new)/rho, the update d = c1 d_prev + c2 (J(u) - u), u += d, and
//            the S6 difference rho |d| = |j~new - j~| of the resulting j~ iterates;
//   stage Q  after a barrier (stage J's reads are done), q_ab of plane zq = zl - 2 (in-plane
//            halo 2; the z derivatives read the ring) into the q plane buffer.
// In 2D the march is the single plane: stage Q in the first phase, stage J in the second.
// Plane loads: per-thread cp.async copies.  The TMA form (3D only) instead loads each plane of u
// and rho - rho0 of a tile whose halo box lies inside the lattice in x and y with tensor copies
// into the ring, one thread issuing them and an mbarrier per ring slot tracking them; tiles on the
// periodic seams, whose boxes wrap, still copy per thread.  Both forms give identical results.
template <int LAT, typename T, typename U, bool TMA>
__device__ __forceinline__ void b_sweep(const DevSim& p, int pair, const Blk bid)
{
    using L = Lat<LAT>;
    constexpr int D = L::D;
    using TL = Tile<D>;
    using SP = SweepPlan<D, T, U>;
    using V2 = typename Vec2<U>::type;
    constexpr int TX = TL::TX, TY = TL::TY, NT = TL::THREADS;
    constexpr int UX = SP::UX, UP = SP::UP, QX = SP::QX, QY = SP::QY, QP = SP::QP, NQ = SP::NQ;
    constexpr int PF = SP::PF, R = SP::R;
    constexpr int HZ = D == 3 ? 4 : 0;
    static_assert(TX * TY == NT, "one J site per thread");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long ring_bar[SP::R];  // one per ring slot (TMA)
    // tensor copies write 128-byte aligned destinations; the dynamic window itself starts after the
    // static barriers on a 16-byte boundary
    unsigned char* sm = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    U* su = reinterpret_cast<U*>(sm);             // [R][D][UP]: u
    U* sq = reinterpret_cast<U*>(sm + SP::OFF_Q);  // [NQB][NQ][QP]: q_ab
    T* sr = reinterpret_cast<T*>(sm + SP::OFF_R);  // [R][UP]: rho - rho0
    auto slot = [](int z) { return D == 3 ? (z + 8 * R) % R : 0; };  // z >= -8
    const int tid = threadIdx.x;
    const int x0 = bid.x * TX, y0 = bid.y * TY;
    const int z0 = D == 3 ? bid.z * p.zb : 0;
    const int z1 = D == 3 ? min(z0 + p.zb, p.nz) : 1;
    const long long NP = (long long)p.nx * p.ny;  // sites per plane
    const T* drho = cp<T>(p.rho);
    const int cur = p.us[pair].cur;
    const U* uold = cp<U>(p.uit[pair][cur]);
    U* unew = mp<U>(p.uit[pair][cur ^ 1]);
    const U c1 = U(p.us[pair].c1), c2 = U(p.us[pair].c2);  // this sweep's update (see k_us_ctl)
    U* dvec = mp<U>(p.dvec[pair]);
    const bool use_d = c1 != U(0), keep_d = p.cheb != 0;
    // the thread's own site (stage J)
    const int ix = tid % TX, iy = tid / TX;
    const int gx = x0 + ix, gy = y0 + iy;
    const bool own = gx < p.nx && gy < p.ny;
    const long long own_xy = (long long)gy * p.nx + gx;
    U dmax = U(0), jmax = U(0);  // residual reductions in the sweep's own precision
    bool bad = false;
    // in-plane offsets of the thread's halo points, wrapped once (true modulo: the halo of a
    // small lattice may exceed it)
    // The halo box starts at x0 - 4, a multiple of 4.  When nx is a multiple of the group G, every
    // group of G consecutive box columns is G consecutive, aligned sites of the lattice (the
    // periodic wrap moves whole groups), and goes in one 16-byte copy per field; otherwise the
    // box goes element by element.
    constexpr int G = 16 / (sizeof(U) > sizeof(T) ? sizeof(U) : sizeof(T));
    constexpr int NG = UP / G, MG = (NG + NT - 1) / NT;
    static_assert(UX % G == 0, "box rows hold whole groups");
    const bool vec = p.aligned16 && p.nx % G == 0;
    int goff[MG];  // in-plane lattice offset of the thread's groups
#pragma unroll
    for (int m = 0; m < MG; ++m) {
        const int t = tid + m * NT, gx = t % (UX / G) * G, gy = t / (UX / G);
        goff[m] = t < NG ? wrapm(x0 - 4 + gx, p.nx) + p.nx * wrapm(y0 - 4 + gy, p.ny) : 0;
    }
    auto fetch = [&](int zl) {
        const long long base = D == 3 ? (long long)wrapc(zl, p.nz) * NP : 0;
        U* du = su + slot(zl) * D * UP;
        T* dr = sr + slot(zl) * UP;
        if (vec) {
#pragma unroll
            for (int m = 0; m < MG; ++m) {
                const int t = tid + m * NT;
                if (t < NG) {
                    const int k = t * G;  // box index of the group's first column
                    const long long g = base + goff[m];
#pragma unroll
                    for (int a = 0; a < D; ++a) cp_async<G * sizeof(U)>(du + a * UP + k, uold + a * p.N + g);
                    cp_async<G * sizeof(T)>(dr + k, drho + g);
                }
            }
        } else {
            for (int k = tid; k < UP; k += NT) {
                const long long g = base + wrapm(x0 - 4 + k % UX, p.nx) + (long long)p.nx * wrapm(y0 - 4 + k / UX, p.ny);
#pragma unroll
                for (int a = 0; a < D; ++a) cp_async<sizeof(U)>(du + a * UP + k, uold + a * p.N + g);
                cp_async<sizeof(T)>(dr + k, drho + g);
            }
        }
    };
    // Tensor copies for tiles whose halo box stays inside the lattice in x and y (CTA-uniform).
    // The box starts at x0 - 4, a multiple of 4 sites, as a tensor copy requires.
    bool tma = false;
    if constexpr (D == 3 && TMA) {
        tma = p.tma != 0 && x0 >= 4 && x0 + TX + 4 <= p.nx && y0 >= 4 && y0 + TY + 4 <= p.ny &&
              (smem_u32(sm) & 127u) == 0;
        if (tma) {
            if (tid == 0) {
#pragma unroll
                for (int k = 0; k < R; ++k) mbar_init(&ring_bar[k], 1);
                fence_mbar_init();
                p.us[pair].tma = 1;  // reported by lbm_stats_get
            }
            __syncthreads();
        }
    }
    unsigned phase = 0;  // parity of each ring slot's barrier phase that the next wait expects
    int aborted_at = INT_MIN;  // plane whose tensor copies timed out
    auto fetch_tma = [&](int zl) {
        if (tid == 0) {
            const int sl = slot(zl);
            const int zz = wrapc(zl, p.nz);
            unsigned long long* bar = &ring_bar[sl];
            fence_proxy_async_smem();
            mbar_expect_tx(bar, unsigned(D * UP * sizeof(U) + UP * sizeof(T)));
            const CUtensorMap* um = &p.tmaps->u[pair][cur];
#pragma unroll
            for (int a = 0; a < D; ++a) tma_load_4d(su + (sl * D + a) * UP, um, bar, x0 - 4, y0 - 4, zz, a);
            tma_load_3d(sr + sl * UP, &p.tmaps->rho, bar, x0 - 4, y0 - 4, zz);
        }
    };
    // stage J inputs of the own site (j0', previous update), fetched one plane ahead
    U pj[3] = {U(0), U(0), U(0)}, pd[3] = {U(0), U(0), U(0)};
    auto fetch_j = [&](int zj) {
        if (own && zj >= z0 && zj < z1) {
            const long long g = (D == 3 ? zj * NP : 0) + own_xy;
#pragma unroll
            for (int a = 0; a < D; ++a) {
                pj[a] = U(plane<T>(p.j0pp, a)[g]);
                if (use_d) pd[a] = dvec[a * p.N + g];
            }
        }
    };
    // A[k][a]: sum over b of d_b q_ab at plane zq - 2 + k of the own site, as far as known
    U A[5][3];
#pragma unroll
    for (int k = 0; k < 5; ++k)
#pragma unroll
        for (int a = 0; a < 3; ++a) A[k][a] = U(0);
    U ju[3] = {U(0), U(0), U(0)}, jr = U(0);  // own u and rho - rho0 of the plane being finished
#pragma unroll
    for (int k = 0; k < PF; ++k) {
        if (tma) fetch_tma(z0 - HZ + k);
        else fetch(z0 - HZ + k);
        cp_async_commit();
    }
    fetch_j(z0);
    // q_ab of plane z lives in the q plane buffer (or one of two, with NQB = 2)
    auto qbuf = [&](int z) { return sq + (SP::NQB == 2 ? (z & 1) : 0) * NQ * QP; };
    auto qplane = [&](int z) { return D == 2 ? z == 0 : (z >= z0 - 2 && z < z1 + 2); };
    // Phase zl: stage J of plane zs = zq - 1, from the q that the previous phase wrote, and stage Q
    // of plane zq = zl - HZ/2 into the q buffer once J has read it.  The J stage of plane zs
    // finishes plane zs - 2 (3D), whose own u and rho - rho0 the previous phase read from the
    // ring; the last phase only finishes.
    for (int zl = z0 - HZ; zl < z1 + HZ + 1; ++zl) {
        if (PF == 0) {  // 2D: the single plane, in the first phase
            if (zl < z1 + HZ) fetch(zl);
            cp_async_commit();
        }
        bool late = false;
        if (tma && zl < z1 + HZ) {  // plane zl's tensor copies have landed (the last phase loads none)
            const int sl = slot(zl);
            late = !mbar_wait(&ring_bar[sl], (phase >> sl) & 1u);
            if (!late) phase ^= 1u << sl;
        } else {
            cp_async_wait<PF == 0 ? 0 : PF - 1>();  // plane zl has landed (this thread's copies)
        }
        // ... and everyone's copies; the previous phase is done
        if (!tma) {
            __syncthreads();
        } else if (__syncthreads_or(late)) {
            // a tensor copy did not land in time: record it and stop the solve (below, once the
            // copies still in flight, planes zl .. zl + PF - 1, have landed or timed out)
            aborted_at = zl;
            break;
        }
        // The ring slot of plane zl + PF held plane zl + PF - R = zl - 5, which only the previous
        // phase read.
        if (PF > 0) {
            if (zl + PF < z1 + HZ) {
                if (tma) fetch_tma(zl + PF);
                else fetch(zl + PF);
            }
            cp_async_commit();
        }
        const int zq = zl - HZ / 2, zs = zq - 1;
        if (qplane(zs)) {  // stage J: plane zs, whose q the previous phase wrote
            const U* qb = qbuf(zs);
            const int qi = (iy + 2) * UX + ix + 2;
            if (zs >= z0 && zs < z1) {  // in-plane derivatives of plane zs
                const U* ql[5];
#pragma unroll
                for (int k = 0; k < 5; ++k) ql[k] = qb;
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    U acc = U(0);
#pragma unroll
                    for (int b = 0; b < 2; ++b) {
                        const int c = sym2<D>(a, b);
                        acc += d1p<U>(ql, b, qi, UX, [&](const U* P, int j) { return P[c * QP + j]; });
                    }
                    A[2][a] += acc;
                }
            }
            if (D == 3) {
                // d_z g(z) = (2/3)(g(z+1) - g(z-1)) - (1/12)(g(z+2) - g(z-2)): the share of
                // g(zs) = q_az(zs) in the planes zs-2 .. zs+2
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    const U v = qb[sym2<D>(a, 2) * QP + qi];
                    A[0][a] -= U(1.0 / 12.0) * v;
                    A[1][a] += U(2.0 / 3.0) * v;
                    A[3][a] -= U(2.0 / 3.0) * v;
                    A[4][a] += U(1.0 / 12.0) * v;
                }
            }
            constexpr int KC = D == 3 ? 0 : 2;  // the finished plane: zs - 2 (3D), zs (2D)
            const int zc = D == 3 ? zs - 2 : zs;
            if (own && zc >= z0 && zc < z1) {
                const long long g = (D == 3 ? zc * NP : 0) + own_xy;
                const U rho = phys<U>(p).rho0 + jr;
                const U irho = U(1) / rho;
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    const U jt_new = -(U(1) / U(12)) * A[KC][a];  // S5
                    // residual of the fixed point u = (j0' + j~(u))/rho, the update d, u += d
                    const U res = (pj[a] + jt_new) * irho - ju[a];
                    U d = c2 * res;
                    if (use_d) d += c1 * pd[a];
                    if (keep_d) dvec[a * p.N + g] = d;
                    unew[a * p.N + g] = ju[a] + d;
                    // S6: |j~new - j~| of the plain iteration from the current iterate is rho |res|.
                    // The accelerated update d can be small while res is not (its momentum term
                    // c1 d_prev cancelling c2 res), and large while res is small (the momentum term
                    // still moving the iterate), so the stop needs both below the tolerance.
                    const U dv = rho * fmax(fabs(res), fabs(d));
                    bad |= !(dv == dv);
                    dmax = fmax(dmax, dv);
                    jmax = fmax(jmax, fabs(jt_new));
                }
            }
            if (D == 3) {
#pragma unroll
                for (int k = 0; k < 4; ++k)
#pragma unroll
                    for (int a = 0; a < 3; ++a) A[k][a] = A[k + 1][a];
#pragma unroll
                for (int a = 0; a < 3; ++a) A[4][a] = U(0);
            }
            fetch_j(zc + 1);
        }
        const int zj = zl - HZ;  // own u and rho - rho0 of the plane the next phase finishes
        if (zj >= z0 && zj < z1) {
            const U* uc = su + slot(zj) * D * UP;
            const int ui = (iy + 4) * UX + ix + 4;
#pragma unroll
            for (int a = 0; a < D; ++a) ju[a] = uc[a * UP + ui];
            jr = U(sr[slot(zj) * UP + ui]);
        }
        if (SP::NQB == 1 && D == 3) __syncthreads();  // stage J's reads of the q plane are done
        if (qplane(zq)) {  // stage Q: plane zq, two x-neighbouring points per thread (64-bit reads)
            U* qb = qbuf(zq);
            const U* pl[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) pl[k] = su + slot(D == 3 ? zq - 2 + k : 0) * D * UP;
            const T* rq = sr + slot(zq) * UP;
            constexpr int PX = UX / 2;  // point pairs per row of the pitch
            for (int t = tid; t < QY * PX; t += NT) {
                const int qx = 2 * (t % PX), qy = t / PX;
                if (qx >= QX) continue;
                const int k = qy * UX + qx;      // even: the pair is 2-element aligned
                const int ui = k + 2 * UX + 2;   // (qy + 2) UX + qx + 2
                U du[2][3][3];                   // [point][a][b] = d_a u_b
#pragma unroll
                for (int b = 0; b < D; ++b) {
                    const U* P = pl[2] + b * UP;
                    const V2 xm = ld2<U>(P + ui - 2), xc = ld2<U>(P + ui), xp = ld2<U>(P + ui + 2);
                    du[0][0][b] = d1v<U>(xm.x, xm.y, xc.y, xp.x);
                    du[1][0][b] = d1v<U>(xm.y, xc.x, xp.x, xp.y);
                    const V2 ym2 = ld2<U>(P + ui - 2 * UX), ym1 = ld2<U>(P + ui - UX);
                    const V2 yp1 = ld2<U>(P + ui + UX), yp2 = ld2<U>(P + ui + 2 * UX);
                    du[0][1][b] = d1v<U>(ym2.x, ym1.x, yp1.x, yp2.x);
                    du[1][1][b] = d1v<U>(ym2.y, ym1.y, yp1.y, yp2.y);
                    if (D == 3) {
                        const V2 zm2 = ld2<U>(pl[0] + b * UP + ui), zm1 = ld2<U>(pl[1] + b * UP + ui);
                        const V2 zp1 = ld2<U>(pl[3] + b * UP + ui), zp2 = ld2<U>(pl[4] + b * UP + ui);
                        du[0][2][b] = d1v<U>(zm2.x, zm1.x, zp1.x, zp2.x);
                        du[1][2][b] = d1v<U>(zm2.y, zm1.y, zp1.y, zp2.y);
                    }
                }
                U qv[2][NQ];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    U P, DP, PM, RPP;
                    eos_full<U>(p, phys<U>(p).rho0 + U(rq[ui + h]), P, DP, PM, RPP);
                    U div = U(0);
#pragma unroll
                    for (int a = 0; a < D; ++a) div += du[h][a][a];
#pragma unroll
                    for (int a = 0; a < D; ++a)
#pragma unroll
                        for (int b = a; b < D; ++b)
                            qv[h][sym2<D>(a, b)] = (a == b ? PM * div : U(0)) + P * (du[h][b][a] + du[h][a][b]);
                }
#pragma unroll
                for (int c = 0; c < NQ; ++c) st2<U>(qb + c * QP + k, qv[0][c], qv[1][c]);
            }
        }
    }
    cp_async_wait<0>();
    if (aborted_at != INT_MIN) {
        if (tid == 0) {
            atomicOr(p.status, STB_TIMEOUT);
            for (int z = aborted_at; z < aborted_at + PF && z < z1 + HZ; ++z)
                (void)mbar_wait(&ring_bar[slot(z)], (phase >> slot(z)) & 1u);
        }
        bad = true;  // the residual reads as infinite: the control kernel ends the solve
    }
    // NaN -> +inf, which orders above every finite residual
    const double dmax_d = bad ? __longlong_as_double(0x7ff0000000000000ll) : double(dmax);
    block_max2(dmax_d, double(jmax), &p.us[pair].resid_bits, &p.us[pair].jmax_bits);
}
template <int LAT, typename T, typename U, bool TMA>
__global__ void __launch_bounds__(Tile<Lat<LAT>::D>::THREADS, sizeof(U) == 4 ? 3 : 1) k_sweep(DevSim p, int pair)
{
    b_sweep<LAT, T, U, TMA>(p, pair, launch_blk());
}

// S2 (tiled): f = kappa rho d_a lap rho with the third-derivative stencil of Sec. IV.E,
// j0' = j0 + (h/2) f, and the start of the u-solve u = (j0' + j~)/rho with j~ of the previous
// step (warm start, Sec. IX item 3) or j~ = 0 (S1).  The CTA marches along z; rho - rho0 of
// each plane (in-plane halo 2) arrives by cp.async in a ring of 5 + PF planes.
template <int D>
struct ForcePlan {
    using TL = Tile<D>;
    static constexpr int RX = TL::TX + 4, RY = TL::TY + 4, RP = RX * RY;
    static constexpr int PF = D == 3 ? 2 : 0;
    static constexpr int R = D == 3 ? 5 + PF : 1;
    __device__ static int slot(int z) { return D == 3 ? (z + 8 * R) % R : 0; }  // z >= -8
};

template <int LAT, typename T, typename U>
__device__ __forceinline__ void b_force(const DevSim& p, int pair, const Blk bid)
{
    using L = Lat<LAT>;
    constexpr int D = L::D;
    using TL = Tile<D>;
    using FP = ForcePlan<D>;
    constexpr int TX = TL::TX, TY = TL::TY, NT = TL::THREADS;
    constexpr int RX = FP::RX, RP = FP::RP, PF = FP::PF;
    constexpr int HZ = D == 3 ? 2 : 0;
    static_assert(TX * TY == NT, "one site per thread");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sr = reinterpret_cast<T*>(smem_raw);  // [R][RY][RX]: rho - rho0
    const int tid = threadIdx.x;
    const int x0 = bid.x * TX, y0 = bid.y * TY;
    const int z0 = D == 3 ? bid.z * p.zb : 0;
    const int z1 = D == 3 ? min(z0 + p.zb, p.nz) : 1;
    const long long NP = (long long)p.nx * p.ny;
    const T* drho = cp<T>(p.rho);
    U* u0 = mp<U>(p.uit[pair][p.us[pair].cur]);
    const int ix = tid % TX, iy = tid / TX;
    const int gx = x0 + ix, gy = y0 + iy;
    const bool own = gx < p.nx && gy < p.ny;
    const long long own_xy = (long long)gy * p.nx + gx;
    // pairs of box columns in one copy when nx is even (see the collision kernel's ring)
    constexpr int G = 2, NG = RP / G, MG = (NG + NT - 1) / NT;
    const bool vec = p.aligned16 && p.nx % G == 0;
    int goff[MG];
#pragma unroll
    for (int m = 0; m < MG; ++m) {
        const int t = tid + m * NT, gx = t % (RX / G) * G, gy = t / (RX / G);
        goff[m] = t < NG ? wrapm(x0 - 2 + gx, p.nx) + p.nx * wrapm(y0 - 2 + gy, p.ny) : 0;
    }
    auto fetch = [&](int zl) {
        const long long base = D == 3 ? (long long)wrapc(zl, p.nz) * NP : 0;
        T* dst = sr + FP::slot(zl) * RP;
        if (vec) {
#pragma unroll
            for (int m = 0; m < MG; ++m) {
                const int t = tid + m * NT;
                if (t < NG) cp_async<G * sizeof(T)>(dst + t * G, drho + base + goff[m]);
            }
        } else {
            for (int k = tid; k < RP; k += NT)
                cp_async<sizeof(T)>(dst + k, drho + base + wrapm(x0 - 2 + k % RX, p.nx) +
                                                 (long long)p.nx * wrapm(y0 - 2 + k / RX, p.ny));
        }
    };
    // own-site inputs (j0, warm-start j~), fetched one plane ahead.  The extrapolated start
    // j~_n + theta (j~_n - j~_n-1) continues the change of the last step.
    T pj[3] = {T(0), T(0), T(0)};
    U pw[3] = {U(0), U(0), U(0)};
    const int ws = p.us[0].wsel;
    const U theta = U(p.wtheta);
    auto fetch_own = [&](int z) {
        if (own && z >= z0 && z < z1) {
            const long long g = (D == 3 ? z * NP : 0) + own_xy;
#pragma unroll
            for (int a = 0; a < D; ++a) {
                pj[a] = plane<T>(p.j0pp, a)[g];
                if (p.warm) {
                    const U jn = plane<U>(p.jwp[ws], a)[g];
                    pw[a] = p.warm == 2 ? jn + theta * (jn - plane<U>(p.jwp[ws ^ 1], a)[g]) : jn;
                }
            }
        }
    };
#pragma unroll
    for (int k = 0; k < PF; ++k) {
        fetch(z0 - HZ + k);
        cp_async_commit();
    }
    fetch_own(z0);
    for (int zl = z0 - HZ; zl < z1 + HZ; ++zl) {
        if (PF == 0) {  // 2D: the single plane, in this one pass
            fetch(zl);
            cp_async_commit();
        }
        cp_async_wait<PF == 0 ? 0 : PF - 1>();  // plane zl has landed (this thread's copies)
        __syncthreads();                         // ... and everyone's; the previous pass's reads are done
        // The slot of plane zl + PF held plane zl + PF - R = zl - 5, which only the previous
        // pass read, so one barrier per plane suffices.
        if (PF > 0) {
            if (zl + PF < z1 + HZ) fetch(zl + PF);
            cp_async_commit();
        }
        const int zc = zl - HZ;
        if (own && zc >= z0 && zc < z1) {
            const T* pl[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) pl[k] = sr + FP::slot(D == 3 ? zc - 2 + k : 0) * RP;
            const int ri = (iy + 2) * RX + ix + 2;
            // rho - rho0 at offset (dx, dy, dz) from the site
            auto R = [&](int dx, int dy, int dz) { return pl[2 + dz][ri + dx + dy * RX]; };
            const long long g = (D == 3 ? zc * NP : 0) + own_xy;
            const T rs = phys<T>(p).rho0 + R(0, 0, 0);
            const U rho = U(rs);
#pragma unroll
            for (int a = 0; a < D; ++a) {
                const int ex = a == 0, ey = a == 1, ez = a == 2;
                const T ax = R(ex, ey, ez) - R(-ex, -ey, -ez);
                const T two = R(2 * ex, 2 * ey, 2 * ez) - R(-2 * ex, -2 * ey, -2 * ez);
                T diag = T(0);
#pragma unroll
                for (int b = 0; b < D; ++b) {
                    if (b == a) continue;
                    const int bx = b == 0, by = b == 1, bz = b == 2;
#pragma unroll
                    for (int sg = -1; sg <= 1; sg += 2)
                        diag += R(ex + sg * bx, ey + sg * by, ez + sg * bz) - R(-ex + sg * bx, -ey + sg * by, -ez + sg * bz);
                }
                // sum_i tau_i d_ia rho(r + d_i): the (2 0) shell has d_a = +-2
                const T lap3 = T(L::T3_AX) * ax + T(L::T3_DIAG) * diag + T(2.0 * L::T3_TWO) * two;
                const T fa = phys<T>(p).kappa * rs * lap3;
                const T j = pj[a] + T(0.5) * fa;  // S2: j0' = j0 + (h/2) f
                plane<T>(p.fpp, a)[g] = fa;
                plane<T>(p.j0pp, a)[g] = j;
                u0[a * p.N + g] = (U(j) + pw[a]) / rho;
            }
        }
        if (zc >= z0 && zc < z1) fetch_own(zc + 1);
        // the own-site inputs of the plane after that into L2, every thread its own site:
        // 0.254 -> 0.232 ms at 256^3 (0.237 with one lane per field and tile row)
        if (D == 3 && own && zc + 2 >= z0 && zc + 2 < z1) {
            const long long g = (long long)(zc + 2) * NP + own_xy;
#pragma unroll
            for (int a = 0; a < D; ++a) {
                prefetch_l2(plane<T>(p.j0pp, a) + g);
                if (p.warm) prefetch_l2(plane<U>(p.jwp[ws], a) + g);
                if (p.warm == 2) prefetch_l2(plane<U>(p.jwp[ws ^ 1], a) + g);
            }
        }
    }
}
template <int LAT, typename T, typename U>
__global__ void __launch_bounds__(Tile<Lat<LAT>::D>::THREADS) k_force(DevSim p, int pair)
{
    b_force<LAT, T, U>(p, pair, launch_blk());
}

// S8 and S10 (tiled): the pointwise rho, u, p of every plane go to the ring
// (halo 2); the first derivatives of u, j = rho u, p, p/rho and p u_b u_c
// at the tile's sites feed derivs_tail.
template <int LAT, typename T, typename U>
__device__ __forceinline__ void b_derivs(const DevSim& p, const Blk bid)
{
    using L = Lat<LAT>;
    constexpr int D = L::D;
    using TL = Tile<D>;
    constexpr int TX = TL::TX, TY = TL::TY;
    constexpr int RX = TX + 4, RY = TY + 4, NP = 6;  // u_x, u_y, u_z, rho, p, p/rho
    constexpr int HZ = D == 3 ? 2 : 0;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sr = reinterpret_cast<T*>(smem_raw);  // [R][NP][RY][RX]
    const int tid = threadIdx.x, nth = blockDim.x;
    const int x0 = bid.x * TX, y0 = bid.y * TY;
    const int z0 = D == 3 ? bid.z * p.zb : 0;
    const int z1 = D == 3 ? min(z0 + p.zb, p.nz) : 1;
    const T* drho = cp<T>(p.rho);
    const U* uu = cp<U>(p.uit[0][p.us[0].cur]);  // S8: the converged u
    constexpr int MR = (RX * RY + TL::THREADS - 1) / TL::THREADS;
    int hoff[MR];  // wrapped in-plane offsets of the halo points
#pragma unroll
    for (int m = 0; m < MR; ++m) {
        const int k = tid + m * nth;
        hoff[m] = k < RX * RY ? wrapm(x0 - 2 + k % RX, p.nx) + p.nx * wrapm(y0 - 2 + k / RX, p.ny) : 0;
    }
    T pr[MR];
    U pt[MR][3];
    auto fetch = [&](int zl) {
        const long long base = D == 3 ? (long long)wrapc(zl, p.nz) * p.nx * p.ny : 0;
#pragma unroll
        for (int m = 0; m < MR; ++m) {
            const int k = tid + m * nth;
            if (k < RX * RY) {
                const long long g = base + hoff[m];
                pr[m] = drho[g];
#pragma unroll
                for (int a = 0; a < D; ++a) pt[m][a] = uu[a * p.N + g];
            }
        }
    };
    fetch(z0 - HZ);
    for (int zl = z0 - HZ; zl < z1 + HZ; ++zl) {
        {
            T* dst = sr + DerivsPlan<D, T>::slot(zl) * NP * RY * RX;
#pragma unroll
            for (int m = 0; m < MR; ++m) {
                const int k = tid + m * nth;
                if (k < RX * RY) {
                    const T rho = phys<T>(p).rho0 + pr[m];
#pragma unroll
                    for (int a = 0; a < 3; ++a) dst[a * RY * RX + k] = a < D ? T(pt[m][a]) : T(0);
                    // p and p/rho as deviations from their values at rho0, from the difference
                    // formula: the derivative stencils (weights summing to zero) see the same
                    // differences without the rounding of the O(1) offsets
                    T cs2, dcs2;
                    cs2_delta<T>(p, pr[m], cs2, dcs2);
                    dst[3 * RY * RX + k] = rho;
                    dst[4 * RY * RX + k] = phys<T>(p).rho0 * dcs2 + pr[m] * cs2;  // p - p(rho0)
                    dst[5 * RY * RX + k] = dcs2;                                   // p/rho - c_s^2(rho0)
                }
            }
            if (zl + 1 < z1 + HZ) fetch(zl + 1);
        }
        __syncthreads();
        const int zc = zl - HZ;
        if (zc + kDerivsLead >= z0 && zc + kDerivsLead < z1 && tid < TX * TY) {
            // j0' of a plane ahead, into L2 while this plane computes
            const int gx = min(x0 + tid % TX, p.nx - 1), gy = min(y0 + tid / TX, p.ny - 1);
            const long long sn = at(p, gx, gy, D == 3 ? zc + kDerivsLead : 0);
#pragma unroll
            for (int a = 0; a < D; ++a) prefetch_l2(plane<T>(p.j0pp, a) + sn);
        }
        if (zc >= z0 && zc < z1) {
            const int gz = D == 3 ? zc : 0;
            const T* pl[5];
            const T p0 = phys<T>(p).rho0 * phys<T>(p).cs0;  // p(rho0)
            DerivsPlan<D, T>::planes(sr, NP * RY * RX, zc, pl);
            constexpr int PS = RY * RX;
            for (int k = tid; k < TX * TY; k += nth) {
                const int ix = k % TX, iy = k / TX;
                const int gx = x0 + ix, gy = y0 + iy;
                if (gx >= p.nx || gy >= p.ny) continue;
                const int ri = (iy + 2) * RX + ix + 2;
                T du[3][3], dp[3], dpr[3], dpuu[3][3][3];
                T divj = T(0);
#pragma unroll
                for (int a = 0; a < D; ++a) {
#pragma unroll
                    for (int b = 0; b < D; ++b)
                        du[a][b] = d1p<T>(pl, a, ri, RX, [&](const T* P, int j) { return P[b * PS + j]; });
                    divj += d1p<T>(pl, a, ri, RX, [&](const T* P, int j) { return P[3 * PS + j] * P[a * PS + j]; });
                    dp[a] = d1p<T>(pl, a, ri, RX, [&](const T* P, int j) { return P[4 * PS + j]; });
                    dpr[a] = d1p<T>(pl, a, ri, RX, [&](const T* P, int j) { return P[5 * PS + j]; });
#pragma unroll
                    for (int b = 0; b < D; ++b)
#pragma unroll
                        for (int c = b; c < D; ++c)
                            dpuu[a][b][c] = d1p<T>(pl, a, ri, RX, [&](const T* P, int j) {
                                return (p0 + P[4 * PS + j]) * P[b * PS + j] * P[c * PS + j];
                            });
                }
                const long long s = at(p, gx, gy, gz);
                const T u[3] = {pl[2][ri], pl[2][PS + ri], pl[2][2 * PS + ri]};
                const T rs = pl[2][3 * PS + ri];
                T jtl[3] = {T(0), T(0), T(0)};  // j~ = rho u - j0' (S8)
#pragma unroll
                for (int a = 0; a < D; ++a) jtl[a] = rs * u[a] - plane<T>(p.j0pp, a)[s];
                derivs_tail<LAT, T>(p, s, du, divj, dp, dpr, dpuu, rs, u, jtl);
            }
        }
        if (DerivsPlan<D, T>::CLOSING_BARRIER) __syncthreads();
    }
}
// The one-simulation kernel keeps its own copy of the body with blockIdx: routing it through
// b_derivs made it 30 % slower (0.67 against 0.52 ms at 256^3), which the other kernels do not show.
// With FP32 fields and u-solve three CTAs share an SM (80 registers, 62 KB of shared memory
// each): 0.474 ms against 0.505 ms for two at 256^3.
template <int LAT, typename T, typename U>
__global__ void __launch_bounds__(Tile<Lat<LAT>::D>::THREADS, sizeof(T) == 4 && sizeof(U) == 4 ? 3 : 2) k_derivs(DevSim p)
{
    using L = Lat<LAT>;
    constexpr int D = L::D;
    using TL = Tile<D>;
    constexpr int TX = TL::TX, TY = TL::TY;
    constexpr int RX = TX + 4, RY = TY + 4, NP = 6;  // u_x, u_y, u_z, rho, p, p/rho
    constexpr int HZ = D == 3 ? 2 : 0;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sr = reinterpret_cast<T*>(smem_raw);  // [R][NP][RY][RX]
    const int tid = threadIdx.x, nth = blockDim.x;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = D == 3 ? int(blockIdx.z) * p.zb : 0;
    const int z1 = D == 3 ? min(z0 + p.zb, p.nz) : 1;
    const T* drho = cp<T>(p.rho);
    const U* uu = cp<U>(p.uit[0][p.us[0].cur]);  // S8: the converged u
    constexpr int MR = (RX * RY + TL::THREADS - 1) / TL::THREADS;
    int hoff[MR];  // wrapped in-plane offsets of the halo points
#pragma unroll
    for (int m = 0; m < MR; ++m) {
        const int k = tid + m * nth;
        hoff[m] = k < RX * RY ? wrapm(x0 - 2 + k % RX, p.nx) + p.nx * wrapm(y0 - 2 + k / RX, p.ny) : 0;
    }
    T pr[MR];
    U pt[MR][3];
    auto fetch = [&](int zl) {
        const long long base = D == 3 ? (long long)wrapc(zl, p.nz) * p.nx * p.ny : 0;
#pragma unroll
        for (int m = 0; m < MR; ++m) {
            const int k = tid + m * nth;
            if (k < RX * RY) {
                const long long g = base + hoff[m];
                pr[m] = drho[g];
#pragma unroll
                for (int a = 0; a < D; ++a) pt[m][a] = uu[a * p.N + g];
            }
        }
    };
    fetch(z0 - HZ);
    for (int zl = z0 - HZ; zl < z1 + HZ; ++zl) {
        {
            T* dst = sr + DerivsPlan<D, T>::slot(zl) * NP * RY * RX;
#pragma unroll
            for (int m = 0; m < MR; ++m) {
                const int k = tid + m * nth;
                if (k < RX * RY) {
                    const T rho = phys<T>(p).rho0 + pr[m];
#pragma unroll
                    for (int a = 0; a < 3; ++a) dst[a * RY * RX + k] = a < D ? T(pt[m][a]) : T(0);
                    // p and p/rho as deviations from their values at rho0, from the difference
                    // formula: the derivative stencils (weights summing to zero) see the same
                    // differences without the rounding of the O(1) offsets
                    T cs2, dcs2;
                    cs2_delta<T>(p, pr[m], cs2, dcs2);
                    dst[3 * RY * RX + k] = rho;
                    dst[4 * RY * RX + k] = phys<T>(p).rho0 * dcs2 + pr[m] * cs2;  // p - p(rho0)
                    dst[5 * RY * RX + k] = dcs2;                                   // p/rho - c_s^2(rho0)
                }
            }
            if (zl + 1 < z1 + HZ) fetch(zl + 1);
        }
        __syncthreads();
        const int zc = zl - HZ;
        if (zc + kDerivsLead >= z0 && zc + kDerivsLead < z1 && tid < TX * TY) {
            // j0' of a plane ahead, into L2 while this plane computes
            const int gx = min(x0 + tid % TX, p.nx - 1), gy = min(y0 + tid / TX, p.ny - 1);
            const long long sn = at(p, gx, gy, D == 3 ? zc + kDerivsLead : 0);
#pragma unroll
            for (int a = 0; a < D; ++a) prefetch_l2(plane<T>(p.j0pp, a) + sn);
        }
        if (zc >= z0 && zc < z1) {
            const int gz = D == 3 ? zc : 0;
            const T* pl[5];
            const T p0 = phys<T>(p).rho0 * phys<T>(p).cs0;  // p(rho0)
            DerivsPlan<D, T>::planes(sr, NP * RY * RX, zc, pl);
            constexpr int PS = RY * RX;
            for (int k = tid; k < TX * TY; k += nth) {
                const int ix = k % TX, iy = k / TX;
                const int gx = x0 + ix, gy = y0 + iy;
                if (gx >= p.nx || gy >= p.ny) continue;
                const int ri = (iy + 2) * RX + ix + 2;
                T du[3][3], dp[3], dpr[3], dpuu[3][3][3];
                T divj = T(0);
#pragma unroll
                for (int a = 0; a < D; ++a) {
#pragma unroll
                    for (int b = 0; b < D; ++b)
                        du[a][b] = d1p<T>(pl, a, ri, RX, [&](const T* P, int j) { return P[b * PS + j]; });
                    divj += d1p<T>(pl, a, ri, RX, [&](const T* P, int j) { return P[3 * PS + j] * P[a * PS + j]; });
                    dp[a] = d1p<T>(pl, a, ri, RX, [&](const T* P, int j) { return P[4 * PS + j]; });
                    dpr[a] = d1p<T>(pl, a, ri, RX, [&](const T* P, int j) { return P[5 * PS + j]; });
#pragma unroll
                    for (int b = 0; b < D; ++b)
#pragma unroll
                        for (int c = b; c < D; ++c)
                            dpuu[a][b][c] = d1p<T>(pl, a, ri, RX, [&](const T* P, int j) {
                                return (p0 + P[4 * PS + j]) * P[b * PS + j] * P[c * PS + j];
                            });
                }
                const long long s = at(p, gx, gy, gz);
                const T u[3] = {pl[2][ri], pl[2][PS + ri], pl[2][2 * PS + ri]};
                const T rs = pl[2][3 * PS + ri];
                T jtl[3] = {T(0), T(0), T(0)};  // j~ = rho u - j0' (S8)
#pragma unroll
                for (int a = 0; a < D; ++a) jtl[a] = rs * u[a] - plane<T>(p.j0pp, a)[s];
                derivs_tail<LAT, T>(p, s, du, divj, dp, dpr, dpuu, rs, u, jtl);
            }
        }
        if (DerivsPlan<D, T>::CLOSING_BARRIER) __syncthreads();
    }
}


// Ring of the collision kernel: the 5 planes of the derivative stencil and PF planes in flight;
// the copy into the next slot starts after the plane's barrier (one barrier per plane).
template <int D>
struct CollidePlan {
    static constexpr int PF = D == 3 ? 1 : 0;
    static constexpr int R = D == 3 ? 5 + PF : 1;
    __device__ static int slot(int z) { return D == 3 ? (z + 8 * R) % R : 0; }  // z >= -8
    template <typename T>
    __device__ static void planes(T* ring, int plane_elems, int z, const T* (&pl)[5])
    {
#pragma unroll
        for (int k = 0; k < 5; ++k) pl[k] = ring + slot(D == 3 ? z - 2 + k : 0) * plane_elems;
    }
};

// S11 (rest) and S12 (tiled): A, B, C of every plane go to the ring (halo 2);
// d_a A, d_g B_ag and d_a C_b at the tile's sites complete Sigma; collide_tail
// then collides and streams.
template <int LAT, typename T, int S, typename U, bool READ>
__device__ __forceinline__ void b_collide(const DevSim& p, int src, const Blk bid)
{
    using L = Lat<LAT>;
    constexpr int D = L::D;
    using AL = AuxLayout<D>;
    using TL = Tile<D>;
    constexpr int TX = TL::TX, TY = TL::TY;
    constexpr int RX = TX + 4, RY = TY + 4, NP = 1 + AL::NB + D;  // A, B, C
    constexpr int HZ = D == 3 ? 2 : 0;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sr = reinterpret_cast<T*>(smem_raw);  // [R][NP][RY][RX]
    const int tid = threadIdx.x, nth = blockDim.x;
    const int x0 = bid.x * TX, y0 = bid.y * TY;
    const int z0 = D == 3 ? bid.z * p.zb : 0;
    const int z1 = D == 3 ? min(z0 + p.zb, p.nz) : 1;
    const T* drho = cp<T>(p.rho);
    const U* uu = cp<U>(p.uit[0][p.us[0].cur]);
    const int ws = p.us[0].wsel;  // the warm-start buffer this step's j~ goes to
    T k1, k2, k3;
    collision_consts<LAT, T>(p, k1, k2, k3);
    // The halo box starts at x0 - 2, an even column: with nx even, each pair of box columns is
    // two aligned lattice sites (the periodic wrap moves whole pairs) and goes in one copy.
    constexpr int G = 2, NG = RX * RY / G, MG = (NG + TL::THREADS - 1) / TL::THREADS;
    const bool vec = p.aligned16 && p.nx % G == 0;
    int goff[MG];  // in-plane lattice offset of the thread's pairs
#pragma unroll
    for (int m = 0; m < MG; ++m) {
        const int t = tid + m * nth, gx = t % (RX / G) * G, gy = t / (RX / G);
        goff[m] = t < NG ? wrapm(x0 - 2 + gx, p.nx) + p.nx * wrapm(y0 - 2 + gy, p.ny) : 0;
    }
    // A, B, C of plane zl into its ring slot, asynchronously
    auto fetch = [&](int zl) {
        const long long base = D == 3 ? (long long)wrapc(zl, p.nz) * p.nx * p.ny : 0;
        T* dst = sr + CollidePlan<D>::slot(zl) * NP * RY * RX;
        if (vec) {
#pragma unroll
            for (int m = 0; m < MG; ++m) {
                const int t = tid + m * nth;
                if (t < NG) {
                    const long long g = base + goff[m];
#pragma unroll
                    for (int c = 0; c < NP; ++c)
                        cp_async<G * sizeof(T)>(dst + c * RY * RX + t * G, auxp<T>(p, AL::A + c) + g);
                }
            }
        } else {
            for (int k = tid; k < RX * RY; k += nth) {
                const long long g = base + wrapm(x0 - 2 + k % RX, p.nx) + (long long)p.nx * wrapm(y0 - 2 + k / RX, p.ny);
#pragma unroll
                for (int c = 0; c < NP; ++c) cp_async<sizeof(T)>(dst + c * RY * RX + k, auxp<T>(p, AL::A + c) + g);
            }
        }
    };
    constexpr int PF = CollidePlan<D>::PF;
#pragma unroll
    for (int k = 0; k < PF; ++k) {
        fetch(z0 - HZ + k);
        cp_async_commit();
    }
    // the thread's site in the tile (one site per thread)
    const int ix = tid % TX, iy = tid / TX;
    const int gx = x0 + ix, gy = y0 + iy;
    for (int zl = z0 - HZ; zl < z1 + HZ; ++zl) {
        const int zc = zl - HZ;
        const int gz = D == 3 ? zc : 0;
        const bool act = zc >= z0 && zc < z1 && gx < p.nx && gy < p.ny;
        // The site's own inputs are loaded before the barrier, so their latency overlaps the
        // wait for the ring; nothing else is live here.
        const long long s = act ? at(p, gx, gy, gz) : 0;
        T drs = T(0), j0s[3] = {T(0), T(0), T(0)}, f[3] = {T(0), T(0), T(0)};
        U ua[3] = {U(0), U(0), U(0)};
        T sigl[6];
        if (act) {
            drs = drho[s];
#pragma unroll
            for (int a = 0; a < D; ++a) {
                ua[a] = uu[a * p.N + s];
                j0s[a] = plane<T>(p.j0pp, a)[s];
                f[a] = plane<T>(p.fpp, a)[s];
            }
#pragma unroll
            for (int q = 0; q < AL::NB; ++q) sigl[q] = auxp<T>(p, AL::SIGL + q)[s];
        }
        if (PF == 0) {  // 2D: the single plane, in this one pass
            fetch(zl);
            cp_async_commit();
        }
        cp_async_wait<0>();  // plane zl has landed (this thread's copies)
        __syncthreads();     // ... and everyone's; the previous pass's reads are done
        // The slot of plane zl + PF held plane zl + PF - R = zl - 5, which only the previous
        // pass read, so one barrier per plane suffices.
        if (PF > 0) {
            if (zl + PF < z1 + HZ) fetch(zl + PF);
            cp_async_commit();
        }
        if (zc + kCollideLead >= z0 && zc + kCollideLead < z1 && tid < TX * TY) {
            // the per-site inputs of a plane ahead, into L2 while this plane computes (every thread
            // its own site: 1.651 ms at 256^3, against 1.662 with one lane per field and tile row)
            const int gx = min(x0 + tid % TX, p.nx - 1), gy = min(y0 + tid / TX, p.ny - 1);
            const long long sn = at(p, gx, gy, D == 3 ? zc + kCollideLead : 0);
#pragma unroll
            for (int c = AL::SIGL; c < AL::XI + AL::NX; ++c) prefetch_l2(auxp<T>(p, c) + sn);
#pragma unroll
            for (int a = 0; a < D; ++a) {
                prefetch_l2(uu + a * p.N + sn);
                prefetch_l2(plane<T>(p.j0pp, a) + sn);
                prefetch_l2(plane<T>(p.fpp, a) + sn);
            }
            prefetch_l2(drho + sn);
            if (Codec<S>::EXACT) prefetch_l2(cp<float>(p.rho_lo) + sn);
        }
        if (act) {
            const T* pl[5];
            CollidePlan<D>::planes(sr, NP * RY * RX, zc, pl);
            constexpr int PS = RY * RX;
            {
                const int ri = (iy + 2) * RX + ix + 2;
                Site r;
                r.x = gx; r.y = gy; r.z = gz; r.s = s;
                const T rs = phys<T>(p).rho0 + drs;
                T u[3] = {T(0), T(0), T(0)}, jtl[3] = {T(0), T(0), T(0)};
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    u[a] = T(ua[a]);
                    const U jta = U(rs) * ua[a] - U(j0s[a]);  // j~ = rho u - j0' (S8)
                    jtl[a] = T(jta);
                    plane<U>(p.jwp[ws], a)[s] = jta;  // the next step's warm start
                }
                T P, DP, PM, RPP;
                eos_full<T>(p, rs, P, DP, PM, RPP);
                T dA[3], divB[3], dC[3][3];
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    dA[a] = d1p<T>(pl, a, ri, RX, [&](const T* P, int j) { return P[j]; });
                    T acc = T(0);
#pragma unroll
                    for (int g2 = 0; g2 < D; ++g2) {
                        const int kb = 1 + sym2<D>(a, g2);
                        acc += d1p<T>(pl, g2, ri, RX, [&](const T* P, int j) { return P[kb * PS + j]; });
                    }
                    divB[a] = acc;
#pragma unroll
                    for (int b = 0; b < D; ++b)
                        dC[a][b] = d1p<T>(pl, a, ri, RX, [&](const T* P, int j) { return P[(1 + AL::NB + b) * PS + j]; });
                }
                T trdC = T(0);
#pragma unroll
                for (int a = 0; a < D; ++a) trdC += dC[a][a];
                T Sig[3][3];
#pragma unroll
                for (int a = 0; a < D; ++a)
#pragma unroll
                    for (int b = a; b < D; ++b) {
                        T v = k1 * (u[a] * (dA[b] + divB[b]) + u[b] * (dA[a] + divB[a]));
                        v += k2 * (-P * (dC[a][b] + dC[b][a]) - (a == b ? PM * trdC : T(0)));
                        v += sigl[sym2<D>(a, b)];
                        Sig[a][b] = v;
                        Sig[b][a] = v;
                    }
                T Xi[10];
#pragma unroll
                for (int q = 0; q < AL::NX; ++q) Xi[q] = auxp<T>(p, AL::XI + q)[s];
                collide_tail<LAT, T, S, READ>(p, src, r, drs, u, f, jtl, Sig, Xi);
            }
        }
    }
}
template <int LAT, typename T, int S, typename U, bool READ>
__global__ void __launch_bounds__(Tile<Lat<LAT>::D>::THREADS, 2) k_collide(DevSim p, int src)
{
    b_collide<LAT, T, S, U, READ>(p, src, launch_blk());
}

// ---------------------------------------------------------------------------
// Batched forms of the step kernels.  A persistent grid walks the work list of every
// simulation in the table: pass `item` is block (or tile) item - start[k] of slot k.  Slots
// that do not take this step, and in the u-solve those whose solve has stopped, are skipped.
// Every block runs the same body as the one-simulation launch, so each simulation's result
// is bitwise the one it gets alone.
// ---------------------------------------------------------------------------
// slot holding work item `item` in the prefix table start[0..n] (a short scan: n <= 32)
__device__ __forceinline__ int batch_slot(const int* start, int n, int item)
{
    int k = 0;
    while (k + 1 < n && start[k + 1] <= item) ++k;
    return k;
}

static __global__ void kb_step_begin(const DevSim* sims, BatchWork* w)
{
    const int k = threadIdx.x;
    if (k < kBatchSlots) w->live[k] = (k < w->nslot && w->todo[k] > 0) ? 1 : 0;
}

static __global__ void kb_step_end(const DevSim* sims, BatchWork* w)
{
    const int k = threadIdx.x;
    if (k < kBatchSlots && w->live[k]) {
        w->src[k] ^= 1;
        w->todo[k] -= 1;
    }
}

template <int LAT, typename T, int S, typename U>
__global__ void __launch_bounds__(256, 3) kb_moments(const DevSim* sims, const BatchWork* w, int pair)
{
    const int n = w->nslot, total = w->mstart[n];
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int k = batch_slot(w->mstart, n, item);
        if (!w->live[k]) continue;
        const int b = item - w->mstart[k], gx = w->mgx[k], gy = w->mgy[k];
        b_moments<LAT, T, S, U>(sims[k], w->src[k], pair, Blk{b % gx, (b / gx) % gy, b / (gx * gy)});
        __syncthreads();
    }
}

// tile coordinates of tile b of slot k
__device__ __forceinline__ Blk batch_tile(const BatchWork* w, int k, int b)
{
    const int gx = w->tgx[k], gy = w->tgy[k];
    return Blk{b % gx, (b / gx) % gy, b / (gx * gy)};
}

template <int LAT, typename T, typename U>
__global__ void __launch_bounds__(Tile<Lat<LAT>::D>::THREADS) kb_force(const DevSim* sims, const BatchWork* w, int pair)
{
    const int n = w->nslot, total = w->tstart[n];
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int k = batch_slot(w->tstart, n, item);
        if (!w->live[k]) continue;
        b_force<LAT, T, U>(sims[k], pair, batch_tile(w, k, item - w->tstart[k]));
        __syncthreads();
    }
}

static __global__ void kb_us_begin(const DevSim* sims, const BatchWork* w, int pair)
{
    const int k = threadIdx.x >> 5;  // one warp per slot (the condition is uniform in the warp)
    if (k < w->nslot && w->live[k]) b_us_begin(sims[k], pair, threadIdx.x & 31);
}

template <int LAT, typename T, typename U>
__global__ void __launch_bounds__(Tile<Lat<LAT>::D>::THREADS, sizeof(U) == 4 ? 2 : 1)
    kb_sweep(const DevSim* sims, const BatchWork* w, int pair)
{
    const int n = w->nslot, total = w->tstart[n];
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int k = batch_slot(w->tstart, n, item);
        if (!w->live[k] || !sims[k].us[pair].running) continue;
        b_sweep<LAT, T, U, false>(sims[k], pair, batch_tile(w, k, item - w->tstart[k]));
        __syncthreads();
    }
}

// One warp: the control step of every slot whose solve is running; the loop goes on while any is.
static __global__ void kb_us_ctl(const DevSim* sims, const BatchWork* w, int pair, cudaGraphConditionalHandle h)
{
    const int k = threadIdx.x;
    bool still = false;
    if (k < w->nslot && w->live[k] && sims[k].us[pair].running) still = !b_us_ctl(sims[k], pair);
    const bool any = __any_sync(0xffffffffu, still);
    if (k == 0) cudaGraphSetConditional(h, any ? 1u : 0u);
}

template <int LAT, typename T, typename U>
__global__ void __launch_bounds__(Tile<Lat<LAT>::D>::THREADS, 2) kb_derivs(const DevSim* sims, const BatchWork* w)
{
    const int n = w->nslot, total = w->tstart[n];
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int k = batch_slot(w->tstart, n, item);
        if (!w->live[k]) continue;
        b_derivs<LAT, T, U>(sims[k], batch_tile(w, k, item - w->tstart[k]));
        __syncthreads();
    }
}

template <int LAT, typename T, int S, typename U, bool READ>
__global__ void __launch_bounds__(Tile<Lat<LAT>::D>::THREADS, 2) kb_collide(const DevSim* sims, const BatchWork* w)
{
    const int n = w->nslot, total = w->tstart[n];
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int k = batch_slot(w->tstart, n, item);
        if (!w->live[k]) continue;
        b_collide<LAT, T, S, U, READ>(sims[k], w->src[k], batch_tile(w, k, item - w->tstart[k]));
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Initial condition, field and population transfer, conservation sums
// ---------------------------------------------------------------------------
// w_k(c_s^2(rho)) in FP64 (initialisation only)
template <int LAT>
__device__ __forceinline__ double lat_weight_d(int k, const DevSim& p, double rho)
{
    double P, DP, PM, RPP;
    eos_full<double>(p, rho, P, DP, PM, RPP);
    return weight<LAT, double>(k, P / rho);
}

template <int LAT, typename T, int S>
__global__ void k_init_eq(DevSim p, const double* rho_in, const double* u_in, int dst)
{
    using L = Lat<LAT>;
    using C = Codec<S>;
    const long long s = gtid();
    if (s >= p.N) return;
    const T rs = T(rho_in[s]);
    T u[3] = {T(0), T(0), T(0)};
    if (u_in)
#pragma unroll
        for (int a = 0; a < L::D; ++a) u[a] = T(u_in[a * p.N + s]);
    const T drs = T(rho_in[s] - p.rho0);
    T cs2, dcs2;
    cs2_delta<T>(p, drs, cs2, dcs2);
    const T cs0 = phys<T>(p).cs0;
    const T ics2 = T(1) / cs2;
    T uu = T(0);
#pragma unroll
    for (int a = 0; a < L::D; ++a) uu += u[a] * u[a];
    // sum of the stored values: a float pair (error-free TwoSum, as in the collision) for the
    // 32-bit arithmetic, whose FP64 adds took most of the kernel's time on GB300; FP64 for the FP64
    // storage and the local-reference storages
    double stored_sum = 0.0;
    float sh = 0.f, sl = 0.f;
    const float* wf = C::LOC ? p.wref[dst] : nullptr;
    const int x = int(s % p.nx), y = int((s / p.nx) % p.ny), z = int(s / ((long long)p.nx * p.ny));
#pragma unroll
    for (int i = 1; i < L::Q; ++i) {
        const int k = L::shell(i);
        const T uc = T(L::cx(i)) * u[0] + T(L::cy(i)) * u[1] + T(L::cz(i)) * u[2];
        const T X = uc * ics2 + T(0.5) * uc * uc * ics2 * ics2 - T(0.5) * uu * ics2;
        const T w = weight<LAT, T>(k, cs2);
        if (C::LOC) {
            // as if sent by the neighbour at -c_i: n^eq here minus that site's reference, in FP64
            const float ref = wf[k * p.N + sender<LAT>(p, x, y, z, i)];
            const double wd = lat_weight_d<LAT>(k, p, rho_in[s]) * rho_in[s];
            const double dev = (wd - double(ref)) + wd * double(X);
            // the decoded float the moments kernel will sum
            stored_sum += double(__fadd_rn(float(pop_put<LAT, S, double>(p, dst, i, s, dev)), ref));
            continue;
        }
        const T dev = w * rs * X + w * drs +
                      phys<T>(p).rho0 * dcs2 *
                          (T(L::wc(k, 1)) + T(L::wc(k, 2)) * (cs2 + cs0) + T(L::wc(k, 3)) * (cs2 * cs2 + cs2 * cs0 + cs0 * cs0));
        const T sv = pop_put<LAT, S, T>(p, dst, i, s, C::DEV ? dev : w * rs * (T(1) + X));
        if constexpr (sizeof(T) == 4) acc2(sh, sl, float(sv));
        else stored_sum += double(sv);
    }
    if (sizeof(T) == 4 && !C::LOC) stored_sum = double(sh) + double(sl);
    // the rest population closes the sum to rho (as the collision does)
    if (C::LOC) stored_sum += double(wf[s]);  // the rest population's own reference
    const double rest = (C::DEV && !C::LOC ? rho_in[s] - p.rho0 : rho_in[s]) - stored_sum;
    pop_put<LAT, S, double>(p, dst, 0, s, rest);
}

// The references w_k(c_s^2(rho)) rho of every site for the initial populations (local-reference
// storages); k_init_eq then stores each population relative to its sender's.
template <int LAT, typename T>
__global__ void k_init_ref(DevSim p, const double* rho_in, int dst)
{
    using L = Lat<LAT>;
    const long long s = gtid();
    if (s >= p.N) return;
    const T drs = T(rho_in[s] - p.rho0);
    T cs2, dcs2;
    cs2_delta<T>(p, drs, cs2, dcs2);
    const T cs0 = phys<T>(p).cs0;
#pragma unroll
    for (int k = 0; k < L::NSHELL; ++k) {
        const T dw0 = weight<LAT, T>(k, cs2) * drs +
                      phys<T>(p).rho0 * dcs2 *
                          (T(L::wc(k, 1)) + T(L::wc(k, 2)) * (cs2 + cs0) + T(L::wc(k, 3)) * (cs2 * cs2 + cs2 * cs0 + cs0 * cs0));
        float corr;
        p.wref[dst][k * p.N + s] = local_ref(p.pf, k, float(dw0), corr);
    }
}

// rho = sum_i n_i of FP64 populations [Q][N] (references for imported populations)
template <int LAT>
__global__ void k_pops_rho(DevSim p, const double* in, double* rho)
{
    const long long s = gtid();
    if (s >= p.N) return;
    double r = 0.0;
#pragma unroll
    for (int i = 0; i < Lat<LAT>::Q; ++i) r += in[(long long)i * p.N + s];
    rho[s] = r;
}

// The value of population i at site s of buffer b in the FP64 export convention (n_i itself).
template <int LAT, int S>
__device__ __forceinline__ double pop_full(const DevSim& p, int b, int i, long long s)
{
    using L = Lat<LAT>;
    using C = Codec<S>;
    const double v = pop_raw<LAT, S, double>(p, b, i, s);
    if (C::LOC) {
        // the decoded value every density sum uses: fl(stored + sender's reference) for the
        // moving populations, the exact pair plus the own reference for the rest population
        if (i == 0) return v + double(p.wref[b][s]);
        const int x = int(s % p.nx), y = int((s / p.nx) % p.ny), z = int(s / ((long long)p.nx * p.ny));
        return double(__fadd_rn(float(v), p.wref[b][L::shell(i) * p.N + sender<LAT>(p, x, y, z, i)]));
    }
    return v + (C::DEV ? p.off[L::shell(i)] : 0.0);
}

template <int LAT, typename T, typename U>
__global__ void k_fields_out(DevSim p, int pair, double* rho_out, double* u_out)
{
    using L = Lat<LAT>;
    const long long s = gtid();
    if (s >= p.N) return;
    const T rs = phys<T>(p).rho0 + cp<T>(p.rho)[s];
    const U* uu = cp<U>(p.uit[pair][p.us[pair].cur]);
    if (rho_out) rho_out[s] = double(rs);
    if (u_out)
#pragma unroll
        for (int a = 0; a < L::D; ++a) u_out[a * p.N + s] = double(uu[a * p.N + s]);
}

template <int LAT, int S>
__global__ void k_pops_out(DevSim p, int src, double* out)
{
    using L = Lat<LAT>;
    using C = Codec<S>;
    const long long s = gtid();
    if (s >= p.N) return;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) out[(long long)i * p.N + s] = pop_full<LAT, S>(p, src, i, s);
}

template <int LAT, int S>
__global__ void k_pops_in(DevSim p, const double* in, int dst)
{
    using L = Lat<LAT>;
    using C = Codec<S>;
    const long long s = gtid();
    if (s >= p.N) return;
    const int x = int(s % p.nx), y = int((s / p.nx) % p.ny), z = int(s / ((long long)p.nx * p.ny));
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        // relative to the reference the decode of buffer dst will add
        const double ref = C::LOC ? double(p.wref[dst][L::shell(i) * p.N + (i == 0 ? s : sender<LAT>(p, x, y, z, i))])
                                  : (C::DEV ? p.off[L::shell(i)] : 0.0);
        pop_put<LAT, S, double>(p, dst, i, s, in[(long long)i * p.N + s] - ref);
    }
}

// FP64 sums of rho and sum_i n_i c_i: fixed grid, fixed tree, so the result is
// independent of scheduling.  Each block writes its 4 partial sums.
constexpr int RED_BLOCK = kRedBlock;
constexpr int RED_GRID = kRedGrid;

template <int LAT, int S>
__global__ void k_red_partial(DevSim p, int src, double* part)
{
    using L = Lat<LAT>;
    using C = Codec<S>;
    __shared__ double sm[4][RED_BLOCK];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long s = blockIdx.x * (long long)RED_BLOCK + threadIdx.x; s < p.N; s += (long long)RED_GRID * RED_BLOCK) {
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            const double v = pop_full<LAT, S>(p, src, i, s);
            acc[0] += v;
            acc[1] += L::cx(i) * v;
            acc[2] += L::cy(i) * v;
            acc[3] += L::cz(i) * v;
        }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) sm[c][threadIdx.x] = acc[c];
    __syncthreads();
    for (int w = RED_BLOCK / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
#pragma unroll
            for (int c = 0; c < 4; ++c) sm[c][threadIdx.x] += sm[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 4) part[blockIdx.x * 4 + threadIdx.x] = sm[threadIdx.x][0];
}

static __global__ void k_red_final(DevSim p, const double* part, int nparts, double* out)
{
    __shared__ double sm[4][RED_BLOCK];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int k = threadIdx.x; k < nparts; k += RED_BLOCK)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[c] += part[k * 4 + c];
#pragma unroll
    for (int c = 0; c < 4; ++c) sm[c][threadIdx.x] = acc[c];
    __syncthreads();
    for (int w = RED_BLOCK / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
#pragma unroll
            for (int c = 0; c < 4; ++c) sm[c][threadIdx.x] += sm[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 4) out[threadIdx.x] = sm[threadIdx.x][0];
}

// ---------------------------------------------------------------------------
// Kernel table of one combination
// ---------------------------------------------------------------------------
template <int LAT, typename T, int S, typename U>
KernelTable make_table(bool read_pops)
{
    KernelTable t{};
    t.moments = (const void*)k_moments<LAT, T, S, U>;
    t.force = (const void*)k_force<LAT, T, U>;
    t.us_begin = (const void*)k_us_begin;
    t.sweep = (const void*)k_sweep<LAT, T, U, false>;
    t.sweep_tma = Lat<LAT>::D == 3 ? (const void*)k_sweep<LAT, T, U, true> : nullptr;
    t.us_ctl = (const void*)k_us_ctl;
    t.derivs = (const void*)k_derivs<LAT, T, U>;
    t.collide = read_pops ? (const void*)k_collide<LAT, T, S, U, true> : (const void*)k_collide<LAT, T, S, U, false>;
    t.init_eq = (const void*)k_init_eq<LAT, T, S>;
    t.init_ref = Codec<S>::LOC ? (const void*)k_init_ref<LAT, T> : nullptr;
    t.pops_rho = (const void*)k_pops_rho<LAT>;
    t.local_ref = Codec<S>::LOC;
    t.fields_out = (const void*)k_fields_out<LAT, T, U>;
    t.pops_out = (const void*)k_pops_out<LAT, S>;
    t.pops_in = (const void*)k_pops_in<LAT, S>;
    t.red_partial = (const void*)k_red_partial<LAT, S>;
    t.red_final = (const void*)k_red_final;
    t.kb_step_begin = (const void*)kb_step_begin;
    t.kb_moments = (const void*)kb_moments<LAT, T, S, U>;
    t.kb_force = (const void*)kb_force<LAT, T, U>;
    t.kb_us_begin = (const void*)kb_us_begin;
    t.kb_sweep = (const void*)kb_sweep<LAT, T, U>;
    t.kb_us_ctl = (const void*)kb_us_ctl;
    t.kb_derivs = (const void*)kb_derivs<LAT, T, U>;
    t.kb_collide = read_pops ? (const void*)kb_collide<LAT, T, S, U, true> : (const void*)kb_collide<LAT, T, S, U, false>;
    t.kb_step_end = (const void*)kb_step_end;
    t.block = 256;
    using TL = Tile<Lat<LAT>::D>;
    t.tile[0] = TL::TX;
    t.tile[1] = TL::TY;
    t.tile_threads = TL::THREADS;
    constexpr int D = Lat<LAT>::D;
    t.smem_sweep = SweepPlan<D, T, U>::BYTES;
    t.sweep_box[0] = SweepPlan<D, T, U>::UX;
    t.sweep_box[1] = SweepPlan<D, T, U>::UY;
    t.smem_force = size_t(ForcePlan<D>::R) * ForcePlan<D>::RP * sizeof(T);
    t.smem_derivs = size_t(DerivsPlan<D, T>::R) * 6 * (TL::TX + 4) * (TL::TY + 4) * sizeof(T);
    t.smem_collide = size_t(CollidePlan<D>::R) * (1 + AuxLayout<D>::NB + D) * (TL::TX + 4) * (TL::TY + 4) * sizeof(T);
    cudaFuncSetAttribute(t.force, cudaFuncAttributeMaxDynamicSharedMemorySize, int(t.smem_force));
    cudaFuncSetAttribute(t.sweep, cudaFuncAttributeMaxDynamicSharedMemorySize, int(t.smem_sweep));
    if (t.sweep_tma) cudaFuncSetAttribute(t.sweep_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, int(t.smem_sweep));
    cudaFuncSetAttribute(t.derivs, cudaFuncAttributeMaxDynamicSharedMemorySize, int(t.smem_derivs));
    cudaFuncSetAttribute(t.collide, cudaFuncAttributeMaxDynamicSharedMemorySize, int(t.smem_collide));
    cudaFuncSetAttribute(t.kb_force, cudaFuncAttributeMaxDynamicSharedMemorySize, int(t.smem_force));
    cudaFuncSetAttribute(t.kb_sweep, cudaFuncAttributeMaxDynamicSharedMemorySize, int(t.smem_sweep));
    cudaFuncSetAttribute(t.kb_derivs, cudaFuncAttributeMaxDynamicSharedMemorySize, int(t.smem_derivs));
    cudaFuncSetAttribute(t.kb_collide, cudaFuncAttributeMaxDynamicSharedMemorySize, int(t.smem_collide));
    t.tsize = sizeof(T);
    t.usize = sizeof(U);
    t.ssize = sizeof(typename Codec<S>::type);
    t.rsize = Codec<S>::SPLIT0 ? sizeof(float2) : 0;
    t.exact = Codec<S>::EXACT;
    return t;
}

}  // namespace lbm
