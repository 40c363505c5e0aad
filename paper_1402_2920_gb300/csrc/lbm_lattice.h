// Velocity sets and weight polynomials of the two lattices, usable in host
// and device code (compile-time tables, so unrolled loops fold them).
#pragma once

namespace lbm {

// ---------------------------------------------------------------------------
// Lattices: Table II (D2Q21) and Table I (D3Q59).  Velocities are ordered by
// shell; inside a shell every vector is followed by its opposite.  Weights are
// w_k(s) = c0 + c1 s + c2 s^2 + c3 s^3 in s = c_s^2, expanded from the tables
// (the D3Q59 rest weight is the one that makes sum_i w_i = 1).
// ---------------------------------------------------------------------------
template <int LAT>
struct Lat;

template <>
struct Lat<0> {
    static constexpr int D = 2, Q = 21, NSHELL = 6;
    static constexpr int NAUX = 13;  // A, B(3), C(2), SigL(3), Xi(4)
    __host__ __device__ static constexpr int cx(int i)
    {
        constexpr int t[21] = {0, 1, -1, 0, 0, 1, -1, 1, -1, 2, -2, 0, 0, 2, -2, 2, -2, 4, -4, 0, 0};
        return t[i];
    }
    __host__ __device__ static constexpr int cy(int i)
    {
        constexpr int t[21] = {0, 0, 0, 1, -1, 1, -1, -1, 1, 0, 0, 2, -2, 2, -2, -2, 2, 0, 0, 4, -4};
        return t[i];
    }
    __host__ __device__ static constexpr int cz(int) { return 0; }
    __host__ __device__ static constexpr int shell(int i)
    {
        constexpr int t[21] = {0, 1, 1, 1, 1, 2, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4, 5, 5, 5, 5};
        return t[i];
    }
    __host__ __device__ static constexpr double wc(int k, int p)
    {
        constexpr double t[6][4] = {{1.0, -21.0 / 8.0, 105.0 / 32.0, -45.0 / 32.0},
                                    {0.0, 32.0 / 45.0, -4.0 / 3.0, 2.0 / 3.0},
                                    {0.0, 0.0, 1.0 / 3.0, -1.0 / 4.0},
                                    {0.0, -1.0 / 18.0, 3.0 / 16.0, -1.0 / 12.0},
                                    {0.0, 0.0, -1.0 / 192.0, 1.0 / 64.0},
                                    {0.0, 1.0 / 1440.0, -1.0 / 384.0, 1.0 / 384.0}};
        return t[k][p];
    }
    // Table III, column d_a d_b d_b (2D): shells (10), (11), (20)
    static constexpr double T3_AX = -2.0, T3_DIAG = 0.5, T3_TWO = 0.25;
};

template <>
struct Lat<1> {
    static constexpr int D = 3, Q = 59, NSHELL = 8;
    static constexpr int NAUX = 26;  // A, B(6), C(3), SigL(6), Xi(10)
    __host__ __device__ static constexpr int cx(int i)
    {
        constexpr int t[59] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0, 1,
                               -1, 1, -1, 1, -1, 1, -1, 2, -2, 0, 0, 0, 0, 2, -2, 2, -2, 2, -2, 2,
                               -2, 0, 0, 0, 0, 2, -2, 2, -2, 2, -2, 2, -2, 4, -4, 0, 0, 0, 0};
        return t[i];
    }
    __host__ __device__ static constexpr int cy(int i)
    {
        constexpr int t[59] = {0, 0, 0, 1, -1, 0, 0, 1, -1, 0, 0, 0, 0, -1, 1, 1, -1, 1, -1, 1,
                               -1, 1, -1, -1, 1, -1, 1, 0, 0, 2, -2, 0, 0, 2, -2, 0, 0, 0, 0, -2,
                               2, 2, -2, 2, -2, 2, -2, 2, -2, -2, 2, -2, 2, 0, 0, 4, -4, 0, 0};
        return t[i];
    }
    __host__ __device__ static constexpr int cz(int i)
    {
        constexpr int t[59] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 1, -1, -1, 1, 1,
                               -1, -1, 1, 1, -1, -1, 1, 0, 0, 0, 0, 2, -2, 0, 0, 2, -2, -2, 2, 0,
                               0, 2, -2, -2, 2, 2, -2, -2, 2, 2, -2, -2, 2, 0, 0, 0, 0, 4, -4};
        return t[i];
    }
    __host__ __device__ static constexpr int shell(int i)
    {
        constexpr int t[59] = {0, 1, 1, 1, 1, 1, 1, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 3,
                               3, 3, 3, 3, 3, 3, 3, 4, 4, 4, 4, 4, 4, 5, 5, 5, 5, 5, 5, 5,
                               5, 5, 5, 5, 5, 6, 6, 6, 6, 6, 6, 6, 6, 7, 7, 7, 7, 7, 7};
        return t[i];
    }
    __host__ __device__ static constexpr double wc(int k, int p)
    {
        constexpr double t[8][4] = {{1.0, -259.0 / 80.0, 273.0 / 64.0, -121.0 / 64.0},
                                    {0.0, 16.0 / 45.0, -2.0 / 3.0, 1.0 / 3.0},
                                    {0.0, 8.0 / 45.0, -1.0 / 3.0, 1.0 / 6.0},
                                    {0.0, -4.0 / 45.0, 1.0 / 3.0, -5.0 / 24.0},
                                    {0.0, -1.0 / 20.0, 17.0 / 96.0, -3.0 / 32.0},
                                    {0.0, -1.0 / 360.0, 1.0 / 192.0, 1.0 / 192.0},
                                    {0.0, 1.0 / 720.0, -1.0 / 192.0, 1.0 / 192.0},
                                    {0.0, 1.0 / 1440.0, -1.0 / 384.0, 1.0 / 384.0}};
        return t[k][p];
    }
    // Table III, column d_a d_b d_b (3D): shells (100), (110), (200)
    static constexpr double T3_AX = -3.0, T3_DIAG = 0.5, T3_TWO = 0.25;
};

}  // namespace lbm
