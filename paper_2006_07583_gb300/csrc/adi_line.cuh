// adi_line.cuh -- device helpers shared by the line kernels: small block algebra, the
// Ricker source, line accessors, right-hand sides of the boundary rows and the generator of
// the uniform middle blocks of a line system (see adi_ops.cuh for the formulation).
#pragma once
#include <cuda_runtime.h>

#include "adi_internal.h"
#include "adi_ops.cuh"

namespace adi {

__device__ __forceinline__ int cfd_idx_g(int N, int j) { return j == 0 ? 0 : (j == N ? 2 * N - 1 : 2 * j); }
__device__ __forceinline__ int cfd_idx_e(int j) { return 2 * j - 1; }

// ---------------------------------------------------------------------------------------
// Small dense helpers.
// ---------------------------------------------------------------------------------------
// Reciprocal: IEEE round-to-nearest in both precisions (the FP32 intrinsic avoids the
// general division sequence).
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

template <typename T, int BS>
__device__ __forceinline__ void mat_inv(const T (&S)[BS][BS], T (&R)[BS][BS]) {
    if constexpr (BS == 2) {
        T det = S[0][0] * S[1][1] - S[0][1] * S[1][0];
        T id = recip(det);
        R[0][0] = S[1][1] * id; R[0][1] = -S[0][1] * id;
        R[1][0] = -S[1][0] * id; R[1][1] = S[0][0] * id;
    } else {
        T c00 = S[1][1] * S[2][2] - S[1][2] * S[2][1];
        T c01 = S[1][2] * S[2][0] - S[1][0] * S[2][2];
        T c02 = S[1][0] * S[2][1] - S[1][1] * S[2][0];
        T det = S[0][0] * c00 + S[0][1] * c01 + S[0][2] * c02;
        T id = recip(det);
        R[0][0] = c00 * id;
        R[0][1] = (S[0][2] * S[2][1] - S[0][1] * S[2][2]) * id;
        R[0][2] = (S[0][1] * S[1][2] - S[0][2] * S[1][1]) * id;
        R[1][0] = c01 * id;
        R[1][1] = (S[0][0] * S[2][2] - S[0][2] * S[2][0]) * id;
        R[1][2] = (S[0][2] * S[1][0] - S[0][0] * S[1][2]) * id;
        R[2][0] = c02 * id;
        R[2][1] = (S[0][1] * S[2][0] - S[0][0] * S[2][1]) * id;
        R[2][2] = (S[0][0] * S[1][1] - S[0][1] * S[1][0]) * id;
    }
}

// Ricker wavelet at time t.
__device__ __forceinline__ double ricker(double amp, double f0, double tdelay, double t) {
    const double pi = 3.14159265358979323846;
    double tau = t - tdelay;
    double q = pi * pi * f0 * f0 * tau * tau;
    return amp * (1.0 - 2.0 * q) * exp(-q);
}

// ---------------------------------------------------------------------------------------
// Line accessors.
// ---------------------------------------------------------------------------------------
template <typename T>
struct Line {
    const LineDesc<T> &d;
    const T *P, *V, *Al;  // pressure, velocity and alpha lines (global or shared memory)
    long long sp, sv;
    __device__ Line(const LineDesc<T> &dd)
        : d(dd), P(dd.p), V(dd.v), Al(dd.alpha), sp(dd.sp), sv(dd.sv) {}
    // the same line staged in shared memory (unit strides)
    __device__ Line(const LineDesc<T> &dd, const T *p, const T *v, const T *al)
        : d(dd), P(p), V(v), Al(al), sp(1), sv(1) {}
    __device__ __forceinline__ T p(int k) const { return P[k * sp]; }
    __device__ __forceinline__ T v(int k) const { return V[k * sv]; }
    __device__ __forceinline__ T al(int k) const { return Al[k * sp]; }
};

// Pressure-line length minus one (index of the far Dirichlet value).
__host__ __device__ __forceinline__ int p_last(int method, int N) {
    return method == kCFD ? N : N + 1;
}

// ---------------------------------------------------------------------------------------
// Right-hand sides of the head/tail rows (solver index i), in the path's precision.
// ---------------------------------------------------------------------------------------
template <typename T>
__device__ T rhs_row(const Line<T> &L, int i) {
    const LineDesc<T> &d = L.d;
    const int N = d.N;
    const T ih = (T)d.inv_h;
    double w[8];
    int c0, n;
    T acc = T(0);
    if (d.method == kCFD) {
        bool is_g = (i == 0) || (i == 2 * N - 1) || (i % 2 == 0);
        int node = i == 0 ? 0 : (i == 2 * N - 1 ? N : (i + 1) / 2);
        if (is_g) {
            n = cfd_Q_row(N, node, &c0, w);
            for (int t = 0; t < n; ++t) acc += (T)w[t] * L.p(c0 + t);
        } else {
            n = cfd_Qbar_row(N, node, &c0, w);
            for (int t = 0; t < n; ++t) acc += (T)w[t] * L.v(c0 + t);
        }
        return acc * ih;
    }
    // MFD: r_c = a_c - alpha_c/h * sum_j D[c-1][j] (v_j - beta/h (G[j][0] p_0 + G[j][N+1] p_L))
    const int c = i + 1;
    const T p0 = L.p(0), pl = L.p(N + 1), bh = (T)(d.beta * d.inv_h);
    n = mfd_D_row(N, c - 1, &c0, w);
    for (int t = 0; t < n; ++t) {
        int node = c0 + t;
        T vt = L.v(node);
        if (node <= 1 || node >= N - 1) {
            double gw[8];
            int g0;
            int ng = mfd_G_row(N, node, &g0, gw);
            T gb = T(0);
            if (g0 == 0) gb += (T)gw[0] * p0;
            if (g0 + ng - 1 == N + 1) gb += (T)gw[ng - 1] * pl;
            vt -= bh * gb;
        }
        acc += (T)w[t] * vt;
    }
    return L.p(c) - L.al(c) * ih * acc;
}

// Middle block b: A (coupling to block b-1), B, C (coupling to block b+1), r.
template <typename T, typename TS, int BS>
__device__ __forceinline__ void middle_block(const Line<TS> &L, const LineShape &s, int b,
                                             T (&A)[BS][BS], T (&B)[BS][BS], T (&C)[BS][BS],
                                             T (&r)[BS]) {
    const LineDesc<TS> &d = L.d;
    const T ih = (T)d.inv_h;
    if constexpr (BS == 2) {
        const int j = 3 + b;  // node
        const T tb = T(3) * (T)d.beta * ih;
        A[0][0] = T(1); A[0][1] = -tb; A[1][0] = -T(3) * ih * (T)L.al(j - 1); A[1][1] = T(1);
        B[0][0] = T(4); B[0][1] = T(0); B[1][0] = T(0); B[1][1] = T(4);
        C[0][0] = T(1); C[0][1] = tb; C[1][0] = T(3) * ih * (T)L.al(j + 1); C[1][1] = T(1);
        r[0] = T(3) * ih * ((T)L.v(j + 1) - (T)L.v(j - 1));
        r[1] = T(3) * ih * ((T)L.p(j + 1) - (T)L.p(j - 1));
    } else {
        const int cb = s.hu + 1 + 3 * b;  // first cell of the block
        const T w0 = (T)mim_w(0), w1 = (T)mim_w(1), w2 = (T)mim_w(2), w3 = (T)mim_w(3);
        const T bh2 = (T)(d.beta * d.inv_h * d.inv_h);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int c = cb + k;
            const T a = (T)L.al(c);
            const T sc = a * bh2;
#pragma unroll
            for (int l = 0; l < 3; ++l) {
                int dA = l - k - 3, dB = l - k, dC = l - k + 3;
                A[k][l] = (dA >= -3) ? -sc * (T)mim_DG(dA + 3) : T(0);
                B[k][l] = (dB == 0 ? T(1) : T(0)) - sc * (T)mim_DG(dB + 3);
                C[k][l] = (dC <= 3) ? -sc * (T)mim_DG(dC + 3) : T(0);
            }
            T dv = w0 * (T)L.v(c - 2) + w1 * (T)L.v(c - 1) + w2 * (T)L.v(c) + w3 * (T)L.v(c + 1);
            r[k] = (T)L.p(c) - a * ih * dv;
        }
    }
}


// Middle block b with the head/tail eliminations folded in (block 0 and block nb-1) and the
// couplings outside the middle system removed.  rH/rT are the head/tail right-hand sides.
template <typename T, typename TS, int BS>
__device__ __forceinline__ void load_block(const Line<TS> &L, const LineShape &s, int b,
                                           const T *rH, const T *rT, T (&A)[BS][BS],
                                           T (&B)[BS][BS], T (&C)[BS][BS], T (&r)[BS]) {
    middle_block<T, TS, BS>(L, s, b, A, B, C, r);
    const TS *th = L.d.tab, *tt = L.d.tab + kTabEnd;
    if (b == 0) {
#pragma unroll
        for (int i = 0; i < BS; ++i) {
#pragma unroll
            for (int j = 0; j < BS; ++j) { B[i][j] -= (T)th[kTabDB + i * BS + j]; A[i][j] = T(0); }
            T acc = T(0);
            for (int k = 0; k < s.hu; ++k) acc += (T)th[kTabK + i * s.hu + k] * rH[k];
            r[i] -= acc;
        }
    }
    if (b == s.nb - 1) {
#pragma unroll
        for (int i = 0; i < BS; ++i) {
#pragma unroll
            for (int j = 0; j < BS; ++j) { B[i][j] -= (T)tt[kTabDB + i * BS + j]; C[i][j] = T(0); }
            T acc = T(0);
            for (int k = 0; k < s.tu; ++k) acc += (T)tt[kTabK + i * s.tu + k] * rT[k];
            r[i] -= acc;
        }
    }
}

// ---------------------------------------------------------------------------------------
// Full line system in solver ordering, FP64, for the boundary elimination.
//   CFD ordering: g_0, e_1, g_1, ..., e_{N-1}, g_{N-1}, g_N  (e_j at 2j-1, g_j at 2j)
//   MFD ordering: u_1 .. u_N (cell c at c-1)
// ---------------------------------------------------------------------------------------
template <typename T>
__device__ inline double line_entry(const LineDesc<T> &d, int row, int col) {
    const int N = d.N;
    const double ih = d.inv_h, beta = d.beta;
    double w[8];
    int c0, n;
    double acc = 0.0;
    if (d.method == kCFD) {
        bool is_g = (row == 0) || (row == 2 * N - 1) || (row % 2 == 0);
        int node = row == 0 ? 0 : (row == 2 * N - 1 ? N : (row + 1) / 2);
        if (is_g) {
            n = cfd_P_row(N, node, &c0, w);
            for (int t = 0; t < n; ++t)
                if (cfd_idx_g(N, c0 + t) == col) acc += w[t];
            n = cfd_Q_row(N, node, &c0, w);
            for (int t = 0; t < n; ++t) {
                int k = c0 + t;
                if (k >= 1 && k <= N - 1 && cfd_idx_e(k) == col)
                    acc += w[t] * ih * (double)d.alpha[k * d.sp];
            }
        } else {
            n = cfd_Pbar_row(N, node, &c0, w);
            for (int t = 0; t < n; ++t)
                if (cfd_idx_e(c0 + t) == col) acc += w[t];
            n = cfd_Qbar_row(N, node, &c0, w);
            for (int t = 0; t < n; ++t)
                if (cfd_idx_g(N, c0 + t) == col) acc += w[t] * ih * beta;
        }
        return acc;
    }
    // MFD Schur row for cell c = row + 1, column cell c' = col + 1.
    const int c = row + 1, cc = col + 1;
    double dw[8], gw[8];
    int d0, g0;
    int nd = mfd_D_row(N, c - 1, &d0, dw);
    double s = 0.0;
    for (int t = 0; t < nd; ++t) {
        int node = d0 + t;
        int ng = mfd_G_row(N, node, &g0, gw);
        int k = cc - g0;
        if (k >= 0 && k < ng) s += dw[t] * gw[k];
    }
    acc = (row == col ? 1.0 : 0.0) - (double)d.alpha[c * d.sp] * beta * ih * ih * s;
    return acc;
}

// Gauss-Jordan inverse with partial pivoting of an n x n matrix (A is destroyed).
__device__ inline bool small_inverse(double *A, int n, double *R) {
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) R[i * n + j] = (i == j) ? 1.0 : 0.0;
    double scale = 0.0;
    for (int i = 0; i < n * n; ++i) scale = fmax(scale, fabs(A[i]));
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int i = c + 1; i < n; ++i)
            if (fabs(A[i * n + c]) > fabs(A[p * n + c])) p = i;
        if (!(fabs(A[p * n + c]) > 1e-13 * scale)) return false;
        if (p != c)
            for (int j = 0; j < n; ++j) {
                double t = A[c * n + j]; A[c * n + j] = A[p * n + j]; A[p * n + j] = t;
                t = R[c * n + j]; R[c * n + j] = R[p * n + j]; R[p * n + j] = t;
            }
        double ip = 1.0 / A[c * n + c];
        for (int j = 0; j < n; ++j) { A[c * n + j] *= ip; R[c * n + j] *= ip; }
        for (int i = 0; i < n; ++i) {
            if (i == c) continue;
            double f = A[i * n + c];
            if (f == 0.0) continue;
            for (int j = 0; j < n; ++j) { A[i * n + j] -= f * A[c * n + j]; R[i * n + j] -= f * R[c * n + j]; }
        }
    }
    return true;
}

}  // namespace adi
