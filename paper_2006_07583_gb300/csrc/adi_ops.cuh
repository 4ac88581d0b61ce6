// adi_ops.cuh -- operator coefficients and the per-line system of the Peaceman-Rachford
// stages, as the GPU path evaluates them.
//
// Line formulation (one x-line in stage 1, one y-line in stage 2).  A line has N cells, a
// pressure line p_0..p_L (p_0, p_L Dirichlet; CFD L = N on the nodes, MFD L = N+1 on
// edges + cell centres), interior pressure carried values a_k, velocities v_0..v_N on the
// nodes, alpha_k = dt/2 kappa_k and beta = dt/2 (density 1).  Stage 1 of Eq. 6 / Eq. 8
// asks for (u*, v*) with
//      u*_k + alpha_k (Dv v*)_k = a_k ,      v*_j + beta (Du u*)_j = v_j ,
// Dv = Pbar^{-1} Qbar (CFD, App. A) or D4 (MFD, App. B), Du = P^{-1} Q or G4 acting on the
// whole pressure line.  Stage 2 (Eq. 10) is the same system along y with (C, w*).
//
//  CFD: unknowns e = Dv v*, g = Du u* (2 per node).  Substituting u* = a - alpha e and
//       v* = v - beta g gives   Pbar e + Qbar (beta g) = Qbar v ,
//                               P g + Q_int (alpha e)  = Q [p_0, a, p_L] ,
//       block tridiagonal in x_j = (e_j, g_j) away from the two ends.
//  MFD: Schur form in u*:  (I - alpha D beta G_int) u* = a - alpha D (v - beta G_bnd p_bnd),
//       heptadiagonal, grouped into 3x3 blocks.
// The Peaceman-Rachford identities then give the next stage's carried values without any
// further derivative:  C = 2 u* - a (+ dt/2 f^{m+1}),  v^{m+1} = 2 v* - v.
//
// The first h_u and last t_u unknowns of each line (where App. A/B use their one-sided
// boundary rows) are eliminated once per line in FP64 into small tables; what remains is a
// uniform block tridiagonal system with block size BS (2 for CFD, 3 for MFD).
#pragma once
#include <cstdint>

namespace adi {

constexpr int kCFD = 0;
constexpr int kMFD = 1;

// ---------------------------------------------------------------------------------------
// App. A (compact FD, fourth order): coefficients of one row, times h for Q and Qbar.
// Columns are node indices 0..N.  Each returns the row length and its first column.
// ---------------------------------------------------------------------------------------
__host__ __device__ inline int cfd_P_row(int N, int r, int *c0, double *w) {
    if (r == 0) { *c0 = 0; w[0] = 6.0; w[1] = 18.0; return 2; }
    if (r == N) { *c0 = N - 1; w[0] = 18.0; w[1] = 6.0; return 2; }
    *c0 = r - 1; w[0] = 1.0; w[1] = 4.0; w[2] = 1.0; return 3;
}
__host__ __device__ inline int cfd_Q_row(int N, int r, int *c0, double *w) {
    if (r == 0) { *c0 = 0; w[0] = -17.0; w[1] = 9.0; w[2] = 9.0; w[3] = -1.0; return 4; }
    if (r == N) { *c0 = N - 3; w[0] = 1.0; w[1] = -9.0; w[2] = -9.0; w[3] = 17.0; return 4; }
    *c0 = r - 1; w[0] = -3.0; w[1] = 0.0; w[2] = 3.0; return 3;
}
// Reduced operators: row for interior node j (1..N-1); Pbar columns are node indices.
__host__ __device__ inline int cfd_Pbar_row(int N, int j, int *c0, double *w) {
    if (j == 1) { *c0 = 1; w[0] = 6.0; w[1] = 6.0; return 2; }
    if (j == N - 1) { *c0 = N - 2; w[0] = 6.0; w[1] = 6.0; return 2; }
    *c0 = j - 1; w[0] = 1.0; w[1] = 4.0; w[2] = 1.0; return 3;
}
__host__ __device__ inline int cfd_Qbar_row(int N, int j, int *c0, double *w) {
    if (j == 1) { *c0 = 0; w[0] = -1.0; w[1] = -9.0; w[2] = 9.0; w[3] = 1.0; return 4; }
    if (j == N - 1) { *c0 = N - 3; w[0] = -1.0; w[1] = -9.0; w[2] = 9.0; w[3] = 1.0; return 4; }
    *c0 = j - 1; w[0] = -3.0; w[1] = 0.0; w[2] = 3.0; return 3;
}

// ---------------------------------------------------------------------------------------
// App. B (mimetic, fourth order, alpha = beta = 0, gamma = 1/24): rows times h.
// D4 is N x (N+1) (cell r+1 <- nodes), G4 is (N+1) x (N+2) (node j <- edges+centres).
// The last rows mirror the printed first rows with a sign change.
// ---------------------------------------------------------------------------------------
__host__ __device__ inline double mim_D0(int c) {
    switch (c) {
    case 0: return -4751.0 / 5192.0;
    case 1: return 909.0 / 1298.0;
    case 2: return 6091.0 / 15576.0;
    case 3: return -1165.0 / 5192.0;
    case 4: return 129.0 / 2596.0;
    default: return -25.0 / 15576.0;
    }
}
__host__ __device__ inline double mim_G0(int c) {
    switch (c) {
    case 0: return -47888.0 / 14245.0;
    case 1: return 1790.0 / 407.0;
    case 2: return -14545.0 / 9768.0;
    case 3: return 8997.0 / 16280.0;
    case 4: return -2335.0 / 22792.0;
    default: return 25.0 / 9768.0;
    }
}
__host__ __device__ inline double mim_G1(int c) {
    switch (c) {
    case 0: return 16.0 / 105.0;
    case 1: return -31.0 / 24.0;
    case 2: return 29.0 / 24.0;
    case 3: return -3.0 / 40.0;
    default: return 1.0 / 168.0;
    }
}
// Interior fourth-order staggered stencil (1/24, -9/8, 9/8, -1/24).
__host__ __device__ inline double mim_w(int c) {
    return c == 0 ? 1.0 / 24.0 : c == 1 ? -9.0 / 8.0 : c == 2 ? 9.0 / 8.0 : -1.0 / 24.0;
}
__host__ __device__ inline int mfd_D_row(int N, int r, int *c0, double *w) {
    if (r == 0) { *c0 = 0; for (int c = 0; c < 6; ++c) w[c] = mim_D0(c); return 6; }
    if (r == N - 1) { *c0 = N - 5; for (int c = 0; c < 6; ++c) w[c] = -mim_D0(5 - c); return 6; }
    *c0 = r - 1; for (int c = 0; c < 4; ++c) w[c] = mim_w(c); return 4;
}
__host__ __device__ inline int mfd_G_row(int N, int j, int *c0, double *w) {
    if (j == 0) { *c0 = 0; for (int c = 0; c < 6; ++c) w[c] = mim_G0(c); return 6; }
    if (j == 1) { *c0 = 0; for (int c = 0; c < 5; ++c) w[c] = mim_G1(c); return 5; }
    if (j == N) { *c0 = N - 4; for (int c = 0; c < 6; ++c) w[c] = -mim_G0(5 - c); return 6; }
    if (j == N - 1) { *c0 = N - 3; for (int c = 0; c < 5; ++c) w[c] = -mim_G1(4 - c); return 5; }
    *c0 = j - 1; for (int c = 0; c < 4; ++c) w[c] = mim_w(c); return 4;
}

// Self-convolution of the interior stencil: interior rows of D4 G4 (times h^2) have the
// seven coefficients c_s = sum_{i+l=s} w_i w_l, s = 0..6, on cells c-3..c+3.
__host__ __device__ inline double mim_DG(int s) {
    double acc = 0.0;
    for (int i = 0; i < 4; ++i) {
        int l = s - i;
        if (l >= 0 && l < 4) acc += mim_w(i) * mim_w(l);
    }
    return acc;
}

// ---------------------------------------------------------------------------------------
// Line partition: head (h_u unknowns), nb middle blocks of BS, tail (t_u unknowns).
// ---------------------------------------------------------------------------------------
struct LineShape {
    int bs, hu, tu, nb, nunk;
};

__host__ __device__ inline LineShape line_shape(int method, int N) {
    LineShape s;
    if (method == kCFD) {
        s.bs = 2; s.hu = 5; s.tu = 5; s.nunk = 2 * N;
        s.nb = N - 5;  // nodes 3 .. N-3
    } else {
        s.bs = 3; s.nunk = N;
        int q = (N - 8) % 3;
        s.hu = q == 0 ? 4 : 5;
        s.tu = q == 2 ? 5 : 4;
        s.nb = (N - s.hu - s.tu) / 3;
    }
    return s;
}

// Per line end table (values in the path's precision, built in FP64):
//   Hinv  [hu x hu] at 0,  HinvE [hu x bs] at 36,  K [bs x hu] at 54,  dB [bs x bs] at 72.
constexpr int kTabHinv = 0;
constexpr int kTabHinvE = 36;
constexpr int kTabK = 54;
constexpr int kTabDB = 72;
constexpr int kTabEnd = 96;   // one line end
constexpr int kTabLine = 192; // head then tail

}  // namespace adi
