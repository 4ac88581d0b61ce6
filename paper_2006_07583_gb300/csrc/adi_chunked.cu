// adi_chunked.cu -- the partitioned (chunked) line solver: one CTA owns a group of whole
// lines of one simulation, every thread owns a chunk of up to M middle blocks of one line.
//
// A line's middle blocks (block tridiagonal, see adi_ops.cuh) are split into T chunks
// separated by single separator blocks:
//     [chunk 0][s_1][chunk 1][s_2] ... [s_{T-1}][chunk T-1]
// Eliminating every chunk interior leaves a block tridiagonal system on the separators.
// Its matrix depends only on alpha, so its block LU (Sinv_k, F_k, Gamma_k) is built once
// per line in FP64 (precompute_sep_kernel).  Per half step:
//   phase A  every chunk runs a forward and a backward block sweep over its blocks (no
//            storage) and hands the particular solution's end values to its separators;
//   phase B  one thread per line runs the separator substitution (forward and backward);
//   phase C  every chunk solves its interior with both neighbouring separators known,
//            keeping the forward factors in registers (checkpoints every SUB blocks,
//            segments recomputed backwards), and writes the carried outputs
//            C = 2 u* - a (+ dt/2 f) and v' = 2 v* - v.
// Phase C's re-reads of the chunk inputs hit L1/L2: the CTA touched them in phase A.
#include <cuda_runtime.h>

#include "adi_internal.h"
#include "adi_line.cuh"
#include "adi_ops.cuh"

namespace adi {

// ---------------------------------------------------------------------------------------
// Chunk geometry: T chunks of lengths base or base+1 (the first rem chunks), each followed
// by one separator block except the last.
// ---------------------------------------------------------------------------------------
struct ChunkGeom {
    int T, base, rem;
};
__host__ __device__ inline ChunkGeom chunk_geom(int nb, int M) {
    ChunkGeom g;
    g.T = (nb + 1 + M) / (M + 1);  // ceil((nb + 1) / (M + 1))
    if (g.T < 1) g.T = 1;
    int inner = nb - (g.T - 1);
    g.base = inner / g.T;
    g.rem = inner % g.T;
    return g;
}
__host__ __device__ inline int chunk_start(const ChunkGeom &g, int c) {
    return c * (g.base + 1) + (c < g.rem ? c : g.rem);
}
__host__ __device__ inline int chunk_len(const ChunkGeom &g, int c) {
    return g.base + (c < g.rem ? 1 : 0);
}

int chunk_count(int method, int N, int M) {
    LineShape s = line_shape(method, N);
    return chunk_geom(s.nb, M).T;
}

// ---------------------------------------------------------------------------------------
// Block algebra helpers (register arrays, compile-time sizes).
// ---------------------------------------------------------------------------------------
template <typename T, int BS>
__device__ __forceinline__ void mm(const T (&X)[BS][BS], const T (&Y)[BS][BS], T (&R)[BS][BS]) {
#pragma unroll
    for (int i = 0; i < BS; ++i)
#pragma unroll
        for (int j = 0; j < BS; ++j) {
            T acc = T(0);
#pragma unroll
            for (int k = 0; k < BS; ++k) acc += X[i][k] * Y[k][j];
            R[i][j] = acc;
        }
}
template <typename T, int BS>
__device__ __forceinline__ void mv(const T (&X)[BS][BS], const T (&y)[BS], T (&r)[BS]) {
#pragma unroll
    for (int i = 0; i < BS; ++i) {
        T acc = T(0);
#pragma unroll
        for (int k = 0; k < BS; ++k) acc += X[i][k] * y[k];
        r[i] = acc;
    }
}

// One elimination step: S = B - A G ; G' = S^{-1} C ; y' = S^{-1} (r - A y).
template <typename T, int BS>
__device__ __forceinline__ void thomas_step(const T (&A)[BS][BS], const T (&B)[BS][BS],
                                            const T (&C)[BS][BS], const T (&r)[BS],
                                            T (&G)[BS][BS], T (&y)[BS]) {
    T S[BS][BS], Si[BS][BS], rr[BS];
#pragma unroll
    for (int i = 0; i < BS; ++i) {
#pragma unroll
        for (int j = 0; j < BS; ++j) {
            T acc = B[i][j];
#pragma unroll
            for (int k = 0; k < BS; ++k) acc -= A[i][k] * G[k][j];
            S[i][j] = acc;
        }
        T acc = r[i];
#pragma unroll
        for (int k = 0; k < BS; ++k) acc -= A[i][k] * y[k];
        rr[i] = acc;
    }
    mat_inv<T, BS>(S, Si);
    mm<T, BS>(Si, C, G);
    mv<T, BS>(Si, rr, y);
}

// ---------------------------------------------------------------------------------------
// FP64 precompute of the separator system, one thread per line.
// sep layout per line: for k = 1..T-1, record k-1 holds Sinv (BS^2), F (BS^2), Gamma (BS^2).
// ---------------------------------------------------------------------------------------
template <typename TS, int BS>
__device__ void sep_precompute_line(const LineDesc<TS> &d, int M, TS *sep) {
    const Line<TS> L(d);
    const LineShape s = line_shape(d.method, d.N);
    const ChunkGeom g = chunk_geom(s.nb, M);
    const double rz[6] = {0, 0, 0, 0, 0, 0};
    // state carried across separators
    double Zn[BS][BS], Gn[BS][BS];      // left chunk's forward spike / Gamma at its last block
    double Gh[BS][BS];                  // Gamma-hat of the previous separator
    double Zprev_valid = 0.0;
    for (int i = 0; i < BS; ++i)
        for (int j = 0; j < BS; ++j) { Zn[i][j] = 0; Gn[i][j] = 0; Gh[i][j] = 0; }
    for (int c = 0; c < g.T; ++c) {
        const int b0 = chunk_start(g, c), n = chunk_len(g, c);
        // backward sweep of chunk c (for the separator on its left, k = c)
        double Zb[BS][BS], Gb[BS][BS];
        {
            double G[BS][BS], Z[BS][BS];
            for (int i = n - 1; i >= 0; --i) {
                double A[BS][BS], B[BS][BS], C[BS][BS], r[BS];
                load_block<double, TS, BS>(L, s, b0 + i, rz, rz, A, B, C, r);
                if (i == n - 1)
                    for (int p = 0; p < BS; ++p)
                        for (int q = 0; q < BS; ++q) C[p][q] = 0.0;  // coupling to x_R removed
                double S[BS][BS], Si[BS][BS];
                for (int p = 0; p < BS; ++p)
                    for (int q = 0; q < BS; ++q) {
                        double acc = B[p][q];
                        if (i < n - 1)
                            for (int k = 0; k < BS; ++k) acc -= C[p][k] * G[k][q];
                        S[p][q] = acc;
                    }
                mat_inv<double, BS>(S, Si);
                double Gn2[BS][BS], Zn2[BS][BS];
                mm<double, BS>(Si, A, Gn2);
                if (i == n - 1) {
                    // spike w.r.t. x_R uses the original C of block n-1
                    double A2[BS][BS], B2[BS][BS], C2[BS][BS], r2[BS];
                    load_block<double, TS, BS>(L, s, b0 + i, rz, rz, A2, B2, C2, r2);
                    mm<double, BS>(Si, C2, Zn2);
                    for (int p = 0; p < BS; ++p)
                        for (int q = 0; q < BS; ++q) Zn2[p][q] = -Zn2[p][q];
                } else {
                    double T1[BS][BS];
                    mm<double, BS>(C, Z, T1);
                    mm<double, BS>(Si, T1, Zn2);
                    for (int p = 0; p < BS; ++p)
                        for (int q = 0; q < BS; ++q) Zn2[p][q] = -Zn2[p][q];
                }
                for (int p = 0; p < BS; ++p)
                    for (int q = 0; q < BS; ++q) { G[p][q] = Gn2[p][q]; Z[p][q] = Zn2[p][q]; }
            }
            for (int p = 0; p < BS; ++p)
                for (int q = 0; q < BS; ++q) { Zb[p][q] = Z[p][q]; Gb[p][q] = G[p][q]; }
        }
        if (c > 0) {
            // separator k = c between chunk c-1 (left) and chunk c (right)
            const int sb = b0 - 1;
            double As[BS][BS], Bs[BS][BS], Cs[BS][BS], rs[BS];
            load_block<double, TS, BS>(L, s, sb, rz, rz, As, Bs, Cs, rs);
            double Ahat[BS][BS], Bhat[BS][BS], Chat[BS][BS], T1[BS][BS], T2[BS][BS];
            mm<double, BS>(As, Zn, Ahat);          // coupling to separator k-1
            for (int p = 0; p < BS; ++p)
                for (int q = 0; q < BS; ++q) Ahat[p][q] *= Zprev_valid;
            mm<double, BS>(As, Gn, T1);
            mm<double, BS>(Cs, Gb, T2);
            for (int p = 0; p < BS; ++p)
                for (int q = 0; q < BS; ++q) Bhat[p][q] = Bs[p][q] - T1[p][q] - T2[p][q];
            mm<double, BS>(Cs, Zb, Chat);          // coupling to separator k+1
            if (c == g.T - 1)
                for (int p = 0; p < BS; ++p)
                    for (int q = 0; q < BS; ++q) Chat[p][q] = 0.0;
            // block Thomas on the separator chain
            double S[BS][BS], Si[BS][BS];
            for (int p = 0; p < BS; ++p)
                for (int q = 0; q < BS; ++q) {
                    double acc = Bhat[p][q];
                    for (int k = 0; k < BS; ++k) acc -= Ahat[p][k] * Gh[k][q];
                    S[p][q] = acc;
                }
            mat_inv<double, BS>(S, Si);
            double F[BS][BS], Gnew[BS][BS];
            mm<double, BS>(Si, Ahat, F);
            mm<double, BS>(Si, Chat, Gnew);
            TS *rec = sep + (size_t)(c - 1) * 3 * BS * BS;
            for (int p = 0; p < BS; ++p)
                for (int q = 0; q < BS; ++q) {
                    rec[p * BS + q] = (TS)Si[p][q];
                    rec[BS * BS + p * BS + q] = (TS)(-F[p][q]);
                    rec[2 * BS * BS + p * BS + q] = (TS)Gnew[p][q];
                    Gh[p][q] = Gnew[p][q];
                }
        }
        // forward sweep of chunk c (for the separator on its right, k = c+1)
        if (c < g.T - 1) {
            double G[BS][BS], Z[BS][BS];
            for (int i = 0; i < n; ++i) {
                double A[BS][BS], B[BS][BS], C[BS][BS], r[BS];
                load_block<double, TS, BS>(L, s, b0 + i, rz, rz, A, B, C, r);
                double S[BS][BS], Si[BS][BS];
                for (int p = 0; p < BS; ++p)
                    for (int q = 0; q < BS; ++q) {
                        double acc = B[p][q];
                        if (i > 0)
                            for (int k = 0; k < BS; ++k) acc -= A[p][k] * G[k][q];
                        S[p][q] = acc;
                    }
                mat_inv<double, BS>(S, Si);
                double Gn2[BS][BS], Zn2[BS][BS], T1[BS][BS];
                mm<double, BS>(Si, C, Gn2);
                if (i == 0) {
                    mm<double, BS>(Si, A, Zn2);  // A of the first block couples to x_L
                } else {
                    mm<double, BS>(A, Z, T1);
                    mm<double, BS>(Si, T1, Zn2);
                }
                for (int p = 0; p < BS; ++p)
                    for (int q = 0; q < BS; ++q) { G[p][q] = Gn2[p][q]; Z[p][q] = -Zn2[p][q]; }
            }
            for (int p = 0; p < BS; ++p)
                for (int q = 0; q < BS; ++q) { Zn[p][q] = Z[p][q]; Gn[p][q] = G[p][q]; }
            Zprev_valid = c > 0 ? 1.0 : 0.0;  // chunk 0 has no left separator
        }
    }
}

template <typename TS>
__global__ void precompute_sep_kernel(const LineDesc<TS> *__restrict__ descs, int nlines) {
    int line = blockIdx.x * blockDim.x + threadIdx.x;
    if (line >= nlines) return;
    const LineDesc<TS> d = descs[line];
    if (d.method == kCFD)
        sep_precompute_line<TS, 2>(d, d.chunkM, d.sep);
    else
        sep_precompute_line<TS, 3>(d, d.chunkM, d.sep);
}

// ---------------------------------------------------------------------------------------
// Outputs.
// ---------------------------------------------------------------------------------------
template <typename T>
struct Out {
    const LineDesc<T> &d;
    int natural;
    T src;
    bool src_done;
    __device__ Out(const LineDesc<T> &dd, int nat) : d(dd), natural(nat), src(T(0)), src_done(false) {}
    __device__ __forceinline__ T source_at(int k) {
        if (k != d.src_k) return T(0);
        if (!src_done) {
            long long m = *d.clock;
            src = (T)(d.src_scale * ricker(d.src_amp, d.src_f0, d.src_tdelay, (double)(m + 1) * d.dt));
            if (d.advance_clock) *d.clock = m + 1;
            src_done = true;
        }
        return src;
    }
    // CFD node j with solution (e, g) (e unused at the ends)
    __device__ __forceinline__ void cfd_node(int j, T e, T g) {
        const T beta = (T)d.beta;
        T vin = d.v[j * d.sv];
        d.vo[j * d.sv] = vin - T(2) * beta * g;
        if (natural && d.w_out) d.w_out[j * d.sv] = vin - beta * g;
        if (j >= 1 && j <= d.N - 1) {
            T pin = d.p[j * d.sp];
            T ae = d.alpha[j * d.sp] * e;
            d.po[j * d.sp] = pin - T(2) * ae + source_at(j);
            if (natural && d.u_out) d.u_out[j * d.sp] = pin - ae;
        }
    }
    // MFD cell c with solution u
    __device__ __forceinline__ void mfd_cell(int c, T u) {
        T pin = d.p[c * d.sp];
        d.po[c * d.sp] = T(2) * u - pin + source_at(c);
        if (natural && d.u_out) d.u_out[c * d.sp] = u;
    }
    // MFD node j with (G u)_j already times 1/h
    __device__ __forceinline__ void mfd_node(int j, T gu) {
        const T beta = (T)d.beta;
        T vin = d.v[j * d.sv];
        d.vo[j * d.sv] = vin - T(2) * beta * gu;
        if (natural && d.w_out) d.w_out[j * d.sv] = vin - beta * gu;
    }
};

// v' at MFD nodes [j0, j1] from a window of cell values: cells[k - c_lo] for k in
// [c_lo, c_hi]; pressure-line index 0 and N+1 are the Dirichlet values.
template <typename T>
__device__ void mfd_nodes_from_window(Out<T> &o, int j0, int j1, const T *cells, int c_lo) {
    const int N = o.d.N;
    const T ih = (T)o.d.inv_h;
    const T p0 = o.d.p[0], pl = o.d.p[(long long)(N + 1) * o.d.sp];
    for (int j = j0; j <= j1; ++j) {
        double gw[8];
        int g0;
        int ng = mfd_G_row(N, j, &g0, gw);
        T acc = T(0);
        for (int t = 0; t < ng; ++t) {
            int k = g0 + t;
            T uk = (k == 0) ? p0 : (k == N + 1 ? pl : cells[k - c_lo]);
            acc += (T)gw[t] * uk;
        }
        o.mfd_node(j, acc * ih);
    }
}

// CFD tail unknowns (e_{N-2}, g_{N-2}, e_{N-1}, g_{N-1}, g_N) from the last middle block.
template <typename T>
__device__ __forceinline__ void cfd_tail_outputs(Out<T> &o, const LineDesc<T> &d, const T *rT,
                                                 T e_last, T g_last) {
    const int N = d.N;
    const T *tt = d.tab + kTabEnd;
    T xt[5];
    for (int i = 0; i < 5; ++i) {
        T acc = T(0);
        for (int k = 0; k < 5; ++k) acc += tt[kTabHinv + i * 5 + k] * rT[k];
        acc -= tt[kTabHinvE + i * 2 + 0] * e_last + tt[kTabHinvE + i * 2 + 1] * g_last;
        xt[i] = acc;
    }
    o.cfd_node(N - 2, xt[0], xt[1]);
    o.cfd_node(N - 1, xt[2], xt[3]);
    o.cfd_node(N, T(0), xt[4]);
}

// ---------------------------------------------------------------------------------------
// The fused partitioned solver.
// ---------------------------------------------------------------------------------------
template <typename T, int BS, int M, int SUB>
__device__ void chunked_body(const LineDesc<T> *__restrict__ descs, int desc0, int nl, int write_natural,
                             T *sm) {
    constexpr int NSEG = M / SUB;
    const int tid = threadIdx.x;
    const LineDesc<T> &d0 = descs[desc0];
    const LineShape s = line_shape(d0.method, d0.N);
    const ChunkGeom g = chunk_geom(s.nb, M);
    const int T_ = g.T;
    const int nthreads = T_ * nl;
    // shared: per line, per separator k (1..T-1): left (BS), right (BS), x (BS)
    T *smL = sm;
    T *smR = sm + (size_t)nl * T_ * BS;
    T *smX = sm + (size_t)2 * nl * T_ * BS;
    auto SL = [&](int l, int k) -> T * { return smL + ((size_t)l * T_ + k) * BS; };
    auto SR = [&](int l, int k) -> T * { return smR + ((size_t)l * T_ + k) * BS; };
    auto SX = [&](int l, int k) -> T * { return smX + ((size_t)l * T_ + k) * BS; };

    const bool active = tid < nthreads;
    const int c = active ? tid / nl : 0;
    const int l = active ? tid % nl : 0;
    const LineDesc<T> &d = descs[desc0 + l];
    const Line<T> L(d);
    const int b0 = chunk_start(g, c), n = chunk_len(g, c);
    const bool first = (c == 0), last = (c == T_ - 1);
    T rH[6], rT[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) { rH[i] = T(0); rT[i] = T(0); }
    if (active && first)
        for (int i = 0; i < s.hu; ++i) rH[i] = rhs_row(L, i);
    if (active && last)
        for (int i = 0; i < s.tu; ++i) rT[i] = rhs_row(L, s.nunk - s.tu + i);

    // ---------------- phase A ----------------
    if (active) {
        if (!last) {  // forward sweep -> y_n, hand r_sigma - A_sigma y_n to separator c+1
            T G[BS][BS], y[BS];
#pragma unroll
            for (int p = 0; p < BS; ++p) { y[p] = T(0); for (int q = 0; q < BS; ++q) G[p][q] = T(0); }
            for (int i = 0; i < n; ++i) {
                T A[BS][BS], B[BS][BS], C[BS][BS], r[BS];
                load_block<T, T, BS>(L, s, b0 + i, rH, rT, A, B, C, r);
                if (i == 0)
#pragma unroll
                    for (int p = 0; p < BS; ++p)
#pragma unroll
                        for (int q = 0; q < BS; ++q) A[p][q] = T(0);
                thomas_step<T, BS>(A, B, C, r, G, y);
            }
            T As[BS][BS], Bs[BS][BS], Cs[BS][BS], rs[BS], t[BS];
            load_block<T, T, BS>(L, s, b0 + n, rH, rT, As, Bs, Cs, rs);
            mv<T, BS>(As, y, t);
            T *dst = SL(l, c + 1);
#pragma unroll
            for (int p = 0; p < BS; ++p) dst[p] = rs[p] - t[p];
        }
        if (!first) {  // backward sweep -> y'_1, hand C_sigma y'_1 to separator c
            T G[BS][BS], y[BS];
#pragma unroll
            for (int p = 0; p < BS; ++p) { y[p] = T(0); for (int q = 0; q < BS; ++q) G[p][q] = T(0); }
            for (int i = n - 1; i >= 0; --i) {
                T A[BS][BS], B[BS][BS], C[BS][BS], r[BS];
                load_block<T, T, BS>(L, s, b0 + i, rH, rT, A, B, C, r);
                if (i == n - 1)
#pragma unroll
                    for (int p = 0; p < BS; ++p)
#pragma unroll
                        for (int q = 0; q < BS; ++q) C[p][q] = T(0);
                thomas_step<T, BS>(C, B, A, r, G, y);  // mirrored recurrence
            }
            T As[BS][BS], Bs[BS][BS], Cs[BS][BS], rs[BS], t[BS];
            load_block<T, T, BS>(L, s, b0 - 1, rH, rT, As, Bs, Cs, rs);
            mv<T, BS>(Cs, y, t);
            T *dst = SR(l, c);
#pragma unroll
            for (int p = 0; p < BS; ++p) dst[p] = t[p];
        }
    }
    __syncthreads();

    // ---------------- phase B: separator chain, one thread per line ----------------
    if (tid < nl && T_ > 1) {
        const int ll = tid;
        const T *sep = descs[desc0 + ll].sep;
        T y[BS];
#pragma unroll
        for (int p = 0; p < BS; ++p) y[p] = T(0);
        for (int k = 1; k < T_; ++k) {
            const T *rec = sep + (size_t)(k - 1) * 3 * BS * BS;
            T rhs[BS], yn[BS];
            const T *Lk = SL(ll, k), *Rk = SR(ll, k);
#pragma unroll
            for (int p = 0; p < BS; ++p) rhs[p] = Lk[p] - Rk[p];
#pragma unroll
            for (int p = 0; p < BS; ++p) {
                T acc = T(0);
#pragma unroll
                for (int q = 0; q < BS; ++q) acc += rec[p * BS + q] * rhs[q] + rec[BS * BS + p * BS + q] * y[q];
                yn[p] = acc;
            }
            T *st = SX(ll, k);
#pragma unroll
            for (int p = 0; p < BS; ++p) { y[p] = yn[p]; st[p] = yn[p]; }
        }
        T x[BS];
#pragma unroll
        for (int p = 0; p < BS; ++p) x[p] = T(0);
        for (int k = T_ - 1; k >= 1; --k) {
            const T *rec = sep + (size_t)(k - 1) * 3 * BS * BS + 2 * BS * BS;
            T *st = SX(ll, k);
            T xn[BS];
#pragma unroll
            for (int p = 0; p < BS; ++p) {
                T acc = st[p];
#pragma unroll
                for (int q = 0; q < BS; ++q) acc -= rec[p * BS + q] * x[q];
                xn[p] = acc;
            }
#pragma unroll
            for (int p = 0; p < BS; ++p) { x[p] = xn[p]; st[p] = xn[p]; }
        }
    }
    __syncthreads();
    if (!active) return;

    // ---------------- phase C ----------------
    Out<T> o(d, write_natural);
    T xL[BS], xR[BS];
#pragma unroll
    for (int p = 0; p < BS; ++p) {
        xL[p] = first ? T(0) : SX(l, c)[p];
        xR[p] = last ? T(0) : SX(l, c + 1)[p];
    }
    // forward sweep with checkpoints after every SUB blocks
    T cpG[NSEG][BS][BS], cpy[NSEG][BS];
    {
        T G[BS][BS], y[BS];
#pragma unroll
        for (int p = 0; p < BS; ++p) { y[p] = T(0); for (int q = 0; q < BS; ++q) G[p][q] = T(0); }
#pragma unroll
        for (int sg = 0; sg < NSEG - 1; ++sg) {
#pragma unroll
            for (int k = 0; k < SUB; ++k) {
                const int i = sg * SUB + k;
                if (i < n) {
                    T A[BS][BS], B[BS][BS], C[BS][BS], r[BS], t[BS];
                    load_block<T, T, BS>(L, s, b0 + i, rH, rT, A, B, C, r);
                    if (i == 0) {
                        mv<T, BS>(A, xL, t);
#pragma unroll
                        for (int p = 0; p < BS; ++p) {
                            r[p] -= first ? T(0) : t[p];
#pragma unroll
                            for (int q = 0; q < BS; ++q) A[p][q] = T(0);
                        }
                    }
                    if (i == n - 1) {
                        mv<T, BS>(C, xR, t);
#pragma unroll
                        for (int p = 0; p < BS; ++p) {
                            r[p] -= last ? T(0) : t[p];
#pragma unroll
                            for (int q = 0; q < BS; ++q) C[p][q] = T(0);
                        }
                    }
                    thomas_step<T, BS>(A, B, C, r, G, y);
                }
            }
#pragma unroll
            for (int p = 0; p < BS; ++p) { cpy[sg][p] = y[p]; for (int q = 0; q < BS; ++q) cpG[sg][p][q] = G[p][q]; }
        }
    }
    // backward: segments from last to first, each recomputed from its checkpoint
    T xn[BS];
#pragma unroll
    for (int p = 0; p < BS; ++p) xn[p] = xR[p];
#pragma unroll
    for (int sg = NSEG - 1; sg >= 0; --sg) {
        if (sg * SUB >= n) continue;
        T Gs[SUB][BS][BS], ys[SUB][BS];
        {
            T G[BS][BS], y[BS];
#pragma unroll
            for (int p = 0; p < BS; ++p) {
                y[p] = sg == 0 ? T(0) : cpy[sg > 0 ? sg - 1 : 0][p];
#pragma unroll
                for (int q = 0; q < BS; ++q) G[p][q] = sg == 0 ? T(0) : cpG[sg > 0 ? sg - 1 : 0][p][q];
            }
#pragma unroll
            for (int k = 0; k < SUB; ++k) {
                const int i = sg * SUB + k;
                if (i < n) {
                    T A[BS][BS], B[BS][BS], C[BS][BS], r[BS], t[BS];
                    load_block<T, T, BS>(L, s, b0 + i, rH, rT, A, B, C, r);
                    if (i == 0) {
                        mv<T, BS>(A, xL, t);
#pragma unroll
                        for (int p = 0; p < BS; ++p) {
                            r[p] -= first ? T(0) : t[p];
#pragma unroll
                            for (int q = 0; q < BS; ++q) A[p][q] = T(0);
                        }
                    }
                    if (i == n - 1) {
                        mv<T, BS>(C, xR, t);
#pragma unroll
                        for (int p = 0; p < BS; ++p) {
                            r[p] -= last ? T(0) : t[p];
#pragma unroll
                            for (int q = 0; q < BS; ++q) C[p][q] = T(0);
                        }
                    }
                    thomas_step<T, BS>(A, B, C, r, G, y);
#pragma unroll
                    for (int p = 0; p < BS; ++p) { ys[k][p] = y[p]; for (int q = 0; q < BS; ++q) Gs[k][p][q] = G[p][q]; }
                }
            }
        }
#pragma unroll
        for (int k = SUB - 1; k >= 0; --k) {
            const int i = sg * SUB + k;
            if (i < n) {
                T x[BS];
#pragma unroll
                for (int p = 0; p < BS; ++p) {
                    T acc = ys[k][p];
#pragma unroll
                    for (int q = 0; q < BS; ++q) acc -= Gs[k][p][q] * xn[q];
                    x[p] = acc;
                }
                const int b = b0 + i;
                if constexpr (BS == 2) {
                    o.cfd_node(3 + b, x[0], x[1]);
                    if (last && i == n - 1) cfd_tail_outputs<T>(o, d, rT, x[0], x[1]);
                } else {
                    const int q0 = s.hu + 1 + 3 * b;
                    o.mfd_cell(q0, x[0]); o.mfd_cell(q0 + 1, x[1]); o.mfd_cell(q0 + 2, x[2]);
                    if (last && i == n - 1) {
                        // nodes q0+1 .. N from this block, the tail cells and p_L
                        const T *tt = d.tab + kTabEnd;
                        T cells[8];
                        cells[0] = x[0]; cells[1] = x[1]; cells[2] = x[2];
                        for (int t2 = 0; t2 < s.tu; ++t2) {
                            T acc = T(0);
                            for (int kk = 0; kk < s.tu; ++kk) acc += tt[kTabHinv + t2 * s.tu + kk] * rT[kk];
#pragma unroll
                            for (int kk = 0; kk < BS; ++kk) acc -= tt[kTabHinvE + t2 * BS + kk] * x[kk];
                            cells[3 + t2] = acc;
                            o.mfd_cell(q0 + 3 + t2, acc);
                        }
                        mfd_nodes_from_window<T>(o, q0 + 1, d.N, cells, q0);
                    } else {
                        const T ih = (T)d.inv_h;
                        const T w0 = (T)mim_w(0), w1 = (T)mim_w(1), w2 = (T)mim_w(2), w3 = (T)mim_w(3);
                        o.mfd_node(q0 + 1, ih * (w0 * x[0] + w1 * x[1] + w2 * x[2] + w3 * xn[0]));
                        o.mfd_node(q0 + 2, ih * (w0 * x[1] + w1 * x[2] + w2 * xn[0] + w3 * xn[1]));
                        o.mfd_node(q0 + 3, ih * (w0 * x[2] + w1 * xn[0] + w2 * xn[1] + w3 * xn[2]));
                    }
                }
#pragma unroll
                for (int p = 0; p < BS; ++p) xn[p] = x[p];
            }
        }
    }
    // xn now holds the chunk's first block.  Separator on the right: outputs by this chunk.
    if (!last) {
        const int b = b0 + n;
        if constexpr (BS == 2) {
            o.cfd_node(3 + b, xR[0], xR[1]);
        } else {
            const int q0 = s.hu + 1 + 3 * b;
            o.mfd_cell(q0, xR[0]); o.mfd_cell(q0 + 1, xR[1]); o.mfd_cell(q0 + 2, xR[2]);
        }
    }
    if constexpr (BS == 2) {
        if (first) {  // head unknowns g0, e1, g1, e2, g2
            const T *th = d.tab;
            T xh[5];
            for (int i = 0; i < 5; ++i) {
                T acc = T(0);
                for (int k = 0; k < 5; ++k) acc += th[kTabHinv + i * 5 + k] * rH[k];
                acc -= th[kTabHinvE + i * 2 + 0] * xn[0] + th[kTabHinvE + i * 2 + 1] * xn[1];
                xh[i] = acc;
            }
            o.cfd_node(0, T(0), xh[0]);
            o.cfd_node(1, xh[1], xh[2]);
            o.cfd_node(2, xh[3], xh[4]);
        }
    } else {
        if (first) {  // head cells 1..hu, then nodes 0 .. hu+1
            const T *th = d.tab;
            T cells[12];
            cells[0] = d.p[0];
            for (int i = 0; i < s.hu; ++i) {
                T acc = T(0);
                for (int k = 0; k < s.hu; ++k) acc += th[kTabHinv + i * s.hu + k] * rH[k];
#pragma unroll
                for (int k = 0; k < BS; ++k) acc -= th[kTabHinvE + i * BS + k] * xn[k];
                cells[1 + i] = acc;
                o.mfd_cell(1 + i, acc);
            }
            cells[s.hu + 1] = xn[0]; cells[s.hu + 2] = xn[1]; cells[s.hu + 3] = xn[2];
            mfd_nodes_from_window<T>(o, 0, s.hu + 1, cells, 0);
        } else {  // nodes c_first-2 .. c_first from the left separator and the first block
            const int q0 = s.hu + 1 + 3 * b0;
            T cells[6] = {xL[0], xL[1], xL[2], xn[0], xn[1], xn[2]};
            const T ih = (T)d.inv_h;
            const T w0 = (T)mim_w(0), w1 = (T)mim_w(1), w2 = (T)mim_w(2), w3 = (T)mim_w(3);
#pragma unroll
            for (int jj = 0; jj < 3; ++jj)
                o.mfd_node(q0 - 2 + jj, ih * (w0 * cells[jj] + w1 * cells[jj + 1] + w2 * cells[jj + 2] + w3 * cells[jj + 3]));
        }
    }
}

template <typename T, int BS, int M, int SUB>
__global__ void __launch_bounds__(256, 2)
line_solve_chunked_kernel(const LineDesc<T> *__restrict__ descs, const int4 *__restrict__ groups,
                          int write_natural) {
    extern __shared__ __align__(16) unsigned char smraw[];
    T *sm = reinterpret_cast<T *>(smraw);
    const int4 gr = groups[blockIdx.x];  // (first descriptor, lines, method, unused)
    chunked_body<T, BS, M, SUB>(descs, gr.x, gr.y, write_natural, sm);
}

int chunk_M(int method) { return method == kCFD ? 32 : 16; }

template <typename T>
cudaError_t launch_precompute_sep(const LineDesc<T> *d, int nlines, cudaStream_t s) {
    if (nlines <= 0) return cudaSuccess;
    precompute_sep_kernel<T><<<(nlines + 63) / 64, 64, 0, s>>>(d, nlines);
    return cudaGetLastError();
}

template <typename T, int BS, int M, int SUB>
cudaError_t launch_chunked_variant(const LineDesc<T> *d, const int4 *groups, int ngroups,
                                   size_t smem_bytes, int write_natural, cudaStream_t s) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(line_solve_chunked_kernel<T, BS, M, SUB>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    line_solve_chunked_kernel<T, BS, M, SUB><<<ngroups, 256, smem_bytes, s>>>(d, groups, write_natural);
    return cudaGetLastError();
}

// groups of one method only (the caller splits mixed batches).
template <typename T>
cudaError_t launch_line_solve_chunked(const LineDesc<T> *d, const int4 *groups, int ngroups,
                                      int method, size_t smem_bytes, int write_natural,
                                      cudaStream_t s) {
    if (ngroups <= 0) return cudaSuccess;
    if (method == kCFD)
        return launch_chunked_variant<T, 2, 32, 8>(d, groups, ngroups, smem_bytes, write_natural, s);
    return launch_chunked_variant<T, 3, 16, 4>(d, groups, ngroups, smem_bytes, write_natural, s);
}

template cudaError_t launch_precompute_sep<float>(const LineDesc<float> *, int, cudaStream_t);
template cudaError_t launch_precompute_sep<double>(const LineDesc<double> *, int, cudaStream_t);
template cudaError_t launch_line_solve_chunked<float>(const LineDesc<float> *, const int4 *, int,
                                                      int, size_t, int, cudaStream_t);
template cudaError_t launch_line_solve_chunked<double>(const LineDesc<double> *, const int4 *, int,
                                                       int, size_t, int, cudaStream_t);

}  // namespace adi
