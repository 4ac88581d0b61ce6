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
// Shared-memory layout of one CTA: staged lines (pressure, velocity, alpha; Lp = N+2 each),
// then the separator hand-over slots SL (left part), SR (right part) and SX (solutions).
// ---------------------------------------------------------------------------------------
__host__ __device__ inline size_t chunked_smem_elems(int N, int nl, int T, int bs) {
    return (size_t)3 * nl * (N + 2) + (size_t)3 * nl * T * bs;
}

// Affine map y -> m y + off on BS-vectors (separator substitution scans).
template <typename T, int BS>
struct Aff {
    T m[BS][BS];
    T off[BS];
};

template <typename T, int BS>
__device__ __forceinline__ void aff_shfl(Aff<T, BS> &dst, const Aff<T, BS> &src, int delta, bool up) {
#pragma unroll
    for (int i = 0; i < BS; ++i) {
#pragma unroll
        for (int j = 0; j < BS; ++j)
            dst.m[i][j] = up ? __shfl_up_sync(0xffffffffu, src.m[i][j], delta)
                             : __shfl_down_sync(0xffffffffu, src.m[i][j], delta);
        dst.off[i] = up ? __shfl_up_sync(0xffffffffu, src.off[i], delta)
                        : __shfl_down_sync(0xffffffffu, src.off[i], delta);
    }
}
// a <- a o b  (apply b first, then a)
template <typename T, int BS>
__device__ __forceinline__ void aff_after(Aff<T, BS> &a, const Aff<T, BS> &b) {
    Aff<T, BS> r;
#pragma unroll
    for (int i = 0; i < BS; ++i) {
        T acc = a.off[i];
#pragma unroll
        for (int k = 0; k < BS; ++k) acc += a.m[i][k] * b.off[k];
        r.off[i] = acc;
#pragma unroll
        for (int j = 0; j < BS; ++j) {
            T s = T(0);
#pragma unroll
            for (int k = 0; k < BS; ++k) s += a.m[i][k] * b.m[k][j];
            r.m[i][j] = s;
        }
    }
    a = r;
}

// Separator chain of one line, one warp: forward y_k = Sinv_k rhs_k + mF_k y_{k-1}, then
// backward x_k = y_k - Gamma_k x_{k+1}, both as warp scans of affine maps (k = 1..K).
template <typename T, int BS>
__device__ void separator_scan(const T *__restrict__ sep, const T *SLl, const T *SRl, T *SXl, int K,
                               int lane) {
    const int per = (K + 31) / 32;
    const int k0 = 1 + lane * per;
    const int k1 = min(K + 1, k0 + per);
    // forward: local composition
    Aff<T, BS> a;
#pragma unroll
    for (int i = 0; i < BS; ++i) {
        a.off[i] = T(0);
#pragma unroll
        for (int j = 0; j < BS; ++j) a.m[i][j] = i == j ? T(1) : T(0);
    }
    for (int k = k0; k < k1; ++k) {
        const T *rec = sep + (size_t)(k - 1) * 3 * BS * BS;
        Aff<T, BS> st;
#pragma unroll
        for (int i = 0; i < BS; ++i) {
            T g = T(0);
#pragma unroll
            for (int q = 0; q < BS; ++q) {
                g += rec[i * BS + q] * (SLl[k * BS + q] - SRl[k * BS + q]);
                st.m[i][q] = rec[BS * BS + i * BS + q];
            }
            st.off[i] = g;
        }
        aff_after<T, BS>(st, a);
        a = st;
    }
    // inclusive scan over lanes (earlier lanes applied first)
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        Aff<T, BS> o;
        aff_shfl<T, BS>(o, a, s, true);
        if (lane >= s) aff_after<T, BS>(a, o);
    }
    T y[BS];
#pragma unroll
    for (int i = 0; i < BS; ++i) {
        T v = __shfl_up_sync(0xffffffffu, a.off[i], 1);
        y[i] = lane == 0 ? T(0) : v;
    }
    for (int k = k0; k < k1; ++k) {
        const T *rec = sep + (size_t)(k - 1) * 3 * BS * BS;
        T yn[BS];
#pragma unroll
        for (int i = 0; i < BS; ++i) {
            T acc = T(0);
#pragma unroll
            for (int q = 0; q < BS; ++q)
                acc += rec[i * BS + q] * (SLl[k * BS + q] - SRl[k * BS + q]) + rec[BS * BS + i * BS + q] * y[q];
            yn[i] = acc;
        }
#pragma unroll
        for (int i = 0; i < BS; ++i) { y[i] = yn[i]; SXl[k * BS + i] = yn[i]; }
    }
    // backward: local composition from the end of the range
#pragma unroll
    for (int i = 0; i < BS; ++i) {
        a.off[i] = T(0);
#pragma unroll
        for (int j = 0; j < BS; ++j) a.m[i][j] = i == j ? T(1) : T(0);
    }
    for (int k = k1 - 1; k >= k0; --k) {
        const T *G = sep + (size_t)(k - 1) * 3 * BS * BS + 2 * BS * BS;
        Aff<T, BS> st;
#pragma unroll
        for (int i = 0; i < BS; ++i) {
#pragma unroll
            for (int q = 0; q < BS; ++q) st.m[i][q] = -G[i * BS + q];
            st.off[i] = SXl[k * BS + i];
        }
        aff_after<T, BS>(st, a);
        a = st;
    }
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        Aff<T, BS> o;
        aff_shfl<T, BS>(o, a, s, false);
        if (lane + s < 32) aff_after<T, BS>(a, o);
    }
    T x[BS];
#pragma unroll
    for (int i = 0; i < BS; ++i) {
        T v = __shfl_down_sync(0xffffffffu, a.off[i], 1);
        x[i] = lane == 31 ? T(0) : v;
    }
    for (int k = k1 - 1; k >= k0; --k) {
        const T *G = sep + (size_t)(k - 1) * 3 * BS * BS + 2 * BS * BS;
        T xn[BS];
#pragma unroll
        for (int i = 0; i < BS; ++i) {
            T acc = SXl[k * BS + i];
#pragma unroll
            for (int q = 0; q < BS; ++q) acc -= G[i * BS + q] * x[q];
            xn[i] = acc;
        }
#pragma unroll
        for (int i = 0; i < BS; ++i) { x[i] = xn[i]; SXl[k * BS + i] = xn[i]; }
    }
}

// ---------------------------------------------------------------------------------------
// One staged line: shared-memory arrays plus the scalars the sweeps need, in registers.
// Outputs are written in place into the staged arrays (natural outputs of stage-2 lines go
// straight to global memory).
// ---------------------------------------------------------------------------------------
template <typename T>
struct Ln {
    T *P, *V;           // staged pressure / velocity line (shared memory)
    const T *Al;        // staged alpha line (shared memory)
    T beta, ih;
    int N, hu, tu, nb, nunk;
    int src_k;          // pressure index of the point source on this line, or -1
    T srcv;             // dt/2 f(t_{m+1}) at the source point
    bool src_hit;       // this thread wrote the source point
    int natural;
    T *u_out, *w_out;   // natural outputs (global), or nullptr
    long long sp, sv;   // strides of u_out / w_out
};

template <typename T, int BS>
__device__ __forceinline__ void mblock(const Ln<T> &L, int b, T (&A)[BS][BS], T (&B)[BS][BS],
                                       T (&C)[BS][BS], T (&r)[BS]) {
    if constexpr (BS == 2) {
        const int j = 3 + b;
        const T t3 = T(3) * L.ih;
        const T tb = t3 * L.beta;
        A[0][0] = T(1); A[0][1] = -tb; A[1][0] = -t3 * L.Al[j - 1]; A[1][1] = T(1);
        B[0][0] = T(4); B[0][1] = T(0); B[1][0] = T(0); B[1][1] = T(4);
        C[0][0] = T(1); C[0][1] = tb; C[1][0] = t3 * L.Al[j + 1]; C[1][1] = T(1);
        r[0] = t3 * (L.V[j + 1] - L.V[j - 1]);
        r[1] = t3 * (L.P[j + 1] - L.P[j - 1]);
    } else {
        const int cb = L.hu + 1 + 3 * b;
        const T w0 = T(1.0 / 24.0), w1 = T(-9.0 / 8.0), w2 = T(9.0 / 8.0), w3 = T(-1.0 / 24.0);
        const T bh2 = L.beta * L.ih * L.ih;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int c = cb + k;
            const T a = L.Al[c];
            const T sc = a * bh2;
#pragma unroll
            for (int l = 0; l < 3; ++l) {
                const int dA = l - k - 3, dB = l - k, dC = l - k + 3;
                A[k][l] = (dA >= -3) ? -sc * (T)mim_DG(dA + 3) : T(0);
                B[k][l] = (dB == 0 ? T(1) : T(0)) - sc * (T)mim_DG(dB + 3);
                C[k][l] = (dC <= 3) ? -sc * (T)mim_DG(dC + 3) : T(0);
            }
            const T dv = w0 * L.V[c - 2] + w1 * L.V[c - 1] + w2 * L.V[c] + w3 * L.V[c + 1];
            r[k] = L.P[c] - a * L.ih * dv;
        }
    }
}

// Boundary-block corrections (head elimination on block 0, tail on block nb-1), held in
// registers by the chunks that own those blocks.
template <typename T, int BS>
struct Corr {
    T dB[BS][BS];
    T dr[BS];
};

template <typename T, int BS>
__device__ __forceinline__ void blk(const Ln<T> &L, int b, const Corr<T, BS> &c0, const Corr<T, BS> &cl,
                                    T (&A)[BS][BS], T (&B)[BS][BS], T (&C)[BS][BS], T (&r)[BS]) {
    mblock<T, BS>(L, b, A, B, C, r);
    if (b == 0) {
#pragma unroll
        for (int i = 0; i < BS; ++i) {
            r[i] -= c0.dr[i];
#pragma unroll
            for (int j = 0; j < BS; ++j) { B[i][j] -= c0.dB[i][j]; A[i][j] = T(0); }
        }
    }
    if (b == L.nb - 1) {
#pragma unroll
        for (int i = 0; i < BS; ++i) {
            r[i] -= cl.dr[i];
#pragma unroll
            for (int j = 0; j < BS; ++j) { B[i][j] -= cl.dB[i][j]; C[i][j] = T(0); }
        }
    }
}

template <typename T>
__device__ __forceinline__ T src_at(Ln<T> &L, int k) {
    if (k != L.src_k) return T(0);
    L.src_hit = true;
    return L.srcv;
}
template <typename T>
__device__ __forceinline__ void out_cfd(Ln<T> &L, int j, T e, T g) {
    T vin = L.V[j];
    L.V[j] = vin - T(2) * L.beta * g;
    if (L.natural) L.w_out[j * L.sv] = vin - L.beta * g;
    if (j >= 1 && j <= L.N - 1) {
        T pin = L.P[j];
        T ae = L.Al[j] * e;
        L.P[j] = pin - T(2) * ae + src_at(L, j);
        if (L.natural) L.u_out[j * L.sp] = pin - ae;
    }
}
template <typename T>
__device__ __forceinline__ void out_mfd_cell(Ln<T> &L, int c, T u) {
    T pin = L.P[c];
    L.P[c] = T(2) * u - pin + src_at(L, c);
    if (L.natural) L.u_out[c * L.sp] = u;
}
template <typename T>
__device__ __forceinline__ void out_mfd_node(Ln<T> &L, int j, T gu) {
    T vin = L.V[j];
    L.V[j] = vin - T(2) * L.beta * gu;
    if (L.natural) L.w_out[j * L.sv] = vin - L.beta * gu;
}

// v' at MFD nodes [j0, j1] from cells[k - c_lo] (k in [c_lo, ...]); pressure indices 0 and
// N+1 are the Dirichlet values.
template <typename T>
__device__ __noinline__ void mfd_nodes_window(Ln<T> &L, int j0, int j1, const T *cells, int c_lo) {
    const int N = L.N;
    const T p0 = L.P[0], pl = L.P[N + 1];
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
        out_mfd_node(L, j, acc * L.ih);
    }
}

// CFD head (g0, e1, g1, e2, g2) from the first middle block.
template <typename T>
__device__ __noinline__ void cfd_head_out(Ln<T> &L, const T *th, const T *rH, T e, T g) {
    T xh[5];
    for (int i = 0; i < 5; ++i) {
        T acc = T(0);
        for (int k = 0; k < 5; ++k) acc += th[kTabHinv + i * 5 + k] * rH[k];
        xh[i] = acc - th[kTabHinvE + i * 2] * e - th[kTabHinvE + i * 2 + 1] * g;
    }
    out_cfd(L, 0, T(0), xh[0]);
    out_cfd(L, 1, xh[1], xh[2]);
    out_cfd(L, 2, xh[3], xh[4]);
}
// CFD tail (e_{N-2}, g_{N-2}, e_{N-1}, g_{N-1}, g_N) from the last middle block.
template <typename T>
__device__ __noinline__ void cfd_tail_out(Ln<T> &L, const T *tt, const T *rT, T e, T g) {
    const int N = L.N;
    T xt[5];
    for (int i = 0; i < 5; ++i) {
        T acc = T(0);
        for (int k = 0; k < 5; ++k) acc += tt[kTabHinv + i * 5 + k] * rT[k];
        xt[i] = acc - tt[kTabHinvE + i * 2] * e - tt[kTabHinvE + i * 2 + 1] * g;
    }
    out_cfd(L, N - 2, xt[0], xt[1]);
    out_cfd(L, N - 1, xt[2], xt[3]);
    out_cfd(L, N, T(0), xt[4]);
}
// MFD head cells 1..hu from the first middle block, then nodes 0 .. hu+1.
template <typename T>
__device__ __noinline__ void mfd_head_out(Ln<T> &L, const T *th, const T *rH, const T *x0) {
    T cells[12];
    cells[0] = L.P[0];
    for (int i = 0; i < L.hu; ++i) {
        T acc = T(0);
        for (int k = 0; k < L.hu; ++k) acc += th[kTabHinv + i * L.hu + k] * rH[k];
        for (int k = 0; k < 3; ++k) acc -= th[kTabHinvE + i * 3 + k] * x0[k];
        cells[1 + i] = acc;
    }
    cells[L.hu + 1] = x0[0]; cells[L.hu + 2] = x0[1]; cells[L.hu + 3] = x0[2];
    for (int i = 0; i < L.hu; ++i) out_mfd_cell(L, 1 + i, cells[1 + i]);
    mfd_nodes_window(L, 0, L.hu + 1, cells, 0);
}
// MFD tail cells from the last middle block (cells q0..q0+2), then nodes q0+1 .. N.
template <typename T>
__device__ __noinline__ void mfd_tail_out(Ln<T> &L, const T *tt, const T *rT, const T *xl, int q0) {
    T cells[8];
    cells[0] = xl[0]; cells[1] = xl[1]; cells[2] = xl[2];
    for (int i = 0; i < L.tu; ++i) {
        T acc = T(0);
        for (int k = 0; k < L.tu; ++k) acc += tt[kTabHinv + i * L.tu + k] * rT[k];
        for (int k = 0; k < 3; ++k) acc -= tt[kTabHinvE + i * 3 + k] * xl[k];
        cells[3 + i] = acc;
    }
    for (int i = 0; i < L.tu; ++i) out_mfd_cell(L, q0 + 3 + i, cells[3 + i]);
    mfd_nodes_window(L, q0 + 1, L.N, cells, q0);
}

// Correction of a boundary block: dB = tab[kTabDB], dr = tab[kTabK] . r_end.
template <typename T, int BS>
__device__ __forceinline__ void load_corr(Corr<T, BS> &c, const T *tab, const T *rend, int m) {
#pragma unroll
    for (int i = 0; i < BS; ++i) {
#pragma unroll
        for (int j = 0; j < BS; ++j) c.dB[i][j] = tab[kTabDB + i * BS + j];
        T acc = T(0);
        for (int k = 0; k < m; ++k) acc += tab[kTabK + i * m + k] * rend[k];
        c.dr[i] = acc;
    }
}

// ---------------------------------------------------------------------------------------
// The fused partitioned solver (one CTA per group of nl consecutive lines of one
// simulation and direction).
// ---------------------------------------------------------------------------------------
template <typename T, int BS, int M, int SUB>
__device__ void chunked_body(const LineDesc<T> *__restrict__ descs, int desc0, int nl, int write_natural,
                             T *sm) {
    constexpr int NSEG = M / SUB;
    const int tid = threadIdx.x;
    const LineDesc<T> &d0 = descs[desc0];
    const int N = d0.N;
    const LineShape s = line_shape(d0.method, N);
    const ChunkGeom g = chunk_geom(s.nb, M);
    const int T_ = g.T;
    const int nthreads = T_ * nl;
    const int Lp = N + 2;
    const int np = p_last(d0.method, N) + 1;  // pressure-line length
    T *sP = sm;
    T *sV = sP + (size_t)nl * Lp;
    T *sA = sV + (size_t)nl * Lp;
    T *smL = sA + (size_t)nl * Lp;
    T *smR = smL + (size_t)nl * T_ * BS;
    T *smX = smR + (size_t)nl * T_ * BS;
    const long long sp = d0.sp, sv = d0.sv;

    // ---------------- stage the lines into shared memory ----------------
    {
        // consecutive lines of one simulation are a fixed stride apart
        const long long lsp = nl > 1 ? (long long)(descs[desc0 + 1].p - d0.p) : 0;
        const long long lsv = nl > 1 ? (long long)(descs[desc0 + 1].v - d0.v) : 0;
        const T *gp = d0.p, *gv = d0.v, *ga = d0.alpha;
        const int per = blockDim.x / nl;
        const int lc = tid % nl, kc = tid / nl;
        if (sp == 1) {
            for (int ll = 0; ll < nl; ++ll)
                for (int k = tid; k < np; k += blockDim.x) {
                    sP[ll * Lp + k] = gp[ll * lsp + k];
                    sA[ll * Lp + k] = ga[ll * lsp + k];
                }
        } else if (tid < per * nl) {
            for (int k = kc; k < np; k += per) {
                sP[lc * Lp + k] = gp[lc * lsp + k * sp];
                sA[lc * Lp + k] = ga[lc * lsp + k * sp];
            }
        }
        if (sv == 1) {
            for (int ll = 0; ll < nl; ++ll)
                for (int k = tid; k <= N; k += blockDim.x) sV[ll * Lp + k] = gv[ll * lsv + k];
        } else if (tid < per * nl) {
            for (int k = kc; k <= N; k += per) sV[lc * Lp + k] = gv[lc * lsv + k * sv];
        }
    }
    __syncthreads();

    const bool active = tid < nthreads;
    const int c = active ? tid / nl : 0;
    const int l = active ? tid % nl : 0;
    const LineDesc<T> &d = descs[desc0 + l];
    Ln<T> L;
    L.P = sP + (size_t)l * Lp; L.V = sV + (size_t)l * Lp; L.Al = sA + (size_t)l * Lp;
    L.beta = (T)d.beta; L.ih = (T)d.inv_h;
    L.N = N; L.hu = s.hu; L.tu = s.tu; L.nb = s.nb; L.nunk = s.nunk;
    L.src_k = d.src_k; L.srcv = T(0); L.src_hit = false;
    L.natural = write_natural && d.u_out != nullptr;
    L.u_out = d.u_out; L.w_out = d.w_out; L.sp = d.snp; L.sv = d.snv;
    const T *th = d.tab, *tt = d.tab + kTabEnd;
    auto SL = [&](int ll, int k) -> T * { return smL + ((size_t)ll * T_ + k) * BS; };
    auto SR = [&](int ll, int k) -> T * { return smR + ((size_t)ll * T_ + k) * BS; };
    auto SX = [&](int ll, int k) -> T * { return smX + ((size_t)ll * T_ + k) * BS; };
    const int b0 = chunk_start(g, c), n = chunk_len(g, c);
    const bool first = (c == 0), last = (c == T_ - 1);
    T rH[6], rT[6];
    Corr<T, BS> c0, cl;
#pragma unroll
    for (int i = 0; i < BS; ++i) {
        c0.dr[i] = cl.dr[i] = T(0);
#pragma unroll
        for (int j = 0; j < BS; ++j) c0.dB[i][j] = cl.dB[i][j] = T(0);
    }
    if (active && (first || last)) {
        const Line<T> Lg(d, L.P, L.V, L.Al);
        if (first) {
            for (int i = 0; i < s.hu; ++i) rH[i] = rhs_row(Lg, i);
            load_corr<T, BS>(c0, th, rH, s.hu);
        }
        if (last) {
            for (int i = 0; i < s.tu; ++i) rT[i] = rhs_row(Lg, s.nunk - s.tu + i);
            load_corr<T, BS>(cl, tt, rT, s.tu);
        }
    }
    if (active && L.src_k >= 0) {
        long long m = *d.clock;
        L.srcv = (T)(d.src_scale * ricker(d.src_amp, d.src_f0, d.src_tdelay, (double)(m + 1) * d.dt));
    }

    // ---------------- phase A ----------------
    if (active) {
        if (!last) {  // forward sweep -> y_n, hand r_sigma - A_sigma y_n to separator c+1
            T G[BS][BS], y[BS];
#pragma unroll
            for (int p = 0; p < BS; ++p) { y[p] = T(0); for (int q = 0; q < BS; ++q) G[p][q] = T(0); }
            for (int i = 0; i < n; ++i) {
                T A[BS][BS], B[BS][BS], C[BS][BS], r[BS];
                blk<T, BS>(L, b0 + i, c0, cl, A, B, C, r);
                if (i == 0)
#pragma unroll
                    for (int p = 0; p < BS; ++p)
#pragma unroll
                        for (int q = 0; q < BS; ++q) A[p][q] = T(0);
                thomas_step<T, BS>(A, B, C, r, G, y);
            }
            T As[BS][BS], Bs[BS][BS], Cs[BS][BS], rs[BS], t[BS];
            mblock<T, BS>(L, b0 + n, As, Bs, Cs, rs);
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
                blk<T, BS>(L, b0 + i, c0, cl, A, B, C, r);
                if (i == n - 1)
#pragma unroll
                    for (int p = 0; p < BS; ++p)
#pragma unroll
                        for (int q = 0; q < BS; ++q) C[p][q] = T(0);
                thomas_step<T, BS>(C, B, A, r, G, y);  // mirrored recurrence
            }
            T As[BS][BS], Bs[BS][BS], Cs[BS][BS], rs[BS], t[BS];
            mblock<T, BS>(L, b0 - 1, As, Bs, Cs, rs);
            mv<T, BS>(Cs, y, t);
            T *dst = SR(l, c);
#pragma unroll
            for (int p = 0; p < BS; ++p) dst[p] = t[p];
        }
    }
    __syncthreads();

    // ---------------- phase B: separator chains, one warp per line ----------------
    if (T_ > 1) {
        const int warp = tid >> 5, lane = tid & 31, nwarps = blockDim.x >> 5;
        for (int ll = warp; ll < nl; ll += nwarps)
            separator_scan<T, BS>(descs[desc0 + ll].sep, SL(ll, 0), SR(ll, 0), SX(ll, 0), T_ - 1, lane);
    }
    __syncthreads();

    // ---------------- phase C ----------------
    T xL[BS], xR[BS];
#pragma unroll
    for (int p = 0; p < BS; ++p) { xL[p] = T(0); xR[p] = T(0); }
    if (active) {
#pragma unroll
        for (int p = 0; p < BS; ++p) {
            xL[p] = first ? T(0) : SX(l, c)[p];
            xR[p] = last ? T(0) : SX(l, c + 1)[p];
        }
        // Segments of SUB blocks from the last to the first; each one re-runs the forward
        // elimination from the chunk start (no stored factors), keeps its SUB factors in
        // registers and back-substitutes.  CFD blocks read the nodes next to them, so the
        // first block of a segment writes its outputs only after the segment below has been
        // recomputed (pending output).
        T xn[BS];
#pragma unroll
        for (int p = 0; p < BS; ++p) xn[p] = xR[p];
        int pend_node = -1;
        T pend_e = T(0), pend_g = T(0);
        const int nseg = (n + SUB - 1) / SUB;
        for (int sg = nseg - 1; sg >= 0; --sg) {
            T G[BS][BS], y[BS];
#pragma unroll
            for (int p = 0; p < BS; ++p) { y[p] = T(0); for (int q = 0; q < BS; ++q) G[p][q] = T(0); }
            // forward, no storage, up to the segment
            for (int i = 0; i < sg * SUB; ++i) {
                T A[BS][BS], B[BS][BS], C[BS][BS], r[BS], t[BS];
                blk<T, BS>(L, b0 + i, c0, cl, A, B, C, r);
                if (i == 0) {
                    mv<T, BS>(A, xL, t);
#pragma unroll
                    for (int p = 0; p < BS; ++p) {
                        r[p] -= t[p];
#pragma unroll
                        for (int q = 0; q < BS; ++q) A[p][q] = T(0);
                    }
                }
                thomas_step<T, BS>(A, B, C, r, G, y);
            }
            // forward over the segment, factors kept
            T Gs[SUB][BS][BS], ys[SUB][BS];
#pragma unroll
            for (int k = 0; k < SUB; ++k) {
                const int i = sg * SUB + k;
                if (i < n) {
                    T A[BS][BS], B[BS][BS], C[BS][BS], r[BS], t[BS];
                    blk<T, BS>(L, b0 + i, c0, cl, A, B, C, r);
                    if (i == 0) {
                        mv<T, BS>(A, xL, t);
#pragma unroll
                        for (int p = 0; p < BS; ++p) {
                            r[p] -= t[p];
#pragma unroll
                            for (int q = 0; q < BS; ++q) A[p][q] = T(0);
                        }
                    }
                    if (i == n - 1) {
                        mv<T, BS>(C, xR, t);
#pragma unroll
                        for (int p = 0; p < BS; ++p) {
                            r[p] -= t[p];
#pragma unroll
                            for (int q = 0; q < BS; ++q) C[p][q] = T(0);
                        }
                    }
                    thomas_step<T, BS>(A, B, C, r, G, y);
#pragma unroll
                    for (int p = 0; p < BS; ++p) { ys[k][p] = y[p]; for (int q = 0; q < BS; ++q) Gs[k][p][q] = G[p][q]; }
                }
            }
            if constexpr (BS == 2) {
                if (pend_node >= 0) { out_cfd(L, pend_node, pend_e, pend_g); pend_node = -1; }
            }
            // back substitution over the segment, outputs
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
                        if (k == 0) { pend_node = 3 + b; pend_e = x[0]; pend_g = x[1]; }
                        else out_cfd(L, 3 + b, x[0], x[1]);
                        if (last && i == n - 1) cfd_tail_out(L, tt, rT, x[0], x[1]);
                    } else {
                        const int q0 = s.hu + 1 + 3 * b;
                        out_mfd_cell(L, q0, x[0]); out_mfd_cell(L, q0 + 1, x[1]); out_mfd_cell(L, q0 + 2, x[2]);
                        if (last && i == n - 1) {
                            mfd_tail_out(L, tt, rT, x, q0);
                        } else {
                            const T w0 = T(1.0 / 24.0), w1 = T(-9.0 / 8.0), w2 = T(9.0 / 8.0), w3 = T(-1.0 / 24.0);
                            out_mfd_node(L, q0 + 1, L.ih * (w0 * x[0] + w1 * x[1] + w2 * x[2] + w3 * xn[0]));
                            out_mfd_node(L, q0 + 2, L.ih * (w0 * x[1] + w1 * x[2] + w2 * xn[0] + w3 * xn[1]));
                            out_mfd_node(L, q0 + 3, L.ih * (w0 * x[2] + w1 * xn[0] + w2 * xn[1] + w3 * xn[2]));
                        }
                    }
#pragma unroll
                    for (int p = 0; p < BS; ++p) xn[p] = x[p];
                }
            }
        }
        if constexpr (BS == 2) {
            if (pend_node >= 0) out_cfd(L, pend_node, pend_e, pend_g);
            if (first) cfd_head_out(L, th, rH, xn[0], xn[1]);
        } else {
            if (first) {
                mfd_head_out(L, th, rH, xn);
            } else {  // nodes c_first-2 .. c_first from the left separator and the first block
                const int q0 = s.hu + 1 + 3 * b0;
                const T w0 = T(1.0 / 24.0), w1 = T(-9.0 / 8.0), w2 = T(9.0 / 8.0), w3 = T(-1.0 / 24.0);
                out_mfd_node(L, q0 - 2, L.ih * (w0 * xL[0] + w1 * xL[1] + w2 * xL[2] + w3 * xn[0]));
                out_mfd_node(L, q0 - 1, L.ih * (w0 * xL[1] + w1 * xL[2] + w2 * xn[0] + w3 * xn[1]));
                out_mfd_node(L, q0, L.ih * (w0 * xL[2] + w1 * xn[0] + w2 * xn[1] + w3 * xn[2]));
            }
        }
        (void)NSEG;
    }
    // the separator on the right of each chunk: outputs after every chunk has read its halo
    __syncthreads();
    if (active && !last) {
        const int b = b0 + n;
        if constexpr (BS == 2) {
            out_cfd(L, 3 + b, xR[0], xR[1]);
        } else {
            const int q0 = s.hu + 1 + 3 * b;
            out_mfd_cell(L, q0, xR[0]); out_mfd_cell(L, q0 + 1, xR[1]); out_mfd_cell(L, q0 + 2, xR[2]);
        }
    }
    if (active && L.src_hit && d.advance_clock) *d.clock = *d.clock + 1;
    __syncthreads();

    // ---------------- write the staged lines back ----------------
    {
        const long long lsp = nl > 1 ? (long long)(descs[desc0 + 1].po - d0.po) : 0;
        const long long lsv = nl > 1 ? (long long)(descs[desc0 + 1].vo - d0.vo) : 0;
        const long long spo = d0.spo, svo = d0.svo;
        T *gp = d0.po, *gv = d0.vo;
        const int per = blockDim.x / nl;
        const int lc = tid % nl, kc = tid / nl;
        if (spo == 1) {
            for (int ll = 0; ll < nl; ++ll)
                for (int k = tid; k < np; k += blockDim.x) gp[ll * lsp + k] = sP[ll * Lp + k];
        } else if (tid < per * nl) {
            for (int k = kc; k < np; k += per) gp[lc * lsp + k * spo] = sP[lc * Lp + k];
        }
        if (svo == 1) {
            for (int ll = 0; ll < nl; ++ll)
                for (int k = tid; k <= N; k += blockDim.x) gv[ll * lsv + k] = sV[ll * Lp + k];
        } else if (tid < per * nl) {
            for (int k = kc; k <= N; k += per) gv[lc * lsv + k * svo] = sV[lc * Lp + k];
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

size_t chunked_smem_bytes(int N, int nl, int T, int bs, size_t esz) {
    return chunked_smem_elems(N, nl, T, bs) * esz;
}

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
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, kChunkSmemMax);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(line_solve_chunked_kernel<T, BS, M, SUB>,
                                 cudaFuncAttributePreferredSharedMemoryCarveout, 100);
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
