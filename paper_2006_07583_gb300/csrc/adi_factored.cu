// adi_factored.cu -- the factored line solver: per-line block-LU factors resident on the
// device, chunks of a line held in registers, forward and backward substitution joined
// across chunks by segmented scans of affine maps.
//
// The middle system of a line (block tridiagonal, blocks A_b, B_b, C_b; head/tail already
// eliminated, see adi_ops.cuh) has the block LU
//     S_b = B_b - A_b G_{b-1},   G_b = S_b^{-1} C_b,
// which depends on alpha only.  It is built once per line in FP64 (precompute) and stored
// as S_b^{-1} in the path's precision, together with two transfer matrices per chunk of M
// consecutive blocks:
//     forward   y_b = S_b^{-1} r_b + F_b y_{b-1},   F_b = -S_b^{-1} A_b,   F_c = prod F_b
//     backward  x_b = y_b - G_b x_{b+1},                                   H_c = prod (-G_b)
// Per half step one thread owns one chunk: it loads the chunk's inputs and factors into
// registers, computes the chunk's local forward solution, a segmented scan over the chunks
// of the line supplies y at the chunk's start, the forward pass is redone with it, a local
// backward pass and a second (suffix) scan supply x after the chunk's end, and the final
// backward pass writes the carried outputs C = 2 u* - a (+ dt/2 f), v' = 2 v* - v.
#include <cuda_runtime.h>

#include "adi_internal.h"
#include "adi_line.cuh"
#include "adi_ops.cuh"

namespace adi {

// Chunks per line (a power of two, at most kFacMaxT) and blocks per chunk.
struct FGeom {
    int T, M;
};
constexpr int kFacMaxT = 512;
__host__ __device__ inline int fac_mmax(int method) { return method == kCFD ? 8 : 3; }
__host__ __device__ inline FGeom fgeom(int nb, int mmax) {
    int need = (nb + mmax - 1) / mmax;
    int T = 1;
    while (T < need && T < kFacMaxT) T <<= 1;
    FGeom g;
    g.T = T;
    g.M = (nb + T - 1) / T;
    return g;
}
// Words of one line's factor record: S^{-1} per block, then (F_c, H_c) per chunk; padded to
// a multiple of four words.
__host__ __device__ inline size_t fac_line_words(int method, int N) {
    LineShape s = line_shape(method, N);
    FGeom g = fgeom(s.nb, fac_mmax(method));
    size_t bs2 = (size_t)s.bs * s.bs;
    size_t w = (size_t)s.nb * bs2 + (size_t)g.T * 2 * bs2;
    return (w + 3) & ~(size_t)3;
}
bool fac_supported(int method, int N) {
    LineShape s = line_shape(method, N);
    return fgeom(s.nb, fac_mmax(method)).M <= fac_mmax(method);
}
size_t fac_words(int method, int N) { return fac_line_words(method, N); }
int fac_chunks(int method, int N) {
    LineShape s = line_shape(method, N);
    return fgeom(s.nb, fac_mmax(method)).T;
}

// ---------------------------------------------------------------------------------------
// Small block helpers.
// ---------------------------------------------------------------------------------------
template <typename T, int BS>
__device__ __forceinline__ void f_mm(const T (&X)[BS][BS], const T (&Y)[BS][BS], T (&R)[BS][BS]) {
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

// ---------------------------------------------------------------------------------------
// FP64 precompute of the factor record, one thread per line.
// ---------------------------------------------------------------------------------------
template <typename TS, int BS>
__device__ void fac_precompute_line(const LineDesc<TS> &d, TS *rec) {
    const Line<TS> L(d);
    const LineShape s = line_shape(d.method, d.N);
    const FGeom g = fgeom(s.nb, fac_mmax(d.method));
    const double rz[6] = {0, 0, 0, 0, 0, 0};
    const size_t bs2 = (size_t)BS * BS;
    TS *chunk_rec = rec + (size_t)s.nb * bs2;
    double G[BS][BS], Fp[BS][BS], Hp[BS][BS];
    for (int p = 0; p < BS; ++p)
        for (int q = 0; q < BS; ++q) { G[p][q] = 0.0; Fp[p][q] = Hp[p][q] = (p == q) ? 1.0 : 0.0; }
    for (int b = 0; b < s.nb; ++b) {
        double A[BS][BS], B[BS][BS], C[BS][BS], r[BS];
        load_block<double, TS, BS>(L, s, b, rz, rz, A, B, C, r);
        double S[BS][BS], Si[BS][BS], Gn[BS][BS], Fb[BS][BS], T1[BS][BS];
        for (int p = 0; p < BS; ++p)
            for (int q = 0; q < BS; ++q) {
                double acc = B[p][q];
                for (int k = 0; k < BS; ++k) acc -= A[p][k] * G[k][q];
                S[p][q] = acc;
            }
        mat_inv<double, BS>(S, Si);
        f_mm<double, BS>(Si, C, Gn);
        f_mm<double, BS>(Si, A, Fb);
        for (int p = 0; p < BS; ++p)
            for (int q = 0; q < BS; ++q) rec[(size_t)b * bs2 + p * BS + q] = (TS)Si[p][q];
        const int c = b / g.M, i = b % g.M;
        if (i == 0)
            for (int p = 0; p < BS; ++p)
                for (int q = 0; q < BS; ++q) Fp[p][q] = Hp[p][q] = (p == q) ? 1.0 : 0.0;
        // Fp <- (-Si A) Fp ;  Hp <- Hp (-Gn)
        f_mm<double, BS>(Fb, Fp, T1);
        for (int p = 0; p < BS; ++p)
            for (int q = 0; q < BS; ++q) Fp[p][q] = -T1[p][q];
        f_mm<double, BS>(Hp, Gn, T1);
        for (int p = 0; p < BS; ++p)
            for (int q = 0; q < BS; ++q) Hp[p][q] = -T1[p][q];
        if (i == g.M - 1 || b == s.nb - 1) {
            for (int p = 0; p < BS; ++p)
                for (int q = 0; q < BS; ++q) {
                    chunk_rec[(size_t)c * 2 * bs2 + p * BS + q] = (TS)Fp[p][q];
                    chunk_rec[(size_t)c * 2 * bs2 + bs2 + p * BS + q] = (TS)Hp[p][q];
                }
        }
        for (int p = 0; p < BS; ++p)
            for (int q = 0; q < BS; ++q) G[p][q] = Gn[p][q];
    }
    // chunks past the end of the line act as identities
    for (int c = (s.nb + g.M - 1) / g.M; c < g.T; ++c)
        for (int p = 0; p < BS; ++p)
            for (int q = 0; q < BS; ++q) {
                chunk_rec[(size_t)c * 2 * bs2 + p * BS + q] = (TS)(p == q ? 1.0 : 0.0);
                chunk_rec[(size_t)c * 2 * bs2 + bs2 + p * BS + q] = (TS)(p == q ? 1.0 : 0.0);
            }
}

template <typename TS>
__global__ void fac_precompute_kernel(const LineDesc<TS> *__restrict__ descs, int nlines) {
    int line = blockIdx.x * blockDim.x + threadIdx.x;
    if (line >= nlines) return;
    const LineDesc<TS> d = descs[line];
    if (d.method == kCFD)
        fac_precompute_line<TS, 2>(d, d.sep);
    else
        fac_precompute_line<TS, 3>(d, d.sep);
}

// ---------------------------------------------------------------------------------------
// Segmented scans of affine maps z -> m z + off over the T chunk-threads of a line.
// Lines occupy aligned groups of T consecutive threads (T a power of two).
// ---------------------------------------------------------------------------------------
template <typename T, int BS>
struct Map {
    T m[BS][BS];
    T off[BS];
};
template <typename T, int BS>
__device__ __forceinline__ void map_id(Map<T, BS> &a) {
#pragma unroll
    for (int i = 0; i < BS; ++i) {
        a.off[i] = T(0);
#pragma unroll
        for (int j = 0; j < BS; ++j) a.m[i][j] = i == j ? T(1) : T(0);
    }
}
// a <- a o b  (b first, then a)
template <typename T, int BS>
__device__ __forceinline__ void map_after(Map<T, BS> &a, const Map<T, BS> &b) {
    Map<T, BS> r;
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
template <typename T, int BS>
__device__ __forceinline__ void map_shfl(Map<T, BS> &dst, const Map<T, BS> &src, int delta, bool up,
                                         int width) {
#pragma unroll
    for (int i = 0; i < BS; ++i) {
#pragma unroll
        for (int j = 0; j < BS; ++j)
            dst.m[i][j] = up ? __shfl_up_sync(0xffffffffu, src.m[i][j], delta, width)
                             : __shfl_down_sync(0xffffffffu, src.m[i][j], delta, width);
        dst.off[i] = up ? __shfl_up_sync(0xffffffffu, src.off[i], delta, width)
                        : __shfl_down_sync(0xffffffffu, src.off[i], delta, width);
    }
}

// Inclusive scan over the chunks of a line.  forward: result(c) = a_c o ... o a_0;
// backward: result(c) = a_c o a_{c+1} o ... o a_{T-1}.  Returns the exclusive value's
// offset applied to zero, i.e. z before chunk c (forward) or after chunk c (backward).
// sm holds 32 maps (warp aggregates, then warp prefixes); all threads of the CTA must
// call it.
template <typename T, int BS>
__device__ void line_scan(Map<T, BS> a, bool forward, int Tl, T (&z)[BS], Map<T, BS> *sm) {
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int width = Tl < 32 ? Tl : 32;
    const int pos = forward ? (lane % width) : (width - 1 - lane % width);
    // warp-level (segment width <= 32) inclusive scan
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        if (s >= width) break;
        Map<T, BS> o;
        map_shfl<T, BS>(o, a, s, forward, width);
        if (pos >= s) map_after<T, BS>(a, o);
    }
    T zz[BS];
    // exclusive value within the warp segment
#pragma unroll
    for (int i = 0; i < BS; ++i) {
        T v = forward ? __shfl_up_sync(0xffffffffu, a.off[i], 1, width)
                      : __shfl_down_sync(0xffffffffu, a.off[i], 1, width);
        zz[i] = pos == 0 ? T(0) : v;
    }
    if (Tl > 32) {
        // combine the warps of a line: warp aggregates go to shared memory, the first warp of
        // each line scans them (exclusive), every warp applies its prefix
        const int wpl = Tl / 32;              // warps per line (<= 16)
        const int wl = warp % wpl;            // warp index within its line
        const int wfirst = warp - wl;
        const int last_lane = forward ? 31 : 0;
        if (lane == last_lane) sm[warp] = a;  // the warp's full composition
        __syncthreads();
        if (wl == 0) {
            // lane t < wpl holds warp aggregate t; scan across them (width = wpl)
            Map<T, BS> w;
            if (lane < wpl) w = sm[wfirst + lane]; else map_id<T, BS>(w);
            const int wpos = forward ? lane : (wpl - 1 - lane);
#pragma unroll
            for (int s2 = 1; s2 < 16; s2 <<= 1) {
                if (s2 >= wpl) break;
                Map<T, BS> o;
                map_shfl<T, BS>(o, w, s2, forward, 32);
                if (lane < wpl && wpos >= s2) map_after<T, BS>(w, o);
            }
            // exclusive prefix for warp `lane`
            Map<T, BS> ex;
            map_shfl<T, BS>(ex, w, 1, forward, 32);
            if (wpos == 0) map_id<T, BS>(ex);
            __syncwarp();
            if (lane < wpl) sm[16 + wfirst + lane] = ex;
        }
        __syncthreads();
        const Map<T, BS> pre = sm[16 + warp];
        // z = (exclusive within warp) o pre, applied to zero
        Map<T, BS> ex;
        map_shfl<T, BS>(ex, a, 1, forward, 32);
        if (pos == 0) map_id<T, BS>(ex);
        map_after<T, BS>(ex, pre);
#pragma unroll
        for (int i = 0; i < BS; ++i) zz[i] = ex.off[i];
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < BS; ++i) z[i] = zz[i];
}

// ---------------------------------------------------------------------------------------
// The kernel.  One CTA = nl lines of one simulation and direction, T threads per line,
// thread (l, c) = (tid / T, tid % T) owns blocks [c M, c M + M) of line l.
// ---------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T fsrc(const LineDesc<T> &d, int k, T srcv, bool &hit) {
    if (k != d.src_k) return T(0);
    hit = true;
    return srcv;
}

template <typename T, int BS, int MM>
__device__ void factored_body(const LineDesc<T> *__restrict__ descs, int desc0, int nl, int natural,
                              Map<T, BS> *smmaps) {
    const int tid = threadIdx.x;
    const LineDesc<T> &d0 = descs[desc0];
    const int N = d0.N;
    const LineShape s = line_shape(d0.method, N);
    const FGeom g = fgeom(s.nb, fac_mmax(d0.method));
    const int Tl = g.T, M = g.M;
    const int l = tid / Tl, c = tid % Tl;
    const bool active = l < nl;
    const LineDesc<T> &d = descs[desc0 + (active ? l : 0)];
    const int b0 = c * M;
    int n = s.nb - b0;
    n = n < 0 ? 0 : (n > M ? M : n);
    if (!active) n = 0;
    const bool has_last = active && n > 0 && b0 + n == s.nb;  // owns block nb-1
    const bool has_first = active && c == 0;                   // owns block 0
    const T ih = (T)d.inv_h, beta = (T)d.beta;
    const T *rec = d.sep;
    const size_t bs2 = (size_t)BS * BS;

    // factors of the chunk
    T Si[MM][BS][BS];
#pragma unroll
    for (int i = 0; i < MM; ++i)
#pragma unroll
        for (int p = 0; p < BS; ++p)
#pragma unroll
            for (int q = 0; q < BS; ++q)
                Si[i][p][q] = (i < n) ? rec[(size_t)(b0 + i) * bs2 + p * BS + q] : T(0);

    // inputs: right-hand sides and the alpha window of the chunk, computed once into
    // registers (32-bit indexing: a line of at most 16384 cells in a field of at most
    // 16386^2 points)
    const T *gp = d.p, *gv = d.v, *ga = d.alpha;
    const int sp = (int)d.sp, sv = (int)d.sv;
    auto P = [&](int k) -> T { return gp[k * sp]; };
    auto V = [&](int k) -> T { return gv[k * sv]; };
    auto AL = [&](int k) -> T { return ga[k * sp]; };
    constexpr int NA = (BS == 2) ? MM + 2 : 3 * MM;  // alpha window
    const int abase = (BS == 2) ? b0 + 2 : s.hu + 1 + 3 * b0;
    T aw[NA];
    T rr[MM][BS];
    {
        const int na = (BS == 2) ? n + 2 : 3 * n;
#pragma unroll
        for (int k = 0; k < NA; ++k) aw[k] = (k < na) ? AL(abase + k) : T(0);
        const T t3 = T(3) * ih;
#pragma unroll
        for (int i = 0; i < MM; ++i) {
            if (i < n) {
                if constexpr (BS == 2) {
                    const int j = b0 + i + 3;
                    rr[i][0] = t3 * (V(j + 1) - V(j - 1));
                    rr[i][1] = t3 * (P(j + 1) - P(j - 1));
                } else {
                    const T w0 = T(1.0 / 24.0), w1 = T(-9.0 / 8.0), w2 = T(9.0 / 8.0), w3 = T(-1.0 / 24.0);
#pragma unroll
                    for (int m = 0; m < 3; ++m) {
                        const int cc = abase + 3 * i + m;
                        const T dv = w0 * V(cc - 2) + w1 * V(cc - 1) + w2 * V(cc) + w3 * V(cc + 1);
                        rr[i][m] = P(cc) - aw[3 * i + m] * ih * dv;
                    }
                }
            } else {
#pragma unroll
                for (int p = 0; p < BS; ++p) rr[i][p] = T(0);
            }
        }
    }

    // boundary right-hand-side corrections (head on block 0, tail on block nb-1)
    if (has_first || has_last) {
        const Line<T> Lg(d);
        if (has_first) {
            for (int p = 0; p < BS; ++p) {
                T acc = T(0);
                for (int k = 0; k < s.hu; ++k) acc += d.tab[kTabK + p * s.hu + k] * rhs_row(Lg, k);
                rr[0][p] -= acc;
            }
        }
        if (has_last) {
            const int il = n - 1;
            for (int p = 0; p < BS; ++p) {
                T acc = T(0);
                for (int k = 0; k < s.tu; ++k)
                    acc += d.tab[kTabEnd + kTabK + p * s.tu + k] * rhs_row(Lg, s.nunk - s.tu + k);
#pragma unroll
                for (int i = 0; i < MM; ++i)
                    if (i == il) rr[i][p] -= acc;
            }
        }
    }

    // couplings of block i: A (to block i-1) and C (to block i+1), zero across the
    // eliminated head/tail
    auto blockAC = [&](int i, T (&A)[BS][BS], T (&C)[BS][BS]) {
        const int b = b0 + i;
        if constexpr (BS == 2) {
            const T t3 = T(3) * ih, tb = t3 * beta;
            A[0][0] = T(1); A[0][1] = -tb; A[1][0] = -t3 * aw[i]; A[1][1] = T(1);
            C[0][0] = T(1); C[0][1] = tb; C[1][0] = t3 * aw[i + 2]; C[1][1] = T(1);
        } else {
            const T bh2 = beta * ih * ih;
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                const T sc = aw[3 * i + m] * bh2;
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const int dA = q - m - 3, dC = q - m + 3;
                    A[m][q] = (dA >= -3) ? -sc * (T)mim_DG(dA + 3) : T(0);
                    C[m][q] = (dC <= 3) ? -sc * (T)mim_DG(dC + 3) : T(0);
                }
            }
        }
        if (b == 0)
#pragma unroll
            for (int p = 0; p < BS; ++p)
#pragma unroll
                for (int q = 0; q < BS; ++q) A[p][q] = T(0);
        if (b == s.nb - 1)
#pragma unroll
            for (int p = 0; p < BS; ++p)
#pragma unroll
                for (int q = 0; q < BS; ++q) C[p][q] = T(0);
    };
    // y <- S^{-1}_i (r_i - A y)
    auto fstep = [&](int i, T (&y)[BS]) {
        T A[BS][BS], C[BS][BS], t[BS];
        blockAC(i, A, C);
#pragma unroll
        for (int p = 0; p < BS; ++p) {
            T acc = rr[i][p];
#pragma unroll
            for (int q = 0; q < BS; ++q) acc -= A[p][q] * y[q];
            t[p] = acc;
        }
#pragma unroll
        for (int p = 0; p < BS; ++p) {
            T acc = T(0);
#pragma unroll
            for (int q = 0; q < BS; ++q) acc += Si[i][p][q] * t[q];
            y[p] = acc;
        }
    };
    // x <- y_i - S^{-1}_i (C x)
    auto bstep = [&](int i, const T (&y)[BS], T (&x)[BS]) {
        T A[BS][BS], C[BS][BS], t[BS];
        blockAC(i, A, C);
#pragma unroll
        for (int p = 0; p < BS; ++p) {
            T acc = T(0);
#pragma unroll
            for (int q = 0; q < BS; ++q) acc += C[p][q] * x[q];
            t[p] = acc;
        }
#pragma unroll
        for (int p = 0; p < BS; ++p) {
            T acc = y[p];
#pragma unroll
            for (int q = 0; q < BS; ++q) acc -= Si[i][p][q] * t[q];
            x[p] = acc;
        }
    };

    // ---- forward: local pass, scan, true pass ----
    T y[BS];
#pragma unroll
    for (int p = 0; p < BS; ++p) y[p] = T(0);
#pragma unroll
    for (int i = 0; i < MM; ++i)
        if (i < n) fstep(i, y);
    Map<T, BS> mp;
    {
        const T *cr = rec + (size_t)s.nb * bs2 + (size_t)c * 2 * bs2;
#pragma unroll
        for (int p = 0; p < BS; ++p) {
            mp.off[p] = y[p];
#pragma unroll
            for (int q = 0; q < BS; ++q) mp.m[p][q] = active ? cr[p * BS + q] : (p == q ? T(1) : T(0));
        }
    }
    T yin[BS];
    line_scan<T, BS>(mp, true, Tl, yin, smmaps);
    T Y[MM][BS];
#pragma unroll
    for (int p = 0; p < BS; ++p) y[p] = yin[p];
#pragma unroll
    for (int i = 0; i < MM; ++i)
        if (i < n) {
            fstep(i, y);
#pragma unroll
            for (int p = 0; p < BS; ++p) Y[i][p] = y[p];
        }

    // ---- backward: local pass, suffix scan, true pass ----
    T x[BS];
#pragma unroll
    for (int p = 0; p < BS; ++p) x[p] = T(0);
#pragma unroll
    for (int i = MM - 1; i >= 0; --i)
        if (i < n) bstep(i, Y[i], x);
    {
        const T *cr = rec + (size_t)s.nb * bs2 + (size_t)c * 2 * bs2 + bs2;
#pragma unroll
        for (int p = 0; p < BS; ++p) {
            mp.off[p] = x[p];
#pragma unroll
            for (int q = 0; q < BS; ++q) mp.m[p][q] = active ? cr[p * BS + q] : (p == q ? T(1) : T(0));
        }
    }
    T xin[BS];
    line_scan<T, BS>(mp, false, Tl, xin, smmaps);
    if (!active) return;

    // ---- true backward pass with outputs ----
    T srcv = T(0);
    bool hit = false;
    if (d.src_k >= 0) {
        long long m = *d.clock;
        srcv = (T)(d.src_scale * ricker(d.src_amp, d.src_f0, d.src_tdelay, (double)(m + 1) * d.dt));
    }
    const bool nat = natural && d.u_out != nullptr;
    T *gpo = d.po, *gvo = d.vo;
    const int spo = (int)d.spo, svo = (int)d.svo;
    auto out_p = [&](int k, T val_out, T val_nat) {
        gpo[k * spo] = val_out + fsrc(d, k, srcv, hit);
        if (nat) d.u_out[k * (int)d.snp] = val_nat;
    };
    auto out_v = [&](int j, T vin, T dv) {  // dv = beta * (D_u u*)_j
        gvo[j * svo] = vin - T(2) * dv;
        if (nat) d.w_out[j * (int)d.snv] = vin - dv;
    };
    T xn[BS];
#pragma unroll
    for (int p = 0; p < BS; ++p) { xn[p] = xin[p]; x[p] = xin[p]; }
    T X0[BS];
#pragma unroll
    for (int p = 0; p < BS; ++p) X0[p] = T(0);
#pragma unroll
    for (int i = MM - 1; i >= 0; --i) {
        if (i < n) {
#pragma unroll
            for (int p = 0; p < BS; ++p) xn[p] = x[p];
            bstep(i, Y[i], x);
            const int b = b0 + i;
            if constexpr (BS == 2) {
                const int j = b + 3;
                const T pin = P(j);
                const T ae = AL(j) * x[0];
                out_p(j, pin - T(2) * ae, pin - ae);
                out_v(j, V(j), beta * x[1]);
            } else {
                const int q0 = s.hu + 1 + 3 * b;
#pragma unroll
                for (int m = 0; m < 3; ++m) out_p(q0 + m, T(2) * x[m] - P(q0 + m), x[m]);
                if (b != s.nb - 1) {
                    // nodes q0+1..q0+3 from this block's cells and the next block's
                    const T w0 = T(1.0 / 24.0), w1 = T(-9.0 / 8.0), w2 = T(9.0 / 8.0), w3 = T(-1.0 / 24.0);
                    const T bi = beta * ih;
                    out_v(q0 + 1, V(q0 + 1), bi * (w0 * x[0] + w1 * x[1] + w2 * x[2] + w3 * xn[0]));
                    out_v(q0 + 2, V(q0 + 2), bi * (w0 * x[1] + w1 * x[2] + w2 * xn[0] + w3 * xn[1]));
                    out_v(q0 + 3, V(q0 + 3), bi * (w0 * x[2] + w1 * xn[0] + w2 * xn[1] + w3 * xn[2]));
                }
            }
            if (b == s.nb - 1) {  // tail unknowns
                const T *tt = d.tab + kTabEnd;
                const Line<T> Lg(d);
                T rT[6], xt[6];
                for (int kk = 0; kk < s.tu; ++kk) rT[kk] = rhs_row(Lg, s.nunk - s.tu + kk);
                for (int t2 = 0; t2 < s.tu; ++t2) {
                    T acc = T(0);
                    for (int kk = 0; kk < s.tu; ++kk) acc += tt[kTabHinv + t2 * s.tu + kk] * rT[kk];
#pragma unroll
                    for (int kk = 0; kk < BS; ++kk) acc -= tt[kTabHinvE + t2 * BS + kk] * x[kk];
                    xt[t2] = acc;
                }
                if constexpr (BS == 2) {
                    // e_{N-2}, g_{N-2}, e_{N-1}, g_{N-1}, g_N
                    const int jn = N - 2;
                    for (int q = 0; q < 2; ++q) {
                        const int j = jn + q;
                        const T pin = d.p[(long long)j * d.sp], vin = d.v[(long long)j * d.sv];
                        const T ae = d.alpha[(long long)j * d.sp] * xt[2 * q];
                        out_p(j, pin - T(2) * ae, pin - ae);
                        out_v(j, vin, beta * xt[2 * q + 1]);
                    }
                    out_v(N, d.v[(long long)N * d.sv], beta * xt[4]);
                } else {
                    // tail cells q0+3 .. N, then nodes q0+1 .. N from the window
                    const int qb = s.hu + 1 + 3 * b;  // first cell of the last block
                    T cells[8];
                    cells[0] = x[0]; cells[1] = x[1]; cells[2] = x[2];
                    for (int t2 = 0; t2 < s.tu; ++t2) {
                        cells[3 + t2] = xt[t2];
                        const int cc = qb + 3 + t2;
                        const T pin = d.p[(long long)cc * d.sp];
                        out_p(cc, T(2) * xt[t2] - pin, xt[t2]);
                    }
                    const T p0 = d.p[0], pl = d.p[(long long)(N + 1) * d.sp];
                    for (int j = qb + 1; j <= N; ++j) {
                        double gw[8];
                        int g0;
                        int ng = mfd_G_row(N, j, &g0, gw);
                        T acc = T(0);
                        for (int t2 = 0; t2 < ng; ++t2) {
                            int kk = g0 + t2;
                            acc += (T)gw[t2] * ((kk == 0) ? p0 : (kk == N + 1 ? pl : cells[kk - qb]));
                        }
                        out_v(j, d.v[(long long)j * d.sv], beta * ih * acc);
                    }
                }
            }
            if (i == 0)
#pragma unroll
                for (int p = 0; p < BS; ++p) X0[p] = x[p];
        }
    }
    if (has_first) {  // head unknowns from block 0
        const T *th = d.tab;
        const Line<T> Lg(d);
        T rH[6], xh[6];
        for (int kk = 0; kk < s.hu; ++kk) rH[kk] = rhs_row(Lg, kk);
        for (int t2 = 0; t2 < s.hu; ++t2) {
            T acc = T(0);
            for (int kk = 0; kk < s.hu; ++kk) acc += th[kTabHinv + t2 * s.hu + kk] * rH[kk];
#pragma unroll
            for (int kk = 0; kk < BS; ++kk) acc -= th[kTabHinvE + t2 * BS + kk] * X0[kk];
            xh[t2] = acc;
        }
        if constexpr (BS == 2) {
            // g0, e1, g1, e2, g2
            out_v(0, d.v[0], beta * xh[0]);
            for (int q = 0; q < 2; ++q) {
                const int j = 1 + q;
                const T pin = d.p[(long long)j * d.sp], vin = d.v[(long long)j * d.sv];
                const T ae = d.alpha[(long long)j * d.sp] * xh[1 + 2 * q];
                out_p(j, pin - T(2) * ae, pin - ae);
                out_v(j, vin, beta * xh[2 + 2 * q]);
            }
        } else {
            T cells[12];
            cells[0] = d.p[0];
            for (int t2 = 0; t2 < s.hu; ++t2) {
                cells[1 + t2] = xh[t2];
                const T pin = d.p[(long long)(1 + t2) * d.sp];
                out_p(1 + t2, T(2) * xh[t2] - pin, xh[t2]);
            }
            cells[s.hu + 1] = X0[0]; cells[s.hu + 2] = X0[1]; cells[s.hu + 3] = X0[2];
            for (int j = 0; j <= s.hu + 1; ++j) {
                double gw[8];
                int g0;
                int ng = mfd_G_row(N, j, &g0, gw);
                T acc = T(0);
                for (int t2 = 0; t2 < ng; ++t2) acc += (T)gw[t2] * cells[g0 + t2];
                out_v(j, d.v[(long long)j * d.sv], beta * ih * acc);
            }
        }
    }
    if (hit && d.advance_clock) *d.clock = *d.clock + 1;
}

template <typename T, int BS, int MM>
__global__ void __launch_bounds__(512, 1)
line_solve_factored_kernel(const LineDesc<T> *__restrict__ descs, const int4 *__restrict__ groups,
                           int natural) {
    __shared__ Map<T, BS> smmaps[32];
    const int4 gr = groups[blockIdx.x];
    factored_body<T, BS, MM>(descs, gr.x, gr.y, natural, smmaps);
}

template <typename T>
cudaError_t launch_fac_precompute(const LineDesc<T> *d, int nlines, cudaStream_t s) {
    if (nlines <= 0) return cudaSuccess;
    fac_precompute_kernel<T><<<(nlines + 63) / 64, 64, 0, s>>>(d, nlines);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_line_solve_factored(const LineDesc<T> *d, const int4 *groups, int ngroups,
                                       int method, int threads, int natural, cudaStream_t s) {
    if (ngroups <= 0) return cudaSuccess;
    if (method == kCFD)
        line_solve_factored_kernel<T, 2, 8><<<ngroups, threads, 0, s>>>(d, groups, natural);
    else
        line_solve_factored_kernel<T, 3, 3><<<ngroups, threads, 0, s>>>(d, groups, natural);
    return cudaGetLastError();
}

template cudaError_t launch_fac_precompute<float>(const LineDesc<float> *, int, cudaStream_t);
template cudaError_t launch_fac_precompute<double>(const LineDesc<double> *, int, cudaStream_t);
template cudaError_t launch_line_solve_factored<float>(const LineDesc<float> *, const int4 *, int, int,
                                                       int, int, cudaStream_t);
template cudaError_t launch_line_solve_factored<double>(const LineDesc<double> *, const int4 *, int,
                                                        int, int, int, cudaStream_t);

}  // namespace adi
