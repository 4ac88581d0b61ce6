// adi_factored.cu -- the factored line solver: persistent CTAs, line inputs staged in shared
// memory by bulk asynchronous copies (a two-stage ring, the next line group in flight while
// the current one is solved), chunks of a line in registers, chunks joined by segmented scans
// of affine maps.
//
// The middle system of a line (block tridiagonal, blocks A_b, B_b, C_b; head/tail already
// eliminated, see adi_ops.cuh) has the block LU
//     S_b = B_b - A_b G_{b-1},   G_b = S_b^{-1} C_b .
// One thread owns a chunk of M consecutive blocks.  The FP64 precompute stores per chunk
// only what the chunk cannot rebuild from its own data:
//     S_{b0}   the Schur complement at the chunk's first block,
//     F_c      prod over the chunk of F_b = -S_b^{-1} A_b   (forward transfer),
//     H_c      prod over the chunk of -G_b                   (backward transfer).
// Per half step a thread rebuilds S_b^{-1} of its blocks from S_{b0} and the alpha values
// on the line (one block recurrence in the path's precision), then
//     forward  y_b = S_b^{-1}(r_b - A_b y_{b-1})   local pass from y = 0,
//              scan of (F_c, y_end) over the chunks -> the true y entering the chunk,
//              correction y_b += delta_b, delta_b = F_b delta_{b-1};
//     backward x_b = y_b - G_b x_{b+1}             local pass from x = 0,
//              suffix scan of (H_c, x_start) -> the true x after the chunk,
//              correction x_b += eps_b, eps_b = -G_b eps_{b+1};
// and writes the carried outputs C = 2 u* - a (+ dt/2 f), v' = 2 v* - v.
#include <cuda_runtime.h>

#include "adi_internal.h"
#include "adi_line.cuh"
#include "adi_ops.cuh"

namespace adi {

constexpr int kFacThreads = 512;              // threads per CTA
constexpr int kFacMaxT = 512;                 // chunks (threads) per line at most
constexpr size_t kFacSmemLimit = 227 * 1024;  // shared memory per CTA
constexpr size_t kFacStaticSmem = 4096;       // reserve for the kernel's static shared memory

// Chunks per line (a power of two, at most kFacMaxT) and blocks per chunk.
struct FGeom {
    int T, M;
};
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
// Elements of one staged line array (pressure, velocity or alpha), a multiple of four.
__host__ __device__ inline int fac_lp(int N) { return (N + 2 + 3) & ~3; }
// End tables: the head/tail eliminations and outputs as linear maps of
//   z = [p window (8), v window (8), x of the adjacent middle block (BS)],
// windows p[0..7], v[0..7] at the head and p[L-7..L], v[N-7..N] at the tail.  Per end:
//   KZ [3][16]  correction of the adjacent block's right-hand side (-K W),
//   HZ [6][19]  the eliminated unknowns (Hinv W | -Hinv E),
//   DZ [8][19]  MFD: h (G u) at the end's velocity nodes,
//   dB [3][3]   diagonal-block correction of the adjacent block.
constexpr int kEndKZ = 0, kEndHZ = 48, kEndDZ = 162, kEndDB = 314;
constexpr int kEndStride = 324, kEndTable = 2 * kEndStride;
// Elements of one line's chunk record: S_b0, F_c, H_c as three arrays of T BSxBS blocks,
// then the two end tables.
__host__ __device__ inline int fac_chunk_elems(int bs, int T) { return (3 * T * bs * bs + 3) & ~3; }
__host__ __device__ inline int fac_rec(int bs, int T) { return fac_chunk_elems(bs, T) + kEndTable; }
__host__ __device__ inline FGeom fac_geom(int method, int N) {
    return fgeom(line_shape(method, N).nb, fac_mmax(method));
}
__host__ __device__ inline int fac_line_elems(int method, int N) {
    LineShape s = line_shape(method, N);
    return 3 * fac_lp(N) + fac_rec(s.bs, fac_geom(method, N).T);
}

// One stage: the group's descriptors, then per line [p | v | alpha | record].
constexpr size_t kDescBytes = sizeof(LineDesc<float>);
static_assert(sizeof(LineDesc<float>) == sizeof(LineDesc<double>), "descriptor sizes differ");
static_assert(kDescBytes % 16 == 0, "descriptor size");
__host__ __device__ inline size_t fac_desc_area(int nl) { return ((size_t)nl * kDescBytes + 127) & ~(size_t)127; }
size_t fac_stage_bytes(int method, int N, int nl, size_t esz) {
    size_t b = fac_desc_area(nl) + (size_t)nl * fac_line_elems(method, N) * esz;
    return (b + 127) & ~(size_t)127;
}
int fac_stages_for(size_t stage_bytes) {
    if (2 * stage_bytes + kFacStaticSmem <= kFacSmemLimit) return 2;
    if (stage_bytes + kFacStaticSmem <= kFacSmemLimit) return 1;
    return 0;
}
// Lines per CTA: as many as the CTA's threads cover, fewer where a two-stage ring of them
// would not fit shared memory.
int fac_lines_per_cta(int method, int N, size_t esz) {
    int T = fac_geom(method, N).T;
    int nl = T >= kFacThreads ? 1 : kFacThreads / T;
    while (nl > 1 && fac_stages_for(fac_stage_bytes(method, N, nl, esz)) < 2) --nl;
    return nl;
}
bool fac_supported(int method, int N, size_t esz) {
    if (fac_geom(method, N).M > fac_mmax(method)) return false;
    return fac_stages_for(fac_stage_bytes(method, N, 1, esz)) > 0;
}
size_t fac_words(int method, int N) {
    return (size_t)fac_rec(line_shape(method, N).bs, fac_geom(method, N).T);
}
int fac_chunks(int method, int N) { return fac_geom(method, N).T; }

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
// FP64 precompute of the chunk records, one thread per line.
// ---------------------------------------------------------------------------------------
template <typename TS, int BS>
__device__ void fac_precompute_line(const LineDesc<TS> &d, TS *rec) {
    const Line<TS> L(d);
    const LineShape s = line_shape(d.method, d.N);
    const FGeom g = fgeom(s.nb, fac_mmax(d.method));
    const double rz[6] = {0, 0, 0, 0, 0, 0};
    constexpr int B2 = BS * BS;
    TS *recS = rec, *recF = rec + (size_t)g.T * B2, *recH = rec + (size_t)2 * g.T * B2;
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
        const int c = b / g.M, i = b % g.M;
        if (i == 0) {
            for (int p = 0; p < BS; ++p)
                for (int q = 0; q < BS; ++q) {
                    recS[(size_t)c * B2 + p * BS + q] = (TS)S[p][q];
                    Fp[p][q] = Hp[p][q] = (p == q) ? 1.0 : 0.0;
                }
        }
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
                    recF[(size_t)c * B2 + p * BS + q] = (TS)Fp[p][q];
                    recH[(size_t)c * B2 + p * BS + q] = (TS)Hp[p][q];
                }
        }
        for (int p = 0; p < BS; ++p)
            for (int q = 0; q < BS; ++q) G[p][q] = Gn[p][q];
    }
    // chunks past the end of the line act as identities
    for (int c = (s.nb + g.M - 1) / g.M; c < g.T; ++c)
        for (int p = 0; p < BS; ++p)
            for (int q = 0; q < BS; ++q) {
                const TS e = (TS)(p == q ? 1.0 : 0.0);
                recS[(size_t)c * B2 + p * BS + q] = e;
                recF[(size_t)c * B2 + p * BS + q] = e;
                recH[(size_t)c * B2 + p * BS + q] = e;
            }
}

// Right-hand side of head/tail row i as coefficients on the windows p[op..op+7] and
// v[ov..ov+7] (the same sums rhs_row evaluates).  False if a term falls outside.
template <typename TS>
__device__ bool rhs_coeffs(const LineDesc<TS> &d, int i, int op, int ov, double (&cp)[8], double (&cv)[8]) {
    for (int k = 0; k < 8; ++k) cp[k] = cv[k] = 0.0;
    const int N = d.N;
    const double ih = d.inv_h;
    bool ok = true;
    auto add = [&](double (&w8)[8], int idx, double val) {
        if (idx < 0 || idx >= 8) ok = false; else w8[idx] += val;
    };
    double w[8];
    int c0, n;
    if (d.method == kCFD) {
        const bool is_g = (i == 0) || (i == 2 * N - 1) || (i % 2 == 0);
        const int node = i == 0 ? 0 : (i == 2 * N - 1 ? N : (i + 1) / 2);
        if (is_g) {
            n = cfd_Q_row(N, node, &c0, w);
            for (int t = 0; t < n; ++t) add(cp, c0 + t - op, w[t] * ih);
        } else {
            n = cfd_Qbar_row(N, node, &c0, w);
            for (int t = 0; t < n; ++t) add(cv, c0 + t - ov, w[t] * ih);
        }
        return ok;
    }
    // r_c = p_c - alpha_c/h sum_j D[c-1][j] (v_j - beta/h (G[j][0] p_0 + G[j][N+1] p_L))
    const int c = i + 1;
    const double a = (double)d.alpha[(long long)c * d.sp], bh = d.beta * ih;
    add(cp, c - op, 1.0);
    n = mfd_D_row(N, c - 1, &c0, w);
    for (int t = 0; t < n; ++t) {
        const int node = c0 + t;
        const double coef = -a * ih * w[t];
        add(cv, node - ov, coef);
        if (node <= 1 || node >= N - 1) {
            double gw[8];
            int g0;
            const int ng = mfd_G_row(N, node, &g0, gw);
            if (g0 == 0) add(cp, 0 - op, -coef * bh * gw[0]);
            if (g0 + ng - 1 == N + 1) add(cp, N + 1 - op, -coef * bh * gw[ng - 1]);
        }
    }
    return ok;
}

// The two end tables of a line (see kEnd*), from the head/tail elimination tables.
template <typename TS, int BS>
__device__ void fac_end_tables(const LineDesc<TS> &d, TS *et) {
    const int N = d.N;
    const LineShape s = line_shape(d.method, N);
    const int pl = p_last(d.method, N);
    const double nan = __longlong_as_double(0x7ff8000000000000ULL);
    for (int end = 0; end < 2; ++end) {
        TS *e = et + end * kEndStride;
        const TS *t = d.tab + end * kTabEnd;
        const int m = end == 0 ? s.hu : s.tu;
        const int r0 = end == 0 ? 0 : s.nunk - s.tu;
        const int op = end == 0 ? 0 : pl - 7, ov = end == 0 ? 0 : N - 7;
        double W[6][16];
        bool ok = true;
        for (int k = 0; k < m; ++k) {
            double cp[8], cv[8];
            ok = rhs_coeffs(d, r0 + k, op, ov, cp, cv) && ok;
            for (int j = 0; j < 8; ++j) { W[k][j] = cp[j]; W[k][8 + j] = cv[j]; }
        }
        for (int i = 0; i < kEndStride; ++i) e[i] = (TS)0;
        for (int p = 0; p < BS; ++p)
            for (int j = 0; j < 16; ++j) {
                double acc = 0.0;
                for (int k = 0; k < m; ++k) acc -= (double)t[kTabK + p * m + k] * W[k][j];
                e[kEndKZ + p * 16 + j] = (TS)(ok ? acc : nan);
            }
        double HZ[6][19];
        for (int q = 0; q < m; ++q) {
            for (int j = 0; j < 16; ++j) {
                double acc = 0.0;
                for (int k = 0; k < m; ++k) acc += (double)t[kTabHinv + q * m + k] * W[k][j];
                HZ[q][j] = acc;
            }
            for (int b = 0; b < 3; ++b) HZ[q][16 + b] = b < BS ? -(double)t[kTabHinvE + q * BS + b] : 0.0;
            for (int j = 0; j < 19; ++j) e[kEndHZ + q * 19 + j] = (TS)(ok ? HZ[q][j] : nan);
        }
        for (int p = 0; p < BS; ++p)
            for (int q = 0; q < BS; ++q) e[kEndDB + p * 3 + q] = t[kTabDB + p * BS + q];
        if (d.method != kMFD) continue;
        // MFD: h (G u)_j at the end's nodes, cells expressed through z
        const int qb = s.hu + 1 + 3 * (s.nb - 1);  // first cell of the last middle block
        const int j0 = end == 0 ? 0 : qb + 1, j1 = end == 0 ? s.hu + 1 : N;
        for (int j = j0; j <= j1; ++j) {
            double row[19];
            for (int k = 0; k < 19; ++k) row[k] = 0.0;
            double gw[8];
            int g0;
            const int ng = mfd_G_row(N, j, &g0, gw);
            bool rok = ok;
            for (int tt = 0; tt < ng; ++tt) {
                const int cc = g0 + tt;
                if (end == 0) {
                    if (cc == 0) row[0] += gw[tt];
                    else if (cc <= s.hu) for (int k = 0; k < 19; ++k) row[k] += gw[tt] * HZ[cc - 1][k];
                    else if (cc <= s.hu + 3) row[16 + cc - s.hu - 1] += gw[tt];
                    else rok = false;
                } else {
                    if (cc == N + 1) row[N + 1 - op] += gw[tt];
                    else if (cc >= qb + 3) for (int k = 0; k < 19; ++k) row[k] += gw[tt] * HZ[cc - qb - 3][k];
                    else if (cc >= qb) row[16 + cc - qb] += gw[tt];
                    else rok = false;
                }
            }
            for (int k = 0; k < 19; ++k) e[kEndDZ + (j - j0) * 19 + k] = (TS)(rok ? row[k] : nan);
        }
    }
}

template <typename TS>
__global__ void fac_precompute_kernel(const LineDesc<TS> *__restrict__ descs, int nlines) {
    int line = blockIdx.x * blockDim.x + threadIdx.x;
    if (line >= nlines) return;
    const LineDesc<TS> d = descs[line];
    const LineShape s = line_shape(d.method, d.N);
    TS *et = d.sep + fac_chunk_elems(s.bs, fac_geom(d.method, d.N).T);
    if (d.method == kCFD) {
        fac_precompute_line<TS, 2>(d, d.sep);
        fac_end_tables<TS, 2>(d, et);
    } else {
        fac_precompute_line<TS, 3>(d, d.sep);
        fac_end_tables<TS, 3>(d, et);
    }
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
// Bulk asynchronous copies (global -> shared) completing on an mbarrier.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_to_smem(void *dst, const void *src, unsigned bytes,
                                             unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Waits for the phase with the given parity; gives up after a bounded number of polls
// (each poll may suspend the thread for a short hardware-defined time).
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity) {
    for (int i = 0; i < (1 << 22); ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__host__ __device__ inline unsigned round16(unsigned b) { return (b + 15u) & ~15u; }

// Thread 0: stage the inputs of one line group (pressure, velocity and alpha lines and the
// chunk records) into shared memory.  Every source line starts on a 16-byte boundary (the
// carried arrays have padded leading dimensions) and the copies, rounded up to 16 bytes,
// stay inside the padded line.
template <typename T>
__device__ void fac_issue(const LineDesc<T> *__restrict__ descs, int4 gr, unsigned char *stage,
                          unsigned long long *bar) {
    const LineDesc<T> &d0 = descs[gr.x];
    const int N = d0.N, method = d0.method;
    const LineShape s = line_shape(method, N);
    const FGeom g = fgeom(s.nb, fac_mmax(method));
    const int Lp = fac_lp(N), R = fac_rec(s.bs, g.T);
    const unsigned bp = round16((unsigned)(p_last(method, N) + 1) * (unsigned)sizeof(T));
    const unsigned bv = round16((unsigned)(N + 1) * (unsigned)sizeof(T));
    const unsigned br = (unsigned)R * (unsigned)sizeof(T);
    const unsigned bd = (unsigned)(gr.y * kDescBytes);
    mbar_expect_tx(bar, bd + (unsigned)gr.y * (2 * bp + bv + br));
    bulk_to_smem(stage, descs + gr.x, bd, bar);
    T *base = (T *)(stage + fac_desc_area(gr.y));
    for (int l = 0; l < gr.y; ++l) {
        const LineDesc<T> &d = descs[gr.x + l];
        T *ln = base + (size_t)l * (3 * Lp + R);
        bulk_to_smem(ln, d.p, bp, bar);
        bulk_to_smem(ln + Lp, d.v, bv, bar);
        bulk_to_smem(ln + 2 * Lp, d.alpha, bp, bar);
        bulk_to_smem(ln + 3 * Lp, d.sep, br, bar);
    }
}

// W consecutive elements of shared memory into registers: 16-byte loads where src is
// 16-byte aligned, element loads otherwise.
template <typename T, int W>
__device__ __forceinline__ void load_window(const T *src, T (&w)[W]) {
    constexpr int per = 16 / (int)sizeof(T);
    static_assert(W % per == 0, "window");
    if ((smem_addr(src) & 15u) == 0) {
#pragma unroll
        for (int k = 0; k < W; k += per) {
            const uint4 q = *reinterpret_cast<const uint4 *>(src + k);
            const T *e = reinterpret_cast<const T *>(&q);
#pragma unroll
            for (int j = 0; j < per; ++j) w[k + j] = e[j];
        }
    } else {
#pragma unroll
        for (int k = 0; k < W; ++k) w[k] = src[k];
    }
}

// ---------------------------------------------------------------------------------------
// One line group from its staged inputs.  nl lines of one simulation and direction, T
// threads per line; thread (l, c) = (tid / T, tid % T) owns blocks [c M, c M + M) of line l.
// ---------------------------------------------------------------------------------------
template <typename T, int BS, int MM>
__device__ __forceinline__ void fac_group(int4 gr, const unsigned char *stage_raw, int natural,
                                          Map<T, BS> *smmaps) {
    constexpr int B2 = BS * BS;
    const int tid = threadIdx.x;
    const LineDesc<T> *descs = (const LineDesc<T> *)stage_raw;  // staged descriptors
    const T *stage = (const T *)(stage_raw + fac_desc_area(gr.y));
    const LineDesc<T> &d0 = descs[0];
    const int N = d0.N;
    const LineShape s = line_shape(d0.method, N);
    const FGeom g = fgeom(s.nb, fac_mmax(d0.method));
    const int Tl = g.T, M = g.M;
    const int Lp = fac_lp(N), R = fac_rec(BS, Tl);
    const int l = tid / Tl, c = tid % Tl;
    const bool active = l < gr.y;
    const LineDesc<T> &d = descs[active ? l : 0];
    const T *sP = stage + (size_t)(active ? l : 0) * (3 * Lp + R);
    const T *sV = sP + Lp, *sA = sP + 2 * Lp, *sR = sP + 3 * Lp;
    const T *eH = sR + fac_chunk_elems(BS, Tl), *eT = eH + kEndStride;  // end tables
    const int pl = p_last(d0.method, N);
    const int b0 = c * M;
    int n = s.nb - b0;
    n = n < 0 ? 0 : (n > M ? M : n);
    if (!active) n = 0;
    const bool has_first = active && c == 0;                   // owns block 0
    const bool has_last = active && n > 0 && b0 + n == s.nb;  // owns block nb-1
    const T ih = (T)d.inv_h, beta = (T)d.beta;

    // ---- alpha window and right-hand sides (from shared memory) ----
    constexpr int NA = (BS == 2) ? MM + 2 : 3 * MM;
    T aw[NA];     // CFD: 3 alpha / h at nodes b0+2 ..;  MFD: alpha at the chunk's cells
    T Y[MM][BS];  // r, then y, then x
    const int cb = s.hu + 1 + 3 * b0;  // MFD: first cell of the chunk
    if constexpr (BS == 2) {
        // windows s[b0 .. b0+MM+3] (the reads stay inside the stage buffer)
        static_assert(MM % 4 == 0, "CFD window length");
        const T c3 = T(3) * ih;
        // node j = b0 + i + 3 is window index i + 3
        {
            T w[MM + 4];
#pragma unroll
            for (int k = 0; k < MM + 4; ++k) w[k] = T(0);
            if (n > 0) load_window<T, MM + 4>(sA + b0, w);
#pragma unroll
            for (int k = 0; k < NA; ++k) aw[k] = (k < n + 2) ? c3 * w[k + 2] : T(0);
        }
        {
            T w[MM + 4];
#pragma unroll
            for (int k = 0; k < MM + 4; ++k) w[k] = T(0);
            if (n > 0) load_window<T, MM + 4>(sV + b0, w);
#pragma unroll
            for (int i = 0; i < MM; ++i) Y[i][0] = (i < n) ? c3 * (w[i + 4] - w[i + 2]) : T(0);
        }
        {
            T w[MM + 4];
#pragma unroll
            for (int k = 0; k < MM + 4; ++k) w[k] = T(0);
            if (n > 0) load_window<T, MM + 4>(sP + b0, w);
#pragma unroll
            for (int i = 0; i < MM; ++i) Y[i][1] = (i < n) ? c3 * (w[i + 4] - w[i + 2]) : T(0);
        }
    } else {
        const int na = 3 * n;
#pragma unroll
        for (int k = 0; k < NA; ++k) aw[k] = (k < na) ? sA[cb + k] : T(0);
#pragma unroll
        for (int i = 0; i < MM; ++i) {
            if (i < n) {
                {
                    const T w0 = T(1.0 / 24.0), w1 = T(-9.0 / 8.0), w2 = T(9.0 / 8.0), w3 = T(-1.0 / 24.0);
#pragma unroll
                    for (int m = 0; m < 3; ++m) {
                        const int cc = cb + 3 * i + m;
                        const T dv = w0 * sV[cc - 2] + w1 * sV[cc - 1] + w2 * sV[cc] + w3 * sV[cc + 1];
                        Y[i][m] = sP[cc] - aw[3 * i + m] * ih * dv;
                    }
                }
            } else {
#pragma unroll
                for (int p = 0; p < BS; ++p) Y[i][p] = T(0);
            }
        }
    }
    // end windows z = [p window, v window, x of the adjacent block] (x filled later)
    auto end_window = [&](bool tail, T (&z)[19]) {
        const int op = tail ? pl - 7 : 0, ov = tail ? N - 7 : 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) { z[k] = sP[op + k]; z[8 + k] = sV[ov + k]; }
#pragma unroll
        for (int k = 16; k < 19; ++k) z[k] = T(0);
    };
    if (has_first) {  // head elimination: r_0 += KZ_head z
        T z[19];
        end_window(false, z);
#pragma unroll
        for (int p = 0; p < BS; ++p) {
            T acc = T(0);
#pragma unroll
            for (int k = 0; k < 16; ++k) acc += eH[kEndKZ + p * 16 + k] * z[k];
            Y[0][p] += acc;
        }
    }
    if (has_last) {  // tail elimination: r_{nb-1} += KZ_tail z
        T z[19];
        end_window(true, z);
        const int il = n - 1;
#pragma unroll
        for (int p = 0; p < BS; ++p) {
            T acc = T(0);
#pragma unroll
            for (int k = 0; k < 16; ++k) acc += eT[kEndKZ + p * 16 + k] * z[k];
#pragma unroll
            for (int i = 0; i < MM; ++i)
                if (i == il) Y[i][p] += acc;
        }
    }

    // ---- block couplings from the alpha window ----
    // A_i (to block i-1), B_i (diagonal, without the head/tail corrections), C_i (to i+1).
    auto blockA = [&](int i, T (&A)[BS][BS]) {
        if constexpr (BS == 2) {
            const T tb = T(3) * ih * beta;
            A[0][0] = T(1); A[0][1] = -tb; A[1][0] = -aw[i]; A[1][1] = T(1);
        } else {
            const T bh2 = beta * ih * ih;
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                const T sc = aw[3 * i + m] * bh2;
#pragma unroll
                for (int q = 0; q < 3; ++q) A[m][q] = (q >= m) ? -sc * (T)mim_DG(q - m) : T(0);
            }
        }
    };
    auto blockC = [&](int i, T (&C)[BS][BS]) {
        if constexpr (BS == 2) {
            const T tb = T(3) * ih * beta;
            C[0][0] = T(1); C[0][1] = tb; C[1][0] = aw[i + 2]; C[1][1] = T(1);
        } else {
            const T bh2 = beta * ih * ih;
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                const T sc = aw[3 * i + m] * bh2;
#pragma unroll
                for (int q = 0; q < 3; ++q) C[m][q] = (q <= m) ? -sc * (T)mim_DG(q - m + 6) : T(0);
            }
        }
    };
    auto blockB = [&](int i, T (&B)[BS][BS]) {
        if constexpr (BS == 2) {
            B[0][0] = T(4); B[0][1] = T(0); B[1][0] = T(0); B[1][1] = T(4);
        } else {
            const T bh2 = beta * ih * ih;
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                const T sc = aw[3 * i + m] * bh2;
#pragma unroll
                for (int q = 0; q < 3; ++q) B[m][q] = (q == m ? T(1) : T(0)) - sc * (T)mim_DG(q - m + 3);
            }
        }
    };

    // ---- factorisation of the chunk and the local forward pass ----
    T Si[MM][BS][BS];
    T y[BS];
#pragma unroll
    for (int p = 0; p < BS; ++p) y[p] = T(0);
    {
        T G[BS][BS];
#pragma unroll
        for (int p = 0; p < BS; ++p)
#pragma unroll
            for (int q = 0; q < BS; ++q) G[p][q] = T(0);
#pragma unroll
        for (int i = 0; i < MM; ++i) {
            if (i < n) {
                T S[BS][BS];
                if (i == 0) {
#pragma unroll
                    for (int p = 0; p < BS; ++p)
#pragma unroll
                        for (int q = 0; q < BS; ++q) S[p][q] = sR[c * B2 + p * BS + q];
                } else {
                    T A[BS][BS], B[BS][BS];
                    blockA(i, A);
                    blockB(i, B);
#pragma unroll
                    for (int p = 0; p < BS; ++p)
#pragma unroll
                        for (int q = 0; q < BS; ++q) {
                            T acc = B[p][q];
#pragma unroll
                            for (int k = 0; k < BS; ++k) acc -= A[p][k] * G[k][q];
                            S[p][q] = acc;
                        }
                    if (b0 + i == s.nb - 1) {
#pragma unroll
                        for (int p = 0; p < BS; ++p)
#pragma unroll
                            for (int q = 0; q < BS; ++q) S[p][q] -= eT[kEndDB + p * 3 + q];
                    }
                }
                mat_inv<T, BS>(S, Si[i]);
                // y <- S^{-1} (r - A y)   (y = 0 entering the chunk)
                T t[BS];
                if (i == 0) {
#pragma unroll
                    for (int p = 0; p < BS; ++p) t[p] = Y[i][p];
                } else {
                    T A[BS][BS];
                    blockA(i, A);
#pragma unroll
                    for (int p = 0; p < BS; ++p) {
                        T acc = Y[i][p];
#pragma unroll
                        for (int q = 0; q < BS; ++q) acc -= A[p][q] * y[q];
                        t[p] = acc;
                    }
                }
#pragma unroll
                for (int p = 0; p < BS; ++p) {
                    T acc = T(0);
#pragma unroll
                    for (int q = 0; q < BS; ++q) acc += Si[i][p][q] * t[q];
                    y[p] = acc;
                    Y[i][p] = acc;
                }
                if (i + 1 < MM) {  // G <- S^{-1} C for the next block
                    T C[BS][BS];
                    blockC(i, C);
                    f_mm<T, BS>(Si[i], C, G);
                }
            }
        }
    }

    // ---- forward scan: the true y entering the chunk ----
    Map<T, BS> mp;
    {
        const T *F = sR + Tl * B2 + c * B2;
#pragma unroll
        for (int p = 0; p < BS; ++p) {
            mp.off[p] = y[p];
#pragma unroll
            for (int q = 0; q < BS; ++q) mp.m[p][q] = active ? F[p * BS + q] : (p == q ? T(1) : T(0));
        }
    }
    T yin[BS];
    line_scan<T, BS>(mp, true, Tl, yin, smmaps);
    {
        // y_b += delta_b,  delta_b = -S_b^{-1} A_b delta_{b-1},  delta entering = yin
        T dl[BS];
#pragma unroll
        for (int p = 0; p < BS; ++p) dl[p] = yin[p];
#pragma unroll
        for (int i = 0; i < MM; ++i) {
            if (i < n) {
                T A[BS][BS], t[BS];
                blockA(i, A);
#pragma unroll
                for (int p = 0; p < BS; ++p) {
                    T acc = T(0);
#pragma unroll
                    for (int q = 0; q < BS; ++q) acc += A[p][q] * dl[q];
                    t[p] = acc;
                }
#pragma unroll
                for (int p = 0; p < BS; ++p) {
                    T acc = T(0);
#pragma unroll
                    for (int q = 0; q < BS; ++q) acc -= Si[i][p][q] * t[q];
                    dl[p] = acc;
                    Y[i][p] += acc;
                }
            }
        }
    }

    // ---- local backward pass (x = 0 after the chunk) ----
    T x[BS];
#pragma unroll
    for (int p = 0; p < BS; ++p) x[p] = T(0);
#pragma unroll
    for (int i = MM - 1; i >= 0; --i) {
        if (i < n) {
            T t[BS];
            if (i == n - 1) {
#pragma unroll
                for (int p = 0; p < BS; ++p) t[p] = T(0);
            } else {
                T C[BS][BS];
                blockC(i, C);
#pragma unroll
                for (int p = 0; p < BS; ++p) {
                    T acc = T(0);
#pragma unroll
                    for (int q = 0; q < BS; ++q) acc += C[p][q] * x[q];
                    t[p] = acc;
                }
            }
#pragma unroll
            for (int p = 0; p < BS; ++p) {
                T acc = Y[i][p];
#pragma unroll
                for (int q = 0; q < BS; ++q) acc -= Si[i][p][q] * t[q];
                x[p] = acc;
                Y[i][p] = acc;
            }
        }
    }

    // ---- backward scan: the true x after the chunk ----
    {
        const T *H = sR + 2 * Tl * B2 + c * B2;
#pragma unroll
        for (int p = 0; p < BS; ++p) {
            mp.off[p] = x[p];
#pragma unroll
            for (int q = 0; q < BS; ++q) mp.m[p][q] = active ? H[p * BS + q] : (p == q ? T(1) : T(0));
        }
    }
    T xin[BS];
    line_scan<T, BS>(mp, false, Tl, xin, smmaps);
    if (!active) return;
    {
        // x_b += eps_b,  eps_b = -S_b^{-1} C_b eps_{b+1},  eps after the chunk = xin
        T ep[BS];
#pragma unroll
        for (int p = 0; p < BS; ++p) ep[p] = xin[p];
#pragma unroll
        for (int i = MM - 1; i >= 0; --i) {
            if (i < n) {
                T t[BS];
                if (b0 + i == s.nb - 1) {
#pragma unroll
                    for (int p = 0; p < BS; ++p) t[p] = T(0);
                } else {
                    T C[BS][BS];
                    blockC(i, C);
#pragma unroll
                    for (int p = 0; p < BS; ++p) {
                        T acc = T(0);
#pragma unroll
                        for (int q = 0; q < BS; ++q) acc += C[p][q] * ep[q];
                        t[p] = acc;
                    }
                }
#pragma unroll
                for (int p = 0; p < BS; ++p) {
                    T acc = T(0);
#pragma unroll
                    for (int q = 0; q < BS; ++q) acc -= Si[i][p][q] * t[q];
                    ep[p] = acc;
                    Y[i][p] += acc;
                }
            }
        }
    }

    // ---- outputs: C = 2 u* - a (+ source), v' = 2 v* - v, optionally natural u, w ----
    bool hit = false;
    const int src_k = d.src_k;
    auto srcval = [&](int k) -> T {
        if (k != src_k) return T(0);
        hit = true;
        const long long m = *d.clock;
        return (T)(d.src_scale * ricker(d.src_amp, d.src_f0, d.src_tdelay, (double)(m + 1) * d.dt));
    };
    T *__restrict__ uo = natural ? d.u_out : nullptr;
    T *__restrict__ wo = natural ? d.w_out : nullptr;
    const bool nat = uo != nullptr;
    T *__restrict__ gpo = d.po;
    T *__restrict__ gvo = d.vo;
    const int spo = (int)d.spo, svo = (int)d.svo, snp = (int)d.snp, snv = (int)d.snv;
    auto out_p = [&](int k, T val_out, T val_nat) {
        gpo[k * spo] = val_out + srcval(k);
        if (nat) uo[k * snp] = val_nat;
    };
    auto out_v = [&](int j, T vin, T dv) {  // dv = beta * (D_u u*)_j
        gvo[j * svo] = vin - T(2) * dv;
        if (nat) wo[j * snv] = vin - dv;
    };
    if constexpr (BS == 2) {
        // node j = b0 + i + 3 is window index i + 3 (16-byte loads of the chunk's windows)
        {
            T wp[MM + 4], wa[MM + 4];
            if (n > 0) {
                load_window<T, MM + 4>(sP + b0, wp);
                load_window<T, MM + 4>(sA + b0, wa);
            }
#pragma unroll
            for (int i = 0; i < MM; ++i)
                if (i < n) {
                    const T pin = wp[i + 3];
                    const T ae = wa[i + 3] * Y[i][0];
                    out_p(b0 + i + 3, pin - T(2) * ae, pin - ae);
                }
        }
        {
            T wv[MM + 4];
            if (n > 0) load_window<T, MM + 4>(sV + b0, wv);
#pragma unroll
            for (int i = 0; i < MM; ++i)
                if (i < n) out_v(b0 + i + 3, wv[i + 3], beta * Y[i][1]);
        }
    } else {
        T xn[BS];  // x of the block after the current one
#pragma unroll
        for (int p = 0; p < BS; ++p) xn[p] = xin[p];
#pragma unroll
        for (int i = MM - 1; i >= 0; --i) {
            if (i < n) {
                const int b = b0 + i;
                const int q0 = cb + 3 * i;
#pragma unroll
                for (int m = 0; m < 3; ++m) out_p(q0 + m, T(2) * Y[i][m] - sP[q0 + m], Y[i][m]);
                if (b != s.nb - 1) {
                    // nodes q0+1..q0+3 from this block's cells and the next block's
                    const T w0 = T(1.0 / 24.0), w1 = T(-9.0 / 8.0), w2 = T(9.0 / 8.0), w3 = T(-1.0 / 24.0);
                    const T bi = beta * ih;
                    out_v(q0 + 1, sV[q0 + 1], bi * (w0 * Y[i][0] + w1 * Y[i][1] + w2 * Y[i][2] + w3 * xn[0]));
                    out_v(q0 + 2, sV[q0 + 2], bi * (w0 * Y[i][1] + w1 * Y[i][2] + w2 * xn[0] + w3 * xn[1]));
                    out_v(q0 + 3, sV[q0 + 3], bi * (w0 * Y[i][2] + w1 * xn[0] + w2 * xn[1] + w3 * xn[2]));
                }
#pragma unroll
                for (int p = 0; p < BS; ++p) xn[p] = Y[i][p];
            }
        }
    }
    T xl[BS];  // x of the chunk's last block
#pragma unroll
    for (int p = 0; p < BS; ++p) xl[p] = Y[0][p];
#pragma unroll
    for (int i = 1; i < MM; ++i)
        if (i == n - 1)
#pragma unroll
            for (int p = 0; p < BS; ++p) xl[p] = Y[i][p];
    if (has_last) {  // tail unknowns: xe = HZ z, z with the last block's x
        T z[19], xe[6];
        end_window(true, z);
#pragma unroll
        for (int p = 0; p < BS; ++p) z[16 + p] = xl[p];
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            T acc = T(0);
#pragma unroll
            for (int k = 0; k < 19; ++k) acc += eT[kEndHZ + q * 19 + k] * z[k];
            xe[q] = acc;
        }
        if constexpr (BS == 2) {
            // e_{N-2}, g_{N-2}, e_{N-1}, g_{N-1}, g_N
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int j = N - 2 + q;
                const T pin = sP[j];
                const T ae = sA[j] * xe[2 * q];
                out_p(j, pin - T(2) * ae, pin - ae);
                out_v(j, sV[j], beta * xe[2 * q + 1]);
            }
            out_v(N, sV[N], beta * xe[4]);
        } else {
            // tail cells after this block, then nodes qb+1 .. N
            const int qb = cb + 3 * (n - 1);
            for (int t2 = 0; t2 < s.tu; ++t2) {
                const int cc = qb + 3 + t2;
                T xv = xe[0];
#pragma unroll
                for (int q = 1; q < 6; ++q)
                    if (q == t2) xv = xe[q];
                out_p(cc, T(2) * xv - sP[cc], xv);
            }
            for (int j = qb + 1; j <= N; ++j) {
                const T *row = eT + kEndDZ + (j - qb - 1) * 19;
                T acc = T(0);
#pragma unroll
                for (int k = 0; k < 19; ++k) acc += row[k] * z[k];
                out_v(j, sV[j], beta * ih * acc);
            }
        }
    }
    if (has_first) {  // head unknowns from block 0: xe = HZ z, z with block 0's x
        T z[19], xe[6];
        end_window(false, z);
#pragma unroll
        for (int p = 0; p < BS; ++p) z[16 + p] = Y[0][p];
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            T acc = T(0);
#pragma unroll
            for (int k = 0; k < 19; ++k) acc += eH[kEndHZ + q * 19 + k] * z[k];
            xe[q] = acc;
        }
        if constexpr (BS == 2) {
            // g0, e1, g1, e2, g2
            out_v(0, sV[0], beta * xe[0]);
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int j = 1 + q;
                const T pin = sP[j];
                const T ae = sA[j] * xe[1 + 2 * q];
                out_p(j, pin - T(2) * ae, pin - ae);
                out_v(j, sV[j], beta * xe[2 + 2 * q]);
            }
        } else {
            // head cells 1 .. hu, then nodes 0 .. hu+1
#pragma unroll
            for (int t2 = 0; t2 < 6; ++t2)
                if (t2 < s.hu) out_p(1 + t2, T(2) * xe[t2] - sP[1 + t2], xe[t2]);
            for (int j = 0; j <= s.hu + 1; ++j) {
                const T *row = eH + kEndDZ + j * 19;
                T acc = T(0);
#pragma unroll
                for (int k = 0; k < 19; ++k) acc += row[k] * z[k];
                out_v(j, sV[j], beta * ih * acc);
            }
        }
    }
    if (hit && d.advance_clock) *d.clock = *d.clock + 1;
}

// ---------------------------------------------------------------------------------------
// The kernel: persistent CTAs walk the line groups g = blockIdx.x, blockIdx.x + gridDim.x,
// ...; with STAGES = 2 thread 0 starts the copies of the next group before the current one
// is solved.  A wait that runs out sets *fault and ends the CTA.
// ---------------------------------------------------------------------------------------
template <typename T, int BS, int MM, int STAGES>
__global__ void __launch_bounds__(kFacThreads, 1)
line_solve_factored_kernel(const LineDesc<T> *__restrict__ descs, const int4 *__restrict__ groups,
                           int ngroups, int natural, unsigned stage_bytes, int *fault) {
    extern __shared__ __align__(128) unsigned char fac_smem[];
    __shared__ Map<T, BS> smmaps[32];
    __shared__ __align__(8) unsigned long long bars[2];
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (STAGES == 2 && tid == 0 && (int)blockIdx.x < ngroups)
        fac_issue<T>(descs, groups[blockIdx.x], fac_smem, &bars[0]);
    int it = 0;
    bool ok = true;
    int g = blockIdx.x;
    for (; g < ngroups; g += gridDim.x, ++it) {
        const int st = STAGES == 2 ? (it & 1) : 0;
        const unsigned par = STAGES == 2 ? (unsigned)((it >> 1) & 1) : (unsigned)(it & 1);
        if (tid == 0) {
            if (STAGES == 2) {
                const int gn = g + (int)gridDim.x;
                if (gn < ngroups)
                    fac_issue<T>(descs, groups[gn], fac_smem + (size_t)(st ^ 1) * stage_bytes, &bars[st ^ 1]);
            } else {
                fac_issue<T>(descs, groups[g], fac_smem, &bars[0]);
            }
        }
        const bool got = mbar_wait(&bars[st], par);
        if (!__syncthreads_and(got)) { ok = false; break; }
        fac_group<T, BS, MM>(groups[g], fac_smem + (size_t)st * stage_bytes, natural, smmaps);
        __syncthreads();
    }
    if (!ok && tid == 0) {
        atomicExch(fault, 1);
        // let copies still in flight land before the CTA's shared memory is released
        const int st = STAGES == 2 ? (it & 1) : 0;
        (void)mbar_wait(&bars[st], STAGES == 2 ? (unsigned)((it >> 1) & 1) : (unsigned)(it & 1));
        if (STAGES == 2 && g + (int)gridDim.x < ngroups)
            (void)mbar_wait(&bars[st ^ 1], (unsigned)(((it + 1) >> 1) & 1));
    }
}

template <typename T>
cudaError_t launch_fac_precompute(const LineDesc<T> *d, int nlines, cudaStream_t s) {
    if (nlines <= 0) return cudaSuccess;
    fac_precompute_kernel<T><<<(nlines + 63) / 64, 64, 0, s>>>(d, nlines);
    return cudaGetLastError();
}

template <typename T, int BS, int MM, int STAGES>
cudaError_t launch_fac_inst(const LineDesc<T> *d, const int4 *groups, int ngroups, size_t stage_bytes,
                            int grid, int natural, int *fault, cudaStream_t s) {
    auto kern = line_solve_factored_kernel<T, BS, MM, STAGES>;
    const size_t dyn = (size_t)STAGES * stage_bytes;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
    kern<<<grid, kFacThreads, dyn, s>>>(d, groups, ngroups, natural, (unsigned)stage_bytes, fault);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_line_solve_factored(const LineDesc<T> *d, const int4 *groups, int ngroups, int method,
                                       size_t stage_bytes, int stages, int grid, int natural, int *fault,
                                       cudaStream_t s) {
    if (ngroups <= 0) return cudaSuccess;
    if (grid > ngroups) grid = ngroups;
    if (method == kCFD)
        return stages == 2 ? launch_fac_inst<T, 2, 8, 2>(d, groups, ngroups, stage_bytes, grid, natural, fault, s)
                           : launch_fac_inst<T, 2, 8, 1>(d, groups, ngroups, stage_bytes, grid, natural, fault, s);
    return stages == 2 ? launch_fac_inst<T, 3, 3, 2>(d, groups, ngroups, stage_bytes, grid, natural, fault, s)
                       : launch_fac_inst<T, 3, 3, 1>(d, groups, ngroups, stage_bytes, grid, natural, fault, s);
}

template cudaError_t launch_fac_precompute<float>(const LineDesc<float> *, int, cudaStream_t);
template cudaError_t launch_fac_precompute<double>(const LineDesc<double> *, int, cudaStream_t);
template cudaError_t launch_line_solve_factored<float>(const LineDesc<float> *, const int4 *, int, int, size_t,
                                                       int, int, int, int *, cudaStream_t);
template cudaError_t launch_line_solve_factored<double>(const LineDesc<double> *, const int4 *, int, int,
                                                        size_t, int, int, int, int *, cudaStream_t);

}  // namespace adi
