// adi_factored.cu -- the factored line solver (default): persistent CTAs, whole lines staged
// in shared memory by bulk asynchronous copies (a two-stage mbarrier ring), uniform chunks of
// MM blocks per thread held in registers, chunks joined by segmented scans of affine maps.
//
// Line system (adi_ops.cuh): every line is  [head region | nb middle blocks | tail region]
// where the middle part is block tridiagonal (blocks A_b, B_b, C_b of size BS) and the two end
// regions hold the one-sided boundary rows of App. A/B.  Here the end regions also absorb the
// remainder of nb modulo MM, so that the middle part is exactly tact * MM blocks and every
// thread runs the same unrolled code on MM blocks with no per-block predication.
//
// FP64 precompute, once per line (time invariant, depends on alpha only):
//   * each end region is eliminated densely: its unknowns become a linear map HZ of
//     z = [p window, v window, x of the adjacent middle block], the adjacent block's right-hand
//     side gets the correction KZ z and its diagonal block the correction dB;
//   * the middle part's block LU  S_b = B_b - A_b G_{b-1},  G_b = S_b^{-1} C_b  is run once and
//     per chunk c only  S at the chunk's first block,  F_c = prod(-S_b^{-1} A_b)  and
//     H_c = prod(-G_b)  are stored.
// Per half step a thread rebuilds S_b^{-1} of its blocks from the stored S and the alpha values,
// then
//   forward   y_b = S_b^{-1}(r_b - A_b y_{b-1})  locally from y = 0; the true y entering the
//             chunk is the exclusive scan of the maps (F_c, y_end) over the chunks; correction
//             y_b += d_b, d_b = -S_b^{-1} A_b d_{b-1};
//   backward  x_b = y_b - G_b x_{b+1} locally from x = 0; the true x after the chunk is the
//             suffix scan of (H_c, x_first); correction x_b += e_b, e_b = -G_b e_{b+1};
// and writes the carried outputs C = 2u* - a (+ dt/2 f), v' = 2v* - v.  The end regions are
// evaluated cooperatively by the warp that owns the adjacent chunk.
//
// The chunk transfers decay geometrically along a line (the line systems are diagonally
// dominant in the block sense).  The precompute finds, per line, the reach R: the smallest
// number of consecutive chunk transfers whose product has infinity norm below tau (2^-40 for
// FP32 records, 2^-70 for FP64).  The scan value of chunk c is then the sequential recurrence
// over the R chunks before (after) it, read from shared memory; what it leaves out is that
// product times a true value of the solution, i.e. below tau relative to the solution.  Lines
// whose reach exceeds kFacMaxReach use the full log-depth scan of affine maps instead (the
// group's kFacOwnFull bit, set on the host from the line's own reach).
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/adi.h"
#include "adi_internal.h"
#include "adi_line.cuh"
#include "adi_ops.cuh"

namespace adi {

constexpr int kFacThreads = 512;              // threads per CTA: 15 compute warps and one staging warp
constexpr int kFacWorkers = kFacThreads - 32; // threads that solve lines
constexpr int kFacMaxT = kFacWorkers;         // chunks (threads) per line at most
constexpr size_t kFacSmemLimit = 227 * 1024;  // shared memory per CTA
constexpr size_t kFacStaticBase = 2048;       // reserve for the kernel's other static shared memory
constexpr int kFacMaxStages = 3;              // staged groups in flight per CTA at most
constexpr int kFacWs = 1024;                  // FP64 workspace of the precompute, per line
// Static shared memory of the kernel for element size esz and block size bs, an upper bound:
// the scan buffers (chunk offsets, two arrays for FP32, one for FP64) plus the rest (checked
// against the compiled kernel before its first launch).
__host__ __device__ inline size_t fac_static_smem(size_t esz, int bs) {
    return kFacStaticBase + (size_t)kFacThreads * bs * (esz == 4 ? 2 : 1) * esz;
}

// One rounding for a*b + c, written out so that the compiler's contraction choices cannot make
// two code paths of the same output round differently.
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// ---------------------------------------------------------------------------------------
// Geometry of a line for the factored solver.
// ---------------------------------------------------------------------------------------
// Blocks per chunk: CFD 9 (an odd stride between the chunks' shared-memory windows keeps
// their loads free of bank conflicts); MFD 3 (a chunk's record, S, F and H of 3 x 3, then costs
// 12 bytes per cell in FP32; two-block chunks cost 18 and ran a batch of 128-1024-cell lines 4 %
// slower), and 2 for lines of at most kFacMfdShort cells, whose end regions would not fit their
// tables with the remainder of three-block chunks.
constexpr int kFacMfdShort = 16;
__host__ __device__ inline int fac_mm(int method, int N) {
    if (method == kCFD) return 9;
    return N <= kFacMfdShort ? 2 : 3;
}
// Threads a whole line needs (see fac_geom): a power of two up to 32, else a multiple of 32.
__host__ __device__ inline int fac_geom_T(int method, int N) {
    const int tact = line_shape(method, N).nb / fac_mm(method, N);
    if (tact > 32) return (tact + 31) & ~31;
    int T = 1;
    while (T < tact) T <<= 1;
    return T;
}
// Kernel variant (one compiled instance per chunk length and method, and for split lines).
__host__ __device__ inline int fac_variant_of(int method, int N) {
    const bool split = fac_geom_T(method, N) > kFacMaxT;
    if (method == kCFD) return split ? 3 : 0;
    return fac_mm(method, N) == 2 ? 1 : (split ? 4 : 2);
}
// End windows: p[op .. op+win) and v[ov .. ov+win); hmax bounds the eliminated unknowns of
// one end (base head/tail plus half of at most MM-1 remainder blocks).
__host__ __device__ inline int fac_win(int method) { return method == kCFD ? 8 : 12; }
__host__ __device__ inline int fac_hmax(int method) { return method == kCFD ? 13 : 8; }

struct FacGeom {
    int method, N, bs, mm;
    int hu, tu;   // eliminated unknowns of the head and tail regions
    int nb;       // middle blocks (tact * mm)
    int tact;     // chunks holding blocks
    int T;        // threads per line: a power of two up to 32, else a multiple of 32
    int first;    // CFD: node of middle block 0; MFD: first cell of middle block 0
    int win, hmax;
};

__host__ __device__ inline FacGeom fac_geom(int method, int N) {
    const LineShape s = line_shape(method, N);
    FacGeom g;
    g.method = method;
    g.N = N;
    g.bs = s.bs;
    g.mm = fac_mm(method, N);
    g.tact = s.nb / g.mm;
    const int k = s.nb - g.tact * g.mm;
    const int kh = k / 2;
    g.hu = s.hu + kh * s.bs;
    g.tu = s.tu + (k - kh) * s.bs;
    g.nb = g.tact * g.mm;
    int T = 1;
    while (T < g.tact) T <<= 1;
    g.T = g.tact > 32 ? ((g.tact + 31) & ~31) : T;
    g.first = method == kCFD ? (g.hu + 1) / 2 : g.hu + 1;
    g.win = fac_win(method);
    g.hmax = fac_hmax(method);
    return g;
}

// Per-end table: KZ [bs][2win] | HZ [hmax][Z] | DZ [hmax+2][Z] (MFD) | dB [bs][bs], Z = 2win+bs.
__host__ __device__ inline int fac_zlen(const FacGeom &g) { return 2 * g.win + g.bs; }
__host__ __device__ inline int fac_e_hz(const FacGeom &g) { return g.bs * 2 * g.win; }
__host__ __device__ inline int fac_e_dz(const FacGeom &g) { return fac_e_hz(g) + g.hmax * fac_zlen(g); }
__host__ __device__ inline int fac_e_db(const FacGeom &g) {
    return fac_e_dz(g) + (g.method == kMFD ? (g.hmax + 2) * fac_zlen(g) : 0);
}
__host__ __device__ inline int fac_e_stride(const FacGeom &g) { return (fac_e_db(g) + g.bs * g.bs + 3) & ~3; }
// Record of one line: S_first, F_c, H_c (tact blocks each, every part padded to a multiple of
// four elements so that each starts on a 16-byte boundary), the head and tail tables, then four
// values: the forward and backward reach of the windowed scans.
__host__ __device__ inline int fac_ru4(int x) { return (x + 3) & ~3; }
__host__ __device__ inline int fac_part(const FacGeom &g) { return fac_ru4(g.tact * g.bs * g.bs); }
__host__ __device__ inline int fac_chunk_elems(const FacGeom &g) { return 3 * fac_part(g); }
__host__ __device__ inline int fac_info(const FacGeom &g) { return fac_chunk_elems(g) + 2 * fac_e_stride(g); }
__host__ __device__ inline int fac_rec(const FacGeom &g) { return fac_info(g) + 4; }
// Elements of one staged line array (pressure, velocity or alpha), a multiple of four.
__host__ __device__ inline int fac_lp(int N) { return (N + 2 + 3) & ~3; }
// Shared-memory scratch of a staged line: the window parts of its end-region rows.
__host__ __device__ inline int fac_end_rows(int method) {
    return 2 * (fac_hmax(method) + (method == kMFD ? fac_hmax(method) + 2 : 0));
}
__host__ __device__ inline int fac_scratch(const FacGeom &g) { return (fac_end_rows(g.method) + 3) & ~3; }
// A staged line: pressure, velocity, alpha (fac_lp each), the record, the scratch.
__host__ __device__ inline int fac_line_elems(const FacGeom &g) { return 3 * fac_lp(g.N) + fac_rec(g) + fac_scratch(g); }

constexpr size_t kDescBytes = sizeof(LineDesc<float>);
static_assert(sizeof(LineDesc<float>) == sizeof(LineDesc<double>), "descriptor sizes differ");
static_assert(kDescBytes % 16 == 0, "descriptor size");
__host__ __device__ inline size_t fac_desc_area(int nl) { return ((size_t)nl * kDescBytes + 127) & ~(size_t)127; }
// A stage: the group (128 bytes), the descriptors, then the lines.
constexpr size_t kFacGroupBytes = 128;
static_assert(sizeof(FacGroup) % 16 == 0 && sizeof(FacGroup) <= kFacGroupBytes, "group header");
__host__ __device__ inline size_t fac_head_bytes(int nl) { return kFacGroupBytes + fac_desc_area(nl); }

size_t fac_stage_bytes(int method, int N, int nl, size_t esz) {
    size_t b = fac_head_bytes(nl) + (size_t)nl * fac_line_elems(fac_geom(method, N)) * esz;
    return (b + 127) & ~(size_t)127;
}
int fac_stages_for(size_t stage_bytes, size_t esz, int method) {
    const size_t st = fac_static_smem(esz, method == kCFD ? 2 : 3);
    for (int k = kFacMaxStages; k >= 1; --k)
        if ((size_t)k * stage_bytes + st <= kFacSmemLimit) return k;
    return 0;
}
// Lines per CTA: as many as the CTA's threads cover, fewer where a two-stage ring of them
// would not fit shared memory.
int fac_lines_per_cta(int method, int N, size_t esz) {
    const int T = fac_geom(method, N).T;
    int nl = T >= kFacWorkers ? 1 : kFacWorkers / T;
    while (nl > 1 && fac_stages_for(fac_stage_bytes(method, N, nl, esz), esz, method) < 2) --nl;
    return nl;
}
bool fac_split_line(int method, int N) { return fac_geom(method, N).T > kFacMaxT; }
bool fac_supported(int method, int N, size_t esz) {
    const FacGeom g = fac_geom(method, N);
    if (g.tact < 1) return false;
    if (g.hu > g.hmax || g.tu > g.hmax) return false;
    if (g.T > kFacMaxT) {  // split into sub-lines (for the largest halo a split line accepts)
        FacGroup tmp[kFacMaxSplit];
        size_t sb = 0;
        return fac_split_groups(method, N, 0, kFacSplitMaxHalo, 1.0, 1.0, esz, tmp, &sb) > 0;
    }
    return fac_stages_for(fac_stage_bytes(method, N, 1, esz), esz, method) > 0;
}
size_t fac_words(int method, int N) { return (size_t)fac_rec(fac_geom(method, N)); }
int fac_chunks(int method, int N) { return fac_geom(method, N).T; }
int fac_variant(int method, int N) { return fac_variant_of(method, N); }
size_t fac_ws_doubles() { return kFacWs; }
static unsigned fac_tdiv(int T) {
    return T > 1 ? (unsigned)(((1ull << 32) + (unsigned long long)T - 1) / (unsigned long long)T) : 0u;
}
FacGroup fac_group_of(int method, int N, int first, int nl, double inv_h, double beta) {
    const FacGeom g = fac_geom(method, N);
    FacGroup r{};
    r.first = first; r.nl = nl; r.N = N; r.T = g.T;
    r.tact = g.tact; r.hu = g.hu; r.tu = g.tu; r.mid = g.first;
    r.lp = fac_lp(N); r.part = fac_part(g);
    r.eh = fac_chunk_elems(g); r.et = r.eh + fac_e_stride(g);
    r.info = fac_info(g); r.pl = p_last(method, N);
    r.ls = fac_line_elems(g); r.scr = 3 * r.lp + fac_rec(g);
    r.ih = inv_h; r.beta = beta; r.ihf = (float)inv_h; r.betaf = (float)beta;
    r.tdiv = fac_tdiv(g.T);
    r.c0 = 0; r.lo = 0; r.pn = r.pl + 1; r.vn = N + 1;
    r.own = (g.tact << 9) | kFacOwnHead | kFacOwnTail;
    r.sp0 = 0; r.sp1 = r.pl + 1; r.sv0 = 0; r.sv1 = N + 1;
    return r;
}

// Sub-lines of a line with more chunks than a CTA has threads.  Sub-line i owns the chunks
// [tact i / K, tact (i+1) / K) and also solves `halo` (rounded so that its first chunk is a
// multiple of four: the record parts it stages then start on 16-byte boundaries) chunks on
// each interior side.  The windowed scans of its owned chunks reach at most `halo` chunks, all
// inside its range; the halo chunks' own scan values are truncated at the range's ends and
// their outputs are not written.  Staged elements cover every stencil read of the range; the
// owned outputs are stored by bulk copies on 4-element-aligned spans and, at the ragged ends
// of a span, by the threads that compute them.
int fac_split_groups(int method, int N, int first, int halo, double inv_h, double beta, size_t esz,
                     FacGroup *out, size_t *stage_bytes) {
    const FacGeom g = fac_geom(method, N);
    if (g.tact < 1 || g.hu > g.hmax || g.tu > g.hmax || halo < 1 || halo > kFacSplitMaxHalo) return 0;
    const int B2 = g.bs * g.bs, pl = p_last(method, N);
    const int per = method == kCFD ? g.mm : 3 * g.mm;  // nodes (CFD) or cells (MFD) per chunk
    const int vsh = method == kCFD ? 0 : 1;             // MFD: a chunk's velocities start one after its cells
    int K = 2;
    while (K <= kFacMaxSplit && (g.tact + K - 1) / K + 2 * halo + 3 > kFacMaxT) ++K;
    if (K > kFacMaxSplit) return 0;
    size_t smax = 0;
    for (int i = 0; i < K; ++i) {
        const int s0 = (int)((long long)g.tact * i / K), s1 = (int)((long long)g.tact * (i + 1) / K);
        const bool head = i == 0, tail = i == K - 1;
        const int c0 = head ? 0 : ((s0 - halo) & ~3);
        const int c1 = tail ? g.tact : std::min(g.tact, s1 + halo);
        const int tl = c1 - c0;
        if (c0 < 0 || tl > kFacMaxT || tl <= 64) return 0;
        FacGroup r{};
        r.first = first; r.nl = 1; r.N = N;
        r.tact = tl; r.T = (tl + 31) & ~31;
        r.hu = g.hu; r.tu = g.tu; r.mid = g.first;
        // staged elements [lo, hi): a CFD chunk reads nodes jb-1 .. jb+mm, an MFD chunk cells
        // cb .. cb+3mm-1 and velocities cb-2 .. cb+3mm
        const int lo = head ? 0 : ((g.first + c0 * per - 2) & ~3);
        const int hp = tail ? pl + 1 : g.first + c1 * per + 1;
        const int hv = tail ? N + 1 : g.first + c1 * per + 1;
        r.lo = lo; r.pn = hp - lo; r.vn = hv - lo;
        r.lp = fac_ru4(r.pn > r.vn ? r.pn : r.vn);
        const int part = fac_ru4(tl * B2), es = fac_e_stride(g);
        r.part = part;
        int off = 3 * part;
        r.eh = head ? off : -1;
        if (head) off += es;
        r.et = tail ? off : -1;
        if (tail) off += es;
        r.info = off;
        r.pl = pl;
        r.scr = 3 * r.lp + off + 4;
        r.ls = r.scr + fac_scratch(g);
        r.ih = inv_h; r.beta = beta; r.ihf = (float)inv_h; r.betaf = (float)beta;
        r.tdiv = fac_tdiv(r.T);
        r.c0 = c0;
        r.own = (s0 - c0) | ((s1 - c0) << 9) | (head ? kFacOwnHead : 0) | (tail ? kFacOwnTail : 0) | kFacOwnSplit;
        const int p0 = head ? 0 : g.first + s0 * per, p1 = tail ? pl + 1 : g.first + s1 * per;
        const int v0 = head ? 0 : g.first + s0 * per + vsh, v1 = tail ? N + 1 : g.first + s1 * per + vsh;
        r.sp0 = fac_ru4(p0); r.sp1 = tail ? p1 : (p1 & ~3);
        r.sv0 = fac_ru4(v0); r.sv1 = tail ? v1 : (v1 & ~3);
        out[i] = r;
        const size_t sb = (fac_head_bytes(1) + (size_t)r.ls * esz + 127) & ~(size_t)127;
        if (sb > smax) smax = sb;
    }
    *stage_bytes = smax;
    return fac_stages_for(smax, esz, method) > 0 ? K : 0;
}
// Table offsets of an end region, as compile-time functions of the block size (fac_e_*).
template <int BS>
struct FacEnd {
    static constexpr int W = BS == 2 ? 8 : 12, HMAX = BS == 2 ? 13 : 8, Z = 2 * W + BS;
    static constexpr int HZ = BS * 2 * W, DZ = HZ + HMAX * Z, DB = DZ + (BS == 3 ? (HMAX + 2) * Z : 0);
};

// ---------------------------------------------------------------------------------------
// Middle block b (A to block b-1, B, C to block b+1) in precision R from alpha values
// al(k) along the pressure line.
// ---------------------------------------------------------------------------------------
template <typename R, int BS, typename AL>
__device__ __forceinline__ void fac_block(const FacGeom &g, double beta, double ih, int b, AL al,
                                          R (&A)[BS][BS], R (&B)[BS][BS], R (&C)[BS][BS]) {
    if constexpr (BS == 2) {
        const int j = g.first + b;
        const R tb = R(3) * (R)beta * (R)ih;
        A[0][0] = R(1); A[0][1] = -tb; A[1][0] = -R(3) * (R)ih * (R)al(j - 1); A[1][1] = R(1);
        B[0][0] = R(4); B[0][1] = R(0); B[1][0] = R(0); B[1][1] = R(4);
        C[0][0] = R(1); C[0][1] = tb; C[1][0] = R(3) * (R)ih * (R)al(j + 1); C[1][1] = R(1);
    } else {
        const int cb = g.first + 3 * b;
        const R bh2 = (R)(beta * ih * ih);
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            const R sc = (R)al(cb + m) * bh2;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                A[m][q] = (q >= m) ? -sc * (R)mim_DG(q - m) : R(0);
                B[m][q] = (q == m ? R(1) : R(0)) - sc * (R)mim_DG(q - m + 3);
                C[m][q] = (q <= m) ? -sc * (R)mim_DG(q - m + 6) : R(0);
            }
        }
    }
}

template <typename R, int BS>
__device__ __forceinline__ void f_mm(const R (&X)[BS][BS], const R (&Y)[BS][BS], R (&Z)[BS][BS]) {
#pragma unroll
    for (int i = 0; i < BS; ++i)
#pragma unroll
        for (int j = 0; j < BS; ++j) {
            R acc = R(0);
#pragma unroll
            for (int k = 0; k < BS; ++k) acc += X[i][k] * Y[k][j];
            Z[i][j] = acc;
        }
}

// ---------------------------------------------------------------------------------------
// FP64 precompute.
// ---------------------------------------------------------------------------------------
// Right-hand side of line row i (solver index) as coefficients on the windows
// p[op .. op+W) and v[ov .. ov+W).  False if a term falls outside them.
template <typename TS>
__device__ bool fac_rhs_coeffs(const LineDesc<TS> &d, int i, int op, int ov, int W, double *cp, double *cv) {
    for (int k = 0; k < W; ++k) cp[k] = cv[k] = 0.0;
    const int N = d.N;
    const double ih = d.inv_h;
    bool ok = true;
    auto add = [&](double *w, int idx, double val) {
        if (idx < 0 || idx >= W) ok = false; else w[idx] += val;
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
    // r_c = p_c - alpha_c/h sum_j D[c-1][j] (v_j - beta/h (G[j][0] p_0 + G[j][N+1] p_{N+1}))
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

// Dense elimination of one end region (end 0: head, 1: tail) into its table; dB of the end
// (bs x bs, row-major) is also returned in dBo.  False if the region is singular.
template <typename TS>
__device__ bool fac_end(const LineDesc<TS> &d, const FacGeom &g, int end, double *ws, TS *et, double *dBo) {
    const int N = d.N, bs = g.bs, W = g.win, Z = fac_zlen(g);
    const int nunk = d.method == kCFD ? 2 * N : N;
    const int m = end == 0 ? g.hu : g.tu;
    const int r0 = end == 0 ? 0 : nunk - g.tu;
    const int j0 = end == 0 ? g.hu : nunk - g.tu - bs;
    const int pl = p_last(d.method, N);
    const int op = end == 0 ? 0 : pl + 1 - W, ov = end == 0 ? 0 : N + 1 - W;
    double *H = ws, *Hi = H + m * m, *E = Hi + m * m, *F = E + m * bs, *Rm = F + bs * m;
    double *HiE = Rm + m * 2 * W, *K = HiE + m * bs, *HZ = K + bs * m;
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) H[i * m + j] = line_entry(d, r0 + i, r0 + j);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < bs; ++j) E[i * bs + j] = line_entry(d, r0 + i, j0 + j);
    for (int i = 0; i < bs; ++i)
        for (int j = 0; j < m; ++j) F[i * m + j] = line_entry(d, j0 + i, r0 + j);
    if (!small_inverse(H, m, Hi)) return false;
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < bs; ++j) {
            double acc = 0.0;
            for (int k = 0; k < m; ++k) acc += Hi[i * m + k] * E[k * bs + j];
            HiE[i * bs + j] = acc;
        }
    for (int i = 0; i < bs; ++i)
        for (int j = 0; j < m; ++j) {
            double acc = 0.0;
            for (int k = 0; k < m; ++k) acc += F[i * m + k] * Hi[k * m + j];
            K[i * m + j] = acc;
        }
    for (int i = 0; i < bs; ++i)
        for (int j = 0; j < bs; ++j) {
            double acc = 0.0;
            for (int k = 0; k < m; ++k) acc += F[i * m + k] * HiE[k * bs + j];
            dBo[i * bs + j] = acc;
        }
    bool ok = true;
    for (int q = 0; q < m; ++q) ok = fac_rhs_coeffs(d, r0 + q, op, ov, W, Rm + q * 2 * W, Rm + q * 2 * W + W) && ok;
    const double nan = __longlong_as_double(0x7ff8000000000000ULL);
    const int e_stride = fac_e_stride(g);
    for (int i = 0; i < e_stride; ++i) et[i] = (TS)0;
    // KZ = -K R
    for (int p = 0; p < bs; ++p)
        for (int k = 0; k < 2 * W; ++k) {
            double acc = 0.0;
            for (int q = 0; q < m; ++q) acc -= K[p * m + q] * Rm[q * 2 * W + k];
            et[p * 2 * W + k] = (TS)(ok ? acc : nan);
        }
    // HZ = [Hinv R | -Hinv E]
    for (int q = 0; q < m; ++q) {
        for (int k = 0; k < 2 * W; ++k) {
            double acc = 0.0;
            for (int q2 = 0; q2 < m; ++q2) acc += Hi[q * m + q2] * Rm[q2 * 2 * W + k];
            HZ[q * Z + k] = acc;
        }
        for (int b = 0; b < bs; ++b) HZ[q * Z + 2 * W + b] = -HiE[q * bs + b];
        for (int k = 0; k < Z; ++k) et[fac_e_hz(g) + q * Z + k] = (TS)(ok ? HZ[q * Z + k] : nan);
    }
    for (int i = 0; i < bs * bs; ++i) et[fac_e_db(g) + i] = (TS)dBo[i];
    if (d.method != kMFD) return true;
    // MFD: h (G u)_j at the end's velocity nodes as maps of z (cells through HZ)
    const int qb = g.first + 3 * (g.nb - 1);  // first cell of the last middle block
    const int jlo = end == 0 ? 0 : qb + 1, jhi = end == 0 ? g.hu + 1 : N;
    const int cell_lo = end == 0 ? 1 : N - g.tu + 1;  // first eliminated cell
    const int adj = end == 0 ? g.hu + 1 : qb;         // first cell of the adjacent block
    for (int j = jlo; j <= jhi; ++j) {
        double *row = HZ + m * Z;  // scratch row after HZ
        for (int k = 0; k < Z; ++k) row[k] = 0.0;
        double gw[8];
        int g0;
        const int ng = mfd_G_row(N, j, &g0, gw);
        bool rok = ok;
        for (int t = 0; t < ng; ++t) {
            const int cc = g0 + t;
            if (cc == 0 || cc == N + 1) {
                const int wi = cc - op;
                if (wi < 0 || wi >= W) rok = false; else row[wi] += gw[t];
            } else if (cc >= cell_lo && cc < cell_lo + m) {
                for (int k = 0; k < Z; ++k) row[k] += gw[t] * HZ[(cc - cell_lo) * Z + k];
            } else if (cc >= adj && cc < adj + bs) {
                row[2 * W + cc - adj] += gw[t];
            } else {
                rok = false;
            }
        }
        for (int k = 0; k < Z; ++k) et[fac_e_dz(g) + (j - jlo) * Z + k] = (TS)(rok ? row[k] : nan);
    }
    return true;
}

template <typename TS, int BS>
__device__ bool fac_chunks_fp64(const LineDesc<TS> &d, const FacGeom &g, const double *dBh, const double *dBt, TS *rec) {
    constexpr int B2 = BS * BS;
    TS *recS = rec, *recF = rec + fac_part(g), *recH = rec + (size_t)2 * fac_part(g);
    auto al = [&](int k) -> double { return (double)d.alpha[(long long)k * d.sp]; };
    double G[BS][BS], Fp[BS][BS], Hp[BS][BS];
    for (int p = 0; p < BS; ++p)
        for (int q = 0; q < BS; ++q) { G[p][q] = 0.0; Fp[p][q] = Hp[p][q] = (p == q) ? 1.0 : 0.0; }
    for (int b = 0; b < g.nb; ++b) {
        double A[BS][BS], B[BS][BS], C[BS][BS];
        fac_block<double, BS>(g, d.beta, d.inv_h, b, al, A, B, C);
        if (b == 0)
            for (int p = 0; p < BS; ++p)
                for (int q = 0; q < BS; ++q) { B[p][q] -= dBh[p * BS + q]; A[p][q] = 0.0; }
        if (b == g.nb - 1)
            for (int p = 0; p < BS; ++p)
                for (int q = 0; q < BS; ++q) { B[p][q] -= dBt[p * BS + q]; C[p][q] = 0.0; }
        double S[BS][BS], Si[BS][BS], Gn[BS][BS], T1[BS][BS];
        for (int p = 0; p < BS; ++p)
            for (int q = 0; q < BS; ++q) {
                double acc = B[p][q];
                for (int k = 0; k < BS; ++k) acc -= A[p][k] * G[k][q];
                S[p][q] = acc;
            }
        double det = BS == 2 ? S[0][0] * S[1][1] - S[0][1] * S[1][0]
                             : S[0][0] * (S[1][1] * S[2][2] - S[1][2] * S[2][1]) -
                                   S[0][1] * (S[1][0] * S[2][2] - S[1][2] * S[2][0]) +
                                   S[0][2] * (S[1][0] * S[2][1] - S[1][1] * S[2][0]);
        if (!(fabs(det) > 0.0) || !isfinite(det)) return false;
        mat_inv<double, BS>(S, Si);
        f_mm<double, BS>(Si, C, Gn);
        const int c = b / g.mm, i = b % g.mm;
        if (i == 0) {
            for (int p = 0; p < BS; ++p)
                for (int q = 0; q < BS; ++q) {
                    recS[(size_t)c * B2 + p * BS + q] = (TS)S[p][q];
                    Fp[p][q] = Hp[p][q] = (p == q) ? 1.0 : 0.0;
                }
        }
        // Fp <- (-Si A) Fp ;  Hp <- Hp (-Gn)
        double Fb[BS][BS];
        f_mm<double, BS>(Si, A, Fb);
        f_mm<double, BS>(Fb, Fp, T1);
        for (int p = 0; p < BS; ++p)
            for (int q = 0; q < BS; ++q) Fp[p][q] = -T1[p][q];
        f_mm<double, BS>(Hp, Gn, T1);
        for (int p = 0; p < BS; ++p)
            for (int q = 0; q < BS; ++q) Hp[p][q] = -T1[p][q];
        if (i == g.mm - 1)
            for (int p = 0; p < BS; ++p)
                for (int q = 0; q < BS; ++q) {
                    recF[(size_t)c * B2 + p * BS + q] = (TS)Fp[p][q];
                    recH[(size_t)c * B2 + p * BS + q] = (TS)Hp[p][q];
                }
        for (int p = 0; p < BS; ++p)
            for (int q = 0; q < BS; ++q) G[p][q] = Gn[p][q];
    }
    return true;
}

// Reach of the windowed scans (see the header): the largest, over the chunks, of the number
// of consecutive stored transfers (forward: F_e F_{e-1} ..., backward: H_s H_{s+1} ...) whose
// product first has infinity norm at most tau, or that reaches the end of the line; at most
// kFacMaxReach + 1 (which selects the full scan).
template <typename TS, int BS>
__device__ int fac_reach(const TS *maps, int tact, double tau, bool forward) {
    constexpr int B2 = BS * BS;
    int reach = 0;
    for (int e = 0; e < tact - 1; ++e) {
        const int first = forward ? e : e + 1;  // chunk whose transfer the window starts with
        double P[BS][BS];
        for (int p = 0; p < BS; ++p)
            for (int q = 0; q < BS; ++q) P[p][q] = p == q ? 1.0 : 0.0;
        int r = 0;
        for (;;) {
            const int k = forward ? first - r : first + r;
            double M[BS][BS], T1[BS][BS];
            for (int p = 0; p < BS; ++p)
                for (int q = 0; q < BS; ++q) M[p][q] = (double)maps[(size_t)k * B2 + p * BS + q];
            f_mm<double, BS>(P, M, T1);
            double nrm = 0.0;
            for (int p = 0; p < BS; ++p) {
                double rs = 0.0;
                for (int q = 0; q < BS; ++q) { P[p][q] = T1[p][q]; rs += fabs(T1[p][q]); }
                nrm = fmax(nrm, rs);
            }
            ++r;
            const bool at_end = forward ? (k == 0) : (k == tact - 1);
            if (nrm <= tau || at_end || r > kFacMaxReach) break;
        }
        reach = max(reach, r);
        if (reach > kFacMaxReach) break;
    }
    return reach;
}

template <typename TS>
__global__ void fac_precompute_kernel(const LineDesc<TS> *__restrict__ descs, int nlines, double *ws,
                                      int *status) {
    const int line = blockIdx.x * blockDim.x + threadIdx.x;
    if (line >= nlines) return;
    const LineDesc<TS> d = descs[line];
    const FacGeom g = fac_geom(d.method, d.N);
    double *w = ws + (size_t)line * kFacWs;
    TS *rec = d.sep;
    TS *eH = rec + fac_chunk_elems(g), *eT = eH + fac_e_stride(g);
    double dBh[9], dBt[9];
    bool ok = fac_end(d, g, 0, w, eH, dBh) && fac_end(d, g, 1, w, eT, dBt);
    if (ok) ok = d.method == kCFD ? fac_chunks_fp64<TS, 2>(d, g, dBh, dBt, rec)
                                  : fac_chunks_fp64<TS, 3>(d, g, dBh, dBt, rec);
    if (!ok) { atomicExch(status, 1); return; }
    const double tau = sizeof(TS) == 4 ? 0x1p-40 : 0x1p-70;
    const TS *F = rec + fac_part(g), *H = rec + (size_t)2 * fac_part(g);
    const int rf = d.method == kCFD ? fac_reach<TS, 2>(F, g.tact, tau, true) : fac_reach<TS, 3>(F, g.tact, tau, true);
    const int rb = d.method == kCFD ? fac_reach<TS, 2>(H, g.tact, tau, false) : fac_reach<TS, 3>(H, g.tact, tau, false);
    TS *info = rec + fac_info(g);
    info[0] = (TS)rf;
    info[1] = (TS)rb;
    info[2] = info[3] = (TS)0;
    atomicMax(status + 1, max(rf, rb));
}

// ---------------------------------------------------------------------------------------
// Affine maps z -> m z + off and their segmented scans over the chunks of a line.
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
__device__ __forceinline__ void map_shfl(Map<T, BS> &dst, const Map<T, BS> &src, int delta, bool up, int width) {
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

// Barrier of the compute warps (named barrier 1; the staging warp does not take part).
__device__ __forceinline__ void workers_sync() {
    asm volatile("bar.sync 1, %0;" ::"r"(kFacWorkers) : "memory");
}

// Scan buffers of a CTA: warp aggregates and warp prefixes.
template <typename T, int BS>
struct ScanSmem {
    Map<T, BS> agg[kFacThreads / 32];
    T pre[kFacThreads / 32][BS];
};

// Exclusive scan over the Tl chunk-threads of each line (lines occupy aligned groups of Tl
// consecutive threads; threads past the last whole line of the CTA take part in the warp
// shuffles only).  forward: z(c) = (a_{c-1} o ... o a_0)(0), the value entering chunk c;
// backward: z(c) = (a_{c+1} o ... o a_{Tl-1})(0), the value after chunk c.  Every thread of
// the CTA must call it with the same Tl.
template <typename T, int BS>
__device__ __forceinline__ void seg_scan(Map<T, BS> a, bool forward, int Tl, T (&z)[BS], ScanSmem<T, BS> &sm) {
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int width = Tl < 32 ? Tl : 32;
    const int pos = forward ? (lane % width) : (width - 1 - lane % width);
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        if (s >= width) break;
        Map<T, BS> o;
        map_shfl<T, BS>(o, a, s, forward, width);
        if (pos >= s) map_after<T, BS>(a, o);
    }
    Map<T, BS> ex;
    map_shfl<T, BS>(ex, a, 1, forward, width);
    if (pos == 0) map_id<T, BS>(ex);
    if (Tl <= 32) {
#pragma unroll
        for (int i = 0; i < BS; ++i) z[i] = ex.off[i];
        return;
    }
    const int nw = Tl >> 5;          // warps per line
    const int wl = warp % nw;        // warp index within its line
    const bool whole = (tid / Tl) < (kFacWorkers / Tl);  // inside a whole line of the CTA
    if (pos == 31) sm.agg[warp] = a;  // the warp's full composition
    workers_sync();
    if (whole && wl == 0 && lane == 0) {
        T p[BS];
#pragma unroll
        for (int i = 0; i < BS; ++i) p[i] = T(0);
        for (int k = 0; k < nw; ++k) {
            const int w = warp + (forward ? k : nw - 1 - k);
#pragma unroll
            for (int i = 0; i < BS; ++i) sm.pre[w][i] = p[i];
            const Map<T, BS> &ag = sm.agg[w];
            T q[BS];
#pragma unroll
            for (int i = 0; i < BS; ++i) {
                T acc = ag.off[i];
#pragma unroll
                for (int k2 = 0; k2 < BS; ++k2) acc += ag.m[i][k2] * p[k2];
                q[i] = acc;
            }
#pragma unroll
            for (int i = 0; i < BS; ++i) p[i] = q[i];
        }
    }
    workers_sync();
#pragma unroll
    for (int i = 0; i < BS; ++i) {
        T acc = ex.off[i];
#pragma unroll
        for (int k = 0; k < BS; ++k) acc += ex.m[i][k] * sm.pre[warp][k];
        z[i] = acc;
    }
}

// Block inverse of the line kernel: the FP32 path takes the hardware reciprocal
// approximation (relative error below 2^-22), FP64 an IEEE division.
__device__ __forceinline__ float fac_rcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double fac_rcp(double x) { return 1.0 / x; }
template <typename T, int BS>
__device__ __forceinline__ void fac_inv(const T (&S)[BS][BS], T (&R)[BS][BS]) {
    if constexpr (BS == 2) {
        const T id = fac_rcp(S[0][0] * S[1][1] - S[0][1] * S[1][0]);
        R[0][0] = S[1][1] * id; R[0][1] = -S[0][1] * id;
        R[1][0] = -S[1][0] * id; R[1][1] = S[0][0] * id;
    } else {
        const T c00 = S[1][1] * S[2][2] - S[1][2] * S[2][1];
        const T c01 = S[1][2] * S[2][0] - S[1][0] * S[2][2];
        const T c02 = S[1][0] * S[2][1] - S[1][1] * S[2][0];
        const T id = fac_rcp(S[0][0] * c00 + S[0][1] * c01 + S[0][2] * c02);
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
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_to_smem(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
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
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity, int polls = 1 << 22) {
    for (int i = 0; i < polls; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__host__ __device__ inline unsigned round16(unsigned b) { return (b + 15u) & ~15u; }

// Bulk copies (shared -> global) of the staged outputs of a solved group, issued by the lanes
// of the staging warp once the compute warps have released the stage (lane k takes lines k,
// k + 32, ...); each line's pressure output (in place of its pressure line) and v' (in place
// of alpha).  Lines shorter than a warp were stored directly by the compute warps.  Returns
// once this lane's copies have read the stage.
template <typename T>
__device__ void fac_store_outputs(const unsigned char *stage, int lane) {
    const FacGroup &gr = *(const FacGroup *)stage;
    if (gr.T < 32) return;
    const LineDesc<T> *descs = (const LineDesc<T> *)(stage + kFacGroupBytes);
    const T *base = (const T *)(stage + fac_head_bytes(gr.nl));
    // stored spans [sp0, sp1) and [sv0, sv1): 4-element-aligned starts, lengths rounded up to
    // 16 bytes only at the line's end (inside the padded line)
    const unsigned pbytes = round16((unsigned)(gr.sp1 - gr.sp0) * (unsigned)sizeof(T));
    const unsigned vbytes = round16((unsigned)(gr.sv1 - gr.sv0) * (unsigned)sizeof(T));
    for (int l = lane; l < gr.nl; l += 32) {
        const T *sp = base + (size_t)l * gr.ls - gr.lo;  // staged element k at sp[k]
        if (pbytes)
            asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(descs[l].po + gr.sp0),
                         "r"(smem_addr(sp + gr.sp0)), "r"(pbytes)
                         : "memory");
        if (vbytes)
            asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(descs[l].vo + gr.sv0),
                         "r"(smem_addr(sp + 2 * gr.lp + gr.sv0)), "r"(vbytes)
                         : "memory");
    }
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// The staging warp: stage one line group (descriptors, then per line the pressure, velocity
// and alpha lines and the record) into shared memory.  Lane 0 announces the group's bytes on the
// stage's "full" barrier (its only arrival) and copies the header and the descriptors; lane k
// reads the descriptors of lines k, k + 32, ... from global memory and issues their copies, so
// that a group of many short lines costs one round trip for its descriptors, not one per line.
// A sub-line of a split line stages its span of the three lines and, of the record, its chunks'
// S, F and H parts, the end tables it holds and the reach.  Every source starts on a 16-byte
// boundary (padded leading dimensions; spans start at multiples of four elements; record parts
// are padded to four elements and sub-line ranges start at multiples of four chunks) and the
// copies, rounded up to 16 bytes, stay inside the padded line or the record.
template <typename T, int BS, bool SPLIT>
__device__ void fac_issue(const LineDesc<T> *__restrict__ descs, const FacGroup *gp, unsigned char *stage,
                          unsigned long long *bar, int lane) {
    const FacGroup &gr = *gp;
    const int Lp = gr.lp, lo = SPLIT ? gr.lo : 0;
    const unsigned bp = round16((unsigned)gr.pn * (unsigned)sizeof(T));
    const unsigned bv = round16((unsigned)gr.vn * (unsigned)sizeof(T));
    const unsigned br = (unsigned)(gr.info + 4) * (unsigned)sizeof(T);  // the staged record
    const unsigned bd = (unsigned)(gr.nl * kDescBytes);
    const unsigned bg = (unsigned)sizeof(FacGroup);
    if (lane == 0) {
        mbar_expect_tx(bar, bg + bd + (unsigned)gr.nl * (2 * bp + bv + br));
        bulk_to_smem(stage, gp, bg, bar);
        bulk_to_smem(stage + kFacGroupBytes, descs + gr.first, bd, bar);
    }
    __syncwarp();  // the group's bytes are announced before any line copy is issued
    T *base = (T *)(stage + fac_head_bytes(gr.nl));
    for (int l = lane; l < gr.nl; l += 32) {
        const LineDesc<T> &d = descs[gr.first + l];
        T *ln = base + (size_t)l * gr.ls;
        bulk_to_smem(ln, d.p + lo, bp, bar);
        bulk_to_smem(ln + Lp, d.v + lo, bv, bar);
        bulk_to_smem(ln + 2 * Lp, d.alpha + lo, bp, bar);
        if constexpr (!SPLIT) {
            bulk_to_smem(ln + 3 * Lp, d.sep, br, bar);
        } else {
            const FacGeom g = fac_geom(BS == 2 ? kCFD : kMFD, gr.N);
            const int pg = fac_part(g), es = fac_e_stride(g);
            const size_t cs = (size_t)gr.c0 * (BS * BS);
            const unsigned bpart = (unsigned)gr.part * (unsigned)sizeof(T);
            const unsigned be = (unsigned)es * (unsigned)sizeof(T);
            T *rec = ln + 3 * Lp;
            const T *src = d.sep;
            bulk_to_smem(rec, src + cs, bpart, bar);
            bulk_to_smem(rec + gr.part, src + pg + cs, bpart, bar);
            bulk_to_smem(rec + 2 * gr.part, src + 2 * pg + cs, bpart, bar);
            if (gr.eh >= 0) bulk_to_smem(rec + gr.eh, src + 3 * pg, be, bar);
            if (gr.et >= 0) bulk_to_smem(rec + gr.et, src + 3 * pg + es, be, bar);
            bulk_to_smem(rec + gr.info, src + 3 * pg + 2 * es, 4u * (unsigned)sizeof(T), bar);
        }
    }
}

// W consecutive shared-memory elements into registers (8-byte loads for float when the
// source is 8-byte aligned).
template <typename T, int W>
__device__ __forceinline__ void load_win(const T *src, T (&w)[W]) {
    if constexpr (sizeof(T) == 4 && W % 2 == 0) {
        if ((smem_addr(src) & 7u) == 0) {
#pragma unroll
            for (int k = 0; k < W; k += 2) {
                const float2 q = *reinterpret_cast<const float2 *>(src + k);
                w[k] = q.x;
                w[k + 1] = q.y;
            }
            return;
        }
    }
#pragma unroll
    for (int k = 0; k < W; ++k) w[k] = src[k];
}

// BS x BS block from shared memory (16-byte load for a 2x2 FP32 block: records are 16-byte
// aligned and 2x2 blocks lie on 16-byte boundaries).
template <typename T, int BS>
__device__ __forceinline__ void load_blk(const T *src, T (&M)[BS][BS]) {
    if constexpr (sizeof(T) == 4 && BS == 2) {
        const float4 q = *reinterpret_cast<const float4 *>(src);
        M[0][0] = q.x; M[0][1] = q.y; M[1][0] = q.z; M[1][1] = q.w;
    } else {
#pragma unroll
        for (int p = 0; p < BS; ++p)
#pragma unroll
            for (int q = 0; q < BS; ++q) M[p][q] = src[p * BS + q];
    }
}

// Windowed scan value of chunk c (see the header): forward, the value entering c from the
// `reach` chunks before it, z <- F_k z + o_k for k = max(0, c - reach) .. c-1; backward, the
// value after c from the chunks after it, z <- H_k z + o_k for k = min(tact-1, c + reach) ..
// c+1.  maps: the line's F or H blocks; off: the line's chunk offsets (BS per chunk).
template <typename T, int BS>
__device__ __forceinline__ void win_scan(bool forward, int c, int tact, int reach, const T *maps, const T *off,
                                         T (&z)[BS]) {
#pragma unroll
    for (int p = 0; p < BS; ++p) z[p] = T(0);
    const int k0 = forward ? max(0, c - reach) : min(tact - 1, c + reach);
    const int n = forward ? c - k0 : k0 - c;
#pragma unroll 4
    for (int t = 0; t < n; ++t) {
        const int k = forward ? k0 + t : k0 - t;
        T M[BS][BS];
        load_blk<T, BS>(maps + k * BS * BS, M);
        T nz[BS];
#pragma unroll
        for (int p = 0; p < BS; ++p) {
            T acc = off[k * BS + p];
#pragma unroll
            for (int q = 0; q < BS; ++q) acc += M[p][q] * z[q];
            nz[p] = acc;
        }
#pragma unroll
        for (int p = 0; p < BS; ++p) z[p] = nz[p];
    }
}

// ---------------------------------------------------------------------------------------
// One line group from its staged inputs: nl lines of one simulation and direction, Tl
// threads per line; thread (l, c) = (tid / Tl, tid % Tl) owns middle blocks [c MM, c MM + MM).
// ---------------------------------------------------------------------------------------
template <typename T, int BS, int MM, bool SPLIT>
__device__ __forceinline__ void fac_group(unsigned char *stage_raw, int natural, ScanSmem<T, BS> &ssm,
                                          T *offf, T *offb) {
    static_assert(MM >= 2, "chunks of at least two blocks");
    using E = FacEnd<BS>;
    constexpr int W = E::W;
    static_assert(2 * W <= 32, "a window row fits one warp");
    constexpr int B2 = BS * BS;
    const int tid = threadIdx.x, lane = tid & 31;
    const FacGroup &gr = *(const FacGroup *)stage_raw;  // staged with the lines
    const LineDesc<T> *descs = (const LineDesc<T> *)(stage_raw + kFacGroupBytes);
    T *stage = (T *)(stage_raw + fac_head_bytes(gr.nl));
    const int N = gr.N, Tl = gr.T, tact = gr.tact;  // tact: chunks of the group's range
    const int Lp = gr.lp;
    const int l = Tl > 1 ? (int)__umulhi((unsigned)tid, gr.tdiv) : tid, c = tid - l * Tl;  // c: local chunk
    // a sub-line of a split line (SPLIT) covers the chunks c0 .. c0 + tact - 1 of its line
    const int cg = SPLIT ? gr.c0 + c : c;  // global chunk
    const int own = gr.own, ol0 = own & 511, ol1 = (own >> 9) & 511;
    const bool full_scan = (own & kFacOwnFull) != 0;
    const bool has_head = !SPLIT || (own & kFacOwnHead) != 0, has_tail = !SPLIT || (own & kFacOwnTail) != 0;
    const bool line_ok = l < gr.nl;
    const bool act = line_ok && c < tact;
    const bool owned = SPLIT ? act && c >= ol0 && c < ol1 : act;  // writes its outputs
    // an owned chunk at either end of a sub-line's owned span has outputs outside the
    // bulk-stored spans
    const bool edge = SPLIT && (c == ol0 || c == ol1 - 1);
    const int ll = line_ok ? l : 0;
    const LineDesc<T> &d = descs[ll];
    T *lb = stage + (size_t)ll * gr.ls;     // the line's staged block
    T *sPw = SPLIT ? lb - gr.lo : lb;       // staged element k of the pressure line at sPw[k]
    const T *sP = sPw;
    const T *sV = sP + Lp, *sA = sP + 2 * Lp, *sR = lb + 3 * Lp;
    const T *eH = sR + gr.eh, *eT = sR + gr.et;
    const int pl = gr.pl;
    constexpr int Z = E::Z;
    const T *sinfo = sR + gr.info;
    T *lofff = offf + (tid - c) * BS, *loffb = offb + (tid - c) * BS;  // this line's chunk offsets
    const T ih = sizeof(T) == 4 ? (T)gr.ihf : (T)gr.ih, beta = sizeof(T) == 4 ? (T)gr.betaf : (T)gr.beta;
    // segment of lanes that evaluates a line end: the whole warp for Tl >= 32, else the line
    const int S = Tl < 32 ? Tl : 32;
    const int ls = c & (S - 1);           // lane index within the segment (S a power of two)
    const int sbase = lane - ls;          // first lane of the segment
    const int wl = c >> 5;                // warp index within the line (Tl >= 32)
    const bool head_seg = has_head && (Tl < 32 || wl == 0);
    const bool tail_seg = has_tail && (Tl < 32 || wl == ((tact - 1) >> 5));
    const bool is_tail = act && has_tail && c == tact - 1;
    const int opT = pl + 1 - W, ovT = N + 1 - W;  // tail windows

    // ---- right-hand sides and the alpha window ----
    constexpr int NA = (BS == 2) ? MM + 2 : 3 * MM;
    T aw[NA];     // CFD: 3 alpha / h at nodes jb-1 .. jb+MM;  MFD: alpha at the chunk's cells
    T Y[MM][BS];  // r, then y, then x
    const int jb = gr.mid + cg * MM;      // CFD: first node of the chunk
    const int cb = gr.mid + 3 * cg * MM;  // MFD: first cell of the chunk
    if (act) {
        if constexpr (BS == 2) {
            const T c3 = T(3) * ih;
            T w[MM + 2];
            load_win<T, MM + 2>(sA + jb - 1, w);
#pragma unroll
            for (int k = 0; k < NA; ++k) aw[k] = c3 * w[k];
            load_win<T, MM + 2>(sV + jb - 1, w);
#pragma unroll
            for (int i = 0; i < MM; ++i) Y[i][0] = c3 * (w[i + 2] - w[i]);
            load_win<T, MM + 2>(sP + jb - 1, w);
#pragma unroll
            for (int i = 0; i < MM; ++i) Y[i][1] = c3 * (w[i + 2] - w[i]);
        } else {
#pragma unroll
            for (int k = 0; k < NA; ++k) aw[k] = sA[cb + k];
            T vw[3 * MM + 3];
#pragma unroll
            for (int k = 0; k < 3 * MM + 3; ++k) vw[k] = sV[cb - 2 + k];
            const T w0 = T(1.0 / 24.0), w1 = T(-9.0 / 8.0), w2 = T(9.0 / 8.0), w3 = T(-1.0 / 24.0);
#pragma unroll
            for (int i = 0; i < MM; ++i)
#pragma unroll
                for (int m = 0; m < 3; ++m) {
                    const int k = 3 * i + m;
                    const T dv = w0 * vw[k] + w1 * vw[k + 1] + w2 * vw[k + 2] + w3 * vw[k + 3];
                    Y[i][m] = sP[cb + k] - aw[k] * ih * dv;
                }
        }
    }

    // ---- head / tail corrections of the adjacent blocks' right-hand sides (KZ z) ----
    auto zval = [&](bool tail, int k) -> T {
        return k < W ? sP[(tail ? opT : 0) + k] : sV[(tail ? ovT : 0) + k - W];
    };
    // Window parts (first 2W terms) of the end-region rows HZ and DZ, known once the line is
    // staged: computed now by threads spread over the line and kept in the line's scratch, so
    // that at the end the end-region lanes add only the adjacent block's BS terms.
    // Row r < NR1 belongs to the head, r >= NR1 to the tail; within an end, HZ rows come first.
    constexpr int NR1 = E::HMAX + (BS == 3 ? E::HMAX + 2 : 0), NR = 2 * NR1;
    T *scr = lb + gr.scr;
    // Lines of at least three warps: the warps other than the head and tail warps compute the
    // rows after their local forward pass (below), while the end warps form KZ z.
    const bool scr_help = Tl >= 96;
    if (line_ok && !scr_help) {
        auto row_win = [&](int r) {
            const bool tail = r >= NR1;
            if (!(tail ? has_tail : has_head)) return;
            const int q = tail ? r - NR1 : r;
            const T *row = (tail ? eT : eH) + (q < E::HMAX ? E::HZ + q * Z : E::DZ + (q - E::HMAX) * Z);
            T a0 = T(0), a1 = T(0);
#pragma unroll
            for (int k = 0; k < 2 * W; k += 2) {
                a0 += row[k] * zval(tail, k);
                a1 += row[k + 1] * zval(tail, k + 1);
            }
            scr[r] = a0 + a1;
        };
        const int stride = Tl >= NR ? Tl / NR : 1;
        if (stride > 1) {
            if (c % stride == 0 && c / stride < NR) row_win(c / stride);
        } else {
            for (int r = c; r < NR; r += Tl) row_win(r);
        }
    }
    auto seg_kz = [&](bool tail, T (&out)[BS]) {
        const T *kz = (tail ? eT : eH);
        if (S == 32) {  // one window term per lane (2W <= 32), then a warp sum
            const int k = ls;
            const bool has = k < 2 * W;
            const T *zp = k < W ? sP + (tail ? opT : 0) + k : sV + (tail ? ovT : 0) + (k - W);
            const T z = has ? *zp : T(0);
#pragma unroll
            for (int p = 0; p < BS; ++p) out[p] = has ? kz[p * 2 * W + k] * z : T(0);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                for (int p = 0; p < BS; ++p) out[p] += __shfl_xor_sync(0xffffffffu, out[p], o);
            return;
        }
#pragma unroll
        for (int p = 0; p < BS; ++p) {
            T acc = T(0);
            for (int k = ls; k < 2 * W; k += S) acc += kz[p * 2 * W + k] * zval(tail, k);
            out[p] = acc;
        }
        for (int o = S >> 1; o > 0; o >>= 1)
#pragma unroll
            for (int p = 0; p < BS; ++p) out[p] += __shfl_xor_sync(0xffffffffu, out[p], o, S);
    };
    if (head_seg) {
        T kz[BS];
        seg_kz(false, kz);
        if (act && c == 0)
#pragma unroll
            for (int p = 0; p < BS; ++p) Y[0][p] += kz[p];
    }
    if (tail_seg) {
        T kz[BS];
        seg_kz(true, kz);
        if (is_tail)
#pragma unroll
            for (int p = 0; p < BS; ++p) Y[MM - 1][p] += kz[p];
    }

    // ---- block couplings from the alpha window ----
    // CFD: A_i = [[1, -tb], [-a_i, 1]], B = 4 I, C_i = [[1, tb], [a_{i+2}, 1]] with a = aw (3 alpha
    // / h at the nodes) and tb = 3 beta / h; its products below are written out, so that no unit
    // or zero entry costs an operation.  MFD: A_i (upper triangular), B_i and C_i (lower
    // triangular) hold the 7-point operator's bands scaled per cell; its products visit the
    // nonzero entries only (the compiler keeps a product with a literal zero).
    const T tb = T(3) * ih * beta;
    auto blockA = [&](int i, T (&A)[BS][BS]) {  // MFD
        const T bh2 = beta * ih * ih;
#pragma unroll
        for (int m = 0; m < BS; ++m) {
            const T sc = aw[3 * i + m] * bh2;
#pragma unroll
            for (int q = 0; q < BS; ++q) A[m][q] = (q >= m) ? -sc * (T)mim_DG(q - m) : T(0);
        }
    };
    auto blockB = [&](int i, T (&B)[BS][BS]) {  // MFD
        const T bh2 = beta * ih * ih;
#pragma unroll
        for (int m = 0; m < BS; ++m) {
            const T sc = aw[3 * i + m] * bh2;
#pragma unroll
            for (int q = 0; q < BS; ++q) B[m][q] = (q == m ? T(1) : T(0)) - sc * (T)mim_DG(q - m + 3);
        }
    };
    auto blockC = [&](int i, T (&C)[BS][BS]) {  // MFD
        const T bh2 = beta * ih * ih;
#pragma unroll
        for (int m = 0; m < BS; ++m) {
            const T sc = aw[3 * i + m] * bh2;
#pragma unroll
            for (int q = 0; q < BS; ++q) C[m][q] = (q <= m) ? -sc * (T)mim_DG(q - m + 6) : T(0);
        }
    };
    // out = A_i v
    auto mulA = [&](int i, const T (&v)[BS], T (&out)[BS]) {
        T r[BS];
        if constexpr (BS == 2) {
            r[0] = v[0] - tb * v[1];
            r[1] = v[1] - aw[i] * v[0];
        } else {
            T A[BS][BS];
            blockA(i, A);
#pragma unroll
            for (int p = 0; p < BS; ++p) {
                T acc = A[p][p] * v[p];
#pragma unroll
                for (int q = p + 1; q < BS; ++q) acc += A[p][q] * v[q];
                r[p] = acc;
            }
        }
#pragma unroll
        for (int p = 0; p < BS; ++p) out[p] = r[p];
    };
    // out = C_i v
    auto mulC = [&](int i, const T (&v)[BS], T (&out)[BS]) {
        T r[BS];
        if constexpr (BS == 2) {
            r[0] = v[0] + tb * v[1];
            r[1] = v[1] + aw[i + 2] * v[0];
        } else {
            T C[BS][BS];
            blockC(i, C);
#pragma unroll
            for (int p = 0; p < BS; ++p) {
                T acc = C[p][0] * v[0];
#pragma unroll
                for (int q = 1; q <= p; ++q) acc += C[p][q] * v[q];
                r[p] = acc;
            }
        }
#pragma unroll
        for (int p = 0; p < BS; ++p) out[p] = r[p];
    };
    // out = -Si t
    auto neg_si = [&](const T (&Si)[BS][BS], const T (&t)[BS], T (&out)[BS]) {
        T r[BS];
#pragma unroll
        for (int p = 0; p < BS; ++p) {
            T acc = Si[p][0] * t[0];
#pragma unroll
            for (int q = 1; q < BS; ++q) acc += Si[p][q] * t[q];
            r[p] = -acc;
        }
#pragma unroll
        for (int p = 0; p < BS; ++p) out[p] = r[p];
    };

    // ---- factorisation and local forward pass ----
    T Si[MM][BS][BS];
    if (act) {
        T G[BS][BS];
#pragma unroll
        for (int i = 0; i < MM; ++i) {
            T S[BS][BS];
            if (i == 0) {
                load_blk<T, BS>(sR + c * B2, S);
            } else {
                // S_i = B_i - A_i G_{i-1}
                if constexpr (BS == 2) {
                    S[0][0] = T(4) - G[0][0] + tb * G[1][0];
                    S[0][1] = tb * G[1][1] - G[0][1];
                    S[1][0] = aw[i] * G[0][0] - G[1][0];
                    S[1][1] = T(4) - G[1][1] + aw[i] * G[0][1];
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
                            for (int k = p; k < BS; ++k) acc -= A[p][k] * G[k][q];
                            S[p][q] = acc;
                        }
                }
                if (i == MM - 1 && is_tail) {
#pragma unroll
                    for (int p = 0; p < BS; ++p)
#pragma unroll
                        for (int q = 0; q < BS; ++q) S[p][q] -= eT[E::DB + p * BS + q];
                }
            }
            fac_inv<T, BS>(S, Si[i]);
            // y_i = Si_i (r_i - A_i y_{i-1})
            T t[BS];
            if (i == 0) {
#pragma unroll
                for (int p = 0; p < BS; ++p) t[p] = Y[0][p];
            } else if constexpr (BS == 2) {
                t[0] = Y[i][0] - Y[i - 1][0] + tb * Y[i - 1][1];
                t[1] = Y[i][1] - Y[i - 1][1] + aw[i] * Y[i - 1][0];
            } else {
                T A[BS][BS];
                blockA(i, A);
#pragma unroll
                for (int p = 0; p < BS; ++p) {
                    T acc = Y[i][p];
#pragma unroll
                    for (int q = p; q < BS; ++q) acc -= A[p][q] * Y[i - 1][q];
                    t[p] = acc;
                }
            }
#pragma unroll
            for (int p = 0; p < BS; ++p) {
                T acc = Si[i][p][0] * t[0];
#pragma unroll
                for (int q = 1; q < BS; ++q) acc += Si[i][p][q] * t[q];
                Y[i][p] = acc;
            }
            if (i + 1 < MM) {  // G_i = Si_i C_i
                if constexpr (BS == 2) {
                    const T a2 = aw[i + 2];
                    G[0][0] = Si[i][0][0] + Si[i][0][1] * a2;
                    G[0][1] = Si[i][0][0] * tb + Si[i][0][1];
                    G[1][0] = Si[i][1][0] + Si[i][1][1] * a2;
                    G[1][1] = Si[i][1][0] * tb + Si[i][1][1];
                } else {
                    T C[BS][BS];
                    blockC(i, C);
#pragma unroll
                    for (int p = 0; p < BS; ++p)
#pragma unroll
                        for (int q = 0; q < BS; ++q) {
                            T acc = Si[i][p][q] * C[q][q];
#pragma unroll
                            for (int k = q + 1; k < BS; ++k) acc += Si[i][p][k] * C[k][q];
                            G[p][q] = acc;
                        }
                }
            }
        }
    }

    // ---- window parts of the end-region rows by the middle warps (one row per half-warp,
    // one or two terms per lane, then a half-warp sum) ----
    if (scr_help && line_ok) {
        const int tw = (tact - 1) >> 5;  // the tail warp (tact > 64, so 2 <= tw)
        if (wl != 0 && wl != tw) {
            const int hi = wl - 1 - (wl > tw ? 1 : 0), nh = (Tl >> 5) - 2;
            const int half = lane >> 4, k = lane & 15;
            for (int r0 = 2 * hi; r0 < NR; r0 += 2 * nh) {  // warp-uniform trip count
                const int r = r0 + half;
                const bool tail = r >= NR1;
                const int q = tail ? r - NR1 : r;
                T a = T(0);
                const bool here = r < NR && (tail ? has_tail : has_head);
                if (here) {
                    const T *row = (tail ? eT : eH) + (q < E::HMAX ? E::HZ + q * Z : E::DZ + (q - E::HMAX) * Z);
                    a = row[k] * zval(tail, k);
                    if (k + 16 < 2 * W) a += row[k + 16] * zval(tail, k + 16);
                }
#pragma unroll
                for (int o = 8; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
                if (k == 0 && here) scr[r] = a;
            }
        }
    }

    // ---- forward scan: the true y entering the chunk; correction ----
    T yin[BS];
    if (full_scan) {
        Map<T, BS> mp;
        if (act) {
            load_blk<T, BS>(sR + gr.part + c * B2, mp.m);
#pragma unroll
            for (int p = 0; p < BS; ++p) mp.off[p] = Y[MM - 1][p];
        } else {
            map_id<T, BS>(mp);
        }
        seg_scan<T, BS>(mp, true, Tl, yin, ssm);
    } else {
        if (act)
#pragma unroll
            for (int p = 0; p < BS; ++p) lofff[c * BS + p] = Y[MM - 1][p];
        workers_sync();
        if (act) win_scan<T, BS>(true, c, tact, (int)sinfo[0], sR + gr.part, lofff, yin);
    }
    if (act) {
        T dl[BS];
#pragma unroll
        for (int p = 0; p < BS; ++p) dl[p] = yin[p];
#pragma unroll
        for (int i = 0; i < MM; ++i) {  // d_i = -Si_i A_i d_{i-1}
            T t[BS];
            mulA(i, dl, t);
            neg_si(Si[i], t, dl);
#pragma unroll
            for (int p = 0; p < BS; ++p) Y[i][p] += dl[p];
        }
        // local backward pass (x = 0 after the chunk): x_i = y_i - Si_i (C_i x_{i+1})
#pragma unroll
        for (int i = MM - 2; i >= 0; --i) {
            T t[BS], u[BS];
            mulC(i, Y[i + 1], t);
            neg_si(Si[i], t, u);
#pragma unroll
            for (int p = 0; p < BS; ++p) Y[i][p] += u[p];
        }
    }

    // ---- backward scan: the true x after the chunk; correction ----
    T xin[BS];
    if (full_scan) {
        Map<T, BS> mp;
        if (act) {
            load_blk<T, BS>(sR + 2 * gr.part + c * B2, mp.m);
#pragma unroll
            for (int p = 0; p < BS; ++p) mp.off[p] = Y[0][p];
        } else {
            map_id<T, BS>(mp);
        }
        seg_scan<T, BS>(mp, false, Tl, xin, ssm);
    } else {
        if (offb == offf) workers_sync();  // one offset buffer: the forward reads are done
        if (act)
#pragma unroll
            for (int p = 0; p < BS; ++p) loffb[c * BS + p] = Y[0][p];
        workers_sync();
        if (act) win_scan<T, BS>(false, c, tact, (int)sinfo[1], sR + 2 * gr.part, loffb, xin);
    }
    if (act) {
        T ep[BS];
#pragma unroll
        for (int p = 0; p < BS; ++p) ep[p] = xin[p];
#pragma unroll
        for (int i = MM - 1; i >= 0; --i) {  // e_i = -Si_i C_i e_{i+1}
            T t[BS];
            mulC(i, ep, t);
            neg_si(Si[i], t, ep);
#pragma unroll
            for (int p = 0; p < BS; ++p) Y[i][p] += ep[p];
        }
    }

    // ---- outputs: C = 2 u* - a (+ source), v' = 2 v* - v, optionally natural u, w ----
    T *__restrict__ gpo = d.po;
    T *__restrict__ gvo = d.vo;
    T *__restrict__ uo = natural ? d.u_out : nullptr;
    T *__restrict__ wo = natural ? d.w_out : nullptr;
    const long long spo = d.spo, svo = d.svo, snp = d.snp, snv = d.snv;
    const int src_k = d.src_k;
    // Lines of at least a warp stage their outputs in shared memory and leave with one bulk
    // copy per line and array: the pressure output in place of the pressure line, v' in
    // place of alpha.  Both are dead once the solve is done, and every thread reads them only
    // at the points it writes, before writing there.  Shorter lines store directly.
    const bool stage_v = Tl >= 32;
    T *sOut = sPw + 2 * Lp;
    // source term dt/2 f(t_{m+1}) added by the thread that wrote pressure point src_k
    // staged in shared memory inside the bulk-stored spans, stored directly outside them
    const int sp0 = gr.sp0, sp1 = gr.sp1, sv0 = gr.sv0, sv1 = gr.sv1;
    auto staged_p = [&](int k) { return SPLIT ? stage_v && k >= sp0 && k < sp1 : stage_v; };
    auto staged_v = [&](int j) { return SPLIT ? stage_v && j >= sv0 && j < sv1 : stage_v; };
    auto add_source = [&]() {
        const long long m = *d.clock;
        const T s = (T)(d.src_scale * ricker(d.src_amp, d.src_f0, d.src_tdelay, (double)(m + 1) * d.dt));
        if (staged_p(src_k)) sPw[src_k] += s; else gpo[src_k * spo] = gpo[src_k * spo] + s;
        if (d.advance_clock) *d.clock = m + 1;
    };
    // the fourth-order staggered difference of four consecutive values, up to the factor 1/h
    auto d4 = [](T a, T b, T c, T d) {
        return fma_rn(T(-1.0 / 24.0), d, fma_rn(T(9.0 / 8.0), c, fma_rn(T(-9.0 / 8.0), b, T(1.0 / 24.0) * a)));
    };
    auto out_p = [&](int k, T val_out, T val_nat) {
        if (staged_p(k)) sPw[k] = val_out; else gpo[k * spo] = val_out;
        if (uo) uo[k * snp] = val_nat;
    };
    // v' = v - 2 c g and the natural w = v - c g, with g the velocity's derivative term and c its
    // factor (beta for CFD, beta/h for MFD).  The carried value is formed exactly as on the
    // staged-only paths below, so that writing natural outputs never changes the trajectory.
    auto out_v = [&](int j, T vin, T cf, T g) {
        const T val = fma_rn(-(T(2) * cf), g, vin);
        if (staged_v(j)) sOut[j] = val; else gvo[j * svo] = val;
        if (wo) wo[j * snv] = fma_rn(-cf, g, vin);
    };
    if (owned) {
        if constexpr (BS == 2) {
            // alpha at the chunk's nodes is aw / (3/h); p and v at the chunk's nodes
            const T inv_c3 = T(1) / (T(3) * ih);
            T wp[MM], wv[MM];
            load_win<T, MM>(sP + jb, wp);
            load_win<T, MM>(sV + jb, wv);
            if (stage_v && !uo && !wo && !edge) {
#pragma unroll
                for (int i = 0; i < MM; ++i) {
                    const T ae = aw[i + 1] * inv_c3 * Y[i][0];
                    sPw[jb + i] = wp[i] - T(2) * ae;
                    sOut[jb + i] = fma_rn(-(T(2) * beta), Y[i][1], wv[i]);
                }
            } else {
#pragma unroll
                for (int i = 0; i < MM; ++i) {
                    const T ae = aw[i + 1] * inv_c3 * Y[i][0];
                    out_p(jb + i, wp[i] - T(2) * ae, wp[i] - ae);
                    out_v(jb + i, wv[i], beta, Y[i][1]);
                }
            }
            if (src_k >= jb && src_k < jb + MM) add_source();
        } else {
            const T bi = beta * ih;
            if (stage_v && !uo && !wo && !edge) {
                // staged outputs only: no per-point branches; the velocities after the last
                // block of the tail chunk belong to the tail region
                const T b2 = T(2) * bi;
#pragma unroll
                for (int i = 0; i < MM; ++i) {
                    const int q0 = cb + 3 * i;
#pragma unroll
                    for (int m = 0; m < 3; ++m) sPw[q0 + m] = T(2) * Y[i][m] - sP[q0 + m];
                    const T xn0 = i + 1 < MM ? Y[i + 1 < MM ? i + 1 : i][0] : xin[0];
                    const T xn1 = i + 1 < MM ? Y[i + 1 < MM ? i + 1 : i][1] : xin[1];
                    const T xn2 = i + 1 < MM ? Y[i + 1 < MM ? i + 1 : i][2] : xin[2];
                    const T d1 = d4(Y[i][0], Y[i][1], Y[i][2], xn0);
                    const T d2 = d4(Y[i][1], Y[i][2], xn0, xn1);
                    const T d3 = d4(Y[i][2], xn0, xn1, xn2);
                    if (i + 1 < MM || !is_tail) {
                        sOut[q0 + 1] = fma_rn(-b2, d1, sV[q0 + 1]);
                        sOut[q0 + 2] = fma_rn(-b2, d2, sV[q0 + 2]);
                        sOut[q0 + 3] = fma_rn(-b2, d3, sV[q0 + 3]);
                    }
                }
                if (src_k >= cb && src_k < cb + 3 * MM) add_source();
            } else {
#pragma unroll
            for (int i = 0; i < MM; ++i) {
                const int q0 = cb + 3 * i;
#pragma unroll
                for (int m = 0; m < 3; ++m) out_p(q0 + m, T(2) * Y[i][m] - sP[q0 + m], Y[i][m]);
                // x of the next block (the next chunk's first block after the last one)
                const int in = i + 1 < MM ? i + 1 : i;
                const T xn0 = i + 1 < MM ? Y[in][0] : xin[0];
                const T xn1 = i + 1 < MM ? Y[in][1] : xin[1];
                const T xn2 = i + 1 < MM ? Y[in][2] : xin[2];
                if (!(i == MM - 1 && is_tail)) {
                    out_v(q0 + 1, sV[q0 + 1], bi, d4(Y[i][0], Y[i][1], Y[i][2], xn0));
                    out_v(q0 + 2, sV[q0 + 2], bi, d4(Y[i][1], Y[i][2], xn0, xn1));
                    out_v(q0 + 3, sV[q0 + 3], bi, d4(Y[i][2], xn0, xn1, xn2));
                }
            }
            if (src_k >= cb && src_k < cb + 3 * MM) add_source();
            }
        }
    }

    // ---- head and tail regions, evaluated by their segments ----
    auto seg_end = [&](bool tail) {
        const T *et = tail ? eT : eH;
        const int src_lane = sbase + ((tail ? tact - 1 : 0) & (S - 1));
        T xJ[BS];
#pragma unroll
        for (int b = 0; b < BS; ++b) xJ[b] = __shfl_sync(0xffffffffu, tail ? Y[MM - 1][b] : Y[0][b], src_lane);
        if (!line_ok) return;
        const int m = tail ? gr.tu : gr.hu;
        const T *pscr = scr + (tail ? NR1 : 0);
        // row = [window part (scratch) | adjacent block's BS terms]
        auto row_dot = [&](const T *row, int r) -> T {
            T acc = pscr[r];
#pragma unroll
            for (int b = 0; b < BS; ++b) acc += row[2 * W + b] * xJ[b];
            return acc;
        };
        if constexpr (BS == 2) {
            const int r0 = tail ? 2 * N - gr.tu : 0;
            if (S == 32) {
                // one row per lane (m <= HMAX < 32); every operand is read before xJ arrives,
                // and alpha by every lane before any lane writes v' over it
                const int q = ls;
                const bool has = q < m;
                const int i = r0 + (has ? q : 0);
                const bool is_g = (i == 0) || (i == 2 * N - 1) || (i % 2 == 0);
                const int node = i == 0 ? 0 : (i == 2 * N - 1 ? N : (i + 1) / 2);
                const T *row = et + E::HZ + (has ? q : 0) * Z;
                const T base = pscr[has ? q : 0], k0 = row[2 * W], k1 = row[2 * W + 1];
                const T al = sA[node], vv = sV[node], pp = sP[node];
                const T x = base + k0 * xJ[0] + k1 * xJ[1];
                if (stage_v) __syncwarp();
                if (has) {
                    if (is_g) {
                        out_v(node, vv, beta, x);
                    } else {
                        const T ae = al * x;
                        out_p(node, pp - T(2) * ae, pp - ae);
                        if (node == src_k) add_source();
                    }
                }
                return;
            }
            // one row per lane (m <= 13 < S when v' is staged): alpha is read by every lane
            // before any lane writes v' over it
            for (int q0 = 0; q0 < m; q0 += S) {
                const int q = q0 + ls;
                const bool has = q < m;
                const int i = r0 + (has ? q : 0);
                const bool is_g = (i == 0) || (i == 2 * N - 1) || (i % 2 == 0);
                const int node = i == 0 ? 0 : (i == 2 * N - 1 ? N : (i + 1) / 2);
                const T x = has ? row_dot(et + E::HZ + q * Z, q) : T(0);
                const T al = sA[node];
                if (stage_v) __syncwarp();
                if (!has) continue;
                if (is_g) {
                    out_v(node, sV[node], beta, x);
                } else {
                    const T ae = al * x;
                    out_p(node, sP[node] - T(2) * ae, sP[node] - ae);
                    if (node == src_k) add_source();
                }
            }
        } else {
            const int cell0 = tail ? N - gr.tu + 1 : 1;
            const int qb = gr.mid + 3 * ((cg - c + tact) * MM - 1);  // first cell of the last middle block
            const int jlo = tail ? qb + 1 : 0, nrow = tail ? N - qb : gr.hu + 2;
            if (S == 32) {
                // one row per lane: pressure rows on lanes 0..15 (m <= HMAX), velocity rows on
                // lanes 16..31 (nrow <= HMAX + 2)
                static_assert(E::HMAX + 2 <= 16, "end rows fit a half-warp");
                const bool vel = ls >= 16;
                const int q = vel ? ls - 16 : ls;
                const bool has = q < (vel ? nrow : m);
                const int qq = has ? q : 0;
                const T x = row_dot(et + (vel ? E::DZ : E::HZ) + qq * Z, vel ? E::HMAX + qq : qq);
                if (has) {
                    if (vel) {
                        out_v(jlo + qq, sV[jlo + qq], beta * ih, x);
                    } else {
                        const int cc = cell0 + qq;
                        out_p(cc, T(2) * x - sP[cc], x);
                        if (cc == src_k) add_source();
                    }
                }
                return;
            }
            for (int q = ls; q < m; q += S) {
                const T x = row_dot(et + E::HZ + q * Z, q);
                const int cc = cell0 + q;
                out_p(cc, T(2) * x - sP[cc], x);
                if (cc == src_k) add_source();
            }
            for (int q = ls; q < nrow; q += S) {
                const int j = jlo + q;
                out_v(j, sV[j], beta * ih, row_dot(et + E::DZ + q * Z, E::HMAX + q));
            }
        }
    };
    __syncwarp();  // scratch rows written by other lanes (lines within one warp, no scan barrier)
    if (head_seg) seg_end(false);
    if (tail_seg) seg_end(true);
    // staged outputs are written to global memory by the staging warp once every compute warp
    // has released the stage; make this thread's shared-memory writes visible to those copies
    if (stage_v) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---------------------------------------------------------------------------------------
// The kernel: persistent CTAs walk the line groups g = blockIdx.x, blockIdx.x + gridDim.x, ...
// through a ring of `stages` shared-memory stages.  The last warp stages the groups: one lane
// waits until the compute warps have released a stage (mbarrier "empty") and starts the bulk
// copies of the next group into it (mbarrier "full").  The 15 compute warps wait for "full",
// solve the group and release the stage.  Every wait is bounded; one that runs out sets *fault
// and the warp carries on with the same iteration count, so no warp is left waiting at a
// barrier and the launch ends (with garbage results and the fault flag set).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void mbar_arrive(unsigned long long *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

template <typename T, int BS, int MM, bool SPLIT>
__global__ void __launch_bounds__(kFacThreads, 1)
line_solve_factored_kernel(const LineDesc<T> *__restrict__ descs, const FacGroup *__restrict__ groups, int ngroups,
                           int natural, unsigned stage_bytes, int stages, int *fault) {
    extern __shared__ __align__(128) unsigned char fac_smem[];
    __shared__ ScanSmem<T, BS> ssm;
    __shared__ __align__(8) unsigned long long full[kFacMaxStages], empty[kFacMaxStages];
    // chunk offsets of the windowed scans: forward and backward buffers for FP32, one for FP64
    constexpr int kBufs = sizeof(T) == 4 ? 2 : 1;
    __shared__ T offs[kBufs][kFacThreads * BS];
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid == 0) {
        for (int k = 0; k < kFacMaxStages; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], kFacWorkers / 32);
        }
        mbar_fence_init();
    }
    __syncthreads();
    // the it-th group of this CTA goes to stage it % stages, as that stage's use-th group
    if (tid >= kFacWorkers) {  // the staging warp; every lane runs the same loop
        int last[kFacMaxStages];
        for (int k = 0; k < kFacMaxStages; ++k) last[k] = -1;
        int st = 0, use = 0;
        for (int gi = blockIdx.x; gi < ngroups; gi += gridDim.x) {
            unsigned char *stage = fac_smem + (size_t)st * stage_bytes;
            if (use > 0) {
                // the previous group of this stage is solved: write its outputs, then refill.
                // The copies that filled it have landed (the compute warps waited for them);
                // if a compute warp's wait ran out they may not have, so every lane waits for
                // them itself before it copies anything into the stage again.
                if (!mbar_wait(&empty[st], (unsigned)((use - 1) & 1))) atomicExch(fault, 1);
                if (!mbar_wait(&full[st], (unsigned)((use - 1) & 1))) atomicExch(fault, 1);
                fac_store_outputs<T>(stage, lane);
                __syncwarp();  // every lane's output copies have read the stage
            }
            fac_issue<T, BS, SPLIT>(descs, groups + gi, stage, &full[st], lane);
            last[st] = use;
            if (++st == stages) { st = 0; ++use; }
        }
        // the last groups of each stage: wait until solved and until their copies have
        // landed (no bulk copy into this CTA's shared memory may outlive it), write outputs
        for (int k = 0; k < stages; ++k)
            if (last[k] >= 0) {
                if (!mbar_wait(&empty[k], (unsigned)(last[k] & 1))) atomicExch(fault, 1);
                if (!mbar_wait(&full[k], (unsigned)(last[k] & 1))) atomicExch(fault, 1);
                fac_store_outputs<T>(fac_smem + (size_t)k * stage_bytes, lane);
            }
        // global visibility of this lane's output copies before the CTA ends
        asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
        return;
    }
    int st = 0, use = 0;
    for (int gi = blockIdx.x; gi < ngroups; gi += gridDim.x) {
        if (!mbar_wait(&full[st], (unsigned)(use & 1))) atomicExch(fault, 1);
        fac_group<T, BS, MM, SPLIT>(fac_smem + (size_t)st * stage_bytes, natural, ssm, offs[0], offs[kBufs - 1]);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[st]);
        if (++st == stages) { st = 0; ++use; }
    }
}

template <typename T>
cudaError_t launch_fac_precompute(const LineDesc<T> *d, int nlines, double *ws, int *status, cudaStream_t s) {
    if (nlines <= 0) return cudaSuccess;
    fac_precompute_kernel<T><<<(nlines + 63) / 64, 64, 0, s>>>(d, nlines, ws, status);
    return cudaGetLastError();
}

template <typename T, int BS, int MM, bool SPLIT>
cudaError_t launch_fac_inst(const LineDesc<T> *d, const FacGroup *groups, int ngroups, size_t stage_bytes, int stages,
                            int grid, int natural, int *fault, cudaStream_t s) {
    auto kern = line_solve_factored_kernel<T, BS, MM, SPLIT>;
    // the host sizes the ring with fac_static_smem, an upper bound of the kernel's own static
    // shared memory: check it against the compiled kernel once
    static const bool static_ok = [&] {
        cudaFuncAttributes a{};
        return cudaFuncGetAttributes(&a, kern) == cudaSuccess && a.sharedSizeBytes <= fac_static_smem(sizeof(T), BS);
    }();
    if (!static_ok) return cudaErrorInvalidConfiguration;
    const size_t dyn = (size_t)stages * stage_bytes;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
    kern<<<grid, kFacThreads, dyn, s>>>(d, groups, ngroups, natural, (unsigned)stage_bytes, stages, fault);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_line_solve_factored(const LineDesc<T> *d, const FacGroup *groups, int ngroups, int variant,
                                       size_t stage_bytes, int stages, int grid, int natural, int *fault,
                                       cudaStream_t s) {
    if (ngroups <= 0) return cudaSuccess;
    if (grid > ngroups) grid = ngroups;
    if (stages < 1 || stages > kFacMaxStages) return cudaErrorInvalidValue;
    switch (variant) {
    case 0: return launch_fac_inst<T, 2, 9, false>(d, groups, ngroups, stage_bytes, stages, grid, natural, fault, s);
    case 1: return launch_fac_inst<T, 3, 2, false>(d, groups, ngroups, stage_bytes, stages, grid, natural, fault, s);
    case 2: return launch_fac_inst<T, 3, 3, false>(d, groups, ngroups, stage_bytes, stages, grid, natural, fault, s);
    case 3: return launch_fac_inst<T, 2, 9, true>(d, groups, ngroups, stage_bytes, stages, grid, natural, fault, s);
    case 4: return launch_fac_inst<T, 3, 3, true>(d, groups, ngroups, stage_bytes, stages, grid, natural, fault, s);
    }
    return cudaErrorInvalidValue;
}

template cudaError_t launch_fac_precompute<float>(const LineDesc<float> *, int, double *, int *, cudaStream_t);
template cudaError_t launch_fac_precompute<double>(const LineDesc<double> *, int, double *, int *, cudaStream_t);
template cudaError_t launch_line_solve_factored<float>(const LineDesc<float> *, const FacGroup *, int, int, size_t, int,
                                                       int, int, int *, cudaStream_t);
template cudaError_t launch_line_solve_factored<double>(const LineDesc<double> *, const FacGroup *, int, int, size_t,
                                                        int, int, int, int *, cudaStream_t);

// The bounded wait's failure path, run on purpose: one thread waits on an mbarrier that
// nothing arrives at, with `polls` polls at most, and records whether the wait gave up (and
// the time it took).  No other thread or copy is involved, so the kernel always ends.
__global__ void wait_timeout_probe_kernel(int polls, int *gave_up, long long *cycles) {
    __shared__ __align__(8) unsigned long long bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    mbar_fence_init();
    const long long t0 = clock64();
    const bool ok = mbar_wait(&bar, 0u, polls);
    *cycles = clock64() - t0;
    *gave_up = ok ? 0 : 1;
}

}  // namespace adi

extern "C" int adi_selftest_wait_timeout(int polls, int *gave_up, long long *cycles) {
    if (polls < 1 || polls > (1 << 22) || !gave_up) return ADI_EINVAL;
    int *d_flag = nullptr;
    long long *d_cyc = nullptr;
    cudaError_t e = cudaMalloc(&d_flag, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&d_cyc, sizeof(long long));
    if (e == cudaSuccess) {
        adi::wait_timeout_probe_kernel<<<1, 32>>>(polls, d_flag, d_cyc);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(gave_up, d_flag, sizeof(int), cudaMemcpyDeviceToHost);
    long long c = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&c, d_cyc, sizeof(long long), cudaMemcpyDeviceToHost);
    if (cycles) *cycles = c;
    if (d_flag) cudaFree(d_flag);
    if (d_cyc) cudaFree(d_cyc);
    if (e != cudaSuccess) { (void)cudaGetLastError(); return e == cudaErrorNoDevice ? ADI_ENOTSUP : ADI_ECUDA; }
    return ADI_OK;
}
