// adi_kernels.cu -- line kernels of the Peaceman-Rachford ADI step (arXiv 2006.07583,
// Sec. 2, Eqs. 6-10 and 12) for sm_103a.
//
//   precompute  FP64, once per line: eliminates the one-sided boundary rows of App. A/B
//               (head and tail of every line system) into small tables.
//   prologue    turns natural fields (u, v, w) into the carried stage-1 state
//               a = u - alpha Dbar_y w + dt/2 f and w* = w - beta D_y u (Eq. 8's A and
//               Alg. 1/2's W*).
//   line_solve  one half step on a set of lines, thread per line: builds the block
//               tridiagonal line system on the fly from alpha and the stencils, block
//               Thomas forward sweep (factors kept in a global scratch), backward sweep,
//               then the carried outputs C = 2u* - a (+ dt/2 f), v' = 2v* - v.
//   finite      NaN/Inf scan of a field.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <vector>

#include "adi_internal.h"
#include "adi_ops.cuh"
#include "adi_line.cuh"

namespace adi {

// One thread per line: head and tail elimination tables.
template <typename T>
__global__ void precompute_kernel(const LineDesc<T> *__restrict__ descs, int nlines,
                                  T *tab_out_base, int *status) {
    int line = blockIdx.x * blockDim.x + threadIdx.x;
    if (line >= nlines) return;
    const LineDesc<T> d = descs[line];
    const LineShape s = line_shape(d.method, d.N);
    T *tab = tab_out_base + (size_t)line * kTabLine;
    const int bs = s.bs;
    for (int end = 0; end < 2; ++end) {
        const int m = end == 0 ? s.hu : s.tu;
        // index ranges: region R (the m eliminated unknowns), adjacent block J (bs)
        const int r0 = end == 0 ? 0 : s.nunk - s.tu;
        const int j0 = end == 0 ? s.hu : s.nunk - s.tu - bs;
        double H[36], Hi[36], E[18], F[18];
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) H[i * m + j] = line_entry(d, r0 + i, r0 + j);
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < bs; ++j) E[i * bs + j] = line_entry(d, r0 + i, j0 + j);
        for (int i = 0; i < bs; ++i)
            for (int j = 0; j < m; ++j) F[i * m + j] = line_entry(d, j0 + i, r0 + j);
        if (!small_inverse(H, m, Hi)) { atomicExch(status, 1); return; }
        T *t = tab + end * kTabEnd;
        for (int i = 0; i < m * m; ++i) t[kTabHinv + i] = (T)Hi[i];
        double HiE[18];
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < bs; ++j) {
                double acc = 0.0;
                for (int k = 0; k < m; ++k) acc += Hi[i * m + k] * E[k * bs + j];
                HiE[i * bs + j] = acc;
                t[kTabHinvE + i * bs + j] = (T)acc;
            }
        for (int i = 0; i < bs; ++i)
            for (int j = 0; j < m; ++j) {
                double acc = 0.0;
                for (int k = 0; k < m; ++k) acc += F[i * m + k] * Hi[k * m + j];
                t[kTabK + i * m + j] = (T)acc;
            }
        for (int i = 0; i < bs; ++i)
            for (int j = 0; j < bs; ++j) {
                double acc = 0.0;
                for (int k = 0; k < m; ++k) acc += F[i * m + k] * HiE[k * bs + j];
                t[kTabDB + i * bs + j] = (T)acc;
            }
    }
}

// ---------------------------------------------------------------------------------------
// Thread-per-line solver.
// ---------------------------------------------------------------------------------------
size_t v1_scratch_words(int method, int N) {
    LineShape s = line_shape(method, N);
    return (size_t)s.nunk + (size_t)s.nb * (s.bs * s.bs + s.bs);
}

template <typename T, int BS>
__device__ void solve_line_v1(const LineDesc<T> &d, T *scr, long long st, int write_natural) {
    const Line<T> L(d);
    const LineShape s = line_shape(d.method, d.N);
    const int N = d.N, hu = s.hu, tu = s.tu, nb = s.nb, nunk = s.nunk;
    auto X = [&](int k) -> T & { return scr[(long long)k * st]; };
    auto Gm = [&](int b, int i, int j) -> T & { return scr[(long long)(nunk + (b * BS + i) * BS + j) * st]; };
    auto Y = [&](int b, int i) -> T & { return scr[(long long)(nunk + nb * BS * BS + b * BS + i) * st]; };
    const T *th = d.tab, *tt = d.tab + kTabEnd;

    T rH[6], rT[6];
    for (int i = 0; i < hu; ++i) rH[i] = rhs_row(L, i);
    for (int i = 0; i < tu; ++i) rT[i] = rhs_row(L, nunk - tu + i);

    // forward sweep
    T Gp[BS][BS], yp[BS];
#pragma unroll
    for (int i = 0; i < BS; ++i) { yp[i] = T(0); for (int j = 0; j < BS; ++j) Gp[i][j] = T(0); }
    for (int b = 0; b < nb; ++b) {
        T A[BS][BS], B[BS][BS], C[BS][BS], r[BS];
        middle_block<T, T, BS>(L, s, b, A, B, C, r);
        if (b == 0) {
            for (int i = 0; i < BS; ++i) {
                for (int j = 0; j < BS; ++j) B[i][j] -= th[kTabDB + i * BS + j];
                T acc = T(0);
                for (int k = 0; k < hu; ++k) acc += th[kTabK + i * hu + k] * rH[k];
                r[i] -= acc;
            }
        }
        if (b == nb - 1) {
            for (int i = 0; i < BS; ++i) {
                for (int j = 0; j < BS; ++j) B[i][j] -= tt[kTabDB + i * BS + j];
                T acc = T(0);
                for (int k = 0; k < tu; ++k) acc += tt[kTabK + i * tu + k] * rT[k];
                r[i] -= acc;
            }
        }
        T S[BS][BS], Si[BS][BS];
#pragma unroll
        for (int i = 0; i < BS; ++i) {
#pragma unroll
            for (int j = 0; j < BS; ++j) {
                T acc = B[i][j];
#pragma unroll
                for (int k = 0; k < BS; ++k) acc -= A[i][k] * Gp[k][j];
                S[i][j] = acc;
            }
            T acc = r[i];
#pragma unroll
            for (int k = 0; k < BS; ++k) acc -= A[i][k] * yp[k];
            r[i] = acc;
        }
        mat_inv<T, BS>(S, Si);
#pragma unroll
        for (int i = 0; i < BS; ++i) {
#pragma unroll
            for (int j = 0; j < BS; ++j) {
                T acc = T(0);
#pragma unroll
                for (int k = 0; k < BS; ++k) acc += Si[i][k] * C[k][j];
                Gp[i][j] = acc;
                Gm(b, i, j) = acc;
            }
        }
        T yn[BS];
#pragma unroll
        for (int i = 0; i < BS; ++i) {
            T acc = T(0);
#pragma unroll
            for (int k = 0; k < BS; ++k) acc += Si[i][k] * r[k];
            yn[i] = acc;
        }
#pragma unroll
        for (int i = 0; i < BS; ++i) { yp[i] = yn[i]; Y(b, i) = yn[i]; }
    }
    // backward sweep: x_b = y_b - Gamma_b x_{b+1}
    T xn[BS];
#pragma unroll
    for (int i = 0; i < BS; ++i) xn[i] = T(0);
    for (int b = nb - 1; b >= 0; --b) {
        T x[BS];
#pragma unroll
        for (int i = 0; i < BS; ++i) {
            T acc = Y(b, i);
#pragma unroll
            for (int k = 0; k < BS; ++k) acc -= Gm(b, i, k) * xn[k];
            x[i] = acc;
        }
#pragma unroll
        for (int i = 0; i < BS; ++i) { xn[i] = x[i]; X(hu + b * BS + i) = x[i]; }
    }
    // eliminated head/tail unknowns
    for (int i = 0; i < hu; ++i) {
        T acc = T(0);
        for (int k = 0; k < hu; ++k) acc += th[kTabHinv + i * hu + k] * rH[k];
        for (int k = 0; k < BS; ++k) acc -= th[kTabHinvE + i * BS + k] * X(hu + k);
        X(i) = acc;
    }
    const int lb = hu + (nb - 1) * BS;
    for (int i = 0; i < tu; ++i) {
        T acc = T(0);
        for (int k = 0; k < tu; ++k) acc += tt[kTabHinv + i * tu + k] * rT[k];
        for (int k = 0; k < BS; ++k) acc -= tt[kTabHinvE + i * BS + k] * X(lb + k);
        X(nunk - tu + i) = acc;
    }

    // source term dt/2 f(t_{m+1}) at the source point of this line
    T src = T(0);
    if (d.src_k >= 0) {
        long long m = *d.clock;
        double t1 = (double)(m + 1) * d.dt;
        src = (T)(d.src_scale * ricker(d.src_amp, d.src_f0, d.src_tdelay, t1));
        if (d.advance_clock) *d.clock = m + 1;
    }

    // epilogue: carried outputs (and natural outputs on request)
    const T beta = (T)d.beta;
    if (d.method == kCFD) {
        for (int j = 0; j <= N; ++j) {
            T g = X(cfd_idx_g(N, j));
            T vin = d.v[j * d.sv];
            d.vo[j * d.svo] = vin - T(2) * beta * g;
            if (write_natural && d.w_out) d.w_out[j * d.snv] = vin - beta * g;
        }
        for (int j = 1; j <= N - 1; ++j) {
            T e = X(cfd_idx_e(j));
            T pin = d.p[j * d.sp];
            T ae = L.al(j) * e;
            d.po[j * d.spo] = pin - T(2) * ae + (j == d.src_k ? src : T(0));
            if (write_natural && d.u_out) d.u_out[j * d.snp] = pin - ae;
        }
    } else {
        const T ih = (T)d.inv_h;
        const T p0 = L.p(0), pl = L.p(N + 1);
        for (int j = 0; j <= N; ++j) {
            double gw[8];
            int g0;
            int ng = mfd_G_row(N, j, &g0, gw);
            T acc = T(0);
            for (int t = 0; t < ng; ++t) {
                int k = g0 + t;  // pressure-line index
                T uk = (k == 0) ? p0 : (k == N + 1 ? pl : X(k - 1));
                acc += (T)gw[t] * uk;
            }
            T gu = acc * ih;
            T vin = d.v[j * d.sv];
            d.vo[j * d.svo] = vin - T(2) * beta * gu;
            if (write_natural && d.w_out) d.w_out[j * d.snv] = vin - beta * gu;
        }
        for (int c = 1; c <= N; ++c) {
            T u = X(c - 1);
            T pin = d.p[c * d.sp];
            d.po[c * d.spo] = T(2) * u - pin + (c == d.src_k ? src : T(0));
            if (write_natural && d.u_out) d.u_out[c * d.snp] = u;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(128) line_solve_v1_kernel(const LineDesc<T> *__restrict__ descs,
                                                           int nlines, T *scratch, long long st,
                                                           int write_natural) {
    int line = blockIdx.x * blockDim.x + threadIdx.x;
    if (line >= nlines) return;
    const LineDesc<T> d = descs[line];
    T *scr = scratch + line;
    if (d.method == kCFD)
        solve_line_v1<T, 2>(d, scr, st, write_natural);
    else
        solve_line_v1<T, 3>(d, scr, st, write_natural);
}

// ---------------------------------------------------------------------------------------
// Prologue: carried state from natural fields, one thread per stage-2 (y) line.
//   a_k  = u_k - alpha_k (Dv w)_k + dt/2 f(t_m)   (interior pressure points) -> d.po
//   w*_j = w_j - beta (Du u)_j                      (all velocity points)     -> d.v
// (d.po of a stage-2 line is the stage-1 input buffer; d.v is the stage-2 input; the
// natural u and w are read through d.u_out and d.w_out.)
// CFD derivatives solve Pbar e = Qbar w and P g = Q u by the Thomas algorithm, with the
// factors of the two constant matrices precomputed (fac: P's sub-diagonal, eliminated
// super-diagonal and inverse pivots, N+1 each, then Pbar's, N-1 each).
// ---------------------------------------------------------------------------------------
template <typename T>
__device__ void thomas_apply(int n, T *rhs, long long st, const T *__restrict__ lo, const T *__restrict__ cu,
                             const T *__restrict__ id) {
    // Solves the n-row system in place: forward d_r = (rhs_r - lo_r d_{r-1}) / den_r, then
    // x_r = d_r - c_r x_{r+1}; the running value stays in a register.
    T d = rhs[0] * id[0];
    rhs[0] = d;
    for (int r = 1; r < n; ++r) {
        d = (rhs[(long long)r * st] - lo[r] * d) * id[r];
        rhs[(long long)r * st] = d;
    }
    T x = d;
    for (int r = n - 2; r >= 0; --r) {
        x = rhs[(long long)r * st] - cu[r] * x;
        rhs[(long long)r * st] = x;
    }
}

// Without precomputed factors (fac == nullptr): the same elimination with each row's factors
// formed on the fly, the eliminated super-diagonal kept in cs (stride st).
template <typename T>
__device__ void thomas_rows(int N, bool reduced, T *rhs, T *cs, long long st) {
    const int n = reduced ? N - 1 : N + 1;
    double w[8];
    int c0;
    T cprev = T(0), d = T(0);
    for (int r = 0; r < n; ++r) {
        if (reduced) cfd_Pbar_row(N, r + 1, &c0, w); else cfd_P_row(N, r, &c0, w);
        T lo = T(0), di, up = T(0);
        if (r == 0) { di = (T)w[0]; up = (T)w[1]; }
        else if (r == n - 1) { lo = (T)w[0]; di = (T)w[1]; }
        else { lo = (T)w[0]; di = (T)w[1]; up = (T)w[2]; }
        const T den = di - lo * cprev;
        cprev = up / den;
        d = (rhs[(long long)r * st] - lo * d) / den;
        cs[(long long)r * st] = cprev;
        rhs[(long long)r * st] = d;
    }
    T x = d;
    for (int r = n - 2; r >= 0; --r) {
        x = rhs[(long long)r * st] - cs[(long long)r * st] * x;
        rhs[(long long)r * st] = x;
    }
}

template <typename T>
__global__ void prologue_kernel(const LineDesc<T> *__restrict__ descs, int nlines, T *scratch,
                                long long st, const T *__restrict__ fac) {
    int line = blockIdx.x * blockDim.x + threadIdx.x;
    if (line >= nlines) return;
    const LineDesc<T> d = descs[line];
    const int N = d.N;
    const T ih = (T)d.inv_h, beta = (T)d.beta;
    T *scr = scratch + line;
    auto S = [&](int k) -> T & { return scr[(long long)k * st]; };
    const T *un = d.u_out;  // natural u along the line (same indexing as p)
    const T *wn = d.w_out;  // natural w along the line (same indexing as v)
    double w[8];
    int c0;
    T src = T(0);
    if (d.src_k >= 0) {
        double t = (double)(*d.clock) * d.dt;
        src = (T)(d.src_scale * ricker(d.src_amp, d.src_f0, d.src_tdelay, t));
    }
    const long long snp = d.snp, snv = d.snv, spo = d.spo;
    if (d.method == kCFD) {
        // g = P^{-1} Q u  (slots 0..N), then w* = w - beta g
        for (int j = 0; j <= N; ++j) {
            int n = cfd_Q_row(N, j, &c0, w);
            T acc = T(0);
            for (int t = 0; t < n; ++t) acc += (T)w[t] * un[(c0 + t) * snp];
            S(j) = acc * ih;
        }
        if (fac) thomas_apply<T>(N + 1, scr, st, fac, fac + (N + 1), fac + 2 * (N + 1));
        else thomas_rows<T>(N, false, scr, scr + (long long)(N + 1) * st, st);
        for (int j = 0; j <= N; ++j) d.v[j * d.sv] = wn[j * snv] - beta * S(j);
        // e = Pbar^{-1} Qbar w  (slots 0..N-2 for nodes 1..N-1), then a = u - alpha e
        for (int j = 1; j <= N - 1; ++j) {
            int n = cfd_Qbar_row(N, j, &c0, w);
            T acc = T(0);
            for (int t = 0; t < n; ++t) acc += (T)w[t] * wn[(c0 + t) * snv];
            S(j - 1) = acc * ih;
        }
        if (fac) {
            const T *fb = fac + 3 * (N + 1);
            thomas_apply<T>(N - 1, scr, st, fb, fb + (N - 1), fb + 2 * (N - 1));
        } else {
            thomas_rows<T>(N, true, scr, scr + (long long)(N + 1) * st, st);
        }
        for (int j = 1; j <= N - 1; ++j) {
            T val = un[j * snp] - d.alpha[j * d.sp] * S(j - 1);
            if (j == d.src_k) val += src;
            d.po[j * spo] = val;
        }
        d.po[0] = un[0];
        d.po[(long long)N * spo] = un[(long long)N * snp];
    } else {
        for (int j = 0; j <= N; ++j) {
            int n = mfd_G_row(N, j, &c0, w);
            T acc = T(0);
            for (int t = 0; t < n; ++t) acc += (T)w[t] * un[(c0 + t) * snp];
            d.v[j * d.sv] = wn[j * snv] - beta * acc * ih;
        }
        for (int c = 1; c <= N; ++c) {
            int n = mfd_D_row(N, c - 1, &c0, w);
            T acc = T(0);
            for (int t = 0; t < n; ++t) acc += (T)w[t] * wn[(c0 + t) * snv];
            T val = un[c * snp] - d.alpha[c * d.sp] * acc * ih;
            if (c == d.src_k) val += src;
            d.po[c * spo] = val;
        }
        d.po[0] = un[0];
        d.po[(long long)(N + 1) * spo] = un[(long long)(N + 1) * snp];
    }
}

// ---------------------------------------------------------------------------------------
// The same prologue spread over the lines' elements.  prologue_stencil_kernel: block (32
// lines, 8 elements); for CFD it leaves (Q u)_j / h (j = 0..N) and (Qbar w)_j / h (j = 1..N-1)
// in the scratch (element k of a line at k * st + line), for MFD it writes w* and a directly.
// prologue_solve_win_kernel (CFD): the two Thomas solves with the precomputed factors, one
// thread per chunk of a line (below).
// ---------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T prologue_src(const LineDesc<T> &d) {
    return (T)(d.src_scale * ricker(d.src_amp, d.src_f0, d.src_tdelay, (double)(*d.clock) * d.dt));
}

// Interior rows of the explicit operators (CFD Q and Qbar: -3, 0, 3; MFD D4 and G4: the
// fourth-order staggered stencil), with the weights as compile-time constants of T; the same
// terms in the same order as the row functions give them, so the sums are the same.  p points
// at the row's first point, s is the stride along the line.
template <typename T>
__device__ __forceinline__ T cfd_interior_dot(const T *p, long long s) {
    T acc = T(0);
    acc += T(-3.0) * p[0];
    acc += T(0.0) * p[s];
    acc += T(3.0) * p[2 * s];
    return acc;
}
template <typename T>
__device__ __forceinline__ T mfd_interior_dot(const T *p, long long s) {
    T acc = T(0);
    acc += T(1.0 / 24.0) * p[0];
    acc += T(-9.0 / 8.0) * p[s];
    acc += T(9.0 / 8.0) * p[2 * s];
    acc += T(-1.0 / 24.0) * p[3 * s];
    return acc;
}

template <typename T>
__global__ void prologue_stencil_kernel(const LineDesc<T> *__restrict__ descs, int nlines, int N, int method,
                                        T *scratch, long long st) {
    // block (32 lines, 8): elements j0 .. j0 + 31 of 32 consecutive lines; lane = line reads the
    // row-major natural fields coalesced.  MFD writes w* and a, which are contiguous along each
    // line, through shared memory, along each line in turn.
    __shared__ T tv[32][33], tp[32][33], tu[32][33];
    // the block's 32 descriptors, copied once with 16-byte loads (each thread would otherwise
    // read its own descriptor's fields, 32 scattered sectors per load)
    __shared__ __align__(16) unsigned char sdesc[32 * sizeof(LineDesc<T>)];
    static_assert(sizeof(LineDesc<T>) % 16 == 0, "descriptor size");
    const int x = threadIdx.x, y = threadIdx.y;
    const int line0 = blockIdx.x * 32, line = line0 + x;
    const int j0 = blockIdx.y * 32;
    {
        const int nl = min(32, nlines - line0);
        const uint4 *src = reinterpret_cast<const uint4 *>(descs + line0);
        uint4 *dst = reinterpret_cast<uint4 *>(sdesc);
        const int nvec = nl * (int)(sizeof(LineDesc<T>) / 16);
        for (int k = y * 32 + x; k < nvec; k += 256) dst[k] = src[k];
    }
    __syncthreads();
    const LineDesc<T> *sd = reinterpret_cast<const LineDesc<T> *>(sdesc);
    if (line < nlines) {
        const LineDesc<T> &d = sd[x];
        const T ih = (T)d.inv_h, beta = (T)d.beta;
        const T *un = d.u_out, *wn = d.w_out;
        const long long snp = d.snp, snv = d.snv;
        double w[8];
        int c0;
        for (int jj = y; jj < 32; jj += 8) {
            const int j = j0 + jj;
            if (j > N + 1) break;
            if (method == kCFD) {
                if (j <= N) {
                    T acc = T(0);
                    if (j >= 1 && j <= N - 1) {
                        acc = cfd_interior_dot(un + (long long)(j - 1) * snp, snp);
                    } else {
                        const int n = cfd_Q_row(N, j, &c0, w);
                        for (int t = 0; t < n; ++t) acc += (T)w[t] * un[(c0 + t) * snp];
                    }
                    scratch[(long long)j * st + line] = acc * ih;
                }
                if (j >= 1 && j <= N - 1) {
                    T acc = T(0);
                    if (j >= 2 && j <= N - 2) {
                        acc = cfd_interior_dot(wn + (long long)(j - 1) * snv, snv);
                    } else {
                        const int n = cfd_Qbar_row(N, j, &c0, w);
                        for (int t = 0; t < n; ++t) acc += (T)w[t] * wn[(c0 + t) * snv];
                    }
                    scratch[(long long)(N + j) * st + line] = acc * ih;
                }
            } else {
                if (j <= N) {
                    T acc = T(0);
                    if (j >= 2 && j <= N - 2) {
                        acc = mfd_interior_dot(un + (long long)(j - 1) * snp, snp);
                    } else {
                        const int n = mfd_G_row(N, j, &c0, w);
                        for (int t = 0; t < n; ++t) acc += (T)w[t] * un[(c0 + t) * snp];
                    }
                    tv[jj][x] = wn[j * snv] - beta * acc * ih;
                }
                tu[jj][x] = un[j * snp];
                if (j >= 1 && j <= N) {
                    // a = u - alpha (D w)/h (+ source), formed below along the line
                    T acc = T(0);
                    if (j >= 2 && j <= N - 1) {
                        acc = mfd_interior_dot(wn + (long long)(j - 2) * snv, snv);
                    } else {
                        const int n = mfd_D_row(N, j - 1, &c0, w);
                        for (int t = 0; t < n; ++t) acc += (T)w[t] * wn[(c0 + t) * snv];
                    }
                    tp[jj][x] = acc;
                }
            }
        }
    }
    if (method == kCFD) return;  // uniform over the block
    __syncthreads();
    // lane = element: 8 lines at a time, 32 consecutive elements each
    for (int l = y; l < 32 && line0 + l < nlines; l += 8) {
        const LineDesc<T> &dl = sd[l];
        const int j = j0 + x;
        if (j > N + 1) continue;
        if (j <= N) dl.v[(long long)j * dl.sv] = tv[x][l];
        T val = tu[x][l];  // j = 0 or N+1: Dirichlet, u itself
        if (j >= 1 && j <= N) {
            val = val - dl.alpha[(long long)j * dl.sp] * tp[x][l] * (T)dl.inv_h;
            if (j == dl.src_k) val += prologue_src(dl);
        }
        dl.po[(long long)j * dl.spo] = val;
    }
}

// The same two Thomas solves spread over chunks of kProR rows of every line, one thread per
// (line, chunk): a line of 4097 rows gives 65 threads instead of one, so the solve is no longer a
// chain of thousands of dependent steps per thread.  Each thread solves the rows of its chunk
// plus a halo of kProH rows on each side that are not at a line end, with the values beyond the
// halo taken as zero.  Away from the two boundary rows P and Pbar are tridiag(1, 4, 1), whose
// inverse decays by a factor 2 - sqrt(3) = 0.268 per row, so what the truncation leaves out is
// 0.268^32 = 5e-19 of the solution: the result equals the whole-line solve to rounding.  A
// window that starts inside the line eliminates from its first row as if it had no
// predecessor; those rows are interior rows, and the start-up factors of that elimination (the
// last kProH values of the factor buffer) join the whole line's factors within kProH rows.
constexpr int kProR = 64, kProH = 32;

// q(r) gives the right-hand side of row r.  The forward values of rows r0..r1-1 go to
// tmp[(r - t0) * ts] and are read back by the backward sweep just before out(r, x) is called for
// the row.
template <typename T, typename QF, typename Out>
__host__ __device__ __forceinline__ void prologue_win_solve(int n, int r0, int r1, QF q, const T *lo, const T *cu,
                                                            const T *id, const T *su_id, T *tmp, long long ts,
                                                            Out out, int t0 = 0) {
    const int s = r0 > 0 ? r0 - kProH : 0;
    const int e = r1 + kProH < n ? r1 + kProH : n;
    T dd = T(0);
#pragma unroll 8
    for (int r = s; r < r0; ++r) dd = (q(r) - dd) * su_id[r - s];  // start-up rows
#pragma unroll 8
    for (int r = r0; r < r1; ++r) {
        dd = (q(r) - lo[r] * dd) * id[r];
        tmp[(long long)(r - t0) * ts] = dd;
    }
    T hh[kProH];
#pragma unroll
    for (int k = 0; k < kProH; ++k) {
        const int r = r1 + k;
        if (r < e) {
            dd = (q(r) - lo[r] * dd) * id[r];
            hh[k] = dd;
        }
    }
    T x = T(0);
#pragma unroll
    for (int k = kProH - 1; k >= 0; --k) {
        const int r = r1 + k;
        if (r < e) x = hh[k] - cu[r] * x;
    }
#pragma unroll 8
    for (int r = r1 - 1; r >= r0; --r) {
        x = tmp[(long long)(r - t0) * ts] - cu[r] * x;
        out(r, x);
    }
}

// grid.y: the chunks of P (N+1 rows) first, then those of Pbar (N-1 rows).  A block is one warp
// of 32 consecutive lines.  The lines' natural fields are row-major, so lane = line reads them
// coalesced; the outputs (w*, a) and alpha are contiguous along each line, so they go through
// shared memory and move along each line in turn, lane = row.  (Loading the window's right-hand
// sides and natural values into shared memory first measured slower: 508-536 against 406 us at
// 4096 lines of 4097 rows.)
template <typename T>
__global__ void __launch_bounds__(32) prologue_solve_win_kernel(const LineDesc<T> *__restrict__ descs, int nlines,
                                                                int N, const T *scratch, long long st,
                                                                const T *__restrict__ fac) {
    __shared__ T tile[kProR][33];  // per line: the forward values, then the chunk's outputs
    __shared__ T tu[kProR][33];    // Pbar chunks: u at the chunk's nodes
    const int lane = threadIdx.x;
    const int line0 = blockIdx.x * 32, line = line0 + lane;
    const int nP = N + 1, nB = N - 1;
    const int chP = (nP + kProR - 1) / kProR;
    const bool isP = (int)blockIdx.y < chP;
    const int c = isP ? (int)blockIdx.y : (int)blockIdx.y - chP;
    const int r0 = c * kProR, r1 = min(isP ? nP : nB, r0 + kProR), nr = r1 - r0;
    const T *su_id = fac + 3 * (N + 1) + 3 * (N - 1);
    if (line < nlines) {
        const LineDesc<T> &d = descs[line];
        const T beta = (T)d.beta;
        const T *un = d.u_out, *wn = d.w_out;
        const long long snp = d.snp, snv = d.snv;
        const T *__restrict__ q = scratch + (isP ? 0 : (long long)(N + 1) * st) + line;
        auto qf = [&](int r) -> T { return q[(long long)r * st]; };
        if (isP) {
            // P g = (Q u)/h over rows 0..N; w*_r = w_r - beta g_r
            const T *lo = fac, *cu = fac + (N + 1), *id = fac + 2 * (N + 1);
            prologue_win_solve<T>(nP, r0, r1, qf, lo, cu, id, su_id, &tile[0][lane], 33,
                                  [&](int r, T g) { tile[r - r0][lane] = wn[(long long)r * snv] - beta * g; }, r0);
        } else {
            // Pbar e = (Qbar w)/h over nodes 1..N-1 (rows 0..N-2); a_j = u_j - alpha_j e_j (+ source)
            const T *fb = fac + 3 * (N + 1);
            const T *lo = fb, *cu = fb + (N - 1), *id = fb + 2 * (N - 1);
            prologue_win_solve<T>(nB, r0, r1, qf, lo, cu, id, su_id, &tile[0][lane], 33, [&](int r, T e) {
                tile[r - r0][lane] = e;
                tu[r - r0][lane] = un[(long long)(r + 1) * snp];
            }, r0);
            if (c == 0) {
                d.po[0] = un[0];
                d.po[(long long)N * d.spo] = un[(long long)N * snp];
            }
        }
    }
    __syncwarp();
    for (int l = 0; l < 32 && line0 + l < nlines; ++l) {
        const LineDesc<T> &dl = descs[line0 + l];
        if (isP) {
            for (int k = lane; k < nr; k += 32) dl.v[(long long)(r0 + k) * dl.sv] = tile[k][l];
        } else {
            for (int k = lane; k < nr; k += 32) {
                const long long j = r0 + k + 1;
                T val = tu[k][l] - dl.alpha[j * dl.sp] * tile[k][l];
                if (j == dl.src_k) val += prologue_src(dl);
                dl.po[j * dl.spo] = val;
            }
        }
    }
}

// Sets *flag if any x[i] is NaN or infinite: 16-byte loads over the aligned body of x (when x
// itself is 16-byte aligned), element loads for the rest.
template <typename T>
__global__ void finite_check_kernel(const T *__restrict__ x, size_t n, int *flag) {
    constexpr int V = 16 / sizeof(T);
    const size_t i0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t nv = ((size_t)x & 15u) == 0 ? n / V : 0;
    bool bad = false;
    if constexpr (sizeof(T) == 4) {
        const float4 *xv = reinterpret_cast<const float4 *>(x);
        for (size_t i = i0; i < nv; i += stride) {
            const float4 q = xv[i];
            bad |= !(isfinite(q.x) && isfinite(q.y) && isfinite(q.z) && isfinite(q.w));
        }
    } else {
        const double2 *xv = reinterpret_cast<const double2 *>(x);
        for (size_t i = i0; i < nv; i += stride) {
            const double2 q = xv[i];
            bad |= !(isfinite(q.x) && isfinite(q.y));
        }
    }
    for (size_t i = nv * V + i0; i < n; i += stride) bad |= !isfinite((double)x[i]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch(flag, 1);
}

// ---------------------------------------------------------------------------------------
// Launchers.
// ---------------------------------------------------------------------------------------
template <typename T>
cudaError_t launch_precompute(const LineDesc<T> *d, int nlines, T *tab, int *status,
                              cudaStream_t s) {
    if (nlines <= 0) return cudaSuccess;
    int tpb = 64;
    precompute_kernel<T><<<(nlines + tpb - 1) / tpb, tpb, 0, s>>>(d, nlines, tab, status);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_line_solve_v1(const LineDesc<T> *d, int nlines, T *scratch, long long st,
                                 int write_natural, cudaStream_t s) {
    if (nlines <= 0) return cudaSuccess;
    int tpb = 128;
    line_solve_v1_kernel<T><<<(nlines + tpb - 1) / tpb, tpb, 0, s>>>(d, nlines, scratch, st,
                                                                    write_natural);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_prologue(const LineDesc<T> *d, int nlines, const T *fac, T *scratch, long long st,
                            cudaStream_t s) {
    if (nlines <= 0) return cudaSuccess;
    int tpb = 128;
    prologue_kernel<T><<<(nlines + tpb - 1) / tpb, tpb, 0, s>>>(d, nlines, scratch, st, fac);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_prologue_lines(const LineDesc<T> *d, int nlines, int N, int method, const T *fac, T *scratch,
                                  long long st, cudaStream_t s) {
    if (nlines <= 0) return cudaSuccess;
    dim3 grid((unsigned)((nlines + 31) / 32), (unsigned)((N + 2 + 31) / 32));
    prologue_stencil_kernel<T><<<grid, dim3(32, 8), 0, s>>>(d, nlines, N, method, scratch, st);
    if (method == kCFD) {
        const unsigned chunks = (unsigned)((N + 1 + kProR - 1) / kProR + (N - 1 + kProR - 1) / kProR);
        prologue_solve_win_kernel<T><<<dim3((unsigned)((nlines + 31) / 32), chunks), 32, 0, s>>>(d, nlines, N,
                                                                                              scratch, st, fac);
    }
    return cudaGetLastError();
}

// Thomas factors of the App. A P (N+1 rows) and Pbar (N-1 rows), for the prologue: per matrix
// the sub-diagonal, the eliminated super-diagonal c_r = up_r / den_r and 1 / den_r, where
// den_r = di_r - lo_r c_{r-1}; built in FP64.
size_t prologue_factor_count(int N) { return (size_t)3 * (N + 1) + 3 * (N - 1) + kProH; }
void prologue_factors(int N, std::vector<double> &out) {
    out.assign(prologue_factor_count(N), 0.0);
    // start-up factors of a window that begins on an interior row (no predecessor): 1 / den_k with
    // den_0 = 4, den_k = 4 - 1 / den_{k-1}
    {
        double *su = out.data() + 3 * (N + 1) + 3 * (N - 1), den = 4.0;
        for (int k = 0; k < kProH; ++k) {
            su[k] = 1.0 / den;
            den = 4.0 - su[k];
        }
    }
    for (int bar = 0; bar < 2; ++bar) {
        const int n = bar ? N - 1 : N + 1;
        double *lo = out.data() + (bar ? 3 * (N + 1) : 0), *cu = lo + n, *id = cu + n;
        double cprev = 0.0;
        for (int r = 0; r < n; ++r) {
            double w[8];
            int c0;
            if (bar) cfd_Pbar_row(N, r + 1, &c0, w); else cfd_P_row(N, r, &c0, w);
            double l = 0.0, di, up = 0.0;
            if (r == 0) { di = w[0]; up = w[1]; }
            else if (r == n - 1) { l = w[0]; di = w[1]; }
            else { l = w[0]; di = w[1]; up = w[2]; }
            const double den = di - l * cprev;
            lo[r] = l;
            cu[r] = up / den;
            id[r] = 1.0 / den;
            cprev = cu[r];
        }
    }
}
template <typename T>
cudaError_t launch_finite_check(const T *x, size_t n, int *flag, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    size_t blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    finite_check_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(x, n, flag);
    return cudaGetLastError();
}

#define ADI_INST(T)                                                                          \
    template cudaError_t launch_precompute<T>(const LineDesc<T> *, int, T *, int *,          \
                                              cudaStream_t);                                 \
    template cudaError_t launch_line_solve_v1<T>(const LineDesc<T> *, int, T *, long long,   \
                                                 int, cudaStream_t);                         \
    template cudaError_t launch_prologue<T>(const LineDesc<T> *, int, const T *, T *, long long,  \
                                            cudaStream_t);                                         \
    template cudaError_t launch_prologue_lines<T>(const LineDesc<T> *, int, int, int, const T *, T *, \
                                                  long long, cudaStream_t);                                   \
    template cudaError_t launch_finite_check<T>(const T *, size_t, int *, cudaStream_t);
ADI_INST(float)
ADI_INST(double)

}  // namespace adi
