// adi_fixed.cu -- the paper's own way of solving the stage systems, for comparison with the
// exact line solves of the default path: the fixed-point iteration of Eq. 9 (Algorithms 3 and
// 4).  Each Peaceman-Rachford stage assembles its explicit right-hand side, then sweeps
//     u_{k+1} = a - alpha (Dv v_k),      v_{k+1} = v^m - beta (Du u_{k+1})
// along every line of its direction until the sum of the Frobenius norms of the two updates
// is at most eps, or kmax sweeps have run.  Dv, Du are the App. A compact operators
// (Pbar^{-1} Qbar, P^{-1} Q: a tridiagonal solve per application) or the App. B mimetic
// stencils (D4, G4).  The norm test runs on the device: every sweep's kernels read a status
// word and return at once when an earlier sweep has converged, so no host round trip sits
// between sweeps.  One thread per line (the paper's GPU decomposition); natural (u, v, w)
// fields in row-major device arrays.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "../../include/adi.h"
#include "adi_internal.h"
#include "adi_line.cuh"
#include "adi_ops.cuh"

namespace adi {
namespace {

// Thomas factors of a tridiagonal operator of n rows: multipliers m_r (r >= 1), inverse
// pivots, super-diagonal.  Built on the host in FP64 from the App. A rows.
template <typename T>
struct FpTri {
    const T *m, *id, *c;
};

// Device-side convergence state of one stage's iteration.
struct FpState {
    double sum[2];  // squared Frobenius norms of the two updates of the current sweep
    int k;          // sweeps done in this stage
    int done;       // the stage's iteration has stopped
    long long sweeps;  // sweeps over the whole call
};

// Du along a line of N cells: CFD P^{-1} Q / h on nodes 0..N (N+1 -> N+1); MFD G4 / h
// (N+2 -> N+1).  x: the pressure line with element stride sx; out: N+1 values, stride so.
template <typename T>
__device__ void fp_du(int method, int N, T ih, const T *x, long long sx, T *out, long long so, FpTri<T> P) {
    double w[6];
    int c0 = 0;
    if (method == kCFD) {
        for (int r = 0; r <= N; ++r) {
            const int n = cfd_Q_row(N, r, &c0, w);
            T acc = T(0);
            for (int i = 0; i < n; ++i) acc += (T)w[i] * x[(long long)(c0 + i) * sx];
            out[(long long)r * so] = acc * ih;
        }
        for (int r = 1; r <= N; ++r) out[(long long)r * so] -= P.m[r] * out[(long long)(r - 1) * so];
        out[(long long)N * so] *= P.id[N];
        for (int r = N - 1; r >= 0; --r)
            out[(long long)r * so] = (out[(long long)r * so] - P.c[r] * out[(long long)(r + 1) * so]) * P.id[r];
    } else {
        for (int j = 0; j <= N; ++j) {
            const int n = mfd_G_row(N, j, &c0, w);
            T acc = T(0);
            for (int i = 0; i < n; ++i) acc += (T)w[i] * x[(long long)(c0 + i) * sx];
            out[(long long)j * so] = acc * ih;
        }
    }
}

// Dv along a line of N cells: CFD Pbar^{-1} Qbar / h (N+1 -> interior nodes 1..N-1); MFD
// D4 / h (N+1 -> cells 1..N).  Written at the pressure-line indices 1..L-1 of out.
template <typename T>
__device__ void fp_dv(int method, int N, T ih, const T *x, long long sx, T *out, long long so, FpTri<T> Pb) {
    double w[6];
    int c0 = 0;
    if (method == kCFD) {
        for (int j = 1; j <= N - 1; ++j) {
            const int n = cfd_Qbar_row(N, j, &c0, w);
            T acc = T(0);
            for (int i = 0; i < n; ++i) acc += (T)w[i] * x[(long long)(c0 + i) * sx];
            out[(long long)j * so] = acc * ih;
        }
        // Pbar rows j = 1..N-1 are factor rows 0..N-2
        for (int j = 2; j <= N - 1; ++j) out[(long long)j * so] -= Pb.m[j - 1] * out[(long long)(j - 1) * so];
        out[(long long)(N - 1) * so] *= Pb.id[N - 2];
        for (int j = N - 2; j >= 1; --j)
            out[(long long)j * so] = (out[(long long)j * so] - Pb.c[j - 1] * out[(long long)(j + 1) * so]) * Pb.id[j - 1];
    } else {
        for (int r = 0; r < N; ++r) {
            const int n = mfd_D_row(N, r, &c0, w);
            T acc = T(0);
            for (int i = 0; i < n; ++i) acc += (T)w[i] * x[(long long)(c0 + i) * sx];
            out[(long long)(r + 1) * so] = acc * ih;
        }
    }
}

// Lines of one direction: line l (first .. first + n - 1) of the pressure-like arrays starts
// at l * lsp with element stride esp, of the velocity arrays at l * lsv with stride esv.
struct FpLines {
    int first, n, N, L;  // L: last pressure index (N for CFD, N+1 for MFD)
    long long lsp, esp, lsv, esv;
};

// Explicit right-hand side of a stage along its explicit direction:
//   ov = vl - beta Du(ul)   (all N+1 velocities),   oa = ul - alpha Dv(vl)   (interior)
template <typename T>
__global__ void fp_rhs_kernel(int method, FpLines g, T ih, T beta, const T *__restrict__ ul, const T *__restrict__ vl,
                              const T *__restrict__ alpha, T *ov, T *oa, FpTri<T> P, FpTri<T> Pb) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.n) return;
    const long long l = g.first + t;
    const T *u = ul + l * g.lsp, *v = vl + l * g.lsv, *al = alpha + l * g.lsp;
    T *o_v = ov + l * g.lsv, *o_a = oa + l * g.lsp;
    fp_du<T>(method, g.N, ih, u, g.esp, o_v, g.esv, P);
    for (int k = 0; k <= g.N; ++k) o_v[k * g.esv] = v[k * g.esv] - beta * o_v[k * g.esv];
    fp_dv<T>(method, g.N, ih, v, g.esv, o_a, g.esp, Pb);
    for (int k = 1; k < g.L; ++k) o_a[k * g.esp] = u[k * g.esp] - al[k * g.esp] * o_a[k * g.esp];
}

// One sweep of Eq. 9 along the implicit direction:
//   oa = a - alpha Dv(vk)   (interior; oa's end values are the Dirichlet data),
//   ov = vb - beta Du(oa).
template <typename T>
__global__ void fp_sweep_kernel(int method, FpLines g, T ih, T beta, const T *__restrict__ a, const T *__restrict__ vk,
                                const T *__restrict__ vb, const T *__restrict__ alpha, T *oa, T *ov, FpTri<T> P,
                                FpTri<T> Pb, const FpState *st) {
    if (st->done) return;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.n) return;
    const long long l = g.first + t;
    const T *av = a + l * g.lsp, *v = vk + l * g.lsv, *b = vb + l * g.lsv, *al = alpha + l * g.lsp;
    T *o_a = oa + l * g.lsp, *o_v = ov + l * g.lsv;
    fp_dv<T>(method, g.N, ih, v, g.esv, o_a, g.esp, Pb);
    for (int k = 1; k < g.L; ++k) o_a[k * g.esp] = av[k * g.esp] - al[k * g.esp] * o_a[k * g.esp];
    fp_du<T>(method, g.N, ih, o_a, g.esp, o_v, g.esv, P);
    for (int k = 0; k <= g.N; ++k) o_v[k * g.esv] = b[k * g.esv] - beta * o_v[k * g.esv];
}

// Squared norm of x - y into *sum (FP64 accumulation).
template <typename T>
__global__ void fp_diff_kernel(const T *__restrict__ x, const T *__restrict__ y, size_t n, double *sum, const FpState *st) {
    if (st->done) return;
    double acc = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double d = (double)x[i] - (double)y[i];
        acc += d * d;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ double part[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) part[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += part[w];
        atomicAdd(sum, s);
    }
}

// End of a sweep: the test of the paper (sum of the two Frobenius norms) against eps and the
// sweep limit; later sweeps of the stage return at once once it has stopped.
__global__ void fp_finish_kernel(FpState *st, double eps, int kmax) {
    if (st->done) return;
    const double test = sqrt(st->sum[0]) + sqrt(st->sum[1]);
    st->sum[0] = st->sum[1] = 0.0;
    st->k += 1;
    st->sweeps += 1;
    if (test <= eps || st->k >= kmax) st->done = 1;
}

__global__ void fp_reset_kernel(FpState *st) {
    st->sum[0] = st->sum[1] = 0.0;
    st->k = 0;
    st->done = 0;
}

template <typename T>
__global__ void fp_copy_kernel(T *dst, const T *__restrict__ src, size_t n, const FpState *st) {
    if (st && st->done) return;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

// Point source dt/2 f(t) / h^2 added to the right-hand side at (is, js).
template <typename T>
__global__ void fp_source_kernel(T *a, long long p, double scale, double amp, double f0, double td, double t) {
    a[p] = (T)((double)a[p] + scale * ricker(amp, f0, td, t));
}

// Host: Thomas factors of the App. A tridiagonal P (rows 0..N) or Pbar (rows 1..N-1).
void tri_factors(int N, bool bar, std::vector<double> &m, std::vector<double> &id, std::vector<double> &c) {
    const int n = bar ? N - 1 : N + 1;
    std::vector<double> a(n, 0.0), b(n, 0.0), s(n, 0.0);
    for (int r = 0; r < n; ++r) {
        double w[6];
        int c0 = 0;
        const int row = bar ? r + 1 : r;
        const int len = bar ? cfd_Pbar_row(N, row, &c0, w) : cfd_P_row(N, row, &c0, w);
        for (int i = 0; i < len; ++i) {
            const int col = (bar ? c0 - 1 : c0) + i;  // Pbar columns are nodes 1..N-1
            if (col == r - 1) a[r] = w[i];
            else if (col == r) b[r] = w[i];
            else if (col == r + 1) s[r] = w[i];
        }
    }
    m.assign(n, 0.0); id.assign(n, 0.0); c = s;
    double d = b[0];
    id[0] = 1.0 / d;
    for (int r = 1; r < n; ++r) {
        m[r] = a[r] / d;
        d = b[r] - m[r] * s[r - 1];
        id[r] = 1.0 / d;
    }
}

struct DevArr {
    void *p = nullptr;
    ~DevArr() { if (p) cudaFree(p); }
};

template <typename T>
int run_fixed(int method, int nx, int ny, double h, double dt, const double *c_field, double *U, double *V,
              double *W, int nsteps, double t0, const double *src, int kmax, double eps, long long *sweeps,
              double *ms_out) {
    const bool cfd = method == ADI_CFD;
    const int ru = cfd ? ny + 1 : ny + 2, cu = cfd ? nx + 1 : nx + 2;  // U shape
    const int rv = ru, cv = nx + 1;                                     // V shape
    const int rw = ny + 1, cw = cu;                                     // W shape
    const size_t nU = (size_t)ru * cu, nV = (size_t)rv * cv, nW = (size_t)rw * cw;
    const int pix = cfd ? nx - 1 : nx, piy = cfd ? ny - 1 : ny;

    // device arrays
    enum { dU, dV, dW, dAl, dA, dUs, dVs, dWs, dUk, dVk, dWk, dUn, dVn, dWn, dNum };
    const size_t sizes[dNum] = {nU, nV, nW, nU, nU, nU, nV, nW, nU, nV, nW, nU, nV, nW};
    DevArr arr[dNum], tri[12], state;
    for (int k = 0; k < dNum; ++k)
        if (cudaMalloc(&arr[k].p, sizes[k] * sizeof(T)) != cudaSuccess) { (void)cudaGetLastError(); return ADI_ENOMEM; }
    if (cudaMalloc(&state.p, sizeof(FpState)) != cudaSuccess) { (void)cudaGetLastError(); return ADI_ENOMEM; }
    auto P = [&](int k) { return (T *)arr[k].p; };
    cudaError_t e = cudaMemset(state.p, 0, sizeof(FpState));

    // inputs: fields, alpha = dt/2 c^2
    {
        std::vector<T> buf(std::max(nU, std::max(nV, nW)));
        auto up = [&](const double *x, size_t n, int k, double scale, bool sq) {
            for (size_t i = 0; i < n; ++i) buf[i] = (T)(sq ? scale * x[i] * x[i] : x[i]);
            if (e == cudaSuccess) e = cudaMemcpy(arr[k].p, buf.data(), n * sizeof(T), cudaMemcpyHostToDevice);
        };
        up(U, nU, dU, 1.0, false);
        up(V, nV, dV, 1.0, false);
        up(W, nW, dW, 1.0, false);
        up(c_field, nU, dAl, 0.5 * dt, true);
    }
    if (e == cudaSuccess) e = cudaMemset(arr[dA].p, 0, nU * sizeof(T));

    // Thomas factors for both line lengths (CFD only)
    FpTri<T> Px{}, Pbx{}, Py{}, Pby{};
    if (cfd) {
        int slot = 0;
        auto make = [&](int N, bool bar) {
            std::vector<double> m, id, c;
            tri_factors(N, bar, m, id, c);
            FpTri<T> t{};
            const T *ptr[3];
            const std::vector<double> *src3[3] = {&m, &id, &c};
            for (int q = 0; q < 3; ++q) {
                std::vector<T> tv(src3[q]->begin(), src3[q]->end());
                if (e == cudaSuccess) e = cudaMalloc(&tri[slot].p, tv.size() * sizeof(T));
                if (e == cudaSuccess) e = cudaMemcpy(tri[slot].p, tv.data(), tv.size() * sizeof(T), cudaMemcpyHostToDevice);
                ptr[q] = (const T *)tri[slot].p;
                ++slot;
            }
            t.m = ptr[0]; t.id = ptr[1]; t.c = ptr[2];
            return t;
        };
        Px = make(nx, false); Pbx = make(nx, true); Py = make(ny, false); Pby = make(ny, true);
    }
    if (e != cudaSuccess) { (void)cudaGetLastError(); return e == cudaErrorMemoryAllocation ? ADI_ENOMEM : ADI_ECUDA; }

    // lines: rows (x-lines, stage 1 implicit, stage 2 explicit) and columns
    FpLines rows{1, piy, nx, cfd ? nx : nx + 1, (long long)cu, 1, (long long)cv, 1};
    FpLines cols{1, pix, ny, cfd ? ny : ny + 1, 1, (long long)cu, 1, (long long)cw};
    const T ih = (T)(1.0 / h), beta = (T)(0.5 * dt);
    const int tb = 128;
    auto blocks = [&](int n) { return (n + tb - 1) / tb; };
    FpState *st = (FpState *)state.p;
    auto copy = [&](int dst, int src, size_t n, const FpState *guard) {
        fp_copy_kernel<T><<<152 * 4, 256>>>(P(dst), P(src), n, guard);
    };
    const double sscale = 0.5 * dt / (h * h);
    const long long sp = src ? (long long)src[0] * cu + (long long)src[1] : 0;

    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0);
    for (int m = 0; m < nsteps; ++m) {
        const double t = t0 + m * dt;
        // ---- stage 1: w* and a explicit along y (columns), then x-line sweeps ----
        copy(dWs, dW, nW, nullptr);
        copy(dUs, dU, nU, nullptr);
        copy(dVs, dV, nV, nullptr);
        fp_rhs_kernel<T><<<blocks(pix), tb>>>(method, cols, ih, beta, P(dU), P(dW), P(dAl), P(dWs), P(dA), Py, Pby);
        if (src) fp_source_kernel<T><<<1, 1>>>(P(dA), sp, sscale, src[2], src[3], src[4], t);
        copy(dUk, dU, nU, nullptr);
        copy(dVk, dV, nV, nullptr);
        fp_reset_kernel<<<1, 1>>>(st);
        for (int k = 0; k < kmax; ++k) {
            fp_sweep_kernel<T><<<blocks(piy), tb>>>(method, rows, ih, beta, P(dA), P(dVk), P(dV), P(dAl), P(dUs),
                                                    P(dVs), Px, Pbx, st);
            fp_diff_kernel<T><<<152 * 2, 256>>>(P(dUs), P(dUk), nU, &st->sum[0], st);
            fp_diff_kernel<T><<<152 * 2, 256>>>(P(dVs), P(dVk), nV, &st->sum[1], st);
            fp_finish_kernel<<<1, 1>>>(st, eps, kmax);
            copy(dUk, dUs, nU, st);
            copy(dVk, dVs, nV, st);
        }
        // ---- stage 2: v^{m+1} and C explicit along x (rows), then y-line sweeps ----
        copy(dVn, dVs, nV, nullptr);
        fp_rhs_kernel<T><<<blocks(piy), tb>>>(method, rows, ih, beta, P(dUs), P(dVs), P(dAl), P(dVn), P(dA), Px, Pbx);
        if (src) fp_source_kernel<T><<<1, 1>>>(P(dA), sp, sscale, src[2], src[3], src[4], t + dt);
        copy(dWn, dWs, nW, nullptr);
        copy(dUn, dUs, nU, nullptr);
        copy(dUk, dUs, nU, nullptr);
        copy(dWk, dW, nW, nullptr);
        fp_reset_kernel<<<1, 1>>>(st);
        for (int k = 0; k < kmax; ++k) {
            fp_sweep_kernel<T><<<blocks(pix), tb>>>(method, cols, ih, beta, P(dA), P(dWk), P(dWs), P(dAl), P(dUn),
                                                    P(dWn), Py, Pby, st);
            fp_diff_kernel<T><<<152 * 2, 256>>>(P(dUn), P(dUk), nU, &st->sum[0], st);
            fp_diff_kernel<T><<<152 * 2, 256>>>(P(dWn), P(dWk), nW, &st->sum[1], st);
            fp_finish_kernel<<<1, 1>>>(st, eps, kmax);
            copy(dUk, dUn, nU, st);
            copy(dWk, dWn, nW, st);
        }
        copy(dU, dUn, nU, nullptr);
        copy(dV, dVn, nV, nullptr);
        copy(dW, dWn, nW, nullptr);
    }
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    FpState hs{};
    if (e == cudaSuccess) e = cudaMemcpy(&hs, state.p, sizeof(FpState), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) {
        std::vector<T> buf(std::max(nU, std::max(nV, nW)));
        auto down = [&](double *x, size_t n, int k) {
            if (e == cudaSuccess) e = cudaMemcpy(buf.data(), arr[k].p, n * sizeof(T), cudaMemcpyDeviceToHost);
            if (e == cudaSuccess)
                for (size_t i = 0; i < n; ++i) x[i] = (double)buf[i];
        };
        down(U, nU, dU);
        down(V, nV, dV);
        down(W, nW, dW);
    }
    if (e != cudaSuccess) { (void)cudaGetLastError(); return ADI_ECUDA; }
    if (sweeps) *sweeps = hs.sweeps;
    if (ms_out) *ms_out = ms;
    return ADI_OK;
}

}  // namespace
}  // namespace adi

extern "C" int adi_fixed_point(int method, int nx, int ny, double h, double dt, const double *c_field, double *u,
                               double *v, double *w, int nsteps, double t0, const double *source, int kmax,
                               double eps, int precision, long long *sweeps, double *device_ms) {
    if ((method != ADI_CFD && method != ADI_MFD) || (precision != ADI_FP32 && precision != ADI_FP64) ||
        nx < ADI_MIN_CELLS || ny < ADI_MIN_CELLS || nx > ADI_MAX_CELLS || ny > ADI_MAX_CELLS ||
        !(std::isfinite(h) && h > 0) || !(std::isfinite(dt) && dt > 0) || !c_field || !u || !v || !w ||
        nsteps < 0 || kmax < 1 || !(eps >= 0.0))
        return ADI_EINVAL;
    if (source) {
        const int piy = method == ADI_CFD ? ny - 1 : ny, pix = method == ADI_CFD ? nx - 1 : nx;
        const int is = (int)source[0], js = (int)source[1];
        if (is < 1 || is > piy || js < 1 || js > pix) return ADI_EINVAL;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) { (void)cudaGetLastError(); return ADI_ENOTSUP; }
    return precision == ADI_FP64
               ? adi::run_fixed<double>(method, nx, ny, h, dt, c_field, u, v, w, nsteps, t0, source, kmax, eps, sweeps, device_ms)
               : adi::run_fixed<float>(method, nx, ny, h, dt, c_field, u, v, w, nsteps, t0, source, kmax, eps, sweeps, device_ms);
}
