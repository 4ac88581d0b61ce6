// adi_api.cu -- host implementation of the C ABI in include/adi.h.
//
// Device state of one simulation (precision T):
//   A      carried pressure, U layout: interior holds a^m (before stage 1) or C (between
//          the stages); outer rows/columns hold the Dirichlet data.
//   Vb     v^m (natural), V layout.
//   Wb     w* (carried), W layout.
//   alpha  dt/2 * c^2 at U's points.
//   Uo, Wo natural u, w, written by the last stage-2 launch of every adi_step call.
//   tab    head/tail elimination tables, one kTabLine record per line (rows then columns).
//   scratch  per-line scratch of the line solver.
// One time step = stage-1 launch over the x-lines + stage-2 launch over the y-lines.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/adi.h"
#include "adi_internal.h"
#include "adi_ops.cuh"

using namespace adi;

namespace {

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct Geometry {
    int method, nx, ny;
    int rows_u, ldu, rows_v, ldv, rows_w, ldw;
    int pix, piy;  // interior pressure counts along x and y
    size_t nU() const { return (size_t)rows_u * ldu; }
    size_t nV() const { return (size_t)rows_v * ldv; }
    size_t nW() const { return (size_t)rows_w * ldw; }
};

Geometry make_geometry(int method, int nx, int ny) {
    Geometry g;
    g.method = method; g.nx = nx; g.ny = ny;
    if (method == ADI_CFD) {
        g.rows_u = g.rows_v = g.rows_w = ny + 1;
        g.ldu = g.ldv = g.ldw = nx + 1;
        g.pix = nx - 1; g.piy = ny - 1;
    } else {
        g.rows_u = ny + 2; g.ldu = nx + 2;
        g.rows_v = ny + 2; g.ldv = nx + 1;
        g.rows_w = ny + 1; g.ldw = nx + 2;
        g.pix = nx; g.piy = ny;
    }
    return g;
}

size_t elem_size(int precision) { return precision == ADI_FP64 ? 8 : 4; }

}  // namespace

struct adi_sim {
    Geometry g;
    int precision = ADI_FP32;
    double h = 0, dt = 0;
    size_t esz = 4;
    DevBuf A, Vb, Wb, alpha, Uo, Wo, tab, scratch, rowd, cold, clock, status;
    long long scratch_stride = 0;
    int n_row = 0, n_col = 0;
    std::vector<unsigned char> h_rowd, h_cold;  // host copies of the descriptors
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    long long steps = 0;
    int sticky = ADI_OK;
    bool in_batch = false;
    cudaStream_t batch_stream = nullptr;
    bool src_on = false;
    int src_i = 0, src_j = 0;
    double src_amp = 0, src_f0 = 0, src_td = 0;
    std::map<int, cudaGraphExec_t> graphs;
};

struct adi_batch_t {
    std::vector<adi_sim *> sims;
    int precision = ADI_FP32;
    DevBuf rowd, cold, scratch;
    int n_row = 0, n_col = 0;
    long long scratch_stride = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int sticky = ADI_OK;
    std::map<int, cudaGraphExec_t> graphs;
};

namespace {

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return ADI_OK;
    if (e == cudaErrorMemoryAllocation) return ADI_ENOMEM;
    if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) return ADI_ENOTSUP;
    return ADI_ECUDA;
}

int dev_alloc(DevBuf &b, size_t bytes) {
    b.bytes = bytes;
    if (bytes == 0) { b.p = nullptr; return ADI_OK; }
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) { b.p = nullptr; (void)cudaGetLastError(); return cuda_status(e); }
    return ADI_OK;
}
void dev_free(DevBuf &b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr; b.bytes = 0;
}

template <typename T>
__global__ void convert_from_double(const double *src, T *dst, size_t n, double scale, int square) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < n) {
        double x = src[i];
        dst[i] = (T)(square ? scale * x * x : scale * x);
    }
}
template <typename T>
__global__ void convert_to_double(const T *src, double *dst, size_t n) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (double)src[i];
}

// Uploads a host double array into a device array of the sim's precision; scale*x or
// scale*x^2 (used for alpha = dt/2 c^2).  staging must hold n doubles.
int upload(adi_sim *s, const double *host, void *dst, size_t n, double *staging, double scale,
           int square) {
    if (n == 0) return ADI_OK;
    cudaError_t e;
    if (host)
        e = cudaMemcpyAsync(staging, host, n * sizeof(double), cudaMemcpyHostToDevice, s->stream);
    else
        e = cudaMemsetAsync(staging, 0, n * sizeof(double), s->stream);
    if (e != cudaSuccess) return cuda_status(e);
    unsigned blocks = (unsigned)((n + 255) / 256);
    if (s->precision == ADI_FP64)
        convert_from_double<double><<<blocks, 256, 0, s->stream>>>(staging, (double *)dst, n, scale, square);
    else
        convert_from_double<float><<<blocks, 256, 0, s->stream>>>(staging, (float *)dst, n, scale, square);
    return cuda_status(cudaGetLastError());
}

template <typename T>
void fill_descs(adi_sim *s, std::vector<LineDesc<T>> &rows, std::vector<LineDesc<T>> &cols) {
    const Geometry &g = s->g;
    T *A = (T *)s->A.p, *V = (T *)s->Vb.p, *W = (T *)s->Wb.p, *Uo = (T *)s->Uo.p, *Wo = (T *)s->Wo.p;
    const T *al = (const T *)s->alpha.p;
    const T *tab = (const T *)s->tab.p;
    LineDesc<T> base;
    std::memset(&base, 0, sizeof(base));
    base.method = g.method;
    base.beta = 0.5 * s->dt;
    base.inv_h = 1.0 / s->h;
    base.dt = s->dt;
    base.clock = (long long *)s->clock.p;
    base.src_k = -1;
    base.src_amp = s->src_amp; base.src_f0 = s->src_f0; base.src_tdelay = s->src_td;
    base.src_scale = s->dt / (2.0 * s->h * s->h);
    rows.assign(g.piy, base);
    cols.assign(g.pix, base);
    for (int r = 0; r < g.piy; ++r) {
        int i = r + 1;  // grid row of this x-line
        LineDesc<T> &d = rows[r];
        d.p = A + (size_t)i * g.ldu;
        d.alpha = al + (size_t)i * g.ldu;
        d.v = V + (size_t)i * g.ldv;
        d.u_out = nullptr; d.w_out = nullptr;
        d.sp = 1; d.sv = 1;
        d.N = g.nx;
        d.tab = tab + (size_t)r * kTabLine;
        if (s->src_on && s->src_i == i) d.src_k = s->src_j;
        d.advance_clock = 0;
    }
    for (int c = 0; c < g.pix; ++c) {
        int j = c + 1;  // grid column of this y-line
        LineDesc<T> &d = cols[c];
        d.p = A + j;
        d.alpha = al + j;
        d.v = W + j;
        d.u_out = Uo + j;
        d.w_out = Wo + j;
        d.sp = g.ldu; d.sv = g.ldw;
        d.N = g.ny;
        d.tab = tab + (size_t)(g.piy + c) * kTabLine;
        if (s->src_on && s->src_j == j) { d.src_k = s->src_i; d.advance_clock = 1; }
    }
}

template <typename T>
int upload_descs(adi_sim *s) {
    std::vector<LineDesc<T>> rows, cols;
    fill_descs<T>(s, rows, cols);
    s->h_rowd.assign((unsigned char *)rows.data(), (unsigned char *)(rows.data() + rows.size()));
    s->h_cold.assign((unsigned char *)cols.data(), (unsigned char *)(cols.data() + cols.size()));
    cudaError_t e = cudaMemcpyAsync(s->rowd.p, rows.data(), rows.size() * sizeof(LineDesc<T>),
                                    cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->cold.p, cols.data(), cols.size() * sizeof(LineDesc<T>),
                            cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    return cuda_status(e);
}

size_t scratch_words_for(const Geometry &g) {
    return std::max(v1_scratch_words(g.method, g.nx), v1_scratch_words(g.method, g.ny));
}

template <typename T>
int run_prologue(adi_sim *s) {
    cudaError_t e = launch_prologue<T>((const LineDesc<T> *)s->cold.p, s->n_col, nullptr, nullptr,
                                       0, 0, (T *)s->scratch.p, s->scratch_stride, s->stream);
    return cuda_status(e);
}

int prologue(adi_sim *s) {
    return s->precision == ADI_FP64 ? run_prologue<double>(s) : run_prologue<float>(s);
}

template <typename T>
int run_precompute(adi_sim *s) {
    cudaError_t e = cudaMemsetAsync(s->status.p, 0, sizeof(int), s->stream);
    if (e == cudaSuccess)
        e = launch_precompute<T>((const LineDesc<T> *)s->rowd.p, s->n_row, (T *)s->tab.p,
                                 (int *)s->status.p, s->stream);
    if (e == cudaSuccess)
        e = launch_precompute<T>((const LineDesc<T> *)s->cold.p, s->n_col,
                                 (T *)s->tab.p + (size_t)s->n_row * kTabLine, (int *)s->status.p,
                                 s->stream);
    int st = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&st, s->status.p, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_status(e);
    return st ? ADI_ESINGULAR : ADI_OK;
}

// Enqueues one full step (both stages) for a set of row and column descriptors.
template <typename T>
cudaError_t enqueue_step(const void *rowd, int n_row, const void *cold, int n_col, void *scratch,
                         long long st, int natural, cudaStream_t stream) {
    cudaError_t e = launch_line_solve_v1<T>((const LineDesc<T> *)rowd, n_row, (T *)scratch, st, 0,
                                            stream);
    if (e != cudaSuccess) return e;
    return launch_line_solve_v1<T>((const LineDesc<T> *)cold, n_col, (T *)scratch, st, natural,
                                   stream);
}

cudaError_t enqueue_steps(int precision, const void *rowd, int n_row, const void *cold, int n_col,
                          void *scratch, long long st, int nsteps, cudaStream_t stream) {
    for (int k = 0; k < nsteps; ++k) {
        int natural = (k == nsteps - 1) ? 1 : 0;
        cudaError_t e = precision == ADI_FP64
                            ? enqueue_step<double>(rowd, n_row, cold, n_col, scratch, st, natural, stream)
                            : enqueue_step<float>(rowd, n_row, cold, n_col, scratch, st, natural, stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Captures nsteps into a graph (cached per step count) and launches it.
cudaError_t run_graph(std::map<int, cudaGraphExec_t> &cache, int precision, const void *rowd,
                      int n_row, const void *cold, int n_col, void *scratch, long long st,
                      int nsteps, cudaStream_t stream) {
    auto it = cache.find(nsteps);
    if (it == cache.end()) {
        cudaStream_t cap;
        cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
        e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) { cudaStreamDestroy(cap); return e; }
        cudaError_t le = enqueue_steps(precision, rowd, n_row, cold, n_col, scratch, st, nsteps, cap);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(cap, &graph);
        cudaStreamDestroy(cap);
        if (le != cudaSuccess) { if (graph) cudaGraphDestroy(graph); return le; }
        if (e != cudaSuccess) return e;
        cudaGraphExec_t exec;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return e;
        it = cache.emplace(nsteps, exec).first;
    }
    return cudaGraphLaunch(it->second, stream);
}

void drop_graphs(std::map<int, cudaGraphExec_t> &cache) {
    for (auto &kv : cache) cudaGraphExecDestroy(kv.second);
    cache.clear();
}

bool finite_positive(const double *x, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!(std::isfinite(x[i]) && x[i] > 0.0)) return false;
    return true;
}
bool all_finite(const double *x, size_t n) {
    if (!x) return true;
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(x[i])) return false;
    return true;
}

size_t desc_size(int precision) {
    return precision == ADI_FP64 ? sizeof(LineDesc<double>) : sizeof(LineDesc<float>);
}

}  // namespace

extern "C" {

int adi_abi_version(void) { return 1; }

const char *adi_strerror(int code) {
    switch (code) {
    case ADI_OK: return "ok";
    case ADI_EINVAL: return "invalid argument";
    case ADI_ENOMEM: return "out of device memory or over budget";
    case ADI_ECUDA: return "CUDA error";
    case ADI_ENONFINITE: return "non-finite value in a field";
    case ADI_ETIMEOUT: return "bounded wait timed out";
    case ADI_EBUSY: return "object is busy";
    case ADI_ENOTSUP: return "no usable CUDA device or unsupported configuration";
    case ADI_ESINGULAR: return "singular line-system block";
    }
    return "unknown error";
}

size_t adi_state_bytes(int method, int nx, int ny, int precision) {
    if ((method != ADI_CFD && method != ADI_MFD) || nx < ADI_MIN_CELLS || ny < ADI_MIN_CELLS ||
        nx > ADI_MAX_CELLS || ny > ADI_MAX_CELLS || (precision != ADI_FP32 && precision != ADI_FP64))
        return 0;
    Geometry g = make_geometry(method, nx, ny);
    size_t esz = elem_size(precision);
    size_t nl = (size_t)g.pix + g.piy;
    size_t fields = (3 * g.nU() + g.nV() + 2 * g.nW()) * esz;  // A, alpha, Uo, Vb, Wb, Wo
    size_t tab = nl * kTabLine * esz;
    size_t scratch = scratch_words_for(g) * std::max(g.pix, g.piy) * esz;
    size_t descs = nl * desc_size(precision);
    return fields + tab + scratch + descs + 2 * sizeof(long long);
}

int adi_create(adi_handle *out, int method, int nx, int ny, double h, double dt,
               const double *c_field, const double *u0, const double *v0, const double *w0,
               int precision) {
    if (!out) return ADI_EINVAL;
    *out = nullptr;
    if ((method != ADI_CFD && method != ADI_MFD) || nx < ADI_MIN_CELLS || ny < ADI_MIN_CELLS ||
        nx > ADI_MAX_CELLS || ny > ADI_MAX_CELLS || (precision != ADI_FP32 && precision != ADI_FP64) ||
        !(std::isfinite(h) && h > 0) || !(std::isfinite(dt) && dt > 0) || !c_field)
        return ADI_EINVAL;
    Geometry g = make_geometry(method, nx, ny);
    if (!finite_positive(c_field, g.nU()) || !all_finite(u0, g.nU()) || !all_finite(v0, g.nV()) ||
        !all_finite(w0, g.nW()))
        return ADI_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) { (void)cudaGetLastError(); return ADI_ENOTSUP; }

    adi_sim *s = new (std::nothrow) adi_sim;
    if (!s) return ADI_ENOMEM;
    s->g = g; s->precision = precision; s->h = h; s->dt = dt; s->esz = elem_size(precision);
    s->n_row = g.piy; s->n_col = g.pix;
    int rc = ADI_OK;
    cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { delete s; return cuda_status(e); }
    s->own_stream = true;
    const size_t esz = s->esz;
    s->scratch_stride = std::max(g.pix, g.piy);
    if (!rc) rc = dev_alloc(s->A, g.nU() * esz);
    if (!rc) rc = dev_alloc(s->alpha, g.nU() * esz);
    if (!rc) rc = dev_alloc(s->Uo, g.nU() * esz);
    if (!rc) rc = dev_alloc(s->Vb, g.nV() * esz);
    if (!rc) rc = dev_alloc(s->Wb, g.nW() * esz);
    if (!rc) rc = dev_alloc(s->Wo, g.nW() * esz);
    if (!rc) rc = dev_alloc(s->tab, (size_t)(g.pix + g.piy) * kTabLine * esz);
    if (!rc) rc = dev_alloc(s->scratch, scratch_words_for(g) * (size_t)s->scratch_stride * esz);
    if (!rc) rc = dev_alloc(s->rowd, (size_t)g.piy * desc_size(precision));
    if (!rc) rc = dev_alloc(s->cold, (size_t)g.pix * desc_size(precision));
    if (!rc) rc = dev_alloc(s->clock, sizeof(long long));
    if (!rc) rc = dev_alloc(s->status, sizeof(int));
    DevBuf staging;
    if (!rc) rc = dev_alloc(staging, std::max(g.nU(), std::max(g.nV(), g.nW())) * sizeof(double));
    if (!rc) rc = cuda_status(cudaMemsetAsync(s->clock.p, 0, sizeof(long long), s->stream));
    // alpha = dt/2 c^2 ; natural U, W ; v ; the carried buffers get the natural values first
    if (!rc) rc = upload(s, c_field, s->alpha.p, g.nU(), (double *)staging.p, 0.5 * dt, 1);
    if (!rc) rc = upload(s, u0, s->Uo.p, g.nU(), (double *)staging.p, 1.0, 0);
    if (!rc) rc = upload(s, v0, s->Vb.p, g.nV(), (double *)staging.p, 1.0, 0);
    if (!rc) rc = upload(s, w0, s->Wo.p, g.nW(), (double *)staging.p, 1.0, 0);
    if (!rc) rc = cuda_status(cudaMemcpyAsync(s->A.p, s->Uo.p, g.nU() * esz, cudaMemcpyDeviceToDevice, s->stream));
    if (!rc) rc = cuda_status(cudaMemcpyAsync(s->Wb.p, s->Wo.p, g.nW() * esz, cudaMemcpyDeviceToDevice, s->stream));
    if (!rc) rc = cuda_status(cudaStreamSynchronize(s->stream));
    dev_free(staging);
    if (!rc) rc = precision == ADI_FP64 ? upload_descs<double>(s) : upload_descs<float>(s);
    if (!rc) rc = precision == ADI_FP64 ? run_precompute<double>(s) : run_precompute<float>(s);
    if (!rc) rc = prologue(s);
    if (!rc) rc = cuda_status(cudaStreamSynchronize(s->stream));
    if (rc) { adi_destroy(s); return rc; }
    *out = s;
    return ADI_OK;
}

int adi_set_stream(adi_handle s, void *stream) {
    if (!s) return ADI_EINVAL;
    if (s->own_stream) { cudaStreamSynchronize(s->stream); cudaStreamDestroy(s->stream); s->own_stream = false; }
    s->stream = (cudaStream_t)stream;
    return ADI_OK;
}

int adi_set_source(adi_handle s, int is, int js, double amp, double f0, double tdelay) {
    if (!s) return ADI_EINVAL;
    if (s->sticky) return s->sticky;
    if (s->in_batch) return ADI_EBUSY;
    const Geometry &g = s->g;
    if (is < 1 || is > g.piy || js < 1 || js > g.pix || !std::isfinite(amp) || !std::isfinite(f0) ||
        !std::isfinite(tdelay))
        return ADI_EINVAL;
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return s->sticky = cuda_status(e);
    s->src_on = true; s->src_i = is; s->src_j = js;
    s->src_amp = amp; s->src_f0 = f0; s->src_td = tdelay;
    int rc = s->precision == ADI_FP64 ? upload_descs<double>(s) : upload_descs<float>(s);
    if (!rc) rc = prologue(s);  // a picks up dt/2 f(t_now) at the source point
    if (!rc) rc = cuda_status(cudaStreamSynchronize(s->stream));
    if (rc) s->sticky = rc;
    return rc;
}

int adi_step(adi_handle s, int nsteps) {
    if (!s || nsteps < 0) return ADI_EINVAL;
    if (s->sticky) return s->sticky;
    if (s->in_batch) return ADI_EBUSY;
    if (nsteps == 0) return ADI_OK;
    cudaError_t e;
    if (nsteps == 1)
        e = enqueue_steps(s->precision, s->rowd.p, s->n_row, s->cold.p, s->n_col, s->scratch.p,
                          s->scratch_stride, 1, s->stream);
    else
        e = run_graph(s->graphs, s->precision, s->rowd.p, s->n_row, s->cold.p, s->n_col,
                      s->scratch.p, s->scratch_stride, nsteps, s->stream);
    if (e != cudaSuccess) return s->sticky = cuda_status(e);
    s->steps += nsteps;
    return ADI_OK;
}

int adi_sync(adi_handle s) {
    if (!s) return ADI_EINVAL;
    if (s->sticky) return s->sticky;
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) s->sticky = cuda_status(e);
    return s->sticky;
}

int adi_read_fields(adi_handle s, double *u, double *v, double *w) {
    if (!s) return ADI_EINVAL;
    if (s->in_batch && s->batch_stream) {
        cudaError_t be = cudaStreamSynchronize(s->batch_stream);
        if (be != cudaSuccess) return s->sticky = cuda_status(be);
    }
    int rc = adi_sync(s);
    if (rc) return rc;
    const Geometry &g = s->g;
    struct { const void *src; double *dst; size_t n; } parts[3] = {
        {s->Uo.p, u, g.nU()}, {s->Vb.p, v, g.nV()}, {s->Wo.p, w, g.nW()}};
    DevBuf tmp;
    rc = dev_alloc(tmp, std::max(g.nU(), std::max(g.nV(), g.nW())) * sizeof(double));
    if (rc) return rc;
    for (auto &pt : parts) {
        if (!pt.dst) continue;
        unsigned blocks = (unsigned)((pt.n + 255) / 256);
        if (s->precision == ADI_FP64)
            convert_to_double<double><<<blocks, 256, 0, s->stream>>>((const double *)pt.src, (double *)tmp.p, pt.n);
        else
            convert_to_double<float><<<blocks, 256, 0, s->stream>>>((const float *)pt.src, (double *)tmp.p, pt.n);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(pt.dst, tmp.p, pt.n * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) { dev_free(tmp); return s->sticky = cuda_status(e); }
    }
    dev_free(tmp);
    return ADI_OK;
}

int adi_set_fields(adi_handle s, const double *u, const double *v, const double *w) {
    if (!s) return ADI_EINVAL;
    if (s->in_batch && s->batch_stream) {
        cudaError_t be = cudaStreamSynchronize(s->batch_stream);
        if (be != cudaSuccess) return s->sticky = cuda_status(be);
    }
    int rc = adi_sync(s);
    if (rc) return rc;
    const Geometry &g = s->g;
    if (!all_finite(u, g.nU()) || !all_finite(v, g.nV()) || !all_finite(w, g.nW())) return ADI_EINVAL;
    DevBuf staging;
    rc = dev_alloc(staging, std::max(g.nU(), std::max(g.nV(), g.nW())) * sizeof(double));
    if (rc) return rc;
    if (!rc && u) rc = upload(s, u, s->Uo.p, g.nU(), (double *)staging.p, 1.0, 0);
    if (!rc && u) rc = cuda_status(cudaMemcpyAsync(s->A.p, s->Uo.p, g.nU() * s->esz, cudaMemcpyDeviceToDevice, s->stream));
    if (!rc && v) rc = upload(s, v, s->Vb.p, g.nV(), (double *)staging.p, 1.0, 0);
    if (!rc && w) rc = upload(s, w, s->Wo.p, g.nW(), (double *)staging.p, 1.0, 0);
    if (!rc) rc = cuda_status(cudaMemcpyAsync(s->Wb.p, s->Wo.p, g.nW() * s->esz, cudaMemcpyDeviceToDevice, s->stream));
    if (!rc) rc = prologue(s);
    if (!rc) rc = cuda_status(cudaStreamSynchronize(s->stream));
    dev_free(staging);
    if (rc) s->sticky = rc;
    return rc;
}

int adi_check_finite(adi_handle s) {
    if (!s) return ADI_EINVAL;
    int rc = adi_sync(s);
    if (rc) return rc;
    cudaError_t e = cudaMemsetAsync(s->status.p, 0, sizeof(int), s->stream);
    const Geometry &g = s->g;
    const void *fields[4] = {s->A.p, s->Vb.p, s->Wb.p, s->Uo.p};
    size_t ns[4] = {g.nU(), g.nV(), g.nW(), g.nU()};
    for (int k = 0; k < 4 && e == cudaSuccess; ++k)
        e = s->precision == ADI_FP64
                ? launch_finite_check<double>((const double *)fields[k], ns[k], (int *)s->status.p, s->stream)
                : launch_finite_check<float>((const float *)fields[k], ns[k], (int *)s->status.p, s->stream);
    int flag = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, s->status.p, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return s->sticky = cuda_status(e);
    if (flag) return s->sticky = ADI_ENONFINITE;
    return ADI_OK;
}

int adi_get_time(adi_handle s, long long *steps, double *t) {
    if (!s) return ADI_EINVAL;
    if (steps) *steps = s->steps;
    if (t) *t = s->steps * s->dt;
    return ADI_OK;
}

int adi_destroy(adi_handle s) {
    if (!s) return ADI_OK;
    if (s->stream) cudaStreamSynchronize(s->stream);
    drop_graphs(s->graphs);
    DevBuf *bufs[] = {&s->A, &s->Vb, &s->Wb, &s->alpha, &s->Uo, &s->Wo, &s->tab, &s->scratch,
                      &s->rowd, &s->cold, &s->clock, &s->status};
    for (DevBuf *b : bufs) dev_free(*b);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    (void)cudaGetLastError();
    delete s;
    return ADI_OK;
}

// ----------------------------------------------------------------------------------------
// Batches: every member's x-lines in one descriptor table, y-lines in another.
// ----------------------------------------------------------------------------------------
int adi_batch_create(adi_batch *out, const adi_handle *sims, int n) {
    if (!out || !sims || n < 1) return ADI_EINVAL;
    *out = nullptr;
    int prec = sims[0] ? sims[0]->precision : -1;
    for (int k = 0; k < n; ++k) {
        if (!sims[k]) return ADI_EINVAL;
        if (sims[k]->precision != prec) return ADI_EINVAL;
        if (sims[k]->in_batch) return ADI_EBUSY;
        if (sims[k]->sticky) return sims[k]->sticky;
        for (int q = 0; q < k; ++q)
            if (sims[q] == sims[k]) return ADI_EINVAL;
    }
    adi_batch_t *b = new (std::nothrow) adi_batch_t;
    if (!b) return ADI_ENOMEM;
    b->precision = prec;
    size_t dsz = desc_size(prec), esz = elem_size(prec);
    std::vector<unsigned char> rows, cols;
    size_t words = 0;
    for (int k = 0; k < n; ++k) {
        adi_sim *s = sims[k];
        cudaStreamSynchronize(s->stream);
        b->sims.push_back(s);
        rows.insert(rows.end(), s->h_rowd.begin(), s->h_rowd.end());
        cols.insert(cols.end(), s->h_cold.begin(), s->h_cold.end());
        words = std::max(words, scratch_words_for(s->g));
    }
    b->n_row = (int)(rows.size() / dsz);
    b->n_col = (int)(cols.size() / dsz);
    b->scratch_stride = std::max(b->n_row, b->n_col);
    int rc = cuda_status(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
    if (!rc) b->own_stream = true;
    if (!rc) rc = dev_alloc(b->rowd, rows.size());
    if (!rc) rc = dev_alloc(b->cold, cols.size());
    if (!rc) rc = dev_alloc(b->scratch, words * (size_t)b->scratch_stride * esz);
    if (!rc) rc = cuda_status(cudaMemcpy(b->rowd.p, rows.data(), rows.size(), cudaMemcpyHostToDevice));
    if (!rc) rc = cuda_status(cudaMemcpy(b->cold.p, cols.data(), cols.size(), cudaMemcpyHostToDevice));
    if (rc) { adi_batch_destroy(b); return rc; }
    for (adi_sim *s : b->sims) { s->in_batch = true; s->batch_stream = b->stream; }
    *out = b;
    return ADI_OK;
}

int adi_batch_set_stream(adi_batch b, void *stream) {
    if (!b) return ADI_EINVAL;
    if (b->own_stream) { cudaStreamSynchronize(b->stream); cudaStreamDestroy(b->stream); b->own_stream = false; }
    b->stream = (cudaStream_t)stream;
    for (adi_sim *s : b->sims) s->batch_stream = b->stream;
    return ADI_OK;
}

int adi_batch_step(adi_batch b, int nsteps) {
    if (!b || nsteps < 0) return ADI_EINVAL;
    if (b->sticky) return b->sticky;
    if (nsteps == 0) return ADI_OK;
    cudaError_t e = run_graph(b->graphs, b->precision, b->rowd.p, b->n_row, b->cold.p, b->n_col,
                              b->scratch.p, b->scratch_stride, nsteps, b->stream);
    if (e != cudaSuccess) {
        b->sticky = cuda_status(e);
        for (adi_sim *s : b->sims) s->sticky = b->sticky;
        return b->sticky;
    }
    for (adi_sim *s : b->sims) s->steps += nsteps;
    return ADI_OK;
}

int adi_batch_half_step(adi_batch b, int stage, int write_natural) {
    if (!b || (stage != 1 && stage != 2)) return ADI_EINVAL;
    if (b->sticky) return b->sticky;
    cudaError_t e;
    const void *d = stage == 1 ? b->rowd.p : b->cold.p;
    int n = stage == 1 ? b->n_row : b->n_col;
    int nat = stage == 2 && write_natural ? 1 : 0;
    if (b->precision == ADI_FP64)
        e = launch_line_solve_v1<double>((const LineDesc<double> *)d, n, (double *)b->scratch.p,
                                         b->scratch_stride, nat, b->stream);
    else
        e = launch_line_solve_v1<float>((const LineDesc<float> *)d, n, (float *)b->scratch.p,
                                        b->scratch_stride, nat, b->stream);
    if (e != cudaSuccess) {
        b->sticky = cuda_status(e);
        for (adi_sim *s : b->sims) s->sticky = b->sticky;
        return b->sticky;
    }
    if (stage == 2)
        for (adi_sim *s : b->sims) s->steps += 1;
    return ADI_OK;
}

int adi_batch_sync(adi_batch b) {
    if (!b) return ADI_EINVAL;
    if (b->sticky) return b->sticky;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        b->sticky = cuda_status(e);
        for (adi_sim *s : b->sims) s->sticky = b->sticky;
    }
    return b->sticky;
}

int adi_batch_destroy(adi_batch b) {
    if (!b) return ADI_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_graphs(b->graphs);
    dev_free(b->rowd); dev_free(b->cold); dev_free(b->scratch);
    for (adi_sim *s : b->sims) { s->in_batch = false; s->batch_stream = nullptr; }
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    (void)cudaGetLastError();
    delete b;
    return ADI_OK;
}

}  // extern "C"
