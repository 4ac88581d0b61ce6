// adi_static.cu -- adi_step_static: one time step of a small simulation whose fields the
// caller keeps in device memory, with every temporary of the library placed in one
// fixed-size device array compiled into libadi.  Nothing is allocated on the device or the
// host heap: the array's address is looked up once per device (cudaGetSymbolAddress) and
// handed to the same kernels the handle path launches with the thread-per-line solver
// (head/tail tables, carried-state prologue, x-line and y-line solves).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/adi.h"
#include "adi_internal.h"
#include "adi_ops.cuh"

using namespace adi;

namespace {

// Capacity of the scratch array.  A grid of ADI_STATIC_MAX_CELLS^2 cells in FP64 needs about
// 2.1 MB (CFD) or 1.8 MB (MFD); the exact need is computed per call and checked.
constexpr size_t kStaticBytes = (size_t)4 << 20;
__device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices];  // device address of g_static_scratch, per device ordinal
std::mutex g_setup_mutex;

int status_of(cudaError_t e) {
    if (e == cudaSuccess) return ADI_OK;
    if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) return ADI_ENOTSUP;
    return ADI_ECUDA;
}

// Address of the scratch array on the current device; the first call for a device looks it
// up with that device current and keeps it for the life of the process (a cudaDeviceReset,
// or a driver context other than the device's primary one, would make the kept address
// stale: the entry point is for processes that keep one primary context per device).
int scratch_on_current_device(unsigned char **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { (void)cudaGetLastError(); return status_of(e); }
    if (dev < 0 || dev >= kMaxDevices) return ADI_ENOTSUP;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) { (void)cudaGetLastError(); return e != cudaSuccess ? status_of(e) : ADI_ECUDA; }
        g_scratch_addr[dev] = p;
    }
    *out = (unsigned char *)g_scratch_addr[dev];
    return ADI_OK;
}

struct Shape {
    int ldu, ldv, ldw;   // row lengths of U, V, W
    int pix, piy;        // interior pressure counts along x (y-lines) and y (x-lines)
    size_t nU, nV, nW;
};

Shape shape_of(int method, int nx, int ny) {
    Shape g;
    if (method == ADI_CFD) {
        g.ldu = g.ldv = g.ldw = nx + 1;
        g.nU = g.nV = g.nW = (size_t)(ny + 1) * (nx + 1);
        g.pix = nx - 1; g.piy = ny - 1;
    } else {
        g.ldu = nx + 2; g.ldv = nx + 1; g.ldw = nx + 2;
        g.nU = (size_t)(ny + 2) * (nx + 2);
        g.nV = (size_t)(ny + 2) * (nx + 1);
        g.nW = (size_t)(ny + 1) * (nx + 2);
        g.pix = nx; g.piy = ny;
    }
    return g;
}

// Byte offsets of the temporaries inside the scratch array (each 256-byte aligned).
struct Layout {
    size_t desc, status, alpha, A, C, W0, W1, tab, scr, end;
    long long st;  // word stride of the per-line solver scratch (lines side by side)
};

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

Layout layout_of(int method, int nx, int ny, const Shape &g, size_t esz) {
    Layout L;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = up256(off + bytes);
        return o;
    };
    const size_t nl = (size_t)g.pix + g.piy;
    L.desc = take(nl * sizeof(LineDesc<double>));  // LineDesc<float> has the same size
    L.status = take(sizeof(int));
    L.alpha = take(g.nU * esz);
    L.A = take(g.nU * esz);
    L.C = take(g.nU * esz);
    L.W0 = take(g.nW * esz);
    L.W1 = take(g.nW * esz);
    L.tab = take(nl * kTabLine * esz);
    L.st = std::max(g.pix, g.piy);
    size_t words = std::max(v1_scratch_words(method, nx), v1_scratch_words(method, ny));
    words = std::max(words, (size_t)(2 * ny + 4));  // the prologue's column solves
    L.scr = take(words * (size_t)L.st * esz);
    L.end = off;
    return L;
}

static_assert(sizeof(LineDesc<float>) == sizeof(LineDesc<double>), "descriptor sizes differ");

// Host staging of the descriptors: static storage, sized for the largest accepted grid.
constexpr int kMaxLines = 2 * ADI_STATIC_MAX_CELLS;
alignas(64) unsigned char g_host_descs[kMaxLines * sizeof(LineDesc<double>)];

template <typename T>
void fill_descs(int method, int nx, int ny, double h, double dt, const Shape &g,
                unsigned char *base, const Layout &L, const T *v_in, T *u_out, T *v_out, T *w_out,
                LineDesc<T> *out) {
    LineDesc<T> b;
    std::memset(&b, 0, sizeof(b));
    b.method = method;
    b.beta = 0.5 * dt;
    b.inv_h = 1.0 / h;
    b.dt = dt;
    b.src_k = -1;  // no source term
    T *A = (T *)(base + L.A), *C = (T *)(base + L.C);
    T *W0 = (T *)(base + L.W0), *W1 = (T *)(base + L.W1);
    const T *al = (const T *)(base + L.alpha);
    const T *tab = (const T *)(base + L.tab);
    for (int r = 0; r < g.piy; ++r) {  // x-lines: grid rows 1 .. piy
        const int i = r + 1;
        LineDesc<T> d = b;
        d.p = A + (size_t)i * g.ldu;
        d.po = C + (size_t)i * g.ldu;
        d.alpha = al + (size_t)i * g.ldu;
        d.v = const_cast<T *>(v_in) + (size_t)i * g.ldv;
        d.vo = v_out + (size_t)i * g.ldv;
        d.sp = d.sv = d.spo = d.svo = d.snp = d.snv = 1;
        d.N = nx;
        d.tab = tab + (size_t)r * kTabLine;
        out[r] = d;
    }
    for (int c = 0; c < g.pix; ++c) {  // y-lines: grid columns 1 .. pix
        const int j = c + 1;
        LineDesc<T> d = b;
        d.p = C + j;
        d.po = A + j;
        d.alpha = al + j;
        d.v = W0 + j;
        d.vo = W1 + j;
        d.u_out = u_out + j;
        d.w_out = w_out + j;
        d.sp = g.ldu; d.sv = g.ldw; d.spo = g.ldu; d.svo = g.ldw; d.snp = g.ldu; d.snv = g.ldw;
        d.N = ny;
        d.tab = tab + (size_t)(g.piy + c) * kTabLine;
        out[g.piy + c] = d;
    }
}

template <typename T>
__global__ void static_alpha_kernel(const T *__restrict__ c, T *__restrict__ alpha, size_t n,
                                    double half_dt) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < n) {
        double x = (double)c[i];
        alpha[i] = (T)(half_dt * x * x);
    }
}

template <typename T>
int step_static(int method, int nx, int ny, double h, double dt, const T *c, const T *u,
                const T *v, const T *w, T *u_out, T *v_out, T *w_out, cudaStream_t s) {
    unsigned char *base = nullptr;
    int rc = scratch_on_current_device(&base);
    if (rc) return rc;
    const Shape g = shape_of(method, nx, ny);
    const Layout L = layout_of(method, nx, ny, g, sizeof(T));
    if (L.end > kStaticBytes) return ADI_ENOMEM;
    const int nl = g.pix + g.piy;
    LineDesc<T> *hd = (LineDesc<T> *)g_host_descs;
    fill_descs<T>(method, nx, ny, h, dt, g, base, L, v, u_out, v_out, w_out, hd);
    LineDesc<T> *dd = (LineDesc<T> *)(base + L.desc);
    int *status = (int *)(base + L.status);
    T *alpha = (T *)(base + L.alpha), *A = (T *)(base + L.A), *C = (T *)(base + L.C);
    T *tab = (T *)(base + L.tab), *scr = (T *)(base + L.scr);
    const size_t esz = sizeof(T);

    cudaError_t e = cudaMemcpyAsync(dd, hd, (size_t)nl * sizeof(LineDesc<T>), cudaMemcpyHostToDevice, s);
    // the singular-pivot flag is the one temporary read before it is written
    if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int), s);
    if (e == cudaSuccess) {
        static_alpha_kernel<T><<<(unsigned)((g.nU + 255) / 256), 256, 0, s>>>(c, alpha, g.nU, 0.5 * dt);
        e = cudaGetLastError();
    }
    // Dirichlet data on the outer rows/columns of both carried pressure arrays; outputs start
    // as copies of the inputs (their outer entries are not updated by the step)
    if (e == cudaSuccess) e = cudaMemcpyAsync(A, u, g.nU * esz, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(C, u, g.nU * esz, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(u_out, u, g.nU * esz, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(v_out, v, g.nV * esz, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(w_out, w, g.nW * esz, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = launch_precompute<T>(dd, nl, tab, status, s);
    // carried state a, w* from the natural fields (read through the y-lines' u_out/w_out)
    if (e == cudaSuccess) e = launch_prologue<T>(dd + g.piy, g.pix, nullptr, scr, L.st, s);
    if (e == cudaSuccess) e = launch_line_solve_v1<T>(dd, g.piy, scr, L.st, 0, s);
    if (e == cudaSuccess) e = launch_line_solve_v1<T>(dd + g.piy, g.pix, scr, L.st, 1, s);
    int singular = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&singular, status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { (void)cudaGetLastError(); return status_of(e); }
    return singular ? ADI_ESINGULAR : ADI_OK;
}

// Every pointer must be device (or managed) memory of the current device: host memory
// handed here by mistake would fault the caller's context in the first copy or kernel, so it
// is refused before anything is enqueued.  cudaPointerGetAttributes allocates nothing.
int check_device_pointers(const void *const ins[4], const void *const outs[3]) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { (void)cudaGetLastError(); return status_of(e); }
    const void *all[7] = {ins[0], ins[1], ins[2], ins[3], outs[0], outs[1], outs[2]};
    for (const void *p : all) {
        cudaPointerAttributes a;
        std::memset(&a, 0, sizeof(a));
        e = cudaPointerGetAttributes(&a, p);
        if (e != cudaSuccess) { (void)cudaGetLastError(); return ADI_EINVAL; }
        if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) return ADI_EINVAL;
        if (a.device != dev) return ADI_EINVAL;
    }
    return ADI_OK;
}

}  // namespace

extern "C" int adi_step_static(int method, int nx, int ny, double h, double dt, int precision,
                               const void *c, const void *u, const void *v, const void *w,
                               void *u_out, void *v_out, void *w_out, void *cuda_stream) {
    if (method != ADI_CFD && method != ADI_MFD) return ADI_EINVAL;
    if (precision != ADI_FP32 && precision != ADI_FP64) return ADI_EINVAL;
    if (nx < ADI_MIN_CELLS || ny < ADI_MIN_CELLS) return ADI_EINVAL;
    if (!(h > 0.0) || !(dt > 0.0) || !std::isfinite(h) || !std::isfinite(dt)) return ADI_EINVAL;
    if (!c || !u || !v || !w || !u_out || !v_out || !w_out) return ADI_EINVAL;
    const void *ins[4] = {c, u, v, w};
    const void *outs[3] = {u_out, v_out, w_out};
    for (int o = 0; o < 3; ++o) {
        for (int i = 0; i < 4; ++i)
            if (outs[o] == ins[i]) return ADI_EINVAL;
        for (int k = o + 1; k < 3; ++k)
            if (outs[o] == outs[k]) return ADI_EINVAL;
    }
    if (nx > ADI_STATIC_MAX_CELLS || ny > ADI_STATIC_MAX_CELLS) return ADI_ENOMEM;
    {
        const int rc = check_device_pointers(ins, outs);
        if (rc) return rc;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (precision == ADI_FP64)
        return step_static<double>(method, nx, ny, h, dt, (const double *)c, (const double *)u,
                                   (const double *)v, (const double *)w, (double *)u_out,
                                   (double *)v_out, (double *)w_out, s);
    return step_static<float>(method, nx, ny, h, dt, (const float *)c, (const float *)u,
                              (const float *)v, (const float *)w, (float *)u_out, (float *)v_out,
                              (float *)w_out, s);
}
