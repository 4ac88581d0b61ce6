// adi_sponge.cu -- absorbing layers: Cerjan's damping, the technique Sec. 2.1 names for the
// CFD formulation.  After every full step, each field value at a point whose distance to the
// nearest wall is delta cells, delta < width, is multiplied by g = exp(-(a (width - delta))^2);
// the pressure's wall values (the Dirichlet data) are left alone.
//
// The line kernels carry (a, v, w*) from step to step, and pointwise damping of the natural
// fields does not commute with the non-local derivatives inside a and w*.  So a simulation with
// layers writes its natural fields every step; this kernel damps them (u, w natural; v, which
// the x-line stage leaves in natural form, in place) and the prologue kernels then rebuild
// the carried state from them, exactly as adi_set_fields does (adi_api.cu).
#include <cuda_runtime.h>

#include "../../include/adi.h"
#include "adi_internal.h"

namespace adi {

namespace {

// Coordinate in cells of index k along an axis of n cells: nodes for CFD and for the unstaggered
// axis of an MFD velocity; cell centres plus the two walls for a staggered MFD axis.
__device__ __forceinline__ double cell_coord(int method, bool staggered, int k, int n) {
    if (method == ADI_CFD || !staggered) return (double)k;
    if (k == 0) return 0.0;
    if (k == n + 1) return (double)n;
    return (double)k - 0.5;
}

__device__ __forceinline__ double damping(double x, double y, int nx, int ny, double width, double a) {
    double d = fmin(fmin(x, (double)nx - x), fmin(y, (double)ny - y));
    if (d >= width) return 1.0;
    const double q = a * (width - d);
    return exp(-q * q);
}

// blockIdx.y: 0 = u (natural, rows_u x ldu, interior only), 1 = v (rows_v x ldv, leading
// dimension ldvp), 2 = w (natural, rows_w x ldw).
template <typename T>
__global__ void sponge_kernel(SpongeRec r) {
    const int f = blockIdx.y;
    const int rows = f == 0 ? r.rows_u : (f == 1 ? r.rows_v : r.rows_w);
    const int cols = f == 0 ? r.ldu : (f == 1 ? r.ldv : r.ldw);
    const long long ld = f == 0 ? r.ldu : (f == 1 ? r.ldvp : r.ldw);
    T *x = (T *)(f == 0 ? r.uo : (f == 1 ? r.v : r.wo));
    const size_t n = (size_t)rows * cols;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(q / cols), j = (int)(q % cols);
        if (f == 0 && (i == 0 || j == 0 || i == rows - 1 || j == cols - 1)) continue;  // walls
        // u: both axes staggered (MFD); v: x on nodes, y staggered; w: x staggered, y on nodes
        const double xc = cell_coord(r.method, f != 1, j, r.nx);
        const double yc = cell_coord(r.method, f != 2, i, r.ny);
        const double g = damping(xc, yc, r.nx, r.ny, r.width, r.a);
        if (g != 1.0) {
            const T val = (T)((double)x[(size_t)i * ld + j] * g);
            x[(size_t)i * ld + j] = val;
            // v's first and last rows are not lines of the x-line stage, which therefore never
            // carries them from one copy to the other: both copies take the damped value
            if (f == 1 && (i == 0 || i == rows - 1)) ((T *)r.v_other)[(size_t)i * ld + j] = val;
        }
    }
}

}  // namespace

template <typename T>
cudaError_t launch_sponge(const SpongeRec &r, cudaStream_t s) {
    const size_t n = (size_t)(r.rows_u > r.rows_v ? r.rows_u : r.rows_v) * (size_t)(r.ldu + 1);
    const size_t want = (n + 255) / 256;
    const unsigned gx = (unsigned)(want < 1 ? 1 : (want > 4096 ? 4096 : want));
    sponge_kernel<T><<<dim3(gx, 3), 256, 0, s>>>(r);
    return cudaGetLastError();
}

template cudaError_t launch_sponge<float>(const SpongeRec &, cudaStream_t);
template cudaError_t launch_sponge<double>(const SpongeRec &, cudaStream_t);

}  // namespace adi
