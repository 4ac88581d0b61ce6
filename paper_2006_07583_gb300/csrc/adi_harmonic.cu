// adi_harmonic.cu -- time-harmonic Dirichlet walls and distributed forcing (the manufactured
// problem of Sec. 4, Eq. 11):  u = B cos(omega t + phb) on U's outer rows and columns,
// f = F cos(omega t + phf) at the interior pressure points.
//
// The line kernels take a line's Dirichlet values from the two end entries of its carried
// pressure line and add nothing but the point source, so the time dependence lives entirely
// in one small launch per stage over the members that have harmonic data, after the stage's
// transpose has put the carried pressure into the next stage's layout:
//   after stage 1 (C, column-major, read by the y-lines of stage 2):
//       C += dt/2 f(t_{m+1}) on the interior; the y-line ends (south/north walls) = u0(t_{m+1});
//   after stage 2 (a, row-major, read by the x-lines of the next stage 1):
//       a += dt/2 f(t_{m+1}) on the interior; the x-line ends (west/east walls) = u0(t_{m+1} +
//       dt/2), the intermediate wall value u* of the next step; the natural output's walls =
//       u0(t_{m+1}); then the member's step clock advances.
// Eqs. 6-7 add dt/2 f(t_m) to stage 1's right-hand side and dt/2 f(t_{m+1}) to stage 2's; in the
// carried form (C = 2u* - a + dt/2 f(t_{m+1}), a' = 2u - C + dt/2 f(t_{m+1})) both stages add the
// forcing at the step's new time level.  Every value of the time factor is evaluated in FP64.
#include <cuda_runtime.h>

#include "../../include/adi.h"
#include "adi_internal.h"

namespace adi {

namespace {

template <typename T>
__device__ __forceinline__ double wall(const HarmDesc &d, int side, int k, double t) {
    // side 0 west, 1 east (index k = row), 2 south, 3 north (index k = column)
    const double *e = d.edges + (side < 2 ? side * d.rows_u : 2 * d.rows_u + (side - 2) * d.ldu);
    return e[k] * cos(d.omega * t + d.phb);
}

// One member per blockIdx.y; the blocks of a member stride over its points.
template <typename T>
__global__ void harmonic_kernel(const HarmDesc *__restrict__ descs, int mode) {
    const HarmDesc &d = descs[blockIdx.y];
    const long long m = *d.clock;
    // modes: 0 after stage 1, 1 after stage 2, 2 natural walls before a prologue,
    // 3 carried state after a prologue (both at the clock's own time)
    const double t = (double)(mode <= 1 ? m + 1 : m) * d.dt;
    const int rows = d.rows_u, cols = d.ldu;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t first = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (mode == 0 || mode == 1 || mode == 3) {
        // forcing on the interior (rows 1 .. rows-2, columns 1 .. cols-2)
        if (d.f_row) {
            const T fs = (T)(0.5 * d.dt * cos(d.omega * t + d.phf));
            const size_t ni = (size_t)(rows - 2) * (cols - 2);
            if (mode == 0) {  // column-major C: column j contiguous
                T *C = (T *)d.c_col;
                const T *F = (const T *)d.f_col;
                for (size_t q = first; q < ni; q += stride) {
                    const size_t j = 1 + q / (rows - 2), i = 1 + q % (rows - 2);
                    C[j * d.ldc + i] += fs * F[j * d.ldc + i];
                }
            } else {          // row-major a
                T *A = (T *)d.a_row;
                const T *F = (const T *)d.f_row;
                for (size_t q = first; q < ni; q += stride) {
                    const size_t i = 1 + q / (cols - 2), j = 1 + q % (cols - 2);
                    A[i * d.lda + j] += fs * F[i * d.lda + j];
                }
            }
        }
    }
    if (mode == 0) {  // the y-line ends at t_{m+1}
        T *C = (T *)d.c_col;
        for (size_t j = first; j < (size_t)cols; j += stride) {
            C[j * d.ldc] = (T)wall<T>(d, 2, (int)j, t);
            C[j * d.ldc + rows - 1] = (T)wall<T>(d, 3, (int)j, t);
        }
    }
    if (mode == 1 || mode == 3) {  // the x-line ends: u* of the coming step at t + dt/2
        T *A = (T *)d.a_row;
        const double th = t + 0.5 * d.dt;
        for (size_t i = first; i < (size_t)rows; i += stride) {
            A[i * d.lda] = (T)wall<T>(d, 0, (int)i, th);
            A[i * d.lda + cols - 1] = (T)wall<T>(d, 1, (int)i, th);
        }
    }
    if (mode == 1 || mode == 2) {  // the natural pressure's walls at t
        T *U = (T *)d.uo;
        for (size_t i = first; i < (size_t)rows; i += stride) {
            U[i * cols] = (T)wall<T>(d, 0, (int)i, t);
            U[i * cols + cols - 1] = (T)wall<T>(d, 1, (int)i, t);
        }
        for (size_t j = first; j < (size_t)cols; j += stride) {
            U[j] = (T)wall<T>(d, 2, (int)j, t);
            U[(size_t)(rows - 1) * cols + j] = (T)wall<T>(d, 3, (int)j, t);
        }
    }
}

// Advances every member's step clock (after the stage-2 launch, once all of its threads
// have read the clock).
__global__ void harmonic_tick_kernel(const HarmDesc *__restrict__ descs, int n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) *descs[k].clock = *descs[k].clock + 1;
}

}  // namespace

template <typename T>
cudaError_t launch_harmonic(const HarmDesc *d, int n, size_t max_points, int mode, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const size_t want = (max_points + 255) / 256;
    const unsigned gx = (unsigned)(want < 1 ? 1 : (want > 2048 ? 2048 : want));
    harmonic_kernel<T><<<dim3(gx, (unsigned)n), 256, 0, s>>>(d, mode);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && mode == 1) {
        harmonic_tick_kernel<<<(n + 127) / 128, 128, 0, s>>>(d, n);
        e = cudaGetLastError();
    }
    return e;
}

template cudaError_t launch_harmonic<float>(const HarmDesc *, int, size_t, int, cudaStream_t);
template cudaError_t launch_harmonic<double>(const HarmDesc *, int, size_t, int, cudaStream_t);

}  // namespace adi
