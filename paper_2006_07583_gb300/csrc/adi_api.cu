// adi_api.cu -- host implementation of the C ABI in include/adi.h.
//
// Device state of one simulation (precision T).  Every line kernel reads and writes its
// lines contiguously: the fields a stage reads are stored with that stage's lines as rows, and
// the carried pressure changes layout between the stages through a tiled transpose after
// each stage.
//   A[0]   carried pressure a^m (stage-1 input), row-major U layout.
//   A[2]   carried C as stage 1 writes it, row-major; transposed into
//   A[1]   carried C (stage-2 input), column-major (column j of U is contiguous, leading
//          dimension ldc).
//   A[3]   carried a as stage 2 writes it, column-major; transposed into A[0].
//          Outer rows/columns of all four hold the Dirichlet data.
//   V[p]   v^m (natural), row-major V layout; W[p] w* (carried), column-major W layout.
//          Each half step reads one copy and writes the other (ping-pong, parity p flips
//          every step), because line kernels read stencil halos that neighbouring chunks
//          are writing.
//   alpha  dt/2 * c^2 at U's points, row-major; alphaT the same, column-major.
//   Uo, Wo natural u, w (row-major), written by the last stage-2 launch of every adi_step.
//   tab    head/tail elimination tables, one kTabLine record per line (rows then columns).
//   sep    per-line records of the chunked or factored solver.
// One time step = stage 1 over the x-lines + stage 2 over the y-lines.  Which kernels run is
// described by an execution plan (Plan): the thread-per-line solver for some members, the
// chunked or factored solver (one launch per method) for the others.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <new>
#include <vector>

#include "../../include/adi.h"
#include "adi_internal.h"
#include "adi_line.cuh"
#include "adi_ops.cuh"

using namespace adi;

namespace {

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return ADI_OK;
    if (e == cudaErrorMemoryAllocation) return ADI_ENOMEM;
    if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) return ADI_ENOTSUP;
    return ADI_ECUDA;
}

// Streaming multiprocessors of the current device (persistent grids).
int sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
        (void)cudaGetLastError();
        return 132;
    }
    return n;
}

int dev_alloc(DevBuf &b, size_t bytes) {
    b.bytes = bytes;
    if (bytes == 0) { b.p = nullptr; return ADI_OK; }
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) { b.p = nullptr; b.bytes = 0; (void)cudaGetLastError(); return cuda_status(e); }
    return ADI_OK;
}
void dev_free(DevBuf &b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr; b.bytes = 0;
}

struct Geometry {
    int method, nx, ny;
    int rows_u, ldu, rows_v, ldv, rows_w, ldw;  // natural (compact, row-major) layouts
    // carried layouts, leading dimensions padded to 32 elements so that every line starts
    // on a 128-byte boundary: lda (a and alpha, row-major), ldvp (v, row-major), ldc (C and
    // alphaT, column-major over U's ldu columns), ldwc (w*, column-major over W's ldw columns)
    int lda, ldvp, ldc, ldwc;
    int pix, piy;  // interior pressure counts along x and y
    size_t nU() const { return (size_t)rows_u * ldu; }
    size_t nV() const { return (size_t)rows_v * ldv; }
    size_t nW() const { return (size_t)rows_w * ldw; }
    size_t nA() const { return (size_t)rows_u * lda; }
    size_t nVp() const { return (size_t)rows_v * ldvp; }
    size_t nC() const { return (size_t)ldu * ldc; }
    size_t nWc() const { return (size_t)ldw * ldwc; }
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
    auto pad = [](int x) { return (x + 31) & ~31; };
    g.lda = pad(g.ldu);
    g.ldvp = pad(g.ldv);
    g.ldc = pad(g.rows_u);
    g.ldwc = pad(g.rows_w);
    return g;
}

size_t elem_size(int precision) { return precision == ADI_FP64 ? 8 : 4; }
size_t desc_size(int precision) {
    return precision == ADI_FP64 ? sizeof(LineDesc<double>) : sizeof(LineDesc<float>);
}
int block_size(int method) { return method == ADI_CFD ? 2 : 3; }

// Chunked-solver limits: chunks per line must fit one CTA of the kernel.
constexpr int kChunkThreads = 256;

int chunks_for(int method, int N) { return chunk_count(method, N, chunk_M(method)); }

bool chunked_ok_dir(int method, int N, size_t esz) {
    int T = chunks_for(method, N);
    return T <= kChunkThreads &&
           chunked_smem_bytes(N, 1, T, block_size(method), esz) <= (size_t)kChunkSmemMax;
}
bool chunked_ok(const Geometry &g, size_t esz) {
    return chunked_ok_dir(g.method, g.nx, esz) && chunked_ok_dir(g.method, g.ny, esz);
}

size_t sep_words(const Geometry &g) {
    int bs = block_size(g.method);
    size_t per = (size_t)3 * bs * bs;
    return ((size_t)g.piy * (chunks_for(g.method, g.nx) - 1) +
            (size_t)g.pix * (chunks_for(g.method, g.ny) - 1)) * per;
}
bool factored_ok(const Geometry &g, size_t esz) {
    return fac_supported(g.method, g.nx, esz) && fac_supported(g.method, g.ny, esz);
}
size_t fac_words_total(const Geometry &g) {
    return (size_t)g.piy * fac_words(g.method, g.nx) + (size_t)g.pix * fac_words(g.method, g.ny);
}
// per-line record words of the sim's solver (0 for the thread-per-line solver)
size_t solver_words(const Geometry &g, int solver) {
    if (solver == ADI_SOLVER_FACTORED) return fac_words_total(g);
    if (solver == ADI_SOLVER_CHUNKED) return sep_words(g);
    return 0;
}
int default_solver(const Geometry &g, size_t esz);

size_t v1_words(const Geometry &g) {
    return std::max(v1_scratch_words(g.method, g.nx), v1_scratch_words(g.method, g.ny));
}

// The factored solver where it applies (adi_autotune measured it fastest from 128^2 to 8192^2
// on GB300), else the chunked one, else one thread per line.
int default_solver(const Geometry &g, size_t esz) {
    if (factored_ok(g, esz)) return ADI_SOLVER_FACTORED;
    if (chunked_ok(g, esz)) return ADI_SOLVER_CHUNKED;
    return ADI_SOLVER_LINE;
}

// An execution plan: which kernels advance a set of simulations.
struct Plan {
    int precision = ADI_FP32;
    // thread-per-line members: descriptors per [parity][direction], and their scratch
    DevBuf v1d[2][2];
    int v1n[2] = {0, 0};
    DevBuf scratch;
    long long scratch_stride = 0;
    // chunked members: all descriptors per [parity][direction], line groups per [dir][method]
    DevBuf cd[2][2];
    DevBuf groups[2][2];
    int ngroups[2][2] = {{0, 0}, {0, 0}};
    size_t smem[2][2] = {{0, 0}, {0, 0}};
    // factored members: descriptors per [parity][direction], groups per [dir][kernel variant]
    DevBuf fd[2][2];
    DevBuf fgroups[2][kFacVariants];
    int nfgroups[2][kFacVariants] = {};
    size_t fstage[2][kFacVariants] = {};  // shared memory of one pipeline stage
    int fstages[2][kFacVariants] = {};    // staged groups in flight per CTA (1 to 3)
    int fgrid[2][kFacVariants] = {};      // persistent CTAs
    int fring[2][kFacVariants] = {};      // ring-depth cap of the launch (0: none)
    // carried-pressure transposes after each stage, one array per member: [dir]
    DevBuf tdesc[2];
    int tcount[2] = {0, 0}, trows[2] = {0, 0}, tcols[2] = {0, 0};
    // natural fields after a stage 2 that writes them: one record per member, per plan parity
    DevBuf ndesc[2];
    int ncount = 0, nrows = 0, ncols = 0;
    DevBuf fault;                            // set by a factored launch whose wait ran out
    // time-harmonic walls and forcing of the members that have them (after each stage)
    DevBuf hdesc;
    int hcount = 0;
    size_t hmax = 0;
    // absorbing layers: per member with layers, what runs after its stage 2 (per plan parity q)
    struct SpongeStep {
        SpongeRec rec[2];         // the natural fields to damp (v: the copy stage 1 wrote)
        const void *ydesc[2];     // y-line descriptors of the next step's parity
        int nlines = 0, N = 0, method = 0;
        void *scr = nullptr;      // prologue scratch, then (CFD) the Thomas factors
        const void *fac = nullptr;
        long long st = 1;
        void *A3 = nullptr, *A0 = nullptr;
        int rows_u = 0, ldu = 0, ldc = 0, lda = 0;
        int harm = -1;            // index of the member's harmonic record, or -1
    };
    std::vector<SpongeStep> sponges;
    std::map<int, cudaGraphExec_t> graphs;
};

void drop_graphs(std::map<int, cudaGraphExec_t> &cache) {
    for (auto &kv : cache) cudaGraphExecDestroy(kv.second);
    cache.clear();
}

void plan_free(Plan &p) {
    drop_graphs(p.graphs);
    for (int d = 0; d < 2; ++d) {
        for (int q = 0; q < 2; ++q) { dev_free(p.v1d[q][d]); dev_free(p.cd[q][d]); dev_free(p.fd[q][d]); }
        for (int m = 0; m < 2; ++m) dev_free(p.groups[d][m]);
        for (int v = 0; v < kFacVariants; ++v) {
            dev_free(p.fgroups[d][v]);
            p.nfgroups[d][v] = 0;
            p.fstage[d][v] = 0;
            p.fstages[d][v] = 0;
            p.fgrid[d][v] = 0;
            p.fring[d][v] = 0;
        }
        p.v1n[d] = 0;
        p.ngroups[d][0] = p.ngroups[d][1] = 0;
        p.smem[d][0] = p.smem[d][1] = 0;
    }
    for (int d = 0; d < 2; ++d) {
        dev_free(p.tdesc[d]);
        p.tcount[d] = p.trows[d] = p.tcols[d] = 0;
        dev_free(p.ndesc[d]);
    }
    p.ncount = p.nrows = p.ncols = 0;
    dev_free(p.scratch);
    dev_free(p.fault);
    dev_free(p.hdesc);
    p.hcount = 0;
    p.hmax = 0;
    p.sponges.clear();
}

// ADI_ETIMEOUT if a launch of the plan gave up waiting for its staged inputs.
int plan_fault(const Plan &p, cudaStream_t stream) {
    if (!p.fault.p) return ADI_OK;
    int f = 0;
    cudaError_t e = cudaMemcpyAsync(&f, p.fault.p, sizeof(int), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_status(e);
    return f ? ADI_ETIMEOUT : ADI_OK;
}

}  // namespace

struct adi_sim {
    Geometry g;
    int precision = ADI_FP32;
    double h = 0, dt = 0;
    size_t esz = 4;
    DevBuf A[4], V[2], W[2], alpha, alphaT, Uo, Wo, tab, sep, cold_all, clock, status;
    // host <-> device staging of the natural fields (FP64) and the prologue's scratch with the
    // Thomas factors after it: allocated by the first adi_set_fields / adi_read_fields /
    // adi_set_source after creation and kept until adi_destroy (adi_create frees its own)
    DevBuf xfer, pro;
    int parity = 0;                           // which V/W copy is current
    int plan_base = 0;                        // parity at which the own plan was built
    std::vector<unsigned char> h_desc[2][2];  // host descriptors [parity][0 = x-lines, 1 = y-lines]
    int nlines[2] = {0, 0};
    int solver = ADI_SOLVER_CHUNKED;
    int fac_reach = 0;                        // largest scan reach of the factored records
    // factored solver's launch parameters (0 = automatic): at most fac_nl_cap lines per CTA,
    // fac_ring_cap staged groups in flight (1: no prefetch); chosen by adi_autotune
    int fac_nl_cap = 0, fac_ring_cap = 0;
    Plan plan;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    long long steps = 0;
    int sticky = ADI_OK;
    bool in_batch = false;
    cudaStream_t batch_stream = nullptr;
    bool src_on = false;
    int src_i = 0, src_j = 0;
    double src_amp = 0, src_f0 = 0, src_td = 0;
    // time-harmonic walls and forcing (adi_set_harmonic): wall amplitudes (FP64), F in both
    // carried layouts (absent without forcing), and this simulation's own record on the device
    bool harm_on = false;
    double h_omega = 0, h_phb = 0, h_phf = 0;
    DevBuf h_edges, h_frow, h_fcol, h_self;
    // absorbing layers (adi_set_sponge): width in cells and strength; the y-line descriptors
    // of both parities and the prologue's scratch (with the CFD Thomas factors) kept on the
    // device for the per-step rebuild of the carried state
    bool sp_on = false;
    double sp_width = 0, sp_a = 0;
    DevBuf sp_desc[2], sp_scr;
};

struct adi_batch_t {
    std::vector<adi_sim *> sims;
    bool timing = false;
    std::vector<cudaEvent_t> ev[2];  // per stage: begin/end pairs of recorded solves
    size_t ev_used[2] = {0, 0};      // events of the pool in use
    std::vector<int> base_parity;  // members' parity when the batch was built
    int parity = 0;                // batch steps taken, mod 2
    int precision = ADI_FP32;
    Plan plan;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int sticky = ADI_OK;
};

namespace {

// The conversions below give each thread one column and a stride of gridDim.y rows (at most 128
// block rows, so a thread converts many rows, with its loads in flight together); both sides
// are coalesced and no thread divides a flat index.
inline dim3 conv_grid(size_t rows, size_t cols) {
    return dim3((unsigned)((cols + 255) / 256), (unsigned)(rows < 128 ? (rows > 0 ? rows : 1) : 128));
}
// Compact row-major double (rows x cols) -> rows with leading dimension ld in T.
template <typename T>
__global__ void convert_from_double(const double *src, T *dst, size_t rows, size_t cols, size_t ld,
                                    double scale, int square) {
    const size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (c >= cols) return;
#pragma unroll 4
    for (size_t r = blockIdx.y; r < rows; r += gridDim.y) {
        const double x = src[r * cols + c];
        dst[r * ld + c] = (T)(square ? scale * x * x : scale * x);
    }
}
// Rows with leading dimension ld in T -> compact row-major double.
template <typename T>
__global__ void convert_to_double(const T *src, double *dst, size_t rows, size_t cols, size_t ld) {
    const size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (c >= cols) return;
#pragma unroll 4
    for (size_t r = blockIdx.y; r < rows; r += gridDim.y) dst[r * cols + c] = (double)src[r * ld + c];
}
// Compact row-major S (rows x cols) -> rows with leading dimension ld in T.
template <typename S, typename T>
__global__ void convert_in(const S *src, T *dst, size_t rows, size_t cols, size_t ld) {
    const size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (c >= cols) return;
#pragma unroll 4
    for (size_t r = blockIdx.y; r < rows; r += gridDim.y) dst[r * ld + c] = (T)src[r * cols + c];
}
// Rows with leading dimension ld in T -> compact row-major D.
template <typename T, typename D>
__global__ void convert_out(const T *src, D *dst, size_t rows, size_t cols, size_t ld) {
    const size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (c >= cols) return;
#pragma unroll 4
    for (size_t r = blockIdx.y; r < rows; r += gridDim.y) dst[r * cols + c] = (D)src[r * ld + c];
}

// The natural fields after a step, from the carried state of its stage 2: a y-line solve leaves
// a = 2u - C (+ the point source's dt/2 f) and w*' = 2w - w*, and keeps its inputs C and w*, so
// u = (a + C)/2 and w = (w*' + w*)/2 on every point the y-lines solve (CFD: u on nodes 1..N-1,
// MFD: cells 1..N; w on 0..N; columns 1..pix).  One record per member and plan parity.
struct NatDesc {
    const void *a, *c;        // A[3] (a) and A[1] (C), column-major: column j at j * ldc
    const void *wn, *wi;      // w*' (the stage's output) and w* (its input), column j at j * ldwc
    void *uo, *wo;            // natural u (row-major, ldu) and w (row-major, ldw)
    const long long *clock;   // the member's step clock (for the point source)
    int ldc, ldwc, ldu, ldw;
    int j1;                   // columns 1 .. j1 - 1
    int ku0, ku1, kw1;        // u rows [ku0, ku1), w rows [0, kw1)
    int src_i, src_j;         // the point source's row and column, or -1
    int clock_ahead;          // 1: the clock has not yet advanced past this step (harmonic walls)
    double dt, src_amp, src_f0, src_td, src_scale;
};

// blockIdx.z: the member; a 32 x 32 tile of (row k, column j) per block.  The carried arrays are
// read along their columns (lane = row) and the natural ones written along their rows (lane =
// column), through shared memory, so both sides are coalesced.
template <typename T>
__global__ void naturalize_kernel(const NatDesc *__restrict__ nd) {
    __shared__ T tu[32][33], tw[32][33];
    const NatDesc d = nd[blockIdx.z];
    const int k0 = blockIdx.y * 32, jb = blockIdx.x * 32;
    if (k0 >= max(d.ku1, d.kw1) || jb >= d.j1) return;  // uniform over the block
    const int tx = threadIdx.x, ty = threadIdx.y;
    const T *a = (const T *)d.a, *c = (const T *)d.c, *wn = (const T *)d.wn, *wi = (const T *)d.wi;
    T src = T(0);
    if (d.src_j >= 0)
        src = (T)(d.src_scale *
                  ricker(d.src_amp, d.src_f0, d.src_td, (double)(*d.clock + d.clock_ahead) * d.dt));
    for (int jj = ty; jj < 32; jj += 8) {
        const int j = jb + jj, k = k0 + tx;
        if (j < 1 || j >= d.j1) continue;
        if (k >= d.ku0 && k < d.ku1) {
            const long long o = (long long)j * d.ldc + k;
            T u = T(0.5) * (a[o] + c[o]);
            if (k == d.src_i && j == d.src_j) u -= T(0.5) * src;
            tu[jj][tx] = u;
        }
        if (k < d.kw1) {
            const long long o = (long long)j * d.ldwc + k;
            tw[jj][tx] = T(0.5) * (wn[o] + wi[o]);
        }
    }
    __syncthreads();
    T *uo = (T *)d.uo, *wo = (T *)d.wo;
    for (int kk = ty; kk < 32; kk += 8) {
        const int k = k0 + kk, j = jb + tx;
        if (j < 1 || j >= d.j1) continue;
        if (k >= d.ku0 && k < d.ku1) uo[(long long)k * d.ldu + j] = tu[tx][kk];
        if (k < d.kw1) wo[(long long)k * d.ldw + j] = tw[tx][kk];
    }
}

// dst[j * ld_dst + i] = src[i * ld_src + j] for a rows x cols array (32 x 32 tiles).
template <typename T>
__global__ void transpose_kernel(const T *__restrict__ src, int rows, int cols, int ld_src,
                                 T *__restrict__ dst, int ld_dst) {
    __shared__ T tile[32][33];
    const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        int i = i0 + r, j = j0 + threadIdx.x;
        if (i < rows && j < cols) tile[r][threadIdx.x] = src[(size_t)i * ld_src + j];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        int j = j0 + r, i = i0 + threadIdx.x;
        if (i < rows && j < cols) dst[(size_t)j * ld_dst + i] = tile[threadIdx.x][r];
    }
}

// One array of a batched transpose: dst[c * ld_dst + r] = src[r * ld_src + c] for r < rows,
// c < cols.
struct TDesc {
    const void *src;
    void *dst;
    int rows, cols, ld_src, ld_dst;
};

// Batched tiled transpose (32 x 32 tiles through shared memory); blockIdx.z picks the array.
template <typename T>
__global__ void transpose_batch_kernel(const TDesc *__restrict__ td) {
    __shared__ T tile[32][33];
    const TDesc d = td[blockIdx.z];
    const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
    if (i0 >= d.rows || j0 >= d.cols) return;  // uniform over the block
    const T *__restrict__ src = (const T *)d.src;
    T *__restrict__ dst = (T *)d.dst;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int i = i0 + r, j = j0 + threadIdx.x;
        if (i < d.rows && j < d.cols) tile[r][threadIdx.x] = src[(size_t)i * d.ld_src + j];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int j = j0 + r, i = i0 + threadIdx.x;
        if (i < d.rows && j < d.cols) dst[(size_t)j * d.ld_dst + i] = tile[threadIdx.x][r];
    }
}

// FP32 batched transpose with 64 x 64 tiles and 16-byte global accesses (16 x 16 threads, four
// float4 rows each).  Leading dimensions are multiples of 32 elements and bases 16-byte
// aligned, so every 4-element group that starts inside a row's leading dimension is a
// valid aligned access; rows past `rows` load as zeros, which only ever land in the
// destination's padding, and destination rows past `cols` are not written.
__global__ void __launch_bounds__(256) transpose_batch64_kernel(const TDesc *__restrict__ td) {
    __shared__ float tile[64][65];
    const TDesc d = td[blockIdx.z];
    const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
    if (i0 >= d.rows || j0 >= d.cols) return;  // uniform over the block
    const float *__restrict__ src = (const float *)d.src;
    float *__restrict__ dst = (float *)d.dst;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int j = j0 + 4 * tx;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int r = ty + 16 * k, i = i0 + r;
        float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < d.rows && j < d.ld_src) q = *reinterpret_cast<const float4 *>(src + (size_t)i * d.ld_src + j);
        tile[r][4 * tx] = q.x; tile[r][4 * tx + 1] = q.y; tile[r][4 * tx + 2] = q.z; tile[r][4 * tx + 3] = q.w;
    }
    __syncthreads();
    const int i = i0 + 4 * tx;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int cc = ty + 16 * k, jj = j0 + cc;
        if (jj < d.cols && i < d.ld_dst) {
            const float4 q = make_float4(tile[4 * tx][cc], tile[4 * tx + 1][cc], tile[4 * tx + 2][cc], tile[4 * tx + 3][cc]);
            *reinterpret_cast<float4 *>(dst + (size_t)jj * d.ld_dst + i) = q;
        }
    }
}

int transpose(adi_sim *s, const void *src, int rows, int cols, int ld_src, void *dst, int ld_dst) {
    dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32)), block(32, 8);
    if (s->precision == ADI_FP64)
        transpose_kernel<double><<<grid, block, 0, s->stream>>>((const double *)src, rows, cols, ld_src,
                                                                 (double *)dst, ld_dst);
    else
        transpose_kernel<float><<<grid, block, 0, s->stream>>>((const float *)src, rows, cols, ld_src,
                                                                (float *)dst, ld_dst);
    return cuda_status(cudaGetLastError());
}

// Uploads a host double array into a device array of the sim's precision; scale*x or
// scale*x^2 (used for alpha = dt/2 c^2).  staging must hold n doubles.
// (host rows x cols, compact; NULL uploads zeros) -> dst rows with leading dimension ld.
int upload(adi_sim *s, const double *host, void *dst, size_t rows, size_t cols, size_t ld,
           double *staging, double scale, int square) {
    const size_t n = rows * cols;
    if (n == 0) return ADI_OK;
    cudaError_t e;
    if (host)
        e = cudaMemcpyAsync(staging, host, n * sizeof(double), cudaMemcpyHostToDevice, s->stream);
    else
        e = cudaMemsetAsync(staging, 0, n * sizeof(double), s->stream);
    if (e != cudaSuccess) return cuda_status(e);
    const dim3 grid = conv_grid(rows, cols);
    if (s->precision == ADI_FP64)
        convert_from_double<double><<<grid, 256, 0, s->stream>>>(staging, (double *)dst, rows, cols, ld, scale, square);
    else
        convert_from_double<float><<<grid, 256, 0, s->stream>>>(staging, (float *)dst, rows, cols, ld, scale, square);
    return cuda_status(cudaGetLastError());
}

// Builds the line descriptors of a simulation ([0] x-lines, [1] y-lines).
template <typename T>
void fill_descs(adi_sim *s, int par, std::vector<LineDesc<T>> &rows, std::vector<LineDesc<T>> &cols) {
    const Geometry &g = s->g;
    T *A0 = (T *)s->A[0].p, *A1 = (T *)s->A[1].p, *A2 = (T *)s->A[2].p, *A3 = (T *)s->A[3].p;
    T *Uo = (T *)s->Uo.p, *Wo = (T *)s->Wo.p;
    T *Vi = (T *)s->V[par].p, *Vn = (T *)s->V[1 - par].p;
    T *Wi = (T *)s->W[par].p, *Wn = (T *)s->W[1 - par].p;
    const T *al = (const T *)s->alpha.p, *alT = (const T *)s->alphaT.p;
    const T *tab = (const T *)s->tab.p;
    T *sep = (T *)s->sep.p;
    const int bs = block_size(g.method);
    const int Mx = chunk_M(g.method);
    const int Tx = chunks_for(g.method, g.nx), Ty = chunks_for(g.method, g.ny);
    const bool fac = s->solver == ADI_SOLVER_FACTORED;
    const size_t rec_x = fac ? fac_words(g.method, g.nx) : (size_t)(Tx - 1) * 3 * bs * bs;
    const size_t rec_y = fac ? fac_words(g.method, g.ny) : (size_t)(Ty - 1) * 3 * bs * bs;
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
    base.chunkM = Mx;
    rows.assign(g.piy, base);
    cols.assign(g.pix, base);
    size_t sep_off = 0;
    for (int r = 0; r < g.piy; ++r) {
        int i = r + 1;  // grid row of this x-line
        LineDesc<T> &d = rows[r];
        d.p = A0 + (size_t)i * g.lda;
        d.po = A2 + (size_t)i * g.lda;  // C row-major; transposed into A1 after the stage
        d.alpha = al + (size_t)i * g.lda;
        d.v = Vi + (size_t)i * g.ldvp;
        d.vo = Vn + (size_t)i * g.ldvp;
        d.u_out = nullptr; d.w_out = nullptr;
        d.sp = 1; d.sv = 1; d.spo = 1; d.svo = 1; d.snp = 1; d.snv = 1;
        d.N = g.nx;
        d.tab = tab + (size_t)r * kTabLine;
        d.sep = sep ? sep + sep_off : nullptr;
        sep_off += rec_x;
        if (s->src_on && s->src_i == i) d.src_k = s->src_j;
        d.advance_clock = 0;
    }
    for (int c = 0; c < g.pix; ++c) {
        int j = c + 1;  // grid column of this y-line
        LineDesc<T> &d = cols[c];
        d.p = A1 + (size_t)j * g.ldc;
        d.po = A3 + (size_t)j * g.ldc;  // a column-major; transposed into A0 after the stage
        d.alpha = alT + (size_t)j * g.ldc;
        d.v = Wi + (size_t)j * g.ldwc;
        d.vo = Wn + (size_t)j * g.ldwc;
        d.u_out = Uo + j;
        d.w_out = Wo + j;
        d.sp = 1; d.sv = 1; d.spo = 1; d.svo = 1; d.snp = g.ldu; d.snv = g.ldw;
        d.N = g.ny;
        d.tab = tab + (size_t)(g.piy + c) * kTabLine;
        d.sep = sep ? sep + sep_off : nullptr;
        sep_off += rec_y;
        // with harmonic data the clock advances after the stage's harmonic launch instead
        if (s->src_on && s->src_j == j) { d.src_k = s->src_i; d.advance_clock = s->harm_on ? 0 : 1; }
    }
}

template <typename T>
void build_host_descs(adi_sim *s) {
    for (int par = 0; par < 2; ++par) {
        std::vector<LineDesc<T>> rows, cols;
        fill_descs<T>(s, par, rows, cols);
        s->h_desc[par][0].assign((unsigned char *)rows.data(), (unsigned char *)(rows.data() + rows.size()));
        s->h_desc[par][1].assign((unsigned char *)cols.data(), (unsigned char *)(cols.data() + cols.size()));
    }
}

// The harmonic record of a simulation with time-harmonic walls (and forcing).
HarmDesc harm_desc_of(const adi_sim *s) {
    const Geometry &g = s->g;
    HarmDesc d;
    d.a_row = s->A[0].p;
    d.c_col = s->A[1].p;
    d.uo = s->Uo.p;
    d.f_row = s->h_frow.p;
    d.f_col = s->h_fcol.p;
    d.edges = (const double *)s->h_edges.p;
    d.clock = (long long *)s->clock.p;
    d.rows_u = g.rows_u; d.ldu = g.ldu; d.lda = g.lda; d.ldc = g.ldc;
    d.dt = s->dt; d.omega = s->h_omega; d.phb = s->h_phb; d.phf = s->h_phf;
    return d;
}

// Builds an execution plan for members (all of one precision).  Plan parity q uses each
// member's descriptors of parity (member's current parity) ^ q.
int plan_build(Plan &p, const std::vector<adi_sim *> &members, cudaStream_t stream) {
    plan_free(p);
    if (members.empty()) return ADI_EINVAL;
    const int prec = members[0]->precision;
    p.precision = prec;
    const size_t dsz = desc_size(prec), esz = elem_size(prec);
    std::vector<unsigned char> v1[2][2], cd[2][2], fdv[2][2];
    std::vector<int4> gr[2][2];
    std::vector<FacGroup> fgr[2][kFacVariants];
    size_t words = 0;
    for (adi_sim *s : members) {
        for (int dir = 0; dir < 2; ++dir) {
            if (s->solver == ADI_SOLVER_LINE) {
                for (int q = 0; q < 2; ++q) {
                    const std::vector<unsigned char> &h = s->h_desc[s->parity ^ q][dir];
                    v1[q][dir].insert(v1[q][dir].end(), h.begin(), h.end());
                }
            } else if (s->solver == ADI_SOLVER_FACTORED) {
                int first = (int)(fdv[0][dir].size() / dsz);
                int n = s->nlines[dir];
                int N = dir == 0 ? s->g.nx : s->g.ny;
                int v = fac_variant(s->g.method, N);
                if (fac_split_line(s->g.method, N)) {
                    // lines longer than a CTA's chunks: sub-lines with a halo of the scan reach
                    FacGroup sub[kFacMaxSplit];
                    for (int st = 0; st < n; ++st) {
                        size_t sb = 0;
                        const int k = fac_split_groups(s->g.method, N, first + st, std::max(1, s->fac_reach),
                                                       1.0 / s->h, 0.5 * s->dt, esz, sub, &sb);
                        if (k == 0) return ADI_ENOTSUP;
                        fgr[dir][v].insert(fgr[dir][v].end(), sub, sub + k);
                        p.fstage[dir][v] = std::max(p.fstage[dir][v], sb);
                    }
                } else {
                    int nl = fac_lines_per_cta(s->g.method, N, esz);
                    if (s->fac_nl_cap > 0) nl = std::min(nl, s->fac_nl_cap);
                    for (int st = 0; st < n; st += nl) {
                        int cnt = std::min(nl, n - st);
                        FacGroup fg = fac_group_of(s->g.method, N, first + st, cnt, 1.0 / s->h, 0.5 * s->dt);
                        // the scans this simulation's lines need, whatever else shares the launch
                        if (s->fac_reach > kFacMaxReach) fg.own |= kFacOwnFull;
                        fgr[dir][v].push_back(fg);
                        p.fstage[dir][v] = std::max(p.fstage[dir][v], fac_stage_bytes(s->g.method, N, cnt, esz));
                    }
                }
                if (s->fac_ring_cap > 0)
                    p.fring[dir][v] = p.fring[dir][v] > 0 ? std::min(p.fring[dir][v], s->fac_ring_cap) : s->fac_ring_cap;
                for (int q = 0; q < 2; ++q) {
                    const std::vector<unsigned char> &h = s->h_desc[s->parity ^ q][dir];
                    fdv[q][dir].insert(fdv[q][dir].end(), h.begin(), h.end());
                }
            } else {
                int first = (int)(cd[0][dir].size() / dsz);
                int n = s->nlines[dir];
                int N = dir == 0 ? s->g.nx : s->g.ny;
                int T = chunks_for(s->g.method, N);
                int bs = block_size(s->g.method);
                // lines per CTA: at most kChunkThreads threads, at least ~128 threads, and
                // enough CTAs to give every SM two of them
                int nl_max = std::max(1, kChunkThreads / T);
                int nl_min = std::min(nl_max, (128 + T - 1) / T);
                int nl = std::max(nl_min, std::min(nl_max, (n + 2 * 152 - 1) / (2 * 152)));
                while (nl > 1 && chunked_smem_bytes(N, nl, T, bs, esz) > (size_t)kChunkSmemMax) --nl;
                for (int st = 0; st < n; st += nl) {
                    int cnt = std::min(nl, n - st);
                    gr[dir][s->g.method].push_back(make_int4(first + st, cnt, s->g.method, 0));
                    size_t sm = chunked_smem_bytes(N, cnt, T, bs, esz);
                    p.smem[dir][s->g.method] = std::max(p.smem[dir][s->g.method], sm);
                }
                for (int q = 0; q < 2; ++q) {
                    const std::vector<unsigned char> &h = s->h_desc[s->parity ^ q][dir];
                    cd[q][dir].insert(cd[q][dir].end(), h.begin(), h.end());
                }
            }
        }
        if (s->solver == ADI_SOLVER_LINE) words = std::max(words, v1_words(s->g));
    }
    int rc = ADI_OK;
    for (int dir = 0; dir < 2 && !rc; ++dir) {
        p.v1n[dir] = (int)(v1[0][dir].size() / dsz);
        for (int q = 0; q < 2 && !rc; ++q) {
            if (!v1[q][dir].empty()) {
                rc = dev_alloc(p.v1d[q][dir], v1[q][dir].size());
                if (!rc) rc = cuda_status(cudaMemcpyAsync(p.v1d[q][dir].p, v1[q][dir].data(), v1[q][dir].size(), cudaMemcpyHostToDevice, stream));
            }
            if (!rc && !cd[q][dir].empty()) {
                rc = dev_alloc(p.cd[q][dir], cd[q][dir].size());
                if (!rc) rc = cuda_status(cudaMemcpyAsync(p.cd[q][dir].p, cd[q][dir].data(), cd[q][dir].size(), cudaMemcpyHostToDevice, stream));
            }
            if (!rc && !fdv[q][dir].empty()) {
                rc = dev_alloc(p.fd[q][dir], fdv[q][dir].size());
                if (!rc) rc = cuda_status(cudaMemcpyAsync(p.fd[q][dir].p, fdv[q][dir].data(), fdv[q][dir].size(), cudaMemcpyHostToDevice, stream));
            }
        }
        for (int v = 0; v < kFacVariants && !rc; ++v) {
            p.nfgroups[dir][v] = (int)fgr[dir][v].size();
            p.fstages[dir][v] = fac_stages_for(p.fstage[dir][v], esz, (v == 0 || v == 3) ? ADI_CFD : ADI_MFD);
            if (p.fring[dir][v] > 0) p.fstages[dir][v] = std::min(p.fstages[dir][v], p.fring[dir][v]);
            p.fgrid[dir][v] = std::min(p.nfgroups[dir][v], sm_count());
            if (p.nfgroups[dir][v] && !p.fstages[dir][v]) { rc = ADI_ENOTSUP; break; }
            if (!fgr[dir][v].empty()) {
                rc = dev_alloc(p.fgroups[dir][v], fgr[dir][v].size() * sizeof(FacGroup));
                if (!rc) rc = cuda_status(cudaMemcpyAsync(p.fgroups[dir][v].p, fgr[dir][v].data(), fgr[dir][v].size() * sizeof(FacGroup), cudaMemcpyHostToDevice, stream));
            }
        }
        for (int m = 0; m < 2 && !rc; ++m) {
            p.ngroups[dir][m] = (int)gr[dir][m].size();
            if (!gr[dir][m].empty()) {
                rc = dev_alloc(p.groups[dir][m], gr[dir][m].size() * sizeof(int4));
                if (!rc) rc = cuda_status(cudaMemcpyAsync(p.groups[dir][m].p, gr[dir][m].data(), gr[dir][m].size() * sizeof(int4), cudaMemcpyHostToDevice, stream));
            }
        }
    }
    // the transposes of the carried pressure after each stage
    for (int dir = 0; dir < 2 && !rc; ++dir) {
        std::vector<TDesc> td;
        for (adi_sim *s : members) {
            const Geometry &g = s->g;
            TDesc t;
            if (dir == 0) {  // C row-major (A[2]) -> column-major (A[1])
                t.src = s->A[2].p; t.dst = s->A[1].p;
                t.rows = g.rows_u; t.cols = g.ldu; t.ld_src = g.lda; t.ld_dst = g.ldc;
            } else {         // a column-major (A[3]) -> row-major (A[0])
                t.src = s->A[3].p; t.dst = s->A[0].p;
                t.rows = g.ldu; t.cols = g.rows_u; t.ld_src = g.ldc; t.ld_dst = g.lda;
            }
            p.trows[dir] = std::max(p.trows[dir], t.rows);
            p.tcols[dir] = std::max(p.tcols[dir], t.cols);
            td.push_back(t);
        }
        p.tcount[dir] = (int)td.size();
        rc = dev_alloc(p.tdesc[dir], td.size() * sizeof(TDesc));
        if (!rc) rc = cuda_status(cudaMemcpyAsync(p.tdesc[dir].p, td.data(), td.size() * sizeof(TDesc),
                                                  cudaMemcpyHostToDevice, stream));
    }
    // the natural fields' records (member parity s->parity ^ q at plan parity q)
    for (int q = 0; q < 2 && !rc; ++q) {
        std::vector<NatDesc> nd;
        for (adi_sim *s : members) {
            const Geometry &g = s->g;
            const int pm = s->parity ^ q;
            NatDesc d;
            std::memset(&d, 0, sizeof(d));
            d.a = s->A[3].p; d.c = s->A[1].p;
            d.wn = s->W[1 - pm].p; d.wi = s->W[pm].p;
            d.uo = s->Uo.p; d.wo = s->Wo.p;
            d.clock = (const long long *)s->clock.p;
            d.ldc = g.ldc; d.ldwc = g.ldwc; d.ldu = g.ldu; d.ldw = g.ldw;
            d.j1 = 1 + g.pix;
            d.ku0 = 1;
            d.ku1 = g.method == ADI_CFD ? g.ny : g.ny + 1;
            d.kw1 = g.ny + 1;
            d.src_i = s->src_on ? s->src_i : -1;
            d.src_j = s->src_on ? s->src_j : -1;
            d.clock_ahead = s->harm_on ? 1 : 0;
            d.dt = s->dt; d.src_amp = s->src_amp; d.src_f0 = s->src_f0; d.src_td = s->src_td;
            d.src_scale = s->dt / (2.0 * s->h * s->h);
            p.nrows = std::max(p.nrows, std::max(d.ku1, d.kw1));
            p.ncols = std::max(p.ncols, d.j1);
            nd.push_back(d);
        }
        p.ncount = (int)nd.size();
        rc = dev_alloc(p.ndesc[q], nd.size() * sizeof(NatDesc));
        if (!rc) rc = cuda_status(cudaMemcpyAsync(p.ndesc[q].p, nd.data(), nd.size() * sizeof(NatDesc),
                                                  cudaMemcpyHostToDevice, stream));
    }
    // the harmonic records of the members with time-harmonic walls
    if (!rc) {
        std::vector<HarmDesc> hd;
        for (adi_sim *s : members)
            if (s->harm_on) {
                hd.push_back(harm_desc_of(s));
                p.hmax = std::max(p.hmax, s->g.nU());
            }
        p.hcount = (int)hd.size();
        if (!hd.empty()) {
            rc = dev_alloc(p.hdesc, hd.size() * sizeof(HarmDesc));
            if (!rc) rc = cuda_status(cudaMemcpyAsync(p.hdesc.p, hd.data(), hd.size() * sizeof(HarmDesc),
                                                      cudaMemcpyHostToDevice, stream));
        }
    }
    // the absorbing layers' per-step work, with each such member's own descriptor copies
    int hidx = 0;
    for (adi_sim *s : members) {
        const int my_h = s->harm_on ? hidx++ : -1;
        if (!s->sp_on || rc) continue;
        const Geometry &g = s->g;
        for (int par = 0; par < 2 && !rc; ++par)
            rc = cuda_status(cudaMemcpyAsync(s->sp_desc[par].p, s->h_desc[par][1].data(), s->h_desc[par][1].size(),
                                             cudaMemcpyHostToDevice, stream));
        Plan::SpongeStep sp;
        for (int q = 0; q < 2; ++q) {
            const int pm = s->parity ^ q;  // the member's parity at plan parity q
            SpongeRec &r = sp.rec[q];
            r.uo = s->Uo.p; r.v = s->V[1 - pm].p; r.wo = s->Wo.p; r.v_other = s->V[pm].p;
            r.method = g.method; r.nx = g.nx; r.ny = g.ny;
            r.rows_u = g.rows_u; r.ldu = g.ldu; r.rows_v = g.rows_v; r.ldv = g.ldv; r.ldvp = g.ldvp;
            r.rows_w = g.rows_w; r.ldw = g.ldw;
            r.width = s->sp_width; r.a = s->sp_a;
            sp.ydesc[q] = s->sp_desc[1 - pm].p;
        }
        sp.nlines = s->nlines[1]; sp.N = g.ny; sp.method = g.method;
        sp.st = std::max(1, s->nlines[1]);
        sp.scr = s->sp_scr.p;
        sp.fac = g.method == ADI_CFD ? (const void *)((unsigned char *)s->sp_scr.p + (size_t)(2 * g.ny + 2) * sp.st * s->esz) : nullptr;
        sp.A3 = s->A[3].p; sp.A0 = s->A[0].p;
        sp.rows_u = g.rows_u; sp.ldu = g.ldu; sp.ldc = g.ldc; sp.lda = g.lda;
        sp.harm = my_h;
        p.sponges.push_back(sp);
    }
    if (!rc) rc = dev_alloc(p.fault, sizeof(int));
    if (!rc) rc = cuda_status(cudaMemsetAsync(p.fault.p, 0, sizeof(int), stream));
    if (!rc && (p.v1n[0] || p.v1n[1])) {
        p.scratch_stride = std::max(p.v1n[0], p.v1n[1]);
        rc = dev_alloc(p.scratch, words * (size_t)p.scratch_stride * esz);
    }
    if (!rc) rc = cuda_status(cudaStreamSynchronize(stream));
    if (rc) plan_free(p);
    return rc;
}

// One stage (dir 0: stage 1 over x-lines, dir 1: stage 2 over y-lines) of a plan at plan
// parity q.
template <typename T>
cudaError_t enqueue_stage(const Plan &p, int q, int dir, int natural, cudaStream_t stream, cudaEvent_t ev0,
                          cudaEvent_t ev1) {
    cudaError_t e = ev0 ? cudaEventRecord(ev0, stream) : cudaSuccess;
    // members with absorbing layers need their natural fields after every step; the line solves
    // leave them to naturalize_kernel below (writing them from the line kernels would put one
    // scattered element per lane into the row-major natural arrays)
    const int nat = dir == 1 ? (natural || !p.sponges.empty() ? 1 : 0) : 0;
    if (e == cudaSuccess && p.v1n[dir])
        e = launch_line_solve_v1<T>((const LineDesc<T> *)p.v1d[q][dir].p, p.v1n[dir], (T *)p.scratch.p,
                                    p.scratch_stride, 0, stream);
    for (int v = 0; v < kFacVariants && e == cudaSuccess; ++v)
        if (p.nfgroups[dir][v])
            e = launch_line_solve_factored<T>((const LineDesc<T> *)p.fd[q][dir].p,
                                              (const FacGroup *)p.fgroups[dir][v].p, p.nfgroups[dir][v], v,
                                              p.fstage[dir][v], p.fstages[dir][v], p.fgrid[dir][v], 0,
                                              (int *)p.fault.p, stream);
    for (int m = 0; m < 2 && e == cudaSuccess; ++m)
        if (p.ngroups[dir][m])
            e = launch_line_solve_chunked<T>((const LineDesc<T> *)p.cd[q][dir].p,
                                             (const int4 *)p.groups[dir][m].p, p.ngroups[dir][m], m,
                                             p.smem[dir][m], 0, stream);
    if (e == cudaSuccess && ev1) e = cudaEventRecord(ev1, stream);
    // natural u and w from the carried state, before anything moves or changes it
    if (e == cudaSuccess && nat && p.ncount) {
        dim3 grid((unsigned)((p.ncols + 31) / 32), (unsigned)((p.nrows + 31) / 32), (unsigned)p.ncount);
        naturalize_kernel<T><<<grid, dim3(32, 8), 0, stream>>>((const NatDesc *)p.ndesc[q].p);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && p.tcount[dir]) {
        if (sizeof(T) == 4) {
            dim3 grid((unsigned)((p.tcols[dir] + 63) / 64), (unsigned)((p.trows[dir] + 63) / 64), (unsigned)p.tcount[dir]);
            transpose_batch64_kernel<<<grid, dim3(16, 16), 0, stream>>>((const TDesc *)p.tdesc[dir].p);
        } else {
            dim3 grid((unsigned)((p.tcols[dir] + 31) / 32), (unsigned)((p.trows[dir] + 31) / 32), (unsigned)p.tcount[dir]);
            transpose_batch_kernel<T><<<grid, dim3(32, 8), 0, stream>>>((const TDesc *)p.tdesc[dir].p);
        }
        e = cudaGetLastError();
    }
    // time-harmonic walls and forcing, in the layout the next stage reads
    if (e == cudaSuccess && p.hcount)
        e = launch_harmonic<T>((const HarmDesc *)p.hdesc.p, p.hcount, p.hmax, dir, stream);
    // absorbing layers: damp the natural fields, rebuild the carried state from them
    if (dir == 1)
        for (const Plan::SpongeStep &sp : p.sponges) {
            if (e != cudaSuccess) break;
            e = launch_sponge<T>(sp.rec[q], stream);
            if (e == cudaSuccess)
                e = launch_prologue_lines<T>((const LineDesc<T> *)sp.ydesc[q], sp.nlines, sp.N, sp.method,
                                             (const T *)sp.fac, (T *)sp.scr, sp.st, stream);
            if (e == cudaSuccess) {  // the prologue wrote a column-major (A[3]); a row-major copy
                dim3 grid((unsigned)((sp.rows_u + 31) / 32), (unsigned)((sp.ldu + 31) / 32)), block(32, 8);
                transpose_kernel<T><<<grid, block, 0, stream>>>((const T *)sp.A3, sp.ldu, sp.rows_u, sp.ldc,
                                                                (T *)sp.A0, sp.lda);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess && sp.harm >= 0)
                e = launch_harmonic<T>((const HarmDesc *)p.hdesc.p + sp.harm, 1, (size_t)sp.rows_u * sp.ldu, 3, stream);
        }
    return e;
}

cudaError_t enqueue_stage_any(const Plan &p, int q, int dir, int natural, cudaStream_t stream,
                              cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr) {
    return p.precision == ADI_FP64 ? enqueue_stage<double>(p, q, dir, natural, stream, ev0, ev1)
                                   : enqueue_stage<float>(p, q, dir, natural, stream, ev0, ev1);
}

// nsteps full steps starting at plan parity q0.
cudaError_t enqueue_steps(const Plan &p, int q0, int nsteps, cudaStream_t stream) {
    for (int k = 0; k < nsteps; ++k) {
        int q = (q0 + k) & 1;
        cudaError_t e = enqueue_stage_any(p, q, 0, 0, stream);
        if (e == cudaSuccess) e = enqueue_stage_any(p, q, 1, k == nsteps - 1 ? 1 : 0, stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Captures nsteps from parity q0 into a graph (cached per (steps, parity)) and launches it.
cudaError_t run_graph(Plan &p, int q0, int nsteps, cudaStream_t stream) {
    const int key = 2 * nsteps + q0;
    auto it = p.graphs.find(key);
    if (it == p.graphs.end()) {
        cudaStream_t cap;
        cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
        e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) { cudaStreamDestroy(cap); return e; }
        cudaError_t le = enqueue_steps(p, q0, nsteps, cap);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(cap, &graph);
        cudaStreamDestroy(cap);
        if (le != cudaSuccess) { if (graph) cudaGraphDestroy(graph); return le; }
        if (e != cudaSuccess) return e;
        cudaGraphExec_t exec;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return e;
        it = p.graphs.emplace(key, exec).first;
    }
    return cudaGraphLaunch(it->second, stream);
}

// Uploads the sim's descriptors of its current parity (x-lines then y-lines) for the
// prologue and the precomputes.
int upload_sim_descs(adi_sim *s) {
    const std::vector<unsigned char> &hx = s->h_desc[s->parity][0], &hy = s->h_desc[s->parity][1];
    size_t bytes = hx.size() + hy.size();
    if (s->cold_all.bytes < bytes) {
        dev_free(s->cold_all);
        int rc = dev_alloc(s->cold_all, bytes);
        if (rc) return rc;
    }
    cudaError_t e = cudaMemcpyAsync(s->cold_all.p, hx.data(), hx.size(), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync((unsigned char *)s->cold_all.p + hx.size(), hy.data(), hy.size(),
                            cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    return cuda_status(e);
}

template <typename T>
int run_prologue_t(adi_sim *s) {
    const LineDesc<T> *cols = (const LineDesc<T> *)((unsigned char *)s->cold_all.p + s->h_desc[s->parity][0].size());
    const long long st = std::max(1, s->nlines[1]);
    const int N = s->g.ny;
    const size_t scr = (size_t)(2 * N + 2) * st, nfac = s->g.method == ADI_CFD ? prologue_factor_count(N) : 0;
    const size_t bytes = (scr + nfac) * sizeof(T);
    cudaError_t e = cudaSuccess;
    if (s->pro.bytes != bytes) {  // first use: scratch plus the CFD Thomas factors of P, Pbar
        dev_free(s->pro);
        int rc = dev_alloc(s->pro, bytes);
        if (rc) return rc;
        if (nfac) {
            std::vector<double> f;
            prologue_factors(N, f);
            std::vector<T> ft(f.begin(), f.end());
            e = cudaMemcpyAsync((T *)s->pro.p + scr, ft.data(), ft.size() * sizeof(T), cudaMemcpyHostToDevice, s->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);  // ft leaves scope
        }
    }
    if (e == cudaSuccess)
        e = launch_prologue_lines<T>(cols, s->nlines[1], N, s->g.method, nfac ? (const T *)s->pro.p + scr : nullptr,
                                     (T *)s->pro.p, st, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_status(e);
    // the prologue wrote a column-major (A[3]), like a stage-2 launch
    const Geometry &g = s->g;
    int rc = transpose(s, s->A[3].p, g.ldu, g.rows_u, g.ldc, s->A[0].p, g.lda);
    if (!rc) rc = cuda_status(cudaStreamSynchronize(s->stream));
    return rc;
}

// One launch of the harmonic kernel for this simulation alone (mode 2 or 3).
int harm_self(adi_sim *s, int mode) {
    if (!s->harm_on) return ADI_OK;
    if (!s->h_self.p) {
        int rc = dev_alloc(s->h_self, sizeof(HarmDesc));
        if (rc) return rc;
    }
    const HarmDesc d = harm_desc_of(s);
    cudaError_t e = cudaMemcpyAsync(s->h_self.p, &d, sizeof(d), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess)
        e = s->precision == ADI_FP64 ? launch_harmonic<double>((const HarmDesc *)s->h_self.p, 1, s->g.nU(), mode, s->stream)
                                     : launch_harmonic<float>((const HarmDesc *)s->h_self.p, 1, s->g.nU(), mode, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);  // d leaves scope
    return cuda_status(e);
}

// Rebuilds the carried state from the natural fields; with time-harmonic data it then adds
// dt/2 f(t_now) and sets the x-line ends to the coming step's u*.
int prologue(adi_sim *s) {
    int rc = s->precision == ADI_FP64 ? run_prologue_t<double>(s) : run_prologue_t<float>(s);
    if (!rc) rc = harm_self(s, 3);
    return rc;
}

// The device step clock follows the host's step count (sources and harmonic data read it).
int sync_clock(adi_sim *s) {
    cudaError_t e = cudaMemcpyAsync(s->clock.p, &s->steps, sizeof(long long), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    return cuda_status(e);
}

template <typename T>
int run_precompute(adi_sim *s) {
    const LineDesc<T> *all = (const LineDesc<T> *)s->cold_all.p;
    int n = s->nlines[0] + s->nlines[1];
    cudaError_t e = cudaMemsetAsync(s->status.p, 0, sizeof(int), s->stream);
    if (e == cudaSuccess) e = launch_precompute<T>(all, n, (T *)s->tab.p, (int *)s->status.p, s->stream);
    int st = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&st, s->status.p, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_status(e);
    if (st) return ADI_ESINGULAR;
    if (s->solver == ADI_SOLVER_CHUNKED) {
        e = launch_precompute_sep<T>(all, n, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    } else if (s->solver == ADI_SOLVER_FACTORED) {
        // FP64 workspace of the dense end eliminations, one slice per line
        DevBuf ws;
        int rc = dev_alloc(ws, (size_t)n * fac_ws_doubles() * sizeof(double));
        if (rc) return rc;
        int out[2] = {0, 0};
        e = cudaMemsetAsync(s->status.p, 0, 2 * sizeof(int), s->stream);
        if (e == cudaSuccess) e = launch_fac_precompute<T>(all, n, (double *)ws.p, (int *)s->status.p, s->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(out, s->status.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        dev_free(ws);
        if (e == cudaSuccess && out[0]) return ADI_ESINGULAR;
        s->fac_reach = out[1];
    }
    return cuda_status(e);
}

// (Re)builds descriptors, separator factors and the plan for the sim's current solver.
int setup_solver(adi_sim *s) {
    dev_free(s->sep);
    int rc = ADI_OK;
    rc = dev_alloc(s->sep, solver_words(s->g, s->solver) * s->esz);
    if (rc) return rc;
    if (s->precision == ADI_FP64) build_host_descs<double>(s); else build_host_descs<float>(s);
    rc = upload_sim_descs(s);
    if (!rc) rc = s->precision == ADI_FP64 ? run_precompute<double>(s) : run_precompute<float>(s);
    if (!rc) rc = plan_build(s->plan, std::vector<adi_sim *>{s}, s->stream);
    s->plan_base = s->parity;
    // a split line whose scan reach exceeds the halo a sub-line can take: use the chunked solver
    if (rc == ADI_ENOTSUP && s->solver == ADI_SOLVER_FACTORED && chunked_ok(s->g, s->esz)) {
        s->solver = ADI_SOLVER_CHUNKED;
        return setup_solver(s);
    }
    return rc;
}

// The FP64 staging buffer of host <-> device field copies (one field), kept once allocated.
// Byte offsets of the three fields' slots in the staging buffer (U, V, W; FP64-sized).
void xfer_slots(const Geometry &g, size_t off[4]) {
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    off[0] = 0;
    off[1] = up(g.nU() * sizeof(double));
    off[2] = off[1] + up(g.nV() * sizeof(double));
    off[3] = off[2] + up(g.nW() * sizeof(double));
}
int xfer_buffer(adi_sim *s) {
    size_t off[4];
    xfer_slots(s->g, off);
    if (s->xfer.bytes >= off[3]) return ADI_OK;
    dev_free(s->xfer);
    return dev_alloc(s->xfer, off[3]);
}

// Copies host fields (FP64, or FP32 with f32) into their slots of the staging buffer and checks
// them there, before any of the simulation's state changes (ADI_EINVAL on NaN/Inf).  staged[k]
// receives the slot of field k, or nullptr for a field not given.
int stage_fields(adi_sim *s, const void *const f[3], bool f32, const void *staged[3]) {
    int rc = xfer_buffer(s);
    if (rc) return rc;
    const Geometry &g = s->g;
    size_t off[4];
    xfer_slots(g, off);
    const size_t n[3] = {g.nU(), g.nV(), g.nW()};
    const size_t hsz = f32 ? sizeof(float) : sizeof(double);
    cudaError_t e = cudaMemsetAsync(s->status.p, 0, sizeof(int), s->stream);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
        staged[k] = nullptr;
        if (!f[k]) continue;
        void *slot = (unsigned char *)s->xfer.p + off[k];
        e = cudaMemcpyAsync(slot, f[k], n[k] * hsz, cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess)
            e = f32 ? launch_finite_check<float>((const float *)slot, n[k], (int *)s->status.p, s->stream)
                    : launch_finite_check<double>((const double *)slot, n[k], (int *)s->status.p, s->stream);
        staged[k] = slot;
    }
    int flag = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, s->status.p, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_status(e);
    return flag ? ADI_EINVAL : ADI_OK;
}

// One staged field (compact rows x cols of FP64, or FP32 with f32) into a device array of the
// simulation's precision with leading dimension ld; nullptr: zeros.
int load_field(adi_sim *s, const void *staged, bool f32, void *dst, size_t rows, size_t cols, size_t ld) {
    if (!staged) return cuda_status(cudaMemsetAsync(dst, 0, rows * ld * s->esz, s->stream));
    const dim3 grid = conv_grid(rows, cols);
    if (s->precision == ADI_FP64) {
        if (f32) convert_in<float, double><<<grid, 256, 0, s->stream>>>((const float *)staged, (double *)dst, rows, cols, ld);
        else convert_in<double, double><<<grid, 256, 0, s->stream>>>((const double *)staged, (double *)dst, rows, cols, ld);
    } else {
        if (f32) convert_in<float, float><<<grid, 256, 0, s->stream>>>((const float *)staged, (float *)dst, rows, cols, ld);
        else convert_in<double, float><<<grid, 256, 0, s->stream>>>((const double *)staged, (float *)dst, rows, cols, ld);
    }
    return cuda_status(cudaGetLastError());
}

// Loads natural fields (staged device copies from stage_fields; nullptr keeps the current
// natural value, or zeros without keep_missing) into both ping-pong copies and rebuilds the
// carried state at the current parity with the prologue (so a member of a batch stays
// consistent with the batch's plan).
int load_state(adi_sim *s, const void *const staged[3], bool f32, bool keep_missing) {
    const Geometry &g = s->g;
    const size_t esz = s->esz;
    const int cur = s->parity;
    int rc = ADI_OK;
    if (staged[1] || !keep_missing) rc = load_field(s, staged[1], f32, s->V[cur].p, g.rows_v, g.ldv, g.ldvp);
    if (!rc) rc = cuda_status(cudaMemcpyAsync(s->V[1 - cur].p, s->V[cur].p, g.nVp() * esz, cudaMemcpyDeviceToDevice, s->stream));
    if (!rc && (staged[0] || !keep_missing)) rc = load_field(s, staged[0], f32, s->Uo.p, g.rows_u, g.ldu, g.ldu);
    if (!rc && (staged[2] || !keep_missing)) rc = load_field(s, staged[2], f32, s->Wo.p, g.rows_w, g.ldw, g.ldw);
    // with time-harmonic walls, u's walls are the harmonic data at the current time
    if (!rc) rc = harm_self(s, 2);
    // all four carried-pressure arrays start from u (their outer rows/columns stay the
    // Dirichlet data: line kernels write interior lines only)
    for (int k = 0; k <= 2 && !rc; k += 2)
        rc = cuda_status(cudaMemcpy2DAsync(s->A[k].p, g.lda * esz, s->Uo.p, g.ldu * esz, g.ldu * esz, g.rows_u,
                                           cudaMemcpyDeviceToDevice, s->stream));
    for (int k = 1; k <= 3 && !rc; k += 2) rc = transpose(s, s->Uo.p, g.rows_u, g.ldu, g.ldu, s->A[k].p, g.ldc);
    for (int k = 0; k < 2 && !rc; ++k) rc = transpose(s, s->Wo.p, g.rows_w, g.ldw, g.ldw, s->W[k].p, g.ldwc);
    if (!rc) rc = cuda_status(cudaStreamSynchronize(s->stream));
    if (!rc) rc = upload_sim_descs(s);  // descriptors of the current parity
    if (!rc) rc = prologue(s);
    return rc;
}

// True when ok(x[i]) holds for every i; large arrays are split over host threads.
template <typename F>
bool all_of_host(const double *x, size_t n, F ok) {
    auto range = [&](size_t lo, size_t hi) {
        bool good = true;
        for (size_t i = lo; i < hi; ++i) good &= ok(x[i]);
        return good;
    };
    const size_t kChunk = (size_t)1 << 20;
    const unsigned hw = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    if (n < 2 * kChunk || hw == 1) return range(0, n);
    const unsigned nt = (unsigned)std::min<size_t>(hw, n / kChunk);
    std::vector<std::thread> th;
    std::vector<char> res(nt, 1);
    for (unsigned t = 0; t < nt; ++t)
        th.emplace_back([&, t] { res[t] = range(n * t / nt, n * (t + 1) / nt) ? 1 : 0; });
    for (auto &x_ : th) x_.join();
    for (char r : res)
        if (!r) return false;
    return true;
}
bool finite_positive(const double *x, size_t n) {
    return all_of_host(x, n, [](double v) { return std::isfinite(v) && v > 0.0; });
}
bool all_finite(const double *x, size_t n) {
    if (!x) return true;
    return all_of_host(x, n, [](double v) { return std::isfinite(v); });
}

bool valid_config(int method, int nx, int ny, int precision) {
    return (method == ADI_CFD || method == ADI_MFD) && nx >= ADI_MIN_CELLS && ny >= ADI_MIN_CELLS &&
           nx <= ADI_MAX_CELLS && ny <= ADI_MAX_CELLS && (precision == ADI_FP32 || precision == ADI_FP64);
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
    if (!valid_config(method, nx, ny, precision)) return 0;
    Geometry g = make_geometry(method, nx, ny);
    size_t esz = elem_size(precision);
    size_t nl = (size_t)g.pix + g.piy;
    // a and C in both layouts, alpha, alphaT, Uo; two v copies; two w* copies and Wo
    size_t fields = (3 * g.nA() + 3 * g.nC() + g.nU() + 2 * g.nVp() + 2 * g.nWc() + g.nW()) * esz;
    size_t tab = nl * kTabLine * esz;
    size_t descs = 2 * nl * desc_size(precision);  // sim copy + plan copy
    int sv = default_solver(g, esz);
    size_t solver = sv == ADI_SOLVER_LINE ? v1_words(g) * (size_t)std::max(g.pix, g.piy) * esz
                                          : solver_words(g, sv) * esz;
    return fields + tab + descs + solver + sizeof(long long) + sizeof(int);
}

int adi_create(adi_handle *out, int method, int nx, int ny, double h, double dt,
               const double *c_field, const double *u0, const double *v0, const double *w0,
               int precision) {
    if (!out) return ADI_EINVAL;
    *out = nullptr;
    if (!valid_config(method, nx, ny, precision) || !(std::isfinite(h) && h > 0) ||
        !(std::isfinite(dt) && dt > 0) || !c_field)
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
    s->nlines[0] = g.piy; s->nlines[1] = g.pix;
    s->solver = default_solver(g, elem_size(precision));
    cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { delete s; return cuda_status(e); }
    s->own_stream = true;
    const size_t esz = s->esz;
    int rc = ADI_OK;
    rc = dev_alloc(s->A[0], g.nA() * esz);
    if (!rc) rc = dev_alloc(s->A[1], g.nC() * esz);
    if (!rc) rc = dev_alloc(s->A[2], g.nA() * esz);
    if (!rc) rc = dev_alloc(s->A[3], g.nC() * esz);
    for (int k = 0; k < 2 && !rc; ++k) {
        rc = dev_alloc(s->V[k], g.nVp() * esz);
        if (!rc) rc = dev_alloc(s->W[k], g.nWc() * esz);
    }
    if (!rc) rc = dev_alloc(s->alpha, g.nA() * esz);
    if (!rc) rc = dev_alloc(s->alphaT, g.nC() * esz);
    if (!rc) rc = dev_alloc(s->Uo, g.nU() * esz);
    if (!rc) rc = dev_alloc(s->Wo, g.nW() * esz);
    // padding entries are read by bulk copies and the finite check: start them at zero
    {
        DevBuf *zb[] = {&s->A[0], &s->A[1], &s->A[2], &s->A[3], &s->V[0], &s->V[1], &s->W[0], &s->W[1],
                        &s->alpha, &s->alphaT};
        for (DevBuf *b : zb)
            if (!rc) rc = cuda_status(cudaMemsetAsync(b->p, 0, b->bytes, s->stream));
    }
    if (!rc) rc = dev_alloc(s->tab, (size_t)(g.pix + g.piy) * kTabLine * esz);
    if (!rc) rc = dev_alloc(s->clock, sizeof(long long));
    if (!rc) rc = dev_alloc(s->status, 2 * sizeof(int));
    if (!rc) rc = cuda_status(cudaMemsetAsync(s->clock.p, 0, sizeof(long long), s->stream));
    if (!rc) {  // alpha = dt/2 c^2
        DevBuf staging;
        rc = dev_alloc(staging, g.nU() * sizeof(double));
        if (!rc) rc = upload(s, c_field, s->alpha.p, g.rows_u, g.ldu, g.lda, (double *)staging.p, 0.5 * dt, 1);
        if (!rc) rc = transpose(s, s->alpha.p, g.rows_u, g.ldu, g.lda, s->alphaT.p, g.ldc);
        if (!rc) rc = cuda_status(cudaStreamSynchronize(s->stream));
        dev_free(staging);
    }
    if (!rc) rc = setup_solver(s);
    if (!rc) {
        const void *f[3] = {u0, v0, w0}, *staged[3];
        rc = stage_fields(s, f, false, staged);
        if (!rc) rc = load_state(s, staged, false, false);
    }
    if (rc) { adi_destroy(s); return rc; }
    dev_free(s->xfer);  // set-up staging is not kept
    dev_free(s->pro);
    *out = s;
    return ADI_OK;
}

int adi_set_solver(adi_handle s, int solver) {
    if (!s || (solver != ADI_SOLVER_LINE && solver != ADI_SOLVER_CHUNKED && solver != ADI_SOLVER_FACTORED))
        return ADI_EINVAL;
    if (s->sticky) return s->sticky;
    if (s->in_batch) return ADI_EBUSY;
    if (solver == ADI_SOLVER_CHUNKED && !chunked_ok(s->g, s->esz)) return ADI_ENOTSUP;
    if (solver == ADI_SOLVER_FACTORED && !factored_ok(s->g, s->esz)) return ADI_ENOTSUP;
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return s->sticky = cuda_status(e);
    if (solver == s->solver) return ADI_OK;
    s->solver = solver;
    int rc = setup_solver(s);
    if (rc) s->sticky = rc;
    return rc;
}

int adi_get_solver(adi_handle s) { return s ? s->solver : -1; }

int adi_get_scan_reach(adi_handle s, int *reach) {
    if (!s || !reach) return ADI_EINVAL;
    *reach = s->solver == ADI_SOLVER_FACTORED ? s->fac_reach : 0;
    return ADI_OK;
}

}  // extern "C"

namespace {

// Solver choices measured by adi_autotune, per (method, nx, ny, precision).
struct TuneResult {
    int solver = ADI_SOLVER_LINE;
    double ms[3] = {-1.0, -1.0, -1.0};
    int nl_cap = 0, ring_cap = 0;  // the factored solver's launch parameters (0 = automatic)
    double ms_launch = -1.0;       // time per step with them
};
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, TuneResult> g_tune;

// The device state a step changes: carried and natural fields and the step clock.
int state_parts(adi_sim *s, DevBuf **parts) {
    DevBuf *list[] = {&s->A[0], &s->A[1], &s->A[2], &s->A[3], &s->V[0], &s->V[1],
                      &s->W[0], &s->W[1], &s->Uo, &s->Wo, &s->clock};
    int n = 0;
    for (DevBuf *b : list) parts[n++] = b;
    return n;
}
// Copies the step state into (save = true) or out of one device buffer, on the sim's stream.
int copy_state(adi_sim *s, DevBuf &buf, bool save) {
    DevBuf *parts[16];
    const int n = state_parts(s, parts);
    size_t total = 0;
    for (int k = 0; k < n; ++k) total += (parts[k]->bytes + 255) & ~(size_t)255;
    if (save) {
        int rc = dev_alloc(buf, total);
        if (rc) return rc;
    }
    size_t off = 0;
    for (int k = 0; k < n; ++k) {
        unsigned char *snap = (unsigned char *)buf.p + off;
        cudaError_t e = save ? cudaMemcpyAsync(snap, parts[k]->p, parts[k]->bytes, cudaMemcpyDeviceToDevice, s->stream)
                             : cudaMemcpyAsync(parts[k]->p, snap, parts[k]->bytes, cudaMemcpyDeviceToDevice, s->stream);
        if (e != cudaSuccess) return cuda_status(e);
        off += (parts[k]->bytes + 255) & ~(size_t)255;
    }
    return cuda_status(cudaStreamSynchronize(s->stream));
}

// Time per step of the sim's current solver: an untimed run of n steps (graph capture
// included), then n timed steps between two events on the sim's stream.
int time_steps(adi_sim *s, int n, double *ms) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    int rc = cuda_status(e);
    if (!rc) rc = adi_step(s, n);
    if (!rc) rc = cuda_status(cudaEventRecord(e0, s->stream));
    if (!rc) rc = adi_step(s, n);
    if (!rc) rc = cuda_status(cudaEventRecord(e1, s->stream));
    if (!rc) rc = adi_sync(s);
    float t = 0.f;
    if (!rc) rc = cuda_status(cudaEventElapsedTime(&t, e0, e1));
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (!rc) *ms = (double)t / n;
    return rc;
}

}  // namespace

extern "C" {

int adi_autotune(adi_handle s, int trials, int force, int *chosen, double *ms_per_step) {
    if (!s || trials < 1) return ADI_EINVAL;
    if (s->sticky) return s->sticky;
    if (s->in_batch) return ADI_EBUSY;
    const auto key = std::make_tuple(s->g.method, s->g.nx, s->g.ny, s->precision);
    TuneResult res;
    bool cached = false;
    if (!force) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) { res = it->second; cached = true; }
    }
    int rc = ADI_OK;
    if (!cached) {
        cudaError_t e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) return s->sticky = cuda_status(e);
        DevBuf snap;
        rc = copy_state(s, snap, true);
        if (rc) { dev_free(snap); return rc == ADI_ENOMEM ? ADI_ENOMEM : (s->sticky = rc); }
        const int parity0 = s->parity, solver0 = s->solver;
        const long long steps0 = s->steps;
        s->fac_nl_cap = 0;  // the solvers are compared with the automatic launch parameters
        s->fac_ring_cap = 0;
        const int n = trials + (trials & 1);  // even: both runs start at the same parity
        double best = 0.0;
        res.solver = -1;
        const int order[3] = {ADI_SOLVER_FACTORED, ADI_SOLVER_CHUNKED, ADI_SOLVER_LINE};
        for (int k = 0; k < 3 && !rc; ++k) {
            const int sv = order[k];
            if ((sv == ADI_SOLVER_FACTORED && !factored_ok(s->g, s->esz)) ||
                (sv == ADI_SOLVER_CHUNKED && !chunked_ok(s->g, s->esz)))
                continue;
            rc = adi_set_solver(s, sv);
            double ms = 0.0;
            if (!rc) rc = time_steps(s, n, &ms);
            // every candidate starts from the saved state
            if (!rc) rc = copy_state(s, snap, false);
            if (rc) break;
            s->parity = parity0;
            s->steps = steps0;
            res.ms[sv] = ms;
            if (res.solver < 0 || ms < best) { best = ms; res.solver = sv; }
        }
        // the factored solver's launch parameters: lines per CTA (the automatic count, then
        // halved down to one) and the staging ring depth (automatic: as many groups in flight
        // as shared memory takes, up to three; then capped at 1 and at 2)
        if (!rc && res.solver == ADI_SOLVER_FACTORED) {
            rc = adi_set_solver(s, ADI_SOLVER_FACTORED);
            const int nl0 = std::max(fac_split_line(s->g.method, s->g.nx) ? 1 : fac_lines_per_cta(s->g.method, s->g.nx, s->esz),
                                     fac_split_line(s->g.method, s->g.ny) ? 1 : fac_lines_per_cta(s->g.method, s->g.ny, s->esz));
            std::vector<int> caps = {0};
            for (int c = nl0 / 2; c >= 1; c /= 2) caps.push_back(c);
            res.ms_launch = res.ms[ADI_SOLVER_FACTORED];
            for (size_t ci = 0; ci < caps.size() && !rc; ++ci)
                for (int ring = 0; ring <= 2 && !rc; ++ring) {
                    if (ci == 0 && ring == 0) continue;  // the automatic choice, timed above
                    s->fac_nl_cap = caps[ci];
                    s->fac_ring_cap = ring;
                    rc = plan_build(s->plan, std::vector<adi_sim *>{s}, s->stream);
                    s->plan_base = s->parity;
                    double ms = 0.0;
                    if (!rc) rc = time_steps(s, n, &ms);
                    if (!rc) rc = copy_state(s, snap, false);
                    if (rc) break;
                    s->parity = parity0;
                    s->steps = steps0;
                    if (ms < res.ms_launch) { res.ms_launch = ms; res.nl_cap = caps[ci]; res.ring_cap = ring; }
                }
        }
        if (rc) {
            dev_free(snap);
            return s->sticky = rc;
        }
        dev_free(snap);
        if (res.solver < 0) res.solver = solver0;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[key] = res;
    }
    s->fac_nl_cap = res.solver == ADI_SOLVER_FACTORED ? res.nl_cap : 0;
    s->fac_ring_cap = res.solver == ADI_SOLVER_FACTORED ? res.ring_cap : 0;
    rc = adi_set_solver(s, res.solver);  // rebuilds the plan with the chosen parameters
    if (rc) return rc;
    if (chosen) *chosen = res.solver;
    if (ms_per_step)
        for (int k = 0; k < 3; ++k) ms_per_step[k] = res.ms[k];
    return ADI_OK;
}

int adi_set_launch(adi_handle s, int lines_per_cta, int ring_depth) {
    if (!s || lines_per_cta < 0 || ring_depth < 0 || ring_depth > 3) return ADI_EINVAL;
    if (s->sticky) return s->sticky;
    if (s->in_batch) return ADI_EBUSY;
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return s->sticky = cuda_status(e);
    s->fac_nl_cap = lines_per_cta;
    s->fac_ring_cap = ring_depth;
    int rc = plan_build(s->plan, std::vector<adi_sim *>{s}, s->stream);
    s->plan_base = s->parity;
    if (rc) s->sticky = rc;
    return rc;
}

int adi_get_launch(adi_handle s, int *lines_per_cta, int *ring_depth) {
    if (!s) return ADI_EINVAL;
    if (lines_per_cta) *lines_per_cta = s->fac_nl_cap;
    if (ring_depth) *ring_depth = s->fac_ring_cap;
    return ADI_OK;
}

int adi_set_harmonic(adi_handle s, const double *B, const double *F, double omega, double phase_b,
                     double phase_f) {
    if (!s) return ADI_EINVAL;
    if (s->sticky) return s->sticky;
    if (s->in_batch) return ADI_EBUSY;
    if (!std::isfinite(omega) || !std::isfinite(phase_b) || !std::isfinite(phase_f)) return ADI_EINVAL;
    const Geometry &g = s->g;
    if (F && !B) return ADI_EINVAL;
    if ((B && !all_finite(B, g.nU())) || (F && !all_finite(F, g.nU()))) return ADI_EINVAL;
    if (!B && !s->harm_on) return ADI_OK;
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return s->sticky = cuda_status(e);
    int rc = ADI_OK;
    if (!B) {  // back to time-independent walls: the ones the fields hold now
        s->harm_on = false;
        dev_free(s->h_edges); dev_free(s->h_frow); dev_free(s->h_fcol); dev_free(s->h_self);
    } else {
        // the wall amplitudes, kept in FP64: west, east (one per row), south, north (per column)
        std::vector<double> ed(2 * (size_t)g.rows_u + 2 * (size_t)g.ldu);
        for (int i = 0; i < g.rows_u; ++i) {
            ed[i] = B[(size_t)i * g.ldu];
            ed[g.rows_u + i] = B[(size_t)i * g.ldu + g.ldu - 1];
        }
        for (int j = 0; j < g.ldu; ++j) {
            ed[2 * (size_t)g.rows_u + j] = B[j];
            ed[2 * (size_t)g.rows_u + g.ldu + j] = B[(size_t)(g.rows_u - 1) * g.ldu + j];
        }
        if (!s->h_edges.p) rc = dev_alloc(s->h_edges, ed.size() * sizeof(double));
        if (!rc) rc = cuda_status(cudaMemcpyAsync(s->h_edges.p, ed.data(), ed.size() * sizeof(double),
                                                  cudaMemcpyHostToDevice, s->stream));
        if (!rc) rc = cuda_status(cudaStreamSynchronize(s->stream));  // ed leaves scope
        if (!rc && F) {  // F in the layouts of both stages' carried pressure
            if (!s->h_frow.p) rc = dev_alloc(s->h_frow, g.nA() * s->esz);
            if (!rc && !s->h_fcol.p) rc = dev_alloc(s->h_fcol, g.nC() * s->esz);
            if (!rc) rc = cuda_status(cudaMemsetAsync(s->h_frow.p, 0, g.nA() * s->esz, s->stream));
            if (!rc) rc = cuda_status(cudaMemsetAsync(s->h_fcol.p, 0, g.nC() * s->esz, s->stream));
            if (!rc) rc = xfer_buffer(s);
            if (!rc) rc = upload(s, F, s->h_frow.p, g.rows_u, g.ldu, g.lda, (double *)s->xfer.p, 1.0, 0);
            if (!rc) rc = transpose(s, s->h_frow.p, g.rows_u, g.ldu, g.lda, s->h_fcol.p, g.ldc);
            if (!rc) rc = cuda_status(cudaStreamSynchronize(s->stream));
        } else if (!rc) {
            dev_free(s->h_frow); dev_free(s->h_fcol);
        }
        if (!rc) {
            s->harm_on = true;
            s->h_omega = omega; s->h_phb = phase_b; s->h_phf = phase_f;
        }
    }
    // descriptors (who advances the clock), the plan (its harmonic records), then the state:
    // walls at the current time, carried state rebuilt from the current fields
    if (!rc) {
        if (s->precision == ADI_FP64) build_host_descs<double>(s); else build_host_descs<float>(s);
        rc = sync_clock(s);
    }
    if (!rc) rc = upload_sim_descs(s);
    if (!rc) rc = plan_build(s->plan, std::vector<adi_sim *>{s}, s->stream);
    s->plan_base = s->parity;
    if (!rc) {
        const void *none[3] = {nullptr, nullptr, nullptr};
        rc = load_state(s, none, false, true);
    }
    dev_free(s->xfer);
    dev_free(s->pro);
    if (rc) s->sticky = rc;
    return rc;
}

int adi_set_sponge(adi_handle s, double width, double a) {
    if (!s) return ADI_EINVAL;
    if (s->sticky) return s->sticky;
    if (s->in_batch) return ADI_EBUSY;
    if (!std::isfinite(width) || !std::isfinite(a) || width < 0 || a < 0) return ADI_EINVAL;
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return s->sticky = cuda_status(e);
    int rc = ADI_OK;
    if (width == 0 || a == 0) {
        if (!s->sp_on) return ADI_OK;
        s->sp_on = false;
        dev_free(s->sp_desc[0]); dev_free(s->sp_desc[1]); dev_free(s->sp_scr);
    } else {
        const Geometry &g = s->g;
        const long long st = std::max(1, s->nlines[1]);
        const int N = g.ny;
        const size_t scr = (size_t)(2 * N + 2) * st, nfac = g.method == ADI_CFD ? prologue_factor_count(N) : 0;
        const size_t dbytes = s->h_desc[0][1].size();
        if (s->sp_desc[0].bytes != dbytes) {
            dev_free(s->sp_desc[0]); dev_free(s->sp_desc[1]);
            rc = dev_alloc(s->sp_desc[0], dbytes);
            if (!rc) rc = dev_alloc(s->sp_desc[1], dbytes);
        }
        if (!rc && s->sp_scr.bytes != (scr + nfac) * s->esz) {
            dev_free(s->sp_scr);
            rc = dev_alloc(s->sp_scr, (scr + nfac) * s->esz);
            if (!rc && nfac) {
                std::vector<double> f;
                prologue_factors(N, f);
                if (s->precision == ADI_FP64) {
                    rc = cuda_status(cudaMemcpyAsync((double *)s->sp_scr.p + scr, f.data(), f.size() * sizeof(double),
                                                     cudaMemcpyHostToDevice, s->stream));
                    if (!rc) rc = cuda_status(cudaStreamSynchronize(s->stream));
                } else {
                    std::vector<float> ff(f.begin(), f.end());
                    rc = cuda_status(cudaMemcpyAsync((float *)s->sp_scr.p + scr, ff.data(), ff.size() * sizeof(float),
                                                     cudaMemcpyHostToDevice, s->stream));
                    if (!rc) rc = cuda_status(cudaStreamSynchronize(s->stream));  // ff leaves scope
                }
            }
        }
        if (!rc) { s->sp_on = true; s->sp_width = width; s->sp_a = a; }
    }
    if (!rc) rc = plan_build(s->plan, std::vector<adi_sim *>{s}, s->stream);
    s->plan_base = s->parity;
    if (rc) s->sticky = rc;
    return rc;
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
    if (s->precision == ADI_FP64) build_host_descs<double>(s); else build_host_descs<float>(s);
    int rc = sync_clock(s);  // the source is evaluated at the current step's time
    if (!rc) rc = upload_sim_descs(s);
    if (!rc) rc = plan_build(s->plan, std::vector<adi_sim *>{s}, s->stream);
    s->plan_base = s->parity;
    if (!rc) rc = prologue(s);  // a picks up dt/2 f(t_now) at the source point
    dev_free(s->pro);           // a one-off: the prologue's scratch is not kept
    if (rc) s->sticky = rc;
    return rc;
}

int adi_step(adi_handle s, int nsteps) {
    if (!s || nsteps < 0) return ADI_EINVAL;
    if (s->sticky) return s->sticky;
    if (s->in_batch) return ADI_EBUSY;
    if (nsteps == 0) return ADI_OK;
    // the own plan's parity 0 is the sim's parity when the plan was built
    const int q0 = s->parity ^ s->plan_base;
    cudaError_t e = nsteps == 1 ? enqueue_steps(s->plan, q0, 1, s->stream)
                                : run_graph(s->plan, q0, nsteps, s->stream);
    if (e != cudaSuccess) return s->sticky = cuda_status(e);
    s->steps += nsteps;
    s->parity ^= nsteps & 1;
    return ADI_OK;
}

int adi_sync(adi_handle s) {
    if (!s) return ADI_EINVAL;
    if (s->sticky) return s->sticky;
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return s->sticky = cuda_status(e);
    int rc = plan_fault(s->plan, s->stream);
    if (rc) s->sticky = rc;
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
    struct { const void *src; double *dst; size_t rows, cols, ld; } parts[3] = {
        {s->Uo.p, u, (size_t)g.rows_u, (size_t)g.ldu, (size_t)g.ldu},
        {s->V[s->parity].p, v, (size_t)g.rows_v, (size_t)g.ldv, (size_t)g.ldvp},
        {s->Wo.p, w, (size_t)g.rows_w, (size_t)g.ldw, (size_t)g.ldw}};
    rc = xfer_buffer(s);
    if (rc) return rc;
    DevBuf &tmp = s->xfer;
    for (auto &pt : parts) {
        if (!pt.dst) continue;
        const size_t n = pt.rows * pt.cols;
        const dim3 grid = conv_grid(pt.rows, pt.cols);
        if (s->precision == ADI_FP64)
            convert_to_double<double><<<grid, 256, 0, s->stream>>>((const double *)pt.src, (double *)tmp.p, pt.rows, pt.cols, pt.ld);
        else
            convert_to_double<float><<<grid, 256, 0, s->stream>>>((const float *)pt.src, (double *)tmp.p, pt.rows, pt.cols, pt.ld);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(pt.dst, tmp.p, n * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) return s->sticky = cuda_status(e);
    }
    return ADI_OK;
}

namespace {
// adi_set_fields / adi_set_fields_f32: stage and check every given field, then load them.
int set_fields_any(adi_handle s, const void *u, const void *v, const void *w, bool f32) {
    if (!s) return ADI_EINVAL;
    if (s->in_batch && s->batch_stream) {
        cudaError_t be = cudaStreamSynchronize(s->batch_stream);
        if (be != cudaSuccess) return s->sticky = cuda_status(be);
    }
    int rc = adi_sync(s);
    if (rc) return rc;
    const void *f[3] = {u, v, w}, *staged[3];
    rc = stage_fields(s, f, f32, staged);
    if (rc == ADI_EINVAL) return rc;
    if (rc) return s->sticky = rc;
    rc = load_state(s, staged, f32, true);
    if (rc) s->sticky = rc;
    return rc;
}
}  // namespace

int adi_set_fields(adi_handle s, const double *u, const double *v, const double *w) {
    return set_fields_any(s, u, v, w, false);
}

int adi_set_fields_f32(adi_handle s, const float *u, const float *v, const float *w) {
    return set_fields_any(s, u, v, w, true);
}

int adi_read_fields_f32(adi_handle s, float *u, float *v, float *w) {
    if (!s) return ADI_EINVAL;
    if (s->in_batch && s->batch_stream) {
        cudaError_t be = cudaStreamSynchronize(s->batch_stream);
        if (be != cudaSuccess) return s->sticky = cuda_status(be);
    }
    int rc = adi_sync(s);
    if (rc) return rc;
    const Geometry &g = s->g;
    struct { const void *src; float *dst; size_t rows, cols, ld; } parts[3] = {
        {s->Uo.p, u, (size_t)g.rows_u, (size_t)g.ldu, (size_t)g.ldu},
        {s->V[s->parity].p, v, (size_t)g.rows_v, (size_t)g.ldv, (size_t)g.ldvp},
        {s->Wo.p, w, (size_t)g.rows_w, (size_t)g.ldw, (size_t)g.ldw}};
    // FP64 fields are converted through the staging buffer; an FP32 field whose rows are padded
    // (v) is first packed there on the device, since a pitched device-to-host copy runs at about
    // half the speed of a contiguous one
    bool need_xfer = s->precision == ADI_FP64;
    for (auto &pt : parts) need_xfer |= pt.dst && pt.ld != pt.cols;
    if (need_xfer) {
        rc = xfer_buffer(s);
        if (rc) return rc;
    }
    cudaError_t e = cudaSuccess;
    for (auto &pt : parts) {
        if (!pt.dst || e != cudaSuccess) continue;
        if (s->precision == ADI_FP32 && pt.ld == pt.cols) {  // straight from the device array
            e = cudaMemcpyAsync(pt.dst, pt.src, pt.rows * pt.cols * sizeof(float), cudaMemcpyDeviceToHost, s->stream);
        } else if (s->precision == ADI_FP32) {
            convert_out<float, float><<<conv_grid(pt.rows, pt.cols), 256, 0, s->stream>>>(
                (const float *)pt.src, (float *)s->xfer.p, pt.rows, pt.cols, pt.ld);
            e = cudaGetLastError();
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(pt.dst, s->xfer.p, pt.rows * pt.cols * sizeof(float), cudaMemcpyDeviceToHost, s->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);  // the staging is reused
        } else {
            const size_t n = pt.rows * pt.cols;
            convert_out<double, float><<<conv_grid(pt.rows, pt.cols), 256, 0, s->stream>>>((const double *)pt.src,
                                                                                           (float *)s->xfer.p, pt.rows,
                                                                                           pt.cols, pt.ld);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaMemcpyAsync(pt.dst, s->xfer.p, n * sizeof(float), cudaMemcpyDeviceToHost, s->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);  // the staging is reused
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return s->sticky = cuda_status(e);
    return ADI_OK;
}

int adi_check_finite(adi_handle s) {
    if (!s) return ADI_EINVAL;
    int rc = adi_sync(s);
    if (rc) return rc;
    cudaError_t e = cudaMemsetAsync(s->status.p, 0, sizeof(int), s->stream);
    const Geometry &g = s->g;
    const void *fields[4] = {s->A[0].p, s->V[s->parity].p, s->W[s->parity].p, s->Uo.p};
    size_t ns[4] = {g.nA(), g.nVp(), g.nWc(), g.nU()};
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
    if (s->in_batch) return ADI_EBUSY;  // a batch or ticket still refers to it
    if (s->stream) cudaStreamSynchronize(s->stream);
    plan_free(s->plan);
    DevBuf *bufs[] = {&s->A[0], &s->A[1], &s->A[2], &s->A[3], &s->V[0], &s->V[1], &s->W[0], &s->W[1], &s->alpha,
                      &s->alphaT, &s->Uo, &s->Wo, &s->tab, &s->sep, &s->cold_all, &s->clock, &s->status,
                      &s->xfer, &s->pro, &s->h_edges, &s->h_frow, &s->h_fcol, &s->h_self,
                      &s->sp_desc[0], &s->sp_desc[1], &s->sp_scr};
    for (DevBuf *b : bufs) dev_free(*b);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    (void)cudaGetLastError();
    delete s;
    return ADI_OK;
}

// ----------------------------------------------------------------------------------------
// Batches: one plan over every member's lines.
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
    for (int k = 0; k < n; ++k) {
        cudaStreamSynchronize(sims[k]->stream);
        b->sims.push_back(sims[k]);
    }
    int rc = cuda_status(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
    if (!rc) b->own_stream = true;
    if (!rc) rc = plan_build(b->plan, b->sims, b->stream);
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

static int batch_fail(adi_batch b, cudaError_t e) {
    b->sticky = cuda_status(e);
    for (adi_sim *s : b->sims) s->sticky = b->sticky;
    return b->sticky;
}

int adi_batch_step(adi_batch b, int nsteps) {
    if (!b || nsteps < 0) return ADI_EINVAL;
    if (b->sticky) return b->sticky;
    if (nsteps == 0) return ADI_OK;
    cudaError_t e = nsteps == 1 ? enqueue_steps(b->plan, b->parity, 1, b->stream)
                                : run_graph(b->plan, b->parity, nsteps, b->stream);
    if (e != cudaSuccess) return batch_fail(b, e);
    b->parity ^= nsteps & 1;
    for (adi_sim *s : b->sims) { s->steps += nsteps; s->parity ^= nsteps & 1; }
    return ADI_OK;
}

int adi_batch_half_step(adi_batch b, int stage, int write_natural) {
    if (!b || (stage != 1 && stage != 2)) return ADI_EINVAL;
    if (b->sticky) return b->sticky;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (b->timing) {
        std::vector<cudaEvent_t> &pool = b->ev[stage - 1];
        size_t &used = b->ev_used[stage - 1];
        while (pool.size() < used + 2) {
            cudaEvent_t ev;
            if (cudaEventCreate(&ev) != cudaSuccess) { (void)cudaGetLastError(); return ADI_ECUDA; }
            pool.push_back(ev);
        }
        e0 = pool[used]; e1 = pool[used + 1];
        used += 2;
    }
    cudaError_t e = enqueue_stage_any(b->plan, b->parity, stage - 1, write_natural ? 1 : 0, b->stream, e0, e1);
    if (e != cudaSuccess) return batch_fail(b, e);
    if (stage == 2) {
        b->parity ^= 1;
        for (adi_sim *s : b->sims) { s->steps += 1; s->parity ^= 1; }
    }
    return ADI_OK;
}

int adi_batch_sync(adi_batch b) {
    if (!b) return ADI_EINVAL;
    if (b->sticky) return b->sticky;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return batch_fail(b, e);
    int rc = plan_fault(b->plan, b->stream);
    if (rc) b->sticky = rc;
    return rc;
}

int adi_batch_set_timing(adi_batch b, int enable) {
    if (!b) return ADI_EINVAL;
    b->timing = enable != 0;
    return ADI_OK;
}

int adi_batch_solve_time(adi_batch b, int stage, double *total_ms, int *count) {
    if (!b || (stage != 1 && stage != 2)) return ADI_EINVAL;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return batch_fail(b, e);
    const std::vector<cudaEvent_t> &pool = b->ev[stage - 1];
    size_t &used = b->ev_used[stage - 1];
    double sum = 0.0;
    for (size_t k = 0; k + 1 < used; k += 2) {
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, pool[k], pool[k + 1]);
        if (e != cudaSuccess) return batch_fail(b, e);
        sum += ms;
    }
    if (total_ms) *total_ms = sum;
    if (count) *count = (int)(used / 2);
    used = 0;
    return ADI_OK;
}

// ----------------------------------------------------------------------------------------
// Asynchronous batches with per-simulation step counts (adi_batch_submit / adi_batch_poll).
// ----------------------------------------------------------------------------------------
namespace {

struct Ticket {
    std::vector<adi_sim *> sims;
    std::vector<Plan *> plans;  // one per phase, kept until the ticket completes
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
};
std::mutex g_ticket_mu;
std::map<int, Ticket *> g_tickets;
int g_next_ticket = 1;

void ticket_free(Ticket *t) {
    if (t->stream) cudaStreamSynchronize(t->stream);
    for (Plan *p : t->plans) { plan_free(*p); delete p; }
    for (adi_sim *s : t->sims) { s->in_batch = false; s->batch_stream = nullptr; }
    if (t->done) cudaEventDestroy(t->done);
    if (t->stream) cudaStreamDestroy(t->stream);
    (void)cudaGetLastError();
    delete t;
}

}  // namespace

int adi_batch_submit(const adi_handle *sims, const int *nsteps, int n, int *ticket) {
    if (!sims || !nsteps || n < 1 || !ticket) return ADI_EINVAL;
    const int prec = sims[0] ? sims[0]->precision : -1;
    for (int k = 0; k < n; ++k) {
        if (!sims[k] || nsteps[k] < 0 || sims[k]->precision != prec) return ADI_EINVAL;
        if (sims[k]->in_batch) return ADI_EBUSY;
        if (sims[k]->sticky) return sims[k]->sticky;
        for (int q = 0; q < k; ++q)
            if (sims[q] == sims[k]) return ADI_EINVAL;
    }
    Ticket *t = new (std::nothrow) Ticket;
    if (!t) return ADI_ENOMEM;
    cudaStream_t up = nullptr;
    int rc = cuda_status(cudaStreamCreateWithFlags(&t->stream, cudaStreamNonBlocking));
    if (!rc) rc = cuda_status(cudaStreamCreateWithFlags(&up, cudaStreamNonBlocking));
    if (!rc) rc = cuda_status(cudaEventCreateWithFlags(&t->done, cudaEventDisableTiming));
    std::vector<int> par0(n);
    for (int k = 0; k < n && !rc; ++k) {
        rc = cuda_status(cudaStreamSynchronize(sims[k]->stream));
        t->sims.push_back(sims[k]);
        par0[k] = sims[k]->parity;
    }
    // Phases: every member with steps left advances together until the smallest remaining
    // count is reached; the members done by then leave.  Each phase's plan is built (on a
    // separate stream, so that nothing waits for the earlier phases' kernels) with every
    // member at the parity it will have when the phase starts.
    // All plans first: a failure here leaves every member untouched.
    std::vector<int> runs;
    int done_steps = 0;
    while (!rc) {
        std::vector<adi_sim *> active;
        int next = 0;
        for (int k = 0; k < n; ++k)
            if (nsteps[k] > done_steps) {
                active.push_back(sims[k]);
                if (next == 0 || nsteps[k] < next) next = nsteps[k];
            }
        if (active.empty()) break;
        for (int k = 0; k < n; ++k) sims[k]->parity = par0[k] ^ (done_steps & 1);
        Plan *p = new (std::nothrow) Plan;
        if (!p) { rc = ADI_ENOMEM; break; }
        t->plans.push_back(p);
        rc = plan_build(*p, active, up);
        runs.push_back(next - done_steps);
        done_steps = next;
    }
    for (int k = 0; k < n; ++k) sims[k]->parity = par0[k];
    if (up) cudaStreamDestroy(up);
    if (rc) {
        ticket_free(t);
        return rc;
    }
    for (size_t i = 0; i < t->plans.size() && !rc; ++i) {
        const int run = runs[i];
        rc = cuda_status(run == 1 ? enqueue_steps(*t->plans[i], 0, 1, t->stream)
                                  : run_graph(*t->plans[i], 0, run, t->stream));
    }
    if (!rc) rc = cuda_status(cudaEventRecord(t->done, t->stream));
    if (rc) {  // some phases may have run: the members' state is no longer known
        ticket_free(t);
        for (int k = 0; k < n; ++k) sims[k]->sticky = rc;
        return rc;
    }
    for (int k = 0; k < n; ++k) {
        sims[k]->parity = par0[k] ^ (nsteps[k] & 1);
        sims[k]->steps += nsteps[k];
        sims[k]->in_batch = true;
        sims[k]->batch_stream = t->stream;
    }
    std::lock_guard<std::mutex> lk(g_ticket_mu);
    *ticket = g_next_ticket++;
    g_tickets[*ticket] = t;
    return ADI_OK;
}

int adi_batch_poll(int ticket, int *done) {
    if (!done) return ADI_EINVAL;
    *done = 0;
    Ticket *t = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_ticket_mu);
        auto it = g_tickets.find(ticket);
        if (it == g_tickets.end()) return ADI_EINVAL;
        t = it->second;
    }
    const cudaError_t q = cudaEventQuery(t->done);
    if (q == cudaErrorNotReady) return ADI_OK;
    int rc = cuda_status(q);
    for (Plan *p : t->plans)
        if (!rc) rc = plan_fault(*p, t->stream);
    {
        std::lock_guard<std::mutex> lk(g_ticket_mu);
        g_tickets.erase(ticket);
    }
    std::vector<adi_sim *> sims = t->sims;
    ticket_free(t);
    if (rc)
        for (adi_sim *s : sims) s->sticky = rc;
    *done = 1;
    return rc;
}

int adi_batch_destroy(adi_batch b) {
    if (!b) return ADI_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (int k = 0; k < 2; ++k)
        for (cudaEvent_t ev : b->ev[k]) cudaEventDestroy(ev);
    plan_free(b->plan);
    for (adi_sim *s : b->sims) { s->in_batch = false; s->batch_stream = nullptr; }
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    (void)cudaGetLastError();
    delete b;
    return ADI_OK;
}

}  // extern "C"
