// adi_internal.h -- declarations shared by the host side (adi_api.cu) and the kernels
// (adi_kernels.cu, adi_chunked.cu).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

namespace adi {

// One grid line of one simulation, as every line kernel sees it.  Pressure-like values
// (a or C, Dirichlet ends included) and alpha share one indexing along the line; the
// velocity line (v in stage 1, w* in stage 2) has N+1 entries.
// Inputs (p, v) and outputs (po, vo) are distinct buffers: line kernels read stencil halos
// of neighbouring chunks while other chunks write, so a half step never updates in place.
template <typename T>
struct alignas(16) LineDesc {  // 16-byte multiple: descriptor arrays are bulk-copied
    T *p;              // pressure line (input), element 0 and element L are the Dirichlet values
    T *v;              // velocity line v_0..v_N (input)
    T *po;             // pressure line (output, same indexing as p)
    T *vo;             // velocity line (output, same indexing as v)
    const T *alpha;    // dt/2 * kappa along the pressure line
    T *u_out;          // natural pressure output (stage-2 lines) or nullptr; also the
                       // natural input of the prologue
    T *w_out;          // natural velocity output (stage-2 lines) or nullptr
    const T *tab;      // head/tail elimination tables (kTabLine values)
    long long sp;      // element stride of p and alpha along the line
    long long sv;      // element stride of v along the line
    long long spo;     // element stride of po along the line
    long long svo;     // element stride of vo along the line
    long long snp;     // element stride of u_out along the line
    long long snv;     // element stride of w_out along the line
    int N;             // cells along the line
    int method;        // kCFD / kMFD
    int src_k;         // index along the pressure line of the point source, or -1
    int advance_clock; // 1: this line's thread advances the simulation clock after use
    long long *clock;  // completed steps of the owning simulation
    double beta;       // dt/2 (density 1)
    double inv_h;
    double dt;
    double src_amp, src_f0, src_tdelay; // Ricker source (amp, f0, delay)
    double src_scale;  // dt / (2 h^2)
    T *sep;            // per-line record of the chunked or factored solver
    int chunkM;        // chunk length (blocks) the separator factors were built for
    int pad2;
};

// Launchers (defined in adi_kernels.cu).
template <typename T>
cudaError_t launch_precompute(const LineDesc<T> *d, int nlines, T *tab_out_base,
                              int *status, cudaStream_t s);
template <typename T>
cudaError_t launch_line_solve_v1(const LineDesc<T> *d, int nlines, T *scratch,
                                 long long scratch_stride, int write_natural, cudaStream_t s);
template <typename T>
cudaError_t launch_prologue(const LineDesc<T> *col_lines, int nlines, const T *u_nat,
                            const T *w_nat, long long u_ld, long long w_ld, T *scratch,
                            long long scratch_stride, cudaStream_t s);
template <typename T>
cudaError_t launch_finite_check(const T *x, size_t n, int *flag, cudaStream_t s);

// Scratch words per line of the thread-per-line solver (solution + block factors).
size_t v1_scratch_words(int method, int N);

// Factored solver (adi_factored.cu).
// One line group of a launch, built on the host: lines [first, first + nl) of one simulation
// and direction, with the geometry every thread of the CTA needs.
// Copied into shared memory with the group's lines.
struct alignas(16) FacGroup {
    int first, nl, N, T;     // first descriptor, lines, cells per line, threads per line
    int tact, hu, tu, mid;   // chunks with blocks, end-region unknowns, first middle node / cell
    int lp, rec, eh, et;     // staged line elements, record elements, head / tail table offsets
    int info, pl, ls, scr;   // scan-reach offset, far Dirichlet index, staged line stride, scratch offset
    double ih, beta;         // 1/h and dt/2 of the simulation
    float ihf, betaf;        // the same in FP32
    unsigned tdiv;           // ceil(2^32 / T) (0 for T = 1): thread / T = umulhi(thread, tdiv)
    int pad1;
};
FacGroup fac_group_of(int method, int N, int first, int nl, double inv_h, double beta);
bool fac_supported(int method, int N, size_t esz);  // chunks fit a CTA, stage fits smem
size_t fac_words(int method, int N);     // elements of one line's record
int fac_chunks(int method, int N);       // threads per line
int fac_variant(int method, int N);      // compiled kernel instance: 0 CFD, 1-2 MFD
constexpr int kFacVariants = 3;
int fac_lines_per_cta(int method, int N, size_t esz);
size_t fac_stage_bytes(int method, int N, int nl, size_t esz);  // shared memory of one stage
int fac_stages_for(size_t stage_bytes, size_t esz);  // 2 (prefetch), 1, or 0 (does not fit)
size_t fac_ws_doubles();                 // FP64 workspace per line of the precompute
// status[0]: set when a line system is singular; status[1]: atomic max of the lines' scan reach
template <typename T>
cudaError_t launch_fac_precompute(const LineDesc<T> *d, int nlines, double *ws, int *status,
                                  cudaStream_t s);
// max_reach: the largest scan reach of the launch's lines (beyond the window limit the
// kernel uses the full scan)
template <typename T>
cudaError_t launch_line_solve_factored(const LineDesc<T> *d, const FacGroup *groups, int ngroups,
                                       int variant, size_t stage_bytes, int stages, int grid,
                                       int natural, int max_reach, int *fault, cudaStream_t s);

// Chunked solver (adi_chunked.cu).
int chunk_M(int method);                 // chunk length in blocks used by the kernel
int chunk_count(int method, int N, int M);  // chunks per line
// dynamic shared memory of one CTA of the chunked kernel (nl lines of N cells, T chunks)
size_t chunked_smem_bytes(int N, int nl, int T, int bs, size_t esz);
constexpr int kChunkSmemMax = 110 * 1024;  // per CTA, so that two CTAs share an SM
template <typename T>
cudaError_t launch_precompute_sep(const LineDesc<T> *d, int nlines, cudaStream_t s);
template <typename T>
cudaError_t launch_line_solve_chunked(const LineDesc<T> *d, const int4 *groups, int ngroups,
                                      int method, size_t smem_bytes, int write_natural,
                                      cudaStream_t s);

}  // namespace adi
