// adi_internal.h -- declarations shared by the host side (adi_api.cu) and the kernels
// (adi_kernels.cu, adi_chunked.cu).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <vector>

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
// fac: the Thomas factors of prologue_factors() in T, or nullptr (formed on the fly; the
// scratch then holds two vectors per line)
template <typename T>
cudaError_t launch_prologue(const LineDesc<T> *col_lines, int nlines, const T *fac, T *scratch,
                            long long scratch_stride, cudaStream_t s);
// CFD: 3 (N+1) + 3 (N-1) Thomas factors of P and Pbar, then the start-up factors of the
// chunked solves (prologue_factor_count(N) values in all)
void prologue_factors(int N, std::vector<double> &out);
size_t prologue_factor_count(int N);
// The prologue over the y-lines of one simulation (N cells each) with one thread per line
// element for the stencils (and, for CFD, one per line for the Thomas solves with fac).
// scratch: 2N elements per line (element k at k * st + line).
template <typename T>
cudaError_t launch_prologue_lines(const LineDesc<T> *col_lines, int nlines, int N, int method, const T *fac,
                                  T *scratch, long long st, cudaStream_t s);
template <typename T>
cudaError_t launch_finite_check(const T *x, size_t n, int *flag, cudaStream_t s);

// Scratch words per line of the thread-per-line solver (solution + block factors).
size_t v1_scratch_words(int method, int N);

// Time-harmonic walls and forcing (adi_harmonic.cu): one record per simulation that has them.
// Walls u = B cos(omega t + phb); forcing f = F cos(omega t + phf); t = clock * dt.
struct HarmDesc {
    void *a_row;          // carried a, row-major (leading dimension lda): the x-lines' input
    void *c_col;          // carried C, column-major (leading dimension ldc): the y-lines' input
    void *uo;             // natural pressure, row-major rows_u x ldu
    const void *f_row;    // F at U's points, row-major (lda), or nullptr (no forcing)
    const void *f_col;    // F column-major (ldc), or nullptr
    const double *edges;  // B on the walls: west [rows_u], east [rows_u], south [ldu], north [ldu]
    long long *clock;     // completed steps of the simulation
    int rows_u, ldu, lda, ldc;
    double dt, omega, phb, phf;
};
// mode 0: after stage 1; 1: after stage 2 (advances the clocks); 2: the natural walls at the
// clock's time; 3: the carried state after a prologue.  max_points: the largest rows_u * ldu.
template <typename T>
cudaError_t launch_harmonic(const HarmDesc *d, int n, size_t max_points, int mode, cudaStream_t s);

// Absorbing layers (adi_sponge.cu): the damped fields of one simulation after a step.
struct SpongeRec {
    void *uo, *v, *wo;          // natural u (rows_u x ldu), natural v (rows_v x ldv, leading
                                // dimension ldvp), natural w (rows_w x ldw)
    void *v_other;              // the other copy of v: its first and last rows, which no x-line
                                // writes, must hold the same damped values
    int method, nx, ny;
    int rows_u, ldu, rows_v, ldv, ldvp, rows_w, ldw;
    double width, a;            // layer width in cells, damping strength
};
template <typename T>
cudaError_t launch_sponge(const SpongeRec &r, cudaStream_t s);

// Factored solver (adi_factored.cu).
// One line group of a launch, built on the host: lines [first, first + nl) of one simulation
// and direction, with the geometry every thread of the CTA needs; or, for a line with more
// chunks than a CTA has threads, one sub-line: the chunks [c0, c0 + tact) of one line, of
// which it writes the outputs of its own chunks and solves the others (a halo of at least the
// scan reach on each interior side) only to feed its own chunks' windowed scans.
// Copied into shared memory with the group's lines.  Offsets below are in elements.
struct alignas(16) FacGroup {
    int first, nl, N, T;     // first descriptor, lines, cells per line, threads per line
    int tact, hu, tu, mid;   // chunks of the group's range, end-region unknowns, first middle node / cell
    int lp, part, eh, et;    // staged array stride; S/F/H part of the staged record; head / tail table (-1: absent)
    int info, pl, ls, scr;   // scan-reach offset in the staged record, far Dirichlet index, staged line stride, scratch
    double ih, beta;         // 1/h and dt/2 of the simulation
    float ihf, betaf;        // the same in FP32
    unsigned tdiv;           // ceil(2^32 / T) (0 for T = 1): thread / T = umulhi(thread, tdiv)
    int c0;                  // global index of the range's first chunk
    int lo, pn, vn;          // first staged line element; staged pressure/alpha and velocity elements
    int own;                 // bits 0-8 first owned local chunk, 9-17 end of owned local chunks,
                             // bit 18 holds the head region, bit 19 the tail region, bit 20 a split line
    int sp0, sp1, sv0, sv1;  // pressure / velocity outputs stored by bulk copies ([sp0, sp1)); the
                             // group's other owned outputs are stored by the threads that compute them
};
constexpr int kFacOwnHead = 1 << 18, kFacOwnTail = 1 << 19, kFacOwnSplit = 1 << 20;
constexpr int kFacOwnFull = 1 << 21;     // the group's lines reach beyond the scan window: full scans
constexpr int kFacMaxReach = 32;         // longest window of the windowed scans
constexpr int kFacMaxSplit = 8;           // sub-lines of one line at most
constexpr int kFacSplitMaxHalo = 16;      // largest scan reach a split line accepts
FacGroup fac_group_of(int method, int N, int first, int nl, double inv_h, double beta);
bool fac_split_line(int method, int N);  // a line of N cells needs more chunks than a CTA has threads
// The sub-line groups of one split line (descriptor `first`) for scans of reach `halo`;
// returns their count (0: not possible) and the largest stage among them.
int fac_split_groups(int method, int N, int first, int halo, double inv_h, double beta, size_t esz,
                     FacGroup *out, size_t *stage_bytes);
bool fac_supported(int method, int N, size_t esz);  // chunks fit a CTA, stage fits smem
size_t fac_words(int method, int N);     // elements of one line's record
int fac_chunks(int method, int N);       // threads per line
int fac_variant(int method, int N);      // compiled kernel instance: 0 CFD, 1-2 MFD, 3-4 split lines
constexpr int kFacVariants = 5;
int fac_lines_per_cta(int method, int N, size_t esz);
size_t fac_stage_bytes(int method, int N, int nl, size_t esz);  // shared memory of one stage
int fac_stages_for(size_t stage_bytes, size_t esz, int method);  // groups in flight that fit: 3, 2, 1 or 0
size_t fac_ws_doubles();                 // FP64 workspace per line of the precompute
// status[0]: set when a line system is singular; status[1]: atomic max of the lines' scan reach
template <typename T>
cudaError_t launch_fac_precompute(const LineDesc<T> *d, int nlines, double *ws, int *status,
                                  cudaStream_t s);
// Each group takes the windowed or the full scans by its own kFacOwnFull bit, so a line's
// arithmetic does not depend on the other lines of the launch.
template <typename T>
cudaError_t launch_line_solve_factored(const LineDesc<T> *d, const FacGroup *groups, int ngroups,
                                       int variant, size_t stage_bytes, int stages, int grid,
                                       int natural, int *fault, cudaStream_t s);

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
