// Host-only check of the prologue's Thomas factors (prologue_factors): for several line
// lengths, P x = b and Pbar x = b solved with the stored factors agree with a dense Gaussian
// elimination of the same App. A matrices, assembled from their row functions -- both as one
// elimination over the whole line and as the chunked, halo-truncated elimination the prologue
// kernel runs (prologue_win_solve, called here on the host for every chunk), which must cover
// every row once and agree to 1e-13.  Built with nvcc and run on the host by
// tests/test_split_geometry.py; it launches no kernel.
#include "../paper_2006_07583_gb300/csrc/adi_kernels.cu"
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>
using namespace adi;

static std::vector<double> dense_solve(std::vector<double> A, std::vector<double> b, int n) {
    for (int k = 0; k < n; ++k) {  // partial pivoting
        int p = k;
        for (int i = k + 1; i < n; ++i)
            if (std::fabs(A[i * n + k]) > std::fabs(A[p * n + k])) p = i;
        if (p != k) {
            for (int j = 0; j < n; ++j) std::swap(A[k * n + j], A[p * n + j]);
            std::swap(b[k], b[p]);
        }
        for (int i = k + 1; i < n; ++i) {
            const double m = A[i * n + k] / A[k * n + k];
            for (int j = k; j < n; ++j) A[i * n + j] -= m * A[k * n + j];
            b[i] -= m * b[k];
        }
    }
    std::vector<double> x(n);
    for (int i = n - 1; i >= 0; --i) {
        double s = b[i];
        for (int j = i + 1; j < n; ++j) s -= A[i * n + j] * x[j];
        x[i] = s / A[i * n + i];
    }
    return x;
}

int main() {
    int bad = 0;
    for (int N : {16, 17, 31, 64, 65, 95, 96, 97, 100, 127, 128, 129, 257, 1001}) {
        std::vector<double> f;
        prologue_factors(N, f);
        for (int bar = 0; bar < 2; ++bar) {
            const int n = bar ? N - 1 : N + 1;
            std::vector<double> A((size_t)n * n, 0.0), b(n);
            for (int r = 0; r < n; ++r) {
                double w[8];
                int c0 = 0;
                const int len = bar ? cfd_Pbar_row(N, r + 1, &c0, w) : cfd_P_row(N, r, &c0, w);
                for (int i = 0; i < len; ++i) A[(size_t)r * n + (bar ? c0 - 1 : c0) + i] = w[i];
                b[r] = std::sin(0.37 * r + 0.1 * N) + 0.5;
            }
            const std::vector<double> xd = dense_solve(A, b, n);
            const double *lo = f.data() + (bar ? 3 * (N + 1) : 0), *cu = lo + n, *id = cu + n;
            std::vector<double> x(b);
            double d = x[0] * id[0];
            x[0] = d;
            for (int r = 1; r < n; ++r) { d = (x[r] - lo[r] * d) * id[r]; x[r] = d; }
            double xv = d;
            for (int r = n - 2; r >= 0; --r) { xv = x[r] - cu[r] * xv; x[r] = xv; }
            double err = 0.0, nrm = 0.0;
            for (int r = 0; r < n; ++r) { err = std::fmax(err, std::fabs(x[r] - xd[r])); nrm = std::fmax(nrm, std::fabs(xd[r])); }
            if (!(err <= 1e-13 * nrm)) { printf("FAIL N %d bar %d err %g\n", N, bar, err); ++bad; }
            // the chunked elimination of the kernel
            const double *su_id = f.data() + 3 * (N + 1) + 3 * (N - 1);
            std::vector<double> tmp(n, 0.0), xc(n, 0.0);
            std::vector<int> hits(n, 0);
            for (int r0 = 0; r0 < n; r0 += kProR) {
                const int r1 = std::min(n, r0 + kProR);
                prologue_win_solve<double>(n, r0, r1, [&](int r) { return b[r]; }, lo, cu, id, su_id, tmp.data(), 1,
                                           [&](int r, double v) { xc[r] = v; ++hits[r]; });
            }
            double errc = 0.0;
            for (int r = 0; r < n; ++r) {
                errc = std::fmax(errc, std::fabs(xc[r] - xd[r]));
                if (hits[r] != 1) { printf("FAIL N %d bar %d row %d written %d times\n", N, bar, r, hits[r]); ++bad; }
            }
            if (!(errc <= 1e-13 * nrm)) { printf("FAIL chunked N %d bar %d err %g\n", N, bar, errc); ++bad; }
        }
    }
    printf("bad %d\n", bad);
    return bad != 0;
}
