// Host-only check of the factored solver's split-line geometry: for lines longer than a CTA's
// chunks, every sub-line's range, halo, staged spans, record parts, end tables and output
// spans are checked against the index pattern the kernel reads and writes (CFD: a chunk reads
// nodes jb-1 .. jb+mm; MFD: cells cb .. cb+3mm-1 and velocities cb-2 .. cb+3mm; the end
// windows of the head and tail; bulk copies 16-byte aligned and inside the line or record),
// and the sub-lines together own every chunk and every output exactly once.  Built with nvcc
// and run on the host by tests/test_split_geometry.py; it launches no kernel.
#include "../paper_2006_07583_gb300/csrc/adi_factored.cu"
#include <cstdio>
#include <vector>
using namespace adi;
static int bad = 0;
#define CHECK(c, ...) do { if (!(c)) { if (bad < 40) { printf("FAIL %s:%d: ", #c, __LINE__); printf(__VA_ARGS__); printf("\n"); } ++bad; } } while (0)

int main() {
    for (int method = 0; method < 2; ++method)
        for (int N : {4300, 4500, 5000, 6000, 8192, 8191, 8190, 8189, 10000, 12345, 16384})
            for (int halo : {1, 3, 4, 8, 12, 16})
                for (size_t esz : {(size_t)4, (size_t)8}) {
                    if (!fac_split_line(method, N)) continue;
                    const FacGeom g = fac_geom(method, N);
                    FacGroup sub[kFacMaxSplit];
                    size_t sb = 0;
                    int K = fac_split_groups(method, N, 7, halo, 1.0, 1.0, esz, sub, &sb);
                    if (K == 0) { printf("no split: method %d N %d halo %d esz %zu\n", method, N, halo, esz); continue; }
                    const int MM = g.mm, B2 = g.bs * g.bs, pl = p_last(method, N);
                    const int W = fac_win(method), per = method == 0 ? MM : 3 * MM;
                    const int pg = fac_part(g), es = fac_e_stride(g), recg = fac_rec(g);
                    std::vector<int> pown(pl + 1, 0), vown(N + 1, 0), chunkown(g.tact, 0);
                    CHECK(sb + fac_static_smem(esz, g.bs) <= kFacSmemLimit, "smem");
                    for (int i = 0; i < K; ++i) {
                        const FacGroup &r = sub[i];
                        const bool head = r.own & kFacOwnHead, tail = r.own & kFacOwnTail;
                        const int ol0 = r.own & 511, ol1 = (r.own >> 9) & 511, tl = r.tact;
                        CHECK(r.T <= kFacMaxT && r.T >= tl && r.T % 32 == 0 && tl > 64, "T %d tl %d", r.T, tl);
                        CHECK(r.c0 % 4 == 0 && r.lo % 4 == 0 && r.lp % 4 == 0 && r.part % 4 == 0, "align");
                        CHECK(r.c0 + tl <= g.tact && ol0 >= 0 && ol1 <= tl && ol0 < ol1, "range");
                        CHECK(head == (r.c0 == 0) && tail == (r.c0 + tl == g.tact), "head/tail");
                        // halo on each interior side at least `halo`
                        if (!head) CHECK(ol0 >= halo, "halo lo %d", ol0);
                        if (!tail) CHECK(tl - ol1 >= halo, "halo hi %d", tl - ol1);
                        for (int c = ol0; c < ol1; ++c) chunkown[r.c0 + c]++;
                        // staged spans cover every read
                        auto inP = [&](int k) { return k >= r.lo && k < r.lo + r.pn && k - r.lo < r.lp; };
                        auto inV = [&](int k) { return k >= r.lo && k < r.lo + r.vn && k - r.lo < r.lp; };
                        CHECK(r.lo + r.pn <= pl + 1 + 3 && r.lo + r.vn <= N + 1 + 3, "span end");
                        CHECK(fac_ru4(r.lo + r.pn) <= fac_ru4(pl + 1) && fac_ru4(r.lo + r.vn) <= fac_ru4(N + 1), "copy end");
                        for (int c = 0; c < tl; ++c) {
                            const int cg = r.c0 + c;
                            if (method == 0) {
                                const int jb = r.mid + cg * MM;
                                for (int k = jb - 1; k <= jb + MM; ++k) { CHECK(inP(k) && inV(k), "cfd read %d c %d", k, c); }
                            } else {
                                const int cb = r.mid + 3 * cg * MM;
                                for (int k = cb; k < cb + 3 * MM; ++k) CHECK(inP(k), "mfd p read %d", k);
                                for (int k = cb - 2; k <= cb + 3 * MM; ++k) CHECK(inV(k), "mfd v read %d", k);
                            }
                        }
                        if (head) { for (int k = 0; k < W; ++k) CHECK(inP(k) && inV(k), "head window"); CHECK(r.eh >= 0, "eh"); }
                        if (tail) {
                            for (int k = pl + 1 - W; k <= pl; ++k) CHECK(inP(k), "tail p window %d", k);
                            for (int k = N + 1 - W; k <= N; ++k) CHECK(inV(k), "tail v window %d", k);
                            CHECK(r.et >= 0, "et");
                        }
                        // record parts inside the global record
                        const size_t cs = (size_t)r.c0 * B2;
                        CHECK(cs + r.part <= (size_t)pg, "S part");
                        CHECK(2 * (size_t)pg + cs + r.part <= 3 * (size_t)pg, "H part");
                        CHECK((cs * esz) % 16 == 0 && (r.part * esz) % 16 == 0 && (es * esz) % 16 == 0, "rec align");
                        CHECK(3 * pg + 2 * es + 4 == recg, "rec size");
                        CHECK(r.info + 4 + 3 * r.lp <= r.scr && r.scr + fac_scratch(g) == r.ls, "layout");
                        // outputs: owned chunks plus end regions; stored spans inside them
                        int p0 = head ? 0 : r.mid + (r.c0 + ol0) * per, p1 = tail ? pl + 1 : r.mid + (r.c0 + ol1) * per;
                        int vs = method == 0 ? 0 : 1;
                        int v0 = head ? 0 : r.mid + (r.c0 + ol0) * per + vs, v1 = tail ? N + 1 : r.mid + (r.c0 + ol1) * per + vs;
                        for (int k = p0; k < p1; ++k) pown[k]++;
                        for (int k = v0; k < v1; ++k) vown[k]++;
                        CHECK(r.sp0 >= p0 && r.sp1 <= (tail ? pl + 1 : p1) && r.sp0 % 4 == 0 && (tail || r.sp1 % 4 == 0), "sp");
                        CHECK(r.sv0 >= v0 && r.sv1 <= (tail ? N + 1 : v1) && r.sv0 % 4 == 0 && (tail || r.sv1 % 4 == 0), "sv");
                        CHECK(r.sp0 >= r.lo && fac_ru4(r.sp1) <= r.lo + r.lp, "sp staged");
                        CHECK(r.sv0 >= r.lo && fac_ru4(r.sv1) <= r.lo + r.lp, "sv staged");
                        // direct-stored elements lie in the first or last owned chunk
                        const int fp0 = r.mid + (r.c0 + ol0) * per, fp1 = r.mid + (r.c0 + ol1 - 1) * per;
                        for (int k = p0; k < p1; ++k)
                            if (k < r.sp0 || k >= r.sp1) CHECK((k >= fp0 && k < fp0 + per) || (k >= fp1 && k < fp1 + per), "direct p %d", k);
                        for (int k = v0; k < v1; ++k)
                            if (k < r.sv0 || k >= r.sv1) CHECK((k >= fp0 + vs && k < fp0 + per + vs) || (k >= fp1 + vs && k < fp1 + per + vs), "direct v %d", k);
                    }
                    for (int c = 0; c < g.tact; ++c) CHECK(chunkown[c] == 1, "chunk %d owned %d times", c, chunkown[c]);
                    for (int k = 0; k <= pl; ++k) CHECK(pown[k] == 1, "p %d owned %d", k, pown[k]);
                    for (int k = 0; k <= N; ++k) CHECK(vown[k] == 1, "v %d owned %d", k, vown[k]);
                }
    // every line length: a supported line fits the CTA (threads, shared memory) as a whole
    // line or as sub-lines, and its end regions fit their tables
    for (int method = 0; method < 2; ++method)
        for (int N = ADI_MIN_CELLS; N <= ADI_MAX_CELLS; N += (N < 600 ? 1 : 37))
            for (size_t esz : {(size_t)4, (size_t)8}) {
                if (!fac_supported(method, N, esz)) continue;
                const FacGeom g = fac_geom(method, N);
                CHECK(g.hu <= g.hmax && g.tu <= g.hmax && g.tact >= 1, "ends N %d", N);
                CHECK(g.nb == g.tact * g.mm, "blocks N %d", N);
                if (!fac_split_line(method, N)) {
                    const int nl = fac_lines_per_cta(method, N, esz);
                    CHECK(nl >= 1 && nl * g.T <= kFacMaxT, "lines per CTA N %d", N);
                    const size_t sb = fac_stage_bytes(method, N, nl, esz);
                    CHECK(fac_stages_for(sb, esz, method) >= 1, "stage N %d", N);
                    CHECK((size_t)fac_stages_for(sb, esz, method) * sb + fac_static_smem(esz, g.bs) <= kFacSmemLimit, "smem N %d", N);
                } else {
                    FacGroup sub[kFacMaxSplit];
                    size_t sb = 0;
                    const int K = fac_split_groups(method, N, 0, kFacSplitMaxHalo, 1.0, 1.0, esz, sub, &sb);
                    CHECK(K >= 2, "split N %d", N);
                    CHECK((size_t)fac_stages_for(sb, esz, method) * sb + fac_static_smem(esz, g.bs) <= kFacSmemLimit, "split smem N %d", N);
                }
            }
    printf("bad %d\n", bad);
    return bad != 0;
}
