// Test-only host build of the tensor-core flush's shared-memory operand
// layout (paper_2412_01737_gb300/csrc/ggf_flush_layout.cuh) and of the panel
// index, so that tests can check the producers' index arithmetic without a
// GPU.  Nothing in the library calls it.
#include "../../paper_2412_01737_gb300/csrc/ggf_flush_layout.cuh"

extern "C" {

// For copy slots idx = 0 .. n - 1: the plane element (row, kq), its byte
// offset in the core-matrix layout and its float offset in a chunk-major panel
// with NP padded rows (rank column kq of chunk 0).
void emu_flush_layout(int n, int NP, int* row, int* kq, unsigned* off, unsigned long long* pan) {
    for (int i = 0; i < n; ++i) {
        stage_elem(i, row[i], kq[i]);
        off[i] = cm_off(row[i], kq[i]);
        pan[i] = (unsigned long long)pidx(row[i], kq[i], NP);
    }
}

}

extern "C" {

// Pre-split blocks: for every (chain c < n, pair p, plane, row < NP, rank
// column k < panel_cols(KRM), k a multiple of 4) in that order, the byte
// offsets hi, lo (and hi2, lo2 for the negated U_i copy, else ~0) of its V
// element (uv = 0) and of its U element (uv = 1), as 10 numbers per record
// (c, p, uv, plane, row, k, hi, lo, hi2, lo2).  Returns the number of records.
long long emu_ps_layout(int cplx, int N, int KRM, int pairs, int n, unsigned long long* rec, long long cap) {
    const bool cx = cplx != 0;
    const int NP = panel_rows(N), KP = panel_cols(KRM), planes = cx ? 2 : 1;
    long long m = 0;
    for (int c = 0; c < n; ++c)
        for (int p = 0; p < pairs; ++p)
            for (int uv = 0; uv < 2; ++uv)
                for (int pl = 0; pl < planes; ++pl)
                    for (int row = 0; row < NP; ++row)
                        for (int k = 0; k < KP; k += 4) {
                            if (m >= cap) return -1;
                            size_t hi, lo, hi2 = ~(size_t)0, lo2 = ~(size_t)0;
                            if (uv == 0) ps_vdst(cx, N, KRM, pairs, c, p, pl, row, k, hi, lo);
                            else ps_udst(cx, N, KRM, pairs, n, c, p, pl, row, k, hi, lo, hi2, lo2);
                            unsigned long long* r = rec + 10 * m;
                            r[0] = c; r[1] = p; r[2] = uv; r[3] = pl; r[4] = row; r[5] = k;
                            r[6] = hi; r[7] = lo; r[8] = hi2; r[9] = lo2;
                            ++m;
                        }
    return m;
}

unsigned long long emu_ps_bytes(int cplx, int N, int KRM, int pairs, int n) {
    return ps_bytes(cplx != 0, N, KRM, pairs, n);
}

unsigned long long emu_ps_off(int cplx, int N, int KRM, int pairs, int n, int uv, int c, int p, int b, int kc) {
    return uv == 0 ? ps_voff(cplx != 0, N, KRM, pairs, c, p, b, kc) : ps_uoff(cplx != 0, N, KRM, pairs, n, c, p, b, kc);
}

}
