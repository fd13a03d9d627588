// Shared-memory operand layout of the tensor-core flush (k_flush_tc.cu): the
// stage planes that the producer warps fill and the MMAs read.  Host and
// device, so that the index arithmetic can be checked without a GPU.
#pragma once
#include <cstdint>
#include "ggf_common.cuh"

namespace {

constexpr int KC = 8;                         // rank columns per stage (one MMA K step)
constexpr int SBO = KC / 4 * 128;             // bytes between 8-row core-matrix groups

// Byte offset of (row, k) inside a K-major no-swizzle operand plane (KC wide):
// 8-row x 16-byte core matrices, 128 bytes apart along K, SBO bytes apart
// between 8-row groups.
GGF_HD uint32_t cm_off(int row, int k) {
    return (uint32_t)((row >> 3) * SBO + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

// Element of a stage plane handled by copy slot idx: row (idx & 7) + 8 (idx >> 4),
// rank columns 4 ((idx >> 3) & 1) .. + 3.  Each 8-thread phase of a warp's
// 16-byte stores then fills one 128-byte run of the core-matrix layout (8 rows
// of one column group), free of bank conflicts; pairing the two column groups
// of a row in neighbouring threads put them 128 bytes apart, on the same banks
// (a 2-way conflict on every split store).  A warp still reads 16 whole rows of
// the chunk-major panel, four 128-byte lines.
GGF_HD void stage_elem(int idx, int& row, int& kq) {
    row = (idx & 7) | ((idx >> 4) << 3);
    kq = 4 * ((idx >> 3) & 1);
}

}  // namespace

// ---- pre-split operand blocks (flush in waves of chains) ---------------------
//
// Before a wave of chains is flushed, every operand value is split once into
// tf32 hi/lo and written to a scratch array in blocks that hold exactly the
// bytes of one stage's V part or U part, in the core-matrix layout above, so
// that one bulk copy per part fills a stage.  Per (chain of the wave, pair,
// row block, rank chunk of KC columns):
//   real pairs     V block  128 rows: [hi 4 KB][lo 4 KB]
//                  U block  256 rows: [hi 8 KB][lo 8 KB]
//   complex pairs  V block  128 rows: [V_r hi][V_r lo][V_i hi][V_i lo] (4 KB each)
//                  U block  128 rows: [hi 12 KB][lo 12 KB], each the composite
//                  [-U_i ; U_r ; U_i] (384 rows) that the complex MMAs read.
// Rows past N and rank columns past the chain's pending rank hold zeros.  The
// scratch is [all V blocks of the wave][all U blocks of the wave], V blocks
// indexed (((chain * pairs + pair) * NP / 128 + block) * chunks + chunk).

constexpr int PS_PLANE = 128 * KC * 4;        // 4 KB: 128 rows x KC tf32

GGF_HD constexpr int ps_urows(bool cplx) { return cplx ? 128 : 256; }
GGF_HD constexpr int ps_vbytes(bool cplx) { return cplx ? 4 * PS_PLANE : 2 * PS_PLANE; }
GGF_HD constexpr int ps_ubytes(bool cplx) { return cplx ? 2 * 3 * PS_PLANE : 2 * 2 * PS_PLANE; }
GGF_HD int ps_chunks(int KRM) { return panel_cols(KRM) / KC; }

// bytes of the V region and of the whole scratch for n chains
GGF_HD size_t ps_vregion(bool cplx, int N, int KRM, int pairs, int n) {
    return (size_t)n * pairs * (panel_rows(N) / 128) * ps_chunks(KRM) * ps_vbytes(cplx);
}
GGF_HD size_t ps_bytes(bool cplx, int N, int KRM, int pairs, int n) {
    return ps_vregion(cplx, N, KRM, pairs, n) +
           (size_t)n * pairs * (panel_rows(N) / ps_urows(cplx)) * ps_chunks(KRM) * ps_ubytes(cplx);
}

// byte offset of the V block (chain c of the wave, pair p, 128-row block jb,
// chunk kc) and of the U block (row block ib of ps_urows rows)
GGF_HD size_t ps_voff(bool cplx, int N, int KRM, int pairs, int c, int p, int jb, int kc) {
    return ((((size_t)c * pairs + p) * (panel_rows(N) / 128) + jb) * ps_chunks(KRM) + kc) * ps_vbytes(cplx);
}
GGF_HD size_t ps_uoff(bool cplx, int N, int KRM, int pairs, int n, int c, int p, int ib, int kc) {
    return ps_vregion(cplx, N, KRM, pairs, n) +
           ((((size_t)c * pairs + p) * (panel_rows(N) / ps_urows(cplx)) + ib) * ps_chunks(KRM) + kc) *
               ps_ubytes(cplx);
}

// Where the split pass writes element (row, k) of a plane (k < panel_cols):
// the byte offsets of its hi and lo copies in the V block (plane 0 = V_r or
// the real V, 1 = V_i) and in the U block (plane 0 = U or U_r, 1 = U_i; for
// U_i also the negated copy, returned in hi2/lo2, else ~0).
GGF_HD void ps_vdst(bool cplx, int N, int KRM, int pairs, int c, int p, int plane, int row, int k, size_t& hi,
                    size_t& lo) {
    const size_t b = ps_voff(cplx, N, KRM, pairs, c, p, row / 128, k / KC);
    const uint32_t o = cm_off(row % 128, k % KC);
    hi = b + (size_t)(2 * plane) * PS_PLANE + o;
    lo = hi + PS_PLANE;
}
GGF_HD void ps_udst(bool cplx, int N, int KRM, int pairs, int n, int c, int p, int plane, int row, int k, size_t& hi,
                    size_t& lo, size_t& hi2, size_t& lo2) {
    const int ur = ps_urows(cplx);
    const size_t b = ps_uoff(cplx, N, KRM, pairs, n, c, p, row / ur, k / KC);
    const size_t half = (size_t)(cplx ? 3 : 2) * PS_PLANE;         // hi part bytes
    const int r = row % ur;
    hi2 = lo2 = ~(size_t)0;
    if (!cplx) {
        hi = b + cm_off(r, k % KC);
    } else if (plane == 0) {
        hi = b + cm_off(128 + r, k % KC);                            // U_r: composite rows 128..255
    } else {
        hi = b + cm_off(256 + r, k % KC);                            // U_i: rows 256..383
        hi2 = b + cm_off(r, k % KC);                                 // -U_i: rows 0..127
        lo2 = hi2 + half;
    }
    lo = hi + half;
}
