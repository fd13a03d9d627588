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
