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
