// Schedule of the grouped tcgen05 launch (written by batched.cu, read by the
// kernel in gemm_tc_tcgen05.cu).  The operands of its problems -- raw e4m3
// residues for p < 16, centred fp16 otherwise -- are stacked, K-major, as
// bytes in a few arrays: one per k-stride bin (128 2^b bytes per row), A rows
// and B^T rows of a problem in the same array, one byte-typed tensor map per
// array.  A problem is then a bin, a kind and two row offsets; only its first
// k elements (rounded up to 32 bytes) of each row are written.
#pragma once

#include <cstdint>

namespace gfp {

constexpr int TC_GROUP_BINS = 10;            // row strides 128 .. 65536 bytes

struct alignas(64) TcGroupProblem {          // 64 bytes
    uint8_t *C;
    int64_t ldc;
    int32_t m, n;
    int32_t rowA0, rowB0;                    // first row of A and of B^T in the bin's array
    int32_t ktiles;                          // k in 128-byte slices
    int16_t bin;                             // stride bin (tensor map index)
    int8_t kind;                             // 0: raw e4m3 (kind::f8f6f4), 1: centred fp16 (kind::f16);
                                             // the kernel tells them apart by `scale`
    int8_t sym;                              // 1: B = A^T, so C = A A^T is symmetric; the schedule
                                             // holds the tiles tn >= tm only and the epilogue also
                                             // writes each tile with tn > tm transposed at (tn, tm)
    uint32_t p, off;                         // off: 0 (raw products are non-negative)
    float scale;                             // 2^18 (raw e4m3), 1 (fp16)
    uint32_t m32;                            // ceil(2^32 / p)
    int32_t klast;                           // 32-wide MMAs in the last k slice (1-4)
    int32_t red;                             // 1: every sum < 2^23 units (mantissa read)
};
static_assert(sizeof(TcGroupProblem) == 64, "layout");

struct TcGroupItem {
    int32_t prob;
    uint16_t tm, tn;
};

struct alignas(64) TcGroupHeader {
    int32_t count, items, grid, nmaps;
    int64_t off_probs, off_items, off_ranges, off_maps;   // byte offsets from the header
};
static_assert(sizeof(TcGroupHeader) == 64, "layout");

}  // namespace gfp
