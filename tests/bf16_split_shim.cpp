// Host build of the library's FP64 -> BF16 rounding and split, for the CPU test that compares
// them bit for bit with the rounding's definition in the oracle (test infrastructure).
#include <cstdint>

#include "bf16split.cuh"

extern "C" void bf16_split_many(const double* x, int64_t n, uint16_t* hi, uint16_t* lo) {
    for (int64_t i = 0; i < n; ++i) dbg::bf16_split(x[i], hi[i], lo[i]);
}

extern "C" void bf16_round_many(const double* x, int64_t n, uint16_t* b) {
    for (int64_t i = 0; i < n; ++i) b[i] = dbg::bf16_bits(x[i]);
}
