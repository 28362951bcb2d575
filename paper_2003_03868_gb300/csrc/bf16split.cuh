// FP64 -> BF16 rounding (round to nearest, ties to even, from the IEEE-754 encodings with
// integer operations) and the split x = hi + lo of the split-BF16 operands (hi = bf16(x),
// lo = bf16(x - hi)).  Host and device: the packing kernel of the tensor-core tier uses it, and
// a host build lets a CPU test compare it bit for bit with the rounding's definition.
#pragma once

#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define BF16_HD __host__ __device__ __forceinline__
#else
#define BF16_HD inline
#endif

namespace dbg {

BF16_HD uint64_t bf16_f64_bits(double x) {
#ifdef __CUDA_ARCH__
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t u;
    std::memcpy(&u, &x, sizeof u);
    return u;
#endif
}

// binary32's range: values below its normal range become signed zero, values rounding past
// its largest finite value infinity; NaN stays NaN.
BF16_HD uint16_t bf16_bits(double x) {
    const uint64_t u = bf16_f64_bits(x);
    const uint16_t sign = (uint16_t)((u >> 48) & 0x8000u);
    const int e = (int)((u >> 52) & 0x7ff);
    if (e == 0x7ff) return (uint16_t)(sign | 0x7f80u | ((u & 0xfffffffffffffull) ? 0x40u : 0u));
    const int eb = e - 1023 + 127;               // biased binary32 exponent
    if (eb < 1) return sign;                     // below the normal range
    const uint64_t mant = u & 0xfffffffffffffull;    // 52 bits; keep 7
    const uint64_t keep = mant >> 45, rest = mant & ((1ull << 45) - 1);
    const uint64_t half = 1ull << 44;
    uint32_t m7 = (uint32_t)keep;
    int ex = eb;
    if (rest > half || (rest == half && (m7 & 1u))) {
        if (++m7 == 128u) {
            m7 = 0;
            ++ex;
        }
    }
    if (ex >= 255) return (uint16_t)(sign | 0x7f80u);
    return (uint16_t)(sign | ((uint32_t)ex << 7) | m7);
}

BF16_HD double bf16_value(uint16_t b) {
    const uint32_t w = (uint32_t)b << 16;
    float f;
#ifdef __CUDA_ARCH__
    f = __uint_as_float(w);
#else
    std::memcpy(&f, &w, sizeof f);
#endif
    return (double)f;
}

// hi = bf16(x) and lo = bf16(x - hi); x - hi is exact in FP64 (hi is x's significand rounded
// to 8 bits), so lo is the rounding of the exact remainder.
BF16_HD void bf16_split(double x, uint16_t& hi, uint16_t& lo) {
    hi = bf16_bits(x);
    lo = bf16_bits(x - bf16_value(hi));
}

}  // namespace dbg
