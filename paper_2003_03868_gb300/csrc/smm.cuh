// Internal interface of the batched block-product kernels: their arguments, the
// runtime launch configuration the tuner chooses among, and the launcher.
#pragma once

#include <cuda_bf16.h>

#include <vector>

#include "common.cuh"

namespace dbg {

// Arguments of one batched block-product launch: C block k = (f_row[k], f_col[k])
// at c_data + f_off[k] sums the products f_pbeg[k] .. f_pbeg[k+1]-1, product p
// being A block prod_a[p] (inner size bs[a_col[prod_a[p]]]) times B block prod_b[p].
struct SmmArgs {
    const int32_t* f_row; const int32_t* f_col; const int64_t* f_off; const int64_t* f_pbeg; const int64_t* f_cin;
    const int32_t* prod_a; const int32_t* prod_b;
    const int32_t* a_col; const int64_t* a_off; const double* a_data;
    const int64_t* b_off; const double* b_data;
    const int64_t* ci_off; const double* ci_data;
    const int32_t* bs;
    double alpha, beta;
    double* c_data; double* c_norm; double* c_dev2;
    int colmajor;    // lane -> element order: 0 row-major (i = idx / n), 1 column-major (i = idx % m)
    int prefetch2;   // 1: fetch the next 32 products' metadata before using the current ones
};

// Launch configuration of one (m, n) shape; none of it changes the arithmetic
// (every C element is summed in the same order whatever the configuration).
struct TuneCfg {
    int tpb = 256;           // threads per CTA (multiple of 32, <= 256)
    int ctas_per_sm = 32;    // grid = min(warps needed / warps per CTA, (SM count) * ctas_per_sm)
    int colmajor = 0;        // FP64 only
    int prefetch2 = 0;       // FP64 only
};

TuneCfg default_cfg(int prec);
// Tuned configuration for (prec, m, n, k), or the default when the table has none.
TuneCfg tune_lookup(int prec, int m, int n, int k);
// Legal configurations the tuner times for a precision.
std::vector<TuneCfg> tune_space(int prec);

// Features of one (m, n, k, configuration) sample for the prediction model.
void mlp_features(int prec, int m, int n, int k, const TuneCfg& c, float* f);

// Fragment-ready BF16 copies of the operands (BF16 products only): block b of A
// at a16 + a_po[b] (m x k padded to 16-multiples), block b of B transposed at
// b16 + b_po[b] (n x k padded to 8 x 16-multiples).  Each block takes its own
// padded size, so mixed block sizes waste no slots.
struct Bf16Packs {
    const __nv_bfloat16* a16 = nullptr;
    const int64_t* a_po = nullptr;
    const __nv_bfloat16* b16 = nullptr;
    const int64_t* b_po = nullptr;
    const __nv_bfloat16* a16_lo = nullptr;   // DBCSR_BF16X3: the residuals lo = bf16(x - hi), same offsets
    const __nv_bfloat16* b16_lo = nullptr;
};
inline bool is_bf16(int prec) { return prec == DBCSR_BF16 || prec == DBCSR_BF16X3; }
// Packed tile size (elements) of an r x c block in a role (0: A, m x k; 1: B, k x n stored n x k).
__host__ __device__ inline int64_t pack_size(int role, int r, int c) {
    return role == 0 ? (int64_t)(16 * ((r + 15) / 16)) * (16 * ((c + 15) / 16))
                     : (int64_t)(8 * ((c + 7) / 8)) * (16 * ((r + 15) / 16));
}

// Launches the kernel of shape (m, n) over the cnt blocks listed in list.
void launch_smm_shape(int prec, int m, int n, int64_t cnt, const int64_t* list, const SmmArgs& sa,
                      const Bf16Packs& pk, const TuneCfg& cfg, cudaStream_t s);

}  // namespace dbg
