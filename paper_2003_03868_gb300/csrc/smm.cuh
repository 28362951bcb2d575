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

// Launch configuration of one (m, n) shape.  tpb, ctas_per_sm, colmajor and prefetch2 leave
// the arithmetic unchanged (every C element is summed in the same order); split picks the
// kernel's work split per C block and changes only the rounding order: of the block norm
// (warp pair) or of one remainder element (K-split).
constexpr int kSplitDefault = -1;   // K-split where m n = 32 EF + 1, else a pair from 6 slots per lane
constexpr int kSplitWarp = 0;       // one warp per C block
constexpr int kSplitPair = 1;       // two warps per C block, half of the element slots each (m n > 32)
constexpr int kSplitK = 2;          // 32 EF elements over the lanes, the last one summed along K (m n = 32 EF + 1)
struct TuneCfg {
    int tpb = 256;           // threads per CTA (multiple of 32, <= 256)
    int ctas_per_sm = 32;    // grid = min(warps needed / warps per CTA, (SM count) * ctas_per_sm)
    int colmajor = 0;        // lane -> element order
    int prefetch2 = 0;       // fetch the next 32 products' metadata ahead
    int split = kSplitDefault;
};

TuneCfg default_cfg(int prec);
// Tuned configuration for (prec, m, n, k), or the default when the table has none.
TuneCfg tune_lookup(int prec, int m, int n, int k);
// Configurations the tuner times (FP64; the tensor-core tier has no per-shape kernels).
std::vector<TuneCfg> tune_space(int prec);
// Whether cfg applies to m x n blocks, and the work split it resolves to.
bool cfg_valid(int m, int n, const TuneCfg& c);
int resolve_split(int m, int n, const TuneCfg& c);

// Features of one (m, n, k, configuration) sample for the prediction model.
void mlp_features(int prec, int m, int n, int k, const TuneCfg& c, float* f);

inline bool is_bf16(int prec) { return prec == DBCSR_BF16 || prec == DBCSR_BF16X3; }

// Launches the FP64 kernel of shape (m, n) over the cnt blocks listed in list.
void launch_smm_shape(int m, int n, int64_t cnt, const int64_t* list, const SmmArgs& sa, const TuneCfg& cfg,
                      cudaStream_t s);

}  // namespace dbg
