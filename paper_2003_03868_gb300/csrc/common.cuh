// Shared declarations of the GB300 block-sparse library: error plumbing,
// stream-ordered device buffers, the matrix object and internal entry points.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <cstring>
#include <functional>
#include <memory>
#include <stdexcept>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "dbcsr_gb.h"

namespace dbg {

// Largest block edge the kernels accept (atom blocks of the workloads are <= 23).
constexpr int kMaxBlock = 32;

// Host work split over threads: f(chunk, begin, end) over [0, n) in up to 16 contiguous chunks
// (one chunk below 2^18 items); chunk c always covers the same range for a given n, so
// results that are combined in chunk order are deterministic.  Returns the chunk count.
template <class F>
int host_chunks(int64_t n, F&& f) {
    const int hw = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    const int nt = n < (1 << 18) ? 1 : hw;
    const int64_t per = (n + nt - 1) / nt;
    std::vector<std::thread> th;
    for (int c = 1; c < nt; ++c)
        th.emplace_back([&, c] { f(c, std::min(n, c * per), std::min(n, (c + 1) * per)); });
    f(0, 0, std::min(n, per));
    for (auto& t : th) t.join();
    return nt;
}

struct Error : std::runtime_error {
    dbcsr_status code;
    Error(dbcsr_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};

[[noreturn]] void fail(dbcsr_status code, const std::string& msg);
void set_last_error(const std::string& msg);
extern std::atomic<int64_t> g_launches;

#define DBG_CK(call)                                                                        \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            if (e_ == cudaErrorMemoryAllocation) {                                          \
                (void)cudaGetLastError();                                                   \
                ::dbg::fail(DBCSR_ENOMEM, std::string(#call) + ": " + cudaGetErrorString(e_)); \
            }                                                                               \
            ::dbg::fail(DBCSR_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
        }                                                                                   \
    } while (0)

// Every kernel launch site is followed by DBG_LAUNCH_CK(): it checks the launch
// and counts it (dbcsr_launch_count).
#define DBG_LAUNCH_CK()                                                                          \
    do {                                                                                         \
        ::dbg::g_launches.fetch_add(1, std::memory_order_relaxed);                               \
        cudaError_t e_ = cudaGetLastError();                                                     \
        if (e_ != cudaSuccess)                                                                   \
            ::dbg::fail(e_ == cudaErrorMemoryAllocation ? DBCSR_ENOMEM : DBCSR_ECUDA,            \
                        std::string("kernel launch at ") + __FILE__ + ":" + std::to_string(__LINE__) + \
                            ": " + cudaGetErrorString(e_));                                      \
    } while (0)

// Sets kernel's dynamic shared-memory limit to dyn bytes before a launch that asks for them.
// The default limit (48 KB) covers static and dynamic shared memory together, so a launch
// just under 48 KB of dynamic memory fails too when the kernel has static arrays; the
// attribute is therefore set for every nonzero request.
template <class K>
inline void allow_dyn_smem(K kernel, size_t dyn) {
    if (dyn > 0) DBG_CK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
}

// The library's stream-ordered memory pool on the current device.  It keeps freed
// memory cached (release threshold = max) so that the per-product stacks and
// matrices are not unmapped at every host synchronisation and mapped again.
cudaMemPool_t library_pool();
// Waits for the device, then returns cached pool memory above keep_bytes to the driver.
void trim_pool(uint64_t keep_bytes);
// Stream-ordered allocation from library_pool().  When the device is out of memory the
// cached free memory is returned to the driver (after the device is idle) and the
// allocation is tried once more; a second failure throws DBCSR_ENOMEM.
void pool_alloc(void** p, size_t bytes, cudaStream_t s);

// Device array allocated and freed in stream order from library_pool().
template <class T>
struct DBuf {
    T* p = nullptr;
    int64_t n = 0;
    cudaStream_t s = nullptr;

    DBuf() = default;
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
    DBuf(DBuf&& o) noexcept : p(o.p), n(o.n), s(o.s) { o.p = nullptr; o.n = 0; }
    DBuf& operator=(DBuf&& o) noexcept {
        if (this != &o) {
            release();
            p = o.p; n = o.n; s = o.s;
            o.p = nullptr; o.n = 0;
        }
        return *this;
    }
    ~DBuf() { release(); }

    void alloc(int64_t count, cudaStream_t stream) {
        release();
        s = stream;
        n = count;
        if (count > 0) pool_alloc((void**)&p, sizeof(T) * (size_t)count, stream);
    }
    void zero() {
        if (n > 0) DBG_CK(cudaMemsetAsync(p, 0, sizeof(T) * (size_t)n, s));
    }
    void release() noexcept {
        if (p) cudaFreeAsync(p, s);
        p = nullptr;
        n = 0;
    }
};

// Pinned host scratch for small device->host readbacks.
struct HostScalars {
    static constexpr int kCap = 256;
    int64_t* i = nullptr;
    double* d = nullptr;
    HostScalars();
    ~HostScalars();
};
HostScalars& host_scalars();

// Groups of block rows (= block columns) read as one dense tile by the tensor-core tier
// (lowtier.cu): at most kGroupWidth rows and kGroupMembers blocks per group.
constexpr int kGroupWidth = 112;
constexpr int kGroupMembers = 16;
constexpr int32_t kMaxBlockRowsLt = 262144;
struct Groups {
    int32_t ngrp = 0, nblk = 0, max_members = 0;
    std::vector<int32_t> h_w;            // host copy of the widths
    DBuf<int32_t> g_of;                  // [nblk] group of every block
    DBuf<int32_t> g_pos;                 // [nblk] first row of the block inside its group
    DBuf<int32_t> g_ptr;                 // [ngrp + 1] members of group k: g_mem[g_ptr[k] .. g_ptr[k+1])
    DBuf<int32_t> g_mem;                 // [nblk] blocks in ascending order per group
    DBuf<int32_t> g_w;                   // [ngrp] rows of every group
    DBuf<int32_t> g_mrec;                // [nblk] per member slot (g_mem order): first row | rows << 8
    DBuf<int32_t> g_midx;                // [nblk] member index of every block inside its group
};

}  // namespace dbg

// The matrix object behind the opaque C handle.
struct dbcsr_matrix_ {
    int32_t nblk = 0;
    int64_t n = 0;                       // matrix dimension = sum of block edges
    cudaStream_t stream = nullptr;
    std::vector<int32_t> h_bs;           // host copy of the block edges
    dbg::DBuf<int32_t> bs;               // [nblk] block edges
    bool finalized = false;

    // block-CSR on the device
    int64_t nnzb = 0, nel = 0;
    dbg::DBuf<int64_t> rp;               // [nblk + 1] row pointers
    dbg::DBuf<int32_t> col;              // [nnzb] block column, ascending per row
    dbg::DBuf<int32_t> row;              // [nnzb] block row of each block
    dbg::DBuf<int64_t> off;              // [nnzb + 1] element offset of each block in data
    dbg::DBuf<double> data;              // [nel] blocks row-major, packed in CSR order
    dbg::DBuf<double> norms;             // [nnzb] Frobenius norms (valid iff norms_valid)
    bool norms_valid = false;

    int plans = 0;                       // live multiply plans that use this matrix's arrays

    // groups of blocks for the tensor-core tier: computed from this matrix (or inherited from
    // the operand of the product that formed it) at its first BF16 product; any partition
    // gives the same products, the groups only decide how dense the tiles are
    std::shared_ptr<dbg::Groups> groups;

    // staging area of put_block(s) before finalize
    std::vector<int32_t> st_row, st_col;
    std::vector<int64_t> st_src;         // element offset of each staged block in st_dev
    dbg::DBuf<double> st_dev;
    int64_t st_dev_used = 0;
};

namespace dbg {

// ---- scan.cu
// out[0..n] = exclusive prefix sum of in[0..n-1]; out[n] = total.  n >= 0.
void scan_exclusive(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s);
void scan_exclusive(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s);
// Deterministic sum of v[0..n-1] into *out (device); fixed reduction tree for a given n.
void det_sum(const double* v, int64_t n, double* out, cudaStream_t s);
// The same sum with a caller-given buffer of kDetSumPartials doubles for the per-CTA partials.
constexpr int kDetSumPartials = 1024;
void det_sum_into(const double* v, int64_t n, double* partials, double* out, cudaStream_t s);

// ---- matrix.cu
void check_finalized(const dbcsr_matrix_* m);
void ensure_norms(dbcsr_matrix_* m);
void compute_block_norms(const dbcsr_matrix_* m, double* norms, double* dev2);
void copy_matrix(dbcsr_matrix_* dst, const dbcsr_matrix_* src);
void scale_shift(dbcsr_matrix_* m, double scale, double shift);
// Keeps the blocks whose flag is nonzero (norms, when given, are compacted too).
void compact(dbcsr_matrix_* m, const int32_t* keep, const double* norms_in);
void filter_matrix(dbcsr_matrix_* m, double eps, const double* norms_in);
int64_t read_i64(const int64_t* dev, cudaStream_t s);
// Reads k scalars and, optionally, one contiguous array of na values, with one synchronisation.
void read_i64s(const int64_t* const* dev, int k, int64_t* out, cudaStream_t s, const int64_t* arr = nullptr,
               int na = 0, int64_t* arr_out = nullptr);
double read_f64(const double* dev, cudaStream_t s);

// ---- add.cu
// A <- alpha A + beta B on the union of the patterns (B may be A).
void add(dbcsr_matrix_* A, double alpha, const dbcsr_matrix_* B, double beta);

// ---- reduce.cu
double trace(dbcsr_matrix_* m);
double trace_product(dbcsr_matrix_* a, dbcsr_matrix_* b);
double gershgorin(dbcsr_matrix_* m, double mu);
// part[b] = <A_b, B_JI^T> for every block b = (I, J) of A (the first stage of trace_product).
void trace_product_parts_into(dbcsr_matrix_* a, dbcsr_matrix_* b, double* part, cudaStream_t s);

// ---- multiply.cu
// sym_result: the caller knows alpha*A*B + beta*C is symmetric in exact arithmetic
// (as every product of the sign iteration is), and the result is made exactly
// symmetric; blocks without a formed twin (J, I) are dropped.
//   kSymMirror:  only blocks I <= J are computed, their twins copied as transposes, and
//                the diagonal blocks replaced by their symmetric parts;
//   kSymAverage: both twins are computed and replaced by their symmetric mean
//                (for operands that commute only approximately, e.g. BF16 products).
constexpr int kSymNone = 0, kSymMirror = 1, kSymAverage = 2;
struct LowTierPlan;
// m <- (m + m^T) / 2 on the blocks that have a twin; blocks without one are dropped.
void symmetrize(dbcsr_matrix_* m);
// A planned product C = alpha A B on fixed patterns: the buffers its numeric phase needs
// and that phase captured as one CUDA graph (dbcsr_multiply_plan).
struct MultPlan {
    cudaGraphExec_t exec = nullptr;
    int64_t kernels = 0;                 // kernel launches per execution
    cudaStream_t stream = nullptr;
    dbcsr_matrix_* A = nullptr;
    dbcsr_matrix_* B = nullptr;
    dbcsr_matrix_* C = nullptr;
    std::vector<DBuf<int32_t>> bufs_i32;
    std::vector<DBuf<int64_t>> bufs_i64;
    std::vector<DBuf<double>> bufs_f64;
    std::vector<DBuf<__nv_bfloat16>> bufs_bf16;
    std::vector<DBuf<uint8_t>> bufs_u8;
    LowTierPlan* lt = nullptr;           // BF16 products: the tensor-core tier's symbolic results
    ~MultPlan();
};
// plan: build a plan instead of a one-off product (beta = 0, C distinct from A and B, no
// symmetric result); C then holds the formed pattern with blocks under eps zeroed.
void multiply(double alpha, dbcsr_matrix_* A, dbcsr_matrix_* B, double beta, dbcsr_matrix_* C, double eps,
              int prec, dbcsr_mult_stats* stats, bool want_dev2, int sym_result = kSymNone, MultPlan* plan = nullptr);
void execute_plan(MultPlan* plan);
// Fails with DBCSR_ESTATE when a live plan uses m's arrays (they must not be replaced).
void check_unplanned(const dbcsr_matrix_* m, const char* where);

// ---- lowtier.cu
// Groups of neighbouring blocks from the strongest couplings (block norms) of m.
std::shared_ptr<Groups> build_groups(dbcsr_matrix_* m);
// Where the tensor-core tier writes: the formed blocks of the product (CSR over block rows,
// computed flags, element offsets, C input) and the result arrays.
struct LowTierOut {
    const int64_t* f_rp; const int32_t* f_col; const uint8_t* f_comp; const int64_t* f_off; const int64_t* f_cin;
    const int64_t* ci_off; const double* ci_data;
    double alpha, beta;
    double* c_data; double* c_norm; double* c_dev2;
};
struct LowTierPlan;
void lowtier_plan_delete(LowTierPlan* p);
// Symbolic phase of a tensor-core product: group tile patterns of A, B and C and the per-C-tile
// stacks.  sym_operands: A and B are exactly symmetric (B's tiles are then read transposed from
// its row-major packing, and from A's packing when B is A).
std::unique_ptr<LowTierPlan, void (*)(LowTierPlan*)> lowtier_prepare(int prec, dbcsr_matrix_* A, dbcsr_matrix_* B,
                                                                     std::shared_ptr<Groups> groups, bool sym_operands,
                                                                     int64_t nform, const int64_t* f_rp,
                                                                     const int32_t* f_row, const int32_t* f_col,
                                                                     const uint8_t* f_comp, cudaStream_t s);
// Numeric phase: packs A and B (their current values), then runs the tensor-core kernel.
void lowtier_pack(LowTierPlan& L, dbcsr_matrix_* A, dbcsr_matrix_* B, cudaStream_t s);
void lowtier_run(LowTierPlan& L, dbcsr_matrix_* A, const LowTierOut& o, cudaStream_t s);
// Fails with DBCSR_ETIMEOUT when a bounded wait of the kernel ran out (synchronises s).
void lowtier_check(LowTierPlan& L, cudaStream_t s);
int64_t lowtier_tiles(const LowTierPlan& L);
// Executed MMA flops (2 M N K per MMA, every split product, padding included) and the bytes
// its bulk copies move into shared memory.
double lowtier_tensor_flops(const LowTierPlan& L);
double lowtier_copy_bytes(const LowTierPlan& L);

// ---- dense.cu
// C[b] = alpha A[b] B[b] + beta C[b] for nb row-major n x n matrices (b < 65536): FP64 on the
// FP64 pipe; FP32 storage on the TF32 tensor cores (split: three products of TF32 halves,
// close to FP32 arithmetic).  C must not alias A or B.
void dense_gemm_f64(int64_t nb, int n, double alpha, const double* A, const double* B, double beta, double* C,
                    cudaStream_t s);
void dense_gemm_tf32(int64_t nb, int n, float alpha, const float* A, const float* B, float beta, float* C, bool split,
                     cudaStream_t s);

// ---- submatrix.cu
dbcsr_status submatrix_sign(dbcsr_matrix_* H, double mu, const dbcsr_sign_opts* opts, dbcsr_matrix_* P,
                            dbcsr_sign_report* rep);

// ---- purify.cu
dbcsr_status purify(dbcsr_matrix_* H, double n_occ, int32_t method, const dbcsr_sign_opts* opts, dbcsr_matrix_* P,
                    dbcsr_sign_report* rep);
dbcsr_status sign_mu_search(dbcsr_matrix_* H, double n_occ, double mu_lo, double mu_hi, const dbcsr_sign_opts* opts,
                            dbcsr_matrix_* P, double* mu_out, int32_t* evaluations, dbcsr_sign_report* rep);

// ---- sqrt.cu
// S^(-1/2) (into Sinv) and, when Ssqrt is given, S^(1/2) by the sign iteration on [[0, S], [1, 0]].
dbcsr_status inverse_sqrt(dbcsr_matrix_* S, const dbcsr_sign_opts* opts, dbcsr_matrix_* Sinv, dbcsr_matrix_* Ssqrt,
                          dbcsr_sign_report* rep);
dbcsr_status inverse_hotelling(dbcsr_matrix_* A, const dbcsr_sign_opts* opts, dbcsr_matrix_* Ainv,
                               dbcsr_sign_report* rep);
dbcsr_status sign_iterate_nonorth(dbcsr_matrix_* K, dbcsr_matrix_* S, double mu, const dbcsr_sign_opts* opts,
                                  dbcsr_matrix_* P, dbcsr_sign_report* rep, dbcsr_sign_report* rep_sqrt);

// ---- sign.cu
// A matrix with m's block sizes and stream, no pattern yet.
std::unique_ptr<dbcsr_matrix_> make_like(const dbcsr_matrix_* m, cudaStream_t s);
// c_0..c_n, c_j = binom(2j, j) / 4^j: the step polynomial p_n(y) = sum_j c_j (1 - y)^j.
std::vector<double> sign_series_coeffs(int n);
// U = p_n(Y) for the step of order n + 1 (Y = filter(X X), or Z Y in the square-root
// iteration): order 2 gives (3 - Y) / 2 with no product; higher orders sum p_n in powers of
// 1 - Y with filtered products (Y is then overwritten with 1 - Y).
std::unique_ptr<dbcsr_matrix_> step_polynomial(dbcsr_matrix_* Y, int order, double eps, int tier, int sym,
                                               const std::function<void(const dbcsr_mult_stats&, int)>& account);
// One update X <- filter(X p_n(Y)) of the sign iteration of order n + 1, given
// Y = filter(X X); products in precision tier with symmetry mode sym, each passed to account.
// Y is overwritten (with 1 - Y for orders above 2, with Y - 1 in order 2's correction form).
void sign_update(dbcsr_matrix_* X, dbcsr_matrix_* Y, int order, bool correction, double eps, int tier, int sym,
                 const std::function<void(const dbcsr_mult_stats&, int)>& account);
dbcsr_status sign_iterate_resume(dbcsr_matrix_* H, dbcsr_matrix_* X0, const dbcsr_sign_report* prev,
                                 const dbcsr_sign_opts* opts, dbcsr_matrix_* P, dbcsr_sign_report* rep);
dbcsr_status sign_iterate(dbcsr_matrix_* H, double mu, const dbcsr_sign_opts* opts, dbcsr_matrix_* P,
                          dbcsr_sign_report* rep);

// Streaming multiprocessors of the current device (cudaDevAttrMultiProcessorCount, queried
// once per device and cached; 152 on a GB300).
int num_sms();

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
// Grid of ceil(work / per) CTAs, at least 1, at most cap (default: 64 CTAs per SM).
inline unsigned grid_for(int64_t work, int per, int64_t cap = -1) {
    if (cap < 0) cap = (int64_t)num_sms() * 64;
    int64_t g = ceil_div(work, per);
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (unsigned)g;
}

}  // namespace dbg
