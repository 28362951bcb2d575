// Autotuner of the batched block-product kernels (the paper's "Batched
// execution": each (m, n, k) kernel is tuned over its parameters on stacks of
// block products, and the best parameter set is kept per (m, n, k)).
//
// Here the parameters of the FP64 block-product kernels are the work split per C block
// (one warp, a warp pair sharing the element slots, or the K-split remainder kernel) and
// the launch-time choices that leave the arithmetic unchanged: threads per CTA, CTAs per
// SM of the grid, the lane-to-element order and double-buffered product metadata.  The
// tensor-core tier (BF16 products) runs one tile shape for every block shape, so it has
// nothing to tune per (m, n, k).  A synthetic stack for (m, n, k) imitates one shape launch
// of a real product: stack_len products over C blocks of 32 products each, with A and B
// blocks drawn at random from pools of about 512 MB together (several times the L2).
#include <algorithm>
#include <cstdio>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <tuple>

#include "common.cuh"
#include "smm.cuh"

namespace dbg {
namespace {

std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, TuneCfg> g_tune;

// The synthetic stack imitates one shape launch of a sign-iteration product: operand
// pools several times larger than L2 (kPoolBytes for A and B together, so products
// miss in L2 as real ones do), C blocks of kProductsPerC products each (one metadata
// batch), and products that draw their A and B blocks at random from the pools.
constexpr int64_t kPoolMin = 20000;
constexpr int64_t kPoolBytes = 512ll << 20;
constexpr int kProductsPerC = 32;

int64_t pool_blocks(int m, int n, int k) {
    return std::max<int64_t>(kPoolMin, kPoolBytes / (8 * ((int64_t)m * k + (int64_t)k * n)));
}

__device__ __forceinline__ uint64_t mix(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_fill_uniform(int64_t n, uint64_t seed, double* __restrict__ x) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = (double)(mix(seed ^ (uint64_t)i) >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

__global__ void k_fill_stack_synth(int64_t nprod, int64_t nc, int64_t npool, uint64_t seed, int m, int n, int k,
                                   int32_t* __restrict__ prod_a, int32_t* __restrict__ prod_b,
                                   int64_t* __restrict__ a_off, int64_t* __restrict__ b_off, int32_t* __restrict__ a_col,
                                   int32_t* __restrict__ f_row, int32_t* __restrict__ f_col, int64_t* __restrict__ f_off,
                                   int64_t* __restrict__ f_pbeg, int64_t* __restrict__ f_cin, int64_t* __restrict__ list) {
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = tid; p < nprod; p += stride) {
        prod_a[p] = (int32_t)(mix(seed + 2 * (uint64_t)p) % (uint64_t)npool);
        prod_b[p] = (int32_t)(mix(seed + 2 * (uint64_t)p + 1) % (uint64_t)npool);
    }
    for (int64_t i = tid; i < npool; i += stride) {
        a_off[i] = i * (int64_t)m * k;
        b_off[i] = i * (int64_t)k * n;
        a_col[i] = 2;                     // block size table {m, n, k}: K blocks have edge k
    }
    for (int64_t c = tid; c <= nc; c += stride) {
        f_pbeg[c] = std::min(c * (int64_t)kProductsPerC, nprod);
        if (c < nc) {
            f_row[c] = 0;
            f_col[c] = 1;
            f_off[c] = c * (int64_t)m * n;
            f_cin[c] = -1;
            list[c] = c;
        }
    }
}

// A synthetic (m, n, k) stack resident on the device.
struct SynthStack {
    int m, n, k;
    int64_t nprod, nc, npool;
    DBuf<double> a, b, c, norm, dev2;
    DBuf<int32_t> prod_a, prod_b, a_col, f_row, f_col, bs;
    DBuf<int64_t> a_off, b_off, f_off, f_pbeg, f_cin, list;
    SmmArgs args{};

    SynthStack(int m_, int n_, int k_, int64_t stack_len, cudaStream_t s) : m(m_), n(n_), k(k_) {
        nprod = stack_len;
        npool = pool_blocks(m, n, k);
        nc = ceil_div(stack_len, kProductsPerC);
        a.alloc(npool * m * k, s);
        b.alloc(npool * k * n, s);
        c.alloc(nc * m * n, s);
        norm.alloc(nc, s);
        dev2.alloc(nc, s);
        prod_a.alloc(nprod, s);
        prod_b.alloc(nprod, s);
        a_col.alloc(npool, s);
        f_row.alloc(nc, s);
        f_col.alloc(nc, s);
        bs.alloc(3, s);
        a_off.alloc(npool, s);
        b_off.alloc(npool, s);
        f_off.alloc(nc, s);
        f_pbeg.alloc(nc + 1, s);
        f_cin.alloc(nc, s);
        list.alloc(nc, s);
        const int32_t hb[3] = {m, n, k};
        DBG_CK(cudaMemcpyAsync(bs.p, hb, sizeof(hb), cudaMemcpyHostToDevice, s));
        k_fill_uniform<<<grid_for(a.n, 256), 256, 0, s>>>(a.n, 0xA5A5ull + (uint64_t)m * 977 + k, a.p);
        DBG_LAUNCH_CK();
        k_fill_uniform<<<grid_for(b.n, 256), 256, 0, s>>>(b.n, 0x5A5Aull + (uint64_t)n * 977 + k, b.p);
        DBG_LAUNCH_CK();
        k_fill_stack_synth<<<grid_for(std::max<int64_t>(nprod, npool), 256), 256, 0, s>>>(
            nprod, nc, npool, 0x1234ull + (uint64_t)(m * 10000 + n * 100 + k), m, n, k, prod_a.p, prod_b.p, a_off.p, b_off.p,
            a_col.p, f_row.p, f_col.p, f_off.p, f_pbeg.p, f_cin.p, list.p);
        DBG_LAUNCH_CK();
        args = SmmArgs{f_row.p, f_col.p, f_off.p, f_pbeg.p, f_cin.p, prod_a.p, prod_b.p, a_col.p, a_off.p, a.p,
                       b_off.p, b.p, nullptr, nullptr, bs.p, 1.0, 0.0, c.p, norm.p, dev2.p, 0, 0};
    }

    // Median time (ms) of `reps` launches with configuration cfg.
    double time(const TuneCfg& cfg, int reps, cudaStream_t s) {
        cudaEvent_t e0, e1;
        DBG_CK(cudaEventCreate(&e0));
        DBG_CK(cudaEventCreate(&e1));
        std::vector<float> t;
        launch_smm_shape(m, n, nc, list.p, args, cfg, s);   // warm-up
        for (int r = 0; r < reps; ++r) {
            DBG_CK(cudaEventRecord(e0, s));
            launch_smm_shape(m, n, nc, list.p, args, cfg, s);
            DBG_CK(cudaEventRecord(e1, s));
            DBG_CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            DBG_CK(cudaEventElapsedTime(&ms, e0, e1));
            t.push_back(ms);
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        std::sort(t.begin(), t.end());
        return t[t.size() / 2];
    }
};

void check_prec(int prec) {
    if (prec != DBCSR_FP64)
        fail(DBCSR_EINVAL, "tune: prec must be DBCSR_FP64 (the tensor-core tier has no per-shape kernels to tune)");
}

void check_triple(int prec, int m, int n, int k) {
    check_prec(prec);
    if (m < 1 || n < 1 || k < 1 || m > kMaxBlock || n > kMaxBlock || k > kMaxBlock)
        fail(DBCSR_EINVAL, "tune: m, n, k must lie in [1, 32]");
}

}  // namespace

std::vector<TuneCfg> tune_space(int prec) {
    check_prec(prec);
    std::vector<TuneCfg> v;
    for (int sp : {kSplitWarp, kSplitPair, kSplitK})
        for (int tpb : {128, 256})
            for (int c : {4, 8, 16, 32})
                for (int cm : {0, 1})
                    for (int pf : {0, 1}) {
                        TuneCfg t;
                        t.tpb = tpb;
                        t.ctas_per_sm = c;
                        t.colmajor = cm;
                        t.prefetch2 = pf;
                        t.split = sp;
                        v.push_back(t);
                    }
    return v;
}

TuneCfg tune_lookup(int prec, int m, int n, int k) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune.find({prec, m, n, k});
    return it == g_tune.end() ? default_cfg(prec) : it->second;
}

}  // namespace dbg

// ------------------------------------------------------------------ C ABI
namespace {
dbg::TuneCfg from_c(const dbcsr_kernel_cfg& c) {
    dbg::TuneCfg t;
    t.tpb = c.tpb;
    t.ctas_per_sm = c.ctas_per_sm;
    t.colmajor = c.colmajor;
    t.prefetch2 = c.prefetch2;
    t.split = c.split;
    return t;
}
dbcsr_kernel_cfg to_c(const dbg::TuneCfg& t) {
    return dbcsr_kernel_cfg{t.tpb, t.ctas_per_sm, t.colmajor, t.prefetch2, t.split};
}

template <class F>
dbcsr_status guard(F&& f) {
    try {
        f();
        dbg::set_last_error("");
        return DBCSR_OK;
    } catch (const dbg::Error& e) {
        dbg::set_last_error(e.what());
        return e.code;
    } catch (const std::exception& e) {
        dbg::set_last_error(e.what());
        return DBCSR_EINVAL;
    }
}
}  // namespace

extern "C" {

dbcsr_status dbcsr_tune_space(int32_t prec, dbcsr_kernel_cfg* out, int32_t cap, int32_t* n) {
    return guard([&] {
        auto v = dbg::tune_space(prec);
        if (n) *n = (int32_t)v.size();
        if (out)
            for (int32_t i = 0; i < std::min<int32_t>(cap, (int32_t)v.size()); ++i) out[i] = to_c(v[i]);
    });
}

dbcsr_status dbcsr_time_config(int32_t prec, int32_t m, int32_t n, int32_t k, int64_t stack_len, int32_t reps,
                               const dbcsr_kernel_cfg* cfgs, int32_t ncfg, double* ms_out) {
    return guard([&] {
        dbg::check_triple(prec, m, n, k);
        if (stack_len < 1 || reps < 1 || ncfg < 1 || !cfgs || !ms_out) dbg::fail(DBCSR_EINVAL, "time_config: bad argument");
        cudaStream_t s = nullptr;
        for (int32_t i = 0; i < ncfg; ++i)
            if (!dbg::cfg_valid(m, n, from_c(cfgs[i])))
                dbg::fail(DBCSR_EINVAL, "time_config: configuration " + std::to_string(i) + " does not apply to the shape");
        dbg::SynthStack st(m, n, k, stack_len, s);
        for (int32_t i = 0; i < ncfg; ++i) ms_out[i] = st.time(from_c(cfgs[i]), reps, s);
    });
}

dbcsr_status dbcsr_autotune(const int32_t* mnk, int32_t ntriples, int32_t prec, int64_t stack_len, int32_t reps,
                            dbcsr_tune_record* recs, int64_t cap, int64_t* nrec) {
    return guard([&] {
        if (!mnk || ntriples < 1 || stack_len < 1 || reps < 1) dbg::fail(DBCSR_EINVAL, "autotune: bad argument");
        const auto space = dbg::tune_space(prec);
        cudaStream_t s = nullptr;
        int64_t w = 0;
        for (int32_t t = 0; t < ntriples; ++t) {
            const int m = mnk[3 * t], n = mnk[3 * t + 1], k = mnk[3 * t + 2];
            dbg::check_triple(prec, m, n, k);
            dbg::SynthStack st(m, n, k, stack_len, s);
            double best = 1e300;
            dbg::TuneCfg best_cfg = dbg::default_cfg(prec);
            for (const auto& c : space) {
                if (!dbg::cfg_valid(m, n, c)) continue;
                const double ms = st.time(c, reps, s);
                if (ms < best) {
                    best = ms;
                    best_cfg = c;
                }
                if (recs && w < cap) {
                    recs[w] = dbcsr_tune_record{m, n, k, prec, to_c(c), ms,
                                                2.0 * m * n * k * (double)stack_len / (ms * 1e-3) * 1e-9};
                }
                ++w;
            }
            std::lock_guard<std::mutex> lock(dbg::g_tune_mu);
            dbg::g_tune[{prec, m, n, k}] = best_cfg;
        }
        if (nrec) *nrec = w;
    });
}

dbcsr_status dbcsr_tune_predicted(int32_t prec, const float* params, const int32_t* mnk, int32_t ntriples,
                                  int64_t stack_len, int32_t reps, double tolerance, int32_t* fell_back) {
    return guard([&] {
        if (!mnk || ntriples < 1 || stack_len < 1 || reps < 1 || !(tolerance == tolerance))
            dbg::fail(DBCSR_EINVAL, "tune_predicted: bad argument");
        for (int32_t t = 0; t < ntriples; ++t) dbg::check_triple(prec, mnk[3 * t], mnk[3 * t + 1], mnk[3 * t + 2]);
        std::vector<dbcsr_kernel_cfg> pred(ntriples);
        const dbcsr_status ps = dbcsr_mlp_predict_best(prec, params, mnk, ntriples, pred.data(), nullptr);
        if (ps != DBCSR_OK) dbg::fail(ps, "tune_predicted: prediction failed");
        const auto space = dbg::tune_space(prec);
        const dbg::TuneCfg dflt = dbg::default_cfg(prec);
        cudaStream_t s = nullptr;
        for (int32_t t = 0; t < ntriples; ++t) {
            const int m = mnk[3 * t], n = mnk[3 * t + 1], k = mnk[3 * t + 2];
            dbg::SynthStack st(m, n, k, stack_len, s);
            // measured time decides on the prediction: kept if within tolerance of the default,
            // otherwise the exhaustive search over the space decides
            dbg::TuneCfg chosen = from_c(pred[t]);
            const double tp = st.time(chosen, reps, s);
            const double td = st.time(dflt, reps, s);
            const bool fb = !(tp <= td * (1.0 + tolerance));
            if (fb) {
                double best = 1e300;
                for (const auto& c : space) {
                    if (!dbg::cfg_valid(m, n, c)) continue;
                    const double ms = st.time(c, reps, s);
                    if (ms < best) {
                        best = ms;
                        chosen = c;
                    }
                }
            }
            if (fell_back) fell_back[t] = fb ? 1 : 0;
            std::lock_guard<std::mutex> lock(dbg::g_tune_mu);
            dbg::g_tune[{prec, m, n, k}] = chosen;
        }
    });
}

dbcsr_status dbcsr_tune_set(int32_t prec, int32_t m, int32_t n, int32_t k, const dbcsr_kernel_cfg* cfg) {
    return guard([&] {
        dbg::check_triple(prec, m, n, k);
        std::lock_guard<std::mutex> lock(dbg::g_tune_mu);
        if (cfg && !dbg::cfg_valid(m, n, from_c(*cfg)))
            dbg::fail(DBCSR_EINVAL, "tune_set: the configuration does not apply to m x n blocks");
        if (!cfg) dbg::g_tune.erase({prec, m, n, k});
        else dbg::g_tune[{prec, m, n, k}] = from_c(*cfg);
    });
}

dbcsr_status dbcsr_tune_get(int32_t prec, int32_t m, int32_t n, int32_t k, dbcsr_kernel_cfg* cfg, int* found) {
    return guard([&] {
        dbg::check_triple(prec, m, n, k);
        std::lock_guard<std::mutex> lock(dbg::g_tune_mu);
        auto it = dbg::g_tune.find({prec, m, n, k});
        if (found) *found = it != dbg::g_tune.end();
        if (cfg) *cfg = to_c(it != dbg::g_tune.end() ? it->second : dbg::default_cfg(prec));
    });
}

dbcsr_status dbcsr_tune_clear(void) {
    return guard([&] {
        std::lock_guard<std::mutex> lock(dbg::g_tune_mu);
        dbg::g_tune.clear();
    });
}

dbcsr_status dbcsr_tune_save(const char* path) {
    return guard([&] {
        if (!path) dbg::fail(DBCSR_EINVAL, "tune_save: null path");
        std::ofstream f(path);
        if (!f) dbg::fail(DBCSR_EINVAL, std::string("tune_save: cannot open ") + path);
        f << "# prec m n k tpb ctas_per_sm colmajor prefetch2 split\n";
        std::lock_guard<std::mutex> lock(dbg::g_tune_mu);
        for (const auto& [key, c] : dbg::g_tune)
            f << std::get<0>(key) << ' ' << std::get<1>(key) << ' ' << std::get<2>(key) << ' ' << std::get<3>(key) << ' '
              << c.tpb << ' ' << c.ctas_per_sm << ' ' << c.colmajor << ' ' << c.prefetch2 << ' ' << c.split << '\n';
    });
}

dbcsr_status dbcsr_tune_load(const char* path) {
    return guard([&] {
        if (!path) dbg::fail(DBCSR_EINVAL, "tune_load: null path");
        std::ifstream f(path);
        if (!f) dbg::fail(DBCSR_EINVAL, std::string("tune_load: cannot open ") + path);
        std::string line;
        std::map<std::tuple<int, int, int, int>, dbg::TuneCfg> tab;
        while (std::getline(f, line)) {
            if (line.empty() || line[0] == '#') continue;
            std::istringstream is(line);
            int prec, m, n, k;
            dbg::TuneCfg c;
            if (!(is >> prec >> m >> n >> k >> c.tpb >> c.ctas_per_sm >> c.colmajor >> c.prefetch2 >> c.split))
                dbg::fail(DBCSR_EINVAL, "tune_load: malformed line: " + line);
            dbg::check_triple(prec, m, n, k);
            if (!dbg::cfg_valid(m, n, c))
                dbg::fail(DBCSR_EINVAL, "tune_load: configuration out of range for the shape: " + line);
            tab[{prec, m, n, k}] = c;
        }
        std::lock_guard<std::mutex> lock(dbg::g_tune_mu);
        for (auto& [key, c] : tab) dbg::g_tune[key] = c;
    });
}

}  // extern "C"
