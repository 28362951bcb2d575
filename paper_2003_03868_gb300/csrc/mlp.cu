// Performance-prediction MLP for the block-product kernels (the paper's
// "Batched execution": autotuning data train a model that predicts near-optimal
// parameters for the (m, n, k) kernels that were not tuned).
//
// Model: features x (nfeat) -> 64 ReLU -> 64 ReLU -> 1 (predicted standardised
// log time), FP32.  Parameters are one flat array:
//   W1[64][nfeat] b1[64] W2[64][64] b2[64] W3[64] b3
// Training: full-batch mean squared error, Adam.  Every kernel is deterministic:
// gradients of a weight are summed by one thread over the samples in order, and
// the loss by a fixed tree.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "smm.cuh"

namespace dbg {
namespace {

constexpr int kH = 64;
constexpr int kMaxFeat = 32;

__host__ __device__ inline int64_t n_params(int nf) { return (int64_t)kH * nf + kH + kH * kH + kH + kH + 1; }

struct Layout {
    int nf;
    const float *W1, *b1, *W2, *b2, *W3, *b3;
};

__host__ __device__ inline Layout layout(const float* p, int nf) {
    Layout L;
    L.nf = nf;
    L.W1 = p;
    L.b1 = L.W1 + kH * nf;
    L.W2 = L.b1 + kH;
    L.b2 = L.W2 + kH * kH;
    L.W3 = L.b2 + kH;
    L.b3 = L.W3 + kH;
    return L;
}

// One warp per sample: h1, h2 (stored for the backward pass) and y.
__global__ void k_mlp_forward(int64_t B, int nf, const float* __restrict__ params, const float* __restrict__ X,
                              float* __restrict__ H1, float* __restrict__ H2, float* __restrict__ Y) {
    const Layout L = layout(params, nf);
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); b < B; b += warps) {
        const float* x = X + b * nf;
        float h1[2], h2[2];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int u = lane + 32 * r;
            float s = L.b1[u];
            for (int f = 0; f < nf; ++f) s = fmaf(L.W1[u * nf + f], x[f], s);
            h1[r] = fmaxf(s, 0.f);
            H1[b * kH + u] = h1[r];
        }
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int u = lane + 32 * r;
            float s = L.b2[u];
            for (int v = 0; v < kH; ++v) {
                const float hv = __shfl_sync(0xffffffffu, h1[v >> 5], v & 31);
                s = fmaf(L.W2[u * kH + v], hv, s);
            }
            h2[r] = fmaxf(s, 0.f);
            H2[b * kH + u] = h2[r];
        }
        float y = L.W3[lane] * h2[0] + L.W3[lane + 32] * h2[1];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
        if (lane == 0) Y[b] = y + L.b3[0];
    }
}

// Per sample: dy = 2 (y - t) / B, dH2 = dy W3 (h2 > 0), dH1 = W2^T dH2 (h1 > 0); err = (y - t)^2.
__global__ void k_mlp_backprop(int64_t B, int nf, const float* __restrict__ params, const float* __restrict__ T,
                               const float* __restrict__ H1, const float* __restrict__ H2, const float* __restrict__ Y,
                               float* __restrict__ DY, float* __restrict__ D2, float* __restrict__ D1,
                               float* __restrict__ ERR) {
    const Layout L = layout(params, nf);
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); b < B; b += warps) {
        const float diff = Y[b] - T[b];
        const float dy = 2.f * diff / (float)B;
        float d2[2];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int u = lane + 32 * r;
            d2[r] = H2[b * kH + u] > 0.f ? dy * L.W3[u] : 0.f;
            D2[b * kH + u] = d2[r];
        }
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int v = lane + 32 * r;
            float s = 0.f;
            for (int u = 0; u < kH; ++u) {
                const float du = __shfl_sync(0xffffffffu, d2[u >> 5], u & 31);
                s = fmaf(L.W2[u * kH + v], du, s);
            }
            D1[b * kH + v] = H1[b * kH + v] > 0.f ? s : 0.f;
        }
        if (lane == 0) {
            DY[b] = dy;
            ERR[b] = diff * diff;
        }
    }
}

// One thread per parameter: its gradient summed over the samples in order.
__global__ void k_mlp_weight_grads(int64_t B, int nf, const float* __restrict__ X, const float* __restrict__ H1,
                                   const float* __restrict__ H2, const float* __restrict__ DY,
                                   const float* __restrict__ D2, const float* __restrict__ D1, float* __restrict__ G) {
    const int64_t P = n_params(nf);
    const int64_t ob1 = kH * nf, oW2 = ob1 + kH, ob2 = oW2 + kH * kH, oW3 = ob2 + kH, ob3 = oW3 + kH;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        float g = 0.f;
        if (i < ob1) {                       // W1[u][f] (offset 0)
            const int u = (int)(i / nf), f = (int)(i % nf);
            for (int64_t b = 0; b < B; ++b) g = fmaf(D1[b * kH + u], X[b * nf + f], g);
        } else if (i < oW2) {                // b1[u]
            const int u = (int)(i - ob1);
            for (int64_t b = 0; b < B; ++b) g += D1[b * kH + u];
        } else if (i < ob2) {                // W2[u][v]
            const int u = (int)((i - oW2) / kH), v = (int)((i - oW2) % kH);
            for (int64_t b = 0; b < B; ++b) g = fmaf(D2[b * kH + u], H1[b * kH + v], g);
        } else if (i < oW3) {                // b2[u]
            const int u = (int)(i - ob2);
            for (int64_t b = 0; b < B; ++b) g += D2[b * kH + u];
        } else if (i < ob3) {                // W3[u]
            const int u = (int)(i - oW3);
            for (int64_t b = 0; b < B; ++b) g = fmaf(DY[b], H2[b * kH + u], g);
        } else {                             // b3
            for (int64_t b = 0; b < B; ++b) g += DY[b];
        }
        G[i] = g;
    }
}

// Adam (Kingma & Ba 2015) with bias correction, step t (1-based).
__global__ void k_adam(int64_t P, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m1,
                       float* __restrict__ m2, float lr, float b1, float b2, float eps, int t) {
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float a = b1 * m1[i] + (1.f - b1) * gi;
        const float v = b2 * m2[i] + (1.f - b2) * gi * gi;
        m1[i] = a;
        m2[i] = v;
        p[i] -= lr * (a / c1) / (sqrtf(v / c2) + eps);
    }
}

// Fixed-tree sum of n floats into *out (one CTA).
__global__ void k_sum_f32(int64_t n, const float* __restrict__ v, float* __restrict__ out) {
    __shared__ float sh[256];
    float s = 0.f;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += v[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

struct MlpWork {
    int64_t B;
    int nf;
    DBuf<float> X, T, H1, H2, Y, DY, D2, D1, ERR, P, G, M1, M2, loss;
    MlpWork(int64_t B_, int nf_, const float* hX, const float* hT, const float* hp, cudaStream_t s) : B(B_), nf(nf_) {
        const int64_t np = n_params(nf);
        X.alloc(B * nf, s);
        H1.alloc(B * kH, s);
        H2.alloc(B * kH, s);
        Y.alloc(B, s);
        P.alloc(np, s);
        DBG_CK(cudaMemcpyAsync(X.p, hX, sizeof(float) * B * nf, cudaMemcpyHostToDevice, s));
        DBG_CK(cudaMemcpyAsync(P.p, hp, sizeof(float) * np, cudaMemcpyHostToDevice, s));
        if (hT) {
            T.alloc(B, s);
            DY.alloc(B, s);
            D2.alloc(B * kH, s);
            D1.alloc(B * kH, s);
            ERR.alloc(B, s);
            G.alloc(np, s);
            M1.alloc(np, s);
            M2.alloc(np, s);
            loss.alloc(1, s);
            M1.zero();
            M2.zero();
            DBG_CK(cudaMemcpyAsync(T.p, hT, sizeof(float) * B, cudaMemcpyHostToDevice, s));
        }
    }
    void forward(cudaStream_t s) {
        k_mlp_forward<<<grid_for(B, 8, num_sms() * 16), 256, 0, s>>>(B, nf, P.p, X.p, H1.p, H2.p, Y.p);
        DBG_LAUNCH_CK();
    }
    void gradient(cudaStream_t s) {
        forward(s);
        k_mlp_backprop<<<grid_for(B, 8, num_sms() * 16), 256, 0, s>>>(B, nf, P.p, T.p, H1.p, H2.p, Y.p, DY.p, D2.p, D1.p,
                                                                ERR.p);
        DBG_LAUNCH_CK();
        const int64_t np = n_params(nf);
        k_mlp_weight_grads<<<grid_for(np, 128), 128, 0, s>>>(B, nf, X.p, H1.p, H2.p, DY.p, D2.p, D1.p, G.p);
        DBG_LAUNCH_CK();
        k_sum_f32<<<1, 256, 0, s>>>(B, ERR.p, loss.p);
        DBG_LAUNCH_CK();
    }
};

void check_feat(int nf, int64_t B) {
    if (nf < 1 || nf > kMaxFeat) fail(DBCSR_EINVAL, "mlp: nfeat must lie in [1, 32]");
    if (B < 1) fail(DBCSR_EINVAL, "mlp: need at least one sample");
}

uint64_t splitmix(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace

// Features of one (m, n, k, configuration) sample, kMlpFeatures of them.
void mlp_features(int prec, int m, int n, int k, const TuneCfg& c, float* f) {
    (void)prec;
    const int mn = m * n;
    const int split = resolve_split(m, n, c);
    const int E = (mn + 31) / 32;                                     // element slots per lane, one warp
    const double lanes = 32.0 * (split == kSplitK ? (mn >> 5) + 1 : E);
    const int el = split == kSplitPair ? (E + 1) / 2 : (split == kSplitK ? (mn >> 5) : E);
    f[0] = m / 32.f;
    f[1] = n / 32.f;
    f[2] = k / 32.f;
    f[3] = (float)(std::log2((double)mn * k) / 15.0);
    f[4] = (float)(mn / lanes);                                       // useful fraction of the lane slots
    f[5] = split == kSplitK ? 1.f : 0.f;                              // K-split remainder kernel
    f[6] = c.tpb / 256.f;
    f[7] = (float)(std::log2((double)c.ctas_per_sm) / 6.0);
    f[8] = (float)c.colmajor;
    f[9] = (float)c.prefetch2;
    f[10] = split == kSplitPair ? 1.f : 0.f;                          // warp pair
    f[11] = el / 32.f;                                                // element slots (registers) per lane
}

// The model trained by dbcsr_predictor_train, one per precision, for the calls that take
// params == NULL.
std::mutex g_pred_mu;
std::map<int, std::vector<float>> g_predictor;

// One timing record of the autotuner as it is read back from a records file.
struct Rec {
    int prec, m, n, k;
    TuneCfg c;
    double ms;
};

std::vector<Rec> read_records(const char* path, int prec) {
    if (!path) fail(DBCSR_EINVAL, "predictor: null path");
    std::ifstream f(path);
    if (!f) fail(DBCSR_EINVAL, std::string("predictor: cannot open ") + path);
    std::vector<Rec> out;
    std::string line;
    while (std::getline(f, line)) {
        if (line.empty() || line[0] == '#') continue;
        std::istringstream is(line);
        Rec r;
        if (!(is >> r.prec >> r.m >> r.n >> r.k >> r.c.tpb >> r.c.ctas_per_sm >> r.c.colmajor >> r.c.prefetch2 >>
              r.c.split >> r.ms))
            fail(DBCSR_EINVAL, "predictor: malformed line: " + line);
        if (r.m < 1 || r.m > kMaxBlock || r.n < 1 || r.n > kMaxBlock || r.k < 1 || r.k > kMaxBlock ||
            !cfg_valid(r.m, r.n, r.c) || !(r.ms > 0.0) || !std::isfinite(r.ms))
            fail(DBCSR_EINVAL, "predictor: record out of range: " + line);
        if (r.prec == prec) out.push_back(r);
    }
    if (out.empty()) fail(DBCSR_EINVAL, std::string("predictor: no records of this precision in ") + path);
    return out;
}

// The training set of the prediction model from the autotuner's timings of one precision:
// the features of every (m, n, k, configuration) and, as the target, the log of its time
// minus the mean log time of its (m, n, k) triple, divided by the standard deviation of
// those centred values over all records (population form, floored at 1e-12).  The model
// thus learns how a configuration changes the time of a triple, not the triple's size.
void predictor_data(const std::vector<Rec>& recs, std::vector<float>& X, std::vector<float>& T) {
    const int nf = DBCSR_MLP_FEATURES;
    const size_t n = recs.size();
    X.assign(n * nf, 0.f);
    T.assign(n, 0.f);
    std::map<std::tuple<int, int, int>, std::pair<double, int64_t>> tri;
    std::vector<double> y(n);
    for (size_t i = 0; i < n; ++i) {
        const Rec& r = recs[i];
        mlp_features(r.prec, r.m, r.n, r.k, r.c, X.data() + i * nf);
        y[i] = std::log(r.ms);
        auto& acc = tri[{r.m, r.n, r.k}];
        acc.first += y[i];
        acc.second += 1;
    }
    std::vector<double> t(n);
    double mean = 0.0;
    for (size_t i = 0; i < n; ++i) {
        const auto& acc = tri[{recs[i].m, recs[i].n, recs[i].k}];
        t[i] = y[i] - acc.first / (double)acc.second;
        mean += t[i];
    }
    mean /= (double)n;
    double var = 0.0;
    for (size_t i = 0; i < n; ++i) var += (t[i] - mean) * (t[i] - mean);
    const double sd = std::max(std::sqrt(var / (double)n), 1e-12);
    for (size_t i = 0; i < n; ++i) T[i] = (float)(t[i] / sd);
}

}  // namespace dbg

extern "C" {

dbcsr_status dbcsr_tune_records_save(const char* path, const dbcsr_tune_record* recs, int64_t n, int32_t append) {
    try {
        if (!path || n < 0 || (n > 0 && !recs)) dbg::fail(DBCSR_EINVAL, "tune_records_save: bad argument");
        std::ofstream f(path, append ? std::ios::app : std::ios::trunc);
        if (!f) dbg::fail(DBCSR_EINVAL, std::string("tune_records_save: cannot open ") + path);
        if (!append) f << "# prec m n k tpb ctas_per_sm colmajor prefetch2 split ms\n";
        f.precision(17);
        for (int64_t i = 0; i < n; ++i) {
            const dbcsr_tune_record& r = recs[i];
            f << r.prec << ' ' << r.m << ' ' << r.n << ' ' << r.k << ' ' << r.cfg.tpb << ' ' << r.cfg.ctas_per_sm << ' '
              << r.cfg.colmajor << ' ' << r.cfg.prefetch2 << ' ' << r.cfg.split << ' ' << r.ms << '\n';
        }
        if (!f) dbg::fail(DBCSR_EINVAL, std::string("tune_records_save: write failed on ") + path);
        dbg::set_last_error("");
        return DBCSR_OK;
    } catch (const dbg::Error& e) {
        dbg::set_last_error(e.what());
        return e.code;
    }
}

dbcsr_status dbcsr_predictor_data(const char* tune_records, int32_t prec, float* X, float* T, int64_t cap,
                                  int64_t* n) {
    try {
        if (!n || cap < 0) dbg::fail(DBCSR_EINVAL, "predictor_data: bad argument");
        const auto recs = dbg::read_records(tune_records, prec);
        std::vector<float> x, t;
        dbg::predictor_data(recs, x, t);
        *n = (int64_t)recs.size();
        const int64_t w = std::min<int64_t>(cap, *n);
        if (w > 0 && X) std::memcpy(X, x.data(), sizeof(float) * w * DBCSR_MLP_FEATURES);
        if (w > 0 && T) std::memcpy(T, t.data(), sizeof(float) * w);
        dbg::set_last_error("");
        return DBCSR_OK;
    } catch (const dbg::Error& e) {
        dbg::set_last_error(e.what());
        return e.code;
    }
}

dbcsr_status dbcsr_predictor_train(const char* tune_records, int32_t prec, uint64_t seed, const dbcsr_mlp_opts* opts,
                                   dbcsr_mlp_report* rep) {
    try {
        if (!opts) dbg::fail(DBCSR_EINVAL, "predictor_train: null opts");
        const auto recs = dbg::read_records(tune_records, prec);
        std::vector<float> X, T;
        dbg::predictor_data(recs, X, T);
        const int nf = DBCSR_MLP_FEATURES;
        std::vector<float> params(dbg::n_params(nf));
        dbcsr_status st = dbcsr_mlp_init(nf, seed, params.data());
        if (st != DBCSR_OK) return st;
        st = dbcsr_mlp_train(nf, params.data(), X.data(), T.data(), (int64_t)recs.size(), opts, rep);
        if (st != DBCSR_OK) return st;
        std::lock_guard<std::mutex> lk(dbg::g_pred_mu);
        dbg::g_predictor[prec] = std::move(params);
        dbg::set_last_error("");
        return DBCSR_OK;
    } catch (const dbg::Error& e) {
        dbg::set_last_error(e.what());
        return e.code;
    }
}

dbcsr_status dbcsr_predictor_params(int32_t prec, float* params) {
    try {
        if (!params) dbg::fail(DBCSR_EINVAL, "predictor_params: null params");
        std::lock_guard<std::mutex> lk(dbg::g_pred_mu);
        auto it = dbg::g_predictor.find(prec);
        if (it == dbg::g_predictor.end()) dbg::fail(DBCSR_ESTATE, "predictor_params: no model trained for this precision");
        std::memcpy(params, it->second.data(), sizeof(float) * it->second.size());
        dbg::set_last_error("");
        return DBCSR_OK;
    } catch (const dbg::Error& e) {
        dbg::set_last_error(e.what());
        return e.code;
    }
}

dbcsr_status dbcsr_mlp_features(int32_t prec, const int32_t* mnk, const dbcsr_kernel_cfg* cfgs, int64_t n,
                                float* out) {
    try {
        if (!mnk || !cfgs || !out || n < 0) dbg::fail(DBCSR_EINVAL, "mlp_features: null argument");
        for (int64_t i = 0; i < n; ++i) {
            dbg::TuneCfg c;
            c.tpb = cfgs[i].tpb;
            c.ctas_per_sm = cfgs[i].ctas_per_sm;
            c.colmajor = cfgs[i].colmajor;
            c.prefetch2 = cfgs[i].prefetch2;
            c.split = cfgs[i].split;
            if (!dbg::cfg_valid(mnk[3 * i], mnk[3 * i + 1], c))
                dbg::fail(DBCSR_EINVAL, "mlp_features: configuration out of range for the shape");
            dbg::mlp_features(prec, mnk[3 * i], mnk[3 * i + 1], mnk[3 * i + 2], c, out + i * DBCSR_MLP_FEATURES);
        }
        dbg::set_last_error("");
        return DBCSR_OK;
    } catch (const dbg::Error& e) {
        dbg::set_last_error(e.what());
        return e.code;
    }
}

dbcsr_status dbcsr_mlp_predict_best(int32_t prec, const float* params, const int32_t* mnk, int32_t ntriples,
                                    dbcsr_kernel_cfg* best, float* best_pred) {
    try {
        if (!mnk || !best || ntriples < 1) dbg::fail(DBCSR_EINVAL, "mlp_predict_best: bad argument");
        std::vector<float> kept;
        if (!params) {
            // the model that dbcsr_predictor_train keeps for this precision
            std::lock_guard<std::mutex> lk(dbg::g_pred_mu);
            auto it = dbg::g_predictor.find(prec);
            if (it == dbg::g_predictor.end())
                dbg::fail(DBCSR_ESTATE, "mlp_predict_best: params NULL and no model trained for this precision");
            kept = it->second;
            params = kept.data();
        }
        const auto space = dbg::tune_space(prec);
        const int nf = DBCSR_MLP_FEATURES;
        const int64_t B = (int64_t)ntriples * (int64_t)space.size();
        std::vector<float> X(B * nf), Y(B);
        for (int32_t t = 0; t < ntriples; ++t)
            for (size_t c = 0; c < space.size(); ++c)
                dbg::mlp_features(prec, mnk[3 * t], mnk[3 * t + 1], mnk[3 * t + 2], space[c],
                                  X.data() + ((int64_t)t * space.size() + c) * nf);
        cudaStream_t s = nullptr;
        dbg::MlpWork w(B, nf, X.data(), nullptr, params, s);
        w.forward(s);
        DBG_CK(cudaMemcpyAsync(Y.data(), w.Y.p, sizeof(float) * B, cudaMemcpyDeviceToHost, s));
        DBG_CK(cudaStreamSynchronize(s));
        for (int32_t t = 0; t < ntriples; ++t) {
            // the lowest prediction among the configurations that apply to the triple's shape
            int64_t arg = -1;
            for (size_t c = 0; c < space.size(); ++c) {
                if (!dbg::cfg_valid(mnk[3 * t], mnk[3 * t + 1], space[c])) continue;
                if (arg < 0 || Y[t * space.size() + c] < Y[t * space.size() + arg]) arg = (int64_t)c;
            }
            const dbg::TuneCfg& b = space[arg];
            best[t] = dbcsr_kernel_cfg{b.tpb, b.ctas_per_sm, b.colmajor, b.prefetch2, b.split};
            if (best_pred) best_pred[t] = Y[t * space.size() + arg];
        }
        dbg::set_last_error("");
        return DBCSR_OK;
    } catch (const dbg::Error& e) {
        dbg::set_last_error(e.what());
        return e.code;
    }
}

int64_t dbcsr_mlp_param_count(int32_t nfeat) { return dbg::n_params(nfeat); }

dbcsr_status dbcsr_mlp_init(int32_t nfeat, uint64_t seed, float* params) {
    try {
        dbg::check_feat(nfeat, 1);
        if (!params) dbg::fail(DBCSR_EINVAL, "mlp_init: null params");
        // Glorot/Xavier uniform: U(-a, a), a = sqrt(6 / (fan_in + fan_out)); biases 0
        uint64_t s = seed;
        auto uni = [&](double a) { return (float)(((dbg::splitmix(s) >> 11) * (2.0 / 9007199254740992.0) - 1.0) * a); };
        const int H = dbg::kH;
        float* p = params;
        for (int i = 0; i < H * nfeat; ++i) *p++ = uni(std::sqrt(6.0 / (nfeat + H)));
        for (int i = 0; i < H; ++i) *p++ = 0.f;
        for (int i = 0; i < H * H; ++i) *p++ = uni(std::sqrt(6.0 / (H + H)));
        for (int i = 0; i < H; ++i) *p++ = 0.f;
        for (int i = 0; i < H; ++i) *p++ = uni(std::sqrt(6.0 / (H + 1)));
        *p++ = 0.f;
        dbg::set_last_error("");
        return DBCSR_OK;
    } catch (const dbg::Error& e) {
        dbg::set_last_error(e.what());
        return e.code;
    }
}

dbcsr_status dbcsr_mlp_forward(int32_t nfeat, const float* params, const float* X, int64_t B, float* y_out) {
    try {
        dbg::check_feat(nfeat, B);
        if (!params || !X || !y_out) dbg::fail(DBCSR_EINVAL, "mlp_forward: null argument");
        cudaStream_t s = nullptr;
        dbg::MlpWork w(B, nfeat, X, nullptr, params, s);
        w.forward(s);
        DBG_CK(cudaMemcpyAsync(y_out, w.Y.p, sizeof(float) * B, cudaMemcpyDeviceToHost, s));
        DBG_CK(cudaStreamSynchronize(s));
        dbg::set_last_error("");
        return DBCSR_OK;
    } catch (const dbg::Error& e) {
        dbg::set_last_error(e.what());
        return e.code;
    }
}

dbcsr_status dbcsr_mlp_loss_grad(int32_t nfeat, const float* params, const float* X, const float* T, int64_t B,
                                 float* loss, float* grad) {
    try {
        dbg::check_feat(nfeat, B);
        if (!params || !X || !T) dbg::fail(DBCSR_EINVAL, "mlp_loss_grad: null argument");
        cudaStream_t s = nullptr;
        dbg::MlpWork w(B, nfeat, X, T, params, s);
        w.gradient(s);
        float l = 0.f;
        DBG_CK(cudaMemcpyAsync(&l, w.loss.p, sizeof(float), cudaMemcpyDeviceToHost, s));
        if (grad)
            DBG_CK(cudaMemcpyAsync(grad, w.G.p, sizeof(float) * dbg::n_params(nfeat), cudaMemcpyDeviceToHost, s));
        DBG_CK(cudaStreamSynchronize(s));
        if (loss) *loss = l / (float)B;
        dbg::set_last_error("");
        return DBCSR_OK;
    } catch (const dbg::Error& e) {
        dbg::set_last_error(e.what());
        return e.code;
    }
}

dbcsr_status dbcsr_mlp_train(int32_t nfeat, float* params, const float* X, const float* T, int64_t B,
                             const dbcsr_mlp_opts* opts, dbcsr_mlp_report* rep) {
    try {
        dbg::check_feat(nfeat, B);
        if (!params || !X || !T || !opts) dbg::fail(DBCSR_EINVAL, "mlp_train: null argument");
        if (opts->epochs < 1 || !(opts->lr > 0)) dbg::fail(DBCSR_EINVAL, "mlp_train: need epochs >= 1 and lr > 0");
        cudaStream_t s = nullptr;
        dbg::MlpWork w(B, nfeat, X, T, params, s);
        const int64_t np = dbg::n_params(nfeat);
        cudaEvent_t e0, e1;
        DBG_CK(cudaEventCreate(&e0));
        DBG_CK(cudaEventCreate(&e1));
        DBG_CK(cudaEventRecord(e0, s));
        float first = 0.f, last = 0.f;
        for (int t = 1; t <= opts->epochs; ++t) {
            w.gradient(s);
            if (t == 1) DBG_CK(cudaMemcpyAsync(&first, w.loss.p, sizeof(float), cudaMemcpyDeviceToHost, s));
            dbg::k_adam<<<dbg::grid_for(np, 256), 256, 0, s>>>(np, w.P.p, w.G.p, w.M1.p, w.M2.p, (float)opts->lr,
                                                               (float)opts->beta1, (float)opts->beta2,
                                                               (float)opts->eps, t);
            DBG_LAUNCH_CK();
        }
        w.forward(s);
        dbg::k_mlp_backprop<<<dbg::grid_for(B, 8, dbg::num_sms() * 16), 256, 0, s>>>(B, nfeat, w.P.p, w.T.p, w.H1.p, w.H2.p,
                                                                          w.Y.p, w.DY.p, w.D2.p, w.D1.p, w.ERR.p);
        DBG_LAUNCH_CK();
        dbg::k_sum_f32<<<1, 256, 0, s>>>(B, w.ERR.p, w.loss.p);
        DBG_LAUNCH_CK();
        DBG_CK(cudaMemcpyAsync(&last, w.loss.p, sizeof(float), cudaMemcpyDeviceToHost, s));
        DBG_CK(cudaEventRecord(e1, s));
        DBG_CK(cudaMemcpyAsync(params, w.P.p, sizeof(float) * np, cudaMemcpyDeviceToHost, s));
        DBG_CK(cudaStreamSynchronize(s));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (rep) {
            rep->loss_first = first / (float)B;
            rep->loss_last = last / (float)B;
            rep->ms = ms;
            rep->epochs = opts->epochs;
        }
        dbg::set_last_error("");
        return DBCSR_OK;
    } catch (const dbg::Error& e) {
        dbg::set_last_error(e.what());
        return e.code;
    }
}

}  // extern "C"
