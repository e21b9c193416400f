// Host side of the C ABI declared in include/core_als.h: handle, workspace,
// structure validation, row planning and kernel launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "core_als.h"
#include "als_eval.h"
#include "als_fp64.cuh"
#include "als_kernels.cuh"

namespace {

using als::Counters;
using als::Params;
using als::Side;

// Row plan of one side: rows bucketed by length - warp rows (n_i <= 32, for
// widths up to 32), three CTA-resident capacities and split rows (longer than
// the largest capacity, cut into Gram chunks); each group sorted by length
// descending so the longest start first. Capacities by padded width F keep
// the staged slice plus histograms within shared memory.
struct BucketCaps {
    int cap[3];
};
BucketCaps bucket_caps(int F) {
    if (F <= 32) return {{128, 512, 1024}};
    if (F == 64) return {{128, 256, 512}};
    return {{64, 128, 256}};
}

struct Plan {
    als_tuning tuning{};
    const int64_t* indptr = nullptr;
    int64_t n_rows = 0, nnz = 0, n_cols = 0;
    int F = 0;
    int n_warp = 0;
    int n_bucket[3] = {0, 0, 0};
    int n_slots = 0, n_chunks = 0, n_super = 0;
    int64_t max_len = 0;
    std::vector<int64_t> host_indptr;  // the indptr the plan was built from
    std::vector<int32_t> blen;         // lengths of the bucket rows, in list order
    bool stale = false;                // the buffers were refilled: re-check before use
    int32_t* d_lists = nullptr;  // [warp | bucket0 | bucket1 | bucket2 | split rows | c_begin | ch_slot | ch_start
                                 //  | sc_slot | sc_start]
    void* d_split = nullptr;     // split-row selection state and scratch
    int off_bucket(int b) const {
        int o = n_warp;
        for (int q = 0; q < b; ++q) o += n_bucket[q];
        return o;
    }
    int off_split() const { return off_bucket(3); }
    int n_cta_like() const { return n_bucket[0] + n_bucket[1] + n_bucket[2] + n_slots; }
};

void free_plan(Plan& p) {
    if (p.d_lists) cudaFree(p.d_lists);
    if (p.d_split) cudaFree(p.d_split);
    p.d_lists = nullptr;
    p.d_split = nullptr;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Layout of Plan::d_split for width F (with_part false: no chunk Grams, for
// the fast variant's factor-wide selection, which assembles nothing).
struct SplitLayout {
    size_t P, Mk, need, cut, done, ghist, arrive, eqc, part, total;
    SplitLayout(int n_slots, int n_chunks, int F, bool with_part = true) {
        size_t o = 0;
        const size_t sc = (size_t)std::max(n_slots, 1) * F * 4;
        P = o; o += align256(sc);
        Mk = o; o += align256(sc);
        need = o; o += align256(sc);
        cut = o; o += align256(sc);
        done = o; o += align256(sc);
        ghist = o; o += align256(sc * 256);
        arrive = o; o += align256((size_t)std::max(n_slots, 1) * 4);
        eqc = o; o += align256((size_t)std::max(n_chunks, 1) * F * 4);
        part = o; o += with_part ? align256((size_t)std::max(n_chunks, 1) * F * (F + 1) * 4) : 256;
        total = o;
    }
};

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

// Workspace of the fast variant's factor-wide selection for a factor of
// n_cols rows at width F: the split-row selection runs on one virtual row
// that holds every row of the factor once (indices 0..n_cols-1).
struct FactorWs {
    int64_t n_cols = -1;
    int F = 0;
    void* mem = nullptr;
    int n_chunks = 0, n_super = 0;
    int64_t* vip = nullptr;     // {0, n_cols}
    int32_t* iota = nullptr;    // 0..n_cols-1
    int32_t* lists = nullptr;   // [row | c_begin | ch_slot | ch_start | sc_slot | sc_start]
    void* split = nullptr;      // SplitLayout(1, n_chunks, F, false)
};

}  // namespace

struct als_handle {
    als_options opt;
    cudaStream_t stream = nullptr;
    // Side streams of a half-sweep (the split-row chain on aux, the warp
    // rows on aux2, the solves of the CTA-resident rows' buckets on aux3,
    // beside their assembly) and their fork/join events; made on first use.
    cudaStream_t aux = nullptr, aux2 = nullptr, aux3 = nullptr;
    cudaStream_t copy = nullptr;  // host-to-device inputs of als_fit_host
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_join2 = nullptr, ev_join3 = nullptr;
    cudaEvent_t ev_bucket[3] = {nullptr, nullptr, nullptr};
    int device = 0;
    std::vector<Plan> plans;
    als_tuning tuning{0, 1, 0, 0.0};
    DevBuf g_aug;     // augmented systems of CTA rows
    DevBuf misc;      // counters + eval partials + error word
    DevBuf host_in;   // device copies for als_fit_host
    DevBuf masks;     // CES masks of the current half-sweep (FP64 fallback)
    DevBuf fb_list;   // rows flagged for the FP64 redo
    DevBuf delta;     // refinement corrections
    DevBuf perms;     // pivot permutations of the stored LU factors (n_f > 32, refinement)
    DevBuf evalbuf;   // partial sums of the objective, ReMSE and ranking kernels
    std::vector<FactorWs> fws;  // fast-variant selection workspaces (by factor size and width)
    int n_sm = 152;
    int64_t launches = 0;
    std::string last_error;
    // Kernel timing (als_profile): events bracketing each launch.
    bool profiling = false;
    struct Timed {
        const char* family;
        cudaEvent_t start, stop;
    };
    std::vector<Timed> timed;
    std::vector<cudaEvent_t> event_pool;
    const char* pending_family = nullptr;
    cudaEvent_t pending_start = nullptr;
    // Captured sweep of als_fit (one cached graph, keyed by its buffers).
    struct {
        const int64_t* ru = nullptr;
        const int64_t* ri = nullptr;
        float* U = nullptr;
        float* M = nullptr;
        cudaGraphExec_t exec = nullptr;
        int64_t launches = 0;
    } fit_graph;
};

namespace {

int set_err(als_handle* h, int code, const char* fmt, ...) {
    if (h) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        h->last_error = buf;
    }
    return code;
}

#define ALS_CUDA(h, call)                                                                       \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return set_err((h), ALS_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));   \
    } while (0)

cudaEvent_t take_event(als_handle* h) {
    if (!h->event_pool.empty()) {
        cudaEvent_t e = h->event_pool.back();
        h->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

// Marks the start of a launch of kernel family `family` (timed when
// profiling is on).
void pre_launch(als_handle* h, const char* family) {
    if (!h->profiling) return;
    h->pending_family = family;
    h->pending_start = take_event(h);
    if (h->pending_start) cudaEventRecord(h->pending_start, h->stream);
}

void post_launch(als_handle* h) {
    if (!h->profiling || !h->pending_start) return;
    cudaEvent_t stop = take_event(h);
    if (!stop) return;
    cudaEventRecord(stop, h->stream);
    h->timed.push_back({h->pending_family, h->pending_start, stop});
    h->pending_start = nullptr;
}

#define ALS_LAUNCH(h, family, ...)                                                               \
    do {                                                                                        \
        pre_launch((h), (family));                                                              \
        __VA_ARGS__;                                                                            \
        post_launch(h);                                                                         \
        (h)->launches++;                                                                        \
        cudaError_t e_ = cudaGetLastError();                                                    \
        if (e_ != cudaSuccess)                                                                  \
            return set_err((h), ALS_ERR_CUDA, "kernel launch failed: %s", cudaGetErrorString(e_)); \
    } while (0)

int ensure(als_handle* h, DevBuf& b, size_t bytes) {
    if (b.bytes >= bytes) return ALS_OK;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    size_t want = std::max(bytes, (size_t)256);
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_err(h, ALS_ERR_OOM, "cudaMalloc(%zu) failed: %s", want, cudaGetErrorString(e));
    }
    b.bytes = want;
    return ALS_OK;
}

// Padded width: 8, 16, 32 for the CUDA-core engine; 32, 64, 128 for the
// tensor-core engines (their tiles start at 32 features).
int padded_width(int f, int precision) {
    const int lo = (precision == ALS_FP32 && f <= 32) ? 8 : 32;
    int F = lo;
    while (F < f) F *= 2;
    return F <= 128 ? F : 0;
}

// Padded width the plans and kernels of a handle use (its options and tuning).
int plan_width(const ::als_handle* h);
int factor_ws(::als_handle* h, int64_t n_cols, int F, FactorWs** out);

// Gram engine for an option set: FP32 runs on CUDA cores up to 32 features
// and as split TF32 on tensor cores above; the other precisions always use
// tensor cores.
int engine_of(int precision, int F) {
    switch (precision) {
        case ALS_FP32: return F <= 32 ? als::ENG_CUDA : als::ENG_TF32X3;
        case ALS_TF32: return als::ENG_TF32;
        case ALS_BF16: return als::ENG_BF16;
        case ALS_FP32_TC: return als::ENG_TF32X3;
        default: return -1;
    }
}

Params make_params(const als_options& o) {
    Params p;
    p.f = o.n_f;
    p.lambda = o.lambda;
    p.budget = o.budget;
    p.min_keep = o.min_keep;
    p.reg_mode = o.reg_mode;
    p.gram_mode = o.gram_mode;
    p.ratio_max = (float)o.pivot_ratio_max;
    p.fixed_keep = o.fixed_keep;
    p.err = nullptr;
    p.gP = nullptr;
    p.gMk = nullptr;
    p.gcut = nullptr;
    return p;
}

int check_options(als_handle* h, const als_options* o) {
    if (!o) return set_err(h, ALS_ERR_ARG, "options are null");
    if (o->n_f < 1) return set_err(h, ALS_ERR_ARG, "n_f must be >= 1");
    if (o->n_f > 128) return set_err(h, ALS_ERR_UNSUPPORTED, "n_f > 128 is not built in this library");
    if (!(o->budget >= 0.0 && o->budget <= 1.0)) return set_err(h, ALS_ERR_ARG, "budget must be in [0, 1]");
    if (!(o->lambda >= 0.0f) || !std::isfinite(o->lambda)) return set_err(h, ALS_ERR_ARG, "lambda must be >= 0");
    if (o->reg_mode != ALS_REG_WEIGHTED && o->reg_mode != ALS_REG_PLAIN) return set_err(h, ALS_ERR_ARG, "bad reg_mode");
    if (o->gram_mode < ALS_GRAM_ASYM || o->gram_mode > ALS_GRAM_FULL) return set_err(h, ALS_ERR_ARG, "bad gram_mode");
    if (o->precision < ALS_FP32 || o->precision > ALS_FP32_TC) return set_err(h, ALS_ERR_ARG, "bad precision");
    if (o->min_keep < 0) return set_err(h, ALS_ERR_ARG, "min_keep must be >= 0");
    if (!(o->pivot_ratio_max > 0.0)) return set_err(h, ALS_ERR_ARG, "pivot_ratio_max must be > 0");
    if (o->fp64_fallback != 0 && o->fp64_fallback != 1) return set_err(h, ALS_ERR_ARG, "fp64_fallback must be 0 or 1");
    if (o->refine_steps < ALS_REFINE_AUTO || o->refine_steps > 3)
        return set_err(h, ALS_ERR_ARG, "refine_steps must be ALS_REFINE_AUTO or 0 to 3");
    if (o->fixed_keep < 0) return set_err(h, ALS_ERR_ARG, "fixed_keep must be >= 0");
    if (o->sketch != ALS_SKETCH_SLICE && o->sketch != ALS_SKETCH_FACTOR)
        return set_err(h, ALS_ERR_ARG, "sketch must be ALS_SKETCH_SLICE or ALS_SKETCH_FACTOR");
    return ALS_OK;
}

int check_csr(als_handle* h, const als_csr* R) {
    if (!R) return set_err(h, ALS_ERR_ARG, "rating structure is null");
    if (R->n_rows < 0 || R->n_cols < 0 || R->nnz < 0) return set_err(h, ALS_ERR_ARG, "negative size");
    if (R->n_rows > 0x7fffffff || R->n_cols > 0x7fffffff) return set_err(h, ALS_ERR_ARG, "more than 2^31-1 rows");
    if (!R->indptr) return set_err(h, ALS_ERR_ARG, "indptr is null");
    if (R->nnz > 0 && (!R->indices || !R->values)) return set_err(h, ALS_ERR_ARG, "indices/values are null");
    return ALS_OK;
}

Counters* counters(als_handle* h) { return reinterpret_cast<Counters*>(h->misc.p); }

int plan_width(const als_handle* h) {
    const int F = padded_width(h->opt.n_f, h->opt.precision);
    return (h->tuning.tc_gram && h->opt.precision == ALS_FP32 && F <= 32) ? 32 : F;
}
// Counters of the refinement's second solve (not reported).
Counters* scratch_counters(als_handle* h) { return reinterpret_cast<Counters*>(reinterpret_cast<char*>(h->misc.p) + 128); }
double* eval_partials(als_handle* h) {
    return reinterpret_cast<double*>(reinterpret_cast<char*>(h->misc.p) + 256);
}
double* eval_out(als_handle* h) { return eval_partials(h) + als::kEvalBlocks; }
unsigned* valid_err(als_handle* h) { return reinterpret_cast<unsigned*>(eval_out(h) + 1); }
constexpr size_t kColmaxOffset = 256 + (als::kEvalBlocks + 1) * sizeof(double) + 64;  // uint32[128]
constexpr size_t kDevErrOffset = kColmaxOffset + 128 * sizeof(uint32_t);
constexpr size_t kMiscBytes = kDevErrOffset + 16;
// Sticky device error word: bit 0 = a bounded device wait ran out. Kernels
// set it; the host reads and clears it when it synchronises for a report.
unsigned* dev_err(als_handle* h) { return reinterpret_cast<unsigned*>(static_cast<char*>(h->misc.p) + kDevErrOffset); }
// Structure check of a reused plan's buffers (k_validate bits, written
// without synchronising); read and cleared with the error word.
unsigned* reuse_err(als_handle* h) { return dev_err(h) + 1; }

// Status of a device error word value read back by the host (which then clears the word).
int dev_err_status(als_handle* h, unsigned e) {
    if (e == 0) return ALS_OK;
    ALS_CUDA(h, cudaMemsetAsync(dev_err(h), 0, sizeof(unsigned), h->stream));
    return set_err(h, ALS_ERR_TIMEOUT,
                   "a bounded device wait ran out (tensor-core completion barrier): results since the last report "
                   "are not valid");
}

// Validate one side's structure on the device and download its indptr.
int validate_csr(als_handle* h, const als_csr* R, std::vector<int64_t>& indptr) {
    cudaStream_t st = h->stream;
    ALS_CUDA(h, cudaMemsetAsync(valid_err(h), 0, sizeof(unsigned), st));
    if (R->n_rows > 0) {
        int blocks = (int)std::min<int64_t>((std::max(R->n_rows, R->nnz) + 255) / 256, (int64_t)h->n_sm * 8);
        ALS_LAUNCH(h, "validate", als::k_validate<<<blocks, 256, 0, st>>>(R->indptr, R->indices, R->values, R->n_rows, R->n_cols, R->nnz,
                                                valid_err(h)));
    }
    indptr.resize(R->n_rows + 1);
    unsigned err = 0;
    ALS_CUDA(h, cudaMemcpyAsync(indptr.data(), R->indptr, sizeof(int64_t) * (R->n_rows + 1), cudaMemcpyDeviceToHost, st));
    ALS_CUDA(h, cudaMemcpyAsync(&err, valid_err(h), sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    ALS_CUDA(h, cudaStreamSynchronize(st));
    if (indptr[0] != 0 || indptr[R->n_rows] != R->nnz) err |= 1u;
    if (err & 1u) return set_err(h, ALS_ERR_CSR, "indptr is not monotone from 0 to nnz");
    if (err & 2u) return set_err(h, ALS_ERR_CSR, "indices out of range, unsorted or duplicated inside a row");
    if (err & 4u) return set_err(h, ALS_ERR_NONFINITE, "non-finite rating value");
    return ALS_OK;
}

// *reused: the plan was found in the cache without a synchronous check; the
// caller then re-checks the indices and values on the device (asynchronously).
int build_plan(als_handle* h, const als_csr* R, Plan** out, bool* reused = nullptr) {
    std::vector<int64_t> indptr;
    bool checked = false;
    if (reused) *reused = false;
    for (size_t q = 0; q < h->plans.size(); ++q) {
        Plan& p = h->plans[q];
        if (p.indptr == R->indptr && p.n_rows == R->n_rows && p.nnz == R->nnz && p.n_cols == R->n_cols &&
            p.tuning.split_at_middle == h->tuning.split_at_middle && p.tuning.warp_rows == h->tuning.warp_rows &&
            p.tuning.tc_gram == h->tuning.tc_gram) {
            if (!p.stale) {
                *out = &p;
                if (reused) *reused = true;
                return ALS_OK;
            }
            // The buffers were refilled: validate the new contents; the plan
            // stands if the row structure (indptr) is unchanged.
            int rc = validate_csr(h, R, indptr);
            if (rc) return rc;
            checked = true;
            if (indptr == p.host_indptr) {
                // Histograms and arrival counts start from zero again (a
                // failed call may have left them dirty).
                const SplitLayout L(p.n_slots, p.n_chunks, p.F);
                ALS_CUDA(h, cudaMemsetAsync(reinterpret_cast<char*>(p.d_split) + L.ghist, 0, L.eqc - L.ghist, h->stream));
                p.stale = false;
                *out = &p;
                return ALS_OK;
            }
            free_plan(p);
            h->plans.erase(h->plans.begin() + q);
            break;
        }
    }
    if (!checked) {
        int rc = validate_csr(h, R, indptr);
        if (rc) return rc;
    }
    cudaStream_t st = h->stream;

    const int F = plan_width(h);
    const BucketCaps caps = bucket_caps(F);
    const int chunk = als::split_chunk(F);
    std::vector<int32_t> warp_rows, bucket[3], split_rows;
    int64_t max_len = 0;
    for (int64_t i = 0; i < R->n_rows; ++i) {
        const int64_t len = indptr[i + 1] - indptr[i];
        max_len = std::max(max_len, len);
        const int top = h->tuning.split_at_middle ? caps.cap[1] : caps.cap[2];
        if (len <= als::kWarpRowMax && F <= 32 && h->tuning.warp_rows) warp_rows.push_back((int32_t)i);
        else if (len <= caps.cap[0]) bucket[0].push_back((int32_t)i);
        else if (len <= caps.cap[1]) bucket[1].push_back((int32_t)i);
        else if (len <= top) bucket[2].push_back((int32_t)i);
        else split_rows.push_back((int32_t)i);
    }
    auto longer = [&](int32_t a, int32_t b) { return indptr[a + 1] - indptr[a] > indptr[b + 1] - indptr[b]; };
    // Warp rows by length too: the eight warps of a CTA then do similar work
    // (a CTA's slot frees only when its slowest warp is done).
    std::stable_sort(warp_rows.begin(), warp_rows.end(), longer);
    for (auto& v : bucket) std::stable_sort(v.begin(), v.end(), longer);
    std::stable_sort(split_rows.begin(), split_rows.end(), longer);
    std::vector<int32_t> c_begin(1, 0), ch_slot, ch_start, sc_slot, sc_start;
    for (size_t q = 0; q < split_rows.size(); ++q) {
        const int64_t len = indptr[split_rows[q] + 1] - indptr[split_rows[q]];
        for (int64_t st = 0; st < len; st += chunk) {
            ch_slot.push_back((int32_t)q);
            ch_start.push_back((int32_t)st);
        }
        for (int64_t st = 0; st < len; st += als::kSplitSuper) {
            sc_slot.push_back((int32_t)q);
            sc_start.push_back((int32_t)st);
        }
        c_begin.push_back((int32_t)ch_slot.size());
    }
    Plan p;
    p.indptr = R->indptr;
    p.n_rows = R->n_rows;
    p.nnz = R->nnz;
    p.n_cols = R->n_cols;
    p.F = F;
    p.tuning = h->tuning;
    p.n_warp = (int)warp_rows.size();
    for (int q = 0; q < 3; ++q) p.n_bucket[q] = (int)bucket[q].size();
    p.n_slots = (int)split_rows.size();
    p.n_chunks = (int)ch_slot.size();
    p.n_super = (int)sc_slot.size();
    p.max_len = max_len;
    p.host_indptr = indptr;
    for (auto& v : bucket)
        for (int32_t r : v) p.blen.push_back((int32_t)(indptr[r + 1] - indptr[r]));
    std::vector<int32_t> lists(warp_rows);
    for (auto& v : bucket) lists.insert(lists.end(), v.begin(), v.end());
    lists.insert(lists.end(), split_rows.begin(), split_rows.end());
    lists.insert(lists.end(), c_begin.begin(), c_begin.end());
    lists.insert(lists.end(), ch_slot.begin(), ch_slot.end());
    lists.insert(lists.end(), ch_start.begin(), ch_start.end());
    lists.insert(lists.end(), sc_slot.begin(), sc_slot.end());
    lists.insert(lists.end(), sc_start.begin(), sc_start.end());
    cudaError_t e = cudaMalloc(&p.d_lists, lists.size() * sizeof(int32_t));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_err(h, ALS_ERR_OOM, "cudaMalloc(plan) failed");
    }
    const SplitLayout L(p.n_slots, p.n_chunks, F);
    e = cudaMalloc(&p.d_split, L.total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_plan(p);
        return set_err(h, ALS_ERR_OOM, "cudaMalloc(split state, %zu bytes) failed", L.total);
    }
    ALS_CUDA(h, cudaMemcpyAsync(p.d_lists, lists.data(), lists.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    // The split histograms and arrival counts start (and stay between
    // passes) at zero.
    ALS_CUDA(h, cudaMemsetAsync(reinterpret_cast<char*>(p.d_split) + L.ghist, 0, L.eqc - L.ghist, st));
    ALS_CUDA(h, cudaStreamSynchronize(st));
    // Keep a small bounded cache of plans.
    if (h->plans.size() >= 8) {
        free_plan(h->plans.front());
        h->plans.erase(h->plans.begin());
        if (h->fit_graph.exec) {  // it may use the evicted plan
            cudaGraphExecDestroy(h->fit_graph.exec);
            h->fit_graph = {};
        }
    }
    h->plans.push_back(p);
    *out = &h->plans.back();
    // The fast variant's selection workspace for this side's design factor,
    // made here so that captured sweeps find it.
    if (h->opt.sketch == ALS_SKETCH_FACTOR && h->opt.gram_mode != ALS_GRAM_FULL && R->n_cols > 0) {
        FactorWs* w = nullptr;
        int rc = factor_ws(h, R->n_cols, F, &w);
        if (rc) return rc;
    }
    return ALS_OK;
}

// Resident CTAs per SM of a kCtaThreads-thread kernel with `smem` bytes of
// dynamic shared memory, from shared memory, registers and warps.
int cta_occupancy(const cudaFuncAttributes& fa, size_t smem) {
    const size_t per_sm = 233472;  // shared memory of one SM
    const size_t reserved = 1024;  // per-CTA reservation
    const int occ_smem = (int)(per_sm / (smem + fa.sharedSizeBytes + reserved));
    const int warps = als::kCtaThreads / 32;
    const int regs_per_warp = ((fa.numRegs * 32 + 255) / 256) * 256;
    const int occ_regs = regs_per_warp > 0 ? 65536 / (regs_per_warp * warps) : 8;
    return std::max(1, std::min({occ_smem, occ_regs, 64 / warps}));
}

// The handle's side streams (aux at the highest priority) and fork/join events.
int ensure_aux(als_handle* h) {
    if (h->ev_bucket[2]) return ALS_OK;
    int least = 0, greatest = 0;
    ALS_CUDA(h, cudaDeviceGetStreamPriorityRange(&least, &greatest));
    if (!h->aux) ALS_CUDA(h, cudaStreamCreateWithPriority(&h->aux, cudaStreamNonBlocking, greatest));
    if (!h->aux2) ALS_CUDA(h, cudaStreamCreateWithPriority(&h->aux2, cudaStreamNonBlocking, least));
    if (!h->aux3) ALS_CUDA(h, cudaStreamCreateWithPriority(&h->aux3, cudaStreamNonBlocking, least));
    if (!h->copy) ALS_CUDA(h, cudaStreamCreateWithPriority(&h->copy, cudaStreamNonBlocking, least));
    for (cudaEvent_t* e : {&h->ev_fork, &h->ev_join, &h->ev_join2, &h->ev_join3, &h->ev_bucket[0], &h->ev_bucket[1],
                           &h->ev_bucket[2]})
        if (!*e) ALS_CUDA(h, cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    return ALS_OK;
}

// Launch shape of a kernel that may hold tensor memory: CUDA-core engines
// get one CTA per work item; tensor-core engines a persistent grid whose
// shared-memory request is padded so that the CTAs resident on one SM never
// need more than its 512 TMEM columns (one accumulator each).
template <class K>
int tc_launch_shape(als_handle* h, K kernel, size_t smem, int eng, uint32_t tmem_cols, int count, int mode,
                    size_t* smem_out, int* grid_out) {
    *smem_out = smem;
    *grid_out = count;
    if (eng == als::ENG_CUDA || mode == 2 || count == 0) return ALS_OK;
    const int limit = std::max(1, (int)(512 / (als::kTcAccums * tmem_cols)));
    const size_t per_sm = 233472;   // shared memory of one SM
    const size_t reserved = 1024;   // per-CTA reservation
    const size_t floor_smem = per_sm / (limit + 1) - reserved + 1;
    *smem_out = std::max(smem, std::min<size_t>(floor_smem, 232448));
    ALS_CUDA(h, cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem_out));
    ALS_CUDA(h, cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared));
    cudaFuncAttributes fa;
    ALS_CUDA(h, cudaFuncGetAttributes(&fa, kernel));
    const int occ = std::min(cta_occupancy(fa, *smem_out), limit);
    *grid_out = std::min(count, h->n_sm * occ);
    return ALS_OK;
}

// One bucket of CTA-resident rows. Its rows are sorted by length, longest
// first (lens: their lengths on the host): one launch per run of rows that
// reach the same number of resident CTAs per SM, its shared memory sized for
// the run's longest row.
template <int F, int ENG>
int launch_cta_bucket(als_handle* h, const Side& side, const Params& p, const int32_t* list, const int32_t* lens,
                      int count, int mode, float* G_aug, uint32_t* masks_out, const uint32_t* tcol) {
    if (count == 0) return ALS_OK;
    using L = als::CtaLayout<F, ENG>;
    auto kern = als::k_cta_rows<F, ENG>;
    cudaFuncAttributes fa;
    ALS_CUDA(h, cudaFuncGetAttributes(&fa, kern));
    // Tensor-core engines hold TMEM: at most 512 columns' worth of accumulators per SM.
    const int limit = ENG == als::ENG_CUDA
                          ? 64
                          : std::max(1, (int)(512 / (als::kTcAccums * als::TcCfg<F, als::tc_prec(ENG)>::TMEM_COLS)));
    auto occ_of = [&](int len) { return std::min(cta_occupancy(fa, L::bytes(std::max(len, 1))), limit); };
    for (int a = 0; a < count;) {
        const int cap = std::max(lens[a], 1);
        const int occ = occ_of(cap);
        const int b = (int)(std::partition_point(lens + a, lens + count, [&](int32_t len) { return occ_of(len) == occ; }) -
                            lens);
        size_t smem = L::bytes(cap);
        ALS_CUDA(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int grid = b - a;
        if constexpr (ENG != als::ENG_CUDA) {
            int rc = tc_launch_shape(h, kern, smem, ENG, als::TcCfg<F, als::tc_prec(ENG)>::TMEM_COLS, b - a, mode,
                                     &smem, &grid);
            if (rc) return rc;
        }
        ALS_LAUNCH(h, "cta_rows", kern<<<grid, als::kCtaThreads, smem, h->stream>>>(
                                      side, p, list + a, b - a, cap, mode, G_aug + (size_t)a * F * (F + 1),
                                      masks_out, tcol));
        a = b;
    }
    return ALS_OK;
}

// Device views of a plan's split rows (chunk lists) and their state.
void split_views(const Plan& pl, int F, als::SplitPlan& sp, als::SplitState& ss) {
    const int32_t* base = pl.d_lists;
    sp.row = base + pl.off_split();
    sp.c_begin = sp.row + pl.n_slots;
    sp.ch_slot = sp.c_begin + pl.n_slots + 1;
    sp.ch_start = sp.ch_slot + pl.n_chunks;
    sp.sc_slot = sp.ch_start + pl.n_chunks;
    sp.sc_start = sp.sc_slot + pl.n_super;
    sp.n_slots = pl.n_slots;
    sp.n_chunks = pl.n_chunks;
    sp.n_super = pl.n_super;
    const SplitLayout L(pl.n_slots, pl.n_chunks, F);
    char* mem = reinterpret_cast<char*>(pl.d_split);
    ss.P = reinterpret_cast<uint32_t*>(mem + L.P);
    ss.Mk = reinterpret_cast<uint32_t*>(mem + L.Mk);
    ss.need = reinterpret_cast<int32_t*>(mem + L.need);
    ss.cut = reinterpret_cast<int32_t*>(mem + L.cut);
    ss.done = reinterpret_cast<int32_t*>(mem + L.done);
    ss.ghist = reinterpret_cast<uint32_t*>(mem + L.ghist);
    ss.arrive = reinterpret_cast<int32_t*>(mem + L.arrive);
    ss.eqc = reinterpret_cast<int32_t*>(mem + L.eqc);
    ss.part = reinterpret_cast<float*>(mem + L.part);
}

// The radix selection of the split rows (per slot and column): init, four
// histogram passes, equal-key counts, the positional cut.
template <int F>
int launch_split_select(als_handle* h, const Side& side, const Params& p, const als::SplitPlan& sp,
                        const als::SplitState& ss, const char* fam_hist) {
    cudaStream_t st = h->stream;
    const int sc = sp.n_slots * F;
    ALS_LAUNCH(h, "split_init", als::k_split_init<F><<<(sc + 255) / 256, 256, 0, st>>>(side, p, sp, ss));
    constexpr int CG = als::split_hist_cols(F);
    const size_t hsmem = (size_t)CG * als::kHistRow * 4;
    ALS_CUDA(h, cudaFuncSetAttribute(als::k_split_hist<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsmem));
    for (int pass = 0; pass < 4; ++pass) {
        ALS_LAUNCH(h, fam_hist, als::k_split_hist<F><<<sp.n_super * (F / CG), als::kCtaThreads, hsmem, st>>>(
                                    side, p, sp, ss, pass));
    }
    ALS_LAUNCH(h, "split_eqcount", als::k_split_eqcount<F><<<sp.n_chunks, als::kCtaThreads, 0, st>>>(side, p, sp, ss));
    ALS_LAUNCH(h, "split_cut", als::k_split_cut<F><<<(sc * 32 + 255) / 256, 256, 0, st>>>(side, p, sp, ss));
    return ALS_OK;
}

__global__ void k_iota(int32_t* __restrict__ dst, int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        dst[e] = (int32_t)e;
}

// The fast variant's selection workspace for a factor of n_cols rows at
// width F (built once, synchronising; a few are kept).
int factor_ws(als_handle* h, int64_t n_cols, int F, FactorWs** out) {
    for (auto& w : h->fws)
        if (w.n_cols == n_cols && w.F == F) {
            *out = &w;
            return ALS_OK;
        }
    FactorWs w;
    w.n_cols = n_cols;
    w.F = F;
    const int chunk = als::split_chunk(F);
    w.n_chunks = (int)((n_cols + chunk - 1) / chunk);
    w.n_super = (int)((n_cols + als::kSplitSuper - 1) / als::kSplitSuper);
    std::vector<int32_t> lists = {0, 0, w.n_chunks};  // row, c_begin
    for (int c = 0; c < w.n_chunks; ++c) lists.push_back(0);
    for (int c = 0; c < w.n_chunks; ++c) lists.push_back(c * chunk);
    for (int q = 0; q < w.n_super; ++q) lists.push_back(0);
    for (int q = 0; q < w.n_super; ++q) lists.push_back(q * als::kSplitSuper);
    const SplitLayout L(1, w.n_chunks, F, false);
    const size_t s_iota = align256((size_t)n_cols * 4), s_lists = align256(lists.size() * 4);
    if (cudaMalloc(&w.mem, 256 + s_iota + s_lists + L.total) != cudaSuccess) {
        cudaGetLastError();
        return set_err(h, ALS_ERR_OOM, "cudaMalloc(fast-variant selection workspace) failed");
    }
    char* base = static_cast<char*>(w.mem);
    w.vip = reinterpret_cast<int64_t*>(base);
    w.iota = reinterpret_cast<int32_t*>(base + 256);
    w.lists = reinterpret_cast<int32_t*>(base + 256 + s_iota);
    w.split = base + 256 + s_iota + s_lists;
    const int64_t vip[2] = {0, n_cols};
    cudaStream_t st = h->stream;
    int rc = ALS_OK;
    if (cudaMemcpyAsync(w.vip, vip, sizeof vip, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(w.lists, lists.data(), lists.size() * 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(static_cast<char*>(w.split) + L.ghist, 0, L.eqc - L.ghist, st) != cudaSuccess)
        rc = ALS_ERR_CUDA;
    if (rc == ALS_OK) {
        k_iota<<<(int)std::min<int64_t>((n_cols + 255) / 256, 4096), 256, 0, st>>>(w.iota, n_cols);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) rc = ALS_ERR_CUDA;
    }
    if (rc) {
        cudaGetLastError();
        cudaFree(w.mem);
        return set_err(h, rc, "building the fast-variant selection workspace failed");
    }
    if (h->fws.size() >= 4) {
        cudaStreamSynchronize(st);
        cudaFree(h->fws.front().mem);
        h->fws.erase(h->fws.begin());
    }
    h->fws.push_back(w);
    *out = &h->fws.back();
    return ALS_OK;
}

// Fast variant (Sec. 3): CES once on the whole design factor Y - the split
// selection on the virtual row of all of Y's rows, budget rule at n =
// n_cols - and its keep rule handed to every row kernel through p.
template <int F>
int launch_factor_sketch(als_handle* h, const Side& side, Params& p) {
    FactorWs* w = nullptr;
    int rc = factor_ws(h, side.n_cols, F, &w);
    if (rc) return rc;
    Side vs = side;
    vs.indptr = w->vip;
    vs.indices = w->iota;
    vs.values = nullptr;
    vs.n_rows = 1;
    als::SplitPlan sp;
    sp.row = w->lists;
    sp.c_begin = sp.row + 1;
    sp.ch_slot = sp.c_begin + 2;
    sp.ch_start = sp.ch_slot + w->n_chunks;
    sp.sc_slot = sp.ch_start + w->n_chunks;
    sp.sc_start = sp.sc_slot + w->n_super;
    sp.n_slots = 1;
    sp.n_chunks = w->n_chunks;
    sp.n_super = w->n_super;
    const SplitLayout L(1, w->n_chunks, F, false);
    char* mem = static_cast<char*>(w->split);
    als::SplitState ss;
    ss.P = reinterpret_cast<uint32_t*>(mem + L.P);
    ss.Mk = reinterpret_cast<uint32_t*>(mem + L.Mk);
    ss.need = reinterpret_cast<int32_t*>(mem + L.need);
    ss.cut = reinterpret_cast<int32_t*>(mem + L.cut);
    ss.done = reinterpret_cast<int32_t*>(mem + L.done);
    ss.ghist = reinterpret_cast<uint32_t*>(mem + L.ghist);
    ss.arrive = reinterpret_cast<int32_t*>(mem + L.arrive);
    ss.eqc = reinterpret_cast<int32_t*>(mem + L.eqc);
    ss.part = reinterpret_cast<float*>(mem + L.part);
    rc = launch_split_select<F>(h, vs, p, sp, ss, "factor_hist");
    if (rc) return rc;
    p.gP = ss.P;
    p.gMk = ss.Mk;
    p.gcut = ss.cut;
    return ALS_OK;
}

template <int F, int ENG>
int launch_split(als_handle* h, const Plan& pl, const Side& side, const Params& p, int mode, float* G_aug,
                 uint32_t* masks_out) {
    if (pl.n_slots == 0) return ALS_OK;
    cudaStream_t st = h->stream;
    als::SplitPlan sp;
    als::SplitState ss;
    split_views(pl, F, sp, ss);
    // The fast variant's rows take the factor-wide rule: no selection here.
    if (p.gP == nullptr) {
        int rc = launch_split_select<F>(h, side, p, sp, ss, "split_hist");
        if (rc) return rc;
    }
    auto gkern = als::k_split_gram<F, ENG>;
    size_t smem = sizeof(als::SplitGramSmem<F, ENG>);
    ALS_CUDA(h, cudaFuncSetAttribute(gkern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // Persistent: every resident CTA takes a contiguous range of chunks.
    int ggrid = pl.n_chunks;
    if constexpr (ENG != als::ENG_CUDA) {
        int rc = tc_launch_shape(h, gkern, smem, ENG, als::TcCfg<F, als::tc_prec(ENG)>::TMEM_COLS, pl.n_chunks, mode,
                                 &smem, &ggrid);
        if (rc) return rc;
    } else {
        int occ = 0;
        ALS_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, gkern, als::kCtaThreads, smem));
        ggrid = std::max(1, std::min(pl.n_chunks, h->n_sm * std::max(occ, 1)));
    }
    const int per = (pl.n_chunks + ggrid - 1) / ggrid;
    ggrid = (pl.n_chunks + per - 1) / per;
    ALS_LAUNCH(h, "split_gram", gkern<<<ggrid, als::kCtaThreads, smem, st>>>(side, p, sp, ss, mode, masks_out, per));
    if (mode != 2)
        ALS_LAUNCH(h, "split_reduce",
                   als::k_split_reduce<F><<<pl.n_slots, als::kCtaThreads, 0, st>>>(side, p, sp, ss, G_aug, per,
                                                                                 als::run_chunks(ENG)));
    return ALS_OK;
}

// Warp-per-row CES and Gram of the rows with at most 32 positions (n_f <= 32);
// mode 0: each warp also solves its row into X_out; 1: the systems go to aug.
template <int F>
int launch_warp_rows(als_handle* h, const Side& side, const Params& p, const int32_t* list, int count, int mode,
                     uint32_t* masks_out, float* aug, float* X_out, int32_t* flags_out, als::Fallback fb) {
    ALS_LAUNCH(h, "warp_rows", als::k_warp_rows<F><<<(count + 7) / 8, 256, 0, h->stream>>>(
                                   side, p, list, count, mode == 2, masks_out, aug, mode == 0 ? X_out : nullptr,
                                   flags_out, counters(h), fb));
    return ALS_OK;
}

// Batched solve of augmented systems listed by `list` (null: identity).
template <int F>
int launch_solve(als_handle* h, float* aug, const int32_t* list, int count, const Params& p, float* X_out,
                 int32_t* flags_out, als::Fallback fb, Counters* cnt = nullptr, int32_t* perm_buf = nullptr,
                 int replay = 0) {
    if (count == 0) return ALS_OK;
    if (cnt == nullptr) cnt = counters(h);
    if constexpr (F <= 32) {
        ALS_LAUNCH(h, "solve_rows", als::k_solve_rows<F><<<(count + 7) / 8, 256, 0, h->stream>>>(
                                        aug, list, count, p, X_out, flags_out, cnt, fb));
    } else if (replay) {
        const size_t smem = (size_t)F * (F + 1) * sizeof(float);
        ALS_CUDA(h, cudaFuncSetAttribute(als::k_solve_replay<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        ALS_LAUNCH(h, "solve_rows", als::k_solve_replay<F><<<count, 32, smem, h->stream>>>(aug, list, count, p, X_out,
                                                                                         perm_buf));
    } else {
        using C = als::RegSolve<F>;
        ALS_CUDA(h, cudaFuncSetAttribute(als::k_solve_reg<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM));
        ALS_LAUNCH(h, "solve_rows", als::k_solve_reg<F><<<count, C::NT, C::SMEM, h->stream>>>(
                                        aug, list, count, p, X_out, flags_out, cnt, fb, perm_buf, perm_buf != nullptr));
    }
    return ALS_OK;
}

// FP64 redo of the rows the solves flagged (fixed grid; reads the list
// length on the device).
template <int F>
int launch_fp64(als_handle* h, const Side& side, const Params& p, const uint32_t* masks, float* X_out,
                int32_t* flags_out) {
    const size_t smem = sizeof(als::Fp64Smem<F>);
    ALS_CUDA(h, cudaFuncSetAttribute(als::k_fp64_rows<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ALS_LAUNCH(h, "fp64_rows", als::k_fp64_rows<F><<<h->n_sm, als::kFp64Threads, smem, h->stream>>>(
                                   side, p, masks, reinterpret_cast<const int32_t*>(h->fb_list.p),
                                   &counters(h)->fb_count, X_out, flags_out, counters(h)));
    return ALS_OK;
}

// mode 0: solve into X_out; 1: assembled systems into G_out/b_out; 2: masks only.
// revalidate: the plan was reused from the cache, so the buffers' indices and
// values are checked again on the device, beside the row work.
template <int F, int ENG>
int run_side(als_handle* h, const Plan& pl, const Side& side, int mode, float* X_out, int32_t* flags_out,
             uint32_t* masks_out, float* G_out, float* b_out, bool revalidate) {
    cudaStream_t st = h->stream;
    Params p = make_params(h->opt);
    p.err = dev_err(h);
    if (h->opt.sketch == ALS_SKETCH_FACTOR && h->opt.gram_mode != ALS_GRAM_FULL && side.n_cols > 0) {
        const int src = launch_factor_sketch<F>(h, side, p);
        if (src) return src;
    }
    const int n_warp = F <= 32 ? pl.n_warp : 0;
    const int n_aug = n_warp + pl.n_cta_like();
    int rc = ensure(h, h->g_aug, (size_t)std::max(n_aug, 1) * F * (F + 1) * sizeof(float));
    if (rc) return rc;
    float* G_aug = reinterpret_cast<float*>(h->g_aug.p);
    // FP64 fallback: keep the masks and collect the flagged rows.
    als::Fallback fb{nullptr, nullptr};
    const bool fallback = mode == 0 && h->opt.fp64_fallback != 0;
    const bool refine = mode == 0 && h->opt.refine_steps > 0;
    if (fallback || refine) {
        constexpr int W = (F + 31) / 32;
        rc = ensure(h, h->masks, (size_t)std::max<int64_t>(pl.nnz, 1) * W * sizeof(uint32_t));
        if (rc) return rc;
        rc = ensure(h, h->fb_list, (size_t)std::max<int64_t>(pl.n_rows, 1) * sizeof(int32_t));
        if (rc) return rc;
        if (masks_out == nullptr) masks_out = reinterpret_cast<uint32_t*>(h->masks.p);
        if (fallback) {
            fb.rows = reinterpret_cast<int32_t*>(h->fb_list.p);
            fb.count = &counters(h)->fb_count;
        }
    }
    // Augmented systems in row-list order: [warp rows | bucket0 | bucket1 |
    // bucket2 | split slots].
    constexpr size_t FF = (size_t)F * (F + 1);
    const int nb = pl.n_bucket[0] + pl.n_bucket[1] + pl.n_bucket[2];
    const int off_split = n_warp + nb;
    float* aug_warp = G_aug;
    float* aug_b0 = aug_warp + (size_t)n_warp * FF;
    float* aug_b1 = aug_b0 + (size_t)pl.n_bucket[0] * FF;
    float* aug_b2 = aug_b1 + (size_t)pl.n_bucket[1] * FF;
    float* aug_split = aug_b2 + (size_t)pl.n_bucket[2] * FF;
    const int32_t* lists = pl.d_lists;
    // Wide systems keep their LU factors (in G_aug) and permutations when a
    // refinement follows: its corrections then need substitutions only.
    int32_t* perm_buf = nullptr;
    if (F > 32 && refine) {
        rc = ensure(h, h->perms, (size_t)std::max(n_aug, 1) * F * sizeof(int32_t));
        if (rc) return rc;
        perm_buf = reinterpret_cast<int32_t*>(h->perms.p);
    }
    // Solve of the list entries [off, off + cnt) (mode 0).
    auto solve_range = [&](int off, int cnt) -> int {
        if (mode != 0 || cnt == 0) return ALS_OK;
        return launch_solve<F>(h, G_aug + (size_t)off * FF, lists + off, cnt, p, X_out, flags_out, fb, nullptr,
                               perm_buf ? perm_buf + (size_t)off * F : nullptr);
    };
    // Three independent groups - split rows, warp rows, CTA-resident rows -
    // write disjoint systems, masks and solutions: each assembles and then
    // solves its own rows, the split-row chain (the longest dependent
    // sequence) on the handle's high-priority stream, the warp rows on a
    // second side stream, the CTA rows on the caller's stream, bucket by
    // bucket, with each bucket's solve on a third side stream as soon as it
    // is assembled (solves wait on latency, assemblies on issue slots). The
    // side streams join before the refinement. Profiling keeps one stream,
    // so that each launch's events time it alone.
    const int groups = (pl.n_slots > 0) + (n_warp > 0) + (nb > 0);
    const int buckets = (pl.n_bucket[0] > 0) + (pl.n_bucket[1] > 0) + (pl.n_bucket[2] > 0);
    const bool overlap = (groups > 1 || buckets > 1) && !h->profiling;
    if (overlap) {
        rc = ensure_aux(h);
        if (rc) return rc;
        ALS_CUDA(h, cudaEventRecord(h->ev_fork, st));
    }
    if (revalidate && pl.n_rows > 0) {
        // On the warp-row stream when the groups overlap (it finishes first).
        if (overlap) {
            ALS_CUDA(h, cudaStreamWaitEvent(h->aux2, h->ev_fork, 0));
            h->stream = h->aux2;
        }
        const int blocks = (int)std::min<int64_t>((std::max(pl.n_rows, pl.nnz) + 255) / 256, (int64_t)h->n_sm * 8);
        ALS_LAUNCH(h, "validate", als::k_validate<<<blocks, 256, 0, h->stream>>>(side.indptr, side.indices,
                                                                              side.values, pl.n_rows, pl.n_cols,
                                                                              pl.nnz, reuse_err(h)));
        h->stream = st;
    }
    if (pl.n_slots > 0) {
        if (overlap) {
            ALS_CUDA(h, cudaStreamWaitEvent(h->aux, h->ev_fork, 0));
            h->stream = h->aux;
        }
        rc = launch_split<F, ENG>(h, pl, side, p, mode, aug_split, masks_out);
        if (!rc) rc = solve_range(off_split, pl.n_slots);
        h->stream = st;
        if (rc) return rc;
        if (overlap) ALS_CUDA(h, cudaEventRecord(h->ev_join, h->aux));
    }
    if constexpr (F <= 32) {
        if (n_warp > 0) {
            if (overlap) {
                ALS_CUDA(h, cudaStreamWaitEvent(h->aux2, h->ev_fork, 0));
                h->stream = h->aux2;
            }
            rc = launch_warp_rows<F>(h, side, p, lists, n_warp, mode, masks_out, aug_warp, X_out, flags_out, fb);
            h->stream = st;
            if (rc) return rc;
            if (overlap) ALS_CUDA(h, cudaEventRecord(h->ev_join2, h->aux2));
        }
    }
    if (nb > 0) {
        // Largest exponent per factor column: the top of the resident rows' CES window.
        uint32_t* tcol = reinterpret_cast<uint32_t*>(static_cast<char*>(h->misc.p) + kColmaxOffset);
        if (p.gP == nullptr) {  // the fast variant selects nothing per row
            ALS_CUDA(h, cudaMemsetAsync(tcol, 0, (size_t)F * sizeof(uint32_t), st));
            const int64_t total = side.n_cols * (int64_t)p.f;
            const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, (int64_t)h->n_sm * 4));
            ALS_LAUNCH(h, "colmax", als::k_colmax<F><<<blocks, 256, 0, st>>>(side.Y, side.n_cols, p.f, tcol));
        }
        // At n_f <= 32 a bucket is assembled in pieces of at most kPieceRows
        // rows, each solved as soon as it is assembled: a piece's systems
        // (50 MB) are still in L2 when its solve reads them.
        constexpr int kPieceRows = 12288;
        for (int b = 2; b >= 0; --b) {
            if (pl.n_bucket[b] == 0) continue;
            float* aug = b == 2 ? aug_b2 : (b == 1 ? aug_b1 : aug_b0);
            const int piece = (F <= 32 && mode == 0) ? kPieceRows : pl.n_bucket[b];
            for (int a0 = 0; a0 < pl.n_bucket[b]; a0 += piece) {
                const int cnt = std::min(piece, pl.n_bucket[b] - a0);
                rc = launch_cta_bucket<F, ENG>(h, side, p, lists + pl.off_bucket(b) + a0,
                                               pl.blen.data() + (pl.off_bucket(b) - pl.n_warp) + a0, cnt, mode,
                                               aug + (size_t)a0 * FF, masks_out, tcol);
                if (rc) return rc;
                if (overlap && mode == 0) {
                    ALS_CUDA(h, cudaEventRecord(h->ev_bucket[b], st));
                    ALS_CUDA(h, cudaStreamWaitEvent(h->aux3, h->ev_bucket[b], 0));
                    h->stream = h->aux3;
                }
                rc = solve_range(pl.off_bucket(b) + a0, cnt);
                h->stream = st;
                if (rc) return rc;
            }
        }
        if (overlap && mode == 0) {
            ALS_CUDA(h, cudaEventRecord(h->ev_join3, h->aux3));
            ALS_CUDA(h, cudaStreamWaitEvent(st, h->ev_join3, 0));
        }
    }
    if (overlap) {
        if (pl.n_slots > 0) ALS_CUDA(h, cudaStreamWaitEvent(st, h->ev_join, 0));
        if (F <= 32 && n_warp > 0) {
            ALS_CUDA(h, cudaStreamWaitEvent(st, h->ev_join2, 0));
        } else if (revalidate && pl.n_rows > 0) {
            ALS_CUDA(h, cudaEventRecord(h->ev_join2, h->aux2));
            ALS_CUDA(h, cudaStreamWaitEvent(st, h->ev_join2, 0));
        }
    }
    if (mode == 1 && n_aug > 0)
        ALS_LAUNCH(h, "unpack_aug", als::k_unpack_aug<F><<<1024, 256, 0, st>>>(G_aug, lists, n_aug, p.f, G_out, b_out));
    // The CTA and split rows (contiguous after the warp rows) are refined;
    // warp rows always assemble in FP32 on CUDA cores.
    struct Seg { const int32_t* list; int count; float* aug; };
    const Seg segs[1] = {{lists + n_warp, pl.n_cta_like(), aug_b0}};
    if (refine) {
        // Refinement steps for the CTA and split rows: residual from the data
        // into the rhs column, a solve with the same G (for n_f > 32 the
        // stored factors: substitutions only), X += delta.
        rc = ensure(h, h->delta, (size_t)std::max<int64_t>(pl.n_rows, 1) * p.f * sizeof(float));
        if (rc) return rc;
        float* D = reinterpret_cast<float*>(h->delta.p);
        for (int step = 0; step < h->opt.refine_steps; ++step)
        for (const Seg& sg : segs) {
            if (sg.count == 0) continue;
            // Resident-bucket rows: a warp each; split rows: a CTA each.
            const int nb = pl.n_bucket[0] + pl.n_bucket[1] + pl.n_bucket[2];
            if (nb > 0)
                ALS_LAUNCH(h, "refine_resid", als::k_refine_resid_warp<F><<<(nb + 7) / 8, 256, 0, st>>>(
                                                  side, p, masks_out, sg.list, nb, sg.aug, X_out));
            if (pl.n_slots > 0) {
                // Chunk partials (FP64) in the split state's chunk-Gram scratch,
                // free once the systems are assembled; then a fixed-order sum.
                als::SplitPlan sp;
                als::SplitState ss;
                split_views(pl, F, sp, ss);
                double* part = reinterpret_cast<double*>(ss.part);
                ALS_LAUNCH(h, "refine_resid", als::k_refine_resid_chunk<F><<<pl.n_chunks, 256, 0, st>>>(
                                                  side, p, sp, masks_out, part, X_out));
                ALS_LAUNCH(h, "refine_resid", als::k_refine_resid_reduce<F><<<pl.n_slots, 128, 0, st>>>(
                                                  side, p, sp, part, sg.aug + (size_t)nb * F * (F + 1), X_out));
            }
            rc = launch_solve<F>(h, sg.aug, sg.list, sg.count, p, D, nullptr, als::Fallback{nullptr, nullptr},
                                 scratch_counters(h), perm_buf ? perm_buf + (size_t)n_warp * F : nullptr,
                                 perm_buf != nullptr);
            if (rc) return rc;
            ALS_LAUNCH(h, "add_rows", als::k_add_rows<<<std::min(1024, (sg.count * p.f + 255) / 256), 256, 0, st>>>(
                                          sg.list, sg.count, p.f, D, X_out));
        }
    }
    if (fallback) {
        rc = launch_fp64<F>(h, side, p, masks_out, X_out, flags_out);
        if (rc) return rc;
    }
    return ALS_OK;
}

// All built (width, engine) pairs.
int run_side_any(als_handle* h, const Plan& pl, const Side& side, int mode, float* X_out, int32_t* flags_out,
                 uint32_t* masks_out, float* G_out, float* b_out, bool revalidate) {
    int F = padded_width(h->opt.n_f, h->opt.precision);
    int eng = engine_of(h->opt.precision, F);
    if (h->tuning.tc_gram && h->opt.precision == ALS_FP32 && F <= 32) {
        F = 32;  // the tensor-core tiles start at 32 features
        eng = als::ENG_TF32X3;
    }
#define ALS_RUN(FF, EE)                                                                          \
    if (F == FF && eng == EE)                                                                     \
        return run_side<FF, EE>(h, pl, side, mode, X_out, flags_out, masks_out, G_out, b_out, revalidate)
    ALS_RUN(8, als::ENG_CUDA);
    ALS_RUN(16, als::ENG_CUDA);
    ALS_RUN(32, als::ENG_CUDA);
    ALS_RUN(32, als::ENG_BF16);
    ALS_RUN(32, als::ENG_TF32);
    ALS_RUN(32, als::ENG_TF32X3);
    ALS_RUN(64, als::ENG_BF16);
    ALS_RUN(64, als::ENG_TF32);
    ALS_RUN(64, als::ENG_TF32X3);
    ALS_RUN(128, als::ENG_BF16);
    ALS_RUN(128, als::ENG_TF32);
    ALS_RUN(128, als::ENG_TF32X3);
#undef ALS_RUN
    return set_err(h, ALS_ERR_UNSUPPORTED, "n_f %d with precision %d is not built", h->opt.n_f, h->opt.precision);
}

int dispatch_side(als_handle* h, const als_csr* R, const float* Y, int mode, float* X_out, int32_t* flags_out,
                  uint32_t* masks_out, float* G_out, float* b_out) {
    int rc = check_csr(h, R);
    if (rc) return rc;
    if (!Y && R->n_cols > 0) return set_err(h, ALS_ERR_ARG, "factor Y is null");
    Plan* pl = nullptr;
    bool reused = false;
    rc = build_plan(h, R, &pl, &reused);
    if (rc) return rc;
    Side side;
    side.indptr = R->indptr;
    side.indices = R->indices;
    side.values = R->values;
    side.Y = Y;
    side.n_rows = R->n_rows;
    side.n_cols = R->n_cols;
    if (mode == 0) ALS_CUDA(h, cudaMemsetAsync(counters(h), 0, sizeof(Counters), h->stream));
    return run_side_any(h, *pl, side, mode, X_out, flags_out, masks_out, G_out, b_out, reused);
}

template <int F>
int solve_systems(als_handle* h, int64_t n_rows, const float* G, const float* b, float* X_out, int32_t* flags_out) {
    cudaStream_t st = h->stream;
    Params p = make_params(h->opt);
    int rc = ensure(h, h->g_aug, (size_t)std::max<int64_t>(n_rows, 1) * F * (F + 1) * sizeof(float));
    if (rc) return rc;
    float* G_aug = reinterpret_cast<float*>(h->g_aug.p);
    ALS_CUDA(h, cudaMemsetAsync(counters(h), 0, sizeof(Counters), st));
    ALS_LAUNCH(h, "pack_aug", als::k_pack_aug<F><<<1024, 256, 0, st>>>(G, b, n_rows, p.f, G_aug));
    return launch_solve<F>(h, G_aug, nullptr, (int)n_rows, p, X_out, flags_out, als::Fallback{nullptr, nullptr});
}

}  // namespace

extern "C" {

void als_default_options(als_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->n_f = 32;
    o->lambda = 0.05f;
    o->budget = 0.25;
    o->min_keep = 0;
    o->reg_mode = ALS_REG_WEIGHTED;
    o->gram_mode = ALS_GRAM_ASYM;
    o->precision = ALS_FP32;
    o->pivot_ratio_max = 1e6;
    o->fp64_fallback = 1;
    o->refine_steps = ALS_REFINE_AUTO;
}

int als_create(als_handle** out, const als_options* opt, void* stream) {
    if (!out) return ALS_ERR_ARG;
    *out = nullptr;
    int rc = check_options(nullptr, opt);
    if (rc) return rc;
    als_handle* h = new als_handle();
    h->opt = *opt;
    if (h->opt.refine_steps == ALS_REFINE_AUTO)
        h->opt.refine_steps = opt->precision == ALS_BF16 ? 2 : (opt->precision == ALS_TF32 ? 1 : 0);
    h->stream = reinterpret_cast<cudaStream_t>(stream);
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return ALS_ERR_CUDA;
    }
    if (cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess || h->n_sm <= 0) {
        cudaGetLastError();
        h->n_sm = 152;
    }
    rc = ensure(h, h->misc, kMiscBytes);
    if (rc) {
        delete h;
        return rc;
    }
    if (cudaMemset(h->misc.p, 0, kMiscBytes) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(h->misc.p);
        delete h;
        return ALS_ERR_CUDA;
    }
    *out = h;
    return ALS_OK;
}

int als_destroy(als_handle* h) {
    if (!h) return ALS_ERR_ARG;
    cudaStreamSynchronize(h->stream);
    for (auto& p : h->plans) free_plan(p);
    for (auto& t : h->timed) {
        cudaEventDestroy(t.start);
        cudaEventDestroy(t.stop);
    }
    for (auto e : h->event_pool) cudaEventDestroy(e);
    if (h->fit_graph.exec) cudaGraphExecDestroy(h->fit_graph.exec);
    for (cudaStream_t s : {h->aux, h->aux2, h->aux3, h->copy})
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : {h->ev_fork, h->ev_join, h->ev_join2, h->ev_join3, h->ev_bucket[0], h->ev_bucket[1],
                          h->ev_bucket[2]})
        if (e) cudaEventDestroy(e);
    for (DevBuf* b : {&h->g_aug, &h->misc, &h->host_in, &h->masks, &h->fb_list, &h->delta, &h->perms, &h->evalbuf})
        if (b->p) cudaFree(b->p);
    for (auto& w : h->fws) cudaFree(w.mem);
    delete h;
    return ALS_OK;
}

int als_set_stream(als_handle* h, void* stream) {
    if (!h) return ALS_ERR_ARG;
    h->stream = reinterpret_cast<cudaStream_t>(stream);
    return ALS_OK;
}

int als_get_options(const als_handle* h, als_options* o) {
    if (!h || !o) return ALS_ERR_ARG;
    *o = h->opt;
    return ALS_OK;
}

int als_prepare(als_handle* h, const als_csr* R) {
    if (!h) return ALS_ERR_ARG;
    int rc = check_csr(h, R);
    if (rc) return rc;
    // A cached plan on these buffers is checked again, synchronously: its
    // structure is re-validated and the plan rebuilt if the rows changed.
    for (Plan& p : h->plans)
        if (p.indptr == R->indptr) p.stale = true;
    Plan* pl = nullptr;
    return build_plan(h, R, &pl);
}

int als_half_sweep(als_handle* h, const als_csr* R, const float* Y, float* X_out, int32_t* flags_out) {
    if (!h) return ALS_ERR_ARG;
    if (!X_out && R && R->n_rows > 0) return set_err(h, ALS_ERR_ARG, "X_out is null");
    return dispatch_side(h, R, Y, 0, X_out, flags_out, nullptr, nullptr, nullptr);
}

int als_select(als_handle* h, const als_csr* R, const float* Y, uint32_t* masks_out) {
    if (!h) return ALS_ERR_ARG;
    if (!masks_out && R && R->nnz > 0) return set_err(h, ALS_ERR_ARG, "masks_out is null");
    return dispatch_side(h, R, Y, 2, nullptr, nullptr, masks_out, nullptr, nullptr);
}

int als_assemble(als_handle* h, const als_csr* R, const float* Y, float* G_out, float* b_out) {
    if (!h) return ALS_ERR_ARG;
    if ((!G_out || !b_out) && R && R->n_rows > 0) return set_err(h, ALS_ERR_ARG, "G_out/b_out is null");
    return dispatch_side(h, R, Y, 1, nullptr, nullptr, nullptr, G_out, b_out);
}

int als_solve(als_handle* h, int64_t n_rows, const float* G, const float* b, float* X_out, int32_t* flags_out) {
    if (!h) return ALS_ERR_ARG;
    if (n_rows < 0 || n_rows > 0x7fffffff) return set_err(h, ALS_ERR_ARG, "bad n_rows");
    if (n_rows == 0) return ALS_OK;
    if (!G || !b || !X_out) return set_err(h, ALS_ERR_ARG, "null buffer");
    switch (padded_width(h->opt.n_f, h->opt.precision)) {
        case 8: return solve_systems<8>(h, n_rows, G, b, X_out, flags_out);
        case 16: return solve_systems<16>(h, n_rows, G, b, X_out, flags_out);
        case 32: return solve_systems<32>(h, n_rows, G, b, X_out, flags_out);
        case 64: return solve_systems<64>(h, n_rows, G, b, X_out, flags_out);
        case 128: return solve_systems<128>(h, n_rows, G, b, X_out, flags_out);
        default: return set_err(h, ALS_ERR_UNSUPPORTED, "n_f not supported");
    }
}

int als_eval_sse(als_handle* h, int64_t n, const int32_t* iu, const int32_t* im, const float* r, const float* U,
                 const float* M, double* sse_host) {
    if (!h || !sse_host) return ALS_ERR_ARG;
    if (n < 0) return set_err(h, ALS_ERR_ARG, "negative count");
    if (n == 0) {
        *sse_host = 0.0;
        return ALS_OK;
    }
    if (!iu || !im || !r || !U || !M) return set_err(h, ALS_ERR_ARG, "null buffer");
    cudaStream_t st = h->stream;
    ALS_LAUNCH(h, "sse", als::k_sse<<<als::kEvalBlocks, als::kEvalThreads, 0, st>>>(n, iu, im, r, U, M, h->opt.n_f, eval_partials(h)));
    ALS_LAUNCH(h, "sum_partials", als::k_sum_partials<<<1, 32, 0, st>>>(eval_partials(h), als::kEvalBlocks, eval_out(h)));
    ALS_CUDA(h, cudaMemcpyAsync(sse_host, eval_out(h), sizeof(double), cudaMemcpyDeviceToHost, st));
    ALS_CUDA(h, cudaStreamSynchronize(st));
    return ALS_OK;
}

int als_eval_sse_async(als_handle* h, int64_t n, const int32_t* iu, const int32_t* im, const float* r,
                       const float* U, const float* M, double* sse_dev) {
    if (!h || !sse_dev) return ALS_ERR_ARG;
    if (n < 0) return set_err(h, ALS_ERR_ARG, "negative count");
    if (n > 0 && (!iu || !im || !r || !U || !M)) return set_err(h, ALS_ERR_ARG, "null buffer");
    cudaStream_t st = h->stream;
    if (n == 0) {
        ALS_CUDA(h, cudaMemsetAsync(sse_dev, 0, sizeof(double), st));
        return ALS_OK;
    }
    ALS_LAUNCH(h, "sse", als::k_sse<<<als::kEvalBlocks, als::kEvalThreads, 0, st>>>(n, iu, im, r, U, M, h->opt.n_f,
                                                                                   eval_partials(h)));
    ALS_LAUNCH(h, "sum_partials", als::k_sum_partials<<<1, 32, 0, st>>>(eval_partials(h), als::kEvalBlocks, sse_dev));
    return ALS_OK;
}

int als_objective(als_handle* h, const als_csr* Ru, const als_csr* Ri, const float* U, const float* M,
                  double* obj_host) {
    if (!h || !obj_host) return ALS_ERR_ARG;
    int rc = check_csr(h, Ru);
    if (!rc) rc = check_csr(h, Ri);
    if (rc) return rc;
    if (Ru->n_rows != Ri->n_cols || Ru->n_cols != Ri->n_rows || Ru->nnz != Ri->nnz)
        return set_err(h, ALS_ERR_ARG, "user and item sides do not describe the same matrix");
    if ((Ru->n_rows > 0 && !U) || (Ri->n_rows > 0 && !M)) return set_err(h, ALS_ERR_ARG, "null factor");
    rc = ensure(h, h->evalbuf, (3 * als_eval::kBlocks + 8) * sizeof(double));
    if (rc) return rc;
    double* part = static_cast<double*>(h->evalbuf.p);
    double* out = part + 3 * als_eval::kBlocks;
    cudaStream_t st = h->stream;
    cudaError_t e = als_eval::objective(st, Ru->indptr, Ru->indices, Ru->values, Ru->n_rows, Ru->nnz, Ri->indptr,
                                        Ri->n_rows, U, M, h->opt.n_f, (double)h->opt.lambda,
                                        h->opt.reg_mode == ALS_REG_PLAIN ? 1 : 0, part, out);
    h->launches += 4;
    if (e != cudaSuccess) return set_err(h, ALS_ERR_CUDA, "objective launch failed: %s", cudaGetErrorString(e));
    ALS_CUDA(h, cudaMemcpyAsync(obj_host, out, sizeof(double), cudaMemcpyDeviceToHost, st));
    ALS_CUDA(h, cudaStreamSynchronize(st));
    return ALS_OK;
}

int als_eval_remse(als_handle* h, int64_t n, const int32_t* iu, const int32_t* im, const float* r, const float* U,
                   const float* M, double* remse_host) {
    if (!h || !remse_host) return ALS_ERR_ARG;
    if (n < 0) return set_err(h, ALS_ERR_ARG, "negative count");
    if (n == 0) {
        *remse_host = NAN;
        return ALS_OK;
    }
    if (!iu || !im || !r || !U || !M) return set_err(h, ALS_ERR_ARG, "null buffer");
    int rc = ensure(h, h->evalbuf, (3 * als_eval::kBlocks + 8) * sizeof(double));
    if (rc) return rc;
    double* part = static_cast<double*>(h->evalbuf.p);
    double* out = part + 3 * als_eval::kBlocks;
    cudaStream_t st = h->stream;
    cudaError_t e = als_eval::sse_and_norm(st, n, iu, im, r, U, M, h->opt.n_f, part, out);
    h->launches += 2;
    if (e != cudaSuccess) return set_err(h, ALS_ERR_CUDA, "ReMSE launch failed: %s", cudaGetErrorString(e));
    double sums[2] = {0.0, 0.0};
    ALS_CUDA(h, cudaMemcpyAsync(sums, out, sizeof sums, cudaMemcpyDeviceToHost, st));
    ALS_CUDA(h, cudaStreamSynchronize(st));
    *remse_host = sums[1] > 0.0 ? std::sqrt(sums[0]) / std::sqrt(sums[1]) : NAN;
    return ALS_OK;
}

int als_eval_ranking(als_handle* h, const als_csr* Rt, const als_csr* rel, const float* U, const float* M,
                     int k_hit, int k_ndcg, int32_t* topk_out, double* hit_host, double* ndcg_host,
                     int64_t* n_eval_host) {
    if (!h || !hit_host || !ndcg_host) return ALS_ERR_ARG;
    int rc = check_csr(h, Rt);
    if (!rc) rc = check_csr(h, rel);
    if (rc) return rc;
    if (rel->n_rows != Rt->n_rows) return set_err(h, ALS_ERR_ARG, "relevant sets must cover the same users");
    if (k_hit < 1 || k_ndcg < 1 || k_hit > als_eval::kRankMaxK || k_ndcg > als_eval::kRankMaxK)
        return set_err(h, ALS_ERR_ARG, "k_hit and k_ndcg must be in 1..%d", als_eval::kRankMaxK);
    if (Rt->n_cols > 1500000) return set_err(h, ALS_ERR_UNSUPPORTED, "more than 1,500,000 items");
    if ((Rt->n_rows > 0 && !U) || (Rt->n_cols > 0 && !M)) return set_err(h, ALS_ERR_ARG, "null factor");
    const int K = std::max(k_hit, k_ndcg);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(Rt->n_rows, (int64_t)h->n_sm * 4));
    rc = ensure(h, h->evalbuf, (3 * (size_t)std::max(grid, als_eval::kBlocks) + 8) * sizeof(double));
    if (rc) return rc;
    double* part = static_cast<double*>(h->evalbuf.p);
    double* out = part + 3 * std::max(grid, als_eval::kBlocks);
    cudaStream_t st = h->stream;
    if (Rt->n_rows == 0) {
        *hit_host = *ndcg_host = NAN;
        if (n_eval_host) *n_eval_host = 0;
        return ALS_OK;
    }
    cudaError_t e = als_eval::rank(st, grid, Rt->n_rows, Rt->n_cols, h->opt.n_f, U, M, Rt->indptr, Rt->indices,
                                   rel->indptr, rel->indices, K, k_hit, k_ndcg, topk_out, part, out);
    h->launches += 2;
    if (e != cudaSuccess) return set_err(h, ALS_ERR_CUDA, "ranking launch failed: %s", cudaGetErrorString(e));
    double sums[3] = {0.0, 0.0, 0.0};
    ALS_CUDA(h, cudaMemcpyAsync(sums, out, sizeof sums, cudaMemcpyDeviceToHost, st));
    ALS_CUDA(h, cudaStreamSynchronize(st));
    *hit_host = sums[2] > 0 ? sums[0] / sums[2] : NAN;
    *ndcg_host = sums[2] > 0 ? sums[1] / sums[2] : NAN;
    if (n_eval_host) *n_eval_host = (int64_t)sums[2];
    return ALS_OK;
}

int als_profile(als_handle* h, int enable) {
    if (!h) return ALS_ERR_ARG;
    ALS_CUDA(h, cudaStreamSynchronize(h->stream));
    for (auto& t : h->timed) {
        h->event_pool.push_back(t.start);
        h->event_pool.push_back(t.stop);
    }
    h->timed.clear();
    h->profiling = enable != 0;
    return ALS_OK;
}

int als_kernel_time(als_handle* h, const char* name, double* ms_host, int64_t* launches_host) {
    if (!h || !ms_host) return ALS_ERR_ARG;
    ALS_CUDA(h, cudaStreamSynchronize(h->stream));
    double total = 0.0;
    int64_t count = 0;
    for (auto& t : h->timed) {
        if (name && std::strcmp(name, t.family) != 0) continue;
        float ms = 0.f;
        ALS_CUDA(h, cudaEventElapsedTime(&ms, t.start, t.stop));
        total += ms;
        ++count;
    }
    *ms_host = total;
    if (launches_host) *launches_host = count;
    return ALS_OK;
}

int als_get_report(als_handle* h, als_report* rep) {
    if (!h || !rep) return ALS_ERR_ARG;
    Counters c;
    unsigned words[2] = {0u, 0u};  // error word, reused-structure check
    ALS_CUDA(h, cudaMemcpyAsync(&c, counters(h), sizeof c, cudaMemcpyDeviceToHost, h->stream));
    ALS_CUDA(h, cudaMemcpyAsync(words, dev_err(h), sizeof words, cudaMemcpyDeviceToHost, h->stream));
    ALS_CUDA(h, cudaStreamSynchronize(h->stream));
    const unsigned e = words[0];
    std::memset(rep, 0, sizeof *rep);
    rep->rows_flagged = (int64_t)c.flagged;
    rep->rows_singular = (int64_t)c.singular;
    rep->rows_fp64 = (int64_t)c.fp64_rows;
    float mr;
    std::memcpy(&mr, &c.max_ratio_bits, sizeof mr);
    rep->max_pivot_ratio = mr;
    rep->test_rmse = NAN;
    rep->objective = NAN;
    if (words[1] != 0u) {
        ALS_CUDA(h, cudaMemsetAsync(reuse_err(h), 0, sizeof(unsigned), h->stream));
        if (e) dev_err_status(h, e);  // clear it too
        if (words[1] & 3u)
            return set_err(h, ALS_ERR_CSR, "refilled buffers of a cached plan hold out-of-range, unsorted or duplicate "
                                           "indices or a bad indptr: results since the last report are not valid");
        return set_err(h, ALS_ERR_NONFINITE, "refilled buffers of a cached plan hold a non-finite rating");
    }
    return dev_err_status(h, e);
}

int als_wait_selftest(als_handle* h, int64_t limit_ns, int keep_record) {
    if (!h) return ALS_ERR_ARG;
    if (limit_ns < 0 || limit_ns > 2000000000ll) return set_err(h, ALS_ERR_ARG, "limit_ns must be in [0, 2e9]");
    ALS_LAUNCH(h, "wait_selftest", als::k_wait_selftest<<<1, 32, 0, h->stream>>>((uint64_t)limit_ns, dev_err(h)));
    if (keep_record) return ALS_OK;  // the next report-reading call returns the timeout
    unsigned e = 0;
    ALS_CUDA(h, cudaMemcpyAsync(&e, dev_err(h), sizeof e, cudaMemcpyDeviceToHost, h->stream));
    ALS_CUDA(h, cudaStreamSynchronize(h->stream));
    return dev_err_status(h, e);
}

int als_sweep(als_handle* h, const als_csr* Ru, const als_csr* Ri, float* U, float* M) {
    if (!h) return ALS_ERR_ARG;
    int rc = als_half_sweep(h, Ru, M, U, nullptr);
    if (rc) return rc;
    return als_half_sweep(h, Ri, U, M, nullptr);
}

// Capture one sweep (users, then items) on the handle's stream into an
// executable graph. Every buffer and plan it touches must already exist.
static int capture_sweep(als_handle* h, const als_csr* Ru, const als_csr* Ri, float* U, float* M,
                         cudaGraphExec_t* exec, int64_t* launches) {
    const bool prof = h->profiling;
    h->profiling = false;
    const int64_t before = h->launches;
    ALS_CUDA(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    int rc = als_sweep(h, Ru, Ri, U, M);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
    h->profiling = prof;
    *launches = h->launches - before;
    h->launches = before;
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return set_err(h, ALS_ERR_CUDA, "stream capture failed: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return set_err(h, ALS_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
    return ALS_OK;
}

int als_fit(als_handle* h, const als_csr* Ru, const als_csr* Ri, int sweeps, float* U, float* M, int64_t n_test,
            const int32_t* tu, const int32_t* tm, const float* tr, als_report* rep) {
    if (!h) return ALS_ERR_ARG;
    if (sweeps < 0) return set_err(h, ALS_ERR_ARG, "negative sweep count");
    if (!Ru || !Ri) return set_err(h, ALS_ERR_ARG, "null rating structure");
    if (Ru->n_rows != Ri->n_cols || Ru->n_cols != Ri->n_rows || Ru->nnz != Ri->nnz)
        return set_err(h, ALS_ERR_ARG, "user and item sides do not describe the same matrix");
    // First sweep directly (it builds plans and workspace), the rest from a
    // captured graph when the stream allows capture and profiling is off.
    const bool use_graph = sweeps >= 2 && h->stream != nullptr && !h->profiling;
    int done = 0;
    if (sweeps > 0) {
        int rc = als_sweep(h, Ru, Ri, U, M);
        if (rc) return rc;
        done = 1;
    }
    if (use_graph) {
        auto& g = h->fit_graph;
        if (!(g.exec && g.ru == Ru->indptr && g.ri == Ri->indptr && g.U == U && g.M == M)) {
            if (g.exec) cudaGraphExecDestroy(g.exec);
            g.exec = nullptr;
            int rc = capture_sweep(h, Ru, Ri, U, M, &g.exec, &g.launches);
            if (rc) return rc;
            g.ru = Ru->indptr;
            g.ri = Ri->indptr;
            g.U = U;
            g.M = M;
        }
        for (; done < sweeps; ++done) {
            ALS_CUDA(h, cudaGraphLaunch(g.exec, h->stream));
            h->launches += g.launches;
        }
    }
    for (; done < sweeps; ++done) {
        int rc = als_sweep(h, Ru, Ri, U, M);
        if (rc) return rc;
    }
    // Always read (and clear) the device error word: a bounded wait that ran
    // out during these sweeps must not pass as ALS_OK.
    als_report local;
    als_report* rp = rep ? rep : &local;
    int rc = als_get_report(h, rp);
    if (rc) return rc;
    if (rep) {
        rep->sweeps_done = sweeps;
        if (n_test > 0) {
            double sse = 0.0;
            rc = als_eval_sse(h, n_test, tu, tm, tr, U, M, &sse);
            if (rc) return rc;
            rep->test_rmse = std::sqrt(sse / (double)n_test);
        }
        rc = als_objective(h, Ru, Ri, U, M, &rep->objective);
        if (rc) return rc;
    }
    return ALS_OK;
}

int als_fit_host(als_handle* h, int64_t n_u, int64_t n_m, int64_t nnz, const int64_t* uip, const int32_t* uix,
                 const float* uv, const int64_t* iip, const int32_t* iix, const float* iv, int sweeps, float* U_host,
                 float* M_host, int64_t n_test, const int32_t* tu, const int32_t* tm, const float* tr,
                 als_report* rep) {
    if (!h) return ALS_ERR_ARG;
    if (n_u < 0 || n_m < 0 || nnz < 0 || n_test < 0) return set_err(h, ALS_ERR_ARG, "negative size");
    if (!uip || !iip || !U_host || !M_host) return set_err(h, ALS_ERR_ARG, "null host buffer");
    const int f = h->opt.n_f;
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t s_uip = al((n_u + 1) * 8), s_iip = al((n_m + 1) * 8), s_ix = al(nnz * 4), s_v = al(nnz * 4);
    const size_t s_U = al(n_u * f * 4), s_M = al(n_m * f * 4), s_t = al(n_test * 4);
    const size_t total = s_uip + s_iip + 2 * s_ix + 2 * s_v + s_U + s_M + 3 * s_t;
    const char* old_base = reinterpret_cast<const char*>(h->host_in.p);
    const size_t old_bytes = h->host_in.bytes;
    int rc = ensure(h, h->host_in, total);
    if (rc) return rc;
    char* base = reinterpret_cast<char*>(h->host_in.p);
    // This call refills the input buffer (perhaps moved): plans keyed on it
    // must re-check its contents before use (kept when the row structure is
    // unchanged), and the captured sweep, which may use them, is dropped.
    for (Plan& p : h->plans) {
        const char* q = reinterpret_cast<const char*>(p.indptr);
        if ((old_base && q >= old_base && q < old_base + old_bytes) || (q >= base && q < base + h->host_in.bytes))
            p.stale = true;
    }
    if (h->fit_graph.exec) {
        cudaGraphExecDestroy(h->fit_graph.exec);
        h->fit_graph = {};
    }
    auto take = [&](size_t b) { char* p = base; base += b; return p; };
    int64_t* d_uip = (int64_t*)take(s_uip);
    int64_t* d_iip = (int64_t*)take(s_iip);
    int32_t* d_uix = (int32_t*)take(s_ix);
    int32_t* d_iix = (int32_t*)take(s_ix);
    float* d_uv = (float*)take(s_v);
    float* d_iv = (float*)take(s_v);
    float* d_U = (float*)take(s_U);
    float* d_M = (float*)take(s_M);
    int32_t* d_tu = (int32_t*)take(s_t);
    int32_t* d_tm = (int32_t*)take(s_t);
    float* d_tr = (float*)take(s_t);
    cudaStream_t st = h->stream;
    if (sweeps < 0) return set_err(h, ALS_ERR_ARG, "negative sweep count");
    rc = ensure_aux(h);
    if (rc) return rc;
    // The user side and M^(0) go in on the caller's stream; the item side and
    // the test set on the copy stream (after the stream's earlier work),
    // where they are also validated while the first user half-sweep runs.
    ALS_CUDA(h, cudaEventRecord(h->ev_fork, st));
    ALS_CUDA(h, cudaStreamWaitEvent(h->copy, h->ev_fork, 0));
    ALS_CUDA(h, cudaMemcpyAsync(d_uip, uip, (n_u + 1) * 8, cudaMemcpyHostToDevice, st));
    ALS_CUDA(h, cudaMemcpyAsync(d_iip, iip, (n_m + 1) * 8, cudaMemcpyHostToDevice, h->copy));
    if (nnz > 0) {
        ALS_CUDA(h, cudaMemcpyAsync(d_uix, uix, nnz * 4, cudaMemcpyHostToDevice, st));
        ALS_CUDA(h, cudaMemcpyAsync(d_uv, uv, nnz * 4, cudaMemcpyHostToDevice, st));
        ALS_CUDA(h, cudaMemcpyAsync(d_iix, iix, nnz * 4, cudaMemcpyHostToDevice, h->copy));
        ALS_CUDA(h, cudaMemcpyAsync(d_iv, iv, nnz * 4, cudaMemcpyHostToDevice, h->copy));
    }
    ALS_CUDA(h, cudaMemcpyAsync(d_M, M_host, n_m * f * 4, cudaMemcpyHostToDevice, st));
    if (n_test > 0) {
        ALS_CUDA(h, cudaMemcpyAsync(d_tu, tu, n_test * 4, cudaMemcpyHostToDevice, h->copy));
        ALS_CUDA(h, cudaMemcpyAsync(d_tm, tm, n_test * 4, cudaMemcpyHostToDevice, h->copy));
        ALS_CUDA(h, cudaMemcpyAsync(d_tr, tr, n_test * 4, cudaMemcpyHostToDevice, h->copy));
    }
    als_csr Ru{n_u, n_m, nnz, d_uip, d_uix, d_uv};
    als_csr Ri{n_m, n_u, nnz, d_iip, d_iix, d_iv};
    int first = 0;  // sweeps done here (the first one, with the item side validated under it)
    if (sweeps > 0) {
        rc = als_half_sweep(h, &Ru, d_M, d_U, nullptr);
        if (rc == ALS_OK) {
            h->stream = h->copy;
            rc = als_prepare(h, &Ri);
            h->stream = st;
        }
        if (rc) {
            cudaStreamSynchronize(h->copy);
            return rc;
        }
        ALS_CUDA(h, cudaEventRecord(h->ev_join3, h->copy));
        ALS_CUDA(h, cudaStreamWaitEvent(st, h->ev_join3, 0));
        rc = als_half_sweep(h, &Ri, d_U, d_M, nullptr);
        if (rc) return rc;
        first = 1;
    } else {
        ALS_CUDA(h, cudaEventRecord(h->ev_join3, h->copy));
        ALS_CUDA(h, cudaStreamWaitEvent(st, h->ev_join3, 0));
    }
    als_report local;
    rc = als_fit(h, &Ru, &Ri, sweeps - first, d_U, d_M, n_test, d_tu, d_tm, d_tr, rep ? rep : &local);
    if (rc) return rc;
    if (rep) rep->sweeps_done = sweeps;
    ALS_CUDA(h, cudaMemcpyAsync(U_host, d_U, n_u * f * 4, cudaMemcpyDeviceToHost, st));
    ALS_CUDA(h, cudaMemcpyAsync(M_host, d_M, n_m * f * 4, cudaMemcpyDeviceToHost, st));
    ALS_CUDA(h, cudaStreamSynchronize(st));
    return ALS_OK;
}

int64_t als_workspace_bytes(const als_handle* h) {
    if (!h) return 0;
    int64_t b = (int64_t)(h->g_aug.bytes + h->misc.bytes + h->host_in.bytes + h->masks.bytes + h->fb_list.bytes);
    for (const auto& p : h->plans)
        b += (int64_t)SplitLayout(p.n_slots, p.n_chunks, p.F).total +
             (int64_t)(p.n_rows + 2 * p.n_chunks + 2 * p.n_super + p.n_slots + 1) * 4;
    return b;
}

int64_t als_launch_count(const als_handle* h) { return h ? h->launches : 0; }

const char* als_status_string(int s) {
    switch (s) {
        case ALS_OK: return "ok";
        case ALS_ERR_ARG: return "invalid argument";
        case ALS_ERR_CSR: return "invalid rating structure (indptr/indices)";
        case ALS_ERR_NONFINITE: return "non-finite rating value";
        case ALS_ERR_CUDA: return "CUDA runtime error";
        case ALS_ERR_TIMEOUT: return "device wait timed out";
        case ALS_ERR_OOM: return "device allocation failed";
        case ALS_ERR_DEVICE_BOUNDS: return "device bounds check fired";
        case ALS_ERR_UNSUPPORTED: return "unsupported option combination";
        default: return "unknown status";
    }
}

const char* als_last_error(const als_handle* h) { return h ? h->last_error.c_str() : "null handle"; }


}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free test SSE (als_eval_sse_static). Its FP64 block partials
// live in this file-scope device array instead of a handle's workspace.
#include <mutex>

namespace {

static __device__ __align__(256) double g_sse_static_partials[ALS_SSE_STATIC_MAX_BLOCKS];

constexpr int kStaticMaxDevices = 64;
std::mutex g_sse_static_mu;
double* g_sse_static_addr[kStaticMaxDevices] = {};
void* g_sse_static_ctx[kStaticMaxDevices] = {};  // the context each address was looked up in

// The current CUDA context (the driver's cuCtxGetCurrent, reached through the
// runtime's entry-point query so that nothing links libcuda directly).
using CtxGetCurrentFn = int (*)(void**);
void* current_context() {
    static CtxGetCurrentFn fn = nullptr;
    static bool looked = false;
    if (!looked) {
        looked = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<CtxGetCurrentFn>(p);
        else
            cudaGetLastError();
    }
    void* ctx = nullptr;
    if (fn == nullptr || fn(&ctx) != 0) return nullptr;
    return ctx;
}

// Device address of the scratch array on the current device, looked up with
// that device current (cudaGetSymbolAddress) once per (device, context): a
// new context, e.g. after cudaDeviceReset, gets a new lookup.
int sse_static_scratch(double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return ALS_ERR_CUDA;
    }
    if (dev < 0 || dev >= kStaticMaxDevices) return ALS_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_sse_static_mu);
    void* ctx = current_context();
    if (g_sse_static_addr[dev] == nullptr || ctx == nullptr || ctx != g_sse_static_ctx[dev]) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_sse_static_partials) != cudaSuccess || ptr == nullptr) {
            cudaGetLastError();
            return ALS_ERR_CUDA;
        }
        g_sse_static_addr[dev] = static_cast<double*>(ptr);
        g_sse_static_ctx[dev] = ctx;
    }
    *out = g_sse_static_addr[dev];
    return ALS_OK;
}

}  // namespace

extern "C" int als_eval_sse_static(int64_t n, const int32_t* iu, const int32_t* im, const float* r, const float* U,
                                   const float* M, int n_f, double* sse_dev, void* cuda_stream) {
    if (!sse_dev || n < 0 || n_f < 1) return ALS_ERR_ARG;
    if (n > ALS_SSE_STATIC_MAX_ENTRIES) return ALS_ERR_ARG;  // beyond the static scratch
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    if (n == 0) return cudaMemsetAsync(sse_dev, 0, sizeof(double), st) == cudaSuccess ? ALS_OK : ALS_ERR_CUDA;
    if (!iu || !im || !r || !U || !M) return ALS_ERR_ARG;
    double* partials = nullptr;
    int rc = sse_static_scratch(&partials);
    if (rc) return rc;
    const int blocks = (int)((n + ALS_SSE_STATIC_ENTRIES_PER_BLOCK - 1) / ALS_SSE_STATIC_ENTRIES_PER_BLOCK);
    als::k_sse<<<blocks, als::kEvalThreads, 0, st>>>(n, iu, im, r, U, M, n_f, partials);
    als::k_sum_partials<<<1, 32, 0, st>>>(partials, blocks, sse_dev);
    return cudaGetLastError() == cudaSuccess ? ALS_OK : ALS_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Autotuner (als_autotune).
#include <map>
#include <mutex>

namespace {

std::mutex g_tune_mu;
std::map<std::vector<int64_t>, als_tuning> g_tune_cache;

// (n_f, precision, log2 length histogram of both sides) of a problem.
int tune_key(als_handle* h, const als_csr* Ru, const als_csr* Ri, std::vector<int64_t>* key) {
    key->assign({h->opt.n_f, h->opt.precision, h->opt.gram_mode});
    for (const als_csr* R : {Ru, Ri}) {
        std::vector<int64_t> ip(R->n_rows + 1);
        ALS_CUDA(h, cudaMemcpy(ip.data(), R->indptr, ip.size() * 8, cudaMemcpyDeviceToHost));
        int64_t hist[40] = {0};
        for (int64_t i = 0; i < R->n_rows; ++i) {
            const int64_t len = ip[i + 1] - ip[i];
            int b = 0;
            while (b < 39 && (int64_t(1) << b) <= len) ++b;
            hist[b]++;
        }
        key->insert(key->end(), hist, hist + 40);
    }
    return ALS_OK;
}

}  // namespace

extern "C" int als_set_tuning(als_handle* h, const als_tuning* t) {
    if (!h || !t) return ALS_ERR_ARG;
    h->tuning = *t;
    h->tuning.split_at_middle = t->split_at_middle ? 1 : 0;
    h->tuning.warp_rows = t->warp_rows ? 1 : 0;
    h->tuning.tc_gram = t->tc_gram ? 1 : 0;
    if (h->fit_graph.exec) {
        cudaGraphExecDestroy(h->fit_graph.exec);
        h->fit_graph = {};
    }
    return ALS_OK;
}

extern "C" int als_get_tuning(const als_handle* h, als_tuning* t) {
    if (!h || !t) return ALS_ERR_ARG;
    *t = h->tuning;
    return ALS_OK;
}

extern "C" int als_autotune(als_handle* h, const als_csr* Ru, const als_csr* Ri, float* U, float* M, int trials,
                            als_tuning* chosen) {
    if (!h || !Ru || !Ri || !U || !M || trials < 1) return ALS_ERR_ARG;
    std::vector<int64_t> key;
    int rc = tune_key(h, Ru, Ri, &key);
    if (rc) return rc;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            rc = als_set_tuning(h, &it->second);
            if (!rc && chosen) *chosen = it->second;
            return rc;
        }
    }
    const bool fp32_small = h->opt.precision == ALS_FP32 && h->opt.n_f <= 32;
    std::vector<als_tuning> cands;
    for (int split = 0; split < 2; ++split)
        for (int warp = 0; warp < 2; ++warp)
            for (int tc = 0; tc < (fp32_small ? 2 : 1); ++tc) {
                if (!warp && h->opt.n_f > 32) continue;
                cands.push_back(als_tuning{split, warp, tc, 0.0});
            }
    // Keep M^(0): every trial starts from it.
    float* M0 = nullptr;
    const size_t mbytes = (size_t)Ri->n_rows * h->opt.n_f * sizeof(float);
    if (cudaMalloc(&M0, std::max<size_t>(mbytes, 4)) != cudaSuccess) {
        cudaGetLastError();
        return set_err(h, ALS_ERR_OOM, "autotune: no memory for M^(0)");
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const als_tuning saved = h->tuning;
    const bool prof = h->profiling;
    h->profiling = false;
    als_tuning best{};
    double best_ms = 1e300;
    rc = cudaMemcpyAsync(M0, M, mbytes, cudaMemcpyDeviceToDevice, h->stream) == cudaSuccess ? ALS_OK : ALS_ERR_CUDA;
    for (size_t c = 0; c < cands.size() && rc == ALS_OK; ++c) {
        rc = als_set_tuning(h, &cands[c]);
        if (!rc) rc = als_sweep(h, Ru, Ri, U, M);  // warm-up: plans and workspace
        if (rc) break;
        cudaEventRecord(e0, h->stream);
        for (int t = 0; t < trials && rc == ALS_OK; ++t) rc = als_sweep(h, Ru, Ri, U, M);
        cudaEventRecord(e1, h->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = ALS_ERR_CUDA;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        cands[c].ms_per_sweep = ms / trials;
        if (cands[c].ms_per_sweep < best_ms) {
            best_ms = cands[c].ms_per_sweep;
            best = cands[c];
        }
        if (cudaMemcpyAsync(M, M0, mbytes, cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess) rc = ALS_ERR_CUDA;
    }
    cudaStreamSynchronize(h->stream);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(M0);
    h->profiling = prof;
    if (rc) {
        als_set_tuning(h, &saved);
        return rc;
    }
    als_set_tuning(h, &best);
    h->tuning.ms_per_sweep = best_ms;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[key] = h->tuning;
    }
    if (chosen) *chosen = h->tuning;
    return ALS_OK;
}

// ---------------------------------------------------------------------------
// Batches of independent problems (als_batch_*).
namespace {

// dst[e] = src[e] + add for e < n.
__global__ void k_shift_i64(int64_t* __restrict__ dst, const int64_t* __restrict__ src, int64_t n, int64_t add) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        dst[e] = src[e] + add;
}
__global__ void k_shift_i32(int32_t* __restrict__ dst, const int32_t* __restrict__ src, int64_t n, int32_t add) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        dst[e] = src[e] + add;
}

struct BatchGroup {
    int n_f = 0;
    als_handle* h = nullptr;
    void* mem = nullptr;
    als_csr users{}, items{};
    float* U = nullptr;
    float* M = nullptr;
    std::vector<int> members;
    std::vector<int64_t> u_off, m_off;
};

}  // namespace

struct als_batch {
    cudaStream_t stream = nullptr;
    std::vector<als_problem> probs;
    std::vector<BatchGroup> groups;
    cudaGraphExec_t exec = nullptr;
    int64_t launches = 0;
};

static void batch_free(als_batch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (auto& g : b->groups) {
        if (g.h) als_destroy(g.h);
        if (g.mem) cudaFree(g.mem);
    }
    delete b;
}

extern "C" int als_batch_create(als_batch** out, const als_options* opt, int n, const als_problem* probs,
                                void* stream) {
    if (!out || !opt || n <= 0 || !probs) return ALS_ERR_ARG;
    *out = nullptr;
    if (stream == nullptr) return ALS_ERR_ARG;  // capture needs a created stream
    // The fast variant selects over a whole factor; a block-diagonal stack
    // would mix the problems' factors in one selection.
    if (opt->sketch == ALS_SKETCH_FACTOR) return ALS_ERR_UNSUPPORTED;
    als_batch* b = new als_batch();
    b->stream = reinterpret_cast<cudaStream_t>(stream);
    b->probs.assign(probs, probs + n);
    for (int q = 0; q < n; ++q) {
        const als_problem& pr = probs[q];
        if (pr.users.n_rows != pr.items.n_cols || pr.users.n_cols != pr.items.n_rows || pr.users.nnz != pr.items.nnz ||
            !pr.U || !pr.M || pr.n_f < 1) {
            batch_free(b);
            return ALS_ERR_ARG;
        }
        auto it = std::find_if(b->groups.begin(), b->groups.end(), [&](const BatchGroup& g) { return g.n_f == pr.n_f; });
        if (it == b->groups.end()) {
            b->groups.emplace_back();
            b->groups.back().n_f = pr.n_f;
            it = b->groups.end() - 1;
        }
        it->members.push_back(q);
    }
    int rc = ALS_OK;
    for (auto& g : b->groups) {
        // Offsets and sizes of the block-diagonal concatenation.
        int64_t nu = 0, nm = 0, nnz = 0;
        for (int q : g.members) {
            g.u_off.push_back(nu);
            g.m_off.push_back(nm);
            nu += probs[q].users.n_rows;
            nm += probs[q].items.n_rows;
            nnz += probs[q].users.nnz;
        }
        if (nu > 0x7fffffff || nm > 0x7fffffff) {
            rc = ALS_ERR_ARG;
            break;
        }
        auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
        const size_t s_up = al((nu + 1) * 8), s_ip = al((nm + 1) * 8), s_ix = al(nnz * 4), s_v = al(nnz * 4);
        const size_t s_U = al(nu * g.n_f * 4), s_M = al(nm * g.n_f * 4);
        if (cudaMalloc(&g.mem, s_up + s_ip + 2 * s_ix + 2 * s_v + s_U + s_M) != cudaSuccess) {
            cudaGetLastError();
            rc = ALS_ERR_OOM;
            break;
        }
        char* base = reinterpret_cast<char*>(g.mem);
        int64_t* up = reinterpret_cast<int64_t*>(base);
        int64_t* ip = reinterpret_cast<int64_t*>(base + s_up);
        int32_t* ux = reinterpret_cast<int32_t*>(base + s_up + s_ip);
        int32_t* ix = reinterpret_cast<int32_t*>(base + s_up + s_ip + s_ix);
        float* uv = reinterpret_cast<float*>(base + s_up + s_ip + 2 * s_ix);
        float* iv = reinterpret_cast<float*>(base + s_up + s_ip + 2 * s_ix + s_v);
        g.U = reinterpret_cast<float*>(base + s_up + s_ip + 2 * s_ix + 2 * s_v);
        g.M = reinterpret_cast<float*>(base + s_up + s_ip + 2 * s_ix + 2 * s_v + s_U);
        int64_t eo = 0;
        for (size_t k = 0; k < g.members.size() && rc == ALS_OK; ++k) {
            const als_problem& pr = probs[g.members[k]];
            const int64_t uo = g.u_off[k], mo = g.m_off[k], e = pr.users.nnz;
            k_shift_i64<<<256, 256, 0, b->stream>>>(up + uo, pr.users.indptr, pr.users.n_rows + 1, eo);
            k_shift_i64<<<256, 256, 0, b->stream>>>(ip + mo, pr.items.indptr, pr.items.n_rows + 1, eo);
            if (e > 0) {
                k_shift_i32<<<1024, 256, 0, b->stream>>>(ux + eo, pr.users.indices, e, (int32_t)mo);
                k_shift_i32<<<1024, 256, 0, b->stream>>>(ix + eo, pr.items.indices, e, (int32_t)uo);
                cudaMemcpyAsync(uv + eo, pr.users.values, e * 4, cudaMemcpyDeviceToDevice, b->stream);
                cudaMemcpyAsync(iv + eo, pr.items.values, e * 4, cudaMemcpyDeviceToDevice, b->stream);
            }
            if (cudaGetLastError() != cudaSuccess) rc = ALS_ERR_CUDA;
            eo += e;
        }
        if (rc) break;
        cudaMemsetAsync(g.M, 0, s_M, b->stream);
        g.users = als_csr{nu, nm, nnz, up, ux, uv};
        g.items = als_csr{nm, nu, nnz, ip, ix, iv};
        als_options o = *opt;
        o.n_f = g.n_f;
        rc = als_create(&g.h, &o, stream);
        if (rc) break;
        // One direct sweep builds the plans (validation included) and workspace.
        rc = als_prepare(g.h, &g.users);
        if (!rc) rc = als_prepare(g.h, &g.items);
        if (!rc) rc = als_sweep(g.h, &g.users, &g.items, g.U, g.M);
        if (rc) break;
    }
    if (rc == ALS_OK) {
        // Capture one sweep of every group.
        if (cudaStreamSynchronize(b->stream) != cudaSuccess ||
            cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            rc = ALS_ERR_CUDA;
        } else {
            for (auto& g : b->groups) {
                const int64_t before = g.h->launches;
                int r2 = als_sweep(g.h, &g.users, &g.items, g.U, g.M);
                b->launches += g.h->launches - before;
                g.h->launches = before;
                if (r2 && rc == ALS_OK) rc = r2;
            }
            cudaGraph_t graph = nullptr;
            if (cudaStreamEndCapture(b->stream, &graph) != cudaSuccess && rc == ALS_OK) rc = ALS_ERR_CUDA;
            if (rc == ALS_OK && cudaGraphInstantiate(&b->exec, graph, 0) != cudaSuccess) rc = ALS_ERR_CUDA;
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
        }
    }
    if (rc) {
        batch_free(b);
        return rc;
    }
    *out = b;
    return ALS_OK;
}

extern "C" int als_batch_fit(als_batch* b, int sweeps) {
    if (!b || sweeps < 0) return ALS_ERR_ARG;
    cudaStream_t st = b->stream;
    for (auto& g : b->groups)
        for (size_t k = 0; k < g.members.size(); ++k) {
            const als_problem& pr = b->probs[g.members[k]];
            if (cudaMemcpyAsync(g.M + g.m_off[k] * g.n_f, pr.M, pr.items.n_rows * g.n_f * 4, cudaMemcpyDeviceToDevice,
                                st) != cudaSuccess)
                return ALS_ERR_CUDA;
        }
    for (int t = 0; t < sweeps; ++t) {
        if (cudaGraphLaunch(b->exec, st) != cudaSuccess) return ALS_ERR_CUDA;
    }
    for (auto& g : b->groups)
        for (size_t k = 0; k < g.members.size(); ++k) {
            const als_problem& pr = b->probs[g.members[k]];
            if (cudaMemcpyAsync(pr.U, g.U + g.u_off[k] * g.n_f, pr.users.n_rows * g.n_f * 4, cudaMemcpyDeviceToDevice,
                                st) != cudaSuccess ||
                cudaMemcpyAsync(pr.M, g.M + g.m_off[k] * g.n_f, pr.items.n_rows * g.n_f * 4, cudaMemcpyDeviceToDevice,
                                st) != cudaSuccess)
                return ALS_ERR_CUDA;
        }
    // Every group's device error word: one small copy each, one synchronisation.
    std::vector<unsigned> words(b->groups.size(), 0u);
    for (size_t q = 0; q < b->groups.size(); ++q)
        if (cudaMemcpyAsync(&words[q], dev_err(b->groups[q].h), sizeof(unsigned), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess)
            return ALS_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return ALS_ERR_CUDA;
    int status = ALS_OK;
    for (size_t q = 0; q < b->groups.size(); ++q)
        if (words[q] != 0u) {
            const cudaStream_t hs = b->groups[q].h->stream;
            b->groups[q].h->stream = st;
            dev_err_status(b->groups[q].h, words[q]);  // clears the word
            b->groups[q].h->stream = hs;
            status = ALS_ERR_TIMEOUT;
        }
    return status;
}

extern "C" int64_t als_batch_launches_per_sweep(const als_batch* b) { return b ? b->launches : 0; }

extern "C" int als_batch_select(als_batch* b, int problem, int side, const float* Y, uint32_t* masks_out) {
    if (!b || problem < 0 || problem >= (int)b->probs.size() || (side != 0 && side != 1) || !Y || !masks_out)
        return ALS_ERR_ARG;
    BatchGroup* grp = nullptr;
    size_t k = 0;
    for (auto& g : b->groups)
        for (size_t q = 0; q < g.members.size(); ++q)
            if (g.members[q] == problem) {
                grp = &g;
                k = q;
            }
    if (!grp) return ALS_ERR_ARG;
    const als_problem& pr = b->probs[problem];
    const als_csr& R = side == 0 ? grp->users : grp->items;
    const int64_t other_rows = side == 0 ? pr.items.n_rows : pr.users.n_rows;
    const int64_t other_off = side == 0 ? grp->m_off[k] : grp->u_off[k];
    const int W = (grp->n_f + 31) / 32;
    int64_t e0 = 0;
    for (size_t q = 0; q < k; ++q) e0 += b->probs[grp->members[q]].users.nnz;
    // The group's design factor with this problem's rows taken from Y (the
    // other problems' rows are left as they are: rows never interact).
    float* Yg = side == 0 ? grp->M : grp->U;
    cudaStream_t st = b->stream;
    if (cudaMemcpyAsync(Yg + other_off * grp->n_f, Y, (size_t)other_rows * grp->n_f * 4, cudaMemcpyDeviceToDevice,
                        st) != cudaSuccess)
        return ALS_ERR_CUDA;
    uint32_t* all = nullptr;
    if (cudaMalloc(&all, (size_t)std::max<int64_t>(R.nnz, 1) * W * 4) != cudaSuccess) {
        cudaGetLastError();
        return ALS_ERR_OOM;
    }
    const cudaStream_t hs = grp->h->stream;
    grp->h->stream = st;
    int rc = als_select(grp->h, &R, Yg, all);
    grp->h->stream = hs;
    if (rc == ALS_OK && cudaMemcpyAsync(masks_out, all + e0 * W, (size_t)pr.users.nnz * W * 4, cudaMemcpyDeviceToDevice,
                                        st) != cudaSuccess)
        rc = ALS_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess && rc == ALS_OK) rc = ALS_ERR_CUDA;
    cudaFree(all);
    return rc;
}

extern "C" int als_batch_destroy(als_batch* b) {
    if (!b) return ALS_ERR_ARG;
    cudaStreamSynchronize(b->stream);
    batch_free(b);
    return ALS_OK;
}

