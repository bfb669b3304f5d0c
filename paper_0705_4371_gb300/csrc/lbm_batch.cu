// lbm_batch.cu -- batched form: many independent D2Q9 runs advanced
// together, replayed as CUDA graphs, with an autotuner over the launch
// strategies whose choices are cached in a JSON file.  Strategies: the
// batched kernel (per step, one stream-collide launch over the work items of
// every run and one launch of every run's selection, lbm_batch_kernels.cuh)
// with two tile shapes, or every run's own
// stream-collide kernel in concurrent graph branches (one chain of steps per
// run).  All compute identical results.
#include <algorithm>
#include <cctype>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_device.cuh"
#include "lbm_internal.h"

using namespace lbm;

namespace {

constexpr int kBatchGraphSteps = 32;   // steps per graph (even: the buffer parity returns)
constexpr int kMaxRuns = 4096;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    return run_fail(code, buf);
}

#define CK(x)                                                                                     \
    do {                                                                                          \
        cudaError_t e_ = (x);                                                                     \
        if (e_ != cudaSuccess)                                                                    \
            return fail(e_ == cudaErrorMemoryAllocation ? LB_ERR_OOM : LB_ERR_CUDA, "%s: %s", #x, \
                        cudaGetErrorString(e_));                                                  \
    } while (0)

int storage_of(int prec) {
    return prec == LB_F64 ? 0 : (prec == LB_F16_DEV ? 2 : (prec == LB_F32 ? 3 : 1));
}

}  // namespace

struct lb_batch {
    std::vector<lb_handle*> runs;
    std::vector<lb_run_desc> desc;
    int storage = 1, eq = 0, variant = 0, rows = 8;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    BatchLaunchers BL{};
    int sm_count = 0, blocks_per_sm = 1, grid = 1;
    int total_tiles = 0;
    long long total_sites = 0;
    // device arrays
    Params* d_params = nullptr;          // [2][nruns]: source buffer 0, 1
    CUtensorMap* d_tmaps = nullptr;      // [2][nruns]
    int* d_tile_base = nullptr;          // [nruns + 1]
    unsigned* d_counters = nullptr;      // [2]: the item counter of each buffer parity
    Params* h_params = nullptr;          // pinned staging of d_params
    std::vector<Params> uploaded;        // what d_params holds
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    // concurrent branches (variant 2): one stream per run, fork and join events
    std::vector<cudaStream_t> rs;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    // timing of direct launches
    bool timing = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
    double acc_ms = 0.0;
    long long acc_n = 0;
};

namespace {

int nruns(const lb_batch* b) { return (int)b->runs.size(); }

void drop_graphs(lb_batch* b) {
    for (auto& g : b->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

// Tile list, tensor maps and grid of the current variant.
int configure(lb_batch* b) {
    drop_graphs(b);
    b->BL = batch_launchers(b->storage, b->eq, std::min(b->variant, kBatchKernelVariants - 1));
    b->rows = b->BL.rows;
    int bps = 1;
    CK(b->BL.setup(&bps));
    b->blocks_per_sm = std::max(1, bps);
    const int n = nruns(b);
    std::vector<int> base(n + 1, 0);
    for (int r = 0; r < n; r++) {
        const lb_run_desc& d = b->desc[r];
        // work items of the run: its edge items (the x = 0 and x = nx - 1
        // columns, 32 x rows sites each) and its tiles
        const long long edge = ((long long)(d.nx > 1 ? 2 : 1) * d.ny + 32 * b->rows - 1) / (32 * b->rows);
        const long long t = edge + (long long)((d.nx + 127) / 128) * ((d.ny + b->rows - 1) / b->rows);
        if (base[r] + t > 0x7fffffffll) return fail(LB_ERR_ARG, "too many tiles in the batch");
        base[r + 1] = base[r] + (int)t;
    }
    b->total_tiles = base[n];
    b->grid = std::max(1, std::min(b->blocks_per_sm * b->sm_count, (b->total_tiles + 3) / 4));
    CK(cudaMemcpyAsync(b->d_tile_base, base.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice, b->stream));
    std::vector<CUtensorMap> tm(2 * (size_t)n);
    for (int c = 0; c < 2; c++)
        for (int r = 0; r < n; r++) {
            const int rc = run_tensor_map(b->runs[r], c, b->rows, &tm[(size_t)c * n + r]);
            if (rc != LB_OK) return rc;
        }
    CK(cudaMemcpyAsync(b->d_tmaps, tm.data(), tm.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice,
                       b->stream));
    CK(cudaMemsetAsync(b->d_counters, 0, 2 * sizeof(unsigned), b->stream));
    CK(cudaStreamSynchronize(b->stream));
    return LB_OK;
}

// Parameters of both source parities; the runs still holding a fresh
// (pre-collision) state get it for their parity-`first` entry.
// Copied only when they changed (a probe, a replay or a fresh state).
int upload_params(lb_batch* b, int first, bool with_prestream) {
    const int n = nruns(b);
    std::vector<Params> p(2 * (size_t)n);
    for (int c = 0; c < 2; c++)
        for (int r = 0; r < n; r++) {
            const bool pre = with_prestream && c == first && run_view(b->runs[r]).prestream;
            p[(size_t)c * n + r] = run_params(b->runs[r], c, pre);
        }
    if (b->uploaded.size() == p.size() && !std::memcmp(b->uploaded.data(), p.data(), p.size() * sizeof(Params)))
        return LB_OK;
    CK(cudaStreamSynchronize(b->stream));   // the staging buffer may still feed a copy
    std::memcpy(b->h_params, p.data(), p.size() * sizeof(Params));
    CK(cudaMemcpyAsync(b->d_params, b->h_params, p.size() * sizeof(Params), cudaMemcpyHostToDevice, b->stream));
    b->uploaded.swap(p);
    return LB_OK;
}

BatchArgs args_of(const lb_batch* b, int c) {
    const int n = nruns(b);
    BatchArgs A;
    A.P = b->d_params + (size_t)c * n;
    A.tm = b->d_tmaps + (size_t)c * n;
    A.tile_base = b->d_tile_base;
    A.nruns = n;
    A.total_tiles = b->total_tiles;
    A.tile_counter = b->d_counters + c;
    return A;
}

// Concurrent branches: every run advances `steps` steps on its own stream
// (the first one reading a fresh state where it has one), between a fork
// and a join on the batch stream.
int branches(lb_batch* b, int c, int steps, bool first_pre) {
    const int n = nruns(b);
    if (b->rs.empty()) {
        b->rs.assign(n, nullptr);
        b->join.assign(n, nullptr);
        for (int r = 0; r < n; r++) {
            CK(cudaStreamCreateWithFlags(&b->rs[r], cudaStreamNonBlocking));
            CK(cudaEventCreateWithFlags(&b->join[r], cudaEventDisableTiming));
        }
        CK(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
    }
    CK(cudaEventRecord(b->fork, b->stream));
    for (int r = 0; r < n; r++) {
        lb_handle* h = b->runs[r];
        CK(cudaStreamWaitEvent(b->rs[r], b->fork, 0));
        const bool pre = first_pre && run_view(h).prestream;
        int cc = c;
        for (int s2 = 0; s2 < steps; s2++) {
            const int rc = run_queue_step(h, cc, pre && s2 == 0, b->rs[r]);
            if (rc != LB_OK) return rc;
            cc = 1 - cc;
        }
        CK(cudaEventRecord(b->join[r], b->rs[r]));
        CK(cudaStreamWaitEvent(b->stream, b->join[r], 0));
    }
    return LB_OK;
}

int launch(lb_batch* b, int c, bool timed, bool first_pre = false) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (timed) {
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        CK(cudaEventRecord(e0, b->stream));
    }
    if (b->variant >= kBatchKernelVariants) {
        const int rc = branches(b, c, 1, first_pre);
        if (rc != LB_OK) return rc;
    } else {
        CK(b->BL.launch(args_of(b, c), b->grid, b->stream));
    }
    if (timed) {
        CK(cudaEventRecord(e1, b->stream));
        b->ev.push_back({e0, e1});
    }
    return LB_OK;
}

int build_graph(lb_batch* b, int start) {
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    int rc = LB_OK;
    if (b->variant >= kBatchKernelVariants) {
        rc = branches(b, start, kBatchGraphSteps, false);
    } else {
        int c = start;
        for (int s = 0; s < kBatchGraphSteps && rc == LB_OK; s++) {
            rc = launch(b, c, false);
            c = 1 - c;
        }
    }
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (rc != LB_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    CK(e);
    e = cudaGraphInstantiate(&b->graph[start], g, 0);
    cudaGraphDestroy(g);
    CK(e);
    return LB_OK;
}

// The runs' common buffer parity; fails when they were stepped apart.
int common_parity(lb_batch* b, int* c) {
    *c = run_view(b->runs[0]).cur;
    for (lb_handle* h : b->runs)
        if (run_view(h).cur != *c)
            return fail(LB_ERR_STATE, "the runs of a batch were stepped apart (lb_step on a single run)");
    return LB_OK;
}

int sum_times(lb_batch* b) {
    for (auto& p : b->ev) {
        float ms = 0.0f;
        CK(cudaEventSynchronize(p.second));
        CK(cudaEventElapsedTime(&ms, p.first, p.second));
        b->acc_ms += ms;
        b->acc_n++;
        cudaEventDestroy(p.first);
        cudaEventDestroy(p.second);
    }
    b->ev.clear();
    return LB_OK;
}

// Autotuner cache: a JSON object, one entry per line,
//   "key": {"variant": v, "ms_per_step": [t0, t1]}
std::string cache_key(const lb_batch* b) {
    int dev = 0;
    cudaDeviceProp prop;
    cudaGetDevice(&dev);
    cudaGetDeviceProperties(&prop, dev);
    unsigned long long h = 1469598103934665603ull;   // FNV-1a over the runs' sizes
    for (const lb_run_desc& d : b->desc) {
        const long long v[2] = {d.nx, d.ny};
        const unsigned char* p = reinterpret_cast<const unsigned char*>(v);
        for (size_t i = 0; i < sizeof(v); i++) h = (h ^ p[i]) * 1099511628211ull;
    }
    std::string name;
    for (const char* s = prop.name; *s; s++)
        name += (std::isalnum((unsigned char)*s) ? *s : '_');
    char buf[256];
    snprintf(buf, sizeof(buf), "%s_sm%d_s%d_e%d_n%d_%016llx", name.c_str(), prop.multiProcessorCount,
             b->storage, b->eq, nruns(b), h);
    return buf;
}

bool cache_lookup(const char* path, const std::string& key, int* variant) {
    std::ifstream f(path);
    if (!f) return false;
    std::string line;
    const std::string pat = "\"" + key + "\": {\"variant\": ";
    while (std::getline(f, line)) {
        const size_t at = line.find(pat);
        if (at == std::string::npos) continue;
        const int v = std::atoi(line.c_str() + at + pat.size());
        if (v >= 0 && v < kBatchVariants) {
            *variant = v;
            return true;
        }
    }
    return false;
}

bool cache_store(const char* path, const std::string& key, int variant, const double* ms) {
    std::vector<std::string> entries;
    {
        std::ifstream f(path);
        std::string line;
        while (f && std::getline(f, line)) {
            const size_t q = line.find('"');
            if (q == std::string::npos || line.find("\"" + key + "\"") != std::string::npos) continue;
            std::string e = line.substr(q);
            while (!e.empty() && (e.back() == ',' || e.back() == ' ')) e.pop_back();
            entries.push_back(e);
        }
    }
    std::ostringstream e;
    e << "\"" << key << "\": {\"variant\": " << variant << ", \"ms_per_step\": [";
    for (int v = 0; v < kBatchVariants; v++) e << (v ? ", " : "") << ms[v];
    e << "]}";
    entries.push_back(e.str());
    std::ofstream o(path, std::ios::trunc);
    if (!o) return false;
    o << "{\n";
    for (size_t i = 0; i < entries.size(); i++) o << "  " << entries[i] << (i + 1 < entries.size() ? "," : "") << "\n";
    o << "}\n";
    return (bool)o;
}

}  // namespace

extern "C" {

int lb_batch_create(const lb_run_desc* runs, int n, void* cuda_stream, lb_batch** out) {
    if (!out) return fail(LB_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!runs || n < 1 || n > kMaxRuns) return fail(LB_ERR_ARG, "need 1 to %d runs", kMaxRuns);
    for (int r = 0; r < n; r++) {
        const lb_run_desc& d = runs[r];
        if (d.lattice != LB_D2Q9) return fail(LB_ERR_ARG, "run %d: the batched form is built for D2Q9", r);
        if (d.equilibrium != LB_EQ_POLY && d.equilibrium != LB_EQ_ENTROPIC)
            return fail(LB_ERR_ARG, "run %d: the batched form runs the polynomial and entropic equilibria", r);
        if (d.equilibrium != runs[0].equilibrium || d.precision != runs[0].precision)
            return fail(LB_ERR_ARG, "run %d: every run of a batch has the same equilibrium and precision", r);
    }
    lb_batch* b = new lb_batch();
    b->desc.assign(runs, runs + n);
    b->storage = storage_of(runs[0].precision);
    b->eq = runs[0].equilibrium;
    auto bail = [&](int rc) {
        lb_batch_destroy(b);
        return rc;
    };
    if (cuda_stream) {
        b->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess)
            return bail(fail(LB_ERR_CUDA, "cudaStreamCreate failed"));
        b->own_stream = true;
    }
    for (int r = 0; r < n; r++) {
        const lb_run_desc& d = runs[r];
        lb_handle* h = nullptr;
        int rc = lb_create(d.lattice, d.nx, d.ny, d.equilibrium, d.nu, d.delta, d.k, &d.bc, d.precision,
                           b->stream, &h);
        if (rc != LB_OK) return bail(rc);
        b->runs.push_back(h);
        // the runs' own kernels (concurrent branches, sequential steps) take
        // 8-row staged tiles with 16 warps per SM: the fastest measured for
        // many small grids side by side (6-row tiles, the single large grid's
        // default, leave too few warps)
        rc = lb_set_tile_shape(h, 4);
        if (rc != LB_OK) return bail(rc);
        b->total_sites += (long long)d.nx * d.ny;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return bail(fail(LB_ERR_CUDA, "device query failed"));
    if (cudaMalloc(&b->d_params, 2 * (size_t)n * sizeof(Params)) != cudaSuccess ||
        cudaMalloc(&b->d_tmaps, 2 * (size_t)n * sizeof(CUtensorMap)) != cudaSuccess ||
        cudaMalloc(&b->d_tile_base, (n + 1) * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&b->d_counters, 2 * sizeof(unsigned)) != cudaSuccess ||
        cudaMallocHost(&b->h_params, 2 * (size_t)n * sizeof(Params)) != cudaSuccess)
        return bail(fail(LB_ERR_OOM, "batch allocation failed"));
    const int rc = configure(b);
    if (rc != LB_OK) return bail(rc);
    *out = b;
    return LB_OK;
}

void lb_batch_destroy(lb_batch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_graphs(b);
    for (auto& p : b->ev) {
        cudaEventDestroy(p.first);
        cudaEventDestroy(p.second);
    }
    for (cudaStream_t st : b->rs)
        if (st) cudaStreamDestroy(st);
    for (cudaEvent_t ev : b->join)
        if (ev) cudaEventDestroy(ev);
    if (b->fork) cudaEventDestroy(b->fork);
    for (lb_handle* h : b->runs) lb_destroy(h);
    if (b->d_params) cudaFree(b->d_params);
    if (b->d_tmaps) cudaFree(b->d_tmaps);
    if (b->d_tile_base) cudaFree(b->d_tile_base);
    if (b->d_counters) cudaFree(b->d_counters);
    if (b->h_params) cudaFreeHost(b->h_params);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

lb_handle* lb_batch_run(lb_batch* b, int r) {
    if (!b || r < 0 || r >= nruns(b)) return nullptr;
    return b->runs[r];
}

int lb_batch_step(lb_batch* b, int n) {
    if (!b) return fail(LB_ERR_ARG, "NULL batch");
    if (n < 0) return fail(LB_ERR_ARG, "n must be >= 0");
    if (n == 0) return LB_OK;
    for (lb_handle* h : b->runs) {
        const int rc = run_check(h);
        if (rc != LB_OK) return rc;
    }
    int c = 0;
    int rc = common_parity(b, &c);
    if (rc != LB_OK) return rc;
    bool any_pre = false;
    for (lb_handle* h : b->runs) any_pre |= run_view(h).prestream;
    rc = upload_params(b, c, any_pre);
    if (rc != LB_OK) return rc;
    int done = 0;
    if (any_pre) {
        // first step after a state upload: the fresh runs read their own sites
        rc = launch(b, c, b->timing, true);
        if (rc != LB_OK) return rc;
        c = 1 - c;
        done = 1;
        rc = upload_params(b, c, false);
        if (rc != LB_OK) return rc;
    }
    while (done < n) {
        if (!b->timing && n - done >= kBatchGraphSteps) {
            if (!b->graph[c]) {
                rc = build_graph(b, c);
                if (rc != LB_OK) return rc;
            }
            CK(cudaGraphLaunch(b->graph[c], b->stream));
            done += kBatchGraphSteps;
        } else {
            rc = launch(b, c, b->timing);
            if (rc != LB_OK) return rc;
            c = 1 - c;
            done++;
        }
    }
    for (lb_handle* h : b->runs) {
        run_advance(h, n);
        rc = run_queue_err(h);
        if (rc != LB_OK) return rc;
    }
    return LB_OK;
}

int lb_batch_step_sequential(lb_batch* b, int n) {
    if (!b) return fail(LB_ERR_ARG, "NULL batch");
    for (lb_handle* h : b->runs) {
        const int rc = lb_step(h, n);
        if (rc != LB_OK) return rc;
    }
    return LB_OK;
}

int lb_batch_sync(lb_batch* b) {
    if (!b) return fail(LB_ERR_ARG, "NULL batch");
    for (lb_handle* h : b->runs) {
        const int rc = lb_sync(h);
        if (rc != LB_OK) return rc;
    }
    return LB_OK;
}

int lb_batch_set_variant(lb_batch* b, int variant) {
    if (!b) return fail(LB_ERR_ARG, "NULL batch");
    if (variant < 0 || variant >= kBatchVariants)
        return fail(LB_ERR_ARG, "variant must be in [0, %d)", kBatchVariants);
    CK(cudaStreamSynchronize(b->stream));
    b->variant = variant;
    return configure(b);
}

int lb_batch_set_timing(lb_batch* b, int enable) {
    if (!b) return fail(LB_ERR_ARG, "NULL batch");
    b->timing = enable != 0;
    return LB_OK;
}

int lb_batch_kernel_times(lb_batch* b, double* ms, long long* launches, int reset) {
    if (!b) return fail(LB_ERR_ARG, "NULL batch");
    const int rc = sum_times(b);
    if (rc != LB_OK) return rc;
    if (ms) *ms = b->acc_ms;
    if (launches) *launches = b->acc_n;
    if (reset) {
        b->acc_ms = 0.0;
        b->acc_n = 0;
    }
    return LB_OK;
}

int lb_batch_autotune(lb_batch* b, int steps, const char* cache_path, int* variant_out) {
    if (!b) return fail(LB_ERR_ARG, "NULL batch");
    if (steps < 1) return fail(LB_ERR_ARG, "steps must be >= 1");
    const std::string key = cache_key(b);
    int v = -1;
    if (cache_path && cache_lookup(cache_path, key, &v)) {
        const int rc = lb_batch_set_variant(b, v);
        if (rc != LB_OK) return rc;
        if (variant_out) *variant_out = v;
        return LB_OK;
    }
    // Each strategy is timed as it runs in production: whole graphs of
    // kBatchGraphSteps steps (steps rounded up to whole graphs), after one
    // graph of warm-up, with events on the batch's stream.
    double ms[kBatchVariants];
    const bool timing = b->timing;
    b->timing = false;
    const int graphs = std::max(1, (steps + kBatchGraphSteps - 1) / kBatchGraphSteps);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        b->timing = timing;
        return fail(LB_ERR_CUDA, "cudaEventCreate failed");
    }
    int rc = lb_batch_step(b, 1);   // leaves a fresh state's first step out of the timing
    for (int t = 0; t < kBatchVariants && rc == LB_OK; t++) {
        rc = lb_batch_set_variant(b, t);
        if (rc == LB_OK) rc = lb_batch_step(b, kBatchGraphSteps);   // warm-up (builds the graph)
        if (rc != LB_OK) break;
        float el = 0.0f;
        if (cudaEventRecord(e0, b->stream) != cudaSuccess) rc = fail(LB_ERR_CUDA, "cudaEventRecord failed");
        if (rc == LB_OK) rc = lb_batch_step(b, graphs * kBatchGraphSteps);
        if (rc == LB_OK && (cudaEventRecord(e1, b->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                            cudaEventElapsedTime(&el, e0, e1) != cudaSuccess))
            rc = fail(LB_ERR_CUDA, "autotune timing failed");
        ms[t] = rc == LB_OK ? (double)el / (graphs * kBatchGraphSteps) : 1e30;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->timing = timing;
    if (rc != LB_OK) return rc;
    v = (int)(std::min_element(ms, ms + kBatchVariants) - ms);
    rc = lb_batch_set_variant(b, v);
    if (rc != LB_OK) return rc;
    if (cache_path && !cache_store(cache_path, key, v, ms))
        return fail(LB_ERR_ARG, "cannot write the autotuner cache %s", cache_path);
    if (variant_out) *variant_out = v;
    return LB_OK;
}

int lb_batch_info(lb_batch* b, long long* out) {
    if (!b || !out) return fail(LB_ERR_ARG, "NULL argument");
    out[0] = nruns(b);
    out[1] = b->total_sites;
    out[2] = b->total_tiles;
    out[3] = b->grid;
    out[4] = b->blocks_per_sm;
    out[5] = b->variant;
    out[6] = b->rows;
    out[7] = kBatchGraphSteps;
    return LB_OK;
}

}  // extern "C"

namespace lbm {

BatchLaunchers batch_launchers(int storage, int eq, int variant) {
    if (storage == 0) return batch_launchers_f64(eq, variant);
    if (storage == 2) return batch_launchers_f16(eq, variant);
    if (storage == 3) return batch_launchers_f32p(eq, variant);
    return batch_launchers_f32(eq, variant);
}

}  // namespace lbm
