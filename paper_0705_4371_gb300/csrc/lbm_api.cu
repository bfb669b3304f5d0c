// lbm_api.cu -- C ABI (include/lbm.h): handle lifecycle, argument checks,
// device memory, step scheduling (direct launches or CUDA graphs), logs and
// the sticky error word.  All compute runs in the kernels of
// lbm_kernels_*.cu; this file only allocates, validates and launches.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "../../include/lbm.h"
#include "lbm_device.cuh"
#include "lbm_internal.h"
#include "lbm_mlp.cuh"

using namespace lbm;

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

#define CK(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(e_ == cudaErrorMemoryAllocation ? LB_ERR_OOM : LB_ERR_CUDA,     \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

constexpr int kGraphSteps = 32;      // steps per captured graph (even: buffers return)
constexpr int kExportChunks = 8;     // row chunks of a host export (copies overlap the conversion)
constexpr int kXferEvents = 16;      // events of one chunked transfer (>= Q planes, >= chunks, + 1)
constexpr int kDefaultLog = 65536;
// Default tile shapes, the fastest measured on GB300: FP32 and FP16 storage
// (plain and deviation) stage 6-row tiles with 2 more in flight per block
// (shape 5; FP16 at 1000 steps of the 4096 x 2048 cylinder: 90.8 k MLUPS
// against 86.8 k with 8-row tiles at three blocks per SM); FP64 storage
// 8-row tiles with 1 more (shape 4).  Small polynomial-f* FP32 grids (up to 600 000 sites:
// one or two staged tiles per resident block, a step of ~20 us dominated by
// latency) run faster register-fed (shape 1): the 600 x 500 channel 15.7 k
// against 13.0 k MLUPS, 1024 x 512 23.2 k against 22.2 k; from 1536 x 768
// on shape 5 is ahead (34.3 k against 31.1 k), and FP16 storage is fastest
// on shape 5 at every size measured.  The energy forms are bound by the Newton solve, not
// by memory: FP64 storage's FP64 finish wants the most resident warps
// (register-fed shape 1); the float-float finish of FP32 / FP16 storage and
// the network's warm start run best in the staged shape 4 (measured at
// 2048 x 1024: Newton start 0.22 ms per step against 0.44 on shape 0 and 0.24
// on shape 5; warm start 0.35 against 0.54 and 0.35).
int default_tile_shape(int lattice, int eq, int precision, long long sites) {
    if (lattice != LB_D2Q9) return 0;
    if (eq < LB_EQ_ENTROPIC_ENERGY) {
        if (precision == LB_F64) return 4;
        if (eq == LB_EQ_POLY && precision != LB_F16_DEV && sites <= 600000) return 1;
        return 5;
    }
    if (precision == LB_F64) return 1;
    return 4;
}

size_t storage_bytes(int prec) { return prec == LB_F64 ? 8 : (prec == LB_F16_DEV ? 2 : 4); }

// Half-width of the band around delta in which the precision form decides
// dS > delta in FP64 rather than in FP32.  The FP32 evaluation of f* leaves
// an error |e_i| <= ~1e-7 W_i in each nonequilibrium component d_i = f_i - f*_i
// (a few roundings of quantities below 0.6 W_i); with dS ~ sum d_i^2 / (2 f*_i),
// its first-order effect on dS is sum |d_i| e_i / f*_i <= 1e-7 sum |d_i| <=
// 1e-7 sqrt(2 rho dS) ~ 1.5e-7 sqrt(dS) near rho = 1, the second-order one is
// below 1e-13, and the FP32 sum itself is within ~1e-6 dS.  The band takes
// twenty times the first-order term, a relative 1e-3 and an absolute 1e-12.
double recheck_band(double delta) {
    const double a = std::fabs(delta);
    return 1e-3 * a + 3e-6 * std::sqrt(a) + 1e-12;
}

}  // namespace

void lbm::set_last_error(const char* msg) { g_last_error = msg; }

struct lb_handle {
    int lattice, Q, nx, ny, nxp, eq, prec, k;
    double nu, beta, delta, rho0;
    lb_boundaries bc;
    cudaStream_t stream;
    bool own_stream;
    Launchers L;
    void* buf[2];
    int cur;                  // buffer holding the current state
    bool prestream;           // current buffer holds pre-collision populations
    long long plane;
    // selection
    unsigned long long* cand_key;
    unsigned* cand_idx;
    unsigned* cand_count;
    long long cand_cap;
    int cand_per_block;
    int* sel_idx;
    int* sel_count;
    long long sel_cap;
    // logs
    int* count_ring;
    double* probe_ring;
    int ring_cap;
    int probe_x, probe_y;
    long long* d_step;
    long long h_step;         // steps queued so far
    unsigned* d_err;
    unsigned* h_err;          // pinned copy
    cudaEvent_t err_ev;
    bool err_ev_pending;
    // replay
    int* replay_cnt;
    long long* replay_off;
    int* replay_idx;
    long long replay_t0, replay_n;
    // graph of kGraphSteps steps starting from buffer 0 (graph_exec[0]) or 1
    cudaGraphExec_t graph_exec[2];
    // timing
    bool timing;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, int>> ev_pairs[2];   // (start, stop) indices per kind
    size_t ev_next;
    double acc_ms[2];
    long long acc_n[2];
    // energy form; the learned form's network (FP32 master copy on the device)
    float* mlp;
    bool mlp_set;
    bool elbm;                // ELBM collision (elbmLB)
    // device staging of FP64 host fields (state import/export, initial
    // fields): allocated on first use and kept, since mapping hundreds of MB
    // per call costs more than the copy itself
    double* stage;
    size_t stage_bytes;
    // streams of the host copies of those transfers (created with the
    // staging buffers), uploads and downloads apart, and the events that
    // order them with the conversion kernels on the run's stream: chunk by
    // chunk, so that one chunk's copy overlaps the conversion of the next
    // (import) or the previous (export).  Downloads have staging of their own
    // (stage_out), so an upload can overlap a download; d2h_done marks the
    // end of the last download, which the next export waits for before
    // overwriting stage_out, and imp_done the end of the last upload's
    // conversions, the only readers of stage, which the next upload's
    // copies wait for.
    cudaStream_t copy_stream, d2h_stream;
    cudaEvent_t xfer_ev[kXferEvents], out_ev[kXferEvents], d2h_done, imp_done;
    double* stage_out;
    size_t stage_out_bytes;
    bool d2h_pending, imp_pending;
    unsigned long long* newton_stats;
    // completion ticket of the stream-collide blocks; tile shape of K1
    unsigned* ticket;
    int tile_shape;
    // overflow list of sites awaiting an exact dS
    unsigned* pend_idx;
    unsigned* pend_count;
    int grid_blocks, sm_count, blocks_per_sm;
    // tensor maps of the two population buffers (shared-memory-staged shapes)
    CUtensorMap tmap[2];
    unsigned* tile_counter;
    // claim order of the staged shapes' tiles: boundary tiles first; two
    // orders of tile_order_n claims, by the parity of the buffer read
    int* tile_order;
    int tile_order_n;
    // slab of a run sharded in x: ghost columns on each side, global x of the
    // first owned column, global nx; the keys of the slab's best candidates;
    // the step's selection among the slab's sites (one replayed step)
    int slab, ghost_l, ghost_r, gx0, gnx;
    bool slab_collided;
    unsigned long long* sel_key;
    int* slab_sel;
    int* slab_cnt;
    long long* slab_off;
};

namespace {

// Inlet populations f*(rho_in, u_in) (Sec. 4.2) in FP64 with the kernels'
// own formulas, converted as the storage holds them: FP64 f; FP32 and FP16
// deviation storage the FP32 value of f - W_i (the FP32 arithmetic of both);
// plain FP32 the FP32 value of f minus the FP32 weight.
template <typename L>
void inlet_values_of(const lb_handle* h, double* gin) {
    double fs[9] = {0};
    feq_rho_u<L, double>(h->eq, h->bc.rho_in, h->bc.u_in[0], h->bc.u_in[1], 0.0, fs);
    for (int i = 0; i < 9; i++) gin[i] = 0.0;
    for (int i = 0; i < L::Q; i++) {
        if (h->prec == LB_F64) gin[i] = fs[i];
        else if (h->prec == LB_F32) gin[i] = (double)((float)fs[i] - (float)L::w(i));
        else gin[i] = (double)(float)(fs[i] - L::w(i));
    }
}
void inlet_values(const lb_handle* h, double* gin) {
    if (h->lattice == LB_D1Q3) inlet_values_of<D1Q3>(h, gin);
    else inlet_values_of<D2Q9>(h, gin);
}

Params make_params(const lb_handle* h, int src, bool prestream) {
    Params P;
    memset(&P, 0, sizeof(P));
    P.nx = h->nx; P.ny = h->ny; P.nxp = h->nxp; P.plane = h->plane;
    P.eq = h->eq; P.beta = h->beta; P.delta = h->delta; P.rho0 = h->rho0; P.k = h->k;
    P.betaf = (float)h->beta; P.rho0f = (float)h->rho0;
    // FP32 threshold: the largest float not above delta, so that a site with
    // FP32 dS > deltaf has dS > delta up to the FP32 rounding of dS itself
    P.deltaf = (float)h->delta;
    if ((double)P.deltaf > h->delta) P.deltaf = std::nextafter(P.deltaf, -INFINITY);
    P.bc[0] = h->bc.kind_x0; P.bc[1] = h->bc.kind_x1; P.bc[2] = h->bc.kind_y0; P.bc[3] = h->bc.kind_y1;
    P.rho_in = h->bc.rho_in; P.ux_in = h->bc.u_in[0]; P.uy_in = h->bc.u_in[1];
    P.ox0 = h->bc.obstacle_x0; P.oy0 = h->bc.obstacle_y0; P.ow = h->bc.obstacle_w; P.oh = h->bc.obstacle_h;
    inlet_values(h, P.gin);
    P.src = h->buf[src];
    P.dst = h->buf[1 - src];
    P.prestream = prestream ? 1 : 0;
    P.cand_key = h->cand_key; P.cand_idx = h->cand_idx; P.cand_count = h->cand_count;
    P.cand_per_block = h->cand_per_block;
    P.sel_idx = h->sel_idx; P.sel_count = h->sel_count;
    P.count_ring = h->count_ring; P.probe_ring = h->probe_x >= 0 ? h->probe_ring : nullptr;
    P.ring_cap = h->ring_cap; P.probe_x = h->probe_x; P.probe_y = h->probe_y;
    P.step = h->d_step; P.err = h->d_err;
    P.replay_cnt = h->replay_cnt; P.replay_off = h->replay_off; P.replay_idx = h->replay_idx;
    P.replay_t0 = h->replay_t0; P.replay_n = h->replay_n;
    P.recheck = (h->prec == LB_F32_DEV || h->prec == LB_F16_DEV) ? 1 : 0;
    P.recheck_band = recheck_band(h->delta);
    P.mlp = h->mlp; P.newton_stats = h->newton_stats;
    P.ticket = h->ticket;
    P.pend_idx = h->pend_idx;
    P.pend_count = h->pend_count;
    P.grid_blocks = h->grid_blocks;
    P.tile_counter = h->tile_counter;
    P.tile_order = h->tile_order ? h->tile_order + (src ? h->tile_order_n : 0) : nullptr;
    P.elbm = h->elbm ? 1 : 0;
    P.wall = h->bc.obstacle_wall;
    P.slab = h->slab;
    P.own_x0 = h->slab ? h->ghost_l : 0;
    P.own_x1 = h->slab ? h->nx - h->ghost_r : h->nx;
    P.sel_key = h->slab ? h->sel_key : nullptr;
    return P;
}

void drop_graphs(lb_handle* h) {
    for (int i = 0; i < 2; i++) {
        if (h->graph_exec[i]) cudaGraphExecDestroy(h->graph_exec[i]);
        h->graph_exec[i] = nullptr;
    }
}

int check_sticky(lb_handle* h, bool wait) {
    if (h->err_ev_pending) {
        cudaError_t q = wait ? cudaEventSynchronize(h->err_ev) : cudaEventQuery(h->err_ev);
        if (q == cudaErrorNotReady) return LB_OK;
        CK(q);
    }
    const unsigned e = *h->h_err;
    if (e & ERR_NONFINITE) return fail(LB_ERR_NONFINITE, "non-finite moments appeared");
    if (e & ERR_NEWTON) return fail(LB_ERR_NEWTON, "a Newton solve did not reach 1e-12");
    if (e & ERR_TIMEOUT) return fail(LB_ERR_TIMEOUT, "a bounded device wait gave up");
    if (e & ERR_REPLAY) return fail(LB_ERR_ARG, "a replayed site index was out of range or solid");
    return LB_OK;
}

int queue_err_readback(lb_handle* h) {
    CK(cudaMemcpyAsync(h->h_err, h->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaEventRecord(h->err_ev, h->stream));
    h->err_ev_pending = true;
    return LB_OK;
}

cudaEvent_t next_event(lb_handle* h) {
    if (h->ev_next >= h->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        h->ev_pool.push_back(e);
    }
    return h->ev_pool[h->ev_next++];
}

// Queue one time step reading buffer src: a single launch (the last block
// of the stream-collide kernel performs the selection and the Ehrenfests'
// step).
int queue_step(lb_handle* h, int src, bool prestream, bool timed) {
    const Params P = make_params(h, src, prestream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (timed) {
        e0 = next_event(h);
        e1 = next_event(h);
        if (!e0 || !e1) return fail(LB_ERR_CUDA, "cudaEventCreate failed");
        CK(cudaEventRecord(e0, h->stream));
    }
    CK(h->L.collide(P, h->tile_shape, &h->tmap[src], h->stream));
    if (timed) {
        CK(cudaEventRecord(e1, h->stream));
        h->ev_pairs[0].push_back({(int)h->ev_next - 2, (int)h->ev_next - 1});
    }
    return LB_OK;
}

int build_graph(lb_handle* h, int start) {
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    int rc = LB_OK;
    int src = start;
    for (int s = 0; s < kGraphSteps && rc == LB_OK; s++) {
        rc = queue_step(h, src, false, false);
        src = 1 - src;
    }
    cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    if (rc != LB_OK) { if (g) cudaGraphDestroy(g); return rc; }
    CK(e);
    e = cudaGraphInstantiate(&h->graph_exec[start], g, 0);
    cudaGraphDestroy(g);
    CK(e);
    return LB_OK;
}

bool valid_kind(int k) { return k >= LB_BB && k <= LB_OUTLET_COPY; }

// Tensor map describing population buffer b as a 3-D array (x: nx, y: ny,
// plane: Q) for staged tiles of R = rows rows: box = (cols + 2 H) x R x 1
// elements, H = 16 bytes of halo on each side (each plane's copy starts at
// the row its populations are pulled from); coordinates outside the array
// read as zero.
int encode_tensor_map(const lb_handle* h, int b, int rows, int cols, CUtensorMap* out) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                         cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
            return fail(LB_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const size_t es = storage_bytes(h->prec);
    const CUtensorMapDataType dt = h->prec == LB_F64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                   : h->prec == LB_F16_DEV ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                           : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const cuuint64_t gdim[3] = {(cuuint64_t)h->nx, (cuuint64_t)h->ny, (cuuint64_t)h->Q};
    const cuuint64_t gstride[2] = {(cuuint64_t)h->nxp * es, (cuuint64_t)h->plane * es};
    const cuuint32_t box[3] = {(cuuint32_t)(cols + 2 * (16 / es)), (cuuint32_t)rows, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = encode(out, dt, 3, h->buf[b], gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(LB_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return LB_OK;
}

// Claim order of the staged tiles (rows x cols sites).  The tiles that take
// the rule-by-rule path (the grid's first and last rows, a ragged last
// column of tiles, the obstacle and its neighbours; the same test as the
// kernel's, whose columns x = 0 and x = nx - 1 go apart) cost several times an
// interior tile: they are spread evenly over the first three quarters of
// the claims, where they overlap interior tiles that keep the memory busy,
// and the last claims are interior tiles of equal cost, so that the blocks
// run out of work together.  Both kinds keep their row-major order, except
// that with reverse the interior tiles come in the opposite order: the steps
// that read buffer 1 use that order, so that each step starts on the tiles
// the previous step wrote last, while they are still in L2 (4096 x 2048:
// 75.2 k against 74.2 k MLUPS).
std::vector<int> staged_tile_order(const lb_handle* h, int rows, int cols, bool reverse) {
    const int tiles_x = (h->nx + cols - 1) / cols, tiles_y = (h->ny + rows - 1) / rows;
    const lb_boundaries& b = h->bc;
    std::vector<int> slow, fast;
    for (int ty = 0; ty < tiles_y; ty++)
        for (int tx = 0; tx < tiles_x; tx++) {
            const int x0 = tx * cols, y0 = ty * rows;
            const bool clean = x0 + cols <= h->nx && y0 >= 1 && y0 + rows <= h->ny - 1 &&
                               (b.obstacle_w == 0 || x0 + cols + 1 <= b.obstacle_x0 ||
                                x0 - 1 >= b.obstacle_x0 + b.obstacle_w || y0 + rows + 1 <= b.obstacle_y0 ||
                                y0 - 1 >= b.obstacle_y0 + b.obstacle_h);
            (clean ? fast : slow).push_back(ty * tiles_x + tx);
        }
    if (reverse) std::reverse(fast.begin(), fast.end());
    const size_t n = slow.size() + fast.size();
    const size_t span = std::max(slow.size(), n * 3 / 4);   // claims the slow tiles are spread over
    std::vector<int> order;
    order.reserve(n);
    size_t js = 0, jf = 0;
    for (size_t c = 0; c < n; c++) {
        // slow tile j goes to claim floor(j * span / nslow)
        const bool take_slow = js < slow.size() && c >= js * span / slow.size();
        if (take_slow || jf == fast.size()) order.push_back(slow[js++]);
        else order.push_back(fast[jf++]);
    }
    return order;
}

int make_tensor_maps(lb_handle* h) {
    const int rows = staged_rows(h->tile_shape);
    if (h->lattice != LB_D2Q9 || rows == 0) return LB_OK;
    const int cols = staged_cols(h->tile_shape);
    for (int b = 0; b < 2; b++) {
        const int rc = encode_tensor_map(h, b, rows, cols, &h->tmap[b]);
        if (rc != LB_OK) return rc;
    }
    std::vector<int> order = staged_tile_order(h, rows, cols, false);
    const std::vector<int> back = staged_tile_order(h, rows, cols, true);
    h->tile_order_n = (int)order.size();
    order.insert(order.end(), back.begin(), back.end());
    if (h->tile_order) cudaFree(h->tile_order);
    h->tile_order = nullptr;
    CK(cudaMalloc(&h->tile_order, order.size() * sizeof(int)));
    CK(cudaMemcpy(h->tile_order, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice));
    return LB_OK;
}

// Persistent grid of the stream-collide kernel: resident blocks per SM for
// the tile shape (occupancy calculator) times the SM count.
int size_grid(lb_handle* h) {
    int dev = 0, bps = 1;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, dev));
    CK(h->L.occupancy(h->tile_shape, &bps));
    h->blocks_per_sm = bps < 1 ? 1 : bps;
    h->grid_blocks = h->blocks_per_sm * h->sm_count;
    return LB_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// What the batched form (lbm_batch.cu) needs of a run.
// ---------------------------------------------------------------------------
namespace lbm {

RunView run_view(const lb_handle* h) {
    RunView v;
    v.lattice = h->lattice;
    v.nx = h->nx;
    v.ny = h->ny;
    v.eq = h->eq;
    v.prec = h->prec;
    v.cur = h->cur;
    v.prestream = h->prestream;
    v.replaying = h->replay_n > 0 && h->h_step < h->replay_t0 + h->replay_n;
    v.step = h->h_step;
    v.stream = h->stream;
    return v;
}

Params run_params(const lb_handle* h, int src, bool prestream) { return make_params(h, src, prestream); }

int run_tensor_map(const lb_handle* h, int buf, int rows, CUtensorMap* out) {
    return encode_tensor_map(h, buf, rows, 128, out);
}

void run_advance(lb_handle* h, long long n) {
    h->h_step += n;
    if (n & 1) h->cur = 1 - h->cur;
    if (n > 0) h->prestream = false;
}

int run_queue_step(lb_handle* h, int src, bool prestream, cudaStream_t st) {
    Params P = make_params(h, src, prestream);
    // beside the batch's other runs (concurrent graph branches) a small run
    // keeps to few blocks, at least four 1024-site tiles each, instead of
    // spreading over the whole GPU as it does when stepped alone
    const long long cap = std::max(1ll, ((long long)h->nx * h->ny + 4095) / 4096);
    P.grid_blocks = (int)std::min((long long)P.grid_blocks, cap);
    CK(h->L.collide(P, h->tile_shape, &h->tmap[src], st));
    return LB_OK;
}

int run_check(lb_handle* h) { return check_sticky(h, false); }

int run_queue_err(lb_handle* h) { return queue_err_readback(h); }

int run_fail(int code, const char* msg) { return fail(code, "%s", msg); }

}  // namespace lbm

extern "C" {

const char* lb_last_error(void) { return g_last_error.c_str(); }

void lb_destroy(lb_handle* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->copy_stream) {
        // transfers still queued read or write the staging buffers freed below
        cudaStreamSynchronize(h->copy_stream);
        cudaStreamSynchronize(h->d2h_stream);
    }
    drop_graphs(h);
    void* ptrs[] = {h->buf[0], h->buf[1], h->cand_key, h->cand_idx, h->cand_count, h->sel_idx,
                    h->sel_count, h->count_ring, h->probe_ring, h->d_step, h->d_err, h->replay_cnt,
                    h->replay_off, h->replay_idx, h->mlp, h->newton_stats, h->ticket,
                    h->pend_idx, h->pend_count, h->tile_counter, h->tile_order, h->stage, h->sel_key,
                    h->slab_sel, h->slab_cnt, h->slab_off};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (h->h_err) cudaFreeHost(h->h_err);
    if (h->err_ev) cudaEventDestroy(h->err_ev);
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    if (h->copy_stream) {
        for (cudaEvent_t e : h->xfer_ev)
            if (e) cudaEventDestroy(e);
        for (cudaEvent_t e : h->out_ev)
            if (e) cudaEventDestroy(e);
        if (h->d2h_done) cudaEventDestroy(h->d2h_done);
        if (h->imp_done) cudaEventDestroy(h->imp_done);
        cudaStreamDestroy(h->copy_stream);
        cudaStreamDestroy(h->d2h_stream);
    }
    if (h->stage_out) cudaFree(h->stage_out);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

int lb_create(int lattice, int nx, int ny, int equilibrium, double nu, double delta, int k,
              const lb_boundaries* bc, int precision, void* cuda_stream, lb_handle** out) {
    if (!out) return fail(LB_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (lattice != LB_D1Q3 && lattice != LB_D2Q9) return fail(LB_ERR_ARG, "unknown lattice %d", lattice);
    if (equilibrium < LB_EQ_POLY || equilibrium > LB_EQ_ENTROPIC_ENERGY_MLP)
        return fail(LB_ERR_ARG, "unknown equilibrium %d", equilibrium);
    if (equilibrium >= LB_EQ_ENTROPIC_ENERGY && lattice != LB_D2Q9)
        return fail(LB_ERR_ARG, "the energy-constrained equilibria are built for D2Q9");
    if (precision < LB_F64 || precision > LB_F16_DEV) return fail(LB_ERR_ARG, "unknown precision %d", precision);
    if (!(nu > 0.0) || !(nu < 1e30)) return fail(LB_ERR_ARG, "nu must be positive and finite");
    if (delta != delta) return fail(LB_ERR_ARG, "delta is NaN");
    if (k < 0) return fail(LB_ERR_ARG, "k must be >= 0");
    if (lattice == LB_D1Q3 && ny != 1) return fail(LB_ERR_ARG, "D1Q3 needs ny = 1");
    if (nx < 3 || (lattice == LB_D2Q9 && ny < 3)) return fail(LB_ERR_ARG, "grid too small");
    if ((long long)(lattice == LB_D1Q3 ? 3 : 9) * ny * ((nx + 31) / 32 * 32) >= (1ll << 31))
        return fail(LB_ERR_ARG, "grid too large (a population array must hold < 2^31 values)");
    lb_boundaries b;
    if (bc) b = *bc;
    else {
        memset(&b, 0, sizeof(b));
        b.kind_x0 = b.kind_x1 = b.kind_y0 = b.kind_y1 = LB_BB;
        b.rho_in = 1.0;
    }
    int kinds[4] = {b.kind_x0, b.kind_x1, b.kind_y0, b.kind_y1};
    for (int i = 0; i < 4; i++)
        if (!valid_kind(kinds[i])) return fail(LB_ERR_ARG, "unknown boundary kind %d", kinds[i]);
    if (b.kind_x0 == LB_FREESLIP || b.kind_x1 == LB_FREESLIP)
        return fail(LB_ERR_ARG, "free-slip is supported on the y sides only");
    if (b.kind_y0 == LB_INLET_EQ || b.kind_y0 == LB_OUTLET_EQ || b.kind_y1 == LB_INLET_EQ ||
        b.kind_y1 == LB_OUTLET_EQ || b.kind_y0 == LB_OUTLET_COPY || b.kind_y1 == LB_OUTLET_COPY)
        return fail(LB_ERR_ARG, "inlet/outlet are supported on the x sides only");
    if ((b.kind_x0 == LB_PERIODIC) != (b.kind_x1 == LB_PERIODIC) ||
        (b.kind_y0 == LB_PERIODIC) != (b.kind_y1 == LB_PERIODIC))
        return fail(LB_ERR_ARG, "periodic sides come in pairs");
    if (b.kind_x0 == LB_INLET_EQ || b.kind_x1 == LB_INLET_EQ) {
        if (!(b.rho_in > 0.0)) return fail(LB_ERR_ARG, "inlet density must be positive");
        if (!(fabs(b.u_in[0]) < 0.5 && fabs(b.u_in[1]) < 0.5)) return fail(LB_ERR_ARG, "inlet speed too large");
    }
    if (b.obstacle_w < 0 || b.obstacle_h < 0) return fail(LB_ERR_ARG, "negative obstacle size");
    if (b.obstacle_wall != LB_WALL_BOUNCE_BACK && b.obstacle_wall != LB_WALL_DIFFUSE)
        return fail(LB_ERR_ARG, "unknown obstacle wall rule %d", b.obstacle_wall);
    if (b.obstacle_w > 0) {
        if (lattice == LB_D1Q3) return fail(LB_ERR_ARG, "no obstacle on D1Q3");
        if (b.obstacle_h <= 0) return fail(LB_ERR_ARG, "obstacle height must be positive");
        if (b.obstacle_x0 < 1 || b.obstacle_x0 + b.obstacle_w > nx - 3 || b.obstacle_y0 < 1 ||
            b.obstacle_y0 + b.obstacle_h > ny - 1)
            return fail(LB_ERR_ARG, "obstacle must keep one fluid site to the walls and two columns to x = nx-1");
    }

    lb_handle* h = new lb_handle();   // value-initialised: every scalar and pointer is zero
    h->lattice = lattice; h->Q = lattice == LB_D1Q3 ? 3 : 9; h->nx = nx; h->ny = ny;
    h->nxp = (nx + 31) / 32 * 32;
    h->eq = equilibrium; h->prec = precision; h->k = k; h->nu = nu; h->delta = delta;
    h->beta = 1.0 / (1.0 + 6.0 * nu);
    // reference density of the deviation arithmetic: every FP32 / FP16 form
    // (plain FP32 storage keeps f - fl32(W_i)); FP64 works on f itself
    h->rho0 = precision == LB_F64 ? 0.0 : 1.0;
    h->bc = b;
    h->plane = (long long)ny * h->nxp;
    h->probe_x = h->probe_y = -1;
    h->tile_shape = default_tile_shape(lattice, equilibrium, precision, (long long)nx * ny);
    h->ring_cap = kDefaultLog;
    h->replay_t0 = -1;
    if (precision == LB_F64) h->L = launchers_f64(lattice, equilibrium);
    else if (precision == LB_F16_DEV) h->L = launchers_f16(lattice, equilibrium);
    else if (precision == LB_F32) h->L = launchers_f32p(lattice, equilibrium);
    else h->L = launchers_f32(lattice, equilibrium);

#define CKH(call)                                                                   \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess) {                                                    \
            int rc_ = fail(e_ == cudaErrorMemoryAllocation ? LB_ERR_OOM : LB_ERR_CUDA, \
                           "%s: %s", #call, cudaGetErrorString(e_));                \
            lb_destroy(h);                                                          \
            return rc_;                                                             \
        }                                                                           \
    } while (0)

    if (cuda_stream) {
        h->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        CKH(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
        h->own_stream = true;
    }
    const size_t pop_bytes = (size_t)h->Q * h->plane * storage_bytes(precision);
    for (int i = 0; i < 2; i++) {
        CKH(cudaMalloc(&h->buf[i], pop_bytes));
        CKH(cudaMemsetAsync(h->buf[i], 0, pop_bytes, h->stream));
    }
    const long long nsites = (long long)nx * ny;
    // candidate list: one slot per site (warps append every site with
    // dS > delta; the list can never overflow)
    h->cand_per_block = std::min(k, 1024);
    h->cand_cap = std::max(1ll, nsites);
    h->sel_cap = std::max(1ll, std::min((long long)k, nsites));
    CKH(cudaMalloc(&h->cand_key, h->cand_cap * sizeof(unsigned long long)));
    CKH(cudaMalloc(&h->cand_idx, h->cand_cap * sizeof(unsigned)));
    CKH(cudaMalloc(&h->cand_count, sizeof(unsigned)));
    CKH(cudaMalloc(&h->sel_idx, std::max(h->sel_cap, (long long)1) * sizeof(int)));
    CKH(cudaMalloc(&h->sel_count, sizeof(int)));
    CKH(cudaMalloc(&h->count_ring, h->ring_cap * sizeof(int)));
    CKH(cudaMalloc(&h->probe_ring, h->ring_cap * sizeof(double)));
    CKH(cudaMalloc(&h->d_step, sizeof(long long)));
    CKH(cudaMalloc(&h->d_err, sizeof(unsigned)));
    CKH(cudaMalloc(&h->newton_stats, 4 * sizeof(unsigned long long)));
    if (h->eq == LB_EQ_ENTROPIC_ENERGY_MLP) {
        CKH(cudaMalloc(&h->mlp, lbm::kMlpParams * sizeof(float)));
        CKH(cudaMemsetAsync(h->mlp, 0, lbm::kMlpParams * sizeof(float), h->stream));
    }
    CKH(cudaMalloc(&h->ticket, sizeof(unsigned)));
    CKH(cudaMemsetAsync(h->ticket, 0, sizeof(unsigned), h->stream));
    CKH(cudaMalloc(&h->pend_idx, std::max(1ll, nsites) * sizeof(unsigned)));
    CKH(cudaMalloc(&h->pend_count, sizeof(unsigned)));
    CKH(cudaMemsetAsync(h->pend_count, 0, sizeof(unsigned), h->stream));
    CKH(cudaMalloc(&h->tile_counter, sizeof(unsigned)));
    CKH(cudaMemsetAsync(h->tile_counter, 0, sizeof(unsigned), h->stream));
    CKH(cudaMallocHost(&h->h_err, sizeof(unsigned)));
    *h->h_err = 0;
    CKH(cudaEventCreateWithFlags(&h->err_ev, cudaEventDisableTiming));
    CKH(cudaMemsetAsync(h->cand_count, 0, sizeof(unsigned), h->stream));
    CKH(cudaMemsetAsync(h->sel_count, 0, sizeof(int), h->stream));
    CKH(cudaMemsetAsync(h->count_ring, 0, h->ring_cap * sizeof(int), h->stream));
    CKH(cudaMemsetAsync(h->probe_ring, 0, h->ring_cap * sizeof(double), h->stream));
    CKH(cudaMemsetAsync(h->d_step, 0, sizeof(long long), h->stream));
    CKH(cudaMemsetAsync(h->d_err, 0, sizeof(unsigned), h->stream));
    CKH(cudaMemsetAsync(h->newton_stats, 0, 4 * sizeof(unsigned long long), h->stream));
    CKH(h->L.set_smem(kSelectStageCap));
    if (size_grid(h) != LB_OK || make_tensor_maps(h) != LB_OK) {
        const std::string msg = g_last_error;
        lb_destroy(h);
        return fail(LB_ERR_CUDA, "%s", msg.c_str());
    }
    CKH(cudaStreamSynchronize(h->stream));
    h->cur = 0;
    h->prestream = true;
#undef CKH
    *out = h;
    return LB_OK;
}

// The handle's staging buffer, at least `bytes` long (the previous calls that
// used it have synchronised with the stream).
static int copy_streams(lb_handle* h) {
    if (!h->copy_stream) {
        CK(cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
        CK(cudaStreamCreateWithFlags(&h->d2h_stream, cudaStreamNonBlocking));
        for (cudaEvent_t& e : h->xfer_ev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        for (cudaEvent_t& e : h->out_ev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&h->d2h_done, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&h->imp_done, cudaEventDisableTiming));
    }
    return LB_OK;
}

// Download staging (exports), at least `bytes` long; a previous download
// may still read it (the caller orders its kernels after d2h_done).
static int staging_out(lb_handle* h, size_t bytes, double** out) {
    if (int rc = copy_streams(h)) return rc;
    if (h->stage_out_bytes < bytes) {
        CK(cudaStreamSynchronize(h->d2h_stream));
        if (h->stage_out) cudaFree(h->stage_out);
        h->stage_out = nullptr;
        h->stage_out_bytes = 0;
        const size_t full = (size_t)std::max(h->Q, 4) * h->nx * h->ny * sizeof(double);
        CK(cudaMalloc(&h->stage_out, std::max(bytes, full)));
        h->stage_out_bytes = std::max(bytes, full);
    }
    *out = h->stage_out;
    return LB_OK;
}

static int staging(lb_handle* h, size_t bytes, double** out) {
    if (int rc = copy_streams(h)) return rc;
    if (h->stage_bytes < bytes) {
        if (h->stage) cudaFree(h->stage);
        h->stage = nullptr;
        h->stage_bytes = 0;
        // room for every use at once: Q population planes or 4 field planes
        const size_t full = (size_t)std::max(h->Q, 4) * h->nx * h->ny * sizeof(double);
        CK(cudaMalloc(&h->stage, std::max(bytes, full)));
        h->stage_bytes = std::max(bytes, full);
    }
    *out = h->stage;
    return LB_OK;
}

int lb_init_equilibrium(lb_handle* h, const double* rho, const double* ux, const double* uy,
                        const double* e2) {
    if (!h || !rho || !ux) return fail(LB_ERR_ARG, "NULL argument");
    const long long N = (long long)h->nx * h->ny;
    for (long long i = 0; i < N; i++)
        if (!(rho[i] > 0.0) || !(fabs(ux[i]) < 0.5) || (uy && !(fabs(uy[i]) < 0.5)))
            return fail(LB_ERR_ARG, "init field out of range at site %lld", i);
    double* d = nullptr;
    const size_t nb = N * sizeof(double);
    if (int rc = staging(h, 4 * nb, &d)) return rc;
    CK(cudaMemcpyAsync(d, rho, nb, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(d + N, ux, nb, cudaMemcpyHostToDevice, h->stream));
    if (uy) CK(cudaMemcpyAsync(d + 2 * N, uy, nb, cudaMemcpyHostToDevice, h->stream));
    if (e2) CK(cudaMemcpyAsync(d + 3 * N, e2, nb, cudaMemcpyHostToDevice, h->stream));
    Params P = make_params(h, 1 - h->cur, true);   // dst = buf[cur]
    CK(h->L.init_eq(P, d, d + N, uy ? d + 2 * N : nullptr, e2 ? d + 3 * N : nullptr, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->prestream = true;
    return LB_OK;
}

// The state is uploaded plane by plane on the copy stream; the run's stream
// converts plane i (k_import) while plane i + 1 is in flight.  The copies
// wait for the previous upload's conversions (they read the same staging;
// the first upload waits for all the work queued so far), not for the
// steps and exports queued after them, so that in a serving loop the next
// upload runs while the run steps and downloads.
static int set_state(lb_handle* h, const double* f, bool async) {
    if (!h || !f) return fail(LB_ERR_ARG, "NULL argument");
    const long long N = (long long)h->nx * h->ny;
    const size_t nb = (size_t)h->Q * N * sizeof(double);
    double* d = nullptr;
    if (h->stage_bytes < nb && h->copy_stream) CK(cudaStreamSynchronize(h->stream));
    if (int rc = staging(h, nb, &d)) return rc;
    Params P = make_params(h, 1 - h->cur, true);
    if (h->imp_pending) {
        CK(cudaStreamWaitEvent(h->copy_stream, h->imp_done, 0));
    } else {
        CK(cudaEventRecord(h->xfer_ev[kXferEvents - 1], h->stream));
        CK(cudaStreamWaitEvent(h->copy_stream, h->xfer_ev[kXferEvents - 1], 0));
    }
    for (int i = 0; i < h->Q; i++) {
        CK(cudaMemcpyAsync(d + i * N, f + i * N, (size_t)N * sizeof(double), cudaMemcpyHostToDevice,
                           h->copy_stream));
        CK(cudaEventRecord(h->xfer_ev[i], h->copy_stream));
        CK(cudaStreamWaitEvent(h->stream, h->xfer_ev[i], 0));
        CK(h->L.import_state(P, d, i, i + 1, h->stream));
    }
    CK(cudaEventRecord(h->imp_done, h->stream));
    h->imp_pending = true;
    h->prestream = true;
    if (!async) CK(cudaStreamSynchronize(h->stream));
    return LB_OK;
}

int lb_set_state(lb_handle* h, const double* f) { return set_state(h, f, false); }
int lb_set_state_async(lb_handle* h, const double* f) { return set_state(h, f, true); }

// Host exports go in row chunks: the run's stream converts chunk c
// (k_export over its sites) while the download stream moves chunk c - 1 to
// the host; each field (mode 0: each population plane) is copied per chunk.
// The kernels first wait for the previous download out of the same staging.
static int export_fields(lb_handle* h, int mode, double* o0, double* o1, double* o2, double* o3,
                         int on_device, bool async = false) {
    const long long N = (long long)h->nx * h->ny;
    if (on_device) {
        Params P = make_params(h, h->cur, h->prestream);
        CK(h->L.export_state(P, mode, o0, o1, o2, o3, 0, N, h->stream));
        return LB_OK;
    }
    double* d = nullptr;
    const int planes = mode == 0 ? h->Q : 1;   // planes of N values per output field
    if (int rc = staging_out(h, (size_t)N * sizeof(double) * (mode == 0 ? h->Q : (mode == 1 ? 4 : 1)), &d))
        return rc;
    if (h->d2h_pending) CK(cudaStreamWaitEvent(h->stream, h->d2h_done, 0));
    Params P = make_params(h, h->cur, h->prestream);
    double* outs[4] = {o0, mode == 1 ? o1 : nullptr, mode == 1 ? o2 : nullptr, mode == 1 ? o3 : nullptr};
    double* dd[4] = {d, outs[1] ? d + N : nullptr, outs[2] ? d + 2 * N : nullptr,
                     outs[3] ? d + 3 * N : nullptr};
    const int chunks = std::min(kExportChunks, h->ny);
    const int rows = (h->ny + chunks - 1) / chunks;
    for (int c = 0; c * rows < h->ny; c++) {
        const long long s0 = (long long)c * rows * h->nx;
        const long long s1 = std::min<long long>((long long)(c + 1) * rows, h->ny) * h->nx;
        CK(h->L.export_state(P, mode, dd[0], dd[1], dd[2], dd[3], s0, s1, h->stream));
        CK(cudaEventRecord(h->out_ev[c], h->stream));
        CK(cudaStreamWaitEvent(h->d2h_stream, h->out_ev[c], 0));
        for (int j = 0; j < 4; j++) {
            if (!outs[j] || !dd[j]) continue;
            for (int q = 0; q < planes; q++)
                CK(cudaMemcpyAsync(outs[j] + q * N + s0, dd[j] + q * N + s0, (size_t)(s1 - s0) * sizeof(double),
                                   cudaMemcpyDeviceToHost, h->d2h_stream));
        }
    }
    CK(cudaEventRecord(h->d2h_done, h->d2h_stream));
    h->d2h_pending = true;
    if (!async) {
        CK(cudaStreamSynchronize(h->d2h_stream));
        CK(cudaStreamSynchronize(h->stream));
    }
    return LB_OK;
}

int lb_get_state(lb_handle* h, double* f) {
    if (!h || !f) return fail(LB_ERR_ARG, "NULL argument");
    return export_fields(h, 0, f, nullptr, nullptr, nullptr, 0);
}

int lb_moments(lb_handle* h, double* rho, double* ux, double* uy, double* e2, int on_device) {
    if (!h || !rho || !ux) return fail(LB_ERR_ARG, "NULL argument");
    return export_fields(h, 1, rho, ux, uy, e2, on_device);
}

int lb_moments_async(lb_handle* h, double* rho, double* ux, double* uy, double* e2) {
    if (!h || !rho || !ux) return fail(LB_ERR_ARG, "NULL argument");
    return export_fields(h, 1, rho, ux, uy, e2, 0, true);
}

int lb_delta_s(lb_handle* h, double* ds, int on_device) {
    if (!h || !ds) return fail(LB_ERR_ARG, "NULL argument");
    return export_fields(h, 2, ds, nullptr, nullptr, nullptr, on_device);
}

int lb_step(lb_handle* h, int n) {
    if (!h) return fail(LB_ERR_ARG, "NULL handle");
    if (n < 0) return fail(LB_ERR_ARG, "n must be >= 0");
    if (h->slab) return fail(LB_ERR_STATE, "a slab steps with lb_slab_collide and lb_slab_apply");
    int rc = check_sticky(h, false);
    if (rc != LB_OK) return rc;
    if (h->eq == LB_EQ_ENTROPIC_ENERGY_MLP && !h->mlp_set)
        return fail(LB_ERR_STATE, "the learned equilibrium needs its network (lb_set_mlp) first");
    int done = 0;
    const bool replaying = h->replay_n > 0 && h->h_step < h->replay_t0 + h->replay_n;
    while (done < n) {
        const bool direct = h->prestream || h->timing || replaying || (n - done) < kGraphSteps;
        if (direct) {
            rc = queue_step(h, h->cur, h->prestream, h->timing);
            if (rc != LB_OK) return rc;
            h->prestream = false;
            h->cur = 1 - h->cur;
            h->h_step++;
            done++;
        } else {
            if (!h->graph_exec[h->cur]) {
                rc = build_graph(h, h->cur);
                if (rc != LB_OK) return rc;
            }
            CK(cudaGraphLaunch(h->graph_exec[h->cur], h->stream));
            h->h_step += kGraphSteps;
            done += kGraphSteps;   // kGraphSteps is even: cur is unchanged
        }
    }
    return queue_err_readback(h);
}

int lb_sync(lb_handle* h) {
    if (!h) return fail(LB_ERR_ARG, "NULL handle");
    CK(cudaStreamSynchronize(h->stream));
    if (h->copy_stream) {
        CK(cudaStreamSynchronize(h->copy_stream));
        CK(cudaStreamSynchronize(h->d2h_stream));
    }
    return check_sticky(h, true);
}

int lb_selected(lb_handle* h, int* idx, int cap, int* count) {
    if (!h || !count || (cap > 0 && !idx)) return fail(LB_ERR_ARG, "NULL argument");
    int c = 0;
    CK(cudaMemcpyAsync(&c, h->sel_count, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    *count = c;
    const int m = std::min(c, cap);
    if (m > 0) {
        CK(cudaMemcpyAsync(idx, h->sel_idx, m * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
    }
    return LB_OK;
}

static int read_ring(lb_handle* h, void* dring, size_t esz, void* out, int n) {
    if (n < 0 || n > h->ring_cap) return fail(LB_ERR_ARG, "n must be in [0, log capacity]");
    if ((long long)n > h->h_step) return fail(LB_ERR_ARG, "only %lld steps were run", h->h_step);
    if (n == 0) return LB_OK;
    std::vector<char> all((size_t)h->ring_cap * esz);
    CK(cudaMemcpyAsync(all.data(), dring, all.size(), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    for (int j = 0; j < n; j++) {
        const long long t = h->h_step - n + j;
        memcpy(static_cast<char*>(out) + j * esz, all.data() + (t % h->ring_cap) * esz, esz);
    }
    return LB_OK;
}

int lb_counts(lb_handle* h, int* per_step, int n) {
    if (!h || (n > 0 && !per_step)) return fail(LB_ERR_ARG, "NULL argument");
    return read_ring(h, h->count_ring, sizeof(int), per_step, n);
}

int lb_set_probe(lb_handle* h, int x, int y) {
    if (!h) return fail(LB_ERR_ARG, "NULL handle");
    if (x < 0 || x >= h->nx || y < 0 || y >= h->ny) return fail(LB_ERR_ARG, "probe outside the grid");
    h->probe_x = x;
    h->probe_y = y;
    drop_graphs(h);
    return LB_OK;
}

int lb_probe(lb_handle* h, double* ux_series, int n) {
    if (!h || (n > 0 && !ux_series)) return fail(LB_ERR_ARG, "NULL argument");
    if (h->probe_x < 0) return fail(LB_ERR_STATE, "no probe set");
    return read_ring(h, h->probe_ring, sizeof(double), ux_series, n);
}

int lb_set_log_capacity(lb_handle* h, int steps) {
    if (!h) return fail(LB_ERR_ARG, "NULL handle");
    if (steps < 1 || steps > (1 << 26)) return fail(LB_ERR_ARG, "capacity out of range");
    CK(cudaStreamSynchronize(h->stream));
    int* cr = nullptr;
    double* pr = nullptr;
    CK(cudaMalloc(&cr, steps * sizeof(int)));
    if (cudaMalloc(&pr, steps * sizeof(double)) != cudaSuccess) {
        cudaFree(cr);
        return fail(LB_ERR_OOM, "log allocation failed");
    }
    cudaMemset(cr, 0, steps * sizeof(int));
    cudaMemset(pr, 0, steps * sizeof(double));
    cudaFree(h->count_ring);
    cudaFree(h->probe_ring);
    h->count_ring = cr;
    h->probe_ring = pr;
    h->ring_cap = steps;
    drop_graphs(h);
    return LB_OK;
}

int lb_replay_selection(lb_handle* h, const int* counts, const int* idx, int nsteps) {
    if (!h || nsteps < 0 || (nsteps > 0 && !counts)) return fail(LB_ERR_ARG, "bad argument");
    std::vector<long long> off(std::max(nsteps, 1));
    long long tot = 0;
    for (int t = 0; t < nsteps; t++) {
        if (counts[t] < 0 || counts[t] > h->sel_cap)
            return fail(LB_ERR_ARG, "replay count %d at step %d outside [0, %lld]", counts[t], t, h->sel_cap);
        off[t] = tot;
        tot += counts[t];
    }
    if (tot > 0 && !idx) return fail(LB_ERR_ARG, "idx is NULL");
    CK(cudaStreamSynchronize(h->stream));
    cudaFree(h->replay_cnt); cudaFree(h->replay_off); cudaFree(h->replay_idx);
    h->replay_cnt = nullptr; h->replay_off = nullptr; h->replay_idx = nullptr;
    CK(cudaMalloc(&h->replay_cnt, std::max(nsteps, 1) * sizeof(int)));
    CK(cudaMalloc(&h->replay_off, std::max(nsteps, 1) * sizeof(long long)));
    CK(cudaMalloc(&h->replay_idx, std::max(tot, 1ll) * sizeof(int)));
    if (nsteps) {
        CK(cudaMemcpy(h->replay_cnt, counts, nsteps * sizeof(int), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(h->replay_off, off.data(), nsteps * sizeof(long long), cudaMemcpyHostToDevice));
    }
    if (tot) CK(cudaMemcpy(h->replay_idx, idx, tot * sizeof(int), cudaMemcpyHostToDevice));
    h->replay_t0 = h->h_step;
    h->replay_n = nsteps;
    drop_graphs(h);
    return LB_OK;
}

int lb_select_only(const double* ds, int n, double delta, int k, int* idx_out, int* count) {
    if (!count || n < 0 || k < 0 || (n > 0 && !ds)) return fail(LB_ERR_ARG, "bad argument");
    if (delta != delta) return fail(LB_ERR_ARG, "delta is NaN");
    *count = 0;
    if (n == 0 || k == 0) return LB_OK;
    if (!idx_out) return fail(LB_ERR_ARG, "idx_out is NULL");
    cudaStream_t st;
    CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    const int per_block = std::min(k, 1024);
    const long long cap = n;
    const long long scap = std::min((long long)k, (long long)n);
    double* d_ds = nullptr;
    unsigned long long* key = nullptr;
    unsigned* cid = nullptr;
    unsigned* ccount = nullptr;
    int* sel = nullptr;
    int* scount = nullptr;
    long long* step = nullptr;
    unsigned* err = nullptr;
    cudaError_t e = cudaSuccess;
    auto ok = [&](cudaError_t x) { if (e == cudaSuccess) e = x; return e == cudaSuccess; };
    ok(cudaMalloc(&d_ds, n * sizeof(double)));
    ok(cudaMalloc(&key, cap * sizeof(unsigned long long)));
    ok(cudaMalloc(&cid, cap * sizeof(unsigned)));
    ok(cudaMalloc(&ccount, sizeof(unsigned)));
    ok(cudaMalloc(&sel, scap * sizeof(int)));
    ok(cudaMalloc(&scount, sizeof(int)));
    ok(cudaMalloc(&step, sizeof(long long)));
    ok(cudaMalloc(&err, sizeof(unsigned)));
    if (e == cudaSuccess) {
        ok(cudaMemcpyAsync(d_ds, ds, n * sizeof(double), cudaMemcpyHostToDevice, st));
        ok(cudaMemsetAsync(ccount, 0, sizeof(unsigned), st));
        ok(cudaMemsetAsync(step, 0, sizeof(long long), st));
        ok(cudaMemsetAsync(err, 0, sizeof(unsigned), st));
        Params P;
        memset(&P, 0, sizeof(P));
        P.nx = n; P.ny = 1; P.nxp = n; P.plane = n; P.delta = delta; P.k = k;
        P.cand_key = key; P.cand_idx = cid; P.cand_count = ccount; P.cand_per_block = per_block;
        P.sel_idx = sel; P.sel_count = scount; P.step = step; P.err = err; P.ring_cap = 1;
        Launchers L = launchers_f64(LB_D1Q3, LB_EQ_POLY);
        ok(L.set_smem(kSelectStageCap));
        ok(launch_emit_from_ds(P, d_ds, n, st));
        ok(L.select(P, kSelectStageCap, 1, st));
        int c = 0;
        ok(cudaMemcpyAsync(&c, scount, sizeof(int), cudaMemcpyDeviceToHost, st));
        ok(cudaStreamSynchronize(st));
        if (e == cudaSuccess) {
            *count = c;
            if (c > 0) ok(cudaMemcpy(idx_out, sel, std::min<long long>(c, scap) * sizeof(int),
                                     cudaMemcpyDeviceToHost));
        }
    }
    void* ptrs[] = {d_ds, key, cid, ccount, sel, scount, step, err};
    for (void* p : ptrs) if (p) cudaFree(p);
    cudaStreamDestroy(st);
    if (e != cudaSuccess)
        return fail(e == cudaErrorMemoryAllocation ? LB_ERR_OOM : LB_ERR_CUDA, "lb_select_only: %s",
                    cudaGetErrorString(e));
    return LB_OK;
}

int lb_set_collision(lb_handle* h, int collision) {
    if (!h) return fail(LB_ERR_ARG, "NULL handle");
    if (collision != LB_COLLISION_LBGK && collision != LB_COLLISION_ELBM)
        return fail(LB_ERR_ARG, "unknown collision %d", collision);
    if (collision == LB_COLLISION_ELBM && h->eq != LB_EQ_ENTROPIC)
        return fail(LB_ERR_ARG, "ELBM uses the entropic quasiequilibria (LB_EQ_ENTROPIC)");
    CK(cudaStreamSynchronize(h->stream));
    h->elbm = collision == LB_COLLISION_ELBM;
    drop_graphs(h);
    return LB_OK;
}

int lb_mlp_param_count(void) { return lbm::kMlpParams; }

int lb_set_mlp(lb_handle* h, const float* params, int n) {
    if (!h || !params) return fail(LB_ERR_ARG, "NULL argument");
    if (n != lb_mlp_param_count()) return fail(LB_ERR_ARG, "expected %d parameters", lb_mlp_param_count());
    if (h->eq != LB_EQ_ENTROPIC_ENERGY_MLP)
        return fail(LB_ERR_STATE, "the run does not use the learned equilibrium");
    for (int i = 0; i < n; i++)
        if (!std::isfinite(params[i])) return fail(LB_ERR_ARG, "parameter %d is not finite", i);
    CK(cudaMemcpyAsync(h->mlp, params, (size_t)n * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->mlp_set = true;
    return LB_OK;
}

int lb_newton_stats(lb_handle* h, long long* it32, long long* it64, long long* sites,
                    long long* fails, int reset) {
    if (!h) return fail(LB_ERR_ARG, "NULL handle");
    unsigned long long s[4] = {0, 0, 0, 0};
    CK(cudaMemcpyAsync(s, h->newton_stats, sizeof(s), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (it32) *it32 = (long long)s[0];
    if (it64) *it64 = (long long)s[1];
    if (sites) *sites = (long long)s[2];
    if (fails) *fails = (long long)s[3];
    if (reset) CK(cudaMemsetAsync(h->newton_stats, 0, sizeof(s), h->stream));
    return LB_OK;
}

int lb_set_timing(lb_handle* h, int enable) {
    if (!h) return fail(LB_ERR_ARG, "NULL handle");
    h->timing = enable != 0;
    return LB_OK;
}

int lb_kernel_times(lb_handle* h, double* collide_ms, long long* collide_launches, double* select_ms,
                    long long* select_launches, int reset) {
    if (!h) return fail(LB_ERR_ARG, "NULL handle");
    CK(cudaStreamSynchronize(h->stream));
    for (int kind = 0; kind < 2; kind++) {
        for (auto& pr : h->ev_pairs[kind]) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, h->ev_pool[pr.first], h->ev_pool[pr.second]));
            h->acc_ms[kind] += ms;
            h->acc_n[kind] += 1;
        }
        h->ev_pairs[kind].clear();
    }
    h->ev_next = 0;
    if (collide_ms) *collide_ms = h->acc_ms[0];
    if (collide_launches) *collide_launches = h->acc_n[0];
    if (select_ms) *select_ms = h->acc_ms[1];
    if (select_launches) *select_launches = h->acc_n[1];
    if (reset) {
        h->acc_ms[0] = h->acc_ms[1] = 0.0;
        h->acc_n[0] = h->acc_n[1] = 0;
    }
    return LB_OK;
}

int lb_set_tile_shape(lb_handle* h, int shape) {
    if (!h) return fail(LB_ERR_ARG, "NULL handle");
    if (shape < 0 || shape >= kTileShapes) return fail(LB_ERR_ARG, "tile shape must be in [0, %d)", kTileShapes);
    if (h->lattice != LB_D2Q9) return fail(LB_ERR_ARG, "tile shapes apply to D2Q9 runs");
    if (shape == 6 && h->eq >= LB_EQ_ENTROPIC_ENERGY)
        return fail(LB_ERR_ARG, "the energy forms take tile shapes 0-5");
    CK(cudaStreamSynchronize(h->stream));
    h->tile_shape = shape;
    drop_graphs(h);
    const int rc = size_grid(h);
    if (rc != LB_OK) return rc;
    return make_tensor_maps(h);
}

// ---------------------------------------------------------------------------
// Slabs of a run sharded in x (the selection of Sec. 3.2 is global: the k
// sites with the largest dS of the whole grid).
// ---------------------------------------------------------------------------

int lb_set_slab(lb_handle* h, int ghost_left, int ghost_right, int global_x0, int global_nx) {
    if (!h) return fail(LB_ERR_ARG, "NULL handle");
    if (h->lattice != LB_D2Q9) return fail(LB_ERR_ARG, "slabs are built for D2Q9");
    if (h->slab) return fail(LB_ERR_STATE, "the handle is already a slab");
    if ((ghost_left != 0 && ghost_left != 1) || (ghost_right != 0 && ghost_right != 1))
        return fail(LB_ERR_ARG, "a slab has at most one ghost column on each side");
    const int own = h->nx - ghost_left - ghost_right;
    if (own < 3) return fail(LB_ERR_ARG, "a slab owns at least three columns");
    if (global_x0 < 0 || global_x0 + own > global_nx) return fail(LB_ERR_ARG, "slab outside the global grid");
    if ((ghost_left == 0) != (global_x0 == 0) || (ghost_right == 0) != (global_x0 + own == global_nx))
        return fail(LB_ERR_ARG, "ghost columns on exactly the sides that face another slab");
    if ((long long)h->ny * global_nx >= (1ll << 31)) return fail(LB_ERR_ARG, "global grid too large");
    if (h->replay_n > 0) return fail(LB_ERR_STATE, "a slab cannot replay selections");
    CK(cudaStreamSynchronize(h->stream));
    const long long cap = std::max(1ll, h->sel_cap);
    CK(cudaMalloc(&h->sel_key, cap * sizeof(unsigned long long)));
    CK(cudaMalloc(&h->slab_sel, cap * sizeof(int)));
    CK(cudaMalloc(&h->slab_cnt, sizeof(int)));
    CK(cudaMalloc(&h->slab_off, sizeof(long long)));
    CK(cudaMemset(h->slab_off, 0, sizeof(long long)));
    h->slab = 1;
    h->ghost_l = ghost_left;
    h->ghost_r = ghost_right;
    h->gx0 = global_x0;
    h->gnx = global_nx;
    drop_graphs(h);
    return LB_OK;
}

int lb_slab_collide(lb_handle* h) {
    if (!h) return fail(LB_ERR_ARG, "NULL handle");
    if (!h->slab) return fail(LB_ERR_STATE, "not a slab (lb_set_slab)");
    if (h->slab_collided) return fail(LB_ERR_STATE, "the previous step's selection was not applied");
    int rc = check_sticky(h, false);
    if (rc != LB_OK) return rc;
    if (h->eq == LB_EQ_ENTROPIC_ENERGY_MLP && !h->mlp_set)
        return fail(LB_ERR_STATE, "the learned equilibrium needs its network (lb_set_mlp) first");
    rc = queue_step(h, h->cur, h->prestream, h->timing);
    if (rc != LB_OK) return rc;
    h->slab_collided = true;
    return LB_OK;
}

int lb_slab_candidates(lb_handle* h, unsigned long long* keys, long long* global_idx, int cap, int* count) {
    if (!h || !count || (cap > 0 && (!keys || !global_idx))) return fail(LB_ERR_ARG, "NULL argument");
    if (!h->slab_collided) return fail(LB_ERR_STATE, "no collided step (lb_slab_collide)");
    int c = 0;
    CK(cudaMemcpyAsync(&c, h->sel_count, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    *count = c;
    const int m = std::min(c, cap);
    if (m > 0) {
        std::vector<int> idx(m);
        CK(cudaMemcpyAsync(idx.data(), h->sel_idx, m * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaMemcpyAsync(keys, h->sel_key, m * sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        for (int j = 0; j < m; j++) {
            const int x = idx[j] % h->nx, y = idx[j] / h->nx;
            global_idx[j] = (long long)y * h->gnx + (h->gx0 + x - h->ghost_l);
        }
    }
    return check_sticky(h, true);
}

int lb_slab_apply(lb_handle* h, const long long* global_idx, int m) {
    if (!h || m < 0 || (m > 0 && !global_idx)) return fail(LB_ERR_ARG, "bad argument");
    if (!h->slab_collided) return fail(LB_ERR_STATE, "no collided step (lb_slab_collide)");
    if (m > h->k) return fail(LB_ERR_ARG, "more selected sites (%d) than k (%d)", m, h->k);
    std::vector<int> own;
    const int own_w = h->nx - h->ghost_l - h->ghost_r;
    for (int j = 0; j < m; j++) {
        const long long g = global_idx[j];
        if (g < 0 || g >= (long long)h->ny * h->gnx) return fail(LB_ERR_ARG, "site %lld outside the grid", g);
        const int gx = (int)(g % h->gnx), y = (int)(g / h->gnx);
        if (gx >= h->gx0 && gx < h->gx0 + own_w) own.push_back(y * h->nx + (gx - h->gx0 + h->ghost_l));
    }
    const int c = (int)own.size();
    CK(cudaMemcpyAsync(h->slab_cnt, &c, sizeof(int), cudaMemcpyHostToDevice, h->stream));
    if (c > 0) CK(cudaMemcpyAsync(h->slab_sel, own.data(), c * sizeof(int), cudaMemcpyHostToDevice, h->stream));
    // the Ehrenfests' step at the slab's selected sites, as one replayed step
    Params P = make_params(h, h->cur, h->prestream);
    P.replay_cnt = h->slab_cnt;
    P.replay_off = h->slab_off;
    P.replay_idx = h->slab_sel;
    P.replay_t0 = h->h_step;
    P.replay_n = 1;
    CK(h->L.select(P, kSelectStageCap, 0, h->stream));
    CK(cudaStreamSynchronize(h->stream));   // the host copies of the lists are local
    h->slab_collided = false;
    h->prestream = false;
    h->cur = 1 - h->cur;
    h->h_step++;
    return queue_err_readback(h);
}

int lb_slab_ghost(lb_handle* h, int side, void* buf, int direction) {
    if (!h || !buf) return fail(LB_ERR_ARG, "NULL argument");
    if (!h->slab) return fail(LB_ERR_STATE, "not a slab (lb_set_slab)");
    if (h->slab_collided) return fail(LB_ERR_STATE, "the step's selection was not applied");
    if (side != 0 && side != 1) return fail(LB_ERR_ARG, "side is 0 (left) or 1 (right)");
    if (direction != 0 && direction != 1) return fail(LB_ERR_ARG, "direction is 0 (pack) or 1 (unpack)");
    if ((side == 0 && !h->ghost_l) || (side == 1 && !h->ghost_r)) return fail(LB_ERR_ARG, "no neighbour on that side");
    // pack: the outgoing populations of the first (left) or last (right)
    // owned column; unpack: the incoming ones into the ghost column
    int col, right;
    if (direction == 0) {
        col = side == 0 ? h->ghost_l : h->nx - 1 - h->ghost_r;
        right = side == 1;
    } else {
        col = side == 0 ? 0 : h->nx - 1;
        right = side == 0;
    }
    Params P = make_params(h, h->cur, false);
    CK(h->L.ghost(P, h->buf[h->cur], col, right, buf, direction, h->stream));
    return LB_OK;
}

int lb_info(lb_handle* h, long long* out, double* beta_out) {
    if (!h || !out) return fail(LB_ERR_ARG, "NULL argument");
    out[0] = h->Q;
    out[1] = h->nxp;
    out[2] = (long long)storage_bytes(h->prec);
    out[3] = 2ll * h->Q * (long long)storage_bytes(h->prec);
    out[4] = 1;
    out[5] = h->grid_blocks;
    out[6] = h->blocks_per_sm;
    out[7] = h->tile_shape;
    if (beta_out) *beta_out = h->beta;
    return LB_OK;
}

}  // extern "C"
