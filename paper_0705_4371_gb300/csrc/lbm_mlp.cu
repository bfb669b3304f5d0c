// lbm_mlp.cu -- learned form: training data for the network that
// warm-starts the energy Newton solve, and its training on the GPU.
//
//   lb_energy_dataset  moments -> energy-constrained multipliers mu by Newton
//                      (FP32 iterations, FP64 finish to 1e-12; Sec. 3.3),
//                      with the network's features and corrections mu - mu0
//   lb_mlp_normalise   input standardisation and output scales from a data set
//   lb_mlp_forward     the network on a batch (the kernels' own evaluation)
//   lb_mlp_grad        mean squared error and its gradient (deterministic)
//   lb_mlp_adam        one Adam update
//   lb_mlp_train       epochs of mini-batch Adam
//
// The forward pass of training is the inference routine (BF16 tensor cores,
// FP32 accumulation), so the network is trained on exactly the arithmetic
// that later evaluates it.  The backward pass runs in FP32 on the BF16
// weights and activations the forward pass used (gradients pass straight
// through the roundings), one sample per thread; per-block partial sums are
// reduced in a fixed order, so every result is reproducible bit for bit.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_device.cuh"
#include "lbm_energy.cuh"
#include "lbm_internal.h"
#include "lbm_mlp.cuh"

using namespace lbm;

namespace {

constexpr int kTrainRows = 64;                   // samples per block (two warps)
constexpr int kLd = kMlpHid + 1;                 // padded activation row
constexpr int kPartial = kMlpTrainable + 1;      // per-block gradient sums and the loss
constexpr int kReduceThreads = 256;
// Adam's constants; 1 - b is stored as its own correctly rounded FP32 value
// (1.0f - 0.999f differs from 0.001 by 1.3e-5 relative)
constexpr double kAdamB1d = 0.9, kAdamB2d = 0.999;
constexpr float kAdamB1 = 0.9f, kAdamB2 = 0.999f, kAdam1mB1 = 0.1f, kAdam1mB2 = 0.001f, kAdamEps = 1e-8f;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    set_last_error(buf);
    return code;
}

#define CK(x)                                                                                     \
    do {                                                                                          \
        cudaError_t e_ = (x);                                                                     \
        if (e_ != cudaSuccess)                                                                    \
            return fail(e_ == cudaErrorMemoryAllocation ? LB_ERR_OOM : LB_ERR_CUDA, "%s: %s", #x, \
                        cudaGetErrorString(e_));                                                  \
    } while (0)

__device__ __forceinline__ float bf16_round(float v) { return bf16_lo(bf16_pack(v, 0.0f)); }

// ---------------------------------------------------------------------------
// Training data: for sample i, the moments (rho, rho u, 2E) with
// 2E = escale_i x (2E of the isothermal entropic equilibrium, Sec. 4.2),
// the multipliers mu of ln(f*_j / W_j) = mu . (1, v_x, v_y, |v|^2) by the
// energy Newton solve from the polynomial start point, the features
// (rho, u_x, u_y, 2E/rho - |u|^2) and the corrections mu - mu0.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_energy_dataset(const double* __restrict__ rho,
                                                         const double* __restrict__ ux,
                                                         const double* __restrict__ uy,
                                                         const double* __restrict__ escale, long long n,
                                                         float* __restrict__ feat, float* __restrict__ dmu,
                                                         double* __restrict__ mu,
                                                         unsigned long long* __restrict__ stats) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    NewtonCount nc = {0, 0, 0, 0};
    if (i < n) {
        const double r = rho[i], u = ux[i], v = uy[i];
        double fi[9];
        feq_entropic<D2Q9, double>(r, u, v, 0.0, fi);
        double e2iso = 0.0;
#pragma unroll
        for (int j = 0; j < 9; j++) e2iso += (double)(D2Q9::cx(j) * D2Q9::cx(j) + D2Q9::cy(j) * D2Q9::cy(j)) * fi[j];
        const double e2 = escale[i] * e2iso;
        float a[3] = {3.0f * (float)u, 3.0f * (float)v, 0.0f};
        double fs[9], a64[3];
        energy_solve(r, u, v, e2 / r, a, fs, nc, 4e-15, a64);
        const double m[4] = {log(fs[0] / D2Q9::w(0)), a64[0], a64[1], a64[2]};
        const double m0[4] = {log(r) - 1.5 * (u * u + v * v), 3.0 * u, 3.0 * v, 0.0};
        const double f[4] = {r, u, v, e2 / r - u * u - v * v};
#pragma unroll
        for (int j = 0; j < 4; j++) {
            feat[i * 4 + j] = (float)f[j];
            dmu[i * 4 + j] = (float)(m[j] - m0[j]);
            if (mu) mu[i * 4 + j] = m[j];
        }
    }
    if (stats) {
        unsigned long long v4[4] = {nc.it32, nc.it64, nc.sites, nc.fails};
#pragma unroll
        for (int j = 0; j < 4; j++) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v4[j] += __shfl_xor_sync(0xffffffffu, v4[j], o);
        }
        if ((threadIdx.x & 31) == 0 && v4[2] > 0)
            for (int j = 0; j < 4; j++) atomicAdd(stats + j, v4[j]);
    }
}

// ---------------------------------------------------------------------------
// Standardisation of the features (mean, 1 / standard deviation) and the
// output scales (root mean square of mu - mu0) from a data set; one block,
// FP64 sums in a fixed order.
// ---------------------------------------------------------------------------
constexpr int kNormThreads = 1024;

__global__ void __launch_bounds__(kNormThreads) k_mlp_normalise(float* __restrict__ p,
                                                                 const float* __restrict__ feat,
                                                                 const float* __restrict__ dmu, long long n) {
    __shared__ double red[12][kNormThreads / 32];
    double acc[12];
#pragma unroll
    for (int j = 0; j < 12; j++) acc[j] = 0.0;
    for (long long i = threadIdx.x; i < n; i += kNormThreads) {
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const double f = feat[i * 4 + j], d = dmu[i * 4 + j];
            acc[j] += f;
            acc[4 + j] += f * f;
            acc[8 + j] += d * d;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < 12; j++) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
        if (lane == 0) red[j][warp] = acc[j];
    }
    __syncthreads();
    if (threadIdx.x < 12) {
        double s = 0.0;
        for (int w = 0; w < kNormThreads / 32; w++) s += red[threadIdx.x][w];
        red[threadIdx.x][0] = s;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        const int j = threadIdx.x;
        const double mean = red[j][0] / (double)n;
        const double var = red[4 + j][0] / (double)n - mean * mean;
        const double sd = var > 0.0 ? sqrt(var) : 0.0;
        const double rms = sqrt(red[8 + j][0] / (double)n);
        p[kMlpMean + j] = (float)mean;
        p[kMlpIstd + j] = sd > 0.0 ? (float)(1.0 / sd) : 1.0f;
        p[kMlpOscale + j] = rms > 0.0 ? (float)rms : 1.0f;
    }
}

// ---------------------------------------------------------------------------
// The network on a batch: y[i][0..3] for features feat[i][0..3].
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_mlp_forward(const float* __restrict__ p,
                                                     const float* __restrict__ feat, long long n,
                                                     float* __restrict__ y) {
    __shared__ MlpSmem ms;
    mlp_fill(ms, p);
    __syncthreads();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < n;
    unsigned p01 = 0u, p23 = 0u;
    if (valid) mlp_inputs(ms, feat[i * 4], feat[i * 4 + 1], feat[i * 4 + 2], feat[i * 4 + 3], p01, p23);
    float out[kMlpOut];
    mlp_warp_forward<false>(ms, p01, p23, out);
    if (valid)
        for (int j = 0; j < kMlpOut; j++) y[i * 4 + j] = out[j];
}

// ---------------------------------------------------------------------------
// Loss gradient, per block of kTrainRows samples: forward pass (capturing
// the BF16 activations), backward pass one sample per thread, and the
// block's sums of every trainable entry's gradient and of the squared
// errors.  Samples i0 .. i0 + n - 1; targets (mu - mu0) / out_scale;
// inv_count = 1 / (4 x batch size) (the loss is the mean over the batch and
// the four outputs).
// ---------------------------------------------------------------------------
struct TrainSmem {
    MlpSmem ms;
    float w2[kMlpHid][kMlpHid];        // BF16-rounded W2, W3 as floats
    float w3[kMlpOut][kMlpHid];
    float h1[kTrainRows][kLd], h2[kTrainRows][kLd];
    float dz1[kTrainRows][kLd], dz2[kTrainRows][kLd];
    float x[kTrainRows][kMlpIn], dy[kTrainRows][kMlpOut];
    float loss[kTrainRows];
};

__global__ void __launch_bounds__(kTrainRows) k_mlp_grad(const float* __restrict__ p,
                                                         const float* __restrict__ feat,
                                                         const float* __restrict__ dmu, long long i0,
                                                         int n, float inv_count,
                                                         float* __restrict__ partial) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TrainSmem& s = *reinterpret_cast<TrainSmem*>(smem_raw);
    const int tid = threadIdx.x;
    mlp_fill(s.ms, p);
    for (int e = tid; e < kMlpHid * kMlpHid; e += kTrainRows)
        s.w2[e / kMlpHid][e % kMlpHid] = bf16_round(p[kMlpW2 + e]);
    for (int e = tid; e < kMlpOut * kMlpHid; e += kTrainRows)
        s.w3[e / kMlpHid][e % kMlpHid] = bf16_round(p[kMlpW3 + e]);
    __syncthreads();
    const int r = tid;
    const int i = blockIdx.x * kTrainRows + r;
    const bool valid = i < n;
    float tg[kMlpOut] = {0.0f, 0.0f, 0.0f, 0.0f};
    unsigned p01 = 0u, p23 = 0u;
    if (valid) {
        const float* f = feat + (i0 + i) * 4;
        const float* d = dmu + (i0 + i) * 4;
        mlp_inputs(s.ms, f[0], f[1], f[2], f[3], p01, p23);
        for (int j = 0; j < kMlpOut; j++) tg[j] = d[j] / s.ms.oscale[j];
    }
    float y[kMlpOut];
    const int w0 = tid & ~31;
    mlp_warp_forward<true>(s.ms, p01, p23, y, &s.h1[w0][0], &s.h2[w0][0], kLd);
    s.x[r][0] = bf16_lo(p01);
    s.x[r][1] = bf16_hi(p01);
    s.x[r][2] = bf16_lo(p23);
    s.x[r][3] = bf16_hi(p23);
    float l = 0.0f;
#pragma unroll
    for (int j = 0; j < kMlpOut; j++) {
        const float d = valid ? y[j] - tg[j] : 0.0f;
        l += d * d;
        s.dy[r][j] = 2.0f * d * inv_count;
    }
    s.loss[r] = l;
    __syncthreads();
    // dz2 = (dy W3) where z2 > 0
    for (int k = 0; k < kMlpHid; k++) {
        float a = 0.0f;
#pragma unroll
        for (int j = 0; j < kMlpOut; j++) a += s.dy[r][j] * s.w3[j][k];
        s.dz2[r][k] = s.h2[r][k] > 0.0f ? a : 0.0f;
    }
    // dz1 = (dz2 W2) where z1 > 0
    float acc[kMlpHid];
#pragma unroll
    for (int k = 0; k < kMlpHid; k++) acc[k] = 0.0f;
    for (int k = 0; k < kMlpHid; k++) {
        const float d = s.dz2[r][k];
#pragma unroll
        for (int k2 = 0; k2 < kMlpHid; k2++) acc[k2] += d * s.w2[k][k2];
    }
#pragma unroll
    for (int k = 0; k < kMlpHid; k++) s.dz1[r][k] = s.h1[r][k] > 0.0f ? acc[k] : 0.0f;
    __syncthreads();
    // the block's sums over its samples, in sample order
    float* out = partial + (size_t)blockIdx.x * kPartial;
    for (int e = tid; e < kMlpTrainable; e += kTrainRows) {
        float a = 0.0f;
        if (e < kMlpB1) {
            const int nn = e / kMlpIn, k = e % kMlpIn;
            for (int q = 0; q < kTrainRows; q++) a += s.dz1[q][nn] * s.x[q][k];
        } else if (e < kMlpW2) {
            const int nn = e - kMlpB1;
            for (int q = 0; q < kTrainRows; q++) a += s.dz1[q][nn];
        } else if (e < kMlpB2) {
            const int nn = (e - kMlpW2) / kMlpHid, k = (e - kMlpW2) % kMlpHid;
            for (int q = 0; q < kTrainRows; q++) a += s.dz2[q][nn] * s.h1[q][k];
        } else if (e < kMlpW3) {
            const int nn = e - kMlpB2;
            for (int q = 0; q < kTrainRows; q++) a += s.dz2[q][nn];
        } else if (e < kMlpB3) {
            const int j = (e - kMlpW3) / kMlpHid, k = (e - kMlpW3) % kMlpHid;
            for (int q = 0; q < kTrainRows; q++) a += s.dy[q][j] * s.h2[q][k];
        } else {
            const int j = e - kMlpB3;
            for (int q = 0; q < kTrainRows; q++) a += s.dy[q][j];
        }
        out[e] = a;
    }
    if (tid == 0) {
        float a = 0.0f;
        for (int q = 0; q < kTrainRows; q++) a += s.loss[q];
        out[kMlpTrainable] = a;
    }
}

// Sum of the block partials (fixed order) -> gradient and loss; then,
// when t > 0, the Adam update of step t (Kingma and Ba, 2015):
//   m <- b1 m + (1 - b1) g,  v <- b2 v + (1 - b2) g^2,
//   p <- p - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
// loss_log (optional) accumulates loss x log_scale.
__global__ void __launch_bounds__(kReduceThreads) k_mlp_reduce(const float* __restrict__ partial, int nblk,
                                                               float* __restrict__ grad, float* loss_out,
                                                               float loss_scale, float* __restrict__ p,
                                                               float* __restrict__ m, float* __restrict__ v,
                                                               float lr, float c1, float c2,
                                                               float* loss_log, float log_scale) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < kMlpTrainable) {
        float g = 0.0f;
        for (int b = 0; b < nblk; b++) g += partial[(size_t)b * kPartial + e];
        if (grad) grad[e] = g;
        if (p) {
            const float mm = kAdamB1 * m[e] + kAdam1mB1 * g;
            const float vv = kAdamB2 * v[e] + kAdam1mB2 * (g * g);
            m[e] = mm;
            v[e] = vv;
            p[e] -= lr * (mm * c1) / (sqrtf(vv * c2) + kAdamEps);
        }
    } else if (e < kMlpParams) {
        if (grad) grad[e] = 0.0f;
    } else if (e == kMlpParams) {
        float a = 0.0f;
        for (int b = 0; b < nblk; b++) a += partial[(size_t)b * kPartial + kMlpTrainable];
        const float loss = a * loss_scale;
        if (loss_out) *loss_out = loss;
        if (loss_log) *loss_log += loss * log_scale;
    }
}

// Adam on a given gradient (every trainable entry).
__global__ void __launch_bounds__(kReduceThreads) k_mlp_adam(float* __restrict__ p, const float* __restrict__ g,
                                                             float* __restrict__ m, float* __restrict__ v,
                                                             float lr, float c1, float c2) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= kMlpTrainable) return;
    const float gg = g[e];
    const float mm = kAdamB1 * m[e] + kAdam1mB1 * gg;
    const float vv = kAdamB2 * v[e] + kAdam1mB2 * (gg * gg);
    m[e] = mm;
    v[e] = vv;
    p[e] -= lr * (mm * c1) / (sqrtf(vv * c2) + kAdamEps);
}

constexpr unsigned reduce_blocks() { return (kMlpParams + 1 + kReduceThreads - 1) / kReduceThreads; }

// one-time opt-in to the training kernel's shared memory (per device)
cudaError_t grad_setup() {
    return cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(TrainSmem));
}

cudaError_t launch_grad(const float* p, const float* feat, const float* dmu, long long i0, int n,
                        float* partial, cudaStream_t st) {
    const unsigned blocks = (unsigned)((n + kTrainRows - 1) / kTrainRows);
    k_mlp_grad<<<blocks, kTrainRows, sizeof(TrainSmem), st>>>(p, feat, dmu, i0, n,
                                                              1.0f / (4.0f * (float)n), partial);
    return cudaGetLastError();
}

// Adam's bias corrections 1 / (1 - b^t)
void adam_corrections(long long t, float& c1, float& c2) {
    c1 = (float)(1.0 / (1.0 - std::pow(kAdamB1d, (double)t)));
    c2 = (float)(1.0 / (1.0 - std::pow(kAdamB2d, (double)t)));
}

// SplitMix64 (Steele, Lea and Flood, 2014)
unsigned long long splitmix64(unsigned long long& s) {
    unsigned long long z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace

extern "C" {

int lb_mlp_init(float* params, int n, unsigned long long seed) {
    if (!params) return fail(LB_ERR_ARG, "params is NULL");
    if (n != kMlpParams) return fail(LB_ERR_ARG, "expected %d parameters", kMlpParams);
    unsigned long long s = seed;
    auto uni = [&]() { return 2.0 * (double)(splitmix64(s) >> 11) * 0x1p-53 - 1.0; };
    for (int i = 0; i < n; i++) params[i] = 0.0f;
    for (int i = 0; i < kMlpHid * kMlpIn; i++) params[kMlpW1 + i] = (float)(uni() * std::sqrt(6.0 / kMlpIn));
    for (int i = 0; i < kMlpHid * kMlpHid; i++) params[kMlpW2 + i] = (float)(uni() * std::sqrt(6.0 / kMlpHid));
    for (int i = 0; i < kMlpOut * kMlpHid; i++) params[kMlpW3 + i] = (float)(uni() * std::sqrt(6.0 / kMlpHid));
    for (int j = 0; j < 4; j++) {
        params[kMlpIstd + j] = 1.0f;
        params[kMlpOscale + j] = 1.0f;
    }
    return LB_OK;
}

int lb_energy_dataset(const double* rho, const double* ux, const double* uy, const double* escale,
                      long long n, float* feat, float* dmu, double* mu, unsigned long long* stats,
                      void* cuda_stream) {
    if (n < 0) return fail(LB_ERR_ARG, "n must be >= 0");
    if (n > 0 && (!rho || !ux || !uy || !escale || !feat || !dmu))
        return fail(LB_ERR_ARG, "NULL argument");
    if (n == 0) return LB_OK;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const long long blocks = (n + 255) / 256;
    if (blocks > 0x7fffffffll) return fail(LB_ERR_ARG, "n too large");
    k_energy_dataset<<<(unsigned)blocks, 256, 0, st>>>(rho, ux, uy, escale, n, feat, dmu, mu, stats);
    CK(cudaGetLastError());
    return LB_OK;
}

int lb_mlp_normalise(float* params, const float* feat, const float* dmu, long long n, void* cuda_stream) {
    if (!params || !feat || !dmu) return fail(LB_ERR_ARG, "NULL argument");
    if (n <= 0) return fail(LB_ERR_ARG, "n must be > 0");
    k_mlp_normalise<<<1, kNormThreads, 0, static_cast<cudaStream_t>(cuda_stream)>>>(params, feat, dmu, n);
    CK(cudaGetLastError());
    return LB_OK;
}

int lb_mlp_forward(const float* params, const float* feat, long long n, float* y, void* cuda_stream) {
    if (n < 0) return fail(LB_ERR_ARG, "n must be >= 0");
    if (n > 0 && (!params || !feat || !y)) return fail(LB_ERR_ARG, "NULL argument");
    if (n == 0) return LB_OK;
    const long long blocks = (n + 127) / 128;
    if (blocks > 0x7fffffffll) return fail(LB_ERR_ARG, "n too large");
    k_mlp_forward<<<(unsigned)blocks, 128, 0, static_cast<cudaStream_t>(cuda_stream)>>>(params, feat, n, y);
    CK(cudaGetLastError());
    return LB_OK;
}

int lb_mlp_grad(const float* params, const float* feat, const float* dmu, int n, float* grad,
                float* loss, void* cuda_stream) {
    if (!params || !feat || !dmu || !grad) return fail(LB_ERR_ARG, "NULL argument");
    if (n <= 0) return fail(LB_ERR_ARG, "n must be > 0");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    CK(grad_setup());
    const int nblk = (n + kTrainRows - 1) / kTrainRows;
    float* partial = nullptr;
    CK(cudaMallocAsync(&partial, (size_t)nblk * kPartial * sizeof(float), st));
    cudaError_t e = launch_grad(params, feat, dmu, 0, n, partial, st);
    if (e == cudaSuccess) {
        k_mlp_reduce<<<reduce_blocks(), kReduceThreads, 0, st>>>(partial, nblk, grad, loss,
                                                                 1.0f / (4.0f * (float)n), nullptr,
                                                                 nullptr, nullptr, 0.0f, 0.0f, 0.0f,
                                                                 nullptr, 0.0f);
        e = cudaGetLastError();
    }
    cudaFreeAsync(partial, st);
    CK(e);
    return LB_OK;
}

int lb_mlp_adam(float* params, const float* grad, float* m, float* v, long long t, double lr,
                void* cuda_stream) {
    if (!params || !grad || !m || !v) return fail(LB_ERR_ARG, "NULL argument");
    if (t < 1) return fail(LB_ERR_ARG, "t must be >= 1");
    if (!(lr >= 0.0) || !std::isfinite(lr)) return fail(LB_ERR_ARG, "lr must be finite and >= 0");
    float c1, c2;
    adam_corrections(t, c1, c2);
    k_mlp_adam<<<(kMlpTrainable + kReduceThreads - 1) / kReduceThreads, kReduceThreads, 0,
                 static_cast<cudaStream_t>(cuda_stream)>>>(params, grad, m, v, (float)lr, c1, c2);
    CK(cudaGetLastError());
    return LB_OK;
}

int lb_mlp_train(float* params, const float* feat, const float* dmu, long long n, int batch, int epochs,
                 double lr0, double lr1, float* loss_log, void* cuda_stream) {
    if (!params || !feat || !dmu) return fail(LB_ERR_ARG, "NULL argument");
    if (n <= 0 || batch <= 0 || epochs < 0) return fail(LB_ERR_ARG, "n, batch must be > 0, epochs >= 0");
    if (batch > (1 << 24)) return fail(LB_ERR_ARG, "batch too large");
    if (!(lr0 > 0.0) || !(lr1 > 0.0) || !std::isfinite(lr0) || !std::isfinite(lr1))
        return fail(LB_ERR_ARG, "learning rates must be positive and finite");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    CK(grad_setup());
    const long long nb = (n + batch - 1) / batch;
    const int nblk_max = (batch + kTrainRows - 1) / kTrainRows;
    float *partial = nullptr, *mv = nullptr;
    CK(cudaMallocAsync(&partial, (size_t)nblk_max * kPartial * sizeof(float), st));
    cudaError_t e = cudaMallocAsync(&mv, 2 * (size_t)kMlpParams * sizeof(float), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(mv, 0, 2 * (size_t)kMlpParams * sizeof(float), st);
    if (e == cudaSuccess && loss_log) e = cudaMemsetAsync(loss_log, 0, (size_t)epochs * sizeof(float), st);
    const long long total = nb * (long long)epochs;
    long long t = 0;
    for (int ep = 0; ep < epochs && e == cudaSuccess; ep++) {
        for (long long b = 0; b < nb && e == cudaSuccess; b++) {
            const long long i0 = b * batch;
            const int nn = (int)std::min<long long>(batch, n - i0);
            const int nblk = (nn + kTrainRows - 1) / kTrainRows;
            const double lr = lr0 * std::pow(lr1 / lr0, total > 1 ? (double)t / (double)(total - 1) : 0.0);
            t++;
            float c1, c2;
            adam_corrections(t, c1, c2);
            e = launch_grad(params, feat, dmu, i0, nn, partial, st);
            if (e != cudaSuccess) break;
            k_mlp_reduce<<<reduce_blocks(), kReduceThreads, 0, st>>>(
                partial, nblk, nullptr, nullptr, 1.0f / (4.0f * (float)nn), params, mv, mv + kMlpParams,
                (float)lr, c1, c2, loss_log ? loss_log + ep : nullptr, (float)(1.0 / (double)nb));
            e = cudaGetLastError();
        }
    }
    if (mv) cudaFreeAsync(mv, st);
    cudaFreeAsync(partial, st);
    CK(e);
    return LB_OK;
}

}  // extern "C"
