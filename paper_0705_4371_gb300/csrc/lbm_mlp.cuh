// lbm_mlp.cuh -- the 4-64-64-4 network that warm-starts the energy Newton
// solve (learned form).  Inputs: the site's features (rho, u_x, u_y,
// theta = 2E/rho - |u|^2), standardised; outputs: the scaled corrections
// (mu - mu0) / out_scale of the four Lagrange multipliers of
// ln(f*_i / W_i) = mu . (1, v_x, v_y, |v|^2) (Sec. 3.3) about the
// polynomial start point mu0 = (ln rho - 3/2 |u|^2, 3 u_x, 3 u_y, 0).
// ReLU hidden layers.
//
// Parameters: one FP32 vector (the master copy)
//   W1[64][4] b1[64] W2[64][64] b2[64] W3[4][64] b3[4] mean[4] inv_std[4]
//   out_scale[4]
// Evaluation is one warp per 32 sites on the tensor cores
// (mma.sync m16n8k16, BF16 operands, FP32 accumulation): the standardised
// inputs, the weights and the hidden activations are rounded to BF16 (round
// to nearest even), biases are added in FP32 (they initialise the
// accumulators).  The hidden layer's output fragments are re-packed in
// registers as the next layer's input fragments, so the activations never
// leave the registers.
#pragma once

#include <cstdint>

namespace lbm {

constexpr int kMlpIn = 4, kMlpHid = 64, kMlpOut = 4;
constexpr int kMlpW1 = 0;
constexpr int kMlpB1 = kMlpW1 + kMlpHid * kMlpIn;      // 256
constexpr int kMlpW2 = kMlpB1 + kMlpHid;               // 320
constexpr int kMlpB2 = kMlpW2 + kMlpHid * kMlpHid;     // 4416
constexpr int kMlpW3 = kMlpB2 + kMlpHid;               // 4480
constexpr int kMlpB3 = kMlpW3 + kMlpOut * kMlpHid;     // 4736
constexpr int kMlpMean = kMlpB3 + kMlpOut;             // 4740
constexpr int kMlpIstd = kMlpMean + kMlpIn;            // 4744
constexpr int kMlpOscale = kMlpIstd + kMlpIn;          // 4748
constexpr int kMlpParams = kMlpOscale + kMlpOut;       // 4752
constexpr int kMlpTrainable = kMlpMean;                // entries below this are trained

// The network's weights in mma fragment order (BF16 pairs), biases and
// normalisation, in shared memory.  [n-tile][k-step][lane] for W2,
// [k-step][lane] for W3 (outputs 4..7 of its n-tile are zero), [n-tile][lane]
// for W1 (its k-step has inputs 0..3; inputs 4..15 are zero).
struct MlpSmem {
    unsigned w1[8][32];
    uint2 w2[8][4][32];
    uint2 w3[4][32];
    float b1[kMlpHid], b2[kMlpHid], b3[8];
    float mean[kMlpIn], istd[kMlpIn], oscale[kMlpOut];
};

// Two FP32 values to a BF16 pair (round to nearest even); lo in the low half.
__device__ __forceinline__ unsigned bf16_pack(float lo, float hi) {
    unsigned d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}
// The same after ReLU (max(x, 0)).
__device__ __forceinline__ unsigned bf16_pack_relu(float lo, float hi) {
    unsigned d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}
__device__ __forceinline__ float bf16_lo(unsigned u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float bf16_hi(unsigned u) { return __uint_as_float(u & 0xffff0000u); }

// D = A B + D, m16n8k16, BF16 A (row) and B (col), FP32 accumulators.
__device__ __forceinline__ void mma_bf16(float* c, unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                         unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Block-cooperative fill of the shared copy from the FP32 parameter vector
// (the caller synchronises before use).
__device__ __forceinline__ void mlp_fill(MlpSmem& s, const float* __restrict__ p) {
    const int tid = threadIdx.x, nt_ = blockDim.x;
    for (int e = tid; e < 8 * 32; e += nt_) {
        const int nt = e >> 5, lane = e & 31, g = lane >> 2, tig = lane & 3;
        const int n = 8 * nt + g, k = 2 * tig;
        s.w1[nt][lane] = tig < 2 ? bf16_pack(p[kMlpW1 + n * kMlpIn + k], p[kMlpW1 + n * kMlpIn + k + 1])
                                 : 0u;
    }
    for (int e = tid; e < 8 * 4 * 32; e += nt_) {
        const int nt = e >> 7, ks = (e >> 5) & 3, lane = e & 31, g = lane >> 2, tig = lane & 3;
        const float* row = p + kMlpW2 + (8 * nt + g) * kMlpHid + 16 * ks + 2 * tig;
        s.w2[nt][ks][lane] = make_uint2(bf16_pack(row[0], row[1]), bf16_pack(row[8], row[9]));
    }
    for (int e = tid; e < 4 * 32; e += nt_) {
        const int ks = e >> 5, lane = e & 31, g = lane >> 2, tig = lane & 3;
        if (g < kMlpOut) {
            const float* row = p + kMlpW3 + g * kMlpHid + 16 * ks + 2 * tig;
            s.w3[ks][lane] = make_uint2(bf16_pack(row[0], row[1]), bf16_pack(row[8], row[9]));
        } else {
            s.w3[ks][lane] = make_uint2(0u, 0u);
        }
    }
    for (int e = tid; e < kMlpHid; e += nt_) {
        s.b1[e] = p[kMlpB1 + e];
        s.b2[e] = p[kMlpB2 + e];
    }
    for (int e = tid; e < 8; e += nt_) s.b3[e] = e < kMlpOut ? p[kMlpB3 + e] : 0.0f;
    for (int e = tid; e < kMlpIn; e += nt_) {
        s.mean[e] = p[kMlpMean + e];
        s.istd[e] = p[kMlpIstd + e];
        s.oscale[e] = p[kMlpOscale + e];
    }
}

// Standardised features (FP32: (f - mean) * inv_std) rounded to two BF16
// pairs (inputs 0, 1 and 2, 3).
__device__ __forceinline__ void mlp_inputs(const MlpSmem& s, float f0, float f1, float f2, float f3,
                                           unsigned& p01, unsigned& p23) {
    p01 = bf16_pack((f0 - s.mean[0]) * s.istd[0], (f1 - s.mean[1]) * s.istd[1]);
    p23 = bf16_pack((f2 - s.mean[2]) * s.istd[2], (f3 - s.mean[3]) * s.istd[3]);
}

// Forward pass of the network for the warp's 32 sites, lane l holding site
// l: inputs (p01, p23) from mlp_inputs, outputs y[0..3].  Every lane of the
// warp must call it (lanes without a site pass zeros and ignore y).
// CAP: also store the hidden activations (BF16 values, after ReLU) of site
// l at h1[l * ld + j], h2[l * ld + j] (training).
template <bool CAP>
__device__ __forceinline__ void mlp_warp_forward(const MlpSmem& s, unsigned p01, unsigned p23, float* y,
                                                 float* h1 = nullptr, float* h2 = nullptr, int ld = 0) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, g = lane >> 2, tig = lane & 3;
#pragma unroll
    for (int m = 0; m < 2; m++) {
        // rows r0, r1 of this 16-site tile; input columns 2 tig, 2 tig + 1
        const int r0 = 16 * m + g, r1 = r0 + 8;
        const unsigned x0lo = __shfl_sync(FULL, p01, r0), x0hi = __shfl_sync(FULL, p23, r0);
        const unsigned x1lo = __shfl_sync(FULL, p01, r1), x1hi = __shfl_sync(FULL, p23, r1);
        const unsigned a0 = tig == 0 ? x0lo : (tig == 1 ? x0hi : 0u);
        const unsigned a1 = tig == 0 ? x1lo : (tig == 1 ? x1hi : 0u);
        // layer 1; its n-tiles 2j, 2j+1 form k-step j of layer 2
        unsigned A2[4][4];
#pragma unroll
        for (int nt = 0; nt < 8; nt++) {
            const float bl = s.b1[8 * nt + 2 * tig], bh = s.b1[8 * nt + 2 * tig + 1];
            float c[4] = {bl, bh, bl, bh};
            mma_bf16(c, a0, a1, 0u, 0u, s.w1[nt][lane], 0u);
            const unsigned u0 = bf16_pack_relu(c[0], c[1]), u1 = bf16_pack_relu(c[2], c[3]);
            A2[nt >> 1][(nt & 1) * 2 + 0] = u0;
            A2[nt >> 1][(nt & 1) * 2 + 1] = u1;
            if constexpr (CAP) {
                const int col = 8 * nt + 2 * tig;
                h1[r0 * ld + col] = bf16_lo(u0);
                h1[r0 * ld + col + 1] = bf16_hi(u0);
                h1[r1 * ld + col] = bf16_lo(u1);
                h1[r1 * ld + col + 1] = bf16_hi(u1);
            }
        }
        // layers 2 and 3: each pair of layer-2 n-tiles is one layer-3 k-step
        float yc[4] = {s.b3[2 * tig], s.b3[2 * tig + 1], s.b3[2 * tig], s.b3[2 * tig + 1]};
#pragma unroll
        for (int jp = 0; jp < 4; jp++) {
            unsigned A3[4];
#pragma unroll
            for (int hh = 0; hh < 2; hh++) {
                const int nt = 2 * jp + hh;
                const float bl = s.b2[8 * nt + 2 * tig], bh = s.b2[8 * nt + 2 * tig + 1];
                float c[4] = {bl, bh, bl, bh};
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    const uint2 b = s.w2[nt][j][lane];
                    mma_bf16(c, A2[j][0], A2[j][1], A2[j][2], A2[j][3], b.x, b.y);
                }
                const unsigned u0 = bf16_pack_relu(c[0], c[1]), u1 = bf16_pack_relu(c[2], c[3]);
                A3[2 * hh] = u0;
                A3[2 * hh + 1] = u1;
                if constexpr (CAP) {
                    const int col = 8 * nt + 2 * tig;
                    h2[r0 * ld + col] = bf16_lo(u0);
                    h2[r0 * ld + col + 1] = bf16_hi(u0);
                    h2[r1 * ld + col] = bf16_lo(u1);
                    h2[r1 * ld + col + 1] = bf16_hi(u1);
                }
            }
            const uint2 b = s.w3[jp][lane];
            mma_bf16(yc, A3[0], A3[1], A3[2], A3[3], b.x, b.y);
        }
        // output j of tile row r sits in lane 4 (r mod 8) + j / 2, register
        // (j mod 2) (+2 for rows 8..15): bring it to lane 16 m + r
#pragma unroll
        for (int j = 0; j < kMlpOut; j++) {
            const int src = 4 * (lane & 7) + (j >> 1);
            const float lo = __shfl_sync(FULL, yc[j & 1], src);
            const float hi = __shfl_sync(FULL, yc[2 + (j & 1)], src);
            if ((lane >> 4) == m) y[j] = (lane & 8) ? hi : lo;
        }
    }
}

// Warm start of the energy Newton solve: multipliers a = (mu_x, mu_y, mu_c)
// of the normalised form from the network, for the warp's 32 sites (every
// lane calls; valid = false lanes get the polynomial start).  Outputs that
// are not finite or implausibly large (|a| > 8) fall back to the polynomial
// start.
__device__ __forceinline__ void mlp_warm_start(const MlpSmem& s, bool valid, float rho, float ux,
                                               float uy, float e2, float* a) {
    const float th = valid ? e2 / rho - ux * ux - uy * uy : 0.0f;
    unsigned p01 = 0u, p23 = 0u;
    if (valid) mlp_inputs(s, rho, ux, uy, th, p01, p23);
    float y[kMlpOut] = {0.0f, 0.0f, 0.0f, 0.0f};
    mlp_warp_forward<false>(s, p01, p23, y);
    a[0] = 3.0f * ux;
    a[1] = 3.0f * uy;
    a[2] = 0.0f;
    if (!valid) return;
    const float c0 = a[0] + s.oscale[1] * y[1];
    const float c1 = a[1] + s.oscale[2] * y[2];
    const float c2 = s.oscale[3] * y[3];
    if (fabsf(c0) <= 8.0f && fabsf(c1) <= 8.0f && fabsf(c2) <= 8.0f) {   // false for NaN
        a[0] = c0;
        a[1] = c1;
        a[2] = c2;
    }
}

}  // namespace lbm
