// Learned warm start: a three-layer message-passing network on the pattern of
// C that predicts a starting factor R0 (unit rows) for the Burer-Monteiro
// solve, trained on the factors the solver returns.  The paper starts from a
// random factor; this network is an addition of this library.
//
// Network (definition shared with the CPU oracle of the tests; F = 16 input
// features, H = 32 hidden, r_out outputs, w_ij = C_ij for i != j,
// s_i = sum_j |w_ij|):
//   x_i  = [1, log(1+deg_i)/4, sum_j w_ij / s_i, C_ii / s_i, 12 SplitMix64 normals]
//   m_i  = sum_j (w_ij / s_i) h_j ;  h_i <- relu(W_s h_i + W_n m_i + b)   (3 layers)
//   o_i  = W_o h_i + b_o ;  r_hat_i = o_i / ||o_i||
//   loss = mean over edges i<j of (r_hat_i . r_hat_j - X*_ij)^2
// Activations are stored in bf16 (or float for checking) with float
// arithmetic; weights are float masters, rounded to bf16 for the forward pass
// in bf16 mode; gradients, Adam moments and every reduction are float/double.
// Weight gradients are summed per block in a fixed order and folded over the
// blocks in a fixed order (deterministic).
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/lorads.h"
#include "common.cuh"
#include "control_dev.cuh"

using namespace lorads;

namespace {

constexpr int kF = 16;            // input features
constexpr int kStruct = 4;        // structural features
constexpr int kH = 32;            // hidden width
constexpr int kLayers = 3;
constexpr int kMaxOut = 32;       // r_out <= 32
constexpr uint64_t kFeatureStream = 0x474E4E;
constexpr int kTile = 32;         // nodes per tile of the dense kernels

int64_t param_count(int r_out) {
    int64_t p = 0;
    int f = kF;
    for (int l = 0; l < kLayers; ++l) {
        p += 2LL * kH * f + kH;
        f = kH;
    }
    return p + (int64_t)r_out * kH + r_out;
}

int64_t layer_offset(int l) {
    int64_t p = 0;
    int f = kF;
    for (int q = 0; q < l; ++q) {
        p += 2LL * kH * f + kH;
        f = kH;
    }
    return p;
}

__device__ __forceinline__ float bf16_round(float v) {
    return __bfloat162float(__float2bfloat16_rn(v));
}

template <typename TA> __device__ __forceinline__ float ld_act(const TA* p) { return float(*p); }
template <> __device__ __forceinline__ float ld_act<__nv_bfloat16>(const __nv_bfloat16* p) {
    return __bfloat162float(*p);
}
template <typename TA> __device__ __forceinline__ TA to_act(float v) { return TA(v); }
template <> __device__ __forceinline__ __nv_bfloat16 to_act<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

template <typename TA> constexpr bool is_bf16() { return std::is_same<TA, __nv_bfloat16>::value; }

// ------------------------------------------------------------------ features
template <typename TA>
__global__ void k_gnn_prep(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           const double* __restrict__ cv, uint64_t seed, TA* __restrict__ x,
                           float* __restrict__ inv_s) {
    const uint64_t golden = 0x9E3779B97F4A7C15ull;
    const uint64_t base = seed ^ (kFeatureStream * golden);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double deg = 0, s = 0, ws = 0, dg = 0;
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            const double w = cv[e];
            if (ci[e] == i) {
                dg += w;
            } else {
                deg += 1;
                s += fabs(w);
                ws += w;
            }
        }
        const double is = s > 0 ? 1.0 / s : 0.0;
        inv_s[i] = (float)is;
        TA* xi = x + i * kF;
        xi[0] = to_act<TA>(1.0f);
        xi[1] = to_act<TA>((float)(log1p(deg) / 4.0));
        xi[2] = to_act<TA>((float)(ws * is));
        xi[3] = to_act<TA>((float)(dg * is));
        for (int k = 0; k < kF - kStruct; ++k)
            xi[kStruct + k] = to_act<TA>((float)normal_at(base, i * (kF - kStruct) + k));
    }
}

// ------------------------------------------------------------------ aggregation
// forward  : out_i = inv_s_i * sum_{j != i} w_ij in_j
// transpose: out_j (+)= sum_{i != j} w_ij inv_s_i in_i   (C symmetric: row j's entries)
// A group of F/4 lanes owns a row; lane l handles features 4l..4l+3.
template <typename TI, typename TO>
__global__ void k_gnn_agg(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                          const double* __restrict__ cv, const float* __restrict__ inv_s, const TI* __restrict__ in,
                          int F, TO* __restrict__ out, int transpose, int accumulate) {
    const int G = F / 4;
    const int lane = threadIdx.x & 31;
    const int lig = lane % G;
    const int rows_per_warp = 32 / G;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = warp * rows_per_warp; base < n; base += nwarps * rows_per_warp) {
        const int64_t i = base + lane / G;
        if (i >= n || lane >= rows_per_warp * G) continue;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            const int j = ci[e];
            if (j == i) continue;
            float w = (float)cv[e];
            if (transpose) w *= inv_s[j];
            const TI* src = in + (int64_t)j * F + 4 * lig;
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[c] = fmaf(w, ld_act<TI>(src + c), acc[c]);
        }
        const float sc = transpose ? 1.0f : inv_s[i];
        TO* dst = out + i * F + 4 * lig;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float v = acc[c] * sc;
            if (accumulate) v += float(dst[c]);
            dst[c] = to_act<TO>(v);
        }
    }
}

// ------------------------------------------------------------------ dense layer
// h_out = relu(W_s h_in + W_n m + b); 8 threads per node, 4 outputs each.
template <typename TA>
__global__ void __launch_bounds__(256)
k_gnn_dense(int64_t n, const TA* __restrict__ hin, const TA* __restrict__ min_, int F,
            const float* __restrict__ theta_l, TA* __restrict__ hout) {
    __shared__ float Ws[kH * kH], Wn[kH * kH], b[kH];
    for (int e = threadIdx.x; e < kH * F; e += blockDim.x) {
        float a = theta_l[e], c = theta_l[kH * F + e];
        if (is_bf16<TA>()) { a = bf16_round(a); c = bf16_round(c); }
        Ws[e] = a;
        Wn[e] = c;
    }
    for (int e = threadIdx.x; e < kH; e += blockDim.x) {
        float a = theta_l[2 * kH * F + e];
        b[e] = is_bf16<TA>() ? bf16_round(a) : a;
    }
    __syncthreads();
    const int sub = threadIdx.x & 7;                 // outputs 4*sub .. 4*sub+3
    for (int64_t i = blockIdx.x * (int64_t)(blockDim.x / 8) + threadIdx.x / 8; i < n;
         i += (int64_t)gridDim.x * (blockDim.x / 8)) {
        float u[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) u[c] = b[4 * sub + c];
        for (int k = 0; k < F; ++k) {
            const float hv = ld_act<TA>(hin + i * F + k);
            const float mv = ld_act<TA>(min_ + i * F + k);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int o = 4 * sub + c;
                u[c] = fmaf(Ws[o * F + k], hv, fmaf(Wn[o * F + k], mv, u[c]));
            }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) hout[i * kH + 4 * sub + c] = to_act<TA>(fmaxf(u[c], 0.0f));
    }
}

// ------------------------------------------------------------------ output layer
template <typename TA>
__global__ void __launch_bounds__(256)
k_gnn_out(int64_t n, const TA* __restrict__ h, const float* __restrict__ theta_o, int r_out,
          float* __restrict__ rhat, float* __restrict__ onrm, double* __restrict__ R, int ld) {
    __shared__ float Wo[kMaxOut * kH], bo[kMaxOut];
    for (int e = threadIdx.x; e < r_out * kH; e += blockDim.x) {
        const float a = theta_o[e];
        Wo[e] = is_bf16<TA>() ? bf16_round(a) : a;
    }
    for (int e = threadIdx.x; e < r_out; e += blockDim.x) {
        const float a = theta_o[r_out * kH + e];
        bo[e] = is_bf16<TA>() ? bf16_round(a) : a;
    }
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float hv[kH];
#pragma unroll
        for (int k = 0; k < kH; ++k) hv[k] = ld_act<TA>(h + i * kH + k);
        float o[kMaxOut];
        float nn = 0.f;
        for (int c = 0; c < r_out; ++c) {
            float v = bo[c];
#pragma unroll
            for (int k = 0; k < kH; ++k) v = fmaf(Wo[c * kH + k], hv[k], v);
            o[c] = v;
            nn = fmaf(v, v, nn);
        }
        const float nrm = sqrtf(nn);
        const float inv = nrm > 0.f ? 1.0f / nrm : 0.f;
        if (onrm) onrm[i] = nrm;
        for (int c = 0; c < r_out; ++c) {
            const float v = o[c] * inv;
            if (rhat) rhat[i * r_out + c] = v;
            if (R) R[i * ld + c] = (double)v;
        }
        if (R)
            for (int c = r_out; c < ld; ++c) R[i * ld + c] = 0.0;
    }
}

// ------------------------------------------------------------------ loss
// One warp per node, lane c holds component c: loss over edges i < j and
// dL/d r_hat_i = (2 / |E|) sum_j (r_hat_i . r_hat_j - t_ij) r_hat_j.
__global__ void __launch_bounds__(256)
k_gnn_loss(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
           const float* __restrict__ rhat, int r_out, const float* __restrict__ target, float two_over_ne,
           float* __restrict__ dr, double* __restrict__ part) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double loss = 0.0;
    for (int64_t i = warp; i < n; i += nwarps) {
        const float ri = lane < r_out ? rhat[i * r_out + lane] : 0.f;
        float g = 0.f;
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            const int j = ci[e];
            if (j == i) continue;
            const float rj = lane < r_out ? rhat[(int64_t)j * r_out + lane] : 0.f;
            float d = ri * rj;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
            const float diff = d - target[e];
            if (j > i && lane == 0) loss += (double)diff * diff;
            g = fmaf(two_over_ne * diff, rj, g);
        }
        if (lane < r_out) dr[i * r_out + lane] = g;
    }
    double acc[1] = {loss};
    block_partials<1>(acc, part);
}

// ------------------------------------------------------------------ backward
// Output layer: do = (dr - r_hat (r_hat . dr)) / ||o||, dh = W_o^T do, and the
// block's partial sums of dW_o = sum do h^T, db_o = sum do.
template <typename TA>
__global__ void __launch_bounds__(256)
k_gnn_out_back(int64_t n, const TA* __restrict__ h, const float* __restrict__ rhat, const float* __restrict__ onrm,
               const float* __restrict__ dr, const float* __restrict__ theta_o, int r_out, float* __restrict__ dh,
               float* __restrict__ gpart, int64_t pstride, int64_t poff) {
    __shared__ float Wo[kMaxOut * kH];
    __shared__ float s_do[kTile][kMaxOut];
    __shared__ float s_h[kTile][kH];
    for (int e = threadIdx.x; e < r_out * kH; e += blockDim.x) {
        const float a = theta_o[e];
        Wo[e] = is_bf16<TA>() ? bf16_round(a) : a;
    }
    const int nent = r_out * kH + r_out;          // owned entries: e = tid, tid + 256, ... (<= 1056)
    float accw[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    __syncthreads();
    const int64_t ntiles = (n + kTile - 1) / kTile;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t i0 = t * kTile;
        // per node (threads 0..kTile-1): do and dh
        if (threadIdx.x < kTile) {
            const int64_t i = i0 + threadIdx.x;
            float dov[kMaxOut];
            if (i < n) {
                float dotv = 0.f;
                for (int c = 0; c < r_out; ++c) dotv = fmaf(rhat[i * r_out + c], dr[i * r_out + c], dotv);
                const float nr = onrm[i];
                const float inv = nr > 0.f ? 1.0f / nr : 0.f;
                for (int c = 0; c < r_out; ++c) dov[c] = (dr[i * r_out + c] - rhat[i * r_out + c] * dotv) * inv;
            } else {
                for (int c = 0; c < r_out; ++c) dov[c] = 0.f;
            }
            for (int c = 0; c < r_out; ++c) s_do[threadIdx.x][c] = dov[c];
            for (int k = 0; k < kH; ++k) {
                float v = 0.f;
                for (int c = 0; c < r_out; ++c) v = fmaf(Wo[c * kH + k], dov[c], v);
                if (i < n) dh[i * kH + k] = v;
                s_h[threadIdx.x][k] = i < n ? ld_act<TA>(h + i * kH + k) : 0.f;
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            const int e = threadIdx.x + q * 256;
            if (e < nent) {
                float a = accw[q];
                if (e < r_out * kH) {
                    const int c = e / kH, k = e % kH;
                    for (int u = 0; u < kTile; ++u) a = fmaf(s_do[u][c], s_h[u][k], a);
                } else {
                    const int c = e - r_out * kH;
                    for (int u = 0; u < kTile; ++u) a += s_do[u][c];
                }
                accw[q] = a;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const int e = threadIdx.x + q * 256;
        if (e < nent) gpart[blockIdx.x * pstride + poff + e] = accw[q];
    }
}

// Hidden layer l: du = dh_out * [h_out > 0]; dh_in = W_s^T du (self part),
// dm = W_n^T du; block partials of dW_s = sum du h_in^T, dW_n = sum du m^T,
// db = sum du.  The neighbour part of dh_in (A^T dm) is added by k_gnn_agg.
template <typename TA>
__global__ void __launch_bounds__(256)
k_gnn_layer_back(int64_t n, const TA* __restrict__ hin, const TA* __restrict__ min_, const TA* __restrict__ hout,
                 int F, const float* __restrict__ dh_out, const float* __restrict__ theta_l,
                 float* __restrict__ dh_in, float* __restrict__ dm, float* __restrict__ gpart, int64_t pstride,
                 int64_t poff) {
    __shared__ float Ws[kH * kH], Wn[kH * kH];
    __shared__ float s_du[kTile][kH];
    __shared__ float s_hin[kTile][kH];
    __shared__ float s_min[kTile][kH];
    for (int e = threadIdx.x; e < kH * F; e += blockDim.x) {
        float a = theta_l[e], c = theta_l[kH * F + e];
        if (is_bf16<TA>()) { a = bf16_round(a); c = bf16_round(c); }
        Ws[e] = a;
        Wn[e] = c;
    }
    const int nent = 2 * kH * F + kH;
    float accw[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) accw[q] = 0.f;
    __syncthreads();
    const int64_t ntiles = (n + kTile - 1) / kTile;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t i0 = t * kTile;
        // stage du, h_in, m of the tile (all threads)
        for (int e = threadIdx.x; e < kTile * kH; e += blockDim.x) {
            const int u = e / kH, o = e % kH;
            const int64_t i = i0 + u;
            float d = 0.f;
            if (i < n && ld_act<TA>(hout + i * kH + o) > 0.f) d = dh_out[i * kH + o];
            s_du[u][o] = d;
        }
        for (int e = threadIdx.x; e < kTile * F; e += blockDim.x) {
            const int u = e / F, k = e % F;
            const int64_t i = i0 + u;
            s_hin[u][k] = i < n ? ld_act<TA>(hin + i * F + k) : 0.f;
            s_min[u][k] = i < n ? ld_act<TA>(min_ + i * F + k) : 0.f;
        }
        __syncthreads();
        // dh_in (self) and dm for each node of the tile
        for (int e = threadIdx.x; e < kTile * F; e += blockDim.x) {
            const int u = e / F, k = e % F;
            const int64_t i = i0 + u;
            if (i >= n) continue;
            float a = 0.f, c = 0.f;
            for (int o = 0; o < kH; ++o) {
                a = fmaf(Ws[o * F + k], s_du[u][o], a);
                c = fmaf(Wn[o * F + k], s_du[u][o], c);
            }
            dh_in[i * F + k] = a;
            dm[i * F + k] = c;
        }
        // weight-gradient partials
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const int e = threadIdx.x + q * 256;
            if (e < nent) {
                float a = accw[q];
                if (e < kH * F) {
                    const int o = e / F, k = e % F;
                    for (int u = 0; u < kTile; ++u) a = fmaf(s_du[u][o], s_hin[u][k], a);
                } else if (e < 2 * kH * F) {
                    const int o = (e - kH * F) / F, k = (e - kH * F) % F;
                    for (int u = 0; u < kTile; ++u) a = fmaf(s_du[u][o], s_min[u][k], a);
                } else {
                    const int o = e - 2 * kH * F;
                    for (int u = 0; u < kTile; ++u) a += s_du[u][o];
                }
                accw[q] = a;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        const int e = threadIdx.x + q * 256;
        if (e < nent) gpart[blockIdx.x * pstride + poff + e] = accw[q];
    }
}

// grad[p] = sum over blocks of gpart[b][p] (fixed order, double accumulation)
__global__ void k_gnn_fold(const float* __restrict__ gpart, int nb, int64_t P, float* __restrict__ grad) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s += gpart[(int64_t)b * P + p];
        grad[p] = (float)s;
    }
}

// Adam (Kingma & Ba 2015) on the float master weights.
__global__ void k_gnn_adam(int64_t P, float* __restrict__ theta, const float* __restrict__ grad,
                           float* __restrict__ m1, float* __restrict__ m2, float lr, float b1, float b2, float eps,
                           float c1, float c2) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
        const float g = grad[p];
        const float a = b1 * m1[p] + (1.f - b1) * g;
        const float b = b2 * m2[p] + (1.f - b2) * g * g;
        m1[p] = a;
        m2[p] = b;
        theta[p] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
    }
}

// X*_ij = r_i . r_j on every stored entry of C (0 on the diagonal)
__global__ void k_gnn_targets(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                              const double* __restrict__ R, int r, int ld, float* __restrict__ t) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            const int j = ci[e];
            double d = 0.0;
            if (j != i)
                for (int c = 0; c < r; ++c) d += R[i * ld + c] * R[(int64_t)j * ld + c];
            t[e] = (float)d;
        }
    }
}

}  // namespace

// ====================================================================== object
struct lorads_gnn {
    int r_out = 0;
    int act = LORADS_BF16;
    int64_t P = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0, nb = 0;
    std::string err;
    float* theta = nullptr;
    float* grad = nullptr;
    float* m1 = nullptr;
    float* m2 = nullptr;
    float* gpart = nullptr;
    int64_t step = 0;
    // per-node workspace (grown on demand)
    int64_t cap = 0;
    void* x = nullptr;           // n x F  (activation type)
    void* h[kLayers] = {};       // n x H
    void* m[kLayers] = {};       // n x F_in
    float* inv_s = nullptr;
    float* rhat = nullptr;       // n x r_out
    float* onrm = nullptr;
    float* dr = nullptr;         // n x r_out
    float* dh = nullptr;         // n x H
    float* dh2 = nullptr;        // n x H
    float* dm = nullptr;         // n x H
    double* lpart = nullptr;     // loss partials
};

namespace {

#define GCK(call)                                                                          \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            cudaGetLastError();                                                            \
            g->err = std::string(#call) + ": " + cudaGetErrorString(e_);                   \
            return e_ == cudaErrorMemoryAllocation ? LORADS_ERR_OOM : LORADS_ERR_CUDA;     \
        }                                                                                  \
    } while (0)

void gfree(void* p) {
    if (p) cudaFree(p);
}

void free_ws(lorads_gnn* g) {
    gfree(g->x);
    for (int l = 0; l < kLayers; ++l) {
        gfree(g->h[l]);
        gfree(g->m[l]);
        g->h[l] = g->m[l] = nullptr;
    }
    gfree(g->inv_s); gfree(g->rhat); gfree(g->onrm); gfree(g->dr); gfree(g->dh); gfree(g->dh2); gfree(g->dm);
    g->x = nullptr;
    g->inv_s = g->rhat = g->onrm = g->dr = g->dh = g->dh2 = g->dm = nullptr;
    g->cap = 0;
}

lorads_status ensure_ws(lorads_gnn* g, int64_t n) {
    if (n <= g->cap) return LORADS_OK;
    free_ws(g);
    const size_t ea = g->act == LORADS_BF16 ? 2 : 4;
    GCK(cudaMalloc(&g->x, (size_t)n * kF * ea));
    for (int l = 0; l < kLayers; ++l) {
        GCK(cudaMalloc(&g->h[l], (size_t)n * kH * ea));
        GCK(cudaMalloc(&g->m[l], (size_t)n * kH * ea));
    }
    GCK(cudaMalloc(&g->inv_s, (size_t)n * 4));
    GCK(cudaMalloc(&g->rhat, (size_t)n * g->r_out * 4));
    GCK(cudaMalloc(&g->onrm, (size_t)n * 4));
    GCK(cudaMalloc(&g->dr, (size_t)n * g->r_out * 4));
    GCK(cudaMalloc(&g->dh, (size_t)n * kH * 4));
    GCK(cudaMalloc(&g->dh2, (size_t)n * kH * 4));
    GCK(cudaMalloc(&g->dm, (size_t)n * kH * 4));
    g->cap = n;
    return LORADS_OK;
}

int grid_for(const lorads_gnn* g, int64_t items, int per_block) {
    int64_t b = (items + per_block - 1) / per_block;
    if (b < 1) b = 1;
    return (int)std::min<int64_t>(b, (int64_t)g->num_sms * 8);
}

// forward pass: features, three layers, output rows (R: optional FP64 n x ld copy)
template <typename TA>
void forward(lorads_gnn* g, int64_t n, const int64_t* rp, const int32_t* ci, const double* cv, uint64_t seed,
             double* R, int ld) {
    cudaStream_t s = g->stream;
    TA* x = static_cast<TA*>(g->x);
    k_gnn_prep<TA><<<grid_for(g, n, 256), 256, 0, s>>>(n, rp, ci, cv, seed, x, g->inv_s);
    const TA* hin = x;
    int F = kF;
    for (int l = 0; l < kLayers; ++l) {
        TA* m = static_cast<TA*>(g->m[l]);
        TA* h = static_cast<TA*>(g->h[l]);
        k_gnn_agg<TA, TA><<<grid_for(g, n * (F / 4), 256), 256, 0, s>>>(n, rp, ci, cv, g->inv_s, hin, F, m, 0, 0);
        k_gnn_dense<TA><<<grid_for(g, n, 32), 256, 0, s>>>(n, hin, m, F, g->theta + layer_offset(l), h);
        hin = h;
        F = kH;
    }
    k_gnn_out<TA><<<grid_for(g, n, 256), 256, 0, s>>>(n, hin, g->theta + layer_offset(kLayers), g->r_out, g->rhat,
                                                       g->onrm, R, ld);
}

template <typename TA>
void backward(lorads_gnn* g, int64_t n, const int64_t* rp, const int32_t* ci, const double* cv) {
    cudaStream_t s = g->stream;
    const int nb = g->nb;
    TA* h3 = static_cast<TA*>(g->h[kLayers - 1]);
    k_gnn_out_back<TA><<<nb, 256, 0, s>>>(n, h3, g->rhat, g->onrm, g->dr, g->theta + layer_offset(kLayers),
                                           g->r_out, g->dh, g->gpart, g->P, layer_offset(kLayers));
    float* dh_out = g->dh;
    float* dh_in = g->dh2;
    for (int l = kLayers - 1; l >= 0; --l) {
        const int F = l == 0 ? kF : kH;
        const TA* hin = l == 0 ? static_cast<const TA*>(g->x) : static_cast<const TA*>(g->h[l - 1]);
        k_gnn_layer_back<TA><<<nb, 256, 0, s>>>(n, hin, static_cast<const TA*>(g->m[l]),
                                                 static_cast<const TA*>(g->h[l]), F, dh_out,
                                                 g->theta + layer_offset(l), dh_in, g->dm, g->gpart, g->P,
                                                 layer_offset(l));
        if (l > 0) {
            // dh_in += A^T dm  (the neighbour part)
            k_gnn_agg<float, float><<<grid_for(g, n * (F / 4), 256), 256, 0, s>>>(n, rp, ci, cv, g->inv_s, g->dm, F,
                                                                                   dh_in, 1, 1);
            float* t = dh_out;
            dh_out = dh_in;
            dh_in = t;
        }
    }
    k_gnn_fold<<<grid_for(g, g->P, 256), 256, 0, s>>>(g->gpart, nb, g->P, g->grad);
}

lorads_status check(lorads_gnn* g, const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        g->err = std::string(what) + ": " + cudaGetErrorString(e);
        return LORADS_ERR_CUDA;
    }
    return LORADS_OK;
}

lorads_status check_graph(lorads_gnn* g, int64_t n, const void* rp, const void* ci, const void* cv) {
    if (n < 1 || n > INT32_MAX) {
        g->err = "n must be in [1, 2^31)";
        return LORADS_ERR_INVALID_ARG;
    }
    if (!rp || !ci || !cv) {
        g->err = "null graph pointer";
        return LORADS_ERR_INVALID_ARG;
    }
    return LORADS_OK;
}

thread_local std::string g_gnn_create_error;

}  // namespace

extern "C" int64_t lorads_gnn_param_count(int32_t r_out) {
    return (r_out < 1 || r_out > kMaxOut) ? -1 : param_count(r_out);
}

extern "C" const char* lorads_gnn_last_error(const lorads_gnn* g) { return g ? g->err.c_str() : "null network"; }

extern "C" const char* lorads_gnn_create_error(void) { return g_gnn_create_error.c_str(); }

extern "C" void lorads_gnn_destroy(lorads_gnn* g) {
    if (!g) return;
    if (g->stream) cudaStreamSynchronize(g->stream);
    free_ws(g);
    gfree(g->theta); gfree(g->grad); gfree(g->m1); gfree(g->m2); gfree(g->gpart); gfree(g->lpart);
    delete g;
}

extern "C" lorads_status lorads_gnn_create(lorads_gnn** out, int32_t r_out, int32_t act_prec, const float* theta0,
                                           void* cuda_stream) {
    if (!out) return LORADS_ERR_INVALID_ARG;
    *out = nullptr;
    if (r_out < 1 || r_out > kMaxOut) {
        g_gnn_create_error = "r_out must be in [1, 32]";
        return LORADS_ERR_INVALID_ARG;
    }
    if (act_prec != LORADS_BF16 && act_prec != LORADS_FP32) {
        g_gnn_create_error = "act_prec must be LORADS_BF16 or LORADS_FP32";
        return LORADS_ERR_INVALID_ARG;
    }
    if (!theta0) {
        g_gnn_create_error = "theta0 (initial parameters) is NULL";
        return LORADS_ERR_INVALID_ARG;
    }
    lorads_gnn* g = new (std::nothrow) lorads_gnn();
    if (!g) return LORADS_ERR_OOM;
    g->r_out = r_out;
    g->act = act_prec;
    g->P = param_count(r_out);
    g->stream = static_cast<cudaStream_t>(cuda_stream);
    auto fail = [&](lorads_status s) {
        g_gnn_create_error = g->err;
        lorads_gnn_destroy(g);
        return s;
    };
#define GCREATE(call)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            cudaGetLastError();                                                            \
            g->err = std::string(#call) + ": " + cudaGetErrorString(e_);                   \
            return fail(e_ == cudaErrorMemoryAllocation ? LORADS_ERR_OOM : LORADS_ERR_CUDA); \
        }                                                                                  \
    } while (0)
    int dev = 0;
    GCREATE(cudaGetDevice(&dev));
    GCREATE(cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, dev));
    g->nb = g->num_sms * 2;
    const size_t pb = (size_t)g->P * sizeof(float);
    GCREATE(cudaMalloc(&g->theta, pb));
    GCREATE(cudaMalloc(&g->grad, pb));
    GCREATE(cudaMalloc(&g->m1, pb));
    GCREATE(cudaMalloc(&g->m2, pb));
    GCREATE(cudaMalloc(&g->gpart, pb * g->nb));
    GCREATE(cudaMalloc(&g->lpart, sizeof(double) * g->num_sms * 8));
    GCREATE(cudaMemcpy(g->theta, theta0, pb, cudaMemcpyHostToDevice));
    GCREATE(cudaMemset(g->m1, 0, pb));
    GCREATE(cudaMemset(g->m2, 0, pb));
    GCREATE(cudaMemset(g->grad, 0, pb));
#undef GCREATE
    *out = g;
    return LORADS_OK;
}

extern "C" lorads_status lorads_gnn_get_params(lorads_gnn* g, float* theta_host, int64_t count) {
    if (!g || !theta_host || count < g->P) return LORADS_ERR_INVALID_ARG;
    GCK(cudaStreamSynchronize(g->stream));
    GCK(cudaMemcpy(theta_host, g->theta, g->P * sizeof(float), cudaMemcpyDeviceToHost));
    return LORADS_OK;
}

extern "C" lorads_status lorads_gnn_set_params(lorads_gnn* g, const float* theta_host, int64_t count) {
    if (!g || !theta_host || count < g->P) return LORADS_ERR_INVALID_ARG;
    GCK(cudaStreamSynchronize(g->stream));
    GCK(cudaMemcpy(g->theta, theta_host, g->P * sizeof(float), cudaMemcpyHostToDevice));
    GCK(cudaMemset(g->m1, 0, g->P * sizeof(float)));
    GCK(cudaMemset(g->m2, 0, g->P * sizeof(float)));
    g->step = 0;
    return LORADS_OK;
}

extern "C" lorads_status lorads_gnn_predict(lorads_gnn* g, int64_t n, const int64_t* c_rowptr,
                                            const int32_t* c_colind, const double* c_val, uint64_t feature_seed,
                                            int32_t ld, double* R_out) {
    if (!g) return LORADS_ERR_INVALID_ARG;
    lorads_status s = check_graph(g, n, c_rowptr, c_colind, c_val);
    if (s != LORADS_OK) return s;
    if (!R_out || ld < g->r_out) {
        g->err = "R_out must be a device n x ld FP64 array with ld >= r_out";
        return LORADS_ERR_INVALID_ARG;
    }
    if ((s = ensure_ws(g, n)) != LORADS_OK) return s;
    if (g->act == LORADS_BF16) forward<__nv_bfloat16>(g, n, c_rowptr, c_colind, c_val, feature_seed, R_out, ld);
    else forward<float>(g, n, c_rowptr, c_colind, c_val, feature_seed, R_out, ld);
    return check(g, "gnn forward");
}

extern "C" lorads_status lorads_gnn_edge_targets(int64_t n, const int64_t* c_rowptr, const int32_t* c_colind,
                                                 const double* R, int32_t r, int32_t ld, float* targets,
                                                 void* cuda_stream) {
    if (n < 1 || !c_rowptr || !c_colind || !R || !targets || r < 1 || ld < r) return LORADS_ERR_INVALID_ARG;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 4096);
    k_gnn_targets<<<grid, 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(n, c_rowptr, c_colind, R, r, ld,
                                                                               targets);
    return cudaGetLastError() == cudaSuccess ? LORADS_OK : LORADS_ERR_CUDA;
}

extern "C" lorads_status lorads_gnn_train_step(lorads_gnn* g, int64_t n, const int64_t* c_rowptr,
                                               const int32_t* c_colind, const double* c_val, uint64_t feature_seed,
                                               const float* targets, int64_t n_edges, float lr, double* loss_out,
                                               float* grad_out) {
    if (!g) return LORADS_ERR_INVALID_ARG;
    lorads_status s = check_graph(g, n, c_rowptr, c_colind, c_val);
    if (s != LORADS_OK) return s;
    if (!targets || n_edges < 1 || !(lr >= 0.0f)) {
        g->err = "targets must be given, n_edges >= 1 and lr >= 0";
        return LORADS_ERR_INVALID_ARG;
    }
    if ((s = ensure_ws(g, n)) != LORADS_OK) return s;
    const bool bf = g->act == LORADS_BF16;
    if (bf) forward<__nv_bfloat16>(g, n, c_rowptr, c_colind, c_val, feature_seed, nullptr, 0);
    else forward<float>(g, n, c_rowptr, c_colind, c_val, feature_seed, nullptr, 0);
    const int nbl = grid_for(g, n * 32, 256);
    k_gnn_loss<<<nbl, 256, 0, g->stream>>>(n, c_rowptr, c_colind, g->rhat, g->r_out, targets,
                                           (float)(2.0 / (double)n_edges), g->dr, g->lpart);
    if (bf) backward<__nv_bfloat16>(g, n, c_rowptr, c_colind, c_val);
    else backward<float>(g, n, c_rowptr, c_colind, c_val);
    if (grad_out) GCK(cudaMemcpyAsync(grad_out, g->grad, g->P * sizeof(float), cudaMemcpyDeviceToDevice, g->stream));
    if (lr > 0.0f) {
        g->step += 1;
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.0f - std::pow(b1, (float)g->step), c2 = 1.0f - std::pow(b2, (float)g->step);
        k_gnn_adam<<<grid_for(g, g->P, 256), 256, 0, g->stream>>>(g->P, g->theta, g->grad, g->m1, g->m2, lr, b1, b2,
                                                                  1e-8f, c1, c2);
    }
    if ((s = check(g, "gnn train step")) != LORADS_OK) return s;
    if (loss_out) {
        std::vector<double> lp(nbl);
        GCK(cudaMemcpyAsync(lp.data(), g->lpart, nbl * sizeof(double), cudaMemcpyDeviceToHost, g->stream));
        GCK(cudaStreamSynchronize(g->stream));
        double L = 0.0;
        for (double v : lp) L += v;
        *loss_out = L / (double)n_edges;
    }
    return LORADS_OK;
}
