// mlp_simt.cu -- FP32 CUDA-core form of the RPNN (Sec. 4.3, Fig. 6): forward, the
// chain-rule backward, the log-MSE loss (Sec. 5.2) and Adam.
//
// Every layer is one launch of a tiled SGEMM with a fused epilogue
//   C = act(sum_seg A_seg B_seg + bias + residual) [* (mask > 0)]
// where each operand is addressed through (row, col) strides, so the same kernel
// serves the forward layers, the data gradients (dY W) and the weight gradients
// (dY^T X).  The block's first layer is two segments: [z^k | o^{k-1}] [V^k | W1^k]^T.
#include <cmath>

#include "common.cuh"

namespace rpnn {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

struct Seg {
    const float* A;
    int64_t sam, sak;   // A(m, k) = A[m*sam + k*sak]
    const float* B;
    int64_t sbk, sbn;   // B(k, n) = B[k*sbk + n*sbn]
    int K;
};

struct Epi {
    const float* bias;  // [N] or null
    const float* res;   // residual [M][ldr] or null
    int64_t ldr;
    const float* mask;  // multiply by (mask > 0), [M][ldm] or null
    int64_t ldm;
    int relu;
    float* C;
    int64_t ldc;
};

__device__ __forceinline__ void load_tiles(const Seg& s, int m0, int n0, int k0, int M, int N,
                                           float (*As)[BM + 4], float (*Bs)[BN + 4]) {
    const int tid = threadIdx.x;
#pragma unroll
    for (int r = 0; r < (BM * BK) / NT; ++r) {
        const int e = tid + r * NT;
        int mm, kk;
        if (s.sak == 1) { mm = e / BK; kk = e % BK; } else { mm = e % BM; kk = e / BM; }
        const int m = m0 + mm, k = k0 + kk;
        As[kk][mm] = (m < M && k < s.K) ? __ldg(s.A + (int64_t)m * s.sam + (int64_t)k * s.sak) : 0.0f;
    }
#pragma unroll
    for (int r = 0; r < (BN * BK) / NT; ++r) {
        const int e = tid + r * NT;
        int kk, nn;
        if (s.sbn == 1) { kk = e / BN; nn = e % BN; } else { kk = e % BK; nn = e / BK; }
        const int n = n0 + nn, k = k0 + kk;
        Bs[kk][nn] = (n < N && k < s.K) ? __ldg(s.B + (int64_t)k * s.sbk + (int64_t)n * s.sbn) : 0.0f;
    }
}

__global__ void __launch_bounds__(NT)
k_gemm(int M_host, const int* __restrict__ M_dev, int N, Seg s0, Seg s1, int nseg, Epi e) {
    const int M = M_dev ? *M_dev : M_host;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    if (m0 >= M) return;
    __shared__ float As[BK][BM + 4];
    __shared__ float Bs[BK][BN + 4];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    float acc[4][4] = {};
    for (int si = 0; si < nseg; ++si) {
        const Seg& s = si == 0 ? s0 : s1;
        for (int k0 = 0; k0 < s.K; k0 += BK) {
            load_tiles(s, m0, n0, k0, M, N, As, Bs);
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                float a[4], b[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
                for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty + 16 * i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx + 16 * j;
            if (n >= N) continue;
            float v = acc[i][j];
            if (e.bias) v += e.bias[n];
            if (e.res) v += e.res[(int64_t)m * e.ldr + n];
            if (e.relu) v = fmaxf(v, 0.0f);
            if (e.mask && !(e.mask[(int64_t)m * e.ldm + n] > 0.0f)) v = 0.0f;
            e.C[(int64_t)m * e.ldc + n] = v;
        }
    }
}

// out[i] = x[i] * (m[i] > 0)
__global__ void k_mask(const float* __restrict__ x, const float* __restrict__ m, int n,
                       float* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = m[i] > 0.0f ? x[i] : 0.0f;
}

// column sums: out[n] = sum_m X[m][n] (bias gradients), fixed order per column
__global__ void k_colsum(const float* __restrict__ X, int M, int N, int64_t ld, float* __restrict__ out) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.0f;
    for (int m = 0; m < M; ++m) s += X[(int64_t)m * ld + n];
    out[n] = s;
}

Seg seg(const float* A, int64_t sam, int64_t sak, const float* B, int64_t sbk, int64_t sbn, int K) {
    Seg s;
    s.A = A; s.sam = sam; s.sak = sak; s.B = B; s.sbk = sbk; s.sbn = sbn; s.K = K;
    return s;
}

Epi epi(float* C, int64_t ldc, const float* bias = nullptr, int relu = 0,
        const float* res = nullptr, int64_t ldr = 0, const float* mask = nullptr, int64_t ldm = 0) {
    Epi e;
    e.C = C; e.ldc = ldc; e.bias = bias; e.relu = relu; e.res = res; e.ldr = ldr;
    e.mask = mask; e.ldm = ldm;
    return e;
}

rpnn_status gemm(int M, const int* M_dev, int N, const Seg& s0, const Seg* s1, const Epi& e,
                 cudaStream_t s) {
    if (M <= 0 || N <= 0) return RPNN_OK;
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM);
    if (grid.y > 65535u) { set_error("GEMM with %d rows exceeds the grid limit", M); return RPNN_ERR_ARG; }
    k_gemm<<<grid, NT, 0, s>>>(M, M_dev, N, s0, s1 ? *s1 : s0, s1 ? 2 : 1, e);
    RPNN_CHECK_LAUNCH();
    return RPNN_OK;
}

// Deterministic log-MSE loss (Sec. 5.2): one block; FP64 tree reduction.
__global__ void k_loss(const float* __restrict__ g, const float* __restrict__ t, int B,
                       double* loss, float* __restrict__ dg) {
    __shared__ double red[1024];
    double s = 0.0;
    for (int i = threadIdx.x; i < B; i += blockDim.x) {
        const double r = log1p((double)g[i]) - log1p((double)t[i]);
        s += r * r;
        dg[i] = (float)(2.0 * r / ((1.0 + (double)g[i]) * (double)B));
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = red[0] / (double)B;
}

__global__ void k_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ grad, int64_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = grad[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

}  // namespace

const ParamLayout& param_layout() {
    static ParamLayout L = [] {
        ParamLayout l{};
        int64_t o = 0;
        for (int k = 0; k < RPNN_K; ++k) {
            l.V[k] = o; o += (int64_t)RPNN_H * RPNN_DIN;
            if (k > 0) { l.W1[k] = o; o += (int64_t)RPNN_H * RPNN_H; } else l.W1[k] = -1;
            l.b1[k] = o; o += RPNN_H;
            l.W2[k] = o; o += (int64_t)RPNN_H * RPNN_H;
            l.b2[k] = o; o += RPNN_H;
        }
        for (int t = 0; t < 3; ++t) {
            const int out = t == 2 ? 1 : RPNN_H;
            l.T[t] = o; o += (int64_t)out * RPNN_H;
            l.bT[t] = o; o += out;
        }
        l.total = o;
        return l;
    }();
    return L;
}

// saved activations per row: o^1..o^10, F1^1..F1^10, o^11, o^12 (each 200), g
size_t mlp_saved_floats_per_row() { return 22 * (size_t)RPNN_H + 1; }

rpnn_status mlp_forward_f32(Ctx& c, const float* desc, int64_t q, const int* q_dev, float* out,
                            float* saved, cudaStream_t s) {
    const ParamLayout& L = param_layout();
    const float* P = c.params32.as<float>();
    const int M = (int)q;
    const int64_t H = RPNN_H, ZS = (int64_t)RPNN_K * RPNN_DESC_STRIDE;
    float *o_prev = nullptr, *o_cur, *f1;
    auto slot = [&](int i) { return saved + (size_t)i * q * H; };
    rpnn_status st;
    for (int k = 0; k < RPNN_K; ++k) {
        if (saved) { o_cur = slot(k); f1 = slot(10 + k); }
        else { o_cur = c.act0.as<float>(); f1 = c.act1.as<float>(); }
        // F1 = relu([z^k | o^{k-1}] [V^k | W1^k]^T + b1)
        Seg z = seg(desc + k * RPNN_DESC_STRIDE, ZS, 1, P + L.V[k], 1, RPNN_DIN, RPNN_DIN);
        if (k > 0) {
            Seg o = seg(o_prev, H, 1, P + L.W1[k], 1, H, RPNN_H);
            st = gemm(M, q_dev, RPNN_H, z, &o, epi(f1, H, P + L.b1[k], 1), s);
        } else {
            st = gemm(M, q_dev, RPNN_H, z, nullptr, epi(f1, H, P + L.b1[k], 1), s);
        }
        if (st) return st;
        // o^k = relu(W2 F1 + b2 + o^{k-1})  (in place when not saving)
        Seg w2 = seg(f1, H, 1, P + L.W2[k], 1, H, RPNN_H);
        st = gemm(M, q_dev, RPNN_H, w2, nullptr, epi(o_cur, H, P + L.b2[k], 1, k > 0 ? o_prev : nullptr, H), s);
        if (st) return st;
        o_prev = o_cur;
    }
    // standard layers
    float* t0 = saved ? slot(20) : c.act1.as<float>();
    float* t1 = saved ? slot(21) : c.act2.as<float>();
    st = gemm(M, q_dev, RPNN_H, seg(o_prev, H, 1, P + L.T[0], 1, H, RPNN_H), nullptr,
              epi(t0, H, P + L.bT[0], 1), s);
    if (st) return st;
    st = gemm(M, q_dev, RPNN_H, seg(t0, H, 1, P + L.T[1], 1, H, RPNN_H), nullptr,
              epi(t1, H, P + L.bT[1], 1), s);
    if (st) return st;
    st = gemm(M, q_dev, 1, seg(t1, H, 1, P + L.T[2], 1, H, RPNN_H), nullptr, epi(out, 1, P + L.bT[2], 1), s);
    if (st) return st;
    if (saved) RPNN_CUDA_TRY(cudaMemcpyAsync(saved + (size_t)22 * q * H, out, q * sizeof(float),
                                             cudaMemcpyDeviceToDevice, s));
    return RPNN_OK;
}

rpnn_status mlp_forward_f32_with(const float* P, const float* desc, int64_t q, float* out, float* s0,
                                 float* s1, float* s2, cudaStream_t s) {
    const ParamLayout& L = param_layout();
    const int M = (int)q;
    const int64_t H = RPNN_H, ZS = (int64_t)RPNN_K * RPNN_DESC_STRIDE;
    float* o = s0;
    float* f1 = s1;
    rpnn_status st;
    for (int k = 0; k < RPNN_K; ++k) {
        Seg z = seg(desc + k * RPNN_DESC_STRIDE, ZS, 1, P + L.V[k], 1, RPNN_DIN, RPNN_DIN);
        if (k > 0) {
            Seg oo = seg(o, H, 1, P + L.W1[k], 1, H, RPNN_H);
            st = gemm(M, nullptr, RPNN_H, z, &oo, epi(f1, H, P + L.b1[k], 1), s);
        } else {
            st = gemm(M, nullptr, RPNN_H, z, nullptr, epi(f1, H, P + L.b1[k], 1), s);
        }
        if (st) return st;
        Seg w2 = seg(f1, H, 1, P + L.W2[k], 1, H, RPNN_H);
        st = gemm(M, nullptr, RPNN_H, w2, nullptr, epi(o, H, P + L.b2[k], 1, k > 0 ? o : nullptr, H), s);
        if (st) return st;
    }
    st = gemm(M, nullptr, RPNN_H, seg(o, H, 1, P + L.T[0], 1, H, RPNN_H), nullptr, epi(s1, H, P + L.bT[0], 1), s);
    if (st) return st;
    st = gemm(M, nullptr, RPNN_H, seg(s1, H, 1, P + L.T[1], 1, H, RPNN_H), nullptr, epi(s2, H, P + L.bT[1], 1), s);
    if (st) return st;
    return gemm(M, nullptr, 1, seg(s2, H, 1, P + L.T[2], 1, H, RPNN_H), nullptr, epi(out, 1, P + L.bT[2], 1), s);
}

rpnn_status mlp_backward_f32(Ctx& c, const float* desc, int64_t q, const float* saved,
                             const float* dout, float* dP, cudaStream_t s) {
    const ParamLayout& L = param_layout();
    const float* P = c.params32.as<float>();
    const int M = (int)q;
    const int64_t H = RPNN_H, ZS = (int64_t)RPNN_K * RPNN_DESC_STRIDE;
    auto slot = [&](int i) { return saved + (size_t)i * q * H; };
    const float* g = saved + (size_t)22 * q * H;
    rpnn_status st = c.act0.reserve((size_t)q * H * sizeof(float));
    if (!st) st = c.act1.reserve((size_t)q * H * sizeof(float));
    if (!st) st = c.act2.reserve((size_t)q * H * sizeof(float));
    if (!st) st = c.t_dg.reserve((size_t)q * sizeof(float));
    if (st) return st;
    float* bufA = c.act0.as<float>();
    float* bufB = c.act1.as<float>();
    float* da = c.act2.as<float>();
    float* da3 = c.t_dg.as<float>();
    const dim3 cs_grid((RPNN_H + 255) / 256);
    // last layer: g = relu(T3 o12 + bT3): da3 = dout * (g > 0)
    k_mask<<<(M + 255) / 256, 256, 0, s>>>(dout, g, M, da3);
    RPNN_CHECK_LAUNCH();
    // dT3[0][j] = sum_m da3[m] o12[m][j]; dbT3 = sum_m da3
    st = gemm(1, nullptr, RPNN_H, seg(da3, 0, 1, slot(21), H, 1, M), nullptr, epi(dP + L.T[2], H), s);
    if (st) return st;
    k_colsum<<<1, 32, 0, s>>>(da3, M, 1, 1, dP + L.bT[2]);
    RPNN_CHECK_LAUNCH();
    // da2 = (da3 T3) * (o12 > 0)
    st = gemm(M, nullptr, RPNN_H, seg(da3, 1, 1, P + L.T[2], H, 1, 1), nullptr,
              epi(bufA, H, nullptr, 0, nullptr, 0, slot(21), H), s);
    if (st) return st;
    // standard layer 2: input o11 (slot 20); layer 1: input o10 (slot 9)
    const float* tin[2] = {slot(9), slot(20)};
    for (int t = 1; t >= 0; --t) {
        // dT = da^T x_in; db = colsum(da)
        st = gemm(RPNN_H, nullptr, RPNN_H, seg(bufA, 1, H, tin[t], H, 1, M), nullptr, epi(dP + L.T[t], H), s);
        if (st) return st;
        k_colsum<<<cs_grid, 256, 0, s>>>(bufA, M, RPNN_H, H, dP + L.bT[t]);
        RPNN_CHECK_LAUNCH();
        // d x_in = da T, masked by (x_in > 0) (x_in is a ReLU output)
        st = gemm(M, nullptr, RPNN_H, seg(bufA, H, 1, P + L.T[t], H, 1, RPNN_H), nullptr,
                  epi(bufB, H, nullptr, 0, nullptr, 0, tin[t], H), s);
        if (st) return st;
        float* tmp = bufA; bufA = bufB; bufB = tmp;
    }
    // bufA = dpre_10 = dl/d(pre-activation of o^10)
    for (int k = RPNN_K - 1; k >= 0; --k) {
        const float* f1 = slot(10 + k);
        // dW2 = dpre^T F1; db2 = colsum(dpre)
        st = gemm(RPNN_H, nullptr, RPNN_H, seg(bufA, 1, H, f1, H, 1, M), nullptr, epi(dP + L.W2[k], H), s);
        if (st) return st;
        k_colsum<<<cs_grid, 256, 0, s>>>(bufA, M, RPNN_H, H, dP + L.b2[k]);
        RPNN_CHECK_LAUNCH();
        // da1 = (dpre W2) * (F1 > 0)
        st = gemm(M, nullptr, RPNN_H, seg(bufA, H, 1, P + L.W2[k], H, 1, RPNN_H), nullptr,
                  epi(da, H, nullptr, 0, nullptr, 0, f1, H), s);
        if (st) return st;
        // dV = da1^T z^k; db1 = colsum(da1)
        st = gemm(RPNN_H, nullptr, RPNN_DIN, seg(da, 1, H, desc + k * RPNN_DESC_STRIDE, ZS, 1, M), nullptr,
                  epi(dP + L.V[k], RPNN_DIN), s);
        if (st) return st;
        k_colsum<<<cs_grid, 256, 0, s>>>(da, M, RPNN_H, H, dP + L.b1[k]);
        RPNN_CHECK_LAUNCH();
        if (k > 0) {
            const float* oprev = slot(k - 1);
            st = gemm(RPNN_H, nullptr, RPNN_H, seg(da, 1, H, oprev, H, 1, M), nullptr, epi(dP + L.W1[k], H), s);
            if (st) return st;
            // dpre_{k-1} = (dpre_k + da1 W1) * (o^{k-1} > 0)
            st = gemm(M, nullptr, RPNN_H, seg(da, H, 1, P + L.W1[k], H, 1, RPNN_H), nullptr,
                      epi(bufB, H, nullptr, 0, bufA, H, oprev, H), s);
            if (st) return st;
            float* tmp = bufA; bufA = bufB; bufB = tmp;
        }
    }
    return RPNN_OK;
}

rpnn_status launch_loss(const float* g, const float* target, int batch, double* loss, float* dg,
                        cudaStream_t s) {
    k_loss<<<1, 1024, 0, s>>>(g, target, batch, loss, dg);
    RPNN_CHECK_LAUNCH();
    return RPNN_OK;
}

rpnn_status launch_adam(float* p, float* m, float* v, const float* grad, int64_t n, int64_t step,
                        const rpnn_adam_cfg& cfg, cudaStream_t s) {
    const double c1 = 1.0 - std::pow((double)cfg.beta1, (double)step);
    const double c2 = 1.0 - std::pow((double)cfg.beta2, (double)step);
    k_adam<<<1024, 256, 0, s>>>(p, m, v, grad, n, cfg.lr, cfg.beta1, cfg.beta2, cfg.eps, (float)c1,
                                (float)c2);
    RPNN_CHECK_LAUNCH();
    return RPNN_OK;
}

}  // namespace rpnn
