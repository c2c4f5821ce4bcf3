// train_bf16.cu -- mixed-precision training form of the network (Sec. 4.3 forward, Sec. 5.2
// chain rule): the forward runs in the persistent tensor-core network kernel in its training
// form (mlp_tc.cu); every data gradient and weight gradient is a BF16 tensor-core GEMM
// (gemm_tc.cu) with FP32 accumulation; biases, residual sums, ReLU masks, saved activations,
// the loss, the gradients and the Adam step stay FP32 (FP32 master weights).  The 1-wide
// output layer's gradients, which have a K or N of 1, run on the FP32 CUDA-core GEMM.
//
// Each 200-wide activation is stored twice by the forward: FP32 [q][200] (residual input,
// ReLU mask) and BF16 transposed [200][ldq] (operand of the weight gradients, which sum over
// the q rows); ldq = q rounded up to 8 elements.  (The BF16 [q][200] slots ahead of the
// transposed ones in the saved buffer are no longer written.)
#include <cuda_bf16.h>

#include "common.cuh"

namespace rpnn {

namespace {

constexpr int H = RPNN_H;
constexpr int VLD = 232;                  // row pitch of V^k in BF16 (226 rounded up to 8)
constexpr int kMaxMats = 64;

// BF16 weight image: V^k [200][232] (K-major for the forward), W1^k and W2^k [200][200]
// and their transposes (K-major for the data gradients), T1, T2 and their transposes.
struct TrainImage {
    int64_t V[RPNN_K], W1[RPNN_K], W2[RPNN_K], W1T[RPNN_K], W2T[RPNN_K], T[2], TT[2];
    int64_t total;
};

const TrainImage& train_image() {
    static TrainImage I = [] {
        TrainImage t{};
        int64_t o = 0;
        for (int k = 0; k < RPNN_K; ++k) {
            t.V[k] = o; o += (int64_t)H * VLD;
            t.W2[k] = o; o += (int64_t)H * H;
            t.W2T[k] = o; o += (int64_t)H * H;
            if (k > 0) {
                t.W1[k] = o; o += (int64_t)H * H;
                t.W1T[k] = o; o += (int64_t)H * H;
            } else {
                t.W1[k] = t.W1T[k] = -1;
            }
        }
        for (int i = 0; i < 2; ++i) {
            t.T[i] = o; o += (int64_t)H * H;
            t.TT[i] = o; o += (int64_t)H * H;
        }
        t.total = o;
        return t;
    }();
    return I;
}

struct MatJob {
    int64_t src, dst;                     // offsets (floats / BF16 elements)
    int rows, cols, ld, transpose;        // source [rows][cols]; destination pitch ld
};
struct MatJobs {
    MatJob j[kMaxMats];
    int n;
};

// blockIdx.y = matrix; destination element (r, c) of a [rows][ld] (or transposed
// [cols][ld]) matrix, padding columns written as zero
__global__ void k_train_image(const float* __restrict__ P, const MatJobs jobs, __nv_bfloat16* __restrict__ img) {
    const MatJob& J = jobs.j[blockIdx.y];
    const int drows = J.transpose ? J.cols : J.rows;
    const int dcols = J.transpose ? J.rows : J.cols;
    const int64_t total = (int64_t)drows * J.ld;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / J.ld), c = (int)(i % J.ld);
        float v = 0.0f;
        if (c < dcols) v = J.transpose ? P[J.src + (int64_t)c * J.cols + r] : P[J.src + (int64_t)r * J.cols + c];
        img[J.dst + i] = __float2bfloat16_rn(v);
    }
}

__device__ __forceinline__ __nv_bfloat16 to_bf16(float v) { return __float2bfloat16_rn(v); }
__device__ __forceinline__ __nv_bfloat16 to_bf16(__nv_bfloat16 v) { return v; }

// z [q][10][240] FP32 or BF16 -> zb [q][10][240] BF16 and zt [10][226][ldq] BF16 (per level,
// transposed); FP32 values are rounded to nearest even, BF16 values copied
// Training descriptors -> BF16 rows zb [q][10][240] (FP32 input only: BF16 input is used in
// place) and the transposed copy zt [10 * 226][ldq] the V^k weight gradients read, through
// 32 x 32 shared-memory tiles (rows m read along the columns, written along m).
template <class T>
__global__ void k_train_desc(const T* __restrict__ z, int64_t q, int64_t ldq, __nv_bfloat16* __restrict__ zb,
                             __nv_bfloat16* __restrict__ zt) {
    const int64_t row = (int64_t)RPNN_K * RPNN_DESC_STRIDE;
    if (zb) {
        const int64_t total = q * row;
        const int64_t stride = (int64_t)gridDim.x * gridDim.y * blockDim.x * blockDim.y;
        const int64_t t0 = ((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * (blockDim.x * blockDim.y) +
                           threadIdx.y * blockDim.x + threadIdx.x;
        for (int64_t i = t0; i < total; i += stride) zb[i] = to_bf16(z[i]);
    }
    __shared__ __nv_bfloat16 tile[32][33];
    const int ncol = RPNN_K * RPNN_DIN;                      // 2260 transposed rows
    const int lc0 = blockIdx.y * 32;
    const int64_t m0 = (int64_t)blockIdx.x * 32;
    for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
        const int64_t m = m0 + yy;
        const int lc = lc0 + threadIdx.x;
        if (m < q && lc < ncol) {
            const int k = lc / RPNN_DIN, c = lc - k * RPNN_DIN;
            tile[yy][threadIdx.x] = to_bf16(z[m * row + (int64_t)k * RPNN_DESC_STRIDE + c]);
        }
    }
    __syncthreads();
    for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
        const int lc = lc0 + yy;
        const int64_t m = m0 + threadIdx.x;
        if (m < q && lc < ncol) zt[(int64_t)lc * ldq + m] = tile[threadIdx.x][yy];
    }
}

__global__ void k_bf16_to_f32(const __nv_bfloat16* __restrict__ in, float* __restrict__ out, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = __bfloat162float(in[i]);
}

// x [q][200] FP32 -> BF16 [q][200] and transposed BF16 [200][ldq], through 32 x 32
// shared-memory tiles
__global__ void k_train_act(const float* __restrict__ x, int64_t q, int64_t ldq, __nv_bfloat16* __restrict__ xb,
                            __nv_bfloat16* __restrict__ xt) {
    __shared__ __nv_bfloat16 tile[32][33];
    const int n0 = blockIdx.y * 32;
    const int64_t m0 = (int64_t)blockIdx.x * 32;
    for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
        const int64_t m = m0 + yy;
        const int n = n0 + threadIdx.x;
        if (m < q && n < H) {
            const __nv_bfloat16 b = __float2bfloat16_rn(x[m * H + n]);
            xb[m * H + n] = b;
            tile[yy][threadIdx.x] = b;
        }
    }
    __syncthreads();
    for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
        const int n = n0 + yy;
        const int64_t m = m0 + threadIdx.x;
        if (m < q && n < H) xt[(int64_t)n * ldq + m] = tile[threadIdx.x][yy];
    }
}

int grid_for(int64_t n, int sms) {
    int64_t b = (n + 255) / 256;
    if (b > (int64_t)sms * 8) b = (int64_t)sms * 8;
    return (int)std::max<int64_t>(b, 1);
}

}  // namespace

int64_t train_ldq(int64_t q) { return (q + 7) & ~(int64_t)7; }

rpnn_status launch_bf16_to_f32(const void* in, float* out, int64_t n, int sms, cudaStream_t s) {
    if (n <= 0) return RPNN_OK;
    k_bf16_to_f32<<<grid_for(n, sms), 256, 0, s>>>(static_cast<const __nv_bfloat16*>(in), out, n);
    RPNN_CHECK_LAUNCH();
    return RPNN_OK;
}

size_t train_bf16_saved32_floats(int64_t q) { return (size_t)22 * H * train_ldq(q) + (size_t)q; }

size_t train_bf16_saved_elems(int64_t q) {
    // 22 activations as BF16 [q][200] and BF16 [200][ldq]; descriptors as BF16 [q][2400]
    // and [10][226][ldq]
    return (size_t)22 * q * H + (size_t)22 * H * train_ldq(q) + (size_t)q * RPNN_K * RPNN_DESC_STRIDE +
           (size_t)RPNN_K * RPNN_DIN * train_ldq(q);
}

rpnn_status train_build_image(Ctx& c, cudaStream_t s) {
    const TrainImage& I = train_image();
    const ParamLayout& L = param_layout();
    rpnn_status st = c.t_w16.reserve((size_t)I.total * 2);
    if (st) return st;
    MatJobs jobs{};
    auto add = [&](int64_t src, int64_t dst, int rows, int cols, int ld, int tr) {
        jobs.j[jobs.n++] = MatJob{src, dst, rows, cols, ld, tr};
    };
    for (int k = 0; k < RPNN_K; ++k) {
        add(L.V[k], I.V[k], H, RPNN_DIN, VLD, 0);
        add(L.W2[k], I.W2[k], H, H, H, 0);
        add(L.W2[k], I.W2T[k], H, H, H, 1);
        if (k > 0) {
            add(L.W1[k], I.W1[k], H, H, H, 0);
            add(L.W1[k], I.W1T[k], H, H, H, 1);
        }
    }
    for (int i = 0; i < 2; ++i) {
        add(L.T[i], I.T[i], H, H, H, 0);
        add(L.T[i], I.TT[i], H, H, H, 1);
    }
    k_train_image<<<dim3(32, jobs.n), 256, 0, s>>>(c.params32.as<float>(), jobs, c.t_w16.as<__nv_bfloat16>());
    RPNN_CHECK_LAUNCH();
    return RPNN_OK;
}

// Forward with saved activations: FP32 slots in the FP32 form's order (o^1..o^10,
// F1^1..F1^10, o^11, o^12), each transposed [200][ldq] so that a warp's 32 rows are 128
// contiguous bytes per column, then g [q] (train_bf16_saved32_floats(q) floats in `saved`);
// BF16 copies in `s16` (train_bf16_saved_elems(q)).
rpnn_status mlp_forward_bf16_train(Ctx& c, const void* desc, int desc_dtype, int64_t q, float* out, float* saved,
                                   uint16_t* s16, cudaStream_t s) {
    const int64_t ldq = train_ldq(q);
    // the transposed weight image the backward reads
    rpnn_status st = train_build_image(c, s);
    if (st) return st;
    uint16_t* zb = s16 + (size_t)22 * q * H + (size_t)22 * H * ldq;
    uint16_t* zt = zb + (size_t)q * RPNN_K * RPNN_DESC_STRIDE;
    const dim3 tgrid((unsigned)((q + 31) / 32), (RPNN_K * RPNN_DIN + 31) / 32);
    // BF16 records are the forward's operand as they are; FP32 ones are rounded into zb
    const void* zfwd = desc;
    if (desc_dtype == RPNN_BF16) {
        k_train_desc<<<tgrid, dim3(32, 8), 0, s>>>(static_cast<const __nv_bfloat16*>(desc), q, ldq, nullptr,
                                                  reinterpret_cast<__nv_bfloat16*>(zt));
    } else {
        k_train_desc<<<tgrid, dim3(32, 8), 0, s>>>(static_cast<const float*>(desc), q, ldq,
                                                  reinterpret_cast<__nv_bfloat16*>(zb),
                                                  reinterpret_cast<__nv_bfloat16*>(zt));
        zfwd = zb;
    }
    RPNN_CHECK_LAUNCH();
    // the 22 layers in the persistent tensor-core network kernel (one 128-row tile per CTA,
    // layer after layer in shared and tensor memory), in its training form: FP32 biases in
    // the epilogue, every ReLU output stored FP32 and BF16 transposed for the backward
    st = mlp_forward_bf16_saving(c, zfwd, q, out, saved, s16 + (size_t)22 * q * H, ldq, s);
    if (st) return st;
    RPNN_CUDA_TRY(cudaMemcpyAsync(saved + (size_t)22 * H * ldq, out, q * sizeof(float), cudaMemcpyDeviceToDevice, s));
    return RPNN_OK;
}

rpnn_status mlp_backward_bf16_train(Ctx& c, int64_t q, const float* saved, const uint16_t* s16, const float* dout,
                                    float* dP, cudaStream_t s, const cudaStream_t* side) {
    const ParamLayout& L = param_layout();
    const TrainImage& I = train_image();
    const int M = (int)q;
    const int64_t ldq = train_ldq(q);
    const uint16_t* W = c.t_w16.as<uint16_t>();
    auto slot = [&](int i) { return saved + (size_t)i * H * ldq; };       // transposed [200][ldq]
    auto slott = [&](int i) { return s16 + (size_t)22 * q * H + (size_t)i * H * ldq; };
    const uint16_t* zt = s16 + (size_t)22 * q * H + (size_t)22 * H * ldq + (size_t)q * RPNN_K * RPNN_DESC_STRIDE;
    // one gradient buffer per layer, each FP32 [q][200] + BF16 [q][200] + BF16 transposed
    // [200][ldq]: nothing is overwritten within a step, so the weight-gradient GEMMs and
    // bias sums may run on the two `side` streams (those of W2 and T on side[0], of V and W1
    // on side[1], each with its own split-K workspace) while the data-gradient chain
    // continues on `s`
    constexpr int NG = 22;
    const size_t per16 = (size_t)q * H + (size_t)H * ldq;
    rpnn_status st = c.t_gb32.reserve((size_t)NG * q * H * sizeof(float));
    if (!st) st = c.t_gb16.reserve((size_t)NG * per16 * 2);
    if (st) return st;
    static_assert(NG + 3 <= kTrainEvents, "gradient-ready events");
    if (side && (int)c.t_events.size() < kTrainEvents) { set_error("weight-gradient stream events missing"); return RPNN_ERR_STATE; }
    struct Buf { float* f; uint16_t* b; uint16_t* t; int id; };
    auto buf = [&](int i) {
        uint16_t* b16 = c.t_gb16.as<uint16_t>() + (size_t)i * per16;
        return Buf{c.t_gb32.as<float>() + (size_t)i * q * H, b16, b16 + (size_t)q * H, i};
    };
    auto out_to = [&](const Buf& b) {
        TgOut o;
        o.C = b.f; o.ldc = H;
        o.Cb = b.b; o.ldb = H;
        o.Ct = b.t; o.ldt = ldq;
        return o;
    };
    // the weight-gradient streams (both s when there are none)
    const cudaStream_t ws[2] = {side ? side[0] : s, side ? side[1] : s};
    DevBuf* wsb[2] = {nullptr, side ? &c.t_ws2 : nullptr};
    // gradient buffer b is complete on s: let weight-gradient stream w use it
    auto ready = [&](const Buf& b, int w) -> rpnn_status {
        if (!side) return RPNN_OK;
        RPNN_CUDA_TRY(cudaEventRecord(c.t_events[b.id], s));
        RPNN_CUDA_TRY(cudaStreamWaitEvent(ws[w], c.t_events[b.id], 0));
        return RPNN_OK;
    };
    auto wgrad = [&](int w, const uint16_t* at, const uint16_t* bt, int N, float* dst) {
        // dW[j][i] = sum_m a[m][j] x[m][i]: A = a^T [200][ldq], B = x^T [N][ldq], K = q
        const TgSeg sg{at, ldq, bt, ldq, M};
        TgOut o;
        o.C = dst; o.ldc = N;
        return tc_gemm(c, H, N, sg, nullptr, o, ws[w], wsb[w]);
    };
    if (side) {
        // the weight-gradient streams start after everything issued on s so far
        RPNN_CUDA_TRY(cudaEventRecord(c.t_events[NG], s));
        RPNN_CUDA_TRY(cudaStreamWaitEvent(ws[0], c.t_events[NG], 0));
        RPNN_CUDA_TRY(cudaStreamWaitEvent(ws[1], c.t_events[NG], 0));
    }
    int next = 0;
    Buf A = buf(next++);
    // output layer (CUDA cores): A.f = dl/d(pre-activation of o^12 ... ) masked, dT3, dbT3
    st = mlp_output_layer_backward_f32(c, slot(21), saved + (size_t)22 * H * ldq, dout, q, dP, A.f, s, ldq);
    if (st) return st;
    k_train_act<<<dim3((unsigned)((q + 31) / 32), (H + 31) / 32), dim3(32, 8), 0, s>>>(
        A.f, q, ldq, reinterpret_cast<__nv_bfloat16*>(A.b), reinterpret_cast<__nv_bfloat16*>(A.t));
    RPNN_CHECK_LAUNCH();
    if ((st = ready(A, 0))) return st;
    // standard layers 2 (input o^11, slot 20) and 1 (input o^10, slot 9)
    for (int t = 1; t >= 0; --t) {
        const int in = t == 1 ? 20 : 9;
        Buf B = buf(next++);
        TgOut o = out_to(B);
        o.mask = slot(in); o.ldm = ldq; o.mask_t = 1;
        const TgSeg sd{A.b, H, W + I.TT[t], H, H};
        st = tc_gemm(c, M, H, sd, nullptr, o, s);
        if (!st) st = ready(B, 0);
        if (!st) st = wgrad(0, A.t, slott(in), H, dP + L.T[t]);
        if (!st) st = colsum_f32(c, A.f, M, H, dP + L.bT[t], ws[0]);
        if (st) return st;
        A = B;
    }
    // blocks k = 10 .. 1; A = dl/d(pre-activation of o^k)
    for (int k = RPNN_K - 1; k >= 0; --k) {
        // da1 = (dpre W2) * (F1 > 0)
        Buf D = buf(next++);
        TgOut o = out_to(D);
        o.mask = slot(10 + k); o.ldm = ldq; o.mask_t = 1;
        const TgSeg sd{A.b, H, W + I.W2T[k], H, H};
        st = tc_gemm(c, M, H, sd, nullptr, o, s);
        if (!st) st = ready(D, 1);
        if (st) return st;
        Buf B{};
        if (k > 0) {
            // dpre_{k-1} = (dpre_k + da1 W1) * (o^{k-1} > 0)
            B = buf(next++);
            TgOut o2 = out_to(B);
            o2.res = A.f; o2.ldr = H;
            o2.mask = slot(k - 1); o2.ldm = ldq; o2.mask_t = 1;
            const TgSeg s1{D.b, H, W + I.W1T[k], H, H};
            st = tc_gemm(c, M, H, s1, nullptr, o2, s);
            if (!st) st = ready(B, 0);
            if (st) return st;
        }
        st = wgrad(0, A.t, slott(10 + k), H, dP + L.W2[k]);
        if (!st) st = colsum_f32(c, A.f, M, H, dP + L.b2[k], ws[0]);
        if (!st) st = wgrad(1, D.t, zt + (size_t)k * RPNN_DIN * ldq, RPNN_DIN, dP + L.V[k]);
        if (!st) st = colsum_f32(c, D.f, M, H, dP + L.b1[k], ws[1]);
        if (!st && k > 0) st = wgrad(1, D.t, slott(k - 1), H, dP + L.W1[k]);
        if (st) return st;
        if (k > 0) A = B;
    }
    if (side) {
        // s continues only after every weight gradient is written
        for (int w = 0; w < 2; ++w) {
            RPNN_CUDA_TRY(cudaEventRecord(c.t_events[NG + 1 + w], ws[w]));
            RPNN_CUDA_TRY(cudaStreamWaitEvent(s, c.t_events[NG + 1 + w], 0));
        }
    }
    return RPNN_OK;
}

}  // namespace rpnn
