// descriptor.cu -- hierarchical stencil descriptor (Sec. 4.2, Fig. 5).
//
// Per shading point: light-aligned frame (z = light, x = normalize(z cross omega),
// y = z cross x, omega = -d), gamma = acos(omega . light), and for each of the 10
// levels the density rho at the 225 points of the 5x5x9 stencil spanning
// [-1,1]x[-1,1]x[-1,3] mean free paths scaled by 2^(k-1), trilinearly interpolated in
// the mip level chosen for that level.  FP32 with explicit _rn intrinsics so the
// rounding sequence is fixed (no contraction):
//   s = inv_h0 * 2^-m, g = (inv_mean * 2^(k-1)) * s, A = g ex, B = g ey, C = g ez,
//   U0 = x s - 0.5, u = fma(oz, C, fma(oy, B, fma(ox, A, U0))),
//   lerp(a, b, f) = fma(f, b - a, a) in x, then y, then z.
// Layout: one block of 256 threads per shading point (grid-stride over points);
// thread t < 225 owns stencil point t for all 10 levels, threads 225..239 write gamma
// and the zero padding.  Each lookup reads one 32-byte corner record (two float4).
#include <cuda_bf16.h>

#include "common.cuh"

namespace rpnn {

namespace {

template <class T> __device__ __forceinline__ T cvt_out(float v);
template <> __device__ __forceinline__ float cvt_out<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 cvt_out<__nv_bfloat16>(float v) {
    return __float2bfloat16_rn(v);
}

__device__ __forceinline__ float lerp_rn(float a, float b, float f) {
    return __fmaf_rn(f, __fsub_rn(b, a), a);
}

struct Frame {
    float ex[3], ey[3], ez[3];
    float gamma;
};

__device__ __forceinline__ Frame make_frame(const float d[3], const float wl[3]) {
    Frame F;
    const float w[3] = {-d[0], -d[1], -d[2]};
    const float* ez = wl;
    float cr[3];
    cr[0] = __fsub_rn(__fmul_rn(ez[1], w[2]), __fmul_rn(ez[2], w[1]));
    cr[1] = __fsub_rn(__fmul_rn(ez[2], w[0]), __fmul_rn(ez[0], w[2]));
    cr[2] = __fsub_rn(__fmul_rn(ez[0], w[1]), __fmul_rn(ez[1], w[0]));
    const float len2 = __fadd_rn(__fadd_rn(__fmul_rn(cr[0], cr[0]), __fmul_rn(cr[1], cr[1])),
                                 __fmul_rn(cr[2], cr[2]));
    if (len2 < 1e-12f) {
        // Duff et al. 2017 basis of z, in FP64 from the FP32 inputs, rounded
        const double n0 = ez[0], n1 = ez[1], n2 = ez[2];
        const double sg = signbit(ez[2]) ? -1.0 : 1.0;   // copysign(1, z)
        const double a = __ddiv_rn(-1.0, __dadd_rn(sg, n2));
        F.ex[0] = __double2float_rn(__dadd_rn(1.0, __dmul_rn(__dmul_rn(__dmul_rn(sg, n0), n0), a)));
        F.ex[1] = __double2float_rn(__dmul_rn(sg, __dmul_rn(__dmul_rn(n0, n1), a)));
        F.ex[2] = __double2float_rn(__dmul_rn(-sg, n0));
    } else {
        const float len = __fsqrt_rn(len2);
        for (int a = 0; a < 3; ++a) F.ex[a] = __fdiv_rn(cr[a], len);
    }
    for (int a = 0; a < 3; ++a) F.ez[a] = ez[a];
    F.ey[0] = __fsub_rn(__fmul_rn(ez[1], F.ex[2]), __fmul_rn(ez[2], F.ex[1]));
    F.ey[1] = __fsub_rn(__fmul_rn(ez[2], F.ex[0]), __fmul_rn(ez[0], F.ex[2]));
    F.ey[2] = __fsub_rn(__fmul_rn(ez[0], F.ex[1]), __fmul_rn(ez[1], F.ex[0]));
    float cg = __fadd_rn(__fadd_rn(__fmul_rn(w[0], wl[0]), __fmul_rn(w[1], wl[1])), __fmul_rn(w[2], wl[2]));
    cg = fminf(fmaxf(cg, -1.0f), 1.0f);
    F.gamma = acosf(cg);
    return F;
}

__device__ __forceinline__ float lookup(const VolumeView& v, int m, const float u[3]) {
    const LevelDesc L = v.lvl[m];
    int i[3];
    float f[3];
    const int dims[3] = {L.ax, L.ay, L.az};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float uu = fminf(fmaxf(u[a], -1.0e6f), 1.0e6f);
        const float fl = floorf(uu);
        f[a] = __fsub_rn(uu, fl);
        i[a] = (int)fl;
    }
    if (i[0] < -1 || i[0] > dims[0] - 1 || i[1] < -1 || i[1] > dims[1] - 1 || i[2] < -1 ||
        i[2] > dims[2] - 1)
        return 0.0f;
    const int64_t r = L.rec_offset +
                      ((int64_t)(i[2] + 1) * (L.ay + 1) + (i[1] + 1)) * (L.ax + 1) + (i[0] + 1);
    const float4 lo = __ldg(v.packed + 2 * r);
    const float4 hi = __ldg(v.packed + 2 * r + 1);
    const float c00 = lerp_rn(lo.x, lo.y, f[0]);
    const float c10 = lerp_rn(lo.z, lo.w, f[0]);
    const float c01 = lerp_rn(hi.x, hi.y, f[0]);
    const float c11 = lerp_rn(hi.z, hi.w, f[0]);
    const float c0 = lerp_rn(c00, c10, f[1]);
    const float c1 = lerp_rn(c01, c11, f[1]);
    return lerp_rn(c0, c1, f[2]);
}

// Thread t < 250 of the block owns stencil column (ix, iy) = (t%25 % 5, t%25 / 5) of
// level k = t / 25 and walks its 9 points along z, so the level set-up and the
// (ox, oy) part of each coordinate are computed once per column; threads 250..255
// write gamma and the zero padding.
template <class OutT>
__global__ void __launch_bounds__(256)
k_descriptor(const VolumeView v, const float* __restrict__ xs, const float* __restrict__ ds,
             const float* __restrict__ wls, int wl_stride, int64_t q_host,
             const int* __restrict__ q_dev, OutT* __restrict__ out) {
    const int64_t q = q_dev ? (int64_t)*q_dev : q_host;
    const int t = threadIdx.x;
    const int k = t / 25, col = t % 25;
    const int ix = col % 5, iy = col / 5;
    const float ox = __fadd_rn(-1.0f, __fmul_rn(0.5f, (float)ix));
    const float oy = __fadd_rn(-1.0f, __fmul_rn(0.5f, (float)iy));
    const int m = k < RPNN_K ? v.mip_of_level[k] : 0;
    const float s = __fmul_rn(v.inv_h0, __int_as_float((127 - m) << 23));   // * 2^-m
    const float gk = __fmul_rn(__fmul_rn(v.inv_mean_f, (float)(1 << (k < RPNN_K ? k : 0))), s);
    for (int64_t qi = blockIdx.x; qi < q; qi += gridDim.x) {
        const float x[3] = {__ldg(xs + 3 * qi), __ldg(xs + 3 * qi + 1), __ldg(xs + 3 * qi + 2)};
        const float d[3] = {__ldg(ds + 3 * qi), __ldg(ds + 3 * qi + 1), __ldg(ds + 3 * qi + 2)};
        const float* wp = wls + (int64_t)wl_stride * qi;
        const float wl[3] = {__ldg(wp), __ldg(wp + 1), __ldg(wp + 2)};
        const Frame F = make_frame(d, wl);
        OutT* row = out + qi * (int64_t)(RPNN_K * RPNN_DESC_STRIDE);
        if (k < RPNN_K) {
            float P[3], C[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float A = __fmul_rn(gk, F.ex[a]), B = __fmul_rn(gk, F.ey[a]);
                C[a] = __fmul_rn(gk, F.ez[a]);
                const float U0 = __fsub_rn(__fmul_rn(x[a], s), 0.5f);
                P[a] = __fmaf_rn(oy, B, __fmaf_rn(ox, A, U0));
            }
            OutT* dst = row + k * RPNN_DESC_STRIDE + col;
#pragma unroll 3
            for (int iz = 0; iz < 9; ++iz) {
                const float oz = __fadd_rn(-1.0f, __fmul_rn(0.5f, (float)iz));
                const float u[3] = {__fmaf_rn(oz, C[0], P[0]), __fmaf_rn(oz, C[1], P[1]),
                                    __fmaf_rn(oz, C[2], P[2])};
                dst[iz * 25] = cvt_out<OutT>(lookup(v, m, u));
            }
        } else {
            for (int e = t - 250; e < RPNN_K * (RPNN_DESC_STRIDE - RPNN_S); e += 6) {
                const int kk = e / (RPNN_DESC_STRIDE - RPNN_S), j = e % (RPNN_DESC_STRIDE - RPNN_S);
                row[kk * RPNN_DESC_STRIDE + RPNN_S + j] = cvt_out<OutT>(j == 0 ? F.gamma : 0.0f);
            }
        }
    }
}

}  // namespace

rpnn_status launch_descriptor(Ctx& c, const VolumeView& vv, const float* x, const float* d,
                              const float* wl, int wl_stride, int64_t q, const int* q_dev,
                              void* out, int dtype, cudaStream_t s) {
    if (q <= 0 && !q_dev) return RPNN_OK;
    int64_t g = q_dev ? (int64_t)c.num_sms * 8 : q;
    if (g > (int64_t)c.num_sms * 8) g = (int64_t)c.num_sms * 8;
    if (dtype == RPNN_F32)
        k_descriptor<float><<<(int)g, 256, 0, s>>>(vv, x, d, wl, wl_stride, q, q_dev, (float*)out);
    else
        k_descriptor<__nv_bfloat16><<<(int)g, 256, 0, s>>>(vv, x, d, wl, wl_stride, q, q_dev,
                                                           (__nv_bfloat16*)out);
    RPNN_CHECK_LAUNCH();
    return RPNN_OK;
}

}  // namespace rpnn
