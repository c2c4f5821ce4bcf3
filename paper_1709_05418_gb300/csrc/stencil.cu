// stencil.cu -- descriptors of other stencil resolutions, for the stencil-size comparison of
// Sec. 7 (Fig. 10, right).
//
// The standard stencil (Sec. 4.2, Fig. 5) has 5 x 5 x 9 points spaced half a mean free path
// over [-1, 1] x [-1, 1] x [-1, 3] (times 2^(k-1) at level k).  The comparison keeps that
// extent and changes the resolution: n x n x (2n - 1) points spaced h = 2 / (n - 1), each
// level reading the mip whose voxel is the largest power of two not above the spacing (so
// n = 5 gives the standard descriptor, bit for bit).  Rows are FP32 [q][RPNN_K][din],
// din = n^2 (2n - 1) + 1 (the points, then gamma), for the FP32 network of any input width
// (rpnn_forward_f32 / rpnn_backward_f32).
//
// This is an experiment path, not the renderer's: every pyramid level is kept as plain
// FP32 (built once per volume), one warp per shading point deals the (level, column) tasks
// to its lanes, and each task walks its column's 2n - 1 points along z.  The arithmetic is
// the standard descriptor's fixed FP32 sequence (light-aligned frame with separately
// rounded products, u = fma(oz, C, fma(oy, B, fma(ox, A, x s - 1/2))), trilinear lerps
// fma(f, b - a, a) in x, y, z order, zero outside the level).
#include <cmath>

#include "common.cuh"

namespace rpnn {

namespace {

constexpr int kStencilMin = 2, kStencilMax = 9;

struct StencilLevel {
    int64_t off;     // level data in the plain pyramid
    int ax, ay, az;  // level dims
    float s, gk;     // inv_h0 2^-m and (inv_mean 2^k) s
};

struct StencilArgs {
    const float* mips;
    StencilLevel lv[RPNN_K];
    int n, nz, din;
    float h;         // point spacing in stencil units
};

__device__ __forceinline__ float lerp_fma(float a, float b, float f) { return __fmaf_rn(f, __fsub_rn(b, a), a); }

__device__ __forceinline__ float voxel(const float* __restrict__ v, const StencilLevel& L, int x, int y, int z) {
    if (x < 0 || y < 0 || z < 0 || x >= L.ax || y >= L.ay || z >= L.az) return 0.0f;
    return __ldg(v + ((int64_t)z * L.ay + y) * L.ax + x);
}

// trilinear lookup at level coordinates u (voxel centres at integers), zero outside
__device__ __forceinline__ float trilinear(const float* __restrict__ v, const StencilLevel& L, float u0, float u1,
                                           float u2) {
    const float c0 = fminf(fmaxf(u0, -1.0e6f), 1.0e6f), c1 = fminf(fmaxf(u1, -1.0e6f), 1.0e6f),
                c2 = fminf(fmaxf(u2, -1.0e6f), 1.0e6f);
    const float l0 = floorf(c0), l1 = floorf(c1), l2 = floorf(c2);
    const int i0 = (int)l0, i1 = (int)l1, i2 = (int)l2;
    if (i0 < -1 || i0 > L.ax - 1 || i1 < -1 || i1 > L.ay - 1 || i2 < -1 || i2 > L.az - 1) return 0.0f;
    const float f0 = __fsub_rn(c0, l0), f1 = __fsub_rn(c1, l1), f2 = __fsub_rn(c2, l2);
    const float c00 = lerp_fma(voxel(v, L, i0, i1, i2), voxel(v, L, i0 + 1, i1, i2), f0);
    const float c10 = lerp_fma(voxel(v, L, i0, i1 + 1, i2), voxel(v, L, i0 + 1, i1 + 1, i2), f0);
    const float c01 = lerp_fma(voxel(v, L, i0, i1, i2 + 1), voxel(v, L, i0 + 1, i1, i2 + 1), f0);
    const float c11 = lerp_fma(voxel(v, L, i0, i1 + 1, i2 + 1), voxel(v, L, i0 + 1, i1 + 1, i2 + 1), f0);
    return lerp_fma(lerp_fma(c00, c10, f1), lerp_fma(c01, c11, f1), f2);
}

struct Frame3 {
    float ex[3], ey[3], ez[3], gamma;
};

// light-aligned frame: ez = wl, ex = normalize(ez x omega), ey = ez x ex (omega = -d);
// a degenerate omega takes ex from Duff et al.'s basis of ez (FP32, fixed rounding sequence)
__device__ __forceinline__ Frame3 light_frame(const float d[3], const float wl[3]) {
    Frame3 F;
    const float w[3] = {-d[0], -d[1], -d[2]};
    float cr[3];
    cr[0] = __fsub_rn(__fmul_rn(wl[1], w[2]), __fmul_rn(wl[2], w[1]));
    cr[1] = __fsub_rn(__fmul_rn(wl[2], w[0]), __fmul_rn(wl[0], w[2]));
    cr[2] = __fsub_rn(__fmul_rn(wl[0], w[1]), __fmul_rn(wl[1], w[0]));
    const float len2 = __fadd_rn(__fadd_rn(__fmul_rn(cr[0], cr[0]), __fmul_rn(cr[1], cr[1])),
                                 __fmul_rn(cr[2], cr[2]));
    if (len2 < 1e-12f) {
        const float sg = signbit(wl[2]) ? -1.0f : 1.0f;
        const float a = __fdiv_rn(-1.0f, __fadd_rn(sg, wl[2]));
        F.ex[0] = __fadd_rn(1.0f, __fmul_rn(__fmul_rn(__fmul_rn(sg, wl[0]), wl[0]), a));
        F.ex[1] = __fmul_rn(sg, __fmul_rn(__fmul_rn(wl[0], wl[1]), a));
        F.ex[2] = __fmul_rn(-sg, wl[0]);
    } else {
        const float len = __fsqrt_rn(len2);
        for (int a = 0; a < 3; ++a) F.ex[a] = __fdiv_rn(cr[a], len);
    }
    for (int a = 0; a < 3; ++a) F.ez[a] = wl[a];
    F.ey[0] = __fsub_rn(__fmul_rn(wl[1], F.ex[2]), __fmul_rn(wl[2], F.ex[1]));
    F.ey[1] = __fsub_rn(__fmul_rn(wl[2], F.ex[0]), __fmul_rn(wl[0], F.ex[2]));
    F.ey[2] = __fsub_rn(__fmul_rn(wl[0], F.ex[1]), __fmul_rn(wl[1], F.ex[0]));
    float cg = __fadd_rn(__fadd_rn(__fmul_rn(w[0], wl[0]), __fmul_rn(w[1], wl[1])), __fmul_rn(w[2], wl[2]));
    cg = fminf(fmaxf(cg, -1.0f), 1.0f);
    F.gamma = acosf(cg);
    return F;
}

// one warp per shading point (grid-stride); lanes take the RPNN_K * n^2 column tasks
__global__ void __launch_bounds__(256) k_stencil(StencilArgs a, const float* __restrict__ xs,
                                                 const float* __restrict__ ds, const float* __restrict__ wls,
                                                 int wl_stride, int64_t q, float* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int cols = a.n * a.n, S = cols * a.nz;
    for (int64_t qi = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); qi < q; qi += warps) {
        const float* wp = wls + (int64_t)wl_stride * qi;
        const float wl[3] = {__ldg(wp), __ldg(wp + 1), __ldg(wp + 2)};
        const float x[3] = {__ldg(xs + 3 * qi), __ldg(xs + 3 * qi + 1), __ldg(xs + 3 * qi + 2)};
        const float d[3] = {__ldg(ds + 3 * qi), __ldg(ds + 3 * qi + 1), __ldg(ds + 3 * qi + 2)};
        const Frame3 F = light_frame(d, wl);
        float* row = out + qi * (int64_t)RPNN_K * a.din;
        for (int task = lane; task < RPNN_K * cols; task += 32) {
            const int k = task / cols, col = task - cols * k;
            const int iy = col / a.n, ix = col - a.n * iy;
            const StencilLevel& L = a.lv[k];
            const float ox = __fadd_rn(-1.0f, __fmul_rn(a.h, (float)ix));
            const float oy = __fadd_rn(-1.0f, __fmul_rn(a.h, (float)iy));
            float P[3], C[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float A = __fmul_rn(L.gk, F.ex[c]), B = __fmul_rn(L.gk, F.ey[c]);
                C[c] = __fmul_rn(L.gk, F.ez[c]);
                const float U0 = __fsub_rn(__fmul_rn(x[c], L.s), 0.5f);
                P[c] = __fmaf_rn(oy, B, __fmaf_rn(ox, A, U0));
            }
            const float* lv = a.mips + L.off;
            float* dst = row + (int64_t)k * a.din + col;
            for (int iz = 0; iz < a.nz; ++iz) {
                const float oz = __fadd_rn(-1.0f, __fmul_rn(a.h, (float)iz));
                dst[(int64_t)iz * cols] = trilinear(lv, L, __fmaf_rn(oz, C[0], P[0]), __fmaf_rn(oz, C[1], P[1]),
                                                    __fmaf_rn(oz, C[2], P[2]));
            }
        }
        for (int k = lane; k < RPNN_K; k += 32) row[(int64_t)k * a.din + S] = F.gamma;
    }
}

// every pyramid level of v as plain FP32, built once per pyramid
rpnn_status stencil_mips(Ctx& c, Volume& v, cudaStream_t s) {
    if (v.stencil_ready) return RPNN_OK;
    int64_t total = 0;
    for (int m = 0; m < v.levels; ++m) {
        v.smip_off[m] = total;
        total += (int64_t)v.dims[m][0] * v.dims[m][1] * v.dims[m][2];
    }
    rpnn_status st = v.stencil_mips.reserve((size_t)total * sizeof(float));
    if (st) return st;
    for (int m = 0; m < v.levels; ++m) {
        st = volume_build_level(c, v, m, v.stencil_mips.as<float>() + v.smip_off[m], s);
        if (st) return st;
    }
    v.stencil_ready = true;
    return RPNN_OK;
}

}  // namespace

int stencil_din(int n_xy) {
    if (n_xy < kStencilMin || n_xy > kStencilMax) return -1;
    return n_xy * n_xy * (2 * n_xy - 1) + 1;
}

rpnn_status stencil_descriptors(Ctx& c, Volume& v, int n_xy, const float* x, const float* d, const float* wl,
                                int wl_stride, int64_t q, float* out, cudaStream_t s) {
    const int din = stencil_din(n_xy);
    if (din < 0) {
        set_error("stencil resolution %d outside [%d, %d]", n_xy, kStencilMin, kStencilMax);
        return RPNN_ERR_ARG;
    }
    if (q == 0) return RPNN_OK;
    rpnn_status st = stencil_mips(c, v, s);
    if (st) return st;
    const VolumeView vw = v.view();
    StencilArgs a{};
    a.mips = v.stencil_mips.as<float>();
    a.n = n_xy;
    a.nz = 2 * n_xy - 1;
    a.din = din;
    const double h = 2.0 / (double)(n_xy - 1);
    a.h = (float)h;
    for (int k = 0; k < RPNN_K; ++k) {
        // the level whose voxel is the largest power of two (in fine voxels) not above the
        // spacing h 2^(k-1) mean free paths, clamped to the pyramid
        const double sk = h * std::ldexp((double)vw.inv_mean_f, k) * (double)vw.inv_h0;
        int m = 0;
        if (sk > 0.0) {
            int ex;
            std::frexp(sk, &ex);
            m = ex - 1;
        }
        m = m < 0 ? 0 : (m > v.levels - 1 ? v.levels - 1 : m);
        StencilLevel& L = a.lv[k];
        L.off = v.smip_off[m];
        L.ax = v.dims[m][0];
        L.ay = v.dims[m][1];
        L.az = v.dims[m][2];
        L.s = std::ldexp(vw.inv_h0, -m);
        L.gk = std::ldexp(vw.inv_mean_f, k) * L.s;
    }
    const int64_t blocks = (q + 7) / 8;
    const int grid = (int)(blocks < (int64_t)c.num_sms * 8 ? blocks : (int64_t)c.num_sms * 8);
    k_stencil<<<grid, 256, 0, s>>>(a, x, d, wl, wl_stride, q, out);
    RPNN_CHECK_LAUNCH();
    return RPNN_OK;
}

}  // namespace rpnn
