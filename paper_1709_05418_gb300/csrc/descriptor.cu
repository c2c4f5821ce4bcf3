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
// Layout: one warp per shading point; each lookup reads one 32-byte corner record with a
// single 256-bit load.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "common.cuh"
#include "desc_lookup.cuh"

namespace rpnn {

namespace {

using namespace desc;

template <class T> __device__ __forceinline__ T cvt_out(float v);
template <> __device__ __forceinline__ float cvt_out<float>(float v) { return v; }
// E4M3: round to nearest even, saturating at +-448 (the descriptor is stored unscaled)
template <> __device__ __forceinline__ __nv_fp8_e4m3 cvt_out<__nv_fp8_e4m3>(float v) { return __nv_fp8_e4m3(v); }
template <> __device__ __forceinline__ __nv_bfloat16 cvt_out<__nv_bfloat16>(float v) {
    return __float2bfloat16_rn(v);
}

// One warp per shading point (8 per block, grid-stride over points, one block-wide
// barrier at the start).  The 250 column tasks (level k, stencil column (ix, iy)) are
// dealt to the lanes in order; a task reads its level's constants from shared memory,
// computes the (ox, oy) part of the coordinate once and walks the 9 points along z
// (fully unrolled: oz = -1 + 0.5 iz are constants).  BF16 rows are assembled in a
// per-warp shared buffer and written with 16-byte stores; FP32 rows are stored
// directly (25 consecutive values per level and z-slice).
//
// BATCH: the shading points of up to RPNN_MAX_BATCH renders, compacted: point j belongs
// to the item i with off[i] <= j < off[i+1], reads its position and direction at
// region_i + j - off[i], and uses item i's volume and light; row j of `out` is written.
// BLEND: some stencil level blends two mip levels (a separate instance, so the plain
// kernel keeps its registers).
template <class OutT, bool BATCH, bool BLEND>
__global__ void __launch_bounds__(256, sizeof(OutT) == 2 ? (BATCH ? 4 : 5) : 4)
k_descriptor(const VolumeView v, const float* __restrict__ xs, const float* __restrict__ ds,
             const float* __restrict__ wls, int wl_stride, int64_t q_host,
             const int* __restrict__ q_dev, OutT* __restrict__ out, const BatchItemDev* __restrict__ items,
             int n_items, const int* __restrict__ off) {
    // row stride per level: 240 values (FP32, BF16) or 256 (E4M3: whole 32-byte K-steps)
    constexpr int DS = sizeof(OutT) == 1 ? 256 : RPNN_DESC_STRIDE;
    constexpr int ROW = RPNN_K * DS;
    constexpr bool STAGE = sizeof(OutT) <= 2;
    constexpr int NI = BATCH ? RPNN_MAX_BATCH : 1;
    __shared__ __align__(16) OutT rowbuf[STAGE ? 8 : 1][STAGE ? ROW : 8];
    __shared__ LevelK lk[NI][RPNN_K];
    __shared__ LevelB lb[BLEND ? NI : 1][RPNN_K];
    __shared__ int s_off[NI + 1];
    __shared__ int64_t s_region[NI];
    __shared__ float s_light[NI][3];
    __shared__ const float4* s_packed[NI];
    if (BATCH) {
        for (int e = threadIdx.x; e < n_items * RPNN_K; e += blockDim.x) {
            lk[e / RPNN_K][e % RPNN_K] = make_level(items[e / RPNN_K].v, e % RPNN_K);
            if (BLEND) lb[e / RPNN_K][e % RPNN_K] = make_blend(items[e / RPNN_K].v, e % RPNN_K);
        }
        for (int i = threadIdx.x; i <= n_items; i += blockDim.x) s_off[i] = off[i];
        for (int i = threadIdx.x; i < n_items; i += blockDim.x) {
            s_region[i] = items[i].region;
            s_packed[i] = items[i].v.packed;
            for (int a = 0; a < 3; ++a) s_light[i][a] = items[i].light[a];
        }
    } else if (threadIdx.x < RPNN_K) {
        lk[0][threadIdx.x] = make_level(v, threadIdx.x);
        if (BLEND) lb[0][threadIdx.x] = make_blend(v, threadIdx.x);
    }
    __syncthreads();
    const int64_t q = BATCH ? (int64_t)s_off[n_items] : (q_dev ? (int64_t)*q_dev : q_host);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t qi = (int64_t)blockIdx.x * 8 + warp; qi < q; qi += (int64_t)gridDim.x * 8) {
        int it = 0;
        int64_t src = qi;
        const float4* packed = v.packed;
        float wl[3];
        if (BATCH) {
            while (it + 1 < n_items && s_off[it + 1] <= qi) ++it;
            src = s_region[it] + (qi - s_off[it]);
            packed = s_packed[it];
            for (int a = 0; a < 3; ++a) wl[a] = s_light[it][a];
        } else {
            const float* wp = wls + (int64_t)wl_stride * qi;
            for (int a = 0; a < 3; ++a) wl[a] = __ldg(wp + a);
        }
        const float x[3] = {__ldg(xs + 3 * src), __ldg(xs + 3 * src + 1), __ldg(xs + 3 * src + 2)};
        const float d[3] = {__ldg(ds + 3 * src), __ldg(ds + 3 * src + 1), __ldg(ds + 3 * src + 2)};
        const Frame F = make_frame(d, wl);
        const LevelK* lki = lk[it];
        const LevelB* lbi = lb[BLEND ? it : 0];
        OutT* grow = out + qi * (int64_t)ROW;
        OutT* row = STAGE ? rowbuf[warp] : grow;
        for (int task = lane; task < RPNN_K * 25; task += 32) {
            const int k = task / 25, col = task - 25 * k;
            const int iy = col / 5, ix = col - 5 * iy;
            const float ox = __fadd_rn(-1.0f, __fmul_rn(0.5f, (float)ix));
            const float oy = __fadd_rn(-1.0f, __fmul_rn(0.5f, (float)iy));
            const LevelK g = lki[k];
            float P[3], C[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float A = __fmul_rn(g.gk, F.ex[a]), B = __fmul_rn(g.gk, F.ey[a]);
                C[a] = __fmul_rn(g.gk, F.ez[a]);
                const float U0 = __fsub_rn(__fmul_rn(x[a], g.s), 0.5f);
                P[a] = __fmaf_rn(oy, B, __fmaf_rn(ox, A, U0));
            }
            OutT* dst = row + k * DS + col;
            const float bw = BLEND ? lbi[k].w : 0.0f;
            if (BLEND && bw > 0.0f) {
                // blended: lerp(rho_m, rho_{m+1}, w), level m + 1 read at its own coordinates
                const LevelB b = lbi[k];
                float P1[3], C1[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const float A = __fmul_rn(b.gk1, F.ex[a]), B = __fmul_rn(b.gk1, F.ey[a]);
                    C1[a] = __fmul_rn(b.gk1, F.ez[a]);
                    const float U0 = __fsub_rn(__fmul_rn(x[a], b.s1), 0.5f);
                    P1[a] = __fmaf_rn(oy, B, __fmaf_rn(ox, A, U0));
                }
#pragma unroll 3
                for (int iz = 0; iz < 9; ++iz) {
                    const float oz = -1.0f + 0.5f * (float)iz;
                    const float r0 = lookup(packed, g.g0, __fmaf_rn(oz, C[0], P[0]), __fmaf_rn(oz, C[1], P[1]),
                                            __fmaf_rn(oz, C[2], P[2]));
                    const float r1 = lookup(packed, b.g1, __fmaf_rn(oz, C1[0], P1[0]), __fmaf_rn(oz, C1[1], P1[1]),
                                            __fmaf_rn(oz, C1[2], P1[2]));
                    dst[iz * 25] = cvt_out<OutT>(lerp_rn(r0, r1, b.w));
                }
            } else {
#pragma unroll
                for (int iz = 0; iz < 9; ++iz) {
                    const float oz = -1.0f + 0.5f * (float)iz;      // exact: -1, -0.5, ..., 3
                    dst[iz * 25] = cvt_out<OutT>(lookup(packed, g.g0, __fmaf_rn(oz, C[0], P[0]),
                                                        __fmaf_rn(oz, C[1], P[1]), __fmaf_rn(oz, C[2], P[2])));
                }
            }
        }
        for (int e = lane; e < RPNN_K * (DS - RPNN_S); e += 32) {
            const int kk = e / (DS - RPNN_S), j = e % (DS - RPNN_S);
            row[kk * DS + RPNN_S + j] = cvt_out<OutT>(j == 0 ? F.gamma : 0.0f);
        }
        if (STAGE) {
            __syncwarp();
            uint4* gdst = reinterpret_cast<uint4*>(grow);
            const uint4* ssrc = reinterpret_cast<const uint4*>(row);
            for (int e = lane; e < ROW * (int)sizeof(OutT) / 16; e += 32) gdst[e] = ssrc[e];
            __syncwarp();
        }
    }
}

template <class OutT, bool BATCH, bool BLEND>
int blocks_per_sm() {
    static int nb = 0;
    if (!nb) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_descriptor<OutT, BATCH, BLEND>, 256, 0) != cudaSuccess ||
            nb <= 0)
            nb = 1;
    }
    return nb;
}

template <class OutT, bool BLEND>
rpnn_status launch_one(Ctx& c, const VolumeView& vv, const float* x, const float* d, const float* wl,
                       int wl_stride, int64_t q, const int* q_dev, void* out, cudaStream_t s) {
    // one resident wave of blocks (8 shading points each), grid-stride beyond that
    const int64_t wave = (int64_t)c.num_sms * blocks_per_sm<OutT, false, BLEND>();
    int64_t g = q_dev ? wave : (q + 7) / 8;
    if (g > wave) g = wave;
    k_descriptor<OutT, false, BLEND><<<(int)g, 256, 0, s>>>(vv, x, d, wl, wl_stride, q, q_dev, (OutT*)out, nullptr, 0,
                                                            nullptr);
    RPNN_CHECK_LAUNCH();
    return RPNN_OK;
}

template <class OutT>
rpnn_status launch_typed(Ctx& c, const VolumeView& vv, const float* x, const float* d, const float* wl,
                         int wl_stride, int64_t q, const int* q_dev, void* out, cudaStream_t s) {
    bool blend = false;
    for (int k = 0; k < RPNN_K; ++k) blend |= vv.mip_w[k] > 0.0f;
    return blend ? launch_one<OutT, true>(c, vv, x, d, wl, wl_stride, q, q_dev, out, s)
                 : launch_one<OutT, false>(c, vv, x, d, wl, wl_stride, q, q_dev, out, s);
}

}  // namespace

rpnn_status launch_descriptor(Ctx& c, const VolumeView& vv, const float* x, const float* d,
                              const float* wl, int wl_stride, int64_t q, const int* q_dev,
                              void* out, int dtype, cudaStream_t s) {
    if (q <= 0 && !q_dev) return RPNN_OK;
    if (dtype == RPNN_F32) return launch_typed<float>(c, vv, x, d, wl, wl_stride, q, q_dev, out, s);
    if (dtype == RPNN_FP8E4M3) return launch_typed<__nv_fp8_e4m3>(c, vv, x, d, wl, wl_stride, q, q_dev, out, s);
    return launch_typed<__nv_bfloat16>(c, vv, x, d, wl, wl_stride, q, q_dev, out, s);
}

rpnn_status launch_descriptor_batch(Ctx& c, const BatchItemDev* items, int n, const float* x, const float* d,
                                    const int* off, int64_t cap, void* out, bool blend, cudaStream_t s) {
    if (n < 1 || n > RPNN_MAX_BATCH) { set_error("batch of %d items", n); return RPNN_ERR_ARG; }
    const int64_t wave = (int64_t)c.num_sms * (blend ? blocks_per_sm<__nv_bfloat16, true, true>()
                                                     : blocks_per_sm<__nv_bfloat16, true, false>());
    int64_t g = (cap + 7) / 8;
    if (g > wave) g = wave;
    if (g < 1) g = 1;
    VolumeView none{};
    if (blend)
        k_descriptor<__nv_bfloat16, true, true><<<(int)g, 256, 0, s>>>(none, x, d, nullptr, 0, cap, nullptr,
                                                                       (__nv_bfloat16*)out, items, n, off);
    else
        k_descriptor<__nv_bfloat16, true, false><<<(int)g, 256, 0, s>>>(none, x, d, nullptr, 0, cap, nullptr,
                                                                        (__nv_bfloat16*)out, items, n, off);
    RPNN_CHECK_LAUNCH();
    return RPNN_OK;
}

}  // namespace rpnn
