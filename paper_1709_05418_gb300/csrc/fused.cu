// fused.cu -- descriptor gather (Sec. 4.2, Fig. 5) fused into the BF16 tcgen05 network
// (Sec. 4.3, Fig. 6): the render's shading points go from (x, d) to the prediction g(z) in
// one persistent kernel, without descriptor rows in global memory.
//
// Same network as k_rpnn_tc (128-query tiles, 22 tensor-core layers, two FP32 accumulators
// in tensor memory, one activation buffer, biases riding in the MMAs), with its descriptor
// ring filled by gather warps instead of TMA copies:
//   warp 0        weight producer: the pre-arranged BF16 weight image, one bulk copy per
//                 ring stage of 64 K-columns;
//   warp 1        tensor-memory owner and MMA issuer (the issue loop of k_rpnn_tc);
//   warps 2-9     epilogue: accumulator -> ReLU -> BF16 activations, in four rounds of
//                 64 columns (one publication each), so 72 registers a thread suffice;
//   warps 10-25   gather: lane = shading point (one 32-row group of the tile per warp and
//                 four warps per group), each warp computes 8-column tasks of a ring stage
//                 (8 consecutive stencil points of its lane's query, in the canonical
//                 (iz*5 + iy)*5 + ix order, then gamma and zeros) with the FP32 arithmetic
//                 of desc_lookup.cuh, rounds them to BF16 and stores them as one 16-byte
//                 unit of the 64-byte-swizzled operand row.
// The ring holds the descriptor in exactly the layout the TMA copies of the row-reading
// kernel produce, and every value is the one k_descriptor would write, so the MMAs, their
// order and the prediction are those of descriptor + network bit for bit.
//
// Adjacent lanes hold adjacent shading points (the compacted query list is in pixel
// order), so at the coarse stencil levels many lanes read the same corner record.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "desc_lookup.cuh"
#include "tc_net.cuh"
#include "tc_ptx.cuh"

namespace rpnn {

namespace {

using namespace net;
using namespace desc;

constexpr int W_STAGES = 3, Z_STAGES = 4;
constexpr int EPI_WARPS = 8;
constexpr int G_FIRST = 2 + EPI_WARPS;          // first gather warp
constexpr int G_WARPS = 16;                     // 4 per 32-row query group
constexpr int NTHREADS = 32 * (G_FIRST + G_WARPS);
constexpr int NPTS = 240;                       // stored width of one descriptor level

constexpr uint32_t OFF_X = 0;
constexpr uint32_t OFF_W = OFF_X + NBLK * BLK_A;               // 57344
constexpr uint32_t OFF_Z = OFF_W + W_STAGES * W_STAGE;         // 137216
constexpr uint32_t OFF_BAR = OFF_Z + Z_STAGES * Z_STAGE;       // 202752
enum {
    B_WFULL = 0, B_WEMPTY = B_WFULL + W_STAGES, B_ZFULL = B_WEMPTY + W_STAGES, B_ZEMPTY = B_ZFULL + Z_STAGES,
    B_ACC = B_ZEMPTY + Z_STAGES, B_BLK, B_PART = B_BLK + NPUB_MAX, B_DRAIN, B_COUNT
};
constexpr uint32_t OFF_TMEM_SLOT = OFF_BAR + BAR_STRIDE * B_COUNT;
constexpr uint32_t OFF_ABORT = OFF_TMEM_SLOT + 8;
constexpr uint32_t OFF_PART = OFF_ABORT + 8;                   // 3 x 128 floats
constexpr uint32_t OFF_LK = (OFF_PART + 3 * 128 * 4 + 15) & ~15u;   // LevelK[10]
constexpr uint32_t OFF_OFS = OFF_LK + RPNN_K * sizeof(LevelK);  // float4[NPTS]: stencil offsets
constexpr uint32_t SMEM_BYTES = OFF_OFS + NPTS * 16 + 64;
static_assert(OFF_W % 1024 == 0 && OFF_Z % 1024 == 0, "swizzled operand blocks must stay 1024-byte aligned");
static_assert(OFF_OFS % 16 == 0 && sizeof(LevelK) % 16 == 0, "shared tables must be 16-byte aligned");
static_assert(SMEM_BYTES <= 232448, "shared memory over the per-block limit");

struct FusedArgs {
    TcArgs net;                 // weight image, bias table, output layer, count, output, status
    VolumeView v;
    const float* xs;            // shading points [q][3]
    const float* ds;            // tracing directions [q][3]
    float wl[3];                // light direction (towards the light)
};

// Stencil point p's offsets in mean free paths: (ox, oy, oz) = -1 + (ix, iy, iz) / 2 for
// p = (iz*5 + iy)*5 + ix < 225; w = 1 marks gamma (p = 225), w = 2 the zero padding.
__device__ __forceinline__ float4 stencil_offset(int p) {
    if (p >= RPNN_S) return make_float4(0.0f, 0.0f, 0.0f, p == RPNN_S ? 1.0f : 2.0f);
    const int iz = p / 25, iy = (p % 25) / 5, ix = p % 5;
    return make_float4(__fadd_rn(-1.0f, __fmul_rn(0.5f, (float)ix)), __fadd_rn(-1.0f, __fmul_rn(0.5f, (float)iy)),
                       -1.0f + 0.5f * (float)iz, 0.0f);
}

// Stencil points p0 .. p0+7 of the lane's shading point at level (g; frame terms A, B, C,
// U0), as BF16 pairs in one 16-byte unit.  cls (stencil_class) selects lookups without
// range tests, with them, or none; the values are those of lookup() in every case.
template <int CLS>
__device__ __forceinline__ uint4 gather_points(const float4* __restrict__ packed, const LevelGeo& g, const float4* ofs,
                                               int p0, const float (&A)[3], const float (&B)[3], const float (&C)[3],
                                               const float (&U0)[3]) {
    uint32_t w[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        float val[2];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const float4 o = ofs[p0 + 2 * h + i];
            float u[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) u[a] = __fmaf_rn(o.z, C[a], __fmaf_rn(o.y, B[a], __fmaf_rn(o.x, A[a], U0[a])));
            val[i] = CLS == kInside ? lookup_in(packed, g, u[0], u[1], u[2]) : lookup(packed, g, u[0], u[1], u[2]);
        }
        w[h] = pack_bf16x2(val[0], val[1]);
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// The level's tail task (columns 224..231): its last point, gamma, zeros.
__device__ __forceinline__ uint4 gather_tail(const float4* __restrict__ packed, const LevelGeo& g, const float4* ofs,
                                             const float (&A)[3], const float (&B)[3], const float (&C)[3],
                                             const float (&U0)[3], float gamma, bool live) {
    const float4 o = ofs[RPNN_S - 1];
    float u[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) u[a] = __fmaf_rn(o.z, C[a], __fmaf_rn(o.y, B[a], __fmaf_rn(o.x, A[a], U0[a])));
    const float last = live ? lookup(packed, g, u[0], u[1], u[2]) : 0.0f;
    return make_uint4(pack_bf16x2(last, live ? gamma : 0.0f), 0u, 0u, 0u);
}

__global__ void __launch_bounds__(NTHREADS, 1) k_rpnn_fused(const __grid_constant__ FusedArgs fa) {
    using F = FmtBF16;
    extern __shared__ __align__(1024) unsigned char sm[];
    const TcArgs& a = fa.net;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t base = tc::smem_u32(sm);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + OFF_ABORT);
    auto bar = [&](int i) { return base + OFF_BAR + BAR_STRIDE * (uint32_t)i; };
    const int64_t Q = a.q_dev ? (int64_t)*a.q_dev : a.q_host;
    const int ntiles = (int)((Q + TM - 1) / TM);
    LevelK* lk = reinterpret_cast<LevelK*>(sm + OFF_LK);
    float4* ofs = reinterpret_cast<float4*>(sm + OFF_OFS);

    if (tid == 0) {
        *abort_flag = (base & 1023u) ? 1 : 0;
        for (int s = 0; s < W_STAGES; ++s) { tc::mbar_init(bar(B_WFULL + s), 1); tc::mbar_init(bar(B_WEMPTY + s), 1); }
        for (int s = 0; s < Z_STAGES; ++s) {
            tc::mbar_init(bar(B_ZFULL + s), G_WARPS);           // one arrival per gather warp
            tc::mbar_init(bar(B_ZEMPTY + s), 1);
        }
        tc::mbar_init(bar(B_ACC), 1);
        for (int b = 0; b < npub<F>(); ++b) tc::mbar_init(bar(B_BLK + b), EPI_WARPS);
        tc::mbar_init(bar(B_PART), EPI_WARPS / 2);
        tc::mbar_init(bar(B_DRAIN), 1);
        tc::fence_mbar_init();
    }
    if (warp == 1) {
        tc::tmem_alloc(base + OFF_TMEM_SLOT, 512);
        tc::tmem_relinquish();
    }
    if (tid < RPNN_K) lk[tid] = make_level(fa.v, tid);
    for (int p = tid; p < NPTS; p += NTHREADS) ofs[p] = stencil_offset(p);
    for (int i = tid; i < (int)(NBLK * BLK_A / 16); i += NTHREADS) reinterpret_cast<uint4*>(sm + OFF_X)[i] = make_uint4(0, 0, 0, 0);
    tc::fence_proxy_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(sm + OFF_TMEM_SLOT);

    if (warp == 0) {
        // ------------------------------------------------------------ weight producer
        if (lane == 0 && !*abort_flag) {
            uint32_t sw = 0, pw = 0, wfills = 0;
            for (int t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x) {
                for (int l = 0; l < NLAYERS && !*abort_flag; ++l) {
                    const int KB = layer_kb<F>(l), nb = layer_blocks<F>(l);
                    for (int k0 = 0; k0 < KB; k0 += SKB) {
                        const int b0 = k0 / 64;
                        const uint32_t bytes = (nb - b0 >= 2 ? 2u : 1u) * BLK_B;
                        if (!tc::mbar_wait(bar(B_WEMPTY + sw), pw ^ 1u, abort_flag)) break;
                        tc::mbar_expect_tx(bar(B_WFULL + sw), bytes);
                        tc::bulk_g2s(base + OFF_W + sw * W_STAGE, a.img + a.img_off[l] + (int64_t)b0 * BLK_B, bytes,
                                     bar(B_WFULL + sw));
                        ++wfills;
                        if (++sw == W_STAGES) { sw = 0; pw ^= 1u; }
                    }
                }
            }
            if (*abort_flag) {
                for (uint32_t s2 = 0; s2 < W_STAGES && s2 < wfills; ++s2)
                    tc::mbar_poll(bar(B_WFULL + s2), ((wfills - 1 - s2) / W_STAGES) & 1u, tc::kSpinLimit);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0 && !*abort_flag) {
            IssueState S;
            S.idesc = tc::idesc_bf16(TM, NP);
            S.abort_addr = base + OFF_ABORT;
            S.hi = (uint32_t)(tc::smem_desc_sw64(base) >> 32);
            S.w0 = (uint32_t)tc::smem_desc_sw64(base + OFF_W);
            S.z0 = (uint32_t)tc::smem_desc_sw64(base + OFF_Z);
            S.x0 = (uint32_t)tc::smem_desc_sw64(base + OFF_X);
            S.wbar0 = bar(B_WFULL);
            S.zbar0 = bar(B_ZFULL);
            S.blk0 = bar(B_BLK);
            S.w = S.w0; S.z = S.z0; S.wbar = S.wbar0; S.zbar = S.zbar0;
            S.sw = 0; S.pw = 0; S.sz = 0; S.pz = 0;
            uint32_t n = 0;
            for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
                for (int l = 0; l < NLAYERS; ++l, ++n) {
                    const uint32_t acc = tmem + (uint32_t)(l & 1) * 256u;
                    tc::tc_fence_after();
                    const uint32_t pb = (uint32_t)(l & 1) ^ 1u;
                    if (l == 0) {
                        issue_layer<W_STAGES, Z_STAGES, false, F::KZB, F::KZB, false>(S, acc, pb);
                        if (n > 0)
                            tc::mbar_wait_issuer(S.blk0 + BAR_STRIDE * (npub<F>() - 1), pb, tc::kSpinLimit, S.abort_addr);
                    } else if (l < 20 && !(l & 1)) {
                        issue_layer<W_STAGES, Z_STAGES, false, F::KZB + F::XB, F::KZB, false>(S, acc, pb);
                    } else if (layer_resid(l)) {
                        issue_layer<W_STAGES, Z_STAGES, false, F::XB, 0, true>(S, acc, pb);
                    } else {
                        issue_layer<W_STAGES, Z_STAGES, false, F::XB, 0, false>(S, acc, pb);
                    }
                    tc::mma_commit(bar(B_ACC));
                }
                if (*abort_flag) break;
            }
            if (*abort_flag) {
                tc::mma_commit(bar(B_DRAIN));
                tc::mbar_poll(bar(B_DRAIN), 0u, tc::kSpinLimit);
            }
        }
    } else if (warp < G_FIRST) {
        // ------------------------------------------------------------ epilogue
        const int quarter = warp & 3;
        const int half = (warp - 2) >> 2;
        const int row = quarter * 32 + lane;
        const int sw = (row >> 1) & 3;
        uint32_t n = 0;
        unsigned char* Xsm = sm + OFF_X;
        float* part = reinterpret_cast<float*>(sm + OFF_PART);
        uint32_t tile_iter = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            float dot = 0.0f, dot1 = 0.0f;       // output-layer quarters: even / odd blocks
            bool ok = true;
            for (int l = 0; l < NLAYERS; ++l, ++n) {
                if (lane == 0) ok = tc::mbar_wait(bar(B_ACC), n & 1u, abort_flag);
                ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
                if (!ok) break;
                tc::tc_fence_after();
                const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (n & 1u) * 256u + 16u * half;
                const EpiArgs ea{Xsm, row, sw, half, lane, bar(B_BLK), a.bias + (size_t)l * NP, a.w3, a.scale, taddr};
                // four rounds of two 32-column blocks (the last has one); each ends with its
                // block pair's publication
                auto rounds = [&](auto kind) {
                    constexpr int K = decltype(kind)::value;
                    float v[32];
                    tc::tmem_ld16x2(taddr, v);
                    epi_blocks<F, K, 0, 2>(ea, v, dot, dot1, l);
                    tc::tmem_ld16x2(taddr + 64u, v);
                    epi_blocks<F, K, 2, 2>(ea, v, dot, dot1, l);
                    tc::tmem_ld16x2(taddr + 128u, v);
                    epi_blocks<F, K, 4, 2>(ea, v, dot, dot1, l);
                    float v1[16];
                    tc::tmem_ld16(taddr + 192u, v1);
                    epi_blocks<F, K, 6, 1>(ea, v1, dot, dot1, l);
                };
                if (l == 0) rounds(std::integral_constant<int, EPI_FIRST>{});
                else if (l == 21) rounds(std::integral_constant<int, EPI_LAST>{});
                else if (layer_keeps_o(l)) rounds(std::integral_constant<int, EPI_KEEP>{});
                else rounds(std::integral_constant<int, EPI_PLAIN>{});
            }
            if (!ok) break;
            // half 1 holds quarters 1 (even blocks) and 3 (odd), half 0 quarters 0 and 2
            if (half) {
                part[row] = dot;
                part[2 * TM + row] = dot1;
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(bar(B_PART));
            } else {
                if (!tc::mbar_wait(bar(B_PART), tile_iter & 1u, abort_flag)) break;
                const int64_t r = (int64_t)t * TM + row;
                if (r < Q) a.out[r] = out_from_quarters(dot, part[row], dot1, part[2 * TM + row], __ldg(a.w3 + NP - 1));
            }
            ++tile_iter;
        }
    } else {
        // ------------------------------------------------------------ gather
        const int gw = warp - G_FIRST;
        const int qg = gw & 3, wq = gw >> 2;        // 32-row query group, task phase
        const int row = qg * 32 + lane;
        const int sw = (row >> 1) & 3;
        const float4* packed = fa.v.packed;
        uint32_t sz = 0, pz = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
            const int64_t qi = (int64_t)t * TM + row;
            const bool valid = qi < Q;
            const int64_t qs = valid ? qi : 0;
            for (int k = 0; k < RPNN_K && ok; ++k) {
                // the frame is recomputed per level from the (cached) query, so only the
                // level's terms A, B, C, U0 stay live across its lookups
                float x[3], d[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) { x[c] = __ldg(fa.xs + 3 * qs + c); d[c] = __ldg(fa.ds + 3 * qs + c); }
                const Frame Fr = make_frame(d, fa.wl);
                const LevelK g = lk[k];
                float A[3], B[3], C[3], U0[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    A[c] = __fmul_rn(g.gk, Fr.ex[c]);
                    B[c] = __fmul_rn(g.gk, Fr.ey[c]);
                    C[c] = __fmul_rn(g.gk, Fr.ez[c]);
                    U0[c] = __fsub_rn(__fmul_rn(x[c], g.s), 0.5f);
                }
                const float gamma = Fr.gamma;
                const int cls = valid ? stencil_class(g.g0, A, B, C, U0) : kOutside;
                for (int st = 0; st < 4; ++st) {
                    // the ring slot is free once the MMAs of its previous contents completed
                    if (lane == 0) ok = tc::mbar_wait(bar(B_ZEMPTY + sz), pz ^ 1u, abort_flag);
                    ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
                    if (!ok) break;
                    unsigned char* slot = sm + OFF_Z + sz * Z_STAGE + row * 64;
                    const int ntask = st < 3 ? 8 : 6;       // stage 3 holds columns 192..239
                    for (int j = wq; j < ntask; j += 4) {
                        const int p0 = 64 * st + 8 * j;
                        uint4 q = make_uint4(0u, 0u, 0u, 0u);
                        if (p0 + 8 > RPNN_S) {
                            if (p0 < RPNN_S) q = gather_tail(packed, g.g0, ofs, A, B, C, U0, gamma, valid);
                        } else if (cls == kInside) {
                            q = gather_points<kInside>(packed, g.g0, ofs, p0, A, B, C, U0);
                        } else if (cls == kMixed) {
                            q = gather_points<kMixed>(packed, g.g0, ofs, p0, A, B, C, U0);
                        }
                        // column 8j of the stage: 32-column block j / 4, 16-byte unit j % 4
                        *reinterpret_cast<uint4*>(slot + (j >> 2) * BLK_A + (((j & 3) ^ sw) << 4)) = q;
                    }
                    tc::fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(bar(B_ZFULL + sz));
                    if (++sz == Z_STAGES) { sz = 0; pz ^= 1u; }
                }
            }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (*abort_flag && tid == 0) atomicOr(a.status, kStatTimeout);
    if (warp == 1) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, 512);
    }
}

}  // namespace

bool fused_supported(const VolumeView& vv) {
    for (int k = 0; k < RPNN_K; ++k)
        if (vv.mip_w[k] > 0.0f) return false;       // blended mip selection: unfused path
    return true;
}

// The render's descriptor + BF16 network stages in one launch: shading points xs / ds
// (q rows, or the device count q_dev with capacity q), light direction wl, predictions to
// out.  The BF16 weight image must be current (mlp_build_bf16_image).
rpnn_status fused_forward_bf16(Ctx& c, const VolumeView& vv, const float* xs, const float* ds, const float wl[3],
                               int64_t q, const int* q_dev, float* out, cudaStream_t s) {
    if (q <= 0) return RPNN_OK;
    if (!fused_supported(vv)) { set_error("fused render: blended mip selection is not fused"); return RPNN_ERR_UNSUPPORTED; }
    const ImageLayout I = image_layout<FmtBF16>();
    const unsigned char* b = c.wimg_bf16.as<unsigned char>();
    FusedArgs fa{};
    fa.net.img = b;
    fa.net.bias = reinterpret_cast<const float*>(b + I.bias_bytes_off);
    fa.net.w3 = reinterpret_cast<const float*>(b + I.w3_bytes_off);
    fa.net.scale = nullptr;
    for (int l = 0; l < NLAYERS; ++l) fa.net.img_off[l] = I.off[l];
    fa.net.q_host = q;
    fa.net.q_dev = q_dev;
    fa.net.out = out;
    fa.net.status = c.status.as<uint32_t>();
    fa.v = vv;
    fa.xs = xs;
    fa.ds = ds;
    for (int i = 0; i < 3; ++i) fa.wl[i] = wl[i];
    static bool attr = false;
    if (!attr) {
        RPNN_CUDA_TRY(cudaFuncSetAttribute(k_rpnn_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
        attr = true;
    }
    const int64_t ntiles = (q + TM - 1) / TM;
    const int grid = (int)std::min<int64_t>(ntiles, c.num_sms);
    k_rpnn_fused<<<grid, NTHREADS, SMEM_BYTES, s>>>(fa);
    RPNN_CHECK_LAUNCH();
    return RPNN_OK;
}

}  // namespace rpnn
