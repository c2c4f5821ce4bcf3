// mlp_tc.cu -- BF16 tensor-core (tcgen05) form of the RPNN forward (Sec. 4.3, Fig. 6).
//
// One persistent kernel runs all 22 matrix layers of the network for 128-query tiles:
//   block k:  F1 = relu([z^k | o^{k-1}] [V^k | W1^k]^T + b1)      (K = 240 + 208)
//             o^k = relu(F1 W2^T + b2 + o^{k-1})                   (K = 208)
//   standard: o11 = relu(o10 T1^T + bT1), o12 = relu(o11 T2^T + bT2)
//   output:   g = relu(T3 . o12 + bT3)  (CUDA cores, in the last epilogue)
// Widths are padded to N = 208 (zero rows) and the descriptor level to K = 240.
//
// Roles (320 threads): warp 0 streams operands through two rings -- weights (64 K-columns
// of the pre-arranged BF16 image per stage, one bulk copy) and, for a block's first layer,
// descriptor tiles (64 columns x 128 queries per stage, two 2-D TMA boxes); warp 1
// allocates tensor memory and one lane issues tcgen05.mma, four K = 16 steps per stage,
// into two alternating FP32 accumulators (so the descriptor part of a block's first layer
// overlaps the previous epilogue); warps 2-9 are the epilogue: tensor memory -> registers,
// ReLU, BF16 activations written back to shared memory for the next layer.
//
// BF16: biases ride in the MMAs: activation column 200 (first padding column) holds 1.0 and
// the weight image carries each layer's bias in that column.  Only block 1's first layer,
// which reads no activation, adds its bias in the epilogue.
//
// FP8 (E4M3, kind::f8f6f4, K = 32 per MMA): the same kernel with the same byte geometry
// (a ring stage is 128 bytes of K = 128 elements); per-tensor scales: the descriptor is
// stored unscaled, every layer's activation output o has a calibrated scale s (o = q s),
// and each layer's weights are quantised so that accumulator units u are common to both
// parts of a block's first layer ([z | o] against [V | W1]).  The epilogue dequantises (x u),
// adds the FP32 bias, applies ReLU and re-quantises (/ s); the residual is kept in the
// accumulator in that layer's units (/ u of the next second layer).
//
// One activation buffer X serves every layer: a layer's epilogue starts only after all
// of that layer's MMAs (the readers of X) have completed.  The residual o^{k-1} of a
// block's second layer therefore cannot stay in X; the previous second layer's epilogue
// writes o^{k-1} (FP32) back into its accumulator instead, and the next second layer
// accumulates onto it.
//
// Operand layout in shared memory (K-major, 64-byte swizzle): blocks of 32 columns; in a
// block, row r occupies 64 bytes at r * 64 and its 16-byte unit j (columns 8j..8j+7)
// sits at unit j ^ ((r >> 1) & 3).  The weight image in global memory is stored in
// exactly this form, and descriptor tiles arrive as 64-byte-swizzled TMA boxes.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "tc_net.cuh"
#include "tc_ptx.cuh"
#include "tmap.h"

namespace rpnn {

namespace {

using namespace net;

constexpr int W_STAGES = 4, Z_STAGES = 4;
constexpr uint32_t OFF_X = 0;
constexpr uint32_t OFF_W = OFF_X + NBLK * BLK_A;               // 57344
constexpr uint32_t OFF_Z = OFF_W + W_STAGES * W_STAGE;         // 163840
constexpr uint32_t OFF_BAR = OFF_Z + Z_STAGES * Z_STAGE;       // 229376
constexpr int EPI_WARPS = 8;
constexpr int NTHREADS = 64 + 32 * EPI_WARPS;

// barrier slots from OFF_BAR, BAR_STRIDE bytes apart
enum {
    B_WFULL = 0, B_WEMPTY = B_WFULL + W_STAGES, B_ZFULL = B_WEMPTY + W_STAGES,
    B_ACC = B_ZFULL + Z_STAGES, B_BLK, B_PART = B_BLK + NPUB_MAX, B_DRAIN, B_COUNT
};
// a descriptor slot is reused 8 or 11 stages after its reader (a first layer's z stages,
// then the 4 stages of layer 1 or of the block's second layer and the first layer's x
// stages); the weight ring proves stages at least W_STAGES + 1 back complete
static_assert(W_STAGES + 1 <= 8 && Z_STAGES == 4, "descriptor slot reuse needs the weight ring's ordering");
constexpr uint32_t OFF_TMEM_SLOT = OFF_BAR + BAR_STRIDE * B_COUNT;
constexpr uint32_t OFF_ABORT = OFF_TMEM_SLOT + 8;
constexpr uint32_t OFF_PART = OFF_ABORT + 8;                  // 3 x 128 floats
constexpr uint32_t SMEM_BYTES = OFF_PART + 3 * 128 * 4 + 64;
static_assert(OFF_W % 1024 == 0 && OFF_Z % 1024 == 0 && W_STAGE % 1024 == 0 && Z_STAGE % 1024 == 0,
              "swizzled operand blocks must stay 1024-byte aligned");
static_assert(SMEM_BYTES <= 232448, "shared memory over the per-block limit");

// TRAIN: the training forward (BF16): FP32 biases in the epilogue, every layer's output
// stored for the backward (TcArgs::tsave), no padding-column bias trick.
template <class F, bool TRAIN>
__global__ void __launch_bounds__(NTHREADS, 1)
k_rpnn_tc(const __grid_constant__ CUtensorMap zmap, const TcArgs a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t base = tc::smem_u32(sm);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + OFF_ABORT);
    auto bar = [&](int i) { return base + OFF_BAR + BAR_STRIDE * (uint32_t)i; };
    auto twait = [&](uint32_t b, uint32_t parity) { return tc::mbar_wait(b, parity, abort_flag); };
    const int64_t Q = a.q_dev ? (int64_t)*a.q_dev : a.q_host;
    const int ntiles = (int)((Q + TM - 1) / TM);

    if (tid == 0) {
        *abort_flag = (base & 1023u) ? 1 : 0;
        for (int s = 0; s < W_STAGES; ++s) { tc::mbar_init(bar(B_WFULL + s), 1); tc::mbar_init(bar(B_WEMPTY + s), 1); }
        for (int s = 0; s < Z_STAGES; ++s) tc::mbar_init(bar(B_ZFULL + s), 1);
        tc::mbar_init(bar(B_ACC), 1);
        for (int b = 0; b < npub<F>(); ++b) tc::mbar_init(bar(B_BLK + b), EPI_WARPS);   // one arrival per warp
        tc::mbar_init(bar(B_PART), EPI_WARPS / 2);
        tc::mbar_init(bar(B_DRAIN), 1);
        tc::fence_mbar_init();
    }
    if (warp == 1) {
        tc::tmem_alloc(base + OFF_TMEM_SLOT, 512);
        tc::tmem_relinquish();
    }
    // the activation buffer starts zeroed: padding bytes an MMA reads but no epilogue writes
    // (FP8: activation bytes 208..223) must hold finite values
    for (int i = tid; i < (int)(NBLK * BLK_A / 16); i += NTHREADS) reinterpret_cast<uint4*>(sm + OFF_X)[i] = make_uint4(0, 0, 0, 0);
    tc::fence_proxy_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(sm + OFF_TMEM_SLOT);

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        // Stages are filled in the order the issuer consumes them; ring positions and
        // phases live in registers.
        if (lane == 0 && !*abort_flag) {
            uint32_t sw = 0, pw = 0, sz = 0, pz = 0;
            uint32_t wfills = 0, zfills = 0;
            for (int t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x) {
                for (int l = 0; l < NLAYERS && !*abort_flag; ++l) {
                    const int KB = layer_kb<F>(l), zkb = layer_zkb<F>(l), nb = layer_blocks<F>(l);
                    for (int k0 = 0; k0 < KB; k0 += SKB) {
                        if (k0 < zkb) {
                            // No wait for the slot: its previous reader is the same stage of
                            // the previous block's first layer (tile's first layer: the previous
                            // tile's last), at least 8 stages back, and the weight fill just
                            // before this point waited for the MMAs of the stage W_STAGES + 1
                            // back to complete (MMAs complete in issue order).
                            const uint32_t st = base + OFF_Z + sz * Z_STAGE;
                            // level l/2, bytes k0 .. k0+127 as two boxes of 64 bytes (x in elements)
                            const int x = ((l / 2) * F::KZB + k0) / F::EB;
                            tc::mbar_expect_tx(bar(B_ZFULL + sz), Z_STAGE);
                            tc::tma_load_2d(st, &zmap, x, t * TM, bar(B_ZFULL + sz));
                            tc::tma_load_2d(st + BLK_A, &zmap, x + 64 / F::EB, t * TM, bar(B_ZFULL + sz));
                            ++zfills;
                            if (++sz == Z_STAGES) { sz = 0; pz ^= 1u; }
                        }
                        const int b0 = k0 / 64;
                        const uint32_t bytes = (nb - b0 >= 2 ? 2u : 1u) * BLK_B;
                        if (!twait(bar(B_WEMPTY + sw), pw ^ 1u)) break;
                        tc::mbar_expect_tx(bar(B_WFULL + sw), bytes);
                        tc::bulk_g2s(base + OFF_W + sw * W_STAGE, a.img + a.img_off[l] + (int64_t)b0 * BLK_B, bytes,
                                     bar(B_WFULL + sw));
                        ++wfills;
                        if (++sw == W_STAGES) { sw = 0; pw ^= 1u; }
                    }
                }
            }
            if (*abort_flag) {
                // drain: wait (bounded) for this thread's copies still in flight, i.e. for
                // the latest fill of every ring slot to have landed
                for (uint32_t s2 = 0; s2 < W_STAGES && s2 < wfills; ++s2)
                    tc::mbar_poll(bar(B_WFULL + s2), ((wfills - 1 - s2) / W_STAGES) & 1u, tc::kSpinLimit);
                for (uint32_t s2 = 0; s2 < Z_STAGES && s2 < zfills; ++s2)
                    tc::mbar_poll(bar(B_ZFULL + s2), ((zfills - 1 - s2) / Z_STAGES) & 1u, tc::kSpinLimit);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        // No shared-memory load and no wait result may sit between MMAs in this thread
        // (each would stall behind the MMAs in flight): waits are output-free asm loops,
        // one per stage of four MMAs, covering the weight stage, the descriptor stage and
        // the activation block the stage needs; the abort flag is read once per tile.
        // Each layer kind is issued by a fully unrolled routine, so every descriptor
        // offset, accumulate flag and wait shape is a compile-time constant: the thread
        // spends its time in waits and MMAs, not in address arithmetic.
        if (lane == 0 && !*abort_flag) {
            IssueState S;
            S.idesc = F::FP8 ? tc::idesc_e4m3(TM, NP) : tc::idesc_bf16(TM, NP);
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
            uint32_t n = 0;                          // layer instance
            for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
                for (int l = 0; l < NLAYERS; ++l, ++n) {
                    const uint32_t acc = tmem + (uint32_t)(l & 1) * 256u;   // n and l share parity
                    // One tcgen05 fence per layer orders this layer's MMAs after the waits
                    // (in the previous layer) that saw epilogue n-2 finish with accumulator
                    // n % 2.  Operands written by TMA or by the epilogue (fence.proxy.async +
                    // mbarrier) need no tcgen05 fence.
                    tc::tc_fence_after();
                    // publication parity of epilogue n-1: n and l share parity
                    const uint32_t pb = (uint32_t)(l & 1) ^ 1u;
                    if (l == 0) {
                        issue_layer<W_STAGES, Z_STAGES, F::FP8, F::KZB, F::KZB, false, false>(S, acc, pb);
                        // a tile's first layer reads no activation; it still waits for the
                        // previous epilogue, so the issuer never runs two phases ahead of it
                        if (n > 0)
                            tc::mbar_wait_issuer(S.blk0 + BAR_STRIDE * (npub<F>() - 1), pb, tc::kSpinLimit, S.abort_addr);
                    } else if (l < 20 && !(l & 1)) {
                        issue_layer<W_STAGES, Z_STAGES, F::FP8, F::KZB + F::XB, F::KZB, false, false>(S, acc, pb);
                    } else if (layer_resid(l) && !TRAIN) {
                        // (the training form adds the residual in its epilogue)
                        issue_layer<W_STAGES, Z_STAGES, F::FP8, F::XB, 0, true>(S, acc, pb);
                    } else {
                        issue_layer<W_STAGES, Z_STAGES, F::FP8, F::XB, 0, false>(S, acc, pb);
                    }
                    tc::mma_commit(bar(B_ACC));
                }
                if (*abort_flag) break;
            }
            if (*abort_flag) {
                // drain: wait (bounded) for the MMAs in flight before tensor memory is freed
                tc::mma_commit(bar(B_DRAIN));
                tc::mbar_poll(bar(B_DRAIN), 0u, tc::kSpinLimit);
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue
        // 8 warps: warp w reads tensor-memory lanes 32*(w%4) .. +31 (its 32 query rows)
        // and, in every 32-column block b, the columns 32b + 16*half .. +15 (half = 0 for
        // warps 2-5, 1 for warps 6-9).  All 7 chunks are loaded in one round trip; each
        // finished block pair is published on its own barrier so the next layer's MMAs can
        // start on it while later blocks are still being written.
        // The E4M3 and training forms read a different FP32 bias row in every layer's
        // epilogue; fetched from L2 there, each row's first use would sit on the layer chain.
        // The table (22 x 208 floats, 18 KB) and the E4M3 scales go to L1 once, here.
        if (F::FP8 || TRAIN) {
            const int et = tid - 64;
            for (int i = et; i < (int)(NLAYERS * NP * 4 / 128); i += 32 * EPI_WARPS)
                asm volatile("prefetch.global.L1 [%0];" ::"l"(a.bias + 32 * i));
            if (F::FP8 && et < (int)(NLAYERS * 16 + 127) / 128)
                asm volatile("prefetch.global.L1 [%0];" ::"l"(a.scale + 32 * et));
        }
        const int quarter = warp & 3;
        const int half = (warp - 2) >> 2;
        const int row = quarter * 32 + lane;
        const int sw = (row >> 1) & 3;
        uint32_t n = 0;
        unsigned char* Xsm = sm + OFF_X;
        float* part = reinterpret_cast<float*>(sm + OFF_PART);     // [3][TM] partial dots
        uint32_t tile_iter = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            float dot = 0.0f, dot1 = 0.0f;      // output-layer quarters: even / odd blocks
            bool ok = true;
            for (int l = 0; l < NLAYERS; ++l, ++n) {
                // one poller per warp: lane 0 waits, the warp follows
                if (lane == 0) ok = twait(bar(B_ACC), n & 1u);
                ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
                if (!ok) break;
                tc::tc_fence_after();
                const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (n & 1u) * 256u + 16u * half;
                float v[NBLK * 16];
                tc::tmem_ld16x7(taddr, v);
                // the FP32 bias row of layer l (BF16 renders add it only for layer 0; the E4M3
                // and training forms for every layer)
                EpiArgs ea{Xsm, row, sw, half, lane, bar(B_BLK), a.bias + (size_t)l * NP, a.w3, a.scale, taddr};
                if (TRAIN) {
                    const int64_t r = (int64_t)t * TM + row;
                    // saved slot of layer l: F1^k (l = 2k - 2) at 10 + k - 1, o^k (l = 2k - 1)
                    // at k - 1, o^11 and o^12 at 20 and 21
                    const int slot = l >= 20 ? l : ((l & 1) ? (l >> 1) : 10 + (l >> 1));
                    if (r < Q) {
                        // both copies transposed [slot][200][ldq]: column j of row r at j * ldq
                        ea.tf = a.tsave + (int64_t)slot * RPNN_H * a.tldq + r;
                        ea.tt = a.tsave_t + (int64_t)slot * RPNN_H * a.tldq + r;
                        ea.tldq = a.tldq;
                        // second layers k >= 2 add o^{k-1} (slot k - 2), which this thread
                        // stored two layers earlier
                        if (layer_resid(l)) ea.tres = a.tsave + (int64_t)((l >> 1) - 1) * RPNN_H * a.tldq + r;
                    }
                }
                // one straight-line routine per layer kind
                if (l == 0) epi_layer<F, EPI_FIRST, TRAIN>(ea, v, dot, dot1, l);
                else if (l == 21) epi_layer<F, EPI_LAST, TRAIN>(ea, v, dot, dot1, l);
                else if (layer_keeps_o(l)) epi_layer<F, EPI_KEEP, TRAIN>(ea, v, dot, dot1, l);
                else epi_layer<F, EPI_PLAIN, TRAIN>(ea, v, dot, dot1, l);
            }
            if (!ok) break;
            // combine the column quarters' partial dot products of the output layer: half 1
            // holds quarters 1 (even blocks) and 3 (odd), half 0 quarters 0 and 2 and adds
            // them in the fixed order (bounded wait)
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
    }
    tc::tc_fence_before();
    __syncthreads();
    if (*abort_flag && tid == 0) atomicOr(a.status, kStatTimeout);
    if (warp == 1) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, 512);
    }
}

// BF16 weight image, FP32 bias table and output layer from the FP32 parameters.
// img_off holds byte offsets; element e of the image is byte 2e.
__global__ void k_build_image(const float* __restrict__ P, ParamLayout L, TcArgs a,
                              __nv_bfloat16* __restrict__ img, float* __restrict__ bias,
                              float* __restrict__ w3, int64_t total) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int l = NLAYERS - 1;
        while (l > 0 && a.img_off[l] > 2 * e) --l;
        // block of 32 columns: 208 rows of 64 bytes, 16-byte unit j of row n stored at
        // unit j ^ ((n >> 1) & 3) (the shared-memory image of a 64-byte swizzle)
        const int64_t r = e - a.img_off[l] / 2;
        const int chunk = (int)(r / (BLK_B / 2));
        const int rem = (int)(r % (BLK_B / 2));
        const int n = rem / 32, pos = rem % 32;
        const int c = chunk * 32 + (((pos / 8) ^ ((n >> 1) & 3)) * 8) + pos % 8;
        constexpr int KZ = FmtBF16::KZB / 2;
        // layers l >= 1 read the activation, whose column 200 is the constant 1: the
        // image holds the layer's bias in that column
        float v = 0.0f;
        if (n < RPNN_H) {
            if (l < 20 && !(l & 1)) {
                const int k = l / 2;
                if (c < RPNN_DIN) v = P[L.V[k] + (int64_t)n * RPNN_DIN + c];
                else if (c >= KZ && c < KZ + RPNN_H) v = P[L.W1[k] + (int64_t)n * RPNN_H + (c - KZ)];
                else if (c == KZ + RPNN_H && l > 0) v = P[L.b1[k] + n];
            } else if (c < RPNN_H) {
                const int64_t off = l < 20 ? L.W2[l / 2] : L.T[l - 20];
                v = P[off + (int64_t)n * RPNN_H + c];
            } else if (c == RPNN_H) {
                v = P[(l < 20 ? L.b2[l / 2] : L.bT[l - 20]) + n];
            }
        }
        img[e] = __float2bfloat16_rn(v);
    }
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (tid < NLAYERS * NP) {
        const int l = (int)(tid / NP), n = (int)(tid % NP);
        float v = 0.0f;
        if (n < RPNN_H) {
            if (l < 20) v = P[((l & 1) ? L.b2[l / 2] : L.b1[l / 2]) + n];
            else v = P[L.bT[l - 20] + n];
        }
        bias[tid] = v;
    }
    // output layer weights, zero padded; the output bias rides in the last slot
    if (tid < NP) w3[tid] = tid < RPNN_H ? P[L.T[2] + tid] : (tid == NP - 1 ? P[L.bT[2]] : 0.0f);
}

// Quantisation factors of the E4M3 image: layer l's descriptor weights (V) are scaled by
// fz[l] and its activation weights (W1, W2, T) by fx[l] before rounding to E4M3.
struct Fp8Factors {
    float fz[NLAYERS], fx[NLAYERS];
};

// E4M3 weight image (same 64-byte-block layout as the BF16 image, one byte per element);
// the FP32 bias table and output layer as for BF16.
__global__ void k_build_image_e4m3(const float* __restrict__ P, ParamLayout L, TcArgs a, Fp8Factors f,
                                   unsigned char* __restrict__ img, float* __restrict__ bias,
                                   float* __restrict__ w3, int64_t total) {
    constexpr int KZ = FmtE4M3::KZB;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int l = NLAYERS - 1;
        while (l > 0 && a.img_off[l] > e) --l;
        const int64_t r = e - a.img_off[l];
        const int chunk = (int)(r / BLK_B);
        const int rem = (int)(r % BLK_B);
        const int n = rem / 64, pos = rem % 64;
        const int c = chunk * 64 + (((pos / 16) ^ ((n >> 1) & 3)) * 16) + pos % 16;
        float v = 0.0f;
        if (n < RPNN_H) {
            if (l < 20 && !(l & 1)) {
                const int k = l / 2;
                if (c < RPNN_DIN) v = P[L.V[k] + (int64_t)n * RPNN_DIN + c] * f.fz[l];
                else if (c >= KZ && c < KZ + RPNN_H) v = P[L.W1[k] + (int64_t)n * RPNN_H + (c - KZ)] * f.fx[l];
            } else if (c < RPNN_H) {
                const int64_t off = l < 20 ? L.W2[l / 2] : L.T[l - 20];
                v = P[off + (int64_t)n * RPNN_H + c] * f.fx[l];
            }
        }
        const __nv_fp8_e4m3 q(v);
        img[e] = *reinterpret_cast<const unsigned char*>(&q);
    }
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (tid < NLAYERS * NP) {
        const int l = (int)(tid / NP), n = (int)(tid % NP);
        float v = 0.0f;
        if (n < RPNN_H) {
            if (l < 20) v = P[((l & 1) ? L.b2[l / 2] : L.b1[l / 2]) + n];
            else v = P[L.bT[l - 20] + n];
        }
        bias[tid] = v;
    }
    if (tid < NP) w3[tid] = tid < RPNN_H ? P[L.T[2] + tid] : (tid == NP - 1 ? P[L.bT[2]] : 0.0f);
}

// largest value of each [q][200] activation slot (non-negative after ReLU: the float bits
// order like the values)
__global__ void k_slot_max(const float* __restrict__ saved, int64_t q, int nslots, unsigned* __restrict__ out) {
    const int slot = blockIdx.y;
    if (slot >= nslots) return;
    const float* x = saved + (size_t)slot * q * RPNN_H;
    unsigned m = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < q * RPNN_H; i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, __float_as_uint(fmaxf(x[i], 0.0f)));
    for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out + slot, m);
}

// Launch of the network kernel in format F on q descriptor rows (q_dev: device count, or
// null).
// TRAIN: tsave / tsave_t / ldq receive the saved activations (TcArgs::tsave).
template <class F, bool TRAIN = false>
rpnn_status forward_tc(Ctx& c, const DevBuf& image, const void* desc, int64_t q, const int* q_dev, float* out,
                       cudaStream_t s, float* tsave = nullptr, uint16_t* tsave_t = nullptr, int64_t ldq = 0) {
    if (q <= 0) return RPNN_OK;
    if ((reinterpret_cast<uintptr_t>(desc) & 15u) != 0) {
        set_error("descriptor rows must be 16-byte aligned");
        return RPNN_ERR_ARG;
    }
    EncodeTiledFn enc = encode_fn();
    if (!enc) { set_error("cuTensorMapEncodeTiled is unavailable"); return RPNN_ERR_UNSUPPORTED; }
    CUtensorMap zmap;
    const cuuint64_t row_elems = (cuuint64_t)RPNN_K * (F::KZB / F::EB);
    const cuuint64_t dims[2] = {row_elems, (cuuint64_t)q};
    const cuuint64_t strides[1] = {row_elems * F::EB};
    const cuuint32_t box[2] = {(cuuint32_t)(64 / F::EB), TM};
    const cuuint32_t es[2] = {1, 1};
    CUresult r = enc(&zmap, F::FP8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                     const_cast<void*>(desc), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) { set_error("cuTensorMapEncodeTiled failed (%d)", (int)r); return RPNN_ERR_CUDA; }
    const ImageLayout I = image_layout<F>();
    const unsigned char* b = image.as<unsigned char>();
    TcArgs a{};
    a.img = b;
    a.bias = reinterpret_cast<const float*>(b + I.bias_bytes_off);
    a.w3 = reinterpret_cast<const float*>(b + I.w3_bytes_off);
    a.scale = F::FP8 ? reinterpret_cast<const float*>(b + I.scale_bytes_off) : nullptr;
    for (int l = 0; l < NLAYERS; ++l) a.img_off[l] = I.off[l];
    a.q_host = q;
    a.q_dev = q_dev;
    a.out = out;
    a.status = c.status.as<uint32_t>();
    a.tsave = tsave;
    a.tsave_t = tsave_t;
    a.tq = q;
    a.tldq = ldq;
    static bool attr = false;
    if (!attr) {
        RPNN_CUDA_TRY(cudaFuncSetAttribute(k_rpnn_tc<F, TRAIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
        attr = true;
    }
    const int64_t ntiles = (q + TM - 1) / TM;
    const int grid = (int)std::min<int64_t>(ntiles, c.num_sms);
    k_rpnn_tc<F, TRAIN><<<grid, NTHREADS, SMEM_BYTES, s>>>(zmap, a);
    RPNN_CHECK_LAUNCH();
    return RPNN_OK;
}

}  // namespace

rpnn_status mlp_build_bf16_image(Ctx& c, cudaStream_t s) {
    const ImageLayout I = image_layout<FmtBF16>();
    rpnn_status st = c.wimg_bf16.reserve(I.total_bytes);
    if (st) return st;
    TcArgs a{};
    for (int l = 0; l < NLAYERS; ++l) a.img_off[l] = I.off[l];
    unsigned char* b = c.wimg_bf16.as<unsigned char>();
    k_build_image<<<c.num_sms * 8, 256, 0, s>>>(c.params32.as<float>(), param_layout(), a,
                                                 reinterpret_cast<__nv_bfloat16*>(b),
                                                 reinterpret_cast<float*>(b + I.bias_bytes_off),
                                                 reinterpret_cast<float*>(b + I.w3_bytes_off), I.img_bytes / 2);
    RPNN_CHECK_LAUNCH();
    return RPNN_OK;
}

rpnn_status mlp_forward_bf16(Ctx& c, const void* desc_bf16, int64_t q, const int* q_dev, float* out,
                             cudaStream_t s) {
    return forward_tc<FmtBF16>(c, c.wimg_bf16, desc_bf16, q, q_dev, out, s);
}

rpnn_status mlp_forward_bf16_saving(Ctx& c, const void* desc_bf16, int64_t q, float* out, float* saved,
                                    uint16_t* saved_t, int64_t ldq, cudaStream_t s) {
    if (q <= 0) return RPNN_OK;
    return forward_tc<FmtBF16, true>(c, c.wimg_bf16, desc_bf16, q, nullptr, out, s, saved, saved_t, ldq);
}

rpnn_status mlp_forward_fp8(Ctx& c, const void* desc_fp8, int64_t q, const int* q_dev, float* out, cudaStream_t s) {
    if (!c.fp8_ready) { set_error("FP8 network: rpnn_calibrate_fp8 has not run since the weights were set"); return RPNN_ERR_STATE; }
    return forward_tc<FmtE4M3>(c, c.wimg_fp8, desc_fp8, q, q_dev, out, s);
}

// Per-tensor FP8 scales for the network of Sec. 4.3: the activation scale of each layer's
// output from its largest value over the calibration descriptors (FP32 network), the
// weight factors so that both parts of a block's first layer share accumulator units, and
// the E4M3 weight image.
rpnn_status mlp_calibrate_fp8(Ctx& c, const float* desc, int64_t q, cudaStream_t s) {
    if (q <= 0) { set_error("calibration needs at least one descriptor"); return RPNN_ERR_ARG; }
    const size_t per_row = mlp_saved_floats_per_row();
    rpnn_status st = c.t_saved.reserve((size_t)q * per_row * sizeof(float));
    if (!st) st = c.t_out.reserve((size_t)q * sizeof(float));
    if (!st) st = c.t_loss.reserve(32 * sizeof(unsigned));
    if (st) return st;
    st = mlp_forward_f32(c, desc, q, nullptr, c.t_out.as<float>(), c.t_saved.as<float>(), s);
    if (st) return st;
    unsigned* mx = c.t_loss.as<unsigned>();
    RPNN_CUDA_TRY(cudaMemsetAsync(mx, 0, 32 * sizeof(unsigned), s));
    k_slot_max<<<dim3(64, 21), 256, 0, s>>>(c.t_saved.as<float>(), q, 21, mx);
    RPNN_CUDA_TRY(cudaGetLastError());
    unsigned hmx[21];
    RPNN_CUDA_TRY(cudaMemcpyAsync(hmx, mx, sizeof hmx, cudaMemcpyDeviceToHost, s));
    std::vector<float> P((size_t)RPNN_NPARAMS);
    RPNN_CUDA_TRY(cudaMemcpyAsync(P.data(), c.params32.p, P.size() * sizeof(float), cudaMemcpyDeviceToHost, s));
    RPNN_CUDA_TRY(cudaStreamSynchronize(s));
    const ParamLayout& L = param_layout();
    auto maxabs = [&](int64_t off, int64_t n) {
        double m = 0.0;
        for (int64_t i = 0; i < n; ++i) m = std::max(m, (double)std::fabs(P[off + i]));
        return m;
    };
    // activation output scales: layer l's output is slot 10 + l/2 (first layers), (l-1)/2
    // (second layers), 20 (first standard layer); E4M3 reaches 448
    double s_out[NLAYERS] = {};
    for (int l = 0; l <= 20; ++l) {
        const int slot = l == 20 ? 20 : ((l & 1) ? (l - 1) / 2 : 10 + l / 2);
        float m;
        std::memcpy(&m, &hmx[slot], 4);
        s_out[l] = (m > 0.0f ? (double)m : 1.0) / 448.0;
    }
    const double s_z = 1.0;                  // descriptor values are stored unscaled
    Fp8Factors f{};
    float table[NLAYERS][4] = {};
    double u[NLAYERS] = {};
    for (int l = 0; l < NLAYERS; ++l) {
        const double s_in = l > 0 ? s_out[l - 1] : 1.0;
        double uz = 0.0, ux = 0.0;
        if (l < 20 && !(l & 1)) {
            const int k = l / 2;
            uz = s_z * maxabs(L.V[k], (int64_t)RPNN_H * RPNN_DIN) / 448.0;
            if (l > 0) ux = s_in * maxabs(L.W1[k], (int64_t)RPNN_H * RPNN_H) / 448.0;
        } else {
            const int64_t off = l < 20 ? L.W2[l / 2] : L.T[l - 20];
            ux = s_in * maxabs(off, (int64_t)RPNN_H * RPNN_H) / 448.0;
        }
        u[l] = std::max(std::max(uz, ux), 1e-30);
        f.fz[l] = (float)(s_z / u[l]);
        f.fx[l] = (float)(s_in / u[l]);
    }
    for (int l = 0; l < NLAYERS; ++l) {
        table[l][0] = (float)u[l];
        table[l][1] = l <= 20 ? (float)(1.0 / s_out[l]) : 1.0f;
        table[l][2] = (layer_keeps_o(l) && l + 2 < NLAYERS) ? (float)(1.0 / u[l + 2]) : 1.0f;
    }
    const ImageLayout I = image_layout<FmtE4M3>();
    st = c.wimg_fp8.reserve(I.total_bytes);
    if (st) return st;
    TcArgs a{};
    for (int l = 0; l < NLAYERS; ++l) a.img_off[l] = I.off[l];
    unsigned char* b = c.wimg_fp8.as<unsigned char>();
    k_build_image_e4m3<<<c.num_sms * 8, 256, 0, s>>>(c.params32.as<float>(), L, a, f, b,
                                                      reinterpret_cast<float*>(b + I.bias_bytes_off),
                                                      reinterpret_cast<float*>(b + I.w3_bytes_off), I.img_bytes);
    RPNN_CHECK_LAUNCH();
    RPNN_CUDA_TRY(cudaMemcpyAsync(b + I.scale_bytes_off, table, sizeof table, cudaMemcpyHostToDevice, s));
    RPNN_CUDA_TRY(cudaStreamSynchronize(s));
    c.fp8_ready = true;
    ++c.epoch;
    return RPNN_OK;
}

}  // namespace rpnn
