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
// Biases ride in the MMAs: activation column 200 (first padding column) holds 1.0 and the
// weight image carries each layer's bias in that column.  Only block 1's first layer,
// which reads no activation, adds its bias in the epilogue.
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

#include <cstdio>
#include <cstdlib>
#include <vector>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace rpnn {

namespace {

constexpr int TM = 128;                 // query rows per tile
constexpr int NP = 208;                 // padded layer width
constexpr int NLAYERS = 22;             // tensor-core layers
constexpr int KZ = 240;                 // padded descriptor level (226 used)
constexpr int SK = 64;                  // K columns per ring stage: four K = 16 MMAs
constexpr uint32_t BLK_A = TM * 64;     // 8192: 32 columns of 128 rows
constexpr uint32_t BLK_B = NP * 64;     // 13312: 32 columns of 208 rows
constexpr int NBLK = 7;                 // 32-column blocks of a 208-wide activation
constexpr int NPUB = 4;                 // epilogue publication points: blocks {0,1} {2,3} {4,5} {6}
constexpr int W_STAGES = 4, Z_STAGES = 3;
constexpr uint32_t W_STAGE = 2 * BLK_B;                        // 26624
constexpr uint32_t Z_STAGE = 2 * BLK_A;                        // 16384
constexpr uint32_t OFF_X = 0;
constexpr uint32_t OFF_W = OFF_X + NBLK * BLK_A;               // 57344
constexpr uint32_t OFF_Z = OFF_W + W_STAGES * W_STAGE;         // 163840
constexpr uint32_t OFF_BAR = OFF_Z + Z_STAGES * Z_STAGE;       // 212992
constexpr uint32_t BAR_STRIDE = 16;
constexpr int EPI_THREADS = 256;         // 8 epilogue warps
constexpr int EPI_WARPS = EPI_THREADS / 32;
constexpr int NTHREADS = 64 + EPI_THREADS;

// barrier slots from OFF_BAR, BAR_STRIDE bytes apart; B_DONE completes its phase 0 at
// setup and stands in for "nothing to wait for" in the issuer's three-barrier poll
enum {
    B_WFULL = 0, B_WEMPTY = B_WFULL + W_STAGES, B_ZFULL = B_WEMPTY + W_STAGES, B_ZEMPTY = B_ZFULL + Z_STAGES,
    B_ACC = B_ZEMPTY + Z_STAGES, B_BLK, B_PART = B_BLK + NPUB, B_DONE, B_COUNT
};
constexpr uint32_t OFF_TMEM_SLOT = OFF_BAR + BAR_STRIDE * B_COUNT;
constexpr uint32_t OFF_ABORT = OFF_TMEM_SLOT + 8;
constexpr uint32_t OFF_PART = OFF_ABORT + 8;                  // 128 floats
constexpr uint32_t SMEM_BYTES = OFF_PART + 128 * 4 + 64;
static_assert(OFF_W % 1024 == 0 && OFF_Z % 1024 == 0 && W_STAGE % 1024 == 0 && Z_STAGE % 1024 == 0,
              "swizzled operand blocks must stay 1024-byte aligned");
static_assert(SMEM_BYTES <= 232448, "shared memory over the per-block limit");

struct TcArgs {
    const __nv_bfloat16* img;   // weight image
    const float* bias;          // [NLAYERS][NP]
    const float* w3;            // [NP] output layer weights (zero padded), bias in [NP-1]
    int64_t img_off[NLAYERS];   // element offset of each layer's image
    int64_t q_host;
    const int* q_dev;
    float* out;
    uint32_t* status;
    unsigned long long* trace;  // optional per-block cycle counters (diagnostics), or null
};

// K extent of layer l: a block's first layer reads [z | o] (240 + 208 columns; block 0
// has no o), every other layer reads the 208-wide activation.
__host__ __device__ constexpr int layer_k(int l) {
    return l == 0 ? KZ : ((l < 20 && !(l & 1)) ? KZ + NP : NP);
}
// leading K columns of layer l that come from the descriptor tile
__host__ __device__ constexpr int layer_zk(int l) { return (l < 20 && !(l & 1)) ? KZ : 0; }
// 32-column blocks of layer l's weight image
__host__ __device__ constexpr int layer_blocks(int l) { return (layer_k(l) + 31) / 32; }
// second layers k >= 1 of a block add the residual o^{k-1}: their accumulator starts
// from it (written back by the epilogue of second layer k-1)
__host__ __device__ constexpr bool layer_resid(int l) { return (l & 1) && l >= 3 && l < 20; }
__host__ __device__ constexpr bool layer_keeps_o(int l) { return (l & 1) && l < 18; }

// two floats -> packed BF16 pair (lo in the low half), round to nearest even; the
// second form also clamps negatives to zero (ReLU)
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}
__device__ __forceinline__ uint32_t pack_relu_bf16x2(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

__global__ void __launch_bounds__(NTHREADS, 1)
k_rpnn_tc(const __grid_constant__ CUtensorMap zmap, const TcArgs a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t base = tc::smem_u32(sm);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + OFF_ABORT);
    auto bar = [&](int i) { return base + OFF_BAR + BAR_STRIDE * (uint32_t)i; };
    // diagnostics: cycles spent in each role's waits, when a.trace is set, and for block
    // 0 a timeline of 4 stamps per layer instance (MMA issue start/end, epilogue start/end)
    long long* tl = (a.trace && blockIdx.x == 0) ? reinterpret_cast<long long*>(a.trace + 1024 * 12) : nullptr;
    unsigned long long cyc_wait = 0, cyc_wait2 = 0;
    const long long cyc_start = clock64();
    auto twait = [&](uint32_t b, uint32_t parity, unsigned long long& acc) {
        const long long t0 = a.trace ? clock64() : 0;
        const bool r = tc::mbar_wait(b, parity, abort_flag);
        if (a.trace) acc += (unsigned long long)(clock64() - t0);
        return r;
    };
    const int64_t Q = a.q_dev ? (int64_t)*a.q_dev : a.q_host;
    const int ntiles = (int)((Q + TM - 1) / TM);

    if (tid == 0) {
        *abort_flag = (base & 1023u) ? 1 : 0;
        for (int s = 0; s < W_STAGES; ++s) { tc::mbar_init(bar(B_WFULL + s), 1); tc::mbar_init(bar(B_WEMPTY + s), 1); }
        for (int s = 0; s < Z_STAGES; ++s) { tc::mbar_init(bar(B_ZFULL + s), 1); tc::mbar_init(bar(B_ZEMPTY + s), 1); }
        tc::mbar_init(bar(B_ACC), 1);
        for (int b = 0; b < NPUB; ++b) tc::mbar_init(bar(B_BLK + b), EPI_WARPS);   // one arrival per warp
        tc::mbar_init(bar(B_PART), EPI_WARPS / 2);
        tc::mbar_init(bar(B_DONE), 1);
        tc::fence_mbar_init();
        tc::mbar_arrive(bar(B_DONE));
    }
    if (warp == 1) {
        tc::tmem_alloc(base + OFF_TMEM_SLOT, 512);
        tc::tmem_relinquish();
    }
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
            for (int t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x) {
                for (int l = 0; l < NLAYERS && !*abort_flag; ++l) {
                    const int K = layer_k(l), zk = layer_zk(l), nb = layer_blocks(l);
                    for (int k0 = 0; k0 < K; k0 += SK) {
                        if (k0 < zk) {
                            if (!twait(bar(B_ZEMPTY + sz), pz ^ 1u, cyc_wait)) break;
                            const uint32_t st = base + OFF_Z + sz * Z_STAGE;
                            const int x = (l / 2) * KZ + k0;    // level l/2, columns k0 .. k0+63
                            tc::mbar_expect_tx(bar(B_ZFULL + sz), Z_STAGE);
                            tc::tma_load_2d(st, &zmap, x, t * TM, bar(B_ZFULL + sz));
                            tc::tma_load_2d(st + BLK_A, &zmap, x + 32, t * TM, bar(B_ZFULL + sz));
                            if (++sz == Z_STAGES) { sz = 0; pz ^= 1u; }
                        }
                        const int b0 = k0 / 32;
                        const uint32_t bytes = (nb - b0 >= 2 ? 2u : 1u) * BLK_B;
                        if (!twait(bar(B_WEMPTY + sw), pw ^ 1u, cyc_wait)) break;
                        tc::mbar_expect_tx(bar(B_WFULL + sw), bytes);
                        tc::bulk_g2s(base + OFF_W + sw * W_STAGE, a.img + a.img_off[l] + (int64_t)b0 * (BLK_B / 2),
                                     bytes, bar(B_WFULL + sw));
                        if (++sw == W_STAGES) { sw = 0; pw ^= 1u; }
                    }
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        // No shared-memory load and no wait result may sit between MMAs in this thread
        // (each would stall behind the MMAs in flight): waits are output-free asm loops,
        // one per stage of four MMAs, covering the weight stage, the descriptor stage and
        // the activation block the stage needs; the abort flag is read once per tile.
        if (lane == 0 && !*abort_flag) {
            const uint32_t idesc = tc::idesc_bf16(TM, NP);
            const uint32_t abort_addr = base + OFF_ABORT;
            const uint32_t none = bar(B_DONE);
            const bool trace = a.trace != nullptr;
            // 64-bit operand descriptors are built once; an MMA only adds constants to them
            // (the start-address field counts 16-byte units: +2 = +32 bytes = 16 columns)
            const uint64_t d_W = tc::smem_desc_sw64(base + OFF_W);
            const uint64_t d_Z = tc::smem_desc_sw64(base + OFF_Z);
            const uint64_t d_X = tc::smem_desc_sw64(base + OFF_X);
            uint32_t n = 0;                          // layer instance
            uint32_t sw = 0, pw = 0, sz = 0, pz = 0; // ring positions and phases
            for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
                for (int l = 0; l < NLAYERS; ++l, ++n) {
                    const uint32_t acc = tmem + (n & 1u) * 256u;
                    if (tl && n < 512) tl[4 * n] = clock64();
                    // One tcgen05 fence per layer orders this layer's MMAs after the waits
                    // (in the previous layer) that saw epilogue n-2 finish with accumulator
                    // n % 2.  Operands written by TMA or by the epilogue (fence.proxy.async +
                    // mbarrier) need no tcgen05 fence.
                    tc::tc_fence_after();
                    const int K = layer_k(l), zk = layer_zk(l);
                    const uint32_t first_acc = layer_resid(l) ? 1u : 0u;
                    // Activation blocks 2p, 2p+1 of epilogue n-1 are published on B_BLK + p;
                    // the epilogue warps publish in order, so a completed publication also
                    // covers every block before it.
                    const uint32_t pb = (n - 1) & 1u;
                    int blk_ready = n > 0 ? -1 : NPUB - 1;
                    for (int k0 = 0; k0 < K; k0 += SK) {
                        const int k1 = min(K, k0 + SK);
                        const bool hz = k0 < zk;
                        const int need = k1 > zk ? (k1 - zk - 1) >> 6 : -1;    // publication
                        uint32_t b2 = none, p2 = 0;
                        if (need > blk_ready) { b2 = bar(B_BLK + need); p2 = pb; blk_ready = need; }
                        const long long tw = trace ? clock64() : 0;
                        tc::mbar_wait_issuer3(bar(B_WFULL + sw), pw, hz ? bar(B_ZFULL + sz) : none, hz ? pz : 0u, b2, p2,
                                              tc::kSpinLimit, abort_addr);
                        if (trace) cyc_wait += (unsigned long long)(clock64() - tw);
                        const uint64_t d_w = d_W + sw * (uint64_t)(W_STAGE >> 4);
                        const uint64_t d_z = d_Z + sz * (uint64_t)(Z_STAGE >> 4);
#pragma unroll
                        for (int j = 0; j < SK / 16; ++j) {
                            const int k = k0 + 16 * j;
                            if (k >= k1) break;
                            const uint64_t d_b = d_w + (uint64_t)(j >> 1) * (BLK_B >> 4) + (uint64_t)(j & 1) * 2u;
                            uint64_t d_a;
                            if (k < zk) d_a = d_z + (uint64_t)(j >> 1) * (BLK_A >> 4) + (uint64_t)(j & 1) * 2u;
                            else {
                                const int c = k - zk;              // column of the activation
                                d_a = d_X + (uint64_t)(c >> 5) * (BLK_A >> 4) + (uint64_t)((c >> 4) & 1) * 2u;
                            }
                            tc::mma_bf16(acc, d_a, d_b, idesc, k > 0 ? 1u : first_acc);
                        }
                        tc::mma_commit(bar(B_WEMPTY + sw));
                        if (++sw == W_STAGES) { sw = 0; pw ^= 1u; }
                        if (hz) {
                            tc::mma_commit(bar(B_ZEMPTY + sz));
                            if (++sz == Z_STAGES) { sz = 0; pz ^= 1u; }
                        }
                    }
                    // a layer that reads no activation (a tile's first) still waits for the
                    // previous epilogue, so the issuer never runs two phases ahead of it
                    if (blk_ready < NPUB - 1) {
                        const long long tb = trace ? clock64() : 0;
                        tc::mbar_wait_issuer(bar(B_BLK + NPUB - 1), pb, tc::kSpinLimit, abort_addr);
                        if (trace) cyc_wait2 += (unsigned long long)(clock64() - tb);
                    }
                    tc::mma_commit(bar(B_ACC));
                    if (tl && n < 512) tl[4 * n + 1] = clock64();
                }
                if (*abort_flag) break;
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue
        // 8 warps: warp w reads tensor-memory lanes 32*(w%4) .. +31 (its 32 query rows)
        // and, in every 32-column block b, the columns 32b + 16*half .. +15 (half = 0 for
        // warps 2-5, 1 for warps 6-9).  All 7 chunks are loaded in one round trip; each
        // finished block is published on its own barrier so the next layer's MMAs can
        // start on it while later blocks are still being written.
        const int quarter = warp & 3;
        const int half = (warp - 2) >> 2;
        const int row = quarter * 32 + lane;
        const int sw = (row >> 1) & 3;
        uint32_t n = 0;
        unsigned char* Xsm = sm + OFF_X;
        float* part = reinterpret_cast<float*>(sm + OFF_PART);     // [TM] partial dots
        uint32_t tile_iter = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            float dot = 0.0f;
            bool ok = true;
            for (int l = 0; l < NLAYERS; ++l, ++n) {
                // one poller per warp: lane 0 waits, the warp follows
                if (lane == 0) ok = twait(bar(B_ACC), n & 1u, cyc_wait);
                ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
                if (tl && n < 512 && warp == 2 && lane == 0) tl[4 * n + 2] = clock64();
                if (!ok) break;
                tc::tc_fence_after();
                const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (n & 1u) * 256u + 16u * half;
                float v[NBLK * 16];
                tc::tmem_ld16x7(taddr, v);
                const bool keep = layer_keeps_o(l);
#pragma unroll
                for (int b = 0; b < NBLK; ++b) {
                    const int c0 = 32 * b + 16 * half;
                    float* w = v + 16 * b;
                    // accumulator columns 200..207 are exactly zero (zero weight rows and
                    // zero start values), so ReLU needs no column mask
                    if (c0 < NP) {
                        if (l == 0) {
                            const float4* b4 = reinterpret_cast<const float4*>(a.bias + c0);
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                const float4 bb = __ldg(b4 + q);
                                w[4 * q] += bb.x; w[4 * q + 1] += bb.y; w[4 * q + 2] += bb.z; w[4 * q + 3] += bb.w;
                            }
                        }
                        if (keep || l == 21) {
#pragma unroll
                            for (int i = 0; i < 16; ++i) w[i] = fmaxf(w[i], 0.0f);
                        }
                        // o^k stays in the accumulator as the next second layer's start value
                        if (keep) tc::tmem_st16(taddr + 32u * b, w);
                        if (l == 21) {
                            const float4* w4 = reinterpret_cast<const float4*>(a.w3 + c0);
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                const float4 ww = __ldg(w4 + q);
                                dot = fmaf(w[4 * q], ww.x, dot); dot = fmaf(w[4 * q + 1], ww.y, dot);
                                dot = fmaf(w[4 * q + 2], ww.z, dot); dot = fmaf(w[4 * q + 3], ww.w, dot);
                            }
                        } else {
                            // BF16 pairs (ReLU folded into the conversion unless already applied)
                            uint4 p0, p1;
                            uint32_t* u0 = reinterpret_cast<uint32_t*>(&p0);
                            uint32_t* u1 = reinterpret_cast<uint32_t*>(&p1);
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                u0[q] = keep ? pack_bf16x2(w[2 * q], w[2 * q + 1]) : pack_relu_bf16x2(w[2 * q], w[2 * q + 1]);
                                u1[q] = keep ? pack_bf16x2(w[8 + 2 * q], w[9 + 2 * q])
                                             : pack_relu_bf16x2(w[8 + 2 * q], w[9 + 2 * q]);
                            }
                            // column 200 carries the constant 1 that multiplies the next layer's bias
                            if (b == NBLK - 1) u1[0] = (u1[0] & 0xFFFF0000u) | 0x3F80u;
                            // 64-byte swizzled row: 16-byte unit u of row r at u ^ ((r >> 1) & 3)
                            unsigned char* rb = Xsm + b * BLK_A + row * 64;
                            *reinterpret_cast<uint4*>(rb + (((2 * half) ^ sw) << 4)) = p0;
                            *reinterpret_cast<uint4*>(rb + (((2 * half + 1) ^ sw) << 4)) = p1;
                        }
                    }
                    if ((b & 1) || b == NBLK - 1) {
                        // publish blocks b-1, b: make the stores visible to the tensor core,
                        // and (last block) complete the accumulator write-back first, since
                        // the MMAs that start from it wait for the last publication
                        tc::fence_proxy_async_smem();
                        if (b == NBLK - 1 && keep) tc::tmem_wait_st();
                        tc::tc_fence_before();
                        __syncwarp();
                        if (lane == 0) tc::mbar_arrive(bar(B_BLK + (b >> 1)));
                    }
                }
                if (tl && n < 512 && warp == 2 && lane == 0) tl[4 * n + 3] = clock64();
            }
            if (!ok) break;
            // combine the two column halves of the output layer's dot product: the
            // second half publishes its partial sums, the first half adds them (bounded wait)
            if (half) {
                part[row] = dot;
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(bar(B_PART));
            } else {
                if (!tc::mbar_wait(bar(B_PART), tile_iter & 1u, abort_flag)) break;
                const int64_t r = (int64_t)t * TM + row;
                if (r < Q) a.out[r] = fmaxf(dot + part[row] + __ldg(a.w3 + NP - 1), 0.0f);
            }
            ++tile_iter;
        }
    }
    if (a.trace && lane == 0 && warp <= 2) {
        unsigned long long* tr = a.trace + (size_t)blockIdx.x * 12 + warp * 3;
        tr[0] = cyc_wait;
        tr[1] = cyc_wait2;
        tr[2] = (unsigned long long)(clock64() - cyc_start);
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
__global__ void k_build_image(const float* __restrict__ P, ParamLayout L, TcArgs a,
                              __nv_bfloat16* __restrict__ img, float* __restrict__ bias,
                              float* __restrict__ w3, int64_t total) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int l = NLAYERS - 1;
        while (l > 0 && a.img_off[l] > e) --l;
        // chunk of 32 columns: 208 rows of 64 bytes, 16-byte unit j of row n stored at
        // unit j ^ ((n >> 1) & 3) (the shared-memory image of a 64-byte swizzle)
        const int64_t r = e - a.img_off[l];
        const int chunk = (int)(r / (BLK_B / 2));
        const int rem = (int)(r % (BLK_B / 2));
        const int n = rem / 32, pos = rem % 32;
        const int c = chunk * 32 + (((pos / 8) ^ ((n >> 1) & 3)) * 8) + pos % 8;
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

struct ImageLayout {
    int64_t off[NLAYERS];
    int64_t img_elems;
    size_t bias_bytes_off, w3_bytes_off, total_bytes;
};

ImageLayout image_layout() {
    ImageLayout I{};
    int64_t o = 0;
    for (int l = 0; l < NLAYERS; ++l) {
        I.off[l] = o;
        o += (int64_t)layer_blocks(l) * (BLK_B / 2);
    }
    I.img_elems = o;
    I.bias_bytes_off = ((size_t)o * 2 + 255) & ~(size_t)255;
    I.w3_bytes_off = I.bias_bytes_off + (size_t)NLAYERS * NP * 4;
    I.total_bytes = I.w3_bytes_off + NP * 4 + 256;
    return I;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess)
            return (EncodeTiledFn) nullptr;
        return (EncodeTiledFn)p;
    }();
    return fn;
}

}  // namespace

rpnn_status mlp_build_bf16_image(Ctx& c, cudaStream_t s) {
    const ImageLayout I = image_layout();
    rpnn_status st = c.wimg_bf16.reserve(I.total_bytes);
    if (st) return st;
    TcArgs a{};
    for (int l = 0; l < NLAYERS; ++l) a.img_off[l] = I.off[l];
    unsigned char* b = c.wimg_bf16.as<unsigned char>();
    k_build_image<<<c.num_sms * 8, 256, 0, s>>>(c.params32.as<float>(), param_layout(), a,
                                                 reinterpret_cast<__nv_bfloat16*>(b),
                                                 reinterpret_cast<float*>(b + I.bias_bytes_off),
                                                 reinterpret_cast<float*>(b + I.w3_bytes_off), I.img_elems);
    RPNN_CHECK_LAUNCH();
    return RPNN_OK;
}

rpnn_status mlp_forward_bf16(Ctx& c, const void* desc_bf16, int64_t q, const int* q_dev, float* out,
                             cudaStream_t s) {
    if (q <= 0) return RPNN_OK;
    if ((reinterpret_cast<uintptr_t>(desc_bf16) & 15u) != 0) {
        set_error("descriptor rows must be 16-byte aligned");
        return RPNN_ERR_ARG;
    }
    EncodeTiledFn enc = encode_fn();
    if (!enc) { set_error("cuTensorMapEncodeTiled is unavailable"); return RPNN_ERR_UNSUPPORTED; }
    CUtensorMap zmap;
    const cuuint64_t dims[2] = {(cuuint64_t)RPNN_K * RPNN_DESC_STRIDE, (cuuint64_t)q};
    const cuuint64_t strides[1] = {(cuuint64_t)RPNN_K * RPNN_DESC_STRIDE * 2};
    const cuuint32_t box[2] = {32, TM};
    const cuuint32_t es[2] = {1, 1};
    CUresult r = enc(&zmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(desc_bf16), dims, strides, box,
                     es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) { set_error("cuTensorMapEncodeTiled failed (%d)", (int)r); return RPNN_ERR_CUDA; }
    const ImageLayout I = image_layout();
    unsigned char* b = c.wimg_bf16.as<unsigned char>();
    TcArgs a{};
    a.img = reinterpret_cast<const __nv_bfloat16*>(b);
    a.bias = reinterpret_cast<const float*>(b + I.bias_bytes_off);
    a.w3 = reinterpret_cast<const float*>(b + I.w3_bytes_off);
    for (int l = 0; l < NLAYERS; ++l) a.img_off[l] = I.off[l];
    a.q_host = q;
    a.q_dev = q_dev;
    a.out = out;
    a.status = c.status.as<uint32_t>();
    // RPNN_TC_TRACE=1: per-role wait cycles of every block, summarised on stderr
    // (synchronises the stream; diagnostics only)
    static unsigned long long* trace_buf = nullptr;
    const bool tracing = getenv("RPNN_TC_TRACE") != nullptr;
    if (tracing && !trace_buf) RPNN_CUDA_TRY(cudaMalloc(&trace_buf, (1024 * 12 + 4 * 512 + 128) * sizeof(unsigned long long)));
    a.trace = tracing ? trace_buf : nullptr;
    static bool attr = false;
    if (!attr) {
        RPNN_CUDA_TRY(cudaFuncSetAttribute(k_rpnn_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
        attr = true;
    }
    const int64_t ntiles = (q + TM - 1) / TM;
    const int grid = (int)std::min<int64_t>(ntiles, c.num_sms);
    if (tracing) RPNN_CUDA_TRY(cudaMemsetAsync(trace_buf, 0, (1024 * 12 + 4 * 512 + 128) * sizeof(unsigned long long), s));
    k_rpnn_tc<<<grid, NTHREADS, SMEM_BYTES, s>>>(zmap, a);
    RPNN_CHECK_LAUNCH();
    if (tracing) {
        std::vector<unsigned long long> h((size_t)grid * 12);
        RPNN_CUDA_TRY(cudaMemcpyAsync(h.data(), trace_buf, h.size() * 8, cudaMemcpyDeviceToHost, s));
        RPNN_CUDA_TRY(cudaStreamSynchronize(s));
        double acc[12] = {};
        for (int b = 0; b < grid; ++b)
            for (int i = 0; i < 12; ++i) acc[i] += (double)h[(size_t)b * 12 + i] / grid;
        fprintf(stderr,
                "[rpnn tc trace] blocks %d  producer: wait_empty %.0f of %.0f cyc | mma: stage polls %.0f "
                "end-of-layer waits %.0f of %.0f | epilogue(w2): wait_acc %.0f of %.0f\n",
                grid, acc[0], acc[2], acc[3], acc[4], acc[5], acc[6], acc[8]);
        std::vector<long long> tlh(4 * 512 + 128);
        RPNN_CUDA_TRY(cudaMemcpy(tlh.data(), trace_buf + 1024 * 12, tlh.size() * 8, cudaMemcpyDeviceToHost));
        // block 0, second tile: per layer, issue span, issue->acc ready, epilogue span, gap
        for (int n = 22; n < 44 && tlh[4 * n + 3]; ++n) {
            const long long* q = &tlh[4 * n];
            fprintf(stderr, "[rpnn tc timeline] layer %2d issue %6lld  to-acc %6lld  epi %6lld  next-issue-gap %6lld\n",
                    n - 22, q[1] - q[0], q[2] - q[0], q[3] - q[2], n < 511 ? q[4] - q[1] : 0LL);
        }
    }
    return RPNN_OK;
}

}  // namespace rpnn
