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
#include "tc_ptx.cuh"
#include "tmap.h"

namespace rpnn {

namespace {

constexpr int TM = 128;                 // query rows per tile
constexpr int NP = 208;                 // padded layer width
constexpr int NLAYERS = 22;             // tensor-core layers
constexpr int SKB = 128;                // K bytes per ring stage: four MMAs of 32 bytes
constexpr uint32_t BLK_A = TM * 64;     // 8192: 64 bytes of K for 128 rows
constexpr uint32_t BLK_B = NP * 64;     // 13312: 64 bytes of K for 208 rows
constexpr int NBLK = 7;                 // 32-column accumulator chunks of a 208-wide layer
constexpr int NPUB_MAX = 4;             // epilogue publications per layer (one per 128 bytes)

// Operand formats.  KZB: bytes of one descriptor level an MMA reads (226 values, padded to
// whole 32-byte K-steps); XB: bytes of the activation an MMA reads (208 values, padded).
struct FmtBF16 {
    static constexpr bool FP8 = false;
    static constexpr int EB = 2, KZB = 480, XB = 416;
};
struct FmtE4M3 {
    static constexpr bool FP8 = true;
    static constexpr int EB = 1, KZB = 256, XB = 224;
};
template <class F> __host__ __device__ constexpr int npub() { return (F::XB + SKB - 1) / SKB; }
constexpr int W_STAGES = 4, Z_STAGES = 4;
constexpr uint32_t W_STAGE = 2 * BLK_B;                        // 26624
constexpr uint32_t Z_STAGE = 2 * BLK_A;                        // 16384
constexpr uint32_t OFF_X = 0;
constexpr uint32_t OFF_W = OFF_X + NBLK * BLK_A;               // 57344
constexpr uint32_t OFF_Z = OFF_W + W_STAGES * W_STAGE;         // 163840
constexpr uint32_t OFF_BAR = OFF_Z + Z_STAGES * Z_STAGE;       // 229376
constexpr uint32_t BAR_STRIDE = 16;
constexpr int EPI_THREADS = 256;         // 8 epilogue warps
constexpr int EPI_WARPS = EPI_THREADS / 32;
constexpr int NTHREADS = 64 + EPI_THREADS;

// barrier slots from OFF_BAR, BAR_STRIDE bytes apart; B_DONE completes its phase 0 at
// setup and stands in for "nothing to wait for" in the issuer's three-barrier poll
enum {
    B_WFULL = 0, B_WEMPTY = B_WFULL + W_STAGES, B_ZFULL = B_WEMPTY + W_STAGES, B_ZEMPTY = B_ZFULL + Z_STAGES,
    B_ACC = B_ZEMPTY + Z_STAGES, B_BLK, B_PART = B_BLK + NPUB_MAX, B_DONE, B_DRAIN, B_COUNT
};
constexpr uint32_t OFF_TMEM_SLOT = OFF_BAR + BAR_STRIDE * B_COUNT;
constexpr uint32_t OFF_ABORT = OFF_TMEM_SLOT + 8;
constexpr uint32_t OFF_PART = OFF_ABORT + 8;                  // 128 floats
constexpr uint32_t SMEM_BYTES = OFF_PART + 128 * 4 + 64;
static_assert(OFF_W % 1024 == 0 && OFF_Z % 1024 == 0 && W_STAGE % 1024 == 0 && Z_STAGE % 1024 == 0,
              "swizzled operand blocks must stay 1024-byte aligned");
static_assert(SMEM_BYTES <= 232448, "shared memory over the per-block limit");

struct TcArgs {
    const unsigned char* img;   // weight image
    const float* bias;          // [NLAYERS][NP]
    const float* w3;            // [NP] output layer weights (zero padded), bias in [NP-1]
    const float* scale;         // FP8: [NLAYERS] x {u, 1/s_out, 1/u of layer l+2, 0}; BF16: null
    int64_t img_off[NLAYERS];   // byte offset of each layer's image
    int64_t q_host;
    const int* q_dev;
    float* out;
    uint32_t* status;
};

// K bytes of layer l: a block's first layer reads [z | o] (block 1 has no o), every other
// layer reads the 208-wide activation.
template <class F> __host__ __device__ constexpr int layer_kb(int l) {
    return l == 0 ? F::KZB : ((l < 20 && !(l & 1)) ? F::KZB + F::XB : F::XB);
}
// leading K bytes of layer l that come from the descriptor tile
template <class F> __host__ __device__ constexpr int layer_zkb(int l) { return (l < 20 && !(l & 1)) ? F::KZB : 0; }
// 64-byte blocks of layer l's weight image
template <class F> __host__ __device__ constexpr int layer_blocks(int l) { return (layer_kb<F>(l) + 63) / 64; }
// second layers k >= 1 of a block add the residual o^{k-1}: their accumulator starts
// from it (written back by the epilogue of second layer k-1)
__host__ __device__ constexpr bool layer_resid(int l) { return (l & 1) && l >= 3 && l < 20; }
__host__ __device__ constexpr bool layer_keeps_o(int l) { return (l & 1) && l < 18; }

// Issue state of the MMA thread: the low 32 bits of the current weight / descriptor stage
// operand descriptors (start address in 16-byte units) and of the activation buffer, the
// common high word, the current ring barriers, positions and phases.
struct IssueState {
    uint32_t idesc, abort_addr, none, hi;
    uint32_t w0, z0, x0, w, z;
    uint32_t wbar0, zbar0, wbar, zbar, blk0;
    uint32_t sw, pw, sz, pz;
};

// D[acc] (+)= A * B^T with operand descriptors given as low words and a common high word;
// `accumulate` is a constant at every call site (the two forms differ only in the flag).
#define RPNN_MMA_LOHI(KIND, PRED)                                                            \
    asm volatile("{\n .reg .b64 da, db;\n .reg .pred p;\n"                                 \
                 " mov.b64 da, {%1, %3};\n mov.b64 db, {%2, %3};\n " PRED "\n"            \
                 " tcgen05.mma.cta_group::1." KIND " [%0], da, db, %4, p;\n}\n"             \
                 ::"r"(acc), "r"(a_lo), "r"(b_lo), "r"(hi), "r"(idesc) : "memory")
template <bool FP8>
__device__ __forceinline__ void mma_lohi(uint32_t acc, uint32_t a_lo, uint32_t b_lo, uint32_t hi, uint32_t idesc,
                                         bool accumulate) {
    if (FP8) {
        if (accumulate) RPNN_MMA_LOHI("kind::f8f6f4", "setp.eq.u32 p, 0, 0;");
        else RPNN_MMA_LOHI("kind::f8f6f4", "setp.ne.u32 p, 0, 0;");
    } else {
        if (accumulate) RPNN_MMA_LOHI("kind::f16", "setp.eq.u32 p, 0, 0;");
        else RPNN_MMA_LOHI("kind::f16", "setp.ne.u32 p, 0, 0;");
    }
}
#undef RPNN_MMA_LOHI

// One layer of KB bytes of K, the first ZKB of them from the descriptor ring, in stages of
// 128 bytes (four MMAs of 32 bytes).  RESID: the accumulator already holds o^{k-1}.
// Activation byte c sits in 64-byte block c / 64 at half (c / 32) % 2; a stage reading
// bytes up to c waits for publication c / 128 of the previous epilogue (parity pb).
template <bool FP8, int KB, int ZKB, bool RESID>
__device__ __forceinline__ void issue_layer(IssueState& S, uint32_t acc, uint32_t pb) {
#pragma unroll
    for (int k0 = 0; k0 < KB; k0 += SKB) {
        const int k1 = k0 + SKB < KB ? k0 + SKB : KB;
        const bool hz = k0 < ZKB;
        const int need = k1 > ZKB ? (k1 - ZKB - 1) >> 7 : -1;
        const uint32_t pub = S.blk0 + BAR_STRIDE * (uint32_t)(need < 0 ? 0 : need);
        if (hz && need >= 0)
            tc::mbar_wait_issuer3(S.wbar, S.pw, S.zbar, S.pz, pub, pb, tc::kSpinLimit, S.abort_addr);
        else if (hz)
            tc::mbar_wait_issuer3(S.wbar, S.pw, S.zbar, S.pz, S.none, 0u, tc::kSpinLimit, S.abort_addr);
        else if (need >= 0)
            tc::mbar_wait_issuer3(S.wbar, S.pw, pub, pb, S.none, 0u, tc::kSpinLimit, S.abort_addr);
        else
            tc::mbar_wait_issuer(S.wbar, S.pw, tc::kSpinLimit, S.abort_addr);
#pragma unroll
        for (int j = 0; j < SKB / 32; ++j) {
            const int k = k0 + 32 * j;
            if (k < k1) {
                const uint32_t b = S.w + (uint32_t)((j >> 1) * (BLK_B >> 4) + (j & 1) * 2);
                const int c = k - ZKB;
                const uint32_t a = k < ZKB ? S.z + (uint32_t)((j >> 1) * (BLK_A >> 4) + (j & 1) * 2)
                                           : S.x0 + (uint32_t)((c >> 6) * (BLK_A >> 4) + ((c >> 5) & 1) * 2);
                mma_lohi<FP8>(acc, a, b, S.hi, S.idesc, k > 0 || RESID);
            }
        }
        tc::mma_commit(S.wbar + BAR_STRIDE * W_STAGES);          // this stage's "empty" barrier
        if (++S.sw == W_STAGES) { S.sw = 0; S.pw ^= 1u; S.w = S.w0; S.wbar = S.wbar0; }
        else { S.w += W_STAGE >> 4; S.wbar += BAR_STRIDE; }
        if (hz) {
            tc::mma_commit(S.zbar + BAR_STRIDE * Z_STAGES);
            if (++S.sz == Z_STAGES) { S.sz = 0; S.pz ^= 1u; S.z = S.z0; S.zbar = S.zbar0; }
            else { S.z += Z_STAGE >> 4; S.zbar += BAR_STRIDE; }
        }
    }
}

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
// four floats -> four E4M3 bytes (round to nearest even, saturating at +-448, ReLU)
__device__ __forceinline__ uint32_t pack_relu_e4m3x4(float a0, float a1, float a2, float a3) {
    uint16_t lo, hi;
    asm("cvt.rn.satfinite.relu.e4m3x2.f32 %0, %1, %2;" : "=h"(lo) : "f"(a1), "f"(a0));
    asm("cvt.rn.satfinite.relu.e4m3x2.f32 %0, %1, %2;" : "=h"(hi) : "f"(a3), "f"(a2));
    return (uint32_t)lo | ((uint32_t)hi << 16);
}

// Epilogue of one layer for one warp: 16 columns of each 32-column block for the warp's
// 32 rows (already loaded from tensor memory into v), published in block pairs.
enum { EPI_PLAIN = 0, EPI_KEEP = 1, EPI_FIRST = 2, EPI_LAST = 3 };
struct EpiArgs {
    unsigned char* X;
    int row, sw, half, lane;
    uint32_t blk_bar;             // publication barrier 0 (the others follow at BAR_STRIDE)
    const float* bias;            // FP32 bias table (BF16: block 1's first layer only)
    const float* w3;              // output layer weights
    const float* scale;           // FP8 per-layer scales, or null
    uint32_t taddr;               // the warp's accumulator columns
};

// KIND: EPI_PLAIN ReLU + BF16; EPI_KEEP also writes o^k back into the accumulator (the next
// second layer's start value); EPI_FIRST adds the FP32 bias (block 1's first layer, whose
// MMAs read no activation column); EPI_LAST is the output layer's ReLU and dot product.
// FP8: every kind dequantises, adds the FP32 bias and quantises its output (see the top).
template <class F, int KIND>
__device__ __forceinline__ void epi_layer(const EpiArgs& e, float (&v)[NBLK * 16], float& dot, int l) {
    float u = 1.0f, qs = 1.0f, ku = 1.0f;
    if (F::FP8) {
        const float4 sc = __ldg(reinterpret_cast<const float4*>(e.scale) + l);
        u = sc.x; qs = sc.y; ku = sc.z;
    }
#pragma unroll
    for (int b = 0; b < NBLK; ++b) {
        const int c0 = 32 * b + 16 * e.half;
        float* w = v + 16 * b;
        // accumulator columns 200..207 are exactly zero (zero weight rows and zero start
        // values), so ReLU needs no column mask
        if (c0 < NP) {
            if (F::FP8) {
#pragma unroll
                for (int i = 0; i < 16; ++i) w[i] *= u;
            }
            if (F::FP8 || KIND == EPI_FIRST) {
                const float4* b4 = reinterpret_cast<const float4*>(e.bias + c0);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 bb = __ldg(b4 + q);
                    w[4 * q] += bb.x; w[4 * q + 1] += bb.y; w[4 * q + 2] += bb.z; w[4 * q + 3] += bb.w;
                }
            }
            if (KIND == EPI_KEEP || KIND == EPI_LAST) {
#pragma unroll
                for (int i = 0; i < 16; ++i) w[i] = fmaxf(w[i], 0.0f);
            }
            if (KIND == EPI_KEEP && !F::FP8) tc::tmem_st16(e.taddr + 32u * b, w);
            if (KIND == EPI_LAST) {
                const float4* w4 = reinterpret_cast<const float4*>(e.w3 + c0);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 ww = __ldg(w4 + q);
                    dot = fmaf(w[4 * q], ww.x, dot); dot = fmaf(w[4 * q + 1], ww.y, dot);
                    dot = fmaf(w[4 * q + 2], ww.z, dot); dot = fmaf(w[4 * q + 3], ww.w, dot);
                }
            } else if (F::FP8) {
                // 16 E4M3 bytes: byte c of the row's activation at 64-byte block c / 64,
                // 16-byte unit (c % 64) / 16, swizzled like the BF16 layout
                uint4 p;
                p.x = pack_relu_e4m3x4(w[0] * qs, w[1] * qs, w[2] * qs, w[3] * qs);
                p.y = pack_relu_e4m3x4(w[4] * qs, w[5] * qs, w[6] * qs, w[7] * qs);
                p.z = pack_relu_e4m3x4(w[8] * qs, w[9] * qs, w[10] * qs, w[11] * qs);
                p.w = pack_relu_e4m3x4(w[12] * qs, w[13] * qs, w[14] * qs, w[15] * qs);
                unsigned char* rb = e.X + (b >> 1) * BLK_A + e.row * 64;
                *reinterpret_cast<uint4*>(rb + (((2 * (b & 1) + e.half) ^ e.sw) << 4)) = p;
                if (KIND == EPI_KEEP) {
                    // o^k in the units of the next second layer's accumulator
#pragma unroll
                    for (int i = 0; i < 16; ++i) w[i] *= ku;
                    tc::tmem_st16(e.taddr + 32u * b, w);
                }
            } else {
                // BF16 pairs (ReLU folded into the conversion unless already applied)
                uint4 p0, p1;
                uint32_t* u0 = reinterpret_cast<uint32_t*>(&p0);
                uint32_t* u1 = reinterpret_cast<uint32_t*>(&p1);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (KIND == EPI_KEEP) {
                        u0[q] = pack_bf16x2(w[2 * q], w[2 * q + 1]);
                        u1[q] = pack_bf16x2(w[8 + 2 * q], w[9 + 2 * q]);
                    } else {
                        u0[q] = pack_relu_bf16x2(w[2 * q], w[2 * q + 1]);
                        u1[q] = pack_relu_bf16x2(w[8 + 2 * q], w[9 + 2 * q]);
                    }
                }
                // column 200 carries the constant 1 that multiplies the next layer's bias
                if (b == NBLK - 1) u1[0] = (u1[0] & 0xFFFF0000u) | 0x3F80u;
                // 64-byte swizzled row: 16-byte unit u of row r at u ^ ((r >> 1) & 3)
                unsigned char* rb = e.X + b * BLK_A + e.row * 64;
                *reinterpret_cast<uint4*>(rb + (((2 * e.half) ^ e.sw) << 4)) = p0;
                *reinterpret_cast<uint4*>(rb + (((2 * e.half + 1) ^ e.sw) << 4)) = p1;
            }
        }
        // publication p covers activation bytes [128 p, 128 p + 128): after chunk b when
        // the chunk ends such a range, or is the last
        constexpr int CB = 32 * F::EB;                    // activation bytes of one chunk
        if (((b + 1) * CB) % SKB == 0 || b == NBLK - 1) {
            const int p = (b * CB) / SKB;
            // make the stores visible to the tensor core, and (last chunk) complete the
            // accumulator write-back first, since the MMAs that start from it wait for the
            // last publication
            tc::fence_proxy_async_smem();
            if (b == NBLK - 1 && KIND == EPI_KEEP) tc::tmem_wait_st();
            tc::tc_fence_before();
            __syncwarp();
            if (e.lane == 0) tc::mbar_arrive(e.blk_bar + BAR_STRIDE * (uint32_t)p);
        }
    }
}

template <class F>
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
        for (int s = 0; s < Z_STAGES; ++s) { tc::mbar_init(bar(B_ZFULL + s), 1); tc::mbar_init(bar(B_ZEMPTY + s), 1); }
        tc::mbar_init(bar(B_ACC), 1);
        for (int b = 0; b < npub<F>(); ++b) tc::mbar_init(bar(B_BLK + b), EPI_WARPS);   // one arrival per warp
        tc::mbar_init(bar(B_PART), EPI_WARPS / 2);
        tc::mbar_init(bar(B_DONE), 1);
        tc::mbar_init(bar(B_DRAIN), 1);
        tc::fence_mbar_init();
        tc::mbar_arrive(bar(B_DONE));
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
                            if (!twait(bar(B_ZEMPTY + sz), pz ^ 1u)) break;
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
            S.none = bar(B_DONE);
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
                        issue_layer<F::FP8, F::KZB, F::KZB, false>(S, acc, pb);
                        // a tile's first layer reads no activation; it still waits for the
                        // previous epilogue, so the issuer never runs two phases ahead of it
                        if (n > 0)
                            tc::mbar_wait_issuer(S.blk0 + BAR_STRIDE * (npub<F>() - 1), pb, tc::kSpinLimit, S.abort_addr);
                    } else if (l < 20 && !(l & 1)) {
                        issue_layer<F::FP8, F::KZB + F::XB, F::KZB, false>(S, acc, pb);
                    } else if (layer_resid(l)) {
                        issue_layer<F::FP8, F::XB, 0, true>(S, acc, pb);
                    } else {
                        issue_layer<F::FP8, F::XB, 0, false>(S, acc, pb);
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
                if (lane == 0) ok = twait(bar(B_ACC), n & 1u);
                ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
                if (!ok) break;
                tc::tc_fence_after();
                const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (n & 1u) * 256u + 16u * half;
                float v[NBLK * 16];
                tc::tmem_ld16x7(taddr, v);
                const EpiArgs ea{Xsm, row, sw, half, lane, bar(B_BLK), a.bias, a.w3, a.scale, taddr};
                // one straight-line routine per layer kind
                if (l == 0) epi_layer<F, EPI_FIRST>(ea, v, dot, l);
                else if (l == 21) epi_layer<F, EPI_LAST>(ea, v, dot, l);
                else if (layer_keeps_o(l)) epi_layer<F, EPI_KEEP>(ea, v, dot, l);
                else epi_layer<F, EPI_PLAIN>(ea, v, dot, l);
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

// Byte layout of a weight image: per layer its 64-byte blocks (208 rows each), then the
// FP32 bias table [NLAYERS][NP], the output layer [NP] and the FP8 scale table [NLAYERS][4].
struct ImageLayout {
    int64_t off[NLAYERS];
    int64_t img_bytes;
    size_t bias_bytes_off, w3_bytes_off, scale_bytes_off, total_bytes;
};

template <class F>
ImageLayout image_layout() {
    ImageLayout I{};
    int64_t o = 0;
    for (int l = 0; l < NLAYERS; ++l) {
        I.off[l] = o;
        o += (int64_t)layer_blocks<F>(l) * BLK_B;
    }
    I.img_bytes = o;
    I.bias_bytes_off = ((size_t)o + 255) & ~(size_t)255;
    I.w3_bytes_off = I.bias_bytes_off + (size_t)NLAYERS * NP * 4;
    I.scale_bytes_off = (I.w3_bytes_off + NP * 4 + 255) & ~(size_t)255;
    I.total_bytes = I.scale_bytes_off + NLAYERS * 16 + 256;
    return I;
}

// Launch of the network kernel in format F on q descriptor rows (q_dev: device count, or
// null).
template <class F>
rpnn_status forward_tc(Ctx& c, const DevBuf& image, const void* desc, int64_t q, const int* q_dev, float* out,
                       cudaStream_t s) {
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
    static bool attr = false;
    if (!attr) {
        RPNN_CUDA_TRY(cudaFuncSetAttribute(k_rpnn_tc<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
        attr = true;
    }
    const int64_t ntiles = (q + TM - 1) / TM;
    const int grid = (int)std::min<int64_t>(ntiles, c.num_sms);
    k_rpnn_tc<F><<<grid, NTHREADS, SMEM_BYTES, s>>>(zmap, a);
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
