// tc_net.cuh -- pieces of the tcgen05 RPNN network kernels (Sec. 4.3, Fig. 6) shared by
// the network kernel that reads descriptor rows from global memory and the fused kernel
// that gathers them itself: tile geometry, operand formats, the per-layer K structure,
// the MMA issue loop of one layer and the epilogue of one layer.
//
// Operand layout in shared memory (K-major, 64-byte swizzle): blocks of 32 columns; in a
// block, row r occupies 64 bytes at r * 64 and its 16-byte unit j (columns 8j..8j+7)
// sits at unit j ^ ((r >> 1) & 3).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace rpnn {
namespace net {

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
constexpr uint32_t W_STAGE = 2 * BLK_B;                        // 26624
constexpr uint32_t Z_STAGE = 2 * BLK_A;                        // 16384
constexpr uint32_t BAR_STRIDE = 16;

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
    // training forward (k_rpnn_tc<FmtBF16, true>): every layer's ReLU output is also stored
    // FP32 and BF16, both transposed [slot][200][ldq], for the backward (slot: o^k at k - 1,
    // F1^k at 10 + k - 1, o^11 at 20, o^12 at 21)
    float* tsave;
    uint16_t* tsave_t;
    int64_t tq, tldq;
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
    uint32_t idesc, abort_addr, hi;
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
// ZCOMMIT: signal each consumed descriptor stage on its "empty" barrier (a kernel whose
// descriptor ring is refilled only after the weight ring proves the stage's MMAs done
// passes false and saves that commit).
// Activation byte c sits in 64-byte block c / 64 at half (c / 32) % 2; a stage reading
// bytes up to c waits for publication c / 128 of the previous epilogue (parity pb).
template <int W_STAGES, int Z_STAGES, bool FP8, int KB, int ZKB, bool RESID, bool ZCOMMIT = true>
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
            tc::mbar_wait_issuer2(S.wbar, S.pw, S.zbar, S.pz, tc::kSpinLimit, S.abort_addr);
        else if (need >= 0)
            tc::mbar_wait_issuer2(S.wbar, S.pw, pub, pb, tc::kSpinLimit, S.abort_addr);
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
            if (ZCOMMIT) tc::mma_commit(S.zbar + BAR_STRIDE * Z_STAGES);
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
    const float* bias;            // this layer's FP32 biases (BF16 renders: used by layer 0 only)
    const float* w3;              // output layer weights
    const float* scale;           // FP8 per-layer scales, or null
    uint32_t taddr;               // the warp's accumulator columns
    float* tf;                    // training forward: this row's column 0 of the transposed FP32 output, or null
    uint16_t* tt;                 // training forward: the same in the transposed BF16 output
    int64_t tldq;                 // their column pitch
    const float* tres;            // training forward: column 0 of this row's transposed FP32 residual o^{k-1}, or null
};

// KIND: EPI_PLAIN ReLU + BF16; EPI_KEEP also writes o^k back into the accumulator (the next
// second layer's start value); EPI_FIRST adds the FP32 bias (block 1's first layer, whose
// MMAs read no activation column); EPI_LAST is the output layer's ReLU and dot product.
// FP8: every kind dequantises, adds the FP32 bias and quantises its output (see the top).
// Blocks B0 .. B0 + NB - 1 of the layer, whose accumulator chunks the caller has loaded
// into v (chunk B0 + i at v[16 i ..]); epi_layer is the whole layer in one call.
// One 16-column chunk of one layer for the warp's 32 rows: columns 32 b + 16 half .. +15,
// accumulator values in w; u, qs, ku are the FP8 scales (1 for BF16).
// TRAIN (training forward, BF16): biases are FP32 and added here for every layer (the
// activation's padding column 200 stays 0), a second layer's residual is added here too
// (from e.tres, after the bias, as the GEMM form adds it; the accumulator starts at zero),
// and the ReLU output also goes to e.tf / e.tt.
template <class F, int KIND, bool TRAIN = false>
__device__ __forceinline__ void epi_chunk(const EpiArgs& e, int b, int half, float* w, float& dot, float u, float qs,
                                          float ku) {
    const int c0 = 32 * b + 16 * half;
    // accumulator columns 200..207 are exactly zero (zero weight rows and zero start
    // values), so ReLU needs no column mask
    if (c0 >= NP) return;
    if (F::FP8) {
#pragma unroll
        for (int i = 0; i < 16; ++i) w[i] *= u;
    }
    if (F::FP8 || KIND == EPI_FIRST || TRAIN) {
        const float4* b4 = reinterpret_cast<const float4*>(e.bias + c0);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 bb = __ldg(b4 + q);
            w[4 * q] += bb.x; w[4 * q + 1] += bb.y; w[4 * q + 2] += bb.z; w[4 * q + 3] += bb.w;
        }
    }
    if (TRAIN && e.tres) {
        // one column at a time: the warp's 32 rows are 128 contiguous bytes; all loads first
        float rr[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) rr[i] = c0 + i < RPNN_H ? e.tres[(int64_t)(c0 + i) * e.tldq] : 0.0f;
#pragma unroll
        for (int i = 0; i < 16; ++i)
            if (c0 + i < RPNN_H) w[i] += rr[i];
    }
    if (KIND == EPI_KEEP || KIND == EPI_LAST || TRAIN) {
#pragma unroll
        for (int i = 0; i < 16; ++i) w[i] = fmaxf(w[i], 0.0f);
    }
    if (TRAIN && e.tf) {
        // columns c0 .. c0 + 15 of the row, the 200 real ones, FP32 and BF16, both transposed
        // (a warp's 32 rows are 128 and 64 contiguous bytes per column)
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            if (c0 + i < RPNN_H) {
                e.tf[(int64_t)(c0 + i) * e.tldq] = w[i];
                e.tt[(int64_t)(c0 + i) * e.tldq] = __bfloat16_as_ushort(__float2bfloat16_rn(w[i]));
            }
        }
    }
    if (KIND == EPI_KEEP && !F::FP8 && !TRAIN) tc::tmem_st16(e.taddr + 32u * b + 16u * (half - e.half), w);
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
        *reinterpret_cast<uint4*>(rb + (((2 * (b & 1) + half) ^ e.sw) << 4)) = p;
        if (KIND == EPI_KEEP) {
            // o^k in the units of the next second layer's accumulator
#pragma unroll
            for (int i = 0; i < 16; ++i) w[i] *= ku;
            tc::tmem_st16(e.taddr + 32u * b + 16u * (half - e.half), w);
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
        if (!TRAIN && c0 == 192) u1[0] = (u1[0] & 0xFFFF0000u) | 0x3F80u;
        // 64-byte swizzled row: 16-byte unit u of row r at u ^ ((r >> 1) & 3)
        unsigned char* rb = e.X + b * BLK_A + e.row * 64;
        *reinterpret_cast<uint4*>(rb + (((2 * half) ^ e.sw) << 4)) = p0;
        *reinterpret_cast<uint4*>(rb + (((2 * half + 1) ^ e.sw) << 4)) = p1;
    }
}

// Publication p of a layer (activation bytes [128 p, 128 p + 128)) after the warp's stores:
// make them visible to the tensor core and, before the last one, complete the accumulator
// write-back (the MMAs that start from it wait for the last publication).
template <int KIND>
__device__ __forceinline__ void epi_publish(const EpiArgs& e, int p, bool last) {
    tc::fence_proxy_async_smem();
    if (last && KIND == EPI_KEEP) tc::tmem_wait_st();
    tc::tc_fence_before();
    __syncwarp();
    if (e.lane == 0) tc::mbar_arrive(e.blk_bar + BAR_STRIDE * (uint32_t)p);
}

template <class F> __device__ __forceinline__ float4 epi_scales(const EpiArgs& e, int l) {
    if (!F::FP8) return make_float4(1.0f, 1.0f, 1.0f, 0.0f);
    return __ldg(reinterpret_cast<const float4*>(e.scale) + l);
}

// Blocks B0 .. B0 + NB - 1 of the layer, whose accumulator chunks (column half e.half of
// each 32-column block) the caller has loaded into v (chunk B0 + i at v[16 i ..]),
// published as each 128-byte range of the activation is complete; epi_layer is the whole
// layer in one call.  The output layer's dot product runs as two FMA chains, over the
// even blocks (dot0) and the odd blocks (dot1), the column quarters of the sum below.
template <class F, int KIND, int B0, int NB, bool TRAIN = false>
__device__ __forceinline__ void epi_blocks(const EpiArgs& e, float (&v)[NB * 16], float& dot0, float& dot1, int l) {
    const float4 sc = epi_scales<F>(e, l);
#pragma unroll
    for (int b = B0; b < B0 + NB; ++b) {
        epi_chunk<F, KIND, TRAIN>(e, b, e.half, v + 16 * (b - B0), (b & 1) ? dot1 : dot0, sc.x, sc.y, sc.z);
        constexpr int CB = 32 * F::EB;                    // activation bytes of one block
        if (((b + 1) * CB) % SKB == 0 || b == NBLK - 1) epi_publish<KIND>(e, (b * CB) / SKB, b == NBLK - 1);
    }
}

template <class F, int KIND, bool TRAIN = false>
__device__ __forceinline__ void epi_layer(const EpiArgs& e, float (&v)[NBLK * 16], float& dot0, float& dot1, int l) {
    epi_blocks<F, KIND, 0, NBLK, TRAIN>(e, v, dot0, dot1, l);
}

// The prediction g = relu(T3 . o12 + bT3) from the column quarters' partial dot products:
// quarter q = 2 (block parity) + (half) holds the FMA chain over its 16-column chunks in
// increasing block order; g = relu(((q0 + q1) + (q2 + q3)) + bT3) in both network kernels.
__device__ __forceinline__ float out_from_quarters(float q0, float q1, float q2, float q3, float b) {
    return fmaxf(__fadd_rn(__fadd_rn(__fadd_rn(q0, q1), __fadd_rn(q2, q3)), b), 0.0f);
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

}  // namespace net
}  // namespace rpnn
