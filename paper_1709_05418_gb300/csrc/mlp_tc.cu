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
    B_ACC = B_ZEMPTY + Z_STAGES, B_BLK, B_PART = B_BLK + NPUB, B_DONE, B_DRAIN, B_COUNT
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

// Issue state of the MMA thread: the low 32 bits of the current weight / descriptor stage
// operand descriptors (start address in 16-byte units) and of the activation buffer, the
// common high word, the current ring barriers, positions and phases.
struct IssueState {
    uint32_t idesc, abort_addr, none, hi;
    uint32_t w0, z0, x0, w, z;
    uint32_t wbar0, zbar0, wbar, zbar, blk0;
    uint32_t sw, pw, sz, pz;
    long long* tr;       // timeline base (block 0, diagnostics) or null
    long long* stamp;    // per-stage stamps of this layer instance, or null
    unsigned long long cyc;
};

// D[acc] (+)= A * B^T with operand descriptors given as low words and a common high word;
// `accumulate` is a constant at every call site (the two forms differ only in the flag).
__device__ __forceinline__ void mma_lohi(uint32_t acc, uint32_t a_lo, uint32_t b_lo, uint32_t hi, uint32_t idesc,
                                         bool accumulate) {
    if (accumulate)
        asm volatile(
            "{\n .reg .b64 da, db;\n .reg .pred p;\n"
            " mov.b64 da, {%1, %3};\n mov.b64 db, {%2, %3};\n setp.eq.u32 p, 0, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], da, db, %4, p;\n}\n"
            ::"r"(acc), "r"(a_lo), "r"(b_lo), "r"(hi), "r"(idesc) : "memory");
    else
        asm volatile(
            "{\n .reg .b64 da, db;\n .reg .pred p;\n"
            " mov.b64 da, {%1, %3};\n mov.b64 db, {%2, %3};\n setp.ne.u32 p, 0, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], da, db, %4, p;\n}\n"
            ::"r"(acc), "r"(a_lo), "r"(b_lo), "r"(hi), "r"(idesc) : "memory");
}

// One layer of K columns, the first ZK of them from the descriptor ring, in stages of 64
// columns (four K = 16 MMAs).  RESID: the accumulator already holds o^{k-1}.  Activation
// column c sits in 32-column block c / 32 at half (c / 16) % 2; a stage reading columns
// up to c waits for publication c / 64 of the previous epilogue (phase parity pb).
template <bool TRACE, int K, int ZK, bool RESID>
__device__ __forceinline__ void issue_layer(IssueState& S, uint32_t acc, uint32_t pb) {
#pragma unroll
    for (int k0 = 0; k0 < K; k0 += SK) {
        const int k1 = k0 + SK < K ? k0 + SK : K;
        const bool hz = k0 < ZK;
        const int need = k1 > ZK ? (k1 - ZK - 1) >> 6 : -1;
        const uint32_t pub = S.blk0 + BAR_STRIDE * (uint32_t)(need < 0 ? 0 : need);
        long long t0 = 0;
        if (TRACE) {
            t0 = clock64();
            if (S.stamp) S.stamp[(k0 / SK) * 3] = t0;
        }
        if (hz && need >= 0)
            tc::mbar_wait_issuer3(S.wbar, S.pw, S.zbar, S.pz, pub, pb, tc::kSpinLimit, S.abort_addr);
        else if (hz)
            tc::mbar_wait_issuer3(S.wbar, S.pw, S.zbar, S.pz, S.none, 0u, tc::kSpinLimit, S.abort_addr);
        else if (need >= 0)
            tc::mbar_wait_issuer3(S.wbar, S.pw, pub, pb, S.none, 0u, tc::kSpinLimit, S.abort_addr);
        else
            tc::mbar_wait_issuer(S.wbar, S.pw, tc::kSpinLimit, S.abort_addr);
        if (TRACE) {
            const long long t1 = clock64();
            S.cyc += (unsigned long long)(t1 - t0);
            if (S.stamp) S.stamp[(k0 / SK) * 3 + 1] = t1;
        }
#pragma unroll
        for (int j = 0; j < SK / 16; ++j) {
            const int k = k0 + 16 * j;
            if (k < k1) {
                const uint32_t b = S.w + (uint32_t)((j >> 1) * (BLK_B >> 4) + (j & 1) * 2);
                const int c = k - ZK;
                const uint32_t a = k < ZK ? S.z + (uint32_t)((j >> 1) * (BLK_A >> 4) + (j & 1) * 2)
                                          : S.x0 + (uint32_t)((c >> 5) * (BLK_A >> 4) + ((c >> 4) & 1) * 2);
                mma_lohi(acc, a, b, S.hi, S.idesc, k > 0 || RESID);
            }
        }
        tc::mma_commit(S.wbar + BAR_STRIDE * W_STAGES);          // this stage's "empty" barrier
        if (TRACE && S.stamp) S.stamp[(k0 / SK) * 3 + 2] = clock64();
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

// Epilogue of one layer for one warp: 16 columns of each 32-column block for the warp's
// 32 rows (already loaded from tensor memory into v), published in block pairs.
enum { EPI_PLAIN = 0, EPI_KEEP = 1, EPI_FIRST = 2, EPI_LAST = 3 };
struct EpiArgs {
    unsigned char* X;
    int row, sw, half, lane;
    uint32_t blk_bar;             // publication barrier 0 (the others follow at BAR_STRIDE)
    const float* bias;            // FP32 bias table (block 1's first layer)
    const float* w3;              // output layer weights
    uint32_t taddr;               // the warp's accumulator columns
    long long *et, *wt, *pt;      // diagnostics stamps or null
};

// KIND: EPI_PLAIN ReLU + BF16; EPI_KEEP also writes o^k back into the accumulator (the next
// second layer's start value); EPI_FIRST adds the FP32 bias (block 1's first layer, whose
// MMAs read no activation column); EPI_LAST is the output layer's ReLU and dot product.
template <int KIND>
__device__ __forceinline__ void epi_layer(const EpiArgs& e, float (&v)[NBLK * 16], float& dot) {
#pragma unroll
    for (int b = 0; b < NBLK; ++b) {
        const int c0 = 32 * b + 16 * e.half;
        float* w = v + 16 * b;
        // accumulator columns 200..207 are exactly zero (zero weight rows and zero start
        // values), so ReLU needs no column mask
        if (c0 < NP) {
            if (KIND == EPI_FIRST) {
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
            if (KIND == EPI_KEEP) tc::tmem_st16(e.taddr + 32u * b, w);
            if (KIND == EPI_LAST) {
                const float4* w4 = reinterpret_cast<const float4*>(e.w3 + c0);
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
        if ((b & 1) || b == NBLK - 1) {
            // publish blocks b-1, b: make the stores visible to the tensor core, and (last
            // block) complete the accumulator write-back first, since the MMAs that start
            // from it wait for the last publication
            if (e.et) e.et[1 + (b >> 1)] = clock64();
            tc::fence_proxy_async_smem();
            if (b == NBLK - 1 && KIND == EPI_KEEP) tc::tmem_wait_st();
            tc::tc_fence_before();
            __syncwarp();
            if (e.et) e.et[5 + (b >> 1)] = clock64();
            if (e.lane == 0) tc::mbar_arrive(e.blk_bar + BAR_STRIDE * (uint32_t)(b >> 1));
            if (e.wt) e.wt[b >> 1] = clock64();
            if (e.pt) e.pt[b >> 1] = clock64();
        }
    }
}

template <bool TRACE>
__global__ void __launch_bounds__(NTHREADS, 1)
k_rpnn_tc(const __grid_constant__ CUtensorMap zmap, const TcArgs a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t base = tc::smem_u32(sm);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + OFF_ABORT);
    auto bar = [&](int i) { return base + OFF_BAR + BAR_STRIDE * (uint32_t)i; };
    // diagnostics: cycles spent in each role's waits, when a.trace is set, and for block
    // 0 a timeline of 4 stamps per layer instance (MMA issue start/end, epilogue start/end)
    long long* tl = (TRACE && blockIdx.x == 0) ? reinterpret_cast<long long*>(a.trace + 1024 * 12) : nullptr;
    unsigned long long cyc_wait = 0, cyc_wait2 = 0;
    const long long cyc_start = clock64();
    auto twait = [&](uint32_t b, uint32_t parity, unsigned long long& acc) {
        const long long t0 = TRACE ? clock64() : 0;
        const bool r = tc::mbar_wait(b, parity, abort_flag);
        if (TRACE) acc += (unsigned long long)(clock64() - t0);
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
        tc::mbar_init(bar(B_DRAIN), 1);
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
            uint32_t wfills = 0, zfills = 0;
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
                            ++zfills;
                            if (++sz == Z_STAGES) { sz = 0; pz ^= 1u; }
                        }
                        const int b0 = k0 / 32;
                        const uint32_t bytes = (nb - b0 >= 2 ? 2u : 1u) * BLK_B;
                        if (!twait(bar(B_WEMPTY + sw), pw ^ 1u, cyc_wait)) break;
                        tc::mbar_expect_tx(bar(B_WFULL + sw), bytes);
                        tc::bulk_g2s(base + OFF_W + sw * W_STAGE, a.img + a.img_off[l] + (int64_t)b0 * (BLK_B / 2),
                                     bytes, bar(B_WFULL + sw));
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
            S.idesc = tc::idesc_bf16(TM, NP);
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
            S.tr = tl;
            S.cyc = 0;
            uint32_t n = 0;                          // layer instance
            for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
                for (int l = 0; l < NLAYERS; ++l, ++n) {
                    const uint32_t acc = tmem + (uint32_t)(l & 1) * 256u;   // n and l share parity
                    if (TRACE && tl && n < 512) tl[4 * n] = clock64();
                    S.stamp = (TRACE && tl && (n == 24 || n == 25)) ? tl + 2048 + (n - 24) * 24 : nullptr;
                    // One tcgen05 fence per layer orders this layer's MMAs after the waits
                    // (in the previous layer) that saw epilogue n-2 finish with accumulator
                    // n % 2.  Operands written by TMA or by the epilogue (fence.proxy.async +
                    // mbarrier) need no tcgen05 fence.
                    tc::tc_fence_after();
                    // publication parity of epilogue n-1: n and l share parity
                    const uint32_t pb = (uint32_t)(l & 1) ^ 1u;
                    if (l == 0) {
                        issue_layer<TRACE, KZ, KZ, false>(S, acc, pb);
                        // a tile's first layer reads no activation; it still waits for the
                        // previous epilogue, so the issuer never runs two phases ahead of it
                        if (n > 0) tc::mbar_wait_issuer(S.blk0 + BAR_STRIDE * (NPUB - 1), pb, tc::kSpinLimit, S.abort_addr);
                    } else if (l < 20 && !(l & 1)) {
                        issue_layer<TRACE, KZ + NP, KZ, false>(S, acc, pb);
                    } else if (layer_resid(l)) {
                        issue_layer<TRACE, NP, 0, true>(S, acc, pb);
                    } else {
                        issue_layer<TRACE, NP, 0, false>(S, acc, pb);
                    }
                    tc::mma_commit(bar(B_ACC));
                    if (TRACE && tl && n < 512) tl[4 * n + 1] = clock64();
                }
                if (*abort_flag) break;
            }
            cyc_wait = S.cyc;
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
                if (lane == 0) ok = twait(bar(B_ACC), n & 1u, cyc_wait);
                ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
                if (TRACE && tl && n < 512 && warp == 2 && lane == 0) tl[4 * n + 2] = clock64();
                if (!ok) break;
                tc::tc_fence_after();
                const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (n & 1u) * 256u + 16u * half;
                float v[NBLK * 16];
                tc::tmem_ld16x7(taddr, v);
                // diagnostics (block 0, warp 2, instances 23 and 24): after the load, before
                // and after each publication's fences
                long long* et = (TRACE && tl && warp == 2 && lane == 0 && (n == 23 || n == 24))
                                    ? tl + 2048 + 64 + (n - 23) * 16 : nullptr;
                if (et) et[0] = clock64();
                long long* wt = (TRACE && tl && lane == 0 && n == 24) ? tl + 2048 + 96 + (warp - 2) * 4 : nullptr;
                long long* pt = (TRACE && tl && warp == 2 && lane == 0 && (n == 23 || n == 24))
                                    ? tl + 2048 + 48 + (n - 23) * 8 : nullptr;
                const EpiArgs ea{Xsm, row, sw, half, lane, bar(B_BLK), a.bias, a.w3, taddr, et, wt, pt};
                // one straight-line routine per layer kind
                if (l == 0) epi_layer<EPI_FIRST>(ea, v, dot);
                else if (l == 21) epi_layer<EPI_LAST>(ea, v, dot);
                else if (layer_keeps_o(l)) epi_layer<EPI_KEEP>(ea, v, dot);
                else epi_layer<EPI_PLAIN>(ea, v, dot);
                if (TRACE && tl && n < 512 && warp == 2 && lane == 0) tl[4 * n + 3] = clock64();
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
    if (TRACE && lane == 0 && warp <= 2) {
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
    // (never while the stream is being captured into a graph: tracing synchronises)
    cudaStreamCaptureStatus capturing = cudaStreamCaptureStatusNone;
    RPNN_CUDA_TRY(cudaStreamIsCapturing(s, &capturing));
    const bool tracing = getenv("RPNN_TC_TRACE") != nullptr && capturing == cudaStreamCaptureStatusNone;
    if (tracing && !trace_buf) RPNN_CUDA_TRY(cudaMalloc(&trace_buf, (1024 * 12 + 4 * 512 + 128) * sizeof(unsigned long long)));
    a.trace = tracing ? trace_buf : nullptr;
    static bool attr = false;
    if (!attr) {
        RPNN_CUDA_TRY(cudaFuncSetAttribute(k_rpnn_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
        RPNN_CUDA_TRY(cudaFuncSetAttribute(k_rpnn_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
        attr = true;
    }
    const int64_t ntiles = (q + TM - 1) / TM;
    const int grid = (int)std::min<int64_t>(ntiles, c.num_sms);
    if (tracing) RPNN_CUDA_TRY(cudaMemsetAsync(trace_buf, 0, (1024 * 12 + 4 * 512 + 128) * sizeof(unsigned long long), s));
    if (tracing) k_rpnn_tc<true><<<grid, NTHREADS, SMEM_BYTES, s>>>(zmap, a);
    else k_rpnn_tc<false><<<grid, NTHREADS, SMEM_BYTES, s>>>(zmap, a);
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
        // block 0, layer instances 24 and 25 (second tile, layers 2 and 3): per stage the
        // poll start / poll end / commit, and the publications of the epilogue feeding it,
        // relative to the layer's issue start
        for (int inst = 0; inst < 2; ++inst) {
            const long long t0 = tlh[4 * (24 + inst)];
            const long long* st = &tlh[2048 + inst * 24];
            const long long* pub = &tlh[2048 + 48 + inst * 8];
            fprintf(stderr, "[rpnn tc stages] inst %d: epilogue %d acc-ready %lld pubs %lld %lld %lld %lld\n", 24 + inst,
                    23 + inst, tlh[4 * (23 + inst) + 2] - t0, pub[0] - t0, pub[1] - t0, pub[2] - t0, pub[3] - t0);
            const long long* et = &tlh[2048 + 64 + inst * 16];
            const long long ea = tlh[4 * (23 + inst) + 2];
            fprintf(stderr, "[rpnn tc epilogue] inst %d (from acc-ready): tmem-ld %lld | pubs: stores %lld %lld %lld %lld"
                            " / fenced %lld %lld %lld %lld\n", 23 + inst, et[0] - ea, et[1] - ea, et[2] - ea, et[3] - ea,
                    et[4] - ea, et[5] - ea, et[6] - ea, et[7] - ea, et[8] - ea);
            if (inst == 1) {
                for (int w = 0; w < 8; ++w)
                    fprintf(stderr, "[rpnn tc epilogue] inst 24 warp %d (scheduler %d): pubs %lld %lld %lld %lld\n", w + 2,
                            (w + 2) & 3, tlh[2048 + 96 + w * 4] - ea, tlh[2048 + 96 + w * 4 + 1] - ea,
                            tlh[2048 + 96 + w * 4 + 2] - ea, tlh[2048 + 96 + w * 4 + 3] - ea);
            }
            for (int j = 0; j < 8 && st[3 * j]; ++j)
                fprintf(stderr, "[rpnn tc stages] inst %d stage %d  poll %6lld .. %6lld  commit %6lld\n", 24 + inst, j,
                        st[3 * j] - t0, st[3 * j + 1] - t0, st[3 * j + 2] - t0);
        }
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
