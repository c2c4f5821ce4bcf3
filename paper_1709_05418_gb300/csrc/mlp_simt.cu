// mlp_simt.cu -- FP32 CUDA-core form of the RPNN (Sec. 4.3, Fig. 6): forward, the
// chain-rule backward, the log-MSE loss (Sec. 5.2) and Adam.
//
// Every layer is one launch of a tiled SGEMM with a fused epilogue
//   C = act(sum_seg A_seg B_seg + bias + residual) [* (mask > 0)]
// where each operand is addressed through (row, col) strides, so the same kernel
// serves the forward layers, the data gradients (dY W) and the weight gradients
// (dY^T X).  The block's first layer is two segments: [z^k | o^{k-1}] [V^k | W1^k]^T.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace rpnn {

namespace {

struct Seg {
    const float* A;
    int64_t sam, sak;   // A(m, k) = A[m*sam + k*sak]
    const float* B;
    int64_t sbk, sbn;   // B(k, n) = B[k*sbk + n*sbn]
    int K;
};

struct Epi {
    const float* bias;  // [N] or null
    const float* res;   // residual [M][ldr] or null
    int64_t ldr;
    const float* mask;  // multiply by (mask > 0): element (m, n) at mask[m * ldm + n * mcs], or null
    int64_t ldm, mcs;
    int relu;
    float* C;
    int64_t ldc;
};

__device__ __forceinline__ float epilogue(const Epi& e, int m, int n, float v) {
    if (e.bias) v += e.bias[n];
    if (e.res) v += e.res[(int64_t)m * e.ldr + n];
    if (e.relu) v = fmaxf(v, 0.0f);
    if (e.mask && !(e.mask[(int64_t)m * e.ldm + (int64_t)n * e.mcs] > 0.0f)) v = 0.0f;
    return v;
}

template <int BM, int BN, int BK, int NT>
__device__ __forceinline__ void load_tiles(const Seg& s, int m0, int n0, int k0, int M, int N,
                                           float (*As)[BM + 4], float (*Bs)[BN + 4]) {
    const int tid = threadIdx.x;
#pragma unroll
    for (int r = 0; r < (BM * BK) / NT; ++r) {
        const int e = tid + r * NT;
        int mm, kk;
        if (s.sak == 1) { mm = e / BK; kk = e % BK; } else { mm = e % BM; kk = e / BM; }
        const int m = m0 + mm, k = k0 + kk;
        As[kk][mm] = (m < M && k < s.K) ? __ldg(s.A + (int64_t)m * s.sam + (int64_t)k * s.sak) : 0.0f;
    }
#pragma unroll
    for (int r = 0; r < (BN * BK) / NT; ++r) {
        const int e = tid + r * NT;
        int kk, nn;
        if (s.sbn == 1) { kk = e / BN; nn = e % BN; } else { kk = e % BK; nn = e / BK; }
        const int n = n0 + nn, k = k0 + kk;
        Bs[kk][nn] = (n < N && k < s.K) ? __ldg(s.B + (int64_t)k * s.sbk + (int64_t)n * s.sbn) : 0.0f;
    }
}

// C tile [BM x BN] per block, [TM x TN] per thread (rows ty + i*BM/TM, columns
// tx + j*BN/TN).  Every output sums its products in increasing k (segment 0, then
// segment 1) with one FMA each, whatever the tile shape, so all tiles give the same bits.
// With splits > 1, block z takes the z-th contiguous run of the K tiles and writes its
// partial sums to ws[z][m][n]; k_splitk_epi adds them in z order and applies the epilogue.
template <int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
k_gemm(int M_host, const int* __restrict__ M_dev, int N, Seg s0, Seg s1, int nseg, Epi e, int splits,
       float* __restrict__ ws) {
    constexpr int NT = (BM / TM) * (BN / TN), CX = BN / TN, RY = BM / TM;
    static_assert((BM * BK) % NT == 0 && (BN * BK) % NT == 0, "tile loads must divide evenly");
    const int M = M_dev ? *M_dev : M_host;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    if (m0 >= M) return;
    __shared__ float As[BK][BM + 4];
    __shared__ float Bs[BK][BN + 4];
    const int tx = threadIdx.x % CX, ty = threadIdx.x / CX;
    float acc[TM][TN] = {};
    const int T0 = (s0.K + BK - 1) / BK;
    const int T = T0 + (nseg > 1 ? (s1.K + BK - 1) / BK : 0);
    const int per = (T + splits - 1) / splits;
    const int tb = (int)blockIdx.z * per, te = min(T, tb + per);
    for (int t = tb; t < te; ++t) {
        const bool first = t < T0;
        const Seg& s = first ? s0 : s1;
        const int k0 = (first ? t : t - T0) * BK;
        load_tiles<BM, BN, BK, NT>(s, m0, n0, k0, M, N, As, Bs);
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float a[TM], b[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + RY * i];
#pragma unroll
            for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx + CX * j];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int m = m0 + ty + RY * i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int n = n0 + tx + CX * j;
            if (n >= N) continue;
            if (splits > 1)
                ws[((int64_t)blockIdx.z * M_host + m) * N + n] = acc[i][j];
            else
                e.C[(int64_t)m * e.ldc + n] = epilogue(e, m, n, acc[i][j]);
        }
    }
}

__global__ void k_splitk_epi(const float* __restrict__ ws, int splits, int M_host, const int* __restrict__ M_dev,
                             int N, Epi e) {
    const int M = M_dev ? *M_dev : M_host;
    const int64_t total = (int64_t)M * N;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int m = (int)(i / N), n = (int)(i % N);
        float v = 0.0f;
        for (int z = 0; z < splits; ++z) v += ws[((int64_t)z * M_host + m) * N + n];
        e.C[(int64_t)m * e.ldc + n] = epilogue(e, m, n, v);
    }
}

// out[i] = x[i] * (m[i] > 0)
__global__ void k_mask(const float* __restrict__ x, const float* __restrict__ m, int n,
                       float* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = m[i] > 0.0f ? x[i] : 0.0f;
}

// column sums: out[n] = sum_m X[m][n] (bias gradients).  Block of 8 x 128 threads per 8
// columns (a warp reads 8 consecutive floats of 4 rows: whole 32-byte sectors): thread
// (x, y) sums rows y, y + 128, ... of column x in increasing order, then the 128 partial sums
// are added in y order (a fixed order for given M).
constexpr int kColsumCols = 8, kColsumRows = 128;
__global__ void __launch_bounds__(kColsumCols * kColsumRows) k_colsum(const float* __restrict__ X, int M, int N,
                                                                   int64_t ld, float* __restrict__ out) {
    __shared__ float part[kColsumRows][kColsumCols + 1];
    const int n = blockIdx.x * kColsumCols + threadIdx.x;
    float s = 0.0f;
    if (n < N)
        for (int m = threadIdx.y; m < M; m += kColsumRows) s += X[(int64_t)m * ld + n];
    part[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0 && n < N) {
        float t = 0.0f;
        for (int y = 0; y < kColsumRows; ++y) t += part[y][threadIdx.x];
        out[n] = t;
    }
}

void launch_colsum(const float* X, int M, int N, int64_t ld, float* out, cudaStream_t s) {
    k_colsum<<<(unsigned)((N + kColsumCols - 1) / kColsumCols), dim3(kColsumCols, kColsumRows), 0, s>>>(X, M, N, ld,
                                                                                                   out);
}

Seg seg(const float* A, int64_t sam, int64_t sak, const float* B, int64_t sbk, int64_t sbn, int K) {
    Seg s;
    s.A = A; s.sam = sam; s.sak = sak; s.B = B; s.sbk = sbk; s.sbn = sbn; s.K = K;
    return s;
}

Epi epi(float* C, int64_t ldc, const float* bias = nullptr, int relu = 0,
        const float* res = nullptr, int64_t ldr = 0, const float* mask = nullptr, int64_t ldm = 0,
        int64_t mcs = 1) {
    Epi e;
    e.C = C; e.ldc = ldc; e.bias = bias; e.relu = relu; e.res = res; e.ldr = ldr;
    e.mask = mask; e.ldm = ldm; e.mcs = mcs;
    return e;
}

// ---- tile shapes and the autotuner ----------------------------------------------------
struct TileShape { int bm, bn, bk, tm, tn; };
constexpr TileShape kTiles[] = {
    {64, 64, 16, 4, 4},    // the default (no tuning)
    {128, 64, 16, 8, 4},
    {64, 128, 16, 4, 8},
    {128, 128, 8, 8, 8},
    {32, 64, 16, 2, 4},
    {128, 32, 16, 8, 2},
};
constexpr int kNumTiles = sizeof(kTiles) / sizeof(kTiles[0]);
constexpr int kSplits[] = {1, 2, 4, 8, 16, 32};
constexpr int kMinSplitK = 1024;

template <int BM, int BN, int BK, int TM, int TN>
void launch_tile(int M, const int* M_dev, int N, const Seg& s0, const Seg& s1, int nseg, const Epi& e,
                 int splits, float* ws, cudaStream_t s) {
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, splits);
    k_gemm<BM, BN, BK, TM, TN><<<grid, (BM / TM) * (BN / TN), 0, s>>>(M, M_dev, N, s0, s1, nseg, e, splits, ws);
}

rpnn_status launch_gemm(int tile, int splits, int M, const int* M_dev, int N, const Seg& s0, const Seg& s1,
                        int nseg, const Epi& e, float* ws, cudaStream_t s) {
    const TileShape& t = kTiles[tile];
    if ((M + t.bm - 1) / t.bm > 65535) { set_error("GEMM with %d rows exceeds the grid limit", M); return RPNN_ERR_ARG; }
    switch (tile) {
        case 0: launch_tile<64, 64, 16, 4, 4>(M, M_dev, N, s0, s1, nseg, e, splits, ws, s); break;
        case 1: launch_tile<128, 64, 16, 8, 4>(M, M_dev, N, s0, s1, nseg, e, splits, ws, s); break;
        case 2: launch_tile<64, 128, 16, 4, 8>(M, M_dev, N, s0, s1, nseg, e, splits, ws, s); break;
        case 3: launch_tile<128, 128, 8, 8, 8>(M, M_dev, N, s0, s1, nseg, e, splits, ws, s); break;
        case 4: launch_tile<32, 64, 16, 2, 4>(M, M_dev, N, s0, s1, nseg, e, splits, ws, s); break;
        default: launch_tile<128, 32, 16, 8, 2>(M, M_dev, N, s0, s1, nseg, e, splits, ws, s); break;
    }
    RPNN_CHECK_LAUNCH();
    if (splits > 1) {
        const int64_t total = (int64_t)M * N;
        int64_t b = (total + 255) / 256;
        if (b > 152 * 8) b = 152 * 8;
        k_splitk_epi<<<(unsigned)b, 256, 0, s>>>(ws, splits, M, M_dev, N, e);
        RPNN_CHECK_LAUNCH();
    }
    return RPNN_OK;
}

GemmKey make_key(int M, int N, const Seg& s0, const Seg* s1, const Epi& e, bool dyn) {
    GemmKey k{};
    k.M = M; k.N = N; k.K0 = s0.K; k.K1 = s1 ? s1->K : 0;
    k.flags = (s0.sak == 1) | (s0.sbn == 1) << 1 | (s1 && s1->sak == 1) << 2 | (s1 && s1->sbn == 1) << 3 |
              (e.bias != nullptr) << 4 | (e.res != nullptr) << 5 | (e.mask != nullptr) << 6 | (int)dyn << 7;
    return k;
}

// Times every admissible (tile, split) on the call's own operands, writing into scratch
// (the caller's output is untouched, so in-place residuals stay valid), and returns the
// fastest.  Synchronises the stream.
rpnn_status tune(Ctx& c, const GemmKey& key, int M, const int* M_dev, int N, const Seg& s0, const Seg& s1,
                 int nseg, const Epi& e, cudaStream_t s, GemmChoice* out) {
    GemmTuner& tu = c.tuner;
    // admissible (tile, split) pairs: tiles no taller than twice the rows; a split only
    // for inner sizes of at least kMinSplitK (the weight gradients, which sum over the
    // batch; forward GEMMs therefore never split and give the default tile's bits), where
    // the tiles alone fill fewer than one wave, keeping >= 4 K tiles per run and at most
    // 8 blocks per SM
    struct Cand { int t, sp; };
    std::vector<Cand> cands;
    int maxsplit = 1;
    const int ksteps16 = (s0.K + 15) / 16 + (nseg > 1 ? (s1.K + 15) / 16 : 0);
    for (int t = 0; t < kNumTiles; ++t) {
        const TileShape& ts = kTiles[t];
        if (t > 0 && ts.bm > 2 * M) continue;
        const int64_t blocks = (int64_t)((N + ts.bn - 1) / ts.bn) * ((M + ts.bm - 1) / ts.bm);
        for (int sp : kSplits) {
            if (sp > 1 && (ksteps16 * 16 < kMinSplitK || blocks >= c.num_sms || blocks * sp > (int64_t)c.num_sms * 8 ||
                           (ksteps16 * 16 / ts.bk) / sp < 4))
                continue;
            cands.push_back({t, sp});
            if (sp > maxsplit) maxsplit = sp;
        }
    }
    rpnn_status st = tu.scratch.reserve((size_t)M * N * sizeof(float));
    if (!st && maxsplit > 1) st = tu.ws.reserve((size_t)maxsplit * M * N * sizeof(float));
    if (st) return st;
    Epi es = e;
    es.C = tu.scratch.as<float>();
    es.ldc = N;
    if (!tu.ev0) {
        RPNN_CUDA_TRY(cudaEventCreate(&tu.ev0));
        RPNN_CUDA_TRY(cudaEventCreate(&tu.ev1));
    }
    GemmChoice best{0, 1, 1e30f, 0.0f};
    for (const Cand& cd : cands) {
        st = launch_gemm(cd.t, cd.sp, M, M_dev, N, s0, s1, nseg, es, tu.ws.as<float>(), s);   // warm
        if (st) return st;
        RPNN_CUDA_TRY(cudaEventRecord(tu.ev0, s));
        for (int r = 0; r < 3; ++r) {
            st = launch_gemm(cd.t, cd.sp, M, M_dev, N, s0, s1, nseg, es, tu.ws.as<float>(), s);
            if (st) return st;
        }
        RPNN_CUDA_TRY(cudaEventRecord(tu.ev1, s));
        RPNN_CUDA_TRY(cudaEventSynchronize(tu.ev1));
        float ms = 0.0f;
        RPNN_CUDA_TRY(cudaEventElapsedTime(&ms, tu.ev0, tu.ev1));
        const float us = ms * 1000.0f / 3.0f;
        if (cd.t == 0 && cd.sp == 1) best.default_us = us;
        if (us < best.us) { best.us = us; best.tile = cd.t; best.splits = cd.sp; }
    }
    tu.table.emplace_back(key, best);
    ++tu.version;
    *out = best;
    return RPNN_OK;
}

// C = epilogue(sum_seg A_seg B_seg).  With a context whose autotuner is on, the tile shape
// and split-K factor are the fastest measured for this shape (timed at its first use,
// outside stream capture); otherwise the default 64 x 64 tile without a split.
rpnn_status gemm(Ctx* c, int M, const int* M_dev, int N, const Seg& s0, const Seg* s1, const Epi& e,
                 cudaStream_t s) {
    if (M <= 0 || N <= 0) return RPNN_OK;
    GemmChoice ch{0, 1, 0.0f, 0.0f};
    const Seg& s1r = s1 ? *s1 : s0;
    const int nseg = s1 ? 2 : 1;
    if (c && c->tuner.enabled) {
        // a choice already made applies under stream capture too; timing new shapes does not
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        RPNN_CUDA_TRY(cudaStreamIsCapturing(s, &cs));
        const GemmKey key = make_key(M, N, s0, s1, e, M_dev != nullptr);
        const GemmChoice* hit = c->tuner.find(key);
        if (hit) {
            ch = *hit;
        } else if (cs == cudaStreamCaptureStatusNone) {
            rpnn_status st = tune(*c, key, M, M_dev, N, s0, s1r, nseg, e, s, &ch);
            if (st) return st;
        }
    }
    float* ws = nullptr;
    if (ch.splits > 1) {
        rpnn_status st = c->tuner.ws.reserve((size_t)ch.splits * M * N * sizeof(float));
        if (st) return st;
        ws = c->tuner.ws.as<float>();
    }
    return launch_gemm(ch.tile, ch.splits, M, M_dev, N, s0, s1r, nseg, e, ws, s);
}

// Deterministic log-MSE loss (Sec. 5.2): one block; FP64 tree reduction.
// log-MSE loss (Sec. 5.2): per element r = log1p(g) - log1p(t) and dl/dg = 2 r / ((1 + g) B)
// in FP64, block sums of r^2 in a fixed tree, then the block sums in block order.  Spread
// over blocks: an FP64 log1p per element on one SM took tens of microseconds per step.
constexpr int kLossThreads = 256, kLossBlocks = 64;
__global__ void k_loss_terms(const float* __restrict__ g, const float* __restrict__ t, int B,
                             double* __restrict__ part, float* __restrict__ dg) {
    __shared__ double red[kLossThreads];
    double s = 0.0;
    for (int i = blockIdx.x * kLossThreads + threadIdx.x; i < B; i += gridDim.x * kLossThreads) {
        const double r = log1p((double)g[i]) - log1p((double)t[i]);
        s += r * r;
        dg[i] = (float)(2.0 * r / ((1.0 + (double)g[i]) * (double)B));
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = kLossThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_loss_sum(const double* __restrict__ part, int nb, int B, double* loss) {
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s += part[b];
        *loss = s / (double)B;
    }
}

__global__ void k_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ grad, int64_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = grad[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

__global__ void k_adam_dev(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                           const float* __restrict__ grad, int64_t n, float lr, float b1, float b2, float eps,
                           const float* __restrict__ cc) {
    const float c1 = cc[0], c2 = cc[1];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = grad[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

__global__ void k_set2(float* __restrict__ cc, float a, float b) {
    cc[0] = a;
    cc[1] = b;
}

}  // namespace

int gemm_tile_index(int bm, int bn, int bk) {
    for (int t = 0; t < kNumTiles; ++t)
        if (kTiles[t].bm == bm && kTiles[t].bn == bn && kTiles[t].bk == bk) return t;
    return -1;
}

void gemm_tile_shape(int tile, int* bm, int* bn, int* bk) {
    const TileShape& t = kTiles[(tile >= 0 && tile < kNumTiles) ? tile : 0];
    *bm = t.bm; *bn = t.bn; *bk = t.bk;
}

ParamLayout param_layout_for(int din) {
    ParamLayout l{};
    int64_t o = 0;
    for (int k = 0; k < RPNN_K; ++k) {
        l.V[k] = o; o += (int64_t)RPNN_H * din;
        if (k > 0) { l.W1[k] = o; o += (int64_t)RPNN_H * RPNN_H; } else l.W1[k] = -1;
        l.b1[k] = o; o += RPNN_H;
        l.W2[k] = o; o += (int64_t)RPNN_H * RPNN_H;
        l.b2[k] = o; o += RPNN_H;
    }
    for (int t = 0; t < 3; ++t) {
        const int out = t == 2 ? 1 : RPNN_H;
        l.T[t] = o; o += (int64_t)out * RPNN_H;
        l.bT[t] = o; o += out;
    }
    l.total = o;
    return l;
}

const ParamLayout& param_layout() {
    static ParamLayout L = param_layout_for(RPNN_DIN);
    return L;
}


// saved activations per row: o^1..o^10, F1^1..F1^10, o^11, o^12 (each 200), g
size_t mlp_saved_floats_per_row() { return 22 * (size_t)RPNN_H + 1; }

rpnn_status rpnn_forward_f32(Ctx* c, const NetDims& nd, const float* P, const float* desc, int64_t q,
                             const int* q_dev, float* out, float* saved, float* const scr[3], cudaStream_t s) {
    const ParamLayout& L = *nd.L;
    const int M = (int)q;
    const int64_t H = RPNN_H, ZS = (int64_t)RPNN_K * nd.stride;
    float *o_prev = nullptr, *o_cur, *f1;
    auto slot = [&](int i) { return saved + (size_t)i * q * H; };
    rpnn_status st;
    for (int k = 0; k < RPNN_K; ++k) {
        if (saved) { o_cur = slot(k); f1 = slot(10 + k); }
        else { o_cur = scr[0]; f1 = scr[1]; }
        // F1 = relu([z^k | o^{k-1}] [V^k | W1^k]^T + b1)
        Seg z = seg(desc + k * nd.stride, ZS, 1, P + L.V[k], 1, nd.din, nd.din);
        if (k > 0) {
            Seg o = seg(o_prev, H, 1, P + L.W1[k], 1, H, RPNN_H);
            st = gemm(c, M, q_dev, RPNN_H, z, &o, epi(f1, H, P + L.b1[k], 1), s);
        } else {
            st = gemm(c, M, q_dev, RPNN_H, z, nullptr, epi(f1, H, P + L.b1[k], 1), s);
        }
        if (st) return st;
        // o^k = relu(W2 F1 + b2 + o^{k-1})  (in place when not saving)
        Seg w2 = seg(f1, H, 1, P + L.W2[k], 1, H, RPNN_H);
        st = gemm(c, M, q_dev, RPNN_H, w2, nullptr, epi(o_cur, H, P + L.b2[k], 1, k > 0 ? o_prev : nullptr, H), s);
        if (st) return st;
        o_prev = o_cur;
    }
    // standard layers
    float* t0 = saved ? slot(20) : scr[1];
    float* t1 = saved ? slot(21) : scr[2];
    st = gemm(c, M, q_dev, RPNN_H, seg(o_prev, H, 1, P + L.T[0], 1, H, RPNN_H), nullptr,
              epi(t0, H, P + L.bT[0], 1), s);
    if (st) return st;
    st = gemm(c, M, q_dev, RPNN_H, seg(t0, H, 1, P + L.T[1], 1, H, RPNN_H), nullptr,
              epi(t1, H, P + L.bT[1], 1), s);
    if (st) return st;
    st = gemm(c, M, q_dev, 1, seg(t1, H, 1, P + L.T[2], 1, H, RPNN_H), nullptr, epi(out, 1, P + L.bT[2], 1), s);
    if (st) return st;
    if (saved) RPNN_CUDA_TRY(cudaMemcpyAsync(saved + (size_t)22 * q * H, out, q * sizeof(float),
                                             cudaMemcpyDeviceToDevice, s));
    return RPNN_OK;
}

rpnn_status mlp_forward_f32(Ctx& c, const float* desc, int64_t q, const int* q_dev, float* out,
                            float* saved, cudaStream_t s) {
    const NetDims nd{&param_layout(), RPNN_DIN, RPNN_DESC_STRIDE};
    float* const scr[3] = {c.act0.as<float>(), c.act1.as<float>(), c.act2.as<float>()};
    return rpnn_forward_f32(&c, nd, c.params32.as<float>(), desc, q, q_dev, out, saved, scr, s);
}

rpnn_status rpnn_backward_f32(Ctx& c, const NetDims& nd, const float* P, const float* desc, int64_t q,
                              const float* saved, const float* dout, float* dP, cudaStream_t s) {
    const ParamLayout& L = *nd.L;
    const int M = (int)q;
    const int64_t H = RPNN_H, ZS = (int64_t)RPNN_K * nd.stride;
    auto slot = [&](int i) { return saved + (size_t)i * q * H; };
    const float* g = saved + (size_t)22 * q * H;
    rpnn_status st = c.act0.reserve((size_t)q * H * sizeof(float));
    if (!st) st = c.act1.reserve((size_t)q * H * sizeof(float));
    if (!st) st = c.act2.reserve((size_t)q * H * sizeof(float));
    if (!st) st = c.t_dg.reserve((size_t)q * sizeof(float));
    if (st) return st;
    float* bufA = c.act0.as<float>();
    float* bufB = c.act1.as<float>();
    float* da = c.act2.as<float>();
    float* da3 = c.t_dg.as<float>();
    // last layer: g = relu(T3 o12 + bT3): da3 = dout * (g > 0)
    k_mask<<<(M + 255) / 256, 256, 0, s>>>(dout, g, M, da3);
    RPNN_CHECK_LAUNCH();
    // dT3[0][j] = sum_m da3[m] o12[m][j]; dbT3 = sum_m da3
    st = gemm(&c, 1, nullptr, RPNN_H, seg(da3, 0, 1, slot(21), H, 1, M), nullptr, epi(dP + L.T[2], H), s);
    if (st) return st;
    launch_colsum(da3, M, 1, 1, dP + L.bT[2], s);
    RPNN_CHECK_LAUNCH();
    // da2 = (da3 T3) * (o12 > 0)
    st = gemm(&c, M, nullptr, RPNN_H, seg(da3, 1, 1, P + L.T[2], H, 1, 1), nullptr,
              epi(bufA, H, nullptr, 0, nullptr, 0, slot(21), H), s);
    if (st) return st;
    // standard layer 2: input o11 (slot 20); layer 1: input o10 (slot 9)
    const float* tin[2] = {slot(9), slot(20)};
    for (int t = 1; t >= 0; --t) {
        // dT = da^T x_in; db = colsum(da)
        st = gemm(&c, RPNN_H, nullptr, RPNN_H, seg(bufA, 1, H, tin[t], H, 1, M), nullptr, epi(dP + L.T[t], H), s);
        if (st) return st;
        launch_colsum(bufA, M, RPNN_H, H, dP + L.bT[t], s);
        RPNN_CHECK_LAUNCH();
        // d x_in = da T, masked by (x_in > 0) (x_in is a ReLU output)
        st = gemm(&c, M, nullptr, RPNN_H, seg(bufA, H, 1, P + L.T[t], H, 1, RPNN_H), nullptr,
                  epi(bufB, H, nullptr, 0, nullptr, 0, tin[t], H), s);
        if (st) return st;
        float* tmp = bufA; bufA = bufB; bufB = tmp;
    }
    // bufA = dpre_10 = dl/d(pre-activation of o^10)
    for (int k = RPNN_K - 1; k >= 0; --k) {
        const float* f1 = slot(10 + k);
        // dW2 = dpre^T F1; db2 = colsum(dpre)
        st = gemm(&c, RPNN_H, nullptr, RPNN_H, seg(bufA, 1, H, f1, H, 1, M), nullptr, epi(dP + L.W2[k], H), s);
        if (st) return st;
        launch_colsum(bufA, M, RPNN_H, H, dP + L.b2[k], s);
        RPNN_CHECK_LAUNCH();
        // da1 = (dpre W2) * (F1 > 0)
        st = gemm(&c, M, nullptr, RPNN_H, seg(bufA, H, 1, P + L.W2[k], H, 1, RPNN_H), nullptr,
                  epi(da, H, nullptr, 0, nullptr, 0, f1, H), s);
        if (st) return st;
        // dV = da1^T z^k; db1 = colsum(da1)
        st = gemm(&c, RPNN_H, nullptr, nd.din, seg(da, 1, H, desc + k * nd.stride, ZS, 1, M), nullptr,
                  epi(dP + L.V[k], nd.din), s);
        if (st) return st;
        launch_colsum(da, M, RPNN_H, H, dP + L.b1[k], s);
        RPNN_CHECK_LAUNCH();
        if (k > 0) {
            const float* oprev = slot(k - 1);
            st = gemm(&c, RPNN_H, nullptr, RPNN_H, seg(da, 1, H, oprev, H, 1, M), nullptr, epi(dP + L.W1[k], H), s);
            if (st) return st;
            // dpre_{k-1} = (dpre_k + da1 W1) * (o^{k-1} > 0)
            st = gemm(&c, M, nullptr, RPNN_H, seg(da, H, 1, P + L.W1[k], H, 1, RPNN_H), nullptr,
                      epi(bufB, H, nullptr, 0, bufA, H, oprev, H), s);
            if (st) return st;
            float* tmp = bufA; bufA = bufB; bufB = tmp;
        }
    }
    return RPNN_OK;
}

rpnn_status mlp_backward_f32(Ctx& c, const float* desc, int64_t q, const float* saved,
                             const float* dout, float* dP, cudaStream_t s) {
    const NetDims nd{&param_layout(), RPNN_DIN, RPNN_DESC_STRIDE};
    return rpnn_backward_f32(c, nd, c.params32.as<float>(), desc, q, saved, dout, dP, s);
}

rpnn_status mlp_output_layer_f32(Ctx& c, const float* t1, int64_t q, float* out, cudaStream_t s) {
    const ParamLayout& L = param_layout();
    const float* P = c.params32.as<float>();
    const int64_t H = RPNN_H;
    return gemm(&c, (int)q, nullptr, 1, seg(t1, H, 1, P + L.T[2], 1, H, RPNN_H), nullptr,
                epi(out, 1, P + L.bT[2], 1), s);
}

rpnn_status mlp_output_layer_backward_f32(Ctx& c, const float* t1, const float* g, const float* dout, int64_t q,
                                          float* dP, float* da2, cudaStream_t s, int64_t ldt1) {
    // t1 = o^12: [q][200] row-major, or (ldt1 > 0) transposed [200][ldt1]
    const int64_t rs = ldt1 > 0 ? 1 : RPNN_H, cs = ldt1 > 0 ? ldt1 : 1;
    const ParamLayout& L = param_layout();
    const float* P = c.params32.as<float>();
    const int M = (int)q;
    const int64_t H = RPNN_H;
    rpnn_status st = c.t_dg.reserve((size_t)q * sizeof(float));
    if (st) return st;
    float* da3 = c.t_dg.as<float>();
    k_mask<<<(M + 255) / 256, 256, 0, s>>>(dout, g, M, da3);
    RPNN_CHECK_LAUNCH();
    st = gemm(&c, 1, nullptr, RPNN_H, seg(da3, 0, 1, t1, rs, cs, M), nullptr, epi(dP + L.T[2], H), s);
    if (st) return st;
    launch_colsum(da3, M, 1, 1, dP + L.bT[2], s);
    RPNN_CHECK_LAUNCH();
    return gemm(&c, M, nullptr, RPNN_H, seg(da3, 1, 1, P + L.T[2], H, 1, 1), nullptr,
                epi(da2, H, nullptr, 0, nullptr, 0, t1, rs, cs), s);
}

rpnn_status colsum_f32(Ctx& c, const float* X, int M, int N, float* out, cudaStream_t s) {
    (void)c;
    launch_colsum(X, M, N, N, out, s);
    RPNN_CHECK_LAUNCH();
    return RPNN_OK;
}

// ---- plain ("all-at-once") MLP of the architecture comparison (Sec. 7, Fig. 10) -------
// hidden layers h_i = relu(W_i h_{i-1} + b_i) (h_{-1} = the input row), output
// g = relu(w_o h_last + b_o); parameters per layer W_i [w_i][w_{i-1}] row-major, then b_i,
// then w_o [1][w_last], b_o.

int64_t dense_param_count(const int* widths, int n, int din) {
    int64_t c = 0, prev = din;
    for (int i = 0; i < n; ++i) {
        c += prev * widths[i] + widths[i];
        prev = widths[i];
    }
    return c + prev + 1;
}

// forward; saved (optional) receives h_0 .. h_{n-1} ([q][w_i] each, consecutive) then g
rpnn_status dense_forward(Ctx& c, const int* widths, int n, int din, const float* P, const float* in, int64_t q,
                          float* out, float* saved, cudaStream_t s) {
    const int M = (int)q;
    const float* x = in;
    int64_t prev = din, off = 0, soff = 0, wmax = 1;
    for (int i = 0; i < n; ++i) wmax = std::max<int64_t>(wmax, widths[i]);
    rpnn_status st = RPNN_OK;
    if (!saved) {
        st = c.act0.reserve((size_t)q * wmax * sizeof(float));
        if (!st) st = c.act1.reserve((size_t)q * wmax * sizeof(float));
        if (st) return st;
    }
    float* bufs[2] = {c.act0.as<float>(), c.act1.as<float>()};
    for (int i = 0; i < n; ++i) {
        const int w = widths[i];
        float* h = saved ? saved + soff : bufs[i & 1];
        st = gemm(&c, M, nullptr, w, seg(x, prev, 1, P + off, 1, prev, (int)prev), nullptr,
                  epi(h, w, P + off + (int64_t)w * prev, 1), s);
        if (st) return st;
        off += (int64_t)w * prev + w;
        soff += (int64_t)q * w;
        x = h;
        prev = w;
    }
    st = gemm(&c, M, nullptr, 1, seg(x, prev, 1, P + off, 1, prev, (int)prev), nullptr, epi(out, 1, P + off + prev, 1), s);
    if (st) return st;
    if (saved) RPNN_CUDA_TRY(cudaMemcpyAsync(saved + soff, out, q * sizeof(float), cudaMemcpyDeviceToDevice, s));
    return RPNN_OK;
}

// gradient of sum_i dout_i g_i into dP (written), from the saved activations
rpnn_status dense_backward(Ctx& c, const int* widths, int n, int din, const float* P, const float* in, int64_t q,
                           const float* saved, const float* dout, float* dP, cudaStream_t s) {
    const int M = (int)q;
    int64_t wmax = 1;
    for (int i = 0; i < n; ++i) wmax = std::max<int64_t>(wmax, widths[i]);
    rpnn_status st = c.act0.reserve((size_t)q * wmax * sizeof(float));
    if (!st) st = c.act1.reserve((size_t)q * wmax * sizeof(float));
    if (!st) st = c.t_dg.reserve((size_t)q * sizeof(float));
    if (st) return st;
    std::vector<int64_t> poff(n + 1), soff(n + 1);
    int64_t o = 0, so = 0, prev = din;
    for (int i = 0; i < n; ++i) {
        poff[i] = o; soff[i] = so;
        o += (int64_t)widths[i] * prev + widths[i];
        so += (int64_t)q * widths[i];
        prev = widths[i];
    }
    poff[n] = o; soff[n] = so;
    const float* g = saved + so;
    float* da = c.t_dg.as<float>();
    k_mask<<<(M + 255) / 256, 256, 0, s>>>(dout, g, M, da);
    RPNN_CHECK_LAUNCH();
    const int64_t wl = n ? widths[n - 1] : din;
    const float* hl = n ? saved + soff[n - 1] : in;
    // output layer: dw_o = da^T h_last, db_o = sum da, dh_last = (da w_o) * (h_last > 0)
    st = gemm(&c, 1, nullptr, (int)wl, seg(da, 0, 1, hl, wl, 1, M), nullptr, epi(dP + poff[n], wl), s);
    if (st) return st;
    launch_colsum(da, M, 1, 1, dP + poff[n] + wl, s);
    RPNN_CHECK_LAUNCH();
    if (n == 0) return RPNN_OK;
    float* cur = c.act0.as<float>();
    float* nxt = c.act1.as<float>();
    st = gemm(&c, M, nullptr, (int)wl, seg(da, 1, 1, P + poff[n], wl, 1, 1), nullptr,
              epi(cur, wl, nullptr, 0, nullptr, 0, hl, wl), s);
    if (st) return st;
    for (int i = n - 1; i >= 0; --i) {
        const int64_t w = widths[i], pw = i ? widths[i - 1] : din;
        const float* xin = i ? saved + soff[i - 1] : in;
        // dW_i = dh_i^T x_{i-1}; db_i = colsum(dh_i)
        st = gemm(&c, (int)w, nullptr, (int)pw, seg(cur, 1, w, xin, pw, 1, M), nullptr, epi(dP + poff[i], pw), s);
        if (st) return st;
        launch_colsum(cur, M, (int)w, w, dP + poff[i] + w * pw, s);
        RPNN_CHECK_LAUNCH();
        if (i > 0) {
            // dh_{i-1} = (dh_i W_i) * (h_{i-1} > 0)
            st = gemm(&c, M, nullptr, (int)pw, seg(cur, w, 1, P + poff[i], pw, 1, (int)w), nullptr,
                      epi(nxt, pw, nullptr, 0, nullptr, 0, xin, pw), s);
            if (st) return st;
            std::swap(cur, nxt);
        }
    }
    return RPNN_OK;
}

rpnn_status launch_loss(Ctx& c, const float* g, const float* target, int batch, double* loss, float* dg,
                        cudaStream_t s) {
    rpnn_status st = c.t_lpart.reserve(kLossBlocks * sizeof(double));
    if (st) return st;
    const int nb = std::max(1, std::min(kLossBlocks, (batch + kLossThreads - 1) / kLossThreads));
    k_loss_terms<<<nb, kLossThreads, 0, s>>>(g, target, batch, c.t_lpart.as<double>(), dg);
    RPNN_CHECK_LAUNCH();
    k_loss_sum<<<1, 32, 0, s>>>(c.t_lpart.as<double>(), nb, batch, loss);
    RPNN_CHECK_LAUNCH();
    return RPNN_OK;
}

rpnn_status launch_adam(float* p, float* m, float* v, const float* grad, int64_t n, int64_t step,
                        const rpnn_adam_cfg& cfg, cudaStream_t s) {
    const double c1 = 1.0 - std::pow((double)cfg.beta1, (double)step);
    const double c2 = 1.0 - std::pow((double)cfg.beta2, (double)step);
    k_adam<<<1024, 256, 0, s>>>(p, m, v, grad, n, cfg.lr, cfg.beta1, cfg.beta2, cfg.eps, (float)c1,
                                (float)c2);
    RPNN_CHECK_LAUNCH();
    return RPNN_OK;
}

rpnn_status launch_adam_corrections(float* cc, int64_t step, const rpnn_adam_cfg& cfg, cudaStream_t s) {
    const double c1 = 1.0 - std::pow((double)cfg.beta1, (double)step);
    const double c2 = 1.0 - std::pow((double)cfg.beta2, (double)step);
    k_set2<<<1, 1, 0, s>>>(cc, (float)c1, (float)c2);
    RPNN_CHECK_LAUNCH();
    return RPNN_OK;
}

rpnn_status launch_adam_dev(float* p, float* m, float* v, const float* grad, int64_t n, const float* cc,
                            const rpnn_adam_cfg& cfg, cudaStream_t s) {
    k_adam_dev<<<1024, 256, 0, s>>>(p, m, v, grad, n, cfg.lr, cfg.beta1, cfg.beta2, cfg.eps, cc);
    RPNN_CHECK_LAUNCH();
    return RPNN_OK;
}

}  // namespace rpnn
