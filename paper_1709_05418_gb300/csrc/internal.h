// internal.h -- host-side state shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include <unordered_map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/rpnn.h"

namespace rpnn {

constexpr int kMaxLevels = 16;
constexpr int kBrick = 8;    // tracking majorant bricks: kBrick^3 voxels
constexpr uint32_t kTrackCapDefault = 1000000u;   // tentative collisions per tracking call

// status bits written by kernels into the context's device status word
enum : uint32_t { kStatIterLimit = 1u, kStatNonFinite = 2u, kStatNegative = 4u, kStatTimeout = 8u,
                  kStatCapacity = 16u };

void set_error(const char* fmt, ...);

// NVTX range for the life of a scope (names a library call or a render stage in profiler
// timelines; costs nothing measurable when no tool is attached)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

#define RPNN_CUDA_TRY(call)                                                              \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            ::rpnn::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),     \
                              __FILE__, __LINE__);                                       \
            return e_ == cudaErrorMemoryAllocation ? RPNN_ERR_OOM : RPNN_ERR_CUDA;       \
        }                                                                                \
    } while (0)

#define RPNN_CHECK_LAUNCH() RPNN_CUDA_TRY(cudaGetLastError())

// A device allocation owned by the context; grows, never shrinks.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    rpnn_status reserve(size_t n);
    void release();
    template <class T> T* as() const { return static_cast<T*>(p); }
};
// advanced by every device allocation or release of a DevBuf (a captured graph's buffer
// pointers stay valid while it is unchanged)
uint64_t devbuf_generation();

// Geometry of one level of the corner-packed pyramid: record (x,y,z) for x in
// [-1, ax-1] holds the 8 trilinear corners of cell (x..x+1, y..y+1, z..z+1).
struct LevelDesc {
    int ax, ay, az;          // level dims
    int64_t rec_offset;      // offset of the level's first record, in records
};

// Everything a kernel needs to read a volume; passed by value.
struct VolumeView {
    const float* raw;        // FP32 grid [nz][ny][nx]
    int n[3];
    float inv_h0;            // max(n)
    float ext[3];            // grid extent in the unit box
    float majorant;
    float albedo, g;
    float inv_mean_f;
    int mip_of_level[RPNN_K];
    const float4* packed;    // corner records (2 float4 per record)
    LevelDesc lvl[kMaxLevels];
    const float* bmaj;       // per-brick majorant [nb2][nb1][nb0] (bricks of kBrick^3 voxels)
    int nb[3];
    float bs;                // brick edge in world units (kBrick / max(n))
    float mip_w[RPNN_K];     // blended descriptor: weight of level mip_of_level[k] + 1 (0: off)
    uint32_t track_cap;      // tentative collisions (and brick steps) per tracking call
    const float* lm;         // first-bounce Lorenz-Mie table (p[N], cdf[N+1], cos[N+1]) or null: HG
    const float* lmc;        // the table after the first bounce (chopped or = lm; null: HG)
    float dscale;            // extinction scale after the first bounce (1 unless chopped)
    float albedo_c;          // albedo after the first bounce (= albedo unless chopped)
};

struct Volume {
    int n[3] = {0, 0, 0};
    float albedo = 0.f, g = 0.f;
    DevBuf raw;              // FP32 copy
    DevBuf packed;           // corner records for the levels the stencil reads
    DevBuf stats;            // device-side statistics scratch
    DevBuf bmaj;             // per-brick tracking majorants
    DevBuf mip_a, mip_b, mip_w;   // separable-pass scratch and taps of the pyramid build
    DevBuf mip_d;                 // the levels the descriptor reads, before corner packing
    int nb[3] = {0, 0, 0};
    bool mip_blend = false;  // descriptor blends levels m_k and m_k + 1
    uint32_t track_cap = 0;  // 0: the default cap (rpnn_set_iteration_cap)
    const float* lm = nullptr;   // the context's Lorenz-Mie table when selected
    const float* lmc = nullptr;  // the table after the first bounce (chopped or = lm)
    float dscale = 1.0f, albedo_c = 0.0f;  // chopped medium (albedo_c 0: = albedo)
    DevBuf stencil_mips;     // every pyramid level as plain FP32, for the stencil-size sweep
    int64_t smip_off[kMaxLevels] = {};   // element offset of each level in stencil_mips
    bool stencil_ready = false;
    bool built = false;
    int levels = 0;
    int dims[kMaxLevels][3] = {};
    rpnn_volume_info info{};
    bool level_packed[kMaxLevels] = {};
    LevelDesc lvl[kMaxLevels] = {};
    VolumeView view() const;
};

// Autotuned SIMT GEMM launches: a shape (rows, columns, the K of each operand segment,
// operand layouts and epilogue kind) maps to the tile shape and split-K factor that ran
// fastest when the shape was first met.
struct GemmKey {
    int M, N, K0, K1, flags;
    bool operator==(const GemmKey& o) const {
        return M == o.M && N == o.N && K0 == o.K0 && K1 == o.K1 && flags == o.flags;
    }
};
struct GemmChoice {
    int tile, splits;     // index into the tile table; K split into this many runs
    float us, default_us; // measured time of the choice and of the default tile
};
struct GemmTuner {
    bool enabled = true;
    uint64_t version = 0;   // advanced by every change of the table or of `enabled`
    std::vector<std::pair<GemmKey, GemmChoice>> table;
    DevBuf scratch, ws;   // tuning output, split-K partial sums
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    const GemmChoice* find(const GemmKey& k) const {
        for (const auto& e : table)
            if (e.first == k) return &e.second;
        return nullptr;
    }
};

// Encoded 2-D tensor maps of BF16 GEMM operands, by what they encode (base address, row
// pitch, inner size, rows, box rows): a pure function of the key, so entries never go stale.
struct TmapKey {
    const void* p;
    int64_t ld;
    int K, rows, box;
    bool operator==(const TmapKey& o) const {
        return p == o.p && ld == o.ld && K == o.K && rows == o.rows && box == o.box;
    }
};
struct TmapKeyHash {
    size_t operator()(const TmapKey& k) const {
        size_t h = std::hash<const void*>()(k.p);
        h = h * 1000003u ^ (size_t)k.ld;
        h = h * 1000003u ^ (size_t)k.K;
        h = h * 1000003u ^ (size_t)k.rows;
        return h * 1000003u ^ (size_t)k.box;
    }
};
struct alignas(64) TmapBytes {
    unsigned char b[128];
};

// One item of a batched render as the batched descriptor kernel reads it: the item's
// volume, the offset of its region in the per-pixel-sample query buffers, its light.
struct BatchItemDev {
    VolumeView v;
    int64_t region;
    float light[4];
};

// A captured batched render: the item list it was captured for (the cache key), the
// context epoch at capture, the graph, and the buffers it owns (stable while it lives).
struct BatchGraph {
    std::vector<rpnn_batch_item> items;
    uint64_t epoch = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t cap = 0;                 // capacity of the compacted query arrays
    int64_t blocks = 0, pixels = 0;  // primary blocks and image pixels of all items
    DevBuf x, d, ps, sample, count, off, desc, g, table, tables;
};

// A captured training step (rpnn_train_step): the configuration it was captured for (the
// cache key, seen once eagerly before capture), the graph, and the staging buffers its
// kernels read the minibatch and Adam's bias corrections from.
struct TrainGraphKey {
    int32_t batch = 0, desc_dtype = 0, precision = 0;
    const void *params = nullptr, *m = nullptr, *v = nullptr, *loss = nullptr;
    float lr = 0, b1 = 0, b2 = 0, eps = 0;
    uint64_t tuner_version = 0, epoch = 0, allocs = 0;
    bool operator==(const TrainGraphKey& o) const {
        return batch == o.batch && desc_dtype == o.desc_dtype && precision == o.precision && params == o.params &&
               m == o.m && v == o.v && loss == o.loss && lr == o.lr && b1 == o.b1 && b2 == o.b2 && eps == o.eps &&
               tuner_version == o.tuner_version && epoch == o.epoch && allocs == o.allocs;
    }
};
struct TrainGraph {
    TrainGraphKey key, seen;
    bool have_seen = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    DevBuf desc, target, adam;        // staged minibatch, {c1, c2} of Adam's bias correction
};

constexpr int kTrainEvents = 25;   // 22 per-layer gradients, fork, two joins

struct Ctx {
    int device = 0;
    int num_sms = 0;
    std::vector<Volume*> vols;
    DevBuf status;           // uint32 status bits
    DevBuf params32;         // FP32 parameters (flat, the documented layout)
    DevBuf wimg_bf16;        // tensor-core weight image
    DevBuf wimg_fp8;         // E4M3 weight image with its scales (after rpnn_calibrate_fp8)
    bool weights_set = false;
    bool fp8_ready = false;  // FP8 image built for the current weights
    // render scratch
    DevBuf q_x, q_d, q_ps, q_count, sample_val, desc, g_out, act0, act1, act2, light;
    // training scratch
    DevBuf t_saved, t_grad, t_dg, t_out, t_loss;
    DevBuf t_lpart;                     // block sums of the loss
    DevBuf t_w16, t_saved16;            // BF16 training: weight image, activation copies
    DevBuf t_gb32, t_gb16;              // BF16 training: per-layer gradients (FP32; BF16 and transposed BF16)
    std::vector<cudaEvent_t> t_events;  // BF16 training: kTrainEvents gradient-ready / fork / join events
    cudaStream_t side_stream[2] = {nullptr, nullptr};   // BF16 training: weight gradients beside the
    DevBuf t_ws2;                       // data-gradient chain; the second stream's split-K workspace
    DevBuf t_desc32;                    // FP32 widening of BF16 training descriptors (FP32 training form)
    int train_precision = RPNN_F32;     // arithmetic of rpnn_train_step / rpnn_mlp_backward
    GemmTuner tuner;
    DevBuf lm_table;         // Lorenz-Mie phase table, uploaded on first use
    DevBuf lmc_table;        // its chopped form, same layout
    std::unordered_map<TmapKey, TmapBytes, TmapKeyHash> tmaps;   // BF16 GEMM operand maps
    // batched render: a captured graph, the stream it is captured on, and an epoch that
    // volume loads, mip builds and weight updates advance (invalidating the graph)
    BatchGraph batch;
    TrainGraph tgraph;               // captured training step
    bool train_graphs = true;        // rpnn_set_train_graphs
    int64_t chunk_rows = 0;          // descriptor/network chunk of a render (0: kChunkRows)
    bool fused = false;              // BF16 renders gather descriptors inside the network kernel
    cudaStream_t capture_stream = nullptr;
    uint64_t epoch = 1;
    // stage timing: one set of 5 events per profiled render
    bool profiling = false;
    std::vector<cudaEvent_t> prof_events;
    size_t prof_used = 0;
    Volume* vol(int id) const {
        return (id >= 0 && id < (int)vols.size()) ? vols[id] : nullptr;
    }
};

// ---- launchers implemented in the .cu files -------------------------------------------
void batch_release(Ctx& c);           // frees the captured batch graph and its buffers
// Batched render helpers (render.cu): the per-item tables of the batched primary, scatter and
// composite kernels (host image of `batch_tables_bytes(n)` bytes, with the primary grid's
// block count and the items' total pixel count), and their launches.
size_t batch_tables_bytes(int n);
void batch_tables(const Ctx& c, const rpnn_batch_item* items, int n, const std::vector<int64_t>& region,
                  std::vector<unsigned char>& out, int64_t* blocks, int64_t* pixels);
rpnn_status launch_primary_batch(Ctx& c, const void* tables, int n, int64_t blocks, float* sample_val, float* qx,
                                 float* qd, uint32_t* qps, int* qcount, cudaStream_t s);
rpnn_status launch_scatter_composite_batch(Ctx& c, const void* tables, int n, int64_t pixels, const float* g,
                                           const uint32_t* qps, const int* off, float* sample_val, cudaStream_t s);
void train_graph_release(Ctx& c);     // frees the captured training step and its buffers
rpnn_status volume_stats(Ctx& c, Volume& v, cudaStream_t s);
rpnn_status volume_brick_majorants(Ctx& c, Volume& v, cudaStream_t s);
rpnn_status volume_build_level(Ctx& c, Volume& v, int level, float* dst, cudaStream_t s);
// levels[0..n-1] into dst[0..n-1] (each [az][ay][ax] FP32), their y and z passes in shared launches
rpnn_status volume_build_levels(Ctx& c, Volume& v, const int* levels, int n, float* const* dst, cudaStream_t s);
rpnn_status volume_pack_levels(Ctx& c, Volume& v, cudaStream_t s);
rpnn_status load_density(Ctx& c, Volume& v, const void* src, int dtype, cudaStream_t s);

rpnn_status launch_descriptor(Ctx& c, const VolumeView& vv, const float* x, const float* d,
                              const float* wl, int wl_stride, int64_t q, const int* q_dev,
                              void* out, int dtype, cudaStream_t s);
// Batched form: compacted query j of item i (off[i] <= j < off[i+1], j < off[n]) reads
// x, d at region_i + j - off[i] and writes descriptor row j.  BF16 output.
// blend: some item's volume blends mip levels (rpnn_set_mip_blend).
rpnn_status launch_descriptor_batch(Ctx& c, const BatchItemDev* items, int n, const float* x, const float* d,
                                    const int* off, int64_t cap, void* out, bool blend, cudaStream_t s);

// Primary stage.  Query outputs (qx, qd, qps, qcount) and inspection outputs (hit, xo,
// dout, Ld; per pixel sample) are each optional.
rpnn_status launch_primary(Ctx& c, const VolumeView& vv, const rpnn_render_desc& rd,
                           float* sample_val, float* qx, float* qd, uint32_t* qps, int* qcount,
                           int* hit, float* xo, float* dout, float* Ld, cudaStream_t s);
// g_off / g_total (device, optional): this render's predictions start at g[*g_off] and
// stop before g[*g_total] (batched renders)
rpnn_status launch_scatter_composite(Ctx& c, const rpnn_render_desc& rd, float alpha,
                                     const float* g, const uint32_t* qps, const int* qcount,
                                     float* sample_val, float* image, bool with_g,
                                     cudaStream_t s, const int* g_off = nullptr,
                                     const int* g_total = nullptr);
// Environment lighting: next-event estimates towards lights j0..n-1 (device dirs [n][3],
// irradiances E [n]) of the *qcount (<= max_q) shading points, added to their samples.
rpnn_status launch_nee_env(Ctx& c, const VolumeView& vv, const rpnn_render_desc& rd, const float* qx,
                           const float* qd, const uint32_t* qps, const int* qcount, int64_t max_q, const float* dirs,
                           const float* E, int j0, int n, float* sample_val, cudaStream_t s);
// Descriptors of an n_xy x n_xy x (2 n_xy - 1) stencil (the stencil-size comparison of
// Sec. 7): FP32 rows [q][RPNN_K][stencil_din(n_xy)], level k's points
// (-1 + h ix, -1 + h iy, -1 + h iz) * 2^(k-1) mean free paths, h = 2 / (n_xy - 1), read from
// the mip level matching that spacing; n_xy = 5 is the standard descriptor.
int stencil_din(int n_xy);
rpnn_status stencil_descriptors(Ctx& c, Volume& v, int n_xy, const float* x, const float* d, const float* wl,
                                int wl_stride, int64_t q, float* out, cudaStream_t s);
// uploads the Lorenz-Mie phase table to c.lm_table once (synchronises s)
rpnn_status phase_lm_upload(Ctx& c, cudaStream_t s);
// fraction of the scattered light in the chopped peak (RPNN_LM_CHOP_BINS bins)
double phase_lm_chop_fraction();
// RPNN_ERR_NONFINITE if any of the n values is NaN or Inf (synchronises s)
rpnn_status check_finite(Ctx& c, const float* p, int64_t n, cudaStream_t s);
// sample_val[qps[i]] += scale * g[i] for i < *qcount
rpnn_status launch_scatter(Ctx& c, float scale, const float* g, const uint32_t* qps, const int* qcount,
                           float* sample_val, cudaStream_t s);
// Rows per descriptor/network chunk of a render.
constexpr int64_t kChunkRows = (int64_t)1 << 20;
// out[i] = clamp(*count - i*rows, 0, rows) for i < n
rpnn_status launch_chunk_counts(Ctx& c, const int* count, int64_t rows, int n, int* out, cudaStream_t s);
rpnn_status launch_records(Ctx& c, const VolumeView& vv, int64_t first, int64_t n,
                           uint64_t seed, float rel_ci, int n_min, int n_max, float* x,
                           float* d, float* wl, float* label, int* npaths, cudaStream_t s);

// FP32 CUDA-core network
rpnn_status mlp_forward_f32(Ctx& c, const float* desc, int64_t q, const int* q_dev,
                            float* out, float* saved, cudaStream_t s);
rpnn_status mlp_backward_f32(Ctx& c, const float* desc, int64_t q, const float* saved,
                             const float* dout, float* dparams, cudaStream_t s);
size_t mlp_saved_floats_per_row();
// block tile (rows, columns, K step) of entry `tile` of the SIMT GEMM tile table
void gemm_tile_shape(int tile, int* bm, int* bn, int* bk);
// index of the tile (bm, bn, bk) in that table, or -1
int gemm_tile_index(int bm, int bn, int bk);
rpnn_status launch_loss(Ctx& c, const float* g, const float* target, int batch, double* loss,
                        float* dg, cudaStream_t s);
rpnn_status launch_adam(float* p, float* m, float* v, const float* grad, int64_t n,
                        int64_t step, const rpnn_adam_cfg& cfg, cudaStream_t s);
// Adam with its bias corrections {1 - b1^step, 1 - b2^step} read from device memory (cc,
// two FP32 values as launch_adam computes them), and the launch that writes them
rpnn_status launch_adam_dev(float* p, float* m, float* v, const float* grad, int64_t n, const float* cc,
                            const rpnn_adam_cfg& cfg, cudaStream_t s);
rpnn_status launch_adam_corrections(float* cc, int64_t step, const rpnn_adam_cfg& cfg, cudaStream_t s);

// BF16 tensor-core GEMM (training): D = epilogue(A0 B0^T + A1 B1^T), A_s [M][K_s] and
// B_s [N][K_s] BF16 with K contiguous (row pitches lda/ldb in elements, multiples of 8;
// 16-byte aligned bases).  The epilogue adds bias [N] and residual, applies ReLU and the
// mask (x * (mask > 0)), and stores any of FP32 C, BF16 Cb and transposed BF16 Ct
// (Ct[n * ldt + m]).  Tile width and split-K are autotuned per shape like the SIMT GEMM.
struct TgSeg {
    const uint16_t* A;
    int64_t lda;
    const uint16_t* B;
    int64_t ldb;
    int K;
};
struct TgOut {
    float* C = nullptr;
    int64_t ldc = 0;
    uint16_t* Cb = nullptr;
    int64_t ldb = 0;
    uint16_t* Ct = nullptr;
    int64_t ldt = 0;
    const float* bias = nullptr;
    const float* res = nullptr;
    int64_t ldr = 0;
    const float* mask = nullptr;
    int64_t ldm = 0;
    int mask_t = 0;                  // mask stored transposed: element (m, n) at mask[n * ldm + m]
    int relu = 0;
};
// split_ws: the split-K workspace (null: the tuner's); GEMMs that may run at the same time
// on different streams need different workspaces
rpnn_status tc_gemm(Ctx& c, int M, int N, const TgSeg& s0, const TgSeg* s1, const TgOut& o, cudaStream_t s,
                    DevBuf* split_ws = nullptr);

// FP32 output layer g = relu(T3 t1 + bT3) and its backward (da3 = dout * (g > 0); dT3, dbT3
// into dP; da2 = (da3 T3) * (t1 > 0)); bias-gradient column sums.  The backward's t1 is
// [q][200] row-major, or (ldt1 > 0) transposed [200][ldt1].
rpnn_status mlp_output_layer_f32(Ctx& c, const float* t1, int64_t q, float* out, cudaStream_t s);
rpnn_status mlp_output_layer_backward_f32(Ctx& c, const float* t1, const float* g, const float* dout, int64_t q,
                                          float* dP, float* da2, cudaStream_t s, int64_t ldt1 = 0);
rpnn_status colsum_f32(Ctx& c, const float* X, int M, int N, float* out, cudaStream_t s);

// Plain ("all-at-once") MLP of the architecture comparison (Sec. 7): n hidden layers of
// widths[i], ReLU everywhere, one ReLU output; FP32 CUDA-core GEMMs
int64_t dense_param_count(const int* widths, int n, int din);
rpnn_status dense_forward(Ctx& c, const int* widths, int n, int din, const float* P, const float* in, int64_t q,
                          float* out, float* saved, cudaStream_t s);
rpnn_status dense_backward(Ctx& c, const int* widths, int n, int din, const float* P, const float* in, int64_t q,
                           const float* saved, const float* dout, float* dP, cudaStream_t s);

// Mixed-precision training form (BF16 tensor-core GEMMs, FP32 master weights and
// activations): saved FP32 slots as mlp_forward_f32, BF16 copies in s16
// (train_bf16_saved_elems(q) elements)
size_t train_bf16_saved_elems(int64_t q);
// FP32 floats of the BF16 training forward's saved activations (22 transposed [200][ldq]
// slots, then g [q])
size_t train_bf16_saved32_floats(int64_t q);
// desc: q rows [10][240] of dtype desc_dtype (RPNN_F32 or RPNN_BF16)
rpnn_status mlp_forward_bf16_train(Ctx& c, const void* desc, int desc_dtype, int64_t q, float* out, float* saved,
                                   uint16_t* s16, cudaStream_t s);
// exact FP32 widening of n BF16 values
rpnn_status launch_bf16_to_f32(const void* in, float* out, int64_t n, int sms, cudaStream_t s);
rpnn_status mlp_backward_bf16_train(Ctx& c, int64_t q, const float* saved, const uint16_t* s16, const float* dout,
                                    float* dP, cudaStream_t s, const cudaStream_t* side = nullptr);

// BF16 tensor-core network
rpnn_status mlp_build_bf16_image(Ctx& c, cudaStream_t s);
// Descriptor gather fused into the BF16 network (the render's two stages in one launch):
// shading points xs / ds ([q][3], or the device count q_dev with capacity q), light wl.
bool fused_supported(const VolumeView& vv);
rpnn_status fused_forward_bf16(Ctx& c, const VolumeView& vv, const float* xs, const float* ds, const float wl[3],
                               int64_t q, const int* q_dev, float* out, cudaStream_t s);
rpnn_status mlp_forward_bf16(Ctx& c, const void* desc_bf16, int64_t q, const int* q_dev,
                             float* out, cudaStream_t s);
// FP8 (E4M3) tensor-core network on [q][10][256] E4M3 descriptors; needs mlp_calibrate_fp8
// The BF16 tensor-core network on descriptor rows as the training forward: FP32 biases,
// every layer's ReLU output stored FP32 at saved + slot * q * 200 and BF16 transposed at
// saved_t + slot * 200 * ldq (slots as the training form's), the prediction in out.
rpnn_status mlp_forward_bf16_saving(Ctx& c, const void* desc_bf16, int64_t q, float* out, float* saved,
                                    uint16_t* saved_t, int64_t ldq, cudaStream_t s);
rpnn_status mlp_forward_fp8(Ctx& c, const void* desc_fp8, int64_t q, const int* q_dev, float* out,
                            cudaStream_t s);
// Per-tensor scales from the FP32 network on q FP32 descriptors [q][10][240]; builds the
// E4M3 weight image (synchronises s)
rpnn_status mlp_calibrate_fp8(Ctx& c, const float* desc, int64_t q, cudaStream_t s);

// parameter layout offsets (floats) of the flat vector
struct ParamLayout {
    int64_t V[RPNN_K], W1[RPNN_K], b1[RPNN_K], W2[RPNN_K], b2[RPNN_K];
    int64_t T[3], bT[3];
    int64_t total;
};
const ParamLayout& param_layout();
ParamLayout param_layout_for(int din);   // the same network with block input width din

// A progressive network's shape: parameter layout, block input width (Sigma^k and gamma)
// and the stored width of one level of a descriptor row.
struct NetDims {
    const ParamLayout* L;
    int din;
    int64_t stride;
};
// The FP32 forward and backward of mlp_forward_f32 / mlp_backward_f32 for any NetDims and
// parameter vector P (the two call these with the standard shape and the context's weights).
// The forward's activations go to `saved` (22 slots of [q][200] and g) or, when it is null,
// to the three [q][200] buffers scr[0..2].  c may be null: every GEMM then runs the default
// tile without split-K and nothing is allocated (tile shapes change no result bit).
rpnn_status rpnn_forward_f32(Ctx* c, const NetDims& nd, const float* P, const float* desc, int64_t q,
                             const int* q_dev, float* out, float* saved, float* const scr[3], cudaStream_t s);
rpnn_status rpnn_backward_f32(Ctx& c, const NetDims& nd, const float* P, const float* desc, int64_t q,
                              const float* saved, const float* dout, float* dP, cudaStream_t s);

}  // namespace rpnn
