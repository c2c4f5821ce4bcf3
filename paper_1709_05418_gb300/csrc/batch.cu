// batch.cu -- batched rendering of several clouds (uneven query counts) as one CUDA graph.
//
// No counterpart in the paper, whose renderer serves one cloud at a time: serving many
// clouds per frame runs every stage once for all of them.  One primary launch (Sec. 4.4)
// covers the pixel samples of all items, each block working on one item and writing its
// queries into that item's region of the per-pixel-sample buffers; a one-thread prefix sum
// turns the per-item counts into offsets of the compacted query list; the descriptor
// (Sec. 4.2) and network (Sec. 4.3) stages run once over that list; one scatter adds every
// item's predictions to its samples and one composite writes every item's image.  The query counts are
// deterministic (Philox-keyed decisions), so the first call runs the primary stages once
// to size the compacted buffers, then captures the whole sequence.
#include <cmath>
#include <cstddef>
#include <cstring>
#include <vector>

#include "internal.h"

namespace rpnn {

namespace {

// off[i] = queries of items 0..i-1; off[n] = total, clamped to the capacity (a status
// bit reports the overflow, which deterministic counts never produce)
__global__ void k_batch_offsets(const int* __restrict__ count, int n, int64_t cap, int* __restrict__ off,
                                uint32_t* status) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    int64_t acc = 0;
    for (int i = 0; i < n; ++i) {
        off[i] = (int)(acc < cap ? acc : cap);
        acc += count[i];
    }
    if (acc > cap) {
        atomicOr(status, kStatCapacity);
        acc = cap;
    }
    off[n] = (int)acc;
}

// the part of rpnn_render_desc that defines a render (its trailing padding excluded)
bool same_desc(const rpnn_render_desc& a, const rpnn_render_desc& b) {
    return std::memcmp(&a, &b, offsetof(rpnn_render_desc, mode) + sizeof(a.mode)) == 0;
}

bool same_items(const std::vector<rpnn_batch_item>& key, const rpnn_batch_item* items, int n) {
    if ((int)key.size() != n) return false;
    for (int i = 0; i < n; ++i)
        if (key[i].vol != items[i].vol || key[i].dev_image != items[i].dev_image ||
            !same_desc(key[i].desc, items[i].desc))
            return false;
    return true;
}

void drop_graph(BatchGraph& B) {
    if (B.exec) cudaGraphExecDestroy(B.exec);
    if (B.graph) cudaGraphDestroy(B.graph);
    B.exec = nullptr;
    B.graph = nullptr;
    B.items.clear();
}

// Enqueues the whole batched render on stream s (captured, or run directly).
rpnn_status enqueue_batch(Ctx& c, const rpnn_batch_item* items, int n, cudaStream_t s) {
    BatchGraph& B = c.batch;
    int* count = B.count.as<int>();
    int* off = B.off.as<int>();
    RPNN_CUDA_TRY(cudaMemsetAsync(count, 0, n * sizeof(int), s));
    rpnn_status st = launch_primary_batch(c, B.tables.p, n, B.blocks, B.sample.as<float>(), B.x.as<float>(),
                                          B.d.as<float>(), B.ps.as<uint32_t>(), count, s);
    if (st) return st;
    k_batch_offsets<<<1, 32, 0, s>>>(count, n, B.cap, off, c.status.as<uint32_t>());
    RPNN_CHECK_LAUNCH();
    bool blend = false;
    for (int i = 0; i < n; ++i) blend |= c.vol(items[i].vol)->mip_blend;
    st = launch_descriptor_batch(c, B.table.as<BatchItemDev>(), n, B.x.as<float>(), B.d.as<float>(),
                                             off, B.cap, B.desc.p, blend, s);
    if (st) return st;
    st = mlp_forward_bf16(c, B.desc.p, B.cap, off + n, B.g.as<float>(), s);
    if (st) return st;
    return launch_scatter_composite_batch(c, B.tables.p, n, B.pixels, B.g.as<float>(), B.ps.as<uint32_t>(), off,
                                          B.sample.as<float>(), s);
}

// Sizes the buffers for this item list, learns the query counts with one direct run of
// the primary stages, and captures the batched render as a graph.
rpnn_status build_batch(Ctx& c, const rpnn_batch_item* items, int n, cudaStream_t s) {
    BatchGraph& B = c.batch;
    drop_graph(B);
    std::vector<int64_t> region(n);
    int64_t P = 0;
    for (int i = 0; i < n; ++i) {
        region[i] = P;
        P += (int64_t)items[i].desc.width * items[i].desc.height * items[i].desc.spp;
    }
    if (P > ((int64_t)1 << 31) - 1) { set_error("batch of %lld pixel samples is too large", (long long)P); return RPNN_ERR_ARG; }
    rpnn_status st = B.x.reserve(P * 3 * sizeof(float));
    if (!st) st = B.d.reserve(P * 3 * sizeof(float));
    if (!st) st = B.ps.reserve(P * sizeof(uint32_t));
    if (!st) st = B.sample.reserve(P * sizeof(float));
    if (!st) st = B.count.reserve(RPNN_MAX_BATCH * sizeof(int));
    if (!st) st = B.off.reserve((RPNN_MAX_BATCH + 1) * sizeof(int));
    if (!st) st = B.table.reserve(RPNN_MAX_BATCH * sizeof(BatchItemDev));
    if (!st) st = B.tables.reserve(batch_tables_bytes(RPNN_MAX_BATCH));
    if (st) return st;
    // the items' tables for the batched primary, scatter and composite kernels
    std::vector<unsigned char> ht;
    batch_tables(c, items, n, region, ht, &B.blocks, &B.pixels);
    RPNN_CUDA_TRY(cudaMemcpyAsync(B.tables.p, ht.data(), ht.size(), cudaMemcpyHostToDevice, s));
    // query counts of this item list
    int* count = B.count.as<int>();
    RPNN_CUDA_TRY(cudaMemsetAsync(count, 0, n * sizeof(int), s));
    st = launch_primary_batch(c, B.tables.p, n, B.blocks, B.sample.as<float>(), B.x.as<float>(), B.d.as<float>(),
                              B.ps.as<uint32_t>(), count, s);
    if (st) return st;
    std::vector<int> h(n);
    RPNN_CUDA_TRY(cudaMemcpyAsync(h.data(), count, n * sizeof(int), cudaMemcpyDeviceToHost, s));
    RPNN_CUDA_TRY(cudaStreamSynchronize(s));
    int64_t total = 0;
    for (int i = 0; i < n; ++i) total += h[i];
    B.cap = ((total > 0 ? total : 1) + 127) / 128 * 128;
    st = B.desc.reserve((size_t)B.cap * RPNN_K * RPNN_DESC_STRIDE * 2);
    if (!st) st = B.g.reserve((size_t)B.cap * sizeof(float));
    if (st) return st;
    std::vector<BatchItemDev> table(n);
    for (int i = 0; i < n; ++i) {
        table[i].v = c.vol(items[i].vol)->view();
        table[i].region = region[i];
        for (int a = 0; a < 3; ++a) table[i].light[a] = items[i].desc.light_dir[a];
        table[i].light[3] = 0.0f;
    }
    RPNN_CUDA_TRY(cudaMemcpy(B.table.p, table.data(), n * sizeof(BatchItemDev), cudaMemcpyHostToDevice));
    // capture on the library's own stream (the caller's may be the legacy default stream)
    if (!c.capture_stream) RPNN_CUDA_TRY(cudaStreamCreateWithFlags(&c.capture_stream, cudaStreamNonBlocking));
    cudaStream_t cs = c.capture_stream;
    RPNN_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    const rpnn_status est = enqueue_batch(c, items, n, cs);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(cs, &graph);
    if (est) {
        if (graph) cudaGraphDestroy(graph);
        return est;
    }
    if (ce != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        set_error("stream capture of the batched render failed: %s", cudaGetErrorString(ce));
        return RPNN_ERR_CUDA;
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    if (ie != cudaSuccess) {
        cudaGraphDestroy(graph);
        set_error("graph instantiation failed: %s", cudaGetErrorString(ie));
        return RPNN_ERR_CUDA;
    }
    B.graph = graph;
    B.exec = exec;
    B.items.assign(items, items + n);
    B.epoch = c.epoch;
    return RPNN_OK;
}

}  // namespace

void batch_release(Ctx& c) {
    BatchGraph& B = c.batch;
    drop_graph(B);
    DevBuf* bufs[] = {&B.x, &B.d, &B.ps, &B.sample, &B.count, &B.off, &B.desc, &B.g, &B.table, &B.tables};
    for (DevBuf* b : bufs) b->release();
}

}  // namespace rpnn

using namespace rpnn;

extern "C" rpnn_status rpnn_render_batch(rpnn_ctx* ctx, const rpnn_batch_item* items, int32_t n_items,
                                         int64_t* out_num_queries, void* stream) {
    if (!ctx) { set_error("null context"); return RPNN_ERR_HANDLE; }
    set_error("%s", "");
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (!items || n_items < 1 || n_items > RPNN_MAX_BATCH) {
        set_error("a batch holds 1 to %d items, got %d", RPNN_MAX_BATCH, n_items);
        return RPNN_ERR_ARG;
    }
    if (!c->weights_set) { set_error("rpnn_set_weights has not run"); return RPNN_ERR_STATE; }
    for (int i = 0; i < n_items; ++i) {
        const rpnn_batch_item& it = items[i];
        const Volume* v = c->vol(it.vol);
        if (!v) { set_error("item %d: no volume %d", i, it.vol); return RPNN_ERR_HANDLE; }
        if (!v->built) { set_error("item %d: volume %d: rpnn_build_mips has not run", i, it.vol); return RPNN_ERR_HANDLE; }
        const rpnn_render_desc& d = it.desc;
        if (d.width <= 0 || d.height <= 0 || d.spp <= 0 || (int64_t)d.width * d.height * d.spp > ((int64_t)1 << 31) - 1) {
            set_error("item %d: bad image size", i);
            return RPNN_ERR_ARG;
        }
        if (d.mode != RPNN_MODE_RPNN || d.precision != RPNN_BF16) {
            set_error("item %d: a batch renders RPNN_MODE_RPNN with RPNN_BF16 precision", i);
            return RPNN_ERR_ARG;
        }
        const float l2 = d.light_dir[0] * d.light_dir[0] + d.light_dir[1] * d.light_dir[1] + d.light_dir[2] * d.light_dir[2];
        if (!(fabsf(l2 - 1.0f) < 1e-4f)) { set_error("item %d: light_dir must be unit length", i); return RPNN_ERR_ARG; }
        if (!it.dev_image) { set_error("item %d: dev_image is null", i); return RPNN_ERR_ARG; }
    }
    cudaStream_t s = (cudaStream_t)stream;
    BatchGraph& B = c->batch;
    if (!(B.exec && B.epoch == c->epoch && same_items(B.items, items, n_items))) {
        const rpnn_status st = build_batch(*c, items, n_items, s);
        if (st) { drop_graph(B); return st; }
    }
    RPNN_CUDA_TRY(cudaGraphLaunch(B.exec, s));
    if (out_num_queries) {
        int h[RPNN_MAX_BATCH];
        RPNN_CUDA_TRY(cudaMemcpyAsync(h, B.count.p, n_items * sizeof(int), cudaMemcpyDeviceToHost, s));
        RPNN_CUDA_TRY(cudaStreamSynchronize(s));
        for (int i = 0; i < n_items; ++i) out_num_queries[i] = h[i];
    }
    return RPNN_OK;
}
