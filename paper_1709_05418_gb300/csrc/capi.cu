// capi.cu -- the C ABI declared in include/rpnn.h: argument checks, ownership, and the
// sequencing of the kernels of each call.
#include <atomic>
#include <cstdarg>
#include <cstring>
#include <new>

#include "common.cuh"

namespace rpnn {

namespace {
thread_local char g_err[1024] = "";
}

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}

static std::atomic<uint64_t> g_devbuf_generation{1};
uint64_t devbuf_generation() { return g_devbuf_generation.load(); }

rpnn_status DevBuf::reserve(size_t n) {
    if (n <= bytes) return RPNN_OK;
    ++g_devbuf_generation;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    // round up to 2 MiB so repeated growth settles quickly
    const size_t want = (n + (2u << 20) - 1) & ~(size_t)((2u << 20) - 1);
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) {
        p = nullptr;
        set_error("cudaMalloc(%zu) failed: %s", want, cudaGetErrorString(e));
        return RPNN_ERR_OOM;
    }
    bytes = want;
    return RPNN_OK;
}

void DevBuf::release() {
    if (p) ++g_devbuf_generation;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
}

}  // namespace rpnn

using namespace rpnn;

namespace {
// Training descriptors as the training precision reads them: the BF16 form reads FP32 or
// BF16 rows itself; the FP32 form reads FP32 rows, so BF16 rows are widened (exactly) into
// context scratch first.  *d32 is the FP32 view (null for the BF16 form).
rpnn_status train_desc(Ctx& c, const void* desc, int dtype, int64_t q, const float** d32, cudaStream_t s) {
    *d32 = nullptr;
    if (c.train_precision == RPNN_BF16) return RPNN_OK;
    if (dtype == RPNN_F32) { *d32 = static_cast<const float*>(desc); return RPNN_OK; }
    const int64_t n = q * RPNN_K * RPNN_DESC_STRIDE;
    rpnn_status st = c.t_desc32.reserve((size_t)n * sizeof(float));
    if (st) return st;
    st = launch_bf16_to_f32(desc, c.t_desc32.as<float>(), n, c.num_sms, s);
    if (st) return st;
    *d32 = c.t_desc32.as<float>();
    return RPNN_OK;
}

// Forward with saved activations in the context's training precision (FP32 CUDA cores,
// or BF16 tensor-core GEMMs with FP32 master weights); the prediction goes to t_out.
rpnn_status train_forward(Ctx& c, const void* desc, int dtype, const float* d32, int64_t q, cudaStream_t s) {
    const size_t saved = c.train_precision == RPNN_BF16 ? train_bf16_saved32_floats(q)
                                                        : mlp_saved_floats_per_row() * (size_t)q;
    rpnn_status st = c.t_saved.reserve(saved * sizeof(float));
    if (!st) st = c.t_out.reserve(q * sizeof(float));
    if (st) return st;
    if (c.train_precision == RPNN_BF16) {
        st = c.t_saved16.reserve(train_bf16_saved_elems(q) * 2);
        if (st) return st;
        return mlp_forward_bf16_train(c, desc, dtype, q, c.t_out.as<float>(), c.t_saved.as<float>(),
                                      c.t_saved16.as<uint16_t>(), s);
    }
    return mlp_forward_f32(c, d32, q, nullptr, c.t_out.as<float>(), c.t_saved.as<float>(), s);
}

// side: a second stream for the BF16 weight gradients (null: everything on s)
rpnn_status train_backward(Ctx& c, const float* d32, int64_t q, const float* dout, float* dP, cudaStream_t s,
                           const cudaStream_t* side = nullptr) {
    if (c.train_precision == RPNN_BF16)
        return mlp_backward_bf16_train(c, q, c.t_saved.as<float>(), c.t_saved16.as<uint16_t>(), dout, dP, s, side);
    return mlp_backward_f32(c, d32, q, c.t_saved.as<float>(), dout, dP, s);
}

rpnn_status check_train_desc(const void* desc, int dtype) {
    (void)desc;
    if (dtype != RPNN_F32 && dtype != RPNN_BF16) { set_error("training descriptors must be F32 or BF16"); return RPNN_ERR_ARG; }
    return RPNN_OK;
}
}  // namespace

#define CHECK_CTX(ctx)                                                        \
    do {                                                                      \
        if (!(ctx)) { set_error("null context"); return RPNN_ERR_HANDLE; }    \
        g_err_clear();                                                        \
    } while (0)

static void g_err_clear() { set_error("%s", ""); }

static Volume* get_vol(Ctx* c, int id, bool need_built) {
    Volume* v = c->vol(id);
    if (!v) { set_error("unknown volume id %d", id); return nullptr; }
    if (need_built && !v->built) { set_error("volume %d: rpnn_build_mips has not run", id); return nullptr; }
    return v;
}

extern "C" {

rpnn_status rpnn_create(rpnn_ctx** out) {
    if (!out) { set_error("out is null"); return RPNN_ERR_ARG; }
    Ctx* c = new (std::nothrow) Ctx();
    if (!c) { set_error("host allocation failed"); return RPNN_ERR_OOM; }
    RPNN_CUDA_TRY(cudaGetDevice(&c->device));
    RPNN_CUDA_TRY(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
    rpnn_status st = c->status.reserve(sizeof(uint32_t));
    if (st) { delete c; return st; }
    RPNN_CUDA_TRY(cudaMemset(c->status.p, 0, sizeof(uint32_t)));
    *out = reinterpret_cast<rpnn_ctx*>(c);
    return RPNN_OK;
}

rpnn_status rpnn_destroy(rpnn_ctx* ctx) {
    if (!ctx) return RPNN_OK;
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    cudaDeviceSynchronize();
    for (Volume* v : c->vols) {
        if (!v) continue;
        v->raw.release(); v->packed.release(); v->stats.release(); v->bmaj.release();
        v->mip_a.release(); v->mip_b.release(); v->mip_w.release(); v->mip_d.release(); v->stencil_mips.release();
        delete v;
    }
    DevBuf* bufs[] = {&c->status, &c->params32, &c->wimg_bf16, &c->wimg_fp8, &c->q_x, &c->q_d, &c->q_ps,
                      &c->q_count, &c->sample_val, &c->desc, &c->g_out, &c->act0, &c->act1,
                      &c->act2, &c->t_saved, &c->t_grad, &c->t_dg, &c->t_out, &c->t_loss, &c->t_lpart, &c->light,
                      &c->tuner.scratch, &c->tuner.ws, &c->t_w16, &c->t_saved16, &c->t_gb32, &c->t_gb16, &c->t_ws2, &c->t_desc32, &c->lm_table, &c->lmc_table};
    for (DevBuf* b : bufs) b->release();
    if (c->tuner.ev0) cudaEventDestroy(c->tuner.ev0);
    if (c->tuner.ev1) cudaEventDestroy(c->tuner.ev1);
    batch_release(*c);
    train_graph_release(*c);
    if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
    for (cudaStream_t ss : c->side_stream)
        if (ss) cudaStreamDestroy(ss);
    for (cudaEvent_t e : c->t_events) cudaEventDestroy(e);
    for (cudaEvent_t e : c->prof_events) cudaEventDestroy(e);
    delete c;
    return RPNN_OK;
}

const char* rpnn_last_error(void) { return g_err; }

rpnn_status rpnn_sync_status(rpnn_ctx* ctx, void* stream) {
    CHECK_CTX(ctx);
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t h = 0;
    RPNN_CUDA_TRY(cudaMemcpyAsync(&h, c->status.p, sizeof h, cudaMemcpyDeviceToHost, s));
    RPNN_CUDA_TRY(cudaMemsetAsync(c->status.p, 0, sizeof h, s));
    RPNN_CUDA_TRY(cudaStreamSynchronize(s));
    if (h & kStatIterLimit) { set_error("a device loop reached its iteration cap"); return RPNN_ERR_ITER_LIMIT; }
    if (h & kStatNonFinite) { set_error("non-finite value met on the device"); return RPNN_ERR_NONFINITE; }
    if (h & kStatTimeout) { set_error("a tensor-core pipeline wait timed out; its results are invalid"); return RPNN_ERR_TIMEOUT; }
    if (h & kStatCapacity) { set_error("batched render: more shading points than its captured capacity"); return RPNN_ERR_STATE; }
    return RPNN_OK;
}

rpnn_status rpnn_load_volume(rpnn_ctx* ctx, const void* dev_density, int32_t dtype, int32_t nx,
                             int32_t ny, int32_t nz, float albedo, float hg_g, int32_t* out_vol,
                             void* stream) {
    CHECK_CTX(ctx);
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (!dev_density || !out_vol) { set_error("null pointer"); return RPNN_ERR_ARG; }
    if (dtype != RPNN_F32 && dtype != RPNN_F16) { set_error("density dtype must be F32 or F16"); return RPNN_ERR_ARG; }
    if (nx <= 0 || ny <= 0 || nz <= 0 || nx > 8192 || ny > 8192 || nz > 8192 ||
        (int64_t)nx * ny * nz > (int64_t)1 << 33) {
        set_error("bad grid size %d x %d x %d", nx, ny, nz);
        return RPNN_ERR_ARG;
    }
    if (!(albedo >= 0.0f && albedo <= 1.0f) || !(hg_g > -1.0f && hg_g < 1.0f)) {
        set_error("albedo must be in [0,1] and hg_g in (-1,1)");
        return RPNN_ERR_ARG;
    }
    Volume* v = new (std::nothrow) Volume();
    if (!v) { set_error("host allocation failed"); return RPNN_ERR_OOM; }
    v->n[0] = nx; v->n[1] = ny; v->n[2] = nz;
    v->albedo = albedo; v->g = hg_g;
    rpnn_status st = load_density(*c, *v, dev_density, dtype, (cudaStream_t)stream);
    if (st) { v->raw.release(); delete v; return st; }
    c->vols.push_back(v);
    *out_vol = (int32_t)c->vols.size() - 1;
    ++c->epoch;
    return RPNN_OK;
}

rpnn_status rpnn_build_mips(rpnn_ctx* ctx, int32_t vol, void* stream) {
    CHECK_CTX(ctx);
    NvtxRange range("rpnn_build_mips");
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    Volume* v = get_vol(c, vol, false);
    if (!v) return RPNN_ERR_HANDLE;
    cudaStream_t s = (cudaStream_t)stream;
    ++c->epoch;
    rpnn_status st = volume_stats(*c, *v, s);
    if (!st) st = volume_brick_majorants(*c, *v, s);
    if (st) return st;
    return volume_pack_levels(*c, *v, s);
}

rpnn_status rpnn_get_volume_info(rpnn_ctx* ctx, int32_t vol, rpnn_volume_info* out) {
    CHECK_CTX(ctx);
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    Volume* v = get_vol(c, vol, true);
    if (!v) return RPNN_ERR_HANDLE;
    if (!out) { set_error("out is null"); return RPNN_ERR_ARG; }
    *out = v->info;
    return RPNN_OK;
}

rpnn_status rpnn_set_phase_function(rpnn_ctx* ctx, int32_t vol, int32_t kind) {
    CHECK_CTX(ctx);
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    Volume* v = get_vol(c, vol, false);
    if (!v) return RPNN_ERR_HANDLE;
    if (kind != RPNN_PHASE_HG && kind != RPNN_PHASE_LORENZ_MIE && kind != RPNN_PHASE_LORENZ_MIE_CHOPPED) {
        set_error("unknown phase function %d", kind);
        return RPNN_ERR_ARG;
    }
    v->lm = v->lmc = nullptr;
    v->dscale = 1.0f;
    v->albedo_c = 0.0f;
    if (kind != RPNN_PHASE_HG) {
        rpnn_status st = phase_lm_upload(*c, nullptr);
        if (st) return st;
        v->lm = c->lm_table.as<float>();
        v->lmc = v->lm;
    }
    if (kind == RPNN_PHASE_LORENZ_MIE_CHOPPED) {
        const double f = phase_lm_chop_fraction(), a = (double)v->albedo;
        v->lmc = c->lmc_table.as<float>();
        v->dscale = (float)(1.0 - f * a);
        v->albedo_c = (float)(a * (1.0 - f) / (1.0 - f * a));
    }
    ++c->epoch;
    return RPNN_OK;
}

rpnn_status rpnn_set_iteration_cap(rpnn_ctx* ctx, int32_t vol, int64_t cap) {
    CHECK_CTX(ctx);
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    Volume* v = get_vol(c, vol, false);
    if (!v) return RPNN_ERR_HANDLE;
    if (cap < 0 || cap > 0xFFFFFFFFll) { set_error("cap must be in [0, 2^32)"); return RPNN_ERR_ARG; }
    v->track_cap = (uint32_t)cap;
    ++c->epoch;
    return RPNN_OK;
}

rpnn_status rpnn_set_mip_blend(rpnn_ctx* ctx, int32_t vol, int32_t on) {
    CHECK_CTX(ctx);
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    Volume* v = get_vol(c, vol, false);
    if (!v) return RPNN_ERR_HANDLE;
    v->mip_blend = on != 0;
    ++c->epoch;                      // captured batch renders hold the volume's view
    return RPNN_OK;
}

rpnn_status rpnn_copy_brick_majorants(rpnn_ctx* ctx, int32_t vol, float* dev_out, void* stream) {
    CHECK_CTX(ctx);
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    Volume* v = get_vol(c, vol, true);
    if (!v) return RPNN_ERR_HANDLE;
    if (!dev_out) { set_error("dev_out is null"); return RPNN_ERR_ARG; }
    RPNN_CUDA_TRY(cudaMemcpyAsync(dev_out, v->bmaj.p, (size_t)v->nb[0] * v->nb[1] * v->nb[2] * sizeof(float),
                                  cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return RPNN_OK;
}

rpnn_status rpnn_copy_mip_level(rpnn_ctx* ctx, int32_t vol, int32_t level, float* dev_out, void* stream) {
    CHECK_CTX(ctx);
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    Volume* v = get_vol(c, vol, true);
    if (!v) return RPNN_ERR_HANDLE;
    if (!dev_out) { set_error("dev_out is null"); return RPNN_ERR_ARG; }
    return volume_build_level(*c, *v, level, dev_out, (cudaStream_t)stream);
}

rpnn_status rpnn_set_weights(rpnn_ctx* ctx, const float* dev_params, int64_t n_params, void* stream) {
    CHECK_CTX(ctx);
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (!dev_params) { set_error("dev_params is null"); return RPNN_ERR_ARG; }
    if (n_params != RPNN_NPARAMS) {
        set_error("expected %d parameters, got %lld", RPNN_NPARAMS, (long long)n_params);
        return RPNN_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    rpnn_status st = c->params32.reserve(n_params * sizeof(float));
    if (st) return st;
    // a NaN or Inf parameter is rejected before it reaches any weight copy (synchronises s)
    st = check_finite(*c, dev_params, n_params, s);
    if (st) return st;
    RPNN_CUDA_TRY(cudaMemcpyAsync(c->params32.p, dev_params, n_params * sizeof(float),
                                  cudaMemcpyDeviceToDevice, s));
    st = mlp_build_bf16_image(*c, s);
    if (st) return st;
    c->weights_set = true;
    c->fp8_ready = false;
    ++c->epoch;
    return RPNN_OK;
}

rpnn_status rpnn_extract_descriptors(rpnn_ctx* ctx, int32_t vol, const float* dev_x, const float* dev_d,
                                     const float* dev_wl, int32_t wl_stride, int64_t q, void* dev_desc,
                                     int32_t desc_dtype, void* stream) {
    CHECK_CTX(ctx);
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    Volume* v = get_vol(c, vol, true);
    if (!v) return RPNN_ERR_HANDLE;
    if (q < 0) { set_error("q < 0"); return RPNN_ERR_ARG; }
    if (q == 0) return RPNN_OK;
    if (!dev_x || !dev_d || !dev_wl || !dev_desc) { set_error("null pointer"); return RPNN_ERR_ARG; }
    if (wl_stride != 0 && wl_stride != 3) { set_error("wl_stride must be 0 or 3"); return RPNN_ERR_ARG; }
    if (desc_dtype != RPNN_F32 && desc_dtype != RPNN_BF16 && desc_dtype != RPNN_FP8E4M3) {
        set_error("desc dtype must be F32, BF16 or FP8E4M3");
        return RPNN_ERR_ARG;
    }
    if ((reinterpret_cast<uintptr_t>(dev_desc) & 15u) != 0) { set_error("dev_desc must be 16-byte aligned"); return RPNN_ERR_ARG; }
    return launch_descriptor(*c, v->view(), dev_x, dev_d, dev_wl, wl_stride, q, nullptr, dev_desc,
                             desc_dtype, (cudaStream_t)stream);
}

static rpnn_status ensure_rows(Ctx* c, int64_t q, bool f32_net) {
    rpnn_status st = RPNN_OK;
    if (f32_net) {
        const size_t b = (size_t)q * RPNN_H * sizeof(float);
        if (!st) st = c->act0.reserve(b);
        if (!st) st = c->act1.reserve(b);
        if (!st) st = c->act2.reserve(b);
    }
    return st;
}

rpnn_status rpnn_mlp_forward(rpnn_ctx* ctx, const void* dev_desc, int32_t desc_dtype, int64_t q,
                             int32_t precision, float* dev_out, void* stream) {
    CHECK_CTX(ctx);
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (!c->weights_set) { set_error("rpnn_set_weights has not run"); return RPNN_ERR_STATE; }
    if (q < 0) { set_error("q < 0"); return RPNN_ERR_ARG; }
    if (q == 0) return RPNN_OK;
    if (!dev_desc || !dev_out) { set_error("null pointer"); return RPNN_ERR_ARG; }
    if (q > (int64_t)1 << 30) { set_error("q too large"); return RPNN_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == RPNN_F32) {
        if (desc_dtype != RPNN_F32) { set_error("the FP32 network reads FP32 descriptors"); return RPNN_ERR_ARG; }
        rpnn_status st = ensure_rows(c, q, true);
        if (st) return st;
        return mlp_forward_f32(*c, (const float*)dev_desc, q, nullptr, dev_out, nullptr, s);
    }
    if (precision == RPNN_BF16) {
        if (desc_dtype != RPNN_BF16) { set_error("the BF16 network reads BF16 descriptors"); return RPNN_ERR_ARG; }
        return mlp_forward_bf16(*c, dev_desc, q, nullptr, dev_out, s);
    }
    if (precision == RPNN_FP8E4M3) {
        if (desc_dtype != RPNN_FP8E4M3) { set_error("the FP8 network reads E4M3 descriptors"); return RPNN_ERR_ARG; }
        return mlp_forward_fp8(*c, dev_desc, q, nullptr, dev_out, s);
    }
    set_error("precision must be RPNN_F32, RPNN_BF16 or RPNN_FP8E4M3");
    return RPNN_ERR_ARG;
}

rpnn_status rpnn_calibrate_fp8(rpnn_ctx* ctx, const float* dev_desc, int64_t q, void* stream) {
    CHECK_CTX(ctx);
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (!c->weights_set) { set_error("rpnn_set_weights has not run"); return RPNN_ERR_STATE; }
    if (!dev_desc || q < 1) { set_error("calibration needs q >= 1 descriptor rows"); return RPNN_ERR_ARG; }
    if (q > (int64_t)1 << 24) { set_error("q too large"); return RPNN_ERR_ARG; }
    rpnn_status st = ensure_rows(c, q, true);
    if (st) return st;
    return mlp_calibrate_fp8(*c, dev_desc, q, (cudaStream_t)stream);
}

static rpnn_status check_desc(const rpnn_render_desc* d) {
    if (!d) { set_error("desc is null"); return RPNN_ERR_ARG; }
    if (d->width <= 0 || d->height <= 0 || d->spp <= 0 ||
        (int64_t)d->width * d->height * d->spp > ((int64_t)1 << 31) - 1) {
        set_error("bad image size %d x %d x %d spp", d->width, d->height, d->spp);
        return RPNN_ERR_ARG;
    }
    if (d->mode < RPNN_MODE_RPNN || d->mode > RPNN_MODE_PATH) { set_error("bad mode"); return RPNN_ERR_ARG; }
    if (d->precision != RPNN_F32 && d->precision != RPNN_BF16 && d->precision != RPNN_FP8E4M3) {
        set_error("bad precision");
        return RPNN_ERR_ARG;
    }
    const float l2 = d->light_dir[0] * d->light_dir[0] + d->light_dir[1] * d->light_dir[1] +
                     d->light_dir[2] * d->light_dir[2];
    if (!(fabsf(l2 - 1.0f) < 1e-4f)) { set_error("light_dir must be unit length"); return RPNN_ERR_ARG; }
    return RPNN_OK;
}

rpnn_status rpnn_trace_primary(rpnn_ctx* ctx, int32_t vol, const rpnn_render_desc* desc, int32_t* dev_hit,
                               float* dev_x, float* dev_d, float* dev_Ld, void* stream) {
    CHECK_CTX(ctx);
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    Volume* v = get_vol(c, vol, true);
    if (!v) return RPNN_ERR_HANDLE;
    rpnn_status st = check_desc(desc);
    if (st) return st;
    if (!dev_hit || !dev_x || !dev_d || !dev_Ld) { set_error("null pointer"); return RPNN_ERR_ARG; }
    return launch_primary(*c, v->view(), *desc, nullptr, nullptr, nullptr, nullptr, nullptr, dev_hit,
                          dev_x, dev_d, dev_Ld, (cudaStream_t)stream);
}

// One render: the camera and light of `desc`, or (n_env > 0) the n_env directional lights
// env_dir [n][3] / env_E [n] (host) in place of desc's light (environment lighting).
static rpnn_status render_impl(Ctx* c, int32_t vol, const rpnn_render_desc* desc, const float* env_dir,
                               const float* env_E, int n_env, float* dev_image, int64_t* out_num_queries,
                               cudaStream_t s) {
    NvtxRange range(n_env > 0 ? "rpnn_render_env" : "rpnn_render");
    Volume* v = get_vol(c, vol, true);
    if (!v) return RPNN_ERR_HANDLE;
    rpnn_status st = check_desc(desc);
    if (st) return st;
    if (!dev_image) { set_error("dev_image is null"); return RPNN_ERR_ARG; }
    const bool net = desc->mode == RPNN_MODE_RPNN;
    if (net && !c->weights_set) { set_error("rpnn_set_weights has not run"); return RPNN_ERR_STATE; }
    if (net && desc->precision == RPNN_FP8E4M3 && !c->fp8_ready) {
        set_error("FP8 render: rpnn_calibrate_fp8 has not run since the weights were set");
        return RPNN_ERR_STATE;
    }
    // the lights: desc's one, or the environment's directions
    const int nl = n_env > 0 ? n_env : 1;
    std::vector<float> lights(4 * (size_t)nl);
    for (int j = 0; j < nl; ++j)
        for (int a = 0; a < 3; ++a) lights[3 * j + a] = n_env > 0 ? env_dir[3 * j + a] : desc->light_dir[a];
    for (int j = 0; j < nl; ++j) lights[3 * nl + j] = n_env > 0 ? env_E[j] : desc->light_E;
    rpnn_render_desc rd0 = *desc;                   // the primary pass carries light 0
    for (int a = 0; a < 3; ++a) rd0.light_dir[a] = lights[a];
    rd0.light_E = lights[3 * nl];
    const bool queries = net || nl > 1;             // shading points are listed for the network or extra lights
    const int64_t P = (int64_t)desc->width * desc->height * desc->spp;
    const bool f32 = desc->precision == RPNN_F32;
    const bool fp8 = desc->precision == RPNN_FP8E4M3;
    // BF16: descriptor and network in one kernel, no descriptor rows in memory
    const bool fused = net && !f32 && !fp8 && c->fused && fused_supported(v->view());
    const size_t desc_row_bytes = fp8 ? (size_t)RPNN_K * RPNN_DESC_STRIDE_FP8 : (size_t)RPNN_K * RPNN_DESC_STRIDE * (f32 ? 4 : 2);
    // the descriptor and network stages run over chunks of at most kChunkRows queries, so
    // the descriptor buffer stays bounded (5 GB BF16) for renders of millions of samples
    const int64_t CH = std::min<int64_t>(P, c->chunk_rows > 0 ? c->chunk_rows : kChunkRows);
    const int nchunks = (int)((P + CH - 1) / CH);
    st = c->sample_val.reserve(P * sizeof(float));
    if (!st) st = c->q_count.reserve((1 + nchunks) * sizeof(int));
    if (!st) st = c->light.reserve(lights.size() * sizeof(float));
    if (queries) {
        if (!st) st = c->q_x.reserve(P * 3 * sizeof(float));
        if (!st) st = c->q_d.reserve(P * 3 * sizeof(float));
        if (!st) st = c->q_ps.reserve(P * sizeof(uint32_t));
    }
    if (net) {
        if (!st) st = c->g_out.reserve(P * sizeof(float));
        if (!st && !fused) st = c->desc.reserve((size_t)CH * desc_row_bytes);
        if (!st) st = ensure_rows(c, CH, f32);
    }
    if (st) return st;
    const VolumeView vv = v->view();
    int* qc = c->q_count.as<int>();
    cudaEvent_t* ev = nullptr;
    if (c->profiling) {
        if (c->prof_events.size() < (c->prof_used + 1) * 5) {
            for (int i = 0; i < 5; ++i) {
                cudaEvent_t e;
                RPNN_CUDA_TRY(cudaEventCreate(&e));
                c->prof_events.push_back(e);
            }
        }
        ev = &c->prof_events[c->prof_used * 5];
        ++c->prof_used;
        RPNN_CUDA_TRY(cudaEventRecord(ev[0], s));
    }
    // light directions (device, [nl][3]) then irradiances ([nl]), read by the descriptor
    // and environment next-event kernels
    RPNN_CUDA_TRY(cudaMemcpyAsync(c->light.p, lights.data(), lights.size() * sizeof(float), cudaMemcpyHostToDevice, s));
    const float* ldir = c->light.as<float>();
    RPNN_CUDA_TRY(cudaMemsetAsync(qc, 0, sizeof(int), s));
    {
        NvtxRange stage("primary");
        st = launch_primary(*c, vv, rd0, c->sample_val.as<float>(), queries ? c->q_x.as<float>() : nullptr,
                            queries ? c->q_d.as<float>() : nullptr, queries ? c->q_ps.as<uint32_t>() : nullptr,
                            queries ? qc : nullptr, nullptr, nullptr, nullptr, nullptr, s);
        if (st) return st;
        if (nl > 1) {
            st = launch_nee_env(*c, vv, rd0, c->q_x.as<float>(), c->q_d.as<float>(), c->q_ps.as<uint32_t>(), qc, P,
                                ldir, ldir + 3 * nl, 1, nl, c->sample_val.as<float>(), s);
            if (st) return st;
        }
    }
    if (ev) RPNN_CUDA_TRY(cudaEventRecord(ev[1], s));
    if (!net && ev) {
        RPNN_CUDA_TRY(cudaEventRecord(ev[2], s));
        RPNN_CUDA_TRY(cudaEventRecord(ev[3], s));
    }
    if (net) {
        // per-chunk query counts (device): clamp(count - i*CH, 0, CH)
        if (nchunks > 1) {
            st = launch_chunk_counts(*c, qc, CH, nchunks, qc + 1, s);
            if (st) return st;
        }
        NvtxRange stage("descriptor+network");
        for (int j = 0; j < nl; ++j) {
            for (int i = 0; i < nchunks; ++i) {
                const int* cnt = nchunks > 1 ? qc + 1 + i : qc;
                const int64_t first = (int64_t)i * CH;
                if (fused) {
                    if (ev && j == nl - 1 && i == nchunks - 1) RPNN_CUDA_TRY(cudaEventRecord(ev[2], s));
                    st = fused_forward_bf16(*c, vv, c->q_x.as<float>() + 3 * first, c->q_d.as<float>() + 3 * first,
                                            &lights[3 * j], CH, cnt, c->g_out.as<float>() + first, s);
                    if (st) return st;
                    continue;
                }
                st = launch_descriptor(*c, vv, c->q_x.as<float>() + 3 * first, c->q_d.as<float>() + 3 * first,
                                       ldir + 3 * j, 0, CH, cnt, c->desc.p,
                                       f32 ? RPNN_F32 : (fp8 ? RPNN_FP8E4M3 : RPNN_BF16), s);
                if (st) return st;
                // (a chunked render attributes its network time to the descriptor stage)
                if (ev && j == nl - 1 && i == nchunks - 1) RPNN_CUDA_TRY(cudaEventRecord(ev[2], s));
                if (f32) st = mlp_forward_f32(*c, c->desc.as<float>(), CH, cnt, c->g_out.as<float>() + first, nullptr, s);
                else if (fp8) st = mlp_forward_fp8(*c, c->desc.p, CH, cnt, c->g_out.as<float>() + first, s);
                else st = mlp_forward_bf16(*c, c->desc.p, CH, cnt, c->g_out.as<float>() + first, s);
                if (st) return st;
            }
            // light j's predictions, weighted by albedo * E_j (the last light's scatter runs
            // with the composite below)
            if (j < nl - 1) {
                st = launch_scatter(*c, v->albedo * lights[3 * nl + j], c->g_out.as<float>(), c->q_ps.as<uint32_t>(),
                                    qc, c->sample_val.as<float>(), s);
                if (st) return st;
            }
        }
        if (ev) RPNN_CUDA_TRY(cudaEventRecord(ev[3], s));
    }
    rpnn_render_desc rdl = *desc;                   // the composite's scatter carries the last light
    rdl.light_E = lights[3 * nl + nl - 1];
    st = launch_scatter_composite(*c, rdl, v->albedo, net ? c->g_out.as<float>() : nullptr,
                                  net ? c->q_ps.as<uint32_t>() : nullptr, qc, c->sample_val.as<float>(),
                                  dev_image, net, s);
    if (st) return st;
    if (ev) RPNN_CUDA_TRY(cudaEventRecord(ev[4], s));
    if (out_num_queries) {
        int h = 0;
        RPNN_CUDA_TRY(cudaMemcpyAsync(&h, qc, sizeof(int), cudaMemcpyDeviceToHost, s));
        RPNN_CUDA_TRY(cudaStreamSynchronize(s));
        *out_num_queries = net ? h : -1;
    }
    return RPNN_OK;
}

rpnn_status rpnn_render(rpnn_ctx* ctx, int32_t vol, const rpnn_render_desc* desc, float* dev_image,
                        int64_t* out_num_queries, void* stream) {
    CHECK_CTX(ctx);
    return render_impl(reinterpret_cast<Ctx*>(ctx), vol, desc, nullptr, nullptr, 0, dev_image, out_num_queries,
                       (cudaStream_t)stream);
}

rpnn_status rpnn_render_env(rpnn_ctx* ctx, int32_t vol, const rpnn_render_desc* desc, const float* dirs,
                            const float* irradiance, int32_t n, float* dev_image, int64_t* out_num_queries,
                            void* stream) {
    CHECK_CTX(ctx);
    if (n < 1 || n > RPNN_MAX_ENV_LIGHTS || !dirs || !irradiance) {
        set_error("environment needs 1..%d directions and irradiances", RPNN_MAX_ENV_LIGHTS);
        return RPNN_ERR_ARG;
    }
    if (desc && desc->mode == RPNN_MODE_PATH) { set_error("environment lighting renders RPNN or SINGLE mode"); return RPNN_ERR_ARG; }
    for (int j = 0; j < n; ++j) {
        const float* w = dirs + 3 * j;
        const float l2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
        if (!(fabsf(l2 - 1.0f) < 1e-4f)) { set_error("direction %d is not unit length", j); return RPNN_ERR_ARG; }
        if (!(irradiance[j] >= 0.0f) || !std::isfinite(irradiance[j])) { set_error("irradiance %d is negative or not finite", j); return RPNN_ERR_ARG; }
    }
    return render_impl(reinterpret_cast<Ctx*>(ctx), vol, desc, dirs, irradiance, n, dev_image, out_num_queries,
                       (cudaStream_t)stream);
}

rpnn_status rpnn_set_fused(rpnn_ctx* ctx, int32_t on) {
    CHECK_CTX(ctx);
    reinterpret_cast<Ctx*>(ctx)->fused = on != 0;
    return RPNN_OK;
}

rpnn_status rpnn_set_render_chunk(rpnn_ctx* ctx, int64_t rows) {
    CHECK_CTX(ctx);
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (rows < 0 || (rows > 0 && rows < 128)) { set_error("chunk rows must be 0 or at least 128"); return RPNN_ERR_ARG; }
    c->chunk_rows = rows;
    return RPNN_OK;
}

static bool dense_args_ok(const int32_t* widths, int32_t n, int32_t din) {
    if (n < 0 || n > 64 || din <= 0 || (n > 0 && !widths)) return false;
    for (int i = 0; i < n; ++i)
        if (widths[i] <= 0 || widths[i] > 16384) return false;
    return true;
}

int64_t rpnn_dense_param_count(const int32_t* widths, int32_t n_hidden, int32_t din) {
    if (!dense_args_ok(widths, n_hidden, din)) return -1;
    return dense_param_count(widths, n_hidden, din);
}

rpnn_status rpnn_dense_forward(rpnn_ctx* ctx, const int32_t* widths, int32_t n_hidden, int32_t din,
                               const float* dev_params, const float* dev_in, int64_t q, float* dev_out,
                               void* stream) {
    CHECK_CTX(ctx);
    if (!dense_args_ok(widths, n_hidden, din)) { set_error("bad layer widths"); return RPNN_ERR_ARG; }
    if (q <= 0 || q > 65535 * 64 || !dev_params || !dev_in || !dev_out) { set_error("bad rows or pointer"); return RPNN_ERR_ARG; }
    return dense_forward(*reinterpret_cast<Ctx*>(ctx), widths, n_hidden, din, dev_params, dev_in, q, dev_out, nullptr,
                         (cudaStream_t)stream);
}

static rpnn_status dense_fwd_saved(Ctx& c, const int32_t* widths, int32_t n, int32_t din, const float* P,
                                   const float* in, int64_t q, cudaStream_t s) {
    int64_t per_row = 1;
    for (int i = 0; i < n; ++i) per_row += widths[i];
    rpnn_status st = c.t_saved.reserve((size_t)per_row * q * sizeof(float));
    if (!st) st = c.t_out.reserve((size_t)q * sizeof(float));
    if (st) return st;
    return dense_forward(c, widths, n, din, P, in, q, c.t_out.as<float>(), c.t_saved.as<float>(), s);
}

rpnn_status rpnn_dense_backward(rpnn_ctx* ctx, const int32_t* widths, int32_t n_hidden, int32_t din,
                                const float* dev_params, const float* dev_in, int64_t q, const float* dev_dout,
                                float* dev_dparams, void* stream) {
    CHECK_CTX(ctx);
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (!dense_args_ok(widths, n_hidden, din)) { set_error("bad layer widths"); return RPNN_ERR_ARG; }
    if (q <= 0 || q > 65535 * 64 || !dev_params || !dev_in || !dev_dout || !dev_dparams) {
        set_error("bad rows or pointer");
        return RPNN_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    rpnn_status st = dense_fwd_saved(*c, widths, n_hidden, din, dev_params, dev_in, q, s);
    if (st) return st;
    return dense_backward(*c, widths, n_hidden, din, dev_params, dev_in, q, c->t_saved.as<float>(), dev_dout,
                          dev_dparams, s);
}

rpnn_status rpnn_dense_train_step(rpnn_ctx* ctx, const int32_t* widths, int32_t n_hidden, int32_t din,
                                  const float* dev_in, const float* dev_target, int32_t batch,
                                  const rpnn_adam_cfg* adam, int64_t step, float* dev_params, float* dev_m,
                                  float* dev_v, double* dev_loss, void* stream) {
    CHECK_CTX(ctx);
    NvtxRange range("rpnn_dense_train_step");
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (!dense_args_ok(widths, n_hidden, din)) { set_error("bad layer widths"); return RPNN_ERR_ARG; }
    if (batch <= 0 || batch > 65535 * 64 || !adam || step < 1 || !dev_in || !dev_target || !dev_params || !dev_m ||
        !dev_v || !dev_loss) {
        set_error("bad batch, step or pointer");
        return RPNN_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t np = dense_param_count(widths, n_hidden, din);
    rpnn_status st = c->t_grad.reserve((size_t)np * sizeof(float));
    if (!st) st = c->sample_val.reserve((size_t)batch * sizeof(float));
    if (!st) st = dense_fwd_saved(*c, widths, n_hidden, din, dev_params, dev_in, batch, s);
    if (st) return st;
    float* dg = c->sample_val.as<float>();
    st = launch_loss(*c, c->t_out.as<float>(), dev_target, batch, dev_loss, dg, s);
    if (!st) st = dense_backward(*c, widths, n_hidden, din, dev_params, dev_in, batch, c->t_saved.as<float>(), dg,
                                 c->t_grad.as<float>(), s);
    if (st) return st;
    return launch_adam(dev_params, dev_m, dev_v, c->t_grad.as<float>(), np, step, *adam, s);
}

// ---------------------------------------------------------------- stencil-size comparison
int64_t rpnn_stencil_param_count(int32_t n_xy) {
    const int din = stencil_din(n_xy);
    return din < 0 ? -1 : param_layout_for(din).total;
}

static bool stencil_shape(int32_t n_xy, ParamLayout* L, NetDims* nd) {
    const int din = stencil_din(n_xy);
    if (din < 0) {
        set_error("stencil resolution %d outside [2, 9]", n_xy);
        return false;
    }
    *L = param_layout_for(din);
    *nd = NetDims{L, din, din};
    return true;
}

rpnn_status rpnn_stencil_descriptors(rpnn_ctx* ctx, int32_t vol, int32_t n_xy, const float* dev_x,
                                     const float* dev_d, const float* dev_wl, int32_t wl_stride, int64_t q,
                                     float* dev_desc, void* stream) {
    CHECK_CTX(ctx);
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    Volume* v = get_vol(c, vol, true);
    if (!v) return RPNN_ERR_HANDLE;
    if (q < 0 || q > kChunkRows) { set_error("q must be in [0, %lld]", (long long)kChunkRows); return RPNN_ERR_ARG; }
    if (wl_stride < 0) { set_error("wl_stride < 0"); return RPNN_ERR_ARG; }
    if (q > 0 && (!dev_x || !dev_d || !dev_wl || !dev_desc)) { set_error("null pointer"); return RPNN_ERR_ARG; }
    return stencil_descriptors(*c, *v, n_xy, dev_x, dev_d, dev_wl, wl_stride, q, dev_desc, (cudaStream_t)stream);
}

rpnn_status rpnn_stencil_forward(rpnn_ctx* ctx, int32_t n_xy, const float* dev_params, const float* dev_desc,
                                 int64_t q, float* dev_out, void* stream) {
    CHECK_CTX(ctx);
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    ParamLayout L;
    NetDims nd;
    if (!stencil_shape(n_xy, &L, &nd)) return RPNN_ERR_ARG;
    if (q <= 0 || q > kChunkRows) { set_error("q must be in [1, %lld]", (long long)kChunkRows); return RPNN_ERR_ARG; }
    if (!dev_params || !dev_desc || !dev_out) { set_error("null pointer"); return RPNN_ERR_ARG; }
    rpnn_status st = ensure_rows(c, q, true);
    if (st) return st;
    float* const scr[3] = {c->act0.as<float>(), c->act1.as<float>(), c->act2.as<float>()};
    return rpnn_forward_f32(c, nd, dev_params, dev_desc, q, nullptr, dev_out, nullptr, scr, (cudaStream_t)stream);
}

// forward with saved activations (t_saved), prediction to t_out
static rpnn_status stencil_fwd_saved(Ctx& c, const NetDims& nd, const float* P, const float* desc, int64_t q,
                                     cudaStream_t s) {
    rpnn_status st = c.t_saved.reserve(mlp_saved_floats_per_row() * q * sizeof(float));
    if (!st) st = c.t_out.reserve(q * sizeof(float));
    if (st) return st;
    return rpnn_forward_f32(&c, nd, P, desc, q, nullptr, c.t_out.as<float>(), c.t_saved.as<float>(), nullptr, s);
}

rpnn_status rpnn_stencil_backward(rpnn_ctx* ctx, int32_t n_xy, const float* dev_params, const float* dev_desc,
                                  int64_t q, const float* dev_dout, float* dev_dparams, void* stream) {
    CHECK_CTX(ctx);
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    ParamLayout L;
    NetDims nd;
    if (!stencil_shape(n_xy, &L, &nd)) return RPNN_ERR_ARG;
    if (q <= 0 || q > kChunkRows) { set_error("q must be in [1, %lld]", (long long)kChunkRows); return RPNN_ERR_ARG; }
    if (!dev_params || !dev_desc || !dev_dout || !dev_dparams) { set_error("null pointer"); return RPNN_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    rpnn_status st = stencil_fwd_saved(*c, nd, dev_params, dev_desc, q, s);
    if (st) return st;
    return rpnn_backward_f32(*c, nd, dev_params, dev_desc, q, c->t_saved.as<float>(), dev_dout, dev_dparams, s);
}

rpnn_status rpnn_stencil_train_step(rpnn_ctx* ctx, int32_t n_xy, const float* dev_desc, const float* dev_target,
                                    int32_t batch, const rpnn_adam_cfg* adam, int64_t step, float* dev_params,
                                    float* dev_m, float* dev_v, double* dev_loss, void* stream) {
    CHECK_CTX(ctx);
    NvtxRange range("rpnn_stencil_train_step");
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    ParamLayout L;
    NetDims nd;
    if (!stencil_shape(n_xy, &L, &nd)) return RPNN_ERR_ARG;
    if (batch <= 0 || batch > kChunkRows || !adam || step < 1 || !dev_desc || !dev_target || !dev_params ||
        !dev_m || !dev_v || !dev_loss) {
        set_error("bad batch, step or pointer");
        return RPNN_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    rpnn_status st = c->t_grad.reserve((size_t)L.total * sizeof(float));
    if (!st) st = c->sample_val.reserve((size_t)batch * sizeof(float));
    if (!st) st = stencil_fwd_saved(*c, nd, dev_params, dev_desc, batch, s);
    if (st) return st;
    float* dg = c->sample_val.as<float>();
    st = launch_loss(*c, c->t_out.as<float>(), dev_target, batch, dev_loss, dg, s);
    if (!st) st = rpnn_backward_f32(*c, nd, dev_params, dev_desc, batch, c->t_saved.as<float>(), dg,
                                    c->t_grad.as<float>(), s);
    if (st) return st;
    return launch_adam(dev_params, dev_m, dev_v, c->t_grad.as<float>(), L.total, step, *adam, s);
}

rpnn_status rpnn_set_autotune_table(rpnn_ctx* ctx, const rpnn_tune_entry* entries, int32_t n) {
    CHECK_CTX(ctx);
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (n < 0 || (!entries && n > 0)) { set_error("bad entries"); return RPNN_ERR_ARG; }
    std::vector<std::pair<GemmKey, GemmChoice>> add;
    for (int32_t i = 0; i < n; ++i) {
        const rpnn_tune_entry& e = entries[i];
        GemmKey k{e.M, e.N, e.K0, e.K1, e.flags};
        GemmChoice ch{0, e.splits, e.us, e.default_us};
        const bool tc = (e.flags & (1 << 8)) != 0;
        if (tc) {
            if (e.tile_m != 128 || e.tile_k != 64 ||
                (e.tile_n != 32 && e.tile_n != 64 && e.tile_n != 128 && e.tile_n != 256)) {
                set_error("entry %d: no tensor-core tile %d x %d x %d", i, e.tile_m, e.tile_n, e.tile_k);
                return RPNN_ERR_ARG;
            }
            ch.tile = e.tile_n;
        } else {
            ch.tile = gemm_tile_index(e.tile_m, e.tile_n, e.tile_k);
            if (ch.tile < 0) {
                set_error("entry %d: no tile %d x %d x %d", i, e.tile_m, e.tile_n, e.tile_k);
                return RPNN_ERR_ARG;
            }
        }
        if (e.splits < 1 || e.splits > 32 || (e.splits & (e.splits - 1))) {
            set_error("entry %d: split %d", i, e.splits);
            return RPNN_ERR_ARG;
        }
        add.emplace_back(k, ch);
    }
    for (const auto& kc : add) {
        bool found = false;
        for (auto& e : c->tuner.table)
            if (e.first == kc.first) { e.second = kc.second; found = true; }
        if (!found) c->tuner.table.push_back(kc);
    }
    ++c->tuner.version;
    return RPNN_OK;
}

rpnn_status rpnn_set_train_precision(rpnn_ctx* ctx, int32_t precision) {
    CHECK_CTX(ctx);
    if (precision != RPNN_F32 && precision != RPNN_BF16) {
        set_error("training precision must be RPNN_F32 or RPNN_BF16");
        return RPNN_ERR_ARG;
    }
    reinterpret_cast<Ctx*>(ctx)->train_precision = precision;
    return RPNN_OK;
}

rpnn_status rpnn_set_autotune(rpnn_ctx* ctx, int32_t on) {
    CHECK_CTX(ctx);
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (c->tuner.enabled != (on != 0)) ++c->tuner.version;
    c->tuner.enabled = on != 0;
    return RPNN_OK;
}

rpnn_status rpnn_get_autotune(rpnn_ctx* ctx, rpnn_tune_entry* out, int32_t cap, int32_t* n) {
    CHECK_CTX(ctx);
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (cap < 0 || !n || (!out && cap > 0)) { set_error("bad output buffer"); return RPNN_ERR_ARG; }
    const auto& t = c->tuner.table;
    *n = (int32_t)t.size();
    for (int32_t i = 0; i < cap && i < (int32_t)t.size(); ++i) {
        const GemmKey& k = t[i].first;
        const GemmChoice& ch = t[i].second;
        int tm = 128, tn = ch.tile, tk = 64;           // tensor-core entries store the tile width
        if (!(k.flags & (1 << 8))) gemm_tile_shape(ch.tile, &tm, &tn, &tk);
        out[i] = rpnn_tune_entry{k.M, k.N, k.K0, k.K1, k.flags, tm, tn, tk, ch.splits, ch.us, ch.default_us};
    }
    return RPNN_OK;
}

rpnn_status rpnn_set_profiling(rpnn_ctx* ctx, int32_t on) {
    CHECK_CTX(ctx);
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    c->profiling = on != 0;
    return RPNN_OK;
}

rpnn_status rpnn_read_profile(rpnn_ctx* ctx, double* ms, int64_t* renders) {
    CHECK_CTX(ctx);
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (!ms || !renders) { set_error("null pointer"); return RPNN_ERR_ARG; }
    for (int i = 0; i < RPNN_NUM_STAGES; ++i) ms[i] = 0.0;
    for (size_t r = 0; r < c->prof_used; ++r) {
        cudaEvent_t* ev = &c->prof_events[r * 5];
        RPNN_CUDA_TRY(cudaEventSynchronize(ev[4]));
        for (int i = 0; i < RPNN_NUM_STAGES; ++i) {
            float t = 0.0f;
            RPNN_CUDA_TRY(cudaEventElapsedTime(&t, ev[i], ev[i + 1]));
            ms[i] += t;
        }
    }
    *renders = (int64_t)c->prof_used;
    c->prof_used = 0;
    return RPNN_OK;
}

rpnn_status rpnn_gen_records(rpnn_ctx* ctx, int32_t vol, int64_t first, int64_t n, uint64_t seed,
                             float rel_ci, int32_t n_min, int32_t n_max, float* dev_x, float* dev_d,
                             float* dev_wl, float* dev_label, int32_t* dev_npaths, void* stream) {
    CHECK_CTX(ctx);
    NvtxRange range("rpnn_gen_records");
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    Volume* v = get_vol(c, vol, true);
    if (!v) return RPNN_ERR_HANDLE;
    if (n < 0 || first < 0 || first + n > ((int64_t)1 << 32)) { set_error("bad record range"); return RPNN_ERR_ARG; }
    if (n == 0) return RPNN_OK;
    if (!dev_x || !dev_d || !dev_wl || !dev_label || !dev_npaths) { set_error("null pointer"); return RPNN_ERR_ARG; }
    if (!(rel_ci > 0.0f) || n_min < 1 || n_max < n_min) { set_error("bad stopping rule"); return RPNN_ERR_ARG; }
    return launch_records(*c, v->view(), first, n, seed, rel_ci, n_min, n_max, dev_x, dev_d, dev_wl,
                          dev_label, dev_npaths, (cudaStream_t)stream);
}

rpnn_status rpnn_mlp_backward(rpnn_ctx* ctx, const void* dev_desc, int32_t desc_dtype, int64_t q,
                              const float* dev_dout, float* dev_dparams, void* stream) {
    CHECK_CTX(ctx);
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (!c->weights_set) { set_error("rpnn_set_weights has not run"); return RPNN_ERR_STATE; }
    if (q <= 0 || q > 65535 * 64) { set_error("q must be in [1, %d]", 65535 * 64); return RPNN_ERR_ARG; }
    if (!dev_desc || !dev_dout || !dev_dparams) { set_error("null pointer"); return RPNN_ERR_ARG; }
    rpnn_status st = check_train_desc(dev_desc, desc_dtype);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const float* d32 = nullptr;
    st = train_desc(*c, dev_desc, desc_dtype, q, &d32, s);
    if (!st) st = train_forward(*c, dev_desc, desc_dtype, d32, q, s);
    if (st) return st;
    return train_backward(*c, d32, q, dev_dout, dev_dparams, s);
}

}  // extern "C"

namespace rpnn {
namespace {

// The arithmetic of one training step on q descriptor rows: forward, log-MSE loss,
// backward, Adam, weight copies.  Adam's bias corrections come from step (host) or, when
// cc is not null, from device memory (the captured form).
rpnn_status train_step_body(Ctx& c, const void* desc, int32_t dtype, const float* target, int64_t q,
                            const rpnn_adam_cfg& adam, int64_t step, const float* cc, float* params, float* m,
                            float* v, double* loss, cudaStream_t s) {
    const float* d32 = nullptr;
    rpnn_status st = train_desc(c, desc, dtype, q, &d32, s);
    if (!st) st = train_forward(c, desc, dtype, d32, q, s);
    if (st) return st;
    float* dg = c.sample_val.as<float>();
    st = launch_loss(c, c.t_out.as<float>(), target, (int)q, loss, dg, s);
    if (st) return st;
    // a captured BF16 step runs the weight gradients on two more streams, beside the
    // data-gradient chain (a direct step keeps one stream: it may time new GEMM shapes)
    const cudaStream_t* side = nullptr;
    cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
    RPNN_CUDA_TRY(cudaStreamIsCapturing(s, &cst));
    if (cst == cudaStreamCaptureStatusActive && c.train_precision == RPNN_BF16 && c.side_stream[1] &&
        (int)c.t_events.size() >= kTrainEvents)
        side = c.side_stream;
    st = train_backward(c, d32, q, dg, c.t_grad.as<float>(), s, side);
    // a direct step sizes the second weight-gradient stream's split-K workspace like the
    // tuner's, so that a later capture allocates nothing
    if (!st && cst == cudaStreamCaptureStatusNone && c.train_precision == RPNN_BF16 && c.tuner.ws.bytes > 0)
        st = c.t_ws2.reserve(c.tuner.ws.bytes);
    if (st) return st;
    st = cc ? launch_adam_dev(params, m, v, c.t_grad.as<float>(), RPNN_NPARAMS, cc, adam, s)
            : launch_adam(params, m, v, c.t_grad.as<float>(), RPNN_NPARAMS, step, adam, s);
    if (st) return st;
    RPNN_CUDA_TRY(cudaMemcpyAsync(c.params32.p, params, (size_t)RPNN_NPARAMS * sizeof(float),
                                  cudaMemcpyDeviceToDevice, s));
    return mlp_build_bf16_image(c, s);
}

void drop_train_graph(TrainGraph& G) {
    if (G.exec) cudaGraphExecDestroy(G.exec);
    if (G.graph) cudaGraphDestroy(G.graph);
    G.exec = nullptr;
    G.graph = nullptr;
}

// Captures the step for configuration `key` on the library's stream, reading the minibatch
// and Adam's corrections from the graph's staging buffers.
rpnn_status capture_train_step(Ctx& c, const TrainGraphKey& key, const rpnn_adam_cfg& adam, float* params, float* m,
                               float* v, double* loss) {
    TrainGraph& G = c.tgraph;
    drop_train_graph(G);
    if (!c.capture_stream) RPNN_CUDA_TRY(cudaStreamCreateWithFlags(&c.capture_stream, cudaStreamNonBlocking));
    // the weight-gradient streams and their events exist before the capture starts
    for (cudaStream_t& ss : c.side_stream)
        if (!ss) RPNN_CUDA_TRY(cudaStreamCreateWithFlags(&ss, cudaStreamNonBlocking));
    while ((int)c.t_events.size() < kTrainEvents) {
        cudaEvent_t ev;
        RPNN_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        c.t_events.push_back(ev);
    }
    cudaStream_t cs = c.capture_stream;
    RPNN_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    const rpnn_status est = train_step_body(c, G.desc.p, key.desc_dtype, G.target.as<float>(), key.batch, adam, 1,
                                            G.adam.as<float>(), params, m, v, loss, cs);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(cs, &graph);
    if (est || ce != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        if (!est) set_error("stream capture of the training step failed: %s", cudaGetErrorString(ce));
        return est ? est : RPNN_ERR_CUDA;
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    if (ie != cudaSuccess) {
        cudaGraphDestroy(graph);
        set_error("graph instantiation failed: %s", cudaGetErrorString(ie));
        return RPNN_ERR_CUDA;
    }
    G.graph = graph;
    G.exec = exec;
    G.key = key;
    return RPNN_OK;
}

}  // namespace

void train_graph_release(Ctx& c) {
    drop_train_graph(c.tgraph);
    c.tgraph.desc.release();
    c.tgraph.target.release();
    c.tgraph.adam.release();
}

}  // namespace rpnn

extern "C" {

rpnn_status rpnn_train_step(rpnn_ctx* ctx, const void* dev_desc, int32_t desc_dtype, const float* dev_target, int32_t batch,
                            const rpnn_adam_cfg* adam, int64_t step, float* dev_params, float* dev_m,
                            float* dev_v, double* dev_loss, void* stream) {
    CHECK_CTX(ctx);
    NvtxRange range("rpnn_train_step");
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (!c->weights_set) { set_error("rpnn_set_weights has not run"); return RPNN_ERR_STATE; }
    if (batch <= 0 || batch > 65535 * 64) { set_error("bad batch %d", batch); return RPNN_ERR_ARG; }
    if (!adam || step < 1) { set_error("adam config missing or step < 1"); return RPNN_ERR_ARG; }
    if (!dev_desc || !dev_target || !dev_params || !dev_m || !dev_v || !dev_loss) {
        set_error("null pointer");
        return RPNN_ERR_ARG;
    }
    rpnn_status st = check_train_desc(dev_desc, desc_dtype);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t q = batch;
    const size_t row_bytes = (size_t)RPNN_K * RPNN_DESC_STRIDE * (desc_dtype == RPNN_BF16 ? 2 : 4);
    st = c->t_grad.reserve((size_t)RPNN_NPARAMS * sizeof(float));
    if (!st) st = c->sample_val.reserve(q * sizeof(float));
    if (!st && c->train_graphs) {
        st = c->tgraph.desc.reserve((size_t)q * row_bytes);
        if (!st) st = c->tgraph.target.reserve((size_t)q * sizeof(float));
        if (!st) st = c->tgraph.adam.reserve(2 * sizeof(float));
    }
    if (st) return st;
    if (!c->train_graphs)
        return train_step_body(*c, dev_desc, desc_dtype, dev_target, q, *adam, step, nullptr, dev_params, dev_m, dev_v,
                               dev_loss, s);
    // The step's launches are the same from step to step: the first step of a configuration
    // runs them directly (the GEMM autotuner decides its tiles there), the second captures
    // them as a graph, later steps replay it after staging the minibatch and Adam's
    // corrections.  The key holds everything the captured launches bake in.
    TrainGraph& G = c->tgraph;
    TrainGraphKey key;
    key.batch = batch; key.desc_dtype = desc_dtype; key.precision = c->train_precision;
    key.params = dev_params; key.m = dev_m; key.v = dev_v; key.loss = dev_loss;
    key.lr = adam->lr; key.b1 = adam->beta1; key.b2 = adam->beta2; key.eps = adam->eps;
    key.tuner_version = c->tuner.version; key.epoch = c->epoch; key.allocs = devbuf_generation();
    if (!(G.exec && G.key == key)) {
        if (!(G.have_seen && G.seen == key)) {
            st = train_step_body(*c, dev_desc, desc_dtype, dev_target, q, *adam, step, nullptr, dev_params, dev_m,
                                 dev_v, dev_loss, s);
            key.tuner_version = c->tuner.version;      // the direct run may have tuned
            key.allocs = devbuf_generation();
            G.seen = key;
            G.have_seen = true;
            return st;
        }
        st = capture_train_step(*c, key, *adam, dev_params, dev_m, dev_v, dev_loss);
        if (st) return st;
    }
    RPNN_CUDA_TRY(cudaMemcpyAsync(G.desc.p, dev_desc, (size_t)q * row_bytes, cudaMemcpyDeviceToDevice, s));
    RPNN_CUDA_TRY(cudaMemcpyAsync(G.target.p, dev_target, (size_t)q * sizeof(float), cudaMemcpyDeviceToDevice, s));
    st = launch_adam_corrections(G.adam.as<float>(), step, *adam, s);
    if (st) return st;
    RPNN_CUDA_TRY(cudaGraphLaunch(G.exec, s));
    return RPNN_OK;
}

rpnn_status rpnn_set_train_graphs(rpnn_ctx* ctx, int32_t on) {
    CHECK_CTX(ctx);
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    c->train_graphs = on != 0;
    if (!c->train_graphs) train_graph_release(*c);
    c->tgraph.have_seen = false;
    return RPNN_OK;
}

}  // extern "C"
