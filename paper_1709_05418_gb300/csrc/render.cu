// render.cu -- Monte Carlo part of the renderer (Sec. 4.4) and the training-record
// generator (Sec. 5.1).
//
// k_primary: one thread per pixel sample.  Pinhole ray with Philox pixel jitter, delta
// tracking to the first real collision (the visible point), next-event estimation of
// the direct in-scattering with a ratio-tracked shadow ray, and either (RPNN mode) an
// appended shading query for the descriptor + network stages, or (path mode) a
// path-traced estimate of the indirect part.  Queries are compacted with one atomic per
// warp so the list stays in pixel order within a warp.
#include <vector>

#include "common.cuh"

namespace rpnn {

namespace {

struct RenderArgs {
    float cam_pos[3], cam_fwd[3], cam_right[3], cam_up[3];
    float tan_half, aspect;
    int W, H, spp;
    uint64_t seed;
    float wl[3];
    float E;
    int mode;   // RPNN_MODE_*
};

// One render of a batch for the batched primary pass: its volume, camera and light, its
// pixel samples, where they start in the batch's per-sample buffers, and its first block.
struct PrimaryItem {
    VolumeView v;
    RenderArgs a;
    int64_t P, region, first_block;
};

// 6 blocks of 128 threads per SM (80 registers, no spills): more rays in flight to hide the
// latency of the density gathers (the batched form, which reads the volume from shared
// memory, takes 5 and 96 registers).  BATCH: the grid covers the pixel samples of up to
// RPNN_MAX_BATCH renders (items[i] from block first_block on); each block copies its item
// into shared memory and works on that render's samples, writing into its region of the
// per-sample buffers and appending its shading points to that region with its own count.
template <bool BATCH>
__global__ void __launch_bounds__(128, BATCH ? 5 : 6)
k_primary(const VolumeView v_, const RenderArgs a_, int64_t P_, float* __restrict__ sample_val,
          float* __restrict__ qx, float* __restrict__ qd, uint32_t* __restrict__ qps,
          int* __restrict__ qcount, int* __restrict__ hit_out, float* __restrict__ x_out,
          float* __restrict__ d_out, float* __restrict__ Ld_out, uint32_t* status,
          const PrimaryItem* __restrict__ items, int n_items) {
    __shared__ __align__(16) PrimaryItem it;
    __shared__ int s_item;
    if (BATCH) {
        if (threadIdx.x == 0) {
            int i = 0;
            while (i + 1 < n_items && items[i + 1].first_block <= (int64_t)blockIdx.x) ++i;
            s_item = i;
        }
        __syncthreads();
        const int* src = reinterpret_cast<const int*>(items + s_item);
        int* dst = reinterpret_cast<int*>(&it);
        for (int w = threadIdx.x; w < (int)(sizeof(PrimaryItem) / sizeof(int)); w += blockDim.x) dst[w] = src[w];
        __syncthreads();
        const int64_t o = it.region;
        sample_val += o;
        qx += 3 * o;
        qd += 3 * o;
        qps += o;
        qcount += s_item;
    }
    const VolumeView& v = BATCH ? it.v : v_;
    const RenderArgs& a = BATCH ? it.a : a_;
    const int64_t P = BATCH ? it.P : P_;
    const int64_t ps = (blockIdx.x - (BATCH ? it.first_block : 0)) * (int64_t)blockDim.x + threadIdx.x;
    const bool active = ps < P;
    int hit = 0;
    float3 x = f3(0.f, 0.f, 0.f), d = f3(0.f, 0.f, 1.f);
    float Ld = 0.0f;
    if (active) {
        const uint32_t pixel = (uint32_t)(ps / a.spp), s = (uint32_t)(ps % a.spp);
        const int px = (int)(pixel % (uint32_t)a.W), py = (int)(pixel / (uint32_t)a.W);
        const Rng rc = make_rng(a.seed, pixel, s, kDomCamera);
        const float4 xi = rc.draw(0);
        const float sx = (2.0f * ((float)px + xi.x) / (float)a.W - 1.0f) * a.tan_half * a.aspect;
        const float sy = (1.0f - 2.0f * ((float)py + xi.y) / (float)a.H) * a.tan_half;
        d = normalize3(f3(a.cam_fwd[0] + sx * a.cam_right[0] + sy * a.cam_up[0],
                          a.cam_fwd[1] + sx * a.cam_right[1] + sy * a.cam_up[1],
                          a.cam_fwd[2] + sx * a.cam_right[2] + sy * a.cam_up[2]));
        const float3 o = f3(a.cam_pos[0], a.cam_pos[1], a.cam_pos[2]);
        uint32_t ctr = 0;
        const int r = delta_track(v, o, d, make_rng(a.seed, pixel, s, kDomPrimary), ctr, x);
        bool capped = r < 0;
        hit = r == 1;
        float val = 0.0f;
        if (hit) {
            const float3 wl = f3(a.wl[0], a.wl[1], a.wl[2]);
            uint32_t c2 = 0;
            Ld = nee(v, true, x, d, wl, a.E, make_rng(a.seed, pixel, s, kDomShadow), c2, capped);
            float Li = 0.0f;
            if (a.mode == RPNN_MODE_PATH)
                Li = path_Li(v, x, d, wl, a.E, make_rng(a.seed, pixel, s, kDomPath), capped);
            val = v.albedo * (Ld + Li);
        }
        if (capped) raise_status(status, kStatIterLimit);
        if (sample_val) sample_val[ps] = val;
        if (hit_out) {
            hit_out[ps] = hit;
            x_out[3 * ps] = x.x; x_out[3 * ps + 1] = x.y; x_out[3 * ps + 2] = x.z;
            d_out[3 * ps] = d.x; d_out[3 * ps + 1] = d.y; d_out[3 * ps + 2] = d.z;
            Ld_out[ps] = Ld;
        }
    }
    if (qcount) {
        const bool want = active && hit;
        const unsigned mask = __ballot_sync(0xffffffffu, want);
        const int lane = threadIdx.x & 31;
        int base = 0;
        if (lane == 0 && mask) base = atomicAdd(qcount, __popc(mask));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (want) {
            const int slot = base + __popc(mask & ((1u << lane) - 1u));
            qx[3 * slot] = x.x; qx[3 * slot + 1] = x.y; qx[3 * slot + 2] = x.z;
            qd[3 * slot] = d.x; qd[3 * slot + 1] = d.y; qd[3 * slot + 2] = d.z;
            qps[slot] = (uint32_t)ps;
        }
    }
}

// sample_val[ps_i] += alpha * E * g_i for every shading query i
__global__ void k_scatter(const float* __restrict__ g, const uint32_t* __restrict__ qps,
                          const int* __restrict__ qcount, const int* __restrict__ g_off,
                          const int* __restrict__ g_total, float scale, float* __restrict__ sample_val) {
    // predictions of this render's queries start at g[*g_off] (batched renders) and no
    // index reaches *g_total
    const int o = g_off ? *g_off : 0;
    int n = *qcount;
    if (g_total && *g_total - o < n) n = *g_total - o;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        sample_val[qps[i]] += scale * g[o + i];
}

// Environment lighting (Sec. 4.4: a distant emitter approximated by directional samples):
// for every shading point i and every light j >= j0, the next-event estimate towards
// direction j with irradiance E_j, added to the point's sample value times the albedo.
// Each direction restarts the point's shadow stream (pixel, sample, shadow domain) at draw
// 0, so direction j's estimate is the one a single-light render with light j makes.
__global__ void __launch_bounds__(128)
k_nee_env(const VolumeView v, const RenderArgs a, const float* __restrict__ qx, const float* __restrict__ qd,
          const uint32_t* __restrict__ qps, const int* __restrict__ qcount, const float* __restrict__ dirs,
          const float* __restrict__ E, int j0, int n, float* __restrict__ sample_val, uint32_t* status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= *qcount) return;
    const uint32_t ps = qps[i];
    const uint32_t pixel = ps / (uint32_t)a.spp, s = ps % (uint32_t)a.spp;
    const float3 x = f3(qx[3 * i], qx[3 * i + 1], qx[3 * i + 2]);
    const float3 d = f3(qd[3 * i], qd[3 * i + 1], qd[3 * i + 2]);
    const Rng rng = make_rng(a.seed, pixel, s, kDomShadow);
    bool capped = false;
    float Ld = 0.0f;
    for (int j = j0; j < n; ++j) {
        uint32_t ctr = 0;
        Ld += nee(v, true, x, d, f3(dirs[3 * j], dirs[3 * j + 1], dirs[3 * j + 2]), E[j], rng, ctr, capped);
    }
    if (capped) raise_status(status, kStatIterLimit);
    sample_val[ps] += v.albedo * Ld;
}

// pixel = mean over its spp samples, summed in sample order
__global__ void k_composite(const float* __restrict__ sample_val, int64_t npix, int spp,
                            float* __restrict__ image) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npix;
         p += (int64_t)gridDim.x * blockDim.x) {
        float acc = 0.0f;
        for (int s = 0; s < spp; ++s) acc += sample_val[p * spp + s];
        image[p] = acc / (float)spp;
    }
}

// One render of a batch for the batched scatter and composite: its region of the per-sample
// buffers, the weight of its predictions (albedo x irradiance), samples per pixel, pixel
// count, first pixel in the batch's pixel numbering, and its image.
struct OutItem {
    int64_t region, npix, first_pixel;
    float scale;
    int spp;
    float* image;
};

// Predictions of all items' shading points (compacted: item i's at off[i] .. off[i+1]) added to
// their samples, sample_val[region_i + qps[region_i + j]] += scale_i g[off[i] + j]
__global__ void k_scatter_batch(const float* __restrict__ g, const uint32_t* __restrict__ qps,
                                const int* __restrict__ off, const OutItem* __restrict__ items, int n_items,
                                float* __restrict__ sample_val) {
    const int total = off[n_items];
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
        int i = 0;
        while (i + 1 < n_items && off[i + 1] <= q) ++i;
        const int64_t o = items[i].region;
        sample_val[o + qps[o + (q - off[i])]] += items[i].scale * g[q];
    }
}

// every item's pixels: mean over its samples, summed in sample order (as k_composite)
__global__ void k_composite_batch(const float* __restrict__ sample_val, const OutItem* __restrict__ items,
                                  int n_items, int64_t total_pixels) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < total_pixels;
         p += (int64_t)gridDim.x * blockDim.x) {
        int i = 0;
        while (i + 1 < n_items && items[i + 1].first_pixel <= p) ++i;
        const OutItem& it = items[i];
        const int64_t px = p - it.first_pixel;
        const float* sv = sample_val + it.region + px * it.spp;
        float acc = 0.0f;
        for (int s = 0; s < it.spp; ++s) acc += sv[s];
        it.image[px] = acc / (float)it.spp;
    }
}

// Kahan-compensated FP32 running sum (hi + lo carries about twice FP32's precision)
struct KahanF {
    float hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add(float v) {
        const float y = __fsub_rn(v, lo);
        const float t = __fadd_rn(hi, y);
        lo = __fsub_rn(__fsub_rn(t, hi), y);
        hi = t;
    }
    // the running sum plus a (small) partial sum, as one float
    __device__ __forceinline__ float with(float v) const { return __fadd_rn(hi, __fsub_rn(v, lo)); }
};

// inclusive prefix sum over the warp's lanes
__device__ __forceinline__ float warp_scan(float v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// Training records (Sec. 5.1); one warp per record.  Lane 0 samples the record (direction,
// origin on the bounding sphere's cross-section, free flight by delta tracking with
// retries, light direction) and the warp traces its label paths 32 at a time, path j on
// lane j % 32 with path j's own random stream.  After each round the stopping rule is
// evaluated at every path count of the round in order -- n >= n_min and
// 1.96 s / sqrt(n) <= rel_ci * mean -- from FP32 prefix sums of L and L^2 over the round
// added to Kahan-compensated running totals; the first count that meets it (or n_max)
// ends the record and its label is the mean of its first n paths.
__global__ void __launch_bounds__(128)
k_records(const VolumeView v, int64_t first, int64_t n, uint64_t seed, float rel_ci, int n_min,
          int n_max, float* __restrict__ xo, float* __restrict__ dout, float* __restrict__ wlo,
          float* __restrict__ label, int* __restrict__ npaths, uint32_t* status) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += nwarps) {
        const uint32_t rec = (uint32_t)(first + i);
        float3 x = f3(0.f, 0.f, 0.f), d = f3(0.f, 0.f, 1.f);
        int found = 0;
        if (lane == 0) {
            const float ext[3] = {v.ext[0], v.ext[1], v.ext[2]};
            const float3 C = f3(0.5f * ext[0], 0.5f * ext[1], 0.5f * ext[2]);
            const float R = 0.5f * sqrtf(ext[0] * ext[0] + ext[1] * ext[1] + ext[2] * ext[2]);
            for (uint32_t att = 0; att < (uint32_t)kRecordAttempts && !found; ++att) {
                const float4 xi = make_rng(seed, rec, att, kDomRecord).draw(0);
                const float cz = 1.0f - 2.0f * xi.x;
                float sp, cp;
                sincosf(2.0f * kPi * xi.y, &sp, &cp);
                const float sz = sqrtf(fmaxf(0.0f, 1.0f - cz * cz));
                d = f3(sz * cp, sz * sp, cz);
                float3 b1, b2;
                duff_basis(d, b1, b2);
                const float rr = R * sqrtf(xi.z);
                float s2, c2;
                sincosf(2.0f * kPi * xi.w, &s2, &c2);
                const float3 o = C + (rr * c2) * b1 + (rr * s2) * b2 + (-2.0f * R) * d;
                uint32_t ctr = 0;
                const int h = delta_track(v, o, d, make_rng(seed, rec, att, kDomRecTrack), ctr, x);
                if (h < 0) raise_status(status, kStatIterLimit);
                found = h == 1;
            }
        }
        found = __shfl_sync(0xffffffffu, found, 0);
        x = f3(__shfl_sync(0xffffffffu, x.x, 0), __shfl_sync(0xffffffffu, x.y, 0), __shfl_sync(0xffffffffu, x.z, 0));
        d = f3(__shfl_sync(0xffffffffu, d.x, 0), __shfl_sync(0xffffffffu, d.y, 0), __shfl_sync(0xffffffffu, d.z, 0));
        float3 wl;
        {
            const float4 xi = make_rng(seed, rec, 0, kDomLight).draw(0);
            const float cz = 1.0f - 2.0f * xi.x;
            float sp, cp;
            sincosf(2.0f * kPi * xi.y, &sp, &cp);
            const float sz = sqrtf(fmaxf(0.0f, 1.0f - cz * cz));
            wl = f3(sz * cp, sz * sp, cz);
        }
        float mean = 0.0f;
        int np = 0;
        bool capped = false;
        if (found) {
            KahanF S, Q;                               // running sums of L and L^2
            for (int base = 0; base < n_max; base += 32) {
                const int j = base + lane;
                float L = 0.0f;
                if (j < n_max) L = path_Li(v, x, d, wl, 1.0f, make_rng(seed, rec, (uint32_t)j, kDomLabel), capped);
                const float pS = warp_scan(L, lane), pQ = warp_scan(L * L, lane);
                const float cnt = (float)(j + 1);
                const float s_j = S.with(pS), q_j = Q.with(pQ);
                const float m_j = s_j / cnt;
                const float var = fmaxf(q_j - s_j * m_j, 0.0f) / fmaxf(cnt - 1.0f, 1.0f);
                const float hw = 1.96f * sqrtf(var / cnt);
                const bool stop = j < n_max && ((j + 1 >= n_min && j > 0 && m_j > 0.0f && hw <= rel_ci * m_j) ||
                                                j + 1 == n_max);
                const uint32_t hit = __ballot_sync(0xffffffffu, stop);
                if (hit) {
                    const int f = __ffs(hit) - 1;
                    mean = __shfl_sync(0xffffffffu, m_j, f);
                    np = base + f + 1;
                    break;
                }
                S.add(__shfl_sync(0xffffffffu, pS, 31));
                Q.add(__shfl_sync(0xffffffffu, pQ, 31));
            }
        } else if (lane == 0) {
            raise_status(status, kStatIterLimit);
        }
        if (__any_sync(0xffffffffu, capped) && lane == 0) raise_status(status, kStatIterLimit);
        if (lane == 0) {
            xo[3 * i] = x.x; xo[3 * i + 1] = x.y; xo[3 * i + 2] = x.z;
            dout[3 * i] = d.x; dout[3 * i + 1] = d.y; dout[3 * i + 2] = d.z;
            wlo[3 * i] = wl.x; wlo[3 * i + 1] = wl.y; wlo[3 * i + 2] = wl.z;
            label[i] = mean;
            npaths[i] = np;
        }
    }
}

RenderArgs make_args(const rpnn_render_desc& rd) {
    RenderArgs a;
    for (int k = 0; k < 3; ++k) {
        a.cam_pos[k] = rd.cam_pos[k]; a.cam_fwd[k] = rd.cam_fwd[k];
        a.cam_right[k] = rd.cam_right[k]; a.cam_up[k] = rd.cam_up[k];
        a.wl[k] = rd.light_dir[k];
    }
    a.tan_half = rd.tan_half_fov_y;
    a.aspect = (float)rd.width / (float)rd.height;
    a.W = rd.width; a.H = rd.height; a.spp = rd.spp;
    a.seed = rd.seed;
    a.E = rd.light_E;
    a.mode = rd.mode;
    return a;
}

}  // namespace

size_t batch_tables_bytes(int n) {
    return ((size_t)n * sizeof(PrimaryItem) + 255) / 256 * 256 + (size_t)n * sizeof(OutItem);
}

void batch_tables(const Ctx& c, const rpnn_batch_item* items, int n, const std::vector<int64_t>& region,
                  std::vector<unsigned char>& out, int64_t* blocks, int64_t* pixels) {
    out.assign(batch_tables_bytes(n), 0);
    PrimaryItem* pi = reinterpret_cast<PrimaryItem*>(out.data());
    OutItem* oi = reinterpret_cast<OutItem*>(out.data() + ((size_t)n * sizeof(PrimaryItem) + 255) / 256 * 256);
    int64_t b = 0, px = 0;
    for (int i = 0; i < n; ++i) {
        const rpnn_render_desc& rd = items[i].desc;
        const Volume* v = c.vol(items[i].vol);
        pi[i].v = v->view();
        pi[i].a = make_args(rd);
        pi[i].P = (int64_t)rd.width * rd.height * rd.spp;
        pi[i].region = region[i];
        pi[i].first_block = b;
        b += (pi[i].P + 127) / 128;
        oi[i].region = region[i];
        oi[i].npix = (int64_t)rd.width * rd.height;
        oi[i].first_pixel = px;
        oi[i].scale = v->albedo * rd.light_E;
        oi[i].spp = rd.spp;
        oi[i].image = items[i].dev_image;
        px += oi[i].npix;
    }
    *blocks = b;
    *pixels = px;
}

rpnn_status launch_primary_batch(Ctx& c, const void* tables, int n, int64_t blocks, float* sample_val, float* qx,
                                 float* qd, uint32_t* qps, int* qcount, cudaStream_t s) {
    const PrimaryItem* pi = static_cast<const PrimaryItem*>(tables);
    k_primary<true><<<(unsigned)blocks, 128, 0, s>>>(VolumeView{}, RenderArgs{}, 0, sample_val, qx, qd, qps, qcount,
                                                     nullptr, nullptr, nullptr, nullptr, c.status.as<uint32_t>(), pi,
                                                     n);
    RPNN_CHECK_LAUNCH();
    return RPNN_OK;
}

rpnn_status launch_scatter_composite_batch(Ctx& c, const void* tables, int n, int64_t pixels, const float* g,
                                           const uint32_t* qps, const int* off, float* sample_val, cudaStream_t s) {
    const OutItem* oi = reinterpret_cast<const OutItem*>(static_cast<const unsigned char*>(tables) +
                                                         ((size_t)n * sizeof(PrimaryItem) + 255) / 256 * 256);
    k_scatter_batch<<<c.num_sms * 8, 256, 0, s>>>(g, qps, off, oi, n, sample_val);
    RPNN_CHECK_LAUNCH();
    int64_t b = (pixels + 255) / 256;
    if (b > c.num_sms * 16) b = c.num_sms * 16;
    k_composite_batch<<<(unsigned)(b > 0 ? b : 1), 256, 0, s>>>(sample_val, oi, n, pixels);
    RPNN_CHECK_LAUNCH();
    return RPNN_OK;
}

rpnn_status launch_primary(Ctx& c, const VolumeView& vv, const rpnn_render_desc& rd,
                           float* sample_val, float* qx, float* qd, uint32_t* qps, int* qcount,
                           int* hit, float* xo, float* dout, float* Ld, cudaStream_t s) {
    const int64_t P = (int64_t)rd.width * rd.height * rd.spp;
    const int64_t blocks = (P + 127) / 128;
    k_primary<false><<<(unsigned)blocks, 128, 0, s>>>(vv, make_args(rd), P, sample_val, qx, qd, qps, qcount,
                                                      hit, xo, dout, Ld, c.status.as<uint32_t>(), nullptr, 0);
    RPNN_CHECK_LAUNCH();
    return RPNN_OK;
}

rpnn_status launch_scatter_composite(Ctx& c, const rpnn_render_desc& rd, float alpha,
                                     const float* g, const uint32_t* qps, const int* qcount,
                                     float* sample_val, float* image, bool with_g, cudaStream_t s,
                                     const int* g_off, const int* g_total) {
    const int64_t npix = (int64_t)rd.width * rd.height;
    if (with_g) {
        k_scatter<<<c.num_sms * 8, 256, 0, s>>>(g, qps, qcount, g_off, g_total, alpha * rd.light_E, sample_val);
        RPNN_CHECK_LAUNCH();
    }
    int64_t b = (npix + 255) / 256;
    if (b > c.num_sms * 16) b = c.num_sms * 16;
    k_composite<<<(unsigned)b, 256, 0, s>>>(sample_val, npix, rd.spp, image);
    RPNN_CHECK_LAUNCH();
    return RPNN_OK;
}

rpnn_status launch_nee_env(Ctx& c, const VolumeView& vv, const rpnn_render_desc& rd, const float* qx,
                           const float* qd, const uint32_t* qps, const int* qcount, int64_t max_q, const float* dirs,
                           const float* E, int j0, int n, float* sample_val, cudaStream_t s) {
    if (max_q <= 0 || j0 >= n) return RPNN_OK;
    k_nee_env<<<(unsigned)((max_q + 127) / 128), 128, 0, s>>>(vv, make_args(rd), qx, qd, qps, qcount, dirs, E, j0, n,
                                                                sample_val, c.status.as<uint32_t>());
    RPNN_CHECK_LAUNCH();
    return RPNN_OK;
}

rpnn_status launch_scatter(Ctx& c, float scale, const float* g, const uint32_t* qps, const int* qcount,
                           float* sample_val, cudaStream_t s) {
    k_scatter<<<c.num_sms * 8, 256, 0, s>>>(g, qps, qcount, nullptr, nullptr, scale, sample_val);
    RPNN_CHECK_LAUNCH();
    return RPNN_OK;
}

namespace {
__global__ void k_count_nonfinite(const float* __restrict__ p, int64_t n, unsigned int* bad) {
    unsigned int b = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b |= !isfinite(p[i]);
    if (__any_sync(0xffffffffu, b) && (threadIdx.x & 31) == 0) atomicOr(bad, 1u);
}
}  // namespace

rpnn_status check_finite(Ctx& c, const float* p, int64_t n, cudaStream_t s) {
    rpnn_status st = c.t_loss.reserve(sizeof(unsigned int));
    if (st) return st;
    unsigned int* bad = c.t_loss.as<unsigned int>();
    RPNN_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(unsigned int), s));
    k_count_nonfinite<<<c.num_sms * 4, 256, 0, s>>>(p, n, bad);
    RPNN_CHECK_LAUNCH();
    unsigned int h = 0;
    RPNN_CUDA_TRY(cudaMemcpyAsync(&h, bad, sizeof(h), cudaMemcpyDeviceToHost, s));
    RPNN_CUDA_TRY(cudaStreamSynchronize(s));
    if (h) { set_error("parameters contain NaN or Inf"); return RPNN_ERR_NONFINITE; }
    return RPNN_OK;
}

namespace {
__global__ void k_chunk_counts(const int* __restrict__ count, int64_t rows, int n, int* __restrict__ out) {
    const int64_t total = *count;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int64_t left = total - (int64_t)i * rows;
        out[i] = (int)(left < 0 ? 0 : (left > rows ? rows : left));
    }
}
}  // namespace

rpnn_status launch_chunk_counts(Ctx& c, const int* count, int64_t rows, int n, int* out, cudaStream_t s) {
    (void)c;
    k_chunk_counts<<<1, 128, 0, s>>>(count, rows, n, out);
    RPNN_CHECK_LAUNCH();
    return RPNN_OK;
}

rpnn_status launch_records(Ctx& c, const VolumeView& vv, int64_t first, int64_t n, uint64_t seed,
                           float rel_ci, int n_min, int n_max, float* x, float* d, float* wl,
                           float* label, int* npaths, cudaStream_t s) {
    // one warp per record, four per block; at most a few waves of blocks (grid-stride)
    const int64_t blocks = std::min<int64_t>((n + 3) / 4, (int64_t)c.num_sms * 16);
    k_records<<<(unsigned)blocks, 128, 0, s>>>(vv, first, n, seed, rel_ci, n_min, n_max, x, d, wl,
                                               label, npaths, c.status.as<uint32_t>());
    RPNN_CHECK_LAUNCH();
    return RPNN_OK;
}

}  // namespace rpnn
