/*
 * rpnn.h -- C ABI of the GB300 (sm_103a) RPNN cloud-rendering hot path.
 *
 * Method: Kallweit, Mueller, McWilliams, Gross, Novak, "Deep Scattering: Rendering
 * Atmospheric Clouds with Radiance-Predicting Neural Networks".  For every shading
 * point the path (a) samples a visible point by delta tracking (Sec. 4.4), (b)
 * gathers the 10-level 5x5x9 light-aligned stencil descriptor from a Gaussian
 * mip pyramid of the mean-free-path-normalised density (Sec. 4.2, Sec. 6), (c) runs
 * the progressive-input residual network (Sec. 4.3, Fig. 6) and adds its indirect
 * prediction to the Monte Carlo single-scattering estimate (Sec. 4.4).  Training
 * (Sec. 5) runs on the same device with the library's own forward/backward kernels.
 *
 * Conventions shared by every entry point
 *  - Return value: RPNN_OK (0) or a negative rpnn_status.  Errors never abort the
 *    process; rpnn_last_error() gives a message for the calling thread.
 *  - Pointers named dev_* are device pointers owned by the caller and borrowed for the
 *    duration of the call (or of the asynchronous work it enqueues).  Everything the
 *    library allocates (volume copies, pyramids, weight images, scratch) is owned by
 *    the context and released by rpnn_destroy.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Calls
 *    enqueue work on it and return without synchronising unless documented otherwise.
 *  - A context is bound to the CUDA device current at rpnn_create; call it from any
 *    thread with that device current.  Calls on one context are not thread-safe.
 *  - Geometry: a density grid of nx*ny*nz voxels (x fastest) is scaled uniformly into
 *    the unit box (Sec. 5): voxel size h0 = 1/max(nx,ny,nz), grid extent
 *    [0, nx*h0] x [0, ny*h0] x [0, nz*h0], voxel (i,j,k) centred at ((i+.5)h0, ...).
 *    Density values are extinction coefficients per unit of that box.
 *  - Directions: `d` is a ray's tracing direction (from the camera into the cloud);
 *    the radiance of Eq. 1 propagates along omega = -d.  `light_dir` points towards
 *    the (directional) light.
 */
#ifndef RPNN_ABI_H_
#define RPNN_ABI_H_
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rpnn_ctx rpnn_ctx;
typedef int32_t rpnn_status;

enum {
    RPNN_OK = 0,
    RPNN_ERR_ARG = -1,          /* invalid argument (size, pointer, value) */
    RPNN_ERR_HANDLE = -2,       /* unknown context or volume id */
    RPNN_ERR_CUDA = -3,         /* a CUDA runtime call failed */
    RPNN_ERR_OOM = -4,          /* device allocation failed */
    RPNN_ERR_ITER_LIMIT = -5,   /* a device loop hit its iteration cap (result truncated) */
    RPNN_ERR_NONFINITE = -6,    /* NaN/Inf met in data the call validates */
    RPNN_ERR_STATE = -7,        /* call order violated (e.g. render before set_weights) */
    RPNN_ERR_UNSUPPORTED = -8,  /* combination not built for this device */
    RPNN_ERR_TIMEOUT = -9       /* a bounded device-side wait gave up (results invalid) */
};

enum { RPNN_F32 = 0, RPNN_F16 = 1, RPNN_BF16 = 2, RPNN_FP8E4M3 = 3 };

enum {
    RPNN_K = 10,            /* stencil levels (Sec. 4.2) */
    RPNN_S = 225,           /* points per level: 5 x 5 x 9 (Sec. 4.2) */
    RPNN_DIN = 226,         /* network input per block: Sigma^k and gamma (Sec. 4.3) */
    RPNN_DESC_STRIDE = 240, /* stored width of one level of a descriptor row */
    RPNN_DESC_STRIDE_FP8 = 256, /* the same for E4M3 rows (whole 32-byte tensor-core K-steps) */
    RPNN_H = 200,           /* hidden width (Sec. 7: every layer has 200 nodes) */
    RPNN_NPARAMS = 1296601  /* flat parameter count, layout below */
};

/* ---- context -------------------------------------------------------------------- */
rpnn_status rpnn_create(rpnn_ctx** out);
rpnn_status rpnn_destroy(rpnn_ctx* ctx);
/* Message of the calling thread's last error ("" if none).  Valid until the next call. */
const char* rpnn_last_error(void);
/* Reads (and clears) the context's device status word; synchronises `stream`.
 * Returns RPNN_OK, RPNN_ERR_ITER_LIMIT, RPNN_ERR_NONFINITE or RPNN_ERR_TIMEOUT. */
rpnn_status rpnn_sync_status(rpnn_ctx* ctx, void* stream);

/* ---- volume (Sec. 4.2 mean-free-path normalisation; Sec. 5 unit box) ---------------- */
/* Copies the caller's density grid (dtype RPNN_F32 or RPNN_F16, nx*ny*nz values, x
 * fastest) into a library-owned FP32 grid and returns its id in *out_vol.  albedo is
 * the single-scattering albedo alpha (mu_s = alpha mu_t, Sec. 3.2), hg_g the
 * Henyey-Greenstein asymmetry (Sec. 5.1).  Values must be finite and >= 0 (checked by
 * rpnn_build_mips). */
rpnn_status rpnn_load_volume(rpnn_ctx* ctx, const void* dev_density, int32_t dtype, int32_t nx,
                             int32_t ny, int32_t nz, float albedo, float hg_g,
                             int32_t* out_vol, void* stream);
/* Computes the volume statistics (majorant, mean over non-zero voxels -- an exact
 * fixed-point sum with 32 fraction bits below the majorant's binary exponent) and the
 * Gaussian mip levels read by the 10 stencil levels (sigma_i = 2^i fine voxels, Sec.
 * 6; truncated at 3 sigma, normalised, zero outside, divided by the mean).  Synchronises
 * `stream` once to read the statistics back.  RPNN_ERR_NONFINITE for negative/NaN/Inf
 * voxels, RPNN_ERR_ARG for an all-zero grid. */
rpnn_status rpnn_build_mips(rpnn_ctx* ctx, int32_t vol, void* stream);

typedef struct {
    int32_t n[3];              /* nx, ny, nz */
    int32_t levels;            /* mip levels 0..levels-1 */
    int32_t dims[16][3];       /* per level: ceil(n / 2^i) */
    int32_t mip_of_level[RPNN_K]; /* mip level read by stencil level k (0-based) */
    double mean;               /* mean extinction over voxels > 0 */
    float inv_mean_f;          /* (float)(1/mean) = one mean free path in world units */
    float majorant;            /* max voxel value */
    int64_t nonzero;           /* voxels > 0 */
    int32_t bricks[3];         /* tracking majorant bricks per axis: ceil(n / 8) */
    float mip_weight[RPNN_K];  /* blended descriptor: weight of level mip_of_level[k] + 1 */
} rpnn_volume_info;
/* Host copy of the statistics (valid after rpnn_build_mips). */
rpnn_status rpnn_get_volume_info(rpnn_ctx* ctx, int32_t vol, rpnn_volume_info* out);
/* Writes mip level `level` as FP32 [dims[2]][dims[1]][dims[0]] into dev_out (building it
 * if the stencil does not use it). */
rpnn_status rpnn_copy_mip_level(rpnn_ctx* ctx, int32_t vol, int32_t level, float* dev_out,
                                void* stream);
/* Blended (fractional) mip selection for the descriptor of volume `vol` (Sec. 6 fixes a
 * Gaussian pyramid but not how a stencil level picks from it; blending is the fractional
 * choice): with on != 0, stencil level k reads (1 - w_k) rho_{m_k} + w_k rho_{m_k + 1},
 * w_k = the fraction of log2(stencil spacing in fine voxels) above m_k (0 where the spacing is
 * outside the pyramid), as lerp(a, b, w) = fma(w, b - a, a) in FP32.  The descriptor then
 * varies continuously with the mean free path instead of jumping where m_k switches (e.g.
 * over an animation), at twice the lookups.  Off by default; applies to later descriptor
 * extractions and renders of the volume. */
rpnn_status rpnn_set_mip_blend(rpnn_ctx* ctx, int32_t vol, int32_t on);
/* Cap on the tentative collisions (and brick steps) of one tracking call through volume
 * `vol` (0 = the default 1,000,000).  A call that reaches it stops, its result is truncated
 * and the device status raises RPNN_ERR_ITER_LIMIT at the next status read (rpnn_sync_status,
 * or a call that reads the count); the context stays usable.  For fault injection in tests
 * and for bounding the time of a render. */
rpnn_status rpnn_set_iteration_cap(rpnn_ctx* ctx, int32_t vol, int64_t cap);
/* Phase function of volume `vol` (Sec. 3.1): RPNN_PHASE_HG (the default; Henyey-Greenstein
 * with the g given at rpnn_load_volume) or RPNN_PHASE_LORENZ_MIE, the cloud droplets'
 * Lorenz-Mie function: the Mie series (Bohren & Huffman 1983) for water spheres (index
 * 1.333) at 0.55 um over Deirmendjian's cumulus C.1 size distribution, averaged over
 * RPNN_LM_BINS bins of 0.1 degree per unit solid angle.  It applies to next-event
 * estimation and to the path tracer's direction sampling (label records, path mode), which
 * samples a bin by its cumulative probability and cos(theta) uniformly inside it.
 * RPNN_PHASE_LORENZ_MIE_CHOPPED (Sec. 3.1, Sec. 5.1): the full function at a path's first
 * bounce (the camera's or a training record's vertex); after it, the function without its
 * diffraction peak (the RPNN_LM_CHOP_BINS bins below 5 degrees, holding the fraction f of
 * the scattered light) renormalised, in a medium of extinction (1 - f albedo) mu_t and
 * albedo (1 - f) albedo / (1 - f albedo); light reaches every vertex (next-event shadow
 * rays) through that thinner medium, camera rays and record sampling see the full one.
 * (The paper's own tables and chop angle are in its unavailable supplement.)  The first
 * Lorenz-Mie selection in a context uploads both tables (context-owned, 43 KB) and
 * synchronises the default stream.  Errors: RPNN_ERR_ARG for another kind, RPNN_ERR_HANDLE
 * for an unknown volume. */
enum { RPNN_PHASE_HG = 0, RPNN_PHASE_LORENZ_MIE = 1, RPNN_PHASE_LORENZ_MIE_CHOPPED = 2 };
#define RPNN_LM_BINS 1800
#define RPNN_LM_CHOP_BINS 50
rpnn_status rpnn_set_phase_function(rpnn_ctx* ctx, int32_t vol, int32_t kind);
/* Host copy of the full (chopped = 0) or chopped table (no device work): bin values
 * p[RPNN_LM_BINS] (per steradian), cumulative probabilities cdf[RPNN_LM_BINS + 1], bin-edge
 * cosines cos_edges[...] and the peak's fraction f; any pointer may be NULL.
 * Errors: RPNN_ERR_ARG unless n == RPNN_LM_BINS. */
rpnn_status rpnn_lorenz_mie_table(int32_t chopped, double* p, double* cdf, double* cos_edges, int32_t n,
                                  double* peak_fraction);
/* Writes the tracking majorant grid as FP32 [bricks[2]][bricks[1]][bricks[0]] into dev_out:
 * delta and ratio tracking (Sec. 4.4) bound the density piecewise by bricks of 8^3 voxels,
 * brick b by the largest of the voxels its trilinear density interpolates (8b - 1 .. 8b + 8
 * per axis, zero outside the grid), and cross empty bricks without drawing. */
rpnn_status rpnn_copy_brick_majorants(rpnn_ctx* ctx, int32_t vol, float* dev_out, void* stream);

/* ---- network parameters (Sec. 4.3) --------------------------------------------------- */
/* Flat FP32 parameter vector, row-major [out][in] matrices, in this order:
 *   for block k = 1..10:  V^k [200][226], W1^k [200][200] (omitted for k = 1: o^0 = 0,
 *                         footnote 1 of Sec. 4.3), b1^k [200], W2^k [200][200], b2^k [200]
 *   standard layers:      [200][200], [200], [200][200], [200], [1][200], [1]
 * 1,296,601 values.  Block: F1 = relu(V z^k + W1 o^{k-1} + b1), F2 = W2 F1 + b2,
 * o^k = relu(F2 + o^{k-1}); standard layer o' = relu(W o + b); g = last output.
 * The library keeps its own FP32 copy and a BF16 tensor-core image; the caller's
 * buffer may be freed after the call returns (the copy is enqueued on `stream`).
 * Parameters are checked first (the call synchronises `stream` for it): a NaN or Inf
 * returns RPNN_ERR_NONFINITE and leaves the previous weights in place. */
rpnn_status rpnn_set_weights(rpnn_ctx* ctx, const float* dev_params, int64_t n_params,
                             void* stream);

/* ---- descriptor (Sec. 4.2, Fig. 5) ---------------------------------------------------- */
/* For q shading points x (dev_x, q*3 FP32, unit-box world coordinates) with tracing
 * directions d (dev_d, q*3 FP32, unit length) and light directions (dev_wl: 3 floats
 * shared by all queries when wl_stride = 0, or q*3 floats when wl_stride = 3; unit
 * length) writes the descriptor rows [q][10][RPNN_DESC_STRIDE] of dtype RPNN_F32 or
 * RPNN_BF16 (or [q][10][RPNN_DESC_STRIDE_FP8] of RPNN_FP8E4M3: the FP32 value rounded to
 * E4M3, nearest even, saturating at 448, unscaled) into dev_desc: per level k the 225
 * densities rho at the stencil points in (iz*5+iy)*5+ix order, then gamma =
 * acos(omega . light) in radians, then zeros.
 * Frame: z = light, x = normalize(z cross omega), y = z cross x (x = first vector of
 * the Duff et al. 2017 basis of z when omega is parallel to z).  The FP32 arithmetic
 * follows one fixed rounding sequence, bit-identical to the FP32 CPU restatement. */
rpnn_status rpnn_extract_descriptors(rpnn_ctx* ctx, int32_t vol, const float* dev_x,
                                     const float* dev_d, const float* dev_wl, int32_t wl_stride,
                                     int64_t q, void* dev_desc, int32_t desc_dtype, void* stream);

/* ---- network forward (Sec. 4.3) -------------------------------------------------------- */
/* g = RPNN(z) for q descriptor rows (layout of rpnn_extract_descriptors; dtype RPNN_F32,
 * RPNN_BF16 or RPNN_FP8E4M3).  precision RPNN_F32: FP32 CUDA-core form; RPNN_BF16: tcgen05
 * tensor cores, BF16 operands, FP32 accumulation (needs desc_dtype RPNN_BF16);
 * RPNN_FP8E4M3: tcgen05, E4M3 operands with per-tensor scales, FP32 accumulation (needs
 * desc_dtype RPNN_FP8E4M3 and rpnn_calibrate_fp8 since the last rpnn_set_weights, else
 * RPNN_ERR_STATE).  dev_out: q FP32. */
rpnn_status rpnn_mlp_forward(rpnn_ctx* ctx, const void* dev_desc, int32_t desc_dtype, int64_t q,
                             int32_t precision, float* dev_out, void* stream);
/* FP8 calibration (the paper trains and runs in FP32; low precision is this library's):
 * runs the FP32 network on q FP32 descriptor rows [q][10][RPNN_DESC_STRIDE] (dev_desc,
 * borrowed for the call), takes each layer's largest activation as its E4M3 range (scale =
 * max / 448), chooses per-layer weight scales, and builds the E4M3 weight image that
 * RPNN_FP8E4M3 renders and forwards use until the next rpnn_set_weights.  Synchronises
 * `stream`.  Errors: RPNN_ERR_STATE (no weights), RPNN_ERR_ARG (q < 1, null), CUDA/OOM. */
rpnn_status rpnn_calibrate_fp8(rpnn_ctx* ctx, const float* dev_desc, int64_t q, void* stream);

/* ---- FP32 network forward without device allocation ----------------------------------------
 * The paper has no counterpart to this entry point.  It serves callers that cannot call
 * cudaMalloc when they run the network: hosts whose device memory is all owned by their own
 * allocator or reserved up front under a fixed budget (a game engine, a serving runtime),
 * and real-time loops that allow no allocation after start-up (cudaMalloc and cudaFree may
 * block and synchronise the device).  It computes g = RPNN(z) for at most
 * RPNN_STATIC_MAX_ROWS rows of FP32 descriptors (layout of rpnn_extract_descriptors) with
 * the caller's FP32 parameter vector (layout above), without a context, through the same
 * routine and the same FP32 CUDA-core GEMM kernel as rpnn_mlp_forward with precision
 * RPNN_F32, with the GEMM's default tile.  The result equals rpnn_mlp_forward's bit for bit:
 * tile shapes change no result bit and a forward GEMM is never split along K.
 *  - Scratch: one static device array of 3 * RPNN_STATIC_MAX_ROWS * 200 floats (9.8 MB),
 *    present on every GPU that loads the library until the process exits.  It keeps the
 *    last call's contents; nothing in it needs to start at zero (every layer writes its
 *    output before the next reads it).
 *  - All calls share that array: calls whose work overlaps on a GPU (two streams, two
 *    threads) race and give wrong results.  Serialise them on one stream.
 *  - Set-up: the first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call before any
 *    stream capture.
 *  - Errors: RPNN_ERR_ARG for q > RPNN_STATIC_MAX_ROWS or null pointers, RPNN_ERR_CUDA when
 *    the set-up lookup fails.  It calls no cudaMalloc, cudaFree or other allocating routine. */
enum { RPNN_STATIC_MAX_ROWS = 4096 };
rpnn_status rpnn_mlp_forward_f32_static(const float* dev_params, const float* dev_desc, int64_t q,
                                        float* dev_out, void* stream);

/* ---- rendering (Sec. 4.4) ---------------------------------------------------------------- */
typedef struct {
    float cam_pos[3], cam_fwd[3], cam_right[3], cam_up[3]; /* pinhole frame (unit vectors) */
    float tan_half_fov_y;
    int32_t width, height, spp;
    uint64_t seed;                /* Philox4x32-10 key */
    float light_dir[3];           /* unit, towards the light */
    float light_E;                /* irradiance of the directional light */
    int32_t precision;            /* RPNN_F32, RPNN_BF16 or RPNN_FP8E4M3 network arithmetic */
    int32_t mode;                 /* RPNN_MODE_* */
} rpnn_render_desc;
enum { RPNN_MODE_RPNN = 0, RPNN_MODE_SINGLE = 1, RPNN_MODE_PATH = 2 };
/* Renders width*height pixels (row-major, y down) into dev_image (FP32, caller-owned):
 * pixel = (1/spp) sum_s alpha * E * (p_HG(d.light) T_light + g(z)), where the first term
 * is next-event estimation with a ratio-tracked shadow ray and g the network's L_i
 * prediction (RPNN_MODE_RPNN), zero (RPNN_MODE_SINGLE), or a path-traced L_i estimate
 * (RPNN_MODE_PATH, the plain Monte Carlo reference).  Rays that miss the cloud give 0.
 * *out_num_queries (host, may be NULL) receives the number of shading points; passing
 * it synchronises `stream`. */
rpnn_status rpnn_render(rpnn_ctx* ctx, int32_t vol, const rpnn_render_desc* desc,
                        float* dev_image, int64_t* out_num_queries, void* stream);
/* Environment lighting (Sec. 4.4: a distant emitter such as a sun-sky model is approximated
 * by directional samples whose predictions are summed): renders as rpnn_render with the n
 * directional lights dirs[j] (host, [n][3], unit, towards the light) of irradiance
 * irradiance[j] (host, [n], >= 0) in place of desc->light_dir / light_E:
 * pixel = (1/spp) sum_s alpha sum_j E_j (p_HG(d.w_j) T_j + g(z_j)), z_j the descriptor in
 * light j's frame.  The visible point of a sample does not depend on the lights and each
 * light's shadow ray uses the stream a single-light render with that light uses, so the
 * result is the sum of the n single-light renders (up to FP32 summation order).
 * desc->mode: RPNN_MODE_RPNN or RPNN_MODE_SINGLE.  The descriptor and network stages run
 * once per light.  Errors: RPNN_ERR_ARG for n outside 1..RPNN_MAX_ENV_LIGHTS, a non-unit
 * direction, a negative or non-finite irradiance, or path mode; otherwise as rpnn_render. */
#define RPNN_MAX_ENV_LIGHTS 1024
rpnn_status rpnn_render_env(rpnn_ctx* ctx, int32_t vol, const rpnn_render_desc* desc, const float* dirs,
                            const float* irradiance, int32_t n, float* dev_image, int64_t* out_num_queries,
                            void* stream);
/* Memory budget of rpnn_render (no counterpart in the paper): the descriptor and network
 * stages run over chunks of at most `rows` shading points (0 = the default 1,048,576
 * rows, i.e. 5 GB of BF16 descriptors; otherwise at least 128).  Results do not depend on
 * the chunking.  Errors: RPNN_ERR_ARG for 0 < rows < 128 or rows < 0. */
rpnn_status rpnn_set_render_chunk(rpnn_ctx* ctx, int64_t rows);
/* Fused descriptor + network stages (off by default; Sec. 4.2 and 4.3 in one kernel, no
 * counterpart in the paper, which names descriptor construction as the bottleneck in
 * Sec. 7): with on != 0 a BF16 render (rpnn_render, rpnn_render_env) gathers each shading
 * point's descriptor inside the tensor-core network kernel, so no descriptor rows are
 * written to or read from device memory and no descriptor buffer is allocated.  The image
 * is bit for bit that of the unfused stages (the same FP32 descriptor arithmetic and BF16
 * rounding, the same MMAs in the same order).  On a GB300 the fused kernel is slower than
 * the two separate kernels (its gather warps share the SM's registers and issue slots with
 * the network's epilogue), so it serves renders whose descriptor buffer would not fit.
 * Renders with blended mip selection (rpnn_set_mip_blend) run unfused.  Never fails for a
 * valid context. */
rpnn_status rpnn_set_fused(rpnn_ctx* ctx, int32_t on);
/* Batched serving (no counterpart in the paper: many clouds, uneven query counts, one
 * frame).  Item i renders volume items[i].vol with items[i].desc into items[i].dev_image
 * (FP32, caller-owned, width*height) exactly as rpnn_render would, bit for bit.  Every
 * stage runs once for all items: one primary launch over all items' pixel samples, a prefix
 * sum of the per-item query counts, one descriptor and one network launch over the
 * compacted shading points, one scatter and one composite; the sequence is captured once as
 * a CUDA graph on a library-owned stream and replayed on `stream` while the item list
 * (volumes, descriptions, image pointers) is unchanged; loading a volume, building mips or setting
 * weights invalidates the captured graph, and so do rpnn_set_mip_blend and
 * rpnn_set_iteration_cap.  Requirements: 1 <= n_items <= RPNN_MAX_BATCH, every item in
 * RPNN_MODE_RPNN with RPNN_BF16 precision.  out_num_queries (host, may be
 * NULL): n_items per-item shading-point counts; passing it synchronises `stream`.
 * Errors: RPNN_ERR_ARG (empty, oversized or mixed batch, bad descriptions, null image),
 * RPNN_ERR_HANDLE, RPNN_ERR_STATE (no weights), RPNN_ERR_OOM, RPNN_ERR_CUDA. */
enum { RPNN_MAX_BATCH = 32 };
typedef struct {
    int32_t vol;
    rpnn_render_desc desc;
    float* dev_image;
} rpnn_batch_item;
rpnn_status rpnn_render_batch(rpnn_ctx* ctx, const rpnn_batch_item* items, int32_t n_items,
                              int64_t* out_num_queries, void* stream);
/* Stage timing (no counterpart in the paper; used to attribute render time).  When on,
 * rpnn_render records CUDA events on its stream at the boundaries of its four stages:
 * primary (tracking + NEE), descriptor, network, composite.  rpnn_read_profile waits for
 * those events, writes the summed device milliseconds of each stage over the renders
 * since the previous read into ms[RPNN_NUM_STAGES] and their number into *renders. */
enum { RPNN_STAGE_PRIMARY = 0, RPNN_STAGE_DESCRIPTOR = 1, RPNN_STAGE_NETWORK = 2,
       RPNN_STAGE_COMPOSITE = 3, RPNN_NUM_STAGES = 4 };
rpnn_status rpnn_set_profiling(rpnn_ctx* ctx, int32_t on);
rpnn_status rpnn_read_profile(rpnn_ctx* ctx, double* ms, int64_t* renders);
/* Primary stage only, for inspection: per pixel-sample ps = pixel*spp + sample writes
 * hit flag (1 hit, 0 miss), x (3 floats), d (3 floats), L_d (E p T, without alpha). */
rpnn_status rpnn_trace_primary(rpnn_ctx* ctx, int32_t vol, const rpnn_render_desc* desc,
                               int32_t* dev_hit, float* dev_x, float* dev_d, float* dev_Ld,
                               void* stream);

/* ---- training (Sec. 5) -------------------------------------------------------------------- */
/* Training records (Sec. 5.1) `first` .. `first+n-1` of stream `seed`: direction uniform
 * on the sphere, origin uniform on the bounding sphere's cross-section, free flight by
 * delta tracking (retried on escape), light direction uniform on the sphere, and L_i by
 * path tracing with next-event estimation until the 95% half-width is within rel_ci of
 * the mean (n_min .. n_max paths).  Outputs (FP32, caller-owned): x, d, wl (n*3 each),
 * label (n), npaths (n int32). */
rpnn_status rpnn_gen_records(rpnn_ctx* ctx, int32_t vol, int64_t first, int64_t n, uint64_t seed,
                             float rel_ci, int32_t n_min, int32_t n_max, float* dev_x,
                             float* dev_d, float* dev_wl, float* dev_label,
                             int32_t* dev_npaths, void* stream);
/* Gradient of sum_i dout_i * g(z_i) w.r.t. the parameters currently set by
 * rpnn_set_weights (the chain rule in the training precision, rpnn_set_train_precision:
 * FP32 CUDA cores by default, or BF16 tensor-core GEMMs), written (not accumulated) to
 * dev_dparams (RPNN_NPARAMS floats).  dev_desc: q rows [10][RPNN_DESC_STRIDE] of desc_dtype
 * RPNN_F32 or RPNN_BF16 (BF16 records take half the memory: 4.8 KB instead of 9.6 KB per
 * row).  The BF16 training form rounds FP32 rows to BF16 itself, so both dtypes give it the
 * same result for BF16-representable rows; the FP32 form widens BF16 rows exactly (into
 * context scratch).  Errors: RPNN_ERR_ARG for another dtype, q outside [1, 4194240] or a
 * null pointer; RPNN_ERR_STATE before rpnn_set_weights. */
rpnn_status rpnn_mlp_backward(rpnn_ctx* ctx, const void* dev_desc, int32_t desc_dtype, int64_t q,
                              const float* dev_dout, float* dev_dparams, void* stream);
typedef struct { float lr, beta1, beta2, eps; } rpnn_adam_cfg;
/* One optimiser step (Sec. 5.2): forward on `batch` descriptor rows (desc_dtype RPNN_F32 or
 * RPNN_BF16, as rpnn_mlp_backward), loss mean (log(1+g) - log(1+L))^2 written as FP64 to
 * *dev_loss (device), backward, Adam (step >= 1, bias-corrected) on the caller's FP32
 * parameters dev_params with moments dev_m, dev_v (RPNN_NPARAMS each, updated in place),
 * then the library's weight copies are refreshed from the updated parameters. */
rpnn_status rpnn_train_step(rpnn_ctx* ctx, const void* dev_desc, int32_t desc_dtype, const float* dev_target,
                            int32_t batch, const rpnn_adam_cfg* adam, int64_t step,
                            float* dev_params, float* dev_m, float* dev_v, double* dev_loss,
                            void* stream);
/* Captured training steps (on by default; no counterpart in the paper): a step's ~100
 * launches are the same from step to step, so the first rpnn_train_step of a configuration
 * (batch, descriptor dtype, training precision, the parameter / moment / loss pointers,
 * the Adam settings, the autotuner's table) runs them directly, the second captures them
 * as a CUDA graph on a library-owned stream, and later steps copy the minibatch into
 * context-owned staging buffers and replay the graph (one launch instead of ~100).  The
 * results are those of the direct steps bit for bit.  Any device allocation by the
 * context, a weight or volume change, or a tuning change makes the next step direct and
 * the one after re-capture.  on == 0 runs every step directly and frees the graph. */
rpnn_status rpnn_set_train_graphs(rpnn_ctx* ctx, int32_t on);

/* ---- plain MLP of the architecture comparison (Sec. 7, Fig. 10) -------------------------
 * The paper compares its progressive network with "all-at-once" MLPs that take the whole
 * descriptor in the first layer: shallow-wide (hidden widths 400, 400, 200, 200, 200) and
 * deep-narrow (22 hidden layers of 200).  Here: n_hidden hidden layers of widths[i] (host
 * array), ReLU after every layer including the 1-wide output; input rows of din FP32
 * values (e.g. descriptor rows [10][240], din = 2400, whose zero padding leaves the matching
 * weights inert).  Parameters (FP32, caller-owned, flat): per hidden layer W [w_i][w_{i-1}]
 * row-major then b [w_i], then w_o [1][w_last], b_o.  FP32 CUDA-core GEMMs (autotuned). */
int64_t rpnn_dense_param_count(const int32_t* widths, int32_t n_hidden, int32_t din);   /* -1: bad args */
rpnn_status rpnn_dense_forward(rpnn_ctx* ctx, const int32_t* widths, int32_t n_hidden, int32_t din,
                               const float* dev_params, const float* dev_in, int64_t q, float* dev_out,
                               void* stream);
/* Gradient of sum_i dout_i g(x_i) w.r.t. the parameters, written to dev_dparams. */
rpnn_status rpnn_dense_backward(rpnn_ctx* ctx, const int32_t* widths, int32_t n_hidden, int32_t din,
                                const float* dev_params, const float* dev_in, int64_t q, const float* dev_dout,
                                float* dev_dparams, void* stream);
/* One Adam step on the log-MSE loss (as rpnn_train_step), parameters and moments updated in
 * place, loss (FP64) to *dev_loss. */
rpnn_status rpnn_dense_train_step(rpnn_ctx* ctx, const int32_t* widths, int32_t n_hidden, int32_t din,
                                  const float* dev_in, const float* dev_target, int32_t batch,
                                  const rpnn_adam_cfg* adam, int64_t step, float* dev_params, float* dev_m,
                                  float* dev_v, double* dev_loss, void* stream);

/* ---- stencil-size comparison (Sec. 7, Fig. 10 right) -------------------------------------
 * The progressive network fed by stencils of other resolutions over the standard extent:
 * n_xy x n_xy x (2 n_xy - 1) points at (-1 + h ix, -1 + h iy, -1 + h iz) * 2^(k-1) mean free
 * paths, h = 2 / (n_xy - 1), n_xy in [2, 9] (5: the standard 5 x 5 x 9 stencil).  Level k
 * reads the mip whose voxel is the largest power of two (fine voxels) not above the spacing
 * h 2^(k-1) mean free paths.  Rows are FP32 [q][RPNN_K][din], din = n_xy^2 (2 n_xy - 1) + 1
 * (points in (iz n_xy + iy) n_xy + ix order, then gamma), unpadded.  The network is the
 * standard one (Sec. 4.3) with V^k of width din: parameters (FP32, caller-owned, flat) in
 * the order of rpnn_set_weights.  FP32 CUDA-core GEMMs; at most 2^20 rows per call.
 * Errors: RPNN_ERR_ARG for n_xy outside [2, 9], a bad row count or a null pointer;
 * RPNN_ERR_HANDLE for an unknown volume or one without rpnn_build_mips.  The first
 * rpnn_stencil_descriptors call on a pyramid builds its levels as plain FP32 (volume-owned,
 * about 1.14x the grid) on the given stream. */
int64_t rpnn_stencil_param_count(int32_t n_xy);   /* -1 for n_xy outside [2, 9] */
/* Descriptors of q shading points (dev_x, dev_d [q][3]; light directions dev_wl [3] per
 * point at stride wl_stride floats, 0 for one shared direction) to dev_desc. */
rpnn_status rpnn_stencil_descriptors(rpnn_ctx* ctx, int32_t vol, int32_t n_xy, const float* dev_x,
                                     const float* dev_d, const float* dev_wl, int32_t wl_stride, int64_t q,
                                     float* dev_desc, void* stream);
rpnn_status rpnn_stencil_forward(rpnn_ctx* ctx, int32_t n_xy, const float* dev_params, const float* dev_desc,
                                 int64_t q, float* dev_out, void* stream);
/* Gradient of sum_i dout_i g(z_i) w.r.t. the parameters, written to dev_dparams. */
rpnn_status rpnn_stencil_backward(rpnn_ctx* ctx, int32_t n_xy, const float* dev_params, const float* dev_desc,
                                  int64_t q, const float* dev_dout, float* dev_dparams, void* stream);
/* One Adam step on the log-MSE loss (as rpnn_train_step), loss (FP64) to *dev_loss. */
rpnn_status rpnn_stencil_train_step(rpnn_ctx* ctx, int32_t n_xy, const float* dev_desc, const float* dev_target,
                                    int32_t batch, const rpnn_adam_cfg* adam, int64_t step, float* dev_params,
                                    float* dev_m, float* dev_v, double* dev_loss, void* stream);

/* Arithmetic of rpnn_train_step and rpnn_mlp_backward: RPNN_F32 (the default; FP32 CUDA-core
 * GEMMs) or RPNN_BF16 (mixed precision: every 200-wide layer and weight gradient is a BF16
 * tcgen05 GEMM with FP32 accumulation; FP32 master weights, biases, residual sums, ReLU
 * masks, loss, gradients and Adam; the 1-wide output layer stays FP32).  No counterpart in
 * the paper, which does not state its training arithmetic.  Errors: RPNN_ERR_ARG for any
 * other value. */
rpnn_status rpnn_set_train_precision(rpnn_ctx* ctx, int32_t precision);
/* GEMM-tile autotuner of the FP32 CUDA-core network (forward, backward, the FP32 render
 * form) and of the BF16 tensor-core training GEMMs (tile width 64/128/256 and split-K; no
 * counterpart in the paper).  With `on` != 0 (the default), the first call of
 * each GEMM shape (rows, columns, inner sizes, operand layouts, epilogue kind) times every
 * admissible tile shape and split-K factor on the call's own operands (writing into
 * library scratch, so the call's output is unaffected), synchronising the stream once, and
 * later calls of that shape use the fastest.  Calls made during CUDA-graph capture use a
 * choice already made, else the default tile.  Tile shapes change no result bit (every
 * output sums its products in increasing k); K is split only for inner sizes of at least
 * 1,024 (the weight gradients, which sum over the batch), whose runs' partial sums are
 * added in run order, so those results differ from the default tile by rounding only and
 * are the same from run to run once the choice is made.  Forward results (rpnn_mlp_forward,
 * the FP32 render form) are therefore bit for bit those of the default tile.  With on == 0 every GEMM uses the default
 * 64 x 64 tile without a split and the table is kept. */
rpnn_status rpnn_set_autotune(rpnn_ctx* ctx, int32_t on);
typedef struct {
    int32_t M, N, K0, K1;          /* rows, columns, inner sizes of the two operand segments */
    int32_t flags;                 /* operand layouts and epilogue kind (library-defined bits) */
    int32_t tile_m, tile_n, tile_k, splits;   /* the choice */
    float us, default_us;          /* its measured time and that of the default tile (us) */
} rpnn_tune_entry;
/* Copies up to `cap` entries of the tuning table into out (host) and the table's size to
 * *n (host).  Errors: RPNN_ERR_ARG for cap < 0, n NULL, or out NULL with cap > 0. */
rpnn_status rpnn_get_autotune(rpnn_ctx* ctx, rpnn_tune_entry* out, int32_t cap, int32_t* n);
/* Restores n tuning decisions (as rpnn_get_autotune wrote them, e.g. from a checkpoint):
 * later calls of those shapes use them without timing, so a resumed training run repeats
 * the arithmetic of the run that wrote them bit for bit.  Entries for shapes already in the
 * table replace them.  Errors: RPNN_ERR_ARG for n < 0, entries NULL with n > 0, or a tile
 * shape or split the library does not have. */
rpnn_status rpnn_set_autotune_table(rpnn_ctx* ctx, const rpnn_tune_entry* entries, int32_t n);

#ifdef __cplusplus
}
#endif
#endif
