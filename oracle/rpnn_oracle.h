/*
 * rpnn_oracle.h -- CPU reference ("oracle") for the RPNN cloud-rendering hot path
 * of Kallweit et al., "Deep Scattering: Rendering Atmospheric Clouds with
 * Radiance-Predicting Neural Networks".
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, plain, obviously-correct
 * statement of what the GPU path computes.  Only the test-suite, the smoke check
 * and the CPU-baseline leg of the benchmark load it.  The product path (the CUDA
 * library) never links, loads or calls it, and the two share no code: this header
 * is the oracle's own.
 *
 * Precision: FP64 throughout, except the "_f32" entry points, which restate the
 * mip pyramid and the descriptor in FP32 with one fixed, documented rounding
 * sequence (used to check the GPU descriptor bit for bit).
 *
 * Parity pins (what fixes each function independently of itself) are in the
 * test-suite; functions that have none say "parity unpinned" below.
 */
#ifndef RPNN_ORACLE_H
#define RPNN_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_K 10          /* stencil levels (Sec. 4.2) */
#define ORC_S 225         /* points per level, 5x5x9 (Sec. 4.2) */
#define ORC_DIN 226       /* per-block input z^k = {Sigma^k, gamma} (Sec. 4.3) */
#define ORC_H 200         /* hidden width (Sec. 7) */
#define ORC_MAX_LEVELS 16

typedef struct orc_ctx orc_ctx;

/* ---- counter-based RNG: Philox4x32-10 (Salmon et al. 2011) ---------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* ---- volume + statistics (Sec. 4.2 mean-free-path normalisation, Sec. 5 unit box) */
/* Copies the FP32 density (x fastest).  Returns NULL on bad input. */
orc_ctx* orc_create(const float* density, int nx, int ny, int nz, double albedo, double hg_g);
void orc_destroy(orc_ctx* c);
/* stats: mean over voxels > 0 (fixed-point definition), the same mean summed in
 * long double (for pinning), inv_mean as FP32, majorant, non-zero count, number of
 * mip levels, and the mip level read by each stencil level. */
typedef struct {
    double mean, mean_ld;
    double inv_mean;       /* 1/mean in FP64 */
    float inv_mean_f;      /* (float)(1/mean) */
    float majorant;
    int64_t nonzero;
    int levels;
    int mip_of_level[ORC_K];
    int dims[ORC_MAX_LEVELS][3];
    double h0, inv_h0;
    double ext[3];
    double mip_weight[ORC_K];   /* blended descriptor: weight of level m_k + 1 (FP64) */
    float mip_weight_f[ORC_K];  /* the same, rounded to FP32 */
} orc_stats;
int orc_get_stats(const orc_ctx* c, orc_stats* out);
/* Blended (fractional) mip selection for the descriptor: stencil level k reads
 * (1 - w_k) rho_{m_k} + w_k rho_{m_k + 1}, w_k the fraction of log2(spacing in fine voxels)
 * above m_k (0 where the spacing is outside the pyramid).  Off by default. */
void orc_set_mip_blend(orc_ctx* c, int on);

/* ---- Gaussian mip pyramid (Sec. 6 "Implementation": sigma_i = 2^i) ---------- */
int orc_gauss_taps(int level, double* w, int cap, int* off); /* -> tap count */
/* level values rho = (G_sigma * mu_t)/mean, FP64, written [nz][ny][nx] */
int orc_mip_level_f64(orc_ctx* c, int level, double* out);
/* FP32 fixed-order restatement (bit-exactness reference) */
int orc_mip_level_f32(orc_ctx* c, int level, float* out);

/* ---- hierarchical descriptor (Sec. 4.2, Fig. 5) ---------------------------- */
/* x: q*3 positions (unit box), d: q*3 camera-ray (tracing) directions, wl: light
 * direction (towards the light).  out: q * 10 * 226 (Sigma^k in (iz*5+iy)*5+ix order,
 * then gamma). */
int orc_descriptor_f64(orc_ctx* c, const double* x, const double* d, const double wl[3],
                       int64_t q, double* out);
int orc_descriptor_f32(orc_ctx* c, const float* x, const float* d, const float wl[3],
                       int64_t q, float* out);
/* The same descriptor for an n x n x (2n - 1) stencil over the standard extent (spacing
 * 2 / (n - 1); the stencil-size comparison of Sec. 7): rows [q][ORC_K][din], din =
 * orc_stencil_din(n) = n^2 (2n - 1) + 1 (-1 for n outside [2, 9]); n = 5 is the standard
 * descriptor without its padding.  Level k reads the mip matching the spacing. */
int orc_stencil_din(int n);
int orc_descriptor_stencil_f64(orc_ctx* c, int n, const double* x, const double* d, const double wl[3],
                               int64_t q, double* out);
int orc_descriptor_stencil_f32(orc_ctx* c, int n, const float* x, const float* d, const float wl[3],
                               int64_t q, float* out);
/* local frame, for pinning: ex, ey, ez, gamma */
void orc_frame_f64(const double d[3], const double wl[3], double ex[3], double ey[3],
                   double ez[3], double* gamma);
/* density of the raw grid at p, trilinear, zero outside (FP64) */
double orc_density(const orc_ctx* c, const double p[3]);

/* ---- Monte Carlo transport (Sec. 4.4; Eq. 1) -------------------------------- */
typedef struct {
    double cam_pos[3], cam_fwd[3], cam_right[3], cam_up[3];
    double tan_half_fov_y;
    int width, height, spp;
    uint64_t seed;
    double light_dir[3];   /* unit, towards the light */
    double light_E;        /* irradiance of the directional light */
} orc_camera;

/* Tracking reads a per-brick majorant: bricks of ORC_BRICK^3 fine voxels, each bounded by
 * the largest voxel its trilinear density interpolates (voxels 8b-1 .. 8b+8 per axis). */
#define ORC_BRICK 8
float orc_brick_majorant(const orc_ctx* c, int bx, int by, int bz);   /* -1 outside */
/* The same estimators against the global majorant (the path tracer's bounces; pins). */
int orc_delta_track_global(const orc_ctx* c, const double o[3], const double d[3], uint64_t seed,
                           uint32_t id0, uint32_t id1, uint32_t domain, uint32_t* ctr,
                           double x[3], double* t_out);
double orc_ratio_track_global(const orc_ctx* c, const double o[3], const double d[3], uint64_t seed,
                              uint32_t id0, uint32_t id1, uint32_t domain, uint32_t* ctr, int* capped);
/* The same estimators in a medium of extinction s mu_t (the chopped medium after the first
 * bounce, Sec. 3.1); s = 1 gives the functions above exactly. */
int orc_delta_track_global_scaled(const orc_ctx* c, const double o[3], const double d[3], double s,
                                  uint64_t seed, uint32_t id0, uint32_t id1, uint32_t domain,
                                  uint32_t* ctr, double x[3], double* t_out);
double orc_ratio_track_scaled(const orc_ctx* c, const double o[3], const double d[3], double s,
                              uint64_t seed, uint32_t id0, uint32_t id1, uint32_t domain,
                              uint32_t* ctr, int* capped);

/* Free flight by delta tracking from o along unit d inside the unit-box grid.
 * RNG counter (id0, id1, step, domain).  Returns 1 on collision (x written, t), 0
 * on escape, -1 if the step cap was reached. */
int orc_delta_track(const orc_ctx* c, const double o[3], const double d[3], uint64_t seed,
                    uint32_t id0, uint32_t id1, uint32_t domain, uint32_t* ctr,
                    double x[3], double* t_out);
/* Ratio-tracking transmittance from o along d to the grid boundary. */
double orc_ratio_track(const orc_ctx* c, const double o[3], const double d[3], uint64_t seed,
                       uint32_t id0, uint32_t id1, uint32_t domain, uint32_t* ctr, int* capped);
/* Lorenz-Mie scattering of one sphere (Bohren & Huffman 1983, App. A): size parameter x,
 * relative refractive index m_re + i m_im; s11[k] = (|S1|^2 + |S2|^2) / 2 at cosines mu[k];
 * extinction and scattering efficiencies. */
int orc_mie_single(double x, double m_re, double m_im, const double* mu, int nmu, double* s11, double* qext,
                   double* qsca);
/* The tabulated cloud phase function (water, 0.55 um, Deirmendjian C.1 droplets): bin means
 * p[ORC_LM_BINS] over 0.1-degree bins of scattering angle, cumulative probabilities
 * cdf[ORC_LM_BINS + 1] and bin-edge cosines cos_edges[ORC_LM_BINS + 1]. */
#define ORC_LM_BINS 1800
int orc_lm_table(double* p, double* cdf, double* cos_edges, int n);
/* Volume phase function: 0 Henyey-Greenstein with the volume's g, 1 the Lorenz-Mie table,
 * 2 the Lorenz-Mie table at a path's first bounce and, after it, the table with its first
 * chop_bins bins (the diffraction peak, fraction f of the scattered light) removed and
 * renormalised, in a medium of extinction (1 - f albedo) mu_t and albedo
 * (1 - f) albedo / (1 - f albedo) (Sec. 3.1).  -1 on a bad kind or bin count. */
int orc_set_phase(orc_ctx* c, int kind, int chop_bins);
void orc_set_phase_lm(orc_ctx* c, int on);     /* orc_set_phase(c, on ? 1 : 0, 0) */
/* f, the extinction scale and the albedo after the first bounce (0, 1, albedo unchopped) */
int orc_chop_params(const orc_ctx* c, double* f, double* dscale, double* albedo_c);
/* the chopped table (kind 2 only): bin values p[n], cumulative probabilities cdf[n + 1] */
int orc_lm_chopped_table(const orc_ctx* c, double* p, double* cdf, int n);
/* Henyey-Greenstein phase function of the cosine between propagation directions. */
double orc_hg(double g, double cos_theta);
/* New tracing direction scattered from tracing direction d, cosine ~ HG(g). */
void orc_sample_hg(double g, const double d[3], double xi0, double xi1, double out[3]);

/* Per pixel-sample primary query: hit flag, x, d, L_d (direct in-scattering). */
int orc_primary(const orc_ctx* c, const orc_camera* cam, int64_t pixel, int sample,
                double x[3], double d[3], double* Ld);

/* Render selected pixels.  mode 0: RPNN (params, may be NULL => L_i = 0);
 * mode 1: plain path tracing (multi-scatter, NEE at every vertex).
 * out[i] = pixel value averaged over spp.  Multithreaded over pixels. */
int orc_render_pixels(orc_ctx* c, const orc_camera* cam, const double* params, int mode,
                      const int64_t* pixels, int64_t npix, double* out, int nthreads);
int orc_render(orc_ctx* c, const orc_camera* cam, const double* params, int mode,
               double* image, int nthreads);

/* ---- RPNN network (Sec. 4.3, Fig. 6) ----------------------------------------- */
typedef struct { int K, din, H, ntail; } orc_net;   /* default {10, 226, 200, 3} */
int64_t orc_net_param_count(const orc_net* n);
/* z: q * K * din.  g: q outputs. */
int orc_mlp_forward(const orc_net* n, const double* params, const double* z, int64_t q,
                    double* g);
/* dparams (zeroed by the caller) += d(sum_i dg_i * g_i)/dparams */
int orc_mlp_backward(const orc_net* n, const double* params, const double* z, int64_t q,
                     const double* dg, double* dparams);
/* Sec. 5.2 loss; writes dl/dg_i when dg != NULL */
double orc_logmse_loss(const double* g, const double* target, int64_t b, double* dg);
/* Adam (Kingma & Ba 2014), step t >= 1, bias-corrected */
void orc_adam(double* p, double* m, double* v, const double* grad, int64_t n, int64_t t,
              double lr, double b1, double b2, double eps);

/* ---- training records (Sec. 5.1) ---------------------------------------------- */
/* Samples record `rec`: ray direction d, shading point x, light direction wl, and
 * estimates L_i by path tracing with NEE until the 95% half-width <= rel_ci*mean
 * (at least n_min, at most n_max paths).  Returns 0, or -1 on a cap. */
int orc_gen_record(const orc_ctx* c, uint64_t seed, int64_t rec, double rel_ci, int n_min,
                   int n_max, double x[3], double d[3], double wl[3], double* label,
                   int64_t* npaths, double* half_width);
/* L_i at a given configuration with a fixed number of paths (no stopping rule);
 * max_bounces > 0 truncates every path after that many collisions (pinning only). */
int orc_estimate_Li(const orc_ctx* c, uint64_t seed, uint32_t rec, const double x[3],
                    const double d[3], const double wl[3], int npaths, int max_bounces,
                    double* mean, double* var);

#ifdef __cplusplus
}
#endif
#endif
