/*
 * rpnn_oracle.c -- CPU reference for the RPNN hot path (TEST INFRASTRUCTURE ONLY).
 *
 * Kallweit et al., "Deep Scattering" (Sec. 3.1 Lorenz-Mie phase function, full and chopped;
 * Sec. 3.2 Eq. 1, Sec. 4.2-4.4, Sec. 5, Sec. 6; Sec. 7's stencil sizes).
 * Plain loops, FP64 unless a function name ends in _f32.  No blocking, fusion or
 * reordering beyond what the paper's definitions state; every reading the paper
 * leaves open is fixed in the comments where it is taken.
 *
 * Only the test-suite, the smoke check and the benchmark's CPU-baseline leg use this
 * file.  It shares no code with the CUDA library.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fopenmp -fPIC -shared (the FP32 paths
 * rely on -ffp-contract=off: every product and sum below is rounded on its own
 * unless written as fmaf()).
 */
#include "rpnn_oracle.h"

#include <complex.h>
#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------------- */
/* RNG streams.  Counter = (id0, id1, step, domain); key = seed (lo, hi).      */
/* ------------------------------------------------------------------------- */
enum {
    DOM_CAMERA = 1,    /* pixel jitter */
    DOM_PRIMARY = 2,   /* delta tracking along the camera ray */
    DOM_SHADOW = 3,    /* ratio tracking towards the light (NEE at the primary hit) */
    DOM_PATH = 4,      /* plain path tracing continuation in renders */
    DOM_RECORD = 5,    /* record sampling: direction + disk point */
    DOM_RECTRACK = 6,  /* record free-flight */
    DOM_LIGHT = 7,     /* record light direction */
    DOM_LABEL = 8      /* label path tracing */
};
#define TRACK_CAP 1000000u    /* tentative collisions per tracking call */
#define BOUNCE_CAP 100000     /* collisions per path */
#define RECORD_ATTEMPTS 4096

/* Philox4x32-10 from Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3" (SC'11): 10 rounds of the Philox S-box with multipliers 0xD2511F53,
 * 0xCD9E8D57 and the Weyl key schedule 0x9E3779B9, 0xBB67AE85. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void draw(uint64_t seed, uint32_t id0, uint32_t id1, uint32_t step, uint32_t dom,
                 double xi[4]) {
    uint32_t ctr[4] = {id0, id1, step, dom};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t r[4];
    orc_philox4x32_10(ctr, key, r);
    for (int i = 0; i < 4; ++i) xi[i] = (double)(r[i] >> 8) * 0x1p-24; /* [0, 1) */
}

/* ------------------------------------------------------------------------- */
/* Volume                                                                      */
/* ------------------------------------------------------------------------- */
struct orc_ctx {
    int n[3];
    float* dens;
    double albedo, g;
    orc_stats st;
    int nb[3];          /* bricks of ORC_BRICK^3 voxels per axis */
    int mip_blend;      /* descriptor blends levels m_k and m_k + 1 (orc_set_mip_blend) */
    int phase_lm;       /* phase function: 0 Henyey-Greenstein (g), 1 tabulated Lorenz-Mie,
                         * 2 Lorenz-Mie at the first bounce, chopped afterwards (orc_set_phase) */
    double chop_f;      /* fraction of scattered light in the chopped forward peak */
    double dscale;      /* extinction scale after the first bounce: 1 - f albedo (1 unchopped) */
    double albedo_c;    /* albedo after the first bounce: albedo (1 - f) / (1 - f albedo) */
    double* lmc_p;      /* chopped table: bin values, cumulative probabilities */
    double* lmc_cdf;
    float* bmaj;        /* per-brick majorant [nb2][nb1][nb0] */
    double* mip64[ORC_MAX_LEVELS];
    float* mip32[ORC_MAX_LEVELS];
};

static int imax3(int a, int b, int c) { int m = a > b ? a : b; return m > c ? m : c; }

/* Mean over non-zero voxels (Sec. 4.2).  Definition used here: every voxel value v>0 is
 * truncated to a fixed-point integer with 32 fraction bits below the majorant's
 * binary exponent, the integers are summed exactly, and the sum is scaled back and
 * divided by the count in FP64.  The result is independent of summation order. */
static void compute_stats(orc_ctx* c) {
    orc_stats* s = &c->st;
    const int64_t nv = (int64_t)c->n[0] * c->n[1] * c->n[2];
    float mx = 0.0f;
    int64_t nz = 0;
    long double sum_ld = 0.0L;
    for (int64_t i = 0; i < nv; ++i) {
        float v = c->dens[i];
        if (v > mx) mx = v;
        if (v > 0.0f) { ++nz; sum_ld += (long double)v; }
    }
    int e = 0;
    frexpf(mx, &e);             /* mx < 2^e */
    int S = 32 - e;
    int64_t isum = 0;
    for (int64_t i = 0; i < nv; ++i) {
        float v = c->dens[i];
        if (v > 0.0f) isum += (int64_t)ldexp((double)v, S);
    }
    s->majorant = mx;
    s->nonzero = nz;
    s->mean = nz ? ldexp((double)isum, -S) / (double)nz : 0.0;
    s->mean_ld = nz ? (double)(sum_ld / (long double)nz) : 0.0;
    s->inv_mean = nz ? 1.0 / s->mean : 0.0;
    s->inv_mean_f = (float)s->inv_mean;
    const int nmax = imax3(c->n[0], c->n[1], c->n[2]);
    s->h0 = 1.0 / (double)nmax;
    s->inv_h0 = (double)nmax;
    for (int a = 0; a < 3; ++a) s->ext[a] = (double)c->n[a] * s->h0;
    /* levels i = 0 .. L-1, level L-1 is the first whose largest dimension is 1 */
    int L = 1;
    while (((nmax + (1 << (L - 1)) - 1) >> (L - 1)) > 1) ++L;
    s->levels = L;
    for (int i = 0; i < ORC_MAX_LEVELS; ++i)
        for (int a = 0; a < 3; ++a) s->dims[i][a] = (c->n[a] + (1 << i) - 1) >> i;
    /* Mip level read by stencil level k (the paper is silent, Sec. 6 only says a
     * Gaussian mipmap is used): the level whose voxel size is the largest power of two
     * not above the stencil spacing 0.5 * 2^(k-1) mean free paths. */
    for (int k = 0; k < ORC_K; ++k) {
        double sk = 0.5 * ldexp((double)s->inv_mean_f, k) * s->inv_h0; /* fine voxels */
        int m = 0;
        if (sk > 0.0) { int ex; frexp(sk, &ex); m = ex - 1; }
        if (m < 0) m = 0;
        if (m > L - 1) m = L - 1;
        s->mip_of_level[k] = m;
        /* fractional level for the blended descriptor: log2 of the spacing; the weight of
         * level m + 1 is its fraction above m (0 where the spacing falls outside the
         * pyramid's range, which keeps the clamped level alone) */
        double w = 0.0;
        if (sk > 0.0) {
            const double mr = log2(sk);
            if (mr > 0.0 && mr < (double)(L - 1)) w = mr - floor(mr);
        }
        s->mip_weight[k] = w;
        s->mip_weight_f[k] = (float)w;
    }
}

void orc_set_mip_blend(orc_ctx* c, int on) { c->mip_blend = on != 0; }

/* Majorant of each brick of ORC_BRICK^3 voxels for tracking (Sec. 7 names spatial
 * acceleration of the Monte Carlo part; per-brick majorants are the standard piecewise-
 * constant bound): brick b covers fine voxel-centre coordinates [8b - 1/2, 8b + 8 - 1/2]
 * per axis, where the trilinear density interpolates voxels 8b - 1 .. 8b + 8, so the
 * largest of those voxels (zero outside the grid) bounds the density in the brick. */
static void compute_brick_majorants(orc_ctx* c) {
    for (int a = 0; a < 3; ++a) c->nb[a] = (c->n[a] + ORC_BRICK - 1) / ORC_BRICK;
    c->bmaj = (float*)calloc((size_t)c->nb[0] * c->nb[1] * c->nb[2], sizeof(float));
    for (int bz = 0; bz < c->nb[2]; ++bz)
        for (int by = 0; by < c->nb[1]; ++by)
            for (int bx = 0; bx < c->nb[0]; ++bx) {
                float m = 0.0f;
                for (int z = bz * ORC_BRICK - 1; z <= bz * ORC_BRICK + ORC_BRICK; ++z)
                    for (int y = by * ORC_BRICK - 1; y <= by * ORC_BRICK + ORC_BRICK; ++y)
                        for (int x = bx * ORC_BRICK - 1; x <= bx * ORC_BRICK + ORC_BRICK; ++x) {
                            if (x < 0 || y < 0 || z < 0 || x >= c->n[0] || y >= c->n[1] || z >= c->n[2]) continue;
                            const float v = c->dens[((size_t)z * c->n[1] + y) * c->n[0] + x];
                            if (v > m) m = v;
                        }
                c->bmaj[((size_t)bz * c->nb[1] + by) * c->nb[0] + bx] = m;
            }
}

float orc_brick_majorant(const orc_ctx* c, int bx, int by, int bz) {
    if (bx < 0 || by < 0 || bz < 0 || bx >= c->nb[0] || by >= c->nb[1] || bz >= c->nb[2]) return -1.0f;
    return c->bmaj[((size_t)bz * c->nb[1] + by) * c->nb[0] + bx];
}

orc_ctx* orc_create(const float* density, int nx, int ny, int nz, double albedo, double hg_g) {
    if (!density || nx <= 0 || ny <= 0 || nz <= 0) return NULL;
    const int64_t nv = (int64_t)nx * ny * nz;
    for (int64_t i = 0; i < nv; ++i)
        if (!(density[i] >= 0.0f) || isinf(density[i])) return NULL;
    orc_ctx* c = (orc_ctx*)calloc(1, sizeof(orc_ctx));
    c->n[0] = nx; c->n[1] = ny; c->n[2] = nz;
    c->dens = (float*)malloc(sizeof(float) * nv);
    memcpy(c->dens, density, sizeof(float) * nv);
    c->albedo = albedo;
    c->albedo_c = albedo;
    c->dscale = 1.0;
    c->g = hg_g;
    compute_stats(c);
    if (c->st.nonzero == 0) { orc_destroy(c); return NULL; }
    compute_brick_majorants(c);
    return c;
}

void orc_destroy(orc_ctx* c) {
    if (!c) return;
    for (int i = 0; i < ORC_MAX_LEVELS; ++i) { free(c->mip64[i]); free(c->mip32[i]); }
    free(c->dens);
    free(c->bmaj);
    free(c->lmc_p);
    free(c->lmc_cdf);
    free(c);
}

int orc_get_stats(const orc_ctx* c, orc_stats* out) {
    if (!c || !out) return -1;
    *out = c->st;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Gaussian mip pyramid of the density (Sec. 6, Implementation; sigma_i = 2^i).      */
/* Readings: sigma in fine voxels; level i sampled at level-i voxel centres, i.e.    */
/* fine coordinate (j + 0.5) 2^i - 0.5; kernel truncated to |offset| <= 3 sigma and */
/* normalised over the truncated support; zero outside the grid (mu_t = 0 on the    */
/* boundary, Eq. 1); values divided by the mean (rho, Sec. 4.2).                     */
/* ------------------------------------------------------------------------- */
int orc_gauss_taps(int level, double* w, int cap, int* off) {
    if (level < 0 || level >= ORC_MAX_LEVELS) return -1;
    const double sigma = ldexp(1.0, level);
    int T;
    if (level == 0) { T = 7; *off = -3; }
    else { T = 6 << level; *off = (1 << (level - 1)) - 3 * (1 << level); }
    if (T > cap) return -1;
    double sum = 0.0;
    for (int m = 0; m < T; ++m) {
        double d = (level == 0) ? (double)(m - 3) : (double)m - 3.0 * sigma + 0.5;
        w[m] = exp(-d * d / (2.0 * sigma * sigma));
        sum += w[m];
    }
    for (int m = 0; m < T; ++m) w[m] /= sum;
    return T;
}

static int level_ok(const orc_ctx* c, int level) {
    return c && level >= 0 && level < c->st.levels;
}

int orc_mip_level_f64(orc_ctx* c, int level, double* out) {
    if (!level_ok(c, level)) return -1;
    const int nx = c->n[0], ny = c->n[1], nz = c->n[2];
    const int ax = c->st.dims[level][0], ay = c->st.dims[level][1], az = c->st.dims[level][2];
    const int T = (level == 0) ? 7 : (6 << level);
    double* w = (double*)malloc(sizeof(double) * T);
    int off;
    orc_gauss_taps(level, w, T, &off);
    const int st = 1 << level;
    double* A = (double*)calloc((size_t)ax * ny * nz, sizeof(double));
    double* B = (double*)calloc((size_t)ax * ay * nz, sizeof(double));
    /* separable: x, then y, then z */
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int j = 0; j < ax; ++j) {
                double acc = 0.0;
                for (int m = 0; m < T; ++m) {
                    int t = j * st + off + m;
                    if (t >= 0 && t < nx) acc += w[m] * (double)c->dens[((size_t)z * ny + y) * nx + t];
                }
                A[((size_t)z * ny + y) * ax + j] = acc;
            }
    for (int z = 0; z < nz; ++z)
        for (int j = 0; j < ay; ++j)
            for (int x = 0; x < ax; ++x) {
                double acc = 0.0;
                for (int m = 0; m < T; ++m) {
                    int t = j * st + off + m;
                    if (t >= 0 && t < ny) acc += w[m] * A[((size_t)z * ny + t) * ax + x];
                }
                B[((size_t)z * ay + j) * ax + x] = acc;
            }
    for (int j = 0; j < az; ++j)
        for (int y = 0; y < ay; ++y)
            for (int x = 0; x < ax; ++x) {
                double acc = 0.0;
                for (int m = 0; m < T; ++m) {
                    int t = j * st + off + m;
                    if (t >= 0 && t < nz) acc += w[m] * B[((size_t)t * ay + y) * ax + x];
                }
                out[((size_t)j * ay + y) * ax + x] = acc * c->st.inv_mean;
            }
    free(A); free(B); free(w);
    return 0;
}

/* FP32 restatement: FP64 weights rounded to FP32; each pass accumulates taps in
 * ascending order, acc = acc + w*v with the product and the sum rounded separately;
 * final value = acc * inv_mean_f. */
int orc_mip_level_f32(orc_ctx* c, int level, float* out) {
    if (!level_ok(c, level)) return -1;
    const int nx = c->n[0], ny = c->n[1], nz = c->n[2];
    const int ax = c->st.dims[level][0], ay = c->st.dims[level][1], az = c->st.dims[level][2];
    const int T = (level == 0) ? 7 : (6 << level);
    double* wd = (double*)malloc(sizeof(double) * T);
    float* w = (float*)malloc(sizeof(float) * T);
    int off;
    orc_gauss_taps(level, wd, T, &off);
    for (int m = 0; m < T; ++m) w[m] = (float)wd[m];
    const int st = 1 << level;
    float* A = (float*)calloc((size_t)ax * ny * nz, sizeof(float));
    float* B = (float*)calloc((size_t)ax * ay * nz, sizeof(float));
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int j = 0; j < ax; ++j) {
                float acc = 0.0f;
                for (int m = 0; m < T; ++m) {
                    int t = j * st + off + m;
                    if (t >= 0 && t < nx) {
                        float p = w[m] * c->dens[((size_t)z * ny + y) * nx + t];
                        acc = acc + p;
                    }
                }
                A[((size_t)z * ny + y) * ax + j] = acc;
            }
    for (int z = 0; z < nz; ++z)
        for (int j = 0; j < ay; ++j)
            for (int x = 0; x < ax; ++x) {
                float acc = 0.0f;
                for (int m = 0; m < T; ++m) {
                    int t = j * st + off + m;
                    if (t >= 0 && t < ny) {
                        float p = w[m] * A[((size_t)z * ny + t) * ax + x];
                        acc = acc + p;
                    }
                }
                B[((size_t)z * ay + j) * ax + x] = acc;
            }
    for (int j = 0; j < az; ++j)
        for (int y = 0; y < ay; ++y)
            for (int x = 0; x < ax; ++x) {
                float acc = 0.0f;
                for (int m = 0; m < T; ++m) {
                    int t = j * st + off + m;
                    if (t >= 0 && t < nz) {
                        float p = w[m] * B[((size_t)t * ay + y) * ax + x];
                        acc = acc + p;
                    }
                }
                out[((size_t)j * ay + y) * ax + x] = acc * c->st.inv_mean_f;
            }
    free(A); free(B); free(w); free(wd);
    return 0;
}

static const double* get_mip64(orc_ctx* c, int level) {
    if (!c->mip64[level]) {
        const int* d = c->st.dims[level];
        double* buf = (double*)malloc(sizeof(double) * (size_t)d[0] * d[1] * d[2]);
        orc_mip_level_f64(c, level, buf);
#pragma omp critical(orc_mip)
        {
            if (!c->mip64[level]) { c->mip64[level] = buf; buf = NULL; }
        }
        free(buf);
    }
    return c->mip64[level];
}

static const float* get_mip32(orc_ctx* c, int level) {
    if (!c->mip32[level]) {
        const int* d = c->st.dims[level];
        float* buf = (float*)malloc(sizeof(float) * (size_t)d[0] * d[1] * d[2]);
        orc_mip_level_f32(c, level, buf);
#pragma omp critical(orc_mip)
        {
            if (!c->mip32[level]) { c->mip32[level] = buf; buf = NULL; }
        }
        free(buf);
    }
    return c->mip32[level];
}

/* ------------------------------------------------------------------------- */
/* Trilinear interpolation at voxel-centre convention, zero outside the grid.  */
/* u is the continuous voxel coordinate (voxel j has its centre at u = j).      */
/* ------------------------------------------------------------------------- */
static double fetch64(const double* v, const int* d, int x, int y, int z) {
    if (x < 0 || y < 0 || z < 0 || x >= d[0] || y >= d[1] || z >= d[2]) return 0.0;
    return v[((size_t)z * d[1] + y) * d[0] + x];
}

static double lerp64(double a, double b, double f) { return a + f * (b - a); }

static double trilinear64(const double* v, const int* d, const double u[3]) {
    double fl[3], f[3];
    int i[3];
    for (int a = 0; a < 3; ++a) {
        fl[a] = floor(u[a]);
        f[a] = u[a] - fl[a];
        if (fl[a] < -1.0 || fl[a] > (double)(d[a] - 1)) return 0.0;
        i[a] = (int)fl[a];
    }
    double c00 = lerp64(fetch64(v, d, i[0], i[1], i[2]), fetch64(v, d, i[0] + 1, i[1], i[2]), f[0]);
    double c10 = lerp64(fetch64(v, d, i[0], i[1] + 1, i[2]), fetch64(v, d, i[0] + 1, i[1] + 1, i[2]), f[0]);
    double c01 = lerp64(fetch64(v, d, i[0], i[1], i[2] + 1), fetch64(v, d, i[0] + 1, i[1], i[2] + 1), f[0]);
    double c11 = lerp64(fetch64(v, d, i[0], i[1] + 1, i[2] + 1), fetch64(v, d, i[0] + 1, i[1] + 1, i[2] + 1), f[0]);
    return lerp64(lerp64(c00, c10, f[1]), lerp64(c01, c11, f[1]), f[2]);
}

static float fetch32(const float* v, const int* d, int x, int y, int z) {
    if (x < 0 || y < 0 || z < 0 || x >= d[0] || y >= d[1] || z >= d[2]) return 0.0f;
    return v[((size_t)z * d[1] + y) * d[0] + x];
}

/* FP32 lerp(a, b, f) = fma(f, b - a, a): one rounding for b - a, one for the fma. */
static float lerp32(float a, float b, float f) { return fmaf(f, b - a, a); }

static float trilinear32(const float* v, const int* d, const float u[3]) {
    float f[3];
    int i[3];
    for (int a = 0; a < 3; ++a) {
        float uu = fminf(fmaxf(u[a], -1.0e6f), 1.0e6f);
        float fl = floorf(uu);
        f[a] = uu - fl;
        i[a] = (int)fl;
        if (i[a] < -1 || i[a] > d[a] - 1) return 0.0f;
    }
    float c00 = lerp32(fetch32(v, d, i[0], i[1], i[2]), fetch32(v, d, i[0] + 1, i[1], i[2]), f[0]);
    float c10 = lerp32(fetch32(v, d, i[0], i[1] + 1, i[2]), fetch32(v, d, i[0] + 1, i[1] + 1, i[2]), f[0]);
    float c01 = lerp32(fetch32(v, d, i[0], i[1], i[2] + 1), fetch32(v, d, i[0] + 1, i[1], i[2] + 1), f[0]);
    float c11 = lerp32(fetch32(v, d, i[0], i[1] + 1, i[2] + 1), fetch32(v, d, i[0] + 1, i[1] + 1, i[2] + 1), f[0]);
    float c0 = lerp32(c00, c10, f[1]);
    float c1 = lerp32(c01, c11, f[1]);
    return lerp32(c0, c1, f[2]);
}

/* raw-grid density for tracking (the paper is silent; trilinear, zero outside) */
double orc_density(const orc_ctx* c, const double p[3]) {
    double u[3];
    for (int a = 0; a < 3; ++a) u[a] = p[a] * c->st.inv_h0 - 0.5;
    /* the raw grid viewed as FP64 values */
    double fl[3], f[3];
    int i[3];
    for (int a = 0; a < 3; ++a) {
        fl[a] = floor(u[a]);
        f[a] = u[a] - fl[a];
        if (fl[a] < -1.0 || fl[a] > (double)(c->n[a] - 1)) return 0.0;
        i[a] = (int)fl[a];
    }
#define RAW(x, y, z) \
    (((x) < 0 || (y) < 0 || (z) < 0 || (x) >= c->n[0] || (y) >= c->n[1] || (z) >= c->n[2]) \
         ? 0.0 : (double)c->dens[((size_t)(z) * c->n[1] + (y)) * c->n[0] + (x)])
    double c00 = lerp64(RAW(i[0], i[1], i[2]), RAW(i[0] + 1, i[1], i[2]), f[0]);
    double c10 = lerp64(RAW(i[0], i[1] + 1, i[2]), RAW(i[0] + 1, i[1] + 1, i[2]), f[0]);
    double c01 = lerp64(RAW(i[0], i[1], i[2] + 1), RAW(i[0] + 1, i[1], i[2] + 1), f[0]);
    double c11 = lerp64(RAW(i[0], i[1] + 1, i[2] + 1), RAW(i[0] + 1, i[1] + 1, i[2] + 1), f[0]);
#undef RAW
    return lerp64(lerp64(c00, c10, f[1]), lerp64(c01, c11, f[1]), f[2]);
}

/* ------------------------------------------------------------------------- */
/* Descriptor (Sec. 4.2).                                                       */
/* Frame: z-axis = light direction wl; x-axis perpendicular to the plane of z and */
/* omega (omega = -d is the propagation direction, Eq. 1 uses x_u = x - u omega),  */
/* x = normalize(z cross omega); y = z cross x.  Degenerate (omega parallel to z):  */
/* x from the orthonormal basis of Duff et al. 2017 built around z.              */
/* gamma = acos(omega . wl), radians.                                            */
/* Stencil point (ix, iy, iz), ix, iy in 0..4, iz in 0..8, index (iz*5+iy)*5+ix,    */
/* offset o = (-1 + ix/2, -1 + iy/2, -1 + iz/2) mean free paths, scaled by        */
/* 2^(k-1) at level k; one mean free path = 1/mean world units.                   */
/* ------------------------------------------------------------------------- */
static void duff_basis(const double n[3], double b1[3], double b2[3]) {
    double sign = copysign(1.0, n[2]);
    double a = -1.0 / (sign + n[2]);
    double b = n[0] * n[1] * a;
    b1[0] = 1.0 + sign * n[0] * n[0] * a; b1[1] = sign * b; b1[2] = -sign * n[0];
    b2[0] = b; b2[1] = sign + n[1] * n[1] * a; b2[2] = -n[1];
}

/* The first vector of the same basis in FP32 with one fixed rounding sequence (the FP32
 * restatement's degenerate frame): sign = copysign(1, z), a = -1 / (sign + z),
 * x = (1 + ((sign x) x) a, sign ((x y) a), -sign x), every operation rounded to float. */
static void duff_x_f32(const float n[3], float b1[3]) {
    const float sign = signbit(n[2]) ? -1.0f : 1.0f;
    const float a = -1.0f / (sign + n[2]);
    b1[0] = 1.0f + ((sign * n[0]) * n[0]) * a;
    b1[1] = sign * ((n[0] * n[1]) * a);
    b1[2] = -sign * n[0];
}

static void cross64(const double a[3], const double b[3], double o[3]) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

void orc_frame_f64(const double d[3], const double wl[3], double ex[3], double ey[3],
                   double ez[3], double* gamma) {
    double w[3] = {-d[0], -d[1], -d[2]};
    for (int a = 0; a < 3; ++a) ez[a] = wl[a];
    double c[3];
    cross64(ez, w, c);
    double len2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
    if (len2 < 1e-12) {
        double b2[3];
        duff_basis(ez, ex, b2);
    } else {
        double len = sqrt(len2);
        for (int a = 0; a < 3; ++a) ex[a] = c[a] / len;
    }
    cross64(ez, ex, ey);
    double cg = w[0] * wl[0] + w[1] * wl[1] + w[2] * wl[2];
    if (cg > 1.0) cg = 1.0;
    if (cg < -1.0) cg = -1.0;
    *gamma = acos(cg);
}

int orc_descriptor_f64(orc_ctx* c, const double* x, const double* d, const double wl[3],
                       int64_t q, double* out) {
    if (!c) return -1;
    const double* lv[ORC_K];
    const double* lv1[ORC_K];
    for (int k = 0; k < ORC_K; ++k) {
        lv[k] = get_mip64(c, c->st.mip_of_level[k]);
        lv1[k] = (c->mip_blend && c->st.mip_weight[k] > 0.0) ? get_mip64(c, c->st.mip_of_level[k] + 1) : NULL;
    }
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < q; ++i) {
        double ex[3], ey[3], ez[3], gamma;
        orc_frame_f64(d + 3 * i, wl, ex, ey, ez, &gamma);
        double* o = out + i * (ORC_K * ORC_DIN);
        for (int k = 0; k < ORC_K; ++k) {
            const int m = c->st.mip_of_level[k];
            const double scale = ldexp(c->st.inv_mean, k);      /* 2^(k-1) mfp, k 1-based */
            const double s_m = ldexp(c->st.inv_h0, -m);          /* level-m voxels per unit */
            const double w = c->st.mip_weight[k];
            for (int iz = 0; iz < 9; ++iz)
                for (int iy = 0; iy < 5; ++iy)
                    for (int ix = 0; ix < 5; ++ix) {
                        double ox = -1.0 + 0.5 * ix, oy = -1.0 + 0.5 * iy, oz = -1.0 + 0.5 * iz;
                        double p[3], u[3];
                        for (int a = 0; a < 3; ++a) {
                            p[a] = x[3 * i + a] + scale * (ox * ex[a] + oy * ey[a] + oz * ez[a]);
                            u[a] = p[a] * s_m - 0.5;
                        }
                        double r = trilinear64(lv[k], c->st.dims[m], u);
                        if (lv1[k]) {   /* blended: (1 - w) rho_m + w rho_{m+1} */
                            for (int a = 0; a < 3; ++a) u[a] = p[a] * (0.5 * s_m) - 0.5;
                            r = (1.0 - w) * r + w * trilinear64(lv1[k], c->st.dims[m + 1], u);
                        }
                        o[k * ORC_DIN + (iz * 5 + iy) * 5 + ix] = r;
                    }
            o[k * ORC_DIN + ORC_S] = gamma;
        }
    }
    return 0;
}

/* FP32 restatement of the same descriptor with one fixed rounding sequence:
 *   omega = -d; c = ez x omega (each product rounded, then the difference);
 *   len2 = (c0*c0 + c1*c1) + c2*c2; ex = c / sqrtf(len2) (correctly rounded ops);
 *   degenerate (len2 < 1e-12): Duff basis in FP32 (duff_x_f32);
 *   ey = ez x ex; cos gamma = (w0*l0 + w1*l1) + w2*l2, clamped; gamma = acosf;
 *   level k (0-based here): s = inv_h0 * 2^-m, g = (inv_mean_f * 2^k) * s,
 *   A = g*ex, B = g*ey, C = g*ez, U0 = x*s - 0.5,
 *   u = fma(oz, C, fma(oy, B, fma(ox, A, U0))) per axis; rho = trilinear32(u). */
int orc_descriptor_f32(orc_ctx* c, const float* x, const float* d, const float wl[3],
                       int64_t q, float* out) {
    if (!c) return -1;
    const float* lv[ORC_K];
    const float* lv1[ORC_K];
    for (int k = 0; k < ORC_K; ++k) {
        lv[k] = get_mip32(c, c->st.mip_of_level[k]);
        lv1[k] = (c->mip_blend && c->st.mip_weight[k] > 0.0) ? get_mip32(c, c->st.mip_of_level[k] + 1) : NULL;
    }
    const float inv_h0 = (float)c->st.inv_h0;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < q; ++i) {
        const float* xi = x + 3 * i;
        const float* di = d + 3 * i;
        float w[3] = {-di[0], -di[1], -di[2]};
        float ez[3] = {wl[0], wl[1], wl[2]};
        float cr[3];
        { float p, r;
          p = ez[1] * w[2]; r = ez[2] * w[1]; cr[0] = p - r;
          p = ez[2] * w[0]; r = ez[0] * w[2]; cr[1] = p - r;
          p = ez[0] * w[1]; r = ez[1] * w[0]; cr[2] = p - r; }
        float len2;
        { float a = cr[0] * cr[0], b = cr[1] * cr[1], e = cr[2] * cr[2]; len2 = (a + b) + e; }
        float ex[3];
        if (len2 < 1e-12f) {
            duff_x_f32(ez, ex);
        } else {
            float len = sqrtf(len2);
            for (int a = 0; a < 3; ++a) ex[a] = cr[a] / len;
        }
        float ey[3];
        { float p, r;
          p = ez[1] * ex[2]; r = ez[2] * ex[1]; ey[0] = p - r;
          p = ez[2] * ex[0]; r = ez[0] * ex[2]; ey[1] = p - r;
          p = ez[0] * ex[1]; r = ez[1] * ex[0]; ey[2] = p - r; }
        float cg;
        { float a = w[0] * wl[0], b = w[1] * wl[1], e = w[2] * wl[2]; cg = (a + b) + e; }
        cg = fminf(fmaxf(cg, -1.0f), 1.0f);
        const float gamma = acosf(cg);
        float* o = out + i * (ORC_K * ORC_DIN);
        for (int k = 0; k < ORC_K; ++k) {
            const int m = c->st.mip_of_level[k];
            const float s = ldexpf(inv_h0, -m);
            const float g = ldexpf(c->st.inv_mean_f, k) * s;
            float A[3], B[3], C[3], U0[3];
            for (int a = 0; a < 3; ++a) {
                A[a] = g * ex[a]; B[a] = g * ey[a]; C[a] = g * ez[a];
                float xs = xi[a] * s;
                U0[a] = xs - 0.5f;
            }
            /* level m + 1: the same formulas with s1 = inv_h0 * 2^-(m+1) */
            const float s1 = ldexpf(inv_h0, -(m + 1));
            const float g1 = ldexpf(c->st.inv_mean_f, k) * s1;
            float A1[3], B1[3], C1[3], U01[3];
            for (int a = 0; a < 3; ++a) {
                A1[a] = g1 * ex[a]; B1[a] = g1 * ey[a]; C1[a] = g1 * ez[a];
                float xs = xi[a] * s1;
                U01[a] = xs - 0.5f;
            }
            for (int iz = 0; iz < 9; ++iz)
                for (int iy = 0; iy < 5; ++iy)
                    for (int ix = 0; ix < 5; ++ix) {
                        const float ox = -1.0f + 0.5f * (float)ix;
                        const float oy = -1.0f + 0.5f * (float)iy;
                        const float oz = -1.0f + 0.5f * (float)iz;
                        float u[3];
                        for (int a = 0; a < 3; ++a)
                            u[a] = fmaf(oz, C[a], fmaf(oy, B[a], fmaf(ox, A[a], U0[a])));
                        float r = trilinear32(lv[k], c->st.dims[m], u);
                        if (lv1[k]) {   /* blended: lerp(rho_m, rho_{m+1}, w) at level m + 1's coordinates */
                            for (int a = 0; a < 3; ++a)
                                u[a] = fmaf(oz, C1[a], fmaf(oy, B1[a], fmaf(ox, A1[a], U01[a])));
                            r = lerp32(r, trilinear32(lv1[k], c->st.dims[m + 1], u), c->st.mip_weight_f[k]);
                        }
                        o[k * ORC_DIN + (iz * 5 + iy) * 5 + ix] = r;
                    }
            o[k * ORC_DIN + ORC_S] = gamma;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Other stencil resolutions (the stencil-size comparison of Sec. 7, Fig. 10):   */
/* n x n x (2n - 1) points over the standard stencil's extent [-1,1]^2 x [-1,3],   */
/* spacing h = 2 / (n - 1) (n = 5: the standard 5 x 5 x 9 stencil), index          */
/* (iz*n + iy)*n + ix, then gamma; level k reads the mip whose voxel is the largest */
/* power of two (fine voxels) not above the spacing h 2^(k-1) mean free paths.      */
/* ------------------------------------------------------------------------- */
int orc_stencil_din(int n) {
    if (n < 2 || n > 9) return -1;
    return n * n * (2 * n - 1) + 1;
}

static int stencil_mip(const orc_ctx* c, int n, int k) {
    const double h = 2.0 / (double)(n - 1);
    const double sk = h * ldexp((double)c->st.inv_mean_f, k) * c->st.inv_h0;   /* fine voxels */
    int m = 0;
    if (sk > 0.0) { int ex; frexp(sk, &ex); m = ex - 1; }
    if (m < 0) m = 0;
    if (m > c->st.levels - 1) m = c->st.levels - 1;
    return m;
}

int orc_descriptor_stencil_f64(orc_ctx* c, int n, const double* x, const double* d, const double wl[3],
                               int64_t q, double* out) {
    const int din = orc_stencil_din(n);
    if (!c || din < 0) return -1;
    const int nz = 2 * n - 1, S = din - 1;
    const double h = 2.0 / (double)(n - 1);
    int mk[ORC_K];
    const double* lv[ORC_K];
    for (int k = 0; k < ORC_K; ++k) { mk[k] = stencil_mip(c, n, k); lv[k] = get_mip64(c, mk[k]); }
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < q; ++i) {
        double ex[3], ey[3], ez[3], gamma;
        orc_frame_f64(d + 3 * i, wl, ex, ey, ez, &gamma);
        double* o = out + i * (int64_t)ORC_K * din;
        for (int k = 0; k < ORC_K; ++k) {
            const double scale = ldexp(c->st.inv_mean, k);
            const double s_m = ldexp(c->st.inv_h0, -mk[k]);
            for (int iz = 0; iz < nz; ++iz)
                for (int iy = 0; iy < n; ++iy)
                    for (int ix = 0; ix < n; ++ix) {
                        const double ox = -1.0 + h * ix, oy = -1.0 + h * iy, oz = -1.0 + h * iz;
                        double u[3];
                        for (int a = 0; a < 3; ++a)
                            u[a] = (x[3 * i + a] + scale * (ox * ex[a] + oy * ey[a] + oz * ez[a])) * s_m - 0.5;
                        o[k * din + (iz * n + iy) * n + ix] = trilinear64(lv[k], c->st.dims[mk[k]], u);
                    }
            o[k * din + S] = gamma;
        }
    }
    return 0;
}

/* FP32 restatement with the standard descriptor's rounding sequence (orc_descriptor_f32)
 * and the offsets -1 + h_f i, h_f = (float)(2 / (n - 1)), each product and sum rounded. */
int orc_descriptor_stencil_f32(orc_ctx* c, int n, const float* x, const float* d, const float wl[3],
                               int64_t q, float* out) {
    const int din = orc_stencil_din(n);
    if (!c || din < 0) return -1;
    const int nz = 2 * n - 1, S = din - 1;
    const float hf = (float)(2.0 / (double)(n - 1));
    int mk[ORC_K];
    const float* lv[ORC_K];
    for (int k = 0; k < ORC_K; ++k) { mk[k] = stencil_mip(c, n, k); lv[k] = get_mip32(c, mk[k]); }
    const float inv_h0 = (float)c->st.inv_h0;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < q; ++i) {
        const float* xi = x + 3 * i;
        const float* di = d + 3 * i;
        float w[3] = {-di[0], -di[1], -di[2]};
        const float* ez = wl;
        float cr[3];
        { float p, r;
          p = ez[1] * w[2]; r = ez[2] * w[1]; cr[0] = p - r;
          p = ez[2] * w[0]; r = ez[0] * w[2]; cr[1] = p - r;
          p = ez[0] * w[1]; r = ez[1] * w[0]; cr[2] = p - r; }
        float len2;
        { float a = cr[0] * cr[0], b = cr[1] * cr[1], e = cr[2] * cr[2]; len2 = (a + b) + e; }
        float ex[3];
        if (len2 < 1e-12f) {
            duff_x_f32(ez, ex);
        } else {
            float len = sqrtf(len2);
            for (int a = 0; a < 3; ++a) ex[a] = cr[a] / len;
        }
        float ey[3];
        { float p, r;
          p = ez[1] * ex[2]; r = ez[2] * ex[1]; ey[0] = p - r;
          p = ez[2] * ex[0]; r = ez[0] * ex[2]; ey[1] = p - r;
          p = ez[0] * ex[1]; r = ez[1] * ex[0]; ey[2] = p - r; }
        float cg;
        { float a = w[0] * wl[0], b = w[1] * wl[1], e = w[2] * wl[2]; cg = (a + b) + e; }
        cg = fminf(fmaxf(cg, -1.0f), 1.0f);
        const float gamma = acosf(cg);
        float* o = out + i * (int64_t)ORC_K * din;
        for (int k = 0; k < ORC_K; ++k) {
            const int m = mk[k];
            const float s = ldexpf(inv_h0, -m);
            const float g = ldexpf(c->st.inv_mean_f, k) * s;
            float A[3], B[3], C[3], U0[3];
            for (int a = 0; a < 3; ++a) {
                A[a] = g * ex[a]; B[a] = g * ey[a]; C[a] = g * ez[a];
                float xs = xi[a] * s;
                U0[a] = xs - 0.5f;
            }
            for (int iz = 0; iz < nz; ++iz)
                for (int iy = 0; iy < n; ++iy)
                    for (int ix = 0; ix < n; ++ix) {
                        float px = hf * (float)ix, py = hf * (float)iy, pz = hf * (float)iz;
                        const float ox = -1.0f + px, oy = -1.0f + py, oz = -1.0f + pz;
                        float u[3];
                        for (int a = 0; a < 3; ++a)
                            u[a] = fmaf(oz, C[a], fmaf(oy, B[a], fmaf(ox, A[a], U0[a])));
                        o[k * din + (iz * n + iy) * n + ix] = trilinear32(lv[k], c->st.dims[m], u);
                    }
            o[k * din + S] = gamma;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Transport                                                                    */
/* ------------------------------------------------------------------------- */
double orc_hg(double g, double ct) {
    double den = 1.0 + g * g - 2.0 * g * ct;
    return (1.0 - g * g) / (4.0 * ORC_PI * den * sqrt(den));
}

/* ray/box clip against [0, ext] */
static int box_clip(const double ext[3], const double o[3], const double d[3], double* t0,
                    double* t1) {
    double tmin = 0.0, tmax = INFINITY;
    for (int a = 0; a < 3; ++a) {
        if (d[a] != 0.0) {
            double ta = (0.0 - o[a]) / d[a], tb = (ext[a] - o[a]) / d[a];
            if (ta > tb) { double t = ta; ta = tb; tb = t; }
            if (ta > tmin) tmin = ta;
            if (tb < tmax) tmax = tb;
        } else if (o[a] < 0.0 || o[a] > ext[a]) {
            return 0;
        }
    }
    *t0 = tmin; *t1 = tmax;
    return tmin < tmax;
}

/* Delta (Woodcock) tracking against the global majorant (Sec. 4.4): the path tracer's
 * bounces (which start inside the medium) use it, and it is the estimator the brick
 * tracking below must agree with in distribution.  Each tentative
 * collision draws one Philox block: xi0 for the exponential step, xi1 for the
 * real/null decision (xi1 * majorant < mu_t).  The extinction is the grid's times s (the
 * chopped medium's optically thinner volume, Sec. 3.1): the majorant s mu_max sets the
 * step, and the real/null ratio s mu_t / (s mu_max) is the unscaled one. */
int orc_delta_track_global_scaled(const orc_ctx* c, const double o[3], const double d[3], double s,
                                  uint64_t seed, uint32_t id0, uint32_t id1, uint32_t domain,
                                  uint32_t* ctr, double x[3], double* t_out) {
    double t0, t1;
    const double maj = (double)c->st.majorant;
    if (maj <= 0.0 || !box_clip(c->st.ext, o, d, &t0, &t1)) return 0;
    const double maj_s = s * maj;
    double t = t0;
    for (uint32_t n = 0; n < TRACK_CAP; ++n) {
        double xi[4];
        draw(seed, id0, id1, (*ctr)++, domain, xi);
        t -= log(1.0 - xi[0]) / maj_s;
        if (t >= t1) return 0;
        double p[3] = {o[0] + t * d[0], o[1] + t * d[1], o[2] + t * d[2]};
        double mu = orc_density(c, p);
        if (xi[1] * maj < mu) {
            x[0] = p[0]; x[1] = p[1]; x[2] = p[2];
            if (t_out) *t_out = t;
            return 1;
        }
    }
    return -1;
}

int orc_delta_track_global(const orc_ctx* c, const double o[3], const double d[3], uint64_t seed,
                           uint32_t id0, uint32_t id1, uint32_t domain, uint32_t* ctr, double x[3],
                           double* t_out) {
    return orc_delta_track_global_scaled(c, o, d, 1.0, seed, id0, id1, domain, ctr, x, t_out);
}

/* Ratio tracking (Novak et al. 2014, cited in Sec. 2) for the shadow-ray
 * transmittance; one Philox block per tentative collision (xi0). */
double orc_ratio_track_global(const orc_ctx* c, const double o[3], const double d[3], uint64_t seed,
                       uint32_t id0, uint32_t id1, uint32_t domain, uint32_t* ctr, int* capped) {
    double t0, t1;
    const double maj = (double)c->st.majorant;
    if (capped) *capped = 0;
    if (maj <= 0.0 || !box_clip(c->st.ext, o, d, &t0, &t1)) return 1.0;
    double t = t0, T = 1.0;
    for (uint32_t n = 0; n < TRACK_CAP; ++n) {
        double xi[4];
        draw(seed, id0, id1, (*ctr)++, domain, xi);
        t -= log(1.0 - xi[0]) / maj;
        if (t >= t1) return T;
        double p[3] = {o[0] + t * d[0], o[1] + t * d[1], o[2] + t * d[2]};
        T *= 1.0 - orc_density(c, p) / maj;
    }
    if (capped) *capped = 1;
    return T;
}

/* Walk over the bricks a ray crosses (3-D DDA): brick b[], the ray parameter at which it
 * leaves the current brick along each axis (tnext) and the parameter span of one brick
 * (tdelta).  Brick size bs = ORC_BRICK fine voxels in world units. */
typedef struct {
    int b[3], step[3];
    double tnext[3], tdelta[3];
} brick_walk;

static void walk_init(const orc_ctx* c, const double o[3], const double d[3], double t0, brick_walk* w) {
    const double bs = (double)ORC_BRICK * c->st.h0;
    for (int a = 0; a < 3; ++a) {
        const double p = o[a] + t0 * d[a];
        int b = (int)floor(p / bs);
        if (b < 0) b = 0;
        if (b > c->nb[a] - 1) b = c->nb[a] - 1;
        w->b[a] = b;
        if (d[a] > 0.0) {
            w->step[a] = 1;
            w->tnext[a] = ((double)(b + 1) * bs - o[a]) / d[a];
            w->tdelta[a] = bs / d[a];
        } else if (d[a] < 0.0) {
            w->step[a] = -1;
            w->tnext[a] = ((double)b * bs - o[a]) / d[a];
            w->tdelta[a] = -bs / d[a];
        } else {
            w->step[a] = 0;
            w->tnext[a] = INFINITY;
            w->tdelta[a] = INFINITY;
        }
    }
}

/* end of the current brick's segment (capped at t1) */
static double walk_exit(const brick_walk* w, double t1) {
    double t = w->tnext[0];
    if (w->tnext[1] < t) t = w->tnext[1];
    if (w->tnext[2] < t) t = w->tnext[2];
    return t < t1 ? t : t1;
}

/* steps into the next brick along the first axis whose boundary comes first; 0 when the
 * ray leaves the grid of bricks */
static int walk_step(const orc_ctx* c, brick_walk* w) {
    int a = 0;
    if (w->tnext[1] < w->tnext[a]) a = 1;
    if (w->tnext[2] < w->tnext[a]) a = 2;
    w->b[a] += w->step[a];
    w->tnext[a] += w->tdelta[a];
    return w->b[a] >= 0 && w->b[a] < c->nb[a];
}

static double walk_majorant(const orc_ctx* c, const brick_walk* w) {
    return (double)c->bmaj[((size_t)w->b[2] * c->nb[1] + w->b[1]) * c->nb[0] + w->b[0]];
}

/* Delta (Woodcock) tracking (Sec. 4.4) with a piecewise-constant majorant.  Each tentative
 * collision draws one Philox block: xi0 gives the optical depth tau = -log(1 - xi0) of
 * the majorant to travel, xi1 the real/null decision (xi1 * mu_b < mu_t).  The ray walks
 * the bricks spending tau at each brick's rate mu_b (mu_b = 0: nothing spent), so the
 * tentative collision falls where the majorant's optical depth from the previous one
 * reaches tau -- the exponential free flight of the piecewise-constant majorant. */
int orc_delta_track(const orc_ctx* c, const double o[3], const double d[3], uint64_t seed,
                    uint32_t id0, uint32_t id1, uint32_t domain, uint32_t* ctr, double x[3],
                    double* t_out) {
    double t0, t1;
    if (c->st.majorant <= 0.0f || !box_clip(c->st.ext, o, d, &t0, &t1)) return 0;
    brick_walk w;
    walk_init(c, o, d, t0, &w);
    double t = t0, tau = 0.0, xi[4] = {0, 0, 0, 0};
    int fresh = 1;                     /* a new block is needed for the next collision */
    for (uint32_t n = 0; n < TRACK_CAP; ++n) {
        const double te = walk_exit(&w, t1);
        const double mu_b = walk_majorant(c, &w);
        if (mu_b > 0.0) {
            if (fresh) {
                draw(seed, id0, id1, (*ctr)++, domain, xi);
                tau = -log(1.0 - xi[0]);
                fresh = 0;
            }
            const double seg = mu_b * (te - t);
            if (tau < seg) {
                t += tau / mu_b;
                fresh = 1;
                double p[3] = {o[0] + t * d[0], o[1] + t * d[1], o[2] + t * d[2]};
                if (xi[1] * mu_b < orc_density(c, p)) {
                    x[0] = p[0]; x[1] = p[1]; x[2] = p[2];
                    if (t_out) *t_out = t;
                    return 1;
                }
                continue;
            }
            tau -= seg;
        }
        if (te >= t1) return 0;
        t = te;
        if (!walk_step(c, &w)) return 0;
    }
    return -1;
}

/* Ratio tracking (Novak et al. 2014, cited in Sec. 2) for the shadow-ray transmittance,
 * over the same walk: one Philox block (xi0 -> optical depth) per tentative collision,
 * T *= 1 - mu_t / mu_b there.  The extinction is the grid's times s (the chopped medium's
 * thinner volume, Sec. 3.1): each brick's majorant rate is s mu_b, the ratio unchanged. */
double orc_ratio_track_scaled(const orc_ctx* c, const double o[3], const double d[3], double s,
                              uint64_t seed, uint32_t id0, uint32_t id1, uint32_t domain,
                              uint32_t* ctr, int* capped) {
    double t0, t1;
    if (capped) *capped = 0;
    if (c->st.majorant <= 0.0f || !box_clip(c->st.ext, o, d, &t0, &t1)) return 1.0;
    brick_walk w;
    walk_init(c, o, d, t0, &w);
    double t = t0, T = 1.0, tau = 0.0;
    int fresh = 1;
    for (uint32_t n = 0; n < TRACK_CAP; ++n) {
        const double te = walk_exit(&w, t1);
        const double mu_b = walk_majorant(c, &w);
        if (mu_b > 0.0) {
            if (fresh) {
                double xi[4];
                draw(seed, id0, id1, (*ctr)++, domain, xi);
                tau = -log(1.0 - xi[0]);
                fresh = 0;
            }
            const double mu_s = s * mu_b;
            const double seg = mu_s * (te - t);
            if (tau < seg) {
                t += tau / mu_s;
                fresh = 1;
                double p[3] = {o[0] + t * d[0], o[1] + t * d[1], o[2] + t * d[2]};
                T *= 1.0 - orc_density(c, p) / mu_b;
                continue;
            }
            tau -= seg;
        }
        if (te >= t1) return T;
        t = te;
        if (!walk_step(c, &w)) return T;
    }
    if (capped) *capped = 1;
    return T;
}

double orc_ratio_track(const orc_ctx* c, const double o[3], const double d[3], uint64_t seed,
                       uint32_t id0, uint32_t id1, uint32_t domain, uint32_t* ctr, int* capped) {
    return orc_ratio_track_scaled(c, o, d, 1.0, seed, id0, id1, domain, ctr, capped);
}

static void normalize3(double v[3]) {
    double l = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    v[0] /= l; v[1] /= l; v[2] /= l;
}

/* Henyey-Greenstein sampling in the tracing convention: the new tracing direction d'
 * has cos(d, d') distributed as p_HG (the phase function of the cosine between
 * propagation directions omega = -d and omega' = -d' is the same cosine). */
void orc_sample_hg(double g, const double d[3], double xi0, double xi1, double out[3]) {
    double ct;
    if (fabs(g) < 1e-3) ct = 1.0 - 2.0 * xi0;
    else {
        double s = (1.0 - g * g) / (1.0 - g + 2.0 * g * xi0);
        ct = (1.0 + g * g - s * s) / (2.0 * g);
    }
    if (ct > 1.0) ct = 1.0;
    if (ct < -1.0) ct = -1.0;
    double st = sqrt(fmax(0.0, 1.0 - ct * ct));
    double phi = 2.0 * ORC_PI * xi1;
    double b1[3], b2[3];
    duff_basis(d, b1, b2);
    for (int a = 0; a < 3; ++a) out[a] = st * cos(phi) * b1[a] + st * sin(phi) * b2[a] + ct * d[a];
    normalize3(out);
}

/* ------------------------------------------------------------------------- */
/* Lorenz-Mie phase function of cloud droplets (Sec. 3.1).                      */
/* The paper's tables and chopping live in its supplement, which is not        */
/* available; here the phase function is computed from the series of Bohren &  */
/* Huffman (1983, App. A) for water droplets (m = 1.333, no absorption) at      */
/* 0.55 um, averaged over Deirmendjian's cumulus C.1 size distribution          */
/* n(r) ~ r^6 exp(-1.5 r) (r in um, mode 4 um), and tabulated as its mean over  */
/* ORC_LM_BINS bins of 0.1 degree of scattering angle (by solid angle): the     */
/* phase function used is that piecewise-constant one, which is sampled        */
/* exactly (bin by its cumulative probability, then cos theta uniform in it).   */
/* ------------------------------------------------------------------------- */
int orc_mie_single(double x, double m_re, double m_im, const double* mu, int nmu, double* s11, double* qext,
                   double* qsca) {
    if (!(x > 0.0) || nmu < 0) return -1;
    const double complex m = m_re + I * m_im, y = m * x;
    const int nstop = (int)(x + 4.0 * cbrt(x) + 2.0);
    const int nmx = (int)fmax((double)nstop, cabs(y)) + 16;
    double complex* D = (double complex*)calloc((size_t)nmx + 1, sizeof(double complex));
    double complex* S1 = (double complex*)calloc((size_t)(nmu > 0 ? nmu : 1), sizeof(double complex));
    double complex* S2 = (double complex*)calloc((size_t)(nmu > 0 ? nmu : 1), sizeof(double complex));
    double* pim1 = (double*)calloc((size_t)(nmu > 0 ? nmu : 1), sizeof(double));   /* pi_{n-1} */
    double* pin = (double*)malloc(sizeof(double) * (size_t)(nmu > 0 ? nmu : 1));    /* pi_n */
    for (int k = 0; k < nmu; ++k) pin[k] = 1.0;
    /* logarithmic derivative D_n(y) by downward recurrence from D_nmx = 0 */
    for (int n = nmx; n > 0; --n) D[n - 1] = (double)n / y - 1.0 / (D[n] + (double)n / y);
    /* Riccati-Bessel functions psi_n, chi_n by upward recurrence, xi_n = psi_n - i chi_n */
    double psi0 = cos(x), psi1 = sin(x), chi0 = -sin(x), chi1 = cos(x);
    double complex xi1 = psi1 - I * chi1;
    double qe = 0.0, qs = 0.0;
    for (int n = 1; n <= nstop; ++n) {
        const double dn = (double)n;
        const double psi = (2.0 * dn - 1.0) / x * psi1 - psi0;
        const double chi = (2.0 * dn - 1.0) / x * chi1 - chi0;
        const double complex xi = psi - I * chi;
        const double complex da = D[n] / m + dn / x, db = m * D[n] + dn / x;
        const double complex an = (da * psi - psi1) / (da * xi - xi1);
        const double complex bn = (db * psi - psi1) / (db * xi - xi1);
        qs += (2.0 * dn + 1.0) * (creal(an) * creal(an) + cimag(an) * cimag(an) + creal(bn) * creal(bn) +
                                  cimag(bn) * cimag(bn));
        qe += (2.0 * dn + 1.0) * creal(an + bn);
        const double fn = (2.0 * dn + 1.0) / (dn * (dn + 1.0));
        for (int k = 0; k < nmu; ++k) {
            const double pi = pin[k], tau = dn * mu[k] * pi - (dn + 1.0) * pim1[k];
            S1[k] += fn * (an * pi + bn * tau);
            S2[k] += fn * (an * tau + bn * pi);
            /* pi_{n+1} = ((2n+1)/n) mu pi_n - ((n+1)/n) pi_{n-1} */
            const double next = (2.0 * dn + 1.0) / dn * mu[k] * pi - (dn + 1.0) / dn * pim1[k];
            pim1[k] = pi;
            pin[k] = next;
        }
        psi0 = psi1; psi1 = psi;
        chi0 = chi1; chi1 = chi;
        xi1 = psi1 - I * chi1;
    }
    for (int k = 0; k < nmu; ++k) {
        const double a1 = cabs(S1[k]), a2 = cabs(S2[k]);
        s11[k] = 0.5 * (a1 * a1 + a2 * a2);
    }
    if (qext) *qext = 2.0 / (x * x) * qe;
    if (qsca) *qsca = 2.0 / (x * x) * qs;
    free(D); free(S1); free(S2); free(pim1); free(pin);
    return 0;
}

static double lm_p[ORC_LM_BINS], lm_cdf[ORC_LM_BINS + 1], lm_cos[ORC_LM_BINS + 1];
static int lm_ready = 0;

static void lm_build(void) {
    const double dth = ORC_PI / ORC_LM_BINS;
    const int nf = 2 * ORC_LM_BINS + 1;                  /* bin edges and midpoints */
    double* mu = (double*)malloc(sizeof(double) * nf);
    double* acc = (double*)calloc((size_t)nf, sizeof(double));
    double* s11 = (double*)malloc(sizeof(double) * nf);
    for (int f = 0; f < nf; ++f) mu[f] = cos(0.5 * dth * f);
    const double lambda = 0.55, k = 2.0 * ORC_PI / lambda;
    for (int ir = 1; ir <= 160; ++ir) {                 /* r = 0.1 .. 16 um */
        const double r = 0.1 * ir, w = pow(r, 6.0) * exp(-1.5 * r);
        orc_mie_single(k * r, 1.333, 0.0, mu, nf, s11, NULL, NULL);
        for (int f = 0; f < nf; ++f) acc[f] += w * s11[f];
    }
    double total = 0.0;
    for (int j = 0; j < ORC_LM_BINS; ++j) {
        const double t0 = dth * j, tm = t0 + 0.5 * dth, t1 = t0 + dth;
        /* Simpson over the bin of i(theta) sin(theta) d theta, per unit solid angle */
        const double integ = (acc[2 * j] * sin(t0) + 4.0 * acc[2 * j + 1] * sin(tm) + acc[2 * j + 2] * sin(t1)) *
                             dth / 6.0;
        const double dcos = cos(t0) - cos(t1);
        lm_p[j] = integ / dcos;
        total += 2.0 * ORC_PI * integ;
    }
    lm_cdf[0] = 0.0;
    for (int j = 0; j < ORC_LM_BINS; ++j) {
        lm_p[j] /= total;
        lm_cos[j] = cos(dth * j);
        lm_cdf[j + 1] = lm_cdf[j] + lm_p[j] * 2.0 * ORC_PI * (cos(dth * j) - cos(dth * (j + 1)));
    }
    lm_cos[ORC_LM_BINS] = -1.0;
    lm_cdf[ORC_LM_BINS] = 1.0;
    free(mu); free(acc); free(s11);
    lm_ready = 1;
}

int orc_lm_table(double* p, double* cdf, double* cos_edges, int n) {
    if (n != ORC_LM_BINS) return -1;
    if (!lm_ready) lm_build();
    for (int j = 0; j < n; ++j) { if (p) p[j] = lm_p[j]; }
    for (int j = 0; j <= n; ++j) { if (cdf) cdf[j] = lm_cdf[j]; if (cos_edges) cos_edges[j] = lm_cos[j]; }
    return 0;
}

/* The chopped table (Sec. 3.1, after Bouthors et al. 2008): the first `chop_bins` bins (the
 * diffraction peak) hold the fraction f of the scattered light; they are removed and the
 * rest renormalised by 1 / (1 - f).  Light scattered into the peak is treated as not
 * scattered at all, so the scattering coefficient drops to (1 - f) mu_s while absorption
 * stays: extinction (1 - f albedo) mu_t, albedo (1 - f) albedo / (1 - f albedo). */
static void chop_build(orc_ctx* c, int chop_bins) {
    const double dth = ORC_PI / ORC_LM_BINS;
    if (!c->lmc_p) c->lmc_p = (double*)malloc(sizeof(double) * ORC_LM_BINS);
    if (!c->lmc_cdf) c->lmc_cdf = (double*)malloc(sizeof(double) * (ORC_LM_BINS + 1));
    double f = 0.0;
    for (int j = 0; j < chop_bins; ++j) f += lm_p[j] * 2.0 * ORC_PI * (cos(dth * j) - cos(dth * (j + 1)));
    c->lmc_cdf[0] = 0.0;
    for (int j = 0; j < ORC_LM_BINS; ++j) {
        c->lmc_p[j] = j < chop_bins ? 0.0 : lm_p[j] / (1.0 - f);
        c->lmc_cdf[j + 1] = c->lmc_cdf[j] + c->lmc_p[j] * 2.0 * ORC_PI * (cos(dth * j) - cos(dth * (j + 1)));
    }
    c->lmc_cdf[ORC_LM_BINS] = 1.0;
    c->chop_f = f;
    c->dscale = 1.0 - f * c->albedo;
    c->albedo_c = c->albedo * (1.0 - f) / (1.0 - f * c->albedo);
}

int orc_set_phase(orc_ctx* c, int kind, int chop_bins) {
    if (!c || kind < 0 || kind > 2 || chop_bins < 0 || chop_bins >= ORC_LM_BINS) return -1;
    if (kind > 0 && !lm_ready) lm_build();
    c->phase_lm = kind;
    c->chop_f = 0.0;
    c->dscale = 1.0;
    c->albedo_c = c->albedo;
    if (kind == 2) chop_build(c, chop_bins);
    return 0;
}

void orc_set_phase_lm(orc_ctx* c, int on) {
    orc_set_phase(c, on ? 1 : 0, 0);
}

int orc_chop_params(const orc_ctx* c, double* f, double* dscale, double* albedo_c) {
    if (!c) return -1;
    if (f) *f = c->chop_f;
    if (dscale) *dscale = c->dscale;
    if (albedo_c) *albedo_c = c->albedo_c;
    return 0;
}

int orc_lm_chopped_table(const orc_ctx* c, double* p, double* cdf, int n) {
    if (!c || c->phase_lm != 2 || n != ORC_LM_BINS) return -1;
    for (int j = 0; j < n; ++j) { if (p) p[j] = c->lmc_p[j]; }
    for (int j = 0; j <= n; ++j) { if (cdf) cdf[j] = c->lmc_cdf[j]; }
    return 0;
}

/* phase function of the volume at cos theta between propagation directions, at the first
 * bounce of a path (the camera's or a record's vertex) or after it */
static double phase_eval(const orc_ctx* c, int first, double ct) {
    if (!c->phase_lm) return orc_hg(c->g, ct);
    const double* tp = (c->phase_lm == 2 && !first) ? c->lmc_p : lm_p;
    if (ct > 1.0) ct = 1.0;
    if (ct < -1.0) ct = -1.0;
    int j = (int)(acos(ct) / (ORC_PI / ORC_LM_BINS));
    if (j > ORC_LM_BINS - 1) j = ORC_LM_BINS - 1;
    return tp[j];
}

/* new tracing direction: HG, or the tabulated Lorenz-Mie function (bin by its cumulative
 * probability xi0, cos theta uniform inside the bin, azimuth 2 pi xi1) */
static void phase_sample(const orc_ctx* c, int first, const double d[3], double xi0, double xi1,
                         double out[3]) {
    if (!c->phase_lm) { orc_sample_hg(c->g, d, xi0, xi1, out); return; }
    const double* cdf = (c->phase_lm == 2 && !first) ? c->lmc_cdf : lm_cdf;
    int lo = 0, hi = ORC_LM_BINS;
    while (hi - lo > 1) {
        const int mid = (lo + hi) / 2;
        if (cdf[mid] <= xi0) lo = mid; else hi = mid;
    }
    const double f = (xi0 - cdf[lo]) / (cdf[lo + 1] - cdf[lo]);
    double ct = lm_cos[lo] - f * (lm_cos[lo] - lm_cos[lo + 1]);
    if (ct > 1.0) ct = 1.0;
    if (ct < -1.0) ct = -1.0;
    const double st = sqrt(fmax(0.0, 1.0 - ct * ct)), phi = 2.0 * ORC_PI * xi1;
    double b1[3], b2[3];
    duff_basis(d, b1, b2);
    for (int a = 0; a < 3; ++a) out[a] = st * cos(phi) * b1[a] + st * sin(phi) * b2[a] + ct * d[a];
    normalize3(out);
}

/* Direct in-scattering by next-event estimation towards the directional light
 * (Sec. 4.4; MIS with phase sampling adds nothing for a delta light).  `first`: the vertex
 * is a path's first bounce, which scatters with the full phase function; the light reaches
 * every vertex through the (chopped medium's) extinction dscale mu_t. */
static double nee(const orc_ctx* c, int first, const double x[3], const double d[3], const double wl[3],
                  double E, uint64_t seed, uint32_t id0, uint32_t id1, uint32_t dom,
                  uint32_t* ctr) {
    double ct = d[0] * wl[0] + d[1] * wl[1] + d[2] * wl[2];
    double T = orc_ratio_track_scaled(c, x, wl, c->dscale, seed, id0, id1, dom, ctr, NULL);
    return E * phase_eval(c, first, ct) * T;
}

/* One path estimate of the indirect in-scattered radiance L_i at vertex x reached with
 * tracing direction d (Sec. 4, L_i excludes the uncollided light): sample a direction
 * from the phase function, find the next collision by delta tracking, survive it
 * with probability albedo, add NEE there, repeat. */
static double path_Li(const orc_ctx* c, const double x0[3], const double d0[3],
                      const double wl[3], double E, uint64_t seed, uint32_t id0,
                      uint32_t id1, uint32_t dom, int max_bounces, int* capped) {
    double x[3] = {x0[0], x0[1], x0[2]}, d[3] = {d0[0], d0[1], d0[2]};
    uint32_t ctr = 0;
    double L = 0.0;
    const int cap = (max_bounces > 0 && max_bounces < BOUNCE_CAP) ? max_bounces : BOUNCE_CAP;
    for (int b = 0; b < cap; ++b) {
        double xi[4];
        draw(seed, id0, id1, ctr++, dom, xi);
        double nd[3];
        /* x0 is the path's first bounce (full phase function); later vertices scatter
         * with the chopped one where the volume is set so (Sec. 3.1) */
        phase_sample(c, b == 0, d, xi[0], xi[1], nd);
        double nx[3];
        /* a bounce starts inside the medium, where bricks hold nearly the global majorant:
         * track it against the global one (crossing bricks there only costs) */
        int hit = orc_delta_track_global_scaled(c, x, nd, c->dscale, seed, id0, id1, dom, &ctr, nx, NULL);
        if (hit < 0) { if (capped) *capped = 1; return L; }
        if (hit == 0) return L;
        draw(seed, id0, id1, ctr++, dom, xi);
        if (!(xi[0] < c->albedo_c)) return L;    /* absorbed */
        L += nee(c, 0, nx, nd, wl, E, seed, id0, id1, dom, &ctr);
        x[0] = nx[0]; x[1] = nx[1]; x[2] = nx[2];
        d[0] = nd[0]; d[1] = nd[1]; d[2] = nd[2];
    }
    if (cap == BOUNCE_CAP && capped) *capped = 1;
    return L;
}

int orc_primary(const orc_ctx* c, const orc_camera* cam, int64_t pixel, int sample,
                double x[3], double d[3], double* Ld) {
    const int W = cam->width, H = cam->height;
    const int px = (int)(pixel % W), py = (int)(pixel / W);
    double xi[4];
    draw(cam->seed, (uint32_t)pixel, (uint32_t)sample, 0, DOM_CAMERA, xi);
    const double aspect = (double)W / (double)H;
    double sx = (2.0 * ((double)px + xi[0]) / (double)W - 1.0) * cam->tan_half_fov_y * aspect;
    double sy = (1.0 - 2.0 * ((double)py + xi[1]) / (double)H) * cam->tan_half_fov_y;
    for (int a = 0; a < 3; ++a) d[a] = cam->cam_fwd[a] + sx * cam->cam_right[a] + sy * cam->cam_up[a];
    normalize3(d);
    uint32_t ctr = 0;
    int hit = orc_delta_track(c, cam->cam_pos, d, cam->seed, (uint32_t)pixel, (uint32_t)sample,
                              DOM_PRIMARY, &ctr, x, NULL);
    if (hit != 1) { *Ld = 0.0; return hit; }
    uint32_t sc = 0;
    *Ld = nee(c, 1, x, d, cam->light_dir, cam->light_E, cam->seed, (uint32_t)pixel,
              (uint32_t)sample, DOM_SHADOW, &sc);
    return 1;
}

int orc_render_pixels(orc_ctx* c, const orc_camera* cam, const double* params, int mode,
                      const int64_t* pixels, int64_t npix, double* out, int nthreads) {
    if (!c || !cam) return -1;
    const orc_net net = {ORC_K, ORC_DIN, ORC_H, 3};
    if (mode == 0 && params) get_mip64(c, c->st.mip_of_level[0]); /* warm (thread-safe anyway) */
    if (nthreads <= 0) nthreads = 1;
    int err = 0;
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads)
    for (int64_t i = 0; i < npix; ++i) {
        double acc = 0.0;
        for (int s = 0; s < cam->spp; ++s) {
            double x[3], d[3], Ld;
            int hit = orc_primary(c, cam, pixels[i], s, x, d, &Ld);
            if (hit < 0) { err = 1; continue; }
            if (hit == 0) continue;
            double Li = 0.0;
            if (mode == 0 && params) {
                double z[ORC_K * ORC_DIN];
                orc_descriptor_f64(c, x, d, cam->light_dir, 1, z);
                orc_mlp_forward(&net, params, z, 1, &Li);
                Li *= cam->light_E;   /* the network predicts for unit irradiance */
            } else if (mode == 1) {
                int capped = 0;
                Li = path_Li(c, x, d, cam->light_dir, cam->light_E, cam->seed,
                             (uint32_t)pixels[i], (uint32_t)s, DOM_PATH, 0, &capped);
                if (capped) err = 1;
            }
            acc += c->albedo * (Ld + Li);
        }
        out[i] = acc / (double)cam->spp;
    }
    return err ? -2 : 0;
}

int orc_render(orc_ctx* c, const orc_camera* cam, const double* params, int mode,
               double* image, int nthreads) {
    const int64_t n = (int64_t)cam->width * cam->height;
    int64_t* pix = (int64_t*)malloc(sizeof(int64_t) * n);
    for (int64_t i = 0; i < n; ++i) pix[i] = i;
    int r = orc_render_pixels(c, cam, params, mode, pix, n, image, nthreads);
    free(pix);
    return r;
}

/* ------------------------------------------------------------------------- */
/* RPNN (Sec. 4.3).  Parameter order (flat, row-major [out][in] matrices):       */
/*   for k = 1..K:  V^k [H][din], W1^k [H][H] (absent for k = 1, o^0 = 0 makes it   */
/*                  inert, footnote 1), b1^k [H], W2^k [H][H], b2^k [H]            */
/*   then ntail standard layers: [H][H],[H] ... and the last one [1][H], [1].      */
/* Block:  F1 = relu(V z + W1 o + b1);  F2 = W2 F1 + b2;  o' = relu(F2 + o).        */
/* Standard layer: o' = relu(W o + b); the final layer's output is g (Sec. 4.3).    */
/* ------------------------------------------------------------------------- */
int64_t orc_net_param_count(const orc_net* n) {
    int64_t c = 0;
    for (int k = 0; k < n->K; ++k) {
        c += (int64_t)n->H * n->din;
        if (k > 0) c += (int64_t)n->H * n->H;
        c += n->H + (int64_t)n->H * n->H + n->H;
    }
    for (int t = 0; t < n->ntail; ++t) {
        int out = (t == n->ntail - 1) ? 1 : n->H;
        c += (int64_t)out * n->H + out;
    }
    return c;
}

typedef struct {
    const double *V, *W1, *b1, *W2, *b2;
} blk_ptrs;

static void net_layout(const orc_net* n, const double* p, blk_ptrs* blk, const double** tw,
                       const double** tb) {
    for (int k = 0; k < n->K; ++k) {
        blk[k].V = p; p += (int64_t)n->H * n->din;
        if (k > 0) { blk[k].W1 = p; p += (int64_t)n->H * n->H; } else blk[k].W1 = NULL;
        blk[k].b1 = p; p += n->H;
        blk[k].W2 = p; p += (int64_t)n->H * n->H;
        blk[k].b2 = p; p += n->H;
    }
    for (int t = 0; t < n->ntail; ++t) {
        int out = (t == n->ntail - 1) ? 1 : n->H;
        tw[t] = p; p += (int64_t)out * n->H;
        tb[t] = p; p += out;
    }
}

/* y[r] = sum_c M[r][c] x[c] (+ y if acc) */
static void matvec(const double* M, const double* x, int rows, int cols, double* y, int acc) {
    for (int r = 0; r < rows; ++r) {
        double s = 0.0;
        for (int c = 0; c < cols; ++c) s += M[(int64_t)r * cols + c] * x[c];
        y[r] = acc ? y[r] + s : s;
    }
}

static double relu(double a) { return a > 0.0 ? a : 0.0; }

/* forward for one query; saves (per block) a1 = pre-ReLU of F1, F1, pre = F2 + o_prev,
 * o after each block, and the tail pre-activations, when `save` is given. */
typedef struct {
    double* o_in;   /* [K][H] o^{k-1} */
    double* a1;     /* [K][H] */
    double* f1;     /* [K][H] */
    double* pre2;   /* [K][H] */
    double* t_in;   /* [ntail][H] */
    double* t_pre;  /* [ntail][H] */
} fwd_save;

static double forward_one(const orc_net* n, const blk_ptrs* blk, const double** tw,
                          const double** tb, const double* z, fwd_save* sv) {
    const int H = n->H;
    double* o = (double*)calloc(H, sizeof(double));
    double* a1 = (double*)malloc(sizeof(double) * H);
    double* f1 = (double*)malloc(sizeof(double) * H);
    double* a2 = (double*)malloc(sizeof(double) * H);
    for (int k = 0; k < n->K; ++k) {
        const double* zk = z + (int64_t)k * n->din;
        if (sv) memcpy(sv->o_in + (int64_t)k * H, o, sizeof(double) * H);
        matvec(blk[k].V, zk, H, n->din, a1, 0);
        if (blk[k].W1) matvec(blk[k].W1, o, H, H, a1, 1);
        for (int r = 0; r < H; ++r) { a1[r] += blk[k].b1[r]; f1[r] = relu(a1[r]); }
        matvec(blk[k].W2, f1, H, H, a2, 0);
        for (int r = 0; r < H; ++r) {
            double pre = a2[r] + blk[k].b2[r] + o[r];
            if (sv) sv->pre2[(int64_t)k * H + r] = pre;
            o[r] = relu(pre);
        }
        if (sv) {
            memcpy(sv->a1 + (int64_t)k * H, a1, sizeof(double) * H);
            memcpy(sv->f1 + (int64_t)k * H, f1, sizeof(double) * H);
        }
    }
    double g = 0.0;
    for (int t = 0; t < n->ntail; ++t) {
        int out = (t == n->ntail - 1) ? 1 : H;
        if (sv) memcpy(sv->t_in + (int64_t)t * H, o, sizeof(double) * H);
        matvec(tw[t], o, out, H, a2, 0);
        for (int r = 0; r < out; ++r) {
            double pre = a2[r] + tb[t][r];
            if (sv) sv->t_pre[(int64_t)t * H + r] = pre;
            a2[r] = relu(pre);
        }
        if (out == 1) g = a2[0];
        else memcpy(o, a2, sizeof(double) * H);
    }
    free(o); free(a1); free(f1); free(a2);
    return g;
}

int orc_mlp_forward(const orc_net* n, const double* params, const double* z, int64_t q,
                    double* g) {
    if (!n || !params || !z || !g || n->ntail < 1) return -1;
    blk_ptrs blk[64];
    const double* tw[16];
    const double* tb[16];
    if (n->K > 64 || n->ntail > 16) return -1;
    net_layout(n, params, blk, tw, tb);
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t i = 0; i < q; ++i)
        g[i] = forward_one(n, blk, tw, tb, z + i * (int64_t)n->K * n->din, NULL);
    return 0;
}

/* Chain rule through the network of one query, accumulating into dparams (serial over
 * queries so the accumulation order is fixed). */
int orc_mlp_backward(const orc_net* n, const double* params, const double* z, int64_t q,
                     const double* dg, double* dparams) {
    if (!n || !params || !z || !dg || !dparams || n->ntail < 1) return -1;
    if (n->K > 64 || n->ntail > 16) return -1;
    const int H = n->H, K = n->K, T = n->ntail;
    blk_ptrs blk[64], dblk[64];
    const double* tw[16];
    const double* tb[16];
    const double* dtw[16];
    const double* dtb[16];
    net_layout(n, params, blk, tw, tb);
    net_layout(n, dparams, dblk, dtw, dtb);
    fwd_save sv;
    sv.o_in = (double*)malloc(sizeof(double) * K * H);
    sv.a1 = (double*)malloc(sizeof(double) * K * H);
    sv.f1 = (double*)malloc(sizeof(double) * K * H);
    sv.pre2 = (double*)malloc(sizeof(double) * K * H);
    sv.t_in = (double*)malloc(sizeof(double) * T * H);
    sv.t_pre = (double*)malloc(sizeof(double) * T * H);
    double* dout = (double*)malloc(sizeof(double) * H);
    double* da = (double*)malloc(sizeof(double) * H);
    double* dprev = (double*)malloc(sizeof(double) * H);
    double* df1 = (double*)malloc(sizeof(double) * H);
    for (int64_t i = 0; i < q; ++i) {
        const double* zi = z + i * (int64_t)K * n->din;
        forward_one(n, blk, tw, tb, zi, &sv);
        /* tail, last layer first */
        dout[0] = dg[i];
        for (int t = T - 1; t >= 0; --t) {
            int out = (t == T - 1) ? 1 : H;
            double* dW = (double*)dtw[t];
            double* db = (double*)dtb[t];
            const double* xin = sv.t_in + (int64_t)t * H;
            for (int r = 0; r < out; ++r) {
                da[r] = sv.t_pre[(int64_t)t * H + r] > 0.0 ? dout[r] : 0.0;
                db[r] += da[r];
                for (int c2 = 0; c2 < H; ++c2) dW[(int64_t)r * H + c2] += da[r] * xin[c2];
            }
            for (int c2 = 0; c2 < H; ++c2) {
                double s = 0.0;
                for (int r = 0; r < out; ++r) s += tw[t][(int64_t)r * H + c2] * da[r];
                dprev[c2] = s;
            }
            memcpy(dout, dprev, sizeof(double) * H);
        }
        /* blocks, last first; dout = dl/do^k */
        for (int k = K - 1; k >= 0; --k) {
            const double* zk = zi + (int64_t)k * n->din;
            const double* oin = sv.o_in + (int64_t)k * H;
            const double* f1 = sv.f1 + (int64_t)k * H;
            double* dV = (double*)dblk[k].V;
            double* dW1 = (double*)dblk[k].W1;
            double* db1 = (double*)dblk[k].b1;
            double* dW2 = (double*)dblk[k].W2;
            double* db2 = (double*)dblk[k].b2;
            /* o^k = relu(pre2): dpre = dout * [pre2 > 0] */
            for (int r = 0; r < H; ++r) da[r] = sv.pre2[(int64_t)k * H + r] > 0.0 ? dout[r] : 0.0;
            /* F2 = W2 F1 + b2 */
            for (int r = 0; r < H; ++r) {
                db2[r] += da[r];
                for (int c2 = 0; c2 < H; ++c2) dW2[(int64_t)r * H + c2] += da[r] * f1[c2];
            }
            for (int c2 = 0; c2 < H; ++c2) {
                double s = 0.0;
                for (int r = 0; r < H; ++r) s += blk[k].W2[(int64_t)r * H + c2] * da[r];
                df1[c2] = sv.a1[(int64_t)k * H + c2] > 0.0 ? s : 0.0;   /* through F1's ReLU */
            }
            /* residual: d o^{k-1} gets dpre directly */
            for (int r = 0; r < H; ++r) dprev[r] = da[r];
            /* a1 = V z + W1 o^{k-1} + b1 */
            for (int r = 0; r < H; ++r) {
                db1[r] += df1[r];
                for (int c2 = 0; c2 < n->din; ++c2) dV[(int64_t)r * n->din + c2] += df1[r] * zk[c2];
                if (dW1)
                    for (int c2 = 0; c2 < H; ++c2) dW1[(int64_t)r * H + c2] += df1[r] * oin[c2];
            }
            if (blk[k].W1)
                for (int c2 = 0; c2 < H; ++c2) {
                    double s = 0.0;
                    for (int r = 0; r < H; ++r) s += blk[k].W1[(int64_t)r * H + c2] * df1[r];
                    dprev[c2] += s;
                }
            memcpy(dout, dprev, sizeof(double) * H);
        }
    }
    free(sv.o_in); free(sv.a1); free(sv.f1); free(sv.pre2); free(sv.t_in); free(sv.t_pre);
    free(dout); free(da); free(dprev); free(df1);
    return 0;
}

/* Sec. 5.2: l = mean_i (log(1 + g_i) - log(1 + L_i))^2 (natural log) */
double orc_logmse_loss(const double* g, const double* target, int64_t b, double* dg) {
    double s = 0.0;
    for (int64_t i = 0; i < b; ++i) {
        double r = log1p(g[i]) - log1p(target[i]);
        s += r * r;
        if (dg) dg[i] = 2.0 * r / ((1.0 + g[i]) * (double)b);
    }
    return s / (double)b;
}

/* Adam (Kingma & Ba 2014, Algorithm 1), bias-corrected */
void orc_adam(double* p, double* m, double* v, const double* grad, int64_t n, int64_t t,
              double lr, double b1, double b2, double eps) {
    const double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
    for (int64_t i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * grad[i];
        v[i] = b2 * v[i] + (1.0 - b2) * grad[i] * grad[i];
        double mh = m[i] / c1, vh = v[i] / c2;
        p[i] -= lr * mh / (sqrt(vh) + eps);
    }
}

/* ------------------------------------------------------------------------- */
/* Training records (Sec. 5.1)                                                  */
/* ------------------------------------------------------------------------- */
int orc_estimate_Li(const orc_ctx* c, uint64_t seed, uint32_t rec, const double x[3],
                    const double d[3], const double wl[3], int npaths, int max_bounces,
                    double* mean, double* var) {
    double mu = 0.0, m2 = 0.0;
    int capped = 0;
    for (int j = 0; j < npaths; ++j) {
        double L = path_Li(c, x, d, wl, 1.0, seed, rec, (uint32_t)j, DOM_LABEL, max_bounces,
                           &capped);
        double delta = L - mu;
        mu += delta / (double)(j + 1);
        m2 += delta * (L - mu);
    }
    *mean = mu;
    *var = npaths > 1 ? m2 / (double)(npaths - 1) : 0.0;
    return capped ? -1 : 0;
}

/* Record sampling: direction uniform on the sphere; ray origin uniform (by area) on the
 * disk of the bounding sphere's cross-section perpendicular to the direction, moved one
 * diameter back; free flight by delta tracking; retry on escape.  Light direction
 * uniform on the sphere.  L_i by path tracing with NEE until the 95% interval
 * half-width 1.96 s / sqrt(n) is within rel_ci of the running mean (Sec. 5.1). */
int orc_gen_record(const orc_ctx* c, uint64_t seed, int64_t rec, double rel_ci, int n_min,
                   int n_max, double x[3], double d[3], double wl[3], double* label,
                   int64_t* npaths, double* half_width) {
    const uint32_t r = (uint32_t)rec;
    const double C[3] = {0.5 * c->st.ext[0], 0.5 * c->st.ext[1], 0.5 * c->st.ext[2]};
    const double R = 0.5 * sqrt(c->st.ext[0] * c->st.ext[0] + c->st.ext[1] * c->st.ext[1] +
                                c->st.ext[2] * c->st.ext[2]);
    int found = 0;
    for (uint32_t a = 0; a < RECORD_ATTEMPTS && !found; ++a) {
        double xi[4];
        draw(seed, r, a, 0, DOM_RECORD, xi);
        double cz = 1.0 - 2.0 * xi[0], phi = 2.0 * ORC_PI * xi[1];
        double sz = sqrt(fmax(0.0, 1.0 - cz * cz));
        d[0] = sz * cos(phi); d[1] = sz * sin(phi); d[2] = cz;
        double b1[3], b2[3];
        duff_basis(d, b1, b2);
        double rr = R * sqrt(xi[2]), ph2 = 2.0 * ORC_PI * xi[3];
        double o[3];
        for (int k = 0; k < 3; ++k)
            o[k] = C[k] + rr * (cos(ph2) * b1[k] + sin(ph2) * b2[k]) - 2.0 * R * d[k];
        uint32_t ctr = 0;
        int hit = orc_delta_track(c, o, d, seed, r, a, DOM_RECTRACK, &ctr, x, NULL);
        if (hit == 1) found = 1;
    }
    if (!found) return -1;
    {
        double xi[4];
        draw(seed, r, 0, 0, DOM_LIGHT, xi);
        double cz = 1.0 - 2.0 * xi[0], phi = 2.0 * ORC_PI * xi[1];
        double sz = sqrt(fmax(0.0, 1.0 - cz * cz));
        wl[0] = sz * cos(phi); wl[1] = sz * sin(phi); wl[2] = cz;
    }
    double mu = 0.0, m2 = 0.0;
    int capped = 0;
    int64_t j = 0;
    double hw = INFINITY;
    for (j = 0; j < n_max; ++j) {
        double L = path_Li(c, x, d, wl, 1.0, seed, r, (uint32_t)j, DOM_LABEL, 0, &capped);
        double delta = L - mu;
        mu += delta / (double)(j + 1);
        m2 += delta * (L - mu);
        int64_t nn = j + 1;
        if (nn >= n_min && nn > 1) {
            hw = 1.96 * sqrt(m2 / (double)(nn - 1) / (double)nn);
            if (mu > 0.0 && hw <= rel_ci * mu) { ++j; break; }
        }
    }
    *label = mu;
    *npaths = j;
    *half_width = hw;
    return capped ? -1 : 0;
}
