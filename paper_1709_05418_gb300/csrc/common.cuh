// common.cuh -- device helpers of the RPNN hot path (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "internal.h"

namespace rpnn {

// Random-number streams: Philox4x32-10 counter (id0, id1, step, domain), key = seed.
enum : uint32_t {
    kDomCamera = 1, kDomPrimary = 2, kDomShadow = 3, kDomPath = 4,
    kDomRecord = 5, kDomRecTrack = 6, kDomLight = 7, kDomLabel = 8
};
constexpr int kBounceCap = 100000;         // collisions per path
constexpr int kRecordAttempts = 4096;
constexpr float kPi = 3.14159265358979323846f;

// Philox4x32-10 (Salmon et al., SC'11).
__device__ __forceinline__ uint4 philox(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k.x += 0x9E3779B9u; k.y += 0xBB67AE85u; }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

__device__ __forceinline__ float u01(uint32_t r) { return (float)(r >> 8) * 0x1p-24f; }

struct Rng {
    uint2 key;
    uint32_t id0, id1, dom;
    __device__ __forceinline__ float4 draw(uint32_t step) const {
        uint4 r = philox(make_uint4(id0, id1, step, dom), key);
        return make_float4(u01(r.x), u01(r.y), u01(r.z), u01(r.w));
    }
};
__device__ __forceinline__ Rng make_rng(uint64_t seed, uint32_t id0, uint32_t id1, uint32_t dom) {
    Rng r;
    r.key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    r.id0 = id0; r.id1 = id1; r.dom = dom;
    return r;
}

__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return f3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 normalize3(float3 a) {
    float l = sqrtf(dot3(a, a));
    return f3(a.x / l, a.y / l, a.z / l);
}

// Orthonormal basis around unit n (Duff et al., "Building an Orthonormal Basis,
// Revisited", JCGT 2017).
__device__ __forceinline__ void duff_basis(float3 n, float3& b1, float3& b2) {
    const float sign = copysignf(1.0f, n.z);
    const float a = -1.0f / (sign + n.z);
    const float b = n.x * n.y * a;
    b1 = f3(1.0f + sign * n.x * n.x * a, sign * b, -sign * n.x);
    b2 = f3(b, sign + n.y * n.y * a, -n.y);
}

// Henyey-Greenstein phase function of the cosine between propagation directions.
__device__ __forceinline__ float hg_eval(float g, float ct) {
    const float den = 1.0f + g * g - 2.0f * g * ct;
    return (1.0f - g * g) / (4.0f * kPi * den * sqrtf(den));
}

// New tracing direction scattered from tracing direction d with cos ~ HG(g).
__device__ __forceinline__ float3 hg_sample(float g, float3 d, float xi0, float xi1) {
    float ct;
    if (fabsf(g) < 1e-3f) ct = 1.0f - 2.0f * xi0;
    else {
        const float s = (1.0f - g * g) / (1.0f - g + 2.0f * g * xi0);
        ct = (1.0f + g * g - s * s) / (2.0f * g);
    }
    ct = fminf(fmaxf(ct, -1.0f), 1.0f);
    const float st = sqrtf(fmaxf(0.0f, 1.0f - ct * ct));
    float sp, cp;
    sincosf(2.0f * kPi * xi1, &sp, &cp);
    float3 b1, b2;
    duff_basis(d, b1, b2);
    return normalize3((st * cp) * b1 + (st * sp) * b2 + ct * d);
}

// The volume's phase function at cos theta between propagation directions: HG (tab null),
// or the table's value in the 0.1-degree bin of theta.  tab is the volume's first-bounce
// table (v.lm) or the one after the first bounce (v.lmc, chopped or the same).
__device__ __forceinline__ float phase_eval(const VolumeView& v, const float* tab, float ct) {
    if (!tab) return hg_eval(v.g, ct);
    const float th = acosf(fminf(fmaxf(ct, -1.0f), 1.0f));
    const int j = min((int)(th * ((float)RPNN_LM_BINS / kPi)), RPNN_LM_BINS - 1);
    return __ldg(tab + j);
}

// New tracing direction from the phase function: HG (tab null), or a table bin chosen by
// its cumulative probability xi0 with cos theta uniform inside it (azimuth 2 pi xi1).
__device__ __forceinline__ float3 phase_sample(const VolumeView& v, const float* tab, float3 d, float xi0,
                                               float xi1) {
    if (!tab) return hg_sample(v.g, d, xi0, xi1);
    const float* cdf = tab + RPNN_LM_BINS;
    const float* cb = tab + 2 * RPNN_LM_BINS + 1;
    int lo = 0, hi = RPNN_LM_BINS;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(cdf + mid) <= xi0) lo = mid; else hi = mid;
    }
    const float c0 = __ldg(cdf + lo), c1 = __ldg(cdf + lo + 1);
    const float f = c1 > c0 ? (xi0 - c0) / (c1 - c0) : 0.0f;
    const float e0 = __ldg(cb + lo), e1 = __ldg(cb + lo + 1);
    const float ct = fminf(fmaxf(e0 - f * (e0 - e1), -1.0f), 1.0f);
    const float st = sqrtf(fmaxf(0.0f, 1.0f - ct * ct));
    float sp, cp;
    sincosf(2.0f * kPi * xi1, &sp, &cp);
    float3 b1, b2;
    duff_basis(d, b1, b2);
    return normalize3((st * cp) * b1 + (st * sp) * b2 + ct * d);
}

// Ray / grid-box clip: [t0, t1] inside [0, ext].
__device__ __forceinline__ bool box_clip(const float ext[3], float3 o, float3 d, float& t0, float& t1) {
    float tmin = 0.0f, tmax = INFINITY;
    const float oo[3] = {o.x, o.y, o.z}, dd[3] = {d.x, d.y, d.z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (dd[a] != 0.0f) {
            float ta = (0.0f - oo[a]) / dd[a], tb = (ext[a] - oo[a]) / dd[a];
            if (ta > tb) { float t = ta; ta = tb; tb = t; }
            tmin = fmaxf(tmin, ta);
            tmax = fminf(tmax, tb);
        } else if (oo[a] < 0.0f || oo[a] > ext[a]) {
            return false;
        }
    }
    t0 = tmin; t1 = tmax;
    return tmin < tmax;
}

// Raw-grid density (trilinear, voxel centres, zero outside) for free-flight sampling.
__device__ __forceinline__ float raw_density(const VolumeView& v, float3 p) {
    const float u[3] = {p.x * v.inv_h0 - 0.5f, p.y * v.inv_h0 - 0.5f, p.z * v.inv_h0 - 0.5f};
    int i[3];
    float f[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float fl = floorf(u[a]);
        f[a] = u[a] - fl;
        i[a] = (int)fl;
        if (i[a] < -1 || i[a] > v.n[a] - 1) return 0.0f;
    }
    const int nx = v.n[0], ny = v.n[1], nz = v.n[2];
    float c[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int x = i[0] + (k & 1), y = i[1] + ((k >> 1) & 1), z = i[2] + (k >> 2);
        const bool in = x >= 0 && y >= 0 && z >= 0 && x < nx && y < ny && z < nz;
        c[k] = in ? __ldg(v.raw + ((size_t)z * ny + y) * nx + x) : 0.0f;
    }
    const float c00 = fmaf(f[0], c[1] - c[0], c[0]), c10 = fmaf(f[0], c[3] - c[2], c[2]);
    const float c01 = fmaf(f[0], c[5] - c[4], c[4]), c11 = fmaf(f[0], c[7] - c[6], c[6]);
    const float c0 = fmaf(f[1], c10 - c00, c00), c1 = fmaf(f[1], c11 - c01, c01);
    return fmaf(f[2], c1 - c0, c0);
}

// Walk over the tracking bricks a ray crosses (3-D DDA): current brick (bx, by, bz), the
// ray parameter at which it is left across each axis (tn*), the parameter span of one
// brick along each axis (td*) and the step direction (s*).
struct BrickWalk {
    int bx, by, bz, sx, sy, sz;
    float tnx, tny, tnz, tdx, tdy, tdz;
};

__device__ __forceinline__ void walk_axis(float o, float d, float t0, float bs, int nb, int& b, int& s, float& tn,
                                          float& td) {
    b = (int)floorf((o + t0 * d) / bs);
    b = min(max(b, 0), nb - 1);
    if (d > 0.0f) { s = 1; tn = ((float)(b + 1) * bs - o) / d; td = bs / d; }
    else if (d < 0.0f) { s = -1; tn = ((float)b * bs - o) / d; td = -bs / d; }
    else { s = 0; tn = INFINITY; td = INFINITY; }
}

__device__ __forceinline__ void walk_init(const VolumeView& v, float3 o, float3 d, float t0, BrickWalk& w) {
    walk_axis(o.x, d.x, t0, v.bs, v.nb[0], w.bx, w.sx, w.tnx, w.tdx);
    walk_axis(o.y, d.y, t0, v.bs, v.nb[1], w.by, w.sy, w.tny, w.tdy);
    walk_axis(o.z, d.z, t0, v.bs, v.nb[2], w.bz, w.sz, w.tnz, w.tdz);
}

// end of the current brick's segment, capped at t1
__device__ __forceinline__ float walk_exit(const BrickWalk& w, float t1) {
    return fminf(fminf(fminf(w.tnx, w.tny), w.tnz), t1);
}

// into the next brick across the first boundary (x before y before z on ties); false
// once the ray leaves the grid of bricks
__device__ __forceinline__ bool walk_step(const VolumeView& v, BrickWalk& w) {
    if (w.tny < w.tnx && w.tny <= w.tnz) { w.by += w.sy; w.tny += w.tdy; return (unsigned)w.by < (unsigned)v.nb[1]; }
    if (w.tnz < w.tnx) { w.bz += w.sz; w.tnz += w.tdz; return (unsigned)w.bz < (unsigned)v.nb[2]; }
    w.bx += w.sx; w.tnx += w.tdx; return (unsigned)w.bx < (unsigned)v.nb[0];
}

__device__ __forceinline__ float walk_majorant(const VolumeView& v, const BrickWalk& w) {
    return __ldg(v.bmaj + ((size_t)w.bz * v.nb[1] + w.by) * v.nb[0] + w.bx);
}

// Delta (Woodcock) tracking with a piecewise-constant majorant.  Each tentative collision
// draws one Philox block at step *ctr: x gives the majorant optical depth to travel,
// tau = -log(1 - x), y the real/null decision (y * mu_b < mu_t).  The ray walks the
// bricks spending tau at each brick's rate mu_b (empty bricks spend nothing), so the
// tentative collision falls where the majorant's optical depth reaches tau.
// 1 = collision at x, 0 = escape, -1 = cap reached.
__device__ __forceinline__ int delta_track(const VolumeView& v, float3 o, float3 d, const Rng& rng,
                                           uint32_t& ctr, float3& x) {
    float t0, t1;
    if (v.majorant <= 0.0f || !box_clip(v.ext, o, d, t0, t1)) return 0;
    BrickWalk w;
    walk_init(v, o, d, t0, w);
    float t = t0, tau = 0.0f, xy = 0.0f;
    bool fresh = true;                  // a new block is needed for the next collision
    for (uint32_t n = 0; n < v.track_cap; ++n) {
        const float te = walk_exit(w, t1);
        const float mu_b = walk_majorant(v, w);
        if (mu_b > 0.0f) {
            if (fresh) {
                const float4 xi = rng.draw(ctr++);
                tau = -logf(1.0f - xi.x);
                xy = xi.y;
                fresh = false;
            }
            const float seg = mu_b * (te - t);
            if (tau < seg) {
                t += tau / mu_b;
                fresh = true;
                const float3 p = o + t * d;
                if (xy * mu_b < raw_density(v, p)) { x = p; return 1; }
                continue;
            }
            tau -= seg;
        }
        if (te >= t1) return 0;
        t = te;
        if (!walk_step(v, w)) return 0;
    }
    return -1;
}

// Delta tracking against the global majorant (one block per tentative collision: x for
// the exponential step, y for the real/null decision), for the path tracer's bounces,
// which start inside the medium where the bricks hold nearly the global majorant anyway.
// The medium behind a first bounce has extinction v.dscale * mu_t (the chopped
// Lorenz-Mie medium; 1 otherwise): the majorant's rate scales, the real/null ratio not.
__device__ __forceinline__ int delta_track_global(const VolumeView& v, float3 o, float3 d, const Rng& rng,
                                                  uint32_t& ctr, float3& x) {
    float t0, t1;
    if (v.majorant <= 0.0f || !box_clip(v.ext, o, d, t0, t1)) return 0;
    const float maj_s = v.majorant * v.dscale;
    float t = t0;
    for (uint32_t n = 0; n < v.track_cap; ++n) {
        const float4 xi = rng.draw(ctr++);
        t -= logf(1.0f - xi.x) / maj_s;
        if (t >= t1) return 0;
        const float3 p = o + t * d;
        if (xi.y * v.majorant < raw_density(v, p)) { x = p; return 1; }
    }
    return -1;
}

// Ratio-tracking transmittance from o along d to the grid boundary over the same walk:
// one block (x -> optical depth) per tentative collision, T *= 1 - mu_t / mu_b there.
// Light travels through the medium of extinction v.dscale * mu_t (see delta_track_global):
// each brick's rate is v.dscale * mu_b, the ratio unchanged.
__device__ __forceinline__ float ratio_track(const VolumeView& v, float3 o, float3 d, const Rng& rng,
                                             uint32_t& ctr, bool& capped) {
    float t0, t1;
    if (v.majorant <= 0.0f || !box_clip(v.ext, o, d, t0, t1)) return 1.0f;
    BrickWalk w;
    walk_init(v, o, d, t0, w);
    float t = t0, T = 1.0f, tau = 0.0f;
    bool fresh = true;
    for (uint32_t n = 0; n < v.track_cap; ++n) {
        const float te = walk_exit(w, t1);
        const float mu_b = walk_majorant(v, w);
        if (mu_b > 0.0f) {
            if (fresh) {
                tau = -logf(1.0f - rng.draw(ctr++).x);
                fresh = false;
            }
            const float mu_s = mu_b * v.dscale;
            const float seg = mu_s * (te - t);
            if (tau < seg) {
                t += tau / mu_s;
                fresh = true;
                T *= 1.0f - raw_density(v, o + t * d) / mu_b;
                continue;
            }
            tau -= seg;
        }
        if (te >= t1) return T;
        t = te;
        if (!walk_step(v, w)) return T;
    }
    capped = true;
    return T;
}

// Next-event estimate towards the directional light (the phase argument is the
// cosine between tracing direction d and the light direction).  `first`: x is a path's
// first bounce (the camera's or a record's vertex), which scatters with the full phase
// function; later vertices use the one after the first bounce.
__device__ __forceinline__ float nee(const VolumeView& v, bool first, float3 x, float3 d, float3 wl, float E,
                                     const Rng& rng, uint32_t& ctr, bool& capped) {
    const float T = ratio_track(v, x, wl, rng, ctr, capped);
    return E * phase_eval(v, first ? v.lm : v.lmc, dot3(d, wl)) * T;
}

// One path estimate of L_i at vertex x reached along tracing direction d: phase
// sampling, delta tracking to the next collision, survival with probability albedo,
// NEE there, repeat.  Draw order per bounce: direction block, tracking blocks,
// survival block, shadow blocks.  x is the path's first bounce (full phase function);
// everything after it uses the medium behind the first bounce (v.lmc, v.dscale,
// v.albedo_c), which is the volume's own unless its Lorenz-Mie function is chopped.
__device__ __forceinline__ float path_Li(const VolumeView& v, float3 x, float3 d, float3 wl, float E,
                                         const Rng& rng, bool& capped) {
    uint32_t ctr = 0;
    float L = 0.0f;
    for (int b = 0; b < kBounceCap; ++b) {
        float4 xi = rng.draw(ctr++);
        const float3 nd = phase_sample(v, b == 0 ? v.lm : v.lmc, d, xi.x, xi.y);
        float3 nx;
        const int hit = delta_track_global(v, x, nd, rng, ctr, nx);
        if (hit < 0) { capped = true; return L; }
        if (hit == 0) return L;
        xi = rng.draw(ctr++);
        if (!(xi.x < v.albedo_c)) return L;
        L += nee(v, false, nx, nd, wl, E, rng, ctr, capped);
        x = nx;
        d = nd;
    }
    capped = true;
    return L;
}

__device__ __forceinline__ void raise_status(uint32_t* status, uint32_t bits) {
    if (status) atomicOr(status, bits);
}

}  // namespace rpnn
