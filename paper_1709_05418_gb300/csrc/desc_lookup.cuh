// desc_lookup.cuh -- FP32 arithmetic of the hierarchical stencil descriptor (Sec. 4.2,
// Fig. 5), shared by every kernel that builds descriptor values, so that they all follow
// one fixed rounding sequence (no contraction, explicit _rn intrinsics):
//   frame: z = light, x = normalize(z cross omega), y = z cross x (omega = -d), with the
//          Duff et al. 2017 basis of z when omega is parallel to z; gamma = acos(omega . z);
//   s = inv_h0 * 2^-m, g = (inv_mean * 2^(k-1)) * s, A = g ex, B = g ey, C = g ez,
//   U0 = x s - 0.5, u = fma(oz, C, fma(oy, B, fma(ox, A, U0))),
//   trilinear lerp(a, b, f) = fma(f, b - a, a) in x, then y, then z, from one 32-byte
//   corner record per lookup.
#pragma once
#include "common.cuh"

namespace rpnn {
namespace desc {

__device__ __forceinline__ float lerp_rn(float a, float b, float f) {
    return __fmaf_rn(f, __fsub_rn(b, a), a);
}

struct Frame {
    float ex[3], ey[3], ez[3];
    float gamma;
};

__device__ __forceinline__ Frame make_frame(const float d[3], const float wl[3]) {
    Frame F;
    const float w[3] = {-d[0], -d[1], -d[2]};
    const float* ez = wl;
    float cr[3];
    cr[0] = __fsub_rn(__fmul_rn(ez[1], w[2]), __fmul_rn(ez[2], w[1]));
    cr[1] = __fsub_rn(__fmul_rn(ez[2], w[0]), __fmul_rn(ez[0], w[2]));
    cr[2] = __fsub_rn(__fmul_rn(ez[0], w[1]), __fmul_rn(ez[1], w[0]));
    const float len2 = __fadd_rn(__fadd_rn(__fmul_rn(cr[0], cr[0]), __fmul_rn(cr[1], cr[1])),
                                 __fmul_rn(cr[2], cr[2]));
    if (len2 < 1e-12f) {
        // Duff et al. 2017 basis of z in FP32: sg = copysign(1, z), a = -1 / (sg + z),
        // x = (1 + sg x^2 a, sg x y a, -sg x), each operation rounded in this order
        const float sg = signbit(ez[2]) ? -1.0f : 1.0f;
        const float a = __fdiv_rn(-1.0f, __fadd_rn(sg, ez[2]));
        F.ex[0] = __fadd_rn(1.0f, __fmul_rn(__fmul_rn(__fmul_rn(sg, ez[0]), ez[0]), a));
        F.ex[1] = __fmul_rn(sg, __fmul_rn(__fmul_rn(ez[0], ez[1]), a));
        F.ex[2] = __fmul_rn(-sg, ez[0]);
    } else {
        const float len = __fsqrt_rn(len2);
        for (int a = 0; a < 3; ++a) F.ex[a] = __fdiv_rn(cr[a], len);
    }
    for (int a = 0; a < 3; ++a) F.ez[a] = ez[a];
    F.ey[0] = __fsub_rn(__fmul_rn(ez[1], F.ex[2]), __fmul_rn(ez[2], F.ex[1]));
    F.ey[1] = __fsub_rn(__fmul_rn(ez[2], F.ex[0]), __fmul_rn(ez[0], F.ex[2]));
    F.ey[2] = __fsub_rn(__fmul_rn(ez[0], F.ex[1]), __fmul_rn(ez[1], F.ex[0]));
    float cg = __fadd_rn(__fadd_rn(__fmul_rn(w[0], wl[0]), __fmul_rn(w[1], wl[1])), __fmul_rn(w[2], wl[2]));
    cg = fminf(fmaxf(cg, -1.0f), 1.0f);
    F.gamma = acosf(cg);
    return F;
}

// Per-level constants of one volume, staged in shared memory once per block: the
// coordinate scale s = inv_h0 * 2^-m and gk = (inv_mean * 2^(k-1)) * s of level k (mip m),
// the level dims, and the record index of cell (0,0,0) with the record strides (records
// cover cells -1 .. n-1 on each axis).
struct LevelGeo {
    float hx, hy, hz;          // 1.5*2^23 + n - 1 per axis: the largest valid t (see lookup)
    uint32_t rbias, sy, sz;    // record index = rbias + bits(t2) sz + bits(t1) sy + bits(t0)
};
// Level k's constants (32 bytes, two 16-byte shared loads) ...
struct __align__(16) LevelK {
    float s, gk;
    LevelGeo g0;
};
// ... and, for a blended descriptor, those of mip level m + 1 with its weight w (w = 0:
// level k reads level m alone)
struct __align__(16) LevelB {
    float s1, gk1, w, pad;
    LevelGeo g1;
    uint32_t pad2[2];
};

// Trilinear lookup from one 32-byte corner record (c0, c1-c0, c2, c3-c2, c4, c5-c4, c6,
// c7-c6).  floor(u) without conversions: t = u + 1.5*2^23 rounded down is floor(u) +
// 1.5*2^23 exactly for |u| < 2^22, and its bit pattern minus that of 1.5*2^23 is the cell
// index; the fraction u - (t - 1.5*2^23) is u - floor(u) exactly.  The cell is inside
// [-1, n-1] iff t lies in [1.5*2^23 - 1, 1.5*2^23 + n - 1], a test that also rejects any
// |u| >= 2^22 (t then falls outside), so out-of-range points read 0 exactly as the
// reference, which clamps |u| to 1e6 first.  The record index folds the bit-pattern
// offsets into r000 (uint32 wrap-around).  The x-lerps use the stored differences, which
// round exactly as lerp_rn's own subtraction.
constexpr float kFloorMagic = 12582912.0f;   // 1.5 * 2^23

__device__ __forceinline__ float lookup(const float4* __restrict__ packed, const LevelGeo& g, float u0, float u1,
                                        float u2) {
    const float t0 = __fadd_rd(u0, kFloorMagic), t1 = __fadd_rd(u1, kFloorMagic), t2 = __fadd_rd(u2, kFloorMagic);
    if (!(t0 >= kFloorMagic - 1.0f && t0 <= g.hx && t1 >= kFloorMagic - 1.0f && t1 <= g.hy &&
          t2 >= kFloorMagic - 1.0f && t2 <= g.hz))
        return 0.0f;
    const float f0 = __fsub_rn(u0, __fsub_rn(t0, kFloorMagic));
    const float f1 = __fsub_rn(u1, __fsub_rn(t1, kFloorMagic));
    const float f2 = __fsub_rn(u2, __fsub_rn(t2, kFloorMagic));
    const uint32_t r = g.rbias + (uint32_t)__float_as_int(t2) * g.sz + (uint32_t)__float_as_int(t1) * g.sy +
                       (uint32_t)__float_as_int(t0);
    float c[8];
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(c[0]), "=f"(c[1]), "=f"(c[2]), "=f"(c[3]), "=f"(c[4]), "=f"(c[5]), "=f"(c[6]), "=f"(c[7])
        : "l"(packed + 2 * (size_t)r));
    const float c00 = __fmaf_rn(f0, c[1], c[0]);
    const float c10 = __fmaf_rn(f0, c[3], c[2]);
    const float c01 = __fmaf_rn(f0, c[5], c[4]);
    const float c11 = __fmaf_rn(f0, c[7], c[6]);
    const float c0 = lerp_rn(c00, c10, f1);
    const float c1 = lerp_rn(c01, c11, f1);
    return lerp_rn(c0, c1, f2);
}

// lookup() for a point known to lie inside the level (stencil_class == kInside): the same
// arithmetic without the range test.
__device__ __forceinline__ float lookup_in(const float4* __restrict__ packed, const LevelGeo& g, float u0, float u1,
                                           float u2) {
    const float t0 = __fadd_rd(u0, kFloorMagic), t1 = __fadd_rd(u1, kFloorMagic), t2 = __fadd_rd(u2, kFloorMagic);
    const float f0 = __fsub_rn(u0, __fsub_rn(t0, kFloorMagic));
    const float f1 = __fsub_rn(u1, __fsub_rn(t1, kFloorMagic));
    const float f2 = __fsub_rn(u2, __fsub_rn(t2, kFloorMagic));
    const uint32_t r = g.rbias + (uint32_t)__float_as_int(t2) * g.sz + (uint32_t)__float_as_int(t1) * g.sy +
                       (uint32_t)__float_as_int(t0);
    float c[8];
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(c[0]), "=f"(c[1]), "=f"(c[2]), "=f"(c[3]), "=f"(c[4]), "=f"(c[5]), "=f"(c[6]), "=f"(c[7])
        : "l"(packed + 2 * (size_t)r));
    const float c00 = __fmaf_rn(f0, c[1], c[0]);
    const float c10 = __fmaf_rn(f0, c[3], c[2]);
    const float c01 = __fmaf_rn(f0, c[5], c[4]);
    const float c11 = __fmaf_rn(f0, c[7], c[6]);
    const float c0 = lerp_rn(c00, c10, f1);
    const float c1 = lerp_rn(c01, c11, f1);
    return lerp_rn(c0, c1, f2);
}

// Where one shading point's stencil lies in a level, from its bounding box: the points
// u = U0 + ox A + oy B + oz C (ox, oy in [-1, 1], oz in [-1, 3]) span, per axis,
// U0 -+ (|A| + |B|) plus the range of oz C.  A level's cells cover u in [-1, n); with a
// margin of 1/64 cell (far above the FP32 rounding of u, a few 2^-12 cells) the box
// decides whether every point is inside (kInside: no range tests needed), every point is
// outside (kOutside: every value is 0), or neither (kMixed: test each point).
enum { kOutside = 0, kInside = 1, kMixed = 2 };
__device__ __forceinline__ int stencil_class(const LevelGeo& g, const float (&A)[3], const float (&B)[3],
                                             const float (&C)[3], const float (&U0)[3]) {
    constexpr float kMargin = 1.0f / 64.0f;
    const float hi[3] = {g.hx - kFloorMagic + 1.0f, g.hy - kFloorMagic + 1.0f, g.hz - kFloorMagic + 1.0f};  // n
    bool inside = true, outside = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float ab = fabsf(A[a]) + fabsf(B[a]);
        const float lo = U0[a] - ab + fminf(-C[a], 3.0f * C[a]);
        const float up = U0[a] + ab + fmaxf(-C[a], 3.0f * C[a]);
        inside = inside && lo >= -1.0f + kMargin && up < hi[a] - kMargin;
        outside = outside || up < -1.0f - kMargin || lo >= hi[a] + kMargin;
    }
    return outside ? kOutside : (inside ? kInside : kMixed);
}


// level k's constants of volume v
__device__ __forceinline__ LevelGeo make_geo(const VolumeView& v, int m) {
    const LevelDesc L = v.lvl[m];
    LevelGeo g;
    g.hx = kFloorMagic + (float)(L.ax - 1);
    g.hy = kFloorMagic + (float)(L.ay - 1);
    g.hz = kFloorMagic + (float)(L.az - 1);
    g.sy = (uint32_t)(L.ax + 1);
    g.sz = (uint32_t)((L.ax + 1) * (L.ay + 1));
    // cell (i0, i1, i2) is record rec_offset + (i2+1) sz + (i1+1) sy + (i0+1), and
    // i = bits(t) - bits(1.5*2^23)
    const uint32_t mb = (uint32_t)__float_as_int(kFloorMagic);
    g.rbias = (uint32_t)L.rec_offset + g.sz + g.sy + 1u - mb * (g.sz + g.sy + 1u);
    return g;
}

// level k's constants of volume v
__device__ __forceinline__ LevelK make_level(const VolumeView& v, int k) {
    const int m = v.mip_of_level[k];
    LevelK g;
    g.s = __fmul_rn(v.inv_h0, __int_as_float((127 - m) << 23));   // * 2^-m
    g.gk = __fmul_rn(__fmul_rn(v.inv_mean_f, (float)(1 << k)), g.s);
    g.g0 = make_geo(v, m);
    return g;
}

__device__ __forceinline__ LevelB make_blend(const VolumeView& v, int k) {
    const int m = v.mip_of_level[k];
    LevelB b{};
    b.w = v.mip_w[k];
    if (b.w > 0.0f) {
        b.s1 = __fmul_rn(v.inv_h0, __int_as_float((126 - m) << 23));   // * 2^-(m+1)
        b.gk1 = __fmul_rn(__fmul_rn(v.inv_mean_f, (float)(1 << k)), b.s1);
        b.g1 = make_geo(v, m + 1);
    }
    return b;
}

}  // namespace desc
}  // namespace rpnn
