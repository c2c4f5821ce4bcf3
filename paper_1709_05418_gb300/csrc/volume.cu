// volume.cu -- per-volume preprocessing: statistics (Sec. 4.2 mean-free-path
// normalisation) and the Gaussian mip pyramid (Sec. 6, sigma_i = 2^i fine voxels),
// stored as corner-packed records for the descriptor gather.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace rpnn {

namespace {

struct DevStats {
    unsigned int max_bits;      // max voxel (non-negative floats order like uint)
    unsigned int bad;           // negative / NaN / Inf seen
    unsigned long long count;   // voxels > 0
    unsigned long long isum;    // fixed-point sum
};

__global__ void k_f16_to_f32(const __half* __restrict__ in, float* __restrict__ out, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = __half2float(in[i]);
}

// The grid is read as 16-byte vectors (the allocation is 256-byte aligned), the last n % 4
// voxels one by one; max, count and the fixed-point sum below are exact in any order.
__device__ __forceinline__ void stats_max_one(float x, unsigned int& mx, unsigned int& bad, unsigned int& cnt) {
    if (!(x >= 0.0f) || isinf(x)) { bad = 1; return; }
    mx = max(mx, __float_as_uint(x));
    cnt += x > 0.0f;
}
__global__ void k_stats_max(const float* __restrict__ v, int64_t n, DevStats* st) {
    unsigned int mx = 0, bad = 0, c32 = 0;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nt = (int64_t)gridDim.x * blockDim.x;
    const float4* v4 = reinterpret_cast<const float4*>(v);
    for (int64_t i = tid; i < n / 4; i += nt) {
        const float4 q = __ldg(v4 + i);
        stats_max_one(q.x, mx, bad, c32); stats_max_one(q.y, mx, bad, c32);
        stats_max_one(q.z, mx, bad, c32); stats_max_one(q.w, mx, bad, c32);
    }
    for (int64_t i = n / 4 * 4 + tid; i < n; i += nt) stats_max_one(v[i], mx, bad, c32);
    unsigned long long cnt = c32;       // a thread counts at most n / threads + 4 voxels
    for (int o = 16; o; o >>= 1) {
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        bad |= __shfl_xor_sync(0xffffffffu, bad, o);
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&st->max_bits, mx);
        if (bad) atomicOr(&st->bad, 1u);
        atomicAdd(&st->count, cnt);
    }
}

// x * 2^S truncated to an integer, for finite x > 0 with x * 2^S < 2^32, from the float's
// bits: x = M * 2^(E - 150) with the 24-bit significand M (hidden bit set unless
// subnormal) and biased exponent E (1 for subnormals), so the product is M shifted by
// E - 150 + S, and a right shift truncates exactly as the real value rounds toward zero.
__device__ __forceinline__ unsigned long long fixed_point(float x, int S) {
    const uint32_t b = __float_as_uint(x);
    const int E = (int)(b >> 23);
    const unsigned long long M = (b & 0x7FFFFFu) | (E ? 0x800000u : 0u);
    const int sh = (E ? E : 1) - 150 + S;
    if (sh >= 0) return M << sh;
    return sh > -24 ? M >> (-sh) : 0ull;
}

// Fixed-point sum: each v > 0 truncated to an integer with S = 32 - e fraction bits,
// where the majorant is below 2^e; the integer sum is exact (< 2^62 for 2^30 voxels)
// and independent of order.
__global__ void k_stats_sum(const float* __restrict__ v, int64_t n, DevStats* st) {
    int e;
    frexpf(__uint_as_float(st->max_bits), &e);
    const int S = 32 - e;
    unsigned long long s = 0;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nt = (int64_t)gridDim.x * blockDim.x;
    const float4* v4 = reinterpret_cast<const float4*>(v);
    for (int64_t i = tid; i < n / 4; i += nt) {
        const float4 q = __ldg(v4 + i);
        if (q.x > 0.0f) s += fixed_point(q.x, S);
        if (q.y > 0.0f) s += fixed_point(q.y, S);
        if (q.z > 0.0f) s += fixed_point(q.z, S);
        if (q.w > 0.0f) s += fixed_point(q.w, S);
    }
    for (int64_t i = n / 4 * 4 + tid; i < n; i += nt) {
        const float x = v[i];
        if (x > 0.0f) s += fixed_point(x, S);
    }
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&st->isum, s);
}

// One separable pass of the Gaussian filter along one axis with decimation: output index
// j along the axis reads fine indices j*st + off + m, m = 0..T-1 (zero outside, so only the
// taps inside the grid are visited), accumulated in ascending m as acc = acc + w*v (no
// contraction); the final pass multiplies by `scale` (1/mean).
// The y or z passes of several levels in one launch (outputs of job j at flattened indices
// first[j] .. first[j+1] - 1), so that the deep levels' few long tap chains run beside the
// others instead of after them.
struct MipJob {
    const float* in;
    float* out;
    const float* w;
    int ix, iy, iz, ox, oy, oz, st, off, T;
    int64_t first;
};
struct MipJobs {
    MipJob j[kMaxLevels];
    int n, axis, apply_scale;
    float scale;
    int64_t total;
};
__global__ void k_mip_pass_multi(const __grid_constant__ MipJobs J) {
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < J.total;
         o += (int64_t)gridDim.x * blockDim.x) {
        int k = 0;
        while (k + 1 < J.n && J.j[k + 1].first <= o) ++k;
        const MipJob& b = J.j[k];
        const int64_t q = o - b.first;
        const int x = (int)(q % b.ox);
        const int y = (int)((q / b.ox) % b.oy);
        const int z = (int)(q / ((int64_t)b.ox * b.oy));
        int j, n;
        int64_t base, stride;
        if (J.axis == 1) { j = y; n = b.iy; base = (int64_t)z * b.iy * b.ix + x; stride = b.ix; }
        else { j = z; n = b.iz; base = (int64_t)y * b.ix + x; stride = (int64_t)b.ix * b.iy; }
        float acc = 0.0f;
        const int t0 = j * b.st + b.off;
        const int mlo = max(0, -t0), mhi = min(b.T, n - t0);
#pragma unroll 8
        for (int m = mlo; m < mhi; ++m)
            acc = __fadd_rn(acc, __fmul_rn(__ldg(b.w + m), __ldg(b.in + base + (int64_t)(t0 + m) * stride)));
        b.out[q] = J.apply_scale ? __fmul_rn(acc, J.scale) : acc;
    }
}

// The x passes of several levels, staged: a block copies R consecutive x lines of the fine
// grid (contiguous in memory) into shared memory once, with coalesced loads (line pitch
// nx + 1 floats), and computes every level's decimated outputs (line r, index j) from them
// with r fastest, so a warp's lanes read different lines at one position (different banks)
// instead of 32 scattered global lines per tap.  Each output's taps in ascending m,
// acc = acc + w*v.
struct MipXJob {
    float* out;
    const float* w;
    int ax, st, off, T;
};
struct MipXJobs {
    MipXJob j[kMaxLevels];
    int n;
};
__global__ void k_mip_pass_x(const float* __restrict__ in, int nx, int64_t nrows, int R,
                             const __grid_constant__ MipXJobs J) {
    extern __shared__ float lines[];
    const int pitch = nx + 1;
    for (int64_t r0 = (int64_t)blockIdx.x * R; r0 < nrows; r0 += (int64_t)gridDim.x * R) {
        const int nr = (int)min((int64_t)R, nrows - r0);
        __syncthreads();                       // the previous lines' readers are done
        // the nr lines are nr * nx consecutive floats: eight loads per thread in flight at once
        const float* src = in + r0 * nx;
        const int total = nr * nx, nb = (int)blockDim.x;
        int e = threadIdx.x;
        for (; e + 7 * nb < total; e += 8 * nb) {
            float v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = __ldg(src + e + k * nb);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int ee = e + k * nb, r = ee / nx;
                lines[r * pitch + ee - r * nx] = v[k];
            }
        }
        for (; e < total; e += nb) {
            const int r = e / nx;
            lines[r * pitch + e - r * nx] = __ldg(src + e);
        }
        __syncthreads();
        for (int k = 0; k < J.n; ++k) {
            const MipXJob& b = J.j[k];
            for (int task = threadIdx.x; task < R * b.ax; task += blockDim.x) {
                const int r = task % R, j = task / R;
                if (r >= nr) continue;
                const float* line = lines + r * pitch;
                const int t0 = j * b.st + b.off;
                const int mlo = max(0, -t0), mhi = min(b.T, nx - t0);
                float acc = 0.0f;
#pragma unroll 4
                for (int m = mlo; m < mhi; ++m) acc = __fadd_rn(acc, __fmul_rn(__ldg(b.w + m), line[t0 + m]));
                b.out[(r0 + r) * b.ax + j] = acc;
            }
        }
    }
}

// Corner packing: record (rx, ry, rz) of a level with dims (ax, ay, az) describes cell
// (rx-1, ry-1, rz-1).  With c[dx + 2 dy + 4 dz] its 8 corner values (zero outside), the
// record holds c0, c1 - c0, c2, c3 - c2, c4, c5 - c4, c6, c7 - c6: the x-differences the
// four x-lerps need, rounded exactly as a lerp rounds them.
__global__ void k_pack(const float* __restrict__ lv, float4* __restrict__ rec, int ax, int ay, int az) {
    const int rx_n = ax + 1, ry_n = ay + 1, rz_n = az + 1;
    const int64_t total = (int64_t)rx_n * ry_n * rz_n;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < total;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int x0 = (int)(r % rx_n) - 1;
        const int y0 = (int)((r / rx_n) % ry_n) - 1;
        const int z0 = (int)(r / ((int64_t)rx_n * ry_n)) - 1;
        float c[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int x = x0 + (k & 1), y = y0 + ((k >> 1) & 1), z = z0 + (k >> 2);
            const bool in = x >= 0 && y >= 0 && z >= 0 && x < ax && y < ay && z < az;
            c[k] = in ? lv[((int64_t)z * ay + y) * ax + x] : 0.0f;
        }
        rec[2 * r] = make_float4(c[0], __fsub_rn(c[1], c[0]), c[2], __fsub_rn(c[3], c[2]));
        rec[2 * r + 1] = make_float4(c[4], __fsub_rn(c[5], c[4]), c[6], __fsub_rn(c[7], c[6]));
    }
}

float bits_to_float(unsigned int b) {
    float f;
    std::memcpy(&f, &b, sizeof f);
    return f;
}

int grid_for(int64_t n, int block, int num_sms) {
    int64_t g = (n + block - 1) / block;
    const int64_t cap = (int64_t)num_sms * 16;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

// Gaussian taps of level i: sigma = 2^i, offsets |d| <= 3 sigma, normalised (FP64,
// rounded to FP32).
std::vector<float> gauss_taps(int level, int* off) {
    const double sigma = std::ldexp(1.0, level);
    int T;
    if (level == 0) { T = 7; *off = -3; }
    else { T = 6 << level; *off = (1 << (level - 1)) - 3 * (1 << level); }
    std::vector<double> w(T);
    double sum = 0.0;
    for (int m = 0; m < T; ++m) {
        const double d = (level == 0) ? (double)(m - 3) : (double)m - 3.0 * sigma + 0.5;
        w[m] = std::exp(-d * d / (2.0 * sigma * sigma));
        sum += w[m];
    }
    std::vector<float> wf(T);
    for (int m = 0; m < T; ++m) wf[m] = (float)(w[m] / sum);
    return wf;
}

}  // namespace

rpnn_status load_density(Ctx& c, Volume& v, const void* src, int dtype, cudaStream_t s) {
    const int64_t n = (int64_t)v.n[0] * v.n[1] * v.n[2];
    rpnn_status st = v.raw.reserve(n * sizeof(float));
    if (st) return st;
    if (dtype == RPNN_F32) {
        RPNN_CUDA_TRY(cudaMemcpyAsync(v.raw.p, src, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
    } else {
        k_f16_to_f32<<<grid_for(n, 256, c.num_sms), 256, 0, s>>>((const __half*)src, v.raw.as<float>(), n);
        RPNN_CHECK_LAUNCH();
    }
    return RPNN_OK;
}

// Per-brick majorant for tracking: brick b (kBrick^3 voxels) bounds the trilinear density
// over its region by the largest of the voxels it interpolates, 8b - 1 .. 8b + 8 per axis
// (zero outside the grid).  One thread per brick; max is exact, so the order is free.
__global__ void k_brick_majorant(const float* __restrict__ raw, int nx, int ny, int nz, int bx, int by, int bz,
                                 float* __restrict__ out) {
    const int64_t nb = (int64_t)bx * by * bz;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nb; i += (int64_t)gridDim.x * blockDim.x) {
        const int x0 = (int)(i % bx) * kBrick - 1, y0 = (int)((i / bx) % by) * kBrick - 1,
                  z0 = (int)(i / ((int64_t)bx * by)) * kBrick - 1;
        float m = 0.0f;
        for (int z = max(z0, 0); z <= min(z0 + kBrick + 1, nz - 1); ++z)
            for (int y = max(y0, 0); y <= min(y0 + kBrick + 1, ny - 1); ++y) {
                const float* r = raw + ((int64_t)z * ny + y) * nx;
                // a fixed-length line with in-grid predicates: its loads are in flight together
#pragma unroll
                for (int dx = 0; dx < kBrick + 2; ++dx) {
                    const int x = x0 + dx;
                    if (x >= 0 && x < nx) m = fmaxf(m, __ldg(r + x));
                }
            }
        out[i] = m;
    }
}

rpnn_status volume_brick_majorants(Ctx& c, Volume& v, cudaStream_t s) {
    for (int a = 0; a < 3; ++a) v.info.bricks[a] = v.nb[a] = (v.n[a] + kBrick - 1) / kBrick;
    const int64_t nb = (int64_t)v.nb[0] * v.nb[1] * v.nb[2];
    rpnn_status st = v.bmaj.reserve((size_t)nb * sizeof(float));
    if (st) return st;
    k_brick_majorant<<<grid_for(nb, 128, c.num_sms), 128, 0, s>>>(v.raw.as<float>(), v.n[0], v.n[1], v.n[2], v.nb[0],
                                                                  v.nb[1], v.nb[2], v.bmaj.as<float>());
    RPNN_CHECK_LAUNCH();
    return RPNN_OK;
}

rpnn_status volume_stats(Ctx& c, Volume& v, cudaStream_t s) {
    const int64_t n = (int64_t)v.n[0] * v.n[1] * v.n[2];
    rpnn_status st = v.stats.reserve(sizeof(DevStats));
    if (st) return st;
    DevStats* ds = v.stats.as<DevStats>();
    RPNN_CUDA_TRY(cudaMemsetAsync(ds, 0, sizeof(DevStats), s));
    const int g = grid_for(n, 256, c.num_sms);
    k_stats_max<<<g, 256, 0, s>>>(v.raw.as<float>(), n, ds);
    RPNN_CHECK_LAUNCH();
    k_stats_sum<<<g, 256, 0, s>>>(v.raw.as<float>(), n, ds);
    RPNN_CHECK_LAUNCH();
    DevStats h;
    RPNN_CUDA_TRY(cudaMemcpyAsync(&h, ds, sizeof(DevStats), cudaMemcpyDeviceToHost, s));
    RPNN_CUDA_TRY(cudaStreamSynchronize(s));
    if (h.bad) { set_error("density has negative, NaN or Inf voxels"); return RPNN_ERR_NONFINITE; }
    if (h.count == 0) { set_error("density grid has no voxel > 0"); return RPNN_ERR_ARG; }
    // mean = (fixed-point sum) 2^-S / count, S = 32 - e with the majorant below 2^e; in
    // IEEE double on the host (each operation correctly rounded)
    int e;
    std::frexp(bits_to_float(h.max_bits), &e);
    const double mean = std::ldexp((double)(long long)h.isum, -(32 - e)) / (double)h.count;
    const float inv_mean_f = (float)(1.0 / mean);
    rpnn_volume_info& I = v.info;
    for (int a = 0; a < 3; ++a) I.n[a] = v.n[a];
    const int nmax = std::max(v.n[0], std::max(v.n[1], v.n[2]));
    int L = 1;
    while (((nmax + (1 << (L - 1)) - 1) >> (L - 1)) > 1) ++L;
    I.levels = v.levels = L;
    for (int i = 0; i < 16; ++i)
        for (int a = 0; a < 3; ++a) I.dims[i][a] = v.dims[i][a] = (v.n[a] + (1 << i) - 1) >> i;
    I.mean = mean;
    I.inv_mean_f = inv_mean_f;
    I.majorant = bits_to_float(h.max_bits);
    I.nonzero = (int64_t)h.count;
    // mip level read by stencil level k: largest power-of-two voxel not above the
    // stencil spacing 0.5 * 2^(k-1) mean free paths (exact frexp of an exact product)
    for (int k = 0; k < RPNN_K; ++k) {
        const double sk = 0.5 * std::ldexp((double)inv_mean_f, k) * (double)nmax;
        int m = 0;
        if (sk > 0.0) { int ex; std::frexp(sk, &ex); m = ex - 1; }
        m = std::max(0, std::min(m, L - 1));
        I.mip_of_level[k] = m;
        // blended descriptor: weight of level m + 1 = fraction of log2(spacing) above m
        // (0 where the spacing is outside the pyramid's range)
        double w = 0.0;
        if (sk > 0.0) {
            const double mr = std::log2(sk);
            if (mr > 0.0 && mr < (double)(L - 1)) w = mr - std::floor(mr);
        }
        I.mip_weight[k] = (float)w;
    }
    return RPNN_OK;
}

rpnn_status volume_build_levels(Ctx& c, Volume& v, const int* levels, int nlev, float* const* dst, cudaStream_t s) {
    if (nlev <= 0) return RPNN_OK;
    if (nlev > kMaxLevels) { set_error("too many mip levels (%d)", nlev); return RPNN_ERR_ARG; }
    const int nx = v.n[0], ny = v.n[1], nz = v.n[2];
    // deepest level first: its long tap chains start with the launch
    std::vector<int> ord(levels, levels + nlev);
    for (int l : ord)
        if (l < 0 || l >= v.levels) { set_error("mip level %d out of range", l); return RPNN_ERR_ARG; }
    std::sort(ord.begin(), ord.end(), [](int a, int b) { return a > b; });
    // taps and scratch of every level side by side (offsets in floats, 16-float aligned);
    // volume-owned, grows and never shrinks: no allocation or synchronisation per build
    std::vector<float> taps;
    std::vector<int> offs(nlev), toff(nlev), T(nlev);
    std::vector<int64_t> aoff(nlev), boff(nlev);
    int64_t asz = 0, bsz = 0;
    for (int k = 0; k < nlev; ++k) {
        const int l = ord[k];
        std::vector<float> w = gauss_taps(l, &offs[k]);
        T[k] = (int)w.size();
        toff[k] = (int)taps.size();
        taps.insert(taps.end(), w.begin(), w.end());
        taps.resize((taps.size() + 15) / 16 * 16, 0.0f);
        aoff[k] = asz; asz += ((int64_t)v.dims[l][0] * ny * nz + 15) / 16 * 16;
        boff[k] = bsz; bsz += ((int64_t)v.dims[l][0] * v.dims[l][1] * nz + 15) / 16 * 16;
    }
    rpnn_status rs = v.mip_w.reserve(taps.size() * sizeof(float));
    if (!rs) rs = v.mip_a.reserve((size_t)asz * sizeof(float));
    if (!rs) rs = v.mip_b.reserve((size_t)bsz * sizeof(float));
    if (rs) return rs;
    float* dw = v.mip_w.as<float>();
    float* A = v.mip_a.as<float>();
    float* B = v.mip_b.as<float>();
    RPNN_CUDA_TRY(cudaMemcpyAsync(dw, taps.data(), taps.size() * sizeof(float), cudaMemcpyHostToDevice, s));
    // the x passes of every level in one launch (the fine grid is read once), R lines of nx
    // floats per block in at most 64 KB of shared memory
    constexpr int kLineBytes = 64 * 1024;
    const int R = std::max(1, std::min(32, kLineBytes / ((nx + 1) * (int)sizeof(float))));
    const int smem = R * (nx + 1) * (int)sizeof(float);
    static bool attr = false;
    if (!attr) {
        RPNN_CUDA_TRY(cudaFuncSetAttribute(k_mip_pass_x, cudaFuncAttributeMaxDynamicSharedMemorySize, kLineBytes));
        attr = true;
    }
    const int64_t nrows = (int64_t)ny * nz;
    MipXJobs XJ{};
    XJ.n = nlev;
    for (int k = 0; k < nlev; ++k) {
        const int l = ord[k];
        XJ.j[k] = MipXJob{A + aoff[k], dw + toff[k], v.dims[l][0], 1 << l, offs[k], T[k]};
    }
    k_mip_pass_x<<<grid_for((nrows + R - 1) / R, 1, c.num_sms), 256, smem, s>>>(v.raw.as<float>(), nx, nrows, R, XJ);
    // y passes of every level in one launch, then the z passes (with the 1/mean scale)
    for (int axis = 1; axis <= 2; ++axis) {
        MipJobs J{};
        J.n = nlev; J.axis = axis; J.apply_scale = axis == 2; J.scale = v.info.inv_mean_f;
        int64_t first = 0;
        for (int k = 0; k < nlev; ++k) {
            const int l = ord[k], ax = v.dims[l][0], ay = v.dims[l][1], az = v.dims[l][2];
            MipJob& b = J.j[k];
            b.w = dw + toff[k]; b.st = 1 << l; b.off = offs[k]; b.T = T[k];
            if (axis == 1) {
                b.in = A + aoff[k]; b.out = B + boff[k];
                b.ix = ax; b.iy = ny; b.iz = nz; b.ox = ax; b.oy = ay; b.oz = nz;
            } else {
                const int kk = (int)(std::find(levels, levels + nlev, l) - levels);
                b.in = B + boff[k]; b.out = dst[kk];
                b.ix = ax; b.iy = ay; b.iz = nz; b.ox = ax; b.oy = ay; b.oz = az;
            }
            b.first = first;
            first += (int64_t)b.ox * b.oy * b.oz;
        }
        J.total = first;
        k_mip_pass_multi<<<grid_for(J.total, 256, c.num_sms), 256, 0, s>>>(J);
    }
    RPNN_CHECK_LAUNCH();
    return RPNN_OK;
}

rpnn_status volume_build_level(Ctx& c, Volume& v, int level, float* dst, cudaStream_t s) {
    return volume_build_levels(c, v, &level, 1, &dst, s);
}

rpnn_status volume_pack_levels(Ctx& c, Volume& v, cudaStream_t s) {
    int64_t total = 0;
    bool need[kMaxLevels] = {};
    for (int k = 0; k < RPNN_K; ++k) {
        need[v.info.mip_of_level[k]] = true;
        if (v.info.mip_weight[k] > 0.0f) need[v.info.mip_of_level[k] + 1] = true;   // blended descriptor
    }
    for (int i = 0; i < v.levels; ++i) {
        v.level_packed[i] = need[i];
        v.lvl[i].ax = v.dims[i][0]; v.lvl[i].ay = v.dims[i][1]; v.lvl[i].az = v.dims[i][2];
        v.lvl[i].rec_offset = total;
        if (need[i]) total += (int64_t)(v.dims[i][0] + 1) * (v.dims[i][1] + 1) * (v.dims[i][2] + 1);
    }
    rpnn_status st = v.packed.reserve(total * 2 * sizeof(float4));
    if (st) return st;
    // the needed levels, built together, each into its own part of a volume-owned buffer
    int lv[kMaxLevels], nl = 0;
    int64_t doff[kMaxLevels], dsz = 0;
    for (int i = 0; i < v.levels; ++i) {
        if (!need[i]) continue;
        doff[nl] = dsz;
        dsz += ((int64_t)v.dims[i][0] * v.dims[i][1] * v.dims[i][2] + 15) / 16 * 16;
        lv[nl++] = i;
    }
    st = v.mip_d.reserve((size_t)std::max<int64_t>(dsz, 1) * sizeof(float));
    if (st) return st;
    float* dst[kMaxLevels];
    for (int k = 0; k < nl; ++k) dst[k] = v.mip_d.as<float>() + doff[k];
    st = volume_build_levels(c, v, lv, nl, dst, s);
    if (st) return st;
    for (int k = 0; k < nl; ++k) {
        const int i = lv[k];
        const int64_t nrec = (int64_t)(v.dims[i][0] + 1) * (v.dims[i][1] + 1) * (v.dims[i][2] + 1);
        k_pack<<<grid_for(nrec, 256, c.num_sms), 256, 0, s>>>(
            dst[k], v.packed.as<float4>() + 2 * v.lvl[i].rec_offset, v.dims[i][0], v.dims[i][1], v.dims[i][2]);
        RPNN_CHECK_LAUNCH();
    }
    RPNN_CUDA_TRY(cudaStreamSynchronize(s));
    v.built = true;
    v.stencil_ready = false;
    return RPNN_OK;
}

VolumeView Volume::view() const {
    VolumeView w{};
    w.raw = raw.as<float>();
    const int nmax = std::max(n[0], std::max(n[1], n[2]));
    for (int a = 0; a < 3; ++a) {
        w.n[a] = n[a];
        w.ext[a] = (float)((double)n[a] / (double)nmax);
    }
    w.inv_h0 = (float)nmax;
    w.majorant = info.majorant;
    w.albedo = albedo;
    w.g = g;
    w.inv_mean_f = info.inv_mean_f;
    for (int k = 0; k < RPNN_K; ++k) w.mip_of_level[k] = info.mip_of_level[k];
    w.packed = packed.as<float4>();
    for (int i = 0; i < kMaxLevels; ++i) w.lvl[i] = lvl[i];
    w.bmaj = bmaj.as<float>();
    for (int a = 0; a < 3; ++a) w.nb[a] = nb[a];
    w.bs = (float)((double)kBrick / (double)nmax);
    for (int k = 0; k < RPNN_K; ++k) w.mip_w[k] = mip_blend ? info.mip_weight[k] : 0.0f;
    w.track_cap = track_cap ? track_cap : kTrackCapDefault;
    w.lm = lm;
    w.lmc = lmc;
    w.dscale = dscale;
    w.albedo_c = albedo_c > 0.0f ? albedo_c : albedo;
    return w;
}

}  // namespace rpnn
