// phase.cu -- the cloud droplets' Lorenz-Mie phase function (Sec. 3.1), computed on the
// host and tabulated for the tracking kernels.
//
// The paper's tables are in its supplement, which is not available; the function here is
// the Mie series (Bohren & Huffman 1983, App. A) for water spheres (relative index 1.333,
// no absorption) at 0.55 um, weighted by Deirmendjian's cumulus C.1 size distribution
// n(r) ~ r^6 exp(-1.5 r) (r in um, 0.1 .. 16 um in steps of 0.1), and averaged over 1,800
// bins of 0.1 degree of scattering angle per unit solid angle (Simpson's rule on the bin's
// edges and midpoint).  The tracking kernels use that piecewise-constant function: they
// read a bin's value for next-event estimation and sample a bin by its cumulative
// probability, then cos(theta) uniformly inside it.
//
// The chopped form (after Bouthors et al. 2008, as Sec. 3.1 takes it) removes the
// diffraction peak, the bins below 5 degrees holding the fraction f of the scattered light,
// and renormalises the rest by 1 / (1 - f); the light scattered into the peak counts as
// not scattered, so the medium behind a path's first bounce has extinction (1 - f albedo)
// mu_t and albedo (1 - f) albedo / (1 - f albedo).
#include <cmath>
#include <complex>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace rpnn {

namespace {

using cplx = std::complex<double>;

// (|S1|^2 + |S2|^2) / 2 of one sphere of size parameter x at the cosines cs[]
void sphere_intensity(double x, cplx m, const std::vector<double>& cs, std::vector<double>& out) {
    const cplx y = m * x;
    const int terms = (int)(x + 4.0 * std::cbrt(x) + 2.0);
    const int start = (int)std::max((double)terms, std::abs(y)) + 16;
    // D_n(y) = psi_n'(y) / psi_n(y), recurred downwards from zero
    std::vector<cplx> D(start + 1, cplx(0.0, 0.0));
    for (int n = start; n >= 1; --n) D[n - 1] = (double)n / y - 1.0 / (D[n] + (double)n / y);
    const size_t na = cs.size();
    std::vector<cplx> s1(na), s2(na);
    std::vector<double> p_prev(na, 0.0), p_cur(na, 1.0);   // angular functions pi_{n-1}, pi_n
    // Riccati-Bessel psi, chi at orders n-2, n-1
    double psi_a = std::cos(x), psi_b = std::sin(x);
    double chi_a = -std::sin(x), chi_b = std::cos(x);
    for (int n = 1; n <= terms; ++n) {
        const double f = (double)(2 * n - 1) / x;
        const double psi_n = f * psi_b - psi_a;
        const double chi_n = f * chi_b - chi_a;
        const cplx xi_n(psi_n, -chi_n), xi_b(psi_b, -chi_b);
        const cplx ta = D[n] / m + (double)n / x;
        const cplx tb = m * D[n] + (double)n / x;
        const cplx a = (ta * psi_n - psi_b) / (ta * xi_n - xi_b);
        const cplx b = (tb * psi_n - psi_b) / (tb * xi_n - xi_b);
        const double w = (double)(2 * n + 1) / ((double)n * (n + 1));
        for (size_t k = 0; k < na; ++k) {
            const double pk = p_cur[k];
            const double tk = n * cs[k] * pk - (n + 1) * p_prev[k];
            s1[k] += w * (a * pk + b * tk);
            s2[k] += w * (a * tk + b * pk);
            const double nxt = ((double)(2 * n + 1) * cs[k] * pk - (double)(n + 1) * p_prev[k]) / (double)n;
            p_prev[k] = pk;
            p_cur[k] = nxt;
        }
        psi_a = psi_b; psi_b = psi_n;
        chi_a = chi_b; chi_b = chi_n;
    }
    out.resize(na);
    for (size_t k = 0; k < na; ++k) out[k] = 0.5 * (std::norm(s1[k]) + std::norm(s2[k]));
}

struct LmTable {
    std::vector<double> p, cdf, cosb;
    std::vector<double> pc, cdfc;   // chopped
    double f = 0.0;                 // fraction in the chopped peak
};

const LmTable& lm_table() {
    static LmTable T;
    static std::once_flag once;
    std::call_once(once, [] {
        const int N = RPNN_LM_BINS;
        const double pi = 3.14159265358979323846, dth = pi / N;
        std::vector<double> cs(2 * N + 1), sum(2 * N + 1, 0.0), one;
        for (int f = 0; f <= 2 * N; ++f) cs[f] = std::cos(0.5 * dth * f);
        const double k = 2.0 * pi / 0.55;
        for (int i = 1; i <= 160; ++i) {
            const double r = 0.1 * i;
            sphere_intensity(k * r, cplx(1.333, 0.0), cs, one);
            const double w = std::pow(r, 6.0) * std::exp(-1.5 * r);
            for (int f = 0; f <= 2 * N; ++f) sum[f] += w * one[f];
        }
        T.p.resize(N);
        T.cdf.assign(N + 1, 0.0);
        T.cosb.resize(N + 1);
        double norm = 0.0;
        for (int j = 0; j < N; ++j) {
            const double a = dth * j, m = a + 0.5 * dth, b = a + dth;
            const double area = (sum[2 * j] * std::sin(a) + 4.0 * sum[2 * j + 1] * std::sin(m) +
                                 sum[2 * j + 2] * std::sin(b)) * dth / 6.0;
            T.p[j] = area / (std::cos(a) - std::cos(b));
            norm += 2.0 * pi * area;
        }
        for (int j = 0; j < N; ++j) {
            T.p[j] /= norm;
            T.cosb[j] = std::cos(dth * j);
            T.cdf[j + 1] = T.cdf[j] + T.p[j] * 2.0 * pi * (std::cos(dth * j) - std::cos(dth * (j + 1)));
        }
        T.cosb[N] = -1.0;
        T.cdf[N] = 1.0;
        const int K = RPNN_LM_CHOP_BINS;
        T.f = T.cdf[K];
        T.pc.assign(N, 0.0);
        T.cdfc.assign(N + 1, 0.0);
        for (int j = K; j < N; ++j) {
            T.pc[j] = T.p[j] / (1.0 - T.f);
            T.cdfc[j + 1] = (T.cdf[j + 1] - T.f) / (1.0 - T.f);
        }
        T.cdfc[N] = 1.0;
    });
    return T;
}

// one table as floats [p (N) | cdf (N + 1) | cos edges (N + 1)]
std::vector<float> pack(const std::vector<double>& p, const std::vector<double>& cdf,
                        const std::vector<double>& cosb) {
    const int N = RPNN_LM_BINS;
    std::vector<float> h(3 * (size_t)N + 2);
    for (int j = 0; j < N; ++j) h[j] = (float)p[j];
    for (int j = 0; j <= N; ++j) {
        h[N + j] = (float)cdf[j];
        h[2 * N + 1 + j] = (float)cosb[j];
    }
    return h;
}

}  // namespace

double phase_lm_chop_fraction() { return lm_table().f; }

rpnn_status phase_lm_upload(Ctx& c, cudaStream_t s) {
    if (c.lm_table.p && c.lmc_table.p) return RPNN_OK;
    const LmTable& T = lm_table();
    const std::vector<float> full = pack(T.p, T.cdf, T.cosb), chopped = pack(T.pc, T.cdfc, T.cosb);
    const size_t bytes = full.size() * sizeof(float);
    rpnn_status st = c.lm_table.reserve(bytes);
    if (!st) st = c.lmc_table.reserve(bytes);
    if (st) return st;
    RPNN_CUDA_TRY(cudaMemcpyAsync(c.lm_table.p, full.data(), bytes, cudaMemcpyHostToDevice, s));
    RPNN_CUDA_TRY(cudaMemcpyAsync(c.lmc_table.p, chopped.data(), bytes, cudaMemcpyHostToDevice, s));
    RPNN_CUDA_TRY(cudaStreamSynchronize(s));
    return RPNN_OK;
}

}  // namespace rpnn

using namespace rpnn;

extern "C" rpnn_status rpnn_lorenz_mie_table(int32_t chopped, double* p, double* cdf, double* cos_edges,
                                              int32_t n, double* peak_fraction) {
    if (n != RPNN_LM_BINS) {
        set_error("the table has %d bins", RPNN_LM_BINS);
        return RPNN_ERR_ARG;
    }
    const LmTable& T = lm_table();
    const std::vector<double>& tp = chopped ? T.pc : T.p;
    const std::vector<double>& tc = chopped ? T.cdfc : T.cdf;
    for (int j = 0; j < n; ++j)
        if (p) p[j] = tp[j];
    for (int j = 0; j <= n; ++j) {
        if (cdf) cdf[j] = tc[j];
        if (cos_edges) cos_edges[j] = T.cosb[j];
    }
    if (peak_fraction) *peak_fraction = T.f;
    return RPNN_OK;
}
