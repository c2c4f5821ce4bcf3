"""CPU oracle for the RPNN hot path (TEST INFRASTRUCTURE ONLY).

A plain C implementation (``rpnn_oracle.c``) of what the GPU library computes,
written from Kallweit et al., "Deep Scattering" (Sec. 3.1 Lorenz-Mie phase function and its
chopped form, Sec. 3.2 Eq. 1, Sec. 4.2-4.4, Sec. 5, Sec. 6, Sec. 7's stencil sizes), wrapped
here with ctypes + numpy; the plain MLPs of the architecture
comparison (Sec. 7) and the environment superposition (Sec. 4.4) are written here in
numpy / Python directly.  Only ``tests/``, the smoke
check and the benchmark's ``cpu_baseline`` / reference leg may import this
package; the CUDA library never calls it and shares no code with it.

Pins (what fixes each function independently of itself) live in
``tests/test_oracle_*.py``.  Parity unpinned: the trained network as a whole
(only its per-layer arithmetic is pinned).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rpnn_oracle.c")
_HDR = os.path.join(_HERE, "rpnn_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liborc.so")
_lock = threading.Lock()
_lib = None

K, S, DIN, H = 10, 225, 226, 200
MAX_LEVELS = 16


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-ffp-contract=off keeps every FP32 op rounded
    on its own, as the FP32 restatements require)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Stats(C.Structure):
    _fields_ = [
        ("mean", C.c_double), ("mean_ld", C.c_double), ("inv_mean", C.c_double),
        ("inv_mean_f", C.c_float), ("majorant", C.c_float), ("nonzero", C.c_int64),
        ("levels", C.c_int), ("mip_of_level", C.c_int * K),
        ("dims", (C.c_int * 3) * MAX_LEVELS), ("h0", C.c_double), ("inv_h0", C.c_double),
        ("ext", C.c_double * 3), ("mip_weight", C.c_double * K), ("mip_weight_f", C.c_float * K),
    ]


class Camera(C.Structure):
    _fields_ = [
        ("cam_pos", C.c_double * 3), ("cam_fwd", C.c_double * 3),
        ("cam_right", C.c_double * 3), ("cam_up", C.c_double * 3),
        ("tan_half_fov_y", C.c_double), ("width", C.c_int), ("height", C.c_int),
        ("spp", C.c_int), ("seed", C.c_uint64), ("light_dir", C.c_double * 3),
        ("light_E", C.c_double),
    ]


class Net(C.Structure):
    _fields_ = [("K", C.c_int), ("din", C.c_int), ("H", C.c_int), ("ntail", C.c_int)]


_dp = C.POINTER(C.c_double)
_fp = C.POINTER(C.c_float)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.orc_create.restype = C.c_void_p
            L.orc_create.argtypes = [_fp, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double]
            L.orc_destroy.argtypes = [C.c_void_p]
            L.orc_get_stats.argtypes = [C.c_void_p, C.POINTER(Stats)]
            L.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32)] * 3
            L.orc_gauss_taps.argtypes = [C.c_int, _dp, C.c_int, C.POINTER(C.c_int)]
            L.orc_mip_level_f64.argtypes = [C.c_void_p, C.c_int, _dp]
            L.orc_mip_level_f32.argtypes = [C.c_void_p, C.c_int, _fp]
            L.orc_descriptor_f64.argtypes = [C.c_void_p, _dp, _dp, _dp, C.c_int64, _dp]
            L.orc_descriptor_f32.argtypes = [C.c_void_p, _fp, _fp, _fp, C.c_int64, _fp]
            L.orc_stencil_din.argtypes = [C.c_int]
            L.orc_descriptor_stencil_f64.argtypes = [C.c_void_p, C.c_int, _dp, _dp, _dp, C.c_int64, _dp]
            L.orc_descriptor_stencil_f32.argtypes = [C.c_void_p, C.c_int, _fp, _fp, _fp, C.c_int64, _fp]
            L.orc_frame_f64.argtypes = [_dp, _dp, _dp, _dp, _dp, _dp]
            L.orc_density.restype = C.c_double
            L.orc_density.argtypes = [C.c_void_p, _dp]
            L.orc_delta_track.argtypes = [C.c_void_p, _dp, _dp, C.c_uint64, C.c_uint32,
                                          C.c_uint32, C.c_uint32, C.POINTER(C.c_uint32),
                                          _dp, _dp]
            L.orc_ratio_track.restype = C.c_double
            L.orc_ratio_track.argtypes = [C.c_void_p, _dp, _dp, C.c_uint64, C.c_uint32,
                                          C.c_uint32, C.c_uint32, C.POINTER(C.c_uint32),
                                          C.POINTER(C.c_int)]
            for name in ("orc_delta_track_global",):
                getattr(L, name).argtypes = L.orc_delta_track.argtypes
            L.orc_ratio_track_global.restype = C.c_double
            L.orc_ratio_track_global.argtypes = L.orc_ratio_track.argtypes
            L.orc_mie_single.argtypes = [C.c_double, C.c_double, C.c_double, _dp, C.c_int, _dp,
                                         C.POINTER(C.c_double), C.POINTER(C.c_double)]
            L.orc_lm_table.argtypes = [_dp, _dp, _dp, C.c_int]
            L.orc_set_phase_lm.argtypes = [C.c_void_p, C.c_int]
            L.orc_set_phase_lm.restype = None
            L.orc_set_phase.argtypes = [C.c_void_p, C.c_int, C.c_int]
            L.orc_chop_params.argtypes = [C.c_void_p, _dp, _dp, _dp]
            L.orc_lm_chopped_table.argtypes = [C.c_void_p, _dp, _dp, C.c_int]
            L.orc_delta_track_global_scaled.argtypes = [C.c_void_p, _dp, _dp, C.c_double, C.c_uint64,
                                                        C.c_uint32, C.c_uint32, C.c_uint32,
                                                        C.POINTER(C.c_uint32), _dp, _dp]
            L.orc_ratio_track_scaled.restype = C.c_double
            L.orc_ratio_track_scaled.argtypes = [C.c_void_p, _dp, _dp, C.c_double, C.c_uint64, C.c_uint32,
                                                 C.c_uint32, C.c_uint32, C.POINTER(C.c_uint32),
                                                 C.POINTER(C.c_int)]
            L.orc_set_mip_blend.argtypes = [C.c_void_p, C.c_int]
            L.orc_set_mip_blend.restype = None
            L.orc_brick_majorant.restype = C.c_float
            L.orc_brick_majorant.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int]
            L.orc_hg.restype = C.c_double
            L.orc_hg.argtypes = [C.c_double, C.c_double]
            L.orc_primary.argtypes = [C.c_void_p, C.POINTER(Camera), C.c_int64, C.c_int,
                                      _dp, _dp, _dp]
            L.orc_render_pixels.argtypes = [C.c_void_p, C.POINTER(Camera), _dp, C.c_int,
                                            C.POINTER(C.c_int64), C.c_int64, _dp, C.c_int]
            L.orc_net_param_count.restype = C.c_int64
            L.orc_net_param_count.argtypes = [C.POINTER(Net)]
            L.orc_mlp_forward.argtypes = [C.POINTER(Net), _dp, _dp, C.c_int64, _dp]
            L.orc_mlp_backward.argtypes = [C.POINTER(Net), _dp, _dp, C.c_int64, _dp, _dp]
            L.orc_logmse_loss.restype = C.c_double
            L.orc_logmse_loss.argtypes = [_dp, _dp, C.c_int64, _dp]
            L.orc_adam.argtypes = [_dp, _dp, _dp, _dp, C.c_int64, C.c_int64, C.c_double,
                                   C.c_double, C.c_double, C.c_double]
            L.orc_gen_record.argtypes = [C.c_void_p, C.c_uint64, C.c_int64, C.c_double,
                                         C.c_int, C.c_int, _dp, _dp, _dp, _dp,
                                         C.POINTER(C.c_int64), _dp]
            L.orc_estimate_Li.argtypes = [C.c_void_p, C.c_uint64, C.c_uint32, _dp, _dp, _dp,
                                          C.c_int, C.c_int, _dp, _dp]
            L.orc_sample_hg.argtypes = [C.c_double, _dp, C.c_double, C.c_double, _dp]
            _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp)


def _f(a):
    return a.ctypes.data_as(_fp)


def _c64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a if shape is None else a.reshape(shape)


def _c32(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a if shape is None else a.reshape(shape)


def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def gauss_taps(level: int):
    cap = 7 if level == 0 else 6 << level
    w = np.zeros(cap, np.float64)
    off = C.c_int()
    n = lib().orc_gauss_taps(level, _d(w), cap, C.byref(off))
    return w[:n], off.value


def hg(g: float, cos_theta: float) -> float:
    return lib().orc_hg(g, cos_theta)


def sample_hg(g: float, d, xi0: float, xi1: float):
    d = _c64(d, (3,))
    out = np.zeros(3)
    lib().orc_sample_hg(g, _d(d), xi0, xi1, _d(out))
    return out


def frame(d, wl):
    d = _c64(d, (3,)); wl = _c64(wl, (3,))
    ex, ey, ez, gam = (np.zeros(3), np.zeros(3), np.zeros(3), np.zeros(1))
    lib().orc_frame_f64(_d(d), _d(wl), _d(ex), _d(ey), _d(ez), _d(gam))
    return ex, ey, ez, float(gam[0])


def net_param_count(K=10, din=226, H=200, ntail=3) -> int:
    n = Net(K, din, H, ntail)
    return int(lib().orc_net_param_count(C.byref(n)))


def stencil_din(n: int) -> int:
    """Block input width of the n x n x (2n - 1) stencil: n^2 (2n - 1) points and gamma."""
    din = int(lib().orc_stencil_din(int(n)))
    if din < 0:
        raise ValueError(f"stencil resolution {n} outside [2, 9]")
    return din


def mlp_forward(params, z, K=10, din=226, H=200, ntail=3):
    n = Net(K, din, H, ntail)
    params = _c64(params)
    z = _c64(z)
    q = z.size // (K * din)
    g = np.zeros(q, np.float64)
    r = lib().orc_mlp_forward(C.byref(n), _d(params), _d(z), q, _d(g))
    assert r == 0
    return g


def mlp_backward(params, z, dg, K=10, din=226, H=200, ntail=3):
    n = Net(K, din, H, ntail)
    params = _c64(params)
    z = _c64(z)
    dg = _c64(dg)
    q = z.size // (K * din)
    dp = np.zeros_like(params)
    r = lib().orc_mlp_backward(C.byref(n), _d(params), _d(z), q, _d(dg), _d(dp))
    assert r == 0
    return dp


def logmse_loss(g, target, want_grad=True):
    g = _c64(g); t = _c64(target)
    dg = np.zeros_like(g)
    l = lib().orc_logmse_loss(_d(g), _d(t), g.size, _d(dg) if want_grad else None)
    return (l, dg) if want_grad else l


def adam(p, m, v, grad, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """In-place Adam on float64 arrays."""
    for a in (p, m, v, grad):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lib().orc_adam(_d(p), _d(m), _d(v), _d(grad), p.size, t, lr, b1, b2, eps)


def dense_forward(params, widths, x):
    """Plain ("all-at-once") MLP of the architecture comparison (Sec. 7, Fig. 10) in FP64:
    h_i = relu(W_i h_{i-1} + b_i) with h_{-1} = x (rows), g = relu(w_o h_last + b_o).
    Parameters flat: per hidden layer W_i [w_i][w_{i-1}] row-major then b_i, then w_o, b_o.
    Returns (g [q], [h_0, ..., h_{n-1}])."""
    p = np.asarray(params, np.float64)
    h = np.asarray(x, np.float64).reshape(len(x), -1)
    acts, o = [], 0
    for w in widths:
        W = p[o:o + w * h.shape[1]].reshape(w, h.shape[1]); o += w * h.shape[1]
        b = p[o:o + w]; o += w
        h = np.maximum(h @ W.T + b, 0.0)
        acts.append(h)
    wo = p[o:o + h.shape[1]]; o += h.shape[1]
    g = np.maximum(h @ wo + p[o], 0.0)
    assert o + 1 == p.size
    return g, acts


def dense_backward(params, widths, x, dout):
    """Gradient of sum_i dout_i g_i with respect to the flat parameters (chain rule, FP64)."""
    p = np.asarray(params, np.float64)
    xin = np.asarray(x, np.float64).reshape(len(x), -1)
    g, acts = dense_forward(p, widths, xin)
    grad = np.zeros_like(p)
    offs, o, prev = [], 0, xin.shape[1]
    for w in widths:
        offs.append((o, prev, w)); o += w * prev + w; prev = w
    da = np.asarray(dout, np.float64) * (g > 0)
    hl = acts[-1] if acts else xin
    grad[o:o + prev] = da @ hl
    grad[o + prev] = da.sum()
    dh = np.outer(da, p[o:o + prev]) * (hl > 0)
    for i in range(len(widths) - 1, -1, -1):
        oi, pw, w = offs[i]
        xi = acts[i - 1] if i else xin
        grad[oi:oi + w * pw] = (dh.T @ xi).ravel()
        grad[oi + w * pw:oi + w * pw + w] = dh.sum(axis=0)
        if i:
            W = p[oi:oi + w * pw].reshape(w, pw)
            dh = (dh @ W) * (acts[i - 1] > 0)
    return grad


LM_BINS = 1800
LM_CHOP_BINS = 50       # the chopped diffraction peak: scattering angles below 5 degrees


def mie_single(x, m_re, m_im, mu):
    """Lorenz-Mie of one sphere: (s11 at cosines mu, Q_ext, Q_sca)."""
    mu = _c64(mu)
    out = np.zeros(mu.size)
    qe, qs = C.c_double(), C.c_double()
    assert lib().orc_mie_single(float(x), float(m_re), float(m_im), _d(mu), mu.size, _d(out),
                                C.byref(qe), C.byref(qs)) == 0
    return out, qe.value, qs.value


def lm_table():
    """The tabulated cloud phase function: (bin means p, cumulative cdf, bin-edge cosines)."""
    p, cdf, ce = np.zeros(LM_BINS), np.zeros(LM_BINS + 1), np.zeros(LM_BINS + 1)
    assert lib().orc_lm_table(_d(p), _d(cdf), _d(ce), LM_BINS) == 0
    return p, cdf, ce


def make_camera(cam: dict) -> Camera:
    c = Camera()
    for k in ("cam_pos", "cam_fwd", "cam_right", "cam_up", "light_dir"):
        arr = getattr(c, k)
        for i in range(3):
            arr[i] = float(cam[k][i])
    c.tan_half_fov_y = float(cam["tan_half_fov_y"])
    c.width, c.height, c.spp = int(cam["width"]), int(cam["height"]), int(cam["spp"])
    c.seed = int(cam["seed"])
    c.light_E = float(cam.get("light_E", 1.0))
    return c


class Volume:
    """One cloud: density grid (x fastest, [nz][ny][nx]), albedo, HG g."""

    def __init__(self, density, albedo=0.99, g=0.85):
        d = _c32(density)
        assert d.ndim == 3
        nz, ny, nx = d.shape
        self._keep = d
        self.shape = d.shape
        self.albedo, self.g = float(albedo), float(g)
        self.h = lib().orc_create(_f(d), nx, ny, nz, self.albedo, self.g)
        if not self.h:
            raise ValueError("oracle rejected the volume (negative/non-finite or all zero)")

    def close(self):
        if self.h:
            lib().orc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def stats(self) -> dict:
        s = Stats()
        lib().orc_get_stats(self.h, C.byref(s))
        return {
            "mean": s.mean, "mean_ld": s.mean_ld, "inv_mean": s.inv_mean,
            "inv_mean_f": s.inv_mean_f, "majorant": s.majorant, "nonzero": s.nonzero,
            "levels": s.levels, "mip_of_level": list(s.mip_of_level),
            "dims": [tuple(s.dims[i]) for i in range(s.levels)],
            "h0": s.h0, "inv_h0": s.inv_h0, "ext": tuple(s.ext),
            "mip_weight": list(s.mip_weight), "mip_weight_f": list(s.mip_weight_f),
        }

    def set_phase_lm(self, on: bool):
        """Tabulated Lorenz-Mie phase function instead of Henyey-Greenstein."""
        lib().orc_set_phase_lm(self.h, 1 if on else 0)

    def set_phase(self, kind: int, chop_bins: int = LM_CHOP_BINS):
        """0 HG, 1 Lorenz-Mie, 2 Lorenz-Mie at the first bounce and chopped (first chop_bins
        bins removed) in the thinner medium after it."""
        assert lib().orc_set_phase(self.h, int(kind), int(chop_bins)) == 0

    def chop_params(self):
        """(peak fraction f, extinction scale, albedo) after the first bounce."""
        f, s, a = C.c_double(), C.c_double(), C.c_double()
        assert lib().orc_chop_params(self.h, C.byref(f), C.byref(s), C.byref(a)) == 0
        return f.value, s.value, a.value

    def lm_chopped_table(self):
        p, cdf = np.zeros(LM_BINS), np.zeros(LM_BINS + 1)
        assert lib().orc_lm_chopped_table(self.h, _d(p), _d(cdf), LM_BINS) == 0
        return p, cdf

    def set_mip_blend(self, on: bool):
        """Blended (fractional) mip selection for descriptors (off by default)."""
        lib().orc_set_mip_blend(self.h, 1 if on else 0)

    def mip_level(self, level: int, f32: bool = False):
        st = self.stats()
        ax, ay, az = st["dims"][level]
        if f32:
            out = np.zeros((az, ay, ax), np.float32)
            r = lib().orc_mip_level_f32(self.h, level, _f(out))
        else:
            out = np.zeros((az, ay, ax), np.float64)
            r = lib().orc_mip_level_f64(self.h, level, _d(out))
        assert r == 0
        return out

    def density(self, p) -> float:
        p = _c64(p, (3,))
        return lib().orc_density(self.h, _d(p))

    def descriptor(self, x, d, wl, f32: bool = False):
        if f32:
            x = _c32(x, (-1, 3)); d = _c32(d, (-1, 3)); wl = _c32(wl, (3,))
            q = x.shape[0]
            out = np.zeros((q, K, DIN), np.float32)
            r = lib().orc_descriptor_f32(self.h, _f(x), _f(d), _f(wl), q, _f(out))
        else:
            x = _c64(x, (-1, 3)); d = _c64(d, (-1, 3)); wl = _c64(wl, (3,))
            q = x.shape[0]
            out = np.zeros((q, K, DIN), np.float64)
            r = lib().orc_descriptor_f64(self.h, _d(x), _d(d), _d(wl), q, _d(out))
        assert r == 0
        return out

    def descriptor_stencil(self, n, x, d, wl, f32: bool = False):
        """Descriptor of the n x n x (2n - 1) stencil (stencil-size comparison): [q][K][din]."""
        din = stencil_din(n)
        if f32:
            x = _c32(x, (-1, 3)); d = _c32(d, (-1, 3)); wl = _c32(wl, (3,))
            q = x.shape[0]
            out = np.zeros((q, K, din), np.float32)
            r = lib().orc_descriptor_stencil_f32(self.h, n, _f(x), _f(d), _f(wl), q, _f(out))
        else:
            x = _c64(x, (-1, 3)); d = _c64(d, (-1, 3)); wl = _c64(wl, (3,))
            q = x.shape[0]
            out = np.zeros((q, K, din), np.float64)
            r = lib().orc_descriptor_stencil_f64(self.h, n, _d(x), _d(d), _d(wl), q, _d(out))
        assert r == 0
        return out

    def delta_track(self, o, d, seed, id0, id1, domain=2, global_majorant=False, scale=None):
        """Delta tracking over the brick majorants (global_majorant: against the single
        global majorant, the estimator the brick form must agree with in distribution;
        scale: against the global majorant in a medium of extinction scale * mu_t)."""
        o = _c64(o, (3,)); d = _c64(d, (3,))
        x = np.zeros(3); t = np.zeros(1)
        ctr = C.c_uint32(0)
        if scale is not None:
            r = lib().orc_delta_track_global_scaled(self.h, _d(o), _d(d), float(scale), seed, id0, id1,
                                                    domain, C.byref(ctr), _d(x), _d(t))
            return r, x, float(t[0])
        fn = lib().orc_delta_track_global if global_majorant else lib().orc_delta_track
        r = fn(self.h, _d(o), _d(d), seed, id0, id1, domain, C.byref(ctr), _d(x), _d(t))
        return r, x, float(t[0])

    def ratio_track(self, o, d, seed, id0, id1, domain=3, global_majorant=False, scale=None):
        o = _c64(o, (3,)); d = _c64(d, (3,))
        ctr = C.c_uint32(0)
        capped = C.c_int(0)
        if scale is not None:
            return lib().orc_ratio_track_scaled(self.h, _d(o), _d(d), float(scale), seed, id0, id1, domain,
                                                C.byref(ctr), C.byref(capped))
        fn = lib().orc_ratio_track_global if global_majorant else lib().orc_ratio_track
        T = fn(self.h, _d(o), _d(d), seed, id0, id1, domain, C.byref(ctr), C.byref(capped))
        return T

    def brick_majorants(self):
        """Per-brick majorant grid [nbz][nby][nbx] (bricks of 8^3 voxels)."""
        nz, ny, nx = self.shape
        nb = [(n + 7) // 8 for n in (nx, ny, nz)]
        out = np.zeros((nb[2], nb[1], nb[0]), np.float32)
        for z in range(nb[2]):
            for y in range(nb[1]):
                for x in range(nb[0]):
                    out[z, y, x] = lib().orc_brick_majorant(self.h, x, y, z)
        return out

    def primary(self, cam: dict, pixel: int, sample: int):
        c = make_camera(cam)
        x = np.zeros(3); d = np.zeros(3); Ld = np.zeros(1)
        hit = lib().orc_primary(self.h, C.byref(c), pixel, sample, _d(x), _d(d), _d(Ld))
        return hit, x, d, float(Ld[0])

    def render_pixels(self, cam: dict, pixels, params=None, mode=0, nthreads=None):
        c = make_camera(cam)
        pix = np.ascontiguousarray(pixels, dtype=np.int64)
        out = np.zeros(pix.size, np.float64)
        p = None if params is None else _c64(params)
        nt = nthreads or os.cpu_count() or 1
        r = lib().orc_render_pixels(self.h, C.byref(c), None if p is None else _d(p), mode,
                                    pix.ctypes.data_as(C.POINTER(C.c_int64)), pix.size,
                                    _d(out), nt)
        if r != 0:
            raise RuntimeError(f"oracle render failed ({r})")
        return out

    def render_pixels_env(self, cam: dict, pixels, dirs, irradiance, params=None, mode=0, nthreads=None):
        """Environment lighting (Sec. 4.4): the distant emitter is a set of directional
        lights (dirs[j] towards the light, irradiance E_j), and a pixel sums each light's
        direct in-scattering and predicted indirect in-scattering over the lights.  The
        visible point does not depend on the light and each light's shadow ray draws the
        same stream, so the sum is taken over single-light renders, in light order."""
        out = None
        for w, e in zip(np.asarray(dirs, np.float64), np.asarray(irradiance, np.float64)):
            cj = dict(cam, light_dir=tuple(float(v) for v in w), light_E=float(e))
            r = self.render_pixels(cj, pixels, params=params, mode=mode, nthreads=nthreads)
            out = r if out is None else out + r
        return out

    def gen_record(self, seed, rec, rel_ci=0.02, n_min=64, n_max=65536):
        x = np.zeros(3); d = np.zeros(3); wl = np.zeros(3); lab = np.zeros(1); hw = np.zeros(1)
        n = C.c_int64(0)
        r = lib().orc_gen_record(self.h, seed, rec, rel_ci, n_min, n_max, _d(x), _d(d), _d(wl),
                                 _d(lab), C.byref(n), _d(hw))
        return {"status": r, "x": x, "d": d, "wl": wl, "label": float(lab[0]),
                "npaths": int(n.value), "half_width": float(hw[0])}

    def estimate_Li(self, seed, rec, x, d, wl, npaths, max_bounces=0):
        x = _c64(x, (3,)); d = _c64(d, (3,)); wl = _c64(wl, (3,))
        m = np.zeros(1); v = np.zeros(1)
        r = lib().orc_estimate_Li(self.h, seed, rec, _d(x), _d(d), _d(wl), npaths, max_bounces,
                                  _d(m), _d(v))
        return r, float(m[0]), float(v[0])
