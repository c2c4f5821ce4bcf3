"""Thin ctypes binding of the C ABI in ``include/rpnn.h``.

Argument marshalling only: every step runs in the CUDA library.  Tensors are
PyTorch CUDA tensors (device memory and streams are PyTorch's); their data
pointers and the current stream are passed straight through.  The methods of
``Context`` carry the C entry points' names without the ``rpnn_`` prefix.
Importing this module does not load the library; creating a ``Context`` does,
and raises if it has not been built or no GPU is present.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import torch

from . import build as _build

K, S, DIN, DESC_STRIDE, H, NPARAMS = 10, 225, 226, 240, 200, 1296601
DESC_STRIDE_FP8 = 256
F32, F16, BF16, FP8 = 0, 1, 2, 3
MODE_RPNN, MODE_SINGLE, MODE_PATH = 0, 1, 2
ERR_NAMES = {0: "OK", -1: "ERR_ARG", -2: "ERR_HANDLE", -3: "ERR_CUDA", -4: "ERR_OOM",
             -5: "ERR_ITER_LIMIT", -6: "ERR_NONFINITE", -7: "ERR_STATE", -8: "ERR_UNSUPPORTED",
             -9: "ERR_TIMEOUT"}


PHASE_HG, PHASE_LORENZ_MIE, PHASE_LORENZ_MIE_CHOPPED = 0, 1, 2
LM_BINS, LM_CHOP_BINS = 1800, 50


class RPNNError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


class RenderDesc(C.Structure):
    _fields_ = [("cam_pos", C.c_float * 3), ("cam_fwd", C.c_float * 3),
                ("cam_right", C.c_float * 3), ("cam_up", C.c_float * 3),
                ("tan_half_fov_y", C.c_float), ("width", C.c_int32), ("height", C.c_int32),
                ("spp", C.c_int32), ("seed", C.c_uint64), ("light_dir", C.c_float * 3),
                ("light_E", C.c_float), ("precision", C.c_int32), ("mode", C.c_int32)]


class BatchItem(C.Structure):
    _fields_ = [("vol", C.c_int32), ("desc", RenderDesc), ("dev_image", C.c_void_p)]


class VolumeInfo(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("levels", C.c_int32), ("dims", (C.c_int32 * 3) * 16),
                ("mip_of_level", C.c_int32 * K), ("mean", C.c_double),
                ("inv_mean_f", C.c_float), ("majorant", C.c_float), ("nonzero", C.c_int64),
                ("bricks", C.c_int32 * 3), ("mip_weight", C.c_float * K)]


class TuneEntry(C.Structure):
    _fields_ = [("M", C.c_int32), ("N", C.c_int32), ("K0", C.c_int32), ("K1", C.c_int32),
                ("flags", C.c_int32), ("tile_m", C.c_int32), ("tile_n", C.c_int32),
                ("tile_k", C.c_int32), ("splits", C.c_int32), ("us", C.c_float),
                ("default_us", C.c_float)]


class AdamCfg(C.Structure):
    _fields_ = [("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float)]


_lib = None
_lock = threading.Lock()
_vp = C.c_void_p


def lib_path() -> str:
    return _build.LIB


def load():
    """Loads the built library (after PyTorch has initialised CUDA, so both share one
    runtime).  Raises when the library is missing or no CUDA device is visible."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the RPNN library runs on the GPU only")
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"CUDA library not built ({_build.LIB}); run build()")
        torch.cuda.init()
        L = C.CDLL(_build.LIB)
        i32, i64, u64, f32 = C.c_int32, C.c_int64, C.c_uint64, C.c_float
        sig = {
            "rpnn_create": [C.POINTER(_vp)],
            "rpnn_destroy": [_vp],
            "rpnn_sync_status": [_vp, _vp],
            "rpnn_load_volume": [_vp, _vp, i32, i32, i32, i32, f32, f32, C.POINTER(i32), _vp],
            "rpnn_build_mips": [_vp, i32, _vp],
            "rpnn_get_volume_info": [_vp, i32, C.POINTER(VolumeInfo)],
            "rpnn_copy_mip_level": [_vp, i32, i32, _vp, _vp],
            "rpnn_copy_brick_majorants": [_vp, i32, _vp, _vp],
            "rpnn_set_mip_blend": [_vp, i32, i32],
            "rpnn_set_iteration_cap": [_vp, i32, i64],
            "rpnn_set_phase_function": [_vp, i32, i32],
            "rpnn_stencil_descriptors": [_vp, i32, i32, _vp, _vp, _vp, i32, i64, _vp, _vp],
            "rpnn_stencil_forward": [_vp, i32, _vp, _vp, i64, _vp, _vp],
            "rpnn_stencil_backward": [_vp, i32, _vp, _vp, i64, _vp, _vp, _vp],
            "rpnn_stencil_train_step": [_vp, i32, _vp, _vp, i32, C.POINTER(AdamCfg), i64, _vp, _vp, _vp, _vp,
                                        _vp],
            "rpnn_set_autotune_table": [_vp, C.POINTER(TuneEntry), i32],
            "rpnn_dense_forward": [_vp, C.POINTER(i32), i32, i32, _vp, _vp, i64, _vp, _vp],
            "rpnn_dense_backward": [_vp, C.POINTER(i32), i32, i32, _vp, _vp, i64, _vp, _vp, _vp],
            "rpnn_dense_train_step": [_vp, C.POINTER(i32), i32, i32, _vp, _vp, i32, C.POINTER(AdamCfg),
                                      i64, _vp, _vp, _vp, _vp, _vp],
            "rpnn_set_weights": [_vp, _vp, i64, _vp],
            "rpnn_extract_descriptors": [_vp, i32, _vp, _vp, _vp, i32, i64, _vp, i32, _vp],
            "rpnn_mlp_forward": [_vp, _vp, i32, i64, i32, _vp, _vp],
            "rpnn_render": [_vp, i32, C.POINTER(RenderDesc), _vp, C.POINTER(i64), _vp],
            "rpnn_render_batch": [_vp, C.POINTER(BatchItem), i32, C.POINTER(i64), _vp],
            "rpnn_render_env": [_vp, i32, C.POINTER(RenderDesc), C.POINTER(f32), C.POINTER(f32), i32, _vp,
                                C.POINTER(i64), _vp],
            "rpnn_set_render_chunk": [_vp, i64],
            "rpnn_set_fused": [_vp, i32],
            "rpnn_set_train_graphs": [_vp, i32],
            "rpnn_calibrate_fp8": [_vp, _vp, i64, _vp],
            "rpnn_trace_primary": [_vp, i32, C.POINTER(RenderDesc), _vp, _vp, _vp, _vp, _vp],
            "rpnn_gen_records": [_vp, i32, i64, i64, u64, f32, i32, i32, _vp, _vp, _vp, _vp,
                                 _vp, _vp],
            "rpnn_mlp_backward": [_vp, _vp, i32, i64, _vp, _vp, _vp],
            "rpnn_train_step": [_vp, _vp, i32, _vp, i32, C.POINTER(AdamCfg), i64, _vp, _vp, _vp,
                                _vp, _vp],
            "rpnn_set_profiling": [_vp, i32],
            "rpnn_set_autotune": [_vp, i32],
            "rpnn_set_train_precision": [_vp, i32],
            "rpnn_get_autotune": [_vp, C.POINTER(TuneEntry), i32, C.POINTER(i32)],
            "rpnn_read_profile": [_vp, C.POINTER(C.c_double), C.POINTER(i64)],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = C.c_int32
        L.rpnn_stencil_param_count.restype = C.c_int64
        L.rpnn_stencil_param_count.argtypes = [C.c_int32]
        L.rpnn_dense_param_count.restype = C.c_int64
        L.rpnn_dense_param_count.argtypes = [C.POINTER(C.c_int32), C.c_int32, C.c_int32]
        L.rpnn_last_error.restype = C.c_char_p
        L.rpnn_last_error.argtypes = []
        _lib = L
        return L


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dtype_code(t):
    if t.dtype == torch.uint8:
        return FP8                          # E4M3 bytes
    return {torch.float32: F32, torch.float16: F16, torch.bfloat16: BF16}[t.dtype]


class Context:
    """One rpnn_ctx bound to the current CUDA device."""

    train_precision = F32

    def __init__(self):
        self.L = load()
        h = C.c_void_p()
        self._check(self.L.rpnn_create(C.byref(h)))
        self.h = h

    def _check(self, rc):
        if rc != 0:
            raise RPNNError(rc, self.L.rpnn_last_error().decode())
        return rc

    def close(self):
        if getattr(self, "h", None):
            self.L.rpnn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- volume ---------------------------------------------------------------------
    def load_volume(self, density: torch.Tensor, albedo=0.99, hg_g=0.85) -> int:
        assert density.dim() == 3
        nz, ny, nx = density.shape
        vid = C.c_int32()
        self._check(self.L.rpnn_load_volume(self.h, _ptr(density), _dtype_code(density), nx, ny,
                                            nz, albedo, hg_g, C.byref(vid), _stream()))
        return vid.value

    def build_mips(self, vol: int):
        self._check(self.L.rpnn_build_mips(self.h, vol, _stream()))

    def get_volume_info(self, vol: int) -> dict:
        i = VolumeInfo()
        self._check(self.L.rpnn_get_volume_info(self.h, vol, C.byref(i)))
        return {"n": tuple(i.n), "levels": i.levels,
                "dims": [tuple(i.dims[k]) for k in range(i.levels)],
                "mip_of_level": list(i.mip_of_level), "mean": i.mean,
                "inv_mean_f": i.inv_mean_f, "majorant": i.majorant, "nonzero": i.nonzero,
                "bricks": tuple(i.bricks), "mip_weight": list(i.mip_weight)}

    def copy_mip_level(self, vol: int, level: int) -> torch.Tensor:
        info = self.get_volume_info(vol)
        ax, ay, az = info["dims"][level]
        out = torch.empty((az, ay, ax), dtype=torch.float32, device="cuda")
        self._check(self.L.rpnn_copy_mip_level(self.h, vol, level, _ptr(out), _stream()))
        return out

    def set_mip_blend(self, vol: int, on: bool):
        """Blended (fractional) mip selection for the volume's descriptors."""
        self._check(self.L.rpnn_set_mip_blend(self.h, vol, 1 if on else 0))

    def copy_brick_majorants(self, vol: int) -> torch.Tensor:
        nb = self.get_volume_info(vol)["bricks"]
        out = torch.empty((nb[2], nb[1], nb[0]), dtype=torch.float32, device="cuda")
        self._check(self.L.rpnn_copy_brick_majorants(self.h, vol, _ptr(out), _stream()))
        return out

    def sync_status(self):
        self._check(self.L.rpnn_sync_status(self.h, _stream()))

    STAGES = ("primary", "descriptor", "network", "composite")

    def set_profiling(self, on: bool):
        self._check(self.L.rpnn_set_profiling(self.h, 1 if on else 0))

    # -- plain ("all-at-once") MLP of the architecture comparison (Sec. 7) -----------
    @staticmethod
    def _widths(widths):
        w = (C.c_int32 * max(1, len(widths)))(*[int(x) for x in widths])
        return w, len(widths)

    def dense_param_count(self, widths, din):
        w, n = self._widths(widths)
        return int(self.L.rpnn_dense_param_count(w, n, din))

    def dense_forward(self, widths, params, x, out=None):
        w, n = self._widths(widths)
        q, din = x.shape[0], x[0].numel()
        if out is None:
            out = torch.empty(q, dtype=torch.float32, device="cuda")
        self._check(self.L.rpnn_dense_forward(self.h, w, n, din, _ptr(params), _ptr(x), q, _ptr(out), _stream()))
        return out

    def dense_backward(self, widths, params, x, dout, out=None):
        w, n = self._widths(widths)
        q, din = x.shape[0], x[0].numel()
        if out is None:
            out = torch.empty(params.numel(), dtype=torch.float32, device="cuda")
        self._check(self.L.rpnn_dense_backward(self.h, w, n, din, _ptr(params), _ptr(x), q, _ptr(dout), _ptr(out),
                                               _stream()))
        return out

    def dense_train_step(self, widths, x, target, params, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999,
                         eps=1e-8, loss=None):
        w, n = self._widths(widths)
        if loss is None:
            loss = torch.empty(1, dtype=torch.float64, device="cuda")
        cfg = AdamCfg(lr, beta1, beta2, eps)
        self._check(self.L.rpnn_dense_train_step(self.h, w, n, x[0].numel(), _ptr(x), _ptr(target), x.shape[0],
                                                 C.byref(cfg), step, _ptr(params), _ptr(m), _ptr(v), _ptr(loss),
                                                 _stream()))
        return loss

    # ---- stencil-size comparison (Sec. 7, Fig. 10 right)
    def stencil_param_count(self, n_xy: int) -> int:
        return int(self.L.rpnn_stencil_param_count(n_xy))

    def stencil_descriptors(self, vol, n_xy, x, d, wl, out=None):
        """FP32 rows [q][10][n_xy^2 (2 n_xy - 1) + 1] of the n_xy x n_xy x (2 n_xy - 1) stencil."""
        q = x.shape[0]
        stride = 3 if wl.dim() == 2 else 0
        if out is None:
            out = torch.empty((q, K, n_xy * n_xy * (2 * n_xy - 1) + 1), dtype=torch.float32, device="cuda")
        self._check(self.L.rpnn_stencil_descriptors(self.h, vol, n_xy, _ptr(x), _ptr(d), _ptr(wl), stride, q,
                                                    _ptr(out), _stream()))
        return out

    def stencil_forward(self, n_xy, params, desc, out=None):
        q = desc.shape[0]
        if out is None:
            out = torch.empty(q, dtype=torch.float32, device="cuda")
        self._check(self.L.rpnn_stencil_forward(self.h, n_xy, _ptr(params), _ptr(desc), q, _ptr(out), _stream()))
        return out

    def stencil_backward(self, n_xy, params, desc, dout, out=None):
        if out is None:
            out = torch.empty(params.numel(), dtype=torch.float32, device="cuda")
        self._check(self.L.rpnn_stencil_backward(self.h, n_xy, _ptr(params), _ptr(desc), desc.shape[0], _ptr(dout),
                                                 _ptr(out), _stream()))
        return out

    def stencil_train_step(self, n_xy, desc, target, params, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999,
                           eps=1e-8, loss=None):
        if loss is None:
            loss = torch.empty(1, dtype=torch.float64, device="cuda")
        cfg = AdamCfg(lr, beta1, beta2, eps)
        self._check(self.L.rpnn_stencil_train_step(self.h, n_xy, _ptr(desc), _ptr(target), desc.shape[0],
                                                   C.byref(cfg), step, _ptr(params), _ptr(m), _ptr(v), _ptr(loss),
                                                   _stream()))
        return loss

    def set_train_precision(self, precision):
        """F32 (default) or BF16 arithmetic for train_step and mlp_backward."""
        self._check(self.L.rpnn_set_train_precision(self.h, precision))
        self.train_precision = precision

    def set_autotune(self, on: bool):
        self._check(self.L.rpnn_set_autotune(self.h, 1 if on else 0))

    def set_autotune_table(self, table: list):
        """Restores tuning decisions written by autotune_table() (e.g. from a checkpoint)."""
        buf = (TuneEntry * max(1, len(table)))()
        for i, e in enumerate(table):
            for f, _ in TuneEntry._fields_:
                setattr(buf[i], f, e[f])
        self._check(self.L.rpnn_set_autotune_table(self.h, buf, len(table)))

    def set_phase_function(self, vol: int, kind: int):
        """PHASE_HG (default), PHASE_LORENZ_MIE (the tabulated cloud-droplet function) or
        PHASE_LORENZ_MIE_CHOPPED (full at a path's first bounce, chopped after it in the
        correspondingly thinner medium)."""
        self._check(self.L.rpnn_set_phase_function(self.h, vol, int(kind)))

    def set_iteration_cap(self, vol: int, cap: int):
        """Tentative collisions per tracking call through the volume (0: the default)."""
        self._check(self.L.rpnn_set_iteration_cap(self.h, vol, int(cap)))

    def autotune_table(self) -> list:
        """The GEMM-tile choices made so far, one dict per shape."""
        n = C.c_int32()
        self._check(self.L.rpnn_get_autotune(self.h, None, 0, C.byref(n)))
        buf = (TuneEntry * max(1, n.value))()
        self._check(self.L.rpnn_get_autotune(self.h, buf, n.value, C.byref(n)))
        return [{f: getattr(buf[i], f) for f, _ in TuneEntry._fields_} for i in range(n.value)]

    def read_profile(self) -> dict:
        ms = (C.c_double * 4)()
        n = C.c_int64()
        self._check(self.L.rpnn_read_profile(self.h, ms, C.byref(n)))
        out = {k: ms[i] for i, k in enumerate(self.STAGES)}
        out["renders"] = n.value
        return out

    # -- network ----------------------------------------------------------------------
    def set_weights(self, params: torch.Tensor):
        assert params.dtype == torch.float32 and params.numel() == NPARAMS
        self._check(self.L.rpnn_set_weights(self.h, _ptr(params), params.numel(), _stream()))

    def extract_descriptors(self, vol, x, d, wl, dtype=torch.float32, out=None):
        """dtype torch.uint8 selects E4M3 rows [q][10][256] (bytes)."""
        q = x.shape[0]
        stride = 3 if wl.dim() == 2 else 0
        if out is None:
            width = DESC_STRIDE_FP8 if dtype == torch.uint8 else DESC_STRIDE
            out = torch.empty((q, K, width), dtype=dtype, device="cuda")
        self._check(self.L.rpnn_extract_descriptors(self.h, vol, _ptr(x), _ptr(d), _ptr(wl),
                                                    stride, q, _ptr(out), _dtype_code(out),
                                                    _stream()))
        return out

    def mlp_forward(self, desc, precision=F32, out=None):
        q = desc.shape[0]
        if out is None:
            out = torch.empty(q, dtype=torch.float32, device="cuda")
        self._check(self.L.rpnn_mlp_forward(self.h, _ptr(desc), _dtype_code(desc), q, precision,
                                            _ptr(out), _stream()))
        return out

    def calibrate_fp8(self, desc):
        """Per-tensor FP8 scales from the FP32 network on these FP32 descriptors."""
        assert desc.dtype == torch.float32
        self._check(self.L.rpnn_calibrate_fp8(self.h, _ptr(desc), desc.shape[0], _stream()))

    def mlp_backward(self, desc, dout, out=None):
        q = desc.shape[0]
        if out is None:
            out = torch.empty(NPARAMS, dtype=torch.float32, device="cuda")
        self._check(self.L.rpnn_mlp_backward(self.h, _ptr(desc), _dtype_code(desc), q, _ptr(dout), _ptr(out),
                                             _stream()))
        return out

    def train_step(self, desc, target, params, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999,
                   eps=1e-8, loss=None):
        if loss is None:
            loss = torch.empty(1, dtype=torch.float64, device="cuda")
        cfg = AdamCfg(lr, beta1, beta2, eps)
        self._check(self.L.rpnn_train_step(self.h, _ptr(desc), _dtype_code(desc), _ptr(target), desc.shape[0],
                                           C.byref(cfg), step, _ptr(params), _ptr(m), _ptr(v),
                                           _ptr(loss), _stream()))
        return loss

    # -- rendering -------------------------------------------------------------------
    @staticmethod
    def render_desc(cam: dict, precision=F32, mode=MODE_RPNN) -> RenderDesc:
        r = RenderDesc()
        for k in ("cam_pos", "cam_fwd", "cam_right", "cam_up", "light_dir"):
            arr = getattr(r, k)
            for i in range(3):
                arr[i] = float(cam[k][i])
        r.tan_half_fov_y = float(cam["tan_half_fov_y"])
        r.width, r.height, r.spp = int(cam["width"]), int(cam["height"]), int(cam["spp"])
        r.seed = int(cam["seed"])
        r.light_E = float(cam.get("light_E", 1.0))
        r.precision, r.mode = int(precision), int(mode)
        return r

    def render(self, vol, cam: dict, precision=F32, mode=MODE_RPNN, image=None,
               want_count=False, desc=None):
        rd = desc if desc is not None else self.render_desc(cam, precision, mode)
        if image is None:
            image = torch.empty((rd.height, rd.width), dtype=torch.float32, device="cuda")
        nq = C.c_int64(-1)
        self._check(self.L.rpnn_render(self.h, vol, C.byref(rd), _ptr(image),
                                       C.byref(nq) if want_count else None, _stream()))
        return (image, nq.value) if want_count else image

    def render_env(self, vol, cam: dict, dirs, irradiance, precision=F32, mode=MODE_RPNN, image=None,
                   want_count=False):
        """Render under n directional lights (dirs [n][3] unit, towards the light; irradiance
        [n]) approximating an environment emitter."""
        import numpy as np
        dirs = np.ascontiguousarray(dirs, dtype=np.float32).reshape(-1, 3)
        irr = np.ascontiguousarray(irradiance, dtype=np.float32).reshape(-1)
        assert dirs.shape[0] == irr.shape[0]
        rd = self.render_desc(cam, precision, mode)
        if image is None:
            image = torch.empty((cam["height"], cam["width"]), dtype=torch.float32, device="cuda")
        nq = C.c_int64(-1)
        fp = C.POINTER(C.c_float)
        self._check(self.L.rpnn_render_env(self.h, vol, C.byref(rd), dirs.ctypes.data_as(fp),
                                           irr.ctypes.data_as(fp), dirs.shape[0], _ptr(image),
                                           C.byref(nq) if want_count else None, _stream()))
        return (image, nq.value) if want_count else image

    def set_render_chunk(self, rows: int):
        self._check(self.L.rpnn_set_render_chunk(self.h, rows))

    def set_train_graphs(self, on: bool):
        """Capture the training step as a CUDA graph after its first run (default) or run
        every step's launches directly."""
        self._check(self.L.rpnn_set_train_graphs(self.h, 1 if on else 0))

    def set_fused(self, on: bool):
        """BF16 renders gather descriptors inside the network kernel (no descriptor buffer)
        or run the descriptor and network stages separately (the default)."""
        self._check(self.L.rpnn_set_fused(self.h, 1 if on else 0))

    def render_batch(self, jobs, images=None, want_counts=False):
        """Renders several clouds in one batched launch sequence (BF16 network): `jobs` is a
        list of (volume, camera dict); `images` (optional) the output tensors, which should
        be reused across calls so the captured graph is replayed.  Returns the images (and
        the per-item shading-point counts)."""
        n = len(jobs)
        arr = (BatchItem * n)()
        out = []
        for i, (vol, cam) in enumerate(jobs):
            rd = self.render_desc(cam, BF16, MODE_RPNN)
            img = images[i] if images is not None else torch.empty((rd.height, rd.width), dtype=torch.float32,
                                                                      device="cuda")
            arr[i].vol = vol
            arr[i].desc = rd
            arr[i].dev_image = _ptr(img)
            out.append(img)
        counts = (C.c_int64 * n)() if want_counts else None
        self._check(self.L.rpnn_render_batch(self.h, arr, n, counts, _stream()))
        return (out, list(counts)) if want_counts else out

    def trace_primary(self, vol, cam: dict):
        rd = self.render_desc(cam)
        P = rd.width * rd.height * rd.spp
        hit = torch.empty(P, dtype=torch.int32, device="cuda")
        x = torch.empty((P, 3), dtype=torch.float32, device="cuda")
        d = torch.empty((P, 3), dtype=torch.float32, device="cuda")
        Ld = torch.empty(P, dtype=torch.float32, device="cuda")
        self._check(self.L.rpnn_trace_primary(self.h, vol, C.byref(rd), _ptr(hit), _ptr(x),
                                              _ptr(d), _ptr(Ld), _stream()))
        return hit, x, d, Ld

    def gen_records(self, vol, first, n, seed, rel_ci=0.02, n_min=64, n_max=65536):
        dev = "cuda"
        x = torch.empty((n, 3), dtype=torch.float32, device=dev)
        d = torch.empty((n, 3), dtype=torch.float32, device=dev)
        wl = torch.empty((n, 3), dtype=torch.float32, device=dev)
        lab = torch.empty(n, dtype=torch.float32, device=dev)
        npaths = torch.empty(n, dtype=torch.int32, device=dev)
        self._check(self.L.rpnn_gen_records(self.h, vol, first, n, seed, rel_ci, n_min, n_max,
                                            _ptr(x), _ptr(d), _ptr(wl), _ptr(lab), _ptr(npaths),
                                            _stream()))
        return x, d, wl, lab, npaths
