"""Tensor-core operand layouts (tcgen05 descriptors, TMEM loads, bulk and TMA copies)
used by the BF16 network kernel, checked with one MMA against numpy."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def probe():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    out = os.path.join(HERE, "_build")
    os.makedirs(out, exist_ok=True)
    so = os.path.join(out, "libtcprobe.so")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17",
                    "-Xcompiler", "-fPIC", "-shared", "-cudart", "shared", "-o", so,
                    os.path.join(HERE, "csrc", "tc_probe.cu")], check=True)
    torch.cuda.init()
    L = ctypes.CDLL(so)
    L.tc_probe.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int, ctypes.c_int] + [ctypes.c_void_p] * 3
    return L


def bf16(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16)


def test_mma_tmem_and_copies(probe):
    rng = np.random.default_rng(0)
    A = bf16(rng.normal(size=(128, 32)))
    B = bf16(rng.normal(size=(208, 32)))
    # B image: k-group major, rows contiguous: element (n, c) at (c//8)*208*8 + n*8 + c%8
    Bn = B.float().numpy()
    img = np.zeros((4, 208, 8), np.float32)
    for g in range(4):
        img[g] = Bn[:, 8 * g:8 * g + 8]
    Bimg = bf16(img.reshape(-1)).cuda()
    T = bf16(rng.normal(size=(100, 64))).cuda()
    D = torch.zeros((128, 208), dtype=torch.float32, device="cuda")
    tma = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    Ad = A.cuda()
    rc = probe.tc_probe(Ad.data_ptr(), Bimg.data_ptr(), T.data_ptr(), 100, 64, D.data_ptr(),
                        tma.data_ptr(), err.data_ptr())
    assert rc == 0 and err.item() == 0, (rc, err.item())
    ref = A.double().numpy() @ B.double().numpy().T
    got = D.cpu().double().numpy()
    assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max()
    boxes = tma.cpu().view(torch.bfloat16).float().numpy().reshape(2, 128, 8)
    Tn = T.float().cpu().numpy()
    exp0 = np.zeros((128, 8), np.float32)
    exp0[:100] = Tn[:, 16:24]
    exp1 = np.zeros((128, 8), np.float32)
    exp1[:36] = Tn[64:100, 8:16]
    assert np.array_equal(boxes[0], exp0) and np.array_equal(boxes[1], exp1)


def sw64_image(B):
    """[rows][64] -> two 32-column blocks, row-major 64-byte rows, 16-byte unit j of row n
    at unit j ^ ((n >> 1) & 3)."""
    rows = B.shape[0]
    img = np.zeros((2, rows, 4, 8), np.float32)
    for blk in range(2):
        for n in range(rows):
            for j in range(4):
                img[blk, n, j ^ ((n >> 1) & 3)] = B[n, 32 * blk + 8 * j:32 * blk + 8 * j + 8]
    return img


def test_mma_sw64_layouts(probe):
    probe.tc_probe_sw64.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int, ctypes.c_int] + [ctypes.c_void_p] * 3
    rng = np.random.default_rng(1)
    A = bf16(rng.normal(size=(128, 64)))
    B = bf16(rng.normal(size=(208, 64)))
    Bimg = bf16(sw64_image(B.float().numpy()).reshape(-1)).cuda()
    T = bf16(rng.normal(size=(100, 64))).cuda()
    D = torch.zeros((128, 208), dtype=torch.float32, device="cuda")
    tma = torch.zeros(8192, dtype=torch.uint8, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    Ad = A.cuda()
    rc = probe.tc_probe_sw64(Ad.data_ptr(), Bimg.data_ptr(), T.data_ptr(), 100, 64, D.data_ptr(),
                             tma.data_ptr(), err.data_ptr())
    assert rc == 0 and err.item() == 0, (rc, err.item())
    ref = A.double().numpy() @ B.double().numpy().T
    got = D.cpu().double().numpy()
    assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max()
    raw = tma.cpu().view(torch.bfloat16).float().numpy().reshape(128, 4, 8)
    box = np.zeros((128, 32), np.float32)
    for r in range(128):
        for j in range(4):
            box[r, 8 * j:8 * j + 8] = raw[r, j ^ ((r >> 1) & 3)]
    exp = np.zeros((128, 32), np.float32)
    exp[:100] = T.float().cpu().numpy()[:, 32:64]
    assert np.array_equal(box, exp)


def sw64_image_bytes(B):
    """[rows][128] bytes -> two 64-byte-wide blocks, row-major 64-byte rows, 16-byte unit j
    of row n at unit j ^ ((n >> 1) & 3)."""
    rows = B.shape[0]
    img = np.zeros((2, rows, 4, 16), np.uint8)
    for blk in range(2):
        for n in range(rows):
            for j in range(4):
                img[blk, n, j ^ ((n >> 1) & 3)] = B[n, 64 * blk + 16 * j:64 * blk + 16 * j + 16]
    return img


def test_mma_fp8_e4m3_layouts(probe):
    """kind::f8f6f4 with E4M3 A and B in the 64-byte-swizzled K-major layout (64 elements
    per row of a block, K = 32 per MMA) and a uint8 TMA box: D = A B^T exactly as the FP32
    sum of the E4M3 products."""
    f8 = getattr(torch, "float8_e4m3fn", None)
    if f8 is None:
        pytest.skip("no float8_e4m3fn in this torch")
    probe.tc_probe_fp8.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int, ctypes.c_int] + [ctypes.c_void_p] * 3
    rng = np.random.default_rng(7)
    A8 = torch.from_numpy(rng.normal(size=(128, 128)).astype(np.float32)).to(f8)
    B8 = torch.from_numpy(rng.normal(size=(208, 128)).astype(np.float32)).to(f8)
    Ab = A8.view(torch.uint8).numpy()
    Bb = B8.view(torch.uint8).numpy()
    Bimg = torch.from_numpy(sw64_image_bytes(Bb).reshape(-1).copy()).cuda()
    T = torch.from_numpy(rng.integers(0, 256, size=(100, 256), dtype=np.uint8)).cuda()
    D = torch.zeros((128, 208), dtype=torch.float32, device="cuda")
    tma = torch.zeros(8192, dtype=torch.uint8, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    Ad = torch.from_numpy(Ab.copy()).cuda()
    rc = probe.tc_probe_fp8(Ad.data_ptr(), Bimg.data_ptr(), T.data_ptr(), 100, 256, D.data_ptr(),
                            tma.data_ptr(), err.data_ptr())
    assert rc == 0 and err.item() == 0, (rc, err.item())
    ref = A8.double().numpy() @ B8.double().numpy().T
    got = D.cpu().double().numpy()
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()
    raw = tma.cpu().numpy().reshape(128, 4, 16)
    box = np.zeros((128, 64), np.uint8)
    for r in range(128):
        for j in range(4):
            box[r, 16 * j:16 * j + 16] = raw[r, j ^ ((r >> 1) & 3)]
    exp = np.zeros((128, 64), np.uint8)
    exp[:100] = T.cpu().numpy()[:, 64:128]
    assert np.array_equal(box, exp)


def test_bounded_wait_gives_up_and_the_context_stays_usable(probe):
    """A wait on a barrier phase nobody completes returns after its poll budget with the
    error set (no hang, no trap), and the device keeps working afterwards."""
    probe.tc_wait_timeout.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    err = torch.zeros(2, dtype=torch.int32, device="cuda")
    cyc = torch.zeros(1, dtype=torch.int64, device="cuda")
    assert probe.tc_wait_timeout(2000, err.data_ptr(), cyc.data_ptr()) == 0
    assert err.tolist() == [1, 1]
    assert int(cyc) > 0
    x = torch.arange(1000, device="cuda", dtype=torch.float32)
    assert float(x.sum()) == 499500.0
