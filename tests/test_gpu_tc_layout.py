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
