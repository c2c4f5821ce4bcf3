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


def test_mma_issue_rate(probe, capsys):
    """Back-to-back tcgen05.mma throughput on resident operands (reported, loosely checked)."""
    probe.tc_mma_rate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    cyc = torch.zeros(2, dtype=torch.int64, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    rates = {}
    cases = [(4, 128, "sw64 N208, 4 warps"), (6, 128, "sw64 N256, 4 warps"), (4, 160, "sw64 N208, 5 warps"),
             (4, 192, "sw64 N208, 6 warps"), (4, 256, "sw64 N208, 8 warps"), (4, 320, "sw64 N208, 10 warps"),
             (4 | 32, 256, "8 warps, 4 exit early"), (4 | 16, 128, "4 warps, wait+fence per 2"),
             (4 | 8, 256, "8 warps, 7 polling")]
    for mode, nt, name in cases:
        n = 4096
        assert probe.tc_mma_rate(n, mode, cyc.data_ptr(), err.data_ptr(), nt) == 0
        assert err.item() == 0
        issue, done = cyc.cpu().tolist()
        macs = 128 * (256 if mode & 2 else 208) * 16
        rates[name] = (issue / n, done / n, macs / (done / n))
    with capsys.disabled():
        for k, (i, d, r) in rates.items():
            print(f"\n[mma rate] {k:28s} issue {i:7.1f} cyc/mma  complete {d:7.1f} cyc/mma  {r:7.0f} MAC/clk")
    for _, d, _ in rates.values():
        assert d > 0


def test_mma_issue_loop_variants(probe, capsys):
    probe.tc_mma_variant.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    cyc = torch.zeros(2, dtype=torch.int64, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    names = ["plain", "wait/2", "fence::after/2", "fence before loop", "commit/2", "wait+commit/2",
             "relaxed try_wait/2", "test_wait/2", "relaxed test_wait/2", "asm try_wait loop/2", "wait/4",
             "bounded asm, no output/2", "abort check + bounded/2", "volatile counter poll/2",
             "acquire counter poll/2", "bounded asm, no output/4"]
    out = []
    for v, name in enumerate(names):
        assert probe.tc_mma_variant(v, 4096, cyc.data_ptr(), err.data_ptr()) == 0
        assert err.item() == 0
        out.append((name, cyc.cpu().tolist()[1] / 4096))
    with capsys.disabled():
        for name, c in out:
            print(f"\n[mma loop] {name:20s} {c:7.1f} cyc/mma")


def test_mma_rate_with_concurrent_copies(probe, capsys):
    probe.tc_mma_with_copies.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    src = torch.zeros(64 * 13312, dtype=torch.uint8, device="cuda")
    cyc = torch.zeros(2, dtype=torch.int64, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    for mode, name in [(0, "bulk copies"), (1, "bulk copies + smem stores"), (2, "bulk copies + tmem loads"),
                       (4, "bulk copies + A rewrites")]:
        assert probe.tc_mma_with_copies(4096, mode, src.data_ptr(), cyc.data_ptr(), err.data_ptr()) == 0
        assert err.item() == 0
        copies, c = cyc.cpu().tolist()
        with capsys.disabled():
            print(f"\n[mma + traffic] {name:26s} {c / 4096:7.1f} cyc/mma, {copies} copies of 13 KB "
                  f"({copies * 13312 / c:5.1f} B/clk)")


def test_mma_rate_through_ring(probe, capsys):
    """MMA rate when every CH MMAs wait for a ring stage and commit it back, on one SM and
    on every SM at once (the network kernel's pipeline without its epilogue), for three
    forms of the issuing thread's wait."""
    probe.tc_mma_ring.argtypes = [ctypes.c_int] * 5 + [ctypes.c_void_p] * 3
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    src = torch.zeros(64 * 13312, dtype=torch.uint8, device="cuda")
    cyc = torch.zeros(nsm + 24, dtype=torch.int64, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    stamps = {}
    forms = ["branch on success", "fall-through", "fall-through, 2 stages", "commit every 2 stages",
             "three-barrier poll", "two commits per stage", "4 distinct operands",
             "4 distinct, + 8 polling warps"]
    out = []
    for ch, wf in [(0, 0), (2, 0), (2, 1), (2, 2), (2, 3), (4, 0), (4, 1), (4, 4), (4, 5), (4, 6), (4, 7), (8, 0)]:
        for copy in ((0,) if ch == 0 else (0, 1, 2, 3)):
            for grid in (1, nsm) if copy < 2 else (nsm,):
                cyc.zero_()
                err.zero_()
                assert probe.tc_mma_ring(ch, wf, 4096, copy, grid, src.data_ptr(), cyc.data_ptr(),
                                         err.data_ptr()) == 0
                c = cyc[:grid].double().cpu()
                if wf >= 6:
                    stamps[(wf, copy, grid)] = cyc[grid:grid + 24].cpu().tolist()
                out.append((ch, forms[wf], copy, grid, c.mean().item() / 4096, c.max().item() / 4096, err.item()))
    with capsys.disabled():
        for ch, form, copy, grid, mean, mx, e in out:
            print(f"\n[mma ring] {ch} MMAs/stage, {form:22s} copy={copy & 1} sleep={copy >> 1} grid={grid:3d}  {mean:7.1f} cyc/mma "
                  f"(max {mx:7.1f}) err={e}")
        for (wf, copy, grid), st in stamps.items():
            t0 = st[0]
            print(f"\n[mma ring stages] wf={wf} copy={copy & 1} sleep={copy >> 1} grid={grid}: " +
                  "  ".join(f"{st[3 * i] - t0}/{st[3 * i + 1] - t0}/{st[3 * i + 2] - t0}" for i in range(8)))
    assert all(o[-1] == 0 for o in out)



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
