"""GEMM-tile autotuner of the FP32 CUDA-core network: a tuned context gives the forward
results of an untuned one (the default tile) bit for bit, weight gradients that match the
FP64 oracle as closely (split-K partial sums change only their rounding), and records one
choice per GEMM shape it met."""
import numpy as np
import pytest

from paper_1709_05418_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1709_05418_gb300 import api
    params = torch.from_numpy(W.he_init(seed=9)).cuda()
    tuned, plain = api.Context(), api.Context()
    plain.set_autotune(False)
    for c in (tuned, plain):
        c.set_weights(params)
    yield api, tuned, plain, params
    tuned.close()
    plain.close()


def zbatch(q, seed):
    g = torch.Generator().manual_seed(seed)
    z = torch.rand((q, 10, 240), generator=g) * 2.0
    z[:, :, 226:] = 0.0
    return z.cuda()


def rel(a, b):
    a, b = a.double(), b.double()
    return float((a - b).norm() / max(float(b.norm()), 1e-30))


@pytest.mark.parametrize("q", [1, 333, 4096, 152 * 64 + 77])
def test_forward_tuned_matches_default_tile(env, q):
    api, tuned, plain, _ = env
    z = zbatch(q, q)
    a = tuned.mlp_forward(z, api.F32)
    b = plain.mlp_forward(z, api.F32)
    # forward GEMMs never split K, and a tile shape changes no bit
    assert torch.equal(a, b), rel(a, b)


@pytest.fixture(scope="module")
def cloud_desc():
    """FP32 descriptors of 333 shading points in the 64^3 blob cloud, from the oracle."""
    import oracle
    vol = oracle.Volume(W.blob_cloud(64, seed=1))
    x, d = W.random_queries((64, 64, 64), 333, seed=11, margin=0.2)
    wl = np.array([0.3, 0.5, -0.8])
    wl /= np.linalg.norm(wl)
    z = vol.descriptor(x.astype(np.float32), d.astype(np.float32), wl.astype(np.float32), f32=True)
    vol.close()
    zp = np.zeros((z.shape[0], 10, 240), np.float32)
    zp[:, :, :226] = z
    return zp


def test_backward_tuned_and_default_tile_both_match_oracle(env, cloud_desc):
    """Both contexts against the FP64 chain rule, per parameter tensor.  (A ReLU network's
    gradient jumps where a pre-activation crosses zero, so on inputs that put one within
    rounding of zero two summation orders can legitimately differ by more than rounding;
    the comparison is therefore with the oracle on a real cloud's descriptors.)"""
    import oracle
    api, tuned, plain, params = env
    z = torch.from_numpy(cloud_desc).cuda()
    q = z.shape[0]
    dout = torch.from_numpy(np.random.default_rng(3).normal(size=q).astype(np.float32)).cuda()
    ref = oracle.mlp_backward(params.double().cpu().numpy(), cloud_desc[:, :, :226].astype(np.float64),
                              dout.double().cpu().numpy())
    parts_r = W.split_params(ref)
    for c in (tuned, plain):
        g = c.mlp_backward(z, dout).double().cpu().numpy()
        parts_g = W.split_params(g)
        for name, rr in parts_r.items():
            if np.linalg.norm(rr) == 0:
                assert np.linalg.norm(parts_g[name]) == 0, name
            else:
                r = float(np.linalg.norm(parts_g[name] - rr) / np.linalg.norm(rr))
                assert r <= 1e-4, (name, r)


def test_table_records_one_choice_per_shape(env):
    api, tuned, plain, _ = env
    t = tuned.autotune_table()
    assert len(t) >= 10
    keys = [(e["M"], e["N"], e["K0"], e["K1"], e["flags"]) for e in t]
    assert len(set(keys)) == len(keys)
    for e in t:
        assert e["tile_m"] in (32, 64, 128) and e["tile_n"] in (32, 64, 128)
        assert e["splits"] >= 1 and e["us"] > 0 and e["us"] <= e["default_us"] * 1.0001
    # the weight-gradient GEMMs (200 x 200 outputs summed over the batch) are in the table;
    # K below 1,024 is never split; the untuned context recorded nothing
    assert any(e["K0"] == 333 and e["M"] == 200 for e in t)
    assert all(e["splits"] == 1 for e in t if e["K0"] + e["K1"] < 1024)
    assert plain.autotune_table() == []


def test_weight_gradient_over_a_long_batch_splits_and_matches_oracle(env, cloud_desc):
    """A batch of 2,048 rows (half the training minibatch): the weight-gradient GEMMs may
    take a split of K; the gradient still matches the FP64 chain rule per parameter tensor."""
    import oracle
    api, tuned, plain, params = env
    reps = -(-2048 // cloud_desc.shape[0])
    zz = np.concatenate([cloud_desc] * reps)[:2048]
    dout = np.random.default_rng(4).normal(size=2048).astype(np.float32)
    g = tuned.mlp_backward(torch.from_numpy(zz).cuda(), torch.from_numpy(dout).cuda()).double().cpu().numpy()
    ref = oracle.mlp_backward(params.double().cpu().numpy(), zz[:, :, :226].astype(np.float64),
                              dout.astype(np.float64))
    parts_g, parts_r = W.split_params(g), W.split_params(ref)
    for name, rr in parts_r.items():
        if np.linalg.norm(rr) == 0:
            assert np.linalg.norm(parts_g[name]) == 0, name
        else:
            r = float(np.linalg.norm(parts_g[name] - rr) / np.linalg.norm(rr))
            assert r <= 1e-4, (name, r)
    t = tuned.autotune_table()
    assert any(e["K0"] == 2048 and e["M"] == 200 for e in t)
