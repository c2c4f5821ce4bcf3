"""Plain ("all-at-once") MLPs of the architecture comparison (Sec. 7, Fig. 10): forward and
parameter gradient against the FP64 oracle (pinned by hand cases and finite differences in
the CPU tests), a training step's loss, and the comparison itself on synthetic records."""
import numpy as np
import pytest

from paper_1709_05418_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import oracle
    from paper_1709_05418_gb300 import api
    ctx = api.Context()
    vol = oracle.Volume(W.blob_cloud(64, seed=1))
    x, d = W.random_queries((64, 64, 64), 333, seed=11, margin=0.2)
    wl = np.array([0.3, 0.5, -0.8])
    wl /= np.linalg.norm(wl)
    z = vol.descriptor(x.astype(np.float32), d.astype(np.float32), wl.astype(np.float32), f32=True)
    vol.close()
    zp = np.zeros((z.shape[0], 10, 240), np.float32)
    zp[:, :, :226] = z
    yield api, ctx, zp
    ctx.close()


@pytest.mark.parametrize("widths", [W.SHALLOW_WIDE, W.DEEP_NARROW])
def test_dense_forward_and_gradient_match_oracle(env, widths):
    import oracle
    api, ctx, zp = env
    params = W.dense_he_init(widths, 2400, seed=3)
    assert ctx.dense_param_count(widths, 2400) == params.size
    z = torch.from_numpy(zp).cuda()
    p = torch.from_numpy(params).cuda()
    g = ctx.dense_forward(widths, p, z).double().cpu().numpy()
    ref, _ = oracle.dense_forward(params.astype(np.float64), widths, zp.reshape(len(zp), -1))
    assert (ref > 0).mean() > 0.5
    assert np.linalg.norm(g - ref) / np.linalg.norm(ref) <= 1e-5
    dout = np.random.default_rng(4).normal(size=len(zp)).astype(np.float32)
    dp = ctx.dense_backward(widths, p, z, torch.from_numpy(dout).cuda()).double().cpu().numpy()
    rg = oracle.dense_backward(params.astype(np.float64), widths, zp.reshape(len(zp), -1), dout.astype(np.float64))
    assert np.linalg.norm(dp - rg) / np.linalg.norm(rg) <= 1e-4


def test_dense_train_step_loss(env):
    import oracle
    api, ctx, zp = env
    widths = W.SHALLOW_WIDE
    params = W.dense_he_init(widths, 2400, seed=5)
    p = torch.from_numpy(params).cuda()
    m, v = torch.zeros_like(p), torch.zeros_like(p)
    target = torch.linspace(0.02, 0.6, len(zp), device="cuda")
    loss = ctx.dense_train_step(widths, torch.from_numpy(zp).cuda(), target, p, m, v, 1)
    ctx.sync_status()
    g, _ = oracle.dense_forward(params.astype(np.float64), widths, zp.reshape(len(zp), -1))
    ref = oracle.logmse_loss(g, target.double().cpu().numpy(), want_grad=False)
    assert abs(float(loss) - ref) <= 1e-5 * ref
    assert torch.isfinite(p).all() and not torch.equal(p.cpu(), torch.from_numpy(params))


def test_architecture_comparison_trains_all_three(env):
    """The comparison runs end to end and every network lowers its validation loss; the
    curves are printed (Fig. 10's full ordering is the paper's finding on its dataset and is
    reported here, with only its widest gap asserted)."""
    from paper_1709_05418_gb300 import ablation, train
    api, ctx, _ = env
    clouds = train.blob_clouds(3, size=48, seed0=340)
    desc, label = train.records(ctx, clouds, 3000, seed=31, rel_ci=0.1, n_min=32, n_max=512)
    tr, va = train.split(desc, label)
    curves, counts = ablation.compare(ctx, tr, va, steps=200, batch=512, eval_every=100)
    for name, c in curves.items():
        print(f"{name} ({counts[name]} parameters): " + ", ".join(f"{s}: {l:.4f}" for s, l in c))
        assert c[-1][1] < 0.85 * c[0][1], (name, c)
    # the progressive network ends lowest of the three in every run so far; asserted only
    # against the deep-narrow MLP, the paper's clearest gap
    assert curves["rpnn"][-1][1] < curves["deep_narrow"][-1][1], curves
