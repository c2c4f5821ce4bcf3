"""Training on the GPU (Sec. 5) and what the trained network gains (Sec. 4.4, Sec. 6):
records are path traced by the library, the network is fitted with the library's own
forward/backward kernels, and a render of a held-out cloud with the trained network is
closer to a converged path-traced reference than the method without the network
(single scattering only, L_i = 0)."""
import numpy as np
import pytest

from paper_1709_05418_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1709_05418_gb300 import api, train
    ctx = api.Context()
    yield api, train, ctx
    ctx.close()


def test_training_reduces_loss_and_beats_single_scattering(env):
    api, train, ctx = env
    clouds = train.blob_clouds(4, size=48, seed0=300)
    desc, label = train.records(ctx, clouds, 6000, seed=11, rel_ci=0.1, n_min=32, n_max=512)
    assert desc.shape == (24000, 10, 240) and torch.isfinite(label).all()
    assert (label > 0).float().mean() > 0.5
    tr, va = train.split(desc, label)
    params = torch.from_numpy(W.he_init(seed=5)).cuda()
    params.mul_(0.5)
    ctx.set_weights(params)
    v0 = train.val_loss(ctx, *va)
    hist = train.fit(ctx, tr, va, params, steps=400, batch=1024, lr=1e-3, eval_every=100)
    v1 = hist[-1][2]
    assert v1 < 0.25 * v0, (v0, hist)
    # held-out cloud, reference by plain path tracing
    held = W.blob_cloud(48, nblobs=8, seed=999)
    vol = ctx.load_volume(torch.from_numpy(held).cuda())
    ctx.build_mips(vol)
    cam = W.camera(held.shape, 40, 40, spp=8, seed=12, light_seed=13)
    ref_cam = dict(cam, spp=512)
    ref = ctx.render(vol, ref_cam, mode=api.MODE_PATH).double()
    ctx.set_weights(params)
    rp = ctx.render(vol, cam, precision=api.F32, mode=api.MODE_RPNN).double()
    ss = ctx.render(vol, cam, mode=api.MODE_SINGLE).double()
    ctx.sync_status()
    mask = ref > 0
    rmse_rpnn = float(torch.sqrt(((rp - ref)[mask] ** 2).mean()))
    rmse_ss = float(torch.sqrt(((ss - ref)[mask] ** 2).mean()))
    assert rmse_rpnn < 0.7 * rmse_ss, (rmse_rpnn, rmse_ss)


def test_autograd_function_matches_oracle_gradient(env):
    """rpnn() under torch.autograd gives the FP64 oracle's parameter gradient (the oracle's
    backward is pinned against finite differences in the CPU tests)."""
    import oracle
    from paper_1709_05418_gb300.autograd import rpnn
    api, train, ctx = env
    rng = np.random.default_rng(31)
    z = np.zeros((300, 10, 240), np.float32)
    z[:, :, :226] = rng.uniform(0, 2, size=(300, 10, 226))
    p = W.he_init(seed=32, bias=0.02, positive_head=True)
    w = rng.normal(size=300)
    pt = torch.from_numpy(p).cuda().requires_grad_(True)
    g = rpnn(pt, torch.from_numpy(z).cuda(), ctx)
    (g.double() * torch.from_numpy(w).cuda()).sum().backward()
    ref_g = oracle.mlp_forward(p.astype(np.float64), z[:, :, :226].astype(np.float64))
    ref = oracle.mlp_backward(p.astype(np.float64), z[:, :, :226].astype(np.float64), w)
    ctx.sync_status()
    assert np.abs(g.detach().cpu().numpy() - ref_g).max() <= 1e-4 * np.abs(ref_g).max()
    got = pt.grad.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - ref) <= 1e-4 * np.linalg.norm(ref)


def test_autograd_function_trains_with_torch_adam(env):
    """The log-MSE loss of Sec. 5.2 through rpnn() and torch.optim.Adam decreases."""
    from paper_1709_05418_gb300.autograd import rpnn
    api, train, ctx = env
    clouds = train.blob_clouds(2, size=40, seed0=400)
    desc, label = train.records(ctx, clouds, 2000, seed=21, rel_ci=0.2, n_min=16, n_max=128)
    p = torch.from_numpy(W.he_init(seed=7)).cuda().mul_(0.5).requires_grad_(True)
    opt = torch.optim.Adam([p], lr=1e-3)
    gen = torch.Generator(device="cuda").manual_seed(3)

    def loss_of(idx):
        g = rpnn(p, desc[idx], ctx)
        return ((torch.log1p(g) - torch.log1p(label[idx])) ** 2).mean()

    with torch.no_grad():
        l0 = loss_of(torch.arange(desc.shape[0], device="cuda")).item()
    for _ in range(150):
        idx = torch.randint(0, desc.shape[0], (512,), device="cuda", generator=gen)
        opt.zero_grad()
        loss_of(idx).backward()
        opt.step()
    with torch.no_grad():
        l1 = loss_of(torch.arange(desc.shape[0], device="cuda")).item()
    assert l1 < 0.5 * l0, (l0, l1)
