"""Mixed-precision training form (Sec. 5.2 with BF16 tensor-core GEMMs, FP32 master weights).

Its parameter gradient is compared with the CPU reference of the same arithmetic
(tests/mixed_precision_ref.py: the FP64 chain rule with each GEMM operand rounded to BF16
where the kernels round it, pinned to the oracle in the CPU tests), at a ragged batch and at
a batch long enough for the weight gradients to split K; its distance from the FP64
oracle's gradient is reported.  A fit lowers the validation loss as the FP32 form's does."""
import numpy as np
import pytest

from paper_1709_05418_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# Against the same-arithmetic reference the kernels differ in FP32 (not FP64) accumulation
# and sums, which can move the BF16 rounding of an activation by one unit.  Where no ReLU
# input is near zero that stays a rounding-level difference (TOL_LINEAR); at He
# initialisation many are, and a unit moved across zero re-routes that row's gradient, so
# two BF16 evaluations differ by a few percent (TOL_FLIPS) -- as BF16 and FP64 differ by
# about 15 %.  Bounds are per parameter tensor, relative L2.
TOL_LINEAR = 5e-3
TOL_FLIPS = 5e-2


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1709_05418_gb300 import api
    ctx = api.Context()
    ctx.set_train_precision(api.BF16)
    params = torch.from_numpy(W.he_init(seed=2)).cuda()
    ctx.set_weights(params)
    yield api, ctx, params
    ctx.close()


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


def per_tensor_errors(g, ref):
    out = {}
    pg, pr = W.split_params(g), W.split_params(ref)
    for name, rr in pr.items():
        nr = np.linalg.norm(rr)
        out[name] = float(np.linalg.norm(pg[name] - rr) / nr) if nr > 0 else float(np.linalg.norm(pg[name]))
    return out


def gradients(ctx, params, zz, dout):
    import oracle
    from mixed_precision_ref import forward_backward
    ctx.set_weights(params)
    g = ctx.mlp_backward(torch.from_numpy(zz).cuda(), torch.from_numpy(dout).cuda()).double().cpu().numpy()
    ctx.sync_status()
    assert np.isfinite(g).all()
    p64 = params.double().cpu().numpy()
    _, ref16 = forward_backward(p64, zz[:, :, :226], dout, bf16=True)
    ref64 = oracle.mlp_backward(p64, zz[:, :, :226].astype(np.float64), dout.astype(np.float64))
    return per_tensor_errors(g, ref16), per_tensor_errors(g, ref64)


def rows_of(cloud_desc, rows):
    reps = -(-rows // cloud_desc.shape[0])
    return np.concatenate([cloud_desc] * reps)[:rows]


@pytest.mark.parametrize("rows", [333, 2048])
def test_bf16_gradient_without_relu_flips(env, cloud_desc, rows):
    """Non-negative weights and positive biases keep every ReLU input positive, so the BF16
    kernels and the reference take the same branches: any wrong operand, transpose, scale or
    missing term shows above rounding level."""
    api, ctx, params = env
    p = params.abs() * 0.05
    L = W.split_params(np.zeros(W.param_count()))
    names = list(L)
    flat = p.cpu().numpy().copy()
    off = 0
    for n in names:
        size = L[n].size
        if n.startswith("b"):
            flat[off:off + size] = 0.01
        off += size
    p = torch.from_numpy(flat).cuda()
    zz = rows_of(cloud_desc, rows)
    dout = np.random.default_rng(3).normal(size=rows).astype(np.float32)
    err, e64 = gradients(ctx, p, zz, dout)
    worst = max(err, key=err.get)
    print(f"BF16 gradient, all ReLUs active, {rows} rows: vs same-arithmetic reference worst {worst} "
          f"{err[worst]:.2e}; vs FP64 oracle worst {max(e64.values()):.2e}")
    assert err[worst] <= TOL_LINEAR, err
    ctx.set_weights(params)


@pytest.mark.parametrize("rows", [333, 2048])
def test_bf16_gradient_at_he_init(env, cloud_desc, rows):
    api, ctx, params = env
    zz = rows_of(cloud_desc, rows)
    dout = np.random.default_rng(3).normal(size=rows).astype(np.float32)
    err, e64 = gradients(ctx, params, zz, dout)
    worst = max(err, key=err.get)
    print(f"BF16 gradient, He init, {rows} rows: vs same-arithmetic reference worst {worst} {err[worst]:.2e}, "
          f"median {np.median(list(err.values())):.2e}; vs FP64 oracle median "
          f"{np.median(list(e64.values())):.2e}, worst {max(e64.values()):.2e}")
    assert err[worst] <= TOL_FLIPS, err


def test_bf16_train_step_loss_matches_reference(env, cloud_desc):
    import oracle
    api, ctx, params = env
    z = torch.from_numpy(cloud_desc).cuda()
    target = torch.linspace(0.01, 0.5, z.shape[0], device="cuda")
    p = params.clone()
    m, v = torch.zeros_like(p), torch.zeros_like(p)
    loss = ctx.train_step(z, target, p, m, v, step=1, lr=1e-3)
    ctx.sync_status()
    from mixed_precision_ref import forward_backward
    p64 = params.double().cpu().numpy()
    g16, _ = forward_backward(p64, cloud_desc[:, :, :226], np.zeros(z.shape[0]), bf16=True)
    ref16 = oracle.logmse_loss(g16, target.double().cpu().numpy(), want_grad=False)
    g64 = oracle.mlp_forward(p64, cloud_desc[:, :, :226].astype(np.float64))
    ref64 = oracle.logmse_loss(g64, target.double().cpu().numpy(), want_grad=False)
    print(f"BF16 training loss {float(loss):.6f}; same-arithmetic reference {ref16:.6f}; FP64 oracle {ref64:.6f}")
    assert abs(float(loss) - ref16) <= 2e-3 * ref16, (float(loss), ref16)
    assert torch.isfinite(p).all() and not torch.equal(p, params)
    ctx.set_weights(params)


def test_bf16_fit_lowers_validation_loss(env):
    from paper_1709_05418_gb300 import train
    api, ctx, _ = env
    clouds = train.blob_clouds(3, size=48, seed0=320)
    desc, label = train.records(ctx, clouds, 4000, seed=21, rel_ci=0.1, n_min=32, n_max=512)
    tr, va = train.split(desc, label)
    params = torch.from_numpy(W.he_init(seed=5)).cuda()
    params.mul_(0.5)
    ctx.set_weights(params)
    v0 = train.val_loss(ctx, *va)
    hist = train.fit(ctx, tr, va, params, steps=300, batch=1024, lr=1e-3, eval_every=100)
    v1 = hist[-1][2]
    assert v1 < 0.3 * v0, (v0, hist)


@pytest.mark.parametrize("precision", ["F32", "BF16"])
def test_bf16_training_records_equal_rounded_fp32_records(env, cloud_desc, precision):
    """rpnn_train_step and rpnn_mlp_backward take BF16 descriptor rows (half the record
    memory).  BF16 rows are the FP32 rows' RNE rounding; fed as BF16, or as the same values
    widened back to FP32, both training forms give the same loss, gradient and update bit
    for bit."""
    api, ctx, params = env
    zb = torch.from_numpy(cloud_desc).cuda().to(torch.bfloat16)
    zf = zb.float()
    target = torch.linspace(0.01, 0.5, zb.shape[0], device="cuda")
    dout = torch.from_numpy(np.random.default_rng(9).normal(size=zb.shape[0]).astype(np.float32)).cuda()
    ctx.set_train_precision(getattr(api, precision))
    try:
        ctx.set_weights(params)
        assert torch.equal(ctx.mlp_backward(zb, dout), ctx.mlp_backward(zf, dout))
        res = []
        for z in (zb, zf):
            p = params.clone()
            m, v = torch.zeros_like(p), torch.zeros_like(p)
            loss = ctx.train_step(z, target, p, m, v, step=1, lr=1e-3)
            res.append((float(loss), p, m, v))
            ctx.set_weights(params)
        assert res[0][0] == res[1][0]
        for a, b in zip(res[0][1:], res[1][1:]):
            assert torch.equal(a, b)
        with pytest.raises(api.RPNNError):
            ctx.train_step(zb.to(torch.float16), target, params.clone(), torch.zeros_like(params),
                           torch.zeros_like(params), step=1)
    finally:
        ctx.set_train_precision(api.BF16)
        ctx.set_weights(params)


def test_autograd_function_bf16_route(env, cloud_desc):
    """In BF16 training precision the autograd Function runs the tensor-core forward on BF16
    descriptors and rpnn_mlp_backward's BF16 gradient; FP32 descriptors are refused."""
    from paper_1709_05418_gb300.autograd import rpnn
    api, ctx, params = env
    zb = torch.from_numpy(cloud_desc).cuda().to(torch.bfloat16)
    p = params.clone().requires_grad_(True)
    g = rpnn(p, zb, ctx)
    ref = ctx.mlp_forward(zb, precision=api.BF16)
    assert torch.equal(g.detach(), ref)
    w = torch.from_numpy(np.random.default_rng(10).normal(size=zb.shape[0]).astype(np.float32)).cuda()
    (g * w).sum().backward()
    ctx.set_weights(params)
    assert torch.equal(p.grad, ctx.mlp_backward(zb, w))
    with pytest.raises(TypeError):
        rpnn(p, zb.float(), ctx)
    ctx.set_weights(params)


@pytest.mark.parametrize("precision", ["F32", "BF16"])
def test_captured_training_steps_equal_direct_steps(env, cloud_desc, precision):
    """rpnn_set_train_graphs: from the third step of a configuration on, a step replays a
    captured graph after staging its minibatch; five steps over two alternating minibatches
    give the parameters, moments and losses of five direct steps bit for bit, with the
    autotuner's tile and split-K choices applied inside the captured GEMMs."""
    api, _, params = env
    # 1,280-row minibatches: the weight gradients' inner size admits split-K
    zb = torch.from_numpy(rows_of(cloud_desc, 2560)).cuda()
    if precision == "BF16":
        zb = zb.to(torch.bfloat16)
    batches = [(zb[:1280].contiguous(), torch.linspace(0.01, 0.5, 1280, device="cuda")),
               (zb[1280:].contiguous(), torch.linspace(0.4, 0.02, 1280, device="cuda"))]
    out, table = [], None
    for graphs in (False, True):
        ctx = api.Context()
        ctx.set_train_precision(getattr(api, precision))
        ctx.set_train_graphs(graphs)
        if table is not None:
            ctx.set_autotune_table(table)       # the direct context's tile and split choices
        p = params.clone()
        m, v = torch.zeros_like(p), torch.zeros_like(p)
        loss = torch.empty(1, dtype=torch.float64, device="cuda")
        ctx.set_weights(p)
        losses = []
        for step in range(1, 6):
            z, t = batches[step % 2]
            ctx.train_step(z, t, p, m, v, step, loss=loss)
            losses.append(float(loss.item()))
        ctx.sync_status()
        out.append((losses, p, m, v))
        if table is None:
            table = ctx.autotune_table()
            print(f"{precision}: {sum(e['splits'] > 1 for e in table)} of {len(table)} tuned shapes split K")
        ctx.close()
    assert out[0][0] == out[1][0]
    for a, b in zip(out[0][1:], out[1][1:]):
        assert torch.equal(a, b)
