"""Checkpoint / resume of training: a context restored from a checkpoint (parameters, Adam
moments, step, training precision, the autotuner's decisions) takes the next step bit for
bit as the run that wrote it, in both training precisions."""
import os

import numpy as np
import pytest

from paper_1709_05418_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["BF16", "F32"])
def test_resume_is_bit_identical(tmp_path, precision):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1709_05418_gb300 import api, train
    prec = getattr(api, precision)
    g = torch.Generator().manual_seed(5)
    z = torch.rand((2048, 10, 240), generator=g) * 1.5
    z[:, :, 226:] = 0.0
    t = torch.rand(2048, generator=g) * 0.4
    z, t = z.cuda(), t.cuda()
    params = torch.from_numpy(W.he_init(seed=6)).cuda()
    m, v = torch.zeros_like(params), torch.zeros_like(params)
    a = api.Context()
    a.set_train_precision(prec)
    a.set_weights(params)
    for step in range(1, 4):
        a.train_step(z, t, params, m, v, step)
    path = os.path.join(tmp_path, "ck.pt")
    train.save_checkpoint(path, a, params, m, v, 3, prec)
    la = a.train_step(z, t, params, m, v, 4)
    a.sync_status()

    b = api.Context()
    pb, mb, vb, step = train.load_checkpoint(path, b)
    assert step == 3
    lb = b.train_step(z, t, pb, mb, vb, step + 1)
    b.sync_status()
    assert torch.equal(la, lb)
    assert torch.equal(params, pb) and torch.equal(m, mb) and torch.equal(v, vb)
    assert any(e["splits"] > 1 for e in b.autotune_table())
    a.close()
    b.close()
