"""Proposal network on the tensor cores vs the FP64 oracle (oracle/mlp.py).

Bars: outputs within 1e-2 of the output RMS element by element (BF16 storage,
FP32 accumulation against FP64 accumulation of the same BF16 values), the loss
within 1e-4 relative, weight gradients with cosine >= 0.999 per layer block and
norm error <= 1e-2; batches span several 128-row tiles with a ragged tail.
"""
import numpy as np
import pytest
import torch

from oracle import mlp as om

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    from paper_2411_11833_b300.build import build_library
    build_library()
    import paper_2411_11833_b300 as p
    torch.cuda.set_device(0)
    return p


def _params(seed):
    th = om.init_params(seed)
    g = np.random.default_rng(seed)
    # non-zero biases so that a bias indexing mistake shows
    o = 0
    for (wr, wc), (bn,) in om.shapes():
        o += wr * wc
        th[o:o + bn] = torch.from_numpy(g.normal(0.0, 0.1, bn))
        o += bn
    return th.numpy().astype(np.float32)


def _batch(B, seed):
    g = np.random.default_rng(seed)
    x = g.normal(0.0, 1.0, (B, om.IN)).astype(np.float32)
    y = g.normal(0.0, 1.0, (B, om.OUT // 2)).astype(np.float32)
    mask = (g.random((B, om.OUT // 2)) < 0.8).astype(np.float32)
    mask[:, 9:] = 0.0                      # 9 targets in use, the rest padding
    return x, y, mask


def _cuda(a):
    return torch.from_numpy(a).cuda()


def _blocks():
    out, o = [], 0
    for (wr, wc), (bn,) in om.shapes():
        out.append(("W", o, o + wr * wc))
        o += wr * wc
        out.append(("b", o, o + bn))
        o += bn
    return out


@pytest.mark.parametrize("B", [1, 128, 300])
def test_forward_matches_oracle(pkg, B):
    th = _params(3)
    x, _, _ = _batch(B, 10 + B)
    net = pkg.Mlp(max_batch=512)
    net.set_params(th)
    out = net.forward(_cuda(x)).cpu().double().numpy()
    ref = om.forward(torch.from_numpy(th).double(), torch.from_numpy(x).double()).numpy()
    scale = np.sqrt((ref ** 2).mean())
    assert np.abs(out - ref).max() <= 1e-2 * scale, np.abs(out - ref).max() / scale
    net.close()


@pytest.mark.parametrize("B", [128, 300, 3000, 16384])
def test_gradient_matches_oracle(pkg, B):
    # 300 rows: a ragged last tile (rows past the batch are zeros in the
    # weight-gradient operands); 3000 rows: row splits of two chunks and splits
    # with no rows at all; 16384 (the benchmark's training batch): 11 chunks per
    # split.  Two calls in a row: the loss and the gradient are accumulators the
    # training kernel zeroes, so the second call must not add onto the first.
    th = _params(5)
    x, y, mask = _batch(B, 20 + B)
    net = pkg.Mlp(max_batch=max(512, B))
    net.set_params(th)
    L, gr = om.loss_and_grad(torch.from_numpy(th).double(), torch.from_numpy(x).double(),
                             torch.from_numpy(y).double(), torch.from_numpy(mask).double())
    gr = gr.numpy()
    for call in range(2):
        loss, g = net.gradient(_cuda(x), _cuda(y), _cuda(mask))
        g = g.cpu().double().numpy()
        assert abs(loss - float(L)) <= 1e-4 * abs(float(L)), (call, loss, float(L))
        for kind, a, b in _blocks():
            u, v = g[a:b], gr[a:b]
            cos = float(u @ v / (np.linalg.norm(u) * np.linalg.norm(v)))
            rel = float(np.linalg.norm(u - v) / np.linalg.norm(v))
            assert cos >= 0.999 and rel <= 1e-2, (call, kind, a, cos, rel)
    net.close()


def test_adam_first_step_moves_against_the_gradient_sign(pkg):
    # Adam's first bias-corrected step is -lr * g / (|g| + eps) = -lr sign(g)
    # wherever |g| >> eps
    th = _params(7)
    x, y, mask = _batch(256, 33)
    net = pkg.Mlp(max_batch=256)
    net.set_params(th)
    lr = 1e-3
    net.train_step(_cuda(x), _cuda(y), _cuda(mask), lr)
    step = net.get_params().astype(np.float64) - th.astype(np.float64)
    _, gr = om.loss_and_grad(torch.from_numpy(th).double(), torch.from_numpy(x).double(),
                             torch.from_numpy(y).double(), torch.from_numpy(mask).double())
    gr = gr.numpy()
    big = np.abs(gr) > 1e-3 * np.abs(gr).max()
    expect = -lr * np.sign(gr[big])
    assert np.mean(np.abs(step[big] - expect) <= 1e-6 + 1e-3 * lr) >= 0.99
    assert np.abs(step).max() <= lr * 1.001
    net.close()


def test_training_fits_a_conditional_gaussian_and_stays_consistent(pkg):
    # targets y = A x + noise of known scale per target: NLL training must fit
    # the means and learn log sigma close to log(noise)
    g = np.random.default_rng(11)
    B = 1024
    A = g.normal(0.0, 0.3, (9, om.IN))
    sig = np.linspace(0.05, 0.4, 9)
    net = pkg.Mlp(max_batch=B)
    th = om.init_params(13).numpy().astype(np.float32)
    net.set_params(th)
    mask = np.zeros((B, 16), np.float32)
    mask[:, :9] = 1.0
    losses = []
    for it in range(300):
        x = g.normal(0.0, 1.0, (B, om.IN)).astype(np.float32)
        y = np.zeros((B, 16), np.float32)
        y[:, :9] = x @ A.T + g.normal(0.0, 1.0, (B, 9)) * sig
        # at 2e-3 throughout, the loss keeps bouncing by ~1 over the last 150 steps (the
        # smallest noise's log sigma sits in a steep valley) and where the run stops
        # depends on the last bits of the gradients; the lower rate settles it
        losses.append(net.train_step(_cuda(x), _cuda(y), _cuda(mask), 2e-3 if it < 200 else 4e-4))
    assert losses[-1] < losses[0] - 3.0, (losses[0], losses[-1])
    # the trained parameters read back drive the oracle to the kernel's outputs
    th1 = net.get_params()
    x = g.normal(0.0, 1.0, (300, om.IN)).astype(np.float32)
    out = net.forward(_cuda(x)).cpu().double().numpy()
    ref = om.forward(torch.from_numpy(th1).double(), torch.from_numpy(x).double()).numpy()
    assert np.abs(out - ref).max() <= 1e-2 * np.sqrt((ref ** 2).mean())
    # learned log sigma near the generating noise (loose: 300 steps)
    ls = ref[:, 16:25].mean(axis=0)
    assert np.all(np.abs(ls - np.log(sig)) < 0.7), ls - np.log(sig)
    net.close()


def test_invalid_arguments_are_refused(pkg):
    from paper_2411_11833_b300 import TampError
    net = pkg.Mlp(max_batch=64)
    with pytest.raises(TampError):
        net.set_params(np.zeros(10, np.float32))
    x, y, mask = _batch(65, 1)
    with pytest.raises(TampError):
        net.gradient(_cuda(x), _cuda(y), _cuda(mask))
    net.close()
