"""Cost-model oracle pins (CPU) and CUDA kernel parity (GPU)."""
import numpy as np
import pytest

from oracle import mlp_oracle as M


def _problem(seed, batch=37):
    rng = np.random.default_rng(seed)
    p = rng.normal(0, 0.3, M.H * M.IN + M.H + M.H * M.H + M.H + M.OUT * M.H + M.OUT)
    x = rng.uniform(0, 1, (batch, M.IN))
    t = rng.normal(0, 1, (batch, M.OUT))
    m = (rng.uniform(0, 1, (batch, M.OUT)) < 0.7).astype(np.float64)
    m[0, :] = 1
    return p, x, t, m


def test_oracle_gradient_matches_finite_differences():
    p, x, t, m = _problem(1)
    g = M.grad(p, x, t, m)
    rng = np.random.default_rng(2)
    idx = np.concatenate([rng.choice(p.size, 200, replace=False), [0, 255, 256, 319, 4416, 4999]])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (M.loss(p + e, x, t, m) - M.loss(p - e, x, t, m)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), i


def test_oracle_forward_special_cases():
    p, x, t, m = _problem(3, batch=5)
    # zero weights and biases except b3: y = b3 for every input
    q = np.zeros_like(p)
    q[-M.OUT:] = np.arange(M.OUT)
    _, _, y = M.forward(q, x)
    assert np.array_equal(y, np.tile(np.arange(M.OUT, dtype=np.float64), (5, 1)))
    # perfect prediction -> zero loss and zero gradient
    _, _, y = M.forward(p, x)
    assert M.loss(p, x, y, m) == 0.0
    assert not np.any(M.grad(p, x, y, m))


@pytest.mark.gpu
def test_cuda_forward_backward_adam_match_float64_oracle():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2410_05934_gb300 import costmodel as CM
    for seed, batch in [(4, 1), (5, 37), (6, 1000)]:
        p, x, t, m = _problem(seed, batch)
        y_gpu, g_gpu, loss_gpu = CM.gpu_forward_backward(p, x, t, m)
        _, _, y_ref = M.forward(p, x)
        g_ref = M.grad(p, x, t, m)
        # FP32 kernels vs float64: relative error of a few ulp per accumulation step
        assert np.allclose(y_gpu, y_ref, rtol=1e-4, atol=1e-4)
        scale = np.abs(g_ref).max()
        assert np.abs(g_gpu - g_ref).max() <= 1e-4 * scale + 1e-6
        assert abs(loss_gpu - M.loss(p, x, t, m)) <= 1e-4 * max(1.0, abs(M.loss(p, x, t, m)))
    # Adam against the float64 update rule
    rng = np.random.default_rng(9)
    p = rng.normal(0, 1, 5000)
    g = rng.normal(0, 1, 5000)
    m0, v0 = rng.normal(0, 0.1, 5000), rng.uniform(0, 0.1, 5000)
    new_p, new_m, new_v = CM.gpu_adam(p, g, m0, v0, lr=1e-2, step=3)
    b1, b2, eps = 0.9, 0.999, 1e-8
    rm = b1 * m0 + (1 - b1) * g
    rv = b2 * v0 + (1 - b2) * g * g
    rp = p - 1e-2 * (rm / (1 - b1 ** 3)) / (np.sqrt(rv / (1 - b2 ** 3)) + eps)
    assert np.allclose(new_m, rm, rtol=1e-5, atol=1e-6) and np.allclose(new_v, rv, rtol=1e-5, atol=1e-7)
    assert np.allclose(new_p, rp, rtol=1e-5, atol=1e-5)
