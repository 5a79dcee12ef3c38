"""Pins of the warm-start network oracle: bfloat16 rounding against torch's conversion, the
backward pass against central finite differences, and the Adam step against its formula."""
import numpy as np
import pytest

from oracle import mlp


def test_bf16_rounding_matches_library_conversion():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    a = np.concatenate([rng.standard_normal(1000).astype(np.float32) * 10 ** rng.uniform(-5, 5, 1000),
                        np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -2.5, 0.0], dtype=np.float32)])
    ref = torch.tensor(a).to(torch.bfloat16).float().numpy()
    np.testing.assert_array_equal(mlp.bf16(a), ref)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(1)
    widths = [7, 9, 8, 5]
    Ws, bs = mlp.init(widths, 3)
    Ws = [w.astype(np.float64) for w in Ws]
    bs = [b.astype(np.float64) + rng.standard_normal(b.shape) * 0.1 for b in bs]
    x = rng.standard_normal((4, 7))
    t = rng.standard_normal((4, 5))
    _, gW, gb = mlp.loss_and_grads(Ws, bs, x, t, rnd=False)
    h = 1e-6
    for l in range(3):
        for (i, j) in [(0, 0), (2, 3), (Ws[l].shape[0] - 1, Ws[l].shape[1] - 1)]:
            Wp = [w.copy() for w in Ws]
            Wm = [w.copy() for w in Ws]
            Wp[l][i, j] += h
            Wm[l][i, j] -= h
            fd = (mlp.loss_and_grads(Wp, bs, x, t, rnd=False)[0] - mlp.loss_and_grads(Wm, bs, x, t, rnd=False)[0]) / (2 * h)
            assert abs(fd - gW[l][i, j]) < 1e-8
        bp = [b.copy() for b in bs]
        bm = [b.copy() for b in bs]
        bp[l][1] += h
        bm[l][1] -= h
        fd = (mlp.loss_and_grads(Ws, bp, x, t, rnd=False)[0] - mlp.loss_and_grads(Ws, bm, x, t, rnd=False)[0]) / (2 * h)
        assert abs(fd - gb[l][1]) < 1e-8


def test_adam_first_step_is_a_signed_learning_rate():
    """With zero moments the bias-corrected first Adam step is -lr * g / (|g| + eps)."""
    g = np.array([0.3, -2.0, 1e-3])
    p, m, v = mlp.adam(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    np.testing.assert_allclose(p, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
