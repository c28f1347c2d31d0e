"""Pins of the FP64 surrogate-network oracle: torch's float64 autograd (a library routine), central finite
differences, and the sign-descent special case of Adam."""
import numpy as np
import pytest
import torch

from oracle import mlp
import workloads


def _torch_net(params):
    l1 = torch.nn.Linear(params["W1"].shape[1], params["W1"].shape[0]).double()
    l2 = torch.nn.Linear(params["W2"].shape[1], params["W2"].shape[0]).double()
    l3 = torch.nn.Linear(params["w3"].shape[0], 1).double()
    with torch.no_grad():
        l1.weight.copy_(torch.from_numpy(params["W1"])); l1.bias.copy_(torch.from_numpy(params["b1"]))
        l2.weight.copy_(torch.from_numpy(params["W2"])); l2.bias.copy_(torch.from_numpy(params["b2"]))
        l3.weight.copy_(torch.from_numpy(params["w3"][None, :])); l3.bias.copy_(torch.from_numpy(params["b3"].reshape(1)))
    return torch.nn.Sequential(l1, torch.nn.GELU(approximate="none"), l2, torch.nn.GELU(approximate="none"), l3), (l1, l2, l3)


def test_gelu_matches_torch():
    z = np.linspace(-8, 8, 2001)
    assert np.allclose(mlp.gelu(z), torch.nn.functional.gelu(torch.from_numpy(z)).numpy(), rtol=1e-14, atol=1e-15)
    zt = torch.from_numpy(z).requires_grad_()
    torch.nn.functional.gelu(zt).sum().backward()
    assert np.allclose(mlp.gelu_grad(z), zt.grad.numpy(), rtol=1e-13, atol=1e-15)


def test_forward_and_gradients_match_torch_autograd():
    p = workloads.mlp_init(37, 16, 12, seed=3)
    p["b1"] = np.random.default_rng(1).standard_normal(16) * 0.1
    p["b3"] = np.array(0.3)
    U = np.random.default_rng(2).standard_normal((9, 37))
    t = np.random.default_rng(5).standard_normal(9)
    L, g = mlp.loss_and_grads(p, U, t)
    net, (l1, l2, l3) = _torch_net(p)
    out = net(torch.from_numpy(U))[:, 0]
    Lt = 0.5 * ((out - torch.from_numpy(t)) ** 2).mean()
    Lt.backward()
    assert abs(L - Lt.item()) < 1e-14 * max(1, abs(L))
    pairs = [("W1", l1.weight), ("b1", l1.bias), ("W2", l2.weight), ("b2", l2.bias), ("w3", l3.weight[0]), ("b3", l3.bias[0])]
    for k, tp in pairs:
        assert np.allclose(g[k], tp.grad.numpy() if k not in ("w3", "b3") else
                           (l3.weight.grad[0].numpy() if k == "w3" else l3.bias.grad[0].numpy()), rtol=1e-11, atol=1e-14), k


def test_gradients_match_finite_differences():
    p = workloads.mlp_init(6, 5, 4, seed=8)
    U = np.random.default_rng(3).standard_normal((7, 6))
    t = np.random.default_rng(4).standard_normal(7)
    _, g = mlp.loss_and_grads(p, U, t)
    h = 1e-6
    for k in ("W1", "b1", "W2", "w3", "b3"):
        flat = p[k].reshape(-1)
        for idx in range(0, flat.size, max(1, flat.size // 5)):
            old = flat[idx]
            flat[idx] = old + h
            Lp, _ = mlp.loss_and_grads(p, U, t)
            flat[idx] = old - h
            Lm, _ = mlp.loss_and_grads(p, U, t)
            flat[idx] = old
            fd = (Lp - Lm) / (2 * h)
            assert abs(fd - g[k].reshape(-1)[idx]) < 1e-7 * max(1.0, abs(fd)), (k, idx)


def test_adam_without_moment_memory_is_sign_descent():
    """beta1 = beta2 = 0, eps -> 0: m = g, v = g^2, so the update is -lr * sign(g)."""
    rng = np.random.default_rng(0)
    params = {"a": rng.standard_normal(20)}
    grads = {"a": rng.standard_normal(20)}
    m = {"a": np.zeros(20)}
    v = {"a": np.zeros(20)}
    before = params["a"].copy()
    mlp.adam_step(params, grads, m, v, t=1, lr=0.01, beta1=0.0, beta2=0.0, eps=0.0)
    assert np.allclose(params["a"], before - 0.01 * np.sign(grads["a"]), rtol=0, atol=1e-15)


def test_adam_matches_torch_optim_adam_over_several_steps():
    """oracle.mlp.adam_step against the library routine torch.optim.Adam (Kingma & Ba 2015, bias-corrected
    moments), FP64, over five steps with different gradients, beta1 != beta2 and a non-negligible eps, so that
    swapping beta1 and beta2, an off-by-one in the bias-correction exponent t or eps inside the square root all
    fail."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    shapes = {"W1": (4, 6), "b1": (4,), "w3": (4,)}
    params = {k: rng.standard_normal(s) for k, s in shapes.items()}
    tparams = {k: torch.tensor(v.copy(), dtype=torch.float64, requires_grad=True) for k, v in params.items()}
    lr, b1, b2, eps = 3e-2, 0.8, 0.95, 1e-3
    opt = torch.optim.Adam(list(tparams.values()), lr=lr, betas=(b1, b2), eps=eps)
    m = {k: np.zeros(s) for k, s in shapes.items()}
    v = {k: np.zeros(s) for k, s in shapes.items()}
    for t in range(1, 6):
        grads = {k: rng.standard_normal(s) * (0.1 * t) for k, s in shapes.items()}
        mlp.adam_step(params, grads, m, v, t, lr=lr, beta1=b1, beta2=b2, eps=eps)
        opt.zero_grad()
        for k in shapes:
            tparams[k].grad = torch.tensor(grads[k], dtype=torch.float64)
        opt.step()
        for k in shapes:
            assert np.allclose(params[k], tparams[k].detach().numpy(), rtol=1e-13, atol=1e-15), (t, k)
