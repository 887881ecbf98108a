"""The differentiable EM update and the unrolled network, checked on CPU in FP64
with the oracle standing in for A / A' and for the element-wise EM steps (the
ratio and the closed-form update with their hand-derived gradients), through
torch.autograd.gradcheck.  The library's own element-wise kernels are compared
with the same oracle functions on the GPU (tests/test_gpu_autograd.py)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2301_09710_gb300.autograd as ag
from paper_2301_09710_gb300 import synthetic


class _OA(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, args):
        ctx.args = args
        return torch.from_numpy(oracle.forward(x.detach().numpy(), *args, nthreads=1))

    @staticmethod
    def backward(ctx, g):
        return torch.from_numpy(oracle.back(g.detach().numpy(), *ctx.args, nthreads=1)), None


class _OB(torch.autograd.Function):
    @staticmethod
    def forward(ctx, v, args):
        ctx.args = args
        return torch.from_numpy(oracle.back(v.detach().numpy(), *args, nthreads=1))

    @staticmethod
    def backward(ctx, g):
        return torch.from_numpy(oracle.forward(g.detach().numpy(), *ctx.args, nthreads=1)), None


class _ORatio(torch.autograd.Function):
    @staticmethod
    def forward(ctx, ybar, y, rbar):
        ctx.save_for_backward(ybar, y, rbar)
        r = None if rbar is None else rbar.detach().numpy()
        return torch.from_numpy(oracle.em_ratio(ybar.detach().numpy(), y.detach().numpy(), r))

    @staticmethod
    def backward(ctx, g):
        ybar, y, rbar = ctx.saved_tensors
        r = None if rbar is None else rbar.numpy()
        return torch.from_numpy(oracle.em_ratio_vjp(ybar.numpy(), y.numpy(), r, g.numpy())), None, None


class _ORoot(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, e, s, u, beta):
        ctx.beta = beta
        ctx.save_for_backward(x, e, s, u)
        un = None if u is None else u.detach().numpy()
        return torch.from_numpy(oracle.em_root(x.detach().numpy(), e.detach().numpy(), s.detach().numpy(), un,
                                               beta))

    @staticmethod
    def backward(ctx, g):
        x, e, s, u = ctx.saved_tensors
        un = None if u is None else u.numpy()
        gx, ge, gu = oracle.em_root_vjp(x.numpy(), e.numpy(), s.numpy(), un, ctx.beta, g.numpy())
        return (torch.from_numpy(gx), torch.from_numpy(ge), None,
                None if u is None else torch.from_numpy(gu), None)


def use_oracle_em(monkeypatch):
    """The element-wise EM steps of autograd.em_update on the FP64 oracle."""
    monkeypatch.setattr(ag, "em_ratio", lambda ybar, y, rbar: _ORatio.apply(ybar, y, rbar))
    monkeypatch.setattr(ag, "em_root", lambda x, e, s, u, beta: _ORoot.apply(x, e, s, u, beta))


@pytest.fixture
def tiny(monkeypatch):
    prob = synthetic.random_problem(21, nx=6, nz=3, nview=4, px=3, pz=3, mu_scale=0.1)
    args = (prob.mu.astype(np.float64), prob.psf.astype(np.float64), 1.0, oracle.default_angles(4))
    monkeypatch.setattr(ag, "project", lambda x, plan: _OA.apply(x, args))
    monkeypatch.setattr(ag, "backproject", lambda v, plan: _OB.apply(v, args))
    use_oracle_em(monkeypatch)
    rng = np.random.default_rng(21)
    y = torch.from_numpy(rng.poisson(4.0, (4, 3, 6)).astype(np.float64))
    s = torch.from_numpy(oracle.sensitivity(*args))
    return prob, args, y, s


@pytest.mark.parametrize("beta", [0.0, 0.3, 30.0])
def test_em_update_gradcheck(tiny, beta):
    prob, args, y, s = tiny
    rng = np.random.default_rng(22)
    x = torch.from_numpy(rng.uniform(0.5, 2.0, prob.x.shape)).requires_grad_(True)
    u = torch.from_numpy(rng.uniform(0.5, 2.0, prob.x.shape)).requires_grad_(beta > 0)
    rbar = torch.full_like(y, 0.2)
    if beta > 0:
        assert torch.autograd.gradcheck(lambda a, b: ag.em_update(a, y, rbar, None, s, b, beta), (x, u),
                                        eps=1e-6, atol=1e-7, rtol=1e-5)
    else:
        assert torch.autograd.gradcheck(lambda a: ag.em_update(a, y, rbar, None, s), (x,),
                                        eps=1e-6, atol=1e-7, rtol=1e-5)


def test_em_update_forward_matches_oracle(tiny):
    prob, args, y, s = tiny
    rng = np.random.default_rng(23)
    x = rng.uniform(0.5, 2.0, prob.x.shape)
    u = rng.uniform(0.5, 2.0, prob.x.shape)
    rbar = np.full(y.shape, 0.2)
    got = ag.em_update(torch.from_numpy(x), y, torch.from_numpy(rbar), None, s, torch.from_numpy(u), 0.7)
    want = oracle.em_step_reg(x, y.numpy(), rbar, u, 0.7, *args)
    np.testing.assert_allclose(got.numpy(), want, rtol=1e-12)


def test_unrolled_network_gradcheck_and_checkpoint_equivalence(tiny):
    prob, args, y, s = tiny
    torch.manual_seed(1)
    cnn = ag.Regularizer3D(channels=2).double()
    for p in cnn.parameters():
        torch.nn.init.normal_(p, std=0.1)
    net = ag.UnrolledEM(None, n_outer=2, n_inner=1, beta=0.5, cnn=cnn)
    net._s = s
    x0 = torch.ones(prob.x.shape, dtype=torch.float64)
    target = torch.from_numpy(prob.x.astype(np.float64))
    # checkpointed and plain unrolling give the same loss and gradients
    l1 = ((net(x0, y) - target) ** 2).mean()
    g1 = torch.autograd.grad(l1, list(cnn.parameters()))
    net.checkpoint = False
    l2 = ((net(x0, y) - target) ** 2).mean()
    g2 = torch.autograd.grad(l2, list(cnn.parameters()))
    assert torch.allclose(l1, l2, rtol=0, atol=0)
    for a, b in zip(g1, g2):
        assert torch.allclose(a, b, rtol=1e-12, atol=1e-15)
    # gradcheck wrt the last layer's weights
    w0 = cnn.c3.weight.detach().clone().requires_grad_(True)

    assert torch.autograd.gradcheck(
        lambda wt: ((_unroll_with_w3(net, cnn, wt, x0, y)) - target).pow(2).mean(), (w0,), eps=1e-6, atol=1e-7,
        rtol=1e-5)


def _unroll_with_w3(net, cnn, w3, x0, y):
    x = x0
    for _ in range(net.n_outer):
        h = torch.relu(cnn.c1(x[None, None]))
        h = torch.relu(cnn.c2(h))
        u = x + torch.nn.functional.conv3d(h, w3, cnn.c3.bias, padding=1)[0, 0]
        x = ag.em_update(x, y, None, None, net._s, u, net.beta)
    return x

