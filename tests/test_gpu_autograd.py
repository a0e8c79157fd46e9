"""Differentiable pair: Project/Backproject autograd functions, gradient checks
against central finite differences and the FP64 oracle gradient, and
least-squares gradient descent on ||P x - y||^2 (512 x 512 x 64 ellipsoid
phantom, 720 angles, 512-pixel detector, Gaussian noise sigma = 1e-2)."""
import numpy as np
import pytest
import torch

import oracle
import synth
import synth.gpu as sgpu
import paper_2209_08450_gb300 as tcp
from paper_2209_08450_gb300 import autograd as ag

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def ellipsoid_volume(n, nz, seed):
    rng = np.random.default_rng(seed)
    ells = synth.random_ellipsoids(rng, 64, n, nz_extent=float(nz))
    zs = np.arange(nz) + 0.5 - nz / 2.0
    return sgpu.rasterize_ellipsoids(ells, n, zs, device=DEV).double().cpu().numpy()


def test_backward_of_each_is_the_other():
    rng = np.random.default_rng(0)
    n, nd, nt = 48, 53, 31
    theta = rng.uniform(0, np.pi, nt)
    x = torch.tensor(rng.normal(size=(2, n, n)), dtype=torch.float32, device=DEV, requires_grad=True)
    g = torch.tensor(rng.normal(size=(2, nt, nd)), dtype=torch.float32, device=DEV)
    y = ag.radon(x, theta, 24.2, nd)
    (gx,) = torch.autograd.grad(y, x, g)
    assert torch.allclose(gx, tcp.backproject(g, theta, 24.2, n=n), atol=0, rtol=0)
    s = torch.tensor(rng.normal(size=(2, nt, nd)), dtype=torch.float32, device=DEV, requires_grad=True)
    v = ag.radon_t(s, theta, 24.2, n)
    h = torch.tensor(rng.normal(size=(2, n, n)), dtype=torch.float32, device=DEV)
    (gs,) = torch.autograd.grad(v, s, h)
    assert torch.allclose(gs, tcp.project(h, theta, 24.2, ndet=nd), atol=0, rtol=0)


def test_gradient_matches_fp64_oracle_and_finite_differences():
    n, nz, nt, nd = 512, 64, 720, 512
    theta = synth.uniform_theta(nt)
    c = nd / 2.0
    xt = ellipsoid_volume(n, nz, 4)
    x_true = torch.tensor(xt, dtype=torch.float32, device=DEV)
    g = torch.Generator(device=DEV)
    g.manual_seed(0)
    y = tcp.project(x_true, theta, c, ndet=nd)
    y = y + 1e-2 * torch.randn(y.shape, generator=g, device=DEV)
    x = (0.5 * x_true + 0.1 * torch.rand(x_true.shape, generator=g, device=DEV)).requires_grad_(True)

    def loss_of(v):
        return torch.sum((ag.radon(v, theta, c, nd).double() - y.double()) ** 2)

    L = loss_of(x)
    (grad,) = torch.autograd.grad(L, x)
    # FP64 oracle gradient 2 P^T (P x - y) on two slices
    for z in (0, 37):
        xz = x[z].detach().double().cpu().numpy()
        yz = y[z].double().cpu().numpy()
        r = oracle.project(xz, theta, c, nd)[0] - yz
        ref = 2.0 * oracle.backproject(r, theta, c, n)[0]
        got = grad[z].double().cpu().numpy()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5
    # Central differences along seeded directions.  L is quadratic, so the
    # difference quotient has no truncation error: what is left is the FP32
    # rounding of the two projections (sums of ~10^3 terms of size ~0.5, so
    # ~1e-3 absolute per projection value), which enters the loss difference
    # as ~2 |r| 1e-3 sqrt(#values) / (2 eps): ~1e-3 of the derivative at
    # eps = 1e-3.  v has O(1) entries so that eps * v is far above the FP32
    # resolution of x.
    for k in range(3):
        v = torch.randn(x.shape, generator=g, device=DEV)
        dd = float(torch.sum(grad.double() * v.double()))
        for eps, tol in ((1e-3, 3e-3), (1e-2, 1e-3)):
            with torch.no_grad():
                fd = float((loss_of(x + eps * v) - loss_of(x - eps * v)) / (2 * eps))
            assert abs(fd - dd) <= tol * abs(dd), (eps, fd, dd)


def test_least_squares_gradient_descent_matches_fp64_and_converges():
    # small case: 50 iterations on the GPU vs the same iteration in FP64
    n, nt, nd = 48, 60, 48
    theta = synth.uniform_theta(nt)
    c = nd / 2.0
    x_true = ellipsoid_volume(n, 2, 1)
    y = oracle.project(x_true, theta, c, nd)
    y += 1e-2 * np.random.default_rng(0).normal(size=y.shape)
    yd = torch.tensor(y, dtype=torch.float32, device=DEV)
    L = 2.0 * ag.operator_norm_sq((1, n, n), theta, c, nd, iters=40)
    step = 1.0 / L
    losses = []
    xg = ag.lsq_gradient_descent(yd, theta, c, n, iters=50, step=step, callback=lambda i, l: losses.append(l))
    xo = np.zeros_like(x_true)
    for _ in range(50):
        xo -= step * 2.0 * oracle.backproject(oracle.project(xo, theta, c, nd) - y, theta, c, n)
    got = xg.double().cpu().numpy()
    assert np.linalg.norm(got - xo) / np.linalg.norm(xo) <= 1e-4
    assert all(b <= a * (1 + 1e-6) for a, b in zip(losses, losses[1:]))
    assert losses[-1] < 0.05 * losses[0]


def test_least_squares_full_size_50_iterations():
    n, nz, nt, nd = 512, 64, 720, 512
    theta = synth.uniform_theta(nt)
    c = nd / 2.0
    x_true = torch.tensor(ellipsoid_volume(n, nz, 4), dtype=torch.float32, device=DEV)
    g = torch.Generator(device=DEV)
    g.manual_seed(1)
    y = tcp.project(x_true, theta, c, ndet=nd)
    y = y + 1e-2 * torch.randn(y.shape, generator=g, device=DEV)
    losses = []
    x = ag.lsq_gradient_descent(y, theta, c, n, iters=50, callback=lambda i, l: losses.append(l))
    assert all(b <= a * (1 + 1e-5) for a, b in zip(losses, losses[1:]))
    assert losses[-1] < 0.02 * losses[0]
    err0 = float(x_true.norm())
    assert float((x - x_true).norm()) < 0.8 * err0
