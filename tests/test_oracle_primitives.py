"""Pins of the oracle's building blocks against closed forms, algebraic
identities and library routines (cutoff, expnorm basis, I/A/S decomposition,
edge basis, LayerNorm, SiLU, channel mixing)."""
import math

import numpy as np
import pytest
import torch

from oracle import tensornet as tn

RC = 5.0


def test_cosine_cutoff_closed_forms():
    assert tn.cosine_cutoff(np.array([0.0]), RC)[0] == 1.0
    assert abs(tn.cosine_cutoff(np.array([RC / 2]), RC)[0] - 0.5) < 1e-15
    assert tn.cosine_cutoff(np.array([RC]), RC)[0] == 0.0
    assert tn.cosine_cutoff(np.array([RC + 1.0]), RC)[0] == 0.0
    # phi(rc - eps) = (1 - cos(pi eps / rc)) / 2 = sin^2(pi eps / (2 rc))
    eps = 1e-2
    assert abs(tn.cosine_cutoff(np.array([RC - eps]), RC)[0] - math.sin(math.pi * eps / (2 * RC)) ** 2) < 1e-15
    # derivative: vanishes at both ends, matches central differences inside
    assert abs(tn.cosine_cutoff_grad(np.array([RC - 1e-12]), RC)[0]) < 1e-11
    d = np.linspace(0.1, 4.9, 17)
    h = 1e-6
    fd = (tn.cosine_cutoff(d + h, RC) - tn.cosine_cutoff(d - h, RC)) / (2 * h)
    assert np.allclose(tn.cosine_cutoff_grad(d, RC), fd, atol=1e-9)


def test_expnorm_special_values():
    K = 32
    mu, beta, alpha = tn.expnorm_params(RC, 0.0, K)
    assert alpha == 1.0
    assert abs(mu[0] - math.exp(-5.0)) < 1e-16 and mu[-1] == 1.0
    assert np.allclose(np.diff(mu), (1 - math.exp(-5.0)) / (K - 1))
    # beta^(-1/2) = (2/K)(1 - exp(-5)): twice the basis spacing times (K-1)/K
    assert abs(beta ** -0.5 - (2.0 / K) * (1 - math.exp(-5.0))) < 1e-15
    e, _ = tn.expnorm(np.array([0.0, RC, RC + 0.5]), RC, 0.0, K)
    assert e[0, -1] == 1.0                      # exp(-0) = 1 = mu_{K-1}, phi(0) = 1
    assert np.all(e[1:] == 0.0)                 # phi vanishes at and beyond rc
    assert np.all(np.diff(e[0]) > 0)            # at d = 0 the last centre is closest


def test_expnorm_peaks_at_centres():
    """Without the cutoff factor the k-th function peaks where exp(-d) = mu_k."""
    K = 32
    mu, _, _ = tn.expnorm_params(RC, 0.0, K)
    d = np.linspace(1e-4, RC - 1e-4, 400001)
    e, _ = tn.expnorm(d, RC, 0.0, K)
    rho = e / tn.cosine_cutoff(d, RC)[:, None]
    for k in range(8, K - 1):  # centres strictly inside (0, rc)
        dk = -math.log(mu[k])
        assert abs(d[np.argmax(rho[:, k])] - dk) < 2e-5


def test_expnorm_derivative():
    d = np.linspace(0.3, 4.95, 41)
    h = 1e-6
    ep, _ = tn.expnorm(d + h, RC, 0.0, 32)
    em, _ = tn.expnorm(d - h, RC, 0.0, 32)
    _, de = tn.expnorm(d, RC, 0.0, 32)
    assert np.allclose(de, (ep - em) / (2 * h), atol=1e-7, rtol=1e-6)


def test_decomposition_identities():
    rng = np.random.default_rng(0)
    X = rng.standard_normal((7, 5, 3, 3))
    I, A, S = tn.decompose(X)
    assert np.allclose(I + A + S, X)
    assert np.allclose(np.trace(S, axis1=-2, axis2=-1), 0)
    assert np.allclose(A, -np.swapaxes(A, -1, -2))
    assert np.allclose(S, np.swapaxes(S, -1, -2))
    assert np.allclose(I, np.trace(X, axis1=-2, axis2=-1)[..., None, None] / 3 * np.eye(3))
    # orthogonal split: the squared norms add up
    assert np.allclose(tn.tensor_norm(X), tn.tensor_norm(I) + tn.tensor_norm(A) + tn.tensor_norm(S))
    # projections are idempotent
    for k, P in enumerate((I, A, S)):
        assert np.allclose(tn.decompose(P)[k], P)
    # adjoint: <decompose(X)_q, G_q> summed = <X, decompose_adjoint(G)>
    G = [rng.standard_normal(X.shape) for _ in range(3)]
    lhs = sum(np.sum(p * g) for p, g in zip((I, A, S), G))
    rhs = np.sum(X * tn.decompose_adjoint(*G))
    assert abs(lhs - rhs) < 1e-10


def test_edge_basis():
    rng = np.random.default_rng(1)
    u = rng.standard_normal((50, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    v = rng.standard_normal((50, 3))
    I0, A0, S0 = tn.edge_basis(u)
    assert np.allclose(I0, np.eye(3))
    assert np.allclose(np.einsum("eab,eb->ea", A0, v), np.cross(u, v))
    assert np.allclose(np.trace(S0, axis1=1, axis2=2), 0)
    assert np.allclose(np.einsum("eab,eb->ea", S0, u), 2.0 / 3.0 * u)
    w = np.cross(u, v)  # perpendicular to u
    assert np.allclose(np.einsum("eab,eb->ea", S0, w), -w / 3.0)
    # the three basis matrices are exactly the I, A and S parts of u u^T + [u]_x + Id
    parts = tn.decompose(I0 + A0 + S0)
    for P, Q in zip(parts, (I0, A0, S0)):
        assert np.allclose(P, Q)


@pytest.mark.parametrize("reflect", [False, True])
def test_edge_basis_transforms_under_o3(reflect):
    """Covariance of the edge basis under an orthogonal R: R S0(u) R^T =
    S0(R u), while the skew part is a pseudo-tensor, R A0(u) R^T =
    det(R) A0(R u) (it flips sign under a reflection, which the O(3) energy
    sees only through squared norms and products of two skew parts)."""
    rng = np.random.default_rng(7)
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    R = Q @ np.diag([1.0, 1.0, -1.0]) if reflect else Q
    u = rng.standard_normal((20, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    _, A0, S0 = tn.edge_basis(u)
    _, A1, S1 = tn.edge_basis(u @ R.T)
    det = np.linalg.det(R)
    assert math.isclose(abs(det), 1.0, rel_tol=1e-12) and (det < 0) == reflect
    assert np.allclose(R @ S0 @ R.T, S1, atol=1e-13)
    assert np.allclose(R @ A0 @ R.T, det * A1, atol=1e-13)


def test_layer_norm_silu_match_torch():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((6, 40))
    g = rng.uniform(0.5, 1.5, 40)
    b = rng.uniform(-0.1, 0.1, 40)
    y, _ = tn.layer_norm(x, g, b)
    ref = torch.nn.functional.layer_norm(torch.tensor(x), (40,), torch.tensor(g), torch.tensor(b), eps=1e-5)
    assert np.allclose(y, ref.numpy(), atol=1e-12)
    assert np.allclose(tn.silu(x), torch.nn.functional.silu(torch.tensor(x)).numpy(), atol=1e-15)
    xt = torch.tensor(x, requires_grad=True)
    torch.nn.functional.silu(xt).sum().backward()
    assert np.allclose(tn.silu_grad(x), xt.grad.numpy(), atol=1e-14)
    # LayerNorm adjoint vs torch autograd
    gy = rng.standard_normal((6, 40))
    xt = torch.tensor(x, requires_grad=True)
    gt = torch.tensor(g, requires_grad=True)
    bt = torch.tensor(b, requires_grad=True)
    torch.nn.functional.layer_norm(xt, (40,), gt, bt, eps=1e-5).backward(torch.tensor(gy))
    _, cache = tn.layer_norm(x, g, b)
    gx, gg, gb = tn.layer_norm_adjoint(gy, g, cache)
    assert np.allclose(gx, xt.grad.numpy(), atol=1e-12)
    assert np.allclose(gg, gt.grad.numpy(), atol=1e-12)
    assert np.allclose(gb, bt.grad.numpy(), atol=1e-12)


def test_mix_is_channel_linear():
    rng = np.random.default_rng(3)
    W = rng.standard_normal((4, 4))
    P = rng.standard_normal((2, 4, 3, 3))
    U = tn.mix(W, P)
    for n in range(2):
        for c in range(4):
            ref = sum(W[c, d] * P[n, d] for d in range(4))
            assert np.allclose(U[n, c], ref)


def test_segment_sum():
    idx = np.array([2, 0, 2, 2, 4])
    vals = np.arange(10.0).reshape(5, 2)
    out = tn.segment_sum(idx, vals, 6)
    ref = np.zeros((6, 2))
    for e, k in enumerate(idx):
        ref[k] += vals[e]
    assert np.array_equal(out, ref)
