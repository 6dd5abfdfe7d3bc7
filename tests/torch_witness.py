"""Independent float64 restatement of the TensorNet energy in plain PyTorch,
differentiated by autograd.  Test-only: it pins the oracle's hand-derived
reverse pass (forces and weight gradients).  It follows the same model
readings as the oracle (see the oracle's module header), written from the
model description rather than from the oracle's code."""
import math

import torch


def _silu(x):
    return torch.nn.functional.silu(x)


def _cross_matrix(u):
    z = torch.zeros_like(u[:, 0])
    return torch.stack([torch.stack([z, -u[:, 2], u[:, 1]], -1),
                        torch.stack([u[:, 2], z, -u[:, 0]], -1),
                        torch.stack([-u[:, 1], u[:, 0], z], -1)], -2)


def _parts(X):
    eye = torch.eye(3, dtype=X.dtype)
    tr = X.diagonal(dim1=-2, dim2=-1).sum(-1)
    I = tr[..., None, None] * eye / 3
    A = (X - X.transpose(-1, -2)) / 2
    S = (X + X.transpose(-1, -2)) / 2 - I
    return I, A, S


def _sqnorm(X):
    return (X ** 2).sum((-1, -2))


def _channel_linear(W, X):
    return torch.einsum("cd,ndab->ncab", W, X)


def energy(params, z, pos, batch, box, i, j, F, K, L, rc=5.0, rl=0.0):
    """Per-system energies.  params: dict of float64 tensors (may require
    grad); pos: float64 tensor (may require grad)."""
    p = params
    N = pos.shape[0]
    r = pos[i] - pos[j]
    if box is not None:
        B = box[batch[i]]
        for ax in (2, 1, 0):
            r = r - torch.round(r[:, ax] / B[:, ax, ax])[:, None] * B[:, ax, :]
    d = torch.sqrt((r * r).sum(-1))
    u = r / d[:, None]
    phi = torch.where(d < rc, 0.5 * (torch.cos(math.pi * d / rc) + 1), torch.zeros_like(d))
    start = math.exp(-(rc - rl))
    mu = torch.linspace(start, 1.0, K, dtype=torch.float64)
    beta = ((2.0 / K) * (1 - start)) ** -2
    alpha = 5.0 / (rc - rl)
    e = phi[:, None] * torch.exp(-beta * (torch.exp(alpha * (rl - d))[:, None] - mu) ** 2)

    eye = torch.eye(3, dtype=torch.float64).expand(len(i), 3, 3)
    bases = (eye, _cross_matrix(u), u[:, :, None] * u[:, None, :] - torch.eye(3, dtype=torch.float64) / 3)
    emb = p["emb"][z]
    Zij = torch.cat([emb[i], emb[j]], 1) @ p["emb2_w"].T + p["emb2_b"]
    raw = []
    for q in range(3):
        fq = e @ p["dproj_w"][q].T + p["dproj_b"][q]
        cq = (phi[:, None] * Zij * fq)[:, :, None, None] * bases[q][:, None]
        raw.append(torch.zeros(N, F, 3, 3, dtype=torch.float64).index_add(0, i, cq))
    nrm = torch.nn.functional.layer_norm(_sqnorm(raw[0] + raw[1] + raw[2]), (F,),
                                         p["emb_ln_g"], p["emb_ln_b"], eps=1e-5)
    s = _silu(_silu(nrm @ p["emb_mlp1_w"].T + p["emb_mlp1_b"]) @ p["emb_mlp2_w"].T + p["emb_mlp2_b"])
    s = s.reshape(N, F, 3)
    X = sum(s[:, :, q, None, None] * _channel_linear(p["emb_mix_w"][q], raw[q]) for q in range(3))

    for l in range(L):
        X = X / (_sqnorm(X) + 1)[..., None, None]
        prt = _parts(X)
        Yq = [_channel_linear(p[f"l{l}_mix1_w"][q], prt[q]) for q in range(3)]
        h = _silu(e @ p[f"l{l}_mlp1_w"].T + p[f"l{l}_mlp1_b"])
        h = _silu(h @ p[f"l{l}_mlp2_w"].T + p[f"l{l}_mlp2_b"])
        h = _silu(h @ p[f"l{l}_mlp3_w"].T + p[f"l{l}_mlp3_b"])
        g = (phi[:, None] * h).reshape(-1, F, 3)
        msg = sum(g[:, :, q, None, None] * Yq[q][j] for q in range(3))
        M = torch.zeros(N, F, 3, 3, dtype=torch.float64).index_add(0, i, msg)
        Y = Yq[0] + Yq[1] + Yq[2]
        T = Y @ M + M @ Y
        tp = _parts(T)
        den = (_sqnorm(tp[0] + tp[1] + tp[2]) + 1)[..., None, None]
        dX = sum(_channel_linear(p[f"l{l}_mix2_w"][q], tp[q] / den) for q in range(3))
        X = X + dX + dX @ dX

    I, A, S = _parts(X)
    hcat = torch.cat([_sqnorm(I), _sqnorm(A), _sqnorm(S)], 1)
    hcat = torch.nn.functional.layer_norm(hcat, (3 * F,), p["out_ln_g"], p["out_ln_b"], eps=1e-5)
    o = _silu(hcat @ p["out_w"].T + p["out_b"])
    Ei = (_silu(o @ p["head1_w"].T + p["head1_b"]) @ p["head2_w"].T)[:, 0] + p["head2_b"][0]
    nsys = int(batch.max()) + 1
    return torch.zeros(nsys, dtype=torch.float64).index_add(0, batch, Ei)
