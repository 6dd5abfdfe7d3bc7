"""TensorNet energy, forces and weight gradients in FP64 (plain definition).

TEST INFRASTRUCTURE ONLY (see the package header).

What is computed.  The paper (Sec. 2, "Background"; Sec. 2.1.1, TensorNet)
states the problem: positions R and embedding indices Z go in; a per-sample
scalar (the energy) and its negative gradient with respect to the positions
(the forces) come out, obtained by automatic differentiation so that the
force field is conservative.  TensorNet is an O(3)-equivariant message
passing network on rank-2 Cartesian tensors: 3x3 features are split into
their scalar (I), vector/skew (A) and symmetric-traceless (S) parts and
node-level 3x3 matrix products replace Clebsch-Gordan tensor products.  The
model is composed of a representation model, an output model giving
per-atom scalars, and a sum over the sample (Sec. 2, Fig. 1).  The hyper-
parameters follow the training example of Sec. 2.4 and Table S4: embedding
dimension F = 128, L = 2 interaction layers, K = 32 "expnorm" radial basis
functions, cosine cutoff on [0, 5] A, SiLU activation, O(3) group, max_z 100.

The layer equations themselves are not printed in the paper; this module
writes out the published TensorNet model at that shape.  Readings where the
paper is silent are listed here and marked [R] below:
  [R1] ||T|| is the squared Frobenius norm sum_ab T_ab^2.
  [R2] the expnorm basis carries the cosine cutoff as a factor.
  [R3] per-edge 3F-vectors are split channel-major: index c*3 + p with
       p = 0 (I), 1 (A), 2 (S).
  [R4] in the embedding, channel mixing comes before the scaling by s.
  [R5] the interaction residual is added to the normalised X.
  [R6] the output concatenation order is (||I||, ||A||, ||S||) in blocks.
  [R7] LayerNorm eps = 1e-5; no prior, mean 0, std 1.
  [R8] pair embedding Z_ij = W_e [emb(z_i); emb(z_j)] + b_e, receiver first.
  [R9] the edge vector is r_ij = r_i - r_j; u = r_ij / d_ij.

Representation: every tensor feature is an array [..., F, 3, 3] of full 3x3
matrices (the CUDA path uses a different, compact 9-coordinate form; the two
share nothing).

Pinned by (tests/test_oracle_*.py): closed forms of the cutoff and basis,
algebraic identities of the decomposition and edge basis, central finite
differences of the energy (forces) and of every weight tensor (weight
gradients), invariance under rotations, reflections, translations,
permutations of like atoms and periodic image shifts, zero net force,
equivariance of forces, cutoff continuity, the isolated-atom closed form,
closed forms on toy inputs of the embedding's edge-to-node sum, of the
channel-major splits, of the interaction layer's messages and node update
and of the output model's input, and an independent float64 autograd
restatement of the reverse pass.
Absolute energies of the composed network have no printed value in the
paper: parity unpinned beyond those properties.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

from .neighbors import minimum_image, neighbor_pairs

LN_EPS = 1e-5
EDGE_CHUNK = 8192


# ------------------------------------------------------------ primitives ---

def silu(x):
    return x / (1.0 + np.exp(-x))


def silu_grad(x):
    s = 1.0 / (1.0 + np.exp(-x))
    return s * (1.0 + x * (1.0 - s))


def cosine_cutoff(d, rc):
    """phi(d) = (cos(pi d / rc) + 1) / 2 for d < rc, else 0 (the phi(d_ij)
    envelope of Sec. 2.1.2, on [cutoff_lower = 0, cutoff_upper = rc])."""
    d = np.asarray(d, dtype=np.float64)
    return np.where(d < rc, 0.5 * (np.cos(math.pi * d / rc) + 1.0), 0.0)


def cosine_cutoff_grad(d, rc):
    d = np.asarray(d, dtype=np.float64)
    return np.where(d < rc, -0.5 * math.pi / rc * np.sin(math.pi * d / rc), 0.0)


def expnorm_params(rc, rl, K):
    """Fixed (non-trainable, Sec. 2.4: trainable_rbf False) expnorm centres
    mu_k and width beta, and the decay alpha = 5 / (rc - rl)."""
    start = math.exp(-(rc - rl))
    mu = np.linspace(start, 1.0, K)
    beta = ((2.0 / K) * (1.0 - start)) ** -2
    alpha = 5.0 / (rc - rl)
    return mu, beta, alpha


def expnorm(d, rc, rl, K):
    """e_k(d) = phi(d) exp(-beta (exp(alpha (rl - d)) - mu_k)^2) [R2]
    (rbf_type 'expnorm', num_rbf K; Sec. 2.4).  Returns (e [E,K], de/dd)."""
    mu, beta, alpha = expnorm_params(rc, rl, K)
    d = np.asarray(d, dtype=np.float64)[:, None]
    ex = np.exp(alpha * (rl - d))
    rho = np.exp(-beta * (ex - mu[None, :]) ** 2)
    phi = cosine_cutoff(d, rc)
    dphi = cosine_cutoff_grad(d, rc)
    drho = rho * (-2.0 * beta * (ex - mu[None, :])) * (-alpha * ex)
    return phi * rho, dphi * rho + phi * drho


def edge_basis(u):
    """I0 = Id, A0 = [u]_x (A0 v = u x v), S0 = u u^T - Id/3, each [E,3,3]."""
    E = u.shape[0]
    I0 = np.broadcast_to(np.eye(3), (E, 3, 3)).copy()
    A0 = np.zeros((E, 3, 3))
    A0[:, 0, 1] = -u[:, 2]
    A0[:, 0, 2] = u[:, 1]
    A0[:, 1, 0] = u[:, 2]
    A0[:, 1, 2] = -u[:, 0]
    A0[:, 2, 0] = -u[:, 1]
    A0[:, 2, 1] = u[:, 0]
    S0 = u[:, :, None] * u[:, None, :] - np.eye(3) / 3.0
    return I0, A0, S0


def decompose(X):
    """X = I + A + S: I = (tr X / 3) Id, A = (X - X^T)/2, S = (X + X^T)/2 - I
    (the scalar / vector / rank-2 split of Sec. 2.1.1)."""
    tr = np.trace(X, axis1=-2, axis2=-1)
    I = tr[..., None, None] / 3.0 * np.eye(3)
    Xt = np.swapaxes(X, -1, -2)
    A = 0.5 * (X - Xt)
    S = 0.5 * (X + Xt) - I
    return I, A, S


def decompose_adjoint(gI, gA, gS):
    """Adjoint of `decompose`: each part is an orthogonal (self-adjoint)
    projection, so dE/dX = P_I(gI) + P_A(gA) + P_S(gS)."""
    return decompose(gI)[0] + decompose(gA)[1] + decompose(gS)[2]


def tensor_norm(X):
    """||X|| = sum_ab X_ab^2 per channel [R1]."""
    return np.sum(X * X, axis=(-2, -1))


def mix(W, P):
    """Channel mixing (a bias-free Linear over the channel axis applied to
    every matrix entry): U[n, c] = sum_c' W[c, c'] P[n, c']."""
    N, F = P.shape[:2]
    return np.matmul(W, P.reshape(N, F, 9)).reshape(N, F, 3, 3)


def mix_adjoint(W, gU, P):
    """Returns (dE/dP, dE/dW) for U = mix(W, P)."""
    N, F = gU.shape[:2]
    g2 = gU.reshape(N, F, 9)
    gP = np.matmul(W.T, g2).reshape(N, F, 3, 3)
    gW = np.einsum("ncx,ndx->cd", g2, P.reshape(N, F, 9))
    return gP, gW


def layer_norm(x, g, b):
    mu = x.mean(-1, keepdims=True)
    var = ((x - mu) ** 2).mean(-1, keepdims=True)
    rstd = 1.0 / np.sqrt(var + LN_EPS)
    xh = (x - mu) * rstd
    return xh * g + b, (xh, rstd)


def layer_norm_adjoint(gy, g, cache):
    xh, rstd = cache
    gxh = gy * g
    gx = rstd * (gxh - gxh.mean(-1, keepdims=True) - xh * (gxh * xh).mean(-1, keepdims=True))
    return gx, (gy * xh).sum(0), gy.sum(0)


def segment_sum(index, values, n):
    """out[k] = sum of values[e] over e with index[e] == k (a sparse
    matrix-vector product used as a plain segmented sum)."""
    E = values.shape[0]
    if E == 0:
        return np.zeros((n,) + values.shape[1:])
    S = sp.csr_matrix((np.ones(E), (index, np.arange(E))), shape=(n, E))
    return np.asarray(S @ values.reshape(E, -1)).reshape((n,) + values.shape[1:])


# --------------------------------------------------------------- model ---

class TensorNet:
    """FP64 TensorNet with the parameters of `synth.init_weights` (names and
    (out, in) Linear layout of `synth.param_spec`)."""

    def __init__(self, params: dict, F=128, K=32, L=2, rc=5.0, rl=0.0):
        self.p = {k: np.asarray(v, dtype=np.float64) for k, v in params.items()}
        self.F, self.K, self.L, self.rc, self.rl = F, K, L, float(rc), float(rl)

    # -------------------------------------------------------- geometry ---
    def geometry(self, pos, batch, box, i, j):
        pos = np.asarray(pos, dtype=np.float64)
        r = pos[i] - pos[j]
        if box is not None:
            B = np.asarray(box, np.float64)
            bi = np.asarray(batch)[i]
            for s in np.unique(bi):
                sel = bi == s
                r[sel] = minimum_image(r[sel], B[s])
        d = np.linalg.norm(r, axis=1)
        u = r / d[:, None]
        return r, d, u

    def edge_filter(self, l, e, phi):
        """g_ij = phi(d) SiLU(W3 SiLU(W2 SiLU(W1 e + b1) + b2) + b3), split
        channel-major [R3] into [E, F, 3]."""
        p = self.p
        a1 = e @ p[f"l{l}_mlp1_w"].T + p[f"l{l}_mlp1_b"]
        h1 = silu(a1)
        a2 = h1 @ p[f"l{l}_mlp2_w"].T + p[f"l{l}_mlp2_b"]
        h2 = silu(a2)
        a3 = h2 @ p[f"l{l}_mlp3_w"].T + p[f"l{l}_mlp3_b"]
        h3 = silu(a3)
        g = phi[:, None] * h3
        return g.reshape(-1, self.F, 3), (a1, h1, a2, h2, a3, h3)

    # ----------------------------------------------- interaction layer ---
    def interaction(self, l, X, e, phi, i, j):
        """Interaction layer l (Sec. 2.1.1) on node tensors X [N, F, 3, 3]:
        X <- X / (||X|| + 1) per channel [R1]; (I, A, S) = decomp(X);
        Y^P = W^P_{l,1} P (one bias-free channel mixing per part P); Y = the
        sum of the three; messages M (see `messages`); then `node_update`.
        Returns (X_out, cache of the layer's intermediates)."""
        qn = tensor_norm(X)
        Xn = X / (qn + 1.0)[..., None, None]
        parts = decompose(Xn)
        Yp = [mix(self.p[f"l{l}_mix1_w"][q], parts[q]) for q in range(3)]
        Y = Yp[0] + Yp[1] + Yp[2]
        M = self.messages(l, e, phi, i, j, Yp, X.shape[0])
        Xout, post = self.node_update(l, Xn, Y, M)
        return Xout, dict(X=X, qn=qn, Xn=Xn, parts=parts, Yp=Yp, Y=Y, M=M, **post)

    def messages(self, l, e, phi, i, j, Yp, N):
        """M_i = sum over the edges (i, j) of g^I_ij Y^I_j + g^A_ij Y^A_j +
        g^S_ij Y^S_j, per channel: the receiver i collects its neighbours'
        parts weighted by the radial filters of `edge_filter`."""
        F, E = self.F, len(i)
        M = np.zeros((N, F, 3, 3))
        for a in range(0, E, EDGE_CHUNK):
            sl = slice(a, min(E, a + EDGE_CHUNK))
            g, _ = self.edge_filter(l, e[sl], phi[sl])
            js = j[sl]
            vals = sum(g[:, :, q, None, None] * Yp[q][js] for q in range(3))
            M += segment_sum(i[sl], vals, N)
        return M

    def node_update(self, l, Xn, Y, M):
        """Node part after the messages: T = Y M + M Y (the O(3) product, per
        channel); (I, A, S) = decomp(T) / (||T|| + 1); dX = sum_P W^P_{l,2} P;
        X_out = Xn + dX + dX dX, the residual on the normalised X [R5].
        Returns (X_out, {T: the parts of T, pn: ||T||, Tn: the scaled parts,
        dX})."""
        T = np.matmul(Y, M) + np.matmul(M, Y)                         # O(3)
        TI, TA, TS = decompose(T)
        pn = tensor_norm(TI + TA + TS)
        den = (pn + 1.0)[..., None, None]
        Tn = (TI / den, TA / den, TS / den)
        dX = sum(mix(self.p[f"l{l}_mix2_w"][q], Tn[q]) for q in range(3))
        Xout = Xn + dX + np.matmul(dX, dX)                            # [R5]
        return Xout, dict(T=(TI, TA, TS), pn=pn, Tn=Tn, dX=dX)

    # --------------------------------------------------------- forward ---
    def forward(self, z, pos, batch, box, pairs=None, n_systems=None):
        """Returns (E_s [S], E_i [N], cache)."""
        p, F = self.p, self.F
        z = np.asarray(z)
        batch = np.asarray(batch)
        N = len(z)
        S_ = int(batch.max()) + 1 if n_systems is None else n_systems
        if pairs is None:
            pairs = neighbor_pairs(pos, batch, box, self.rc)
        i, j = (np.asarray(a, dtype=np.int64) for a in pairs)
        E = len(i)
        r, d, u = self.geometry(pos, batch, box, i, j)
        phi = cosine_cutoff(d, self.rc)
        e, _ = expnorm(d, self.rc, self.rl, self.K)
        I0, A0, S0 = edge_basis(u)
        basis = (I0, A0, S0)

        # embedding: Z_ij [R8], f^P = W^P e + b^P, P_i = sum_j phi Z_ij f^P_ij P0
        emb = p["emb"][z]
        Zcat = np.concatenate([emb[i], emb[j]], axis=1)
        Zij = Zcat @ p["emb2_w"].T + p["emb2_b"]
        f = np.einsum("pck,ek->epc", p["dproj_w"], e) + p["dproj_b"][None]
        coef = phi[:, None, None] * Zij[:, None, :] * f               # [E,3,F]
        Praw = [np.zeros((N, F, 3, 3)) for _ in range(3)]
        for a in range(0, E, EDGE_CHUNK):
            sl = slice(a, min(E, a + EDGE_CHUNK))
            for q in range(3):
                vals = coef[sl, q, :, None, None] * basis[q][sl, None, :, :]
                Praw[q] += segment_sum(i[sl], vals, N)
        Xraw = Praw[0] + Praw[1] + Praw[2]
        q0 = tensor_norm(Xraw)
        n0, ln0 = layer_norm(q0, p["emb_ln_g"], p["emb_ln_b"])
        as1 = n0 @ p["emb_mlp1_w"].T + p["emb_mlp1_b"]
        hs1 = silu(as1)
        as2 = hs1 @ p["emb_mlp2_w"].T + p["emb_mlp2_b"]
        s = silu(as2).reshape(N, F, 3)                                # [R3]
        U = [mix(p["emb_mix_w"][q], Praw[q]) for q in range(3)]       # [R4]
        X = sum(s[:, :, q, None, None] * U[q] for q in range(3))

        layers = []
        for l in range(self.L):
            X, cache_l = self.interaction(l, X, e, phi, i, j)
            layers.append(cache_l)

        # output model [R6, R7]
        I, A, S = decompose(X)
        h = np.concatenate([tensor_norm(I), tensor_norm(A), tensor_norm(S)], axis=1)
        hn, lno = layer_norm(h, p["out_ln_g"], p["out_ln_b"])
        ao = hn @ p["out_w"].T + p["out_b"]
        o = silu(ao)
        at = o @ p["head1_w"].T + p["head1_b"]
        t = silu(at)
        Ei = (t @ p["head2_w"].T)[:, 0] + p["head2_b"][0]
        Es = np.zeros(S_)
        np.add.at(Es, batch, Ei)
        cache = dict(z=z, batch=batch, i=i, j=j, r=r, d=d, u=u, phi=phi, e=e, basis=basis,
                     emb=emb, Zcat=Zcat, Zij=Zij, f=f, coef=coef, Praw=Praw, Xraw=Xraw,
                     ln0=ln0, n0=n0, as1=as1, hs1=hs1, as2=as2, s=s, U=U, layers=layers,
                     Xfinal=X, IAS=(I, A, S), h=h, lno=lno, hn=hn, ao=ao, o=o, at=at, t=t,
                     N=N, S=S_)
        return Es, Ei, cache

    # -------------------------------------------------------- backward ---
    def backward(self, c, seed=None, want_weights=True):
        """Analytic reverse pass of `forward` (hand-derived adjoints).

        seed [S] weights the per-system energies (default all ones):
        returns (dE/dpos [N,3], {name: dE/dparam}) for E = sum_s seed_s E_s.
        Forces are -dE/dpos."""
        p, F, N = self.p, self.F, c["N"]
        i, j, E = c["i"], c["j"], len(c["i"])
        seed = np.ones(c["S"]) if seed is None else np.asarray(seed, np.float64)
        G = {k: np.zeros_like(v) for k, v in p.items()}

        # output model
        gEi = seed[c["batch"]]
        G["head2_w"][0] = gEi @ c["t"]
        G["head2_b"][0] = gEi.sum()
        gat = gEi[:, None] * p["head2_w"][0][None, :] * silu_grad(c["at"])
        G["head1_w"] = gat.T @ c["o"]
        G["head1_b"] = gat.sum(0)
        gao = (gat @ p["head1_w"]) * silu_grad(c["ao"])
        G["out_w"] = gao.T @ c["hn"]
        G["out_b"] = gao.sum(0)
        gh, G["out_ln_g"], G["out_ln_b"] = layer_norm_adjoint(gao @ p["out_w"], p["out_ln_g"], c["lno"])
        I, A, S = c["IAS"]
        gX = decompose_adjoint(2.0 * gh[:, :F, None, None] * I,
                               2.0 * gh[:, F:2 * F, None, None] * A,
                               2.0 * gh[:, 2 * F:, None, None] * S)

        # per-edge accumulators: dE/dd and dE/du
        gd = np.zeros(E)
        gu = np.zeros((E, 3))
        gphi = np.zeros(E)
        ge = np.zeros((E, self.K))

        for l in reversed(range(self.L)):
            Ly = c["layers"][l]
            dX, Xn = Ly["dX"], Ly["Xn"]
            # X_out = Xn + dX + dX dX
            gdX = gX + np.matmul(gX, np.swapaxes(dX, -1, -2)) + np.matmul(np.swapaxes(dX, -1, -2), gX)
            gXn = gX.copy()
            # dX = sum_q mix(W2_q, Tn_q)
            gTn = []
            for q in range(3):
                gT_q, G[f"l{l}_mix2_w"][q] = mix_adjoint(p[f"l{l}_mix2_w"][q], gdX, Ly["Tn"][q])
                gTn.append(gT_q)
            TI, TA, TS = Ly["T"]
            den = (Ly["pn"] + 1.0)[..., None, None]
            gpn = -sum(np.sum(gTn[q] * Ly["T"][q], axis=(-2, -1)) for q in range(3)) / den[..., 0, 0] ** 2
            Tsum = TI + TA + TS
            gparts = [gTn[q] / den + 2.0 * Tsum * gpn[..., None, None] for q in range(3)]
            gT = decompose_adjoint(*gparts)
            # T = Y M + M Y
            Y, M = Ly["Y"], Ly["M"]
            gY = np.matmul(gT, np.swapaxes(M, -1, -2)) + np.matmul(np.swapaxes(M, -1, -2), gT)
            gM = np.matmul(np.swapaxes(Y, -1, -2), gT) + np.matmul(gT, np.swapaxes(Y, -1, -2))
            # messages M_i = sum_e sum_q g_q(e) Yp_q[j_e]
            gYp = [gY.copy(), gY.copy(), gY.copy()]
            Yp = Ly["Yp"]
            gW1 = G[f"l{l}_mlp1_w"]
            for a in range(0, E, EDGE_CHUNK):
                sl = slice(a, min(E, a + EDGE_CHUNK))
                g, (a1, h1, a2, h2, a3, h3) = self.edge_filter(l, c["e"][sl], c["phi"][sl])
                gMi = gM[i[sl]]
                gg = np.zeros_like(g)
                for q in range(3):
                    gg[:, :, q] = np.sum(gMi * Yp[q][j[sl]], axis=(-2, -1))
                    gYp[q] += segment_sum(j[sl], g[:, :, q, None, None] * gMi, N)
                gg = gg.reshape(-1, 3 * F)
                gphi[sl] += np.sum(gg * h3, axis=1)
                ga3 = gg * c["phi"][sl][:, None] * silu_grad(a3)
                G[f"l{l}_mlp3_w"] += ga3.T @ h2
                G[f"l{l}_mlp3_b"] += ga3.sum(0)
                ga2 = (ga3 @ p[f"l{l}_mlp3_w"]) * silu_grad(a2)
                G[f"l{l}_mlp2_w"] += ga2.T @ h1
                G[f"l{l}_mlp2_b"] += ga2.sum(0)
                ga1 = (ga2 @ p[f"l{l}_mlp2_w"]) * silu_grad(a1)
                gW1 += ga1.T @ c["e"][sl]
                G[f"l{l}_mlp1_b"] += ga1.sum(0)
                ge[sl] += ga1 @ p[f"l{l}_mlp1_w"]
            # Yp_q = mix(W1_q, part_q(Xn))
            gparts = []
            for q in range(3):
                gP, G[f"l{l}_mix1_w"][q] = mix_adjoint(p[f"l{l}_mix1_w"][q], gYp[q], Ly["parts"][q])
                gparts.append(gP)
            gXn += decompose_adjoint(*gparts)
            # Xn = X / (||X|| + 1)
            X = Ly["X"]
            dq = (Ly["qn"] + 1.0)[..., None, None]
            gX = gXn / dq - 2.0 * X * np.sum(gXn * X, axis=(-2, -1))[..., None, None] / dq ** 2

        # embedding: X0 = sum_q s_q mix(Wt_q, Praw_q)
        s, U, Praw = c["s"], c["U"], c["Praw"]
        gs = np.stack([np.sum(gX * U[q], axis=(-2, -1)) for q in range(3)], axis=-1)   # [N,F,3]
        gPraw = []
        for q in range(3):
            gPq, G["emb_mix_w"][q] = mix_adjoint(p["emb_mix_w"][q], s[:, :, q, None, None] * gX, Praw[q])
            gPraw.append(gPq)
        gas2 = gs.reshape(N, 3 * F) * silu_grad(c["as2"])
        G["emb_mlp2_w"] = gas2.T @ c["hs1"]
        G["emb_mlp2_b"] = gas2.sum(0)
        gas1 = (gas2 @ p["emb_mlp2_w"]) * silu_grad(c["as1"])
        G["emb_mlp1_w"] = gas1.T @ c["n0"]
        G["emb_mlp1_b"] = gas1.sum(0)
        gq0, G["emb_ln_g"], G["emb_ln_b"] = layer_norm_adjoint(gas1 @ p["emb_mlp1_w"], p["emb_ln_g"], c["ln0"])
        gXraw = 2.0 * c["Xraw"] * gq0[..., None, None]
        gPraw = [gPraw[q] + gXraw for q in range(3)]
        # Praw_q[i] = sum_e coef[e,q,:] basis_q[e]
        I0, A0, S0 = c["basis"]
        coef, f, Zij, phi = c["coef"], c["f"], c["Zij"], c["phi"]
        gcoef = np.zeros_like(coef)
        for a in range(0, E, EDGE_CHUNK):
            sl = slice(a, min(E, a + EDGE_CHUNK))
            for q in range(3):
                gPi = gPraw[q][i[sl]]                                           # [e,F,3,3]
                gcoef[sl, q, :] = np.einsum("efab,eab->ef", gPi, c["basis"][q][sl])
                gB = np.einsum("ef,efab->eab", coef[sl, q, :], gPi)
                if q == 1:    # <G, [u]_x> = u . (G21 - G12, G02 - G20, G10 - G01)
                    gu[sl] += np.stack([gB[:, 2, 1] - gB[:, 1, 2], gB[:, 0, 2] - gB[:, 2, 0],
                                        gB[:, 1, 0] - gB[:, 0, 1]], axis=1)
                elif q == 2:  # <G, u u^T - Id/3> -> (G + G^T) u
                    gu[sl] += np.einsum("eab,eb->ea", gB + np.swapaxes(gB, 1, 2), c["u"][sl])
        # coef = phi Z f
        gphi += np.einsum("eqc,ec,eqc->e", gcoef, Zij, f)
        gZ = np.einsum("eqc,e,eqc->ec", gcoef, phi, f)
        gf = gcoef * phi[:, None, None] * Zij[:, None, :]
        G["dproj_w"] = np.einsum("eqc,ek->qck", gf, c["e"])
        G["dproj_b"] = gf.sum(0)
        ge += np.einsum("eqc,qck->ek", gf, p["dproj_w"])
        G["emb2_w"] = gZ.T @ c["Zcat"]
        G["emb2_b"] = gZ.sum(0)
        gZcat = gZ @ p["emb2_w"]
        np.add.at(G["emb"], c["z"][i], gZcat[:, :F])
        np.add.at(G["emb"], c["z"][j], gZcat[:, F:])

        # geometry: e(d), phi(d), u = r/d, r = mic(r_i - r_j)
        d, u = c["d"], c["u"]
        _, dedd = expnorm(d, self.rc, self.rl, self.K)
        gd += np.sum(ge * dedd, axis=1) + gphi * cosine_cutoff_grad(d, self.rc)
        gr = gd[:, None] * u + (gu - np.sum(gu * u, axis=1)[:, None] * u) / d[:, None]
        gpos = segment_sum(i, gr, N) - segment_sum(j, gr, N)
        return gpos, (G if want_weights else None)

    # ------------------------------------------------------ convenience ---
    def energy_forces(self, z, pos, batch, box, pairs=None, n_systems=None, want_weights=False,
                      seed=None):
        Es, Ei, c = self.forward(z, pos, batch, box, pairs, n_systems)
        gpos, G = self.backward(c, seed=seed, want_weights=want_weights)
        return Es, Ei, -gpos, G
