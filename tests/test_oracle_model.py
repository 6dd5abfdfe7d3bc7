"""Pins of the oracle's TensorNet energy, forces and weight gradients:
central finite differences, an autograd witness, the invariances the model
fixes (Sec. 2.1.1: O(3) equivariance; translation, permutation and periodic
image invariance), zero net force, cutoff continuity and the isolated-atom
closed form."""
import math

import numpy as np
import pytest
import torch

from oracle.neighbors import neighbor_pairs
from oracle import tensornet as tn
from oracle.tensornet import TensorNet
from paper_2402_17660_gb300 import synth

from . import torch_witness

SMALL = synth.ModelShape(F=16, K=8, L=2)
FULL = synth.ModelShape()


def _model(shape=SMALL, seed=0):
    W = synth.init_weights(shape, seed)
    return W, TensorNet(W, F=shape.F, K=shape.K, L=shape.L)


def _pbc_small(seed=0, n=30, L=10.5):
    """A periodic box just over 2 cutoffs wide at low density."""
    rng = np.random.default_rng(seed)
    s = synth.random_cluster(n, seed=seed, side=L, min_dist=1.2)
    pos = s.pos.astype(np.float64) + rng.uniform(-L, L, (n, 3)).round() * 0  # inside the box
    box = (np.eye(3) * L)[None].astype(np.float32)
    return s.z, pos.astype(np.float32), s.batch, box


def _fd_forces(m, z, pos, batch, box, h=1e-5):
    pos = pos.astype(np.float64)
    fd = np.zeros_like(pos)
    for a in range(len(pos)):
        for k in range(3):
            pp = pos.copy()
            pp[a, k] += h
            pm = pos.copy()
            pm[a, k] -= h
            fd[a, k] = -(m.forward(z, pp, batch, box)[0].sum() - m.forward(z, pm, batch, box)[0].sum()) / (2 * h)
    return fd


def _rms(F):
    return np.sqrt(np.mean(np.sum(F * F, axis=1)))


@pytest.mark.parametrize("case", ["cluster", "pbc"])
def test_forces_match_finite_differences(case):
    W, m = _model()
    if case == "cluster":
        s = synth.random_cluster(10, seed=5, side=4.0)
        z, pos, batch, box = s.z, s.pos, s.batch, None
    else:
        z, pos, batch, box = _pbc_small(1, n=12)
    _, _, F, _ = m.energy_forces(z, pos, batch, box)
    fd = _fd_forces(m, z, pos, batch, box)
    assert np.max(np.abs(F - fd)) <= 1e-7 * max(_rms(F), 1.0)


def test_forces_match_finite_differences_full_width():
    W, m = _model(FULL)
    s = synth.random_cluster(6, seed=9, side=3.0)
    _, _, F, _ = m.energy_forces(s.z, s.pos, s.batch, None)
    fd = _fd_forces(m, s.z, s.pos, s.batch, None)
    assert np.max(np.abs(F - fd)) <= 1e-7 * max(_rms(F), 1.0)


def test_weight_gradients_match_directional_fd():
    W, m = _model()
    s = synth.random_cluster(10, seed=6, side=4.0)
    pos = s.pos.astype(np.float64)
    _, _, _, G = m.energy_forces(s.z, pos, s.batch, None, want_weights=True)
    rng = np.random.default_rng(0)
    h = 1e-5
    for name in W:
        v = rng.standard_normal(W[name].shape)
        Wp = {k: np.asarray(x, np.float64).copy() for k, x in W.items()}
        Wm = {k: x.copy() for k, x in Wp.items()}
        Wp[name] = Wp[name] + h * v
        Wm[name] = Wm[name] - h * v
        ep = TensorNet(Wp, F=16, K=8, L=2).forward(s.z, pos, s.batch, None)[0][0]
        em = TensorNet(Wm, F=16, K=8, L=2).forward(s.z, pos, s.batch, None)[0][0]
        fd = (ep - em) / (2 * h)
        an = float(np.sum(G[name] * v))
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-2), name


@pytest.mark.parametrize("case", ["cluster", "pbc", "batch"])
def test_reverse_pass_matches_autograd_witness(case):
    W, m = _model()
    if case == "cluster":
        s = synth.random_cluster(14, seed=7, side=4.5)
        z, pos, batch, box = s.z, s.pos, s.batch, None
    elif case == "pbc":
        z, pos, batch, box = _pbc_small(2, n=20)
    else:
        s = synth.molecule_batch(3, nmin=5, nmax=9, seed=4)
        z, pos, batch, box = s.z, s.pos, s.batch, None
    i, j = neighbor_pairs(pos, batch, box, 5.0)
    seed = np.linspace(0.5, 1.5, int(batch.max()) + 1)
    Es, _, c = m.forward(z, pos, batch, box, pairs=(i, j))
    gpos, G = m.backward(c, seed=seed)
    P = {k: torch.tensor(np.asarray(v, np.float64), requires_grad=True) for k, v in W.items()}
    X = torch.tensor(pos.astype(np.float64), requires_grad=True)
    bt = None if box is None else torch.tensor(box.astype(np.float64))
    Et = torch_witness.energy(P, torch.tensor(z).long(), X, torch.tensor(batch).long(), bt,
                              torch.tensor(i), torch.tensor(j), F=16, K=8, L=2)
    assert np.allclose(Et.detach().numpy(), Es, rtol=1e-12, atol=1e-12)
    (Et * torch.tensor(seed)).sum().backward()
    assert np.allclose(gpos, X.grad.numpy(), rtol=1e-9, atol=1e-11)
    for k in W:
        assert np.allclose(G[k], P[k].grad.numpy(), rtol=1e-9, atol=1e-11), k


def _random_orthogonal(seed, reflect):
    rng = np.random.default_rng(seed)
    Q, R = np.linalg.qr(rng.standard_normal((3, 3)))
    Q = Q * np.sign(np.diag(R))
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    if reflect:
        Q = Q @ np.diag([1.0, 1.0, -1.0])
    return Q


@pytest.mark.parametrize("reflect", [False, True])
def test_rotation_reflection_invariance_and_force_equivariance(reflect):
    W, m = _model(FULL)
    s = synth.random_cluster(20, seed=8)
    pos = s.pos.astype(np.float64)
    E0, _, F0, _ = m.energy_forces(s.z, pos, s.batch, None)
    Q = _random_orthogonal(3, reflect)
    E1, _, F1, _ = m.energy_forces(s.z, pos @ Q.T, s.batch, None)
    assert abs(E1[0] - E0[0]) <= 1e-12 * max(1.0, abs(E0[0]))
    assert np.allclose(F1, F0 @ Q.T, atol=1e-11)


def test_translation_permutation_and_zero_net_force():
    W, m = _model()
    s = synth.random_cluster(24, seed=10)
    pos = s.pos.astype(np.float64)
    E0, Ei0, F0, _ = m.energy_forces(s.z, pos, s.batch, None)
    assert np.allclose(F0.sum(0), 0.0, atol=1e-12)
    E1, _, F1, _ = m.energy_forces(s.z, pos + np.array([3.1, -7.2, 0.4]), s.batch, None)
    assert abs(E1[0] - E0[0]) < 1e-12 * max(1.0, abs(E0[0]))
    perm = np.random.default_rng(1).permutation(len(pos))
    E2, Ei2, F2, _ = m.energy_forces(s.z[perm], pos[perm], s.batch, None)
    assert abs(E2[0] - E0[0]) < 1e-12 * max(1.0, abs(E0[0]))
    assert np.allclose(F2, F0[perm], atol=1e-12)
    assert np.allclose(Ei2, Ei0[perm], atol=1e-12)


def test_periodic_image_shift_invariance():
    W, m = _model()
    z, pos, batch, box = _pbc_small(3, n=24)
    pos = pos.astype(np.float64)
    E0, _, F0, _ = m.energy_forces(z, pos, batch, box)
    assert np.allclose(F0.sum(0), 0.0, atol=1e-12)
    shifted = pos.copy()
    shifted[::3] += np.array([10.5, -21.0, 31.5])        # lattice vectors of the box
    E1, _, F1, _ = m.energy_forces(z, shifted, batch, box)
    assert abs(E1[0] - E0[0]) < 1e-12 * max(1.0, abs(E0[0]))
    assert np.allclose(F1, F0, atol=1e-12)


def test_triclinic_cell_equivalent_to_cube_gives_same_energy_forces():
    """Same lattice, other basis (a = (L,0,0), b = (L,L,0), c = (0,L,L)):
    the model sees the same pairs and vectors, so energy and forces agree
    to rounding; a shift of atoms by lattice vectors of the tilted basis
    changes nothing either."""
    W, m = _model()
    s = synth.water_box(6, 18.6, seed=3)
    L = 18.6
    skew = np.array([[[L, 0, 0], [L, L, 0], [0, L, L]]], np.float32)
    pos = s.pos.astype(np.float64)
    E0, _, F0, _ = m.energy_forces(s.z, pos, s.batch, s.box)
    E1, _, F1, _ = m.energy_forces(s.z, pos, s.batch, skew)
    assert abs(E1[0] - E0[0]) < 1e-11 * max(1.0, abs(E0[0]))
    assert np.allclose(F1, F0, atol=1e-10 * _rms(F0))
    shifted = pos.copy()
    shifted[1::3] += skew[0, 0] - 2 * skew[0, 1] + skew[0, 2]
    E2, _, F2, _ = m.energy_forces(s.z, shifted, s.batch, skew)
    assert abs(E2[0] - E0[0]) < 1e-11 * max(1.0, abs(E0[0]))
    assert np.allclose(F2, F0, atol=1e-10 * _rms(F0))


def test_triclinic_forces_match_finite_differences():
    W, m = _model()
    s = synth.triclinic_water(4, 12.416, seed=3)
    pos = s.pos.astype(np.float64)[:24]
    z, batch = s.z[:24], s.batch[:24]
    _, _, F, _ = m.energy_forces(z, pos, batch, s.box)
    fd = _fd_forces(m, z, pos, batch, s.box)
    assert np.abs(F - fd).max() <= 1e-7 * _rms(F) + 1e-9


def test_batch_equals_separate_systems():
    W, m = _model()
    s = synth.molecule_batch(4, nmin=6, nmax=12, seed=5)
    Es, Ei, F, _ = m.energy_forces(s.z, s.pos, s.batch, None)
    for k in range(4):
        sel = s.batch == k
        Ek, _, Fk, _ = m.energy_forces(s.z[sel], s.pos[sel], np.zeros(sel.sum(), np.int32), None)
        assert abs(Ek[0] - Es[k]) < 1e-12 * max(1.0, abs(Es[k]))
        assert np.allclose(Fk, F[sel], atol=1e-12)


def test_isolated_atoms_reduce_to_output_mlp():
    """Atoms farther apart than the cutoff have zero tensor features, so each
    atom's energy is the output head applied to the LayerNorm shift alone:
    an ordinary MLP (evaluated here with torch.nn layers)."""
    W, m = _model()
    pos = np.array([[0.0, 0, 0], [6.0, 0, 0], [0, 12.0, 0]])
    z = np.array([1, 6, 8], np.int32)
    Es, Ei, F, _ = m.energy_forces(z, pos, np.zeros(3, np.int32), None)
    assert np.all(F == 0)
    F_ = SMALL.F
    net = torch.nn.Sequential(torch.nn.Linear(3 * F_, F_), torch.nn.SiLU(),
                              torch.nn.Linear(F_, F_ // 2), torch.nn.SiLU(),
                              torch.nn.Linear(F_ // 2, 1)).double()
    with torch.no_grad():
        for lin, wn, bn in ((net[0], "out_w", "out_b"), (net[2], "head1_w", "head1_b"),
                            (net[4], "head2_w", "head2_b")):
            lin.weight.copy_(torch.tensor(W[wn].astype(np.float64)))
            lin.bias.copy_(torch.tensor(W[bn].astype(np.float64)))
        ref = net(torch.tensor(W["out_ln_b"].astype(np.float64))).item()
    assert np.allclose(Ei, ref, atol=1e-13)


def test_cutoff_continuity():
    """A pair at d = rc - eps differs from the isolated pair by O(eps^4):
    phi(rc - eps) = O(eps^2) multiplies every tensor feature of the pair, and
    the energy sees features only through squared norms."""
    W, m = _model()
    z = np.array([6, 8], np.int32)
    b = np.zeros(2, np.int32)
    far = m.forward(z, np.array([[0.0, 0, 0], [20.0, 0, 0]]), b, None)[0][0]
    dE = []
    for eps in (4e-2, 2e-2, 1e-2):
        dE.append(m.forward(z, np.array([[0.0, 0, 0], [5.0 - eps, 0, 0]]), b, None)[0][0] - far)
    assert abs(dE[0]) > 0
    assert abs(dE[1] / dE[0] - 1 / 16) < 0.005 and abs(dE[2] / dE[1] - 1 / 16) < 0.005


def test_edge_filter_vanishes_with_its_slope_at_the_cutoff():
    """C8: g(d) = 0 for d >= rc, and g(rc - eps) = O(eps^2) (so dg/dd -> 0):
    the cutoff factor phi carries the whole d-dependence there, since the
    expnorm basis (with its own phi factor) stays finite."""
    W, m = _model()
    K = SMALL.K
    for d in (5.0, 5.3, 7.0):
        e, _ = tn.expnorm(np.array([d]), 5.0, 0.0, K)
        g, _ = m.edge_filter(0, e, tn.cosine_cutoff(np.array([d]), 5.0))
        assert np.all(g == 0.0)
    gs = []
    for eps in (4e-2, 2e-2, 1e-2):
        d = np.array([5.0 - eps])
        e, _ = tn.expnorm(d, 5.0, 0.0, K)
        g, _ = m.edge_filter(1, e, tn.cosine_cutoff(d, 5.0))
        gs.append(np.abs(g).max())
    # phi ~ (pi eps / 2 rc)^2 and the basis itself carries another phi, so the
    # filter's leading behaviour is eps^2 times a bounded factor: halving eps
    # divides it by 4 to within the factor's own variation
    assert gs[0] > 0
    assert abs(gs[1] / gs[0] - 0.25) < 0.02 and abs(gs[2] / gs[1] - 0.25) < 0.02


def test_zero_layer_model_runs_and_is_invariant():
    shape = synth.ModelShape(F=16, K=8, L=0)
    W = synth.init_weights(shape, 1)
    m = TensorNet(W, F=16, K=8, L=0)
    s = synth.random_cluster(12, seed=12)
    pos = s.pos.astype(np.float64)
    E0, _, F0, _ = m.energy_forces(s.z, pos, s.batch, None)
    Q = _random_orthogonal(5, True)
    E1, _, F1, _ = m.energy_forces(s.z, pos @ Q.T, s.batch, None)
    assert abs(E1[0] - E0[0]) < 1e-12 * max(1, abs(E0[0]))
    assert np.allclose(F1, F0 @ Q.T, atol=1e-12)
    fd = _fd_forces(m, s.z, pos, s.batch, None)
    assert np.max(np.abs(F0 - fd)) <= 1e-7 * max(_rms(F0), 1.0)


# ------------------------------------------- interaction node update (C9) ---
# One-channel toy layers whose outputs are worked out by hand.  The mixing
# weights are scalars per part: W_{l,1} = (2, 3, 5) and W_{l,2} = (2, 3, 5)
# for (I, A, S), so a dropped or merged decomposition changes the result.

def _toy(F=1, K=2, mlp3_b=(0.0, 0.0, 0.0)):
    w = np.array([2.0, 3.0, 5.0]).reshape(3, 1, 1)
    p = {"l0_mix1_w": w, "l0_mix2_w": w,
         "l0_mlp1_w": np.zeros((F, K)), "l0_mlp1_b": np.zeros(F),
         "l0_mlp2_w": np.zeros((2 * F, F)), "l0_mlp2_b": np.zeros(2 * F),
         "l0_mlp3_w": np.zeros((3 * F, 2 * F)), "l0_mlp3_b": np.asarray(mlp3_b, np.float64)}
    return TensorNet(p, F=F, K=K, L=1)


def _one(A):
    return np.asarray(A, np.float64)[None, None]        # [N=1, F=1, 3, 3]


def test_node_update_commuting_factors():
    """Y = diag(1, 2, 3) and M = diag(4, 5, 6) commute, so T = YM + MY =
    2 YM = diag(8, 20, 36), symmetric; ||T|| = 64 + 400 + 1296 = 1760.  The
    parts of T are I = (64/3) Id and S = T - I, with no A part, so
    dX = (2 I + 5 S) / 1761 = (5 T - 3 (64/3) Id) / 1761 = diag(-24, 36, 116) / 1761,
    and X_out = Xn + dX + dX^2 (dX diagonal)."""
    m = _toy()
    Xn = _one(np.eye(3) * 0.5)
    Xout, c = m.node_update(0, Xn, _one(np.diag([1.0, 2, 3])), _one(np.diag([4.0, 5, 6])))
    TI, TA, TS = c["T"]
    T = (TI + TA + TS)[0, 0]
    assert np.allclose(T, np.diag([8.0, 20, 36]), atol=1e-13)
    assert np.allclose(T, T.T, atol=0)
    assert np.allclose(TA, 0.0, atol=0)
    assert np.isclose(c["pn"][0, 0], 1760.0, rtol=1e-15)
    D = np.diag([-24.0, 36.0, 116.0]) / 1761.0
    assert np.allclose(c["dX"][0, 0], D, atol=1e-15)
    assert np.allclose(Xout[0, 0], 0.5 * np.eye(3) + D + D @ D, atol=1e-15)


def test_node_update_identity_factor():
    """Y = Id gives T = 2M for any M.  With M = [[1,2,3],[4,5,6],[7,8,10]]:
    tr T = 32, ||T|| = 4 * 304 = 1216, A(T) = M - M^T, S(T) = M + M^T - (32/3) Id,
    so dX = (2 (32/3) Id + 3 (M - M^T) + 5 (M + M^T) - (160/3) Id) / 1217
          = [[-22, 24, 38], [36, 18, 64], [62, 76, 68]] / 1217."""
    m = _toy()
    Mm = np.array([[1.0, 2, 3], [4, 5, 6], [7, 8, 10]])
    Xn = _one(np.zeros((3, 3)))
    Xout, c = m.node_update(0, Xn, _one(np.eye(3)), _one(Mm))
    assert np.allclose(sum(c["T"])[0, 0], 2 * Mm, atol=1e-13)
    assert np.isclose(c["pn"][0, 0], 1216.0, rtol=1e-15)
    D = np.array([[-22.0, 24, 38], [36, 18, 64], [62, 76, 68]]) / 1217.0
    assert np.allclose(c["dX"][0, 0], D, atol=1e-15)
    assert np.allclose(Xout[0, 0], D + D @ D, atol=1e-15)


def test_interaction_normalise_decompose_mix():
    """X = [[1,2,0],[0,1,0],[0,0,1]]: ||X|| = 7, so Xn = X / 8; its parts are
    I = Id/8, A = [[0,1,0],[-1,0,0],0]/8, S = [[0,1,0],[1,0,0],0]/8, and with
    W_{l,1} = (2, 3, 5) Y = (2 Id + 3 A + 5 S) * 8 / 8 = [[2,8,0],[2,2,0],[0,0,2]] / 8.
    An isolated atom has M = 0, so T = 0, dX = 0 and X_out = Xn."""
    m = _toy()
    X = _one([[1.0, 2, 0], [0, 1, 0], [0, 0, 1]])
    e = np.zeros((0, 2))
    Xout, c = m.interaction(0, X, e, np.zeros(0), np.zeros(0, np.int64), np.zeros(0, np.int64))
    assert np.isclose(c["qn"][0, 0], 7.0, rtol=1e-15)
    assert np.allclose(c["Xn"], X / 8.0, atol=1e-16)
    assert np.allclose(c["Y"][0, 0], np.array([[2.0, 8, 0], [2, 2, 0], [0, 0, 2]]) / 8.0, atol=1e-15)
    assert np.allclose(c["M"], 0.0, atol=0) and np.allclose(c["dX"], 0.0, atol=0)
    assert np.allclose(Xout, X / 8.0, atol=1e-16)


def test_interaction_layer_two_atoms_closed_form():
    """Two atoms d = rc/3 apart (phi = 3/4) with isotropic features X_0 = 2 Id,
    X_1 = Id.  Radial MLP weights zero and last bias b = ln 3 on the I plane
    give g^I = phi SiLU(ln 3) = (3/4)(3/4) ln 3 = (9/16) ln 3 on every edge.
    Then Xn_0 = 2/13 Id (||X_0|| = 12), Xn_1 = 1/4 Id (||X_1|| = 3);
    Y = 2 Xn (the I weight): Y_0 = 4/13 Id, Y_1 = 1/2 Id; M_0 = g Y_1 =
    (9/32) ln 3 Id, M_1 = g Y_0 = (9/52) ln 3 Id (each atom receives its
    neighbour's Y); T_k = 2 Y_k M_k = t Id with t = (9/52) ln 3 for both
    atoms; dX_k = 2 t / (3 t^2 + 1) Id (I weight 2, ||T|| = 3 t^2);
    X_out = Xn + dX + dX^2."""
    rc = 5.0
    m = _toy(mlp3_b=(math.log(3.0), 0.0, 0.0))
    m.rc = rc
    pos = np.array([[0.0, 0, 0], [rc / 3, 0, 0]])
    i = np.array([0, 1])
    j = np.array([1, 0])
    d = np.linalg.norm(pos[i] - pos[j], axis=1)
    phi = tn.cosine_cutoff(d, rc)
    assert np.allclose(phi, 0.75, atol=1e-15)
    e, _ = tn.expnorm(d, rc, 0.0, 2)
    X = np.stack([_one(2 * np.eye(3))[0], _one(np.eye(3))[0]])
    Xout, c = m.interaction(0, X, e, phi, i, j)
    ln3 = math.log(3.0)
    assert np.allclose(c["M"][0, 0], 9 / 32 * ln3 * np.eye(3), atol=1e-15)
    assert np.allclose(c["M"][1, 0], 9 / 52 * ln3 * np.eye(3), atol=1e-15)
    for k, (xn, t) in enumerate(((2 / 13, 9 / 52 * ln3), (1 / 4, 9 / 52 * ln3))):
        dx = 2 * t / (3 * t * t + 1)
        assert np.allclose(c["dX"][k, 0], dx * np.eye(3), atol=1e-15)
        assert np.allclose(Xout[k, 0], (xn + dx + dx * dx) * np.eye(3), atol=1e-15)


def _two_atom_embedding(d=2.0):
    """Two atoms (H receiver 0 at the origin, C at (0, 0, d)), F = 2, K = 4,
    no interaction layer.  Radial projections are constants (dproj_w = 0),
    the pair embedding is asymmetric in its two halves, and the embedding
    mixing of every class swaps the two channels."""
    shape = synth.ModelShape(F=2, K=4, L=0, max_z=10)
    W = synth.init_weights(shape, seed=5)
    W["emb"][:] = 0.0
    W["emb"][1] = (1.0, 0.0)
    W["emb"][6] = (0.0, 1.0)
    W["emb2_w"] = np.array([[1.0, 2.0, 3.0, 4.0], [0.0, 1.0, 0.0, -1.0]], np.float32)
    W["emb2_b"] = np.array([0.5, -0.5], np.float32)
    W["dproj_w"][:] = 0.0
    W["dproj_b"] = np.array([[1.0, 2.0], [3.0, -1.0], [0.5, 4.0]], np.float32)   # [p][c]: I, A, S
    W["emb_mix_w"] = np.array([[[0.0, 1.0], [1.0, 0.0]]] * 3, np.float32)
    m = TensorNet(W, F=2, K=4, L=0)
    z = np.array([1, 6], np.int32)
    pos = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, d]])
    _, _, c = m.forward(z, pos, np.zeros(2, np.int32), None)
    return W, c


def test_embedding_edge_sum_closed_form():
    """The embedding's edge-to-node sum (Sec. 2.1.1) on two atoms along z.
    Receiver 0 sees r_01 = r_0 - r_1 = -d z (u = -z), receiver 1 sees u = +z.
    The pair embeddings, receiver first: Z_01 = W_e (1, 0, 0, 1) + b_e =
    (5.5, -1.5) and Z_10 = W_e (0, 1, 1, 0) + b_e = (5.5, 0.5).  With constant
    projections f^p = b^p and phi = (cos(2 pi / 5) + 1) / 2 at d = 2 A, channel c
    of receiver i is phi Z_i[c] (b^I[c] Id + b^A[c] [u]_x + b^S[c] (u u^T - Id/3)),
    with [-z]_x = [[0, 1, 0], [-1, 0, 0], [0, 0, 0]] (so that [u]_x v = u x v)
    and u u^T - Id/3 = diag(-1/3, -1/3, 2/3) for u = +-z.  Its squared norm is
    (phi Z)^2 (3 (b^I)^2 + 2 (b^A)^2 + (2/3) (b^S)^2), the three parts being
    orthogonal.  Caught: an edge vector r_j - r_i or a transposed skew part
    (the A block flips sign), the sender-first pair embedding (channel 1
    swaps -1.5 and 0.5), an S part without the -Id/3, a dropped cutoff factor,
    an unsquared norm."""
    W, c = _two_atom_embedding()
    phi = 0.5 * (math.cos(math.pi * 2.0 / 5.0) + 1.0)
    Z = {0: np.array([5.5, -1.5]), 1: np.array([5.5, 0.5])}
    skew = {0: np.array([[0, 1, 0], [-1, 0, 0], [0, 0, 0]], float), 1: np.array([[0, -1, 0], [1, 0, 0], [0, 0, 0]], float)}
    S0 = np.diag([-1.0 / 3, -1.0 / 3, 2.0 / 3])
    bI, bA, bS = (W["dproj_b"][p].astype(np.float64) for p in range(3))
    for i in (0, 1):
        for ch in (0, 1):
            want = phi * Z[i][ch] * (bI[ch] * np.eye(3) + bA[ch] * skew[i] + bS[ch] * S0)
            assert np.allclose(c["Xraw"][i, ch], want, rtol=1e-12, atol=1e-12), (i, ch)
            q0 = (phi * Z[i][ch]) ** 2 * (3 * bI[ch] ** 2 + 2 * bA[ch] ** 2 + (2.0 / 3.0) * bS[ch] ** 2)
            assert math.isclose(tn.tensor_norm(c["Xraw"])[i, ch], q0, rel_tol=1e-12)


def test_embedding_mixes_before_scaling():
    """Reading R4 on the same two atoms: each class's channel mixing (here a
    swap of the two channels) acts on the summed edge features before the
    per-channel scale s of the receiver, so X[c] = sum_p s[c, p] P_p[1 - c].
    Scaling first would give sum_p s[1 - c, p] P_p[1 - c]; the two channels'
    scales differ, so the test tells them apart."""
    _, c = _two_atom_embedding()
    s = c["s"]                      # [N, F, 3]
    P = c["Praw"]                   # three [N, F, 3, 3]
    assert np.abs(s[:, 0, :] - s[:, 1, :]).max() > 1e-3
    I, A, S = c["IAS"]              # no interaction layer: the embedding X, decomposed
    X = I + A + S
    for i in (0, 1):
        for ch in (0, 1):
            want = sum(s[i, ch, p] * P[p][i, 1 - ch] for p in range(3))
            assert np.allclose(X[i, ch], want, rtol=1e-12, atol=1e-12), (i, ch)
            wrong = sum(s[i, 1 - ch, p] * P[p][i, 1 - ch] for p in range(3))
            assert not np.allclose(X[i, ch], wrong, rtol=1e-6, atol=1e-9)


def test_output_concatenates_class_norms_in_blocks():
    """Reading R6 on the same two atoms: the output model's input is
    (||I||, ||A||, ||S||) of the final features in blocks of F channels.  With
    the channel-swap mixing, the class-p part of X[c] is s[c, p] P_p[1 - c], so
    its squared norm is s[c, p]^2 (phi Z[1 - c] b^p[1 - c])^2 n_p with
    n_I = 3, n_A = 2, n_S = 2/3 (the norms of Id, [u]_x and u u^T - Id/3).
    Caught: another block order, channel-major interleaving, unsquared norms."""
    W, c = _two_atom_embedding()
    phi = 0.5 * (math.cos(math.pi * 2.0 / 5.0) + 1.0)
    Z = {0: np.array([5.5, -1.5]), 1: np.array([5.5, 0.5])}
    b = [W["dproj_b"][p].astype(np.float64) for p in range(3)]
    n = (3.0, 2.0, 2.0 / 3.0)
    s = c["s"]
    for i in (0, 1):
        want = np.array([s[i, ch, p] ** 2 * (phi * Z[i][1 - ch] * b[p][1 - ch]) ** 2 * n[p]
                         for p in range(3) for ch in range(2)])
        assert np.allclose(c["h"][i], want, rtol=1e-10, atol=1e-14), (i, c["h"][i], want)


def test_interaction_messages_sum_over_every_neighbour():
    """Three atoms on a line, 0 at the origin, 1 at rc/3 and 2 at -rc/2, with
    isotropic features X_k = c_k Id (c = 1, 2, 3).  Every pair is within the
    cutoff, with phi(rc/3) = 3/4, phi(rc/2) = 1/2 and phi(5 rc/6) =
    (1 - sqrt(3)/2)/2.  With the radial MLP giving g^I = phi SiLU(ln 3) =
    (3/4) ln 3 phi, Xn_k = c_k/(3 c_k^2 + 1) Id and Y_k = 2 Xn_k, atom 0
    receives M_0 = (3/4) ln 3 (phi_01 Y_1 + phi_02 Y_2), the sum over both of
    its neighbours with their own filters; T_0 = 2 Y_0 M_0 = t Id and
    dX_0 = 2 t / (3 t^2 + 1) Id.  Caught: a mean over neighbours, a single
    neighbour, one filter for all edges."""
    rc = 5.0
    m = _toy(mlp3_b=(math.log(3.0), 0.0, 0.0))
    m.rc = rc
    pos = np.array([[0.0, 0, 0], [rc / 3, 0, 0], [-rc / 2, 0, 0]])
    i = np.array([0, 0, 1, 1, 2, 2])
    j = np.array([1, 2, 0, 2, 0, 1])
    d = np.linalg.norm(pos[i] - pos[j], axis=1)
    phi = tn.cosine_cutoff(d, rc)
    e, _ = tn.expnorm(d, rc, 0.0, 2)
    c_ = np.array([1.0, 2.0, 3.0])
    X = np.stack([_one(ck * np.eye(3))[0] for ck in c_])
    Xout, cache = m.interaction(0, X, e, phi, i, j)
    ln3 = math.log(3.0)
    phis = {(0, 1): 0.75, (0, 2): 0.5, (1, 2): 0.5 * (1.0 - math.sqrt(3.0) / 2.0)}
    y = 2.0 * c_ / (3.0 * c_ ** 2 + 1.0)
    for k in range(3):
        mk = 0.75 * ln3 * sum(phis[tuple(sorted((k, n)))] * y[n] for n in range(3) if n != k)
        assert np.allclose(cache["M"][k, 0], mk * np.eye(3), rtol=1e-13, atol=1e-15), k
        t = 2.0 * y[k] * mk
        dx = 2.0 * t / (3.0 * t * t + 1.0)
        xn = c_[k] / (3.0 * c_[k] ** 2 + 1.0)
        assert np.allclose(Xout[k, 0], (xn + dx + dx * dx) * np.eye(3), rtol=1e-13, atol=1e-15), k


def test_per_edge_and_per_atom_splits_are_channel_major():
    """Reading R3 in the oracle's layout: a 3F vector splits as index c*3 + p
    (p = I, A, S).  With zero weights before the last bias, the radial filter
    of an edge is g[c][p] = phi SiLU(b3[c*3 + p]) and the embedding's scales
    are s[c][p] = SiLU(b2[c*3 + p]), for distinct biases; a plane-major split
    (index p*F + c) fails both."""
    F = 2
    b = np.array([0.1, 0.2, 0.3, 0.4, 0.5, 0.6])
    m = _toy(F=F, mlp3_b=b)
    phi = np.array([0.75])
    g, _ = m.edge_filter(0, np.zeros((1, 2)), phi)
    for c in range(F):
        for p in range(3):
            assert math.isclose(g[0, c, p], 0.75 * tn.silu(b[c * 3 + p]), rel_tol=1e-15)
    shape = synth.ModelShape(F=F, K=4, L=0, max_z=10)
    W = synth.init_weights(shape, seed=3)
    W["emb_mlp2_w"][:] = 0.0
    W["emb_mlp2_b"] = b.astype(np.float32)
    _, _, c_ = TensorNet(W, F=F, K=4, L=0).forward(np.array([1, 6], np.int32),
                                                     np.array([[0.0, 0, 0], [0, 0, 2.0]]), np.zeros(2, np.int32), None)
    b32 = W["emb_mlp2_b"].astype(np.float64)
    for c in range(F):
        for p in range(3):
            assert np.allclose(c_["s"][:, c, p], tn.silu(b32[c * 3 + p]), rtol=1e-15, atol=0)
