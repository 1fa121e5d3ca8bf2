"""Learned preconditioner on the GPU against the FP64 oracle: the
shifted-Poisson CG targets, the conv net's forward pass, loss and weight
gradients (through the C ABI), the grid-level inference, and training.

Tolerances: FP64 CG after 200 iterations agrees with the oracle's to 1e-8
relative (the iteration is not converged to rounding, so rounding-order
differences stay small).  The network runs in FP32 with BF16 weights and
inputs; the oracle is given the same BF16-rounded values and computes in
FP64, so outputs agree to FP32 accumulation accuracy (1e-5 relative) and
gradients, which sum ~1e4 products, to 1e-4.
"""
import numpy as np
import pytest

import workloads as wl
from tests.helpers import SMALL_ATOMS, SMALL_E, SMALL_H, SMALL_RADIUS, lib_to_oracle_index, oracle_system

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _grid(spec=None):
    from paper_1306_2953_gb300 import api
    if spec is None:
        g_ora, _, atoms, _ = oracle_system("atoms", SMALL_ATOMS, SMALL_E, SMALL_RADIUS, SMALL_H)
        lg = api.Grid.spheres(np.array(SMALL_ATOMS), SMALL_RADIUS, SMALL_H)
    else:
        g_ora, _, atoms, _ = oracle_system("mol", spec)
        lg = api.Grid.spheres(atoms, spec.radius, spec.h)
    return lg, g_ora, lib_to_oracle_index(g_ora, lg.ijk())


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_shifted_poisson_cg_parity(dtype):
    from oracle import precond as op
    from paper_1306_2953_gb300 import api
    lg, g_ora, idx = _grid(wl.MOL20.system)
    Hs = api.Hamiltonian(lg, np.full(lg.npts, 1.0))
    r = wl.random_block(g_ora.npts, 8, 21)
    t = torch.float64 if dtype == "f64" else torch.float32
    if dtype == "f32":
        r = r.astype(np.float32).astype(np.float64)
    X = api.shifted_poisson_cg(Hs, torch.from_numpy(np.ascontiguousarray(r[idx])).to(t).cuda(), 200)
    ref = op.shifted_poisson_cg(g_ora, r, 1.0, 200)[idx]
    err = np.linalg.norm(X.double().cpu().numpy() - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert err.max() <= (1e-8 if dtype == "f64" else 1e-4)


def _tiles(ntiles=3, D=9, seed=0):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((ntiles, D, D, D)).astype(np.float32)
    mask = (rng.uniform(size=(ntiles, D, D, D)) > 0.25)
    x *= mask
    tgt = rng.standard_normal((ntiles, D, D, D)).astype(np.float32)
    valid = np.zeros((D, D, D), dtype=bool)
    valid[2:-2, 2:-2, 2:-2] = True
    return x, mask, tgt, valid


def test_convnet_forward_and_gradients_match_oracle():
    from oracle import precond as op
    from paper_1306_2953_gb300 import api
    ws = wl.conv_init(5)
    w = np.concatenate([a.reshape(a.shape[0], a.shape[1], 27).ravel() for a in ws]).astype(np.float32)
    x, mask, tgt, valid = _tiles()
    dev = lambda a, t=torch.float32: torch.from_numpy(np.ascontiguousarray(a)).to(t).cuda()
    y, g, loss = api.convnet_tiles(dev(w), dev(x), dev(mask.astype(np.uint8), torch.uint8), dev(tgt),
                                   dev(valid.astype(np.uint8), torch.uint8))
    # oracle on the same BF16-rounded weights and inputs, FP64
    wq = [op.bf16_round(a).astype(np.float64) for a in ws]
    xq = op.bf16_round(x).astype(np.float64)
    yr, cache = op.net_forward(xq, mask, wq)
    lr, gy = op.tile_loss(yr, tgt.astype(np.float64), valid[None] & mask)
    gr = op.net_backward(gy, cache, wq)
    grf = np.concatenate([a.reshape(a.shape[0], a.shape[1], 27).ravel() for a in gr])
    yg = y.cpu().numpy()
    assert np.abs(yg - yr).max() <= 1e-5 * np.abs(yr).max()
    assert abs(loss - lr) <= 1e-5 * lr
    gg = g.cpu().numpy()
    assert np.abs(gg - grf).max() <= 1e-4 * np.abs(grf).max()


def _flat_weights(ws):
    return np.concatenate([a.reshape(a.shape[0], a.shape[1], 27).ravel() for a in ws]).astype(np.float32)


def test_learned_apply_on_grid_matches_oracle():
    from oracle import precond as op
    from paper_1306_2953_gb300 import api
    lg, g_ora, idx = _grid()
    Hs = api.Hamiltonian(lg, np.zeros(lg.npts))
    ws = wl.conv_init(9)
    R = wl.gaussian_sum_block(g_ora.coords, 8, 3).astype(np.float32)
    W = api.precond_apply(Hs, torch.from_numpy(_flat_weights(ws)).cuda(),
                          torch.from_numpy(np.ascontiguousarray(R[idx])).cuda()).cpu().numpy()
    # the oracle's network on the same BF16 input (r * (1/rms) in FP32, then
    # rounded) and BF16 weights, scaled back by rms
    wq = [op.bf16_round(a).astype(np.float64) for a in ws]
    rms = np.sqrt(np.mean(R.astype(np.float64) ** 2, axis=0))
    mask = g_ora.map >= 0
    ref = np.zeros((g_ora.npts, R.shape[1]))
    for s in range(R.shape[1]):
        xq = op.bf16_round(R[:, s] * np.float32(1.0 / rms[s])).astype(np.float64)
        vol, _ = op.grid_volume(g_ora, xq)
        y, _ = op.net_forward(vol[None], mask[None], wq)
        ref[g_ora.map[mask], s] = rms[s] * y[0][mask]
    ref = ref[idx]
    err = np.linalg.norm(W - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert err.max() <= 1e-5


def test_training_reduces_loss():
    from paper_1306_2953_gb300 import api
    lg, g_ora, idx = _grid(wl.MOL20.system)
    Hs = api.Hamiltonian(lg, np.full(lg.npts, 1.0))
    R = torch.from_numpy(wl.random_block(lg.npts, 16, 4).astype(np.float32)).cuda()
    X = api.shifted_poisson_cg(Hs, R, 200)
    w = torch.from_numpy(_flat_weights(wl.conv_init(1))).cuda()
    losses = api.precond_train(Hs, R, X, w, n_tiles=512, epochs=6, batch=64, seed=7)
    assert losses[-1] < 0.8 * losses[0], losses


def test_learned_preconditioner_speeds_up_early_sweeps():
    """What the trained network gains over the method without it: on the
    20-atom molecule, trained on the method's own Ritz residuals and their
    200-iteration shifted-Poisson CG solutions, the learned preconditioner
    leaves a smaller largest residual after five FP32 sweeps than the plain
    filter does from the same start."""
    from paper_1306_2953_gb300 import _lib, api
    w_ = wl.MOL20
    s = w_.system
    lg, g_ora, idx = _grid(s)
    atoms = wl.atom_positions(s)
    pr = api.Projectors(lg, atoms, wl.kb_couplings(s), s.r_c, s.r_cut)
    g_o, H_o, _, _ = oracle_system("mol", s)
    H = api.Hamiltonian(lg, wl.local_potential(g_o.coords, atoms)[idx], pr)
    psi0 = torch.from_numpy(wl.random_block(lg.npts, w_.n_states, w_.seed).astype(np.float32)).cuda()

    def run(kind, weights=None):
        S = api.Solver(H, psi0, w_.block, 1e-4, precond=kind)
        if weights is not None:
            S.set_precond_weights(weights)
        for _ in range(5):
            _, res, _ = S.step()
        return float(res.max())

    S0 = api.Solver(H, psi0, w_.block, 1e-4, precond=_lib.RS_PRECOND_LEARNED)
    R = S0.residual(0, 32).float().contiguous()
    Hs = api.Hamiltonian(lg, np.full(lg.npts, 1.0))
    X = api.shifted_poisson_cg(Hs, R, 200)
    X = X / X.pow(2).mean(dim=0, keepdim=True).sqrt()
    w = torch.from_numpy(_flat_weights(wl.conv_init(11))).cuda()
    api.precond_train(Hs, R, X, w, n_tiles=10000, epochs=5, batch=64, seed=11)
    learned = run(_lib.RS_PRECOND_LEARNED, w)
    plain = run(_lib.RS_PRECOND_FILTER)
    assert learned < 0.7 * plain, (learned, plain)
