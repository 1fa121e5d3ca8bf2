"""Learned preconditioner on the GPU against the FP64 oracle: the
shifted-Poisson CG targets, the conv net's forward pass, loss and weight
gradients (through the C ABI), the grid-level inference, and training.

Tolerances: FP64 CG after 200 iterations agrees with the oracle's to 1e-8
relative (the iteration is not converged to rounding, so rounding-order
differences stay small).  The network runs in FP32 with BF16 weights and
inputs; the oracle is given the same BF16-rounded values and computes in
FP64, so outputs agree to FP32 accumulation accuracy (1e-5 relative) and
gradients, which sum ~1e4 products, to 1e-4.

Training (Adam on the FP32 master weights, BF16 weights in the network):
after T steps the weight change w_T - w_0 of the GPU agrees with the
oracle's, stepped on the same tiles from the same weights, to 1e-2
relative in norm (the BF16-weight bound of the gradient pin).  Adam's first
steps move each weight by about lr * sign(g), so a gradient entry whose
sign the FP32 rounding flips moves that weight the other way; the test
allows that only where |g| is below 1e-3 of the largest gradient entry.
"""
import os
import tempfile

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


def test_convnet_at_training_tile_size_matches_oracle():
    """The training tiles' own size, 22^3 (a 16^3 interior plus 3 points of
    halo), where the weight-gradient kernel stages two planes per CTA."""
    from oracle import precond as op
    from paper_1306_2953_gb300 import api
    ws = wl.conv_init(6)
    w = np.concatenate([a.reshape(a.shape[0], a.shape[1], 27).ravel() for a in ws]).astype(np.float32)
    D = 22
    x, mask, tgt, valid = _tiles(ntiles=3, D=D, seed=4)
    valid[:] = False
    valid[3:-3, 3:-3, 3:-3] = True
    dev = lambda a, t=torch.float32: torch.from_numpy(np.ascontiguousarray(a)).to(t).cuda()
    y, g, loss = api.convnet_tiles(dev(w), dev(x), dev(mask.astype(np.uint8), torch.uint8), dev(tgt),
                                   dev(valid.astype(np.uint8), torch.uint8))
    wq = [op.bf16_round(a).astype(np.float64) for a in ws]
    yr, cache = op.net_forward(op.bf16_round(x).astype(np.float64), mask, wq)
    lr, gy = op.tile_loss(yr, tgt.astype(np.float64), valid[None] & mask)
    grf = np.concatenate([a.reshape(a.shape[0], a.shape[1], 27).ravel() for a in op.net_backward(gy, cache, wq)])
    assert np.abs(y.cpu().numpy() - yr).max() <= 1e-5 * np.abs(yr).max()
    assert abs(loss - lr) <= 1e-5 * lr
    assert np.abs(g.cpu().numpy() - grf).max() <= 1e-4 * np.abs(grf).max()


def test_adam_training_steps_match_oracle():
    """rs_precond_train_tiles (the GPU forward, backward and Adam kernels)
    against the oracle's net_forward / net_backward / Adam over the same
    seeded 22^3 tiles at the training batch size: 128 tiles in batches of
    64, two epochs (four Adam steps)."""
    from oracle import precond as op
    from paper_1306_2953_gb300 import api
    D, ntiles, batch, epochs, lr = 22, 128, 64, 2, 1e-3
    x, mask, tgt, valid = _tiles(ntiles=ntiles, D=D, seed=12)
    valid[:] = False
    valid[3:-3, 3:-3, 3:-3] = True
    ws0 = wl.conv_init(3)
    w = torch.from_numpy(_flat_weights(ws0)).cuda()
    dev = lambda a, t=torch.float32: torch.from_numpy(np.ascontiguousarray(a)).to(t).cuda()
    losses = api.precond_train_tiles(w, dev(x), dev(mask.astype(np.uint8), torch.uint8), dev(tgt),
                                     dev(valid.astype(np.uint8), torch.uint8), batch, epochs, lr)
    w_gpu = w.cpu().numpy().astype(np.float64)
    # the oracle: FP64 master weights, used in BF16 (rounded through FP32)
    params = [a.astype(np.float32).astype(np.float64) for a in ws0]
    opt = op.Adam(params, lr=lr)
    xq = op.bf16_round(x).astype(np.float64)
    ora_losses, gmax = [], []
    for ep in range(epochs):
        tot = 0.0
        for t0 in range(0, ntiles, batch):
            wq = [op.bf16_round(p.astype(np.float32)).astype(np.float64) for p in params]
            y, cache = op.net_forward(xq[t0:t0 + batch], mask[t0:t0 + batch], wq)
            l, gy = op.tile_loss(y, tgt[t0:t0 + batch].astype(np.float64), valid[None] & mask[t0:t0 + batch])
            grads = op.net_backward(gy, cache, wq)
            gmax.append(np.concatenate([gg.ravel() for gg in grads]))
            params = opt.step(params, grads)
            tot += l
        ora_losses.append(tot / (ntiles // batch))
    w_ora = np.concatenate([p.reshape(p.shape[0], p.shape[1], 27).ravel() for p in params])
    w0 = _flat_weights(ws0).astype(np.float64)
    d_gpu, d_ora = w_gpu - w0, w_ora - w0
    assert np.linalg.norm(d_gpu - d_ora) <= 1e-2 * np.linalg.norm(d_ora)
    # element by element: a weight may move the other way only where a
    # gradient entry is too small for its sign to survive FP32 rounding
    small = np.min(np.abs(np.stack(gmax)), axis=0) <= 1e-3 * np.abs(np.stack(gmax)).max()
    big_diff = np.abs(d_gpu - d_ora) > 0.1 * lr
    assert not np.any(big_diff & ~small), np.nonzero(big_diff & ~small)
    # the epoch losses use each side's own BF16 weights, which may differ by
    # one BF16 unit where the master weights straddle a rounding boundary
    assert np.allclose(losses, ora_losses, rtol=1e-3)


def test_precond_save_load_roundtrip(tmp_path):
    """rs_precond_save writes the solver's weights; rs_precond_load reads them
    into another solver, which saves the same bytes back and steps alike (an
    FP32 solver: its projection integrals are FP32 sums in atomic order, so
    two runs agree to FP32 rounding of H psi, ~1e-6 relative, not bitwise);
    corrupted or foreign files are refused."""
    from paper_1306_2953_gb300 import _lib, api
    from paper_1306_2953_gb300._lib import RsError
    lg, g_ora, idx = _grid()
    H = api.Hamiltonian(lg, np.zeros(lg.npts))
    psi0 = torch.from_numpy(np.ascontiguousarray(wl.random_block(g_ora.npts, 16, 2)[idx])).float().cuda()
    w = torch.from_numpy(_flat_weights(wl.conv_init(4))).cuda()
    a = api.Solver(H, psi0, 16, 1e-4, precond=_lib.RS_PRECOND_LEARNED)
    a.set_precond_weights(w)
    path = tmp_path / "w.rsnn"
    a.save_precond(str(path))
    raw = path.read_bytes()
    assert raw[:4] == b"RSNN" and len(raw) == 12 + 4 * 2160 + 4
    b = api.Solver(H, psi0, 16, 1e-4, precond=_lib.RS_PRECOND_LEARNED)
    b.load_precond(str(path))
    b.save_precond(str(tmp_path / "w2.rsnn"))
    assert (tmp_path / "w2.rsnn").read_bytes() == raw
    ea, ra, _ = a.step()
    eb, rb, _ = b.step()
    assert torch.allclose(ea, eb, rtol=1e-6, atol=0) and torch.allclose(ra, rb, rtol=1e-3, atol=1e-9)
    bad = bytearray(raw)
    bad[100] ^= 1
    (tmp_path / "bad.rsnn").write_bytes(bytes(bad))
    with pytest.raises(RsError):
        b.load_precond(str(tmp_path / "bad.rsnn"))
    with pytest.raises(RsError):
        api.Solver(H, psi0, 16, 1e-4).load_precond(str(path))   # not a learned solver


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
    S0.train_precond(lg, torch.from_numpy(_flat_weights(wl.conv_init(11))).cuda(), n_res=32, n_tiles=10000,
                     epochs=5, batch=64, seed=11)
    w = torch.empty(2160, dtype=torch.float32, device="cuda")
    path = os.path.join(tempfile.mkdtemp(), "w.rsnn")
    S0.save_precond(path)
    raw = np.frombuffer(open(path, "rb").read()[12:12 + 4 * 2160], dtype="<f4")
    w.copy_(torch.from_numpy(raw.copy()))
    learned = run(_lib.RS_PRECOND_LEARNED, w)
    plain = run(_lib.RS_PRECOND_FILTER)
    assert learned < 0.7 * plain, (learned, plain)
