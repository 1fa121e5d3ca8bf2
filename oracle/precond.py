"""Oracle: training targets and the learned convolutional preconditioner.

TEST INFRASTRUCTURE.  Neither part is in the paper (its preconditioner is
the filter of Sec. III); both follow the definitions stated here.

Training target: plain conjugate gradients for exactly ``n_iter``
iterations from x_0 = 0 on  (-1/2 Lap + sigma) x = r,  with the 25-point
kinetic stencil of Sec. V.A, x = 0 off the grid, sigma = 1 Ha (so the
operator is symmetric positive definite), one independent system per
column.

Network: y = L3(relu(L2(relu(L1(xhat))))) on the lattice, with
xhat = r / rms(r) (rms over the grid points of that column), bias-free 3^3
cross-correlation layers 1 -> C -> C -> 1 with zero padding, every layer's
output set to zero off the grid, and the preconditioned residual
K r = rms(r) * y.  Loss: mean squared error against the CG solution scaled
the same way, over the interior points of each training tile.  Optimiser:
Adam (Kingma & Ba 2015) with lr = 1e-3, beta = (0.9, 0.999), eps = 1e-8.
Weights are kept in FP32 and used in BF16 (round to nearest even).
"""
from __future__ import annotations

import numpy as np

from .grid import Grid
from .hamiltonian import Hamiltonian


def shifted_poisson_cg(grid: Grid, R: np.ndarray, sigma: float = 1.0, n_iter: int = 200) -> np.ndarray:
    """n_iter CG iterations on (-1/2 Lap + sigma) x = r for every column of R."""
    op = Hamiltonian(grid, np.full(grid.npts, sigma))
    B = np.array(R.reshape(len(R), -1), dtype=np.float64)
    X = np.zeros_like(B)
    Rr = B.copy()
    Pp = Rr.copy()
    rr = np.sum(Rr * Rr, axis=0)
    for _ in range(n_iter):
        Ap = op.apply(Pp)
        pAp = np.sum(Pp * Ap, axis=0)
        alpha = np.where(pAp != 0, rr / np.where(pAp != 0, pAp, 1.0), 0.0)
        X += alpha * Pp
        Rr -= alpha * Ap
        rr_new = np.sum(Rr * Rr, axis=0)
        beta = np.where(rr != 0, rr_new / np.where(rr != 0, rr, 1.0), 0.0)
        Pp = Rr + beta * Pp
        rr = rr_new
    return X.reshape(R.shape)


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 precision (nearest, ties to even),
    returned as float32."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def conv3(x: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Zero-padded 3^3 cross-correlation: x [B, ci, X, Y, Z], w [co, ci, 3, 3, 3]
    -> [B, co, X, Y, Z],  y(p) = sum_ci sum_d w[:, ci, d+1] x[ci, p+d]."""
    B, ci, X, Y, Z = x.shape
    xp = np.zeros((B, ci, X + 2, Y + 2, Z + 2))
    xp[:, :, 1:-1, 1:-1, 1:-1] = x
    y = np.zeros((B, w.shape[0], X, Y, Z))
    for a in range(3):
        for b in range(3):
            for c in range(3):
                y += np.einsum("oi,bixyz->boxyz", w[:, :, a, b, c], xp[:, :, a:a + X, b:b + Y, c:c + Z])
    return y


def conv3_grad_w(g: np.ndarray, x: np.ndarray) -> np.ndarray:
    """dL/dw for y = conv3(x, w) given g = dL/dy."""
    B, ci, X, Y, Z = x.shape
    xp = np.zeros((B, ci, X + 2, Y + 2, Z + 2))
    xp[:, :, 1:-1, 1:-1, 1:-1] = x
    gw = np.zeros((g.shape[1], ci, 3, 3, 3))
    for a in range(3):
        for b in range(3):
            for c in range(3):
                gw[:, :, a, b, c] = np.einsum("boxyz,bixyz->oi", g, xp[:, :, a:a + X, b:b + Y, c:c + Z])
    return gw


def conv3_grad_x(g: np.ndarray, w: np.ndarray) -> np.ndarray:
    """dL/dx for y = conv3(x, w) given g = dL/dy (the transposed correlation)."""
    B, co, X, Y, Z = g.shape
    gp = np.zeros((B, co, X + 2, Y + 2, Z + 2))
    gp[:, :, 1:-1, 1:-1, 1:-1] = g
    gx = np.zeros((B, w.shape[1], X, Y, Z))
    for a in range(3):
        for b in range(3):
            for c in range(3):
                # x[p] feeds y[p - d] with d = (a-1, b-1, c-1)
                gx += np.einsum("oi,boxyz->bixyz", w[:, :, a, b, c],
                                gp[:, :, 2 - a:2 - a + X, 2 - b:2 - b + Y, 2 - c:2 - c + Z])
    return gx


def net_forward(xhat: np.ndarray, mask: np.ndarray, ws):
    """xhat [B, X, Y, Z], mask [B, X, Y, Z] (1 on grid points) -> (y, cache)."""
    m = mask[:, None].astype(np.float64)
    x0 = xhat[:, None].astype(np.float64) * m
    z1 = conv3(x0, ws[0])
    a1 = np.maximum(z1, 0.0) * m
    z2 = conv3(a1, ws[1])
    a2 = np.maximum(z2, 0.0) * m
    y = conv3(a2, ws[2]) * m
    return y[:, 0], (x0, z1, a1, z2, a2, m)


def net_backward(gy: np.ndarray, cache, ws):
    """Gradients of the loss w.r.t. the three weight tensors given gy = dL/dy."""
    x0, z1, a1, z2, a2, m = cache
    g3 = gy[:, None] * m
    gw3 = conv3_grad_w(g3, a2)
    ga2 = conv3_grad_x(g3, ws[2])
    g2 = ga2 * m * (z2 > 0)
    gw2 = conv3_grad_w(g2, a1)
    ga1 = conv3_grad_x(g2, ws[1])
    g1 = ga1 * m * (z1 > 0)
    gw1 = conv3_grad_w(g1, x0)
    return [gw1, gw2, gw3]


def tile_loss(y: np.ndarray, target: np.ndarray, valid: np.ndarray):
    """Mean squared error over the valid points; returns (loss, dL/dy)."""
    n = max(int(valid.sum()), 1)
    d = (y - target) * valid
    return float(np.sum(d * d) / n), 2.0 * d / n


class Adam:
    def __init__(self, params, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.m = [np.zeros_like(p, dtype=np.float64) for p in params]
        self.v = [np.zeros_like(p, dtype=np.float64) for p in params]
        self.t = 0

    def step(self, params, grads):
        self.t += 1
        out = []
        for i, (p, g) in enumerate(zip(params, grads)):
            self.m[i] = self.b1 * self.m[i] + (1 - self.b1) * g
            self.v[i] = self.b2 * self.v[i] + (1 - self.b2) * g * g
            mh = self.m[i] / (1 - self.b1 ** self.t)
            vh = self.v[i] / (1 - self.b2 ** self.t)
            out.append(p - self.lr * mh / (np.sqrt(vh) + self.eps))
        return out


def grid_volume(grid: Grid, values: np.ndarray):
    """Scatter per-point values [np] onto the grid's bounding-box volume;
    returns (volume, mask)."""
    vol = np.zeros(grid.map.shape)
    mask = grid.map >= 0
    vol[mask] = values[grid.map[mask]]
    return vol, mask


def apply_learned(grid: Grid, R: np.ndarray, ws) -> np.ndarray:
    """K r for each column of R [np, nst] with the network weights ``ws``
    (used as given; round them to BF16 beforehand for the BF16 model)."""
    R2 = R.reshape(len(R), -1)
    out = np.zeros_like(R2, dtype=np.float64)
    mask = grid.map >= 0
    for s in range(R2.shape[1]):
        r = R2[:, s].astype(np.float64)
        rms = np.sqrt(np.mean(r * r))
        if rms == 0:
            continue
        vol, _ = grid_volume(grid, r / rms)
        y, _ = net_forward(vol[None], mask[None], ws)
        out[grid.map[mask], s] = rms * y[0][mask]
    return out.reshape(R.shape)
