"""Pins of the oracle's current deposit (Sec. 4, Eq. 18, readings A12-A13).

* Flat space, gamma off: Umeda's zig-zag with midpoint transverse weights.  For trilinear
  node charge, d(uvw) = du v w + u dv w + u v dw + du dv dw / 4 (bars = segment midpoints),
  so the deposit satisfies continuity exactly in 2-D and, in 3-D, up to the closed-form
  cubic term q/4 * prod_ax (+-dx_ax) per segment and node.  Both are checked to roundoff.
* A hand-worked single-cell move (tests/golden/umeda_single_cell.json).
* Flat face weights are bilinear; curved weights sum to one and converge with Q to a
  reference quadrature of the same integrand computed here with scipy.
"""
import json
import os

import numpy as np
import pytest

import oracle as O

RNG = np.random.default_rng(4242)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def cic_rho(N, x, q):
    """Trilinear (cloud-in-cell) charge at the nodes."""
    rho = np.zeros((N, N, N))
    for p in range(x.shape[1]):
        i0 = np.floor(x[:3, p]).astype(int)
        w = x[:3, p] - i0
        for dk in (0, 1):
            for dj in (0, 1):
                for di in (0, 1):
                    W = (w[0] if di else 1 - w[0]) * (w[1] if dj else 1 - w[1]) * (w[2] if dk else 1 - w[2])
                    rho[i0[2] + dk, i0[1] + dj, i0[0] + di] += q * W
    return rho


def div_nodes(J):
    """Backward-difference divergence of edge-centred J at the nodes."""
    div = np.zeros_like(J[0])
    div[:, :, 1:] += J[0][:, :, 1:] - J[0][:, :, :-1]
    div[:, :, 0] += J[0][:, :, 0]
    div[:, 1:, :] += J[1][:, 1:, :] - J[1][:, :-1, :]
    div[:, 0, :] += J[1][:, 0, :]
    div[1:, :, :] += J[2][1:, :, :] - J[2][:-1, :, :]
    div[0, :, :] += J[2][0, :, :]
    return div


def zigzag_segments(x1, x2):
    """Umeda's relay point: two straight segments, each inside one cell."""
    c1 = np.floor(x1)
    c2 = np.floor(x2)
    xr = np.minimum(np.minimum(c1, c2) + 1.0, np.maximum(np.maximum(c1, c2), 0.5 * (x1 + x2)))
    return [(x1, xr, c1.astype(int)), (xr, x2, c2.astype(int))]


def cubic_defect(N, x1, x2, q):
    """q/4 * prod_ax (s_ax * dx_ax) at the 8 nodes of each segment's cell, s = +1 for the
    upper node on that axis, -1 for the lower."""
    out = np.zeros((N, N, N))
    for a, b, cell in zigzag_segments(x1, x2):
        dx = b - a
        for dk in (0, 1):
            for dj in (0, 1):
                for di in (0, 1):
                    s = np.array([1 if di else -1, 1 if dj else -1, 1 if dk else -1])
                    out[cell[2] + dk, cell[1] + dj, cell[0] + di] += 0.25 * q * np.prod(s * dx)
    return out


def test_flat_continuity_closed_form():
    N, dt, q = 14, 0.4, 0.37
    for t in range(40):
        o = O.Oracle(N, N, N, 0.0, 0.0, 1.0, dt)
        x1 = RNG.uniform(4, 9, 3)
        x2 = x1 + RNG.uniform(-0.95, 0.95, 3)
        if t % 4 == 0:
            x2[2] = x1[2]  # 2-D move: exactly conserving
        o.deposit(x1, x2, q, 1.0)
        _, _, J = o.get_fields()
        res = cic_rho(N, x2.reshape(3, 1), q) - cic_rho(N, x1.reshape(3, 1), q) + dt * div_nodes(J)
        pred = cubic_defect(N, x1, x2, q)
        assert np.abs(res - pred).max() < 1e-15
        if t % 4 == 0:
            assert np.abs(res).max() < 1e-15


def test_gamma_factor_scales_flux():
    N = 12
    x1, x2 = np.array([5.2, 5.7, 6.1]), np.array([5.9, 5.4, 6.3])
    o1 = O.Oracle(N, N, N, 2.0, 1.0, 1.0, 0.4)
    o2 = O.Oracle(N, N, N, 2.0, 1.0, 1.0, 0.4)
    o1.deposit(x1, x2, 0.5, 1.0)
    o2.deposit(x1, x2, 0.5, 1.7)
    assert np.allclose(o2.get_fields()[2], 1.7 * o1.get_fields()[2], rtol=1e-15, atol=0)


def test_golden_single_cell_move():
    """Hand-worked: q = 1, dt = 1, m = 0, move (10.25, 10.5, 10.5) -> (10.75, 10.5, 10.5).
    Relay at the midpoint 10.5; two segments of 0.25, each with transverse weights 1/2 x 1/2,
    so each of the four J^x edges of cell (10, 10, 10) receives 2 * 0.25 * 0.25 = 0.125."""
    with open(os.path.join(GOLDEN, "umeda_single_cell.json")) as f:
        gold = json.load(f)
    N = gold["N"]
    o = O.Oracle(N, N, N, 0.0, 0.0, 1.0, gold["dt"])
    o.deposit(np.array(gold["x1"]), np.array(gold["x2"]), gold["q"], 1.0)
    _, _, J = o.get_fields()
    expect = np.zeros_like(J)
    for comp, k, j, i, v in gold["J"]:
        expect[comp, k, j, i] = v
    assert np.abs(J - expect).max() < 1e-16


def test_flat_face_weights_are_bilinear():
    N = 12
    o = O.Oracle(N, N, N, 0.0, 0.0, 1.0, 0.4)
    for K in range(3):
        cell = np.array([4, 5, 6])
        P = cell + RNG.uniform(0, 1, 3)
        W = o.face_weights(K, P, cell)
        I, Jx = (K + 1) % 3, (K + 2) % 3
        wi, wj = P[I] - cell[I], P[Jx] - cell[Jx]
        assert np.allclose(W, [(1 - wi) * (1 - wj), wi * (1 - wj), (1 - wi) * wj, wi * wj], atol=1e-15)


def test_curved_face_weights_quadrature():
    """Eq. 18 sub-areas: weights sum to 1, and Q = 8 matches an adaptive scipy integral of
    sqrt(g_II g_JJ - g_IJ^2) (metric from the pinned Eq. 4) to 1e-10."""
    from scipy.integrate import dblquad

    N, m, a = 24, 3.0, 2.7
    oq = {Q: O.Oracle(N, N, N, m, a, 1.0, 0.4, quad_order=Q) for Q in (1, 2, 4, 8)}
    Xc = oq[2].centre
    errs = {Q: [] for Q in oq}
    for K in range(3):
        cell = np.array([15, 13, 16])
        P = cell + np.array([0.3, 0.8, 0.45])
        I, Jx = (K + 1) % 3, (K + 2) % 3

        def integrand(xj, xi):
            pos = np.zeros(3)
            pos[K] = P[K]
            pos[I] = xi
            pos[Jx] = xj
            g = O.metric(pos - Xc, m, a)
            return np.sqrt(g[I, I] * g[Jx, Jx] - g[I, Jx] ** 2)

        def area(i0, i1, j0, j1):
            return dblquad(integrand, i0, i1, j0, j1, epsabs=1e-13, epsrel=1e-13)[0]

        ci, cj = cell[I], cell[Jx]
        A = [area(P[I], ci + 1, P[Jx], cj + 1), area(ci, P[I], P[Jx], cj + 1),
             area(P[I], ci + 1, cj, P[Jx]), area(ci, P[I], cj, P[Jx])]
        Wref = np.array(A) / sum(A)
        for Q, o in oq.items():
            W = o.face_weights(K, P, cell)
            assert W.sum() == pytest.approx(1.0, abs=1e-15)
            errs[Q].append(np.abs(W - Wref).max())
    assert max(errs[8]) < 1e-10
    assert max(errs[4]) < max(errs[2]) < max(errs[1])
    # curvature matters here: the weights differ from bilinear
    assert max(errs[1]) > 1e-6
