"""Charge density and Gauss-law residual of the library (grpic_charge_density,
grpic_gauss_residual).

* rho (and J^4/c with gamma) against cloud-in-cell in numpy on the GPU's own particle state;
* the residual field against div E - 4 pi rho computed in numpy from the GPU's own d and rho;
* flat space, gamma-free deposit, FP64: over every step the residual changes by exactly
  -4 pi times the closed-form 3-D continuity defect of the moves the GPU made (the zig-zag
  deposit and the E step keep Gauss's law up to that term), on nodes away from the boundary.
"""
import numpy as np
import pytest

from parity_util import small_kerr
from test_oracle_deposit import cubic_defect
from paper_0904_0232_gb300.grpic import GRPIC_NO_GAMMA_IN_J, Simulation

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _cic(shape, x, w):
    rho = np.zeros(shape)
    i0 = np.floor(x[:3]).astype(int)
    f = x[:3] - i0
    for dk in (0, 1):
        for dj in (0, 1):
            for di in (0, 1):
                W = (f[0] if di else 1 - f[0]) * (f[1] if dj else 1 - f[1]) * (f[2] if dk else 1 - f[2])
                np.add.at(rho, (i0[2] + dk, i0[1] + dj, i0[0] + di), w * W)
    return rho


def _div_E(d):
    E = -d
    div = np.zeros_like(E[0])
    div[:, :, 1:] += E[0][:, :, 1:] - E[0][:, :, :-1]
    div[:, 1:, :] += E[1][:, 1:, :] - E[1][:, :-1, :]
    div[1:, :, :] += E[2][1:, :, :] - E[2][:-1, :, :]
    return div


@pytest.mark.parametrize("prec", ["fp64", "fp32_mixed"])
def test_charge_density_and_residual_field(prec):
    wl = small_kerr(n=24, ppc=1, seed=51)
    sim = Simulation(wl.nx, wl.ny, wl.nz, wl.m, wl.a, wl.c, wl.dt, precision=prec)
    sim.set_uniform_field(B=(0.0, 0.0, wl.B0))
    for s, sp in enumerate(wl.species):
        sim.load_particles(s, sp.q_over_m, sp.q_macro, sp.x4, sp.usp, sp.ids, umode=1)
    sim.step(2)
    shape = (wl.nz, wl.ny, wl.nx)
    rho_ref = np.zeros(shape)
    j4_ref = np.zeros(shape)
    for s, sp in enumerate(wl.species):
        x, u, _ = sim.get_particles(s)
        rho_ref += _cic(shape, x, sp.q_macro)
        j4_ref += _cic(shape, x, sp.q_macro * u[3] / wl.c)
    # both sides weigh the same stored positions in FP64; only the order of the atomic adds differs
    tol = 1e-12
    rho = sim.charge_density()
    j4 = sim.charge_density(with_gamma=True)
    scale = np.abs(rho_ref).max()
    assert np.abs(rho - rho_ref).max() <= tol * scale
    assert np.abs(j4 - j4_ref).max() <= tol * np.abs(j4_ref).max()
    res, mx = sim.gauss_residual()
    d, _, _ = sim.get_fields()
    ref = _div_E(d) - 4 * np.pi * rho_ref
    assert np.abs(res - ref).max() <= 1e-9 * max(1.0, np.abs(ref).max())
    inner = ref[2:-2, 2:-2, 2:-2]
    assert abs(mx - np.abs(inner).max()) <= 1e-9 * max(1.0, np.abs(inner).max())


def test_gauss_law_flat_space_closed_form():
    N, c, dt, q = 20, 1.0, 0.4, 0.05
    rng = np.random.default_rng(52)
    n = 40
    x = np.vstack([rng.uniform(8, 12, (3, n)), np.zeros((1, n))])
    usp = rng.normal(0, 0.3, (3, n))
    u = np.vstack([usp, np.sqrt(1 + (usp ** 2).sum(0))])
    sim = Simulation(N, N, N, 0.0, 0.0, c, dt, precision="fp64", flags=GRPIC_NO_GAMMA_IN_J)
    sim.set_uniform_field(B=(0.0, 0.0, 0.2))
    sim.load_particles(0, -1.0, -q, x, u, np.arange(n, dtype=np.uint32))
    sim.load_particles(1, 1.0, q, x + np.array([[0.3], [0.1], [-0.2], [0.0]]), u[[1, 0, 2, 3]],
                       np.arange(n, dtype=np.uint32))
    charge = (-q, q)
    sl = (slice(4, N - 4),) * 3

    def positions():
        out = []
        for s in (0, 1):
            xs, _, ids = sim.get_particles(s)
            out.append(xs[:, np.argsort(ids)])
        return out

    G, _ = sim.gauss_residual()
    for _ in range(6):
        before = positions()
        sim.step(1)
        after = positions()
        pred = np.zeros((N, N, N))
        for s in (0, 1):
            for p in range(n):
                pred += cubic_defect(N, before[s][:3, p], after[s][:3, p], charge[s])
        G1, _ = sim.gauss_residual()
        assert np.abs((G1 - G)[sl] + 4 * np.pi * pred[sl]).max() < 1e-13
        G = G1
