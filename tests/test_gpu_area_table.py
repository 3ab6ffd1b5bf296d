"""The far-field deposit from per-cell polynomial fits of the Eq. 18 integrand (grpic_tuning.area_table)
against the oracle's Gauss quadrature, and against the per-node deposit of the same library.

The workload puts a hole of m = 3 cells, a = 0.9m, in a 48^3 box: the far-field radius is then
r_fp64 + |a| + 4 = 18.7 cells, which the fits' own radius (4 + (m / 4.5e-7)^(1/6) = 17.7) does not
raise, so both deposit forms see the same warps take the far-field code, and about three quarters of
the particles take the fits."""
import numpy as np
import pytest

from parity_util import (TOL, check_j, compare_whole_state, gpu_from_oracle, oracle_start, particle_errors, rel_l2,
                         small_kerr, well_conditioned)
from paper_0904_0232_gb300 import synth
from paper_0904_0232_gb300.grpic import (GRPIC_STAGE_PUSH_DEPOSIT, GRPIC_STAGE_SORT, GRPIC_STAGE_ZERO_J, GrpicError,
                                         Simulation)

pytestmark = pytest.mark.gpu
M, A = 3.0, 2.7


@pytest.fixture(autouse=True, scope="module")
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _workload(n=48, seed=21):
    return small_kerr(n=n, ppc=1, seed=seed, m=M, a=A)


def _far_fraction(wl):
    near = 4 * M + A + 4
    assert near >= 4 + (M / 4.5e-7) ** (1 / 6)
    cen = np.array([(wl.nx - 1) / 2, (wl.ny - 1) / 2, (wl.nz - 1) / 2]).reshape(3, 1)
    R = np.concatenate([np.sqrt(((sp.x4[:3] - cen) ** 2).sum(0)) for sp in wl.species])
    return (R >= near).mean()


def _stage(wl, fields, table):
    ref = oracle_start(wl, fields=fields)
    sim = gpu_from_oracle(ref, wl, "fp32_mixed")
    sim.set_tuning(far_min_blocks=4, near_blocks_per_sm=1, sort_interval=1, overlap=0, split=0, j_tile=0, spread=16,
                   area_table=table)
    ref.zero_j()
    ref.push_deposit()
    sim.stage(GRPIC_STAGE_ZERO_J)
    sim.stage(GRPIC_STAGE_PUSH_DEPOSIT)
    sim.stage(GRPIC_STAGE_SORT)  # drops the particles the push removed, as the oracle's push does
    return ref, sim


def test_push_deposit_against_oracle():
    """One push + deposit in random non-uniform fields: every particle and every J node against the
    oracle within the FP32 bounds (J off the nodes of face-ambiguous splits, and the total flux)."""
    wl = _workload()
    assert _far_fraction(wl) > 0.7
    fields = synth.random_fields((wl.nz, wl.ny, wl.nx), 6, 0.02)
    ref, sim = _stage(wl, fields, 1)
    for s in range(len(wl.species)):
        ex, e4, eu = particle_errors(sim, ref, s)
        assert max(ex, e4, eu) <= TOL["fp32_mixed"]["particles"], (s, ex, e4, eu)
    J = sim.get_fields()[2]
    Jr = ref.get_fields()[2]
    check_j(J, Jr, ref, len(wl.species), "fp32_mixed")
    print("area table J rel L2", rel_l2(J, Jr))
    sim.close()


def test_same_as_per_node_deposit():
    """The same start deposited by the fits and by the Gauss nodes of the library: the pushes agree to
    FP32 rounding, and J, node by node, to 1e-6 of its largest value -- a tenth of the oracle bound,
    so a fit that is off at that level cannot hide in the FP32 tolerance."""
    wl = _workload(seed=22)
    fields = synth.random_fields((wl.nz, wl.ny, wl.nx), 7, 0.02)
    _, tab = _stage(wl, fields, 1)
    _, lat = _stage(wl, fields, 0)
    for s in range(len(wl.species)):
        xt, ut, it = tab.get_particles(s)
        xl, ul, il = lat.get_particles(s)
        ot, ol = np.argsort(it), np.argsort(il)
        assert np.array_equal(it[ot], il[ol])
        assert np.abs(xt[:, ot] - xl[:, ol]).max() <= 2e-7 * wl.nx
        assert np.abs(ut[:, ot] - ul[:, ol]).max() <= 2e-7 * max(1.0, np.abs(ul).max())
    Jt = tab.get_fields()[2]
    Jl = lat.get_fields()[2]
    assert np.abs(Jt - Jl).max() <= 1e-6 * np.abs(Jl).max(), np.abs(Jt - Jl).max() / np.abs(Jl).max()
    assert rel_l2(Jt, Jl) <= 1e-6, rel_l2(Jt, Jl)
    print("table vs nodes: J max", np.abs(Jt - Jl).max() / np.abs(Jl).max(), "rel L2", rel_l2(Jt, Jl))
    tab.close()
    lat.close()


def test_whole_steps_against_oracle():
    """Three whole cycles with the fits, every particle, J node and field value against the oracle
    after every step."""
    wl = well_conditioned(_workload(n=40, seed=23), 3, threads=0)
    ref = oracle_start(wl)
    sim = gpu_from_oracle(ref, wl, "fp32_mixed")
    sim.set_tuning(far_min_blocks=4, near_blocks_per_sm=1, sort_interval=1, overlap=0, split=0, j_tile=0, spread=16,
                   area_table=1)
    rec = []
    for step in range(3):
        ref.step(1)
        sim.step(1)
        compare_whole_state(sim, ref, len(wl.species), "fp32_mixed", step, rec)
    print("area table whole steps", rec)
    sim.close()


def test_tuning_round_trip_and_refusals():
    """area_table excludes the J tile; the fits are kept when it is switched off and on again; an FP64
    context keeps the setting and ignores it (its deposit is the FP64 quadrature)."""
    wl = _workload(n=24)
    sim = Simulation(wl.nx, wl.ny, wl.nz, wl.m, wl.a, wl.c, wl.dt, precision="fp32_mixed")
    sim.set_tuning(area_table=1)
    assert sim.tuning()["area_table"] == 1
    with pytest.raises(GrpicError):
        sim.set_tuning(area_table=1, j_tile=1)
    assert sim.tuning()["area_table"] == 1 and sim.tuning()["j_tile"] == 0
    sim.set_tuning(area_table=0)
    sim.set_tuning(area_table=1)
    sim.close()
    f64 = Simulation(wl.nx, wl.ny, wl.nz, wl.m, wl.a, wl.c, wl.dt, precision="fp64")
    f64.set_tuning(area_table=1)
    assert f64.tuning()["area_table"] == 1
    with pytest.raises(GrpicError):
        f64.set_tuning(area_table=1, j_tile=1)
    f64.close()
