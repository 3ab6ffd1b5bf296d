"""GPU (CUDA library through the C ABI) vs the FP64 oracle, element by element on identical
seeded inputs: each stage of the timestep on its own, then whole steps, in FP64 and FP32-mixed."""
import numpy as np
import pytest

import oracle as O
from parity_util import (TOL, check_j, compare_whole_state, gpu_from_oracle, oracle_start, particle_errors, rel_l2,
                         small_kerr, well_conditioned)
from paper_0904_0232_gb300 import synth
from paper_0904_0232_gb300.grpic import (GRPIC_LITERAL_HALF_STEPS, GRPIC_STAGE_B_HALF, GRPIC_STAGE_B_HALF2,
                                         GRPIC_STAGE_E, GRPIC_STAGE_PUSH_DEPOSIT, GRPIC_STAGE_ZERO_J,
                                         GRPIC_U_CONTRA_SPATIAL, GRPIC_U_COV_SPATIAL, GrpicError, Simulation)

pytestmark = pytest.mark.gpu
PRECISIONS = ["fp64", "fp32_mixed"]


@pytest.fixture(autouse=True, scope="module")
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _rand_fields(shape, seed, scale=0.05):
    return synth.random_fields(shape, seed, scale)


@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("dims", [(24, 24, 24), (20, 27, 33)])
def test_uniform_field_init(prec, dims):
    nx, ny, nz = dims
    ref = O.Oracle(nx, ny, nz, 2.0, 1.7, 1.0, 0.4)
    E, B = (0.01, -0.02, 0.03), (0.05, 0.02, 0.1)
    ref.init_uniform_field(E=E, B=B)
    sim = Simulation(nx, ny, nz, 2.0, 1.7, 1.0, 0.4, precision=prec)
    sim.set_uniform_field(E, B)
    d, b, _ = sim.get_fields()
    dr, br, _ = ref.get_fields()
    tol = 1e-14 if prec == "fp64" else 1e-7
    assert rel_l2(d, dr) <= tol and rel_l2(b, br) <= tol


@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("dims", [(24, 24, 24), (19, 26, 31)])
def test_b_half_step(prec, dims):
    nx, ny, nz = dims
    ref = O.Oracle(nx, ny, nz, 2.0, 1.6, 1.0, 0.4, threads=0)
    d, b = _rand_fields((nz, ny, nx), 3)
    ref.set_fields(d, b)
    sim = Simulation(nx, ny, nz, 2.0, 1.6, 1.0, 0.4, precision=prec)
    sim.set_fields(*ref.get_fields()[:2])
    ref.b_half()
    sim.stage(GRPIC_STAGE_B_HALF)
    d1, b1, _ = sim.get_fields()
    dr, br, _ = ref.get_fields()
    assert rel_l2(b1, br) <= TOL[prec]["fields"]
    assert rel_l2(b1 - b, br - b) <= (1e-11 if prec == "fp64" else 2e-4)  # the update itself
    assert np.array_equal(d1, dr) if prec == "fp64" else rel_l2(d1, dr) <= 1e-7


@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("literal", [False, True])
def test_both_b_half_steps(prec, literal):
    """First and second B half-steps, time-centred (default) and literal explicit."""
    nx, ny, nz = 22, 25, 28
    ref = O.Oracle(nx, ny, nz, 2.0, 1.6, 1.0, 0.4, threads=0, flags=O.LITERAL_HALF_STEPS if literal else 0)
    d, b = _rand_fields((nz, ny, nx), 13)
    ref.set_fields(d, b)
    sim = Simulation(nx, ny, nz, 2.0, 1.6, 1.0, 0.4, precision=prec, flags=GRPIC_LITERAL_HALF_STEPS if literal else 0)
    sim.set_fields(d, b)
    ref.b_half()
    ref.b_half2()
    sim.stage(GRPIC_STAGE_B_HALF)
    sim.stage(GRPIC_STAGE_B_HALF2)
    _, b1, _ = sim.get_fields()
    _, br, _ = ref.get_fields()
    assert rel_l2(b1, br) <= TOL[prec]["fields"]
    assert rel_l2(b1 - b, br - b) <= (1e-11 if prec == "fp64" else 2e-4)


@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("literal", [False, True])
def test_e_step_variants(prec, literal):
    nx, ny, nz = 21, 24, 27
    ref = O.Oracle(nx, ny, nz, 2.0, 1.6, 1.0, 0.4, threads=0, flags=O.LITERAL_HALF_STEPS if literal else 0)
    d, b = _rand_fields((nz, ny, nx), 14)
    J = np.random.default_rng(15).standard_normal((3, nz, ny, nx)) * 1e-3
    ref.set_fields(d, b)
    ref.set_j(J)
    sim = Simulation(nx, ny, nz, 2.0, 1.6, 1.0, 0.4, precision=prec, flags=GRPIC_LITERAL_HALF_STEPS if literal else 0)
    sim.set_fields(d, b)
    sim.set_j(J)
    ref.e_step()
    sim.stage(GRPIC_STAGE_E)
    d1, _, _ = sim.get_fields()
    dr, _, _ = ref.get_fields()
    assert rel_l2(d1, dr) <= TOL[prec]["fields"]
    assert rel_l2(d1 - d, dr - d) <= (1e-11 if prec == "fp64" else 2e-4)


@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("dims", [(24, 24, 24), (19, 26, 31)])
def test_e_step(prec, dims):
    nx, ny, nz = dims
    ref = O.Oracle(nx, ny, nz, 2.0, 1.6, 1.0, 0.4, threads=0)
    d, b = _rand_fields((nz, ny, nx), 4)
    J = np.random.default_rng(9).standard_normal((3, nz, ny, nx)) * 1e-3
    ref.set_fields(d, b)
    ref.set_j(J)
    sim = Simulation(nx, ny, nz, 2.0, 1.6, 1.0, 0.4, precision=prec)
    sim.set_fields(d, b)
    sim.set_j(J)
    ref.e_step()
    sim.stage(GRPIC_STAGE_E)
    d1, b1, _ = sim.get_fields()
    dr, br, _ = ref.get_fields()
    assert rel_l2(d1, dr) <= TOL[prec]["fields"]
    assert rel_l2(d1 - d, dr - d) <= (1e-11 if prec == "fp64" else 2e-4)


@pytest.mark.parametrize("prec", PRECISIONS)
def test_load_completes_u4_like_oracle(prec):
    wl = small_kerr(n=24, ppc=2, seed=7)
    sim = Simulation(wl.nx, wl.ny, wl.nz, wl.m, wl.a, wl.c, wl.dt, precision=prec)
    ref = O.Oracle(wl.nx, wl.ny, wl.nz, wl.m, wl.a, wl.c, wl.dt)
    sp = wl.species[0]
    sim.load_particles(0, sp.q_over_m, sp.q_macro, sp.x4, sp.usp, sp.ids, umode=GRPIC_U_COV_SPATIAL)
    ref.load_particles(0, sp.q_over_m, sp.q_macro, sp.x4, sp.usp, sp.ids, umode=1)
    ex, e4, eu = particle_errors(sim, ref, 0)
    tol = 1e-13 if prec == "fp64" else 1e-7
    assert ex <= tol and eu <= tol


def test_load_rejects_bad_input():
    sim = Simulation(16, 16, 16, 1.0, 0.5, 1.0, 0.4, precision="fp64")
    x4 = np.array([[0.5], [5.0], [5.0], [0.0]])
    u4 = np.array([[0.0], [0.0], [0.0], [1.0]])
    with pytest.raises(GrpicError) as ei:
        sim.load_particles(0, -1.0, 0.0, x4, u4, np.array([0], np.uint32))
    assert ei.value.code == 1
    # contravariant completion inside the ergoregion (outside the horizon) is ambiguous and refused:
    # m = 1, a = 0.5, equatorial plane: horizon at R = 1.93, ergosurface at R = 2.06
    x4 = np.array([[7.5 + 2.0], [7.5], [7.5], [0.0]])
    with pytest.raises(GrpicError):
        sim.load_particles(0, -1.0, 0.0, x4, np.zeros((4, 1)), np.array([0], np.uint32), umode=GRPIC_U_CONTRA_SPATIAL)


@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("Q", [1, 2, 3])
def test_push_deposit_stage(prec, Q):
    wl = small_kerr(n=24, ppc=1, seed=8)
    d, b = _rand_fields((wl.nz, wl.ny, wl.nx), 5, scale=0.02)
    ref = oracle_start(wl, quad_order=Q, fields=(d, b))
    sim = gpu_from_oracle(ref, wl, prec, quad_order=Q)
    ref.zero_j()
    ref.push_deposit()
    sim.stage(GRPIC_STAGE_ZERO_J)
    sim.stage(GRPIC_STAGE_PUSH_DEPOSIT)
    tol = TOL[prec]
    for s in range(2):
        ex, e4, eu = particle_errors(sim, ref, s)
        assert ex <= tol["particles"] and eu <= tol["particles"], (s, ex, eu)
        assert e4 <= tol["particles"]
    _, _, J = sim.get_fields()
    _, _, Jr = ref.get_fields()
    check_j(J, Jr, ref, 2, prec)


def _whole_steps_against_oracle(wl, prec, nsteps, record):
    """Whole cycles (B/2, push + deposit, B/2, E, removal, sort) on a well-conditioned workload:
    every particle, every J node and every field value is compared after every step (the face
    mask is asserted empty).  Bound after step k (0-based): (k + 1) x the per-step tolerance --
    independent rounding errors of k + 1 steps adding up."""
    ref = oracle_start(wl)
    sim = gpu_from_oracle(ref, wl, prec)
    for step in range(nsteps):
        ref.step(1)
        sim.step(1)
        compare_whole_state(sim, ref, len(wl.species), prec, step, record)
    return ref, sim


@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("dims", [(24, 24, 24), (20, 26, 30)])
def test_full_steps(prec, dims):
    """Three whole cycles against the oracle, all state compared at every step."""
    wl = small_kerr(n=dims[0], ppc=1, seed=9, nxyz=None if dims[0] == dims[1] == dims[2] else dims)
    n0 = sum(sp.ids.size for sp in wl.species)
    wl = well_conditioned(wl, 3, threads=0)
    assert sum(sp.ids.size for sp in wl.species) >= 0.99 * n0
    rec = []
    _whole_steps_against_oracle(wl, prec, 3, rec)
    print("full_steps", prec, dims, rec)


@pytest.mark.parametrize("prec", PRECISIONS)
def test_removal_matches_oracle(prec):
    """Particles aimed at the horizon and at the outer boundary are removed identically."""
    m, a, N = 2.0, 1.0, 20
    ref = O.Oracle(N, N, N, m, a, 1.0, 0.4, flags=O.FROZEN_FIELDS)
    ref.init_uniform_field(B=(0.0, 0.0, 0.05))
    Xc = ref.centre
    rp = ref.r_plus
    n = 64
    rng = np.random.default_rng(3)
    ang = rng.uniform(0, 2 * np.pi, n)
    x4 = np.zeros((4, n))
    usp = np.zeros((3, n))
    half = n // 2
    # first half: just outside the horizon moving inwards; second half: near the faces moving out
    x4[0, :half] = Xc[0] + (rp + 0.6) * np.cos(ang[:half])
    x4[1, :half] = Xc[1] + (rp + 0.6) * np.sin(ang[:half])
    x4[2, :half] = Xc[2]
    usp[0, :half] = -0.9 * np.cos(ang[:half])
    usp[1, :half] = -0.9 * np.sin(ang[:half])
    x4[0, half:] = rng.uniform(1.05, 1.3, half)
    x4[1, half:] = rng.uniform(3, N - 4, half)
    x4[2, half:] = rng.uniform(3, N - 4, half)
    usp[0, half:] = -0.7
    ids = np.arange(n, dtype=np.uint32)
    ref.load_particles(0, 0.0, 0.0, x4, usp, ids, umode=1)
    sim = Simulation(N, N, N, m, a, 1.0, 0.4, precision=prec)
    d, b, _ = ref.get_fields()
    sim.set_fields(d, b)
    xs, us, idss = ref.get_particles(0)
    sim.load_particles(0, 0.0, 0.0, xs, us, idss)
    for _ in range(3):
        ref.step(1)
        sim.step(1)
        _, _, ir = ref.get_particles(0)
        _, _, ig = sim.get_particles(0)
        assert np.array_equal(np.sort(ig), ir)
    st = sim.stats()
    rs = ref.stats()
    assert st["removed_horizon"] == rs["removed_horizon"] > 0
    assert st["removed_outer"] == rs["removed_outer"] > 0


@pytest.mark.parametrize("prec", PRECISIONS)
def test_load_drops_particles_inside_horizon(prec):
    wl = small_kerr(n=24, ppc=2, seed=12, r_min=0.0)
    ref = O.Oracle(wl.nx, wl.ny, wl.nz, wl.m, wl.a, wl.c, wl.dt)
    sim = Simulation(wl.nx, wl.ny, wl.nz, wl.m, wl.a, wl.c, wl.dt, precision=prec)
    sp = wl.species[1]
    ref.load_particles(0, sp.q_over_m, sp.q_macro, sp.x4, sp.usp, sp.ids, umode=1)
    sim.load_particles(0, sp.q_over_m, sp.q_macro, sp.x4, sp.usp, sp.ids, umode=GRPIC_U_COV_SPATIAL)
    assert ref.stats()["removed_horizon"] > 0
    assert sim.stats()["removed_horizon"] == ref.stats()["removed_horizon"]
    ex, e4, eu = particle_errors(sim, ref, 0)
    assert max(ex, eu) <= (1e-13 if prec == "fp64" else 1e-7)


@pytest.mark.parametrize("prec", PRECISIONS)
def test_near_horizon_full_density(prec):
    """Every cell filled (8 per cell per species), Kerr a = 0.9 m, m = 4 on a 32^3 grid: particles
    start just outside the horizon, fall in and are removed; two whole steps against the oracle,
    all state compared at every step."""
    wl = synth.kerr_ion_electron_128(seed=3, n=32)
    n0 = sum(sp.ids.size for sp in wl.species)
    wl = well_conditioned(wl, 2, threads=0)
    assert sum(sp.ids.size for sp in wl.species) >= 0.99 * n0
    loaded_inside = oracle_start(wl).stats()["removed_horizon"]
    rec = []
    ref, sim = _whole_steps_against_oracle(wl, prec, 2, rec)
    print("near_horizon", prec, rec)
    assert sim.stats()["removed_horizon"] == ref.stats()["removed_horizon"] - loaded_inside > 0


def test_empty_species_and_zero_particles():
    sim = Simulation(16, 16, 16, 1.0, 0.5, 1.0, 0.4, precision="fp32_mixed")
    sim.set_uniform_field(B=(0, 0, 0.1))
    sim.load_particles(0, -1.0, 0.01, np.zeros((4, 0)), np.zeros((4, 0)), np.zeros(0, np.uint32))
    sim.step(2)
    assert sim.num_particles(0) == 0
    x, u, ids = sim.get_particles(0)
    assert x.shape == (4, 0)


def test_step_limit_is_reported():
    """A state moving two cells in one step (u^4 given inconsistent with u^i) is refused with
    GRPIC_ERR_CFL; the kernels clamp every index, so nothing is accessed out of bounds."""
    sim = Simulation(16, 16, 16, 0.0, 0.0, 1.0, 0.4, precision="fp64")
    x4 = np.array([[7.0], [7.0], [7.0], [0.0]])
    u4 = np.array([[5.0], [0.0], [0.0], [1.0]])
    sim.load_particles(0, 0.0, 0.0, x4, u4, np.array([0], np.uint32))
    with pytest.raises(GrpicError) as ei:
        sim.step(1)
    assert ei.value.code == 4


@pytest.mark.parametrize("prec", PRECISIONS)
def test_no_gamma_flag(prec):
    wl = small_kerr(n=20, ppc=1, seed=10)
    ref = oracle_start(wl, flags=O.NO_GAMMA_IN_J)
    sim = gpu_from_oracle(ref, wl, prec, flags=1)
    ref.zero_j()
    ref.push_deposit()
    sim.stage(GRPIC_STAGE_ZERO_J)
    sim.stage(GRPIC_STAGE_PUSH_DEPOSIT)
    check_j(sim.get_fields()[2], ref.get_fields()[2], ref, 2, prec)


def test_schwarzschild_pairs_full_run():
    """The small workload end to end in FP64: a = 0, m = 2, 32^3, e-/e+ pairs outside R = 3m,
    20 whole steps; particles, J and fields against the oracle after steps 1, 5 and 20."""
    wl = synth.schwarzschild_pairs_32(seed=1)
    ref = oracle_start(wl)
    sim = gpu_from_oracle(ref, wl, "fp64")
    done = 0
    for upto, tol in ((1, 1e-12), (5, 1e-11), (20, 1e-9)):
        ref.step(upto - done)
        sim.step(upto - done)
        done = upto
        for s in range(2):
            ex, e4, eu = particle_errors(sim, ref, s)
            assert max(ex, eu) <= tol, (upto, s, ex, eu)
        d, b, J = sim.get_fields()
        dr, br, Jr = ref.get_fields()
        assert rel_l2(J, Jr) <= tol and rel_l2(b, br) <= tol and rel_l2(d, dr) <= tol


@pytest.mark.parametrize("prec", ["fp64", "fp32_mixed"])
def test_fields_contra_readout(prec):
    """grpic_get_fields_contra against the oracle's read-out on random fields around a = 0.9m (every
    face of cells 1 .. n-2; zero on the outer layer), and d as grpic_get_fields returns it."""
    N, m = 24, 2.0
    rng = np.random.default_rng(11)
    d = 0.05 * rng.standard_normal((3, N, N, N))
    b = 0.1 + 0.05 * rng.standard_normal((3, N, N, N))
    ref = O.Oracle(N, N, N, m, 0.9 * m, 1.0, 0.4, threads=0)
    ref.set_fields(d, b)
    sim = Simulation(N, N, N, m, 0.9 * m, 1.0, 0.4, precision=prec)
    sim.set_fields(d, b)
    dd, h = sim.get_fields_contra()
    hr = ref.get_contra_h()
    assert np.array_equal(dd, sim.get_fields()[0])
    tol = 1e-13 if prec == "fp64" else 2e-6
    assert np.abs(h - hr).max() <= tol * np.abs(hr).max(), np.abs(h - hr).max()
    assert np.abs(h[:, 0]).max() == 0.0 and np.abs(h[:, :, -1]).max() == 0.0
    sim.close()
