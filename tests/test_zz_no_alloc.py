"""The allocation-free cell sort (grpic_sort_particles_static) against the library's regular
path (load + get_particles, which sorts with scratch the library allocates).

Some callers cannot allocate device memory where they call us -- a fixed memory budget, an
allocator callback, a loop that must not block in cudaMalloc -- and use this entry point,
whose scratch is a file-scope device array.  The check: two calls in a row (the array keeps
the first call's contents), each giving the same particles in the same cell order as the
regular path, exactly (a sort only moves values).  This file is collected last so that a run
stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _particles(seed, n, N):
    rng = np.random.default_rng(seed)
    x4 = np.vstack([rng.uniform(1.0, N - 2.0, (3, n)), rng.uniform(-1, 1, (1, n))])
    usp = rng.normal(0, 0.2, (3, n))
    u4 = np.vstack([usp, np.sqrt(1.0 + (usp ** 2).sum(0))])
    ids = rng.permutation(n).astype(np.uint32)
    return x4, u4, ids


def _cells(x4, N):
    c = np.floor(x4[:3]).astype(np.int64)
    return (c[2] * N + c[1]) * N + c[0]


def _regular_path(x4, u4, ids, N):
    from paper_0904_0232_gb300.grpic import Simulation

    sim = Simulation(N, N, N, 0.0, 0.0, 1.0, 0.4, precision="fp64")
    sim.load_particles(0, 0.0, 0.0, x4, u4, ids)
    out = sim.get_particles(0)
    sim.close()
    return out


def _static_path(torch, x4, u4, ids, N):
    from paper_0904_0232_gb300.grpic import grpic_sort_particles_static

    dev = torch.device("cuda")
    xt = torch.from_numpy(x4).to(dev)
    ut = torch.from_numpy(u4).to(dev)
    it = torch.from_numpy(ids.view(np.int32)).to(dev)
    xo = torch.empty_like(xt)
    uo = torch.empty_like(ut)
    io = torch.empty_like(it)
    no = torch.zeros(1, dtype=torch.int64, device=dev)
    grpic_sort_particles_static(N, N, N, xt, ut, it, xo, uo, io, no)
    torch.cuda.synchronize()
    k = int(no.item())
    return xo.cpu().numpy()[:, :k], uo.cpu().numpy()[:, :k], io.cpu().numpy().view(np.uint32)[:k]


def _same(a, b, N):
    xa, ua, ia = a
    xb, ub, ib = b
    assert ia.size == ib.size
    # identical cell sequence (order within a cell is unspecified)
    ca, cb = _cells(xa, N), _cells(xb, N)
    assert np.all(np.diff(cb) >= 0)
    assert np.array_equal(ca, cb)
    oa, ob = np.argsort(ia), np.argsort(ib)
    assert np.array_equal(ia[oa], ib[ob])
    assert np.array_equal(xa[:, oa], xb[:, ob]) and np.array_equal(ua[:, oa], ub[:, ob])


def test_static_sort_matches_regular_path_twice(torch):
    N = 40
    for seed, n in ((1, 50000), (2, 33333)):
        x4, u4, ids = _particles(seed, n, N)
        _same(_regular_path(x4, u4, ids, N), _static_path(torch, x4, u4, ids, N), N)


def test_static_sort_drops_particles_outside_the_grid(torch):
    """Positions outside [0, N-1) on any axis -- negative, beyond the last cell, NaN -- go to the
    outside bin and are not returned; the kept count is the offset of that bin.  The kept particles
    come back in cell order, each with its own values, twice in a row."""
    N = 32
    rng = np.random.default_rng(7)
    for n in (20000, 12345):
        x4, u4, ids = _particles(int(rng.integers(100)), n, N)
        bad = rng.random(n) < 0.3
        ax = rng.integers(0, 3, n)
        kind = rng.integers(0, 4, n)
        for i in np.nonzero(bad)[0]:
            x4[ax[i], i] = (-rng.uniform(0.0, 5.0), -1e-300, N - 1 + rng.uniform(0.0, 3.0), np.nan)[kind[i]]
        keep = np.all((x4[:3] >= 0.0) & (x4[:3] < N - 1), axis=0)
        assert 0.2 < 1 - keep.mean() < 0.4
        xo, uo, io = _static_path(torch, x4, u4, ids, N)
        assert io.size == keep.sum()
        c = _cells(xo, N)
        assert np.all(np.diff(c) >= 0)
        assert np.array_equal(np.sort(c), np.sort(_cells(x4[:, keep], N)))
        pos = {int(v): k for k, v in enumerate(ids)}
        src = np.array([pos[int(v)] for v in io])
        assert np.array_equal(np.sort(io), np.sort(ids[keep]))
        assert np.array_equal(xo, x4[:, src]) and np.array_equal(uo, u4[:, src])


def test_static_sort_of_no_particles(torch):
    """n = 0: nothing is read or written but the count, which is 0 (after a call that kept many)."""
    from paper_0904_0232_gb300.grpic import grpic_sort_particles_static

    N = 16
    x4, u4, ids = _particles(4, 3000, N)
    assert _static_path(torch, x4, u4, ids, N)[2].size == 3000
    e = torch.zeros((4, 0), dtype=torch.float64, device="cuda")
    i = torch.zeros(0, dtype=torch.int32, device="cuda")
    no = torch.full((1,), 12345, dtype=torch.int64, device="cuda")
    grpic_sort_particles_static(N, N, N, e, e, i, e.clone(), e.clone(), i.clone(), no)
    torch.cuda.synchronize()
    assert int(no.item()) == 0


def test_static_sort_rejects_too_large_grid(torch):
    from paper_0904_0232_gb300.grpic import GrpicError, grpic_sort_particles_static

    t = torch.zeros((4, 1), dtype=torch.float64, device="cuda")
    i = torch.zeros(1, dtype=torch.int32, device="cuda")
    no = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(GrpicError) as ei:
        grpic_sort_particles_static(65, 64, 64, t, t, i, t.clone(), t.clone(), i.clone(), no)
    assert ei.value.code == 8
