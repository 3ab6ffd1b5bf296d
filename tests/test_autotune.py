"""The autotuner's search and cache, on a fake context whose step time is a known function of
the launch-shape choices (no GPU)."""
from paper_0904_0232_gb300 import autotune
from paper_0904_0232_gb300.grpic import GrpicError


class FakeSim:
    def __init__(self, cost):
        self.cost = cost
        self.t = dict(far_min_blocks=5, near_blocks_per_sm=2, sort_interval=1, overlap=1, split=0, j_tile=0, spread=0,
                      area_table=0)
        self.calls = 0
        self.refused = 0

    def tuning(self):
        return dict(self.t)

    def set_tuning(self, far_min_blocks, near_blocks_per_sm, sort_interval, overlap, split, j_tile, spread,
                   area_table=0):
        # like the library: the area fits and the J tile exclude each other
        if j_tile and area_table:
            self.refused += 1
            raise GrpicError(1, "grpic_set_tuning", "tuning out of range")  # GRPIC_ERR_INVALID
        self.t = dict(far_min_blocks=far_min_blocks, near_blocks_per_sm=near_blocks_per_sm,
                      sort_interval=sort_interval, overlap=overlap, split=split, j_tile=j_tile, spread=spread,
                      area_table=area_table)


def timer(sim, steps):
    sim.calls += 1
    return sim.cost(**sim.t)


def separable(far_min_blocks, near_blocks_per_sm, sort_interval, overlap, split, j_tile, spread=0, area_table=0):
    return ({4: 3.0, 5: 1.0, 6: 2.0}[far_min_blocks] + {1: 0.5, 2: 0.7, 4: 0.2}[near_blocks_per_sm]
            + {1: 0.9, 2: 0.3, 4: 0.4}[sort_interval] + {0: 0.05, 1: 0.0}[overlap] + {0: 0.1, 1: 0.0}[split]
            + {0: 0.0, 1: 0.02}[j_tile] + {0: 0.03, 1: 0.0}[area_table])


def test_coordinate_descent_finds_separable_minimum(tmp_path):
    sim = FakeSim(separable)
    r = autotune.tune(sim, "w", cache=str(tmp_path / "t.json"), timer=timer, device="fake")
    assert r["tuning"] == dict(far_min_blocks=5, near_blocks_per_sm=4, sort_interval=2, overlap=1, split=1, j_tile=0,
                               spread=0, area_table=1)
    assert sim.t == r["tuning"] and not r["cached"]
    assert abs(r["ms_per_step"] - separable(**r["tuning"])) < 1e-12


def test_coupled_cost_second_round(tmp_path):
    # the best near setting depends on the far setting: one round is not enough
    def coupled(far_min_blocks, near_blocks_per_sm, sort_interval, overlap, split, j_tile, spread=0, area_table=0):
        table = {(4, 1): 1.0, (4, 2): 5.0, (4, 4): 5.0, (5, 1): 5.0, (5, 2): 3.0, (5, 4): 5.0,
                 (6, 1): 5.0, (6, 2): 5.0, (6, 4): 0.5}
        return table[(far_min_blocks, near_blocks_per_sm)] + 0.1 * sort_interval + 0.01 * overlap
    sim = FakeSim(coupled)
    r = autotune.tune(sim, "c", cache=str(tmp_path / "t.json"), timer=timer, device="fake", rounds=3)
    best = min(coupled(f, n, 1, 0, 0, 0) for f in (4, 5, 6) for n in (1, 2, 4))
    assert r["ms_per_step"] <= coupled(5, 2, 1, 1, 0, 0)  # never worse than the start
    assert r["tuning"]["sort_interval"] == 1
    assert r["ms_per_step"] >= best


def test_drift_of_the_step_time_cancels(tmp_path):
    """The state evolves while tuning (each trial advances it) and the step time grows with it:
    timing every value forward and backward cancels a linear drift that would otherwise favour
    the values tried first."""
    def cost(far_min_blocks, near_blocks_per_sm, sort_interval, overlap, split, j_tile, spread=0, area_table=0):
        return {1: 1.0, 2: 0.96, 4: 0.92}[sort_interval] + 0.01 * far_min_blocks

    class Drifting(FakeSim):
        def __init__(self):
            super().__init__(cost)

    def drift_timer(sim, steps):
        sim.calls += 1
        return sim.cost(**sim.t) + 0.05 * sim.calls

    sim = Drifting()
    r = autotune.tune(sim, "d", cache=str(tmp_path / "t.json"), timer=drift_timer, device="fake",
                      choices={"sort_interval": (1, 2, 4)}, rounds=1)
    assert r["tuning"]["sort_interval"] == 4


def test_cache_reused(tmp_path):
    cache = str(tmp_path / "t.json")
    sim = FakeSim(separable)
    autotune.tune(sim, "w", cache=cache, timer=timer, device="fake")
    sim2 = FakeSim(separable)
    r = autotune.tune(sim2, "w", cache=cache, timer=timer, device="fake")
    assert r["cached"] and sim2.calls == 0 and sim2.t == r["tuning"]
    # another device or workload signature does not hit
    assert autotune.cached("w", cache, device="other") is None
    assert autotune.cached("x", cache, device="fake") is None


def test_batch_tuning(tmp_path):
    chosen = []
    times = {4: 9.0, 8: 6.0, 16: 7.0}
    r = autotune.tune_batch(lambda k: times[chosen[-1]] * k, chosen.append, "b",
                            cache=str(tmp_path / "t.json"), device="fake")
    assert r["tuning"] == {"batch_blocks_per_sm": 8} and chosen[-1] == 8


def test_refused_combination_is_skipped(tmp_path):
    """A combination the context refuses (here the J tile with the area fits) is timed with the
    conflicting knob back at its first choice: the J tile, chosen first, gives way to the fits
    it excludes, which are cheaper."""
    def cost(far_min_blocks, near_blocks_per_sm, sort_interval, overlap, split, j_tile, spread=0, area_table=0):
        return 1.0 - 0.1 * j_tile - 0.3 * area_table
    sim = FakeSim(cost)
    r = autotune.tune(sim, "r", cache=str(tmp_path / "t.json"), timer=timer, device="fake",
                      choices={"j_tile": (0, 1), "area_table": (0, 1)}, rounds=2)
    assert r["tuning"]["area_table"] == 1 and r["tuning"]["j_tile"] == 0
    assert sim.refused > 0 and abs(r["ms_per_step"] - 0.7) < 1e-12
