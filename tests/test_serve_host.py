"""Host-side request generation of the serving driver (no GPU): the request specs are drawn
within the stated ranges and repeat for a seed, and the absorbing layers a client asks for
scale with the box."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
from paper_0904_0232_gb300 import serve  # noqa: E402


def test_sample_requests_within_ranges_and_seeded():
    full = serve.MIXES["full"]
    a = serve.sample_requests(200, 5, **full)
    b = serve.sample_requests(200, 5, **full)
    assert a == b and a != serve.sample_requests(200, 6, **full)
    for k, r in enumerate(a):
        assert r["n"] in full["grids"]
        assert full["ppc"][0] <= r["ppc"] <= full["ppc"][1]
        assert full["steps"][0] <= r["nsteps"] <= full["steps"][1]
        assert 1.0 <= r["m"] <= 4.0 and 0.0 <= r["a"] <= 0.99 * r["m"]
        assert r["seed"] == 1000 + k
    # every grid of the mix is drawn at this sample size
    assert {r["n"] for r in a} == set(full["grids"])


def test_layers_for_scale_with_the_box():
    for n, w in ((16, 4), (32, 4), (48, 6), (64, 8), (128, 8), (384, 8)):
        lay = serve.layers_for(n)
        assert lay == {"absorb_inner": 0.3, "absorb_outer": 0.2, "absorb_width": w}, (n, lay)
