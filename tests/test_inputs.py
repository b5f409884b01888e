"""The seeded synthetic input generators (CPU): shapes, orderings and ranges
of the workloads the benchmark and the studies use."""
import numpy as np

from paper_2109_00661_gb300 import inputs as I


def test_random_models_ranges_and_seeding():
    m = I.random_models(4096, seed=3)
    assert m["nlayers"].min() >= 1 and m["nlayers"].max() <= 10
    L = m["nlayers"]
    used = np.arange(10)[None, :] < L[:, None]
    assert np.all((m["logsig"][used] >= -4.0) & (m["logsig"][used] <= 0.0))
    assert np.all((m["logh"][used] >= np.log10(2.0)) & (m["logh"][used] <= np.log10(200.0)))
    assert np.all((m["m"][used] >= 0.0) & (m["m"][used] < 1.0))
    assert np.all((m["logtau"][used] >= -6.0) & (m["logtau"][used] <= -1.0))
    assert np.all((m["c"][used] >= 0.1) & (m["c"][used] <= 1.0))
    again = I.random_models(4096, seed=3)
    assert all(np.array_equal(m[k], again[k]) for k in m)
    assert not np.array_equal(m["logsig"], I.random_models(4096, seed=4)["logsig"])


def test_detectability_grid_layout():
    depths, ms = (10.0, 40.0, 80.0), (0.0, 0.25, 0.5, 0.8)
    g = I.detectability_grid(depths, ms, 0.032)
    assert g["nlayers"].shape == (12,) and np.all(g["nlayers"] == 3)
    # depth-major: sounding d * len(ms) + j has depth depths[d] and m = ms[j]
    for d, z in enumerate(depths):
        for j, mv in enumerate(ms):
            s = d * len(ms) + j
            assert np.isclose(10 ** g["logh"][s, 0], z) and np.isclose(10 ** g["logh"][s, 1], 20.0)
            assert g["m"][s, 1] == mv and g["m"][s, 0] == 0.0 and g["m"][s, 2] == 0.0
            assert np.allclose(10 ** g["logsig"][s], [0.01, 0.1, 0.032])
    assert np.allclose(10 ** g["logtau"], 4.07e-4) and np.all(g["c"] == 1.0)


def test_flight_line_section():
    truth, x = I.flight_line(101)
    depth = 10 ** truth["logh"][:, 0]
    m = truth["m"][:, 1]
    assert np.isclose(x[0], 0.0) and np.isclose(x[-1], 1.0)
    assert np.isclose(depth.min(), 20.0) and np.isclose(depth.max(), 80.0)
    assert np.isclose(m.min(), 0.0) and np.isclose(m.max(), 0.5)
    assert np.argmax(m) == 50 and np.argmax(depth) == 50  # the most chargeable, and deepest, at the centre
