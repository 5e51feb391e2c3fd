"""The seeded input recipes hold the shapes and ranges they state (no GPU):
the many-channel set, the served-case stream and the cavity placement."""
import math

import numpy as np

from paper_2410_23802_gb300 import workloads as W


def _no_overlap(case, gap=2.0):
    x, y, r = np.array(case.x), np.array(case.y), np.array(case.radius)
    for i in range(len(x)):
        d = np.hypot(x[i + 1:] - x[i], y[i + 1:] - y[i])
        assert (d >= r[i + 1:] + r[i] + gap - 1e-9).all()


def test_channels_recipe():
    cases = W.channels()
    assert len(cases) == 256
    assert [c.params["nx"] for c in W.channels()] == [c.params["nx"] for c in cases]  # seeded
    for c in cases:
        w = c.params["nx"]
        D = 2 * c.radius[0]
        assert 64 <= w <= 256 and c.params["ny"] == 4 * w
        assert 0.1 * w <= D <= 0.25 * w
        assert c.x == [w / 2.0] and c.y == [3.0 * w]
        assert 1.1 <= c.params["rho_ratio"] <= 2.0 and 0.1 <= c.params["k_ratio_default"] <= 10.0
        assert c.params["cv_ratio"] == 1.5 and c.params["thermal_wall"] == (0, 0, 0, 0)
    widths = np.array([c.params["nx"] for c in cases])
    assert widths.min() < 80 and widths.max() > 240  # the whole range is drawn


def test_served_stream_recipe():
    items = W.served_cases(n=60)
    gaps = np.array([g for g, _, _ in items])
    assert (gaps > 0).all() and 0.5 < gaps.mean() < 2.0  # exponential, mean 1
    precisions = [c.params["precision"] for _, c, _ in items]
    assert set(precisions) == {"fp32", "fp16"}
    for _, c, steps in items:
        side = c.params["nx"]
        n = len(c.x)
        D = 2 * c.radius[0]
        assert steps == 2000 and c.params["ny"] == side
        assert 64 <= side <= 1024 and 1 <= n <= 512 and 8.0 <= D <= 24.0
        assert n == 1 or n * math.pi * D * D / 4 <= 0.3 * 0.6 * side * side
        assert min(c.y) - c.radius[0] >= 0.4 * side  # upper 60 %
        _no_overlap(c)


def test_cavity_placement_recipe():
    c = W.cavity(side=512, n=128)
    r = c.radius[0]
    assert all(r + 2 <= x <= 512 - r - 2 for x in c.x)
    assert all(0.4 * 512 + r + 2 <= y <= 512 - r - 2 for y in c.y)
    _no_overlap(c)
