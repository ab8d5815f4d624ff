"""The serving configuration's request stream (host logic, CPU)."""
import math

import numpy as np

from paper_1811_04384_gb300.serving import poisson_stream


def test_poisson_stream_recipe():
    s = poisson_stream(4000, rate=200.0, seed=13)
    t = np.array([x[0] for x in s])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert (gaps > 0).all()
    assert abs(gaps.mean() - 1 / 200) < 4 * (1 / 200) / math.sqrt(len(gaps))
    Ls = {x[1] for x in s}
    assert Ls == {64, 128, 256, 512, 1024, 2048, 4096}
    Ts = np.array([1 / x[2] for x in s])
    assert Ts.min() >= 1.5 and Ts.max() <= 3.5
    sw = np.array([x[4] for x in s])
    assert sw.min() >= 100 and sw.max() <= 10000
    # log-uniform: the median is near sqrt(100 * 10000) = 1000
    assert 850 < np.median(sw) < 1150
    assert poisson_stream(10, seed=13) == poisson_stream(10, seed=13)
