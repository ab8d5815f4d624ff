"""Memory-safety substitute for a sanitizer (compute-sanitizer is closed on
this pool): the library built with -DISING_CHECKED range-checks every
lattice-word index of every kernel family and records an out-of-range one
instead of accessing it.  The small-lattice battery (every L class, every
execution path, batch, server, both layouts and both chains) runs against
that build in a child process, matches the oracle, and leaves no record."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_small_lattice_battery_under_the_checked_build():
    from paper_1811_04384_gb300 import build
    lib = build.build(checked=True)
    env = dict(os.environ, ISING_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "helpers", "checked_battery.py")],
                       capture_output=True, text=True, env=env, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["ok"] and out["checked"] and out["violation"] == 0
    assert out["cases"] >= 30
