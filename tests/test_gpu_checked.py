"""The checked build (libdsr_check.so: device-side bounds and handle checks
that record the first failure and skip the access, short retry caps) runs
the applications (game of life, wa-tor, batched wa-tor, traffic,
sugarscape) to the same results with no failed check. Each case runs
in a child process, because a process loads one of the two libraries."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys
sys.path.insert(0, {root!r})
sys.path.insert(0, {tests!r})
import numpy as np, torch
import oracle as O
from paper_1809_07444_gb300 import _lib as L
assert L.LIB_PATH.endswith("libdsr_check.so"), L.LIB_PATH
from paper_1809_07444_gb300 import workloads as WL
from paper_1809_07444_gb300.apps import Gol, Wator, WatorBatch, Traffic, Sugarscape
from helpers import check_invariants

g, gr = Gol(64, 64, WL.gol_initial(64, 64, 1)), O.Gol(64, 64, WL.gol_initial(64, 64, 1))
for _ in range(20):
    g.step(1); gr.step(1)
    assert g.hash() == gr.hash()
k0 = WL.wator_initial(96, 96, 2)
w, wr = Wator(96, 96, k0, 2), O.Wator(96, 96, k0, seed=2)
for _ in range(40):
    w.step(1); wr.step(1)
    assert w.hash() == wr.hash()
b = WatorBatch(64 << 20, max_instances=8)
refs = []
for i, s in enumerate([20, 33, 64]):
    kk = WL.wator_initial(s, s, 40 + i)
    refs.append((b.add(s, s, kk, 40 + i), O.Wator(s, s, kk, seed=40 + i)))
for _ in range(20):
    b.step(1)
    for slot, r in refs:
        r.step(1)
        assert b.hash(slot) == r.hash()
v0 = WL.traffic_initial(37, 211, 3, 0.3)
t, tr = Traffic(37, 211, v0, 5), O.Traffic(37, 211, v0, 5)
for _ in range(30):
    t.step(1); tr.step(1)
    assert t.hash() == tr.hash()
cap, ag = WL.sugarscape_initial(37, 29, 3, 0.3)
sg, sr = Sugarscape(37, 29, cap, ag, 7), O.Sugarscape(37, 29, cap, ag, 7)
for _ in range(30):
    sg.step(1); sr.step(1)
    assert sg.hash() == sr.hash()
for hp in (g.heap, w.heap, t.heap, sg.heap):
    st = hp.stats()
    assert st["error_flags"] == 0, st
    check_invariants(hp)
print("checked ok")
"""


def test_checked_build_runs_clean():
    env = dict(os.environ, DSR_LIBRARY="check")
    code = SCRIPT.format(root=ROOT, tests=os.path.join(ROOT, "tests"))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "checked ok" in r.stdout
