"""The checked build (DOPE_CHECKED): every shared-memory index of the block
solver and the resident kernel is tested against its array, and an index
outside it is recorded instead of touching memory.  Solves on every kernel
family run with the checks on: no index may fall outside its array, and the
results must equal the ordinary library's bit for bit.  The checked library is
loaded in a child process (the binding picks it with DOPE_LIBRARY=checked)."""
import hashlib
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, instance factory, extra context arguments)
CASES = '''
from paper_1704_03116_gb300 import inputs
CASES = [
    ("resident_windows_8conn", lambda: inputs.ellipses_rgb(size=256, lam=4.0), {}),
    ("resident_4conn_mode2", lambda: inputs.random_instance((96, 96), 4, (16, 16), lam=2.0, seed=1),
     {"launch_mode": 2}),
    ("persistent_worklists_3d", lambda: inputs.ellipsoids3d(shape=(32, 64, 64)), {"threads": 512}),
    ("persistent_worklists_8conn", lambda: inputs.random_instance((128, 96), 8, (16, 32), lam=3.0, seed=2),
     {"threads": 256, "mu0": 2.0}),
    ("mode1", lambda: inputs.random_instance((64, 64), 8, (16, 16), lam=3.0, seed=3), {"launch_mode": 1}),
    ("overlap_grow2", lambda: inputs.random_instance((64, 64), 8, (16, 16), lam=2.0, seed=4),
     {"grow": (2, 2), "max_iter": 6}),
    ("kernel5x5", lambda: inputs.ellipses_rgb(size=128, lam=1.0, conn=24, block=(32, 32)), {}),
    ("nonsubmodular", lambda: inputs.nonsubmodular_instance(size=64), {"lsa_steps": 16}),
]
'''

CHILD = CASES + '''
import hashlib, json, sys
import numpy as np
from paper_1704_03116_gb300 import dope
out = {}
for name, make, kw in CASES:
    d = make()
    kw = dict(kw)
    kw.setdefault("mu0", d["mu0"])
    g = dope.Dope(d["grid"], d["conn"], d["block"], d["lam"], **kw)
    g.set_unaries(d["u"])
    g.set_weights(d["wq"])
    lab, E, it = g.solve(allow_notconv=True)
    out[name] = [hashlib.sha256(lab.tobytes()).hexdigest(), E, it]
# the batched launch on three of them
gs = [dope.Dope.from_instance(make()) for name, make, kw in CASES[:3]]
res = dope.iterate_batch(gs, 1000)
out["batch"] = [[hashlib.sha256(g.labels()[0].tobytes()).hexdigest(), int(g.labels()[1]), r[0]] for g, r in zip(gs, res)]
try:
    out["check"] = dope.dope_check_status(clear=True)
except dope.DopeError as e:
    out["check"] = "unsupported" if e.status == dope.DOPE_EUNSUPPORTED else "error %d" % e.status
print(json.dumps(out))
'''


def _run(env_lib):
    env = dict(os.environ)
    if env_lib:
        env["DOPE_LIBRARY"] = env_lib
    else:
        env.pop("DOPE_LIBRARY", None)
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_checked_build_finds_no_bad_index_and_changes_nothing():
    from paper_1704_03116_gb300 import _build
    _build.build()
    _build.build(checked=True)
    ref = _run(None)
    got = _run("checked")
    assert ref["check"] == "unsupported"          # the ordinary library has no checks
    assert got["check"] is None, f"shared-memory index outside its array: (length, index) = {got['check']}"
    for key in ref:
        if key != "check":
            assert got[key] == ref[key], key
