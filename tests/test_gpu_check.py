"""pm_surface_check and the bounds-checked build (-DPM_BOUNDS_CHECK).

* Every kind of built surface passes the device consistency check: quadrilateral
  patches before and after their coefficient, a clone, triangle patches, and a
  c != 0 surface.
* The checked library (libparametrix_checked.so, selected with PM_LIBRARY in a
  child process) runs the check before and a finite scan after every apply and
  returns exactly the normal library's results in every precision.
"""

import json
import os
import subprocess
import sys

import numpy as np
import pytest

from workloads import make_workload

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2401_12501_gb300 as pm
    c = pm.Context(0)
    yield c
    c.close()


def test_surfaces_pass_the_consistency_check(ctx):
    import paper_2401_12501_gb300 as pm
    from workloads import ellipsoid_coefficient
    from workloads.trisurfaces import tri_ellipsoid
    wl = make_workload("ellipsoid_small")
    s = pm.Surface.from_fixture(ctx, wl.surface)
    s.check()                                            # geometry and weights only
    s.set_coeff(wl.coeff.a, wl.coeff.grad_a)
    s.apply_R(np.ones(wl.N), "ff")
    s.check()
    c = s.clone()
    c.set_coeff(2.0 * wl.coeff.a, 2.0 * wl.coeff.grad_a)
    c.check()
    c.set_coeff_c(wl.coeff.a, wl.coeff.grad_a, -3.0 - wl.surface.nodes[:, 0])
    c.check()                                            # complex corrections included
    t = tri_ellipsoid(0, 5)
    ts = pm.Surface.from_fixture(ctx, t)
    co = ellipsoid_coefficient(t)
    ts.set_coeff(co.a, co.grad_a)
    ts.check()
    for x in (s, c, ts):
        x.close()


_CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, {root!r})
import paper_2401_12501_gb300 as pm
from workloads import make_workload
wl = make_workload("ellipsoid_small")
ctx = pm.Context(0)
s = pm.Surface.from_fixture(ctx, wl.surface)
s.set_coeff(wl.coeff.a, wl.coeff.grad_a)
sig = np.random.default_rng(5).standard_normal(wl.N) + 1.0
out = {{}}
for prec in ("fp64", "fp32", "ff"):
    out["R_" + prec] = s.apply_R(sig, prec).tolist()
    out["K_" + prec] = s.apply_K(sig, prec).tolist()
print(json.dumps(out))
"""


def _run(env_lib):
    env = dict(os.environ)
    if env_lib:
        env["PM_LIBRARY"] = env_lib
    r = subprocess.run([sys.executable, "-c", _CHILD.format(root=ROOT)], capture_output=True,
                       text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_checked_build_gives_the_same_results():
    from paper_2401_12501_gb300 import build
    checked = build.build(checked=True)
    plain = _run(None)
    chk = _run(checked)
    for k in plain:
        assert np.array_equal(np.array(plain[k]), np.array(chk[k])), k
