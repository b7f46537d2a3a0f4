"""The bounds-checked build (libmdp_checked.so, MDP_CHECKED=1): every batched kernel validates
its block's work item (subdomain, columns, workspace slices, tables, pivot flags, output range)
and the gamma indices it writes through, records the first violation as MDP_ERR_BOUNDS and skips
the access. Run in a child process that loads the checked library: small parity cases against
the oracle (forward and adjoint, both AP types), the same batch under two tile shapes (races),
and host-side fault injection -- a corrupted tile descriptor must be caught by the checks without
a GPU fault, a corrupted factor entry by the parity check."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import os, sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
import workloads as W
from oracle.projection import APSystem
import paper_2103_12172_gb300 as mdp
from paper_2103_12172_gb300 import _lib, MdpError
assert _lib.LIB_PATH.endswith("libmdp_checked.so"), _lib.LIB_PATH

def err(a, b):
    return float((np.abs(a - b).max(axis=1) / np.abs(b).max(axis=1)).max())

def plan_of(subs, tile=0):
    return mdp.Plan(subs, tile_cols=tile)

# parity: forward (Q and P) and adjoint, n = 17, 33, 65, both AP types
for n in (17, 33, 65):
    for ap in (W.AP_DIRICHLET4, W.AP_DIRX_SOMMY):
        sub = W.small_subdomain(n, 6.0 + n / 16.0, ap, 2)
        plan = plan_of([sub])
        G, nc, _, _ = plan.layout(0)
        S = APSystem(sub)
        for kind in ("Q", "P"):
            got = plan.project(kind=kind).cpu().numpy().reshape(nc, G)
            assert err(got, S.columns(kind=kind)) < 1e-10, (n, ap, kind)
        cot = W.random_complex((nc, G), seed=n + ap)
        gx, gk = plan.adjoint(torch.from_numpy(cot.ravel()).cuda())
        rx, rk = S.adjoint(cot, kind="Q")
        assert err(gx.cpu().numpy().reshape(nc, G), rx) < 1e-10, (n, ap)
        assert abs(gk.item() - rk) < 1e-9 * abs(rk), (n, ap)
        plan.status()
        plan.close()
# the same batch under two tile shapes (several items, several waves): equal to rounding
subs = [W.unit_subdomain(i, 0, 65, 7.0 + i, W.AP_DIRX_SOMMY, 3) for i in range(3)]
a = plan_of(subs, 8).project().cpu().numpy()
b = plan_of(subs, 0).project().cpu().numpy()
assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()
# a corrupted tile descriptor: caught by the checks, every access through it skipped
sub = W.small_subdomain(65, 9.0, W.AP_DIRX_SOMMY, 2)
os.environ["MDP_FAULT_INJECT"] = "desc"
bad = plan_of([sub])
del os.environ["MDP_FAULT_INJECT"]
bad.project()
torch.cuda.synchronize()
try:
    bad.status()
    raise SystemExit("corrupted descriptor not reported")
except MdpError as e:
    assert e.code == _lib.MDP_ERR_BOUNDS, e.code
bad.close()
# the context is intact: a clean plan still matches the oracle
G, nc, _, _ = plan_of([sub]).layout(0)
ok = plan_of([sub]).project().cpu().numpy().reshape(nc, G)
assert err(ok, APSystem(sub).columns()) < 1e-10
# a corrupted factor entry: no bounds violation, the parity check catches the wrong numbers
os.environ["MDP_FAULT_INJECT"] = "factor"
wrong = plan_of([sub])
del os.environ["MDP_FAULT_INJECT"]
got = wrong.project().cpu().numpy().reshape(nc, G)
wrong.status()
assert err(got, APSystem(sub).columns()) > 1e-6
print("checked build ok")
'''


def test_checked_library_builds_and_exports_the_same_symbols():
    """The bounds-checked twin compiles for sm_103a and exports every symbol of libmdp.so."""
    from paper_2103_12172_gb300 import _build
    lib = _build.build(checked=True)
    base = _build.build()

    def exported(path):
        out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
        return {line.split()[-1] for line in out.splitlines() if " T mdp_" in line}

    assert exported(lib) == exported(base) and "mdp_project_batch" in exported(lib)


@pytest.mark.gpu
def test_checked_build_parity_races_and_fault_injection():
    from paper_2103_12172_gb300 import _build
    _build.build(checked=True)
    env = dict(os.environ, MDP_LIB_CHECKED="1")
    env.pop("MDP_FAULT_INJECT", None)
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "checked build ok" in r.stdout
