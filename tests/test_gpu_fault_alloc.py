"""Host-side fault injection (SKEI_FAULT_ALLOC=n fails the library's n-th
device allocation in the process): every failing allocation is reported as
SKEI_ENOMEM by the call that needed it, nothing of that call is left
allocated, and the same process then creates plans and batches and runs
operators normally.  No GPU fault is involved: the allocation is refused on
the host before it reaches the driver."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys, torch
sys.path.insert(0, sys.argv[2])
from paper_2411_05771_gb300 import skei as S
k = int(sys.argv[1])
def attempt(make):
    try:
        return "ok", make()
    except RuntimeError as e:
        return ("enomem" if "(-2)" in str(e) else "other: " + str(e)), None
# a plan makes 3 device allocations (angle table, status word, filter spectrum)
first, plan = attempt(lambda: S.Plan(64, 60))
if plan is None:
    plan = S.Plan(64, 60)
x = torch.rand((1, 64, 64), device="cuda")
out = torch.empty((1, 60, plan.n_det), device="cuda")
# a batch then makes its own 3 (item table, work queue, task list)
second, batch = attempt(lambda: S.Batch(S.PROJ_FWD, [S.BatchItem(plan, x, out)]))
if batch is None:
    batch = S.Batch(S.PROJ_FWD, [S.BatchItem(plan, x, out)])
batch.run()
y = S.proj_fwd(plan, x)
torch.cuda.synchronize()
print(first, second, bool(torch.equal(out, y)), plan.status())
"""


@pytest.mark.parametrize("k,first,second", [
    (1, "enomem", "ok"), (2, "enomem", "ok"), (3, "enomem", "ok"),
    (4, "ok", "enomem"), (5, "ok", "enomem"), (6, "ok", "enomem"),
    (0, "ok", "ok"),          # no injection
])
def test_failed_allocation_is_reported_and_recovered(k, first, second):
    env = dict(os.environ, SKEI_FAULT_ALLOC=str(k))
    r = subprocess.run([sys.executable, "-c", CHILD, str(k), ROOT], env=env,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    got = r.stdout.split()[-4:]
    assert got == [first, second, "True", "0"], r.stdout
