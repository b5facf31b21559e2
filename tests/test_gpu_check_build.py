"""GPU tests of the checked build (include/kpm.h, KPM_CHECK): the library
compiled with bounds checks in the staged sweep, loaded in a child process
with KPM_CHECK=1.

On valid inputs the checks change nothing: the moments of both forms and
of a batched ensemble must equal the normal build's bit for bit, with the
device error word clear.  A chunk record corrupted through the checked
build's test hook (an inline run whose rows end past the vector block, a
staged length past the stage, an overflow offset past the overflow array)
must stop the launch before any copy, with kpm_check_device_error
reporting the range error (KPM_EINVAL), and leave the context usable once
the record is restored."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from kpm_inputs import hamiltonians as ham

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json
import numpy as np
from paper_1410_5242_gb300 import kpm
from kpm_inputs import hamiltonians as ham

assert kpm.CHECKED and kpm.lib.kpm_checked_build() == 1
out = {}
h = ham.ti_hamiltonian(16, 16, 12, gamma=1.0, seed=4)
a, b = kpm.scale_from_bounds(*kpm.gershgorin(h), 0.01)
for name, prec in (("fp32", kpm.PREC_FP32), ("fp64", kpm.PREC_FP64)):
    with kpm.create(h, a, b, precision=prec) as ctx:
        assert ctx.get_launch(32)["stages"] >= 1
        out[name] = ctx.moments(40, 32, 3).tolist()
        ctx.check_device_error()
g = ham.ti_hamiltonian(9, 7, 6, gamma=2.0, seed=3)
ctxs = []
for m in (h, g):
    a2, b2 = kpm.scale_from_bounds(*kpm.gershgorin(m), 0.01)
    ctxs.append(kpm.create(m, a2, b2, precision=kpm.PREC_FP32))
out["batch"] = [e.tolist() for e in kpm.moments_batch(ctxs, [24, 16], [16, 32], [5, 6])]
for c in ctxs:
    c.close()
# corrupted records, through the test hook: (word, x, y) of chunk 5's record
def status(f):
    try:
        f()
        return "no error"
    except kpm.KPMError as e:
        return e.status


out["corrupt"] = {}
C = 32
with kpm.create(h, a, b, precision=kpm.PREC_FP32) as ctx:
    rows = ctx.info()["n_pad"]
    ref = ctx.moments(8, 32, 3)
    # inline run 0 (the chunk's own rows) moved to end 24 rows past the block
    ctx.test_corrupt_record(5, 3, rows - 8, 32)
    out["corrupt"]["run_past_block"] = status(lambda: ctx.moments(8, 32, 3))
    ctx.test_corrupt_record(5, 3, 5 * C, C)  # restored
    out["restored_equal"] = bool(np.array_equal(ctx.moments(8, 32, 3), ref))
for name, words in (("length_past_stage", [(1, 4000, 1)]),
                    ("overflow_offset", [(1, 13 | (6 << 16), 40), (2, 1 << 30, 0)])):
    with kpm.create(h, a, b, precision=kpm.PREC_FP32) as ctx:
        for w, x, y in words:
            ctx.test_corrupt_record(5, w, x, y)
        out["corrupt"][name] = status(lambda: ctx.moments(8, 32, 3))
print(json.dumps(out))
'''


@pytest.fixture(scope="module")
def kpm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1410_5242_gb300 import build
    build.build()
    build.build(check=True)
    from paper_1410_5242_gb300 import kpm as k
    return k


def run_child():
    env = dict(os.environ, KPM_CHECK="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_checked_build_matches_normal_build(kpm):
    """Both forms and a batch: the checked build's moments equal the normal
    build's bit for bit, and the checked build's hook is refused by the
    normal build."""
    got = run_child()
    h = ham.ti_hamiltonian(16, 16, 12, gamma=1.0, seed=4)
    a, b = kpm.scale_from_bounds(*kpm.gershgorin(h), 0.01)
    for name, prec in (("fp32", kpm.PREC_FP32), ("fp64", kpm.PREC_FP64)):
        with kpm.create(h, a, b, precision=prec) as ctx:
            ref = ctx.moments(40, 32, 3)
        np.testing.assert_array_equal(np.array(got[name]), ref)
    g = ham.ti_hamiltonian(9, 7, 6, gamma=2.0, seed=3)
    ctxs = []
    for m in (h, g):
        a2, b2 = kpm.scale_from_bounds(*kpm.gershgorin(m), 0.01)
        ctxs.append(kpm.create(m, a2, b2, precision=kpm.PREC_FP32))
    ref = kpm.moments_batch(ctxs, [24, 16], [16, 32], [5, 6])
    for c in ctxs:
        c.close()
    for x, y in zip(got["batch"], ref):
        np.testing.assert_array_equal(np.array(x), y)
    assert kpm.lib.kpm_checked_build() == 0
    with kpm.create(h, a, b, precision=kpm.PREC_FP32) as ctx:
        with pytest.raises(kpm.KPMError) as e:
            ctx.test_corrupt_record(5, 3, 0, 1)
        assert e.value.status == kpm.KPM_EUNSUPPORTED
    # corrupted records stop the launch with a range error
    assert got["corrupt"] == {"run_past_block": kpm.KPM_EINVAL,
                              "length_past_stage": kpm.KPM_EINVAL,
                              "overflow_offset": kpm.KPM_EINVAL}, got["corrupt"]
    assert got["restored_equal"]
