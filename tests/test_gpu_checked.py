"""GPU runs of the bounds-checked build (the stand-in for memory sanitizers,
which this GPU pool does not offer).

The library is rebuilt with -DHOTRG_CHECKED=1: every mapped access of the
FP64 GEMMs, the operand gathers, the tensor-core epilogues and the fused
projection kernel's output stores is compared with
the capacity of its buffer, and an access outside it is skipped and reported as
HOTRG_EBOUNDS instead of being performed.  The checked library runs, in a child
process (a process loads one build), the step paths of every precision mode on
single contexts and on a batch of two concurrent cut groups; each must finish
without a bounds report and still match the FP64 oracle.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys
sys.path.insert(0, %(root)r)
import numpy as np
import paper_2602_05900_gb300 as pkg
from oracle import hotrg as ref
lib = pkg.load()
assert lib._name.endswith("libhotrg_checked.so"), lib._name
cases = [("fp64", 8, 10, 1e-12), ("tf32", 16, 8, 2e-4), ("bf16x3", 12, 8, 5e-5), ("bf16xs", 12, 8, 1e-10)]
for prec, D_cut, nsteps, tol in cases:
    want = ref.run(ref.ising_initial_tensor(0.44, 0.01), D_cut, nsteps).ln_z_per_site
    with pkg.Hotrg(pkg.ising_tensor(0.44, 0.01), D_cut, prec) as h:
        got = h.run(nsteps).ln_z_per_site()
    err = abs(got / want - 1)
    print(prec, D_cut, err)
    assert err < tol, (prec, err)
T0s = [pkg.ising_tensor(0.42), pkg.ising_tensor(0.46), pkg.ising_tensor(0.44)]
with pkg.HotrgBatch(T0s, [8, 12, 8], "fp64") as bt:
    lz = bt.run(8).ln_z_per_site()
for T0, D, v in zip([0.42, 0.46, 0.44], [8, 12, 8], lz):
    want = ref.run(ref.ising_initial_tensor(T0), D, 8).ln_z_per_site
    assert abs(v / want - 1) < 1e-12, (T0, D, v, want)
# TF32 batch with the fused projection kernel on (the D_cut = 16 group runs it)
from paper_2602_05900_gb300.capi import OPT_FUSED_CHAIN
with pkg.HotrgBatch(T0s, [16, 12, 16], "tf32") as bt:
    bt.set_option(OPT_FUSED_CHAIN, 1)
    lz = bt.run(8).ln_z_per_site()
for T0, D, v in zip([0.42, 0.46, 0.44], [16, 12, 16], lz):
    want = ref.run(ref.ising_initial_tensor(T0), D, 8).ln_z_per_site
    assert abs(v / want - 1) < 5e-4, (T0, D, v, want)     # TF32 whole-job bound (beta = 0.44 is near critical)
print("CHECKED_OK")
"""


@pytest.fixture(scope="module")
def checked_lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_05900_gb300 import build
    return build.build(checked=True)


def test_checked_build_runs_every_path_without_bounds_reports(checked_lib):
    env = dict(os.environ, HOTRG_LIB=checked_lib)
    r = subprocess.run([sys.executable, "-c", SCRIPT % {"root": ROOT}], env=env, capture_output=True,
                       text=True, timeout=900, cwd=ROOT)
    print(r.stdout[-3000:], r.stderr[-3000:])
    assert r.returncode == 0, r.stderr[-3000:]
    assert "CHECKED_OK" in r.stdout
