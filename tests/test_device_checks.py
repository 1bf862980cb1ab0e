"""The build with device-side checks (GFP_DEVICE_CHECKS): kernels that meet
input outside their contract record it in an error word instead of faulting,
and gfp_context_check reports it as GFP_ERR_INVALID.  The inputs used here
stay inside every buffer (the kernels skip a column >= k and read no pairs
for a decreasing row_ptr), so the release build runs them harmlessly too."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
import numpy as np, torch
sys.path.insert(0, {root!r})
from paper_cs_0404008_gb300 import gfpdot as g
assert g.lib_path().endswith("debug/libgfpdot.so"), g.lib_path()
g.load()
ctx = g.Context(0)
p, m, k, nb = 65521, 6, 40, 8
dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.uint32).view(np.int32)).cuda()
B = dev(np.arange(k * nb, dtype=np.uint32).reshape(k, nb) % p)
C = torch.zeros((m, nb), dtype=torch.int32, device="cuda")
rp = np.array([0, 2, 4, 6, 8, 10, 12], np.uint32)
col = np.array([0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11], np.uint32)
val = np.ones(12, np.uint32)
out = []
g.gfp_matmul_block_csr(ctx, p, k, dev(rp), dev(col), dev(val), B, C)
out.append(g.gfp_context_check(ctx))          # clean input
bad = col.copy(); bad[5] = k + 3              # a column outside the matrix
g.gfp_matmul_block_csr(ctx, p, k, dev(rp), dev(bad), dev(val), B, C)
out.append(g.gfp_context_check(ctx))
out.append(g.gfp_context_check(ctx))          # the check cleared the record
rp2 = rp.copy(); rp2[3] = 1                   # row_ptr decreases (rows 2 and 3)
g.gfp_matmul_block_csr(ctx, p, k, dev(rp2), dev(col), dev(val), B, C)
out.append(g.gfp_context_check(ctx))
x = dev(np.ones(64, np.uint32))
o = torch.zeros(4, dtype=torch.int32, device="cuda")
g.gfp_dot_batched(ctx, [(p, x, x, 64), (p, x, x, 17)], o)
out.append(g.gfp_context_check(ctx))          # clean batched dot
print("RESULT", out)
"""


def test_debug_build_exports_the_same_abi():
    from paper_cs_0404008_gb300 import build
    rel, dbg = build.build(), build.build(debug=True)
    syms = []
    for path in (rel, dbg):
        out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True,
                             text=True).stdout
        syms.append(sorted(l.split()[-1] for l in out.splitlines()
                           if " T " in l and l.split()[-1].startswith("gfp_")))
    assert syms[0] == syms[1] and len(syms[0]) > 40


@pytest.mark.gpu
def test_device_checks_report_contract_violations():
    env = dict(os.environ, GFPDOT_DEBUG="1")
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT)], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, (r.stdout + r.stderr)[-3000:]
    line = [l for l in r.stdout.splitlines() if l.startswith("RESULT")][-1]
    ok, invalid = 0, -1
    assert line == f"RESULT {[ok, invalid, ok, invalid, ok]}", line
