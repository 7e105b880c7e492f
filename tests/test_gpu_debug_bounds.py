"""The bounds-checking build (libapiccontact_debug.so, -DAPIC_DEBUG_BOUNDS):
on the device every tile-node, page-table, item-size, cell-bit,
permutation and sort-output index of the kernels is checked before use; a
failed check records a bit and skips the access.  Across the entry points
and scene kinds below no check may fire, and the results still match the
oracle.  It runs in a child process so that the environment switch that
selects the debug library does not touch this session's library."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
import torch
sys.path.insert(0, ROOT)
from paper_2108_02259_gb300 import apic, build, scenes
import oracle
assert apic.LIB_PATH.endswith("libapiccontact_debug.so")
build.build(debug=True)
assert apic.load().apic_debug_build() == 1
dev = torch.device("cuda:0")
def t(a, d):
    return torch.as_tensor(np.ascontiguousarray(a), device=dev, dtype=d)
def dev_args(s, dt=np.float32):
    f = s.astype(dt)
    td = torch.float32 if dt == np.float32 else torch.float64
    return t(f.x, torch.float64), t(f.v, td), t(f.C, td), t(f.m, td), t(f.nrm, td), t(f.body, torch.int32)
out = {}
rng = np.random.default_rng(5)
cases = [("two cubes", scenes.two_cubes(mu=0.3, n_iter=4), None),
         ("four bodies small", scenes.four_bodies(scale=0.05), None),
         ("32-body cloud, negative coordinates", scenes.random_cloud(3000, n_bodies=32, seed=3, h=0.1, n_iter=1,
                                                                    origin=(10.0, -20.0, 5.0), spread=1.3), None),
         ("dense 4-body cloud, per-pair mu", scenes.random_cloud(20000, n_bodies=4, seed=9, h=0.05, n_iter=3),
          np.full((4, 4), 0.3) + 0.1 * np.eye(4))]
apic.debug_flags(clear=True)
with apic.Context(0) as ctx:
    for label, s, mp in cases:
        for variant in (0, 1, 5, 7):
            ctx.set_variant(variant)
            X, V, Cc, M, NR, B = dev_args(s)
            r = apic.contact_step(ctx, X, V, Cc, M, NR, B, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies, mu_pair=mp)
            torch.cuda.synchronize()
            out[f"{label}, variant {variant}"] = apic.debug_flags(clear=True)
        rv, rC, _ = oracle.contact_step(s.x, s.v, s.C, s.m, s.nrm, s.body, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies,
                                        mu_pair=mp)
        out[f"{label}, v err"] = float(np.abs(r.v.cpu().double().numpy() - rv).max() / np.abs(s.v).max())
    ctx.set_variant(-1)
    s = cases[1][1]
    X, V, Cc, M, NR, B = dev_args(s, np.float64)
    apic.contact_step(ctx, X, V, Cc, M, NR, B, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies)
    torch.cuda.synchronize()
    out["fp64"] = apic.debug_flags(clear=True)
    X, V, Cc, M, NR, B = dev_args(s)
    apic.contact_step(ctx, X, V, Cc, M, NR, B, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies,
                      flags=apic.APIC_DETERMINISTIC)
    apic.contact_step(ctx, X, V, Cc, M, None, B, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies)
    torch.cuda.synchronize()
    out["deterministic and mass normals"] = apic.debug_flags(clear=True)
    sc = scenes.batch_of_scenes(12, seed=4)
    bs = [apic.BatchScene(*dev_args(x), x.h, x.mu, n_bodies=x.n_bodies) for x in sc]
    apic.contact_step_batched(ctx, bs, sc[0].n_iter)
    torch.cuda.synchronize()
    out["batch of 12 scenes"] = apic.debug_flags(clear=True)
    big = scenes.four_bodies()
    X, V, Cc, M, NR, B = dev_args(big)
    for _ in range(3):  # the page-table box reused across steps
        apic.contact_step(ctx, X, V, Cc, M, NR, B, big.h, big.mu, big.n_iter, n_bodies=big.n_bodies)
    torch.cuda.synchronize()
    out["200k nodes, three steps"] = apic.debug_flags(clear=True)
s = cases[0][1]
X, V, Cc, M, NR, B = dev_args(s)
apic.contact_step_static(X, V, Cc, M, NR, B, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies)
torch.cuda.synchronize()
out["no-allocation entry point"] = apic.debug_flags(clear=True)
print("RESULT " + json.dumps(out))
"""


@pytest.mark.gpu
def test_no_bounds_check_fires():
    env = dict(os.environ, APIC_DEBUG_BOUNDS="1")
    r = subprocess.run([sys.executable, "-c", f"ROOT = {ROOT!r}\n" + CHILD], env=env, capture_output=True,
                       text=True, timeout=1200, cwd=ROOT)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    line = [x for x in r.stdout.splitlines() if x.startswith("RESULT ")][-1]
    res = json.loads(line[len("RESULT "):])
    for k, v in res.items():
        if k.endswith("v err"):
            assert v <= 1e-5, (k, v)
        else:
            assert v == 0, (k, v)


def test_normal_build_has_no_checks():
    """The library the rest of the suite uses is the normal build (its
    kernels carry no checks) and reports no bits."""
    from paper_2108_02259_gb300 import apic, build

    build.build()
    lib = apic.load()
    assert lib.apic_debug_build() == 0
