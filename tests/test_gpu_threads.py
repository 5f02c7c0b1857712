"""Contexts created and used from several host threads at once (the C ABI's
rule is one context per host thread): the one-time per-device set-up of
kernel attributes and persistent grid sizes runs under a lock.  Run in a
fresh process so that the set-up really happens while the threads race."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys, threading
import numpy as np
sys.path.insert(0, sys.argv[1]); sys.path.insert(0, sys.argv[1] + '/tests')
import torch
import oracle
from gpu_util import oracle_fixed, to_dev
from paper_1910_09020_gb300 import binding, synth

n, m, E = 4000, 100, 6
reads, refs = synth.pairs_fixed(91, 0, n, m, synth.SHORT_POISSON)
want_acc, want_obs = oracle_fixed(reads, refs, E)
torch.zeros(1, device='cuda')  # the CUDA context, before the race
T = 4
start = threading.Barrier(T)
out = [None] * T
errors = []

def work(i):
    try:
        start.wait()
        F = binding.Filter(0)  # ss_create: the one-time set-up
        try:
            q = F.pack(to_dev(reads.reshape(-1)), m=m, n=n)
            r = F.pack(to_dev(refs.reshape(-1)), m=m, n=n)
            got = []
            for flags in (binding.SS_MODE_PLAIN, binding.SS_MODE_BUCKETED):
                acc, obs = F.filter(q, r, m=m, e=E, n=n, flags=flags)
                F.sync()
                got.append((acc.cpu().numpy(), obs.cpu().numpy()))
            out[i] = got
        finally:
            F.close()
    except Exception as e:  # reported by the parent
        errors.append(repr(e))

ts = [threading.Thread(target=work, args=(i,)) for i in range(T)]
for t in ts:
    t.start()
for t in ts:
    t.join()
assert not errors, errors
for i in range(T):
    for acc, obs in out[i]:
        assert (acc == want_acc).all() and (obs == want_obs).all(), i
print("ok")
"""


def test_contexts_from_several_host_threads():
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), (
        r.stdout[-2000:] + r.stderr[-4000:])
