"""A program that leaves its handles to the garbage collector exits cleanly.

The child process below creates a context, keys, a batch and a gallery,
searches, and exits without closing anything; the binding closes the live
handles at interpreter exit (newest first).  The child must exit with
status 0 after printing its marker.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
sys.path.insert(0, {root!r})
import numpy as np, torch
import paper_2003_12197_gb300 as H
import workloads as W
dev = torch.device("cuda", 0)
H.build_library()
ctx = H.Context(0)
keys = H.hers_keygen(ctx, 5)
m, d = 5000, 16
nb = H.hers_blocks_for(m)
feats = torch.from_numpy(W.gallery_features(m, d, 6)).to(dev)
gal, _ = H.hers_encrypt_gallery(ctx, keys, feats, 7)
pct = H.hers_encrypt_probe(ctx, keys, feats[3].clone(), 8)
pr = H.hers_probe_prepare(ctx, pct)
sc = H.hers_search(ctx, keys, gal, nb, d, pr)
batch = H.Batch(ctx, keys, [(gal, nb, d, pr)])
batch.run()
scores = H.hers_decrypt_scores(ctx, keys, sc, m).cpu().numpy()
assert int(np.argmax(scores)) == 3
H.hers_check(ctx)
print("searched", flush=True)
"""


def test_exit_without_closing_handles():
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT)], capture_output=True, text=True,
                       timeout=600)
    assert "searched" in r.stdout, r.stdout + r.stderr
    assert r.returncode == 0, f"exit status {r.returncode}: {r.stderr[-2000:]}"
