"""The autotuner's choice outlives the process: a second process with the
same cache file gets the same knobs without timing any candidate (best_ms is
0), and a job in another corpus-size bucket is tuned afresh."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, sys
sys.path.insert(0, sys.argv[1])
import numpy as np, torch
from paper_2511_14955_gb300 import binding as B, synth
data, off, _ = synth.make_corpus("markov_2mb", m=int(sys.argv[2]))
d = torch.from_numpy(data).cuda()
o = torch.from_numpy(off.view(np.int64)).cuda()
t, ms = B.autotune(d, o, n=5, k=512, candidates=2048, base_n=2)
print(json.dumps({"tuning": t, "best_ms": ms}))
'''


def child(cache, m):
    env = dict(os.environ, INTERGRAMS_TUNE_CACHE=str(cache))
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, str(m)], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_second_process_takes_the_cached_choice(tmp_path):
    cache = tmp_path / "sub" / "autotune.txt"
    first = child(cache, 40)
    assert first["best_ms"] > 0 and cache.exists()
    assert len(cache.read_text().splitlines()) == 1
    second = child(cache, 40)
    assert second["best_ms"] == 0 and second["tuning"] == first["tuning"]
    assert len(cache.read_text().splitlines()) == 1
    other = child(cache, 4)  # a smaller corpus: another size bucket
    assert other["best_ms"] > 0
    assert len(cache.read_text().splitlines()) == 2


def test_unreadable_lines_are_ignored(tmp_path):
    cache = tmp_path / "autotune.txt"
    cache.write_text("garbage\nNVIDIA 1 2 3\n")
    out = child(cache, 40)
    assert out["best_ms"] > 0
    assert len(cache.read_text().splitlines()) == 3
