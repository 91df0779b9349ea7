"""The host C code (the oracle and the corpus generator) under AddressSanitizer
and UndefinedBehaviorSanitizer (no GPU).

Both libraries are rebuilt with -fsanitize=address,undefined into a scratch
directory; a child Python process (libasan preloaded) points the loaders at
them, runs the oracle and generator pins, then the oracle's functions on a
full-size 2 MiB workload and the generator on every workload's law. Any
out-of-bounds access, use after free or undefined behaviour aborts the child.
"""
import os
import shutil
import subprocess
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
FLAGS = ["-O1", "-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined", "-fno-sanitize-recover=undefined",
         "-std=c11", "-Wall", "-shared", "-fPIC"]

CHILD = r'''
import sys
from pathlib import Path


def main():
    root, ora, syn = sys.argv[1], Path(sys.argv[2]), Path(sys.argv[3])
    sys.path.insert(0, root)
    import numpy as np
    import pytest
    from oracle import oracle as O
    O.LIB = ora
    from paper_2511_14955_gb300 import _build, synth
    _build.build_synth = lambda force=False: syn
    # the multi-process harness runs the same C calls in worker processes
    # that load the library by its default path: it is left out here
    rc = pytest.main(["-q", "-x", "-p", "no:cacheprovider", "-m", "not gpu and not slow", "-k", "not sharded",
                      f"{root}/tests/test_oracle.py", f"{root}/tests/test_synth.py"])
    if rc:
        sys.exit(int(rc))
    data, off, _ = synth.make_corpus("markov_2mb", seed=1)
    ik, ic = O.intergrams(data, off, 4, 1024, 4096, base_n=1)
    ek, ec = O.exhaustive(data, off, 4, 1 << 22, count_mode=O.EQ1_EVERY_OCCURRENCE)
    rp, cols = O.features(data, off, ik)
    pk, pc = O.count_pass(data, off, 4, None, count_mode=O.EQ1_EVERY_OCCURRENCE)
    assert len(ic) == 1024 and int(ec.sum()) == int(np.maximum(np.diff(off.astype(np.int64)) - 3, 0).sum())
    assert int(pc.sum()) == int(ec.sum())
    for name in synth.WORKLOADS:
        synth.make_corpus(name, seed=2, m=3, max_len=1 << 16)
    maps = open("/proc/self/maps").read()
    assert str(ora) in maps and str(syn) in maps, "the sanitized libraries were not the ones loaded"
    print("sanitized run clean")


if __name__ == "__main__":
    main()
'''


def test_host_c_clean_under_asan_and_ubsan(tmp_path):
    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("gcc not available")
    asan = subprocess.run([gcc, "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    if not asan or not os.path.isabs(asan) or not os.path.exists(asan):
        pytest.skip("libasan not available")
    ora, syn = tmp_path / "liboracle.so", tmp_path / "libsynth.so"
    for out, srcs, libs in ((ora, [ROOT / "oracle" / "intergrams_oracle.c"], []),
                            (syn, [ROOT / "paper_2511_14955_gb300" / "csrc" / "synth.c"], ["-lm", "-lpthread"])):
        r = subprocess.run([gcc, *FLAGS, "-o", str(out), *map(str, srcs), *libs], capture_output=True, text=True)
        if r.returncode != 0:
            pytest.skip("sanitizer build unavailable: " + r.stderr[-300:])
    child = tmp_path / "child.py"
    child.write_text(CHILD)
    env = dict(os.environ, LD_PRELOAD=asan, ASAN_OPTIONS="detect_leaks=0:abort_on_error=0",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    r = subprocess.run([sys.executable, str(child), str(ROOT), str(ora), str(syn)], cwd=str(tmp_path), env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and "sanitized run clean" in r.stdout, (r.stdout[-3000:], r.stderr[-3000:])
