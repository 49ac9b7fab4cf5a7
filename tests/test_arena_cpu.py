"""The serving form's admission arena (csrc/arena.h, host code): a random
script of allocations and releases against a brute-force model that keeps a
byte map of the range and takes the lowest-addressed run of free bytes that
fits.  Checks offsets, failures, usage and peak, and that released blocks
coalesce (the free list always equals the maximal free runs of the byte map)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2509_21963_gb300", "csrc")


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("arena") / "arena_harness")
    subprocess.run([cxx, "-std=c++17", "-O1", f"-I{CSRC}", "-o", exe,
                    os.path.join(ROOT, "tests", "arena_harness.cpp")], check=True)
    return exe


class Model:
    """Byte map of the range in 256-byte units; first fit over free runs."""

    def __init__(self, cap):
        self.units = cap // 256
        self.busy = np.zeros(self.units, dtype=bool)
        self.used = self.peak = 0

    def runs(self):
        out, i = [], 0
        while i < self.units:
            if self.busy[i]:
                i += 1
                continue
            j = i
            while j < self.units and not self.busy[j]:
                j += 1
            out.append((i * 256, (j - i) * 256))
            i = j
        return out

    def alloc(self, nbytes):
        need = max(1, -(-max(nbytes, 1) // 256))
        for off, size in self.runs():
            if size >= need * 256:
                u = off // 256
                self.busy[u:u + need] = True
                self.used += need * 256
                self.peak = max(self.peak, self.used)
                return off
        return None

    def release(self, off, nbytes):
        need = max(1, -(-max(nbytes, 1) // 256))
        assert self.busy[off // 256:off // 256 + need].all()
        self.busy[off // 256:off // 256 + need] = False
        self.used -= need * 256


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_arena_matches_first_fit_model(harness, seed):
    rng = np.random.default_rng(seed)
    cap = 256 * 4096
    model = Model(cap)
    script, expect, live, next_id = [f"I {cap}"], [], {}, 0
    for step in range(3000):
        if live and (rng.random() < 0.45 or len(live) > 60):
            tid = int(rng.choice(list(live)))
            off, nbytes = live.pop(tid)
            script.append(f"R {tid}")
            model.release(off, nbytes)
        else:
            nbytes = int(rng.choice([0, 1, 255, 256, 257]) if rng.random() < 0.2
                         else rng.integers(1, 60000))
            off = model.alloc(nbytes)
            script.append(f"A {next_id} {nbytes}")
            expect.append(f"A {next_id} {off if off is not None else 'fail'}")
            if off is not None:
                live[next_id] = (off, nbytes)
            next_id += 1
        if step % 250 == 0:
            script.append("S")
            runs = model.runs()
            expect.append(f"S {model.used} {model.peak} {len(runs)}")
            expect.extend(f"F {o} {s}" for o, s in runs)
    for tid, (off, nbytes) in list(live.items()):  # everything back: one free block
        script.append(f"R {tid}")
        model.release(off, nbytes)
    script.append("S")
    expect.append(f"S 0 {model.peak} 1")
    expect.append(f"F 0 {cap}")
    p = subprocess.run([harness], input="\n".join(script) + "\n", capture_output=True,
                       text=True, check=True)
    assert p.stdout.split("\n")[:-1] == expect
