"""The batch arena's offset bookkeeping (csrc/arena.h) against a plain model (CPU).

A batch admits lattices against one HBM region; its FreeList places each block
first-fit in 256-byte granules and merges free neighbours on release.  The model
here keeps only the live blocks: free space is their complement (so it is merged
by construction), and first fit is the lowest gap that holds the rounded size.  A
release that failed to merge shows up as a different offset or a spurious "full"
at a later allocation, and in the free list the dumps compare.
"""
import os
import random
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GRANULE = 256


@pytest.fixture(scope="module")
def arena_bin(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    exe = str(tmp_path_factory.mktemp("arena") / "arena_check")
    subprocess.run([gxx, "-std=c++17", "-O1", "-Wall", "-I", os.path.join(ROOT, "paper_1903_11714_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "arena_check.cpp"), "-o", exe], check=True)
    return exe


def up(n):
    return -(-n // GRANULE) * GRANULE


class Model:
    def __init__(self, size):
        self.size = up(size)
        self.live = {}  # offset -> rounded length

    def gaps(self):
        out, pos = [], 0
        for off in sorted(self.live):
            if off > pos:
                out.append((pos, off - pos))
            pos = off + self.live[off]
        if pos < self.size:
            out.append((pos, self.size - pos))
        return out

    def alloc(self, n):
        need = up(n)
        for off, length in self.gaps():
            if length >= need:
                self.live[off] = need
                return off
        return -1

    def free(self, off):
        del self.live[off]

    def dump(self):
        used = sum(self.live.values())
        return " ".join([str(used)] + [f"{o}:{n}" for o, n in self.gaps()])


def run_script(exe, lines):
    r = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    return r.stdout.split("\n")[:len(lines)]


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_free_list_matches_the_model(arena_bin, seed):
    rng = random.Random(seed)
    size = rng.choice([1 << 20, (1 << 20) + 100, 3 << 18])
    m = Model(size)
    script, want = [f"reset {size}"], ["ok"]
    sizes = {}
    for step in range(3000):
        if m.live and (rng.random() < 0.45 or not m.gaps()):
            off = rng.choice(sorted(m.live))
            script.append(f"free {off} {sizes.pop(off)}")
            want.append("ok")
            m.free(off)
        else:
            # lattice-like blocks: planes of 64..2048-sided lattices plus a history,
            # and odd sizes that are not whole granules
            n = rng.choice([64, 128, 256, 512, 1024, 2048]) ** 2 // 8 + 16 * rng.randrange(1, 600)
            if rng.random() < 0.2:
                n = rng.randrange(1, 5000)
            off = m.alloc(n)
            script.append(f"alloc {n}")
            want.append(str(off))
            if off >= 0:
                sizes[off] = n
        if step % 97 == 0:
            script.append("dump")
            want.append(m.dump())
    for off in sorted(m.live):  # return everything: one block spanning the region
        script.append(f"free {off} {sizes[off]}")
        want.append("ok")
        m.free(off)
    script.append("dump")
    want.append(f"0 0:{up(size)}")
    got = run_script(arena_bin, script)
    for k, (g, w) in enumerate(zip(got, want)):
        assert g == w, (k, script[k], g, w)
    assert len(got) == len(want)


def test_whole_region_and_exact_fits(arena_bin):
    lines = ["reset 1000", "alloc 1024", "alloc 1", "dump", "free 0 1024", "alloc 300", "alloc 300",
             "alloc 300", "dump", "free 512 300", "alloc 257", "alloc 256", "free 0 300", "dump", "alloc 512", "dump"]
    got = run_script(arena_bin, lines)
    assert got == ["ok", "0", "-1", "1024",          # 1000 rounds up to 1024: one block takes it all
                   "ok", "0", "512", "-1", "1024",   # 512-byte blocks; the third does not fit
                   "ok", "512", "-1", "ok",           # 257 takes the freed 512 gap; nothing left for 256
                   "512 0:512",                       # freeing 0 leaves one gap at the bottom
                   "0", "1024"]                       # which a 512-byte block fills exactly
