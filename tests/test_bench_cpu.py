"""Host arithmetic of bench.py's roofline object (CPU, no GPU).

* The counter records are tied to the kernel sources by a hash of the code
  without comments, so a comment edit keeps a record current and a code edit
  makes it stale (string literals, which hold inline PTX, count as code).
* `achieved` = the busier integer pipe's busy cycles x 16 lanes per site x sites
  per launch / launch time (or, for records without pipe cycles, the executed
  ALU-pipe operations), against 64 lanes per clock per SM x 152 SMs x the SM clock;
  `traffic` is the record's DRAM bytes per site x sites, and null once the record is
  stale.
"""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_code_only_drops_comments_and_keeps_strings():
    a = 'int x = 1; // one\n/* block\n comment */ asm("add.u32 %0, %1; // kept");\n'
    b = 'int   x = 1;\n asm("add.u32 %0, %1; // kept");'
    assert bench.code_only(a) == bench.code_only(b)
    assert "// kept" in bench.code_only(a)
    assert bench.code_only(a) != bench.code_only(a.replace("x = 1", "x = 2"))
    assert bench.code_only(a) != bench.code_only(a.replace("add.u32", "sub.u32"))


@pytest.mark.parametrize("kernel", sorted(bench.KERNEL_SOURCES))
def test_every_counter_record_names_its_capture(kernel):
    with open(os.path.join(ROOT, "profiles", f"{kernel}_counters.json")) as f:
        d = json.load(f)
    assert d["kernel"] == kernel
    assert "--clock-control none" in d["command"]
    assert len(d["kernel_source_hash"]) == 16
    c = bench.committed_counters(kernel)
    assert c is not None and c["alu_ops_per_site"] > 0 and c["inst_slots_per_site"] >= c["alu_ops_per_site"]


def fake_counters(current):
    return {"current": current, "inst_slots_per_site": 6.0, "alu_ops_per_site": 3.5, "pipe_cycles_per_site": None,
            "dram_bytes_per_site": 0.4, "capture": "ncu ..."}


def test_roofline_arithmetic(monkeypatch):
    monkeypatch.setattr(bench, "committed_counters", lambda k: fake_counters(True))
    sites, t, mhz = 2.0 ** 31, 6.0e-4, 2070.0
    r = bench.kernel_roofline("packed_half_sweep", sites, t, mhz, {"hbm_gbs": 6778.7})
    peak = 64 * 152 * mhz * 1e6 / 1e12
    assert r["bound"] == "alu" and r["unit"] == "Tops/s"
    assert r["peak"] == pytest.approx(peak) and r["peak"] == pytest.approx(20.137, abs=1e-3)
    assert r["achieved"] == pytest.approx(3.5 * sites / t / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / peak)
    assert r["traffic"] == pytest.approx(0.4 * sites)
    assert r["counters"] == "current"
    assert r["issue_view"]["peak"] == pytest.approx(2 * peak)
    assert r["issue_view"]["achieved"] == pytest.approx(6.0 * sites / t / 1e12)
    # the HBM view: 0.375 algorithmic bytes per updated site of a half-sweep (= per site and sweep)
    assert r["hbm_achieved_gbs"] == pytest.approx(0.375 * sites / t / 1e9)
    assert r["hbm_peak_gbs"] == 6778.7


def test_roofline_binds_on_the_busier_pipe(monkeypatch):
    """With pipe cycles in the record, the pipe with more busy cycles per site binds:
    achieved = 16 lanes x busy cycles x sites / time."""
    def counters(pipes):
        return lambda k: {**fake_counters(True), "pipe_cycles_per_site": pipes}

    sites, t, mhz = 2.0 ** 31, 5.0e-4, 2070.0
    peak = 64 * 152 * mhz * 1e6 / 1e12
    monkeypatch.setattr(bench, "committed_counters", counters({"alu": 0.16, "fmaheavy": 0.19}))
    r = bench.kernel_roofline("packed_half_sweep", sites, t, mhz, {})
    assert r["pipe"].startswith("FMA-heavy")
    assert r["achieved"] == pytest.approx(16 * 0.19 * sites / t / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / peak)
    assert r["pipe_views"][bench.PIPE_NAMES["alu"]]["frac"] == pytest.approx(16 * 0.16 * sites / t / 1e12 / peak)
    monkeypatch.setattr(bench, "committed_counters", counters({"alu": 0.21, "fmaheavy": 0.12}))
    r = bench.kernel_roofline("packed_half_sweep", sites, t, mhz, {})
    assert r["pipe"].startswith("ALU") and r["achieved"] == pytest.approx(16 * 0.21 * sites / t / 1e12)


def test_stale_counters_null_the_traffic(monkeypatch):
    monkeypatch.setattr(bench, "committed_counters", lambda k: fake_counters(False))
    r = bench.kernel_roofline("packed_half_sweep", 1e6, 1e-5, 2070.0, {})
    assert r["traffic"] is None and r["counters"].startswith("stale")
    monkeypatch.setattr(bench, "committed_counters", lambda k: None)
    r = bench.kernel_roofline("packed_half_sweep", 1e6, 1e-5, 2070.0, {})
    assert r["achieved"] is None and r["frac"] is None and r["traffic"] is None


def profile_commands():
    """Command lines in profiles/*.md (backslash continuations joined)."""
    out = []
    pdir = os.path.join(ROOT, "profiles")
    for name in sorted(os.listdir(pdir)):
        if not name.endswith(".md"):
            continue
        text = open(os.path.join(pdir, name)).read().replace("\\\n", " ")
        for line in text.splitlines():
            line = line.split("#")[0].strip().strip("`")
            if line.startswith(("ncu ", "python bench.py")):
                out.append((name, line))
    return out


def test_profile_commands_still_run_as_written():
    """Each summary's commands run committed files only: bench.py with options it
    still accepts, and every ncu with --clock-control none."""
    cmds = profile_commands()
    assert {n for n, _ in cmds} == {f for f in os.listdir(os.path.join(ROOT, "profiles")) if f.endswith(".md")}
    for name, line in cmds:
        assert "_work" not in line, (name, line)
        if line.startswith("ncu "):
            assert "--clock-control none" in line, (name, line)
            assert "python bench.py" in line, (name, line)
        argv = line.split("python bench.py", 1)[1].split()
        bench.make_parser().parse_args(argv)


def test_expected_calls_per_word_matches_a_simulation():
    """E[calls] of the counted model against a direct simulation of the bit-plane
    comparison: n sites with random 32-bit U and a fixed T, read four planes per call
    from the top; a word draws call k iff some site is undecided after 4k planes."""
    import numpy as np

    rng = np.random.default_rng(7)
    T = 0x2BEC3A1F
    for n in (0, 1, 3, 16, 32):
        words = 20000
        calls = np.zeros(words)
        if n:
            U = rng.integers(0, 2 ** 32, size=(words, n), dtype=np.uint64)
            # planes read by each site: the position (from the top) of the first bit
            # where U and T differ, plus one
            diff = U ^ np.uint64(T)
            planes = 32 - np.floor(np.log2(diff.astype(np.float64))).astype(int)
            calls = np.ceil(planes.max(axis=1) / 4.0)
        assert np.mean(calls) == pytest.approx(float(bench.expected_calls_per_word(n)), abs=0.02), n
    assert float(bench.expected_calls_per_word(0)) == 0.0
    assert float(bench.expected_calls_per_word(1)) == pytest.approx(sum(2.0 ** (-4 * k) for k in range(8)))


def test_tested_sites_per_word_by_brute_force():
    """Per-word tested-site counts against a site-by-site loop over the plane layout."""
    import numpy as np

    rng = np.random.default_rng(3)
    L, R, first = 128, 5, 7
    rows = rng.choice(np.array([-1, 1], dtype=np.int8), size=(R + 2, L))
    got = bench.tested_sites_per_word(rows, True, False, first_row=first)
    want = []
    for i in range(R):
        gi = first + i
        for colour in (0, 1):
            for w in range(L // 64):
                cnt = 0
                for b in range(32):
                    j = 2 * (32 * w + b) + ((gi + colour) & 1)
                    s = rows[i + 1, j]
                    n = sum(int(x != s) for x in (rows[i, j], rows[i + 2, j], rows[i + 1, (j - 1) % L],
                                                   rows[i + 1, (j + 1) % L]))
                    cnt += n == 1
                want.append(cnt)
    assert list(got) == want
    both = bench.tested_sites_per_word(rows, True, True, first_row=first)
    assert np.all(both >= got) and both.sum() > got.sum()


def test_algorithmic_view_arithmetic():
    """All sites tested with one threshold: E = expected_calls_per_word(32); the views are
    E products x 2 lane-cycles / 32 (FMA-heavy) and (34 E + 15) / 32 (ALU) per site."""
    import numpy as np

    rows = np.ones((4, 128), dtype=np.int8)  # all aligned: every site has n = 0
    v = bench.algorithmic_view(rows, 2 ** 32, 5 << 28, 1e12, 2070.0)
    E = float(bench.expected_calls_per_word(32))
    assert v["calls_per_word"] == pytest.approx(E) and v["tested_sites_per_word"] == 32
    peak = 64 * 152 * 2070.0 * 1e6 / 1e12
    alu = (34 * E + 15) / 32
    assert v["views"][bench.PIPE_NAMES["alu"]]["frac"] == pytest.approx(alu * 1e12 / 1e12 / peak)
    assert v["views"][bench.PIPE_NAMES["fmaheavy"]]["lane_cycles_per_site"] == pytest.approx(E)
    assert v["frac"] == pytest.approx(max(alu, E) / peak)
    # a threshold of 2^32 (accept all) or 0 tests nothing
    assert bench.algorithmic_view(rows, 2 ** 32, 2 ** 32, 1e12, 2070.0)["calls_per_word"] == 0.0


def test_full_size_traffic_is_preferred():
    """A record with a one-pass full-size DRAM capture reports that capture's bytes per
    site (the cube's re-reads, if any, depend on its size)."""
    with open(os.path.join(ROOT, "profiles", "cubic_half_sweep_counters.json")) as f:
        d = json.load(f)
    fs = d["full_size"]
    c = bench.committed_counters("cubic_half_sweep")
    want = (fs["dram_bytes_read_per_launch"] + fs["dram_bytes_write_per_launch"]) / fs["sites_per_launch"]
    assert c["dram_bytes_per_site"] == pytest.approx(want)
    assert "--clock-control none" in fs["command"]
    # at most the algorithmic bytes plus 5 %: each plane read once, the target written once
    assert fs["dram_bytes_read_per_launch"] + fs["dram_bytes_write_per_launch"] <= 1.05 * fs["algorithmic_bytes_per_launch"]


def test_saturated_capacity_counts_the_work_of_unfinished_requests():
    """Requests all admitted at t = 0 advance in lockstep: at the time the half-way
    request finishes, each unfinished one has done as many sweeps as the longest
    finished one.  Three requests of 100, 200, 400 sweeps (L = 64, 128, 256) and one of
    800 (L = 64): after two finish (at t = 2.0 s, the 200-sweep one), the others have
    done 200 sweeps each."""
    from types import SimpleNamespace as R
    res = [R(L=256, sweeps=400, finished=4.0), R(L=64, sweeps=100, finished=1.0),
           R(L=64, sweeps=800, finished=8.0), R(L=128, sweeps=200, finished=2.0)]
    work = 64 * 64 * 100 + 128 * 128 * 200 + 256 * 256 * 200 + 64 * 64 * 200
    assert bench.saturated_capacity(res) == pytest.approx(work / 2.0, rel=1e-15)
    # a request shorter than the finished ones' longest (collected later) counts whole
    res.append(R(L=64, sweeps=150, finished=2.5))
    work5 = 64 * 64 * 100 + 64 * 64 * 150 + 128 * 128 * 200 + 256 * 256 * 200 + 64 * 64 * 200
    assert bench.saturated_capacity(res) == pytest.approx(work5 / 2.0, rel=1e-15)
