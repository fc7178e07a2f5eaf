"""bench.py's reference arm runs on the host alone (the oracle on a bounded,
seeded sample), so its JSON line can be checked here without a GPU; under a
multi-rank launch only rank 0 prints."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(args, env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT,
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    return [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]


def test_reference_arm_line():
    lines = run_bench(["--impl", "reference", "--steps", "1", "--warmup", "0", "--n", "12"])
    assert len(lines) == 1
    j = lines[0]
    assert j["impl"] == "reference" and j["unit"] == "nodes/s" and j["value"] > 0
    assert j["higher_is_better"] is True and j["steps"] == 1 and j["warmup"] == 0
    assert j["cpu_baseline"]["kind"] == "oracle" and j["cpu_baseline"]["cores"] >= 1
    assert j["cpu_baseline"]["value"] == j["value"] and j["cpu_baseline"]["sample"]
    assert j["e2e"] == {"value": j["value"], "unit": j["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert j["config"]["n"] == 12 and j["vs_baseline"] is None


def test_reference_arm_other_ranks_print_nothing():
    lines = run_bench(["--impl", "reference", "--steps", "1", "--warmup", "0", "--n", "12"],
                      {"WORLD_SIZE": "2", "RANK": "1", "LOCAL_RANK": "1"})
    assert lines == []


def test_reference_arm_depth_matches_the_library():
    """The reference arm restates the library's default depth instead of loading
    libnq; the two rules agree for every board size."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2511_12009_gb300 import nq
    for n in range(1, 32):
        assert bench.default_depth(n) == nq.default_depth(n), n


def test_reference_arm_does_not_load_the_library():
    code = ("import sys, runpy; sys.argv = ['bench.py', '--impl', 'reference', '--steps', '1', "
            "'--warmup', '0', '--n', '10']; runpy.run_path('bench.py', run_name='__main__'); "
            "print('LOADED' if any(m.startswith('paper_2511_12009_gb300') for m in sys.modules) "
            "else 'CLEAN')")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip().splitlines()[-1] == "CLEAN"


def test_served_answer_check_catches_a_wrong_answer():
    """The served bench's exactness check: answers equal to OEIS for boards
    without queens and to the oracle for a seeded sample pass; one wrong
    answer in either group fails it. (Small stream, boards N <= 12.)"""
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    import synth_inputs
    oracle.build()
    reqs = synth_inputs.request_stream(7, 60, 6, 12, 0, 3, rate_per_s=1.0)
    q = json.load(open(os.path.join(ROOT, "tests", "golden", "oeis_a000170.json")))["Q"]
    right = {i: (q[str(r["n"])] if not r["queens"] else oracle.count_constrained(r["n"], r["queens"])[0])
             for i, r in enumerate(reqs)}
    chk = bench.check_served_answers(reqs, right, sample=1000, n16=0)
    assert chk["exact"] and chk["mismatches"] == 0
    assert chk["constrained_vs_oracle"] == sum(1 for r in reqs if r["queens"])
    k0 = next(i for i, r in enumerate(reqs) if not r["queens"])
    k1 = next(i for i, r in enumerate(reqs) if r["queens"])
    for i in (k0, k1):
        wrong = dict(right)
        wrong[i] += 1
        assert not bench.check_served_answers(reqs, wrong, sample=1000, n16=0)["exact"]
