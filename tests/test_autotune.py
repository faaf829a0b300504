"""Host logic of the autotuner (coordinate descent and its cache), no GPU."""
import json

from paper_1809_07444_gb300 import autotune as AT


def _bowl(best):
    # separable score with a unique optimum at `best`; one setting cannot run
    rank = {k: {v: i for i, v in enumerate(AT.SPACE[k])} for k in AT.ORDER}

    def measure(t):
        if t["threads"] == 512 and t["fanout"] == 16:
            return None
        return 100.0 - sum(abs(rank[k][t[k]] - rank[k][best[k]]) * (3 - i) for i, k in enumerate(AT.ORDER))
    return measure


def test_search_finds_the_optimum_of_a_separable_score():
    for best in ({"threads": 512, "cap_min": 32, "fanout": 32}, {"threads": 128, "cap_min": 64, "fanout": 16},
                 dict(AT.DEFAULT)):
        got, v, table = AT.search(_bowl(best))
        assert got == best and v == 100.0
        # every setting measured once, far fewer than the full grid of 18
        assert len(table) <= 3 + 2 + 3 + 4


def test_search_skips_settings_that_cannot_run():
    calls = []

    def measure(t):
        calls.append(dict(t))
        return None if t["cap_min"] == 32 else float(t["threads"])
    got, v, table = AT.search(measure)
    assert got["threads"] == 512 and got["cap_min"] == 64 and v == 512.0
    assert table[(512, 32, 64)] is None  # tried after threads moved to 512


def test_tuned_caches_by_key(tmp_path):
    path = str(tmp_path / "cache.json")
    n = []

    def measure(t):
        n.append(1)
        return float(t["threads"]) + (1.0 if t["fanout"] == 32 else 0.0)
    t1, v1, table = AT.tuned("dev/workload", measure, path=path)
    assert t1 == {"threads": 512, "cap_min": 64, "fanout": 32} and table is not None
    k = len(n)
    t2, v2, table2 = AT.tuned("dev/workload", measure, path=path)
    assert t2 == t1 and v2 == v1 and table2 is None and len(n) == k  # cache hit, nothing measured
    data = json.load(open(path))
    assert data["dev/workload"]["tuning"] == t1
    AT.tuned("dev/workload", measure, path=path, refresh=True)
    assert len(n) > k
