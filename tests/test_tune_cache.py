"""The delay autotuner's cache: keys, round trip, and cache hits that need no GPU."""
import json

import ggf_inputs as gi


def test_key_and_round_trip(tmp_path, monkeypatch):
    from paper_2412_01737_gb300 import tune
    p = gi.make_problem(4, gi.U1, 2, 2)
    assert tune.key_of(p, 12, 1) == "L4_g1_nv2_K2_c12_p1"
    path = tmp_path / "sub" / "cache.json"
    data = {"a": {"delay": 8, "ms": {"4": 2.0, "8": 1.5}}}
    tune._store(str(path), data)
    assert tune._load(str(path)) == data
    assert tune._load(str(tmp_path / "missing.json")) == {}
    (tmp_path / "bad.json").write_text("{not json")
    assert tune._load(str(tmp_path / "bad.json")) == {}


def test_cache_hit_returns_stored_choice(tmp_path, monkeypatch):
    from paper_2412_01737_gb300 import tune
    p = gi.make_problem(3, gi.Z2, 1, 1)
    links = gi.cold_links(p, 5)
    path = tmp_path / "cache.json"
    path.write_text(json.dumps({tune.key_of(p, 5, 1): {"delay": 16, "ms": {"4": 3.0, "16": 1.0}}}))
    monkeypatch.setenv("GGF_TUNE_CACHE", str(path))
    best, ms = tune.tune_delay(p, links, 1)
    assert best == 16 and ms == {4: 3.0, 16: 1.0}
