"""The autotuners' JSON cache on the host (no GPU): malformed files read as empty, entries that are
not candidates are tuned again, and concurrent writers leave a whole file behind."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture()
def at(tmp_path, monkeypatch):
    if not os.path.exists(os.path.join(ROOT, "paper_2308_09839_gb300", "libmf.so")):
        from paper_2308_09839_gb300 import build
        build.build()
    monkeypatch.setenv("MF_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    from paper_2308_09839_gb300 import autotune
    return autotune


def test_malformed_cache_reads_as_empty(at, tmp_path):
    path = tmp_path / "tune.json"
    assert at._load() == {}
    for text in ("[1, 2]", "{not json", "17", ""):
        path.write_text(text)
        assert at._load() == {}


def test_store_then_load_leaves_no_temporary(at, tmp_path):
    at._store({"gpu|apply|laplace|(8, 8, 8)": 16})
    assert at._load() == {"gpu|apply|laplace|(8, 8, 8)": 16}
    assert sorted(os.listdir(tmp_path)) == ["tune.json"]


def test_only_candidates_are_taken_from_the_cache(at):
    c = {"a": 8, "b": "8", "c": True, "d": 7, "e": 8.0, "f": None}
    assert at._cached(c, "a", at.CANDIDATES) == 8
    for k in ("b", "c", "d", "e", "f", "missing"):
        assert at._cached(c, k, at.CANDIDATES) is None
    assert at._cached({"z": 0}, "z", at.APPLY_CANDIDATES) == 0
    assert at._cached({"z": 0}, "z", at.CANDIDATES) is None


def test_concurrent_writers_leave_a_whole_file(at, tmp_path):
    code = ("import sys; from paper_2308_09839_gb300 import autotune as a\n"
            "w = int(sys.argv[1])\n"
            "for i in range(40): a._store({f'writer{w}': i, 'pad': 'x' * 20000})\n")
    env = dict(os.environ, MF_AUTOTUNE_CACHE=str(tmp_path / "tune.json"))
    procs = [subprocess.Popen([sys.executable, "-c", code, str(w)], cwd=ROOT, env=env) for w in range(3)]
    for p in procs:
        assert p.wait(timeout=300) == 0
    d = json.loads((tmp_path / "tune.json").read_text())
    assert len(d) == 2 and d["pad"] == "x" * 20000 and any(d.get(f"writer{w}") == 39 for w in range(3))
    assert sorted(os.listdir(tmp_path)) == ["tune.json"]


class _FakeMesh:
    physics, dims, device = "laplace", (8, 8, 40), "cpu"
    info = {"n_dof": 9 * 9 * 41}

    def apply(self, x, y):
        pass


class _FakeEvent:
    def __init__(self, enable_timing=False):
        pass

    def record(self):
        pass

    def elapsed_time(self, other):
        return 1.0


def test_tune_apply_uses_valid_cache_entries_and_retunes_the_rest(at, monkeypatch):
    """tune_apply's host logic with the device parts faked: a cached candidate is used as is; an entry
    that is not a candidate is tuned again (every candidate equally fast: the first, 0, wins) and the
    cache is rewritten."""
    import torch
    calls = []
    monkeypatch.setattr(at, "_device_key", lambda: "gpu")
    monkeypatch.setattr(at.mf, "mf_set_tile_segment", lambda mesh, seg: calls.append(seg))
    monkeypatch.setattr(torch.cuda, "Event", _FakeEvent)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda: None)
    key = "gpu|apply|laplace|(8, 8, 40)"
    at._store({key: 16})
    assert at.tune_apply(_FakeMesh(), reps=1) == 16 and calls == [16]
    at._store({key: 7})
    calls.clear()
    assert at.tune_apply(_FakeMesh(), reps=1) == 0
    assert calls == [0, 8, 12, 16, 20, 24, 32, 0]  # segments above the 41 node planes are skipped
    assert at._load() == {key: 0}
