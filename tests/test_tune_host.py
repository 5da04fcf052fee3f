"""The tuning cache without a GPU: cv_tune_cache_put / cv_tune_cache_get on a
JSON file (round trip, replacement, several keys, the CVX_TUNE_CACHE default
path, malformed files and keys).  The measuring side, cv_plan_tune, is
covered by tests/test_gpu_tune.py."""
import json

import pytest

import paper_2401_13185_gb300 as cvx


def test_put_get_round_trip(tmp_path):
    path = str(tmp_path / "tune.json")
    assert cvx.cv_tune_cache_get(path, "sm152/prec4/K8") is None          # no file yet
    cvx.cv_tune_cache_put(path, "sm152/prec4/K8", (cvx.CV_STRATEGY_SMALL_FOLDS, 0), 1.25)
    cvx.cv_tune_cache_put(path, "sm152/prec4/K16", (cvx.CV_STRATEGY_FOLD_GROUPED, 76), 2.5)
    o, ms = cvx.cv_tune_cache_get(path, "sm152/prec4/K8")
    assert (o.strategy, o.ctas, ms) == (cvx.CV_STRATEGY_SMALL_FOLDS, 0, 1.25)
    o, ms = cvx.cv_tune_cache_get(path, "sm152/prec4/K16")
    assert (o.strategy, o.ctas, ms) == (cvx.CV_STRATEGY_FOLD_GROUPED, 76, 2.5)
    assert (o.fold_begin, o.fold_end, o.xtx_layout, o.reserved, o.wait_limit_ns) == (0, 0, 0, 0, 0)
    assert cvx.cv_tune_cache_get(path, "sm152/prec4/K32") is None
    # the file is plain JSON: one object of {"strategy", "ctas", "ms"} entries
    d = json.load(open(path))
    assert d == {"sm152/prec4/K8": {"strategy": 2, "ctas": 0, "ms": 1.25},
                 "sm152/prec4/K16": {"strategy": 1, "ctas": 76, "ms": 2.5}}


def test_put_replaces_an_entry(tmp_path):
    path = str(tmp_path / "tune.json")
    cvx.cv_tune_cache_put(path, "a/b", (1, 10), 3.0)
    cvx.cv_tune_cache_put(path, "a/b", (0, 0), 1.0)
    o, ms = cvx.cv_tune_cache_get(path, "a/b")
    assert (o.strategy, o.ctas, ms) == (0, 0, 1.0)
    assert len(json.load(open(path))) == 1


def test_environment_variable_names_the_default_file(tmp_path, monkeypatch):
    path = tmp_path / "env.json"
    monkeypatch.setenv("CVX_TUNE_CACHE", str(path))
    cvx.cv_tune_cache_put(None, "k2^3", (1, 5), 0.5)
    assert path.exists()
    o, ms = cvx.cv_tune_cache_get(None, "k2^3")
    assert (o.strategy, o.ctas, ms) == (1, 5, 0.5)
    monkeypatch.delenv("CVX_TUNE_CACHE")
    assert cvx.cv_tune_cache_get(None, "k2^3") is None      # no file named: nothing cached
    cvx.cv_tune_cache_put(None, "k2^3", (1, 5), 0.5)         # and nothing written


def test_malformed_files_keep_what_parses(tmp_path):
    path = tmp_path / "bad.json"
    path.write_text('{"ok/1": {"strategy": 1, "ctas": 4, "ms": 2}, "bad": {"strategy": }, "late": {}}')
    o, ms = cvx.cv_tune_cache_get(str(path), "ok/1")
    assert (o.strategy, o.ctas, ms) == (1, 4, 2.0)
    assert cvx.cv_tune_cache_get(str(path), "late") is None
    path.write_text("not json at all")
    assert cvx.cv_tune_cache_get(str(path), "ok/1") is None
    # an entry with an unknown strategy or a negative ctas is not taken
    path.write_text('{"x": {"strategy": 9, "ctas": 0, "ms": 1}, "y": {"strategy": 0, "ctas": -2, "ms": 1}}')
    assert cvx.cv_tune_cache_get(str(path), "x") is None
    assert cvx.cv_tune_cache_get(str(path), "y") is None
    # put over a malformed file rewrites it with the entries that parsed
    path.write_text('{"keep": {"ctas": 3, "ms": 1.5, "strategy": 1}, oops')
    cvx.cv_tune_cache_put(str(path), "new", (0, 0), 0.25)
    assert json.load(open(path)) == {"keep": {"strategy": 1, "ctas": 3, "ms": 1.5},
                                     "new": {"strategy": 0, "ctas": 0, "ms": 0.25}}


def test_bad_arguments_are_rejected(tmp_path):
    path = str(tmp_path / "t.json")
    for key in ("", 'quote"d', "sp ace", "brace{"):
        with pytest.raises(cvx.CVError) as e:
            cvx.cv_tune_cache_put(path, key, (0, 0), 1.0)
        assert e.value.name == "CV_ERR_INVALID_ARG"
    for opts, ms in (((3, 0), 1.0), ((0, -1), 1.0), ((0, 0), -1.0), ((0, 0), float("nan"))):
        with pytest.raises(cvx.CVError):
            cvx.cv_tune_cache_put(path, "k", opts, ms)
    with pytest.raises(cvx.CVError):
        cvx.cv_tune_cache_put(str(tmp_path / "no" / "such" / "dir.json"), "k", (0, 0), 1.0)
