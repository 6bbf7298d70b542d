"""The launch-shape tuning table (biot_tune_get / biot_tune_put / biot_tune_cache_path):
host-only, no GPU.  Each case runs in a fresh process, since the library reads the cache
file once per process."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(code, cache, **env):
    e = dict(os.environ, BIOT_TUNE_CACHE=str(cache), **env)
    out = subprocess.run([sys.executable, "-c", "from paper_1801_04984_gb300 import binding as B\n" + code],
                         cwd=ROOT, env=e, capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    return out.stdout.strip()


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1801_04984_gb300 import build
    build.build()


def test_put_persists_across_processes_as_json(tmp_path):
    cache = tmp_path / "sub" / "dir" / "tune.json"  # missing directories are created
    assert _run("print(B.tune_cache_path())", cache) == str(cache)
    _run("B.tune_put('elast3_zrun|GPU_sm152|129x129x129|cols3', 22); B.tune_put('k2', 7)", cache)
    data = json.load(open(cache))
    assert data == {"elast3_zrun|GPU_sm152|129x129x129|cols3": 22, "k2": 7}
    got = _run("print(B.tune_get('elast3_zrun|GPU_sm152|129x129x129|cols3'), B.tune_get('k2'), B.tune_get('absent'))", cache)
    assert got.split() == ["22", "7", "-1"]
    # a later put keeps the earlier entries and replaces its own
    _run("B.tune_put('k2', 9)", cache)
    assert json.load(open(cache)) == {"elast3_zrun|GPU_sm152|129x129x129|cols3": 22, "k2": 9}


def test_malformed_or_missing_file_is_ignored(tmp_path):
    cache = tmp_path / "tune.json"
    assert _run("print(B.tune_get('k'))", cache) == "-1"
    cache.write_text('{"k": 5, "broken": }')
    # what parses before the damage is kept; the damaged entry is dropped
    assert _run("print(B.tune_get('k'), B.tune_get('broken'))", cache).split() == ["5", "-1"]
    cache.write_text("not json at all")
    assert _run("print(B.tune_get('k'))", cache) == "-1"
    _run("B.tune_put('k', 3)", cache)  # rewritten as a valid object
    assert json.load(open(cache)) == {"k": 3}


def test_invalid_keys_are_rejected(tmp_path):
    cache = tmp_path / "tune.json"
    code = ("import sys\n"
            "for k in ('', 'a\"b', 'a\\\\b'):\n"
            "    try:\n"
            "        B.tune_put(k, 1)\n"
            "    except B.BiotError:\n"
            "        continue\n"
            "    sys.exit('accepted %r' % k)\n")
    _run(code, cache)
    assert not cache.exists()
