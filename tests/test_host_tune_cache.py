"""Host logic of the launch-shape autotuner's cache (sl_tune), on CPU: the JSON reader and writer
compiled with the host compiler.  Written files are valid JSON that round-trips; files written by
another JSON writer with string values are read; anything else (a non-object, a non-string
value, a truncated file) is refused; a missing file is an empty cache."""
import json
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1910_06476_gb300", "csrc")


@pytest.fixture(scope="module")
def rt(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("host compiler not available")
    exe = str(tmp_path_factory.mktemp("tune") / "tune_cache_rt")
    r = subprocess.run([gxx, "-O1", "-std=c++17", "-I", CSRC, os.path.join(ROOT, "tests", "host", "tune_cache_rt.cpp"),
                        "-o", exe], capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail(r.stderr[-2000:])
    return exe


def read(rt, path):
    out = subprocess.run([rt, "read", str(path)], capture_output=True, text=True, check=True).stdout.splitlines()
    if out[0] == "bad":
        return None
    return dict(line.split("\t") for line in out[1:])


def test_round_trip_and_valid_json(rt, tmp_path):
    p = tmp_path / "c.json"
    pairs = {"k2c_tile|dev=NVIDIA GB300|n=9|kx=512|ky=512|nel=262144|mapped=0|cons=3|fit=0|bv=0|rk=4|vel=0": "tile=2",
             "k2m_per_sm|dev=NVIDIA GB300|n=8|kx=2048|ky=2048|nel=4194304|mapped=0|cons=7|fit=0|bv=0|rk=4|vel=2":
                 "p1=2,p2=0"}
    args = [x for kv in pairs.items() for x in kv]
    subprocess.run([rt, "write", str(p)] + args, check=True)
    assert json.loads(p.read_text()) == pairs
    assert read(rt, p) == pairs
    assert not (tmp_path / "c.json.tmp").exists()


def test_reads_other_writers_and_missing_files(rt, tmp_path):
    p = tmp_path / "other.json"
    p.write_text(json.dumps({"a|n=4": "tile=1", "b": "p1=0,p2=1"}, indent=4))
    assert read(rt, p) == {"a|n=4": "tile=1", "b": "p1=0,p2=1"}
    p.write_text("{}")
    assert read(rt, p) == {}
    assert read(rt, tmp_path / "absent.json") == {}


@pytest.mark.parametrize("text", ["[1, 2]", '{"a": 1}', '{"a": "b"', '{"a" "b"}', '{"a": "b",}', "nonsense"])
def test_refuses_malformed_files(rt, tmp_path, text):
    p = tmp_path / "bad.json"
    p.write_text(text)
    assert read(rt, p) is None
