"""The batch autotuner's cache file (tune_cache.cpp, host only): entries
round-trip, a store replaces its own key and keeps the others, the file
stays valid JSON, hand-written entries in the documented shape are read,
and lines that are not entries are skipped.  The file's functions are
compiled here with a small driver (g++, no GPU)."""
import json
import os
import shutil
import subprocess

import pytest

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_1710_01048_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include <cstring>
#include <string>
namespace wq {
std::string tune_cache_clean_key(const std::string &raw);
bool tune_cache_lookup(const char *path, const std::string &key, int cfg[4], double *ms);
bool tune_cache_store(const char *path, const std::string &key, const int cfg[4], double ms);
}
// usage: drv store PATH KEY c0 c1 c2 c3 ms | drv lookup PATH KEY | drv clean KEY
int main(int argc, char **argv) {
  if (argc >= 3 && !std::strcmp(argv[1], "clean")) {
    std::printf("%s\n", wq::tune_cache_clean_key(argv[2]).c_str());
    return 0;
  }
  if (argc == 9 && !std::strcmp(argv[1], "store")) {
    int c[4];
    for (int i = 0; i < 4; i++) c[i] = std::atoi(argv[4 + i]);
    return wq::tune_cache_store(argv[2], argv[3], c, std::atof(argv[8])) ? 0 : 1;
  }
  if (argc == 4 && !std::strcmp(argv[1], "lookup")) {
    int c[4];
    double ms = 0;
    if (!wq::tune_cache_lookup(argv[2], argv[3], c, &ms)) {
      std::printf("miss\n");
      return 0;
    }
    std::printf("%d %d %d %d %.17g\n", c[0], c[1], c[2], c[3], ms);
    return 0;
  }
  return 2;
}
"""


@pytest.fixture(scope="module")
def drv(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("tc")
    src = d / "drv.cpp"
    src.write_text(DRIVER.replace("#include <cstring>", "#include <cstring>\n#include <cstdlib>"))
    exe = d / "drv"
    subprocess.run(["g++", "-std=c++17", "-O1", str(src), os.path.join(CSRC, "tune_cache.cpp"), "-o", str(exe)],
                   check=True, capture_output=True)
    return str(exe)


def run(drv, *args):
    r = subprocess.run([drv, *map(str, args)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return r.stdout.strip()


def test_round_trip_and_replace(drv, tmp_path):
    f = tmp_path / "c.json"
    assert run(drv, "lookup", f, "k1") == "miss"  # no file
    run(drv, "store", f, "v1|GPU A|fp64", 32, 2, 3, 1, 1.5)
    run(drv, "store", f, "v1|GPU A|mixed", 16, 1, 1, 0, 0.25)
    assert run(drv, "lookup", f, "v1|GPU A|fp64") == "32 2 3 1 1.5"
    assert run(drv, "lookup", f, "v1|GPU A|mixed") == "16 1 1 0 0.25"
    assert run(drv, "lookup", f, "v1|GPU B|fp64") == "miss"
    run(drv, "store", f, "v1|GPU A|fp64", 24, 1, 2, 0, 0.75)
    d = json.loads(f.read_text())
    assert d == {"v1|GPU A|fp64": {"config": [24, 1, 2, 0], "ms": 0.75},
                 "v1|GPU A|mixed": {"config": [16, 1, 1, 0], "ms": 0.25}}
    assert not [p for p in os.listdir(tmp_path) if ".tmp." in p]


def test_hand_written_entries_and_foreign_lines(drv, tmp_path):
    f = tmp_path / "c.json"
    f.write_text('{\n  "a":{"config":[8,1,1,1],"ms":2e-1},\n'
                 '  "broken": {"config": [8, 1, 1], "ms": 1},\n'
                 '  "neg": {"config": [8, -1, 1, 0], "ms": 1},\n'
                 '  "b" : { "config" : [ 32 , 2 , 3 , 0 ] , "ms" : 4 }\n}\n')
    assert run(drv, "lookup", f, "a") == "8 1 1 1 0.20000000000000001"
    assert run(drv, "lookup", f, "b") == "32 2 3 0 4"
    assert run(drv, "lookup", f, "broken") == "miss"
    assert run(drv, "lookup", f, "neg") == "miss"
    run(drv, "store", f, "c", 16, 1, 1, 0, 3)
    assert set(json.loads(f.read_text())) == {"a", "b", "c"}  # foreign lines are dropped on rewrite


def test_keys_are_json_safe(drv, tmp_path):
    assert run(drv, "clean", 'x"y\\z') == "x_y_z"
    f = tmp_path / "c.json"
    k = run(drv, "clean", 'GPU "quoted"')
    run(drv, "store", f, k, 32, 1, 1, 0, 1)
    assert json.loads(f.read_text()) == {"GPU _quoted_": {"config": [32, 1, 1, 0], "ms": 1}}
