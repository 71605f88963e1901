"""C-ABI checks that need no GPU: the library builds, loads, and exports every
entry point the headers under include/ declare; host-only paths validate
arguments; the product package never touches the oracle."""
import ctypes
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = sorted(os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
                 if f.endswith(".h"))


def _built_lib():
    import __graft_entry__ as g
    b = g._load_pkg_build()
    return b.build()


def declared_functions():
    names = set()
    for h in HEADERS:
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(epsm_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("epsm_create", "epsm_search", "epsm_search_batch", "epsm_destroy",
                     "epsm_status_str", "epsm_server_create", "epsm_server_submit",
                     "epsm_server_poll", "epsm_server_replay"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib_path = _built_lib()
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(lib_path)
    for n in declared_functions():
        assert hasattr(lib, n)


def test_status_strings_and_null_context():
    _built_lib()
    import paper_1209_6449_gb300 as epsm
    assert epsm.epsm_status_str(0) == "EPSM_OK"
    assert epsm.epsm_status_str(5) == "EPSM_ERR_TIMEOUT"
    lib = epsm._lib
    cnt = ctypes.c_uint64(7)
    # NULL context / bad m are rejected on the host before any CUDA call
    assert lib.epsm_search(None, None, 0, b"a", 1, None, 0, ctypes.byref(cnt), None) == 1
    assert lib.epsm_search_async(None, None, 0, b"a", 1, None, 0, None, None) == 1
    assert lib.epsm_destroy(None) == 0
    assert lib.epsm_variant_for(None, 4) == 0
    assert lib.epsm_wait_probe(None, 1000, None) == 1


def test_server_arguments_checked_on_the_host():
    _built_lib()
    import paper_1209_6449_gb300 as epsm
    lib = epsm._lib
    rid = ctypes.c_uint64()
    assert lib.epsm_server_create(None, 0, None) == 1
    assert lib.epsm_server_destroy(None) == 0
    assert lib.epsm_server_submit(None, 0, b"ab", 2, ctypes.byref(rid)) == 1
    assert lib.epsm_server_upload(None, b"ab", 2, ctypes.byref(rid)) == 1
    assert lib.epsm_server_poll(None, None, 4, 0) == 0
    assert lib.epsm_server_release(None, 1) == 1
    assert lib.epsm_server_read(None, 1, None, 0) == 1
    assert lib.epsm_server_inject_fault(None, 0, 1) == 1


def test_missing_library_fails_loudly(tmp_path):
    _built_lib()
    from paper_1209_6449_gb300 import _native
    with pytest.raises(ImportError):
        _native.load(str(tmp_path / "nope.so"))


def test_package_does_not_reach_the_oracle():
    pkg = os.path.join(ROOT, "paper_1209_6449_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".inc")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "liboracle" not in txt and "epsm_oracle" not in txt, f
    code = ("import sys; sys.path.insert(0, %r); import paper_1209_6449_gb300; "
            "assert 'oracle' not in sys.modules; print('clean')" % ROOT)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True)
    assert out.returncode == 0 and "clean" in out.stdout, out.stderr


def test_shipped_tuning_table_is_consistent():
    """tuning.json (written by the autotuner on a GPU) names, for every
    alphabet class, text-length bucket and m in 1..32, a variant that covers
    m, a launch shape and a fingerprint width in range."""
    import json
    path = os.path.join(ROOT, "paper_1209_6449_gb300", "tuning.json")
    if not os.path.exists(path):
        pytest.skip("no tuning table shipped")
    with open(path) as f:
        tab = json.load(f)
    assert tab["version"] == 2
    cover = {1: range(1, 5), 2: range(4, 16), 3: range(8, 16), 4: range(15, 33), 5: range(7, 17),
             6: range(2, 17), 7: range(5, 17), 8: range(23, 33)}
    names = {1: "direct", 2: "prefix4", 3: "prefix8", 4: "block8", 5: "block4", 6: "code2",
             7: "adapt", 8: "block8s"}
    assert {"dna", "protein", "text", "mixed"} <= set(tab["classes"])
    for cls, rows in tab["classes"].items():
        assert sorted(int(b) for b in rows) == [0, 1, 2], cls
        for b, by_m in rows.items():
            assert sorted(int(m) for m in by_m) == list(range(1, 33)), (cls, b)
            for m, r in by_m.items():
                assert int(m) in cover[r["variant"]], (cls, b, m, r)
                assert r["name"] == names[r["variant"]]
                assert r["shape"] in (0, 1) and 8 <= r["kbits"] <= 14


def test_tuning_bucket_bounds_match_header():
    import re as _re
    from paper_1209_6449_gb300 import _native
    src = open(os.path.join(ROOT, "include", "epsm.h")).read()
    b1 = int(_re.search(r"EPSM_BUCKET1_MIN \((\d+)ull << (\d+)\)", src).group(1)) << 20
    b2 = int(_re.search(r"EPSM_BUCKET2_MIN \((\d+)ull << (\d+)\)", src).group(1)) << 20
    assert _native.BUCKET_MIN == (0, b1, b2)
    assert [_native.text_bucket(n) for n in (0, b1 - 1, b1, b2 - 1, b2)] == [0, 0, 1, 1, 2]
