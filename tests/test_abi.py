"""CPU checks of the C-ABI boundary: the library builds for sm_103a, loads,
and exports every entry point include/rtucker.h declares; host-only calls
work without a GPU; the product package never touches the oracle."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rtucker.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(rt\w*|rtucker\w*|rhtucker\w*)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2603_21379_gb300 import build
    build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_path_entry_points():
    names = declared_functions()
    for must in ["rtucker_indices", "rtucker_sketch", "rtucker_factors", "rtucker_core", "rtucker_decompose",
                 "rtucker_decompose_host", "rtucker_decompose_host_async", "rtucker_decompose_batched", "rtucker_relerr", "rhtucker_decompose",
                 "rhtucker_relerr", "rt_create", "rt_destroy", "rt_sync", "rt_last_error"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls(lib):
    lib.rt_status_string.restype = ctypes.c_char_p
    assert lib.rt_status_string(0) == b"ok"
    assert lib.rt_status_string(1) == b"invalid argument"
    assert lib.rt_version() >= 1
    # null handle / null output pointers are rejected before any CUDA call
    lib.rt_destroy.argtypes = [ctypes.c_void_p]
    assert lib.rt_destroy(None) == 1
    lib.rt_create.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    assert lib.rt_create(None, None) == 1


def test_binding_names_match_c_abi():
    import paper_2603_21379_gb300 as pkg
    for n in declared_functions():
        if n.startswith(("rtucker_", "rhtucker_")):
            assert hasattr(pkg, n), n


def test_product_path_never_touches_oracle():
    pkg = os.path.join(ROOT, "paper_2603_21379_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"\boracle\b", src), f


def test_options_struct_matches_the_header():
    # the binding's rt_options: same int32 fields, same order, same size as the header
    import paper_2603_21379_gb300 as rt
    text = open(HEADER).read()
    body = re.search(r"typedef struct \{(.*?)\} rt_options;", text, flags=re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"int32_t\s+(\w+)(?:\[(\d+)\])?;", body)
    header = [(name, int(count) if count else 1) for name, count in fields]
    ours = []
    for name, ctype in rt._Options._fields_:
        ours.append((name, getattr(ctype, "_length_", 1)))
    assert header == ours
    assert ctypes.sizeof(rt._Options) == 4 * sum(c for _, c in header)


def test_option_marshalling():
    import paper_2603_21379_gb300 as rt
    assert rt._opts("fp32") is None                      # defaults: no struct
    o = rt._opts("bf16", overlap=True, graph=True, core="ffma")._obj
    assert (o.prec, o.overlap, o.use_graph, o.core) == (1, 1, 1, 2)
    assert list(o.reserved) == [0] * len(o.reserved)
    assert rt._opts("fp32", core="tc")._obj.core == 1
    with pytest.raises(ValueError):
        rt._opts("fp16")
    assert rt._opts("fp32", core="tune")._obj.core == 3
    with pytest.raises(ValueError):
        rt._opts("fp32", core="wmma")
    assert rt._opts("fp32", qr="householder")._obj.qr == 1
    assert rt._opts("fp32", qr="cholesky")._obj.qr == 2
    with pytest.raises(ValueError):
        rt._opts("fp32", qr="givens")


def test_product_never_uses_the_scratch_folder():
    # nothing tracked imports, reads or runs a file of the untracked working folder
    import subprocess
    try:
        files = subprocess.run(["git", "ls-files"], cwd=ROOT, capture_output=True, text=True,
                               check=True).stdout.split()
    except (OSError, subprocess.CalledProcessError):
        pytest.skip("not a git checkout")
    pat = re.compile(r"(?<![\w.])_work[/\\.]|import\s+_work|['\"]_work['\"]")
    hits = []
    for f in files:
        if f == ".gitignore" or not f.endswith((".py", ".cu", ".cuh", ".h", ".cpp", ".sh", ".toml", ".cfg")):
            continue
        with open(os.path.join(ROOT, f), errors="ignore") as fh:
            for i, line in enumerate(fh, 1):
                if pat.search(line):
                    hits.append("%s:%d" % (f, i))
    assert not hits, hits


def test_fp8_storage_sizes(lib):
    # packed float8 storage: codes, then at the element count rounded up to 256 one
    # float32 scale per slab of the last two modes, the whole rounded up to 16 bytes
    lib.rt_fp8_bytes.restype = ctypes.c_size_t
    lib.rt_fp8_scale_offset.restype = ctypes.c_size_t

    def call(fn, n):
        return fn(len(n), (ctypes.c_int64 * len(n))(*n))
    assert call(lib.rt_fp8_scale_offset, [3, 2, 12, 20]) == 1536
    assert call(lib.rt_fp8_bytes, [3, 2, 12, 20]) == 1536 + 6 * 4 + 8
    assert call(lib.rt_fp8_bytes, [300, 200]) == 60160 + 16        # one slab
    assert call(lib.rt_fp8_bytes, [128] * 4) == 128 ** 4 + 4 * 128 ** 2
    assert call(lib.rt_fp8_bytes, [7]) == 0 and call(lib.rt_fp8_bytes, [4, 0, 3]) == 0
