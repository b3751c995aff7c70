"""The C ABI on the host (no GPU needed): the library loads, exports every
function include/gbblas.h declares, and rejects invalid arguments with the
documented status before touching any device.  Pointers here are fake
addresses that are never dereferenced: every call below returns during host
validation (or through a host-side injected fault)."""
import os
import re
import subprocess
import sys
import textwrap

import pytest

import paper_2108_02025_gb300 as gb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gbblas.h")

P = 1 << 20          # fake, 256-byte aligned device addresses
Q = 1 << 30
R = 1 << 34
W = 1 << 36


def declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|int64_t|size_t|void|const char \*)\s*(gb_\w+)\s*\(", text, re.M)))


def test_every_declared_symbol_is_exported():
    names = declared()
    assert len(names) == 23
    for name in names:
        assert hasattr(gb.lib(), name), name
    assert sorted(gb.EXPORTS) == names


def test_version_and_status_strings():
    assert gb.gb_version() >= 100
    for s in (0, -100, -101, -102, -103, -5, 7):
        assert isinstance(gb.gb_status_string(s), str) and gb.gb_status_string(s)
    assert "argument" in gb.gb_status_string(-4)


@pytest.mark.parametrize("f", ["gb_dgemv", "gb_sgemv"])
def test_gemv_validation(f):
    g = getattr(gb, f)
    nb = gb.gb_workspace_bytes(gb.OP_GEMV, gb.F64 if f == "gb_dgemv" else gb.F32, 0, 64, 1 << 20)
    assert nb > 0
    assert g(2, 4, 4, 1.0, P, 4, Q, R, None, 0, 0) == -1
    assert g(0, -1, 4, 1.0, P, 4, Q, R, None, 0, 0) == -2
    assert g(0, 4, -1, 1.0, P, 4, Q, R, None, 0, 0) == -3
    assert g(0, 4, 5, 1.0, P, 4, Q, R, None, 0, 0) == -6          # row-major lda < n
    assert g(1, 5, 4, 1.0, P, 4, Q, R, None, 0, 0) == -6          # col-major lda < m
    assert g(0, 4, 4, 1.0, None, 4, Q, R, None, 0, 0) == -5
    assert g(0, 4, 4, 1.0, P, 4, None, R, None, 0, 0) == -7
    assert g(0, 4, 4, 1.0, P, 4, Q, None, None, 0, 0) == -8
    assert g(0, 4, 4, 1.0, P, 4, Q, P + 8, None, 0, 0) == -8      # c overlaps A
    assert g(0, 4, 4, 1.0, P, 4, Q, Q, None, 0, 0) == -8          # c overlaps x
    assert g(0, 64, 1 << 20, 1.0, P, 1 << 20, Q, R, None, nb, 0) == -9     # workspace missing
    assert g(0, 64, 1 << 20, 1.0, P, 1 << 20, Q, R, W + 4, nb, 0) == -9    # misaligned
    assert g(0, 64, 1 << 20, 1.0, P, 1 << 20, Q, R, W, nb - 8, 0) == gb.GB_ERR_WORKSPACE
    # quick returns: nothing is read, NULL pointers are fine
    assert g(0, 0, 4, 1.0, None, 4, None, None, None, 0, 0) == 0
    assert g(0, 4, 0, 1.0, None, 4, None, None, None, 0, 0) == 0
    assert g(0, 4, 4, 0.0, None, 4, None, None, None, 0, 0) == 0


@pytest.mark.parametrize("f", ["gb_ddot", "gb_sdot"])
def test_dot_validation(f):
    g = getattr(gb, f)
    n = 1 << 24
    nb = gb.gb_workspace_bytes(gb.OP_DOT, gb.F64 if f == "gb_ddot" else gb.F32, 0, 0, n)
    assert nb > 0
    assert g(-1, P, Q, R, W, nb, 0) == -1
    assert g(n, None, Q, R, W, nb, 0) == -2
    assert g(n, P, None, R, W, nb, 0) == -3
    assert g(n, P, Q, None, W, nb, 0) == -4
    assert g(n, P, Q, P + 64, W, nb, 0) == -4                      # alpha inside x
    assert g(n, P, Q, R, None, nb, 0) == -5
    assert g(n, P, Q, R, W, nb - 1, 0) == gb.GB_ERR_WORKSPACE
    assert g(0, None, None, None, None, 0, 0) == 0


@pytest.mark.parametrize("f", ["gb_dger", "gb_sger"])
def test_ger_validation(f):
    g = getattr(gb, f)
    assert g(3, 4, 4, 1.0, P, Q, R, 4, 0) == -1
    assert g(0, -4, 4, 1.0, P, Q, R, 4, 0) == -2
    assert g(0, 4, -4, 1.0, P, Q, R, 4, 0) == -3
    assert g(0, 4, 8, 1.0, P, Q, R, 4, 0) == -8
    assert g(1, 8, 4, 1.0, P, Q, R, 4, 0) == -8
    assert g(0, 4, 4, 1.0, None, Q, R, 4, 0) == -5
    assert g(0, 4, 4, 1.0, P, None, R, 4, 0) == -6
    assert g(0, 4, 4, 1.0, P, Q, None, 4, 0) == -7
    assert g(0, 4, 4, 1.0, P, Q, P + 8, 4, 0) == -7                # C overlaps x
    assert g(0, 4, 4, 0.0, None, None, None, 4, 0) == 0
    assert g(0, 0, 4, 1.0, None, None, None, 4, 0) == 0


def test_copy_to_host_validation():
    assert gb.gb_copy_to_host(None, None, 0, 0) == gb.GB_OK     # nothing to copy
    assert gb.gb_copy_to_host(None, P, 64, 0) == -1              # no destination
    assert gb.gb_copy_to_host(Q, None, 64, 0) == -2              # no source


def test_workspace_bytes():
    wb = gb.gb_workspace_bytes
    assert wb(gb.OP_GER, gb.F64, 0, 1000, 1000) == 0
    assert wb(gb.OP_GEMV, gb.F64, 0, 1048576, 64) == 0                # many rows: no split
    assert wb(gb.OP_GEMV, gb.F32, 0, 64, 1 << 20) > 0                 # wide: split sum
    assert wb(gb.OP_GEMV, gb.F32, 1, 64, 1 << 20) > 0
    assert wb(gb.OP_DOT, gb.F64, 0, 0, 1000) == 0                     # small DOT: one block
    assert wb(gb.OP_DOT, gb.F64, 0, 0, 1 << 28) > 0
    assert wb(gb.OP_GEMV, 7, 0, 64, 1 << 20) == 0                     # invalid dtype
    assert wb(gb.OP_GEMV, gb.F32, 5, 64, 1 << 20) == 0                # invalid layout
    assert wb(gb.OP_GEMV, gb.F32, 0, -1, 10) == 0
    # a pure function: same arguments, same size
    assert wb(gb.OP_GEMV, gb.F32, 0, 64, 1 << 20) == wb(gb.OP_GEMV, gb.F32, 0, 64, 1 << 20)


def test_fault_injection_is_host_side():
    """GB_FAULT_INJECT=<op>:<k> makes the k-th valid call return
    GB_ERR_INJECTED before anything is enqueued; invalid calls do not count."""
    code = textwrap.dedent(f"""
        import sys
        sys.path.insert(0, {ROOT!r})
        import paper_2108_02025_gb300 as gb
        P, Q, R = {P}, {Q}, {R}
        assert gb.gb_dger(0, -1, 4, 1.0, P, Q, R, 4, 0) == -2   # invalid: not counted
        assert gb.gb_sger(0, 4, 4, 1.0, P, Q, R, 4, 0) == gb.GB_ERR_INJECTED
        assert gb.gb_dgemv(0, -1, 4, 1.0, P, 4, Q, R, None, 0, 0) == -2
        print("ok")
    """)
    env = dict(os.environ, GB_FAULT_INJECT="ger:1")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0 and "ok" in r.stdout, r.stderr


def test_no_cpu_fallback_when_library_missing(tmp_path):
    """Without libgbblas.so the package refuses to import."""
    code = textwrap.dedent(f"""
        import sys
        sys.path.insert(0, {ROOT!r})
        try:
            import paper_2108_02025_gb300
        except ImportError as e:
            print("refused:", e)
    """)
    env = dict(os.environ, GBBLAS_LIB=str(tmp_path / "missing.so"))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=120)
    assert "refused" in r.stdout, (r.stdout, r.stderr)


def test_headers_are_plain_c_and_link_from_c(tmp_path):
    """include/gbblas.h and include/gbserve.h compile as C99 with every
    warning an error, and a C program links against libgbblas.so and calls
    host-only entry points (no device is touched)."""
    import shutil
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use.c"
    src.write_text(textwrap.dedent("""
        #include <stdio.h>
        #include "gbblas.h"
        #include "gbserve.h"
        int main(void) {
          gb_request r = {0};
          r.op = GB_REQ_GEMV; r.m = 10; r.n = 10;
          printf("%d %zu %zu %s\\n", gb_version() > 0,
                 gb_workspace_bytes(GB_OP_GEMV, GB_F64, GB_ROW_MAJOR, -1, 5),
                 gb_engine_request_bytes(&r), gb_status_string(GB_ERR_WORKSPACE) != 0 ? "ok" : "no");
          return 0;
        }
    """))
    inc = os.path.join(ROOT, "include")
    libdir = os.path.dirname(gb.LIB_PATH)
    exe = tmp_path / "use"
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", inc, str(src), "-o", str(exe),
                        "-L", libdir, "-lgbblas", f"-Wl,-rpath,{libdir}"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stderr
    assert out.stdout.split() == ["1", "0", "1024", "ok"]
