"""Host-side checks of the C ABI: the library builds, loads, exports every symbol
that include/*.h declares, and rejects bad arguments before touching a GPU."""
import ctypes
import glob
import os
import re

import pytest

from oracle.radic_oracle import is_prime
from tests.conftest import ROOT


@pytest.fixture(scope="module")
def lib():
    from paper_1508_01326_gb300 import build as B
    from paper_1508_01326_gb300 import _lib as L

    B.build()
    return L.lib()


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(radic_[a-z0-9_]+)\s*\(", text):
            names.append(m.group(1))
    return sorted(set(names))


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ["radic_det", "radic_terms", "radic_unrank", "radic_workspace_bytes", "radic_primes"]:
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_struct_layouts_match_header(tmp_path):
    # The binding's ctypes structures against the header compiled as C: the
    # offset of every field and the size of every structure.
    import shutil
    import subprocess

    from paper_1508_01326_gb300 import _lib as L

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"radic_options": L.RadicOptions, "radic_batch_tuning": L.RadicBatchTuning}
    lines = ['#include <stdio.h>', '#include "radic.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append('  printf("radic_result size %zu\\n", sizeof(radic_result));')
    for fname in ["value", "abs_sum", "err_bound", "exact_lo", "exact_hi", "minors", "flagged", "status", "n_primes",
                  "tier", "exact_exp"]:
        lines.append(f'  printf("radic_result {fname} %zu\\n", offsetof(radic_result, {fname}));')
    lines.append("  return 0;\n}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-x", "c", "-std=c11", f"-I{os.path.join(ROOT, 'include')}", str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    got = {}
    for row in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        sname, field, value = row.split()
        got[(sname, field)] = int(value)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
    # the binding reads radic_result as 16 eight-byte words (parse_result)
    assert got[("radic_result", "size")] == 8 * L.RESULT_WORDS
    order = ["value", "abs_sum", "err_bound", "exact_lo", "exact_hi", "minors", "flagged", "status", "n_primes", "tier",
             "exact_exp"]
    for word, fname in enumerate(order):
        assert got[("radic_result", fname)] == 8 * word, fname


def test_host_only_calls(lib):
    assert lib.radic_version() >= 10000
    assert lib.radic_status_string(0) == b"ok"
    assert lib.radic_status_string(1) == b"invalid argument"
    buf = (ctypes.c_uint32 * 4)()
    assert lib.radic_primes(buf, 4) == 4
    primes = list(buf)
    assert len(set(primes)) == 4
    for p in primes:
        assert is_prime(p) and (1 << 30) < p < (1 << 31)


def test_invalid_arguments_rejected_without_gpu(lib):
    from paper_1508_01326_gb300 import _lib as L

    dummy = ctypes.c_void_p(0x1000)
    # NULL matrix
    assert lib.radic_det(None, 3, 5, 5, 3, 0, None, dummy, dummy, 1 << 20, None) == 1
    # lda < n
    assert lib.radic_det(dummy, 3, 5, 4, 3, 0, None, dummy, dummy, 1 << 20, None) == 1
    # per-term exact residues of a real dtype (radic_det takes real inputs in
    # the exact mode, radic_terms does not)
    assert lib.radic_terms(dummy, 3, 5, 5, 3, 2, None, 0, 1, dummy, None) == 1
    # unknown dtype, unknown mode
    assert lib.radic_det(dummy, 3, 5, 5, 9, 0, None, dummy, dummy, 1 << 20, None) == 1
    assert lib.radic_det(dummy, 3, 5, 5, 3, 7, None, dummy, dummy, 1 << 20, None) == 1
    # sizes out of range
    for m, n in [(0, 5), (3, 0), (33, 40), (3, 65)]:
        assert lib.radic_det(dummy, m, n, max(n, 1), 3, 0, None, dummy, dummy, 1 << 20, None) == 1
    # unrank: rank range outside [0, C(n, m))
    assert lib.radic_unrank(8, 5, 56, 1, dummy, None, None) == 1
    assert lib.radic_unrank(8, 5, 50, 7, dummy, None, None) == 1
    assert lib.radic_unrank(8, 9, 0, 1, dummy, None, None) == 1
    assert lib.radic_terms(dummy, 5, 8, 8, 3, 0, None, 0, 57, dummy, None) == 1
    opts = L.make_options(mapping="thread")
    assert lib.radic_workspace_bytes(0, 8, 0, ctypes.byref(opts)) == 0
