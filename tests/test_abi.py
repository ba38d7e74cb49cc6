"""The C-ABI library builds for sm_103a and exports every entry point that
include/hbperm.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import shutil

import pytest

from paper_2605_08048_gb300 import hbperm as H


@pytest.fixture(scope="module")
def built():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no CUDA toolkit")
    from paper_2605_08048_gb300 import build
    return build.build()


def test_exports_every_declared_symbol(built):
    names = H.declared_symbols()
    assert {"hb_align", "hb_perm_test", "hb_perm_test_batched", "hb_perm_labels"} <= set(names)
    lib = ctypes.CDLL(built)
    missing = [s for s in names if not hasattr(lib, s)]
    assert not missing


def test_header_struct_layouts_match_binding(tmp_path):
    """sizeof/offsetof of the header's structs, compiled by the C compiler,
    equal the ctypes mirrors of the binding."""
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = tmp_path / "layout.c"
    fields_o = [f for f, _ in H.hb_opts._fields_]
    fields_r = [f for f, _ in H.hb_result._fields_]
    fields_l = [f for f, _ in H.hb_layout_counts._fields_]
    body = ['#include <stdio.h>', '#include <stddef.h>', '#include "hbperm.h"', "int main(void){",
            'printf("%zu %zu %zu\\n", sizeof(hb_opts), sizeof(hb_result), sizeof(hb_layout_counts));']
    body += [f'printf("%zu\\n", offsetof(hb_opts, {f}));' for f in fields_o]
    body += [f'printf("%zu\\n", offsetof(hb_result, {f}));' for f in fields_r]
    body += [f'printf("%zu\\n", offsetof(hb_layout_counts, {f}));' for f in fields_l]
    body += ["return 0;}"]
    src.write_text("\n".join(body))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(root, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    vals = [int(v) for v in out]
    assert vals[0] == ctypes.sizeof(H.hb_opts) and vals[1] == ctypes.sizeof(H.hb_result)
    assert vals[2] == ctypes.sizeof(H.hb_layout_counts)
    offs = [getattr(H.hb_opts, f).offset for f in fields_o] + [getattr(H.hb_result, f).offset for f in fields_r]
    offs += [getattr(H.hb_layout_counts, f).offset for f in fields_l]
    assert vals[3:] == offs


def test_binding_refuses_without_library(tmp_path, monkeypatch):
    monkeypatch.setattr(H, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(H, "_lib", None)
    with pytest.raises(RuntimeError):
        H.lib()


def test_results_array_mirrors_hb_result():
    """The structured numpy type of batched results has hb_result's layout,
    and Results gives the same dicts as hb_result.as_dict on the same bytes."""
    assert H.RESULT_DTYPE.itemsize == ctypes.sizeof(H.hb_result)
    for k, _ in H.hb_result._fields_:
        assert H.RESULT_DTYPE.fields[k][1] == getattr(H.hb_result, k).offset
    arr = H.np.zeros(3, dtype=H.RESULT_DTYPE)
    arr["p"] = [0.5, 0.25, 1.0]
    arr["count"] = [4, 7, 2**40]
    arr["status"] = [0, 3, -1]
    arr["band_max"] = [1e-9, 0.0, 2.5]
    view = (H.hb_result * 3).from_buffer(arr)
    res = H.Results(arr)
    assert len(res) == 3
    assert [r for r in res] == [v.as_dict() for v in view]
    assert res[1:] == [view[1].as_dict(), view[2].as_dict()]
    assert list(res.column("count")) == [4, 7, 2**40]
    assert res == H.Results(arr.copy()) and res == [v.as_dict() for v in view]
    other = arr.copy()
    other["count"][2] += 1
    assert res != H.Results(other)


def test_binding_checks_shapes_before_calling_the_library():
    """The library reads sum(n + m) rows from the pointer it is given, so the
    binding rejects a packed tensor of another row count, size lists of
    different lengths, and pairs whose X and Y differ in dtype or dimension,
    before any call (no context or GPU is needed to see the error)."""
    torch = pytest.importorskip("torch")
    o = H.make_opts(B=99)
    XY = torch.zeros((30, 16), dtype=torch.bfloat16)
    with pytest.raises(ValueError, match="rows"):
        H.hb_perm_test_batched(None, XY, [10, 5], [10, 4], o)
    with pytest.raises(ValueError, match="one entry per pair"):
        H.hb_perm_test_batched(None, XY, [10, 5], [15], o)
    with pytest.raises(ValueError, match="2-D"):
        H.hb_perm_test_batched(None, XY.reshape(-1), [10, 5], [10, 5], o)
    with pytest.raises(ValueError, match="contiguous"):
        H.hb_perm_test_batched(None, torch.zeros((16, 30), dtype=torch.bfloat16).t(), [10, 5], [10, 5], o)
    X, Y = torch.zeros((4, 16)), torch.zeros((5, 8))
    for call in (lambda: H.hb_perm_test(None, X, Y, o), lambda: H.hb_align(None, X, Y),
                 lambda: H.hb_align_noalloc(X, Y)):
        with pytest.raises(ValueError, match="dimension"):
            call()
    with pytest.raises(ValueError, match="dtype"):
        H.hb_perm_test(None, X, torch.zeros((5, 16), dtype=torch.bfloat16), o)
