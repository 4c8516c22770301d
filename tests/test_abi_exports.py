"""The C-ABI library loads without a GPU and exports every function that
include/pic_gb300.h declares (no compute call is made)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "pic_gb300.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:int|void|char|int64_t)\s*\*?\s*(\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    from paper_1607_04069_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_the_same_functions():
    import paper_1607_04069_gb300 as P
    L = P.lib()
    for n in _declared():
        fn = getattr(L, n)
        assert fn.restype is not None or n.endswith("_destroy")


def test_ctypes_structs_match_the_header(tmp_path):
    """Size and field offsets of every struct the binding mirrors, as the C
    compiler lays them out from include/pic_gb300.h."""
    import shutil
    import subprocess
    import pytest
    import paper_1607_04069_gb300 as P
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    mirrors = {"pic_params": P.PicParams, "tp_source": P.TpSource, "pic_server_opts": P.ServerOpts,
               "pic_request_info": P.RequestInfo, "pic_server_stats": P.ServerStats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pic_gb300.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in mirrors.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def test_missing_library_fails_loudly(monkeypatch):
    """Without the built engine the binding raises instead of falling back
    to anything else: every entry point goes through lib()."""
    import pytest
    import paper_1607_04069_gb300 as P
    monkeypatch.setattr(P, "_lib", None)
    monkeypatch.setattr(P, "LIB_PATH", os.path.join(ROOT, "no-such-dir", "libpic_gb300.so"))
    with pytest.raises(ImportError, match="missing"):
        P.lib()
    with pytest.raises(ImportError):
        P.default_params()


def test_stateless_ops_reject_mismatched_operands():
    """op_sort_noalloc, op_deposit and op_poisson check dtypes, sizes and the
    device before any call into the library: a float64 pos with a float32
    pos_out would have the kernel write 8 bytes into 4-byte slots."""
    import pytest
    torch = pytest.importorskip("torch")
    import paper_1607_04069_gb300 as P
    n = 8
    f32 = lambda: torch.zeros(n, dtype=torch.float32)
    i64 = lambda: torch.zeros(n, dtype=torch.int64)
    pos64 = torch.zeros(n, dtype=torch.float64)
    args = dict(vx=f32(), vy=f32(), vz=f32(), ids=i64(), n_cells=64, vx_out=f32(), vy_out=f32(),
                vz_out=f32(), ids_out=i64())
    with pytest.raises(ValueError, match="pos_out"):
        P.op_sort_noalloc(pos64, pos_out=torch.zeros(n, dtype=torch.float32), **args)
    with pytest.raises(ValueError, match="pos must be"):
        P.op_sort_noalloc(torch.zeros(n, dtype=torch.int64), pos_out=torch.zeros(n, dtype=torch.int64), **args)
    bad = dict(args, ids=torch.zeros(n, dtype=torch.int32))
    with pytest.raises(ValueError, match="ids"):
        P.op_sort_noalloc(pos64, pos_out=torch.zeros(n, dtype=torch.float64), **bad)
    bad = dict(args, vy=torch.zeros(n, dtype=torch.float64))
    with pytest.raises(ValueError, match="vy"):
        P.op_sort_noalloc(pos64, pos_out=torch.zeros(n, dtype=torch.float64), **bad)
    with pytest.raises(ValueError, match="n_out"):
        P.op_sort_noalloc(pos64, pos_out=torch.zeros(n, dtype=torch.float64), n_out=torch.zeros(1), **args)
    with pytest.raises(ValueError, match="room"):
        P.op_sort_noalloc(pos64, pos_out=torch.zeros(n - 1, dtype=torch.float64), **args)
    with pytest.raises(ValueError, match="CUDA"):          # right dtypes, host memory
        P.op_sort_noalloc(pos64, pos_out=torch.zeros(n, dtype=torch.float64), **args)
    with pytest.raises(ValueError, match="contiguous"):
        P.op_sort_noalloc(torch.zeros(2 * n, dtype=torch.float64)[::2], pos_out=pos64.clone(), **args)
    with pytest.raises(ValueError, match="q must"):
        P.op_deposit(torch.zeros(n, dtype=torch.int32), 64, q=torch.zeros(64, dtype=torch.int64))
    with pytest.raises(ValueError, match="q must"):
        P.op_deposit(torch.zeros(n, dtype=torch.int32), 64, q=torch.zeros(65, dtype=torch.float64))
    with pytest.raises(ValueError, match="pos must"):
        P.op_deposit(torch.zeros(n, dtype=torch.float32), 64)
    with pytest.raises(ValueError, match="q_e"):
        P.op_poisson(torch.zeros(65, dtype=torch.int64), torch.zeros(64, dtype=torch.int64), 64, 1e-4, 1.0, 0.0)
