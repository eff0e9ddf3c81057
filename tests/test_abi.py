"""The C-ABI library builds, loads, and exports every symbol its header
declares; host-side argument checks answer without a GPU."""
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def rq():
    import paper_2605_16007_gb300 as rq

    rq.build()
    return rq


def declared_functions():
    src = open(os.path.join(ROOT, "include", "rq.h")).read()
    return re.findall(r"^RQ_API\s+[\w\s\*]+?\b(rq_\w+)\s*\(", src, flags=re.M)


def test_header_declares_the_api():
    names = declared_functions()
    for must in ("rq_build", "rq_search", "rq_search_mixed", "rq_free", "rq_export",
                 "rq_import", "rq_server_create", "rq_submit", "rq_wait"):
        assert must in names


def test_every_declared_symbol_is_exported(rq):
    out = subprocess.run(["nm", "-D", "--defined-only", rq.LIB], capture_output=True,
                         text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    lib = rq.lib()
    for n in declared_functions():
        assert hasattr(lib, n)


def test_status_strings_and_version(rq):
    assert rq.rq_status_str(0) == "ok"
    assert rq.rq_status_str(rq.RQ_ERR_INVALID_ARG) == "invalid argument"
    assert rq.rq_version() >= 10000


@pytest.mark.parametrize("n,dim,nlist", [(10, 8, 11), (10, 0, 2), (10, 5000, 2), (0, 8, 1)])
def test_build_rejects_bad_sizes_on_host(rq, n, dim, nlist):
    base = np.zeros((max(n, 1), max(dim, 1)), np.float32)
    lib = rq.lib()
    import ctypes as C

    h = C.c_void_p()
    st = lib.rq_build(rq._ptr(base), 0, n, dim, nlist, 0, None, C.byref(h))
    assert st == rq.RQ_ERR_INVALID_ARG
    assert lib.rq_last_error().decode()


def test_search_rejects_null_index(rq):
    lib = rq.lib()
    st = lib.rq_search(None, None, 1, 1, 1, 1, None, None, None, None)
    assert st == rq.RQ_ERR_INVALID_ARG


def test_import_rejects_foreign_file(rq, tmp_path):
    p = tmp_path / "junk.bin"
    p.write_bytes(b"NOPE" + b"\0" * 64)
    with pytest.raises(rq.RQError) as e:
        rq.rq_import(str(p))
    assert e.value.status == rq.RQ_ERR_IO
    with pytest.raises(rq.RQError) as e:
        rq.rq_import(str(tmp_path / "missing.bin"))
    assert e.value.status == rq.RQ_ERR_IO
