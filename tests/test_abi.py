"""CPU checks of the C-ABI boundary: the library builds, loads, exports every symbol that
include/uaamg.h declares, and refuses to compute without a GPU (no CPU fallback)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    from paper_1302_2547_gb300 import build as B

    return B.build()


def _declared():
    text = open(os.path.join(ROOT, "include", "uaamg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(uaamg_[A-Za-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("uaamg_setup", "uaamg_solve", "uaamg_free"):
        assert must in names


def test_library_exports_every_declared_symbol(built):
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\bT (uaamg_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    from paper_1302_2547_gb300 import _lib as U

    assert set(U.EXPORTS) == set(_declared())
    L = ctypes.CDLL(built)
    for n in _declared():
        getattr(L, n)


def test_default_params_and_status_strings(built):
    from paper_1302_2547_gb300 import _lib as U

    p = U.uaamg_default_params()
    assert (p.coarse_size, p.max_levels, p.max_agg_size, p.pass_mode) == (64, 25, 5, 1)
    assert (p.pre, p.post, p.kcycle_inner, p.precision, p.max_iter) == (1, 1, 2, 1, 200)
    assert p.sra_rounds == 0
    assert U.status_string(0) == "ok" and "CSR" in U.status_string(2)


def test_params_are_checked_before_any_device_work(built):
    from paper_1302_2547_gb300 import _lib as U
    from paper_1302_2547_gb300 import inputs as I

    A = I.grid2d(8)
    for bad in ({"max_agg_size": 1}, {"kcycle_inner": 3}, {"precision": 7},
                {"max_levels": 0}, {"pass_mode": 4}, {"pre": -1}, {"sra_rounds": -1},
                {"sra_rounds": 65}, {"profile_class": 6}, {"wait_limit_ns": -1}):
        with pytest.raises(U.UaamgError) as e:
            U.uaamg_setup(A.rowptr, A.col, A.val, U.uaamg_default_params(**bad))
        assert e.value.status == 1


def test_no_cpu_fallback_without_a_gpu(built):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1302_2547_gb300 import _lib as U
    from paper_1302_2547_gb300 import inputs as I

    A = I.grid2d(8)
    with pytest.raises(U.UaamgError) as e:
        U.uaamg_setup(A.rowptr, A.col, A.val)
    assert e.value.status == 7  # UAAMG_ERR_CUDA


def test_product_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_1302_2547_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                for pat in (r"^\s*(from|import)\s+oracle\b", r"liboracle", r"oracle/",
                            r"uaamg_oracle"):
                    assert not re.search(pat, text, flags=re.M), (f, pat)


def test_binding_constants_match_the_header():
    """Every UAAMG_* constant that the Python binding restates has the header's value."""
    from paper_1302_2547_gb300 import _lib as U

    text = open(os.path.join(ROOT, "include", "uaamg.h")).read()
    defs = {m.group(1): int(m.group(2))
            for m in re.finditer(r"#define\s+(UAAMG_\w+)\s+(-?\d+)", text)}
    restated = [n for n in dir(U) if n.startswith("UAAMG_")]
    assert len(restated) >= 10
    for name in restated:
        assert name in defs, name
        assert getattr(U, name) == defs[name], name


def test_binding_structs_match_the_c_layout(tmp_path):
    """The ctypes mirrors of uaamg_csr, uaamg_params and uaamg_stats have the C layout:
    a probe compiled against include/uaamg.h prints every field's offset and the size."""
    from paper_1302_2547_gb300 import _lib as U

    structs = {"uaamg_csr": U.uaamg_csr, "uaamg_params": U.uaamg_params,
               "uaamg_stats": U.uaamg_stats, "uaamg_answer": U.uaamg_answer}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "uaamg.h"',
             'int main(void) {']
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ['  return 0;', '}']
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "probe"
    subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src),
                           "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    got = {}
    for line in out.splitlines():
        cname, key, val = line.split()
        got[(cname, key)] = int(val)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def test_binding_structs_have_every_header_field():
    """Field names and order of the ctypes mirrors equal the header's declarations (a field
    missing at the end could hide in the padding of the size check)."""
    from paper_1302_2547_gb300 import _lib as U

    text = open(os.path.join(ROOT, "include", "uaamg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    for cname, py in (("uaamg_csr", U.uaamg_csr), ("uaamg_params", U.uaamg_params),
                      ("uaamg_stats", U.uaamg_stats), ("uaamg_answer", U.uaamg_answer)):
        body = re.search(r"typedef struct %s \{(.*?)\} %s;" % (cname, cname), text, re.S).group(1)
        names = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            # "const int32_t* rowptr" / "int32_t pre, post": the declarators follow the type
            parts = [p.strip() for p in decl.split(",")]
            names.append(re.findall(r"(\w+)\s*$", parts[0])[0])
            names += [re.findall(r"(\w+)\s*$", p)[0] for p in parts[1:]]
        assert names == [f for f, _ in py._fields_], cname


def test_static_aggregation_wrapper_rejects_bad_arguments(built):
    """The binding of uaamg_aggregate_static checks dtypes, lengths and the device of every
    array before the C call, which cannot see the length of a device buffer (CPU only: every
    case here is refused before any device work)."""
    import torch

    from paper_1302_2547_gb300 import _lib as U

    n = 6
    rp = torch.arange(n + 1, dtype=torch.int32)
    cc = torch.arange(n, dtype=torch.int32)
    vv = torch.ones(n, dtype=torch.float64)
    ag = torch.zeros(n, dtype=torch.int32)
    bad = [((rp.long(), cc, vv, ag), "rowptr must be int32"),
           ((rp, cc.long(), vv, ag), "col must be int32"),
           ((rp, cc, vv.float(), ag), "val must be float64"),
           ((rp, cc, vv, ag.long()), "agg must be int32"),
           ((rp, cc, vv, ag[: n - 1]), "fewer than n"),
           ((rp, cc[: n - 1], vv, ag), "same length"),
           ((rp[:1], cc, vv, ag), "n + 1 >= 2"),
           ((rp.numpy(), cc, vv, ag), "CUDA tensors only (rowptr)"),
           ((rp, cc, vv, ag), "CUDA tensors only")]
    for args, msg in bad:
        with pytest.raises(ValueError, match=re.escape(msg)):
            U.uaamg_aggregate_static(*args)
