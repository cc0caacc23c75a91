"""CPU checks of the C ABI: the CUDA library builds for sm_103a, loads without a
GPU, exports every function include/sfl.h declares, and the Python ctypes
mirror has the exact C struct layouts.  No compute call is made."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sfl.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*\**\s+\**(s[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2605_22281_gb300 import builder
    path = builder.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("sfl_plan_create", "sfl_plan_destroy", "sflsqr_solve", "sflsmr_solve", "sflsqr_solve_host",
                 "sflsmr_solve_host", "sfl_sketch_export", "sfl_sketch_apply", "sfl_error_string"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_error_strings_without_gpu(lib):
    lib.sfl_error_string.restype = ctypes.c_char_p
    assert lib.sfl_error_string(0) == b"ok"
    assert b"invalid" in lib.sfl_error_string(1)


def test_ctypes_layout_matches_c():
    from paper_2605_22281_gb300 import _native as N
    structs = {"sfl_csr": N.Csr, "sfl_plan_opts": N.PlanOpts, "sfl_opts": N.Opts, "sfl_info": N.Info,
               "sfl_plan_stats": N.PlanStats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "sfl.h"', 'int main(void) {']
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "layout.c")
        exe = os.path.join(d, "layout")
        open(c, "w").write("\n".join(lines))
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for line in out:
        if line.strip():
            cname, field, val = line.split()
            got[(cname, field)] = int(val)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def _fake_tensor(is_cuda=True, dtype="f64", contiguous=True, dim=1, device="cuda:0", numel=100):
    """An object with the tensor attributes the no-alloc argument check reads
    (no CUDA device is needed to build it)."""
    import types

    import torch
    dt = {"f64": torch.float64, "f32": torch.float32}[dtype]
    return types.SimpleNamespace(is_cuda=is_cuda, dtype=dt, is_contiguous=lambda: contiguous, dim=lambda: dim,
                                 device=device, numel=lambda: numel)


def test_noalloc_arguments_are_rejected_before_any_launch():
    """A wrong v or out raises ValueError on the host, before the library is
    loaded or any kernel could write s doubles through a bad pointer."""
    from paper_2605_22281_gb300 import api as G
    ok_v = _fake_tensor()
    G.check_noalloc_args(64, ok_v, None)
    G.check_noalloc_args(64, ok_v, _fake_tensor(numel=64))
    bad = [
        (_fake_tensor(is_cuda=False), None),                 # v on the host
        (_fake_tensor(dtype="f32"), None),                   # v not FP64 (no silent conversion)
        (_fake_tensor(contiguous=False), None),              # v strided
        (ok_v, _fake_tensor(dtype="f32", numel=64)),         # out FP32
        (ok_v, _fake_tensor(numel=63)),                      # out shorter than s
        (ok_v, _fake_tensor(contiguous=False, numel=64)),    # out strided
        (ok_v, _fake_tensor(is_cuda=False, numel=64)),       # out on the host
        (ok_v, _fake_tensor(device="cuda:1", numel=64)),     # out on another device
    ]
    for v, out in bad:
        with pytest.raises(ValueError):
            G.check_noalloc_args(64, v, out)
