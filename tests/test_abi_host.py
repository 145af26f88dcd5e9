"""The C ABI library without a GPU: it builds, loads, exports every entry
point declared in include/rdbayes.h, its struct layout matches the header as
compiled by the host C compiler, invalid descriptions are rejected with
EINVAL before any device work, and without a device it fails loudly
(RD_ECUDA) instead of falling back to the CPU."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_1605_04718_gb300 as rd
from paper_1605_04718_gb300 import build as rdbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rdbayes.h")


@pytest.fixture(scope="module")
def lib():
    rdbuild.build()
    return rd.load()


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^(?:rd_status|const char\*)\s+(rd_\w+)\(", text, re.M)))


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert names and set(names) == set(rd.EXPORTS)
    nm = subprocess.run(["nm", "-D", "--defined-only", rd.LIB_PATH], capture_output=True,
                        text=True, check=True).stdout
    exported = set(re.findall(r"\s[TW]\s+(rd_\w+)$", nm, re.M))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(lib, n)


def test_desc_layout_matches_header(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "rdbayes.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu\\n\", sizeof(rd_problem_desc),"
        " offsetof(rd_problem_desc, tau), offsetof(rd_problem_desc, fixed),"
        " offsetof(rd_problem_desc, step_space), offsetof(rd_problem_desc, w_max));return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    got = list(map(int, subprocess.run([str(exe)], capture_output=True, text=True,
                                       check=True).stdout.split()))
    D = rd.rd_problem_desc
    assert got == [ctypes.sizeof(D), D.tau.offset, D.fixed.offset, D.step_space.offset,
                   D.w_max.offset]


def _valid_desc(**kw):
    args = dict(dim=2, nx=[64], tau=2.5e-4, n_steps=10, param_map=[0, 1, 2, 3],
                fixed=[0.1, 0.9, 10, 200, 0], prior_kind=[rd.RD_PRIOR_LOGNORMAL] * 4,
                prior_p0=[0.1, 0.9, 10, 200], prior_p1=[0.5] * 4, step_space=[rd.RD_STEP_LOG] * 4)
    args.update(kw)
    return rd.make_desc(**args)


@pytest.mark.parametrize("bad", [
    dict(dim=3), dict(nx=[60]), dict(nx=[256]), dict(tau=-1.0), dict(n_steps=0),
    dict(dim=1, nx=[64], precision=rd.RD_PREC_F32), dict(nx=[64, 32, 16, 40]),
    dict(param_map=[0, 0, 2, 3]), dict(prior_p0=[0.1, 0.9, -1, 200]),
    dict(dim=1, nx=[512]), dict(solver=rd.RD_SOLVER_THOMAS),
])
def test_invalid_descriptions_rejected(lib, bad):
    desc = _valid_desc(**bad)
    h = ctypes.c_void_p()
    code = lib.rd_problem_create(ctypes.byref(desc), None, ctypes.byref(h))
    assert code == rd.RD_EINVAL
    assert rd.rd_last_error()


def test_no_device_fails_loudly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    h = ctypes.c_void_p()
    code = lib.rd_problem_create(ctypes.byref(_valid_desc()), None, ctypes.byref(h))
    assert code == rd.RD_ECUDA
    assert "device" in rd.rd_last_error()


def test_null_handles_are_rejected(lib):
    assert lib.rd_set_initial_state(None, 0, None, None) == rd.RD_EINVAL
    assert lib.rd_evaluate_batch(None, 1, None, None, None, None, None) == rd.RD_EINVAL
    assert lib.rd_chains_run(None, 1) == rd.RD_EINVAL
    assert lib.rd_sync(None) == rd.RD_EINVAL
