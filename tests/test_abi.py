"""The C ABI without a GPU: libpdlp.so loads, exports every function include/pdlp.h
declares, and the ctypes structures match the C layout (checked against a gcc-built
offsetof probe of the header)."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pdlp.h")


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pdlp_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2501_07018_gb300 import binding

    if not os.path.exists(binding.LIB_PATH):
        import __graft_entry__

        __graft_entry__.build()
    return binding.load_library()


def test_exports_every_declared_symbol(lib):
    names = _declared_functions()
    assert {"pdlp_solve", "pdlp_params_default", "pdlp_last_error"} <= set(names)
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (pdlp_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(lib, n)


def test_struct_layout_matches_header(lib):
    from paper_2501_07018_gb300 import binding

    fields = {
        "pdlp_params": [f for f, _ in binding.Params._fields_],
        "pdlp_stats": [f for f, _ in binding.Stats._fields_],
        "pdlp_csr": [f for f, _ in binding.Csr._fields_],
        "pdlp_problem": [f for f, _ in binding.Problem._fields_],
        "pdlp_unrolled_problem": [f for f, _ in binding.UnrolledProblem._fields_],
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void){"]
    for st, fs in fields.items():
        lines.append(f'printf("{st} size %zu\\n", sizeof({st}));')
        for f in fs:
            lines.append(f'printf("{st} {f} %zu\\n", offsetof({st}, {f}));')
    lines.append("return 0;}")
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "probe.c")
        exe = os.path.join(d, "probe")
        open(c, "w").write("\n".join(lines))
        subprocess.run(["gcc", "-std=c99", "-o", exe, c], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    got = {}
    for line in out.splitlines():
        st, f, v = line.split()
        got[(st, f)] = int(v)
    for st, cls in (("pdlp_params", binding.Params), ("pdlp_stats", binding.Stats),
                    ("pdlp_csr", binding.Csr), ("pdlp_problem", binding.Problem),
                    ("pdlp_unrolled_problem", binding.UnrolledProblem)):
        assert got[(st, "size")] == ctypes.sizeof(cls), st
        for f, _ in cls._fields_:
            assert got[(st, f)] == getattr(cls, f).offset, (st, f)


def test_params_default_values(lib):
    from paper_2501_07018_gb300 import binding

    p = binding.default_params()
    assert p.eps_rel_kkt == 1e-8 and p.ruiz_iters == 10 and p.pc_alpha == 1.0
    assert p.check_period == 64 and p.beta_suff == 0.1 and p.beta_nec == 0.9
    assert p.beta_art == 0.5 and p.theta == 0.5 and p.eps_zero == 1e-10
    assert p.precision == 0 and p.inputs_on_device == 0


def test_binding_constants_match_header(lib):
    from paper_2501_07018_gb300 import binding

    defs = dict(re.findall(r"#define\s+(PDLP_\w+)\s+\(?(-?\d+)\)?", open(HEADER).read()))
    assert int(defs["PDLP_TRACE_HEADER"]) == binding.TRACE_HEADER
    assert int(defs["PDLP_POLISH_LOG_COLS"]) == binding.POLISH_LOG_COLS
    assert int(defs["PDLP_FP32_BULK"]) == binding.FP32_BULK and int(defs["PDLP_FP64"]) == binding.FP64
    for code, name in binding.STATUS_NAMES.items():
        key = {"INVALID_ARGUMENT": "PDLP_INVALID_ARGUMENT", "OUT_OF_MEMORY": "PDLP_OUT_OF_MEMORY",
               "CUDA_ERROR": "PDLP_CUDA_ERROR"}.get(name, "PDLP_" + name)
        assert int(defs[key]) == code, name
    p = binding.default_params()
    assert p.feasibility_polishing == 0 and p.polish_log_cap == 0 and not p.polish_log
    assert p.detect_infeasibility == 1 and p.eps_infeas == 1e-9 and p.reduced_costs == 0
