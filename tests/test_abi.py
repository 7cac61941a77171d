"""The C ABI: the library builds for sm_103a, loads, and exports every entry
point that include/pmcim.h declares. No compute call is made here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pmcim.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pmcim_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2312_13117_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_library_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name


def test_binding_names_match_header():
    from paper_2312_13117_gb300 import pmcim
    assert sorted(pmcim.EXPORTS) == _declared()


def test_status_strings_and_defaults(lib):
    from paper_2312_13117_gb300 import pmcim
    pmcim.load()
    o = pmcim.pmcim_default_options()
    assert (o.tol_ind, o.tol_svd, o.tol_verify) == (0.1, 1e-6, 1e-6)
    assert o.max_split_depth == 8 and o.precision == pmcim.PREC_FP64
    assert o.tol_ir == 1e-11 and o.indicator_N == 0 and o.max_ir_sweeps == 6
    # the binding's struct has the header's size: the last field lands where the library writes it
    assert ctypes.sizeof(pmcim.pmcim_options) == pmcim.pmcim_options.fp64_tile.offset + 4
    assert o.residual_fp64 == 0 and o.fp64_tile == 0
    lib.pmcim_status_string.restype = ctypes.c_char_p
    assert lib.pmcim_status_string(-5) == b"output capacity exceeded"


def test_no_cpu_fallback_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import numpy as np
    from paper_2312_13117_gb300 import pmcim
    with pytest.raises(pmcim.PmcimError) as e:
        pmcim.Problem(4, [(np.eye(4), 0, 0, 0.0)])
    assert e.value.code == -3  # PMCIM_ECUDA


def test_debug_wait_limits_reject_negative(lib):
    """The wait-limit setter validates on the host (no device call)."""
    from paper_2312_13117_gb300 import pmcim
    pmcim.load()
    with pytest.raises(pmcim.PmcimError) as e:
        pmcim.debug_wait_limits(-1, 0)
    assert e.value.code == -1   # PMCIM_EINVAL
    pmcim.debug_wait_limits(0, 0)


def test_term_kinds_match_header():
    """The scalar-function kinds, the boundary-integral term's included, agree between the header, the
    binding, the input generators and the oracle."""
    src = open(os.path.join(ROOT, "include", "pmcim.h")).read()
    kinds = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define PMCIM_F_(\w+)\s+(\d+)", src)}
    assert kinds == {"MONOMIAL": 0, "EXP_NEG": 1, "HELMHOLTZ_DLP": 2}
    from paper_2312_13117_gb300 import pmcim
    import oracle
    import workloads
    assert (pmcim.F_MONOMIAL, pmcim.F_EXP_NEG, pmcim.F_HELMHOLTZ_DLP) == (0, 1, 2)
    assert (workloads.MONOMIAL, workloads.EXP_NEG, workloads.HELMHOLTZ_DLP) == (0, 1, 2)
    assert (oracle.MONOMIAL, oracle.EXP_NEG, oracle.HELMHOLTZ_DLP) == (0, 1, 2)


def test_no_cpu_fallback_for_boundary_terms_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import workloads as w
    from paper_2312_13117_gb300 import pmcim
    W = w.scattering_disk(n=16, l=2)
    with pytest.raises(pmcim.PmcimError) as e:
        pmcim.Problem(W.problem.n, W.problem.terms)
    assert e.value.code == -3  # PMCIM_ECUDA


def test_header_compiles_as_c99_and_cxx(tmp_path):
    """include/pmcim.h is a plain C header: it compiles with -std=c99 -pedantic and as C++."""
    import shutil
    import subprocess
    src = tmp_path / "use_header.c"
    src.write_text('#include "pmcim.h"\n'
                   "int main(void) {\n"
                   "  pmcim_options o;\n"
                   "  pmcim_default_options(&o);\n"
                   "  pmcim_fterm f = {PMCIM_F_HELMHOLTZ_DLP, 0, 0.0, 0.5, 0.0};\n"
                   "  (void)f;\n"
                   "  return o.precision;\n"
                   "}\n")
    inc = "-I" + os.path.join(ROOT, "include")
    for cc, flags in (("gcc", ["-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror"]),
                      ("g++", ["-std=c++11", "-Wall", "-Werror", "-x", "c++"])):
        if not shutil.which(cc):
            pytest.skip(cc + " not found")
        subprocess.run([cc, *flags, "-fsyntax-only", inc, str(src)], check=True)
