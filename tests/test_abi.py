"""The C-ABI library loads and exports every declared symbol; argument checks
that run before any device work (no compute calls, no GPU needed)."""
import ctypes as C
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent


@pytest.fixture(scope="module")
def lib():
    from paper_2512_06715_gb300 import build
    build.build()
    from paper_2512_06715_gb300 import pdhg
    return pdhg.lib()


def _declared(header: str) -> list[str]:
    text = (ROOT / "include" / header).read_text()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)   # comments are not declarations
    text = re.sub(r"//[^\n]*", " ", text)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?(?:\w+\s+)+\**\s*(\w+)\s*\(", text, re.M)))


def test_every_declared_symbol_is_exported(lib):
    from paper_2512_06715_gb300 import pdhg
    names = _declared("pdhg.h")
    assert "pdhg_solve" in names and "pdhg_solve_batched" in names and "pdhg_backward" in names
    for name in names:
        assert hasattr(lib, name), name
        assert name in pdhg._SIGS, f"{name} has no Python signature"
    gen = C.CDLL(str(ROOT / "paper_2512_06715_gb300" / "lib" / "libucgen.so"))
    for name in _declared("uc_lp.h"):
        assert hasattr(gen, name), name


def test_opts_default(lib):
    from paper_2512_06715_gb300 import pdhg
    o = pdhg.default_opts()
    assert o.tol == 1e-8 and o.check_every == 64 and o.ruiz_iters == 10
    assert o.beta_sufficient == 0.2 and o.beta_necessary == 0.8 and o.beta_artificial == 0.36
    assert o.precision == pdhg.PREC_FP64
    assert o.kernel_variant == -1 and o.kernel_grid == 0 and o.autotune == 1
    assert o.infeas_tol == 1e-8 and o.ir_fold_checks == 16 and o.launch_overlap == 0


def test_invalid_arguments_rejected_on_host(lib):
    from paper_2512_06715_gb300 import pdhg
    ws = C.c_void_p()
    assert lib.pdhg_workspace_create(None, None, C.byref(ws), None) == -1
    assert b"NULL" in lib.pdhg_last_error()
    prob = pdhg.pdhg_problem(0, 5, 0, 0, 1, 1, 1, 1, 1, 1, 1)
    assert lib.pdhg_workspace_create(C.byref(prob), None, C.byref(ws), None) == -1
    prob = pdhg.pdhg_problem(5, 5, 7, 0, 1, 1, 1, 1, 1, 1, 1)  # m_eq > m
    assert lib.pdhg_workspace_create(C.byref(prob), None, C.byref(ws), None) == -1
    prob = pdhg.pdhg_problem(1 << 31, 5, 0, 0, 1, 1, 1, 1, 1, 1, 1)
    assert lib.pdhg_workspace_create(C.byref(prob), None, C.byref(ws), None) == -5
    o = pdhg.default_opts()
    o.check_every = 32
    prob = pdhg.pdhg_problem(5, 5, 0, 5, 1, 1, 1, 1, 1, 1, 1)
    assert lib.pdhg_workspace_create(C.byref(prob), C.byref(o), C.byref(ws), None) == -5
    o = pdhg.default_opts()
    o.precision = 7
    assert lib.pdhg_workspace_create(C.byref(prob), C.byref(o), C.byref(ws), None) == -1
    for field, bad in (("kernel_variant", 3), ("kernel_variant", -2), ("kernel_variant", 22), ("kernel_grid", -1),
                       ("kernel_grid", 8193), ("launch_overlap", 2), ("ir_fold_checks", -1)):
        o = pdhg.default_opts()
        setattr(o, field, bad)
        assert lib.pdhg_workspace_create(C.byref(prob), C.byref(o), C.byref(ws), None) == -1
    assert lib.pdhg_solve(None, None, None, None, None) == -1
    assert not ws.value


def test_generator_rejects_bad_sizes():
    from paper_2512_06715_gb300.instances import build_instance
    with pytest.raises(ValueError, match="n_line"):
        build_instance(4, 2, 3, 3)
