"""The allocation-free rescaling entry point (pdhg_rescale_noalloc).

It serves callers that cannot call cudaMalloc -- code running where another
framework's caching allocator owns the device memory, code with a memory
budget fixed up front, or code that must not risk an allocation's implicit
synchronisation.  Its only scratch is a fixed file-scope device array, so this
test checks, through the C ABI, that two calls in a row give the same factors
as the workspace path (pdhg_prepare + pdhg_get_scaling), and that a problem
larger than the fixed scratch is refused before any device work.

The file is named to be collected last, so a run that stops at the first
failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2512_06715_gb300.instances import workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_06715_gb300 import build
    build.build()


@pytest.mark.parametrize("name", ["uc24_g33_T24", "uc4224_g600_T24"])
def test_noalloc_rescaling_matches_workspace(name):
    from paper_2512_06715_gb300 import pdhg
    inst = workload(name)
    ws = pdhg.Workspace.from_instance(inst, pdhg.default_opts())
    ws.prepare()
    Dr_ref, Dc_ref = (t.cpu().numpy() for t in ws.scaling())
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):  # the shared scratch keeps the previous call's contents
        Dr = torch.full((inst.m,), np.nan, dtype=torch.float64, device="cuda")
        Dc = torch.full((inst.n,), np.nan, dtype=torch.float64, device="cuda")
        rc = pdhg.lib().pdhg_rescale_noalloc(C.byref(ws.prob), 10, 1, Dr.data_ptr(), Dc.data_ptr(),
                                             stream)
        assert rc == 0, pdhg.lib().pdhg_last_error()
        torch.cuda.synchronize()
        assert np.allclose(Dr.cpu().numpy(), Dr_ref, rtol=1e-12, atol=0)
        assert np.allclose(Dc.cpu().numpy(), Dc_ref, rtol=1e-12, atol=0)
    ws.close()


def test_noalloc_rejects_too_many_columns():
    from paper_2512_06715_gb300 import pdhg
    big = pdhg.pdhg_problem((1 << 21) + 1, 10, 0, 0, 1, 1, 1, 0, 0, 0, 0)
    Dr = torch.empty(10, dtype=torch.float64, device="cuda")
    rc = pdhg.lib().pdhg_rescale_noalloc(C.byref(big), 10, 1, Dr.data_ptr(), Dr.data_ptr(), None)
    assert rc == -5
    assert b"exceeds the fixed scratch" in pdhg.lib().pdhg_last_error()
