"""The allocation-free entry point dvbe_conserved_noalloc, checked against
dvbe_conserved.

It exists for callers that cannot let a library allocate device memory
(a framework that has reserved the GPU's memory for its own pool, or a
time-critical loop where cudaMalloc / cudaFree must not run).  The test
allocates its input and output buffers itself (through torch, as such a
caller would), calls the entry point twice in a row through the C ABI and
compares both results with the allocating entry point.  This file is named
to be collected last.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    from paper_1511_00242_gb300 import build
    build.build()
    import paper_1511_00242_gb300 as dv
    if not torch.cuda.is_available():
        pytest.fail("CUDA is not available")
    return torch, dv


@pytest.mark.parametrize("precision", ["f64", "f32", "bf16_dev"])
def test_noalloc_conserved_matches_allocating_call(env, precision):
    torch, dv = env
    case, fields = W.cavity(70, Re=300, stretch_beta=1.3)
    (rho, ux, uy), _ = W.random_state(case, 11)
    with dv.Solver(case, precision=precision) as s:
        s.init_equilibrium(rho, ux, uy)
        s.step(7)
        ref = s.conserved()
        ptr, pitch, plane, eb = s.device_state()
        assert plane == pitch * case["ny"]
        dx = torch.tensor(np.diff(case["xf"]), dtype=torch.float64, device="cuda")
        dy = torch.tensor(np.diff(case["yf"]), dtype=torch.float64, device="cuda")
        for _ in range(2):  # two calls in a row share the scratch array
            out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
            dv.dvbe_conserved_noalloc(ptr, precision, case["nx"], case["ny"], pitch, dx.data_ptr(),
                                      dy.data_ptr(), case["RT"], 1.0, 0.0, out.data_ptr())
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-15 * abs(ref[0]))


def test_noalloc_rejects_meshes_beyond_its_scratch(env):
    torch, dv = env
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    dummy = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(dv.DvbeError) as e:
        dv.dvbe_conserved_noalloc(dummy.data_ptr(), "f32", 8193, 4096, 8200, dummy.data_ptr(),
                                  dummy.data_ptr(), W.RT_LATTICE, 1.0, 0.0, out.data_ptr())
    assert e.value.status == dv.DVBE_ERR_INVALID_ARG
    assert "cells" in str(e.value)
