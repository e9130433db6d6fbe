"""wl_forces_noalloc, the allocation-free variant of the pressure-force reduction.

Some callers cannot allocate device memory where they need the force (for example
inside a CUDA-graph capture, where cudaMalloc is not allowed, or under an allocator
that owns the whole device).  This entry point takes the pressure and face
coefficients they already hold and keeps its scratch in a fixed device array.  Each
test calls it twice in a row through the C ABI (the second call reuses the array
the first one left behind) and checks it against wl_forces on the same state.  With
precision 0 both read the same FP32 pressure and sum it in FP64 in different orders, so
they agree to FP64 rounding (bar 1e-10 relative).  With the default double-float
pressure (precision 1) the caller's FP32 pressure is that pressure rounded to FP32 (what
wl_get_field returns), so the results differ by that rounding (bar 1e-4 relative, the
force bar of the parity tests).
This file is collected last so that a run stopping at the first failure has already
run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CASES = [
    dict(dims=(128, 64), nu=0.064, U=(1.0, 0.0), body=dict(kind=1, center=(32.0, 32.0), radius=8.0), periodic=0),
    dict(dims=(96, 48, 48), nu=0.02, U=(1.0, 0.0, 0.0), body=dict(kind=1, center=(30.0, 24.3, 23.6), radius=7.0),
         periodic=4),
]


@pytest.mark.parametrize("precision", [0, 1], ids=["fp32_pressure", "double_float_pressure"])
@pytest.mark.parametrize("case", CASES, ids=["cylinder2d", "sphere3d"])
def test_forces_noalloc_matches_wl_forces(case, precision):
    import torch

    from paper_2304_08159_gb300 import Sim, wl

    # precision 0: the FP32 pressure wl_get_field returns is the one wl_forces reads;
    # precision 1 (the default): wl_forces reads ph + pl, the caller holds it rounded to FP32
    sim = Sim(case["dims"], case["nu"], case["U"], body=case["body"], periodic=case["periodic"],
              precision=precision)
    sim.step(4)
    torch.cuda.synchronize()
    ref = sim.forces()
    assert np.abs(ref).max() > 0.0
    p = sim.get(wl.WL_FIELD_P, device=True).contiguous()
    L = sim.get(wl.WL_FIELD_MU0, device=True).contiguous()
    D = len(case["dims"])
    F = torch.empty(D, dtype=torch.float64, device=p.device)
    body = wl.make_body(case["body"])
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        F.fill_(float("nan"))
        rc = wl.wl_forces_noalloc(case["dims"], case["periodic"], body, 1.0, p.data_ptr(), L.data_ptr(),
                                  F.data_ptr(), stream)
        assert rc == wl.WL_OK
        torch.cuda.synchronize()
        got = F.cpu().numpy()
        assert np.all(np.isfinite(got))
        dev = np.abs(got - ref).max() / np.abs(ref).max()
        print(f"wl_forces_noalloc {case['dims']} precision {precision}: max deviation {dev:.2e} of max|F|")
        # precision 0: both sum the same FP32 field in FP64 (in different orders), so they
        # agree to FP64 rounding; the default precision adds the FP32 rounding of ph + pl
        bar = 1e-10 if precision == 0 else 1e-4
        assert np.allclose(got, ref, rtol=bar, atol=bar * np.abs(ref).max())
    sim.close()


def test_forces_noalloc_rejects_oversized_grid():
    """Grids beyond the fixed scratch are refused before any device work."""
    from paper_2304_08159_gb300 import wl

    body = wl.make_body(dict(kind=1, center=(10.0, 10.0, 10.0), radius=4.0))
    rc = wl.wl_forces_noalloc((1024, 1024, 128), 0, body, 1.0, 1, 1, 1, None)
    assert rc == wl.WL_EINVAL
