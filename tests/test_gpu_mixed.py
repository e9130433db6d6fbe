"""Mixed-precision multigrid: the coarse levels (between the fine and the coarsest
one) stored in BF16 or FP16, every operation in FP32, the fine-level residual and
pressure and the FP64 coarsest solve unchanged.  The V-cycle is then a perturbed
preconditioner of an exact outer iteration (iterative refinement), so the solves
must reach the same tolerance and the results must meet the same bars against the
FP64 oracle as the FP32 path (velocity relative L2 <= 1e-5 after 10 steps, pressure
<= 2e-4 at tol 1e-6 and <= 1e-5 at tol 1e-8, C_D <= 1e-4), with at most a couple of
extra V-cycles.  Each test prints the measured error against the oracle.
"""
import numpy as np
import pytest

from tests.gpu_cases import CASES_2D, CASES_3D, make_pair, rel_l2, active_mask

pytestmark = pytest.mark.gpu

MODES = ["bf16", "fp16"]


def _levels_16bit(sim):
    # levels strictly between the fine and the coarsest one are stored in 16 bits
    return max(0, len(sim.levels()) - 2)


@pytest.mark.parametrize("cp", MODES)
@pytest.mark.parametrize("case", [CASES_3D[0], CASES_3D[2], CASES_3D[4], CASES_2D[0], CASES_2D[3]],
                         ids=lambda c: c["id"])
def test_mixed_vcycles_converge_to_oracle_solution(case, cp):
    """From x = 0, V-cycles with 16-bit coarse levels contract the residual about as
    fast as the FP32 cycles and converge to the oracle's solution of A x = z."""
    from paper_2304_08159_gb300 import wl

    sim, ref = make_pair(case, coarse_precision=cp)
    f32, _ = make_pair(case, oracle=False)
    assert _levels_16bit(sim) >= 1
    rng = np.random.default_rng(105)
    z = ref.poisson_apply(rng.standard_normal(sim.shape))
    z32 = z.astype(np.float32)
    res = {}
    for name, s in (("mixed", sim), ("fp32", f32)):
        s.set(wl.WL_FIELD_P, np.zeros(sim.shape, np.float32))
        s.set(wl.WL_FIELD_Z, z32)
        res[name] = [s.gmg_vcycle() for _ in range(10)]
    zmax = np.abs(z32).max()
    rm, rf = np.array(res["mixed"]), np.array(res["fp32"])
    # per-cycle contraction over the first cycles, compared with the FP32 cycles
    rate_m = (rm[4] / rm[0]) ** 0.25
    rate_f = (rf[4] / rf[0]) ** 0.25
    print(f"{case['id']} {cp}: contraction {rate_m:.3f} (fp32 {rate_f:.3f}), final {rm[-1]:.2e}")
    assert rate_m <= max(0.25, 1.5 * rate_f), (rate_m, rate_f)
    assert rm[-1] <= 1e-5 * zmax, rm
    act = active_mask(ref)
    xo, _, _ = ref.pcg(z32.astype(np.float64), tol=1e-12 * zmax)
    xg = sim.get(wl.WL_FIELD_P).astype(np.float64)
    xg = (xg - xg[act].mean()) * act
    xo = (xo - xo[act].mean()) * act
    well = ref.poisson_diag() >= 1e-2
    err = np.abs(xg - xo)[well].max() / np.abs(xo).max()
    print(f"  max |x - x_oracle| / max|x_oracle| = {err:.2e}")
    assert err <= 1e-4, err


@pytest.mark.parametrize("cp", MODES)
def test_mixed_cylinder_10_steps_parity(cp):
    """The 128x64 cylinder (R = 8, Re = 250), 10 adaptive steps at tol 1e-6 with 16-bit
    coarse levels: the FP32 path's bars against the FP64 oracle."""
    case = dict(id="c1", dims=(128, 64), nu=0.064, U=(1.0, 0.0), periodic=0,
                body=dict(kind=1, center=(32.0, 32.0), radius=8.0))
    sim, ref = make_pair(case, coarse_precision=cp)
    f32, _ = make_pair(case, oracle=False)
    sim.step(10)
    f32.step(10)
    ref.step(10, tol=1e-10)
    rc, last, tot, worst = sim.status()
    _, _, tot32, _ = f32.status()
    assert rc == 0 and worst <= 1e-6, (rc, last, tot, worst)
    assert tot <= tot32 + 4, (tot, tot32)
    ug, uo = sim.get(0).astype(np.float64), ref.get_u()
    eu = rel_l2(ug, uo)
    act = active_mask(ref)
    pg, po = sim.get(1).astype(np.float64), ref.get_p()
    pg = (pg - pg[act].mean()) * act
    po = (po - po[act].mean()) * act
    ep = rel_l2(pg, po)
    Fg, Fo = sim.forces(), ref.forces()
    ecd = abs(Fg[0] - Fo[0]) / abs(Fo[0])
    print(f"cylinder {cp}: V-cycles {tot} (fp32 {tot32}); rel L2 u {eu:.2e}, p {ep:.2e}; C_D rel {ecd:.2e}")
    assert eu <= 1e-5 and ep <= 2e-4 and ecd <= 1e-4, (eu, ep, ecd)


@pytest.mark.parametrize("cp", MODES)
def test_mixed_sphere_steps_parity_tight(cp):
    """A 3-D sphere (64x32x32, two 16-bit levels) for 5 steps at tol 1e-8: velocity and
    pressure within 1e-5 of the oracle, drag within 1e-4."""
    case = dict(id="s64", dims=(64, 32, 32), nu=0.02, U=(1.0, 0.0, 0.0), periodic=0,
                body=dict(kind=1, center=(20.3, 15.8, 16.2), radius=6.0))
    sim, ref = make_pair(case, tol=1e-8, coarse_precision=cp)
    assert _levels_16bit(sim) == 2
    sim.step(5)
    ref.step(5, tol=1e-12)
    rc, last, tot, worst = sim.status()
    assert rc == 0 and worst <= 1e-8, (rc, last, tot, worst)
    eu = rel_l2(sim.get(0).astype(np.float64), ref.get_u())
    act = active_mask(ref)
    pg, po = sim.get(1).astype(np.float64), ref.get_p()
    pg = (pg - pg[act].mean()) * act
    po = (po - po[act].mean()) * act
    ep = rel_l2(pg, po)
    Fg, Fo = sim.forces(), ref.forces()
    ed = abs(Fg[0] - Fo[0]) / abs(Fo[0])
    print(f"sphere {cp}: V-cycles {tot}; rel L2 u {eu:.2e}, p {ep:.2e}; drag rel {ed:.2e}")
    assert eu <= 1e-5 and ep <= 1e-5 and ed <= 1e-4, (eu, ep, ed)


def test_mixed_graph_and_host_loop_agree():
    """With 16-bit coarse levels the CUDA-graph step and the host-driven loop still
    give the same bits (the conversion is deterministic)."""
    case = dict(id="g", dims=(64, 32, 32), nu=0.02, U=(1.0, 0.0, 0.0), periodic=4,
                body=dict(kind=1, center=(20.0, 16.0, 16.0), radius=5.0))
    a, _ = make_pair(case, oracle=False, use_graph=True, coarse_precision="bf16")
    b, _ = make_pair(case, oracle=False, use_graph=False, coarse_precision="bf16")
    a.step(3)
    b.step(3)
    assert np.array_equal(a.get(0), b.get(0))
    assert np.array_equal(a.get(1), b.get(1))
