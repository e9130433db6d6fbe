"""GPU parity of the hand-written adjoint (wl_grad_forward / wl_grad_backward) against
the FP64 oracle's reverse-mode derivative (itself pinned by central differences in
tests/test_oracle_adjoint.py) and against central differences of the GPU forward.

Bars:
  * forces recorded by the differentiated rollout: as the forward parity tests (C_D
    relative <= 1e-4 at Poisson tol 1e-8);
  * dJ/dtheta against the oracle's: relative to max|dJ/dtheta| <= 5e-5.  The GPU runs the
    same discrete adjoint in FP32: a few hundred roundings (6e-8 each) per face and
    step, summed over the band and over up to 50 steps, and 100 adjoint solves stopped at
    1e-7 relative, ~1e-5 of the largest terms;
  * dJ/dtheta against central differences of the FP32 forward (h = 1e-3, the 2-D
    cylinder 256x128 case): relative to max|FD| <= 2e-3.  The difference quotient carries
    the forward's FP32/solver noise (~1e-7 of J ~ 10) divided by 2h, ~5e-4, plus the
    O(h^2) error and limiter switches crossed within +-h.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

CASES = [
    dict(id="cyl48x32", dims=(48, 32), nu=0.05, U=(1.0, 0.0), periodic=0,
         body=dict(kind=1, center=(14.3, 15.7), radius=5.0), nsteps=4, dt=0.3),
    dict(id="xper40x32", dims=(40, 32), nu=0.03, U=(0.8, 0.1), periodic=1,
         body=dict(kind=1, center=(19.6, 15.2), radius=4.6), nsteps=3, dt=0.25),
    dict(id="sph24x16x16", dims=(24, 16, 16), nu=0.04, U=(1.0, 0.0, 0.0), periodic=0,
         body=dict(kind=1, center=(8.4, 7.7, 8.2), radius=3.3), nsteps=2, dt=0.3),
]


def _gpu(case, tol=1e-8, every=2):
    from paper_2304_08159_gb300 import Sim

    sim = Sim(case["dims"], case["nu"], case["U"], body=case["body"], periodic=case["periodic"], tol=tol,
              dt_fixed=case["dt"])
    F = sim.grad_forward(case["nsteps"], every)
    return sim, F


@pytest.mark.parametrize("case", CASES, ids=lambda c: c["id"])
def test_adjoint_matches_oracle_gradient(case):
    D = len(case["dims"])
    rng = np.random.default_rng(21)
    gF = rng.standard_normal((case["nsteps"], D))
    sim, Fg = _gpu(case)
    tb = sim.grad_backward(gF)
    ref = O.Oracle(case["dims"], case["nu"], U=case["U"], periodic=case["periodic"], body=case["body"])
    ref.set_ic(0)
    Fo, tbo = ref.rollout_grad(case["nsteps"], case["dt"], gF, tol=1e-12)
    fscale = np.abs(Fo).max()
    assert np.abs(Fg - Fo).max() <= 1e-4 * fscale, (Fg, Fo)
    err = np.abs(tb - tbo).max() / np.abs(tbo).max()
    print(f"{case['id']}: dJ/dtheta gpu {tb} oracle {tbo} rel err {err:.2e}")
    assert err <= 5e-5, (tb, tbo)
    # the state after the backward pass is the one after the rollout again
    from paper_2304_08159_gb300 import wl

    u_after = sim.get(wl.WL_FIELD_U).astype(np.float64)
    assert np.abs(u_after - ref.get_u()).max() <= 1e-4 * np.abs(ref.get_u()).max()
    sim.close()


def test_adjoint_checkpoint_interval_independent():
    """Recomputing from checkpoints every 1, 2 or 4 steps gives the same gradient bits:
    the recomputed steps repeat the rollout's bits, and every adjoint kernel sums in a
    fixed order (gathers and fixed-order block partials, no atomics)."""
    case = CASES[0]
    gF = np.random.default_rng(22).standard_normal((case["nsteps"], 2))
    out = []
    for every in (1, 2, 4):
        sim, _ = _gpu(case, every=every)
        out.append(sim.grad_backward(gF))
        sim.close()
    for t in out[1:]:
        assert np.array_equal(t, out[0]), out


DET_CASES = CASES + [
    # the band across the periodic x side: the gather's wrapped targets and images
    dict(id="xper40x32_seam", dims=(40, 32), nu=0.03, U=(0.8, 0.1), periodic=1,
         body=dict(kind=1, center=(1.3, 15.2), radius=4.6), nsteps=3, dt=0.25),
    # 3-D, periodic in z with the band across the z side
    dict(id="sph24x16x16_zper", dims=(24, 16, 16), nu=0.04, U=(1.0, 0.0, 0.0), periodic=4,
         body=dict(kind=1, center=(8.4, 7.7, 0.6), radius=3.3), nsteps=2, dt=0.3),
]


@pytest.mark.parametrize("case", DET_CASES, ids=lambda c: c["id"])
def test_adjoint_bitwise_repeatable(case):
    """Two backward passes after one rollout, and a second sim's rollout and backward pass,
    give identical gradient bits; the seam cases (band across a periodic side) also match
    the oracle's gradient at the 5e-5 bar."""
    D = len(case["dims"])
    gF = np.random.default_rng(23).standard_normal((case["nsteps"], D))
    sim, F1 = _gpu(case)
    t1 = sim.grad_backward(gF)
    t1b = sim.grad_backward(gF)
    sim.close()
    sim, F2 = _gpu(case)
    t2 = sim.grad_backward(gF)
    sim.close()
    assert np.array_equal(F1, F2)
    assert np.array_equal(t1, t1b) and np.array_equal(t1, t2), (t1, t1b, t2)
    if case["id"].endswith(("seam", "zper")):
        ref = O.Oracle(case["dims"], case["nu"], U=case["U"], periodic=case["periodic"], body=case["body"])
        ref.set_ic(0)
        _, tbo = ref.rollout_grad(case["nsteps"], case["dt"], gF, tol=1e-12)
        err = np.abs(t1 - tbo).max() / np.abs(tbo).max()
        print(f"{case['id']}: dJ/dtheta gpu {t1} oracle {tbo} rel err {err:.2e}")
        assert err <= 5e-5, (t1, tbo)


def _cd_c5(theta, nsteps, tol, every=10, with_grad=False):
    """Mean drag coefficient of the 2-D cylinder case (256x128, Re 200 on the diameter,
    U = 1, fixed dt 0.1) for the body theta = (R, cx, cy)."""
    from paper_2304_08159_gb300 import Sim

    R = theta[0]
    sim = Sim((256, 128), 24.0 / 200.0, (1.0, 0.0), body=dict(kind=1, center=(theta[1], theta[2]), radius=R),
              tol=tol, dt_fixed=0.1)
    F = sim.grad_forward(nsteps, every)
    J = F[:, 0].mean() / R  # C_D = F_x / (U^2/2 * 2R)
    tb = None
    if with_grad:
        g = np.zeros_like(F)
        g[:, 0] = 1.0 / (nsteps * R)
        tb = sim.grad_backward(g)
        tb[0] -= J / R  # the 1/R of the coefficient itself
    sim.close()
    return J, tb


def test_c5_drag_gradient_fd_and_oracle():
    """The adjoint configuration: 2-D cylinder 256x128, R = 12 at (64, 64), Re = 200, mean
    drag coefficient over 50 steps at fixed dt, checkpoints every 10 steps.  dJ/d(R, cx,
    cy) against central differences of the GPU forward (h = 1e-3) and against the FP64
    oracle's gradient."""
    theta = np.array([12.0, 64.0, 64.0])
    nsteps = 50
    J, tb = _cd_c5(theta, nsteps, tol=1e-8, with_grad=True)
    h = 1e-3
    fd = np.zeros(3)
    for t in range(3):
        e = np.zeros(3)
        e[t] = h
        fd[t] = (_cd_c5(theta + e, nsteps, 1e-8)[0] - _cd_c5(theta - e, nsteps, 1e-8)[0]) / (2 * h)
    err_fd = np.abs(tb - fd).max() / np.abs(fd).max()
    ref = O.Oracle((256, 128), 24.0 / 200.0, U=(1.0, 0.0), body=dict(kind=1, center=(64.0, 64.0), radius=12.0))
    ref.set_ic(0)
    g = np.zeros((nsteps, 2))
    g[:, 0] = 1.0 / (nsteps * 12.0)
    Fo, tbo = ref.rollout_grad(nsteps, 0.1, g, tol=1e-11)
    Jo = Fo[:, 0].mean() / 12.0
    tbo = tbo.copy()
    tbo[0] -= Jo / 12.0
    err_or = np.abs(tb - tbo).max() / np.abs(tbo).max()
    print(f"C5: C_D {J:.6f} (oracle {Jo:.6f}); dC_D/d(R,cx,cy) adjoint {tb}, FD {fd}, oracle {tbo}; "
          f"rel err vs FD {err_fd:.2e}, vs oracle {err_or:.2e}")
    assert abs(J - Jo) <= 1e-4 * abs(Jo)
    assert err_or <= 5e-5, (tb, tbo)
    assert err_fd <= 2e-3, (tb, fd)


def test_autograd_function_drag_coefficient():
    """torch.autograd through the rollout: the mean drag coefficient's gradient equals the
    library's theta-cotangent plus the coefficient's own 1/R term."""
    import torch

    from paper_2304_08159_gb300.grad import rollout_forces

    theta = torch.tensor([6.0, 20.3, 16.1], dtype=torch.float64, requires_grad=True)
    F = rollout_forces(theta, dims=(64, 32), nu=12.0 / 200.0, U=(1.0, 0.0), nsteps=6, dt=0.2, every=3, tol=1e-8)
    J = F[:, 0].mean() / (0.5 * 2 * theta[0])
    J.backward()
    Jv, tb = _small(theta.detach().numpy(), 6)
    assert abs(J.item() - Jv) <= 1e-12 * abs(Jv)
    assert np.abs(theta.grad.numpy() - tb).max() <= 1e-5 * np.abs(tb).max(), (theta.grad, tb)


def _small(theta, nsteps):
    from paper_2304_08159_gb300 import Sim

    R = theta[0]
    sim = Sim((64, 32), 12.0 / 200.0, (1.0, 0.0), body=dict(kind=1, center=(theta[1], theta[2]), radius=R), tol=1e-8,
              dt_fixed=0.2)
    F = sim.grad_forward(nsteps, 3)
    J = F[:, 0].mean() / R
    g = np.zeros_like(F)
    g[:, 0] = 1.0 / (nsteps * R)
    tb = sim.grad_backward(g)
    tb[0] -= J / R
    sim.close()
    return J, tb


TORUS = dict(id="torus20x18x18", dims=(20, 18, 18), nu=0.04, U=(1.0, 0.05, -0.05), periodic=0,
             body=dict(kind=2, center=(8.6, 8.7, 9.2), radius=4.3, radius2=1.9), nsteps=3, dt=0.3)


def test_torus_adjoint_matches_oracle_and_central_differences():
    """The torus (the paper's donut): dJ/d(R, r, c_x, c_y, c_z) against the FP64 oracle's
    gradient (pinned by central differences on the CPU) at the 5e-5 bar, bitwise equal
    on a second run, and against central differences of the GPU forward (h = 1e-3) at
    the 2e-3 bar the cylinder's FD check uses."""
    case = TORUS
    gF = np.random.default_rng(24).standard_normal((case["nsteps"], 3))
    sim, Fg = _gpu(case)
    tb = sim.grad_backward(gF)
    tb2 = sim.grad_backward(gF)
    sim.close()
    assert tb.shape == (5,) and np.array_equal(tb, tb2)
    ref = O.Oracle(case["dims"], case["nu"], U=case["U"], periodic=case["periodic"], body=case["body"])
    ref.set_ic(0)
    Fo, tbo = ref.rollout_grad(case["nsteps"], case["dt"], gF, tol=1e-12)
    assert np.abs(Fg - Fo).max() <= 1e-4 * np.abs(Fo).max()
    err = np.abs(tb - tbo).max() / np.abs(tbo).max()
    b = case["body"]
    theta = np.array([b["radius"], b["radius2"]] + list(b["center"]))

    def J(th):
        c = dict(case)
        c["body"] = dict(kind=2, radius=th[0], radius2=th[1], center=tuple(th[2:]))
        s, F = _gpu(c)
        s.close()
        return float((F * gF).sum())

    h = 1e-3
    fd = np.array([(J(theta + h * e) - J(theta - h * e)) / (2 * h) for e in np.eye(5)])
    err_fd = np.abs(tb - fd).max() / np.abs(fd).max()
    print(f"torus: dJ/dtheta gpu {tb} oracle {tbo} FD {fd}; rel err vs oracle {err:.2e}, vs FD {err_fd:.2e}")
    assert err <= 5e-5, (tb, tbo)
    assert err_fd <= 2e-3, (tb, fd)


def test_torus_autograd():
    """torch.autograd through a torus rollout gives the library's theta-cotangent."""
    import torch

    from paper_2304_08159_gb300.grad import rollout_forces

    case = TORUS
    b = case["body"]
    theta = torch.tensor([b["radius"], b["radius2"]] + list(b["center"]), dtype=torch.float64, requires_grad=True)
    F = rollout_forces(theta, dims=case["dims"], nu=case["nu"], U=case["U"], nsteps=case["nsteps"], dt=case["dt"],
                       every=2, tol=1e-8, torus=True)
    J = F[:, 0].sum()
    J.backward()
    sim, _ = _gpu(case)
    g = np.zeros((case["nsteps"], 3))
    g[:, 0] = 1.0
    tb = sim.grad_backward(g)
    sim.close()
    assert np.array_equal(theta.grad.numpy(), tb), (theta.grad, tb)


def test_grad_argument_checks():
    from paper_2304_08159_gb300 import Sim, wl

    sim = Sim((32, 16), 0.05, (1.0, 0.0), body=dict(kind=1, center=(8.0, 8.0), radius=3.0))  # adaptive dt
    with pytest.raises(wl.WLError):
        sim.grad_forward(2, 1)
    sim.close()
    sim = Sim((32, 16), 0.05, (1.0, 0.0), body=dict(kind=1, center=(8.0, 8.0), radius=3.0), dt_fixed=0.2)
    with pytest.raises(wl.WLError):
        sim.grad_backward(np.zeros((2, 2)))  # no forward rollout yet
    sim.close()
