"""Pins of the oracle's reverse-mode derivative (adjoint) of the time step, all on the
CPU in FP64.  Each transpose is checked against the derivative it must be:

* dot-product tests <J dv, w> = <dv, J^T w> with J dv taken by central differences of
  the oracle's own forward routine (convdiff!, one BDIM stage, project!);
* the differentiated rollout's dJ/dtheta against central differences of J over whole
  forward rollouts with the body moved (theta = radius and centre);
* the force adjoint against the buoyancy closed form dF/dR = -2 pi R g (2-D) for the
  hydrostatic pressure p = g y, within the kernel's O(eps^2/R^2) error.
"""
import numpy as np
import pytest

import oracle as O

CASES = [
    dict(dims=(24, 20), nu=0.05, U=(1.0, 0.0), periodic=0, body=dict(kind=1, center=(9.3, 10.4), radius=4.2)),
    dict(dims=(20, 16), nu=0.03, U=(0.7, 0.2), periodic=1, body=dict(kind=1, center=(10.1, 7.6), radius=3.7)),
    dict(dims=(12, 10, 10), nu=0.04, U=(1.0, 0.1, -0.1), periodic=4,
         body=dict(kind=1, center=(5.6, 4.8, 5.3), radius=2.6)),
]
IDS = ["cyl2d", "xper2d", "sph3d"]


def _make(case, **kw):
    o = O.Oracle(case["dims"], case["nu"], U=case["U"], periodic=case["periodic"], body=case["body"], **kw)
    o.set_ic(0)
    return o


def _rand_u(o, rng, U, scale=0.4):
    return np.stack([U[c] + scale * rng.standard_normal(o.shape) for c in range(o.D)])


@pytest.mark.parametrize("advect", [True, False])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_convdiff_adjoint_dot(case, advect):
    o = _make(case, advect=advect)
    rng = np.random.default_rng(1)
    u = _rand_u(o, rng, case["U"])
    du = rng.standard_normal(u.shape)
    rb = rng.standard_normal(u.shape)
    h = 1e-6
    jdu = (o.convdiff(u + h * du) - o.convdiff(u - h * du)) / (2 * h)
    lhs = float((jdu * rb).sum())
    rhs = float((du * o.convdiff_adjoint(u, rb)).sum())
    assert abs(lhs - rhs) <= (1e-7 if advect else 1e-9) * abs(lhs), (lhs, rhs)


@pytest.mark.parametrize("stage", [1, 2])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_stage_adjoint_dot(case, stage):
    o = _make(case)
    rng = np.random.default_rng(2 + stage)
    u0 = _rand_u(o, rng, case["U"], 0.2)
    u1 = _rand_u(o, rng, case["U"], 0.2) if stage == 2 else None
    ob = rng.standard_normal(u0.shape)
    dt = 0.3
    u0b, u1b, _, _ = o.stage_adjoint(stage, dt, u0, u1, ob)
    h = 1e-6
    for which in ([0] if stage == 1 else [0, 1]):
        d = rng.standard_normal(u0.shape)
        if which == 0:
            jd = (o.bdim_stage(stage, dt, u0 + h * d, u1) - o.bdim_stage(stage, dt, u0 - h * d, u1)) / (2 * h)
            rhs = float((d * u0b).sum())
        else:
            jd = (o.bdim_stage(stage, dt, u0, u1 + h * d) - o.bdim_stage(stage, dt, u0, u1 - h * d)) / (2 * h)
            rhs = float((d * u1b).sum())
        lhs = float((jd * ob).sum())
        assert abs(lhs - rhs) <= 1e-7 * abs(lhs), (which, lhs, rhs)


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_project_adjoint_dot(case):
    """project! is linear in the velocity: <P dv, ubar> + <p(dv), pbar> = <dv, vbar>."""
    o = _make(case)
    rng = np.random.default_rng(7)
    mu0 = o.mu0()
    v = _rand_u(o, rng, case["U"], 0.3) * mu0
    dv = rng.standard_normal(v.shape) * mu0
    ub = rng.standard_normal(v.shape)
    pb = rng.standard_normal(o.shape)
    w, dt = 0.5, 0.4

    def proj(vel):
        o.set_u(vel)
        o.set_p(np.zeros(o.shape))
        o.project(w, dt, tol=1e-13)
        return o.get_u(), o.get_p()

    u1, p1 = proj(v + dv)
    u0, p0 = proj(v)
    lhs = float(((u1 - u0) * ub).sum() + ((p1 - p0) * pb).sum())
    vb, _ = o.project_adjoint(v, w, dt, ub, pb)
    rhs = float((dv * vb).sum())
    assert abs(lhs - rhs) <= 1e-8 * abs(lhs), (lhs, rhs)


def _J(case, theta, nsteps, dt, gF):
    c = dict(case)
    b = dict(case["body"])
    b["radius"] = theta[0]
    b["center"] = tuple(theta[1:])
    c["body"] = b
    o = _make(c)
    F, tb = o.rollout_grad(nsteps, dt, gF, tol=1e-13)
    return float((F * gF).sum()), tb


@pytest.mark.parametrize("case,nsteps", [(CASES[0], 4), (CASES[1], 3), (CASES[2], 2)], ids=IDS)
def test_rollout_grad_matches_central_differences(case, nsteps):
    """dJ/d(R, c) of J = sum_n gF_n . F_n over a rollout at fixed dt, against central
    differences of J over whole rollouts with the body moved (h = 1e-5)."""
    D = len(case["dims"])
    rng = np.random.default_rng(11)
    gF = rng.standard_normal((nsteps, D))
    theta = np.array([case["body"]["radius"]] + list(case["body"]["center"]))
    dt = 0.3
    J0, tb = _J(case, theta, nsteps, dt, gF)
    h = 1e-5
    fd = np.zeros_like(theta)
    for t in range(theta.size):
        e = np.zeros_like(theta)
        e[t] = h
        fd[t] = (_J(case, theta + e, nsteps, dt, gF)[0] - _J(case, theta - e, nsteps, dt, gF)[0]) / (2 * h)
    scale = np.abs(fd).max()
    assert scale > 0
    assert np.abs(tb - fd).max() <= 1e-5 * scale, (tb, fd)


TORUS = dict(dims=(16, 18, 18), nu=0.04, U=(1.0, 0.05, -0.05), periodic=0,
             body=dict(kind=2, center=(7.6, 8.7, 9.2), radius=4.3, radius2=1.9))


def _J_torus(theta, nsteps, dt, gF):
    c = dict(TORUS)
    c["body"] = dict(kind=2, radius=theta[0], radius2=theta[1], center=tuple(theta[2:]))
    o = _make(c)
    F, tb = o.rollout_grad(nsteps, dt, gF, tol=1e-13)
    return float((F * gF).sum()), tb


def test_torus_rollout_grad_matches_central_differences():
    """The torus (ring radius R in the y-z plane, tube radius r, centre c): dJ/d(R, r, c)
    over a 2-step rollout against central differences of J with the body changed
    (h = 1e-5), every one of the five components."""
    nsteps, dt = 2, 0.3
    gF = np.random.default_rng(12).standard_normal((nsteps, 3))
    b = TORUS["body"]
    theta = np.array([b["radius"], b["radius2"]] + list(b["center"]))
    J0, tb = _J_torus(theta, nsteps, dt, gF)
    assert tb.shape == (5,)
    h = 1e-5
    fd = np.zeros(5)
    for t in range(5):
        e = np.zeros(5)
        e[t] = h
        fd[t] = (_J_torus(theta + e, nsteps, dt, gF)[0] - _J_torus(theta - e, nsteps, dt, gF)[0]) / (2 * h)
    print("torus dJ/dtheta", tb, "FD", fd)
    assert np.abs(tb - fd).max() <= 1e-5 * np.abs(fd).max(), (tb, fd)


def test_torus_force_adjoint_theta_matches_central_differences():
    """The torus force weights' theta part alone (p fixed): every component of every force
    direction against central differences of the discrete force (h = 1e-6)."""
    rng = np.random.default_rng(13)
    b = TORUS["body"]
    theta = np.array([b["radius"], b["radius2"]] + list(b["center"]))
    p = rng.standard_normal(tuple(reversed(TORUS["dims"])))

    def make(th):
        c = dict(TORUS)
        c["body"] = dict(kind=2, radius=th[0], radius2=th[1], center=tuple(th[2:]))
        return _make(c)

    for d in range(3):
        Fbar = np.zeros(3)
        Fbar[d] = 1.0
        _, _, tb = make(theta).force_adjoint(p, Fbar)
        h = 1e-6
        for t in range(5):
            e = np.zeros(5)
            e[t] = h
            fd = (make(theta + e).force_adjoint(p, Fbar)[0][d] - make(theta - e).force_adjoint(p, Fbar)[0][d]) / (2 * h)
            assert abs(tb[t] - fd) <= 1e-6 * max(np.abs(tb).max(), 1e-12), (d, t, tb[t], fd)


def test_force_adjoint_buoyancy_closed_form():
    """Hydrostatic p = g y around a circle: F_y = -g pi R^2 up to O(eps^2/R^2), so
    dF_y/dR = -2 pi R g and dF_y/dc = 0.  The force adjoint's theta part (p held fixed)
    is the exact derivative of the discrete force (central differences, every component);
    the cell-centred kernel sum moves with the body's offset from the grid by a few
    percent, so the closed forms are checked on the mean over 16 seeded sub-cell offsets."""
    g, R = 0.7, 9.0
    y = np.arange(48) + 0.5
    p = g * np.repeat(y[:, None], 48, axis=1)
    Fbar = np.array([0.0, 1.0])

    def make(theta):
        case = dict(dims=(48, 48), nu=0.05, U=(1.0, 0.0), periodic=0,
                    body=dict(kind=1, center=(theta[1], theta[2]), radius=theta[0]))
        return _make(case)

    rng = np.random.default_rng(5)
    tbs = []
    for k in range(16):
        theta = np.array([R, 23.0 + rng.random(), 24.0 + rng.random()])
        o = make(theta)
        F, pb, tb = o.force_adjoint(p, Fbar)
        assert abs(F[1] + g * np.pi * R**2) <= 0.02 * g * np.pi * R**2
        tbs.append(tb)
        if k == 0:
            h = 1e-6
            for t in range(3):
                e = np.zeros(3)
                e[t] = h
                fd = (make(theta + e).force_adjoint(p, Fbar)[0][1] - make(theta - e).force_adjoint(p, Fbar)[0][1]) / (2 * h)
                assert abs(tb[t] - fd) <= 1e-6 * np.abs(tb).max(), (t, tb[t], fd)
            # pbar is the cotangent of p: <pbar, dp> = dF_y for a random dp
            dp = rng.standard_normal(p.shape)
            F1 = o.force_adjoint(p + dp, Fbar)[0][1]
            assert abs((F1 - F[1]) - float((pb * dp).sum())) <= 1e-10 * abs(F1 - F[1])
    m = np.mean(tbs, axis=0)
    ref = 2 * np.pi * R * g
    assert abs(m[0] + ref) <= 0.05 * ref, m
    assert np.abs(m[1:]).max() <= 0.05 * ref, m
