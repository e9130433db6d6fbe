"""Pins of the FP64 oracle against what the mathematics fixes.

Each test checks one routine of the oracle against something other than the
oracle itself: a hand-worked table (tests/golden/), a closed form, an invariant,
a textbook solver (numpy least squares) or brute force on a tiny case.  Together
they are chosen so that a dropped term, a wrong sign, a wrong index or a swapped
operand in the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _table(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                rows.append([float(v) for v in line.split()])
    return np.array(rows)


# --------------------------------------------------------------------------- BDIM kernel
def test_kernel_moments_golden():
    """K0, K1 at hand-worked points (golden/kernel_moments.txt)."""
    for s, k0, k1 in _table("kernel_moments.txt"):
        assert abs(O.K0(s) - k0) < 1e-15
        assert abs(O.K1(s) - k1) < 1e-15


def test_kernel_moments_derivatives():
    """K0' = K and K1' = -s K (central differences), clamped outside [-1, 1]."""
    h = 1e-5
    for s in np.linspace(-0.95, 0.95, 39):
        K = 0.5 * (1 + math.cos(math.pi * s))
        d0 = (O.K0(s + h) - O.K0(s - h)) / (2 * h)
        d1 = (O.K1(s + h) - O.K1(s - h)) / (2 * h)
        assert abs(d0 - K) < 1e-8
        assert abs(d1 + s * K) < 1e-8
    # outside the support the moments are exactly those of the empty / full range
    assert O.K0(3.0) == 1.0 and O.K0(1.0) == 1.0 and O.K0(-1.0) == 0.0 and O.K0(-3.0) == 0.0
    assert O.K1(3.0) == 0.0 and O.K1(-1.0) == 0.0


@pytest.mark.parametrize("R", [8, 12, 16])
def test_body_volume_circle(R):
    """sum over faces of (1 - mu0) = pi R^2 up to O(eps^2/R^2)."""
    o = O.Oracle((128, 64), 0.064, U=(1, 0), body=dict(kind=1, center=(64, 32), radius=R))
    m = o.mu0()
    for c in range(2):
        rel = (1 - m[c]).sum() / (math.pi * R * R) - 1
        assert abs(rel) < 0.2 / R**2


def test_body_volume_sphere():
    R = 12
    o = O.Oracle((64, 64, 64), 0.01, U=(1, 0, 0), body=dict(kind=1, center=(32, 32, 32), radius=R))
    m = o.mu0()
    V = 4.0 / 3.0 * math.pi * R**3
    for c in range(3):
        assert abs((1 - m[c]).sum() / V - 1) < 0.5 / R**2


def test_body_volume_torus():
    """Sum of (1 - mu0) over the faces is the torus volume 2 pi^2 R r^2 up to the
    kernel's O(eps^2 / r^2) smearing: for a symmetric kernel the excess is eps^2 times
    the integrated mean curvature (4 pi^2 R for a torus) up to a constant, so the
    relative error times r^2 is the same constant for every tube radius."""
    scaled = []
    for R, r, n in ((12, 4, 64), (10, 5, 64), (16, 6, 80)):
        o = O.Oracle((n, n, n), 0.01, U=(1, 0, 0), body=dict(kind=2, center=(n / 2, n / 2, n / 2), radius=R, radius2=r))
        m = o.mu0()
        V = 2.0 * math.pi**2 * R * r**2
        for c in range(3):
            err = (1 - m[c]).sum() / V - 1
            assert abs(err) < 0.5 / r**2
            scaled.append(err * r**2)
    assert max(scaled) - min(scaled) < 0.1 * max(abs(x) for x in scaled)


def test_mu1_direction_and_band():
    """mu1 is eps*K1(d/eps) times the outward normal; zero outside |d| < eps."""
    o = O.Oracle((48, 40), 0.05, U=(1, 0), body=dict(kind=1, center=(20.3, 19.7), radius=6.5))
    mu1 = o.mu1()
    cnt = 0
    for c in range(2):
        for j in range(40):
            for i in range(48):
                x = np.array([i + 0.5, j + 0.5])
                x[c] -= 0.5
                r = np.hypot(x[0] - 20.3, x[1] - 19.7)
                d = r - 6.5
                n = (x - np.array([20.3, 19.7])) / r
                if abs(d) >= 1.0:
                    assert np.all(mu1[c, :, j, i] == 0.0)
                    continue
                cnt += 1
                # K1 by Simpson quadrature of t K(t) over [d, 1]
                t = np.linspace(d, 1.0, 2001)
                f = t * 0.5 * (1 + np.cos(np.pi * t))
                k1 = (t[1] - t[0]) / 3 * (f[0] + f[-1] + 4 * f[1:-1:2].sum() + 2 * f[2:-1:2].sum())
                assert np.allclose(mu1[c, :, j, i], k1 * n, atol=1e-12)
    assert cnt > 50


# --------------------------------------------------------------------------- convection
def test_koren_psi_golden():
    for r, p in _table("koren_psi.txt"):
        assert abs(O.psi(r) - p) < 1e-15


def test_face_value_exact_for_quadratic_averages():
    """With the limiter inactive the kappa=1/3 value reproduces q(0) exactly for cell
    averages of a quadratic q over [-2,-1], [-1,0], [0,1] (third order)."""
    rng = np.random.default_rng(1)
    hits = 0
    for _ in range(200):
        a, b, c = rng.normal(size=3)
        avg = lambda x0, x1: a + b * (x0 + x1) / 2 + c * (x1**3 - x0**3) / (3 * (x1 - x0))
        uu, cc, dd = avg(-2, -1), avg(-1, 0), avg(0, 1)
        if dd == cc:
            continue
        r = (cc - uu) / (dd - cc)
        if 0.4 < r < 4.0:  # unlimited branch psi = (2+r)/3
            hits += 1
            assert abs(O.face_value(uu, cc, dd) - a) < 1e-13
    assert hits > 20


def test_face_value_limited_cases():
    # extremum (r < 0) -> first order upwind (phi = c); flat downwind -> c; steep -> capped
    assert O.face_value(1.0, 2.0, 1.5) == 2.0
    assert O.face_value(0.3, 0.7, 0.7) == 0.7
    # r = (c-u)/(d-c) = 10 -> psi = 2 -> phi = d
    assert abs(O.face_value(-9.0, 1.0, 2.0) - 2.0) < 1e-15


def _random_u(o, rng, scale=1.0):
    return scale * rng.standard_normal((o.D,) + o.shape)


@pytest.mark.parametrize("dims,per", [((16, 12), 3), ((16, 12), 0), ((10, 8, 6), 7), ((10, 8, 6), 2)])
def test_free_stream_preserved(dims, per):
    """A uniform velocity has zero convection-diffusion residual exactly."""
    U = (0.7, -0.3, 0.2)[: len(dims)]
    o = O.Oracle(dims, 0.1, U=U, periodic=per)
    u = np.empty((len(dims),) + o.shape)
    for c in range(len(dims)):
        u[c] = U[c]
    r = o.convdiff(u)
    assert np.abs(r).max() == 0.0


def test_convdiff_diffusion_only_is_discrete_laplacian():
    """With advection off, r = nu * (5-point discrete Laplacian) on a periodic grid,
    checked against numpy.roll (an independent statement of the second difference)."""
    rng = np.random.default_rng(3)
    o = O.Oracle((12, 10), 0.37, periodic=3, advect=False)
    u = _random_u(o, rng)
    r = o.convdiff(u)
    for c in range(2):
        lap = sum(np.roll(u[c], 1, a) + np.roll(u[c], -1, a) - 2 * u[c] for a in (0, 1))
        assert np.allclose(r[c], 0.37 * lap, atol=1e-13)


def test_convection_is_conservative_periodic():
    """Flux form: the residual sums to zero over a periodic domain (momentum)."""
    rng = np.random.default_rng(4)
    o = O.Oracle((10, 8, 6), 0.02, periodic=7)
    r = o.convdiff(_random_u(o, rng))
    for c in range(3):
        assert abs(r[c].sum()) < 1e-12


def test_upwind_transport_direction():
    """Uniform u_x = 1 advecting a tangential profile v(x): r_v = -(phi_{i+1} - phi_i)
    with phi the upwind (left) limited value; for a linear ramp away from the
    wrap the unlimited kappa=1/3 value is exact, so r_v = -slope."""
    o = O.Oracle((32, 4), 0.0, periodic=3)
    u = np.zeros((2,) + o.shape)
    u[0] = 1.0
    x = np.arange(32) + 0.5
    u[1] = 0.1 * x[None, :]
    r = o.convdiff(u)
    assert np.allclose(r[0], 0.0, atol=1e-14)
    assert np.allclose(r[1][:, 4:28], -0.1, atol=1e-13)


def test_tvd_step_advection():
    """Heun + Koren limiter (no body, no viscosity) advecting a step: no new extrema."""
    o = O.Oracle((64, 4), 0.0, periodic=3)
    u = np.zeros((2,) + o.shape)
    u[0] = 1.0
    u[1][:, 10:30] = 1.0
    dt = 0.4
    lo, hi = u[1].min(), u[1].max()
    for _ in range(60):
        u1 = o.bdim_stage(1, dt, u)
        u = o.bdim_stage(2, dt, u, u1)
        assert u[1].min() >= lo - 1e-12 and u[1].max() <= hi + 1e-12
    assert np.allclose(u[0], 1.0, atol=1e-14)
    # the step moved by 60*0.4 = 24 cells: centre of mass of the profile
    xc = (u[1][0] * (np.arange(64) + 0.5)).sum() / u[1][0].sum()
    assert abs(xc - (20.0 + 24.0)) < 0.5


# --------------------------------------------------------------------------- BC
def test_bc_ghost_values():
    """Ghost and boundary faces follow the BC: Dirichlet normal, zero-gradient
    tangential, periodic wrap, including the corners."""
    rng = np.random.default_rng(5)
    o = O.Oracle((6, 5), 0.1, U=(1.5, -0.5), periodic=1)  # x periodic, y walls
    u = rng.standard_normal((2,) + o.shape)
    o.set_u(u)
    P = o.get_u_padded()  # (2, 9, 10): index [c, j+2, i+2]
    g = lambda c, i, j: P[c, j + 2, i + 2]
    ui = lambda c, i, j: u[c, j, i]
    for j in range(-2, 7):
        for i in range(-2, 8):
            iw = i % 6
            # y is a wall: v normal Dirichlet on j in {-2,-1,0,5,6}
            if j in (-2, -1, 0, 5, 6):
                assert g(1, i, j) == -0.5
            else:
                assert g(1, i, j) == ui(1, iw, j)
            jc = min(max(j, 0), 4)
            assert g(0, i, j) == ui(0, iw, jc)


# --------------------------------------------------------------------------- Poisson
def _dense_matrix(o, level=0):
    dims = o.level_dims(level)
    n = int(np.prod(dims))
    A = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        A[:, k] = o.poisson_apply(e, level).ravel()
    return A


def test_poisson_operator_fourier_modes():
    """Constant coefficients, periodic: A cos(2 pi m.x/N) = -sum_d 4 sin^2(pi m_d/N_d) cos(...)."""
    o = O.Oracle((12, 8, 6), 0.1, periodic=7)
    z, y, x = np.meshgrid(np.arange(6), np.arange(8), np.arange(12), indexing="ij")
    for m in [(1, 0, 0), (2, 3, 1), (5, 1, 2)]:
        ph = 2 * np.pi * (m[0] * x / 12 + m[1] * y / 8 + m[2] * z / 6)
        lam = -sum(4 * np.sin(np.pi * m[d] / n) ** 2 for d, n in enumerate((12, 8, 6)))
        for f in (np.cos(ph), np.sin(ph)):
            assert np.allclose(o.poisson_apply(f), lam * f, atol=1e-12)


def test_poisson_operator_neumann_walls():
    """Non-periodic: boundary faces carry no flux, so A has zero column and row sums."""
    o = O.Oracle((7, 5), 0.1, U=(1, 0), body=dict(kind=1, center=(3.2, 2.6), radius=1.4))
    A = _dense_matrix(o)
    assert np.allclose(A.sum(0), 0, atol=1e-14) and np.allclose(A.sum(1), 0, atol=1e-14)
    assert np.allclose(A, A.T, atol=1e-15)
    # eigenvalues <= 0 (negative semi-definite)
    assert np.linalg.eigvalsh(A).max() < 1e-12


@pytest.mark.parametrize("body", [None, dict(kind=1, center=(8.3, 7.6), radius=3.1)])
@pytest.mark.parametrize("dims", [(16, 16), (16, 12)])
def test_dense_pcg_vcycle_vs_lstsq(body, dims):
    """Dense GE (mean-zero), PCG and repeated V-cycles all match numpy least squares."""
    o = O.Oracle(dims, 0.1, U=(1, 0), body=body)
    rng = np.random.default_rng(7)
    A = _dense_matrix(o)
    dg = o.poisson_diag().ravel()
    act = dg > 0
    z = A @ rng.standard_normal(A.shape[0])  # consistent right-hand side
    xa = np.zeros_like(z)
    sol = np.linalg.lstsq(A[np.ix_(act, act)], z[act], rcond=None)[0]
    xa[act] = sol - sol.mean()
    xd = o.dense_solve(z).ravel()
    assert np.abs(xd - xa).max() < 1e-10
    xp, it, res = o.pcg(z, tol=1e-12)
    xp = xp.ravel()
    xp[act] -= xp[act].mean()
    assert res <= 1e-12 and np.abs(xp - xa).max() < 1e-10
    x = np.zeros(o.shape)
    for _ in range(60):
        x, r = o.vcycle(x, z.reshape(o.shape), pre=0, post=4)
        if r < 1e-12:
            break
    assert r < 1e-12
    xv = x.ravel().copy()
    xv[act] -= xv[act].mean()
    assert np.abs(xv - xa).max() < 1e-10


def test_coarse_coefficients_constant_case():
    """No body, periodic: the half-sum coarse face coefficient equals the
    re-discretised one, 2^(D-2), on every level."""
    for dims, val in [((32, 16), 1.0), ((16, 16, 16), 2.0)]:
        o = O.Oracle(dims, 0.1, periodic=(1 << len(dims)) - 1)
        for l in range(1, o.nlevels()):
            L = o.level_L(l)
            assert np.all(L == val ** l)


def test_levels_rule():
    o = O.Oracle((128, 64), 0.064, U=(1, 0))
    assert [o.level_dims(l) for l in range(o.nlevels())] == [(128, 64), (64, 32), (32, 16), (16, 8), (8, 4)]
    o = O.Oracle((24, 20, 12), 0.1, periodic=7)
    assert [o.level_dims(l) for l in range(o.nlevels())] == [(24, 20, 12), (12, 10, 6), (6, 5, 3)]


def test_vcycle_contracts():
    """One V(0,4) cycle contracts the residual of a body problem by a fixed factor."""
    o = O.Oracle((64, 32, 32), 0.01, U=(1, 0, 0), body=dict(kind=1, center=(16, 16, 16), radius=8))
    rng = np.random.default_rng(8)
    z = o.poisson_apply(rng.standard_normal(o.shape))
    x = np.zeros(o.shape)
    rs = []
    for _ in range(5):
        x, r = o.vcycle(x, z, 0, 4)
        rs.append(r)
    rates = np.array(rs[1:]) / np.array(rs[:-1])
    assert rates.max() < 0.15


# --------------------------------------------------------------------------- projection
def test_projection_divergence_and_mass():
    """After project!, |div u| <= tol; with walls the net boundary flux is zero and
    the divergence telescopes to it."""
    o = O.Oracle((40, 24), 0.05, U=(1, 0), body=dict(kind=1, center=(12.2, 11.9), radius=4))
    rng = np.random.default_rng(9)
    # a blended field (zero on the solid faces, as after BDIM) so that cells with
    # no equation carry no divergence
    u = o.mu0() * (1.0 + 0.2 * rng.standard_normal((2,) + o.shape))
    o.set_u(u)
    z0 = o.divergence()
    # sum of div over all cells = outflow - inflow through the walls = U*ny - U*ny = 0
    assert abs(z0.sum()) < 1e-11
    it, res = o.project(1.0, 0.3, tol=1e-10)
    assert res <= 1e-10
    assert np.abs(o.divergence()).max() <= 1.0001e-10


def test_projection_removes_gradient_part():
    """Periodic, no body: projecting u = v + grad(phi), v divergence-free, returns v
    and p = phi / (w dt) (up to a constant)."""
    o = O.Oracle((16, 16), 0.1, periodic=3)
    rng = np.random.default_rng(10)
    phi = rng.standard_normal(o.shape)
    # staggered gradient: (grad phi)_c[I] = phi[I] - phi[I - e_c]
    gx = phi - np.roll(phi, 1, axis=1)
    gy = phi - np.roll(phi, 1, axis=0)
    # divergence-free v from a streamfunction on cell corners
    psi = rng.standard_normal(o.shape)
    vx = np.roll(psi, -1, axis=0) - psi
    vy = -(np.roll(psi, -1, axis=1) - psi)
    u = np.stack([vx + gx, vy + gy])
    o.set_u(u)
    w, dt = 0.5, 0.8
    o.project(w, dt, tol=1e-13)
    assert np.abs(o.get_u() - np.stack([vx, vy])).max() < 1e-11
    p = o.get_p()
    ref = phi / (w * dt)
    assert np.abs((p - p.mean()) - (ref - ref.mean())).max() < 1e-10


# --------------------------------------------------------------------------- full step
def test_cfl_uniform_closed_form():
    o = O.Oracle((32, 16), 0.064, U=(1, 0))
    o.set_ic(0)
    assert abs(o.dt - 1.0 / (1.0 + 4 * 0.064)) < 1e-15
    o = O.Oracle((8, 8, 8), 0.01, U=(0.5, -0.25, 0.125))
    o.set_ic(0)
    assert abs(o.dt - 1.0 / (0.5 + 0.25 + 0.125 + 6 * 0.01)) < 1e-15
    o = O.Oracle((8, 8), 1e-9, U=(1e-12, 0))
    o.set_ic(0)
    assert o.dt == 10.0  # cap


@pytest.mark.parametrize("dims", [(32, 32), (16, 16, 16)])
def test_stokes_mode_closed_form(dims):
    """Advection off, fixed dt: every Heun step multiplies the (discretely
    divergence-free) Taylor-Green mode by g = 1 + l dt + (l dt)^2/2,
    l = -nu sum_d 4 sin^2(k/2) over the directions the mode varies in."""
    D = len(dims)
    nu, dt = 0.05, 0.5
    o = O.Oracle(dims, nu, periodic=(1 << D) - 1, advect=False)
    o.set_ic(1)
    u0 = o.get_u()
    k = 2 * np.pi / dims[0]
    lam = -nu * D * 4 * np.sin(k / 2) ** 2
    g = 1 + lam * dt + (lam * dt) ** 2 / 2
    o.step(4, tol=1e-12, dt_fixed=dt)
    assert np.abs(o.get_u() - g**4 * u0).max() < 1e-14


def test_tgv_2d_energy_decay_converges():
    """2-D Taylor-Green is an exact Navier-Stokes solution, E = E0 exp(-4 nu k^2 t);
    the error in E falls at least at second order under refinement (Re = 100,
    dt = 1/4 cell per unit velocity)."""
    errs = []
    for N in (16, 32, 64):
        L = N / (2 * np.pi)
        nu = L / 100.0
        o = O.Oracle((N, N), nu, periodic=3)
        o.set_ic(1)
        E0 = o.kinetic_energy()
        T = 0.5 * L
        nst = int(round(T / 0.25))
        o.step(nst, tol=1e-12, dt_fixed=T / nst)
        k = 2 * np.pi / N
        Eex = E0 * np.exp(-4 * nu * k * k * T)
        errs.append(abs(o.kinetic_energy() - Eex) / Eex)
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) >= 2.0, (errs, orders)


def test_tgv_3d_energy_decays_and_divergence():
    """3-D TGV: kinetic energy never increases, |div u| <= tol after each step,
    periodic momentum is conserved to rounding."""
    N = 24
    L = N / (2 * np.pi)
    o = O.Oracle((N, N, N), L / 1600.0, periodic=7)
    o.set_ic(1)
    E = o.kinetic_energy()
    mom0 = o.get_u().sum(axis=(1, 2, 3))
    for _ in range(6):
        o.step(1, tol=1e-10)
        E2 = o.kinetic_energy()
        assert E2 <= E * (1 + 1e-14)
        E = E2
        assert np.abs(o.divergence()).max() <= 1.0001e-10
    assert np.abs(o.get_u().sum(axis=(1, 2, 3)) - mom0).max() < 1e-10


def test_cylinder_mirror_symmetry():
    """The 128x64 cylinder case is symmetric about y = 32: u(x, 64-y) = u,
    v(x, 64-y) = -v, to 1e-12 after 50 steps with no noise injected."""
    o = O.Oracle((128, 64), 0.064, U=(1, 0), body=dict(kind=1, center=(32, 32), radius=8))
    o.set_ic(0)
    o.step(50, tol=1e-12)
    u = o.get_u()
    assert np.abs(u[0] - u[0][::-1, :]).max() < 1e-12
    assert np.abs(u[1][1:] + u[1][1:][::-1]).max() < 1e-12
    assert np.all(u[1][0] == 0.0)
    F = o.forces()
    assert abs(F[1]) < 1e-10 and F[0] > 0


def test_body_faces_blocked():
    """Inside the body (d <= -eps) BDIM sets the velocity to the body velocity (0)."""
    o = O.Oracle((64, 32), 0.064, U=(1, 0), body=dict(kind=1, center=(20, 16), radius=6))
    o.set_ic(0)
    o.step(3, tol=1e-10)
    u = o.get_u()
    mu0 = o.mu0()
    assert np.abs(u[mu0 == 0.0]).max() == 0.0


# --------------------------------------------------------------------------- forces
@pytest.mark.parametrize("R", [8, 16])
def test_buoyancy_circle(R):
    """p = g x_d gives F_d = -g pi R^2 (divergence theorem) up to O(eps^2/R^2)."""
    o = O.Oracle((128, 64), 0.064, U=(1, 0), body=dict(kind=1, center=(64, 32), radius=R))
    ny, nx = o.shape
    X, Y = np.meshgrid(np.arange(nx) + 0.5, np.arange(ny) + 0.5)
    for d, field in enumerate((X, Y)):
        o.set_p(2.0 * field)
        F = o.forces()
        assert abs(F[d] / (-2.0 * math.pi * R * R) - 1) < 0.5 / R**2 + 1e-3
        assert abs(F[1 - d]) < 1e-9


def test_buoyancy_sphere():
    R = 12
    o = O.Oracle((64, 64, 64), 0.01, U=(1, 0, 0), body=dict(kind=1, center=(32, 32, 32), radius=R))
    nz, ny, nx = o.shape
    Z, Y, X = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5, indexing="ij")
    o.set_p(X)
    F = o.forces()
    assert abs(F[0] / (-4.0 / 3.0 * math.pi * R**3) - 1) < 0.5 / R**2
    assert abs(F[1]) < 1e-9 and abs(F[2]) < 1e-9


def test_buoyancy_torus():
    """p = x on a torus whose axis is x: F = -V e_x with V = 2 pi^2 R r^2, no side force."""
    R, r = 12, 4
    o = O.Oracle((64, 64, 64), 0.01, U=(1, 0, 0), body=dict(kind=2, center=(32, 32, 32), radius=R, radius2=r))
    nz, ny, nx = o.shape
    Z, Y, X = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5, indexing="ij")
    o.set_p(X)
    F = o.forces()
    assert abs(F[0] / (-2.0 * math.pi**2 * R * r**2) - 1) < 0.5 / r**2
    assert abs(F[1]) < 1e-9 and abs(F[2]) < 1e-9


def test_force_ignores_constant_pressure():
    o = O.Oracle((64, 40), 0.064, U=(1, 0), body=dict(kind=1, center=(21.3, 18.9), radius=5))
    o.set_p(np.full(o.shape, 7.0))
    assert np.abs(o.forces()).max() < 1e-12


# --------------------------------------------------------------------------- sampled SDF body
def _node_grid(dims):
    """Node coordinates (i, j[, k]) of a grid of cells `dims`, arrays shaped reversed(dims + 1)."""
    idx = np.indices(tuple(d + 1 for d in reversed(dims))).astype(float)
    return list(reversed(list(idx)))  # x, y[, z]


def _K0(s):
    s = np.clip(s, -1.0, 1.0)
    return 0.5 + 0.5 * s + np.sin(np.pi * s) / (2 * np.pi)


@pytest.mark.parametrize("dims,a,b", [
    ((24, 16), (0.8, -0.6), 9.3),
    ((20, 16, 12), (0.6, 0.48, 0.64), 9.1),
], ids=["2d", "3d"])
def test_sampled_sdf_planar_is_exact(dims, a, b):
    """A body given by its signed distance at the nodes: multilinear interpolation
    reproduces a linear distance exactly, so for a tilted half-space every face's mu0 is
    K0(d(x_f)/eps) and mu1 is eps K1(d/eps) times the plane's normal, to rounding."""
    a = np.array(a) / np.linalg.norm(a)
    X = _node_grid(dims)
    nodes = sum(a[d] * X[d] for d in range(len(dims))) - b
    o = O.Oracle(dims, 0.05, U=(1.0,) + (0.0,) * (len(dims) - 1), body=dict(kind=3, nodes=nodes))
    mu0, mu1 = o.mu0(), o.mu1()
    centres = list(reversed(list(np.indices(o.shape).astype(float))))
    for c in range(len(dims)):
        x = [centres[d] + 0.5 for d in range(len(dims))]
        x[c] = x[c] - 0.5
        d = sum(a[e] * x[e] for e in range(len(dims))) - b
        assert np.abs(mu0[c] - _K0(d)).max() < 1e-13
        k1 = np.vectorize(O.K1)(d)
        for e in range(len(dims)):
            assert np.abs(mu1[c, e] - k1 * a[e]).max() < 1e-13


def test_sampled_sdf_sphere_volume_and_buoyancy():
    """A sphere's distance sampled at the nodes: the solid volume sum (1 - mu0) and the
    buoyancy of p = x match (4/3) pi R^3 within the interpolation's O(h^2/R) error."""
    R, c, dims = 6.0, (10.3, 8.1, 6.2), (20, 16, 12)
    X = _node_grid(dims)
    nodes = np.sqrt(sum((X[d] - c[d]) ** 2 for d in range(3))) - R
    o = O.Oracle(dims, 0.05, U=(1.0, 0.0, 0.0), body=dict(kind=3, nodes=nodes))
    V = 4.0 / 3.0 * math.pi * R**3
    for comp in range(3):
        assert abs((1 - o.mu0()[comp]).sum() / V - 1) < 0.02
    nz, ny, nx = o.shape
    Z, Y, Xc = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5, indexing="ij")
    o.set_p(Xc)
    F = o.forces()
    assert abs(F[0] / (-V) - 1) < 0.03, F
    assert np.abs(F[1:]).max() < 0.03 * V


def _shear_y2(o, D):
    """u_x = y^2 sampled at the x-faces (y = j + 1/2), other components 0."""
    y = np.arange(o.shape[-2]) + 0.5
    u = np.zeros((D,) + o.shape)
    u[0] = (y**2)[:, None] if D == 2 else (y**2)[None, :, None]
    return u


@pytest.mark.parametrize("D,body,volume,bar", [
    (2, dict(kind=1, radius=9.0), math.pi * 81.0, 0.01),
    (3, dict(kind=1, radius=7.0), 4.0 / 3.0 * math.pi * 343.0, 0.02),
    (3, dict(kind=2, radius=8.0, radius2=3.0), 2.0 * math.pi**2 * 8.0 * 9.0, 0.03),
], ids=["circle", "sphere", "torus"])
def test_viscous_force_closed_form(D, body, volume, bar):
    """For u = (y^2, 0, 0) the strain rate has S_xy = S_yx = y, so by the divergence
    theorem the viscous surface force is 2 nu (div S) V = (2 nu V, 0, 0) with V the body's
    volume; the kernel-weighted cell sum matches it up to O(eps^2/r^2) (mean over seeded
    sub-cell offsets of the body)."""
    nu = 0.04
    n = 48 if D == 2 else 32
    rng = np.random.default_rng(5)
    Fs = []
    for _ in range(6 if D == 2 else 3):
        b = dict(body)
        b["center"] = tuple(n / 2 + rng.random() for _ in range(D))
        o = O.Oracle((n,) * D, nu, U=(0.0,) * D, body=b)
        o.set_ic(0)
        o.set_u(_shear_y2(o, D))
        Fs.append(o.viscous_force())
    F = np.mean(Fs, axis=0)
    ref = 2 * nu * volume
    assert abs(F[0] / ref - 1) < bar, (F, ref)
    assert np.abs(F[1:]).max() < 0.01 * ref, F


@pytest.mark.parametrize("D", [2, 3])
def test_viscous_force_vanishes_for_rigid_motion(D):
    """A uniform translation and a rigid rotation have zero strain rate; the centred
    differences are exact for linear fields, so the force is zero to rounding."""
    n = 24
    b = dict(kind=1, center=(12.3,) * D if D == 2 else (12.3, 11.8, 12.1), radius=5.0)
    o = O.Oracle((n,) * D, 0.05, U=(0.0,) * D, body=b)
    o.set_ic(0)
    # u_x on x-faces (x = i, y = j + 1/2), u_y on y-faces (x = i + 1/2, y = j): rotation about z
    idx = np.indices(o.shape).astype(float)  # (k,) j, i
    i, j = idx[-1], idx[-2]
    u = np.zeros((D,) + o.shape)
    u[0] = 0.3 - 0.7 * (j + 0.5 - 12.0)
    u[1] = -0.2 + 0.7 * (i + 0.5 - 12.0)
    if D == 3:
        u[2] = 0.1
    o.set_u(u)
    assert np.abs(o.viscous_force()).max() < 1e-10


def test_bdim_blend_linear_field():
    """With dt = 0 the stage reduces to the blend u' = mu0 u0 + mu1 . grad u0; for a
    linear field the central difference is the exact gradient, so the blend is
    checked against the analytic slope (mu0 and mu1 are pinned above)."""
    o = O.Oracle((40, 32), 0.05, U=(1, 0), body=dict(kind=1, center=(19.4, 15.8), radius=5.2))
    ny, nx = o.shape
    j, i = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    # u_x at (i, j+1/2), u_y at (i+1/2, j)
    ux = 0.3 + 0.1 * i + 0.2 * (j + 0.5)
    uy = -0.4 + 0.05 * (i + 0.5) - 0.15 * j
    u0 = np.stack([ux, uy])
    out = o.bdim_stage(1, 0.0, u0)
    mu0, mu1 = o.mu0(), o.mu1()
    grad = [(0.1, 0.2), (0.05, -0.15)]
    sl = (slice(4, ny - 4), slice(4, nx - 4))  # away from the walls
    for c in range(2):
        ref = mu0[c] * u0[c] + mu1[c, 0] * grad[c][0] + mu1[c, 1] * grad[c][1]
        assert np.abs(out[c][sl] - ref[sl]).max() < 1e-13


def test_cfl_nonuniform_field():
    """dt uses the largest per-cell out-flux sum_c max(0,u_c[I+e_c]) + max(0,-u_c[I])."""
    o = O.Oracle((8, 6), 0.01, periodic=3)
    u = np.zeros((2,) + o.shape)
    u[0][2, 3] = -2.0   # lower x-face of cell (3,2): out-flux 2 from that cell
    u[0][2, 4] = 3.0    # upper x-face of cell (3,2): out-flux 3 -> cell (3,2) sums to 5
    u[1][5, 1] = -1.5   # cell (1,5) lower y-face: 1.5
    o.set_u(u)
    assert abs(o.cfl() - 1.0 / (5.0 + 4 * 0.01)) < 1e-15


def test_multigrid_projection_reaches_tol():
    """project! with the V-cycle solver stops at ||z - A x||_inf <= tol and lands
    within the tolerance-induced gap of the tight PCG projection."""
    def run(solver, tol):
        o = O.Oracle((64, 32), 0.064, U=(1, 0), body=dict(kind=1, center=(16, 16), radius=5))
        rng = np.random.default_rng(11)
        o.set_u(o.mu0() * (1.0 + 0.1 * rng.standard_normal((2,) + o.shape)))
        it, res = o.project(1.0, 0.5, tol=tol, maxit=40 if solver else 100000, solver=solver)
        return o, it, res
    o1, it1, res1 = run(1, 1e-9)
    assert res1 <= 1e-9 and 3 <= it1 <= 20
    assert np.abs(o1.divergence()).max() <= 1.0001e-9
    o0, _, _ = run(0, 1e-12)
    assert np.abs(o1.get_u() - o0.get_u()).max() < 1e-7
