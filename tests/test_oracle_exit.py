"""Pins of the oracle's convective exit on the upper x face (a reading: the paper's BC!
names the boundary conditions only).  The exit normal velocity is carried out at U_x by
the Heun stages and the exit plane is shifted so that the flux out equals the flux in.
Pinned by invariants, on the CPU in FP64:

* a uniform free stream is a fixed point (exactly);
* after every step the exit plane carries out exactly the inflow (mean of the exit
  velocity = U_x to rounding), and every projection converges with max|div u| <= tol
  (the Neumann problem is solvable only with that balance);
* a flow that is mirror-symmetric about the channel's mid-plane stays so;
* the wake leaves: a domain cut close behind a cylinder stays closer (upstream of the
  cut) to a three-times longer domain with the convective exit than with the Dirichlet
  exit.
"""
import numpy as np

import oracle as O


def _case(exit_on, dims=(64, 32), body=None, nu=0.02, U=(1.0, 0.0)):
    o = O.Oracle(dims, nu, U=U, body=body)
    if exit_on:
        o.set_exit(True)
    o.set_ic(0)
    return o


def test_free_stream_is_fixed_point():
    o = _case(True, dims=(48, 24, 16), U=(0.8, 0.0, 0.0))
    o.step(3, tol=1e-12)
    u = o.get_u()
    assert np.abs(u[0] - 0.8).max() <= 1e-14 and np.abs(u[1:]).max() <= 1e-14
    assert np.abs(o.get_exit() - 0.8).max() <= 1e-14


def test_exit_flux_balance_and_divergence():
    body = dict(kind=1, center=(20.0, 16.3), radius=5.0)
    o = _case(True, dims=(64, 32), body=body, nu=0.03)
    for _ in range(6):
        o.step(1, tol=1e-11)
        e = o.get_exit()
        assert abs(e.mean() - 1.0) <= 1e-12
        assert np.abs(o.divergence()).max() <= 1e-10
    # the exit plane is not uniform: the wake reached it
    assert np.abs(e - 1.0).max() > 1e-6


def test_mirror_symmetry_with_exit():
    body = dict(kind=1, center=(20.0, 16.0), radius=5.0)
    o = _case(True, dims=(64, 32), body=body, nu=0.03)
    o.step(8, tol=1e-12)
    u = o.get_u()
    # u(x, 32 - y) = u, v at face j mirrors to face 32 - j with a sign change
    assert np.abs(u[0] - u[0][::-1, :]).max() <= 1e-10
    v = u[1]
    assert np.abs(v[1:, :] + v[1:, :][::-1, :]).max() <= 1e-10
    e = o.get_exit()
    assert np.abs(e - e[::-1]).max() <= 1e-10


def test_truncated_domain_close_to_long_domain():
    """An outflow condition should let the wake leave: cutting the 2-D cylinder's domain
    24 cells behind the body perturbs the flow upstream of the cut far less with the
    convective exit than with the Dirichlet exit (which forces u_x = U across the wake),
    measured against a domain three times as long (30 steps at fixed dt)."""
    def run(nx, exit_on):
        o = O.Oracle((nx, 32), 0.02, U=(1.0, 0.0), body=dict(kind=1, center=(12.0, 16.3), radius=4.0))
        if exit_on:
            o.set_exit(True)
        o.set_ic(0)
        o.step(30, tol=1e-11, dt_fixed=0.25)
        return o.get_u()

    ref = run(128, False)
    err = {e: np.abs(run(40, e)[:, :, :36] - ref[:, :, :36]).max() for e in (True, False)}
    assert err[True] <= err[False] / 3.0, err
