"""wl_profile_step on a fine level split into band and uniform tiles: the two launches of
each fine sweep and residual pass are timed on their own streams (the *_uni and *_bandt
classes) beside the pair's wall time, once per pair; on a level that does not split they
are absent.  The profiled steps are the same steps as wl_step (identical state)."""
import numpy as np
import pytest

from tests.gpu_cases import make_pair

pytestmark = pytest.mark.gpu

CASE = dict(id="sphere128x64x64", dims=(128, 64, 64), nu=0.02, U=(1.0, 0.0, 0.0), periodic=0,
            body=dict(kind=1, center=(40.0, 32.3, 31.7), radius=6.0))


def test_split_launches_timed_one_by_one(monkeypatch):
    monkeypatch.setenv("WL_UNIFORM_ALL", "1")  # split every level, whatever its band fraction
    a, _ = make_pair(CASE, oracle=False)
    b, _ = make_pair(CASE, oracle=False)
    monkeypatch.delenv("WL_UNIFORM_ALL")
    assert a.level_split(0)[0] == 1
    prof = a.profile_step(2)
    b.step(2)
    for cls in ("sweep_fine", "resid_fine"):
        ms, n = prof[cls]
        assert n > 0 and ms > 0.0
        for part in ("_uni", "_bandt"):
            pms, pn = prof[cls + part]
            assert pn == n, (cls, part, pn, n)
            # each launch starts after the pair's first event and ends before its last
            assert 0.0 < pms <= ms * 1.001, (cls, part, pms, ms)
    # the host-driven steps are the graph steps
    assert np.array_equal(a.get(0), b.get(0))
    assert np.array_equal(a.get(1), b.get(1))


def test_unsplit_level_has_no_split_classes(monkeypatch):
    monkeypatch.setenv("WL_NO_UNIFORM", "1")
    a, _ = make_pair(CASE, oracle=False)
    monkeypatch.delenv("WL_NO_UNIFORM")
    assert a.level_split(0)[0] == 0
    prof = a.profile_step(1)
    assert prof["sweep_fine"][1] > 0
    for cls in ("sweep_fine_uni", "sweep_fine_bandt", "resid_fine_uni", "resid_fine_bandt"):
        assert prof[cls][1] == 0, cls
