"""Seeded inputs shared by the GPU parity tests: grid/body configurations and a
helper that builds the same case on both sides.  Holds none of the method's
arithmetic."""
import numpy as np

def sampled_nodes(dims, sdf):
    """The signed distance sdf(x, y[, z]) sampled at the nodes of a grid of cells `dims`
    (node (i, j[, k]) at position (i, j[, k])), shaped reversed(dims + 1), in FP32 (the
    library's input type, so that both sides see the same values)."""
    idx = np.indices(tuple(d + 1 for d in reversed(dims))).astype(float)
    return sdf(*reversed(list(idx))).astype(np.float32)


def rounded_box(centre, half, r):
    """Exact signed distance of a box of half-sides `half` with edges rounded by r."""
    def f(*x):
        q = [np.abs(x[d] - centre[d]) - half[d] for d in range(len(x))]
        outside = np.sqrt(sum(np.maximum(v, 0.0) ** 2 for v in q))
        inside = np.minimum(np.maximum.reduce(q), 0.0)
        return outside + inside - r
    return f


CASES_2D = [
    dict(id="cyl64x32", dims=(64, 32), nu=0.064, U=(1.0, 0.0), periodic=0,
         body=dict(kind=1, center=(16.0, 16.0), radius=5.0)),
    dict(id="ragged37x29", dims=(37, 29), nu=0.03, U=(0.8, 0.1), periodic=0,
         body=dict(kind=1, center=(15.3, 13.7), radius=4.2)),
    dict(id="per32", dims=(32, 32), nu=0.02, U=(0.0, 0.0), periodic=3, body=None),
    dict(id="xper96x40", dims=(96, 40), nu=0.05, U=(1.0, 0.0), periodic=1,
         body=dict(kind=1, center=(30.5, 20.0), radius=6.0)),
    dict(id="sdfbox48x32", dims=(48, 32), nu=0.05, U=(1.0, 0.0), periodic=0,
         body=dict(kind=3, nodes=sampled_nodes((48, 32), rounded_box((16.3, 15.6), (4.0, 2.5), 1.5)))),
]
CASES_3D = [
    dict(id="sph40x24x20", dims=(40, 24, 20), nu=0.02, U=(1.0, 0.0, 0.0), periodic=0,
         body=dict(kind=1, center=(14.2, 11.9, 10.3), radius=4.5)),
    dict(id="per16", dims=(16, 16, 16), nu=0.01, U=(0.0, 0.0, 0.0), periodic=7, body=None),
    dict(id="zper64x32x32", dims=(64, 32, 32), nu=0.01, U=(1.0, 0.0, 0.0), periodic=4,
         body=dict(kind=1, center=(20.0, 16.0, 16.0), radius=6.0)),
    dict(id="ragged35x21x19", dims=(35, 21, 19), nu=0.015, U=(0.6, 0.2, -0.1), periodic=2,
         body=dict(kind=1, center=(12.7, 10.1, 9.4), radius=3.6)),
    dict(id="torus48x32x32", dims=(48, 32, 32), nu=0.02, U=(1.0, 0.0, 0.0), periodic=0,
         body=dict(kind=2, center=(14.0, 16.3, 15.8), radius=8.0, radius2=3.0)),
    dict(id="sdfbox40x24x20", dims=(40, 24, 20), nu=0.02, U=(1.0, 0.0, 0.0), periodic=0,
         body=dict(kind=3, nodes=sampled_nodes((40, 24, 20), rounded_box((13.7, 12.2, 9.9), (3.0, 2.0, 2.5), 1.2)))),
]


def make_pair(case, oracle=True, **kw):
    from paper_2304_08159_gb300 import Sim
    import oracle as O

    opts = dict(tol=1e-6)
    opts.update(kw)
    sim = Sim(case["dims"], case["nu"], case["U"], body=case["body"], periodic=case["periodic"], **opts)
    ref = None
    if oracle:
        ref = O.Oracle(case["dims"], case["nu"], U=case["U"], periodic=case["periodic"], body=case["body"])
        ref.set_ic(0)
    return sim, ref


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def active_mask(ref):
    return ref.poisson_diag() > 0
