"""The library's FP64 exponential (Tang's table-driven method) against
CUDA's exp and an extended-precision reference: within 1.5 ulp of the exact
value, at most 2 ulp from CUDA's exp (each is within about 1 ulp of exact),
identical outside |x| < 704 (where it defers to the library)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def ulp_distance(a, b):
    ia = a.view(np.int64)
    ib = b.view(np.int64)
    # map to a monotone integer line
    ia = np.where(ia < 0, np.int64(-0x8000000000000000) - ia, ia)
    ib = np.where(ib < 0, np.int64(-0x8000000000000000) - ib, ib)
    return np.abs(ia - ib)


def test_pj_exp_within_one_ulp_of_cuda_exp():
    import torch
    import paper_1809_01029_gb300 as pj
    from paper_1809_01029_gb300 import build
    build.build()
    h = pj.pj_mech_create(synth.make_mechanism("h2co13"))
    rng = np.random.default_rng(3)
    x = np.concatenate([
        rng.uniform(-745.0, 710.0, 2_000_000),
        rng.uniform(-1.0, 1.0, 1_000_000),
        rng.uniform(-80.0, 80.0, 1_000_000),
        np.linspace(-704.5, -703.5, 10001), np.linspace(703.5, 704.5, 10001),
        np.arange(-2000, 2000) * (np.log(2) / 256),       # table nodes and reduction boundaries
        np.arange(-2000, 2000) * (np.log(2) / 512),
        [0.0, -0.0, 1e-300, -1e-300, 5e-324, 708.0, 709.78, 709.79, -708.3, -745.1, -745.2, 1e3, -1e3,
         np.inf, -np.inf, np.nan],
    ])
    d = torch.from_numpy(x).cuda()
    yo = torch.empty_like(d)
    yl = torch.empty_like(d)
    pj.pj_diag_exp(h, len(x), d, yo, yl)
    yo = yo.cpu().numpy()
    yl = yl.cpu().numpy()
    fin = np.isfinite(yl)
    assert np.array_equal(np.isnan(yo), np.isnan(yl))
    assert np.array_equal(yo[~fin & ~np.isnan(yl)], yl[~fin & ~np.isnan(yl)])
    dist = ulp_distance(yo[fin], yl[fin])
    assert dist.max() <= 2, (int(dist.max()), x[fin][np.argmax(dist)])
    big = np.abs(x) >= 704
    assert np.array_equal(yo[big & fin], yl[big & fin])
    # error against an extended-precision exp (long double), in ulps of the result
    sm = np.flatnonzero(np.abs(x) < 700)[:400000]
    exact = np.exp(x[sm].astype(np.longdouble))
    ulp = np.spacing(exact.astype(np.float64)).astype(np.longdouble)
    err = np.abs(yo[sm].astype(np.longdouble) - exact) / ulp
    assert float(err.max()) <= 1.5, float(err.max())
