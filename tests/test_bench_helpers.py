"""Host-side measurement helpers of bench.py (CPU): the per-output error
measure, the analytic derivatives of the sinusoid test fields (checked against
central differences of the fields themselves) and the FP64 oracle's
reordering spread."""
import math

import numpy as np

import bench
from paper_2405_13165_gb300 import clouds as C


def _field_values(modes, x):
    """u, v, w, p of the sinusoid modes at points x [N,3] (FP64)."""
    out = np.zeros((x.shape[0], 4))
    for f, kx, ky, kz, phi in modes:
        out[:, f] += np.sin(x @ np.array([kx, ky, kz]) + phi)
    return out


def test_error_per_output_measures():
    rng = np.random.default_rng(3)
    b = rng.normal(size=(50, 16))
    e = bench.error_per_output(b.copy(), b)
    assert all(v["normwise"] == 0.0 and v["p99"] == 0.0 for v in e.values())
    a = b.copy()
    col = 5   # v.dy
    a[7, col] += 1e-3 * np.abs(b[:, col]).max()
    e = bench.error_per_output(a, b)
    assert math.isclose(e[bench.COLUMNS[col]]["normwise"], 1e-3, rel_tol=1e-3)
    assert all(v["normwise"] == 0.0 for k, v in e.items() if k != bench.COLUMNS[col])


def test_sinusoid_modes_reproduce_the_generated_fields():
    c = C.config_small()
    assert len(c.field_modes) == 16   # 4 fields x 4 modes
    got = _field_values(c.field_modes, c.pos_h[:, :3].astype(np.float64))
    np.testing.assert_allclose(got, c.vp, rtol=0, atol=2e-6)   # vp is stored in FP32


def test_analytic_derivatives_match_central_differences():
    """3D rows: gradient and Laplacian; film rows (on z = 0, normal +z): the
    in-plane gradient and Laplacian.  Outputs set to fourth-order central
    differences of the fields give the analytic figure ~0."""
    c = C.config_small()
    rows = np.concatenate([np.flatnonzero(c.model == 0)[:40], np.flatnonzero(c.model == 1)[:40]])
    sub = c.take(rows)
    x = sub.pos_h[:, :3].astype(np.float64)
    film = sub.model == 1
    h = 1e-3
    out = np.zeros((sub.n, 4, 4))
    for a in range(3):
        d = np.zeros(3)
        d[a] = h
        fp, fm = _field_values(c.field_modes, x + d), _field_values(c.field_modes, x - d)
        fp2, fm2 = _field_values(c.field_modes, x + 2 * d), _field_values(c.field_modes, x - 2 * d)
        f0 = _field_values(c.field_modes, x)
        grad = (8 * (fp - fm) - (fp2 - fm2)) / (12 * h)
        second = (-fp2 + 16 * fp - 30 * f0 + 16 * fm - fm2) / (12 * h * h)
        if a == 2:
            grad[film] = 0.0
            second[film] = 0.0
        out[:, :, a] = grad
        out[:, :, 3] += second
    r = bench.analytic_consistency(sub, out.reshape(sub.n, 16))
    assert r["max_normwise"] < 1e-6, r["per_output"]
    # a dropped sign in the Laplacian is caught
    out[:, :, 3] *= -1.0
    r = bench.analytic_consistency(sub, out.reshape(sub.n, 16))
    assert r["per_output"]["u.lap"]["normwise"] > 1.0


def test_oracle_reorder_spread_is_at_rounding_on_the_small_cloud():
    r = bench.oracle_reorder_spread(C.cell_sorted(C.config_small()))
    assert 0.0 < r["max_normwise"] < 1e-10
