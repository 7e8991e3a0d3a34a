"""Measured WCET curves (§3, Fig. 1's blocker method): the fit of
C(m) = a / m + b on the host, and on the GPU the placement (the kernel under
test on exactly m SMs, disjoint from the blocker's) and the expected
scaling and interference."""
import numpy as np
import pytest

import paper_2105_10312_gb300 as gpa


def test_fit_recovers_the_model_exactly():
    m = np.array([1, 2, 3, 8, 19, 76, 152])
    for a, b in ((3.0, 0.5), (0.25, 0.0), (0.0, 1.5), (12.5, 0.031)):
        fa, fb = gpa.fit_wcet(m, a / m + b)
        assert fa == pytest.approx(a, rel=1e-12, abs=1e-12) and fb == pytest.approx(b, rel=1e-12, abs=1e-12)


def test_fit_is_the_least_squares_solution():
    rng = np.random.default_rng(5)
    m = rng.integers(1, 153, 40)
    y = 2.0 / m + 0.3 + rng.normal(0, 0.05, 40)
    fa, fb = gpa.fit_wcet(m, y)
    X = np.stack([1.0 / m, np.ones(40)], axis=1)
    (ra, rb), *_ = np.linalg.lstsq(X, y, rcond=None)
    assert fa == pytest.approx(ra, rel=1e-9) and fb == pytest.approx(rb, rel=1e-9)


def test_fit_skips_failed_points_and_rejects_degenerate_input():
    m = np.array([1, 2, 4, 8])
    y = 4.0 / m + 1.0
    y_bad = y.copy()
    y_bad[1] = -1.0  # no valid repetition at m = 2
    assert gpa.fit_wcet(m, y_bad) == pytest.approx((4.0, 1.0))
    for mm, yy in (([4, 4, 4], [1.0, 1.1, 0.9]), ([1, 2], [-1.0, 3.0]), ([1], [2.0])):
        with pytest.raises(gpa.GpaError) as ei:
            gpa.fit_wcet(np.array(mm), np.array(yy))
        assert ei.value.code == gpa.ERR_ARG


@pytest.mark.gpu
def test_placement_and_scaling_on_the_gpu(ctx):
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    m = [4, sms // 4, sms // 2, sms]
    comp, used = gpa.measure_wcet(ctx, "COMPUTE", m, 1 << 24, reps=3)
    assert list(used) == m, used
    # compute time scales with 1 / m (measured: C(4) = 19 C(152), against 38 for an ideal 1 / m)
    assert (comp > 0).all() and comp[0] > 0.25 * (sms / 4) * comp[-1]
    a, b = gpa.fit_wcet(m, comp)
    assert a > 0 and abs(a / m[0] + b - comp[0]) < 0.2 * comp[0]
    vadd, used = gpa.measure_wcet(ctx, "VADD", m, 1 << 24, reps=3)
    assert list(used) == m and (vadd > 0).all() and vadd[0] > vadd[-1]
    # half the SMs streaming HBM (about 4 TB/s) beside a memory-bound kernel
    # on the other half: measured 1.13x slower; repetitions agree within 1 %
    vi, used_i = gpa.measure_wcet(ctx, "VADD", [sms // 2], 1 << 24, reps=3, interfere=True)
    assert used_i[0] == sms // 2 and vi[0] > 1.05 * vadd[2]
    for k, n in (("TRANSPOSE", 2048), ("STENCIL", 2048)):
        t, u = gpa.measure_wcet(ctx, k, [8, sms], n, reps=2)
        assert list(u) == [8, sms] and t[0] > t[1] > 0


@pytest.mark.gpu
def test_probe_kernels_compute_what_they_claim(ctx):
    """Each kernel the measurement times, run on seeded data, against NumPy:
    the vector add and the transpose exactly; the stencil sweep and the
    64-step multiply-add chain within float32 rounding (the device fuses
    multiply and add, NumPy does not; the chain contracts, |a| < 1)."""
    rng = np.random.default_rng(9)
    for n, ctas in ((1, 1), (1000003, 0), (4099, 3)):
        a = rng.standard_normal(n).astype(np.float32)
        b = rng.standard_normal(n).astype(np.float32)
        assert np.array_equal(gpa.probe_run(ctx, "VADD", n, a, b, ctas=ctas), a + b)
    for n in (32, 100, 1031):
        a = rng.standard_normal((n, n)).astype(np.float32)
        assert np.array_equal(gpa.probe_run(ctx, "TRANSPOSE", n, a).reshape(n, n), a.T)
        p = np.pad(a.astype(np.float64), 1, mode="edge")
        want = a + 0.1 * (p[1:-1, :-2] + p[1:-1, 2:] + p[:-2, 1:-1] + p[2:, 1:-1] - 4 * a.astype(np.float64))
        got = gpa.probe_run(ctx, "STENCIL", n, a).reshape(n, n)
        assert np.allclose(got, want, rtol=1e-5, atol=1e-5)
    x = rng.uniform(-0.99, 0.99, 100003).astype(np.float32)
    y = np.ones_like(x, dtype=np.float64)
    for _ in range(64):
        y = y * x + 0.5
    got = gpa.probe_run(ctx, "COMPUTE", len(x), x)
    assert np.allclose(got, y, rtol=1e-5, atol=1e-5)
    with pytest.raises(gpa.GpaError) as ei:
        gpa.probe_run(ctx, "TRANSPOSE", 16, np.zeros(256, np.float32))
    assert ei.value.code == gpa.ERR_RANGE


@pytest.mark.gpu
def test_measure_rejects_bad_arguments(ctx):
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for kw, code in ((dict(kernel="VADD", m=[0], n=1024), gpa.ERR_RANGE),
                     (dict(kernel="VADD", m=[sms + 1], n=1024), gpa.ERR_RANGE),
                     (dict(kernel="TRANSPOSE", m=[4], n=16), gpa.ERR_RANGE),
                     (dict(kernel="VADD", m=[4], n=1024, reps=0), gpa.ERR_RANGE)):
        with pytest.raises(gpa.GpaError) as ei:
            gpa.measure_wcet(ctx, **kw)
        assert ei.value.code == code
