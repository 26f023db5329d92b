"""Pins of the oracle's adaptive RKF45 (Sect. 2.1.1 names Runge-Kutta-Fehlberg
beside RK4 and Euler-forward).

On the linear solid-body rotation field (bilinear interpolation is exact
there), one trial of length h maps X to R4(hA) X (fourth order) and R5(hA) X
(fifth order), with the published stability polynomials of the Fehlberg 4(5)
pair, R4(z) = 1 + z + z^2/2 + z^3/6 + z^4/24 + z^5/104 and R5(z) = 1 + z +
z^2/2 + z^3/6 + z^4/24 + z^5/120 + z^6/2080.  The step-size controller is
pinned by exact step counts, since the trial error on a circle depends on h
only.
"""
import numpy as np
import pytest

import oracle as O
import synth

DAY = 86400.0


def _poly(z, coeffs):
    return sum(c * z ** i for i, c in enumerate(coeffs))


R4 = [1.0, 1.0, 1 / 2, 1 / 6, 1 / 24, 1 / 104]
R5 = [1.0, 1.0, 1 / 2, 1 / 6, 1 / 24, 1 / 120, 1 / 2080]


def _rotation():
    spec = synth.solid_body_rotation()
    f = O.Field(spec.lon, spec.lat, spec.depth, spec.times, spec.data)
    return f, 2 * np.pi / DAY


def _matrix_poly(coeffs, M):
    out = np.zeros_like(M)
    P = np.eye(2)
    for c in coeffs:
        out = out + c * P
        P = P @ M
    return out


@pytest.mark.parametrize("h", [300.0, 1800.0, -900.0])
def test_trial_is_the_fehlberg_stability_polynomials(h):
    f, w = _rotation()
    A = np.array([[0.0, -w], [w, 0.0]])
    x0 = np.array([1000.0, 2500.0])
    r, x4, err = O.rkf45_trial(f, 0.0, x0[0], x0[1], 0.0, h)
    assert r == 0
    want4 = _matrix_poly(R4, h * A) @ x0
    want5 = _matrix_poly(R5, h * A) @ x0
    np.testing.assert_allclose(x4[:2], want4, rtol=0, atol=1e-9)
    e = np.max(np.abs(want5 - want4))
    assert abs(err - e) <= 1e-9 + 1e-6 * e, (err, e)


def test_fourth_order_convergence_to_the_circle():
    """Fixed steps (tolerance never exceeded, no doubling): the distance to
    the exact circle after one rotation falls 16-fold per halving of h."""
    f, w = _rotation()
    errs = []
    for h in (1800.0, 900.0, 450.0):
        st = dict(lon=np.array([1000.0]), lat=np.array([2500.0]), depth=np.zeros(1),
                  time=np.zeros(1), ids=np.zeros(1, np.uint64), step=np.zeros(1, np.uint32),
                  status=np.zeros(1, np.uint8))
        k = O.Kernel(O.RKF45, rk45_tol=1e9, rk45_hmin=1.0, rk45_hmax=h)
        O.run(f, k, st["lon"], st["lat"], st["depth"], st["time"], st["ids"], st["step"],
              st["status"], h, DAY, DAY, nthreads=1)
        assert st["step"][0] == int(round(DAY / h))
        errs.append(np.hypot(st["lon"][0] - 1000.0, st["lat"][0] - 2500.0))
    assert 14.0 < errs[0] / errs[1] < 18.0 and 14.0 < errs[1] / errs[2] < 18.0, errs


def _steps(f, tol, h, hmax, T, stops=None, dt_sign=1.0):
    st = dict(lon=np.array([1000.0]), lat=np.array([2500.0]), depth=np.zeros(1),
              time=np.zeros(1), ids=np.zeros(1, np.uint64), step=np.zeros(1, np.uint32),
              status=np.zeros(1, np.uint8))
    hstep = np.zeros(1)
    k = O.Kernel(O.RKF45, rk45_tol=tol, rk45_hmin=1.0, rk45_hmax=hmax)
    times = []
    for ts in (stops or []) + [dt_sign * T]:
        O.run(f, k, st["lon"], st["lat"], st["depth"], st["time"], st["ids"], st["step"],
              st["status"], dt_sign * h, ts, dt_sign * T, nthreads=1, hstep=hstep)
        times.append(st["time"][0])
    return int(st["step"][0]), hstep[0], times


def test_step_size_controller_by_exact_counts():
    f, w = _rotation()
    h = 600.0
    _, _, e_h = O.rkf45_trial(f, 0.0, 1000.0, 2500.0, 0.0, h)
    _, _, e_2h = O.rkf45_trial(f, 0.0, 1000.0, 2500.0, 0.0, 2 * h)
    assert 25.0 < e_2h / e_h < 40.0             # fifth-order local error
    T = 6 * 3600.0
    # tolerance below the error at h, above 10x the error at h/2: every
    # trial at h is rejected, h/2 is accepted and doubles back to h
    n, hp, _ = _steps(f, e_h / 2.0, h, h, T)
    assert n == int(T / (h / 2)) and hp == h
    # tolerance above the error at h but below 10x it: steps of h, no doubling
    n, hp, _ = _steps(f, e_h * 2.0, h, 8 * h, T)
    assert n == int(T / h) and hp == h
    # small errors: the step doubles after each step up to the maximum 4h
    n, hp, _ = _steps(f, e_2h * 100.0, h, 4 * h, T)
    assert n == 2 + int(np.ceil((T - 3 * h) / (4 * h))) and hp == 4 * h   # last one shortened
    # backward in time: the same counts
    n, hp, _ = _steps(f, e_h / 2.0, h, h, T, dt_sign=-1.0)
    assert n == int(T / (h / 2)) and hp == -h


def test_steps_land_on_output_and_end_times():
    """Steps are shortened to land on each stop (output) time and on the end
    time; the shortened step neither doubles nor changes the particle's step
    length."""
    f, w = _rotation()
    stops = [1000.0, 5000.0, 5001.0]
    n, hp, times = _steps(f, 1e9, 900.0, 900.0, 7777.0, stops=stops)
    assert times == stops + [7777.0]
    # 0-900-1000 | 1000-1900-2800-3700-4600-5000 | 5000-5001 | 5001-5901-6801-7701-7777
    assert n == 2 + 5 + 1 + 4 and hp == 900.0
