"""Gradient-driven calibration on the GPU (Sec. 3.2 triaxial target).

Three small triaxial cells, consolidated to the paper's confining stresses
5, 15 and 25 kPa and loaded by a short shear, give one residual each:
(sigma_1 - K sigma_3) / sigma_3 averaged over a 40-step window, K from the
friction angle of Table 1.  The Jacobian of the residuals in (mu_t, mu_r) from
the hand-written adjoint equals central differences of the same windows
(h = 1e-3 relative), and so does the Gauss-Newton step built from it.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def windows():
    from paper_2501_05300_gb300 import calibrate, dem, triaxial
    K = triaxial.K_of_phi(34.0)
    out = []
    for s3 in (5e3, 15e3, 25e3):
        bed, _ = calibrate.consolidated_cell(dem, 1500, s3, seed=2601)
        bed.set_material(mu_t=0.3, mu_r=0.02)
        triaxial.shear(bed, s3, 0.5, 0.004)
        start = bed.save_checkpoint()
        out.append(calibrate.FailureWindow(bed, start, s3, K, strain=0.0, steps=40, reshear=False))
    yield out
    for w in out:
        w.bed.close()


def test_gauss_newton_step_agrees_with_central_differences(windows):
    from paper_2501_05300_gb300 import calibrate
    theta = np.array([1.0, 0.3, 0.02])
    free = [1, 2]
    r, J = [], []
    for w in windows:
        v, g = w.evaluate(theta)
        r.append(v)
        J.append(g[free])
        assert w.last["sigma1"] > w.last["sigma3"] > 0      # a loaded, sheared sample
    r, J = np.array(r), np.array(J)
    Jfd = np.zeros_like(J)
    for j, i in enumerate(free):
        h = 1e-3 * theta[i]
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        for k, w in enumerate(windows):
            Jfd[k, j] = (w.evaluate(tp, grad=False)[0] - w.evaluate(tm, grad=False)[0]) / (2 * h)
    assert np.abs(Jfd).max() > 0
    assert np.abs(J - Jfd).max() <= 1e-2 * np.abs(Jfd).max(), (J, Jfd)
    d = calibrate.gauss_newton_step(r, J, damping=1e-3)
    dfd = calibrate.gauss_newton_step(r, Jfd, damping=1e-3)
    assert np.linalg.norm(d - dfd) <= 2e-2 * np.linalg.norm(dfd), (d, dfd)
    # the residual of the same window is reproducible (restore + record)
    again = windows[0].evaluate(theta, grad=False)[0]
    assert again == r[0]
