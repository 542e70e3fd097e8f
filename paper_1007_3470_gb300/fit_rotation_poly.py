"""Fit the polynomials of the FP32 small rotation (kSin*, kCos* in
csrc/hfs_phase.cuh): sin(theta) = theta + theta^3 P(theta^2) with P of degree 2
and cos(theta) - 1 = theta^2 Q(theta^2) with Q of degree 3 on |theta| <= pi/4.

Method: Lawson's algorithm (iteratively reweighted least squares, which
converges to the minimax solution) on Chebyshev nodes, minimising the
relative error; the coefficients are then rounded to FP32 one at a time, the
later ones refitted to the residual after each rounding.  Run as a script to
print the coefficients and the error of the rounded set."""
import numpy as np


def _nodes(m=4000, margin=2e-7):
    a = (np.pi / 4) * (1 + margin)
    th = a * np.cos((np.arange(m) + 0.5) * np.pi / m)
    return th[th > 0]


def _lawson(basis, target, den, iters=400):
    w = np.ones_like(target)
    c = None
    for _ in range(iters):
        sw = np.sqrt(w) / den
        c, *_ = np.linalg.lstsq(basis * sw[:, None], target * sw, rcond=None)
        err = np.abs((basis @ c - target) / den)
        w = w * err
        w /= w.sum()
    return c


def fit():
    th = _nodes()
    s = th * th
    sin_t = (np.sin(th) - th) / th ** 3          # P(s)
    cm1 = -2.0 * np.sin(th / 2) ** 2             # cos(theta) - 1 without cancellation
    cos_t = cm1 / s                              # Q(s)
    out = []
    for target, den, npow in ((sin_t, np.sin(th) / th ** 3, 3), (cos_t, np.abs(cos_t), 4)):
        fixed = []
        for k in range(npow):
            resid = target - sum(c * s ** j for j, c in enumerate(fixed))
            basis = np.stack([s ** j for j in range(k, npow)], axis=1)
            fixed.append(float(np.float32(_lawson(basis, resid, den)[0])))
        out.append(fixed)
    return out


def errors(sin_c, cos_c, n=200001):
    th = np.linspace(1e-4, np.pi / 4 * (1 + 2e-7), n)
    s = th * th
    p = th + th ** 3 * np.polyval(list(reversed(sin_c)), s)
    q = s * np.polyval(list(reversed(cos_c)), s)
    cm1 = -2.0 * np.sin(th / 2) ** 2
    return float(np.max(np.abs(p / np.sin(th) - 1))), float(np.max(np.abs(q / cm1 - 1)))


if __name__ == "__main__":
    sc, cc = fit()
    print("sin:", ["%.9e" % c for c in sc])
    print("cos-1:", ["%.9e" % c for c in cc])
    print("relative errors (sin, cos-1): %.3e %.3e" % errors(sc, cc))
