"""The polynomials of the FP32 small rotation (sin theta, cos theta - 1 on
|theta| <= pi/4, after the quarter turn is split off) meet the error bounds
stated beside them, and are what the committed fitting procedure produces."""
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "paper_1007_3470_gb300", "csrc", "hfs_phase.cuh")


def _constants():
    text = open(HEADER).read()
    # as the compiler reads them: the decimal literal rounded to FP32
    vals = {m.group(1): float(np.float32(float(m.group(2))))
            for m in re.finditer(r"(k(?:Sin|Cos)\d)\s*=\s*([-+0-9.e]+)f", text)}
    return [vals["kSin3"], vals["kSin5"], vals["kSin7"]], [vals["kCos2"], vals["kCos4"], vals["kCos6"], vals["kCos8"]]


def test_rotation_polynomials_meet_stated_bounds():
    from paper_1007_3470_gb300 import fit_rotation_poly as F
    sc, cc = _constants()
    assert len(sc) == 3 and len(cc) == 4 and cc[0] == -0.5
    es, ec = F.errors(sc, cc)
    assert es <= 4.0e-9 and ec <= 8.9e-10
    # against sin / cos themselves at a few angles, including the interval end
    th = np.array([1e-3, 0.1, 0.5, np.pi / 4])
    s = th * th
    sn = th + th ** 3 * (sc[0] + s * (sc[1] + s * sc[2]))
    cm1 = s * (cc[0] + s * (cc[1] + s * (cc[2] + s * cc[3])))
    np.testing.assert_allclose(sn, np.sin(th), rtol=5e-9, atol=0)
    np.testing.assert_allclose(cm1, -2 * np.sin(th / 2) ** 2, rtol=1e-9, atol=0)
    # |1 + cm1 - i sn|^2 - 1: the magnitude error per rotation stays far below one FP32 ulp
    assert np.max(np.abs((1 + cm1) ** 2 + sn ** 2 - 1)) < 5e-9


def test_fitting_procedure_reproduces_the_constants():
    from paper_1007_3470_gb300 import fit_rotation_poly as F
    sc, cc = _constants()
    fs, fc = F.fit()
    for a, b in zip(sc + cc, fs + fc):
        ulp = np.spacing(np.float32(abs(a)))
        assert abs(a - b) <= 2 * ulp, (a, b)
