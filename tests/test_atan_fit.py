"""The atan polynomial of the rollout kernels is reproducible: the minimax fit
(csrc/atan_minimax.py, Remez exchange for the absolute error of
atan(a) = a p(a^2) on [0, 1]) regenerates the float32 literals that the
scalar and the packed atan2 forms (device.cuh) share, its error equioscillates as a minimax error must (Chebyshev's
alternation theorem: at least degree + 2 extrema of equal size and
alternating sign), and the float32 coefficients stay within 2.2e-8."""
import importlib.util
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2302_11719_gb300", "csrc")


def _fit_module():
    spec = importlib.util.spec_from_file_location("atan_minimax",
                                                  os.path.join(CSRC, "atan_minimax.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _literals():
    s = open(os.path.join(CSRC, "device.cuh")).read()
    vals = {int(k): float(v.rstrip("f")) for k, v in
            re.findall(r"constexpr float ATAN_P(\d) = ([-0-9.e+]+f);", s)}
    return [vals[k] for k in range(8, -1, -1)]


def test_fit_regenerates_the_kernel_coefficients():
    A = _fit_module()
    lit = _literals()
    assert len(lit) == 9
    assert A.float32_coefficients() == [float(np.float32(v)) for v in lit]
    # the scalar and the two packed atan2 use these constants; no source holds a copy
    dev = open(os.path.join(CSRC, "device.cuh")).read()
    assert dev.count("ATAN_P8") == 4          # defined, used by atan2_poly, atan2_2, atan2_2_lat
    for f in os.listdir(CSRC):
        if f.endswith((".cu", ".cuh")):
            assert open(os.path.join(CSRC, f)).read().count("%.9e" % lit[0]) == (f == "device.cuh")


def test_fit_is_minimax_and_accurate():
    A = _fit_module()
    c, err = A.fit()
    assert err < 1.0e-8
    s = np.linspace(0.0, 1.0, 200001)
    e = np.sqrt(s) * (A.poly(c, s) - A.f(s))
    # alternation: sign changes of the error between its extrema of near-maximal size
    big = np.abs(e) > 0.98 * np.max(np.abs(e))
    signs = np.sign(e[big])
    runs = 1 + np.count_nonzero(np.diff(signs))
    assert runs >= A.DEGREE + 2
    # the float32 literals evaluated exactly
    lit = np.array(_literals(), dtype=np.float64)
    a = np.linspace(0.0, 1.0, 400001)
    assert np.max(np.abs(a * np.polyval(lit, a * a) - np.arctan(a))) <= 2.2e-8
