"""The arctangent polynomial of the step kernels: the coefficients in mdg_step.cu are the
ones paper_2606_08039_gb300/csrc/fit_atan.py fits (Lawson's near-minimax fit of atan on
[0, 1], rounded to float32), and their float32 evaluation stays within 1.4e-7 rad. CPU only:
the CUDA source is read as text."""
import importlib.util
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2606_08039_gb300", "csrc")


def _fit_module():
    spec = importlib.util.spec_from_file_location("fit_atan", os.path.join(CSRC, "fit_atan.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _kernel_coefficients():
    src = open(os.path.join(CSRC, "mdg_step.cu")).read()
    body = src[src.index("float atan2_fast(float y, float x)"):]
    body = body[:body.index("float r = a * p;")]
    vals = [float(v) for v in re.findall(r"(-?\d+\.\d+(?:e-?\d+)?)f", body)]
    # the Horner chain: fmaf(s, c7, c6), then fmaf(p, s, c5) ... fmaf(p, s, c0)
    horner = vals[vals.index(1.17549435e-38) + 1:] if 1.17549435e-38 in vals else vals
    c7, c6, rest = horner[0], horner[1], horner[2:]
    return np.array(list(reversed(rest)) + [c6, c7], dtype=np.float32)


def test_kernel_coefficients_are_the_fit():
    fit = _fit_module()
    c = fit.fit()
    k = _kernel_coefficients()
    assert k.shape == c.shape == (fit.N_TERMS,)
    np.testing.assert_array_equal(k, c)


def test_float32_error_bound():
    fit = _fit_module()
    assert fit.float32_error(_kernel_coefficients()) < 1.4e-7
