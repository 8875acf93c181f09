"""Coefficients of the arctangent polynomial of mdg_step.cu (atan2_fast).

atan(a) on [0, 1] is approximated by the odd polynomial a * P(a^2), P of degree 7. The
coefficients come from a near-minimax fit of the absolute error by Lawson's algorithm
(iteratively reweighted least squares: each pass multiplies a grid point's weight by its
error, which drives the weighted least-squares solution towards equal-ripple error), and
are rounded to float32. Prints them with the error of the float32 Horner evaluation
(fused multiply-adds, as on the GPU) against float64 arctan.

    python paper_2606_08039_gb300/csrc/fit_atan.py
"""
import numpy as np

N_TERMS = 8


def fit(n_terms: int = N_TERMS, passes: int = 400) -> np.ndarray:
    a = np.linspace(0.0, 1.0, 20001)
    f = np.arctan(a)
    basis = np.stack([a ** (2 * k + 1) for k in range(n_terms)], axis=1)
    w = np.full(a.shape, 1.0 / a.size)
    for _ in range(passes):
        sw = np.sqrt(w)
        c, *_ = np.linalg.lstsq(basis * sw[:, None], f * sw, rcond=None)
        e = np.abs(basis @ c - f)
        w = w * e
        w /= w.sum()
    return c.astype(np.float32)


def float32_error(c: np.ndarray) -> float:
    a = np.linspace(0.0, 1.0, 2000001).astype(np.float32)
    s = (a * a).astype(np.float32)
    p = np.full(a.shape, c[-1], dtype=np.float32)
    for k in range(len(c) - 2, -1, -1):  # one rounding per fused multiply-add
        p = (p.astype(np.float64) * s + np.float64(c[k])).astype(np.float32)
    r = (p.astype(np.float64) * a).astype(np.float32)
    return float(np.max(np.abs(r.astype(np.float64) - np.arctan(a.astype(np.float64)))))


if __name__ == "__main__":
    c = fit()
    for k, v in enumerate(c):
        print(f"c{k} = {float(v):.9g}f")
    print(f"max |error| of the float32 evaluation on [0, 1]: {float32_error(c):.3g} rad")
