"""Coefficients of the float32 complementary error function of the real-space pair kernels.

The kernels need erfc(x) and exp(-x^2) of the same argument (potential and force of one pair), so
erfc is written as erfc(x) = exp(-x^2) R(x) and only R is approximated: R(x) = erfcx(x), the
scaled complementary error function, is smooth and slowly varying on x >= 0, and
R(x) ~ t (c_1 + c_2 t + ... + c_n t^(n-1)) with t = 1 / (1 + p x)
is the form of Hastings' approximations (Abramowitz & Stegun 7.1.25-7.1.26).  Here n = 8 and the
coefficients are fitted to the RELATIVE error of R on 0 <= x <= 6.5 (the kernels use x = alpha r
up to alpha r_c and x = eta r up to 6.5, beyond which erfc(eta r) is dropped) by iteratively
reweighted least squares toward the minimax solution.  The fit's relative error is below 4e-8,
under the float32 rounding of the evaluation itself, so float32 sums of many pairs carry no
systematic approximation error (7.1.26's 1.5e-7 absolute error is 3e-5 relative at x = 2).

Run as a script to print the table used in csrc/cpm_step.cu (PairMath<float>).
"""
import numpy as np
from scipy.special import erfcx

X_MAX = 6.5
N_TERMS = 8
P = 0.42


def fit(n=N_TERMS, p=P, x_max=X_MAX, iters=60):
    x = np.linspace(0.0, x_max, 20001)
    R = erfcx(x)
    t = 1.0 / (1.0 + p * x)
    V = np.stack([t ** (k + 1) for k in range(n)], axis=1)
    w = np.ones_like(x)
    for _ in range(iters):
        c = np.linalg.lstsq(V * (w / R)[:, None], R * (w / R), rcond=None)[0]
        e = (V @ c - R) / R
        w = w * (np.abs(e) / np.abs(e).max() + 1e-3) ** 0.5
    return c, float(np.max(np.abs((V @ c - R) / R)))


if __name__ == "__main__":
    c, err = fit()
    print(f"// p = {P}, n = {N_TERMS}, max relative error of R on [0, {X_MAX}]: {err:.2e}")
    print(", ".join(f"{v:.9e}f" for v in c))
