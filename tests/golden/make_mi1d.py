"""Writes mi1d_sharp.txt: the paper's closed-form 1D matrix-inclusion strain at the nodes.

Sec. 2.1 eq. FieStnDisIncMat1D: E(x) = E_bar + s_IM nu_tilde(x) E_bar with s_IM = S_IM / S_bar,
i.e. E = E_bar S(x) / S_bar, evaluated with grid averages on the nodes x_i = (i - 1) h of
Sec. 3.1 for the example of Sec. 4 (c_l = l/4, c_r = 3l/4, C_I / C_M = 100, sharp interface,
E_bar = 1).  The nodes never fall on an interface for the grids used here (n = 10, 50, 90 as in
the paper's 1D figures, and n = 18, 54, 162, lengths 2 3^k that the GPU's FFTs accept).
This script evaluates only that closed form.
"""
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def closed_form(n, C_M=1.0, C_I=100.0):
    l = 1.0
    h = l / n
    x = np.arange(n) * h
    nu = ((x > l / 4) & (x < 3 * l / 4)).astype(float)
    S_M, S_I = 1.0 / C_M, 1.0 / C_I
    S = S_M + (S_I - S_M) * nu
    S_bar = S.mean()
    s_IM = (S_I - S_M) / S_bar
    return 1.0 + s_IM * (nu - nu.mean()), nu


if __name__ == "__main__":
    with open(os.path.join(HERE, "mi1d_sharp.txt"), "w") as f:
        f.write("# 1D periodic matrix-inclusion, sharp interface, C_I/C_M = 100, c_l = l/4, c_r = 3l/4\n")
        f.write("# closed form E_i / E_bar (Sec. 2.1 eq. FieStnDisIncMat1D with grid averages)\n")
        f.write("# columns: n i nu_i E_i/E_bar\n")
        for n in (10, 50, 90, 18, 54, 162):
            E, nu = closed_form(n)
            for i in range(n):
                f.write("%d %d %.1f %.17e\n" % (n, i, nu[i], E[i]))
