"""Error bars for correlated Monte Carlo time series (test helper).

Blocking analysis (H. Flyvbjerg and H. G. Petersen, J. Chem. Phys. 91, 461
(1989)): the series is averaged in pairs repeatedly; the standard error of the
mean estimated from the blocked series grows until the blocks are longer than
the autocorrelation time and then levels off.  The largest estimate over the
levels that keep at least 64 blocks is returned, which errs on the safe side.
"""
import numpy as np


def mean_and_error(x):
    x = np.asarray(x, dtype=np.float64)
    mean = float(x.mean())
    best = 0.0
    y = x.copy()
    while len(y) >= 64:
        err = float(y.std(ddof=1) / np.sqrt(len(y)))
        best = max(best, err)
        n2 = len(y) // 2
        y = 0.5 * (y[0:2 * n2:2] + y[1:2 * n2:2])
    return mean, best


def z_score(x, exact):
    mean, err = mean_and_error(x)
    if err == 0.0:
        return 0.0 if mean == exact else float("inf")
    return (mean - exact) / err
