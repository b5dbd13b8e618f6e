"""Truncated decoupling of a strictly diagonally dominant tridiagonal system
(windows with halos) -- TEST INFRASTRUCTURE.

Not a method of the paper: an approximation that drops the couplings beyond
a halo of h rows around each window, so every window is solved on its own.

Definition
  Windows of R kept rows: window w keeps rows [wR, min((w+1)R, n)).  It is
  solved as the tridiagonal system on its extended rows
  [max(0, wR - h), min(n, (w+1)R + h)) with the couplings that leave that
  range cut (a of the first extended row and c of the last taken as 0); the
  result on the kept rows is the window's answer.  With h >= n (or R >= n)
  every window is the whole system and the answer is the exact solution.

Error bound (derived here, not from the paper)
  For a tridiagonal matrix with q = max_i (|a_i| + |c_i|) / |b_i| < 1, column
  j of the inverse decays away from j: for u = A^{-1} e_j and d > 0 the
  homogeneous rows give |u_i| <= q max(|u_{i-1}|, |u_{i+1}|), so the maximum
  over i >= j + d is at most q times the maximum over i >= j + d - 1, and by
  induction |A^{-1}_{ij}| <= q^{|i-j|} ||A^{-1}||_inf
                          <= q^{|i-j|} / ((1 - q) min_i |b_i|).
  The error of a window, e = x_window - x, solves A_w e = s where s is zero
  except s_first = -a_cut x_{first-1} and s_last = -c_cut x_{last+1}.  On the
  kept rows, d_l and d_r rows away from the two ends of the extended range,
      |e_i| <= (|a_cut| q^{d_l} + |c_cut| q^{d_r}) / ((1 - q) min |b|) * ||x||_inf
  with q and min |b| taken over the window's extended rows of A_w (cut
  couplings zero).  `truncated` returns this bound per window.
"""
from __future__ import annotations

import numpy as np

from . import thomas


def windows(n: int, R: int, h: int):
    """(kept start, kept end, extended start, extended end) per window."""
    out = []
    for k0 in range(0, n, R):
        k1 = min(k0 + R, n)
        out.append((k0, k1, max(0, k0 - h), min(n, k1 + h)))
    return out


def truncated(a, b, c, d, R: int, h: int):
    """Windowed solve; returns (x, bounds) with bounds[w] the relative error
    bound of window w (0 where nothing was cut)."""
    a, b, c, d = (np.asarray(v, dtype=np.float64) for v in (a, b, c, d))
    n = b.size
    x = np.empty(n)
    bounds = []
    for k0, k1, e0, e1 in windows(n, R, h):
        aw, bw, cw, dw = a[e0:e1].copy(), b[e0:e1], c[e0:e1].copy(), d[e0:e1]
        a_cut = a[e0] if e0 > 0 else 0.0
        c_cut = c[e1 - 1] if e1 < n else 0.0
        aw[0] = 0.0
        cw[-1] = 0.0
        xw = thomas(aw, bw, cw, dw)
        x[k0:k1] = xw[k0 - e0:k1 - e0]
        q = float(np.max((np.abs(aw) + np.abs(cw)) / np.abs(bw)))
        bmin = float(np.min(np.abs(bw)))
        dl, dr = k0 - e0, (e1 - 1) - (k1 - 1)
        bounds.append((abs(a_cut) * q ** dl + abs(c_cut) * q ** dr) / ((1.0 - q) * bmin))
    return x, np.array(bounds)
