"""Distribution checks of generated variates, computed on the device with torch.

These are measurements of the library's outputs, not part of generation:
  - ks_grid: the Kolmogorov-Smirnov distance between the empirical distribution
    function of x and Phi, evaluated at the K - 1 points q_k = Phi^-1(k / K);
    the supremum between grid points can exceed it by at most 1 / K.
  - ks_bf16_exact: for bfloat16 outputs, the exact KS distance between the
    empirical distribution and that of RN_bf16(Z), Z ~ N(0, 1) (both are step
    functions on the bfloat16 values), plus the distance to Phi itself, which
    rounding alone keeps near density x half a bfloat16 spacing.
  - tail_mass: the fraction of |x| > t against P(|RN_dtype(Z)| > t).
  - serial_chi2: independence of outputs `lag` apart within each stream: a chi-square
    test on the pairs' cells in a k x k grid of equal-probability bins of Phi.
  - error_vs_f64: each narrow output against the binary64 output of the same
    streams: how many representable steps it lies from the nearest value
    RN_dtype(z64), and its distance from z64 in the narrow type's ulps.
"""

from __future__ import annotations

import math

import numpy as np

CHUNK = 1 << 26
MANT_BITS = {"f64": 53, "f32": 24, "bf16": 8}


def _ndtr(x):
    from scipy.special import ndtr
    return ndtr(x)


def ks_grid(torch, x, K: int = 1 << 20, chunk: int = CHUNK) -> dict:
    from scipy.special import kolmogorov, ndtri
    q = ndtri(np.arange(1, K, dtype=np.float64) / K)
    phi_q = _ndtr(q)
    edges = torch.from_numpy(q).to(x.device)
    hist = torch.zeros(K, dtype=torch.int64, device=x.device)
    n = x.numel()
    for a in range(0, n, chunk):
        c = x[a:a + chunk].double()
        # bucket k holds q_{k} < x <= q_{k+1}: cumsum(hist)[k] = #{x <= q_{k+1}}
        hist += torch.bincount(torch.bucketize(c, edges, right=False), minlength=K)
    F = hist.cumsum(0)[:-1].cpu().numpy().astype(np.float64) / n
    d = float(np.max(np.abs(F - phi_q)))
    return {"n": n, "grid_points": K - 1, "D": d, "sqrt_n_D": d * math.sqrt(n),
            "p_value": float(kolmogorov(d * math.sqrt(n)))}


def ks_bf16_exact(torch, x, chunk: int = CHUNK) -> dict:
    from scipy.special import kolmogorov
    hist = torch.zeros(65536, dtype=torch.int64, device=x.device)
    n = x.numel()
    xi = x.view(torch.int16)
    for a in range(0, n, chunk):
        hist += torch.bincount(xi[a:a + chunk].int() & 0xFFFF, minlength=65536)
    counts = hist.cpu().numpy().astype(np.float64)
    with np.errstate(invalid="ignore"):   # the NaN patterns
        vals = (np.arange(65536, dtype=np.uint32) << 16).view(np.float32).astype(np.float64)
    fin = np.isfinite(vals)
    uniq, inv = np.unique(vals[fin], return_inverse=True)    # merges -0 and +0
    cc = np.bincount(inv, weights=counts[fin], minlength=len(uniq))
    assert cc.sum() == n, "non-finite outputs"
    F = np.cumsum(cc) / n
    # P(RN(Z) <= v_k) = Phi(midpoint between v_k and v_{k+1}) (ties have measure zero)
    G = np.append(_ndtr((uniq[:-1] + uniq[1:]) / 2), 1.0)
    d_round = float(np.max(np.abs(F - G)))
    # against Phi itself: the empirical CDF jumps at each value; check both sides of each jump
    phi_v = _ndtr(uniq)
    F_left = np.concatenate([[0.0], F[:-1]])
    d_phi = float(max(np.max(np.abs(F - phi_v)), np.max(np.abs(F_left - phi_v))))
    return {"n": n, "D_vs_rounded_normal": d_round, "sqrt_n_D": d_round * math.sqrt(n),
            "p_value": float(kolmogorov(d_round * math.sqrt(n))), "D_vs_phi": d_phi}


def _next_up(t: float, dtype: str) -> float:
    if dtype == "f64":
        return float(np.nextafter(np.float64(t), np.inf))
    if dtype == "f32":
        return float(np.nextafter(np.float32(t), np.float32(np.inf)))
    b = (np.array([t], dtype=np.float32).view(np.uint32)[0] >> 16) + 1   # bfloat16 bits, t > 0
    return float(np.array([b << 16], dtype=np.uint32).view(np.float32)[0])


def tail_mass(torch, x, dtype: str, t: float = 3.0, chunk: int = CHUNK) -> dict:
    n = x.numel()
    cnt = 0
    for a in range(0, n, chunk):
        cnt += int((x[a:a + chunk].abs() > t).sum().item())
    # RN(z) > t exactly when z is beyond the midpoint to the next value up
    # (t = 3 has an even last significand bit in every type, so a tie rounds to t)
    mid = (t + _next_up(t, dtype)) / 2
    expect = float(2 * _ndtr(-mid))
    obs = cnt / n
    sd = math.sqrt(expect * (1 - expect) / n)
    return {"threshold": t, "observed": obs, "expected": expect, "rel_error": obs / expect - 1,
            "z_score": (obs - expect) / sd}


def round_to_precision(torch, z64, p: int):
    """RN-even of binary64 values to p significand bits, by integer arithmetic on
    the bits (one rounding; normal results assumed), returned as binary64."""
    k = 53 - p
    b = z64.contiguous().view(torch.int64)
    r = ((b + ((1 << (k - 1)) - 1) + ((b >> k) & 1)) >> k) << k
    return r.view(torch.float64)


def error_vs_f64(torch, x, z64, dtype: str, chunk: int = CHUNK) -> dict:
    """x (f32 or bf16) against z64, the binary64 outputs of the same streams:
    steps (adjacent values) from RN_dtype(z64), and distance from z64 in ulps."""
    p = MANT_BITS[dtype]
    ity = torch.int32 if dtype == "f32" else torch.int16
    n = x.numel()
    worst, not_nearest, total_abs, max_rel, max_steps = 0.0, 0, 0.0, 0.0, 0
    for a in range(0, n, chunk):
        r = z64[a:a + chunk]
        xc = x[a:a + chunk]
        rn = round_to_precision(torch, r, p).to(x.dtype)      # exact: representable
        steps = (xc.view(ity).int() - rn.view(ity).int()).abs()
        max_steps = max(max_steps, int(steps.max().item()))
        not_nearest += int((steps != 0).sum().item())
        d = (xc.double() - r).abs()
        nz = r != 0
        _, e = torch.frexp(r)                        # |r| in [2^(e-1), 2^e)
        ulp = torch.exp2((e - p).to(torch.float64))
        u = torch.where(nz, d / ulp, torch.zeros_like(d))
        worst = max(worst, float(u.max().item()))
        total_abs += float(d.sum().item())
        rel = torch.where(nz, d / r.abs(), torch.zeros_like(d))
        max_rel = max(max_rel, float(rel.max().item()))
    return {"max_steps_from_nearest": max_steps, "max_err_ulp": worst,
            "outputs_not_nearest": not_nearest, "frac_not_nearest": not_nearest / max(n, 1),
            "mean_abs_err": total_abs / n, "max_rel_err": max_rel}


def serial_chi2(torch, x, stream_len: int, lag: int = 1, k: int = 16) -> dict:
    """x: packed stream-major outputs, streams of stream_len; pairs (x_t, x_{t+lag})
    are taken within streams only."""
    from scipy.special import ndtri
    from scipy.stats import chi2 as chi2_dist
    edges = torch.from_numpy(ndtri(np.arange(1, k, dtype=np.float64) / k)).to(x.device)
    q = torch.bucketize(x.double().view(-1, stream_len), edges)          # (streams, len)
    cells = (q[:, :-lag] * k + q[:, lag:]).reshape(-1)
    counts = torch.bincount(cells, minlength=k * k).double()
    n = counts.sum()
    expect = n / (k * k)
    stat = float(((counts - expect) ** 2 / expect).sum().item())
    dof = k * k - 1
    return {"lag": lag, "cells": k * k, "pairs": int(n.item()), "chi2": stat, "dof": dof,
            "p_value": float(chi2_dist.sf(stat, dof))}
