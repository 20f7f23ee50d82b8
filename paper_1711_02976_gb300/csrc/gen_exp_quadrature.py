#!/usr/bin/env python3
"""Derive the plane-wave (exponential) quadratures used by the M2X/X2X/X2L
operators and write them to ``exp_quadrature.h``.

The multipole-to-local step of the adaptive FMM (the "new version" FMM the
paper builds on, Sec. 1 and Sec. 3.2, M-to-I, I-to-I, I-to-L in Fig. "op") rests
on the integral representation, for z > 0,

    1/r = (1/2 pi) int_0^inf e^{-lambda z} int_0^{2 pi} e^{i lambda (x cos a + y sin a)} da dlambda.

The paper does not print the discretisation, so it is derived here.  In box
units (box side 1) every V-list pair has a point-to-point offset with
1 <= z <= 4 along the direction axis and |x|, |y| <= 4 across it, so
rho = sqrt(x^2 + y^2) <= 4 sqrt(2).

1. lambda: nodes lambda_k and weights w_k (k < s) such that
       sum_k w_k e^{-lambda_k z} J0(lambda_k rho) = 1/sqrt(z^2 + rho^2)
   to a chosen maximum relative error over that region.  The starting point
   for the smallest s comes from a pivoted QR of a fine Gauss-Legendre rule;
   each larger s starts from the previous solution plus one node beyond the
   largest.  Nodes and weights are then refined by nonlinear least squares on
   log(lambda), log(w) with reweighting towards the maximum error.
2. alpha: node k uses an M_k-point trapezoid rule in alpha; M_k is the
   smallest even count whose aliasing error at z = 1 stays within the node's
   share of the error budget.  M_k even lets the operators store only
   alpha_j, j < M_k/2 (the rest are complex conjugates).

Run:  python gen_exp_quadrature.py  (a few minutes; writes exp_quadrature.h)
"""
from __future__ import annotations

import math
import os
import sys

import numpy as np
import scipy.linalg as sl
import scipy.optimize as so
from scipy.special import j0, j1

RHO_MAX = 4.0 * math.sqrt(2.0)


def set_grid(nz, nrho):
    """Fit grid over the V-list region: nz values of z in [1, 4], nrho of rho."""
    global ZS, RS, Z, RH, F
    ZS = np.linspace(1.0, 4.0, nz)
    RS = np.linspace(0.0, RHO_MAX, nrho)
    Z, RH = [a.ravel() for a in np.meshgrid(ZS, RS, indexing="ij")]
    F = 1.0 / np.sqrt(Z ** 2 + RH ** 2)


set_grid(31, 41)


def _unpack(p, s):
    return np.exp(p[:s]), np.exp(p[s:])


def _resid(p, s, wgt):
    lam, w = _unpack(p, s)
    E = np.exp(-lam[None, :] * Z[:, None]) * j0(lam[None, :] * RH[:, None])
    return (E @ w / F - 1.0) * wgt


def _jac(p, s, wgt):
    lam, w = _unpack(p, s)
    E = np.exp(-lam[None, :] * Z[:, None])
    J0 = j0(lam[None, :] * RH[:, None])
    J1 = j1(lam[None, :] * RH[:, None])
    dl = w[None, :] * E * (-Z[:, None] * J0 - RH[:, None] * J1) / F[:, None] * lam[None, :]
    dw = E * J0 / F[:, None] * w[None, :]
    return np.hstack([dl, dw]) * wgt[:, None]


def _refine(p, s, rounds=25):
    wgt = np.ones_like(F)
    best = (np.inf, p)
    for _ in range(rounds):
        r = so.least_squares(_resid, p, jac=_jac, args=(s, wgt), method="trf", max_nfev=400,
                             xtol=1e-15, ftol=1e-15, gtol=1e-15)
        p = r.x
        e = np.abs(_resid(p, s, np.ones_like(F)))
        if e.max() < best[0]:
            best = (e.max(), p.copy())
        wgt = wgt * (e / e.max()) ** 0.3 + 1e-6
        wgt /= wgt.max()
    return best


def _qr_start(s):
    x, w = np.polynomial.legendre.leggauss(16)
    edges = np.linspace(0.0, 40.0, 41)
    lam = np.concatenate([(x + 1) / 2 * (b - a) + a for a, b in zip(edges[:-1], edges[1:])])
    om = np.concatenate([w / 2 * (b - a) for a, b in zip(edges[:-1], edges[1:])])
    A = om[None, :] * np.exp(-lam[None, :] * Z[:, None]) * j0(lam[None, :] * RH[:, None]) / F[:, None]
    _, _, piv = sl.qr(A, pivoting=True, mode="economic")
    cols = piv[:s]
    wts, *_ = np.linalg.lstsq(A[:, cols], np.ones_like(F), rcond=None)
    l0, w0 = lam[cols], np.abs(om[cols] * wts) + 1e-8
    o = np.argsort(l0)
    return np.concatenate([np.log(l0[o]), np.log(w0[o])])


def lambda_rules(s_lo, s_hi):
    """Yield (s, max_rel_err, lambda, w) for s = s_lo..s_hi by continuation."""
    err, p = _refine(_qr_start(s_lo), s_lo)
    lam, w = _unpack(p, s_lo)
    yield s_lo, err, lam, w
    for s in range(s_lo + 1, s_hi + 1):
        lam_new = np.append(lam, lam[-1] + (lam[-1] - lam[-2]))
        w_new = np.append(w, 0.5 * w[-1])
        err, p = _refine(np.concatenate([np.log(lam_new), np.log(w_new)]), s)
        lam, w = _unpack(p, s)
        o = np.argsort(lam)
        lam, w = lam[o], w[o]
        yield s, err, lam, w


def choose_m(lam, w, budget):
    """Smallest even M_k with w_k e^{-lambda_k} |trapezoid - J0| <= budget * 1/r."""
    ms = []
    rs = np.linspace(0.0, RHO_MAX, 200)
    phis = np.linspace(0.0, math.pi / 2, 9)
    for l, ww in zip(lam, w):
        m = 2
        while True:
            al = 2 * math.pi * np.arange(m) / m
            e = 0.0
            for ph in phis:
                tr = np.mean(np.cos(l * rs[:, None] * np.cos(al[None, :] - ph)), axis=1)
                e = max(e, float(np.max(ww * math.exp(-l) * np.abs(tr - j0(l * rs)) * np.sqrt(1 + rs ** 2))))
            if e <= budget:
                break
            m += 2
        ms.append(m)
    return ms


def total_error(lam, w, ms):
    """Max relative error of the full (lambda, alpha) rule over the V-list region."""
    rs = np.linspace(0.0, RHO_MAX, 81)
    worst = 0.0
    for ph in np.linspace(0.0, math.pi / 2, 7):
        acc = np.zeros((ZS.size, rs.size))
        for l, ww, m in zip(lam, w, ms):
            al = 2 * math.pi * np.arange(m) / m
            tr = np.mean(np.cos(l * rs[:, None] * np.cos(al[None, :] - ph)), axis=1)
            acc += ww * np.exp(-l * ZS)[:, None] * tr[None, :]
        ref = 1.0 / np.sqrt(ZS[:, None] ** 2 + rs[None, :] ** 2)
        worst = max(worst, float(np.max(np.abs(acc / ref - 1.0))))
    return worst


SETTINGS = [
    # name, digits, target max relative error of the lambda rule, s range[, fine phase]
    ("D3", 3, 3.0e-4, (8, 12)),
    ("D6", 6, 3.0e-7, (14, 22)),
    # intermediate rules the autotuner may pair with a 6-digit accuracy target
    ("D4", 4, 3.0e-5, (10, 16)),
    ("D5", 5, 3.0e-6, (12, 19)),
    # the 9-digit setting: its largest nodes oscillate across rho faster than the
    # default grid resolves, so the rule met on that grid is refined (and s raised
    # by continuation) on a finer grid until it meets the second target there
    ("D9", 9, 7.0e-10, (22, 31), (3.5e-10, 36, (41, 161))),
]


def main(out_path):
    blocks = []
    for name, digits, target, (s_lo, s_hi), *fine in SETTINGS:
        set_grid(31, 41)
        chosen = None
        for s, err, lam, w in lambda_rules(s_lo, s_hi):
            print(f"{name}: s={s} lambda-rule max rel err {err:.3e}", flush=True)
            if err <= target:
                chosen = (s, err, lam, w)
                break
        if chosen is None:
            raise SystemExit(f"{name}: no rule met {target}")
        s, err, lam, w = chosen
        if fine:
            ftarget, fs_hi, (nz, nrho) = fine[0]
            set_grid(nz, nrho)
            while True:
                err, pp = _refine(np.concatenate([np.log(lam), np.log(w)]), s)
                lam, w = _unpack(pp, s)
                o = np.argsort(lam)
                lam, w = lam[o], w[o]
                print(f"{name}: s={s} fine-grid lambda-rule max rel err {err:.3e}", flush=True)
                if err <= ftarget:
                    break
                if s >= fs_hi:
                    raise SystemExit(f"{name}: no rule met {ftarget} on the fine grid")
                lam, w, s = np.append(lam, lam[-1] + (lam[-1] - lam[-2])), np.append(w, 0.5 * w[-1]), s + 1
        ms = choose_m(lam, w, err / s)
        tot = total_error(lam, w, ms)
        print(f"{name}: s={s} M={ms} S={sum(ms)} total max rel err {tot:.3e}", flush=True)
        blocks.append((name, digits, s, err, tot, lam, w, ms))
    with open(out_path, "w") as fh:
        fh.write("// Generated by gen_exp_quadrature.py -- do not edit by hand.\n")
        fh.write("// Plane-wave quadratures for 1/r in box units: nodes lambda_k, weights w_k,\n")
        fh.write("// trapezoid counts M_k (even).  Region: 1 <= z <= 4, rho <= 4 sqrt(2).\n")
        fh.write("#pragma once\n\n")
        for name, digits, s, err, tot, lam, w, ms in blocks:
            fh.write(f"// {digits}-digit setting: lambda-rule max rel err {err:.3e}, "
                     f"with alpha rule {tot:.3e}; total terms {sum(ms)}\n")
            fh.write(f"#define RPY_EXPQ_{name}_S {s}\n")
            fh.write(f"static const double rpy_expq_{name.lower()}_lambda[{s}] = {{\n")
            fh.write(",\n".join(f"    {v:.17e}" for v in lam) + "};\n")
            fh.write(f"static const double rpy_expq_{name.lower()}_weight[{s}] = {{\n")
            fh.write(",\n".join(f"    {v:.17e}" for v in w) + "};\n")
            fh.write(f"static const int rpy_expq_{name.lower()}_m[{s}] = {{" + ", ".join(str(m) for m in ms) + "};\n\n")
    print("wrote", out_path)


if __name__ == "__main__":
    here = os.path.dirname(os.path.abspath(__file__))
    main(sys.argv[1] if len(sys.argv) > 1 else os.path.join(here, "exp_quadrature.h"))
