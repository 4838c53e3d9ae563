"""Exact brute-force ray caster for tiny cubes (rational arithmetic).

TEST INFRASTRUCTURE.  It pins the FP64 oracle (``vr_oracle.c``) by computing
the same rendering (paper §3.1, process item 3, with this project's readings)
through *different formulations* in exact rational arithmetic:

* ray/box: the visible segment is found by enumerating the crossings of the
  ray with the six face planes (plus the origin when it lies inside), not by
  the slab test;
* trilinear interpolation: the explicit weighted sum of the eight corners,
  sum_{abc} w_a(fx) w_b(fy) w_c(fz) V[i0+a, j0+b, k0+c], w_0 = 1-f, w_1 = f;
* lookup table: the piecewise-linear interpolant written in the hat-function
  basis, sum_i max(0, 1 - |x - i|) L'[i];
* compositing: the closed product form A_k = 1 - prod_{j<=k} (1 - alpha_j),
  C_k = sum_{j<=k} alpha_j rgb_j prod_{i<j} (1 - alpha_i), not the recurrence.

Square roots (ray normalisation) and fractional powers (opacity correction)
are exact when the argument is a perfect rational square / the exponent is an
integer, and otherwise evaluated with 60 significant digits.  Pure Python:
only for cubes of a few voxels per side and a handful of rays.
"""
from __future__ import annotations

import math
from decimal import Decimal, getcontext
from fractions import Fraction as Fr

getcontext().prec = 60


def _fr(x) -> Fr:
    return x if isinstance(x, Fr) else Fr(x)


def _sqrt(x: Fr) -> Fr:
    if x < 0:
        raise ValueError
    n, d = x.numerator, x.denominator
    rn, rd = math.isqrt(n), math.isqrt(d)
    if rn * rn == n and rd * rd == d:
        return Fr(rn, rd)
    return Fr((Decimal(n) / Decimal(d)).sqrt())


def _pow(base: Fr, e: Fr) -> Fr:
    if e.denominator == 1:
        return base ** e.numerator
    if base == 0:
        return Fr(0)
    if e.denominator == 2:
        return _sqrt(base) ** e.numerator
    b = Decimal(base.numerator) / Decimal(base.denominator)
    ed = Decimal(e.numerator) / Decimal(e.denominator)
    return Fr((b.ln() * ed).exp())


def ray(cam, w, h, px, py):
    """cam = (proj, eye, fwd, du, dv) with exactly representable numbers."""
    proj, eye, fwd, du, dv = cam
    u = Fr(2 * px + 1, 2) - Fr(w, 2)
    v = Fr(2 * py + 1, 2) - Fr(h, 2)
    eye, fwd, du, dv = ([_fr(c) for c in vec] for vec in (eye, fwd, du, dv))
    if proj == 0:
        o = [eye[a] + u * du[a] + v * dv[a] for a in range(3)]
        d = list(fwd)
    else:
        o = list(eye)
        d = [fwd[a] + u * du[a] + v * dv[a] for a in range(3)]
    nrm = _sqrt(sum(c * c for c in d))
    return o, [c / nrm for c in d]


def segment(o, d, dims):
    """[t_in, t_out] of the ray (t >= 0) inside the box [0, n-1]^3, or None."""
    hi = [Fr(n - 1) for n in dims]

    def inside(p):
        return all(0 <= p[a] <= hi[a] for a in range(3))

    ts = []
    if inside(o):
        ts.append(Fr(0))
    for a in range(3):
        if d[a] == 0:
            continue
        for face in (Fr(0), hi[a]):
            t = (face - o[a]) / d[a]
            if t < 0:
                continue
            p = [o[b] + t * d[b] for b in range(3)]
            p[a] = face
            if inside(p):
                ts.append(t)
    if not ts:
        return None
    return min(ts), max(ts)


def trilinear(V, dims, p):
    """V indexed V[z][y][x] (exact numbers); p inside the box."""
    i0, f = [], []
    for a in range(3):
        c = min(math.floor(p[a]), dims[a] - 2)
        i0.append(c)
        f.append(p[a] - c)
    s = Fr(0)
    for c in (0, 1):
        for b in (0, 1):
            for a in (0, 1):
                wgt = ((f[0] if a else 1 - f[0]) * (f[1] if b else 1 - f[1])
                       * (f[2] if c else 1 - f[2]))
                s += wgt * _fr(V[i0[2] + c][i0[1] + b][i0[0] + a])
    return s


def corrected_table(lut, step):
    out = []
    for r, g, b, a in lut:
        out.append((_fr(r), _fr(g), _fr(b), 1 - _pow(1 - _fr(a), _fr(step))))
    return out


def classify(lutc, v_lo, v_hi, s):
    n = len(lutc)
    x = (s - _fr(v_lo)) / (_fr(v_hi) - _fr(v_lo))
    x = min(max(x, Fr(0)), Fr(1)) * (n - 1)
    rgba = [Fr(0)] * 4
    for i in range(n):
        hat = 1 - abs(x - i)
        if hat > 0:
            for c in range(4):
                rgba[c] += hat * lutc[i][c]
    return rgba


def render_pixel(V, dims, cam, w, h, px, py, mode, step, lut=None, v_lo=0,
                 v_hi=1, clip=0, term_alpha=1):
    """Exact result: MIP/SUM -> one number (None for a MIP miss); COMPOSITE ->
    [C_r, C_g, C_b, A].  Also returns the number of evaluated samples."""
    step = _fr(step)
    o, d = ray(cam, w, h, px, py)
    seg = segment(o, d, dims)
    K = 0 if seg is None else math.floor((seg[1] - seg[0]) / step) + 1
    samples = []
    for k in range(K):
        t = seg[0] + k * step
        samples.append(trilinear(V, dims, [o[a] + t * d[a] for a in range(3)]))
    if mode == 0:
        return (max(samples) if samples else None), K
    if mode == 2:
        return sum((s * step for s in samples), Fr(0)), K
    lutc = corrected_table(lut, step)
    alphas, colours = [], []
    count = K
    for k, s in enumerate(samples):
        if s < _fr(clip):
            continue
        rgba = classify(lutc, v_lo, v_hi, s)
        alphas.append(rgba[3])
        colours.append(rgba[:3])
        transmit = Fr(1)
        for a in alphas:
            transmit *= 1 - a
        if 1 - transmit >= _fr(term_alpha):
            count = k + 1
            break
    C = [Fr(0)] * 3
    trans = Fr(1)
    for a, rgb in zip(alphas, colours):
        for c in range(3):
            C[c] += a * rgb[c] * trans
        trans *= 1 - a
    return C + [1 - trans], count
