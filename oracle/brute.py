"""Brute-force restatement of the model-based render (O2), pure Python.

TEST INFRASTRUCTURE ONLY.  For tiny inputs (volumes of a few thousand
voxels, a handful of scanlines): every quantity is evaluated by its direct
definition, with no running sums and no separable filtering:

* remaining energy E(u) = E0 exp(-f int_0^y alpha dv) (App. B.2) as a fresh
  sum over all samples above u, for every u;
* the image I = P (x) R_imp + E (P (x) T) (App. B.2: the reflection
  impulses blurred; the backscatter B = E . P (x) T, the scatter pattern
  blurred and then scaled by the energy at the pixel itself), each
  convolution as the full 2-D sum over the PSF support;
* its own Philox-4x32-10 (Salmon et al., SC 2011) on Python integers and its
  own Box-Muller transform.

It follows the same readings as the C oracle (see ``ussim_oracle.c``) and
exists to catch structural mistakes there (scan offsets, filter order,
padding, counter layout).  Output: dict of numpy arrays.
"""
from __future__ import annotations

import math

import numpy as np

F32 = np.float32
MASK = 0xFFFFFFFF


def philox(ctr, key, rounds=10):
    """Philox-4x32: multiply words 0 and 2 by the two round multipliers,
    mix the high halves with words 1, 3 and the key, bump the key by the
    Weyl increments between rounds."""
    c = [int(x) & MASK for x in ctr]
    k = [int(x) & MASK for x in key]
    mult = (0xD2511F53, 0xCD9E8D57)
    weyl = (0x9E3779B9, 0xBB67AE85)
    for r in range(rounds):
        if r:
            k = [(k[0] + weyl[0]) & MASK, (k[1] + weyl[1]) & MASK]
        prod_a = mult[0] * c[0]
        prod_b = mult[1] * c[2]
        c = [((prod_b >> 32) ^ c[1] ^ k[0]) & MASK, prod_b & MASK,
             ((prod_a >> 32) ^ c[3] ^ k[1]) & MASK, prod_a & MASK]
    return c


def _uniform(w):
    return ((w >> 9) * 2 + 1) / 2.0 ** 24


def _phi(x):
    return 0.5 * math.erfc(-x / math.sqrt(2.0))


def _taps(sigma, spacing):
    if sigma <= 0:
        return [1.0]
    K = math.ceil(3.0 * sigma / spacing)
    raw = [math.exp(-0.5 * (k * spacing / sigma) ** 2) for k in range(-K, K + 1)]
    tot = math.fsum(raw)
    return [r / tot for r in raw]


def render(labels, hu, voxel_mm, table, probe, options, pose, env=0, seed=0, step=0):
    nz, ny, nx = labels.shape
    NL, NS = probe.n_lines, probe.n_samples
    M = np.asarray(pose, F32).reshape(3, 4)
    inv_h = F32(1.0 / float(F32(voxel_mm)))
    dr64 = float(F32(probe.depth_mm)) / NS
    dr = F32(dr64)
    r0 = F32(probe.radius_mm)
    curv = probe.kind == 1
    dth = float(F32(probe.fan_deg)) * math.pi / 180.0 / (NL - 1) if (curv and NL > 1) else 0.0

    def coords(l, s):
        sf = F32(s)
        if curv:
            th = (l - 0.5 * (NL - 1)) * dth
            rho = F32(r0 + F32(sf * dr))
            x = F32(rho * F32(math.sin(th)))
            z = F32(F32(rho * F32(math.cos(th))) - r0)
        else:
            x = F32((l - 0.5 * (NL - 1)) * float(F32(probe.pitch_mm)))
            z = F32(sf * dr)
        u = []
        for c in range(3):
            pc = F32(F32(F32(M[c, 0] * x) + F32(M[c, 2] * z)) + M[c, 3])
            u.append(F32(pc * inv_h))
        return u

    def vox_hu(i, j, k):
        if 0 <= i < nx and 0 <= j < ny and 0 <= k < nz:
            return float(hu[k, j, i])
        return 0.0

    lab = np.zeros((NL, NS), np.int64)
    nn = np.full((NL, NS), -1, np.int64)
    huv = np.zeros((NL, NS))
    for l in range(NL):
        for s in range(NS):
            u = coords(l, s)
            ii = [math.floor(float(F32(uc + F32(0.5)))) for uc in u]
            if all(0 <= ii[c] < n for c, n in enumerate((nx, ny, nz))):
                nn[l, s] = (ii[2] * ny + ii[1]) * nx + ii[0]
                lab[l, s] = labels[ii[2], ii[1], ii[0]]
            f = [math.floor(float(uc)) for uc in u]
            t = [float(F32(u[c] - F32(f[c]))) for c in range(3)]
            # interpolate along x, then y, then z
            plane = []
            for dz in (0, 1):
                row = []
                for dy in (0, 1):
                    a = vox_hu(f[0], f[1] + dy, f[2] + dz)
                    b = vox_hu(f[0] + 1, f[1] + dy, f[2] + dz)
                    row.append(a + t[0] * (b - a))
                plane.append(row[0] + t[1] * (row[1] - row[0]))
            huv[l, s] = plane[0] + t[2] * (plane[1] - plane[0])

    alpha = [float(F32(t.alpha_db_cm_mhz)) * math.log(10.0) / 200.0 for t in table]   # Np / (mm MHz)

    def Z(l, s):
        if options.z_mode == 0:
            return max(huv[l, s] + 1024.0, 1.0)
        return float(F32(table[lab[l, s]].z_mrayl))

    def refl(l, s):
        if s >= NS - 1:
            return 0.0
        return (Z(l, s + 1) - Z(l, s)) / (Z(l, s + 1) + Z(l, s))

    def G(l, s):
        return 1 if (s < NS - 1 and lab[l, s + 1] != lab[l, s]) else 0

    h = float(F32(voxel_mm))

    def cos_theta(l, s):
        if not G(l, s):
            return 1.0
        below = lab[l, s + 1]
        dlat = (float(F32(probe.radius_mm)) + s * dr64) * dth if curv else float(F32(probe.pitch_mm))
        W = math.ceil(2.0 * h / dr64)
        D = min(max(math.ceil(h / dlat), 1), 8)
        lp, lm = min(l + D, NL - 1), max(l - D, 0)
        window = [min(max(q, 0), NS - 1) for q in range(s - W + 1, s + W + 1)]
        dM = sum(int(lab[lp, q] == below) for q in window) - sum(int(lab[lm, q] == below) for q in window)
        tan_t = abs(dM) * dr64 / ((lp - lm) * dlat) if lp > lm else 0.0
        return 1.0 / math.sqrt(1.0 + tan_t * tan_t)

    f_mhz = float(F32(probe.f_mhz))
    e0 = float(F32(probe.e0))

    def increment(l, v):
        inc = -f_mhz * alpha[lab[l, v]] * dr64
        if options.transmission and G(l, v):
            r = refl(l, v)
            inc += math.log(max(1.0 - r * r, 1e-30))
        return inc

    key0 = (seed & MASK) ^ ((step * 0x9E3779B9) & MASK)
    key1 = (seed >> 32) & MASK

    S = np.zeros((NL, NS))
    R = np.zeros((NL, NS))
    Tm = np.zeros((NL, NS))
    E = np.zeros((NL, NS))
    CT = np.zeros((NL, NS))
    for l in range(NL):
        for s in range(NS):
            Es = e0 * math.exp(math.fsum(increment(l, v) for v in range(s)))
            E[l, s] = Es
            ct = cos_theta(l, s)
            CT[l, s] = ct
            rimp = 0.0
            if G(l, s):
                a = abs(ct * refl(l, s))
                rimp = Es * (a * a if options.refl_power == 2 else a)
            tis = table[lab[l, s]]
            if options.speckle:
                w = philox([s >> 1, l, env, 0], [key0, key1])
                u0, u1 = _uniform(w[0]), _uniform(w[1])
                rad = math.sqrt(-2.0 * math.log(u0))
                n0 = rad * (math.sin(2 * math.pi * u1) if s % 2 else math.cos(2 * math.pi * u1))
                mu1 = float(F32(tis.mu1))
                t1 = 0 if mu1 == -math.inf else (2 ** 32 if mu1 == math.inf
                                                  else math.floor(_phi(mu1) * 2.0 ** 32))
                T = n0 * float(F32(tis.sigma0)) + float(F32(tis.mu0)) if w[2 + (s & 1)] < t1 else 0.0
            else:
                T = float(F32(tis.mu0))
            R[l, s] = rimp
            Tm[l, s] = T
            S[l, s] = rimp + Es * T

    wax = _taps(float(F32(probe.psf_sigma_ax_mm)), dr64)
    dlat_mid = ((float(F32(probe.radius_mm)) + 0.5 * float(F32(probe.depth_mm))) * dth
                if curv else float(F32(probe.pitch_mm)))
    wlat = _taps(float(F32(probe.psf_sigma_lat_mm)), dlat_mid)
    Ka, Kl = len(wax) // 2, len(wlat) // 2
    def blur(X, l, s):
        acc = []
        for j in range(-Kl, Kl + 1):
            for k in range(-Ka, Ka + 1):
                if 0 <= l + j < NL and 0 <= s + k < NS:
                    acc.append(wlat[j + Kl] * wax[k + Ka] * X[l + j, s + k])
        return math.fsum(acc)

    I = np.zeros((NL, NS))
    for l in range(NL):
        for s in range(NS):
            I[l, s] = blur(R, l, s) + E[l, s] * blur(Tm, l, s)

    dyn = float(F32(probe.dyn_range_db))
    Y = np.zeros((NL, NS))
    for l in range(NL):
        for s in range(NS):
            db = 20.0 * math.log10(max(I[l, s], 1e-30) / e0)
            Y[l, s] = min(1.0, max(0.0, (db + dyn) / dyn))

    frame = np.zeros((probe.out_h, probe.out_w))
    if not curv:
        frame[:, :] = Y.T
    else:
        half = 0.5 * math.radians(float(F32(probe.fan_deg)))
        R0, D = float(F32(probe.radius_mm)), float(F32(probe.depth_mm))
        xmax = (R0 + D) * math.sin(half)
        zmin, zmax = R0 * math.cos(half), R0 + D
        H, W = probe.out_h, probe.out_w
        for r in range(H):
            for c in range(W):
                x = -xmax + (c + 0.5) * 2 * xmax / W
                z = zmin + (r + 0.5) * (zmax - zmin) / H
                fl = math.atan2(x, z) / dth + 0.5 * (NL - 1)
                fs = (math.hypot(x, z) - R0) / dr64
                if not (0 <= fl <= NL - 1 and 0 <= fs <= NS - 1):
                    continue
                l0 = min(int(math.floor(fl)), NL - 2)
                s0 = min(int(math.floor(fs)), NS - 2)
                a, b = fl - l0, fs - s0
                top = Y[l0, s0] + a * (Y[l0 + 1, s0] - Y[l0, s0])
                bot = Y[l0, s0 + 1] + a * (Y[l0 + 1, s0 + 1] - Y[l0, s0 + 1])
                frame[r, c] = top + b * (bot - top)

    return {"frame": frame, "envelope": I, "logimg": Y, "S": S, "T": Tm, "E": E, "cos_theta": CT,
            "hu": huv, "nn_index": nn, "label": lab}
