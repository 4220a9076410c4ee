"""FP64 oracle for the bispectrum multipoles (Sec. II.C and III.B of the paper).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Steps and the passages they follow
----------------------------------
shells          thin shells of width dk about centres k_i (eq. shell), in integer
                k_f units: shell s holds modes with lo_s <= |n| < lo_s + width,
                lo_s = first + s*step - width/2.
shell_field     F_k^(l)(x) = sum_{n in shell} F_l(n) e^{+ik.x} (eq. F_k), an
                unnormalised inverse DFT of the shell-filtered field.
triangle_sum    sum_x F_{k1}^(l) F_{k2}^(0) F_{k3}^(0) = N^3 sum over closed
                triangles (eq. Factorize, discrete orthogonality); with F^(2) on
                the two larger sides for the split hexadecapole (eq. Bhexa2).
counts          N_T (eq. NT) as an exact integer: per-mode rounded FP64
                convolution C_bc(n) of the shell indicators, summed over shell a.
bispectrum      B^(l) = (2l+1) <F_l F_0 F_0>_T / I_33 - N^(l) (eqs. BispMono,
                BispQuad) with the thin-shell shot noise of eq. SNbisp2thin:
                (2l+1)/I_33 [<F_l F^w_0*>_{k1} + sum_{i=2,3} L_l(q^_1.q^_i)
                <F_0 F^w_l*>_{ki}] - 2 S_3/I_33 delta_l0.  Cosines come from the
                shell centres by the law of cosines (closure q_1+q_2+q_3 = 0).
                Triangles are ordered by the largest side, k1 >= k2 >= k3
                (Sec. II.C), i.e. shell indices a >= b >= c.

Parity: shell fields, triangle sums and counts are pinned by brute-force
enumeration; the thin-shell shot noise of l = 0 by the single-object identity
(one galaxy on a node and randoms on every node leave B_0 = -2 alpha^2/nbar^2
for every triangle, every term of eq. SNbisp2thin being of order one there);
and for l = 0, 2, 4 against F_l and F^w_l summed directly over objects on
nodes (the definitions below eq. SNbisp2, with no grid, moment field or FFT),
assembled per eq. SNbisp2thin.
"""
from __future__ import annotations

import math

import numpy as np

from . import power as _pw
from .power import irfftn, rfftn


def legendre_poly(l, mu):
    mu = np.asarray(mu, dtype=np.float64)
    if l == 0:
        return np.ones_like(mu)
    if l == 2:
        return 0.5 * (3.0 * mu * mu - 1.0)
    if l == 4:
        return (35.0 * mu ** 4 - 30.0 * mu * mu + 3.0) / 8.0
    raise ValueError(l)


def shell_bounds(bshells):
    """(lo_s, hi_s, centre_s) in k_f units for (first, step, width, S)."""
    first, step, width, S = bshells
    c = np.array([first + s * step for s in range(S)], dtype=np.float64)
    lo = c - 0.5 * width
    return lo, lo + width, c


def shell_index(N, bshells):
    """Shell of every half-spectrum mode (-1 outside all shells, at n = 0 and
    on Nyquist planes) and the mode's full-grid weight."""
    lo, hi, _ = shell_bounds(bshells)
    nx, ny, nz = _pw.mode_vectors(N)
    n2 = np.broadcast_to(nx * nx + ny * ny + nz * nz, (N, N, N // 2 + 1))
    idx = np.full(n2.shape, -1, dtype=np.int64)
    for s in range(len(lo)):
        m = (n2 >= lo[s] ** 2) & (n2 < hi[s] ** 2)
        idx[m] = s
    nyq = (np.abs(nx) == N // 2) | (np.abs(ny) == N // 2) | (np.abs(nz) == N // 2)
    idx[np.broadcast_to(nyq, idx.shape)] = -1
    idx[n2 == 0] = -1
    wt = np.broadcast_to(np.where(nx == 0, 1.0, 2.0), idx.shape)
    return idx, wt


def shell_field(Fl, sidx, s, N):
    """F_k^(l)(x) for shell s: unnormalised inverse DFT of F_l on the shell."""
    return irfftn(np.where(sidx == s, Fl, 0.0), (N, N, N)) * float(N) ** 3


def triangle_list(S):
    """All shell triples a >= b >= c (k1 >= k2 >= k3)."""
    return [(a, b, c) for a in range(S) for b in range(a + 1) for c in range(b + 1)]


class Counter:
    """Exact N_T by rounded FP64 convolution of shell indicators."""

    def __init__(self, N, bshells):
        self.N = N
        self.sidx, self.wt = shell_index(N, bshells)
        self._j = {}
        self._C = {}

    def _jfield(self, s):
        if s not in self._j:
            self._j[s] = irfftn((self.sidx == s).astype(np.float64), (self.N,) * 3) * float(self.N) ** 3
        return self._j[s]

    def _conv(self, b, c):
        key = (b, c)
        if key not in self._C:
            C = rfftn(self._jfield(b) * self._jfield(c)) / float(self.N) ** 3
            self._C[key] = np.rint(C.real)
        return self._C[key]

    def count(self, a, b, c):
        C = self._conv(b, c)
        m = self.sidx == a
        return int(np.rint(np.sum(self.wt[m] * C[m])))

    def counts_for_pair(self, b, c, keep=True):
        """N_T(a, b, c) for every shell a at once: the same per-mode rounded
        convolution C_bc, summed over each shell with the full-grid weights.
        keep=False drops C_bc afterwards (large grids)."""
        C = self._conv(b, c)
        sel = self.sidx >= 0
        S = int(self.sidx.max()) + 1
        out = np.rint(np.bincount(self.sidx[sel], weights=self.wt[sel] * C[sel], minlength=S)).astype(np.int64)
        if not keep:
            del self._C[(b, c)]
        return out


def bispectrum(gal, ran, geom, bshells, ells=(0, 2, 4), tris=None, zero_area=False):
    """B^(l) for the given triangles (default: all a >= b >= c with N_T > 0)."""
    g = _pw._geom(geom)
    N = int(g["N"])
    Fl, Fwl, sc = _pw.survey_fields(gal, ran, g, lmax=max(ells), with_w2=True)
    return bispectrum_from_fields(Fl, Fwl, sc, N, bshells, ells, tris, zero_area=zero_area)


def shell_means(Fl, Fwl, sidx, wt, S, ells):
    """Shell means of Re F_l F^w_0* and Re F_0 F^w_l* and mode counts."""
    sel = sidx >= 0
    si = sidx[sel]
    w = wt[sel]
    nm = np.bincount(si, weights=w, minlength=S)
    sn1, sn2 = {}, {}
    for l in ells:
        sn1[l] = np.bincount(si, weights=w * (Fl[l] * np.conj(Fwl[0])).real[sel], minlength=S) / nm
        sn2[l] = np.bincount(si, weights=w * (Fl[0] * np.conj(Fwl[l])).real[sel], minlength=S) / nm
    return nm, sn1, sn2


def bispectrum_from_fields(Fl, Fwl, sc, N, bshells, ells=(0, 2, 4), tris=None, counts=None, cache_fields=None,
                           zero_area=False):
    """B^(l), N^(l), T^(l) and N_T for the given triangles from the Legendre
    fields.  counts: optional mapping (a, b, c) -> N_T written earlier by this
    module's Counter (skips the convolution counter).  cache_fields: at most
    that many shell fields are kept (least recently used dropped), for large
    grids; None keeps them all.  Neither changes the arithmetic.
    zero_area=True (needs l = 0 and 2) adds the split hexadecapole of eq.
    Bhexa2: T22 = sum_x F_a^(2) F_b^(2) F_c^(0) (delta_2 on the two larger
    sides) and B4b = [35/2 T22 - 5 T2 - 7/2 T0] / (N^3 N_T I_33), the
    combination of eq. Bhexa2 formed from the raw sums (no shot-noise
    subtraction: as for P_4b, the self terms of the split product cancel
    against the 7/2 monopole term on zero-area triangles)."""
    from collections import OrderedDict
    S = bshells[3]
    sidx, wt = shell_index(N, bshells)
    _, _, cen = shell_bounds(bshells)
    nm, sn1, sn2 = shell_means(Fl, Fwl, sidx, wt, S, ells)
    counter = None if counts is not None else Counter(N, bshells)
    cache = OrderedDict()

    def field(l, s):
        if (l, s) in cache:
            cache.move_to_end((l, s))
        else:
            if cache_fields is not None:
                while len(cache) >= max(1, cache_fields):
                    cache.popitem(last=False)
            cache[(l, s)] = shell_field(Fl[l], sidx, s, N)
        return cache[(l, s)]

    all_tris = triangle_list(S) if tris is None else list(tris)
    out = dict(tri=[], NT=[], centre_closed=[], nmodes_shell=nm, I33=sc["I33"], S3=sc["S3"])
    for l in ells:
        out[f"T{l}"] = []
        out[f"B{l}"] = []
        out[f"N{l}"] = []
    if zero_area:
        out["T22"], out["B4b"] = [], []
    N3 = float(N) ** 3
    for (a, b, c) in all_tris:
        nt = counts[(a, b, c)] if counter is None else counter.count(a, b, c)
        if tris is None and nt == 0:
            continue
        out["tri"].append((a, b, c))
        out["NT"].append(nt)
        out["centre_closed"].append(bool(cen[b] + cen[c] >= cen[a]))
        mu12 = np.clip((cen[c] ** 2 - cen[a] ** 2 - cen[b] ** 2) / (2 * cen[a] * cen[b]), -1.0, 1.0)
        mu13 = np.clip((cen[b] ** 2 - cen[a] ** 2 - cen[c] ** 2) / (2 * cen[a] * cen[c]), -1.0, 1.0)
        I0b, I0c = field(0, b), field(0, c)
        for l in ells:
            T = float(np.sum(field(l, a) * I0b * I0c))
            pref = 2 * l + 1
            noise = pref / sc["I33"] * (sn1[l][a] + float(legendre_poly(l, mu12)) * sn2[l][b]
                                         + float(legendre_poly(l, mu13)) * sn2[l][c])
            if l == 0:
                noise -= 2.0 * sc["S3"] / sc["I33"]
            out[f"T{l}"].append(T)
            out[f"N{l}"].append(noise)
            out[f"B{l}"].append(pref * T / (N3 * nt * sc["I33"]) - noise if nt > 0 else float("nan"))
        if zero_area:
            T22 = float(np.sum(field(2, a) * field(2, b) * I0c))
            out["T22"].append(T22)
            T0, T2 = out["T0"][-1], out["T2"][-1]
            out["B4b"].append((17.5 * T22 - 5.0 * T2 - 3.5 * T0) / (N3 * nt * sc["I33"]) if nt > 0
                              else float("nan"))
    for k in list(out):
        if isinstance(out[k], list):
            out[k] = np.asarray(out[k])
    return out
