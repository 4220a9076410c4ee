"""FP64 oracle for the power-spectrum multipoles (Sec. III.A of the paper).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Plain numpy/scipy in
float64, one field at a time, no grouping or fusion: every step is the
definition it cites.

Steps and the passages they follow
----------------------------------
scalars        alpha (Sec. III.A, above eq. F0; weighted reading), I_22 (eq. I22def),
               N_0 (eq. N0true) and its FKP expectation alpha(1+alpha) sum_r w^2,
               I_33 = alpha sum_r nbar^2 w^3 (the normalisation eq. BispMono divides by,
               left undefined by the paper; FKP-type reading), S_3 (last term of
               eq. Noise0), L^ab at k = 0 (eq. Lab).
assign         interpolation of objects to grid nodes (eq. mapFFT): CIC, TSC or
               PCS; interlaced pairs of grids (Sec. III.A after eq. mapFFT).
moments        F x^_a x^_b and F x^_a x^_b x^_c x^_d about the observer
               (eqs. Qij, Qijkl, Qab) with x^ taken at the grid node, or
               (xhat="object") sum w x^_a x^_b (...) W with x^ of each object.
legendre       F_0 (eq. F0), F_2 (eqs. F2, delta2b), F_4 (eqs. delta4, delta4b) from
               one 3-D FFT per moment field, sign e^{-ik.x}.
bin_power      shell average (eq. shell) in half-open bins and P_0, P_2, P_4
               (eqs. P0_impl, P2_impl, P4_impl), P_4b (eqs. P4fast, P4_implb; constant
               35/2 and the 7/2 N_0 self-pair term of |F_2|^2), and P_6b, P_8b by
               the same line-of-sight split (Sec. II.B after eq. P4fast).
"""
from __future__ import annotations

import math

import numpy as np

try:
    import scipy.fft as _sfft

    def rfftn(a):
        return _sfft.rfftn(a, workers=-1)

    def irfftn(a, s):
        return _sfft.irfftn(a, s=s, workers=-1)
except Exception:  # pragma: no cover
    def rfftn(a):
        return np.fft.rfftn(a)

    def irfftn(a, s):
        return np.fft.irfftn(a, s=s)


# The 6 distinct components of the symmetric rank-2 tensor and their
# multiplicities in k^_a k^_b Q_ab (eq. delta2b): diagonal 1, off-diagonal 2.
RANK2 = [((0, 0), 1), ((1, 1), 1), ((2, 2), 1),
         ((0, 1), 2), ((1, 2), 2), ((2, 0), 2)]

# The 15 distinct components of the symmetric rank-4 tensor and their
# multiplicities in k^k^k^k^ Q (eq. delta4b): 1 (x3), 4 (x6), 6 (x3), 12 (x3).
RANK4 = [((0, 0, 0, 0), 1), ((1, 1, 1, 1), 1), ((2, 2, 2, 2), 1),
         ((0, 0, 0, 1), 4), ((0, 0, 0, 2), 4), ((1, 1, 1, 0), 4),
         ((1, 1, 1, 2), 4), ((2, 2, 2, 0), 4), ((2, 2, 2, 1), 4),
         ((0, 0, 1, 1), 6), ((1, 1, 2, 2), 6), ((2, 2, 0, 0), 6),
         ((0, 0, 1, 2), 12), ((1, 1, 0, 2), 12), ((2, 2, 0, 1), 12)]


# ---------------------------------------------------------------------------
# Geometry helpers
# ---------------------------------------------------------------------------

def _geom(g):
    """Normalise a geometry dict: L, N, assign (2 CIC / 3 TSC), origin,
    observer (None for an observer at infinity, then los), compensate,
    P_fkp, alpha_mode (0 = W_g/W_r, 1 = N_g/N_r)."""
    out = dict(g)
    out.setdefault("origin", (0.0, 0.0, 0.0))
    out.setdefault("observer", (0.0, 0.0, 0.0))
    out.setdefault("los", (0.0, 0.0, 1.0))
    out.setdefault("compensate", True)
    out.setdefault("P_fkp", 1e4)
    out.setdefault("alpha_mode", 0)
    out.setdefault("assign", 2)
    out.setdefault("interlace", False)
    return out


def fkp_weights(nbar, P_fkp):
    """FKP weight w = 1/(1 + nbar P_FKP) (the weighting named above eq. F0)."""
    return 1.0 / (1.0 + np.asarray(nbar, dtype=np.float64) * P_fkp)


def _cat(c, P_fkp):
    pos = np.stack([np.asarray(c["x"], dtype=np.float64),
                    np.asarray(c["y"], dtype=np.float64),
                    np.asarray(c["z"], dtype=np.float64)], axis=1)
    nbar = np.asarray(c["nbar"], dtype=np.float64)
    if c.get("w") is not None:
        w = np.asarray(c["w"], dtype=np.float64)
    else:
        w = fkp_weights(nbar, P_fkp)
    return pos, w, nbar


def _los_unit(pos, g):
    """x^ of each position about the observer (x^ = 0 at the observer itself);
    the fixed line of sight when the observer is at infinity."""
    if g["observer"] is None:
        los = np.asarray(g["los"], dtype=np.float64)
        los = los / np.linalg.norm(los)
        return np.broadcast_to(los, pos.shape).copy()
    d = pos - np.asarray(g["observer"], dtype=np.float64)[None, :]
    r = np.linalg.norm(d, axis=1)
    out = np.zeros_like(d)
    nz = r > 0
    out[nz] = d[nz] / r[nz, None]
    return out


# ---------------------------------------------------------------------------
# a1: scalars
# ---------------------------------------------------------------------------

def scalars(gal, ran, geom):
    """alpha, I_22, I_33, N_0 (true and FKP forms), S_3 and L^ab at k=0."""
    g = _geom(geom)
    _, wg, _ = _cat(gal, g["P_fkp"])
    pr, wr, nr = _cat(ran, g["P_fkp"])
    Wg, Wr = wg.sum(), wr.sum()
    alpha = Wg / Wr if g["alpha_mode"] == 0 else wg.size / wr.size
    xh = _los_unit(pr, g)
    lab = np.array([np.sum(xh[:, a] * xh[:, b] * wr) for (a, b), _ in RANK2]) / Wr
    return dict(
        W_g=Wg, W_r=Wr, alpha=alpha,
        I22=alpha * np.sum(nr * wr ** 2),
        I33=alpha * np.sum(nr ** 2 * wr ** 3),
        N0=np.sum(wg ** 2) + alpha ** 2 * np.sum(wr ** 2),
        N0_fkp=alpha * (1.0 + alpha) * np.sum(wr ** 2),
        S3=np.sum(wg ** 3) - alpha ** 3 * np.sum(wr ** 3),
        Lab=lab,  # order xx, yy, zz, xy, yz, zx
        n_gal=wg.size, n_ran=wr.size,
    )


# ---------------------------------------------------------------------------
# a2: gridding (eq. mapFFT)
# ---------------------------------------------------------------------------

def assign(pos, values, geom):
    """Sum of values * W(x_node - x_j) on the N^3 grid [z][y][x], FP64.

    u = (x - origin)/H.  CIC: i0 = floor(u), d = u - i0, weights (1-d, d) on
    (i0, i0+1).  TSC: i0 = floor(u + 1/2), d = u - i0, weights
    (1/2 - d)^2/2, 3/4 - d^2, (1/2 + d)^2/2 on (i0-1, i0, i0+1).  PCS (the
    paper's fourth-order interpolation, Sec. III.A after eq. mapFFT): i0 =
    floor(u), d = u - i0, the cubic B-spline weights (1-d)^3/6,
    (4 - 6d^2 + 3d^3)/6, (1 + 3d + 3d^2 - 3d^3)/6, d^3/6 on (i0-1, ..., i0+2).
    Node indices are taken mod N.
    """
    g = _geom(geom)
    N, L, p = int(g["N"]), float(g["L"]), int(g["assign"])
    H = L / N
    u = (pos - np.asarray(g["origin"], dtype=np.float64)[None, :]) / H
    taps = []  # per axis: list of (index offset array, weight array)
    for a in range(3):
        if p == 2:
            i0 = np.floor(u[:, a])
            d = u[:, a] - i0
            taps.append([(i0, 1.0 - d), (i0 + 1, d)])
        elif p == 3:
            i0 = np.floor(u[:, a] + 0.5)
            d = u[:, a] - i0
            taps.append([(i0 - 1, 0.5 * (0.5 - d) ** 2), (i0, 0.75 - d * d),
                         (i0 + 1, 0.5 * (0.5 + d) ** 2)])
        elif p == 4:
            i0 = np.floor(u[:, a])
            d = u[:, a] - i0
            taps.append([(i0 - 1, (1.0 - d) ** 3 / 6.0), (i0, (4.0 - 6.0 * d * d + 3.0 * d ** 3) / 6.0),
                         (i0 + 1, (1.0 + 3.0 * d + 3.0 * d * d - 3.0 * d ** 3) / 6.0), (i0 + 2, d ** 3 / 6.0)])
        else:
            raise ValueError("assign must be 2 (CIC), 3 (TSC) or 4 (PCS)")
    grid = np.zeros(N * N * N)
    for iz, wz in taps[2]:
        jz = np.mod(iz.astype(np.int64), N)
        for iy, wy in taps[1]:
            jy = np.mod(iy.astype(np.int64), N)
            for ix, wx in taps[0]:
                jx = np.mod(ix.astype(np.int64), N)
                grid += np.bincount((jz * N + jy) * N + jx, weights=values * wx * wy * wz,
                                    minlength=N * N * N)
    return grid.reshape(N, N, N)


def fkp_grids(gal, ran, geom, with_w2=False):
    """F(x) = sum_g w W - alpha sum_r w W and, optionally,
    F^w(x) = sum_g w^2 W + alpha^2 sum_r w^2 W (the w^2-weighted field of
    eq. SNbisp2)."""
    g = _geom(geom)
    sc = scalars(gal, ran, g)
    pg, wg, _ = _cat(gal, g["P_fkp"])
    pr, wr, _ = _cat(ran, g["P_fkp"])
    a = sc["alpha"]
    F = assign(pg, wg, g) - a * assign(pr, wr, g)
    Fw = None
    if with_w2:
        Fw = assign(pg, wg ** 2, g) + a * a * assign(pr, wr ** 2, g)
    return F, Fw, sc


# ---------------------------------------------------------------------------
# a3-a5: moments, FFTs, Legendre fields
# ---------------------------------------------------------------------------

def node_xhat(geom):
    """x^ at every grid node origin + iH, as three [z][y][x] arrays."""
    g = _geom(geom)
    N, L = int(g["N"]), float(g["L"])
    H = L / N
    o = np.asarray(g["origin"], dtype=np.float64)
    if g["observer"] is None:
        los = np.asarray(g["los"], dtype=np.float64)
        los = los / np.linalg.norm(los)
        return [np.full((N, N, N), los[a]) for a in range(3)]
    ob = np.asarray(g["observer"], dtype=np.float64)
    X = (o[0] + H * np.arange(N) - ob[0])[None, None, :]
    Y = (o[1] + H * np.arange(N) - ob[1])[None, :, None]
    Z = (o[2] + H * np.arange(N) - ob[2])[:, None, None]
    r = np.sqrt(X * X + Y * Y + Z * Z)
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = np.where(r > 0, 1.0 / r, 0.0)
    return [X * inv, Y * inv, Z * inv]


def mode_vectors(N):
    """Integer mode components (nx, ny, nz) broadcast over the rfft
    half-spectrum [kz][ky][kx], n_a in (-N/2, N/2]."""
    n1 = np.fft.fftfreq(N, d=1.0 / N)
    nh = np.fft.rfftfreq(N, d=1.0 / N)
    return nh[None, None, :], n1[None, :, None], n1[:, None, None]


def window(N, p):
    """Assignment window prod_a sinc(pi n_a / N)^p on the half-spectrum."""
    nx, ny, nz = mode_vectors(N)
    return (np.sinc(nx / N) * np.sinc(ny / N) * np.sinc(nz / N)) ** p


def legendre(grid, geom, lmax=4, compensate=None, moment=None):
    """F_0, F_2, F_4 on the rfft half-spectrum of a real field.

    F_2 = 3/2 sum_ab k^_a k^_b Q_ab - F_0/2            (eqs. F2, delta2b)
    F_4 = 35/8 sum_abcd k^k^k^k^ Q_abcd - 5/2 F_2 - 7/8 F_0   (eqs. delta4, delta4b)
    with Q the FFT (sign e^{-ik.x}) of the moment field of each distinct
    tensor component (a, b, ...): grid * x^_a x^_b (...) with x^ at the grid
    node, or moment((a, b, ...)) when given (the per-object fields of
    object_moments); n = 0 gets k^ = 0.  Divided by the assignment window
    when compensating.
    """
    g = _geom(geom)
    N = int(g["N"])
    comp = g["compensate"] if compensate is None else compensate
    F0 = rfftn(grid)
    out = {0: F0}
    if lmax >= 2:
        nx, ny, nz = mode_vectors(N)
        nn = np.sqrt(nx * nx + ny * ny + nz * nz)
        with np.errstate(divide="ignore", invalid="ignore"):
            inv = np.where(nn > 0, 1.0 / nn, 0.0)
        kh = [nx * inv, ny * inv, nz * inv]
        if moment is None:
            xh = node_xhat(g)

            def moment(e):
                out_e = grid
                for a in e:
                    out_e = out_e * xh[a]
                return out_e
        S2 = np.zeros_like(F0)
        for (a, b), m in RANK2:
            S2 += m * kh[a] * kh[b] * rfftn(moment((a, b)))
        F2 = 1.5 * S2 - 0.5 * F0
        out[2] = F2
        if lmax >= 4:
            S4 = np.zeros_like(F0)
            for (a, b, c, d), m in RANK4:
                S4 += m * kh[a] * kh[b] * kh[c] * kh[d] * rfftn(moment((a, b, c, d)))
            out[4] = 35.0 / 8.0 * S4 - 2.5 * F2 - 7.0 / 8.0 * F0
    if comp:
        W = window(N, int(g["assign"]))
        out = {l: v / W for l, v in out.items()}
    return out


def shifted_geometry(geom):
    """The second grid of an interlaced pair: nodes at origin + (i + 1/2) H."""
    g = _geom(geom)
    H = float(g["L"]) / int(g["N"])
    g2 = dict(g)
    g2["origin"] = tuple(float(o) + 0.5 * H for o in g["origin"])
    return g2


def interlace_fields(F1, F2, N):
    """F_l = [F_l^(1) + e^{-i pi (n_x + n_y + n_z)/N} F_l^(2)] / 2.  The
    second grid's nodes sit half a cell further along every axis, so its DFT
    refers to an origin shifted by H/2 (1, 1, 1); the phase refers it back to
    the first grid's origin, and the average cancels the aliased images of
    odd order (the interlaced grids of Sec. III.A, after eq. mapFFT)."""
    nx, ny, nz = mode_vectors(N)
    ph = np.exp(-1j * np.pi * (nx + ny + nz) / N)
    return {l: 0.5 * (F1[l] + ph * F2[l]) for l in F1}


def object_moments(gal, ran, geom, alpha):
    """The moment fields with x^ taken at each object (eq. Qab read with the
    object's own line of sight): component e = (a, b, ...) is
    sum_g w x^_a x^_b (...) W - alpha sum_r w x^_a x^_b (...) W, the
    products of x^ formed per object before the interpolation."""
    g = _geom(geom)
    pg, wg, _ = _cat(gal, g["P_fkp"])
    pr, wr, _ = _cat(ran, g["P_fkp"])
    xg, xr = _los_unit(pg, g), _los_unit(pr, g)

    def moment(e):
        mg, mr = wg.copy(), wr.copy()
        for a in e:
            mg = mg * xg[:, a]
            mr = mr * xr[:, a]
        return assign(pg, mg, g) - alpha * assign(pr, mr, g)
    return moment


def survey_fields(gal, ran, geom, lmax=4, with_w2=False):
    """F_l (and F^w_l) of a survey: the Legendre fields of its grid, or with
    interlace=True of the interlaced pair of grids, compensated by the
    window after the average.  xhat="object" in the geometry takes the
    moments with each object's own x^ (object_moments; one grid, no F^w)."""
    g = _geom(geom)
    F, Fw, sc = fkp_grids(gal, ran, g, with_w2=with_w2)
    if g.get("xhat", "node") == "object":
        if g.get("interlace") or with_w2:
            raise ValueError("per-object moments: one grid and no F^w")
        return legendre(F, g, lmax=lmax, moment=object_moments(gal, ran, g, sc["alpha"])), None, sc
    if not g.get("interlace"):
        Fl = legendre(F, g, lmax=lmax)
        Fwl = legendre(Fw, g, lmax=lmax) if with_w2 else None
        return Fl, Fwl, sc
    N = int(g["N"])
    g2 = shifted_geometry(g)
    F2, Fw2, _ = fkp_grids(gal, ran, g2, with_w2=with_w2)
    Fl = interlace_fields(legendre(F, g, lmax, compensate=False), legendre(F2, g2, lmax, compensate=False), N)
    Fwl = None
    if with_w2:
        Fwl = interlace_fields(legendre(Fw, g, lmax, compensate=False), legendre(Fw2, g2, lmax, compensate=False), N)
    if g["compensate"]:
        W = window(N, int(g["assign"]))
        Fl = {l: v / W for l, v in Fl.items()}
        if Fwl is not None:
            Fwl = {l: v / W for l, v in Fwl.items()}
    return Fl, Fwl, sc


# ---------------------------------------------------------------------------
# a5: binning and P_l
# ---------------------------------------------------------------------------

def bin_edges(kmin, dk, nbins):
    return kmin + dk * np.arange(nbins + 1)


def mode_bins(N, L, kmin, dk, nbins):
    """Bin index of every half-spectrum mode (-1 when not binned) and its
    full-grid weight (1 on the kx = 0 plane, 2 otherwise).  A mode is binned
    when n != 0, no component equals N/2, and k = k_f |n| lies in a half-open
    bin [kmin + i dk, kmin + (i+1) dk)."""
    nx, ny, nz = mode_vectors(N)
    kf = 2.0 * math.pi / L
    k = kf * np.sqrt(nx * nx + ny * ny + nz * nz)
    k = np.broadcast_to(k, (N, N, N // 2 + 1))
    edges = bin_edges(kmin, dk, nbins)
    b = np.searchsorted(edges, k, side="right") - 1
    nyq = (np.abs(nx) == N // 2) | (np.abs(ny) == N // 2) | (np.abs(nz) == N // 2)
    valid = (b >= 0) & (b < nbins) & ~np.broadcast_to(nyq, b.shape) & (k > 0)
    b = np.where(valid, b, -1)
    wt = np.broadcast_to(np.where(nx == 0, 1.0, 2.0), b.shape)
    return b, wt, k


def bin_power(F, geom, bins, I22, N0):
    """Shell averages (eq. shell) of |F_0|^2, Re F_2 F_0*, Re F_4 F_0*, |F_2|^2
    and P_0, P_2, P_4, P_4b (eqs. P0_impl, P2_impl, P4_impl, P4_implb)."""
    g = _geom(geom)
    N, L = int(g["N"]), float(g["L"])
    kmin, dk, nb = bins
    b, wt, k = mode_bins(N, L, kmin, dk, nb)
    sel = b >= 0
    bi = b[sel]
    w = wt[sel]

    def acc(v):
        return np.bincount(bi, weights=w * v[sel], minlength=nb)

    F0 = F[0]
    nmodes = acc(np.ones(b.shape))
    sk = acc(k)
    s00 = acc(np.abs(F0) ** 2)
    res = dict(nmodes=np.rint(nmodes).astype(np.int64))
    with np.errstate(divide="ignore", invalid="ignore"):
        res["k_eff"] = sk / nmodes
        res["mono_raw"] = s00 / nmodes / I22
        res["P0"] = (s00 / nmodes - N0) / I22
        if 2 in F:
            s20 = acc((F[2] * np.conj(F0)).real)
            s22 = acc(np.abs(F[2]) ** 2)
            res["P2"] = 5.0 * s20 / nmodes / I22
            res["P4b"] = (17.5 * s22 - 5.0 * s20 - 3.5 * s00) / nmodes / I22
        if 4 in F:
            s40 = acc((F[4] * np.conj(F0)).real)
            res["P4"] = 9.0 * s40 / nmodes / I22
            # l = 6 and 8 by the line-of-sight split of Sec. II.B (the remark
            # after eq. P4fast): L_6 and L_8 written through L_2 L_4 and L_4^2,
            #   L_2 L_4 = 2/7 L_2 + 20/77 L_4 + 5/11 L_6,
            #   L_4^2 = 1/9 + 100/693 L_2 + 162/1001 L_4 + 20/99 L_6 + 490/1287 L_8,
            # with each product's two factors taken about different lines of
            # sight (F_2 F_4*, |F_4|^2).  The L_6 term of L_4^2 uses the split
            # L_6; the self-pair shot noise of |F_4|^2 (N_0/9) cancels against
            # the 1/9 |F_0|^2 term.
            s42 = acc((F[4] * np.conj(F[2])).real)
            s44 = acc(np.abs(F[4]) ** 2)
            s60 = 11.0 / 5.0 * (s42 - 2.0 / 7.0 * s20 - 20.0 / 77.0 * s40)
            s80 = 1287.0 / 490.0 * (s44 - s00 / 9.0 - 100.0 / 693.0 * s20 - 162.0 / 1001.0 * s40
                                    - 20.0 / 99.0 * s60)
            res["P6b"] = 13.0 * s60 / nmodes / I22
            res["P8b"] = 17.0 * s80 / nmodes / I22
    return res


def power(gal, ran, geom, bins, lmax=4):
    """P_0, P_2, P_4, P_4b of a survey (gridded FFT estimator, FP64)."""
    g = _geom(geom)
    Fl, _, sc = survey_fields(gal, ran, g, lmax=lmax)
    res = bin_power(Fl, g, bins, sc["I22"], sc["N0"])
    res.update({k: sc[k] for k in ("alpha", "I22", "I33", "N0", "N0_fkp", "S3", "Lab", "W_g", "W_r")})
    return res


def power_from_grid(grid, geom, bins, I22=1.0, N0=0.0, lmax=4):
    """The same estimator applied to a given real grid F(x)."""
    g = _geom(geom)
    Fl = legendre(np.asarray(grid, dtype=np.float64), g, lmax=lmax)
    return bin_power(Fl, g, bins, I22, N0)
