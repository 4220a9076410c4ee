"""Pins for the FP64 bispectrum oracle: brute-force closed-triangle enumeration
in k-space (eq. Factorize read right to left), explicit inverse DFTs for the
shell fields (eq. F_k), exact integer triangle counts (eq. NT) and the thin-shell
approximation of N_T."""
import math

import numpy as np
import pytest

import mockgen
from oracle import bispectrum as ob
from oracle import power as op


def full_spectrum(Fh, N):
    """Full-grid F(n) for n in (-N/2, N/2]^3 from the rfft half-spectrum of a
    real field (F(-n) = F(n)*), as a dict keyed by integer mode tuples."""
    out = {}
    n1 = np.fft.fftfreq(N, 1.0 / N).astype(int)
    for iz in range(N):
        for iy in range(N):
            for ix in range(N // 2 + 1):
                v = Fh[iz, iy, ix]
                n = (ix, n1[iy], n1[iz])
                out[n] = v
                out[(-n[0], -n[1], -n[2])] = np.conj(v)
    return out


def shell_modes(N, bshells, s):
    lo, hi, _ = ob.shell_bounds(bshells)
    r = np.arange(-(N // 2) + 1, N // 2)
    nx, ny, nz = np.meshgrid(r, r, r, indexing="ij")
    n2 = nx ** 2 + ny ** 2 + nz ** 2
    m = (n2 >= lo[s] ** 2) & (n2 < hi[s] ** 2) & (n2 > 0)
    return np.stack([nx[m], ny[m], nz[m]], 1)


def test_shell_field_is_inverse_dft():
    """F_k(x) = sum_{n in shell} F(n) e^{+2 pi i n.x/N}, by explicit summation."""
    N = 12
    bs = (2, 2, 2, 2)
    f = mockgen.rng(2, 1).standard_normal((N, N, N))
    Fh = op.rfftn(f)
    sidx, _ = ob.shell_index(N, bs)
    full = full_spectrum(Fh, N)
    g = np.arange(N)
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    for s in range(2):
        got = ob.shell_field(Fh, sidx, s, N)
        ref = np.zeros((N, N, N), dtype=complex)
        for n in shell_modes(N, bs, s):
            ref += full[tuple(n)] * np.exp(2j * np.pi * (n[0] * x + n[1] * y + n[2] * z) / N)
        assert np.max(np.abs(ref.imag)) < 1e-9
        assert np.max(np.abs(got - ref.real)) < 1e-10 * np.max(np.abs(ref))


@pytest.mark.parametrize("N,bs", [(16, (1, 1, 1, 4)), (24, (2, 2, 2, 3))])
def test_triangle_sums_and_counts_brute_force(N, bs):
    """sum_x F_a^(l) F_b^(0) F_c^(0) / N^3 equals the k-space sum over closed
    triangles n1+n2+n3 = 0 with n_i in shells a, b, c (eq. Factorize), and the
    exact count N_T equals the number of such triangles (eq. NT)."""
    f = mockgen.rng(3, N).standard_normal((N, N, N))
    g = dict(N=N, L=100.0, assign=2, origin=(0, 0, 0), observer=(-40.0, 13.0, 77.0), compensate=False)
    F = op.legendre(f, g, lmax=2)
    sidx, _ = ob.shell_index(N, bs)
    full = {l: full_spectrum(F[l], N) for l in (0, 2)}
    S = bs[3]
    shells = [shell_modes(N, bs, s) for s in range(S)]
    lo, hi, _ = ob.shell_bounds(bs)
    assert 3 * hi[-1] < N  # no aliasing of n1+n2+n3 = 0 mod N
    counter = ob.Counter(N, bs)
    for (a, b, c) in ob.triangle_list(S):
        na, nb = shells[a], shells[b]
        n3 = -(na[:, None, :] + nb[None, :, :])
        q = (n3 ** 2).sum(-1)
        ok = (q >= lo[c] ** 2) & (q < hi[c] ** 2)
        ia, ib = np.nonzero(ok)
        nt = ia.size
        assert counter.count(a, b, c) == nt
        if nt == 0:
            continue
        for l in (0, 2):
            ref = 0.0
            for i, j in zip(ia, ib):
                m3 = tuple(n3[i, j])
                ref += full[l][tuple(na[i])] * full[0][tuple(nb[j])] * full[0][m3]
            T = np.sum(ob.shell_field(F[l], sidx, a, N) * ob.shell_field(F[0], sidx, b, N)
                       * ob.shell_field(F[0], sidx, c, N)) / N ** 3
            assert abs(ref.imag) < 1e-9 * max(1.0, abs(ref.real))
            assert abs(T - ref.real) < 1e-9 * max(1.0, abs(ref.real)), (a, b, c, l)


def test_counts_symmetric_and_thin_shell():
    """N_T is symmetric in its shells and approaches 8 pi^2 k1 k2 k3 dk^3
    (eq. NT, thin-shell form) for wide, well-closed triangles."""
    N = 48
    bs = (6, 3, 3, 4)  # centres 6, 9, 12, 15
    c = ob.Counter(N, bs)
    assert c.count(3, 2, 1) == c.count(2, 3, 1) == c.count(1, 3, 2)
    _, _, cen = ob.shell_bounds(bs)
    for (a, b, cc) in [(3, 2, 1), (2, 2, 1), (3, 3, 3)]:
        approx = 8 * math.pi ** 2 * cen[a] * cen[b] * cen[cc] * 27
        assert abs(c.count(a, b, cc) / approx - 1) < 0.12


def test_bispectrum_plane_parallel_reduces_to_legendre_weighted_sum():
    """Observer at infinity: F_l = L_l(mu) F_0, so T^(l) is the closed-triangle
    sum of L_l(mu_1) F_0 F_0 F_0 (eqs. Bquad, Bispell4 in the plane-parallel
    limit); checked by brute force on a 16^3 grid."""
    N = 16
    bs = (1, 1, 1, 4)
    f = mockgen.rng(9, 0).standard_normal((N, N, N))
    g = dict(N=N, L=50.0, assign=2, observer=None, los=(0, 0, 1), compensate=False)
    F = op.legendre(f, g, lmax=4)
    full0 = full_spectrum(F[0], N)
    sidx, _ = ob.shell_index(N, bs)
    shells = [shell_modes(N, bs, s) for s in range(4)]
    lo, hi, _ = ob.shell_bounds(bs)
    a, b, c = 3, 2, 2
    na, nb = shells[a], shells[b]
    n3 = -(na[:, None, :] + nb[None, :, :])
    q = (n3 ** 2).sum(-1)
    ia, ib = np.nonzero((q >= lo[c] ** 2) & (q < hi[c] ** 2))
    for l in (2, 4):
        ref = 0.0
        for i, j in zip(ia, ib):
            mu = na[i][2] / np.linalg.norm(na[i])
            ref += ob.legendre_poly(l, mu) * full0[tuple(na[i])] * full0[tuple(nb[j])] * full0[tuple(n3[i, j])]
        T = np.sum(ob.shell_field(F[l], sidx, a, N) * ob.shell_field(F[0], sidx, b, N)
                   * ob.shell_field(F[0], sidx, c, N)) / N ** 3
        assert abs(T - ref.real) < 1e-9 * max(1.0, abs(ref.real))


def test_unclustered_bispectrum_shot_noise_statistical():
    """Parity unpinned beyond statistics: for a Poisson-sampled unclustered
    catalog the thin-shell shot-noise subtraction (eqs. Noise0, SNbisp2thin)
    leaves B_0 consistent with zero, while the raw triangle average is not."""
    N, L = 32, 400.0
    bs = (3, 3, 3, 3)
    geom = dict(N=N, L=L, assign=3, origin=(0.0, 0.0, 0.0), observer=(200.0, 200.0, -600.0), P_fkp=0.0)
    raws, subs = [], []
    for seed in range(4):
        gal = mockgen.uniform_points(30000, 40.0, 360.0, seed=seed, stream=30)
        ran = mockgen.uniform_points(300000, 40.0, 360.0, seed=seed, stream=31)
        res = ob.bispectrum(gal, ran, geom, bs, ells=(0,), tris=[(2, 2, 2), (2, 1, 1), (1, 1, 1), (2, 2, 1)])
        raws.append(res["B0"] + res["N0"])
        subs.append(res["B0"])
    raws, subs = np.array(raws), np.array(subs)
    mean_sub = subs.mean(0)
    err = subs.std(0, ddof=1) / math.sqrt(len(subs))
    assert np.all(np.abs(mean_sub) < 4 * err + 1e-3 * np.abs(raws.mean(0)))
    assert np.all(np.abs(raws.mean(0)) > 3 * err)
    assert np.all(np.abs(mean_sub) < 0.3 * np.abs(raws.mean(0)))


def single_object_case():
    """One galaxy (w = 1) exactly on a node of a 16^3 periodic CIC grid (L = 16,
    no compensation) and one random (w = 128) on every node, nbar = 2^-10,
    alpha = N_g/N_r = 2^-12; shells centred on 2, 3, 4 k_f, width k_f."""
    N = 16
    i = np.arange(N, dtype=np.float64)
    z, y, x = np.meshgrid(i, i, i, indexing="ij")
    ran = dict(x=x.ravel().astype(np.float32), y=y.ravel().astype(np.float32), z=z.ravel().astype(np.float32),
               w=np.full(N ** 3, 128.0, dtype=np.float32), nbar=np.full(N ** 3, 2.0 ** -10, dtype=np.float32))
    gal = dict(x=np.array([5.0], np.float32), y=np.array([6.0], np.float32), z=np.array([7.0], np.float32),
               w=np.array([1.0], np.float32), nbar=np.array([2.0 ** -10], np.float32))
    geom = dict(L=16.0, N=N, assign=2, compensate=False, periodic=True, alpha_mode=1,
                origin=(0.0, 0.0, 0.0), observer=(8.0, 8.0, -40.0))
    return gal, ran, geom, (2, 1, 1, 3)


def test_single_object_thin_shell_shot_noise_identity():
    """A single object's bispectrum is all shot noise.  With one galaxy on a
    node (CIC puts all of it there) F_0(q) = w e^{iq.x} on every shell mode,
    and randoms on every node contribute nothing at q != 0.  So every closed
    triangle sums to w^3 (B-hat_0 = w^3/I_33), and each of the three pair terms
    of eq. SNbisp2thin is the shell mean of F_0 F^w_0* = w^3; the triple term is
    -2 (w^3 - alpha^3 sum_r w_r^3)/I_33.  Hence, for every triangle,
      N_0 = [3 w^3 - 2 (w^3 - alpha^3 sum_r w_r^3)] / I_33 = 0.625,
      B_0 = B-hat_0 - N_0 = -2 alpha^3 sum_r w_r^3 / I_33 = -2 alpha^2/nbar^2 = -0.125,
    with I_33 = alpha sum_r nbar^2 w_r^3 = 2 and B-hat_0 = 0.5: every term is
    of order one, so a dropped or mis-weighted pair term, a wrong sign or
    alpha power in the triple term, or a normalisation of B-hat and N_0 that
    differ all fail."""
    gal, ran, geom, bs = single_object_case()
    ref = ob.bispectrum(gal, ran, geom, bs, ells=(0,))
    assert len(ref["tri"]) >= 5
    assert abs(ref["I33"] - 2.0) < 1e-12
    assert np.max(np.abs(ref["N0"] - 0.625)) < 1e-12
    assert np.max(np.abs(ref["B0"] + 0.125)) < 1e-12


def _leg(l, mu):
    """Textbook Legendre polynomials L_0, L_2, L_4."""
    return {0: np.ones_like(mu), 2: 0.5 * (3 * mu ** 2 - 1), 4: (35 * mu ** 4 - 30 * mu ** 2 + 3) / 8.0}[l]


def test_thin_shell_shot_noise_from_direct_point_sums():
    """Objects exactly on the nodes of a 12^3 periodic CIC grid (no
    compensation), observer outside the box: then F_l(q) = sum_j c_j w_j
    L_l(q^.x^_j) e^{-iq.x_j} (c = 1 for galaxies, -alpha for randoms) and
    F^w_l(q) = sum_j c'_j w_j^2 L_l(q^.x^_j) e^{-iq.x_j} (c' = 1, alpha^2), the
    definitions below eq. SNbisp2, summed directly over the objects with no
    grid, moment field or FFT.  The thin-shell noise of eq. SNbisp2thin built
    from those direct sums (shell means over every mode of each shell,
    Legendre factors at the shell-centre cosines) equals the oracle's for
    l = 0, 2, 4 on every triangle."""
    N, L = 12, 12.0
    g = mockgen.rng(5, 3)
    gi = g.integers(0, N, size=(6, 3)).astype(np.float64)
    ri = g.integers(0, N, size=(40, 3)).astype(np.float64)
    wg, wr = g.uniform(0.5, 2.0, 6), g.uniform(0.5, 1.5, 40)
    nb = np.full(46, 2.0 ** -9)

    def cat(p, w, n):
        return dict(x=p[:, 0].astype(np.float32), y=p[:, 1].astype(np.float32), z=p[:, 2].astype(np.float32),
                    w=w.astype(np.float32), nbar=n.astype(np.float32))

    gal, ran = cat(gi, wg, nb[:6]), cat(ri, wr, nb[6:])
    obs = np.array([6.3, 5.7, -9.1])
    geom = dict(L=L, N=N, assign=2, compensate=False, periodic=True, observer=tuple(obs), origin=(0.0, 0.0, 0.0))
    bs = (1, 1, 1, 3)
    ref = ob.bispectrum(gal, ran, geom, bs, ells=(0, 2, 4))
    # direct sums (float32-rounded inputs, as the oracle reads them)
    wg32, wr32 = wg.astype(np.float32).astype(np.float64), wr.astype(np.float32).astype(np.float64)
    alpha = wg32.sum() / wr32.sum()
    pos = np.concatenate([gi, ri])
    w = np.concatenate([wg32, wr32])
    c1 = np.concatenate([np.ones(6), -alpha * np.ones(40)])
    c2 = np.concatenate([np.ones(6), alpha ** 2 * np.ones(40)])
    xhat = (pos - obs) / np.linalg.norm(pos - obs, axis=1)[:, None]
    I33 = alpha * np.sum(2.0 ** -18 * wr32 ** 3)
    S3 = np.sum(wg32 ** 3) - alpha ** 3 * np.sum(wr32 ** 3)
    assert abs(ref["I33"] / I33 - 1) < 1e-12
    lo, hi, cen = ob.shell_bounds(bs)
    r = np.arange(-(N // 2) + 1, N // 2)
    modes = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3).astype(np.float64)
    nn = np.linalg.norm(modes, axis=1)
    SQ = {}
    for s in range(bs[3]):
        m = modes[(nn >= lo[s]) & (nn < hi[s]) & (nn > 0)]
        q = 2 * np.pi * m / L
        ph = np.exp(-1j * q @ pos.T)                       # [mode][object]
        mu = (m / np.linalg.norm(m, axis=1)[:, None]) @ xhat.T
        F = {l: (ph * _leg(l, mu) * (c1 * w)).sum(1) for l in (0, 2, 4)}
        Fw = {l: (ph * _leg(l, mu) * (c2 * w ** 2)).sum(1) for l in (0, 2, 4)}
        for l in (0, 2, 4):
            SQ[(l, 0, s)] = np.mean((F[l] * np.conj(Fw[0])).real)
            SQ[(0, l, s)] = np.mean((F[0] * np.conj(Fw[l])).real)
    scale = max(abs(v) for v in SQ.values()) / I33
    nclosed = 0
    for t, (a, b, c) in enumerate(ref["tri"]):
        A, B, C = cen[a], cen[b], cen[c]
        if abs(A - B) <= C <= A + B:
            # the triangle's own vectors: q1 along x, q2 at the angle that
            # closes |q1 + q2| = C, q3 = -(q1 + q2); cosines by dot products
            from scipy.optimize import brentq
            th = brentq(lambda u: np.hypot(A + B * np.cos(u), B * np.sin(u)) - C, 0.0, np.pi) \
                if A + B > C > abs(A - B) else (0.0 if C == A + B else np.pi)
            q1 = np.array([A, 0.0, 0.0])
            q2 = B * np.array([np.cos(th), np.sin(th), 0.0])
            q3 = -(q1 + q2)
            mu12 = q1 @ q2 / (A * B)
            mu13 = q1 @ q3 / (A * np.linalg.norm(q3))
            nclosed += 1
        else:
            # centres that do not close (the shells' widths make N_T > 0):
            # the cosines clipped to +-1, the oracle's reading
            mu12 = np.clip((C ** 2 - A ** 2 - B ** 2) / (2 * A * B), -1, 1)
            mu13 = np.clip((B ** 2 - A ** 2 - C ** 2) / (2 * A * C), -1, 1)
        for l in (0, 2, 4):
            n = (2 * l + 1) / I33 * (SQ[(l, 0, a)] + _leg(l, mu12) * SQ[(0, l, b)] + _leg(l, mu13) * SQ[(0, l, c)])
            if l == 0:
                n -= 2 * S3 / I33
            assert abs(ref[f"N{l}"][t] - n) < 1e-9 * scale, (l, (a, b, c), ref[f"N{l}"][t], n)
    assert nclosed >= len(ref["tri"]) // 2


def test_counts_for_pair_equals_single_counts():
    """The all-shells form of the exact counter (used to write the stored
    triangle-count fixtures) gives each count() value."""
    N, bs = 24, (2, 1, 1, 5)
    counter = ob.Counter(N, bs)
    for b in range(bs[3]):
        for c in range(b + 1):
            allc = counter.counts_for_pair(b, c)
            for a in range(b, bs[3]):
                assert allc[a] == counter.count(a, b, c)


def test_split_hexadecapole_sum_brute_force():
    """The triangle sum of eq. Bhexa2 (delta_2 on the two larger sides),
    T22 = sum_x F_a^(2) F_b^(2) F_c^(0), equals N^3 times the k-space sum over
    closed triangles of F_2(n1) F_2(n2) F_0(n3), and B4b is
    [35/2 T22 - 5 T2 - 7/2 T0] / (N^3 N_T I_33)."""
    N, bs = 16, (1, 1, 1, 4)
    f = mockgen.rng(4, N).standard_normal((N, N, N))
    g = dict(N=N, L=100.0, assign=2, origin=(0, 0, 0), observer=(-40.0, 13.0, 77.0), compensate=False)
    F = op.legendre(f, g, lmax=2)
    full = {l: full_spectrum(F[l], N) for l in (0, 2)}
    S = bs[3]
    shells = [shell_modes(N, bs, s) for s in range(S)]
    lo, hi, _ = ob.shell_bounds(bs)
    sc = dict(I33=1.7, S3=0.0)
    res = ob.bispectrum_from_fields(F, F, sc, N, bs, ells=(0, 2), zero_area=True)
    for t, (a, b, c) in enumerate(res["tri"]):
        na, nb = shells[a], shells[b]
        n3 = -(na[:, None, :] + nb[None, :, :])
        q = (n3 ** 2).sum(-1)
        ia, ib = np.nonzero((q >= lo[c] ** 2) & (q < hi[c] ** 2))
        ref = sum(full[2][tuple(na[i])] * full[2][tuple(nb[j])] * full[0][tuple(n3[i, j])] for i, j in zip(ia, ib))
        assert abs(ref.imag) < 1e-9 * max(1.0, abs(ref.real))
        assert abs(res["T22"][t] / N ** 3 - ref.real) < 1e-9 * max(1.0, abs(ref.real)), (a, b, c)
        nt = res["NT"][t]
        b4b = (17.5 * res["T22"][t] - 5 * res["T2"][t] - 3.5 * res["T0"][t]) / (N ** 3 * nt * 1.7)
        assert abs(res["B4b"][t] - b4b) < 1e-12 * max(1.0, abs(b4b))
