"""Pins for the FP64 power-spectrum oracle: each check compares the oracle with
something other than itself (an explicit DFT, a direct 1-LOS Yamamoto sum, a
closed form, a lattice identity, the constants the paper prints)."""
import json
import math
import os

import numpy as np
import pytest
from scipy.special import eval_legendre

import mockgen
from oracle import power as op

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


# ---------------------------------------------------------------------------
# brute-force helpers (no FFT)
# ---------------------------------------------------------------------------

def explicit_dft(f):
    """F(n) = sum_x f(x) exp(-2 pi i n.x / N) by an explicit N^3 x N^3 sum,
    returned on the rfft half-spectrum [nz][ny][nx]."""
    N = f.shape[0]
    g = np.arange(N)
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    xv = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)
    nx, ny, nz = np.meshgrid(np.arange(N // 2 + 1), g, g, indexing="ij")
    # order the half-spectrum as [nz][ny][nx]
    nz, ny, nx = np.meshgrid(g, g, np.arange(N // 2 + 1), indexing="ij")
    nv = np.stack([nx.ravel(), ny.ravel(), nz.ravel()], axis=1)
    ph = (nv @ xv.T) % N
    E = np.exp(-2j * np.pi * ph / N)
    return (E @ f.ravel()).reshape(N, N, N // 2 + 1)


def full_modes(N):
    """All integer mode vectors n with components in (-N/2, N/2)."""
    r = np.arange(-(N // 2) + 1, N // 2)
    nx, ny, nz = np.meshgrid(r, r, r, indexing="ij")
    return np.stack([nx.ravel(), ny.ravel(), nz.ravel()], axis=1)


def direct_yamamoto(pos, w, xhat, modes, kf, l):
    """F_l(k) = sum_j w_j exp(-i k.x_j) L_l(k^.x^_j) for each mode (1-LOS form)."""
    k = modes * kf
    kn = np.linalg.norm(k, axis=1)
    kh = np.where(kn[:, None] > 0, k / np.where(kn > 0, kn, 1.0)[:, None], 0.0)
    ph = np.exp(-1j * (k @ pos.T))
    mu = kh @ xhat.T
    return (ph * eval_legendre(l, mu) * w[None, :]).sum(axis=1)


def lattice_bins(modes, kf, kmin, dk, nb):
    k = kf * np.linalg.norm(modes, axis=1)
    b = np.full(k.shape, -1)
    for i in range(nb):
        lo, hi = kmin + i * dk, kmin + (i + 1) * dk
        b[(k >= lo) & (k < hi) & (k > 0)] = i
    return b


# ---------------------------------------------------------------------------
# FFT and gridding
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("N", [6, 8, 10, 12])
def test_fft_is_the_dft(N):
    f = mockgen.rng(1, N).standard_normal((N, N, N))
    ref = explicit_dft(f)
    got = op.rfftn(f)
    assert np.max(np.abs(got - ref)) < 1e-11 * np.max(np.abs(ref))


def _bspline(s, p):
    """The centred B-spline of order p (textbook piecewise polynomials)."""
    s = np.abs(s)
    if p == 2:
        return np.where(s < 1, 1 - s, 0.0)
    if p == 3:
        return np.where(s < 0.5, 0.75 - s * s, np.where(s < 1.5, 0.5 * (1.5 - s) ** 2, 0.0))
    return np.where(s < 1, (4 - 6 * s * s + 3 * s ** 3) / 6, np.where(s < 2, (2 - s) ** 3 / 6, 0.0))


@pytest.mark.parametrize("p", [2, 3, 4])
def test_assignment_is_the_bspline_kernel(p):
    """Each node gets w * prod_a B_p(node_a - u_a): the order-p B-spline
    (CIC p=2, TSC p=3, PCS p=4) of the distance in cells, with periodic
    wrap."""
    N, L = 8, 8.0
    g = dict(N=N, L=L, assign=p, origin=(0.0, 0.0, 0.0))
    pts = np.array([[3.25, 4.0, 0.1], [7.9, 0.5, 2.5], [0.0, 6.49, 5.51]])
    w = np.array([1.0, 0.5, 2.0])
    grid = op.assign(pts, w, g)
    ref = np.zeros((N, N, N))
    nodes = np.arange(N)
    for j in range(len(w)):
        fac = []
        for a in range(3):
            d = nodes - pts[j, a]
            d = (d + N / 2) % N - N / 2  # periodic distance
            fac.append(_bspline(d, p))
        ref += w[j] * fac[2][:, None, None] * fac[1][None, :, None] * fac[0][None, None, :]
    assert np.max(np.abs(grid - ref)) < 1e-14
    assert abs(grid.sum() - w.sum()) < 1e-13


# ---------------------------------------------------------------------------
# Legendre fields
# ---------------------------------------------------------------------------

def test_single_object_closed_form():
    """One object at a node: F_l(k) F_0*(k) = w^2 L_l(k^.x^_j) for every mode."""
    N, L = 16, 16.0
    obs = (-3.3, 2.7, -5.1)
    g = dict(N=N, L=L, assign=2, origin=(0.0, 0.0, 0.0), observer=obs, compensate=False)
    pos = np.array([[5.0, 9.0, 12.0]])
    w = np.array([0.7])
    grid = op.assign(pos, w, g)
    F = op.legendre(grid, g, lmax=4)
    xh = (pos[0] - np.array(obs)) / np.linalg.norm(pos[0] - np.array(obs))
    nx, ny, nz = op.mode_vectors(N)
    nn = np.sqrt(nx ** 2 + ny ** 2 + nz ** 2)
    mu = (nx * xh[0] + ny * xh[1] + nz * xh[2]) / np.where(nn > 0, nn, 1.0)
    m = np.broadcast_to(nn > 0, F[0].shape)
    for l in (2, 4):
        got = (F[l] * np.conj(F[0])).real
        ref = np.broadcast_to(w[0] ** 2 * eval_legendre(l, mu), got.shape)
        assert np.max(np.abs(got[m] - ref[m])) < 1e-13
        assert np.max(np.abs((F[l] * np.conj(F[0])).imag[m])) < 1e-13


def test_direct_yamamoto_sum_on_nodes():
    """Objects on nodes, CIC, no compensation: gridding is exact and the node
    x^ is the object x^, so the FFT estimator equals the direct 1-LOS sum
    (eqs. 1LOS, deltaell, mapFFT) mode by mode, and so do P_0, P_2, P_4."""
    N, L = 16, 32.0
    H = L / N
    origin = (10.0, -20.0, 5.0)
    obs = (-100.0, 40.0, -30.0)
    g = dict(N=N, L=L, assign=2, origin=origin, observer=obs, compensate=False)
    cat, _ = mockgen.node_points(150, N, L, origin, seed=3)
    pos = np.stack([cat["x"], cat["y"], cat["z"]], 1).astype(np.float64)
    w = 0.2 + mockgen.rng(3, 11).random(150)
    grid = op.assign(pos, w, g)
    F = op.legendre(grid, g, lmax=4)
    xh = pos - np.array(obs)
    xh /= np.linalg.norm(xh, axis=1)[:, None]
    kf = 2 * math.pi / L
    # on the half spectrum
    nx, ny, nz = op.mode_vectors(N)
    hm = np.stack(np.broadcast_arrays(nx, ny, nz), -1).reshape(-1, 3)
    rel = pos - np.array(origin)  # the DFT's phase origin is the box corner
    for l in (0, 2, 4):
        ref = direct_yamamoto(rel, w, xh, hm, kf, l).reshape(F[0].shape)
        nz0 = np.linalg.norm(hm, axis=1).reshape(F[0].shape) > 0
        err = np.max(np.abs(F[l][nz0] - ref[nz0]))
        assert err < 1e-11 * np.max(np.abs(ref)), (l, err)
    # P_l through the estimator vs a direct full-grid lattice average
    bins = (0.5 * kf, kf, 6)
    res = op.bin_power(F, g, bins, I22=1.0, N0=0.0)
    modes = full_modes(N)
    b = lattice_bins(modes, kf, *bins)
    Fd = {l: direct_yamamoto(rel, w, xh, modes, kf, l) for l in (0, 2, 4)}
    for i in range(bins[2]):
        s = b == i
        assert res["nmodes"][i] == s.sum()
        p0 = np.mean(np.abs(Fd[0][s]) ** 2)
        assert abs(res["P0"][i] - p0) < 1e-11 * p0
        for l, pref in ((2, 5.0), (4, 9.0)):
            pl = pref * np.mean((Fd[l][s] * np.conj(Fd[0][s])).real)
            assert abs(res[f"P{l}"][i] - pl) < 1e-11 * p0


def test_plane_parallel_kaiser_fixed_amplitude():
    """Observer at infinity, |F_0(n)|^2 = A(|n|)(1 + f mu^2)^2: then
    F_l = L_l(mu) F_0 and P_l = (2l+1) <L_l(mu)(1+f mu^2)^2 A> over the bin's
    lattice modes exactly (Sec. I Kaiser limit; Sec. II.B plane-parallel
    remark); P_4b = P_4 mode by mode (eqs. factorizeL4, P4fast)."""
    N, L, f = 32, 500.0, 0.7

    def amp(nx, ny, nz):
        n2 = nx * nx + ny * ny + nz * nz
        mu2 = np.where(n2 > 0, nz * nz / np.where(n2 > 0, n2, 1), 0.0)
        return (1.0 + np.sqrt(n2)) ** -1.5 * (1 + f * mu2) ** 2 * 1e6

    field = mockgen.random_phase_field(N, amp, seed=5)
    g = dict(N=N, L=L, assign=2, observer=None, los=(0, 0, 1), compensate=False)
    kf = 2 * math.pi / L
    bins = (0.5 * kf, kf, 15)
    res = op.power_from_grid(field, g, bins)
    modes = full_modes(N)
    b = lattice_bins(modes, kf, *bins)
    n2 = (modes ** 2).sum(1)
    mu = np.where(n2 > 0, modes[:, 2] / np.sqrt(np.where(n2 > 0, n2, 1)), 0)
    A = amp(modes[:, 0], modes[:, 1], modes[:, 2])
    for i in range(bins[2]):
        s = b == i
        for l, key in ((0, "P0"), (2, "P2"), (4, "P4")):
            ref = (2 * l + 1) * np.mean(eval_legendre(l, mu[s]) * A[s])
            scale = np.mean(A[s])
            assert abs(res[key][i] - ref) < 1e-11 * scale, (i, l)
        assert abs(res["P4b"][i] - res["P4"][i]) < 1e-11 * np.mean(A[s])
        # the split hexacontatetrapole and l = 8 multipoles: with F_l = L_l F_0
        # the split products are the one-line-of-sight ones, so P_6b and P_8b
        # are (2l+1) <L_l(mu) (1 + f mu^2)^2 A> exactly (which vanish in the
        # continuum for the Kaiser factor, but not on the lattice)
        for l, key in ((6, "P6b"), (8, "P8b")):
            ref = (2 * l + 1) * np.mean(eval_legendre(l, mu[s]) * A[s])
            assert abs(res[key][i] - ref) < 1e-10 * np.mean(A[s]), (i, l)


def test_split_multipoles_of_one_object_have_no_shot_noise_on_a_sphere():
    """One object on a node, plane-parallel (observer at infinity), no
    compensation: F_l = L_l(mu) w e^{-ik.x} mode by mode, so the split
    multipoles are (2l+1) <L_l(mu)> w^2 over each bin's modes: the shot-noise
    self-pair terms of |F_4|^2 and F_4 F_2* cancel as they do for P_4b, and
    what is left is the lattice's anisotropy, which the direct mode sum
    gives.  Checks the normalisations of the l = 6 and 8 combinations
    independently of the Kaiser factor."""
    N, L = 24, 24.0
    g = dict(N=N, L=L, assign=2, origin=(0.0, 0.0, 0.0), observer=None, los=(0.2, -0.3, 0.93), compensate=False)
    grid = op.assign(np.array([[4.0, 7.0, 11.0]]), np.array([0.9]), g)
    kf = 2 * math.pi / L
    bins = (0.5 * kf, kf, 11)
    res = op.power_from_grid(grid, g, bins)
    los = np.array(g["los"]) / np.linalg.norm(g["los"])
    modes = full_modes(N)
    b = lattice_bins(modes, kf, *bins)
    n2 = (modes ** 2).sum(1)
    mu = np.where(n2 > 0, modes @ los / np.sqrt(np.where(n2 > 0, n2, 1)), 0)
    for i in range(bins[2]):
        s = b == i
        for l, key in ((4, "P4b"), (6, "P6b"), (8, "P8b")):
            ref = (2 * l + 1) * np.mean(eval_legendre(l, mu[s])) * 0.81
            assert abs(res[key][i] - ref) < 1e-11, (i, l, res[key][i], ref)


def test_plane_parallel_isotropic_quadrupole_vanishes():
    """Isotropic amplitude A(|n|), observer at infinity: every lattice sphere
    is symmetric under axis permutations, so sum mu^2 = count/3 and P_2 = 0."""
    N, L = 24, 400.0
    field = mockgen.random_phase_field(N, lambda nx, ny, nz: 1.0 / (1.0 + nx * nx + ny * ny + nz * nz), seed=6)
    g = dict(N=N, L=L, assign=2, observer=None, los=(0, 0, 1), compensate=False)
    kf = 2 * math.pi / L
    res = op.power_from_grid(field, g, (0.5 * kf, kf, 11))
    assert np.all(np.abs(res["P2"]) < 1e-12 * res["P0"])


def test_kaiser_ratios_gaussian_amplitudes():
    """Rayleigh amplitudes: P_2/P_0 and P_4/P_0 follow the continuum Kaiser
    ratios (4f/3 + 4f^2/7)/(1 + 2f/3 + f^2/5) and (8f^2/35)/(...) within
    sample variance once averaged over many modes (Sec. I, Kaiser limit)."""
    N, L, f = 48, 1000.0, 0.7
    g0 = mockgen.rng(21, 0)
    n1 = np.fft.fftfreq(N, 1.0 / N)
    nh = np.fft.rfftfreq(N, 1.0 / N)
    nz, ny, nx = np.meshgrid(n1, n1, nh, indexing="ij")
    n2 = nx ** 2 + ny ** 2 + nz ** 2
    mu2 = np.where(n2 > 0, nz ** 2 / np.where(n2 > 0, n2, 1), 0)
    Fk = (g0.standard_normal(n2.shape) + 1j * g0.standard_normal(n2.shape)) * (1 + f * mu2)
    field = np.fft.irfftn(Fk, s=(N, N, N))
    gg = dict(N=N, L=L, assign=2, observer=None, compensate=False)
    kf = 2 * math.pi / L
    res = op.power_from_grid(field, gg, (4.5 * kf, 8 * kf, 2))
    den = 1 + 2 * f / 3 + f * f / 5
    r2 = np.sum(res["P2"] * res["nmodes"]) / np.sum(res["P0"] * res["nmodes"])
    r4 = np.sum(res["P4"] * res["nmodes"]) / np.sum(res["P0"] * res["nmodes"])
    assert abs(r2 - (4 * f / 3 + 4 * f * f / 7) / den) < 0.03
    assert abs(r4 - (8 * f * f / 35) / den) < 0.03


# ---------------------------------------------------------------------------
# scalars, weights, L^ab
# ---------------------------------------------------------------------------

def test_scalars_closed_form_uniform():
    """Constant nbar and FKP weight: alpha = N_g/N_r, I_22 = N_g nbar w^2,
    N_0 = N_g w^2 (1 + N_g/N_r), I_33 = N_g nbar^2 w^3, S_3 = N_g w^3 (1 - (N_g/N_r)^2);
    nbar = 2^-13 with P_FKP = 2^13 gives w = 1/2 exactly (eqs. I22def, N0true, Noise0)."""
    ng, nr = 300, 4000
    gal = mockgen.uniform_points(ng, 100.0, 200.0, seed=1)
    ran = mockgen.uniform_points(nr, 100.0, 200.0, seed=2)
    sc = op.scalars(gal, ran, dict(N=8, L=300.0, P_fkp=8192.0))
    nb, w, a = 2.0 ** -13, 0.5, ng / nr
    assert abs(sc["alpha"] - a) < 1e-15
    assert abs(sc["I22"] - ng * nb * w * w) < 1e-15 * ng * nb
    assert abs(sc["N0"] - ng * w * w * (1 + a)) < 1e-12
    assert abs(sc["N0_fkp"] - a * (1 + a) * nr * w * w) < 1e-12
    assert abs(sc["I33"] - ng * nb * nb * w ** 3) < 1e-20
    assert abs(sc["S3"] - ng * w ** 3 * (1 - a * a)) < 1e-12


def test_Lab_trace_and_permutation():
    """L^ab at k=0 (eq. Lab): trace 1 since x^.x^ = 1 (the paper's DR11 values
    sum to 1 within their printed digits, eq. Qat0); permuting the catalog's
    axes permutes L^ab."""
    gold = json.load(open(GOLDEN))["Lab_DR11"]
    assert abs(gold["xx"] + gold["yy"] + gold["zz"] - 1.0) < gold["trace_tolerance"]
    ran = mockgen.uniform_points(5000, 0.0, 100.0, seed=4)
    gal = mockgen.uniform_points(50, 0.0, 100.0, seed=5)
    geom = dict(N=8, L=100.0, observer=(-30.0, 10.0, 200.0))
    lab = op.scalars(gal, ran, geom)["Lab"]
    assert abs(lab[0] + lab[1] + lab[2] - 1.0) < 1e-14
    perm = dict(x=ran["y"], y=ran["z"], z=ran["x"], nbar=ran["nbar"])
    geom2 = dict(N=8, L=100.0, observer=(10.0, 200.0, -30.0))
    lab2 = op.scalars(gal, perm, geom2)["Lab"]
    # new (x,y,z) = old (y,z,x): L'xx = Lyy, L'yy = Lzz, L'zz = Lxx, L'xy = Lyz, L'yz = Lzx, L'zx = Lxy
    assert np.allclose(lab2, [lab[1], lab[2], lab[0], lab[4], lab[5], lab[3]], atol=1e-13)


# ---------------------------------------------------------------------------
# the constants printed in the paper
# ---------------------------------------------------------------------------

def test_paper_constants_and_multiplicities():
    gold = json.load(open(GOLDEN))
    mu = np.linspace(-1, 1, 41)
    L2, L4, L6 = (eval_legendre(l, mu) for l in (2, 4, 6))
    c4 = gold["factorizeL4"]
    assert np.allclose(L4, c4["a"] * L2 ** 2 + c4["b"] * L2 + c4["c"], atol=1e-14)
    c6 = gold["factorizeL6"]
    assert np.allclose(L6, c6["a"] * L2 ** 3 + c6["b"] * L2 ** 2 + c6["c"] * L2 + c6["d"], atol=1e-14)
    # P4fast constants reproduce 9 L4 from L2 (eq. P4fast with F_2 = L_2 F_0)
    p4 = gold["P4fast"]
    assert np.allclose(p4["a"] * L2 ** 2 + p4["b"] * 5 * L2 + p4["c"], 9 * L4, atol=1e-13)
    # every index tuple of the symmetric tensors is covered once, with the
    # paper's multiplicities (eqs. delta2b, delta4b)
    import itertools
    for comps, rank, key in ((op.RANK2, 2, "delta2"), (op.RANK4, 4, "delta4")):
        table = {tuple(sorted(c)): m for c, m in comps}
        assert len(table) == gold[key]["n_components"]
        cnt = {}
        for t in itertools.product(range(3), repeat=rank):
            cnt[tuple(sorted(t))] = cnt.get(tuple(sorted(t)), 0) + 1
        assert cnt == table
    hist = {}
    for _, m in op.RANK4:
        hist[str(m)] = hist.get(str(m), 0) + 1
    assert hist == gold["delta4"]["multiplicity_counts"]


def test_mode_counts_match_lattice():
    N, L = 20, 100.0
    kf = 2 * math.pi / L
    b, wt, _ = op.mode_bins(N, L, 0.5 * kf, kf, 9)
    got = np.bincount(b[b >= 0], weights=wt[b >= 0], minlength=9)
    ref = np.bincount(lattice_bins(full_modes(N), kf, 0.5 * kf, kf, 9) + 1, minlength=10)[1:]
    assert np.array_equal(np.rint(got).astype(int), ref)


def test_mockgen_counts():
    sv = mockgen.survey_small()
    gal, ran = mockgen.catalog(sv, 0)
    assert abs(gal["x"].size - 2e4) < 6 * math.sqrt(2e4) + 0.15 * 2e4
    assert ran["x"].size == 200_000
    r = np.sqrt(ran["x"].astype(float) ** 2 + ran["y"].astype(float) ** 2 + ran["z"].astype(float) ** 2)
    assert r.min() >= 299.9 and r.max() <= 900.1


# ---------------------------------------------------------------------------
# window compensation (reading: divide each mode by the assignment window)
# and the monopole's shot-noise subtraction (eq. P0_impl)
# ---------------------------------------------------------------------------

def kernel_ft(p, q):
    """int B_p(t) e^{-iqt} dt of the order-p B-spline kernel (``_bspline``,
    which test_assignment_is_the_bspline_kernel pins against the oracle's
    gridding), by 24-point Gauss-Legendre quadrature on each polynomial piece
    of the kernel.  The kernel is even, so the transform is real.  No sinc
    formula is used: this derives the window from the kernel itself."""
    x, wq = np.polynomial.legendre.leggauss(24)
    edges = {2: [-1.0, 0.0, 1.0], 3: [-1.5, -0.5, 0.5, 1.5], 4: [-2.0, -1.0, 0.0, 1.0, 2.0]}[p]
    q = np.asarray(q, dtype=np.float64)
    out = np.zeros_like(q)
    for a, b in zip(edges[:-1], edges[1:]):
        t = 0.5 * (b - a) * x + 0.5 * (a + b)
        out += 0.5 * (b - a) * (np.cos(np.multiply.outer(q, t)) * (wq * _bspline(t, p))).sum(-1)
    return out


def kernel_window(N, p):
    """prod_a W_p(2 pi n_a / N) on the rfft half-spectrum [nz][ny][nx]."""
    n1 = np.fft.fftfreq(N, 1.0 / N)
    nh = np.fft.rfftfreq(N, 1.0 / N)
    wx, w1 = kernel_ft(p, 2 * np.pi * nh / N), kernel_ft(p, 2 * np.pi * n1 / N)
    return w1[:, None, None] * w1[None, :, None] * wx[None, None, :]


@pytest.mark.parametrize("p", [2, 3, 4])
@pytest.mark.parametrize("N", [8, 12, 30])
def test_window_is_the_kernel_fourier_transform(p, N):
    """The compensation window of mode n is the product over axes of the
    continuous Fourier transform of the assignment kernel at k_a H = 2 pi
    n_a/N (grid units).  A window in the wrong variable (e.g. sinc of pi^2
    n/N), the wrong power, or one axis left out fails."""
    ref = kernel_window(N, p)
    got = op.window(N, p)
    assert got.shape == ref.shape
    assert np.max(np.abs(got - ref)) < 1e-13


@pytest.mark.parametrize("p", [2, 3])
def test_compensated_fields_of_an_object_on_a_node(p):
    """One object of weight w exactly on a node, compensate on.  The node
    weights of the kernel at integer offsets are B_p(0) and B_p(+-1) (CIC:
    1, 0; TSC: 3/4, 1/8), so the uncompensated F_0(n) = w e^{-ik.x_j} prod_a
    [B_p(0) + 2 B_p(1) cos(2 pi n_a/N)], and every compensated field is that
    divided by the kernel window (quadrature above).  With the observer at
    infinity x^ is the line of sight at every node, so F_2 and F_4 are
    L_l(k^.los) F_0 mode by mode, compensated alike."""
    N, L = 16, 16.0
    los = np.array([0.3, -0.5, 0.81])
    los = los / np.linalg.norm(los)
    g = dict(N=N, L=L, assign=p, origin=(0.0, 0.0, 0.0), observer=None, los=tuple(los), compensate=True)
    j = np.array([5.0, 9.0, 12.0])
    w = 0.7
    F = op.legendre(op.assign(j[None, :], np.array([w]), g), g, lmax=4)
    nx, ny, nz = op.mode_vectors(N)
    b0, b1 = float(_bspline(np.array(0.0), p)), float(_bspline(np.array(1.0), p))
    disc = [b0 + 2 * b1 * np.cos(2 * np.pi * n / N) for n in (nx, ny, nz)]
    ph = np.exp(-2j * np.pi * (nx * j[0] + ny * j[1] + nz * j[2]) / N)
    F0 = w * ph * disc[0] * disc[1] * disc[2] / kernel_window(N, p)
    assert np.max(np.abs(F[0] - F0)) < 1e-12 * np.max(np.abs(F0))
    nn = np.sqrt(nx * nx + ny * ny + nz * nz)
    mu = (nx * los[0] + ny * los[1] + nz * los[2]) / np.where(nn > 0, nn, 1.0)
    m = np.broadcast_to(nn > 0, F0.shape)
    for l in (2, 4):
        ref = eval_legendre(l, mu) * F0
        assert np.max(np.abs(F[l][m] - ref[m])) < 1e-12 * np.max(np.abs(F0)), l


def test_monopole_shot_noise_subtraction_single_galaxy():
    """One galaxy (w = 1) on a node of a 16^3 CIC grid and randoms (w_r =
    128, nbar = 2^-10) on every node, alpha = N_g/N_r = 2^-12, compensation
    off.  The randoms sum to zero at every k != 0 (a full lattice sum of
    e^{-ik.x}), so |F_0|^2 = w^2 = 1 on every mode, and eq. P0_impl gives in
    every bin
        mono_raw = w^2 / I_22 = 1/16,
        P_0 = (w^2 - N_0) / I_22 = -alpha^2 sum_r w_r^2 / I_22 = -1/4,
    with I_22 = alpha sum_r nbar w_r^2 = 16 and N_0 = w^2 + alpha^2 sum_r w_r^2
    = 5 written out here.  Subtracting N_0 before the shell average, or
    dividing it by the mode count, fails in every bin."""
    from tests.test_oracle_bispectrum import single_object_case
    gal, ran, geom, _ = single_object_case()
    nr = ran["x"].size
    alpha = 1.0 / nr
    I22 = alpha * nr * 2.0 ** -10 * 128.0 ** 2
    N0 = 1.0 + alpha ** 2 * nr * 128.0 ** 2
    assert (I22, N0) == (16.0, 5.0)
    kf = 2 * math.pi / geom["L"]
    res = op.power(gal, ran, geom, (0.5 * kf, kf, 7))
    assert np.all(res["nmodes"] > 0)
    assert abs(res["I22"] - I22) < 1e-12 and abs(res["N0"] - N0) < 1e-12
    assert np.max(np.abs(res["mono_raw"] - 1.0 / 16)) < 1e-12
    assert np.max(np.abs(res["P0"] + 0.25)) < 1e-12


# ---------------------------------------------------------------------------
# interlaced grids (Sec. III.A, after eq. mapFFT)
# ---------------------------------------------------------------------------

def alias_sums(p, N, n, u, M=4000):
    """Per axis, A = sum_m W(n + mN) e^{-2 pi i (n + mN) u / N} and B = the
    same sum with (-1)^m, |m| <= M, W(q) = [sin(pi q/N)/(pi q/N)]^p written out
    here (the kernel's Fourier transform; the window test above checks it
    against the kernel by quadrature).  By Poisson summation the grid's DFT of
    one object at u is prod_a A_a, and the second grid's (nodes at i + 1/2),
    referred back to the first grid's origin, is prod_a B_a."""
    m = np.arange(-M, M + 1)
    q = n[:, None] + m[None, :] * N
    x = np.pi * q / N
    with np.errstate(divide="ignore", invalid="ignore"):
        W = np.where(q == 0, 1.0, (np.sin(x) / np.where(q == 0, 1.0, x)) ** p)
    e = W * np.exp(-2j * np.pi * q * u / N)
    return e.sum(1), (e * np.where(m % 2 == 0, 1.0, -1.0)[None, :]).sum(1)


@pytest.mark.parametrize("p", [2, 3, 4])
def test_interlaced_grid_keeps_only_even_alias_images(p):
    """One object at a generic position, compensation off.  The interlaced
    F_0 = [F^(1) + e^{-i pi (n_x+n_y+n_z)/N} F^(2)]/2 must equal
    (prod_a A_a + prod_a B_a)/2 = the sum over alias images m with m_x + m_y +
    m_z even only: the odd images cancel.  A wrong sign or half-cell in the
    phase, or the shift applied to the wrong grid, fails."""
    N, L = 12, 12.0
    u = np.array([3.37, 7.81, 5.06])
    g = dict(N=N, L=L, assign=p, origin=(0.0, 0.0, 0.0), observer=(6.3, -4.0, 2.2), compensate=False,
             interlace=True, periodic=True, alpha_mode=1)
    w = np.array([1.0], np.float32)
    cat = dict(x=np.array([u[0]], np.float32), y=np.array([u[1]], np.float32), z=np.array([u[2]], np.float32),
               w=w, nbar=np.ones(1, np.float32))
    # a zero-weight random (alpha = N_g/N_r = 1): F is the galaxy's grid alone
    ran = dict(x=np.array([1.0], np.float32), y=np.array([1.0], np.float32), z=np.array([1.0], np.float32),
               w=np.array([0.0], np.float32), nbar=np.ones(1, np.float32))
    Fl, _, _ = op.survey_fields(cat, ran, g, lmax=0)
    uu = np.array([float(np.float32(v)) for v in u])
    n1 = np.fft.fftfreq(N, 1.0 / N)
    nh = np.fft.rfftfreq(N, 1.0 / N)
    M = 200000 if p == 2 else 4000  # the CIC image sum converges slowest
    Ax, Bx = alias_sums(p, N, nh, uu[0], M)
    Ay, By = alias_sums(p, N, n1, uu[1], M)
    Az, Bz = alias_sums(p, N, n1, uu[2], M)
    A = Az[:, None, None] * Ay[None, :, None] * Ax[None, None, :]
    B = Bz[:, None, None] * By[None, :, None] * Bx[None, None, :]
    ref = 0.5 * (A + B)
    assert np.max(np.abs(Fl[0] - ref)) < 1e-9
    # and not the plain (non-interlaced) grid, whose images of odd order remain
    g1 = dict(g, interlace=False)
    F1, _, _ = op.survey_fields(cat, ran, g1, lmax=0)
    assert np.max(np.abs(F1[0] - A)) < 1e-9
    assert np.max(np.abs(F1[0] - ref)) > 1e-3


def test_object_moments_are_the_gridded_direct_sum():
    """Per-object line of sight (xhat="object"): the moment fields carry each
    object's own x^, so F_l(k) = sum_j w_j L_l(k^.x^_j) sum_n W(x_n - x_j)
    e^{-ik.x_n} exactly, whatever the positions.  Checked mode by mode against
    that sum done by brute force (CIC weights written out per object, no
    grid, no FFT), for galaxies minus alpha times randoms off the nodes; and
    with everything on nodes the per-object fields equal the node-x^ fields."""
    N, L = 12, 24.0
    H = L / N
    origin = (3.0, -7.0, 11.0)
    obs = (-40.0, 25.0, -18.0)
    g = dict(N=N, L=L, assign=2, origin=origin, observer=obs, compensate=False, xhat="object")
    r = mockgen.rng(21, 3)
    ng, nr = 40, 90

    def cat(n):
        p = np.asarray(origin)[None, :] + H * (1.0 + (N - 3.0) * r.random((n, 3)))
        return {"x": p[:, 0], "y": p[:, 1], "z": p[:, 2], "nbar": 1e-4 * (1.0 + r.random(n)),
                "w": 0.3 + r.random(n)}
    gal, ran = cat(ng), cat(nr)
    Fl, _, sc = op.survey_fields(gal, ran, g, lmax=4)
    alpha = sc["alpha"]
    # brute force
    kf = 2 * math.pi / L
    nx, ny, nz = op.mode_vectors(N)
    hm = np.stack(np.broadcast_arrays(nx, ny, nz), -1).reshape(-1, 3)
    kn = np.linalg.norm(hm, axis=1)
    kh = np.where(kn[:, None] > 0, hm / np.where(kn > 0, kn, 1.0)[:, None], 0.0)
    ref = {l: np.zeros(hm.shape[0], dtype=complex) for l in (0, 2, 4)}
    for c, sgn in ((gal, 1.0), (ran, -alpha)):
        pos = np.stack([c["x"], c["y"], c["z"]], 1)
        xh = (pos - np.asarray(obs)) / np.linalg.norm(pos - np.asarray(obs), axis=1)[:, None]
        u = (pos - np.asarray(origin)) / H
        i0 = np.floor(u)
        d = u - i0
        for j in range(pos.shape[0]):
            mu = kh @ xh[j]
            for ox in (0, 1):
                for oy in (0, 1):
                    for oz in (0, 1):
                        wt = ((d[j, 0] if ox else 1 - d[j, 0]) * (d[j, 1] if oy else 1 - d[j, 1])
                              * (d[j, 2] if oz else 1 - d[j, 2]))
                        node = (i0[j] + (ox, oy, oz)) % N
                        ph = np.exp(-2j * np.pi * (hm @ node) / N)
                        for l in (0, 2, 4):
                            ref[l] += sgn * c["w"][j] * wt * eval_legendre(l, mu) * ph
    nz0 = kn > 0
    for l in (0, 2, 4):
        got = Fl[l].reshape(-1)
        err = np.max(np.abs(got[nz0] - ref[l][nz0]))
        assert err < 1e-12 * np.max(np.abs(ref[0])), (l, err)
    # on the nodes the object's x^ is the node's: the two readings agree
    cg, _ = mockgen.node_points(60, 16, 32.0, origin, seed=5)
    cr, _ = mockgen.node_points(120, 16, 32.0, origin, seed=6)
    gn = dict(g, N=16, L=32.0)
    Fo, _, _ = op.survey_fields(cg, cr, gn, lmax=4)
    Fn, _, _ = op.survey_fields(cg, cr, dict(gn, xhat="node"), lmax=4)
    for l in (0, 2, 4):
        assert np.max(np.abs(Fo[l] - Fn[l])) < 1e-12 * np.max(np.abs(Fn[0]))
    # off the nodes they differ (the variant is not a relabelling)
    Fnode, _, _ = op.survey_fields(gal, ran, dict(g, xhat="node"), lmax=4)
    assert np.max(np.abs(Fnode[2] - Fl[2])) > 1e-4 * np.max(np.abs(Fl[0]))
