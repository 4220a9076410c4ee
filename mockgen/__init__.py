"""Seeded synthetic survey catalogs shaped like the paper's BOSS-like setup.

This module is the one input generator shared by the FP64 oracle (``oracle/``)
and the CUDA path (``paper_1506_02729_gb300``).  It holds none of the
estimator's arithmetic: no gridding kernel, no moment field, no Legendre
recombination, no binning.  It only draws catalogs:

1. a Gaussian field on a generation grid with a truncated power-law P(k),
2. its lognormal transform, Poisson-sampled into objects,
3. linear radial redshift-space displacement s = x + f (Psi . x^) x^ (the
   radial mapping of Sec. I, eq. RSDmap, with u = -Psi),
4. a survey footprint and a radial selection nbar(r) applied in redshift space,
5. uniform randoms in the footprint, distributed like nbar(r).

All draws come from numpy's counter-based Philox generator keyed by
(seed, stream).  Galaxies are shuffled so that catalog order carries no
spatial locality.  Positions and nbar are float32 (the catalog format of the
library's C ABI); both sides read the same float32 values.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

try:  # threaded FFTs when available; plain numpy otherwise
    import scipy.fft as _fft

    def _rfftn(a):
        return _fft.rfftn(a, workers=-1)

    def _irfftn(a, s):
        return _fft.irfftn(a, s=s, workers=-1)
except Exception:  # pragma: no cover
    def _rfftn(a):
        return np.fft.rfftn(a)

    def _irfftn(a, s):
        return np.fft.irfftn(a, s=s)


def rng(seed: int, stream: int) -> np.random.Generator:
    """Philox-keyed generator for (seed, stream)."""
    return np.random.Generator(np.random.Philox(key=[int(seed), int(stream)]))


@dataclasses.dataclass
class Survey:
    """Geometry and selection of one synthetic survey."""
    L: float                       # box side, Mpc/h
    N: int                         # estimator grid side
    assign: int                    # 2 = CIC, 3 = TSC
    origin: tuple                  # box corner (Mpc/h)
    observer: tuple                # observer position (Mpc/h)
    footprint: str                 # "cap" or "octant"
    cap_axis: tuple = (0.0, 0.0, 1.0)
    cap_area_deg2: float = 10000.0
    rmin: float = 0.0
    rmax: float = 0.0
    nbar_kind: str = "uniform"     # "uniform" or "gauss"
    nbar_peak: float = 3e-4
    nbar_r0: float = 0.0
    nbar_sigma: float = 1.0
    n_gal_target: float | None = None  # rescales nbar so that E[N_g] = target
    random_ratio: float = 50.0     # N_r = ratio * E[N_g]
    n_random: int | None = None    # overrides random_ratio when set
    P_fkp: float = 1e4
    pk_amp: float = 2e4            # P(k) = amp (k/k0)^index, (Mpc/h)^3
    pk_k0: float = 0.02
    pk_index: float = -1.5
    growth_f: float = 0.7
    gen_grid: int = 256            # grid the lognormal field is drawn on

    def nbar(self, r):
        r = np.asarray(r, dtype=np.float64)
        if self.nbar_kind == "uniform":
            out = np.full_like(r, self.nbar_peak)
        else:
            out = self.nbar_peak * np.exp(-0.5 * ((r - self.nbar_r0) / self.nbar_sigma) ** 2)
        return out * self._nbar_scale

    # ---- footprint -------------------------------------------------------
    def _cap_cos(self):
        omega = self.cap_area_deg2 * (math.pi / 180.0) ** 2
        return 1.0 - omega / (2.0 * math.pi)

    def solid_angle(self):
        if self.footprint == "cap":
            return 2.0 * math.pi * (1.0 - self._cap_cos())
        return 4.0 * math.pi / 8.0

    def in_footprint(self, d):
        """d: (n,3) unit vectors from the observer."""
        if self.footprint == "cap":
            ax = np.asarray(self.cap_axis, dtype=np.float64)
            ax = ax / np.linalg.norm(ax)
            return d @ ax >= self._cap_cos()
        return np.all(d > 0.0, axis=1)

    def expected_ngal_unscaled(self):
        rr = np.linspace(self.rmin, self.rmax, 8193)
        saved = getattr(self, "_nbar_scale", 1.0)
        self._nbar_scale = 1.0
        f = rr ** 2 * self.nbar(rr)
        self._nbar_scale = saved
        trap = getattr(np, "trapezoid", None) or getattr(np, "trapz")
        return self.solid_angle() * trap(f, rr)

    def __post_init__(self):
        self._nbar_scale = 1.0
        if self.n_gal_target is not None:
            self._nbar_scale = self.n_gal_target / self.expected_ngal_unscaled()

    def expected_ngal(self):
        return self.expected_ngal_unscaled() * self._nbar_scale

    def geometry(self):
        """Plain-dict geometry both sides read (no derived arithmetic)."""
        return dict(L=float(self.L), N=int(self.N), assign=int(self.assign),
                    origin=tuple(float(v) for v in self.origin),
                    observer=tuple(float(v) for v in self.observer),
                    P_fkp=float(self.P_fkp))


# --------------------------------------------------------------------------
# The configurations the library is exercised on (sizes of the paper's BOSS
# setup and a small case for parity runs).
# --------------------------------------------------------------------------

def survey_small(N=64, assign=2):
    """L=1000 box, observer 3 cells inside the corner, octant shell 300<r<900,
    ~2e4 galaxies (uniform nbar rescaled to that count), 2e5 randoms."""
    L = 1000.0
    H = L / N
    return Survey(L=L, N=N, assign=assign, origin=(-3 * H,) * 3, observer=(0.0, 0.0, 0.0),
                  footprint="octant", rmin=300.0, rmax=900.0, nbar_kind="uniform",
                  nbar_peak=3e-4, n_gal_target=2.0e4, n_random=200_000, P_fkp=1e4,
                  gen_grid=64)


def survey_boss(N=512, assign=3, random_ratio=50.0, gen_grid=256):
    """L=3500 box, observer at the centre, 10,000 deg^2 cap about (2,1,1.5),
    1100<r<1700, Gaussian nbar(r) peaking at 4e-4 (sigma 117.4), ~7e5 galaxies,
    50x randoms, FKP P0=1e4."""
    L = 3500.0
    return Survey(L=L, N=N, assign=assign, origin=(0.0, 0.0, 0.0),
                  observer=(1750.0, 1750.0, 1750.0), footprint="cap",
                  cap_axis=(2.0, 1.0, 1.5), cap_area_deg2=10000.0, rmin=1100.0, rmax=1700.0,
                  nbar_kind="gauss", nbar_peak=4e-4, nbar_r0=1400.0, nbar_sigma=117.4,
                  random_ratio=random_ratio, P_fkp=1e4, gen_grid=gen_grid)


# --------------------------------------------------------------------------
# Field and catalog generation
# --------------------------------------------------------------------------

def _kgrid(n, box):
    kf = 2.0 * math.pi / box
    k1 = np.fft.fftfreq(n, d=1.0 / n) * kf
    kx = np.fft.rfftfreq(n, d=1.0 / n) * kf
    return k1, kx


def gaussian_field(sv: Survey, seed: int):
    """Gaussian delta_G and displacement Psi (delta = -div Psi) on the
    generation grid, P(k) truncated at the generation grid's Nyquist k."""
    n = sv.gen_grid
    g = rng(seed, 1).standard_normal((n, n, n))
    G = _rfftn(g)
    del g
    k1, kx = _kgrid(n, sv.L)
    kz = k1[:, None, None]
    ky = k1[None, :, None]
    kxx = kx[None, None, :]
    k2 = kz ** 2 + ky ** 2 + kxx ** 2
    k = np.sqrt(k2)
    knyq = math.pi * n / sv.L
    vcell = (sv.L / n) ** 3
    with np.errstate(divide="ignore", invalid="ignore"):
        pk = sv.pk_amp * (k / sv.pk_k0) ** sv.pk_index
    pk[0, 0, 0] = 0.0
    pk[k > knyq] = 0.0
    G *= np.sqrt(pk / vcell)
    delta = _irfftn(G, (n, n, n))
    psi = []
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = np.where(k2 > 0, 1.0 / k2, 0.0)
    for kc in (kxx, ky, kz):
        psi.append(_irfftn(1j * kc * inv * G, (n, n, n)))
    return delta, psi


def _cic_interp(field, u):
    """Periodic CIC read of field[z][y][x] at grid coordinates u=(ux,uy,uz)."""
    n = field.shape[0]
    i0 = np.floor(u).astype(np.int64)
    d = u - i0
    out = np.zeros(u.shape[0])
    for dz in (0, 1):
        wz = d[:, 2] if dz else 1.0 - d[:, 2]
        iz = (i0[:, 2] + dz) % n
        for dy in (0, 1):
            wy = d[:, 1] if dy else 1.0 - d[:, 1]
            iy = (i0[:, 1] + dy) % n
            for dx in (0, 1):
                wx = d[:, 0] if dx else 1.0 - d[:, 0]
                ix = (i0[:, 0] + dx) % n
                out += wx * wy * wz * field[iz, iy, ix]
    return out


def _unit(v):
    r = np.linalg.norm(v, axis=1)
    return v / r[:, None], r


def galaxies(sv: Survey, seed: int):
    """Lognormal, Poisson-sampled, radially redshift-space-distorted galaxies."""
    n = sv.gen_grid
    H = sv.L / n
    delta, psi = gaussian_field(sv, seed)
    sig2 = float(np.var(delta))
    dln = np.exp(delta - 0.5 * sig2) - 1.0
    del delta
    rr = np.linspace(sv.rmin, sv.rmax, 4097)
    n_env = float(np.max(sv.nbar(rr)))
    r2 = rng(seed, 2)
    counts = r2.poisson(np.clip(n_env * (1.0 + dln) * H ** 3, 0.0, None))
    del dln
    idx = np.nonzero(counts.ravel())[0]
    cnt = counts.ravel()[idx]
    cell = np.repeat(idx, cnt)
    iz, rem = np.divmod(cell, n * n)
    iy, ix = np.divmod(rem, n)
    u = np.stack([ix, iy, iz], axis=1).astype(np.float64) + r2.random((cell.size, 3))
    x = np.asarray(sv.origin)[None, :] + u * H
    obs = np.asarray(sv.observer)[None, :]
    d, r = _unit(x - obs)
    keep = (r > sv.rmin - 40.0) & (r < sv.rmax + 40.0)
    x, u, d, r = x[keep], u[keep], d[keep], r[keep]
    # displacement at the object (real space), radial RSD: s = x + f (Psi.x^) x^
    pr = sum(_cic_interp(psi[a], u - 0.5) * d[:, a] for a in range(3))
    s = x + sv.growth_f * pr[:, None] * d
    ds, rs = _unit(s - obs)
    sel = (rs >= sv.rmin) & (rs < sv.rmax) & sv.in_footprint(ds)
    s, rs = s[sel], rs[sel]
    acc = r2.random(s.shape[0]) < sv.nbar(rs) / n_env
    s, rs = s[acc], rs[acc]
    perm = rng(seed, 3).permutation(s.shape[0])
    s, rs = s[perm], rs[perm]
    return _pack(s, sv.nbar(rs))


def randoms(sv: Survey, seed: int, count: int | None = None):
    """Uniform randoms in the footprint, radially distributed like r^2 nbar(r)."""
    if count is None:
        count = sv.n_random if sv.n_random is not None else int(round(sv.random_ratio * sv.expected_ngal()))
    g = rng(seed, 4)
    rr = np.linspace(sv.rmin, sv.rmax, 16385)
    pdf = rr ** 2 * sv.nbar(rr)
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (pdf[1:] + pdf[:-1]) * np.diff(rr))])
    cdf /= cdf[-1]
    r = np.interp(g.random(count), cdf, rr)
    if sv.footprint == "cap":
        ax = np.asarray(sv.cap_axis, dtype=np.float64)
        ax /= np.linalg.norm(ax)
        tmp = np.array([1.0, 0.0, 0.0]) if abs(ax[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
        e1 = np.cross(ax, tmp)
        e1 /= np.linalg.norm(e1)
        e2 = np.cross(ax, e1)
        c0 = sv._cap_cos()
        ct = c0 + (1.0 - c0) * g.random(count)
        st = np.sqrt(np.clip(1.0 - ct * ct, 0.0, None))
        ph = 2.0 * math.pi * g.random(count)
        d = (ct[:, None] * ax[None, :] + (st * np.cos(ph))[:, None] * e1[None, :]
             + (st * np.sin(ph))[:, None] * e2[None, :])
    else:
        d = np.abs(g.standard_normal((count, 3)))
        d /= np.linalg.norm(d, axis=1)[:, None]
    s = np.asarray(sv.observer)[None, :] + r[:, None] * d
    return _pack(s, sv.nbar(r))


def _pack(s, nbar):
    return dict(x=np.ascontiguousarray(s[:, 0], dtype=np.float32),
                y=np.ascontiguousarray(s[:, 1], dtype=np.float32),
                z=np.ascontiguousarray(s[:, 2], dtype=np.float32),
                nbar=np.ascontiguousarray(nbar, dtype=np.float32))


def catalog(sv: Survey, seed: int, random_seed: int | None = None):
    """(galaxies, randoms) for one mock."""
    return galaxies(sv, seed), randoms(sv, seed if random_seed is None else random_seed)


# --------------------------------------------------------------------------
# Small hand-built inputs for pinned tests
# --------------------------------------------------------------------------

def uniform_points(n, lo, hi, seed, stream=7, nbar=2.0 ** -13):
    """n float32 points uniform in the box [lo, hi)^3, with a constant nbar
    column (default 2^-13, exact in float32)."""
    g = rng(seed, stream)
    s = lo + (hi - lo) * g.random((n, 3))
    return _pack(s, np.full(n, nbar))


def node_points(n, N, L, origin, seed, margin=2, stream=8):
    """n float32 points placed exactly on grid nodes origin + i*L/N (L/N a power
    of two keeps the coordinates exact in float32)."""
    g = rng(seed, stream)
    i = g.integers(margin, N - margin, size=(n, 3))
    s = np.asarray(origin)[None, :] + i * (L / N)
    return _pack(s, np.full(n, 1e-4)), i


def random_phase_field(N, amp_of_n, seed, stream=9):
    """Real field on an N^3 periodic grid whose DFT has |F(n)|^2 = amp_of_n(n)
    exactly and random phases (Hermitian), returned as float64 [z][y][x].
    amp_of_n receives integer mode vectors (nx, ny, nz) broadcast over the
    rfft half-spectrum and returns |F|^2."""
    g = rng(seed, stream)
    n1 = np.fft.fftfreq(N, d=1.0 / N)
    nh = np.fft.rfftfreq(N, d=1.0 / N)
    nz = n1[:, None, None]
    ny = n1[None, :, None]
    nx = nh[None, None, :]
    a2 = np.broadcast_to(amp_of_n(nx, ny, nz), (N, N, N // 2 + 1))
    ph = np.exp(2j * math.pi * g.random((N, N, N // 2 + 1)))
    F = np.sqrt(a2) * ph
    # Hermitian projection by a real-space round trip, then rescale amplitudes
    f = np.fft.irfftn(F, s=(N, N, N))
    F2 = np.fft.rfftn(f)
    mag = np.abs(F2)
    with np.errstate(divide="ignore", invalid="ignore"):
        F2 = np.where(mag > 0, F2 / mag * np.sqrt(a2), 0.0)
    return np.fft.irfftn(F2, s=(N, N, N))
