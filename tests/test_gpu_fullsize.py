"""GPU parity at the workloads' full sizes (slow): every P_l bin of the
BOSS-like survey on the 256^3 and 384^3 grids of the mixed-grid mocks and on
the 360^3 bispectrum grid, B_0 with 27 shells to k = 0.15 on 256^3 and 384^3,
B_0,2,4 with 37 shells to k = 0.2 on 360^3 on a stratified sample of at least
200 triangles (every largest-side shell a; equilateral, squeezed and folded
shapes), and the whole exact N_T list against the stored counts of the FP64
oracle's convolution counter (tests/golden/triangle_counts_360_s37.txt,
written by tests/golden/make_triangle_counts.py)."""
import os

import numpy as np
import pytest

import mockgen
from oracle import bispectrum as ob
from oracle import power as op
from tests.helpers import P_TOL, p_errors, to_device
from tests.test_gpu_bispectrum import B_TOL, b_errors

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")

GOLD = os.path.join(os.path.dirname(__file__), "golden", "triangle_counts_360_s37.txt")
BINS = (0.0, 0.005, 60)


def stored_counts(S):
    """(a, b, c) -> N_T for the triangles of the first S shells (3 k_f wide,
    centres 3(s+1) k_f): with 3 n_max < N the counts do not depend on N."""
    out = {}
    for line in open(GOLD):
        if line.startswith("#"):
            continue
        a, b, c, n = (int(v) for v in line.split())
        if a < S:
            out[(a, b, c)] = n
    return out


def stratified_sample(counts, per_a, extra, seed):
    """Per largest-side shell a: the equilateral triangle, the most squeezed
    (smallest c), a folded one (c_b + c_c = c_a, i.e. b + c = a - 1, b as
    close to c as possible), the one with the most closed triangles, and
    `per_a - 4` random others; then `extra` random triangles."""
    g = np.random.default_rng(seed)
    keys = sorted(counts)
    by_a = {}
    for t in keys:
        by_a.setdefault(t[0], []).append(t)
    pick = set()
    for a, ts in by_a.items():
        if (a, a, a) in counts:
            pick.add((a, a, a))
        pick.add(min(ts, key=lambda t: (t[2], -t[1])))
        folded = [t for t in ts if t[1] + t[2] == a - 1]
        if folded:
            pick.add(min(folded, key=lambda t: t[1] - t[2]))
        pick.add(max(ts, key=lambda t: counts[t]))
        rest = [t for t in ts if t not in pick]
        for i in g.permutation(len(rest))[:max(0, per_a - 4)]:
            pick.add(rest[i])
    rest = [t for t in keys if t not in pick]
    for i in g.permutation(len(rest))[:extra]:
        pick.add(rest[i])
    return sorted(pick)


def _mock(N, random_ratio, seed):
    sv = mockgen.survey_boss(N=N, random_ratio=random_ratio)
    gal, ran = mockgen.catalog(sv, seed)
    return sv, gal, ran


def _check_triangle_list(b, counts):
    tri = [tuple(t) for t in b["tri"].astype(int)]
    assert tri == sorted(counts), "triangle list differs from the stored exact counts"
    assert np.array_equal(b["NT"], np.array([counts[t] for t in tri], dtype=np.int64))
    return tri


@pytest.mark.parametrize("N", [256, 384])
def test_mixed_grid_power_and_b0_match_oracle(N):
    """A mixed-grid mock (BOSS-like, 30x randoms) on 256^3 or 384^3: P_0,2,4,
    P_4b in all 60 bins (nmodes bit-exact), the 27-shell triangle list and N_T
    exact, B_0 on a stratified sample against the FP64 oracle."""
    import paper_1506_02729_gb300 as fkp
    sv, gal, ran = _mock(N, 30.0, 40 + N)
    geom = sv.geometry()
    bs = (3, 3, 3, 27)
    plan = fkp.Plan(geom, BINS, bshells=bs, want=fkp.FKP_P0 | fkp.FKP_P2 | fkp.FKP_P4 | fkp.FKP_P4B | fkp.FKP_B0)
    dg, dr = to_device(gal), to_device(ran)
    p, b = plan.bispectrum(dg, dr, contraction=fkp.FKP_CONTRACT_BF16X6)
    _, bf = plan.bispectrum(dg, dr, contraction=fkp.FKP_CONTRACT_FP32)
    counts = stored_counts(27)
    tri = _check_triangle_list(b, counts)
    # P_l through the full oracle
    F, Fw, sc = op.fkp_grids(gal, ran, geom, with_w2=True)
    Fl = op.legendre(F, geom, lmax=4)
    ref = op.bin_power(Fl, geom, BINS, sc["I22"], sc["N0"])
    assert np.array_equal(p["nmodes"], ref["nmodes"])
    err = p_errors(p, ref)
    assert max(err.values()) < P_TOL, err
    # B_0 on a sample
    sample = stratified_sample(counts, 2, 20, seed=N)
    Fl0 = {0: Fl[0]}
    del Fl
    Fwl0 = {0: op.legendre(Fw, geom, lmax=0)[0]}
    rb = ob.bispectrum_from_fields(Fl0, Fwl0, sc, N, bs, ells=(0,), tris=sample, counts=counts, cache_fields=12)
    idx = [tri.index(t) for t in sample]
    m = rb["NT"] >= 100
    den = np.maximum(np.abs(rb["B0"][m]), np.abs(rb["T0"][m]) / (float(N) ** 3 * rb["NT"][m] * rb["I33"]))
    for mode, bb in (("bf16x6", b), ("fp32", bf)):
        err = float(np.max(np.abs(bb["B0"][idx][m] - rb["B0"][m]) / den))
        assert err < B_TOL, (mode, err)


def test_bispectrum_360_stratified_triangles_and_exact_counts():
    """The bispectrum workload (BOSS-like catalog, 360^3 TSC, 37 shells to
    k = 0.2): the whole triangle list with exact N_T, P_l in all bins, and
    B_0,2,4 of every contraction mode on >= 200 stratified triangles against
    the FP64 oracle."""
    import paper_1506_02729_gb300 as fkp
    sv, gal, ran = _mock(360, 50.0, 0)
    geom = sv.geometry()
    bs = (3, 3, 3, 37)
    plan = fkp.Plan(geom, BINS, bshells=bs, want=127)
    dg, dr = to_device(gal), to_device(ran)
    runs = [plan.bispectrum(dg, dr, contraction=c) for c in (0, 1, 2)]
    counts = stored_counts(37)
    tri = _check_triangle_list(runs[0][1], counts)
    F, Fw, sc = op.fkp_grids(gal, ran, geom, with_w2=True)
    Fl = op.legendre(F, geom, lmax=4)
    ref = op.bin_power(Fl, geom, BINS, sc["I22"], sc["N0"])
    for p, _ in runs:
        assert np.array_equal(p["nmodes"], ref["nmodes"])
        err = p_errors(p, ref)
        assert max(err.values()) < P_TOL, err
    sample = stratified_sample(counts, 6, 60, seed=360)
    assert len(sample) >= 200 and len({t[0] for t in sample}) == 37
    Fwl = op.legendre(Fw, geom, lmax=4)
    del F, Fw
    rb = ob.bispectrum_from_fields(Fl, Fwl, sc, 360, bs, ells=(0, 2, 4), tris=sample, counts=counts,
                                   cache_fields=16)
    idx = [tri.index(t) for t in sample]
    for mode, (_, bb) in zip(("fp32", "bf16x3", "bf16x6"), runs):
        got = {k: bb[k][idx] for k in ("B0", "B2", "B4")}
        err = b_errors(got, rb, rb["I33"], 360.0 ** 3)
        print(f"B errors against the oracle, {mode}: " + ", ".join(f"B{l} {v:.2e}" for l, v in err.items()))
        assert max(err.values()) < B_TOL, (mode, err)
