"""GPU parity of the bispectrum path (C ABI) against the FP64 oracle."""
import math

import numpy as np
import pytest

import mockgen
from oracle import bispectrum as ob
from oracle import power as op
from tests.helpers import to_device

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

B_TOL = 1e-4      # B_l against the FP64 oracle (triangles with N_T >= 100)
SN_TOL = 1e-5     # shot-noise terms (shell means of F_l F^w products)
ALL = 1 | 2 | 4 | 8 | 16 | 32 | 64


def _fkp():
    import paper_1506_02729_gb300 as fkp
    return fkp


def b_errors(got, ref, I33, N3):
    """Max error per multipole relative to max(|B_ref|, |T^0_ref|/(N^3 N_T I_33))
    over triangles with N_T >= 100."""
    m = ref["NT"] >= 100
    mono = np.abs(ref["T0"][m]) / (N3 * ref["NT"][m] * I33)
    out = {}
    for l in (0, 2, 4):
        d = np.maximum(np.abs(ref[f"B{l}"][m]), mono)
        out[l] = float(np.max(np.abs(got[f"B{l}"][m] - ref[f"B{l}"][m]) / d))
    return out


@pytest.fixture(scope="module")
def small_b():
    sv = mockgen.survey_small(N=64, assign=3)
    gal, ran = mockgen.catalog(sv, 2)
    geom = sv.geometry()
    kf = 2 * math.pi / sv.L
    bs = (3, 3, 3, 6)
    ref = ob.bispectrum(gal, ran, geom, bs)
    return sv, gal, ran, geom, bs, ref, kf


@pytest.mark.parametrize("contraction", [0, 2], ids=["fp32", "bf16x6_tcgen05"])
def test_small_bispectrum_matches_oracle(small_b, contraction):
    fkp = _fkp()
    sv, gal, ran, geom, bs, ref, kf = small_b
    plan = fkp.Plan(geom, (0.5 * kf, kf, 32), bshells=bs, want=ALL)
    p, b = plan.bispectrum(to_device(gal), to_device(ran), contraction=contraction)
    assert plan.ntri == len(ref["tri"])
    assert np.array_equal(b["tri"].astype(int), np.asarray(ref["tri"]))
    assert np.array_equal(b["NT"], ref["NT"])
    assert np.array_equal(b["centre_closed"].astype(bool), ref["centre_closed"])
    N3 = float(sv.N) ** 3
    err = b_errors(b, ref, ref["I33"], N3)
    assert max(err.values()) < B_TOL, err
    for l in (0, 2, 4):
        d = np.maximum(np.abs(ref[f"N{l}"]), np.abs(ref["N0"]))
        assert np.max(np.abs(b[f"N{l}"] - ref[f"N{l}"]) / d) < SN_TOL, l
    assert abs(b["I33"] / ref["I33"] - 1) < 1e-10


def test_3way_split_matches_fp32_contraction(small_b):
    """The 3-way split (6 products) on the tensor cores against the FP32
    CUDA-core contraction on the same device shell fields: this isolates the
    contraction's error from the FFTs'.  Same denominators and triangle set
    (N_T >= 100) as the oracle comparison."""
    fkp = _fkp()
    sv, gal, ran, geom, bs, ref, kf = small_b
    plan = fkp.Plan(geom, (0.5 * kf, kf, 32), bshells=bs, want=ALL)
    dg, dr = to_device(gal), to_device(ran)
    b32 = plan.bispectrum(dg, dr, contraction=0)[1]
    b6 = plan.bispectrum(dg, dr, contraction=2)[1]
    err = b_errors(b6, b32, float(b32["I33"]), float(sv.N) ** 3)
    assert max(err.values()) < B_TOL, err


def _split_diff_units(small_b, mode_a, mode_b):
    """Largest |T_a - T_b| over the triangle sums (N_T >= 100, l = 0, 2, 4) of
    two contraction modes on the same device fields, in units of 2^-17
    sqrt(sum_x t^2), t = F_a^(l) F_b^(0) F_c^(0) (shell fields from the
    oracle)."""
    fkp = _fkp()
    sv, gal, ran, geom, bs, ref, kf = small_b
    plan = fkp.Plan(geom, (0.5 * kf, kf, 32), bshells=bs, want=ALL)
    dg, dr = to_device(gal), to_device(ran)
    ba = plan.bispectrum(dg, dr, contraction=mode_a)[1]
    bb = plan.bispectrum(dg, dr, contraction=mode_b)[1]
    F = op.fkp_grids(gal, ran, geom)[0]
    Fl = op.legendre(F, geom, lmax=4)
    sidx, _ = ob.shell_index(sv.N, bs)
    I = {(l, s): ob.shell_field(Fl[l], sidx, s, sv.N) for l in (0, 2, 4) for s in range(bs[3])}
    worst = 0.0
    for t, (a, b, c) in enumerate(ref["tri"]):
        if ref["NT"][t] < 100:
            continue
        for l in (0, 2, 4):
            q = math.sqrt(float(np.sum((I[(l, a)] * I[(0, b)] * I[(0, c)]) ** 2)))
            worst = max(worst, abs(ba[f"T{l}"][t] - bb[f"T{l}"][t]) / (2.0 ** -17 * q))
    return worst


def test_hi_lo_split_follows_its_error_model(small_b):
    """The 2-way split (3 products) drops lo*lo and the rounding of lo, each
    ~2^-18 of a product, with random sign: over the N^3 points the error of a
    triangle sum random-walks to ~2^-17 sqrt(sum_x t^2), t = F_a^(l) F_b^(0)
    F_c^(0) (measured spread: median 0.4-0.7, max 3.6 of those units with
    256-point tensor-memory runs).  The FP32 rounding of the tensor-memory
    accumulation (runs of 96 accumulating MMAs: 512 points for the 2-way
    split, 256 for the 3-way one) adds to the difference of the two splits
    (max 6.3 units on this case with 1,024-point runs, 1.6 with these runs).
    Against the 3-way split on the same
    fields, every triangle sum (N_T >= 100, l = 0, 2, 4) stays within 8 units;
    the shell fields for sum_x t^2 come from the oracle."""
    w = _split_diff_units(small_b, 1, 2)
    assert w < 8.0, w


def test_counts_match_oracle_convolution():
    """Exact integer N_T from the GPU enumeration against the oracle's rounded
    FP64 convolution, on a grid and shell set with over 200 triangles."""
    fkp = _fkp()
    N = 96
    bs = (3, 3, 3, 10)
    gal = mockgen.uniform_points(200, 400.0, 600.0, seed=3)
    ran = mockgen.uniform_points(2000, 400.0, 600.0, seed=4)
    geom = dict(L=1000.0, N=N, assign=2, origin=(0.0, 0.0, 0.0), observer=(500.0, 500.0, -2000.0))
    plan = fkp.Plan(geom, (0.0, 0.01, 10), bshells=bs, want=FKP_B0())
    _, b = plan.bispectrum(to_device(gal), to_device(ran))
    counter = ob.Counter(N, bs)
    for t, (a, bb, c) in enumerate(b["tri"].astype(int)):
        assert b["NT"][t] == counter.count(a, bb, c), (a, bb, c)
    # every triple with a positive count is listed
    listed = {tuple(x) for x in b["tri"].astype(int)}
    for tri in ob.triangle_list(bs[3]):
        if tri not in listed:
            assert counter.count(*tri) == 0, tri


def FKP_B0():
    return 1 | 16


def test_aliasing_shells_are_rejected():
    fkp = _fkp()
    with pytest.raises(fkp.FKPError) as e:
        fkp.Plan(dict(L=1000.0, N=48), (0.0, 0.01, 4), bshells=(3, 3, 3, 6), want=FKP_B0())
    assert e.value.code == -2


@pytest.mark.parametrize("contraction", [0, 1, 2], ids=["fp32", "bf16x3_tcgen05", "bf16x6_tcgen05"])
def test_single_object_shot_noise_identity(contraction):
    """One galaxy on a node and randoms on every node (the oracle's pinned
    case): every triangle's B_0 = -2 alpha^2/nbar^2 = -0.125 with N_0 = 0.625
    and B-hat_0 = 0.5, through each contraction."""
    from tests.test_oracle_bispectrum import single_object_case
    fkp = _fkp()
    gal, ran, geom, bs = single_object_case()
    ref = ob.bispectrum(gal, ran, geom, bs, ells=(0,))
    plan = fkp.Plan(geom, (0.0, 2 * math.pi / geom["L"], 8), bshells=bs, want=FKP_B0())
    _, b = plan.bispectrum(to_device(gal), to_device(ran), contraction=contraction)
    assert np.array_equal(b["tri"].astype(int), np.asarray(ref["tri"]))
    assert np.array_equal(b["NT"], ref["NT"])
    assert abs(b["I33"] - 2.0) < 1e-12
    assert np.max(np.abs(b["N0"] - 0.625)) < 1e-5
    assert np.max(np.abs(b["B0"] + 0.125)) < 1e-5


def test_cached_randoms_bispectrum(small_b):
    """B_l with the plan's cached random grids (R and R^w without alpha)
    equals B_l with the random catalog passed in, and the oracle."""
    fkp = _fkp()
    sv, gal, ran, geom, bs, ref, kf = small_b
    plan = fkp.Plan(geom, (0.5 * kf, kf, 32), bshells=bs, want=ALL)
    dg, dr = to_device(gal), to_device(ran)
    plan.cache_randoms(dr)
    _, full = plan.bispectrum(dg, dr, contraction=0)
    _, cached = plan.bispectrum(dg, None, contraction=0)
    assert np.array_equal(cached["NT"], full["NT"])
    assert cached["I33"] == full["I33"] and cached["S3"] == full["S3"]
    N3 = float(sv.N) ** 3
    # each random term is rounded to the grid's fixed point after, not before,
    # the alpha product: relative input differences ~1e-8, which the B_4 sums'
    # cancellations enlarge
    assert max(b_errors(cached, full, full["I33"], N3).values()) < 5e-5
    assert max(b_errors(cached, ref, ref["I33"], N3).values()) < B_TOL


def test_interlaced_pcs_bispectrum_matches_oracle():
    """B_0,2,4 with PCS assignment on an interlaced pair of grids (the
    paper's setup, Sec. III.A and III.C) against the FP64 oracle."""
    fkp = _fkp()
    sv = mockgen.survey_small(N=64, assign=4)
    gal, ran = mockgen.catalog(sv, 3)
    geom = dict(sv.geometry(), interlace=True, periodic=True)
    kf = 2 * math.pi / sv.L
    bs = (3, 3, 3, 6)
    ref = ob.bispectrum(gal, ran, geom, bs)
    plan = fkp.Plan(geom, (0.5 * kf, kf, 32), bshells=bs, want=ALL)
    for c in (0, 2):
        _, b = plan.bispectrum(to_device(gal), to_device(ran), contraction=c)
        assert np.array_equal(b["NT"], ref["NT"])
        assert max(b_errors(b, ref, ref["I33"], 64.0 ** 3).values()) < B_TOL
        for l in (0, 2, 4):
            d = np.maximum(np.abs(ref[f"N{l}"]), np.abs(ref["N0"]))
            assert np.max(np.abs(b[f"N{l}"] - ref[f"N{l}"]) / d) < SN_TOL, l


@pytest.mark.parametrize("contraction", [0, 2], ids=["fp32", "bf16x6_tcgen05"])
def test_split_hexadecapole_bispectrum_matches_oracle(small_b, contraction):
    """B_4b of eq. Bhexa2 (delta_2 on the two larger sides: T22 = sum_x
    F_a^(2) F_b^(2) F_c^(0), extra columns of the contraction) against the
    FP64 oracle, graded by |T0|/(N^3 N_T I_33) like the other multipoles."""
    fkp = _fkp()
    sv, gal, ran, geom, bs, _, kf = small_b
    ref = ob.bispectrum(gal, ran, geom, bs, zero_area=True)
    plan = fkp.Plan(geom, (0.5 * kf, kf, 32), bshells=bs, want=ALL | fkp.FKP_B4B)
    _, b = plan.bispectrum(to_device(gal), to_device(ran), contraction=contraction)
    assert np.array_equal(b["NT"], ref["NT"])
    m = ref["NT"] >= 100
    N3 = float(sv.N) ** 3
    den = np.maximum(np.abs(ref["B4b"][m]), np.abs(ref["T0"][m]) / (N3 * ref["NT"][m] * ref["I33"]))
    assert np.max(np.abs(b["B4b"][m] - ref["B4b"][m]) / den) < B_TOL
    assert max(b_errors(b, ref, ref["I33"], N3).values()) < B_TOL


def test_bispectrum_graph_replay_equals_plain_launches(small_b):
    """The bispectrum path is captured into a CUDA graph on the second call
    with the same device catalogs and contraction and replayed afterwards;
    another contraction mode runs plain launches.  Replays equal plain
    launches bit for bit."""
    fkp = _fkp()
    sv, gal, ran, geom, bs, ref, kf = small_b
    plan = fkp.Plan(geom, (0.5 * kf, kf, 32), bshells=bs, want=ALL)
    dg, dr = to_device(gal), to_device(ran)
    runs = [plan.bispectrum(dg, dr, contraction=c) for c in (2, 2, 2, 0, 2)]
    assert [p["graph"] for p, _ in runs] == [0, 1, 1, 0, 1]
    plan.set_graphs(False)
    p0, b0 = plan.bispectrum(dg, dr, contraction=2)
    assert p0["graph"] == 0
    for p, b in (runs[0], runs[1], runs[2], runs[4]):
        for k in ("B0", "B2", "B4", "N0", "T0"):
            assert np.array_equal(b[k], b0[k], equal_nan=True), k
        assert np.array_equal(p["P0"], p0["P0"], equal_nan=True)
    assert max(b_errors(b0, ref, ref["I33"], float(sv.N) ** 3).values()) < B_TOL
