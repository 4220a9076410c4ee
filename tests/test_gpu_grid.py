"""Element-wise parity of the gridded fields F and F^w (eq. mapFFT; the F^w of
eq. SNbisp2) with the FP64 oracle's mass assignment, through fkp_grid."""
import math

import numpy as np
import pytest

import mockgen
from oracle import power as op

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

UNIT = 2.0 ** -40   # fkp_grid's fixed-point unit
B_ALL = 1 | 2 | 4 | 8 | 16 | 32 | 64


def _fkp():
    import paper_1506_02729_gb300 as fkp
    return fkp


def _dev(c):
    return {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in c.items()}


def _abs_fields(gal, ran, geom, alpha):
    """sum_g |w| W + alpha sum_r |w| W and the same with w^2: the scale of the
    rounding of each cell (FP32 positions and tap weights on the GPU)."""
    g = op._geom(geom)
    pg, wg, _ = op._cat(gal, g["P_fkp"])
    pr, wr, _ = op._cat(ran, g["P_fkp"])
    A = op.assign(pg, np.abs(wg), g) + abs(alpha) * op.assign(pr, np.abs(wr), g)
    Aw = op.assign(pg, wg * wg, g) + alpha * alpha * op.assign(pr, wr * wr, g)
    return A, Aw


def _plan(geom, bisp=True):
    """A plan with the bispectrum outputs (F and F^w gridded together) or,
    bisp=False, a power-spectrum plan (F alone: the accumulation kernel's
    single-grid form)."""
    fkp = _fkp()
    kf = 2 * math.pi / geom["L"]
    if not bisp:
        return fkp.Plan(geom, (0.5 * kf, kf, 8))
    return fkp.Plan(geom, (0.5 * kf, kf, 8), bshells=(3, 3, 3, 4), want=B_ALL)


def _exact_setup(assign, seed=4, interlace=False):
    """The small survey's catalogs on a box whose cell is 16 (L = 1024, N =
    64, origin -48), positions rounded to multiples of 2^-10: then the GPU's
    FP32 u = (x - origin)/H is exact, and only the tap weights' and values'
    FP32 roundings (a few 2^-24 of each term) separate it from the oracle."""
    sv = mockgen.survey_small(N=64, assign=assign)
    gal, ran = mockgen.catalog(sv, seed)
    for c in (gal, ran):
        for k in ("x", "y", "z"):
            c[k] = (np.round(c[k].astype(np.float64) * 1024.0) / 1024.0).astype(np.float32)
    geom = dict(sv.geometry(), L=1024.0, origin=(-48.0, -48.0, -48.0), periodic=True, interlace=interlace)
    return sv, gal, ran, geom


REL = 1e-6   # of each cell's sum of |terms|: a few FP32 roundings per term


@pytest.mark.parametrize("assign,interlace", [(2, False), (3, False), (4, False), (4, True)],
                         ids=["cic", "tsc", "pcs", "pcs_second_grid"])
def test_grid_matches_oracle_assignment(assign, interlace):
    """F and F^w cell by cell against the oracle's assignment (CIC, TSC, PCS;
    for the interlaced plan, its second grid against the oracle's grid with
    the origin moved by half a cell)."""
    sv, gal, ran, geom = _exact_setup(assign, interlace=interlace)
    plan = _plan(geom)
    F, Fw = plan.grid(_dev(gal), _dev(ran), which=1 if interlace else 0, with_w=True)
    g_or = op.shifted_geometry(dict(geom, interlace=False)) if interlace else dict(geom, interlace=False)
    Fo, Fwo, sc = op.fkp_grids(gal, ran, g_or, with_w2=True)
    A, Aw = _abs_fields(gal, ran, g_or, sc["alpha"])
    got, gotw = F * UNIT, Fw * UNIT
    assert np.all(np.abs(got - Fo) <= REL * A + 1e-11), float(np.max(np.abs(got - Fo) - REL * A))
    assert np.all(np.abs(gotw - Fwo) <= REL * Aw + 1e-11), float(np.max(np.abs(gotw - Fwo) - REL * Aw))
    # cells no tap reaches are exactly zero
    assert np.all(F[A == 0] == 0) and np.all(Fw[Aw == 0] == 0)
    assert np.count_nonzero(A) > 50000


@pytest.mark.parametrize("assign", [2, 3], ids=["cic", "tsc"])
def test_power_plan_grid_matches_oracle(assign):
    """A power-spectrum plan grids F alone (the accumulation kernel's
    single-grid form, the one the power-spectrum path times): cell by cell
    against the oracle's assignment, and bit for bit the F of a bispectrum
    plan, which grids F and F^w together."""
    sv, gal, ran, geom = _exact_setup(assign)
    F = _plan(geom, bisp=False).grid(_dev(gal), _dev(ran))
    Fb, _ = _plan(geom).grid(_dev(gal), _dev(ran), with_w=True)
    assert np.array_equal(F, Fb)
    Fo, _, sc = op.fkp_grids(gal, ran, geom, with_w2=False)
    A, _ = _abs_fields(gal, ran, geom, sc["alpha"])
    assert np.all(np.abs(F * UNIT - Fo) <= REL * A + 1e-11), float(np.max(np.abs(F * UNIT - Fo) - REL * A))
    assert np.all(F[A == 0] == 0)
    assert np.count_nonzero(A) > 50000


@pytest.mark.parametrize("bisp", [True, False], ids=["F_and_Fw", "F_alone"])
def test_grid_does_not_depend_on_object_order_or_accumulation_form(bisp):
    """The gridding adds each tap's rounded value as an integer: as two 32-bit
    words, or as one 64-bit word for a work item whose sum of |w| passes 1000.
    Galaxy weights k/1024 (k uniform in 0..250, mean 0.122) and randoms of
    weight 1 (alpha near 0.122) put the tiles' full work items of 8160
    objects on both sides of that bound (29 of them here), and which objects
    share an item follows the objects' order.  Both forms and every order
    give the same grid, bit for bit (the weights keep W_g and W_r, hence
    alpha, exact whatever the order of their sums); the oracle agrees within
    the rounding bound."""
    # two random catalogs (200000 objects, thousands per tile), one as the
    # galaxies
    sv, _, gal, geom = _exact_setup(3, seed=11)
    _, _, ran, _ = _exact_setup(3, seed=12)
    r = np.random.default_rng(1506)
    gal["w"] = (r.integers(0, 251, len(gal["x"])) / 1024.0).astype(np.float32)
    ran["w"] = np.ones(len(ran["x"]), dtype=np.float32)
    plan = _plan(geom, bisp=bisp)

    def grid(g, rr):
        return plan.grid(g, rr, with_w=True) if bisp else (plan.grid(g, rr), None)

    F1, Fw1 = grid(_dev(gal), _dev(ran))
    pg, pr = r.permutation(len(gal["x"])), r.permutation(len(ran["x"]))
    gal2 = {k: v[pg] for k, v in gal.items()}
    ran2 = {k: v[pr] for k, v in ran.items()}
    F2, Fw2 = grid(_dev(gal2), _dev(ran2))
    F3, Fw3 = grid(gal2, ran2)  # host catalogs
    assert np.array_equal(F1, F2) and np.array_equal(F1, F3)
    Fo, Fwo, sc = op.fkp_grids(gal, ran, geom, with_w2=True)
    A, Aw = _abs_fields(gal, ran, geom, sc["alpha"])
    assert np.all(np.abs(F1 * UNIT - Fo) <= REL * A + 1e-11)
    if bisp:
        assert np.array_equal(Fw1, Fw2) and np.array_equal(Fw1, Fw3)
        assert np.all(np.abs(Fw1 * UNIT - Fwo) <= REL * Aw + 1e-11)


def test_grid_rejects_bad_requests():
    fkp = _fkp()
    sv = mockgen.survey_small(N=64, assign=3)
    gal, ran = mockgen.catalog(sv, 4)
    kf = 2 * math.pi / sv.L
    p_only = fkp.Plan(dict(sv.geometry(), periodic=True), (0.5 * kf, kf, 8))
    with pytest.raises(fkp.FKPError):
        p_only.grid(_dev(gal), _dev(ran), with_w=True)   # no F^w grid without bispectrum outputs
    with pytest.raises(fkp.FKPError):
        p_only.grid(_dev(gal), _dev(ran), which=1)       # no second grid without interlacing
    F = p_only.grid(_dev(gal), _dev(ran))
    assert F.shape == (64, 64, 64) and F.dtype == np.int64
