"""GPU: several mocks in one fused call (fkp_power_batch) against one call per
mock and against the FP64 oracle."""
import math

import numpy as np
import pytest

import mockgen
from oracle import power as op
from tests.helpers import P_TOL, p_errors, to_device

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _fkp():
    import paper_1506_02729_gb300 as fkp
    return fkp


def _bins(L):
    kf = 2 * math.pi / L
    return (0.5 * kf, kf, 32)


def _subsample(cat, frac, seed):
    """A random subset of a catalog (uneven mock sizes)."""
    n = len(cat["x"])
    keep = np.sort(np.random.default_rng(seed).choice(n, max(1, int(n * frac)), replace=False))
    return {k: (None if v is None else np.asarray(v)[keep]) for k, v in cat.items()}


@pytest.fixture(scope="module")
def mocks():
    """Three mocks of the 64^3 survey: different seeds, galaxy and random
    counts differing by up to 4x."""
    sv = mockgen.survey_small()
    out = []
    for seed, fg, fr in ((0, 1.0, 1.0), (1, 0.35, 0.6), (2, 0.7, 0.25)):
        gal, ran = mockgen.catalog(sv, seed)
        out.append((_subsample(gal, fg, 10 + seed), _subsample(ran, fr, 20 + seed)))
    return sv, out


def _same(a, b):
    """Batch against single call: identical grid, scalars and bins, bit for bit
    (integer gridding, order-independent bin sums)."""
    assert np.array_equal(a["nmodes"], b["nmodes"])
    for k in ("alpha", "I22", "I33", "N0", "W_g", "W_r", "n_gal", "n_ran"):
        assert a[k] == b[k], k
    for k in ("P0", "P2", "P4", "P4b", "k_eff", "mono_raw"):
        assert np.array_equal(a[k], b[k], equal_nan=True), k


def test_batch_equals_single_calls(mocks):
    fkp = _fkp()
    sv, ms = mocks
    plan = fkp.Plan(sv.geometry(), _bins(sv.L))
    dev = [(to_device(g), to_device(r)) for g, r in ms]
    single = [plan.power(g, r) for g, r in dev]
    batch = plan.power_batch([g for g, _ in dev], [r for _, r in dev])
    assert len(batch) == 3
    assert len({b["n_gal"] for b in batch}) == 3
    for a, b in zip(batch, single):
        _same(a, b)
    # a mock's values do not depend on its batch-mates or its position
    alone = plan.power_batch([dev[2][0]], [dev[2][1]])
    _same(alone[0], single[2])
    rev = plan.power_batch([g for g, _ in dev[::-1]], [r for _, r in dev[::-1]])
    for a, b in zip(rev, single[::-1]):
        _same(a, b)


def test_batch_matches_oracle(mocks):
    """The sparsest mock of a batch against the FP64 oracle."""
    fkp = _fkp()
    sv, ms = mocks
    geom, bins = sv.geometry(), _bins(sv.L)
    gal, ran = ms[1]
    ref = op.power(gal, ran, geom, bins)
    plan = fkp.Plan(geom, bins)
    got = plan.power_batch([to_device(g) for g, _ in ms], [to_device(r) for _, r in ms])[1]
    assert np.array_equal(got["nmodes"], ref["nmodes"])
    err = p_errors(got, ref)
    assert max(err.values()) < P_TOL, err
    for k in ("alpha", "I22", "N0"):
        assert abs(got[k] / ref[k] - 1) < 1e-10, k


def test_batch_ragged_grid_host_catalogs_and_growth(mocks):
    """A 60^3 periodic grid (generic-N kernels), host and device catalogs mixed,
    and a batch larger than the plan's first one (the workspace grows)."""
    fkp = _fkp()
    sv0, ms = mocks
    sv = mockgen.survey_small(N=60, assign=3)
    geom = dict(sv.geometry(), periodic=True)
    kf = 2 * math.pi / sv.L
    plan = fkp.Plan(geom, (0.0, 1.7 * kf, 14))
    cats = [(ms[0][0], ms[0][1]), (to_device(ms[1][0]), to_device(ms[1][1])), (ms[2][0], to_device(ms[2][1]))]
    single = [plan.power(g, r) for g, r in cats]
    two = plan.power_batch([c[0] for c in cats[:2]], [c[1] for c in cats[:2]])
    three = plan.power_batch([c[0] for c in cats], [c[1] for c in cats])
    for a, b in zip(two, single[:2]):
        _same(a, b)
    for a, b in zip(three, single):
        _same(a, b)


def test_batch_rejects_an_empty_random_catalog(mocks):
    fkp = _fkp()
    sv, ms = mocks
    plan = fkp.Plan(sv.geometry(), _bins(sv.L))
    empty = {k: (None if v is None else np.asarray(v)[:0]) for k, v in ms[0][1].items()}
    with pytest.raises(fkp.FKPError) as e:
        plan.power_batch([ms[0][0], ms[1][0]], [ms[0][1], empty])
    assert e.value.code == -1
    # the plan stays usable
    _same(plan.power_batch([ms[0][0]], [ms[0][1]])[0], plan.power(ms[0][0], ms[0][1]))
