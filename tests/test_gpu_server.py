"""The continuous-batching server: results in a mix of concurrent requests of
different sizes and grids equal the standalone results; admission by device
footprint; rejection, timeout and failure paths (all host-side)."""
import math

import numpy as np
import pytest

import mockgen
from tests.helpers import P_TOL, p_errors, to_device

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

B_TOL = 1e-4


def _fkp():
    import paper_1506_02729_gb300 as fkp
    return fkp


def _sub(cat, frac, seed):
    n = cat["x"].size
    idx = np.sort(mockgen.rng(seed, 40).choice(n, size=int(n * frac), replace=False))
    return {k: v[idx] for k, v in cat.items()}


@pytest.fixture(scope="module")
def requests():
    sv = mockgen.survey_small()
    gal, ran = mockgen.catalog(sv, 3)
    kf = 2 * math.pi / sv.L
    out = []
    for i, (N, assign, frac, B) in enumerate([(64, 2, 1.0, False), (60, 3, 0.7, False), (48, 2, 0.5, False),
                                              (64, 3, 0.9, True)]):
        s = mockgen.survey_small(N=N, assign=assign)
        geom = dict(s.geometry(), periodic=True)
        g, r = _sub(gal, frac, i), _sub(ran, frac, 10 + i)
        out.append(dict(geom=geom, pbins=(0.5 * kf, kf, 20), gal=g, ran=r, B=B))
    return out


def test_results_in_the_mix_equal_standalone(requests):
    fkp = _fkp()
    srv = fkp.Server(nslots=3)
    tickets = []
    for rq in requests:
        dg, dr = to_device(rq["gal"]), to_device(rq["ran"])
        if rq["B"]:
            t = srv.submit(rq["geom"], rq["pbins"], dg, dr, want=127, bshells=(3, 3, 3, 6),
                           contraction=fkp.FKP_CONTRACT_BF16X3)
        else:
            t = srv.submit(rq["geom"], rq["pbins"], dg, dr)
        tickets.append((t, rq, dg, dr))
    for t, rq, dg, dr in tickets:
        p, b, lat = srv.wait(t)
        assert lat > 0
        plan = fkp.Plan(rq["geom"], rq["pbins"], bshells=(3, 3, 3, 6) if rq["B"] else None,
                        want=127 if rq["B"] else 15)
        if rq["B"]:
            ps, bs = plan.bispectrum(dg, dr, contraction=fkp.FKP_CONTRACT_BF16X3)
            assert np.array_equal(b["NT"], bs["NT"])
            for k in ("B0", "B2", "B4", "N0", "N2", "N4"):
                assert np.array_equal(b[k], bs[k], equal_nan=True), k
        else:
            ps = plan.power(dg, dr)
        assert np.array_equal(p["nmodes"], ps["nmodes"])
        for k in ("P0", "P2", "P4", "P4b"):  # the same result in the mix as alone, bit for bit
            assert np.array_equal(p[k], ps[k], equal_nan=True), k
    st = srv.stats()
    assert st["completed"] == len(requests) and st["failed"] == 0
    assert st["peak_running"] >= 2  # requests overlapped on the device
    srv.close()


def test_admission_by_footprint_serialises(requests):
    fkp = _fkp()
    rq = requests[0]
    dg, dr = to_device(rq["gal"]), to_device(rq["ran"])
    probe = fkp.Server(nslots=1)
    probe.wait(probe.submit(rq["geom"], rq["pbins"], dg, dr))
    one = probe.stats()["peak_bytes"]
    probe.close()
    srv = fkp.Server(nslots=3, budget=int(one * 1.5))
    ts = [srv.submit(rq["geom"], rq["pbins"], dg, dr) for _ in range(4)]
    res = [srv.wait(t)[0] for t in ts]
    st = srv.stats()
    assert st["completed"] == 4 and st["peak_running"] == 1
    assert st["peak_bytes"] <= st["budget_bytes"]
    for r in res[1:]:
        assert np.array_equal(r["P0"], res[0]["P0"], equal_nan=True)
    srv.close()


def test_oversized_request_is_rejected(requests):
    fkp = _fkp()
    rq = requests[0]
    srv = fkp.Server(nslots=1, budget=1 << 20)
    with pytest.raises(fkp.FKPError) as e:
        srv.submit(rq["geom"], rq["pbins"], to_device(rq["gal"]), to_device(rq["ran"]))
    assert e.value.code == -3
    assert srv.stats()["rejected"] == 1
    srv.close()


def test_wait_timeout_and_failed_request(requests):
    fkp = _fkp()
    rq = requests[0]
    srv = fkp.Server(nslots=1)
    sv = mockgen.survey_boss(N=256, random_ratio=5.0, gen_grid=64)
    big_g, big_r = mockgen.catalog(sv, 0)
    t1 = srv.submit(sv.geometry(), (0.0, 0.005, 40), to_device(big_g), to_device(big_r))
    t2 = srv.submit(rq["geom"], rq["pbins"], to_device(rq["gal"]), to_device(rq["ran"]))
    with pytest.raises(fkp.FKPError) as e:
        srv.wait(t2, timeout_ms=0)
    assert e.value.code == -4
    srv.wait(t1)
    srv.wait(t2)
    bad = dict(rq["geom"], N=98)  # 98 = 2 * 7^2 has no radix plan: the worker's plan creation fails
    t3 = srv.submit(bad, rq["pbins"], to_device(rq["gal"]), to_device(rq["ran"]))
    with pytest.raises(fkp.FKPError) as e:
        srv.wait(t3)
    assert e.value.code == -1
    assert srv.stats()["failed"] == 1
    srv.close()
