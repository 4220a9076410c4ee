"""The entry point that allocates no device memory (for callers that may not
call cudaMalloc once running: processes that reserve all device memory for
their own pool, loops that forbid allocation after start-up, plugin hosts
without an allocator) gives the same multipoles as the plan-based
fkp_power_from_grid, on two calls in a row.  Collected last on purpose."""
import math

import numpy as np
import pytest

import mockgen
from tests.helpers import P_TOL, p_errors

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _field(N, seed):
    return mockgen.random_phase_field(
        N, lambda nx, ny, nz: 1.0 / (1.0 + nx * nx + ny * ny + nz * nz) ** 0.75, seed=seed).astype(np.float32)


def test_no_alloc_entry_point_matches_plan_path_twice():
    import paper_1506_02729_gb300 as fkp
    N, L = 64, 800.0
    geom = dict(N=N, L=L, assign=3, origin=(0.0, 0.0, 0.0), observer=(300.0, -120.0, 410.0), compensate=True,
                periodic=True)
    kf = 2 * math.pi / L
    bins = (0.5 * kf, kf, 31)
    for seed in (11, 12):
        F = torch.from_numpy(_field(N, seed)).cuda()
        ref = fkp.Plan(geom, bins).power_from_grid(F, 2.0, 0.25)
        got = fkp.power_from_grid_noalloc(geom, bins, F, 2.0, 0.25)
        assert np.array_equal(got["nmodes"], ref["nmodes"])
        err = p_errors(got, ref)
        assert max(err.values()) < P_TOL, err


def test_no_alloc_entry_point_rejects_large_grids():
    import paper_1506_02729_gb300 as fkp
    F = torch.zeros((96, 96, 96), dtype=torch.float32, device="cuda")
    with pytest.raises(fkp.FKPError) as e:
        fkp.power_from_grid_noalloc(dict(N=96, L=100.0), (0.0, 0.1, 8), F)
    assert e.value.code == -1 and "N <= 64" in str(e.value)
