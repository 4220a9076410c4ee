"""The entry point that allocates no device memory (for callers that may not
call cudaMalloc once running: processes that reserve all device memory for
their own pool, loops that forbid allocation after start-up, plugin hosts
without an allocator) gives the same multipoles as the plan-based
fkp_power_from_grid and as the FP64 oracle, on two calls in a row, for the
compiled 64^3 passes and for the runtime-sized ones (60^3: radix 5 and 3,
48^3: radix 3) that run on buffers strided for 64^3 inside the static array;
and after a warm-up call its calls leave the device's free memory and the
allocator untouched.  Collected last on purpose."""
import math

import numpy as np
import pytest

import mockgen
from oracle import power as op
from tests.helpers import P_TOL, p_errors

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _field(N, seed):
    return mockgen.random_phase_field(
        N, lambda nx, ny, nz: 1.0 / (1.0 + nx * nx + ny * ny + nz * nz) ** 0.75, seed=seed).astype(np.float32)


@pytest.mark.parametrize("N", [64, 60, 48])
def test_no_alloc_entry_point_matches_plan_path_and_oracle_twice(N):
    import paper_1506_02729_gb300 as fkp
    L = 800.0
    geom = dict(N=N, L=L, assign=3, origin=(0.0, 0.0, 0.0), observer=(300.0, -120.0, 410.0), compensate=True,
                periodic=True)
    kf = 2 * math.pi / L
    bins = (0.5 * kf, kf, N // 2 - 1)
    for seed in (11, 12):
        f = _field(N, seed)
        F = torch.from_numpy(f).cuda()
        ref = fkp.Plan(geom, bins).power_from_grid(F, 2.0, 0.25)
        got = fkp.power_from_grid_noalloc(geom, bins, F, 2.0, 0.25)
        assert np.array_equal(got["nmodes"], ref["nmodes"])
        err = p_errors(got, ref)
        assert max(err.values()) < P_TOL, err
        orc = op.power_from_grid(f.astype(np.float64), geom, bins, 2.0, 0.25)
        assert np.array_equal(got["nmodes"], orc["nmodes"])
        err = p_errors(got, orc)
        assert max(err.values()) < P_TOL, err


def test_no_alloc_calls_leave_device_memory_untouched():
    import paper_1506_02729_gb300 as fkp
    N, L = 64, 800.0
    geom = dict(N=N, L=L, assign=2, origin=(0.0, 0.0, 0.0), observer=(-50.0, 20.0, 900.0), periodic=True)
    kf = 2 * math.pi / L
    bins = (0.5 * kf, kf, 20)
    F = torch.from_numpy(_field(N, 13)).cuda()
    first = fkp.power_from_grid_noalloc(geom, bins, F)  # maps the library's module and array
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    stats0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    res = [fkp.power_from_grid_noalloc(geom, bins, F) for _ in range(2)]
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == stats0
    for r in res:
        assert np.array_equal(r["nmodes"], first["nmodes"])
        assert np.array_equal(r["P0"], first["P0"], equal_nan=True)


def test_no_alloc_entry_point_rejects_large_grids():
    import paper_1506_02729_gb300 as fkp
    F = torch.zeros((96, 96, 96), dtype=torch.float32, device="cuda")
    with pytest.raises(fkp.FKPError) as e:
        fkp.power_from_grid_noalloc(dict(N=96, L=100.0), (0.0, 0.1, 8), F)
    assert e.value.code == -1 and "N <= 64" in str(e.value)
