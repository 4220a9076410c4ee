"""GPU parity of the power-spectrum path (C ABI) against the FP64 oracle."""
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


def _bins_small(L):
    kf = 2 * math.pi / L
    return (0.5 * kf, kf, 32)  # bins centred on integer multiples of k_f up to k_N


@pytest.fixture(scope="module")
def small_mock():
    sv = mockgen.survey_small()
    gal, ran = mockgen.catalog(sv, 0)
    return sv, gal, ran


def _oracle_power(gal, ran, geom, bins):
    return op.power(gal, ran, geom, bins)


def test_small_survey_matches_oracle(small_mock):
    """L=1000, 64^3, CIC, octant survey: P_0, P_2, P_4, P_4b, nmodes, k_eff,
    alpha, I_22, N_0, L^ab against the FP64 oracle."""
    fkp = _fkp()
    sv, gal, ran = small_mock
    geom = sv.geometry()
    bins = _bins_small(sv.L)
    ref = _oracle_power(gal, ran, geom, bins)
    plan = fkp.Plan(geom, bins)
    got = plan.power(to_device(gal), to_device(ran))
    assert np.array_equal(got["nmodes"], ref["nmodes"])
    err = p_errors(got, ref)
    assert max(err.values()) < P_TOL, err
    m = ref["nmodes"] > 0
    assert np.max(np.abs(got["k_eff"][m] / ref["k_eff"][m] - 1)) < 1e-6
    # the scalars are FP64 on the GPU (weights, products and sums)
    for k in ("alpha", "I22", "I33", "N0", "N0_fkp", "S3", "W_g", "W_r"):
        assert abs(got[k] / ref[k] - 1) < 1e-10, k
    assert np.max(np.abs(got["Lab"] - ref["Lab"])) < 1e-6
    assert abs(got["Lab"][:3].sum() - 1) < 1e-6


@pytest.mark.parametrize("N,assign", [(60, 3), (48, 2), (90, 3)])
def test_ragged_grids_match_oracle(small_mock, N, assign):
    """Non-power-of-two grids (radix 2, 3, 5 stages and ragged kx tiles),
    both assignment orders."""
    fkp = _fkp()
    sv0, gal, ran = small_mock
    sv = mockgen.survey_small(N=N, assign=assign)
    geom = dict(sv.geometry(), periodic=True)  # the octant reaches within 2 cells of the far faces
    kf = 2 * math.pi / sv.L
    bins = (0.0, 1.7 * kf, 14)
    ref = _oracle_power(gal, ran, geom, bins)
    got = fkp.Plan(geom, bins).power(to_device(gal), to_device(ran))
    assert np.array_equal(got["nmodes"], ref["nmodes"])
    err = p_errors(got, ref)
    assert max(err.values()) < P_TOL, err


def test_host_catalogs_equal_device_catalogs(small_mock):
    """The host-pointer path (copies inside the call) gives the same fixed-point
    grid, so the same P_l, bit for bit."""
    fkp = _fkp()
    sv, gal, ran = small_mock
    plan = fkp.Plan(sv.geometry(), _bins_small(sv.L))
    a = plan.power(gal, ran)
    b = plan.power(to_device(gal), to_device(ran))
    for k in ("P0", "P2", "P4", "P4b", "k_eff"):
        assert np.array_equal(a[k], b[k], equal_nan=True), k
    assert a["alpha"] == b["alpha"] and a["I22"] == b["I22"]


def test_repeat_runs_agree(small_mock):
    """Bit-reproducible P_l: repeated calls, plain launches after graph replay
    and a plan with other x- and y-pass launch shapes give identical bins
    (integer gridding and bin sums, fixed-order FP64 reductions)."""
    fkp = _fkp()
    sv, gal, ran = small_mock
    plan = fkp.Plan(sv.geometry(), _bins_small(sv.L))
    g, r = to_device(gal), to_device(ran)
    a = plan.power(g, r)
    b = plan.power(g, r)
    plan.set_graphs(False)
    c = plan.power(g, r)
    other = fkp.Plan(sv.geometry(), _bins_small(sv.L))
    other.set_schedule(8, 512, other.schedule()["z_threads"])  # another x/y launch shape, same z-pass shape
    d = other.power(g, r)
    for k in ("P0", "P2", "P4", "P4b", "k_eff"):
        for x in (b, c, d):
            assert np.array_equal(a[k], x[k], equal_nan=True), k


@pytest.mark.parametrize("N", [64, 60])
def test_every_pass_schedule_matches_oracle(small_mock, N):
    """The tuner picks among x-pass grid sizes and y/z-pass block shapes; every
    candidate gives P_l within the tolerance of the oracle (compile-time FFT at
    64, runtime FFT at 60), and the tuned choice is one of them."""
    fkp = _fkp()
    sv0, gal, ran = small_mock
    sv = mockgen.survey_small(N=N, assign=2)
    geom = dict(sv.geometry(), periodic=True)
    kf = 2 * math.pi / sv.L
    bins = (0.0, 1.7 * kf, 14)
    ref = _oracle_power(gal, ran, geom, bins)
    plan = fkp.Plan(geom, bins)
    sch = plan.schedule()
    assert sch["x_mult"] in (1, 2, 4, 8) and sch["y_threads"] in (256, 512) and sch["z_threads"] in (256, 512)
    assert all(t > 0 for t in sch["tuned_ms"])
    g, r = to_device(gal), to_device(ran)
    for xm, yt, zt in [(1, 256, 256), (8, 512, 512), (2, 256, 512), (4, 512, 256)]:
        plan.set_schedule(xm, yt, zt)
        got = plan.power(g, r)
        err = p_errors(got, ref)
        assert max(err.values()) < P_TOL, (xm, yt, zt, err)
    with pytest.raises(fkp.FKPError):
        plan.set_schedule(3, 256, 512)


@pytest.mark.parametrize("N", [128, 256])
def test_fused_last_stage_sizes_match_oracle(small_mock, N):
    """At these sizes the y-pass takes its last FFT stage's outputs from
    registers into the k_y sums: P_l within the tolerance of the oracle for
    each moment set (P_0 alone, P_0 and P_2, all multipoles: 1, 6 and 16
    fields, so 1, 3 and 9 k_z-power groups), both y-pass block shapes, and an
    interlaced PCS pair."""
    fkp = _fkp()
    sv0, gal, ran = small_mock
    sv = mockgen.survey_small(N=N, assign=3)
    geom = dict(sv.geometry())
    kf = 2 * math.pi / sv.L
    bins = (0.5 * kf, kf, 24)
    ref = _oracle_power(gal, ran, geom, bins)
    g, r = to_device(gal), to_device(ran)
    sets = [(fkp.FKP_P0, ("P0",)), (fkp.FKP_P0 | fkp.FKP_P2, ("P0", "P2")),
            (fkp.FKP_P0 | fkp.FKP_P2 | fkp.FKP_P4 | fkp.FKP_P4B, ("P0", "P2", "P4", "P4b"))]
    for want, keys in sets:
        plan = fkp.Plan(geom, bins, want=want)
        zt = plan.schedule()["z_threads"]
        for yt in (256, 512):
            plan.set_schedule(8, yt, zt)
            err = p_errors(plan.power(g, r), ref, keys)
            assert max(err.values()) < P_TOL, (want, yt, err)
    # the second grid of an interlaced pair enters the z-pass sums with its
    # half-cell phase
    geom_i = dict(geom, assign=4, interlace=True, periodic=True)
    ref_i = _oracle_power(gal, ran, geom_i, bins)
    err = p_errors(fkp.Plan(geom_i, bins).power(g, r), ref_i)
    assert max(err.values()) < P_TOL, err


def test_graph_replay_equals_plain_launches(small_mock):
    """The second call with the same device catalogs captures a CUDA graph and
    later calls replay it; another catalog runs plain launches and the graph
    still serves the first one.  Replayed results equal plain ones, bit for
    bit."""
    fkp = _fkp()
    sv, gal, ran = small_mock
    plan = fkp.Plan(sv.geometry(), _bins_small(sv.L))
    g, r = to_device(gal), to_device(ran)
    half = {k: v[: v.shape[0] // 2] for k, v in g.items()}
    flags, res = [], []
    for gg in (g, g, g, half, g):
        out = plan.power(gg, r)
        flags.append(out["graph"])
        res.append(out)
    assert flags == [0, 1, 1, 0, 1]
    assert all(out["timing_ms"][7] > 0 for out in res)
    plan.set_graphs(False)
    plain = plan.power(g, r)
    assert plain["graph"] == 0
    for out in (res[0], res[1], res[2], res[4]):
        for k in ("P0", "P2", "P4", "P4b"):
            assert np.array_equal(out[k], plain[k], equal_nan=True), k
    assert not np.allclose(res[3]["P0"], plain["P0"], equal_nan=True)


def test_periodic_kaiser_from_grid():
    """Plane-parallel field with |F_0|^2 = A(|n|)(1+f mu^2)^2 through
    fkp_power_from_grid against the oracle on the same float32 field."""
    fkp = _fkp()
    N, L, f = 64, 1000.0, 0.7

    def amp(nx, ny, nz):
        n2 = nx * nx + ny * ny + nz * nz
        mu2 = np.where(n2 > 0, nz * nz / np.where(n2 > 0, n2, 1), 0.0)
        return (1.0 + np.sqrt(n2)) ** -1.5 * (1 + f * mu2) ** 2 * 1e6

    field = mockgen.random_phase_field(N, amp, seed=5).astype(np.float32)
    geom = dict(N=N, L=L, assign=2, observer=None, los=(0, 0, 1), compensate=False, periodic=True)
    kf = 2 * math.pi / L
    bins = (0.5 * kf, kf, 31)
    ref = op.power_from_grid(field.astype(np.float64), geom, bins, I22=1.0, N0=0.0)
    got = fkp.Plan(geom, bins).power_from_grid(torch.from_numpy(field).cuda(), 1.0, 0.0)
    assert np.array_equal(got["nmodes"], ref["nmodes"])
    err = p_errors(got, ref)
    assert max(err.values()) < P_TOL, err


def test_radial_observer_inside_box_from_grid():
    """Observer inside the box (radial x^ varies over the grid) on a random
    smooth field: every multipole against the oracle."""
    fkp = _fkp()
    N, L = 48, 600.0
    field = mockgen.random_phase_field(N, lambda nx, ny, nz: 1.0 / (1.0 + nx * nx + ny * ny + nz * nz), seed=8)
    field = field.astype(np.float32)
    geom = dict(N=N, L=L, assign=3, origin=(0.0, 0.0, 0.0), observer=(210.0, -90.0, 333.0), compensate=True,
                periodic=True)
    kf = 2 * math.pi / L
    bins = (0.5 * kf, kf, 23)
    ref = op.power_from_grid(field.astype(np.float64), geom, bins, I22=2.0, N0=0.5)
    got = fkp.Plan(geom, bins).power_from_grid(torch.from_numpy(field).cuda(), 2.0, 0.5)
    err = p_errors(got, ref)
    assert max(err.values()) < P_TOL, err


def test_observer_on_a_grid_node_from_grid():
    """Observer exactly on a grid node (x^ = 0 there) with a spike of F at that
    node: the trace-reduced moment fields must still give every multipole of
    the 22-field oracle, in which the node contributes to F_0 only."""
    fkp = _fkp()
    N, L = 48, 600.0
    field = mockgen.random_phase_field(N, lambda nx, ny, nz: 1.0 / (1.0 + nx * nx + ny * ny + nz * nz), seed=9)
    field = field.astype(np.float32)
    field[12, 20, 24] += 40.0 * np.abs(field).max()  # node (x, y, z) = (24, 20, 12) = the observer
    geom = dict(N=N, L=L, assign=2, origin=(0.0, 0.0, 0.0), observer=(300.0, 250.0, 150.0), compensate=False,
                periodic=True)
    kf = 2 * math.pi / L
    bins = (0.5 * kf, kf, 23)
    ref = op.power_from_grid(field.astype(np.float64), geom, bins, I22=1.0, N0=0.0)
    got = fkp.Plan(geom, bins).power_from_grid(torch.from_numpy(field).cuda(), 1.0, 0.0)
    err = p_errors(got, ref)
    assert max(err.values()) < P_TOL, err


def test_object_near_box_face_is_rejected():
    fkp = _fkp()
    sv = mockgen.survey_small()
    gal = mockgen.uniform_points(100, 100.0, 500.0, seed=1)
    ran = mockgen.uniform_points(1000, 100.0, 500.0, seed=2)
    gal["x"][5] = sv.origin[0] + 0.5 * sv.L / sv.N  # inside the first cell
    plan = fkp.Plan(sv.geometry(), _bins_small(sv.L))
    with pytest.raises(fkp.FKPError) as e:
        plan.power(to_device(gal), to_device(ran))
    assert e.value.code == -2
    # the plan stays usable afterwards
    gal["x"][5] = 300.0
    plan.power(to_device(gal), to_device(ran))


def test_bad_plans_are_rejected():
    fkp = _fkp()
    with pytest.raises(fkp.FKPError):
        fkp.Plan(dict(L=100.0, N=98), (0.0, 0.1, 4))  # 98 = 2 * 7^2
    with pytest.raises(fkp.FKPError):
        fkp.Plan(dict(L=100.0, N=64, assign=5), (0.0, 0.1, 4))
    with pytest.raises(fkp.FKPError):
        fkp.Plan(dict(L=100.0, N=64), (0.0, -0.1, 4))


@pytest.mark.slow
def test_boss_512_full_size_matches_oracle():
    """The benchmark workload: L=3500, 512^3, TSC, 7e5 galaxies and 3.5e7
    randoms, 60 bins of 0.005 h/Mpc: every P_l bin against the FP64 oracle."""
    fkp = _fkp()
    sv = mockgen.survey_boss()
    gal, ran = mockgen.catalog(sv, 0)
    geom = sv.geometry()
    bins = (0.0, 0.005, 60)
    got = fkp.Plan(geom, bins).power(to_device(gal), to_device(ran))
    ref = op.power(gal, ran, geom, bins)
    assert np.array_equal(got["nmodes"], ref["nmodes"])
    err = p_errors(got, ref)
    assert max(err.values()) < P_TOL, err
    for k in ("alpha", "I22", "I33", "N0", "S3", "W_g", "W_r"):
        assert abs(got[k] / ref[k] - 1) < 1e-10, k


def test_bounded_wait_gives_up_and_the_context_stays_usable(small_mock):
    """The passes' bounded mbarrier wait, on a barrier that nothing arrives at
    (the library's diagnostic kernel), gives up after its poll limit and the
    call returns FKP_ETIMEOUT; the same context then still computes P_l."""
    fkp = _fkp()
    rc, msg = fkp.selftest_bounded_wait(0, 2000)
    assert rc == -4, msg
    assert "gave up" in msg
    sv, gal, ran = small_mock
    geom = sv.geometry()
    bins = _bins_small(sv.L)
    got = fkp.Plan(geom, bins).power(to_device(gal), to_device(ran))
    ref = _oracle_power(gal, ran, geom, bins)
    assert max(p_errors(got, ref).values()) < P_TOL


def test_cached_randoms_equal_the_full_path_and_the_oracle(small_mock):
    """One random catalog gridded once onto the plan without alpha (R = sum_r
    w W), then mocks that share it grid only their galaxies and form F = G -
    alpha R: the scalars equal those of passing the randoms (the same
    per-block FP64 partial sums), P_l agree with that path to 1e-6 of the
    monopole (each random term is rounded to the 2^-40 grid after the alpha
    product rather than before) and with the FP64 oracle to the P_l bar; the
    fused batch with rans=None likewise; an empty catalog drops the cache."""
    fkp = _fkp()
    sv, gal, ran = small_mock
    geom = sv.geometry()
    bins = _bins_small(sv.L)
    plan = fkp.Plan(geom, bins)
    dr = to_device(ran)
    plan.cache_randoms(dr)
    gals = [gal, mockgen.catalog(sv, 5, random_seed=0)[0]]
    for gg in gals:
        dg = to_device(gg)
        full = plan.power(dg, dr)
        cached = plan.power(dg, None)
        for k in ("alpha", "I22", "I33", "N0", "S3", "W_g", "W_r", "n_ran"):
            assert cached[k] == full[k], k
        assert np.array_equal(cached["Lab"], full["Lab"])
        assert np.array_equal(cached["nmodes"], full["nmodes"])
        assert max(p_errors(cached, full).values()) < 1e-6
        ref = _oracle_power(gg, ran, geom, bins)
        assert max(p_errors(cached, ref).values()) < P_TOL
    batch = plan.power_batch([to_device(gg) for gg in gals], None)
    for gg, b in zip(gals, batch):
        assert max(p_errors(b, plan.power(to_device(gg), None)).values()) < 1e-6
    plan.cache_randoms({k: v[:0] for k, v in dr.items()})
    with pytest.raises(fkp.FKPError) as e:
        plan.power(to_device(gal), None)
    assert e.value.code == -6


@pytest.mark.parametrize("assign,interlace", [(4, False), (4, True), (2, True), (3, True)],
                         ids=["pcs", "pcs_interlaced", "cic_interlaced", "tsc_interlaced"])
def test_pcs_and_interlaced_grids_match_oracle(small_mock, assign, interlace):
    """Fourth-order (PCS) assignment and interlaced pairs of grids (the
    paper's choice, Sec. III.A after eq. mapFFT), window-compensated: P_l of
    the small survey against the FP64 oracle, which averages the two grids'
    Legendre fields with the half-cell phase and compensates by sinc^p."""
    fkp = _fkp()
    sv0, gal, ran = small_mock
    geom = dict(sv0.geometry(), assign=assign, interlace=interlace, periodic=True)
    bins = _bins_small(sv0.L)
    ref = _oracle_power(gal, ran, geom, bins)
    plan = fkp.Plan(geom, bins)
    got = plan.power(to_device(gal), to_device(ran))
    assert np.array_equal(got["nmodes"], ref["nmodes"])
    err = p_errors(got, ref)
    assert max(err.values()) < P_TOL, err
    for k in ("alpha", "I22", "N0"):
        assert abs(got[k] / ref[k] - 1) < 1e-10, k
    if interlace:
        # the randoms cached on both grids of the pair
        plan.cache_randoms(to_device(ran))
        cached = plan.power(to_device(gal), None)
        assert max(p_errors(cached, got).values()) < 1e-6  # random terms rounded after, not before, alpha
        with pytest.raises(fkp.FKPError):
            plan.power_from_grid(torch.zeros((sv0.N,) * 3, device="cuda"))


def test_interlacing_removes_odd_aliases_of_a_poisson_sample():
    """What interlacing is for: the shot noise of an unclustered sample
    aliases into the high-k power of a single grid (the odd-order images of
    the window), and the interlaced pair cancels the odd images.  Uniform
    galaxies and randoms in a periodic box, CIC, compensated, so that
    <|F_0|^2> = N_0 at every k without aliasing: near the Nyquist frequency
    <|F_0|^2>/N_0 of the interlaced estimate is much closer to 1 than that of
    the single grid (both through the GPU path)."""
    fkp = _fkp()
    N, L = 64, 1000.0
    g = mockgen.rng(21, 0)

    def uniform(n):
        pts = {k: g.uniform(0, L, n).astype(np.float32) for k in ("x", "y", "z")}
        return dict(pts, w=np.ones(n, np.float32), nbar=np.full(n, 3e5 / L ** 3, np.float32))

    gal, ran = uniform(300000), uniform(1500000)
    kf = 2 * math.pi / L
    bins = (0.5 * kf, kf, 31)
    out = {}
    for il in (False, True):
        geom = dict(L=L, N=N, assign=2, origin=(0.0, 0.0, 0.0), observer=(-500.0, 300.0, 2000.0),
                    periodic=True, interlace=il)
        r = fkp.Plan(geom, bins).power(to_device(gal), to_device(ran))
        out[il] = r["mono_raw"] * r["I22"] / r["N0"]  # <|F_0|^2> / N_0: 1 for unaliased shot noise
    # bins |n| = 25..31: the compensated single grid's aliased shot noise sits
    # 8-31 % above N_0, the interlaced pair's 0.3-0.9 % (sums over images)
    hi = slice(24, 31)
    assert np.mean(np.abs(out[False][hi] - 1)) > 0.1
    assert np.mean(np.abs(out[True][hi] - 1)) < 0.3 * np.mean(np.abs(out[False][hi] - 1))


def test_split_multipoles_p6b_p8b_match_oracle(small_mock):
    """P_6b and P_8b by the line-of-sight split (Sec. II.B after eq. P4fast:
    the 22 fields of l <= 4 also give l = 6 and 8) against the FP64 oracle,
    graded like the other multipoles (by max(|P_ref|, raw monopole))."""
    fkp = _fkp()
    sv, gal, ran = small_mock
    geom = sv.geometry()
    bins = _bins_small(sv.L)
    want = fkp.FKP_P0 | fkp.FKP_P2 | fkp.FKP_P4 | fkp.FKP_P4B | fkp.FKP_P6B | fkp.FKP_P8B
    got = fkp.Plan(geom, bins, want=want).power(to_device(gal), to_device(ran))
    ref = _oracle_power(gal, ran, geom, bins)
    err = p_errors(got, ref, keys=("P0", "P2", "P4", "P4b", "P6b", "P8b"))
    assert max(err.values()) < P_TOL, err


@pytest.mark.parametrize("assign,want", [(3, "all"), (2, "p02")], ids=["tsc_all", "cic_p0_p2"])
def test_per_object_line_of_sight_matches_oracle(small_mock, assign, want):
    """FKP_XHAT_OBJECT: every moment field gridded with each object's own x^
    (eq. Qab read per object) against the oracle's per-object reading, and
    measurably apart from the node-x^ estimator (about 1e-3 of the monopole
    in P_2 on this survey, a hundred times the tolerance)."""
    fkp = _fkp()
    sv0, gal, ran = small_mock
    sv = mockgen.survey_small(N=64, assign=assign)
    geom = sv.geometry()
    bins = _bins_small(sv.L)
    keys = ("P0", "P2", "P4", "P4b") if want == "all" else ("P0", "P2")
    flags = (fkp.FKP_P0 | fkp.FKP_P2 | fkp.FKP_P4 | fkp.FKP_P4B) if want == "all" else (fkp.FKP_P0 | fkp.FKP_P2)
    ref = _oracle_power(gal, ran, dict(geom, xhat="object"), bins)
    g, r = to_device(gal), to_device(ran)
    plan = fkp.Plan(geom, bins, want=flags | fkp.FKP_XHAT_OBJECT)
    got = plan.power(g, r)
    assert np.array_equal(got["nmodes"], ref["nmodes"])
    err = p_errors(got, ref, keys)
    assert max(err.values()) < P_TOL, err
    node = fkp.Plan(geom, bins, want=flags).power(g, r)
    assert p_errors(node, ref, keys)["P2"] > 10 * P_TOL
    # F itself is the node plan's grid, bit for bit
    assert np.array_equal(plan.grid(g, r), fkp.Plan(geom, bins, want=flags).grid(g, r))


def test_per_object_plans_refuse_what_they_cannot_do(small_mock):
    fkp = _fkp()
    sv0, gal, ran = small_mock
    geom = sv0.geometry()
    bins = _bins_small(sv0.L)
    X = fkp.FKP_XHAT_OBJECT
    with pytest.raises(fkp.FKPError) as e:
        fkp.Plan(geom, bins, bshells=(3, 3, 3, 4), want=fkp.FKP_P0 | fkp.FKP_B0 | X)
    assert e.value.code == -1
    with pytest.raises(fkp.FKPError) as e:
        fkp.Plan(dict(geom, assign=4, interlace=True), bins, want=fkp.FKP_P0 | fkp.FKP_P2 | X)
    assert e.value.code == -1
    plan = fkp.Plan(geom, bins, want=fkp.FKP_P0 | fkp.FKP_P2 | fkp.FKP_P4 | X)
    for call in (lambda: plan.cache_randoms(to_device(ran)),
                 lambda: plan.power_batch([to_device(gal)], [to_device(ran)]),
                 lambda: plan.power_from_grid(torch.zeros((sv0.N,) * 3, device="cuda"))):
        with pytest.raises(fkp.FKPError) as e:
            call()
        assert e.value.code == -6
