"""Python binding of libfkp.so, the GB300 library for the FKP power-spectrum
and bispectrum multipole estimators of Scoccimarro (2015).

The binding only marshals arguments: every step of the estimator runs in the
library's CUDA kernels.  PyTorch tensors (or numpy arrays for host catalogs)
are passed by pointer.  If the compiled library is missing the import of
this package still succeeds, but every call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libfkp.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "fkp.h")

FKP_P0, FKP_P2, FKP_P4, FKP_P4B = 1, 2, 4, 8
FKP_B0, FKP_B2, FKP_B4 = 16, 32, 64
FKP_P6B, FKP_P8B, FKP_B4B = 128, 256, 512
FKP_XHAT_OBJECT = 1024  # modifier: moments with each object's own line of sight
FKP_CONTRACT_FP32, FKP_CONTRACT_BF16X3, FKP_CONTRACT_BF16X6 = 0, 1, 2
ERRORS = {-1: "FKP_EINVAL", -2: "FKP_EGEOM", -3: "FKP_ENOMEM", -4: "FKP_ETIMEOUT", -5: "FKP_ECUDA",
          -6: "FKP_ESTATE"}
EXPORTS = ["fkp_context_create", "fkp_context_destroy", "fkp_plan_create", "fkp_plan_destroy", "fkp_plan_sizes",
           "fkp_power", "fkp_power_from_grid", "fkp_bispectrum", "fkp_last_error", "fkp_version",
           "fkp_power_from_grid_noalloc", "fkp_server_create", "fkp_server_submit", "fkp_server_poll",
           "fkp_server_wait", "fkp_server_stats", "fkp_server_destroy", "fkp_check_tables",
           "fkp_plan_set_graphs", "fkp_plan_schedule", "fkp_plan_set_schedule", "fkp_power_batch",
           "fkp_selftest_bounded_wait", "fkp_plan_cache_randoms", "fkp_grid"]


class FKPError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Catalog(C.Structure):
    _fields_ = [("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p), ("w", C.c_void_p), ("nbar", C.c_void_p),
                ("n", C.c_int64), ("on_device", C.c_int)]


class Geometry(C.Structure):
    _fields_ = [("L", C.c_double), ("origin", C.c_double * 3), ("observer", C.c_double * 3),
                ("observer_at_infinity", C.c_int), ("los", C.c_double * 3), ("N", C.c_int), ("assign", C.c_int),
                ("compensate", C.c_int), ("periodic", C.c_int), ("P_fkp", C.c_double), ("alpha_mode", C.c_int),
                ("interlace", C.c_int)]


class PBins(C.Structure):
    _fields_ = [("kmin", C.c_double), ("dk", C.c_double), ("nbins", C.c_int)]


class BShells(C.Structure):
    _fields_ = [("first", C.c_int), ("step", C.c_int), ("width", C.c_int), ("nshells", C.c_int)]


_DP = C.POINTER(C.c_double)


class PowerOut(C.Structure):
    _fields_ = [("k_eff", _DP), ("P0", _DP), ("P2", _DP), ("P4", _DP), ("P4b", _DP), ("mono_raw", _DP),
                ("nmodes", C.POINTER(C.c_int64)), ("alpha", C.c_double), ("I22", C.c_double), ("I33", C.c_double),
                ("N0", C.c_double), ("N0_fkp", C.c_double), ("S3", C.c_double), ("W_g", C.c_double),
                ("W_r", C.c_double), ("Lab", C.c_double * 6), ("n_gal", C.c_int64), ("n_ran", C.c_int64),
                ("timing_ms", C.c_float * 8), ("graph", C.c_int), ("P6b", _DP), ("P8b", _DP)]


class BispOut(C.Structure):
    _fields_ = [("tri", C.POINTER(C.c_int16)), ("NT", C.POINTER(C.c_int64)), ("centre_closed", C.POINTER(C.c_uint8)),
                ("B0", _DP), ("B2", _DP), ("B4", _DP), ("N0", _DP), ("N2", _DP), ("N4", _DP),
                ("T0", _DP), ("T2", _DP), ("T4", _DP), ("I33", C.c_double), ("S3", C.c_double),
                ("B4b", _DP), ("T22", _DP)]


class Request(C.Structure):
    _fields_ = [("geom", Geometry), ("pbins", PBins), ("bshells", BShells), ("want", C.c_uint32),
                ("contraction", C.c_int), ("gal", Catalog), ("ran", Catalog), ("pout", C.POINTER(PowerOut)),
                ("bout", C.POINTER(BispOut))]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64), ("rejected", C.c_int64),
                ("queued", C.c_int64), ("running", C.c_int), ("peak_running", C.c_int),
                ("bytes_in_use", C.c_size_t), ("peak_bytes", C.c_size_t), ("budget_bytes", C.c_size_t)]


_lib = None


def lib():
    """The loaded library; raises when it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'` (no CPU fallback exists)")
        L = C.CDLL(LIB_PATH)
        vp = C.c_void_p
        L.fkp_context_create.argtypes = [C.c_int, C.c_size_t, C.POINTER(vp)]
        L.fkp_context_destroy.argtypes = [vp]
        L.fkp_context_destroy.restype = None
        L.fkp_plan_create.argtypes = [vp, C.POINTER(Geometry), C.POINTER(PBins), C.POINTER(BShells), C.c_uint32,
                                      C.POINTER(vp)]
        L.fkp_plan_destroy.argtypes = [vp]
        L.fkp_plan_destroy.restype = None
        L.fkp_plan_sizes.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_size_t)]
        L.fkp_power.argtypes = [vp, C.POINTER(Catalog), C.POINTER(Catalog), vp, C.POINTER(PowerOut)]
        L.fkp_power_from_grid.argtypes = [vp, vp, C.c_double, C.c_double, vp, C.POINTER(PowerOut)]
        L.fkp_power_batch.argtypes = [vp, C.c_int, C.POINTER(Catalog), C.POINTER(Catalog), vp, C.POINTER(PowerOut)]
        L.fkp_bispectrum.argtypes = [vp, C.POINTER(Catalog), C.POINTER(Catalog), C.c_int, vp, C.POINTER(PowerOut),
                                     C.POINTER(BispOut)]
        L.fkp_power_from_grid_noalloc.argtypes = [C.POINTER(Geometry), C.POINTER(PBins), vp, C.c_double,
                                                  C.c_double, vp, C.POINTER(PowerOut)]
        L.fkp_server_create.argtypes = [C.c_int, C.c_int, C.c_size_t, C.POINTER(vp)]
        L.fkp_server_submit.argtypes = [vp, C.POINTER(Request), C.POINTER(C.c_uint64)]
        L.fkp_server_poll.argtypes = [vp, C.c_uint64, C.POINTER(C.c_int)]
        L.fkp_server_wait.argtypes = [vp, C.c_uint64, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double)]
        L.fkp_server_stats.argtypes = [vp, C.POINTER(ServerStats)]
        L.fkp_server_destroy.argtypes = [vp]
        L.fkp_server_destroy.restype = None
        L.fkp_last_error.restype = C.c_char_p
        L.fkp_check_tables.argtypes = []
        L.fkp_plan_set_graphs.argtypes = [vp, C.c_int]
        L.fkp_plan_schedule.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                        C.POINTER(C.c_float)]
        L.fkp_plan_set_schedule.argtypes = [vp, C.c_int, C.c_int, C.c_int]
        L.fkp_version.restype = C.c_char_p
        L.fkp_selftest_bounded_wait.argtypes = [C.c_int, C.c_uint]
        L.fkp_plan_cache_randoms.argtypes = [vp, C.POINTER(Catalog), vp]
        L.fkp_grid.argtypes = [vp, C.POINTER(Catalog), C.POINTER(Catalog), C.c_int, vp, vp, vp]
        _lib = L
    return _lib


def _check(rc):
    if rc != 0:
        raise FKPError(rc, lib().fkp_last_error().decode())


_contexts = {}


def context(device=0, budget=0):
    key = (device, budget)
    if key not in _contexts:
        h = C.c_void_p()
        _check(lib().fkp_context_create(device, budget, C.byref(h)))
        _contexts[key] = h
    return _contexts[key]


def _ptr(a):
    if a is None:
        return None, 0
    if hasattr(a, "data_ptr"):  # torch tensor
        if a.dtype.__repr__() != "torch.float32" or not a.is_contiguous():
            raise TypeError("catalog tensors must be contiguous float32")
        return a.data_ptr(), 1 if a.is_cuda else 0
    arr = np.ascontiguousarray(a, dtype=np.float32)
    return arr.ctypes.data, 0


def check_field(F, N, device):
    """Raises, before any launch, unless F is what the C calls read: a
    contiguous float32 CUDA tensor of N^3 values on `device` (the plan's, or
    the current device for the entry point without a plan).  A wrong dtype
    or size would make the x-pass read past the end of the buffer."""
    if not (hasattr(F, "is_cuda") and F.is_cuda and F.is_contiguous()):
        raise TypeError("F must be a contiguous CUDA float32 tensor")
    import torch
    if F.dtype != torch.float32:
        raise TypeError(f"F must be float32, not {F.dtype}")
    if F.numel() != int(N) ** 3:
        raise ValueError(f"F holds {F.numel()} values; the grid needs N^3 = {int(N) ** 3}")
    if F.device.index != device:
        raise ValueError(f"F is on cuda:{F.device.index}, the call runs on cuda:{device}")


def make_catalog(cat, device=None):
    """Catalog struct from a dict with x, y, z, nbar and optional w (torch
    tensors on one device, or host arrays).  Returns (struct, keepalive).
    With `device` set, device tensors must be on that CUDA device."""
    keep = []
    ptrs = {}
    dev = None
    n = None
    for k in ("x", "y", "z", "w", "nbar"):
        a = cat.get(k)
        if a is None:
            ptrs[k] = None
            continue
        if not hasattr(a, "data_ptr"):
            a = np.ascontiguousarray(a, dtype=np.float32)
        keep.append(a)
        if device is not None and getattr(a, "is_cuda", False) and a.device.index != device:
            raise ValueError(f"catalog tensor on cuda:{a.device.index}, the plan runs on cuda:{device}")
        p, d = _ptr(a)
        ptrs[k] = p
        dev = d if dev is None else dev
        if d != dev:
            raise ValueError("catalog arrays must all be on the device or all on the host")
        m = a.shape[0]
        n = m if n is None else n
        if m != n:
            raise ValueError("catalog arrays differ in length")
    c = Catalog(ptrs["x"], ptrs["y"], ptrs["z"], ptrs["w"], ptrs["nbar"], n or 0, dev or 0)
    return c, keep


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    return getattr(stream, "cuda_stream", stream)


def geometry(g):
    """Geometry struct from a dict (keys of mockgen.Survey.geometry() plus
    optional observer=None/los, compensate, periodic, alpha_mode, interlace)."""
    obs = g.get("observer", (0.0, 0.0, 0.0))
    inf = obs is None
    return Geometry(float(g["L"]), (C.c_double * 3)(*g.get("origin", (0.0, 0.0, 0.0))),
                    (C.c_double * 3)(*((0.0, 0.0, 0.0) if inf else obs)), 1 if inf else 0,
                    (C.c_double * 3)(*g.get("los", (0.0, 0.0, 1.0))), int(g["N"]), int(g.get("assign", 2)),
                    1 if g.get("compensate", True) else 0, 1 if g.get("periodic", False) else 0,
                    float(g.get("P_fkp", 1e4)), int(g.get("alpha_mode", 0)), 1 if g.get("interlace", False) else 0)


class Plan:
    """One geometry, binning and set of outputs; owns the device workspace."""

    def __init__(self, geom, pbins, bshells=None, want=FKP_P0 | FKP_P2 | FKP_P4 | FKP_P4B, device=0, budget=0):
        self.geom = dict(geom)
        self.want = want
        self.device = int(device)
        self._g = geometry(geom)
        self._pb = PBins(float(pbins[0]), float(pbins[1]), int(pbins[2]))
        self._bs = BShells(*[int(v) for v in bshells]) if bshells is not None else None
        self._h = C.c_void_p()
        _check(lib().fkp_plan_create(context(device, budget), C.byref(self._g), C.byref(self._pb),
                                     C.byref(self._bs) if self._bs is not None else None, want, C.byref(self._h)))
        nb, nt, ws = C.c_int(), C.c_int(), C.c_size_t()
        _check(lib().fkp_plan_sizes(self._h, C.byref(nb), C.byref(nt), C.byref(ws)))
        self.nbins, self.ntri, self.workspace_bytes = nb.value, nt.value, ws.value

    def close(self):
        if self._h:
            lib().fkp_plan_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _pout(self):
        nb = self.nbins
        arr = {k: np.full(nb, np.nan) for k in ("k_eff", "P0", "P2", "P4", "P4b", "mono_raw", "P6b", "P8b")}
        arr["nmodes"] = np.zeros(nb, dtype=np.int64)
        o = PowerOut()
        for k in ("k_eff", "P0", "P2", "P4", "P4b", "mono_raw", "P6b", "P8b"):
            setattr(o, k, arr[k].ctypes.data_as(_DP))
        o.nmodes = arr["nmodes"].ctypes.data_as(C.POINTER(C.c_int64))
        return o, arr

    @staticmethod
    def _scalars(o, arr):
        for k in ("alpha", "I22", "I33", "N0", "N0_fkp", "S3", "W_g", "W_r", "n_gal", "n_ran"):
            arr[k] = getattr(o, k)
        arr["Lab"] = np.array(list(o.Lab))
        arr["timing_ms"] = np.array(list(o.timing_ms))
        arr["graph"] = int(o.graph)
        return arr

    def schedule(self):
        """The FFT passes' launch schedule (tuned when the plan was made)."""
        xm, yt, zt = C.c_int(), C.c_int(), C.c_int()
        ms = (C.c_float * 3)()
        _check(lib().fkp_plan_schedule(self._h, C.byref(xm), C.byref(yt), C.byref(zt), ms))
        return {"x_mult": xm.value, "y_threads": yt.value, "z_threads": zt.value, "tuned_ms": list(ms)}

    def set_schedule(self, x_mult, y_threads, z_threads):
        """Overrides the tuned schedule for this plan."""
        _check(lib().fkp_plan_set_schedule(self._h, int(x_mult), int(y_threads), int(z_threads)))

    def set_graphs(self, enable):
        """CUDA-graph replay of the device-catalog power path (default on)."""
        _check(lib().fkp_plan_set_graphs(self._h, 1 if enable else 0))

    def cache_randoms(self, ran, stream=None):
        """Grids a random catalog once onto the plan (without alpha) for later
        calls with ran=None; an empty catalog drops the cache."""
        cr, k2 = make_catalog(ran, self.device)
        _check(lib().fkp_plan_cache_randoms(self._h, C.byref(cr), _stream_handle(stream)))

    def power(self, gal, ran, stream=None):
        """P_0, P_2, P_4, P_4b and the scalars for one survey (ran=None: the
        plan's cached random catalog)."""
        cg, k1 = make_catalog(gal, self.device)
        cr, k2 = make_catalog(ran, self.device) if ran is not None else (None, None)
        o, arr = self._pout()
        _check(lib().fkp_power(self._h, C.byref(cg), C.byref(cr) if cr is not None else None,
                               _stream_handle(stream), C.byref(o)))
        return self._scalars(o, arr)

    def grid(self, gal, ran, which=0, with_w=False, stream=None):
        """The gridded fields F (and F^w with with_w) of one survey as int64
        numpy arrays [z][y][x] in units of 2^-40 (ran=None: the plan's cached
        random catalog; which=1: an interlaced plan's second grid)."""
        N = self.geom["N"]
        cg, k1 = make_catalog(gal, self.device)
        cr, k2 = make_catalog(ran, self.device) if ran is not None else (None, None)
        F = np.empty((N, N, N), dtype=np.int64)
        Fw = np.empty((N, N, N), dtype=np.int64) if with_w else None
        _check(lib().fkp_grid(self._h, C.byref(cg), C.byref(cr) if cr is not None else None, int(which),
                              F.ctypes.data, Fw.ctypes.data if Fw is not None else None, _stream_handle(stream)))
        return (F, Fw) if with_w else F

    def power_batch(self, gals, rans, stream=None):
        """P_0, P_2, P_4, P_4b and the scalars of several mocks on this plan's
        grid: each mock gridded on its own, then one launch per FFT pass for
        all of them.  Returns one result dict per mock."""
        if not gals or (rans is not None and len(gals) != len(rans)):
            raise ValueError("need equal, non-zero numbers of galaxy and random catalogs (rans=None: the cache)")
        n = len(gals)
        cg, cr, keep = (Catalog * n)(), (Catalog * n)(), []
        for k in range(n):
            cg[k], k1 = make_catalog(gals[k], self.device)
            keep.append(k1)
            if rans is not None:
                cr[k], k2 = make_catalog(rans[k], self.device)
                keep.append(k2)
        outs = (PowerOut * n)()
        arrs = []
        for k in range(n):
            o, arr = self._pout()
            outs[k] = o
            arrs.append(arr)
        _check(lib().fkp_power_batch(self._h, n, cg, cr if rans is not None else None, _stream_handle(stream),
                                     outs))
        return [self._scalars(outs[k], arrs[k]) for k in range(n)]

    def power_from_grid(self, F, I22=1.0, N0=0.0, stream=None):
        """The estimator on a given device field F (torch float32 CUDA tensor
        [N][N][N], layout [z][y][x])."""
        check_field(F, self.geom["N"], self.device)
        o, arr = self._pout()
        _check(lib().fkp_power_from_grid(self._h, F.data_ptr(), float(I22), float(N0), _stream_handle(stream),
                                         C.byref(o)))
        return self._scalars(o, arr)

    def bispectrum(self, gal, ran, contraction=FKP_CONTRACT_FP32, stream=None):
        """P_l and B_l (closed triangles a >= b >= c with N_T > 0)."""
        cg, k1 = make_catalog(gal, self.device)
        cr, k2 = make_catalog(ran, self.device) if ran is not None else (None, None)
        o, parr = self._pout()
        nt = self.ntri
        b = {"tri": np.zeros((nt, 3), dtype=np.int16), "NT": np.zeros(nt, dtype=np.int64),
             "centre_closed": np.zeros(nt, dtype=np.uint8)}
        for k in ("B0", "B2", "B4", "N0", "N2", "N4", "T0", "T2", "T4", "B4b", "T22"):
            b[k] = np.full(nt, np.nan)
        bo = BispOut()
        bo.tri = b["tri"].ctypes.data_as(C.POINTER(C.c_int16))
        bo.NT = b["NT"].ctypes.data_as(C.POINTER(C.c_int64))
        bo.centre_closed = b["centre_closed"].ctypes.data_as(C.POINTER(C.c_uint8))
        for k in ("B0", "B2", "B4", "N0", "N2", "N4", "T0", "T2", "T4", "B4b", "T22"):
            setattr(bo, k, b[k].ctypes.data_as(_DP))
        _check(lib().fkp_bispectrum(self._h, C.byref(cg), C.byref(cr) if cr is not None else None,
                                    int(contraction), _stream_handle(stream), C.byref(o), C.byref(bo)))
        b["I33"], b["S3"] = bo.I33, bo.S3
        return self._scalars(o, parr), b


def power_from_grid_noalloc(geom, pbins, F, I22=1.0, N0=0.0, stream=None):
    """The estimator on a device field F for small grids (even N <= 64,
    nbins <= 64) through the entry point that allocates no device memory
    (its buffers live in a static device array shared by all calls on a
    device; calls must not overlap on the GPU)."""
    import torch
    check_field(F, int(geom["N"]), torch.cuda.current_device())
    g = geometry(geom)
    pb = PBins(float(pbins[0]), float(pbins[1]), int(pbins[2]))
    nb = pb.nbins
    arr = {k: np.full(nb, np.nan) for k in ("k_eff", "P0", "P2", "P4", "P4b", "mono_raw", "P6b", "P8b")}
    arr["nmodes"] = np.zeros(nb, dtype=np.int64)
    o = PowerOut()
    for k in ("k_eff", "P0", "P2", "P4", "P4b", "mono_raw", "P6b", "P8b"):
        setattr(o, k, arr[k].ctypes.data_as(_DP))
    o.nmodes = arr["nmodes"].ctypes.data_as(C.POINTER(C.c_int64))
    _check(lib().fkp_power_from_grid_noalloc(C.byref(g), C.byref(pb), F.data_ptr(), float(I22), float(N0),
                                             _stream_handle(stream), C.byref(o)))
    return Plan._scalars(o, arr)


def _bout(nt):
    b = {"tri": np.zeros((nt, 3), dtype=np.int16), "NT": np.zeros(nt, dtype=np.int64),
         "centre_closed": np.zeros(nt, dtype=np.uint8)}
    for k in ("B0", "B2", "B4", "N0", "N2", "N4", "T0", "T2", "T4", "B4b", "T22"):
        b[k] = np.full(nt, np.nan)
    bo = BispOut()
    bo.tri = b["tri"].ctypes.data_as(C.POINTER(C.c_int16))
    bo.NT = b["NT"].ctypes.data_as(C.POINTER(C.c_int64))
    bo.centre_closed = b["centre_closed"].ctypes.data_as(C.POINTER(C.c_uint8))
    for k in ("B0", "B2", "B4", "N0", "N2", "N4", "T0", "T2", "T4", "B4b", "T22"):
        setattr(bo, k, b[k].ctypes.data_as(_DP))
    return bo, b


def max_triangles(bshells):
    """Upper bound on the triangle count of a shell set (all a >= b >= c)."""
    S = int(bshells[3])
    return S * (S + 1) * (S + 2) // 6


class Server:
    """Continuous-batching server: requests (catalogs + geometry + outputs)
    are admitted by device footprint and run concurrently on `nslots`
    streams.  The catalogs passed to submit() are kept referenced until
    their ticket is waited for."""

    def __init__(self, nslots=3, budget=0, device=0):
        self._h = C.c_void_p()
        _check(lib().fkp_server_create(device, nslots, budget, C.byref(self._h)))
        self._live = {}

    def submit(self, geom, pbins, gal, ran, want=FKP_P0 | FKP_P2 | FKP_P4 | FKP_P4B, bshells=None,
               contraction=FKP_CONTRACT_BF16X3):
        cg, k1 = make_catalog(gal)
        cr, k2 = make_catalog(ran)
        pb = PBins(float(pbins[0]), float(pbins[1]), int(pbins[2]))
        bs = BShells(*[int(v) for v in bshells]) if bshells is not None else BShells(1, 1, 1, 1)
        tmp = Plan.__new__(Plan)
        tmp.nbins = pb.nbins
        o, parr = tmp._pout()
        bo, barr = (None, None)
        if bshells is not None:
            bo, barr = _bout(max_triangles(bshells))
        req = Request(geometry(geom), pb, bs, int(want), int(contraction), cg, cr, C.pointer(o),
                      C.pointer(bo) if bo is not None else None)
        t = C.c_uint64()
        _check(lib().fkp_server_submit(self._h, C.byref(req), C.byref(t)))
        self._live[t.value] = (req, o, parr, bo, barr, k1, k2, gal, ran)
        return t.value

    def poll(self, ticket):
        d = C.c_int()
        _check(lib().fkp_server_poll(self._h, ticket, C.byref(d)))
        return bool(d.value)

    def wait(self, ticket, timeout_ms=-1):
        """(power dict, bispectrum dict or None, latency in ms); raises the
        request's own error if it failed."""
        st, lat = C.c_int(), C.c_double()
        _check(lib().fkp_server_wait(self._h, ticket, int(timeout_ms), C.byref(st), C.byref(lat)))
        req, o, parr, bo, barr, *_ = self._live.pop(ticket)
        _check(st.value)
        p = Plan._scalars(o, parr)
        if barr is not None:
            n = int(np.count_nonzero(barr["NT"]))
            barr = {k: (v[:n] if hasattr(v, "shape") and v.shape[:1] == (len(barr["NT"]),) else v)
                    for k, v in barr.items()}
            barr["I33"], barr["S3"] = bo.I33, bo.S3
        return p, barr, lat.value

    def stats(self):
        s = ServerStats()
        _check(lib().fkp_server_stats(self._h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in ServerStats._fields_}

    def close(self):
        if self._h:
            lib().fkp_server_destroy(self._h)
            self._h = C.c_void_p()
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def selftest_bounded_wait(device=0, polls=1000):
    """Return code of the library's bounded-wait diagnostic (FKP_ETIMEOUT,
    -4, is the expected outcome) and its message."""
    rc = lib().fkp_selftest_bounded_wait(int(device), int(polls))
    return rc, lib().fkp_last_error().decode()


def check_tables():
    """Host-only check of the moment-field / k_z-group tables (no GPU)."""
    _check(lib().fkp_check_tables())


def version():
    return lib().fkp_version().decode()
